"""The C-ABI library builds, loads and exports every entry point that
include/alens.h declares.  No GPU needed: no compute call is made."""
import re
import subprocess
from pathlib import Path

import pytest

import paper_2109_08206_gb300 as A

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def libpath():
    return A.build()


def test_header_declares_the_four_step_calls():
    names = A.exported_symbols()
    for n in ("aLENS_build_neighbors", "aLENS_assemble_constraints", "aLENS_solve_lcp", "aLENS_step"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", str(libpath)], capture_output=True, text=True,
                         check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = [n for n in A.exported_symbols() if n not in exported]
    assert not missing, missing
    # and nothing else of ours leaks out
    ours = {n for n in exported if n.startswith("aLENS_")}
    assert ours == set(A.exported_symbols())


def test_library_loads_and_binds(libpath):
    L = A.lib()
    for n in A.exported_symbols():
        assert hasattr(L, n)
    assert L.aLENS_status_string(0).decode() == "ok"
    assert "timed out" in L.aLENS_status_string(4).decode()


def test_ctypes_structs_match_header():
    import ctypes as C
    text = (ROOT / "include" / "alens.h").read_text()
    # field order of aLENS_params and aLENS_info as declared
    def fields(struct):
        body = re.search(r"typedef struct \{([^}]*)\}\s*" + struct + ";", text).group(1)
        return re.findall(r"\b(?:double|int32_t|int64_t|float)\s+(\w+)", body)
    assert [f for f, _ in A.Params._fields_] == fields("aLENS_params")
    assert [f for f, _ in A.Info._fields_] == fields("aLENS_info")
    assert C.sizeof(A.Params) == 9 * 8 + 2 * 4


def test_product_path_does_not_touch_the_oracle():
    # the package and the CUDA sources never import, include or name the oracle
    for p in list((ROOT / "paper_2109_08206_gb300").rglob("*.py")) + \
            list((ROOT / "paper_2109_08206_gb300" / "csrc").glob("*")) + [ROOT / "include" / "alens.h"]:
        t = p.read_text()
        assert "import oracle" not in t and "from oracle" not in t and "alens_oracle" not in t, p


def test_batch_tables_are_laid_out_like_the_header():
    """BatchSpec (host-side marshalling of aLENS_step_batch's tables): one
    aLENS_system per system, scalar boxes widened to three edges, rod
    offsets as int64; a rod_offset of the wrong length is refused before
    any call."""
    systems = [((10.0, 11.0, 12.0), 3.0), (20.0, 4.5)]
    spec = A.BatchSpec(systems, [0, 5, 9])
    assert spec.n_systems == 2
    assert list(spec.tab[0].box) == [10.0, 11.0, 12.0] and spec.tab[0].length == 3.0
    assert list(spec.tab[1].box) == [20.0, 20.0, 20.0] and spec.tab[1].length == 4.5
    assert list(spec.off) == [0, 5, 9]
    with pytest.raises(ValueError):
        A.BatchSpec(systems, [0, 5])
