"""Trajectories (aLENS_run) and their parts through the C ABI, against the
oracle: the counter-based generator's raw words bit for bit, the Brownian
forces, multi-step runs with walls and springs (float64 and mixed), the warm
start (same trajectory within tolerance, fewer iterations on a loaded pile),
a run split into calls equal to one call, and confinement at 2e4 rods.
"""
import numpy as np
import pytest

import oracle as O
from paper_2109_08206_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2109_08206_gb300 as A  # noqa: E402

from test_gpu_parity import dev, host, periodic_diff  # noqa: E402
from test_gpu_springs import springs_dev  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    A.build()
    assert torch.cuda.is_available()


def ctx_of(s, precision=A.FP64, tol=1e-12, max_pairs=None):
    p = A.params_of(s, precision=precision, tol=tol, max_iter=400000)
    return A.Context(p, s.n, max_pairs or max(256, 14 * s.n))


@pytest.mark.parametrize("seed,step", [(0, 0), (12345, 7), (2**40 + 3, 2**33 + 5)])
def test_generator_words_bit_exact(seed, step):
    s = W.tiny_system(1, 300, box=40.0)
    with ctx_of(s) as ctx:
        got = host(ctx.random_words(300, seed, step)).view(np.uint32)
    for i in (0, 1, 2, 150, 299):
        for h in range(2):
            ctr = [i, step & 0xFFFFFFFF, step >> 32, h]
            want = O.philox4x32(ctr, [seed & 0xFFFFFFFF, seed >> 32])
            assert np.array_equal(got[i, 4 * h:4 * h + 4], want)


def test_generator_first_word_block_is_published_known_answer():
    """Rod 0, step 0, seed 0 is Philox4x32-10 at counter 0 and key 0, whose
    output its authors publish (Salmon et al., SC'11): the GPU generator is
    pinned to the definition itself, not only to the oracle."""
    import json
    from pathlib import Path
    kat = json.loads((Path(__file__).parent / "golden" / "philox4x32_10_kat.json").read_text())
    v = kat["vectors"][0]
    assert all(int(w, 16) == 0 for w in v["ctr"] + v["key"])
    s = W.tiny_system(1, 4, box=40.0)
    with ctx_of(s) as ctx:
        got = host(ctx.random_words(4, 0, 0)).view(np.uint32)
    assert [int(w) for w in got[0, :4]] == [int(w, 16) for w in v["out"]]


def test_brownian_forces_match_oracle():
    s = W.tiny_system(2, 500, box=40.0, length=4.0)
    fext = np.random.default_rng(1).standard_normal((s.n, 6))
    with ctx_of(s) as ctx:
        for step in (0, 17):
            got = host(ctx.brownian(dev(s.quat), 1.7, 99, step, dev(fext)))
            want = O.brownian(s.quat, O.problem_of(s), 1.7, 99, step, fext)
            np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("precision,tol,bar", [(A.FP64, 1e-12, 1e-6), (A.MIXED, 1e-7, 1e-4)])
def test_run_with_walls_and_springs_matches_oracle(precision, tol, bar):
    s = W.tiny_system(31, 40, box=12.0, length=3.0, forces="none")
    s.x[:, 2] = 2.2 + (s.x[:, 2] / 12.0) * 5.6   # inside the walls at z = 1.5 and 8.5
    sp = W.spring_set(s, 8, seed=3, kappa=30.0, rest=1.2)
    walls = (2, 1.5, 8.5)
    K = 12
    with ctx_of(s, precision, tol) as ctx:
        ctx.set_walls(*walls)
        ctx.set_springs(*springs_dev(sp))
        x, q = dev(s.x), dev(s.quat)
        info, stats = ctx.run(x, q, K, kT=1.0, seed=21)
        assert info.status == 0 and len(stats) == K
        assert any(st["n_walls"] > 0 for st in stats)
        xg, qg = host(x), host(q)
    xo, qo, st_o = O.trajectory(s.x, s.quat, O.problem_of(s), K, 1.0, 21, springs=sp, walls=walls, tol=1e-13)
    assert np.abs(periodic_diff(xg, xo, s.box)).max() <= bar
    assert np.abs(qg - qo).max() <= bar
    assert [st["n_pairs"] for st in stats] == [d["n_pairs"] for d in st_o]


def test_warm_start_same_trajectory_fewer_iterations():
    # a pile pushed onto a wall by a steady load: contacts persist from step
    # to step, so the previous step's forces are a good start (with fresh
    # thermal noise every step, or a fast-moving suspension, they are not:
    # measured on the 2e4-rod workload, the iteration counts are then alike)
    s = W.tiny_system(31, 60, box=12.0, length=3.0, forces="none")
    s.x[:, 2] = 2.2 + (s.x[:, 2] / 12.0) * 5.6
    f = np.zeros((s.n, 6))
    f[:, 2] = -200.0
    out = {}
    tol = 1e-8
    for warm in (False, True):
        with ctx_of(s, A.FP64, tol, max_pairs=2000) as ctx:
            ctx.set_walls(2, 1.5, 8.5)
            x, q = dev(s.x), dev(s.quat)
            info, stats = ctx.run(x, q, 5, kT=0.0, seed=5, f_ext=dev(f), warm_start=warm)
            x5 = host(x)
            info, stats2 = ctx.run(x, q, 195, kT=0.0, seed=5, first_step=5, f_ext=dev(f), warm_start=warm)
            assert all(st["residual"] <= tol for st in stats + stats2)
            out[warm] = (x5, [st["iters"] for st in stats + stats2])
    assert np.abs(periodic_diff(out[True][0], out[False][0], s.box)).max() < 1e-5
    it_cold, it_warm = out[False][1], out[True][1]
    assert it_warm[0] == it_cold[0]                 # the first step has nothing to start from
    assert sum(it_warm[50:]) < 0.85 * sum(it_cold[50:])


def test_split_run_equals_one_run():
    s = W.tiny_system(44, 60, box=12.0, length=3.0, forces="none")
    res = []
    for chunks in ((6,), (2, 4)):
        with ctx_of(s, A.MIXED, 1e-7) as ctx:
            x, q = dev(s.x), dev(s.quat)
            first = 0
            for c in chunks:
                ctx.run(x, q, c, kT=1.0, seed=8, first_step=first)
                first += c
            res.append((host(x), host(q)))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_confinement_at_2e4_rods():
    s = W.workload("n20k_phi015")
    box = s.box[2]
    lo, hi = 5.0, box - 12.0 - 5.0
    inside = (s.x[:, 2] > lo + 6.0) & (s.x[:, 2] < hi - 6.0)
    x0 = s.x.copy()
    x0[~inside, 2] = lo + 6.0 + (x0[~inside, 2] / box) * (hi - lo - 12.0)   # start away from the walls
    s.x = x0
    f = np.zeros((s.n, 6))
    f[:, 2] = -5000.0   # push everything towards the lower wall (about 0.12 D per step)
    with ctx_of(s, A.MIXED, 1e-6) as ctx:
        ctx.set_walls(2, lo, hi)
        x, q = dev(s.x), dev(s.quat)
        info, stats = ctx.run(x, q, 40, kT=1.0, seed=9, f_ext=dev(f))
        assert info.status == 0
        assert stats[-1]["n_walls"] > 200
        z = host(x)[:, 2]
        p = O.axis(host(q))
        lowest = z - np.abs(p[:, 2]) * s.length / 2 - s.diameter / 2
        # residual overlaps with the wall stay of the order of the step's linearisation error
        assert lowest.min() > lo - 0.25
        assert z.min() > lo and z.max() < hi
