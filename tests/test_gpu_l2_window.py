"""aLENS_set_l2_window: the global-memory solver's L2 residency of the
constraint states changes addresses' cache treatment only, so a step with
it and one without give the same bits.

The 4e5-rod nematic pack (2.1e6 constraints, about 290 MB of solver data)
is the workload where the window applies: its shares do not fit shared
memory, so the two-barrier kernel reads from global memory.
"""
import numpy as np
import pytest

from paper_2109_08206_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2109_08206_gb300 as A  # noqa: E402


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module", autouse=True)
def _built():
    A.build()
    assert torch.cuda.is_available()


def test_l2_window_changes_no_bit():
    s = W.workload("n400k_nematic")
    p = A.params_of(s, precision=A.MIXED, tol=1e-5, max_iter=1_000_000)
    outs = []
    for enable in (True, False):
        with A.Context(p, s.n, 12 * s.n) as ctx:
            ctx.set_l2_window(enable)
            xd, qd = dev(s.x), dev(s.quat)
            gam = torch.empty(ctx.max_pairs, dtype=torch.float64, device="cuda")
            info = ctx.step(xd, qd, dev(s.f_nc), gamma_out=gam)
            outs.append((host(xd), host(qd), host(gam)[:info.n_pairs], info.iters, info.residual, info.solver))
    assert outs[0][5] == 3 and outs[1][5] == 3   # the global-memory two-barrier kernel ran
    for a, b in zip(outs[0][:3], outs[1][:3]):
        assert np.array_equal(a, b)
    assert outs[0][3:5] == outs[1][3:5]
