"""aLENS_set_step_graph: the single-system step recorded as a CUDA graph.

A recorded step launches the one-barrier solver with the whole shared-memory
budget of its launch shape and checks on the device that every block's share
fits; kernels sized by the constraint count run for the capacity and read the
count on the device.  Its results must equal those of steps without a graph
bit for bit, a share that does not fit must fall back to a step without a
graph with nothing moved, and a step whose pairs exceed the capacity must
move nothing and report the required count.
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


def run_steps(s, precision, tol, graph, k_steps=4, fault_at=None, max_pairs=None):
    """k_steps steps from the same state with every output requested."""
    p = A.params_of(s, precision=precision, tol=tol, max_iter=1_000_000)
    out = []
    with A.Context(p, s.n, max_pairs or 12 * s.n) as ctx:
        if graph:
            ctx.set_step_graph(True)
        xd, qd, fd = dev(s.x), dev(s.quat), dev(s.f_nc)
        pr = torch.empty((ctx.max_pairs, 3), dtype=torch.int32, device="cuda")
        gam = torch.empty(ctx.max_pairs, dtype=torch.float64, device="cuda")
        vel = torch.empty((s.n, 6), dtype=torch.float64, device="cuda")
        for k in range(k_steps):
            xd.copy_(dev(s.x)); qd.copy_(dev(s.quat))
            if fault_at == k:
                ctx.inject_fault(2)
            info = ctx.step(xd, qd, fd, pairs_out=pr, gamma_out=gam, vel_out=vel)
            m = info.n_pairs
            out.append((host(xd), host(qd), host(pr)[:m], host(gam)[:m], host(vel), info.as_dict()))
    return out


def assert_same(eager, graph, solver=None):
    for k, (e, g) in enumerate(zip(eager, graph)):
        for a, b in zip(e[:5], g[:5]):
            assert np.array_equal(a, b), k
        for f in ("n_pairs", "n_overlap", "iters", "status", "residual", "min_gap"):
            assert e[5][f] == g[5][f], (k, f)
        if solver is not None:
            assert g[5]["solver"] == solver, k


@pytest.mark.parametrize("name,precision,tol", [("n1000_box40", A.MIXED, 1e-5), ("n1000_box40", A.FP64, 1e-8),
                                                ("n100k_phi010", A.MIXED, 1e-5)])
def test_step_graph_replay_equals_eager(name, precision, tol):
    """The first step runs without a graph, the second records and runs it,
    the last two replay it: every output and counter equals the steps
    without a graph, the replays run the one-barrier solver, and the
    recorded step's launch count repeats."""
    s = W.workload(name)
    eager = run_steps(s, precision, tol, graph=False)
    graph = run_steps(s, precision, tol, graph=True)
    assert eager[0][5]["solver"] == 1   # the workload takes the one-barrier solver
    assert_same(eager, graph, solver=1)
    assert graph[3][5]["launches"] == graph[2][5]["launches"]
    assert graph[2][5]["ms_solve"] > 0.0


def test_step_graph_redo_falls_back_without_moving():
    """A recorded step whose shares do not fit its launch (forced by the test
    hook at the recording) moves nothing on the device and the call runs the
    step without a graph: the results still equal the eager steps, and the
    key stays eager afterwards."""
    s = W.workload("n1000_box40")
    eager = run_steps(s, A.MIXED, 1e-5, graph=False)
    graph = run_steps(s, A.MIXED, 1e-5, graph=True, fault_at=1)
    assert_same(eager, graph)


def test_step_graph_capacity_leaves_the_state_untouched():
    """Replays with the same buffers but a denser arrangement: the pairs
    exceed the capacity, so nothing moves and CAPACITY comes back with the
    required count, as from a step without a graph."""
    s = W.workload("n1000_box40")
    p = A.params_of(s, precision=A.MIXED, tol=1e-5, max_iter=1_000_000)
    dense = s.x * 0.55   # the same rods packed into a corner of the box
    with A.Context(p, s.n, 12 * s.n) as big:
        need = big.step(dev(dense), dev(s.quat), dev(s.f_nc), check=False).n_pairs
        fits = big.step(dev(s.x), dev(s.quat), dev(s.f_nc)).n_pairs
    cap = (need + fits) // 2
    assert fits <= cap < need
    with A.Context(p, s.n, cap) as ctx:
        ctx.set_step_graph(True)
        xd, qd, fd = dev(s.x), dev(s.quat), dev(s.f_nc)
        for k in range(3):   # eager, recorded, replayed: the sparse arrangement fits
            xd.copy_(dev(s.x)); qd.copy_(dev(s.quat))
            assert ctx.step(xd, qd, fd).status == 0
        for k in range(2):   # replays of the dense arrangement
            xd.copy_(dev(dense)); qd.copy_(dev(s.quat))
            with pytest.raises(A.AlensError) as e:
                ctx.step(xd, qd, fd)
            assert e.value.status == 2 and e.value.extra["n_pairs"] == need, k
            assert np.array_equal(host(xd), dense) and np.array_equal(host(qd), s.quat)


def test_step_graph_keeps_eager_where_the_share_does_not_fit():
    """FP64 at 1e5 rods runs the two-barrier solver (a block's share does not
    fit shared memory): the key stays eager and the results are those of
    steps without a graph."""
    s = W.workload("n100k_phi010")
    eager = run_steps(s, A.FP64, 1e-5, graph=False, k_steps=3)
    graph = run_steps(s, A.FP64, 1e-5, graph=True, k_steps=3)
    assert all(g[5]["solver"] != 1 for g in graph)
    assert_same(eager, graph)
