"""Adjoint of the step (aLENS_step_adjoint) through the C ABI.

Small systems: the CUDA gradient against the oracle's adjoint (itself pinned
by central differences of the oracle's forward step, tests/test_oracle_adjoint.py)
element by element — float64 to 1e-7 relative to the largest entry, mixed
(float32 CG operator, float32 BBPGD forward) to 1e-3.  The 2e4-rod
differentiation workload: the oracle's sparse adjoint on its own forward
step, element by element at the same bars; central differences (h = 1e-6)
of the CUDA float64 forward step's loss for sampled centre and orientation
coordinates and the viscosity, plus agreement of the mixed gradient with
the float64 one.  Also the path through a loss on the post-step quaternions,
free drift, determinism, invalid input and the torch.autograd wrapper.
"""
import numpy as np
import pytest

import oracle as O
from oracle import adjoint as ADJ
from paper_2109_08206_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2109_08206_gb300 as A  # noqa: E402

from test_gpu_parity import dev, host  # noqa: E402

SMALL = [(1, 20, 9.0, 3.0), (2, 30, 10.0, 3.0), (3, 16, 8.0, 4.0), (4, 12, 7.0, 3.0)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    A.build()
    assert torch.cuda.is_available()


def small(seed, n, box, L):
    s = W.tiny_system(300 + seed, n, box=box, length=L)
    s.f_nc *= 30.0
    T = s.x + 0.01 * np.random.default_rng(seed).standard_normal(s.x.shape)
    return s, T


def ctx_for(s, precision, tol=None, max_pairs=None):
    tol = tol if tol is not None else (1e-13 if precision == A.FP64 else 1e-7)
    p = A.params_of(s, precision=precision, tol=tol, max_iter=300_000)
    return A.Context(p, s.n, max_pairs or max(64, 12 * s.n))


def gpu_forward(ctx, s, x=None, quat=None, eta=None):
    """(x' unwrapped, quat', pairs, gamma) of one CUDA step from (x, quat)."""
    if eta is not None:
        p = ctx.params
        p.viscosity = eta
        ctx.set_params(p)
    x0 = dev(s.x if x is None else x)
    q0 = dev(s.quat if quat is None else quat)
    xw, qw = x0.clone(), q0.clone()
    vel = torch.empty((s.n, 6), dtype=torch.float64, device="cuda")
    pr = torch.empty((ctx.max_pairs, 3), dtype=torch.int32, device="cuda")
    gam = torch.empty(ctx.max_pairs, dtype=torch.float64, device="cuda")
    info = ctx.step(xw, qw, dev(s.f_nc), pairs_out=pr, gamma_out=gam, vel_out=vel)
    assert info.status == 0
    m = info.n_pairs
    xn = x0 + ctx.params.dt * vel[:, :3]
    return xn, qw, pr[:m].clone(), gam[:m].clone(), x0, q0


def gpu_grad(ctx, s, T, wq=None):
    xn, qn, pr, gam, x0, q0 = gpu_forward(ctx, s)
    gxn = 2.0 * (xn - dev(T))
    gx, gq, gf, geta, info = ctx.step_adjoint(x0, q0, dev(s.f_nc), pr, gam, gxn, None if wq is None else dev(wq))
    return host(gx), host(gq), host(gf), geta, info, host(pr), host(gam)


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


@pytest.mark.parametrize("seed,n,box,L", SMALL)
@pytest.mark.parametrize("precision,bar", [(A.FP64, 1e-7), (A.MIXED, 1e-3)])
def test_adjoint_matches_oracle_adjoint(seed, n, box, L, precision, bar):
    s, T = small(seed, n, box, L)
    with ctx_for(s, precision) as ctx:
        gx, gq, gf, geta, info, pairs, gam = gpu_grad(ctx, s, T)
    ref_L, ref, fw = ADJ.loss_and_grad(s.x, s.quat, s.f_nc, O.problem_of(s), T)
    assert np.array_equal(pairs, fw["pairs"])
    if precision == A.FP64:
        assert np.array_equal(gam > 0, fw["gamma"] > 0)
    assert info.iters > 0
    assert rel(gx, ref["x"]) < bar
    assert rel(gq, ref["quat"]) < bar
    assert rel(gf, ref["fnc"]) < bar
    assert geta == pytest.approx(ref["eta"], rel=bar, abs=bar * abs(ref["eta"]) + 1e-12)


def test_adjoint_through_quaternion_loss():
    s, T = small(2, 30, 10.0, 3.0)
    w = np.random.default_rng(5).standard_normal(s.quat.shape)
    with ctx_for(s, A.FP64) as ctx:
        gx, gq, gf, geta, info, _, _ = gpu_grad(ctx, s, T, wq=w)
    fw = ADJ.forward(s.x, s.quat, s.f_nc, O.problem_of(s))
    ref = ADJ.step_adjoint(s.x, s.quat, s.f_nc, O.problem_of(s), 2.0 * (fw["x"] - T), w, fw=fw)
    assert rel(gx, ref["x"]) < 1e-7
    assert rel(gq, ref["quat"]) < 1e-7
    assert geta == pytest.approx(ref["eta"], rel=1e-7)


def test_adjoint_free_drift_and_determinism():
    s = W.tiny_system(11, 3, box=40.0, length=3.0)
    s.x = np.array([[5.0, 5, 5], [20, 20, 20], [33, 8, 25]])
    T = s.x + 0.1
    with ctx_for(s, A.FP64) as ctx:
        a = gpu_grad(ctx, s, T)
        b = gpu_grad(ctx, s, T)
    xn = s.x + s.dt * ADJ.forward(s.x, s.quat, s.f_nc, O.problem_of(s))["U"][:, :3]
    np.testing.assert_allclose(a[0], 2.0 * (xn - T), rtol=1e-13, atol=1e-15)
    assert a[4].n_pairs == 0
    for u, v in zip(a[:3], b[:3]):
        assert np.array_equal(u, v)
    # a contact system twice: bit-identical
    s, T = small(1, 20, 9.0, 3.0)
    with ctx_for(s, A.MIXED) as ctx:
        a = gpu_grad(ctx, s, T)
        b = gpu_grad(ctx, s, T)
    for u, v in zip(a[:3], b[:3]):
        assert np.array_equal(u, v)
    assert a[3] == b[3]


def test_adjoint_rejects_bad_pairs():
    s, T = small(1, 20, 9.0, 3.0)
    with ctx_for(s, A.FP64) as ctx:
        xn, qn, pr, gam, x0, q0 = gpu_forward(ctx, s)
        bad = pr.clone()
        bad[0, 1] = s.n + 5   # out of range
        with pytest.raises(A.AlensError) as e:
            ctx.step_adjoint(x0, q0, dev(s.f_nc), bad, gam, 2.0 * (xn - dev(T)))
        assert e.value.status == 1


def test_autograd_function_matches_adjoint():
    from paper_2109_08206_gb300.autograd import constrained_step
    s, T = small(3, 16, 8.0, 4.0)
    with ctx_for(s, A.FP64) as ctx:
        x = dev(s.x).requires_grad_(True)
        q = dev(s.quat).requires_grad_(True)
        f = dev(s.f_nc).requires_grad_(True)
        eta = torch.tensor(s.viscosity, dtype=torch.float64, device="cuda", requires_grad=True)
        xn, qn = constrained_step(ctx, x, q, f, eta)
        loss = ((xn - dev(T)) ** 2).sum()
        loss.backward()
        ref_L, ref, _ = ADJ.loss_and_grad(s.x, s.quat, s.f_nc, O.problem_of(s), T)
        assert float(loss.detach()) == pytest.approx(ref_L, rel=1e-10)
        assert rel(host(x.grad), ref["x"]) < 1e-7
        assert rel(host(q.grad), ref["quat"]) < 1e-7
        assert rel(host(f.grad), ref["fnc"]) < 1e-7
        assert float(eta.grad) == pytest.approx(ref["eta"], rel=1e-7)


def test_autograd_backward_uses_its_forward_parameters():
    """Two forwards on one context with different viscosities (and a
    different dt and precision in between) before the first backward: each
    backward gives the oracle gradient at its own forward's parameters, and
    the context keeps the parameters it held before the backward."""
    from paper_2109_08206_gb300.autograd import constrained_step
    s, T = small(2, 30, 10.0, 3.0)
    with ctx_for(s, A.FP64) as ctx:
        outs = []
        for eta_v in (0.7, 1.9):
            x = dev(s.x).requires_grad_(True)
            q = dev(s.quat).requires_grad_(True)
            f = dev(s.f_nc).requires_grad_(True)
            eta = torch.tensor(eta_v, dtype=torch.float64, device="cuda", requires_grad=True)
            xn, qn = constrained_step(ctx, x, q, f, eta)
            outs.append((eta_v, x, q, f, eta, ((xn - dev(T)) ** 2).sum()))
        p = ctx.params
        p.dt = 2e-3
        p.precision = A.MIXED
        ctx.set_params(p)
        before = bytes(ctx.params)
        for eta_v, x, q, f, eta, loss in outs:
            loss.backward()
            s2 = W.RodSystem(x=s.x, quat=s.quat, f_nc=s.f_nc, box=s.box, diameter=s.diameter, length=s.length,
                             viscosity=eta_v, dt=s.dt, delta_c=s.delta_c)
            ref_L, ref, _ = ADJ.loss_and_grad(s.x, s.quat, s.f_nc, O.problem_of(s2), T)
            assert float(loss.detach()) == pytest.approx(ref_L, rel=1e-10)
            assert rel(host(x.grad), ref["x"]) < 1e-7
            assert rel(host(q.grad), ref["quat"]) < 1e-7
            assert rel(host(f.grad), ref["fnc"]) < 1e-7
            assert float(eta.grad) == pytest.approx(ref["eta"], rel=1e-7)
            assert bytes(ctx.params) == before


# ----------------------------------------------------- the 2e4-rod workload

@pytest.fixture(scope="module")
def n20k():
    s = W.workload("n20k_phi015")
    return s, W.loss_targets(s)


def loss_of(ctx, s, T, **kw):
    xn = gpu_forward(ctx, s, **kw)[0]
    return float(((xn - dev(T)) ** 2).sum())


def test_n20k_gradient_against_central_differences(n20k):
    # float64 (a float32 forward's own solve error, about tol D/h in the
    # gradient, swamps a 1e-6 difference; the mixed gradient is compared
    # with the float64 one below)
    s, T = n20k
    h, bar = 1e-6, 2e-4
    with ctx_for(s, A.FP64, tol=1e-13) as ctx:
        gx, gq, gf, geta, info, pairs, gam = gpu_grad(ctx, s, T)
        assert info.status == 0
        rng = np.random.default_rng(3)
        # sampled rods in contact (their gradients carry the constraint terms)
        act = np.unique(pairs[gam > 0][:, :2])
        rods = rng.choice(act, size=6, replace=False)
        for i in rods:
            k = int(rng.integers(3))
            xp, xm = s.x.copy(), s.x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            fd = (loss_of(ctx, s, T, x=xp) - loss_of(ctx, s, T, x=xm)) / (2 * h)
            assert gx[i, k] == pytest.approx(fd, rel=bar, abs=bar * np.abs(gx).max())
            v = np.linalg.svd(s.quat[i].reshape(1, 4))[2][1 + k]
            qp, qm = s.quat.copy(), s.quat.copy()
            qp[i] = (s.quat[i] + h * v) / np.linalg.norm(s.quat[i] + h * v)
            qm[i] = (s.quat[i] - h * v) / np.linalg.norm(s.quat[i] - h * v)
            fd = (loss_of(ctx, s, T, quat=qp) - loss_of(ctx, s, T, quat=qm)) / (2 * h)
            assert gq[i] @ v == pytest.approx(fd, rel=bar, abs=bar * np.abs(gq).max())
        eta0 = s.viscosity
        fd = (loss_of(ctx, s, T, eta=eta0 + h) - loss_of(ctx, s, T, eta=eta0 - h)) / (2 * h)
        assert geta == pytest.approx(fd, rel=bar)


@pytest.fixture(scope="module")
def n20k_oracle(n20k):
    """The float64 oracle's own step (brute-force pairs, FISTA to 1e-13) and
    its sparse adjoint (MINRES on the active system) at 2e4 rods."""
    s, T = n20k
    return ADJ.loss_and_grad(s.x, s.quat, s.f_nc, O.problem_of(s), T, sparse=True, tol=1e-13)


@pytest.mark.parametrize("precision,tol,bar", [(A.FP64, 1e-13, 1e-7), (A.MIXED, 1e-6, 1e-3)])
def test_n20k_gradient_against_sparse_oracle(n20k, n20k_oracle, precision, tol, bar):
    """Element by element (relative to the largest entry) against an
    independent gradient: the oracle's own pair list, solve and sparse
    adjoint on the 2e4-rod differentiation workload."""
    s, T = n20k
    L_o, g_o, fw = n20k_oracle
    with ctx_for(s, precision, tol=tol) as ctx:
        gx, gq, gf, geta, info, pairs, gam = gpu_grad(ctx, s, T)
    assert np.array_equal(pairs, fw["pairs"])
    act_gpu, act_orc = gam > 0, fw["gamma"] > 0
    if precision == A.FP64:
        assert np.array_equal(act_gpu, act_orc)
    err = {k: rel(v, g_o[k]) for k, v in (("x", gx), ("quat", gq), ("fnc", gf))}
    print(f"\nn20k gradient vs sparse oracle ({'fp64' if precision == A.FP64 else 'mixed'}): {err}, "
          f"eta {geta / g_o['eta'] - 1:.2e}, active {int(act_gpu.sum())} / {int(act_orc.sum())}")
    for k, e in err.items():
        assert e < bar, (k, e)
    assert geta == pytest.approx(g_o["eta"], rel=bar)


def test_n20k_mixed_gradient_close_to_fp64(n20k):
    s, T = n20k
    out = {}
    # mixed at 1e-6: on this workload's initial overlaps (velocities of
    # several hundred D/s) the float32 rounding of the reference velocity
    # puts the mixed step's attainable residual near 6e-7
    for prec in (A.FP64, A.MIXED):
        with ctx_for(s, prec, tol=1e-12 if prec == A.FP64 else 1e-6) as ctx:
            out[prec] = gpu_grad(ctx, s, T)
    g64, g32 = out[A.FP64], out[A.MIXED]
    assert rel(g32[0], g64[0]) < 1e-3
    assert rel(g32[1], g64[1]) < 1e-3
    assert g32[3] == pytest.approx(g64[3], rel=1e-3)


def test_adjoint_bounded_wait_times_out_and_context_recovers():
    # one block of the CG leaves before its first grid-wide arrival; the
    # others' bounded waits run out, the call returns TIMEOUT, nothing hangs,
    # and the next call on the same context is exact again
    s, T = small(2, 30, 10.0, 3.0)
    with ctx_for(s, A.FP64) as ctx:
        xn, qn, pr, gam, x0, q0 = gpu_forward(ctx, s)
        ctx.set_wait_limit(0.2)
        ctx.inject_fault(1)
        with pytest.raises(A.AlensError) as e:
            ctx.step_adjoint(x0, q0, dev(s.f_nc), pr, gam, 2.0 * (xn - dev(T)))
        assert e.value.status == 4
        ctx.set_wait_limit(5.0)
        gx, gq, gf, geta, info = ctx.step_adjoint(x0, q0, dev(s.f_nc), pr, gam, 2.0 * (xn - dev(T)))
    ref_L, ref, fw = ADJ.loss_and_grad(s.x, s.quat, s.f_nc, O.problem_of(s), T)
    assert rel(host(gx), ref["x"]) < 1e-7
