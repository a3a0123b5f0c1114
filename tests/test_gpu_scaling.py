"""Diagonal scaling of the BBPGD iteration (aLENS_set_scaling) through the C ABI.

The scaled iteration solves the same CQP (Appendix Eq. suppcqpdef) for
gamma = S gamma~, so every exponent beta must reach the oracle's answer
within the tolerance: the oracle's residual of the returned gamma, U = M D
gamma, and post-step centres, for the unscaled iteration (beta = 0), the
default (0.5) and Jacobi scaling (1), in float64 and mixed precision, on
collisions alone, with bilateral springs (whose compliance is scaled by
sigma^2) and with confining walls (one-sided rows).  Out-of-range exponents
are refused.
"""
import numpy as np
import pytest

import oracle as O
from paper_2109_08206_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2109_08206_gb300 as A  # noqa: E402

from test_gpu_parity import dev, host, make_ctx, periodic_diff, rel_l2  # noqa: E402
from test_gpu_springs import springs_dev  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    A.build()
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def n1000():
    s = W.workload("n1000_box40")
    pb = O.problem_of(s)
    pairs = O.find_pairs(s.x, s.quat, pb)
    asm = O.assemble(s.x, s.quat, s.f_nc, pb, pairs)
    ref = O.step(s.x, s.quat, s.f_nc, pb, tol=1e-13)
    return s, pb, pairs, asm, ref


@pytest.mark.parametrize("beta", [0.0, 0.5, 1.0])
@pytest.mark.parametrize("precision,tol,ubar", [(A.FP64, 1e-9, 1e-6), (A.MIXED, 1e-6, 1e-3)])
def test_scaled_solve_reaches_the_oracle(n1000, beta, precision, tol, ubar):
    s, pb, pairs, asm, ref = n1000
    with make_ctx(s, precision, tol) as ctx:
        ctx.set_scaling(beta)
        g, info = ctx.solve_lcp(dev(s.quat), dev(pairs, torch.int32), dev(asm["dgeom"]), dev(asm["q"]))
        g = host(g)
    assert info.status == 0 and info.residual <= tol
    assert (g >= 0).all()
    # the residual the solver reports is that of the unscaled problem
    _, r = O.gradient(s.quat, pb, pairs, asm["dgeom"], asm["q"], g)
    assert r <= tol * 1.05 + (1e-9 if precision == A.FP64 else 2e-7)
    Ug = O.mobility_apply(s.quat, pb, O.apply_D(s.n, pairs, asm["dgeom"], g))
    Uo = O.mobility_apply(s.quat, pb, O.apply_D(s.n, pairs, asm["dgeom"], ref["gamma"]))
    assert rel_l2(Ug, Uo) <= ubar


def test_scaled_and_unscaled_steps_agree(n1000):
    s, pb, pairs, asm, ref = n1000
    out = {}
    for beta in (0.0, 0.5, 1.0):
        x, q = dev(s.x), dev(s.quat)
        with make_ctx(s, A.FP64, 1e-10) as ctx:
            ctx.set_scaling(beta)
            gam = torch.empty(ctx.max_pairs, dtype=torch.float64, device="cuda")
            info = ctx.step(x, q, dev(s.f_nc), gamma_out=gam)
            assert info.status == 0 and info.residual <= 1e-10
            out[beta] = (host(x), host(q), host(gam)[:info.n_pairs], info.iters)
    for beta in (0.5, 1.0):
        assert np.abs(periodic_diff(out[beta][0], out[0.0][0], s.box)).max() <= 1e-7
        assert np.abs(out[beta][1] - out[0.0][1]).max() <= 1e-7
    assert np.abs(periodic_diff(out[0.5][0], ref["x"], s.box)).max() <= 1e-6


@pytest.mark.parametrize("beta", [0.0, 1.0])
def test_scaled_springs_match_the_oracle(beta):
    s = W.tiny_system(17, 60, box=12.0, length=3.0)
    s.f_nc *= 10.0
    sp = W.spring_set(s, 20, seed=4, kappa=40.0, rest=1.0)
    with make_ctx(s, A.FP64, 1e-11) as ctx:
        ctx.set_scaling(beta)
        ctx.set_springs(*springs_dev(sp))
        x, q = dev(s.x), dev(s.quat)
        info = ctx.step(x, q, dev(s.f_nc))
        assert info.status == 0
        xg = host(x)
    ref = O.step(s.x, s.quat, s.f_nc, O.problem_of(s), tol=1e-13, springs=sp)
    assert np.abs(periodic_diff(xg, ref["x"], s.box)).max() <= 1e-6


@pytest.mark.parametrize("beta", [0.0, 1.0])
def test_scaled_walls_match_the_oracle(beta):
    s = W.tiny_system(31, 40, box=12.0, length=3.0, forces="none")
    s.x[:, 2] = 2.2 + (s.x[:, 2] / 12.0) * 5.6
    f = np.zeros((s.n, 6))
    f[:, 2] = -300.0
    walls = (2, 1.5, 8.5)
    with make_ctx(s, A.FP64, 1e-11) as ctx:
        ctx.set_scaling(beta)
        ctx.set_walls(*walls)
        x, q = dev(s.x), dev(s.quat)
        info, stats = ctx.run(x, q, 6, kT=0.0, seed=3, f_ext=dev(f))
        assert info.status == 0 and any(st["n_walls"] > 0 for st in stats)
        xg = host(x)
    xo, _, _ = O.trajectory(s.x, s.quat, O.problem_of(s), 6, 0.0, 3, f_ext=f, walls=walls, tol=1e-13)
    assert np.abs(periodic_diff(xg, xo, s.box)).max() <= 1e-6


def test_scaling_refuses_out_of_range_exponents(n1000):
    s = n1000[0]
    with make_ctx(s, A.FP64, 1e-8) as ctx:
        for bad in (-0.1, 1.5, float("nan")):
            with pytest.raises(A.AlensError) as e:
                ctx.set_scaling(bad)
            assert e.value.status == 1
        ctx.set_scaling(0.0)
