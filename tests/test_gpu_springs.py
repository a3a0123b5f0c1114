"""Bilateral spring constraints (aLENS_set_springs + aLENS_step) against the
oracle's combined solve, through the C ABI.

Bars as for the collision step: post-step centres within 1e-6 D (float64) /
2e-5 D (mixed), quaternions alike, U to 1e-6 / 1e-3 relative L2, the
collision pair list bit-exact; the spring forces (unique: the compliance
makes the spring block definite) to the same relative bars; the oracle's
mixed KKT residual of the GPU forces within tolerance.  At 1e5 rods with
5e4 springs: KKT of the GPU forces evaluated by the oracle.
"""
import numpy as np
import pytest

import oracle as O
from paper_2109_08206_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2109_08206_gb300 as A  # noqa: E402

from test_gpu_parity import compare_pairs, dev, host, periodic_diff  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    A.build()
    assert torch.cuda.is_available()


def springs_dev(sp):
    return (dev(sp["ends"], torch.int32), dev(sp["arms"]), dev(sp["kappa"]), dev(sp["rest"]))


def gpu_step(s, sp, precision, tol, max_pairs=None):
    p = A.params_of(s, precision=precision, tol=tol, max_iter=400000)
    nb = 0 if sp is None else len(sp["kappa"])
    with A.Context(p, s.n, max_pairs or max(64, 12 * s.n + nb)) as ctx:
        if sp is not None:
            ctx.set_springs(*springs_dev(sp))
        x, q = dev(s.x), dev(s.quat)
        vel = torch.empty((s.n, 6), dtype=torch.float64, device="cuda")
        pr = torch.empty((ctx.max_pairs, 3), dtype=torch.int32, device="cuda")
        gam = torch.empty(ctx.max_pairs, dtype=torch.float64, device="cuda")
        info = ctx.step(x, q, dev(s.f_nc), pairs_out=pr, gamma_out=gam, vel_out=vel, check=False)
        mu = info.n_pairs
        return info, host(x), host(q), host(vel), host(pr)[:mu], host(gam)[:mu + nb]


CASES = [(51, 18, 9.0, 3.0, 6, 50.0), (52, 30, 10.0, 3.0, 12, 10.0), (53, 40, 12.0, 4.0, 20, 1e4),
         (54, 24, 8.0, 3.0, 10, 0.5)]


@pytest.mark.parametrize("seed,n,box,L,nb,kappa", CASES)
@pytest.mark.parametrize("precision,tol,xbar,ubar", [(A.FP64, 1e-11, 1e-6, 1e-6), (A.MIXED, 1e-6, 2e-5, 1e-3)])
def test_springs_match_oracle(seed, n, box, L, nb, kappa, precision, tol, xbar, ubar):
    s = W.tiny_system(seed, n, box=box, length=L)
    s.f_nc *= 20.0
    sp = W.spring_set(s, nb, seed=seed, kappa=kappa, rest=1.5)
    ref = O.step(s.x, s.quat, s.f_nc, O.problem_of(s), tol=1e-13, springs=sp)
    info, x, q, vel, pairs, gam = gpu_step(s, sp, precision, tol)
    assert info.status == 0 and info.residual <= tol
    compare_pairs(pairs, ref["pairs"], s)
    assert np.abs(periodic_diff(x, ref["x"], s.box)).max() <= xbar
    assert np.abs(q - ref["quat"]).max() <= xbar
    assert np.linalg.norm(vel - ref["U"]) <= ubar * np.linalg.norm(ref["U"])
    mu = pairs.shape[0]
    gb, gb_ref = gam[mu:], ref["gamma"][mu:]
    assert np.linalg.norm(gb - gb_ref) <= ubar * max(np.linalg.norm(gb_ref), 1e-12)
    # the oracle's mixed residual of the GPU forces
    _, r = O.gradient(s.quat, O.problem_of(s), ref["all_pairs"], ref["all_dgeom"], ref["all_q"], gam,
                      comp=ref["comp"])
    assert r <= tol * 1.05 + (1e-9 if precision == A.FP64 else 2e-7)


def test_centre_spring_backward_euler_on_gpu():
    s = W.tiny_system(1, 2, box=60.0, length=4.0)
    s.x = np.array([[20.0, 20.0, 20.0], [23.0, 20.0, 20.0]])
    s.quat = np.tile([1.0, 0.0, 0.0, 0.0], (2, 1))
    s.f_nc = np.zeros((2, 6))
    kappa, rest = 10.0, 1.5
    sp = {"ends": np.array([[0, 1]], dtype=np.int32), "arms": np.zeros((1, 2)), "kappa": np.array([kappa]),
          "rest": np.array([rest])}
    info, x, q, vel, pairs, gam = gpu_step(s, sp, A.FP64, 1e-13)
    assert info.status == 0 and pairs.shape[0] == 0
    zperp = O.drag(1.0, s.length, 1.0)[0]
    want = rest + (3.0 - rest) / (1.0 + s.dt * 2.0 * kappa / zperp)
    assert np.linalg.norm(x[1] - x[0]) == pytest.approx(want, rel=1e-12)


def test_bad_springs_are_rejected_and_nothing_moves():
    s = W.tiny_system(52, 30, box=10.0, length=3.0)
    p = A.params_of(s, precision=A.FP64, tol=1e-10)
    for bad in ({"ends": [[0, 0]], "kappa": [1.0]}, {"ends": [[0, 30]], "kappa": [1.0]},
                {"ends": [[0, 1]], "kappa": [0.0]}):
        sp = {"ends": np.array(bad["ends"], dtype=np.int32), "arms": np.zeros((1, 2)),
              "kappa": np.array(bad["kappa"]), "rest": np.ones(1)}
        with A.Context(p, s.n, 400) as ctx:
            ctx.set_springs(*springs_dev(sp))
            x = dev(s.x)
            info = ctx.step(x, dev(s.quat), dev(s.f_nc), check=False)
            assert info.status == 1
            assert np.array_equal(host(x), s.x)
            ctx.set_springs()   # removed: the context steps again
            info = ctx.step(x, dev(s.quat), dev(s.f_nc), check=False)
            assert info.status == 0


def test_springs_in_a_batch_and_across_systems():
    systems = [W.tiny_system(61 + k, 20, box=9.0, length=3.0) for k in range(3)]
    off, x, quat, fnc, spec = W.batch_arrays(systems)
    sps = [W.spring_set(s, 5, seed=70 + k, kappa=20.0) for k, s in enumerate(systems)]
    ends = np.concatenate([sp["ends"] + off[k] for k, sp in enumerate(sps)]).astype(np.int32)
    sp_all = {"ends": ends, "arms": np.concatenate([sp["arms"] for sp in sps]),
              "kappa": np.concatenate([sp["kappa"] for sp in sps]), "rest": np.concatenate([sp["rest"] for sp in sps])}
    p = A.make_params(9.0, 1.0, 3.0, 1.0, 1e-3, 1.0, 1e-11, 400000, A.FP64)
    with A.Context(p, int(off[-1]), 2000) as ctx:
        ctx.set_springs(*springs_dev(sp_all))
        xd, qd = dev(x), dev(quat)
        vel = torch.empty((int(off[-1]), 6), dtype=torch.float64, device="cuda")
        info = ctx.step_batch(spec, off, xd, qd, dev(fnc), vel_out=vel)
        assert info.status == 0
        for k, s in enumerate(systems):
            ref = O.step(s.x, s.quat, s.f_nc, O.problem_of(s), tol=1e-13, springs=sps[k])
            lo, hi = off[k], off[k + 1]
            assert np.abs(periodic_diff(host(xd)[lo:hi], ref["x"], s.box)).max() <= 1e-6
            U = host(vel)[lo:hi]
            assert np.linalg.norm(U - ref["U"]) <= 1e-6 * np.linalg.norm(ref["U"])
        # a spring between two systems is refused
        bad = dict(sp_all)
        bad["ends"] = sp_all["ends"].copy()
        bad["ends"][0, 1] = off[1] + 3
        ctx.set_springs(*springs_dev(bad))
        info = ctx.step_batch(spec, off, dev(x), dev(quat), dev(fnc), check=False)
        assert info.status == 1


@pytest.mark.parametrize("precision,tol", [(A.MIXED, 1e-5), (A.FP64, 1e-6)])
def test_n100k_with_bilateral_springs_kkt(precision, tol):
    s = W.workload("n100k_phi010", n_springs=0)
    sp = W.spring_set(s, 50_000, seed=21)
    pb = O.problem_of(s)
    info, x, q, vel, pairs, gam = gpu_step(s, sp, precision, tol, max_pairs=12 * s.n + 50_000)
    assert info.status == 0 and info.residual <= tol
    mu = pairs.shape[0]
    asm = O.assemble(s.x, s.quat, s.f_nc, pb, pairs)
    sb = O.assemble_springs(s.x, s.quat, s.f_nc, pb, sp["ends"], sp["arms"], sp["kappa"], sp["rest"])
    allp = np.concatenate([pairs, sb["pairs"]])
    dg = np.concatenate([asm["dgeom"], sb["dgeom"]])
    qq = np.concatenate([asm["q"], sb["q"]])
    comp = np.concatenate([-np.ones(mu), sb["comp"]])
    _, r = O.gradient(s.quat, pb, allp, dg, qq, gam, comp=comp)
    assert r <= tol * 1.05 + (2e-7 if precision == A.MIXED else 1e-9)
    assert gam[:mu].min() >= 0.0
    # the update: U = M (F_nc + D gamma) recomputed by the oracle
    F = O.apply_D(s.n, allp, dg, gam) + s.f_nc
    U = O.mobility_apply(s.quat, pb, F)
    assert np.linalg.norm(vel - U) <= 1e-6 * np.linalg.norm(U)
