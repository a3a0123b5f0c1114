"""Pins of the oracle's constraint assembly and mobility.

- D against finite differences of the distance function: the paper's
  theorem grad_C Phi G = D^T (Appendix "Symmetry of the geometrically
  constrained optimization problem").  Phi is re-evaluated as a minimum
  distance at perturbed configurations, so a wrong sign, a swapped torque arm
  or a transposed cross product fails here.
- zero net force and zero net torque about the origin for every column.
- M: the parallel/perpendicular eigen-structure of the slender-rod mobility,
  symmetric positive definiteness, and the printed value of the slender-body
  drag coefficient (Section 3).
- D^T M D symmetric positive semi-definite (Appendix, SPSD of the CQP matrix).
"""
import json
import math
from pathlib import Path

import numpy as np
import pytest

import oracle as O
from paper_2109_08206_gb300 import workloads as W

GOLD = Path(__file__).parent / "golden"


def qmul(a, b):
    s1, v1, s2, v2 = a[0], a[1:], b[0], b[1:]
    return np.concatenate([[s1 * s2 - v1 @ v2], s1 * v2 + s2 * v1 + np.cross(v1, v2)])


def rotate(quat, omega_hat, eps):
    r = np.concatenate([[math.cos(eps / 2)], math.sin(eps / 2) * np.asarray(omega_hat)])
    return qmul(r, quat)


def _close_pairs(seed=21, n=40):
    s = W.tiny_system(seed, n, box=16.0, length=4.0)
    pb = O.problem_of(s)
    pairs = O.find_pairs(s.x, s.quat, pb)
    return s, pb, pairs


def test_D_matches_finite_difference_of_distance():
    s, pb, pairs = _close_pairs()
    assert pairs.shape[0] >= 10
    a = O.assemble(s.x, s.quat, s.f_nc, pb, pairs)
    eps = 1e-6
    checked = 0
    for c, (i, j, code) in enumerate(pairs[:25]):
        if a["phi"][c] + pb.diameter < 1e-3:
            continue  # centrelines touching: Phi is not differentiable there
        one = np.array([[i, j, code]], dtype=np.int32)
        col = np.zeros(12)
        for side, rod in ((0, i), (1, j)):
            for k in range(3):
                num = []
                for sg in (+1, -1):
                    x = s.x.copy(); x[rod, k] += sg * eps
                    num.append(O.pair_gaps(x, s.quat, pb, one)[0])
                col[6 * side + k] = (num[0] - num[1]) / (2 * eps)
                num = []
                for sg in (+1, -1):
                    q = s.quat.copy(); w = np.zeros(3); w[k] = 1.0
                    q[rod] = rotate(q[rod], w, sg * eps)
                    num.append(O.pair_gaps(s.x, q, pb, one)[0])
                col[6 * side + 3 + k] = (num[0] - num[1]) / (2 * eps)
        dg = a["dgeom"][c]
        want = np.concatenate([dg[0:3], dg[3:6], -dg[0:3], -dg[6:9]])
        np.testing.assert_allclose(col, want, atol=2e-6)
        checked += 1
    assert checked >= 10


def test_zero_net_force_and_torque_per_column():
    s, pb, pairs = _close_pairs(23, 50)
    a = O.assemble(s.x, s.quat, s.f_nc, pb, pairs)
    xw = O.wrap(s.x, s.box)
    box = np.asarray(s.box)
    for c, (i, j, code) in enumerate(pairs):
        k = np.array([code % 3 - 1, (code // 3) % 3 - 1, code // 9 - 1])
        e = a["dgeom"][c, 0:3]
        xP, xQ = xw[i], xw[j] + k * box          # Q at the image it was paired with
        torque = np.cross(xP, e) + a["dgeom"][c, 3:6] - np.cross(xQ, e) - a["dgeom"][c, 6:9]
        np.testing.assert_allclose(torque, 0.0, atol=1e-12 * (1 + np.abs(xP).max()))
        r = xP + a["yP"][c] - xQ - a["yQ"][c]
        assert np.linalg.norm(r) - pb.diameter == pytest.approx(a["phi"][c], abs=1e-12)
        assert abs(np.linalg.norm(e) - 1.0) < 1e-14
        # e is along r: P is pushed away from Q when gamma > 0
        assert r @ e == pytest.approx(np.linalg.norm(r), abs=1e-12)


def test_mobility_eigenstructure_and_spd():
    rng = np.random.default_rng(2)
    pb = O.problem(40.0, 1.0, 10.0, 1.0, 1e-3, 1.0)
    zp, zpar, zr, zs = O.drag(1.0, 10.0, 1.0)
    assert zpar == pytest.approx(zp / 2) and zr == pytest.approx(zp * 100 / 12)
    axes = W.unit_axes_isotropic(rng, 5)
    quat = W.quat_from_axis(axes)
    for r in range(5):
        p = axes[r]
        u = np.cross(p, rng.standard_normal(3)); u /= np.linalg.norm(u)
        F = np.zeros((4, 6)); F[0, 0:3] = p; F[1, 0:3] = u; F[2, 3:6] = p; F[3, 3:6] = u
        U = O.mobility_apply(np.tile(quat[r], (4, 1)), pb, F)
        np.testing.assert_allclose(U[0, 0:3], p / zpar, atol=1e-15)
        np.testing.assert_allclose(U[1, 0:3], u / zp, atol=1e-15)
        np.testing.assert_allclose(U[2, 3:6], p / zs, atol=1e-15)
        np.testing.assert_allclose(U[3, 3:6], u / zr, atol=1e-15)
        assert np.abs(U[0:2, 3:6]).max() == 0 and np.abs(U[2:4, 0:3]).max() == 0
        M = O.mobility_apply(np.tile(quat[r], (6, 1)), pb, np.eye(6))
        np.testing.assert_allclose(M, M.T, atol=1e-16)
        assert np.linalg.eigvalsh(M).min() > 0


def test_printed_drag_coefficient():
    g = json.loads((GOLD / "drag_coefficient.json").read_text())
    inp, pr = g["inputs"], g["printed"]
    zeta_perp = O.drag(inp["eta_pN_s_per_um2"], inp["length_um"], inp["diameter_um"])[0]
    # printed to one significant figure
    assert abs(zeta_perp - pr["drag_pN_s_per_um"]) <= 0.5e-3
    tau = zeta_perp / (inp["n_motors"] * inp["k_pN_per_um"])
    assert abs(tau - pr["relaxation_time_s"]) <= 0.5e-6


def test_cqp_matrix_is_spsd():
    s, pb, pairs = _close_pairs(31, 30)
    a = O.assemble(s.x, s.quat, s.f_nc, pb, pairs)
    A = O.dense_A(s.quat, pb, pairs, a["dgeom"])
    np.testing.assert_allclose(A, A.T, atol=1e-15 * np.abs(A).max())
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.min() >= -1e-12 * ev.max()


def test_q_is_gap_rate_plus_free_drift():
    # q = Phi/h + D^T M F_nc (Appendix, block A): compare with the pieces
    s, pb, pairs = _close_pairs(37, 40)
    a = O.assemble(s.x, s.quat, s.f_nc, pb, pairs)
    U = O.mobility_apply(s.quat, pb, s.f_nc)
    want = a["phi"] / pb.dt + O.apply_Dt(pairs, a["dgeom"], U)
    np.testing.assert_allclose(a["q"], want, rtol=1e-13, atol=1e-10)
    # D^T is the adjoint of D: <D g, U> = <g, D^T U>
    rng = np.random.default_rng(0)
    gam = rng.standard_normal(pairs.shape[0])
    F = O.apply_D(s.n, pairs, a["dgeom"], gam)
    assert np.sum(F * U) == pytest.approx(gam @ O.apply_Dt(pairs, a["dgeom"], U), rel=1e-12)
