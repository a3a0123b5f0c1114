"""Bilateral (spring) constraints in the oracle, pinned by closed forms.

Appendix: Phi_b is the distance between two fixed points of particles P and
Q, K [Phi_b - Phi_b^0] = -gamma_b, linearised as Eq. linearconstraints b and
solved together with the collisions (Eq. blockdef D, F: the diagonal
compliance K^{-1}/h and no projection).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2109_08206_gb300 import workloads as W


def two_rods(gap_axis=0, ell=3.0, box=60.0, length=4.0):
    """Two parallel rods along z, centres ell apart along x."""
    x = np.array([[20.0, 20.0, 20.0], [20.0 + ell, 20.0, 20.0]])
    quat = np.tile([1.0, 0.0, 0.0, 0.0], (2, 1))   # axis e_z
    return x, quat, O.problem(box, 1.0, length, 1.0, 1e-3, 1.0)


def test_centre_spring_is_backward_euler_of_the_overdamped_spring():
    # spring between the two centres, perpendicular to both rods: the
    # linearised step is backward Euler for d(ell)/dt = -(2 kappa / zeta_perp)(ell - ell0)
    for ell, kappa, rest in [(3.0, 10.0, 1.5), (2.5, 1e3, 4.0), (5.0, 0.3, 2.0)]:
        x, quat, pb = two_rods(ell=ell)
        sp = {"ends": [[0, 1]], "arms": [[0.0, 0.0]], "kappa": [kappa], "rest": [rest]}
        out = O.step(x, quat, np.zeros((2, 6)), pb, tol=1e-14, springs=sp)
        assert out["pairs"].shape[0] == 0
        zperp = O.drag(1.0, pb.length, 1.0)[0]
        lam = 2.0 * kappa / zperp
        want = rest + (ell - rest) / (1.0 + pb.dt * lam)
        got = np.linalg.norm(out["x"][1] - out["x"][0])
        assert got == pytest.approx(want, rel=1e-12)
        # the spring force is Hookean at the new (linearised) length: gamma = -kappa (ell' - ell0)
        assert out["gamma"][0] == pytest.approx(-kappa * (want - rest), rel=1e-10)


def test_stiff_spring_holds_its_rest_length_to_first_order():
    x, quat, pb = two_rods(ell=3.0)
    sp = {"ends": [[0, 1]], "arms": [[1.2, -0.7]], "kappa": [1e12], "rest": [2.9]}
    rng = np.random.default_rng(2)
    f = rng.standard_normal((2, 6))
    out = O.step(x, quat, f, pb, tol=1e-14, springs=sp)
    sb = out["springs"]
    # linearised length after the step: Phi_b + h D_b^T U
    U = out["U"]
    dg = sb["dgeom"][0]
    dtu = dg[:3] @ (U[0, :3] - U[1, :3]) + dg[3:6] @ U[0, 3:] - dg[6:9] @ U[1, 3:]
    # Eq. linearconstraints b: Phi_b + h D_b^T U - Phi_b^0 = -gamma_b / kappa (1e-9 here)
    gb = out["gamma"][-1]
    assert sb["length"][0] + pb.dt * dtu == pytest.approx(2.9 - gb / 1e12, abs=1e-12)
    assert abs(gb / 1e12) < 1e-8


def test_soft_spring_matches_the_explicit_spring_force():
    # kappa h / zeta -> 0: the implicit spring force tends to the explicit
    # Hookean force -kappa (ell - ell0) e on P (and its torque y_P x F), the
    # opposite on Q
    x, quat, pb = two_rods(ell=3.0)
    q2 = np.array([[math.cos(0.3), math.sin(0.3), 0.0, 0.0], [math.cos(0.5), 0.0, math.sin(0.5), 0.0]])
    sP, sQ, kappa, rest = 1.1, -0.6, 1e-4, 2.0
    sp = {"ends": [[0, 1]], "arms": [[sP, sQ]], "kappa": [kappa], "rest": [rest]}
    out = O.step(x, q2, np.zeros((2, 6)), pb, tol=1e-15, springs=sp)
    p = O.axis(q2)
    a, b = x[0] + sP * p[0], x[1] + sQ * p[1]
    ell = np.linalg.norm(a - b)
    e = (a - b) / ell
    F = np.zeros((2, 6))
    F[0, :3] = -kappa * (ell - rest) * e
    F[0, 3:] = np.cross(sP * p[0], F[0, :3])
    F[1, :3] = -F[0, :3]
    F[1, 3:] = np.cross(sQ * p[1], F[1, :3])
    U_explicit = O.mobility_apply(q2, pb, F)
    np.testing.assert_allclose(out["U"], U_explicit, rtol=1e-6, atol=1e-9 * np.abs(U_explicit).max())


def test_springs_with_collisions_satisfy_the_mixed_kkt_conditions():
    s = W.tiny_system(41, 18, box=9.0, length=3.0)
    s.f_nc *= 10.0
    sp = W.spring_set(s, 6, seed=4, kappa=50.0, rest=1.5)
    pb = O.problem_of(s)
    out = O.step(s.x, s.quat, s.f_nc, pb, tol=1e-13, springs=sp)
    mu = out["pairs"].shape[0]
    assert mu > 0 and out["all_pairs"].shape[0] == mu + 6
    g, r = O.gradient(s.quat, pb, out["all_pairs"], out["all_dgeom"], out["all_q"], out["gamma"], comp=out["comp"])
    gu, gb = g[:mu], g[mu:]
    gam_u = out["gamma"][:mu]
    assert gam_u.min() >= 0.0
    assert gu.min() >= -1e-9 * np.abs(out["all_q"]).max()
    assert np.abs(gam_u * gu).max() <= 1e-9 * (1 + np.abs(gam_u).max() * np.abs(gu).max())
    assert np.abs(gb).max() <= 1e-9 * (1 + np.abs(out["all_q"]).max())
    # two independent solvers agree (when the system is small enough to enumerate)
    m = out["all_pairs"].shape[0]
    if m <= 20:
        ge, _ = O.solve_enum(s.quat, pb, out["all_pairs"], out["all_dgeom"], out["all_q"], comp=out["comp"])
        ga, _, _ = O.solve_apgd(s.quat, pb, out["all_pairs"], out["all_dgeom"], out["all_q"], tol=1e-13,
                                comp=out["comp"])
        np.testing.assert_allclose(ga, ge, rtol=1e-6, atol=1e-8 * np.abs(ge).max())


def test_combined_matrix_is_spsd_with_the_compliance_on_the_diagonal():
    s = W.tiny_system(42, 14, box=8.0, length=3.0)
    sp = W.spring_set(s, 5, seed=5, kappa=7.0, rest=1.0)
    pb = O.problem_of(s)
    pairs = O.find_pairs(s.x, s.quat, pb)
    a = O.assemble(s.x, s.quat, s.f_nc, pb, pairs)
    sb = O.assemble_springs(s.x, s.quat, s.f_nc, pb, sp["ends"], sp["arms"], sp["kappa"], sp["rest"])
    allp = np.concatenate([pairs, sb["pairs"]])
    dg = np.concatenate([a["dgeom"], sb["dgeom"]])
    comp = np.concatenate([-np.ones(len(pairs)), sb["comp"]])
    A0 = O.dense_A(s.quat, pb, allp, dg)
    A1 = O.dense_A(s.quat, pb, allp, dg, comp=comp)
    np.testing.assert_allclose(A1, A1.T, atol=1e-12 * np.abs(A1).max())
    d = np.diag(A1 - A0)
    np.testing.assert_allclose(d[len(pairs):], 1.0 / (pb.dt * 7.0), rtol=1e-14)
    assert np.abs(d[:len(pairs)]).max() == 0.0
    assert np.linalg.eigvalsh(A1).min() > 0.0   # the compliance makes the spring block definite
