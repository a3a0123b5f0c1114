"""Pins of the oracle's complementarity solve and update.

Closed forms (two head-on rods, two rods touching side by side or crossed at
their centres, separated rods), agreement of two independent solvers
(active-set enumeration and accelerated projected gradient), KKT conditions
and optimality of the objective (Appendix, Eq. suppcqpdef and its KKT
equivalence), plus the update's invariants (free drift, spin about the rod
axis, unit quaternions) and the first-order linearisation error of the
scheme (Appendix, end of "Temporal discretization").
"""
import numpy as np
import pytest

import oracle as O
from paper_2109_08206_gb300 import workloads as W

H = 1e-3


def two_rods(dx, p, q, fnc=None, box=60.0):
    x = np.array([[30.0, 30.0, 30.0], [30.0, 30.0, 30.0]])
    x[0] += np.asarray(dx, dtype=float)
    quat = W.quat_from_axis(np.array([p, q], dtype=float))
    f = np.zeros((2, 6)) if fnc is None else np.asarray(fnc, dtype=float)
    pb = O.problem(box, 1.0, 10.0, 1.0, H, 1.0)
    return x, quat, f, pb


def solve_both(x, quat, f, pb):
    pairs = O.find_pairs(x, quat, pb)
    a = O.assemble(x, quat, f, pb, pairs)
    ge, mask = O.solve_enum(quat, pb, pairs, a["dgeom"], a["q"])
    ga, res, it = O.solve_apgd(quat, pb, pairs, a["dgeom"], a["q"], tol=1e-13)
    return pairs, a, ge, mask, ga, res


def test_head_on_overlap_closed_form():
    zp, zpar, _, _ = O.drag(1.0, 10.0, 1.0)
    x, quat, f, pb = two_rods([0, 0, 10.8], [0, 0, 1], [0, 0, 1])     # gap -0.2
    pairs, a, ge, mask, ga, res = solve_both(x, quat, f, pb)
    assert pairs.shape[0] == 1 and a["phi"][0] == pytest.approx(-0.2, abs=1e-13)
    want = 0.2 * zpar / (2 * H)
    assert ge[0] == pytest.approx(want, rel=1e-12)
    assert ga[0] == pytest.approx(want, rel=1e-10)
    xo, qo, U = O.update(x, quat, f, pb, pairs, a["dgeom"], ge)
    # pure axial translation: the linearisation is exact and the gap closes to 0
    assert O.pair_gaps(xo, qo, pb, pairs)[0] == pytest.approx(0.0, abs=1e-12)


@pytest.mark.parametrize("p,q,dx", [([0, 0, 1], [0, 0, 1], [0.9, 0, 0]),
                                    ([1, 0, 0], [0, 1, 0], [0, 0, 0.9])])
def test_centre_contact_closed_form(p, q, dx):
    zp = O.drag(1.0, 10.0, 1.0)[0]
    x, quat, f, pb = two_rods(dx, p, q)
    pairs, a, ge, mask, ga, res = solve_both(x, quat, f, pb)
    assert a["phi"][0] == pytest.approx(-0.1, abs=1e-13)
    want = 0.1 * zp / (2 * H)
    assert ge[0] == pytest.approx(want, rel=1e-12)
    assert ga[0] == pytest.approx(want, rel=1e-10)


def test_separated_rods_drift_freely():
    fnc = [[5, 0, 0, 0, 0, 1], [-5, 0, 0, 0, 0, 0]]       # pushing apart along x
    x, quat, f, pb = two_rods([1.5, 0, 0], [0, 0, 1], [0, 0, 1], fnc)   # gap 0.5
    pairs, a, ge, mask, ga, res = solve_both(x, quat, f, pb)
    assert pairs.shape[0] == 1 and ge[0] == 0.0 and ga[0] == 0.0
    xo, qo, U = O.update(x, quat, f, pb, pairs, a["dgeom"], ge)
    np.testing.assert_allclose(U, O.mobility_apply(quat, pb, f), atol=1e-16)


def _random_tiny(seed, n=8, box=9.0, length=3.0, nematic=None):
    s = W.tiny_system(seed, n, box=box, length=length, nematic_spread=nematic)
    s.f_nc *= 50.0
    return s


def test_enumeration_and_apgd_agree_on_tiny_systems():
    seen = 0
    for seed in range(60):
        s = _random_tiny(seed)
        pb = O.problem_of(s)
        pairs = O.find_pairs(s.x, s.quat, pb)
        if not (2 <= pairs.shape[0] <= 12):
            continue
        a = O.assemble(s.x, s.quat, s.f_nc, pb, pairs)
        ge, mask = O.solve_enum(s.quat, pb, pairs, a["dgeom"], a["q"])
        assert mask >= 0
        ga, res, it = O.solve_apgd(s.quat, pb, pairs, a["dgeom"], a["q"], tol=1e-12)
        assert res <= 1e-12
        # M D gamma (hence U and x') is unique even when gamma is not
        _, _, Ue = O.update(s.x, s.quat, s.f_nc, pb, pairs, a["dgeom"], ge)
        _, _, Ua = O.update(s.x, s.quat, s.f_nc, pb, pairs, a["dgeom"], ga)
        np.testing.assert_allclose(Ua, Ue, atol=1e-7 * (1 + np.abs(Ue).max()))
        A = O.dense_A(s.quat, pb, pairs, a["dgeom"])
        act = ge > 0
        if act.any() and np.linalg.matrix_rank(A[np.ix_(act, act)]) == act.sum() and \
                np.linalg.matrix_rank(A) == A.shape[0]:
            np.testing.assert_allclose(ga, ge, rtol=1e-8, atol=1e-8 * (1 + ge.max()))
        seen += 1
    assert seen >= 15


def test_kkt_and_objective_optimality():
    rng = np.random.default_rng(4)
    s = W.tiny_system(77, 80, box=14.0, length=4.0)
    s.f_nc *= 30.0
    pb = O.problem_of(s)
    pairs = O.find_pairs(s.x, s.quat, pb)
    a = O.assemble(s.x, s.quat, s.f_nc, pb, pairs)
    g0, res, it = O.solve_apgd(s.quat, pb, pairs, a["dgeom"], a["q"], tol=1e-12)
    assert res <= 1e-12
    g, r = O.gradient(s.quat, pb, pairs, a["dgeom"], a["q"], g0)
    assert (g0 >= 0).all()
    assert (H * g).min() >= -1e-9            # linearised post-step gap >= 0
    assert np.abs(g0 * H * g).max() <= 1e-9 * (1 + g0.max())
    A = O.dense_A(s.quat, pb, pairs, a["dgeom"])
    f = lambda v: 0.5 * v @ A @ v + a["q"] @ v
    f0 = f(g0)
    for _ in range(50):
        v = rng.standard_normal(g0.shape[0])
        assert f0 <= f(np.maximum(0.0, g0 + 1e-3 * v)) + 1e-9 * abs(f0)


def test_free_rod_update():
    pb = O.problem(40.0, 1.0, 10.0, 1.0, H, 1.0)
    x = np.array([[1.0, 2.0, 39.9995]])
    axis = np.array([[0.0, 0.6, 0.8]])
    quat = W.quat_from_axis(axis)
    f = np.array([[3.0, -1.0, 2.0, 0.0, 0.0, 0.0]])
    zp, zpar, _, _ = O.drag(1.0, 10.0, 1.0)
    p = axis[0]
    Ut = (p @ f[0, :3]) * p / zpar + (f[0, :3] - (p @ f[0, :3]) * p) / zp
    xo, qo, U = O.update(x, quat, f, pb, np.zeros((0, 3), np.int32), np.zeros((0, 9)), np.zeros(0))
    want = x[0] + H * Ut
    want = want - 40.0 * np.floor(want / 40.0)
    np.testing.assert_allclose(xo[0], want, atol=1e-13)
    np.testing.assert_allclose(qo, quat, atol=1e-15)


def test_spin_about_axis_keeps_axis():
    pb = O.problem(40.0, 1.0, 10.0, 1.0, H, 1.0)
    rng = np.random.default_rng(8)
    axis = W.unit_axes_isotropic(rng, 20)
    quat = W.quat_from_axis(axis)
    f = np.zeros((20, 6)); f[:, 3:6] = 500.0 * axis
    xo, qo, U = O.update(np.full((20, 3), 5.0), quat, f, pb, np.zeros((0, 3), np.int32), np.zeros((0, 9)),
                         np.zeros(0))
    np.testing.assert_allclose(O.axis(qo), axis, atol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(qo, axis=1), 1.0, atol=1e-15)
    assert np.abs(qo - quat).max() > 1e-3      # the quaternion did turn


def test_unit_quaternions_after_step():
    s = W.tiny_system(5, 60, box=16.0, length=4.0)
    pb = O.problem_of(s)
    out = O.step(s.x, s.quat, s.f_nc * 100, pb, tol=1e-11)
    np.testing.assert_allclose(np.linalg.norm(out["quat"], axis=1), 1.0, atol=1e-15)
    assert out["residual"] <= 1e-11


def test_linearisation_error_is_second_order_per_step():
    # Two crossed rods touching off-centre, pressed together: after one step
    # the linearised gap is exactly 0, the true gap differs by O(h^2)
    # because of the rotation (global error O(h), Appendix, end of
    # "Temporal discretization").
    viol = []
    for h in (4e-3, 2e-3, 1e-3):
        fnc = [[0, 0, -400.0, 0, 0, 0], [0, 0, 400.0, 0, 0, 0]]
        x = np.array([[30.0 + 2.0, 30.0 + 1.0, 31.0], [30.0, 30.0, 30.0]])
        quat = W.quat_from_axis(np.array([[1.0, 0.3, 0], [0.2, 1.0, 0]]) /
                                np.linalg.norm([[1.0, 0.3, 0], [0.2, 1.0, 0]], axis=1, keepdims=True))
        pb = O.problem(60.0, 1.0, 10.0, 1.0, h, 1.0)
        pairs = O.find_pairs(x, quat, pb)
        a = O.assemble(x, quat, np.array(fnc), pb, pairs)
        g, res, it = O.solve_apgd(quat, pb, pairs, a["dgeom"], a["q"], tol=1e-14)
        xo, qo, U = O.update(x, quat, np.array(fnc), pb, pairs, a["dgeom"], g)
        viol.append(abs(O.pair_gaps(xo, qo, pb, pairs)[0]))
    r1, r2 = viol[0] / viol[1], viol[1] / viol[2]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0, viol
