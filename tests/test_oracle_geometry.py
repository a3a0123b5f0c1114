"""Pins of the oracle's geometry: rod axis, segment-segment distance, pair list.

Each check compares the oracle with something other than itself: closed
forms, a library rotation, brute-force minimisation over a fine grid, or a
hand-built lattice whose pair list is known by construction.
"""
import json
import math
from pathlib import Path

import numpy as np
import pytest

import oracle as O
from paper_2109_08206_gb300 import workloads as W

GOLD = Path(__file__).parent / "golden"


def test_axis_special_cases():
    # identity leaves e_z; a quarter turn about x takes e_z to -e_y; about y to +e_x
    c = math.cos(math.pi / 4)
    q = np.array([[1, 0, 0, 0], [c, c, 0, 0], [c, 0, c, 0], [0, 1, 0, 0]], dtype=float)
    p = O.axis(q)
    np.testing.assert_allclose(p, [[0, 0, 1], [0, -1, 0], [1, 0, 0], [0, 0, -1]], atol=1e-15)


def test_axis_matches_library_rotation():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(7)
    q = rng.standard_normal((200, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    ref = Rotation.from_quat(q[:, [1, 2, 3, 0]]).apply([0.0, 0.0, 1.0])
    np.testing.assert_allclose(O.axis(q), ref, atol=1e-14)


def test_generator_quaternion_maps_ez_to_axis():
    rng = np.random.default_rng(3)
    a = W.unit_axes_isotropic(rng, 500)
    a[0] = [0, 0, -1]
    a[1] = [0, 0, 1]
    np.testing.assert_allclose(O.axis(W.quat_from_axis(a)), a, atol=1e-14)


L = 10.0
ez, ex, ey = np.array([0, 0, 1.0]), np.array([1.0, 0, 0]), np.array([0, 1.0, 0])


def test_head_on_collinear():
    d, s, t = O.segment_closest([0, 0, 13.0], ez, ez, L)
    assert d == pytest.approx(3.0, abs=1e-14)
    assert (s, t) == (-5.0, 5.0)


def test_parallel_side_by_side_midpoint_rule():
    # dx = x_P - x_Q = (0.7, 0, -2): P sits 2 below Q, so Q's points project onto
    # P's axis at s = t + 2 in [-3, 7]; the overlap with [-5, 5] is [-3, 5],
    # its middle s* = 1, and t* = s* - 2 = -1.
    d, s, t = O.segment_closest([0.7, 0, -2.0], ez, ez, L)
    assert d == pytest.approx(0.7, abs=1e-14)
    assert s == pytest.approx(1.0, abs=1e-14)
    assert t == pytest.approx(-1.0, abs=1e-14)
    # anti-parallel rods: same distance
    d2, _, _ = O.segment_closest([0.7, 0, -2.0], ez, -ez, L)
    assert d2 == pytest.approx(0.7, abs=1e-14)


def test_crossed_perpendicular_interior():
    d, s, t = O.segment_closest([1.5, -2.0, 0.8], ex, ey, L)
    assert d == pytest.approx(0.8, abs=1e-14)
    assert s == pytest.approx(-1.5, abs=1e-14) and t == pytest.approx(-2.0, abs=1e-14)


def test_crossed_line_distance_formula():
    rng = np.random.default_rng(11)
    for _ in range(50):
        p = rng.standard_normal(3); p /= np.linalg.norm(p)
        q = rng.standard_normal(3); q /= np.linalg.norm(q)
        n = np.cross(p, q)
        h = rng.uniform(-1, 1)
        s0, t0 = rng.uniform(-3, 3, 2)
        # centres placed so the lines cross at parameters (s0, t0), offset h along n
        dx = -s0 * p + t0 * q + h * n / np.linalg.norm(n)
        d, s, t = O.segment_closest(dx, p, q, L)
        assert d == pytest.approx(abs(dx @ n) / np.linalg.norm(n), abs=1e-12)


def test_end_to_end_skew():
    d, s, t = O.segment_closest([8.0, 0, 0], ex, ey, L)
    assert d == pytest.approx(3.0, abs=1e-14)
    assert s == -5.0 and t == pytest.approx(0.0, abs=1e-14)


def _brute_min(dx, p, q, length, m=2001):
    from scipy.optimize import minimize
    g = np.linspace(-length / 2, length / 2, m)
    r = dx[None, None, :] + g[:, None, None] * p[None, None, :] - g[None, :, None] * q[None, None, :]
    f = np.einsum("abk,abk->ab", r, r)
    a, b = np.unravel_index(np.argmin(f), f.shape)
    fun = lambda st: float(np.sum((dx + st[0] * p - st[1] * q) ** 2))
    res = minimize(fun, [g[a], g[b]], method="L-BFGS-B", bounds=[(-length / 2, length / 2)] * 2,
                   options={"ftol": 1e-16, "gtol": 1e-14, "maxiter": 500})
    return math.sqrt(min(res.fun, f[a, b]))


def test_distance_vs_brute_force_grid():
    rng = np.random.default_rng(5)
    for k in range(40):
        p = rng.standard_normal(3); p /= np.linalg.norm(p)
        q = rng.standard_normal(3); q /= np.linalg.norm(q)
        if k % 8 == 0:   # nearly parallel
            q = p + 1e-4 * rng.standard_normal(3); q /= np.linalg.norm(q)
        dx = rng.uniform(-4, 4, 3)
        d, s, t = O.segment_closest(dx, p, q, 4.0)
        ref = _brute_min(dx, p, q, 4.0)
        assert d <= ref + 1e-9
        assert d == pytest.approx(ref, abs=1e-7)
        assert abs(s) <= 2.0 and abs(t) <= 2.0
        assert math.sqrt(np.sum((dx + s * p - t * q) ** 2)) == pytest.approx(d, abs=1e-13)


def test_lattice_pairs_known_by_construction():
    # 7x7 square lattice of z-aligned rods, spacing 1.8: each rod has 4 nearest
    # neighbours at surface gap 0.8 < delta_c = 1; diagonals (gap 1.55) and all
    # z-images (centre offset 12.6 along z) are out.  98 pairs in total.
    a, nside, bz = 1.8, 7, 12.6
    xs = []
    for ix in range(nside):
        for iy in range(nside):
            xs.append([ix * a + 0.3, iy * a + 0.3, 6.0 + 0.01 * ((ix * 7 + iy) % 5)])
    x = np.array(xs)
    quat = np.tile([1.0, 0, 0, 0], (x.shape[0], 1))
    pb = O.problem((nside * a, nside * a, bz), 1.0, 10.0, 1.0, 1e-3, 1.0)
    pairs = O.find_pairs(x, quat, pb)
    assert pairs.shape[0] == nside * nside * 2
    gaps = O.pair_gaps(x, quat, pb, pairs)
    np.testing.assert_allclose(gaps, 0.8, atol=1e-12)
    idx = lambda ix, iy: ix * nside + iy
    expect = set()
    for ix in range(nside):
        for iy in range(nside):
            for jx, jy in (((ix + 1) % nside, iy), (ix, (iy + 1) % nside)):
                i, j = idx(ix, iy), idx(jx, jy)
                expect.add((min(i, j), max(i, j)))
    assert {(int(i), int(j)) for i, j, _ in pairs} == expect
    # wrapped neighbours carry a non-zero image shift along x or y only
    codes = {int(c) for _, _, c in pairs}
    assert codes <= {13, 12, 14, 10, 16}
    assert any(c != 13 for c in codes)
    # sorted by (i, j, code)
    keys = [tuple(r) for r in pairs.tolist()]
    assert keys == sorted(keys)


def test_four_rod_golden_columns():
    g = json.loads((GOLD / "four_rod_columns.json").read_text())
    pb = O.problem(g["box"], g["diameter"], g["length"], 1.0, 1e-3, g["delta_c"])
    x, quat = np.array(g["x"]), np.array(g["quat"])
    pairs = O.find_pairs(x, quat, pb)
    assert pairs.tolist() == g["pairs"]
    a = O.assemble(x, quat, np.zeros((4, 6)), pb, pairs)
    np.testing.assert_allclose(a["phi"], g["phi"], atol=1e-14)
    np.testing.assert_allclose(a["dgeom"], g["dgeom"], atol=1e-14)
    # the 24 x 2 dense D built column by column from unit gamma
    for c, col in enumerate(("column_0", "column_1")):
        gam = np.zeros(2); gam[c] = 1.0
        F = O.apply_D(4, pairs, a["dgeom"], gam)
        for rod in range(4):
            want = g["D_dense_6x4_by_rod"][col].get(f"rod_{rod}", [0.0] * 6)
            np.testing.assert_allclose(F[rod], want, atol=1e-14)


def test_sampled_rows_match_full_list():
    s = W.tiny_system(9, 60, box=20.0, length=6.0)
    pb = O.problem_of(s)
    full = O.find_pairs(s.x, s.quat, pb)
    rows = [3, 17, 42]
    part = O.find_pairs(s.x, s.quat, pb, rows=rows)
    sel = full[np.isin(full[:, 0], rows) | np.isin(full[:, 1], rows)]
    assert part.tolist() == sel.tolist()
