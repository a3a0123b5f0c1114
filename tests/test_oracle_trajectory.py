"""Trajectories in the oracle: the counter-based Brownian generator, the
Brownian force's fluctuation-dissipation covariance, free diffusion
(Stokes-Einstein: a step's displacement has covariance 2 kT h M), flat
confining walls, and the first-order convergence in h of the residual
overlaps that the linearised constraints leave (Appendix, "Temporal
discretization": residual overlaps vanish as h -> 0 at first order).
"""
import json
import math
from pathlib import Path

import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_2109_08206_gb300 import workloads as W


def test_normals_are_standard_and_independent():
    z = np.array([O.normals6(12345, 7 + (i % 5), i) for i in range(20000)])   # [20000, 6]
    n = z.size
    assert abs(z.mean()) < 4.0 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 4.0 * math.sqrt(2.0 / n)
    assert stats.kstest(z.ravel(), "norm").pvalue > 1e-4
    c = np.corrcoef(z.T)
    assert np.abs(c - np.eye(6)).max() < 4.0 / math.sqrt(z.shape[0])


def test_generator_matches_published_known_answers():
    """Philox4x32-10 against the known-answer vectors its authors publish
    (Salmon et al., SC'11): pins word order, the hi/lo halves of the
    products and the key schedule, which the statistics below cannot see."""
    kat = json.loads((Path(__file__).parent / "golden" / "philox4x32_10_kat.json").read_text())
    assert len(kat["vectors"]) == 3
    for v in kat["vectors"]:
        ctr = [int(w, 16) for w in v["ctr"]]
        key = [int(w, 16) for w in v["key"]]
        out = [int(w) for w in O.philox4x32(ctr, key)]
        assert out == [int(w, 16) for w in v["out"]], (v, [hex(w) for w in out])


def test_generator_words_differ_across_counters_and_seeds():
    seen = set()
    for seed in (1, 2):
        for step in (0, 1, 2**32 + 1):
            for i in range(200):
                w = O.philox4x32([i, step & 0xFFFFFFFF, step >> 32, 0], [seed & 0xFFFFFFFF, seed >> 32])
                seen.add(tuple(int(v) for v in w))
    assert len(seen) == 2 * 3 * 200
    # one counter bit flipped: every output word changes
    a = O.philox4x32([5, 0, 0, 0], [9, 0])
    b = O.philox4x32([4, 0, 0, 0], [9, 0])
    assert np.all(a != b)


def test_brownian_force_covariance_is_2kT_over_h_times_the_drag():
    pb = O.problem(50.0, 1.0, 6.0, 1.3, 1e-3, 1.0)
    kT = 2.0
    th = np.array([[math.cos(0.4), 0.3 * math.sin(0.4), -0.5 * math.sin(0.4), math.sqrt(1 - 0.34) * math.sin(0.4)]])
    th /= np.linalg.norm(th)
    p = O.axis(th)[0]
    F = np.array([O.brownian(th, pb, kT, 99, k)[0] for k in range(40000)])
    zp, zpar, zr, zs = O.drag(pb.viscosity, pb.length, pb.diameter)
    a = 2.0 * kT / pb.dt
    e1 = np.cross(p, [1.0, 0, 0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(p, e1)
    for blk, (zpar_, zperp_) in ((slice(0, 3), (zpar, zp)), (slice(3, 6), (zs, zr))):
        f = F[:, blk]
        for d, want in ((p, a * zpar_), (e1, a * zperp_), (e2, a * zperp_)):
            assert np.var(f @ d) == pytest.approx(want, rel=5.0 * math.sqrt(2.0 / F.shape[0]))
        assert abs(np.mean((f @ p) * (f @ e1))) < 5.0 * math.sqrt(a * zpar_ * a * zperp_ / F.shape[0])


def test_free_rods_diffuse_with_kT_times_the_mobility():
    # dilute rods, no contacts: one step's displacement along p has variance
    # 2 kT h / zeta_par, across p 2 kT h / zeta_perp per direction
    s = W.tiny_system(5, 400, box=400.0, length=4.0, forces="none")
    pb = O.problem_of(s)
    kT = 1.0
    zp, zpar, _, _ = O.drag(pb.viscosity, pb.length, pb.diameter)
    par, perp = [], []
    p = O.axis(s.quat)
    for k in range(40):
        f = O.brownian(s.quat, pb, kT, 3, k)
        out = O.step(s.x, s.quat, f, pb)
        assert out["pairs"].shape[0] == 0
        dx = out["x"] - O.wrap(s.x, pb.box)
        dx -= np.asarray(pb.box) * np.round(dx / np.asarray(pb.box))
        a = np.sum(dx * p, axis=1)
        par.append(a)
        perp.append(np.linalg.norm(dx - a[:, None] * p, axis=1) ** 2)
    par, perp = np.concatenate(par), np.concatenate(perp)
    n = par.size
    assert np.var(par) == pytest.approx(2 * kT * pb.dt / zpar, rel=5 * math.sqrt(2.0 / n))
    assert np.mean(perp) == pytest.approx(2 * 2 * kT * pb.dt / zp, rel=5 * math.sqrt(1.0 / n))


def test_flat_rod_pushed_into_a_wall_stops_at_contact():
    pb = O.problem(30.0, 1.0, 5.0, 1.0, 1e-3, 1.0)
    x = np.array([[15.0, 15.0, 2.0 + 0.5 + 0.3]])
    q = np.array([[math.cos(math.pi / 4), math.sin(math.pi / 4), 0.0, 0.0]])   # axis along -y: flat on the wall
    f = np.array([[0.0, 0.0, -500.0, 0.0, 0.0, 0.0]])
    for _ in range(30):
        out = O.step(x, q, f, pb, tol=1e-14, walls=(2, 2.0, 28.0))
        x, q = out["x"], out["quat"]
    # translation only: the linearised gap is the exact gap; the rod rests
    # on the wall on both ends, which share the load, and does not rock
    assert x[0, 2] - 0.5 == pytest.approx(2.0, abs=1e-12)
    w = out["walls"]["pairs"]
    assert w.shape[0] == 2 and np.all(w[:, 1] == -1) and sorted(w[:, 2].tolist()) == [0, 1]
    assert np.sum(out["gamma"][-2:]) == pytest.approx(500.0, rel=1e-9)
    assert np.abs(O.axis(q)[0, 2]) < 1e-12


def test_wall_column_acts_on_the_rod_alone():
    s = W.tiny_system(8, 12, box=10.0, length=3.0)
    pb = O.problem(s.box, 1.0, 3.0, 1.0, 1e-3, 1.0)
    wb = O.assemble_walls(s.x, s.quat, s.f_nc, pb, 1, 1.5, 8.0)
    assert wb["pairs"].shape[0] > 0
    g = np.zeros(wb["pairs"].shape[0])
    g[0] = 1.0
    F = O.apply_D(s.n, wb["pairs"], wb["dgeom"], g)
    i = wb["pairs"][0, 0]
    others = np.delete(np.arange(s.n), i)
    assert np.abs(F[others]).max() == 0.0
    assert np.abs(F[i, :3]).max() == 1.0          # the unit normal


def test_residual_overlaps_converge_at_first_order_in_h():
    s = W.tiny_system(91, 40, box=9.0, length=3.0, forces="none")
    worst = []
    for h in (1e-3, 5e-4, 2.5e-4):
        pb = O.problem(s.box, 1.0, 3.0, 1.0, h, 1.0)
        K = int(round(0.02 / h))
        _, _, st = O.trajectory(s.x, s.quat, pb, K, 1.0, 7, tol=1e-12)
        worst.append(-min(d["min_gap"] for d in st[K // 5:]))
    r1, r2 = worst[0] / worst[1], worst[1] / worst[2]
    assert worst[2] > 0
    assert 1.4 < r1 < 3.0 and 1.4 < r2 < 3.0


def test_split_trajectory_equals_one_call():
    s = W.tiny_system(12, 25, box=9.0, length=3.0, forces="none")
    pb = O.problem_of(s)
    xa, qa, _ = O.trajectory(s.x, s.quat, pb, 6, 1.0, 5)
    x1, q1, _ = O.trajectory(s.x, s.quat, pb, 2, 1.0, 5)
    x2, q2, _ = O.trajectory(x1, q1, pb, 4, 1.0, 5, first_step=2)
    np.testing.assert_array_equal(xa, x2)
    np.testing.assert_array_equal(qa, q2)
