"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on
the same seeded inputs.

Bars:
- pair lists: bit-exact (i, j, image) triples, sorted, on every input (all
  inputs are fixed by their seeds): no mismatch is excused.  A failure
  prints the oracle's float64 gaps of the differing pairs.
- assembly (float64 both sides): Phi and q to 1e-12 relative, D records to
  1e-9 absolute (closest-point arms are ill-conditioned for near-parallel
  rods).
- solve: U = M D gamma (unique even when gamma is not) to 1e-5 relative L2 in
  float64 mode and 1e-3 in mixed mode; gamma itself to the same bars when the
  oracle's active-set block is full rank; the oracle's own residual of the
  GPU gamma must meet the tolerance.
- step: post-step centres within 1e-6 D (float64) / 1e-5 D (mixed) of the
  oracle's, quaternions likewise.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2109_08206_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2109_08206_gb300 as A  # noqa: E402


def dev(a, dtype=None):
    dtype = dtype or torch.float64
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module", autouse=True)
def _built():
    A.build()
    assert torch.cuda.is_available()


def make_ctx(s, precision=A.FP64, tol=None, max_pairs=None, max_iter=200000):
    p = A.params_of(s, precision=precision, tol=tol, max_iter=max_iter)
    mp = max_pairs or max(64, 12 * s.n)
    return A.Context(p, s.n, mp)


def compare_pairs(gpu, orc, s):
    """Pair lists equal as sorted (i, j, image) triples; returns 0 (kept for
    callers that assert it).  On a mismatch the message carries the differing
    triples and the oracle's float64 gaps minus delta_c."""
    gpu = np.asarray(gpu).reshape(-1, 3)
    orc = np.asarray(orc).reshape(-1, 3)
    keys = [tuple(r) for r in gpu.tolist()]
    assert keys == sorted(keys), "GPU pair list not sorted by (i, j, image)"
    if gpu.shape == orc.shape and np.array_equal(gpu, orc):
        return 0
    g, o = set(keys), {tuple(r) for r in orc.tolist()}
    diff = np.array(sorted(g ^ o), dtype=np.int32).reshape(-1, 3)
    gaps = O.pair_gaps(s.x, s.quat, O.problem_of(s), diff) if diff.size else np.zeros(0)
    raise AssertionError(f"{diff.shape[0]} pairs differ (GPU {gpu.shape[0]}, oracle {orc.shape[0]}): "
                         f"{diff[:5].tolist()} gap - delta_c {(gaps[:5] - s.delta_c).tolist()}")


def periodic_diff(a, b, box):
    d = a - b
    bx = np.asarray(box)
    return d - bx * np.round(d / bx)


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


# --------------------------------------------------------------------- n1000

@pytest.fixture(scope="module")
def n1000():
    s = W.workload("n1000_box40")
    pb = O.problem_of(s)
    pairs = O.find_pairs(s.x, s.quat, pb)
    asm = O.assemble(s.x, s.quat, s.f_nc, pb, pairs)
    gam, res, it = O.solve_apgd(s.quat, pb, pairs, asm["dgeom"], asm["q"], tol=1e-12, max_iter=2_000_000)
    assert res <= 1e-11
    xo, qo, Uo = O.update(s.x, s.quat, s.f_nc, pb, pairs, asm["dgeom"], gam)
    return s, pb, pairs, asm, gam, (xo, qo, Uo)


def test_neighbors_n1000_bit_exact(n1000):
    s, pb, pairs, *_ = n1000
    with make_ctx(s) as ctx:
        got = host(ctx.build_neighbors(dev(s.x), dev(s.quat)))
    assert compare_pairs(got, pairs, s) == 0
    assert got.shape[0] > 4000


def test_assemble_n1000(n1000):
    s, pb, pairs, asm, *_ = n1000
    with make_ctx(s) as ctx:
        phi, dg, q = ctx.assemble_constraints(dev(s.x), dev(s.quat), dev(s.f_nc), dev(pairs, torch.int32))
        phi, dg, q = host(phi), host(dg), host(q)
    np.testing.assert_allclose(phi, asm["phi"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(dg, asm["dgeom"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(q, asm["q"], rtol=1e-12, atol=1e-9)


def _active_full_rank(s, pb, pairs, dgeom, gam):
    act = gam > 0
    if act.sum() == 0 or act.sum() > 2500:
        return False
    sub = pairs[act]
    A_ = O.dense_A(s.quat, pb, sub, dgeom[act])
    return np.linalg.matrix_rank(A_, tol=1e-10 * np.abs(A_).max()) == act.sum()


@pytest.mark.parametrize("precision,tol,bar", [(A.FP64, 1e-8, 1e-5), (A.MIXED, 1e-6, 1e-3)])
def test_solve_n1000(n1000, precision, tol, bar):
    s, pb, pairs, asm, gam_o, (xo, qo, Uo) = n1000
    with make_ctx(s, precision, tol) as ctx:
        g, info = ctx.solve_lcp(dev(s.quat), dev(pairs, torch.int32), dev(asm["dgeom"]), dev(asm["q"]))
        g = host(g)
    assert info.status == 0 and info.residual <= tol and info.iters > 0
    assert (g >= 0).all()
    # the oracle's own residual of the GPU answer
    _, r = O.gradient(s.quat, pb, pairs, asm["dgeom"], asm["q"], g)
    assert r <= tol * 1.05 + (1e-9 if precision == A.FP64 else 2e-7)
    Ug = O.mobility_apply(s.quat, pb, O.apply_D(s.n, pairs, asm["dgeom"], g))
    Uo_c = O.mobility_apply(s.quat, pb, O.apply_D(s.n, pairs, asm["dgeom"], gam_o))
    assert rel_l2(Ug, Uo_c) <= bar
    if _active_full_rank(s, pb, pairs, asm["dgeom"], gam_o):
        assert rel_l2(g, gam_o) <= bar


@pytest.mark.parametrize("precision,tol,bar", [(A.FP64, 1e-8, 1e-5), (A.MIXED, 1e-6, 1e-3)])
@pytest.mark.parametrize("barriers", [1, 2])
def test_solve_n1000_both_schedules(n1000, precision, tol, bar, barriers):
    """The one-barrier solver (ghost copies of cross-block constraints, step
    length one iteration late) and the two-barrier solver both reach the
    oracle's optimum; aLENS_info names the kernel that ran."""
    s, pb, pairs, asm, gam_o, (xo, qo, Uo) = n1000
    with make_ctx(s, precision, tol) as ctx:
        ctx.set_solver_schedule(barriers)
        g, info = ctx.solve_lcp(dev(s.quat), dev(pairs, torch.int32), dev(asm["dgeom"]), dev(asm["q"]))
        g = host(g)
        with pytest.raises(A.AlensError):
            ctx.set_solver_schedule(3)
    assert info.solver == barriers   # 1: one barrier, 2: two barriers, shares in shared memory
    assert info.status == 0 and info.residual <= tol and info.iters > 0
    assert (g >= 0).all()
    _, r = O.gradient(s.quat, pb, pairs, asm["dgeom"], asm["q"], g)
    assert r <= tol * 1.05 + (1e-9 if precision == A.FP64 else 2e-7)
    # the reported residual is that of the returned gamma: to rounding in
    # float64; in mixed mode to the float32 reference passes' accuracy (the
    # rod forces are rounded to float32 before q + D^T U cancels to a
    # gradient a million times smaller: a few per cent at tol 1e-6)
    assert r == pytest.approx(info.residual, rel=1e-6 if precision == A.FP64 else 0.1)
    Ug = O.mobility_apply(s.quat, pb, O.apply_D(s.n, pairs, asm["dgeom"], g))
    Uo_c = O.mobility_apply(s.quat, pb, O.apply_D(s.n, pairs, asm["dgeom"], gam_o))
    assert rel_l2(Ug, Uo_c) <= bar


@pytest.mark.parametrize("max_iter", [1, 2, 5])
def test_iteration_cap_is_exact(n1000, max_iter):
    """A solve stopped by max_iter reports exactly max_iter iterations and the
    residual of the gamma it returns (one-barrier and two-barrier)."""
    s, pb, pairs, asm, *_ = n1000
    for barriers in (1, 2):
        with make_ctx(s, A.FP64, 1e-8, max_iter=max_iter) as ctx:
            ctx.set_solver_schedule(barriers)
            g, info = ctx.solve_lcp(dev(s.quat), dev(pairs, torch.int32), dev(asm["dgeom"]), dev(asm["q"]),
                                    check=False)
            g = host(g)
        assert info.status == 3 and info.iters == max_iter, (barriers, info.iters)
        _, r = O.gradient(s.quat, pb, pairs, asm["dgeom"], asm["q"], g)
        assert r == pytest.approx(info.residual, rel=1e-6), barriers


@pytest.mark.parametrize("precision,tol,xbar", [(A.FP64, 1e-8, 1e-6), (A.MIXED, 1e-6, 1e-5)])
def test_step_n1000(n1000, precision, tol, xbar):
    s, pb, pairs, asm, gam_o, (xo, qo, Uo) = n1000
    x, q = dev(s.x), dev(s.quat)
    vel = torch.empty((s.n, 6), dtype=torch.float64, device="cuda")
    with make_ctx(s, precision, tol) as ctx:
        gam = torch.empty(ctx.max_pairs, dtype=torch.float64, device="cuda")
        pr = torch.empty((ctx.max_pairs, 3), dtype=torch.int32, device="cuda")
        info = ctx.step(x, q, dev(s.f_nc), pairs_out=pr, gamma_out=gam, vel_out=vel)
        m = info.n_pairs
        got_pairs = host(pr)[:m]
    assert info.status == 0 and info.residual <= tol
    assert m == pairs.shape[0] and np.array_equal(got_pairs, pairs)
    assert info.n_overlap == int((asm["phi"] < 0).sum())
    assert info.min_gap == pytest.approx(asm["phi"].min(), abs=1e-12)
    dx = periodic_diff(host(x), xo, s.box)
    assert np.abs(dx).max() <= xbar * s.diameter
    np.testing.assert_allclose(host(q), qo, atol=xbar)
    np.testing.assert_allclose(np.linalg.norm(host(q), axis=1), 1.0, atol=1e-14)
    assert rel_l2(host(vel), Uo) <= (1e-6 if precision == A.FP64 else 1e-3)


def test_step_is_deterministic(n1000):
    s = n1000[0]
    outs = []
    for _ in range(2):
        x, q = dev(s.x), dev(s.quat)
        with make_ctx(s, A.MIXED, 1e-6) as ctx:
            gam = torch.empty(ctx.max_pairs, dtype=torch.float64, device="cuda")
            info = ctx.step(x, q, dev(s.f_nc), gamma_out=gam)
            outs.append((host(x), host(q), host(gam)[:info.n_pairs], info.iters))
    assert outs[0][3] == outs[1][3]
    for a, b in zip(outs[0][:3], outs[1][:3]):
        assert np.array_equal(a, b)


# ---------------------------------------------------------------- tiny systems

TINY = [(seed, n, box, L) for seed, (n, box, L) in enumerate(
    [(12, 14.0, 3.0), (30, 14.0, 3.0), (40, 11.0, 3.0), (25, 6.0, 3.0), (20, 5.5, 3.0), (60, 16.0, 4.0),
     (33, 9.0, 2.0), (50, 14.0, 3.0), (8, 7.0, 3.0), (45, 12.0, 5.0)])]


@pytest.mark.parametrize("seed,n,box,L", TINY)
@pytest.mark.parametrize("precision", [A.FP64, A.MIXED])
def test_step_tiny(seed, n, box, L, precision):
    s = W.tiny_system(100 + seed, n, box=box, length=L, nematic_spread=0.05 if seed % 3 == 0 else None)
    s.f_nc *= 30.0
    pb = O.problem_of(s)
    ref = O.step(s.x, s.quat, s.f_nc, pb, tol=1e-12)
    tol = 1e-10 if precision == A.FP64 else 1e-6
    x, q = dev(s.x), dev(s.quat)
    with make_ctx(s, precision, tol) as ctx:
        pr = torch.empty((ctx.max_pairs, 3), dtype=torch.int32, device="cuda")
        info = ctx.step(x, q, dev(s.f_nc), pairs_out=pr)
        m = info.n_pairs
        got = host(pr)[:m]
    assert compare_pairs(got, ref["pairs"], s) == 0
    assert info.status == 0
    xbar = 1e-6 if precision == A.FP64 else 2e-5
    assert np.abs(periodic_diff(host(x), ref["x"], s.box)).max() <= xbar
    assert np.abs(host(q) - ref["quat"]).max() <= xbar


def test_adversarial_geometry():
    # parallel, anti-parallel, crossed, collinear and skew pairs placed at
    # gaps just inside / outside delta_c and overlapping; small box so that
    # periodic images matter
    rng = np.random.default_rng(17)
    ez = np.array([0, 0, 1.0])
    xs, axes = [], []
    def add(c, a):
        xs.append(c); axes.append(a / np.linalg.norm(a))
    base = np.array([3.0, 3.0, 3.0])
    for k, gap in enumerate([0.5, 0.999999, 1.000001, -0.3, 0.0, 1e-9]):
        o = base + np.array([k * 4.0, 0, 0])
        add(o, ez); add(o + np.array([1.0 + gap, 0, 0.3]), ez)                    # parallel side by side
        add(o + np.array([0, 6.0, 0]), ez); add(o + np.array([0, 6.0, 11.0 + gap]), -ez)   # collinear head-on
        add(o + np.array([0, 12.0, 0]), np.array([1.0, 0, 0]))                    # collinear chain along x
        add(o + np.array([0.25, 12.0, 1.0 + gap]), np.array([0, 1.0, 0]))          # crossed
    for _ in range(6):  # near-parallel skew pairs
        o = rng.uniform(0, 30, 3)
        a = ez + 1e-7 * rng.standard_normal(3)
        add(o, ez); add(o + np.array([1.5, 0, 2.0]), a)
    x = np.array(xs); axis = np.array(axes)
    box = (30.0, 30.0, 30.0)
    s = W.RodSystem(x=x - 30.0 * np.floor(x / 30.0), quat=W.quat_from_axis(axis),
                    f_nc=rng.standard_normal((x.shape[0], 6)) * 10, box=box, tol=1e-10)
    pb = O.problem_of(s)
    ref = O.find_pairs(s.x, s.quat, pb)
    with make_ctx(s) as ctx:
        got = host(ctx.build_neighbors(dev(s.x), dev(s.quat)))
        phi, dg, q = ctx.assemble_constraints(dev(s.x), dev(s.quat), dev(s.f_nc), dev(ref, torch.int32))
    assert compare_pairs(got, ref, s) == 0
    a = O.assemble(s.x, s.quat, s.f_nc, pb, ref)
    np.testing.assert_allclose(host(phi), a["phi"], atol=1e-12)
    np.testing.assert_allclose(host(dg), a["dgeom"], atol=1e-6)


def _rotation(rng):
    qv = rng.standard_normal(4)
    w, x, y, z = qv / np.linalg.norm(qv)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_float32_screen_boundary():
    """The neighbour search drops a candidate on a float32 closest-point
    distance only when 1 - (p.q)^2 exceeds 1e-4 and the distance clears
    D + delta_c by a margin (0.02 D + 2e-6 box); nearer-parallel pairs go to
    the float64 decision.  Pairs placed just on the float32 side of that
    cut (1 - (p.q)^2 from 1.0005e-4 to 1e-3) with float64 gaps within the
    margin of delta_c, in interior, end-to-side and end-to-end closest-point
    configurations, rotated at random and placed at coordinates up to the
    box edge (200 D): the list must equal the oracle's exactly (Appendix
    "Implementation": a pair is a constraint iff its gap is below delta_c)."""
    rng = np.random.default_rng(29)
    L, D, dc = 10.0, 1.0, 1.0
    box = 200.0
    xs, axes, want_gap = [], [], []
    for det in (1.0005e-4, 1.001e-4, 1.01e-4, 1.1e-4, 2e-4, 1e-3):
        th = math.asin(math.sqrt(det))
        for eps in (-1e-3, -1e-5, -1e-7, 1e-7, 1e-5, 1e-3, 1.5e-2):
            for kind in range(3):
                R = _rotation(rng)
                p = np.array([0.0, 0.0, 1.0])
                q = np.array([math.sin(th), 0.0, math.cos(th)])
                h = D + dc + eps
                # P along p through the origin; the closest point of Q lies
                # at distance h from P in every configuration
                if kind == 0:     # interior closest points, separation along y
                    cq = np.array([0.0, h, 0.0])
                elif kind == 1:   # Q's lower end against the middle of P's side
                    cq = np.array([0.0, h, 0.0]) + 0.5 * L * q
                else:             # Q's lower end against P's upper end
                    cq = np.array([0.0, h, 0.5 * L]) + 0.5 * L * q
                o = rng.uniform(0.0, box, 3)
                if rng.uniform() < 0.5:   # near the far corner, where float32 rounding is largest
                    o = box - rng.uniform(0.0, 12.0, 3)
                xs += [o, o + R @ cq]
                axes += [R @ p, R @ q]
    x = np.array(xs)
    s = W.RodSystem(x=x - box * np.floor(x / box), quat=W.quat_from_axis(np.array(axes)),
                    f_nc=np.zeros((x.shape[0], 6)), box=(box, box, box), tol=1e-10)
    pb = O.problem_of(s)
    ref = O.find_pairs(s.x, s.quat, pb)
    # the constructed pairs do probe the cut: many of them sit within the
    # screen margin of delta_c with 1 - (p.q)^2 above 1e-4 in float64
    built = np.arange(0, x.shape[0], 2)
    ax = O.axis(s.quat)
    dets = 1.0 - np.einsum("ij,ij->i", ax[built], ax[built + 1]) ** 2
    assert (dets > 1e-4).all()
    with make_ctx(s) as ctx:
        got = host(ctx.build_neighbors(dev(s.x), dev(s.quat)))
    assert compare_pairs(got, ref, s) == 0
    # both sides of delta_c are represented among the constructed pairs
    cand = np.stack([built, built + 1, np.full(built.shape, 13)], 1).astype(np.int32)
    dx = s.x[built] - s.x[built + 1]
    shift = np.round(dx / box).astype(int)   # minimum image: x_i - x_j - k box
    cand[:, 2] = (shift[:, 0] + 1) + 3 * (shift[:, 1] + 1) + 9 * (shift[:, 2] + 1)
    gaps = O.pair_gaps(s.x, s.quat, pb, cand)
    near = np.abs(gaps - dc) < 0.02 + 2e-6 * box
    assert (near & (gaps < dc)).sum() >= 20 and (near & (gaps >= dc)).sum() >= 20


def test_float32_keep_band():
    """The neighbour search also keeps a candidate on its float32
    closest-point distance alone when that distance is below D + delta_c by
    the keep margin 2 sqrt(3) (4 u B + L u + 200 u) + 1e-5 D (u = 2^-24, B
    the power of two above the box; 2.7e-4 D at box 200): the float closest
    points are points of the two segments, so their exact distance bounds
    the minimum from above, and the float evaluation errs by at most half
    the margin.  Pairs at general angles with float64 gaps on both sides of
    delta_c - margin and of delta_c, in interior, end-to-side and end-to-end
    closest-point configurations, rotated at random and placed at
    coordinates in the box edge's binade, where float32 rounding is largest:
    the list must equal the oracle's exactly (Appendix "Implementation": a
    pair is a constraint iff its gap is below delta_c)."""
    rng = np.random.default_rng(31)
    L, D, dc = 10.0, 1.0, 1.0
    box = 200.0
    u, B = 2.0 ** -24, 256.0
    kmargin = 2.0 * math.sqrt(3.0) * (4.0 * u * B + L * u + 200.0 * u) + 1e-5 * D
    xs, axes = [], []
    for ang in (0.05, 0.3, 0.9, 1.5707):
        for eps in (-2 * kmargin, -1.2 * kmargin, -kmargin - 1e-6, -kmargin + 1e-6, -0.8 * kmargin, -0.5 * kmargin,
                    -1e-5, -1e-7, 1e-7, 1e-5, 0.5 * kmargin, 2 * kmargin):
            for kind in range(3):
                R = _rotation(rng)
                p = np.array([0.0, 0.0, 1.0])
                q = np.array([math.sin(ang), 0.0, math.cos(ang)])
                h = D + dc + eps
                if kind == 0:     # interior closest points, separation along y
                    cq = np.array([0.0, h, 0.0])
                elif kind == 1:   # Q's lower end against the middle of P's side
                    cq = np.array([0.0, h, 0.0]) + 0.5 * L * q
                else:             # Q's lower end against P's upper end
                    cq = np.array([0.0, h, 0.5 * L]) + 0.5 * L * q
                # coordinates in [130, 200): the binade of the box edge, where
                # float32 rounding is largest
                o = box - rng.uniform(0.0, 70.0, 3)
                xs += [o, o + R @ cq]
                axes += [R @ p, R @ q]
    x = np.array(xs)
    s = W.RodSystem(x=x - box * np.floor(x / box), quat=W.quat_from_axis(np.array(axes)),
                    f_nc=np.zeros((x.shape[0], 6)), box=(box, box, box), tol=1e-10)
    pb = O.problem_of(s)
    ref = O.find_pairs(s.x, s.quat, pb)
    with make_ctx(s, max_pairs=100_000) as ctx:
        got = host(ctx.build_neighbors(dev(s.x), dev(s.quat)))
    assert compare_pairs(got, ref, s) == 0
    # the constructed pairs straddle the keep threshold and delta_c
    built = np.arange(0, x.shape[0], 2)
    cand = np.stack([built, built + 1, np.full(built.shape, 13)], 1).astype(np.int32)
    shift = np.round((s.x[built] - s.x[built + 1]) / box).astype(int)
    cand[:, 2] = (shift[:, 0] + 1) + 3 * (shift[:, 1] + 1) + 9 * (shift[:, 2] + 1)
    gaps = O.pair_gaps(s.x, s.quat, pb, cand)
    assert (gaps < dc - kmargin).sum() >= 20 and ((gaps > dc - kmargin) & (gaps < dc)).sum() >= 20
    assert (gaps >= dc).sum() >= 20


# ------------------------------------------------------------------ edge cases

def test_empty_and_isolated_rods():
    s = W.tiny_system(3, 5, box=200.0, length=3.0)
    pb = O.problem_of(s)
    ref = O.step(s.x, s.quat, s.f_nc, pb)
    assert ref["pairs"].shape[0] == 0
    x, q = dev(s.x), dev(s.quat)
    with make_ctx(s) as ctx:
        info = ctx.step(x, q, dev(s.f_nc))
        assert info.n_pairs == 0 and info.status == 0 and info.iters == 0
        assert np.abs(periodic_diff(host(x), ref["x"], s.box)).max() <= 1e-12
        e = torch.empty((0, 3), dtype=torch.float64, device="cuda")
        e4 = torch.empty((0, 4), dtype=torch.float64, device="cuda")
        e6 = torch.empty((0, 6), dtype=torch.float64, device="cuda")
        info = ctx.step(e, e4, e6)
        assert info.n_pairs == 0 and info.status == 0


def test_capacity_reports_required_count(n1000):
    s, pb, pairs, *_ = n1000
    with make_ctx(s, max_pairs=100) as ctx:
        with pytest.raises(A.AlensError) as ei:
            ctx.build_neighbors(dev(s.x), dev(s.quat))
        assert ei.value.status == 2 and ei.value.extra == pairs.shape[0]
        with pytest.raises(A.AlensError) as ei:
            ctx.step(dev(s.x), dev(s.quat), dev(s.f_nc))
        assert ei.value.status == 2 and ei.value.extra["n_pairs"] == pairs.shape[0]


def test_invalid_inputs_leave_state_untouched(n1000):
    s, pb, pairs, asm, *_ = n1000
    bad = s.quat.copy()
    bad[7] *= 1.01
    x, q = dev(s.x), dev(bad)
    with make_ctx(s) as ctx:
        with pytest.raises(A.AlensError) as ei:
            ctx.step(x, q, dev(s.f_nc))
        assert ei.value.status == 1
        assert np.array_equal(host(x), s.x) and np.array_equal(host(q), bad)
        xn = s.x.copy(); xn[3, 1] = np.nan
        with pytest.raises(A.AlensError):
            ctx.build_neighbors(dev(xn), dev(s.quat))
        shuffled = pairs[::-1].copy()
        with pytest.raises(A.AlensError) as ei:
            ctx.solve_lcp(dev(s.quat), dev(shuffled, torch.int32), dev(asm["dgeom"][::-1]), dev(asm["q"][::-1]))
        assert ei.value.status == 1
        # the context still works afterwards
        got = host(ctx.build_neighbors(dev(s.x), dev(s.quat)))
        assert np.array_equal(got, pairs)


def test_not_converged_reports_residual(n1000):
    s, pb, pairs, asm, *_ = n1000
    with make_ctx(s, A.FP64, 1e-8, max_iter=3) as ctx:
        g, info = ctx.solve_lcp(dev(s.quat), dev(pairs, torch.int32), dev(asm["dgeom"]), dev(asm["q"]), check=False)
        assert info.status == 3 and info.iters == 3 and info.residual > 1e-8
        _, r = O.gradient(s.quat, pb, pairs, asm["dgeom"], asm["q"], host(g))
        assert r == pytest.approx(info.residual, rel=1e-6)


def test_bounded_wait_times_out_and_context_recovers(n1000):
    # one block of the solver leaves before its first grid-wide arrival; the
    # others' bounded waits run out, the call returns TIMEOUT, nothing hangs
    s, pb, pairs, asm, *_ = n1000
    with make_ctx(s, A.FP64, 1e-8) as ctx:
        ctx.set_wait_limit(0.2)
        ctx.inject_fault(1)
        g, info = ctx.solve_lcp(dev(s.quat), dev(pairs, torch.int32), dev(asm["dgeom"]), dev(asm["q"]), check=False)
        assert info.status == 4
        ctx.set_wait_limit(5.0)
        g, info = ctx.solve_lcp(dev(s.quat), dev(pairs, torch.int32), dev(asm["dgeom"]), dev(asm["q"]))
        assert info.status == 0 and info.residual <= 1e-8


def test_warm_start_converges_immediately(n1000):
    s, pb, pairs, asm, gam_o, _ = n1000
    with make_ctx(s, A.FP64, 1e-8) as ctx:
        g, info = ctx.solve_lcp(dev(s.quat), dev(pairs, torch.int32), dev(asm["dgeom"]), dev(asm["q"]),
                                gamma=dev(gam_o))
    assert info.status == 0 and info.iters == 0


# ------------------------------------------------------ full-size (1e5 rods)

@pytest.fixture(scope="module")
def n100k():
    return W.workload("n100k_phi010")


@pytest.mark.parametrize("precision,tol", [(A.FP64, 1e-6), (A.MIXED, 1e-5)])
def test_n100k_step_properties(n100k, precision, tol):
    s = n100k
    pb = O.problem_of(s)
    x, q = dev(s.x), dev(s.quat)
    with make_ctx(s, precision, tol, max_pairs=1_000_000) as ctx:
        gam = torch.empty(ctx.max_pairs, dtype=torch.float64, device="cuda")
        pr = torch.empty((ctx.max_pairs, 3), dtype=torch.int32, device="cuda")
        vel = torch.empty((s.n, 6), dtype=torch.float64, device="cuda")
        info = ctx.step(x, q, dev(s.f_nc), pairs_out=pr, gamma_out=gam, vel_out=vel)
        m = info.n_pairs
        pairs, g = host(pr)[:m], host(gam)[:m]
    assert info.status == 0 and info.residual <= tol and 2e5 < m < 6e5
    # pair list: every pair touching 150 sampled rods, against the oracle
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(s.n, 150, replace=False))
    ref = O.find_pairs(s.x, s.quat, pb, rows=rows)
    sel = pairs[np.isin(pairs[:, 0], rows) | np.isin(pairs[:, 1], rows)]
    assert compare_pairs(sel, ref, s) == 0
    # KKT of the GPU answer, evaluated by the oracle on its own assembly
    asm = O.assemble(s.x, s.quat, s.f_nc, pb, pairs)
    assert (g >= 0).all()
    gr, r = O.gradient(s.quat, pb, pairs, asm["dgeom"], asm["q"], g)
    assert r <= tol * 1.05 + (1e-9 if precision == A.FP64 else 1e-6)
    # U = M (F_nc + D gamma) from the oracle's arithmetic on the GPU gamma
    U = O.mobility_apply(s.quat, pb, s.f_nc + O.apply_D(s.n, pairs, asm["dgeom"], g))
    assert rel_l2(host(vel), U) <= (1e-9 if precision == A.FP64 else 1e-4)
    xo = O.wrap(O.wrap(s.x, s.box) + s.dt * U[:, :3], s.box)
    assert np.abs(periodic_diff(host(x), xo, s.box)).max() <= (1e-9 if precision == A.FP64 else 1e-5)


def test_n100k_mixed_in_every_launch_shape(n100k):
    # the autotuner picks the solver's launch shape among these for the timed
    # steps; each must give a gamma that the oracle finds optimal, the same
    # pair list and a post-step state within the mixed-precision bars
    import paper_2109_08206_gb300.autotune as T
    s = n100k
    pb = O.problem_of(s)
    tol = 1e-5
    out = {}
    kinds = set()
    for shape in T.SINGLE_CANDIDATES:
        for barriers in (1, 2):
            x, q = dev(s.x), dev(s.quat)
            with make_ctx(s, A.MIXED, tol, max_pairs=1_000_000) as ctx:
                ctx.set_launch(*shape)
                ctx.set_solver_schedule(barriers)
                gam = torch.empty(ctx.max_pairs, dtype=torch.float64, device="cuda")
                pr = torch.empty((ctx.max_pairs, 3), dtype=torch.int32, device="cuda")
                vel = torch.empty((s.n, 6), dtype=torch.float64, device="cuda")
                info = ctx.step(x, q, dev(s.f_nc), pairs_out=pr, gamma_out=gam, vel_out=vel)
                m = info.n_pairs
                assert info.status == 0 and info.residual <= tol, shape
                assert barriers == 1 or info.solver in (2, 3)
                kinds.add(info.solver)
                out[shape + (barriers,)] = (host(pr)[:m], host(gam)[:m], host(vel), host(x), info.iters)
    # the default shape runs the one-barrier kernel at this size
    assert 1 in kinds and 2 in kinds
    pairs = out[T.SINGLE_CANDIDATES[0] + (1,)][0]
    asm = O.assemble(s.x, s.quat, s.f_nc, pb, pairs)
    for shape, (pr, g, vel, xg, iters) in out.items():
        assert np.array_equal(pr, pairs), shape
        assert (g >= 0).all()
        _, r = O.gradient(s.quat, pb, pairs, asm["dgeom"], asm["q"], g)
        assert r <= tol * 1.05 + 1e-6, (shape, r)
        U = O.mobility_apply(s.quat, pb, s.f_nc + O.apply_D(s.n, pairs, asm["dgeom"], g))
        assert rel_l2(vel, U) <= 1e-4, shape
        xo = O.wrap(O.wrap(s.x, s.box) + s.dt * U[:, :3], s.box)
        assert np.abs(periodic_diff(xg, xo, s.box)).max() <= 1e-5, shape


# -------------------------------------------- 4e5 rods, nematic, mixed precision

@pytest.fixture(scope="module")
def n400k():
    return W.workload("n400k_nematic")


def test_n400k_nematic_mixed_against_oracle_and_fp64(n400k):
    # the dense nematic pack: FP32-mixed iterations at tol 1e-5; errors
    # reported against the float64 oracle (KKT of the GPU answer) and the
    # float64 GPU step
    s = n400k
    pb = O.problem_of(s)
    mp = 12 * s.n
    res = {}
    for prec in (A.MIXED, A.FP64):
        x, q = dev(s.x), dev(s.quat)
        with make_ctx(s, prec, 1e-5, max_pairs=mp) as ctx:
            gam = torch.empty(mp, dtype=torch.float64, device="cuda")
            pr = torch.empty((mp, 3), dtype=torch.int32, device="cuda")
            info = ctx.step(x, q, dev(s.f_nc), pairs_out=pr, gamma_out=gam)
            m = info.n_pairs
            res[prec] = (info, host(x), host(q), host(pr)[:m], host(gam)[:m])
    info, x32, q32, pairs, g32 = res[A.MIXED]
    assert info.status == 0 and info.residual <= 1e-5 and 1e6 < info.n_pairs < 4e6
    assert np.array_equal(pairs, res[A.FP64][3])
    rng = np.random.default_rng(1)
    rows = np.sort(rng.choice(s.n, 40, replace=False))
    ref = O.find_pairs(s.x, s.quat, pb, rows=rows)
    assert compare_pairs(pairs[np.isin(pairs[:, 0], rows) | np.isin(pairs[:, 1], rows)], ref, s) == 0
    asm = O.assemble(s.x, s.quat, s.f_nc, pb, pairs)
    _, r = O.gradient(s.quat, pb, pairs, asm["dgeom"], asm["q"], g32)
    print(f"\nn400k mixed: {info.iters} iterations, GPU residual {info.residual:.3e}, "
          f"oracle residual of the mixed gamma {r:.3e}, "
          f"max |x_mixed - x_fp64| = {np.abs(periodic_diff(x32, res[A.FP64][1], s.box)).max():.3e} D")
    assert r <= 1.05e-5 + 1e-6
    assert np.abs(periodic_diff(x32, res[A.FP64][1], s.box)).max() <= 1e-4 * s.diameter
