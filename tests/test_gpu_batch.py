"""Batched step (aLENS_step_batch) through the C ABI, against the oracle run
system by system.

Each system of a batch is an independent periodic suspension with its own
box and rod length; the oracle steps every system alone.  Bars as for the
single-system step: pair lists bit-exact per system (global indices shifted
by the system's rod offset, no mismatch excused), post-step
centres and quaternions within 1e-6 D (float64) / 2e-5 D (mixed), U within
1e-6 / 1e-3 relative L2.  Small systems with one or two cells per edge make
several periodic images of one pair close (each is a separate constraint).
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


def small_batch():
    """Ten shrunken ensemble systems plus hand-made ones with anisotropic
    boxes of one to three cells per edge, varied lengths and an empty system."""
    systems = W.ensemble(seed=1000, count=10, scale=0.03)
    extra = [
        W.random_system(71, 60, (8.5, 13.0, 20.0), length=4.0, forces="unit", tol=1e-10, name="aniso_1_2_3"),
        W.random_system(72, 0, 9.0, length=5.0, forces="unit", tol=1e-10, name="empty"),
        W.random_system(73, 90, (12.0, 7.2, 12.0), length=5.0, forces="unit", nematic_spread=0.05, tol=1e-10,
                        name="nematic_2_1_2"),
        W.random_system(74, 2, 6.0, length=3.0, forces="unit", tol=1e-10, name="two_rods"),
    ]
    for s in extra:
        s.f_nc *= 30.0
    return systems[:4] + extra[:2] + systems[4:] + extra[2:]


def batch_ctx(systems, precision, tol, max_iter=400000):
    s0 = systems[0]
    p = A.make_params(s0.box, s0.diameter, s0.length, s0.viscosity, s0.dt, s0.delta_c, tol, max_iter, precision)
    n = sum(s.n for s in systems)
    return A.Context(p, max(n, 1), max(64, 12 * n))


def run_batch(systems, precision, tol, shape=None):
    off, x, quat, fnc, spec = W.batch_arrays(systems)
    xd, qd = dev(x), dev(quat)
    n = int(off[-1])
    vel = torch.empty((max(n, 1), 6), dtype=torch.float64, device="cuda")
    with batch_ctx(systems, precision, tol) as ctx:
        if shape is not None:
            ctx.set_batch_launch(*shape)
        pr = torch.empty((ctx.max_pairs, 3), dtype=torch.int32, device="cuda")
        gam = torch.empty(ctx.max_pairs, dtype=torch.float64, device="cuda")
        info = ctx.step_batch(spec, off, xd, qd, dev(fnc), pairs_out=pr, gamma_out=gam, vel_out=vel[:n])
        m = info.n_pairs
        its, res = ctx.batch_results(len(systems))
        # the aggregate is the worst system
        assert info.iters == its.max() and info.residual == res.max()
        assert np.all(res <= tol)
        return off, host(xd), host(qd), host(pr)[:m], host(gam)[:m], host(vel)[:n], info


def split_pairs(pairs, off):
    """Per-system pair lists in local indices; asserts no pair joins two systems."""
    sys_i = np.searchsorted(off, pairs[:, 0], side="right") - 1
    sys_j = np.searchsorted(off, pairs[:, 1], side="right") - 1
    assert np.array_equal(sys_i, sys_j), "a pair joins two systems"
    out = []
    for s in range(len(off) - 1):
        sel = pairs[sys_i == s].copy()
        sel[:, :2] -= off[s]
        out.append(sel)
    return out


@pytest.mark.parametrize("precision,tol,xbar,ubar", [(A.FP64, 1e-10, 1e-6, 1e-6), (A.MIXED, 1e-6, 2e-5, 1e-3)])
def test_batch_matches_oracle_per_system(precision, tol, xbar, ubar):
    systems = small_batch()
    off, x, q, pairs, gam, vel, info = run_batch(systems, precision, tol)
    assert info.status == 0 and info.residual <= tol
    per = split_pairs(pairs, off)
    total_overlap = 0
    for k, s in enumerate(systems):
        lo, hi = off[k], off[k + 1]
        if s.n == 0:
            assert per[k].shape[0] == 0
            continue
        pb = O.problem_of(s)
        ref = O.step(s.x, s.quat, s.f_nc, pb, tol=1e-12)
        compare_pairs(per[k], ref["pairs"], s)
        total_overlap += int((ref["phi"] < 0).sum())
        assert np.abs(periodic_diff(x[lo:hi], ref["x"], s.box)).max() <= xbar * s.diameter, s.name
        assert np.abs(q[lo:hi] - ref["quat"]).max() <= xbar, s.name
        U = vel[lo:hi]
        assert np.linalg.norm(U - ref["U"]) <= ubar * np.linalg.norm(ref["U"]) + 1e-12, s.name
        # the oracle's residual of the batch's gamma restricted to this system
        if per[k].shape[0] > 0:
            sel = (pairs[:, 0] >= lo) & (pairs[:, 0] < hi)
            asm = O.assemble(s.x, s.quat, s.f_nc, pb, per[k])
            _, r = O.gradient(s.quat, pb, per[k], asm["dgeom"], asm["q"], gam[sel])
            assert r <= tol * 1.05 + (1e-9 if precision == A.FP64 else 2e-7), s.name
    assert info.n_overlap == total_overlap
    assert sum(p.shape[0] for p in per) == info.n_pairs > 0


def test_prepared_tables_equal_lists():
    """A BatchSpec built once gives the same step as the systems and offsets
    passed as lists, bit for bit."""
    systems = small_batch()
    off, x, quat, fnc, spec = W.batch_arrays(systems)
    prepared = A.BatchSpec(spec, off)
    outs = []
    with batch_ctx(systems, A.MIXED, 1e-6) as ctx:
        for tables, offsets in ((spec, off), (prepared, None), (prepared, None)):
            xd, qd = dev(x), dev(quat)
            info = ctx.step_batch(tables, offsets, xd, qd, dev(fnc))
            assert info.status == 0
            outs.append((host(xd), host(qd), info.iters, info.n_pairs))
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1]) and o[2:] == outs[0][2:]
    with pytest.raises(ValueError):
        A.BatchSpec(spec, off[:-1])


def uneven_batch():
    """Three systems of the ensemble's kind (nematic domains, thermal forces):
    two of 2,000 and 1,500 rods and one of 300."""
    out = []
    for seed, n in ((81, 2000), (82, 1500), (83, 300)):
        box = W.box_for_fraction(n, 1.0, 10.0, 0.1)
        out.append(W.random_system(seed, n, box, length=10.0, nematic_spread=0.3, forces="thermal", tol=1e-8,
                                   name=f"uneven_{n}"))
    return out


@pytest.mark.parametrize("precision,tol,xbar,ubar", [(A.FP64, 1e-10, 1e-6, 1e-6), (A.MIXED, 1e-6, 2e-5, 1e-3)])
def test_paired_systems_match_oracle(precision, tol, xbar, ubar):
    """One-block clusters: the two larger systems hold more than 4096
    constraints each and far more than half of a cluster's mean share, so
    two clusters solve each of them together (aLENS_batch_groups: 2 blocks),
    and the smallest is solved by one.  Every system matches the oracle as
    in the other batches, and a second step from the same state repeats the
    first bit for bit (the pairing depends only on the systems and the
    launch)."""
    systems = uneven_batch()
    off, x, quat, fnc, spec = W.batch_arrays(systems)
    n = int(off[-1])
    outs = []
    with batch_ctx(systems, precision, tol) as ctx:
        ctx.set_batch_launch(1024, 1)
        pr = torch.empty((ctx.max_pairs, 3), dtype=torch.int32, device="cuda")
        gam = torch.empty(ctx.max_pairs, dtype=torch.float64, device="cuda")
        vel = torch.empty((n, 6), dtype=torch.float64, device="cuda")
        for rep in range(2):
            xd, qd = dev(x), dev(quat)
            info = ctx.step_batch(spec, off, xd, qd, dev(fnc), pairs_out=pr, gamma_out=gam, vel_out=vel)
            assert info.status == 0 and info.residual <= tol
            m = info.n_pairs
            outs.append((host(xd), host(qd), host(pr)[:m], host(gam)[:m], host(vel)))
            groups = ctx.batch_groups(len(systems))
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
    xg, qg, pairs, gamg, velg = outs[0]
    per = split_pairs(pairs, off)
    ms = [p.shape[0] for p in per]
    assert ms[0] >= 4096 and ms[1] >= 4096 and ms[2] < 4096, ms
    assert list(groups) == [2, 2, 1], (list(groups), ms)
    for k, s in enumerate(systems):
        lo, hi = off[k], off[k + 1]
        pb = O.problem_of(s)
        ref = O.step(s.x, s.quat, s.f_nc, pb, tol=1e-12)
        compare_pairs(per[k], ref["pairs"], s)
        assert np.abs(periodic_diff(xg[lo:hi], ref["x"], s.box)).max() <= xbar * s.diameter, s.name
        assert np.abs(qg[lo:hi] - ref["quat"]).max() <= xbar, s.name
        assert np.linalg.norm(velg[lo:hi] - ref["U"]) <= ubar * np.linalg.norm(ref["U"]), s.name
        sel = (pairs[:, 0] >= lo) & (pairs[:, 0] < hi)
        asm = O.assemble(s.x, s.quat, s.f_nc, pb, per[k])
        _, r = O.gradient(s.quat, pb, per[k], asm["dgeom"], asm["q"], gamg[sel])
        assert r <= tol * 1.05 + (1e-9 if precision == A.FP64 else 2e-7), s.name


def test_pairs_off_without_cooperative_cluster_launch():
    """The test hook that makes the context run as on a device refusing a
    cooperative launch with clusters: the same uneven batch is solved with
    one cluster per system (aLENS_batch_groups: 1 block each), still to the
    oracle's answer."""
    systems = uneven_batch()
    off, x, quat, fnc, spec = W.batch_arrays(systems)
    n = int(off[-1])
    tol = 1e-6
    with batch_ctx(systems, A.MIXED, tol) as ctx:
        ctx.set_batch_launch(1024, 1)
        ctx.inject_fault(3)
        vel = torch.empty((n, 6), dtype=torch.float64, device="cuda")
        xd, qd = dev(x), dev(quat)
        info = ctx.step_batch(spec, off, xd, qd, dev(fnc), vel_out=vel)
        assert info.status == 0 and info.residual <= tol
        assert list(ctx.batch_groups(len(systems))) == [1, 1, 1]
        xg, velg = host(xd), host(vel)
    for k, s in enumerate(systems):
        lo, hi = off[k], off[k + 1]
        ref = O.step(s.x, s.quat, s.f_nc, O.problem_of(s), tol=1e-12)
        assert np.abs(periodic_diff(xg[lo:hi], ref["x"], s.box)).max() <= 2e-5 * s.diameter, s.name
        assert np.linalg.norm(velg[lo:hi] - ref["U"]) <= 1e-3 * np.linalg.norm(ref["U"]), s.name


def test_pair_wait_times_out_and_context_recovers():
    """The test hook that makes the second cluster of every pair skip its
    system: the first cluster's bounded waits run out (wait limit 0.2 s), the
    call returns TIMEOUT and moves no rod, and the next call on the same
    context pairs and solves as before."""
    systems = uneven_batch()
    off, x, quat, fnc, spec = W.batch_arrays(systems)
    with batch_ctx(systems, A.MIXED, 1e-6) as ctx:
        ctx.set_batch_launch(1024, 1)
        ctx.set_wait_limit(0.2)
        ctx.inject_fault(1)
        xd, qd = dev(x), dev(quat)
        with pytest.raises(A.AlensError) as e:
            ctx.step_batch(spec, off, xd, qd, dev(fnc))
        assert e.value.status == 4
        assert np.array_equal(host(xd), x) and np.array_equal(host(qd), quat)
        info = ctx.step_batch(spec, off, xd, qd, dev(fnc))
        assert info.status == 0
        assert list(ctx.batch_groups(len(systems))) == [2, 2, 1]


@pytest.mark.parametrize("precision", [A.FP64, A.MIXED])
def test_batch_of_one_equals_single_step(precision):
    # one system through the batch tables (per-system geometry, per-rod drags;
    # a batch of one uses the single-system solver) must reproduce the
    # single-system step bit for bit
    s = W.tiny_system(5, 60, box=11.0, length=3.0)
    s.f_nc *= 30.0
    tol = 1e-10 if precision == A.FP64 else 1e-6
    outs = []
    for batched in (False, True):
        x, q = dev(s.x), dev(s.quat)
        with batch_ctx([s], precision, tol) as ctx:
            gam = torch.empty(ctx.max_pairs, dtype=torch.float64, device="cuda")
            vel = torch.empty((s.n, 6), dtype=torch.float64, device="cuda")
            if batched:
                info = ctx.step_batch([(s.box, s.length)], [0, s.n], x, q, dev(s.f_nc), gamma_out=gam, vel_out=vel)
            else:
                info = ctx.step(x, q, dev(s.f_nc), gamma_out=gam, vel_out=vel)
            outs.append((host(x), host(q), host(gam)[:info.n_pairs], host(vel), info.iters))
    assert outs[0][4] == outs[1][4]
    for a, b in zip(outs[0][:4], outs[1][:4]):
        assert np.array_equal(a, b)


def test_batch_tables_reused_and_replaced():
    systems = small_batch()[:5]
    off, x, quat, fnc, spec = W.batch_arrays(systems)
    with batch_ctx(systems, A.FP64, 1e-10) as ctx:
        launches = []
        for _ in range(2):
            xd, qd = dev(x), dev(quat)
            info = ctx.step_batch(spec, off, xd, qd, dev(fnc))
            launches.append(info.launches)
        # the second call with the same systems does not rebuild the rod -> system table
        assert launches[1] == launches[0] - 1
        # a different length for one system takes effect (checked against the oracle)
        s = systems[1]
        s2 = W.random_system(99, s.n, s.box, length=s.length * 0.5, forces="unit", tol=1e-10)
        spec2 = list(spec)
        spec2[1] = (s2.box, s2.length)
        x2, q2 = x.copy(), quat.copy()
        x2[off[1]:off[2]], q2[off[1]:off[2]] = s2.x, s2.quat
        f2 = fnc.copy()
        f2[off[1]:off[2]] = s2.f_nc
        xd, qd = dev(x2), dev(q2)
        info = ctx.step_batch(spec2, off, xd, qd, dev(f2))
        assert info.status == 0
        ref = O.step(s2.x, s2.quat, s2.f_nc, O.problem_of(s2), tol=1e-12)
        got = host(xd)[off[1]:off[2]]
        assert np.abs(periodic_diff(got, ref["x"], s2.box)).max() <= 1e-6


def test_batch_rejects_bad_tables():
    systems = small_batch()[:3]
    off, x, quat, fnc, spec = W.batch_arrays(systems)
    with batch_ctx(systems, A.FP64, 1e-10) as ctx:
        xd = dev(x)
        bad = [
            (spec, [1] + list(off[1:])),                          # first offset not 0
            (spec, [0, off[2], off[1], off[3]]),                  # decreasing
            (spec, list(off[:-1]) + [ctx.max_rods + 1]),          # beyond the context
            ([spec[0], ((3.0, 3.0, 3.0), 10.0), spec[2]], off),   # box smaller than L + D + delta_c
            ([spec[0], (spec[1][0], -1.0), spec[2]], off),        # negative length
        ]
        for sp, of in bad:
            with pytest.raises(A.AlensError) as e:
                ctx.step_batch(sp, of, xd, dev(quat), dev(fnc))
            assert e.value.status == 1
        assert np.array_equal(host(xd), x)   # nothing written
        # the context still works after the refusals
        info = ctx.step_batch(spec, off, xd, dev(quat), dev(fnc))
        assert info.status == 0


def test_full_ensemble_sampled_systems():
    # the 256-system ensemble (about 1.3 million rods, float32 iterations,
    # every system solved to the tolerance on its own), in every launch shape
    # the autotuner may pick for the timed steps (the default 1024 x 8 among
    # them): the smallest, a middle and the largest system against the oracle
    import paper_2109_08206_gb300.autotune as T
    systems = W.ensemble(seed=1000, count=256)
    tol = 1e-5
    order = np.argsort([s.n for s in systems])
    picks = (int(order[0]), int(order[len(order) // 2]), int(order[-1]))
    refs = {k: O.step(systems[k].x, systems[k].quat, systems[k].f_nc, O.problem_of(systems[k]), tol=1e-10)
            for k in picks}
    for shape in T.BATCH_CANDIDATES:
        off, x, q, pairs, gam, vel, info = run_batch(systems, A.MIXED, tol, shape)
        assert info.status == 0 and info.residual <= tol, shape
        for k in picks:
            s, ref = systems[k], refs[k]
            lo, hi = off[k], off[k + 1]
            sel = (pairs[:, 0] >= lo) & (pairs[:, 0] < hi)
            mine = pairs[sel].copy()
            mine[:, :2] -= lo
            compare_pairs(mine, ref["pairs"], s)
            U = vel[lo:hi]
            assert np.linalg.norm(U - ref["U"]) <= 1e-3 * np.linalg.norm(ref["U"]), (s.name, shape)
            assert np.abs(periodic_diff(x[lo:hi], ref["x"], s.box)).max() <= 1e-4 * s.diameter, (s.name, shape)


def test_autotune_batch_picks_and_caches():
    import paper_2109_08206_gb300.autotune as T
    systems = small_batch()
    off, x, quat, fnc, spec = W.batch_arrays(systems)
    xd, qd, fd = dev(x), dev(quat), dev(fnc)
    with batch_ctx(systems, A.MIXED, 1e-6) as ctx:
        shape, times = T.tune_batch(ctx, spec, off, xd, qd, fd, A.MIXED)
        assert shape in T.BATCH_CANDIDATES and len(times) == len(T.BATCH_CANDIDATES)
        assert np.array_equal(host(xd), x)   # inputs restored
        info = ctx.step_batch(spec, off, xd, qd, fd)
        assert info.status == 0
        assert T.apply_cached(ctx, "batch", A.MIXED, int(off[-1]), info.n_pairs, len(systems))



@pytest.mark.parametrize("precision,tol", [(A.FP64, 1e-10), (A.MIXED, 1e-6)])
def test_batch_graph_replay_equals_eager_steps(precision, tol):
    """aLENS_set_batch_graph: four steps of the small batch from one state;
    the first runs without a graph, the second records the graph, the last
    two replay it.  Every output equals that of steps without a graph bit
    for bit, the step's counters come back, and a context that changes its
    buffers starts over without a graph."""
    systems = small_batch()
    off, x, quat, fnc, spec = W.batch_arrays(systems)
    n = int(off[-1])

    def steps(graph):
        out = []
        with batch_ctx(systems, precision, tol) as ctx:
            if graph:
                ctx.set_batch_graph(True)
            xd, qd, fd = dev(x), dev(quat), dev(fnc)
            pr = torch.empty((ctx.max_pairs, 3), dtype=torch.int32, device="cuda")
            gam = torch.empty(ctx.max_pairs, dtype=torch.float64, device="cuda")
            vel = torch.empty((n, 6), dtype=torch.float64, device="cuda")
            for k in range(4):
                xd.copy_(dev(x)); qd.copy_(dev(quat))
                info = ctx.step_batch(spec, off, xd, qd, fd, pairs_out=pr, gamma_out=gam, vel_out=vel)
                m = info.n_pairs
                its, res = ctx.batch_results(len(systems))
                out.append((host(xd), host(qd), host(pr)[:m], host(gam)[:m], host(vel), info.as_dict(), its, res))
            if graph:
                # new buffers: another key, so this step runs without the graph and still matches
                x2, q2 = dev(x), dev(quat)
                info = ctx.step_batch(spec, off, x2, q2, fd)
                assert np.array_equal(host(x2), out[0][0]) and info.n_pairs == out[0][5]["n_pairs"]
        return out

    eager, graph = steps(False), steps(True)
    for k in range(4):
        for a, b in zip(eager[k][:5], graph[k][:5]):
            assert np.array_equal(a, b), k
        ie, ig = eager[k][5], graph[k][5]
        for f in ("n_pairs", "n_overlap", "iters", "status", "residual", "min_gap"):
            assert ie[f] == ig[f], (k, f)
        assert np.array_equal(eager[k][6], graph[k][6]) and np.array_equal(eager[k][7], graph[k][7])
        assert ig["ms_solve"] > 0.0 and ig["solver"] == 4
    assert graph[3][5]["launches"] == graph[2][5]["launches"]


def test_batch_graph_capacity_leaves_the_state_untouched():
    """A replayed graph whose pairs exceed the capacity moves no rod and
    reports CAPACITY with the required count, like a step without a graph."""
    systems = small_batch()
    off, x, quat, fnc, spec = W.batch_arrays(systems)
    n = int(off[-1])
    with batch_ctx(systems, A.FP64, 1e-10) as big:
        need = big.step_batch(spec, off, dev(x), dev(quat), dev(fnc)).n_pairs
    s0 = systems[0]
    p = A.make_params(s0.box, s0.diameter, s0.length, s0.viscosity, s0.dt, s0.delta_c, 1e-10, 400000, A.FP64)
    with A.Context(p, n, need - 1) as ctx:
        ctx.set_batch_graph(True)
        xd, qd, fd = dev(x), dev(quat), dev(fnc)
        for k in range(3):   # eager, recorded, replayed
            with pytest.raises(A.AlensError) as e:
                ctx.step_batch(spec, off, xd, qd, fd)
            assert e.value.status == 2 and e.value.extra["n_pairs"] == need, k
            assert np.array_equal(host(xd), x) and np.array_equal(host(qd), quat)
