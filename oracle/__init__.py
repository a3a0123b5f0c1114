"""Python handle on the plain FP64 CPU oracle (``alens_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark use it to check and time the CUDA path.  The product
library never imports it.  Arrays go in and out as float64 / int32 numpy
arrays; the C side does all arithmetic.

Parity pins: every function here is checked by ``tests/test_oracle_*.py``
against closed forms, brute force, library routines or invariants; none is
"parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "alens_oracle.c"
_LIB = _HERE / "_build" / "liborc.so"


class Problem(C.Structure):
    _fields_ = [("box", C.c_double * 3), ("diameter", C.c_double), ("length", C.c_double),
                ("viscosity", C.c_double), ("dt", C.c_double), ("delta_c", C.c_double)]


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (-O2 -ffp-contract=off, OpenMP)."""
    if _LIB.exists() and not force and _LIB.stat().st_mtime >= _SRC.stat().st_mtime:
        return _LIB
    _LIB.parent.mkdir(parents=True, exist_ok=True)
    tmp = _LIB.with_suffix(f".{os.getpid()}.tmp")
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-fvisibility=hidden", str(_SRC), "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(str(build()))
        d, i64, vp = C.c_double, C.c_int64, C.c_void_p
        P = C.POINTER(Problem)
        sig = {
            "orc_set_threads": (C.c_int, [C.c_int]),
            "orc_drag": (None, [d, d, d, vp]),
            "orc_axis": (None, [i64, vp, vp]),
            "orc_wrap": (None, [i64, vp, vp, vp]),
            "orc_segment_closest": (d, [vp, vp, vp, d, vp, vp]),
            "orc_find_pairs": (i64, [i64, vp, vp, P, vp, i64]),
            "orc_find_pairs_rows": (i64, [i64, vp, vp, P, vp, i64, vp, i64]),
            "orc_pair_gaps": (None, [i64, vp, vp, P, i64, vp, vp]),
            "orc_mobility_apply": (None, [i64, vp, P, vp, vp]),
            "orc_assemble": (None, [i64, vp, vp, vp, P, i64, vp, vp, vp, vp, vp, vp]),
            "orc_apply_D": (None, [i64, i64, vp, vp, vp, vp]),
            "orc_apply_Dt": (None, [i64, vp, vp, vp, vp]),
            "orc_gradient": (d, [i64, vp, P, i64, vp, vp, vp, vp, vp, vp]),
            "orc_dense_A": (None, [i64, vp, P, i64, vp, vp, vp, vp]),
            "orc_solve_enum": (i64, [i64, vp, P, i64, vp, vp, vp, vp, vp]),
            "orc_solve_apgd": (d, [i64, vp, P, i64, vp, vp, vp, vp, vp, d, i64, vp]),
            "orc_assemble_springs": (None, [i64, vp, vp, vp, P, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
            "orc_philox4x32": (None, [vp, vp, vp]),
            "orc_normals6": (None, [C.c_uint64, C.c_uint64, i64, vp]),
            "orc_brownian": (None, [i64, vp, P, d, C.c_uint64, C.c_uint64, vp, vp]),
            "orc_assemble_walls": (i64, [i64, vp, vp, vp, P, C.c_int, d, d, i64, vp, vp, vp, vp]),
            "orc_update": (None, [i64, vp, vp, vp, P, i64, vp, vp, vp, vp, vp, vp]),
            "orc_step": (i64, [i64, vp, vp, vp, P, d, i64, i64, vp, vp, vp, vp, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def problem(box, diameter=1.0, length=10.0, viscosity=1.0, dt=1e-3, delta_c=None) -> Problem:
    b = box if np.ndim(box) else (box, box, box)
    return Problem((C.c_double * 3)(*[float(v) for v in b]), float(diameter), float(length),
                   float(viscosity), float(dt), float(diameter if delta_c is None else delta_c))


def problem_of(sys) -> Problem:
    """Problem parameters of a ``workloads.RodSystem``."""
    return problem(sys.box, sys.diameter, sys.length, sys.viscosity, sys.dt, sys.delta_c)


def set_threads(n: int) -> int:
    """Threads of the oracle's parallel loops (n <= 0 leaves them); returns
    the count in force before the call."""
    return int(lib().orc_set_threads(int(n)))


def drag(eta, length, diameter):
    out = np.zeros(4)
    lib().orc_drag(eta, length, diameter, _p(out))
    return out  # zeta_perp, zeta_par, zeta_rot, zeta_spin


def axis(quat):
    q = _f64(quat, (-1, 4))
    out = np.zeros((q.shape[0], 3))
    lib().orc_axis(q.shape[0], _p(q), _p(out))
    return out


def wrap(x, box):
    xx = _f64(x, (-1, 3))
    b = _f64(box if np.ndim(box) else [box] * 3)
    out = np.zeros_like(xx)
    lib().orc_wrap(xx.shape[0], _p(xx), _p(b), _p(out))
    return out


def segment_closest(dx, p, q, length):
    dx, p, q = _f64(dx), _f64(p), _f64(q)
    s, t = C.c_double(), C.c_double()
    d = lib().orc_segment_closest(_p(dx), _p(p), _p(q), float(length), C.byref(s), C.byref(t))
    return d, s.value, t.value


def find_pairs(x, quat, pb: Problem, rows=None):
    x, quat = _f64(x, (-1, 3)), _f64(quat, (-1, 4))
    n = x.shape[0]
    if rows is None:
        cnt = lib().orc_find_pairs(n, _p(x), _p(quat), C.byref(pb), None, 0)
        out = np.zeros((max(cnt, 1), 3), dtype=np.int32)
        cnt2 = lib().orc_find_pairs(n, _p(x), _p(quat), C.byref(pb), _p(out), cnt)
    else:
        r = np.ascontiguousarray(np.unique(np.asarray(rows, dtype=np.int64)))
        cnt = lib().orc_find_pairs_rows(n, _p(x), _p(quat), C.byref(pb), _p(r), r.shape[0], None, 0)
        out = np.zeros((max(cnt, 1), 3), dtype=np.int32)
        cnt2 = lib().orc_find_pairs_rows(n, _p(x), _p(quat), C.byref(pb), _p(r), r.shape[0], _p(out), cnt)
    assert cnt2 == cnt
    return out[:cnt]


def pair_gaps(x, quat, pb: Problem, pairs):
    x, quat = _f64(x, (-1, 3)), _f64(quat, (-1, 4))
    pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 3)
    out = np.zeros(pr.shape[0])
    lib().orc_pair_gaps(x.shape[0], _p(x), _p(quat), C.byref(pb), pr.shape[0], _p(pr), _p(out))
    return out


def mobility_apply(quat, pb: Problem, F):
    quat, F = _f64(quat, (-1, 4)), _f64(F, (-1, 6))
    U = np.zeros_like(F)
    lib().orc_mobility_apply(quat.shape[0], _p(quat), C.byref(pb), _p(F), _p(U))
    return U


def assemble(x, quat, fnc, pb: Problem, pairs):
    x, quat, fnc = _f64(x, (-1, 3)), _f64(quat, (-1, 4)), _f64(fnc, (-1, 6))
    pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 3)
    m = pr.shape[0]
    phi, dg, q = np.zeros(m), np.zeros((m, 9)), np.zeros(m)
    yp, yq = np.zeros((m, 3)), np.zeros((m, 3))
    lib().orc_assemble(x.shape[0], _p(x), _p(quat), _p(fnc), C.byref(pb), m, _p(pr), _p(phi), _p(dg), _p(q),
                       _p(yp), _p(yq))
    return {"phi": phi, "dgeom": dg, "q": q, "yP": yp, "yQ": yq}


def apply_D(n, pairs, dgeom, gamma):
    pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 3)
    dg, g = _f64(dgeom, (-1, 9)), _f64(gamma)
    F = np.zeros((n, 6))
    lib().orc_apply_D(n, pr.shape[0], _p(pr), _p(dg), _p(g), _p(F))
    return F


def apply_Dt(pairs, dgeom, U):
    pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 3)
    dg, U = _f64(dgeom, (-1, 9)), _f64(U, (-1, 6))
    out = np.zeros(pr.shape[0])
    lib().orc_apply_Dt(pr.shape[0], _p(pr), _p(dg), _p(U), _p(out))
    return out


def _comp(comp):
    return None if comp is None else _f64(comp)


def gradient(quat, pb: Problem, pairs, dgeom, q, gamma, comp=None):
    """g = (D^T M D + diag(comp+)) gamma + q and the residual; comp (nullable)
    marks bilateral constraints (>= 0: compliance 1/(h kappa)) among unilateral ones (< 0)."""
    quat = _f64(quat, (-1, 4))
    pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 3)
    dg, q, gm, cp = _f64(dgeom, (-1, 9)), _f64(q), _f64(gamma), _comp(comp)
    g = np.zeros(pr.shape[0])
    r = lib().orc_gradient(quat.shape[0], _p(quat), C.byref(pb), pr.shape[0], _p(pr), _p(dg), _p(q), _p(cp),
                           _p(gm), _p(g))
    return g, r


def dense_A(quat, pb: Problem, pairs, dgeom, comp=None):
    quat = _f64(quat, (-1, 4))
    pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 3)
    dg, cp = _f64(dgeom, (-1, 9)), _comp(comp)
    m = pr.shape[0]
    A = np.zeros((m, m))
    lib().orc_dense_A(quat.shape[0], _p(quat), C.byref(pb), m, _p(pr), _p(dg), _p(cp), _p(A))
    return A


def solve_enum(quat, pb: Problem, pairs, dgeom, q, comp=None):
    quat = _f64(quat, (-1, 4))
    pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 3)
    dg, q, cp = _f64(dgeom, (-1, 9)), _f64(q), _comp(comp)
    gm = np.zeros(pr.shape[0])
    mask = lib().orc_solve_enum(quat.shape[0], _p(quat), C.byref(pb), pr.shape[0], _p(pr), _p(dg), _p(q), _p(cp),
                                _p(gm))
    return gm, mask


def solve_apgd(quat, pb: Problem, pairs, dgeom, q, tol=1e-12, max_iter=1_000_000, gamma0=None, comp=None):
    quat = _f64(quat, (-1, 4))
    pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 3)
    dg, q, cp = _f64(dgeom, (-1, 9)), _f64(q), _comp(comp)
    gm = np.zeros(pr.shape[0]) if gamma0 is None else _f64(gamma0).copy()
    it = C.c_int64()
    r = lib().orc_solve_apgd(quat.shape[0], _p(quat), C.byref(pb), pr.shape[0], _p(pr), _p(dg), _p(q), _p(cp),
                             _p(gm), float(tol), int(max_iter), C.byref(it))
    return gm, r, it.value


def assemble_springs(x, quat, fnc, pb: Problem, ends, arms, kappa, rest):
    """Bilateral constraints of the springs: dict with pairs (P, Q, image),
    dgeom, q, length (Phi_b) and comp = 1/(h kappa)."""
    x, quat, fnc = _f64(x, (-1, 3)), _f64(quat, (-1, 4)), _f64(fnc, (-1, 6))
    en = np.ascontiguousarray(ends, dtype=np.int32).reshape(-1, 2)
    ar, kp, rs = _f64(arms, (-1, 2)), _f64(kappa), _f64(rest)
    nb = en.shape[0]
    pr = np.zeros((nb, 3), dtype=np.int32)
    dg, q, ln, cp = np.zeros((nb, 9)), np.zeros(nb), np.zeros(nb), np.zeros(nb)
    lib().orc_assemble_springs(x.shape[0], _p(x), _p(quat), _p(fnc), C.byref(pb), nb, _p(en), _p(ar), _p(kp),
                               _p(rs), _p(pr), _p(dg), _p(q), _p(ln), _p(cp))
    return {"pairs": pr, "dgeom": dg, "q": q, "length": ln, "comp": cp}


def update(x, quat, fnc, pb: Problem, pairs, dgeom, gamma):
    x, quat, fnc = _f64(x, (-1, 3)), _f64(quat, (-1, 4)), _f64(fnc, (-1, 6))
    pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 3)
    dg, gm = _f64(dgeom, (-1, 9)), _f64(gamma)
    xo, qo, U = np.zeros_like(x), np.zeros_like(quat), np.zeros((x.shape[0], 6))
    lib().orc_update(x.shape[0], _p(x), _p(quat), _p(fnc), C.byref(pb), pr.shape[0], _p(pr), _p(dg), _p(gm),
                     _p(xo), _p(qo), _p(U))
    return xo, qo, U


def philox4x32(ctr, key):
    """Philox4x32-10 of four 32-bit counter words and a two-word key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32(_p(c), _p(k), _p(out))
    return out


def normals6(seed, step, i):
    z = np.zeros(6)
    lib().orc_normals6(int(seed), int(step), int(i), _p(z))
    return z


def brownian(quat, pb: Problem, kT, seed, step, f_ext=None):
    """F_nc of one trajectory step: f_ext plus the Brownian force and torque."""
    quat = _f64(quat, (-1, 4))
    out = np.zeros((quat.shape[0], 6))
    fe = None if f_ext is None else _f64(f_ext, (-1, 6))
    lib().orc_brownian(quat.shape[0], _p(quat), C.byref(pb), float(kT), int(seed), int(step), _p(fe), _p(out))
    return out


def assemble_walls(x, quat, fnc, pb: Problem, axis_w, lo, hi):
    """One-sided wall constraints: dict pairs (i, -1, 2 side + end), dgeom, q, phi."""
    x, quat, fnc = _f64(x, (-1, 3)), _f64(quat, (-1, 4)), _f64(fnc, (-1, 6))
    n = x.shape[0]
    cnt = lib().orc_assemble_walls(n, _p(x), _p(quat), _p(fnc), C.byref(pb), int(axis_w), float(lo), float(hi), 0,
                                   None, None, None, None)
    pr = np.zeros((max(cnt, 1), 3), dtype=np.int32)
    dg, q, ph = np.zeros((max(cnt, 1), 9)), np.zeros(max(cnt, 1)), np.zeros(max(cnt, 1))
    lib().orc_assemble_walls(n, _p(x), _p(quat), _p(fnc), C.byref(pb), int(axis_w), float(lo), float(hi), cnt,
                             _p(pr), _p(dg), _p(q), _p(ph))
    return {"pairs": pr[:cnt], "dgeom": dg[:cnt], "q": q[:cnt], "phi": ph[:cnt]}


def step(x, quat, fnc, pb: Problem, tol=1e-12, max_iter=1_000_000, max_pairs=None, springs=None, walls=None):
    """One full constrained step; returns a dict of every intermediate.

    ``springs`` (nullable): dict of ends [nb, 2], arms [nb, 2], kappa [nb],
    rest [nb]: bilateral constraints solved together with the collisions
    (Eq. linearconstraints b).  ``walls`` (nullable): (axis, lo, hi), two
    flat confining walls (one-sided constraints).  ``gamma`` holds the
    collision forces, then the wall forces, then the spring forces."""
    x, quat, fnc = _f64(x, (-1, 3)), _f64(quat, (-1, 4)), _f64(fnc, (-1, 6))
    pairs = find_pairs(x, quat, pb)
    asm = assemble(x, quat, fnc, pb, pairs)
    if springs is None and walls is None:
        gamma, res, iters = solve_apgd(quat, pb, pairs, asm["dgeom"], asm["q"], tol=tol, max_iter=max_iter)
        xo, qo, U = update(x, quat, fnc, pb, pairs, asm["dgeom"], gamma)
        return {"pairs": pairs, **asm, "gamma": gamma, "residual": res, "iters": iters, "x": xo, "quat": qo, "U": U}
    rows_p, rows_d, rows_q = [pairs.reshape(-1, 3)], [asm["dgeom"].reshape(-1, 9)], [asm["q"]]
    comps = [-np.ones(pairs.shape[0])]
    wb = sb = None
    if walls is not None:
        wb = assemble_walls(x, quat, fnc, pb, *walls)
        rows_p.append(wb["pairs"]); rows_d.append(wb["dgeom"]); rows_q.append(wb["q"])
        comps.append(-np.ones(wb["pairs"].shape[0]))
    if springs is not None:
        sb = assemble_springs(x, quat, fnc, pb, springs["ends"], springs["arms"], springs["kappa"], springs["rest"])
        rows_p.append(sb["pairs"]); rows_d.append(sb["dgeom"]); rows_q.append(sb["q"]); comps.append(sb["comp"])
    allp = np.concatenate(rows_p).astype(np.int32)
    dg = np.concatenate(rows_d)
    q = np.concatenate(rows_q)
    comp = np.concatenate(comps)
    if allp.shape[0] <= 20:
        gamma, _ = solve_enum(quat, pb, allp, dg, q, comp=comp)
        res = gradient(quat, pb, allp, dg, q, gamma, comp=comp)[1]
        iters = 0
    else:
        gamma, res, iters = solve_apgd(quat, pb, allp, dg, q, tol=tol, max_iter=max_iter, comp=comp)
    xo, qo, U = update(x, quat, fnc, pb, allp, dg, gamma)
    return {"pairs": pairs, **asm, "springs": sb, "walls": wb, "all_pairs": allp, "all_dgeom": dg, "all_q": q,
            "comp": comp, "gamma": gamma, "residual": res, "iters": iters, "x": xo, "quat": qo, "U": U}


def trajectory(x, quat, pb: Problem, n_steps, kT, seed, first_step=0, f_ext=None, springs=None, walls=None,
               tol=1e-12):
    """n_steps constrained Brownian steps (F_nc = f_ext + the Brownian force
    of step first_step + k); returns (x, quat, per-step list of dicts with
    the pair count, residual and minimum gap)."""
    x, quat = _f64(x, (-1, 3)).copy(), _f64(quat, (-1, 4)).copy()
    stats = []
    for k in range(n_steps):
        fnc = brownian(quat, pb, kT, seed, first_step + k, f_ext)
        out = step(x, quat, fnc, pb, tol=tol, springs=springs, walls=walls)
        gaps = [out["phi"]] if out["pairs"].shape[0] else []
        if out.get("walls") is not None and out["walls"]["pairs"].shape[0]:
            gaps.append(out["walls"]["phi"])
        stats.append({"n_pairs": int(out["pairs"].shape[0]), "residual": out["residual"],
                      "min_gap": float(np.min(np.concatenate(gaps))) if gaps else float("inf")})
        x, quat = out["x"], out["quat"]
    return x, quat, stats


def step_native(x, quat, fnc, pb: Problem, tol, max_iter, max_pairs):
    """The whole step inside one C call (used to time the oracle)."""
    x, quat, fnc = _f64(x, (-1, 3)), _f64(quat, (-1, 4)), _f64(fnc, (-1, 6))
    n = x.shape[0]
    pairs = np.zeros((max_pairs, 3), dtype=np.int32)
    gamma = np.zeros(max_pairs)
    xo, qo, U = np.zeros_like(x), np.zeros_like(quat), np.zeros((n, 6))
    res, it = C.c_double(), C.c_int64()
    np_ = lib().orc_step(n, _p(x), _p(quat), _p(fnc), C.byref(pb), float(tol), int(max_iter), int(max_pairs),
                         _p(pairs), _p(gamma), _p(xo), _p(qo), _p(U), C.byref(res), C.byref(it))
    return {"n_pairs": np_, "pairs": pairs[:max(np_, 0)], "gamma": gamma[:max(np_, 0)], "x": xo, "quat": qo,
            "U": U, "residual": res.value, "iters": it.value}
