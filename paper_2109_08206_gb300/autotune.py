"""Launch-shape autotuner for the BBPGD kernels.

The solver's launch shape changes only how the work is spread, never what is
computed (each candidate runs the same BBPGD to the same tolerance), so the
tuner times the solve phase of one real step per candidate and keeps the
cheapest.  For a single system the score is the solve time per BBPGD
iteration: the shape also sets the order of the float32 block sums, and the
Barzilai-Borwein iteration count reacts to that order by tens of per cent in
either direction without any trend, so a whole-solve time would mostly rank
the luck of that count.  A batch scores its whole solve time, in which the
counts of hundreds of systems average out.  Results are cached in
``_build/tune.json`` per workload class:
kind (single system or batch), precision, and the bucketed ratios that set
the per-iteration work - constraints per rod (N_c/N, half-octave buckets) and
rods per system (octave buckets).  ``apply_cached`` sets a cached shape on a
context without timing anything.

Single system: (threads per block, blocks per SM) of the cooperative solver
(aLENS_set_launch).  Batch: (threads per block, blocks per cluster) of the
per-system solver (aLENS_set_batch_launch).
"""
from __future__ import annotations

import json
import math
from pathlib import Path

_CACHE = Path(__file__).resolve().parent / "_build" / "tune.json"

SINGLE_CANDIDATES = ((768, 1), (1024, 1), (512, 1), (512, 2), (256, 4))
TIE = 0.01   # a candidate must beat an earlier one by this fraction to be preferred
BATCH_CANDIDATES = ((1024, 8), (1024, 4), (512, 4), (512, 2))


def workload_key(kind: str, precision: int, n_rods: int, n_pairs: int, n_systems: int = 1) -> str:
    ratio = max(n_pairs, 1) / max(n_rods, 1)
    per_sys = max(n_rods, 1) / max(n_systems, 1)
    return f"{kind}:p{precision}:c{round(2 * math.log2(ratio))}:r{round(math.log2(per_sys))}"


def _load() -> dict:
    try:
        return json.loads(_CACHE.read_text())
    except (OSError, ValueError):
        return {}


def _store(key: str, shape, cost: dict):
    d = _load()
    d[key] = {"shape": list(shape), "cost": cost, "unit": cost_unit(key.split(":")[0])}
    _CACHE.parent.mkdir(parents=True, exist_ok=True)
    _CACHE.write_text(json.dumps(d, indent=1, sort_keys=True))


def cached(key: str):
    e = _load().get(key)
    return tuple(e["shape"]) if e else None


def apply(ctx, kind: str, shape):
    """Set a launch shape ("single": threads x blocks per SM, "batch":
    threads x blocks per cluster) on a context, e.g. one tuned on another
    input of the same workload class."""
    if kind == "batch":
        ctx.set_batch_launch(*shape)
    else:
        ctx.set_launch(*shape)


_set = apply


def cost_unit(kind: str) -> str:
    return "ms per batched solve" if kind == "batch" else "us per BBPGD iteration"


def _cost(kind: str, info) -> float:
    if kind == "batch":
        return info.ms_solve
    return 1e3 * info.ms_solve / max(info.iters, 1)


def _tune(ctx, kind, key, run, candidates, reps):
    times = {}
    for shape in candidates:
        _set(ctx, kind, shape)
        best = math.inf
        for _ in range(reps):
            info = run()
            if info.status not in (0, 3):   # OK or NOT_CONVERGED: the timing is valid
                break
            best = min(best, _cost(kind, info))
        times[f"{shape[0]}x{shape[1]}"] = best
    # the first candidate within TIE of the best: timing noise between
    # near-equal shapes does not flip the pick
    best = min(times.values())
    shape = next(s for s in candidates if times[f"{s[0]}x{s[1]}"] <= best * (1.0 + TIE))
    _set(ctx, kind, shape)
    _store(key, shape, times)
    return shape, times


def tune_single(ctx, x, quat, f_nc, precision: int, candidates=SINGLE_CANDIDATES, reps: int = 2):
    """Time aLENS_step's solve for each (threads, blocks per SM); x and quat
    are restored before every step.  Returns (best shape, {shape: us per
    iteration})."""
    x0, q0 = x.clone(), quat.clone()

    def run():
        x.copy_(x0)
        quat.copy_(q0)
        return ctx.step(x, quat, f_nc, check=False)

    info = run()
    key = workload_key("single", precision, x.shape[0], info.n_pairs)
    out = _tune(ctx, "single", key, run, candidates, reps)
    x.copy_(x0)
    quat.copy_(q0)
    return out


def tune_batch(ctx, systems, rod_offset, x, quat, f_nc, precision: int, candidates=BATCH_CANDIDATES,
               reps: int = 2):
    """Time aLENS_step_batch's solve for each (threads, blocks per cluster).
    Returns (best shape, {shape: ms per solve})."""
    x0, q0 = x.clone(), quat.clone()

    def run():
        x.copy_(x0)
        quat.copy_(q0)
        return ctx.step_batch(systems, rod_offset, x, quat, f_nc, check=False)

    info = run()
    key = workload_key("batch", precision, x.shape[0], info.n_pairs, len(systems))
    out = _tune(ctx, "batch", key, run, candidates, reps)
    x.copy_(x0)
    quat.copy_(q0)
    return out


def apply_cached(ctx, kind: str, precision: int, n_rods: int, n_pairs: int, n_systems: int = 1) -> bool:
    """Set the cached shape for this workload class, if one was tuned."""
    shape = cached(workload_key(kind, precision, n_rods, n_pairs, n_systems))
    if shape is None:
        return False
    _set(ctx, kind, shape)
    return True
