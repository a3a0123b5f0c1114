"""Benchmark of the collision-constraint step: rod-steps/s at 1e5 rods.

One step = neighbour search + constraint assembly + BBPGD solve + update
(the whole hot path) over the 100,000-rod suspension (volume fraction 0.10,
isotropic, thermal forces plus 50,000 explicit crosslinker springs; seeded,
synthetic).  Every timed step starts from the same input state, restored
outside the timed region, and L2 is flushed (256 MB write) between steps.
``--workload ensemble256`` times the batched step (aLENS_step_batch) of the
256-system ensemble instead (about 1.28 million rods in one call).

Reported (one JSON line on rank 0):
  value        rod-steps/s of the FP32-mixed step at residual <= 1e-5 (device
               events on the library's stream around aLENS_step, inputs
               resident in HBM);
  fp64         the same for the FP64-plain step at the same residual;
  e2e          the same metric through the C ABI with host buffers: pinned
               host -> device copy of x, quat, f_nc, the step, and the
               device -> host copy of x and quat inside the timed region;
  roofline     the BBPGD kernel (dominant): algorithmic bytes per launch
               (iterations x per-iteration bytes of the solve) / its event time
               vs the measured HBM copy bandwidth;
  cpu_baseline the CPU oracle timed on a bounded spatial sample of the same
               workload on this host's cores.
  --impl reference times that oracle alone (the reference arm).
Multi-GPU (torchrun): independent replicas, one per rank, no collective on
the data path; value = rods x steps of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "rod-steps/s at 1e5 rods, FP32-mixed vs FP64 plain at residual ≤1e-5"
METRIC_ENSEMBLE = "rod-steps/s of the 256-system batched ensemble (one call), FP32-mixed vs FP64 plain at residual ≤1e-5"
METRIC_SPRINGS = ("rod-steps/s at 1e5 rods with 5e4 bilateral spring constraints, FP32-mixed vs FP64 plain at "
                  "residual ≤1e-5")
METRIC_TRAJ = ("rod-steps/s of a 1e5-rod Brownian trajectory (10 steps per call, warm start), FP32-mixed vs FP64 "
               "plain at residual ≤1e-5")
METRIC_GRAD = ("rod-steps/s of one step plus its adjoint (gradient of the post-step centre loss) at 2e4 rods, "
               "FP32-mixed vs FP64 plain at residual ≤1e-5")


METRIC_N1000 = "rod-steps/s at 1e3 rods (periodic cube of side 40), FP64 plain at residual ≤1e-8"
METRIC_N400K = ("rod-steps/s at 4e5 rods (nematic bundle, volume fraction 0.25), FP32-mixed vs FP64 plain at "
                "residual ≤1e-5")


def metric_of(workload):
    return {"ensemble256": METRIC_ENSEMBLE, "n20k_grad": METRIC_GRAD,
            "n100k_springs": METRIC_SPRINGS, "n100k_traj": METRIC_TRAJ,
            "n1000_box40": METRIC_N1000, "n400k_nematic": METRIC_N400K}.get(workload, METRIC)
UNIT = "rod-steps/s"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="n100k_phi010")
    ap.add_argument("--tol", type=float, default=1e-5)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--sample-rods", type=int, default=10000, help="rods in the oracle's spatial sample")
    ap.add_argument("--no-tune", action="store_true", help="keep the default solver launch shape")
    ap.add_argument("--scaling", type=float, default=None,
                    help="diagonal scaling exponent of the BBPGD iteration (default: the library's, 0.5)")
    ap.add_argument("--barriers", type=int, default=None, choices=[1, 2],
                    help="grid barriers per BBPGD iteration (default: the library's, one where it fits)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="precision of the headline step (fp64: the float64 step is the value and no mixed arm runs)")
    ap.add_argument("--shape", default=None,
                    help="solver launch shape THREADSxBLOCKS (per SM, or per cluster for a batch); skips tuning")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        try:
            d = json.loads(p.read_text())
            for k in ("hbm_gbs", "hbm_GBps", "hbm"):
                if k in d and isinstance(d[k], (int, float)):
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi samples (200 ms) during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id):
        self.idx = device_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            sel = ["-i", str(self.idx)] if self.idx is not None else []
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "50", *sel], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [v.strip() for v in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def solve_bytes_per_iter(n, m, w):
    """Algorithmic bytes of one BBPGD iteration: per constraint 24w + 24
    (D record read by the rod gather and by D^T, gamma x3, g x2, q, two CSR
    entries), per rod 15w + 4 (axis, U write, U read, row pointer)."""
    return m * (24 * w + 24) + n * (15 * w + 4)


def step_other_bytes(n, m, w):
    """Algorithmic bytes of a step outside the BBPGD iterations: the
    neighbour search and assembly, N (56 + 24) + N_c (12 + 32 + 11w + 8)
    (rod state and keys in, pair list, records, q and Phi out), and the
    update, N (2 x 56 + 6w) (rod state in and out, the constraint velocity)."""
    return n * (56 + 24) + m * (12 + 32 + 11 * w + 8) + n * (2 * 56 + 6 * w)


PROFILE_RECORD = "profiles/k_bbpgd1_n100k_mixed.json"


def traffic_from_profile(kernel_src: Path, shape, kernel: str):
    """DRAM bytes of one BBPGD launch from the committed ncu record
    (``profiles/k_bbpgd1_n100k_mixed.json``), only if the solver source is
    unchanged since the capture (its sha256 is recorded there), the capture
    ran in the same launch shape and the same kernel ran."""
    path = ROOT / PROFILE_RECORD
    if not path.exists():
        return None
    try:
        rec = json.loads(path.read_text())
    except ValueError:
        return None
    sha = hashlib.sha256(kernel_src.read_bytes()).hexdigest()[:16]
    if rec.get("solve_cu_sha256_16") != sha or rec.get("kernel") != kernel:
        return None
    if shape is None or rec.get("launch_shape") != f"{shape[0]}x{shape[1]}":
        return None
    return float(rec["dram_bytes_per_launch"])


def spatial_sample(s, target):
    """Rods of the workload whose centres fall in the cube [0, a)^3, with a
    chosen so that about `target` rods fall inside; the cube is treated as a
    periodic system of its own (same density, orientations and forces)."""
    from paper_2109_08206_gb300 import workloads as W
    box = np.asarray(s.box)
    frac = (target / s.n) ** (1.0 / 3.0)
    a = max(float(box.min() * frac), s.length + s.diameter + s.delta_c + 1e-6)
    sel = np.all(s.x < a, axis=1)
    sub = W.RodSystem(x=s.x[sel].copy(), quat=s.quat[sel].copy(), f_nc=s.f_nc[sel].copy(), box=(a, a, a),
                      diameter=s.diameter, length=s.length, viscosity=s.viscosity, dt=s.dt, delta_c=s.delta_c,
                      tol=s.tol, name=s.name + "_sample")
    return sub, a


def ensemble_sample(systems, target, seed=7):
    """Systems of the ensemble in a seeded random order until about `target`
    rods are taken (the oracle's CPU sample of the batched workload)."""
    rng = np.random.default_rng(seed)
    take, rods = [], 0
    for k in rng.permutation(len(systems)):
        if rods >= target:
            break
        take.append(int(k))
        rods += systems[k].n
    return take, rods


class SingleJob:
    """One system stepped by aLENS_step (recorded once as a CUDA graph and
    replayed, where the step runs the one-barrier solver)."""

    graph = True

    def __init__(self, s):
        self.s = s
        self.n = s.n
        self.name = s.name

    def context(self, A, precision, tol, stream):
        p = A.params_of(self.s, precision=precision, tol=tol, max_iter=1_000_000)
        ctx = A.Context(p, self.n, 12 * self.n, stream=stream)
        if self.graph:
            ctx.set_step_graph(True)
        return ctx

    def step(self, ctx, x, q, f, **kw):
        return ctx.step(x, q, f, **kw)

    def tune(self, T, ctx, x, q, f, precision):
        return T.tune_single(ctx, x, q, f, precision)

    def solve_bytes(self, ctx, info, w):
        """Algorithmic bytes of the BBPGD launch of the last step."""
        return info["iters"] * solve_bytes_per_iter(self.n, info["n_pairs"], w)

    def arrays(self):
        return self.s.x, self.s.quat, self.s.f_nc

    def periodic_box(self):
        return np.broadcast_to(np.asarray(self.s.box, dtype=np.float64), (self.n, 3))

    def config(self, W, m):
        s = self.s
        c = {"workload": s.name, "rods": self.n, "pairs": m, "box": round(float(s.box[0]), 3),
             "volume_fraction": round(self.n * W.rod_volume(s.diameter, s.length) / float(np.prod(s.box)), 4),
             "springs": s.meta.get("springs")}
        if self.graph:
            c["step"] = "one aLENS_step call, replayed as a captured CUDA graph where it runs the one-barrier solver"
        return c

    def cpu(self, args):
        sub, a = spatial_sample(self.s, args.sample_rods)
        t_cpu, out = oracle_step_time(sub, args.tol)
        return sub.n, t_cpu, (f"{sub.n} rods of {self.s.name} with centres in a periodic sub-cube of edge {a:.2f}; "
                              f"one full oracle step (brute-force pairs, FISTA to residual {args.tol:g}, update), "
                              f"{t_cpu:.2f} s")


class BatchJob:
    """The ensemble stepped by one aLENS_step_batch call."""

    def __init__(self, systems):
        from paper_2109_08206_gb300 import workloads as W
        self.systems = systems
        self.off, self.x, self.quat, self.f_nc, self.spec = W.batch_arrays(systems)
        self.n = int(self.off[-1])
        self.name = f"ensemble{len(systems)}"
        self.ms = None   # per-system constraint counts (set by the first step with pairs_out)
        self.tables = None

    def context(self, A, precision, tol, stream):
        s0 = self.systems[0]
        p = A.make_params(s0.box, s0.diameter, s0.length, s0.viscosity, s0.dt, s0.delta_c, tol, 1_000_000,
                          precision)
        ctx = A.Context(p, self.n, 12 * self.n, stream=stream)
        ctx.set_batch_graph(True)   # the step recorded once as a CUDA graph, then replayed
        return ctx

    def step(self, ctx, x, q, f, **kw):
        if self.tables is None:   # the C tables of the batch, built once
            import paper_2109_08206_gb300 as A
            self.tables = A.BatchSpec(self.spec, self.off)
        return ctx.step_batch(self.tables, None, x, q, f, **kw)

    def tune(self, T, ctx, x, q, f, precision):
        return T.tune_batch(ctx, self.spec, self.off, x, q, f, precision)

    def count_pairs(self, pairs):
        sys_i = np.searchsorted(self.off, pairs[:, 0], side="right") - 1
        self.ms = np.bincount(sys_i, minlength=len(self.systems))

    def solve_bytes(self, ctx, info, w):
        its, _ = ctx.batch_results(len(self.systems))
        ns = np.diff(self.off)
        return float(np.sum(its * (self.ms * (24 * w + 24) + ns * (15 * w + 4))))

    def arrays(self):
        return self.x, self.quat, self.f_nc

    def periodic_box(self):
        return np.repeat(np.asarray([s.box for s in self.systems], dtype=np.float64), np.diff(self.off), axis=0)

    def config(self, W, m):
        return {"workload": self.name, "systems": len(self.systems), "rods": self.n, "pairs": m,
                "rods_per_system": [int(np.diff(self.off).min()), int(np.diff(self.off).max())],
                "step": "one aLENS_step_batch call, replayed as a captured CUDA graph",
                "orientation": f"nematic domains, spread {W.ENSEMBLE_SPREAD} rad about a random director each"}

    def cpu(self, args):
        take, rods = ensemble_sample(self.systems, args.sample_rods)
        t_cpu = 0.0
        for k in take:
            t, _ = oracle_step_time(self.systems[k], args.tol)
            t_cpu += t
        return rods, t_cpu, (f"{len(take)} whole systems of the ensemble ({rods} rods, seeded random pick), "
                             f"each one full oracle step (brute-force pairs, FISTA to residual {args.tol:g}, "
                             f"update), {t_cpu:.2f} s in total")


def cg_bytes_per_iter(n, m, w):
    """Algorithmic bytes of one CG iteration of the adjoint, m the ACTIVE
    constraints (the CG works on the active set only): per constraint
    12w + 60 (rod pass: its record arms and (r, p, Ap) gathered from both
    ends, with the list entries) and 21w + 76 (constraint pass: record, both
    ends' velocities, list entry and end indices, (r, p, Ap, lambda) read and
    written); per rod 9w + 8 (row pointers, axis, velocity write)."""
    return m * (33 * w + 136) + n * (9 * w + 8)


class GradJob(SingleJob):
    """One step and its adjoint (aLENS_step + aLENS_step_adjoint) for the loss
    sum |x' - target|^2 of the differentiation workload."""

    graph = False

    class Out:
        def __init__(self, d):
            self.d = d

        def as_dict(self):
            return self.d

    def __init__(self, s):
        super().__init__(s)
        from paper_2109_08206_gb300 import workloads as W
        self.name = s.name + "_grad"
        self.T = W.loss_targets(s)
        self._bufs = None
        self._active = None   # active constraints of the workload's step (counted once)

    def step(self, ctx, x, q, f, **kw):
        import torch
        if self._bufs is None or self._bufs[0].shape[0] < ctx.max_pairs:
            dev = x.device
            self._bufs = (torch.empty((ctx.max_pairs, 3), dtype=torch.int32, device=dev),
                          torch.empty(ctx.max_pairs, dtype=torch.float64, device=dev),
                          torch.empty((self.n, 6), dtype=torch.float64, device=dev),
                          torch.as_tensor(self.T, device=dev),
                          torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        pr, gm, vel, T, e0, e1 = self._bufs
        x0, q0 = x.clone(), q.clone()
        info = ctx.step(x, q, f, pairs_out=pr, gamma_out=gm, vel_out=vel)
        m = info.n_pairs
        stream = torch.cuda.current_stream()
        e0.record(stream)
        xn = x0 + ctx.params.dt * vel[:, :3]
        gx, gq, gf, geta, ainfo = ctx.step_adjoint(x0, q0, f, pr[:m], gm[:m], 2.0 * (xn - T))
        e1.record(stream)
        e1.synchronize()
        d = info.as_dict()
        if self._active is None:   # the first (untimed) step: the same input every step
            self._active = int((gm[:m] > 0).sum().item())
        d.update({"cg_iters": ainfo.iters, "cg_residual": ainfo.residual, "ms_adjoint": e0.elapsed_time(e1),
                  "launches": d["launches"] + ainfo.launches, "active": self._active})
        return GradJob.Out(d)

    def tune(self, T, ctx, x, q, f, precision):
        return T.tune_single(ctx, x, q, f, precision)

    def cpu(self, args):
        """The oracle's step and dense adjoint on a spatial sample (about 500
        rods: the dense adjoint holds (6n)^2 mobility entries)."""
        import oracle as O
        from oracle import adjoint as ADJ
        sub, a = spatial_sample(self.s, min(args.sample_rods, 500))
        from paper_2109_08206_gb300 import workloads as W
        T = W.loss_targets(sub)
        t0 = time.perf_counter()
        ADJ.loss_and_grad(sub.x, sub.quat, sub.f_nc, O.problem_of(sub), T)
        t = time.perf_counter() - t0
        return sub.n, t, (f"{sub.n} rods of {self.s.name} with centres in a periodic sub-cube of edge {a:.2f}; "
                          f"oracle step (exact or FISTA solve) and its dense adjoint, {t:.2f} s")

    def config(self, W, m):
        c = super().config(W, m)
        c["workload"] = self.name
        c["loss"] = "sum of squared post-step centre displacements from seeded targets (sigma 0.01)"
        return c


class SpringJob(SingleJob):
    """The 1e5-rod suspension with its 50,000 crosslinkers as bilateral
    spring constraints (aLENS_set_springs) instead of explicit forces."""

    graph = False

    def __init__(self, s, springs):
        super().__init__(s)
        self.sp = springs
        self.name = s.name + "_bilateral"
        self.nb = len(springs["kappa"])

    def context(self, A, precision, tol, stream):
        import torch
        p = A.params_of(self.s, precision=precision, tol=tol, max_iter=1_000_000)
        ctx = A.Context(p, self.n, 12 * self.n + self.nb, stream=stream)
        dev = torch.device("cuda", torch.cuda.current_device())
        sp = self.sp
        ctx.set_springs(torch.as_tensor(sp["ends"], dtype=torch.int32, device=dev),
                        torch.as_tensor(sp["arms"], device=dev), torch.as_tensor(sp["kappa"], device=dev),
                        torch.as_tensor(sp["rest"], device=dev))
        return ctx

    def solve_bytes(self, ctx, info, w):
        return info["iters"] * solve_bytes_per_iter(self.n, info["n_pairs"] + self.nb, w)

    def config(self, W, m):
        c = super().config(W, m)
        c.update({"workload": self.name, "springs": None, "bilateral_springs": self.nb,
                  "spring_model": "kappa 10, rest 1.5, attachment arclengths uniform"})
        return c

    def cpu(self, args):
        import oracle as O
        sub, a = spatial_sample(self.s, args.sample_rods)
        from paper_2109_08206_gb300 import workloads as W
        nb = max(1, int(round(self.nb * sub.n / self.n)))
        sp = W.spring_set(sub, nb, seed=21)
        t0 = time.perf_counter()
        O.step(sub.x, sub.quat, sub.f_nc, O.problem_of(sub), tol=args.tol, springs=sp)
        t = time.perf_counter() - t0
        return sub.n, t, (f"{sub.n} rods of {self.s.name} with centres in a periodic sub-cube of edge {a:.2f} and "
                          f"{nb} springs; one oracle step with the bilateral constraints, {t:.2f} s")


class TrajJob(SingleJob):
    """A Brownian trajectory of the 1e5-rod suspension: every timed call is
    aLENS_run over `steps_per_call` steps (kT = 1, Brownian forces drawn on
    the device, the workload's own forces held as f_ext, warm start)."""

    graph = False

    steps_per_call = 10

    class Out:
        def __init__(self, d):
            self.d = d

        def as_dict(self):
            return self.d

    def __init__(self, s):
        super().__init__(s)
        self.name = s.name + "_trajectory"

    def step(self, ctx, x, q, f, **kw):
        info, stats = ctx.run(x, q, self.steps_per_call, kT=1.0, seed=77, first_step=0, f_ext=f, warm_start=True,
                              check=False)
        d = info.as_dict()
        d["iters"] = info.iters / self.steps_per_call   # per constrained step
        d["stats"] = stats
        return TrajJob.Out(d)

    def solve_bytes(self, ctx, info, w):
        return sum(st["iters"] * solve_bytes_per_iter(self.n, st["n_pairs"], w) for st in info["stats"])

    def config(self, W, m):
        c = super().config(W, m)
        c.update({"workload": self.name, "steps_per_call": self.steps_per_call, "kT": 1.0,
                  "brownian": "Philox4x32-10 on the device, covariance 2 kT M^-1 / h", "warm_start": True})
        return c

    def cpu(self, args):
        import oracle as O
        sub, a = spatial_sample(self.s, min(args.sample_rods, 4000))
        K = 3
        t0 = time.perf_counter()
        O.trajectory(sub.x, sub.quat, O.problem_of(sub), K, 1.0, 77, f_ext=sub.f_nc, tol=args.tol)
        t = time.perf_counter() - t0
        return sub.n * K, t, (f"{sub.n} rods of {self.s.name} with centres in a periodic sub-cube of edge {a:.2f}; "
                              f"{K} oracle trajectory steps (Brownian forces, FISTA to {args.tol:g}), {t:.2f} s")


SEEDS = {"n1000_box40": 1, "n100k_phi010": 2, "n400k_nematic": 3, "n20k_phi015": 5}


def make_job(name, sibling=False):
    """The named workload; sibling=True draws another input of the same class
    (every seed shifted by 1000), on which the launch shape is tuned."""
    from paper_2109_08206_gb300 import workloads as W
    d = 1000 if sibling else 0
    if name == "n100k_traj":
        return TrajJob(W.workload("n100k_phi010", seed=2 + d))
    if name == "n100k_springs":
        s = W.workload("n100k_phi010", n_springs=0, seed=2 + d)
        return SpringJob(s, W.spring_set(s, 50_000, seed=21 + d))
    if name == "ensemble256":
        return BatchJob(W.ensemble(seed=1000 + d, count=256))
    if name == "n20k_grad":
        return GradJob(W.workload("n20k_phi015", seed=5 + d))
    return SingleJob(W.workload(name, seed=SEEDS[name] + d))


def oracle_step_time(s, tol, reps=1):
    import oracle as O
    pb = O.problem_of(s)
    times, out = [], None
    for _ in range(reps):
        t0 = time.perf_counter()
        out = O.step_native(s.x, s.quat, s.f_nc, pb, tol, 10_000_000, max(64, 30 * s.n))
        times.append(time.perf_counter() - t0)
    return statistics.median(times), out


def cpu_cores():
    try:
        return int(os.environ.get("OMP_NUM_THREADS") or len(os.sched_getaffinity(0)))
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    """The host CPU as lscpu names it (model, else vendor), and nproc."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        info = {}
        for l in out.splitlines():
            k, _, v = l.partition(":")
            info[k.strip()] = v.strip()
        name = info.get("Model name") or info.get("Vendor ID")
    except Exception:
        pass
    return name, os.cpu_count()


def cpu_baseline_record(job, args):
    """The oracle on the job's bounded CPU sample, median of 3 runs with all
    host cores and median of 3 (1 when a run exceeds 12 s) with one thread."""
    import oracle as O
    reps_all = 3
    times = []
    sample = None
    for _ in range(reps_all):
        rods, t, sample = job.cpu(args)
        times.append(t)
    t_all = statistics.median(times)
    before = O.set_threads(1)
    try:
        t1 = []
        for k in range(3):
            rods1, t, _ = job.cpu(args)
            t1.append(t)
            if t > 12.0:
                break
    finally:
        O.set_threads(before)
    model, nproc = cpu_model()
    return {"value": rods / t_all, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": sample + f"; median of {reps_all} runs on all cores",
            "single_thread": {"value": rods1 / statistics.median(t1), "runs": len(t1),
                              "s_per_step": statistics.median(t1)},
            "s_per_step": t_all, "nproc": nproc, "cpu_model": model}


def replica_time(ms_local, pg=None, device=None):
    """Step time of a replicas run: the slowest rank's (MAX all-reduce; the
    ranks run independent systems, so this is the only collective)."""
    if pg is None:
        return ms_local
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def replica_value(ms_step, rods_per_rank, world_size):
    """Whole-job rod-steps/s: rods of all ranks over the slowest rank's step time."""
    return world_size * rods_per_rank / (ms_step / 1e3)


# ------------------------------------------------------------ reference arm

def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    job = make_job(args.workload)
    for _ in range(max(0, min(args.warmup, 1))):
        job.cpu(args)
    times = []
    for _ in range(args.steps):
        rods, t, sample = job.cpu(args)
        times.append(t)
    t = statistics.mean(times)
    v = rods / t
    line = {"impl": "reference", "metric": metric_of(args.workload), "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload} (oracle on a {rods}-rod sample)", "rods": rods,
                       "tol": args.tol},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def run_ours(args):
    import torch
    import paper_2109_08206_gb300 as A
    from paper_2109_08206_gb300 import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    A.build()
    dev = torch.device("cuda", local)
    job = make_job(args.workload)
    n = job.n
    hx0, hq0, hf0 = job.arrays()
    stream = torch.cuda.Stream(device=dev)
    x0 = torch.as_tensor(hx0, device=dev)
    q0 = torch.as_tensor(hq0, device=dev)
    f = torch.as_tensor(hf0, device=dev)
    x, q = x0.clone(), q0.clone()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    max_pairs = 12 * n

    def make_ctx(precision):
        ctx = job.context(A, precision, args.tol, stream)
        if args.scaling is not None:
            ctx.set_scaling(args.scaling)
        if args.barriers is not None:
            ctx.set_solver_schedule(args.barriers)
        return ctx

    def timed(ctx, K, W_, host=None, w=4):
        """K timed steps after W_ warm-ups; returns per-step ms, infos and the
        algorithmic bytes of each step's BBPGD launch."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        infos, sbytes = [], []
        with torch.cuda.stream(stream):
            for k in range(W_ + K):
                if host is None:
                    x.copy_(x0); q.copy_(q0)
                flush.fill_(float(k))
                if k >= W_:
                    ev[k - W_][0].record(stream)
                if host is None:
                    info = job.step(ctx, x, q, f)
                else:
                    hx, hq, hf, ox, oq = host
                    x.copy_(hx, non_blocking=True); q.copy_(hq, non_blocking=True); f.copy_(hf, non_blocking=True)
                    info = job.step(ctx, x, q, f)
                    ox.copy_(x, non_blocking=True); oq.copy_(q, non_blocking=True)
                if k >= W_:
                    ev[k - W_][1].record(stream)
                    infos.append(info.as_dict())
                    sbytes.append(job.solve_bytes(ctx, infos[-1], w))
            stream.synchronize()
        return [a.elapsed_time(b) for a, b in ev], infos, sbytes

    def barrier():
        torch.cuda.synchronize()
        if pg is not None:
            pg.barrier()

    def max_over_ranks(v):
        return replica_time(v, pg, dev)

    # ---- untimed: the solver's launch shape, tuned on another input of the
    # same workload class (every seed shifted), so that the timed input is
    # not the one the shape was picked on; for a batch, the per-system
    # constraint counts
    import paper_2109_08206_gb300.autotune as T
    kind = "batch" if isinstance(job, BatchJob) else "single"
    default_shape = T.BATCH_CANDIDATES[0] if kind == "batch" else T.SINGLE_CANDIDATES[0]
    sib = None if (args.no_tune or args.shape) else make_job(args.workload, sibling=True)
    if args.shape:
        default_shape = tuple(int(v) for v in args.shape.lower().split("x"))

    def tune_on_sibling(precision):
        sx, sq, sf = (torch.as_tensor(v, device=dev) for v in sib.arrays())
        sctx = sib.context(A, precision, args.tol, stream)
        if args.scaling is not None:
            sctx.set_scaling(args.scaling)
        if args.barriers is not None:
            sctx.set_solver_schedule(args.barriers)
        try:
            return sib.tune(T, sctx, sx, sq, sf, precision)
        finally:
            sctx.close()

    head = A.FP64 if args.precision == "fp64" else A.MIXED
    wh = 8 if head == A.FP64 else 4   # bytes per working-precision value
    if head == A.FP64:
        args.skip_fp64 = True   # the headline is the float64 step itself
    ctx = make_ctx(head)
    if args.shape:
        T.apply(ctx, kind, default_shape)
    tuned = None
    if sib is not None:
        shape, times = tune_on_sibling(head)
        T.apply(ctx, kind, shape)
        tuned = {"shape": list(shape), "cost": times, "cost_unit": T.cost_unit(kind),
                 "tuned_on": f"{sib.name}, another seed of the same workload class"}
    shape_now = tuple(tuned["shape"]) if tuned else default_shape
    if isinstance(job, BatchJob):
        pr = torch.empty((max_pairs, 3), dtype=torch.int32, device=dev)
        xx, qq = x0.clone(), q0.clone()
        inf = job.step(ctx, xx, qq, f, pairs_out=pr)
        job.count_pairs(pr[: inf.n_pairs].cpu().numpy())
        del pr, xx, qq

    # ---- FP32-mixed: the headline
    barrier()
    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        gpu_id = gpu_id if gpu_id.startswith("GPU-") else "GPU-" + gpu_id
    except Exception:
        gpu_id = None
    clk = Clocks(gpu_id).__enter__()   # sampled across every timed region below
    t0 = time.perf_counter()
    ms, infos, sbytes = timed(ctx, args.steps, args.warmup, w=wh)
    barrier()
    wall = time.perf_counter() - t0
    ms_step = max_over_ranks(statistics.mean(ms))
    spc = getattr(job, "steps_per_call", 1)   # constrained steps in one timed call
    value = replica_value(ms_step, n * spc, ws)
    it = [i["iters"] for i in infos]
    ms_solve = statistics.mean(i["ms_solve"] for i in infos)
    m = infos[-1]["n_pairs"]
    res = max(i["residual"] for i in infos)
    launches = sum(i["launches"] for i in infos)
    b_iter = solve_bytes_per_iter(n, m, wh)
    alg_bytes = statistics.mean(sbytes)
    peak, peak_kind = peaks()
    achieved = alg_bytes / (ms_solve / 1e3) / 1e9
    solver = infos[-1].get("solver")
    tn = "double" if head == A.FP64 else "float"
    kernel = {1: f"k_bbpgd1<{tn}>", 2: f"k_bbpgd<{tn},1>", 3: f"k_bbpgd<{tn},0>",
              4: f"k_bbpgd_sys<{tn}>"}.get(solver, f"k_bbpgd<{tn}>")
    traffic = traffic_from_profile(ROOT / "paper_2109_08206_gb300" / "csrc" / "solve.cu", shape_now, kernel) \
        if args.workload == "n100k_phi010" else None   # the committed capture is of this workload
    # the whole step against the same peak: solve bytes plus the search,
    # assembly and update bytes (the adjoint's are not counted: no step fraction for it)
    step_bytes = alg_bytes + spc * step_other_bytes(n, m, wh)
    step_frac = None if isinstance(job, GradJob) else step_bytes / (ms_step / 1e3) / 1e9 / peak

    # ---- the library's default launch shape on the timed input (the
    # headline runs the shape tuned on the sibling input)
    default_run = None
    if tuned and tuple(tuned["shape"]) != tuple(default_shape):
        T.apply(ctx, kind, default_shape)
        msd, infd, _ = timed(ctx, max(3, args.steps // 2), 1, w=wh)
        T.apply(ctx, kind, shape_now)
        msd_step = max_over_ranks(statistics.mean(msd))
        default_run = {"shape": list(default_shape), "value": replica_value(msd_step, n * spc, ws),
                       "ms_per_step": msd_step, "bbpgd_iters": statistics.mean(i["iters"] for i in infd),
                       "ms_solve": statistics.mean(i["ms_solve"] for i in infd)}

    # ---- FP64 plain at the same residual
    fp64 = None
    if not args.skip_fp64:
        ctx64 = make_ctx(A.FP64)
        shape64 = default_shape
        if args.shape:
            T.apply(ctx64, kind, default_shape)
        if sib is not None:
            shape64, _ = tune_on_sibling(A.FP64)
            T.apply(ctx64, kind, shape64)
        ms64, inf64, sb64 = timed(ctx64, max(2, args.steps // 2), 1, w=8)
        ms64_step = max_over_ranks(statistics.mean(ms64))
        ms64_solve = statistics.mean(i["ms_solve"] for i in inf64)
        fp64 = {"value": replica_value(ms64_step, n * spc, ws), "unit": UNIT, "ms_per_step": ms64_step,
                "launch_shape": list(shape64),
                "solver_kernel": {1: "k_bbpgd1<double>", 2: "k_bbpgd<double,1>", 3: "k_bbpgd<double,0>",
                                  4: "k_bbpgd_sys<double>"}.get(inf64[-1].get("solver")),
                "roofline_frac": statistics.mean(sb64) / (ms64_solve / 1e3) / 1e9 / peak,
                "step_frac": None if isinstance(job, GradJob) else
                (statistics.mean(sb64) + spc * step_other_bytes(n, inf64[-1]["n_pairs"], 8))
                / (ms64_step / 1e3) / 1e9 / peak,
                "bbpgd_iters": statistics.mean(i["iters"] for i in inf64),
                **({"cg_iters": statistics.mean(i["cg_iters"] for i in inf64),
                    "ms_adjoint": statistics.mean(i["ms_adjoint"] for i in inf64)} if "cg_iters" in inf64[0] else {}),
                "residual": max(i["residual"] for i in inf64),
                "ms_solve": statistics.mean(i["ms_solve"] for i in inf64),
                "solve_bytes_per_launch": statistics.mean(sb64)}
        ctx64.close()

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.skip_e2e:
        hx = torch.as_tensor(hx0).pin_memory(); hq = torch.as_tensor(hq0).pin_memory()
        hf = torch.as_tensor(hf0).pin_memory()
        ox = torch.empty_like(hx).pin_memory(); oq = torch.empty_like(hq).pin_memory()
        mse, _, _ = timed(ctx, args.steps, 1, host=(hx, hq, hf, ox, oq))
        mse_step = max_over_ranks(statistics.mean(mse))
        e2e = {"value": replica_value(mse_step, n * spc, ws), "unit": UNIT, "ms_per_step": mse_step,
               "h2d_bytes_per_step": int(hx.numel() * 8 + hq.numel() * 8 + hf.numel() * 8),
               "d2h_bytes_per_step": int(ox.numel() * 8 + oq.numel() * 8)}
    clk.__exit__(None, None, None)

    # ---- the mixed step's deviation from the float64 step (outside the timed regions)
    mixed_vs_fp64 = None
    if not args.skip_fp64:
        outs = {}
        plain = type(job) is SingleJob
        for prec in (A.MIXED, A.FP64):
            c2 = make_ctx(prec)
            xx, qq = x0.clone(), q0.clone()
            gam = torch.empty(max_pairs, dtype=torch.float64, device=dev)
            kw = {"gamma_out": gam}
            if plain:
                kw["pairs_out"] = torch.empty((max_pairs, 3), dtype=torch.int32, device=dev)
            inf = SingleJob.step(job, c2, xx, qq, f, **kw) if isinstance(job, (GradJob, TrajJob)) \
                else job.step(c2, xx, qq, f, **kw)
            outs[prec] = (xx, qq, gam[: inf.n_pairs].clone(),
                          kw["pairs_out"][: inf.n_pairs].clone() if plain else None)
            c2.close()
        dx = outs[A.MIXED][0] - outs[A.FP64][0]
        boxt = torch.as_tensor(job.periodic_box(), device=dev)
        dx = dx - boxt * torch.round(dx / boxt)
        g32, g64 = outs[A.MIXED][2], outs[A.FP64][2]
        mixed_vs_fp64 = {"max_dx_over_D": float(dx.abs().max()),
                         "gamma_rel_l2": float(torch.linalg.norm(g32 - g64) / torch.linalg.norm(g64)),
                         "max_dquat": float((outs[A.MIXED][1] - outs[A.FP64][1]).abs().max())}
        if plain and rank == 0:
            # the float64 oracle's residual (rod diameters) of each step's
            # gamma, on its own assembly of the same pair list
            import oracle as O
            s = job.s
            pb = O.problem_of(s)
            for prec, key in ((A.MIXED, "oracle_residual_mixed"), (A.FP64, "oracle_residual_fp64")):
                pr_h = outs[prec][3].cpu().numpy()
                asm = O.assemble(s.x, s.quat, s.f_nc, pb, pr_h)
                _, r = O.gradient(s.quat, pb, pr_h, asm["dgeom"], asm["q"], outs[prec][2].cpu().numpy())
                mixed_vs_fp64[key] = float(r)
    ctx.close()

    if rank != 0:
        return
    cpu = None
    if not args.skip_cpu and ws == 1:
        cpu = cpu_baseline_record(job, args)
    config = job.config(W, m)
    config.update({"tol": args.tol, "scaling_beta": 0.5 if args.scaling is None else args.scaling,
                   "l2": "flushed (256 MB write) between steps; inputs restored outside the timed region",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"})
    line = {
        "metric": metric_of(args.workload), "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if head == A.FP64 else "f32-mixed (f64 geometry, reference passes and residual test)",
        "data": "synthetic",
        "config": config,
        "bbpgd_iters": statistics.mean(it), "residual": res, "launch_shape": tuned,
        "solver_kernel": {0: None, 1: "one grid barrier per iteration", 2: "two barriers, shared-memory shares",
                          3: "two barriers, global memory", 4: "per-system clusters"}.get(infos[-1].get("solver")),
        "phase_ms": {k: statistics.mean(i[k] for i in infos) for k in ("ms_build", "ms_assemble", "ms_solve",
                                                                         "ms_update", "ms_adjoint") if k in infos[0]},
        "adjoint": None if "cg_iters" not in infos[0] else {
            "cg_iters": statistics.mean(i["cg_iters"] for i in infos),
            "cg_residual": max(i["cg_residual"] for i in infos),
            "ms": statistics.mean(i["ms_adjoint"] for i in infos),
            "active_constraints": infos[0].get("active", m),
            "cg_bytes_per_iter": cg_bytes_per_iter(n, infos[0].get("active", m), 4),
            "cg_GBps_algorithmic": statistics.mean(i["cg_iters"] for i in infos)
                                   * cg_bytes_per_iter(n, infos[0].get("active", m), 4)
                                   / (statistics.mean(i["ms_adjoint"] for i in infos) / 1e3) / 1e9},
        "fp64": fp64, "e2e": e2e, "mixed_vs_fp64": mixed_vs_fp64,
        "roofline": {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "algorithmic_bytes_per_launch": alg_bytes, "bytes_per_iter": b_iter,
                     "step_frac": step_frac, "step_bytes": step_bytes},
        "default_shape": default_run,
        "cpu_baseline": cpu, "gpu_launches": launches, "clocks": clk.summary(), "wall_s": wall,
    }
    print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
