"""GB300 library for the hard-body collision-constraint step of aLENS
(Yan et al., arXiv 2109.08206): cell-list neighbours, segment-segment
constraint assembly, BBPGD complementarity solve and the rod update, as
hand-written CUDA kernels for sm_103a behind the C ABI of ``include/alens.h``.

This module is argument marshalling only: it loads ``_build/libalens.so``
with ctypes and passes raw device pointers of torch tensors (PyTorch is used
for device memory and streams).  Every step of the computation runs in the
library's kernels; there is no CPU fallback, and importing the bindings
fails loudly when the library has not been built (run ``build()``).
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

__all__ = ["build", "lib", "Params", "Info", "System", "Context", "BatchSpec", "AlensError", "FP64", "MIXED", "STATUS"]

_PKG = Path(__file__).resolve().parent
_LIB_PATH = _PKG / "_build" / "libalens.so"

FP64, MIXED = 0, 1
STATUS = {0: "OK", 1: "INVALID", 2: "CAPACITY", 3: "NOT_CONVERGED", 4: "TIMEOUT", 5: "CUDA", 6: "NOMEM",
          7: "NOT_IMPLEMENTED"}


class Params(C.Structure):
    """aLENS_params (include/alens.h)."""
    _fields_ = [("box", C.c_double * 3), ("diameter", C.c_double), ("length", C.c_double),
                ("viscosity", C.c_double), ("dt", C.c_double), ("delta_c", C.c_double), ("tol", C.c_double),
                ("max_iter", C.c_int32), ("precision", C.c_int32)]


class Info(C.Structure):
    """aLENS_info (include/alens.h)."""
    _fields_ = [("n_pairs", C.c_int64), ("n_overlap", C.c_int64), ("iters", C.c_int32), ("status", C.c_int32),
                ("residual", C.c_double), ("min_gap", C.c_double), ("ms_build", C.c_float),
                ("ms_assemble", C.c_float), ("ms_solve", C.c_float), ("ms_update", C.c_float),
                ("launches", C.c_int32), ("solver", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class StepStats(C.Structure):
    """aLENS_step_stats (include/alens.h): one step of a trajectory."""
    _fields_ = [("n_pairs", C.c_int64), ("n_walls", C.c_int64), ("iters", C.c_int32), ("status", C.c_int32),
                ("residual", C.c_double), ("min_gap", C.c_double), ("ms_step", C.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class System(C.Structure):
    """aLENS_system (include/alens.h): one system of a batch."""
    _fields_ = [("box", C.c_double * 3), ("length", C.c_double)]


class AlensError(RuntimeError):
    def __init__(self, status: int, where: str, extra=None):
        self.status = status
        self.extra = extra
        msg = f"{where}: {STATUS.get(status, status)} ({_status_string(status)})"
        if isinstance(extra, dict) and "iters" in extra:
            msg += f" iters={extra['iters']} residual={extra['residual']:.3e} n_pairs={extra['n_pairs']}"
        if status == 5:   # ALENS_ERR_CUDA: the runtime error behind it
            try:
                msg += f" [{lib().aLENS_last_cuda_error().decode()}]"
            except Exception:
                pass
        super().__init__(msg)


def build(force: bool = False, verbose: bool = False) -> Path:
    """Compile the CUDA library for sm_103a (see nvcc_build.py)."""
    from . import nvcc_build
    return nvcc_build.build(force=force, verbose=verbose)


_lib = None


def lib():
    """The loaded C library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not _LIB_PATH.exists():
            raise RuntimeError(f"CUDA library missing: {_LIB_PATH} (call paper_2109_08206_gb300.build())")
        L = C.CDLL(str(_LIB_PATH))
        vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        PP, IP = C.POINTER(Params), C.POINTER(Info)
        sig = {
            "aLENS_create": (i32, [PP, i64, i64, vp, C.POINTER(vp)]),
            "aLENS_destroy": (None, [vp]),
            "aLENS_set_params": (i32, [vp, PP]),
            "aLENS_status_string": (C.c_char_p, [i32]),
            "aLENS_build_neighbors": (i32, [vp, i64, vp, vp, vp, i64, C.POINTER(i64)]),
            "aLENS_assemble_constraints": (i32, [vp, i64, vp, vp, vp, i64, vp, vp, vp, vp]),
            "aLENS_solve_lcp": (i32, [vp, i64, vp, i64, vp, vp, vp, vp, IP]),
            "aLENS_step": (i32, [vp, i64, vp, vp, vp, vp, vp, vp, IP]),
            "aLENS_step_batch": (i32, [vp, i32, C.POINTER(System), C.POINTER(i64), vp, vp, vp, vp, vp, vp, IP]),
            "aLENS_batch_results": (i32, [vp, i32, vp, vp]),
            "aLENS_batch_groups": (i32, [vp, i32, vp]),
            "aLENS_step_adjoint": (i32, [vp, i64, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp,
                                         C.POINTER(d), IP]),
            "aLENS_set_batch_launch": (i32, [vp, i32, i32]),
            "aLENS_set_springs": (i32, [vp, i64, vp, vp, vp, vp]),
            "aLENS_set_walls": (i32, [vp, i32, d, d]),
            "aLENS_brownian": (i32, [vp, i64, vp, d, C.c_uint64, i64, vp, vp]),
            "aLENS_random_words": (i32, [vp, i64, C.c_uint64, i64, vp]),
            "aLENS_run": (i32, [vp, i64, vp, vp, vp, i64, d, C.c_uint64, i64, i32, C.POINTER(StepStats), IP]),
            "aLENS_set_wait_limit": (i32, [vp, d]),
            "aLENS_set_scaling": (i32, [vp, d]),
            "aLENS_inject_fault": (i32, [vp, i32]),
            "aLENS_set_launch": (i32, [vp, i32, i32]),
            "aLENS_set_solver_schedule": (i32, [vp, i32]),
            "aLENS_set_batch_graph": (i32, [vp, i32]),
            "aLENS_set_step_graph": (i32, [vp, i32]),
            "aLENS_set_l2_window": (i32, [vp, i32]),
            "aLENS_last_cuda_error": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    """Names declared by include/alens.h (parsed from the header)."""
    import re
    text = (_PKG.parent / "include" / "alens.h").read_text()
    return sorted(set(re.findall(r"\b(aLENS_[a-z0-9_]+)\s*\(", text)))


def _status_string(s: int) -> str:
    try:
        return lib().aLENS_status_string(int(s)).decode()
    except Exception:
        return "?"


def make_params(box, diameter=1.0, length=10.0, viscosity=1.0, dt=1e-3, delta_c=None, tol=1e-8,
                max_iter=100000, precision=FP64) -> Params:
    b = box if hasattr(box, "__len__") else (box, box, box)
    return Params((C.c_double * 3)(*[float(v) for v in b]), float(diameter), float(length), float(viscosity),
                  float(dt), float(diameter if delta_c is None else delta_c), float(tol), int(max_iter),
                  int(precision))


def params_of(sys, precision=FP64, tol=None, max_iter=100000) -> Params:
    """Params of a ``workloads.RodSystem``."""
    return make_params(sys.box, sys.diameter, sys.length, sys.viscosity, sys.dt, sys.delta_c,
                       sys.tol if tol is None else tol, max_iter, precision)


def _ptr(t, dtype, shape_tail=None):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"expected a contiguous {dtype} tensor, got {t.dtype}")
    if shape_tail is not None and tuple(t.shape[1:]) != tuple(shape_tail):
        raise ValueError(f"expected shape [*, {shape_tail}], got {tuple(t.shape)}")
    return C.c_void_p(t.data_ptr())


class BatchSpec:
    """The C tables of a batch (aLENS_system array and rod offsets), built
    once for repeated Context.step_batch calls on the same systems."""

    def __init__(self, systems, rod_offset):
        ns = len(systems)
        if len(rod_offset) != ns + 1:
            raise ValueError("rod_offset needs n_systems + 1 entries")
        self.n_systems = ns
        self.tab = (System * ns)()
        for s, (box, length) in enumerate(systems):
            b = box if hasattr(box, "__len__") else (box, box, box)
            self.tab[s] = System((C.c_double * 3)(*[float(v) for v in b]), float(length))
        self.off = (C.c_int64 * (ns + 1))(*[int(v) for v in rod_offset])


class Context:
    """One aLENS_ctx: workspaces for up to max_rods rods and max_pairs constraints,
    bound to a CUDA stream (default: torch's current stream at creation)."""

    def __init__(self, params: Params, max_rods: int, max_pairs: int, stream=None):
        import torch
        self._lib = lib()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.params = params
        self.max_rods, self.max_pairs = int(max_rods), int(max_pairs)
        h = C.c_void_p()
        st = self._lib.aLENS_create(C.byref(params), self.max_rods, self.max_pairs,
                                    C.c_void_p(stream.cuda_stream), C.byref(h))
        if st != 0:
            raise AlensError(st, "aLENS_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.aLENS_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -------------------------------------------------------------- settings
    def set_params(self, params: Params):
        st = self._lib.aLENS_set_params(self._h, C.byref(params))
        if st != 0:
            raise AlensError(st, "aLENS_set_params")
        self.params = params

    def set_wait_limit(self, seconds: float):
        st = self._lib.aLENS_set_wait_limit(self._h, float(seconds))
        if st != 0:
            raise AlensError(st, "aLENS_set_wait_limit")

    def set_scaling(self, beta: float):
        """Diagonal scaling exponent of the BBPGD iteration (0 = unscaled)."""
        st = self._lib.aLENS_set_scaling(self._h, float(beta))
        if st != 0:
            raise AlensError(st, "aLENS_set_scaling")

    def inject_fault(self, mode: int):
        st = self._lib.aLENS_inject_fault(self._h, int(mode))
        if st != 0:
            raise AlensError(st, "aLENS_inject_fault")

    def set_launch(self, threads: int, blocks_per_sm: int = 0):
        st = self._lib.aLENS_set_launch(self._h, int(threads), int(blocks_per_sm))
        if st != 0:
            raise AlensError(st, "aLENS_set_launch")

    def set_solver_schedule(self, barriers: int):
        """1: one grid barrier per BBPGD iteration where it fits (default); 2: two."""
        st = self._lib.aLENS_set_solver_schedule(self._h, int(barriers))
        if st != 0:
            raise AlensError(st, "aLENS_set_solver_schedule")

    # ------------------------------------------------------------ entry points
    def build_neighbors(self, x, quat, pairs=None):
        """Sorted pair list [m, 3] int32 (i, j, image) on the device."""
        import torch
        n = x.shape[0]
        if pairs is None:
            pairs = torch.empty((self.max_pairs, 3), dtype=torch.int32, device=x.device)
        cnt = C.c_int64()
        st = self._lib.aLENS_build_neighbors(self._h, n, _ptr(x, torch.float64, (3,)), _ptr(quat, torch.float64, (4,)),
                                             _ptr(pairs, torch.int32, (3,)), pairs.shape[0], C.byref(cnt))
        if st != 0:
            raise AlensError(st, "aLENS_build_neighbors", cnt.value)
        return pairs[:cnt.value]

    def assemble_constraints(self, x, quat, f_nc, pairs):
        """(phi [m], dgeom [m, 9], q [m]) float64 on the device."""
        import torch
        n, m = x.shape[0], pairs.shape[0]
        dev = x.device
        phi = torch.empty(m, dtype=torch.float64, device=dev)
        dgeom = torch.empty((m, 9), dtype=torch.float64, device=dev)
        q = torch.empty(m, dtype=torch.float64, device=dev)
        st = self._lib.aLENS_assemble_constraints(
            self._h, n, _ptr(x, torch.float64, (3,)), _ptr(quat, torch.float64, (4,)),
            _ptr(f_nc, torch.float64, (6,)), m, _ptr(pairs.contiguous(), torch.int32, (3,)),
            _ptr(phi, torch.float64), _ptr(dgeom, torch.float64, (9,)), _ptr(q, torch.float64))
        if st != 0:
            raise AlensError(st, "aLENS_assemble_constraints")
        return phi, dgeom, q

    def solve_lcp(self, quat, pairs, dgeom, q, gamma=None, check=True):
        """BBPGD solve; returns (gamma [m] float64, Info)."""
        import torch
        m = pairs.shape[0]
        if gamma is None:
            gamma = torch.zeros(m, dtype=torch.float64, device=quat.device)
        info = Info()
        st = self._lib.aLENS_solve_lcp(self._h, quat.shape[0], _ptr(quat, torch.float64, (4,)), m,
                                       _ptr(pairs.contiguous(), torch.int32, (3,)), _ptr(dgeom, torch.float64, (9,)),
                                       _ptr(q, torch.float64), _ptr(gamma, torch.float64), C.byref(info))
        if check and st != 0:
            raise AlensError(st, "aLENS_solve_lcp", info.as_dict())
        return gamma, info

    def step(self, x, quat, f_nc, pairs_out=None, gamma_out=None, vel_out=None, check=True):
        """One constrained step in place on x, quat (device float64).  Returns Info."""
        import torch
        info = Info()
        st = self._lib.aLENS_step(self._h, x.shape[0], _ptr(x, torch.float64, (3,)), _ptr(quat, torch.float64, (4,)),
                                  _ptr(f_nc, torch.float64, (6,)), _ptr(pairs_out, torch.int32, (3,)),
                                  _ptr(gamma_out, torch.float64), _ptr(vel_out, torch.float64, (6,)), C.byref(info))
        if check and st != 0:
            raise AlensError(st, "aLENS_step", info.as_dict())
        return info

    def step_batch(self, systems, rod_offset, x, quat, f_nc, pairs_out=None, gamma_out=None, vel_out=None,
                   check=True):
        """One constrained step of a batch of independent systems, in place on x, quat.

        ``systems``: sequence of (box, length) with box a 3-sequence or a scalar;
        ``rod_offset``: n_systems + 1 integers, system s owning rods
        [rod_offset[s], rod_offset[s+1]).  Or ``systems`` = a BatchSpec of
        both (``rod_offset`` then ignored), which saves rebuilding the C
        tables on every call.  Returns Info (aggregated over the batch).
        """
        import torch
        spec = systems if isinstance(systems, BatchSpec) else BatchSpec(systems, rod_offset)
        ns, tab, off = spec.n_systems, spec.tab, spec.off
        info = Info()
        st = self._lib.aLENS_step_batch(self._h, ns, tab, off, _ptr(x, torch.float64, (3,)),
                                        _ptr(quat, torch.float64, (4,)), _ptr(f_nc, torch.float64, (6,)),
                                        _ptr(pairs_out, torch.int32, (3,)), _ptr(gamma_out, torch.float64),
                                        _ptr(vel_out, torch.float64, (6,)), C.byref(info))
        if check and st != 0:
            raise AlensError(st, "aLENS_step_batch", info.as_dict())
        return info

    def batch_results(self, n_systems: int):
        """(iters [S] int32, residual [S] float64) numpy arrays of the last step_batch."""
        import numpy as np
        it = np.zeros(n_systems, dtype=np.int32)
        res = np.zeros(n_systems, dtype=np.float64)
        st = self._lib.aLENS_batch_results(self._h, int(n_systems), it.ctypes.data_as(C.c_void_p),
                                           res.ctypes.data_as(C.c_void_p))
        if st != 0:
            raise AlensError(st, "aLENS_batch_results")
        return it, res

    def batch_groups(self, n_systems: int):
        """Blocks that solved each system of the last step_batch (int32 [S])."""
        import numpy as np
        b = np.zeros(n_systems, dtype=np.int32)
        st = self._lib.aLENS_batch_groups(self._h, int(n_systems), b.ctypes.data_as(C.c_void_p))
        if st != 0:
            raise AlensError(st, "aLENS_batch_groups")
        return b

    def set_batch_graph(self, enable: bool = True):
        """Record aLENS_step_batch as a CUDA graph and replay it (see include/alens.h)."""
        st = self._lib.aLENS_set_batch_graph(self._h, int(bool(enable)))
        if st != 0:
            raise AlensError(st, "aLENS_set_batch_graph")

    def set_step_graph(self, enable: bool = True):
        """Record aLENS_step as a CUDA graph and replay it (see include/alens.h)."""
        st = self._lib.aLENS_set_step_graph(self._h, int(bool(enable)))
        if st != 0:
            raise AlensError(st, "aLENS_set_step_graph")

    def set_l2_window(self, enable: bool = True):
        """L2 residency of the global-memory solver's states (see include/alens.h)."""
        st = self._lib.aLENS_set_l2_window(self._h, int(bool(enable)))
        if st != 0:
            raise AlensError(st, "aLENS_set_l2_window")

    def set_batch_launch(self, threads: int, cluster_blocks: int):
        st = self._lib.aLENS_set_batch_launch(self._h, int(threads), int(cluster_blocks))
        if st != 0:
            raise AlensError(st, "aLENS_set_batch_launch")

    def step_adjoint(self, x, quat, f_nc, pairs, gamma, dL_dx_new=None, dL_dquat_new=None, check=True):
        """Gradient of a loss of the post-step state through one aLENS_step.

        x, quat, f_nc: the state the forward step started from; pairs, gamma:
        its pairs_out and gamma_out (device, first n_pairs rows).  Returns
        (dL/dx [n,3], dL/dquat [n,4] (tangent), dL/dF_nc [n,6], dL/deta, Info).
        """
        import torch
        n, m = x.shape[0], pairs.shape[0]
        gx = torch.empty((n, 3), dtype=torch.float64, device=x.device)
        gq = torch.empty((n, 4), dtype=torch.float64, device=x.device)
        gf = torch.empty((n, 6), dtype=torch.float64, device=x.device)
        geta = C.c_double()
        info = Info()
        st = self._lib.aLENS_step_adjoint(
            self._h, n, _ptr(x, torch.float64, (3,)), _ptr(quat, torch.float64, (4,)),
            _ptr(f_nc, torch.float64, (6,)), m, _ptr(pairs.contiguous(), torch.int32, (3,)),
            _ptr(gamma.contiguous(), torch.float64), _ptr(dL_dx_new, torch.float64, (3,)),
            _ptr(dL_dquat_new, torch.float64, (4,)), _ptr(gx, torch.float64, (3,)), _ptr(gq, torch.float64, (4,)),
            _ptr(gf, torch.float64, (6,)), C.byref(geta), C.byref(info))
        if check and st != 0:
            raise AlensError(st, "aLENS_step_adjoint", info.as_dict())
        return gx, gq, gf, geta.value, info

    def set_springs(self, ends=None, arms=None, kappa=None, rest=None):
        """Bilateral springs solved with every later step (device tensors:
        ends [nb, 2] int32, arms [nb, 2], kappa [nb], rest [nb] float64);
        no arguments removes them."""
        import torch
        nb = 0 if ends is None else int(ends.shape[0])
        st = self._lib.aLENS_set_springs(
            self._h, nb, _ptr(None if nb == 0 else ends.contiguous(), torch.int32, (2,)),
            _ptr(None if nb == 0 else arms.contiguous(), torch.float64, (2,)),
            _ptr(None if nb == 0 else kappa.contiguous(), torch.float64),
            _ptr(None if nb == 0 else rest.contiguous(), torch.float64))
        if st != 0:
            raise AlensError(st, "aLENS_set_springs")
        self._springs = (ends, arms, kappa, rest) if nb > 0 else None   # keep the caller's tensors alive

    def set_walls(self, axis: int = -1, lo: float = 0.0, hi: float = 0.0):
        """Two flat confining walls normal to `axis` at lo < hi (axis -1 removes them)."""
        st = self._lib.aLENS_set_walls(self._h, int(axis), float(lo), float(hi))
        if st != 0:
            raise AlensError(st, "aLENS_set_walls")

    def brownian(self, quat, kT: float, seed: int, step: int, f_ext=None):
        """[n, 6] non-constraint force of trajectory step `step` (f_ext + Brownian)."""
        import torch
        out = torch.empty((quat.shape[0], 6), dtype=torch.float64, device=quat.device)
        st = self._lib.aLENS_brownian(self._h, quat.shape[0], _ptr(quat, torch.float64, (4,)), float(kT), int(seed),
                                      int(step), _ptr(f_ext, torch.float64, (6,)), _ptr(out, torch.float64, (6,)))
        if st != 0:
            raise AlensError(st, "aLENS_brownian")
        return out

    def random_words(self, n: int, seed: int, step: int):
        """[n, 8] int32 view of the generator's raw 32-bit words (device)."""
        import torch
        out = torch.empty((n, 8), dtype=torch.int32, device="cuda")
        st = self._lib.aLENS_random_words(self._h, int(n), int(seed), int(step), C.c_void_p(out.data_ptr()))
        if st != 0:
            raise AlensError(st, "aLENS_random_words")
        return out

    def run(self, x, quat, n_steps: int, kT: float, seed: int, first_step: int = 0, f_ext=None,
            warm_start: bool = True, check=True):
        """n_steps Brownian constrained steps in place; returns (Info, [StepStats dicts])."""
        import torch
        stats = (StepStats * max(int(n_steps), 1))()
        info = Info()
        st = self._lib.aLENS_run(self._h, x.shape[0], _ptr(x, torch.float64, (3,)), _ptr(quat, torch.float64, (4,)),
                                 _ptr(f_ext, torch.float64, (6,)), int(n_steps), float(kT), int(seed),
                                 int(first_step), int(bool(warm_start)), stats, C.byref(info))
        if check and st != 0:
            raise AlensError(st, "aLENS_run", info.as_dict())
        return info, [stats[k].as_dict() for k in range(int(n_steps))]
