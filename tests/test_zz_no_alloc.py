"""The allocation-free solve (aLENS_solve_lcp_noalloc), called through the C ABI.

It serves callers that may not allocate device memory (a memory manager
owning the device budget, or a loop where cudaMalloc would stall other
work): its workspace is a static device array of the library.  Checked
against the context-based aLENS_solve_lcp on the same inputs, twice in a row
(the shared array keeps the previous call's contents), at its size limits
(4096 rods and 16384 constraints, where a slip in the workspace layout would
overrun the array), with the device's free memory unchanged across a call,
and for the sizes it rejects.  The file name makes pytest collect it last.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_2109_08206_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2109_08206_gb300 as A  # noqa: E402

MAX_RODS, MAX_PAIRS = 4096, 16384   # ALENS_NOALLOC_MAX_RODS / _PAIRS in include/alens.h


def noalloc_fn():
    L = A.lib()
    fn = L.aLENS_solve_lcp_noalloc
    vp, i64 = C.c_void_p, C.c_int64
    fn.restype = C.c_int32
    fn.argtypes = [C.POINTER(A.Params), i64, vp, i64, vp, vp, vp, vp, vp, C.POINTER(A.Info)]
    return fn


def ptr(t):
    return C.c_void_p(t.data_ptr())


def call_noalloc(params, quat, pairs, dgeom, q, gamma):
    info = A.Info()
    st = noalloc_fn()(C.byref(params), quat.shape[0], ptr(quat), pairs.shape[0], ptr(pairs), ptr(dgeom), ptr(q),
                      ptr(gamma), C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(info))
    torch.cuda.synchronize()
    return st, info


@pytest.fixture(scope="module")
def problem():
    A.build()
    s = W.workload("n1000_box40")
    pb = O.problem_of(s)
    pairs = O.find_pairs(s.x, s.quat, pb)
    asm = O.assemble(s.x, s.quat, s.f_nc, pb, pairs)
    dev = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    return s, pb, dev(s.quat), dev(pairs, torch.int32), dev(asm["dgeom"]), dev(asm["q"]), asm


@pytest.mark.parametrize("precision,tol,bar", [(A.FP64, 1e-8, 1e-5), (A.MIXED, 1e-6, 1e-3)])
def test_noalloc_matches_context_solve_twice(problem, precision, tol, bar):
    s, pb, quat, pairs, dgeom, q, asm = problem
    assert s.n <= MAX_RODS and pairs.shape[0] <= MAX_PAIRS
    params = A.params_of(s, precision=precision, tol=tol, max_iter=200000)
    with A.Context(params, s.n, 12 * s.n) as ctx:
        ref, rinfo = ctx.solve_lcp(quat, pairs, dgeom, q)
        ref = ref.cpu().numpy()
    for _ in range(2):
        gamma = torch.zeros(pairs.shape[0], dtype=torch.float64, device="cuda")
        st, info = call_noalloc(params, quat, pairs, dgeom, q, gamma)
        assert st == 0 and info.status == 0 and info.residual <= tol and info.iters > 0
        g = gamma.cpu().numpy()
        assert np.linalg.norm(g - ref) <= bar * np.linalg.norm(ref)
        _, r = O.gradient(s.quat, pb, pairs.cpu().numpy(), asm["dgeom"], asm["q"], g)
        assert r <= tol * 1.05 + (1e-9 if precision == A.FP64 else 2e-7)


def test_noalloc_rejects_sizes_beyond_its_limits(problem):
    s, pb, quat, pairs, dgeom, q, asm = problem
    params = A.params_of(s, precision=A.FP64, tol=1e-8)
    big = torch.zeros((MAX_RODS + 1, 4), dtype=torch.float64, device="cuda")
    gamma = torch.zeros(pairs.shape[0], dtype=torch.float64, device="cuda")
    st, _ = call_noalloc(params, big, pairs, dgeom, q, gamma)
    assert st == 2   # ALENS_ERR_CAPACITY
    assert np.all(gamma.cpu().numpy() == 0.0)


@pytest.fixture(scope="module")
def largest():
    """4096 rods and exactly 16384 constraints: the first 16384 pairs (in
    sorted order) of a seeded suspension dense enough to have more."""
    s = W.random_system(41, MAX_RODS, 64.0, forces="unit", tol=1e-8)
    pb = O.problem_of(s)
    pairs = O.find_pairs(s.x, s.quat, pb)
    assert pairs.shape[0] > MAX_PAIRS
    pairs = pairs[:MAX_PAIRS]
    asm = O.assemble(s.x, s.quat, s.f_nc, pb, pairs)
    dev = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    return s, pb, dev(s.quat), dev(pairs, torch.int32), dev(asm["dgeom"]), dev(asm["q"]), asm, pairs


@pytest.mark.parametrize("precision,tol,bar", [(A.FP64, 1e-8, 1e-5), (A.MIXED, 1e-6, 1e-3)])
def test_noalloc_at_its_limits_allocates_nothing(largest, precision, tol, bar):
    s, pb, quat, pairs, dgeom, q, asm, pairs_h = largest
    assert quat.shape[0] == MAX_RODS and pairs.shape[0] == MAX_PAIRS
    params = A.params_of(s, precision=precision, tol=tol, max_iter=200000)
    with A.Context(params, s.n, MAX_PAIRS) as ctx:
        ref, _ = ctx.solve_lcp(quat, pairs, dgeom, q)
        ref = ref.cpu().numpy()
    gammas = [torch.zeros(MAX_PAIRS, dtype=torch.float64, device="cuda") for _ in range(3)]
    torch.cuda.synchronize()
    st, _ = call_noalloc(params, quat, pairs, dgeom, q, gammas[0])   # loads whatever loads lazily
    assert st == 0
    for g in gammas[1:]:
        free0 = torch.cuda.mem_get_info()[0]
        st, info = call_noalloc(params, quat, pairs, dgeom, q, g)
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 == free0, (free0, free1)
        assert st == 0 and info.status == 0 and info.residual <= tol and info.iters > 0
        gh = g.cpu().numpy()
        assert np.linalg.norm(gh - ref) <= bar * np.linalg.norm(ref)
        _, r = O.gradient(s.quat, pb, pairs_h, asm["dgeom"], asm["q"], gh)
        assert r <= tol * 1.05 + (1e-9 if precision == A.FP64 else 2e-7)


def test_noalloc_rejects_one_pair_too_many(largest):
    s, pb, quat, pairs, dgeom, q, asm, pairs_h = largest
    params = A.params_of(s, precision=A.FP64, tol=1e-8)
    more = torch.cat([pairs, pairs[-1:]])
    d2 = torch.cat([dgeom, dgeom[-1:]])
    q2 = torch.cat([q, q[-1:]])
    gamma = torch.zeros(MAX_PAIRS + 1, dtype=torch.float64, device="cuda")
    st, _ = call_noalloc(params, quat, more, d2, q2, gamma)
    assert st == 2   # ALENS_ERR_CAPACITY, before any work is queued
    assert np.all(gamma.cpu().numpy() == 0.0)
