// Barzilai-Borwein projected gradient descent (BBPGD) on the CQP
//     min_gamma  1/2 gamma^T (D^T M D) gamma + q^T gamma,   gamma >= 0
// (Appendix Eq. suppcqpdef; Section "Instantiation in a massively parallel
// computing environment": each iteration costs one gradient
// grad f = D^T M D gamma + q, i.e. O(N_u) work).
//
// The paper defers the details of its BBPGD to earlier work, so the
// iteration follows the published projected BB method (Barzilai & Borwein
// 1988; projected form as in Dai & Fletcher 2005):
//   gamma_{k+1} = max(0, gamma_k - alpha_k g_k),
//   s_k = gamma_{k+1} - gamma_k, y_k = g_{k+1} - g_k (= A s_k),
//   alpha_{k+1} from the pair (s_{k-1}, y_{k-1}) of the iteration before,
//     s.s / s.y and s.y / y.y in turn (alternating BB1/BB2): the
//     Barzilai-Borwein step taken one iteration late, a gradient method with
//     retards (Friedlander, Martinez, Molina & Raydan, SIAM J. Numer. Anal.
//     36, 1999), which lets the one-barrier solver below form the step
//     length from sums that arrive with the next barrier; every solver kernel
//     uses it, so all of them run one method;
//   alpha_0 = pi.pi / pi.A.pi for the projected gradient pi at gamma_0, for
//   the first two steps and whenever s.y <= 0 or the step is not finite.
// Stop when (h/D) max |pi_c| <= tol (pi the projected gradient) or after
// max_iter iterations.
//
// One persistent cooperative kernel runs the whole loop, one block per SM.
// Rods are numbered in cell order; block b owns an even share of rods
// [r0, r1) and the constraints they own [c0, c1) (owner = lower-ranked end).
// When they fit, the block keeps its own constraints' records, q, gamma and
// g, and its rods' axes and velocities in shared memory for the whole solve
// (at 1e5 rods the mixed working set, about 30 MB, spreads over the SMs'
// shared memory); global memory then carries what other blocks read: the
// velocities, and the state of constraints whose other rod is another
// block's (the rest of the state is written once when the solve ends).
// Without that fit every block works from the global arrays.  Per
// iteration:
//   phase A (one thread per rod, rods taken in ascending order of their
//     entry counts so that a warp's loops have similar lengths):
//     delta_{k+1} of every constraint touching the rod is formed on the fly
//     from (delta_k, g_k, gamma_ref) and alpha_k, summed into the rod's
//     force and torque F = D delta (owned range contiguous, other-side list
//     in CSR order), and dU = M F is stored;
//   grid barrier;
//   phase B (one thread per owned constraint): delta_{k+1} again (same
//     inputs and rounding), g_{k+1} = gref + D^T dU, and the partial sums
//     s.s, s.y, y.y and max |pi| (per thread, per warp and per block in a
//     fixed order);
//   grid barrier; warps 0-3 of every block then reduce the per-block
//     partials in the same fixed order, so all blocks take identical step
//     decisions.
// Two grid barriers per iteration.  Each barrier wait is bounded in time
// and in polls; a wait that runs out raises ALENS_ERR_TIMEOUT in the device
// status word and every block leaves.
//
// Global layout: the state (delta, g, gamma_ref, gamma_lo) of each
// constraint in two ping-pong [m][4] buffers, U as [rod][6], D records SoA
// [9][m] in owner-major order.
// T = double (float64 plain) or float (mixed: the D, M, D^T work, the sums
// and the step sizes in float32).  max |pi| is exact in either, and the
// stopping test takes the float64 decision (h/D) max |pi| <= tol in both:
// in float32 as max |pi| <= pi_tol, the largest float for which the float64
// product stays within tol.  The per-iteration reductions and decisions stay
// off float64 in the mixed solver because this part's float64 latency is
// about ten times float32's (an add 62 cycles, a divide 561).
#include <cooperative_groups.h>
#include <float.h>

#include <cmath>
#include <limits>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace alens {

// CSR entries whose loads a thread issues together (float64 values need the
// registers twice over)
template <typename T> struct Batch { static constexpr int v = 1; };
constexpr int kRefresh = 64;   // float32 iterations between reference refreshes

template <typename T> struct V2;
template <> struct V2<float> { using t = float2; };
template <> struct V2<double> { using t = double2; };

template <typename T>
__device__ __forceinline__ void ld_pair(const T* p, int c, T& a, T& b)
{
    typename V2<T>::t v = reinterpret_cast<const typename V2<T>::t*>(p)[c];
    a = v.x;
    b = v.y;
}

template <typename T>
__device__ __forceinline__ void ld_u6(const T* U, int i, T u[6])
{
    const typename V2<T>::t* p = reinterpret_cast<const typename V2<T>::t*>(U + 6 * (size_t)i);
    typename V2<T>::t a = p[0], b = p[1], c = p[2];
    u[0] = a.x; u[1] = a.y; u[2] = b.x; u[3] = b.y; u[4] = c.x; u[5] = c.y;
}

// Other-side arms of CSR entry k, packed as [m][8] (e, arm x e, 2 pad).
__device__ __forceinline__ void ld_arm(const float* qe, int k, float v[6])
{
    const float4 a = __ldg(reinterpret_cast<const float4*>(qe) + 2 * (size_t)k);
    const float2 b = __ldg(reinterpret_cast<const float2*>(qe) + 4 * (size_t)k + 2);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y;
}
__device__ __forceinline__ void ld_arm(const double* qe, int k, double v[6])
{
    const double2* p = reinterpret_cast<const double2*>(qe) + 4 * (size_t)k;
    const double2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
}

template <typename T>
__device__ __forceinline__ void st_u6(T* U, int i, const T u[6])
{
    typename V2<T>::t* p = reinterpret_cast<typename V2<T>::t*>(U + 6 * (size_t)i);
    typename V2<T>::t a, b, c;
    a.x = u[0]; a.y = u[1]; b.x = u[2]; b.y = u[3]; c.x = u[4]; c.y = u[5];
    p[0] = a; p[1] = b; p[2] = c;
}

// Constraint state (delta, g, gamma_ref, gamma_lo) of constraint c in a
// [m][4] buffer: one vector load (float32) or two (float64).  The iterate
// is gamma = gamma_ref + gamma_lo + delta: in float32 (gamma_ref, gamma_lo)
// is an unevaluated sum carrying about 48 bits (gamma_lo is 0 in float64).
__device__ __forceinline__ void ld_state(const float* p, int c, float& d, float& g, float& gr, float& gl)
{
    const float4 v = reinterpret_cast<const float4*>(p)[c];
    d = v.x; g = v.y; gr = v.z; gl = v.w;
}
__device__ __forceinline__ void ld_state(const double* p, int c, double& d, double& g, double& gr, double& gl)
{
    const double2* q = reinterpret_cast<const double2*>(p) + 2 * (size_t)c;
    const double2 a = q[0], b = q[1];
    d = a.x; g = a.y; gr = b.x; gl = b.y;
}
__device__ __forceinline__ float gl_of_state(const float* p, int c) { return p[4 * (size_t)c + 3]; }
__device__ __forceinline__ double gl_of_state(const double* p, int c) { return p[4 * (size_t)c + 3]; }

// (delta, g) and (gamma_ref, gamma_lo) halves of a state
template <typename T>
__device__ __forceinline__ void st_dg(T* p, int c, T d, T g)
{
    typename V2<T>::t v;
    v.x = d; v.y = g;
    reinterpret_cast<typename V2<T>::t*>(p)[2 * (size_t)c] = v;
}
template <typename T>
__device__ __forceinline__ void st_ref(T* p, int c, T gr, T gl)
{
    typename V2<T>::t v;
    v.x = gr; v.y = gl;
    reinterpret_cast<typename V2<T>::t*>(p)[2 * (size_t)c + 1] = v;
}

// Exact sum: a + b = s + e.
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T& s, T& e)
{
    s = a + b;
    const T bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Sum-of-products accumulator.  COMP (float32 reference passes): an
// unevaluated (hi, lo) pair fed by error-free transformations - the product
// split through one FMA, the sum through TwoSum - so large contact forces
// that cancel on a rod, or q and D^T U that cancel in a gradient entry, lose
// no digits.  Otherwise a plain sum.
template <typename T, bool COMP>
struct Acc {
    T hi, lo;
    __device__ __forceinline__ void init(T v) { hi = v; lo = T(0); }
    __device__ __forceinline__ void add_prod(T a, T b)
    {
        if (!COMP) {
            hi += a * b;
        } else {
            const T p = a * b;
            const T ep = fma(a, b, -p);
            T sum, es;
            two_sum(hi, p, sum, es);
            hi = sum;
            lo += es + ep;
        }
    }
    // a term far below hi (a product with a low part): into lo directly
    __device__ __forceinline__ void add_lo(T x) { lo += x; }
    __device__ __forceinline__ T value() const { return COMP ? hi + lo : hi; }
};

template <typename T>
struct SolveArgs {
    int n, m, np, mp;
    const int* __restrict__ rowP;
    const int* __restrict__ rowQ;
    const int* __restrict__ qlist;
    const int* __restrict__ ci;
    const int* __restrict__ cj;
    const T* __restrict__ rec;
    const T* __restrict__ qe;
    const T* __restrict__ q;
    const T* __restrict__ ax;
    T* gg0;     // [m][4] (delta, g, gamma_ref, 0): written inside the kernel, plain (coherent) loads only
    T* gg1;
    T* U;       // [n][6] velocity increment M D delta
    T* U2;      // [n][6] second increment buffer (one-barrier solver)
    T* Uref;    // [n][6] reference velocity M D gamma_ref
    T* gref;    // [m] reference gradient q + D^T Uref (blocks working from global memory)
    double* partials;
    unsigned* bar;
    int* flags;
    double* out;   // [0] residual, [1] alpha0
    T inv_perp, inv_par, inv_rot, inv_spin;
    const T* __restrict__ mobr;   // [4][np] per-rod inverse drags (batches), or NULL for the uniform ones
    const T* __restrict__ comp;   // [mp] per constraint: < 0 collision, >= 0 spring compliance 1/(h kappa); NULL: all collisions
    const T* __restrict__ rec_lo; // float32: low parts of rec, qe and q for the reference passes (else NULL)
    const T* __restrict__ qe_lo;
    const T* __restrict__ pe;   // [mp][8] owner-side records (null: read rec)
    const T* __restrict__ q_lo;
    const T* __restrict__ lop;    // [mp][8] float32: rec_lo rows, owner side / other side (null: read rec_lo)
    const T* __restrict__ loq;
    const T* __restrict__ isc;    // [mp] 1/sigma_c of the diagonal scaling (1 when unscaled)
    double hD, tol;
    T pi_tol;      // stopping threshold on max |pi| (float32: see above)
    int max_iter;
    int refresh;   // refresh the reference every this many iterations (0: never)
    int zero_start;   // gamma_0 = 0 (the one-barrier solver's initial reference needs no rod pass)
    int sort_ns;   // global-memory blocks sort their rods (shared memory for the order was given)
    int sort_cap;  // rods the order's scratch holds (a larger share keeps the rank order)
    long long wait_cycles;
    int fault;
    // a step recorded as a graph: the one-barrier kernel was launched with
    // fit_cap bytes of shared memory and reads its shares' need here (null:
    // the need was checked on the host)
    const unsigned long long* need1_dev;
    long long fit_cap;
    const int* __restrict__ bstart;   // [gridDim.x + 1] rod-rank boundaries of the blocks
};

// A block's own rods [r0, r1) and constraints [c0, c1), with their
// shared-memory copies (valid when the block is staged).
template <typename T>
struct Own {
    int r0, r1, c0, c1, q0, q1, cap_c, cap_r, cap_q;
    T* rec;      // [9][cap_c]
    T* gref;     // [cap_c] q + D^T Uref
    T* ds;       // [cap_c] delta (phase B updates it in place, one thread per entry)
    T* grs;      // [cap_c] g (phase B updates it in place, one thread per entry)
    T* gam;      // [cap_c] gamma_ref
    T* ax;       // [3][cap_r]
    T* U;        // [6][cap_r] delta velocity (the reference velocity during a refresh)
    int* cj;     // [cap_c] other end (rank)
    unsigned short* ci;   // [cap_c] owner, local index
    int* rowP;   // [cap_r + 1] owned ranges (global constraint ids)
    int* rowQ;   // [cap_r + 1] other-side ranges (global CSR positions)
    int* qlist;  // [cap_q] other-side constraint ids of the block's rods
    unsigned short* perm;   // [cap_r] the order in which the rod phase's threads take the rods
};

// Shared-memory bytes of a block's share: per owned constraint 13 values
// and 6 bytes of indices, per rod 9 values, two row pointers and a 16-bit
// slot of the rod order, per other-side entry one id (owner indices are
// 16-bit: at most 65535 rods).
__host__ __device__ inline size_t staged_bytes(int esize, size_t cap_c, size_t cap_r, size_t cap_q)
{
    return (13 * cap_c + 9 * cap_r) * (size_t)esize + (cap_c + 2 * cap_r + 2 + cap_q) * sizeof(int) +
           (((cap_c + cap_r) * sizeof(unsigned short) + 3) & ~(size_t)3);
}

template <typename T>
__device__ void carve(Own<T>& o, unsigned char* base)
{
    T* t = reinterpret_cast<T*>(base);
    const size_t C = o.cap_c, R = o.cap_r;
    o.rec = t; t += 9 * C;
    o.gref = t; t += C;
    o.ds = t; t += C;
    o.grs = t; t += C;
    o.gam = t; t += C;
    o.ax = t; t += 3 * R;
    o.U = t; t += 6 * R;
    int* ip = reinterpret_cast<int*>(t);
    o.cj = ip; ip += C;
    o.rowP = ip; ip += R + 1;
    o.rowQ = ip; ip += R + 1;
    o.qlist = ip; ip += o.cap_q;
    o.ci = reinterpret_cast<unsigned short*>(ip);
    o.perm = o.ci + C;
}

// Rod order of the rod phase: ascending (owned, other-side) entry counts,
// so that the 32 rods of a warp run loops of about the same lengths (a warp
// runs each loop as long as its longest rod's).  Rank sort on unique keys
// (count pair, then the block-local index, < 65536) in the scratch key and
// rk ([nr] each); rowP and rowQ point at the block's first rod's row
// pointers.
__device__ void sort_rods(const int* rowP, const int* rowQ, int nr, unsigned* key, int* rk, unsigned short* perm)
{
    for (int li = threadIdx.x; li < nr; li += blockDim.x) {
        const int no = min(rowP[li + 1] - rowP[li], 255), nq = min(rowQ[li + 1] - rowQ[li], 255);
        key[li] = ((unsigned)(no << 8 | nq) << 16) | (unsigned)li;
    }
    __syncthreads();
    for (int li = threadIdx.x; li < nr; li += blockDim.x) {
        const unsigned kk = key[li];
        int r = 0;
        for (int lj = 0; lj < nr; ++lj) r += key[lj] < kk;
        rk[li] = r;
    }
    __syncthreads();
    for (int li = threadIdx.x; li < nr; li += blockDim.x) perm[rk[li]] = (unsigned short)li;
    __syncthreads();
}

template <typename T>
__device__ void stage_in(const SolveArgs<T>& a, Own<T>& o)
{
    const int nr = o.r1 - o.r0, nc = o.c1 - o.c0;
    const size_t mp = a.mp, np = a.np;
    for (int li = threadIdx.x; li <= nr; li += blockDim.x) {
        o.rowP[li] = a.rowP[o.r0 + li];
        o.rowQ[li] = a.rowQ[o.r0 + li];
    }
    for (int li = threadIdx.x; li < nr; li += blockDim.x)
        for (int w = 0; w < 3; ++w) o.ax[w * o.cap_r + li] = a.ax[w * np + o.r0 + li];
#pragma unroll 1
    for (int lc = threadIdx.x; lc < nc; lc += blockDim.x) {
        const int c = o.c0 + lc;
#pragma unroll
        for (int w = 0; w < 9; ++w) o.rec[w * o.cap_c + lc] = a.rec[w * mp + c];
        o.cj[lc] = a.cj[c];
        o.ci[lc] = (unsigned short)(a.ci[c] - o.r0);
        T d, g, gr, gl;
        ld_state(a.gg0, c, d, g, gr, gl);
        o.ds[lc] = d;
        o.gam[lc] = gr;
        o.grs[lc] = T(0);
    }
    for (int k = threadIdx.x; k < o.q1 - o.q0; k += blockDim.x) o.qlist[k] = a.qlist[o.q0 + k];
    // the keys and ranks of the rod order live in the velocity array, which
    // the first rod phase writes before anyone reads it (6 cap_r values hold
    // 2 nr words)
    __syncthreads();
    sort_rods(o.rowP, o.rowQ, nr, reinterpret_cast<unsigned*>(o.U), reinterpret_cast<int*>(o.U) + nr, o.perm);
}

// Rod phase modes: A_STEP forms delta_{k+1} = max(-gamma_ref, delta - alpha g)
// (the owner stores it) and stores dU = M D delta_{k+1}; A_PG sums pi.A.pi
// for the projected gradient pi (returned, nothing stored); A_REF stores the
// reference velocity Uref = M D gamma_ref with compensated sums over the
// split (hi + lo) records, and clears dU.
enum { A_STEP = 0, A_PG = 1, A_REF = 2 };
// Constraint phase modes: B_STEP g_{k+1} = gref + D^T dU and the BB sums;
// B_REF gref = q + D^T Uref (compensated, split records and q), then
// g = gref (delta is 0 there) and pi.pi, max |pi| at gamma_ref.
enum { B_STEP = 0, B_REF = 2 };

// bil: a spring (bilateral) constraint, whose force has no sign constraint
// (Eq. linearconstraints b): no projection.
template <int MODE, typename T>
__device__ __forceinline__ T a_value(T d, T g, T gr, T alpha, bool bil)
{
    if (MODE == A_REF) return gr;
    if (MODE == A_STEP) {
        const T v = fma(-alpha, g, d);   // one rounding, the same in both phases that form it
        return (bil || v > -gr) ? v : -gr;
    }
    return (bil || d > -gr) ? g : (g < T(0) ? g : T(0));   // projected gradient at gamma = gr + d
}

template <typename T>
__device__ __forceinline__ T comp_of(const SolveArgs<T>& a, int c)
{
    return a.comp ? __ldg(&a.comp[c]) : T(-1);
}

template <typename T, int MODE, bool ST>
__device__ __forceinline__ T phase_a(const SolveArgs<T>& a, const Own<T>& o, int cur, T alpha)
{
    constexpr bool COMP = MODE == A_REF && sizeof(T) == 4;
    T fmf = T(0);
    const size_t mp = a.mp, np = a.np;
    constexpr int B = Batch<T>::v;
    constexpr int BO = ST ? 1 : B;   // owned entries come from shared memory when staged
    const T* gc = cur ? a.gg1 : a.gg0;
    T* gn = cur ? a.gg0 : a.gg1;
    const T* sdc = o.ds;   // shared copy (staged blocks)
#pragma unroll 1
    for (int t = threadIdx.x; t < o.r1 - o.r0; t += blockDim.x) {
        const int li = o.perm ? (int)o.perm[t] : t, i = o.r0 + li;
        Acc<T, COMP> Fa[6];
#pragma unroll
        for (int w = 0; w < 6; ++w) Fa[w].init(T(0));
        {   // owned constraints: loads of up to BO entries issued together
            const int b = ST ? o.rowP[li] : a.rowP[i], e = ST ? o.rowP[li + 1] : a.rowP[i + 1];
#pragma unroll 1
            for (int c = b; c < e; c += BO) {
                T dv[BO], gv[BO], rv_[BO], gl[BO], rv[BO][6];
#pragma unroll
                for (int u = 0; u < BO; ++u) {
                    if (c + u < e) {
                        if (ST) {
                            const int lc = c + u - o.c0;
                            dv[u] = sdc[lc];
                            gv[u] = o.grs[lc];
                            rv_[u] = o.gam[lc];
                            if (MODE == A_REF && COMP) gl[u] = gc[4 * (size_t)(c + u) + 3];
#pragma unroll
                            for (int w = 0; w < 6; ++w) rv[u][w] = o.rec[w * o.cap_c + lc];
                        } else {
                            ld_state(gc, c + u, dv[u], gv[u], rv_[u], gl[u]);
                            if (sizeof(T) == 4 && a.pe) {   // float64 is bound by its arithmetic instead
                                ld_arm(a.pe, c + u, rv[u]);
                            } else {
#pragma unroll
                                for (int w = 0; w < 6; ++w) rv[u][w] = a.rec[w * mp + c + u];
                            }
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < BO; ++u) {
                    if (c + u < e) {
                        const T cmp = comp_of(a, c + u);
                        const T v = a_value<MODE, T>(dv[u], gv[u], rv_[u], alpha, cmp >= T(0));
                        if (MODE == A_PG && cmp >= T(0)) fmf += cmp * v * v;   // the spring's compliance term
                        // phase B forms delta_{k+1} again from the same values (staged
                        // blocks, float32); float64, bound by its arithmetic, stores it
                        if (MODE == A_STEP && !ST && sizeof(T) == 8) gn[4 * (size_t)(c + u)] = v;
#pragma unroll
                        for (int w = 0; w < 6; ++w) Fa[w].add_prod(v, rv[u][w]);
                        if (MODE == A_REF && COMP) {   // gamma_lo and the records' low parts
#pragma unroll
                            for (int w = 0; w < 6; ++w)
                                Fa[w].add_lo(v * __ldg(&a.rec_lo[w * mp + c + u]) + gl[u] * rv[u][w]);
                        }
                    }
                }
            }
        }
        {   // constraints owned by other rods: ids first, then their state and arms
            // (from shared memory when the owner is one of the block's rods)
            const int b = ST ? o.rowQ[li] : a.rowQ[i], e = ST ? o.rowQ[li + 1] : a.rowQ[i + 1];
#pragma unroll 1
            for (int k = b; k < e; k += B) {
                int cid[B];
#pragma unroll
                for (int u = 0; u < B; ++u)
                    cid[u] = k + u < e ? (ST ? o.qlist[k + u - o.q0] : __ldg(&a.qlist[k + u])) : -1;
                T dv[B], gv[B], rv_[B], gl[B], qv[B][6];
#pragma unroll
                for (int u = 0; u < B; ++u) {
                    if (cid[u] >= 0) {
                        if (ST && cid[u] >= o.c0 && cid[u] < o.c1) {
                            const int lc = cid[u] - o.c0;
                            dv[u] = sdc[lc];
                            gv[u] = o.grs[lc];
                            rv_[u] = o.gam[lc];
                            if (MODE == A_REF && COMP) gl[u] = gc[4 * (size_t)cid[u] + 3];
#pragma unroll
                            for (int w = 0; w < 3; ++w) {
                                qv[u][w] = o.rec[w * o.cap_c + lc];
                                qv[u][3 + w] = o.rec[(6 + w) * o.cap_c + lc];
                            }
                        } else {
                            ld_state(gc, cid[u], dv[u], gv[u], rv_[u], gl[u]);
                            ld_arm(a.qe, k + u, qv[u]);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < B; ++u) {
                    if (cid[u] >= 0) {
                        const T v = a_value<MODE, T>(dv[u], gv[u], rv_[u], alpha, comp_of(a, cid[u]) >= T(0));
#pragma unroll
                        for (int w = 0; w < 6; ++w) Fa[w].add_prod(-v, qv[u][w]);
                        if (MODE == A_REF && COMP) {
                            T ql[6];
                            ld_arm(a.qe_lo, k + u, ql);
#pragma unroll
                            for (int w = 0; w < 6; ++w) Fa[w].add_lo(-(v * ql[w] + gl[u] * qv[u][w]));
                        }
                    }
                }
            }
        }
        T F[6];
#pragma unroll
        for (int w = 0; w < 6; ++w) F[w] = Fa[w].value();
        T p0, p1, p2;
        if (ST) {
            p0 = o.ax[li]; p1 = o.ax[o.cap_r + li]; p2 = o.ax[2 * o.cap_r + li];
        } else {
            p0 = a.ax[i]; p1 = a.ax[np + i]; p2 = a.ax[2 * np + i];
        }
        T ip = a.inv_perp, ipa = a.inv_par, ir = a.inv_rot, is = a.inv_spin;
        if (a.mobr) {
            ip = __ldg(&a.mobr[i]); ipa = __ldg(&a.mobr[np + i]);
            ir = __ldg(&a.mobr[2 * np + i]); is = __ldg(&a.mobr[3 * np + i]);
        }
        const T pf = p0 * F[0] + p1 * F[1] + p2 * F[2];
        const T pt = p0 * F[3] + p1 * F[4] + p2 * F[5];
        const T cf = pf * (ipa - ip), ct = pt * (is - ir);
        T Uv[6] = {F[0] * ip + p0 * cf, F[1] * ip + p1 * cf, F[2] * ip + p2 * cf,
                   F[3] * ir + p0 * ct, F[4] * ir + p1 * ct, F[5] * ir + p2 * ct};
        if (MODE == A_PG) {
#pragma unroll
            for (int w = 0; w < 6; ++w) fmf += F[w] * Uv[w];
        } else {
            // staged steps publish dU after the rod loop, coalesced (copy_out_du)
            if (!(ST && MODE == A_STEP)) st_u6(MODE == A_REF ? a.Uref : a.U, i, Uv);
            if (MODE == A_REF) {
                const T z[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
                st_u6(a.U, i, z);   // dU = 0: delta is 0 after a reference pass
            }
            if (ST) {
#pragma unroll
                for (int w = 0; w < 6; ++w) o.U[w * o.cap_r + li] = Uv[w];
            }
        }
    }
    return fmf;
}

// A staged step's dU for the other blocks: the block's rods [r0, r1) are
// contiguous in the [n][6] global array, so after the rod loop the block
// copies its shared [6][cap_r] values out with consecutive threads writing
// consecutive pairs.  The rod loop's own stores would be three scattered
// 8-byte stores per rod (its threads take the rods in count order), which
// the grid barrier's release then waits for.
template <typename T>
__device__ __forceinline__ void copy_out_du(const SolveArgs<T>& a, const Own<T>& o)
{
    __syncthreads();
    const int nr = o.r1 - o.r0;
    typename V2<T>::t* g = reinterpret_cast<typename V2<T>::t*>(a.U + 6 * (size_t)o.r0);
    for (int k = threadIdx.x; k < 3 * nr; k += blockDim.x) {
        const int r = k / 3, w = 2 * (k - 3 * r);
        typename V2<T>::t v;
        v.x = o.U[w * o.cap_r + r];
        v.y = o.U[(w + 1) * o.cap_r + r];
        g[k] = v;
    }
}

// Constraint phase for the block's owned constraints (modes above).  In
// B_STEP the new state (delta_{k+1}, g_{k+1}, gamma_ref) goes to buffer nx,
// and acc0..2 = s.s, s.y, y.y against buffer cur; acc3 = max |pi|.
template <typename T, int MODE, bool ST>
__device__ __forceinline__ void phase_b(const SolveArgs<T>& a, const Own<T>& o, int cur, int nx, T alpha, T acc[4])
{
    constexpr bool COMP = MODE != B_STEP && sizeof(T) == 4;
    const size_t mp = a.mp;
    T* gnew = nx ? a.gg1 : a.gg0;
    const T* gold = cur ? a.gg1 : a.gg0;
    const T* Uu = MODE == B_STEP ? a.U : a.Uref;
    const int nc = o.c1 - o.c0;
#pragma unroll 1
    for (int lc = threadIdx.x; lc < nc; lc += blockDim.x) {
        const int c = o.c0 + lc;
        T Ui[6], Uj[6], r[9], base, dm, gam, dold = T(0), gro = T(0);
        bool xstate = false;
        if (ST) {
            const int il = o.ci[lc], j = o.cj[lc];
            xstate = j >= 0 && (j < o.r0 || j >= o.r1);
#pragma unroll
            for (int w = 0; w < 6; ++w) Ui[w] = o.U[w * o.cap_r + il];
            if (j < 0) {   // a wall: no other side
#pragma unroll
                for (int w = 0; w < 6; ++w) Uj[w] = T(0);
            } else if (j >= o.r0 && j < o.r1) {
#pragma unroll
                for (int w = 0; w < 6; ++w) Uj[w] = o.U[w * o.cap_r + (j - o.r0)];
            } else {
                ld_u6(Uu, j, Uj);
            }
#pragma unroll
            for (int w = 0; w < 9; ++w) r[w] = o.rec[w * o.cap_c + lc];
            base = MODE == B_STEP ? o.gref[lc] : a.q[c];
            gam = o.gam[lc];
            if (MODE == B_STEP) {
                // delta_{k+1} as the rod phase formed it (same inputs, same rounding)
                dold = o.ds[lc];
                gro = o.grs[lc];
                dm = a_value<A_STEP, T>(dold, gro, gam, alpha, comp_of(a, c) >= T(0));
                o.ds[lc] = dm;
            } else {
                dm = o.ds[lc];
            }
        } else {
            ld_u6(Uu, a.ci[c], Ui);
            const int j = a.cj[c];
            if (j < 0) {   // a wall: no other side
#pragma unroll
                for (int w = 0; w < 6; ++w) Uj[w] = T(0);
            } else {
                ld_u6(Uu, j, Uj);
            }
#pragma unroll
            for (int w = 0; w < 9; ++w) r[w] = a.rec[w * mp + c];
            base = MODE == B_STEP ? a.gref[c] : a.q[c];
            T gl;
            if (MODE == B_STEP && sizeof(T) == 4) {
                // delta_{k+1} as the rod phase formed it (same inputs, same rounding)
                ld_state(gold, c, dold, gro, gam, gl);
                dm = a_value<A_STEP, T>(dold, gro, gam, alpha, comp_of(a, c) >= T(0));
            } else {
                T gdummy;
                ld_state(gnew, c, dm, gdummy, gam, gl);
                if (MODE == B_STEP) {
                    T g2, gl2;
                    ld_state(gold, c, dold, gro, g2, gl2);
                }
            }
        }
        Acc<T, COMP> du;
        du.init(base);
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            du.add_prod(r[u], Ui[u]);
            du.add_prod(-r[u], Uj[u]);
            du.add_prod(r[3 + u], Ui[3 + u]);
            du.add_prod(-r[6 + u], Uj[3 + u]);
        }
        // springs: + (1/(h kappa)) gamma (Eq. blockdef F); the increment's
        // part in a step, the whole force in a reference pass
        const T cmp = comp_of(a, c);
        const bool bil = cmp >= T(0);
        if (bil) {
            if (MODE == B_STEP) {
                du.add_prod(cmp, dm);
            } else {
                const T glo = gl_of_state(gnew, c);
                du.add_prod(cmp, gam);
                du.add_lo(cmp * glo);
            }
        }
        if (MODE == B_REF && COMP) {
            // low parts of q and of the record
            T rl[9];
#pragma unroll
            for (int w = 0; w < 9; ++w) rl[w] = __ldg(&a.rec_lo[w * mp + c]);
            T t = __ldg(&a.q_lo[c]);
#pragma unroll
            for (int u = 0; u < 3; ++u)
                t += rl[u] * (Ui[u] - Uj[u]) + rl[3 + u] * Ui[3 + u] - rl[6 + u] * Uj[3 + u];
            du.add_lo(t);
        }
        const T gr = du.value();
        if (MODE == B_REF) {
            if (ST) o.gref[lc] = gr;
            else a.gref[c] = gr;
        }
        // g of the new iterate (for B_REF: gamma_ref itself, delta = 0)
        if (ST) {
            o.grs[lc] = gr;
            // the state other blocks read in the next rod phase: in a step,
            // only that of constraints whose other rod is another block's
            if (MODE != B_STEP || xstate) st_dg(gnew, c, dm, gr);
        } else if (MODE == B_STEP && sizeof(T) == 4) {
            st_dg(gnew, c, dm, gr);
        } else {
            gnew[4 * (size_t)c + 1] = gr;
        }
        const T pi = (bil || dm > -gam) ? gr : (gr < T(0) ? gr : T(0));
        // the residual is taken on the unscaled projected gradient pi / sigma_c
        const T api = (pi < T(0) ? -pi : pi) * __ldg(&a.isc[c]);
        acc[3] = api > acc[3] ? api : acc[3];
        if (MODE == B_REF) {
            acc[0] += pi * pi;
        } else {
            const T sv = dm - dold, yv = gr - gro;
            acc[0] += sv * sv;
            acc[1] += sv * yv;
            acc[2] += yv * yv;
        }
    }
}

// Refresh, first half: (gamma_ref, gamma_lo) absorbs delta as a
// double-float sum (TwoSum, then renormalised so that |gamma_lo| is at most
// half an ulp of gamma_ref) and delta becomes 0, in shared memory and in
// both global state buffers.  A constraint held at the bound (delta =
// -gamma_ref) gets gamma = 0 exactly.
template <typename T, bool ST>
__device__ __forceinline__ void fold_delta(const SolveArgs<T>& a, const Own<T>& o, int cur)
{
    T* gc = cur ? a.gg1 : a.gg0;
    T* go = cur ? a.gg0 : a.gg1;
    T* sdc = o.ds;
    const int nc = o.c1 - o.c0;
#pragma unroll 1
    for (int lc = threadIdx.x; lc < nc; lc += blockDim.x) {
        const int c = o.c0 + lc;
        T d, g, gr, gl;
        ld_state(gc, c, d, g, gr, gl);
        if (ST) {
            d = sdc[lc]; g = o.grs[lc]; gr = o.gam[lc];
        }
        const bool bil = comp_of(a, c) >= T(0);   // springs: no bound
        T hi = T(0), lo = T(0);
        if (bil || d > -gr) {
            T s, e;
            two_sum(gr, d, s, e);
            const T l = gl + e;
            hi = s + l;
            lo = l - (hi - s);
            if (!bil && (hi < T(0) || (hi == T(0) && lo < T(0)))) { hi = T(0); lo = T(0); }
        }
        if (ST) {
            sdc[lc] = T(0);
            o.gam[lc] = hi;
        }
        st_dg(gc, c, T(0), g);
        st_ref(gc, c, hi, lo);
        st_ref(go, c, hi, lo);
    }
}

// Block partial of (sum, sum, sum, max) in the working precision (warp
// shuffles, then warp 0 over the warp results, fixed order); lane 0 stores
// it for the cross-block sum.
template <typename T>
__device__ __forceinline__ void block_partial(T v[4], T (*red)[4], T* dst, int stride)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int u = 0; u < 3; ++u) v[u] += __shfl_down_sync(0xffffffffu, v[u], o);
        T mx = __shfl_down_sync(0xffffffffu, v[3], o);
        v[3] = mx > v[3] ? mx : v[3];
    }
    if (lane == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) red[warp][u] = v[u];
    }
    __syncthreads();
    if (warp == 0) {
        T w[4] = {T(0), T(0), T(0), T(0)};
        if (lane < nw) {
#pragma unroll
            for (int u = 0; u < 4; ++u) w[u] = red[lane][u];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int u = 0; u < 3; ++u) w[u] += __shfl_down_sync(0xffffffffu, w[u], o);
            T mx = __shfl_down_sync(0xffffffffu, w[3], o);
            w[3] = mx > w[3] ? mx : w[3];
        }
        if (lane == 0) {
#pragma unroll
            for (int u = 0; u < 4; ++u) dst[u * stride] = w[u];
        }
    }
}

// After a barrier: warps 0-3 each reduce one component of the per-block
// partials ([4][nb]: a warp reads one contiguous row) in the working
// precision in a fixed order, the first 12 loads of every lane in flight
// together (one L2 round trip for up to 384 blocks: 304 at 512 threads x 2
// blocks per SM), and the four totals are broadcast through shared memory.
template <typename T>
__device__ __forceinline__ void grid_total(const T* partials, int nb, T* bc, T out[4])
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 4) {
        const T* row = partials + (size_t)warp * nb;
        T xs[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const int b = lane + 32 * k;
            xs[k] = b < nb ? __ldcg(row + b) : T(0);
        }
        T w = T(0);
        if (warp == 3) {   // max |pi| (every entry >= 0)
#pragma unroll
            for (int k = 0; k < 12; ++k) w = xs[k] > w ? xs[k] : w;
            for (int b = lane + 384; b < nb; b += 32) {
                const T x = __ldcg(row + b);
                w = x > w ? x : w;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T y = __shfl_down_sync(0xffffffffu, w, o);
                w = y > w ? y : w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) w += xs[k];
            for (int b = lane + 384; b < nb; b += 32) w += __ldcg(row + b);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
        }
        if (lane == 0) bc[warp] = w;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) out[u] = bc[u];
}

// The stopping test's complement: (h/D) max |pi| > tol, decided in float64
// (float64 iterations) or by the equivalent float32 threshold.
__device__ __forceinline__ bool above_tol(const SolveArgs<double>& a, double pimax) { return a.hD * pimax > a.tol; }
__device__ __forceinline__ bool above_tol(const SolveArgs<float>& a, float pimax) { return pimax > a.pi_tol; }

// Step-size bookkeeping, done by thread 0 alone (every other thread only
// reads the broadcast).
// Pass kinds of the loop: a step, a reference pass, the line step of alpha_0.
enum { P_STEP = 0, P_REF = 1, P_PG = 2 };

template <typename T>
struct StepState {
    T alpha0, pimax;   // max |pi| of the last test: the residual is (h/D) pimax
    double pp;         // pi.pi at gamma_0 (for alpha_0)
    T pss, psy, pyy;   // the previous step's s.s, s.y, y.y (the step length lags one iteration)
    int have, hist;    // previous sums held; BB1/BB2 alternation counter
    int iters, cur, done;
    int since;   // iterations since the last reference refresh
    __device__ __forceinline__ double residual(double hD) const { return hD * (double)pimax; }
};

template <typename T>
struct Shared {
    T red[32][4];
    T bc[4];
    T part[4];   // this block's partial (cluster solver: read by the cluster's blocks)
    T alpha;
    int done, ok, kind, cur, sys, pair;
};

// Synchronisation of the blocks that share one problem.
// Grid: all blocks of a cooperative launch, bounded barrier on a global
// counter, partials in global memory.
template <typename T>
struct GridSync {
    unsigned* bar;
    int* flags;
    long long wait_cycles;
    T* partials;   // [4][nb]
    unsigned nb, epoch;
    template <typename SH>
    __device__ __forceinline__ bool barrier(SH& sh)
    {
        return grid_barrier(bar, nb * ++epoch, flags, wait_cycles, &sh.ok);
    }
    template <typename SH>
    __device__ __forceinline__ T* slot(SH&) { return partials + blockIdx.x; }
    __device__ __forceinline__ int stride() const { return (int)nb; }
    template <typename SH>
    __device__ __forceinline__ void total(SH& sh, T tot[4]) { grid_total(partials, nb, sh.bc, tot); }
};

// Cluster: the blocks of one thread-block cluster, hardware cluster barrier,
// partials in each block's shared memory read through distributed shared
// memory (every block sums them in the same order: identical decisions).
struct ClusterSync {
    template <typename SH>
    __device__ __forceinline__ bool barrier(SH&)
    {
        cg::this_cluster().sync();
        return true;
    }
    template <typename SH>
    __device__ __forceinline__ auto slot(SH& sh) { return sh.part; }
    __device__ __forceinline__ int stride() const { return 1; }
    template <typename SH, typename T>
    __device__ __forceinline__ void total(SH& sh, T tot[4])
    {
        cg::cluster_group cl = cg::this_cluster();
        if (threadIdx.x < 4) {
            const int u = threadIdx.x;
            const unsigned cs = cl.num_blocks();
            T w = T(0);
            for (unsigned r = 0; r < cs; ++r) {
                const T x = cl.map_shared_rank(sh.part, r)[u];
                w = u == 3 ? (x > w ? x : w) : w + x;
            }
            sh.bc[u] = w;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u) tot[u] = sh.bc[u];
    }
};

// Batches: a cluster alone, or two clusters on one system (a pair).  A pair
// synchronises its blocks like the grid solver, on a bounded barrier over a
// counter of its own, with the block sums in global memory; a cluster alone
// uses the hardware cluster barrier and distributed shared memory.
template <typename T>
struct BatchSync {
    unsigned* bar;       // the pair's arrival counter (null: a cluster alone)
    int* flags;
    long long wait_cycles;
    T* partials;         // the pair's [4][nb] block sums
    unsigned nb, epoch;  // the pair's blocks, barriers passed
    int rank;            // this block's rank in the pair
    template <typename SH>
    __device__ __forceinline__ bool barrier(SH& sh)
    {
        if (bar) return grid_barrier(bar, nb * ++epoch, flags, wait_cycles, &sh.ok);
        cg::this_cluster().sync();
        return true;
    }
    template <typename SH>
    __device__ __forceinline__ T* slot(SH& sh) { return bar ? partials + rank : sh.part; }
    __device__ __forceinline__ int stride() const { return bar ? (int)nb : 1; }
    template <typename SH>
    __device__ __forceinline__ void total(SH& sh, T tot[4])
    {
        if (bar) grid_total(partials, (int)nb, sh.bc, tot);
        else ClusterSync().total(sh, tot);
    }
};

// Smallest rank r in [lo, hi] whose cumulative work W(r) = kOwnWork *
// rowP[r] + kOtherWork * rowQ[r] + kRodWork * r reaches target (an
// other-side entry, gathered from another block, costs about twice an owned
// one in the two-barrier kernels); W is strictly increasing and W(hi) >=
// target.  One warp: 32 probes per round, then a final scan of at most 32
// ranks.  The one-barrier kernel's blocks were timed under other weights
// (owned : other-side : rod = 4:1:4, 4:1:2, 3:1:3, 2:1:2; four seeds at 1e5
// rods): the first two push some shares past the shared-memory budget, the
// others cost 0.5-1.7 % more per iteration than 1:2:2.
constexpr int kOwnWork = 1;
constexpr int kRodWork = 2;
constexpr int kOtherWork = 2;
__device__ __forceinline__ long long rank_work(const int* rowP, const int* rowQ, int r)
{
    return (long long)kOwnWork * rowP[r] + (long long)kOtherWork * rowQ[r] + (long long)kRodWork * r;
}
__device__ __forceinline__ int find_rank(const int* rowP, const int* rowQ, int lo, int hi, long long target)
{
    const int lane = threadIdx.x & 31;
    while (hi - lo >= 32) {
        const long long span = hi - lo;
        const int p = lo + (int)(span * (lane + 1) / 33);
        const long long w = rank_work(rowP, rowQ, p);
        const unsigned ge = __ballot_sync(0xffffffffu, w >= target);
        if (ge == 0) {
            lo = __shfl_sync(0xffffffffu, p, 31) + 1;
        } else {
            const int f = __ffs(ge) - 1;
            const int pf = __shfl_sync(0xffffffffu, p, f);
            const int pb = __shfl_sync(0xffffffffu, p, f > 0 ? f - 1 : 0);
            if (f > 0) lo = pb + 1;
            hi = pf;
        }
    }
    const int p = lo + lane;
    bool ge = false;
    if (p <= hi) ge = rank_work(rowP, rowQ, p) >= target;
    const unsigned m = __ballot_sync(0xffffffffu, ge);
    return m ? lo + __ffs(m) - 1 : hi;
}

// The BBPGD loop over the problem shared by the blocks that SY synchronises.
// On return thread 0 holds the step state; sh.cur is the final buffer.
template <typename T, bool ST, typename SY>
__device__ __forceinline__ void solve_loop(const SolveArgs<T>& a, const Own<T>& o, Shared<T>& sh, SY& sy,
                                           StepState<T>& st)
{
    T* mine = sy.slot(sh);
    T tot[4];
    T v[4];
    st.alpha0 = T(1);
    st.pimax = T(0);
    st.pp = 0.0;
    st.pss = st.psy = st.pyy = T(0);
    st.have = 0;
    st.hist = 0;
    st.cur = 0;
    st.since = 0;
    st.iters = 0;
    if (threadIdx.x == 0) {
        sh.cur = 0;
        sh.kind = P_REF;
    }
    __syncthreads();
    int cur = 0, k = 0;           // k: steps taken
    bool first = true;            // the first pass: the reference is gamma_0 (delta = 0)
    // Every pass ends in the same reduction and decision code, and each
    // pass's code appears once: the persistent kernel's code must stay
    // within the instruction cache (inlined copies made every warp stall on
    // instruction fetch after each barrier).
    for (;;) {
        const int kind = sh.kind;
        const bool initial = first;   // this pass is the reference pass at gamma_0
        const int nx = cur ^ 1;
        v[0] = v[1] = v[2] = v[3] = T(0);
        if (kind == P_STEP) {
            phase_a<T, A_STEP, ST>(a, o, cur, sh.alpha);
            if (ST) copy_out_du(a, o);
            if (!sy.barrier(sh)) return;
            phase_b<T, B_STEP, ST>(a, o, cur, nx, sh.alpha, v);
        } else if (kind == P_REF) {
            // the reference takes the iterate; Uref = M D gamma_ref, gref =
            // q + D^T Uref and g are recomputed from the split records with
            // compensated sums, and pi.pi and max |pi| with them
            if (!first) {
                fold_delta<T, ST>(a, o, cur);
                if (!sy.barrier(sh)) return;
            }
            first = false;
            phase_a<T, A_REF, ST>(a, o, cur, T(0));
            if (!sy.barrier(sh)) return;
            phase_b<T, B_REF, ST>(a, o, cur, cur, T(0), v);
        } else {
            // pi.A.pi for alpha_0 = pi.pi / pi.A.pi (exact line step along
            // the projected gradient at gamma_0)
            v[0] = phase_a<T, A_PG, ST>(a, o, cur, T(0));
            // every block has read the partials (grid_total) before any rewrites them
            if (!sy.barrier(sh)) return;
        }
        block_partial(v, sh.red, mine, sy.stride());
        if (!sy.barrier(sh)) return;
        sy.total(sh, tot);
        if (kind == P_STEP) cur = nx;
        if (threadIdx.x == 0) {
            int next = P_STEP;
            if (kind == P_STEP) {
                const T ss = tot[0], sy = tot[1], yy = tot[2];
                st.pimax = tot[3];
                st.cur = cur;
                st.iters = k + 1;
                const bool below = !above_tol(a, tot[3]);
                // the step length of step k + 1 from (s_{k-1}, y_{k-1}): the
                // same one-iteration lag as the one-barrier solver, so every
                // solver kernel runs one method (alpha_0 until a pair is held)
                T an = st.alpha0;
                if (st.have) {
                    an = (st.hist & 1) == 0 ? st.pss / st.psy : st.psy / st.pyy;
                    if (!(st.psy > T(0)) || !isfinite(an) || !(an > T(0))) an = st.alpha0;
                    ++st.hist;
                }
                st.pss = ss;
                st.psy = sy;
                st.pyy = yy;
                st.have = 1;
                sh.alpha = an;
                // float32: a residual below tol is confirmed on a fresh
                // reference before the loop stops (the increments since the
                // last refresh carry float32 rounding); after a refresh that
                // did not confirm it, the next try waits two iterations
                st.done = below && a.refresh == 0;
                ++st.since;
                const bool refresh = a.refresh > 0 && ((below && st.since >= 3) || st.since >= a.refresh);
                if (refresh) {
                    st.since = 0;
                    next = P_REF;
                } else if (k + 1 >= a.max_iter) {
                    st.done = 1;
                }
            } else if (kind == P_REF) {
                st.pimax = tot[3];
                st.done = !above_tol(a, tot[3]) || k >= a.max_iter;
                if (initial) {   // gamma_0: the line step comes next
                    st.pp = (double)tot[0];
                    next = P_PG;
                }
            } else {
                const double pap = (double)tot[0];
                double alpha0 = st.pp / pap;
                if (!(pap > 0.0) || !isfinite(alpha0) || !(alpha0 > 0.0) || !isfinite((T)alpha0)) alpha0 = 1.0;
                st.alpha0 = (T)alpha0;
                sh.alpha = (T)alpha0;
                st.done = 0;
            }
            sh.kind = next;
            sh.done = st.done;
        }
        __syncthreads();
        if (kind == P_STEP) ++k;
        if (sh.done) break;
    }
    if (ST) {
        // the final state of every owned constraint (a step stores only the
        // state that other blocks read)
        T* gf = cur ? a.gg1 : a.gg0;
        for (int lc = threadIdx.x; lc < o.c1 - o.c0; lc += blockDim.x) st_dg(gf, o.c0 + lc, o.ds[lc], o.grs[lc]);
    }
    if (threadIdx.x == 0) sh.cur = st.cur;
    __syncthreads();
}

// One warp per block boundary b in [0, nb]: the work-balanced split.
__global__ void k_partition(int n, int m, int nb, const int* __restrict__ rowP, const int* __restrict__ rowQ,
                            int* __restrict__ bstart)
{
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b > nb) return;   // uniform per warp
    const long long total = rank_work(rowP, rowQ, n);
    const int r = b == nb ? n : find_rank(rowP, rowQ, 0, n, total * b / nb);
    if ((threadIdx.x & 31) == 0) bstart[b] = r;
}

// Largest shared-memory share over the blocks (bytes, for element size esize)
// and the largest rod count of a block.
__global__ void k_stage_need(int nb, int esize, const int* __restrict__ bstart, const int* __restrict__ rowP,
                             const int* __restrict__ rowQ, unsigned long long* __restrict__ need,
                             unsigned long long* __restrict__ maxrods)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int r0 = bstart[b], r1 = bstart[b + 1];
    const size_t nc = rowP[r1] - rowP[r0], nq = rowQ[r1] - rowQ[r0], nr = r1 - r0;
    const size_t bytes = staged_bytes(esize, nc, nr, nq);
    atomicMax(need, (unsigned long long)bytes);
    atomicMax(maxrods, (unsigned long long)nr);
}

template <typename T, bool ST>
__global__ void __launch_bounds__(1024, 1) k_bbpgd(SolveArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ Shared<T> sh;
    if (a.fault == 1 && blockIdx.x == 0) return;   // test hook: this block never arrives
    Own<T> o;
    o.r0 = a.bstart[blockIdx.x];
    o.r1 = a.bstart[blockIdx.x + 1];
    o.c0 = a.rowP[o.r0];
    o.c1 = a.rowP[o.r1];
    o.q0 = a.rowQ[o.r0];
    o.q1 = a.rowQ[o.r1];
    // the carve uses the block's own counts (all of them fit: checked on launch)
    o.cap_c = o.c1 - o.c0;
    o.cap_r = o.r1 - o.r0;
    o.cap_q = o.q1 - o.q0;
    o.perm = nullptr;
    if (ST) {
        carve(o, dyn);
        stage_in(a, o);
    } else if (a.sort_ns) {
        // global-memory blocks: the rod order alone in shared memory
        const int nr = o.r1 - o.r0;
        unsigned* key = reinterpret_cast<unsigned*>(dyn);
        int* rk = reinterpret_cast<int*>(key + nr);
        o.perm = reinterpret_cast<unsigned short*>(rk + nr);
        sort_rods(a.rowP + o.r0, a.rowQ + o.r0, nr, key, rk, o.perm);
    }
    GridSync<T> sy;
    sy.bar = a.bar; sy.flags = a.flags; sy.wait_cycles = a.wait_cycles;
    sy.partials = reinterpret_cast<T*>(a.partials);
    sy.nb = gridDim.x; sy.epoch = 0;
    StepState<T> st;   // meaningful in thread 0 only
    solve_loop<T, ST>(a, o, sh, sy, st);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.out[1] = (double)st.alpha0;
        a.flags[F_FINAL] = st.cur;
        a.flags[F_ITERS] = st.iters;
        a.out[0] = st.residual(a.hD);
    }
}

// ---------------------------------------------------------------------
// One grid barrier per iteration (staged blocks).
//
// The loop above exchanges two things between blocks in every iteration:
// the velocities dU, which the constraint phase gathers, and the state of
// constraints whose ends lie in different blocks, which the rod phase
// gathers; each needs its own grid barrier, and the step-length sums ride
// on the second.  Here a block also keeps a copy ("ghost") of every
// constraint that another block owns but whose other end is one of its
// rods, and updates it with the owner's arithmetic on the same inputs
// (the same delta, g and alpha, the same two velocities, the same order of
// operations), so that owner and ghost stay equal bit for bit and the rod
// phase reads nothing but shared memory.  Only dU and the block sums cross
// blocks, and both travel on one barrier:
//   constraint phase k (every owned and ghost constraint):
//       delta_k = max(-gamma_ref, delta_{k-1} - alpha_{k-1} g_{k-1}),
//       g_k = gref + D^T dU_k, and for owned constraints the sums of
//       s.s, s.y, y.y (s = delta_k - delta_{k-1}, y = g_k - g_{k-1}) and
//       max |pi_k|;
//   step decision from the sums of constraint phase k-1 (published by the
//       last barrier, fetched into shared memory by cp.async while the
//       constraint phase runs): alpha_k = BB(s_{k-2}, y_{k-2}), i.e. the
//       Barzilai-Borwein step of the published method taken one iteration
//       late (a gradient method with retards: Friedlander, Martinez, Molina
//       & Raydan, SIAM J. Numer. Anal. 36, 1999);
//   rod phase k: delta_{k+1} formed on the fly, dU_{k+1} = M D delta_{k+1},
//       copied out to one of two global buffers (they alternate, so a block
//       never overwrites velocities another block may still be reading);
//   grid barrier (block sums in one of two buffers, alternating alike).
// A residual below tol, 64 float32 iterations, or max_iter start a
// reference refresh of the iterate the slots hold (the same compensated
// passes as above, two extra barriers); the loop stops only on the residual
// of a fresh reference, so the returned gamma (delta = 0 there) carries the
// residual it reports, in float64 and float32 alike.

// A block's share: rods [r0, r1), owned constraints [c0, c1) in slots
// [0, nc), ghosts in slots [nc, nt).
template <typename T>
struct Own1 {
    int r0, r1, c0, c1, q0, q1, nc, ng, nt, cap_r, nbp;
    T* tot;      // [4][nbp] last barrier's block sums (cp.async target)
    T* rec;      // [9][nt]
    T* gref;     // [nt] q + D^T Uref
    T* ds;       // [nt] delta
    T* grs;      // [nt] g
    T* gam;      // [nt] gamma_ref
    T* ax;       // [3][cap_r]
    T* U;        // [6][cap_r] this iteration's dU (the reference velocity during a refresh)
    int* oth;    // [nt] rank of the slot's other end: Q for owned slots, the owner for ghosts (-1: a wall)
    int* gid;    // [ng] constraint id of ghost slot nc + g
    int* rowP;   // [cap_r + 1] owned ranges (constraint ids; slot = id - c0)
    int* rowQ;   // [cap_r + 1] other-side ranges (CSR positions)
    unsigned short* loc;    // [nt] local index of the slot's rod in this block (P owned, Q ghost), | kBil
    unsigned short* qslot;  // [q1 - q0] slot of each other-side entry, | kBil
    unsigned short* perm;   // [cap_r] rod order of the rod phase
};
constexpr unsigned kBil = 0x8000u;   // bilateral (spring) constraint: no projection
constexpr int kMaxSlots = 0x7fff;

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// Shared-memory bytes of a one-barrier block share (nt slots of which ng
// ghosts, nr rods, nq other-side entries, nb blocks).
__host__ __device__ inline size_t staged1_bytes(int esize, size_t nt, size_t ng, size_t nr, size_t nq, size_t nb)
{
    const size_t nbp = (nb + 3) & ~(size_t)3;
    return align16(4 * nbp * esize) + align16((13 * nt + 9 * nr) * esize) +
           align16((nt + ng + 2 * nr + 2) * sizeof(int)) + align16((nt + nq + nr) * sizeof(unsigned short));
}

template <typename T>
__device__ void carve1(Own1<T>& o, unsigned char* base)
{
    const size_t nt = o.nt, R = o.cap_r;
    o.tot = reinterpret_cast<T*>(base);
    base += align16(4 * (size_t)o.nbp * sizeof(T));
    T* t = reinterpret_cast<T*>(base);
    o.rec = t; t += 9 * nt;
    o.gref = t; t += nt;
    o.ds = t; t += nt;
    o.grs = t; t += nt;
    o.gam = t; t += nt;
    o.ax = t; t += 3 * R;
    o.U = t; t += 6 * R;
    base += align16((13 * nt + 9 * R) * sizeof(T));
    int* ip = reinterpret_cast<int*>(base);
    o.oth = ip; ip += nt;
    o.gid = ip; ip += o.ng;
    o.rowP = ip; ip += R + 1;
    o.rowQ = ip; ip += R + 1;
    base += align16((nt + o.ng + 2 * R + 2) * sizeof(int));
    unsigned short* sp = reinterpret_cast<unsigned short*>(base);
    o.loc = sp; sp += nt;
    o.qslot = sp; sp += o.q1 - o.q0;
    o.perm = sp;
}

template <typename T>
struct Shared1 {
    T red[32][4];
    T tot[4];   // grid totals of the last barrier's block sums (warps 1-4, one each)
    T alpha;
    int kind, ng;
};

// Stage one slot (owned or ghost) of constraint c from the global arrays.
template <typename T>
__device__ __forceinline__ void stage_slot(const SolveArgs<T>& a, const Own1<T>& o, int t, int c, int li, int other,
                                           unsigned bil)
{
    const size_t mp = a.mp, nt = o.nt;
#pragma unroll
    for (int w = 0; w < 9; ++w) o.rec[w * nt + t] = a.rec[w * mp + c];
    T d, g, gr, gl;
    ld_state(a.gg0, c, d, g, gr, gl);
    o.ds[t] = d;
    o.gam[t] = gr;
    o.grs[t] = gl;   // gamma_lo until the first reference pass replaces it by g
    o.gref[t] = T(0);
    o.oth[t] = other;
    o.loc[t] = (unsigned short)(li | bil);
}

template <typename T>
__device__ void stage_in1(const SolveArgs<T>& a, Own1<T>& o, unsigned char* dyn, Shared1<T>& sh)
{
    const int nr = o.r1 - o.r0, nq = o.q1 - o.q0;
    // ghosts: other-side entries of the block's rods that another block owns
    if (threadIdx.x == 0) sh.ng = 0;
    __syncthreads();
    int cnt = 0;
    for (int k = threadIdx.x; k < nq; k += blockDim.x) {
        const int c = a.qlist[o.q0 + k];
        cnt += c < o.c0 || c >= o.c1;
    }
    if (cnt) atomicAdd(&sh.ng, cnt);
    __syncthreads();
    o.ng = sh.ng;
    o.nt = o.nc + o.ng;
    carve1(o, dyn);
    __syncthreads();
    if (threadIdx.x == 0) sh.ng = 0;
    for (int li = threadIdx.x; li <= nr; li += blockDim.x) {
        o.rowP[li] = a.rowP[o.r0 + li];
        o.rowQ[li] = a.rowQ[o.r0 + li];
    }
    for (int li = threadIdx.x; li < nr; li += blockDim.x)
        for (int w = 0; w < 3; ++w) o.ax[w * o.cap_r + li] = a.ax[w * (size_t)a.np + o.r0 + li];
    const bool has_comp = a.comp != nullptr;
#pragma unroll 1
    for (int t = threadIdx.x; t < o.nc; t += blockDim.x) {
        const int c = o.c0 + t;
        const unsigned bil = has_comp && a.comp[c] >= T(0) ? kBil : 0u;
        stage_slot(a, o, t, c, a.ci[c] - o.r0, a.cj[c], bil);
    }
    __syncthreads();   // sh.ng is 0 again before the slots are numbered
#pragma unroll 1
    for (int k = threadIdx.x; k < nq; k += blockDim.x) {
        const int c = a.qlist[o.q0 + k];
        const unsigned bil = has_comp && a.comp[c] >= T(0) ? kBil : 0u;
        int t;
        if (c < o.c0 || c >= o.c1) {
            // the slot order of ghosts does not enter any result
            const int g = atomicAdd(&sh.ng, 1);
            t = o.nc + g;
            o.gid[g] = c;
            stage_slot(a, o, t, c, a.cj[c] - o.r0, a.ci[c], bil);
        } else {
            t = c - o.c0;
        }
        o.qslot[k] = (unsigned short)(t | bil);
    }
    __syncthreads();
    sort_rods(o.rowP, o.rowQ, nr, reinterpret_cast<unsigned*>(o.U), reinterpret_cast<int*>(o.U) + nr, o.perm);
}

template <typename T>
__device__ __forceinline__ int slot_gid(const Own1<T>& o, int t)
{
    return t < o.nc ? o.c0 + t : o.gid[t - o.nc];
}

// Rod phase over the block's rods, every entry from shared memory (modes
// as for phase_a: A_STEP forms delta_{k+1} with alpha and leaves dU in
// shared memory; A_PG returns this thread's share of pi.A.pi; A_REF leaves
// Uref = M D gamma_ref (compensated in float32) in shared memory and in
// the global Uref).
// The six low parts of one side of constraint c: e's, then the arm's (rec_lo
// rows 0-2 and 3-5 for the owner, 0-2 and 6-8 for the other side, arm0 = 3
// or 6), from the side's 32-byte row when there is one.
template <typename T>
__device__ __forceinline__ void lo_side(const T* rows, const T* rec_lo, size_t mp, int c, int arm0, T out[6])
{
    if (sizeof(T) == 4 && rows) {
        const float4* r = reinterpret_cast<const float4*>(rows + 8 * (size_t)c);
        const float4 x = __ldg(r), y = __ldg(r + 1);
        out[0] = (T)x.x; out[1] = (T)x.y; out[2] = (T)x.z;
        out[3] = (T)x.w; out[4] = (T)y.x; out[5] = (T)y.y;
        return;
    }
#pragma unroll
    for (int w = 0; w < 3; ++w) {
        out[w] = __ldg(&rec_lo[w * mp + c]);
        out[3 + w] = __ldg(&rec_lo[(arm0 + w) * mp + c]);
    }
}

template <typename T, int MODE>
__device__ __forceinline__ T rod_pass1(const SolveArgs<T>& a, const Own1<T>& o, T alpha)
{
    constexpr bool COMP = MODE == A_REF && sizeof(T) == 4;
    const bool has_comp = a.comp != nullptr;
    const size_t mp = a.mp, np = a.np, nt = o.nt;
    T fmf = T(0);
#pragma unroll 1
    for (int tt = threadIdx.x; tt < o.r1 - o.r0; tt += blockDim.x) {
        const int li = (int)o.perm[tt], i = o.r0 + li;
        Acc<T, COMP> Fa[6];
#pragma unroll
        for (int w = 0; w < 6; ++w) Fa[w].init(T(0));
        {   // owned constraints: slots [rowP[li] - c0, rowP[li + 1] - c0)
            const int e = o.rowP[li + 1] - o.c0;
#pragma unroll 1
            for (int t = o.rowP[li] - o.c0; t < e; ++t) {
                const T dv = o.ds[t], gv = o.grs[t], gr = o.gam[t];
                T rv[6];
#pragma unroll
                for (int w = 0; w < 6; ++w) rv[w] = o.rec[w * nt + t];
                const bool bil = has_comp && (o.loc[t] & kBil);
                const T v = a_value<MODE, T>(dv, gv, gr, alpha, bil);
                if (MODE == A_PG && bil) fmf += __ldg(&a.comp[o.c0 + t]) * v * v;   // the spring's compliance term
#pragma unroll
                for (int w = 0; w < 6; ++w) Fa[w].add_prod(v, rv[w]);
                if (COMP) {   // gamma_lo (held in grs during a reference pass) and the records' low parts
                    const int c = o.c0 + t;
                    const T gl = gv;
                    T rl[6];
                    lo_side(a.lop, a.rec_lo, mp, c, 3, rl);
#pragma unroll
                    for (int w = 0; w < 6; ++w) Fa[w].add_lo(v * rl[w] + gl * rv[w]);
                }
            }
        }
        {   // constraints owned by other rods (owned or ghost slots)
            const int e = o.rowQ[li + 1] - o.q0;
#pragma unroll 1
            for (int k = o.rowQ[li] - o.q0; k < e; ++k) {
                const unsigned qs = o.qslot[k];
                const int t = (int)(qs & kMaxSlots);
                const T dv = o.ds[t], gv = o.grs[t], gr = o.gam[t];
                T qv[6];
#pragma unroll
                for (int w = 0; w < 3; ++w) {
                    qv[w] = o.rec[w * nt + t];
                    qv[3 + w] = o.rec[(6 + w) * nt + t];
                }
                const T v = a_value<MODE, T>(dv, gv, gr, alpha, has_comp && (qs & kBil));
#pragma unroll
                for (int w = 0; w < 6; ++w) Fa[w].add_prod(-v, qv[w]);
                if (COMP) {
                    const int c = slot_gid(o, t);
                    const T gl = gv;
                    T ql[6];
                    lo_side(a.loq, a.rec_lo, mp, c, 6, ql);
#pragma unroll
                    for (int w = 0; w < 6; ++w) Fa[w].add_lo(-(v * ql[w] + gl * qv[w]));
                }
            }
        }
        T F[6];
#pragma unroll
        for (int w = 0; w < 6; ++w) F[w] = Fa[w].value();
        const T p0 = o.ax[li], p1 = o.ax[o.cap_r + li], p2 = o.ax[2 * o.cap_r + li];
        T ip = a.inv_perp, ipa = a.inv_par, ir = a.inv_rot, is = a.inv_spin;
        if (a.mobr) {
            ip = __ldg(&a.mobr[i]); ipa = __ldg(&a.mobr[np + i]);
            ir = __ldg(&a.mobr[2 * np + i]); is = __ldg(&a.mobr[3 * np + i]);
        }
        const T pf = p0 * F[0] + p1 * F[1] + p2 * F[2];
        const T pt = p0 * F[3] + p1 * F[4] + p2 * F[5];
        const T cf = pf * (ipa - ip), ct = pt * (is - ir);
        const T Uv[6] = {F[0] * ip + p0 * cf, F[1] * ip + p1 * cf, F[2] * ip + p2 * cf,
                         F[3] * ir + p0 * ct, F[4] * ir + p1 * ct, F[5] * ir + p2 * ct};
        if (MODE == A_PG) {
#pragma unroll
            for (int w = 0; w < 6; ++w) fmf += F[w] * Uv[w];
        } else {
#pragma unroll
            for (int w = 0; w < 6; ++w) o.U[w * o.cap_r + li] = Uv[w];
            if (MODE == A_REF) st_u6(a.Uref, i, Uv);
        }
    }
    return fmf;
}

// The block's dU (shared [6][cap_r]) into its contiguous range of the
// global [n][6] buffer dst, consecutive threads writing consecutive pairs.
template <typename T>
__device__ __forceinline__ void copy_out1(T* dst, const Own1<T>& o)
{
    __syncthreads();
    const int nr = o.r1 - o.r0;
    typename V2<T>::t* g = reinterpret_cast<typename V2<T>::t*>(dst + 6 * (size_t)o.r0);
    for (int k = threadIdx.x; k < 3 * nr; k += blockDim.x) {
        const int r = k / 3, w = 2 * (k - 3 * r);
        typename V2<T>::t v;
        v.x = o.U[w * o.cap_r + r];
        v.y = o.U[(w + 1) * o.cap_r + r];
        g[k] = v;
    }
}

// Uref = 0 for the block's rods: shared memory and its rows of the global
// Uref (the velocity the step reports if gamma_0 already meets the tolerance).
template <typename T>
__device__ __forceinline__ void zero_uref1(const SolveArgs<T>& a, const Own1<T>& o)
{
    const int nr = o.r1 - o.r0;
    for (int k = threadIdx.x; k < 6 * o.cap_r; k += blockDim.x) o.U[k] = T(0);
    typename V2<T>::t z;
    z.x = T(0);
    z.y = T(0);
    typename V2<T>::t* g = reinterpret_cast<typename V2<T>::t*>(a.Uref + 6 * (size_t)o.r0);
    for (int k = threadIdx.x; k < 3 * nr; k += blockDim.x) g[k] = z;
}

// The two velocities of slot t, P side first: Ui of the owner, Uj of the
// other end (0 for a wall).  Local rods from shared memory, others from the
// global buffer Ug.
template <typename T>
__device__ __forceinline__ void slot_velocities(const Own1<T>& o, int t, const T* Ug, T Ui[6], T Uj[6])
{
    const int li = (int)(o.loc[t] & kMaxSlots);
    const int ro = o.oth[t];
    T Ul[6], Uo[6];
#pragma unroll
    for (int w = 0; w < 6; ++w) Ul[w] = o.U[w * o.cap_r + li];
    if (ro < 0) {
#pragma unroll
        for (int w = 0; w < 6; ++w) Uo[w] = T(0);
    } else if (ro >= o.r0 && ro < o.r1) {
#pragma unroll
        for (int w = 0; w < 6; ++w) Uo[w] = o.U[w * o.cap_r + (ro - o.r0)];
    } else {
        ld_u6(Ug, ro, Uo);
    }
    const bool own = t < o.nc;
#pragma unroll
    for (int w = 0; w < 6; ++w) {
        Ui[w] = own ? Ul[w] : Uo[w];
        Uj[w] = own ? Uo[w] : Ul[w];
    }
}

// Constraint phase of a step over every slot: delta_k from
// (delta_{k-1}, g_{k-1}, alpha_{k-1}) exactly as the rod phase formed it,
// g_k = gref + D^T dU_k (+ the spring's compliance term), and for owned
// slots acc = (s.s, s.y, y.y, max |pi|).
template <typename T>
__device__ __forceinline__ void con_pass_step1(const SolveArgs<T>& a, const Own1<T>& o, T alpha, const T* Ug, T acc[4])
{
    const bool has_comp = a.comp != nullptr;
    const size_t nt = o.nt;
#pragma unroll 1
    for (int t = threadIdx.x; t < o.nt; t += blockDim.x) {
        T Ui[6], Uj[6], r[9];
        slot_velocities(o, t, Ug, Ui, Uj);
#pragma unroll
        for (int w = 0; w < 9; ++w) r[w] = o.rec[w * nt + t];
        const T dold = o.ds[t], gro = o.grs[t], gam = o.gam[t];
        const int c = slot_gid(o, t);
        const T cmp = has_comp ? __ldg(&a.comp[c]) : T(-1);
        const bool bil = cmp >= T(0);
        const T dm = a_value<A_STEP, T>(dold, gro, gam, alpha, bil);
        Acc<T, false> du;
        du.init(o.gref[t]);
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            du.add_prod(r[u], Ui[u]);
            du.add_prod(-r[u], Uj[u]);
            du.add_prod(r[3 + u], Ui[3 + u]);
            du.add_prod(-r[6 + u], Uj[3 + u]);
        }
        if (bil) du.add_prod(cmp, dm);
        const T gr = du.value();
        o.ds[t] = dm;
        o.grs[t] = gr;
        if (t < o.nc) {
            const T pi = (bil || dm > -gam) ? gr : (gr < T(0) ? gr : T(0));
            const T api = (pi < T(0) ? -pi : pi) * __ldg(&a.isc[c]);
            acc[3] = api > acc[3] ? api : acc[3];
            const T sv = dm - dold, yv = gr - gro;
            acc[0] += sv * sv;
            acc[1] += sv * yv;
            acc[2] += yv * yv;
        }
    }
}

// Constraint phase of a refresh over every slot: gref = q + D^T Uref from
// the split records and q with compensated sums (float32), g = gref, and
// for owned slots acc = (pi.pi, 0, 0, max |pi|) at gamma_ref.  ZERO: Uref
// is 0 (gamma_ref = 0), so no velocity is read and the records' products
// (all zero) are left out of the sums.
template <typename T, bool ZERO = false>
__device__ __forceinline__ void con_pass_ref1(const SolveArgs<T>& a, const Own1<T>& o, T acc[4])
{
    constexpr bool COMP = sizeof(T) == 4;
    const bool has_comp = a.comp != nullptr;
    const size_t nt = o.nt, mp = a.mp;
#pragma unroll 1
    for (int t = threadIdx.x; t < o.nt; t += blockDim.x) {
        T Ui[6], Uj[6], r[9];
        if (!ZERO) {
            slot_velocities(o, t, a.Uref, Ui, Uj);
#pragma unroll
            for (int w = 0; w < 9; ++w) r[w] = o.rec[w * nt + t];
        }
        const int c = slot_gid(o, t);
        const T gam = o.gam[t];
        Acc<T, COMP> du;
        du.init(__ldg(&a.q[c]));
        if (!ZERO) {
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                du.add_prod(r[u], Ui[u]);
                du.add_prod(-r[u], Uj[u]);
                du.add_prod(r[3 + u], Ui[3 + u]);
                du.add_prod(-r[6 + u], Uj[3 + u]);
            }
        }
        const T cmp = has_comp ? __ldg(&a.comp[c]) : T(-1);
        const bool bil = cmp >= T(0);
        if (bil) {
            du.add_prod(cmp, gam);
            du.add_lo(cmp * o.grs[t]);   // gamma_lo, before g takes its place below
        }
        if (COMP) {
            T tl = __ldg(&a.q_lo[c]);
            if (!ZERO) {
                T lp[6], lq[6];   // (e, y_P x e) and (e, y_Q x e) low parts
                lo_side(a.lop, a.rec_lo, mp, c, 3, lp);
                lo_side(a.loq, a.rec_lo, mp, c, 6, lq);
#pragma unroll
                for (int u = 0; u < 3; ++u)
                    tl += lp[u] * (Ui[u] - Uj[u]) + lp[3 + u] * Ui[3 + u] - lq[3 + u] * Uj[3 + u];
            }
            du.add_lo(tl);
        }
        const T gr = du.value();
        o.gref[t] = gr;
        o.grs[t] = gr;
        if (t < o.nc) {
            const T dm = o.ds[t];   // 0 after the fold
            const T pi = (bil || dm > -gam) ? gr : (gr < T(0) ? gr : T(0));
            const T api = (pi < T(0) ? -pi : pi) * __ldg(&a.isc[c]);
            acc[3] = api > acc[3] ? api : acc[3];
            acc[0] += pi * pi;
        }
    }
}

// Refresh, first half: every slot folds delta into (gamma_ref, gamma_lo)
// as fold_delta does, from the previous reference's gamma_lo in gprev;
// ghosts repeat their owner's arithmetic on the same inputs, so both hold
// the same reference without waiting for each other.  gamma_ref goes to
// gam, gamma_lo to grs (the reference passes' low part, until the constraint
// pass replaces it by g), and owned slots publish (gamma_ref, gamma_lo) in
// gnew, the other state buffer (ghosts are still reading gprev).
template <typename T>
__device__ __forceinline__ void fold1(const SolveArgs<T>& a, const Own1<T>& o, const T* gprev, T* gnew)
{
    const bool has_comp = a.comp != nullptr;
#pragma unroll 1
    for (int t = threadIdx.x; t < o.nt; t += blockDim.x) {
        const int c = slot_gid(o, t);
        const T d = o.ds[t], gr = o.gam[t], gl = gl_of_state(gprev, c);
        const bool bil = has_comp && (o.loc[t] & kBil);
        T hi = T(0), lo = T(0);
        if (bil || d > -gr) {
            T s, e;
            two_sum(gr, d, s, e);
            const T l = gl + e;
            hi = s + l;
            lo = l - (hi - s);
            if (!bil && (hi < T(0) || (hi == T(0) && lo < T(0)))) { hi = T(0); lo = T(0); }
        }
        o.gam[t] = hi;
        o.grs[t] = lo;
        o.ds[t] = T(0);
        if (t < o.nc) st_ref(gnew, c, hi, lo);
    }
}

// cp.async of the last barrier's block sums ([4][nbp] of buffer src) into
// shared memory; the threads that issue it wait for it in tot_wait.
template <typename T>
__device__ __forceinline__ void tot_fetch(const Own1<T>& o, const T* src)
{
    const int chunks = (int)(4 * (size_t)o.nbp * sizeof(T) / 16);
    if ((int)threadIdx.x < chunks) {
        for (int q = threadIdx.x; q < chunks; q += blockDim.x) {
            const unsigned dst = (unsigned)__cvta_generic_to_shared(reinterpret_cast<unsigned char*>(o.tot) + 16 * (size_t)q);
            const unsigned char* s = reinterpret_cast<const unsigned char*>(src) + 16 * (size_t)q;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(s) : "memory");
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
}
__device__ __forceinline__ void tot_wait() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Warp w's share of the block sums: each warp's (sum, sum, sum, max) into red[w].
template <typename T>
__device__ __forceinline__ void warp_partial(T v[4], T (*red)[4])
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int u = 0; u < 3; ++u) v[u] += __shfl_down_sync(0xffffffffu, v[u], o);
        const T mx = __shfl_down_sync(0xffffffffu, v[3], o);
        v[3] = mx > v[3] ? mx : v[3];
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) red[threadIdx.x >> 5][u] = v[u];
    }
}

// Warp 0 after a block barrier: the block's sums over red, lane 0 stores
// them in dst ([4][stride]).
template <typename T>
__device__ __forceinline__ void block_store(T (*red)[4], T* dst, int stride)
{
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    T w[4] = {T(0), T(0), T(0), T(0)};
    if (lane < nw) {
#pragma unroll
        for (int u = 0; u < 4; ++u) w[u] = red[lane][u];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int u = 0; u < 3; ++u) w[u] += __shfl_down_sync(0xffffffffu, w[u], o);
        const T mx = __shfl_down_sync(0xffffffffu, w[3], o);
        w[3] = mx > w[3] ? mx : w[3];
    }
    if (lane == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) dst[u * stride + blockIdx.x] = w[u];
    }
}

// One warp: the grid total of row u of the fetched block sums (sums for
// u < 3, the maximum for u = 3), in a fixed order, so every block gets the
// same numbers; every lane returns it.
template <typename T>
__device__ __forceinline__ T row_total(const Own1<T>& o, int nb, int u)
{
    const int lane = threadIdx.x & 31;
    const T* row = o.tot + (size_t)u * o.nbp;
    T w = T(0);
    for (int b = lane; b < nb; b += 32) {
        const T x = row[b];
        w = u == 3 ? (x > w ? x : w) : w + x;
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const T y = __shfl_xor_sync(0xffffffffu, w, s);
        w = u == 3 ? (y > w ? y : w) : w + y;
    }
    return w;
}

// The four totals, one warp each: warps 1-4 store them in shared memory and
// meet on a named barrier (warp 0 meanwhile stores the block's own sums).
template <typename T>
__device__ __forceinline__ void warps_totals(const Own1<T>& o, int nb, T* tot)
{
    const int u = (int)(threadIdx.x >> 5) - 1;
    const T w = row_total(o, nb, u);
    if ((threadIdx.x & 31) == 0) tot[u] = w;
    asm volatile("bar.sync 1, 128;\n" ::: "memory");
}

// Loop states: what the last constraint phase was (its sums are what the
// last barrier published), and the decision taken for the next rod phase.
enum { C_NONE1 = 0, C_STEP1 = 1, C_REF1 = 2 };
enum { K_STEP1 = 0, K_REF1 = 1, K_STOP1 = 2 };

template <typename T>
__global__ void __launch_bounds__(1024, 1) k_bbpgd1(SolveArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ Shared1<T> sh;
    if (a.need1_dev) {
        // recorded step: every block reads the same need, so either all run
        // or all leave before their first barrier and ask for an eager step
        const unsigned long long need = *a.need1_dev;
        if (need == 0 || need > (unsigned long long)a.fit_cap) {
            if (blockIdx.x == 0 && threadIdx.x == 0) a.flags[F_SOLVE_ERR] = kSolveRedo;
            return;
        }
    }
    if (a.fault == 1 && blockIdx.x == 0) return;   // test hook: this block never arrives
    Own1<T> o;
    o.r0 = a.bstart[blockIdx.x];
    o.r1 = a.bstart[blockIdx.x + 1];
    o.c0 = a.rowP[o.r0];
    o.c1 = a.rowP[o.r1];
    o.q0 = a.rowQ[o.r0];
    o.q1 = a.rowQ[o.r1];
    o.nc = o.c1 - o.c0;
    o.cap_r = o.r1 - o.r0;
    const int nb = (int)gridDim.x;
    o.nbp = (nb + 3) & ~3;
    stage_in1(a, o, dyn, sh);
    T* part = reinterpret_cast<T*>(a.partials);   // [2][4][nbp]
    const size_t pstride = 4 * (size_t)o.nbp;
    unsigned epoch = 0;
    int* s_ok = &sh.ng;   // the barrier's broadcast word (ng is not needed after staging)
    auto barrier = [&]() { return grid_barrier(a.bar, (unsigned)nb * ++epoch, a.flags, a.wait_cycles, s_ok); };
    const int warp = threadIdx.x >> 5;
    // step state, kept by thread 32 (warp 1, lane 0)
    T alpha0 = T(1), pimax = T(0);
    int k = 0, since = 0, hist = 0;
    bool ok = true;

    // initial reference at gamma_0 and the line step alpha_0 = pi.pi / pi.A.pi;
    // from gamma_0 = 0, Uref = M D gamma_0 = 0 needs no rod pass and no
    // other block's velocities
    if (a.zero_start) {
        zero_uref1(a, o);
        __syncthreads();
    } else {
        rod_pass1<T, A_REF>(a, o, T(0));
        ok = barrier();
    }
    int pw = 0;   // block-sum buffer the next barrier publishes
    if (ok) {
        T v[4] = {T(0), T(0), T(0), T(0)};
        if (a.zero_start) con_pass_ref1<T, true>(a, o, v);
        else con_pass_ref1(a, o, v);
        __syncthreads();   // gref and g of every slot before the line step reads them
        v[1] = rod_pass1<T, A_PG>(a, o, T(0));
        warp_partial(v, sh.red);
        __syncthreads();
        if (warp == 0) block_store(sh.red, part + pw * pstride, o.nbp);
        ok = barrier();
    }
    if (ok) {
        tot_fetch(o, part + pw * pstride);
        tot_wait();
        __syncthreads();
        if (warp >= 1 && warp <= 4) {
            warps_totals(o, nb, sh.tot);
            const T* tot = sh.tot;
            if (threadIdx.x == 32) {
                pimax = tot[3];
                const double pap = (double)tot[1];
                double al = (double)tot[0] / pap;
                if (!(pap > 0.0) || !isfinite(al) || !(al > 0.0) || !isfinite((T)al)) al = 1.0;
                alpha0 = (T)al;
                sh.alpha = alpha0;
                sh.kind = (!above_tol(a, pimax) || a.max_iter <= 0) ? K_STOP1 : K_STEP1;
            }
        }
        __syncthreads();
        pw ^= 1;
    }
    int cprev = C_NONE1;      // the constraint phase whose sums the last barrier published
    bool rstep = false;       // the last rod phase formed a step (its delta is still to be stored)
    T alpha_prev = T(0);
    int db = 0;               // dU buffer the next step's rod phase writes
    int nref = 0;             // refreshes taken: the reference lives in state buffer nref & 1
    while (ok && sh.kind != K_STOP1) {
        const int pr = pw ^ 1;   // buffer the last barrier published
        if (cprev != C_NONE1) tot_fetch(o, part + pr * pstride);
        T v[4] = {T(0), T(0), T(0), T(0)};
        if (rstep) con_pass_step1(a, o, alpha_prev, db ? a.U : a.U2, v);
        const int ccur = rstep ? C_STEP1 : C_NONE1;
        warp_partial(v, sh.red);
        tot_wait();
        __syncthreads();
        if (warp == 0) {
            block_store(sh.red, part + pw * pstride, o.nbp);
        } else if (warp <= 4) {
            if (cprev != C_NONE1) warps_totals(o, nb, sh.tot);
            const T* tot = sh.tot;
            if (threadIdx.x == 32) {
                if (rstep) ++k;
                int kind = K_STEP1;
                T an = sh.alpha;
                if (cprev == C_STEP1) {
                    // sums of (s_{k-2}, y_{k-2}) and max |pi| at the iterate before the slots'
                    pimax = tot[3];
                    ++since;
                    const bool below = !above_tol(a, pimax);
                    if ((below && since >= 2) || (a.refresh > 0 && since >= a.refresh) || k >= a.max_iter) {
                        kind = K_REF1;
                    } else {
                        const T ss = tot[0], sy = tot[1], yy = tot[2];
                        an = (hist & 1) == 0 ? ss / sy : sy / yy;
                        if (!(sy > T(0)) || !isfinite(an) || !(an > T(0))) an = alpha0;
                        ++hist;
                    }
                } else if (cprev == C_REF1) {
                    // the fresh reference's exact residual: the slots' step from it is dropped on a stop
                    pimax = tot[3];
                    since = 0;
                    if (!above_tol(a, pimax) || k - 1 >= a.max_iter) {
                        kind = K_STOP1;
                        --k;
                    }
                } else if (k >= a.max_iter) {
                    kind = K_REF1;   // the cap reached before any step's sums came back
                }
                sh.alpha = an;
                sh.kind = kind;
            }
        }
        __syncthreads();
        const int kind = sh.kind;
        if (kind == K_STOP1) break;
        int cpub = ccur;
        if (kind == K_REF1) {
            fold1(a, o, nref & 1 ? a.gg1 : a.gg0, nref & 1 ? a.gg0 : a.gg1);
            ++nref;
            __syncthreads();
            rod_pass1<T, A_REF>(a, o, T(0));
            if (!(ok = barrier())) break;
            T w[4] = {T(0), T(0), T(0), T(0)};
            con_pass_ref1(a, o, w);
            warp_partial(w, sh.red);
            __syncthreads();
            if (warp == 0) block_store(sh.red, part + pw * pstride, o.nbp);
            cpub = C_REF1;
        }
        const T al = sh.alpha;
        rod_pass1<T, A_STEP>(a, o, al);
        copy_out1(db ? a.U2 : a.U, o);
        alpha_prev = al;
        rstep = true;
        db ^= 1;
        if (!(ok = barrier())) break;
        pw ^= 1;
        cprev = cpub;
    }
    if (!ok) return;
    // every solve ends on a fresh reference: gamma = gamma_ref + gamma_lo
    // (state buffer nref & 1) and delta = 0, so dU = 0
    T* gfin = nref & 1 ? a.gg1 : a.gg0;
    for (int t = threadIdx.x; t < o.nc; t += blockDim.x) st_dg(gfin, o.c0 + t, T(0), o.gref[t]);
    {
        typename V2<T>::t z;
        z.x = T(0);
        z.y = T(0);
        typename V2<T>::t* g = reinterpret_cast<typename V2<T>::t*>(a.U + 6 * (size_t)o.r0);
        for (int q = threadIdx.x; q < 3 * (o.r1 - o.r0); q += blockDim.x) g[q] = z;
    }
    if (blockIdx.x == 0 && threadIdx.x == 32) {
        a.out[1] = (double)alpha0;
        a.flags[F_FINAL] = nref & 1;
        a.flags[F_ITERS] = k;
        a.out[0] = a.hD * (double)pimax;
    }
}

// One thread block per solver block b (kNeedThreads threads): the
// one-barrier kernel's shared-memory share (ghosts counted from the block's
// other-side entries); a share whose slot or rod count exceeds the 15-bit
// local indices does not fit.
constexpr int kNeedThreads = 256;
__global__ void __launch_bounds__(kNeedThreads)
k_stage_need1(int nb, int esize, const int* __restrict__ bstart, const int* __restrict__ rowP,
              const int* __restrict__ rowQ, const int* __restrict__ qlist, unsigned long long* __restrict__ need)
{
    __shared__ int wsum[kNeedThreads / 32];
    const int b = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (b >= nb) return;   // uniform per block
    const int r0 = bstart[b], r1 = bstart[b + 1];
    const int c0 = rowP[r0], c1 = rowP[r1], q0 = rowQ[r0], q1 = rowQ[r1];
    int ng = 0;
    for (int k = q0 + (int)threadIdx.x; k < q1; k += kNeedThreads) {
        const int c = qlist[k];
        ng += c < c0 || c >= c1;
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) ng += __shfl_down_sync(0xffffffffu, ng, s);
    if (lane == 0) wsum[warp] = ng;
    __syncthreads();
    if (threadIdx.x == 0) {
        ng = 0;
        for (int w = 0; w < kNeedThreads / 32; ++w) ng += wsum[w];
        const size_t nt = (size_t)(c1 - c0) + ng, nr = r1 - r0;
        unsigned long long bytes = staged1_bytes(esize, nt, ng, nr, q1 - q0, nb);
        if (nt > (size_t)kMaxSlots || nr > (size_t)kMaxSlots) bytes = ~0ull;
        atomicMax(need, bytes);
    }
}

// Batches: every cluster takes whole systems from a queue (largest first)
// and runs the BBPGD of each on its own, with the system's own step sizes,
// residual and stopping test.  A system's rods are the contiguous ranks
// [sysoff[s], sysoff[s+1]) and its constraints the contiguous owner-major
// range they own, so each block of the cluster takes a work-balanced share
// of them exactly as the grid solver does.  The queue's entries (qent:
// system, pair code) list the largest systems twice: the two clusters that
// take them solve the system together as one group of twice the blocks (a
// pair; code = 2 * pair + member), so that no single system's solve outlasts
// the rest of the queue.  Which systems are paired depends only on the
// systems and the launch, so every step computes the same numbers.  The
// final state is left in buffer 0; per-system iterations and residuals are
// written out, and the largest of each into the step's counters.
template <typename T>
__global__ void __launch_bounds__(1024, 1)
k_bbpgd_sys(SolveArgs<T> a, const long long* __restrict__ sysoff, const int* __restrict__ qent,
            const int* __restrict__ qn, unsigned* __restrict__ pair_bar, unsigned long long* __restrict__ queue,
            int* __restrict__ sys_iters, int* __restrict__ sys_blocks, double* __restrict__ sys_res)
{
    extern __shared__ __align__(16) unsigned char dyn[];   // rod order scratch (when a.sort_ns)
    __shared__ Shared<T> sh;
    __shared__ int bounds[2];
    cg::cluster_group cl = cg::this_cluster();
    const int crank = (int)cl.block_rank(), cs = (int)cl.num_blocks();
    const int nq = *qn;
    for (;;) {
        if (crank == 0 && threadIdx.x == 0) {
            const unsigned long long k = atomicAdd(queue, 1ull);
            sh.sys = k < (unsigned long long)nq ? qent[2 * k] : -1;
            sh.pair = k < (unsigned long long)nq ? qent[2 * k + 1] : -1;
        }
        cl.sync();
        const int s = *cl.map_shared_rank(&sh.sys, 0);
        const int pc = *cl.map_shared_rank(&sh.pair, 0);
        cl.sync();   // every block has the entry before block 0 takes the next one
        if (s < 0) break;
        const int member = pc >= 0 ? (pc & 1) : 0;
        if (a.fault == 1 && member == 1) {   // test hook: a pair's second cluster never arrives
            __syncthreads();
            continue;
        }
        const int gs = pc >= 0 ? 2 * cs : cs, grank = member * cs + crank;   // the group's blocks, this one's rank
        const int R0 = (int)sysoff[s], R1 = (int)sysoff[s + 1];
        if (threadIdx.x < 64) {   // warp w finds end w of this block's share
            const int w = threadIdx.x >> 5, k = grank + w;
            const long long W0 = rank_work(a.rowP, a.rowQ, R0), W1 = rank_work(a.rowP, a.rowQ, R1);
            const int r = k == 0 ? R0 : (k == gs ? R1 : find_rank(a.rowP, a.rowQ, R0, R1, W0 + (W1 - W0) * k / gs));
            if ((threadIdx.x & 31) == 0) bounds[w] = r;
        }
        __syncthreads();
        Own<T> o;
        o.perm = nullptr;
        o.r0 = bounds[0];
        o.r1 = bounds[1];
        if (a.sort_ns && o.r1 - o.r0 <= a.sort_cap) {   // the block's share in entry-count order
            const int nr = o.r1 - o.r0;
            unsigned* key = reinterpret_cast<unsigned*>(dyn);
            int* rk = reinterpret_cast<int*>(key + nr);
            o.perm = reinterpret_cast<unsigned short*>(rk + nr);
            sort_rods(a.rowP + o.r0, a.rowQ + o.r0, nr, key, rk, o.perm);
        }
        o.c0 = a.rowP[o.r0];
        o.c1 = a.rowP[o.r1];
        o.q0 = a.rowQ[o.r0];
        o.q1 = a.rowQ[o.r1];
        o.cap_c = o.c1 - o.c0;
        o.cap_r = o.r1 - o.r0;
        o.cap_q = o.q1 - o.q0;
        BatchSync<T> sy;
        sy.bar = pc >= 0 ? pair_bar + (pc >> 1) : nullptr;
        sy.flags = a.flags;
        sy.wait_cycles = a.wait_cycles;
        sy.partials = reinterpret_cast<T*>(a.partials) + (pc >= 0 ? (size_t)(pc >> 1) * 4 * kPairBlocks : 0);
        sy.nb = (unsigned)gs;
        sy.epoch = 0;
        sy.rank = grank;
        StepState<T> st;
        solve_loop<T, false>(a, o, sh, sy, st);
        if (sh.cur == 1) {
            for (int c = o.c0 + threadIdx.x; c < o.c1; c += blockDim.x) {
                T d, g, gr, gl;
                ld_state(a.gg1, c, d, g, gr, gl);
                st_dg(a.gg0, c, d, g);
                st_ref(a.gg0, c, gr, gl);
            }
        }
        if (grank == 0 && threadIdx.x == 0) {
            sys_iters[s] = st.iters;
            sys_blocks[s] = gs;
            const double res = st.residual(a.hD);
            sys_res[s] = res;
            atomicMax(&a.flags[F_ITERS], st.iters);
            const double r = res < 0.0 ? 0.0 : res;   // a NaN stays NaN (its bits order above every number)
            atomicMax(reinterpret_cast<unsigned long long*>(a.out), (unsigned long long)__double_as_longlong(r));
        }
        __syncthreads();   // bounds and sh are rewritten for the next system
    }
}

// Queue order of the systems: descending constraint count (ties by index).
__global__ void k_sys_order(int ns, const long long* __restrict__ sysoff, const int* __restrict__ rowP,
                            int* __restrict__ order)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    const int ms = rowP[sysoff[s + 1]] - rowP[sysoff[s]];
    int pos = 0;
    for (int t = 0; t < ns; ++t) {
        const int mt = rowP[sysoff[t + 1]] - rowP[sysoff[t]];
        pos += mt > ms || (mt == ms && t < s);
    }
    order[pos] = s;
}

// The queue of the per-system solver: the first K systems of the order are
// paired (listed twice), the others listed once.  A system is paired if it
// is among the max_pairs largest, holds at least 4096 constraints per
// block of one cluster (below that the pair's grid-style barriers cost more
// than the extra blocks save) and more than half of one cluster's mean
// share of the batch's constraints.  One block; also zeroes the pairs'
// barrier counters.
__global__ void k_sys_queue(int ns, const long long* __restrict__ sysoff, const int* __restrict__ rowP,
                            const int* __restrict__ order, int nclusters, int cs, int max_pairs,
                            int* __restrict__ qent, int* __restrict__ qn, unsigned* __restrict__ pair_bar)
{
    __shared__ int npair;
    if (threadIdx.x == 0) {
        const long long total = (long long)rowP[sysoff[ns]] - rowP[sysoff[0]];
        const int cap = max_pairs;
        int k = 0;
        while (k < cap && k < ns) {
            const int sy = order[k];
            const long long m = (long long)rowP[sysoff[sy + 1]] - rowP[sysoff[sy]];
            if (m < 4096LL * cs || 2LL * nclusters * m <= total) break;
            ++k;
        }
        npair = k;
        *qn = ns + k;
    }
    __syncthreads();
    const int K = npair;
    for (int t = threadIdx.x; t < kMaxPairs; t += blockDim.x) pair_bar[t] = 0u;
    for (int e = threadIdx.x; e < ns + K; e += blockDim.x) {
        const bool paired = e < 2 * K;   // entry e = 2 * pair + member
        qent[2 * e] = paired ? order[e >> 1] : order[e - K];
        qent[2 * e + 1] = paired ? e : -1;
    }
}

// gamma back in the caller's pair order.
template <typename T>
__global__ void k_gamma_out(int m, const int* __restrict__ flags, const int* __restrict__ perm, const T* gg0,
                            const T* gg1, const double* __restrict__ scale64, double* __restrict__ out,
                            const unsigned long long* __restrict__ mdev)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= count_of(m, mdev)) return;
    if (flags[F_SOLVE_ERR] != 0) return;
    const T* g = flags[F_FINAL] == 0 ? gg0 : gg1;
    // sigma_c (gamma_ref + gamma_lo + delta): the scaled iterate mapped back
    out[perm[c]] = scale64[c] * (((double)g[4 * (size_t)c + 2] + (double)g[4 * (size_t)c + 3]) + (double)g[4 * (size_t)c]);
}

__global__ void k_rank(int n, const int* __restrict__ sorted_id, int* __restrict__ rank)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) rank[sorted_id[k]] = k;
}

cudaError_t launch_rank(aLENS_ctx* ctx, int n)
{
    if (n <= 0) return cudaSuccess;
    k_rank<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, ctx->sorted_id, ctx->rank);
    ++ctx->launches;
    return cudaGetLastError();
}

// Largest value f of type T with hD * (double)f <= tol in float64 (the
// float64 product is monotone in f, so max |pi| <= f exactly when the float64
// residual test passes); -1 when no f >= 0 passes.
template <typename T>
static T pi_threshold(double hD, double tol)
{
    if (!(hD * 0.0 <= tol)) return T(-1);
    T f = (T)(tol / hD);
    if (!(f >= T(0))) f = T(0);
    while (f > T(0) && !(hD * (double)f <= tol)) f = std::nextafter(f, T(0));
    for (;;) {
        const T g = std::nextafter(f, std::numeric_limits<T>::infinity());
        if (!(g < std::numeric_limits<T>::infinity()) || !(hD * (double)g <= tol)) break;
        f = g;
    }
    return f;
}

template <typename T>
static SolveArgs<T> make_args(aLENS_ctx* ctx, const SolveBufs<T>& sb, int n, int m)
{
    SolveArgs<T> a;
    a.n = n; a.m = m; a.np = (int)ctx->max_rods; a.mp = (int)ctx->max_pairs;
    a.rowP = ctx->rowP; a.rowQ = ctx->rowQ; a.qlist = ctx->qlist; a.ci = ctx->ci; a.cj = ctx->cj;
    a.rec = sb.rec; a.qe = sb.qe; a.q = sb.q; a.ax = sb.ax;
    a.gg0 = sb.gg[0]; a.gg1 = sb.gg[1]; a.U = sb.U; a.U2 = sb.U2; a.Uref = sb.Uref; a.gref = sb.gref;
    // float32 iterations work on increments over a reference that takes
    // the iterate every kRefresh iterations (and to confirm convergence);
    // float64 needs no refresh
    a.refresh = sizeof(T) == 4 ? kRefresh : 0;
    a.partials = ctx->partials; a.bar = ctx->bar; a.flags = ctx->dflags;
    a.out = reinterpret_cast<double*>(ctx->dcount + C_RESID);
    a.inv_perp = (T)ctx->mob.inv_perp; a.inv_par = (T)ctx->mob.inv_par;
    a.inv_rot = (T)ctx->mob.inv_rot; a.inv_spin = (T)ctx->mob.inv_spin;
    a.mobr = ctx->cur_systab ? sb.mobr : nullptr;
    a.rec_lo = sb.rec_lo; a.qe_lo = sb.qe_lo; a.q_lo = sb.q_lo;
    a.lop = sb.lop; a.loq = sb.loq;
    a.pe = sb.pe;
    a.isc = sb.isc;
    a.comp = ctx->cur_comp ? sb.comp : nullptr;
    a.hD = ctx->p.dt / ctx->p.diameter; a.tol = ctx->p.tol; a.max_iter = ctx->p.max_iter;
    a.pi_tol = pi_threshold<T>(a.hD, a.tol);
    a.wait_cycles = (long long)(ctx->wait_s * ctx->clock_khz * 1e3);
    a.fault = 0;
    a.need1_dev = nullptr;
    a.fit_cap = 0;
    a.sort_ns = 0;
    a.sort_cap = 0;
    a.zero_start = ctx->zero_start;
    a.bstart = ctx->bstart;
    return a;
}

// The global-memory solver on data beyond L2 (its records, about 100 bytes
// per constraint, and two 16-byte states stream through L2 every
// iteration): the states, which both phases read and the rod phase gathers
// through the Q-side lists, are kept in L2 by an access-policy window over
// the two state buffers (the first whole, the second up to the last
// constraint) marked persisting, with the context's persisting set-aside
// raised to hold them (as far as the device allows).  Addresses only: the
// kernel and its arithmetic are unchanged.  At 4e5 rods this takes 7 % off
// the solve.  Not while the stream is being captured (the set-aside is not
// a stream operation).
template <typename T>
static bool state_window(aLENS_ctx* ctx, const T* gg0, const T* gg1, int m, cudaAccessPolicyWindow& w)
{
    if (ctx->l2_window_off || ctx->l2_window_max <= 0 || ctx->l2_persist_max <= 0 ||
        (long long)m * 136 <= (long long)ctx->l2_bytes)
        return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return false;
    }
    const size_t used = 2 * (size_t)m * 4 * sizeof(T);
    const size_t want = used < (size_t)ctx->l2_persist_max ? used : (size_t)ctx->l2_persist_max;
    size_t cur = 0;
    if (cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (cur < want) {
        if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (!ctx->persist_set) ctx->persist_prev = cur;
        ctx->persist_set = want;
    }
    cudaCtxResetPersistingL2Cache();   // the last solve's persisting lines back to normal
    const char* base = reinterpret_cast<const char*>(gg0);
    size_t bytes = (size_t)(reinterpret_cast<const char*>(gg1 + 4 * (size_t)m) - base);
    if (bytes > (size_t)ctx->l2_window_max) bytes = (size_t)ctx->l2_window_max;
    w.base_ptr = const_cast<char*>(base);
    w.num_bytes = bytes;
    w.hitRatio = 1.0f;
    w.hitProp = cudaAccessPropertyPersisting;
    w.missProp = cudaAccessPropertyStreaming;
    return true;
}

template <typename T>
static cudaError_t solve_typed(aLENS_ctx* ctx, const SolveBufs<T>& sb, int n, int m)
{
    SolveArgs<T> a = make_args(ctx, sb, n, m);
    a.fault = ctx->fault_mode;
    ctx->fault_mode = 0;

    const int threads = ctx->solve_threads;
    const int bps = ctx->solve_bps > 0 ? ctx->solve_bps : 1;
    // enough blocks that each has at least a warp of rods
    long long want = ((long long)n + 31) / 32;
    long long blocks = (long long)bps * ctx->num_sms;
    if (want < blocks) blocks = want < 1 ? 1 : want;
    if (blocks > ctx->max_blocks) blocks = ctx->max_blocks;
    // work-balanced split, then the largest shared-memory share: stage every
    // block's data when all shares fit the opt-in budget (one readback)
    cudaError_t e;
    const int nbw = (int)blocks + 1;
    k_partition<<<(nbw * 32 + 255) / 256, 256, 0, ctx->stream>>>(n, m, (int)blocks, ctx->rowP, ctx->rowQ, ctx->bstart);
    ++ctx->launches;
    // counters C_SMEM, and C_MAXRODS and C_SMEM1 (adjacent)
    if ((e = cudaMemsetAsync(ctx->dcount + C_SMEM, 0, sizeof(unsigned long long), ctx->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(ctx->dcount + C_MAXRODS, 0, 2 * sizeof(unsigned long long), ctx->stream)) != cudaSuccess)
        return e;
    k_stage_need<<<((int)blocks + 127) / 128, 128, 0, ctx->stream>>>((int)blocks, (int)sizeof(T), ctx->bstart, ctx->rowP,
                                                                  ctx->rowQ, ctx->dcount + C_SMEM,
                                                                  ctx->dcount + C_MAXRODS);
    ++ctx->launches;
    if (ctx->solve_barriers == 1) {
        k_stage_need1<<<(int)blocks, kNeedThreads, 0, ctx->stream>>>((int)blocks, (int)sizeof(T), ctx->bstart,
                                                                      ctx->rowP, ctx->rowQ, ctx->qlist,
                                                                      ctx->dcount + C_SMEM1);
        ++ctx->launches;
    }
    // one readback of the counters C_SMEM .. C_SMEM1 (into the pinned host status
    // buffer; the allocation-free entry point has none and reads into the stack)
    unsigned long long local[C_SMEM1 - C_SMEM + 1];
    unsigned long long* hb = ctx->hcount ? ctx->hcount + C_SMEM : local;
    if ((e = cudaMemcpyAsync(hb, ctx->dcount + C_SMEM, (C_SMEM1 - C_SMEM + 1) * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, ctx->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
        return e;
    const unsigned long long need = hb[0], maxrods = hb[C_MAXRODS - C_SMEM], need1 = hb[C_SMEM1 - C_SMEM];
    const int optin = ctx->smem_optin;
    const long long budget = (long long)optin / bps - (long long)sizeof(Shared<T>) - 1024;
    if ((e = cudaMemsetAsync(ctx->bar, 0, 4 * sizeof(unsigned), ctx->stream)) != cudaSuccess) return e;
    // (warps 1-4 form the step decision: at least 160 threads)
    if (ctx->solve_barriers == 1 && threads >= 256 && need1 > 0 && (long long)need1 <= budget) {
        // one grid barrier per iteration: every block's share and its ghosts fit
        const void* fn1 = (const void*)k_bbpgd1<T>;
        const int ti = sizeof(T) == 4 ? 0 : 1;
        const long long budget1 = (long long)optin - (long long)sizeof(Shared1<T>) - 1024;   // one block per SM
        if (!ctx->attr1_set[ti]) {
            // the limit for the largest budget once; a launch asks for its own need
            if ((e = cudaFuncSetAttribute(fn1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget1)) !=
                cudaSuccess)
                return e;
            ctx->attr1_set[ti] = 1;
        }
        // occupancy only falls as shared memory grows: checked once per shape at the full budget
        const int key = threads * 64 + bps;
        if (ctx->occ1_key[ti] != key) {
            int per_sm1 = 0;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm1, fn1, threads, (size_t)budget)) !=
                cudaSuccess)
                return e;
            ctx->occ1_ok[ti] = per_sm1 >= bps;
            ctx->occ1_key[ti] = key;
        }
        if (ctx->occ1_ok[ti] && (long long)bps * ctx->num_sms >= blocks) {
            void* args1[] = {&a};
            ++ctx->launches;
            ctx->last_solver = 1;
            return cudaLaunchCooperativeKernel(fn1, dim3((unsigned)blocks), dim3(threads), args1, (size_t)need1,
                                               ctx->stream);
        }
    }
    if ((e = launch_setup_qe(ctx)) != cudaSuccess) return e;   // the two-barrier kernels read qe
    const bool staged = (long long)need <= budget && (long long)n / blocks < 60000;
    // global-memory blocks still take their rods in count order when the
    // order (10 bytes of scratch per rod) fits
    const long long sort_bytes = 10 * (long long)maxrods;
    a.sort_ns = sizeof(T) == 8 && !staged && maxrods > 0 && maxrods < 65536 && sort_bytes <= budget;
    a.sort_cap = (int)maxrods;
    const size_t smem = staged ? (size_t)need : (a.sort_ns ? (size_t)sort_bytes : 0);
    const void* fn = staged ? (const void*)k_bbpgd<T, true> : (const void*)k_bbpgd<T, false>;
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem)) != cudaSuccess) return e;
    if ((long long)per_sm * ctx->num_sms < blocks) return cudaErrorCooperativeLaunchTooLarge;
    void* args[] = {&a};
    ++ctx->launches;
    ctx->last_solver = staged ? 2 : 3;
    cudaAccessPolicyWindow win;
    if (!staged && sizeof(T) == 4 && state_window(ctx, sb.gg[0], sb.gg[1], m, win)) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        at[1].id = cudaLaunchAttributeAccessPolicyWindow;
        at[1].val.accessPolicyWindow = win;
        cfg.gridDim = dim3((unsigned)blocks);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = ctx->stream;
        cfg.attrs = at;
        cfg.numAttrs = 2;
        return cudaLaunchKernelExC(&cfg, fn, args);
    }
    return cudaLaunchCooperativeKernel(fn, dim3((unsigned)blocks), dim3(threads), args, smem, ctx->stream);
}

// Batches: the per-system solver on thread-block clusters (one launch).
template <typename T>
static cudaError_t solve_batch_typed(aLENS_ctx* ctx, const SolveBufs<T>& sb, int n, int m)
{
    SolveArgs<T> a = make_args(ctx, sb, n, m);
    a.fault = ctx->fault_mode == 1 ? 1 : 0;
    ctx->fault_mode = 0;
    const int ns = ctx->batch_n;
    cudaError_t e;
    if ((e = launch_setup_qe(ctx)) != cudaSuccess) return e;   // the per-system solver reads qe
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)ctx->batch_cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    // rod order scratch: 10 bytes per rod for twice a cluster block's even
    // share of the largest system (a block with a larger share keeps the
    // rank order); kept small, since this solver reads its data through L1
    long long max_sys = 0;
    for (int s = 0; s < ns; ++s) {
        const long long r = ctx->batch_off_host[s + 1] - ctx->batch_off_host[s];
        if (r > max_sys) max_sys = r;
    }
    const long long cap = 2 * ((max_sys + ctx->batch_cluster - 1) / ctx->batch_cluster);
    a.sort_cap = (int)(cap < 65535 ? cap : 65535);
    const long long sort_bytes = 10 * (long long)a.sort_cap;
    a.sort_ns = sizeof(T) == 8 && cap > 0 && sort_bytes <= 64 * 1024;
    const size_t smem = a.sort_ns ? (size_t)sort_bytes : 0;
    // the attribute is the largest dynamic shared memory a launch may ask
    // for: raised when a batch needs more, never lowered, so that no call is
    // made when nothing changes (a batched step may be recorded as a graph)
    static size_t smem_set[64];
    const int dv = ctx->device >= 0 && ctx->device < 64 ? ctx->device : 0;
    if (smem > smem_set[dv]) {
        if ((e = cudaFuncSetAttribute(k_bbpgd_sys<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        smem_set[dv] = smem;
    }
    cfg.blockDim = dim3((unsigned)ctx->batch_threads);
    cfg.gridDim = dim3((unsigned)ctx->batch_cluster);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int max_active = 0;
    if ((e = cudaOccupancyMaxActiveClusters(&max_active, k_bbpgd_sys<T>, &cfg)) != cudaSuccess) return e;
    if (max_active < 1) return cudaErrorInvalidConfiguration;
    int* qent = ctx->sys_order + ns;
    int* qn = qent + 2 * ((size_t)ns + kMaxPairs);
    unsigned* pair_bar = reinterpret_cast<unsigned*>(qn + 1);
    k_sys_order<<<(ns + 127) / 128, 128, 0, ctx->stream>>>(ns, ctx->sysoff, ctx->rowP, ctx->sys_order);
    ++ctx->launches;
    // Pairs wait for each other, so they need every cluster resident at
    // once: a cooperative launch (tried by the first batched solve of the
    // context; without it the solver runs without pairs).
    cudaLaunchAttribute attr2[2] = {attr[0], {}};
    attr2[1].id = cudaLaunchAttributeCooperative;
    attr2[1].val.cooperative = 1;
    for (int pass = 0; pass < 2; ++pass) {
        const int cap = max_active / 4 < kMaxPairs ? max_active / 4 : kMaxPairs;
        const int max_pairs = ctx->batch_coop != 0 ? cap : 0;
        // a cluster per queue entry at most (every system, and the pairs' second entries)
        const int nclusters = max_active < ns + max_pairs ? max_active : ns + max_pairs;
        k_sys_queue<<<1, 256, 0, ctx->stream>>>(ns, ctx->sysoff, ctx->rowP, ctx->sys_order, nclusters,
                                                ctx->batch_cluster, max_pairs, qent, qn, pair_bar);
        ++ctx->launches;
        if ((e = cudaMemsetAsync(ctx->dcount + C_QUEUE, 0, sizeof(unsigned long long), ctx->stream)) != cudaSuccess)
            return e;
        cfg.gridDim = dim3((unsigned)(nclusters * ctx->batch_cluster));
        cfg.attrs = max_pairs > 0 ? attr2 : attr;
        cfg.numAttrs = max_pairs > 0 ? 2 : 1;
        e = cudaLaunchKernelEx(&cfg, k_bbpgd_sys<T>, a, (const long long*)ctx->sysoff, (const int*)qent,
                               (const int*)qn, pair_bar, ctx->dcount + C_QUEUE, ctx->sys_iters,
                               ctx->sys_iters + ctx->max_systems, ctx->sys_res);
        if (e == cudaSuccess) {
            if (max_pairs > 0) ctx->batch_coop = 1;
            break;
        }
        // a refused cooperative cluster launch enqueued nothing: queue again without pairs
        if (max_pairs == 0 || ctx->batch_coop == 1) return e;
        cudaGetLastError();
        ctx->batch_coop = 0;
    }
    if (e != cudaSuccess) return e;
    ++ctx->launches;
    ctx->last_solver = 4;
    return cudaSuccess;
}

cudaError_t launch_solve(aLENS_ctx* ctx, int n, int m, int precision)
{
    const bool per_system = ctx->cur_systab != nullptr && ctx->batch_n > 1;
    if (precision == ALENS_MIXED)
        return per_system ? solve_batch_typed<float>(ctx, ctx->sb32, n, m) : solve_typed<float>(ctx, ctx->sb32, n, m);
    return per_system ? solve_batch_typed<double>(ctx, ctx->sb64, n, m) : solve_typed<double>(ctx, ctx->sb64, n, m);
}

// The single-system solve of a step recorded as a CUDA graph: no readback.
// The one-barrier kernel is launched with the full shared-memory budget of
// the launch shape, and its blocks check the need of the shares (computed
// on the device by k_stage_need1) against it: a share that does not fit
// makes every block leave before its first barrier with kSolveRedo in
// F_SOLVE_ERR, the update and the outputs then leave everything untouched,
// and the caller runs the step eagerly.  graph1_possible says whether the
// launch shape can take this path at all.
template <typename T>
static long long graph1_budget(const aLENS_ctx* ctx)
{
    const int bps = ctx->solve_bps > 0 ? ctx->solve_bps : 1;
    return (long long)ctx->smem_optin / bps - (long long)sizeof(Shared<T>) - 1024;
}

template <typename T>
static cudaError_t graph1_check(aLENS_ctx* ctx, bool& ok)
{
    ok = false;
    const int threads = ctx->solve_threads, bps = ctx->solve_bps > 0 ? ctx->solve_bps : 1;
    if (ctx->solve_barriers != 1 || threads < 256) return cudaSuccess;
    const void* fn1 = (const void*)k_bbpgd1<T>;
    const int ti = sizeof(T) == 4 ? 0 : 1;
    const long long budget1 = (long long)ctx->smem_optin - (long long)sizeof(Shared1<T>) - 1024;
    cudaError_t e;
    if (!ctx->attr1_set[ti]) {
        if ((e = cudaFuncSetAttribute(fn1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget1)) != cudaSuccess)
            return e;
        ctx->attr1_set[ti] = 1;
    }
    int per_sm1 = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm1, fn1, threads, (size_t)graph1_budget<T>(ctx))) !=
        cudaSuccess)
        return e;
    ok = per_sm1 >= bps;
    return cudaSuccess;
}

template <typename T>
static cudaError_t solve_graph1_typed(aLENS_ctx* ctx, const SolveBufs<T>& sb, int n, int m)
{
    SolveArgs<T> a = make_args(ctx, sb, n, m);
    const bool force_redo = ctx->fault_mode == 2;   // test hook: the recorded need never fits
    ctx->fault_mode = 0;
    const int threads = ctx->solve_threads;
    const int bps = ctx->solve_bps > 0 ? ctx->solve_bps : 1;
    long long want = ((long long)n + 31) / 32;
    long long blocks = (long long)bps * ctx->num_sms;
    if (want < blocks) blocks = want < 1 ? 1 : want;
    if (blocks > ctx->max_blocks) blocks = ctx->max_blocks;
    const long long budget = graph1_budget<T>(ctx);
    a.need1_dev = ctx->dcount + C_SMEM1;
    a.fit_cap = force_redo ? 0 : budget;
    cudaError_t e;
    const int nbw = (int)blocks + 1;
    k_partition<<<(nbw * 32 + 255) / 256, 256, 0, ctx->stream>>>(n, m, (int)blocks, ctx->rowP, ctx->rowQ, ctx->bstart);
    ++ctx->launches;
    if ((e = cudaMemsetAsync(ctx->dcount + C_SMEM1, 0, sizeof(unsigned long long), ctx->stream)) != cudaSuccess) return e;
    k_stage_need1<<<(int)blocks, kNeedThreads, 0, ctx->stream>>>((int)blocks, (int)sizeof(T), ctx->bstart,
                                                                  ctx->rowP, ctx->rowQ, ctx->qlist,
                                                                  ctx->dcount + C_SMEM1);
    ++ctx->launches;
    if ((e = cudaMemsetAsync(ctx->bar, 0, 4 * sizeof(unsigned), ctx->stream)) != cudaSuccess) return e;
    void* args1[] = {&a};
    ++ctx->launches;
    ctx->last_solver = 1;
    return cudaLaunchCooperativeKernel((const void*)k_bbpgd1<T>, dim3((unsigned)blocks), dim3(threads), args1,
                                       (size_t)budget, ctx->stream);
}

cudaError_t graph1_possible(aLENS_ctx* ctx, int precision, bool& ok)
{
    return precision == ALENS_MIXED ? graph1_check<float>(ctx, ok) : graph1_check<double>(ctx, ok);
}

cudaError_t launch_solve_graph1(aLENS_ctx* ctx, int n, int m, int precision)
{
    return precision == ALENS_MIXED ? solve_graph1_typed<float>(ctx, ctx->sb32, n, m)
                                    : solve_graph1_typed<double>(ctx, ctx->sb64, n, m);
}

cudaError_t launch_gamma_out(aLENS_ctx* ctx, int m, int precision, double* gamma_out)
{
    if (m <= 0 || !gamma_out) return cudaSuccess;
    int b = (m + 255) / 256;
    if (precision == ALENS_MIXED) {
        k_gamma_out<float><<<b, 256, 0, ctx->stream>>>(m, ctx->dflags, ctx->perm, ctx->sb32.gg[0], ctx->sb32.gg[1],
                                                       ctx->scale64, gamma_out, ctx->mdev);
    } else {
        k_gamma_out<double><<<b, 256, 0, ctx->stream>>>(m, ctx->dflags, ctx->perm, ctx->sb64.gg[0], ctx->sb64.gg[1],
                                                        ctx->scale64, gamma_out, ctx->mdev);
    }
    ++ctx->launches;
    return cudaGetLastError();
}

}  // namespace alens
