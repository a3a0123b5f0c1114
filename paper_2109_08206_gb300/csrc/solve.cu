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
//   s = gamma_{k+1} - gamma_k, y = g_{k+1} - g_k (= A s),
//   alpha_{k+1} = s.s / s.y on even k, s.y / y.y on odd k (alternating BB1/BB2),
//   alpha_0 = pi.pi / pi.A.pi for the projected gradient pi at gamma_0,
//   and alpha_0 again whenever s.y <= 0 or the step is not finite.
// Stop when (h/D) max |pi_c| <= tol (pi the projected gradient) or after
// max_iter iterations.
//
// One persistent cooperative kernel runs the whole loop, one block per SM.
// Per iteration:
//   phase A (one thread per rod, the block's rods an even share in cell
//     order): gamma_{k+1} of every constraint touching the rod is formed on
//     the fly from (gamma_k, g_k) and alpha_k (the owning rod stores it),
//     summed into the rod's force and torque F = D gamma (owned range
//     contiguous, other-side list in CSR order), and U = M F is stored;
//   grid barrier;
//   phase B (one thread per constraint, the block's owned range): g_{k+1} =
//     q + D^T U, and the partial
//     sums s.s, s.y, y.y and max |pi|: per thread and per warp in the working
//     precision, across warps and blocks in float64, in a fixed order;
//   grid barrier; warp 0 of every block then reduces the per-block partials
//     in the same fixed order, so all blocks take identical step decisions.
// Two grid barriers per iteration.  Each barrier wait is bounded in time
// and in polls; a wait that runs out raises ALENS_ERR_TIMEOUT in the device
// status word and every block leaves.
//
// Layout: (gamma, g) interleaved per constraint in two ping-pong buffers,
// U as [rod][6] (one or two sectors per gather), D records SoA [9][m].
// T = double (float64 plain) or float (mixed: the D, M, D^T work, per-thread
// and per-warp sums in float32; the cross-warp and cross-block sums, the
// residual test and the step sizes in float64; max |pi| is exact in either).
#include <float.h>

#include "internal.cuh"

namespace alens {

enum { A_RAW = 0, A_STEP = 1, A_PG = 2 };
constexpr int kRoundB = 1;  // constraints per thread and round in phase B
// CSR entries whose loads a thread issues together (float64 values need the
// registers twice over)
template <typename T> struct Batch { static constexpr int v = sizeof(T) == 4 ? 2 : 1; };

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

template <typename T>
__device__ __forceinline__ void st_u6(T* U, int i, const T u[6])
{
    typename V2<T>::t* p = reinterpret_cast<typename V2<T>::t*>(U + 6 * (size_t)i);
    typename V2<T>::t a, b, c;
    a.x = u[0]; a.y = u[1]; b.x = u[2]; b.y = u[3]; c.x = u[4]; c.y = u[5];
    p[0] = a; p[1] = b; p[2] = c;
}

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
    T* gg0;     // written inside the kernel: plain (coherent) loads only
    T* gg1;
    T* U;
    double* partials;
    unsigned* bar;
    int* flags;
    double* out;   // [0] residual, [1] alpha0
    T inv_perp, inv_par, inv_rot, inv_spin;
    double hD, tol;
    int max_iter;
    long long wait_cycles;
    int fault;
};

template <int MODE, typename T>
__device__ __forceinline__ T a_value(T g, T gr, T alpha)
{
    if (MODE == A_RAW) return g;
    if (MODE == A_STEP) {
        T v = g - alpha * gr;
        return v > T(0) ? v : T(0);
    }
    return g > T(0) ? gr : (gr < T(0) ? gr : T(0));
}

// Rod-parallel half of the gradient: F = D gamma' and U = M F for the
// block's rods [r0, r1), gamma' per MODE (A_RAW: gamma itself; A_STEP:
// max(0, gamma - alpha g), stored by the P-side rod; A_PG: the projected
// gradient, returning the thread's share of pi.A.pi = sum_rods F.M.F
// instead of storing U).  Two threads per rod: the even lane sums the rod's
// P-range (contiguous), the odd lane its Q-side list; one shuffle combines them.
template <typename T, int MODE>
__device__ __forceinline__ T phase_a(const SolveArgs<T>& a, int r0, int r1, const T* gc, T* gn, T alpha)
{
    T fmf = T(0);
    const size_t mp = a.mp, np = a.np;
    constexpr int kBatch = Batch<T>::v;
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        T F[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        {
            // the rod's own constraints: loads of up to kBatch entries issued together
            const int b = a.rowP[i], e = a.rowP[i + 1];
            for (int c = b; c < e; c += kBatch) {
                T gv[kBatch], grv[kBatch], rv[kBatch][6];
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    if (c + u < e) {
                        ld_pair(gc, c + u, gv[u], grv[u]);
#pragma unroll
                        for (int w = 0; w < 6; ++w) rv[u][w] = a.rec[w * mp + c + u];
                    }
                }
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    if (c + u < e) {
                        T v = a_value<MODE, T>(gv[u], grv[u], alpha);
                        if (MODE == A_STEP) gn[2 * (size_t)(c + u)] = v;
#pragma unroll
                        for (int w = 0; w < 6; ++w) F[w] += v * rv[u][w];
                    }
                }
            }
        }
        {
            // constraints owned by other rods: ids first, then their (gamma, g) and arms
            const int b = a.rowQ[i], e = a.rowQ[i + 1];
            for (int k = b; k < e; k += kBatch) {
                int cid[kBatch];
#pragma unroll
                for (int u = 0; u < kBatch; ++u) cid[u] = k + u < e ? a.qlist[k + u] : -1;
                T gv[kBatch], grv[kBatch], qv[kBatch][6];
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    if (cid[u] >= 0) {
                        ld_pair(gc, cid[u], gv[u], grv[u]);
#pragma unroll
                        for (int w = 0; w < 6; ++w) qv[u][w] = a.qe[w * mp + k + u];
                    }
                }
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    if (cid[u] >= 0) {
                        T v = a_value<MODE, T>(gv[u], grv[u], alpha);
#pragma unroll
                        for (int w = 0; w < 6; ++w) F[w] -= v * qv[u][w];
                    }
                }
            }
        }
        {
            T p0 = a.ax[i], p1 = a.ax[np + i], p2 = a.ax[2 * np + i];
            T pf = p0 * F[0] + p1 * F[1] + p2 * F[2];
            T pt = p0 * F[3] + p1 * F[4] + p2 * F[5];
            T cf = pf * (a.inv_par - a.inv_perp), ct = pt * (a.inv_spin - a.inv_rot);
            T Uv[6] = {F[0] * a.inv_perp + p0 * cf, F[1] * a.inv_perp + p1 * cf, F[2] * a.inv_perp + p2 * cf,
                       F[3] * a.inv_rot + p0 * ct,  F[4] * a.inv_rot + p1 * ct,  F[5] * a.inv_rot + p2 * ct};
            if (MODE == A_PG) {
#pragma unroll
                for (int u = 0; u < 6; ++u) fmf += F[u] * Uv[u];
            } else {
                st_u6(a.U, i, Uv);
            }
        }
    }
    return fmf;
}

// Constraint-parallel half: g_new = q + D^T U, written into the y slot of
// the new (gamma, g) pair, plus the thread's partial sums.
// FIRST: acc0 = pi.pi; otherwise acc0..2 = s.s, s.y, y.y; acc3 = max |pi|.
template <typename T, bool FIRST>
__device__ __forceinline__ void phase_b(const SolveArgs<T>& a, int c0, int c1, T* gnew, const T* gold, T acc[4])
{
    const size_t mp = a.mp;
    const int nt = blockDim.x;
    // two constraints per thread and round; every load of both is issued
    // before the first store
    for (int cA = c0 + threadIdx.x; cA < c1; cA += kRoundB * nt) {
        const int cB = cA + nt;
        const bool hasB = kRoundB > 1 && cB < c1;
        int idx[2] = {cA, hasB ? cB : cA};
        T Ui[2][6], Uj[2][6], r[2][9], qq[2], gm[2], go[2], gro[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = idx[h];
            ld_u6(a.U, a.ci[c], Ui[h]);
            ld_u6(a.U, a.cj[c], Uj[h]);
#pragma unroll
            for (int w = 0; w < 9; ++w) r[h][w] = a.rec[w * mp + c];
            qq[h] = a.q[c];
            gm[h] = gnew[2 * (size_t)c];
            if (!FIRST) ld_pair(gold, c, go[h], gro[h]);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && !hasB) break;
            const int c = idx[h];
            T du = T(0);
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                du += r[h][u] * (Ui[h][u] - Uj[h][u]);
                du += r[h][3 + u] * Ui[h][3 + u];
                du -= r[h][6 + u] * Uj[h][3 + u];
            }
            const T gr = qq[h] + du;
            gnew[2 * (size_t)c + 1] = gr;
            const T g1 = gm[h];
            T pi = g1 > T(0) ? gr : (gr < T(0) ? gr : T(0));
            T api = pi < T(0) ? -pi : pi;
            acc[3] = api > acc[3] ? api : acc[3];
            if (FIRST) {
                acc[0] += pi * pi;
            } else {
                T sv = g1 - go[h], yv = gr - gro[h];
                acc[0] += sv * sv;
                acc[1] += sv * yv;
                acc[2] += yv * yv;
            }
        }
    }
}

// Block partial of (sum, sum, sum, max): warp shuffles in T, then warp 0
// combines the warp results in float64 and lane 0 stores them.  Fixed order.
template <typename T>
__device__ __forceinline__ void block_partial(T v[4], double (*red)[4], double* dst)
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
        for (int u = 0; u < 4; ++u) red[warp][u] = (double)v[u];
    }
    __syncthreads();
    if (warp == 0) {
        double w[4] = {0.0, 0.0, 0.0, 0.0};
        if (lane < nw) {
#pragma unroll
            for (int u = 0; u < 4; ++u) w[u] = red[lane][u];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int u = 0; u < 3; ++u) w[u] += __shfl_down_sync(0xffffffffu, w[u], o);
            double mx = __shfl_down_sync(0xffffffffu, w[3], o);
            w[3] = mx > w[3] ? mx : w[3];
        }
        if (lane == 0) {
#pragma unroll
            for (int u = 0; u < 4; ++u) dst[u] = w[u];
        }
    }
}

// Bounded grid barrier on a monotone arrival counter: block b's k-th arrival
// waits until the counter reaches k * gridDim.x.  The wait gives up after
// wait_cycles clock cycles or 2^28 polls, records ALENS_ERR_TIMEOUT and
// returns false; it also returns false as soon as any block has recorded an
// error, so every block leaves.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned target, int* flags, long long wait_cycles)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        long long t0 = clock64();
        for (unsigned polls = 0;; ++polls) {
            unsigned v = ld_acquire_u32(count);
            if ((int)(v - target) >= 0) break;
            if (ld_volatile_i32(&flags[F_SOLVE_ERR]) != 0) break;
            if (clock64() - t0 > wait_cycles || polls > (1u << 28)) {
                atomicCAS(&flags[F_SOLVE_ERR], 0, ALENS_ERR_TIMEOUT);
                break;
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ld_volatile_i32(&flags[F_SOLVE_ERR]) == 0;
}

// After a barrier: warp 0 reduces the per-block partials in float64 in a
// fixed order and broadcasts the four totals through shared memory.
__device__ __forceinline__ void grid_total(const double* partials, int nb, double* bc, double out[4])
{
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double w[4] = {0.0, 0.0, 0.0, 0.0};
        for (int b = lane; b < nb; b += 32) {
            const volatile double* pb = partials + 4 * (size_t)b;
            w[0] += pb[0];
            w[1] += pb[1];
            w[2] += pb[2];
            double mx = pb[3];
            w[3] = mx > w[3] ? mx : w[3];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int u = 0; u < 3; ++u) w[u] += __shfl_down_sync(0xffffffffu, w[u], o);
            double mx = __shfl_down_sync(0xffffffffu, w[3], o);
            w[3] = mx > w[3] ? mx : w[3];
        }
        if (lane == 0) {
#pragma unroll
            for (int u = 0; u < 4; ++u) bc[u] = w[u];
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) out[u] = bc[u];
}

// Step-size bookkeeping, done by thread 0 alone (float64 division is slow
// on this part; every other thread only reads the broadcast).
struct StepState {
    double alpha0, alpha, res;
    int iters, cur, done;
};

template <typename T>
__global__ void __launch_bounds__(1024, 1) k_bbpgd(SolveArgs<T> a)
{
    __shared__ double red[32][4];
    __shared__ double bc[4];
    __shared__ T s_alpha;
    __shared__ int s_done;
    if (a.fault == 1 && blockIdx.x == 0) return;   // test hook: this block never arrives
    const unsigned nb = gridDim.x;
    double* mine = a.partials + 4 * (size_t)blockIdx.x;
    unsigned epoch = 0;
    // this block's rods (an even split) and the P-side constraints they own
    const int per = (a.n + (int)nb - 1) / (int)nb;
    const int r0 = min(a.n, (int)blockIdx.x * per), r1 = min(a.n, r0 + per);
    const int c0 = a.rowP[r0], c1 = a.rowP[r1];
    double tot[4];
    T v[4];
    StepState st;   // meaningful in thread 0 only

    // U = M D gamma_0
    phase_a<T, A_RAW>(a, r0, r1, a.gg0, nullptr, T(0));
    if (!grid_barrier(a.bar, nb * ++epoch, a.flags, a.wait_cycles)) return;
    // g_0 and the projected gradient at gamma_0
    v[0] = v[1] = v[2] = v[3] = T(0);
    phase_b<T, true>(a, c0, c1, a.gg0, nullptr, v);
    block_partial(v, red, mine);
    if (!grid_barrier(a.bar, nb * ++epoch, a.flags, a.wait_cycles)) return;
    grid_total(a.partials, nb, bc, tot);
    if (threadIdx.x == 0) {
        st.res = a.hD * tot[3];
        st.iters = 0;
        st.cur = 0;
        st.done = !(st.res > a.tol && a.max_iter > 0);
        s_done = st.done;
    }
    __syncthreads();
    if (!s_done) {
        const double pp = tot[0];
        // alpha_0 = pi.pi / pi.A.pi (exact line step along the projected gradient)
        v[0] = phase_a<T, A_PG>(a, r0, r1, a.gg0, nullptr, T(0));
        v[1] = v[2] = v[3] = T(0);
        // every block has read the partials (grid_total) before any rewrites them
        if (!grid_barrier(a.bar, nb * ++epoch, a.flags, a.wait_cycles)) return;
        block_partial(v, red, mine);
        if (!grid_barrier(a.bar, nb * ++epoch, a.flags, a.wait_cycles)) return;
        grid_total(a.partials, nb, bc, tot);
        if (threadIdx.x == 0) {
            const double pap = tot[0];
            double alpha0 = pp / pap;
            if (!(pap > 0.0) || !isfinite(alpha0) || !(alpha0 > 0.0)) alpha0 = 1.0;
            st.alpha0 = st.alpha = alpha0;
            s_alpha = (T)alpha0;
        }
        __syncthreads();
        int cur = 0;
        for (int k = 0; k < a.max_iter; ++k) {
            const int nx = cur ^ 1;
            T* gc = cur ? a.gg1 : a.gg0;
            T* gn = cur ? a.gg0 : a.gg1;
            phase_a<T, A_STEP>(a, r0, r1, gc, gn, s_alpha);
            if (!grid_barrier(a.bar, nb * ++epoch, a.flags, a.wait_cycles)) return;
            v[0] = v[1] = v[2] = v[3] = T(0);
            phase_b<T, false>(a, c0, c1, gn, gc, v);
            block_partial(v, red, mine);
            if (!grid_barrier(a.bar, nb * ++epoch, a.flags, a.wait_cycles)) return;
            grid_total(a.partials, nb, bc, tot);
            cur = nx;
            if (threadIdx.x == 0) {
                const double ss = tot[0], sy = tot[1], yy = tot[2];
                st.res = a.hD * tot[3];
                st.cur = cur;
                st.iters = k + 1;
                st.done = !(st.res > a.tol);
                if (!st.done) {
                    double an = (k & 1) == 0 ? ss / sy : sy / yy;
                    if (!(sy > 0.0) || !isfinite(an) || !(an > 0.0)) an = st.alpha0;
                    st.alpha = an;
                    s_alpha = (T)an;
                }
                s_done = st.done;
            }
            __syncthreads();
            if (s_done) break;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) a.out[1] = st.alpha0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.flags[F_FINAL] = st.cur;
        a.flags[F_ITERS] = st.iters;
        a.out[0] = st.res;
    }
}

// gamma back in the caller's pair order.
template <typename T>
__global__ void k_gamma_out(int m, const int* __restrict__ flags, const int* __restrict__ perm, const T* gg0,
                            const T* gg1, double* __restrict__ out)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    if (flags[F_SOLVE_ERR] != 0) return;
    const T* g = flags[F_FINAL] == 0 ? gg0 : gg1;
    out[perm[c]] = (double)g[2 * (size_t)c];
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

template <typename T>
static cudaError_t solve_typed(aLENS_ctx* ctx, const SolveBufs<T>& sb, int n, int m)
{
    SolveArgs<T> a;
    a.n = n; a.m = m; a.np = (int)ctx->max_rods; a.mp = (int)ctx->max_pairs;
    a.rowP = ctx->rowP; a.rowQ = ctx->rowQ; a.qlist = ctx->qlist; a.ci = ctx->ci; a.cj = ctx->cj;
    a.rec = sb.rec; a.qe = sb.qe; a.q = sb.q; a.ax = sb.ax;
    a.gg0 = sb.gg[0]; a.gg1 = sb.gg[1]; a.U = sb.U;
    a.partials = ctx->partials; a.bar = ctx->bar; a.flags = ctx->dflags;
    a.out = reinterpret_cast<double*>(ctx->dcount + C_RESID);
    a.inv_perp = (T)ctx->mob.inv_perp; a.inv_par = (T)ctx->mob.inv_par;
    a.inv_rot = (T)ctx->mob.inv_rot; a.inv_spin = (T)ctx->mob.inv_spin;
    a.hD = ctx->p.dt / ctx->p.diameter; a.tol = ctx->p.tol; a.max_iter = ctx->p.max_iter;
    a.wait_cycles = (long long)(ctx->wait_s * ctx->clock_khz * 1e3);
    a.fault = ctx->fault_mode;
    ctx->fault_mode = 0;

    int threads = ctx->solve_threads;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bbpgd<T>, threads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (ctx->solve_bps > 0 && ctx->solve_bps < per_sm) per_sm = ctx->solve_bps;
    // enough blocks that each has at least a warp of rods
    long long want = ((long long)n + 31) / 32;
    long long blocks = (long long)per_sm * ctx->num_sms;
    if (want < blocks) blocks = want < 1 ? 1 : want;
    if (blocks > ctx->max_blocks) blocks = ctx->max_blocks;
    if ((e = cudaMemsetAsync(ctx->bar, 0, 4 * sizeof(unsigned), ctx->stream)) != cudaSuccess) return e;
    void* args[] = {&a};
    ++ctx->launches;
    return cudaLaunchCooperativeKernel((const void*)k_bbpgd<T>, dim3((unsigned)blocks), dim3(threads), args, 0,
                                       ctx->stream);
}

cudaError_t launch_solve(aLENS_ctx* ctx, int n, int m, int precision)
{
    if (precision == ALENS_MIXED) return solve_typed<float>(ctx, ctx->sb32, n, m);
    return solve_typed<double>(ctx, ctx->sb64, n, m);
}

cudaError_t launch_gamma_out(aLENS_ctx* ctx, int m, int precision, double* gamma_out)
{
    if (m <= 0 || !gamma_out) return cudaSuccess;
    int b = (m + 255) / 256;
    if (precision == ALENS_MIXED) {
        k_gamma_out<float><<<b, 256, 0, ctx->stream>>>(m, ctx->dflags, ctx->perm, ctx->sb32.gg[0], ctx->sb32.gg[1], gamma_out);
    } else {
        k_gamma_out<double><<<b, 256, 0, ctx->stream>>>(m, ctx->dflags, ctx->perm, ctx->sb64.gg[0], ctx->sb64.gg[1], gamma_out);
    }
    ++ctx->launches;
    return cudaGetLastError();
}

}  // namespace alens
