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
// One persistent cooperative kernel runs the whole loop.  Per iteration:
//   phase A (one thread per rod): gamma_{k+1} of every constraint touching
//     the rod is formed on the fly from gamma_k, g_k and alpha_k (the P-side
//     rod stores it), summed into the rod's force and torque F = D gamma
//     (P-range contiguous, Q-side list in CSR order), and U = M F is stored;
//   grid barrier;
//   phase B (one thread per constraint): g_{k+1} = q + D^T U, plus the four
//     float64 partial reductions s.s, s.y, y.y and max |pi|, reduced per block
//     with warp shuffles in a fixed order;
//   grid barrier; every block then reduces the per-block partials in the
//     same fixed order, so all blocks take identical step decisions.
// Two grid barriers per iteration.  Each barrier wait is bounded in time
// and iterations; a wait that runs out raises ALENS_ERR_TIMEOUT in the
// device status word and every block leaves.
// T = double (float64 plain) or float (mixed: the D, M, D^T work in float32,
// every reduction and the residual in float64).
#include <float.h>

#include "internal.cuh"

namespace alens {

enum { A_RAW = 0, A_STEP = 1, A_PG = 2 };

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
    T* gam0;    // written inside the kernel: no __restrict__/const (no non-coherent loads)
    T* gam1;
    T* grad0;
    T* grad1;
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

template <typename T, int MODE>
__device__ __forceinline__ double phase_a(const SolveArgs<T>& a, const T* gc, const T* grc, T* gn, T alpha)
{
    double fmf = 0.0;
    const int stride = gridDim.x * blockDim.x;
    const size_t mp = a.mp, np = a.np;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        T F[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        int b = a.rowP[i], e = a.rowP[i + 1];
        for (int c = b; c < e; ++c) {
            T v = a_value<MODE, T>(gc[c], grc[c], alpha);
            if (MODE == A_STEP) gn[c] = v;
#pragma unroll
            for (int u = 0; u < 6; ++u) F[u] += v * a.rec[u * mp + c];
        }
        b = a.rowQ[i];
        e = a.rowQ[i + 1];
        for (int k = b; k < e; ++k) {
            int c = a.qlist[k];
            T v = a_value<MODE, T>(gc[c], grc[c], alpha);
#pragma unroll
            for (int u = 0; u < 6; ++u) F[u] -= v * a.qe[u * mp + k];
        }
        T p0 = a.ax[i], p1 = a.ax[np + i], p2 = a.ax[2 * np + i];
        T pf = p0 * F[0] + p1 * F[1] + p2 * F[2];
        T pt = p0 * F[3] + p1 * F[4] + p2 * F[5];
        T cf = pf * (a.inv_par - a.inv_perp), ct = pt * (a.inv_spin - a.inv_rot);
        T Uv[6] = {F[0] * a.inv_perp + p0 * cf, F[1] * a.inv_perp + p1 * cf, F[2] * a.inv_perp + p2 * cf,
                   F[3] * a.inv_rot + p0 * ct,  F[4] * a.inv_rot + p1 * ct,  F[5] * a.inv_rot + p2 * ct};
        if (MODE == A_PG) {
#pragma unroll
            for (int u = 0; u < 6; ++u) fmf += (double)F[u] * (double)Uv[u];
        } else {
#pragma unroll
            for (int u = 0; u < 6; ++u) a.U[u * np + i] = Uv[u];
        }
    }
    return fmf;
}

// g_new = q + D^T U for every constraint, plus the partial reductions:
// FIRST: acc0 = pi.pi, acc3 = max |pi|; otherwise acc0..2 = s.s, s.y, y.y,
// acc3 = max |pi|, with s = gnew - gold and y = grnew - grold.
template <typename T, bool FIRST>
__device__ __forceinline__ void phase_b(const SolveArgs<T>& a, const T* gnew, const T* gold, const T* grold,
                                        T* grnew, double acc[4])
{
    const int stride = gridDim.x * blockDim.x;
    const size_t mp = a.mp, np = a.np;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.m; c += stride) {
        int i = a.ci[c], j = a.cj[c];
        T du = T(0);
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            T e = a.rec[u * mp + c];
            du += e * (a.U[u * np + i] - a.U[u * np + j]);
            du += a.rec[(3 + u) * mp + c] * a.U[(3 + u) * np + i];
            du -= a.rec[(6 + u) * mp + c] * a.U[(3 + u) * np + j];
        }
        T gr = a.q[c] + du;
        grnew[c] = gr;
        T gm = gnew[c];
        T pi = gm > T(0) ? gr : (gr < T(0) ? gr : T(0));
        double api = fabs((double)pi);
        acc[3] = api > acc[3] ? api : acc[3];
        if (FIRST) {
            acc[0] += (double)pi * (double)pi;
        } else {
            double s = (double)gm - (double)gold[c];
            double y = (double)gr - (double)grold[c];
            acc[0] += s * s;
            acc[1] += s * y;
            acc[2] += y * y;
        }
    }
}

// Block reduction of 4 values (sums in 0..2, max in 3); result broadcast to
// every thread through shared memory.  Fixed order: deterministic.
__device__ __forceinline__ void block_reduce4(double v[4], double (*red)[4], double* bc)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int u = 0; u < 3; ++u) v[u] += __shfl_down_sync(0xffffffffu, v[u], o);
        double m = __shfl_down_sync(0xffffffffu, v[3], o);
        v[3] = m > v[3] ? m : v[3];
    }
    if (lane == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) red[warp][u] = v[u];
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
            double m = __shfl_down_sync(0xffffffffu, w[3], o);
            w[3] = m > w[3] ? m : w[3];
        }
        if (lane == 0) {
#pragma unroll
            for (int u = 0; u < 4; ++u) bc[u] = w[u];
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = bc[u];
    __syncthreads();
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

// Every block reduces the per-block partials in the same fixed order.
__device__ __forceinline__ void grid_reduce4(const double* partials, int nb, double v[4], double (*red)[4],
                                             double* bc)
{
    v[0] = v[1] = v[2] = v[3] = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const volatile double* pb = partials + 4 * (size_t)b;
        v[0] += pb[0];
        v[1] += pb[1];
        v[2] += pb[2];
        double m = pb[3];
        v[3] = m > v[3] ? m : v[3];
    }
    block_reduce4(v, red, bc);
}

template <typename T>
__global__ void __launch_bounds__(512) k_bbpgd(SolveArgs<T> a)
{
    __shared__ double red[32][4];
    __shared__ double bc[4];
    if (a.fault == 1 && blockIdx.x == 0) return;   // test hook: this block never arrives
    const unsigned nb = gridDim.x;
    unsigned epoch = 0;
    T* gam[2] = {a.gam0, a.gam1};
    T* grad[2] = {a.grad0, a.grad1};
    double v[4];

    // U = M D gamma_0
    phase_a<T, A_RAW>(a, gam[0], grad[0], nullptr, T(0));
    if (!grid_barrier(a.bar, nb * ++epoch, a.flags, a.wait_cycles)) return;
    // g_0 and the projected gradient at gamma_0
    v[0] = v[1] = v[2] = v[3] = 0.0;
    phase_b<T, true>(a, gam[0], nullptr, nullptr, grad[0], v);
    block_reduce4(v, red, bc);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) a.partials[4 * (size_t)blockIdx.x + u] = v[u];
    }
    if (!grid_barrier(a.bar, nb * ++epoch, a.flags, a.wait_cycles)) return;
    grid_reduce4(a.partials, nb, v, red, bc);
    const double pp = v[0];
    double res = a.hD * v[3];
    int cur = 0, iters = 0;
    if (res > a.tol && a.max_iter > 0) {
        // alpha_0 = pi.pi / pi.A.pi (exact line step along the projected gradient)
        double fmf = phase_a<T, A_PG>(a, gam[0], grad[0], nullptr, T(0));
        v[0] = fmf; v[1] = v[2] = v[3] = 0.0;
        block_reduce4(v, red, bc);
        if (!grid_barrier(a.bar, nb * ++epoch, a.flags, a.wait_cycles)) return;   // all reads of partials done
        if (threadIdx.x == 0) a.partials[4 * (size_t)blockIdx.x] = v[0];
        if (threadIdx.x == 0) {
            a.partials[4 * (size_t)blockIdx.x + 1] = 0.0;
            a.partials[4 * (size_t)blockIdx.x + 2] = 0.0;
            a.partials[4 * (size_t)blockIdx.x + 3] = 0.0;
        }
        if (!grid_barrier(a.bar, nb * ++epoch, a.flags, a.wait_cycles)) return;
        grid_reduce4(a.partials, nb, v, red, bc);
        const double pap = v[0];
        double alpha0 = pp / pap;
        if (!(pap > 0.0) || !isfinite(alpha0) || !(alpha0 > 0.0)) alpha0 = 1.0;
        double alpha = alpha0;
        for (int k = 0; k < a.max_iter; ++k) {
            const int nx = cur ^ 1;
            phase_a<T, A_STEP>(a, gam[cur], grad[cur], gam[nx], (T)alpha);
            if (!grid_barrier(a.bar, nb * ++epoch, a.flags, a.wait_cycles)) return;
            v[0] = v[1] = v[2] = v[3] = 0.0;
            phase_b<T, false>(a, gam[nx], gam[cur], grad[cur], grad[nx], v);
            block_reduce4(v, red, bc);
            if (threadIdx.x == 0) {
#pragma unroll
                for (int u = 0; u < 4; ++u) a.partials[4 * (size_t)blockIdx.x + u] = v[u];
            }
            if (!grid_barrier(a.bar, nb * ++epoch, a.flags, a.wait_cycles)) return;
            grid_reduce4(a.partials, nb, v, red, bc);
            const double ss = v[0], sy = v[1], yy = v[2];
            res = a.hD * v[3];
            cur = nx;
            iters = k + 1;
            if (!(res > a.tol)) break;
            double an = (k & 1) == 0 ? ss / sy : sy / yy;
            if (!(sy > 0.0) || !isfinite(an) || !(an > 0.0)) an = alpha0;
            alpha = an;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) a.out[1] = alpha0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.flags[F_FINAL] = cur;
        a.flags[F_ITERS] = iters;
        a.out[0] = res;
    }
}

template <typename T>
__global__ void k_gamma_out(int m, const int* __restrict__ flags, const T* g0, const T* g1, double* __restrict__ out)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    if (flags[F_SOLVE_ERR] != 0) return;
    const T* g = flags[F_FINAL] == 0 ? g0 : g1;
    out[c] = (double)g[c];
}

template <typename T>
static cudaError_t solve_typed(aLENS_ctx* ctx, const SolveBufs<T>& sb, int n, int m)
{
    SolveArgs<T> a;
    a.n = n; a.m = m; a.np = (int)ctx->max_rods; a.mp = (int)ctx->max_pairs;
    a.rowP = ctx->rowP; a.rowQ = ctx->rowQ; a.qlist = ctx->qlist; a.ci = ctx->ci; a.cj = ctx->cj;
    a.rec = sb.rec; a.qe = sb.qe; a.q = sb.q; a.ax = sb.ax;
    a.gam0 = sb.gam[0]; a.gam1 = sb.gam[1]; a.grad0 = sb.grad[0]; a.grad1 = sb.grad[1]; a.U = sb.U;
    a.partials = ctx->partials; a.bar = ctx->bar; a.flags = ctx->dflags;
    a.out = reinterpret_cast<double*>(ctx->dcount + 4);
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
    long long want = ((long long)(n > m ? n : m) + threads - 1) / threads;
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
        k_gamma_out<float><<<b, 256, 0, ctx->stream>>>(m, ctx->dflags, ctx->sb32.gam[0], ctx->sb32.gam[1], gamma_out);
        ++ctx->launches;
    } else {
        k_gamma_out<double><<<b, 256, 0, ctx->stream>>>(m, ctx->dflags, ctx->sb64.gam[0], ctx->sb64.gam[1], gamma_out);
        ++ctx->launches;
    }
    return cudaGetLastError();
}

}  // namespace alens
