// Multi-step trajectories: confining walls, Brownian forces and the warm
// start of the constraint forces from the previous step.
//
// Walls (Appendix: a collision with an external boundary keeps only the
// particle's side of the column): two flat walls normal to one axis at
// coordinates lo < hi.  The lowest point of a segment over a plane is one of
// its ends (both when it lies flat), so each end y = s p, s = -L/2 and
// +L/2, is a contact candidate with each wall: gap Phi = x_w + s p_w - lo -
// D/2 and normal +e_w for the lower wall, Phi = hi - x_w - s p_w - D/2 and
// -e_w for the upper one.  Each candidate with Phi < delta_c is a one-sided
// row (i, -1, 2 side + end) placed after the collisions, in (rod, side, end)
// order.
//
// Brownian forces (the paper's F_B, drawn from a counter-based generator so
// that every step is reproducible on its own): Philox4x32-10 (Salmon,
// Moraes, Dror & Shaw, SC'11) with key = seed and counters (rod, step, w),
// uniforms (x + 0.5) 2^-32, Box-Muller pairs, and the force and torque
// sqrt(2 kT / h) [sqrt(zeta_par) (p.xi) p + sqrt(zeta_perp) (xi - (p.xi) p)]
// (rotation with zeta_spin, zeta_rot): covariance 2 kT M^-1 / h, so that the
// step's displacement has covariance 2 kT h M (fluctuation-dissipation).
//
// Warm start: every row of a step gets the previous step's force of the same
// constraint - a collision (i, j, image) or a wall contact (i, wall, end)
// found by binary search in the previous step's sorted keys, a spring by its
// index while the spring list is unchanged - and 0 otherwise.
#include <math.h>

#include "internal.cuh"

namespace alens {

namespace {

__device__ __forceinline__ void philox4x32(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

__device__ __forceinline__ void words8(unsigned long long seed, unsigned long long step, int i, uint32_t w[8])
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t c[4] = {(uint32_t)i, (uint32_t)step, (uint32_t)(step >> 32), (uint32_t)h};
        philox4x32(c, (uint32_t)seed, (uint32_t)(seed >> 32));
#pragma unroll
        for (int k = 0; k < 4; ++k) w[4 * h + k] = c[k];
    }
}

}  // namespace

__global__ void k_random_words(int n, unsigned long long seed, unsigned long long step, uint32_t* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t w[8];
    words8(seed, step, i, w);
#pragma unroll
    for (int k = 0; k < 8; ++k) out[8 * (size_t)i + k] = w[k];
}

__global__ void k_brownian(int n, Mob mob, double kT, double dt, unsigned long long seed, unsigned long long step,
                           const double* __restrict__ quat, const double* __restrict__ fext, double* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t w[8];
    words8(seed, step, i, w);
    double z[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double u1 = ((double)w[2 * k] + 0.5) * (1.0 / 4294967296.0);
        const double u2 = ((double)w[2 * k + 1] + 0.5) * (1.0 / 4294967296.0);
        const double r = sqrt(-2.0 * log(u1));
        z[2 * k] = r * cos(2.0 * M_PI * u2);
        z[2 * k + 1] = r * sin(2.0 * M_PI * u2);
    }
    double p0, p1, p2;
    quat_axis(quat[4 * (size_t)i], quat[4 * (size_t)i + 1], quat[4 * (size_t)i + 2], quat[4 * (size_t)i + 3], p0, p1,
              p2);
    const double p[3] = {p0, p1, p2};
    const double a = sqrt(2.0 * kT / dt);
    // drag coefficients zeta = 1 / (inverse drag)
    const double sp = sqrt(1.0 / mob.inv_par), sq = sqrt(1.0 / mob.inv_perp);
    const double ss = sqrt(1.0 / mob.inv_spin), sr = sqrt(1.0 / mob.inv_rot);
    const double pt = p[0] * z[0] + p[1] * z[1] + p[2] * z[2];
    const double pr = p[0] * z[3] + p[1] * z[4] + p[2] * z[5];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const double ft = a * (sp * pt * p[m] + sq * (z[m] - pt * p[m]));
        const double fr = a * (ss * pr * p[m] + sr * (z[3 + m] - pr * p[m]));
        out[6 * (size_t)i + m] = (fext ? fext[6 * (size_t)i + m] : 0.0) + ft;
        out[6 * (size_t)i + 3 + m] = (fext ? fext[6 * (size_t)i + 3 + m] : 0.0) + fr;
    }
}

// Per rod: how many wall contact candidates it has (0-4), and the total.
__global__ void k_count_walls(int n, int np, int axis_w, double lo, double hi, double half, double diameter,
                              double delta_c, const double* __restrict__ xw, const double* __restrict__ axis,
                              int* __restrict__ cnt, unsigned long long* __restrict__ counters)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int c = 0;
    if (i < n) {
        const double pw = axis[axis_w * (size_t)np + i], x = xw[axis_w * (size_t)np + i];
        for (int end = 0; end < 2; ++end) {
            const double tip = x + (end == 0 ? -half : half) * pw;
            if (tip - lo - 0.5 * diameter < delta_c) ++c;
            if (hi - tip - 0.5 * diameter < delta_c) ++c;
        }
        cnt[i] = c;
    }
    unsigned long long tot = (unsigned long long)c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, o);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(&counters[C_WALLS], tot);
}

// Rows row0 + start[i] .. of rod i's wall contacts.
__global__ void k_emit_walls(int n, int np, int row0, int axis_w, double lo, double hi, double half, double diameter,
                             double delta_c, double dt, const double* __restrict__ xw, const double* __restrict__ axis,
                             const double* __restrict__ unc, const int* __restrict__ start, int32_t* __restrict__ pairs,
                             double* __restrict__ phi, double* __restrict__ dgeom, double* __restrict__ q,
                             unsigned long long* __restrict__ counters)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double p[3] = {axis[i], axis[np + i], axis[2 * (size_t)np + i]};
    const double pw = p[axis_w], x = xw[axis_w * (size_t)np + i];
    int row = row0 + start[i];
    for (int side = 0; side < 2; ++side)
        for (int end = 0; end < 2; ++end) {
            const double sg = side == 0 ? 1.0 : -1.0;   // normal into the domain
            const double s = end == 0 ? -half : half;
            const double tip = x + s * pw;
            const double ph = side == 0 ? tip - lo - 0.5 * diameter : hi - tip - 0.5 * diameter;
            if (!(ph < delta_c)) continue;
            double e[3] = {0.0, 0.0, 0.0};
            e[axis_w] = sg;
            const double y[3] = {s * p[0], s * p[1], s * p[2]};
            const double ye[3] = {y[1] * e[2] - y[2] * e[1], y[2] * e[0] - y[0] * e[2], y[0] * e[1] - y[1] * e[0]};
            double* dg = dgeom + 9 * (size_t)row;
            double dtu = 0.0;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                dg[m] = e[m];
                dg[3 + m] = ye[m];
                dg[6 + m] = 0.0;
                dtu += e[m] * unc[m * (size_t)np + i] + ye[m] * unc[(3 + m) * (size_t)np + i];
            }
            pairs[3 * (size_t)row] = i;
            pairs[3 * (size_t)row + 1] = -1;
            pairs[3 * (size_t)row + 2] = 2 * side + end;
            phi[row] = ph;
            q[row] = ph / dt + dtu;
            if (ph < 0.0) atomicAdd(&counters[C_OVERLAP], 1ull);
            const long long b = __double_as_longlong(ph);
            atomicMin((long long*)&counters[C_MINGAP], b >= 0 ? b : b ^ 0x7fffffffffffffffLL);
            ++row;
        }
}

// Keys of the rows: collisions and wall contacts (i, j or 0, image or
// 2 side + end) packed so that the emitted order is ascending; springs by
// index.
__global__ void k_row_keys(int m, int mu, int mw, const int32_t* __restrict__ pairs,
                           unsigned long long* __restrict__ keys)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    unsigned long long k;
    if (r < mu + mw) {
        const unsigned i = (unsigned)pairs[3 * (size_t)r];
        const int j = pairs[3 * (size_t)r + 1];
        const unsigned code = (unsigned)pairs[3 * (size_t)r + 2];
        k = ((unsigned long long)i << 32) | ((unsigned long long)(r < mu ? (unsigned)j : 0u) << 5) | code;
    } else {
        k = (unsigned long long)(r - mu - mw);
    }
    keys[r] = k;
}

__device__ __forceinline__ int find_key(const unsigned long long* keys, int lo, int hi, unsigned long long k)
{
    while (lo < hi) {   // first index in [lo, hi) with keys >= k
        const int mid = (lo + hi) >> 1;
        if (keys[mid] < k) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// gamma_in of every row from the previous step's (keys, gamma).
__global__ void k_warm(int m, int mu, int mw, const unsigned long long* __restrict__ keys,
                       const unsigned long long* __restrict__ pkeys, const double* __restrict__ pgam, int pmu, int pmw,
                       int pms, int springs_same, double* __restrict__ gin)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    const unsigned long long k = keys[r];
    double g = 0.0;
    if (r < mu) {
        const int f = find_key(pkeys, 0, pmu, k);
        if (f < pmu && pkeys[f] == k) g = pgam[f];
    } else if (r < mu + mw) {
        const int f = find_key(pkeys, pmu, pmu + pmw, k);
        if (f < pmu + pmw && pkeys[f] == k) g = pgam[f];
    } else if (springs_same && (long long)k < pms) {
        g = pgam[pmu + pmw + (int)k];
    }
    gin[r] = g;
}

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }

cudaError_t launch_count_walls(aLENS_ctx* ctx, int n)
{
    if (n <= 0 || ctx->wall_axis < 0) return cudaSuccess;
    k_count_walls<<<nblk(n, 256), 256, 0, ctx->stream>>>(n, (int)ctx->max_rods, ctx->wall_axis, ctx->wall_lo,
                                                         ctx->wall_hi, ctx->geo.half, ctx->p.diameter, ctx->p.delta_c,
                                                         ctx->xw, ctx->axis, ctx->cntQ, ctx->dcount);
    ++ctx->launches;
    return cudaGetLastError();
}

cudaError_t launch_emit_walls(aLENS_ctx* ctx, int n, int row0)
{
    if (n <= 0 || ctx->wall_axis < 0) return cudaSuccess;
    cudaError_t e = exclusive_scan(ctx, ctx->cntQ, ctx->curQ, n);
    if (e != cudaSuccess) return e;
    k_emit_walls<<<nblk(n, 256), 256, 0, ctx->stream>>>(n, (int)ctx->max_rods, row0, ctx->wall_axis, ctx->wall_lo,
                                                        ctx->wall_hi, ctx->geo.half, ctx->p.diameter, ctx->p.delta_c,
                                                        ctx->p.dt, ctx->xw, ctx->axis, ctx->unc, ctx->curQ, ctx->pairs,
                                                        ctx->phi, ctx->dgeom, ctx->q64, ctx->dcount);
    ++ctx->launches;
    return cudaGetLastError();
}

cudaError_t launch_brownian(aLENS_ctx* ctx, int n, const double* quat, double kT, unsigned long long seed,
                            unsigned long long step, const double* fext, double* out)
{
    if (n <= 0) return cudaSuccess;
    k_brownian<<<nblk(n, 128), 128, 0, ctx->stream>>>(n, ctx->mob, kT, ctx->p.dt, seed, step, quat, fext, out);
    ++ctx->launches;
    return cudaGetLastError();
}

cudaError_t launch_random_words(aLENS_ctx* ctx, int n, unsigned long long seed, unsigned long long step,
                                uint32_t* out)
{
    if (n <= 0) return cudaSuccess;
    k_random_words<<<nblk(n, 128), 128, 0, ctx->stream>>>(n, seed, step, out);
    ++ctx->launches;
    return cudaGetLastError();
}

cudaError_t launch_warm(aLENS_ctx* ctx, int m, int mu, int mw, double* gin)
{
    if (m <= 0) return cudaSuccess;
    k_row_keys<<<nblk(m, 256), 256, 0, ctx->stream>>>(m, mu, mw, ctx->pairs, ctx->row_keys);
    ++ctx->launches;
    const int same = ctx->prev_sp_version == ctx->sp_version;
    k_warm<<<nblk(m, 256), 256, 0, ctx->stream>>>(m, mu, mw, ctx->row_keys, ctx->prev_keys, ctx->prev_gam,
                                                  (int)ctx->prev_mu, (int)ctx->prev_mw, (int)ctx->prev_ms, same, gin);
    ++ctx->launches;
    return cudaGetLastError();
}

cudaError_t launch_keep_keys(aLENS_ctx* ctx, int m, int mu, int mw)
{
    // this step's row keys become the previous step's (its forces are written by the caller)
    if (m > 0) {
        k_row_keys<<<nblk(m, 256), 256, 0, ctx->stream>>>(m, mu, mw, ctx->pairs, ctx->prev_keys);
        ++ctx->launches;
    }
    ctx->prev_mu = mu;
    ctx->prev_mw = mw;
    ctx->prev_ms = m - mu - mw;
    ctx->prev_sp_version = ctx->sp_version;
    return cudaGetLastError();
}

}  // namespace alens
