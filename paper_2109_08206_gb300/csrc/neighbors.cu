// Neighbour search: pack rods, bin them into a Morton-ordered cell list,
// find every pair (and periodic image) with surface gap below delta_c.
//
// Appendix "Implementation": only close pairs whose minimal distance is
// below delta_c enter the constraint problem.  The paper uses a BVH; on one
// GPU a uniform cell grid with cell edge >= L + D + delta_c is enough, since
// two rods whose centres are farther apart than L + D + delta_c cannot have
// a surface gap below delta_c.
//
// Pipeline: k_pack (wrap centres, rod axis R(theta) e_z, cell key, M F_nc)
// -> counting sort by cell key -> k_search (one warp per rod, rods visited
// in cell order; lanes stride over the 27 neighbour cells; a float32 screen
// with a safety margin, then the float64 keep/drop decision; warp-aggregated
// appends into a per-rod list in shared memory, sorted there by (j, image))
// -> scan of per-rod counts -> k_emit (pairs in (i, j, image) order).
#include "internal.cuh"

namespace alens {

__global__ void k_pack(int n, int np, const double* __restrict__ x, const double* __restrict__ quat,
                       const double* __restrict__ fnc, Geo g, Mob mob, bool cells, double* __restrict__ xw,
                       double* __restrict__ axis, double* __restrict__ unc, float4* __restrict__ pos32,
                       float4* __restrict__ ax32, uint32_t* __restrict__ cellkey, int* __restrict__ cell_count,
                       int* __restrict__ flags)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = quat[4 * (size_t)i], a = quat[4 * (size_t)i + 1], b = quat[4 * (size_t)i + 2],
           c = quat[4 * (size_t)i + 3];
    double nq = s * s + a * a + b * b + c * c;
    bool bad = !(fabs(nq - 1.0) <= 2e-6);
    double p[3];
    quat_axis(s, a, b, c, p[0], p[1], p[2]);
    double w[3];
    int cc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double v = x[3 * (size_t)i + k];
        bad |= !isfinite(v);
        w[k] = wrap_coord(v, g.box[k]);
        int ck = (int)(w[k] / g.cs[k]);
        cc[k] = ck < 0 ? 0 : (ck >= g.nc[k] ? g.nc[k] - 1 : ck);
        xw[k * (size_t)np + i] = w[k];
        axis[k * (size_t)np + i] = p[k];
    }
    if (bad) {
        if (atomicCAS(&flags[F_ERR], 0, ALENS_ERR_INVALID) == 0) flags[F_ERR_ROD] = i;
    }
    pos32[i] = make_float4((float)w[0], (float)w[1], (float)w[2], 0.f);
    ax32[i] = make_float4((float)p[0], (float)p[1], (float)p[2], 0.f);
    if (cells) {
        uint32_t key = morton3(cc[0], cc[1], cc[2]);
        cellkey[i] = key;
        atomicAdd(&cell_count[key], 1);
    }
    if (unc) {
        // U_nc = M F_nc: M_t = p p^T / zeta_par + (I - p p^T) / zeta_perp, same for rotation
        double F[6];
        if (fnc) {
#pragma unroll
            for (int k = 0; k < 6; ++k) F[k] = fnc[6 * (size_t)i + k];
        } else {
#pragma unroll
            for (int k = 0; k < 6; ++k) F[k] = 0.0;
        }
        double pf = p[0] * F[0] + p[1] * F[1] + p[2] * F[2];
        double pt = p[0] * F[3] + p[1] * F[4] + p[2] * F[5];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            unc[k * (size_t)np + i] = F[k] * mob.inv_perp + p[k] * pf * (mob.inv_par - mob.inv_perp);
            unc[(3 + k) * (size_t)np + i] = F[3 + k] * mob.inv_rot + p[k] * pt * (mob.inv_spin - mob.inv_rot);
        }
    }
}

__global__ void k_cell_scatter(int n, const uint32_t* __restrict__ cellkey, const int* __restrict__ cell_start,
                               int* __restrict__ cell_cursor, const float4* __restrict__ pos32,
                               const float4* __restrict__ ax32, int* __restrict__ sorted_id,
                               float4* __restrict__ spos32, float4* __restrict__ sax32)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t key = cellkey[i];
    int pos = cell_start[key] + atomicAdd(&cell_cursor[key], 1);
    sorted_id[pos] = i;
    spos32[pos] = pos32[i];
    sax32[pos] = ax32[i];
}

// Order rods inside each cell by id, so that the cell-sorted layout (and the
// order in which the search meets candidates) does not depend on atomics.
__global__ void k_cell_order(int nkeys, const int* __restrict__ cell_start, int* __restrict__ sorted_id,
                             float4* __restrict__ spos32, float4* __restrict__ sax32)
{
    int key = blockIdx.x * blockDim.x + threadIdx.x;
    if (key >= nkeys) return;
    int b = cell_start[key], e = cell_start[key + 1];
    for (int u = b + 1; u < e; ++u) {
        int id = sorted_id[u];
        float4 ps = spos32[u], as = sax32[u];
        int v = u - 1;
        while (v >= b && sorted_id[v] > id) {
            sorted_id[v + 1] = sorted_id[v];
            spos32[v + 1] = spos32[v];
            sax32[v + 1] = sax32[v];
            --v;
        }
        sorted_id[v + 1] = id;
        spos32[v + 1] = ps;
        sax32[v + 1] = as;
    }
}

// Float32 lower-level screen of one candidate: returns false only when the
// pair is certainly farther than delta_c (with margin); near-parallel pairs
// always pass to the float64 decision.
__device__ __forceinline__ bool screen32(const float4& pi, const float4& ai, const float4& pj, const float4& aj,
                                         float sx, float sy, float sz, const Geo& g)
{
    float dx[3] = {pi.x - pj.x - sx, pi.y - pj.y - sy, pi.z - pj.z - sz};
    float r2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
    if (!(r2 < g.rcut_screen2)) return false;
    float p[3] = {ai.x, ai.y, ai.z}, q[3] = {aj.x, aj.y, aj.z};
    float b = p[0] * q[0] + p[1] * q[1] + p[2] * q[2];
    float det = 1.0f - b * b;
    if (det <= kParallelDet32) return true;   // near-parallel: decide in float64
    float s, t;
    float d = segment_closest<float>(dx, p, q, (float)g.half, kParallelDet32, s, t);
    return d - (float)g.diameter < g.gap_screen;
}

__device__ __forceinline__ bool decide64(int i, int j, int k0, int k1, int k2, int np, const double* __restrict__ xw,
                                         const double* __restrict__ axis, const Geo& g)
{
    double dx[3], p[3], q[3];
    int kk[3] = {k0, k1, k2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dx[k] = __dsub_rn(__dsub_rn(xw[k * (size_t)np + i], xw[k * (size_t)np + j]), __dmul_rn((double)kk[k], g.box[k]));
        p[k] = axis[k * (size_t)np + i];
        q[k] = axis[k * (size_t)np + j];
    }
    double s, t;
    double d = segment_closest<double>(dx, p, q, g.half, kParallelDet64, s, t);
    return d - g.diameter < g.delta_c;
}

__global__ void __launch_bounds__(kSearchWarps * 32)
k_search(int n, int np, Geo g, const int* __restrict__ sorted_id, const float4* __restrict__ spos32,
         const float4* __restrict__ sax32, const uint32_t* __restrict__ cellkey, const double* __restrict__ xw,
         const double* __restrict__ axis, const int* __restrict__ cell_start, int* __restrict__ rod_count,
         long long* __restrict__ rod_tmpstart, uint32_t* __restrict__ tmp_keys, long long cap,
         unsigned long long* __restrict__ counters, int* __restrict__ flags)
{
    __shared__ uint32_t list[kSearchWarps][kPairsPerRodCap];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = blockIdx.x * kSearchWarps + warp;
    if (k >= n) return;   // uniform per warp
    uint32_t* L = list[warp];
    const int i = sorted_id[k];
    const float4 pi = spos32[k], ai = sax32[k];
    int cc[3];
    {
        uint32_t key = cellkey[i];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            uint32_t v = 0;
            for (int bit = 0; bit < g.bits; ++bit) v |= ((key >> (3 * bit + a)) & 1u) << bit;
            cc[a] = (int)v;
        }
    }
    int cnt = 0;
    for (int o = 0; o < 27; ++o) {
        int d[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
        int c[3], sh[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            c[a] = cc[a] + d[a];
            sh[a] = 0;
            if (c[a] < 0) { c[a] += g.nc[a]; sh[a] = -1; }
            else if (c[a] >= g.nc[a]) { c[a] -= g.nc[a]; sh[a] = 1; }
        }
        const uint32_t code = (uint32_t)((sh[0] + 1) + 3 * (sh[1] + 1) + 9 * (sh[2] + 1));
        const uint32_t key = morton3(c[0], c[1], c[2]);
        const int beg = cell_start[key], end = cell_start[key + 1];
        const float sx = (float)sh[0] * g.boxf[0], sy = (float)sh[1] * g.boxf[1], sz = (float)sh[2] * g.boxf[2];
        for (int base = beg; base < end; base += 32) {
            int m = base + lane;
            bool keep = false;
            int j = 0;
            if (m < end) {
                j = sorted_id[m];
                if (j > i && screen32(pi, ai, spos32[m], sax32[m], sx, sy, sz, g))
                    keep = decide64(i, j, sh[0], sh[1], sh[2], np, xw, axis, g);
            }
            unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                int pos = cnt + __popc(bal & ((1u << lane) - 1u));
                if (pos < kPairsPerRodCap) L[pos] = ((uint32_t)j << 5) | code;
            }
            cnt += __popc(bal);
        }
    }
    __syncwarp();
    if (cnt > kPairsPerRodCap) {
        if (lane == 0 && atomicCAS(&flags[F_ERR], 0, ALENS_ERR_CAPACITY) == 0) flags[F_ERR_ROD] = i;
        cnt = kPairsPerRodCap;
    }
    // bitonic sort of L[0..cnt) padded to a power of two
    int P = 1;
    while (P < cnt) P <<= 1;
    for (int u = cnt + lane; u < P; u += 32) L[u] = 0xffffffffu;
    __syncwarp();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = lane; t < (P >> 1); t += 32) {
                int lo = 2 * t - (t & (stride - 1));
                int hi = lo + stride;
                bool up = (lo & size) == 0;
                uint32_t a = L[lo], b = L[hi];
                if ((a > b) == up) { L[lo] = b; L[hi] = a; }
            }
            __syncwarp();
        }
    }
    long long start = 0;
    if (lane == 0) {
        start = (long long)atomicAdd(&counters[C_PAIRS], (unsigned long long)cnt);
        rod_count[i] = cnt;
        rod_tmpstart[i] = start;
    }
    start = __shfl_sync(0xffffffffu, start, 0);
    for (int u = lane; u < cnt; u += 32)
        if (start + u < cap) tmp_keys[start + u] = L[u];
}

__global__ void k_emit(int n, const int* __restrict__ rod_count, const long long* __restrict__ rod_tmpstart,
                       const int* __restrict__ rowP, const uint32_t* __restrict__ tmp_keys, int32_t* __restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = rod_count[i];
    long long s = rod_tmpstart[i];
    long long o = rowP[i];
    for (int u = 0; u < c; ++u) {
        uint32_t key = tmp_keys[s + u];
        out[3 * (o + u) + 0] = i;
        out[3 * (o + u) + 1] = (int32_t)(key >> 5);
        out[3 * (o + u) + 2] = (int32_t)(key & 31u);
    }
}

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }

cudaError_t launch_pack(aLENS_ctx* ctx, int n, const double* x, const double* quat, const double* fnc, bool cells)
{
    if (n <= 0) return cudaSuccess;
    k_pack<<<nblk(n, 256), 256, 0, ctx->stream>>>(n, (int)ctx->max_rods, x, quat, fnc, ctx->geo, ctx->mob, cells,
                                                   ctx->xw, ctx->axis, ctx->unc, ctx->pos32, ctx->ax32,
                                                   ctx->cellkey, ctx->cell_count, ctx->dflags);
    ++ctx->launches;
    return cudaGetLastError();
}

cudaError_t launch_cell_sort(aLENS_ctx* ctx, int n)
{
    int nkeys = 1 << (3 * ctx->geo.bits);
    cudaError_t e = exclusive_scan(ctx, ctx->cell_count, ctx->cell_start, nkeys);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        k_cell_scatter<<<nblk(n, 256), 256, 0, ctx->stream>>>(n, ctx->cellkey, ctx->cell_start, ctx->cell_cursor,
                                                              ctx->pos32, ctx->ax32, ctx->sorted_id, ctx->spos32,
                                                              ctx->sax32);
        ++ctx->launches;
    }
    k_cell_order<<<nblk(nkeys, 256), 256, 0, ctx->stream>>>(nkeys, ctx->cell_start, ctx->sorted_id, ctx->spos32,
                                                            ctx->sax32);
    ++ctx->launches;
    return cudaGetLastError();
}

cudaError_t launch_search(aLENS_ctx* ctx, int n, long long cap)
{
    if (n <= 0) return cudaSuccess;
    k_search<<<nblk(n, kSearchWarps), kSearchWarps * 32, 0, ctx->stream>>>(
        n, (int)ctx->max_rods, ctx->geo, ctx->sorted_id, ctx->spos32, ctx->sax32, ctx->cellkey, ctx->xw, ctx->axis,
        ctx->cell_start, ctx->rod_count, ctx->rod_tmpstart, ctx->tmp_keys, cap, ctx->dcount, ctx->dflags);
    ++ctx->launches;
    return cudaGetLastError();
}

cudaError_t launch_emit_pairs(aLENS_ctx* ctx, int n, int32_t* pairs_out)
{
    cudaError_t e = exclusive_scan(ctx, ctx->rod_count, ctx->rowP, n);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        k_emit<<<nblk(n, 256), 256, 0, ctx->stream>>>(n, ctx->rod_count, ctx->rod_tmpstart, ctx->rowP,
                                                      ctx->tmp_keys, pairs_out);
        ++ctx->launches;
    }
    return cudaGetLastError();
}

}  // namespace alens
