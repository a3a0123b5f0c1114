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
// that drops or keeps a candidate when its float distance is clear of
// D + delta_c by proven margins and flags the rest; warp-aggregated appends
// into a per-rod list in shared memory, sorted there by (j, image)) ->
// k_decide (the float64 keep/drop decision of the flagged candidates) ->
// scan of per-rod counts -> k_emit (pairs in (i, j, image) order).
#include <climits>

#include "internal.cuh"

namespace alens {

__global__ void k_pack(int n, int np, const double* __restrict__ x, const double* __restrict__ quat,
                       const double* __restrict__ fnc, Geo g0, Mob mob0, const SysGeo* __restrict__ systab,
                       const int* __restrict__ sysid, bool cells, double* __restrict__ xw,
                       double* __restrict__ axis, double* __restrict__ unc, float4* __restrict__ pos32,
                       float4* __restrict__ ax32, uint32_t* __restrict__ cellkey, int* __restrict__ cell_count,
                       int* __restrict__ flags)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Geo& g = geo_of(g0, systab, sysid, i);
    const Mob& mob = systab ? systab[sysid[i]].mob : mob0;
    const uint32_t key_base = systab ? (uint32_t)systab[sysid[i]].key_base : 0u;
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
        int ck = cell_index(w[k], g.cs[k], g.inv_cs[k]);
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
        uint32_t key = key_base + morton3(cc[0], cc[1], cc[2]);
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
                               int* __restrict__ cell_cursor, int* __restrict__ sorted_id)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t key = cellkey[i];
    sorted_id[cell_start[key] + atomicAdd(&cell_cursor[key], 1)] = i;
}

// Rods of each cell in ascending id, so that the cell-sorted order (which the
// solver also uses to number rods) does not depend on the atomics above.
// One warp per cell: the cell's ids (distinct) are staged in shared memory;
// up to 32 go to their ranks (the count of smaller ids), longer cells (the
// dense nematic domains hold a few hundred) through a bitonic network,
// len log^2 len work instead of len^2.  A cell longer than kSortCap (none in
// the benchmark workloads) is sorted in place by lane 0.
constexpr int kSortCap = 1024;
constexpr int kSortWarps = 4;
__global__ void __launch_bounds__(kSortWarps * 32)
k_cell_sort_ids(int nkeys, const int* __restrict__ cell_start, int* __restrict__ sorted_id)
{
    __shared__ int buf[kSortWarps][kSortCap];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int key = blockIdx.x * kSortWarps + warp;
    if (key >= nkeys) return;   // uniform per warp
    const int b = cell_start[key], e = cell_start[key + 1], len = e - b;
    if (len <= 1) return;
    if (len > kSortCap) {
        if (lane == 0) {
            for (int u = b + 1; u < e; ++u) {
                int x = sorted_id[u], w = u - 1;
                while (w >= b && sorted_id[w] > x) { sorted_id[w + 1] = sorted_id[w]; --w; }
                sorted_id[w + 1] = x;
            }
        }
        return;
    }
    int* sv = buf[warp];
    for (int u = lane; u < len; u += 32) sv[u] = sorted_id[b + u];
    if (len > 32) {
        // bitonic network over the cell's ids padded to a power of two
        int P = 64;
        while (P < len) P <<= 1;
        for (int u = len + lane; u < P; u += 32) sv[u] = INT_MAX;
        __syncwarp();
        for (int size = 2; size <= P; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int t = lane; t < (P >> 1); t += 32) {
                    const int lo = 2 * t - (t & (stride - 1)), hi = lo + stride;
                    const bool up = (lo & size) == 0;
                    const int x = sv[lo], y = sv[hi];
                    if ((x > y) == up) { sv[lo] = y; sv[hi] = x; }
                }
                __syncwarp();
            }
        }
        for (int u = lane; u < len; u += 32) sorted_id[b + u] = sv[u];
        return;
    }
    __syncwarp();
    // up to 32 ids: each goes to its rank, the count of smaller ids
    const int x = lane < len ? sv[lane] : 0;
    int r = 0;
    for (int t = 0; t < len; ++t) r += sv[t] < x;
    if (lane < len) sorted_id[b + r] = x;
}

__global__ void k_cell_gather(int n, const int* __restrict__ sorted_id, const float4* __restrict__ pos32,
                              const float4* __restrict__ ax32, float4* __restrict__ spos32, float4* __restrict__ sax32)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int i = sorted_id[k];
    spos32[k] = pos32[i];
    sax32[k] = ax32[i];
}

// Float32 screen of one candidate: kScreenDrop when the pair is certainly
// farther apart than delta_c, kScreenKeep when it is certainly closer, and
// kScreenDecide for the float64 decision otherwise.  The clamped
// closest-point pair below is always a valid point pair of the two
// segments.  Drop: away from near-parallel axes it is the optimum up to
// rounding, so its squared distance exceeds (D + delta_c + margin)^2 only if
// the float64 gap exceeds delta_c.  Keep: its exact distance bounds the
// pair's minimum from above, and its float distance is within the keep
// margin of that exact distance (make_geo), so a float distance below
// D + delta_c - margin means a gap below delta_c.  Unit axes are taken as
// unit (a = c = 1); near-parallel pairs (1 - (p.q)^2 <= 1e-4) always go on
// to the float64 decision.
enum { kScreenDrop = 0, kScreenKeep = 1, kScreenDecide = 2 };

// Low word of a candidate key: j << 5 | image code (j < 2^26), with bit 31
// set while the float64 decision is pending; kDropped marks a candidate that
// decision dropped.
constexpr uint32_t kUndecided = 0x80000000u;
constexpr uint32_t kKeyMask = 0x7fffffffu;
constexpr uint32_t kDropped = 0xffffffffu;
constexpr int kCandPiece = 384;   // candidates a search warp lists in shared memory at a time (multiple of 32)

__device__ __forceinline__ int screen32(const float4& pi, const float4& ai, const float4& pj, const float4& aj,
                                        float sx, float sy, float sz, const Geo& g)
{
    float dx[3] = {pi.x - pj.x - sx, pi.y - pj.y - sy, pi.z - pj.z - sz};
    float r2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
    if (!(r2 < g.rcut_screen2)) return kScreenDrop;
    float b = ai.x * aj.x + ai.y * aj.y + ai.z * aj.z;
    float det = 1.0f - b * b;
    if (det <= kParallelDet32) return kScreenDecide;
    float d = ai.x * dx[0] + ai.y * dx[1] + ai.z * dx[2];
    float e = aj.x * dx[0] + aj.y * dx[1] + aj.z * dx[2];
    const float hl = g.half_f;
    float s = fminf(fmaxf(__fdividef(b * e - d, det), -hl), hl);
    float t = b * s + e;
    if (t < -hl || t > hl) {
        t = fminf(fmaxf(t, -hl), hl);
        s = fminf(fmaxf(b * t - d, -hl), hl);
    }
    float r0 = dx[0] + s * ai.x - t * aj.x;
    float r1 = dx[1] + s * ai.y - t * aj.y;
    float r2b = dx[2] + s * ai.z - t * aj.z;
    const float d2 = r0 * r0 + r1 * r1 + r2b * r2b;
    if (d2 < g.keep_d2) return kScreenKeep;
    return d2 < g.screen_d2 ? kScreenDecide : kScreenDrop;
}

// Float64 keep/drop decision of pair (i, j) at image shift k: surface gap
// |r| - D < delta_c at the closest points.
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

__device__ __forceinline__ void decode_cell(uint32_t key, int bits, int cc[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        uint32_t v = 0;
        for (int bit = 0; bit < bits; ++bit) v |= ((key >> (3 * bit + a)) & 1u) << bit;
        cc[a] = (int)v;
    }
}

// The candidate pairs (i, j > i) of the rod at cell-sorted position k, for
// one warp.  Lanes 0-26 fetch the rod ranges of the 27 neighbour cells at
// once (each cell with the periodic image shift that brings it next to i's
// cell), cut to the suffix of ids above i; the warp walks the concatenated
// candidates in two passes (below); the candidates j > i that the float32
// screen keeps or cannot settle go to L with a warp ballot and are sorted
// there by (j, image) with a bitonic network.  Returns their count and,
// unless COUNT_ONLY, leaves their keys (j << 5 | image, bit 31 while the
// float64 decision is pending) sorted in L; COUNT_ONLY takes that decision
// inline.  Q, E and T are the warp's ring [64], candidate list [kCandPiece]
// and image offsets [27] in shared memory.
template <bool COUNT_ONLY>
__device__ __forceinline__ int search_rod(int k, int i, int np, const Geo& g0, const SysGeo* __restrict__ systab,
                                          const int* __restrict__ sysid, const int* __restrict__ sorted_id,
                                          const float4* __restrict__ spos32, const float4* __restrict__ sax32,
                                          const uint32_t* __restrict__ cellkey, const double* __restrict__ xw,
                                          const double* __restrict__ axis, const int* __restrict__ cell_start,
                                          int* __restrict__ flags, uint32_t* L, uint32_t* Q, uint32_t* E, float4* T)
{
    const int lane = threadIdx.x & 31;
    const float4 pi = spos32[k], ai = sax32[k];
    const Geo& g = geo_of(g0, systab, sysid, i);
    const uint32_t key_base = systab ? (uint32_t)systab[sysid[i]].key_base : 0u;
    int cc[3];
    decode_cell(cellkey[i] - key_base, g.bits, cc);
    // the 27 neighbour cells, one per lane: each with the periodic image
    // shift that brings it next to i's cell (as a code and as a float
    // offset), its rod range and its image code
    int cbeg = 0, ccnt = 0;
    uint32_t ccode = 0;
    float csx = 0.0f, csy = 0.0f, csz = 0.0f;
    if (lane < 27) {
        const int d[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
        int c[3], sh[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            c[a] = cc[a] + d[a];
            sh[a] = 0;
            if (c[a] < 0) { c[a] += g.nc[a]; sh[a] = -1; }
            else if (c[a] >= g.nc[a]) { c[a] -= g.nc[a]; sh[a] = 1; }
        }
        ccode = (uint32_t)((sh[0] + 1) + 3 * (sh[1] + 1) + 9 * (sh[2] + 1));
        csx = (float)sh[0] * g.boxf[0];
        csy = (float)sh[1] * g.boxf[1];
        csz = (float)sh[2] * g.boxf[2];
        const uint32_t key = key_base + morton3(c[0], c[1], c[2]);
        int b = cell_start[key], e = cell_start[key + 1];
        // a cell's ids ascend (k_cell_sort_ids): the candidates j > i are a
        // suffix of its range, found by a binary search
        while (b < e) {
            const int mid = (b + e) >> 1;
            if (sorted_id[mid] > i) e = mid;
            else b = mid + 1;
        }
        cbeg = b;
        ccnt = cell_start[key + 1] - b;
    }
    // inclusive prefix of the cells' counts: candidate t lies in the cell o
    // with incl[o - 1] <= t < incl[o]
    int incl = ccnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int excl = incl - ccnt;   // this lane's cell: candidates [excl, incl)
    if (lane < 27) T[ccode] = make_float4(csx, csy, csz, 0.0f);   // equal codes, equal offsets
    int cnt = 0;
    // Two passes over the candidates of all 27 cells.  A: the candidates,
    // listed in shared memory kCandPiece at a time as m | code << 26 (each
    // cell's lane writes its part of the piece), are tested in chunks of 32
    // lanes for the centre distance alone (the screen's first test, about
    // one candidate in seven passes) and the passes are queued in a per-warp
    // ring.  B: every 32 queued candidates (and the rest at the end) take the
    // whole float32 screen with all lanes busy.
    int qh = 0, qn = 0;   // warp-uniform ring head and length (qn < 32 before each chunk)
    for (int pb = 0, base = 0; base < total || qn > 0;) {
        if (base < total) {
            if (base == pb) {   // list the next piece [pb, pb + kCandPiece)
                __syncwarp();   // the last piece's entries are read
                const int u0 = max(pb - excl, 0), u1 = min(incl, pb + kCandPiece) - excl;
                for (int u = u0; u < u1; ++u) E[excl + u - pb] = (uint32_t)(cbeg + u) | (ccode << 26);
                __syncwarp();
            }
            const int t = base + lane;
            bool near = false;
            uint32_t e = 0u;
            if (t < total) {
                e = E[t - pb];
                const float4 sft = T[e >> 26];
                const float4 pj = spos32[e & 0x3ffffffu];
                const float dx = pi.x - pj.x - sft.x, dy = pi.y - pj.y - sft.y, dz = pi.z - pj.z - sft.z;
                near = dx * dx + dy * dy + dz * dz < g.rcut_screen2;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, near);
            if (near) Q[(qh + qn + __popc(bal & ((1u << lane) - 1u))) & 63] = e;
            qn += __popc(bal);
            base += 32;
            if (base >= pb + kCandPiece) pb += kCandPiece;
            __syncwarp();
        }
        if (qn >= 32 || (base >= total && qn > 0)) {
            const int take = qn < 32 ? qn : 32;
            const uint32_t e = lane < take ? Q[(qh + lane) & 63] : 0u;
            qh = (qh + take) & 63;
            qn -= take;
            __syncwarp();   // read before the next chunk reuses the slots
            bool keep = false;
            int j = 0, sc = kScreenDrop;
            const uint32_t code = e >> 26;
            if (lane < take) {
                const int m = (int)(e & 0x3ffffffu);
                const int s0 = (int)(code % 3u) - 1, s1 = (int)((code / 3u) % 3u) - 1, s2 = (int)(code / 9u) - 1;
                sc = screen32(pi, ai, spos32[m], sax32[m], (float)s0 * g.boxf[0], (float)s1 * g.boxf[1],
                              (float)s2 * g.boxf[2], g);
                keep = sc != kScreenDrop;
                if (keep) j = sorted_id[m];
                // counting decides in float64 here; the listing pass leaves it to k_decide
                if (COUNT_ONLY && sc == kScreenDecide) keep = decide64(i, j, s0, s1, s2, np, xw, axis, g);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (!COUNT_ONLY && keep) {
                const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
                if (pos < kPairsPerRodCap)
                    L[pos] = ((uint32_t)j << 5) | code | (sc == kScreenDecide ? kUndecided : 0u);
            }
            cnt += __popc(bal);
        }
    }
    if (COUNT_ONLY) return cnt;
    __syncwarp();
    if (cnt > kPairsPerRodCap) {
        if (lane == 0 && atomicCAS(&flags[F_ERR], 0, ALENS_ERR_CAPACITY) == 0) flags[F_ERR_ROD] = i;
        cnt = kPairsPerRodCap;
    }
    // bitonic sort of L[0..cnt) padded to a power of two
    int P = 1;
    while (P < cnt) P <<= 1;
    for (int u = cnt + lane; u < P; u += 32) L[u] = kKeyMask;
    __syncwarp();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = lane; t < (P >> 1); t += 32) {
                int lo = 2 * t - (t & (stride - 1));
                int hi = lo + stride;
                bool up = (lo & size) == 0;
                uint32_t a = L[lo], b = L[hi];
                if (((a & kKeyMask) > (b & kKeyMask)) == up) { L[lo] = b; L[hi] = a; }
            }
            __syncwarp();
        }
    }
    return cnt;
}

// One warp per rod i (rods taken in cell order for locality of the candidate
// loads), search_rod finding its pairs; they are written to the candidate
// buffer as 64-bit keys (i << 32 | kUndecided? | j << 5 | image), their
// count to rod_count and the total, and k_decide takes the float64 decision
// of the flagged few.  The candidate buffer and the pair total take one
// atomic per block (per rod they would queue on one L2 address): thread 0
// reserves the block's candidates and hands each warp its start; the
// block's warps past n only join that count.  COUNT_ONLY: only the total
// (used when the candidate buffer overflows).
template <bool COUNT_ONLY>
__global__ void __launch_bounds__(kSearchWarps * 32)
k_search(int n, int np, Geo g0, const SysGeo* __restrict__ systab, const int* __restrict__ sysid,
         const int* __restrict__ sorted_id, const float4* __restrict__ spos32,
         const float4* __restrict__ sax32, const uint32_t* __restrict__ cellkey, const double* __restrict__ xw,
         const double* __restrict__ axis, const int* __restrict__ cell_start, int* __restrict__ rod_ncand,
         int* __restrict__ rod_count, long long* __restrict__ rod_tmpstart, unsigned long long* __restrict__ cand,
         long long cand_cap, unsigned long long* __restrict__ counters, int* __restrict__ flags)
{
    __shared__ uint32_t list[COUNT_ONLY ? 1 : kSearchWarps][COUNT_ONLY ? 1 : kPairsPerRodCap];
    __shared__ uint32_t ring[kSearchWarps][64];
    __shared__ uint32_t elist[kSearchWarps][kCandPiece];
    __shared__ float4 Tsh[kSearchWarps][27];
    __shared__ int wcnt[kSearchWarps];
    __shared__ long long wstart[kSearchWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = blockIdx.x * kSearchWarps + warp;
    uint32_t* L = list[COUNT_ONLY ? 0 : warp];
    int i = 0, cnt = 0;
    if (k < n) {   // uniform per warp
        i = sorted_id[k];
        cnt = search_rod<COUNT_ONLY>(k, i, np, g0, systab, sysid, sorted_id, spos32, sax32, cellkey, xw, axis,
                                     cell_start, flags, L, ring[warp], elist[warp], Tsh[warp]);
    }
    if (lane == 0) wcnt[warp] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < kSearchWarps; ++w) tot += wcnt[w];
        long long st = COUNT_ONLY || tot == 0 ? 0 : (long long)atomicAdd(&counters[C_CAND], (unsigned long long)tot);
        if (tot) atomicAdd(&counters[C_PAIRS], (unsigned long long)tot);
        for (int w = 0; w < kSearchWarps; ++w) {
            wstart[w] = st;
            st += wcnt[w];
        }
    }
    __syncthreads();
    if (COUNT_ONLY || k >= n) return;
    const long long start = wstart[warp];
    if (lane == 0) {
        rod_ncand[i] = cnt;
        rod_count[i] = cnt;
        rod_tmpstart[i] = start;
    }
    const unsigned long long hi = (unsigned long long)(unsigned)i << 32;
    for (int u = lane; u < cnt; u += 32)
        if (start + u < cand_cap) cand[start + u] = hi | L[u];
}

// Float64 decision of the candidates the float32 screen left undecided.  A
// few per cent of the candidates carry the flag and the FP64 pipe executes a
// warp instruction at full cost however few lanes are active, so each block
// first gathers the flagged candidates of a chunk of kDecideChunk keys into
// a list in shared memory (warp ballots) and then decides that list with
// full warps: a kept candidate loses its flag, a dropped one becomes
// kDropped and leaves its rod's count and the total.  Chunks go to blocks
// round robin; the list holds a whole chunk, so any flagged fraction fits.
constexpr int kDecideThreads = 256;
constexpr int kDecideChunk = 4 * kDecideThreads;
constexpr int kDecideBlocksPerSM = 4;   // about 6e5 candidates decided in one round of chunks

__global__ void __launch_bounds__(kDecideThreads)
k_decide(int np, Geo g0, const SysGeo* __restrict__ systab, const int* __restrict__ sysid,
         const unsigned long long* counters_ro, unsigned long long* __restrict__ cand, long long cand_cap,
         const double* __restrict__ xw, const double* __restrict__ axis, int* __restrict__ rod_count,
         unsigned long long* counters)
{
    __shared__ int list[kDecideChunk];
    __shared__ int nlist;
    long long total = (long long)counters_ro[C_CAND];
    if (total > cand_cap) total = cand_cap;
    const int lane = threadIdx.x & 31;
    for (long long base = (long long)blockIdx.x * kDecideChunk; base < total;
         base += (long long)gridDim.x * kDecideChunk) {
        if (threadIdx.x == 0) nlist = 0;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kDecideChunk / kDecideThreads; ++r) {
            const int off = r * kDecideThreads + threadIdx.x;
            const bool f = base + off < total && ((uint32_t)cand[base + off] & kUndecided);
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            int at = 0;
            if (lane == 0 && bal) at = atomicAdd(&nlist, __popc(bal));
            at = __shfl_sync(0xffffffffu, at, 0);
            if (f) list[at + __popc(bal & ((1u << lane) - 1u))] = off;
        }
        __syncthreads();
        const int nl = nlist;
        for (int u0 = threadIdx.x - lane; u0 < nl; u0 += kDecideThreads) {   // whole warps
            const int u = u0 + lane;
            bool drop = false;
            if (u < nl) {
                const long long k = base + list[u];
                const unsigned long long key = cand[k];
                const uint32_t lo = (uint32_t)key;
                const int i = (int)(key >> 32);
                const int j = (int)((lo & kKeyMask) >> 5);
                const int code = (int)(lo & 31u);
                const bool kp = decide64(i, j, code % 3 - 1, (code / 3) % 3 - 1, code / 9 - 1, np, xw, axis,
                                         geo_of(g0, systab, sysid, i));
                cand[k] = (key & 0xffffffff00000000ull) | (kp ? (lo & kKeyMask) : kDropped);
                if (!kp) {
                    atomicSub(&rod_count[i], 1);
                    drop = true;
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, drop);
            if (lane == 0 && bal) atomicAdd(&counters[C_PAIRS], 0ull - (unsigned long long)__popc(bal));
        }
        __syncthreads();   // the list is rebuilt for the next chunk
    }
}

// Pairs of rod i in (j, image) order: its segment of the candidate buffer
// less the candidates k_decide dropped.
__global__ void k_emit(int n, const int* __restrict__ rod_ncand, const long long* __restrict__ rod_tmpstart,
                       const int* __restrict__ rowP, const unsigned long long* __restrict__ cand,
                       int32_t* __restrict__ out, long long cap)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = rod_ncand[i];
    long long s = rod_tmpstart[i];
    long long o = rowP[i];
    for (int u = 0; u < c; ++u) {
        if (o >= cap) break;   // more pairs than the output holds (a step without readbacks reports CAPACITY)
        const uint32_t key = (uint32_t)cand[s + u];
        if (key == kDropped) continue;
        out[3 * o + 0] = i;
        out[3 * o + 1] = (int32_t)(key >> 5);
        out[3 * o + 2] = (int32_t)(key & 31u);
        ++o;
    }
}

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }

cudaError_t launch_pack(aLENS_ctx* ctx, int n, const double* x, const double* quat, const double* fnc, bool cells)
{
    if (n <= 0) return cudaSuccess;
    k_pack<<<nblk(n, 256), 256, 0, ctx->stream>>>(n, (int)ctx->max_rods, x, quat, fnc, ctx->geo, ctx->mob,
                                                   ctx->cur_systab, ctx->cur_sysid, cells,
                                                   ctx->xw, ctx->axis, ctx->unc, ctx->pos32, ctx->ax32,
                                                   ctx->cellkey, ctx->cell_count, ctx->dflags);
    ++ctx->launches;
    return cudaGetLastError();
}

cudaError_t launch_cell_sort(aLENS_ctx* ctx, int n)
{
    int nkeys = ctx->cur_nkeys;
    cudaError_t e = exclusive_scan(ctx, ctx->cell_count, ctx->cell_start, nkeys);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        k_cell_scatter<<<nblk(n, 256), 256, 0, ctx->stream>>>(n, ctx->cellkey, ctx->cell_start, ctx->cell_cursor,
                                                              ctx->sorted_id);
        ++ctx->launches;
        k_cell_sort_ids<<<nblk(nkeys, kSortWarps), kSortWarps * 32, 0, ctx->stream>>>(nkeys, ctx->cell_start,
                                                                                       ctx->sorted_id);
        ++ctx->launches;
        k_cell_gather<<<nblk(n, 256), 256, 0, ctx->stream>>>(n, ctx->sorted_id, ctx->pos32, ctx->ax32, ctx->spos32,
                                                             ctx->sax32);
        ++ctx->launches;
    }
    return cudaGetLastError();
}

cudaError_t launch_search(aLENS_ctx* ctx, int n)
{
    if (n <= 0) return cudaSuccess;
    k_search<false><<<nblk(n, kSearchWarps), kSearchWarps * 32, 0, ctx->stream>>>(
        n, (int)ctx->max_rods, ctx->geo, ctx->cur_systab, ctx->cur_sysid, ctx->sorted_id, ctx->spos32, ctx->sax32,
        ctx->cellkey, ctx->xw, ctx->axis, ctx->cell_start, ctx->rod_ncand, ctx->rod_count, ctx->rod_tmpstart, ctx->cand,
        ctx->cand_cap, ctx->dcount, ctx->dflags);
    ++ctx->launches;
    k_decide<<<ctx->num_sms * kDecideBlocksPerSM, kDecideThreads, 0, ctx->stream>>>((int)ctx->max_rods, ctx->geo, ctx->cur_systab,
                                                        ctx->cur_sysid, ctx->dcount, ctx->cand, ctx->cand_cap,
                                                        ctx->xw, ctx->axis, ctx->rod_count, ctx->dcount);
    ++ctx->launches;
    return cudaGetLastError();
}

cudaError_t launch_search_count(aLENS_ctx* ctx, int n)
{
    if (n <= 0) return cudaSuccess;
    k_search<true><<<nblk(n, kSearchWarps), kSearchWarps * 32, 0, ctx->stream>>>(
        n, (int)ctx->max_rods, ctx->geo, ctx->cur_systab, ctx->cur_sysid, ctx->sorted_id, ctx->spos32, ctx->sax32,
        ctx->cellkey, ctx->xw, ctx->axis, ctx->cell_start, ctx->rod_ncand, ctx->rod_count, ctx->rod_tmpstart, ctx->cand,
        ctx->cand_cap, ctx->dcount, ctx->dflags);
    ++ctx->launches;
    return cudaGetLastError();
}

cudaError_t launch_emit_pairs(aLENS_ctx* ctx, int n, int32_t* pairs_out)
{
    cudaError_t e = exclusive_scan(ctx, ctx->rod_count, ctx->rowP, n);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        k_emit<<<nblk(n, 256), 256, 0, ctx->stream>>>(n, ctx->rod_ncand, ctx->rod_tmpstart, ctx->rowP, ctx->cand,
                                                      pairs_out, ctx->max_pairs);
        ++ctx->launches;
    }
    return cudaGetLastError();
}

// The step's capacity test on the device: the kept pairs fit the constraint
// arrays and every candidate fit its buffer, else ALENS_ERR_CAPACITY.
// C_MEFF is the constraint count the later kernels of the step take (0
// after a failure, so that they do nothing).
__global__ void k_check_capacity(long long max_pairs, long long cand_cap, unsigned long long* counters, int* flags)
{
    if (threadIdx.x != 0) return;
    const unsigned long long mu = counters[C_PAIRS];
    const bool over = mu > (unsigned long long)max_pairs || counters[C_CAND] > (unsigned long long)cand_cap;
    if (over) atomicCAS(&flags[F_ERR], 0, ALENS_ERR_CAPACITY);
    counters[C_MEFF] = (over || flags[F_ERR] != 0) ? 0ull : mu;
}

cudaError_t launch_check_capacity(aLENS_ctx* ctx)
{
    k_check_capacity<<<1, 32, 0, ctx->stream>>>(ctx->max_pairs, ctx->cand_cap, ctx->dcount, ctx->dflags);
    ++ctx->launches;
    return cudaGetLastError();
}

// The step's pair list to the caller: *mdev triples (i, j, image).
__global__ void k_copy_pairs(long long cap, const unsigned long long* __restrict__ mdev, const int32_t* __restrict__ src,
                             int32_t* __restrict__ dst)
{
    const long long m = (long long)count_of((int)cap, mdev);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < 3 * m; k += (long long)gridDim.x * blockDim.x)
        dst[k] = src[k];
}

cudaError_t launch_copy_pairs(aLENS_ctx* ctx, int32_t* pairs_out)
{
    k_copy_pairs<<<ctx->num_sms * 4, 256, 0, ctx->stream>>>(ctx->max_pairs, ctx->mdev, ctx->pairs, pairs_out);
    ++ctx->launches;
    return cudaGetLastError();
}

}  // namespace alens
