// Exclusive prefix sum of int32 counts (CSR row pointers, cell starts).
// Two launches: per-tile totals, then per-tile scans, each block adding the
// totals of the tiles before it (a few thousand at most) for its offset.
// Integer sums: exact and deterministic.
#include "internal.cuh"

namespace alens {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;                       // per thread
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int block_exclusive_scan(int v, int* smem, int& total)
{
    // warp inclusive scan
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        int w = lane < nw ? smem[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        smem[32 + lane] = w;   // inclusive warp totals
    }
    __syncthreads();
    total = smem[32 + ((blockDim.x >> 5) - 1)];
    int before = warp > 0 ? smem[32 + warp - 1] : 0;
    int r = before + x - v;
    __syncthreads();
    return r;
}

__global__ void k_tile_sums(const int* __restrict__ in, int n, int* __restrict__ sums)
{
    __shared__ int smem[64];
    long long base = (long long)blockIdx.x * kScanTile;
    int acc = 0;
    for (int k = 0; k < kScanItems; ++k) {
        long long idx = base + (long long)k * kScanThreads + threadIdx.x;
        if (idx < n) acc += in[idx];
    }
    int total;
    block_exclusive_scan(acc, smem, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_tile_scan(const int* __restrict__ in, int n, const int* __restrict__ sums, int* __restrict__ out)
{
    __shared__ int smem[64];
    __shared__ int pre;
    if (threadIdx.x < 32) {   // this tile's offset: the totals of the tiles before it
        int a = 0;
        for (int t = threadIdx.x; t < (int)blockIdx.x; t += 32) a += sums[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (threadIdx.x == 0) pre = a;
    }
    __syncthreads();
    long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    int v[kScanItems];
    int acc = 0;
    for (int k = 0; k < kScanItems; ++k) {
        long long idx = base + k;
        v[k] = idx < n ? in[idx] : 0;
        acc += v[k];
    }
    int total;
    int ex = block_exclusive_scan(acc, smem, total) + pre;
    for (int k = 0; k < kScanItems; ++k) {
        long long idx = base + k;
        if (idx < n) out[idx] = ex;
        ex += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = pre + total;
}

// k_tile_sums sums a tile in strided order and k_tile_scan scans it in
// blocked order; both cover the same kScanTile elements, so the tile totals agree.
cudaError_t exclusive_scan(aLENS_ctx* ctx, const int* counts, int* out, int n)
{
    int ntiles = n > 0 ? (n + kScanTile - 1) / kScanTile : 1;
    if (ntiles + 1 > ctx->scan_tmp_len) return cudaErrorInvalidValue;
    k_tile_sums<<<ntiles, kScanThreads, 0, ctx->stream>>>(counts, n, ctx->scan_tmp);
    ++ctx->launches;
    k_tile_scan<<<ntiles, kScanThreads, 0, ctx->stream>>>(counts, n, ctx->scan_tmp, out);
    ++ctx->launches;
    return cudaGetLastError();
}

}  // namespace alens
