// aLENS_solve_lcp_noalloc: the BBPGD solve of aLENS_solve_lcp for callers
// that must not allocate device memory.
//
// Who needs it: a host application or plugin that runs inside a memory
// manager owning the whole device-memory budget (no cudaMalloc outside its
// pool), and latency-critical loops where cudaMalloc / cudaFree would take
// the allocator lock or synchronise the device at the wrong moment.  Such a
// caller cannot create an aLENS_ctx (aLENS_create allocates its workspaces),
// so this entry point takes its workspace from one statically sized device
// array instead.
//
// The workspace is the file-scope array g_noalloc_scratch below: every GPU
// that loads this library holds it (kNoallocScratchBytes) until the process
// exits.  Host code may not use the array's name as a device address, so
// the first call on each device (with that device current) looks the
// address up with cudaGetSymbolAddress and keeps it; make that first call
// before any stream capture.  A cudaDeviceReset unloads the module and
// leaves the kept address stale, so the entry point is not for use on a
// device after a reset.  All calls share the array and it keeps the
// last call's contents: the counters the solver needs at zero are cleared on
// every call, and two calls whose work overlaps on the GPU (on different
// streams, or from different host threads) race on it.
#include <math.h>
#include <mutex>
#include <string.h>

#include "internal.cuh"

using namespace alens;

namespace {

constexpr int kNoallocMaxRods = ALENS_NOALLOC_MAX_RODS;
constexpr int kNoallocMaxPairs = ALENS_NOALLOC_MAX_PAIRS;
constexpr int kNoallocMaxBlocks = 1024;
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

constexpr size_t kRodInts = align256(sizeof(int) * (kNoallocMaxRods + 1));
constexpr size_t kPairInts = align256(sizeof(int) * kNoallocMaxPairs);
constexpr size_t kSolveWs =
    align256(sizeof(double) * (29 * (size_t)kNoallocMaxPairs + 25 * (size_t)kNoallocMaxRods + 112));
constexpr size_t kPairDoubles = align256(sizeof(double) * kNoallocMaxPairs);
constexpr size_t kPartials = align256(sizeof(double) * 8 * (kNoallocMaxBlocks + 4));
constexpr size_t kBstart = align256(sizeof(int) * (kNoallocMaxBlocks + 1));
constexpr int kScanTmpLen = (kNoallocMaxRods + 4095) / 4096 + 2;
constexpr size_t kSmall = align256(16 * sizeof(unsigned)) + align256(F_NFLAGS * sizeof(int)) +
                          align256(C_NCOUNT * sizeof(unsigned long long)) + align256(kScanTmpLen * sizeof(int));
constexpr size_t kNoallocScratchBytes =
    6 * kRodInts + 4 * kPairInts + kPairDoubles + kSolveWs + kPartials + kBstart + kSmall;

// the header states the size as 5.19 MB
static_assert(kNoallocScratchBytes > 5180000 && kNoallocScratchBytes < 5195000, "noalloc scratch size changed");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_lock;
unsigned char* g_base[kMaxDevices];

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_base(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_lock);
    if (!g_base[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_base[dev] = (unsigned char*)p;
    }
    *out = g_base[dev];
    return cudaSuccess;
}

bool params_valid(const aLENS_params* p)
{
    return p && p->diameter > 0 && p->length > 0 && p->viscosity > 0 && p->dt > 0 && p->tol >= 0 &&
           p->max_iter >= 0 && p->max_iter <= 10000000 && 2.0 * p->length / p->diameter > 1.0 &&
           (p->precision == ALENS_FP64 || p->precision == ALENS_MIXED);
}

}  // namespace

extern "C" aLENS_status aLENS_solve_lcp_noalloc(const aLENS_params* params, int64_t n, const double* quat,
                                                int64_t n_pairs, const int32_t* pairs, const double* dgeom,
                                                const double* q, double* gamma, void* cuda_stream, aLENS_info* info)
{
    if (!params_valid(params) || n < 0 || n_pairs < 0) return ALENS_ERR_INVALID;
    if (n > kNoallocMaxRods || n_pairs > kNoallocMaxPairs) return ALENS_ERR_CAPACITY;
    if (n > 0 && !quat) return ALENS_ERR_INVALID;
    if (n_pairs > 0 && (!pairs || !dgeom || !q || !gamma)) return ALENS_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ALENS_ERR_CUDA;
    unsigned char* base = nullptr;
    if (scratch_base(dev, &base) != cudaSuccess) return ALENS_ERR_CUDA;

    // a context on the host stack whose workspaces are slices of the array
    aLENS_ctx c;
    memset(&c, 0, sizeof(c));
    c.p = *params;
    c.max_rods = kNoallocMaxRods;
    c.max_pairs = kNoallocMaxPairs;
    c.stream = (cudaStream_t)cuda_stream;
    c.device = dev;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return ALENS_ERR_CUDA;
    if (!prop.cooperativeLaunch) return ALENS_ERR_CUDA;
    c.num_sms = prop.multiProcessorCount;
    c.smem_optin = (int)prop.sharedMemPerBlockOptin;
    int clk = 0;
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
    c.clock_khz = clk > 0 ? clk : 2.1e6;
    c.max_blocks = c.num_sms * 8 < kNoallocMaxBlocks ? c.num_sms * 8 : kNoallocMaxBlocks;
    c.wait_s = 5.0;
    c.scale_beta = kDefaultScaleBeta;
    c.solve_threads = 1024;
    c.solve_barriers = 1;
    c.wall_axis = -1;
    double zperp = 4.0 * M_PI * params->viscosity * params->length / log(2.0 * params->length / params->diameter);
    c.mob.inv_perp = 1.0 / zperp;
    c.mob.inv_par = 2.0 / zperp;
    c.mob.inv_rot = 12.0 / (zperp * params->length * params->length);
    c.mob.inv_spin = 1.0 / (M_PI * params->viscosity * params->diameter * params->diameter * params->length);

    size_t o = 0;
    auto take = [&](size_t bytes) { unsigned char* r = base + o; o += align256(bytes); return r; };
    c.rod_count = (int*)take(kRodInts);
    c.cntQ = (int*)take(kRodInts);
    c.curQ = (int*)take(kRodInts);
    c.curP = (int*)take(kRodInts);
    c.rowP = (int*)take(kRodInts);
    c.rowQ = (int*)take(kRodInts);
    c.perm = (int*)take(kPairInts);
    c.qlist = (int*)take(kPairInts);
    c.ci = (int*)take(kPairInts);
    c.cj = (int*)take(kPairInts);
    c.scale64 = (double*)take(kPairDoubles);
    c.solve_ws = take(kSolveWs);
    c.partials = (double*)take(kPartials);
    c.bstart = (int*)take(kBstart);
    c.bar = (unsigned*)take(16 * sizeof(unsigned));
    c.dflags = (int*)take(F_NFLAGS * sizeof(int));
    c.dcount = (unsigned long long*)take(C_NCOUNT * sizeof(unsigned long long));
    c.scan_tmp = (int*)take(kScanTmpLen * sizeof(int));
    c.scan_tmp_len = kScanTmpLen;
    {
        const size_t mp = kNoallocMaxPairs, np = kNoallocMaxRods;
        double* b64 = (double*)c.solve_ws;
        size_t u = 0;
        auto c64 = [&](size_t cnt) { double* r = b64 + u; u = (u + cnt + 7) & ~(size_t)7; return r; };
        c.sb64.gg[0] = c64(4 * mp); c.sb64.gg[1] = c64(4 * mp); c.sb64.U = c64(6 * np); c.sb64.U2 = c64(6 * np);
        c.sb64.Uref = c64(6 * np);
        c.sb64.gref = c64(mp);
        c.sb64.rec = c64(9 * mp); c.sb64.qe = c64(8 * mp); c.sb64.q = c64(mp); c.sb64.ax = c64(3 * np);
        c.sb64.mobr = c64(4 * np);
        c.sb64.comp = c64(mp);
        c.sb64.isc = c64(mp);
        float* b32 = (float*)c.solve_ws;
        size_t v = 0;
        auto c32 = [&](size_t cnt) { float* r = b32 + v; v = (v + cnt + 7) & ~(size_t)7; return r; };
        c.sb32.gg[0] = c32(4 * mp); c.sb32.gg[1] = c32(4 * mp); c.sb32.U = c32(6 * np); c.sb32.U2 = c32(6 * np);
        c.sb32.Uref = c32(6 * np);
        c.sb32.gref = c32(mp);
        c.sb32.rec = c32(9 * mp); c.sb32.qe = c32(8 * mp); c.sb32.q = c32(mp); c.sb32.ax = c32(3 * np);
        c.sb32.mobr = c32(4 * np);
        c.sb32.comp = c32(mp);
        c.sb32.isc = c32(mp);
        // the float32 views use at most half of the workspace: room for the low parts
        c.sb32.rec_lo = c32(9 * mp); c.sb32.qe_lo = c32(8 * mp); c.sb32.q_lo = c32(mp);
    }

    int hflags[F_NFLAGS];
    unsigned long long hcount[C_NCOUNT];
    auto read = [&]() -> bool {
        return cudaMemcpyAsync(hflags, c.dflags, sizeof(hflags), cudaMemcpyDeviceToHost, c.stream) == cudaSuccess &&
               cudaMemcpyAsync(hcount, c.dcount, sizeof(hcount), cudaMemcpyDeviceToHost, c.stream) == cudaSuccess &&
               cudaStreamSynchronize(c.stream) == cudaSuccess;
    };
    // everything that must start at zero on every call
    if (cudaMemsetAsync(c.dflags, 0, F_NFLAGS * sizeof(int), c.stream) != cudaSuccess ||
        cudaMemsetAsync(c.dcount, 0, C_NCOUNT * sizeof(unsigned long long), c.stream) != cudaSuccess)
        return ALENS_ERR_CUDA;
    if (launch_solve_setup_check(&c, (int)n, (int)n_pairs, pairs) != cudaSuccess || !read()) return ALENS_ERR_CUDA;
    if (hflags[F_ERR] != 0) return (aLENS_status)hflags[F_ERR];
    if (launch_solve_setup(&c, (int)n, (int)n_pairs, pairs, dgeom, q, gamma, quat, params->precision, nullptr) !=
        cudaSuccess)
        return ALENS_ERR_CUDA;
    if (n_pairs > 0 && launch_solve(&c, (int)n, (int)n_pairs, params->precision) != cudaSuccess) return ALENS_ERR_CUDA;
    if (!read()) return ALENS_ERR_CUDA;
    double res = 0.0;
    memcpy(&res, &hcount[C_RESID], sizeof(res));
    aLENS_status st = ALENS_OK;
    if (hflags[F_SOLVE_ERR] != 0) st = (aLENS_status)hflags[F_SOLVE_ERR];
    else if (hflags[F_ERR] != 0) st = (aLENS_status)hflags[F_ERR];
    else if (n_pairs > 0 && !(res <= params->tol)) st = ALENS_ERR_NOT_CONVERGED;
    if (st == ALENS_OK || st == ALENS_ERR_NOT_CONVERGED) {
        if (launch_gamma_out(&c, (int)n_pairs, params->precision, gamma) != cudaSuccess ||
            cudaStreamSynchronize(c.stream) != cudaSuccess)
            return ALENS_ERR_CUDA;
    }
    if (info) {
        memset(info, 0, sizeof(*info));
        info->n_pairs = n_pairs;
        info->iters = n_pairs > 0 ? hflags[F_ITERS] : 0;
        info->status = (int32_t)st;
        info->residual = n_pairs > 0 ? res : 0.0;
        info->min_gap = INFINITY;
        info->launches = c.launches;
    }
    return st;
}
