// Host side of the C ABI (include/alens.h): context and workspaces,
// argument checks, and the order of launches of each entry point.
#include <float.h>

#include <algorithm>
#include <limits.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "internal.cuh"

using namespace alens;

namespace {

// the CUDA error behind the calling thread's last ALENS_ERR_CUDA (aLENS_last_cuda_error)
static thread_local cudaError_t g_last_cuda_error = cudaSuccess;

#define CK(call)                                   \
    do {                                           \
        cudaError_t err__ = (call);                \
        if (err__ != cudaSuccess) {                \
            g_last_cuda_error = err__;             \
            return ALENS_ERR_CUDA;                 \
        }                                          \
    } while (0)

bool params_ok(const aLENS_params* p)
{
    if (!p) return false;
    if (!(p->diameter > 0) || !(p->length > 0) || !(p->viscosity > 0) || !(p->dt > 0) || !(p->delta_c >= 0)) return false;
    if (!(p->tol >= 0) || p->max_iter < 0 || p->max_iter > 10000000) return false;
    if (p->precision != ALENS_FP64 && p->precision != ALENS_MIXED) return false;
    if (!(2.0 * p->length / p->diameter > 1.0)) return false;   // ln(2L/D) > 0
    double rcut = p->length + p->diameter + p->delta_c;
    for (int k = 0; k < 3; ++k)
        if (!(p->box[k] >= rcut) || !isfinite(p->box[k])) return false;
    return true;
}

// Cell grid and drag coefficients for a parameter set.  Returns the Morton
// bits needed (or -1 if the grid exceeds 2^kMaxMortonBits cells per edge).
int make_geo(const aLENS_params* p, Geo* g, Mob* mob)
{
    memset(g, 0, sizeof(*g));
    g->diameter = p->diameter;
    g->length = p->length;
    g->half = 0.5 * p->length;
    g->delta_c = p->delta_c;
    g->dt = p->dt;
    g->rcut = p->length + p->diameter + p->delta_c;
    double maxbox = 0.0;
    int maxnc = 1;
    for (int k = 0; k < 3; ++k) {
        g->box[k] = p->box[k];
        g->boxf[k] = (float)p->box[k];
        int nc = (int)floor(p->box[k] / (g->rcut * (1.0 + 1e-9)));
        if (nc < 1) nc = 1;
        g->nc[k] = nc;
        g->cs[k] = p->box[k] / nc;
        g->inv_cs[k] = 1.0 / g->cs[k];
        if (p->box[k] > maxbox) maxbox = p->box[k];
        if (nc > maxnc) maxnc = nc;
    }
    int bits = 0;
    while ((1 << bits) < maxnc) ++bits;
    g->bits = bits;
    // float32 screen margin: covers rounding of coordinates of size maxbox
    // and of the float segment distance (see the search kernel)
    double margin = 0.02 * p->diameter + 2e-6 * maxbox;
    g->rcut_screen2 = (float)((g->rcut + margin) * (g->rcut + margin));
    double dmax = p->diameter + p->delta_c + margin;
    g->screen_d2 = (float)(dmax * dmax);
    // keep side of the float32 screen: the float closest points are points
    // of the two segments (clamped to half_f, at most one float ulp past the
    // ends), so their exact distance bounds the pair's minimum distance from
    // above; the float evaluation of that distance is off by at most
    // sqrt(3) (4 u B + 2 (L/2) u + 200 u) with u = 2^-24 and B the power of
    // two above the box (positions and the image shift rounded to float, the
    // axes rounded, a few float operations on values below 2^5 + L/2).  Twice
    // that, plus 1e-5 D, below D + delta_c keeps the pair without float64.
    double B = 1.0;
    while (B < maxbox) B *= 2.0;
    const double u = 1.0 / 16777216.0;
    const double kmargin = 2.0 * sqrt(3.0) * (4.0 * u * B + p->length * u + 200.0 * u) + 1e-5 * p->diameter;
    const double dkeep = p->diameter + p->delta_c - kmargin;
    g->keep_d2 = dkeep > 0.0 ? (float)(dkeep * dkeep) : 0.0f;
    g->half_f = (float)(0.5 * p->length);
    double zperp = 4.0 * M_PI * p->viscosity * p->length / log(2.0 * p->length / p->diameter);
    mob->inv_perp = 1.0 / zperp;
    mob->inv_par = 2.0 / zperp;
    mob->inv_rot = 12.0 / (zperp * p->length * p->length);
    mob->inv_spin = 1.0 / (M_PI * p->viscosity * p->diameter * p->diameter * p->length);
    return bits <= kMaxMortonBits ? bits : -1;
}

template <typename P>
cudaError_t dmalloc(P** ptr, size_t bytes)
{
    return cudaMalloc((void**)ptr, bytes > 0 ? bytes : 16);
}

void free_all(aLENS_ctx* c)
{
    void* ptrs[] = {c->xw, c->axis, c->unc, c->pos32, c->ax32, c->cellkey, c->sorted_id, c->spos32, c->sax32,
                    c->cell_count, c->cell_start, c->cell_cursor, c->rod_count, c->rod_ncand, c->rod_tmpstart, c->cand,
                    c->rowP, c->rowQ, c->cntQ, c->curQ, c->qlist, c->perm, c->rank, c->curP, c->ci, c->cj, c->pairs, c->phi, c->dgeom,
                    c->q64, c->scale64, c->solve_ws, c->partials, c->bstart, c->bar, c->dflags, c->dcount, c->scan_tmp,
                    c->systab, c->sysid, c->sysoff, c->sys_order, c->sys_iters, c->sys_res, c->adj_ws,
                    c->sp_ends, c->sp_arms, c->sp_kappa, c->sp_rest, c->comp64, c->fnc_buf, c->gin_buf,
                    c->row_keys, c->prev_keys, c->prev_gam};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    free(c->batch_host);
    free(c->batch_off_host);
    if (c->hflags) cudaFreeHost(c->hflags);
    if (c->hcount) cudaFreeHost(c->hcount);
    for (int k = 0; k < 8; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
}

__global__ void k_reset_counters(unsigned long long* cnt, int* flags)
{
    int t = threadIdx.x;
    if (t < C_NCOUNT) cnt[t] = t == C_MINGAP ? (unsigned long long)LLONG_MAX : 0ull;
    if (t < F_NFLAGS) flags[t] = 0;
}

aLENS_status reset_status(aLENS_ctx* c)
{
    k_reset_counters<<<1, 32, 0, c->stream>>>(c->dcount, c->dflags);
    ++c->launches;
    return cudaGetLastError() == cudaSuccess ? ALENS_OK : ALENS_ERR_CUDA;
}

aLENS_status read_status(aLENS_ctx* c)
{
    CK(cudaMemcpyAsync(c->hflags, c->dflags, sizeof(int) * F_NFLAGS, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(c->hcount, c->dcount, sizeof(unsigned long long) * C_NCOUNT, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return ALENS_OK;
}

double decode_gap(unsigned long long k)
{
    long long b = (long long)k;
    if (b == LLONG_MAX) return INFINITY;
    long long bits = b >= 0 ? b : b ^ 0x7fffffffffffffffLL;
    double v;
    memcpy(&v, &bits, sizeof(v));
    return v;
}

// Records a step's timing event.  While a graph is being recorded the event
// must stay an event of the graph (a plain record during capture only orders
// the captured work and is never recorded when the graph runs).
cudaError_t record_event(aLENS_ctx* c, cudaEvent_t e)
{
    return c->mdev ? cudaEventRecordWithFlags(e, c->stream, cudaEventRecordExternal) : cudaEventRecord(e, c->stream);
}

float elapsed(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        ms = -1.f;
        cudaGetLastError();   // a timing that cannot be read is not an error of the step
    }
    return ms;
}

bool rods_ok(aLENS_ctx* c, int64_t n) { return c && n >= 0 && n <= c->max_rods; }

// Every entry point but aLENS_step_batch works on the one system of the
// context's parameters.
void single_mode(aLENS_ctx* c)
{
    c->cur_systab = nullptr;
    c->cur_sysid = nullptr;
    c->cur_comp = nullptr;
    c->cur_nkeys = 1 << (3 * c->geo.bits);
}

// sysid[i] = the system whose rod range [off[s], off[s+1]) holds rod i.
__global__ void k_fill_sysid(int n, int ns, const long long* __restrict__ off, int* __restrict__ sysid)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = ns - 1;   // last s with off[s] <= i
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    sysid[i] = lo;
}

// Grows the cell arrays to hold nkeys cell keys (contents are reset by every search).
aLENS_status grow_keys(aLENS_ctx* c, long long nkeys)
{
    if (nkeys <= c->max_keys) return ALENS_OK;
    CK(cudaStreamSynchronize(c->stream));
    int* na[3] = {nullptr, nullptr, nullptr};
    int* nscan = nullptr;
    int tiles = (int)((std::max((long long)c->max_rods, nkeys) + 4095) / 4096) + 2;
    bool ok = true;
    for (int k = 0; k < 3; ++k) ok &= dmalloc(&na[k], ((size_t)nkeys + 1) * sizeof(int)) == cudaSuccess;
    if (tiles > c->scan_tmp_len) ok &= dmalloc(&nscan, (size_t)tiles * sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        for (int k = 0; k < 3; ++k) if (na[k]) cudaFree(na[k]);
        if (nscan) cudaFree(nscan);
        return ALENS_ERR_NOMEM;
    }
    cudaFree(c->cell_count); cudaFree(c->cell_start); cudaFree(c->cell_cursor);
    c->cell_count = na[0]; c->cell_start = na[1]; c->cell_cursor = na[2];
    if (nscan) { cudaFree(c->scan_tmp); c->scan_tmp = nscan; c->scan_tmp_len = tiles; }
    c->max_keys = (int)nkeys;
    return ALENS_OK;
}

// Validates the batch description and puts its tables on the device:
// per-system geometry (cell keys offset so that the systems' key ranges are
// disjoint and in system order) and the system id of every rod.
aLENS_status batch_tables(aLENS_ctx* c, int ns, const aLENS_system* sys, const int64_t* off)
{
    if (ns < 1 || ns > (1 << 20) || !sys || !off || off[0] != 0) return ALENS_ERR_INVALID;
    for (int s = 0; s < ns; ++s)
        if (off[s + 1] < off[s]) return ALENS_ERR_INVALID;
    if (off[ns] > c->max_rods) return ALENS_ERR_INVALID;
    const bool same = c->batch_n == ns && c->batch_host && c->batch_off_host &&
                      memcmp(c->batch_host, sys, sizeof(aLENS_system) * ns) == 0 &&
                      memcmp(c->batch_off_host, off, sizeof(int64_t) * (ns + 1)) == 0;
    if (same) {
        c->cur_nkeys = c->batch_keys;
        return ALENS_OK;
    }
    ++c->tables_epoch;   // a recorded batched step no longer applies
    SysGeo* tab = (SysGeo*)calloc((size_t)ns, sizeof(SysGeo));
    long long* loff = (long long*)malloc(sizeof(long long) * (ns + 1));
    if (!tab || !loff) { free(tab); free(loff); return ALENS_ERR_NOMEM; }
    long long keys = 0;
    aLENS_status st = ALENS_OK;
    for (int s = 0; s < ns && st == ALENS_OK; ++s) {
        aLENS_params p = c->p;
        for (int k = 0; k < 3; ++k) p.box[k] = sys[s].box[k];
        p.length = sys[s].length;
        int bits;
        if (!params_ok(&p) || (bits = make_geo(&p, &tab[s].g, &tab[s].mob)) < 0) { st = ALENS_ERR_INVALID; break; }
        tab[s].key_base = (int)keys;
        keys += 1ll << (3 * bits);
        if (keys > (1ll << 30)) st = ALENS_ERR_INVALID;
    }
    for (int s = 0; s <= ns; ++s) loff[s] = (long long)off[s];
    if (st == ALENS_OK) st = grow_keys(c, keys);
    if (st == ALENS_OK && ns > c->max_systems) {
        cudaStreamSynchronize(c->stream);
        void* old[] = {c->systab, c->sysoff, c->sys_order, c->sys_iters, c->sys_res};
        for (void* q : old)
            if (q) cudaFree(q);
        c->systab = nullptr; c->sysoff = nullptr; c->sys_order = nullptr; c->sys_iters = nullptr;
        c->sys_res = nullptr; c->max_systems = 0;
        if (dmalloc(&c->systab, sizeof(SysGeo) * ns) != cudaSuccess ||
            dmalloc(&c->sysoff, sizeof(long long) * (ns + 1)) != cudaSuccess ||
            dmalloc(&c->sys_order, sizeof(int) * sys_queue_ints(ns)) != cudaSuccess ||
            dmalloc(&c->sys_iters, 2 * sizeof(int) * ns) != cudaSuccess ||   // iterations, then blocks
            dmalloc(&c->sys_res, sizeof(double) * ns) != cudaSuccess) {
            cudaGetLastError();
            st = ALENS_ERR_NOMEM;
        } else {
            c->max_systems = ns;
        }
    }
    if (st == ALENS_OK && !c->sysid && dmalloc(&c->sysid, sizeof(int) * (size_t)c->max_rods) != cudaSuccess) {
        cudaGetLastError();
        st = ALENS_ERR_NOMEM;
    }
    void* hs = nullptr;
    int64_t* ho = nullptr;
    if (st == ALENS_OK) {
        hs = malloc(sizeof(aLENS_system) * ns);
        ho = (int64_t*)malloc(sizeof(int64_t) * (ns + 1));
        if (!hs || !ho) st = ALENS_ERR_NOMEM;
    }
    if (st == ALENS_OK) {
        // pageable sources: the calls return once the data is staged
        if (cudaMemcpyAsync(c->systab, tab, sizeof(SysGeo) * ns, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
            cudaMemcpyAsync(c->sysoff, loff, sizeof(long long) * (ns + 1), cudaMemcpyHostToDevice, c->stream) !=
                cudaSuccess)
            st = ALENS_ERR_CUDA;
    }
    if (st == ALENS_OK && off[ns] > 0) {
        int n = (int)off[ns];
        k_fill_sysid<<<(n + 255) / 256, 256, 0, c->stream>>>(n, ns, c->sysoff, c->sysid);
        ++c->launches;
        if (cudaGetLastError() != cudaSuccess) st = ALENS_ERR_CUDA;
    }
    free(tab);
    free(loff);
    if (st != ALENS_OK) {
        free(hs); free(ho);
        c->batch_n = 0;   // the device tables may be stale
        return st;
    }
    memcpy(hs, sys, sizeof(aLENS_system) * ns);
    memcpy(ho, off, sizeof(int64_t) * (ns + 1));
    free(c->batch_host); free(c->batch_off_host);
    c->batch_host = hs; c->batch_off_host = ho;
    c->batch_n = ns;
    c->batch_keys = (int)keys;
    c->cur_nkeys = (int)keys;
    return ALENS_OK;
}

// Runs the solver on the layout already set up; fills info.
aLENS_status run_solver(aLENS_ctx* c, int n, int m, aLENS_info* info, cudaEvent_t e0, cudaEvent_t e1)
{
    CK(record_event(c, e0));
    if (m > 0) CK(launch_solve(c, n, m, c->p.precision));
    CK(record_event(c, e1));
    (void)info;
    return ALENS_OK;
}

}  // namespace

extern "C" {

const char* aLENS_status_string(aLENS_status s)
{
    switch (s) {
        case ALENS_OK: return "ok";
        case ALENS_ERR_INVALID: return "invalid argument or input";
        case ALENS_ERR_CAPACITY: return "buffer capacity exceeded";
        case ALENS_ERR_NOT_CONVERGED: return "solver reached max_iter before the tolerance";
        case ALENS_ERR_TIMEOUT: return "a bounded grid-wide wait timed out";
        case ALENS_ERR_CUDA: return "CUDA runtime error";
        case ALENS_ERR_NOMEM: return "out of device memory";
        case ALENS_ERR_NOT_IMPLEMENTED: return "not implemented";
    }
    return "unknown status";
}

aLENS_status aLENS_create(const aLENS_params* params, int64_t max_rods, int64_t max_pairs, void* cuda_stream,
                          aLENS_ctx** out)
{
    if (!out) return ALENS_ERR_INVALID;
    *out = nullptr;
    if (!params_ok(params) || max_rods < 1 || max_pairs < 1 || max_rods > (1 << 26) || max_pairs > INT_MAX / 9)
        return ALENS_ERR_INVALID;
    Geo geo;
    Mob mob;
    if (make_geo(params, &geo, &mob) < 0) return ALENS_ERR_INVALID;
    aLENS_ctx* c = (aLENS_ctx*)calloc(1, sizeof(aLENS_ctx));
    if (!c) return ALENS_ERR_NOMEM;
    c->p = *params;
    c->geo = geo;
    c->mob = mob;
    c->max_rods = max_rods;
    c->max_pairs = max_pairs;
    c->stream = (cudaStream_t)cuda_stream;
    c->wait_s = 5.0;
    c->scale_beta = kDefaultScaleBeta;
    c->solve_threads = 768;   // the lowest time per iteration of 512, 768 and 1024 at 1e5 rods on 152 SMs
    c->solve_bps = 0;
    c->solve_barriers = 1;
    c->batch_threads = 1024;
    c->batch_cluster = 8;
    c->wall_axis = -1;
    if (cudaGetDevice(&c->device) != cudaSuccess) { free(c); return ALENS_ERR_CUDA; }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) { free(c); return ALENS_ERR_CUDA; }
    c->num_sms = prop.multiProcessorCount;
    c->smem_optin = (int)prop.sharedMemPerBlockOptin;
    int clk = 0;
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, c->device);
    c->clock_khz = clk > 0 ? clk : 2.1e6;
    c->coop_ok = prop.cooperativeLaunch;
    c->batch_coop = -1;
    cudaDeviceGetAttribute(&c->l2_bytes, cudaDevAttrL2CacheSize, c->device);
    cudaDeviceGetAttribute(&c->l2_window_max, cudaDevAttrMaxAccessPolicyWindowSize, c->device);
    cudaDeviceGetAttribute(&c->l2_persist_max, cudaDevAttrMaxPersistingL2CacheSize, c->device);
    c->max_keys = 1 << (3 * geo.bits);
    c->max_blocks = c->num_sms * 8;
    size_t np = (size_t)max_rods, mp = (size_t)max_pairs;
    int scan_tiles = (int)((std::max(np, (size_t)c->max_keys) + 4095) / 4096) + 2;
    c->scan_tmp_len = scan_tiles;
    bool ok = true;
    ok &= dmalloc(&c->xw, 3 * np * sizeof(double)) == cudaSuccess;
    ok &= dmalloc(&c->axis, 3 * np * sizeof(double)) == cudaSuccess;
    ok &= dmalloc(&c->unc, 6 * np * sizeof(double)) == cudaSuccess;
    ok &= dmalloc(&c->pos32, np * sizeof(float4)) == cudaSuccess;
    ok &= dmalloc(&c->ax32, np * sizeof(float4)) == cudaSuccess;
    ok &= dmalloc(&c->cellkey, np * sizeof(uint32_t)) == cudaSuccess;
    ok &= dmalloc(&c->sorted_id, np * sizeof(int)) == cudaSuccess;
    ok &= dmalloc(&c->spos32, np * sizeof(float4)) == cudaSuccess;
    ok &= dmalloc(&c->sax32, np * sizeof(float4)) == cudaSuccess;
    ok &= dmalloc(&c->cell_count, ((size_t)c->max_keys + 1) * sizeof(int)) == cudaSuccess;
    ok &= dmalloc(&c->cell_start, ((size_t)c->max_keys + 1) * sizeof(int)) == cudaSuccess;
    ok &= dmalloc(&c->cell_cursor, ((size_t)c->max_keys + 1) * sizeof(int)) == cudaSuccess;
    ok &= dmalloc(&c->rod_count, (np + 1) * sizeof(int)) == cudaSuccess;
    ok &= dmalloc(&c->rod_ncand, np * sizeof(int)) == cudaSuccess;
    ok &= dmalloc(&c->rod_tmpstart, np * sizeof(long long)) == cudaSuccess;
    c->cand_cap = 2 * (long long)mp + 4096;
    ok &= dmalloc(&c->cand, (size_t)c->cand_cap * sizeof(unsigned long long)) == cudaSuccess;
    ok &= dmalloc(&c->rowP, (np + 1) * sizeof(int)) == cudaSuccess;
    ok &= dmalloc(&c->rowQ, (np + 1) * sizeof(int)) == cudaSuccess;
    ok &= dmalloc(&c->cntQ, (np + 1) * sizeof(int)) == cudaSuccess;
    ok &= dmalloc(&c->curQ, (np + 1) * sizeof(int)) == cudaSuccess;
    ok &= dmalloc(&c->qlist, mp * sizeof(int)) == cudaSuccess;
    ok &= dmalloc(&c->perm, mp * sizeof(int)) == cudaSuccess;
    ok &= dmalloc(&c->rank, np * sizeof(int)) == cudaSuccess;
    ok &= dmalloc(&c->curP, (np + 1) * sizeof(int)) == cudaSuccess;
    ok &= dmalloc(&c->ci, mp * sizeof(int)) == cudaSuccess;
    ok &= dmalloc(&c->cj, mp * sizeof(int)) == cudaSuccess;
    ok &= dmalloc(&c->pairs, 3 * mp * sizeof(int32_t)) == cudaSuccess;
    ok &= dmalloc(&c->phi, mp * sizeof(double)) == cudaSuccess;
    ok &= dmalloc(&c->dgeom, 9 * mp * sizeof(double)) == cudaSuccess;
    ok &= dmalloc(&c->q64, mp * sizeof(double)) == cudaSuccess;
    ok &= dmalloc(&c->scale64, mp * sizeof(double)) == cudaSuccess;
    // solver buffers, sized for float64; the float32 views alias the same memory
    // every slice starts on a 64-byte boundary (vector loads): 8 elements of slack each
    size_t solve_elems = 9 * mp + 8 * mp + mp + 3 * np + 8 * mp + 18 * np + mp + 4 * np + mp + mp + 8 * 14 + 8 * mp;
    ok &= dmalloc((char**)&c->solve_ws, solve_elems * sizeof(double)) == cudaSuccess;
    ok &= dmalloc(&c->partials, ((size_t)c->max_blocks + 4) * 8 * sizeof(double)) == cudaSuccess;
    ok &= dmalloc(&c->bstart, ((size_t)c->max_blocks + 1) * sizeof(int)) == cudaSuccess;
    ok &= dmalloc(&c->bar, 4 * sizeof(unsigned)) == cudaSuccess;
    ok &= dmalloc(&c->dflags, F_NFLAGS * sizeof(int)) == cudaSuccess;
    ok &= dmalloc(&c->dcount, C_NCOUNT * sizeof(unsigned long long)) == cudaSuccess;
    ok &= dmalloc(&c->scan_tmp, (size_t)scan_tiles * sizeof(int)) == cudaSuccess;
    ok &= cudaMallocHost((void**)&c->hflags, F_NFLAGS * sizeof(int)) == cudaSuccess;
    ok &= cudaMallocHost((void**)&c->hcount, C_NCOUNT * sizeof(unsigned long long)) == cudaSuccess;
    for (int k = 0; k < 8 && ok; ++k) ok &= cudaEventCreate(&c->ev[k]) == cudaSuccess;
    ok &= cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) == cudaSuccess;
    ok &= cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    ok &= cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_all(c);
        free(c);
        return ALENS_ERR_NOMEM;
    }
    {
        // (gamma, g) pairs first and U next keep their vector loads aligned
        double* base = (double*)c->solve_ws;
        size_t o = 0;
        auto carve64 = [&](size_t cnt) { double* r = base + o; o = (o + cnt + 7) & ~(size_t)7; return r; };
        SolveBufs<double>& s = c->sb64;
        s.gg[0] = carve64(4 * mp); s.gg[1] = carve64(4 * mp); s.U = carve64(6 * np); s.U2 = carve64(6 * np);
        s.Uref = carve64(6 * np);
        s.gref = carve64(mp);
        s.rec = carve64(9 * mp); s.qe = carve64(8 * mp); s.q = carve64(mp); s.ax = carve64(3 * np);
        s.mobr = carve64(4 * np);
        s.comp = carve64(mp);
        s.isc = carve64(mp);
        s.pe = nullptr;   // the float64 rod phase reads rec (its arithmetic bounds it)
        s.lop = nullptr;
        s.loq = nullptr;
        float* fb = (float*)c->solve_ws;
        size_t f = 0;
        auto carve32 = [&](size_t cnt) { float* r = fb + f; f = (f + cnt + 7) & ~(size_t)7; return r; };
        SolveBufs<float>& t = c->sb32;
        t.gg[0] = carve32(4 * mp); t.gg[1] = carve32(4 * mp); t.U = carve32(6 * np); t.U2 = carve32(6 * np);
        t.Uref = carve32(6 * np);
        t.gref = carve32(mp);
        t.rec = carve32(9 * mp); t.qe = carve32(8 * mp); t.q = carve32(mp); t.ax = carve32(3 * np);
        t.mobr = carve32(4 * np);
        t.comp = carve32(mp);
        t.isc = carve32(mp);
        t.pe = carve32(8 * mp);
        // the float32 views use at most 71 mp + 25 np of the workspace's
        // 74 mp + 50 np floats: room for the owner-side records, the low
        // parts and their rows
        t.rec_lo = carve32(9 * mp); t.qe_lo = carve32(8 * mp); t.q_lo = carve32(mp);
        t.lop = carve32(8 * mp); t.loq = carve32(8 * mp);
    }
    if (cudaMemsetAsync(c->cell_cursor, 0, ((size_t)c->max_keys + 1) * sizeof(int), c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        free_all(c);
        free(c);
        return ALENS_ERR_CUDA;
    }
    *out = c;
    return ALENS_OK;
}

void aLENS_destroy(aLENS_ctx* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    if (c->persist_set) {   // the persisting L2 set-aside back to what it was, unless changed since
        int dev = -1;
        const bool other = cudaGetDevice(&dev) == cudaSuccess && dev != c->device;
        if (other) cudaSetDevice(c->device);   // the limit belongs to the context's device
        size_t cur = 0;
        if (cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) == cudaSuccess && cur == c->persist_set)
            cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, c->persist_prev);
        cudaCtxResetPersistingL2Cache();
        if (other) cudaSetDevice(dev);
        cudaGetLastError();
    }
    free_all(c);
    free(c);
}

aLENS_status aLENS_set_params(aLENS_ctx* c, const aLENS_params* params)
{
    if (!c || !params_ok(params)) return ALENS_ERR_INVALID;
    Geo geo;
    Mob mob;
    int bits = make_geo(params, &geo, &mob);
    if (bits < 0) return ALENS_ERR_INVALID;
    if ((1 << (3 * bits)) > c->max_keys) return ALENS_ERR_CAPACITY;
    c->p = *params;
    c->geo = geo;
    c->mob = mob;
    c->batch_n = 0;   // batch tables derive from the parameters: rebuild on the next batch
    c->prev_valid = 0;
    return ALENS_OK;
}

aLENS_status aLENS_set_wait_limit(aLENS_ctx* c, double seconds)
{
    if (!c || !(seconds > 0) || seconds > 3600) return ALENS_ERR_INVALID;
    c->wait_s = seconds;
    return ALENS_OK;
}

aLENS_status aLENS_set_scaling(aLENS_ctx* c, double beta)
{
    if (!c || !(beta >= 0.0 && beta <= 1.0)) return ALENS_ERR_INVALID;
    c->scale_beta = beta;
    return ALENS_OK;
}

static void drop_graph(aLENS_ctx* c);

aLENS_status aLENS_inject_fault(aLENS_ctx* c, int32_t mode)
{
    if (!c || mode < 0 || mode > 3) return ALENS_ERR_INVALID;
    if (mode == 3) {   // as after a refused cooperative cluster launch: no pairs from now on
        c->batch_coop = 0;
        drop_graph(c);
        return ALENS_OK;
    }
    c->fault_mode = mode;
    return ALENS_OK;
}

aLENS_status aLENS_set_launch(aLENS_ctx* c, int32_t threads, int32_t blocks_per_sm)
{
    if (!c || threads < 32 || threads > 1024 || threads % 32 != 0 || blocks_per_sm < 0) return ALENS_ERR_INVALID;
    c->solve_threads = threads;
    c->solve_bps = blocks_per_sm;
    return ALENS_OK;
}

aLENS_status aLENS_set_solver_schedule(aLENS_ctx* c, int32_t barriers)
{
    if (!c || (barriers != 1 && barriers != 2)) return ALENS_ERR_INVALID;
    c->solve_barriers = barriers;
    return ALENS_OK;
}

// Pack + cell list + search; leaves the per-rod kept counts and the
// candidate keys in the context and the pair total in hcount[C_PAIRS].
// Synchronises once (twice if the candidate buffer overflowed, to count the
// pairs exactly).
// The search's kernels (no host readback): pack, cell list, pair search
// and the float64 decision.
static aLENS_status search_kernels(aLENS_ctx* c, int n, const double* x, const double* quat, const double* fnc)
{
    int nkeys = c->cur_nkeys;
    aLENS_status st = reset_status(c);
    if (st != ALENS_OK) return st;
    CK(cudaMemsetAsync(c->cell_count, 0, ((size_t)nkeys + 1) * sizeof(int), c->stream));
    CK(cudaMemsetAsync(c->cell_cursor, 0, ((size_t)nkeys + 1) * sizeof(int), c->stream));
    CK(cudaMemsetAsync(c->rod_count, 0, ((size_t)n + 1) * sizeof(int), c->stream));
    CK(launch_pack(c, n, x, quat, fnc, true));
    if (c->wall_axis >= 0 && c->cur_systab == nullptr) {
        CK(cudaMemsetAsync(c->cntQ, 0, ((size_t)n + 1) * sizeof(int), c->stream));
        CK(launch_count_walls(c, n));
    }
    CK(launch_cell_sort(c, n));
    CK(launch_search(c, n));
    return ALENS_OK;
}

static aLENS_status search_phase(aLENS_ctx* c, int n, const double* x, const double* quat, const double* fnc)
{
    aLENS_status st = search_kernels(c, n, x, quat, fnc);
    if (st != ALENS_OK) return st;
    if ((st = read_status(c)) != ALENS_OK) return st;
    if (c->hflags[F_ERR] != 0) return (aLENS_status)c->hflags[F_ERR];
    if ((long long)c->hcount[C_CAND] > c->cand_cap) {
        // candidate buffer too small: count the pairs exactly, report CAPACITY
        CK(reset_status(c) == ALENS_OK ? cudaSuccess : cudaErrorUnknown);
        CK(launch_search_count(c, n));
        if ((st = read_status(c)) != ALENS_OK) return st;
        return ALENS_ERR_CAPACITY;
    }
    return ALENS_OK;
}

aLENS_status aLENS_build_neighbors(aLENS_ctx* c, int64_t n, const double* x, const double* quat, int32_t* pairs,
                                   int64_t pairs_cap, int64_t* n_pairs)
{
    if (c) { c->launches = 0; c->last_solver = 0; single_mode(c); }
    if (!rods_ok(c, n) || !n_pairs || (n > 0 && (!x || !quat)) || pairs_cap < 0 || (pairs_cap > 0 && !pairs))
        return ALENS_ERR_INVALID;
    long long cap = std::min<long long>(pairs_cap, c->max_pairs);
    aLENS_status st = search_phase(c, (int)n, x, quat, nullptr);
    long long total = (long long)c->hcount[C_PAIRS];
    *n_pairs = total;
    if (st != ALENS_OK) return st;
    if (total > cap) return ALENS_ERR_CAPACITY;
    CK(launch_emit_pairs(c, (int)n, pairs));
    CK(cudaStreamSynchronize(c->stream));
    return ALENS_OK;
}

aLENS_status aLENS_assemble_constraints(aLENS_ctx* c, int64_t n, const double* x, const double* quat,
                                        const double* f_nc, int64_t n_pairs, const int32_t* pairs, double* phi,
                                        double* dgeom, double* q)
{
    if (c) { c->launches = 0; c->last_solver = 0; single_mode(c); }
    if (!rods_ok(c, n) || n_pairs < 0 || n_pairs > c->max_pairs) return ALENS_ERR_INVALID;
    if (n > 0 && (!x || !quat)) return ALENS_ERR_INVALID;
    if (n_pairs > 0 && (!pairs || !phi || !dgeom || !q)) return ALENS_ERR_INVALID;
    aLENS_status st = reset_status(c);
    if (st != ALENS_OK) return st;
    CK(launch_pack(c, (int)n, x, quat, f_nc, false));
    CK(launch_assemble(c, (int)n, (int)n_pairs, pairs, phi, dgeom, q));
    if ((st = read_status(c)) != ALENS_OK) return st;
    if (c->hflags[F_ERR] != 0) return (aLENS_status)c->hflags[F_ERR];
    return ALENS_OK;
}

static void fill_info(aLENS_ctx* c, aLENS_info* info, int64_t m, aLENS_status st)
{
    if (!info) return;
    info->n_pairs = m;
    info->n_overlap = (int64_t)c->hcount[C_OVERLAP];
    info->min_gap = decode_gap(c->hcount[C_MINGAP]);
    info->iters = c->hflags[F_ITERS];
    double res;
    memcpy(&res, &c->hcount[C_RESID], sizeof(res));
    info->residual = m > 0 ? res : 0.0;
    info->status = (int32_t)st;
    info->launches = c->launches;
    info->solver = c->last_solver;
}

static aLENS_status solve_status(aLENS_ctx* c, int64_t m)
{
    if (c->hflags[F_SOLVE_ERR] != 0) return (aLENS_status)c->hflags[F_SOLVE_ERR];
    if (c->hflags[F_ERR] != 0) return (aLENS_status)c->hflags[F_ERR];
    if (m > 0) {
        double res;
        memcpy(&res, &c->hcount[C_RESID], sizeof(res));
        if (!(res <= c->p.tol)) return ALENS_ERR_NOT_CONVERGED;
    }
    return ALENS_OK;
}

aLENS_status aLENS_solve_lcp(aLENS_ctx* c, int64_t n, const double* quat, int64_t n_pairs, const int32_t* pairs,
                             const double* dgeom, const double* q, double* gamma, aLENS_info* info)
{
    if (c) { c->launches = 0; c->last_solver = 0; single_mode(c); }
    if (!rods_ok(c, n) || n_pairs < 0 || n_pairs > c->max_pairs) return ALENS_ERR_INVALID;
    if (n > 0 && !quat) return ALENS_ERR_INVALID;
    if (n_pairs > 0 && (!pairs || !dgeom || !q || !gamma)) return ALENS_ERR_INVALID;
    if (n_pairs > 0 && !c->coop_ok) return ALENS_ERR_CUDA;
    aLENS_status st = reset_status(c);
    if (st != ALENS_OK) return st;
    CK(cudaEventRecord(c->ev[0], c->stream));
    CK(launch_solve_setup_check(c, (int)n, (int)n_pairs, pairs));
    if ((st = read_status(c)) != ALENS_OK) return st;
    if (c->hflags[F_ERR] != 0) return (aLENS_status)c->hflags[F_ERR];
    CK(launch_solve_setup(c, (int)n, (int)n_pairs, pairs, dgeom, q, gamma, quat, c->p.precision, nullptr));
    if ((st = run_solver(c, (int)n, (int)n_pairs, info, c->ev[1], c->ev[2])) != ALENS_OK) return st;
    if ((st = read_status(c)) != ALENS_OK) return st;
    if (c->hflags[F_ERR] != 0) return (aLENS_status)c->hflags[F_ERR];
    st = solve_status(c, n_pairs);
    if (st == ALENS_OK || st == ALENS_ERR_NOT_CONVERGED) {
        CK(launch_gamma_out(c, (int)n_pairs, c->p.precision, gamma));
        CK(cudaStreamSynchronize(c->stream));
    }
    fill_info(c, info, n_pairs, st);
    if (info) {
        info->ms_build = 0.f;
        info->ms_assemble = elapsed(c->ev[0], c->ev[1]);
        info->ms_solve = elapsed(c->ev[1], c->ev[2]);
        info->ms_update = 0.f;
    }
    return st;
}

}  // extern "C"

// The step on the system(s) selected by cur_systab / cur_sysid / cur_nkeys.
// Trajectories: warm = start from the previous step's forces (matched row by
// row), keep = record this step's rows and forces for the next step.
struct StepOpts {
    bool warm = false;
    bool keep = false;
};

// The launch helpers enqueue on ctx->stream: while a StreamSwap lives, that
// is stream s.
struct StreamSwap {
    aLENS_ctx* c;
    cudaStream_t own;
    StreamSwap(aLENS_ctx* c_, cudaStream_t s) : c(c_), own(c_->stream) { c->stream = s; }
    ~StreamSwap() { c->stream = own; }
};

// The solver layout (ranks, owner-major CSR, Q-side offsets, the rods' axes
// and drags) needs the pair list but none of the assembled values, so it
// runs on the side stream while the assembly, bound by the FP64 pipe, runs
// on the step's stream; the step's stream waits for ev_join before the
// records are filled.  Same kernels and arguments as in sequence.
static aLENS_status fork_layout(aLENS_ctx* c, int n, int m, const double* quat)
{
    CK(cudaEventRecord(c->ev_fork, c->stream));
    CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    {
        StreamSwap on(c, c->side);
        CK(launch_rank(c, n));
        CK(launch_solve_layout(c, n, m, c->pairs, quat, c->p.precision, c->rank));
    }
    CK(cudaEventRecord(c->ev_join, c->side));
    return ALENS_OK;
}

static aLENS_status step_impl(aLENS_ctx* c, int64_t n, double* x, double* quat, const double* f_nc,
                              int32_t* pairs_out, double* gamma_out, double* vel_out, aLENS_info* info,
                              StepOpts opt = StepOpts(), int64_t* walls_out = nullptr)
{
    CK(cudaEventRecord(c->ev[0], c->stream));
    aLENS_status st = search_phase(c, (int)n, x, quat, f_nc);
    if (st != ALENS_OK) {
        if (info) { memset(info, 0, sizeof(*info)); info->status = st; info->n_pairs = (int64_t)c->hcount[C_PAIRS]; }
        return st;
    }
    const bool walls = c->wall_axis >= 0 && c->cur_systab == nullptr;
    const long long mu = (long long)c->hcount[C_PAIRS];                  // collisions
    const long long mw = walls ? (long long)c->hcount[C_WALLS] : 0;     // wall contacts
    const long long m = mu + mw + c->sp_n;                               // then springs
    if (walls_out) *walls_out = mw;
    if (m > c->max_pairs) {
        if (info) { memset(info, 0, sizeof(*info)); info->status = ALENS_ERR_CAPACITY; info->n_pairs = mu; }
        return ALENS_ERR_CAPACITY;
    }
    CK(launch_emit_pairs(c, (int)n, c->pairs));
    CK(cudaEventRecord(c->ev[1], c->stream));
    // walls and springs append constraints after the assembly: then the layout follows it
    const bool beside = !walls && c->sp_n == 0;
    if (beside && (st = fork_layout(c, (int)n, (int)m, quat)) != ALENS_OK) return st;
    CK(launch_assemble(c, (int)n, (int)mu, c->pairs, c->phi, c->dgeom, c->q64));
    if (walls) CK(launch_emit_walls(c, (int)n, (int)mu));
    if (c->sp_n > 0) {
        CK(launch_assemble_springs(c, (int)n, (int)(mu + mw)));
        if ((st = read_status(c)) != ALENS_OK) return st;
        if (c->hflags[F_ERR] != 0) {   // a bad spring: nothing moved
            if (info) { memset(info, 0, sizeof(*info)); info->status = c->hflags[F_ERR]; info->n_pairs = mu; }
            return (aLENS_status)c->hflags[F_ERR];
        }
        c->cur_comp = c->comp64;
    }
    const double* gin = nullptr;
    if (opt.warm && c->prev_valid) {
        CK(launch_warm(c, (int)m, (int)mu, (int)mw, c->gin_buf));
        gin = c->gin_buf;
    }
    if (beside) {
        CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    } else {
        CK(launch_rank(c, (int)n));
        CK(launch_solve_layout(c, (int)n, (int)m, c->pairs, quat, c->p.precision, c->rank));
    }
    CK(launch_solve_fill(c, (int)n, (int)m, c->pairs, c->dgeom, c->q64, gin, c->p.precision, c->rank));
    if ((st = run_solver(c, (int)n, (int)m, info, c->ev[2], c->ev[3])) != ALENS_OK) return st;
    c->cur_comp = nullptr;
    CK(launch_update(c, (int)n, (int)m, x, quat, c->p.precision, vel_out, c->rank));
    CK(cudaEventRecord(c->ev[4], c->stream));
    if (gamma_out) CK(launch_gamma_out(c, (int)m, c->p.precision, gamma_out));
    if (opt.keep) {
        CK(launch_gamma_out(c, (int)m, c->p.precision, c->prev_gam));
        CK(launch_keep_keys(c, (int)m, (int)mu, (int)mw));
    }
    if (pairs_out && mu > 0)
        CK(cudaMemcpyAsync(pairs_out, c->pairs, sizeof(int32_t) * 3 * (size_t)mu, cudaMemcpyDeviceToDevice, c->stream));
    if ((st = read_status(c)) != ALENS_OK) return st;
    st = solve_status(c, m);
    if (opt.keep) c->prev_valid = st == ALENS_OK || st == ALENS_ERR_NOT_CONVERGED;
    fill_info(c, info, m, st);
    if (info) {
        info->n_pairs = mu;
        info->ms_build = elapsed(c->ev[0], c->ev[1]);
        info->ms_assemble = elapsed(c->ev[1], c->ev[2]);
        info->ms_solve = elapsed(c->ev[2], c->ev[3]);
        info->ms_update = elapsed(c->ev[3], c->ev[4]);
    }
    return st;
}

// A batched step without host readbacks, for recording as a CUDA graph:
// every kernel that depends on the constraint count is launched for the
// capacity and reads the count from the device (C_MEFF, set by the
// capacity check; 0 after a failure, and the update then leaves the rods
// untouched).  The caller reads the status back after the graph runs.
static aLENS_status step_graph_body(aLENS_ctx* c, int64_t n, double* x, double* quat, const double* f_nc,
                                    int32_t* pairs_out, double* gamma_out, double* vel_out, bool single)
{
    const int mcap = (int)c->max_pairs;
    c->mdev = c->dcount + C_MEFF;
    CK(record_event(c, c->ev[0]));
    aLENS_status st = search_kernels(c, (int)n, x, quat, f_nc);
    if (st == ALENS_OK) {
        CK(launch_check_capacity(c));
        CK(launch_emit_pairs(c, (int)n, c->pairs));
        CK(record_event(c, c->ev[1]));
        st = fork_layout(c, (int)n, mcap, quat);
    }
    if (st == ALENS_OK) {
        CK(launch_assemble(c, (int)n, mcap, c->pairs, c->phi, c->dgeom, c->q64));
        CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
        CK(launch_solve_fill(c, (int)n, mcap, c->pairs, c->dgeom, c->q64, nullptr, c->p.precision, c->rank));
        if (single) {
            CK(record_event(c, c->ev[2]));
            CK(launch_solve_graph1(c, (int)n, mcap, c->p.precision));
            CK(record_event(c, c->ev[3]));
        } else {
            st = run_solver(c, (int)n, mcap, nullptr, c->ev[2], c->ev[3]);
        }
    }
    if (st == ALENS_OK) {
        CK(launch_update(c, (int)n, mcap, x, quat, c->p.precision, vel_out, c->rank));
        CK(record_event(c, c->ev[4]));
        if (gamma_out) CK(launch_gamma_out(c, mcap, c->p.precision, gamma_out));
        if (pairs_out) CK(launch_copy_pairs(c, pairs_out));
    }
    c->mdev = nullptr;
    return st;
}

static void drop_graph(aLENS_ctx* c)
{
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
    c->graph_state = 0;
}

// The key of a recorded batched step: everything its launches bake in.
static aLENS_ctx::GraphKey graph_key(const aLENS_ctx* c, int64_t n, const double* x, const double* quat,
                                     const double* f_nc, const int32_t* pairs_out, const double* gamma_out,
                                     const double* vel_out)
{
    aLENS_ctx::GraphKey k;
    memset(&k, 0, sizeof(k));
    k.n = n;
    k.ptr[0] = x; k.ptr[1] = quat; k.ptr[2] = f_nc; k.ptr[3] = pairs_out; k.ptr[4] = gamma_out; k.ptr[5] = vel_out;
    k.p = c->p;
    k.beta = c->scale_beta;
    k.threads = c->batch_threads;
    k.cluster = c->batch_cluster;
    k.tables = c->tables_epoch;
    k.kind = 1;
    return k;
}

// The key of a recorded single-system step.
static aLENS_ctx::GraphKey single_key(const aLENS_ctx* c, int64_t n, const double* x, const double* quat,
                                      const double* f_nc, const int32_t* pairs_out, const double* gamma_out,
                                      const double* vel_out)
{
    aLENS_ctx::GraphKey k = graph_key(c, n, x, quat, f_nc, pairs_out, gamma_out, vel_out);
    k.threads = c->solve_threads;
    k.cluster = c->solve_bps;
    k.tables = 0;
    k.kind = 2;
    k.barriers = c->solve_barriers;
    return k;
}

// Records the step of the current key on a private stream (recording enqueues
// nothing: the graph runs on the context's stream) and instantiates it.
static aLENS_status record_step(aLENS_ctx* c, int64_t n, double* x, double* quat, const double* f_nc,
                                int32_t* pairs_out, double* gamma_out, double* vel_out, bool single)
{
    c->launches = 0;
    if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    cudaStream_t own = c->stream;
    c->stream = c->cap_stream;
    cudaError_t be = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    aLENS_status st = be == cudaSuccess ? step_graph_body(c, n, x, quat, f_nc, pairs_out, gamma_out, vel_out, single)
                                        : ALENS_ERR_CUDA;
    cudaGraph_t g = nullptr;
    const cudaError_t ce = be == cudaSuccess ? cudaStreamEndCapture(c->stream, &g) : be;
    c->stream = own;
    if (st != ALENS_OK || ce != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        drop_graph(c);
        return st != ALENS_OK ? st : ALENS_ERR_CUDA;
    }
    c->graph = g;
    if (cudaGraphInstantiate(&c->gexec, g, 0) != cudaSuccess) {
        cudaGetLastError();
        drop_graph(c);
        return ALENS_ERR_CUDA;
    }
    c->graph_launches = c->launches;
    c->graph_state = 2;
    return ALENS_OK;
}

// The outcome of a replayed step, read back after the graph ran.
static aLENS_status graph_outcome(aLENS_ctx* c, int64_t n, aLENS_info* info)
{
    aLENS_status st = read_status(c);
    if (st != ALENS_OK) return st;
    const long long mu = (long long)c->hcount[C_PAIRS];
    if (c->hflags[F_ERR] == ALENS_ERR_CAPACITY) {
        long long need = mu;
        if ((long long)c->hcount[C_CAND] > c->cand_cap) {
            // candidates overflowed: count the pairs exactly (nothing moved)
            CK(reset_status(c) == ALENS_OK ? cudaSuccess : cudaErrorUnknown);
            CK(launch_search_count(c, (int)n));
            if ((st = read_status(c)) != ALENS_OK) return st;
            need = (long long)c->hcount[C_PAIRS];
        }
        if (info) { memset(info, 0, sizeof(*info)); info->status = ALENS_ERR_CAPACITY; info->n_pairs = need; }
        return ALENS_ERR_CAPACITY;
    }
    if (c->hflags[F_ERR] != 0) {
        if (info) { memset(info, 0, sizeof(*info)); info->status = c->hflags[F_ERR]; info->n_pairs = mu; }
        return (aLENS_status)c->hflags[F_ERR];
    }
    st = solve_status(c, mu);
    fill_info(c, info, mu, st);
    if (info) {
        info->n_pairs = mu;
        info->ms_build = elapsed(c->ev[0], c->ev[1]);
        info->ms_assemble = elapsed(c->ev[1], c->ev[2]);
        info->ms_solve = elapsed(c->ev[2], c->ev[3]);
        info->ms_update = elapsed(c->ev[3], c->ev[4]);
    }
    return st;
}

// Replays (recording it first when needed) the graph of a batched step and
// reads its outcome back.  Returns ALENS_ERR_NOT_IMPLEMENTED when the step
// is to run eagerly instead (the first step of a new key).
static aLENS_status step_batch_graph(aLENS_ctx* c, int64_t n, double* x, double* quat, const double* f_nc,
                                     int32_t* pairs_out, double* gamma_out, double* vel_out, aLENS_info* info)
{
    const aLENS_ctx::GraphKey k = graph_key(c, n, x, quat, f_nc, pairs_out, gamma_out, vel_out);
    const bool same = c->graph_state > 0 && memcmp(&k, &c->gkey, sizeof(k)) == 0;
    if (!same) {
        drop_graph(c);
        c->gkey = k;
        c->graph_state = 1;   // this key runs eagerly once (tables, attributes, allocations settle)
        return ALENS_ERR_NOT_IMPLEMENTED;
    }
    if (c->graph_state == 1) {
        const aLENS_status rs = record_step(c, n, x, quat, f_nc, pairs_out, gamma_out, vel_out, false);
        if (rs != ALENS_OK) return rs;
    }
    CK(cudaGraphLaunch(c->gexec, c->stream));
    c->launches = c->graph_launches;
    c->last_solver = 4;
    return graph_outcome(c, n, info);
}

// The same for a single-system step: the first step of a key runs eagerly
// (ALENS_ERR_NOT_IMPLEMENTED), and a key whose eager step did not run the
// one-barrier solver, or whose replay found a share too big for the
// recorded launch (kSolveRedo: nothing moved), stays eager.
static aLENS_status step_single_graph(aLENS_ctx* c, int64_t n, double* x, double* quat, const double* f_nc,
                                      int32_t* pairs_out, double* gamma_out, double* vel_out, aLENS_info* info)
{
    const aLENS_ctx::GraphKey k = single_key(c, n, x, quat, f_nc, pairs_out, gamma_out, vel_out);
    const bool same = c->graph_state > 0 && memcmp(&k, &c->gkey, sizeof(k)) == 0;
    if (!same) {
        drop_graph(c);
        c->gkey = k;
        c->graph_state = 1;
        return ALENS_ERR_NOT_IMPLEMENTED;
    }
    if (c->graph_state == 3) return ALENS_ERR_NOT_IMPLEMENTED;
    if (c->graph_state == 1) {
        bool ok = false;
        CK(graph1_possible(c, c->p.precision, ok));
        if (!ok) {
            c->graph_state = 3;
            return ALENS_ERR_NOT_IMPLEMENTED;
        }
        const aLENS_status rs = record_step(c, n, x, quat, f_nc, pairs_out, gamma_out, vel_out, true);
        if (rs != ALENS_OK) return rs;
    }
    CK(cudaGraphLaunch(c->gexec, c->stream));
    c->launches = c->graph_launches;
    c->last_solver = 1;
    CK(cudaMemcpyAsync(c->hflags, c->dflags, sizeof(int) * F_NFLAGS, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (c->hflags[F_SOLVE_ERR] == kSolveRedo) {
        drop_graph(c);
        c->gkey = k;
        c->graph_state = 3;
        return ALENS_ERR_NOT_IMPLEMENTED;
    }
    return graph_outcome(c, n, info);
}

extern "C" {

aLENS_status aLENS_step(aLENS_ctx* c, int64_t n, double* x, double* quat, const double* f_nc, int32_t* pairs_out,
                        double* gamma_out, double* vel_out, aLENS_info* info)
{
    if (c) { c->launches = 0; c->last_solver = 0; single_mode(c); }
    if (!rods_ok(c, n) || (n > 0 && (!x || !quat))) return ALENS_ERR_INVALID;
    if (!c->coop_ok) return ALENS_ERR_CUDA;
    // graph mode: plain steps (no springs, walls or bounded-wait test hook)
    const bool graphable = c->step_graph && n > 0 && c->sp_n == 0 && c->wall_axis < 0 && c->fault_mode != 1;
    aLENS_status st = ALENS_ERR_NOT_IMPLEMENTED;
    if (graphable) st = step_single_graph(c, n, x, quat, f_nc, pairs_out, gamma_out, vel_out, info);
    if (st != ALENS_ERR_NOT_IMPLEMENTED) return st;
    c->launches = 0;
    st = step_impl(c, n, x, quat, f_nc, pairs_out, gamma_out, vel_out, info);
    // a key whose eager step did not run the one-barrier solver stays eager
    if (graphable && c->graph_state == 1 && c->last_solver != 1) c->graph_state = 3;
    return st;
}

aLENS_status aLENS_set_springs(aLENS_ctx* c, int64_t n_springs, const int32_t* ends, const double* arms,
                               const double* kappa, const double* rest)
{
    if (!c || n_springs < 0 || n_springs > c->max_pairs) return ALENS_ERR_INVALID;
    if (n_springs > 0 && (!ends || !arms || !kappa || !rest)) return ALENS_ERR_INVALID;
    if (n_springs > c->sp_cap) {
        CK(cudaStreamSynchronize(c->stream));
        void* old[] = {c->sp_ends, c->sp_arms, c->sp_kappa, c->sp_rest};
        for (void* q : old)
            if (q) cudaFree(q);
        c->sp_ends = nullptr; c->sp_arms = nullptr; c->sp_kappa = nullptr; c->sp_rest = nullptr;
        c->sp_cap = 0;
        c->sp_n = 0;
        const size_t nb = (size_t)n_springs;
        if (dmalloc(&c->sp_ends, 2 * nb * sizeof(int32_t)) != cudaSuccess ||
            dmalloc(&c->sp_arms, 2 * nb * sizeof(double)) != cudaSuccess ||
            dmalloc(&c->sp_kappa, nb * sizeof(double)) != cudaSuccess ||
            dmalloc(&c->sp_rest, nb * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return ALENS_ERR_NOMEM;
        }
        c->sp_cap = n_springs;
    }
    if (n_springs > 0 && !c->comp64) {
        if (dmalloc(&c->comp64, (size_t)c->max_pairs * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return ALENS_ERR_NOMEM;
        }
    }
    const size_t nb = (size_t)n_springs;
    if (nb > 0) {
        CK(cudaMemcpyAsync(c->sp_ends, ends, 2 * nb * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(c->sp_arms, arms, 2 * nb * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(c->sp_kappa, kappa, nb * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(c->sp_rest, rest, nb * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    }
    c->sp_n = n_springs;
    ++c->sp_version;
    return ALENS_OK;
}

aLENS_status aLENS_set_walls(aLENS_ctx* c, int32_t axis, double lo, double hi)
{
    if (!c || axis < -1 || axis > 2) return ALENS_ERR_INVALID;
    if (axis >= 0) {
        const double box = c->p.box[axis];
        const double rcut = c->p.length + c->p.diameter + c->p.delta_c;
        if (!(lo >= 0.0) || !(hi > lo) || !(hi <= box) || !(box - (hi - lo) >= rcut)) return ALENS_ERR_INVALID;
    }
    c->wall_axis = axis;
    c->wall_lo = lo;
    c->wall_hi = hi;
    c->prev_valid = 0;
    return ALENS_OK;
}

aLENS_status aLENS_brownian(aLENS_ctx* c, int64_t n, const double* quat, double kT, uint64_t seed, int64_t step,
                            const double* f_ext, double* out)
{
    if (!rods_ok(c, n) || (n > 0 && (!quat || !out)) || !(kT >= 0.0) || step < 0) return ALENS_ERR_INVALID;
    c->launches = 0; c->last_solver = 0;
    CK(launch_brownian(c, (int)n, quat, kT, seed, (unsigned long long)step, f_ext, out));
    CK(cudaStreamSynchronize(c->stream));
    return ALENS_OK;
}

aLENS_status aLENS_random_words(aLENS_ctx* c, int64_t n, uint64_t seed, int64_t step, uint32_t* out)
{
    if (!rods_ok(c, n) || (n > 0 && !out) || step < 0) return ALENS_ERR_INVALID;
    c->launches = 0; c->last_solver = 0;
    CK(launch_random_words(c, (int)n, seed, (unsigned long long)step, out));
    CK(cudaStreamSynchronize(c->stream));
    return ALENS_OK;
}

aLENS_status aLENS_run(aLENS_ctx* c, int64_t n, double* x, double* quat, const double* f_ext, int64_t n_steps,
                       double kT, uint64_t seed, int64_t first_step, int32_t warm_start, aLENS_step_stats* stats,
                       aLENS_info* info)
{
    if (c) { c->launches = 0; c->last_solver = 0; single_mode(c); }
    if (!rods_ok(c, n) || (n > 0 && (!x || !quat)) || n_steps < 0 || !(kT >= 0.0) || first_step < 0)
        return ALENS_ERR_INVALID;
    if (!c->coop_ok) return ALENS_ERR_CUDA;
    const size_t np = (size_t)c->max_rods, mp = (size_t)c->max_pairs;
    if (!c->fnc_buf) {
        bool ok = dmalloc(&c->fnc_buf, 6 * np * sizeof(double)) == cudaSuccess &&
                  dmalloc(&c->gin_buf, mp * sizeof(double)) == cudaSuccess &&
                  dmalloc(&c->row_keys, mp * sizeof(unsigned long long)) == cudaSuccess &&
                  dmalloc(&c->prev_keys, mp * sizeof(unsigned long long)) == cudaSuccess &&
                  dmalloc(&c->prev_gam, mp * sizeof(double)) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            void* bufs[] = {c->fnc_buf, c->gin_buf, c->row_keys, c->prev_keys, c->prev_gam};
            for (void* q : bufs)
                if (q) cudaFree(q);
            c->fnc_buf = nullptr; c->gin_buf = nullptr; c->row_keys = nullptr; c->prev_keys = nullptr;
            c->prev_gam = nullptr;
            return ALENS_ERR_NOMEM;
        }
        c->prev_valid = 0;
    }
    StepOpts opt;
    opt.warm = warm_start != 0;
    opt.keep = true;
    aLENS_info agg;
    memset(&agg, 0, sizeof(agg));
    agg.min_gap = INFINITY;
    int launches = 0;
    aLENS_status st = ALENS_OK;
    for (int64_t k = 0; k < n_steps; ++k) {
        c->launches = 0; c->last_solver = 0;
        CK(launch_brownian(c, (int)n, quat, kT, seed, (unsigned long long)(first_step + k), f_ext, c->fnc_buf));
        aLENS_info si;
        memset(&si, 0, sizeof(si));
        int64_t mw = 0;
        st = step_impl(c, n, x, quat, c->fnc_buf, nullptr, nullptr, nullptr, &si, opt, &mw);
        launches += c->launches;
        if (stats) {
            aLENS_step_stats& o = stats[k];
            o.n_pairs = si.n_pairs;
            o.n_walls = mw;
            o.iters = si.iters;
            o.status = (int32_t)st;
            o.residual = si.residual;
            o.min_gap = si.min_gap;
            o.ms_step = si.ms_build + si.ms_assemble + si.ms_solve + si.ms_update;
        }
        agg.n_pairs = si.n_pairs;
        agg.n_overlap = si.n_overlap;
        agg.iters += si.iters;
        if (si.residual > agg.residual) agg.residual = si.residual;
        if (si.min_gap < agg.min_gap) agg.min_gap = si.min_gap;
        agg.ms_build += si.ms_build;
        agg.ms_assemble += si.ms_assemble;
        agg.ms_solve += si.ms_solve;
        agg.ms_update += si.ms_update;
        if (st != ALENS_OK && st != ALENS_ERR_NOT_CONVERGED) break;
    }
    agg.status = (int32_t)st;
    agg.launches = launches;
    if (info) *info = agg;
    return st;
}

aLENS_status aLENS_step_adjoint(aLENS_ctx* c, int64_t n, const double* x, const double* quat, const double* f_nc,
                                int64_t n_pairs, const int32_t* pairs, const double* gamma, const double* dL_dx_new,
                                const double* dL_dquat_new, double* dL_dx, double* dL_dquat, double* dL_dfnc,
                                double* dL_deta, aLENS_info* info)
{
    if (c) { c->launches = 0; c->last_solver = 0; single_mode(c); }
    if (!rods_ok(c, n) || n_pairs < 0 || n_pairs > c->max_pairs) return ALENS_ERR_INVALID;
    if (n > 0 && (!x || !quat || !dL_dx || !dL_dquat)) return ALENS_ERR_INVALID;
    if (n_pairs > 0 && (!pairs || !gamma)) return ALENS_ERR_INVALID;
    if (c->sp_n > 0 || c->wall_axis >= 0) return ALENS_ERR_NOT_IMPLEMENTED;   // collisions only
    if (cudaGetLastError() != cudaSuccess) return ALENS_ERR_CUDA;
    if (adjoint_reserve(c) != cudaSuccess) { cudaGetLastError(); return ALENS_ERR_NOMEM; }
    aLENS_status st = reset_status(c);
    if (st != ALENS_OK) return st;
    const int m = (int)n_pairs;
    CK(launch_pack(c, (int)n, x, quat, f_nc, false));
    CK(launch_solve_setup_check(c, (int)n, m, pairs));
    if ((st = read_status(c)) != ALENS_OK) return st;
    if (c->hflags[F_ERR] != 0) return (aLENS_status)c->hflags[F_ERR];
    CK(launch_assemble(c, (int)n, m, pairs, c->phi, c->dgeom, c->q64));
    // the adjoint's operator reads the solver's records as D itself: set
    // them up unscaled
    const double beta = c->scale_beta;
    c->scale_beta = 0.0;
    const cudaError_t se = launch_solve_setup(c, (int)n, m, pairs, c->dgeom, c->q64, gamma, quat, c->p.precision, nullptr);
    c->scale_beta = beta;
    CK(se);
    int iters = 0;
    double rel = 0.0;
    CK(launch_adjoint(c, (int)n, m, quat, f_nc, pairs, gamma, dL_dx_new, dL_dquat_new, dL_dx, dL_dquat, dL_dfnc,
                      &iters, &rel, dL_deta));
    if ((st = read_status(c)) != ALENS_OK) return st;
    if (c->hflags[F_SOLVE_ERR] != 0) return (aLENS_status)c->hflags[F_SOLVE_ERR];   // a CG grid wait ran out
    if (c->hflags[F_ERR] != 0) return (aLENS_status)c->hflags[F_ERR];
    const double tol = c->p.precision == ALENS_MIXED ? 1e-7 : 1e-13;
    st = (m > 0 && !(rel <= tol)) ? ALENS_ERR_NOT_CONVERGED : ALENS_OK;
    if (info) {
        memset(info, 0, sizeof(*info));
        info->n_pairs = n_pairs;
        info->iters = iters;
        info->residual = rel;
        info->status = (int32_t)st;
        info->min_gap = INFINITY;
        info->launches = c->launches;
    }
    return st;
}

aLENS_status aLENS_set_batch_launch(aLENS_ctx* c, int32_t threads, int32_t cluster_blocks)
{
    if (!c || threads < 32 || threads > 1024 || threads % 32 != 0) return ALENS_ERR_INVALID;
    if (cluster_blocks != 1 && cluster_blocks != 2 && cluster_blocks != 4 && cluster_blocks != 8)
        return ALENS_ERR_INVALID;
    c->batch_threads = threads;
    c->batch_cluster = cluster_blocks;
    return ALENS_OK;
}

aLENS_status aLENS_batch_results(aLENS_ctx* c, int32_t n_systems, int32_t* iters, double* residual)
{
    if (!c || n_systems < 1 || n_systems != c->last_batch_n) return ALENS_ERR_INVALID;
    if (n_systems == 1) {
        if (iters) iters[0] = c->hflags[F_ITERS];
        if (residual) memcpy(residual, &c->hcount[C_RESID], sizeof(double));
        return ALENS_OK;
    }
    if (iters) CK(cudaMemcpyAsync(iters, c->sys_iters, sizeof(int32_t) * n_systems, cudaMemcpyDeviceToHost, c->stream));
    if (residual)
        CK(cudaMemcpyAsync(residual, c->sys_res, sizeof(double) * n_systems, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return ALENS_OK;
}

aLENS_status aLENS_batch_groups(aLENS_ctx* c, int32_t n_systems, int32_t* blocks)
{
    if (!c || !blocks || n_systems < 1 || n_systems != c->last_batch_n) return ALENS_ERR_INVALID;
    if (n_systems == 1) {
        blocks[0] = 0;
        return ALENS_OK;
    }
    CK(cudaMemcpyAsync(blocks, c->sys_iters + c->max_systems, sizeof(int32_t) * n_systems, cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return ALENS_OK;
}

aLENS_status aLENS_step_batch(aLENS_ctx* c, int32_t n_systems, const aLENS_system* systems, const int64_t* rod_offset,
                              double* x, double* quat, const double* f_nc, int32_t* pairs_out, double* gamma_out,
                              double* vel_out, aLENS_info* info)
{
    if (c) { c->launches = 0; c->last_solver = 0; single_mode(c); }
    if (!c || n_systems < 1 || !systems || !rod_offset) return ALENS_ERR_INVALID;
    const int64_t n = rod_offset[n_systems];
    if (!rods_ok(c, n) || (n > 0 && (!x || !quat))) return ALENS_ERR_INVALID;
    if (!c->coop_ok) return ALENS_ERR_CUDA;
    if (c->wall_axis >= 0) return ALENS_ERR_NOT_IMPLEMENTED;   // walls belong to single systems
    aLENS_status st = batch_tables(c, n_systems, systems, rod_offset);
    if (st != ALENS_OK) { single_mode(c); return st; }
    c->cur_systab = c->systab;
    c->cur_sysid = c->sysid;
    c->last_batch_n = 0;
    st = ALENS_ERR_NOT_IMPLEMENTED;
    // a batch of one runs the single-system solver, which reads its shared-memory need back
    const bool graphable = c->batch_graph && n > 0 && n_systems > 1 && c->sp_n == 0 && c->fault_mode == 0;
    if (graphable) st = step_batch_graph(c, n, x, quat, f_nc, pairs_out, gamma_out, vel_out, info);
    if (st == ALENS_ERR_NOT_IMPLEMENTED) st = step_impl(c, n, x, quat, f_nc, pairs_out, gamma_out, vel_out, info);
    if (st == ALENS_OK || st == ALENS_ERR_NOT_CONVERGED) c->last_batch_n = n_systems;
    single_mode(c);
    return st;
}

const char* aLENS_last_cuda_error(void) { return cudaGetErrorName(g_last_cuda_error); }

aLENS_status aLENS_set_batch_graph(aLENS_ctx* c, int32_t enable)
{
    if (!c || (enable != 0 && enable != 1)) return ALENS_ERR_INVALID;
    if (!enable) drop_graph(c);
    c->batch_graph = enable;
    return ALENS_OK;
}

aLENS_status aLENS_set_step_graph(aLENS_ctx* c, int32_t enable)
{
    if (!c || (enable != 0 && enable != 1)) return ALENS_ERR_INVALID;
    if (!enable) drop_graph(c);
    c->step_graph = enable;
    return ALENS_OK;
}

aLENS_status aLENS_set_l2_window(aLENS_ctx* c, int32_t enable)
{
    if (!c || (enable != 0 && enable != 1)) return ALENS_ERR_INVALID;
    c->l2_window_off = !enable;
    return ALENS_OK;
}

}  // extern "C"
