// Internal declarations of the GB300 collision-constraint library.
// Device helpers shared by the kernels, the context layout, and the host
// launchers that context.cu strings together.  Nothing here is part of the
// C ABI (include/alens.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/alens.h"

namespace alens {

// ---------------------------------------------------------------- constants

constexpr int kSearchWarps = 8;          // warps per block of the neighbour search
constexpr int kPairsPerRodCap = 512;     // per-rod (i < j) list held in shared memory
constexpr double kParallelDet64 = 1e-12; // a c - b^2 below this (relative) = parallel
constexpr float kParallelDet32 = 1e-4f;  // float screen: below this go straight to float64
constexpr int kMaxMortonBits = 7;        // at most 128 cells per edge

// device status words (one int array, see Ctx::dflags)
enum Flag : int {
    F_ERR = 0,        // first error code seen by any kernel (aLENS_status)
    F_ERR_ROD = 1,    // offending rod / pair index for INVALID or per-rod overflow
    F_SOLVE_ERR = 2,  // solver kernel: ALENS_ERR_TIMEOUT when a grid wait ran out, kSolveRedo (below)
    F_FINAL = 3,      // solver kernel: buffer index that holds the final gamma
    F_ITERS = 4,      // solver kernel: iterations taken
    F_NFLAGS = 16
};
// F_SOLVE_ERR of a recorded single-system step whose shares did not fit the
// shared memory it was launched with: nothing moved, the host steps eagerly
constexpr int kSolveRedo = 1 << 20;
// The batched solver's pairs (two clusters on one system): at most kMaxPairs
// per launch, each of at most kPairBlocks blocks (two clusters of 8)
constexpr int kMaxPairs = 16;
constexpr int kPairBlocks = 16;
inline size_t sys_queue_ints(int ns) { return (size_t)ns + 2 * ((size_t)ns + kMaxPairs) + 1 + kMaxPairs; }
// 64-bit counters (Ctx::dcount)
enum Count : int { C_PAIRS = 0, C_OVERLAP = 1, C_MINGAP = 2, C_CAND = 3, C_RESID = 4, C_ALPHA0 = 5, C_SMEM = 6,
                   C_QUEUE = 7, C_WALLS = 8, C_MAXRODS = 9, C_SMEM1 = 10, C_MEFF = 11, C_NCOUNT = 12 };

// Constraint count of a launch: m itself, or, for a step that runs without
// host readbacks (a captured graph: grids sized for the capacity m), the
// count the device holds in *mdev, at most m.
__device__ __forceinline__ int count_of(int m, const unsigned long long* mdev)
{
    if (!mdev) return m;
    const unsigned long long v = *mdev;
    return v < (unsigned long long)m ? (int)v : m;
}

// ------------------------------------------------------------ plain structs

struct Geo {                 // everything the geometry kernels need
    double box[3];
    double cs[3];            // cell edge per axis (>= L + D + delta_c)
    double inv_cs[3];        // 1 / cs (cell_index's first guess)
    int nc[3];               // cells per axis
    int bits;                // Morton bits per axis
    double diameter, length, half, delta_c, dt;
    double rcut;             // L + D + delta_c: centre-distance bound for a close pair
    float boxf[3];
    float rcut_screen2;      // (rcut + margin)^2 for the float pre-screen
    float screen_d2;         // (D + delta_c + margin)^2 for the float segment screen
    float keep_d2;           // (D + delta_c - keep margin)^2: below it the float distance keeps the pair
    float half_f;            // L/2 in float
};

// Default exponent of the solver's diagonal scaling sigma_c = A_cc^(-beta/2).
constexpr double kDefaultScaleBeta = 0.5;

struct Mob {                 // inverse drag coefficients of one rod (all rods alike)
    double inv_perp, inv_par, inv_rot, inv_spin;
};

struct SysGeo {              // one system of a batch: its geometry, drags and cell keys
    Geo g;
    Mob mob;
    int key_base;            // first cell key of the system in the batch's key space
    int pad;
};

// Geometry of rod i: its system's entry when a batch table is given.
__device__ __forceinline__ const Geo& geo_of(const Geo& g, const SysGeo* systab, const int* sys, int i)
{
    return systab ? systab[sys[i]].g : g;
}

// ------------------------------------------------------------- device helpers

__host__ __device__ inline uint32_t spread_bits3(uint32_t v)
{
    // insert two zero bits between each of the low 10 bits
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__host__ __device__ inline uint32_t morton3(int cx, int cy, int cz)
{
    return spread_bits3((uint32_t)cx) | (spread_bits3((uint32_t)cy) << 1) | (spread_bits3((uint32_t)cz) << 2);
}

// Wrap one coordinate into [0, b).
__device__ __forceinline__ double wrap_coord(double v, double b)
{
    // v - b floor(v / b).  For v in [-b, 2b) the floor of the rounded
    // quotient is -1, 0 or 1 on the same sides of -b, 0, b and 2b as v: the
    // double just below b (2b) divided by b rounds to a double below 1 (2),
    // since b's unit in the last place is at least 2^-53 b.  Those cases
    // need no division and give the same bits (v - b is exact on [b, 2b]).
    double w;
    if (v >= 0.0 && v < b) w = __dadd_rn(v, 0.0);   // + 0.0: -0 becomes +0, as v - b * 0 does
    else if (v < 0.0 && v >= -b) w = __dadd_rn(v, b);
    else if (v >= b && v < 2.0 * b) w = __dsub_rn(v, b);
    else w = __dsub_rn(v, __dmul_rn(b, floor(__ddiv_rn(v, b))));
    if (!(w < b) || w < 0.0) w = 0.0;
    return w;
}

// (int)(w / cs) for a wrapped coordinate w >= 0: the product with 1 / cs is
// within about 1e-12 of the rounded quotient (fewer than 2^10 cells), so its
// floor is the quotient's unless it lies within 1e-9 of an integer, where
// the division decides.
__device__ __forceinline__ int cell_index(double w, double cs, double inv_cs)
{
    const double q = __dmul_rn(w, inv_cs), f = floor(q), r = q - f;
    if (r > 1e-9 && r < 1.0 - 1e-9) return (int)f;
    return (int)__ddiv_rn(w, cs);
}

// Rod axis R(theta) e_z of a quaternion (s, a, b, c).
__device__ __forceinline__ void quat_axis(double s, double a, double b, double c, double& p0, double& p1,
                                          double& p2)
{
    p0 = 2.0 * (a * c + s * b);
    p1 = 2.0 * (b * c - s * a);
    p2 = s * s - a * a - b * b + c * c;
}

template <typename T>
__device__ __forceinline__ T clampv(T v, T lo, T hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

// a b + c rounded once (FUSED) or twice.  The float64 keep/drop decision
// rounds twice, like the oracle it must match bit for bit; the assembly of
// Phi, D and q, which matches within tolerances, fuses.
template <bool FUSED, typename T>
__device__ __forceinline__ T madd(T a, T b, T c)
{
    if constexpr (FUSED) return fma(a, b, c);
    else return a * b + c;
}

template <bool FUSED, typename T>
__device__ __forceinline__ T dot3(const T u[3], const T v[3])
{
    if constexpr (FUSED) return fma(u[2], v[2], fma(u[1], v[1], u[0] * v[0]));
    else return u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
}

// Closest points of two segments {x_P + s p} and {x_Q + t q}, |s|,|t| <= hl,
// given dx = x_P - x_Q.  Clamped-projection method: take the unconstrained
// optimum s of the two infinite lines, clamp it, project onto Q for t; if
// that t leaves Q, clamp t and re-project onto P.  Parallel segments
// (det <= eps a c) whose projections overlap take s at the middle of the
// overlap and t as its clamped projection.  Leaves r = dx + s p - t q and
// returns |r|.
template <typename T, bool FUSED = false>
__device__ __forceinline__ T segment_closest(const T dx[3], const T p[3], const T q[3], T hl, T det_eps, T& s_out,
                                             T& t_out, T r_out[3] = nullptr)
{
    const T a = dot3<FUSED>(p, p), b = dot3<FUSED>(p, q), c = dot3<FUSED>(q, q);
    const T d = dot3<FUSED>(p, dx), e = dot3<FUSED>(q, dx);
    const T det = madd<FUSED>(a, c, -(b * b));
    T s, t;
    bool done = false;
    if (det > det_eps * a * c) {
        s = clampv(madd<FUSED>(b, e, -(c * d)) / det, -hl, hl);
    } else {
        // projections of Q's ends onto P's axis
        T e1 = (-b * hl - d) / a, e2 = (b * hl - d) / a;
        T lo = e1 < e2 ? e1 : e2, hi = e1 < e2 ? e2 : e1;
        T olo = lo < -hl ? -hl : lo, ohi = hi > hl ? hl : hi;
        if (olo <= ohi) {
            s = T(0.5) * (olo + ohi);
            t = clampv(madd<FUSED>(b, s, e) / c, -hl, hl);
            done = true;
        } else {
            s = hi < -hl ? -hl : hl;   // P's end nearest to Q's projection
        }
    }
    if (!done) {
        t = madd<FUSED>(b, s, e) / c;
        if (t < -hl) {
            t = -hl;
            s = clampv(madd<FUSED>(b, t, -d) / a, -hl, hl);
        } else if (t > hl) {
            t = hl;
            s = clampv(madd<FUSED>(b, t, -d) / a, -hl, hl);
        }
    }
    T r[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if constexpr (FUSED) r[k] = fma(-t, q[k], fma(s, p[k], dx[k]));
        else r[k] = dx[k] + s * p[k] - t * q[k];
    }
    s_out = s;
    t_out = t;
    if (r_out) {
#pragma unroll
        for (int k = 0; k < 3; ++k) r_out[k] = r[k];
    }
    return sqrt(dot3<FUSED>(r, r));
}

// ------------------------------------------------------------ scoped atomics

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int* p)
{
    return *(const volatile int*)p;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded grid barrier on a monotone arrival counter: block b's k-th arrival
// waits until the counter reaches k * gridDim.x.  Arrival is a release
// reduction and the wait an acquire poll by thread 0, whose verdict the
// block reads from shared memory.  The wait gives up after wait_cycles clock
// cycles or 2^28 polls, records ALENS_ERR_TIMEOUT and returns false; it also
// returns false as soon as any block has recorded an error, so every block
// leaves.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned target, int* flags, long long wait_cycles,
                                             int* s_ok)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        red_release_add(count, 1u);
        long long t0 = clock64();
        int ok = 1;
        for (unsigned polls = 0;; ++polls) {
            unsigned v = ld_acquire_u32(count);
            if ((int)(v - target) >= 0) break;
            if (ld_volatile_i32(&flags[F_SOLVE_ERR]) != 0) { ok = 0; break; }
            if (clock64() - t0 > wait_cycles || polls > (1u << 28)) {
                atomicCAS(&flags[F_SOLVE_ERR], 0, ALENS_ERR_TIMEOUT);
                ok = 0;
                break;
            }
        }
        if (ok && ld_volatile_i32(&flags[F_SOLVE_ERR]) != 0) ok = 0;
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// ------------------------------------------------------------- context

template <typename T>
struct SolveBufs {           // typed views into the solver workspace
    T* rec;                  // [9][mp]  e, y_P x e, y_Q x e
    T* qe;                   // [mp][8]  per Q-side entry: e, y_Q x e, 2 pad (CSR order)
    T* pe;                   // [mp][8]  per constraint: e, y_P x e, 2 pad (owner order; null: read rec)
    T* q;                    // [mp]
    T* ax;                   // [3][np]
    T* gg[2];                // [mp][4] x 2: (delta, g, gamma_ref, 0), ping-pong
    T* U;                    // [np][6] velocity increment M D delta
    T* U2;                   // [np][6] second increment buffer (the one-barrier solver alternates U, U2)
    T* Uref;                 // [np][6] reference velocity M D gamma_ref
    T* gref;                 // [mp] reference gradient q + D^T Uref
    T* mobr;                 // [4][np] per-rod inverse drags (batches)
    // float32 only: low parts of the float64 inputs (x = hi + lo to about
    // 48 bits), read by the reference passes
    T* rec_lo;               // [9][mp]
    T* qe_lo;                // [mp][8]
    T* q_lo;                 // [mp]
    T* lop;                  // [mp][8] rec_lo of the owner side (e, y_P x e, 2 pad) as one row
    T* loq;                  // [mp][8] rec_lo of the other side (e, y_Q x e, 2 pad) (null: read rec_lo)
    T* comp;                 // [mp] < 0 collision, >= 0 spring compliance 1/(h kappa) (solver order)
    T* isc;                  // [mp] 1 / sigma_c: the constraint's scaling undone (solver order)
};

}  // namespace alens

struct aLENS_ctx {
    aLENS_params p;
    int64_t max_rods, max_pairs;
    cudaStream_t stream;
    int device, num_sms;
    double clock_khz;
    alens::Geo geo;
    alens::Mob mob;
    int max_keys;            // histogram size allocated (power of 8)

    // rod workspaces, pitch max_rods
    double* xw;              // [3][np] wrapped centres
    double* axis;            // [3][np]
    double* unc;             // [6][np] M F_nc
    float4* pos32;           // [np]
    float4* ax32;            // [np]
    uint32_t* cellkey;       // [np]
    int* sorted_id;          // [np]
    float4* spos32;          // [np] cell-sorted copies
    float4* sax32;           // [np]
    int* cell_count;         // [max_keys + 1]
    int* cell_start;         // [max_keys + 1]
    int* cell_cursor;        // [max_keys]
    int* rod_count;          // [np + 1] kept pairs per rod (i < j side)
    int* rod_ncand;          // [np] screened candidates per rod
    long long* rod_tmpstart; // [np] start of the rod's candidate segment
    unsigned long long* cand;// [cand_cap] candidate keys (i << 32 | undecided << 31 | j << 5 | image)
    long long cand_cap;
    int* rowP;               // [np + 1]
    int* rowQ;               // [np + 1]
    int* cntQ;               // [np + 1]
    int* curQ;               // [np]
    int* qlist;              // [mp] Q-side CSR: internal constraint ids per rod rank
    int* perm;               // [mp] internal (owner-major) constraint -> caller constraint
    int* rank;               // [np] solver position of each rod (cell-sorted order)
    int* curP;               // [np + 1]
    int* ci;                 // [mp]
    int* cj;                 // [mp]
    int32_t* pairs;          // [mp][3] internal pair list of a step
    double* phi;             // [mp]
    double* dgeom;           // [mp][9]
    double* q64;             // [mp]
    double* scale64;         // [mp] sigma_c of the solver's diagonal scaling (solver order)
    double scale_beta;       // sigma_c = A_cc^(-beta/2); 0: the unscaled iteration
    void* solve_ws;          // typed solver buffers (sized for double)
    alens::SolveBufs<double> sb64;
    alens::SolveBufs<float> sb32;
    double* partials;        // [max_blocks + 4][8]: [4][nb] block sums, or [2][4][nb] (one-barrier solver)
    int max_blocks;
    int* bstart;             // [max_blocks + 1] solver block boundaries (rod ranks)
    unsigned* bar;           // [4]
    int* dflags;             // [F_NFLAGS]
    unsigned long long* dcount;  // [C_NCOUNT]
    int* scan_tmp;           // block sums for the scans
    int scan_tmp_len;

    // host side
    int* hflags;             // pinned mirror of dflags
    unsigned long long* hcount;
    cudaEvent_t ev[8];
    double wait_s;
    int fault_mode;
    int solve_threads, solve_bps;
    int solve_barriers;      // 1: one-barrier solver where its share fits (default); 2: the two-barrier kernels
    int smem_optin;          // the device's opt-in shared memory per block (bytes)
    int l2_bytes;            // the device's L2 size, its largest access-policy window and
    int l2_window_max;       // its largest persisting set-aside (bytes)
    int l2_persist_max;
    size_t persist_prev;     // the context's persisting set-aside before this context raised it
    size_t persist_set;      // the set-aside this context set (0: untouched)
    int l2_window_off;       // aLENS_set_l2_window(ctx, 0)
    int attr1_set[2];        // the one-barrier kernel's dynamic shared-memory limit is set (float, double)
    int occ1_key[2];         // launch shape (threads * 64 + blocks per SM) whose occupancy was checked ...
    int occ1_ok[2];          // ... and whether that many blocks per SM fit at the full budget
    int last_solver;         // kernel of the last single-system solve: 1 one-barrier, 2 two-barrier staged, 3 two-barrier global
    int zero_start;          // the last setup started from gamma = 0 (no caller gamma)
    int qe_pending;          // the last setup's CSR-ordered other-side copies (qe) are still to be written
    int qe_m, qe_prec;       // ... for this many constraints in this precision
    // batched steps as a captured CUDA graph (aLENS_set_batch_graph)
    const unsigned long long* mdev;   // while recording a graph: the device's constraint count (else NULL)
    int batch_graph;         // graph mode on (batched steps)
    int step_graph;          // graph mode on (single-system steps, aLENS_set_step_graph)
    cudaGraph_t graph;
    cudaGraphExec_t gexec;
    cudaStream_t cap_stream; // the graph is recorded here (the legacy default stream cannot be captured)
    cudaStream_t side;       // the solver layout's kernels, beside the assembly (non-blocking)
    cudaEvent_t ev_fork, ev_join;  // side waits for ev_fork; the step's stream for ev_join
    int graph_launches;      // kernels in the graph
    int graph_state;         // 0 nothing, 1 the key below ran eagerly once, 2 a graph of it is instantiated,
                             // 3 the key stays eager (its solver reads back, or a recorded step redid)
    struct GraphKey {
        int64_t n;
        const void* ptr[6];  // x, quat, f_nc, pairs_out, gamma_out, vel_out
        aLENS_params p;
        double beta;
        int threads, cluster, tables;
        int kind, barriers;  // 1 batched step, 2 single-system step; the solver schedule
    } gkey;
    int tables_epoch;        // bumped whenever the batch tables change
    int coop_ok;
    int batch_coop;          // cooperative launch with clusters: -1 untried, 0 refused, 1 works
    int launches;            // kernels launched since the entry point began
    // batches (aLENS_step_batch): per-system table and per-rod system id;
    // NULL outside a batched step
    alens::SysGeo* systab;   // [max_systems] device
    int* sysid;              // [np] device
    long long* sysoff;       // [max_systems + 1] device rod offsets
    int max_systems;
    const alens::SysGeo* cur_systab;   // set for the duration of a batched step
    const int* cur_sysid;
    int cur_nkeys;           // cell keys of the step (batch: all systems)
    int batch_n;             // systems described by the tables now on the device
    int batch_keys;          // their cell keys
    void* batch_host;        // host copy of the last aLENS_system array (to skip re-uploads)
    int64_t* batch_off_host; // host copy of the last rod offsets
    int* sys_order;          // [max_systems] queue order of the per-system solver, then the
                             // queue entries [2 (max_systems + kMaxPairs)], their count and
                             // the pairs' barrier counters [kMaxPairs] (sys_queue_ints ints)
    int* sys_iters;          // [2][max_systems] iterations of each system's solve, then the blocks that solved it
    double* sys_res;         // [max_systems] final residual of each system
    int last_batch_n;        // systems of the last completed aLENS_step_batch (0: none)
    void* adj_ws;            // adjoint workspace (allocated by the first aLENS_step_adjoint)
    // springs (aLENS_set_springs): bilateral constraints appended to every step's collisions
    int32_t* sp_ends;        // [sp_cap][2] rods P, Q
    double* sp_arms;         // [sp_cap][2] attachment arclengths on P and Q
    double* sp_kappa;        // [sp_cap]
    double* sp_rest;         // [sp_cap]
    int64_t sp_n, sp_cap;
    double* comp64;          // [mp] pair order: -1 collisions, 1/(h kappa) springs (allocated with the springs)
    const double* cur_comp;  // comp64 while a step with springs is set up and solved, else NULL
    int64_t sp_version;      // bumped by every aLENS_set_springs (warm start matches springs by index)
    // walls (aLENS_set_walls): axis (-1: none) and the two wall coordinates
    int wall_axis;
    double wall_lo, wall_hi;
    // trajectories (aLENS_run): forces of a step, warm start from the previous step
    double* fnc_buf;         // [np][6]
    double* gin_buf;         // [mp]
    unsigned long long* row_keys;   // [mp] keys of this step's rows
    unsigned long long* prev_keys;  // [mp] keys of the previous step's rows
    double* prev_gam;        // [mp] the previous step's forces
    int64_t prev_mu, prev_mw, prev_ms, prev_sp_version;
    int prev_valid;
    int batch_threads;       // per-system solver: threads per block
    int batch_cluster;       // per-system solver: blocks per cluster
};

namespace alens {

// scan.cu: exclusive scan of counts[0..n) into out[0..n], out[n] = total.
cudaError_t exclusive_scan(aLENS_ctx* ctx, const int* counts, int* out, int n);

// neighbors.cu
cudaError_t launch_pack(aLENS_ctx* ctx, int n, const double* x, const double* quat, const double* fnc, bool cells);
cudaError_t launch_cell_sort(aLENS_ctx* ctx, int n);
// Screens candidates (float32) into the candidate buffer and decides them
// (float64); per-rod kept counts in rod_count, totals in dcount.
cudaError_t launch_search(aLENS_ctx* ctx, int n);
// Exact pair count only (float64 inline), for a candidate-buffer overflow.
cudaError_t launch_search_count(aLENS_ctx* ctx, int n);
cudaError_t launch_emit_pairs(aLENS_ctx* ctx, int n, int32_t* pairs_out);
cudaError_t launch_check_capacity(aLENS_ctx* ctx);
cudaError_t launch_copy_pairs(aLENS_ctx* ctx, int32_t* pairs_out);

// assemble.cu
cudaError_t launch_assemble(aLENS_ctx* ctx, int n, int m, const int32_t* pairs, double* phi, double* dgeom,
                            double* q);
// Validates a caller's pair list (ranges, i < j, sorted by i) and counts
// the P and Q sides; launch_solve_setup must follow only if no error flag was raised.
cudaError_t launch_solve_setup_check(aLENS_ctx* ctx, int n, int m, const int32_t* pairs);
// rank (nullable): solver position of each rod (identity when NULL).
// launch_solve_setup = launch_solve_layout (from the pair list alone) then
// launch_solve_fill (from the assembled values); a step may run the layout
// beside the assembly.
cudaError_t launch_solve_layout(aLENS_ctx* ctx, int n, int m, const int32_t* pairs, const double* quat,
                                int precision, const int* rank);
cudaError_t launch_solve_fill(aLENS_ctx* ctx, int n, int m, const int32_t* pairs, const double* dgeom,
                              const double* q, const double* gamma_in, int precision, const int* rank);
cudaError_t launch_solve_setup(aLENS_ctx* ctx, int n, int m, const int32_t* pairs, const double* dgeom,
                               const double* q, const double* gamma_in, const double* quat, int precision,
                               const int* rank);
// rank[sorted_id[k]] = k: the cell-sorted position of every rod.
cudaError_t launch_rank(aLENS_ctx* ctx, int n);

// solve.cu
cudaError_t launch_solve(aLENS_ctx* ctx, int n, int m, int precision);
// The other-side copies qe of the last setup, if still pending: the
// global-memory solvers and the adjoint read them, the one-barrier solver
// does not.
cudaError_t launch_setup_qe(aLENS_ctx* ctx);
// The single-system solve of a step recorded as a graph (no readback; the
// kernel checks on the device that its shares fit and otherwise flags
// kSolveRedo), and whether the context's launch shape allows it.
cudaError_t launch_solve_graph1(aLENS_ctx* ctx, int n, int m, int precision);
cudaError_t graph1_possible(aLENS_ctx* ctx, int precision, bool& ok);
cudaError_t launch_gamma_out(aLENS_ctx* ctx, int m, int precision, double* gamma_out);

// Springs: rows mu .. mu + nb of the internal constraint list (pairs, phi,
// dgeom, q) and comp64 for every row (collisions -1).
cudaError_t launch_assemble_springs(aLENS_ctx* ctx, int n, int mu);

// trajectory.cu: walls (count during the search, rows after the
// collisions), Brownian forces, raw generator words, warm start.
cudaError_t launch_count_walls(aLENS_ctx* ctx, int n);
cudaError_t launch_emit_walls(aLENS_ctx* ctx, int n, int row0);
cudaError_t launch_brownian(aLENS_ctx* ctx, int n, const double* quat, double kT, unsigned long long seed,
                            unsigned long long step, const double* fext, double* out);
cudaError_t launch_random_words(aLENS_ctx* ctx, int n, unsigned long long seed, unsigned long long step,
                                uint32_t* out);
cudaError_t launch_warm(aLENS_ctx* ctx, int m, int mu, int mw, double* gin);
cudaError_t launch_keep_keys(aLENS_ctx* ctx, int m, int mu, int mw);

// adjoint.cu: workspace (once) and the adjoint pipeline after pack, assembly
// and the solver setup of the forward step's pair list (identity ranks).
cudaError_t adjoint_reserve(aLENS_ctx* ctx);
cudaError_t launch_adjoint(aLENS_ctx* ctx, int n, int m, const double* quat, const double* fnc,
                           const int32_t* pairs, const double* gamma, const double* gxn, const double* gqn,
                           double* out_x, double* out_q, double* out_f, int* cg_iters, double* cg_rel,
                           double* deta);

// update.cu
cudaError_t launch_update(aLENS_ctx* ctx, int n, int m, double* x, double* quat, int precision, double* vel_out,
                          const int* rank);

}  // namespace alens
