// Adjoint of one constrained step: the gradient of a scalar loss L(x', theta')
// with respect to the step's inputs (centres, orientations, viscosity and
// non-constraint forces), on the pair list and active set of the forward
// step (Appendix Eq. constrainedeom_euler a-c with the constraint problem of
// Eq. suppcqpdef; KKT on the active set A = {c : gamma_c > 0}:
// (A gamma + q)_A = 0, gamma elsewhere 0).
//
//   u      = dL/dU through the update (x' = x + h U_t, theta' = normalise(
//            theta + h Psi(theta) Omega));
//   b      = D^T M u,  A_AA lambda_A = b_A  (conjugate gradients with the
//            solver's own D, M, D^T records; b_A lies in the range of A_AA,
//            so CG from 0 reaches the minimum-norm multiplier when A_AA is
//            singular);
//   w      = D lambda,  nu = M (u - w);
//   dL     = direct update terms + (u - w)^T dM F_tot + nu^T (dD gamma)
//            - (dD lambda)^T U - lambda^T dPhi / h,
// with F_tot = F_nc + D gamma and U = M F_tot.  dPhi = e.(dDx + s dp_P - t dq)
// (the closest-point parameters are stationary or clamped); the derivative of
// the D column follows s*, t* through their branch: both free (2x2
// stationarity system), one clamped (1-D condition), or both clamped.
// Parallel segments (the midpoint reading) hold s*, t* fixed.  The mobility
// terms use dM_t/dp = (1/zeta_par - 1/zeta_perp) d(p p^T) (rotation alike)
// and dM/d eta = -M / eta.  Orientation gradients are projected onto the
// unit quaternion's tangent space.
//
// Everything runs in float64 except the CG operator, which uses the
// solver's records in its working precision (float32 in mixed mode).  The
// CG loop is one persistent cooperative kernel, one block per SM: per
// iteration a rod pass (F = D_A p, Up = M F), a grid barrier, a constraint
// pass (Ap and p.Ap), a grid-wide sum, the update, and a second grid-wide
// sum; every block sums the per-block partials in block order, so all take
// the same step lengths and the result is deterministic.  The setup and
// the passes before and after the loop are ordinary kernels whose scalar
// reductions finish in the last block to arrive.
#include <float.h>

#include "internal.cuh"

namespace alens {

namespace {

__device__ __forceinline__ void cross(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ double dot(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// U = M(p) F for one rod (M_t = I/zp + (1/zpar - 1/zp) p p^T, rotation alike).
__device__ __forceinline__ void mob_apply(const Mob& mb, const double p[3], const double F[6], double U[6])
{
    const double pf = dot(p, F), pt = p[0] * F[3] + p[1] * F[4] + p[2] * F[5];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        U[k] = F[k] * mb.inv_perp + p[k] * pf * (mb.inv_par - mb.inv_perp);
        U[3 + k] = F[3 + k] * mb.inv_rot + p[k] * pt * (mb.inv_spin - mb.inv_rot);
    }
}

// Sum of v over the block (every thread passes its value); thread 0 gets it.
__device__ __forceinline__ double block_sum(double v, double* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (warp == 0) {
        s = lane < nw ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    __syncthreads();
    return s;
}

// Block partial into partials[blockIdx.x]; the last block to arrive sums
// the partials in block order and returns true (with the total in *tot,
// valid in thread 0 of that block).
__device__ __forceinline__ bool last_block_total(double part, double* partials, unsigned* counter, double* tot)
{
    __shared__ double red[32];
    __shared__ int last;
    const double s = block_sum(part, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s;
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        last = t == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    if (threadIdx.x < 32) {
        // warp 0: lane l sums partials l, l + 32, ... (loads in flight
        // together), then a fixed shuffle tree
        __threadfence();
        double acc = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += 32) acc += __ldcg(&partials[b]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) {
            *tot = acc;
            *counter = 0u;   // ready for the next reduction
        }
    }
    return true;
}

enum { S_RR = 0, S_RR0, S_ALPHA, S_BETA, S_ETA, S_TOL2, S_NSCAL = 8 };
enum { I_DONE = 0, I_ITERS, I_MAXIT, I_NI = 4 };

}  // namespace

// Rod pass 1: F_tot = F_nc + D gamma, U = M F_tot; the update's adjoint
// (u = dL/dU, direct dL/dx and dL/dtheta); Mu = M u.
__global__ void k_adj_rods1(int n, int np, Mob mob, double h, const double* __restrict__ axis,
                            const double* __restrict__ quat, const double* __restrict__ fnc,
                            const double* __restrict__ gamma, const double* __restrict__ dgeom,
                            const int* __restrict__ rowP, const int* __restrict__ rowQ,
                            const int* __restrict__ qlist, const double* __restrict__ gxn,
                            const double* __restrict__ gqn, double* __restrict__ Ftot, double* __restrict__ U,
                            double* __restrict__ u, double* __restrict__ Mu, double* __restrict__ gx,
                            double* __restrict__ gq)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double F[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) F[k] = fnc ? fnc[6 * (size_t)i + k] : 0.0;
    for (int c = rowP[i]; c < rowP[i + 1]; ++c) {
        const double g = gamma[c];
        const double* d = dgeom + 9 * (size_t)c;
#pragma unroll
        for (int k = 0; k < 6; ++k) F[k] += g * d[k];
    }
    for (int k = rowQ[i]; k < rowQ[i + 1]; ++k) {
        const int c = qlist[k];
        const double g = gamma[c];
        const double* d = dgeom + 9 * (size_t)c;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            F[a] -= g * d[a];
            F[3 + a] -= g * d[6 + a];
        }
    }
    const double p[3] = {axis[i], axis[np + i], axis[2 * (size_t)np + i]};
    double Ui[6];
    mob_apply(mob, p, F, Ui);
    double ui[6] = {0, 0, 0, 0, 0, 0}, gxi[3] = {0, 0, 0}, gqi[4] = {0, 0, 0, 0};
    if (gxn) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gxi[a] = gxn[3 * (size_t)i + a];   // x' = x + h U_t
            ui[a] = h * gxi[a];
        }
    }
    if (gqn) {
        // theta' = phi/|phi|, phi = (s - h/2 v.Om, v + h/2 (s Om - v x Om))
        const double s = quat[4 * (size_t)i];
        const double v[3] = {quat[4 * (size_t)i + 1], quat[4 * (size_t)i + 2], quat[4 * (size_t)i + 3]};
        const double om[3] = {Ui[3], Ui[4], Ui[5]};
        double vxo[3];
        cross(v, om, vxo);
        double ph[4] = {s - 0.5 * h * dot(v, om), 0, 0, 0};
#pragma unroll
        for (int a = 0; a < 3; ++a) ph[1 + a] = v[a] + 0.5 * h * (s * om[a] - vxo[a]);
        const double nrm = sqrt(ph[0] * ph[0] + ph[1] * ph[1] + ph[2] * ph[2] + ph[3] * ph[3]);
        double qn[4], gin[4], proj = 0.0;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            qn[a] = ph[a] / nrm;
            gin[a] = gqn[4 * (size_t)i + a];
            proj += qn[a] * gin[a];
        }
        double g[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) g[a] = (gin[a] - qn[a] * proj) / nrm;   // dL/dphi
        const double gv[3] = {g[1], g[2], g[3]};
        double oxg[3], gxv[3];
        cross(om, gv, oxg);
        cross(gv, v, gxv);
        gqi[0] = g[0] + 0.5 * h * dot(gv, om);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gqi[1 + a] = gv[a] + 0.5 * h * (-g[0] * om[a] - oxg[a]);
            ui[3 + a] = 0.5 * h * (-g[0] * v[a] + s * gv[a] - gxv[a]);
        }
    }
    double Mui[6];
    mob_apply(mob, p, ui, Mui);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        Ftot[6 * (size_t)i + k] = F[k];
        U[6 * (size_t)i + k] = Ui[k];
        u[6 * (size_t)i + k] = ui[k];
        Mu[6 * (size_t)i + k] = Mui[k];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) gx[3 * (size_t)i + a] = gxi[a];
#pragma unroll
    for (int a = 0; a < 4; ++a) gq[4 * (size_t)i + a] = gqi[a];
}

// b = D^T M u on the active set; CG start lambda = 0, r = b_A, p = 0, Ap = 0,
// alpha = beta = 0.  The CG state of constraint c is one 32-byte record
// cgs[c] = (r, p, Ap, lambda), so that a gather by constraint id touches one
// sector.
__global__ void k_adj_b(int m, const int32_t* __restrict__ pairs, const double* __restrict__ dgeom,
                        const double* __restrict__ gamma, const double* __restrict__ Mu, double* __restrict__ lam,
                        double* __restrict__ cgs, double* __restrict__ partials, unsigned* counter, double* scal,
                        int* iflag, double tol)
{
    double acc = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        const int i = pairs[3 * (size_t)c], j = pairs[3 * (size_t)c + 1];
        const double* d = dgeom + 9 * (size_t)c;
        double b = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            b += d[a] * (Mu[6 * (size_t)i + a] - Mu[6 * (size_t)j + a]) + d[3 + a] * Mu[6 * (size_t)i + 3 + a] -
                 d[6 + a] * Mu[6 * (size_t)j + 3 + a];
        const double rc = gamma[c] > 0.0 ? b : 0.0;
        double2* st = reinterpret_cast<double2*>(cgs) + 2 * (size_t)c;
        st[0] = make_double2(rc, 0.0);    // r, p
        st[1] = make_double2(0.0, 0.0);   // Ap, lambda
        lam[c] = 0.0;
        acc += rc * rc;
    }
    double tot;
    if (last_block_total(acc, partials, counter, &tot) && threadIdx.x == 0) {
        scal[S_RR] = tot;
        scal[S_RR0] = tot;
        scal[S_BETA] = 0.0;
        scal[S_TOL2] = tol * tol * tot;
        iflag[I_ITERS] = 0;
        iflag[I_DONE] = !(tot > 0.0) ? 1 : 0;
    }
}

// Active-set lists of the CG: per rod, the counts of its active owned
// constraints and active other-side entries, then (after the scans) the
// lists themselves in CSR order.
__global__ void k_act_count(int n, const int* __restrict__ rowP, const int* __restrict__ rowQ,
                            const int* __restrict__ qlist, const double* __restrict__ gamma, int* __restrict__ cA,
                            int* __restrict__ cB)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int na = 0, nb = 0;
    for (int c = rowP[i]; c < rowP[i + 1]; ++c) na += gamma[c] > 0.0;
    for (int k = rowQ[i]; k < rowQ[i + 1]; ++k) nb += gamma[qlist[k]] > 0.0;
    cA[i] = na;
    cB[i] = nb;
}

__global__ void k_act_fill(int n, const int* __restrict__ rowP, const int* __restrict__ rowQ,
                           const int* __restrict__ qlist, const double* __restrict__ gamma,
                           const int* __restrict__ aP, const int* __restrict__ aQ, int* __restrict__ alist,
                           int* __restrict__ bk, int* __restrict__ bc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int t = aP[i];
    for (int c = rowP[i]; c < rowP[i + 1]; ++c)
        if (gamma[c] > 0.0) alist[t++] = c;
    t = aQ[i];
    for (int k = rowQ[i]; k < rowQ[i + 1]; ++k) {
        const int c = qlist[k];
        if (gamma[c] > 0.0) {
            bk[t] = k;
            bc[t] = c;
            ++t;
        }
    }
}

// Arguments of the persistent CG.
template <typename T>
struct CgArgs {
    int n, m, np, mp;
    const int* __restrict__ rowP;
    const int* __restrict__ rowQ;
    const int* __restrict__ qlist;
    const int* __restrict__ ci;
    const int* __restrict__ cj;
    const T* __restrict__ rec;
    const T* __restrict__ qe;
    const T* __restrict__ ax;
    T inv_perp, inv_par, inv_rot, inv_spin;
    // the active set {c : gamma_c > 0}: per rod, its active owned constraints
    // alist[aP[i] .. aP[i+1]) and active other-side entries (arm record bk,
    // constraint bc) [aQ[i] .. aQ[i+1]); alist[0 .. aP[n]) lists every active
    // constraint
    const int* __restrict__ aP;
    const int* __restrict__ aQ;
    const int* __restrict__ alist;
    const int* __restrict__ bk;
    const int* __restrict__ bc;
    const T* __restrict__ pe;   // [m][8] owned-side arms per constraint (e, y_P x e, 2 pad)
    double* cgs;         // [m][4] (r, p, Ap, lambda) per constraint
    double* lam;         // [m] lambda, copied out of cgs when the CG ends
    T* Up;               // [n][6] rod velocities of the direction
    double* partials;    // [2][gridDim.x]: the two sums of an iteration
    unsigned* bar;       // monotone grid-barrier counter
    int* flags;          // device status: ALENS_ERR_TIMEOUT when a wait runs out
    double* scal;
    int* iflag;
    long long wait_cycles;
    int fault;           // test hook (aLENS_inject_fault): 1 = block 0 leaves before its first arrival
};

// Float64 arithmetic is scarce on this part (a warp-wide add occupies the
// SM's float64 pipe for many cycles), so the CG's sums avoid shuffle trees
// over every warp.  Block sums of v[0..3]: every thread puts its values in
// vals[u][thread]; warp w adds, for value u = w % 4, the rows (32 threads
// each) w / 4, w / 4 + G, ... (G = warps / 4 groups) of the first `rows`
// rows lane by lane into its own row; warp u < 4 then adds the G group rows
// lane by lane and finishes with a shuffle tree.  Only the first `rows` rows
// can hold non-zero values (threads that had no constraint add nothing).
// Lane 0 of warp u stores the block sum of value u in part[u * gridDim.x +
// blockIdx.x].  Needs blockDim.x a multiple of 128.
__device__ __forceinline__ void block_sums4(const double v[4], double (*vals)[1024], int rows, double* part)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, groups = (int)(blockDim.x >> 7);
#pragma unroll
    for (int u = 0; u < 4; ++u) vals[u][threadIdx.x] = v[u];
    __syncthreads();
    {
        const int u = warp & 3, g = warp >> 2;
        if (g < rows) {
            double s = vals[u][g * 32 + lane];
            for (int k = g + groups; k < rows; k += groups) s += vals[u][k * 32 + lane];
            vals[u][g * 32 + lane] = s;   // row g is read by this warp alone
        }
    }
    __syncthreads();
    if (warp < 4) {
        const int gmax = rows < groups ? rows : groups;
        double s = vals[warp][lane];
        for (int g = 1; g < gmax; ++g) s += vals[warp][g * 32 + lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) part[warp * gridDim.x + blockIdx.x] = s;
    }
}

// Grid totals of the four block sums, the same values in every block: a grid
// barrier, then warp u < 4 of every block adds the partials of value u in
// block order (lanes strided, then a fixed shuffle tree) into tot[u].
__device__ __forceinline__ bool grid_totals4(const double* part, unsigned* bar, unsigned& epoch, int* flags,
                                             long long wait_cycles, int* s_ok, double* tot)
{
    if (!grid_barrier(bar, ++epoch * gridDim.x, flags, wait_cycles, s_ok)) return false;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < 4) {
        double acc = 0.0;
        for (unsigned b = lane; b < gridDim.x; b += 32) acc += __ldcg(&part[warp * gridDim.x + b]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) tot[warp] = acc;
    }
    __syncthreads();
    return true;
}

// CG on A_AA lambda_A = b_A from the state k_adj_b left (lambda = 0, r =
// b_A, p = 0, Ap = 0, r.r and the stopping bound in scal).  Block b takes a
// contiguous share of the rods (kCgLanes lanes per rod, each over every
// kCgLanes-th entry of the rod's lists, the force summed over the lanes by
// shuffles) and of the constraints (a thread each).  Iteration k finds in
// memory r_{k-1}, p_{k-1}, Ap_{k-1} and lambda_{k-1}, and holds alpha_{k-1},
// beta_{k-1} (all zero for k = 0, when r holds r_0):
//   rod pass:   r_k = r_{k-1} - alpha Ap_{k-1}, p_k = r_k + beta p_{k-1}
//               (formed where they are read), F = D_A p_k, Up = M F
//               (working precision);
//   constraint: the same r_k and p_k, lambda_k = lambda_{k-1} + alpha p_{k-1},
//               stored with Ap_k = (D^T Up)_A;
//   one grid sum of p_k.Ap_k, r_k.Ap_k, Ap_k.Ap_k and r_k.r_k.
// Then alpha_k = r_k.r_k / p_k.Ap_k and beta_k = r_{k+1}.r_{k+1} / r_k.r_k,
// with r_{k+1}.r_{k+1} = r_k.r_k - 2 alpha_k r_k.Ap_k + alpha_k^2 Ap_k.Ap_k
// expanded from r_{k+1} = r_k - alpha_k Ap_k; the same iterates as the
// textbook loop, with two grid-wide synchronisations an iteration instead
// of three.  Stops with lambda_k when r_k.r_k <= tol^2 r_0.r_0, when k
// reaches max_iter, or when alpha_k <= 0; k is the iteration count.
constexpr int kCgLanes = 8;

// Owned-side arms in constraint order, one 8-value record per constraint
// (e, y_P x e, two pad values), for the CG's gathers by constraint id.
template <typename T>
__global__ void k_cg_arms(int m, int mp, const T* __restrict__ rec, T* __restrict__ pe)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    T* o = pe + 8 * (size_t)c;
#pragma unroll
    for (int w = 0; w < 6; ++w) o[w] = rec[w * (size_t)mp + c];
    o[6] = T(0);
    o[7] = T(0);
}

__device__ __forceinline__ void ld_cgs(const double* cgs, int c, double& r, double& p, double& ap, double& lam)
{
    const double2* q = reinterpret_cast<const double2*>(cgs) + 2 * (size_t)c;
    const double2 a = q[0], b = q[1];
    r = a.x; p = a.y; ap = b.x; lam = b.y;
}

template <typename T>
__global__ void __launch_bounds__(1024, 1) k_cg(CgArgs<T> a)
{
    __shared__ double vals[4][1024];
    __shared__ double tot[4];
    __shared__ double sc[4];   // alpha, beta, r.r, stop flag (thread 0 writes them)
    __shared__ int s_ok;
    if (a.iflag[I_DONE]) return;   // written by k_adj_b before the launch: uniform
    if (a.fault == 1 && blockIdx.x == 0) return;   // test hook: the others' bounded waits run out
    const size_t mp = a.mp, np = a.np;
    const int r0 = (int)((long long)a.n * blockIdx.x / gridDim.x);
    const int r1 = (int)((long long)a.n * (blockIdx.x + 1) / gridDim.x);
    const int na = a.aP[a.n];   // active constraints
    const int c0 = (int)((long long)na * blockIdx.x / gridDim.x);
    const int c1 = (int)((long long)na * (blockIdx.x + 1) / gridDim.x);
    const int sub = threadIdx.x & (kCgLanes - 1);
    constexpr int kRodsPerWarp = 32 / kCgLanes;
    const double tol2 = a.scal[S_TOL2];
    const int maxit = a.iflag[I_MAXIT];
    double rr = a.scal[S_RR], beta = 0.0, alpha = 0.0;
    unsigned epoch = 0;
    int it = 0;
    for (;; ++it) {
        // the loop runs while the warp's first rod is in range (uniform per warp:
        // every lane takes part in the shuffles)
        for (int base = r0 + (int)(threadIdx.x >> 5) * kRodsPerWarp; base < r1;
             base += (int)(blockDim.x >> 5) * kRodsPerWarp) {
            const int i = base + (int)((threadIdx.x & 31) / kCgLanes);
            T F[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
            if (i < r1) {
                for (int t = a.aP[i] + sub; t < a.aP[i + 1]; t += kCgLanes) {
                    const int c = a.alist[t];
                    const T* p8 = a.pe + 8 * (size_t)c;
                    T pv6[6];
#pragma unroll
                    for (int w = 0; w < 6; ++w) pv6[w] = p8[w];
                    double rc, pc, apc, lc;
                    ld_cgs(a.cgs, c, rc, pc, apc, lc);
                    const T v = (T)(fma(-alpha, apc, rc) + beta * pc);
#pragma unroll
                    for (int w = 0; w < 6; ++w) F[w] += v * pv6[w];
                }
                for (int t = a.aQ[i] + sub; t < a.aQ[i + 1]; t += kCgLanes) {
                    const int c = a.bc[t];
                    const T* q8 = a.qe + 8 * (size_t)a.bk[t];
                    T qv[6];
#pragma unroll
                    for (int w = 0; w < 6; ++w) qv[w] = q8[w];
                    double rc, pc, apc, lc;
                    ld_cgs(a.cgs, c, rc, pc, apc, lc);
                    const T v = (T)(fma(-alpha, apc, rc) + beta * pc);
#pragma unroll
                    for (int w = 0; w < 6; ++w) F[w] -= v * qv[w];
                }
            }
#pragma unroll
            for (int o = 1; o < kCgLanes; o <<= 1) {
#pragma unroll
                for (int w = 0; w < 6; ++w) F[w] += __shfl_xor_sync(0xffffffffu, F[w], o);
            }
            if (sub != 0 || i >= r1) continue;
            const T p0 = a.ax[i], p1 = a.ax[np + i], p2 = a.ax[2 * np + i];
            const T pf = p0 * F[0] + p1 * F[1] + p2 * F[2], pt = p0 * F[3] + p1 * F[4] + p2 * F[5];
            const T cf = pf * (a.inv_par - a.inv_perp), ct = pt * (a.inv_spin - a.inv_rot);
            T* o = a.Up + 6 * (size_t)i;
            o[0] = F[0] * a.inv_perp + p0 * cf; o[1] = F[1] * a.inv_perp + p1 * cf; o[2] = F[2] * a.inv_perp + p2 * cf;
            o[3] = F[3] * a.inv_rot + p0 * ct; o[4] = F[4] * a.inv_rot + p1 * ct; o[5] = F[5] * a.inv_rot + p2 * ct;
        }
        if (!grid_barrier(a.bar, ++epoch * gridDim.x, a.flags, a.wait_cycles, &s_ok)) return;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};   // p.Ap, r.Ap, Ap.Ap, r.r
        for (int t = c0 + threadIdx.x; t < c1; t += blockDim.x) {
            const int c = a.alist[t];
            const T* ui = a.Up + 6 * (size_t)a.ci[c];
            const T* uj = a.Up + 6 * (size_t)a.cj[c];
            T s = T(0);
#pragma unroll
            for (int w = 0; w < 3; ++w)
                s += a.rec[w * mp + c] * (ui[w] - uj[w]) + a.rec[(3 + w) * mp + c] * ui[3 + w] -
                     a.rec[(6 + w) * mp + c] * uj[3 + w];
            const double ap = (double)s;
            double rold, pold, apold, lold;
            ld_cgs(a.cgs, c, rold, pold, apold, lold);
            const double rn = fma(-alpha, apold, rold);
            const double pn = rn + beta * pold;
            double2* stc = reinterpret_cast<double2*>(a.cgs) + 2 * (size_t)c;
            stc[0] = make_double2(rn, pn);
            stc[1] = make_double2(ap, lold + alpha * pold);
            acc[0] += pn * ap;
            acc[1] += rn * ap;
            acc[2] += ap * ap;
            acc[3] += rn * rn;
        }
        const int busy = c1 - c0 < (int)blockDim.x ? c1 - c0 : (int)blockDim.x;   // threads that held a constraint
        block_sums4(acc, vals, (busy + 31) >> 5, a.partials);
        if (!grid_totals4(a.partials, a.bar, epoch, a.flags, a.wait_cycles, &s_ok, tot)) return;
        // the step scalars in one thread (every block finds the same totals)
        if (threadIdx.x == 0) {
            const double rk = tot[3], pap = tot[0];
            double al = alpha, be = beta, stop = 0.0;
            if (!(rk > tol2) || it >= maxit) {
                stop = 1.0;
            } else {
                al = pap > 0.0 ? rk / pap : 0.0;
                if (!(al > 0.0)) {
                    stop = 1.0;
                } else {
                    const double rrn = rk - 2.0 * al * tot[1] + al * al * tot[2];
                    be = rrn > 0.0 ? rrn / rk : 0.0;
                }
            }
            sc[0] = al; sc[1] = be; sc[2] = rk; sc[3] = stop;
        }
        __syncthreads();
        alpha = sc[0];
        beta = sc[1];
        rr = sc[2];
        if (sc[3] != 0.0) break;
    }
    // lambda of the block's active constraints for the passes after the CG
    for (int t = c0 + threadIdx.x; t < c1; t += blockDim.x) {
        const int c = a.alist[t];
        a.lam[c] = a.cgs[4 * (size_t)c + 3];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.scal[S_RR] = rr;
        a.scal[S_ALPHA] = alpha;
        a.scal[S_BETA] = beta;
        a.iflag[I_ITERS] = it;
        a.iflag[I_DONE] = 1;
    }
}

// Rod pass 2: w = D lambda, a = u - w, nu = M a (= dL/dF_nc), the mobility's
// axis term and the viscosity partial -(a . U) / eta.
__global__ void k_adj_rods2(int n, int np, Mob mob, double eta, const double* __restrict__ axis,
                            const double* __restrict__ lam, const double* __restrict__ dgeom,
                            const int* __restrict__ rowP, const int* __restrict__ rowQ,
                            const int* __restrict__ qlist, const double* __restrict__ Ftot,
                            const double* __restrict__ U, const double* __restrict__ u, double* __restrict__ nu,
                            double* __restrict__ gp, double* __restrict__ partials, unsigned* counter, double* scal)
{
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double w[6] = {0, 0, 0, 0, 0, 0};
        for (int c = rowP[i]; c < rowP[i + 1]; ++c) {
            const double l = lam[c];
            const double* d = dgeom + 9 * (size_t)c;
#pragma unroll
            for (int k = 0; k < 6; ++k) w[k] += l * d[k];
        }
        for (int k = rowQ[i]; k < rowQ[i + 1]; ++k) {
            const int c = qlist[k];
            const double l = lam[c];
            const double* d = dgeom + 9 * (size_t)c;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                w[a] -= l * d[a];
                w[3 + a] -= l * d[6 + a];
            }
        }
        const double p[3] = {axis[i], axis[np + i], axis[2 * (size_t)np + i]};
        double a[6], F[6], Ui[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            a[k] = u[6 * (size_t)i + k] - w[k];
            F[k] = Ftot[6 * (size_t)i + k];
            Ui[k] = U[6 * (size_t)i + k];
        }
        double nui[6];
        mob_apply(mob, p, a, nui);
        const double ct = mob.inv_par - mob.inv_perp, cr = mob.inv_spin - mob.inv_rot;
        const double pF = dot(p, F), pa = dot(p, a);
        const double pFr = p[0] * F[3] + p[1] * F[4] + p[2] * F[5], par = p[0] * a[3] + p[1] * a[4] + p[2] * a[5];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            gp[3 * (size_t)i + k] = ct * (pF * a[k] + pa * F[k]) + cr * (pFr * a[3 + k] + par * F[3 + k]);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            nu[6 * (size_t)i + k] = nui[k];
            acc -= a[k] * Ui[k];
        }
    }
    double tot;
    if (last_block_total(acc, partials, counter, &tot) && threadIdx.x == 0) scal[S_ETA] = tot / eta;
}

// Constraint pass: the geometric part for every constraint, as contributions
// to d/dDx (rod P +, rod Q -), d/dp_P and d/dp_Q ([m][9]).
__global__ void k_adj_geo(int m, int np, Geo g, double h, const int32_t* __restrict__ pairs,
                          const double* __restrict__ xw, const double* __restrict__ axis,
                          const double* __restrict__ dgeom, const double* __restrict__ gamma,
                          const double* __restrict__ lam, const double* __restrict__ nu,
                          const double* __restrict__ U, double* __restrict__ geo)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    const int i = pairs[3 * (size_t)c], j = pairs[3 * (size_t)c + 1], code = pairs[3 * (size_t)c + 2];
    const int kk[3] = {code % 3 - 1, (code / 3) % 3 - 1, code / 9 - 1};
    double dx[3], pa[3], pb[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dx[a] = __dsub_rn(__dsub_rn(xw[a * (size_t)np + i], xw[a * (size_t)np + j]), __dmul_rn((double)kk[a], g.box[a]));
        pa[a] = axis[a * (size_t)np + i];
        pb[a] = axis[a * (size_t)np + j];
    }
    double s, t;
    const double rho = segment_closest<double>(dx, pa, pb, g.half, kParallelDet64, s, t);
    const double* d = dgeom + 9 * (size_t)c;
    const double e[3] = {d[0], d[1], d[2]};
    double r[3], yP[3], yQ[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        yP[a] = s * pa[a];
        yQ[a] = t * pb[a];
        r[a] = dx[a] + yP[a] - yQ[a];
    }
    const double gc = gamma[c], lc = lam[c];
    double at[3], aP[3], aQ[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        at[a] = gc * (nu[6 * (size_t)i + a] - nu[6 * (size_t)j + a]) - lc * (U[6 * (size_t)i + a] - U[6 * (size_t)j + a]);
        aP[a] = gc * nu[6 * (size_t)i + 3 + a] - lc * U[6 * (size_t)i + 3 + a];
        aQ[a] = gc * nu[6 * (size_t)j + 3 + a] - lc * U[6 * (size_t)j + 3 + a];
    }
    double c1[3], c2[3], be[3], bP[3], bQ[3];
    cross(aP, yP, c1);
    cross(aQ, yQ, c2);
#pragma unroll
    for (int a = 0; a < 3; ++a) be[a] = at[a] + c1[a] - c2[a];
    cross(e, aP, bP);
    cross(e, aQ, bQ);
#pragma unroll
    for (int a = 0; a < 3; ++a) bQ[a] = -bQ[a];
    double kap[3] = {0, 0, 0};
    if (rho > 0.0) {
        const double eb = dot(e, be);
#pragma unroll
        for (int a = 0; a < 3; ++a) kap[a] = (be[a] - e[a] * eb) / rho;
    }
    const double lh = lc / h;
    double gdx[3], gpa[3], gpb[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        gdx[a] = kap[a] - lh * e[a];
        gpa[a] = s * (kap[a] + bP[a]) - lh * s * e[a];
        gpb[a] = t * (bQ[a] - kap[a]) + lh * t * e[a];
    }
    double ks[3], kt[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ks[a] = kap[a] + bP[a];
        kt[a] = bQ[a] - kap[a];
    }
    const double sig_s = dot(ks, pa), sig_t = dot(kt, pb);
    const double A = dot(pa, pa), B = dot(pa, pb), C = dot(pb, pb);
    const double det = A * C - B * B;
    const bool parallel = !(det > kParallelDet64 * A * C);
    const bool s_free = fabs(s) < g.half, t_free = fabs(t) < g.half;
    // R1 = dDx.pa + dpa.(s pa + r) - dpb.(t pa);  R2 = dDx.pb + dpa.(s pb) + dpb.(r - t pb)
    double c_1 = 0.0, c_2 = 0.0;   // the closest-point terms are -c_1 R1 - c_2 R2
    if (!parallel && s_free && t_free) {
        // J^T xi = sigma, J = [[A, -B], [B, -C]]
        const double dj = -A * C + B * B;
        c_1 = (-C * sig_s - B * sig_t) / dj;
        c_2 = (B * sig_s + A * sig_t) / dj;
    } else if (!parallel && s_free) {
        c_1 = sig_s / A;
    } else if (!parallel && t_free) {
        c_2 = -sig_t / C;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        gdx[a] -= c_1 * pa[a] + c_2 * pb[a];
        gpa[a] -= c_1 * (s * pa[a] + r[a]) + c_2 * s * pb[a];
        gpb[a] -= -c_1 * t * pa[a] + c_2 * (r[a] - t * pb[a]);
    }
    double* o = geo + 9 * (size_t)c;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o[a] = gdx[a];
        o[3 + a] = gpa[a];
        o[6 + a] = gpb[a];
    }
}

// Rod pass 3: gather the constraint terms, map d/dp to the quaternion
// (p = (2(ac + sb), 2(bc - sa), s^2 - a^2 - b^2 + c^2)), project onto the
// tangent space and write the caller's arrays.
__global__ void k_adj_rods3(int n, const double* __restrict__ quat, const int* __restrict__ rowP,
                            const int* __restrict__ rowQ, const int* __restrict__ qlist,
                            const double* __restrict__ geo, const double* __restrict__ gx,
                            const double* __restrict__ gq, const double* __restrict__ gp,
                            const double* __restrict__ nu, double* __restrict__ out_x, double* __restrict__ out_q,
                            double* __restrict__ out_f)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double X[3], P[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        X[a] = gx[3 * (size_t)i + a];
        P[a] = gp[3 * (size_t)i + a];
    }
    for (int c = rowP[i]; c < rowP[i + 1]; ++c) {
        const double* o = geo + 9 * (size_t)c;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            X[a] += o[a];
            P[a] += o[3 + a];
        }
    }
    for (int k = rowQ[i]; k < rowQ[i + 1]; ++k) {
        const double* o = geo + 9 * (size_t)qlist[k];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            X[a] -= o[a];
            P[a] += o[6 + a];
        }
    }
    const double s = quat[4 * (size_t)i], qa = quat[4 * (size_t)i + 1], qb = quat[4 * (size_t)i + 2],
                 qc = quat[4 * (size_t)i + 3];
    double G[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) G[a] = gq[4 * (size_t)i + a];
    G[0] += 2.0 * (qb * P[0] - qa * P[1] + s * P[2]);
    G[1] += 2.0 * (qc * P[0] - s * P[1] - qa * P[2]);
    G[2] += 2.0 * (s * P[0] + qc * P[1] - qb * P[2]);
    G[3] += 2.0 * (qa * P[0] + qb * P[1] + qc * P[2]);
    const double th[4] = {s, qa, qb, qc};
    const double pr = G[0] * th[0] + G[1] * th[1] + G[2] * th[2] + G[3] * th[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) out_x[3 * (size_t)i + a] = X[a];
#pragma unroll
    for (int a = 0; a < 4; ++a) out_q[4 * (size_t)i + a] = G[a] - th[a] * pr;
    if (out_f) {
#pragma unroll
        for (int k = 0; k < 6; ++k) out_f[6 * (size_t)i + k] = nu[6 * (size_t)i + k];
    }
}

// ---------------------------------------------------------------- host side

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }

cudaError_t adjoint_reserve(aLENS_ctx* ctx)
{
    if (ctx->adj_ws) return cudaSuccess;
    const size_t np = (size_t)ctx->max_rods, mp = (size_t)ctx->max_pairs;
    // per rod: Ftot, U, u, Mu, nu, Up (6 each), gx, gp (3), gq (4); per constraint: lam, the CG
    // state (r, p, Ap, lambda), geo (9; the CG's owned-side arm records live there until k_adj_geo)
    // (each slice is rounded up to 8 doubles: 13 slices, at most 91 doubles of padding)
    const size_t doubles = np * (6 * 6 + 3 + 3 + 4) + mp * (1 + 4 + 9) + S_NSCAL + 128;
    // then the flags and the CG's active-set lists (ints): counts and row
    // pointers of the owned and other-side lists, the lists (3 mp)
    const size_t ints = I_NI + 4 * (np + 1) + 3 * mp + 64;
    cudaError_t e = cudaMalloc(&ctx->adj_ws, doubles * sizeof(double) + ints * sizeof(int));
    if (e != cudaSuccess) {
        ctx->adj_ws = nullptr;
        return e;
    }
    return cudaSuccess;
}

cudaError_t launch_adjoint(aLENS_ctx* ctx, int n, int m, const double* quat, const double* fnc,
                           const int32_t* pairs, const double* gamma, const double* gxn, const double* gqn,
                           double* out_x, double* out_q, double* out_f, int* cg_iters, double* cg_rel,
                           double* deta)
{
    const size_t np = (size_t)ctx->max_rods, mp = (size_t)ctx->max_pairs;
    double* base = (double*)ctx->adj_ws;
    size_t o = 0;
    auto take = [&](size_t cnt) { double* r = base + o; o += (cnt + 7) & ~(size_t)7; return r; };
    double* Ftot = take(6 * np);
    double* U = take(6 * np);
    double* u = take(6 * np);
    double* Mu = take(6 * np);
    double* nu = take(6 * np);
    double* Upd = take(6 * np);   // CG rod velocities (working precision view)
    double* gx = take(3 * np);
    double* gp = take(3 * np);
    double* gq = take(4 * np);
    double* lam = take(mp);
    double* cgs = take(4 * mp);
    double* geo = take(9 * mp);
    double* scal = take(S_NSCAL);
    int* iflag = (int*)(base + o);
    int* cA = iflag + 16;       // [np] active owned constraints per rod
    int* cB = cA + np;          // [np] active other-side entries per rod
    int* aP = cB + np;          // [np + 1]
    int* aQ = aP + np + 1;      // [np + 1]
    int* alist = aQ + np + 1;   // [mp]
    int* bk = alist + mp;       // [mp]
    int* bc = bk + mp;          // [mp]
    cudaStream_t st = ctx->stream;
    const int mixed = ctx->p.precision == ALENS_MIXED;
    const double h = ctx->p.dt;
    const int G = ctx->num_sms < ctx->max_blocks ? ctx->num_sms : ctx->max_blocks;
    unsigned* counter = ctx->bar;   // the solver's barrier words are free here
    cudaError_t e;
    if ((e = cudaMemsetAsync(ctx->bar, 0, 4 * sizeof(unsigned), st)) != cudaSuccess) return e;
    const int maxit = ctx->p.max_iter > 0 ? ctx->p.max_iter : 1;
    if ((e = cudaMemsetAsync(iflag, 0, I_NI * sizeof(int), st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(iflag + I_MAXIT, &maxit, sizeof(int), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(lam, 0, sizeof(double) * (m > 0 ? m : 1), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(scal, 0, sizeof(double) * S_NSCAL, st)) != cudaSuccess) return e;
    k_adj_rods1<<<nblk(n, 128), 128, 0, st>>>(n, (int)np, ctx->mob, h, ctx->axis, quat, fnc, gamma, ctx->dgeom,
                                              ctx->rowP, ctx->rowQ, ctx->qlist, gxn, gqn, Ftot, U, u, Mu, gx, gq);
    ++ctx->launches;
    const double tol = mixed ? 1e-7 : 1e-13;
    int iters = 0;
    double rel = 0.0;
    if (m > 0) {
        if ((e = launch_setup_qe(ctx)) != cudaSuccess) return e;   // the CG reads the forward step's qe
        k_adj_b<<<G, 256, 0, st>>>(m, pairs, ctx->dgeom, gamma, Mu, lam, cgs, ctx->partials, counter, scal, iflag,
                                   tol);
        ++ctx->launches;
        if (mixed)
            k_cg_arms<float><<<nblk(m, 256), 256, 0, st>>>(m, (int)mp, ctx->sb32.rec, reinterpret_cast<float*>(geo));
        else
            k_cg_arms<double><<<nblk(m, 256), 256, 0, st>>>(m, (int)mp, ctx->sb64.rec, geo);
        ++ctx->launches;
        // the active set as lists (the CG touches active constraints only)
        k_act_count<<<nblk(n, 128), 128, 0, st>>>(n, ctx->rowP, ctx->rowQ, ctx->qlist, gamma, cA, cB);
        ++ctx->launches;
        if ((e = exclusive_scan(ctx, cA, aP, n)) != cudaSuccess || (e = exclusive_scan(ctx, cB, aQ, n)) != cudaSuccess)
            return e;
        k_act_fill<<<nblk(n, 128), 128, 0, st>>>(n, ctx->rowP, ctx->rowQ, ctx->qlist, gamma, aP, aQ, alist, bk, bc);
        ++ctx->launches;
        // the persistent CG: one block per SM (cooperative launch)
        const void* fn = mixed ? (const void*)k_cg<float> : (const void*)k_cg<double>;
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 1024, 0)) != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
        const long long wait = (long long)(ctx->wait_s * ctx->clock_khz * 1e3);
        const int fault = ctx->fault_mode;   // a pending hook is taken by this launch
        ctx->fault_mode = 0;
        if (mixed) {
            const SolveBufs<float>& sb = ctx->sb32;
            CgArgs<float> ca{n, m, (int)np, (int)mp, ctx->rowP, ctx->rowQ, ctx->qlist, ctx->ci, ctx->cj, sb.rec, sb.qe,
                             sb.ax, (float)ctx->mob.inv_perp, (float)ctx->mob.inv_par, (float)ctx->mob.inv_rot,
                             (float)ctx->mob.inv_spin, aP, aQ, alist, bk, bc, reinterpret_cast<const float*>(geo), cgs,
                             lam, (float*)Upd, ctx->partials,
                             ctx->bar + 2, ctx->dflags, scal, iflag, wait, fault};
            void* args[] = {&ca};
            if ((e = cudaLaunchCooperativeKernel(fn, dim3((unsigned)G), dim3(1024), args, 0, st)) != cudaSuccess)
                return e;
        } else {
            const SolveBufs<double>& sb = ctx->sb64;
            CgArgs<double> ca{n, m, (int)np, (int)mp, ctx->rowP, ctx->rowQ, ctx->qlist, ctx->ci, ctx->cj, sb.rec,
                              sb.qe, sb.ax, ctx->mob.inv_perp, ctx->mob.inv_par, ctx->mob.inv_rot, ctx->mob.inv_spin,
                              aP, aQ, alist, bk, bc, geo, cgs, lam, Upd, ctx->partials, ctx->bar + 2, ctx->dflags, scal,
                              iflag, wait,
                              fault};
            void* args[] = {&ca};
            if ((e = cudaLaunchCooperativeKernel(fn, dim3((unsigned)G), dim3(1024), args, 0, st)) != cudaSuccess)
                return e;
        }
        ++ctx->launches;
        int hflag[I_NI];
        if ((e = cudaMemcpyAsync(hflag, iflag, sizeof(hflag), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return e;
        iters = hflag[I_ITERS];
        double hs[S_NSCAL];
        if ((e = cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return e;
        rel = hs[S_RR0] > 0.0 ? sqrt(hs[S_RR] / hs[S_RR0]) : 0.0;
    }
    k_adj_rods2<<<G, 128, 0, st>>>(n, (int)np, ctx->mob, ctx->p.viscosity, ctx->axis, lam, ctx->dgeom, ctx->rowP,
                                   ctx->rowQ, ctx->qlist, Ftot, U, u, nu, gp, ctx->partials, counter, scal);
    ++ctx->launches;
    if (m > 0) {
        k_adj_geo<<<nblk(m, 128), 128, 0, st>>>(m, (int)np, ctx->geo, h, pairs, ctx->xw, ctx->axis, ctx->dgeom, gamma,
                                                lam, nu, U, geo);
        ++ctx->launches;
    }
    k_adj_rods3<<<nblk(n, 128), 128, 0, st>>>(n, quat, ctx->rowP, ctx->rowQ, ctx->qlist, geo, gx, gq, gp, nu, out_x,
                                              out_q, out_f);
    ++ctx->launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    double hs[S_NSCAL];
    if ((e = cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return e;
    if (deta) *deta = hs[S_ETA];
    *cg_iters = iters;
    *cg_rel = rel;
    return cudaSuccess;
}

}  // namespace alens
