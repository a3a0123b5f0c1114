// Constraint assembly and the solver's sparse layout.
//
// Appendix "Symmetry ...": each collision constraint is one sparse column
// D_PQ = [e_P, y_P x e_P, e_Q, y_Q x e_Q] with e_P = r/|r| = -e_Q and
// r = x_P + y_P - x_Q - y_Q between the closest points.  Appendix Eq.
// blockdef: q = Phi/h + D^T M F_nc.
//
// k_assemble: one thread per pair; float64 closest points, Phi, the 9 values
// (e, y_P x e, y_Q x e) and q, with fused multiply-adds and one reciprocal
// for the normal (the FP64 pipe bounds the kernel; the keep/drop decision
// upstream rounds unfused, like the oracle).  Overlap count and minimum gap
// are reduced per warp before one atomic each.
//
// Solver layout (k_setup_*): constraint-major records in the solver's
// working precision, the P-side CSR (pairs sorted by i make each rod's
// P-constraints one contiguous range), and a Q-side CSR (per rod j, the ids
// of constraints with Q = j, sorted ascending) with a copy of (e, y_Q x e)
// laid out in CSR order so that the rod-parallel gather reads it
// contiguously.
#include <float.h>

#include <climits>

#include "internal.cuh"

namespace alens {

__device__ __forceinline__ long long gap_key(double v)
{
    long long b = __double_as_longlong(v);
    return b >= 0 ? b : b ^ 0x7fffffffffffffffLL;
}

__global__ void k_assemble(int m, int n, int np, Geo g0, const SysGeo* __restrict__ systab,
                           const int* __restrict__ sysid, const int32_t* __restrict__ pairs,
                           const double* __restrict__ xw, const double* __restrict__ axis,
                           const double* __restrict__ unc, double* __restrict__ phi, double* __restrict__ dgeom,
                           double* __restrict__ q, unsigned long long* __restrict__ counters, int* __restrict__ flags,
                           const unsigned long long* __restrict__ mdev)
{
    m = count_of(m, mdev);
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    bool active = c < m;
    bool overlap = false;
    long long key = LLONG_MAX;
    if (active) {
        int i = pairs[3 * (size_t)c], j = pairs[3 * (size_t)c + 1], code = pairs[3 * (size_t)c + 2];
        if (!(i >= 0 && i < j && j < n && code >= 0 && code < 27)) {
            if (atomicCAS(&flags[F_ERR], 0, ALENS_ERR_INVALID) == 0) flags[F_ERR_ROD] = c;
            active = false;
        } else if (systab && sysid[i] != sysid[j]) {   // a batch pair must stay inside one system
            if (atomicCAS(&flags[F_ERR], 0, ALENS_ERR_INVALID) == 0) flags[F_ERR_ROD] = c;
            active = false;
        } else {
            const Geo& g = geo_of(g0, systab, sysid, i);
            int kk[3] = {code % 3 - 1, (code / 3) % 3 - 1, code / 9 - 1};
            double dx[3], p[3], qv[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                dx[a] = __dsub_rn(__dsub_rn(xw[a * (size_t)np + i], xw[a * (size_t)np + j]),
                                  __dmul_rn((double)kk[a], g.box[a]));
                p[a] = axis[a * (size_t)np + i];
                qv[a] = axis[a * (size_t)np + j];
            }
            double s, t, r[3];
            const double dist = segment_closest<double, true>(dx, p, qv, g.half, kParallelDet64, s, t, r);
            double yP[3], yQ[3], e[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                yP[a] = s * p[a];
                yQ[a] = t * qv[a];
            }
            if (dist > 0.0) {
                const double inv = 1.0 / dist;
#pragma unroll
                for (int a = 0; a < 3; ++a) e[a] = r[a] * inv;
            } else {
                // centrelines touch: normal of the two axes, turned towards P;
                // collinear axes: along the axis, towards P; coincident: e_x
                double nx = p[1] * qv[2] - p[2] * qv[1], ny = p[2] * qv[0] - p[0] * qv[2],
                       nz = p[0] * qv[1] - p[1] * qv[0];
                double nn = sqrt(nx * nx + ny * ny + nz * nz);
                if (nn > 1e-12) {
                    double sg = (nx * dx[0] + ny * dx[1] + nz * dx[2]) < 0.0 ? -1.0 : 1.0;
                    e[0] = sg * nx / nn; e[1] = sg * ny / nn; e[2] = sg * nz / nn;
                } else {
                    double pd = p[0] * dx[0] + p[1] * dx[1] + p[2] * dx[2];
                    if (pd != 0.0) {
                        double sg = pd < 0.0 ? -1.0 : 1.0;
                        double pn = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
                        e[0] = sg * p[0] / pn; e[1] = sg * p[1] / pn; e[2] = sg * p[2] / pn;
                    } else {
                        e[0] = 1.0; e[1] = 0.0; e[2] = 0.0;
                    }
                }
            }
            const double ta[3] = {fma(yP[1], e[2], -(yP[2] * e[1])), fma(yP[2], e[0], -(yP[0] * e[2])),
                                  fma(yP[0], e[1], -(yP[1] * e[0]))};
            const double tb[3] = {fma(yQ[1], e[2], -(yQ[2] * e[1])), fma(yQ[2], e[0], -(yQ[0] * e[2])),
                                  fma(yQ[0], e[1], -(yQ[1] * e[0]))};
            double* dg = dgeom + 9 * (size_t)c;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                dg[a] = e[a];
                dg[3 + a] = ta[a];
                dg[6 + a] = tb[a];
            }
            double ph = dist - g.diameter;
            double dtu = 0.0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                dtu = fma(e[a], unc[a * (size_t)np + i] - unc[a * (size_t)np + j], dtu);
                dtu = fma(ta[a], unc[(3 + a) * (size_t)np + i], dtu);
                dtu = fma(-tb[a], unc[(3 + a) * (size_t)np + j], dtu);
            }
            phi[c] = ph;
            q[c] = ph / g.dt + dtu;
            overlap = ph < 0.0;
            key = gap_key(ph);
        }
    }
    unsigned bal = __ballot_sync(0xffffffffu, overlap);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        long long other = __shfl_down_sync(0xffffffffu, key, o);
        key = other < key ? other : key;
    }
    if ((threadIdx.x & 31) == 0) {
        if (bal) atomicAdd(&counters[C_OVERLAP], (unsigned long long)__popc(bal));
        if (key != LLONG_MAX) atomicMin((long long*)&counters[C_MINGAP], key);
    }
}

// Validation of a caller's pair list: ranges, i < j, sorted by i.
__global__ void k_check_pairs(int m, int n, const int32_t* __restrict__ pairs, int* __restrict__ flags)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    int i = pairs[3 * (size_t)c], j = pairs[3 * (size_t)c + 1], code = pairs[3 * (size_t)c + 2];
    bool ok = i >= 0 && i < j && j < n && code >= 0 && code < 27;
    if (ok && c > 0 && pairs[3 * (size_t)(c - 1)] > i) ok = false;
    if (!ok && atomicCAS(&flags[F_ERR], 0, ALENS_ERR_INVALID) == 0) flags[F_ERR_ROD] = c;
}

// The solver numbers rods by rank (their position in the cell-sorted order
// when one is given, else their id) and gives each constraint to the
// endpoint of lower rank (the "owner"; the other endpoint is its Q side).
// A wall row (j = -1) has no other side: rq = -1, owner i.
__device__ __forceinline__ void owner_other(const int32_t* pairs, const int* rank, int c, int& ro, int& rq, bool& flip)
{
    int i = pairs[3 * (size_t)c], j = pairs[3 * (size_t)c + 1];
    if (j < 0) {
        ro = rank ? rank[i] : i;
        rq = -1;
        flip = false;
        return;
    }
    int ri = rank ? rank[i] : i, rj = rank ? rank[j] : j;
    flip = ri > rj;
    ro = flip ? rj : ri;
    rq = flip ? ri : rj;
}

__global__ void k_count_sides(int m, const int32_t* __restrict__ pairs, const int* __restrict__ rank,
                              int* __restrict__ cntP, int* __restrict__ cntQ, const unsigned long long* __restrict__ mdev)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= count_of(m, mdev)) return;
    int ro, rq;
    bool flip;
    owner_other(pairs, rank, c, ro, rq, flip);
    atomicAdd(&cntP[ro], 1);
    if (rq >= 0) atomicAdd(&cntQ[rq], 1);
}

__global__ void k_scatter_owner(int m, const int32_t* __restrict__ pairs, const int* __restrict__ rank,
                                const int* __restrict__ rowP, int* __restrict__ curP, int* __restrict__ perm,
                                const unsigned long long* __restrict__ mdev)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= count_of(m, mdev)) return;
    int ro, rq;
    bool flip;
    owner_other(pairs, rank, c, ro, rq, flip);
    perm[rowP[ro] + atomicAdd(&curP[ro], 1)] = c;
}

// Ascending order inside every CSR segment (segments are short), so that
// the layout does not depend on the order of the atomics above.  A segment
// of up to kSegRegs entries is loaded at once and each entry stored at its
// rank (the entries are distinct constraint ids); a longer one is sorted in
// place.
constexpr int kSegRegs = 16;
__global__ void k_sort_segments(int n, const int* __restrict__ row, int* __restrict__ list)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int b = row[r], e = row[r + 1];
    if (e - b <= kSegRegs) {
        const int len = e - b;
        int v[kSegRegs];
#pragma unroll
        for (int u = 0; u < kSegRegs; ++u) v[u] = u < len ? list[b + u] : INT_MAX;
#pragma unroll
        for (int u = 0; u < kSegRegs; ++u) {
            if (u < len) {
                int k = 0;
#pragma unroll
                for (int t = 0; t < kSegRegs; ++t) k += v[t] < v[u];
                list[b + k] = v[u];
            }
        }
        return;
    }
    for (int u = b + 1; u < e; ++u) {
        int v = list[u];
        int w = u - 1;
        while (w >= b && list[w] > v) {
            list[w + 1] = list[w];
            --w;
        }
        list[w + 1] = v;
    }
}

// One rod's part of a constraint's diagonal entry D_c^T M D_c: e.M_t.e +
// a.M_r.a for the normal e and the rod's arm cross normal a (Eq. blockdef
// M with the rod's drag tensors; the signs of e and a do not matter).  In
// float32: the entry only sets the scaling, which needs to be positive and
// consistent, not exact.
template <typename T>
__device__ __forceinline__ float rod_quad(const double* e, const double* a, const T* ax, int np, int r, float ip,
                                          float ipa, float ir, float is)
{
    const float p0 = (float)ax[r], p1 = (float)ax[np + r], p2 = (float)ax[2 * (size_t)np + r];
    const float e0 = (float)e[0], e1 = (float)e[1], e2 = (float)e[2];
    const float a0 = (float)a[0], a1 = (float)a[1], a2 = (float)a[2];
    const float pe = p0 * e0 + p1 * e1 + p2 * e2, pa = p0 * a0 + p1 * a1 + p2 * a2;
    const float ee = e0 * e0 + e1 * e1 + e2 * e2, aa = a0 * a0 + a1 * a1 + a2 * a2;
    return ip * ee + (ipa - ip) * (pe * pe) + ir * aa + (is - ir) * (pa * pa);
}

// Internal constraint cc (owner-major) <- caller constraint perm[cc].  When
// the owner is the caller's Q rod the column is written from its side:
// e' = -e, (owner arm x e') = -(y_Q x e), (other arm x e') = -(y_P x e).
// With beta > 0 the solver works on the diagonally scaled problem gamma =
// sigma gamma~ (aLENS_set_scaling): the record and q are multiplied by
// sigma_c = (D_c^T M D_c + C_c)^(-beta/2) (evaluated in float32, so a
// float value held exactly in float64), the compliance by sigma_c^2 and the
// starting gamma divided by sigma_c; sigma_c and 1/sigma_c (working
// precision) are kept for the output and the residual.
template <typename T>
__global__ void k_setup_fill(int m, int mp, const int* __restrict__ perm, const int32_t* __restrict__ pairs,
                             const int* __restrict__ rank, const double* __restrict__ dgeom,
                             const double* __restrict__ q64, const double* __restrict__ gin,
                             const int* __restrict__ rowQ, int* __restrict__ curQ, int* __restrict__ qlist,
                             int* __restrict__ ci, int* __restrict__ cj, T* __restrict__ rec, T* __restrict__ qT,
                             T* __restrict__ gg0, T* __restrict__ gg1, T* __restrict__ rec_lo, T* __restrict__ q_lo,
                             const double* __restrict__ comp64, T* __restrict__ compT, int np, const T* __restrict__ ax,
                             const T* __restrict__ mobr, Mob mob0, double beta, double* __restrict__ scale64,
                             T* __restrict__ isc, T* __restrict__ lop, T* __restrict__ loq,
                             const unsigned long long* __restrict__ mdev)
{
    int cc = blockIdx.x * blockDim.x + threadIdx.x;
    if (cc >= count_of(m, mdev)) return;
    int c = perm[cc];
    int ro, rq;
    bool flip;
    owner_other(pairs, rank, c, ro, rq, flip);
    ci[cc] = ro;
    cj[cc] = rq;
    const double* dg = dgeom + 9 * (size_t)c;
    double r[9];
    if (!flip) {
#pragma unroll
        for (int u = 0; u < 9; ++u) r[u] = dg[u];
    } else {
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            r[u] = -dg[u];
            r[3 + u] = -dg[6 + u];
            r[6 + u] = -dg[3 + u];
        }
    }
    double cmp = comp64 ? comp64[c] : -1.0;
    double sig = 1.0;
    if (beta > 0.0) {
        // the rods' axes and drags in rank order (written just before)
        auto part = [&](const double* arm, int rr) {
            if (mobr)
                return rod_quad(r, arm, ax, np, rr, (float)mobr[rr], (float)mobr[np + rr], (float)mobr[2 * (size_t)np + rr],
                                (float)mobr[3 * (size_t)np + rr]);
            return rod_quad(r, arm, ax, np, rr, (float)mob0.inv_perp, (float)mob0.inv_par, (float)mob0.inv_rot,
                            (float)mob0.inv_spin);
        };
        float a = part(r + 3, ro);
        if (rq >= 0) a += part(r + 6, rq);   // rq < 0: a wall
        if (cmp >= 0.0) a += (float)cmp;
        if (a > 0.0f && isfinite(a)) {
            const float sf = exp2f(-0.5f * (float)beta * log2f(a));
            if (sf > 0.0f && isfinite(sf)) sig = (double)sf;
        }
    }
    scale64[cc] = sig;
    // sig is a float value: for float, 1/sig in float is (T)(1.0 / sig)
    // (double rounding is innocuous for a quotient at 53 >= 2 * 24 + 2 bits)
    isc[cc] = sizeof(T) == 4 ? (T)__fdiv_rn(1.0f, (float)sig) : (T)(1.0 / sig);
    T lo[9];
#pragma unroll
    for (int u = 0; u < 9; ++u) {
        const double rs = r[u] * sig;
        const T hi = (T)rs;
        rec[u * (size_t)mp + cc] = hi;
        lo[u] = sizeof(T) == 4 ? (T)(rs - (double)hi) : T(0);   // float32: the rounding error
        if (rec_lo) rec_lo[u * (size_t)mp + cc] = lo[u];
    }
    if (lop) {   // the same low parts as one row per side (the one-barrier reference passes gather them)
        T* p = lop + 8 * (size_t)cc;
        T* q = loq + 8 * (size_t)cc;
#pragma unroll
        for (int u = 0; u < 6; ++u) p[u] = lo[u];
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            q[u] = lo[u];
            q[3 + u] = lo[6 + u];
        }
        p[6] = p[7] = q[6] = q[7] = T(0);
    }
    const double qs = q64[c] * sig;
    const T qh = (T)qs;
    qT[cc] = qh;
    if (q_lo) q_lo[cc] = (T)(qs - (double)qh);
    if (comp64) compT[cc] = (T)(cmp >= 0.0 ? cmp * (sig * sig) : cmp);
    double v = gin ? gin[c] / sig : 0.0;
    if (!(v > 0.0) && !(cmp >= 0.0)) v = 0.0;   // collisions start at gamma >= 0, springs anywhere
    // solver state (delta, g, gamma_ref, gamma_lo) in both buffers: gamma_0
    // (split into a working-precision value and its rounding error) is the
    // first reference
    const T vh = (T)v;
    for (int b = 0; b < 2; ++b) {
        T* st = (b ? gg1 : gg0) + 4 * (size_t)cc;
        st[0] = T(0);
        st[1] = T(0);
        st[2] = vh;
        st[3] = (T)(v - (double)vh);
    }
    if (rq >= 0) qlist[rowQ[rq] + atomicAdd(&curQ[rq], 1)] = cc;
}

// Other-side arms in CSR order, one 8-value record per entry (e, arm x e,
// two pad values) so that the solver's gather is one or two vector loads;
// and the same record of each constraint's owner side in owner order (the
// global-memory rod phase walks a rod's owned constraints from lanes that
// hold unrelated rods, so six scalar columns would cost six sectors).
template <typename T>
__global__ void k_setup_qe(int m, int mp, const int* __restrict__ qlist, const T* __restrict__ rec,
                           T* __restrict__ qe, const T* __restrict__ rec_lo, T* __restrict__ qe_lo,
                           T* __restrict__ pe, const unsigned long long* __restrict__ mdev)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count_of(m, mdev)) return;
    if (pe) {   // constraint k's owner side as one record: the global rod phase reads it whole
        T* o = pe + 8 * (size_t)k;
#pragma unroll
        for (int u = 0; u < 6; ++u) o[u] = rec[u * (size_t)mp + k];
        o[6] = T(0);
        o[7] = T(0);
    }
    int c = qlist[k];
    T* o = qe + 8 * (size_t)k;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
        o[u] = rec[u * (size_t)mp + c];
        o[3 + u] = rec[(6 + u) * (size_t)mp + c];
    }
    o[6] = T(0);
    o[7] = T(0);
    if (rec_lo) {
        T* l = qe_lo + 8 * (size_t)k;
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            l[u] = rec_lo[u * (size_t)mp + c];
            l[3 + u] = rec_lo[(6 + u) * (size_t)mp + c];
        }
        l[6] = T(0);
        l[7] = T(0);
    }
}

template <typename T>
__global__ void k_setup_rods(int n, int np, const double* __restrict__ quat, const int* __restrict__ rank,
                             const SysGeo* __restrict__ systab, const int* __restrict__ sysid, T* __restrict__ ax,
                             T* __restrict__ mobr)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double p0, p1, p2;
    quat_axis(quat[4 * (size_t)i], quat[4 * (size_t)i + 1], quat[4 * (size_t)i + 2], quat[4 * (size_t)i + 3], p0, p1,
              p2);
    int r = rank ? rank[i] : i;
    ax[r] = (T)p0;
    ax[np + r] = (T)p1;
    ax[2 * (size_t)np + r] = (T)p2;
    if (systab) {   // batches: the drags of the rod's system
        const Mob& mb = systab[sysid[i]].mob;
        mobr[r] = (T)mb.inv_perp;
        mobr[np + r] = (T)mb.inv_par;
        mobr[2 * (size_t)np + r] = (T)mb.inv_rot;
        mobr[3 * (size_t)np + r] = (T)mb.inv_spin;
    }
}

// Spring b (bilateral constraint; Appendix: Phi_b is the distance between
// two fixed points of particles P and Q, K [Phi_b - Phi_b^0] = -gamma_b;
// Eqs. linearconstraints b, blockdef D and F): the point at arclength s_P on
// rod P and the point at s_Q on rod Q, taken over their minimum periodic
// image; Phi_b = |r|, e = r / |r| and the D column (e, y_P x e | -e,
// -(y_Q x e)) exactly as for a collision.  Row mu + b of the constraint list:
// pairs (P, Q, image), phi = Phi_b, dgeom, q = (Phi_b - rest)/h + D^T M F_nc,
// comp64 = 1/(h kappa).  Rows below mu (collisions) get comp64 = -1.
__global__ void k_assemble_springs(int nb, int n, int np, int mu, Geo g0, const SysGeo* __restrict__ systab,
                                   const int* __restrict__ sysid, const int32_t* __restrict__ ends,
                                   const double* __restrict__ arms, const double* __restrict__ kappa,
                                   const double* __restrict__ rest, const double* __restrict__ xw,
                                   const double* __restrict__ axis, const double* __restrict__ unc,
                                   int32_t* __restrict__ pairs, double* __restrict__ phi, double* __restrict__ dgeom,
                                   double* __restrict__ q, double* __restrict__ comp64, int* __restrict__ flags)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < mu) comp64[t] = -1.0;
    if (t >= nb) return;
    const int b = t, i = ends[2 * (size_t)b], j = ends[2 * (size_t)b + 1];
    const double sP = arms[2 * (size_t)b], sQ = arms[2 * (size_t)b + 1], kp = kappa[b], r0 = rest[b];
    bool ok = i >= 0 && i < n && j >= 0 && j < n && i != j && kp > 0.0 && isfinite(kp) && isfinite(sP) &&
              isfinite(sQ) && isfinite(r0);
    if (ok && systab && sysid[i] != sysid[j]) ok = false;   // a batch spring stays inside one system
    if (!ok) {
        if (atomicCAS(&flags[F_ERR], 0, ALENS_ERR_INVALID) == 0) flags[F_ERR_ROD] = mu + b;
        return;
    }
    const Geo& g = geo_of(g0, systab, sysid, i);
    double yP[3], yQ[3], r[3], e[3];
    int k[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        yP[a] = sP * axis[a * (size_t)np + i];
        yQ[a] = sQ * axis[a * (size_t)np + j];
        const double d = xw[a * (size_t)np + i] + yP[a] - xw[a * (size_t)np + j] - yQ[a];
        int kk = (int)nearbyint(d / g.box[a]);
        kk = kk > 1 ? 1 : (kk < -1 ? -1 : kk);
        k[a] = kk;
        r[a] = d - (double)kk * g.box[a];
    }
    const double len = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) e[a] = len > 0.0 ? r[a] / len : (a == 0 ? 1.0 : 0.0);
    const double ta[3] = {yP[1] * e[2] - yP[2] * e[1], yP[2] * e[0] - yP[0] * e[2], yP[0] * e[1] - yP[1] * e[0]};
    const double tb[3] = {yQ[1] * e[2] - yQ[2] * e[1], yQ[2] * e[0] - yQ[0] * e[2], yQ[0] * e[1] - yQ[1] * e[0]};
    const size_t row = (size_t)mu + b;
    double* dg = dgeom + 9 * row;
    double dtu = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dg[a] = e[a];
        dg[3 + a] = ta[a];
        dg[6 + a] = tb[a];
        dtu += e[a] * (unc[a * (size_t)np + i] - unc[a * (size_t)np + j]);
        dtu += ta[a] * unc[(3 + a) * (size_t)np + i] - tb[a] * unc[(3 + a) * (size_t)np + j];
    }
    pairs[3 * row] = i;
    pairs[3 * row + 1] = j;
    pairs[3 * row + 2] = (k[0] + 1) + 3 * (k[1] + 1) + 9 * (k[2] + 1);
    phi[row] = len;
    q[row] = (len - r0) / g.dt + dtu;
    comp64[row] = 1.0 / (g.dt * kp);
}

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }

cudaError_t launch_assemble_springs(aLENS_ctx* ctx, int n, int mu)
{
    const int nb = (int)ctx->sp_n;
    const int work = nb > mu ? nb : mu;
    if (work <= 0) return cudaSuccess;
    k_assemble_springs<<<nblk(work, 256), 256, 0, ctx->stream>>>(
        nb, n, (int)ctx->max_rods, mu, ctx->geo, ctx->cur_systab, ctx->cur_sysid, ctx->sp_ends, ctx->sp_arms,
        ctx->sp_kappa, ctx->sp_rest, ctx->xw, ctx->axis, ctx->unc, ctx->pairs, ctx->phi, ctx->dgeom, ctx->q64,
        ctx->comp64, ctx->dflags);
    ++ctx->launches;
    return cudaGetLastError();
}

cudaError_t launch_assemble(aLENS_ctx* ctx, int n, int m, const int32_t* pairs, double* phi, double* dgeom, double* q)
{
    if (m <= 0) return cudaSuccess;
    k_assemble<<<nblk(m, 256), 256, 0, ctx->stream>>>(m, n, (int)ctx->max_rods, ctx->geo, ctx->cur_systab,
                                                      ctx->cur_sysid, pairs, ctx->xw, ctx->axis, ctx->unc, phi, dgeom, q,
                                                      ctx->dcount, ctx->dflags, ctx->mdev);
    ++ctx->launches;
    return cudaGetLastError();
}

template <typename T>
static cudaError_t setup_rods_typed(aLENS_ctx* ctx, const SolveBufs<T>& sb, int n, const double* quat,
                                    const int* rank)
{
    if (n > 0) {
        k_setup_rods<T><<<nblk(n, 256), 256, 0, ctx->stream>>>(n, (int)ctx->max_rods, quat, rank, ctx->cur_systab,
                                                                ctx->cur_sysid, sb.ax, sb.mobr);
        ++ctx->launches;
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t setup_typed(aLENS_ctx* ctx, const SolveBufs<T>& sb, int n, int m, const int32_t* pairs,
                               const double* dgeom, const double* q, const double* gamma_in, const int* rank)
{
    int mp = (int)ctx->max_pairs, np = (int)ctx->max_rods;
    cudaStream_t st = ctx->stream;
    if (m <= 0) return cudaGetLastError();
    // the low-part rows serve the single-system one-barrier solver only
    const bool batch = ctx->cur_systab != nullptr && ctx->batch_n > 1;
    k_setup_fill<T><<<nblk(m, 256), 256, 0, st>>>(m, mp, ctx->perm, pairs, rank, dgeom, q, gamma_in, ctx->rowQ,
                                                  ctx->curQ, ctx->qlist, ctx->ci, ctx->cj, sb.rec, sb.q, sb.gg[0], sb.gg[1],
                                                  sb.rec_lo, sb.q_lo, ctx->cur_comp, sb.comp, np, sb.ax,
                                                  ctx->cur_systab ? sb.mobr : (const T*)nullptr, ctx->mob, ctx->scale_beta,
                                                  ctx->scale64, sb.isc, batch ? (T*)nullptr : sb.lop,
                                                  batch ? (T*)nullptr : sb.loq, ctx->mdev);
    ++ctx->launches;
    k_sort_segments<<<nblk(n, 128), 128, 0, st>>>(n, ctx->rowQ, ctx->qlist);
    ++ctx->launches;
    ctx->qe_pending = 1;   // written by launch_setup_qe where a solver or the adjoint reads it
    ctx->qe_m = m;
    ctx->qe_prec = sizeof(T) == 4 ? ALENS_MIXED : ALENS_FP64;
    return cudaGetLastError();
}

cudaError_t launch_setup_qe(aLENS_ctx* ctx)
{
    if (!ctx->qe_pending) return cudaSuccess;
    ctx->qe_pending = 0;
    const int m = ctx->qe_m, mp = (int)ctx->max_pairs;
    if (m <= 0) return cudaSuccess;
    if (ctx->qe_prec == ALENS_MIXED) {
        const SolveBufs<float>& sb = ctx->sb32;
        k_setup_qe<float><<<nblk(m, 256), 256, 0, ctx->stream>>>(m, mp, ctx->qlist, sb.rec, sb.qe, sb.rec_lo, sb.qe_lo,
                                                                  sb.pe, ctx->mdev);
    } else {
        const SolveBufs<double>& sb = ctx->sb64;
        k_setup_qe<double><<<nblk(m, 256), 256, 0, ctx->stream>>>(m, mp, ctx->qlist, sb.rec, sb.qe, sb.rec_lo,
                                                                   sb.qe_lo, sb.pe, ctx->mdev);
    }
    ++ctx->launches;
    return cudaGetLastError();
}

// Validates a caller's pair list (ranges, i < j, sorted by i).
cudaError_t launch_solve_setup_check(aLENS_ctx* ctx, int n, int m, const int32_t* pairs)
{
    if (m > 0) {
        k_check_pairs<<<nblk(m, 256), 256, 0, ctx->stream>>>(m, n, pairs, ctx->dflags);
        ++ctx->launches;
    }
    return cudaGetLastError();
}

// Owner-major constraint layout over rod ranks, the Q-side CSR, and the
// typed solver buffers.  The pair list must have passed the check.
// The solver's layout from the pair list alone (no assembled values): the
// owner-major CSR (rowP, perm in ascending order per rod), the Q-side
// counts and offsets (rowQ) and the rods' axes and drags in rank order.
cudaError_t launch_solve_layout(aLENS_ctx* ctx, int n, int m, const int32_t* pairs, const double* quat,
                                int precision, const int* rank)
{
    cudaStream_t st = ctx->stream;
    cudaError_t e;
    size_t bytes = sizeof(int) * ((size_t)n + 1);
    if ((e = cudaMemsetAsync(ctx->rod_count, 0, bytes, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ctx->cntQ, 0, bytes, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ctx->curQ, 0, bytes, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ctx->curP, 0, bytes, st)) != cudaSuccess) return e;
    if (m > 0) {
        k_count_sides<<<nblk(m, 256), 256, 0, st>>>(m, pairs, rank, ctx->rod_count, ctx->cntQ, ctx->mdev);
        ++ctx->launches;
    }
    if ((e = exclusive_scan(ctx, ctx->rod_count, ctx->rowP, n)) != cudaSuccess) return e;
    if ((e = exclusive_scan(ctx, ctx->cntQ, ctx->rowQ, n)) != cudaSuccess) return e;
    if (m > 0) {
        k_scatter_owner<<<nblk(m, 256), 256, 0, st>>>(m, pairs, rank, ctx->rowP, ctx->curP, ctx->perm, ctx->mdev);
        ++ctx->launches;
        k_sort_segments<<<nblk(n, 128), 128, 0, st>>>(n, ctx->rowP, ctx->perm);
        ++ctx->launches;
    }
    if (precision == ALENS_MIXED) return setup_rods_typed<float>(ctx, ctx->sb32, n, quat, rank);
    return setup_rods_typed<double>(ctx, ctx->sb64, n, quat, rank);
}

// The records, q and the starting state from the assembled values, on the
// layout of launch_solve_layout.
cudaError_t launch_solve_fill(aLENS_ctx* ctx, int n, int m, const int32_t* pairs, const double* dgeom,
                              const double* q, const double* gamma_in, int precision, const int* rank)
{
    ctx->qe_pending = 0;
    ctx->zero_start = gamma_in == nullptr;
    if (precision == ALENS_MIXED) return setup_typed<float>(ctx, ctx->sb32, n, m, pairs, dgeom, q, gamma_in, rank);
    return setup_typed<double>(ctx, ctx->sb64, n, m, pairs, dgeom, q, gamma_in, rank);
}

cudaError_t launch_solve_setup(aLENS_ctx* ctx, int n, int m, const int32_t* pairs, const double* dgeom,
                               const double* q, const double* gamma_in, const double* quat, int precision,
                               const int* rank)
{
    cudaError_t e = launch_solve_layout(ctx, n, m, pairs, quat, precision, rank);
    if (e != cudaSuccess) return e;
    return launch_solve_fill(ctx, n, m, pairs, dgeom, q, gamma_in, precision, rank);
}

}  // namespace alens
