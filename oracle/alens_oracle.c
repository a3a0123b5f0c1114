/*
 * Plain FP64 CPU oracle for the collision-constraint step of aLENS
 * (Yan et al., "Towards the cellular-scale simulation of motor-driven
 * cytoskeletal assemblies", arXiv 2109.08206).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code, header, table or helper
 * with the CUDA path.
 *
 * Built with -O2 -ffp-contract=off (no fused multiply-add), so every product
 * and sum is rounded on its own.  Slow and obvious on purpose:
 *   - pairs by brute force over all i < j and all 27 periodic image shifts;
 *   - closest points of two segments by enumerating the interior stationary
 *     point and the four edges of the parameter square;
 *   - the complementarity problem by active-set enumeration (tiny systems)
 *     or by accelerated projected gradient (FISTA with restart), not by the
 *     Barzilai-Borwein iteration the GPU path uses.
 *
 * Readings of passages the paper leaves open (they are parameters or fixed
 * rules on both sides):
 *   R1 drag: zeta_perp = 4 pi eta L / ln(2L/D) (the coefficient the paper
 *      quotes in Section 3 "Filament dynamics"), zeta_par = zeta_perp / 2,
 *      zeta_rot = zeta_perp L^2 / 12, zeta_spin = pi eta D^2 L.
 *   R2 L is the cylinder length (caps excluded).
 *   R3 Phi is the surface gap |r| - D; a pair is kept iff Phi < delta_c.
 *   R4 parallel segments (det <= 1e-12 a c) whose projections overlap take
 *      s* at the middle of the overlap and t* as its clamped projection;
 *      touching centrelines take e = unit(p_i x p_j) turned so e.dx >= 0,
 *      or, for collinear axes, e = sign(dx.p_i) p_i, or e_x.
 *   R5 every image shift k in {-1,0,1}^3 with |dx| < L + D + delta_c is its
 *      own constraint, keyed (i, j, code), code = (kx+1)+3(ky+1)+9(kz+1),
 *      dx = x_i - x_j - k*box.
 *   R6 residual r = (h/D) max_c |pi_c|, pi_c = g_c if gamma_c > 0 else
 *      min(g_c, 0), g = D^T M D gamma + q (projected gradient, in rod
 *      diameters of linearised gap).
 *   R7 quaternions (s, v), body axis e_z, lab-frame angular velocity,
 *      linear update then renormalisation.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_API __attribute__((visibility("default")))

typedef struct {
    double box[3];
    double diameter;
    double length;
    double viscosity;
    double dt;
    double delta_c;
} orc_problem;

/* ---------------------------------------------------------------- helpers */

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double* a, const double* b, double* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Drag coefficients (reading R1).  Section 3 quotes 4 pi eta L / log(2L/D). */
/* Threads of the parallel loops (timing the CPU baseline on one core and
 * on all of them); returns the count in force before the call.  No effect
 * without OpenMP. */
ORC_API int orc_set_threads(int n)
{
#ifdef _OPENMP
    const int before = omp_get_max_threads();
    if (n > 0) omp_set_num_threads(n);
    return before;
#else
    (void)n;
    return 1;
#endif
}

ORC_API void orc_drag(double eta, double L, double D, double out[4])
{
    double zperp = 4.0 * M_PI * eta * L / log(2.0 * L / D);
    out[0] = zperp;                 /* perpendicular translation */
    out[1] = zperp / 2.0;           /* parallel translation */
    out[2] = zperp * L * L / 12.0;  /* rotation about an axis normal to the rod */
    out[3] = M_PI * eta * D * D * L;/* spin about the rod axis */
}

/* Rod axis p = R(theta) e_z for unit quaternion theta = (s, v): third column of
 * the rotation matrix the quaternion generates (Appendix "Symmetry of the
 * geometrically constrained optimization problem", y = R Y). */
ORC_API void orc_axis(int64_t n, const double* quat, double* axis)
{
    for (int64_t i = 0; i < n; ++i) {
        const double* q = quat + 4 * i;
        double s = q[0], a = q[1], b = q[2], c = q[3];
        axis[3 * i + 0] = 2.0 * (a * c + s * b);
        axis[3 * i + 1] = 2.0 * (b * c - s * a);
        axis[3 * i + 2] = s * s - a * a - b * b + c * c;
    }
}

/* Wrap a coordinate into [0, box). */
static double wrap1(double v, double b)
{
    double w = v - b * floor(v / b);
    if (w >= b) w = 0.0;
    if (w < 0.0) w = 0.0;
    return w;
}

ORC_API void orc_wrap(int64_t n, const double* x, const double box[3], double* xw)
{
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) xw[3 * i + k] = wrap1(x[3 * i + k], box[k]);
}

/* |dx + s p - t q|^2 */
static double seg_f(const double* dx, const double* p, const double* q, double s, double t)
{
    double r0 = dx[0] + s * p[0] - t * q[0];
    double r1 = dx[1] + s * p[1] - t * q[1];
    double r2 = dx[2] + s * p[2] - t * q[2];
    return r0 * r0 + r1 * r1 + r2 * r2;
}

/* Closest points of segments P = {s p : |s| <= L/2} and Q = {dx' + t q} where
 * the offset between centres is dx = x_P - x_Q (Appendix Fig. "pairwise
 * geometry": r = x_P + y_P - x_Q - y_Q with y_P = s p, y_Q = t q).
 * Minimises f(s, t) = |dx + s p - t q|^2 over [-L/2, L/2]^2 by checking the
 * interior stationary point and then the minimum on each of the four edges
 * (each a clamped one-dimensional projection).  Reading R4 for parallel
 * segments.  Returns |r| at the minimiser. */
ORC_API double orc_segment_closest(const double* dx, const double* p, const double* q, double L,
                                   double* s_out, double* t_out)
{
    const double hl = 0.5 * L;
    double a = dot3(p, p), b = dot3(p, q), c = dot3(q, q);
    double d = dot3(p, dx), e = dot3(q, dx);
    double det = a * c - b * b;
    if (det > 1e-12 * a * c) {
        double s0 = (b * e - c * d) / det;
        double t0 = (a * e - b * d) / det;
        if (fabs(s0) <= hl && fabs(t0) <= hl) {
            *s_out = s0; *t_out = t0;
            return sqrt(seg_f(dx, p, q, s0, t0));
        }
    } else {
        /* parallel: points of Q project onto P's axis at s = (b t - d)/a */
        double e1 = (b * (-hl) - d) / a, e2 = (b * hl - d) / a;
        double lo = e1 < e2 ? e1 : e2, hi = e1 < e2 ? e2 : e1;
        if (lo < -hl) lo = -hl;
        if (hi > hl) hi = hl;
        if (lo <= hi) {
            double s0 = 0.5 * (lo + hi);
            double t0 = clampd((b * s0 + e) / c, -hl, hl);
            *s_out = s0; *t_out = t0;
            return sqrt(seg_f(dx, p, q, s0, t0));
        }
    }
    /* the four edges of the parameter square */
    double best = INFINITY, bs = 0.0, bt = 0.0;
    for (int edge = 0; edge < 4; ++edge) {
        double s, t;
        if (edge < 2) {
            s = edge == 0 ? -hl : hl;
            t = clampd((b * s + e) / c, -hl, hl);
        } else {
            t = edge == 2 ? -hl : hl;
            s = clampd((b * t - d) / a, -hl, hl);
        }
        double f = seg_f(dx, p, q, s, t);
        if (f < best) { best = f; bs = s; bt = t; }
    }
    *s_out = bs; *t_out = bt;
    return sqrt(best);
}

/* Unit normal e for a pair given r (Appendix: e_P = r/|r| = -e_Q), with the
 * reading R4 when |r| = 0. */
static void pair_normal(const double* r, double dist, const double* dx, const double* p, const double* q,
                        double* e)
{
    if (dist > 0.0) {
        e[0] = r[0] / dist; e[1] = r[1] / dist; e[2] = r[2] / dist;
        return;
    }
    double n[3];
    cross3(p, q, n);
    double nn = sqrt(dot3(n, n));
    if (nn > 1e-12) {
        double sg = dot3(n, dx) < 0.0 ? -1.0 : 1.0;
        e[0] = sg * n[0] / nn; e[1] = sg * n[1] / nn; e[2] = sg * n[2] / nn;
        return;
    }
    double pd = dot3(p, dx);
    if (pd != 0.0) {
        double sg = pd < 0.0 ? -1.0 : 1.0;
        double pn = sqrt(dot3(p, p));
        e[0] = sg * p[0] / pn; e[1] = sg * p[1] / pn; e[2] = sg * p[2] / pn;
        return;
    }
    e[0] = 1.0; e[1] = 0.0; e[2] = 0.0;
}

static void image_shift(int code, int k[3])
{
    k[0] = code % 3 - 1;
    k[1] = (code / 3) % 3 - 1;
    k[2] = code / 9 - 1;
}

/* ------------------------------------------------------------------ pairs */

/* Surface gap of pair (i, j) at image code: Phi = |r| - D (reading R3).
 * Returns 0 and leaves *gap untouched when the centre distance is not below
 * L + D + delta_c (no segment point can then be within delta_c). */
static int pair_gap(const double* xw, const double* axis, const orc_problem* pb, int64_t i, int64_t j,
                    int code, double* gap, double* s, double* t, double* dx)
{
    int k[3];
    image_shift(code, k);
    for (int c = 0; c < 3; ++c) dx[c] = xw[3 * i + c] - xw[3 * j + c] - (double)k[c] * pb->box[c];
    double rcut = pb->length + pb->diameter + pb->delta_c;
    if (dot3(dx, dx) >= rcut * rcut) return 0;
    double d = orc_segment_closest(dx, axis + 3 * i, axis + 3 * j, pb->length, s, t);
    *gap = d - pb->diameter;
    return 1;
}

/* All pairs (i < j, image) whose surface gap is below delta_c, in (i, j, code)
 * order (Appendix "Implementation": close pairs whose minimal distance is
 * below delta_c).  Writes at most cap pairs (int32 triples) and returns the
 * full count. */
ORC_API int64_t orc_find_pairs(int64_t n, const double* x, const double* quat, const orc_problem* pb,
                               int32_t* pairs, int64_t cap)
{
    double* xw = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double* axis = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    orc_wrap(n, x, pb->box, xw);
    orc_axis(n, quat, axis);
    int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    /* pass 1: count per i */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0;
        for (int64_t j = i + 1; j < n; ++j)
            for (int code = 0; code < 27; ++code) {
                double gap, s, t, dx[3];
                if (pair_gap(xw, axis, pb, i, j, code, &gap, &s, &t, dx) && gap < pb->delta_c) ++c;
            }
        cnt[i + 1] = c;
    }
    for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    int64_t total = cnt[n];
    if (total <= cap && pairs) {
        /* pass 2: write, each i into its own slot range */
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t i = 0; i < n; ++i) {
            int64_t o = cnt[i];
            for (int64_t j = i + 1; j < n; ++j)
                for (int code = 0; code < 27; ++code) {
                    double gap, s, t, dx[3];
                    if (pair_gap(xw, axis, pb, i, j, code, &gap, &s, &t, dx) && gap < pb->delta_c) {
                        pairs[3 * o + 0] = (int32_t)i;
                        pairs[3 * o + 1] = (int32_t)j;
                        pairs[3 * o + 2] = code;
                        ++o;
                    }
                }
        }
    }
    free(cnt); free(xw); free(axis);
    return total;
}

static int cmp_triple(const void* a, const void* b)
{
    const int32_t* u = (const int32_t*)a;
    const int32_t* v = (const int32_t*)b;
    for (int k = 0; k < 3; ++k)
        if (u[k] != v[k]) return u[k] < v[k] ? -1 : 1;
    return 0;
}

/* The pairs of the full list that involve at least one rod of rows[0..nrows):
 * for every listed rod r and every other rod j, each image of the pair is
 * tested in the canonical orientation (min(r,j), max(r,j)); when r > j the
 * image shift is negated (code -> 26 - code).  Sorted, duplicates removed.
 * Returns the count; writes at most cap triples. */
ORC_API int64_t orc_find_pairs_rows(int64_t n, const double* x, const double* quat, const orc_problem* pb,
                                    const int64_t* rows, int64_t nrows, int32_t* pairs, int64_t cap)
{
    double* xw = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double* axis = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    orc_wrap(n, x, pb->box, xw);
    orc_axis(n, quat, axis);
    /* one growable buffer per listed rod, filled in parallel, then joined */
    int32_t** bufs = (int32_t**)calloc((size_t)(nrows > 0 ? nrows : 1), sizeof(int32_t*));
    int64_t* used = (int64_t*)calloc((size_t)(nrows > 0 ? nrows : 1), sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t a = rows[r], room = 64, u = 0;
        int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)room);
        for (int64_t j = 0; j < n; ++j) {
            if (j == a) continue;
            int64_t i = a < j ? a : j, jj = a < j ? j : a;
            for (int code = 0; code < 27; ++code) {
                double gap, s, t, dx[3];
                if (pair_gap(xw, axis, pb, i, jj, code, &gap, &s, &t, dx) && gap < pb->delta_c) {
                    if (u == room) {
                        room *= 2;
                        buf = (int32_t*)realloc(buf, sizeof(int32_t) * 3 * (size_t)room);
                    }
                    buf[3 * u] = (int32_t)i; buf[3 * u + 1] = (int32_t)jj; buf[3 * u + 2] = code;
                    ++u;
                }
            }
        }
        bufs[r] = buf;
        used[r] = u;
    }
    int64_t total = 0;
    for (int64_t r = 0; r < nrows; ++r) total += used[r];
    int32_t* all = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(total > 0 ? total : 1));
    int64_t o = 0;
    for (int64_t r = 0; r < nrows; ++r) {
        memcpy(all + 3 * o, bufs[r], sizeof(int32_t) * 3 * (size_t)used[r]);
        o += used[r];
        free(bufs[r]);
    }
    qsort(all, (size_t)total, 3 * sizeof(int32_t), cmp_triple);
    int64_t u = 0;
    for (int64_t k = 0; k < total; ++k) {
        if (u > 0 && cmp_triple(all + 3 * k, all + 3 * (u - 1)) == 0) continue;
        if (u != k) memcpy(all + 3 * u, all + 3 * k, 3 * sizeof(int32_t));
        ++u;
    }
    if (pairs && u <= cap) memcpy(pairs, all, sizeof(int32_t) * 3 * (size_t)u);
    free(all); free(bufs); free(used); free(xw); free(axis);
    return u;
}

/* Surface gaps of given pairs (for near-threshold accounting in tests). */
ORC_API void orc_pair_gaps(int64_t n, const double* x, const double* quat, const orc_problem* pb,
                           int64_t npairs, const int32_t* pairs, double* gap_out)
{
    double* xw = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double* axis = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    orc_wrap(n, x, pb->box, xw);
    orc_axis(n, quat, axis);
    for (int64_t c = 0; c < npairs; ++c) {
        int k[3];
        image_shift(pairs[3 * c + 2], k);
        int64_t i = pairs[3 * c], j = pairs[3 * c + 1];
        double dx[3], s, t;
        for (int m = 0; m < 3; ++m) dx[m] = xw[3 * i + m] - xw[3 * j + m] - (double)k[m] * pb->box[m];
        gap_out[c] = orc_segment_closest(dx, axis + 3 * i, axis + 3 * j, pb->length, &s, &t) - pb->diameter;
    }
    free(xw); free(axis);
}

/* --------------------------------------------------------------- mobility */

/* U = M F for one rod (Eq. U = M F, Appendix "Constraint quadratic
 * programming"; M block-diagonal 6x6, reading R1):
 *   U_t = (p p^T)/zeta_par F + (I - p p^T)/zeta_perp F
 *   W   = (p p^T)/zeta_spin T + (I - p p^T)/zeta_rot T                    */
static void mobility_rod(const double* p, const double* zeta, const double* F, double* U)
{
    double pf = dot3(p, F), pt = dot3(p, F + 3);
    for (int k = 0; k < 3; ++k) {
        double fpar = pf * p[k], tpar = pt * p[k];
        U[k] = fpar / zeta[1] + (F[k] - fpar) / zeta[0];
        U[3 + k] = tpar / zeta[3] + (F[3 + k] - tpar) / zeta[2];
    }
}

ORC_API void orc_mobility_apply(int64_t n, const double* quat, const orc_problem* pb, const double* F,
                                double* U)
{
    double zeta[4];
    orc_drag(pb->viscosity, pb->length, pb->diameter, zeta);
    double* axis = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    orc_axis(n, quat, axis);
#pragma omp parallel for
    for (int64_t i = 0; i < n; ++i) mobility_rod(axis + 3 * i, zeta, F + 6 * i, U + 6 * i);
    free(axis);
}

/* --------------------------------------------------------------- assembly */

/* Per pair: Phi, the D column and q (Appendix Eq. blockdef A, and the column
 * D_PQ = [e_P, y_P x e_P, e_Q, y_Q x e_Q] with e_Q = -e_P).
 * dgeom[c] = (e[3], y_P x e[3], y_Q x e[3]); the column acting on rod Q is
 * (-e, -(y_Q x e)).  q_c = Phi_c / h + D_c^T M F_nc. */
ORC_API void orc_assemble(int64_t n, const double* x, const double* quat, const double* fnc,
                          const orc_problem* pb, int64_t npairs, const int32_t* pairs, double* phi,
                          double* dgeom, double* q, double* yp_out, double* yq_out)
{
    double zeta[4];
    orc_drag(pb->viscosity, pb->length, pb->diameter, zeta);
    double* xw = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double* axis = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double* unc = (double*)malloc(sizeof(double) * 6 * (size_t)(n > 0 ? n : 1));
    orc_wrap(n, x, pb->box, xw);
    orc_axis(n, quat, axis);
    for (int64_t i = 0; i < n; ++i) mobility_rod(axis + 3 * i, zeta, fnc + 6 * i, unc + 6 * i);
#pragma omp parallel for
    for (int64_t c = 0; c < npairs; ++c) {
        int64_t i = pairs[3 * c], j = pairs[3 * c + 1];
        int k[3];
        image_shift(pairs[3 * c + 2], k);
        double dx[3], s, t;
        for (int m = 0; m < 3; ++m) dx[m] = xw[3 * i + m] - xw[3 * j + m] - (double)k[m] * pb->box[m];
        const double* pi_ = axis + 3 * i;
        const double* pj_ = axis + 3 * j;
        double dist = orc_segment_closest(dx, pi_, pj_, pb->length, &s, &t);
        double yP[3], yQ[3], r[3], e[3];
        for (int m = 0; m < 3; ++m) {
            yP[m] = s * pi_[m];
            yQ[m] = t * pj_[m];
            r[m] = dx[m] + yP[m] - yQ[m];
        }
        pair_normal(r, dist, dx, pi_, pj_, e);
        double* dg = dgeom + 9 * c;
        dg[0] = e[0]; dg[1] = e[1]; dg[2] = e[2];
        cross3(yP, e, dg + 3);
        cross3(yQ, e, dg + 6);
        phi[c] = dist - pb->diameter;
        const double* ui = unc + 6 * i;
        const double* uj = unc + 6 * j;
        double dtu = dot3(e, ui) + dot3(dg + 3, ui + 3) - dot3(e, uj) - dot3(dg + 6, uj + 3);
        q[c] = phi[c] / pb->dt + dtu;
        if (yp_out) { yp_out[3 * c] = yP[0]; yp_out[3 * c + 1] = yP[1]; yp_out[3 * c + 2] = yP[2]; }
        if (yq_out) { yq_out[3 * c] = yQ[0]; yq_out[3 * c + 1] = yQ[1]; yq_out[3 * c + 2] = yQ[2]; }
    }
    free(xw); free(axis); free(unc);
}

/* Bilateral (spring) constraints (Appendix: Phi_b is the distance between
 * two fixed points of particles P and Q, K [Phi_b - Phi_b^0] = -gamma_b;
 * Eqs. linearconstraints b and blockdef D, F).  Spring b joins the point at
 * arclength arms[b][0] on rod ends[b][0] (P) to arclength arms[b][1] on rod
 * ends[b][1] (Q): r = x_P + s_P p_P - x_Q - s_Q p_Q over the minimum periodic
 * image of the two points, Phi_b = |r|, e = r / |r|, and the D column is
 * (e, y_P x e | -e, -(y_Q x e)) with y = s p, exactly as for a collision.
 * Outputs per spring: pairs (P, Q, image code), dgeom, q = (Phi_b -
 * rest)/h + D^T M F_nc, the length Phi_b and comp = 1/(h kappa). */
ORC_API void orc_assemble_springs(int64_t n, const double* x, const double* quat, const double* fnc,
                                  const orc_problem* pb, int64_t nb, const int32_t* ends, const double* arms,
                                  const double* kappa, const double* rest, int32_t* pairs, double* dgeom,
                                  double* q, double* length, double* comp)
{
    double zeta[4];
    orc_drag(pb->viscosity, pb->length, pb->diameter, zeta);
    size_t nn = (size_t)(n > 0 ? n : 1);
    double* xw = (double*)malloc(sizeof(double) * 3 * nn);
    double* axis = (double*)malloc(sizeof(double) * 3 * nn);
    orc_wrap(n, x, pb->box, xw);
    orc_axis(n, quat, axis);
    for (int64_t b = 0; b < nb; ++b) {
        int64_t i = ends[2 * b], j = ends[2 * b + 1];
        const double *pi_ = axis + 3 * i, *pj_ = axis + 3 * j;
        double yP[3], yQ[3], r[3], e[3];
        int k[3];
        for (int m = 0; m < 3; ++m) {
            yP[m] = arms[2 * b] * pi_[m];
            yQ[m] = arms[2 * b + 1] * pj_[m];
            double d = xw[3 * i + m] + yP[m] - xw[3 * j + m] - yQ[m];
            k[m] = (int)nearbyint(d / pb->box[m]);
            if (k[m] > 1) k[m] = 1;
            if (k[m] < -1) k[m] = -1;
            r[m] = d - (double)k[m] * pb->box[m];
        }
        double len = sqrt(dot3(r, r));
        for (int m = 0; m < 3; ++m) e[m] = len > 0.0 ? r[m] / len : (m == 0 ? 1.0 : 0.0);
        pairs[3 * b] = (int32_t)i;
        pairs[3 * b + 1] = (int32_t)j;
        pairs[3 * b + 2] = (int32_t)((k[0] + 1) + 3 * (k[1] + 1) + 9 * (k[2] + 1));
        double* dg = dgeom + 9 * b;
        dg[0] = e[0]; dg[1] = e[1]; dg[2] = e[2];
        cross3(yP, e, dg + 3);
        cross3(yQ, e, dg + 6);
        double ui[6], uj[6];
        mobility_rod(pi_, zeta, fnc + 6 * i, ui);
        mobility_rod(pj_, zeta, fnc + 6 * j, uj);
        double dtu = dot3(e, ui) + dot3(dg + 3, ui + 3) - dot3(e, uj) - dot3(dg + 6, uj + 3);
        length[b] = len;
        q[b] = (len - rest[b]) / pb->dt + dtu;
        comp[b] = 1.0 / (pb->dt * kappa[b]);
    }
    free(xw); free(axis);
}

/* F = D gamma: force and torque on every rod (Eq. dmap F_u = D_u gamma_u). */
ORC_API void orc_apply_D(int64_t n, int64_t npairs, const int32_t* pairs, const double* dgeom,
                         const double* gamma, double* F)
{
    memset(F, 0, sizeof(double) * 6 * (size_t)n);
    for (int64_t c = 0; c < npairs; ++c) {
        int64_t i = pairs[3 * c], j = pairs[3 * c + 1];
        const double* dg = dgeom + 9 * c;
        double g = gamma[c];
        for (int m = 0; m < 3; ++m) {
            F[6 * i + m] += g * dg[m];
            F[6 * i + 3 + m] += g * dg[3 + m];
            if (j < 0) continue;   /* a wall: one-sided column */
            F[6 * j + m] -= g * dg[m];
            F[6 * j + 3 + m] -= g * dg[6 + m];
        }
    }
}

/* out = D^T U */
ORC_API void orc_apply_Dt(int64_t npairs, const int32_t* pairs, const double* dgeom, const double* U,
                          double* out)
{
#pragma omp parallel for
    for (int64_t c = 0; c < npairs; ++c) {
        int64_t i = pairs[3 * c], j = pairs[3 * c + 1];
        const double* dg = dgeom + 9 * c;
        out[c] = dot3(dg, U + 6 * i) + dot3(dg + 3, U + 6 * i + 3);
        if (j >= 0) out[c] -= dot3(dg, U + 6 * j) + dot3(dg + 6, U + 6 * j + 3);
    }
}

/* ------------------------------------------------------------------ solve */

typedef struct {
    int64_t n, npairs;
    const int32_t* pairs;
    const double* dgeom;
    const double* q;
    const double* comp;   /* NULL, or per constraint: < 0 unilateral, >= 0 bilateral compliance 1/(h kappa) */
    double* axis;
    double zeta[4];
    double* F;   /* 6n scratch */
    double* U;   /* 6n scratch */
} orc_qp;

static int is_bilateral(const orc_qp* qp, int64_t c) { return qp->comp && qp->comp[c] >= 0.0; }

/* out = (D^T M D + diag(0, K^{-1}/h)) v   (Eq. blockdef B, C, E, F) */
static void qp_matvec(orc_qp* qp, const double* v, double* out)
{
    orc_apply_D(qp->n, qp->npairs, qp->pairs, qp->dgeom, v, qp->F);
#pragma omp parallel for
    for (int64_t i = 0; i < qp->n; ++i) mobility_rod(qp->axis + 3 * i, qp->zeta, qp->F + 6 * i, qp->U + 6 * i);
    orc_apply_Dt(qp->npairs, qp->pairs, qp->dgeom, qp->U, out);
    if (qp->comp)
        for (int64_t c = 0; c < qp->npairs; ++c)
            if (qp->comp[c] >= 0.0) out[c] += qp->comp[c] * v[c];
}

static double qp_residual(const orc_qp* qp, const double* gamma, const double* g, const orc_problem* pb)
{
    double m = 0.0;
    for (int64_t c = 0; c < qp->npairs; ++c) {
        /* bilateral entries are free: their projected gradient is g */
        double pg = (gamma[c] > 0.0 || is_bilateral(qp, c)) ? g[c] : (g[c] < 0.0 ? g[c] : 0.0);
        double a = fabs(pg);
        if (a > m) m = a;
    }
    return pb->dt / pb->diameter * m;
}

static int qp_init(orc_qp* qp, int64_t n, const double* quat, const orc_problem* pb, int64_t npairs,
                   const int32_t* pairs, const double* dgeom, const double* q, const double* comp)
{
    qp->n = n; qp->npairs = npairs; qp->pairs = pairs; qp->dgeom = dgeom; qp->q = q; qp->comp = comp;
    orc_drag(pb->viscosity, pb->length, pb->diameter, qp->zeta);
    size_t nn = (size_t)(n > 0 ? n : 1);
    qp->axis = (double*)malloc(sizeof(double) * 3 * nn);
    qp->F = (double*)malloc(sizeof(double) * 6 * nn);
    qp->U = (double*)malloc(sizeof(double) * 6 * nn);
    orc_axis(n, quat, qp->axis);
    return 0;
}

static void qp_free(orc_qp* qp) { free(qp->axis); free(qp->F); free(qp->U); }

/* g = D^T M D gamma + q and the residual (reading R6). */
ORC_API double orc_gradient(int64_t n, const double* quat, const orc_problem* pb, int64_t npairs,
                            const int32_t* pairs, const double* dgeom, const double* q, const double* comp,
                            const double* gamma, double* g)
{
    orc_qp qp;
    qp_init(&qp, n, quat, pb, npairs, pairs, dgeom, q, comp);
    qp_matvec(&qp, gamma, g);
    for (int64_t c = 0; c < npairs; ++c) g[c] += q[c];
    double r = qp_residual(&qp, gamma, g, pb);
    qp_free(&qp);
    return r;
}

/* Dense A = D^T M D for small problems (column c = A e_c). */
ORC_API void orc_dense_A(int64_t n, const double* quat, const orc_problem* pb, int64_t npairs,
                         const int32_t* pairs, const double* dgeom, const double* comp, double* A)
{
    orc_qp qp;
    qp_init(&qp, n, quat, pb, npairs, pairs, dgeom, NULL, comp);
    double* ec = (double*)calloc((size_t)npairs, sizeof(double));
    double* col = (double*)malloc(sizeof(double) * (size_t)npairs);
    for (int64_t c = 0; c < npairs; ++c) {
        ec[c] = 1.0;
        qp_matvec(&qp, ec, col);
        ec[c] = 0.0;
        for (int64_t r = 0; r < npairs; ++r) A[r * npairs + c] = col[r];
    }
    free(ec); free(col);
    qp_free(&qp);
}

/* Solve A_SS x = b by Gaussian elimination with partial pivoting; returns 0
 * if a pivot falls below tiny (singular), 1 otherwise. */
static int small_solve(int m, double* A, double* b, double tiny)
{
    for (int k = 0; k < m; ++k) {
        int piv = k;
        for (int r = k + 1; r < m; ++r)
            if (fabs(A[r * m + k]) > fabs(A[piv * m + k])) piv = r;
        if (fabs(A[piv * m + k]) <= tiny) return 0;
        if (piv != k) {
            for (int c = 0; c < m; ++c) { double t = A[k * m + c]; A[k * m + c] = A[piv * m + c]; A[piv * m + c] = t; }
            double t = b[k]; b[k] = b[piv]; b[piv] = t;
        }
        for (int r = k + 1; r < m; ++r) {
            double f = A[r * m + k] / A[k * m + k];
            for (int c = k; c < m; ++c) A[r * m + c] -= f * A[k * m + c];
            b[r] -= f * b[k];
        }
    }
    for (int k = m - 1; k >= 0; --k) {
        double s = b[k];
        for (int c = k + 1; c < m; ++c) s -= A[k * m + c] * b[c];
        b[k] = s / A[k * m + k];
    }
    return 1;
}

/* Exact solution of the CQP (Eq. suppcqpdef) for tiny problems by
 * enumerating active sets: for every subset S that contains every bilateral
 * constraint, solve A_SS gamma_S = -q_S and accept the first subset whose
 * KKT conditions hold (gamma_S >= 0 on its unilateral entries, g_c >= 0 off
 * S).  A solution with a non-singular A_SS always exists for an SPSD A.
 * Returns the accepted subset's bitmask, or -1. */
ORC_API int64_t orc_solve_enum(int64_t n, const double* quat, const orc_problem* pb, int64_t npairs,
                               const int32_t* pairs, const double* dgeom, const double* q, const double* comp,
                               double* gamma)
{
    if (npairs > 20) return -1;
    int m = (int)npairs;
    int64_t must = 0;
    for (int c = 0; c < m; ++c)
        if (comp && comp[c] >= 0.0) must |= (int64_t)1 << c;
    double* A = (double*)malloc(sizeof(double) * (size_t)(m * m + 1));
    orc_dense_A(n, quat, pb, npairs, pairs, dgeom, comp, A);
    double amax = 0.0, qmax = 0.0;
    for (int c = 0; c < m; ++c) {
        if (A[c * m + c] > amax) amax = A[c * m + c];
        if (fabs(q[c]) > qmax) qmax = fabs(q[c]);
    }
    double* sub = (double*)malloc(sizeof(double) * (size_t)(m * m + 1));
    double* rhs = (double*)malloc(sizeof(double) * (size_t)(m + 1));
    int idx[32];
    int64_t found = -1;
    for (int64_t mask = 0; mask < ((int64_t)1 << m) && found < 0; ++mask) {
        if ((mask & must) != must) continue;
        int k = 0;
        for (int c = 0; c < m; ++c) if (mask >> c & 1) idx[k++] = c;
        for (int r = 0; r < k; ++r) {
            for (int c = 0; c < k; ++c) sub[r * k + c] = A[idx[r] * m + idx[c]];
            rhs[r] = -q[idx[r]];
        }
        if (k > 0 && !small_solve(k, sub, rhs, 1e-10 * amax)) continue;
        int ok = 1;
        for (int r = 0; r < k; ++r)
            if (!(must >> idx[r] & 1) && rhs[r] < -1e-12 * (1.0 + qmax / (amax > 0 ? amax : 1.0))) { ok = 0; break; }
        if (!ok) continue;
        for (int c = 0; c < m; ++c) gamma[c] = 0.0;
        for (int r = 0; r < k; ++r) gamma[idx[r]] = (must >> idx[r] & 1) ? rhs[r] : (rhs[r] > 0.0 ? rhs[r] : 0.0);
        for (int c = 0; c < m && ok; ++c) {
            if (mask >> c & 1) continue;
            double g = q[c];
            for (int r = 0; r < m; ++r) g += A[c * m + r] * gamma[r];
            if (g < -1e-9 * (1.0 + qmax)) ok = 0;
        }
        if (ok) found = mask;
    }
    free(A); free(sub); free(rhs);
    return found;
}

/* Accelerated projected gradient (FISTA, Beck & Teboulle 2009) with the
 * gradient restart of O'Donoghue & Candes 2015 on the CQP
 *   min 1/2 gamma^T A gamma + q^T gamma,  gamma >= 0,  A = D^T M D
 * (Eq. suppcqpdef; the paper solves it with BBPGD, the GPU path does too;
 * the oracle uses a different method that converges to the same KKT point).
 * Step 1/Lip with Lip = 1.1 x the power-iteration estimate of lambda_max(A).
 * Stops when the residual (reading R6) is <= tol or after max_iter
 * iterations; the residual is evaluated every 10 iterations.
 * gamma holds the start on entry (negative entries are projected to 0) and
 * the result on exit.  Returns the final residual; *iters gets the count. */
ORC_API double orc_solve_apgd(int64_t n, const double* quat, const orc_problem* pb, int64_t npairs,
                              const int32_t* pairs, const double* dgeom, const double* q, const double* comp,
                              double* gamma, double tol, int64_t max_iter, int64_t* iters)
{
    orc_qp qp;
    qp_init(&qp, n, quat, pb, npairs, pairs, dgeom, q, comp);
    size_t m = (size_t)(npairs > 0 ? npairs : 1);
    double* v = (double*)malloc(sizeof(double) * m);
    double* w = (double*)malloc(sizeof(double) * m);
    double* z = (double*)malloc(sizeof(double) * m);
    double* gz = (double*)malloc(sizeof(double) * m);
    double* gn = (double*)malloc(sizeof(double) * m);
    /* power iteration for lambda_max */
    for (int64_t c = 0; c < npairs; ++c) v[c] = 1.0 + 0.25 * (double)((c * 7919) % 13) / 13.0;
    double lam = 0.0;
    for (int it = 0; it < 200 && npairs > 0; ++it) {
        double nv = 0.0;
        for (int64_t c = 0; c < npairs; ++c) nv += v[c] * v[c];
        nv = sqrt(nv);
        if (nv == 0.0) break;
        for (int64_t c = 0; c < npairs; ++c) v[c] /= nv;
        qp_matvec(&qp, v, w);
        double rq = 0.0;
        for (int64_t c = 0; c < npairs; ++c) rq += v[c] * w[c];
        lam = rq;
        memcpy(v, w, sizeof(double) * (size_t)npairs);
    }
    double lip = 1.1 * lam;
    if (!(lip > 0.0)) lip = 1.0;
    for (int64_t c = 0; c < npairs; ++c) {
        if (!(gamma[c] > 0.0) && !is_bilateral(&qp, c)) gamma[c] = 0.0;
        z[c] = gamma[c];
    }
    double t = 1.0, res = INFINITY;
    int64_t it = 0;
    for (;;) {
        if (it % 10 == 0) {
            qp_matvec(&qp, gamma, gn);
            for (int64_t c = 0; c < npairs; ++c) gn[c] += q[c];
            res = qp_residual(&qp, gamma, gn, pb);
            if (res <= tol || it >= max_iter) break;
        }
        qp_matvec(&qp, z, gz);
        for (int64_t c = 0; c < npairs; ++c) gz[c] += q[c];
        double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        double restart = 0.0;
        for (int64_t c = 0; c < npairs; ++c) {
            double gnew = z[c] - gz[c] / lip;
            if (gnew < 0.0 && !is_bilateral(&qp, c)) gnew = 0.0;   /* projection on the unilateral block only */
            w[c] = gnew;
            restart += gz[c] * (gnew - gamma[c]);
        }
        double beta = (t - 1.0) / tn;
        if (restart > 0.0) { tn = 1.0; beta = 0.0; }
        for (int64_t c = 0; c < npairs; ++c) {
            z[c] = w[c] + beta * (w[c] - gamma[c]);
            gamma[c] = w[c];
        }
        t = tn;
        ++it;
    }
    if (iters) *iters = it;
    free(v); free(w); free(z); free(gz); free(gn);
    qp_free(&qp);
    return res;
}

/* -------------------------------------------------------- Brownian forces */

/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11, "Parallel random
 * numbers: as easy as 1, 2, 3"): ten rounds of two 32x32->64 multiplications
 * (multipliers 0xD2511F53 and 0xCD9E8D57) whose high halves are mixed with
 * the other counter words and the key; the key is bumped by the Weyl
 * constants 0x9E3779B9 and 0xBB67AE85 between rounds. */
ORC_API void orc_philox4x32(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Six standard normals for rod i at step k from seed: Philox with key =
 * (seed low, seed high) and counters (i, k low, k high, w) for w = 0, 1;
 * each word gives u = (x + 0.5) 2^-32 in (0, 1) and each pair (u1, u2) two
 * normals by Box-Muller: sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2). */
ORC_API void orc_normals6(uint64_t seed, uint64_t step, int64_t i, double z[6])
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    double u[8];
    for (int w = 0; w < 2; ++w) {
        const uint32_t ctr[4] = {(uint32_t)i, (uint32_t)step, (uint32_t)(step >> 32), (uint32_t)w};
        uint32_t o[4];
        orc_philox4x32(ctr, key, o);
        for (int k = 0; k < 4; ++k) u[4 * w + k] = ((double)o[k] + 0.5) * (1.0 / 4294967296.0);
    }
    for (int k = 0; k < 3; ++k) {
        const double r = sqrt(-2.0 * log(u[2 * k]));
        z[2 * k] = r * cos(2.0 * M_PI * u[2 * k + 1]);
        z[2 * k + 1] = r * sin(2.0 * M_PI * u[2 * k + 1]);
    }
}

/* Brownian force and torque of every rod at step k, consistent with the
 * mobility (fluctuation-dissipation: covariance 2 kT M^-1 / h per rod):
 *   F = sqrt(2 kT / h) [sqrt(zeta_par) (p.xi) p + sqrt(zeta_perp) (xi - (p.xi) p)],
 *   T = sqrt(2 kT / h) [sqrt(zeta_spin) (p.chi) p + sqrt(zeta_rot) (chi - (p.chi) p)],
 * xi, chi = the six normals of (seed, k, i); added to f_ext (nullable) into out. */
ORC_API void orc_brownian(int64_t n, const double* quat, const orc_problem* pb, double kT, uint64_t seed,
                          uint64_t step, const double* f_ext, double* out)
{
    double zeta[4];
    orc_drag(pb->viscosity, pb->length, pb->diameter, zeta);
    double* axis = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    orc_axis(n, quat, axis);
    const double a = sqrt(2.0 * kT / pb->dt);
    for (int64_t i = 0; i < n; ++i) {
        double z[6];
        orc_normals6(seed, step, i, z);
        const double* p = axis + 3 * i;
        const double pt = dot3(p, z), pr = dot3(p, z + 3);
        for (int m = 0; m < 3; ++m) {
            double ft = a * (sqrt(zeta[1]) * pt * p[m] + sqrt(zeta[0]) * (z[m] - pt * p[m]));
            double fr = a * (sqrt(zeta[3]) * pr * p[m] + sqrt(zeta[2]) * (z[3 + m] - pr * p[m]));
            out[6 * i + m] = (f_ext ? f_ext[6 * i + m] : 0.0) + ft;
            out[6 * i + 3 + m] = (f_ext ? f_ext[6 * i + 3 + m] : 0.0) + fr;
        }
    }
    free(axis);
}

/* ------------------------------------------------------------------ walls */

/* Confinement by two flat walls normal to axis w at coordinates lo < hi
 * (Appendix: a collision with an external boundary keeps only the
 * particle's side of the column).  The lowest point of a segment over a
 * plane is one of its ends (both, when it lies flat), so each end of a rod,
 * y = s p with s = -L/2 and s = +L/2, is a contact candidate with each wall:
 * gap Phi = x_w + s p_w - lo - D/2 and normal e = +e_w for the lower wall,
 * Phi = hi - x_w - s p_w - D/2 and e = -e_w for the upper one.  A row is
 * made when Phi < delta_c: pairs (i, -1, 2 side + end), dgeom (e, y x e, 0),
 * q = Phi/h + (e, y x e).U_nc, phi.  Rows are in (rod, side, end) order.
 * Returns the row count (rows written only if cap allows). */
ORC_API int64_t orc_assemble_walls(int64_t n, const double* x, const double* quat, const double* fnc,
                                   const orc_problem* pb, int axis_w, double lo, double hi, int64_t cap,
                                   int32_t* pairs, double* dgeom, double* q, double* phi)
{
    double zeta[4];
    orc_drag(pb->viscosity, pb->length, pb->diameter, zeta);
    const double hl = 0.5 * pb->length;
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i) {
        double th[4] = {quat[4 * i], quat[4 * i + 1], quat[4 * i + 2], quat[4 * i + 3]};
        double p[3];
        orc_axis(1, th, p);
        const double xw = wrap1(x[3 * i + axis_w], pb->box[axis_w]);
        for (int side = 0; side < 2; ++side)
        for (int end = 0; end < 2; ++end) {
            const double sg = side == 0 ? 1.0 : -1.0;   /* normal into the domain */
            const double pw = p[axis_w];
            const double s = end == 0 ? -hl : hl;
            const double tip = xw + s * pw;
            const double ph = side == 0 ? tip - lo - 0.5 * pb->diameter : hi - tip - 0.5 * pb->diameter;
            if (!(ph < pb->delta_c)) continue;
            if (cnt < cap) {
                double e[3] = {0.0, 0.0, 0.0}, y[3], ye[3];
                e[axis_w] = sg;
                for (int m = 0; m < 3; ++m) y[m] = s * p[m];
                cross3(y, e, ye);
                pairs[3 * cnt] = (int32_t)i;
                pairs[3 * cnt + 1] = -1;
                pairs[3 * cnt + 2] = 2 * side + end;
                double* dg = dgeom + 9 * cnt;
                for (int m = 0; m < 3; ++m) { dg[m] = e[m]; dg[3 + m] = ye[m]; dg[6 + m] = 0.0; }
                double U[6];
                mobility_rod(p, zeta, fnc + 6 * i, U);
                q[cnt] = ph / pb->dt + dot3(e, U) + dot3(ye, U + 3);
                phi[cnt] = ph;
            }
            ++cnt;
        }
    }
    return cnt;
}

/* ----------------------------------------------------------------- update */

/* C^{k+1} = C^k + h G U (Eq. constrainedeom_euler a), U = M (F_nc + D gamma):
 *   x' = wrap(x + h U_t),
 *   theta' = normalise(theta + h Psi(theta) Omega),
 *   Psi(theta) Omega = 1/2 [ -v.Omega ; s Omega - v x Omega ]
 * (Appendix, Psi = 1/2 [-p^T; sI - P], P_ij = eps_ikj p_k, so P Omega = v x Omega).
 * U_out (nullable) receives U = M (F_nc + D gamma). */
ORC_API void orc_update(int64_t n, const double* x, const double* quat, const double* fnc, const orc_problem* pb,
                        int64_t npairs, const int32_t* pairs, const double* dgeom, const double* gamma,
                        double* x_out, double* quat_out, double* U_out)
{
    double zeta[4];
    orc_drag(pb->viscosity, pb->length, pb->diameter, zeta);
    size_t nn = (size_t)(n > 0 ? n : 1);
    double* F = (double*)malloc(sizeof(double) * 6 * nn);
    double* axis = (double*)malloc(sizeof(double) * 3 * nn);
    orc_apply_D(n, npairs, pairs, dgeom, gamma, F);
    orc_axis(n, quat, axis);
    for (int64_t i = 0; i < n; ++i) {
        double Fi[6], Ui[6];
        for (int k = 0; k < 6; ++k) Fi[k] = fnc[6 * i + k] + F[6 * i + k];
        mobility_rod(axis + 3 * i, zeta, Fi, Ui);
        if (U_out) for (int k = 0; k < 6; ++k) U_out[6 * i + k] = Ui[k];
        for (int k = 0; k < 3; ++k) x_out[3 * i + k] = wrap1(wrap1(x[3 * i + k], pb->box[k]) + pb->dt * Ui[k], pb->box[k]);
        const double* th = quat + 4 * i;
        double s = th[0];
        const double* v = th + 1;
        const double* om = Ui + 3;
        double vxo[3];
        cross3(v, om, vxo);
        double qn[4];
        qn[0] = s + pb->dt * 0.5 * (-dot3(v, om));
        for (int k = 0; k < 3; ++k) qn[1 + k] = v[k] + pb->dt * 0.5 * (s * om[k] - vxo[k]);
        double nq = sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
        for (int k = 0; k < 4; ++k) quat_out[4 * i + k] = qn[k] / nq;
    }
    free(F); free(axis);
}

/* ------------------------------------------------------------- full step */

/* One constrained step: pairs -> assembly -> solve -> update.  Arrays sized
 * by the caller: pairs cap = max_pairs triples.  Returns the pair count
 * (or -count-1 if max_pairs was too small; nothing else is then written). */
ORC_API int64_t orc_step(int64_t n, const double* x, const double* quat, const double* fnc, const orc_problem* pb,
                         double tol, int64_t max_iter, int64_t max_pairs, int32_t* pairs, double* gamma,
                         double* x_out, double* quat_out, double* U_out, double* residual, int64_t* iters)
{
    int64_t np = orc_find_pairs(n, x, quat, pb, pairs, max_pairs);
    if (np > max_pairs) return -np - 1;
    size_t m = (size_t)(np > 0 ? np : 1);
    double* phi = (double*)malloc(sizeof(double) * m);
    double* dg = (double*)malloc(sizeof(double) * 9 * m);
    double* q = (double*)malloc(sizeof(double) * m);
    orc_assemble(n, x, quat, fnc, pb, np, pairs, phi, dg, q, NULL, NULL);
    for (int64_t c = 0; c < np; ++c) gamma[c] = 0.0;
    double r = orc_solve_apgd(n, quat, pb, np, pairs, dg, q, NULL, gamma, tol, max_iter, iters);
    if (residual) *residual = r;
    orc_update(n, x, quat, fnc, pb, np, pairs, dg, gamma, x_out, quat_out, U_out);
    free(phi); free(dg); free(q);
    return np;
}
