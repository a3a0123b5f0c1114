/*
 * alens.h - C ABI of the GB300 library for the hard-body collision-constraint
 * step of aLENS (Yan et al., arXiv 2109.08206).
 *
 * One step takes N rigid spherocylinders (diameter D, cylinder length L) in a
 * periodic box with given non-constraint forces F_nc and a time step h, and
 *   1. finds every rod pair (and periodic image) whose surface gap is below
 *      delta_c                    (Appendix "Implementation", near-neighbour
 *                                  detection with threshold delta_c),
 *   2. builds the gap Phi, the sparse constraint matrix D and
 *      q = Phi/h + D^T M F_nc     (Appendix Eq. blockdef, block A; Eq. dmap),
 *   3. solves the convex QP  min 1/2 g^T (D^T M D) g + q^T g,  g >= 0
 *      by Barzilai-Borwein projected gradient descent
 *                                 (Appendix Eq. suppcqpdef; Section
 *                                  "Instantiation...": BBPGD),
 *   4. moves the rods: U = M (F_nc + D gamma), C' = C + h G U
 *                                 (Appendix Eq. constrainedeom_euler a-c).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Array arguments are DEVICE pointers to caller-owned, contiguous,
 *   row-major memory on the context's device.  The library never frees a
 *   caller pointer and keeps none after a call returns.
 * - x      [n][3] float64  rod centres (any real value; wrapped into [0, box)).
 * - quat   [n][4] float64  unit quaternions (s, v1, v2, v3); the rod axis is
 *                          p = R(quat) e_z.  |quat| must be within 1e-6 of 1.
 * - f_nc   [n][6] float64  non-constraint force (3) then torque (3), lab frame.
 * - pairs  [m][3] int32    (i, j, image) with i < j, sorted by (i, j, image);
 *                          image = (kx+1) + 3(ky+1) + 9(kz+1), k in {-1,0,1}^3,
 *                          and the centre offset of the pair is
 *                          dx = x_i - x_j - k * box (wrapped centres).
 * - dgeom  [m][9] float64  per constraint (e, y_P x e, y_Q x e): e = r/|r| is
 *                          the unit normal from Q to P, y_P / y_Q the contact
 *                          arms from the rod centres; the column of D acting on
 *                          rod P is (e, y_P x e), on rod Q (-e, -(y_Q x e)).
 * - phi    [m] float64     surface gap |r| - D (negative when overlapping).
 * - gamma  [m] float64     constraint force magnitudes (>= 0, repulsive).
 * - Mobility per rod (the paper quotes only the slender-body coefficient
 *   4 pi eta L / ln(2L/D)): zeta_perp = 4 pi eta L / ln(2L/D),
 *   zeta_par = zeta_perp/2, zeta_rot = zeta_perp L^2/12, zeta_spin =
 *   pi eta D^2 L; M_t = p p^T/zeta_par + (I - p p^T)/zeta_perp and
 *   M_r = p p^T/zeta_spin + (I - p p^T)/zeta_rot.
 * - Residual (the paper does not define one): r = (h/D) max_c |pi_c| with
 *   pi_c = g_c if gamma_c > 0 else min(g_c, 0), g = D^T M D gamma + q; it is
 *   the worst linearised post-step gap error in rod diameters.
 * - All work is ordered on the context's CUDA stream.  Entry points that
 *   return counts or an aLENS_info synchronise that stream before returning.
 * - Errors are returned, never raised: ALENS_ERR_INVALID before any output
 *   is written, ALENS_ERR_CAPACITY with the required size, ALENS_ERR_TIMEOUT
 *   when a bounded device wait ran out (the context stays usable),
 *   ALENS_ERR_NOT_CONVERGED with outputs and the residual filled in.
 * - A context is not thread-safe; use one per host thread.
 */
#ifndef ALENS_H
#define ALENS_H

#include <stdint.h>

#if defined(__GNUC__)
#define ALENS_API __attribute__((visibility("default")))
#else
#define ALENS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ALENS_OK = 0,
    ALENS_ERR_INVALID = 1,        /* bad argument or input (NaN, non-unit quaternion, box too small) */
    ALENS_ERR_CAPACITY = 2,       /* a buffer is too small; the required count is reported */
    ALENS_ERR_NOT_CONVERGED = 3,  /* max_iter reached; outputs and residual are valid */
    ALENS_ERR_TIMEOUT = 4,        /* a bounded grid-wide wait gave up; outputs undefined */
    ALENS_ERR_CUDA = 5,           /* a CUDA runtime call failed */
    ALENS_ERR_NOMEM = 6,          /* workspace allocation failed */
    ALENS_ERR_NOT_IMPLEMENTED = 7
} aLENS_status;

typedef enum {
    ALENS_FP64 = 0,   /* every stage in float64 */
    ALENS_MIXED = 1   /* solver iterations (D, M, D^T, their sums and step sizes)
                         in float32 on a float64-accurate reference refreshed
                         every 64 iterations (the reference passes use
                         compensated float32 sums over the float64 records
                         split into float32 pairs); geometry, pair decisions
                         and the stopping decision in float64 */
} aLENS_precision;

typedef struct {
    double box[3];      /* periodic edge lengths; each >= length + diameter + delta_c */
    double diameter;    /* D (the paper's D_fil) */
    double length;      /* L, cylinder length without the caps */
    double viscosity;   /* eta; every drag coefficient is proportional to it */
    double dt;          /* h */
    double delta_c;     /* pair threshold on the surface gap (paper: delta_c = D) */
    double tol;         /* residual tolerance, rod diameters */
    int32_t max_iter;   /* BBPGD iteration cap */
    int32_t precision;  /* aLENS_precision */
} aLENS_params;

typedef struct {
    int64_t n_pairs;    /* constraints in the step */
    int64_t n_overlap;  /* constraints with phi < 0 */
    int32_t iters;      /* BBPGD iterations taken */
    int32_t status;     /* aLENS_status of the call */
    double residual;    /* final residual (rod diameters) */
    double min_gap;     /* min phi over the constraints (+inf if none) */
    float ms_build;     /* device time of the neighbour search */
    float ms_assemble;  /* device time of the assembly and CSR build */
    float ms_solve;     /* device time of the BBPGD kernel alone */
    float ms_update;    /* device time of the update */
    int32_t launches;   /* kernels the call launched */
    int32_t solver;     /* solver kernel of the call: 0 none, 1 one grid barrier per
                           iteration, 2 two barriers with shared-memory shares,
                           3 two barriers from global memory, 4 per-system clusters */
} aLENS_info;

typedef struct aLENS_ctx aLENS_ctx;

/* Create a context on the current CUDA device.  Workspaces for up to
 * max_rods rods and max_pairs constraints are allocated here and owned by
 * the context.  cuda_stream is a cudaStream_t (NULL = legacy default
 * stream).  Returns INVALID for bad parameters, NOMEM/CUDA on failure. */
ALENS_API aLENS_status aLENS_create(const aLENS_params* params, int64_t max_rods, int64_t max_pairs,
                          void* cuda_stream, aLENS_ctx** out);

/* Release every workspace of the context (synchronises its stream).  NULL is ignored. */
ALENS_API void aLENS_destroy(aLENS_ctx* ctx);

/* Replace the step parameters.  Returns CAPACITY if the new box needs more
 * cells than the context allocated at create time, INVALID for bad values. */
ALENS_API aLENS_status aLENS_set_params(aLENS_ctx* ctx, const aLENS_params* params);

/* Static description of a status code. */
ALENS_API const char* aLENS_status_string(aLENS_status status);

/* Neighbour search (Appendix "Implementation": close pairs whose minimal
 * distance is below delta_c).  Writes the sorted pair list into pairs
 * (capacity pairs_cap triples) and the count into *n_pairs (host pointer).
 * On CAPACITY *n_pairs is the required count and pairs is unspecified.
 * The keep/drop decision of every pair is taken in float64. */
ALENS_API aLENS_status aLENS_build_neighbors(aLENS_ctx* ctx, int64_t n, const double* x, const double* quat,
                                   int32_t* pairs, int64_t pairs_cap, int64_t* n_pairs);

/* Constraint assembly for a sorted pair list (Appendix Eq. blockdef A and
 * the column D_PQ = [e_P, y_P x e_P, e_Q, y_Q x e_Q], e_Q = -e_P):
 * phi[m], dgeom[m][9] and q[m] = phi/h + D^T M f_nc, all float64. */
ALENS_API aLENS_status aLENS_assemble_constraints(aLENS_ctx* ctx, int64_t n, const double* x, const double* quat,
                                        const double* f_nc, int64_t n_pairs, const int32_t* pairs,
                                        double* phi, double* dgeom, double* q);

/* BBPGD solve of the CQP (Appendix Eq. suppcqpdef) for given D (dgeom) and
 * q.  gamma is read as the start (negative entries projected to 0; pass
 * zeros for a cold start) and overwritten with the solution.  info (host
 * pointer, may be NULL) receives iterations and residual. */
ALENS_API aLENS_status aLENS_solve_lcp(aLENS_ctx* ctx, int64_t n, const double* quat, int64_t n_pairs,
                             const int32_t* pairs, const double* dgeom, const double* q, double* gamma,
                             aLENS_info* info);

/* One full constrained step: neighbours -> assembly -> BBPGD -> update.
 * x and quat are updated in place (x wrapped into [0, box), quat
 * renormalised).  gamma_out (nullable, capacity max_pairs of the context)
 * receives gamma in pair order; vel_out (nullable, [n][6]) receives
 * U = M (f_nc + D gamma).  pairs_out (nullable, capacity max_pairs triples)
 * receives the pair list.  info (host pointer, may be NULL). */
ALENS_API aLENS_status aLENS_step(aLENS_ctx* ctx, int64_t n, double* x, double* quat, const double* f_nc,
                        int32_t* pairs_out, double* gamma_out, double* vel_out, aLENS_info* info);

/* ------------------------------------------------------------------------
 * Bilateral (spring) constraints: doubly bound crosslinkers (Appendix: Phi_b
 * is the distance between two fixed points of particles P and Q, and
 * K [Phi_b - Phi_b^0] = -gamma_b; linearised as Eq. linearconstraints b and
 * solved with the collisions as one CQP, Eq. suppcqpdef, whose matrix gains
 * the diagonal compliance K^{-1}/h on the spring block (Eq. blockdef F) and
 * whose spring forces are not projected).
 * ends  [n_springs][2] int32: rods P and Q of each spring (P != Q, any order).
 * arms  [n_springs][2] float64: arclengths s_P, s_Q of the attachment points
 *       along the rods' axes from their centres (y = s p).
 * kappa [n_springs] float64 > 0: stiffness; rest [n_springs]: rest length.
 * All DEVICE pointers; the context copies them (stream-ordered) and every
 * later aLENS_step / aLENS_step_batch solves them with that step's
 * collisions: the point pair is taken over its minimum periodic image, the
 * column is (e, y_P x e | -e, -(y_Q x e)) as for a collision, and
 * gamma_out holds the collision forces followed by the spring forces
 * (gamma_b > 0 pushes the points apart, gamma_b = -kappa (Phi_b' - rest)
 * at the linearised new length).  Capacity: collisions + springs <=
 * max_pairs.  n_springs = 0 removes the springs.  A spring whose rods are
 * out of range, equal, in different systems of a batch, or whose kappa is
 * not positive makes the step return INVALID with nothing moved.  Not
 * covered by aLENS_step_adjoint (NOT_IMPLEMENTED while springs are set). */
ALENS_API aLENS_status aLENS_set_springs(aLENS_ctx* ctx, int64_t n_springs, const int32_t* ends, const double* arms,
                                         const double* kappa, const double* rest);

/* ------------------------------------------------------------------------
 * Multi-step trajectories (Appendix Eq. constrainedeom_euler repeated in
 * time, with the Brownian force F_B among the non-constraint forces).
 *
 * aLENS_set_walls: two flat confining walls normal to axis (0, 1, 2; -1
 * removes them) at coordinates lo < hi (Appendix: a collision with an
 * external boundary keeps only the particle's side of the D column).  The
 * lowest point of a rod over a plane is one of its ends (both when it lies
 * flat), so each end y = s p (s = -L/2, +L/2) is a contact candidate with
 * each wall: gap Phi = x_axis + s p_axis - lo - D/2 and normal +e_axis for
 * the lower wall (the upper wall alike, normal -e_axis); every candidate
 * with Phi < delta_c is a unilateral constraint solved with the collisions,
 * its force listed after the collisions (and before the springs) in
 * gamma_out, in (rod, wall, end) order.  Requires 0 <= lo < hi <= box[axis]
 * and box[axis] - (hi - lo) >= L + D + delta_c, so that no pair interacts
 * through the periodic boundary across the walls.  Single systems only
 * (aLENS_step_batch returns NOT_IMPLEMENTED while walls are set); not
 * covered by aLENS_step_adjoint. */
ALENS_API aLENS_status aLENS_set_walls(aLENS_ctx* ctx, int32_t axis, double lo, double hi);

/* The non-constraint force of trajectory step `step`: out [n][6] = f_ext
 * (nullable) + the Brownian force and torque of every rod, with covariance
 * 2 kT M^-1 / h per rod (fluctuation-dissipation: the step's displacement
 * then has covariance 2 kT h M):
 *   F = sqrt(2 kT / h) [sqrt(zeta_par) (p.xi) p + sqrt(zeta_perp) (xi - (p.xi) p)]
 *   T = sqrt(2 kT / h) [sqrt(zeta_spin) (p.chi) p + sqrt(zeta_rot) (chi - (p.chi) p)]
 * where (xi, chi) are six standard normals of (seed, step, rod): the
 * counter-based generator Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11)
 * with key (seed low, seed high) and counters (rod, step low, step high, w),
 * w = 0, 1, each 32-bit word x giving u = (x + 0.5) 2^-32, each pair of
 * words two normals by Box-Muller.  quat, f_ext, out: device. */
ALENS_API aLENS_status aLENS_brownian(aLENS_ctx* ctx, int64_t n, const double* quat, double kT, uint64_t seed,
                                      int64_t step, const double* f_ext, double* out);

/* The eight raw generator words of every rod for (seed, step) (device
 * out [n][8]): the counters w = 0 then w = 1 of aLENS_brownian. */
ALENS_API aLENS_status aLENS_random_words(aLENS_ctx* ctx, int64_t n, uint64_t seed, int64_t step, uint32_t* out);

typedef struct {
    int64_t n_pairs;    /* collisions of the step */
    int64_t n_walls;    /* wall contacts of the step */
    int32_t iters;      /* BBPGD iterations */
    int32_t status;     /* aLENS_status of the step */
    double residual;
    double min_gap;     /* min Phi over collisions and wall contacts */
    float ms_step;      /* device time of the step (search to update) */
} aLENS_step_stats;

/* n_steps constrained steps of x, quat in place; step k (k = 0 ..
 * n_steps-1) uses the forces of aLENS_brownian(first_step + k), so that a
 * long run split into calls reproduces the run done in one call.  Walls and
 * springs set on the context take part.  warm_start != 0 starts every
 * solve from the previous step's forces, matched per constraint (a
 * collision by (i, j, image), a wall contact by (rod, wall, end), a spring
 * by its index while the spring list is unchanged), instead of from 0.
 * stats (HOST array [n_steps], nullable) receives per-step figures; info
 * aggregates (iterations summed, residual max, min_gap min, phase times
 * summed).  The first call allocates the trajectory buffers (6 doubles per
 * rod and 4 words per constraint of the context's capacity).  Stops at the
 * first step whose status is neither OK nor NOT_CONVERGED. */
ALENS_API aLENS_status aLENS_run(aLENS_ctx* ctx, int64_t n, double* x, double* quat, const double* f_ext,
                                 int64_t n_steps, double kT, uint64_t seed, int64_t first_step, int32_t warm_start,
                                 aLENS_step_stats* stats, aLENS_info* info);

/* ------------------------------------------------------------------------
 * Batched step of independent periodic systems.  The paper steps one system
 * (distributed over many processes); an ensemble of many small, uneven
 * systems is stepped here in one call, each system with the step of
 * aLENS_step (Appendix Eq. blockdef A, Eq. suppcqpdef, Eq.
 * constrainedeom_euler a-c).
 *
 * systems    [n_systems] HOST array: periodic box and cylinder length of each
 *            system; each box edge >= length + diameter + delta_c.  Diameter,
 *            viscosity, dt, delta_c, tol, max_iter and precision are the
 *            context's parameters, shared by every system.
 * rod_offset [n_systems + 1] HOST array: system s owns rods
 *            [rod_offset[s], rod_offset[s+1]) of x, quat, f_nc and vel_out;
 *            rod_offset[0] = 0, non-decreasing, last entry = the rod count
 *            (<= max_rods of the context).  Empty systems are allowed.
 * x, quat, f_nc, pairs_out, gamma_out, vel_out, info: as for aLENS_step,
 *            over all rods of the batch with global rod indices.  No pair
 *            joins two systems, so each system's pairs form one contiguous
 *            run of pairs_out (they are sorted by i).
 *
 * Every system's constraint problem is solved by its own BBPGD run (its own
 * step sizes, residual and stopping test), all of them in one launch of the
 * per-system solver (thread-block clusters taking systems from a queue,
 * largest first; the largest systems of an uneven batch are solved by two
 * clusters together, see aLENS_batch_groups); a batch of one system uses
 * the solver of aLENS_step.
 * info aggregates the batch: pair, overlap and launch counts summed,
 * iterations and residual the largest over the systems (so the call
 * returns OK only when every system met the tolerance), minimum gap over
 * all constraints.  aLENS_batch_results gives the per-system figures.  The first call with more systems or cell
 * keys than any call before grows the context's tables (this allocates and
 * synchronises); later calls with the same systems reuse the uploaded tables.
 * Errors as for aLENS_step; INVALID also for a bad table or a system whose
 * cell grid would exceed 2^7 cells along an edge. */
typedef struct {
    double box[3];    /* periodic edge lengths of the system */
    double length;    /* cylinder length L of its rods */
} aLENS_system;

ALENS_API aLENS_status aLENS_step_batch(aLENS_ctx* ctx, int32_t n_systems, const aLENS_system* systems,
                                        const int64_t* rod_offset, double* x, double* quat, const double* f_nc,
                                        int32_t* pairs_out, double* gamma_out, double* vel_out, aLENS_info* info);

/* Batched steps as a captured CUDA graph (the paper has no batch mode: a
 * batch serves many independent systems in one call).  enable = 1:
 * aLENS_step_batch of two or more systems records its whole step - search,
 * assembly, the per-system solver launch, update and outputs - as one CUDA
 * graph and replays it on later calls.  A step has no host readback inside
 * the graph: kernels sized by the constraint count are launched for the
 * context's capacity and read the count on the device, and a step whose
 * pairs exceed the capacity changes nothing and returns ALENS_ERR_CAPACITY
 * with the required count (counted again outside the graph when the
 * candidate buffer overflowed).  The graph is kept for one key: the batch
 * tables, n, the six array pointers of the call, the parameters, the
 * scaling exponent and the batch launch shape.  The first call with a new
 * key runs without a graph, the second records the graph and runs it, later
 * calls replay it; a call with another key starts over.  Steps with
 * springs, and the fault hook, always run without a graph.  Results equal
 * those of steps without a graph bit for bit.  enable = 0 releases the
 * graph.  ALENS_ERR_INVALID for other values. */
ALENS_API aLENS_status aLENS_set_batch_graph(aLENS_ctx* ctx, int32_t enable);

/* CUDA-graph mode for aLENS_step (single systems; Appendix "Implementation":
 * the step's kernels, recorded once and replayed, with no host round trip
 * inside the step).  enable = 1: the first call with a new key (n, the six
 * array pointers, parameters, scaling exponent, solver launch shape and
 * schedule) runs without a graph; if that step ran the one-barrier solver
 * (aLENS_info.solver = 1), the second call records the step and runs it,
 * and later calls replay it.  In the recorded step the solver is launched
 * with the whole shared-memory budget of its launch shape and checks on the
 * device that every block's share fits; when one does not (the pairs moved
 * into a denser arrangement), nothing moves and the call runs the step
 * without a graph, as do all later calls with that key.  Kernels sized by
 * the constraint count are launched for the context's capacity and read the
 * count on the device; a step whose pairs exceed the capacity changes
 * nothing and returns ALENS_ERR_CAPACITY with the required count.  Steps
 * with springs or walls, and the timeout test hook, always run without a
 * graph.  Results equal those of steps without a graph bit for bit.  The
 * graph slot is shared with aLENS_set_batch_graph (one key per context).
 * enable = 0 releases the graph.  ALENS_ERR_INVALID for other values. */
ALENS_API aLENS_status aLENS_set_step_graph(aLENS_ctx* ctx, int32_t enable);

/* L2 residency of the solver's constraint states (enable = 1, the
 * default).  Where the two-barrier solver reads its data from global memory
 * and those data exceed the device's L2 (about 136 bytes per constraint),
 * its launch carries an access-policy window that marks the two state
 * buffers persisting in L2 while the records stream, and the context raises
 * its persisting L2 set-aside to hold the states, as far as the device
 * allows; aLENS_destroy puts the set-aside back.  Addresses only: every
 * result is the same with enable = 0.  A launch being recorded into a CUDA
 * graph takes no window.  INVALID for other values. */
ALENS_API aLENS_status aLENS_set_l2_window(aLENS_ctx* ctx, int32_t enable);

/* Name of the CUDA runtime error behind the calling thread's last
 * ALENS_ERR_CUDA from a context entry point ("cudaSuccess" if none);
 * a static string. */
ALENS_API const char* aLENS_last_cuda_error(void);

/* ------------------------------------------------------------------------
 * Adjoint of aLENS_step (reverse-mode gradient of a scalar loss L(x', quat')
 * of the post-step state).  The paper does not differentiate its step; this
 * differentiates the same step (Appendix Eq. constrainedeom_euler a-c with
 * the constraint problem of Eq. suppcqpdef) on the forward step's pair list
 * and active set {c : gamma_c > 0}, where the KKT conditions read
 * (D^T M D gamma + q)_c = 0:
 *   u = dL/dU through the update; b = D^T M u; lambda solves
 *   (D^T M D)_AA lambda_A = b_A by conjugate gradients (from 0: the
 *   minimum-norm multiplier when the block is singular); then the
 *   derivatives of q, D (closest points on their branch: both parameters
 *   free, one clamped, both clamped; parallel segments with s*, t* held)
 *   and of M (axes, viscosity).
 * x, quat, f_nc: the state the forward aLENS_step started from (device,
 *   as for aLENS_step; the caller keeps a copy, aLENS_step overwrote them).
 * pairs [n_pairs][3], gamma [n_pairs]: that step's pairs_out and gamma_out.
 * dL_dx_new [n][3], dL_dquat_new [n][4]: dL/dx' and dL/dquat' (either may
 *   be NULL = zero).  x' is the unwrapped x + h U_t.
 * Outputs (device): dL_dx [n][3]; dL_dquat [n][4], the gradient projected
 *   onto the unit quaternion's tangent space; dL_dfnc [n][6] (nullable);
 *   dL_deta (HOST pointer, nullable): derivative with respect to the
 *   viscosity, to which every drag coefficient is proportional.
 * The CG operator runs in the context's precision (float32 records in mixed
 * mode), everything else in float64.  info: iters = CG iterations,
 * residual = final relative CG residual |r|/|b_A| (tolerance 1e-13 in
 * FP64, 1e-7 mixed; NOT_CONVERGED with the outputs filled if max_iter CG
 * iterations did not reach it).  The CG loop is one persistent cooperative
 * kernel with bounded grid-wide waits: TIMEOUT when one runs out (see
 * aLENS_set_wait_limit).  The first call allocates the adjoint's
 * workspace (46 doubles and 4 ints per rod, 13 doubles and 3 ints per
 * constraint of the context's capacity).
 * Single systems only (batches: call it per system). */
ALENS_API aLENS_status aLENS_step_adjoint(aLENS_ctx* ctx, int64_t n, const double* x, const double* quat,
                                          const double* f_nc, int64_t n_pairs, const int32_t* pairs,
                                          const double* gamma, const double* dL_dx_new, const double* dL_dquat_new,
                                          double* dL_dx, double* dL_dquat, double* dL_dfnc, double* dL_deta,
                                          aLENS_info* info);

/* Per-system results of the last aLENS_step_batch on this context: iters
 * and residual are HOST arrays of n_systems entries (either may be NULL);
 * n_systems must equal that call's.  For a batch of one system the values
 * are those of its info.  Synchronises the context's stream. */
ALENS_API aLENS_status aLENS_batch_results(aLENS_ctx* ctx, int32_t n_systems, int32_t* iters, double* residual);

/* Blocks that solved each system in the last aLENS_step_batch: one
 * cluster's blocks (aLENS_set_batch_launch), or twice as many for a system
 * that two clusters solved together.  The per-system solver pairs clusters
 * on the largest systems (at most a quarter of its clusters' count, each
 * with at least 4096 constraints per block of one cluster and more than
 * half of one cluster's mean share of the batch's constraints), so that no
 * single system's solve outlasts the rest of the queue; the choice depends
 * only on the systems and the launch shape.  blocks is a HOST array of
 * n_systems entries; n_systems must equal that call's.  For a batch of one
 * system the entry is 0 (the single-system solver ran).  Synchronises the
 * context's stream. */
ALENS_API aLENS_status aLENS_batch_groups(aLENS_ctx* ctx, int32_t n_systems, int32_t* blocks);

/* Launch shape of the per-system solver of aLENS_step_batch: threads per
 * block (multiple of 32, <= 1024; default 1024) and blocks per cluster
 * (1, 2, 4 or 8; default 8).  For tuning. */
ALENS_API aLENS_status aLENS_set_batch_launch(aLENS_ctx* ctx, int32_t threads, int32_t cluster_blocks);

/* Bound on every grid-wide wait inside the solver kernel, in seconds
 * (default 5).  A wait that runs out makes the call return ALENS_ERR_TIMEOUT. */
ALENS_API aLENS_status aLENS_set_wait_limit(aLENS_ctx* ctx, double seconds);

/* Diagonal scaling of the BBPGD iteration (Appendix Eq. suppcqpdef is
 * solved for gamma = S gamma~ with S = diag(sigma_c)): the iteration runs on
 * the records sigma_c D_c, q~_c = sigma_c q_c and the compliance sigma_c^2
 * C_c, with sigma_c = (D_c^T M D_c + C_c)^(-beta/2) computed in float64 when
 * the solve is set up.  The minimiser, the residual (taken on the unscaled
 * projected gradient) and every output are those of the unscaled problem;
 * only the path and the iteration count change.  beta in [0, 1]: 0 is the
 * unscaled iteration, 1 Jacobi scaling; default 0.5.  INVALID otherwise. */
ALENS_API aLENS_status aLENS_set_scaling(aLENS_ctx* ctx, double beta);

/* Test hook: mode 1 makes one thread block of the next solver launch (the
 * BBPGD of a step or solve, or the CG of aLENS_step_adjoint) leave before
 * its first grid-wide arrival, so that the other blocks' bounded waits run
 * out and the call returns ALENS_ERR_TIMEOUT; in the batched solver, the
 * second cluster of every pair (aLENS_batch_groups) skips its system, so
 * that the first cluster's bounded waits run out.  mode 2 makes the next
 * recorded single-system step (aLENS_set_step_graph) find its shares too
 * big for its launch, so that the call falls back to a step without a
 * graph.  These clear themselves after one launch or recording; mode 0
 * disables them.  mode 3 makes the context's batched solver run as on a
 * device that refuses a cooperative launch with clusters: every system is
 * solved by one cluster from then on (drops a recorded batched step). */
ALENS_API aLENS_status aLENS_inject_fault(aLENS_ctx* ctx, int32_t mode);

/* Launch shape of the solver kernel: threads per block (multiple of 32,
 * <= 1024; default 768) and blocks per SM (0 = one).  For tuning. */
ALENS_API aLENS_status aLENS_set_launch(aLENS_ctx* ctx, int32_t threads, int32_t blocks_per_sm);

/* Grid-wide synchronisations per BBPGD iteration (Appendix "Implementation":
 * the BBPGD iterations are the step's dominant cost).  barriers = 1
 * (default): where every block's share of the constraints, plus a copy of
 * each constraint another block owns that touches one of its rods, fits in
 * shared memory, the solver synchronises the grid once per iteration and
 * takes the Barzilai-Borwein step length one iteration late; elsewhere it
 * falls back to barriers = 2, the two-barrier iteration with the current
 * step length.  Both stop on the residual of the returned gamma and reach
 * the same minimiser; iteration counts differ.  For tuning and tests;
 * ALENS_ERR_INVALID for any other value. */
ALENS_API aLENS_status aLENS_set_solver_schedule(aLENS_ctx* ctx, int32_t barriers);

/* ------------------------------------------------------------------------
 * Allocation-free solve.  The paper has no counterpart: this entry point
 * exists for callers that may not allocate device memory - a host
 * application or plugin whose memory manager owns the whole device budget,
 * or a latency-critical loop where cudaMalloc / cudaFree would take the
 * allocator lock or synchronise the device.  Such callers cannot create an
 * aLENS_ctx, because aLENS_create allocates its workspaces.
 *
 * It runs the same BBPGD solve as aLENS_solve_lcp (same arguments and
 * outputs, params->box and delta_c unused) with its workspace in one static
 * device array of the library (5.19 MB, held on every GPU that loads the
 * library until the process exits), and calls no allocating routine.
 * Limits: n <= ALENS_NOALLOC_MAX_RODS and n_pairs <= ALENS_NOALLOC_MAX_PAIRS;
 * larger problems return ALENS_ERR_CAPACITY before any work is queued.
 * The first call on a device (with that device current) looks up the
 * array's device address and keeps it for the life of the process; make it
 * before any stream capture.  cudaDeviceReset (or anything else that
 * destroys the device's primary context) unloads the library's device code
 * and leaves that address stale: do not call this entry point on a device
 * after resetting it.  Every call
 * reuses the same array (the counters that must start at zero are cleared
 * on each call), so calls whose GPU work overlaps - on different streams or
 * from different host threads - race; serialise them.  The call
 * synchronises cuda_stream.  info (may be NULL) gets iterations and
 * residual; its timing fields are 0. */
#define ALENS_NOALLOC_MAX_RODS 4096
#define ALENS_NOALLOC_MAX_PAIRS 16384
ALENS_API aLENS_status aLENS_solve_lcp_noalloc(const aLENS_params* params, int64_t n, const double* quat,
                                               int64_t n_pairs, const int32_t* pairs, const double* dgeom,
                                               const double* q, double* gamma, void* cuda_stream,
                                               aLENS_info* info);

#ifdef __cplusplus
}
#endif

#endif /* ALENS_H */
