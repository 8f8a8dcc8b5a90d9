/* rbfgb.h — C ABI of the GB300 (sm_103a) meshless porous-media solvers.
 *
 * The library implements the hot path of Strzelczyk, Rot, Kosec & Matyka,
 * "Cross-validation of meshless Navier-Stokes solvers in porous media flows"
 * (arXiv 2404.14195): RBF-FD stencil weights (PHS + monomials), the explicit
 * artificial-compressibility Navier-Stokes step (MNS) and the two-relaxation-time
 * meshless lattice Boltzmann step (MLBM) on scattered nodes, and the permeability
 * and drag reductions.  The calls follow the paper's statement of the problem:
 * nodes and geometry in; stencils and weights; step to steady state; drag
 * coefficient and permeability out.
 *
 * Conventions (every call):
 *  - returns RBF_OK (0) or a negative RBF_E* code; rbf_last_error() gives the
 *    message of the last failure on that context (owned by the context);
 *  - host arrays passed in are owned by the caller and copied before return;
 *    host arrays passed out are written before return (the call synchronises
 *    the context's stream);
 *  - node arrays are in the caller's node order (the library reorders nodes
 *    along a Morton curve internally and maps back on output);
 *  - a context is bound to one device and one CUDA stream; calls on one context
 *    are not thread-safe; all device work is ordered on that stream;
 *  - there is no CPU fallback: without a usable CUDA device rbf_create fails
 *    with RBF_ECUDA.
 */
#ifndef RBFGB_H
#define RBFGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    RBF_OK = 0,
    RBF_EINVAL = -1,        /* bad argument, size or call order */
    RBF_ECUDA = -2,         /* CUDA runtime or launch error */
    RBF_ESINGULAR = -3,     /* a stencil's saddle-point system had a zero pivot */
    RBF_EDIVERGED = -4,     /* non-finite field values appeared */
    RBF_ENOTCONVERGED = -5, /* step cap reached before the stopping criterion */
    RBF_ETIMEOUT = -6,      /* a device-side wait hit its iteration cap */
    RBF_ENOMEM = -7         /* device allocation failed */
};

enum { RBF_SOLVER_ACM = 0, RBF_SOLVER_LBM = 1 };
/* RBF_FP32C (ACM only): FP32 weights and FP32 stencil arithmetic, with u, v, w
 * and p carried as pairs of floats hi + lo (compensated summation of every field
 * update; stencil gathers read hi).  Per-step increments near the steady state
 * lie far below one float ulp of the fields; plain FP32 rounds them away and the
 * explicit iteration stalls short of the steady state, the pairs keep them.
 * rbf_get_fields returns hi + lo; rbf_set_fields splits each value into the
 * pair. */
/* RBF_FP32R (MLBM only): FP32 steps that converge to the FP64 fixed point.  The
 * state is f = f_b + d with an FP64 base f_b and an FP32 correction d.  Every
 * 64 steps a refresh folds d into f_b, takes one FP64 step of f_b and keeps its
 * residual r = F(f_b) - f_b in FP32 (d = r); the other steps advance only the
 * correction in FP32, d <- S(d) + r, with S the FP32 step without the body force
 * (the force is inside r).  At the steady state r vanishes in FP64, so the
 * result is the FP64 step's fixed point, while 63 of 64 steps move FP32 data.
 * Plain FP32 populations round every step's state to 2^-24 of the populations'
 * size; when the per-step forcing is a small fraction of it (the steady lattice
 * velocity is ~10^4 steps of forcing on the paper's resolutions) those roundings
 * add up to a bias of ~1e-4 in k/d^2.  Outputs read f_b + d in FP64. */
enum { RBF_FP64 = 0, RBF_FP32 = 1, RBF_FP32C = 2, RBF_FP32R = 3 };
enum { RBF_FLUID = 0, RBF_WALL = 1 };
/* operator ids for rbf_get_weights */
enum {
    RBF_OP_DX = 0, RBF_OP_DY = 1, RBF_OP_DZ = 2, RBF_OP_LAP = 3, /* ACM node operators */
    RBF_OP_LBM0 = 16                                            /* LBM: RBF_OP_LBM0 + k, k = 1..q-1 */
};

typedef struct rbf_ctx rbf_ctx;

/* Create a context on `device`.  cuda_stream: a cudaStream_t to order all work
 * on, or NULL for a stream the context creates and owns. */
int rbf_create(rbf_ctx **out, int device, void *cuda_stream);
int rbf_destroy(rbf_ctx *ctx);
const char *rbf_last_error(const rbf_ctx *ctx);

/* Nodes of the discretisation (meshless discretisation section).  n >= 2.
 *  xyz    n x 3 doubles in the periodic unit cell [0,1)^3 (cell side d = 1);
 *  type   n bytes, RBF_FLUID or RBF_WALL (wall nodes lie on the grain surface);
 *  normal n x 3 doubles; on wall nodes the unit normal pointing out of the solid
 *         into the fluid, ignored on fluid nodes (may be NULL if no wall nodes).
 * Resets stencils, weights and fields. */
int rbf_set_nodes(rbf_ctx *ctx, int64_t n, const double *xyz, const uint8_t *type,
                  const double *normal);

/* The grain: a sphere of radius r centred at c in the periodic cell (case
 * definition section).  Used for the solid mask of the permeability probes, the
 * wall area A of the drag quadrature and the porosity in the drag coefficient. */
int rbf_set_sphere(rbf_ctx *ctx, const double c[3], double r);

/* Stencils S_i: the n_l nearest nodes of every node by periodic distance, ordered
 * by (squared distance, caller's node index), so S_i(1) = i (meshless
 * discretisation section).  Wall nodes also get a Neumann stencil: the node
 * itself and its n_l - 1 nearest fluid nodes.  2 <= n_l <= 64. */
int rbf_build_stencils(rbf_ctx *ctx, int n_l);

/* Copy the stencils out: idx (n x n_l) caller's node indices. */
int rbf_get_stencils(rbf_ctx *ctx, int32_t *idx);

typedef struct {
    int64_t n_systems;   /* saddle systems solved */
    int64_t n_singular;  /* systems with a zero pivot (their weights are NaN) */
    double h_min;        /* smallest internodal distance min_i delta_i */
} rbf_weight_report;

/* RBF-FD weights, Eqs. operatorApprox, rbfScaling and augmentedSystem: PHS
 * r^phs_k (odd, >= 3) in the distance scaled by delta_i (distance from x_i to its
 * nearest neighbour), augmented with the C(mono_m + 3, 3) monomials of degree
 * <= mono_m; solved per node in FP64 by LU with partial pivoting.
 *  solver RBF_SOLVER_ACM: d/dx, d/dy, d/dz, Laplacian at every node, plus the
 *         gradient on every wall node's Neumann stencil.
 *  solver RBF_SOLVER_LBM: interpolation to the departure points x_i - dx e_k
 *         (k = 1..q-1, q = 15 or 19) at every node (MLBM section, L = 1), plus
 *         the gradient at wall nodes for the stress tensor.
 * Requires n_l >= C(mono_m + 3, 3).  rep may be NULL.  Returns RBF_ESINGULAR when
 * any system was singular (weights of those nodes are NaN). */
int rbf_compute_weights(rbf_ctx *ctx, int phs_k, int mono_m, int solver, int q, double dx,
                        rbf_weight_report *rep);

/* Copy one operator's FP64 weights out: out (n x n_l), caller's node order, row i
 * the weights of node i over its stencil rbf_get_stencils()[i]. */
int rbf_get_weights(rbf_ctx *ctx, int op, double *out);

typedef struct {
    int precision;   /* RBF_FP64, RBF_FP32, RBF_FP32C (ACM) or RBF_FP32R (LBM): storage and arithmetic of the steps */
    double nu;       /* kinematic viscosity */
    double g[3];     /* body acceleration */
    double rho;      /* density (ACM) / reference density (LBM); 0 -> 1 */
    /* ACM (MNS section) */
    double dt;       /* time step; <= 0 -> cfl * h_min^2 / (2 nu) */
    double cfl;      /* 0 -> 0.1 */
    double beta;     /* compressibility parameter of Eq. MNS_C; 0 -> 10 */
    double v_ref;    /* reference speed of Eq. MNS_C; <= 0 -> 0.01 |g| d^2 / nu */
    int n_p;         /* pressure iterations per step; 0 -> 3 */
    /* LBM (MLBM section) */
    double tau_plus; /* 0 -> 0.8 */
    double magic;    /* TRT Lambda = (tau+ - 1/2)(tau- - 1/2); 0 -> 3/16 */
} rbf_params;

/* Allocate and initialise the fields of the solver chosen in
 * rbf_compute_weights: ACM v = p = 0; LBM f = f_eq(rho = 1, v = 0) (MLBM section's
 * initial condition).  Resets the step counter. */
int rbf_init(rbf_ctx *ctx, const rbf_params *p);

/* Advance nsteps explicit steps (MNS or MLBM algorithm of the appendix). */
int rbf_step(rbf_ctx *ctx, int nsteps);

/* Fields in physical units, caller's node order: uvwp (n x 4) = (u, v, w, p).
 * LBM: v = (dx/dt) v_lb of the last pre-collision state, p = rho_ref (dx/dt)^2
 * c_s^2 (rho_lb - <rho_lb>) / <rho_lb>, <rho_lb> the node mean: the meshless
 * streaming does not conserve mass, and at the steady state the whole density
 * field keeps growing in proportion while v stays put, so the pressure is
 * taken relative to the current mean density (rbf_drag uses the same p). */
int rbf_get_fields(rbf_ctx *ctx, double *uvwp);
/* Set the ACM state (u, v, w, p) (a warm start or a restart); C of Eq. MNS_C is
 * recomputed from the new velocity.  LBM contexts: RBF_EINVAL. */
int rbf_set_fields(rbf_ctx *ctx, const double *uvwp);

/* LBM populations, unshifted, FP64, q x n (population-major), caller's node
 * order: the post-collision state the next step streams. */
int rbf_lbm_get_populations(rbf_ctx *ctx, double *f);
int rbf_lbm_set_populations(rbf_ctx *ctx, const double *f);

/* Which populations of a wall node are unknown in the streaming step and taken
 * from the opposite direction (Eq. interpolated_bounceback_mlbm):
 *   rule 0 (default): e_k . n > 0, n the wall normal (out of the solid; an exactly
 *          zero product counts as known);
 *   rule 1: the solid check of the touching-limit study (section "Permeability
 *          and drag coefficient for various porosities"): k is unknown when the
 *          departure point x + dx e_k' = x - dx e_k lies inside the solid, i.e.
 *          strictly closer than r to the nearest centre of the periodic sphere
 *          array (FP64, products and sums rounded separately, min image by rint).
 * The rule persists in the context: set it before or after rbf_compute_weights
 * (LBM), which recomputes the masks; rule 1 needs rbf_set_sphere.  Either call
 * may follow rbf_init (the next step uses the new masks).  Bad rule or missing
 * sphere -> RBF_EINVAL. */
int rbf_lbm_set_unknown_rule(rbf_ctx *ctx, int rule);
/* The unknown-population masks, caller's node order: bit k of mask[i] set when
 * population k of node i is bounced back (0 for fluid nodes).  mask: host array
 * of n uint32.  Needs LBM weights. */
int rbf_lbm_get_unknown_mask(rbf_ctx *ctx, uint32_t *mask);

/* Permeability, Eq. k_definition: probes on an m_p x m_p midpoint grid on each of
 * the planes x = 0, .2, .4, .6, .8; fluid probes interpolate v_x from their own
 * n_l nearest nodes (L = 1 weights centred at the probe), solid probes count as
 * zero; q = probe mean; k/d^2 = q nu / |g|.  FP64 accumulation (compensated FP32:
 * of hi + lo).  Needs rbf_set_sphere.  The probe set is built on the first call
 * and when m_p changes; a rebuild that fails keeps the previous probe set
 * (and its m_p) unchanged. */
int rbf_permeability(rbf_ctx *ctx, int m_p, double *k_over_d2, double *q);

/* Hydrodynamic force on the grain, Eqs. stress_tensor_force and
 * integration_force, F = (A / N_b) sum_b sigma . n over wall nodes, and the drag
 * coefficient K = F_x / (6 pi r phi q mu) of Eq. K_definition with q from
 * rbf_permeability(m_p).  FP64 accumulation (compensated FP32: of hi + lo). */
int rbf_drag(rbf_ctx *ctx, int m_p, double F[3], double *K);

/* Pointwise velocity difference of two solutions on the same nodes (the
 * cross-validation of the section "Pointwise comparison of the meshless
 * solvers", Eq. pointwise_error): per node, in the caller's node order,
 *   dv[i]    = |v_a(x_i) - v_b(x_i)|_2
 *   delta[i] = dv[i] / |v_b(x_i)|_2   (NaN where v_b(x_i) = 0, e.g. wall nodes)
 * with velocities in physical units (LBM: lattice velocity times dx/dt_LBM, the
 * same conversion as rbf_get_fields; compensated FP32: hi + lo).  The paper's
 * delta takes a = the MLBM context and b = the MNS context; any two initialised
 * contexts with the same node count on one device are accepted (the nodes are
 * not compared: the caller gives both the same rbf_set_case input).
 * delta, dv: host arrays of n doubles, either may be NULL.  a == b, different
 * devices or node counts -> RBF_EINVAL.  Runs on a's stream, then b's; both
 * streams are synchronised on return.  */
int rbf_pointwise_difference(rbf_ctx *a, rbf_ctx *b, double *delta, double *dv);

/* Relative velocity change |v - v_prev|_2 / |v|_2 over fluid nodes over the last
 * step (ACM), FP64 accumulation; computed when the last rbf_step ran with
 * residual tracking (rbf_solve does).  */
typedef struct {
    int64_t max_steps;   /* step cap */
    int check_every;     /* steps between convergence checks; 0 -> 100 */
    double tol;          /* ACM: relative velocity change per step; LBM: relative
                            change of k/d^2 between checks */
    int m_p;             /* probes per plane side for LBM checks; 0 -> 32 */
} rbf_solve_opts;

typedef struct {
    int64_t steps;       /* steps taken by this call */
    double residual;     /* last criterion value */
    double k_over_d2;    /* permeability at the end (probe grid m_p) */
    int converged;
} rbf_solve_result;

/* Step until the criterion holds or max_steps: returns RBF_OK or
 * RBF_ENOTCONVERGED (res filled in both cases), RBF_EDIVERGED on non-finite
 * fields.  ACM runs as one persistent cooperative kernel that checks the residual
 * on the device every check_every steps (RBF_ETIMEOUT if its grid barrier times
 * out); LBM steps in CUDA graphs and checks k/d^2 on the host. */
int rbf_solve(rbf_ctx *ctx, const rbf_solve_opts *opts, rbf_solve_result *res);

/* Device time of the last rbf_step (milliseconds, CUDA events on the context
 * stream), and the mean duration of one launch of the dominant step kernel over
 * that call (the fused LBM kernel; the ACM predictor).  */
int rbf_last_step_timing(rbf_ctx *ctx, double *total_ms, double *kernel_ms, int64_t *kernel_launches);

/* Advance nsteps steps with eager launches, timing every kernel launch with a
 * CUDA event pair on the context stream.  kernel_ms[c] receives the mean
 * duration (ms) of one launch of kernel class c; *n_classes the number of
 * classes: LBM 1 (the fused step); ACM 4 (predictor, pressure, wall pressure,
 * correction).  kernel_ms must hold 4 doubles.  1 <= nsteps <= 4096. */
int rbf_profile_steps(rbf_ctx *ctx, int nsteps, double *kernel_ms, int *n_classes);

/* Schedule of the fused LBM step (all compute the same step; only the thread
 * mapping and the population layout differ): 0 one node per thread, 256-thread
 * blocks; 1 one opposite-population pair per warp, (q-1)/2 warps per 32-node
 * slice, moments reduced in shared memory, stencil loop unrolled 5 deep
 * (default); 2 as 0 with 128-thread blocks; 3, 4, 5 as 1 unrolled 3, 6, 2 deep.
 * 0-5 keep the populations as the rest population plus interleaved opposite
 * pairs; 6 and 7 keep each node's q populations in one record of q rounded up
 * to a multiple of 4 values, read with 16-byte loads: 6 one node per thread,
 * 256-thread blocks; 7 the same with registers capped so that five blocks fit
 * on an SM; 8 and 9 as 6 in blocks of 128 and 64 threads (finer blocks spread
 * the nodes more evenly over the SMs); 10 as 6, launched as a programmatic
 * dependent launch (the next step's blocks are scheduled while this step drains
 * and wait on the grid dependency before touching memory).  Switching between the two layouts on an initialised LBM
 * context rewrites the state (one kernel launch); the populations, as
 * rbf_lbm_get_populations reports them, are unchanged.
 * On a context whose weights were computed for RBF_SOLVER_ACM the code selects the
 * mapping of the ACM sweeps of rbf_step instead: block + 1000 G, with block =
 * 64, 128 or 256 threads and G = 2 or 4 lanes per node, each lane summing every
 * G-th stencil column (write 0 for one lane per node, i.e. the code is the block
 * size; default 256).  RBF_EINVAL for any other code. */
int rbf_set_kernel_variant(rbf_ctx *ctx, int variant);

#define RBF_TUNE_MAX 16
typedef struct {
    int solver;          /* RBF_SOLVER_ACM or RBF_SOLVER_LBM */
    int n_candidates;
    int code[RBF_TUNE_MAX];  /* schedule codes of rbf_set_kernel_variant (rbf_autotune; LBM or
                                ACM) or persistent schedule codes (rbf_autotune_persistent) */
    double ms_per_step[RBF_TUNE_MAX];
    int chosen;          /* the fastest candidate, now in use */
} rbf_tune_report;

/* Autotuner: time every candidate schedule of the step kernels on this
 * context's own case (LBM: the eleven fused-step schedules; ACM: the sweep codes
 * 256, 128, 64, 2128, 2256, 4128, 4256 of rbf_set_kernel_variant), trial_steps steps each with CUDA events on
 * the context stream, keep the fastest.  The fields are saved before and restored
 * after the trials, so the state and step count are unchanged.  Needs rbf_init;
 * allocates a temporary copy of the state.  2 <= trial_steps <= 2000. */
int rbf_autotune(rbf_ctx *ctx, int trial_steps, rbf_tune_report *rep);

/* Autotuner of the persistent ACM driver (rbf_solve): time the schedules 256,
 * 128, 64, 32 (threads per block, one node per lane), 2128, 4128, 8128, 4256
 * (2, 4, 8, 4 lanes per node; codes as at rbf_set_persistent_block; the grid is
 * as many blocks as cover the work, at most the co-resident count, synchronised
 * by a software grid barrier) and, where the device can place them, one
 * thread-block cluster of 16 or 8 CTAs synchronised by the hardware cluster
 * barrier (codes -16, -8), over trial_steps steps each, CUDA events around the
 * launch, and keep the fastest for this context's later rbf_solve calls.  Fields
 * and step parity are saved before and restored after the trials.  ACM contexts
 * only; 2 <= trial_steps <= 20000.  rep->code[c] is the code of candidate c. */
int rbf_autotune_persistent(rbf_ctx *ctx, int trial_steps, rbf_tune_report *rep);
/* Schedule of the persistent ACM driver for this context, as a code:
 *   block + 1000 G   a cooperative grid of `block` (32, 64, 128, 256; default 256)
 *                    threads per block whose sweeps give each node G lanes (2, 4
 *                    or 8; write 0 for G = 1, i.e. the code is the block size):
 *                    the lanes split the node's stencil columns and combine their
 *                    partial sums with shuffles, multiplying the warps at work on
 *                    small cells;
 *   -8, -16          one cluster of 8 / 16 CTAs of 256 threads, G = 1.
 * A batch launches with its first cell's setting.  With G = 1 the schedule
 * changes only the order of the FP64 residual partial sums; G > 1 also changes
 * the order of the stencil sums (rounding only). */
int rbf_set_persistent_block(rbf_ctx *ctx, int code);

/* Wall-clock limit of one wait at a grid barrier of the persistent ACM driver
 * (rbf_solve, rbf_batch_solve with this context as the first cell): a block that
 * waits longer for the others raises the launch's error flag, every block leaves
 * its step loop at its next barrier, and the call returns RBF_ETIMEOUT; the
 * fields are then those of an unfinished step (call rbf_init or rbf_set_fields
 * before the next solve).  The paper has no counterpart; this is the driver's
 * failure detection.  Default 2 s; 1e-9 <= seconds <= 60, else RBF_EINVAL.  The
 * cluster schedules (codes -8, -16) synchronise with the hardware cluster barrier
 * and do not use it. */
int rbf_set_wait_limit(rbf_ctx *ctx, double seconds);

/* Number of kernel launches issued by this context since creation. */
int64_t rbf_launch_count(const rbf_ctx *ctx);

/* Physical time step of one rbf_step: ACM delta t = cfl h_min^2 / (2 nu) (the MNS
 * section) or the rbf_params value; LBM delta t = nu_lb dx^2 / nu (Eq.
 * conversion_factors).  Needs rbf_init.  For the stopping criterion of
 * Eq. stopCrit, whose window Delta t is in physical time. */
int rbf_time_step(rbf_ctx *ctx, double *dt);

/* ---- batched cells ----------------------------------------------------------
 * Many periodic cells (their own nodes, sphere and stencil size N_L), e.g. a
 * porosity sweep (the paper's section on various porosities).  The weight systems
 * of every node of every cell are solved in one launch (and the wall Neumann
 * systems of every cell in a second one); the ACM steps of all cells run in one
 * persistent cooperative launch, each cell stopping at its own criterion.
 * Each cell is an ordinary rbf_ctx (borrow it with rbf_batch_cell to read fields,
 * permeability or drag; it is owned by the batch). */
typedef struct rbf_batch rbf_batch;
typedef struct {
    int64_t steps;       /* steps this cell took in the last rbf_batch_solve */
    double residual;     /* its last relative velocity change */
    double k_over_d2;    /* its permeability (probe grid m_p) */
    int status;          /* 0 converged, 1 step cap, 2 non-finite */
} rbf_batch_cell_result;
int rbf_batch_create(rbf_batch **out, int device, void *cuda_stream);
int rbf_batch_destroy(rbf_batch *b);
const char *rbf_batch_last_error(const rbf_batch *b);
/* Add a cell (arguments as rbf_set_nodes, rbf_set_sphere and rbf_build_stencils);
 * returns the cell's index (>= 0) or a negative RBF_E* code.  At most 128 cells. */
int rbf_batch_add_cell(rbf_batch *b, int64_t n, const double *xyz, const uint8_t *type, const double *normal,
                       const double c[3], double r, int n_l);
/* Stencils of every cell, then the ACM weights (PHS r^phs_k + monomials of degree
 * <= mono_m) of all cells in one launch.  rep: totals and the smallest h_min. */
int rbf_batch_build(rbf_batch *b, int phs_k, int mono_m, rbf_weight_report *rep);
/* rbf_init on every cell (ACM; each cell gets its own dt from its own h_min). */
int rbf_batch_init(rbf_batch *b, const rbf_params *p);
/* Steady solve of all cells in one persistent launch: per-cell stop when the
 * relative velocity change (checked every opts->check_every steps) is below
 * opts->tol, or at opts->max_steps.  res: one entry per cell.  Returns RBF_OK
 * when every cell converged, RBF_ENOTCONVERGED otherwise (res filled),
 * RBF_ETIMEOUT if a grid barrier of the persistent kernel timed out. */
int rbf_batch_solve(rbf_batch *b, const rbf_solve_opts *opts, rbf_batch_cell_result *res);
/* rbf_autotune_persistent over all cells of the batch in one launch per trial
 * (the choice applies to every cell). */
int rbf_batch_autotune(rbf_batch *b, int trial_steps, rbf_tune_report *rep);
int rbf_batch_num_cells(const rbf_batch *b);
rbf_ctx *rbf_batch_cell(rbf_batch *b, int cell);

/* ---- learned warm start ------------------------------------------------------
 * The paper has no network; this is the build's warm start for the steady ACM
 * solve.  A multilayer perceptron maps 34 features of a node (sin and cos of
 * 2 pi n.x for 16 integer wave vectors n, periodic in the cell; the grain radius
 * r; the signed wall distance phi_sdf) to (u, v, w, p) divided by |g| d^2 / nu.
 * Layers 64 -> 128 -> 128 -> 128 -> 128 -> 16 (features zero-padded from 34 to 64,
 * outputs 4..15 unused and held at zero), GELU (tanh form) after the first four.
 * Forward and backward run as BF16 tensor-core GEMMs (tcgen05, FP32 accumulation
 * in tensor memory); Adam (beta1 0.9, beta2 0.999, eps 1e-8) on FP32 masters.
 * Loss: mean squared error over the 4 outputs.  Parameters are one FP32 vector:
 * per layer W (fan_out x fan_in, row-major) then b (fan_out), layers in order. */
typedef struct rbf_mlp rbf_mlp;
int64_t rbf_mlp_num_params(void);
int rbf_mlp_create(rbf_mlp **out, int device, void *cuda_stream);
int rbf_mlp_destroy(rbf_mlp *mlp);
const char *rbf_mlp_last_error(const rbf_mlp *mlp);
/* Set / get the FP32 parameters (rbf_mlp_num_params() floats); set also resets
 * the Adam moments and step counters. */
int rbf_mlp_set_params(rbf_mlp *mlp, const float *theta);
int rbf_mlp_get_params(rbf_mlp *mlp, float *theta);
/* Training samples (copied): n node positions (n x 3), per-sample radius and wall
 * distance, targets (n x 4, already divided by |g| d^2 / nu). */
int rbf_mlp_set_data(rbf_mlp *mlp, int64_t n, const double *xyz, const float *radius, const float *sdf,
                     const float *target);
/* `steps` Adam steps on mini-batches of `batch` samples (a multiple of 128) drawn
 * with the counter-based SplitMix64: sample = splitmix64(seed * 2^32 + s * batch +
 * b) mod n for draw s (counted since rbf_mlp_set_params).  loss_hist (steps
 * floats, may be NULL) receives each step's mean squared error.  Returns
 * RBF_ETIMEOUT if a tensor-core wait exceeded its limit. */
int rbf_mlp_train(rbf_mlp *mlp, int steps, int batch, double lr, uint64_t seed, float *loss_hist);
/* Gradient (rbf_mlp_num_params() floats, packed like the parameters) and mean
 * squared error of the given samples (batch a multiple of 128), no update. */
int rbf_mlp_gradient(rbf_mlp *mlp, int batch, const int64_t *sample_idx, float *grad, double *loss);
/* Network output for n points: out (n x 4) in the scaled units of the targets. */
int rbf_mlp_predict(rbf_mlp *mlp, int64_t n, const double *xyz, const float *radius, const float *sdf, float *out);
/* Warm start: write scale[c] x output c of the prediction at the context's nodes
 * into its ACM fields (c = 0..3: u, v, w, p; velocity zero on wall nodes; the low
 * words of an RBF_FP32C context zeroed) and recompute C of Eq. MNS_C.  The
 * context must be an initialised ACM context with a sphere, on the same device.
 * scale: 4 doubles (host). */
int rbf_mlp_warm_start(rbf_mlp *mlp, rbf_ctx *ctx, const double *scale);
int64_t rbf_mlp_launch_count(const rbf_mlp *mlp);
/* Training-step schedule (rbf_mlp_train, rbf_mlp_gradient): 1 (default) two fused
 * kernels per step, each CTA carrying 128-row tiles through all five layers with
 * the weights resident in shared memory (forward, then backward with the weight
 * and bias gradients added by vector reductions, so their summation order varies
 * from run to run); 0 one tensor-core GEMM launch per layer and pass with
 * split-batch weight gradients reduced in a fixed order.  Same rounding points in
 * both. */
int rbf_mlp_set_fused(rbf_mlp *mlp, int fused);

/* Permeability exactly as rbf_permeability(m_p), for callers that cannot allocate
 * device memory at this point: for example code whose device memory is owned by
 * another allocator (a framework's caching pool, or an arena sized at start-up
 * that leaves nothing for cudaMalloc), or a loop in which the device-wide
 * synchronisation of cudaMalloc / cudaFree is not acceptable.  The paper has no
 * counterpart; this is a deployment variant of the probe reduction.
 *  - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 *  - Its scratch (4096 block partials and their sum) is one static device array
 *    of 4097 doubles (32,776 bytes) that every GPU loading the library holds
 *    until exit.  rbf_create looks up the array's device address (with the
 *    context's device current) and the context keeps it, so the address is
 *    valid for the context's whole life; this call looks nothing up.
 *  - The probe set must already exist: call rbf_permeability(ctx, m_p, ...) once
 *    first (it builds the probes, which allocates), else RBF_EINVAL.
 *  - At most 1,048,576 fluid probes; more returns RBF_EINVAL.
 *  - All calls share the one array, so calls that overlap on the GPU (other
 *    contexts or streams on the same device) race; serialise them.  Each call
 *    overwrites the partials it uses, so nothing needs clearing.
 *  - Compensated FP32 (RBF_FP32C) reads hi + lo, like rbf_permeability.
 *  - Writes *k_over_d2 and *q (either may be NULL) before returning. */
int rbf_permeability_static(rbf_ctx *ctx, int m_p, double *k_over_d2, double *q);

#ifdef __cplusplus
}
#endif
#endif
