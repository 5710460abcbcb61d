/*
 * frsg.h - C ABI of the GB300 flux reconstruction stochastic Galerkin (FR-SG) library.
 *
 * The library advances the stochastic Galerkin system of a hyperbolic conservation law
 * (Xiao, Kusch, Koellermeier, Frank, arXiv 2112.05946, §2.1, Eq. 6) discretised in
 * physical space by flux reconstruction (§3) with the Radau (DG) correction, in random
 * space by an orthonormal Legendre gPC expansion of one uniform variable z ~ U(-1, 1)
 * with Gauss quadrature (§2.1, Eqs. 2-5), stabilised by the detector-switched modal
 * filter (§4.1-4.2) and the positivity-preserving limiter (§4.3), in time by the
 * three-stage strong-stability-preserving Runge-Kutta scheme.
 *
 * Conventions shared by every call:
 *  - State layout ("uhat"): element x solution point x gPC mode x variable, row major,
 *    uhat[((e * Np + j) * M + k) * S + s], Np = (P+1)^dim, M = N + 1.  In 2D the element
 *    index is e = ey * nx + ex and the point index j = b * (P+1) + a (a along x).
 *    Nodal-in-z arrays use the same order with Q quadrature nodes in place of M modes.
 *  - A context owns every device buffer it allocates; caller pointers are borrowed for
 *    the duration of the call only.  DEVICE pointers must live on the context's device;
 *    work is stream-ordered on the context's stream (no hidden device synchronisation,
 *    except in calls that return host data, which synchronise that stream).
 *  - Errors are returned as frsg_status; nothing throws across the ABI.  The message of
 *    the last error is kept in the context (fr_sg_last_error).  Errors found by kernels
 *    (non-finite values, inadmissible element means) are latched in a device word and
 *    reported by the next call that synchronises (fr_sg_check, or any call with host output).
 *  - Precision: FRSG_FP64 keeps the state in double; FRSG_FP32 and FRSG_FP32_TC keep it in
 *    float and compute the residual in float, with the limiter's exact test, the time-step
 *    reduction and the moments in double.  Calls that take "void*" state use the context's
 *    precision (float for both float forms); calls that take "double*" always use double.
 */
#ifndef FRSG_H
#define FRSG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct frsg_ctx frsg_ctx;

typedef enum {
    FRSG_OK = 0,
    FRSG_E_INVAL = 1,        /* bad argument or unsupported combination of sizes */
    FRSG_E_NOMEM = 2,        /* device or host allocation failed */
    FRSG_E_CUDA = 3,         /* a CUDA runtime call failed */
    FRSG_E_NONFINITE = 4,    /* a kernel produced NaN or Inf */
    FRSG_E_POSITIVITY = 5,   /* an element mean has rho <= 0 or p <= 0 (§4.3 cannot apply) */
    FRSG_E_TIMEOUT = 6,      /* a bounded device wait gave up */
    FRSG_E_UNSUPPORTED = 7   /* valid request the library does not implement */
} frsg_status;

enum { FRSG_BC_PERIODIC = 0, FRSG_BC_DIRICHLET = 1, FRSG_BC_OUTFLOW = 2, FRSG_BC_REFLECT = 3 };
enum { FRSG_EQ_ADVECTION = 0, FRSG_EQ_BURGERS = 1, FRSG_EQ_EULER = 2 };
enum { FRSG_FILTER_NONE = 0, FRSG_FILTER_EXP = 1, FRSG_FILTER_L2 = 2, FRSG_FILTER_LASSO = 3 };
/* Interface flux: local Lax-Friedrichs, or HLL with the Davis signal speeds
 * S_L = min(lambda_min(u_L), lambda_min(u_R)), S_R = max(lambda_max(u_L), lambda_max(u_R)). */
enum { FRSG_FLUX_LLF = 0, FRSG_FLUX_HLL = 1 };
/* Precision forms.  FRSG_FP32_TC: the FP32 form with the Galerkin projection of the residual
 * (§2.1, Eq. 6 with the quadrature of Eq. 5) on the tensor cores (tcgen05 MMA, tf32 operands
 * split into a tf32 part and a float remainder, three products accumulated in FP32: float
 * accuracy); 2D elements with P = 3, Q = 8 and at most 8 gPC modes (FRSG_E_INVAL otherwise),
 * tiles of 4 or 8 elements. */
enum { FRSG_FP64 = 0, FRSG_FP32 = 1, FRSG_FP32_TC = 2 };
enum { FRSG_HOST = 0, FRSG_DEVICE = 1 };

/* Problem description.  Plain old data; struct_size must be sizeof(frsg_config). */
typedef struct {
    uint32_t struct_size;
    int32_t dim;              /* 1 or 2 */
    int32_t nx, ny;           /* elements along x (and y); uniform mesh (§3.1, line and quad maps) */
    double x0, x1, y0, y1;    /* domain [x0, x1] (x [y0, y1]) */
    int32_t bc[4];            /* x-left, x-right, y-bottom, y-top: FRSG_BC_*; periodic pairs must match */
    int32_t P;                /* polynomial degree in x: P+1 Gauss-Legendre solution points (§3.2) */
    int32_t N;                /* gPC degree: M = N+1 orthonormal Legendre modes (§2.1, Eq. 2) */
    int32_t Q;                /* Gauss points in z for the Galerkin projection (§2.1, Eq. 5) */
    int32_t equation;         /* FRSG_EQ_* */
    double adv_speed;         /* advection speed a (FRSG_EQ_ADVECTION) */
    double gamma;             /* ratio of specific heats (FRSG_EQ_EULER) */
    int32_t filter;           /* FRSG_FILTER_*: exponential (§4.1.1), L2 (§4.1.2) or Lasso (§4.1.3,
                                 1D only: soft threshold with strengths picked per element and
                                 variable so that the top physical and random modes vanish) */
    int32_t sensor;           /* 1: filter only elements with theta < 0.99 (§4.2); 0: every element */
    double f_alpha, f_s;      /* exponential filter strength alpha and order s (N_* = 0) */
    double f_eps1, f_eps2;    /* L2 filter damping of the last physical / random mode (§4.1.2, Eq. 39) */
    double s0, kappa;         /* detector parameters (§4.2, Eq. 47), log10 scale */
    int32_t limiter;          /* 1: positivity-preserving limiter on every stage input (§4.3) */
    int32_t precision;        /* FRSG_FP64, FRSG_FP32 or FRSG_FP32_TC */
    int32_t flux;             /* FRSG_FLUX_LLF (§3.3) or FRSG_FLUX_HLL (Euler setup tables of §5.3-5.4),
                                 evaluated pointwise at every z-node of every face */
} frsg_config;

/* Create a context: validates the configuration, builds the tables of §2.1 and §3 on
 * the host (Gauss-Legendre points and weights, Lagrange derivative matrix, Radau
 * correction derivatives, gPC evaluation and projection matrices, Vandermonde),
 * uploads them, allocates the state and two stage buffers on the current device.
 * stream: a cudaStream_t (NULL = legacy default stream).
 * Limits: dim 1 with 1 <= P <= 4, or dim 2 with 1 <= P <= 3; 0 <= N <= 15; 1 <= Q <= 32;
 * nx, ny >= 1 (>= 2 along a periodic direction).
 * Returns FRSG_E_INVAL (with *out = NULL) for anything else. */
frsg_status fr_sg_init(const frsg_config* cfg, void* stream, frsg_ctx** out);

/* Release every resource of the context.  NULL is accepted. */
void fr_sg_destroy(frsg_ctx* ctx);

/* Message of the last failed call on this context ("" if none).  Owned by the context. */
const char* fr_sg_last_error(const frsg_ctx* ctx);

/* Sizes: E elements, Np points per element, M modes, S variables, Q z-nodes.
 * Any output pointer may be NULL. */
frsg_status fr_sg_sizes(const frsg_ctx* ctx, int* E, int* Np, int* M, int* S, int* Q);

/* Replace the stream used by all later calls. */
frsg_status fr_sg_set_stream(frsg_ctx* ctx, void* stream);

/* Host copies of the node coordinates the library uses: x[E*Np] (and y[E*Np] in 2D, else
 * ignored; may be NULL) of the solution points, z[Q] of the random-space nodes.  A caller
 * evaluates initial or boundary data at these nodes for the two projection calls below. */
frsg_status fr_sg_get_nodes(const frsg_ctx* ctx, double* x, double* y, double* z);

/* Host copies of the quadrature weights the library uses: wx[Np] Gauss-Legendre weights of
 * the solution points on the reference element (tensor products in 2D; they sum to 2^dim),
 * wz[Q] probability weights of the z-nodes (they sum to 1).  Either pointer may be NULL. */
frsg_status fr_sg_get_quadrature(const frsg_ctx* ctx, double* wx, double* wz);

/* Dirichlet ghost state of one boundary side (0..3 as in cfg->bc), given as host values
 * g[Q][S] at the z-nodes; projected onto the gPC modes like the initial data (§2.1, Eq. 6,
 * third line).  The ghost state is constant along the side. */
frsg_status fr_sg_set_boundary_nodal(frsg_ctx* ctx, int side, const double* g);

/* Initial condition from values at the solution points and z-nodes: u0[E][Np][Q][S]
 * (double, HOST or DEVICE per `where`), projected on the device:
 * uhat_k(x_j) = sum_q w_q u0(x_j, z_q) Phi_k(z_q)   (§2.1, Eq. 6, third line, with Eq. 5). */
frsg_status fr_sg_set_initial_nodal(frsg_ctx* ctx, const double* u0, int where);

/* Galerkin projection of nodal values onto the gPC modes, out of place and without touching
 * the context's state (§2.1, Eq. 6, third line): uhat[e][j][k][s] = sum_q wz_q Phi_k(z_q)
 * u0[e][j][q][s].  u0 [E][Np][Q][S] and uhat [E][Np][M][S]: DEVICE double arrays on the
 * context's stream (FRSG_E_INVAL for FRSG_HOST).  Asynchronous. */
frsg_status fr_sg_project(frsg_ctx* ctx, const double* u0, double* uhat, int where);

/* Transpose of fr_sg_project, for gradients with respect to the initial data and the
 * parameters it depends on: g[e][j][q][s] = sum_k wz_q Phi_k(z_q) gbar[e][j][k][s].  gbar
 * [E][Np][M][S] and g [E][Np][Q][S]: DEVICE double arrays.  Asynchronous. */
frsg_status fr_sg_project_transpose(frsg_ctx* ctx, const double* gbar, double* g, int where);

/* Copy the state in (set) or out (get) in the canonical double layout [E][Np][M][S],
 * converting from or to float in FRSG_FP32 contexts.  HOST variants synchronise. */
frsg_status fr_sg_set_state(frsg_ctx* ctx, const double* uhat, int where);
frsg_status fr_sg_get_state(frsg_ctx* ctx, double* uhat, int where);

/* Semi-discrete residual dudt = L(u) of the FR-SG system, no limiter and no filter:
 * z-evaluation (§2.1, Eq. 2), flux (§3.2, Eq. 15), Galerkin projection (Eq. 6), face
 * interpolation and the interface flux (LLF or HLL, §3.3), total-flux derivative
 * with the Radau correction (§3.4, Eq. 21; 2D §3.5, Eq. 24).  u and dudt: DEVICE arrays
 * [E][Np][M][S] in the context's precision, 16-byte aligned (FRSG_E_INVAL otherwise: the
 * kernels move four-variable states with vector loads and stores); they must not overlap.
 * Boundary ghost states come from the context. */
frsg_status fr_sg_rhs(frsg_ctx* ctx, const void* u, void* dudt);

/* Advance the context's state by nsteps steps of size dt of the SSP-RK3 scheme, each
 * stage being: limit the stage input (§4.3, if enabled), Euler update with the residual,
 * SSP combination, detector and filter (§4.1-4.2, if enabled) - the forward-Euler
 * sequence of §4.3, Eq. 53 applied per stage.  The exponential filter uses dt (§4.1.1).
 * Asynchronous; errors found on the device are reported by fr_sg_check.
 * use_graph = 1 replays the three stage launches from a captured CUDA graph. */
frsg_status fr_sg_rk_step(frsg_ctx* ctx, double dt, int nsteps, int use_graph);

/* One call from a state to a state: copy uhat_in in (as fr_sg_set_state), take nsteps steps
 * of fr_sg_rk_step, copy the result out to uhat_out (as fr_sg_get_state).  where: FRSG_HOST
 * (host arrays; an FRSG_FP32 context reads and writes pinned ones in place from its
 * conversion kernels, and copies others through a staging buffer) or FRSG_DEVICE (device arrays), both
 * double [E][Np][M][S]; uhat_in and uhat_out may be the same array.  A HOST call synchronises
 * once, at the end, instead of once per copy; a DEVICE call is asynchronous.  FRSG_E_INVAL
 * for null arrays, a bad where, dt <= 0 or nsteps < 0 (the state is then unchanged); device
 * errors as fr_sg_rk_step. */
frsg_status fr_sg_advance(frsg_ctx* ctx, const double* uhat_in, double* uhat_out, int where, double dt, int nsteps,
                          int use_graph);
/* fr_sg_advance with the arrays in the context's own precision: double for FRSG_FP64, float
 * [E][Np][M][S] for FRSG_FP32 and FRSG_FP32_TC.  The same steps; a float context moves half
 * the bytes over the host link (it rounds a double input to float anyway, and widening its
 * float state to double is exact, so nothing is lost).  Host arrays go through the copy
 * engines (pinned ones without staging).  Errors as fr_sg_advance. */
frsg_status fr_sg_advance_native(frsg_ctx* ctx, const void* uhat_in, void* uhat_out, int where, double dt, int nsteps,
                                 int use_graph);

/* Advance the context's state by nsteps steps of size dt of the classical four-stage
 * Runge-Kutta scheme (the integrator of the advection study, §5.1 setup table):
 * y1 = u + dt/2 L(u), y2 = u + dt/2 L(y1), y3 = u + dt L(y2),
 * u <- u + dt/6 (L(u) + 2 L(y1) + 2 L(y2) + L(y3)).  Each stage limits its input (§4.3, if
 * enabled) and runs the detector and filter on its output y_i and on the new state (§4.1-4.2,
 * if enabled); the weighted sum of the residuals is not filtered.  The first call allocates
 * one more state-sized device buffer, kept until fr_sg_destroy.  Decisions loaded by
 * fr_sg_set_replay are consumed one row per stage (four per step); steps taken while rows
 * remain run without the graph.  use_graph = 1 replays the four stage launches from a
 * captured CUDA graph.  Asynchronous; device errors as fr_sg_rk_step. */
frsg_status fr_sg_rk4_step(frsg_ctx* ctx, double dt, int nsteps, int use_graph);

/* Issue stage `stage` (0, 1, 2) of one SSP-RK3 step of size dt: stage 0 reads the state
 * and writes the first stage buffer, stage 1 reads it and writes the second, stage 2 reads
 * the second and writes the state.  Calling stages 0, 1, 2 in order is one
 * fr_sg_rk_step(ctx, dt, 1, 0); separate calls let a caller time or interleave stages. */
frsg_status fr_sg_stage(frsg_ctx* ctx, int stage, double dt);

/* Events (cudaEvent_t, created by the caller) that fr_sg_stage records on the context's
 * stream: before_limiter before the limiter launch (§4.3), before_stage between it and the
 * stage kernel, after_stage after the stage kernel (before the float forms' cell-mean update,
 * which follows it), so that a caller can time each kernel of
 * a stage with the same launches as fr_sg_rk_step (replayed decisions are not consumed while
 * events are set).  Any may be NULL; all NULL (the default) records nothing.  The events are
 * borrowed until they are replaced. */
frsg_status fr_sg_set_timing_events(frsg_ctx* ctx, void* before_limiter, void* before_stage, void* after_stage);

/* Detector + filter (§4.1-4.2) on the current state with step size dt. */
frsg_status fr_sg_filter(frsg_ctx* ctx, double dt);

/* Positivity-preserving limiter (§4.3, Eqs. 48-52) on the current state (Euler only). */
frsg_status fr_sg_limit(frsg_ctx* ctx);

/* Mean and variance over z at each solution point: mean = uhat_0, var = sum_{k>=1} uhat_k^2
 * (orthonormal basis, §2.1, Eq. 3).  mean, var: double [E][Np][S], HOST or DEVICE. */
frsg_status fr_sg_moments(frsg_ctx* ctx, double* mean, double* var, int where);

/* FP64 cell means of the gPC mean mode: mbar[e][s] = sum_j (w_j / 2^dim) uhat[e][j][0][s], the
 * element mean over r (and s) and z (§4.3), host or device double [E][S].  In the float forms
 * (FRSG_FP32, FRSG_FP32_TC) these means are carried in FP64 from step to step: every SSP-RK3
 * stage moves them by the difference of the interface fluxes' mean-mode projections on the
 * element's faces, one stored value per face (so that the sum over a periodic mesh is conserved
 * to FP64 rounding: the filter keeps the mean, §4.1, Lambda_00 = 1, and the limiter scales about
 * it, §4.3), and the float state's mean mode is shifted by a constant per element and variable
 * to match them.  A state written directly (fr_sg_set_state, fr_sg_set_initial_nodal,
 * fr_sg_advance, fr_sg_filter), an RK4 step or a batch step re-anchors them on the float state.
 * In FRSG_FP64 they are computed from the state.  A HOST call synchronises. */
frsg_status fr_sg_cell_means(frsg_ctx* ctx, double* mbar, int where);

/* dt = cfl * h / lambda_max, lambda_max the largest flux-Jacobian spectral radius over
 * solution points and z-nodes of the current state, h the smallest element width.
 * Synchronises; *dt is a host double. */
frsg_status fr_sg_cfl_dt(frsg_ctx* ctx, double cfl, double* dt);

/* Decisions of the three stages of the last fr_sg_rk_step step (or of the last
 * fr_sg_filter / fr_sg_limit call, in row 0): filter_on[3][E] (1 = detector flagged the
 * element and the filter ran), beta[3][E] (limiter scaling, 1 = untouched).  Host arrays;
 * either may be NULL.  Synchronises. */
frsg_status fr_sg_get_decisions(frsg_ctx* ctx, uint8_t* filter_on, double* beta);

/* Replay mode: when flags is non-NULL, the next stages take their filter decisions from
 * flags[nstages][E] (host array, copied) in order instead of the detector, one row per
 * stage, until the rows run out; NULL switches replay off.  Graph replay is disabled
 * while rows remain. */
frsg_status fr_sg_set_replay(frsg_ctx* ctx, const uint8_t* flags, int nstages);

/* Synchronise the context's stream and report (and clear) errors latched by kernels. */
frsg_status fr_sg_check(frsg_ctx* ctx);

/* Batch of independent 1D problems advanced together (uneven sizes, degrees and gPC orders).
 * The paper treats one problem at a time; a batch exists so that many small uncertain
 * instances fill the GPU.  fr_sg_batch_create takes n existing contexts (borrowed; they must
 * outlive the batch), all 1D, scalar (advection or Burgers), without limiter, with the same
 * equation and precision (FRSG_E_INVAL otherwise), and builds per-problem stage arguments and
 * a tile list (at most 256/Q elements per tile, largest tiles first).
 * fr_sg_batch_rk_step advances every member by nsteps SSP-RK3 steps, member i with step size
 * dt[i] (host array of n): each stage is ONE persistent launch over all tiles of all members
 * (grid = SMs x resident CTAs), the three stages replayed from a captured CUDA graph when
 * use_graph = 1.  Each member's state, decisions and error word stay in its context. */
typedef struct frsg_batch frsg_batch;
frsg_status fr_sg_batch_create(frsg_ctx* const* ctxs, int n, void* stream, frsg_batch** out);
void fr_sg_batch_destroy(frsg_batch* b);
frsg_status fr_sg_batch_rk_step(frsg_batch* b, const double* dt, int nsteps, int use_graph);
uint64_t fr_sg_batch_launch_count(const frsg_batch* b);
/* Tile count, persistent grid size and dynamic shared memory per CTA of the batched launch. */
frsg_status fr_sg_batch_info(const frsg_batch* b, int* ntiles, int* grid, size_t* smem);

/* Batched discrete adjoint (the adjoint below for every member of a batch at once): members
 * FRSG_FP64, periodic, LLF flux, no filter or the exponential / L2 filter (FRSG_E_UNSUPPORTED
 * otherwise).
 * fr_sg_batch_forward_record advances every member by nsteps SSP-RK3 steps, member i with step
 * size dt[i] (host array of n), one persistent launch per stage over all members' tiles, and
 * keeps on the device each member's state every checkpoint_every steps and the filter decision
 * of every stage (arenas owned by the batch, grown on demand).
 * fr_sg_batch_adjoint maps nset cotangent sets at once: lambda_T[c n + i] (DEVICE double
 * [E_i][Np_i][M_i], member i of set c) to grad_u0[c n + i] (same layout; host arrays of nset n
 * device pointers, 1 <= nset <= 64).  Each segment between checkpoints is recomputed for all
 * members with the recorded decisions, then walked back: one launch per stage covers every
 * member and every set, the filter transpose applied to the cotangent tile in shared memory.
 * The members' states are not touched.
 * fr_sg_batch_forward_replay advances every member from its current state by nsteps <= the
 * recorded steps with the recorded step sizes and filter decisions (the frozen-decision forward
 * map the adjoint differentiates; for finite-difference checks), keeping nothing.
 * fr_sg_batch_integral_moments: per member i, q[2 i] = E[I] and q[2 i + 1] = Var[I] of
 * I(z) = integral of u(x, z) over the domain for the members' current states (host array of
 * 2 n; the orthonormal gPC basis of §2.1, Eq. 3: E[I] is mode 0 of I, Var[I] the sum of the
 * squares of its other modes), and their gradients with respect to the gPC coefficients in
 * dmean[i] / dvar[i] (device pointers, layout of the state; either table may be NULL).  Needs a
 * recorded run (its member tables); synchronises the batch's stream. */
frsg_status fr_sg_batch_forward_record(frsg_batch* b, const double* dt, int nsteps, int checkpoint_every);
frsg_status fr_sg_batch_forward_replay(frsg_batch* b, int nsteps);
frsg_status fr_sg_batch_adjoint(frsg_batch* b, int nset, double* const* lambda_T, double* const* grad_u0);
frsg_status fr_sg_batch_integral_moments(frsg_batch* b, double* q, double* const* dmean, double* const* dvar);

/* Discrete adjoint of fr_sg_rk_step for 1D FRSG_FP64 contexts with no filter, the
 * exponential or the L2 filter: periodic advection / Burgers with the LLF flux, or Euler with
 * the LLF or HLL flux, any 1D boundary kind, with or without the positivity limiter
 * (FRSG_E_UNSUPPORTED otherwise).  The paper has no adjoint; it is the exact transpose of the
 * linearised scheme of §2.1-§4.3 with the filter decisions of the forward run frozen, the
 * Lax-Friedrichs dissipation max(lambda_L, lambda_R) and the HLL branch and signal speeds
 * min / max differentiated along the branch the forward values take (ties shared equally), and the
 * limiter differentiated through its scalings beta_1 and beta_2 (eps held constant; the
 * minimising points are those of the forward values).
 *
 * fr_sg_forward_record advances the state by nsteps steps of size dt (as fr_sg_rk_step) and
 * keeps, on the device, a checkpoint of the state every checkpoint_every steps and the
 * filter decision of every stage.  Allocates its buffers on first use (and when a longer
 * run needs more).
 * fr_sg_adjoint then maps lambda_T = dQ/du(T) (DEVICE double [E][Np][M][S]) to
 * grad_u0 = dQ/du(0) (DEVICE double, same layout) for the recorded run: each segment between
 * checkpoints is recomputed with the recorded decisions replayed, then walked backwards
 * stage by stage.  The context's state is the recorded final state again when it returns. */
frsg_status fr_sg_forward_record(frsg_ctx* ctx, double dt, int nsteps, int checkpoint_every);
frsg_status fr_sg_adjoint(frsg_ctx* ctx, const double* lambda_T, double* grad_u0);

/* Elements per CTA of the stage kernel (the tile): te >= 1 sets it, te = 0 restores the
 * automatic choice.  Returns FRSG_E_INVAL when the tile does not fit in shared memory or
 * exceeds 512 threads.  *te_out (may be NULL) receives the tile in use. */
frsg_status fr_sg_set_tile(frsg_ctx* ctx, int te, int* te_out);

/* Layout of the 1D stage kernel: 0 = one thread per (z-node, element), looping over the
 * element's solution points; 1 (the default for 1D) = one thread per (z-node, point,
 * element); 2 = layout 0, with the three stages of an SSP-RK3 step in ONE cooperative launch
 * separated by grid-wide barriers (1D without limiter; a barrier that waits longer than
 * about 2 s latches FRSG_E_TIMEOUT and the kernel returns); 3 = the three stages of an SSP-RK3
 * step in ONE launch without grid barriers: each CTA loads its tile with three elements of
 * halo on each side and recomputes the halo's stages on chip, in layout 1's arithmetic (1D
 * without limiter; FRSG_E_UNSUPPORTED when no tile fits: 7*Q*(P+1) > 1024, or every tile's
 * grid too large to be resident at once).  Before storing the step, a
 * CTA waits until the CTAs reading its elements as halo have loaded them (a wait longer than
 * about 2 s latches FRSG_E_TIMEOUT and the CTA stores nothing, while other CTAs may have stored:
 * the state is then partly advanced and must be reloaded); the tile is the number of
 * elements a CTA finishes, and the launch is refused (FRSG_E_CUDA from the step) when its
 * grid cannot be resident at once.  With layout 3, single stages (fr_sg_stage, fr_sg_rhs,
 * the recorded run) run layout 1.  All compute the same stage; the tile is re-chosen
 * automatically.  2D contexts accept only 0 (FRSG_E_UNSUPPORTED otherwise). */
frsg_status fr_sg_set_variant(frsg_ctx* ctx, int variant);

/* Test hook of the one-launch step (layout 3 of fr_sg_set_variant).  wait_cycles > 0 bounds the
 * neighbour wait before the final store to that many SM clock cycles (0 restores the default of
 * about 2 s).  hold_tile >= 0 (layout 3 only; FRSG_E_UNSUPPORTED otherwise, FRSG_E_INVAL past the
 * last tile) adds 2^40 to that tile's launch counter, as if a CTA reading its elements as halo had
 * never loaded them: in the next step that tile's wait cannot be met, so after wait_cycles it
 * latches FRSG_E_TIMEOUT (reported by fr_sg_check) and stores nothing, while the other tiles store
 * their new elements; the counters are re-zeroed before the step after.  After FRSG_E_TIMEOUT from
 * this layout the state is therefore partly advanced: reload it before stepping on.  Drops the
 * cached step graphs.  Synchronises. */
frsg_status fr_sg_test_fused_wait(frsg_ctx* ctx, long long wait_cycles, int hold_tile);

/* Autotuner: times graph-replayed SSP-RK3 steps from the context's current state with its last
 * step size (1e-3 if none was set), so it should run on a representative admissible state, e.g.
 * after the initial state and one step (reps per candidate, default 20; CUDA
 * events on the context's stream around each step, the L2 cache overwritten before it, so that
 * every candidate reads its state from HBM) for every layout (1D) and tile that fits, re-times
 * the three fastest in five interleaved rounds, keeps the best and caches the choice per
 * (dim, P, N, Q, S, precision, elements, filter, equation, interface flux, limiter) for the
 * process.  A cached shape is not re-timed.  Saves and restores the state (two temporary
 * device allocations: the state and twice the L2 size); overwrites the stage buffers and the
 * decision rows; replayed decisions are not consumed.  Synchronises.  variant_out / te_out
 * (may be NULL) receive the choice. */
frsg_status fr_sg_autotune(frsg_ctx* ctx, int reps, int* variant_out, int* te_out);

/* Write the process-wide autotuner cache to a text file (one line per problem shape), or
 * merge such a file into it, so that a later process reuses the choices without timing.
 * Host only; FRSG_E_INVAL for a NULL path, an unreadable or unwritable file, or a malformed
 * line (nothing is merged then). */
frsg_status fr_sg_tune_cache_save(const char* path);
frsg_status fr_sg_tune_cache_load(const char* path);

/* Number of kernel launches issued on this context since creation (graph replays count
 * each captured kernel).  Host counter; never synchronises. */
uint64_t fr_sg_launch_count(const frsg_ctx* ctx);

/* Allocation-free variant of fr_sg_rk_step for 1D problems in FRSG_FP64.  The paper has no
 * counterpart: this entry point exists for callers, not for the method.
 *
 * Some callers may not allocate device memory.  Examples are code whose GPU memory is owned
 * by another allocator (a framework's caching pool, or an arena reserved at start-up) and
 * code on a latency-critical path: cudaMalloc and cudaFree can synchronise the device and
 * fragment the owner's pool, so such callers must not trigger them.  This call takes the
 * caller's input and output state and allocates nothing: no context, no cudaMalloc, no
 * cudaFree, no allocating library routine, and only fixed-size host storage.  Its scratch
 * (two stage buffers, the tables, the step size, the ghost modes and an error word) is one
 * static __device__ array of 8 MiB, which every GPU that loads this library keeps until the
 * process exits.  A problem whose stage buffers and tables do not fit (about 500,000 state
 * values) is rejected with FRSG_E_INVAL and a message on stderr.
 *
 * cfg: as for fr_sg_init, with dim = 1 and precision = FRSG_FP64 (FRSG_E_UNSUPPORTED otherwise).
 * ghost_modes: host [4][M][S] gPC modes of the Dirichlet sides' ghost states (the modes that
 *   fr_sg_set_boundary_nodal computes), or NULL when no side is Dirichlet (FRSG_E_INVAL when a
 *   Dirichlet side has none).
 * u_in, u_out: device double [E][Np][M][S]; u_out receives the state after nsteps steps of
 *   size dt of the same scheme as fr_sg_rk_step (limiter, residual, SSP combination, detector
 *   and filter per stage); u_in == u_out is allowed.
 * stream: a cudaStream_t.  The work is enqueued there and the call synchronises that stream
 *   before it returns, so that it can report the errors kernels latch (FRSG_E_NONFINITE,
 *   FRSG_E_POSITIVITY).  A call that fails after it has queued work (FRSG_E_CUDA) also waits
 *   for that work before it returns.
 * The first call on a device looks up the device address of the static array, with that
 * device current; make that first call before any stream capture.  Every call shares the
 * array and leaves its contents behind: each call clears what must start at zero (the
 * error word) and overwrites the rest before reading it.  Calls that overlapped on the GPU
 * would race on the shared array, so the library runs them one at a time: a call holds a
 * process-wide lock until its stream work has finished. */
frsg_status fr_sg_rk_step_noalloc(const frsg_config* cfg, const double* ghost_modes, const double* u_in,
                                  double* u_out, double dt, int nsteps, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FRSG_H */
