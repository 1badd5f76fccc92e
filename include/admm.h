/*
 * admm.h -- C ABI of libadmm.so, a GB300 (sm_103a) FP64 implementation of the
 * component-decomposed two-level ADMM for AC optimal power flow of Kim & Kim,
 * "Accelerated Computation and Tracking of AC Optimal Power Flow Solutions
 * Using GPUs" (arXiv 2110.06879).
 *
 * One handle holds one grid -- or a batch of independent grids ("scenarios",
 * admm_create_batch) -- resident on the current CUDA device.  Every iteration
 * of Algorithm 1 runs on the device, for all scenarios at once:
 *   branch_tron  -- eq. branch per branch (TRON inside an augmented Lagrangian on
 *                   the line limits, Section II-C / III-B); a persistent launch in
 *                   which each lane solves one branch at a time from a work queue;
 *   bus_dual     -- eq. qp-bound for generators, eq. qp-bus per bus over a CSR
 *                   incidence map (no atomics), the z update (eq. qp-bound with
 *                   infinite bounds), the y update (Section III-B) and the
 *                   primal/dual residual reduction with a device convergence flag;
 * captured once as a CUDA graph whose conditional WHILE node repeats the
 * iteration until the device flag says stop, so a solve costs one graph launch
 * and one stream synchronisation (Section III: no host-device traffic during
 * the iteration).
 *
 * Conventions
 *   - Every pointer argument is a HOST pointer unless its name starts with d_.
 *   - The caller owns every buffer it passes; the library copies inputs during
 *     the call and writes outputs before it returns.  The handle owns all device
 *     memory it allocates, until admm_destroy.
 *   - Indices are 0-based int32.  Powers, voltages and impedances are per unit on
 *     base_mva; angles (and the branch shift) in radians; costs in $/MW^2h,
 *     $/MWh and $/h (MATPOWER units: c2' = c2 base^2, c1' = c1 base on per-unit
 *     power).
 *   - Functions return ADMM_OK (0) or a status below; no exception crosses the
 *     ABI.  A handle is not thread-safe; calls on one handle must be serialised.
 *   - Canonical coupling order (length m = 2 ngen + 8 nbranch), used by every
 *     per-coupling output: [2g] p_g, [2g+1] q_g for generator g, then for branch
 *     l at 2 ngen + 8 l + k, k = 0..7: p_ij, q_ij, p_ji, q_ji, w_i(ij),
 *     theta_i(ij), w_j(ij), theta_j(ij) (Section II-B duplicated variables,
 *     i = from bus, j = to bus).
 */
#ifndef ADMM_H
#define ADMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct admm_handle admm_handle;   /* opaque; owned by the library */

enum {
    ADMM_OK = 0,                 /* converged (or the requested work finished)     */
    ADMM_NOT_CONVERGED = 1,      /* iteration caps reached; state stays valid       */
    ADMM_ERR_INVALID_ARG = -1,   /* rejected input; nothing changed                 */
    ADMM_ERR_CUDA = -2,          /* a CUDA call failed; see admm_last_error()       */
    ADMM_ERR_NUMERICAL = -3,     /* a residual became NaN/Inf; iteration stopped    */
    ADMM_ERR_OOM = -4            /* device allocation failed                        */
};

/* Grid data (eq. acopf, Section II-A).  Every bus must have at least one
 * incident branch; branches may not connect a bus to itself.  tap == 0 means 1.
 * rate_a <= 0 means an unlimited line. */
typedef struct {
    int32_t nbus, nbranch, ngen, ref_bus;
    double base_mva;
    const double *pd, *qd, *gs, *bs, *vmin, *vmax;                   /* [nbus]    */
    const int32_t *f_bus, *t_bus;                                    /* [nbranch] */
    const double *r, *x, *b, *tap, *shift, *rate_a;                  /* [nbranch] */
    const int32_t *gen_bus;                                          /* [ngen]    */
    const double *pmin, *pmax, *qmin, *qmax, *c2, *c1, *c0;          /* [ngen]    */
} admm_grid;

/* Method parameters.  rho_pq / rho_va are the fixed penalties of Table 1
 * (generation and flow couplings / voltage couplings), obj_scale the objective
 * multiplier of Section IV-A, line_limit_frac the 99% tightening of
 * Section IV-A, max_outer / max_inner the caps of Section IV-A.  The remaining
 * constants are this library's readings of what the paper leaves open (outer
 * update, line-limit augmented Lagrangian, TRON tolerances). */
typedef struct {
    double rho_pq, rho_va, obj_scale, line_limit_frac;
    double beta0;          /* initial outer penalty; <= 0 selects 10 rho_va        */
    double beta_factor;    /* beta growth when ||z|| stalls (6)                      */
    double z_decay;        /* ||z|| must fall below this fraction per outer step (0.8) */
    double beta_max;       /* cap on beta (1e12)                                     */
    double lambda_max;     /* projection bound of the outer multiplier (1e12)        */
    double tol_in0;        /* inner tolerance at outer step k: max(tol, tol_in0 *    */
    double tol_in_decay;   /*   tol_in_decay^k)  (1e-2, 0.5)                         */
    double al_rho0;        /* initial rho-tilde of a branch solve; <= 0: 25 rho_pq / rbar^2,
                              rbar the tightened rating (rho_pq without a limit)  */
    double al_tol;         /* line-limit AL stops when max|h| <= al_tol (1e-6)       */
    double al_decay;       /* rho-tilde grows unless max|h| fell below this share (0.1)  */
    double al_rho_factor;  /* rho-tilde growth (100)                                 */
    double al_rho_max;     /* cap on rho-tilde (1e12)                                */
    double tron_gtol;      /* TRON: ||P(x-g)-x||_inf <= gtol max(1, start value) (1e-10) */
    double tron_ftol;      /* TRON: model trusted when the predicted decrease is below
                              ftol max(1,|f|), f = sum rho/2 (u-t)^2 + AL terms (1e-12) */
    double tron_xtol;      /* TRON: stop on ||s||_inf <= xtol max(1, ||x||_inf) (1e-13) */
    int32_t two_level;     /* 1: two-level algorithm; 0: z == 0 (one level)          */
    int32_t max_outer, max_inner;   /* 20, 1000 (Section IV-A)                        */
    int32_t al_max_iter;   /* 20 */
    int32_t tron_max_iter; /* 200 */
    int32_t use_graph;     /* 1: conditional-WHILE CUDA graph; 0: stream launches   */
    int32_t branch_blocks; /* resident blocks of 128 branch lanes; 0: two per SM when the
                              branches fill them, else one per SM              */
    int32_t graph_body_iters; /* iterations per body of the WHILE node, 1..16 (1); the
                                 loop still stops after exactly the iteration that
                                 converges or reaches max_iter                       */
    int32_t beta_rule;     /* outer penalty growth at an outer update: 0 (default) times
                              beta_factor when ||z|| > z_decay ||z_prev||; 1 (adaptive)
                              times min(beta_factor, max(1, (||z|| / (z_decay ||z_prev||))^2)) */
    int32_t lanes_per_branch; /* lanes solving one branch subproblem: 1 (0 means 1) or 2
                                 (a lane pair splits the two line ends' flows and the
                                 rows of the 6x6 products; the iterates agree with the
                                 one-lane kernel to rounding, not bitwise)           */
} admm_options;

typedef struct {
    int32_t iters;          /* inner iterations of the last solve                    */
    int32_t outer_iters;    /* outer updates of the last solve                       */
    int32_t status;         /* return code of the last solve                         */
    int32_t tron_failures;  /* TRON solves that hit tron_max_iter in the last solve  */
    double primal_res;      /* ||u - xbar||_2 over all couplings (last iteration)    */
    double dual_res;        /* ||rho (xbar - xbar_prev)||_2                          */
    double z_norm;          /* ||z||_2                                               */
    double primal_z;        /* ||u - xbar + z||_2 (inner residual)                   */
    double beta;            /* current outer penalty                                 */
    double eps_pri;         /* sqrt(m) tol + tol max(||u||, ||xbar||) (last iteration) */
    double eps_dual;        /* sqrt(m) tol + tol ||y||                               */
    double objective;       /* generation cost at the last admm_get_solution        */
    double max_viol;        /* ||c(x)||_inf at the last admm_get_solution           */
} admm_residuals;

/* Fill *o with the defaults listed above (rho_pq 10, rho_va 1e3, Table 1). */
void admm_default_options(admm_options *o);

/* Validate the grid, compute the pi-model admittances (Section II-A), build
 * the bus->incident-component CSR map (rows: branch ends in increasing branch
 * id, from-end first, then generators in increasing id), allocate the device
 * state on the current device and cold-start it (Section IV-B).
 * o == NULL selects the defaults.  On success *out owns the handle. */
int admm_create(const admm_grid *g, const admm_options *o, admm_handle **out);

/* A batch of nscen independent grids in one handle (grids[0..nscen-1], each
 * validated like admm_create).  Their components are concatenated into one set
 * of device arrays (a flattened component index); every iteration solves all
 * branch subproblems of all running scenarios in one persistent launch and all
 * bus rows in one launch, while each scenario keeps its own loop counters,
 * penalties, tolerance and stopping decision (a per-scenario convergence mask).
 * Bus blocks never straddle scenarios, so a scenario's reductions -- and thus
 * its iterates -- are the same as when it is solved alone.  Per-scenario calls
 * (set_loads*, set_gen_bounds, set_ramp_limit, get_solution, get_residuals,
 * get_vector, get_csr) address the scenario chosen by admm_select_scenario
 * (0 after creation).  admm_create is the batch of one. */
int admm_create_batch(const admm_grid *grids, int32_t nscen, const admm_options *o,
                      admm_handle **out);
void admm_destroy(admm_handle *h);

/* Number of scenarios of the handle (0 for NULL). */
int32_t admm_scenario_count(admm_handle *h);
/* Address scenario s (0 <= s < count) with the per-scenario calls. */
int admm_select_scenario(admm_handle *h, int32_t s);

/* Run all device work of this handle on the given cudaStream_t (NULL: the
 * legacy default stream).  The stream must outlive its use by the handle.
 * Work already queued on the previous stream is ordered before everything
 * queued on the new one (an event recorded on the old stream, waited on by
 * the new); the call does not block the host. */
int admm_set_stream(admm_handle *h, void *cuda_stream);

/* Replace the bus loads (host arrays [nbus]) -- the tracking input of
 * Section IV-C.  admm_set_loads_device takes device pointers instead; both are
 * ordered on the handle's stream. */
int admm_set_loads(admm_handle *h, const double *pd, const double *qd);
int admm_set_loads_device(admm_handle *h, const double *d_pd, const double *d_qd);

/* Replace the generator real-power bounds (host arrays [ngen]), e.g. ramp
 * limits around the previous dispatch when tracking (Section IV-C). */
int admm_set_gen_bounds(admm_handle *h, const double *pmin, const double *pmax);

/* Ramp limit of Section IV-C for the next solve: the generator real-power
 * bounds become [max(pmin, pg - frac pmax), min(pmax, pg + frac pmax)] around
 * the current dispatch pg (on the device), where pmin, pmax are the bounds last
 * given to admm_create or admm_set_gen_bounds (the paper uses frac = 0.02).
 * The next admm_set_gen_bounds replaces them.  Ordered on the handle's stream. */
int admm_set_ramp_limit(admm_handle *h, double frac);

/* Algorithm 1.  warm_start = 0 re-initialises every variable (Section IV-B);
 * 1 keeps all primal, dual and penalty values (Section IV-C) and restarts only
 * the loop counters.  The tests are the standard ADMM ones with absolute and
 * relative tolerance tol (they loosen with the number m of couplings, as
 * Section IV-B notes): stops with ADMM_OK when ||u - xbar|| <= eps_pri,
 * ||rho dxbar|| <= eps_dual and (two-level only) ||z|| <= eps_pri, where
 * eps_pri = sqrt(m) tol + tol max(||u||, ||xbar||) and
 * eps_dual = sqrt(m) tol + tol ||y||; the inner loop ends when
 * ||u - xbar + z|| and ||rho dxbar|| pass the same tests at tol_in.  Otherwise
 * ADMM_NOT_CONVERGED after max_iter inner iterations or max_outer outer
 * updates.  Blocks until done. */
int admm_solve(admm_handle *h, double rho_pq, double rho_va, double tol, int32_t max_iter,
               int32_t warm_start);
/* Same, without waiting: the work is enqueued on the handle's stream; read the
 * outcome with admm_get_residuals after synchronising that stream.  With
 * several scenarios both calls start every scenario with the same arguments;
 * admm_solve returns ADMM_OK only when all of them converged (the most severe
 * error otherwise). */
int admm_solve_async(admm_handle *h, double rho_pq, double rho_va, double tol, int32_t max_iter,
                     int32_t warm_start);

/* Continuous batching.  admm_slot_begin (re)starts scenario s alone -- cold
 * (warm_start = 0, Section IV-B) or from its resident state (1, Section IV-C)
 * -- with its own penalties, tolerance and iteration cap; other scenarios keep
 * running or idle.  admm_run enqueues at most max_iters iterations of the
 * batched loop (one CUDA-graph launch) over the scenarios that are running;
 * it returns early on the device once none is.  Both are asynchronous on the
 * handle's stream; scenarios begun while a run is queued join the next run.
 * admm_slot_status waits for the stream and writes, per scenario, 2 while it is
 * still running or else its solve status (ADMM_OK, ADMM_NOT_CONVERGED, ...),
 * and its iteration count; either pointer may be NULL. */
int admm_slot_begin(admm_handle *h, int32_t s, double rho_pq, double rho_va, double tol,
                    int32_t max_iter, int32_t warm_start);
int admm_run(admm_handle *h, int32_t max_iters);
int admm_slot_status(admm_handle *h, int32_t *status, int32_t *iters);

/* Section IV-A solution: pg, qg [ngen] from the generator subproblems, vm, va
 * [nbus] from the bus subproblems (vm = sqrt(w)), branch flows pf, qf, pt, qt
 * [nbranch] recomputed from the bus voltages.  Any pointer may be NULL.  Also
 * computes the objective and ||c(x)||_inf reported by admm_get_residuals. */
int admm_get_solution(admm_handle *h, double *pg, double *qg, double *vm, double *va, double *pf,
                      double *qf, double *pt, double *qt);
int admm_get_residuals(admm_handle *h, admm_residuals *out);

/* Per-iteration residual history of scenario 0's last solve: rows of 4
 * doubles (primal, dual, z_norm, primal_z); returns the number of rows written
 * (at most cap; the device keeps the last 65536 iterations). */
int32_t admm_get_history(admm_handle *h, double *out, int32_t cap);

/* Copy one state vector to a host buffer, in canonical order:
 *   ADMM_VEC_U, _XBAR, _Z, _Y, _LAMBDA, _RHO : [m] per coupling
 *   ADMM_VEC_BRANCH_X  : [nbranch][6] v_i, v_j, theta_i(ij), theta_j(ij), s_ij, s_ji
 *   ADMM_VEC_BRANCH_LT : [nbranch][2] lambda-tilde of the two line-limit rows
 *   ADMM_VEC_BUS       : [nbus][2] w, theta
 *   ADMM_VEC_ADMITTANCE: [nbranch][8] g_ii b_ii g_ij b_ij g_ji b_ji g_jj b_jj */
enum { ADMM_VEC_U = 0, ADMM_VEC_XBAR = 1, ADMM_VEC_Z = 2, ADMM_VEC_Y = 3, ADMM_VEC_LAMBDA = 4,
       ADMM_VEC_BRANCH_X = 5, ADMM_VEC_BRANCH_LT = 6, ADMM_VEC_BUS = 7, ADMM_VEC_RHO = 8,
       ADMM_VEC_ADMITTANCE = 9 };
int admm_get_vector(admm_handle *h, int32_t which, double *out);

/* The CSR bus -> incident-component map: row_ptr [nbus+1], col [2 nbranch + ngen]
 * with entry 2l (+1) the from (to) end of branch l and 2 nbranch + g generator g. */
int admm_get_csr(admm_handle *h, int32_t *row_ptr, int32_t *col);

/* Counters of the last run (summed over all branches): TRON calls, TRON
 * iterations, gradient/Hessian evaluations, function evaluations, Cauchy
 * trials, CG iterations, projected-search trials, AL passes, TRON cap hits. */
int admm_get_stats(admm_handle *h, int64_t *out9);

/* Checkpoint: the full iteration state of every scenario as an opaque host
 * blob.  Call with buf == NULL to get the size in *len.  admm_set_state accepts
 * only a blob of the same shape; a following warm solve continues the saved
 * trajectory. */
int admm_get_state(admm_handle *h, void *buf, size_t *len);
int admm_set_state(admm_handle *h, const void *buf, size_t len);

/* One scenario's iteration state as an opaque host blob (paging a grid out
 * of a handle and back into this or another handle that holds the same grid
 * as one of its scenarios): the same arrays as admm_get_state, restricted to
 * scenario s, and its outer penalty and pending outer step.  Inputs (loads,
 * generator bounds) are not part of it.  Call with buf == NULL to get the
 * size in *len.  admm_set_scenario_state accepts a blob of the same shape
 * (bus, branch, generator and slot counts) only for a scenario that is not
 * running; a following warm start of that scenario continues the saved
 * trajectory bitwise.  Both synchronise the handle's stream. */
int admm_get_scenario_state(admm_handle *h, int32_t s, void *buf, size_t *len);
int admm_set_scenario_state(admm_handle *h, int32_t s, const void *buf, size_t len);

/* Device bytes admm_create_batch would allocate for these grids (the one
 * state allocation of the handle; the iteration graph and the CUDA context
 * come on top), without touching the device: what a server admits against a
 * device-memory budget.  Only the sizes of the grids are read. */
int admm_device_bytes(const admm_grid *grids, int32_t nscen, size_t *bytes);

/* Tracing: run `iters` inner iterations from the current state (warm, no
 * convergence stop) with stream launches and CUDA events around each kernel on
 * the handle's stream; ms_out[0] = mean branch_tron time, ms_out[1] = mean
 * bus_dual time, ms_out[2] = mean time of one whole iteration, in ms.  Blocks. */
int admm_profile_iterations(admm_handle *h, int32_t iters, double *ms_out);

/* Allocation-free z / y update (the paper has no counterpart; it serves
 * callers).  Some callers cannot call cudaMalloc: a control loop whose device
 * memory is fixed once at start-up, or a program whose device memory all
 * belongs to another allocator and which must not let a library allocate
 * behind its back.  This entry point runs the z update, the y update and the
 * residual norms of one inner iteration, elementwise over the m couplings, on
 * buffers the caller owns, and allocates nothing: its only scratch (per-block
 * partial sums and a ticket counter) is a static device array of 128 KiB +
 * 32 B that every GPU loading the library keeps until the process exits.
 *   m                  couplings, 1 <= m <= 16,777,216 (larger m is rejected
 *                      with ADMM_ERR_INVALID_ARG)
 *   d_u, d_xbar        component-side values and bus-side copies [m]
 *   d_xbar_prev        bus-side copies of the previous iteration [m]
 *   d_rho, d_lambda    penalties and outer multipliers [m]
 *   beta, two_level    outer penalty (>= 0); two_level = 0 keeps z at 0
 *   d_z, d_y           in: previous z, y; out: updated z, y [m]
 *   d_norms            out [4]: ||u - xbar||, ||u - xbar + z||,
 *                      ||rho (xbar - xbar_prev)||, ||z|| (Euclidean)
 *   cuda_stream        stream the work is ordered on (NULL: legacy stream)
 * All d_ pointers are device pointers on the current device.  The first call
 * on each device looks up the scratch array's device address (with that
 * device current); make that first call before any stream capture.  Every
 * call shares the one scratch array, so calls whose work overlaps on a GPU
 * race: order them on one stream.  Returns ADMM_OK, ADMM_ERR_INVALID_ARG or
 * ADMM_ERR_CUDA; the work is asynchronous. */
int admm_dual_update_noalloc(int64_t m, const double *d_u, const double *d_xbar,
                             const double *d_xbar_prev, const double *d_rho,
                             const double *d_lambda, double beta, int32_t two_level,
                             double *d_z, double *d_y, double *d_norms, void *cuda_stream);

/* Autotuner over the launch shape.  (1) Lanes per branch and resident
 * branch_tron blocks: one lane with 1/2, 3/4, 1, 3/2 or 2 blocks of 128 lanes
 * per SM, two lanes with 1 or 2 blocks per SM; each candidate is timed on the
 * same `iters` warm iterations of every scenario replayed from a device copy
 * of the current state, twice (forward and reverse order); the fastest mean
 * branch_tron time wins.  (2) With the graph path, iterations per body of the
 * WHILE node (1, 2, 4), each timed through the graph over 4 * iters replayed
 * iterations.  The choice is kept for later solves (the graph is rebuilt) and
 * the state is put back, so the tuner changes no iteration of the current
 * state; the block count and the graph shape never change a result, the lane
 * count changes iterates at rounding level.  Allocates one temporary device
 * buffer the size of the iteration state (ADMM_ERR_OOM if that fails).
 * Outputs may be NULL: *blocks_out the block count, *body_out the iterations
 * per graph body, *ms_best the fastest mean branch_tron time in ms,
 * *lanes_out the lanes per branch. */
int admm_autotune(admm_handle *h, int32_t iters, int32_t *blocks_out, int32_t *body_out,
                  double *ms_best, int32_t *lanes_out);

/* Roofline calibration (the paper has no counterpart): one launch of an
 * FP64-FMA-only kernel (2 blocks of 256 threads per SM, eight independent FMA
 * chains per thread, `iters` trips) on the given stream (NULL: legacy stream),
 * timed with CUDA events; blocks until done.  out3[0] = achieved GFLOP/s,
 * out3[1] = SM clock in MHz during the launch (clock64 cycles over global-timer
 * nanoseconds on one SM), out3[2] = FMAs per clock per SM sub-partition.
 * Allocates and frees two small device buffers.  Returns ADMM_OK,
 * ADMM_ERR_INVALID_ARG (iters < 1, out3 NULL), ADMM_ERR_OOM or ADMM_ERR_CUDA. */
int admm_fp64_peak(int32_t iters, void *cuda_stream, double *out3);

const char *admm_status_string(int status);
/* Text of the last error recorded by any call in this process (thread-local). */
const char *admm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
