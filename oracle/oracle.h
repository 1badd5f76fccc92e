/*
 * CPU oracle for the component-decomposed two-level ADMM for ACOPF
 * (Kim & Kim, "Accelerated Computation and Tracking of AC Optimal Power Flow
 * Solutions Using GPUs", arXiv 2110.06879).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded FP64
 * restatement of Algorithm 1 and of every subproblem it solves (eq. acopf,
 * eq. branch, eq. qp-bound, eq. qp-bus, the multiplier rules of Section III-B).
 * Only the test-suite, the smoke check and the CPU-baseline leg of the bench
 * may load it.  It shares no code with the CUDA library.
 *
 * Parity status: the paper prints no worked example, so every function here is
 * pinned by mathematics instead (closed forms, KKT conditions, brute force,
 * finite differences, complex power S = V (Y V)^*, an independent NLP solve of
 * the whole tiny ACOPF); see tests/test_oracle_*.py.
 *
 * Index conventions (shared with the library's public header because they
 * define the canonical output layout, not because code is shared):
 *   coupling vector, length m = 2 ngen + 8 nbranch:
 *     [2g + 0] p_g,  [2g + 1] q_g                       (generator g)
 *     [2 ngen + 8l + k], k = 0..7 :
 *        p_ij, q_ij, p_ji, q_ji, w_i(ij), theta_i(ij), w_j(ij), theta_j(ij)
 *   branch variables (6 per branch): v_i, v_j, theta_i(ij), theta_j(ij), s_ij, s_ji
 *   bus incidence row of bus i: branch ends in increasing branch id (from-end
 *   entry 2l, to-end entry 2l + 1), then generators (entry 2 nbranch + g) in
 *   increasing id.
 */
#ifndef ORACLE_H
#define ORACLE_H

#include <stdint.h>

typedef struct {
    int32_t nbus, nbranch, ngen, ref_bus;
    double base_mva;
    const double *pd, *qd, *gs, *bs, *vmin, *vmax;                    /* [nbus]    */
    const int32_t *f_bus, *t_bus;                                     /* [nbranch] */
    const double *r, *x, *b, *tap, *shift, *rate_a;                   /* [nbranch] */
    const int32_t *gen_bus;                                           /* [ngen]    */
    const double *pmin, *pmax, *qmin, *qmax, *c2, *c1, *c0;           /* [ngen]    */
} ora_grid;

typedef struct {
    double rho_pq, rho_va, obj_scale, line_limit_frac;
    double beta0, beta_factor, z_decay, beta_max, lambda_max, tol_in0, tol_in_decay;
    double al_rho0, al_tol, al_decay, al_rho_factor, al_rho_max;
    double tron_gtol, tron_ftol, tron_xtol;
    int32_t two_level, max_outer, max_inner, al_max_iter, tron_max_iter, beta_rule;
} ora_options;

/* One branch subproblem (eq. branch) with all data it needs. */
typedef struct {
    double Y[8];            /* g_ii b_ii g_ij b_ij g_ji b_ji g_jj b_jj           */
    double lo[6], hi[6];    /* bounds of (v_i, v_j, th_i, th_j, s_ij, s_ji)       */
    double xbar[8], z[8], y[8], rho[8];   /* coupling data, order as above      */
    double lt[2];           /* lambda-tilde of the two line-limit equalities     */
    double rt;              /* rho-tilde                                         */
    double alpha;           /* Cauchy step length carried into the next TRON
                               call and back out of it (<= 0: start at 1)       */
} ora_branch_prob;

/* counters of one branch solve (or summed over many) */
typedef struct {
    int64_t tron_calls, tron_iters, fgh_evals, f_evals, cauchy_trials,
            cg_iters, ps_trials, al_passes, tron_maxiter_hits;
} ora_stats;

typedef struct ora ora;

/* whole-problem interface */
ora *ora_create(const ora_grid *g, const ora_options *o);
void ora_destroy(ora *p);
void ora_cold_start(ora *p);
int ora_set_loads(ora *p, const double *pd, const double *qd);
int ora_set_gen_bounds(ora *p, const double *pmin, const double *pmax);
void ora_set_ramp_limit(ora *p, double frac);
int ora_solve(ora *p, double tol, int32_t max_iter, int32_t warm_start);
int ora_get(const ora *p, int32_t which, double *out);
void ora_get_residuals(const ora *p, double *dres, int32_t *ires);
int32_t ora_get_history(const ora *p, double *out, int32_t cap);
void ora_get_stats(const ora *p, ora_stats *s);
void ora_get_csr(const ora *p, int32_t *row_ptr, int32_t *col);
void ora_get_admittance(const ora *p, double *Y8);
void ora_finalize(const ora *p, double *pg, double *qg, double *vm, double *va,
                  double *pf, double *qf, double *pt, double *qt, double *obj_maxviol);

/* single-subproblem interface (pins) */
void ora_admittance(double r, double x, double b, double tap, double shift, double *Y8);
void ora_branch_fgh(const ora_branch_prob *bp, const double *x, double *f, double *g, double *H);
void ora_branch_flows(const double *Y8, const double *x, double *flows4);
int ora_tron(ora_branch_prob *bp, double *x, const ora_options *o, ora_stats *st);
void ora_branch_solve(ora_branch_prob *bp, double *x, const ora_options *o, ora_stats *st);
double ora_gen_solve(double cost2, double cost1, double rho, double xbar, double z, double y,
                     double lo, double hi);

/* vector ids for ora_get */
enum { ORA_U = 0, ORA_XBAR = 1, ORA_Z = 2, ORA_Y = 3, ORA_LAMBDA = 4, ORA_BRANCH_X = 5,
       ORA_BRANCH_LT = 6, ORA_BUS = 7, ORA_RHO = 8 };

#endif
