/*
 * CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * A plain single-threaded FP64 restatement of the paper's method, written for
 * reading against the paper, not for speed:
 *   Section II-A  eq. acopf and the pi-model admittances        -> ora_admittance
 *   Section II-C  eq. branch (branch augmented Lagrangian)       -> branch_fgh
 *   Section III-B TRON (Lin-More) with Steihaug CG              -> ora_tron
 *   Section II-C  augmented Lagrangian on the line limits       -> ora_branch_solve
 *   Section III-B eq. qp-bound (generators, z), eq. qp-bus, multiplier rules
 *   Section III   Algorithm 1 (two-level loop)                  -> ora_solve
 *   Section IV-A/B solution extraction, initialisation          -> ora_finalize, ora_cold_start
 * Readings of points the paper leaves open are listed next to the code that
 * takes them.  Compile with -ffp-contract=off.
 */
#include "oracle.h"

#include <complex.h>
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NV 6                   /* branch variables */
#define TWO_PI 6.283185307179586476925286766559

/* ------------------------------------------------------------------ */
/* Section II-A: admittance entries of the pi model with turns ratio a  */
/* ------------------------------------------------------------------ */
void ora_admittance(double r, double x, double b, double tap, double shift, double *Y8)
{
    double complex ys = 1.0 / (r + I * x);             /* series admittance */
    double complex ysh = I * b;                         /* total line charging */
    double t = (tap == 0.0) ? 1.0 : tap;                /* tap 0 means 1 */
    double complex a = t * cexp(I * shift);
    double complex yii = (ys + 0.5 * ysh) / (creal(a) * creal(a) + cimag(a) * cimag(a));
    double complex yij = -ys / conj(a);
    double complex yji = -ys / a;
    double complex yjj = ys + 0.5 * ysh;
    Y8[0] = creal(yii); Y8[1] = cimag(yii);
    Y8[2] = creal(yij); Y8[3] = cimag(yij);
    Y8[4] = creal(yji); Y8[5] = cimag(yji);
    Y8[6] = creal(yjj); Y8[7] = cimag(yjj);
}

/* ------------------------------------------------------------------ */
/* Flow expressions eq. (pij)-(qji) with w_i = v_i^2, wR = v_i v_j cos(th),  */
/* wI = v_i v_j sin(th), th = th_i - th_j (Section II-C), and their first  */
/* and second derivatives with respect to (v_i, v_j, th_i, th_j).          */
/* Each flow has the shape  a_self * v_k^2 + v_i v_j T(th),                 */
/* T(th) = alpha cos th + beta sin th.                                      */
/* ------------------------------------------------------------------ */
typedef struct { double val, d[NV], h[NV][NV]; } fterm;

static void flow_term(double a_self, int self_is_i, double alpha, double beta,
                      double vi, double vj, double c, double s, fterm *o)
{
    double T = alpha * c + beta * s;
    double Tp = -alpha * s + beta * c;      /* dT/dth  */
    double vv = vi * vj;
    memset(o, 0, sizeof(*o));
    double vk = self_is_i ? vi : vj;
    o->val = a_self * vk * vk + vv * T;
    o->d[0] = (self_is_i ? 2.0 * a_self * vi : 0.0) + vj * T;
    o->d[1] = (self_is_i ? 0.0 : 2.0 * a_self * vj) + vi * T;
    o->d[2] = vv * Tp;
    o->d[3] = -vv * Tp;
    o->h[0][0] = self_is_i ? 2.0 * a_self : 0.0;
    o->h[1][1] = self_is_i ? 0.0 : 2.0 * a_self;
    o->h[0][1] = T;
    o->h[0][2] = vj * Tp;
    o->h[0][3] = -vj * Tp;
    o->h[1][2] = vi * Tp;
    o->h[1][3] = -vi * Tp;
    o->h[2][2] = -vv * T;
    o->h[2][3] = vv * T;
    o->h[3][3] = -vv * T;
    for (int a = 0; a < NV; ++a)
        for (int b = 0; b < a; ++b) o->h[a][b] = o->h[b][a];
}

/* u_c(x) for the eight couplings of a branch, with derivatives */
static void branch_couplings(const double *Y, const double *x, fterm u[8])
{
    double vi = x[0], vj = x[1], th = x[2] - x[3];
    double c = cos(th), s = sin(th);
    double gii = Y[0], bii = Y[1], gij = Y[2], bij = Y[3];
    double gji = Y[4], bji = Y[5], gjj = Y[6], bjj = Y[7];
    flow_term(gii, 1, gij, bij, vi, vj, c, s, &u[0]);     /* p_ij eq. (pij) */
    flow_term(-bii, 1, -bij, gij, vi, vj, c, s, &u[1]);   /* q_ij eq. (qij) */
    flow_term(gjj, 0, gji, -bji, vi, vj, c, s, &u[2]);    /* p_ji eq. (pji) */
    flow_term(-bjj, 0, -bji, -gji, vi, vj, c, s, &u[3]);  /* q_ji eq. (qji) */
    /* w_i(ij) = v_i^2, theta_i(ij), w_j(ij) = v_j^2, theta_j(ij) */
    for (int k = 4; k < 8; ++k) memset(&u[k], 0, sizeof(fterm));
    u[4].val = vi * vi; u[4].d[0] = 2.0 * vi; u[4].h[0][0] = 2.0;
    u[5].val = x[2];    u[5].d[2] = 1.0;
    u[6].val = vj * vj; u[6].d[1] = 2.0 * vj; u[6].h[1][1] = 2.0;
    u[7].val = x[3];    u[7].d[3] = 1.0;
}

void ora_branch_flows(const double *Y8, const double *x, double *flows4)
{
    fterm u[8];
    branch_couplings(Y8, x, u);
    for (int k = 0; k < 4; ++k) flows4[k] = u[k].val;
}

/*
 * eq. branch: F(x) = sum_c [ y_c r_c + rho_c/2 r_c^2 ],  r_c = u_c(x) - xbar_c + z_c
 *                  + sum_e [ lt_e h_e + rt/2 h_e^2 ],  h_e = p_e^2 + q_e^2 + s_e
 * and its exact gradient and Hessian by the chain rule.
 */
void ora_branch_fgh(const ora_branch_prob *bp, const double *x, double *f, double *g, double *H)
{
    fterm u[8];
    branch_couplings(bp->Y, x, u);
    double F = 0.0;
    if (g) memset(g, 0, NV * sizeof(double));
    if (H) memset(H, 0, NV * NV * sizeof(double));
    for (int c = 0; c < 8; ++c) {
        double rc = u[c].val - bp->xbar[c] + bp->z[c];
        F += bp->y[c] * rc + 0.5 * bp->rho[c] * rc * rc;
        double wgt = bp->y[c] + bp->rho[c] * rc;
        for (int a = 0; a < NV; ++a) {
            if (g) g[a] += wgt * u[c].d[a];
            if (H)
                for (int b = 0; b < NV; ++b)
                    H[a * NV + b] += bp->rho[c] * u[c].d[a] * u[c].d[b] + wgt * u[c].h[a][b];
        }
    }
    for (int e = 0; e < 2; ++e) {
        const fterm *P = &u[2 * e], *Q = &u[2 * e + 1];
        int si = 4 + e;
        double h = P->val * P->val + Q->val * Q->val + x[si];
        F += bp->lt[e] * h + 0.5 * bp->rt * h * h;
        double dh[NV], d2h[NV][NV];
        for (int a = 0; a < NV; ++a) {
            dh[a] = 2.0 * P->val * P->d[a] + 2.0 * Q->val * Q->d[a];
            for (int b = 0; b < NV; ++b)
                d2h[a][b] = 2.0 * (P->d[a] * P->d[b] + P->val * P->h[a][b]
                                   + Q->d[a] * Q->d[b] + Q->val * Q->h[a][b]);
        }
        dh[si] += 1.0;
        double wgt = bp->lt[e] + bp->rt * h;
        for (int a = 0; a < NV; ++a) {
            if (g) g[a] += wgt * dh[a];
            if (H)
                for (int b = 0; b < NV; ++b)
                    H[a * NV + b] += bp->rt * dh[a] * dh[b] + wgt * d2h[a][b];
        }
    }
    if (f) *f = F;
}

/* ------------------------------------------------------------------ */
/* TRON: trust-region Newton method for bound constraints (Lin & More  */
/* 1999) with the Steihaug (1983) treatment of negative curvature,     */
/* Section III-B.  Fixed constants of this implementation:              */
/* ------------------------------------------------------------------ */
#define T_MU0 0.01          /* sufficient decrease (Cauchy, projected search) */
#define T_ETA0 1e-3         /* step acceptance */
#define T_ETA1 0.25         /* radius shrink below */
#define T_ETA2 0.75         /* radius expansion above */
#define T_SIGMA1 0.25
#define T_SIGMA3 4.0
#define T_CAUCHY_TRIALS 20
#define T_PS_TRIALS 20
#define T_CG_RTOL 0.1
#define T_CG_MAXIT 12
#define T_CHOL_TRIES 20

static double dot(const double *a, const double *b)
{
    double s = 0.0;
    for (int i = 0; i < NV; ++i) s += a[i] * b[i];
    return s;
}
static double nrm2(const double *a) { return sqrt(dot(a, a)); }
static double proj1(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* model q(s) = g's + s'Hs/2 */
static double qmodel(const double *g, const double *H, const double *s)
{
    double Hs[NV];
    for (int i = 0; i < NV; ++i) {
        Hs[i] = 0.0;
        for (int j = 0; j < NV; ++j) Hs[i] += H[i * NV + j] * s[j];
    }
    return dot(g, s) + 0.5 * dot(s, Hs);
}

/* s(alpha) = P(x - alpha g) - x */
static void pstep(const double *x, const double *g, double alpha, const double *lo,
                  const double *hi, double *s)
{
    for (int i = 0; i < NV; ++i) s[i] = proj1(x[i] - alpha * g[i], lo[i], hi[i]) - x[i];
}

/* norm-inf of P(x - g) - x: the stationarity measure */
static double pgnorm(const double *x, const double *g, const double *lo, const double *hi)
{
    double m = 0.0;
    for (int i = 0; i < NV; ++i) {
        double d = fabs(proj1(x[i] - g[i], lo[i], hi[i]) - x[i]);
        if (d > m) m = d;
    }
    return m;
}

/* Generalised Cauchy step: search alpha along the projected gradient path
 * for q(s) <= mu0 g's and ||s|| <= delta; backtrack by 0.1 when the start
 * fails, otherwise extrapolate by 10 while the conditions still hold and the
 * path still moves (alpha below the largest breakpoint). */
static void cauchy(const double *x, const double *g, const double *H, const double *lo,
                   const double *hi, double delta, double *alpha, double *s, ora_stats *st)
{
    double brmax = 0.0;
    for (int i = 0; i < NV; ++i) {
        double bp = 0.0;
        if (g[i] > 0.0 && x[i] > lo[i]) bp = (x[i] - lo[i]) / g[i];
        else if (g[i] < 0.0 && x[i] < hi[i]) bp = (x[i] - hi[i]) / g[i];
        if (bp > brmax) brmax = bp;
    }
    double a = *alpha;
    pstep(x, g, a, lo, hi, s);
    st->cauchy_trials++;
    int ok = nrm2(s) <= delta && qmodel(g, H, s) <= T_MU0 * dot(g, s);
    if (!ok) {
        for (int t = 0; t < T_CAUCHY_TRIALS; ++t) {
            a *= 0.1;
            pstep(x, g, a, lo, hi, s);
            st->cauchy_trials++;
            if (nrm2(s) <= delta && qmodel(g, H, s) <= T_MU0 * dot(g, s)) break;
        }
    } else {
        double sn[NV];
        for (int t = 0; t < T_CAUCHY_TRIALS; ++t) {
            if (a >= brmax) break;
            double an = a * 10.0;
            pstep(x, g, an, lo, hi, sn);
            st->cauchy_trials++;
            if (nrm2(sn) <= delta && qmodel(g, H, sn) <= T_MU0 * dot(g, sn)) {
                a = an;
                memcpy(s, sn, sizeof(sn));
            } else {
                break;
            }
        }
    }
    *alpha = a;
}

/* tau >= 0 with ||a + tau p|| = delta (a inside the ball) */
static double boundary_tau(const double *a, const double *p, double delta)
{
    double pp = dot(p, p), ap = dot(a, p), aa = dot(a, a);
    double rad = delta * delta - aa;
    if (rad < 0.0) rad = 0.0;
    double disc = sqrt(ap * ap + pp * rad);
    if (pp == 0.0) return 0.0;
    return ap > 0.0 ? rad / (ap + disc) : (disc - ap) / pp;
}

/* Preconditioner of the free block A (n x n, row-major, stride NV): Cholesky
 * factor of D^-1 A D^-1 + sigma I with D = diag(sqrt|A_ii|) (1 where A_ii = 0),
 * sigma = 0 if all A_ii > 0 else 1e-3, doubled until the factorisation
 * succeeds -- Lin-More's incomplete Cholesky is complete for a dense 6x6. */
static void precond_factor(const double *A, int n, double *L, double *dsc)
{
    int pos = 1;
    for (int i = 0; i < n; ++i) {
        double a = A[i * NV + i];
        dsc[i] = a != 0.0 ? sqrt(fabs(a)) : 1.0;
        if (!(a > 0.0)) pos = 0;
    }
    double sigma = pos ? 0.0 : 1e-3;
    for (int tries = 0; tries < T_CHOL_TRIES; ++tries) {
        int ok = 1;
        for (int j = 0; j < n && ok; ++j) {
            double d = A[j * NV + j] / (dsc[j] * dsc[j]) + sigma;
            for (int k = 0; k < j; ++k) d -= L[j * NV + k] * L[j * NV + k];
            if (!(d > 0.0)) { ok = 0; break; }
            L[j * NV + j] = sqrt(d);
            for (int i = j + 1; i < n; ++i) {
                double v = A[i * NV + j] / (dsc[i] * dsc[j]);
                for (int k = 0; k < j; ++k) v -= L[i * NV + k] * L[j * NV + k];
                L[i * NV + j] = v / L[j * NV + j];
            }
        }
        if (ok) return;
        sigma = sigma * 2.0 > 1e-3 ? sigma * 2.0 : 1e-3;
    }
    /* give up: identity in the scaled space */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) L[i * NV + j] = (i == j) ? 1.0 : 0.0;
}

/* z = M^-1 r with M = D L L' D */
static void precond_solve(const double *L, const double *dsc, int n, const double *r, double *z)
{
    double t[NV];
    for (int i = 0; i < n; ++i) {
        double v = r[i] / dsc[i];
        for (int k = 0; k < i; ++k) v -= L[i * NV + k] * t[k];
        t[i] = v / L[i * NV + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double v = t[i];
        for (int k = i + 1; k < n; ++k) v -= L[k * NV + i] * t[k];
        t[i] = v / L[i * NV + i];
    }
    for (int i = 0; i < n; ++i) z[i] = t[i] / dsc[i];
}

/* Subspace step (one pass): Steihaug PCG on the free variables of the Cauchy
 * point for min q(sc + w), ||sc + w|| <= delta, then a projected backtracking
 * search along w. Returns the full step in s. */
static void subspace(const double *x, const double *g, const double *H, const double *lo,
                     const double *hi, double delta, const double *sc, double *s, ora_stats *st)
{
    int fr[NV], n = 0;
    double xc[NV];
    for (int i = 0; i < NV; ++i) {
        xc[i] = x[i] + sc[i];
        if (xc[i] > lo[i] && xc[i] < hi[i]) fr[n++] = i;
    }
    memcpy(s, sc, NV * sizeof(double));
    if (n == 0) return;
    /* gradient of q at sc */
    double gc[NV];
    for (int i = 0; i < NV; ++i) {
        gc[i] = g[i];
        for (int j = 0; j < NV; ++j) gc[i] += H[i * NV + j] * sc[j];
    }
    double A[NV * NV], L[NV * NV], dsc[NV];
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) A[a * NV + b] = H[fr[a] * NV + fr[b]];
    precond_factor(A, n, L, dsc);

    double w[NV] = {0}, r[NV], zz[NV], p[NV], q[NV];
    for (int a = 0; a < n; ++a) r[a] = -gc[fr[a]];
    double rn0 = 0.0;
    for (int a = 0; a < n; ++a) rn0 += r[a] * r[a];
    rn0 = sqrt(rn0);
    if (rn0 == 0.0) return;
    precond_solve(L, dsc, n, r, zz);
    for (int a = 0; a < n; ++a) p[a] = zz[a];
    double rz = 0.0;
    for (int a = 0; a < n; ++a) rz += r[a] * zz[a];
    double tol = T_CG_RTOL * rn0;
    for (int it = 0; it < T_CG_MAXIT; ++it) {
        st->cg_iters++;
        double kappa = 0.0;
        for (int a = 0; a < n; ++a) {
            q[a] = 0.0;
            for (int b = 0; b < n; ++b) q[a] += A[a * NV + b] * p[b];
            kappa += p[a] * q[a];
        }
        /* full-space vectors for the trust-region test */
        double cur[NV], pf[NV];
        for (int i = 0; i < NV; ++i) { cur[i] = sc[i]; pf[i] = 0.0; }
        for (int a = 0; a < n; ++a) { cur[fr[a]] += w[a]; pf[fr[a]] = p[a]; }
        if (kappa <= 0.0) {                       /* negative curvature */
            double tau = boundary_tau(cur, pf, delta);
            for (int a = 0; a < n; ++a) w[a] += tau * p[a];
            break;
        }
        double alpha = rz / kappa;
        double nxt[NV];
        for (int i = 0; i < NV; ++i) nxt[i] = cur[i] + alpha * pf[i];
        if (nrm2(nxt) >= delta) {                 /* trust-region boundary */
            double tau = boundary_tau(cur, pf, delta);
            for (int a = 0; a < n; ++a) w[a] += tau * p[a];
            break;
        }
        for (int a = 0; a < n; ++a) { w[a] += alpha * p[a]; r[a] -= alpha * q[a]; }
        double rn = 0.0;
        for (int a = 0; a < n; ++a) rn += r[a] * r[a];
        if (sqrt(rn) <= tol) break;
        precond_solve(L, dsc, n, r, zz);
        double rz1 = 0.0;
        for (int a = 0; a < n; ++a) rz1 += r[a] * zz[a];
        double beta = rz1 / rz;
        rz = rz1;
        for (int a = 0; a < n; ++a) p[a] = zz[a] + beta * p[a];
    }
    /* projected search along w from the Cauchy point */
    double wf[NV] = {0};
    for (int a = 0; a < n; ++a) wf[fr[a]] = w[a];
    double qc = qmodel(g, H, sc);
    double beta = 1.0;
    for (int t = 0; t < T_PS_TRIALS; ++t) {
        st->ps_trials++;
        double sb[NV], d[NV];
        for (int i = 0; i < NV; ++i) {
            sb[i] = proj1(xc[i] + beta * wf[i], lo[i], hi[i]) - x[i];
            d[i] = sb[i] - sc[i];
        }
        if (qmodel(g, H, sb) <= qc + T_MU0 * dot(gc, d)) {
            memcpy(s, sb, sizeof(sb));
            return;
        }
        beta *= 0.5;
    }
}

/* One TRON solve of the bound-constrained branch problem from x.
 * Stops (status 0) on ||P(x - g) - x||_inf <= gtol * max(1, that norm at the
 * start) or on a step with ||s||_inf <= xtol * max(1, ||x||_inf); status 1
 * after tron_max_iter iterations; status 2 when the radius falls below
 * 1e-14 max(1, ||x||_inf) or the model predicts no decrease.
 * The initial radius is ||P(x0 - g0) - x0||_2.  The Cauchy search starts from
 * the alpha the branch's previous TRON call ended with (bp->alpha; 1 for the
 * first call) and hands its last alpha back in bp->alpha.
 * A step whose predicted decrease is at most ftol * max(1, |f + K|) lies below
 * the rounding level of f; the model is trusted for it (ratio taken as 1).
 * K = sum_c y_c^2 / (2 rho_c) turns F into its completed-square form
 * sum_c rho_c/2 (u_c - t_c)^2 + AL terms, t_c = xbar_c - z_c - y_c/rho_c,
 * a sum of non-negative terms whose size sets the rounding level of f - ft;
 * the test is then the same whichever way the constant of eq. branch is
 * written. */
int ora_tron(ora_branch_prob *bp, double *x, const ora_options *o, ora_stats *st)
{
    const double *lo = bp->lo, *hi = bp->hi;
    double f, g[NV], H[NV * NV];
    for (int i = 0; i < NV; ++i) x[i] = proj1(x[i], lo[i], hi[i]);
    ora_branch_fgh(bp, x, &f, g, H);
    st->tron_calls++;
    st->fgh_evals++;
    double pg0 = pgnorm(x, g, lo, hi);
    double gtol = o->tron_gtol * (pg0 > 1.0 ? pg0 : 1.0);
    double sp[NV];
    pstep(x, g, 1.0, lo, hi, sp);
    double delta = nrm2(sp);
    double alpha = bp->alpha > 0.0 ? bp->alpha : 1.0;
    double K = 0.0;
    for (int c = 0; c < 8; ++c) K += bp->y[c] * bp->y[c] / (2.0 * bp->rho[c]);
    int status = 1;
    for (int k = 0; k < o->tron_max_iter; ++k) {
        if (pgnorm(x, g, lo, hi) <= gtol) { status = 0; break; }
        st->tron_iters++;
        double sc[NV], s[NV];
        cauchy(x, g, H, lo, hi, delta, &alpha, sc, st);
        subspace(x, g, H, lo, hi, delta, sc, s, st);
        double xn = 0.0, sn = 0.0;
        for (int i = 0; i < NV; ++i) {
            if (fabs(x[i]) > xn) xn = fabs(x[i]);
            if (fabs(s[i]) > sn) sn = fabs(s[i]);
        }
        if (sn <= o->tron_xtol * (xn > 1.0 ? xn : 1.0)) { status = 0; break; }
        double xt[NV];
        for (int i = 0; i < NV; ++i) xt[i] = proj1(x[i] + s[i], lo[i], hi[i]);
        double ft;
        ora_branch_fgh(bp, xt, &ft, NULL, NULL);
        st->f_evals++;
        double prered = -qmodel(g, H, s);
        double actred = f - ft;
        double snorm = nrm2(s);
        if (k == 0 && snorm < delta) delta = snorm;
        double fa = fabs(f + K) > 1.0 ? fabs(f + K) : 1.0;
        double ratio;
        if (prered <= 0.0) ratio = -1.0;
        else if (prered <= o->tron_ftol * fa) ratio = 1.0;
        else ratio = actred / prered;
        if (ratio < T_ETA1) delta = T_SIGMA1 * (snorm < delta ? snorm : delta);
        else if (ratio > T_ETA2) delta = (T_SIGMA3 * snorm > delta) ? T_SIGMA3 * snorm : delta;
        if (ratio > T_ETA0) {
            memcpy(x, xt, sizeof(xt));
            f = ft;
            ora_branch_fgh(bp, x, NULL, g, H);
            st->fgh_evals++;
        }
        if (prered <= 0.0) { status = 2; break; }
        xn = 0.0;
        for (int i = 0; i < NV; ++i) if (fabs(x[i]) > xn) xn = fabs(x[i]);
        if (delta <= 1e-14 * (xn > 1.0 ? xn : 1.0)) { status = 2; break; }
    }
    if (status == 1) st->tron_maxiter_hits++;
    bp->alpha = alpha;
    return status;
}

/* Augmented Lagrangian loop on p^2 + q^2 + s = 0 of both branch ends
 * (Section II-C; the schedule is this implementation's reading): rho-tilde
 * starts at the value the caller sets (bp->rt), each pass solves eq. branch by TRON, then
 * lt += rt h; stop when max|h| <= al_tol, else rt *= al_rho_factor (capped)
 * when max|h| did not fall below al_decay times its previous value.  The
 * Cauchy alpha of each TRON call carries into the next one (bp->alpha). */
void ora_branch_solve(ora_branch_prob *bp, double *x, const ora_options *o, ora_stats *st)
{
    double hprev = INFINITY;
    for (int a = 0; a < o->al_max_iter; ++a) {
        st->al_passes++;
        ora_tron(bp, x, o, st);
        double fl[4];
        ora_branch_flows(bp->Y, x, fl);
        double h0 = fl[0] * fl[0] + fl[1] * fl[1] + x[4];
        double h1 = fl[2] * fl[2] + fl[3] * fl[3] + x[5];
        bp->lt[0] += bp->rt * h0;
        bp->lt[1] += bp->rt * h1;
        double hm = fabs(h0) > fabs(h1) ? fabs(h0) : fabs(h1);
        if (hm <= o->al_tol) break;
        if (hm > o->al_decay * hprev) {
            double rn = bp->rt * o->al_rho_factor;
            bp->rt = rn < o->al_rho_max ? rn : o->al_rho_max;
        }
        hprev = hm;
    }
}

/* eq. qp-bound for one generator variable: minimise cost2 x^2 + cost1 x
 * + y (x - xbar + z) + rho/2 (x - xbar + z)^2 over [lo, hi], i.e.
 * Q = 2 cost2 + rho, c = rho (xbar - z) - y - cost1, x* = max(lo, min(hi, c/Q)). */
double ora_gen_solve(double cost2, double cost1, double rho, double xbar, double z, double y,
                     double lo, double hi)
{
    double Q = 2.0 * cost2 + rho;
    double c = rho * (xbar - z) - y - cost1;
    double v = c / Q;
    return v < lo ? lo : (v > hi ? hi : v);
}

/* ------------------------------------------------------------------ */
/* Whole problem                                                       */
/* ------------------------------------------------------------------ */
#define HIST_CAP 200000

struct ora {
    int nb, nl, ng, ref, m;
    double base;
    double *pd, *qd, *gs, *bs, *vmin, *vmax;
    int *fb, *tb;
    double *rate, *Y;
    int *gb;
    double *pmin, *pmax, *qmin, *qmax, *c2, *c1, *c0;   /* c2, c1 per unit */
    double *pbase_lo, *pbase_hi;                          /* bounds set by the caller */
    ora_options o;
    int *row, *col;
    /* state */
    double *u, *xbar, *z, *y, *lam, *rho, *bx, *lt, *bus;
    double *balpha;             /* per branch: Cauchy alpha of its last TRON call */
    double beta, tol_in, zprev;
    int outer, inner;
    /* results */
    int iters, total_iters, status;
    double pri, pri_z, dual, zn;
    double nu, nx, ny;          /* ||u||, ||xbar||, ||y|| of the last iteration */
    ora_stats st;
    double *hist;
    int nhist;
};

static double *dup_d(const double *a, int n)
{
    double *p = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    if (a && n > 0) memcpy(p, a, sizeof(double) * n);
    return p;
}
static int *dup_i(const int32_t *a, int n)
{
    int *p = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) p[i] = a[i];
    return p;
}

/* coupling index helpers */
static int cg_p(const ora *p, int g) { (void)p; return 2 * g; }
static int cb(const ora *p, int l, int k) { return 2 * p->ng + 8 * l + k; }

ora *ora_create(const ora_grid *g, const ora_options *o)
{
    ora *p = (ora *)calloc(1, sizeof(ora));
    p->nb = g->nbus; p->nl = g->nbranch; p->ng = g->ngen; p->ref = g->ref_bus;
    p->base = g->base_mva;
    p->m = 2 * p->ng + 8 * p->nl;
    p->o = *o;
    p->pd = dup_d(g->pd, p->nb); p->qd = dup_d(g->qd, p->nb);
    p->gs = dup_d(g->gs, p->nb); p->bs = dup_d(g->bs, p->nb);
    p->vmin = dup_d(g->vmin, p->nb); p->vmax = dup_d(g->vmax, p->nb);
    p->fb = dup_i(g->f_bus, p->nl); p->tb = dup_i(g->t_bus, p->nl);
    p->rate = dup_d(g->rate_a, p->nl);
    p->Y = dup_d(NULL, 8 * p->nl);
    for (int l = 0; l < p->nl; ++l)
        ora_admittance(g->r[l], g->x[l], g->b[l], g->tap[l], g->shift[l], &p->Y[8 * l]);
    p->gb = dup_i(g->gen_bus, p->ng);
    p->pmin = dup_d(g->pmin, p->ng); p->pmax = dup_d(g->pmax, p->ng);
    p->pbase_lo = dup_d(g->pmin, p->ng); p->pbase_hi = dup_d(g->pmax, p->ng);
    p->qmin = dup_d(g->qmin, p->ng); p->qmax = dup_d(g->qmax, p->ng);
    p->c2 = dup_d(NULL, p->ng); p->c1 = dup_d(NULL, p->ng); p->c0 = dup_d(g->c0, p->ng);
    /* costs to per-unit power: c2' = c2 base^2, c1' = c1 base (MATPOWER units) */
    for (int k = 0; k < p->ng; ++k) {
        p->c2[k] = g->c2[k] * p->base * p->base;
        p->c1[k] = g->c1[k] * p->base;
    }
    /* incidence rows: counting sort of entries (branch ends, then gens) by bus;
     * entries are visited in increasing entry id, so each row is ordered. */
    int ne = 2 * p->nl + p->ng;
    p->row = (int *)calloc(p->nb + 1, sizeof(int));
    p->col = (int *)malloc(sizeof(int) * (ne > 0 ? ne : 1));
    for (int e = 0; e < ne; ++e) {
        int bus = e < 2 * p->nl ? ((e & 1) ? p->tb[e >> 1] : p->fb[e >> 1]) : p->gb[e - 2 * p->nl];
        p->row[bus + 1]++;
    }
    for (int i = 0; i < p->nb; ++i) p->row[i + 1] += p->row[i];
    int *fill = (int *)malloc(sizeof(int) * (p->nb > 0 ? p->nb : 1));
    for (int i = 0; i < p->nb; ++i) fill[i] = p->row[i];
    for (int e = 0; e < ne; ++e) {
        int bus = e < 2 * p->nl ? ((e & 1) ? p->tb[e >> 1] : p->fb[e >> 1]) : p->gb[e - 2 * p->nl];
        p->col[fill[bus]++] = e;
    }
    free(fill);
    int m = p->m;
    p->u = dup_d(NULL, m); p->xbar = dup_d(NULL, m); p->z = dup_d(NULL, m);
    p->y = dup_d(NULL, m); p->lam = dup_d(NULL, m); p->rho = dup_d(NULL, m);
    p->bx = dup_d(NULL, 6 * p->nl); p->lt = dup_d(NULL, 2 * p->nl);
    p->balpha = dup_d(NULL, p->nl);
    p->bus = dup_d(NULL, 2 * p->nb);
    p->hist = dup_d(NULL, 4 * HIST_CAP);
    /* penalties: rho_pq for generator and flow couplings, rho_va for w, theta */
    for (int k = 0; k < p->ng; ++k) { p->rho[2 * k] = o->rho_pq; p->rho[2 * k + 1] = o->rho_pq; }
    for (int l = 0; l < p->nl; ++l)
        for (int k = 0; k < 8; ++k) p->rho[cb(p, l, k)] = k < 4 ? o->rho_pq : o->rho_va;
    ora_cold_start(p);
    return p;
}

void ora_destroy(ora *p)
{
    if (!p) return;
    free(p->pbase_lo); free(p->pbase_hi);
    double *d[] = {p->pd, p->qd, p->gs, p->bs, p->vmin, p->vmax, p->rate, p->Y, p->pmin,
                   p->pmax, p->qmin, p->qmax, p->c2, p->c1, p->c0, p->u, p->xbar, p->z,
                   p->y, p->lam, p->rho, p->bx, p->lt, p->bus, p->hist, p->balpha};
    for (unsigned i = 0; i < sizeof(d) / sizeof(d[0]); ++i) free(d[i]);
    free(p->fb); free(p->tb); free(p->gb); free(p->row); free(p->col);
    free(p);
}

static double s_lower(const ora *p, int l)
{
    /* eq. branch bound on the slack, read as -rbar^2 with rbar the rating
     * tightened to line_limit_frac (Section IV-A); no rating = no limit */
    double r = p->rate[l];
    if (!(r > 0.0)) return -1e20;
    double rb = p->o.line_limit_frac * r;
    return -rb * rb;
}

static void branch_bounds(const ora *p, int l, double *lo, double *hi)
{
    int i = p->fb[l], j = p->tb[l];
    lo[0] = p->vmin[i]; hi[0] = p->vmax[i];
    lo[1] = p->vmin[j]; hi[1] = p->vmax[j];
    lo[2] = -TWO_PI; hi[2] = TWO_PI;
    lo[3] = -TWO_PI; hi[3] = TWO_PI;
    lo[4] = s_lower(p, l); hi[4] = 0.0;
    lo[5] = lo[4]; hi[5] = 0.0;
}

/* Section IV-B initialisation: generation and voltage magnitudes at the
 * middle of their bounds, angles zero, flows from those voltages, all
 * multipliers zero; bus copies equal to the component values. */
void ora_cold_start(ora *p)
{
    for (int k = 0; k < p->ng; ++k) {
        p->u[2 * k] = 0.5 * (p->pmin[k] + p->pmax[k]);
        p->u[2 * k + 1] = 0.5 * (p->qmin[k] + p->qmax[k]);
    }
    for (int i = 0; i < p->nb; ++i) {
        double v = 0.5 * (p->vmin[i] + p->vmax[i]);
        p->bus[2 * i] = v * v;
        p->bus[2 * i + 1] = 0.0;
    }
    for (int l = 0; l < p->nl; ++l) {
        double *x = &p->bx[6 * l];
        int i = p->fb[l], j = p->tb[l];
        x[0] = 0.5 * (p->vmin[i] + p->vmax[i]);
        x[1] = 0.5 * (p->vmin[j] + p->vmax[j]);
        x[2] = 0.0; x[3] = 0.0;
        double fl[4];
        ora_branch_flows(&p->Y[8 * l], x, fl);
        double slo = s_lower(p, l);
        x[4] = proj1(-(fl[0] * fl[0] + fl[1] * fl[1]), slo, 0.0);
        x[5] = proj1(-(fl[2] * fl[2] + fl[3] * fl[3]), slo, 0.0);
        p->lt[2 * l] = 0.0; p->lt[2 * l + 1] = 0.0;
        p->balpha[l] = 1.0;
        for (int k = 0; k < 4; ++k) p->u[cb(p, l, k)] = fl[k];
        p->u[cb(p, l, 4)] = x[0] * x[0];
        p->u[cb(p, l, 5)] = 0.0;
        p->u[cb(p, l, 6)] = x[1] * x[1];
        p->u[cb(p, l, 7)] = 0.0;
    }
    memcpy(p->xbar, p->u, sizeof(double) * p->m);
    memset(p->z, 0, sizeof(double) * p->m);
    memset(p->y, 0, sizeof(double) * p->m);
    memset(p->lam, 0, sizeof(double) * p->m);
    /* beta0 <= 0 selects the default reading beta0 = 10 rho_va */
    p->beta = p->o.beta0 > 0.0 ? p->o.beta0 : 10.0 * p->o.rho_va;
    p->outer = 0; p->inner = 0; p->zprev = INFINITY;
    p->total_iters = 0;
    p->pri = p->pri_z = p->dual = p->zn = 0.0;
}

int ora_set_loads(ora *p, const double *pd, const double *qd)
{
    memcpy(p->pd, pd, sizeof(double) * p->nb);
    memcpy(p->qd, qd, sizeof(double) * p->nb);
    return 0;
}

int ora_set_gen_bounds(ora *p, const double *pmin, const double *pmax)
{
    memcpy(p->pmin, pmin, sizeof(double) * p->ng);
    memcpy(p->pmax, pmax, sizeof(double) * p->ng);
    memcpy(p->pbase_lo, pmin, sizeof(double) * p->ng);
    memcpy(p->pbase_hi, pmax, sizeof(double) * p->ng);
    return 0;
}

/* Section IV-C ramp limit |p_{t+1} - p_t| <= frac * pmax around the current
 * dispatch, on the bounds last set by the caller (lower kept <= upper). */
void ora_set_ramp_limit(ora *p, double frac)
{
    for (int k = 0; k < p->ng; ++k) {
        double pg = p->u[2 * k], r = frac * p->pbase_hi[k];
        double hi = pg + r < p->pbase_hi[k] ? pg + r : p->pbase_hi[k];
        double lo = pg - r > p->pbase_lo[k] ? pg - r : p->pbase_lo[k];
        p->pmin[k] = lo < hi ? lo : hi;
        p->pmax[k] = hi;
    }
}

/* Algorithm 1, x-update of the generators: eq. qp-bound with the scaled cost */
static void update_generators(ora *p)
{
    double so = p->o.obj_scale;
    for (int k = 0; k < p->ng; ++k) {
        int cp = cg_p(p, k), cq = cp + 1;
        p->u[cp] = ora_gen_solve(so * p->c2[k], so * p->c1[k], p->rho[cp], p->xbar[cp], p->z[cp],
                                 p->y[cp], p->pmin[k], p->pmax[k]);
        p->u[cq] = ora_gen_solve(0.0, 0.0, p->rho[cq], p->xbar[cq], p->z[cq], p->y[cq],
                                 p->qmin[k], p->qmax[k]);
    }
}

/* rho-tilde at the start of a branch solve (reading of this implementation;
 * Section II-C gives no schedule): al_rho0 when set, else
 * 25 rho_pq / rbar^2 with rbar the tightened rating: 100 times the penalty
 * rho_pq / (2 rbar)^2 under which rt/2 h^2 on h = p^2 + q^2 + s weighs a
 * deviation dS of the apparent flow at the limit (dh = 2 rbar dS) like the
 * coupling penalty rho_pq/2 dS^2 -- one growth step ahead, since the first
 * passes at that weight seldom cut the violation enough to avoid the growth
 * (capped at al_rho_max); rho_pq for a line without a limit. */
static double al_rho_start(const ora *p, int l)
{
    if (p->o.al_rho0 > 0.0) return p->o.al_rho0;
    double rb2 = -s_lower(p, l);
    if (!(rb2 < 1e19)) return p->o.rho_pq;
    double r = 25.0 * p->o.rho_pq / rb2;
    return r < p->o.al_rho_max ? r : p->o.al_rho_max;
}

/* Algorithm 1, x-update of the branches: eq. branch by the AL loop around TRON,
 * warm-started from the branch's previous solution clipped to its bounds */
static void update_branches(ora *p, int l0, int l1)
{
    for (int l = l0; l < l1; ++l) {
        ora_branch_prob bp;
        memcpy(bp.Y, &p->Y[8 * l], sizeof(bp.Y));
        branch_bounds(p, l, bp.lo, bp.hi);
        for (int k = 0; k < 8; ++k) {
            int c = cb(p, l, k);
            bp.xbar[k] = p->xbar[c]; bp.z[k] = p->z[c]; bp.y[k] = p->y[c]; bp.rho[k] = p->rho[c];
        }
        bp.lt[0] = p->lt[2 * l]; bp.lt[1] = p->lt[2 * l + 1];
        bp.rt = al_rho_start(p, l);
        bp.alpha = p->balpha[l];
        double *x = &p->bx[6 * l];
        ora_branch_solve(&bp, x, &p->o, &p->st);
        p->lt[2 * l] = bp.lt[0]; p->lt[2 * l + 1] = bp.lt[1];
        p->balpha[l] = bp.alpha;
        double fl[4];
        ora_branch_flows(bp.Y, x, fl);
        for (int k = 0; k < 4; ++k) p->u[cb(p, l, k)] = fl[k];
        p->u[cb(p, l, 4)] = x[0] * x[0];
        p->u[cb(p, l, 5)] = x[2];
        p->u[cb(p, l, 6)] = x[1] * x[1];
        p->u[cb(p, l, 7)] = x[3];
    }
}

/* Algorithm 1, xbar-update: eq. qp-bus per bus.  The bus variables are the pooled
 * w_i and theta_i and one copy per incident generator (p, q) and branch end
 * (p, q of the flow leaving bus i).  Coupling c contributes
 * rho_c/2 (xbar - t_c)^2 with target t_c = u_c + z_c + y_c/rho_c, so
 * Q = diag(rho) (pooled: sum of rho), c = Q t, and A x = b holds
 *   P row: sum p_g(i) - sum p_l(i) - gs w = pd   (eq. pg)
 *   Q row: sum q_g(i) - sum q_l(i) + bs w = qd   (eq. qg)
 * mu = (A Q^-1 A')^-1 (A Q^-1 c - b),  x = Q^-1 (c - A' mu).
 * theta_i is not in A: theta_i = its pooled target (0 at the reference bus,
 * Section IV-B). */
static void update_buses(ora *p)
{
    int maxv = 0;
    for (int i = 0; i < p->nb; ++i) {
        int d = p->row[i + 1] - p->row[i];
        if (d > maxv) maxv = d;
    }
    int cap = 2 * maxv + 1;
    double *Qd = (double *)malloc(sizeof(double) * cap);
    double *cv = (double *)malloc(sizeof(double) * cap);
    double *A0 = (double *)malloc(sizeof(double) * cap);
    double *A1 = (double *)malloc(sizeof(double) * cap);
    int *cpl = (int *)malloc(sizeof(int) * cap);
    for (int i = 0; i < p->nb; ++i) {
        /* pooled w and theta */
        double qw = 0.0, cw = 0.0, qt = 0.0, ct = 0.0;
        int nv = 1;     /* variable 0 is w */
        for (int k = p->row[i]; k < p->row[i + 1]; ++k) {
            int e = p->col[k];
            if (e < 2 * p->nl) {
                int l = e >> 1, end = e & 1;
                int cP = cb(p, l, end ? 2 : 0), cQ = cb(p, l, end ? 3 : 1);
                int cW = cb(p, l, end ? 6 : 4), cT = cb(p, l, end ? 7 : 5);
                double tW = p->u[cW] + p->z[cW] + p->y[cW] / p->rho[cW];
                double tT = p->u[cT] + p->z[cT] + p->y[cT] / p->rho[cT];
                qw += p->rho[cW]; cw += p->rho[cW] * tW;
                qt += p->rho[cT]; ct += p->rho[cT] * tT;
                /* flow copies: -1 in their balance row */
                Qd[nv] = p->rho[cP]; cv[nv] = p->rho[cP] * (p->u[cP] + p->z[cP] + p->y[cP] / p->rho[cP]);
                A0[nv] = -1.0; A1[nv] = 0.0; cpl[nv] = cP; nv++;
                Qd[nv] = p->rho[cQ]; cv[nv] = p->rho[cQ] * (p->u[cQ] + p->z[cQ] + p->y[cQ] / p->rho[cQ]);
                A0[nv] = 0.0; A1[nv] = -1.0; cpl[nv] = cQ; nv++;
            } else {
                int g = e - 2 * p->nl;
                int cP = 2 * g, cQ = 2 * g + 1;
                Qd[nv] = p->rho[cP]; cv[nv] = p->rho[cP] * (p->u[cP] + p->z[cP] + p->y[cP] / p->rho[cP]);
                A0[nv] = 1.0; A1[nv] = 0.0; cpl[nv] = cP; nv++;
                Qd[nv] = p->rho[cQ]; cv[nv] = p->rho[cQ] * (p->u[cQ] + p->z[cQ] + p->y[cQ] / p->rho[cQ]);
                A0[nv] = 0.0; A1[nv] = 1.0; cpl[nv] = cQ; nv++;
            }
        }
        Qd[0] = qw; cv[0] = cw; A0[0] = -p->gs[i]; A1[0] = p->bs[i]; cpl[0] = -1;
        /* M = A Q^-1 A',  rhs = A Q^-1 c - b */
        double M00 = 0.0, M01 = 0.0, M11 = 0.0, r0 = -p->pd[i], r1 = -p->qd[i];
        for (int v = 0; v < nv; ++v) {
            M00 += A0[v] * A0[v] / Qd[v];
            M01 += A0[v] * A1[v] / Qd[v];
            M11 += A1[v] * A1[v] / Qd[v];
            r0 += A0[v] * cv[v] / Qd[v];
            r1 += A1[v] * cv[v] / Qd[v];
        }
        double det = M00 * M11 - M01 * M01;
        double mu0 = (M11 * r0 - M01 * r1) / det;
        double mu1 = (M00 * r1 - M01 * r0) / det;
        double w = (cv[0] - A0[0] * mu0 - A1[0] * mu1) / Qd[0];
        double th = (i == p->ref) ? 0.0 : ct / qt;
        p->bus[2 * i] = w;
        p->bus[2 * i + 1] = th;
        for (int v = 1; v < nv; ++v) p->xbar[cpl[v]] = (cv[v] - A0[v] * mu0 - A1[v] * mu1) / Qd[v];
        for (int k = p->row[i]; k < p->row[i + 1]; ++k) {
            int e = p->col[k];
            if (e < 2 * p->nl) {
                int l = e >> 1, end = e & 1;
                p->xbar[cb(p, l, end ? 6 : 4)] = w;
                p->xbar[cb(p, l, end ? 7 : 5)] = th;
            }
        }
    }
    free(Qd); free(cv); free(A0); free(A1); free(cpl);
}

/* One inner iteration of Algorithm 1 (x-, xbar-, z- and y-updates) with its residuals:
 * primal = ||u - xbar||, primal_z = ||u - xbar + z||,
 * dual = ||rho (xbar - xbar_prev)||, zn = ||z||, all Euclidean. */
static void iterate(ora *p, int l0, int l1)
{
    int m = p->m;
    double *xprev = dup_d(p->xbar, m);
    update_generators(p);
    update_branches(p, l0, l1);
    update_buses(p);
    double sp = 0.0, spz = 0.0, sd = 0.0, sz = 0.0, su = 0.0, sx = 0.0, sy = 0.0;
    for (int c = 0; c < m; ++c) {
        double r0 = p->u[c] - p->xbar[c];
        /* Algorithm 1, z-update: eq. qp-bound with (l, u) = (-inf, inf):
         * minimise lam z + beta/2 z^2 + y (r0 + z) + rho/2 (r0 + z)^2 */
        if (p->o.two_level) {
            double Q = p->beta + p->rho[c];
            double cz = -(p->lam[c] + p->y[c] + p->rho[c] * r0);
            p->z[c] = cz / Q;
        } else {
            p->z[c] = 0.0;
        }
        /* Algorithm 1, y-update: y <- y + rho (A x + B xbar + z) */
        p->y[c] += p->rho[c] * (r0 + p->z[c]);
        double dx = p->rho[c] * (p->xbar[c] - xprev[c]);
        sp += r0 * r0;
        spz += (r0 + p->z[c]) * (r0 + p->z[c]);
        sd += dx * dx;
        sz += p->z[c] * p->z[c];
        su += p->u[c] * p->u[c];
        sx += p->xbar[c] * p->xbar[c];
        sy += p->y[c] * p->y[c];
    }
    free(xprev);
    p->pri = sqrt(sp); p->pri_z = sqrt(spz); p->dual = sqrt(sd); p->zn = sqrt(sz);
    p->nu = sqrt(su); p->nx = sqrt(sx); p->ny = sqrt(sy);
    if (p->nhist < HIST_CAP) {
        double *h = &p->hist[4 * p->nhist++];
        h[0] = p->pri; h[1] = p->dual; h[2] = p->zn; h[3] = p->pri_z;
    }
}

/* Stopping tolerances (reading of "the termination conditions of SunSun21",
 * Section IV-A, which loosen as the number of consensus constraints grows,
 * Section IV-B): the standard ADMM test of Boyd et al. (2011, Sec. 3.3.1) with
 * absolute and relative tolerance both equal to t,
 *   eps_pri(t)  = sqrt(m) t + t max(||u||, ||xbar||),
 *   eps_dual(t) = sqrt(m) t + t ||y||. */
static double eps_pri(const ora *p, double t)
{
    double a = p->nu > p->nx ? p->nu : p->nx;
    return sqrt((double)p->m) * t + t * a;
}
static double eps_dual(const ora *p, double t) { return sqrt((double)p->m) * t + t * p->ny; }

/* Algorithm 1, outer update (readings of this implementation):
 * lam <- Proj_[-lambda_max, lambda_max](lam + beta z); beta <- beta_factor beta
 * (capped) when ||z|| did not fall below z_decay times its value at the
 * previous outer update; the inner tolerance halves each outer update.
 * The adaptive variant (beta_rule 1, Section V's sensitivity to the penalties)
 * grows beta by (||z|| / (z_decay ||z_prev||))^2, kept within [1, beta_factor]:
 * no growth while ||z|| falls fast enough, the full factor when it stalls. */
static void outer_update(ora *p, double tol)
{
    for (int c = 0; c < p->m; ++c) {
        double v = p->lam[c] + p->beta * p->z[c];
        p->lam[c] = proj1(v, -p->o.lambda_max, p->o.lambda_max);
    }
    if (p->o.beta_rule == 1) {
        double r = p->zn / (p->o.z_decay * p->zprev);     /* 0 while zprev is infinite */
        double f = r * r;
        if (!(f > 1.0)) f = 1.0;
        if (f > p->o.beta_factor) f = p->o.beta_factor;
        double b = p->beta * f;
        p->beta = b < p->o.beta_max ? b : p->o.beta_max;
    } else if (p->zn > p->o.z_decay * p->zprev) {
        double b = p->beta * p->o.beta_factor;
        p->beta = b < p->o.beta_max ? b : p->o.beta_max;
    }
    p->zprev = p->zn;
    p->outer++;
    p->inner = 0;
    double ti = p->o.tol_in0 * pow(p->o.tol_in_decay, p->outer);
    p->tol_in = ti > tol ? ti : tol;
}

/* Algorithm 1: repeat { inner ADMM until converged; outer update } until
 * ||z|| <= eps_pri(tol).  Returns 0 when ||u - xbar|| <= eps_pri(tol),
 * ||rho dxbar|| <= eps_dual(tol) and ||z|| <= eps_pri(tol);
 * 1 when max_iter or max_outer is reached first, -3 on a non-finite residual.
 * warm_start = 0 reinitialises (Section IV-B); 1 keeps every primal, dual and
 * penalty value (Section IV-C) and restarts only the loop counters. */
int ora_solve(ora *p, double tol, int32_t max_iter, int32_t warm_start)
{
    if (!warm_start) ora_cold_start(p);
    p->outer = 0; p->inner = 0; p->zprev = INFINITY;
    p->tol_in = p->o.tol_in0 > tol ? p->o.tol_in0 : tol;
    p->iters = 0;
    p->nhist = 0;
    memset(&p->st, 0, sizeof(p->st));
    p->status = 1;
    while (p->iters < max_iter) {
        iterate(p, 0, p->nl);
        p->iters++;
        p->total_iters++;
        if (!isfinite(p->pri) || !isfinite(p->dual) || !isfinite(p->zn)) { p->status = -3; break; }
        double ep = eps_pri(p, tol), ed = eps_dual(p, tol);
        if (p->pri <= ep && p->dual <= ed && (!p->o.two_level || p->zn <= ep)) {
            p->status = 0;
            break;
        }
        if (p->o.two_level) {
            p->inner++;
            if ((p->pri_z <= eps_pri(p, p->tol_in) && p->dual <= eps_dual(p, p->tol_in)) ||
                p->inner >= p->o.max_inner) {
                outer_update(p, tol);
                if (p->outer >= p->o.max_outer) break;
            }
        }
    }
    return p->status;
}

int ora_get(const ora *p, int32_t which, double *out)
{
    switch (which) {
    case ORA_U: memcpy(out, p->u, sizeof(double) * p->m); return 0;
    case ORA_XBAR: memcpy(out, p->xbar, sizeof(double) * p->m); return 0;
    case ORA_Z: memcpy(out, p->z, sizeof(double) * p->m); return 0;
    case ORA_Y: memcpy(out, p->y, sizeof(double) * p->m); return 0;
    case ORA_LAMBDA: memcpy(out, p->lam, sizeof(double) * p->m); return 0;
    case ORA_BRANCH_X: memcpy(out, p->bx, sizeof(double) * 6 * p->nl); return 0;
    case ORA_BRANCH_LT: memcpy(out, p->lt, sizeof(double) * 2 * p->nl); return 0;
    case ORA_BUS: memcpy(out, p->bus, sizeof(double) * 2 * p->nb); return 0;
    case ORA_RHO: memcpy(out, p->rho, sizeof(double) * p->m); return 0;
    default: return -1;
    }
}

/* dres: pri, dual, zn, pri_z, beta, tol_in, ||u||, ||xbar||, ||y||;
 * ires: iters, outer, status, total */
void ora_get_residuals(const ora *p, double *dres, int32_t *ires)
{
    dres[0] = p->pri; dres[1] = p->dual; dres[2] = p->zn; dres[3] = p->pri_z;
    dres[4] = p->beta; dres[5] = p->tol_in;
    dres[6] = p->nu; dres[7] = p->nx; dres[8] = p->ny;
    ires[0] = p->iters; ires[1] = p->outer; ires[2] = p->status; ires[3] = p->total_iters;
}

int32_t ora_get_history(const ora *p, double *out, int32_t cap)
{
    int n = p->nhist < cap ? p->nhist : cap;
    memcpy(out, p->hist, sizeof(double) * 4 * n);
    return n;
}

void ora_get_stats(const ora *p, ora_stats *s) { *s = p->st; }

void ora_get_csr(const ora *p, int32_t *row_ptr, int32_t *col)
{
    for (int i = 0; i <= p->nb; ++i) row_ptr[i] = p->row[i];
    for (int k = 0; k < p->row[p->nb]; ++k) col[k] = p->col[k];
}

void ora_get_admittance(const ora *p, double *Y8) { memcpy(Y8, p->Y, sizeof(double) * 8 * p->nl); }

/* Section IV-A solution: generation from the generator subproblems, voltage
 * from the bus subproblems (v = sqrt(w)), flows recomputed from the bus
 * voltages.  obj_maxviol[0] = generation cost (unscaled),
 * obj_maxviol[1] = ||c(x)||_inf over the power balance of every bus, the line
 * limits (full rating) and the voltage bounds. */
void ora_finalize(const ora *p, double *pg, double *qg, double *vm, double *va,
                  double *pf, double *qf, double *pt, double *qt, double *obj_maxviol)
{
    double *v = dup_d(NULL, p->nb), *a = dup_d(NULL, p->nb);
    double *bp = dup_d(NULL, p->nb), *bq = dup_d(NULL, p->nb);
    double viol = 0.0, obj = 0.0;
    for (int i = 0; i < p->nb; ++i) {
        double w = p->bus[2 * i];
        v[i] = sqrt(w > 0.0 ? w : 0.0);
        a[i] = p->bus[2 * i + 1];
        double w2 = v[i] * v[i];
        bp[i] = -p->pd[i] - p->gs[i] * w2;
        bq[i] = -p->qd[i] + p->bs[i] * w2;
        double dv = v[i] - p->vmax[i];
        if (p->vmin[i] - v[i] > dv) dv = p->vmin[i] - v[i];
        if (dv > viol) viol = dv;
        if (vm) vm[i] = v[i];
        if (va) va[i] = a[i];
    }
    for (int k = 0; k < p->ng; ++k) {
        double P = p->u[2 * k], Q = p->u[2 * k + 1];
        bp[p->gb[k]] += P;
        bq[p->gb[k]] += Q;
        obj += p->c2[k] * P * P + p->c1[k] * P + p->c0[k];
        if (pg) pg[k] = P;
        if (qg) qg[k] = Q;
    }
    for (int l = 0; l < p->nl; ++l) {
        int i = p->fb[l], j = p->tb[l];
        double x[6] = {v[i], v[j], a[i], a[j], 0.0, 0.0}, fl[4];
        ora_branch_flows(&p->Y[8 * l], x, fl);
        bp[i] -= fl[0]; bq[i] -= fl[1];
        bp[j] -= fl[2]; bq[j] -= fl[3];
        if (p->rate[l] > 0.0) {
            double sf = sqrt(fl[0] * fl[0] + fl[1] * fl[1]) - p->rate[l];
            double st = sqrt(fl[2] * fl[2] + fl[3] * fl[3]) - p->rate[l];
            if (sf > viol) viol = sf;
            if (st > viol) viol = st;
        }
        if (pf) pf[l] = fl[0];
        if (qf) qf[l] = fl[1];
        if (pt) pt[l] = fl[2];
        if (qt) qt[l] = fl[3];
    }
    for (int i = 0; i < p->nb; ++i) {
        if (fabs(bp[i]) > viol) viol = fabs(bp[i]);
        if (fabs(bq[i]) > viol) viol = fabs(bq[i]);
    }
    obj_maxviol[0] = obj;
    obj_maxviol[1] = viol;
    free(v); free(a); free(bp); free(bq);
}
