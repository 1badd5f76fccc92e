// branch_tron: the branch x-update of Algorithm 1 (line 3) -- one thread per
// branch solves eq. branch (Section II-C): minimise over
// x = (v_i, v_j, theta_i(ij), theta_j(ij), s_ij, s_ji) within bounds
//   sum_c rho_c/2 (u_c(x) - t_c)^2 + sum_e [lt_e h_e + rt/2 h_e^2],
//   h_e = p_e^2 + q_e^2 + s_e,
// where t_c = xbar_c - z_c - y_c/rho_c are the targets written by the bus kernel
// (the paper's y r + rho/2 r^2 terms up to a constant).  The line limits are
// handled by an augmented Lagrangian loop around a trust-region Newton method
// for bound constraints (Lin-More TRON with Steihaug CG, Section III-B).
//
// Everything lives in registers: the 6x6 Hessian is packed (21 entries), the
// free-variable subspace of TRON is expressed with masks instead of index
// compaction so every loop has a compile-time trip count, and one sincos per
// function evaluation serves the four flows, their gradients and Hessians.
// The FP64 pipe is the bound (GB300 FP64 is a small fraction of FP32), so the
// code spends no FP64 work on anything that is not part of the method.
#include "admm_internal.cuh"

namespace admm {
namespace {

constexpr double kMu0 = 0.01, kEta0 = 1e-3, kEta1 = 0.25, kEta2 = 0.75;
constexpr double kSigma1 = 0.25, kSigma3 = 4.0, kCgRtol = 0.1;
constexpr int kCauchyTrials = 20, kPsTrials = 20, kCgMaxit = 12, kCholTries = 20;

// packed symmetric index (i <= j or j <= i)
__host__ __device__ constexpr int P(int i, int j)
{
    return i <= j ? (i * (11 - i)) / 2 + j : (j * (11 - j)) / 2 + i;
}

struct Prob {
    double Y[8];
    double lo[6], hi[6];
    double t[8];
    double rpq, rva, lt0, lt1, rt;
};

struct Cnt {
    int tron_calls, tron_iters, fgh, f, cauchy, cg, ps, al, maxhit;
};

__device__ __forceinline__ double clampd(double v, double lo, double hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

// One flow a_self v_k^2 + v_i v_j (alpha cos th + beta sin th), its gradient in
// (v_i, v_j, th) and Hessian entries (ii, jj, ij, i-th, j-th, th-th).
struct Flow {
    double F, d0, d1, d2, h00, h11, h01, h02, h12, h22;
};

template <bool kSelfI>
__device__ __forceinline__ void flow(double a, double al, double be, double vi, double vj,
                                     double vv, double c, double s, Flow &o, bool deriv)
{
    double T = al * c + be * s;
    double vk = kSelfI ? vi : vj;
    o.F = a * vk * vk + vv * T;
    if (!deriv) return;
    double Tp = be * c - al * s;
    o.d0 = (kSelfI ? 2.0 * a * vi : 0.0) + vj * T;
    o.d1 = (kSelfI ? 0.0 : 2.0 * a * vj) + vi * T;
    o.d2 = vv * Tp;
    o.h00 = kSelfI ? 2.0 * a : 0.0;
    o.h11 = kSelfI ? 0.0 : 2.0 * a;
    o.h01 = T;
    o.h02 = vj * Tp;
    o.h12 = vi * Tp;
    o.h22 = -vv * T;
}

__device__ __forceinline__ void flows4(const Prob &p, const double *x, Flow f[4], bool deriv)
{
    double vi = x[0], vj = x[1];
    double s, c;
    sincos(x[2] - x[3], &s, &c);
    double vv = vi * vj;
    flow<true>(p.Y[0], p.Y[2], p.Y[3], vi, vj, vv, c, s, f[0], deriv);      // p_ij
    flow<true>(-p.Y[1], -p.Y[3], p.Y[2], vi, vj, vv, c, s, f[1], deriv);    // q_ij
    flow<false>(p.Y[6], p.Y[4], -p.Y[5], vi, vj, vv, c, s, f[2], deriv);    // p_ji
    flow<false>(-p.Y[7], -p.Y[5], -p.Y[4], vi, vj, vv, c, s, f[3], deriv);  // q_ji
}

__device__ __forceinline__ double fval(const Prob &p, const double *x)
{
    Flow fl[4];
    flows4(p, x, fl, false);
    double r0 = fl[0].F - p.t[0], r1 = fl[1].F - p.t[1], r2 = fl[2].F - p.t[2],
           r3 = fl[3].F - p.t[3];
    double rwi = x[0] * x[0] - p.t[4], rti = x[2] - p.t[5];
    double rwj = x[1] * x[1] - p.t[6], rtj = x[3] - p.t[7];
    double h0 = fl[0].F * fl[0].F + fl[1].F * fl[1].F + x[4];
    double h1 = fl[2].F * fl[2].F + fl[3].F * fl[3].F + x[5];
    double f = 0.5 * p.rpq * (r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3)
             + 0.5 * p.rva * (rwi * rwi + rti * rti + rwj * rwj + rtj * rtj);
    f += p.lt0 * h0 + 0.5 * p.rt * h0 * h0;
    f += p.lt1 * h1 + 0.5 * p.rt * h1 * h1;
    return f;
}

// gradient and packed Hessian (f not needed by callers)
__device__ __forceinline__ void fgh(const Prob &p, const double *x, double *g, double *H)
{
    Flow fl[4];
    flows4(p, x, fl, true);
    double h0 = fl[0].F * fl[0].F + fl[1].F * fl[1].F + x[4];
    double h1 = fl[2].F * fl[2].F + fl[3].F * fl[3].F + x[5];
    double mu0 = p.lt0 + p.rt * h0, mu1 = p.lt1 + p.rt * h1;
    double mu[4] = {mu0, mu0, mu1, mu1};
    // coefficient of each flow gradient and of each flow Hessian
    double G0 = 0.0, G1 = 0.0, G2 = 0.0;
    double A00 = 0.0, A11 = 0.0, A01 = 0.0, A02 = 0.0, A12 = 0.0, A22 = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double ck = p.rpq * (fl[k].F - p.t[k]) + 2.0 * mu[k] * fl[k].F;
        double wk = p.rpq + 2.0 * mu[k];
        G0 += ck * fl[k].d0;
        G1 += ck * fl[k].d1;
        G2 += ck * fl[k].d2;
        A00 += ck * fl[k].h00 + wk * fl[k].d0 * fl[k].d0;
        A11 += ck * fl[k].h11 + wk * fl[k].d1 * fl[k].d1;
        A01 += ck * fl[k].h01 + wk * fl[k].d0 * fl[k].d1;
        A02 += ck * fl[k].h02 + wk * fl[k].d0 * fl[k].d2;
        A12 += ck * fl[k].h12 + wk * fl[k].d1 * fl[k].d2;
        A22 += ck * fl[k].h22 + wk * fl[k].d2 * fl[k].d2;
    }
    // gradients of h_e in (v_i, v_j, th)
    double e00 = 2.0 * (fl[0].F * fl[0].d0 + fl[1].F * fl[1].d0);
    double e01 = 2.0 * (fl[0].F * fl[0].d1 + fl[1].F * fl[1].d1);
    double e02 = 2.0 * (fl[0].F * fl[0].d2 + fl[1].F * fl[1].d2);
    double e10 = 2.0 * (fl[2].F * fl[2].d0 + fl[3].F * fl[3].d0);
    double e11 = 2.0 * (fl[2].F * fl[2].d1 + fl[3].F * fl[3].d1);
    double e12 = 2.0 * (fl[2].F * fl[2].d2 + fl[3].F * fl[3].d2);
    const double rt = p.rt;
    A00 += rt * (e00 * e00 + e10 * e10);
    A11 += rt * (e01 * e01 + e11 * e11);
    A01 += rt * (e00 * e01 + e10 * e11);
    A02 += rt * (e00 * e02 + e10 * e12);
    A12 += rt * (e01 * e02 + e11 * e12);
    A22 += rt * (e02 * e02 + e12 * e12);
    double vi = x[0], vj = x[1];
    double rwi = vi * vi - p.t[4], rwj = vj * vj - p.t[6];
    g[0] = G0 + p.rva * rwi * 2.0 * vi;
    g[1] = G1 + p.rva * rwj * 2.0 * vj;
    g[2] = G2 + p.rva * (x[2] - p.t[5]);
    g[3] = -G2 + p.rva * (x[3] - p.t[7]);
    g[4] = mu0;
    g[5] = mu1;
    H[P(0, 0)] = A00 + p.rva * (4.0 * vi * vi + 2.0 * rwi);
    H[P(0, 1)] = A01;
    H[P(0, 2)] = A02;
    H[P(0, 3)] = -A02;
    H[P(0, 4)] = rt * e00;
    H[P(0, 5)] = rt * e10;
    H[P(1, 1)] = A11 + p.rva * (4.0 * vj * vj + 2.0 * rwj);
    H[P(1, 2)] = A12;
    H[P(1, 3)] = -A12;
    H[P(1, 4)] = rt * e01;
    H[P(1, 5)] = rt * e11;
    H[P(2, 2)] = A22 + p.rva;
    H[P(2, 3)] = -A22;
    H[P(2, 4)] = rt * e02;
    H[P(2, 5)] = rt * e12;
    H[P(3, 3)] = A22 + p.rva;
    H[P(3, 4)] = -rt * e02;
    H[P(3, 5)] = -rt * e12;
    H[P(4, 4)] = rt;
    H[P(4, 5)] = 0.0;
    H[P(5, 5)] = rt;
}

__device__ __forceinline__ double dot6(const double *a, const double *b)
{
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) s += a[i] * b[i];
    return s;
}

__device__ __forceinline__ void hmul(const double *H, const double *v, double *o)
{
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < 6; ++j) s += H[P(i, j)] * v[j];
        o[i] = s;
    }
}

__device__ __forceinline__ double qmodel(const double *g, const double *H, const double *s)
{
    double Hs[6];
    hmul(H, s, Hs);
    return dot6(g, s) + 0.5 * dot6(s, Hs);
}

__device__ __forceinline__ void pstep(const Prob &p, const double *x, const double *g,
                                      double a, double *s)
{
#pragma unroll
    for (int i = 0; i < 6; ++i) s[i] = clampd(x[i] - a * g[i], p.lo[i], p.hi[i]) - x[i];
}

__device__ __forceinline__ double pgnorm(const Prob &p, const double *x, const double *g)
{
    double m = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) m = fmax(m, fabs(clampd(x[i] - g[i], p.lo[i], p.hi[i]) - x[i]));
    return m;
}

__device__ __forceinline__ bool cauchy_ok(const double *g, const double *H, const double *s,
                                          double delta)
{
    return sqrt(dot6(s, s)) <= delta && qmodel(g, H, s) <= kMu0 * dot6(g, s);
}

// generalised Cauchy step along the projected-gradient path
__device__ void cauchy(const Prob &p, const double *x, const double *g, const double *H,
                       double delta, double &alpha, double *s, Cnt &c)
{
    double brmax = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double bp = 0.0;
        if (g[i] > 0.0 && x[i] > p.lo[i]) bp = (x[i] - p.lo[i]) / g[i];
        else if (g[i] < 0.0 && x[i] < p.hi[i]) bp = (x[i] - p.hi[i]) / g[i];
        brmax = fmax(brmax, bp);
    }
    double a = alpha;
    pstep(p, x, g, a, s);
    c.cauchy++;
    if (!cauchy_ok(g, H, s, delta)) {
        for (int t = 0; t < kCauchyTrials; ++t) {
            a *= 0.1;
            pstep(p, x, g, a, s);
            c.cauchy++;
            if (cauchy_ok(g, H, s, delta)) break;
        }
    } else {
        for (int t = 0; t < kCauchyTrials; ++t) {
            if (a >= brmax) break;
            double an = a * 10.0, sn[6];
            pstep(p, x, g, an, sn);
            c.cauchy++;
            if (!cauchy_ok(g, H, sn, delta)) break;
            a = an;
#pragma unroll
            for (int i = 0; i < 6; ++i) s[i] = sn[i];
        }
    }
    alpha = a;
}

__device__ __forceinline__ double boundary_tau(const double *a, const double *pv, double delta)
{
    double pp = dot6(pv, pv), ap = dot6(a, pv), aa = dot6(a, a);
    double rad = fmax(delta * delta - aa, 0.0);
    double disc = sqrt(ap * ap + pp * rad);
    if (pp == 0.0) return 0.0;
    return ap > 0.0 ? rad / (ap + disc) : (disc - ap) / pp;
}

// Preconditioner: Cholesky of the scaled free block plus sigma I (identity on
// fixed variables); L packed lower-triangular, d the diagonal scaling.
__device__ void precond_factor(const double *H, const bool *fr, double *L, double *d)
{
    bool pos = true;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double a = H[P(i, i)];
        d[i] = (fr[i] && a != 0.0) ? sqrt(fabs(a)) : 1.0;
        if (fr[i] && !(a > 0.0)) pos = false;
    }
    double sigma = pos ? 0.0 : 1e-3;
    for (int tries = 0; tries < kCholTries; ++tries) {
        bool ok = true;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            double dd = fr[j] ? H[P(j, j)] / (d[j] * d[j]) + sigma : 1.0;
#pragma unroll
            for (int k = 0; k < j; ++k) dd -= L[P(j, k)] * L[P(j, k)];
            ok = ok && (dd > 0.0);
            double ljj = sqrt(fmax(dd, 1e-300));
            L[P(j, j)] = ljj;
#pragma unroll
            for (int i = j + 1; i < 6; ++i) {
                double v = (fr[i] && fr[j]) ? H[P(i, j)] / (d[i] * d[j]) : 0.0;
#pragma unroll
                for (int k = 0; k < j; ++k) v -= L[P(i, k)] * L[P(j, k)];
                L[P(i, j)] = v / ljj;
            }
        }
        if (ok) return;
        sigma = fmax(sigma * 2.0, 1e-3);
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) L[P(i, j)] = (i == j) ? 1.0 : 0.0;
    }
}

__device__ __forceinline__ void precond_solve(const double *L, const double *d, const double *r,
                                              double *z)
{
    double t[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double v = r[i] / d[i];
#pragma unroll
        for (int k = 0; k < i; ++k) v -= L[P(i, k)] * t[k];
        t[i] = v / L[P(i, i)];
    }
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        double v = t[i];
#pragma unroll
        for (int k = i + 1; k < 6; ++k) v -= L[P(k, i)] * t[k];
        t[i] = v / L[P(i, i)];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) z[i] = t[i] / d[i];
}

// Subspace step: Steihaug PCG on the free variables of the Cauchy point, then
// a projected backtracking search along the CG direction.
__device__ void subspace(const Prob &p, const double *x, const double *g, const double *H,
                         double delta, const double *sc, double *s, Cnt &c)
{
    bool fr[6];
    double xc[6];
    bool any = false;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        xc[i] = x[i] + sc[i];
        fr[i] = xc[i] > p.lo[i] && xc[i] < p.hi[i];
        any = any || fr[i];
        s[i] = sc[i];
    }
    if (!any) return;
    double gc[6];
    hmul(H, sc, gc);
#pragma unroll
    for (int i = 0; i < 6; ++i) gc[i] += g[i];
    double L[21], d[6];
    precond_factor(H, fr, L, d);
    double w[6], r[6], z[6], pv[6], q[6];
    double rn0 = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        w[i] = 0.0;
        r[i] = fr[i] ? -gc[i] : 0.0;
        rn0 += r[i] * r[i];
    }
    rn0 = sqrt(rn0);
    if (rn0 == 0.0) return;
    precond_solve(L, d, r, z);
    double rz = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        pv[i] = fr[i] ? z[i] : 0.0;
        rz += r[i] * pv[i];
    }
    const double tol = kCgRtol * rn0;
    for (int it = 0; it < kCgMaxit; ++it) {
        c.cg++;
        hmul(H, pv, q);
        double kappa = 0.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            q[i] = fr[i] ? q[i] : 0.0;
            kappa += pv[i] * q[i];
        }
        double cur[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) cur[i] = sc[i] + w[i];
        if (kappa <= 0.0) {
            double tau = boundary_tau(cur, pv, delta);
#pragma unroll
            for (int i = 0; i < 6; ++i) w[i] += tau * pv[i];
            break;
        }
        double al = rz / kappa, nx[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) nx[i] = cur[i] + al * pv[i];
        if (sqrt(dot6(nx, nx)) >= delta) {
            double tau = boundary_tau(cur, pv, delta);
#pragma unroll
            for (int i = 0; i < 6; ++i) w[i] += tau * pv[i];
            break;
        }
        double rn = 0.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            w[i] += al * pv[i];
            r[i] -= al * q[i];
            rn += r[i] * r[i];
        }
        if (sqrt(rn) <= tol) break;
        precond_solve(L, d, r, z);
        double rz1 = 0.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            z[i] = fr[i] ? z[i] : 0.0;
            rz1 += r[i] * z[i];
        }
        double be = rz1 / rz;
        rz = rz1;
#pragma unroll
        for (int i = 0; i < 6; ++i) pv[i] = z[i] + be * pv[i];
    }
    double qc = qmodel(g, H, sc);
    double beta = 1.0;
    for (int t = 0; t < kPsTrials; ++t) {
        c.ps++;
        double sb[6], dd[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            sb[i] = clampd(xc[i] + beta * w[i], p.lo[i], p.hi[i]) - x[i];
            dd[i] = sb[i] - sc[i];
        }
        if (qmodel(g, H, sb) <= qc + kMu0 * dot6(gc, dd)) {
#pragma unroll
            for (int i = 0; i < 6; ++i) s[i] = sb[i];
            return;
        }
        beta *= 0.5;
    }
}

// TRON on eq. branch from x; returns 0 converged, 1 iteration cap, 2 stalled
__device__ int tron(const Prob &p, double *x, const DevOpts &O, Cnt &c)
{
#pragma unroll
    for (int i = 0; i < 6; ++i) x[i] = clampd(x[i], p.lo[i], p.hi[i]);
    double g[6], H[21];
    double f = fval(p, x);
    fgh(p, x, g, H);
    c.tron_calls++;
    c.fgh++;
    const double pg0 = pgnorm(p, x, g);
    const double gtol = O.tron_gtol * fmax(pg0, 1.0);
    double sp[6];
    pstep(p, x, g, 1.0, sp);
    double delta = sqrt(dot6(sp, sp));
    double alpha = 1.0;
    int status = 1;
    for (int k = 0; k < O.tron_max_iter; ++k) {
        if (pgnorm(p, x, g) <= gtol) { status = 0; break; }
        c.tron_iters++;
        double sc[6], s[6];
        cauchy(p, x, g, H, delta, alpha, sc, c);
        subspace(p, x, g, H, delta, sc, s, c);
        double xn = 0.0, sn = 0.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            xn = fmax(xn, fabs(x[i]));
            sn = fmax(sn, fabs(s[i]));
        }
        if (sn <= O.tron_xtol * fmax(xn, 1.0)) { status = 0; break; }
        double xt[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) xt[i] = clampd(x[i] + s[i], p.lo[i], p.hi[i]);
        double ft = fval(p, xt);
        c.f++;
        double prered = -qmodel(g, H, s);
        double actred = f - ft;
        double snorm = sqrt(dot6(s, s));
        if (k == 0 && snorm < delta) delta = snorm;
        double fa = fmax(fabs(f), 1.0);
        double ratio;
        if (prered <= 0.0) ratio = -1.0;
        else if (prered <= O.tron_ftol * fa) ratio = 1.0;
        else ratio = actred / prered;
        if (ratio < kEta1) delta = kSigma1 * fmin(snorm, delta);
        else if (ratio > kEta2) delta = fmax(delta, kSigma3 * snorm);
        if (ratio > kEta0) {
#pragma unroll
            for (int i = 0; i < 6; ++i) x[i] = xt[i];
            f = ft;
            fgh(p, x, g, H);
            c.fgh++;
        }
        if (prered <= 0.0) { status = 2; break; }
        xn = 0.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) xn = fmax(xn, fabs(x[i]));
        if (delta <= 1e-14 * fmax(xn, 1.0)) { status = 2; break; }
    }
    if (status == 1) c.maxhit++;
    return status;
}

__device__ __forceinline__ void warp_add_u64(unsigned long long *dst, int v)
{
    unsigned int s = __reduce_add_sync(0xffffffffu, (unsigned int)v);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(dst, (unsigned long long)s);
}

}  // namespace

__global__ void __launch_bounds__(kBranchBlock) branch_tron_kernel(DevGrid G, DevOpts O)
{
    Ctrl *ctrl = G.ctrl;
    if (ctrl->done) return;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    const int nl = G.nl;
    Cnt c = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (l < nl) {
        Prob p;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            p.Y[k] = G.Y[k * nl + l];
            p.t[k] = G.bt[k * nl + l];
        }
        p.lo[0] = G.lim[0 * nl + l]; p.hi[0] = G.lim[1 * nl + l];
        p.lo[1] = G.lim[2 * nl + l]; p.hi[1] = G.lim[3 * nl + l];
        p.lo[2] = -kTwoPi; p.hi[2] = kTwoPi;
        p.lo[3] = -kTwoPi; p.hi[3] = kTwoPi;
        p.lo[4] = G.lim[4 * nl + l]; p.hi[4] = 0.0;
        p.lo[5] = p.lo[4]; p.hi[5] = 0.0;
        p.rpq = ctrl->rho_pq;
        p.rva = ctrl->rho_va;
        p.lt0 = G.blt[l];
        p.lt1 = G.blt[nl + l];
        p.rt = O.al_rho0 > 0.0 ? O.al_rho0 : p.rpq;
        double x[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) x[k] = G.bx[k * nl + l];
        // augmented Lagrangian on p^2 + q^2 + s = 0 of both ends
        double hprev = __longlong_as_double(0x7ff0000000000000LL);
        Flow fl[4];
        for (int a = 0; a < O.al_max_iter; ++a) {
            c.al++;
            tron(p, x, O, c);
            flows4(p, x, fl, false);
            double h0 = fl[0].F * fl[0].F + fl[1].F * fl[1].F + x[4];
            double h1 = fl[2].F * fl[2].F + fl[3].F * fl[3].F + x[5];
            p.lt0 += p.rt * h0;
            p.lt1 += p.rt * h1;
            double hm = fmax(fabs(h0), fabs(h1));
            if (hm <= O.al_tol) break;
            if (hm > O.al_decay * hprev) p.rt = fmin(p.rt * O.al_rho_factor, O.al_rho_max);
            hprev = hm;
        }
        if (O.al_max_iter <= 0) flows4(p, x, fl, false);
#pragma unroll
        for (int k = 0; k < 6; ++k) G.bx[k * nl + l] = x[k];
        G.blt[l] = p.lt0;
        G.blt[nl + l] = p.lt1;
        G.bu[0 * nl + l] = fl[0].F;
        G.bu[1 * nl + l] = fl[1].F;
        G.bu[2 * nl + l] = fl[2].F;
        G.bu[3 * nl + l] = fl[3].F;
        G.bu[4 * nl + l] = x[0] * x[0];
        G.bu[5 * nl + l] = x[2];
        G.bu[6 * nl + l] = x[1] * x[1];
        G.bu[7 * nl + l] = x[3];
    }
    unsigned long long *st = ctrl->stats;
    warp_add_u64(&st[ST_TRON_CALLS], c.tron_calls);
    warp_add_u64(&st[ST_TRON_ITERS], c.tron_iters);
    warp_add_u64(&st[ST_FGH], c.fgh);
    warp_add_u64(&st[ST_F], c.f);
    warp_add_u64(&st[ST_CAUCHY], c.cauchy);
    warp_add_u64(&st[ST_CG], c.cg);
    warp_add_u64(&st[ST_PS], c.ps);
    warp_add_u64(&st[ST_AL], c.al);
    warp_add_u64(&st[ST_TRON_MAXHIT], c.maxhit);
}

}  // namespace admm
