// branch_tron: the branch part of the x-update of Algorithm 1.  Every branch
// solves eq. branch (Section II-C): minimise over
// x = (v_i, v_j, theta_i(ij), theta_j(ij), s_ij, s_ji) within bounds
//   sum_c rho_c/2 (u_c(x) - t_c)^2 + sum_e [lt_e h_e + rt/2 h_e^2],
//   h_e = p_e^2 + q_e^2 + s_e,
// where t_c = xbar_c - z_c - y_c/rho_c are the targets written by the bus kernel
// (the paper's y r + rho/2 r^2 terms up to a constant).  The line limits are
// handled by an augmented Lagrangian loop around a trust-region Newton method
// for bound constraints (Lin-More TRON with Steihaug CG, Section III-B).
//
// GB300 design.  FP64 runs at about 1.7 FMA per clock per SM (0.42 per
// sub-partition, measured: one warp instruction per ~76 cycles; FP32 is ~76
// times faster), so the kernel is bound by FP64 warp instructions, and a warp
// instruction costs the same whether 32 lanes or 1 lane are active.  Branch
// problems need very different amounts of work (1 to several AL passes, 1 to
// dozens of TRON iterations), so one-branch-per-thread with a fixed assignment
// leaves most lanes idle.  Instead the grid is persistent and every lane pulls
// a new branch from a queue as soon as its branch is finished; each trip of
// the main loop performs exactly one TRON iteration in every lane that has one
// to do, so the expensive code runs with nearly full warps.  One lane solves
// one branch (its Hessian and preconditioner factor packed, 21 entries each,
// in shared memory, everything else in registers; the TRON free set handled
// with masks so all loops have fixed trip counts); the branch data the
// evaluations read (admittances and targets) sit in shared memory too.  The
// function, gradient and Hessian are evaluated together at every trial point
// (one sincos), since nearly every trial step is accepted; after a rejected
// step the gradient and Hessian are re-evaluated at the kept point.
#include "admm_internal.cuh"

namespace admm {
namespace {

constexpr double kMu0 = 0.01, kEta0 = 1e-3, kEta1 = 0.25, kEta2 = 0.75;
constexpr double kSigma1 = 0.25, kSigma3 = 4.0, kCgRtol = 0.1;
constexpr int kCauchyTrials = 20, kPsTrials = 20, kCgMaxit = 12, kCholTries = 20;
constexpr unsigned kFull = 0xffffffffu;

// packed symmetric index
__host__ __device__ constexpr int P(int i, int j)
{
    return i <= j ? (i * (11 - i)) / 2 + j : (j * (11 - j)) / 2 + i;
}

// A lane's packed symmetric matrices (the Hessian and the preconditioner's
// factor) and its scratch live in shared memory: held in registers each
// matrix costs 42 of the 255 registers a lane has, and the subspace step then
// spills.  Entries are stored in pairs, the block's lanes interleaved pair by
// pair (entry k of lane t at (k / 2) * 2 kBranchBlock + 2 t + k % 2), so that
// two consecutive entries are one 16-byte access.
struct SMat {
    double *p;   // the lane's first pair
    __device__ __forceinline__ double &operator[](int k) const
    {
        return p[(k >> 1) * (2 * kBranchBlock) + (k & 1)];
    }
};

struct Cnt {
    int tron_calls, tron_iters, fgh, f, cauchy, cg, ps, al, maxhit;
};

// Order-preserving integer images of doubles (NaN excluded, -0 == +0).
// GB300 executes double compare / min / max on the FP64 pipe at the FP64 rate,
// so every comparison, min, max and clamp of the solver runs on these keys on
// the integer pipe instead; only arithmetic uses the FP64 pipe.
__device__ __forceinline__ long long okey(double v)
{
    const long long b = __double_as_longlong(v);
    const long long m = b & 0x7fffffffffffffffLL;
    return b < 0 ? -m : m;
}
__device__ __forceinline__ bool dlt(double a, double b) { return okey(a) < okey(b); }
__device__ __forceinline__ bool dle(double a, double b) { return okey(a) <= okey(b); }
__device__ __forceinline__ bool dpos(double a) { return __double_as_longlong(a) > 0; }   // a > 0
__device__ __forceinline__ bool dneg(double a) { return okey(a) < 0; }                   // a < 0
__device__ __forceinline__ double dmaxi(double a, double b) { return dlt(a, b) ? b : a; }
__device__ __forceinline__ double dmini(double a, double b) { return dlt(b, a) ? b : a; }
__device__ __forceinline__ double dabsi(double a)
{
    return __longlong_as_double(__double_as_longlong(a) & 0x7fffffffffffffffLL);
}
// max of |a| over values: the bits of non-negative doubles order like integers
__device__ __forceinline__ double amax(double m, double a)
{
    const long long ba = __double_as_longlong(a) & 0x7fffffffffffffffLL;
    return ba > __double_as_longlong(m) ? __longlong_as_double(ba) : m;
}

// v * 2^-k for k >= 0 by an exponent shift on the integer pipe: exact for
// a normal v whose exponent stays normal; 0 where the result would be
// subnormal (and for v = 0)
__device__ __forceinline__ double pow2_scale(double v, int k)
{
    const long long b = __double_as_longlong(v);
    const long long e = (b >> 52) & 0x7ff;
    return e > k ? __longlong_as_double(b - ((long long)k << 52)) : 0.0;
}

// v * 2^k for k >= 0 by an exponent step on the integer pipe: exact for a
// normal v whose result stays finite; v itself for 0, subnormals, infinities,
// NaN and results that would overflow
__device__ __forceinline__ double pow2_up(double v, int k)
{
    const long long b = __double_as_longlong(v);
    const long long e = (b >> 52) & 0x7ff;
    return (e != 0 && e + k < 0x7ff) ? __longlong_as_double(b + ((long long)k << 52)) : v;
}
__device__ __forceinline__ double twice(double v) { return pow2_up(v, 1); }

// Two lanes per branch (kL = 2): lanes 2k and 2k+1 hold the same branch and
// the same state, bit for bit; the parts of a trip that split cleanly (the two
// line ends' flows, rows of 6x6 products, halves of 6-vector dot products)
// are computed half on each lane and exchanged.  Every combined value is a
// single sum mine + partner's, which is the same on both lanes (IEEE addition
// commutes), so both lanes keep taking the same decisions.  m is the mask of
// the lanes executing the call; pairs are always both in or both out, and
// every lane named in m must reach the call: never place one of these products
// behind a short-circuit (&&, ||, ?:) that some lanes of m skip.
__device__ __forceinline__ bool odd_lane() { return (threadIdx.x & 1) != 0; }
__device__ __forceinline__ double partner(unsigned m, double v) { return __shfl_xor_sync(m, v, 1); }

// bounds of one branch: v_i, v_j from the buses, theta copies +-2 pi, slacks;
// kept with their keys
struct Bounds {
    double vlo_i, vhi_i, vlo_j, vhi_j, slo;
    long long kvlo_i, kvhi_i, kvlo_j, kvhi_j, kslo;
    __device__ __forceinline__ void set_keys()
    {
        kvlo_i = okey(vlo_i); kvhi_i = okey(vhi_i); kvlo_j = okey(vlo_j); kvhi_j = okey(vhi_j);
        kslo = okey(slo);
    }
    __device__ __forceinline__ double lo(int i) const
    {
        return i == 0 ? vlo_i : i == 1 ? vlo_j : i < 4 ? -kTwoPi : slo;
    }
    __device__ __forceinline__ double hi(int i) const
    {
        return i == 0 ? vhi_i : i == 1 ? vhi_j : i < 4 ? kTwoPi : 0.0;
    }
    __device__ __forceinline__ long long klo(int i) const
    {
        return i == 0 ? kvlo_i : i == 1 ? kvlo_j : i < 4 ? -0x401921FB54442D18LL : kslo;
    }
    __device__ __forceinline__ long long khi(int i) const
    {
        return i == 0 ? kvhi_i : i == 1 ? kvhi_j : i < 4 ? 0x401921FB54442D18LL : 0LL;
    }
    // P_[lo_i, hi_i](v)
    __device__ __forceinline__ double clamp(int i, double v) const
    {
        const long long k = okey(v);
        return k < klo(i) ? lo(i) : (k > khi(i) ? hi(i) : v);
    }
    __device__ __forceinline__ bool above_lo(int i, double v) const { return okey(v) > klo(i); }
    __device__ __forceinline__ bool below_hi(int i, double v) const { return okey(v) < khi(i); }
};

// One line end's two flows p and q.  A flow is a v_k^2 + v_i v_j T(th) with
// T = al cos th + be sin th, T' = dT/dth = be cos th - al sin th; an end's q
// flow has the angle factors (Tq, Tq') = (-sg T', sg T) of its p flow's, with
// sg = +1 at the from end and -1 at the to end, so the pair shares the six
// products of (v_j, v_i, v_i v_j) with (T, T').  Adds the end's terms to the
// gradient and Hessian sums (ck = rho_pq r + 2 mu F and wk = rho_pq + 2 mu per
// flow, mu = lt + rt h of the end) and returns the end's halves of
// grad h = 2 sum F dF in e0..e2.  from: the from end (self term in v_i); a
// constant for one lane per branch, the lane's end (a selection, not a branch
// of the code) for two.
struct EndSums {
    double G0, G1, G2, A00, A11, A01, A02, A12, A22, fq;
};

__device__ __forceinline__ void end_terms(bool from, double ap, double aq, double vi, double vj, double vv,
                                          double T, double Tp, double Fp, double Fq, double tp,
                                          double tq, double rpq, double mu, EndSums &E,
                                          double &e0, double &e1, double &e2)
{
    const double jT = vj * T, iT = vi * T, vT = vv * T;
    const double jP = vj * Tp, iP = vi * Tp, vP = vv * Tp;
    // the q flow's v_j Tq, v_i Tq, vv Tq and v_j Tq', v_i Tq', vv Tq'
    const double Tq = from ? -Tp : Tp;
    const double jTq = from ? -jP : jP, iTq = from ? -iP : iP, vTq = from ? -vP : vP;
    const double jPq = from ? jT : -jT, iPq = from ? iT : -iT, vPq = from ? vT : -vT;
    const double vk = from ? vi : vj;
    // doublings (2 mu, 2 a, 2 (...)) are exponent steps on the integer pipe
    const double m2 = twice(mu), wk = rpq + m2;
    const double ap2 = twice(ap), aq2 = twice(aq);
    // dF = (2a v_i + v_j T, v_i T, vv T') (from end) or (v_j T, 2a v_j + v_i T, vv T');
    // d2F: self term 2a, (0,1) T, (0,2) v_j T', (1,2) v_i T', (2,2) -vv T
    const double dp0 = from ? ap2 * vk + jT : jT;
    const double dp1 = from ? iT : ap2 * vk + iT;
    const double dq0 = from ? aq2 * vk + jTq : jTq;
    const double dq1 = from ? iTq : aq2 * vk + iTq;
    const double dp2 = vP, dq2 = vPq;
    const double rp = Fp - tp, rq = Fq - tq;
    E.fq += rp * rp + rq * rq;
    const double cp = rpq * rp + m2 * Fp, cq = rpq * rq + m2 * Fq;
    E.G0 += cp * dp0 + cq * dq0;
    E.G1 += cp * dp1 + cq * dq1;
    E.G2 += cp * dp2 + cq * dq2;
    const double sd = twice(cp * ap + cq * aq);          // c times the self second derivative
    if (from) E.A00 += sd; else E.A11 += sd;
    E.A00 += wk * (dp0 * dp0 + dq0 * dq0);
    E.A11 += wk * (dp1 * dp1 + dq1 * dq1);
    E.A01 += (cp * T + cq * Tq) + wk * (dp0 * dp1 + dq0 * dq1);
    E.A02 += (cp * jP + cq * jPq) + wk * (dp0 * dp2 + dq0 * dq2);
    E.A12 += (cp * iP + cq * iPq) + wk * (dp1 * dp2 + dq1 * dq2);
    E.A22 += -(cp * vT + cq * vTq) + wk * (dp2 * dp2 + dq2 * dq2);
    e0 = twice(Fp * dp0 + Fq * dq0);
    e1 = twice(Fp * dp1 + Fq * dq1);
    e2 = twice(Fp * dp2 + Fq * dq2);
}

// f, gradient, packed Hessian and the four flows of eq. branch at x.
// Y and t live in shared memory with stride kBranchBlock.  The flow values
// come first (h and the multipliers mu need all four), then each end's terms.
__device__ __forceinline__ void evaluate1(const double *sY, const double *sT, double rpq, double rva,
                                          double lt0, double lt1, double rt, const double *x,
                                          double &f, double *g, SMat H, double *F)
{
    const double vi = x[0], vj = x[1];
    double s, c;
    sincos(x[2] - x[3], &s, &c);
    const double vv = vi * vj;
    constexpr int S = kBranchBlock;
    const double gii = sY[0 * S], bii = sY[1 * S], gij = sY[2 * S], bij = sY[3 * S];
    const double gji = sY[4 * S], bji = sY[5 * S], gjj = sY[6 * S], bjj = sY[7 * S];
    // eqs. (pij)-(qji): p_ij = g_ii v_i^2 + vv T_i, q_ij = -b_ii v_i^2 - vv T'_i with
    // (al, be) = (g_ij, b_ij); p_ji = g_jj v_j^2 + vv T_j, q_ji = -b_jj v_j^2 + vv T'_j
    // with (al, be) = (g_ji, -b_ji)
    const double Ti = gij * c + bij * s, Tpi = bij * c - gij * s;
    const double Tj = gji * c - bji * s, Tpj = -bji * c - gji * s;
    const double wi = vi * vi, wj = vj * vj;
    F[0] = gii * wi + vv * Ti;
    F[1] = -bii * wi - vv * Tpi;
    F[2] = gjj * wj + vv * Tj;
    F[3] = -bjj * wj + vv * Tpj;
    const double h0 = F[0] * F[0] + F[1] * F[1] + x[4];
    const double h1 = F[2] * F[2] + F[3] * F[3] + x[5];
    const double mu0 = lt0 + rt * h0, mu1 = lt1 + rt * h1;
    EndSums E = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    double e00, e01, e02, e10, e11, e12;
    end_terms(true, gii, -bii, vi, vj, vv, Ti, Tpi, F[0], F[1], sT[0 * S], sT[1 * S], rpq, mu0,
                    E, e00, e01, e02);
    end_terms(false, gjj, -bjj, vi, vj, vv, Tj, Tpj, F[2], F[3], sT[2 * S], sT[3 * S], rpq, mu1,
                     E, e10, e11, e12);
    // the AL terms' Gauss-Newton part rt grad h grad h'
    const double r00 = rt * e00, r01 = rt * e01, r02 = rt * e02;
    const double r10 = rt * e10, r11 = rt * e11, r12 = rt * e12;
    const double A00 = E.A00 + (r00 * e00 + r10 * e10);
    const double A11 = E.A11 + (r01 * e01 + r11 * e11);
    const double A01 = E.A01 + (r00 * e01 + r10 * e11);
    const double A02 = E.A02 + (r00 * e02 + r10 * e12);
    const double A12 = E.A12 + (r01 * e02 + r11 * e12);
    const double A22 = E.A22 + (r02 * e02 + r12 * e12);
    const double rwi = wi - sT[4 * S], rti = x[2] - sT[5 * S];
    const double rwj = wj - sT[6 * S], rtj = x[3] - sT[7 * S];
    const double hrt = pow2_scale(rt, 1), trva = twice(rva);
    f = pow2_scale(rpq, 1) * E.fq + pow2_scale(rva, 1) * (rwi * rwi + rti * rti + rwj * rwj + rtj * rtj)
      + lt0 * h0 + hrt * h0 * h0 + lt1 * h1 + hrt * h1 * h1;
    g[0] = E.G0 + trva * rwi * vi;
    g[1] = E.G1 + trva * rwj * vj;
    g[2] = E.G2 + rva * rti;
    g[3] = -E.G2 + rva * rtj;
    g[4] = mu0;
    g[5] = mu1;
    H[P(0, 0)] = A00 + rva * (4.0 * wi + twice(rwi));
    H[P(0, 1)] = A01;
    H[P(0, 2)] = A02;
    H[P(0, 3)] = -A02;
    H[P(0, 4)] = r00;
    H[P(0, 5)] = r10;
    H[P(1, 1)] = A11 + rva * (4.0 * wj + twice(rwj));
    H[P(1, 2)] = A12;
    H[P(1, 3)] = -A12;
    H[P(1, 4)] = r01;
    H[P(1, 5)] = r11;
    H[P(2, 2)] = A22 + rva;
    H[P(2, 3)] = -A22;
    H[P(2, 4)] = r02;
    H[P(2, 5)] = r12;
    H[P(3, 3)] = A22 + rva;
    H[P(3, 4)] = -r02;
    H[P(3, 5)] = -r12;
    H[P(4, 4)] = rt;
    H[P(4, 5)] = 0.0;
    H[P(5, 5)] = rt;
}

// The same with two lanes per branch: the even lane takes the from end's two
// flows (p_ij, q_ij), the odd lane the to end's (p_ji, q_ji); each forms its
// end's shares of the gradient and Hessian sums, the pair swaps them and both
// assemble f, g and H from (from-end share + to-end share).
__device__ __forceinline__ void evaluate2(unsigned m, const double *sY, const double *sT,
                                          double rpq, double rva, double lt0, double lt1,
                                          double rt, const double *x, double &f, double *g,
                                          SMat H, double *F)
{
    const bool od = odd_lane();
    const double vi = x[0], vj = x[1];
    double s, c;
    sincos(x[2] - x[3], &s, &c);
    const double vv = vi * vj;
    constexpr int S = kBranchBlock;
    // my end's p flow (al, be) and self coefficients, as in evaluate1
    const double al = od ? sY[4 * S] : sY[2 * S];                 // g_ji : g_ij
    const double be = od ? -sY[5 * S] : sY[3 * S];                // -b_ji : b_ij
    const double ap = od ? sY[6 * S] : sY[0 * S];                 // g_jj : g_ii
    const double aq = od ? -sY[7 * S] : -sY[1 * S];               // -b_jj : -b_ii
    const double T = al * c + be * s, Tp = be * c - al * s;
    const double wk2 = od ? vj * vj : vi * vi;
    const double vP = vv * Tp;
    const double Fp = ap * wk2 + vv * T;
    const double Fq = aq * wk2 + (od ? vP : -vP);
    const double hm = Fp * Fp + Fq * Fq + (od ? x[5] : x[4]);
    const double mum = (od ? lt1 : lt0) + rt * hm;
    EndSums E = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    double em0, em1, em2;
    end_terms(!od, ap, aq, vi, vj, vv, T, Tp, Fp, Fq, sT[(od ? 2 : 0) * S], sT[(od ? 3 : 1) * S],
              rpq, mum, E, em0, em1, em2);
    // swap with the partner; (from, to) in a fixed order on both lanes
    const double pG0 = partner(m, E.G0), pG1 = partner(m, E.G1), pG2 = partner(m, E.G2);
    const double pA00 = partner(m, E.A00), pA11 = partner(m, E.A11), pA01 = partner(m, E.A01);
    const double pA02 = partner(m, E.A02), pA12 = partner(m, E.A12), pA22 = partner(m, E.A22);
    const double pfq = partner(m, E.fq), ph = partner(m, hm);
    const double pe0 = partner(m, em0), pe1 = partner(m, em1), pe2 = partner(m, em2);
    const double pFp = partner(m, Fp), pFq = partner(m, Fq);
    const double G0 = E.G0 + pG0, G1 = E.G1 + pG1, G2 = E.G2 + pG2;
    const double fq = E.fq + pfq;
    const double h0 = od ? ph : hm, h1 = od ? hm : ph;
    const double mu0 = lt0 + rt * h0, mu1 = lt1 + rt * h1;
    const double e00 = od ? pe0 : em0, e01 = od ? pe1 : em1, e02 = od ? pe2 : em2;
    const double e10 = od ? em0 : pe0, e11 = od ? em1 : pe1, e12 = od ? em2 : pe2;
    F[0] = od ? pFp : Fp;
    F[1] = od ? pFq : Fq;
    F[2] = od ? Fp : pFp;
    F[3] = od ? Fq : pFq;
    const double r00 = rt * e00, r01 = rt * e01, r02 = rt * e02;
    const double r10 = rt * e10, r11 = rt * e11, r12 = rt * e12;
    const double A00 = (E.A00 + pA00) + (r00 * e00 + r10 * e10);
    const double A11 = (E.A11 + pA11) + (r01 * e01 + r11 * e11);
    const double A01 = (E.A01 + pA01) + (r00 * e01 + r10 * e11);
    const double A02 = (E.A02 + pA02) + (r00 * e02 + r10 * e12);
    const double A12 = (E.A12 + pA12) + (r01 * e02 + r11 * e12);
    const double A22 = (E.A22 + pA22) + (r02 * e02 + r12 * e12);
    const double wi = vi * vi, wj = vj * vj;
    const double rwi = wi - sT[4 * S], rti = x[2] - sT[5 * S];
    const double rwj = wj - sT[6 * S], rtj = x[3] - sT[7 * S];
    const double hrt = pow2_scale(rt, 1), trva = twice(rva);
    f = pow2_scale(rpq, 1) * fq + pow2_scale(rva, 1) * (rwi * rwi + rti * rti + rwj * rwj + rtj * rtj)
      + lt0 * h0 + hrt * h0 * h0 + lt1 * h1 + hrt * h1 * h1;
    g[0] = G0 + trva * rwi * vi;
    g[1] = G1 + trva * rwj * vj;
    g[2] = G2 + rva * rti;
    g[3] = -G2 + rva * rtj;
    g[4] = mu0;
    g[5] = mu1;
    H[P(0, 0)] = A00 + rva * (4.0 * wi + twice(rwi));
    H[P(0, 1)] = A01;
    H[P(0, 2)] = A02;
    H[P(0, 3)] = -A02;
    H[P(0, 4)] = r00;
    H[P(0, 5)] = r10;
    H[P(1, 1)] = A11 + rva * (4.0 * wj + twice(rwj));
    H[P(1, 2)] = A12;
    H[P(1, 3)] = -A12;
    H[P(1, 4)] = r01;
    H[P(1, 5)] = r11;
    H[P(2, 2)] = A22 + rva;
    H[P(2, 3)] = -A22;
    H[P(2, 4)] = r02;
    H[P(2, 5)] = r12;
    H[P(3, 3)] = A22 + rva;
    H[P(3, 4)] = -r02;
    H[P(3, 5)] = -r12;
    H[P(4, 4)] = rt;
    H[P(4, 5)] = 0.0;
    H[P(5, 5)] = rt;
}

template <int kL>
__device__ __forceinline__ void evaluate(unsigned m, const double *sY, const double *sT, double rpq,
                                         double rva, double lt0, double lt1, double rt,
                                         const double *x, double &f, double *g, SMat H, double *F)
{
    if constexpr (kL == 1) evaluate1(sY, sT, rpq, rva, lt0, lt1, rt, x, f, g, H, F);
    else evaluate2(m, sY, sT, rpq, rva, lt0, lt1, rt, x, f, g, H, F);
}

template <int kL = 1>
__device__ __forceinline__ double dot6(const double *a, const double *b, unsigned m = kFull)
{
    double s = 0.0;
    if constexpr (kL == 1) {
#pragma unroll
        for (int i = 0; i < 6; ++i) s += a[i] * b[i];
        return s;
    } else {
        const bool od = odd_lane();   // even lane: entries 0..2, odd lane: 3..5
#pragma unroll
        for (int i = 0; i < 3; ++i) s += (od ? a[3 + i] : a[i]) * (od ? b[3 + i] : b[i]);
        return s + partner(m, s);
    }
}

template <int kL = 1>
__device__ __forceinline__ void hmul(SMat H, const double *v, double *o, unsigned m = kFull)
{
    if constexpr (kL == 1) {
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            double s = 0.0;
#pragma unroll
            for (int j = 0; j < 6; ++j) s += H[P(i, j)] * v[j];
            o[i] = s;
        }
    } else {
        const bool od = odd_lane();   // even lane: rows 0..2, odd lane: rows 3..5
        double r[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            double s = 0.0;
#pragma unroll
            for (int j = 0; j < 6; ++j) s += H[od ? P(3 + i, j) : P(i, j)] * v[j];
            r[i] = s;
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double q = partner(m, r[i]);
            o[i] = od ? q : r[i];
            o[3 + i] = od ? r[i] : q;
        }
    }
}

// q(s) = g's + s'Hs/2 using the symmetry of H (two lanes: from H s by rows)
template <int kL = 1>
__device__ __forceinline__ double qmodel(const double *g, SMat H, const double *s, unsigned m = kFull)
{
    if constexpr (kL == 1) {
        double q = 0.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            double t = g[i] + 0.5 * H[P(i, i)] * s[i];
#pragma unroll
            for (int j = i + 1; j < 6; ++j) t += H[P(i, j)] * s[j];
            q += s[i] * t;
        }
        return q;
    } else {
        double hs[6];
        hmul<2>(H, s, hs, m);
        return dot6<2>(g, s, m) + 0.5 * dot6<2>(s, hs, m);
    }
}

// v'Hv / 2 (one lane: from the packed triangle, 33 operations against 42 for
// H v and a dot product; two lanes: from H v by rows)
template <int kL = 1>
__device__ __forceinline__ double half_quad(SMat H, const double *v, unsigned m = kFull)
{
    if constexpr (kL == 1) {
        double q = 0.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            double t = pow2_scale(H[P(i, i)], 1) * v[i];
#pragma unroll
            for (int j = i + 1; j < 6; ++j) t += H[P(i, j)] * v[j];
            q += v[i] * t;
        }
        return q;
    } else {
        double hv[6];
        hmul<2>(H, v, hv, m);
        return 0.5 * dot6<2>(v, hv, m);
    }
}

__device__ __forceinline__ void pstep(const Bounds &B, const double *x, const double *g, double a,
                                      double *s)
{
#pragma unroll
    for (int i = 0; i < 6; ++i) s[i] = B.clamp(i, x[i] - a * g[i]) - x[i];
}

__device__ __forceinline__ double pgnorm(const Bounds &B, const double *x, const double *g)
{
    double m = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) m = amax(m, B.clamp(i, x[i] - g[i]) - x[i]);
    return m;
}


// A Cauchy trial past a breakpoint of the projected path (rare): the projected
// step t = P(x - a g) - x and its q(t), |t|^2 and g't, kept out of line so
// that the code of the common path stays small.  Warp-collective for kL = 2.
struct V6 {
    double v[6];
};
struct Q3 {
    double q, tt, gt;
};
template <int kL>
__device__ __noinline__ Q3 cauchy_full(const Bounds B, const V6 x, const V6 g, double a, SMat H)
{
    double t[6];
    pstep(B, x.v, g.v, a, t);
    Q3 r;
    r.q = qmodel<kL>(g.v, H, t);
    r.tt = dot6<kL>(t, t);
    r.gt = dot6<kL>(g.v, t);
    return r;
}

// The loops below (Cauchy trials, Cholesky retries, CG, projected search)
// have data-dependent trip counts.  They are written warp-uniform: every lane
// of the warp runs every trip, exits are decided with __any_sync, and lanes
// that are finished (or have no TRON iteration this trip, flag `on`) keep
// their values by selection.  Lanes at different trips would otherwise be
// scheduled apart and the warp would run their FP64 work one group after
// another.  Inactive lanes compute on stale registers only (no memory access).

// Generalised Cauchy step along the projected-gradient path: from the carried
// alpha (the previous TRON iteration's, or the branch's previous TRON call's
// at the first iteration), backtrack by 0.1 while the sufficient-decrease / radius test fails, or
// extrapolate by 10 while it holds and the path still moves.  Until the path
// meets a bound, s(alpha) = -alpha g_P (g_P: g without the components pinned at
// a bound), so |s|^2, g's and q(s) follow from |g_P|^2 and g_P' H g_P computed
// once; trials past a breakpoint evaluate the projection in full.  qsc
// returns q(s) of the step chosen, from the same closed form or evaluation.
template <int kL>
__device__ __forceinline__ void cauchy(bool on, const Bounds &B, const double *x, const double *g,
                                       SMat H, double d2, double &alpha, double *s,
                                       double &qsc, Cnt &c)
{
    bool path[6];
    double room[6], gp[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const bool gp_pos = dpos(g[i]);
        path[i] = (gp_pos && B.above_lo(i, x[i])) || (dneg(g[i]) && B.below_hi(i, x[i]));
        room[i] = (gp_pos ? x[i] : B.hi(i)) - (gp_pos ? B.lo(i) : x[i]);
        gp[i] = path[i] ? g[i] : 0.0;
    }
    const double G2 = dot6<kL>(gp, gp), hGHG = half_quad<kL>(H, gp);   // |g_P|^2, g_P' H g_P / 2
    // sufficient decrease and radius test at alpha = a (uniform across the
    // warp), with q(s(a)) in q; `past`: a is past every breakpoint of the path
    auto ok_at = [&](double a, bool need, double &q, bool &past) -> bool {
        bool unc = true;
        past = true;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const double ag = a * dabsi(g[i]);
            unc = unc && (!path[i] || dle(ag, room[i]));
            past = past && (!path[i] || dle(room[i], ag));
        }
        const double gs = -a * G2, a2 = a * a;
        q = gs + a2 * hGHG;
        bool ok = dle(a2 * G2, d2) && dle(q, kMu0 * gs);
        if (__any_sync(kFull, need && !unc)) {
            // every lane forms every product (no short-circuit): with two
            // lanes per branch the products exchange values within the pair
            V6 xv, gv;
#pragma unroll
            for (int i = 0; i < 6; ++i) { xv.v[i] = x[i]; gv.v[i] = g[i]; }
            const Q3 r = cauchy_full<kL>(B, xv, gv, a, H);
            const double qf = r.q;
            const bool okf = dle(r.tt, d2) && dle(qf, kMu0 * r.gt);
            ok = unc ? ok : okf;
            q = unc ? q : qf;
        }
        return ok;
    };
    double a = alpha, qa = 0.0;
    bool pa;                           // a is past every breakpoint
    if (on) c.cauchy++;
    const bool back = !ok_at(a, on, qa, pa);
    bool go = on;
    for (int t = 0; t < kCauchyTrials; ++t) {
        // the path stops moving once a is past every breakpoint
        if (go && !back) go = !pa;
        if (!__any_sync(kFull, go)) break;
        const double an = a * (back ? 0.1 : 10.0);
        if (go) c.cauchy++;
        double qn;
        bool pn;
        const bool ok = ok_at(an, go, qn, pn);
        if (go && (back || ok)) {
            a = an;
            qa = qn;
            pa = pn;
        }
        if (ok == back) go = false;    // backtracking found a point / extrapolation failed
    }
    pstep(B, x, g, a, s);
    qsc = qa;
    if (on) alpha = a;
}

template <int kL>
__device__ __forceinline__ double boundary_tau(const double *a, const double *pv, double d2)
{
    const double pp = dot6<kL>(pv, pv), ap = dot6<kL>(a, pv), aa = dot6<kL>(a, a);
    const double rad = dmaxi(d2 - aa, 0.0);
    const double disc = sqrt(ap * ap + pp * rad);
    if (!dpos(pp)) return 0.0;
    return dpos(ap) ? rad / (ap + disc) : (disc - ap) / pp;
}

// One Cholesky pass of M + sigma I on the free block (identity on fixed
// variables), M = H (kPlain, sigma = 0) or the scaled matrix D^-1 H D^-1
// (ds = diag(D^-1)); the diagonal of the factor keeps the reciprocal pivots.
// The pass runs in registers; lanes with write == true store the factor to L.
template <bool kPlain>
__device__ __forceinline__ double scaled_entry(SMat H, const double *ds, int i, int j)
{
    return kPlain ? H[P(i, j)] : H[P(i, j)] * ds[i] * ds[j];
}

template <bool kPlain>
__device__ __forceinline__ bool chol_pass(SMat H, const double *ds, const bool *fr, double sigma,
                                          bool write, SMat L)
{
    double l[21];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        double dd = fr[j] ? (kPlain ? H[P(j, j)] : scaled_entry<false>(H, ds, j, j) + sigma) : 1.0;
#pragma unroll
        for (int k = 0; k < j; ++k) dd -= l[P(j, k)] * l[P(j, k)];
        ok = ok && dpos(dd);
        const double linv = rsqrt(dmaxi(dd, 1e-300));
        l[P(j, j)] = linv;
#pragma unroll
        for (int i = j + 1; i < 6; ++i) {
            double v = (fr[i] && fr[j]) ? scaled_entry<kPlain>(H, ds, i, j) : 0.0;
#pragma unroll
            for (int k = 0; k < j; ++k) v -= l[P(i, k)] * l[P(j, k)];
            l[P(i, j)] = v * linv;
        }
    }
    if (write) {
#pragma unroll
        for (int k = 0; k < 21; ++k) L[k] = l[k];
    }
    return ok;
}

// k-th shift of the schedule sigma_0 = (pos ? 0 : 1e-3),
// sigma_{t+1} = max(2 sigma_t, 1e-3): 1e-3 * 2^(k - pos), or 0 at k = 0 when
// pos.  Doubling is exact, so adding to the exponent gives the doubled value
// bit for bit.
__device__ __forceinline__ double shift_at(int k, bool pos)
{
    const int e = pos ? k - 1 : k;
    return e < 0 ? 0.0 : __longlong_as_double(__double_as_longlong(1e-3) + ((long long)e << 52));
}

// Preconditioner: Cholesky factor of D^-1 A D^-1 + sigma I on the free block,
// D = diag(sqrt|A_ii|), sigma the first shift of the schedule above (at most
// kCholTries of them) for which the factorisation succeeds.  A positive
// definite block is first factored unscaled: then D L L' D = L0 L0' exactly,
// so the preconditioned CG iterates are the same.  The first successful shift
// is found by bisection over the schedule's indices (about 5 factorisations
// instead of up to 20 in sequence): A + sigma I stays positive definite as
// sigma grows, so success is monotone in the index and bisection finds the
// same shift as trying the shifts in order.  Dv receives the diagonal of D^-1
// (lanes with a scaled factor only).  The scaled path is rare and kept out of
// line, so that the code of the common path stays small.
__device__ __noinline__ void precond_scaled(bool need, SMat H, unsigned frm, SMat L, SMat Dv)
{
    bool fr[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) fr[i] = (frm >> i) & 1u;
    bool pos = true;
    double ds[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const double a = H[P(i, i)];
        ds[i] = (fr[i] && okey(a) != 0) ? rsqrt(dabsi(a)) : 1.0;
        pos = pos && (!fr[i] || dpos(a));
    }
#pragma unroll
    for (int i = 0; i < 6; ++i)
        if (need) Dv[i] = ds[i];
    // first success in [lo, hi]; hi == kCholTries: none found yet.  `held`:
    // L holds the factor at hi (the lane's last pass succeeded)
    int lo = 0, hi = kCholTries;
    bool srch = need, held = false;
    for (int t = 0; t < 8; ++t) {
        if (!__any_sync(kFull, srch)) break;
        const int mid = (lo + hi) >> 1;
        const bool ok = chol_pass<false>(H, ds, fr, shift_at(mid, pos), srch, L);
        if (srch) {
            hi = ok ? mid : hi;
            lo = ok ? lo : mid + 1;
            held = ok;
        }
        srch = srch && lo < hi;
    }
    const bool redo = need && hi < kCholTries && !held;
    if (__any_sync(kFull, redo)) chol_pass<false>(H, ds, fr, shift_at(hi, pos), redo, L);
    if (__any_sync(kFull, need && hi >= kCholTries)) {   // give up: identity in the scaled space
#pragma unroll
        for (int i = 0; i < 6; ++i) {
#pragma unroll
            for (int j = 0; j <= i; ++j)
                if (need && hi >= kCholTries) L[P(i, j)] = (i == j) ? 1.0 : 0.0;
        }
    }
}

// Returns whether the lane's factor is the scaled one (warp-collective).
__device__ __forceinline__ bool precond_factor(bool on, SMat H, const bool *fr, SMat L, SMat Dv)
{
    const bool plain = chol_pass<true>(H, nullptr, fr, 0.0, true, L);
    const bool need = on && !plain;
    if (!__any_sync(kFull, need)) return false;
    unsigned frm = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) frm |= fr[i] ? 1u << i : 0u;
    precond_scaled(need, H, frm, L, Dv);
    return need;
}

// z = M^-1 r, M = D L L' D (D = I unless `scaled`); anys: some lane of the
// warp has a scaled factor (multiplying by 1 leaves the others' values as
// they are)
__device__ __forceinline__ void precond_solve(SMat L, SMat Dv, bool scaled, bool anys, const double *r,
                                              double *z)
{
    double t[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double v = anys ? r[i] * (scaled ? Dv[i] : 1.0) : r[i];
#pragma unroll
        for (int k = 0; k < i; ++k) v -= L[P(i, k)] * t[k];
        t[i] = v * L[P(i, i)];
    }
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        double v = t[i];
#pragma unroll
        for (int k = i + 1; k < 6; ++k) v -= L[P(k, i)] * t[k];
        t[i] = v * L[P(i, i)];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) z[i] = anys ? t[i] * (scaled ? Dv[i] : 1.0) : t[i];
}

// Subspace step: Steihaug PCG on the free variables of the Cauchy point, then
// a projected backtracking search along the CG direction.
template <int kL>
__device__ __forceinline__ void subspace(bool on, const Bounds &B, const double *x, const double *g,
                                         SMat H, SMat L, SMat S, double d2, const double *sc, double qc,
                                         double *s, double &qs, Cnt &c)
{
    qs = qc;                 // q(s) for the step returned: the Cauchy point's, or
                             // the accepted search point's below
    bool fr[6];
    double xc[6];
    bool any = false;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        xc[i] = x[i] + sc[i];
        fr[i] = B.above_lo(i, xc[i]) && B.below_hi(i, xc[i]);
        any = any || fr[i];
        s[i] = sc[i];
    }
    const bool act = on && any;
    if (!__any_sync(kFull, act)) return;
    double gc[6];
    hmul<kL>(H, sc, gc);
#pragma unroll
    for (int i = 0; i < 6; ++i) gc[i] += g[i];
    const SMat Dv = S;                     // the scratch holds D^-1 until CG ends
    const bool scaled = precond_factor(act, H, fr, L, Dv);
    const bool anys = __any_sync(kFull, scaled);
    // hwb: H times the boundary step tau p, which CG adds to w without
    // updating r; elsewhere H w = r0 - r on the free variables (r0 = -gc)
    double w[6], r[6], z[6], pv[6], q[6], hwb[6];
    double rn0 = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        w[i] = 0.0;
        hwb[i] = 0.0;
        r[i] = fr[i] ? -gc[i] : 0.0;
        rn0 += r[i] * r[i];
    }
    const bool cgon = act && dpos(rn0);
    if (!__any_sync(kFull, cgon)) return;
    precond_solve(L, Dv, scaled, anys, r, z);
    double rz = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        pv[i] = fr[i] ? z[i] : 0.0;
        rz += r[i] * pv[i];
    }
    const double tol2 = kCgRtol * kCgRtol * rn0;
    bool go = cgon;
    for (int it = 0; it < kCgMaxit; ++it) {
        if (!__any_sync(kFull, go)) break;
        if (go) c.cg++;
        hmul<kL>(H, pv, q);
        double kappa = 0.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            q[i] = fr[i] ? q[i] : 0.0;
            kappa += pv[i] * q[i];
        }
        double cur[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) cur[i] = sc[i] + w[i];
        const double al = rz / kappa;
        double nx2 = 0.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const double v = cur[i] + al * pv[i];
            nx2 += v * v;
        }
        // negative curvature or the trust-region boundary: stop on the boundary
        const bool bnd = go && (!dpos(kappa) || dle(d2, nx2));
        if (__any_sync(kFull, bnd)) {
            const double tau = boundary_tau<kL>(cur, pv, d2);
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                w[i] = bnd ? w[i] + tau * pv[i] : w[i];
                hwb[i] = bnd ? tau * q[i] : hwb[i];
            }
        }
        go = go && !bnd;
        double rn = 0.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            w[i] = go ? w[i] + al * pv[i] : w[i];
            r[i] = go ? r[i] - al * q[i] : r[i];
            rn += r[i] * r[i];
        }
        go = go && !dle(rn, tol2);
        if (!__any_sync(kFull, go)) break;
        precond_solve(L, Dv, scaled, anys, r, z);
        double rz1 = 0.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            z[i] = fr[i] ? z[i] : 0.0;
            rz1 += r[i] * z[i];
        }
        const double be = rz1 / rz;
        rz = go ? rz1 : rz;
#pragma unroll
        for (int i = 0; i < 6; ++i) pv[i] = go ? z[i] + be * pv[i] : pv[i];
    }
    // Projected search along w from the Cauchy point.  While xc + beta w
    // stays inside the bounds (beta below every free variable's
    // breakpoint), q(sc + beta w) = q(sc) + beta gc'w + beta^2/2 w'Hw in
    // closed form, with H w from the CG recurrences.  Past a breakpoint the
    // projected step is sc + beta w + e, e_i = bound_i - (xc_i + beta w_i) on
    // the variables past theirs, and q = q(sc + beta w) + gc'e + beta (Hw)'e
    // + e'He/2, formed over those variables only.  The scratch S (free once
    // CG is done) keeps H w in S[0..5] and e in S[6..11].
    double gw = 0.0, whw = 0.0, room[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const double hw = fr[i] ? (-gc[i] - r[i]) + hwb[i] : 0.0;
        S[i] = hw;
        gw += gc[i] * w[i];
        whw += w[i] * hw;
        room[i] = dpos(w[i]) ? B.hi(i) - xc[i] : xc[i] - B.lo(i);
    }
    double beta = 1.0;
    bool ps = cgon;
    for (int t = 0; t < kPsTrials; ++t) {
        if (!__any_sync(kFull, ps)) break;
        if (ps) c.ps++;
        // beta = 2^-t: beta |w_i|, beta gw and beta^2 whw / 2 are exact
        // exponent shifts, done on the integer pipe
        bool unc = true;
#pragma unroll
        for (int i = 0; i < 6; ++i) unc = unc && (!fr[i] || dle(pow2_scale(dabsi(w[i]), t), room[i]));
        const double bgw = pow2_scale(gw, t);
        double qb = (qc + bgw) + pow2_scale(whw, 2 * t + 1);
        bool okp = ps && dle(qb, qc + kMu0 * bgw);
        if (__any_sync(kFull, ps && !unc)) {
            double ge = 0.0, he = 0.0, ehe = 0.0;
#pragma unroll
            for (int i = 0; i < 6; ++i) S[6 + i] = 0.0;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                const double bwi = pow2_scale(dabsi(w[i]), t);
                const bool cl = fr[i] && !dle(bwi, room[i]);
                if (__any_sync(kFull, cl)) {
                    const double ei = cl ? (dpos(w[i]) ? room[i] - bwi : bwi - room[i]) : 0.0;
                    ge += gc[i] * ei;
                    he += S[i] * ei;
                    double th = 0.5 * H[P(i, i)] * ei;
#pragma unroll
                    for (int j = 0; j < i; ++j) th += H[P(i, j)] * S[6 + j];
                    ehe += ei * th;
                    S[6 + i] = ei;
                }
            }
            const double qf = qb + (ge + pow2_scale(he, t)) + ehe;
            const bool okf = ps && dle(qf, qc + kMu0 * (bgw + ge));
            qb = unc ? qb : qf;
            okp = unc ? okp : okf;
        }
        if (__any_sync(kFull, okp)) {
#pragma unroll
            for (int i = 0; i < 6; ++i) s[i] = okp ? B.clamp(i, xc[i] + beta * w[i]) - x[i] : s[i];
        }
        qs = okp ? qb : qs;
        ps = ps && !okp;
        beta = pow2_scale(beta, 1);                 // 2^-(t+1), exact
    }
}

__device__ __forceinline__ void warp_add_u64(unsigned long long *dst, int v)
{
    const unsigned int s = __reduce_add_sync(kFull, (unsigned int)v);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(dst, (unsigned long long)s);
}

// Scheduling class of a branch that took `trips` loop trips (0 = hardest).
__device__ __forceinline__ int trip_class(int trips)
{
    return trips >= 64 ? 0 : trips >= 48 ? 1 : trips >= 32 ? 2 : trips >= 24 ? 3
         : trips >= 16 ? 4 : trips >= 8 ? 5 : trips >= 4 ? 6 : 7;
}

// File the branches some lanes finished (filed >= 0) into the class lists of
// the next iteration (warp-collective; one atomic per class and warp).
__device__ __forceinline__ void file_branches(Ctrl *ctrl, int32_t *lnxt, int nl, int nxt, int lane,
                                              int filed, int fcls)
{
    if (!__any_sync(kFull, filed >= 0)) return;
#pragma unroll
    for (int cl = 0; cl < kClasses; ++cl) {
        const unsigned m = __ballot_sync(kFull, filed >= 0 && fcls == cl);
        if (m) {
            const int leader = __ffs(m) - 1;
            unsigned base = 0;
            if (lane == leader) base = atomicAdd(&ctrl->cls_count[nxt][cl], (unsigned)__popc(m));
            base = __shfl_sync(kFull, base, leader);
            if (filed >= 0 && fcls == cl)
                lnxt[(size_t)cl * nl + base + __popc(m & ((1u << lane) - 1u))] = filed;
        }
    }
}

// LS_REEVAL_DONE: the solve stopped right after a rejected step; the flows the
// AL update needs are re-evaluated at the kept point first
enum LaneState { LS_IDLE = 0, LS_INIT = 1, LS_ITER = 2, LS_REEVAL = 3, LS_DONE = 4, LS_REEVAL_DONE = 5 };

}  // namespace

// The kernel body, for kL = 1 or 2 lanes per branch.
template <int kL>
__device__ __forceinline__ void branch_tron_body(DevGrid G, DevOpts O)
{
    // dynamic shared memory: Y[8], t[8] per lane with stride kBranchBlock,
    // then the packed Hessian, the preconditioner's factor and a scratch of 12
    // in pairs (SMat)
    extern __shared__ double sh[];
    __shared__ unsigned cstart[kClasses + 1];  // queue positions where the classes start
    const SMat H{sh + 16 * kBranchBlock + 2 * threadIdx.x};
    const SMat Lf{sh + 38 * kBranchBlock + 2 * threadIdx.x};
    const SMat Sc{sh + 60 * kBranchBlock + 2 * threadIdx.x};
    Ctrl *ctrl = G.ctrl;
    if (ctrl->done) return;                    // uniform across the grid
    const int nl = G.nl;
    const int lane = threadIdx.x & 31;
    const double *sY = sh + threadIdx.x;
    const double *sT = sh + 8 * kBranchBlock + threadIdx.x;
    double rpq = 1.0, rva = 1.0, rt0 = 1.0;   // penalties of the lane's branch's scenario
    Cnt c = {0, 0, 0, 0, 0, 0, 0, 0, 0};

    // queue order: the classes filed by the previous iteration, hardest first
    const int cur = ctrl->total_iters & 1, nxt = cur ^ 1;
    if (threadIdx.x == 0) {
        unsigned acc = 0;
        cstart[0] = 0;
        for (int k = 0; k < kClasses; ++k) cstart[k + 1] = (acc += ctrl->cls_count[cur][k]);
    }
    __syncthreads();
    const bool ordered = cstart[kClasses] == (unsigned)nl;
    // branch slots: one per lane, or one per lane pair (the even lane, `lead`,
    // takes part in the queue, files, writes and counts); the first `slots`
    // positions of the queue are dealt across all warps
    const bool lead = kL == 1 || !odd_lane();
    const unsigned slots = gridDim.x * blockDim.x / kL;
    const unsigned spw = 32 / kL;                    // slots per warp
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    const bool bsync = gridDim.x >= 2u * (unsigned)O.num_sms;   // uniform across the grid
    const int32_t *lcur = G.cls_list + (size_t)cur * kClasses * nl;
    int32_t *lnxt = G.cls_list + (size_t)nxt * kClasses * nl;

    int b = -1, state = LS_IDLE, apass = 0, k = 0, trips = 0;
    bool exhausted = false;
    Bounds B{1.0, 1.0, 1.0, 1.0, 0.0, 0, 0, 0, 0, 0};
    double x[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, xt[6], g[6], F[4] = {0.0, 0.0, 0.0, 0.0};
    // the trust radius is kept squared (dsq): its tests and updates need only
    // squares, which saves a square root per step
    double f = 0.0, dsq = 0.0, alpha = 1.0, gtol = 0.0, prered = 0.0, snorm2 = 0.0;
    double lt0 = 0.0, lt1 = 0.0, rt = rt0, hprev = 0.0;

    while (true) {
        bool eval = false;
        // (T) one TRON iteration up to its trial point, or the stop of the solve
        bool go_t = false;
        if (state == LS_ITER) {
            if (k >= O.tron_max_iter) {
                c.maxhit++;
                state = LS_DONE;
            } else if (dle(pgnorm(B, x, g), gtol)) {
                state = LS_DONE;
            } else {
                c.tron_iters++;
                go_t = true;
            }
        }
        if (__any_sync(kFull, go_t)) {
            double sc[6], s[6];
            double qs = 0.0, qsc = 0.0;
            cauchy<kL>(go_t, B, x, g, H, dsq, alpha, sc, qsc, c);
            subspace<kL>(go_t, B, x, g, H, Lf, Sc, dsq, sc, qsc, s, qs, c);
            const double s2 = dot6<kL>(s, s);
            if (go_t) {
                double xn = 0.0, sn = 0.0;
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    xn = amax(xn, x[i]);
                    sn = amax(sn, s[i]);
                }
                if (dle(sn, O.tron_xtol * dmaxi(xn, 1.0))) {
                    state = LS_DONE;
                } else {
                    prered = -qs;
                    c.f++;
                    if (!dpos(prered)) {
                        state = LS_DONE;          // no decrease predicted: stalled
                    } else {
#pragma unroll
                        for (int i = 0; i < 6; ++i) xt[i] = B.clamp(i, x[i] + s[i]);
                        snorm2 = s2;
                        eval = true;
                    }
                }
            }
        }
        // (A) a finished TRON solve: line-limit multiplier update (Section II-C);
        // the next pass starts in this same trip
        int filed = -1, fcls = 0;
        if (state == LS_DONE) {
            const double h0 = F[0] * F[0] + F[1] * F[1] + x[4];
            const double h1 = F[2] * F[2] + F[3] * F[3] + x[5];
            lt0 += rt * h0;
            lt1 += rt * h1;
            const double hm = amax(dabsi(h0), h1);
            bool fin = dle(hm, O.al_tol);
            if (!fin) {
                if (dlt(O.al_decay * hprev, hm)) rt = dmini(rt * O.al_rho_factor, O.al_rho_max);
                hprev = hm;
                fin = apass >= O.al_max_iter;
            }
            if (fin) {
                if (lead) {
#pragma unroll
                    for (int i = 0; i < 6; ++i) G.bx[i * nl + b] = x[i];
                    G.blt[b] = lt0;
                    G.blt[nl + b] = lt1;
                    G.balpha[b] = alpha;
#pragma unroll
                    for (int i = 0; i < 4; ++i) G.bu[i * nl + b] = F[i];
                    G.bu[4 * nl + b] = x[0] * x[0];
                    G.bu[5 * nl + b] = x[2];
                    G.bu[6 * nl + b] = x[1] * x[1];
                    G.bu[7 * nl + b] = x[3];
                    filed = b;
                }
                fcls = trip_class(trips);
                b = -1;
                state = LS_IDLE;
            } else {
                state = LS_INIT;
            }
        }
        // (F) file finished branches by the work they took
        file_branches(ctrl, lnxt, nl, nxt, lane, filed, fcls);
        // (R) refill idle lanes from the branch queue (one atomic per warp);
        // branches of scenarios that are not iterating are filed and skipped
        for (int rep = 0; rep < 64; ++rep) {
            const unsigned need = __ballot_sync(kFull, lead && state == LS_IDLE && !exhausted);
            if (!need) break;
            const int leader = __ffs(need) - 1;
            unsigned base = 0;
            if (lane == leader) base = atomicAdd(&ctrl->branch_next, (unsigned)__popc(need));
            base = __shfl_sync(kFull, base, leader);
            unsigned idx = base + __popc(need & ((1u << lane) - 1u));
            if constexpr (kL == 2) idx = __shfl_sync(kFull, idx, lane & ~1);   // the pair's slot
            int skip = -1;
            if (state == LS_IDLE && !exhausted) {
                // the first fill hands each warp 32 consecutive positions:
                // deal the ranks across the warps instead (rank = lane-in-fill
                // x warps + warp), so that the hardest branches spread over all
                // warps rather than filling the first ones, and a grid with
                // fewer branches than lanes occupies every warp.  Positions
                // whose rank is past the end hold no branch; every position
                // below `lanes` is still drawn, since each lane draws at least
                // once and draws take consecutive positions.
                const unsigned r = idx < slots ? (idx % spw) * nwarps + idx / spw : idx;
                if (r < (unsigned)nl) {
                    int bb = (int)r;
                    if (ordered) {
                        int cl = 0;
                        for (int q = 1; q < kClasses; ++q) cl = r >= cstart[q] ? q : cl;
                        bb = lcur[(size_t)cl * nl + (r - cstart[cl])];
                    }
                    const SCtrl *sc = G.sc + G.br_scen[bb];
                    if (!sc->active || sc->done) {
                        skip = bb;
                    } else {
                        b = bb;
                        rpq = sc->rho_pq;
                        rva = sc->rho_va;
                        trips = 0;
                        double *my = sh + threadIdx.x;
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            my[i * kBranchBlock] = G.Y[i * nl + b];
                            my[(8 + i) * kBranchBlock] = G.bt[i * nl + b];
                        }
                        B.vlo_i = G.lim[0 * nl + b];
                        B.vhi_i = G.lim[1 * nl + b];
                        B.vlo_j = G.lim[2 * nl + b];
                        B.vhi_j = G.lim[3 * nl + b];
                        B.slo = G.lim[4 * nl + b];
                        B.set_keys();
                        // rho-tilde starts at 25 rho_pq / rbar^2: 100 times the
                        // penalty on h = p^2 + q^2 + s that weighs a flow deviation
                        // at the limit like the coupling penalty does (rho_pq
                        // without a limit)
                        {
                            const double rb2 = -B.slo;
                            const double r = 25.0 * rpq / rb2;
                            rt0 = O.al_rho0 > 0.0 ? O.al_rho0
                                : (rb2 < 1e19 ? (r < O.al_rho_max ? r : O.al_rho_max) : rpq);
                        }
#pragma unroll
                        for (int i = 0; i < 6; ++i) x[i] = G.bx[i * nl + b];
                        lt0 = G.blt[b];
                        lt1 = G.blt[nl + b];
                        alpha = G.balpha[b];
                        rt = rt0;
                        hprev = __longlong_as_double(0x7ff0000000000000LL);
                        apass = 0;
                        state = LS_INIT;
                    }
                } else {
                    exhausted = true;
                }
            }
            file_branches(ctrl, lnxt, nl, nxt, lane, lead ? skip : -1, kClasses - 1);
        }
        // done when every lane is idle and the queue is drained.  With two or
        // more blocks per SM the block's warps also meet here every trip: the
        // four warps of a block then run the same part of the code at the
        // same time (fewer instruction-fetch stalls; measured 9 % faster on the
        // 70,000-bus grid), while the SM's other block fills the waits.  With
        // one block per SM the barrier would only add waiting.
        if (bsync) {
            if (!__syncthreads_or(state != LS_IDLE || !exhausted)) break;
        } else if (!__any_sync(kFull, state != LS_IDLE || !exhausted)) {
            break;
        }
        // (I) a TRON solve starts from the current point; a rejected step gets
        // its gradient and Hessian back at the kept point
        if (state == LS_INIT) {
            apass++;
            c.al++;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                x[i] = B.clamp(i, x[i]);
                xt[i] = x[i];
            }
            eval = true;
        } else if (state == LS_REEVAL || state == LS_REEVAL_DONE) {
#pragma unroll
            for (int i = 0; i < 6; ++i) xt[i] = x[i];
            eval = true;
        }
        // (E) the one evaluation site of the trip
        double fe = 0.0;
        const unsigned em = __ballot_sync(kFull, eval);
        if (eval) evaluate<kL>(em, sY, sT, rpq, rva, lt0, lt1, rt, xt, fe, g, H, F);
        if (b >= 0) ++trips;
        // (Q) after the evaluation
        const unsigned im = __ballot_sync(kFull, state == LS_INIT);
        if (state == LS_INIT) {
            f = fe;
            c.tron_calls++;
            c.fgh++;
            // the projected-gradient step P(x - g) - x gives both the stopping
            // threshold (its max norm) and the first trust radius (its 2-norm)
            double sp[6], pg0 = 0.0;
            pstep(B, x, g, 1.0, sp);
#pragma unroll
            for (int i = 0; i < 6; ++i) pg0 = amax(pg0, sp[i]);
            gtol = O.tron_gtol * dmaxi(pg0, 1.0);
            dsq = dot6<kL>(sp, sp, im);
            alpha = dpos(alpha) ? alpha : 1.0;   // carried from the previous call
            k = 0;
            state = LS_ITER;
        } else if (state == LS_REEVAL) {
            state = LS_ITER;
        } else if (state == LS_REEVAL_DONE) {
            state = LS_DONE;
        } else if (state == LS_ITER && eval) {
            const double actred = f - fe;
            if (k == 0 && dlt(snorm2, dsq)) dsq = snorm2;
            const double fa = dmaxi(dabsi(f), 1.0);
            // ratio = actred / prered (1 when the model is trusted) against
            // eta0, eta1, eta2, compared as actred against eta prered (prered > 0).
            // The model is trusted when prered is below tron_ftol max(1, |f|),
            // f in its completed-square form sum rho/2 (u - t)^2 + AL terms:
            // the rounding level of f - ft, whichever way the constant of
            // eq. branch is written
            const bool trusted = dle(prered, O.tron_ftol * fa);
            static_assert(kEta1 == 0.25, "eta1 scaling is an exponent step");
            const bool below1 = !trusted && dlt(actred, pow2_scale(prered, 2));
            const bool above2 = trusted || dlt(kEta2 * prered, actred);
            const bool above0 = trusted || dlt(kEta0 * prered, actred);
            // sigma1^2 = 2^-4 and sigma3^2 = 2^4: exponent steps
            static_assert(kSigma1 * kSigma1 == 0.0625 && kSigma3 * kSigma3 == 16.0, "radius factors");
            if (below1) dsq = pow2_scale(dmini(snorm2, dsq), 4);
            else if (above2) dsq = dmaxi(dsq, pow2_up(snorm2, 4));
            if (above0) {
#pragma unroll
                for (int i = 0; i < 6; ++i) x[i] = xt[i];
                f = fe;
                c.fgh++;
            } else {
                state = LS_REEVAL;
            }
            double xn = 0.0;
#pragma unroll
            for (int i = 0; i < 6; ++i) xn = amax(xn, x[i]);
            const double xm = dmaxi(xn, 1.0);
            if (dle(dsq, 1e-28 * xm * xm))
                state = state == LS_REEVAL ? LS_REEVAL_DONE : LS_DONE;
            ++k;
        }
    }
    // counters: once per branch (the lead lane of a pair)
    unsigned long long *st = ctrl->stats;
    const int on = lead ? 1 : 0;
    warp_add_u64(&st[ST_TRON_CALLS], on * c.tron_calls);
    warp_add_u64(&st[ST_TRON_ITERS], on * c.tron_iters);
    warp_add_u64(&st[ST_FGH], on * c.fgh);
    warp_add_u64(&st[ST_F], on * c.f);
    warp_add_u64(&st[ST_CAUCHY], on * c.cauchy);
    warp_add_u64(&st[ST_CG], on * c.cg);
    warp_add_u64(&st[ST_PS], on * c.ps);
    warp_add_u64(&st[ST_AL], on * c.al);
    warp_add_u64(&st[ST_TRON_MAXHIT], on * c.maxhit);
}

__global__ void __launch_bounds__(kBranchBlock, kBranchBlocksPerSM)
branch_tron_kernel(DevGrid G, DevOpts O)
{
    branch_tron_body<1>(G, O);
}

// two lanes per branch (a lane pair shares each branch's work, see evaluate2)
__global__ void __launch_bounds__(kBranchBlock, kBranchBlocksPerSM)
branch_tron2_kernel(DevGrid G, DevOpts O)
{
    branch_tron_body<2>(G, O);
}

}  // namespace admm
