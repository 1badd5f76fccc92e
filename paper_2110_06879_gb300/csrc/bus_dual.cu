// bus_dual: the generator x-update, the bus xbar-update, the z-update and the y-update of Algorithm 1
// fused into one pass over the bus -> incident-component CSR map, plus the
// residual reduction and the loop control of the two-level algorithm.
//
// A block owns a run of consecutive buses (at most kBusPerBlock, at most
// kSlotCap incidence slots, split on the host) and works in three phases:
// (A) one thread per slot -- generator updates (eq. qp-bound, the generator's
// own slot) and every coupling's target u + z + y/rho; (B) one thread per bus
// -- the row's sums in CSR order from shared memory and the bus closed form;
// (C) one thread per slot -- bus copies, z, y, residual sums.  Every coupling
// is owned by exactly one bus (the bus its copy lives on), so the gather needs
// no atomics and sums in a fixed order (deterministic), and the per-slot
// phases keep the lanes busy whatever the row lengths.  The outer multiplier update
// lambda <- Proj(lambda + beta z) is applied lazily: lambda is read only by the
// z update, so the bus row applies a pending outer update to its slots just
// before it updates z.  Bus blocks never straddle scenarios (each scenario's
// buses start on a block boundary), so every block writes its partial sums for
// exactly one scenario; the scenario's last block to finish (atomic ticket)
// sums them in block order, evaluates that scenario's stopping tests and outer
// step.  A scenario's result is therefore the same whether it is solved alone
// or batched with others.  control_kernel ends each iteration: it sets the
// CUDA-graph conditional while any scenario is still running.
#include "admm_internal.cuh"

namespace admm {
namespace {

__device__ __forceinline__ double clampd(double v, double lo, double hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

// block-wide sum of 4 values, result valid in thread 0
template <int kBlock, int kN>
__device__ __forceinline__ void block_sum(double (&v)[kN], double (*sh)[kN])
{
#pragma unroll
    for (int k = 0; k < kN; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kN; ++k) sh[w][k] = v[k];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < kN; ++k) v[k] = lane < kBlock / 32 ? sh[lane][k] : 0.0;
#pragma unroll
        for (int k = 0; k < kN; ++k) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        }
    }
}


__device__ __forceinline__ void flows_at(const double *Y, int nl, int l, double vi, double vj,
                                         double th, double out[4])
{
    double s, c;
    sincos(th, &s, &c);
    double gii = Y[0 * nl + l], bii = Y[1 * nl + l], gij = Y[2 * nl + l], bij = Y[3 * nl + l];
    double gji = Y[4 * nl + l], bji = Y[5 * nl + l], gjj = Y[6 * nl + l], bjj = Y[7 * nl + l];
    double vv = vi * vj;
    out[0] = gii * vi * vi + vv * (gij * c + bij * s);
    out[1] = -bii * vi * vi + vv * (-bij * c + gij * s);
    out[2] = gjj * vj * vj + vv * (gji * c - bji * s);
    out[3] = -bjj * vj * vj + vv * (-bji * c - gji * s);
}

}  // namespace

// pi-model entries of Section II-A from (r, x, b, tap, shift), and the bounds of
// every branch subproblem.
__global__ void admittance_kernel(DevGrid G)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    const int nl = G.nl;
    if (l >= nl) return;
    double r = G.raw[0 * nl + l], x = G.raw[1 * nl + l], b = G.raw[2 * nl + l];
    double tap = G.raw[3 * nl + l], sh = G.raw[4 * nl + l], rate = G.raw[5 * nl + l];
    if (tap == 0.0) tap = 1.0;
    double den = r * r + x * x;
    double ys_r = r / den, ys_i = -x / den;          // 1 / (r + jx)
    double ar = tap * cos(sh), ai = tap * sin(sh);   // a = tap e^{j shift}
    double a2 = ar * ar + ai * ai;
    // y_ii = (ys + j b/2) / |a|^2
    G.Y[0 * nl + l] = ys_r / a2;
    G.Y[1 * nl + l] = (ys_i + 0.5 * b) / a2;
    // y_ij = -ys / conj(a) = -ys a / |a|^2
    G.Y[2 * nl + l] = -(ys_r * ar - ys_i * ai) / a2;
    G.Y[3 * nl + l] = -(ys_r * ai + ys_i * ar) / a2;
    // y_ji = -ys / a = -ys conj(a) / |a|^2
    G.Y[4 * nl + l] = -(ys_r * ar + ys_i * ai) / a2;
    G.Y[5 * nl + l] = -(ys_i * ar - ys_r * ai) / a2;
    // y_jj = ys + j b/2
    G.Y[6 * nl + l] = ys_r;
    G.Y[7 * nl + l] = ys_i + 0.5 * b;
    int i = G.f_bus[l], j = G.t_bus[l];
    G.lim[0 * nl + l] = G.bus[4 * G.nb + i];
    G.lim[1 * nl + l] = G.bus[5 * G.nb + i];
    G.lim[2 * nl + l] = G.bus[4 * G.nb + j];
    G.lim[3 * nl + l] = G.bus[5 * G.nb + j];
    double rb = G.line_limit_frac * rate;
    G.lim[4 * nl + l] = rate > 0.0 ? -rb * rb : -1e20;
}

// Section IV-B initialisation (cold start) of one scenario.  Thread roles:
// its branches, its incidence slots, its buses, its generators, and one more
// thread for the scenario's outer state.
__global__ void cold_start_kernel(DevGrid G, Range R, double beta_init)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int nl = G.nl, nb = G.nb, ng = G.ng, ns = G.ns;
    const double *vmin = G.bus + 4 * nb, *vmax = G.bus + 5 * nb;
    const int nbr = R.b1 - R.b0, nsl = R.k1 - R.k0, nbu = R.i1 - R.i0, nge = R.g1 - R.g0;
    if (t < nbr) {
        const int l = R.b0 + t, i = G.f_bus[l], j = G.t_bus[l];
        double vi = 0.5 * (vmin[i] + vmax[i]), vj = 0.5 * (vmin[j] + vmax[j]);
        double fl[4];
        flows_at(G.Y, nl, l, vi, vj, 0.0, fl);
        double slo = G.lim[4 * nl + l];
        double x[6] = {vi, vj, 0.0, 0.0, clampd(-(fl[0] * fl[0] + fl[1] * fl[1]), slo, 0.0),
                       clampd(-(fl[2] * fl[2] + fl[3] * fl[3]), slo, 0.0)};
        for (int k = 0; k < 6; ++k) G.bx[k * nl + l] = x[k];
        G.blt[l] = 0.0;
        G.blt[nl + l] = 0.0;
        G.balpha[l] = 1.0;
        double u[8] = {fl[0], fl[1], fl[2], fl[3], vi * vi, 0.0, vj * vj, 0.0};
        for (int k = 0; k < 8; ++k) {
            G.bu[k * nl + l] = u[k];
            G.bt[k * nl + l] = u[k];        // xbar = u, z = y = 0
        }
        return;
    }
    int q = t - nbr;
    if (q < nsl) {
        const int k = R.k0 + q;
        const int e = G.col[k];
        double cp, cq;
        if (e < 2 * nl) {
            int l = e >> 1, end = e & 1, i = G.f_bus[l], j = G.t_bus[l];
            double vi = 0.5 * (vmin[i] + vmax[i]), vj = 0.5 * (vmin[j] + vmax[j]);
            double fl[4];
            flows_at(G.Y, nl, l, vi, vj, 0.0, fl);
            cp = end ? fl[2] : fl[0];
            cq = end ? fl[3] : fl[1];
        } else {
            int g = e - 2 * nl;
            cp = 0.5 * (G.glim[0 * ng + g] + G.glim[1 * ng + g]);
            cq = 0.5 * (G.glim[2 * ng + g] + G.glim[3 * ng + g]);
        }
        G.sx[k] = cp;
        G.sx[ns + k] = cq;
        for (int c = 0; c < 4; ++c) {
            G.sz[c * ns + k] = 0.0;
            G.sy[c * ns + k] = 0.0;
            G.sl[c * ns + k] = 0.0;
        }
        return;
    }
    q -= nsl;
    if (q < nbu) {
        const int i = R.i0 + q;
        double v = 0.5 * (vmin[i] + vmax[i]);
        G.bw[i] = v * v;
        G.bth[i] = 0.0;
        return;
    }
    q -= nbu;
    if (q < nge) {
        const int g = R.g0 + q;
        G.gu[g] = 0.5 * (G.glim[0 * ng + g] + G.glim[1 * ng + g]);
        G.gu[ng + g] = 0.5 * (G.glim[2 * ng + g] + G.glim[3 * ng + g]);
        return;
    }
    if (q == nge) {   // the scenario's outer state
        SCtrl *c = G.sc + R.s;
        c->beta = beta_init;
        c->pending = 0;
        c->total_iters = 0;
    }
}

// Start (or restart) the loops of scenarios [s0, s1): Algorithm 1 restarts its
// counters; the primal, dual and penalty values stay (warm start).
__global__ void slot_begin_kernel(DevGrid G, DevOpts O, int32_t s0, int32_t s1, SolveParams P)
{
    const int s = s0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= s1) return;
    SCtrl *c = G.sc + s;
    c->tol = P.tol;
    c->rho_pq = P.rho_pq;
    c->rho_va = P.rho_va;
    c->max_iter = P.max_iter;
    c->iter = 0;
    c->inner = 0;
    c->outer = 0;
    c->status = CS_RUNNING;
    c->done = P.max_iter <= 0 ? 1 : 0;
    c->active = 1;
    c->zprev = __longlong_as_double(0x7ff0000000000000LL);
    c->tol_in = fmax(O.tol_in0, P.tol);
    c->counter = 0;
}

// Start one run of the iteration loop over every active scenario.
__global__ void run_begin_kernel(DevGrid G, int32_t run_max)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    Ctrl *c = G.ctrl;
    int live = 0;
    for (int s = 0; s < G.S; ++s) live += (G.sc[s].active && !G.sc[s].done) ? 1 : 0;
    c->run_iter = 0;
    c->run_max = run_max;
    c->n_live = live;
    c->done = (live == 0 || run_max <= 0) ? 1 : 0;
    c->branch_next = 0;
    for (int k = 0; k < kNumStats; ++k) c->stats[k] = 0;
}

__global__ void __launch_bounds__(kBusBlock)
bus_dual_kernel(DevGrid G, DevOpts O)
{
    __shared__ double sh[kBusBlock / 32][7];
    __shared__ bool last;
    // per slot of the block: contributions to its bus's P row, Q row, pooled
    // w and pooled theta sums, whether it is a branch end, and its bus
    __shared__ double sA[4][kSlotCap];
    __shared__ unsigned short sBusOf[kSlotCap];
    __shared__ unsigned char sIsBr[kSlotCap];
    // per bus of the block: mu_P, mu_Q, w, theta, w - w_prev, theta - theta_prev
    __shared__ double sB[6][kBusPerBlock];
    if (G.ctrl->done) return;
    const int sid = G.blk_scen[blockIdx.x];
    SCtrl *c = G.sc + sid;
    if (!c->active || c->done) return;      // this scenario is not iterating
    const int nb = G.nb, nl = G.nl, ng = G.ng, ns = G.ns;
    const int blk0 = G.blk_off[sid], nblk_s = G.blk_off[sid + 1] - blk0;
    const int i0 = G.blk_bus[blockIdx.x], nbus = G.blk_bus[blockIdx.x + 1] - i0;
    const int k0 = G.row_ptr[i0], nslot = G.row_ptr[i0 + nbus] - k0;
    const double rpq = c->rho_pq, rva = c->rho_va, beta = c->beta;
    // reciprocals once per block: a division costs about ten FP64 instructions
    const double irpq = 1.0 / rpq, irva = 1.0 / rva;
    const double izpq = 1.0 / (beta + rpq), izva = 1.0 / (beta + rva);
    const bool pending = c->pending != 0;
    const double bused = c->beta_used, lmax = O.lambda_max;
    const bool two = O.two_level != 0;
    const double so = O.obj_scale;

    // (A) one thread per slot: generator updates (eq. qp-bound) and every
    // coupling's target t = u + z + y/rho, as the slot's share of the bus sums
    for (int q = threadIdx.x; q < nslot; q += kBusBlock) {
        const int k = k0 + q;
        const int e = G.col[k];
        const double zP = G.sz[k], zQ = G.sz[ns + k], yP = G.sy[k], yQ = G.sy[ns + k];
        if (e < 2 * nl) {
            const int l = e >> 1, end = e & 1;
            const double uP = G.bu[(end ? 2 : 0) * nl + l], uQ = G.bu[(end ? 3 : 1) * nl + l];
            const double uW = G.bu[(end ? 6 : 4) * nl + l], uT = G.bu[(end ? 7 : 5) * nl + l];
            const double tW = uW + G.sz[2 * ns + k] + G.sy[2 * ns + k] * irva;
            const double tT = uT + G.sz[3 * ns + k] + G.sy[3 * ns + k] * irva;
            sA[0][q] = -(uP + zP + yP * irpq);      // a flow copy enters its row with -1
            sA[1][q] = -(uQ + zQ + yQ * irpq);
            sA[2][q] = rva * tW;
            sA[3][q] = rva * tT;
            sIsBr[q] = 1;
        } else {
            const int g = e - 2 * nl;
            // eq. qp-bound: Q = 2 s_o c2' + rho, c = rho (xbar - z) - y - s_o c1'
            const double xP = G.sx[k], xQ = G.sx[ns + k];
            double pg = (rpq * (xP - zP) - yP - so * G.gc[ng + g]) / (2.0 * so * G.gc[g] + rpq);
            double qg = (rpq * (xQ - zQ) - yQ) * irpq;
            pg = clampd(pg, G.glim[0 * ng + g], G.glim[1 * ng + g]);
            qg = clampd(qg, G.glim[2 * ng + g], G.glim[3 * ng + g]);
            G.gu[g] = pg;
            G.gu[ng + g] = qg;
            sA[0][q] = pg + zP + yP * irpq;
            sA[1][q] = qg + zQ + yQ * irpq;
            sA[2][q] = 0.0;
            sA[3][q] = 0.0;
            sIsBr[q] = 0;
        }
    }
    __syncthreads();

    // (B) one thread per bus: the row's sums in CSR order, then eq. qp-bus:
    // pooled w (A column (-gs, bs)) and the 2x2 solve; theta the pooled target
    if (threadIdx.x < nbus) {
        const int i = i0 + threadIdx.x;
        const int r0 = G.row_ptr[i] - k0, r1 = G.row_ptr[i + 1] - k0;
        double rP = 0.0, rQ = 0.0, cw = 0.0, ct = 0.0;
        int nbr = 0;
        for (int q = r0; q < r1; ++q) {
            rP += sA[0][q];
            rQ += sA[1][q];
            cw += sA[2][q];
            ct += sA[3][q];
            nbr += sIsBr[q];
            sBusOf[q] = (unsigned short)threadIdx.x;
        }
        // every copy has weight rho_pq in the P and Q rows (M = A Q^-1 A'),
        // every branch end weight rho_va in the pooled w and theta
        const double nrow = (double)(r1 - r0);
        const double qw = (double)nbr * rva;
        const double gs = G.bus[2 * nb + i], bs = G.bus[3 * nb + i];
        const double iqw = 1.0 / qw;
        const double tw = cw * iqw;
        const double M00 = nrow * irpq + gs * gs * iqw;
        const double M11 = nrow * irpq + bs * bs * iqw;
        const double M01 = -gs * bs * iqw;
        rP += -gs * tw - G.bus[i];
        rQ += bs * tw - G.bus[nb + i];
        const double det = M00 * M11 - M01 * M01;
        const double idet = 1.0 / det;
        const double mu0 = (M11 * rP - M01 * rQ) * idet;
        const double mu1 = (M00 * rQ - M01 * rP) * idet;
        const double w = (cw + gs * mu0 - bs * mu1) * iqw;
        const double th = (i == c->ref) ? 0.0 : ct / qw;
        sB[0][threadIdx.x] = mu0;
        sB[1][threadIdx.x] = mu1;
        sB[2][threadIdx.x] = w;
        sB[3][threadIdx.x] = th;
        sB[4][threadIdx.x] = w - G.bw[i];
        sB[5][threadIdx.x] = th - G.bth[i];
        G.bw[i] = w;
        G.bth[i] = th;
    }
    __syncthreads();

    // (C) one thread per slot: bus copies, lazy outer update, z, y,
    // residual sums, branch targets
    // |u-xbar|^2, |u-xbar+z|^2, |rho dxbar|^2, |z|^2, |u|^2, |xbar|^2, |y|^2
    double acc[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int q = threadIdx.x; q < nslot; q += kBusBlock) {
        const int k = k0 + q;
        const int e = G.col[k];
        const bool isb = e < 2 * nl;
        const int nc = isb ? 4 : 2;
        const int l = e >> 1, end = e & 1;
        const int bl = sBusOf[q];
        const double mu0 = sB[0][bl], mu1 = sB[1][bl];
        double u[4];
        if (isb) {
            u[0] = G.bu[(end ? 2 : 0) * nl + l];
            u[1] = G.bu[(end ? 3 : 1) * nl + l];
            u[2] = G.bu[(end ? 6 : 4) * nl + l];
            u[3] = G.bu[(end ? 7 : 5) * nl + l];
        } else {
            u[0] = G.gu[e - 2 * nl];
            u[1] = G.gu[ng + e - 2 * nl];
            u[2] = u[3] = 0.0;
        }
        const double sgn = isb ? 1.0 : -1.0;   // A = -1 for flow copies, +1 for generators
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            if (cc >= nc) break;
            const bool pq = cc < 2;
            const double rho = pq ? rpq : rva, irho = pq ? irpq : irva, iz = pq ? izpq : izva;
            const double zc = G.sz[cc * ns + k], yc = G.sy[cc * ns + k];
            double xb, dual;
            if (pq) {
                const double tc = u[cc] + zc + yc * irho;
                xb = tc + sgn * (cc == 0 ? mu0 : mu1) * irho;
                dual = rho * (xb - G.sx[cc * ns + k]);
                G.sx[cc * ns + k] = xb;
            } else {
                xb = sB[cc == 2 ? 2 : 3][bl];
                dual = rho * sB[cc == 2 ? 4 : 5][bl];
            }
            double lc = G.sl[cc * ns + k];
            if (pending) {
                lc = clampd(lc + bused * zc, -lmax, lmax);
                G.sl[cc * ns + k] = lc;
            }
            const double r0c = u[cc] - xb;
            const double zn = two ? -(lc + yc + rho * r0c) * iz : 0.0;
            const double yn = yc + rho * (r0c + zn);
            G.sz[cc * ns + k] = zn;
            G.sy[cc * ns + k] = yn;
            acc[0] += r0c * r0c;
            acc[1] += (r0c + zn) * (r0c + zn);
            acc[2] += dual * dual;
            acc[3] += zn * zn;
            acc[4] += u[cc] * u[cc];
            acc[5] += xb * xb;
            acc[6] += yn * yn;
            if (isb) {
                // component index in bt: from end {0,1,4,5}, to end {2,3,6,7}
                const int comp = (cc < 2 ? cc : cc + 2) + (end ? 2 : 0);
                G.bt[comp * nl + l] = xb - zn - yn * irho;
            }
        }
    }
    block_sum<kBusBlock, 7>(acc, sh);
    if (threadIdx.x == 0) {
        double *pp = G.partials + 8 * blockIdx.x;
        for (int k = 0; k < 7; ++k) pp[k] = acc[k];
        __threadfence();
        unsigned int ticket = atomicAdd(&c->counter, 1u);
        last = ticket == (unsigned)nblk_s - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the scenario's last block: fixed-order sum of its block partials
    double v[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblk_s; b += blockDim.x) {
        const volatile double *pp = G.partials + 8 * (blk0 + b);
        for (int k = 0; k < 7; ++k) v[k] += pp[k];
    }
    block_sum<kBusBlock, 7>(v, sh);
    if (threadIdx.x != 0) return;
    c->counter = 0;
    const double pri = sqrt(v[0]), pri_z = sqrt(v[1]), dual = sqrt(v[2]), zn = sqrt(v[3]);
    c->pri = pri; c->pri_z = pri_z; c->dual = dual; c->zn = zn;
    // standard ADMM tolerances (absolute and relative both t):
    // eps_pri(t) = sqrt(m) t + t max(|u|, |xbar|), eps_dual(t) = sqrt(m) t + t |y|
    const double sqm = sqrt((double)c->m);
    const double nux = fmax(sqrt(v[4]), sqrt(v[5])), ny = sqrt(v[6]);
    const double ep = sqm * c->tol + c->tol * nux, ed = sqm * c->tol + c->tol * ny;
    c->eps_pri = ep;
    c->eps_dual = ed;
    if (sid == 0) {
        double *h = G.hist + 4 * (c->iter % kHistCap);
        h[0] = pri; h[1] = dual; h[2] = zn; h[3] = pri_z;
    }
    c->iter += 1;
    c->total_iters += 1;
    int stop = 0;
    c->pending = 0;
    if (!isfinite(pri) || !isfinite(dual) || !isfinite(zn)) {
        c->status = -3;
        stop = 1;
    } else if (pri <= ep && dual <= ed && (!two || zn <= ep)) {
        c->status = 0;
        stop = 1;
    } else {
        if (two) {
            c->inner += 1;
            const double epi = sqm * c->tol_in + c->tol_in * nux;
            const double edi = sqm * c->tol_in + c->tol_in * ny;
            if ((pri_z <= epi && dual <= edi) || c->inner >= O.max_inner) {
                // outer step: lambda <- Proj(lambda + beta z) (applied lazily),
                // beta grows when ||z|| stalled
                c->pending = 1;
                c->beta_used = c->beta;
                if (O.beta_rule == 1) {
                    // adaptive: grow by the squared shortfall of the decrease
                    // (no growth the first time, zprev being infinite)
                    const double r = zn / (O.z_decay * c->zprev);
                    const double f = fmin(O.beta_factor, fmax(1.0, r * r));
                    c->beta = fmin(c->beta * f, O.beta_max);
                } else if (zn > O.z_decay * c->zprev) {
                    c->beta = fmin(c->beta * O.beta_factor, O.beta_max);
                }
                c->zprev = zn;
                c->outer += 1;
                c->inner = 0;
                c->tol_in = fmax(O.tol_in0 * pow(O.tol_in_decay, (double)c->outer), c->tol);
                if (c->outer >= O.max_outer) {
                    c->status = 1;
                    stop = 1;
                }
            }
        }
        if (!stop && c->iter >= c->max_iter) {
            c->status = 1;
            stop = 1;
        }
    }
    if (stop) {
        c->done = 1;
        atomicSub(&G.ctrl->n_live, 1);
    }
}

// End of one iteration: the next branch_tron queue, the scheduling classes,
// and whether the loop goes on (some scenario still running, run cap not hit).
__global__ void control_kernel(DevGrid G, cudaGraphConditionalHandle cond, int32_t use_cond)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    Ctrl *c = G.ctrl;
    int stop = c->done;
    if (!stop) {
        c->run_iter += 1;
        c->total_iters += 1;
        c->branch_next = 0;
        // the branch lists filled by this iteration become the next queue order;
        // the ones it consumed are emptied to be filled next
        const int nxt = (c->total_iters + 1) & 1;
        for (int r = 0; r < kClasses; ++r) c->cls_count[nxt][r] = 0u;
        stop = (c->n_live <= 0 || c->run_iter >= c->run_max) ? 1 : 0;
        c->done = stop;
    }
    if (use_cond) cudaGraphSetConditional(cond, stop ? 0u : 1u);
}

// Ramp limit of Section IV-C around the current dispatch pg:
// pmin' = max(pmin, pg - frac pmax), pmax' = min(pmax, pg + frac pmax) on the
// bounds last set by the caller (pmin' kept <= pmax').
__global__ void ramp_limit_kernel(DevGrid G, Range R, double frac)
{
    const int g = R.g0 + blockIdx.x * blockDim.x + threadIdx.x;
    const int ng = G.ng;
    if (g >= R.g1) return;
    const double lo = G.gbase[g], hi = G.gbase[ng + g], pg = G.gu[g];
    const double r = frac * hi;
    const double nhi = fmin(hi, pg + r);
    G.glim[g] = fmin(fmax(lo, pg - r), nhi);
    G.glim[ng + g] = nhi;
}

// After the loop: apply an outer multiplier update still pending.
__global__ void flush_lambda_kernel(DevGrid G, DevOpts O)
{
    const int ns = G.ns;
    const double lmax = O.lambda_max;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 4 * ns; t += gridDim.x * blockDim.x) {
        const SCtrl *c = G.sc + G.slot_scen[t % ns];
        if (c->pending) G.sl[t] = clampd(G.sl[t] + c->beta_used * G.sz[t], -lmax, lmax);
    }
}

__global__ void clear_pending_kernel(DevGrid G)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < G.S) G.sc[s].pending = 0;
}

// Section IV-A solution extraction and ||c(x)||_inf.  Roles: [0, nb) buses
// (voltage, balance mismatch over the CSR row, voltage bounds), [nb, nb + nl)
// branches (flows from bus voltages, line limits), [nb + nl, ...) generators
// (cost).  The last block reduces the per-block max violation and cost.
__global__ void __launch_bounds__(kFinBlock)
finalize_kernel(DevGrid G, Range R, double *pg, double *qg, double *vm, double *va, double *pf,
                double *qf, double *pt, double *qt, int32_t nblk)
{
    __shared__ double sh[kFinBlock / 32][2];
    __shared__ bool last;
    const int nb = G.nb, nl = G.nl, ng = G.ng;
    const int nbs = R.i1 - R.i0, nls = R.b1 - R.b0, ngs = R.g1 - R.g0;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double viol = 0.0, obj = 0.0;
    // outputs are indexed locally within the scenario
    if (t < nbs) {
        const int i = R.i0 + t;
        const double v = sqrt(fmax(G.bw[i], 0.0));
        if (vm) vm[t] = v;
        if (va) va[t] = G.bth[i];
        const double w2 = v * v;
        double bp = -G.bus[i] - G.bus[2 * nb + i] * w2;
        double bq = -G.bus[nb + i] + G.bus[3 * nb + i] * w2;
        for (int k = G.row_ptr[i]; k < G.row_ptr[i + 1]; ++k) {
            const int e = G.col[k];
            if (e < 2 * nl) {
                const int l = e >> 1, end = e & 1, fi = G.f_bus[l], tj = G.t_bus[l];
                double fl[4];
                flows_at(G.Y, nl, l, sqrt(fmax(G.bw[fi], 0.0)), sqrt(fmax(G.bw[tj], 0.0)),
                         G.bth[fi] - G.bth[tj], fl);
                bp -= end ? fl[2] : fl[0];
                bq -= end ? fl[3] : fl[1];
            } else {
                bp += G.gu[e - 2 * nl];
                bq += G.gu[ng + e - 2 * nl];
            }
        }
        viol = fmax(fmax(fabs(bp), fabs(bq)), fmax(v - G.bus[5 * nb + i], G.bus[4 * nb + i] - v));
    } else if (t < nbs + nls) {
        const int l = R.b0 + t - nbs, lo = t - nbs, fi = G.f_bus[l], tj = G.t_bus[l];
        double fl[4];
        flows_at(G.Y, nl, l, sqrt(fmax(G.bw[fi], 0.0)), sqrt(fmax(G.bw[tj], 0.0)),
                 G.bth[fi] - G.bth[tj], fl);
        if (pf) pf[lo] = fl[0];
        if (qf) qf[lo] = fl[1];
        if (pt) pt[lo] = fl[2];
        if (qt) qt[lo] = fl[3];
        const double rate = G.raw[5 * nl + l];
        if (rate > 0.0)
            viol = fmax(sqrt(fl[0] * fl[0] + fl[1] * fl[1]), sqrt(fl[2] * fl[2] + fl[3] * fl[3])) - rate;
    } else if (t < nbs + nls + ngs) {
        const int go = t - nbs - nls, g = R.g0 + go;
        const double P = G.gu[g];
        if (pg) pg[go] = P;
        if (qg) qg[go] = G.gu[ng + g];
        obj = G.gc[g] * P * P + G.gc[ng + g] * P + G.gc[2 * ng + g];
    }
    // block max of viol, block sum of obj
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        viol = fmax(viol, __shfl_down_sync(0xffffffffu, viol, o));
        obj += __shfl_down_sync(0xffffffffu, obj, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sh[w][0] = viol; sh[w][1] = obj; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double mv = 0.0, so = 0.0;
        for (int k = 0; k < kFinBlock / 32; ++k) { mv = fmax(mv, sh[k][0]); so += sh[k][1]; }
        G.fin_partials[2 * blockIdx.x] = mv;
        G.fin_partials[2 * blockIdx.x + 1] = so;
        __threadfence();
        unsigned int ticket = atomicAdd(&G.sc[R.s].fin_counter, 1u);
        last = ticket == (unsigned)nblk - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double mv = 0.0, so = 0.0;
    for (int b = 0; b < nblk; ++b) {
        const volatile double *pp = G.fin_partials + 2 * b;
        mv = fmax(mv, pp[0]);
        so += pp[1];
    }
    G.sc[R.s].max_viol = mv;
    G.sc[R.s].objective = so;
    G.sc[R.s].fin_counter = 0;
}

}  // namespace admm
