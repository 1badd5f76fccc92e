// bus_dual: the generator x-update, the bus xbar-update, the z-update and the y-update of Algorithm 1
// fused into one pass over the bus -> incident-component CSR map, plus the
// residual reduction and the loop control of the two-level algorithm.
//
// One thread owns one bus row.  Every coupling is owned by exactly one bus (the
// bus its copy lives on), so the gather needs no atomics and sums in CSR order
// (deterministic).  Generators are owned by their bus too: their closed-form
// update (eq. qp-bound) uses only the slot values of that row, so it runs in
// the same thread before the bus update.  The outer multiplier update
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
    if (G.ctrl->done) return;
    const int sid = G.blk_scen[blockIdx.x];
    SCtrl *c = G.sc + sid;
    if (!c->active || c->done) return;      // this scenario is not iterating
    const int nb = G.nb, nl = G.nl, ng = G.ng, ns = G.ns;
    const int blk0 = G.blk_off[sid], nblk_s = G.blk_off[sid + 1] - blk0;
    const int i = G.bus_off[sid] + (blockIdx.x - blk0) * blockDim.x + threadIdx.x;
    const int i_end = G.bus_off[sid + 1];
    const double rpq = c->rho_pq, rva = c->rho_va, beta = c->beta;
    // reciprocals once per block: a division costs about ten FP64 instructions
    const double irpq = 1.0 / rpq, irva = 1.0 / rva;
    const double izpq = 1.0 / (beta + rpq), izva = 1.0 / (beta + rva);
    const bool pending = c->pending != 0;
    const double bused = c->beta_used, lmax = O.lambda_max;
    const bool two = O.two_level != 0;
    // |u-xbar|^2, |u-xbar+z|^2, |rho dxbar|^2, |z|^2, |u|^2, |xbar|^2, |y|^2
    double acc[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (i < i_end) {
        const int r0 = G.row_ptr[i], r1 = G.row_ptr[i + 1];
        const double so = O.obj_scale;
        // pass 1: generator updates, then the bus QP sums
        double M00 = 0.0, M11 = 0.0, rP = 0.0, rQ = 0.0;
        double qw = 0.0, cw = 0.0, qt = 0.0, ct = 0.0;
        for (int k = r0; k < r1; ++k) {
            const int e = G.col[k];
            const double zP = G.sz[k], zQ = G.sz[ns + k], yP = G.sy[k], yQ = G.sy[ns + k];
            if (e < 2 * nl) {
                const int l = e >> 1, end = e & 1;
                const double uP = G.bu[(end ? 2 : 0) * nl + l], uQ = G.bu[(end ? 3 : 1) * nl + l];
                const double uW = G.bu[(end ? 6 : 4) * nl + l], uT = G.bu[(end ? 7 : 5) * nl + l];
                const double zW = G.sz[2 * ns + k], zT = G.sz[3 * ns + k];
                const double yW = G.sy[2 * ns + k], yT = G.sy[3 * ns + k];
                const double tP = uP + zP + yP * irpq, tQ = uQ + zQ + yQ * irpq;
                const double tW = uW + zW + yW * irva, tT = uT + zT + yT * irva;
                M00 += irpq;
                M11 += irpq;
                rP -= tP;
                rQ -= tQ;
                qw += rva; cw += rva * tW;
                qt += rva; ct += rva * tT;
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
                const double tP = pg + zP + yP * irpq, tQ = qg + zQ + yQ * irpq;
                M00 += irpq;
                M11 += irpq;
                rP += tP;
                rQ += tQ;
            }
        }
        // eq. qp-bus: pooled w (A column (-gs, bs)), then the 2x2 solve
        const double gs = G.bus[2 * nb + i], bs = G.bus[3 * nb + i];
        const double iqw = 1.0 / qw;
        const double tw = cw * iqw;
        M00 += gs * gs * iqw;
        M11 += bs * bs * iqw;
        const double M01 = -gs * bs * iqw;
        rP += -gs * tw - G.bus[i];
        rQ += bs * tw - G.bus[nb + i];
        const double det = M00 * M11 - M01 * M01;
        const double idet = 1.0 / det;
        const double mu0 = (M11 * rP - M01 * rQ) * idet;
        const double mu1 = (M00 * rQ - M01 * rP) * idet;
        const double w = (cw + gs * mu0 - bs * mu1) * iqw;
        const double th = (i == c->ref) ? 0.0 : ct / qt;
        const double dw = w - G.bw[i], dth = th - G.bth[i];
        G.bw[i] = w;
        G.bth[i] = th;
        // pass 2: bus copies, lazy outer update, z, y, residuals, branch targets
        for (int k = r0; k < r1; ++k) {
            const int e = G.col[k];
            const bool isb = e < 2 * nl;
            const int nc = isb ? 4 : 2;
            const int l = e >> 1, end = e & 1;
            double u[4], rho[4], irho[4], iz[4];
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
            rho[0] = rho[1] = rpq;
            rho[2] = rho[3] = rva;
            irho[0] = irho[1] = irpq;
            irho[2] = irho[3] = irva;
            iz[0] = iz[1] = izpq;
            iz[2] = iz[3] = izva;
            const double sgn = isb ? 1.0 : -1.0;   // A = -1 for flow copies, +1 for generators
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (c >= nc) break;
                const double zc = G.sz[c * ns + k], yc = G.sy[c * ns + k];
                double xb, dual;
                if (c < 2) {
                    const double tc = u[c] + zc + yc * irho[c];
                    xb = tc + sgn * (c == 0 ? mu0 : mu1) * irho[c];
                    dual = rho[c] * (xb - G.sx[c * ns + k]);
                    G.sx[c * ns + k] = xb;
                } else {
                    xb = c == 2 ? w : th;
                    dual = rho[c] * (c == 2 ? dw : dth);
                }
                double lc = G.sl[c * ns + k];
                if (pending) {
                    lc = clampd(lc + bused * zc, -lmax, lmax);
                    G.sl[c * ns + k] = lc;
                }
                const double r0c = u[c] - xb;
                const double zn = two ? -(lc + yc + rho[c] * r0c) * iz[c] : 0.0;
                const double yn = yc + rho[c] * (r0c + zn);
                G.sz[c * ns + k] = zn;
                G.sy[c * ns + k] = yn;
                acc[0] += r0c * r0c;
                acc[1] += (r0c + zn) * (r0c + zn);
                acc[2] += dual * dual;
                acc[3] += zn * zn;
                acc[4] += u[c] * u[c];
                acc[5] += xb * xb;
                acc[6] += yn * yn;
                if (isb) {
                    // component index in bt: from end {0,1,4,5}, to end {2,3,6,7}
                    const int comp = (c < 2 ? c : c + 2) + (end ? 2 : 0);
                    G.bt[comp * nl + l] = xb - zn - yn * irho[c];
                }
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
                if (zn > O.z_decay * c->zprev) c->beta = fmin(c->beta * O.beta_factor, O.beta_max);
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
