// Internal device-side definitions of libadmm (not part of the public ABI).
//
// Device layout (structure of arrays, FP64 unless noted; nl branches, ng
// generators, nb buses, ns = 2 nl + ng incidence slots in CSR order):
//   branch params  Y[8][nl] (g_ii b_ii g_ij b_ij g_ji b_ji g_jj b_jj),
//                  lim[5][nl] (vmin_i, vmax_i, vmin_j, vmax_j, s lower bound)
//   branch state   bx[6][nl] (v_i v_j th_i th_j s_ij s_ji), blt[2][nl] (lambda-tilde),
//                  balpha[nl] (Cauchy step length of the last TRON call)
//   branch I/O     bt[8][nl] targets xbar - z - y/rho written by the bus kernel,
//                  bu[8][nl] component-side coupling values written by branch_tron
//   generators     gc[3][ng] (c2' c1' c0 per-unit costs), glim[4][ng], gu[2][ng]
//   buses          bus[6][nb] (pd qd gs bs vmin vmax), bw[nb], bth[nb], row_ptr[nb+1]
//   slots          col[ns] (int32 entry id), sx[2][ns] bus-side p/q copies,
//                  sz, sy, sl [4][ns]: z, y, lambda of the slot's couplings
//                  (p, q, w, theta for a branch end; p, q for a generator)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace admm {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int kHistCap = 65536;      // residual history ring (rows of 4 doubles)
constexpr int kNumStats = 9;

// Counters of one solve, summed over branches.
enum StatId { ST_TRON_CALLS = 0, ST_TRON_ITERS, ST_FGH, ST_F, ST_CAUCHY, ST_CG, ST_PS, ST_AL,
              ST_TRON_MAXHIT };

// Loop status kept on the device.
enum { CS_RUNNING = 2 };

// Per-scenario state of Algorithm 1.  A handle holds S scenarios (independent
// grids) concatenated into one set of arrays; each scenario runs its own loop
// counters, penalties, tolerances and stopping decision.
struct SCtrl {
    double tol, rho_pq, rho_va;
    double beta, beta_used, tol_in, zprev;
    double pri, dual, zn, pri_z, eps_pri, eps_dual;
    double objective, max_viol;
    int32_t max_iter, iter, inner, outer, status, done, pending, active;
    int32_t total_iters, ref, m, pad;
    unsigned int counter;          // last-block ticket of bus_dual for this scenario
    unsigned int fin_counter;      // last-block ticket of finalize for this scenario
};

// scheduling classes of branch_tron by loop trips: >= 64, 48, 32, 24, 16, 8, 4, < 4
constexpr int kClasses = 8;

// Whole-handle state of one run of the iteration loop.
struct Ctrl {
    int32_t run_iter, run_max, n_live, done;
    int32_t total_iters, pad0;
    unsigned int branch_next;      // work queue head of branch_tron (reset every iteration)
    unsigned int pad1;
    // longest-first scheduling of branch_tron: branches filed by the loop trips
    // they needed (kClasses classes), double-buffered by iteration parity
    unsigned int cls_count[2][kClasses];
    unsigned long long stats[kNumStats];
};

struct DevOpts {
    double obj_scale;
    double beta0, beta_factor, z_decay, beta_max, lambda_max, tol_in0, tol_in_decay;
    double al_rho0, al_tol, al_decay, al_rho_factor, al_rho_max;
    double tron_gtol, tron_ftol, tron_xtol;
    int32_t two_level, max_outer, max_inner, al_max_iter, tron_max_iter, beta_rule;
    int32_t num_sms;               // SMs of the device (branch_tron's trip barrier)
    int32_t pad_;
};

struct DevGrid {
    int32_t nb, nl, ng, ns, S;
    int32_t nblk_bus;              // blocks of the bus_dual launch (aligned per scenario)
    int32_t nblk_branch;           // blocks of the (persistent) branch_tron launch
    int32_t pad_;
    // scenario layout: index ranges [off[s], off[s+1]) of each scenario
    const int32_t *bus_off, *br_off, *gen_off, *slot_off, *blk_off;
    const int32_t *blk_scen;       // [nblk_bus] scenario of each bus block
    const int32_t *blk_bus;        // [nblk_bus + 1] first bus of each bus block (global)
    const int32_t *br_scen;        // [nl] scenario of each branch
    const int32_t *slot_scen;      // [ns] scenario of each incidence slot
    SCtrl *sc;                     // [S]
    // branches
    const int32_t *f_bus, *t_bus;
    double *Y, *lim, *bx, *blt, *bt, *bu;
    double *balpha;
    const double *raw;             // r x b tap shift rate [6][nl] for the admittance kernel
    // generators
    const int32_t *gen_bus;
    double *gc, *glim, *gu;
    double *gbase;                 // [2][ng] pmin, pmax as last set by the caller
    // buses
    double *bus, *bw, *bth;
    const int32_t *row_ptr, *col;
    // slots
    double *sx, *sz, *sy, *sl;
    // scratch and control
    int32_t *cls_list;             // [2][kClasses][nl] branch ids per (parity, class)
    double *partials;              // [nblk_bus][8]
    double *fin_partials;          // [nblk_fin][2] (one scenario at a time)
    double *hist;                  // [kHistCap][4], scenario 0 only
    Ctrl *ctrl;
    double line_limit_frac;
};

struct SolveParams {
    double tol, rho_pq, rho_va;
    int32_t max_iter, warm;
};

// index ranges of one scenario, for the kernels that work on one scenario
struct Range {
    int32_t s, b0, b1, k0, k1, i0, i1, g0, g1;
};

// kernels
__global__ void admittance_kernel(DevGrid G);
__global__ void cold_start_kernel(DevGrid G, Range R, double beta_init);
__global__ void slot_begin_kernel(DevGrid G, DevOpts O, int32_t s0, int32_t s1, SolveParams P);
__global__ void run_begin_kernel(DevGrid G, int32_t run_max);
__global__ void branch_tron_kernel(DevGrid G, DevOpts O);
__global__ void branch_tron2_kernel(DevGrid G, DevOpts O);   // two lanes per branch
__global__ void bus_dual_kernel(DevGrid G, DevOpts O);
__global__ void control_kernel(DevGrid G, cudaGraphConditionalHandle cond, int32_t use_cond);
__global__ void flush_lambda_kernel(DevGrid G, DevOpts O);
__global__ void clear_pending_kernel(DevGrid G);
__global__ void ramp_limit_kernel(DevGrid G, Range R, double frac);
__global__ void finalize_kernel(DevGrid G, Range R, double *pg, double *qg, double *vm,
                                double *va, double *pf, double *qf, double *pt, double *qt,
                                int32_t nblk);

constexpr int kBranchBlock = 128;
constexpr int kBranchBlocksPerSM = 1;   // launch bound: 255 registers a lane (two blocks still fit an SM)
// dynamic shared memory of a branch_tron block: per lane, the branch data
// (Y[8], t[8]), the packed Hessian and the preconditioner's packed factor (21
// doubles each, stored in 11 pairs) and a scratch of 12 (the preconditioner's
// scaling during CG, H w and the clamped part of a projected step in the
// search)
constexpr size_t kBranchSmem = (size_t)(16 + 2 * 22 + 12) * kBranchBlock * sizeof(double);
constexpr int kBusBlock = 256;      // threads of a bus_dual block
constexpr int kBusPerBlock = 256;   // at most this many buses per bus_dual block
constexpr int kSlotCap = 768;       // at most this many incidence slots per bus_dual block
constexpr int kFinBlock = 256;

}  // namespace admm
