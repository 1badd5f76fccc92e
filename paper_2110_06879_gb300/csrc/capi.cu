// C ABI of libadmm (include/admm.h): handle life cycle, host-side setup
// (validation, CSR incidence map), device allocation, the iteration graph and
// the copy-out of results.  All numerical work runs in the kernels of
// branch_tron.cu and bus_dual.cu.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/admm.h"
#include "admm_internal.cuh"

namespace {
// NVTX range around one C-ABI call, for Nsight timelines (no cost without a tool)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace

using namespace admm;

namespace {

thread_local std::string g_err;

void set_err(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

#define CK(call)                                                                     \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            set_err("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                    __LINE__);                                                       \
            return e_ == cudaErrorMemoryAllocation ? ADMM_ERR_OOM : ADMM_ERR_CUDA;   \
        }                                                                            \
    } while (0)

constexpr int kMaxBodyIters = 16;
constexpr uint64_t kStateMagic = 0x41444d4d53543032ull;   // "ADMMST02"

}  // namespace

struct admm_handle {
    int32_t S = 0;                        // scenarios
    int32_t nb = 0, nl = 0, ng = 0, ns = 0;   // totals over scenarios
    admm_options opts{};
    DevGrid G{};
    DevOpts O{};
    cudaStream_t stream = nullptr;
    void *dmem = nullptr;        // one device allocation, carved into the arrays
    size_t dbytes = 0;
    double *dout = nullptr;      // finalize outputs [2 nb + 4 nl + 2 ng]
    Ctrl *hctrl = nullptr;       // pinned host mirror of the control block
    SCtrl *hsc = nullptr;        // pinned host mirror of the scenario control blocks
    // host copies of the layout (global indices)
    std::vector<int32_t> row_ptr, col, f_bus, t_bus, gen_bus;
    std::vector<int32_t> bus_off, br_off, gen_off, slot_off, blk_off;
    std::vector<double> base_mva;
    int32_t sel = 0;             // scenario addressed by the per-scenario calls
    int nblk_branch = 0, nblk_bus = 0, nblk_fin = 0, nblk_flush = 0;
    int lanes = 1;               // lanes per branch of branch_tron (1 or 2)
    int sms = 152;               // SMs of the device
    // iteration graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t begin_node = nullptr;
    int32_t begin_run_max = 0;
    void *begin_args[2] = {nullptr, nullptr};
    bool graph_ok = false;
};

extern "C" void admm_default_options(admm_options *o)
{
    std::memset(o, 0, sizeof(*o));
    o->rho_pq = 10.0;
    o->rho_va = 1000.0;
    o->obj_scale = 1.0;
    o->line_limit_frac = 0.99;
    o->beta0 = 0.0;
    o->beta_factor = 6.0;
    o->z_decay = 0.8;
    o->beta_max = 1e12;
    o->lambda_max = 1e12;
    o->tol_in0 = 1e-2;
    o->tol_in_decay = 0.5;
    o->al_rho0 = 0.0;
    o->al_tol = 1e-6;
    o->al_decay = 0.1;
    o->al_rho_factor = 100.0;
    o->al_rho_max = 1e12;
    o->tron_gtol = 1e-10;
    o->tron_ftol = 1e-12;
    o->tron_xtol = 1e-13;
    o->two_level = 1;
    o->max_outer = 20;
    o->max_inner = 1000;
    o->al_max_iter = 20;
    o->tron_max_iter = 200;
    o->use_graph = 1;
    o->branch_blocks = 0;
    o->graph_body_iters = 1;
}

extern "C" const char *admm_last_error(void) { return g_err.c_str(); }

extern "C" const char *admm_status_string(int s)
{
    switch (s) {
    case ADMM_OK: return "ADMM_OK";
    case ADMM_NOT_CONVERGED: return "ADMM_NOT_CONVERGED";
    case ADMM_ERR_INVALID_ARG: return "ADMM_ERR_INVALID_ARG";
    case ADMM_ERR_CUDA: return "ADMM_ERR_CUDA";
    case ADMM_ERR_NUMERICAL: return "ADMM_ERR_NUMERICAL";
    case ADMM_ERR_OOM: return "ADMM_ERR_OOM";
    default: return "ADMM_UNKNOWN_STATUS";
    }
}

namespace {

bool finite_all(const double *a, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

int validate(const admm_grid *g, const admm_options *o)
{
    if (!g) { set_err("grid is NULL"); return ADMM_ERR_INVALID_ARG; }
    if (g->nbus < 1 || g->nbranch < 1 || g->ngen < 0) {
        set_err("need nbus >= 1, nbranch >= 1, ngen >= 0");
        return ADMM_ERR_INVALID_ARG;
    }
    long long ns = 2LL * g->nbranch + g->ngen, m = 2LL * g->ngen + 8LL * g->nbranch;
    if (m > 0x7fffffffLL || ns > 0x7fffffffLL) { set_err("grid too large"); return ADMM_ERR_INVALID_ARG; }
    if (g->ref_bus < 0 || g->ref_bus >= g->nbus) { set_err("ref_bus out of range"); return ADMM_ERR_INVALID_ARG; }
    if (!(g->base_mva > 0.0)) { set_err("base_mva must be positive"); return ADMM_ERR_INVALID_ARG; }
    const double *bus_arrays[] = {g->pd, g->qd, g->gs, g->bs, g->vmin, g->vmax};
    const double *br_arrays[] = {g->r, g->x, g->b, g->tap, g->shift, g->rate_a};
    const double *gen_arrays[] = {g->pmin, g->pmax, g->qmin, g->qmax, g->c2, g->c1, g->c0};
    for (auto a : bus_arrays)
        if (!a || !finite_all(a, g->nbus)) { set_err("bus array NULL or not finite"); return ADMM_ERR_INVALID_ARG; }
    for (auto a : br_arrays)
        if (!a || !finite_all(a, g->nbranch)) { set_err("branch array NULL or not finite"); return ADMM_ERR_INVALID_ARG; }
    if (g->ngen > 0) {
        for (auto a : gen_arrays)
            if (!a || !finite_all(a, g->ngen)) { set_err("generator array NULL or not finite"); return ADMM_ERR_INVALID_ARG; }
        if (!g->gen_bus) { set_err("gen_bus is NULL"); return ADMM_ERR_INVALID_ARG; }
    }
    if (!g->f_bus || !g->t_bus) { set_err("f_bus/t_bus NULL"); return ADMM_ERR_INVALID_ARG; }
    std::vector<int> deg(g->nbus, 0);
    for (int l = 0; l < g->nbranch; ++l) {
        int f = g->f_bus[l], t = g->t_bus[l];
        if (f < 0 || f >= g->nbus || t < 0 || t >= g->nbus) { set_err("branch %d: bus index out of range", l); return ADMM_ERR_INVALID_ARG; }
        if (f == t) { set_err("branch %d connects bus %d to itself", l, f); return ADMM_ERR_INVALID_ARG; }
        if (g->r[l] == 0.0 && g->x[l] == 0.0) { set_err("branch %d has zero impedance", l); return ADMM_ERR_INVALID_ARG; }
        deg[f]++; deg[t]++;
    }
    for (int k = 0; k < g->ngen; ++k)
        if (g->gen_bus[k] >= 0 && g->gen_bus[k] < g->nbus) deg[g->gen_bus[k]]++;
    for (int i = 0; i < g->nbus; ++i) {
        if (deg[i] == 0) { set_err("bus %d has no incident branch", i); return ADMM_ERR_INVALID_ARG; }
        if (deg[i] > kSlotCap) {
            set_err("bus %d has %d incident branch ends and generators (at most %d)", i, deg[i], kSlotCap);
            return ADMM_ERR_INVALID_ARG;
        }
        if (!(g->vmin[i] > 0.0) || g->vmin[i] > g->vmax[i]) { set_err("bus %d: need 0 < vmin <= vmax", i); return ADMM_ERR_INVALID_ARG; }
    }
    for (int k = 0; k < g->ngen; ++k) {
        if (g->gen_bus[k] < 0 || g->gen_bus[k] >= g->nbus) { set_err("generator %d: bus out of range", k); return ADMM_ERR_INVALID_ARG; }
        if (g->pmin[k] > g->pmax[k] || g->qmin[k] > g->qmax[k]) { set_err("generator %d: empty bounds", k); return ADMM_ERR_INVALID_ARG; }
        if (g->c2[k] < 0.0) { set_err("generator %d: negative quadratic cost", k); return ADMM_ERR_INVALID_ARG; }
    }
    if (o) {
        if (!(o->rho_pq > 0.0) || !(o->rho_va > 0.0)) { set_err("penalties must be positive"); return ADMM_ERR_INVALID_ARG; }
        if (o->branch_blocks < 0) { set_err("branch_blocks must be >= 0"); return ADMM_ERR_INVALID_ARG; }
        if (o->graph_body_iters < 1 || o->graph_body_iters > kMaxBodyIters) {
            set_err("graph_body_iters must be in 1..%d", kMaxBodyIters);
            return ADMM_ERR_INVALID_ARG;
        }
        if (o->beta_rule < 0 || o->beta_rule > 1) { set_err("beta_rule must be 0 or 1"); return ADMM_ERR_INVALID_ARG; }
        if (o->lanes_per_branch < 0 || o->lanes_per_branch > 2) {
            set_err("lanes_per_branch must be 0, 1 or 2");
            return ADMM_ERR_INVALID_ARG;
        }
        if (o->max_outer < 1 || o->max_inner < 1 || o->tron_max_iter < 1 || o->al_max_iter < 1) {
            set_err("iteration caps must be >= 1");
            return ADMM_ERR_INVALID_ARG;
        }
    }
    return ADMM_OK;
}

// carve 256-byte aligned sub-buffers out of one allocation
struct Carver {
    size_t off = 0;
    template <class T>
    size_t take(size_t n)
    {
        size_t o = off;
        off += ((n * sizeof(T) + 255) / 256) * 256;
        return o;
    }
};

// Offsets of every device array in the handle's single allocation.
struct Layout {
    size_t fb, tb, Y, lim, bx, blt, bt, bu, raw, balpha, gb, gc, glim, gu, gbase, bus, bw, bth,
        rp, col, sx, sz, sy, sl, cls, part, fpart, hist, ctrl, sc, offs, blks, brs, sls, out, blkb;
    size_t bytes;
};

// Sizes of one handle: totals over its scenarios, bus blocks (bus_dual) and
// finalize blocks, the largest scenario (output staging).
struct Sizes {
    long long nb = 0, nl = 0, ng = 0, ns = 0;
    int S = 0, nblk_bus = 0, nblk_fin = 1, maxnb = 1, maxnl = 1, maxng = 1;
};

// Bus blocks of bus_dual for one grid: consecutive buses, at most
// kBusPerBlock of them and at most kSlotCap incidence slots (branch ends and
// generators) per block.  Returns the block count; `starts` (if given)
// receives the first bus (local index) of each block.  Needs every bus's
// slot count <= kSlotCap (checked in validate).
// Buses per bus_dual block: kBusPerBlock, or half of it when the handle's
// buses would not give every SM a block (the 10k-bus grid then runs 79 blocks
// on 79 SMs instead of 40; measured 0.058 -> 0.045 ms a launch, while the
// 70k-bus grid is faster with the full size).
int bus_block_size(const admm_grid *grids, int S)
{
    long long nb = 0;
    for (int s = 0; s < S; ++s) nb += grids[s].nbus;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 152;
    cudaGetLastError();
    return (nb + kBusPerBlock - 1) / kBusPerBlock < sms ? kBusPerBlock / 2 : kBusPerBlock;
}

int bus_block_starts(const admm_grid &g, std::vector<int32_t> *starts, int bpb)
{
    std::vector<int> deg(g.nbus, 0);
    for (int l = 0; l < g.nbranch; ++l) { deg[g.f_bus[l]]++; deg[g.t_bus[l]]++; }
    for (int k = 0; k < g.ngen; ++k) deg[g.gen_bus[k]]++;
    int n = 0, i = 0;
    while (i < g.nbus) {
        if (starts) starts->push_back(i);
        int cnt = 0, slots = 0;
        while (i < g.nbus && cnt < bpb && slots + deg[i] <= kSlotCap) {
            slots += deg[i];
            ++cnt;
            ++i;
        }
        ++n;
    }
    return n;
}

Sizes sizes_of(const admm_grid *grids, int S)
{
    Sizes z;
    z.S = S;
    const int bpb = bus_block_size(grids, S);
    for (int s = 0; s < S; ++s) {
        const admm_grid &g = grids[s];
        z.nb += g.nbus; z.nl += g.nbranch; z.ng += g.ngen;
        z.nblk_bus += bus_block_starts(g, nullptr, bpb);
        const int nf = (g.nbus + g.nbranch + g.ngen + kFinBlock - 1) / kFinBlock;
        z.nblk_fin = nf > z.nblk_fin ? nf : z.nblk_fin;
        z.maxnb = g.nbus > z.maxnb ? g.nbus : z.maxnb;
        z.maxnl = g.nbranch > z.maxnl ? g.nbranch : z.maxnl;
        z.maxng = g.ngen > z.maxng ? g.ngen : z.maxng;
    }
    z.ns = 2 * z.nl + z.ng;
    return z;
}

Layout layout_of(const Sizes &z)
{
    const size_t nb = z.nb, nl = z.nl, ng = z.ng, ns = z.ns, S = z.S;
    Carver cv;
    Layout L;
    L.fb = cv.take<int32_t>(nl); L.tb = cv.take<int32_t>(nl);
    L.Y = cv.take<double>(8 * nl); L.lim = cv.take<double>(5 * nl);
    L.bx = cv.take<double>(6 * nl); L.blt = cv.take<double>(2 * nl);
    L.bt = cv.take<double>(8 * nl); L.bu = cv.take<double>(8 * nl);
    L.raw = cv.take<double>(6 * nl);
    L.balpha = cv.take<double>(nl);
    L.gb = cv.take<int32_t>(ng > 0 ? ng : 1);
    L.gc = cv.take<double>(3 * ng + 1); L.glim = cv.take<double>(4 * ng + 1);
    L.gu = cv.take<double>(2 * ng + 1);
    L.gbase = cv.take<double>(2 * ng + 1);
    L.bus = cv.take<double>(6 * nb); L.bw = cv.take<double>(nb); L.bth = cv.take<double>(nb);
    L.rp = cv.take<int32_t>(nb + 1); L.col = cv.take<int32_t>(ns);
    L.sx = cv.take<double>(2 * ns); L.sz = cv.take<double>(4 * ns);
    L.sy = cv.take<double>(4 * ns); L.sl = cv.take<double>(4 * ns);
    L.cls = cv.take<int32_t>(2 * (size_t)kClasses * nl);
    L.part = cv.take<double>(8 * (size_t)z.nblk_bus); L.fpart = cv.take<double>(2 * (size_t)z.nblk_fin);
    L.hist = cv.take<double>(4 * (size_t)kHistCap);
    L.ctrl = cv.take<Ctrl>(1);
    L.sc = cv.take<SCtrl>(S);
    L.offs = cv.take<int32_t>(5 * (S + 1));
    L.blks = cv.take<int32_t>(z.nblk_bus); L.brs = cv.take<int32_t>(nl); L.sls = cv.take<int32_t>(ns);
    L.blkb = cv.take<int32_t>(z.nblk_bus + 1);
    L.out = cv.take<double>(2 * (size_t)z.maxnb + 4 * (size_t)z.maxnl + 2 * (size_t)z.maxng + 1);
    L.bytes = cv.off;
    return L;
}

// branch_tron with one or two lanes per branch
void *branch_func(int lanes)
{
    return lanes == 2 ? (void *)branch_tron2_kernel : (void *)branch_tron_kernel;
}

void launch_branch(int lanes, int nbk, cudaStream_t s, const DevGrid &G, const DevOpts &O)
{
    if (lanes == 2) branch_tron2_kernel<<<nbk, kBranchBlock, kBranchSmem, s>>>(G, O);
    else branch_tron_kernel<<<nbk, kBranchBlock, kBranchSmem, s>>>(G, O);
}

// the branch kernels take more than the default 48 KB of dynamic shared memory
int branch_smem_setup()
{
    for (void *f : {(void *)branch_tron_kernel, (void *)branch_tron2_kernel})
        CK(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBranchSmem));
    return ADMM_OK;
}

// blocks that give every branch a slot (128 / lanes slots per block)
int branch_blocks_needed(int nl, int lanes)
{
    const int per = kBranchBlock / lanes;
    return (nl + per - 1) / per;
}

int launch_check(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_err("%s launch failed: %s", what, cudaGetErrorString(e));
        return ADMM_ERR_CUDA;
    }
    return ADMM_OK;
}

Range range_of(const admm_handle *h, int s)
{
    Range R;
    R.s = s;
    R.b0 = h->br_off[s]; R.b1 = h->br_off[s + 1];
    R.k0 = h->slot_off[s]; R.k1 = h->slot_off[s + 1];
    R.i0 = h->bus_off[s]; R.i1 = h->bus_off[s + 1];
    R.g0 = h->gen_off[s]; R.g1 = h->gen_off[s + 1];
    return R;
}

// run_begin -> WHILE { branch_tron -> bus_dual -> control } -> flush -> clear
int build_graph(admm_handle *h)
{
    cudaGraph_t graph;
    CK(cudaGraphCreate(&graph, 0));
    h->graph = graph;
    h->begin_args[0] = &h->G;
    h->begin_args[1] = &h->begin_run_max;
    cudaKernelNodeParams kp{};
    kp.func = (void *)run_begin_kernel;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(32);
    kp.kernelParams = h->begin_args;
    CK(cudaGraphAddKernelNode(&h->begin_node, graph, nullptr, 0, &kp));
    cudaGraphConditionalHandle cond;
    CK(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    CK(cudaGraphAddNode(&wnode, graph, &h->begin_node, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    void *bargs[2] = {&h->G, &h->O};
    cudaKernelNodeParams bp{};
    bp.func = branch_func(h->lanes);
    bp.gridDim = dim3(h->nblk_branch);
    bp.blockDim = dim3(kBranchBlock);
    bp.sharedMemBytes = (unsigned)kBranchSmem;
    bp.kernelParams = bargs;
    cudaKernelNodeParams up{};
    up.func = (void *)bus_dual_kernel;
    up.gridDim = dim3(h->nblk_bus);
    up.blockDim = dim3(kBusBlock);
    up.kernelParams = bargs;
    int32_t use_cond = 1;
    void *cargs[3] = {&h->G, &cond, &use_cond};
    cudaKernelNodeParams ccp{};
    ccp.func = (void *)control_kernel;
    ccp.gridDim = dim3(1);
    ccp.blockDim = dim3(32);
    ccp.kernelParams = cargs;
    // graph_body_iters iterations per body: once a control kernel has set the
    // device stop flag, the kernels after it in the body return at once
    cudaGraphNode_t bnode, unode, cnode = nullptr, fnode, pnode;
    for (int r = 0; r < h->opts.graph_body_iters; ++r) {
        CK(cudaGraphAddKernelNode(&bnode, body, cnode ? &cnode : nullptr, cnode ? 1 : 0, &bp));
        CK(cudaGraphAddKernelNode(&unode, body, &bnode, 1, &up));
        CK(cudaGraphAddKernelNode(&cnode, body, &unode, 1, &ccp));
    }
    cudaKernelNodeParams fp{};
    fp.func = (void *)flush_lambda_kernel;
    fp.gridDim = dim3(h->nblk_flush);
    fp.blockDim = dim3(256);
    fp.kernelParams = bargs;
    CK(cudaGraphAddKernelNode(&fnode, graph, &wnode, 1, &fp));
    void *pargs[1] = {&h->G};
    cudaKernelNodeParams pp{};
    pp.func = (void *)clear_pending_kernel;
    pp.gridDim = dim3((h->S + 255) / 256);
    pp.blockDim = dim3(256);
    pp.kernelParams = pargs;
    CK(cudaGraphAddKernelNode(&pnode, graph, &fnode, 1, &pp));
    CK(cudaGraphInstantiate(&h->exec, graph, 0));
    h->graph_ok = true;
    return ADMM_OK;
}

void destroy_graph(admm_handle *h)
{
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->exec = nullptr;
    h->graph = nullptr;
    h->graph_ok = false;
}

int cold_start(admm_handle *h, int s, double rho_va)
{
    const Range R = range_of(h, s);
    const double beta_init = h->opts.beta0 > 0.0 ? h->opts.beta0 : 10.0 * rho_va;
    const int n = (R.b1 - R.b0) + (R.k1 - R.k0) + (R.i1 - R.i0) + (R.g1 - R.g0) + 1;
    cold_start_kernel<<<(n + 255) / 256, 256, 0, h->stream>>>(h->G, R, beta_init);
    return launch_check("cold_start_kernel");
}

int slot_begin(admm_handle *h, int s0, int s1, double rho_pq, double rho_va, double tol,
               int32_t max_iter, int32_t warm)
{
    int rc;
    if (!warm)
        for (int s = s0; s < s1; ++s)
            if ((rc = cold_start(h, s, rho_va)) != ADMM_OK) return rc;
    SolveParams sp{tol, rho_pq, rho_va, max_iter, warm};
    slot_begin_kernel<<<(s1 - s0 + 255) / 256, 256, 0, h->stream>>>(h->G, h->O, s0, s1, sp);
    return launch_check("slot_begin_kernel");
}

// one run of the loop over the active scenarios, at most run_max iterations
int run_async(admm_handle *h, int32_t run_max)
{
    int rc;
    if (h->opts.use_graph && h->graph_ok) {
        h->begin_run_max = run_max;
        cudaKernelNodeParams kp{};
        kp.func = (void *)run_begin_kernel;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(32);
        kp.kernelParams = h->begin_args;
        CK(cudaGraphExecKernelNodeSetParams(h->exec, h->begin_node, &kp));
        CK(cudaGraphLaunch(h->exec, h->stream));
        return ADMM_OK;
    }
    run_begin_kernel<<<1, 32, 0, h->stream>>>(h->G, run_max);
    if ((rc = launch_check("run_begin_kernel")) != ADMM_OK) return rc;
    cudaGraphConditionalHandle none = 0;
    for (int it = 0; it < run_max; ++it) {
        launch_branch(h->lanes, h->nblk_branch, h->stream, h->G, h->O);
        bus_dual_kernel<<<h->nblk_bus, kBusBlock, 0, h->stream>>>(h->G, h->O);
        control_kernel<<<1, 32, 0, h->stream>>>(h->G, none, 0);
        if ((rc = launch_check("iteration kernels")) != ADMM_OK) return rc;
        // poll the device flag now and then so a finished run stops enqueuing
        if ((it & 63) == 63) {
            CK(cudaMemcpyAsync(h->hctrl, h->G.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            if (h->hctrl->done) break;
        }
    }
    flush_lambda_kernel<<<h->nblk_flush, 256, 0, h->stream>>>(h->G, h->O);
    clear_pending_kernel<<<(h->S + 255) / 256, 256, 0, h->stream>>>(h->G);
    return launch_check("flush_lambda_kernel");
}

int sync_sc(admm_handle *h)
{
    CK(cudaMemcpyAsync(h->hsc, h->G.sc, sizeof(SCtrl) * h->S, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(h->hctrl, h->G.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return ADMM_OK;
}

}  // namespace

extern "C" int admm_create_batch(const admm_grid *grids, int32_t nscen, const admm_options *o,
                                 admm_handle **out)
{
    NvtxRange nvtx_("admm_create_batch");
    if (!out) { set_err("out is NULL"); return ADMM_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!grids || nscen < 1) { set_err("need at least one grid"); return ADMM_ERR_INVALID_ARG; }
    int rc;
    long long tot_nb = 0, tot_nl = 0, tot_ng = 0;
    for (int s = 0; s < nscen; ++s) {
        if ((rc = validate(&grids[s], o)) != ADMM_OK) {
            g_err = "scenario " + std::to_string(s) + ": " + g_err;
            return rc;
        }
        tot_nb += grids[s].nbus; tot_nl += grids[s].nbranch; tot_ng += grids[s].ngen;
    }
    if (8 * tot_nl + 2 * tot_ng > 0x7fffffffLL || 2 * tot_nl + tot_ng > 0x7fffffffLL) {
        set_err("batch too large");
        return ADMM_ERR_INVALID_ARG;
    }
    admm_handle *h = new admm_handle();
    if (o) h->opts = *o; else admm_default_options(&h->opts);
    const admm_options &op = h->opts;
    const int S = nscen;
    h->S = S;
    h->nb = (int)tot_nb; h->nl = (int)tot_nl; h->ng = (int)tot_ng;
    h->ns = 2 * h->nl + h->ng;
    const int nb = h->nb, nl = h->nl, ng = h->ng, ns = h->ns;
    h->bus_off.assign(S + 1, 0); h->br_off.assign(S + 1, 0); h->gen_off.assign(S + 1, 0);
    h->slot_off.assign(S + 1, 0); h->blk_off.assign(S + 1, 0);
    h->base_mva.resize(S);
    const int bpb = bus_block_size(grids, S);
    for (int s = 0; s < S; ++s) {
        h->bus_off[s + 1] = h->bus_off[s] + grids[s].nbus;
        h->br_off[s + 1] = h->br_off[s] + grids[s].nbranch;
        h->gen_off[s + 1] = h->gen_off[s] + grids[s].ngen;
        h->blk_off[s + 1] = h->blk_off[s] + bus_block_starts(grids[s], nullptr, bpb);
        h->base_mva[s] = grids[s].base_mva;
    }
    // concatenated topology in global indices
    h->f_bus.resize(nl); h->t_bus.resize(nl); h->gen_bus.resize(ng);
    std::vector<int32_t> br_scen(nl), blk_scen(h->blk_off[S]), slot_scen(ns);
    for (int s = 0; s < S; ++s) {
        const admm_grid &g = grids[s];
        for (int l = 0; l < g.nbranch; ++l) {
            h->f_bus[h->br_off[s] + l] = h->bus_off[s] + g.f_bus[l];
            h->t_bus[h->br_off[s] + l] = h->bus_off[s] + g.t_bus[l];
            br_scen[h->br_off[s] + l] = s;
        }
        for (int k = 0; k < g.ngen; ++k) h->gen_bus[h->gen_off[s] + k] = h->bus_off[s] + g.gen_bus[k];
        for (int b = h->blk_off[s]; b < h->blk_off[s + 1]; ++b) blk_scen[b] = s;
    }
    // first bus (global) of every bus_dual block, and the end
    std::vector<int32_t> blk_bus;
    blk_bus.reserve(h->blk_off[S] + 1);
    for (int s = 0; s < S; ++s) {
        std::vector<int32_t> st;
        bus_block_starts(grids[s], &st, bpb);
        for (int32_t b : st) blk_bus.push_back(h->bus_off[s] + b);
    }
    blk_bus.push_back(h->bus_off[S]);
    // CSR bus -> incident entries by a stable counting sort over entry ids
    h->row_ptr.assign(nb + 1, 0);
    h->col.assign(ns, 0);
    auto bus_of = [&](int e) { return e < 2 * nl ? ((e & 1) ? h->t_bus[e >> 1] : h->f_bus[e >> 1]) : h->gen_bus[e - 2 * nl]; };
    for (int e = 0; e < ns; ++e) h->row_ptr[bus_of(e) + 1]++;
    for (int i = 0; i < nb; ++i) h->row_ptr[i + 1] += h->row_ptr[i];
    {
        std::vector<int32_t> fill(h->row_ptr.begin(), h->row_ptr.end() - 1);
        for (int e = 0; e < ns; ++e) h->col[fill[bus_of(e)]++] = e;
    }
    for (int s = 0; s <= S; ++s) h->slot_off[s] = h->row_ptr[h->bus_off[s]];
    for (int s = 0; s < S; ++s)
        for (int k = h->slot_off[s]; k < h->slot_off[s + 1]; ++k) slot_scen[k] = s;
    {
        // branch_tron is persistent: its blocks pull branches from a queue and
        // none waits on another, so any block count is correct
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            sms = 152;
        cudaGetLastError();
        h->sms = sms;
        h->lanes = op.lanes_per_branch == 2 ? 2 : 1;
        const int need = branch_blocks_needed(nl, h->lanes);
        // default: two blocks per SM (two warps per sub-partition hide part of
        // the FP64 latency) when the branches fill every slot of them, else one
        const int cap = op.branch_blocks > 0 ? op.branch_blocks : (need >= 2 * sms ? 2 * sms : sms);
        h->nblk_branch = need < cap ? need : cap;
    }
    h->nblk_bus = h->blk_off[S];
    const Sizes zs = sizes_of(grids, S);
    h->nblk_fin = zs.nblk_fin;
    h->nblk_flush = (4 * ns + 255) / 256 < 1184 ? (4 * ns + 255) / 256 : 1184;
    // device layout
    const Layout Lo = layout_of(zs);
    h->dbytes = Lo.bytes;
    if ((rc = branch_smem_setup()) != ADMM_OK) { delete h; return rc; }
    cudaError_t e = cudaMalloc(&h->dmem, h->dbytes);
    if (e != cudaSuccess) {
        set_err("cudaMalloc(%zu) failed: %s", h->dbytes, cudaGetErrorString(e));
        delete h;
        return e == cudaErrorMemoryAllocation ? ADMM_ERR_OOM : ADMM_ERR_CUDA;
    }
    if (cudaMallocHost(&h->hctrl, sizeof(Ctrl)) != cudaSuccess ||
        cudaMallocHost(&h->hsc, sizeof(SCtrl) * S) != cudaSuccess) {
        set_err("cudaMallocHost failed");
        admm_destroy(h);
        return ADMM_ERR_CUDA;
    }
    char *base = (char *)h->dmem;
    DevGrid &G = h->G;
    G.nb = nb; G.nl = nl; G.ng = ng; G.ns = ns; G.S = S;
    G.nblk_bus = h->nblk_bus;
    G.nblk_branch = h->nblk_branch;
    G.f_bus = (int32_t *)(base + Lo.fb); G.t_bus = (int32_t *)(base + Lo.tb);
    G.Y = (double *)(base + Lo.Y); G.lim = (double *)(base + Lo.lim);
    G.bx = (double *)(base + Lo.bx); G.blt = (double *)(base + Lo.blt);
    G.bt = (double *)(base + Lo.bt); G.bu = (double *)(base + Lo.bu);
    G.raw = (double *)(base + Lo.raw);
    G.balpha = (double *)(base + Lo.balpha);
    G.gen_bus = (int32_t *)(base + Lo.gb);
    G.gc = (double *)(base + Lo.gc); G.glim = (double *)(base + Lo.glim); G.gu = (double *)(base + Lo.gu);
    G.gbase = (double *)(base + Lo.gbase);
    G.bus = (double *)(base + Lo.bus); G.bw = (double *)(base + Lo.bw); G.bth = (double *)(base + Lo.bth);
    G.row_ptr = (int32_t *)(base + Lo.rp); G.col = (int32_t *)(base + Lo.col);
    G.sx = (double *)(base + Lo.sx); G.sz = (double *)(base + Lo.sz);
    G.sy = (double *)(base + Lo.sy); G.sl = (double *)(base + Lo.sl);
    G.cls_list = (int32_t *)(base + Lo.cls);
    G.partials = (double *)(base + Lo.part); G.fin_partials = (double *)(base + Lo.fpart);
    G.hist = (double *)(base + Lo.hist);
    G.ctrl = (Ctrl *)(base + Lo.ctrl);
    G.sc = (SCtrl *)(base + Lo.sc);
    int32_t *offs = (int32_t *)(base + Lo.offs);
    G.bus_off = offs; G.br_off = offs + (S + 1); G.gen_off = offs + 2 * (S + 1);
    G.slot_off = offs + 3 * (S + 1); G.blk_off = offs + 4 * (S + 1);
    G.blk_scen = (int32_t *)(base + Lo.blks); G.br_scen = (int32_t *)(base + Lo.brs);
    G.slot_scen = (int32_t *)(base + Lo.sls);
    G.blk_bus = (int32_t *)(base + Lo.blkb);
    G.line_limit_frac = op.line_limit_frac;
    h->dout = (double *)(base + Lo.out);
    DevOpts &O = h->O;
    O.obj_scale = op.obj_scale;
    O.beta0 = op.beta0; O.beta_factor = op.beta_factor; O.z_decay = op.z_decay;
    O.beta_max = op.beta_max; O.lambda_max = op.lambda_max;
    O.tol_in0 = op.tol_in0; O.tol_in_decay = op.tol_in_decay;
    O.al_rho0 = op.al_rho0; O.al_tol = op.al_tol; O.al_decay = op.al_decay;
    O.al_rho_factor = op.al_rho_factor; O.al_rho_max = op.al_rho_max;
    O.tron_gtol = op.tron_gtol; O.tron_ftol = op.tron_ftol; O.tron_xtol = op.tron_xtol;
    O.two_level = op.two_level; O.max_outer = op.max_outer; O.max_inner = op.max_inner;
    O.al_max_iter = op.al_max_iter; O.tron_max_iter = op.tron_max_iter;
    O.beta_rule = op.beta_rule;
    O.num_sms = h->sms;
    O.pad_ = 0;
    // uploads (host staging in the device layout)
    {
        std::vector<double> bus(6 * (size_t)nb), raw(6 * (size_t)nl), gc(3 * (size_t)ng + 1),
            glim(4 * (size_t)ng + 1);
        std::vector<SCtrl> sc(S);
        for (int s = 0; s < S; ++s) {
            const admm_grid &g = grids[s];
            const int i0 = h->bus_off[s], l0 = h->br_off[s], k0 = h->gen_off[s];
            const double *ba[6] = {g.pd, g.qd, g.gs, g.bs, g.vmin, g.vmax};
            for (int k = 0; k < 6; ++k)
                std::memcpy(&bus[(size_t)k * nb + i0], ba[k], sizeof(double) * g.nbus);
            const double *ra[6] = {g.r, g.x, g.b, g.tap, g.shift, g.rate_a};
            for (int k = 0; k < 6; ++k)
                std::memcpy(&raw[(size_t)k * nl + l0], ra[k], sizeof(double) * g.nbranch);
            for (int k = 0; k < g.ngen; ++k) {
                const int q = k0 + k;
                gc[q] = g.c2[k] * g.base_mva * g.base_mva;
                gc[ng + q] = g.c1[k] * g.base_mva;
                gc[2 * (size_t)ng + q] = g.c0[k];
                glim[q] = g.pmin[k];
                glim[ng + q] = g.pmax[k];
                glim[2 * (size_t)ng + q] = g.qmin[k];
                glim[3 * (size_t)ng + q] = g.qmax[k];
            }
            std::memset(&sc[s], 0, sizeof(SCtrl));
            sc[s].ref = i0 + g.ref_bus;
            sc[s].m = 2 * g.ngen + 8 * g.nbranch;
            sc[s].done = 1;
            sc[s].rho_pq = op.rho_pq;
            sc[s].rho_va = op.rho_va;
        }
        std::vector<int32_t> offv(5 * (size_t)(S + 1));
        for (int s = 0; s <= S; ++s) {
            offv[s] = h->bus_off[s];
            offv[(S + 1) + s] = h->br_off[s];
            offv[2 * (S + 1) + s] = h->gen_off[s];
            offv[3 * (S + 1) + s] = h->slot_off[s];
            offv[4 * (S + 1) + s] = h->blk_off[s];
        }
        auto up = [&](void *dst, const void *src, size_t bytes) {
            return bytes == 0 || cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
        };
        if (cudaMemset(h->dmem, 0, h->dbytes) != cudaSuccess || !up(G.bus, bus.data(), bus.size() * 8) ||
            !up((void *)G.raw, raw.data(), raw.size() * 8) || !up(G.gc, gc.data(), gc.size() * 8) ||
            !up(G.glim, glim.data(), glim.size() * 8) || !up(G.gbase, glim.data(), 2 * (size_t)ng * 8) ||
            !up((void *)G.f_bus, h->f_bus.data(), nl * 4) || !up((void *)G.t_bus, h->t_bus.data(), nl * 4) ||
            !up((void *)G.gen_bus, h->gen_bus.data(), (size_t)ng * 4) ||
            !up((void *)G.row_ptr, h->row_ptr.data(), (nb + 1) * 4) || !up((void *)G.col, h->col.data(), ns * 4) ||
            !up(G.sc, sc.data(), sizeof(SCtrl) * S) || !up(offs, offv.data(), offv.size() * 4) ||
            !up((void *)G.blk_scen, blk_scen.data(), blk_scen.size() * 4) ||
            !up((void *)G.blk_bus, blk_bus.data(), blk_bus.size() * 4) ||
            !up((void *)G.br_scen, br_scen.data(), br_scen.size() * 4) ||
            !up((void *)G.slot_scen, slot_scen.data(), slot_scen.size() * 4)) {
            set_err("upload failed: %s", cudaGetErrorString(cudaGetLastError()));
            admm_destroy(h);
            return ADMM_ERR_CUDA;
        }
    }
    admittance_kernel<<<(nl + 255) / 256, 256, 0, h->stream>>>(G);
    if ((rc = launch_check("admittance_kernel")) != ADMM_OK) { admm_destroy(h); return rc; }
    for (int s = 0; s < S; ++s)
        if ((rc = cold_start(h, s, op.rho_va)) != ADMM_OK) { admm_destroy(h); return rc; }
    if (op.use_graph) {
        rc = build_graph(h);
        if (rc != ADMM_OK) {
            // fall back to stream launches (conditional graph nodes unavailable)
            destroy_graph(h);
            cudaGetLastError();
            h->opts.use_graph = 0;
        }
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        set_err("setup failed: %s", cudaGetErrorString(cudaGetLastError()));
        admm_destroy(h);
        return ADMM_ERR_CUDA;
    }
    *out = h;
    return ADMM_OK;
}

extern "C" int admm_device_bytes(const admm_grid *grids, int32_t nscen, size_t *bytes)
{
    if (!grids || nscen < 1 || !bytes) { set_err("need grids, nscen >= 1 and bytes"); return ADMM_ERR_INVALID_ARG; }
    for (int s = 0; s < nscen; ++s)
        if (grids[s].nbus < 1 || grids[s].nbranch < 1 || grids[s].ngen < 0) {
            set_err("scenario %d: need nbus >= 1, nbranch >= 1, ngen >= 0", s);
            return ADMM_ERR_INVALID_ARG;
        }
    *bytes = layout_of(sizes_of(grids, nscen)).bytes;
    return ADMM_OK;
}

extern "C" int admm_create(const admm_grid *g, const admm_options *o, admm_handle **out)
{
    if (!g) { set_err("grid is NULL"); return ADMM_ERR_INVALID_ARG; }
    return admm_create_batch(g, 1, o, out);
}

extern "C" void admm_destroy(admm_handle *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    destroy_graph(h);
    if (h->dmem) cudaFree(h->dmem);
    if (h->hctrl) cudaFreeHost(h->hctrl);
    if (h->hsc) cudaFreeHost(h->hsc);
    delete h;
}

extern "C" int32_t admm_scenario_count(admm_handle *h) { return h ? h->S : 0; }

extern "C" int admm_select_scenario(admm_handle *h, int32_t s)
{
    if (!h || s < 0 || s >= h->S) { set_err("scenario out of range"); return ADMM_ERR_INVALID_ARG; }
    h->sel = s;
    return ADMM_OK;
}

extern "C" int admm_set_stream(admm_handle *h, void *s)
{
    if (!h) { set_err("handle is NULL"); return ADMM_ERR_INVALID_ARG; }
    cudaStream_t ns = (cudaStream_t)s;
    if (ns != h->stream) {
        // order the handle's work queued on the old stream before the new one's
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaError_t e = cudaEventRecord(ev, h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ns, ev, 0);
        cudaEventDestroy(ev);
        CK(e);
    }
    h->stream = ns;
    return ADMM_OK;
}

extern "C" int admm_set_loads(admm_handle *h, const double *pd, const double *qd)
{
    NvtxRange nvtx_("admm_set_loads");
    if (!h || !pd || !qd) { set_err("NULL argument"); return ADMM_ERR_INVALID_ARG; }
    const int i0 = h->bus_off[h->sel], n = h->bus_off[h->sel + 1] - i0;
    if (!finite_all(pd, n) || !finite_all(qd, n)) { set_err("loads not finite"); return ADMM_ERR_INVALID_ARG; }
    CK(cudaMemcpyAsync(h->G.bus + i0, pd, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->G.bus + h->nb + i0, qd, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    return ADMM_OK;
}

extern "C" int admm_set_loads_device(admm_handle *h, const double *d_pd, const double *d_qd)
{
    if (!h || !d_pd || !d_qd) { set_err("NULL argument"); return ADMM_ERR_INVALID_ARG; }
    const int i0 = h->bus_off[h->sel], n = h->bus_off[h->sel + 1] - i0;
    CK(cudaMemcpyAsync(h->G.bus + i0, d_pd, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(h->G.bus + h->nb + i0, d_qd, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
    return ADMM_OK;
}

extern "C" int admm_set_gen_bounds(admm_handle *h, const double *pmin, const double *pmax)
{
    if (!h || !pmin || !pmax) { set_err("NULL argument"); return ADMM_ERR_INVALID_ARG; }
    const int g0 = h->gen_off[h->sel], n = h->gen_off[h->sel + 1] - g0;
    for (int k = 0; k < n; ++k)
        if (!(pmin[k] <= pmax[k]) || !std::isfinite(pmin[k]) || !std::isfinite(pmax[k])) {
            set_err("generator %d: empty or non-finite bounds", k);
            return ADMM_ERR_INVALID_ARG;
        }
    if (n == 0) return ADMM_OK;
    const int ng = h->ng;
    CK(cudaMemcpyAsync(h->G.glim + g0, pmin, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->G.glim + ng + g0, pmax, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->G.gbase + g0, pmin, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->G.gbase + ng + g0, pmax, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    return ADMM_OK;
}

extern "C" int admm_set_ramp_limit(admm_handle *h, double frac)
{
    if (!h) { set_err("handle is NULL"); return ADMM_ERR_INVALID_ARG; }
    if (!(frac >= 0.0) || !std::isfinite(frac)) { set_err("ramp fraction must be >= 0"); return ADMM_ERR_INVALID_ARG; }
    const Range R = range_of(h, h->sel);
    if (R.g1 == R.g0) return ADMM_OK;
    ramp_limit_kernel<<<(R.g1 - R.g0 + 255) / 256, 256, 0, h->stream>>>(h->G, R, frac);
    return launch_check("ramp_limit_kernel");
}

extern "C" int admm_solve_async(admm_handle *h, double rho_pq, double rho_va, double tol,
                                int32_t max_iter, int32_t warm_start)
{
    NvtxRange nvtx_("admm_solve_async");
    if (!h) { set_err("handle is NULL"); return ADMM_ERR_INVALID_ARG; }
    if (!(rho_pq > 0.0) || !(rho_va > 0.0) || !(tol >= 0.0) || max_iter < 0) {
        set_err("need rho > 0, tol >= 0, max_iter >= 0");
        return ADMM_ERR_INVALID_ARG;
    }
    h->opts.rho_pq = rho_pq;
    h->opts.rho_va = rho_va;
    int rc = slot_begin(h, 0, h->S, rho_pq, rho_va, tol, max_iter, warm_start);
    if (rc != ADMM_OK) return rc;
    if (max_iter == 0) return ADMM_OK;
    return run_async(h, max_iter);
}

extern "C" int admm_solve(admm_handle *h, double rho_pq, double rho_va, double tol, int32_t max_iter,
                          int32_t warm_start)
{
    NvtxRange nvtx_("admm_solve");
    int rc = admm_solve_async(h, rho_pq, rho_va, tol, max_iter, warm_start);
    if (rc != ADMM_OK) return rc;
    if ((rc = sync_sc(h)) != ADMM_OK) return rc;
    int st = ADMM_OK;
    for (int s = 0; s < h->S; ++s) {
        int q = h->hsc[s].status == CS_RUNNING ? ADMM_NOT_CONVERGED : h->hsc[s].status;
        if (max_iter == 0) q = ADMM_NOT_CONVERGED;
        if (q < 0) st = q < st ? q : st;
        else if (st >= 0 && q > st) st = q;
    }
    return st;
}

extern "C" int admm_slot_begin(admm_handle *h, int32_t s, double rho_pq, double rho_va, double tol,
                               int32_t max_iter, int32_t warm_start)
{
    NvtxRange nvtx_("admm_slot_begin");
    if (!h || s < 0 || s >= h->S) { set_err("scenario out of range"); return ADMM_ERR_INVALID_ARG; }
    if (!(rho_pq > 0.0) || !(rho_va > 0.0) || !(tol >= 0.0) || max_iter < 0) {
        set_err("need rho > 0, tol >= 0, max_iter >= 0");
        return ADMM_ERR_INVALID_ARG;
    }
    return slot_begin(h, s, s + 1, rho_pq, rho_va, tol, max_iter, warm_start);
}

extern "C" int admm_run(admm_handle *h, int32_t max_iters)
{
    NvtxRange nvtx_("admm_run");
    if (!h || max_iters < 0) { set_err("bad argument"); return ADMM_ERR_INVALID_ARG; }
    if (max_iters == 0) return ADMM_OK;
    return run_async(h, max_iters);
}

extern "C" int admm_slot_status(admm_handle *h, int32_t *status, int32_t *iters)
{
    if (!h) { set_err("handle is NULL"); return ADMM_ERR_INVALID_ARG; }
    int rc = sync_sc(h);
    if (rc != ADMM_OK) return rc;
    for (int s = 0; s < h->S; ++s) {
        const SCtrl &c = h->hsc[s];
        if (status) status[s] = !c.done ? CS_RUNNING : c.status == CS_RUNNING ? ADMM_NOT_CONVERGED : c.status;
        if (iters) iters[s] = c.iter;
    }
    return ADMM_OK;
}

extern "C" int admm_get_residuals(admm_handle *h, admm_residuals *out)
{
    if (!h || !out) { set_err("NULL argument"); return ADMM_ERR_INVALID_ARG; }
    int rc = sync_sc(h);
    if (rc != ADMM_OK) return rc;
    const SCtrl &c = h->hsc[h->sel];
    out->iters = c.iter;
    out->outer_iters = c.outer;
    out->status = c.status == CS_RUNNING ? ADMM_NOT_CONVERGED : c.status;
    out->tron_failures = (int32_t)h->hctrl->stats[ST_TRON_MAXHIT];
    out->primal_res = c.pri;
    out->dual_res = c.dual;
    out->z_norm = c.zn;
    out->primal_z = c.pri_z;
    out->beta = c.beta;
    out->eps_pri = c.eps_pri;
    out->eps_dual = c.eps_dual;
    out->objective = c.objective;
    out->max_viol = c.max_viol;
    return ADMM_OK;
}

extern "C" int admm_get_solution(admm_handle *h, double *pg, double *qg, double *vm, double *va,
                                 double *pf, double *qf, double *pt, double *qt)
{
    NvtxRange nvtx_("admm_get_solution");
    if (!h) { set_err("handle is NULL"); return ADMM_ERR_INVALID_ARG; }
    const Range R = range_of(h, h->sel);
    const int nb = R.i1 - R.i0, nl = R.b1 - R.b0, ng = R.g1 - R.g0;
    double *d = h->dout;
    double *dvm = d, *dva = d + nb, *dpf = d + 2 * nb, *dqf = dpf + nl, *dpt = dqf + nl,
           *dqt = dpt + nl, *dpg = dqt + nl, *dqg = dpg + ng;
    const int nblk = (nb + nl + ng + kFinBlock - 1) / kFinBlock;
    finalize_kernel<<<nblk, kFinBlock, 0, h->stream>>>(h->G, R, dpg, dqg, dvm, dva, dpf, dqf, dpt,
                                                       dqt, nblk);
    int rc = launch_check("finalize_kernel");
    if (rc != ADMM_OK) return rc;
    struct { double *host; const double *dev; int n; } cp[] = {
        {pg, dpg, ng}, {qg, dqg, ng}, {vm, dvm, nb}, {va, dva, nb},
        {pf, dpf, nl}, {qf, dqf, nl}, {pt, dpt, nl}, {qt, dqt, nl}};
    for (auto &c : cp)
        if (c.host && c.n > 0)
            CK(cudaMemcpyAsync(c.host, c.dev, sizeof(double) * c.n, cudaMemcpyDeviceToHost, h->stream));
    return sync_sc(h);
}

extern "C" int32_t admm_get_history(admm_handle *h, double *out, int32_t cap)
{
    if (!h || !out || cap < 0) { set_err("bad argument"); return ADMM_ERR_INVALID_ARG; }
    if (sync_sc(h) != ADMM_OK) return ADMM_ERR_CUDA;
    const int total = h->hsc[0].iter;
    int n = total > kHistCap ? kHistCap : total;   // the ring keeps the last kHistCap rows
    if (n > cap) n = cap;
    std::vector<double> all(4 * (size_t)kHistCap);
    if (cudaMemcpy(all.data(), h->G.hist, all.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_err("history copy failed");
        return ADMM_ERR_CUDA;
    }
    const int first = total > kHistCap ? total - kHistCap : 0;
    for (int r = 0; r < n; ++r)
        std::memcpy(out + 4 * (size_t)r, &all[4 * (size_t)((first + r) % kHistCap)], 4 * sizeof(double));
    return n;
}

namespace {

int fetch(admm_handle *h, const double *dev, size_t n, std::vector<double> &v)
{
    v.resize(n);
    if (n == 0) return ADMM_OK;
    CK(cudaMemcpyAsync(v.data(), dev, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return ADMM_OK;
}

}  // namespace

extern "C" int admm_get_vector(admm_handle *h, int32_t which, double *out)
{
    if (!h || !out) { set_err("NULL argument"); return ADMM_ERR_INVALID_ARG; }
    const int nb = h->nb, nl = h->nl, ng = h->ng, ns = h->ns;
    const Range R = range_of(h, h->sel);
    const int ngs = R.g1 - R.g0, nbs = R.i1 - R.i0;
    std::vector<double> a, b, c;
    int rc = ADMM_OK;
    // canonical order within the scenario: its generators, then its branches
    auto cb = [&](int l, int k) { return 2 * (size_t)ngs + 8 * (size_t)(l - R.b0) + k; };
    auto sync = [&]() -> int { CK(cudaStreamSynchronize(h->stream)); return ADMM_OK; };
    switch (which) {
    case ADMM_VEC_U:
        if ((rc = fetch(h, h->G.bu, 8 * (size_t)nl, a)) || (rc = fetch(h, h->G.gu, 2 * (size_t)ng, b)) || (rc = sync())) return rc;
        for (int g = R.g0; g < R.g1; ++g) { out[2 * (g - R.g0)] = b[g]; out[2 * (g - R.g0) + 1] = b[ng + g]; }
        for (int l = R.b0; l < R.b1; ++l)
            for (int k = 0; k < 8; ++k) out[cb(l, k)] = a[(size_t)k * nl + l];
        return ADMM_OK;
    case ADMM_VEC_XBAR:
    case ADMM_VEC_Z:
    case ADMM_VEC_Y:
    case ADMM_VEC_LAMBDA: {
        const double *src = which == ADMM_VEC_Z ? h->G.sz : which == ADMM_VEC_Y ? h->G.sy : h->G.sl;
        if (which == ADMM_VEC_XBAR) {
            if ((rc = fetch(h, h->G.sx, 2 * (size_t)ns, a)) || (rc = fetch(h, h->G.bw, nb, b)) ||
                (rc = fetch(h, h->G.bth, nb, c)) || (rc = sync()))
                return rc;
        } else if ((rc = fetch(h, src, 4 * (size_t)ns, a)) || (rc = sync())) {
            return rc;
        }
        for (int i = R.i0; i < R.i1; ++i) {
            for (int k = h->row_ptr[i]; k < h->row_ptr[i + 1]; ++k) {
                const int e = h->col[k];
                if (e < 2 * nl) {
                    const int l = e >> 1, end = e & 1;
                    const size_t cp = cb(l, end ? 2 : 0), cq = cb(l, end ? 3 : 1);
                    const size_t cw = cb(l, end ? 6 : 4), ct = cb(l, end ? 7 : 5);
                    if (which == ADMM_VEC_XBAR) {
                        out[cp] = a[k]; out[cq] = a[ns + k]; out[cw] = b[i]; out[ct] = c[i];
                    } else {
                        out[cp] = a[k]; out[cq] = a[ns + k]; out[cw] = a[2 * (size_t)ns + k];
                        out[ct] = a[3 * (size_t)ns + k];
                    }
                } else {
                    const int g = e - 2 * nl - R.g0;
                    out[2 * g] = a[k];
                    out[2 * g + 1] = a[ns + k];
                }
            }
        }
        return ADMM_OK;
    }
    case ADMM_VEC_RHO: {
        if ((rc = sync_sc(h)) != ADMM_OK) return rc;
        const double rp = h->hsc[h->sel].rho_pq, rv = h->hsc[h->sel].rho_va;
        for (int g = 0; g < ngs; ++g) { out[2 * g] = rp; out[2 * g + 1] = rp; }
        for (int l = R.b0; l < R.b1; ++l)
            for (int k = 0; k < 8; ++k) out[cb(l, k)] = k < 4 ? rp : rv;
        return ADMM_OK;
    }
    case ADMM_VEC_BRANCH_X:
    case ADMM_VEC_BRANCH_LT:
    case ADMM_VEC_ADMITTANCE: {
        const int w = which == ADMM_VEC_BRANCH_X ? 6 : which == ADMM_VEC_BRANCH_LT ? 2 : 8;
        const double *src = which == ADMM_VEC_BRANCH_X ? h->G.bx : which == ADMM_VEC_BRANCH_LT ? h->G.blt : h->G.Y;
        if ((rc = fetch(h, src, (size_t)w * nl, a)) || (rc = sync())) return rc;
        for (int l = R.b0; l < R.b1; ++l)
            for (int k = 0; k < w; ++k) out[(size_t)(l - R.b0) * w + k] = a[(size_t)k * nl + l];
        return ADMM_OK;
    }
    case ADMM_VEC_BUS:
        if ((rc = fetch(h, h->G.bw, nb, a)) || (rc = fetch(h, h->G.bth, nb, b)) || (rc = sync())) return rc;
        for (int i = 0; i < nbs; ++i) { out[2 * i] = a[R.i0 + i]; out[2 * i + 1] = b[R.i0 + i]; }
        return ADMM_OK;
    default:
        set_err("unknown vector id %d", which);
        return ADMM_ERR_INVALID_ARG;
    }
}

extern "C" int admm_get_csr(admm_handle *h, int32_t *row_ptr, int32_t *col)
{
    if (!h || !row_ptr || !col) { set_err("NULL argument"); return ADMM_ERR_INVALID_ARG; }
    const Range R = range_of(h, h->sel);
    const int nls = R.b1 - R.b0;
    for (int i = R.i0; i <= R.i1; ++i) row_ptr[i - R.i0] = h->row_ptr[i] - R.k0;
    for (int k = R.k0; k < R.k1; ++k) {
        const int e = h->col[k];
        col[k - R.k0] = e < 2 * h->nl ? e - 2 * R.b0 : 2 * nls + (e - 2 * h->nl - R.g0);
    }
    return ADMM_OK;
}

extern "C" int admm_get_stats(admm_handle *h, int64_t *out9)
{
    if (!h || !out9) { set_err("NULL argument"); return ADMM_ERR_INVALID_ARG; }
    int rc = sync_sc(h);
    if (rc != ADMM_OK) return rc;
    for (int k = 0; k < kNumStats; ++k) out9[k] = (int64_t)h->hctrl->stats[k];
    return ADMM_OK;
}

namespace {

// state arrays of a handle, in blob order
struct StatePart {
    double *dev;
    size_t n;
};

std::vector<StatePart> state_parts(admm_handle *h)
{
    const size_t nl = h->nl, ng = h->ng, nb = h->nb, ns = h->ns;
    return {{h->G.bx, 6 * nl}, {h->G.blt, 2 * nl}, {h->G.bt, 8 * nl}, {h->G.bu, 8 * nl},
            {h->G.gu, 2 * ng}, {h->G.bw, nb},      {h->G.bth, nb},    {h->G.sx, 2 * ns},
            {h->G.sz, 4 * ns}, {h->G.sy, 4 * ns},  {h->G.sl, 4 * ns}, {h->G.balpha, nl}};
}

constexpr int kScalarsPerScenario = 4;   // beta, total iterations, beta_used, pending
constexpr uint64_t kScenMagic = 0x41444d4d53433031ull;   // "ADMMSC01"

// The same arrays by index space, for the state of one scenario: rows of
// length nl (branches), ng (generators), nb (buses) or ns (slots).
enum Space { SP_BR = 0, SP_GEN, SP_BUS, SP_SLOT };
struct ScenPart {
    double *dev;
    int rows;
    Space sp;
};

std::vector<ScenPart> scenario_parts(admm_handle *h)
{
    const DevGrid &G = h->G;
    return {{G.bx, 6, SP_BR},   {G.blt, 2, SP_BR},   {G.bt, 8, SP_BR},   {G.bu, 8, SP_BR},
            {G.gu, 2, SP_GEN},  {G.bw, 1, SP_BUS},   {G.bth, 1, SP_BUS}, {G.sx, 2, SP_SLOT},
            {G.sz, 4, SP_SLOT}, {G.sy, 4, SP_SLOT},  {G.sl, 4, SP_SLOT}, {G.balpha, 1, SP_BR}};
}

// [offset, count) of scenario s and the row stride in each index space
void scen_range(const admm_handle *h, int s, Space sp, size_t &off, size_t &cnt, size_t &stride)
{
    const std::vector<int32_t> &o = sp == SP_BR ? h->br_off : sp == SP_GEN ? h->gen_off
                                  : sp == SP_BUS ? h->bus_off : h->slot_off;
    off = (size_t)o[s];
    cnt = (size_t)(o[s + 1] - o[s]);
    stride = sp == SP_BR ? h->nl : sp == SP_GEN ? h->ng : sp == SP_BUS ? h->nb : h->ns;
}

size_t scen_blob_bytes(admm_handle *h, int s)
{
    size_t n = 0;
    for (auto &p : scenario_parts(h)) {
        size_t off, cnt, stride;
        scen_range(h, s, p.sp, off, cnt, stride);
        n += (size_t)p.rows * cnt;
    }
    return 6 * sizeof(uint64_t) + kScalarsPerScenario * sizeof(double) + n * sizeof(double);
}

}  // namespace

extern "C" int admm_get_scenario_state(admm_handle *h, int32_t s, void *buf, size_t *len)
{
    NvtxRange nvtx_("admm_get_scenario_state");
    if (!h || !len || s < 0 || s >= h->S) { set_err("bad argument"); return ADMM_ERR_INVALID_ARG; }
    const size_t need = scen_blob_bytes(h, s);
    if (!buf) { *len = need; return ADMM_OK; }
    if (*len < need) { set_err("state buffer too small (%zu < %zu)", *len, need); return ADMM_ERR_INVALID_ARG; }
    int rc = sync_sc(h);
    if (rc != ADMM_OK) return rc;
    uint64_t *hdr = (uint64_t *)buf;
    hdr[0] = kScenMagic;
    hdr[1] = (uint64_t)(h->bus_off[s + 1] - h->bus_off[s]);
    hdr[2] = (uint64_t)(h->br_off[s + 1] - h->br_off[s]);
    hdr[3] = (uint64_t)(h->gen_off[s + 1] - h->gen_off[s]);
    hdr[4] = (uint64_t)(h->slot_off[s + 1] - h->slot_off[s]);
    hdr[5] = 0;
    double *sc = (double *)(hdr + 6);
    const SCtrl &c = h->hsc[s];
    sc[0] = c.beta;
    sc[1] = (double)c.total_iters;
    sc[2] = c.pending ? c.beta_used : 0.0;
    sc[3] = (double)c.pending;
    double *p = sc + kScalarsPerScenario;
    for (auto &pt : scenario_parts(h)) {
        size_t off, cnt, stride;
        scen_range(h, s, pt.sp, off, cnt, stride);
        for (int r = 0; r < pt.rows; ++r) {
            if (cnt)
                CK(cudaMemcpyAsync(p, pt.dev + r * stride + off, cnt * sizeof(double),
                                   cudaMemcpyDeviceToHost, h->stream));
            p += cnt;
        }
    }
    CK(cudaStreamSynchronize(h->stream));
    *len = need;
    return ADMM_OK;
}

extern "C" int admm_set_scenario_state(admm_handle *h, int32_t s, const void *buf, size_t len)
{
    NvtxRange nvtx_("admm_set_scenario_state");
    if (!h || !buf || s < 0 || s >= h->S) { set_err("bad argument"); return ADMM_ERR_INVALID_ARG; }
    const uint64_t *hdr = (const uint64_t *)buf;
    if (len != scen_blob_bytes(h, s) || len < 6 * sizeof(uint64_t) || hdr[0] != kScenMagic ||
        hdr[1] != (uint64_t)(h->bus_off[s + 1] - h->bus_off[s]) ||
        hdr[2] != (uint64_t)(h->br_off[s + 1] - h->br_off[s]) ||
        hdr[3] != (uint64_t)(h->gen_off[s + 1] - h->gen_off[s]) ||
        hdr[4] != (uint64_t)(h->slot_off[s + 1] - h->slot_off[s])) {
        set_err("scenario state blob does not match scenario %d of this handle", s);
        return ADMM_ERR_INVALID_ARG;
    }
    int rc = sync_sc(h);
    if (rc != ADMM_OK) return rc;
    SCtrl &c = h->hsc[s];
    if (c.active && !c.done) { set_err("scenario %d is running", s); return ADMM_ERR_INVALID_ARG; }
    const double *sc = (const double *)(hdr + 6);
    c.beta = sc[0];
    c.total_iters = (int32_t)sc[1];
    c.beta_used = sc[2];
    c.pending = (int32_t)sc[3];
    const double *p = sc + kScalarsPerScenario;
    for (auto &pt : scenario_parts(h)) {
        size_t off, cnt, stride;
        scen_range(h, s, pt.sp, off, cnt, stride);
        for (int r = 0; r < pt.rows; ++r) {
            if (cnt)
                CK(cudaMemcpyAsync(pt.dev + r * stride + off, p, cnt * sizeof(double),
                                   cudaMemcpyHostToDevice, h->stream));
            p += cnt;
        }
    }
    CK(cudaMemcpyAsync(h->G.sc + s, &c, sizeof(SCtrl), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return ADMM_OK;
}

extern "C" int admm_get_state(admm_handle *h, void *buf, size_t *len)
{
    NvtxRange nvtx_("admm_get_state");
    if (!h || !len) { set_err("NULL argument"); return ADMM_ERR_INVALID_ARG; }
    auto parts = state_parts(h);
    size_t n = 0;
    for (auto &p : parts) n += p.n;
    const size_t need = 5 * sizeof(uint64_t) + kScalarsPerScenario * (size_t)h->S * sizeof(double) +
                        n * sizeof(double);
    if (!buf) { *len = need; return ADMM_OK; }
    if (*len < need) { set_err("state buffer too small (%zu < %zu)", *len, need); return ADMM_ERR_INVALID_ARG; }
    int rc = sync_sc(h);
    if (rc != ADMM_OK) return rc;
    uint64_t *hdr = (uint64_t *)buf;
    hdr[0] = kStateMagic; hdr[1] = (uint64_t)h->nb; hdr[2] = (uint64_t)h->nl; hdr[3] = (uint64_t)h->ng;
    hdr[4] = (uint64_t)h->S;
    double *sc = (double *)(hdr + 5);
    for (int s = 0; s < h->S; ++s) {
        const SCtrl &c = h->hsc[s];
        sc[4 * s] = c.beta;
        sc[4 * s + 1] = (double)c.total_iters;
        sc[4 * s + 2] = c.pending ? c.beta_used : 0.0;
        sc[4 * s + 3] = (double)c.pending;
    }
    double *p = sc + kScalarsPerScenario * h->S;
    for (auto &pt : parts) {
        if (pt.n) CK(cudaMemcpyAsync(p, pt.dev, pt.n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        p += pt.n;
    }
    CK(cudaStreamSynchronize(h->stream));
    *len = need;
    return ADMM_OK;
}

extern "C" int admm_set_state(admm_handle *h, const void *buf, size_t len)
{
    NvtxRange nvtx_("admm_set_state");
    if (!h || !buf) { set_err("NULL argument"); return ADMM_ERR_INVALID_ARG; }
    auto parts = state_parts(h);
    size_t n = 0;
    for (auto &p : parts) n += p.n;
    const size_t need = 5 * sizeof(uint64_t) + kScalarsPerScenario * (size_t)h->S * sizeof(double) +
                        n * sizeof(double);
    const uint64_t *hdr = (const uint64_t *)buf;
    if (len != need || hdr[0] != kStateMagic || hdr[1] != (uint64_t)h->nb || hdr[2] != (uint64_t)h->nl ||
        hdr[3] != (uint64_t)h->ng || hdr[4] != (uint64_t)h->S) {
        set_err("state blob does not match this handle");
        return ADMM_ERR_INVALID_ARG;
    }
    int rc = sync_sc(h);
    if (rc != ADMM_OK) return rc;
    const double *sc = (const double *)(hdr + 5);
    for (int s = 0; s < h->S; ++s) {
        SCtrl &c = h->hsc[s];
        c.beta = sc[4 * s];
        c.total_iters = (int32_t)sc[4 * s + 1];
        c.beta_used = sc[4 * s + 2];
        c.pending = (int32_t)sc[4 * s + 3];
    }
    std::memset(h->hctrl->cls_count, 0, sizeof(h->hctrl->cls_count));   // queue order restarts
    const double *p = sc + kScalarsPerScenario * h->S;
    for (auto &pt : parts) {
        if (pt.n) CK(cudaMemcpyAsync(pt.dev, p, pt.n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        p += pt.n;
    }
    CK(cudaMemcpyAsync(h->G.sc, h->hsc, sizeof(SCtrl) * h->S, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->G.ctrl, h->hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return ADMM_OK;
}

namespace {

// every device region an iteration writes and a later iteration reads: the
// state arrays, the scheduling class lists and the control blocks
std::vector<std::pair<void *, size_t>> replay_parts(admm_handle *h)
{
    std::vector<std::pair<void *, size_t>> out;
    for (auto &p : state_parts(h)) out.push_back({p.dev, p.n * sizeof(double)});
    out.push_back({h->G.cls_list, 2 * (size_t)kClasses * h->nl * sizeof(int32_t)});
    out.push_back({h->G.ctrl, sizeof(Ctrl)});
    out.push_back({h->G.sc, (size_t)h->S * sizeof(SCtrl)});
    return out;
}

int replay_copy(admm_handle *h, char *snap, bool save)
{
    size_t off = 0;
    for (auto &p : replay_parts(h)) {
        if (p.second)
            CK(cudaMemcpyAsync(save ? (void *)(snap + off) : p.first, save ? p.first : (void *)(snap + off),
                               p.second, cudaMemcpyDeviceToDevice, h->stream));
        off += (p.second + 255) & ~(size_t)255;
    }
    return ADMM_OK;
}

}  // namespace

extern "C" int admm_autotune(admm_handle *h, int32_t iters, int32_t *blocks_out, int32_t *body_out,
                             double *ms_best, int32_t *lanes_out)
{
    NvtxRange nvtx_("admm_autotune");
    if (!h || iters < 1) { set_err("bad argument"); return ADMM_ERR_INVALID_ARG; }
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 152;
    cudaGetLastError();
    // (lanes per branch, blocks) candidates
    constexpr int kCand = 7;
    const int cand[kCand] = {sms / 2, (3 * sms) / 4, sms, (3 * sms) / 2, 2 * sms, sms, 2 * sms};
    const int clan[kCand] = {1, 1, 1, 1, 1, 2, 2};
    double tot[kCand] = {0, 0, 0, 0, 0, 0, 0};
    auto blocks_of = [&](int c) {
        const int need = branch_blocks_needed(h->nl, clan[c]);
        return cand[c] < need ? (cand[c] > 0 ? cand[c] : 1) : need;
    };
    // candidates that come out as the same launch (blocks capped at the
    // branches' need) are timed once: timing one shape several times and
    // keeping its best would favour it over shapes timed once
    bool dup[kCand];
    for (int c = 0; c < kCand; ++c) {
        dup[c] = false;
        for (int e = 0; e < c; ++e)
            dup[c] = dup[c] || (clan[e] == clan[c] && blocks_of(e) == blocks_of(c));
    }
    size_t bytes = 0;
    for (auto &p : replay_parts(h)) bytes += (p.second + 255) & ~(size_t)255;
    char *snap = nullptr;
    CK(cudaMalloc(&snap, bytes));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = replay_copy(h, snap, true);
    if (rc == ADMM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
        set_err("cudaEventCreate failed");
        rc = ADMM_ERR_CUDA;
    }
    cudaGraphConditionalHandle none = 0;
    // two passes, the second in reverse order; every candidate replays the
    // same `iters` iterations from the same saved state
    for (int pass = 0; pass < 2 && rc == ADMM_OK; ++pass) {
        for (int k = 0; k < kCand && rc == ADMM_OK; ++k) {
            const int c = pass == 0 ? k : kCand - 1 - k;
            if (dup[c]) continue;
            const int nbk = blocks_of(c);
            DevGrid G = h->G;
            G.nblk_branch = nbk;
            if ((rc = replay_copy(h, snap, false)) != ADMM_OK) break;
            if ((rc = slot_begin(h, 0, h->S, h->opts.rho_pq, h->opts.rho_va, 0.0, iters, 1)) != ADMM_OK) break;
            run_begin_kernel<<<1, 32, 0, h->stream>>>(h->G, iters);
            for (int it = 0; it < iters && rc == ADMM_OK; ++it) {
                float ms = 0.f;
                if (cudaEventRecord(e0, h->stream) != cudaSuccess) { rc = ADMM_ERR_CUDA; break; }
                launch_branch(clan[c], nbk, h->stream, G, h->O);
                if (cudaEventRecord(e1, h->stream) != cudaSuccess) { rc = ADMM_ERR_CUDA; break; }
                bus_dual_kernel<<<h->nblk_bus, kBusBlock, 0, h->stream>>>(h->G, h->O);
                control_kernel<<<1, 32, 0, h->stream>>>(h->G, none, 0);
                if ((rc = launch_check("autotune iteration")) != ADMM_OK) break;
                if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                    set_err("autotune timing failed");
                    rc = ADMM_ERR_CUDA;
                    break;
                }
                tot[c] += ms;
            }
        }
    }
    int best = 0;
    for (int c = 1; c < kCand; ++c)
        if (!dup[c] && tot[c] < tot[best]) best = c;
    const int nbk = blocks_of(best);
    if (rc == ADMM_OK) {
        h->nblk_branch = nbk;
        h->G.nblk_branch = nbk;
        h->opts.branch_blocks = nbk;
        h->lanes = clan[best];
        h->opts.lanes_per_branch = clan[best];
    }
    // graph shape: iterations per body of the WHILE node, timed through the
    // graph itself over 4 * iters iterations replayed from the same state
    constexpr int kBodyCand = 3;
    const int bc[kBodyCand] = {1, 2, 4};
    double bt[kBodyCand] = {0, 0, 0};
    bool tuned_body = false;
    if (rc == ADMM_OK && h->opts.use_graph) {
        for (int pass = 0; pass < 2 && rc == ADMM_OK; ++pass) {
            for (int k = 0; k < kBodyCand && rc == ADMM_OK; ++k) {
                const int c = pass == 0 ? k : kBodyCand - 1 - k;
                h->opts.graph_body_iters = bc[c];
                destroy_graph(h);
                if ((rc = build_graph(h)) != ADMM_OK) break;
                if ((rc = replay_copy(h, snap, false)) != ADMM_OK) break;
                if ((rc = slot_begin(h, 0, h->S, h->opts.rho_pq, h->opts.rho_va, 0.0, 4 * iters, 1)) != ADMM_OK)
                    break;
                float ms = 0.f;
                if (cudaEventRecord(e0, h->stream) != cudaSuccess) { rc = ADMM_ERR_CUDA; break; }
                if ((rc = run_async(h, 4 * iters)) != ADMM_OK) break;
                if (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                    set_err("autotune timing failed");
                    rc = ADMM_ERR_CUDA;
                    break;
                }
                bt[c] += ms;
            }
        }
        tuned_body = rc == ADMM_OK;
    }
    int bbest = 0;
    for (int c = 1; c < kBodyCand; ++c)
        if (bt[c] < bt[bbest]) bbest = c;
    h->opts.graph_body_iters = tuned_body ? bc[bbest] : 1;
    // leave the solve where it was
    if (rc == ADMM_OK) rc = replay_copy(h, snap, false);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess && rc == ADMM_OK) {
        set_err("autotune: %s", cudaGetErrorString(cudaGetLastError()));
        rc = ADMM_ERR_CUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(snap);
    if (h->opts.use_graph) {
        destroy_graph(h);
        if (build_graph(h) != ADMM_OK) {
            destroy_graph(h);
            cudaGetLastError();
            h->opts.use_graph = 0;
        }
    }
    if (rc != ADMM_OK) return rc;
    if (blocks_out) *blocks_out = nbk;
    if (body_out) *body_out = h->opts.graph_body_iters;
    if (lanes_out) *lanes_out = h->lanes;
    if (ms_best) *ms_best = tot[best] / (2.0 * iters);
    return ADMM_OK;
}

extern "C" int admm_profile_iterations(admm_handle *h, int32_t iters, double *ms_out)
{
    NvtxRange nvtx_("admm_profile_iterations");
    if (!h || !ms_out || iters < 1) { set_err("bad argument"); return ADMM_ERR_INVALID_ARG; }
    int rc = slot_begin(h, 0, h->S, h->opts.rho_pq, h->opts.rho_va, 0.0, iters, 1);
    if (rc != ADMM_OK) return rc;
    run_begin_kernel<<<1, 32, 0, h->stream>>>(h->G, iters);
    if ((rc = launch_check("run_begin_kernel")) != ADMM_OK) return rc;
    std::vector<cudaEvent_t> ev(2 * (size_t)iters + 1);
    for (auto &e : ev) CK(cudaEventCreate(&e));
    cudaGraphConditionalHandle none = 0;
    CK(cudaEventRecord(ev[0], h->stream));
    for (int it = 0; it < iters; ++it) {
        launch_branch(h->lanes, h->nblk_branch, h->stream, h->G, h->O);
        CK(cudaEventRecord(ev[2 * it + 1], h->stream));
        bus_dual_kernel<<<h->nblk_bus, kBusBlock, 0, h->stream>>>(h->G, h->O);
        control_kernel<<<1, 32, 0, h->stream>>>(h->G, none, 0);
        CK(cudaEventRecord(ev[2 * it + 2], h->stream));
    }
    flush_lambda_kernel<<<h->nblk_flush, 256, 0, h->stream>>>(h->G, h->O);
    clear_pending_kernel<<<(h->S + 255) / 256, 256, 0, h->stream>>>(h->G);
    if ((rc = launch_check("profiled iteration")) != ADMM_OK) return rc;
    CK(cudaStreamSynchronize(h->stream));
    double tb = 0.0, tu = 0.0;
    for (int it = 0; it < iters; ++it) {
        float a = 0.f, b = 0.f;
        CK(cudaEventElapsedTime(&a, ev[2 * it], ev[2 * it + 1]));
        CK(cudaEventElapsedTime(&b, ev[2 * it + 1], ev[2 * it + 2]));
        tb += a;
        tu += b;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    ms_out[0] = tb / iters;
    ms_out[1] = tu / iters;
    ms_out[2] = (tb + tu) / iters;
    return ADMM_OK;
}
