// Host side of the shearsim C ABI: simulation objects, device memory, CUDA
// graphs of a time step and of a solve, and the state-access calls.
//
// A time step is one CUDA graph: cell binning and sorting, pair search, the
// fused pair/assembly kernel, the solve (one cooperative persistent launch,
// FP64 or mixed; with SHEARSIM_PERSISTENT=0 the two-kernel iteration as a
// conditional WHILE node whose body holds an IF node for the true-residual
// check), the stress, and the position update.  The host launches nsteps
// graphs back to back and reads the device state once at the end.  If
// conditional graph nodes are unavailable the same kernels are launched from
// a host loop instead (SHEARSIM_HOST_LOOP=1 forces that mode).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace ss;


#include "sim_impl.cuh"

namespace ss_host {

std::string g_create_error;

Launch launch_of(const sp_sim* s, cudaStream_t st) { return Launch{st, s->num_sms}; }

bool mixed(const sp_sim* s) { return s->p.precision == SP_PREC_MIXED; }

bool warm_from_prev(const sp_sim* s) { return s->p.warm_start == SP_WARM_PREV || s->learned; }

template <class T>
int dev_alloc(sp_sim* s, T** ptr, size_t count)
{
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(T) * std::max<size_t>(count, 1));
    if (e != cudaSuccess) {
        s->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? SP_ERR_OOM : SP_ERR_CUDA;
    }
    *ptr = static_cast<T*>(q);
    return SP_OK;
}

namespace {
// Work arrays of xi = p(A) g for this simulation's sizes (the form of its solver).
int fdt_alloc(sp_sim* s, FdtBuffers& V)
{
    const size_t bytes = s->kp.mixed ? sizeof(float4) * 2 * (size_t)s->kp.npad : sizeof(double) * 3 * (size_t)s->kp.npad;
    int rc = SP_OK;
    auto A_ = [&](int r) { if (rc == SP_OK) rc = r; };
    for (auto& p : V.v) {
        char* q = nullptr;
        A_(dev_alloc(s, &q, bytes));
        p = q;
    }
    A_(dev_alloc(s, &V.cs, 2 + kFdtMaxDegree + 1));
    A_(dev_alloc(s, &V.csf, 2 + kFdtMaxDegree + 1));
    A_(dev_alloc(s, &V.bound, 1));
    return rc;
}

void fdt_free(FdtBuffers& V)
{
    for (auto& p : V.v) {
        cudaFree(p);
        p = nullptr;
    }
    cudaFree(V.cs);
    cudaFree(V.csf);
    cudaFree(V.bound);
    V = FdtBuffers{};
}
}  // namespace


void free_graphs(sp_sim* s)
{
    if (s->step_exec) cudaGraphExecDestroy(s->step_exec);
    if (s->step_graph) cudaGraphDestroy(s->step_graph);
    s->step_exec = nullptr;
    s->step_graph = nullptr;
    for (int k = 0; k < 2; ++k) {
        if (s->solve_exec[k]) cudaGraphExecDestroy(s->solve_exec[k]);
        if (s->solve_graph[k]) cudaGraphDestroy(s->solve_graph[k]);
        s->solve_exec[k] = nullptr;
        s->solve_graph[k] = nullptr;
    }
}

int alloc_pairs(sp_sim* s, long long cap)
{
    DevBuffers& B = s->B;
    cudaFree(B.col);
    cudaFree(B.val);
    cudaFree(B.val32);
    cudaFree(B.img);
    cudaFree(B.hcol);
    cudaFree(B.hval);
    cudaFree(B.hlo);
    B.hlo = nullptr;
    cudaFree(B.val32lo);
    B.val32lo = nullptr;
    B.col = nullptr;
    B.val = nullptr;
    B.val32 = nullptr;
    B.img = nullptr;
    B.hcol = nullptr;
    B.hval = nullptr;
    SS_TRY(dev_alloc(s, &B.col, (size_t)cap));
    SS_TRY(dev_alloc(s, &B.val, (size_t)cap));
    SS_TRY(dev_alloc(s, &B.val32, (size_t)cap));
    SS_TRY(dev_alloc(s, &B.img, (size_t)cap));
    s->kp.hcopy = 0;
    if (mixed(s)) {   // low parts of the weights; halo lists of the on-chip solve
        // systems small enough for the on-chip solve get a second region for
        // the lists of blocks whose entries cannot stay on chip, so that the
        // blocks can split the rows at any row (their halo lists then take
        // entry shares that do not follow the sliced layout's windows)
        const bool second = (long long)s->kp.n <= 2048ll * s->num_sms && 2 * cap < 0x7fffffffll;
        const size_t hcap = (size_t)cap * (second ? 2 : 1);
        SS_TRY(dev_alloc(s, &B.val32lo, (size_t)cap));
        SS_TRY(dev_alloc(s, &B.hcol, hcap));
        SS_TRY(dev_alloc(s, &B.hval, hcap));
        SS_TRY(dev_alloc(s, &B.hlo, hcap));
        if (second) s->kp.hcopy = cap;
    }
    s->nnz_cap = cap;
    s->st_host->nnz_cap = cap;
    SS_CUDA(cudaMemcpyAsync(&B.st->nnz_cap, &cap, sizeof(cap), cudaMemcpyHostToDevice, s->stream));
    return SP_OK;
}

int check_params(const sp_params* p, std::string& why)
{
    if (!p) { why = "params is NULL"; return SP_ERR_INVALID_ARG; }
    if (p->n < 2 || p->n > (1ll << 27)) { why = "n must be in [2, 2^27]"; return SP_ERR_INVALID_ARG; }
    if (!(p->rc > 0) || !(p->dt > 0) || !(p->zeta > 0) || !(p->kT >= 0) || !(p->alpha >= 0) ||
        !std::isfinite(p->kappa) || !std::isfinite(p->eps) || !(p->cg_tol > 0) || p->cg_max_iter < 1) {
        why = "rc, dt, zeta, cg_tol must be > 0; kT, alpha >= 0; kappa, eps finite; cg_max_iter >= 1";
        return SP_ERR_INVALID_ARG;
    }
    for (int a = 0; a < 3; ++a) {
        if (!(p->L[a] > 0) || !std::isfinite(p->L[a])) { why = "box edges must be > 0"; return SP_ERR_INVALID_ARG; }
        if (p->L[a] < 2.0 * p->rc) { why = "box edge below 2 r_c"; return SP_ERR_BOX_TOO_SMALL; }
    }
    if (p->precision != SP_PREC_FP64 && p->precision != SP_PREC_MIXED) { why = "unknown precision"; return SP_ERR_INVALID_ARG; }
    if (p->warm_start != SP_WARM_NONE && p->warm_start != SP_WARM_PREV) { why = "unknown warm start"; return SP_ERR_INVALID_ARG; }
    return SP_OK;
}

// lambda^2 = r_c^2 / (2 ln 20): the weight exp(-r^2 / 2 lambda^2) is 5 % at r_c.
double lambda2_of(double rc) { return rc * rc / (2.0 * std::log(20.0)); }

void derive(const sp_params& p, KParams& k, int npad)
{
    k.n = (int)p.n;
    k.npad = npad;
    for (int a = 0; a < 3; ++a) k.L[a] = p.L[a];
    k.rc2 = p.rc * p.rc;
    const double l2 = lambda2_of(p.rc);
    k.two_lambda2 = 2.0 * l2;
    k.w_scale = 256.0 / k.two_lambda2;
    k.pcfg = 0;   // tile configuration of the persistent solver (sp_autotune)
    k.res_smem = kResSmemBytes;
    k.alpha = p.alpha;
    k.mixed = p.precision == SP_PREC_MIXED ? 1 : 0;
    k.alpha_hi = (float)p.alpha;
    k.alpha_lo = (float)(p.alpha - (double)k.alpha_hi);
    k.zeta = p.zeta;
    k.kappa = p.kappa;
    k.dt = p.dt;
    k.c_ev = p.eps * 0.1 * p.kT / l2;          // (v/lambda^3) kT / lambda^2 with v/lambda^3 = 0.1
    k.noise_amp = std::sqrt(2.0 * p.zeta * p.kT / p.dt);
    auto split = [](double v, float& hi, float& lo) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
    };
    split(k.noise_amp / p.zeta, k.amp_z_hi, k.amp_z_lo);
    split(k.c_ev / p.zeta, k.cev_z_hi, k.cev_z_lo);
    split(p.kappa, k.kap_hi, k.kap_lo);
    split(0.5 * p.L[1], k.hly_hi, k.hly_lo);
    split(p.alpha * p.kappa * p.L[1], k.akl_hi, k.akl_lo);
    k.seed = p.seed;
    // cells: edge >= r_c (1 + 1e-9) so that rounding never moves a partner
    // within r_c out of the 3 x 3 x 3 block; in a sparse box the cells are
    // made coarser, so the cell index slots stay within a small multiple of n
    int nc[3];
    for (int a = 0; a < 3; ++a) {
        nc[a] = (int)std::floor(p.L[a] / (p.rc * (1.0 + 1e-9)));
        nc[a] = std::min(std::max(nc[a], 1), 4096);
    }
    auto slots = [&]() {
        long long t = 512;
        for (int a = 0; a < 3; ++a) t *= (nc[a] + 7) / 8;
        return t;
    };
    const long long slot_cap = std::min<long long>(std::max<long long>(8ll * p.n, 1ll << 15), 1ll << 30);
    while (slots() > slot_cap) {
        int a = 0;
        for (int b = 1; b < 3; ++b)
            if (nc[b] > nc[a]) a = b;
        nc[a] = std::max(3, nc[a] / 2);
    }
    for (int a = 0; a < 3; ++a) {
        k.nc[a] = nc[a];
        k.inv_cw[a] = (double)nc[a] / p.L[a];
        k.ntile[a] = (nc[a] + 7) / 8;
    }
    long long ncell = slots();
    if (k.nc[0] < 3 && k.nc[1] < 3 && k.nc[2] < 3) {
        k.nc[0] = k.nc[1] = k.nc[2] = 1;
        k.ntile[0] = k.ntile[1] = k.ntile[2] = 1;
        k.inv_cw[0] = 1.0 / p.L[0];
        k.inv_cw[1] = 1.0 / p.L[1];
        k.inv_cw[2] = 1.0 / p.L[2];
        ncell = 1;
    }
    k.ncell = (int)ncell;
    k.nslots = (k.n + 255) / 256 * 256;
    k.nchunks = k.nslots / 32;
    k.fast_cells = (k.nc[0] >= 3 && k.nc[1] >= 3 && k.nc[2] >= 3) ? 1 : 0;
    // FP32 pre-filter margin on |R|^2: 2^-24 (256 L r_c + 64 r_c^2) bounds the
    // FP32 rounding of positions, image shifts, differences, squares and sums
    const double Lmax = std::max(p.L[0], std::max(p.L[1], p.L[2]));
    const double margin = std::ldexp(256.0 * Lmax * p.rc + 64.0 * p.rc * p.rc, -24);
    k.rc2_lo = (float)(k.rc2 - margin);
    k.rc2_hi = (float)(k.rc2 + margin);
    for (int a = 0; a < 3; ++a) {
        k.Lf[a] = (float)p.L[a];
        k.Llo[a] = (float)(p.L[a] - (double)k.Lf[a]);
    }
    k.wsc_hi = (float)k.w_scale;
    k.wsc_lo = (float)(k.w_scale - (double)k.wsc_hi);
    k.tol2 = p.cg_tol * p.cg_tol;
    // mixed solver: each FP32 inner solve reduces the residual by 10^-4 before
    // the FP64 residual is recomputed (well above FP32 attainable accuracy)
    k.inner2 = 1e-8;
    k.max_iter = p.cg_max_iter;
    for (int a = 0; a < 3; ++a) {
        k.fix_inv[a] = 4294967296.0 / p.L[a];
        k.fix_scale[a] = (float)(p.L[a] / 4294967296.0);
    }
    k.w_exp2 = (float)(-1.4426950408889634 / k.two_lambda2);
    k.c_ev_f = (float)k.c_ev;
    k.za_f = (float)(k.zeta * k.alpha);
    k.kly_f = (float)(k.kappa * k.L[1]);
}

// --------------------------------------------------------------- enqueueing

long long enqueue_build(sp_sim* s, cudaStream_t cs, cudaStream_t side, cudaEvent_t* ev, bool split_x)
{
    KParams& P = s->kp;
    DevBuffers& B = s->B;
    Launch L = launch_of(s, cs);
    const bool warm = warm_from_prev(s);
    long long launches = 0;
    if (P.ncell == 1) {
        launch_identity_gather(P, B, warm, L);
        launches += 1;
    } else {
        launch_bin(P, B, L);
        launches += 1 + launch_scan(B.cell_count, B.cell_start, P.ncell, B.scan_tmp, 0, B.st, 0, L);
        launches += launch_scatter_sort_gather(P, B, warm, L);
    }
    if (side && ev && split_x) {   // x0 (just gathered) split into double-floats beside the search and assembly
        cudaEventRecord(ev[0], cs);
        cudaStreamWaitEvent(side, ev[0], 0);
        launch_cg_split_x(P, B, launch_of(s, side));
        cudaEventRecord(ev[1], side);
        launches += 1;
    }
    launches += launch_nbr_count(P, B, !s->use_inj && P.noise_amp != 0.0, L, side, (side && ev) ? ev + 2 : nullptr);
    launch_sell_plan(P, B, L);
    launches += 1 + launch_scan(B.chunk_len32, B.chunk_off, P.nchunks, B.scan_tmp, s->nnz_cap, B.st, 2, L);
    return launches;
}

// Conditional WHILE node holding one CG iteration, with an IF node for the
// true-residual check, appended to the graph being captured on cs.
int capture_cg_loop(sp_sim* s, cudaStream_t cs)
{
    KParams& P = s->kp;
    DevBuffers& B = s->B;
    const bool mx = mixed(s);
    cudaStreamCaptureStatus cst;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    SS_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphConditionalHandle h_loop;
    SS_CUDA(cudaGraphConditionalHandleCreate(&h_loop, g, 1u, cudaGraphCondAssignDefault));
    cudaGraphNodeParams wp = {cudaGraphNodeTypeConditional};
    wp.conditional.handle = h_loop;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    SS_CUDA(cudaGraphAddNode(&wnode, g, deps, nullptr, nd, &wp));
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    SS_CUDA(cudaStreamUpdateCaptureDependencies(cs, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));

    cudaStream_t bs = s->cap_stream[2];
    SS_CUDA(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    cudaGraphConditionalHandle h_check;
    SS_CUDA(cudaGraphConditionalHandleCreate(&h_check, body, 0u, cudaGraphCondAssignDefault));
    CgLaunch C{1, (unsigned long long)h_loop, (unsigned long long)h_check};
    launch_cg_spmv(P, B, mx, launch_of(s, bs));
    launch_cg_update(P, B, mx, C, launch_of(s, bs));
    cudaGraph_t bg = nullptr;
    SS_CUDA(cudaStreamGetCaptureInfo(bs, &cst, nullptr, &bg, &deps, nullptr, &nd));
    cudaGraphNodeParams ip = {cudaGraphNodeTypeConditional};
    ip.conditional.handle = h_check;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t inode;
    SS_CUDA(cudaGraphAddNode(&inode, bg, deps, nullptr, nd, &ip));
    cudaGraph_t ifbody = ip.conditional.phGraph_out[0];
    SS_CUDA(cudaStreamUpdateCaptureDependencies(bs, &inode, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaStream_t is = s->cap_stream[3];
    SS_CUDA(cudaStreamBeginCaptureToGraph(is, ifbody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    launch_cg_true_residual(P, B, mx, true, C, launch_of(s, is));
    SS_CUDA(cudaStreamEndCapture(is, &ifbody));
    SS_CUDA(cudaStreamEndCapture(bs, &body));
    return SP_OK;
}

// CG driven from the host: iterations in chunks, the device state polled
// between chunks (kernels after convergence return at once).
int host_cg_loop(sp_sim* s, long long* launches)
{
    KParams& P = s->kp;
    DevBuffers& B = s->B;
    const bool mx = mixed(s);
    CgLaunch C{0, 0, 0};
    Launch L = launch_of(s, s->stream);
    const int chunk = 8;
    for (int it = 0; it < P.max_iter + kMaxCgRestarts + chunk; it += chunk) {
        for (int k = 0; k < chunk; ++k) {
            launch_cg_spmv(P, B, mx, L);
            launch_cg_update(P, B, mx, C, L);
            launch_cg_true_residual(P, B, mx, false, C, L);
            *launches += cg_kernels_per_iteration(mx) + cg_kernels_per_check(mx);
        }
        SS_CUDA(cudaMemcpyAsync(s->st_host, B.st, sizeof(DevState), cudaMemcpyDeviceToHost, s->stream));
        SS_CUDA(cudaStreamSynchronize(s->stream));
        const DevState& h = *s->st_host;
        if (h.done || h.error || h.overflow) break;
    }
    return SP_OK;
}

// Everything of a solve after assembly: init, loop, finish, stress.
int enqueue_solve(sp_sim* s, cudaStream_t cs, bool from_x, bool in_graph, long long* launches, bool with_stress,
                  bool x_split)
{
    KParams& P = s->kp;
    DevBuffers& B = s->B;
    Launch L = launch_of(s, cs);
    if (mixed(s) && s->persistent && cg_persistent_on_chip(P, B, L)) {
        // the on-chip solve forms its initial residual itself (one pass over
        // its rows' entries, beside placing them in shared memory)
        KParams Pf = P;
        Pf.fused_init = from_x ? 2 : 1;
        if (from_x && !x_split) {
            launch_cg_split_x(P, B, L);
            *launches += 1;
        }
        SS_CUDA(launch_cg32_persistent(Pf, B, L));
        *launches += 1;
        launch_cg_finish(P, B, true, L);
        *launches += 1;
        if (with_stress) {
            launch_stress(P, B, true, L);
            *launches += 1;
        }
        return SP_OK;
    }
    if (!mixed(s) && s->persistent) {   // the FP64 solve in one cooperative launch
        SS_CUDA(launch_cg64_persistent(P, B, from_x ? 1 : 0, L));
        *launches += 1;
        launch_cg_finish(P, B, false, L);
        *launches += 1;
        if (with_stress) {
            launch_stress(P, B, false, L);
            *launches += 1;
        }
        return SP_OK;
    }
    *launches += launch_cg_init(P, B, from_x, mixed(s), L);
    if (mixed(s) && s->persistent) {
        SS_CUDA(launch_cg32_persistent(P, B, L));
        *launches += 1 + cg_persistent_prelaunches(P, B, L);
    } else if (in_graph) {
        SS_TRY(capture_cg_loop(s, cs));
    } else {
        SS_TRY(host_cg_loop(s, launches));
    }
    launch_cg_finish(P, B, mixed(s), L);
    *launches += 1;
    if (with_stress) {
        launch_stress(P, B, mixed(s), L);
        *launches += 1;
    }
    return SP_OK;
}

int capture_step_graph(sp_sim* s)
{
    free_graphs(s);
    cudaStream_t cs = s->cap_stream[0];
    cudaStream_t side = s->cap_stream[1];
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    for (cudaEvent_t& x : ev)
        if (cudaEventCreateWithFlags(&x, cudaEventDisableTiming) != cudaSuccess) {
            for (cudaEvent_t y : ev)
                if (y) cudaEventDestroy(y);
            s->err = "cudaEventCreateWithFlags failed";
            return SP_ERR_CUDA;
        }
    const bool warm = warm_from_prev(s);
    // the on-chip solve from the previous velocities: their split into
    // double-floats runs beside the pair search and the assembly
    const bool side_split = mixed(s) && s->persistent && warm && !s->learned &&
                            cg_persistent_on_chip(s->kp, s->B, launch_of(s, cs));
    SS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    long long launches = enqueue_build(s, cs, side, ev, side_split);
    launches += launch_nbr_fill(s->kp, s->B, true, s->use_inj, mixed(s), launch_of(s, cs));
    if (s->fdt_degree > 0)   // the right-hand side with A^(1/2)-correlated noise
        launches += enqueue_fdt_noise(s->kp, s->B, s->fdt, s->fdt_degree, s->use_inj, cs);
    if (s->learned) {
        launch_mp_infer(s->kp, s->B, s->mp, launch_of(s, cs));
        launches += mp_infer_launches();
    }
    if (side_split) cudaStreamWaitEvent(cs, ev[1], 0);
    int rc = enqueue_solve(s, cs, warm, true, &launches, false, side_split);
    // the stress and the position update read the step's state and write
    // different arrays: the stress runs on a second captured stream beside the
    // update, and the new image offset is committed after both
    if (rc == SP_OK) {
        cudaEventRecord(ev[4], cs);
        cudaStreamWaitEvent(side, ev[4], 0);
        launch_stress(s->kp, s->B, mixed(s), launch_of(s, side));
        cudaEventRecord(ev[5], side);
        launch_integrate(s->kp, s->B, launch_of(s, cs), false);
        cudaStreamWaitEvent(cs, ev[5], 0);
        launch_commit_step(s->B, launch_of(s, cs));
        launches += 3;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (rc != SP_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) {
        s->err = std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e);
        return SP_ERR_CUDA;
    }
    s->step_graph = g;
    SS_CUDA(cudaGraphInstantiate(&s->step_exec, g, 0));
    s->fixed_launches_step = launches;
    return SP_OK;
}

int capture_solve_graph(sp_sim* s, int from_x)
{
    cudaStream_t cs = s->cap_stream[0];
    SS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    long long launches = 0;
    int rc = enqueue_solve(s, cs, from_x != 0, true, &launches);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (rc != SP_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) {
        s->err = std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e);
        return SP_ERR_CUDA;
    }
    s->solve_graph[from_x] = g;
    SS_CUDA(cudaGraphInstantiate(&s->solve_exec[from_x], g, 0));
    s->fixed_launches_solve = launches;
    return SP_OK;
}

// The capture streams must wait for the simulation stream and vice versa:
// graphs are launched on the simulation stream, so no extra ordering is needed.

int read_state(sp_sim* s)
{
    SS_CUDA(cudaMemcpyAsync(s->st_host, s->B.st, sizeof(DevState), cudaMemcpyDeviceToHost, s->stream));
    SS_CUDA(cudaStreamSynchronize(s->stream));
    return SP_OK;
}

template <class T>
int write_field(sp_sim* s, T* dev_field, T value)
{
    SS_CUDA(cudaMemcpyAsync(dev_field, &value, sizeof(T), cudaMemcpyHostToDevice, s->stream));
    SS_CUDA(cudaStreamSynchronize(s->stream));
    return SP_OK;
}

int set_device(sp_sim* s)
{
    SS_CUDA(cudaSetDevice(s->p.device));
    return SP_OK;
}

// The message of a failure raised on the device (DevState::error).
const char* status_text(int status)
{
    switch (status) {
    case SP_ERR_NOT_CONVERGED: return "CG did not converge";
    case SP_ERR_NONFINITE: return "non-finite value in CG";
    case SP_ERR_TIMEOUT: return "a grid-barrier wait of the persistent solver ran past the wait limit";
    case SP_ERR_INVALID_ARG:
        return "positions must be finite and lie in [0, L) (the simulation's positions are undefined until "
               "valid ones are set)";
    default: return "device-side failure";
    }
}

// After a failed step or solve, clear the sticky flags so the simulation stays usable.
int clear_flags(sp_sim* s)
{
    DevState* d = s->B.st;
    SS_TRY(write_field(s, &d->error, 0));
    SS_TRY(write_field(s, &d->overflow, 0));
    // a persistent solve that stopped on an error may have left arrivals behind
    SS_TRY(write_field(s, &d->bar_count, 0u));
    SS_TRY(write_field(s, &d->bar_exit, 0u));
    return SP_OK;
}

int grow_pairs(sp_sim* s)
{
    long long need = s->st_host->nnz_slots;
    long long cap = std::max<long long>((long long)(need * 1.25) + 1024, s->nnz_cap * 3 / 2);
    if (cap > 0x7fffffffll) {
        s->err = "pair count exceeds 2^31";
        return SP_ERR_OOM;
    }
    SS_CUDA(cudaStreamSynchronize(s->stream));
    free_graphs(s);
    SS_TRY(alloc_pairs(s, cap));
    SS_TRY(write_field(s, &s->B.st->overflow, 0));
    return SP_OK;
}

int ensure_step_graph(sp_sim* s)
{
    if (s->host_loop || s->step_exec) return SP_OK;
    int rc = capture_step_graph(s);
    if (rc != SP_OK) {
        // conditional graph nodes unavailable: fall back to the host-driven loop
        cudaGetLastError();
        free_graphs(s);
        s->host_loop = true;
        std::fprintf(stderr, "shearsim: CUDA graph capture failed (%s); using host-driven CG loop\n",
                     s->err.c_str());
    }
    return SP_OK;
}

int do_build(sp_sim* s)
{
    for (int attempt = 0; attempt < 4; ++attempt) {
        long long launches = enqueue_build(s, s->stream);
        (void)launches;
        launch_nbr_fill(s->kp, s->B, false, s->use_inj, mixed(s), launch_of(s, s->stream));
        SS_TRY(read_state(s));
        if (!s->st_host->overflow) break;
        SS_TRY(grow_pairs(s));
    }
    if (s->st_host->overflow) {
        s->err = "pair capacity could not be grown";
        return SP_ERR_OOM;
    }
    // the new cell order becomes the state order
    const size_t np = (size_t)s->kp.npad;
    SS_CUDA(cudaMemcpyAsync(s->B.pos_s, s->B.pos_w, sizeof(double) * 3 * np, cudaMemcpyDeviceToDevice, s->stream));
    SS_CUDA(cudaMemcpyAsync(s->B.id_s, s->B.id_w, sizeof(int) * s->kp.n, cudaMemcpyDeviceToDevice, s->stream));
    SS_CUDA(cudaMemcpyAsync(s->B.v_s, s->B.x, sizeof(double) * 3 * np, cudaMemcpyDeviceToDevice, s->stream));
    SS_CUDA(cudaStreamSynchronize(s->stream));
    s->built = true;
    s->assembled = false;
    return SP_OK;
}

}  // namespace ss_host

using namespace ss_host;

// Error text of calls that have no simulation object (creation, the
// allocation-free solve); sp_last_error(NULL) returns it.
std::string& sp_global_error() { return g_create_error; }

// ======================================================================= ABI

extern "C" {

double sp_kappa_from_kappa_tau(double kappa_tau, double rc, double zeta, double kT)
{
    if (!(kT > 0)) return NAN;
    const double tau = lambda2_of(rc) * zeta / kT;   // Rouse time, §Method
    return kappa_tau / tau;
}

const char* sp_last_error(const sp_sim* s)
{
    return s ? s->err.c_str() : g_create_error.c_str();
}

int sp_sim_destroy(sp_sim* s)
{
    if (!s) return SP_OK;
    cudaSetDevice(s->p.device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    free_graphs(s);
    DevBuffers& B = s->B;
    vc_free(s->vc);
    fdt_free(s->fdt);
    void* ptrs[] = {B.pos_s, B.id_s, B.v_s, B.pos_w, B.pos32, B.id_w, B.cell_of, B.slot, B.perm,
                    B.cell_count, B.cell_start, B.row_cnt, B.slot_row, B.row_slot, B.chunk_len32,
                    B.chunk_off, B.col, B.img, B.val, B.val32, B.val32lo, B.hcol, B.hval, B.diag, B.partials_df,
                    B.diag32lo, B.bdf, B.xdf, B.rdf, B.rlo, B.hlo,
                    B.dinv, B.diag32, B.dinv32, B.b, B.x, B.r, B.p, B.q, B.z, B.s64, B.r4, B.p4, B.q4, B.d4,
                    B.posfix, B.res_hist, B.xi_inj, B.exp_tab, B.exp_tab_df, B.rng_tab, B.pos32lo, B.cand_j, B.cand_img, B.noise3, B.partials, B.scan_tmp, B.stage, B.st};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (s->mp_alloc) {
        MpBuffers& M = s->mp;
        void* mps[] = {M.x0, M.a0, M.y, M.a1, M.dy, M.g1, M.master, M.m, M.v, M.grad, M.gpart, M.dpart, M.wb, M.scal,
                       M.part, M.ticket};
        for (void* q : mps)
            if (q) cudaFree(q);
    }
    if (s->st_host) cudaFreeHost(s->st_host);
    if (s->fcg) cudaFree(s->fcg);
    for (auto& c : s->cap_stream)
        if (c) cudaStreamDestroy(c);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return SP_OK;
}

int sp_sim_create(const sp_params* p, const double* pos_host, sp_sim** out)
{
    g_create_error.clear();
    if (!out) {
        g_create_error = "out is NULL";
        return SP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    std::string why;
    int rc = check_params(p, why);
    if (rc != SP_OK) {
        g_create_error = why;
        return rc;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || p->device < 0 || p->device >= ndev) {
        cudaGetLastError();
        g_create_error = "no CUDA device with the requested ordinal";
        return SP_ERR_NO_DEVICE;
    }
    sp_sim* s = new sp_sim();
    s->p = *p;
    auto fail = [&](int code) {
        g_create_error = s->err;
        sp_sim_destroy(s);
        return code;
    };
    if (cudaSetDevice(p->device) != cudaSuccess) {
        s->err = "cudaSetDevice failed";
        return fail(SP_ERR_CUDA);
    }
    cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    cg_prepare();
    if (s->num_sms < 1) s->num_sms = 1;
    const char* hl = std::getenv("SHEARSIM_HOST_LOOP");
    s->host_loop = hl && hl[0] == '1';
    const char* pe = std::getenv("SHEARSIM_PERSISTENT");
    s->persistent = !(pe && pe[0] == '0');
    if (p->stream) {
        s->stream = (cudaStream_t)p->stream;
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            s->err = "cudaStreamCreate failed";
            return fail(SP_ERR_CUDA);
        }
        s->own_stream = true;
    }
    for (auto& c : s->cap_stream) {
        if (cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking) != cudaSuccess) {
            s->err = "cudaStreamCreate failed";
            return fail(SP_ERR_CUDA);
        }
    }
    const int n = (int)p->n;
    const int npad = (n + 63) / 64 * 64;
    derive(*p, s->kp, npad);
    // a smaller shared-memory budget for the on-chip solve (its entries then
    // fit on fewer SMs): only to exercise the fallback of blocks that do not fit
    if (const char* rsm = std::getenv("SHEARSIM_RESIDENT_SMEM"))
        s->kp.res_smem = std::min(std::max(std::atoi(rsm), 0), kResSmemBytes);
    DevBuffers& B = s->B;
    const size_t v3 = 3 * (size_t)npad;
    int a = SP_OK;
    auto A = [&](int r) { if (a == SP_OK) a = r; };
    A(dev_alloc(s, &B.pos_s, v3));
    A(dev_alloc(s, &B.pos_w, v3));
    A(dev_alloc(s, &B.pos32, v3));
    A(dev_alloc(s, &B.pos32lo, v3));
    A(dev_alloc(s, &B.v_s, v3));
    A(dev_alloc(s, &B.id_s, n));
    A(dev_alloc(s, &B.id_w, n));
    A(dev_alloc(s, &B.cell_of, n));
    A(dev_alloc(s, &B.slot, n));
    A(dev_alloc(s, &B.perm, n));
    A(dev_alloc(s, &B.cell_count, s->kp.ncell));
    A(dev_alloc(s, &B.cell_start, (size_t)s->kp.ncell + 1));
    A(dev_alloc(s, &B.row_cnt, n));
    A(dev_alloc(s, &B.cand_j, (size_t)kCandCap * npad));
    A(dev_alloc(s, &B.noise3, v3));
    A(dev_alloc(s, &B.cand_img, (size_t)kCandCap * npad));
    A(dev_alloc(s, &B.slot_row, (size_t)s->kp.nslots));
    A(dev_alloc(s, &B.row_slot, n));
    A(dev_alloc(s, &B.chunk_len32, (size_t)s->kp.nchunks));
    A(dev_alloc(s, &B.chunk_off, (size_t)s->kp.nchunks + 1));
    A(dev_alloc(s, &B.diag, n));
    A(dev_alloc(s, &B.dinv, n));
    A(dev_alloc(s, &B.diag32, n));
    A(dev_alloc(s, &B.dinv32, n));
    A(dev_alloc(s, &B.b, v3));
    A(dev_alloc(s, &B.x, v3));
    A(dev_alloc(s, &B.r, v3));
    A(dev_alloc(s, &B.p, v3));
    A(dev_alloc(s, &B.q, v3));
    A(dev_alloc(s, &B.z, v3));
    if (!mixed(s)) A(dev_alloc(s, &B.s64, 2 * v3));
    A(dev_alloc(s, &B.r4, (size_t)npad));
    if (mixed(s)) {   // double-float forms of the mixed solver's true residuals
        A(dev_alloc(s, &B.diag32lo, (size_t)npad));
        A(dev_alloc(s, &B.bdf, 2 * (size_t)npad));
        A(dev_alloc(s, &B.xdf, 2 * (size_t)npad));
        A(dev_alloc(s, &B.rdf, 2 * (size_t)npad));
        A(dev_alloc(s, &B.rlo, (size_t)s->num_sms * kResLoStride));
        A(dev_alloc(s, &B.posfix, (size_t)npad));
        A(dev_alloc(s, &B.res_hist, (size_t)s->kp.nslots));
    }
    A(dev_alloc(s, &B.p4, (size_t)npad));
    A(dev_alloc(s, &B.q4, (size_t)npad));
    A(dev_alloc(s, &B.d4, (size_t)npad));
    A(dev_alloc(s, &B.partials, 8 * (size_t)kMaxPartials));
    A(dev_alloc(s, &B.partials_df, 4 * (size_t)kMaxPartials));
    A(dev_alloc(s, &B.exp_tab, (size_t)kExpTab));
    A(dev_alloc(s, &B.exp_tab_df, (size_t)kExpTab));
    A(dev_alloc(s, &B.rng_tab, (size_t)kRngTab));
    A(dev_alloc(s, &B.scan_tmp, (size_t)(std::max(std::max(n, s->kp.ncell), s->kp.nchunks) / 4096 + 2)));
    A(dev_alloc(s, &B.stage, 3 * (size_t)n));
    A(dev_alloc(s, &B.st, 1));
    if (a != SP_OK) return fail(a);
    if (cudaMallocHost(&s->st_host, sizeof(DevState)) != cudaSuccess) {
        s->err = "cudaMallocHost failed";
        return fail(SP_ERR_OOM);
    }
    std::memset(s->st_host, 0, sizeof(DevState));
    s->st_host->noise_step = -1;   // no normals drawn yet
    s->st_host->bar_timeout_ns = kDefaultWaitLimitNs;
    if (cudaMemcpyAsync(B.st, s->st_host, sizeof(DevState), cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
        cudaMemsetAsync(B.v_s, 0, sizeof(double) * v3, s->stream) != cudaSuccess ||
        cudaMemsetAsync(B.x, 0, sizeof(double) * v3, s->stream) != cudaSuccess ||
        cudaMemsetAsync(B.pos_s, 0, sizeof(double) * v3, s->stream) != cudaSuccess ||
        cudaMemsetAsync(B.pos_w, 0, sizeof(double) * v3, s->stream) != cudaSuccess ||
        upload_exp_table(B.exp_tab, B.exp_tab_df, s->stream) != cudaSuccess ||
        upload_rng_table(B.rng_tab, s->stream) != cudaSuccess) {
        s->err = "initialising device state failed";
        return fail(SP_ERR_CUDA);
    }
    rc = alloc_pairs(s, std::max<long long>(1024, 20ll * n));
    if (rc != SP_OK) return fail(rc);
    if (pos_host) {
        // identity order: row k holds particle k
        std::vector<int> ids(n);
        for (int i = 0; i < n; ++i) ids[i] = i;
        for (int i = 0; i < 3 * n; ++i) {
            const double v = pos_host[i];
            const double L = p->L[i % 3];
            if (!(v >= 0.0) || !(v < L)) {
                s->err = "initial positions must lie in [0, L)";
                return fail(SP_ERR_INVALID_ARG);
            }
        }
        if (cudaMemcpy(B.id_s, ids.data(), sizeof(int) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(B.stage, pos_host, sizeof(double) * 3 * n, cudaMemcpyHostToDevice) != cudaSuccess) {
            s->err = "copying initial positions failed";
            return fail(SP_ERR_CUDA);
        }
        launch_gather_by_id(B.stage, B.id_s, n, npad, B.pos_s, s->stream);
    } else {
        launch_uniform_positions(s->kp, B, launch_of(s, s->stream));
    }
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) {
        s->err = std::string("initialisation: ") + cudaGetErrorString(cudaGetLastError());
        return fail(SP_ERR_CUDA);
    }
    *out = s;
    return SP_OK;
}

int sp_build_neighbors(sp_sim* s)
{
    if (!s) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    return do_build(s);
}

int sp_assemble(sp_sim* s)
{
    if (!s) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    if (!s->built) {
        s->err = "sp_assemble needs sp_build_neighbors after the last position change";
        return SP_ERR_INVALID_ARG;
    }
    launch_assemble_only(s->kp, s->B, s->use_inj, mixed(s), launch_of(s, s->stream));
    SS_CUDA(cudaGetLastError());
    SS_CUDA(cudaStreamSynchronize(s->stream));
    s->assembled = true;
    return SP_OK;
}

int sp_solve_velocities(sp_sim* s, const double* v0_dev, sp_solve_info* info)
{
    if (!s) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    if (!s->assembled) {
        s->err = "sp_solve_velocities needs sp_assemble first";
        return SP_ERR_INVALID_ARG;
    }
    const int n = s->kp.n;
    const size_t np = (size_t)s->kp.npad;
    int from_x = 0;
    if (v0_dev) {
        for (int a = 0; a < 3; ++a)
            SS_CUDA(cudaMemcpyAsync(s->B.x + a * np, v0_dev + (size_t)a * n, sizeof(double) * n,
                                    cudaMemcpyDeviceToDevice, s->stream));
        from_x = 1;
    } else if (warm_from_prev(s)) {
        from_x = 1;   // x holds the previous velocities (gathered by the build) or the network's guess
    }
    long long launches = 0;
    if (!s->host_loop && !s->solve_exec[from_x]) {
        if (capture_solve_graph(s, from_x) != SP_OK) {
            cudaGetLastError();
            std::fprintf(stderr, "shearsim: solve graph capture failed (%s); using host-driven CG loop\n",
                         s->err.c_str());
            free_graphs(s);
            s->host_loop = true;
        }
    }
    if (s->host_loop) {
        SS_TRY(enqueue_solve(s, s->stream, from_x != 0, false, &launches));
    } else {
        SS_CUDA(cudaGraphLaunch(s->solve_exec[from_x], s->stream));
    }
    SS_TRY(read_state(s));
    const DevState& h = *s->st_host;
    int status = h.error ? h.error : (h.overflow ? SP_ERR_OOM : h.status);
    if (info) {
        info->status = status;
        info->iterations = h.iter;
        info->residual = h.last_res;
        info->bnorm = std::sqrt(h.bnorm2);
        info->offchip_blocks = h.res_offchip;
        info->host_driven = s->host_loop ? 1 : 0;
    }
    SS_CUDA(cudaMemcpyAsync(s->B.v_s, s->B.x, sizeof(double) * 3 * np, cudaMemcpyDeviceToDevice, s->stream));
    if (h.error) {
        SS_TRY(clear_flags(s));
        s->err = status_text(status);
    }
    SS_CUDA(cudaStreamSynchronize(s->stream));
    return status;
}

namespace {
// nsteps steps; with pos_out, the positions after them are copied out (by
// particle id) in the same stream before the one synchronisation that reads
// the step statistics (again after a pair-storage regrowth).
int run_steps(sp_sim* s, int32_t nsteps, double* pos_out, sp_step_info* info)
{
    SS_TRY(ensure_step_graph(s));
    launch_reset_step_stats(s->B.st, s->stream);
    long long launches = 1;
    long long done = 0;
    int status = SP_OK;
    for (int guard = 0; done < nsteps && guard < 8; ++guard) {
        const long long todo = nsteps - done;
        if (s->host_loop) {
            for (long long k = 0; k < todo; ++k) {
                launches += enqueue_build(s, s->stream);
                launches += launch_nbr_fill(s->kp, s->B, true, s->use_inj, mixed(s), launch_of(s, s->stream));
                if (s->fdt_degree > 0)
                    launches += enqueue_fdt_noise(s->kp, s->B, s->fdt, s->fdt_degree, s->use_inj, s->stream);
                if (s->learned) {
                    launch_mp_infer(s->kp, s->B, s->mp, launch_of(s, s->stream));
                    launches += mp_infer_launches();
                }
                SS_TRY(enqueue_solve(s, s->stream, warm_from_prev(s), false, &launches));
                launch_integrate(s->kp, s->B, launch_of(s, s->stream));
                launches += 2;   // the update and the commit of the new offset
                SS_TRY(read_state(s));
                if (s->st_host->error || s->st_host->overflow) break;
            }
        } else {
            for (long long k = 0; k < todo; ++k) SS_CUDA(cudaGraphLaunch(s->step_exec, s->stream));
        }
        if (pos_out) {
            launch_scatter_by_id(s->B.pos_s, s->kp.npad, s->B.id_s, s->kp.n, s->B.stage, s->stream);
            SS_CUDA(cudaMemcpyAsync(pos_out, s->B.stage, sizeof(double) * 3 * s->kp.n, cudaMemcpyDeviceToHost,
                                    s->stream));
        }
        SS_TRY(read_state(s));
        done = s->st_host->steps_in_call;
        if (s->st_host->overflow) {
            SS_TRY(grow_pairs(s));
            SS_TRY(ensure_step_graph(s));
            continue;
        }
        if (s->st_host->error) {
            status = s->st_host->error;
            s->err = status_text(status);
            SS_TRY(clear_flags(s));
            break;
        }
    }
    const DevState& h = *s->st_host;
    if (!s->host_loop) {
        launches += h.steps_in_call * s->fixed_launches_step;
        if (!s->persistent)
            launches += h.iter_sum * cg_kernels_per_iteration(mixed(s)) + h.true_checks * cg_kernels_per_check(mixed(s));
    }
    if (info) {
        info->status = status;
        info->max_iterations = h.iter_max;
        info->steps_done = h.steps_in_call;
        info->cg_iterations = h.iter_sum;
        info->last_residual = h.last_res;
        info->stress_xy = h.stress_xy;
        info->kernel_launches = launches;
        info->delta = h.delta;
        info->step = h.step;
        info->host_driven = s->host_loop ? 1 : 0;
    }
    s->built = false;
    s->assembled = false;
    if (status == SP_OK && h.steps_in_call < nsteps) {
        s->err = "steps stopped early";
        return SP_ERR_CUDA;
    }
    return status;
}
}  // namespace

int64_t sp_state_record_bytes(void) { return (int64_t)sizeof(DevState); }

int sp_step(sp_sim* s, int32_t nsteps, sp_step_info* info)
{
    if (!s || nsteps < 0) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    return run_steps(s, nsteps, nullptr, info);
}

int sp_step_host(sp_sim* s, const double* pos_in, double delta, int32_t nsteps, double* pos_out,
                 sp_step_info* info)
{
    if (!s || !pos_in || !pos_out || nsteps < 0) return SP_ERR_INVALID_ARG;
    if (!(delta >= 0.0) || !(delta < s->p.L[0])) {
        s->err = "delta must lie in [0, L_x)";
        return SP_ERR_INVALID_ARG;
    }
    SS_TRY(set_device(s));
    // positions by particle id into the state order; the offset through the
    // pinned state mirror (an asynchronous copy, read before the mirror is
    // next written by the statistics read-back in the same stream)
    SS_CUDA(cudaMemcpyAsync(s->B.stage, pos_in, sizeof(double) * 3 * s->kp.n, cudaMemcpyHostToDevice, s->stream));
    launch_gather_positions(s->B.stage, s->B.id_s, s->kp.n, s->kp.npad, s->B.pos_s, s->kp, s->B.st, s->stream);
    s->st_host->delta = delta;
    SS_CUDA(cudaMemcpyAsync(&s->B.st->delta, &s->st_host->delta, sizeof(double), cudaMemcpyHostToDevice, s->stream));
    s->built = false;
    s->assembled = false;
    return run_steps(s, nsteps, pos_out, info);
}

int sp_profile_step(sp_sim* s, sp_kernel_profile* out)
{
    if (!s || !out) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    std::memset(out, 0, sizeof(*out));
    KParams& P = s->kp;
    DevBuffers& B = s->B;
    const bool mx = mixed(s);
    Launch L = launch_of(s, s->stream);
    CgLaunch C{0, 0, 0};
    std::vector<cudaEvent_t> ev;
    std::vector<int> cls;   // class of the interval ending at each event
    auto mark = [&](int c) -> int {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return SP_ERR_CUDA;
        cudaEventRecord(e, s->stream);
        ev.push_back(e);
        cls.push_back(c);
        return SP_OK;
    };
    enum { START = -1, SORT = 0, SPMV, UPDATE, TRUE_RES, DIRECTION, OTHER, COUNT, FILL, PERSIST, INIT, STRESS,
           INTEGRATE, MPNN, ASSEMBLE };
    launch_reset_step_stats(B.st, s->stream);
    int rc = mark(START);
    if (rc == SP_OK) {
        const bool warm = s->p.warm_start == SP_WARM_PREV;
        if (P.ncell == 1) {
            launch_identity_gather(P, B, warm, L);
        } else {
            launch_bin(P, B, L);
            launch_scan(B.cell_count, B.cell_start, P.ncell, B.scan_tmp, 0, B.st, 0, L);
            launch_scatter_sort_gather(P, B, warm, L);
        }
        mark(SORT);
        launch_nbr_count(P, B, !s->use_inj && P.noise_amp != 0.0, L);
        launch_sell_plan(P, B, L);
        launch_scan(B.chunk_len32, B.chunk_off, P.nchunks, B.scan_tmp, s->nnz_cap, B.st, 2, L);
        mark(COUNT);
        launch_assemble_only(P, B, s->use_inj, mx, L);   // places the collected pairs and assembles
        rc = mark(ASSEMBLE);
        if (rc == SP_OK && s->learned) {
            launch_mp_infer(P, B, s->mp, L);
            rc = mark(MPNN);
        }
    }
    const bool pers = s->persistent;
    // as a step runs it: the on-chip solve forms its initial residual itself
    // (init_ms then holds only the split of x0 into double-floats)
    const bool fused = pers && cg_persistent_on_chip(P, B, L);
    if (rc == SP_OK && pers && !mx) {   // the FP64 solve in one cooperative launch (it forms r itself)
        rc = mark(INIT);
        if (rc == SP_OK && launch_cg64_persistent(P, B, warm_from_prev(s) ? 1 : 0, L) != cudaSuccess) rc = SP_ERR_CUDA;
        if (rc == SP_OK) rc = mark(PERSIST);
        out->persistent_blocks = cg64_persistent_grid(P, L);
        out->persistent_init = 1;
    }
    if (rc == SP_OK && (!pers || mx)) {
        if (!fused)
            launch_cg_init(P, B, warm_from_prev(s), mx, L);
        else if (warm_from_prev(s))
            launch_cg_split_x(P, B, L);
        rc = mark(INIT);
    }
    if (rc == SP_OK && pers && mx) {
        KParams Pf = P;
        Pf.fused_init = fused ? (warm_from_prev(s) ? 2 : 1) : 0;
        if (launch_cg32_persistent(Pf, B, L) != cudaSuccess) rc = SP_ERR_CUDA;
        if (rc == SP_OK) rc = mark(PERSIST);
        out->persistent_blocks = cg_persistent_grid(P, B, L);
        out->persistent_init = fused ? 1 : 0;
    }
    for (int it = 0; rc == SP_OK && !pers && it < P.max_iter + kMaxCgRestarts + 8; ++it) {
        launch_cg_spmv(P, B, mx, L);
        mark(SPMV);
        launch_cg_update(P, B, mx, C, L);
        rc = mark(UPDATE);
        if (rc != SP_OK) break;
        rc = read_state(s);
        if (rc != SP_OK) break;
        if (s->st_host->check_true) {
            launch_cg_true_residual(P, B, mx, false, C, L);
            rc = mark(TRUE_RES);
            if (rc != SP_OK) break;
            rc = read_state(s);
            if (rc != SP_OK) break;
        }
        const DevState& h = *s->st_host;
        if (h.done || h.error || h.overflow) break;
    }
    if (rc == SP_OK) {
        launch_cg_finish(P, B, mx, L);
        mark(OTHER);
        launch_stress(P, B, mixed(s), L);
        mark(STRESS);
        launch_integrate(P, B, L);
        rc = mark(INTEGRATE);
    }
    if (rc == SP_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = SP_ERR_CUDA;
    if (rc == SP_OK) rc = read_state(s);
    // back-to-back launches of the two loop kernels on the system just solved
    // (probe mode: same work, solver scalars untouched), one event pair each
    if (rc == SP_OK && !s->st_host->error && !s->st_host->overflow) {
        const int reps = 20;
        cudaEvent_t e[3];
        for (auto& x : e) cudaEventCreate(&x);
        cudaEventRecord(e[0], s->stream);
        for (int k = 0; k < reps; ++k) launch_cg_spmv(P, B, mx, L, 1);
        cudaEventRecord(e[1], s->stream);
        for (int k = 0; k < reps; ++k) launch_cg_update(P, B, mx, C, L, 1);
        cudaEventRecord(e[2], s->stream);
        if (cudaEventSynchronize(e[2]) == cudaSuccess) {
            float a = 0.f, b = 0.f;
            cudaEventElapsedTime(&a, e[0], e[1]);
            cudaEventElapsedTime(&b, e[1], e[2]);
            out->spmv_probe_ms = a / reps;
            out->update_probe_ms = b / reps;
            out->probe_reps = reps;
        } else {
            rc = SP_ERR_CUDA;
        }
        for (auto& x : e) cudaEventDestroy(x);
    }
    double* acc[] = {&out->sort_ms, &out->spmv_ms, &out->update_ms, &out->true_residual_ms,
                     &out->direction_ms, &out->other_ms, &out->count_ms, &out->fill_ms, &out->persistent_ms,
                     &out->init_ms, &out->stress_ms, &out->integrate_ms, &out->mpnn_ms,
                     &out->assemble_ms};
    for (size_t k = 1; rc == SP_OK && k < ev.size(); ++k) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[k - 1], ev[k]);
        *acc[cls[k]] += ms;
    }
    for (auto e : ev) cudaEventDestroy(e);
    if (rc != SP_OK) {
        if (s->err.empty()) s->err = "profiling step failed";
        return rc;
    }
    out->build_ms = out->sort_ms + out->count_ms + out->fill_ms + out->assemble_ms;
    out->other_ms += out->init_ms + out->stress_ms + out->integrate_ms;
    const DevState& h = *s->st_host;
    if (h.overflow) {
        // the pair storage was too small for this step: grow it and report the failure
        SS_TRY(grow_pairs(s));
        s->err = "pair storage grown during profiling; repeat the call";
        return SP_ERR_OOM;
    }
    out->cg_iterations = h.iter;
    out->spmv_launches = h.iter;
    out->update_launches = h.iter;
    out->direction_launches = 0;   // fused into the SpMV kernel
    out->true_residual_launches = pers ? 0 : (int)h.true_checks * cg_kernels_per_check(mx);
    out->true_checks = (int)h.true_checks;
    if (pers) {
        out->spmv_launches = 0;
        out->update_launches = 0;
    }
    out->n = P.n;
    out->nnz = h.nnz;
    out->nnz_slots = h.nnz_slots;
    out->precision = s->p.precision;
    s->built = false;
    s->assembled = false;
    if (h.error) {
        int status = h.error;
        SS_TRY(clear_flags(s));
        return status;
    }
    return SP_OK;
}

int sp_stress_xy(sp_sim* s, double* sigma)
{
    if (!s || !sigma) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    SS_TRY(read_state(s));
    *sigma = s->st_host->stress_xy;
    return SP_OK;
}

int sp_get_positions(sp_sim* s, double* pos_host)
{
    if (!s || !pos_host) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    launch_scatter_by_id(s->B.pos_s, s->kp.npad, s->B.id_s, s->kp.n, s->B.stage, s->stream);
    SS_CUDA(cudaMemcpyAsync(pos_host, s->B.stage, sizeof(double) * 3 * s->kp.n, cudaMemcpyDeviceToHost, s->stream));
    SS_CUDA(cudaStreamSynchronize(s->stream));
    return SP_OK;
}

int sp_set_positions(sp_sim* s, const double* pos_host, double delta)
{
    if (!s || !pos_host) return SP_ERR_INVALID_ARG;
    if (!(delta >= 0.0) || !(delta < s->p.L[0])) {
        s->err = "delta must lie in [0, L_x)";
        return SP_ERR_INVALID_ARG;
    }
    SS_TRY(set_device(s));
    SS_CUDA(cudaMemcpyAsync(s->B.stage, pos_host, sizeof(double) * 3 * s->kp.n, cudaMemcpyHostToDevice, s->stream));
    launch_gather_positions(s->B.stage, s->B.id_s, s->kp.n, s->kp.npad, s->B.pos_s, s->kp, s->B.st, s->stream);
    SS_CUDA(cudaMemcpyAsync(&s->B.st->delta, &delta, sizeof(double), cudaMemcpyHostToDevice, s->stream));
    SS_CUDA(cudaStreamSynchronize(s->stream));
    s->built = false;
    s->assembled = false;
    SS_TRY(read_state(s));
    if (s->st_host->error == SP_ERR_INVALID_ARG) {
        SS_TRY(clear_flags(s));
        s->err = status_text(SP_ERR_INVALID_ARG);
        return SP_ERR_INVALID_ARG;
    }
    return SP_OK;
}

int sp_get_velocities(sp_sim* s, double* v_host)
{
    if (!s || !v_host) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    launch_scatter_by_id(s->B.x, s->kp.npad, s->B.id_w, s->kp.n, s->B.stage, s->stream);
    SS_CUDA(cudaMemcpyAsync(v_host, s->B.stage, sizeof(double) * 3 * s->kp.n, cudaMemcpyDeviceToHost, s->stream));
    SS_CUDA(cudaStreamSynchronize(s->stream));
    return SP_OK;
}

int sp_get_state(sp_sim* s, double* delta, int64_t* step)
{
    if (!s) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    SS_TRY(read_state(s));
    if (delta) *delta = s->st_host->delta;
    if (step) *step = s->st_host->step;
    return SP_OK;
}

int sp_set_step(sp_sim* s, int64_t step)
{
    if (!s || step < 0) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    long long v = step;
    SS_TRY(write_field(s, &s->B.st->step, v));
    return SP_OK;
}

int sp_solve_flexible(sp_sim* s, int32_t net_every, sp_solve_info* info)
{
    if (!s || net_every < 0) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    if (mixed(s)) {
        s->err = "sp_solve_flexible needs an SP_PREC_FP64 simulation";
        return SP_ERR_INVALID_ARG;
    }
    if (!s->assembled) {
        s->err = "sp_solve_flexible needs sp_assemble first";
        return SP_ERR_INVALID_ARG;
    }
    if (net_every > 0 && !s->mp_alloc) {
        s->err = "sp_solve_flexible with net_every > 0 needs the network (sp_mpnn_enable)";
        return SP_ERR_INVALID_ARG;
    }
    if (!s->fcg) SS_TRY(dev_alloc(s, &s->fcg, 1));
    const size_t np = (size_t)s->kp.npad;
    // start from zero unless the simulation starts from the previous velocities
    // (which the build gathered into x); the network's warm-start guess is not used here
    if (s->p.warm_start != SP_WARM_PREV) SS_CUDA(cudaMemsetAsync(s->B.x, 0, sizeof(double) * 3 * np, s->stream));
    long long launches = 0;
    SS_TRY(fcg_solve(s->kp, s->B, net_every > 0 ? &s->mp : nullptr, net_every, s->fcg, &s->fcg_host,
                     launch_of(s, s->stream), &launches));
    const FcgState& h = s->fcg_host;
    int status = h.status;
    if (status == SP_OK && !(h.last_res <= s->p.cg_tol)) status = SP_ERR_NOT_CONVERGED;
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->status = status;
        info->iterations = h.iter;
        info->residual = h.last_res;
        info->bnorm = std::sqrt(h.bb);
        info->host_driven = 1;
    }
    SS_CUDA(cudaMemcpyAsync(s->B.v_s, s->B.x, sizeof(double) * 3 * np, cudaMemcpyDeviceToDevice, s->stream));
    SS_CUDA(cudaStreamSynchronize(s->stream));
    if (status != SP_OK) s->err = status_text(status);
    return status;
}

int sp_device_code_version(int32_t device, int32_t* binary_version, int32_t* ptx_version)
{
    if (!binary_version || !ptx_version) return SP_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        g_create_error = "no CUDA device with the requested ordinal";
        return SP_ERR_NO_DEVICE;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    int bin = 0, ptx = 0;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = device_code_version(&bin, &ptx);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        g_create_error = std::string("cudaFuncGetAttributes: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return SP_ERR_CUDA;
    }
    *binary_version = bin;
    *ptx_version = ptx;
    return SP_OK;
}

int sp_set_wait_limit(sp_sim* s, double seconds)
{
    if (!s || !(seconds > 0.0) || !(seconds <= 60.0)) {
        if (s) s->err = "the wait limit must lie in (0, 60] seconds";
        return SP_ERR_INVALID_ARG;
    }
    SS_TRY(set_device(s));
    const unsigned long long ns = std::max(1ull, (unsigned long long)std::llround(seconds * 1e9));
    SS_TRY(write_field(s, &s->B.st->bar_timeout_ns, ns));
    s->st_host->bar_timeout_ns = ns;
    return SP_OK;
}

int sp_get_order(sp_sim* s, int64_t* ids_host)
{
    if (!s || !ids_host) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    std::vector<int> ids(s->kp.n);
    SS_CUDA(cudaMemcpyAsync(ids.data(), s->B.id_w, sizeof(int) * s->kp.n, cudaMemcpyDeviceToHost, s->stream));
    SS_CUDA(cudaStreamSynchronize(s->stream));
    for (int i = 0; i < s->kp.n; ++i) ids_host[i] = ids[i];
    return SP_OK;
}

int sp_get_num_pairs(sp_sim* s, int64_t* npairs)
{
    if (!s || !npairs) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    SS_TRY(read_state(s));
    *npairs = s->st_host->nnz / 2;
    return SP_OK;
}

namespace {
// The pairs of the current matrix on the host, as (row, col, weight) entries
// in row order (rows in cell order).
int fetch_entries(sp_sim* s, std::vector<int>& rows, std::vector<int>& cols, std::vector<double>& vals,
                  std::vector<int>& ids)
{
    const int n = s->kp.n;
    SS_TRY(read_state(s));
    const long long slots = s->st_host->nnz_slots;
    std::vector<int> cnt(n), row_slot(n), chunk_off(s->kp.nchunks + 1), col(slots);
    std::vector<double> val(slots);
    std::vector<float> vh, vl;   // the mixed path keeps its weights as double-floats only
    ids.resize(n);
    SS_CUDA(cudaMemcpyAsync(cnt.data(), s->B.row_cnt, sizeof(int) * n, cudaMemcpyDeviceToHost, s->stream));
    SS_CUDA(cudaMemcpyAsync(row_slot.data(), s->B.row_slot, sizeof(int) * n, cudaMemcpyDeviceToHost, s->stream));
    SS_CUDA(cudaMemcpyAsync(chunk_off.data(), s->B.chunk_off, sizeof(int) * (s->kp.nchunks + 1),
                            cudaMemcpyDeviceToHost, s->stream));
    SS_CUDA(cudaMemcpyAsync(col.data(), s->B.col, sizeof(int) * slots, cudaMemcpyDeviceToHost, s->stream));
    if (mixed(s)) {
        vh.resize(slots);
        vl.resize(slots);
        SS_CUDA(cudaMemcpyAsync(vh.data(), s->B.val32, sizeof(float) * slots, cudaMemcpyDeviceToHost, s->stream));
        SS_CUDA(cudaMemcpyAsync(vl.data(), s->B.val32lo, sizeof(float) * slots, cudaMemcpyDeviceToHost, s->stream));
    } else {
        SS_CUDA(cudaMemcpyAsync(val.data(), s->B.val, sizeof(double) * slots, cudaMemcpyDeviceToHost, s->stream));
    }
    SS_CUDA(cudaMemcpyAsync(ids.data(), s->B.id_w, sizeof(int) * n, cudaMemcpyDeviceToHost, s->stream));
    SS_CUDA(cudaStreamSynchronize(s->stream));
    if (mixed(s))
        for (long long e = 0; e < slots; ++e) val[e] = (double)vh[e] + (double)vl[e];
    rows.clear();
    cols.clear();
    vals.clear();
    for (int r = 0; r < n; ++r) {
        const int slot = row_slot[r];
        const int base = chunk_off[slot >> 5] + (slot & 31);
        for (int k = 0; k < cnt[r]; ++k) {
            rows.push_back(r);
            cols.push_back(col[base + 32 * k]);
            vals.push_back(val[base + 32 * k]);
        }
    }
    return SP_OK;
}
}  // namespace

int sp_get_neighbors(sp_sim* s, int64_t cap, int64_t* pairs_host, int64_t* npairs)
{
    if (!s || !npairs) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    std::vector<int> rows, cols, ids;
    std::vector<double> vals;
    SS_TRY(fetch_entries(s, rows, cols, vals, ids));
    long long m = 0;
    for (size_t e = 0; e < rows.size(); ++e) {
        const int a = ids[rows[e]], b = ids[cols[e]];
        if (a < b) {
            if (pairs_host && m < cap) {
                pairs_host[2 * m] = a;
                pairs_host[2 * m + 1] = b;
            }
            ++m;
        }
    }
    *npairs = m;
    if (pairs_host && m > cap) {
        s->err = "pair capacity too small";
        return SP_ERR_INVALID_ARG;
    }
    return SP_OK;
}

int sp_get_system(sp_sim* s, double* diag_host, double* b_host, double* w_host)
{
    if (!s) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    const int n = s->kp.n;
    const size_t np = (size_t)s->kp.npad;
    std::vector<int> rows, cols, ids;
    std::vector<double> vals;
    SS_TRY(fetch_entries(s, rows, cols, vals, ids));
    if (diag_host) {
        std::vector<double> d(n);
        if (mixed(s)) {   // double-float A_ii
            std::vector<float> h(n), l(n);
            SS_CUDA(cudaMemcpy(h.data(), s->B.diag32, sizeof(float) * n, cudaMemcpyDeviceToHost));
            SS_CUDA(cudaMemcpy(l.data(), s->B.diag32lo, sizeof(float) * n, cudaMemcpyDeviceToHost));
            for (int r = 0; r < n; ++r) d[r] = (double)h[r] + (double)l[r];
        } else {
            SS_CUDA(cudaMemcpy(d.data(), s->B.diag, sizeof(double) * n, cudaMemcpyDeviceToHost));
        }
        for (int r = 0; r < n; ++r) diag_host[ids[r]] = d[r];
    }
    if (b_host) {
        std::vector<double> b(3 * np);
        if (mixed(s)) {   // double-float rows (hi, lo)
            std::vector<float> f(8 * np);
            SS_CUDA(cudaMemcpy(f.data(), s->B.bdf, sizeof(float) * 8 * np, cudaMemcpyDeviceToHost));
            for (size_t r = 0; r < np; ++r)
                for (int a = 0; a < 3; ++a) b[a * np + r] = (double)f[8 * r + a] + (double)f[8 * r + 4 + a];
        } else {
            SS_CUDA(cudaMemcpy(b.data(), s->B.b, sizeof(double) * 3 * np, cudaMemcpyDeviceToHost));
        }
        for (int r = 0; r < n; ++r)
            for (int a = 0; a < 3; ++a) b_host[3 * (size_t)ids[r] + a] = b[a * np + r];
    }
    if (w_host) {
        long long m = 0;
        for (size_t e = 0; e < rows.size(); ++e)
            if (ids[rows[e]] < ids[cols[e]]) w_host[m++] = vals[e];
    }
    return SP_OK;
}

int sp_set_noise(sp_sim* s, const double* xi_host)
{
    if (!s) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    SS_CUDA(cudaStreamSynchronize(s->stream));
    if (xi_host) {
        if (!s->B.xi_inj) SS_TRY(dev_alloc(s, &s->B.xi_inj, 3 * (size_t)s->kp.n));
        SS_CUDA(cudaMemcpy(s->B.xi_inj, xi_host, sizeof(double) * 3 * s->kp.n, cudaMemcpyHostToDevice));
        s->use_inj = true;
    } else {
        s->use_inj = false;
    }
    free_graphs(s);   // the kernels' arguments changed
    return SP_OK;
}

int sp_philox_blocks(int32_t device, uint64_t seed, uint64_t step, int64_t count, const int64_t* ids_host,
                     uint64_t* out_host)
{
    if (count < 0 || (count > 0 && (!ids_host || !out_host))) return SP_ERR_INVALID_ARG;
    if (count == 0) return SP_OK;
    if (cudaSetDevice(device) != cudaSuccess) return SP_ERR_NO_DEVICE;
    long long* ids = nullptr;
    unsigned long long* out = nullptr;
    if (cudaMalloc(&ids, sizeof(long long) * count) != cudaSuccess) return SP_ERR_OOM;
    if (cudaMalloc(&out, sizeof(unsigned long long) * 4 * count) != cudaSuccess) {
        cudaFree(ids);
        return SP_ERR_OOM;
    }
    int rc = SP_OK;
    if (cudaMemcpy(ids, ids_host, sizeof(long long) * count, cudaMemcpyHostToDevice) != cudaSuccess) rc = SP_ERR_CUDA;
    if (rc == SP_OK) {
        launch_philox_blocks(seed, step, count, ids, out, 0);
        if (cudaMemcpy(out_host, out, sizeof(unsigned long long) * 4 * count, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = SP_ERR_CUDA;
    }
    cudaFree(ids);
    cudaFree(out);
    return rc;
}

int sp_normals(int32_t device, uint64_t seed, uint64_t step, int64_t count, const int64_t* ids_host,
               int32_t precision, double* out_host)
{
    if (count < 0 || (count > 0 && (!ids_host || !out_host))) return SP_ERR_INVALID_ARG;
    if (precision != SP_PREC_FP64 && precision != SP_PREC_MIXED) return SP_ERR_INVALID_ARG;
    if (count == 0) return SP_OK;
    if (cudaSetDevice(device) != cudaSuccess) return SP_ERR_NO_DEVICE;
    long long* ids = nullptr;
    double* out = nullptr;
    float4* tab = nullptr;
    int rc = SP_OK;
    if (cudaMalloc(&ids, sizeof(long long) * count) != cudaSuccess || cudaMalloc(&out, sizeof(double) * 3 * count) != cudaSuccess ||
        cudaMalloc(&tab, sizeof(float4) * kRngTab) != cudaSuccess)
        rc = SP_ERR_OOM;
    if (rc == SP_OK && (cudaMemcpy(ids, ids_host, sizeof(long long) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
                        upload_rng_table(tab, 0) != cudaSuccess))
        rc = SP_ERR_CUDA;
    if (rc == SP_OK) {
        launch_normals(tab, seed, step, count, ids, out, precision == SP_PREC_MIXED ? 1 : 0, 0);
        if (cudaMemcpy(out_host, out, sizeof(double) * 3 * count, cudaMemcpyDeviceToHost) != cudaSuccess) rc = SP_ERR_CUDA;
    }
    cudaGetLastError();
    cudaFree(ids);
    cudaFree(out);
    cudaFree(tab);
    return rc;
}

int sp_sqrt_apply(sp_sim* s, int32_t degree, const double* g_host, double* xi_host, double* lambda_max,
                  double* steps_ms)
{
    if (!s || !g_host || !xi_host) return SP_ERR_INVALID_ARG;
    if (degree < 1 || degree > kFdtMaxDegree) {
        s->err = "sqrt_apply: degree must be in [1, 4096]";
        return SP_ERR_INVALID_ARG;
    }
    if (!s->assembled) {
        s->err = "sqrt_apply: assemble the system first";
        return SP_ERR_INVALID_ARG;
    }
    SS_TRY(set_device(s));
    const KParams& P = s->kp;
    DevBuffers& B = s->B;
    const int n = P.n, np = P.npad;
    FdtBuffers V;
    double* planes = nullptr;   // g, then xi, as FP64 planes in the rows' order
    int rc = fdt_alloc(s, V);
    if (rc == SP_OK) rc = dev_alloc(s, &planes, 3 * (size_t)np);
    unsigned long long bbits = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == SP_OK) {
        if (cudaMemcpyAsync(B.stage, g_host, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
            rc = SP_ERR_CUDA;
    }
    if (rc == SP_OK) {
        launch_gather_by_id(B.stage, B.id_w, n, np, planes, s->stream);
        if (P.mixed)
            cheb_split(P, planes, static_cast<float4*>(V.v[0]), s->stream);
        else
            cudaMemcpyAsync(V.v[0], planes, sizeof(double) * 3 * np, cudaMemcpyDeviceToDevice, s->stream);
        if (steps_ms) {
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            cudaEventRecord(e0, s->stream);
        }
        enqueue_cheb(P, B, V, degree, s->stream);
        if (steps_ms) cudaEventRecord(e1, s->stream);
        if (P.mixed)
            cheb_join(P, static_cast<float4*>(V.v[4]), planes, s->stream);
        else
            cudaMemcpyAsync(planes, V.v[4], sizeof(double) * 3 * np, cudaMemcpyDeviceToDevice, s->stream);
        launch_scatter_by_id(planes, np, B.id_w, n, B.stage, s->stream);
        if (cudaMemcpyAsync(xi_host, B.stage, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(&bbits, V.bound, sizeof(bbits), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
            cudaStreamSynchronize(s->stream) != cudaSuccess)
            rc = SP_ERR_CUDA;
    }
    if (rc == SP_OK) {
        double lmax = 1.0;
        std::memcpy(&lmax, &bbits, sizeof(lmax));
        if (lambda_max) *lambda_max = lmax;
        if (steps_ms) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            *steps_ms = ms;
        }
    }
    if (rc == SP_ERR_CUDA) s->err = std::string("sqrt_apply: ") + cudaGetErrorString(cudaGetLastError());
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    fdt_free(V);
    cudaFree(planes);
    return rc;
}

int sp_set_fdt_noise(sp_sim* s, int32_t degree)
{
    if (!s) return SP_ERR_INVALID_ARG;
    if (degree < 0 || degree > kFdtMaxDegree) {
        s->err = "fdt noise: degree must be in [0, 4096]";
        return SP_ERR_INVALID_ARG;
    }
    SS_TRY(set_device(s));
    SS_CUDA(cudaStreamSynchronize(s->stream));
    if (degree > 0 && !s->fdt.v[0]) SS_TRY(fdt_alloc(s, s->fdt));
    s->fdt_degree = degree;
    free_graphs(s);   // the step graph is captured again with (or without) the noise pass
    return SP_OK;
}

static void vc_info(const VcStats& st, long long n, sp_vcorr_info* info)
{
    if (!info) return;
    info->pairs_ms = st.pairs_ms;
    info->boundary_pairs = st.band_pairs;
    info->pairs = n * (n - 1) / 2;
}

int sp_velocity_correlation(sp_sim* s, int32_t nbins, double rmax, double* sum_host, int64_t* count_host,
                            double* vsq_host, sp_vcorr_info* info)
{
    if (!s || !sum_host || !count_host || !vsq_host) return SP_ERR_INVALID_ARG;
    if (nbins < 1 || nbins > kVcMaxBins || !(rmax > 0.0) || !std::isfinite(rmax)) {
        s->err = "velocity correlation: needs 1 <= nbins <= 1024 and rmax > 0";
        return SP_ERR_INVALID_ARG;
    }
    SS_TRY(set_device(s));
    SS_TRY(read_state(s));
    const long long n = s->kp.n;
    if (vc_reserve(s->vc, n) != cudaSuccess) {
        cudaGetLastError();
        s->err = "velocity correlation: device allocation failed";
        return SP_ERR_OOM;
    }
    // positions and the last solve's velocities, both in particle-id order
    launch_scatter_by_id(s->B.pos_s, s->kp.npad, s->B.id_s, s->kp.n, s->vc.pos_n3, s->stream);
    launch_scatter_by_id(s->B.x, s->kp.npad, s->B.id_w, s->kp.n, s->vc.v_n3, s->stream);
    VcStats st{};
    const char* e = nullptr;
    const int rc = run_velocity_correlation(s->vc, n, s->p.L, s->st_host->delta, s->kp.kappa, nbins, rmax, s->stream,
                                            sum_host, reinterpret_cast<long long*>(count_host), vsq_host, &st, &e);
    if (e) s->err = e;
    if (rc == SP_OK) vc_info(st, n, info);
    return rc;
}

int sp_velocity_correlation_host(int32_t device, int64_t n, const double* L3, double delta, double kappa,
                                 const double* pos_host, const double* v_host, int32_t nbins, double rmax,
                                 double* sum_host, int64_t* count_host, double* vsq_host, sp_vcorr_info* info)
{
    if (n < 1 || !L3 || !pos_host || !v_host || !sum_host || !count_host || !vsq_host) return SP_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return SP_ERR_NO_DEVICE;
    }
    VcBuffers V{};
    int rc = SP_OK;
    if (vc_reserve(V, n) != cudaSuccess) rc = SP_ERR_OOM;
    if (rc == SP_OK && (cudaMemcpy(V.pos_n3, pos_host, sizeof(double) * 3 * n, cudaMemcpyHostToDevice) != cudaSuccess ||
                        cudaMemcpy(V.v_n3, v_host, sizeof(double) * 3 * n, cudaMemcpyHostToDevice) != cudaSuccess))
        rc = SP_ERR_CUDA;
    VcStats st{};
    const char* e = nullptr;
    if (rc == SP_OK)
        rc = run_velocity_correlation(V, n, L3, delta, kappa, nbins, rmax, 0, sum_host,
                                      reinterpret_cast<long long*>(count_host), vsq_host, &st, &e);
    if (e) sp_global_error() = e;
    if (rc == SP_OK) vc_info(st, n, info);
    cudaGetLastError();
    vc_free(V);
    return rc;
}

int sp_structure_factor(sp_sim* s, int32_t nkx, int32_t nky, int32_t grid, double* S_host,
                        double* qx_host, double* qy_host)
{
    if (!s || !S_host || nkx < 0 || nky < 0 || grid < 0) return SP_ERR_INVALID_ARG;
    if (grid > 0 && (grid < 8 || grid > 8192 || 4 * nkx >= grid || 4 * nky >= grid)) {
        s->err = "structure factor: grid must be in [8, 8192] with |kx|, |ky| < grid / 4";
        return SP_ERR_INVALID_ARG;
    }
    if ((long long)(2 * nkx + 1) * (2 * nky + 1) > (1ll << 24)) {
        s->err = "structure factor: too many modes";
        return SP_ERR_INVALID_ARG;
    }
    SS_TRY(set_device(s));
    SS_TRY(read_state(s));
    const double delta = s->st_host->delta;
    const size_t m = (size_t)(2 * nkx + 1) * (2 * nky + 1);
    double *S = nullptr, *qx = nullptr, *qy = nullptr, *tw = nullptr;
    unsigned long long* g = nullptr;
    double2* A = nullptr;
    int rc = SP_OK;
    auto A_ = [&](int r) { if (rc == SP_OK) rc = r; };
    A_(dev_alloc(s, &S, m));
    A_(dev_alloc(s, &qx, m));
    A_(dev_alloc(s, &qy, m));
    if (grid > 0) {
        A_(dev_alloc(s, &tw, 2 * (size_t)grid));
        A_(dev_alloc(s, &g, (size_t)grid * grid));
        A_(dev_alloc(s, &A, (size_t)(2 * nkx + 1) * grid));
    }
    if (rc == SP_OK && grid > 0) {
        // twiddle table (cos, sin)(2 pi m / G), m = 0..G-1
        std::vector<double> t(2 * (size_t)grid);
        const double two_pi = 6.283185307179586476925286766559;
        for (int k = 0; k < grid; ++k) {
            t[2 * k] = std::cos(two_pi * k / grid);
            t[2 * k + 1] = std::sin(two_pi * k / grid);
        }
        if (cudaMemcpyAsync(tw, t.data(), sizeof(double) * t.size(), cudaMemcpyHostToDevice, s->stream) !=
            cudaSuccess)
            rc = SP_ERR_CUDA;
        if (rc == SP_OK) SS_CUDA(cudaStreamSynchronize(s->stream));
    }
    if (rc == SP_OK) {
        if (run_structure_factor(s->kp, s->B, delta, grid, nkx, nky, tw, g, A, S, qx, qy, s->stream) != cudaSuccess)
            rc = SP_ERR_CUDA;
    }
    if (rc == SP_OK) {
        if (cudaMemcpyAsync(S_host, S, sizeof(double) * m, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
            (qx_host && cudaMemcpyAsync(qx_host, qx, sizeof(double) * m, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess) ||
            (qy_host && cudaMemcpyAsync(qy_host, qy, sizeof(double) * m, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess) ||
            cudaStreamSynchronize(s->stream) != cudaSuccess)
            rc = SP_ERR_CUDA;
    }
    if (rc == SP_ERR_CUDA && s->err.empty()) s->err = std::string("structure factor: ") + cudaGetErrorString(cudaGetLastError());
    void* ptrs[] = {S, qx, qy, tw, g, A};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    return rc;
}

int sp_mpnn_num_params(void) { return kMpParams; }

int sp_mpnn_enable(sp_sim* s, uint64_t seed, const float* weights_host)
{
    if (!s) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    MpBuffers& M = s->mp;
    if (!s->mp_alloc) {
        const size_t rows = 3 * (size_t)s->kp.n;
        int a = SP_OK;
        auto A = [&](int r) { if (a == SP_OK) a = r; };
        A(dev_alloc(s, &M.x0, rows));
        A(dev_alloc(s, &M.a0, rows));
        A(dev_alloc(s, &M.y, rows));
        A(dev_alloc(s, &M.a1, rows));
        A(dev_alloc(s, &M.dy, rows));
        A(dev_alloc(s, &M.g1, rows));
        A(dev_alloc(s, &M.master, kMpParams));
        A(dev_alloc(s, &M.m, kMpParams));
        A(dev_alloc(s, &M.v, kMpParams));
        A(dev_alloc(s, &M.grad, kMpParams));
        A(dev_alloc(s, &M.gpart, (size_t)1024 * kMpParams));
        A(dev_alloc(s, &M.dpart, (size_t)1024 * 12));
        A(dev_alloc(s, &M.wb, (size_t)mp_weights_bf16_count()));
        A(dev_alloc(s, &M.scal, 4));
        A(dev_alloc(s, &M.part, (size_t)kMaxPartials));
        A(dev_alloc(s, &M.ticket, 4));
        s->mp_alloc = true;   // freed by sp_sim_destroy even if an allocation failed
        if (a != SP_OK) return a;
        if (mp_prepare() != 0) {
            s->err = "could not enable the shared memory of the training kernel";
            return SP_ERR_CUDA;
        }
    }
    std::vector<float> w(kMpParams, 0.f);
    if (weights_host) {
        std::memcpy(w.data(), weights_host, sizeof(float) * kMpParams);
    } else {
        // scaled normal hidden weights; readout = the previous-velocity guess
        std::mt19937_64 gen(seed);
        std::normal_distribution<double> nd(0.0, 1.0);
        for (int k = 0; k < kMpOffW2; ++k) w[k] = (float)(nd(gen) / std::sqrt(6.0));
        for (int k = kMpOffW2; k < kMpOffO; ++k) w[k] = (float)(nd(gen) / 8.0);
        w[kMpOffO + 9] = 1.f;
    }
    SS_CUDA(cudaMemsetAsync(M.wb, 0, sizeof(__nv_bfloat16) * mp_weights_bf16_count(), s->stream));
    SS_CUDA(cudaMemsetAsync(M.m, 0, sizeof(float) * kMpParams, s->stream));
    SS_CUDA(cudaMemsetAsync(M.v, 0, sizeof(float) * kMpParams, s->stream));
    SS_CUDA(cudaMemsetAsync(M.ticket, 0, sizeof(unsigned int) * 4, s->stream));
    SS_CUDA(cudaMemsetAsync(M.scal, 0, sizeof(double) * 4, s->stream));
    SS_CUDA(cudaMemcpyAsync(M.master, w.data(), sizeof(float) * kMpParams, cudaMemcpyHostToDevice, s->stream));
    launch_mp_convert(M, s->stream);
    SS_CUDA(cudaStreamSynchronize(s->stream));
    s->mp_t = 0;
    s->learned = true;
    free_graphs(s);
    return SP_OK;
}

int sp_mpnn_set_prior(sp_sim* s, int32_t use_vprev)
{
    if (!s || !s->mp_alloc || (use_vprev != 0 && use_vprev != 1)) return SP_ERR_INVALID_ARG;
    s->mp.zero_vprev = use_vprev ? 0 : 1;
    free_graphs(s);   // the captured step graph holds the network's buffers by value
    return SP_OK;
}

int sp_mpnn_disable(sp_sim* s)
{
    if (!s) return SP_ERR_INVALID_ARG;
    s->learned = false;
    free_graphs(s);
    return SP_OK;
}

int sp_mpnn_get_weights(sp_sim* s, float* w_host)
{
    if (!s || !w_host || !s->mp_alloc) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    SS_CUDA(cudaMemcpyAsync(w_host, s->mp.master, sizeof(float) * kMpParams, cudaMemcpyDeviceToHost, s->stream));
    SS_CUDA(cudaStreamSynchronize(s->stream));
    return SP_OK;
}

int sp_mpnn_set_weights(sp_sim* s, const float* w_host)
{
    if (!s || !w_host || !s->mp_alloc) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    SS_CUDA(cudaMemcpyAsync(s->mp.master, w_host, sizeof(float) * kMpParams, cudaMemcpyHostToDevice, s->stream));
    launch_mp_convert(s->mp, s->stream);
    SS_CUDA(cudaStreamSynchronize(s->stream));
    return SP_OK;
}

int sp_mpnn_forward(sp_sim* s, double* guess_host)
{
    if (!s || !s->mp_alloc) return SP_ERR_INVALID_ARG;
    if (!s->assembled) {
        s->err = "sp_mpnn_forward needs sp_assemble first";
        return SP_ERR_INVALID_ARG;
    }
    SS_TRY(set_device(s));
    launch_mp_infer(s->kp, s->B, s->mp, launch_of(s, s->stream));
    SS_CUDA(cudaGetLastError());
    if (guess_host) {
        launch_scatter_by_id(s->B.x, s->kp.npad, s->B.id_w, s->kp.n, s->B.stage, s->stream);
        SS_CUDA(cudaMemcpyAsync(guess_host, s->B.stage, sizeof(double) * 3 * s->kp.n, cudaMemcpyDeviceToHost,
                                s->stream));
    }
    SS_CUDA(cudaStreamSynchronize(s->stream));
    return SP_OK;
}

int sp_mpnn_train_step(sp_sim* s, float lr, double* loss, float* grad_host)
{
    if (!s || !s->mp_alloc || !(lr >= 0.f)) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    if (lr > 0.f) s->mp_t += 1;   // a gradient-only call (lr = 0) is no Adam step
    launch_mp_train(s->kp, s->B, s->mp, lr, std::max(s->mp_t, 1), launch_of(s, s->stream));
    SS_CUDA(cudaGetLastError());
    if (loss) SS_CUDA(cudaMemcpyAsync(loss, s->mp.scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    if (grad_host)
        SS_CUDA(cudaMemcpyAsync(grad_host, s->mp.grad, sizeof(float) * kMpParams, cudaMemcpyDeviceToHost, s->stream));
    SS_CUDA(cudaStreamSynchronize(s->stream));
    return SP_OK;
}

}  // extern "C"
