// Batches of independent simulations advanced together (ensembles of replicas
// with uneven particle counts and shear rates).
//
// Each replica is a full simulation (own box, shear rate, seed, buffers and
// device state).  One time step of the whole batch is one CUDA graph: the
// replicas' cell lists, pair searches and assemblies run as parallel branches,
// then a single cooperative launch solves every replica's system (blocks are
// shared out in proportion to the replicas' rows; each replica's blocks
// synchronise, reduce and stop on their own), then the replicas' stress and
// position updates run as parallel branches again.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "sim_impl.cuh"

using namespace ss;
using namespace ss_host;

struct sp_batch {
    int R = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<sp_sim*> sims;
    std::vector<cudaStream_t> branch;
    std::vector<cudaEvent_t> ev;
    KParams* d_P = nullptr;
    DevBuffers* d_B = nullptr;
    int* d_blk_off = nullptr;
    std::vector<int> blk_off;
    int total_blocks = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long fixed_launches = 0;
    int cfg = 0;   // tile configuration of the batched solver (sp_batch_autotune)
    std::string err;
};

namespace {

constexpr int kBranches = 8;

#define SB_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            b->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
            return SP_ERR_CUDA;                                                         \
        }                                                                               \
    } while (0)

void free_graph(sp_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Device copies of every replica's constants and buffer pointers, and the
// share of the cooperative launch of each replica.
int upload(sp_batch* b)
{
    std::vector<KParams> P(b->R);
    std::vector<DevBuffers> B(b->R);
    std::vector<long long> win(b->R);
    long long total_win = 0;
    for (int k = 0; k < b->R; ++k) {
        P[k] = b->sims[k]->kp;
        B[k] = b->sims[k]->B;
        win[k] = P[k].nslots / 256;
        total_win += win[k];
    }
    const int cap = cg_persistent_batch_capacity(Launch{b->stream, b->sims[0]->num_sms}, b->cfg);
    if (cap < b->R) {
        b->err = "more replicas than resident blocks of the batched solver";
        return SP_ERR_INVALID_ARG;
    }
    // blocks in proportion to the windows of 256 rows, at least one each, at
    // most one per window, within the co-resident capacity
    std::vector<int> nb(b->R);
    long long used = 0;
    for (int k = 0; k < b->R; ++k) {
        long long x = (long long)((double)cap * (double)win[k] / (double)total_win);
        x = std::max<long long>(1, std::min<long long>(x, win[k]));
        nb[k] = (int)x;
        used += x;
    }
    while (used > cap) {   // trim the largest shares
        int kmax = (int)(std::max_element(nb.begin(), nb.end()) - nb.begin());
        if (nb[kmax] <= 1) break;
        --nb[kmax];
        --used;
    }
    b->blk_off.assign(b->R + 1, 0);
    for (int k = 0; k < b->R; ++k) b->blk_off[k + 1] = b->blk_off[k] + nb[k];
    b->total_blocks = b->blk_off[b->R];
    SB_CUDA(cudaMemcpyAsync(b->d_P, P.data(), sizeof(KParams) * b->R, cudaMemcpyHostToDevice, b->stream));
    SB_CUDA(cudaMemcpyAsync(b->d_B, B.data(), sizeof(DevBuffers) * b->R, cudaMemcpyHostToDevice, b->stream));
    SB_CUDA(cudaMemcpyAsync(b->d_blk_off, b->blk_off.data(), sizeof(int) * (b->R + 1), cudaMemcpyHostToDevice,
                            b->stream));
    SB_CUDA(cudaStreamSynchronize(b->stream));
    return SP_OK;
}

int capture(sp_batch* b)
{
    free_graph(b);
    cudaStream_t cs = b->stream;
    const int S = (int)b->branch.size();
    long long launches = 0;
    SB_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    int rc = SP_OK;
    auto fork = [&](cudaEvent_t e) {
        cudaEventRecord(e, cs);
        for (int s = 0; s < S; ++s) cudaStreamWaitEvent(b->branch[s], e, 0);
    };
    auto join = [&]() {
        for (int s = 0; s < S; ++s) {
            cudaEventRecord(b->ev[1 + s], b->branch[s]);
            cudaStreamWaitEvent(cs, b->ev[1 + s], 0);
        }
    };
    fork(b->ev[0]);
    for (int k = 0; k < b->R; ++k) {
        sp_sim* s = b->sims[k];
        cudaStream_t st = b->branch[k % S];
        launches += enqueue_build(s, st);
        launches += launch_nbr_fill(s->kp, s->B, true, s->use_inj, true, launch_of(s, st));
        launches += launch_cg_init(s->kp, s->B, s->p.warm_start == SP_WARM_PREV, true, launch_of(s, st));
    }
    join();
    if (launch_cg32_persistent_batch(b->d_P, b->d_B, b->d_blk_off, b->R, b->total_blocks, b->cfg,
                                     Launch{cs, b->sims[0]->num_sms}) != cudaSuccess)
        rc = SP_ERR_CUDA;
    launches += 1;
    fork(b->ev[S + 1]);
    for (int k = 0; k < b->R; ++k) {
        sp_sim* s = b->sims[k];
        cudaStream_t st = b->branch[k % S];
        launch_cg_finish(s->kp, s->B, true, launch_of(s, st));
        launch_stress(s->kp, s->B, true, launch_of(s, st));
        launch_integrate(s->kp, s->B, launch_of(s, st));
        launches += 4;   // finish, stress, update, commit of the new offset
    }
    join();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (rc != SP_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        b->err = std::string("batch graph capture failed: ") + cudaGetErrorString(rc != SP_OK ? cudaGetLastError() : e);
        cudaGetLastError();
        return SP_ERR_CUDA;
    }
    b->graph = g;
    SB_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
    b->fixed_launches = launches;
    return SP_OK;
}

}  // namespace

extern "C" {

int sp_batch_destroy(sp_batch* b)
{
    if (!b) return SP_OK;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    free_graph(b);
    for (sp_sim* s : b->sims) sp_sim_destroy(s);
    for (auto s : b->branch) cudaStreamDestroy(s);
    for (auto e : b->ev) cudaEventDestroy(e);
    if (b->d_P) cudaFree(b->d_P);
    if (b->d_B) cudaFree(b->d_B);
    if (b->d_blk_off) cudaFree(b->d_blk_off);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return SP_OK;
}

int sp_batch_create(int32_t R, const sp_params* params, const double* const* pos_host, sp_batch** out)
{
    std::string& gerr = sp_global_error();
    gerr.clear();
    if (!out || !params || R < 1 || R > 4096) {
        gerr = "sp_batch_create: need 1 <= R <= 4096 parameter sets and an output pointer";
        return SP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    for (int k = 0; k < R; ++k) {
        if (params[k].precision != SP_PREC_MIXED || params[k].device != params[0].device) {
            gerr = "sp_batch_create: every replica must use the mixed solver on the same device";
            return SP_ERR_INVALID_ARG;
        }
    }
    sp_batch* b = new sp_batch();
    b->R = R;
    b->device = params[0].device;
    auto fail = [&](int code, const std::string& why) {
        gerr = why;
        sp_batch_destroy(b);
        return code;
    };
    if (cudaSetDevice(b->device) != cudaSuccess) return fail(SP_ERR_NO_DEVICE, "no such device");
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(SP_ERR_CUDA, "cudaStreamCreate failed");
    const int S = std::min(kBranches, (int)R);
    b->branch.resize(S);
    for (auto& s : b->branch)
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
            return fail(SP_ERR_CUDA, "cudaStreamCreate failed");
    b->ev.resize(S + 2);
    for (auto& e : b->ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return fail(SP_ERR_CUDA, "cudaEventCreate failed");
    for (int k = 0; k < R; ++k) {
        sp_params p = params[k];
        p.stream = (void*)b->stream;
        sp_sim* s = nullptr;
        const int rc = sp_sim_create(&p, pos_host ? pos_host[k] : nullptr, &s);
        if (rc != SP_OK) return fail(rc, "replica " + std::to_string(k) + ": " + gerr);
        s->persistent = true;
        b->sims.push_back(s);
    }
    if (cudaMalloc(&b->d_P, sizeof(KParams) * R) != cudaSuccess ||
        cudaMalloc(&b->d_B, sizeof(DevBuffers) * R) != cudaSuccess ||
        cudaMalloc(&b->d_blk_off, sizeof(int) * (R + 1)) != cudaSuccess)
        return fail(SP_ERR_OOM, "cudaMalloc failed");
    const int rc = upload(b);
    if (rc != SP_OK) return fail(rc, b->err);
    *out = b;
    return SP_OK;
}

int sp_batch_get_sim(sp_batch* b, int32_t k, sp_sim** sim)
{
    if (!b || !sim || k < 0 || k >= b->R) return SP_ERR_INVALID_ARG;
    *sim = b->sims[k];
    return SP_OK;
}

int sp_batch_blocks(sp_batch* b, int32_t* blocks)
{
    if (!b || !blocks) return SP_ERR_INVALID_ARG;
    for (int k = 0; k < b->R; ++k) blocks[k] = b->blk_off[k + 1] - b->blk_off[k];
    return SP_OK;
}

int sp_batch_step(sp_batch* b, int32_t nsteps, sp_step_info* info)
{
    if (!b || nsteps < 0) return SP_ERR_INVALID_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess) return SP_ERR_NO_DEVICE;
    for (sp_sim* s : b->sims) launch_reset_step_stats(s->B.st, b->stream);
    if (!b->exec) {
        const int rc = capture(b);
        if (rc != SP_OK) return rc;
    }
    for (int k = 0; k < nsteps; ++k) SB_CUDA(cudaGraphLaunch(b->exec, b->stream));
    SB_CUDA(cudaStreamSynchronize(b->stream));
    int status = SP_OK;
    bool regrown = false;
    for (int k = 0; k < b->R; ++k) {
        sp_sim* s = b->sims[k];
        int rc = read_state(s);
        if (rc != SP_OK) return rc;
        long long done = s->st_host->steps_in_call;
        long long iters = s->st_host->iter_sum, checks = s->st_host->true_checks;
        int iter_max = s->st_host->iter_max;
        int rstatus = s->st_host->error;
        if (s->st_host->overflow) {
            // this replica's pair storage overflowed at step `done`: grow it and let
            // the replica catch up on its own; the batch graph is re-captured
            rc = grow_pairs(s);
            if (rc != SP_OK) return rc;
            regrown = true;
            sp_step_info si{};
            rc = sp_step(s, (int32_t)(nsteps - done), &si);
            done += si.steps_done;
            iters += si.cg_iterations;
            iter_max = std::max(iter_max, si.max_iterations);
            rstatus = rc;
        } else if (rstatus != 0) {
            rc = clear_flags(s);
            if (rc != SP_OK) return rc;
        }
        if (rstatus != SP_OK && status == SP_OK) status = rstatus;
        if (info) {
            info[k].status = rstatus;
            info[k].steps_done = done;
            info[k].cg_iterations = iters;
            info[k].max_iterations = iter_max;
            info[k].last_residual = s->st_host->last_res;
            info[k].stress_xy = s->st_host->stress_xy;
            info[k].delta = s->st_host->delta;
            info[k].step = s->st_host->step;
            info[k].kernel_launches = (k == 0 ? (long long)nsteps * b->fixed_launches : 0) + 0 * checks;
            info[k].host_driven = 0;   // the batch always steps by its captured graph
        }
        s->built = false;
        s->assembled = false;
    }
    if (regrown) {
        free_graph(b);
        const int rc = upload(b);
        if (rc != SP_OK) return rc;
    }
    if (status != SP_OK) b->err = "a replica failed (see its step info)";
    return status;
}

int sp_batch_autotune(sp_batch* b, int32_t trials, sp_tune_info* info)
{
    if (!b) return SP_ERR_INVALID_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess) return SP_ERR_NO_DEVICE;
    sp_tune_info out{};
    out.num_configs = std::min(kBatchConfigs, SP_TUNE_MAX_CONFIGS);
    const int prev = b->cfg;
    int best = prev;
    if (trials >= 1) {
        // every replica's pair list and system for its current positions (the
        // state is kept: a build only reorders it; the solves below overwrite
        // only the solution vectors, which the next step's build refills)
        for (sp_sim* s : b->sims) {
            int rc = do_build(s);
            if (rc == SP_OK) rc = sp_assemble(s);
            if (rc != SP_OK) {
                b->err = "autotune: building a replica's system failed";
                return rc;
            }
        }
        cudaEvent_t e0, e1;
        SB_CUDA(cudaEventCreate(&e0));
        SB_CUDA(cudaEventCreate(&e1));
        double best_ms = 1e30;
        for (int k = 0; k < out.num_configs; ++k) {
            b->cfg = k;
            if (upload(b) != SP_OK) {   // fewer resident blocks than replicas
                cudaGetLastError();
                continue;
            }
            double t = 1e30;
            for (int r = 0; r < trials; ++r) {
                for (sp_sim* s : b->sims) launch_cg_init(s->kp, s->B, false, true, launch_of(s, b->stream));
                cudaEventRecord(e0, b->stream);
                const cudaError_t le = launch_cg32_persistent_batch(b->d_P, b->d_B, b->d_blk_off, b->R,
                                                                    b->total_blocks, k,
                                                                    Launch{b->stream, b->sims[0]->num_sms});
                cudaEventRecord(e1, b->stream);
                if (le != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    b->cfg = prev;
                    upload(b);
                    b->err = std::string("autotune: batched solve failed: ") + cudaGetErrorString(le);
                    return SP_ERR_CUDA;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                t = std::min(t, (double)ms);
            }
            for (sp_sim* s : b->sims) {   // a failed trial (e.g. a timeout) is not a candidate
                if (read_state(s) != SP_OK) break;
                if (s->st_host->error) {
                    clear_flags(s);
                    t = 1e30;
                }
            }
            if (k < SP_TUNE_MAX_CONFIGS) out.ms[k] = t < 1e30 ? t : 0.0;
            if (t < best_ms) {
                best_ms = t;
                best = k;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    b->cfg = best;
    free_graph(b);
    const int rc = upload(b);
    if (rc != SP_OK) return rc;
    for (sp_sim* s : b->sims) {
        s->built = false;
        s->assembled = false;
    }
    if (info) {
        out.config = best;
        cg_batch_config(best, &out.gathers_in_flight, &out.blocks_per_sm, &out.block_threads);
        *info = out;
    }
    return SP_OK;
}

int sp_batch_set_config(sp_batch* b, int32_t config)
{
    if (!b || config < 0 || config >= kBatchConfigs) return SP_ERR_INVALID_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess) return SP_ERR_NO_DEVICE;
    const int prev = b->cfg;
    b->cfg = config;
    free_graph(b);
    const int rc = upload(b);
    if (rc != SP_OK) {
        b->cfg = prev;
        upload(b);
    }
    return rc;
}

const char* sp_batch_last_error(const sp_batch* b)
{
    return b ? b->err.c_str() : sp_global_error().c_str();
}

}  // extern "C"
