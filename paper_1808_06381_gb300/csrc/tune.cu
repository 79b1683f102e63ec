// sp_autotune: choice of the persistent solver's tile configuration for one
// simulation by timing (all configurations run the same iteration; only the
// grouping of the dot products' partial sums, hence their rounding, differs).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>

#include "shearsim.h"
#include "sim_impl.cuh"

using namespace ss;
using namespace ss_host;

namespace {

std::mutex g_cache_mutex;

std::string tune_key(const sp_sim* s, long long nnz)
{
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, s->p.device);
    std::string name(prop.name);
    for (char& c : name)
        if (c == ' ' || c == '|') c = '_';
    const long long row_len = s->kp.n > 0 ? (long long)std::llround((double)nnz / (double)s->kp.n) : 0;
    std::ostringstream k;
    k << name << "|sm" << s->num_sms << "|n" << s->kp.n << "|row" << row_len;
    return k.str();
}

int cache_lookup(const std::string& path, const std::string& key)
{
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    std::ifstream f(path);
    std::string k;
    int cfg, found = -1;
    while (f >> k >> cfg)
        if (k == key && cfg >= 0 && cfg < kPersistentConfigs) found = cfg;   // the last line wins
    return found;
}

void cache_store(const std::string& path, const std::string& key, int cfg)
{
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    std::ofstream f(path, std::ios::app);
    if (f) f << key << ' ' << cfg << '\n';
}

}  // namespace

extern "C" int sp_set_solver_config(sp_sim* s, int32_t config, sp_tune_info* info)
{
    if (!s || config < 0 || config >= std::min(kPersistentConfigs, SP_TUNE_MAX_CONFIGS)) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    s->kp.pcfg = config;
    free_graphs(s);   // captured graphs hold the previous configuration's kernel
    if (info) {
        sp_tune_info out{};
        out.config = config;
        out.num_configs = std::min(kPersistentConfigs, SP_TUNE_MAX_CONFIGS);
        cg_persistent_config(config, &out.gathers_in_flight, &out.blocks_per_sm, &out.pipelined, &out.block_threads,
                             &out.resident, &out.matrix_free);
        *info = out;
    }
    return SP_OK;
}

extern "C" int sp_autotune(sp_sim* s, int32_t trials, sp_tune_info* info)
{
    if (!s) return SP_ERR_INVALID_ARG;
    SS_TRY(set_device(s));
    sp_tune_info out{};
    out.num_configs = std::min(kPersistentConfigs, SP_TUNE_MAX_CONFIGS);
    auto finish = [&](int cfg) {
        s->kp.pcfg = cfg;
        free_graphs(s);   // captured graphs hold the previous configuration's kernel
        out.config = cfg;
        cg_persistent_config(cfg, &out.gathers_in_flight, &out.blocks_per_sm, &out.pipelined, &out.block_threads,
                             &out.resident, &out.matrix_free);
        if (info) *info = out;
        return SP_OK;
    };
    if (!mixed(s) || !s->persistent || trials < 1) return finish(s->kp.pcfg);

    // the system of the current positions (noise of the current step counter)
    SS_TRY(do_build(s));
    launch_assemble_only(s->kp, s->B, s->use_inj, mixed(s), launch_of(s, s->stream));
    SS_CUDA(cudaStreamSynchronize(s->stream));
    s->assembled = true;
    SS_TRY(read_state(s));
    const long long nnz = s->st_host->nnz;

    const char* path = std::getenv("SHEARSIM_TUNE_CACHE");
    const std::string key = tune_key(s, nnz);
    if (path && *path) {
        const int cfg = cache_lookup(path, key);
        if (cfg >= 0) {
            out.from_cache = 1;
            return finish(cfg);
        }
    }

    // keep the previous velocities (the next step's warm start)
    const size_t vbytes = sizeof(double) * 3 * (size_t)s->kp.npad;
    double* v_save = nullptr;
    SS_CUDA(cudaMalloc(&v_save, vbytes));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = SP_OK;
    if (cudaMemcpyAsync(v_save, s->B.v_s, vbytes, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = SP_ERR_CUDA;
    const int prev = s->kp.pcfg;
    int best = prev;
    double best_ms = 0.0;
    for (int c = 0; rc == SP_OK && c < out.num_configs; ++c) {
        if (!cg_persistent_usable(c, s->kp, s->B, launch_of(s, s->stream))) continue;   // ms[c] stays 0
        s->kp.pcfg = c;
        double cmin = 0.0;
        for (int t = 0; rc == SP_OK && t <= trials; ++t) {   // the first solve warms up
            long long launches = 0;
            cudaEventRecord(e0, s->stream);
            rc = enqueue_solve(s, s->stream, false, false, &launches);
            cudaEventRecord(e1, s->stream);
            if (rc == SP_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = SP_ERR_CUDA;
            if (rc == SP_OK) rc = read_state(s);
            if (rc == SP_OK && s->st_host->error) rc = s->st_host->error;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rc == SP_OK && t > 0 && (cmin == 0.0 || ms < cmin)) cmin = ms;
        }
        out.ms[c] = cmin;
        if (rc == SP_OK && (best_ms == 0.0 || cmin < best_ms)) {
            best_ms = cmin;
            best = c;
        }
    }
    if (cudaMemcpyAsync(s->B.v_s, v_save, vbytes, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        rc = rc == SP_OK ? SP_ERR_CUDA : rc;
    cudaFree(v_save);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc != SP_OK) {
        s->kp.pcfg = prev;
        if (s->st_host->error) clear_flags(s);
        if (s->err.empty()) s->err = "autotuning solve failed";
        return rc;
    }
    if (path && *path) cache_store(path, key, best);
    return finish(best);
}
