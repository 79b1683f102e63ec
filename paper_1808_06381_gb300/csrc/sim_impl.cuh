// Private host-side declarations shared by the translation units of the
// shearsim library (simulation object and the enqueueing helpers).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "internal.cuh"

// One simulation: parameters, device buffers, streams and captured graphs.
struct sp_sim {
    sp_params p{};
    ss::KParams kp{};
    ss::DevBuffers B{};
    ss::DevState* st_host = nullptr;  // pinned mirror of the device state
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // capture streams: [0] the graph's main stream, [1] its side branch (normals,
    // split of x0, stress), [2] the body of the CG loop's WHILE node, [3] the
    // body of its IF node; a stream still joined to one capture cannot begin
    // another, so the side branch and the node bodies never share one
    cudaStream_t cap_stream[4] = {nullptr, nullptr, nullptr, nullptr};
    int num_sms = 0;
    long long nnz_cap = 0;
    bool use_inj = false;
    bool host_loop = false;       // CG loop driven from the host
    bool persistent = true;       // mixed solver: one cooperative launch per solve
    bool built = false;           // pairs match the current positions
    bool assembled = false;
    cudaGraph_t step_graph = nullptr;
    cudaGraphExec_t step_exec = nullptr;
    cudaGraph_t solve_graph[2] = {nullptr, nullptr};   // [from_x]
    cudaGraphExec_t solve_exec[2] = {nullptr, nullptr};
    long long fixed_launches_step = 0;
    long long fixed_launches_solve = 0;
    ss::MpBuffers mp{};           // learned warm start (allocated by sp_mpnn_enable)
    bool mp_alloc = false;
    bool learned = false;         // run the network before every solve of a step
    int mp_t = 0;                 // Adam step counter
    ss::VcBuffers vc{};           // velocity correlation (allocated by its first call)
    ss::FdtBuffers fdt{};         // A^(1/2)-correlated noise in the steps (sp_set_fdt_noise)
    int fdt_degree = 0;           // 0: independent noise per particle (the paper's)
    ss::FcgState* fcg = nullptr;  // flexible solve's device state (allocated by its first call)
    ss::FcgState fcg_host{};
    std::string err;
};

// Error propagation inside functions that hold an sp_sim* named s.
#define SS_CUDA(call)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            s->err = std::string(#call) + ": " + cudaGetErrorString(e_);                     \
            return SP_ERR_CUDA;                                                              \
        }                                                                                    \
    } while (0)

#define SS_TRY(expr)                 \
    do {                                \
        int rc_ = (expr);               \
        if (rc_ != SP_OK) return rc_;   \
    } while (0)

namespace ss_host {
ss::Launch launch_of(const sp_sim* s, cudaStream_t st);
bool mixed(const sp_sim* s);
// side/ev (optional): the step's normals run on side beside the pair search
// (ev[2], ev[3]); with split_x also the split of x0 into double-floats right
// after the gather (ev[0], ev[1]; the caller waits for ev[1])
long long enqueue_build(sp_sim* s, cudaStream_t cs, cudaStream_t side = nullptr, cudaEvent_t* ev = nullptr,
                        bool split_x = false);
int read_state(sp_sim* s);
int grow_pairs(sp_sim* s);
int clear_flags(sp_sim* s);
int set_device(sp_sim* s);
void free_graphs(sp_sim* s);
bool warm_from_prev(const sp_sim* s);   // the solve starts from x (previous velocities or the network's guess)
int do_build(sp_sim* s);                // pair list for the current positions (grows storage if needed)
// init, loop, finish and stress of one solve, enqueued on cs
// with_stress = false: the caller launches the stress kernel itself
// x_split: xdf already holds x0 (split beside the build)
int enqueue_solve(sp_sim* s, cudaStream_t cs, bool from_x, bool in_graph, long long* launches,
                  bool with_stress = true, bool x_split = false);
}  // namespace ss_host

std::string& sp_global_error();
