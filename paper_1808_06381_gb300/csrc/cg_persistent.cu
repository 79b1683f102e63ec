// Persistent mixed-precision CG: the whole solve of Eq. algebra (arXiv
// 1808.06381, §Method) in one cooperative launch.
//
// Same iteration as the mixed solver of cg.cu (Jacobi-preconditioned CG: FP32
// SpMV with the direction update fused, FP32 update of r and of the
// correction d, double-float dot products, FP64 residual replacement), but
// the iteration loop runs inside the kernel: a block owns whole windows of
// 256 rows, two grid-wide reductions per iteration, and the CG scalars
// decided by thread 0 of every block from identical totals, so every block
// takes the same decisions.  A block writes the solver vectors of its own
// rows only; its gathers of r (and of x in the FP64 residual) read rows that
// other blocks wrote before the last barrier.
//
// Grid barrier: one arrival counter that only grows during a launch (barrier
// k is passed once k x blocks have arrived; one release-add per block, polled
// with acquire loads), reset by the last block to leave the launch.  After
// the barrier every block sums all blocks' partial sums itself, in one fixed
// order.  The launch is
// cooperative (all blocks resident), and every wait is bounded by the global
// timer: a block that waits longer than the simulation's wait limit
// (DevState::bar_timeout_ns, 2 s unless sp_set_wait_limit changed it) sets
// SP_ERR_TIMEOUT and leaves the solve, so no GPU can hang on it.
#include <math.h>

#include <mutex>

#include "internal.cuh"

namespace ss {

namespace {


struct PShared {
    float2 df[32];
    double d[32];
    float2 dfk[2][32];   // per-warp sums of the grid reductions
    double dk[4][32];
    double bcast[4];
    float bcastf[2];     // the same totals rounded to FP32 (the on-chip iteration's scalars)
    int flag;
    // decided by thread 0 (FP64 scalars once per block, not once per thread)
    float alpha_f, beta_f;
    int action;   // 0 continue, 1 replace the residual, 2 stop
    // thread 0's CG state, kept here rather than in every thread's registers
    double rho, rr_restart, bnorm2, last_res;
    double alpha_d, beta_d;   // the pipelined FP64 solve's scalars (its reductions overwrite bcast)
    float rho_f, target_f;   // on-chip iteration: rho and its stopping target in FP32
    int iter, restarts, status;
};

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_add_release_gpu(unsigned int* p, unsigned int v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Arrival at barrier k of the launch by thread 0 (target = k x blocks): one
// release-add on a counter that only grows during the launch, then polls
// until it reaches the target.  No block releases the others, so the wait
// after the last arrival is one poll.  The writes of every thread of every
// block before the barrier are visible to every thread after it (release by
// each arrival, acquire by the polls, block barriers on both sides).  Returns
// 0, or SP_ERR_TIMEOUT (also raised in st->error) when the wait ran past the
// simulation's limit.  The solvers take every other stopping decision
// identically in every block from identical totals, so nothing else has to
// travel with the barrier; a block that timed out leaves, and the others time
// out at the next barrier it misses.
__device__ __forceinline__ int barrier_thread0(DevState* st, unsigned int target)
{
    red_add_release_gpu(&st->bar_count, 1u);
    const unsigned long long t0 = global_ns();
    const unsigned long long limit = st->bar_timeout_ns;   // set by the host between launches
    for (;;) {
        if (ld_acquire_gpu(&st->bar_count) >= target) return 0;
        if (global_ns() - t0 > limit) {   // a timer read per poll: polls are L2 round trips anyway
            atomicCAS(&st->error, 0, (int)SP_ERR_TIMEOUT);
            return (int)SP_ERR_TIMEOUT;
        }
    }
}

// Every block of a launch leaves through here (with its system's state and
// block count): the last one to leave, when no block polls the counter any
// more, resets the barrier for the next launch.
__device__ __forceinline__ void barrier_leave(DevState* st, int nb)
{
    __syncthreads();
    if (threadIdx.x == 0 && atomicAdd(&st->bar_exit, 1u) == (unsigned)nb - 1) {
        st->bar_count = 0u;
        st->bar_exit = 0u;
    }
}

// Grid barrier (the blocks of one system).  Returns false when the solve
// must stop (an error was raised anywhere, including a barrier timeout).
__device__ __forceinline__ bool grid_sync(DevState* st, unsigned int& gen, PShared& sh, int nb)
{
    __syncthreads();
    if (threadIdx.x == 0) sh.flag = barrier_thread0(st, (gen + 1u) * (unsigned int)nb);
    __syncthreads();
    gen += 1u;
    return sh.flag == 0;
}

// Grid-wide sums of K double-float values: every block publishes its block
// sums, passes the barrier, then sums all blocks' partials itself, in the
// same fixed order in every block (so all blocks hold identical totals).
// The K values go through one warp-level pass each and one block barrier;
// warp 0 alone forms the block's sums, arrives, and sums the other blocks'
// partials after the release, so a reduction costs two block barriers.
// Consecutive calls must use alternating partial sets: a block may still be
// reading one set when a faster block writes the next.
constexpr int kPartialsPerLane = 8;   // covers grids of up to 256 blocks in one round of loads

struct NoPost {
    template <class T>
    __device__ void operator()(const T&) const {}
};

// post(totals) runs on thread 0 before the closing block barrier, so the
// scalars it derives are visible to every thread when the call returns.
template <int K, class OutT, class Post = NoPost>
__device__ __forceinline__ bool grid_allreduce_df(DevState* st, unsigned int& gen, PShared& sh,
                                                  const dfloat (&v)[K], float2* partials, OutT (&out)[K],
                                                  int bid, int nb, Post post = Post())
{
    static_assert(K <= 2, "two values at most");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    dfloat w[K];
    constexpr bool f32 = sizeof(OutT) == sizeof(float);
    // FP32 totals (the iteration's scalars): every level of the sums in FP32
    // (trees and short runs, ~1e-6 of the summed magnitudes; the scalars are
    // FP32 anyway), in one fixed order, so every block holds the same totals
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if constexpr (f32) {
            float f = __fadd_rn(v[k].hi, v[k].lo);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
            w[k] = dfloat{f, 0.f};
        } else {
            w[k] = warp_sum_df(v[k]);
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) sh.dfk[k][warp] = make_float2(w[k].hi, w[k].lo);
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float2 a = lane < nw ? sh.dfk[k][lane] : make_float2(0.f, 0.f);
            if constexpr (f32) {
                float f = a.x;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
                w[k] = dfloat{f, 0.f};
            } else {
                w[k] = warp_sum_df(dfloat{a.x, a.y});
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) partials[k * kMaxPartials + bid] = make_float2(w[k].hi, w[k].lo);
            sh.flag = barrier_thread0(st, (gen + 1u) * (unsigned int)nb);
        }
        __syncwarp();   // orders thread 0's acquire before the other lanes' loads
        // all of a lane's loads are issued before the first sum (one latency)
        if constexpr (f32) {   // the blocks' FP32 sums, summed in FP32 in a fixed order
            float pv[K][kPartialsPerLane];   // the high parts only (the low ones are 0)
#pragma unroll
            for (int k = 0; k < K; ++k)
#pragma unroll
                for (int u = 0; u < kPartialsPerLane; ++u) {
                    const int b = lane + 32 * u;
                    pv[k][u] = b < nb ? __ldcg(&partials[k * kMaxPartials + b].x) : 0.f;
                }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                float a = 0.f;
#pragma unroll
                for (int u = 0; u < kPartialsPerLane; ++u) a += pv[k][u];
                for (int b = lane + 32 * kPartialsPerLane; b < nb; b += 32) a += __ldcg(&partials[k * kMaxPartials + b].x);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                if (lane == 0) sh.bcastf[k] = a;   // no FP64 operation on the iteration's path
            }
        } else {
            float2 pv[K][kPartialsPerLane];
#pragma unroll
            for (int k = 0; k < K; ++k)
#pragma unroll
                for (int u = 0; u < kPartialsPerLane; ++u) {
                    const int b = lane + 32 * u;
                    pv[k][u] = b < nb ? __ldcg(partials + k * kMaxPartials + b) : make_float2(0.f, 0.f);
                }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                dfloat a{0.f, 0.f};
#pragma unroll
                for (int u = 0; u < kPartialsPerLane; ++u) a = df_add(a, dfloat{pv[k][u].x, pv[k][u].y});
                for (int b = lane + 32 * kPartialsPerLane; b < nb; b += 32) {
                    const float2 p = __ldcg(partials + k * kMaxPartials + b);
                    a = df_add(a, dfloat{p.x, p.y});
                }
                a = warp_sum_df(a);
                if (lane == 0) sh.bcast[k] = (double)a.hi + (double)a.lo;
            }
        }
        if (lane == 0) {
            OutT t[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if constexpr (sizeof(OutT) == sizeof(float))
                    t[k] = sh.bcastf[k];
                else
                    t[k] = sh.bcast[k];
            }
            post(t);
        }
    }
    __syncthreads();
    gen += 1u;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if constexpr (sizeof(OutT) == sizeof(float))
            out[k] = sh.bcastf[k];
        else
            out[k] = sh.bcast[k];
    }
    return sh.flag == 0;
}

template <int K>
__device__ __forceinline__ bool grid_allreduce(DevState* st, unsigned int& gen, PShared& sh,
                                               const dfloat (&v)[K], float2* partials, double (&out)[K],
                                               int bid, int nb)
{
    return grid_allreduce_df<K, double>(st, gen, sh, v, partials, out, bid, nb);
}

// The same for FP64 values (the rare FP64 residual replacement).
template <int K>
__device__ __forceinline__ bool grid_allreduce(DevState* st, unsigned int& gen, PShared& sh,
                                               const double (&v)[K], double* partials, double (&out)[K],
                                               int bid, int nb)
{
    static_assert(K <= 4, "four values at most");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] = warp_sum(v[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) sh.dk[k][warp] = w[k];
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k) w[k] = warp_sum(lane < nw ? sh.dk[k][lane] : 0.0);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) partials[k * kMaxPartials + bid] = w[k];
            sh.flag = barrier_thread0(st, (gen + 1u) * (unsigned int)nb);
        }
        __syncwarp();
        double pv[K][kPartialsPerLane];
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int u = 0; u < kPartialsPerLane; ++u) {
                const int b = lane + 32 * u;
                pv[k][u] = b < nb ? __ldcg(partials + k * kMaxPartials + b) : 0.0;
            }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double a = 0.0;
#pragma unroll
            for (int u = 0; u < kPartialsPerLane; ++u) a += pv[k][u];
            for (int b = lane + 32 * kPartialsPerLane; b < nb; b += 32) a += __ldcg(partials + k * kMaxPartials + b);
            a = warp_sum(a);
            if (lane == 0) sh.bcast[k] = a;
        }
    }
    __syncthreads();
    gen += 1u;
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = sh.bcast[k];
    return sh.flag == 0;
}

// s = sum_j w_ij D^-1_j r_j (FP32).  Rows of r written by other blocks before
// the last barrier are visible to plain loads (the barrier's acquire orders
// them), so the gathers may hit L1: rows of neighbouring particles are
// gathered by many rows of the same block.
template <int KB, bool PIPE>
__device__ __forceinline__ void p_row_sum32(const int* __restrict__ col, const float* __restrict__ val,
                                            const float4* r, int e0, int e1, float& s0, float& s1, float& s2)
{
    s0 = s1 = s2 = 0.f;
    int j[KB];
    float w[KB];
    auto load_batch = [&](int eb, int (&jj)[KB], float (&ww)[KB]) {
#pragma unroll
        for (int u = 0; u < KB; ++u) {
            const int e = eb + 32 * u;
            jj[u] = 0;
            ww[u] = 0.f;
            if (e < e1) {
                jj[u] = ld_stream(col + e);
                ww[u] = ld_stream(val + e);
            }
        }
    };
    if (PIPE) load_batch(e0, j, w);
    for (int eb = e0; eb < e1; eb += 32 * KB) {
        if (!PIPE) load_batch(eb, j, w);
        float4 g[KB];
#pragma unroll
        for (int u = 0; u < KB; ++u) {
            g[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (w[u] != 0.f) g[u] = r[j[u]];
        }
        // PIPE: the next batch's columns and weights are requested while this
        // batch's gathers are in flight, so each batch waits one latency, not two
        float wc[KB];
#pragma unroll
        for (int u = 0; u < KB; ++u) wc[u] = w[u];
        if (PIPE) load_batch(eb + 32 * KB, j, w);
#pragma unroll
        for (int u = 0; u < KB; ++u) {
            const float ww = wc[u] * g[u].w;
            s0 = fmaf(ww, g[u].x, s0);
            s1 = fmaf(ww, g[u].y, s1);
            s2 = fmaf(ww, g[u].z, s2);
        }
    }
}

// ---- matrix-free SpMV (the streaming solve's inner iteration without the
// stored weights).  The weight of Eq. algebra's pair term, w_ij =
// exp(-|R_ij|^2 / 2 lambda^2) (§Method; the pair list, and with it the 5 %
// truncation, is the assembly's), recomputed in FP32 from the positions in
// 32-bit fixed point of each box edge (one unit L / 2^32, ~3e-8 of a
// particle spacing at the benchmark's densities).  Differences of fixed-point
// coordinates wrap modulo 2^32, which is the periodic minimum image in x and
// z; in y the wrap also yields the Lees-Edwards image crossing m (-1, 0, 1),
// whose x shift m delta is a fixed-point constant of the step, so the
// separation is exact integer arithmetic up to the positions' rounding.  A
// pair of the list lies within r_c < L / 2 of every edge, so the wrapped
// image is the pair's image.  The weights agree with the assembled ones to
// ~3e-7 (relative); the residual replacements use the assembled double-float
// weights, so the solve still meets its tolerance on the assembled system.
__device__ __forceinline__ unsigned int fixed_coord(double x, double inv)
{
    return (unsigned int)(unsigned long long)__double2ll_rn(x * inv);   // x in [0, L): modulo 2^32
}

// delta / L_x in fixed point (modulo 2^32)
__device__ __forceinline__ unsigned int fixed_shift(double delta, const KParams& P)
{
    const double f = delta / P.L[0];
    return (unsigned int)(unsigned long long)__double2ll_rn((f - floor(f)) * 4294967296.0);
}

__device__ __forceinline__ float pair_weight_fixed(uint4 a, uint4 b, unsigned int dfix, const KParams& P)
{
    const int dy = (int)(a.y - b.y);
    const int m = (int)(((long long)a.y - (long long)b.y - (long long)dy) >> 32);   // y images crossed
    const int dx = (int)(a.x - b.x - (unsigned int)m * dfix);
    const int dz = (int)(a.z - b.z);
    const float fx = (float)dx * P.fix_scale[0], fy = (float)dy * P.fix_scale[1], fz = (float)dz * P.fix_scale[2];
    return exp2f(P.w_exp2 * fmaf(fx, fx, fmaf(fy, fy, fz * fz)));
}

// s = sum_j w_ij D^-1_j r_j (FP32) with w_ij recomputed from the fixed-point
// positions pf; the row's padding entries (column = the row itself) are
// skipped.  r gathers through plain loads (other blocks wrote it before the
// last barrier), the positions through the read-only path.
template <int KB, bool PIPE>
__device__ __forceinline__ void p_row_sum32_mf(const KParams& P, const int* __restrict__ col, const float4* r,
                                               const uint4* __restrict__ pf, uint4 pi, int row, unsigned int dfix,
                                               int e0, int e1, float& s0, float& s1, float& s2)
{
    s0 = s1 = s2 = 0.f;
    int j[KB];
    auto load_batch = [&](int eb, int (&jj)[KB]) {
#pragma unroll
        for (int u = 0; u < KB; ++u) {
            const int e = eb + 32 * u;
            jj[u] = e < e1 ? ld_stream(col + e) : row;
        }
    };
    if (PIPE) load_batch(e0, j);
    for (int eb = e0; eb < e1; eb += 32 * KB) {
        if (!PIPE) load_batch(eb, j);
        float4 g[KB];
        uint4 q[KB];
        bool on[KB];
#pragma unroll
        for (int u = 0; u < KB; ++u) {
            on[u] = j[u] != row;
            g[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            q[u] = pi;
            if (on[u]) {
                g[u] = r[j[u]];
                q[u] = __ldg(pf + j[u]);
            }
        }
        if (PIPE) load_batch(eb + 32 * KB, j);
#pragma unroll
        for (int u = 0; u < KB; ++u) {
            if (!on[u]) continue;
            const float ww = pair_weight_fixed(pi, q[u], dfix, P) * g[u].w;
            s0 = fmaf(ww, g[u].x, s0);
            s1 = fmaf(ww, g[u].y, s1);
            s2 = fmaf(ww, g[u].z, s2);
        }
    }
}

// The fixed-point positions of the rows (from the double-float positions of
// the step's assembly).
__global__ void k32_pos_fixed(KParams P, DevBuffers B)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const int np = P.npad;
    uint4 q;
    q.x = fixed_coord((double)B.pos32[i] + (double)B.pos32lo[i], P.fix_inv[0]);
    q.y = fixed_coord((double)B.pos32[np + i] + (double)B.pos32lo[np + i], P.fix_inv[1]);
    q.z = fixed_coord((double)B.pos32[2 * np + i] + (double)B.pos32lo[2 * np + i], P.fix_inv[2]);
    q.w = 0u;
    B.posfix[i] = q;
}

}  // namespace

// x += d of one row in double-float (the correction d accumulated in FP32
// since the last fold).
__device__ __forceinline__ void fold_correction(const DevBuffers& B, int i, float4 d)
{
    const float4 xh = B.xdf[2 * i], xl = B.xdf[2 * i + 1];
    const dfloat a = df_add(dfloat{xh.x, xl.x}, d.x), b = df_add(dfloat{xh.y, xl.y}, d.y),
                 c = df_add(dfloat{xh.z, xl.z}, d.z);
    B.xdf[2 * i] = make_float4(a.hi, b.hi, c.hi, 0.f);
    B.xdf[2 * i + 1] = make_float4(a.lo, b.lo, c.lo, 0.f);
}

// The true residual r = b - A x of one row (slot of the sliced layout) in
// double-float; returns (fp32(r), D^-1) and |fp32(r)|^2 in rs.
template <int KB>
__device__ __forceinline__ float4 true_residual_row(const KParams& P, const DevBuffers& B, int slot, int row,
                                                    float& rs)
{
    dfloat s[3], r[3];
    row_sum_df<KB>(B.col, B.val32, B.val32lo, B.xdf, B.chunk_off[slot >> 5] + (slot & 31),
                   B.chunk_off[(slot >> 5) + 1], s);
    residual_df(P, B, row, s, r);
    rs = r[0].hi * r[0].hi + r[1].hi * r[1].hi + r[2].hi * r[2].hi;
    return make_float4(r[0].hi, r[1].hi, r[2].hi, B.dinv32[row]);
}

// The solution of one row in FP64 from its double-float form.
__device__ __forceinline__ void store_x64(const DevBuffers& B, int np, int i)
{
    const float4 xh = B.xdf[2 * i], xl = B.xdf[2 * i + 1];
    B.x[i] = (double)xh.x + (double)xl.x;
    B.x[np + i] = (double)xh.y + (double)xl.y;
    B.x[2 * np + i] = (double)xh.z + (double)xl.z;
}

// Slot of thread t (0..255 of its window group) in the group's k-th window.
// The chunks of a window hold rows of decreasing length; warp c takes chunk c
// of even windows and chunk 7 - c of odd ones, so a warp's rows over two
// windows have about equal total length (the slowest warp sets the pace of
// every phase).
__device__ __forceinline__ int chunk_lane(int k, int t)
{
    return (k & 1) ? (t ^ 0xE0) : t;
}

// The solve of one system by blocks bid = 0..nb-1 of the launch (all of the
// launch for a single system; a share of it in a batch).  Expects r4 = (r, D^-1)
// with r = b - A x, p4 = q4 = d4 = 0 and the scalars, from the set-up kernel.
// A block of 256 G threads is G window groups of 256; group g takes the
// block's windows wb + g, wb + g + G, ... (one row per thread and window).
template <int KB, bool PIPE, bool MF = false>
__device__ __forceinline__ void persistent_solve(const KParams& P, const DevBuffers& B, int bid, int nb,
                                                 PShared& sh)
{
    DevState* st = B.st;
    if (threadIdx.x == 0) sh.flag = 0;
    __syncthreads();
    if (st->error | st->overflow | st->done) return;   // uniform: set before the launch
    unsigned int gen = 0u;   // barriers passed in this launch (the counter starts at 0)

    const int nwin = P.nslots / 256;
    const int wb = (int)((long long)bid * nwin / nb);
    const int we = (int)((long long)(bid + 1) * nwin / nb);
    const int G = blockDim.x >> 8;                              // window groups
    const int t = threadIdx.x & 255, wg = wb + (threadIdx.x >> 8);   // lane in window, first window
    const int np = P.npad;
    const float alpha_e = (float)P.alpha;
    const unsigned int dfix = MF ? fixed_shift(st->delta, P) : 0u;

    // CG scalars: thread 0 keeps them in FP64 and makes every decision; the
    // other threads see the FP32 step lengths and the action code.
    if (threadIdx.x == 0) {
        sh.rho = st->rho;
        sh.rr_restart = st->rr_restart;
        sh.bnorm2 = st->bnorm2;
        sh.last_res = st->last_res;
        sh.iter = 0;
        sh.restarts = 0;
        sh.status = SP_OK;
        sh.beta_f = 0.f;
    }
    __syncthreads();

    // partial-sum sets: set 0 for p.q, 1-2 for r.r and r.z, the FP64 array for
    // the true residual; a block still reading one set after a barrier is
    // never overtaken by a faster block writing the same set (its next write
    // lies behind at least one more barrier)
    for (;;) {
        // ---- SpMV with the fused direction update; p.q
        dfloat pq{0.f, 0.f};
        const float betaf = sh.beta_f;
        // the row and entry range of the next window are loaded while this one
        // is processed (they do not change during the solve)
        int slot = wg * 256 + chunk_lane(0, t);
        int row = wg < we ? B.slot_row[slot] : -1;
        int e0 = wg < we ? B.chunk_off[slot >> 5] + (slot & 31) : 0;
        int e1 = wg < we ? B.chunk_off[(slot >> 5) + 1] : 0;
        for (int w = wg, k = 0; w < we; w += G, ++k) {
            int nrow = -1, ne0 = 0, ne1 = 0;
            if (w + G < we) {
                const int ns = (w + G) * 256 + chunk_lane(k + 1, t);
                nrow = B.slot_row[ns];
                ne0 = B.chunk_off[ns >> 5] + (ns & 31);
                ne1 = B.chunk_off[(ns >> 5) + 1];
            }
            if (row >= 0) {
                const float4 ri = B.r4[row];
                const float d = __ldg(B.diag32 + row);
                float4 qo = make_float4(0.f, 0.f, 0.f, 0.f), po = qo;
                if (betaf != 0.f) {
                    qo = B.q4[row];
                    po = B.p4[row];
                }
                float s0, s1, s2;
                if constexpr (MF)
                    p_row_sum32_mf<KB, PIPE>(P, B.col, B.r4, B.posfix, B.posfix[row], row, dfix, e0, e1, s0, s1,
                                             s2);
                else
                    p_row_sum32<KB, PIPE>(B.col, B.val32, B.r4, e0, e1, s0, s1, s2);
                const float z0 = ri.w * ri.x, z1 = ri.w * ri.y, z2 = ri.w * ri.z;
                float q0 = fmaf(d, z0, -alpha_e * s0);
                float q1 = fmaf(d, z1, -alpha_e * s1);
                float q2 = fmaf(d, z2, -alpha_e * s2);
                float p0 = z0, p1 = z1, p2 = z2;
                if (betaf != 0.f) {
                    q0 = fmaf(betaf, qo.x, q0);
                    q1 = fmaf(betaf, qo.y, q1);
                    q2 = fmaf(betaf, qo.z, q2);
                    p0 = fmaf(betaf, po.x, p0);
                    p1 = fmaf(betaf, po.y, p1);
                    p2 = fmaf(betaf, po.z, p2);
                }
                B.q4[row] = make_float4(q0, q1, q2, 0.f);
                B.p4[row] = make_float4(p0, p1, p2, 0.f);
                pq = df_add(pq, p0 * q0 + p1 * q1 + p2 * q2);
            }
            row = nrow;
            e0 = ne0;
            e1 = ne1;
        }
        {
            const dfloat v[1] = {pq};
            double tot[1];
            if (!grid_allreduce<1>(st, gen, sh, v, B.partials_df, tot, bid, nb)) break;
            if (threadIdx.x == 0) {
                sh.action = 0;
                if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
                    sh.status = SP_ERR_NONFINITE;
                    sh.action = 2;
                } else {
                    sh.alpha_f = (float)(sh.rho / tot[0]);
                }
            }
        }
        __syncthreads();
        if (sh.action == 2) break;

        // ---- update of d and r (own rows); r.r and r.D^-1 r
        const float af = sh.alpha_f;
        dfloat rr{0.f, 0.f}, rz{0.f, 0.f};
        for (int w = wg; w < we; w += G) {
            const int i = w * 256 + t;
            if (i < P.n) {
                const float4 p = B.p4[i], q = B.q4[i];
                float4 d = B.d4[i], r = B.r4[i];
                d.x = fmaf(af, p.x, d.x);
                d.y = fmaf(af, p.y, d.y);
                d.z = fmaf(af, p.z, d.z);
                r.x = fmaf(-af, q.x, r.x);
                r.y = fmaf(-af, q.y, r.y);
                r.z = fmaf(-af, q.z, r.z);
                B.d4[i] = d;
                B.r4[i] = r;
                const float rs = r.x * r.x + r.y * r.y + r.z * r.z;
                rr = df_add(rr, rs);
                rz = df_add(rz, r.w * rs);
            }
        }
        {
            const dfloat v[2] = {rr, rz};
            double tot[2];
            if (!grid_allreduce<2>(st, gen, sh, v, B.partials_df + kMaxPartials, tot, bid, nb)) break;
            if (threadIdx.x == 0) {
                ++sh.iter;
                sh.action = 0;
                if (!isfinite(tot[0]) || !isfinite(tot[1])) {
                    sh.status = SP_ERR_NONFINITE;
                    sh.action = 2;
                } else {
                    sh.beta_f = (float)(tot[1] / sh.rho);
                    sh.rho = tot[1];
                    const double target = fmax(P.inner2 * sh.rr_restart, kInnerFinal2 * P.tol2 * sh.bnorm2);
                    if (tot[0] <= target || sh.iter >= P.max_iter) sh.action = 1;
                }
            }
        }
        __syncthreads();
        if (sh.action == 2) break;
        if (sh.action == 0) continue;

        // ---- residual replacement: x += d (own rows, double-float), then
        // r = b - A x in double-float
        for (int w = wg; w < we; w += G) {
            const int i = w * 256 + t;
            if (i < P.n) {
                fold_correction(B, i, B.d4[i]);
                B.d4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        if (!grid_sync(st, gen, sh, nb)) break;
        double trr = 0.0, trz = 0.0;
        for (int w = wg, k = 0; w < we; w += G, ++k) {
            const int slot = w * 256 + chunk_lane(k, t);
            const int row = B.slot_row[slot];
            if (row >= 0) {
                float rs;
                const float4 rf = true_residual_row<2>(P, B, slot, row, rs);
                B.r4[row] = rf;
                trr += (double)rs;
                trz += (double)(rf.w * rs);
            }
        }
        {
            const double v[2] = {trr, trz};
            double tot[2];
            if (!grid_allreduce<2>(st, gen, sh, v, B.partials, tot, bid, nb)) break;
            if (threadIdx.x == 0) {
                sh.last_res = sqrt(tot[0] / sh.bnorm2);
                if (bid == 0) st->true_checks += 1;
                sh.action = 0;
                if (!isfinite(tot[0])) {
                    sh.status = SP_ERR_NONFINITE;
                    sh.action = 2;
                } else if (tot[0] <= P.tol2 * sh.bnorm2) {
                    sh.action = 2;   // converged
                } else if (sh.iter >= P.max_iter || sh.restarts >= kMaxCgRestarts + 8) {
                    sh.status = SP_ERR_NOT_CONVERGED;
                    sh.action = 2;
                } else {
                    ++sh.restarts;
                    sh.rho = tot[1];
                    sh.beta_f = 0.f;
                    sh.rr_restart = tot[0];
                }
            }
        }
        __syncthreads();
        if (sh.action == 2) break;
    }
    // the solution in FP64 (own rows)
    for (int w = wg; w < we; w += G) {
        const int i = w * 256 + t;
        if (i < P.n) store_x64(B, np, i);
    }
    // every block's thread 0 holds the same scalars; block 0 records them
    if (bid == 0 && threadIdx.x == 0) {
        st->iter = sh.iter;
        st->restarts = sh.restarts;
        st->last_res = sh.last_res;
        st->done = 1;
        if (st->error == 0 && sh.status != SP_OK) {
            st->status = sh.status;
            st->error = sh.status;
        } else if (st->error != 0) {
            st->status = st->error;
        } else {
            st->status = SP_OK;
        }
    }
}

// ------------------------------------------------------------ on-chip solve
// The same iteration for systems whose rows fit on the chip: a block holds
// one contiguous range of at most 2048 rows within at most kResWindows
// windows, a thread of a block of BS owns at most RPT rows (BS RPT = 2048)
// and keeps their solver vectors (r, p, q, d) in registers for the whole
// solve; the block keeps z = D^-1 r of its rows (D^-1 in the fourth lane) and
// the matrix entries that couple two of its rows (packed words, below) in
// shared memory.  Only the entries that couple its rows to other blocks' rows
// ("halo" entries, about a sixth with the tiled Morton row order) and those
// rows' r are read from global memory in the iteration; an entry is local
// when its column lies in the block's row range.  The set-up at the start of
// the solve sorts each row's entries into the two lists; a chunk whose local
// entries find no room in shared memory keeps all its entries in the halo
// list, and a block whose halo lists do not fit its share of the list buffers
// gathers every entry from copies of its rows' sliced lists (slower, same
// result).
constexpr int kResWindows = 8;                       // 2048 rows per block
constexpr int kResMaxBlocks = 192;                   // blocks the entry-balanced split serves
constexpr int kResChunks = kResWindows * 8;
constexpr int kResHalo = 4;                          // halo gathers in flight per thread
constexpr int kResSetupBatch = 6;                    // entries requested at a time in the set-up
constexpr int kResCheckBatch = 4;                    // gathers in flight in the off-chip blocks' true residual
constexpr int kResCheckLocal = 8;                    // low parts requested at a time in the on-chip check

// A local entry of the on-chip solve in one 32-bit word, so that one
// shared-memory load serves the column and the weight: the column (11 bits:
// a block holds fewer than 2048 rows) and the FP32 weight rounded to 18
// mantissa bits, its exponent in 3 bits (a weight of the 5 % truncation lies
// in (0.05, 1], five binades from 2^-5).  Word 0 is column 0 with weight 0
// (padding); a real weight never encodes as 0.  The iteration's products use
// the rounded weight (2^-19 relative: the inner FP32 solve converges as
// fast); the residual replacements add the stored low part, which the
// placement takes as (w_hi - rounded) + w_lo.
__device__ __forceinline__ unsigned int pack_entry(int col, float w, float& rounded)
{
    unsigned int b = (__float_as_uint(w) + 0x10u) & ~0x1Fu;   // to 18 mantissa bits, to nearest
    const int e = min(max((int)(b >> 23) - 122, 0), 7);
    const unsigned int code = ((unsigned int)e << 18) | ((b >> 5) & 0x3FFFFu);
    rounded = __uint_as_float((((code >> 18) + 122u) << 23) | ((code & 0x3FFFFu) << 5));
    return (unsigned int)col | (code << 11);
}

__device__ __forceinline__ int entry_col(unsigned int word) { return (int)(word & 0x7FFu); }

__device__ __forceinline__ float entry_weight(unsigned int word)
{
    const unsigned int code = word >> 11;
    return code ? __uint_as_float((((code >> 18) + 122u) << 23) | ((code & 0x3FFFFu) << 5)) : 0.f;
}

struct RShared {
    int loff[kResChunks];    // shared-memory offset of the chunk's local entries
    int nloc[kResChunks];    // local entries per row of the chunk (its longest row's count)
    int nhalo[kResChunks];   // halo entries per row of the chunk
    int hoff[kResChunks];    // global offset of the chunk's halo list
    unsigned long long spill;   // chunks whose local entries found no room: all their entries in the halo list
    short bnd[kResMaxBlocks + 1];  // first window of every block (entry-balanced split by windows; < 2^15)
    int rbnd[kResMaxBlocks + 1];   // first row of every block (entry-balanced split by rows)
    int split_ok;
    int nlocal;              // entries of the local lists (every chunk's, padding included)
    int mode;                // 0: on chip; 1: the block's lists did not fit at all, all gathers global
};

__device__ __forceinline__ void res_halo_batch(const DevBuffers& B, int hb, int kb, int nh, float& s0, float& s1,
                                               float& s2)
{
    int j[kResHalo];
    float w[kResHalo];
#pragma unroll
    for (int u = 0; u < kResHalo; ++u) {
        j[u] = 0;
        w[u] = 0.f;
        if (kb + u < nh) {   // L1-cached: every iteration reads the same lists
            j[u] = B.hcol[hb + 32 * (kb + u)];
            w[u] = B.hval[hb + 32 * (kb + u)];
        }
    }
    float4 g[kResHalo];
#pragma unroll
    for (int u = 0; u < kResHalo; ++u) {
        g[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (w[u] != 0.f) g[u] = B.r4[j[u]];
    }
#pragma unroll
    for (int u = 0; u < kResHalo; ++u) {
        const float ww = w[u] * g[u].w;
        s0 = fmaf(ww, g[u].x, s0);
        s1 = fmaf(ww, g[u].y, s1);
        s2 = fmaf(ww, g[u].z, s2);
    }
}

// Thread t owns the rows at positions u BS + t (even u) and u BS + BS - 1 - t
// (odd u), u < RPT, below R, of the block's R rows sorted by halo count,
// then local count, both descending: a warp's 32 rows have about equal
// counts (little padding in either list), and each thread pairs heavier rows
// with lighter ones.
template <int BS, int RPT>
__device__ __forceinline__ void resident_solve(const KParams& P, const DevBuffers& B, int bid, int nb, PShared& sh,
                                               RShared& rs, float4* dyn, int smem_bytes)
{
    DevState* st = B.st;
    const bool fused = P.fused_init != 0;   // the initial residual is formed here
    if (threadIdx.x == 0) sh.flag = 0;
    __syncthreads();
    if (st->error | st->overflow | (fused ? 0 : st->done)) return;   // uniform: set before the launch
    unsigned int gen = 0u;   // barriers passed in this launch (the counter starts at 0)

    const int nwin = P.nslots / 256;
    // The block's rows.  Every block computes the same split of the rows into
    // nb shares with about equal numbers of matrix entries (a sheared run
    // clusters, and its dense regions carry up to ~1.3x the mean entries per
    // row): block b starts where the sliced layout's entry count reaches
    // T_b = b E / nb, at the row interpolated inside that window of 256 rows
    // (a window's rows are spatially compact, so their lengths are similar).
    // A window at a share's edge is read by both blocks, each keeping its own
    // rows.  Where a share would be empty, hold more than 2048 rows or touch
    // more than kResWindows windows, or no separate region exists for the
    // lists of blocks whose entries cannot stay on chip, the shares are whole
    // windows with about equal entries instead (block b from the first window
    // that starts at or after T_b), and failing that equal numbers of windows.
    int wb = (int)((long long)bid * nwin / nb), we = (int)((long long)(bid + 1) * nwin / nb);
    int rb = wb * 256, re = min(we * 256, P.n);
    int hbase = -1, hcap = 0;   // the block's range of the halo lists (set below for the window split)
    {
        const long long E = B.chunk_off[nwin * 8];
        const bool split = nb <= kResMaxBlocks && E > 0;
        for (int b = threadIdx.x; b <= min(nb, kResMaxBlocks); b += BS) {
            rs.bnd[b] = -1;   // every interior boundary is set by the window that holds T_b
            rs.rbnd[b] = -1;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            rs.bnd[0] = 0;
            rs.bnd[min(nb, kResMaxBlocks)] = (short)nwin;
            rs.rbnd[0] = 0;
            rs.rbnd[min(nb, kResMaxBlocks)] = P.n;
        }
        if (split) {
            for (int w = threadIdx.x; w < nwin; w += BS) {
                const long long lo = B.chunk_off[w * 8], hi = B.chunk_off[(w + 1) * 8];
                const int b0 = max(1, (int)(lo * nb / E)), b1 = min(nb - 1, (int)(hi * nb / E) + 1);
                for (int b = b0; b <= b1; ++b) {
                    const long long T = (long long)b * E / nb;
                    if (T > lo && T <= hi) rs.bnd[b] = (short)(w + 1);
                    if (T >= lo && T < hi) rs.rbnd[b] = min(w * 256 + (int)((T - lo) * 256 / (hi - lo)), P.n);
                }
            }
        }
        __syncthreads();
        if (split && threadIdx.x == 0) {
            // a share ends within the kResWindows-th window from the one it
            // starts in (so it holds at most 2048 rows and the rows of a block
            // whose lists cannot stay on chip map to its threads' slots), and
            // leaves at least a row to every later share; boundaries that
            // miss T_b stay monotone, and a share the clamp leaves invalid is
            // caught below
            int prev = 0;   // carried in a register: one dependent chain of integer operations per share
            for (int b = 1; b < nb; ++b) {
                int r = rs.rbnd[b];
                if (r < 0) break;
                r = min(r, (prev / 256 + kResWindows) * 256);
                r = min(r, P.n - (nb - b));
                prev = max(r, prev + 1);
                rs.rbnd[b] = prev;
            }
        }
        __syncthreads();
        int bad_w = !split, bad_r = !split || P.hcopy <= 0;
        if (split)
            for (int b = threadIdx.x; b < nb; b += BS) {
                const int nw = rs.bnd[b + 1] - rs.bnd[b];
                bad_w |= rs.bnd[b] < 0 || nw < 1 || nw > kResWindows;
                const int r0 = rs.rbnd[b], r1 = rs.rbnd[b + 1];
                bad_r |= r0 < 0 || r1 - r0 < 1 || r1 - r0 > kResWindows * 256 ||
                         (r1 + 255) / 256 - r0 / 256 > kResWindows;
            }
        if (!__syncthreads_or(bad_r)) {
            rb = rs.rbnd[bid];
            re = rs.rbnd[bid + 1];
            wb = rb / 256;
            we = (re + 255) / 256;
            hbase = (int)((long long)bid * E / nb);
            hcap = (int)((long long)(bid + 1) * E / nb) - hbase;
        } else if (!__syncthreads_or(bad_w)) {
            wb = rs.bnd[bid];
            we = rs.bnd[bid + 1];
            rb = wb * 256;
            re = min(we * 256, P.n);
        }
        if (hbase < 0) {
            hbase = B.chunk_off[wb * 8];
            hcap = B.chunk_off[we * 8] - hbase;
        }
    }
    const int R = re - rb;                               // the block's rows: rb .. re - 1
    float4* zbuf = dyn;                                  // [R] z of the block's rows (D^-1 in w)
    const int cap = max(smem_bytes - R * (int)sizeof(float4), 0) / 4;
    unsigned int* sent = reinterpret_cast<unsigned int*>(dyn + R);   // packed local entries
    float* __restrict__ rlo = B.rlo + (size_t)bid * kResLoStride;   // low parts of the local weights
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int np = P.npad;
    const float alpha_e = (float)P.alpha;
    // requests in flight per thread in the set-up and in the true residual of
    // blocks whose entries are off chip (the 1024-thread form has half the registers)
    constexpr int KS = BS >= 1024 ? 4 : kResSetupBatch, KC = BS >= 1024 ? 2 : kResCheckBatch;

    // ---- set-up 1: local and halo entry counts of every row of the block
    // (read in slot order, so that a warp's loads are coalesced), sort keys
    // (halo desc, local desc, row asc) sorted by a bitonic network; keys,
    // counts and the inverse permutation borrow the space of zbuf (14 bytes
    // per row of its 16)
    const int t = threadIdx.x & 255, g = threadIdx.x >> 8;
    int npow = 1;
    while (npow < R) npow <<= 1;
    unsigned int* skey = reinterpret_cast<unsigned int*>(zbuf);
    unsigned int* scnt = skey + npow;
    unsigned short* sinv = reinterpret_cast<unsigned short*>(scnt + R);
    for (int i = R + (int)threadIdx.x; i < npow; i += BS) skey[i] = 0xffffffffu;
    // a thread's slots are slot t of the windows wb + g, wb + g + BS / 256, ...
    // (at most kWin of them: every split keeps a block within kResWindows
    // windows); their rows and chunk bounds are requested together
    constexpr int kWin = kResWindows / (BS / 256);
    if (we - wb > kResWindows) {   // never: every split keeps a block within kResWindows windows
        // leave before any row is placed; the other blocks' barrier waits end
        // at their limit, and the solve reports the error
        if (threadIdx.x == 0) atomicCAS(&st->error, 0, (int)SP_ERR_INVALID_ARG);
        return;
    }
    int srow[kWin], sc0[kWin], sc1[kWin];
#pragma unroll
    for (int k = 0; k < kWin; ++k) {
        const int slot = (wb + g + (BS / 256) * k) * 256 + t;
        const bool in = wb + g + (BS / 256) * k < we;
        srow[k] = in ? B.slot_row[slot] : -1;
        sc0[k] = in ? B.chunk_off[slot >> 5] : 0;
        sc1[k] = in ? B.chunk_off[(slot >> 5) + 1] : 0;
    }
#pragma unroll
    for (int k = 0; k < kWin; ++k) {
        const int slot = (wb + g + (BS / 256) * k) * 256 + t;
        const int row = srow[k];
        if (row < rb || row >= re) continue;   // no row, or another block's (a window at a share's edge)
        const int e1 = sc1[k];
        int nl = 0, nh = 0;
        unsigned long long hist = 0ull;   // local entries per bank group (column mod 8), 8 bits each
        // the columns alone: a padding entry of the sliced layout points at its
        // own row (and has weight 0), a real partner never does
        for (int eb = sc0[k] + (slot & 31); eb < e1; eb += 32 * 2 * KS) {
            int j[2 * KS];
#pragma unroll
            for (int u = 0; u < 2 * KS; ++u) {
                const int e = eb + 32 * u;
                j[u] = e < e1 ? ld_stream(B.col + e) : row;
            }
#pragma unroll
            for (int u = 0; u < 2 * KS; ++u) {
                if (j[u] != row) {
                    if (j[u] >= rb && j[u] < re) {
                        ++nl;
                        hist += 1ull << (8 * ((j[u] - rb) & 7));
                    } else {
                        ++nh;
                    }
                }
            }
        }
        const int i = row - rb;
        scnt[i] = (unsigned)nl | ((unsigned)nh << 16);
        B.res_hist[slot] = hist;   // read back by this thread when it places the row's entries
        skey[i] = ((unsigned)(31 - min(nh, 31)) << 17) | ((unsigned)(63 - min(nl, 63)) << 11) | (unsigned)i;
    }
    __syncthreads();
    for (int k = 2; k <= npow; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int h = threadIdx.x; h < npow / 2; h += blockDim.x) {
                const int i = 2 * h - (h & (j - 1)), l = i + j;
                const unsigned int a = skey[i], b = skey[l];
                if ((a > b) == ((i & k) == 0)) {
                    skey[i] = b;
                    skey[l] = a;
                }
            }
            __syncthreads();
        }
    }
    for (int pos = threadIdx.x; pos < R; pos += BS) sinv[skey[pos] & 2047u] = (unsigned short)pos;

    // ---- set-up 2: the own rows, the chunk maxima, the offsets of both lists
    static_assert(BS * RPT == kResWindows * 256 && BS % 256 == 0, "a block holds 2048 rows");
    int row[RPT];
    {
        int cl[RPT], ch[RPT];
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            const int pos = u * BS + ((u & 1) ? BS - 1 - (int)threadIdx.x : (int)threadIdx.x);
            const bool own = pos < R;
            row[u] = -1;
            cl[u] = ch[u] = 0;
            if (own) {
                const int i = (int)(skey[pos] & 2047u);
                row[u] = rb + i;
                cl[u] = (int)(scnt[i] & 0xffffu);
                ch[u] = (int)(scnt[i] >> 16);
            }
            const int ml = __reduce_max_sync(0xffffffffu, cl[u]);
            const int mh = __reduce_max_sync(0xffffffffu, ch[u]);
            if (lane == 0) {
                rs.nloc[u * (BS / 32) + warp] = ml;
                rs.nhalo[u * (BS / 32) + warp] = mh;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // a chunk whose local entries find no room in shared memory keeps them
        // in its halo list (gathered from global memory, like the entries to
        // other blocks); the other chunks stay on chip
        int lo = 0, ho = 0;
        unsigned long long spill = 0ull;
        for (int c = 0; c < kResChunks; ++c) {
            rs.loff[c] = lo;
            if (lo + 32 * rs.nloc[c] > cap) {
                spill |= 1ull << c;
                rs.nhalo[c] += rs.nloc[c];
                rs.nloc[c] = 0;
            }
            lo += 32 * rs.nloc[c];
            rs.hoff[c] = hbase + ho;
            ho += 32 * rs.nhalo[c];
        }
        rs.spill = spill;
        rs.nlocal = lo;
        rs.mode = ho <= hcap ? 0 : 1;
        if (rs.mode != 0) {
            // the halo lists cannot hold the block's entries: every entry is
            // gathered, from lists that are the sliced layout's own (each row's
            // entries copied below to the same positions, offset by hcopy),
            // each thread's rows those of its own slots (chunk_lane)
            for (int c = 0; c < kResChunks; ++c) {
                const int u = c / (BS / 32), wp = c % (BS / 32);
                const int w = wb + (wp >> 3) + (BS / 256) * u;
                rs.loff[c] = 0;
                rs.nloc[c] = 0;
                rs.hoff[c] = hbase;
                rs.nhalo[c] = 0;
                if (w < we) {
                    const int sc = w * 8 + ((u & 1) ? (wp & 7) ^ 7 : (wp & 7));
                    rs.hoff[c] = (int)P.hcopy + B.chunk_off[sc];
                    rs.nhalo[c] = (B.chunk_off[sc + 1] - B.chunk_off[sc]) / 32;
                }
            }
            rs.nlocal = 0;
        }
        const int off = (rs.mode != 0 || spill != 0ull) ? 1 : 0;   // some or all entries gathered globally
        if (fused)   // summed by block 0 at the end (the counter is not reset before this launch)
            B.partials[3 * kMaxPartials + bid] = (double)off;
        else if (off)
            atomicAdd(&st->res_offchip, 1);
    }
    __syncthreads();
    const bool onchip = rs.mode == 0;
    if (onchip) {   // lanes of the last chunk without a row keep these (column 0, weight 0)
        for (int e = threadIdx.x; e < rs.nlocal; e += BS) {
            sent[e] = 0u;
        }
        __syncthreads();   // before any entry is placed
    }
    if (!onchip) {   // the sliced layout's own assignment and lists, every gather global
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            const int w = wb + g + (BS / 256) * u;
            const int slot = w * 256 + chunk_lane(u, t);
            row[u] = w < we ? B.slot_row[slot] : -1;
            if (row[u] < rb || row[u] >= re) row[u] = -1;   // a window at the edge of a row share
            if (row[u] < 0) continue;
            const int e1 = B.chunk_off[(slot >> 5) + 1];
            for (int e = B.chunk_off[slot >> 5] + (slot & 31); e < e1; e += 32) {
                B.hcol[P.hcopy + e] = B.col[e];
                B.hval[P.hcopy + e] = B.val32[e];
                B.hlo[P.hcopy + e] = B.val32lo[e];
            }
        }
    }

    // the initial residual of the fused form, row by row: r = b - (A_ii x0 -
    // alpha s) from the row's double-float sum s (x0 from xdf), or r = b with
    // x = 0; r4, rdf and the sums ||b||^2, r.r, r.D^-1 r
    double bb = 0.0, rr0 = 0.0, rz0 = 0.0;
    auto init_row = [&](int rw, const dfloat (&sd)[3]) {
        dfloat rd[3];
        if (P.fused_init == 2) {
            residual_df(P, B, rw, sd, rd);
        } else {
            const float4 bh = B.bdf[2 * rw], bl = B.bdf[2 * rw + 1];
            rd[0] = dfloat{bh.x, bl.x};
            rd[1] = dfloat{bh.y, bl.y};
            rd[2] = dfloat{bh.z, bl.z};
            B.xdf[2 * rw] = make_float4(0.f, 0.f, 0.f, 0.f);
            B.xdf[2 * rw + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int c = 0; c < 3; ++c) B.x[c * np + rw] = 0.0;
        }
        const float di = B.dinv32[rw];
        const float4 bh = B.bdf[2 * rw];
        bb += (double)(bh.x * bh.x + bh.y * bh.y + bh.z * bh.z);
        const float rsq = rd[0].hi * rd[0].hi + rd[1].hi * rd[1].hi + rd[2].hi * rd[2].hi;
        B.r4[rw] = make_float4(rd[0].hi, rd[1].hi, rd[2].hi, di);
        B.rdf[2 * rw] = make_float4(rd[0].hi, rd[1].hi, rd[2].hi, 0.f);
        B.rdf[2 * rw + 1] = make_float4(rd[0].lo, rd[1].lo, rd[2].lo, 0.f);
        rr0 += (double)rsq;
        rz0 += (double)(di * rsq);
    };
    const bool from_x = P.fused_init == 2;

    // ---- set-up 3: place the entries (read in slot order; each row's lists
    // go to the chunk and lane of the thread that owns the row); in the fused
    // form the same pass sums A x0 for the initial residual
    if (onchip) {
        for (int w = wb + g; w < we; w += BS / 256) {
            const int slot = w * 256 + t;
            const int row = B.slot_row[slot];
            if (row < rb || row >= re) continue;
            const int pos = sinv[row - rb];
            const int u = pos / BS, rem = pos - u * BS;
            const int owner = (u & 1) ? BS - 1 - rem : rem;
            const int c = u * (BS / 32) + (owner >> 5);
            const int lo = rs.loff[c] + (owner & 31), nl = rs.nloc[c], nh = rs.nhalo[c];
            const int hb = rs.hoff[c] + (owner & 31);
            const int e1 = B.chunk_off[(slot >> 5) + 1];
            const bool spilled = (rs.spill >> c) & 1ull;   // every entry of the row to its halo list
            // The order of the row's local entries.  Its owner reads entry k
            // in step k of the local sums together with the other 7 lanes of
            // its quarter warp (one 16-byte gather of z each; lanes that hit
            // the same 16-byte bank group, column mod 8, at different columns
            // are served one after another).  Entry positions k whose group is
            // (k + l) mod 8, l the owner's lane in its quarter, keep the
            // quarter's gathers of a step on 8 different groups: each group's
            // entries take its positions k = (g - l) mod 8 + 8 m first, the
            // rest fill the positions left over, lowest first, in column
            // order.  Position k < nlr belongs to group (k + l) mod 8 as its
            // (k / 8)-th; it is left over when that group has at most k / 8
            // entries (E, counted in set-up 1, 8 bits per group).  M counts
            // the entries placed per group (4 bits, saturating: a group has at
            // most 8 positions below 64).  The left-over positions are a 64-bit
            // mask: a row of more than 64 local entries keeps column order.
            const int nlr = (int)(scnt[row - rb] & 0xffffu), ql = owner & 7;
            const bool bank_order = nlr <= 64;
            unsigned long long free_pos = 0ull;
            {   // group h's positions from its E_h-th on: every 8th bit from (h - l) mod 8 + 8 E_h
                const unsigned long long E = B.res_hist[slot];
#pragma unroll
                for (int h = 0; h < 8; ++h) {
                    const int k0 = ((h - ql) & 7) + 8 * (int)((E >> (8 * h)) & 0xffull);
                    if (k0 < 64) free_pos |= 0x0101010101010101ull << k0;
                }
                free_pos &= nlr >= 64 ? ~0ull : (1ull << nlr) - 1ull;
            }
            unsigned int M = 0u;
            int kl = 0, kh = 0;
            auto local_pos = [&](int gg) {   // position of the next local entry of group gg
                if (!bank_order) return kl;
                const int m = (int)((M >> (4 * gg)) & 15u);
                if (m < 15) M += 1u << (4 * gg);
                const int d = (gg - ql) & 7;
                if (d + 8 * m < nlr) return d + 8 * m;
                // as many positions are left over as entries go beyond their
                // group's, so a bit is set (0 keeps even a miscount in bounds)
                const int k = max(__ffsll((long long)free_pos) - 1, 0);
                free_pos &= free_pos - 1ull;
                return k;
            };
            dfloat sd[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            for (int eb = B.chunk_off[slot >> 5] + (slot & 31); eb < e1; eb += 32 * KS) {
                int j[KS];
                float v[KS], vl[KS];
#pragma unroll
                for (int u = 0; u < KS; ++u) {
                    const int e = eb + 32 * u;
                    j[u] = e < e1 ? ld_stream(B.col + e) : 0;
                    v[u] = e < e1 ? ld_stream(B.val32 + e) : 0.f;
                    vl[u] = e < e1 ? ld_stream(B.val32lo + e) : 0.f;
                }
                if (from_x) {   // the row's sum of w_ij x0_j (as row_sum_df)
                    float4 xh[KS], xl[KS];
#pragma unroll
                    for (int u = 0; u < KS; ++u) {
                        xh[u] = xl[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (v[u] != 0.f) {
                            xh[u] = B.xdf[2 * j[u]];
                            xl[u] = B.xdf[2 * j[u] + 1];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < KS; ++u) {
                        const dfloat wd{v[u], vl[u]};
                        sd[0] = df_add(sd[0], df_mul(wd, dfloat{xh[u].x, xl[u].x}));
                        sd[1] = df_add(sd[1], df_mul(wd, dfloat{xh[u].y, xl[u].y}));
                        sd[2] = df_add(sd[2], df_mul(wd, dfloat{xh[u].z, xl[u].z}));
                    }
                }
#pragma unroll
                for (int u = 0; u < KS; ++u) {
                    if (v[u] == 0.f) continue;
                    if (!spilled && j[u] != row && j[u] >= rb && j[u] < re) {   // as counted in set-up 1
                        const int k = local_pos((j[u] - rb) & 7);
                        float vr;
                        sent[lo + 32 * k] = pack_entry(j[u] - rb, v[u], vr);
                        rlo[lo + 32 * k] = __fadd_rn(__fsub_rn(v[u], vr), vl[u]);   // v - vr exact
                        ++kl;
                    } else {
                        B.hcol[hb + 32 * kh] = j[u];
                        B.hval[hb + 32 * kh] = v[u];
                        B.hlo[hb + 32 * kh] = vl[u];
                        ++kh;
                    }
                }
            }
            for (; kl < nl; ++kl) {   // padding: weight 0 at a record of the position's own bank group
                sent[lo + 32 * kl] = (unsigned int)(R >= 8 ? (kl + ql) & 7 : 0);   // weight 0
                rlo[lo + 32 * kl] = 0.f;
            }
            for (; kh < nh; ++kh) {
                B.hcol[hb + 32 * kh] = row;
                B.hval[hb + 32 * kh] = 0.f;
                B.hlo[hb + 32 * kh] = 0.f;
            }
            if (fused) init_row(row, sd);
        }
    }
    __syncthreads();   // sinv (in zbuf) is read until here
    if (onchip) {
        // every local column indexes one of the block's rows; an entry that
        // does not (a broken invariant of the placement) is neutralised and
        // raises an error rather than read outside zbuf
        int bad = 0;
        for (int e = threadIdx.x; e < rs.nlocal; e += BS) {
            if (entry_col(sent[e]) >= R) {
                sent[e] = 0u;
                bad = 1;
            }
        }
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(&st->error, 0, (int)SP_ERR_INVALID_ARG);
    }

    // ---- the initial residual (fused form): r = b - A x0 in double-float, or
    // r = b with x = 0, for the block's rows in slot order, with ||b||^2,
    // r.r and r.D^-1 r summed over the grid (as the initial-residual kernel)
    bool start_done = false;
    double init_tot[3] = {0.0, 0.0, 0.0};
    if (fused) {
        if (threadIdx.x == 0) {
            sh.status = SP_OK;
            sh.last_res = 0.0;
        }
        if (!onchip) {   // the placement pass did not run: the rows' sums here
            for (int w = wb + g, k = 0; w < we; w += BS / 256, ++k) {
                const int slot = w * 256 + chunk_lane(k, t);
                const int rw = B.slot_row[slot];
                if (rw < rb || rw >= re) continue;
                dfloat sd[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
                if (from_x)
                    row_sum_df<KC>(B.col, B.val32, B.val32lo, B.xdf, B.chunk_off[slot >> 5] + (slot & 31),
                                   B.chunk_off[(slot >> 5) + 1], sd);
                init_row(rw, sd);
            }
        }
        const double v[3] = {bb, rr0, rz0};
        if (!grid_allreduce<3>(st, gen, sh, v, B.partials, init_tot, bid, nb)) start_done = true;
        if (threadIdx.x == 0 && !start_done) {
            sh.status = SP_OK;
            sh.action = 0;
            sh.last_res = 1.0;
            const double bb2 = init_tot[0], rr2 = init_tot[1];
            if (!isfinite(bb2) || !isfinite(rr2)) {
                sh.status = SP_ERR_NONFINITE;
                sh.action = 2;
            } else if (bb2 == 0.0) {
                sh.action = 2;   // b = 0: the solution is v = 0 (written by the finishing kernel)
                sh.last_res = 0.0;
            } else if (rr2 <= P.tol2 * bb2) {
                sh.action = 2;   // x0 already meets the tolerance (exact r)
                sh.last_res = sqrt(rr2 / bb2);
            }
            if (bid == 0) {
                st->bnorm2 = bb2;
                st->rr = rr2;
                st->rr_restart = rr2;
                st->rho = init_tot[2];
                st->beta = 0.0;
                st->iter = 0;
                st->restarts = 0;
                st->check_true = 0;
                st->status = 0;
                st->zero_b = (isfinite(bb2) && bb2 == 0.0) ? 1 : 0;
                st->done = 0;
            }
        }
        __syncthreads();
        if (start_done || sh.action == 2) start_done = true;
    }

    // Rows whose r (and d) other blocks gather: on chip, those with an entry
    // to another block's row (pairs are symmetric, so exactly the rows of the
    // other blocks' halo lists; a warp's rows of one index u share their
    // chunk's halo count, sorted first); every row of a block with entries
    // off chip (a spilled chunk, or all of them: its own gathers read them
    // too).  Fewer stores before each barrier's release.
    unsigned int pub = 0u;
#pragma unroll
    for (int u = 0; u < RPT; ++u)
        if (!onchip || rs.spill != 0ull || rs.nhalo[u * (BS / 32) + warp] != 0) pub |= 1u << u;

    // ---- load r and D^-1 of the own rows.  An own row's z = D^-1 r is kept in
    // zbuf with D^-1 in its w (rather than in registers: the kernel is at its
    // 128-register limit), so the direction update reads z there
    float r[RPT][3], p[RPT][3], q[RPT][3], d[RPT][3];
    auto dv_of = [&](int u) { return zbuf[row[u] - rb].w; };
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
#pragma unroll
        for (int c = 0; c < 3; ++c) r[u][c] = p[u][c] = q[u][c] = d[u][c] = 0.f;
    }
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
        if (row[u] < 0) continue;
        const float4 r4 = B.r4[row[u]];
        r[u][0] = r4.x;
        r[u][1] = r4.y;
        r[u][2] = r4.z;
        zbuf[row[u] - rb] = make_float4(r4.w * r4.x, r4.w * r4.y, r4.w * r4.z, r4.w);
    }
    if (threadIdx.x == 0) {
        if (fused) {
            sh.rho = init_tot[2];
            sh.rr_restart = init_tot[1];
            sh.bnorm2 = init_tot[0];
        } else {
            sh.rho = st->rho;
            sh.rr_restart = st->rr_restart;
            sh.bnorm2 = st->bnorm2;
            sh.last_res = st->last_res;
            sh.status = SP_OK;
        }
        sh.iter = 0;
        sh.restarts = 0;
        sh.beta_f = 0.f;
        // the iteration's scalars in FP32 (its vectors are FP32; the FP64
        // divisions cost ~0.5 us per iteration on GB300's FP64 pipe)
        sh.rho_f = (float)sh.rho;
        sh.target_f = (float)fmax(P.inner2 * sh.rr_restart, kInnerFinal2 * P.tol2 * sh.bnorm2);
    }
    __syncthreads();

    while (!start_done) {
        // ---- SpMV with the fused direction update; p.q
        dfloat pq{0.f, 0.f};
        const float betaf = sh.beta_f;
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            if (row[u] < 0) continue;
            const float di = __ldg(B.diag32 + row[u]);
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;
            {
                const int c = u * (BS / 32) + warp;
                const int lo = rs.loff[c] + lane, nl = rs.nloc[c], nh = rs.nhalo[c];
                const int hb = rs.hoff[c] + lane;
                // the first halo batch is requested before the local sum, so
                // its latency runs under the shared-memory work
                int j[kResHalo];
                float w[kResHalo];
#pragma unroll
                for (int k = 0; k < kResHalo; ++k) {
                    j[k] = 0;
                    w[k] = 0.f;
                    if (k < nh) {   // L1-cached: every iteration reads the same lists
                        j[k] = B.hcol[hb + 32 * k];
                        w[k] = B.hval[hb + 32 * k];
                    }
                }
                float4 gh[kResHalo];
#pragma unroll
                for (int k = 0; k < kResHalo; ++k) {
                    gh[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (w[k] != 0.f) gh[k] = B.r4[j[k]];
                }
                for (int k = 0; k < nl; ++k) {
                    const unsigned int ew = sent[lo + 32 * k];
                    const float wl = entry_weight(ew);
                    const float4 zj = zbuf[entry_col(ew)];
                    s0 = fmaf(wl, zj.x, s0);
                    s1 = fmaf(wl, zj.y, s1);
                    s2 = fmaf(wl, zj.z, s2);
                }
#pragma unroll
                for (int k = 0; k < kResHalo; ++k) {
                    const float ww = w[k] * gh[k].w;
                    s0 = fmaf(ww, gh[k].x, s0);
                    s1 = fmaf(ww, gh[k].y, s1);
                    s2 = fmaf(ww, gh[k].z, s2);
                }
                for (int kb = kResHalo; kb < nh; kb += kResHalo) res_halo_batch(B, hb, kb, nh, s0, s1, s2);
            }
            const float4 zo = zbuf[row[u] - rb];   // D^-1 r of the row, as the update wrote it
            const float z0 = zo.x, z1 = zo.y, z2 = zo.z;
            float q0 = fmaf(di, z0, -alpha_e * s0);
            float q1 = fmaf(di, z1, -alpha_e * s1);
            float q2 = fmaf(di, z2, -alpha_e * s2);
            if (betaf != 0.f) {
                q0 = fmaf(betaf, q[u][0], q0);
                q1 = fmaf(betaf, q[u][1], q1);
                q2 = fmaf(betaf, q[u][2], q2);
                p[u][0] = fmaf(betaf, p[u][0], z0);
                p[u][1] = fmaf(betaf, p[u][1], z1);
                p[u][2] = fmaf(betaf, p[u][2], z2);
            } else {
                p[u][0] = z0;
                p[u][1] = z1;
                p[u][2] = z2;
            }
            q[u][0] = q0;
            q[u][1] = q1;
            q[u][2] = q2;
            pq.hi += p[u][0] * q[u][0] + p[u][1] * q[u][1] + p[u][2] * q[u][2];   // FP32, as the block sums
        }
        {
            const dfloat v[1] = {pq};
            float tot[1];
            if (!grid_allreduce_df<1, float>(st, gen, sh, v, B.partials_df, tot, bid, nb,
                                              [&](const float (&t)[1]) {
                                                  sh.action = 0;
                                                  if (!(t[0] > 0.f) || !isfinite(t[0])) {
                                                      sh.status = SP_ERR_NONFINITE;
                                                      sh.action = 2;
                                                  } else {
                                                      sh.alpha_f = sh.rho_f / t[0];
                                                  }
                                              }))
                break;
        }
        if (sh.action == 2) break;

        // ---- update of d and r; r.r and r.D^-1 r; z of the own rows published
        const float af = sh.alpha_f;
        dfloat rr{0.f, 0.f}, rz{0.f, 0.f};
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            if (row[u] < 0) continue;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                d[u][c] = fmaf(af, p[u][c], d[u][c]);
                r[u][c] = fmaf(-af, q[u][c], r[u][c]);
            }
            const float rsq = r[u][0] * r[u][0] + r[u][1] * r[u][1] + r[u][2] * r[u][2];
            const float dvu = dv_of(u);
            rr.hi += rsq;   // FP32, as the block sums
            rz.hi += dvu * rsq;
            if (pub & (1u << u)) B.r4[row[u]] = make_float4(r[u][0], r[u][1], r[u][2], dvu);
            zbuf[row[u] - rb] = make_float4(dvu * r[u][0], dvu * r[u][1], dvu * r[u][2], dvu);
        }
        {
            const dfloat v[2] = {rr, rz};
            float tot[2];
            if (!grid_allreduce_df<2, float>(st, gen, sh, v, B.partials_df + kMaxPartials, tot, bid, nb,
                                              [&](const float (&t)[2]) {
                                                  ++sh.iter;
                                                  sh.action = 0;
                                                  if (!isfinite(t[0]) || !isfinite(t[1])) {
                                                      sh.status = SP_ERR_NONFINITE;
                                                      sh.action = 2;
                                                  } else {
                                                      sh.beta_f = t[1] / sh.rho_f;
                                                      sh.rho_f = t[1];
                                                      if (t[0] <= sh.target_f || sh.iter >= P.max_iter)
                                                          sh.action = 1;
                                                  }
                                              }))
                break;
        }
        if (sh.action == 2) break;
        if (sh.action == 0) continue;

        // ---- residual replacement: x += d (double-float) and the true residual
        // r = b - A x.  On chip it follows from the last one, b - A (x + d) =
        // (b - A x) - A d, with A d in double-float (weights hi + lo, d exact
        // as FP32): the local half from shared memory (d of the block's rows in
        // zbuf), the halo half from d published in global memory; the residual
        // itself kept as a double-float record per row (rdf).  A block whose
        // entries are all off chip forms A d the same way from its lists.
        {
            // every row's x record is requested before the first is updated
            float4 xh[RPT], xl[RPT];
#pragma unroll
            for (int u = 0; u < RPT; ++u) {
                xh[u] = xl[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (row[u] >= 0) {
                    xh[u] = B.xdf[2 * row[u]];
                    xl[u] = B.xdf[2 * row[u] + 1];
                }
            }
#pragma unroll
            for (int u = 0; u < RPT; ++u) {
                if (row[u] < 0) continue;
                const float4 df = make_float4(d[u][0], d[u][1], d[u][2], dv_of(u));
                const dfloat a = df_add(dfloat{xh[u].x, xl[u].x}, df.x), b = df_add(dfloat{xh[u].y, xl[u].y}, df.y),
                             c = df_add(dfloat{xh[u].z, xl[u].z}, df.z);
                B.xdf[2 * row[u]] = make_float4(a.hi, b.hi, c.hi, 0.f);
                B.xdf[2 * row[u] + 1] = make_float4(a.lo, b.lo, c.lo, 0.f);
                if (pub & (1u << u)) B.d4[row[u]] = make_float4(df.x, df.y, df.z, 0.f);
                zbuf[row[u] - rb] = df;   // d, D^-1 in w
                // r, p and q are set anew after the check (beta = 0), so none of
                // them holds a register through it
#pragma unroll
                for (int c = 0; c < 3; ++c) r[u][c] = p[u][c] = q[u][c] = 0.f;
            }
        }
        if (!grid_sync(st, gen, sh, nb)) break;
        double trr = 0.0, trz = 0.0;
        {
#pragma unroll
            for (int u = 0; u < RPT; ++u) {
                if (row[u] < 0) continue;
                const int c = u * (BS / 32) + warp;
                const int lo = rs.loff[c] + lane, nl = rs.nloc[c], nh = rs.nhalo[c];
                const int hb = rs.hoff[c] + lane;
                // the row's residual record and A_ii are requested first (they
                // arrive under the sums)
                const float4 rh = B.rdf[2 * row[u]], rl = B.rdf[2 * row[u] + 1];
                const dfloat dg{B.diag32[row[u]], B.diag32lo[row[u]]};
                // A d in double-float: each product of a high weight part splits
                // exactly (pr + e); the pr are summed by TwoSum, every low-order
                // term (e, the low part's product, the TwoSum errors) goes into
                // one FP32 compensation
                float sh[3] = {0.f, 0.f, 0.f}, sc[3] = {0.f, 0.f, 0.f};
                auto add = [&](float wh, float wl, float4 dj) {
                    const float dd[3] = {dj.x, dj.y, dj.z};
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const float pr = __fmul_rn(wh, dd[a]);
                        const dfloat t = two_sum(sh[a], pr);
                        sh[a] = t.hi;
                        sc[a] = __fadd_rn(sc[a], __fadd_rn(t.lo, fmaf(wl, dd[a], fmaf(wh, dd[a], -pr))));
                    }
                };
                // loads in batches (one latency per batch): the low parts of the
                // local weights, then the halo entries and their gathers of d
                for (int kb = 0; kb < nl; kb += kResCheckLocal) {
                    float wl[kResCheckLocal];
#pragma unroll
                    for (int k = 0; k < kResCheckLocal; ++k)
                        wl[k] = kb + k < nl ? ld_stream(rlo + lo + 32 * (kb + k)) : 0.f;
#pragma unroll
                    for (int k = 0; k < kResCheckLocal; ++k) {
                        if (kb + k < nl) {
                            const int e = lo + 32 * (kb + k);
                            add(entry_weight(sent[e]), wl[k], zbuf[entry_col(sent[e])]);
                        }
                    }
                }
                for (int kb = 0; kb < nh; kb += kResHalo) {
                    int j[kResHalo];
                    float wh[kResHalo], wl[kResHalo];
#pragma unroll
                    for (int k = 0; k < kResHalo; ++k) {
                        j[k] = 0;
                        wh[k] = wl[k] = 0.f;
                        if (kb + k < nh) {
                            const int e = hb + 32 * (kb + k);
                            j[k] = ld_stream(B.hcol + e);
                            wh[k] = ld_stream(B.hval + e);
                            wl[k] = ld_stream(B.hlo + e);
                        }
                    }
                    float4 dj[kResHalo];
#pragma unroll
                    for (int k = 0; k < kResHalo; ++k) {
                        dj[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (wh[k] != 0.f) dj[k] = B.d4[j[k]];
                    }
#pragma unroll
                    for (int k = 0; k < kResHalo; ++k) add(wh[k], wl[k], dj[k]);
                }
                dfloat s[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) s[a] = two_sum(sh[a], sc[a]);
                const dfloat al{P.alpha_hi, P.alpha_lo};
                const dfloat ro[3] = {{rh.x, rl.x}, {rh.y, rl.y}, {rh.z, rl.z}};
                dfloat rn[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const dfloat ad = df_add(df_mul(dg, dfloat{d[u][a], 0.f}), df_neg(df_mul(al, s[a])));
                    rn[a] = df_add(ro[a], df_neg(ad));
                    r[u][a] = rn[a].hi;
                    d[u][a] = 0.f;
                }
                B.rdf[2 * row[u]] = make_float4(rn[0].hi, rn[1].hi, rn[2].hi, 0.f);
                B.rdf[2 * row[u] + 1] = make_float4(rn[0].lo, rn[1].lo, rn[2].lo, 0.f);
                const float rsq = r[u][0] * r[u][0] + r[u][1] * r[u][1] + r[u][2] * r[u][2];
                trr += (double)rsq;
                trz += (double)(dv_of(u) * rsq);
            }
            __syncthreads();   // zbuf (d) read by every row before it changes
#pragma unroll
            for (int u = 0; u < RPT; ++u) {
                if (row[u] < 0) continue;
                const float dvu = dv_of(u);
                if (pub & (1u << u)) B.r4[row[u]] = make_float4(r[u][0], r[u][1], r[u][2], dvu);
                zbuf[row[u] - rb] = make_float4(dvu * r[u][0], dvu * r[u][1], dvu * r[u][2], dvu);
            }
        }
        {
            const double v[2] = {trr, trz};
            double tot[2];
            if (!grid_allreduce<2>(st, gen, sh, v, B.partials, tot, bid, nb)) break;
            if (threadIdx.x == 0) {
                sh.last_res = sqrt(tot[0] / sh.bnorm2);
                if (bid == 0) st->true_checks += 1;
                sh.action = 0;
                if (!isfinite(tot[0])) {
                    sh.status = SP_ERR_NONFINITE;
                    sh.action = 2;
                } else if (tot[0] <= P.tol2 * sh.bnorm2) {
                    sh.action = 2;   // converged
                } else if (sh.iter >= P.max_iter || sh.restarts >= kMaxCgRestarts + 8) {
                    sh.status = SP_ERR_NOT_CONVERGED;
                    sh.action = 2;
                } else {
                    ++sh.restarts;
                    sh.rho = tot[1];
                    sh.beta_f = 0.f;
                    sh.rr_restart = tot[0];
                    sh.rho_f = (float)tot[1];
                    sh.target_f = (float)fmax(P.inner2 * sh.rr_restart, kInnerFinal2 * P.tol2 * sh.bnorm2);
                }
            }
        }
        __syncthreads();
        if (sh.action == 2) break;
    }
    if (!(fused && sh.iter == 0)) {   // a solve that met the tolerance at x0 keeps x0 as it was
#pragma unroll
        for (int u = 0; u < RPT; ++u)
            if (row[u] >= 0) store_x64(B, np, row[u]);
    }
    if (bid == 0 && threadIdx.x == 0) {
        if (fused) {   // every block wrote its mode before the first grid reduction
            int off = 0;
            for (int b = 0; b < nb; ++b) off += B.partials[3 * kMaxPartials + b] != 0.0 ? 1 : 0;
            st->res_offchip = off;
        }
        st->iter = sh.iter;
        st->restarts = sh.restarts;
        st->last_res = sh.last_res;
        st->done = 1;
        if (st->error == 0 && sh.status != SP_OK) {
            st->status = sh.status;
            st->error = sh.status;
        } else if (st->error != 0) {
            st->status = st->error;
        } else {
            st->status = SP_OK;
        }
    }
}

template <int BS, int RPT>
__global__ void __launch_bounds__(BS, 1) k32_cg_resident(KParams P, DevBuffers B, int smem_bytes)
{
    extern __shared__ float4 res_dyn[];
    __shared__ PShared sh;
    __shared__ RShared rs;
    resident_solve<BS, RPT>(P, B, blockIdx.x, gridDim.x, sh, rs, res_dyn, smem_bytes);
    barrier_leave(B.st, gridDim.x);
}

// ------------------------------------------------------ FP64 persistent solve
// The FP64 solve in one cooperative launch, every scalar decided by thread 0
// of every block from identical totals; the recurrence residual arms an FP64
// true-residual check that accepts or restarts.
// Large systems (TPR = 1): the FP64 solver's iteration as the two-kernel form
// of cg.cu (Jacobi-PCG with the direction update fused into the SpMV: q = A z
// + beta q, p = z + beta p; x += alpha p, r -= alpha q, z = D^-1 r), two grid
// reductions per iteration (the barrier of the second one also publishes z
// for the next SpMV); a block owns whole windows of 256 rows, one thread per
// row, warps take the windows' chunks in zig-zag order (as the mixed
// streaming solve).
// Small systems (TPR = 4, fewer than two windows per SM): pipelined CG, one
// grid reduction per iteration (below), where the barriers are a large share
// of an iteration; a block owns a run of chunks of 32 rows and four
// neighbouring lanes share a row, each summing every fourth of its entries,
// so a row's gathers are in flight together; GB300 issues FP64 at ~2 FMA per
// clock per SM, so a small system is also spread over as many SMs as it has
// chunk pairs.  Gathered vectors go through plain (coherent) loads: other
// blocks wrote them before the last barrier.
constexpr int kBatch64 = 6;

// s_a = sum over the row's entries k = sub, sub + TPR, ... of w_k v_a[col_k]
template <int TPR>
__device__ __forceinline__ void p_row_sum64(const int* __restrict__ col, const double* __restrict__ val,
                                            const double* v, int np, int e0, int e1, int sub, bool active,
                                            double& s0, double& s1, double& s2)
{
    s0 = s1 = s2 = 0.0;
    if (active) {
        for (int eb = e0 + 32 * sub; eb < e1; eb += 32 * TPR * kBatch64) {
            int j[kBatch64];
            double w[kBatch64];
#pragma unroll
            for (int u = 0; u < kBatch64; ++u) {
                const int e = eb + 32 * TPR * u;
                j[u] = 0;
                w[u] = 0.0;
                if (e < e1) {
                    j[u] = ld_stream(col + e);
                    w[u] = __ldg(val + e);
                }
            }
            double g0[kBatch64], g1[kBatch64], g2[kBatch64];
#pragma unroll
            for (int u = 0; u < kBatch64; ++u) {
                g0[u] = g1[u] = g2[u] = 0.0;
                if (w[u] != 0.0) {
                    g0[u] = v[j[u]];
                    g1[u] = v[np + j[u]];
                    g2[u] = v[2 * np + j[u]];
                }
            }
#pragma unroll
            for (int u = 0; u < kBatch64; ++u) {
                s0 += w[u] * g0[u];
                s1 += w[u] * g1[u];
                s2 += w[u] * g2[u];
            }
        }
    }
#pragma unroll
    for (int o = 1; o < TPR; o <<= 1) {   // the row's lanes are neighbours in the warp
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
}

// The block's rows in slot order: calls f(slot, sub, active) the same number
// of times in every thread of the block (the shuffles of p_row_sum64 need
// whole warps).
template <int TPR, class F>
__device__ __forceinline__ void for_each_slot64(const KParams& P, int bid, int nb, F f)
{
    if (TPR == 1) {
        const int nwin = P.nslots / 256;
        const int wb = (int)((long long)bid * nwin / nb), we = (int)((long long)(bid + 1) * nwin / nb);
        const int G = blockDim.x >> 8, t = threadIdx.x & 255;
        for (int w = wb + (int)(threadIdx.x >> 8), k = 0; w < we; w += G, ++k) f(w * 256 + chunk_lane(k, t), 0, true);
    } else {
        const int s0 = 32 * (int)((long long)bid * P.nchunks / nb);
        const int s1 = 32 * (int)((long long)(bid + 1) * P.nchunks / nb);
        const int per = blockDim.x / TPR;
        for (int base = s0; base < s1; base += per) {
            const int slot = base + (int)threadIdx.x / TPR;
            f(slot, (int)threadIdx.x % TPR, slot < s1);
        }
    }
}

template <int TPR>
__device__ __forceinline__ void persistent_solve64(const KParams& P, const DevBuffers& B, int bid, int nb,
                                                   PShared& sh, int from_x)
{
    DevState* st = B.st;
    if (threadIdx.x == 0) sh.flag = 0;
    __syncthreads();
    if (st->error | st->overflow) return;   // uniform: set before the launch
    unsigned int gen = 0u;   // barriers passed in this launch (the counter starts at 0)
    const int np = P.npad;
    double* x = B.x;
    double* r = B.r;
    double* z = B.z;
    double* p = B.p;
    double* q = B.q;
    auto row_of = [&](int slot, bool active) { return active ? B.slot_row[slot] : -1; };
    auto ends = [&](int slot, int& e0, int& e1) {
        e0 = B.chunk_off[slot >> 5] + (slot & 31);
        e1 = B.chunk_off[(slot >> 5) + 1];
    };

    // r = b - A x0 (or b, x = 0); z = D^-1 r; p = q = 0; ||b||^2, r.r, r.z
    {
        double bb = 0.0, rr = 0.0, rz = 0.0;
        for_each_slot64<TPR>(P, bid, nb, [&](int slot, int sub, bool active) {
            const int row = row_of(slot, active);
            int e0 = 0, e1 = 0;
            if (row >= 0) ends(slot, e0, e1);
            double s0 = 0.0, s1 = 0.0, s2 = 0.0;
            if (from_x) p_row_sum64<TPR>(B.col, B.val, x, np, e0, e1, sub, row >= 0, s0, s1, s2);
            if (row < 0 || sub != 0) return;
            const double sv[3] = {s0, s1, s2};
            const double d = B.diag[row], di = B.dinv[row];
            double rs = 0.0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int k2 = c * np + row;
                const double bk = B.b[k2];
                double rk = bk;
                if (from_x)
                    rk = bk - (d * x[k2] - P.alpha * sv[c]);
                else
                    x[k2] = 0.0;
                r[k2] = rk;
                z[k2] = di * rk;
                p[k2] = 0.0;
                q[k2] = 0.0;
                bb += bk * bk;
                rs += rk * rk;
            }
            rr += rs;
            rz += di * rs;
        });
        const double v[3] = {bb, rr, rz};
        double tot[3];
        if (!grid_allreduce<3>(st, gen, sh, v, B.partials, tot, bid, nb)) goto done;
        if (threadIdx.x == 0) {
            sh.bnorm2 = tot[0];
            sh.rho = tot[2];
            sh.rr_restart = tot[1];
            sh.iter = 0;
            sh.restarts = 0;
            sh.status = SP_OK;
            sh.last_res = tot[0] > 0.0 ? sqrt(tot[1] / tot[0]) : 0.0;
            sh.action = 0;
            sh.bcast[3] = 0.0;   // beta
            if (!isfinite(tot[0]) || !isfinite(tot[1])) {
                sh.status = SP_ERR_NONFINITE;
                sh.action = 2;
            } else if (tot[0] == 0.0 || tot[1] <= P.tol2 * tot[0]) {
                sh.action = 2;   // b = 0 (x = 0 then) or the start meets the tolerance
            }
            if (bid == 0) {
                st->bnorm2 = tot[0];
                st->zero_b = tot[0] == 0.0 ? 1 : 0;
            }
        }
        __syncthreads();
        if (sh.action == 2) goto done;
    }
    for (;;) {
        // ---- q = A z + beta q; p = z + beta p; p.q
        const double beta = sh.bcast[3];
        double pq = 0.0;
        for_each_slot64<TPR>(P, bid, nb, [&](int slot, int sub, bool active) {
            const int row = row_of(slot, active);
            int e0 = 0, e1 = 0;
            if (row >= 0) ends(slot, e0, e1);
            double s0, s1, s2;
            p_row_sum64<TPR>(B.col, B.val, z, np, e0, e1, sub, row >= 0, s0, s1, s2);
            if (row < 0 || sub != 0) return;
            const double sv[3] = {s0, s1, s2};
            const double d = B.diag[row];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int k2 = c * np + row;
                const double zk = z[k2];
                const double az = d * zk - P.alpha * sv[c];
                const double qk = beta == 0.0 ? az : az + beta * q[k2];
                const double pk = beta == 0.0 ? zk : zk + beta * p[k2];
                q[k2] = qk;
                p[k2] = pk;
                pq += pk * qk;
            }
        });
        {
            const double v[1] = {pq};
            double tot[1];
            if (!grid_allreduce<1>(st, gen, sh, v, B.partials + kMaxPartials, tot, bid, nb)) break;
            if (threadIdx.x == 0) {
                sh.action = 0;
                if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
                    sh.status = SP_ERR_NONFINITE;
                    sh.action = 2;
                } else {
                    sh.bcast[2] = sh.rho / tot[0];   // alpha
                }
            }
            __syncthreads();
            if (sh.action == 2) break;
        }
        // ---- x += alpha p; r -= alpha q; z = D^-1 r (own rows); r.r, r.z
        const double a = sh.bcast[2];
        double rr = 0.0, rz = 0.0;
        for_each_slot64<TPR>(P, bid, nb, [&](int slot, int sub, bool active) {
            const int i = row_of(slot, active);
            if (i < 0 || sub != 0) return;
            const double di = B.dinv[i];
            double rs = 0.0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int k2 = c * np + i;
                x[k2] += a * p[k2];
                const double rk = r[k2] - a * q[k2];
                r[k2] = rk;
                z[k2] = di * rk;
                rs += rk * rk;
            }
            rr += rs;
            rz += di * rs;
        });
        {
            const double v[2] = {rr, rz};
            double tot[2];
            if (!grid_allreduce<2>(st, gen, sh, v, B.partials + 2 * kMaxPartials, tot, bid, nb)) break;
            if (threadIdx.x == 0) {
                ++sh.iter;
                sh.action = 0;
                if (!isfinite(tot[0]) || !isfinite(tot[1])) {
                    sh.status = SP_ERR_NONFINITE;
                    sh.action = 2;
                } else {
                    sh.bcast[3] = tot[1] / sh.rho;   // beta
                    sh.rho = tot[1];
                    if (tot[0] <= P.tol2 * sh.bnorm2 || sh.iter >= P.max_iter) sh.action = 1;
                }
            }
            __syncthreads();
            if (sh.action == 2) break;
            if (sh.action == 0) continue;
        }
        // ---- the FP64 true residual r = b - A x (z = D^-1 r): accept, restart or give up
        {
            double trr = 0.0, trz = 0.0;
            for_each_slot64<TPR>(P, bid, nb, [&](int slot, int sub, bool active) {
                const int row = row_of(slot, active);
                int e0 = 0, e1 = 0;
                if (row >= 0) ends(slot, e0, e1);
                double s0, s1, s2;
                p_row_sum64<TPR>(B.col, B.val, x, np, e0, e1, sub, row >= 0, s0, s1, s2);
                if (row < 0 || sub != 0) return;
                const double sv[3] = {s0, s1, s2};
                const double d = B.diag[row], di = B.dinv[row];
                double rs = 0.0;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int k2 = c * np + row;
                    const double rk = B.b[k2] - (d * x[k2] - P.alpha * sv[c]);
                    r[k2] = rk;
                    z[k2] = di * rk;
                    rs += rk * rk;
                }
                trr += rs;
                trz += di * rs;
            });
            const double v[2] = {trr, trz};
            double tot[2];
            if (!grid_allreduce<2>(st, gen, sh, v, B.partials, tot, bid, nb)) break;
            if (threadIdx.x == 0) {
                sh.last_res = sqrt(tot[0] / sh.bnorm2);
                if (bid == 0) st->true_checks += 1;
                sh.action = 0;
                if (!isfinite(tot[0])) {
                    sh.status = SP_ERR_NONFINITE;
                    sh.action = 2;
                } else if (tot[0] <= P.tol2 * sh.bnorm2) {
                    sh.action = 2;   // converged
                } else if (sh.iter >= P.max_iter || sh.restarts >= kMaxCgRestarts + 8) {
                    sh.status = SP_ERR_NOT_CONVERGED;
                    sh.action = 2;
                } else {
                    ++sh.restarts;
                    sh.rho = tot[1];
                    sh.bcast[3] = 0.0;
                }
            }
            __syncthreads();
            if (sh.action == 2) break;
        }
    }
done:
    if (bid == 0 && threadIdx.x == 0) {
        st->iter = sh.iter;
        st->restarts = sh.restarts;
        st->last_res = sh.last_res;
        st->done = 1;
        if (st->error == 0 && sh.status != SP_OK) {
            st->status = sh.status;
            st->error = sh.status;
        } else if (st->error != 0) {
            st->status = st->error;
        } else {
            st->status = SP_OK;
        }
    }
}

// s_a = sum over the row's entries k = sub, sub + TPR, ... of w_k D^-1_col v_a[col_k]
template <int TPR>
__device__ __forceinline__ void p_row_sum64_scaled(const int* __restrict__ col, const double* __restrict__ val,
                                                   const double* __restrict__ dinv, const double* v, int np, int e0,
                                                   int e1, int sub, bool active, double& s0, double& s1, double& s2)
{
    s0 = s1 = s2 = 0.0;
    if (active) {
        for (int eb = e0 + 32 * sub; eb < e1; eb += 32 * TPR * kBatch64) {
            int j[kBatch64];
            double w[kBatch64];
#pragma unroll
            for (int u = 0; u < kBatch64; ++u) {
                const int e = eb + 32 * TPR * u;
                j[u] = 0;
                w[u] = 0.0;
                if (e < e1) {
                    j[u] = ld_stream(col + e);
                    w[u] = __ldg(val + e);
                }
            }
            double g0[kBatch64], g1[kBatch64], g2[kBatch64], dj[kBatch64];
#pragma unroll
            for (int u = 0; u < kBatch64; ++u) {
                g0[u] = g1[u] = g2[u] = dj[u] = 0.0;
                if (w[u] != 0.0) {
                    dj[u] = __ldg(dinv + j[u]);
                    g0[u] = v[j[u]];
                    g1[u] = v[np + j[u]];
                    g2[u] = v[2 * np + j[u]];
                }
            }
#pragma unroll
            for (int u = 0; u < kBatch64; ++u) {
                const double ww = w[u] * dj[u];
                s0 += ww * g0[u];
                s1 += ww * g1[u];
                s2 += ww * g2[u];
            }
        }
    }
#pragma unroll
    for (int o = 1; o < TPR; o <<= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
}

// Small systems: pipelined CG (Ghysels & Vanroose, Parallel Computing 40, 2014)
// with the Jacobi preconditioner, FP64, one grid reduction per iteration.  With
// u = D^-1 r and m = D^-1 w formed where they are used, per iteration:
//   gamma = (r, u), delta = (w, u), ||r||^2           (the barrier's reduction)
//   beta = gamma / gamma_old, alpha = gamma / (delta - beta gamma / alpha_old)
//   n = A m;  z = n + beta z;  s = w + beta s;  p = u + beta p;
//   x += alpha p;  r -= alpha s;  w -= alpha z
// so the reduction of the next iteration's scalars and the publication of w
// for its SpMV share one barrier (w double-buffered: the SpMV reads the
// iteration's w while the update writes the next one).  The recurrence
// residual arms an FP64 true residual b - A x, which ends the solve or
// restarts the recurrences from it.
__device__ __forceinline__ void pipelined_solve64(const KParams& P, const DevBuffers& B, int bid, int nb, PShared& sh,
                                                  int from_x)
{
    constexpr int TPR = 4;
    DevState* st = B.st;
    if (threadIdx.x == 0) sh.flag = 0;
    __syncthreads();
    if (st->error | st->overflow) return;   // uniform: set before the launch
    unsigned int gen = 0u;
    const int np = P.npad;
    double* x = B.x;
    double* r = B.r;
    double* z = B.z;
    double* p = B.p;
    double* sv = B.s64;
    double* wbuf[2] = {B.q, B.s64 + 3 * (size_t)np};
    int cur = 0;        // the w buffer of the current iteration
    int pset = 0;       // partial-sum set of the next reduction (consecutive ones differ)
    auto row_of = [&](int slot, bool active) { return active ? B.slot_row[slot] : -1; };
    auto ends = [&](int slot, int& e0, int& e1) {
        e0 = B.chunk_off[slot >> 5] + (slot & 31);
        e1 = B.chunk_off[(slot >> 5) + 1];
    };
    auto partials = [&]() {   // two sets of up to three sums each
        double* q = B.partials + (size_t)pset * 4 * kMaxPartials;
        pset ^= 1;
        return q;
    };
    // w = A D^-1 r into wbuf[cur]; z = s = p = 0; gamma, delta, ||r||^2 (after a barrier that published r)
    auto restart_w = [&](double (&tot)[3]) -> bool {
        double g = 0.0, d = 0.0, rr = 0.0;
        double* w = wbuf[cur];
        for_each_slot64<TPR>(P, bid, nb, [&](int slot, int sub, bool active) {
            const int row = row_of(slot, active);
            int e0 = 0, e1 = 0;
            if (row >= 0) ends(slot, e0, e1);
            double s0, s1, s2;
            p_row_sum64_scaled<TPR>(B.col, B.val, B.dinv, r, np, e0, e1, sub, row >= 0, s0, s1, s2);
            if (row < 0 || sub >= 3) return;   // lane c: component c
            const double sm = sub == 0 ? s0 : (sub == 1 ? s1 : s2);
            const double dg = B.diag[row], di = B.dinv[row];
            {
                const int k2 = sub * np + row;
                const double rk = r[k2], uk = di * rk;
                const double wk = dg * uk - P.alpha * sm;
                w[k2] = wk;
                z[k2] = 0.0;
                sv[k2] = 0.0;
                p[k2] = 0.0;
                g += rk * uk;
                d += wk * uk;
                rr += rk * rk;
            }
        });
        const double v[3] = {g, d, rr};
        return grid_allreduce<3>(st, gen, sh, v, partials(), tot, bid, nb);
    };
    // the true residual r = b - A x (after a barrier that published x); ||r||^2
    auto true_residual = [&](double (&tot)[1], bool first) -> bool {
        double rr = 0.0, bb = 0.0;
        for_each_slot64<TPR>(P, bid, nb, [&](int slot, int sub, bool active) {
            const int row = row_of(slot, active);
            int e0 = 0, e1 = 0;
            if (row >= 0) ends(slot, e0, e1);
            double s0 = 0.0, s1 = 0.0, s2 = 0.0;
            if (!first || from_x) p_row_sum64<TPR>(B.col, B.val, x, np, e0, e1, sub, row >= 0, s0, s1, s2);
            if (row < 0 || sub >= 3) return;   // lane c: component c
            const double sm = sub == 0 ? s0 : (sub == 1 ? s1 : s2);
            const double dg = B.diag[row];
            {
                const int k2 = sub * np + row;
                const double bk = B.b[k2];
                double rk = bk;
                if (!first || from_x)
                    rk = bk - (dg * x[k2] - P.alpha * sm);
                else
                    x[k2] = 0.0;
                r[k2] = rk;
                rr += rk * rk;
                bb += bk * bk;
            }
        });
        if (first) {
            const double v[2] = {rr, bb};
            double t2[2];
            if (!grid_allreduce<2>(st, gen, sh, v, partials(), t2, bid, nb)) return false;
            if (threadIdx.x == 0) sh.bnorm2 = t2[1];
            tot[0] = t2[0];
            return true;
        }
        const double v[1] = {rr};
        return grid_allreduce<1>(st, gen, sh, v, partials(), tot, bid, nb);
    };

    double t3[3], t1[1];
    bool first = true;   // beta = 0: the first iteration of the solve or of a restart
    if (!true_residual(t1, true)) goto done;
    if (threadIdx.x == 0) {
        sh.iter = 0;
        sh.restarts = 0;
        sh.status = SP_OK;
        sh.last_res = sh.bnorm2 > 0.0 ? sqrt(t1[0] / sh.bnorm2) : 0.0;
        sh.action = 0;
        if (!isfinite(sh.bnorm2) || !isfinite(t1[0])) {
            sh.status = SP_ERR_NONFINITE;
            sh.action = 2;
        } else if (sh.bnorm2 == 0.0 || t1[0] <= P.tol2 * sh.bnorm2) {
            sh.action = 2;   // b = 0 (x = 0 then) or the start meets the tolerance
        }
        if (bid == 0) {
            st->bnorm2 = sh.bnorm2;
            st->zero_b = sh.bnorm2 == 0.0 ? 1 : 0;
        }
    }
    __syncthreads();
    if (sh.action == 2) goto done;
    if (!restart_w(t3)) goto done;
    for (;;) {
        // ---- the scalars of this iteration (thread 0, identical totals in every block)
        if (threadIdx.x == 0) {
            const double g = t3[0], d = t3[1], rr = t3[2];
            sh.action = 0;
            if (!isfinite(g) || !isfinite(d) || !isfinite(rr)) {
                sh.status = SP_ERR_NONFINITE;
                sh.action = 2;
            } else if (rr <= P.tol2 * sh.bnorm2 || sh.iter >= P.max_iter) {
                sh.action = 1;   // the true residual decides
            } else {
                const double beta = first ? 0.0 : g / sh.rho;
                const double den = first ? d : d - beta * g / sh.alpha_d;   // (p, A p) of the new direction
                if (!(den > 0.0)) {
                    sh.action = 1;   // lost to rounding near convergence: the true residual decides
                } else {
                    sh.beta_d = beta;
                    sh.alpha_d = g / den;
                    sh.rho = g;
                }
            }
        }
        __syncthreads();
        first = false;
        if (sh.action == 2) break;
        if (sh.action == 1) {
            if (!true_residual(t1, false)) break;
            if (threadIdx.x == 0) {
                sh.last_res = sqrt(t1[0] / sh.bnorm2);
                if (bid == 0) st->true_checks += 1;
                sh.action = 0;
                if (!isfinite(t1[0])) {
                    sh.status = SP_ERR_NONFINITE;
                    sh.action = 2;
                } else if (t1[0] <= P.tol2 * sh.bnorm2) {
                    sh.action = 2;   // converged
                } else if (sh.iter >= P.max_iter || sh.restarts >= kMaxCgRestarts + 8) {
                    sh.status = SP_ERR_NOT_CONVERGED;
                    sh.action = 2;
                } else {
                    ++sh.restarts;
                }
            }
            __syncthreads();
            if (sh.action == 2) break;
            if (!restart_w(t3)) break;
            first = true;
            continue;
        }
        // ---- n = A D^-1 w; the recurrences (w into the other buffer); the next reduction
        const double a = sh.alpha_d, beta = sh.beta_d;
        const double* w = wbuf[cur];
        double* wn = wbuf[cur ^ 1];
        double g = 0.0, d = 0.0, rr = 0.0;
        for_each_slot64<TPR>(P, bid, nb, [&](int slot, int sub, bool active) {
            const int row = row_of(slot, active);
            int e0 = 0, e1 = 0;
            if (row >= 0) ends(slot, e0, e1);
            double s0, s1, s2;
            p_row_sum64_scaled<TPR>(B.col, B.val, B.dinv, w, np, e0, e1, sub, row >= 0, s0, s1, s2);
            // every lane of the row holds the sums: lane c updates component c
            // (a third of the FP64 instructions per warp of a lane doing all three)
            if (row < 0 || sub >= 3) return;
            const double sm = sub == 0 ? s0 : (sub == 1 ? s1 : s2);
            const double dg = B.diag[row], di = B.dinv[row];
            {
                const int k2 = sub * np + row;
                const double wk = w[k2];
                const double nk = dg * (di * wk) - P.alpha * sm;   // (A m)_k, m = D^-1 w
                const double zk = nk + beta * z[k2];
                const double sk = wk + beta * sv[k2];
                const double pk = di * r[k2] + beta * p[k2];
                z[k2] = zk;
                sv[k2] = sk;
                p[k2] = pk;
                x[k2] += a * pk;
                const double rk = r[k2] - a * sk;
                r[k2] = rk;
                const double wnk = wk - a * zk;
                wn[k2] = wnk;
                const double uk = di * rk;
                g += rk * uk;
                d += wnk * uk;
                rr += rk * rk;
            }
        });
        cur ^= 1;
        const double v[3] = {g, d, rr};
        if (!grid_allreduce<3>(st, gen, sh, v, partials(), t3, bid, nb)) break;
        if (threadIdx.x == 0) ++sh.iter;
    }
done:
    if (bid == 0 && threadIdx.x == 0) {
        st->iter = sh.iter;
        st->restarts = sh.restarts;
        st->last_res = sh.last_res;
        st->done = 1;
        if (st->error == 0 && sh.status != SP_OK) {
            st->status = sh.status;
            st->error = sh.status;
        } else if (st->error != 0) {
            st->status = st->error;
        } else {
            st->status = SP_OK;
        }
    }
}

template <int TPR>
__global__ void __launch_bounds__(512, 1) k64_cg_persistent(KParams P, DevBuffers B, int from_x)
{
    __shared__ PShared sh;
    if (TPR == 1)
        persistent_solve64<1>(P, B, blockIdx.x, gridDim.x, sh, from_x);
    else
        pipelined_solve64(P, B, blockIdx.x, gridDim.x, sh, from_x);
    barrier_leave(B.st, gridDim.x);
}

// Tile configurations of the single-system kernel: gathers in flight per
// thread (KB) against resident blocks per SM (MINB, which caps the registers
// at 65536 / (256 MINB)), with or without requesting the next batch's
// columns during the current gathers (PIPE).  Chosen per system by the
// autotuner.
template <int KB, int MINB, bool PIPE, int BS, bool MF = false>
__global__ void __launch_bounds__(BS, MINB) k32_cg_persistent(KParams P, DevBuffers B)
{
    __shared__ PShared sh;
    persistent_solve<KB, PIPE, MF>(P, B, blockIdx.x, gridDim.x, sh);
    barrier_leave(B.st, gridDim.x);
}

// Batch: block b serves replica k with blk_off[k] <= b < blk_off[k + 1]; each
// replica's blocks synchronise and reduce among themselves only, and leave
// when their replica has converged.  Tile configurations (gathers in flight
// KB, resident blocks per SM MINB, threads per block BS) are chosen by
// sp_batch_autotune.
template <int KB, int MINB, int BS>
__global__ void __launch_bounds__(BS, MINB) k32_cg_persistent_batch(const KParams* __restrict__ Ps,
                                                                   const DevBuffers* __restrict__ Bs,
                                                                   const int* __restrict__ blk_off, int R)
{
    __shared__ PShared sh;
    __shared__ int rep;
    if (threadIdx.x == 0) {
        int lo = 0, hi = R - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (blk_off[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
        }
        rep = lo;
    }
    __syncthreads();
    const int k = rep;
    persistent_solve<KB, false>(Ps[k], Bs[k], (int)blockIdx.x - blk_off[k], blk_off[k + 1] - blk_off[k], sh);
    barrier_leave(Bs[k].st, blk_off[k + 1] - blk_off[k]);
}

namespace {
// kResSmemBytes (220 KB): the largest carve-out; more blocks keep every local entry
// on chip (at 190 KB the densest blocks of some steps fell back to global gathers),
// and the halo gathers keep ~28 KB of L1

struct PCfg {
    int kb, minb, pipe, bs;
    const void* fn;
    int occ;
    int resident;   // 1: the on-chip solve (k32_cg_resident), dynamic shared memory kResSmemBytes
    int mf;         // 1: the streaming solve with the matrix-free SpMV (weights recomputed)
};
PCfg g_pcfg[kPersistentConfigs] = {   // entry 0: the default without autotuning
    {6, 1, 0, 1024, (const void*)k32_cg_persistent<6, 1, false, 1024>, 0, 0},
    {8, 1, 0, 1024, (const void*)k32_cg_persistent<8, 1, false, 1024>, 0, 0},
    {6, 4, 0, 256, (const void*)k32_cg_persistent<6, 4, false, 256>, 0, 0},
    {8, 4, 0, 256, (const void*)k32_cg_persistent<8, 4, false, 256>, 0, 0},
    {4, 4, 0, 256, (const void*)k32_cg_persistent<4, 4, false, 256>, 0, 0},
    {4, 4, 1, 256, (const void*)k32_cg_persistent<4, 4, true, 256>, 0, 0},
    {5, 4, 1, 256, (const void*)k32_cg_persistent<5, 4, true, 256>, 0, 0},
    {6, 3, 1, 256, (const void*)k32_cg_persistent<6, 3, true, 256>, 0, 0},
    {kResHalo, 1, 0, 1024, (const void*)k32_cg_resident<1024, 2>, 0, 1},
    {kResHalo, 1, 0, 512, (const void*)k32_cg_resident<512, 4>, 0, 1},
    {4, 1, 0, 512, (const void*)k32_cg_persistent<4, 1, false, 512, true>, 0, 0, 1},
    {4, 3, 0, 256, (const void*)k32_cg_persistent<4, 3, false, 256, true>, 0, 0, 1},
};
struct BCfg {
    int kb, minb, bs;
    const void* fn;
    int occ;
};
BCfg g_bcfg[kBatchConfigs] = {   // entry 0: the default without autotuning
    {6, 4, 256, (const void*)k32_cg_persistent_batch<6, 4, 256>, 0},
    {4, 4, 256, (const void*)k32_cg_persistent_batch<4, 4, 256>, 0},
    {8, 4, 256, (const void*)k32_cg_persistent_batch<8, 4, 256>, 0},
    {6, 2, 512, (const void*)k32_cg_persistent_batch<6, 2, 512>, 0},
    {6, 1, 1024, (const void*)k32_cg_persistent_batch<6, 1, 1024>, 0},
    {8, 1, 1024, (const void*)k32_cg_persistent_batch<8, 1, 1024>, 0},
};
std::once_flag g_pocc_once;
void pocc_init()
{
    std::call_once(g_pocc_once, [] {
        for (auto& c : g_pcfg) {
            int smem = 0;
            if (c.resident) {
                smem = kResSmemBytes;
                if (cudaFuncSetAttribute(c.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
                    c.occ = 0;
                    continue;
                }
            }
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ, c.fn, c.bs, smem) != cudaSuccess) c.occ = 0;
        }
        for (auto& c : g_bcfg)
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ, c.fn, c.bs, 0) != cudaSuccess) c.occ = 0;
        cudaGetLastError();
    });
}

long long grid_of(const PCfg& c, const KParams& P, Launch L)
{
    const long long groups = c.bs / 256;   // windows a block processes at once
    long long g = std::min<long long>((long long)L.num_sms * c.occ, (P.nslots / 256 + groups - 1) / groups);
    if (g > kMaxPartials) g = kMaxPartials;
    return g;
}

// The on-chip solve needs its halo lists and at most kResWindows windows per block.
bool resident_fits(const PCfg& c, const KParams& P, const DevBuffers& B, Launch L)
{
    if (!B.hcol || !B.hval || !B.hlo || !B.rlo || !B.rdf || !B.res_hist) return false;
    const long long g = grid_of(c, P, L);   // at most one block per SM: rlo holds num_sms blocks
    return g >= 1 && g <= L.num_sms && (P.nslots / 256 + g - 1) / g <= kResWindows;
}

// The configuration a launch uses: the chosen one, or entry 0 where the
// chosen one is the on-chip solve and the system does not fit it.
const PCfg& cfg_of(const KParams& P, const DevBuffers& B, Launch L)
{
    pocc_init();
    const int k = (P.pcfg >= 0 && P.pcfg < kPersistentConfigs) ? P.pcfg : 0;
    if (g_pcfg[k].resident && !resident_fits(g_pcfg[k], P, B, L)) return g_pcfg[0];
    return g_pcfg[k];
}
}  // namespace

int cg_persistent_batch_capacity(Launch L, int cfg)
{
    pocc_init();
    if (cfg < 0 || cfg >= kBatchConfigs) return 0;
    return L.num_sms * g_bcfg[cfg].occ;
}

void cg_batch_config(int k, int* gathers, int* blocks_per_sm, int* block_threads)
{
    const BCfg& c = g_bcfg[(k >= 0 && k < kBatchConfigs) ? k : 0];
    *gathers = c.kb;
    *blocks_per_sm = c.minb;
    *block_threads = c.bs;
}

cudaError_t launch_cg32_persistent_batch(const KParams* Ps_dev, const DevBuffers* Bs_dev, const int* blk_off_dev,
                                         int R, int total_blocks, int cfg, Launch L)
{
    if (cfg < 0 || cfg >= kBatchConfigs) return cudaErrorInvalidValue;
    if (total_blocks < 1 || total_blocks > cg_persistent_batch_capacity(L, cfg))
        return cudaErrorCooperativeLaunchTooLarge;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)total_blocks);
    lc.blockDim = dim3((unsigned)g_bcfg[cfg].bs);
    lc.dynamicSmemBytes = 0;
    lc.stream = L.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    void* args[] = {const_cast<KParams**>(&Ps_dev), const_cast<DevBuffers**>(&Bs_dev), const_cast<int**>(&blk_off_dev),
                    &R};
    return cudaLaunchKernelExC(&lc, g_bcfg[cfg].fn, args);
}

void cg_persistent_config(int k, int* gathers, int* blocks_per_sm, int* pipelined, int* block_threads,
                          int* resident, int* matrix_free)
{
    const PCfg& c = g_pcfg[(k >= 0 && k < kPersistentConfigs) ? k : 0];
    *gathers = c.kb;
    *blocks_per_sm = c.minb;
    *pipelined = c.pipe;
    *block_threads = c.bs;
    *resident = c.resident;
    *matrix_free = c.mf;
}

int cg_persistent_prelaunches(const KParams& P, const DevBuffers& B, Launch L)
{
    return cfg_of(P, B, L).mf ? 1 : 0;
}

bool cg_persistent_usable(int k, const KParams& P, const DevBuffers& B, Launch L)
{
    pocc_init();
    if (k < 0 || k >= kPersistentConfigs || g_pcfg[k].occ < 1) return false;
    return !g_pcfg[k].resident || resident_fits(g_pcfg[k], P, B, L);
}

bool cg_persistent_on_chip(const KParams& P, const DevBuffers& B, Launch L)
{
    return cfg_of(P, B, L).resident != 0;
}

int cg_persistent_grid(const KParams& P, const DevBuffers& B, Launch L)
{
    return (int)grid_of(cfg_of(P, B, L), P, L);
}

// FP64 persistent solve.  Systems of at least two windows of 256 rows per SM:
// blocks of 512 threads (two windows at a time), one per SM, one thread per
// row.  Smaller ones: blocks of two chunks of 32 rows with four threads per
// row (256 threads), as many blocks as chunk pairs up to one per SM.
void cg64_shape(const KParams& P, Launch L, int* grid, int* threads, int* tpr)
{
    const int nwin = P.nslots / 256;
    const int cap = std::min(L.num_sms, kMaxPartials);
    if (nwin >= 2 * L.num_sms) {
        *grid = std::min(cap, (nwin + 1) / 2);
        *threads = 512;
        *tpr = 1;
    } else {
        const int nch = std::max(P.nchunks, 1);
        const int g = std::max(1, std::min(cap, (nch + 1) / 2));
        *grid = g;
        *threads = 4 * 32 * std::min(4, (nch + g - 1) / g);
        *tpr = 4;
    }
}

cudaError_t launch_cg64_persistent(const KParams& P, DevBuffers& B, int from_x, Launch L)
{
    int g = 1, bs = 32, tpr = 1;
    cg64_shape(P, L, &g, &bs, &tpr);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)g);
    cfg.blockDim = dim3((unsigned)bs);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = L.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void* args[] = {const_cast<KParams*>(&P), &B, &from_x};
    return cudaLaunchKernelExC(&cfg, tpr == 1 ? (const void*)k64_cg_persistent<1> : (const void*)k64_cg_persistent<4>,
                               args);
}

int cg64_persistent_grid(const KParams& P, Launch L)
{
    int g = 1, bs = 32, tpr = 1;
    cg64_shape(P, L, &g, &bs, &tpr);
    return g;
}

cudaError_t launch_cg32_persistent(const KParams& P, DevBuffers& B, Launch L)
{
    const PCfg& c = cfg_of(P, B, L);
    const int g = (int)grid_of(c, P, L);
    if (g < 1) return cudaErrorCooperativeLaunchTooLarge;
    if (c.mf) {
        if (!B.posfix || !B.pos32lo) return cudaErrorInvalidValue;
        k32_pos_fixed<<<(P.n + 255) / 256, 256, 0, L.stream>>>(P, B);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)g);
    cfg.blockDim = dim3((unsigned)c.bs);
    int smem = std::min(std::max(P.res_smem, 0), kResSmemBytes);
    cfg.dynamicSmemBytes = c.resident ? smem : 0;
    cfg.stream = L.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void* args[] = {const_cast<KParams*>(&P), &B, &smem};
    return cudaLaunchKernelExC(&cfg, c.fn, args);
}

}  // namespace ss
