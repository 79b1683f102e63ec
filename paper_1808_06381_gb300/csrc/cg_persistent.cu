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
// Grid barrier: one arrival counter (acquire-release atomic), a generation
// word on its own line that the last arriving block releases, and the error
// flag copied next to it by that block.  After the barrier every block sums
// all blocks' partial sums itself, in one fixed order.  The launch is
// cooperative (all blocks resident), and every wait is bounded by the global
// timer: a block that waits longer than kBarrierTimeoutNs sets
// SP_ERR_TIMEOUT and leaves the solve, so no GPU can hang on it.
#include <math.h>

#include <mutex>

#include "internal.cuh"

namespace ss {

namespace {

constexpr int kPBlock = 256;
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;   // 2 s

struct PShared {
    float2 df[32];
    double d[32];
    double bcast[4];
    int flag;
    // decided by thread 0 (FP64 scalars once per block, not once per thread)
    float alpha_f, beta_f;
    int action;   // 0 continue, 1 replace the residual, 2 stop
    // thread 0's CG state, kept here rather than in every thread's registers
    double rho, rr_restart, bnorm2, last_res;
    int iter, restarts, status;
};

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned int* p, unsigned int v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned int atom_add_acq_rel_gpu(unsigned int* p, unsigned int v)
{
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Arrival and release by thread 0; returns the error flag (0 = continue).
// The writes of every thread of every block before the barrier are visible
// to every thread after it (release by each arrival, acquire by the waiters,
// and the block barriers on both sides).
__device__ __forceinline__ int barrier_thread0(DevState* st, unsigned int target, int nb)
{
    if (atom_add_acq_rel_gpu(&st->bar_count, 1u) == (unsigned)nb - 1) {
        const int e = *(volatile int*)&st->error;
        st->bar_err = e;
        st->bar_count = 0u;
        st_release_gpu(&st->bar_gen, target);
        return e;
    }
    const unsigned long long t0 = global_ns();
    for (unsigned int polls = 1;; ++polls) {
        if (ld_acquire_gpu(&st->bar_gen) == target) return *(volatile int*)&st->bar_err;
        if ((polls & 255u) == 0u && global_ns() - t0 > kBarrierTimeoutNs) {
            atomicCAS(&st->error, 0, (int)SP_ERR_TIMEOUT);
            return (int)SP_ERR_TIMEOUT;
        }
    }
}

// Grid barrier (the blocks of one system).  Returns false when the solve
// must stop (an error was raised anywhere, including a barrier timeout).
__device__ __forceinline__ bool grid_sync(DevState* st, unsigned int& gen, PShared& sh, int nb)
{
    __syncthreads();
    if (threadIdx.x == 0) sh.flag = barrier_thread0(st, gen + 1u, nb);
    __syncthreads();
    gen += 1u;
    return sh.flag == 0;
}

// Grid-wide sums of K double-float values: every block publishes its block
// sums, passes the barrier, then sums all blocks' partials itself, in the
// same fixed order in every block (so all blocks hold identical totals).
// Consecutive calls must use alternating partial sets: a block may still be
// reading one set when a faster block writes the next.
template <int K>
__device__ __forceinline__ bool grid_allreduce(DevState* st, unsigned int& gen, PShared& sh,
                                               const dfloat (&v)[K], float2* partials, double (&out)[K],
                                               int bid, int nb)
{
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const dfloat t = block_sum_df(v[k], sh.df);
        if (threadIdx.x == 0) partials[k * kMaxPartials + bid] = make_float2(t.hi, t.lo);
    }
    if (threadIdx.x == 0) sh.flag = barrier_thread0(st, gen + 1u, nb);
    __syncthreads();
    gen += 1u;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        dfloat a{0.f, 0.f};
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const float2 p = __ldcg(partials + k * kMaxPartials + b);
            a = df_add(a, dfloat{p.x, p.y});
        }
        const dfloat t = block_sum_df(a, sh.df);
        if (threadIdx.x == 0) sh.bcast[k] = (double)t.hi + (double)t.lo;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = sh.bcast[k];
    return sh.flag == 0;
}

// The same for FP64 values (the rare FP64 residual replacement).
template <int K>
__device__ __forceinline__ bool grid_allreduce(DevState* st, unsigned int& gen, PShared& sh,
                                               const double (&v)[K], double* partials, double (&out)[K],
                                               int bid, int nb)
{
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double t = block_sum(v[k], sh.d);
        if (threadIdx.x == 0) partials[k * kMaxPartials + bid] = t;
    }
    if (threadIdx.x == 0) sh.flag = barrier_thread0(st, gen + 1u, nb);
    __syncthreads();
    gen += 1u;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double a = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) a += __ldcg(partials + k * kMaxPartials + b);
        const double t = block_sum(a, sh.d);
        if (threadIdx.x == 0) sh.bcast[k] = t;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = sh.bcast[k];
    return sh.flag == 0;
}

constexpr int kBatchP = 6;    // FP32 gathers in flight per thread (batch kernel; see kPersistentCfg)
constexpr int kBatchP64 = 2;  // FP64 gathers in flight (the rare FP64 residual replacement)

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

// s_a = sum_j w_ij x_a[j] (FP64 planes).
__device__ __forceinline__ void p_row_sum64(const int* __restrict__ col, const double* __restrict__ val,
                                            const double* x, int np, int e0, int e1, double& s0, double& s1,
                                            double& s2)
{
    s0 = s1 = s2 = 0.0;
    for (int eb = e0; eb < e1; eb += 32 * kBatchP64) {
        int j[kBatchP64];
        double w[kBatchP64];
#pragma unroll
        for (int u = 0; u < kBatchP64; ++u) {
            const int e = eb + 32 * u;
            j[u] = 0;
            w[u] = 0.0;
            if (e < e1) {
                j[u] = __ldg(col + e);
                w[u] = __ldg(val + e);
            }
        }
#pragma unroll
        for (int u = 0; u < kBatchP64; ++u) {
            if (w[u] != 0.0) {
                s0 += w[u] * __ldcg(x + j[u]);
                s1 += w[u] * __ldcg(x + np + j[u]);
                s2 += w[u] * __ldcg(x + 2 * np + j[u]);
            }
        }
    }
}

}  // namespace

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
template <int KB, bool PIPE>
__device__ __forceinline__ void persistent_solve(const KParams& P, const DevBuffers& B, int bid, int nb,
                                                 PShared& sh)
{
    DevState* st = B.st;
    if (threadIdx.x == 0) sh.flag = 0;
    __syncthreads();
    if (st->error | st->overflow | st->done) return;   // uniform: set before the launch
    unsigned int gen = 0u;   // used by thread 0 only
    if (threadIdx.x == 0) gen = *(volatile unsigned int*)&st->bar_gen;

    const int nwin = P.nslots / 256;
    const int wb = (int)((long long)bid * nwin / nb);
    const int we = (int)((long long)(bid + 1) * nwin / nb);
    const int G = blockDim.x >> 8;                              // window groups
    const int t = threadIdx.x & 255, wg = wb + (threadIdx.x >> 8);   // lane in window, first window
    const int np = P.npad;
    const float alpha_e = (float)P.alpha;

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
                    const double target = fmax(P.inner2 * sh.rr_restart, 0.25 * P.tol2 * sh.bnorm2);
                    if (tot[0] <= target || sh.iter >= P.max_iter) sh.action = 1;
                }
            }
        }
        __syncthreads();
        if (sh.action == 2) break;
        if (sh.action == 0) continue;

        // ---- residual replacement: x += d (own rows), then r = b - A x in FP64
        for (int w = wg; w < we; w += G) {
            const int i = w * 256 + t;
            if (i < P.n) {
                const float4 d = B.d4[i];
                B.x[i] += (double)d.x;
                B.x[np + i] += (double)d.y;
                B.x[2 * np + i] += (double)d.z;
                B.d4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        if (!grid_sync(st, gen, sh, nb)) break;
        double trr = 0.0, trz = 0.0;
        for (int w = wg, k = 0; w < we; w += G, ++k) {
            const int slot = w * 256 + chunk_lane(k, t);
            const int row = B.slot_row[slot];
            if (row >= 0) {
                const int e0 = B.chunk_off[slot >> 5] + (slot & 31);
                const int e1 = B.chunk_off[(slot >> 5) + 1];
                double s[3];
                p_row_sum64(B.col, B.val, B.x, np, e0, e1, s[0], s[1], s[2]);
                const double d = B.diag[row];
                const float di = B.dinv32[row];
                double rk[3];
                double rs = 0.0;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int k = c * np + row;
                    rk[c] = B.b[k] - (d * B.x[k] - P.alpha * s[c]);
                    rs += rk[c] * rk[c];
                }
                B.r4[row] = make_float4((float)rk[0], (float)rk[1], (float)rk[2], di);
                trr += rs;
                trz += (double)di * rs;
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

// Tile configurations of the single-system kernel: gathers in flight per
// thread (KB) against resident blocks per SM (MINB, which caps the registers
// at 65536 / (256 MINB)), with or without requesting the next batch's
// columns during the current gathers (PIPE).  Chosen per system by the
// autotuner.
template <int KB, int MINB, bool PIPE, int BS>
__global__ void __launch_bounds__(BS, MINB) k32_cg_persistent(KParams P, DevBuffers B)
{
    __shared__ PShared sh;
    persistent_solve<KB, PIPE>(P, B, blockIdx.x, gridDim.x, sh);
}

// Batch: block b serves replica k with blk_off[k] <= b < blk_off[k + 1]; each
// replica's blocks synchronise and reduce among themselves only, and leave
// when their replica has converged.
__global__ void __launch_bounds__(kPBlock, 4) k32_cg_persistent_batch(const KParams* __restrict__ Ps,
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
    persistent_solve<kBatchP, false>(Ps[k], Bs[k], (int)blockIdx.x - blk_off[k], blk_off[k + 1] - blk_off[k], sh);
}

namespace {
struct PCfg {
    int kb, minb, pipe, bs;
    const void* fn;
    int occ;
};
PCfg g_pcfg[kPersistentConfigs] = {   // entry 0: the default without autotuning
    {6, 1, 0, 1024, (const void*)k32_cg_persistent<6, 1, false, 1024>, 0},
    {8, 1, 0, 1024, (const void*)k32_cg_persistent<8, 1, false, 1024>, 0},
    {6, 4, 0, 256, (const void*)k32_cg_persistent<6, 4, false, 256>, 0},
    {8, 4, 0, 256, (const void*)k32_cg_persistent<8, 4, false, 256>, 0},
    {4, 4, 0, 256, (const void*)k32_cg_persistent<4, 4, false, 256>, 0},
    {4, 4, 1, 256, (const void*)k32_cg_persistent<4, 4, true, 256>, 0},
    {5, 4, 1, 256, (const void*)k32_cg_persistent<5, 4, true, 256>, 0},
    {6, 3, 1, 256, (const void*)k32_cg_persistent<6, 3, true, 256>, 0},
};
int g_pocc_batch = 0;
std::once_flag g_pocc_once;
void pocc_init()
{
    std::call_once(g_pocc_once, [] {
        for (auto& c : g_pcfg)
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ, c.fn, c.bs, 0) != cudaSuccess) c.occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_pocc_batch, k32_cg_persistent_batch, kPBlock, 0) !=
            cudaSuccess)
            g_pocc_batch = 0;
        cudaGetLastError();
    });
}
const PCfg& cfg_of(const KParams& P)
{
    const int k = (P.pcfg >= 0 && P.pcfg < kPersistentConfigs) ? P.pcfg : 0;
    return g_pcfg[k];
}
}  // namespace

int cg_persistent_batch_capacity(Launch L)
{
    pocc_init();
    return L.num_sms * g_pocc_batch;
}

cudaError_t launch_cg32_persistent_batch(const KParams* Ps_dev, const DevBuffers* Bs_dev, const int* blk_off_dev,
                                         int R, int total_blocks, Launch L)
{
    if (total_blocks < 1 || total_blocks > cg_persistent_batch_capacity(L)) return cudaErrorCooperativeLaunchTooLarge;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)total_blocks);
    cfg.blockDim = dim3(kPBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = L.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k32_cg_persistent_batch, Ps_dev, Bs_dev, blk_off_dev, R);
}

void cg_persistent_config(int k, int* gathers, int* blocks_per_sm, int* pipelined, int* block_threads)
{
    const PCfg& c = g_pcfg[(k >= 0 && k < kPersistentConfigs) ? k : 0];
    *gathers = c.kb;
    *blocks_per_sm = c.minb;
    *pipelined = c.pipe;
    *block_threads = c.bs;
}

int cg_persistent_grid(const KParams& P, Launch L)
{
    pocc_init();
    const PCfg& c = cfg_of(P);
    const long long groups = c.bs / 256;   // windows a block processes at once
    long long g = std::min<long long>((long long)L.num_sms * c.occ, (P.nslots / 256 + groups - 1) / groups);
    if (g > kMaxPartials) g = kMaxPartials;
    return (int)g;
}

cudaError_t launch_cg32_persistent(const KParams& P, DevBuffers& B, Launch L)
{
    const int g = cg_persistent_grid(P, L);
    if (g < 1) return cudaErrorCooperativeLaunchTooLarge;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)g);
    cfg.blockDim = dim3((unsigned)cfg_of(P).bs);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = L.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void* args[] = {const_cast<KParams*>(&P), &B};
    return cudaLaunchKernelExC(&cfg, cfg_of(P).fn, args);
}

}  // namespace ss
