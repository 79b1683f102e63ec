// Learned warm start for the velocity solve: a small message-passing network
// that guesses v = A^-1 b before CG (the paper has no learned part; the
// solve it accelerates is Eq. algebra of arXiv 1808.06381, §Method).
//
// Per node i and Cartesian component c (row r = 3 i + c), shared weights:
//   s = RMS of b;  x0 = (b / A_ii, vprev, b) / s
//   a0 = M x0 with (M u)_i = sum_j alpha w_ij / A_ii u_j       (message pass 1)
//   h1 = tanh([x0, a0] W1);  h2 = tanh(h1 W2);  y = h2 W3       (6 -> 64 -> 64 -> 4)
//   a1 = M y                                                     (message pass 2)
//   guess = s [y, a1, x0] . o
// The message passes run on the narrow features (like an SpMV of the solver);
// the MLP of inference is one kernel on the tcgen05 tensor cores (BF16
// operands in shared memory, FP32 accumulators in tensor memory, 128-row
// tiles; k_mp_mlp_fwd_tc).  Training (MSE to the converged velocities)
// recomputes the forward and runs the backward on the same tensor cores
// (k_mp_mlp_bwd_tc: activation gradients and the weight gradients as
// products over each tile's rows, accumulated in tensor memory across a
// block's tiles), then a deterministic reduction over blocks and Adam on FP32
// master weights.
#include <cuda_bf16.h>
#include <math.h>

#include <cstring>
#include <random>
#include <vector>

#include "sim_impl.cuh"

namespace ss {

namespace {

constexpr int kTileRows = 128;
constexpr int kMaxGradBlocks = 1024;

__device__ __forceinline__ unsigned smem_addr(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned*>(&v);
}

// Weight layouts in the packed BF16 array (element offsets).
constexpr int kW1T = 0;                 // [64][16]: W1 transposed, k padded 6 -> 16
constexpr int kW2T = kW1T + 64 * 16;    // [64][64]: W2 transposed
constexpr int kW3T = kW2T + 64 * 64;    // [8][64]:  W3 transposed, n padded 4 -> 8
constexpr int kW2N = kW3T + 8 * 64;     // [64][64]: W2 as is (backward)
constexpr int kW3P = kW2N + 64 * 64;    // [64][16]: W3 as is, k padded 4 -> 16 (backward)
constexpr int kWB = kW3P + 64 * 16;

// tanh by the hardware approximation (one MUFU operation, relative error
// below 2^-10): finer than the BF16 rounding the activations get next.
__device__ __forceinline__ float tanh_fast(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ------------------------------------------- forward MLP on tcgen05 tensor cores
//
// The three layers of a tile of 128 rows as 5th-generation tensor-core MMAs
// (tcgen05.mma, kind::f16, BF16 operands from shared memory, FP32
// accumulators in tensor memory), M = 128 rows: layer 1 [x0, a0] (K 6 -> 16)
// x W1 (N = 64), layer 2 h1 x W2 (K = N = 64, four K = 16 steps), layer 3 h2 x
// W3 (N 4 -> 16).  One thread issues the MMAs and commits them to an
// mbarrier; the four warps read the accumulators back with tcgen05.ld (warp w
// owns rows 32w..32w+31, its lane quarter of tensor memory), apply tanh, and
// store BF16 into the next layer's operand tile.  Operands use the
// no-swizzle K-major layout of 8 x 16-byte core matrices: element (r, k) of an
// R x K tile sits at ((r / 8) (K / 8) + k / 8) 128 + (r % 8) 16 + (k % 8) 2
// bytes, so the leading (K) core-matrix stride is 128 bytes and the stride
// between 8-row groups K / 8 x 128 bytes.  64 columns of tensor memory are
// reused by the three layers.  Every wait is bounded.
namespace tc {

constexpr int kRows = 128;
constexpr int kTmemCols = 64;
constexpr long long kWaitLimit = 1ll << 24;

__device__ __forceinline__ int core_off(int r, int k, int K)   // byte offset in a core-matrix tile
{
    return ((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ unsigned long long smem_desc(const void* base, int K)
{
    const unsigned long long addr = smem_addr(base);
    const unsigned long long lbo = 128, sbo = (unsigned long long)(K >> 3) * 128;
    return ((addr >> 4) & 0x3FFFull) | (((lbo >> 4) & 0x3FFFull) << 16) | (((sbo >> 4) & 0x3FFFull) << 32) |
           (1ull << 46);   // descriptor version 1; base offset 0, no swizzle
}

__host__ __device__ constexpr unsigned idesc_bf16(int M, int N)
{
    return (1u << 4)                  // D: FP32
           | (1u << 7) | (1u << 10)   // A, B: BF16
           | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);   // both K-major
}

__device__ __forceinline__ void mma(unsigned tmem_d, unsigned long long a, unsigned long long b, unsigned idesc,
                                    int accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void commit(void* mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
                 : "memory");
}

// bounded wait for the mbarrier phase with the given parity; false on timeout
__device__ __forceinline__ bool wait_phase(void* mbar, unsigned parity)
{
    const unsigned a = smem_addr(mbar);
    for (long long it = 0; it < kWaitLimit; ++it) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void ld16(unsigned taddr, float (&v)[16])
{
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

}  // namespace tc

}  // namespace

// y = h2 W3 with h2 = tanh(tanh([x0, a0] W1) W2), 128 rows per tile (see tc above).
__global__ void __launch_bounds__(128) k_mp_mlp_fwd_tc(int rows, MpBuffers M, DevState* st)
{
    using namespace tc;
    __shared__ __align__(128) unsigned char sA1[kRows * 16 * 2];   // [128][16] inputs
    __shared__ __align__(128) unsigned char sB1[64 * 16 * 2];      // [64][16]  W1^T
    __shared__ __align__(128) unsigned char sA2[kRows * 64 * 2];   // [128][64] h1, then h2
    __shared__ __align__(128) unsigned char sB2[64 * 64 * 2];      // [64][64]  W2^T
    __shared__ __align__(128) unsigned char sB3[16 * 64 * 2];      // [16][64]  W3^T (n padded 4 -> 16)
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ unsigned tmem_base;
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5;

    // weights (BF16, already transposed and padded) into core-matrix tiles
    for (int e = tid; e < 64 * 16; e += blockDim.x)
        *reinterpret_cast<__nv_bfloat16*>(sB1 + core_off(e / 16, e % 16, 16)) = M.wb[kW1T + e];
    for (int e = tid; e < 64 * 64; e += blockDim.x)
        *reinterpret_cast<__nv_bfloat16*>(sB2 + core_off(e / 64, e % 64, 64)) = M.wb[kW2T + e];
    for (int e = tid; e < 16 * 64; e += blockDim.x) {
        const int n = e / 64, k = e % 64;
        *reinterpret_cast<__nv_bfloat16*>(sB3 + core_off(n, k, 64)) =
            n < 8 ? M.wb[kW3T + n * 64 + k] : __float2bfloat16_rn(0.f);
    }
    if (tid == 0) {
        failed = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = tmem_base;
    const unsigned tlane = tmem + ((unsigned)(warp * 32) << 16);   // this warp's lane quarter
    const unsigned id1 = idesc_bf16(kRows, 64), id3 = idesc_bf16(kRows, 16);
    unsigned phase = 0;

    for (int base = blockIdx.x * kRows; base < rows && !failed; base += gridDim.x * kRows) {
        const int r = base + tid;   // this thread's row (tile row tid)
        {   // layer-1 operand: [x0, a0] in BF16, k 6..15 zero
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 x = r < rows ? M.x0[r] : z, a = r < rows ? M.a0[r] : z;
            uint4 lo, hi;
            lo.x = pack_bf16(x.x, x.y);
            lo.y = pack_bf16(x.z, a.x);
            lo.z = pack_bf16(a.y, a.z);
            lo.w = 0u;
            hi = make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4*>(sA1 + core_off(tid, 0, 16)) = lo;
            *reinterpret_cast<uint4*>(sA1 + core_off(tid, 8, 16)) = hi;
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0) {
            mma(tmem, smem_desc(sA1, 16), smem_desc(sB1, 16), id1, 0);
            commit(&mbar);
        }
        if (!wait_phase(&mbar, phase)) atomicExch(&failed, 1);
        phase ^= 1u;
        fence_after();
        // h1 = tanh(D), BF16 into the layer-2 operand
#pragma unroll
        for (int c = 0; c < 64; c += 16) {
            float v[16];
            ld16(tlane + c, v);
#pragma unroll
            for (int q = 0; q < 16; q += 8) {
                uint4 w;
                w.x = pack_bf16(tanh_fast(v[q]), tanh_fast(v[q + 1]));
                w.y = pack_bf16(tanh_fast(v[q + 2]), tanh_fast(v[q + 3]));
                w.z = pack_bf16(tanh_fast(v[q + 4]), tanh_fast(v[q + 5]));
                w.w = pack_bf16(tanh_fast(v[q + 6]), tanh_fast(v[q + 7]));
                *reinterpret_cast<uint4*>(sA2 + core_off(tid, c + q, 64)) = w;
            }
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0) {
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)   // K = 16 per step: two core matrices, 256 bytes
                mma(tmem, smem_desc(sA2 + ks * 256, 64), smem_desc(sB2 + ks * 256, 64), id1, ks > 0);
            commit(&mbar);
        }
        if (!wait_phase(&mbar, phase)) atomicExch(&failed, 1);
        phase ^= 1u;
        fence_after();
        // h2 = tanh(D) overwrites h1 (layer 2 has read it)
#pragma unroll
        for (int c = 0; c < 64; c += 16) {
            float v[16];
            ld16(tlane + c, v);
#pragma unroll
            for (int q = 0; q < 16; q += 8) {
                uint4 w;
                w.x = pack_bf16(tanh_fast(v[q]), tanh_fast(v[q + 1]));
                w.y = pack_bf16(tanh_fast(v[q + 2]), tanh_fast(v[q + 3]));
                w.z = pack_bf16(tanh_fast(v[q + 4]), tanh_fast(v[q + 5]));
                w.w = pack_bf16(tanh_fast(v[q + 6]), tanh_fast(v[q + 7]));
                *reinterpret_cast<uint4*>(sA2 + core_off(tid, c + q, 64)) = w;
            }
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0) {
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                mma(tmem, smem_desc(sA2 + ks * 256, 64), smem_desc(sB3 + ks * 256, 64), id3, ks > 0);
            commit(&mbar);
        }
        if (!wait_phase(&mbar, phase)) atomicExch(&failed, 1);
        phase ^= 1u;
        fence_after();
        {
            float v[16];
            ld16(tlane, v);
            if (r < rows) M.y[r] = make_float4(v[0], v[1], v[2], v[3]);
        }
        fence_before();
        __syncthreads();   // the next tile's MMAs overwrite tensor memory and the operands
        fence_after();
    }
    if (failed && tid == 0) atomicCAS(&st->error, 0, (int)SP_ERR_TIMEOUT);
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// ------------------------------------------ training backward on tcgen05
//
// One tile of 128 rows at a time, one thread per row, 128 threads; every
// product is a tcgen05.mma with M = 128 (BF16 operands in the no-swizzle
// K-major core-matrix layout above, FP32 accumulators in tensor memory):
//   h1 = tanh(X W1), h2 = tanh(h1 W2)             (forward recomputed; K 16, 64)
//   dp2 = (dY W3^T) (1 - h2^2)                     (A = dY [128][16], B = W3 [64][16])
//   dp1 = (dp2 W2^T) (1 - h1^2)                    (A = dp2 [128][64], B = W2 [64][64])
// and the weight gradients as products over the tile's rows (K = 128), with
// the tile's activations written transposed into the A and B operands:
//   [h1^T; h2^T] (128 x 128) x dp2^T (64 x 128)^T -> rows 0-63: dW2 = h1^T dp2
//   [h1^T; h2^T]             x dY^T  (16 x 128)^T -> rows 64-127: dW3 = h2^T dY
//   [dp1^T; 0]               x X^T   (16 x 128)^T -> rows 0-63: dW1^T = dp1^T X
// The three gradient accumulators stay in tensor memory across all the
// block's tiles and are read back once: one partial gradient per block,
// summed over blocks in a fixed order (k_mp_grad_reduce).  Tensor memory:
// columns 0-63 for the activations' products (reused), 64-127 dW2, 128-143
// dW3, 144-159 dW1^T.  The derivative of tanh uses the BF16 activations the
// products use.  Every wait is bounded.
namespace tcb {
constexpr int kBRows = 128;
constexpr int kBTmemCols = 256;
constexpr int kColW2 = 64, kColW3 = 128, kColW1 = 144;
// dynamic shared memory layout (byte offsets, 128-byte aligned)
constexpr int oW1T = 0;                      // [64][16]  W1^T          (B, layer 1)
constexpr int oW2T = oW1T + 64 * 16 * 2;     // [64][64]  W2^T          (B, layer 2)
constexpr int oW3P = oW2T + 64 * 64 * 2;     // [64][16]  W3 (k 4 -> 16) (B, dh2)
constexpr int oW2N = oW3P + 64 * 16 * 2;     // [64][64]  W2            (B, dh1)
constexpr int oX = oW2N + 64 * 64 * 2;       // [128][16] [x0, a0]      (A, layer 1)
constexpr int oH1 = oX + kBRows * 16 * 2;     // [128][64] h1            (A, layer 2)
constexpr int oDY = oH1 + kBRows * 64 * 2;    // [128][16] dY            (A, dh2)
constexpr int oP2 = oDY + kBRows * 16 * 2;    // [128][64] dp2           (A, dh1)
constexpr int oAT1 = oP2 + kBRows * 64 * 2;   // [128][128] [h1^T; h2^T] (A, dW2 and dW3)
constexpr int oAT2 = oAT1 + 128 * 128 * 2;   // [128][128] [dp1^T; 0]   (A, dW1^T)
constexpr int oBP2 = oAT2 + 128 * 128 * 2;   // [64][128] dp2^T         (B, dW2)
constexpr int oBDY = oBP2 + 64 * 128 * 2;    // [16][128] dY^T          (B, dW3)
constexpr int oBX = oBDY + 16 * 128 * 2;     // [16][128] X^T           (B, dW1^T)
constexpr int kSmem = oBX + 16 * 128 * 2;
}  // namespace tcb

int mp_bwd_tc_smem_bytes() { return tcb::kSmem + 128; }

__global__ void __launch_bounds__(128, 1) k_mp_mlp_bwd_tc(int rows, MpBuffers M, DevState* st)
{
    using namespace tc;
    using namespace tcb;
    extern __shared__ __align__(128) unsigned char sm_raw[];
    // the operand tiles start on a 128-byte boundary (the launch adds 128 bytes)
    unsigned char* sm = sm_raw + ((128u - (smem_addr(sm_raw) & 127u)) & 127u);
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ unsigned tmem_base;
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5;
    auto put = [&](int off, int r, int k, int K, float v) {
        *reinterpret_cast<__nv_bfloat16*>(sm + off + core_off(r, k, K)) = __float2bfloat16_rn(v);
    };
    auto get = [&](int off, int r, int k, int K) {
        return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(sm + off + core_off(r, k, K)));
    };
    // weights (BF16 layouts of k_mp_adam) into core-matrix tiles
    for (int e = tid; e < 64 * 16; e += blockDim.x) {
        *reinterpret_cast<__nv_bfloat16*>(sm + oW1T + core_off(e / 16, e % 16, 16)) = M.wb[kW1T + e];
        *reinterpret_cast<__nv_bfloat16*>(sm + oW3P + core_off(e / 16, e % 16, 16)) = M.wb[kW3P + e];
    }
    for (int e = tid; e < 64 * 64; e += blockDim.x) {
        *reinterpret_cast<__nv_bfloat16*>(sm + oW2T + core_off(e / 64, e % 64, 64)) = M.wb[kW2T + e];
        *reinterpret_cast<__nv_bfloat16*>(sm + oW2N + core_off(e / 64, e % 64, 64)) = M.wb[kW2N + e];
    }
    // rows 64-127 of [dp1^T; 0], rows 4-15 of dY^T and 6-15 of X^T stay zero
    for (int e = tid; e < 64 * 128; e += blockDim.x) put(oAT2, 64 + e / 128, e % 128, 128, 0.f);
    for (int e = tid; e < 12 * 128; e += blockDim.x) put(oBDY, 4 + e / 128, e % 128, 128, 0.f);
    for (int e = tid; e < 10 * 128; e += blockDim.x) put(oBX, 6 + e / 128, e % 128, 128, 0.f);
    if (tid == 0) {
        failed = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(kBTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = tmem_base;
    const unsigned tlane = tmem + ((unsigned)(warp * 32) << 16);   // this warp's lane quarter
    const unsigned id64 = idesc_bf16(kBRows, 64), id16 = idesc_bf16(kBRows, 16);
    unsigned phase = 0;
    int acc = 0;   // the gradient products accumulate after the block's first tile
    auto sync_mma = [&]() {   // operands written by all threads -> visible to the MMA issuer
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
    };
    auto wait_mma = [&]() {
        if (!wait_phase(&mbar, phase)) atomicExch(&failed, 1);
        phase ^= 1u;
        fence_after();
    };

    for (int base = blockIdx.x * kBRows; base < rows && !failed; base += gridDim.x * kBRows) {
        const int r = base + tid;   // this thread's row (tile row tid)
        {   // X = [x0, a0] (k 6..15 zero) and dY (k 4..15 zero): rows, and transposed
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 x = r < rows ? M.x0[r] : z, a = r < rows ? M.a0[r] : z, d = r < rows ? M.dy[r] : z;
            const float xs[6] = {x.x, x.y, x.z, a.x, a.y, a.z}, ds[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                put(oX, tid, k, 16, k < 6 ? xs[k] : 0.f);
                put(oDY, tid, k, 16, k < 4 ? ds[k] : 0.f);
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) put(oBX, k, tid, 128, xs[k]);
#pragma unroll
            for (int k = 0; k < 4; ++k) put(oBDY, k, tid, 128, ds[k]);
        }
        sync_mma();
        if (tid == 0) {
            mma(tmem, smem_desc(sm + oX, 16), smem_desc(sm + oW1T, 16), id64, 0);
            commit(&mbar);
        }
        wait_mma();
        // h1 = tanh(D): row operand and rows 0-63 of [h1^T; h2^T]
#pragma unroll
        for (int c = 0; c < 64; c += 16) {
            float v[16];
            ld16(tlane + c, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const float h = tanh_fast(v[q]);
                put(oH1, tid, c + q, 64, h);
                put(oAT1, c + q, tid, 128, h);
            }
        }
        sync_mma();
        if (tid == 0) {
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                mma(tmem, smem_desc(sm + oH1 + ks * 256, 64), smem_desc(sm + oW2T + ks * 256, 64), id64, ks > 0);
            commit(&mbar);
        }
        wait_mma();
        // h2 = tanh(D): rows 64-127 of [h1^T; h2^T]
#pragma unroll
        for (int c = 0; c < 64; c += 16) {
            float v[16];
            ld16(tlane + c, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) put(oAT1, 64 + c + q, tid, 128, tanh_fast(v[q]));
        }
        sync_mma();
        if (tid == 0) {   // dh2 = dY W3^T
            mma(tmem, smem_desc(sm + oDY, 16), smem_desc(sm + oW3P, 16), id64, 0);
            commit(&mbar);
        }
        wait_mma();
        // dp2 = dh2 (1 - h2^2): row operand and transposed
#pragma unroll
        for (int c = 0; c < 64; c += 16) {
            float v[16];
            ld16(tlane + c, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const float h = get(oAT1, 64 + c + q, tid, 128);
                const float g = v[q] * (1.f - h * h);
                put(oP2, tid, c + q, 64, g);
                put(oBP2, c + q, tid, 128, g);
            }
        }
        sync_mma();
        if (tid == 0) {   // dh1 = dp2 W2^T
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                mma(tmem, smem_desc(sm + oP2 + ks * 256, 64), smem_desc(sm + oW2N + ks * 256, 64), id64, ks > 0);
            commit(&mbar);
        }
        wait_mma();
        // dp1 = dh1 (1 - h1^2), transposed into rows 0-63 of [dp1^T; 0]
#pragma unroll
        for (int c = 0; c < 64; c += 16) {
            float v[16];
            ld16(tlane + c, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const float h = get(oH1, tid, c + q, 64);
                put(oAT2, c + q, tid, 128, v[q] * (1.f - h * h));
            }
        }
        sync_mma();
        if (tid == 0) {   // the weight gradients, summed over the tile's rows (K = 128)
#pragma unroll
            for (int ks = 0; ks < 8; ++ks) {
                const int a = acc | (ks > 0);
                mma(tmem + kColW2, smem_desc(sm + oAT1 + ks * 256, 128), smem_desc(sm + oBP2 + ks * 256, 128), id64, a);
                mma(tmem + kColW3, smem_desc(sm + oAT1 + ks * 256, 128), smem_desc(sm + oBDY + ks * 256, 128), id16, a);
                mma(tmem + kColW1, smem_desc(sm + oAT2 + ks * 256, 128), smem_desc(sm + oBX + ks * 256, 128), id16, a);
            }
            commit(&mbar);
        }
        wait_mma();   // the next tile overwrites the operands
        acc = 1;
        fence_before();
        __syncthreads();
        fence_after();
    }
    // this block's partial gradient (zero if it had no tile)
    float* gp = M.gpart + (size_t)blockIdx.x * kMpParams;
    if (acc && !failed) {
        if (warp < 2) {   // rows 0-63: dW2[i][h] (i = row) and dW1^T[i][f]
            const int i = tid;
#pragma unroll
            for (int c = 0; c < 64; c += 16) {
                float v[16];
                ld16(tlane + kColW2 + c, v);
#pragma unroll
                for (int q = 0; q < 16; ++q) gp[kMpOffW2 + i * 64 + c + q] = v[q];
            }
            float v[16];
            ld16(tlane + kColW1, v);
#pragma unroll
            for (int f = 0; f < 6; ++f) gp[kMpOffW1 + f * 64 + i] = v[f];
        } else {          // rows 64-127: dW3[h][m] (h = row - 64)
            const int h = tid - 64;
            float v[16];
            ld16(tlane + kColW3, v);
#pragma unroll
            for (int m = 0; m < 4; ++m) gp[kMpOffW3 + h * 4 + m] = v[m];
        }
    } else {
        for (int e = tid; e < kMpOffO; e += blockDim.x) gp[e] = 0.f;
    }
    if (failed && tid == 0) atomicCAS(&st->error, 0, (int)SP_ERR_TIMEOUT);
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kBTmemCols) : "memory");
}

namespace {
}  // namespace

// -------------------------------------------------------------- kernels

// Component c of b at row i: the mixed path keeps b as double-floats only.
__device__ __forceinline__ double b_at(const DevBuffers& B, int np, int c, int i)
{
    if (B.bdf) {
        const float4 h = B.bdf[2 * i], l = B.bdf[2 * i + 1];
        return c == 0 ? (double)h.x + (double)l.x : (c == 1 ? (double)h.y + (double)l.y : (double)h.z + (double)l.z);
    }
    return B.b[c * np + i];
}

// s = sqrt(sum b^2 / 3n) (1 if b = 0)
__global__ void k_mp_scale(KParams P, DevBuffers B, MpBuffers M)
{
    const int np = P.npad;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x)
        for (int c = 0; c < 3; ++c) {
            const double b = M.in ? M.in[c * np + i] : b_at(B, np, c, i);
            acc += b * b;
        }
    const double v[1] = {acc};
    if (publish_partials<1>(v, M.part, &M.ticket[0])) {
        double out[1];
        reduce_partials<1>(M.part, out);
        if (threadIdx.x == 0) {
            const double s = sqrt(out[0] / (3.0 * P.n));
            M.scal[0] = s > 0.0 ? s : 1.0;
        }
    }
}

// x0 rows (b / A_ii, vprev, b) / s, with vprev = the current x (the previous velocities).
__global__ void k_mp_input(KParams P, DevBuffers B, MpBuffers M)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const int np = P.npad;
    const float inv = (float)(1.0 / M.scal[0]);
    const double di = B.bdf ? (double)B.dinv32[i] : B.dinv[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double b = M.in ? M.in[c * np + i] : b_at(B, np, c, i);
        const float vp = M.zero_vprev ? 0.f : (float)B.x[c * np + i] * inv;
        M.x0[3 * i + c] = make_float4((float)(b * di) * inv, vp, (float)b * inv, 0.f);
    }
}

// out = M in (mode 0), out = M^T in (mode 1), out += M^T in (mode 2); three rows per node.
__global__ void k_mp_aggregate(KParams P, DevBuffers B, const float4* __restrict__ in, float4* __restrict__ out,
                               int mode)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const int slot = B.row_slot[i];
    const int base = B.chunk_off[slot >> 5] + (slot & 31);
    const int cnt = B.row_cnt[i];
    const float ae = (float)P.alpha;
    float4 s[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) s[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 0; k < cnt; ++k) {
        const int e = base + 32 * k;
        const int j = B.col[e];
        float w = ae * B.val32[e];
        if (mode != 0) w *= B.dinv32[j];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 u = in[3 * j + c];
            s[c].x = fmaf(w, u.x, s[c].x);
            s[c].y = fmaf(w, u.y, s[c].y);
            s[c].z = fmaf(w, u.z, s[c].z);
            s[c].w = fmaf(w, u.w, s[c].w);
        }
    }
    const float di = mode == 0 ? B.dinv32[i] : 1.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float4 r = make_float4(s[c].x * di, s[c].y * di, s[c].z * di, s[c].w * di);
        if (mode == 2) {
            const float4 o = out[3 * i + c];
            r = make_float4(r.x + o.x, r.y + o.y, r.z + o.z, r.w + o.w);
        }
        out[3 * i + c] = r;
    }
}

// Second message pass fused with the output: a1 = M y for node i, then
// guess = s [y, a1, x0] . o written as the start vector of CG (a1 is kept
// for training).
__global__ void k_mp_aggregate_output(KParams P, DevBuffers B, MpBuffers M)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const int slot = B.row_slot[i];
    const int base = B.chunk_off[slot >> 5] + (slot & 31);
    const int cnt = B.row_cnt[i];
    const float ae = (float)P.alpha;
    float4 acc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 0; k < cnt; ++k) {
        const int e = base + 32 * k;
        const int j = B.col[e];
        const float w = ae * B.val32[e];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 u = M.y[3 * j + c];
            acc[c].x = fmaf(w, u.x, acc[c].x);
            acc[c].y = fmaf(w, u.y, acc[c].y);
            acc[c].z = fmaf(w, u.z, acc[c].z);
            acc[c].w = fmaf(w, u.w, acc[c].w);
        }
    }
    const float di = B.dinv32[i];
    const double s = M.scal[0];
    const float* o = M.master + kMpOffO;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int r = 3 * i + c;
        const float4 a = make_float4(acc[c].x * di, acc[c].y * di, acc[c].z * di, acc[c].w * di);
        M.a1[r] = a;
        const float4 y = M.y[r], x = M.x0[r];
        const float out = y.x * o[0] + y.y * o[1] + y.z * o[2] + y.w * o[3] + a.x * o[4] + a.y * o[5] + a.z * o[6] +
                          a.w * o[7] + x.x * o[8] + x.y * o[9] + x.z * o[10];
        (M.out ? M.out : B.x)[c * P.npad + i] = s * (double)out;
    }
}

// Loss rows: e = out - vstar / s, dout = 2 e / 3n; dy = dout o[0:4], g1 = dout o[4:8];
// per block: sum e^2 and the readout gradient sum dout [y, a1, x0].
__global__ void k_mp_loss(KParams P, DevBuffers B, MpBuffers M)
{
    const double s = M.scal[0];
    const float* o = M.master + kMpOffO;
    const int rows = 3 * P.n;
    double acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = 0.0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
        const int i = r / 3, c = r - 3 * i;
        const float4 y = M.y[r], a = M.a1[r], x = M.x0[r];
        const float out = y.x * o[0] + y.y * o[1] + y.z * o[2] + y.w * o[3] + a.x * o[4] + a.y * o[5] + a.z * o[6] +
                          a.w * o[7] + x.x * o[8] + x.y * o[9] + x.z * o[10];
        const double e = (double)out - B.x[c * P.npad + i] / s;
        const float d = (float)(2.0 * e / rows);
        M.dy[r] = make_float4(d * o[0], d * o[1], d * o[2], d * o[3]);
        M.g1[r] = make_float4(d * o[4], d * o[5], d * o[6], d * o[7]);
        const float f[11] = {y.x, y.y, y.z, y.w, a.x, a.y, a.z, a.w, x.x, x.y, x.z};
        acc[0] += e * e;
#pragma unroll
        for (int k = 0; k < 11; ++k) acc[1 + k] += (double)(d * f[k]);
    }
    __shared__ double sh[32];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const double t = block_sum(acc[k], sh);
        if (threadIdx.x == 0) M.dpart[blockIdx.x * 12 + k] = t;
    }
}

// grad = sum over blocks (fixed order); the readout's gradient and the loss from the loss blocks.
__global__ void k_mp_grad_reduce(MpBuffers M, int nblocks_mlp, int nblocks_loss, int rows)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < kMpOffO) {
        float s = 0.f;
        for (int b = 0; b < nblocks_mlp; ++b) s += M.gpart[(size_t)b * kMpParams + p];
        M.grad[p] = s;
    } else if (p < kMpParams) {
        double s = 0.0;
        for (int b = 0; b < nblocks_loss; ++b) s += M.dpart[b * 12 + 1 + (p - kMpOffO)];
        M.grad[p] = (float)s;
    } else if (p == kMpParams) {
        double s = 0.0;
        for (int b = 0; b < nblocks_loss; ++b) s += M.dpart[b * 12];
        M.scal[1] = s / rows;
    }
}

// Adam (Kingma & Ba 2015) on the FP32 masters, then the BF16 layouts for the kernels.
__global__ void k_mp_adam(MpBuffers M, float lr, int t)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kMpParams) return;
    if (lr != 0.f) {
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        const float gp = M.grad[p];
        const float m = b1 * M.m[p] + (1.f - b1) * gp;
        const float v = b2 * M.v[p] + (1.f - b2) * gp * gp;
        M.m[p] = m;
        M.v[p] = v;
        const float mh = m / (1.f - powf(b1, (float)t));
        const float vh = v / (1.f - powf(b2, (float)t));
        M.master[p] -= lr * mh / (sqrtf(vh) + eps);
    }
    const __nv_bfloat16 w = __float2bfloat16_rn(M.master[p]);
    if (p < kMpOffW2) {
        const int f = p / 64, i = p % 64;     // W1[f][i]
        M.wb[kW1T + i * 16 + f] = w;
    } else if (p < kMpOffW3) {
        const int q = p - kMpOffW2, i = q / 64, h = q % 64;   // W2[i][h]
        M.wb[kW2T + h * 64 + i] = w;
        M.wb[kW2N + i * 64 + h] = w;
    } else if (p < kMpOffO) {
        const int q = p - kMpOffW3, h = q / 4, m = q % 4;     // W3[h][m]
        M.wb[kW3T + m * 64 + h] = w;
        M.wb[kW3P + h * 16 + m] = w;
    }
}

// ------------------------------------------------------------------ launchers

void launch_mp_infer(const KParams& P, DevBuffers& B, MpBuffers& M, Launch L)
{
    const int rows = 3 * P.n;
    k_mp_scale<<<grid_for(P.n, kVecBlock, L.num_sms * 4), kVecBlock, 0, L.stream>>>(P, B, M);
    k_mp_input<<<grid_for(P.n, kVecBlock, 1 << 30), kVecBlock, 0, L.stream>>>(P, B, M);
    k_mp_aggregate<<<grid_for(P.n, 128, 1 << 30), 128, 0, L.stream>>>(P, B, M.x0, M.a0, 0);
    k_mp_mlp_fwd_tc<<<grid_for(rows, tc::kRows, L.num_sms * 6), tc::kRows, 0, L.stream>>>(rows, M, B.st);
    k_mp_aggregate_output<<<grid_for(P.n, 128, 1 << 30), 128, 0, L.stream>>>(P, B, M);
}

int mp_infer_launches() { return 5; }

void launch_mp_apply(const KParams& P, DevBuffers& B, const MpBuffers& M, const double* in, double* out, Launch L)
{
    MpBuffers A = M;
    A.in = in;
    A.out = out;
    A.zero_vprev = 1;
    launch_mp_infer(P, B, A, L);
}

void launch_mp_train(const KParams& P, DevBuffers& B, MpBuffers& M, float lr, int t, Launch L)
{
    const int rows = 3 * P.n;
    const int nloss = grid_for(rows, kVecBlock, std::min(kMaxGradBlocks, L.num_sms * 4));
    k_mp_loss<<<nloss, kVecBlock, 0, L.stream>>>(P, B, M);
    k_mp_aggregate<<<grid_for(P.n, 128, 1 << 30), 128, 0, L.stream>>>(P, B, M.g1, M.dy, 2);
    const int nmlp = grid_for(rows, kTileRows, std::min(kMaxGradBlocks, L.num_sms));
    k_mp_mlp_bwd_tc<<<nmlp, 128, mp_bwd_tc_smem_bytes(), L.stream>>>(rows, M, B.st);
    k_mp_grad_reduce<<<grid_for(kMpParams + 1, kVecBlock, 1 << 30), kVecBlock, 0, L.stream>>>(M, nmlp, nloss, rows);
    k_mp_adam<<<grid_for(kMpParams, kVecBlock, 1 << 30), kVecBlock, 0, L.stream>>>(M, lr, t);
}

int mp_prepare()
{
    return (int)cudaFuncSetAttribute(k_mp_mlp_bwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     mp_bwd_tc_smem_bytes());
}

int mp_weights_bf16_count() { return kWB; }

void launch_mp_convert(MpBuffers& M, cudaStream_t s)
{
    k_mp_adam<<<grid_for(kMpParams, kVecBlock, 1 << 30), kVecBlock, 0, s>>>(M, 0.f, 1);
}

}  // namespace ss
