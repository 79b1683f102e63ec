// Internal declarations of the shearsim CUDA library (sm_103a).
// Device helpers shared by the kernels of this library, the per-simulation
// device state, and host launchers for the kernels of each translation unit.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "shearsim.h"

namespace ss {

constexpr int kMaxCgRestarts = 4;    // true-residual restarts per solve before giving up
// Mixed solver: the inner FP32 iteration that may end the solve stops once its
// recursive ||r||^2 <= kInnerFinal2 tol^2 ||b||^2.  The recursion started from
// a true residual at most ~1e-4 ||b|| (or from the initial residual), so FP32
// rounding and the rounded weights move it from the true residual by ~1e-10
// ||b||, far inside the 10 % margin; the true residual in double-float decides.
constexpr double kInnerFinal2 = 0.81;
constexpr int kVecBlock = 256;       // threads per block of the streaming kernels

// Constants of one simulation, passed by value to every kernel.
struct KParams {
    int n;              // particles (rows)
    int npad;           // stride between the x, y, z planes of a vector
    double L[3];
    double rc2;         // r_c^2: pair kept iff |R|^2 < rc2
    double two_lambda2; // 2 lambda^2, lambda^2 = r_c^2 / (2 ln 20)
    double w_scale;     // 256 / (2 lambda^2): index scale of the weight table
    double alpha, zeta, kappa, dt;
    double c_ev;        // eps * 0.1 * kT / lambda^2
    double noise_amp;   // sqrt(2 zeta kT / dt)
    unsigned long long seed;
    int nc[3];          // cells per axis (cell edge >= r_c)
    double inv_cw[3];   // cells per unit length
    int ncell;          // cell index slots: tiles of 8^3 cells, ntile[0] * ntile[1] * ntile[2] * 512
    int ntile[3];       // tiles per axis
    int nslots;         // rows rounded up to a multiple of 256
    int nchunks;        // nslots / 32
    int fast_cells;     // every axis has >= 3 cells: FP32 pre-filter with exact fallback
    float rc2_lo;       // FP32 distance^2 below this: certainly |R|^2 < r_c^2
    float rc2_hi;       // FP32 distance^2 at or above this: certainly |R|^2 >= r_c^2
    float Lf[3];        // box edges in FP32
    float Llo[3];       // L - Lf: the box edges as double-floats (Lf, Llo)
    float wsc_hi, wsc_lo; // w_scale as a double-float
    double tol2;        // cg_tol^2
    double inner2;      // mixed solver: inner FP32 solve stops at ||r||^2 <= inner2 * ||r_restart||^2
    int max_iter;
    int mixed;          // 1: the mixed path (double-float assembly and normals)
    float alpha_hi, alpha_lo;   // alpha as a double-float (mixed solver's residuals)
    // the mixed assembly's row finish in double-float: b = amp_z g + cev_z f
    // (+ kappa (y - L_y / 2) + akl sum n w for the x component)
    float amp_z_hi, amp_z_lo;   // noise_amp / zeta
    float cev_z_hi, cev_z_lo;   // c_ev / zeta
    float kap_hi, kap_lo;       // kappa
    float hly_hi, hly_lo;       // L_y / 2
    float akl_hi, akl_lo;       // alpha kappa L_y
    int pcfg;           // tile configuration of the persistent solver (index, autotuned)
    int res_smem;       // shared memory the on-chip solve uses (<= kResSmemBytes; less only to test its fallback)
    int fused_init;     // on-chip solve: 0 after the initial-residual kernel; 1 forms r = b itself (x0 = 0), 2 r = b - A x0
    long long hcopy;    // on-chip solve: where hcol / hval / hlo hold a second copy region (the lists of blocks
                        // whose entries all stay off chip, at their sliced positions + hcopy); 0: none, and the
                        // blocks then take whole windows
    // matrix-free SpMV of the streaming mixed solve: positions in 32-bit fixed
    // point of each box edge (one unit L / 2^32), w = 2^(w_exp2 |R|^2)
    double fix_inv[3];  // 2^32 / L
    float fix_scale[3]; // L / 2^32
    float w_exp2;       // -log2(e) / (2 lambda^2)
    float c_ev_f, za_f, kly_f;  // c_ev, zeta alpha and kappa L_y in FP32 (the mixed path's stress)
};

constexpr int kPersistentConfigs = 12;
constexpr int kResSmemBytes = 190 * 1024;   // on-chip solve: dynamic shared memory per block
constexpr int kResLoStride = 49152;          // >= kResSmemBytes / 4: local entries of one block

// Scalars that live on the device so that a whole step runs without the host.
struct DevState {
    double delta;             // Lees-Edwards image offset of the image at y + L_y
    long long step;           // step counter (noise key)
    long long nnz;            // off-diagonal entries of the current matrix (2 x pairs)
    long long nnz_slots;      // entries including the padding of the sliced layout
    long long nnz_cap;        // capacity of col / val / img
    int overflow;             // sticky: nnz exceeded nnz_cap
    int error;                // sticky: first failing sp_status of a step (0 = none)
    // conjugate gradients
    double bnorm2, rho, alpha, beta, rr, pq, rr_true, rr_restart;
    int iter, restarts, done, status, check_true, zero_b;
    // mixed precision bookkeeping
    int since_replace;
    // statistics accumulated over the steps of one sp_step call
    long long iter_sum;
    int iter_max;
    int steps_in_call;
    long long true_checks;
    double last_res;
    double stress_xy;
    unsigned int ticket[4];
    // grid barriers of the persistent solvers: arrivals counted up through a
    // launch (barrier k of a launch is passed once k x blocks have arrived),
    // and on its own line the blocks that have left the launch (the last one
    // resets both, so every launch starts from 0)
    alignas(128) unsigned int bar_count;
    alignas(128) unsigned int bar_exit;
    long long noise_step;     // step whose normals noise3 holds (-1: none)
    int res_offchip;          // on-chip solve: blocks whose rows did not fit on their SM (last solve)
    double delta_next;        // the offset the position update advanced to (committed after the stress)
    unsigned long long bar_timeout_ns;   // limit of one grid-barrier wait of the persistent solvers
};

constexpr unsigned long long kDefaultWaitLimitNs = 2000000000ull;   // 2 s

// Device buffers of one simulation (all in the current cell order unless noted).
struct DevBuffers {
    // state (order of the previous build)
    double* pos_s;   // [3][npad]
    int* id_s;       // [n]
    double* v_s;     // [3][npad] velocities of the last solve
    // work arrays of the current step (cell order)
    double* pos_w;   // [3][npad]
    float* pos32;    // [3][npad] FP32 copy of pos_w for the pair pre-filter
    float* pos32lo;  // [3][npad] pos_w - pos32: positions as double-floats (pos32, pos32lo)
    int* id_w;       // [n]
    int* cell_of;    // [n] cell of each row: in the state order while binning, then (written by the
                     // per-cell sort) in the cell order of the current rows, where the pair search reads it
    int* slot;       // [n]
    int* perm;       // [n] new row -> state row
    int* cell_count; // [ncell]
    int* cell_start; // [ncell + 1]
    // Matrix in sliced ELLPACK (SELL-32-sigma256): rows are ranked by length
    // (descending) inside windows of 256, the ranked rows form chunks of 32,
    // and entry k of the row in slot s sits at chunk_off[s / 32] + 32 k + s % 32.
    int* row_cnt;    // [n] off-diagonal entries of each row
    double* noise3;  // [3][npad] the step's thermal normals by row, drawn during the pair search
    int* cand_j;     // [kCandCap][npad] partners of each row as found by the pair search
    unsigned char* cand_img; // [kCandCap][npad] their image codes
    int* slot_row;   // [nslots] row of each slot (-1: padding slot)
    int* row_slot;   // [n]
    int* chunk_len32;// [nchunks] 32 x the longest row of each chunk
    int* chunk_off;  // [nchunks + 1]
    int* col;        // [nnz_cap] partner row (padding entries: the row itself)
    unsigned char* img; // [nnz_cap] image of the partner: (a+2) | (m+1) << 3 | (c+1) << 5
    double* val;     // [nnz_cap] pair weights w_ij (A_ij = -alpha w_ij); padding 0
    float* val32;    // [nnz_cap] FP32 copy for the mixed solver
    float* val32lo;  // [nnz_cap] mixed: val32 + val32lo is the weight as a double-float
    int* hcol;       // [nnz_cap] on-chip solve: each block's entries to other blocks' rows (mixed only)
    float* hval;     // [nnz_cap] their weights
    float* hlo;      // [nnz_cap] the low parts of those weights (double-float)
    float* rlo;      // [SMs][kResLoStride] on-chip solve: the local entries' weight low parts, per block
                     // in its shared-memory layout
    unsigned long long* res_hist; // [nslots] on-chip solve set-up: each row's local entries per bank
                                  // group of z (column mod 8), 8 bits each
    double* diag;    // [n] A_ii
    double* dinv;    // [n] 1 / A_ii
    float* diag32;   // [n]
    float* dinv32;   // [n]
    double* b;       // [3][npad]
    double* x;       // [3][npad] solution (velocities)
    double* r;       // [3][npad]
    double* p;       // [3][npad]
    double* q;       // [3][npad]
    double* z;       // [3][npad] D^-1 r (FP64 solver)
    double* s64;     // [6][npad] FP64 pipelined solve of small systems: s, and the second buffer of w
                     // (w in q and s64 + 3 npad in turn, z in z)
    uint4* posfix;   // [npad] mixed: positions in 32-bit fixed point of the box edges (x, y, z, 0), built
                     // before each matrix-free solve
    float4* r4;      // [npad] mixed solver vectors, (x, y, z, 0) per row
    float4* p4;
    float4* q4;
    float4* d4;      // correction accumulated since the last fold into x
    // mixed solver, double-float forms (hi + lo) for its true residuals b - A x
    float* diag32lo; // [npad] A_ii = diag32 + diag32lo
    float4* bdf;     // [2 npad] b of row i: hi at 2i, lo at 2i + 1, each (x, y, z, 0)
    float4* xdf;     // [2 npad] x the same way (one 32-byte record per row, one sector per gather)
    float4* rdf;     // [2 npad] the true residual b - A x the same way (initial residual; on-chip checks)
    double* xi_inj;  // [n][3] injected normals by id (or null)
    double* exp_tab; // [kExpTab] exp(-k / 256), computed on the host
    float2* exp_tab_df; // [kExpTab] the same as double-floats
    float4* rng_tab;    // [kRngTab] double-float tables of the mixed path's normals (computed on the host)
    double* partials;// [kMaxPartials * 8]
    float2* partials_df; // [kMaxPartials * 4] double-float partial sums (mixed solver)
    int* scan_tmp;   // block sums of the scans
    double* stage;   // [n][3] staging for host transfers
    DevState* st;
};

constexpr int kMaxPartials = 4096;
constexpr int kExpTab = 1024;
// Double-float tables of the mixed path's Box-Muller normals: ln c and 1 / c
// for c = j / 128, j = kLnTabBase + k; then (ln 2, 1 / 3); then cos and sin
// of 2 pi j / 64; then (2 pi, -1 / 6).  Entries (hi, lo, hi, lo).
constexpr int kLnTabBase = 90;
constexpr int kLnTab = 96;
constexpr int kTrigTab = 64;
constexpr int kRngConstLn = kLnTab;                 // (ln 2, 1 / 3)
constexpr int kRngTrig = kLnTab + 1;                // cos, sin of 2 pi j / 64
constexpr int kRngConstTrig = kRngTrig + kTrigTab;  // (2 pi, -1 / 6)
constexpr int kRngTab = kRngConstTrig + 1;
constexpr int kCandCap = 64;    // partners kept per row by the search (rows with more are searched again; the
                                 // clustered steady state of a sheared run has many rows above 32)
constexpr int kMaxSmIds = 1024;   // weight table: exp(-t) for t < 4 (pairs have t < ln 20)

// Learned warm start (mpnn.cu): flat FP32 weights W1 [6][64], W2 [64][64],
// W3 [64][4], o [11] (row-major, in that order).
constexpr int kMpOffW1 = 0;
constexpr int kMpOffW2 = 6 * 64;
constexpr int kMpOffW3 = kMpOffW2 + 64 * 64;
constexpr int kMpOffO = kMpOffW3 + 64 * 4;
constexpr int kMpParams = kMpOffO + 11;

struct MpBuffers {
    float4* x0;      // [3n] rows 3i + c: (b / A_ii, vprev, b, 0) / s
    float4* a0;      // [3n] M x0
    float4* y;       // [3n] MLP output (4 message features)
    float4* a1;      // [3n] M y
    float4* dy;      // [3n] training: dLoss / dy
    float4* g1;      // [3n] training: dLoss / da1
    float* master;   // [kMpParams] FP32 weights
    float* m;        // [kMpParams] Adam first moment
    float* v;        // [kMpParams] Adam second moment
    float* grad;     // [kMpParams]
    float* gpart;    // [blocks][kMpParams] per-block weight gradients
    double* dpart;   // [blocks][12] per-block loss and readout gradient
    __nv_bfloat16* wb;  // BF16 weight layouts for the tensor-core kernels
    double* scal;    // [0] = s (RMS of b), [1] = last loss
    double* part;    // [kMaxPartials] partial sums of the scale reduction
    unsigned int* ticket;
    // inference on another vector (the flexible solve's preconditioner): input
    // planes [3][npad] in place of b (NULL: b), output planes (NULL: x, the
    // start vector of CG), and the vprev feature set to 0
    const double* in;
    double* out;
    int zero_vprev;
};

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block (blockDim.x a multiple of 32, <= 1024); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh)
{
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (w == 0) v = warp_sum(v);
    return v;
}

// Publish this block's partial sums, then return true in exactly one block
// (the last one to arrive).  That block may then read every block's
// partials: no block ever waits for another.
template <int K>
__device__ __forceinline__ bool publish_partials(const double (&vals)[K], double* partials,
                                                 unsigned int* ticket)
{
    __shared__ double sh[32];
    __shared__ bool last;
    double tot[K];
#pragma unroll
    for (int k = 0; k < K; ++k) tot[k] = block_sum(vals[k], sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) partials[k * kMaxPartials + blockIdx.x] = tot[k];
        __threadfence();
        const unsigned int t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        if (threadIdx.x == 0) *ticket = 0u;
    }
    return last;
}

// In the last block: sum the K partial arrays in a fixed order (deterministic).
template <int K>
__device__ __forceinline__ void reduce_partials(const double* partials, double (&out)[K])
{
    __shared__ double sh[32];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double v = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x)
            v += __ldcg(partials + k * kMaxPartials + i);
        out[k] = block_sum(v, sh);
    }
}

// Lees-Edwards minimum image R_ij = R_i - R_j with every operation rounded
// exactly as written (no contraction), so the pair predicate is reproducible
// bit for bit on any IEEE machine.  n = round(y_ij / L_y) is the vertical image
// index of the boundary correction V_ij = kappa L_y n x (§Method).
__device__ __forceinline__ double min_image(const KParams& P, double delta, double xi, double yi,
                                            double zi, double xj, double yj, double zj,
                                            double& dx, double& dy, double& dz)
{
    dx = __dsub_rn(xi, xj);
    dy = __dsub_rn(yi, yj);
    dz = __dsub_rn(zi, zj);
    const double n = round(__ddiv_rn(dy, P.L[1]));
    dy = __dsub_rn(dy, __dmul_rn(n, P.L[1]));
    dx = __dsub_rn(dx, __dmul_rn(n, delta));
    dx = __dsub_rn(dx, __dmul_rn(P.L[0], round(__ddiv_rn(dx, P.L[0]))));
    dz = __dsub_rn(dz, __dmul_rn(P.L[2], round(__ddiv_rn(dz, P.L[2]))));
    return n;
}

__device__ __forceinline__ double sq_norm_exact(double dx, double dy, double dz)
{
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Loads of data that no thread writes during the kernel and that is read
// once per pass (matrix columns and values): non-coherent path, not
// allocated in L1, so L1 keeps the gathered vector rows.
__device__ __forceinline__ int ld_stream(const int* p)
{
    int v;
    asm("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_stream(const float* p)
{
    float v;
    asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ void philox4x64_10(unsigned long long c[4], unsigned long long k0,
                                              unsigned long long k1)
{
    const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const unsigned long long hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        const unsigned long long hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        const unsigned long long n0 = hi1 ^ c[1] ^ k0;
        const unsigned long long n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// Three N(0,1) draws for particle `id` at `step`: one Philox block (counter
// (id, step, 0, 0), key (seed, 0)), Box-Muller on 53-bit uniforms.
__device__ __forceinline__ void normals3(unsigned long long seed, unsigned long long step,
                                         unsigned long long id, double& g0, double& g1, double& g2)
{
    unsigned long long c[4] = {id, step, 0ull, 0ull};
    philox4x64_10(c, seed, 0ull);
    const double s53 = 1.0 / 9007199254740992.0;
    const double u1 = (double)((c[0] >> 11) + 1ull) * s53;
    const double u2 = (double)(c[1] >> 11) * s53;
    const double u3 = (double)((c[2] >> 11) + 1ull) * s53;
    const double u4 = (double)(c[3] >> 11) * s53;
    const double r1 = sqrt(-2.0 * log(u1));
    const double r2 = sqrt(-2.0 * log(u3));
    double s, co;
    sincospi(2.0 * u2, &s, &co);
    g0 = r1 * co;
    g1 = r1 * s;
    g2 = r2 * cospi(2.0 * u4);
}

__device__ __forceinline__ double wrap_box(double x, double L)
{
    x = x - L * floor(x / L);
    if (x >= L) x = x - L;
    if (x < 0.0) x = 0.0;
    return x;
}

__device__ __forceinline__ int cell_coord(double x, double inv_cw, int nc)
{
    int c = (int)floor(x * inv_cw);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

// Index of cell (cx, cy, cz) in the row order: the cells are grouped in
// tiles of 8 x 8 x 8 (tiles in x-fastest order, Morton order inside a tile),
// so any run of consecutive rows covers a compact region of space and the
// solver's gathers of neighbouring rows reuse cache lines.  Slots of cells
// outside the box stay empty.
__device__ __forceinline__ int spread3(int v)
{
    return (v & 1) | ((v & 2) << 2) | ((v & 4) << 4);
}

__device__ __forceinline__ int cell_index(const KParams& P, int cx, int cy, int cz)
{
    const int t = ((cz >> 3) * P.ntile[1] + (cy >> 3)) * P.ntile[0] + (cx >> 3);
    return (t << 9) | spread3(cx & 7) | (spread3(cy & 7) << 1) | (spread3(cz & 7) << 2);
}

// Image code of a pair: the partner's image sits at R_j + a L_x x + m (L_y y + delta x) + c L_z z.
__device__ __forceinline__ unsigned char image_code(int a, int m, int c)
{
    return (unsigned char)((a + 2) | ((m + 1) << 3) | ((c + 1) << 5));
}

// Exact separation R_i - (image of R_j) for a pair whose image indices are
// known: the canonical minimum-image operations of min_image() with n = m
// and the two rounded quotients replaced by a and c (equal for any pair
// within r_c), so the result is bit-identical and needs no division.
__device__ __forceinline__ double image_separation(const KParams& P, double delta, double xi, double yi,
                                                   double zi, double xj, double yj, double zj,
                                                   unsigned char code, double& dx, double& dy,
                                                   double& dz)
{
    const double a = (double)((int)(code & 7) - 2);
    const double n = (double)((int)((code >> 3) & 3) - 1);
    const double c = (double)((int)((code >> 5) & 3) - 1);
    dx = __dsub_rn(__dsub_rn(__dsub_rn(xi, xj), __dmul_rn(n, delta)), __dmul_rn(P.L[0], a));
    dy = __dsub_rn(__dsub_rn(yi, yj), __dmul_rn(n, P.L[1]));
    dz = __dsub_rn(__dsub_rn(zi, zj), __dmul_rn(P.L[2], c));
    return n;
}

// Double-float accumulation (Knuth's TwoSum): a sum kept as an unevaluated
// pair hi + lo of FP32 numbers, about 44 significant bits, using only the FP32
// pipes (GB300 issues FP64 at a small fraction of the FP32 rate).
struct dfloat {
    float hi, lo;
};

__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    const float t = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float hi = __fadd_rn(s, t);
    return dfloat{hi, __fsub_rn(t, __fsub_rn(hi, s))};
}

__device__ __forceinline__ dfloat df_add(dfloat a, float x) { return df_add(a, dfloat{x, 0.f}); }

// Error-free building blocks (Knuth's TwoSum, Dekker's FastTwoSum, and the
// product error by one fused multiply-add), explicit round-to-nearest
// intrinsics so that no contraction changes them.
__device__ __forceinline__ dfloat two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return dfloat{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ dfloat fast_two_sum(float a, float b)   // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return dfloat{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ dfloat df_sqr(dfloat a)
{
    const float p = __fmul_rn(a.hi, a.hi);
    const float e = fmaf(__fmul_rn(2.f, a.hi), a.lo, fmaf(a.hi, a.hi, -p));
    return fast_two_sum(p, e);
}

__device__ __forceinline__ dfloat df_neg(dfloat a) { return dfloat{-a.hi, -a.lo}; }

__device__ __forceinline__ double df_to_double(dfloat a) { return (double)a.hi + (double)a.lo; }

// The double-float nearest a double: hi = fp32(x), lo = fp32(x - hi).
__device__ __forceinline__ dfloat df_split(double x)
{
    const float hi = __double2float_rn(x);
    return dfloat{hi, __double2float_rn(x - (double)hi)};
}

// ---- the same normals in double-float arithmetic on the FP32 pipes (the
// mixed path): each step below is within a few units of 2^-47 of its FP64
// counterpart, so the normals agree with the FP64 ones to ~1e-13.

// u = m 2^-53 (m < 2^53 an integer) as a double-float.
__device__ __forceinline__ dfloat df_u53(unsigned long long m)
{
    const float h = __ull2float_rn(m);
    const long long rem = (long long)m - (long long)(unsigned long long)h;   // exact, |rem| < 2^29
    const float s = 1.1102230246251565e-16f;                                  // 2^-53 (exact)
    return dfloat{h * s, __ll2float_rn(rem) * s};
}

// ln u for u = k 2^-53 in (0, 1] (k the integer): u = 2^e m with m in
// [sqrt(1/2), sqrt(2)), c = j / 128 the table point nearest m, t = (m - c) / c
// (|t| < 0.0056), ln u = e ln 2 + ln c + ln(1 + t) with the series of
// ln(1 + t): t, t^2 and t^3 terms in double-float, the rest (t^4 .. t^7) in
// FP32.  Next to u = 1 (c = 1), where ln u is as small as 1 - u, t = -(2^53 -
// k) 2^-53 is taken exactly from the integer, so ln u keeps its relative
// accuracy.
__device__ __forceinline__ dfloat df_log_unit(dfloat u, unsigned long long k53, const float4* __restrict__ tab)
{
    int e;
    float mh = frexpf(u.hi, &e);
    if (mh < 0.70710678f) {
        mh *= 2.f;
        e -= 1;
    }
    const float ml = ldexpf(u.lo, -e);   // exact
    const int j = __float2int_rn(mh * 128.f);
    const float4 lc = __ldg(tab + (j - kLnTabBase));
    const float4 k = __ldg(tab + kRngConstLn);
    dfloat t;
    if (e == 0 && j == 128) {   // u in [1 - 1/256, 1]: 2^53 - k < 2^45, exact as a double-float
        const long long v = (1ll << 53) - (long long)k53;
        const float vh = __ll2float_rn(v);
        const float s = 1.1102230246251565e-16f;   // 2^-53
        t = dfloat{-vh * s, -__ll2float_rn(v - (long long)vh) * s};
    } else {
        const dfloat mc = two_sum(__fsub_rn(mh, (float)j * 0.0078125f), ml);   // m - c (the difference is exact)
        t = df_mul(mc, dfloat{lc.z, lc.w});
    }
    const dfloat t2 = df_sqr(t);
    const dfloat t3 = df_mul(t2, t);
    const float th = t.hi;
    const float tail = __fmul_rn(__fmul_rn(t2.hi, t2.hi),
                                 fmaf(th, fmaf(th, fmaf(th, 1.f / 7.f, -1.f / 6.f), 0.2f), -0.25f));
    dfloat s = df_add(t, dfloat{-0.5f * t2.hi, -0.5f * t2.lo});
    s = df_add(s, df_mul(t3, dfloat{k.z, k.w}));
    s = df_add(s, dfloat{tail, 0.f});
    s = df_add(s, dfloat{lc.x, lc.y});
    return df_add(s, df_mul(dfloat{(float)e, 0.f}, dfloat{k.x, k.y}));
}

// sqrt(x), x >= 0: one Newton step from the FP32 root (the square of the
// FP32 root exact by one fused multiply-add).
__device__ __forceinline__ dfloat df_sqrt(dfloat x)
{
    if (!(x.hi > 0.f)) return dfloat{0.f, 0.f};
    const float y = sqrtf(x.hi);
    const float p = __fmul_rn(y, y), pe = fmaf(y, y, -p);
    const float r = __fadd_rn(__fsub_rn(x.hi, p), __fsub_rn(x.lo, pe));
    return fast_two_sum(y, __fdiv_rn(r, __fmul_rn(2.f, y)));
}

// cos(2 pi u), sin(2 pi u) for u in [0, 1]: u = j / 64 + r (|r| <= 1/128),
// theta = 2 pi r, the two series to theta^7 and theta^6 (leading terms in
// double-float), combined with the table's cos and sin of 2 pi j / 64.
__device__ __forceinline__ void df_sincos2pi(dfloat u, const float4* __restrict__ tab, dfloat& sn, dfloat& cs)
{
    const int j = __float2int_rn(u.hi * 64.f);
    const dfloat r = two_sum(__fsub_rn(u.hi, (float)j * 0.015625f), u.lo);   // the difference is exact
    const float4 k = __ldg(tab + kRngConstTrig);
    const dfloat th = df_mul(r, dfloat{k.x, k.y});
    const dfloat t2 = df_sqr(th);
    dfloat s = df_add(th, df_mul(df_mul(t2, th), dfloat{k.z, k.w}));
    s = df_add(s, dfloat{__fmul_rn(__fmul_rn(th.hi, __fmul_rn(t2.hi, t2.hi)), fmaf(t2.hi, -1.f / 5040.f, 1.f / 120.f)),
                         0.f});
    dfloat c = df_add(dfloat{1.f, 0.f}, dfloat{-0.5f * t2.hi, -0.5f * t2.lo});
    c = df_add(c, dfloat{__fmul_rn(__fmul_rn(t2.hi, t2.hi), fmaf(t2.hi, -1.f / 720.f, 1.f / 24.f)), 0.f});
    const float4 a = __ldg(tab + kRngTrig + (j & (kTrigTab - 1)));
    const dfloat ca{a.x, a.y}, sa{a.z, a.w};
    cs = df_add(df_mul(ca, c), df_neg(df_mul(sa, s)));
    sn = df_add(df_mul(sa, c), df_mul(ca, s));
}

// normals3 in double-float: the same Philox block and Box-Muller formulas.
__device__ __forceinline__ void normals3_df(const float4* __restrict__ tab, unsigned long long seed,
                                            unsigned long long step, unsigned long long id, dfloat& g0, dfloat& g1,
                                            dfloat& g2)
{
    unsigned long long c[4] = {id, step, 0ull, 0ull};
    philox4x64_10(c, seed, 0ull);
    const unsigned long long k1 = (c[0] >> 11) + 1ull, k3 = (c[2] >> 11) + 1ull;
    const dfloat l1 = df_log_unit(df_u53(k1), k1, tab);
    const dfloat l3 = df_log_unit(df_u53(k3), k3, tab);
    const dfloat r1 = df_sqrt(dfloat{-2.f * l1.hi, -2.f * l1.lo});
    const dfloat r2 = df_sqrt(dfloat{-2.f * l3.hi, -2.f * l3.lo});
    dfloat s, co, s4, c4;
    df_sincos2pi(df_u53(c[1] >> 11), tab, s, co);
    df_sincos2pi(df_u53(c[3] >> 11), tab, s4, c4);
    g0 = df_mul(r1, co);
    g1 = df_mul(r1, s);
    g2 = df_mul(r2, c4);
}


// s_c = sum_j w_ij x_c[j] in double-float over the entries [e0, e1) (stride
// 32) of one slot of the sliced layout: weights val32 + val32lo, x as the
// double-float records of xdf.  KB entries are requested at a time.
template <int KB>
__device__ __forceinline__ void row_sum_df(const int* __restrict__ col, const float* __restrict__ wh,
                                           const float* __restrict__ wl, const float4* xdf,
                                           int e0, int e1, dfloat (&s)[3])
{
    s[0] = s[1] = s[2] = dfloat{0.f, 0.f};
    for (int eb = e0; eb < e1; eb += 32 * KB) {
        int j[KB];
        float h[KB], l[KB];
#pragma unroll
        for (int u = 0; u < KB; ++u) {
            const int e = eb + 32 * u;
            j[u] = 0;
            h[u] = l[u] = 0.f;
            if (e < e1) {
                j[u] = ld_stream(col + e);
                h[u] = ld_stream(wh + e);
                l[u] = ld_stream(wl + e);
            }
        }
        float4 xh[KB], xl[KB];
#pragma unroll
        for (int u = 0; u < KB; ++u) {
            xh[u] = xl[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (h[u] != 0.f) {
                xh[u] = xdf[2 * j[u]];
                xl[u] = xdf[2 * j[u] + 1];
            }
        }
#pragma unroll
        for (int u = 0; u < KB; ++u) {
            const dfloat w{h[u], l[u]};
            s[0] = df_add(s[0], df_mul(w, dfloat{xh[u].x, xl[u].x}));
            s[1] = df_add(s[1], df_mul(w, dfloat{xh[u].y, xl[u].y}));
            s[2] = df_add(s[2], df_mul(w, dfloat{xh[u].z, xl[u].z}));
        }
    }
}

// r = b - (A_ii x - alpha s) of one row in double-float, from the row's sum s
// of row_sum_df (Eq. algebra: A = I + alpha L_w with L_w's off-diagonal -w_ij).
__device__ __forceinline__ void residual_df(const KParams& P, const DevBuffers& B, int row, const dfloat (&s)[3],
                                            dfloat (&r)[3])
{
    const dfloat d{B.diag32[row], B.diag32lo[row]}, al{P.alpha_hi, P.alpha_lo};
    const float4 xh = B.xdf[2 * row], xl = B.xdf[2 * row + 1], bh = B.bdf[2 * row], bl = B.bdf[2 * row + 1];
    const dfloat x[3] = {{xh.x, xl.x}, {xh.y, xl.y}, {xh.z, xl.z}};
    const dfloat b[3] = {{bh.x, bl.x}, {bh.y, bl.y}, {bh.z, bl.z}};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const dfloat t = df_add(df_mul(d, x[c]), df_neg(df_mul(al, s[c])));
        r[c] = df_add(b[c], df_neg(t));
    }
}

__device__ __forceinline__ dfloat warp_sum_df(dfloat v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dfloat w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = df_add(v, w);
    }
    return v;
}

// Block sum of double-float values; valid in thread 0.
__device__ __forceinline__ dfloat block_sum_df(dfloat v, float2* sh)
{
    v = warp_sum_df(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = make_float2(v.hi, v.lo);
    __syncthreads();
    const int nw = blockDim.x >> 5;
    dfloat t{0.f, 0.f};
    if (threadIdx.x < nw) t = dfloat{sh[threadIdx.x].x, sh[threadIdx.x].y};
    if (w == 0) t = warp_sum_df(t);
    return t;
}

// Double-float counterpart of publish_partials / reduce_partials: every block
// publishes its sums, and the last block to arrive returns the totals (as
// doubles, in thread 0) after summing the partials in a fixed order.
template <int K>
__device__ __forceinline__ bool publish_reduce_df(dfloat (&vals)[K], float2* partials, unsigned int* ticket,
                                                  double (&out)[K])
{
    __shared__ float2 sh[32];
    __shared__ bool last;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const dfloat t = block_sum_df(vals[k], sh);
        if (threadIdx.x == 0) partials[k * kMaxPartials + blockIdx.x] = make_float2(t.hi, t.lo);
    }
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        dfloat v{0.f, 0.f};
        for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
            const float2 p = __ldcg(partials + k * kMaxPartials + i);
            v = df_add(v, dfloat{p.x, p.y});
        }
        const dfloat t = block_sum_df(v, sh);
        out[k] = (double)t.hi + (double)t.lo;
    }
    if (threadIdx.x == 0) *ticket = 0u;
    return true;
}

// ------------------------------------------------------------------ launchers

inline int grid_for(long long work, int per_block, int max_blocks)
{
    long long g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (int)g;
}

struct Launch {
    cudaStream_t stream;
    int num_sms;
};

// neighbors.cu
void launch_bin(const KParams& P, DevBuffers& B, Launch L);
// mode 0: plain scan; mode 2: the total is the matrix size with padding
// (st->nnz_slots), and exceeding cap_check raises the overflow flag.  Both
// return the kernels they launched.
int launch_scan(const int* in, int* out, int n, int* block_tmp, long long cap_check, DevState* st, int mode,
                Launch L);
void launch_sell_plan(const KParams& P, DevBuffers& B, Launch L);
int launch_scatter_sort_gather(const KParams& P, DevBuffers& B, bool warm, Launch L);
void launch_identity_gather(const KParams& P, DevBuffers& B, bool warm, Launch L);
// The step's pair search; with draw_noise it also draws the thermal normals
// of every row (FP64 Box-Muller, overlapping the search's memory latency).
// side/ev (optional): the normals run on side between ev[0] and ev[1], beside
// the search, and L.stream waits for them; returns the kernels launched
int launch_nbr_count(const KParams& P, DevBuffers& B, bool draw_noise, Launch L, cudaStream_t side = nullptr,
                     cudaEvent_t* ev = nullptr);
// Pair fill (columns and image codes), followed, with assemble, by the FP64
// assembly of the matrix and right-hand side; returns the kernels launched.
int launch_nbr_fill(const KParams& P, DevBuffers& B, bool assemble, bool use_inj, bool df, Launch L);
void launch_assemble_only(const KParams& P, DevBuffers& B, bool use_inj, bool df, Launch L);
// Fills the weight tables exp_tab and exp_tab_df (host computation, one copy each).
cudaError_t upload_exp_table(double* exp_tab, float2* exp_tab_df, cudaStream_t stream);
cudaError_t upload_rng_table(float4* rng_tab, cudaStream_t stream);
void launch_normals(const float4* tab, unsigned long long seed, unsigned long long step, long long count,
                    const long long* ids, double* out, int df, cudaStream_t s);
void launch_uniform_positions(const KParams& P, DevBuffers& B, Launch L);
void launch_philox_blocks(unsigned long long seed, unsigned long long step, long long count,
                          const long long* ids, unsigned long long* out, cudaStream_t s);

// cg.cu
struct CgLaunch {
    int use_cond;                       // call cudaGraphSetConditional (inside a graph)
    unsigned long long h_loop, h_check; // cudaGraphConditionalHandle values
};
// One CG iteration is two kernels: spmv (q = A z + beta q, p = z + beta p, p.q)
// and update (x or d += alpha p, r -= alpha q, r.r, r.z).  The true-residual
// check is one kernel (FP64) or two (mixed: fold d into x, then FP64 residual).
int launch_cg_init(const KParams& P, DevBuffers& B, bool from_x, bool mixed, Launch L);
// probe = 1: time the kernel on the current system without touching the solver state
void launch_cg_spmv(const KParams& P, DevBuffers& B, bool mixed, Launch L, int probe = 0);
void launch_cg_update(const KParams& P, DevBuffers& B, bool mixed, const CgLaunch& C, Launch L,
                      int probe = 0);
void launch_cg_true_residual(const KParams& P, DevBuffers& B, bool mixed, bool always_check,
                             const CgLaunch& C, Launch L);
void launch_cg_finish(const KParams& P, DevBuffers& B, bool mixed, Launch L);
int cg_kernels_per_iteration(bool mixed);
void cg_prepare();   // resident-block counts of the solver kernels (once per process)
// cg_persistent.cu: the whole mixed solve (after launch_cg_init) in one cooperative launch
// (preceded, for a matrix-free configuration, by the fixed-point positions'
// kernel: cg_persistent_prelaunches kernels before the solve)
cudaError_t launch_cg32_persistent(const KParams& P, DevBuffers& B, Launch L);
int cg_persistent_prelaunches(const KParams& P, const DevBuffers& B, Launch L);
// The FP64 solver as one cooperative launch (r = b - A x0 with from_x, else x = 0).
cudaError_t launch_cg64_persistent(const KParams& P, DevBuffers& B, int from_x, Launch L);
int cg64_persistent_grid(const KParams& P, Launch L);
// Whether the persistent solve of this system runs on chip (and so can form
// its initial residual itself: launch it with fused_init set and without
// launch_cg_init, after launch_cg_split_x where it starts from x).
bool cg_persistent_on_chip(const KParams& P, const DevBuffers& B, Launch L);
void launch_cg_split_x(const KParams& P, DevBuffers& B, Launch L);
int cg_persistent_grid(const KParams& P, const DevBuffers& B, Launch L);
// Tile configuration k of the persistent solver: gathers in flight, blocks per
// SM, next batch requested during the current gathers (1) or not (0), threads
// per block (256 G: G windows at a time), on-chip solve (1) or not (0),
// weights recomputed from positions in the iteration (1) or read (0).
void cg_persistent_config(int k, int* gathers, int* blocks_per_sm, int* pipelined, int* block_threads,
                          int* resident, int* matrix_free);
// Whether configuration k can solve this system (the on-chip solve needs at
// most 2048 rows per block and its halo lists).
bool cg_persistent_usable(int k, const KParams& P, const DevBuffers& B, Launch L);
// A batch of systems in one cooperative launch: blocks [blk_off[k], blk_off[k+1]) solve system k.
constexpr int kBatchConfigs = 6;   // tile configurations of the batched solver (sp_batch_autotune)
int cg_persistent_batch_capacity(Launch L, int cfg);
void cg_batch_config(int k, int* gathers, int* blocks_per_sm, int* block_threads);
cudaError_t launch_cg32_persistent_batch(const KParams* Ps_dev, const DevBuffers* Bs_dev, const int* blk_off_dev,
                                         int R, int total_blocks, int cfg, Launch L);
int cg_kernels_per_check(bool mixed);

// fcg.cu: flexible CG (FCG(1)) in FP64 whose preconditioner is the network
// (every net_every iterations, net != NULL) or Jacobi; x holds the start
// vector; the state's status, iterations and true residual on return.
struct FcgState {
    double bb, rr, pq, alpha, beta, last_res;
    int iter, done, status;
    unsigned int ticket;
};
int fcg_solve(const KParams& P, DevBuffers& B, const MpBuffers* net, int net_every, FcgState* S, FcgState* S_host,
              Launch L, long long* launches);

// mpnn.cu
void launch_mp_infer(const KParams& P, DevBuffers& B, MpBuffers& M, Launch L);
int mp_infer_launches();
// The network applied to the planes `in` ([3][npad], in place of b, with the
// vprev feature 0), its output written to `out` (the flexible solve's
// preconditioner; same 5 kernels as the warm start).
void launch_mp_apply(const KParams& P, DevBuffers& B, const MpBuffers& M, const double* in, double* out, Launch L);
void launch_mp_train(const KParams& P, DevBuffers& B, MpBuffers& M, float lr, int t, Launch L);
int mp_prepare();
int mp_weights_bf16_count();
void launch_mp_convert(MpBuffers& M, cudaStream_t s);

// integrate.cu
// commit = false: the new offset stays in delta_next until launch_commit_step
// (so that a stress kernel running beside the update still reads the step's offset)
void launch_integrate(const KParams& P, DevBuffers& B, Launch L, bool commit = true);
void launch_commit_step(DevBuffers& B, Launch L);
void launch_stress(const KParams& P, DevBuffers& B, bool mixed, Launch L);
void launch_scatter_by_id(const double* planes, int npad, const int* ids, int n, double* out_n3,
                          cudaStream_t s);
void launch_gather_by_id(const double* in_n3, const int* ids, int n, int npad, double* planes,
                         cudaStream_t s);
// The same for positions given by a caller: a coordinate that is not finite or
// lies outside [0, L_a) sets st->error to SP_ERR_INVALID_ARG (the steps that
// follow then do nothing and report it).
void launch_gather_positions(const double* in_n3, const int* ids, int n, int npad, double* planes,
                             const KParams& P, DevState* st, cudaStream_t s);
void launch_reset_step_stats(DevState* st, cudaStream_t s);
// Architecture of the device code the current device runs (cudaFuncGetAttributes
// of one of this library's kernels): 10 major + minor, e.g. 103 for sm_103.
cudaError_t device_code_version(int* binary_version, int* ptx_version);
// sfactor.cu: S(q) at q_z = 0 for kx in [-nkx, nkx], ky in [-nky, nky] (kx slowest);
// G = 0: direct sum over particles; G > 0: CIC grid of G x G in the sheared frame.
cudaError_t run_structure_factor(const KParams& P, const DevBuffers& B, double delta, int G, int nkx, int nky,
                                 const double* twiddle_dev, unsigned long long* grid_dev, double2* A_dev,
                                 double* S_dev, double* qx_dev, double* qy_dev, cudaStream_t s);

// fdt.cu: xi = p(A) g ~ A^(1/2) g (Chebyshev interpolant of sqrt on [1, lambda_max])
cudaError_t cheb_bound(const KParams& P, DevBuffers& B, unsigned long long* out_dev, cudaStream_t s);
// Work arrays of xi = p(A) g: v[0] holds g, v[1..3] the rotating T_k, v[4] xi;
// each 3 npad doubles (FP64 path) or 2 npad float4 records (mixed path).
struct FdtBuffers {
    void* v[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    double* cs = nullptr;            // [2 + 4097] interval map and coefficients
    float2* csf = nullptr;           // the same as double-floats
    unsigned long long* bound = nullptr;
};
constexpr int kFdtMaxDegree = 4096;
// xi = p(A) g with g already in V.v[0]; returns the kernels launched
int enqueue_cheb(const KParams& P, DevBuffers& B, FdtBuffers& V, int degree, cudaStream_t s);
// the step's right-hand side with A^(1/2)-correlated noise: g from the assembly's
// normals into V.v[0], xi = p(A) g, b += (amp / zeta) (xi - g); returns the kernels launched
int enqueue_fdt_noise(const KParams& P, DevBuffers& B, FdtBuffers& V, int degree, bool use_inj, cudaStream_t s);
// cs: [0] 2 / (b - a), [1] (b + a) / (b - a), [2 + k] c_k (k <= degree); csf: the same as double-floats
cudaError_t cheb_coeffs(const unsigned long long* bound, int degree, double* cs, float2* csf, cudaStream_t s);
cudaError_t cheb_step(const KParams& P, DevBuffers& B, const double* tc, const double* tp, double* tn, double* y,
                      const double* cs, int k, cudaStream_t s);
cudaError_t cheb_step_df(const KParams& P, DevBuffers& B, const float4* tc, const float4* tp, float4* tn, float4* y,
                         const float2* csf, int k, cudaStream_t s);
cudaError_t cheb_split(const KParams& P, const double* g, float4* t, cudaStream_t s);
cudaError_t cheb_join(const KParams& P, const float4* y, double* out, cudaStream_t s);

// vcorr.cu: velocity cross-correlation versus distance (Fig. vv)
constexpr int kVcMaxBins = 1024;
struct VcBuffers {
    double* pos_n3 = nullptr;   // [n][3] positions (particle order of the caller)
    double* v_n3 = nullptr;     // [n][3] velocities
    float4* p4 = nullptr;       // [n] FP32 positions
    float4* u4 = nullptr;       // [n] FP32 velocities relative to the imposed flow
    unsigned long long* sum = nullptr;   // [kVcMaxBins] fixed-point sums of the products
    unsigned long long* cnt = nullptr;   // [kVcMaxBins] pair counts
    int2* band = nullptr;       // [band_cap] pairs decided in FP64
    unsigned int* misc = nullptr;        // [4] listed pairs, bits of max |u|^2, position flag
    double* part = nullptr;     // per-block sums of |u|^2
    double* scal = nullptr;     // [2] <|u|^2>, fixed-point scale
    int2* tiles = nullptr;      // (I, first J) of every block
    long long n_cap = 0, band_cap = 0, tiles_cap = 0, tiles_n = 0, tiles_for = 0;
    cudaEvent_t ev[2] = {nullptr, nullptr};
};
struct VcStats {
    double pairs_ms;            // the all-pairs kernel (CUDA events on the caller's stream)
    long long band_pairs;       // pairs decided in FP64
    long long blocks;           // blocks of the all-pairs kernel
};
void vc_free(VcBuffers& V);
cudaError_t vc_reserve(VcBuffers& V, long long n);
// Inputs in V.pos_n3 / V.v_n3 (n rows, positions in [0, L)); results to the host.
int run_velocity_correlation(VcBuffers& V, long long n, const double L[3], double delta, double kappa, int nbins,
                             double rmax, cudaStream_t s, double* sum_host, long long* cnt_host, double* vsq_host,
                             VcStats* stats, const char** err);

}  // namespace ss
