// Velocity cross-correlation versus distance (arXiv 1808.06381, §Results,
// Fig. vv): the average inter-chain velocity product <v_c . v_c'> / <v_c^2>
// as a function of the inter-chain distance |R_cc'|.
//
// u_c = v_c - kappa (y_c - L_y/2) x is the velocity relative to the imposed
// flow (the Lees-Edwards image of c' moves with v_c' + kappa L_y n x and so
// carries the same u).  Every pair c < c' whose minimum-image distance r is
// below rmax adds u_c . u_c' to bin floor(r nbins / rmax) and counts there.
//
// All pairs are visited (n^2 / 2): one block per 512 particles c (two per
// thread) and a run of 256-particle tiles of c' staged in shared memory, every
// pair in FP32.  The
// decisions that make the result exact are taken in FP64 where FP32 could get
// them wrong: a pair whose FP32 image index, bin or cut-off test lies within
// the FP32 error bound of a boundary is appended to a list, and a second
// kernel decides those pairs with the FP64 operations of the definition, so
// the counts are exact.  The products go into per-warp shared-memory
// histograms as 2^-20-scaled fixed-point integers (scale from the largest
// |u|^2), so the sums do not depend on the order of the additions.
#include <math.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace ss {

namespace {

constexpr int kVcTile = 256;               // particles per tile; threads per block
constexpr int kVcWarps = kVcTile / 32;
constexpr int kVcPrepBlocks = 1024;        // vsq partial sums

// rint(x) for |x| < 2^22 by the 1.5 2^23 shift (two FP32 additions instead of
// a rounding instruction); ties go to even like rintf
__device__ __forceinline__ float rint_shift(float x)
{
    return __fsub_rn(__fadd_rn(x, 12582912.f), 12582912.f);
}

struct VcConst {
    int n, nbins, ntile, chunk;
    float Lf[3], iLf[3], df;   // box edges, their inverses, delta (FP32)
    float r2_hi;               // FP32 |R|^2 >= r2_hi: certainly |R| >= rmax
    float r_band;              // FP32 |R| > r_band: decided in FP64
    float inv_f;               // nbins / rmax
    float eb;                  // FP32 bin position within eb of an edge: decided in FP64
    float half[3];             // |component| > half[a] (L_a/2 less the FP32 error): image decided in FP64
    double delta, kappa, rmax2, inv;
    double invL[3];            // 1 / L_a (FP64)
};

// FP32 copies of the positions and of u; FP64 sums of |u|^2 per block and the
// largest FP32 |u|^2 (its bits, non-negative floats order like integers).
__global__ void __launch_bounds__(kVcTile) k_vc_prep(VcConst C, KParams P, const double* __restrict__ pos,
                                                       const double* __restrict__ v, float4* __restrict__ p4,
                                                       float4* __restrict__ u4, double* __restrict__ part,
                                                       unsigned int* __restrict__ umax, int* __restrict__ flag)
{
    __shared__ double ssum[kVcWarps];
    __shared__ float smax[kVcWarps];
    double s = 0.0;
    float m = 0.f;
    for (int i = blockIdx.x * kVcTile + threadIdx.x; i < C.n; i += gridDim.x * kVcTile) {
        const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
        if (!(x >= 0.0 && x < P.L[0] && y >= 0.0 && y < P.L[1] && z >= 0.0 && z < P.L[2])) atomicOr(flag, 1);
        const double ux = v[3 * i] - C.kappa * (y - 0.5 * P.L[1]), uy = v[3 * i + 1], uz = v[3 * i + 2];
        s += ux * ux + uy * uy + uz * uz;
        const float4 uf = make_float4((float)ux, (float)uy, (float)uz, 0.f);
        p4[i] = make_float4((float)x, (float)y, (float)z, 0.f);
        u4[i] = uf;
        m = fmaxf(m, uf.x * uf.x + uf.y * uf.y + uf.z * uf.z);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    s = warp_sum(s);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
        ssum[warp] = s;
        smax[warp] = m;
    }
    __syncthreads();
    if (warp == 0) {
        s = lane < kVcWarps ? ssum[lane] : 0.0;
        m = lane < kVcWarps ? smax[lane] : 0.f;
        s = warp_sum(s);
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) {
            part[blockIdx.x] = s;
            atomicMax(umax, __float_as_uint(m));
        }
    }
}

// vsq = (1/n) sum |u|^2 (partials summed in a fixed order) and the
// fixed-point scale S = 2^(20 - e) with max |u_f|^2 < 2^e, so that every FP32
// product times S stays below 2^21 in magnitude.
__global__ void k_vc_scale(int n, int nparts, const double* __restrict__ part, const unsigned int* __restrict__ umax,
                           double* __restrict__ scal)
{
    double s = 0.0;
    for (int k = threadIdx.x; k < nparts; k += 32) s += part[k];
    s = warp_sum(s);
    if (threadIdx.x == 0) {
        scal[0] = s / (double)n;
        const float m = __uint_as_float(*umax);
        int e = 0;
        if (m > 0.f) frexp((double)m, &e);
        scal[1] = ldexp(1.0, 20 - e);
    }
}

// One pair (i, j), i < j: the FP32 minimum image and distance; the pair goes
// to the per-warp histogram, or to the FP64 list when one of its decisions
// lies within the FP32 error bound of a boundary.
__device__ __forceinline__ void vc_pair(const VcConst& C, float4 pi, float4 ui, int i, float4 pj,
                                        const float4* su, int jj, int j, float S, unsigned long long* hsw,
                                        int2* band, unsigned int* band_n, unsigned int band_cap)
{
    float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
    const float ny = rint_shift(dy * C.iLf[1]);
    dy = fmaf(-ny, C.Lf[1], dy);
    dx = fmaf(-ny, C.df, dx);
    dx = fmaf(-rint_shift(dx * C.iLf[0]), C.Lf[0], dx);
    dz = fmaf(-rint_shift(dz * C.iLf[2]), C.Lf[2], dz);
    // an image index taken within the FP32 error of a tie leaves that
    // component within the same error of half the box edge
    const bool tie = fabsf(dx) > C.half[0] || fabsf(dy) > C.half[1] || fabsf(dz) > C.half[2];
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (!(j > i)) return;
    bool push = tie;
    if (!tie && r2 < C.r2_hi) {
        // |R| from the reciprocal square root (within 3 ulp; the bands allow for it)
        const float r = r2 * rsqrtf(fmaxf(r2, 1e-30f));
        const float t = r * C.inv_f;
        const float tk = __fadd_rd(t, 8388608.f);   // 2^23 + floor(t) (0 <= t < 2^23)
        const float fr = t - (tk - 8388608.f);      // exact
        if (r > C.r_band || fr < C.eb || fr > 1.f - C.eb) {
            push = true;
        } else {
            const int k = __float_as_int(tk) - 0x4B000000;
            const float4 uj = su[jj];
            const float dot = fmaf(ui.x, uj.x, fmaf(ui.y, uj.y, ui.z * uj.z));
            // round(dot S) by the 1.5 2^23 shift (|dot S| < 2^21)
            const int q = __float_as_int(fmaf(dot, S, 12582912.f)) - 0x4B400000;
            atomicAdd(hsw + k, (1ull << 40) + (unsigned long long)(long long)q);
        }
    }
    if (push) {   // rare (a few per thousand pairs)
        const unsigned int idx = atomicAdd(band_n, 1u);
        if (idx < band_cap) band[idx] = make_int2(i, j);
    }
}

// Block (I, J0): particles i = 512 I + tid and 512 I + 256 + tid against the
// c' tiles J0 .. J0 + chunk - 1 (256 particles each).
__global__ void __launch_bounds__(kVcTile) k_vc_pairs(VcConst C, const float4* __restrict__ p4,
                                                        const float4* __restrict__ u4, const int2* __restrict__ tiles,
                                                        const double* __restrict__ scal,
                                                        unsigned long long* __restrict__ gsum,
                                                        unsigned long long* __restrict__ gcnt,
                                                        int2* __restrict__ band, unsigned int* __restrict__ band_n,
                                                        unsigned int band_cap)
{
    extern __shared__ float4 vc_smem[];
    float4* sp = vc_smem;                  // [kVcTile] positions of the c' tile
    float4* su = sp + kVcTile;             // [kVcTile] their u
    // per-warp histograms, one 64-bit word per bin: count 2^40 + fixed-point sum
    // (a warp adds at most 32 x 2 x 16 x 256 = 2^18 pairs to a bin, so the count
    // fits the top 24 bits and the sum, below 2^18 (2^20 + 1) in magnitude, the
    // low 40 bits in two's complement)
    unsigned long long* hs = reinterpret_cast<unsigned long long*>(su + kVcTile);   // [warps][nbins]
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int k = tid; k < kVcWarps * C.nbins; k += kVcTile) hs[k] = 0ull;
    const int2 tb = tiles[blockIdx.x];
    const int I = tb.x, J0 = tb.y, J1 = min(C.ntile - 1, J0 + C.chunk - 1);
    const int i0 = I * 2 * kVcTile + tid, i1 = i0 + kVcTile;
    // a particle past n pairs with no j (index n + 2^30 is above every j)
    const int e0 = i0 < C.n ? i0 : (1 << 30), e1 = i1 < C.n ? i1 : (1 << 30);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 pi0 = i0 < C.n ? p4[i0] : z4, ui0 = i0 < C.n ? u4[i0] : z4;
    const float4 pi1 = i1 < C.n ? p4[i1] : z4, ui1 = i1 < C.n ? u4[i1] : z4;
    const float S = (float)scal[1];
    unsigned long long* hsw = hs + warp * C.nbins;
    for (int J = J0; J <= J1; ++J) {
        __syncthreads();   // the histograms are zeroed; the previous tile is no longer read
        const int jt = J * kVcTile + tid;
        if (jt < C.n) {
            sp[tid] = p4[jt];
            su[tid] = u4[jt];
        }
        __syncthreads();
        const int jn = min(kVcTile, C.n - J * kVcTile);
#pragma unroll 2
        for (int jj = 0; jj < jn; ++jj) {
            const int j = J * kVcTile + jj;
            const float4 pj = sp[jj];
            vc_pair(C, pi0, ui0, e0, pj, su, jj, j, S, hsw, band, band_n, band_cap);
            vc_pair(C, pi1, ui1, e1, pj, su, jj, j, S, hsw, band, band_n, band_cap);
        }
    }
    __syncthreads();
    for (int k = tid; k < C.nbins; k += kVcTile) {
        long long s = 0;
        unsigned long long c = 0ull;
        for (int w = 0; w < kVcWarps; ++w) {
            const unsigned long long h = hs[w * C.nbins + k];
            const long long sw = (long long)(h << 24) >> 24;   // the low 40 bits, sign-extended
            s += sw;
            c += (h - (unsigned long long)sw) >> 40;
        }
        if (c) {
            atomicAdd(gsum + k, (unsigned long long)s);
            atomicAdd(gcnt + k, c);
        }
    }
}

// round(a / L) as the definition computes it (quotient rounded to FP64, then
// rounded half away from zero), with the division taken only where the
// product by 1/L (within 2^-50 of the quotient for |a / L| < 2) lies near a
// half-integer.
__device__ __forceinline__ double round_quotient(double a, double L, double invL)
{
    const double q = __dmul_rn(a, invL);
    const double f = fabs(q - trunc(q));
    return fabs(f - 0.5) < 0x1p-46 ? round(__ddiv_rn(a, L)) : round(q);
}

// The Lees-Edwards minimum image with every operation of the definition
// (the same results as min_image()).
__device__ __forceinline__ void vc_min_image(const KParams& P, const VcConst& C, double xi, double yi, double zi,
                                             double xj, double yj, double zj, double& dx, double& dy, double& dz)
{
    dx = __dsub_rn(xi, xj);
    dy = __dsub_rn(yi, yj);
    dz = __dsub_rn(zi, zj);
    const double n = round_quotient(dy, P.L[1], C.invL[1]);
    dy = __dsub_rn(dy, __dmul_rn(n, P.L[1]));
    dx = __dsub_rn(dx, __dmul_rn(n, C.delta));
    dx = __dsub_rn(dx, __dmul_rn(P.L[0], round_quotient(dx, P.L[0], C.invL[0])));
    dz = __dsub_rn(dz, __dmul_rn(P.L[2], round_quotient(dz, P.L[2], C.invL[2])));
}

// The listed pairs with the FP64 operations of the definition (the minimum
// image rounded exactly as written, |R|^2 < rmax^2, floor(sqrt(|R|^2) nbins /
// rmax)); products in FP64, rounded to the same fixed point.
__global__ void k_vc_band(VcConst C, KParams P, const double* __restrict__ pos, const double* __restrict__ v,
                          const int2* __restrict__ band, const unsigned int* __restrict__ band_n,
                          unsigned int band_cap, const double* __restrict__ scal,
                          unsigned long long* __restrict__ gsum, unsigned long long* __restrict__ gcnt)
{
    const unsigned int m = min(*band_n, band_cap);
    const double S = scal[1];
    for (unsigned int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
        const int2 pr = band[t];
        const int i = pr.x, j = pr.y;
        double dx, dy, dz;
        vc_min_image(P, C, pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], pos[3 * j], pos[3 * j + 1], pos[3 * j + 2],
                     dx, dy, dz);
        const double r2 = sq_norm_exact(dx, dy, dz);
        if (!(r2 < C.rmax2)) continue;
        long long k = (long long)floor(__dmul_rn(__dsqrt_rn(r2), C.inv));
        if (k > C.nbins - 1) k = C.nbins - 1;
        const double yi = pos[3 * i + 1], yj = pos[3 * j + 1];
        const double uxi = v[3 * i] - C.kappa * (yi - 0.5 * P.L[1]);
        const double uxj = v[3 * j] - C.kappa * (yj - 0.5 * P.L[1]);
        const double dot = uxi * uxj + v[3 * i + 1] * v[3 * j + 1] + v[3 * i + 2] * v[3 * j + 2];
        atomicAdd(gsum + k, (unsigned long long)llrint(dot * S));
        atomicAdd(gcnt + k, 1ull);
    }
}

size_t pairs_smem(int nbins)
{
    return sizeof(float4) * 2 * kVcTile + sizeof(unsigned long long) * kVcWarps * nbins;
}

template <class T>
cudaError_t vc_alloc(T** p, long long count)
{
    cudaFree(*p);
    *p = nullptr;
    return cudaMalloc(p, sizeof(T) * (size_t)count);
}

}  // namespace

void vc_free(VcBuffers& V)
{
    void* ptrs[] = {V.pos_n3, V.v_n3, V.p4, V.u4, V.sum, V.cnt, V.band, V.misc, V.part, V.scal, V.tiles};
    for (void* q : ptrs) cudaFree(q);
    if (V.ev[0]) cudaEventDestroy(V.ev[0]);
    if (V.ev[1]) cudaEventDestroy(V.ev[1]);
    V = VcBuffers{};
}

// Buffers for n particles (kept and reused while n does not grow).
cudaError_t vc_reserve(VcBuffers& V, long long n)
{
    cudaError_t e = cudaSuccess;
    auto T = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    if (!V.sum) {   // the fixed-size part
        T(vc_alloc(&V.sum, kVcMaxBins));
        T(vc_alloc(&V.cnt, kVcMaxBins));
        T(vc_alloc(&V.misc, 4));
        T(vc_alloc(&V.part, kVcPrepBlocks));
        T(vc_alloc(&V.scal, 2));
        // initial capacity of the boundary-pair list (grown on demand; a small
        // value set through the environment exercises the growth)
        long long bc = 1 << 20;
        if (const char* env = getenv("SHEARSIM_VCORR_BAND_CAP")) bc = std::max(1ll, atoll(env));
        T(vc_alloc(&V.band, bc));
        if (e == cudaSuccess) V.band_cap = bc;
        T(cudaEventCreate(&V.ev[0]));
        T(cudaEventCreate(&V.ev[1]));
        if (e != cudaSuccess) {
            vc_free(V);
            return e;
        }
    }
    if (n > V.n_cap) {
        V.n_cap = 0;
        T(vc_alloc(&V.pos_n3, 3 * n));
        T(vc_alloc(&V.v_n3, 3 * n));
        T(vc_alloc(&V.p4, n));
        T(vc_alloc(&V.u4, n));
        if (e == cudaSuccess) V.n_cap = n;
    }
    return e;
}

int run_velocity_correlation(VcBuffers& V, long long n, const double L[3], double delta, double kappa, int nbins,
                             double rmax, cudaStream_t s, double* sum_host, long long* cnt_host, double* vsq_host,
                             VcStats* stats, const char** err)
{
    if (n < 1 || n > (1ll << 30) || nbins < 1 || nbins > kVcMaxBins || !(rmax > 0.0) || !std::isfinite(rmax) ||
        !(delta >= 0.0) || !(delta < L[0]) || !std::isfinite(kappa)) {
        if (err) *err = "velocity correlation: needs n >= 1, 1 <= nbins <= 1024, rmax > 0, 0 <= delta < L_x";
        return SP_ERR_INVALID_ARG;
    }
    for (int a = 0; a < 3; ++a)
        if (!(L[a] > 0.0) || !std::isfinite(L[a])) {
            if (err) *err = "velocity correlation: box edges must be positive";
            return SP_ERR_INVALID_ARG;
        }
    if (vc_reserve(V, n) != cudaSuccess) {
        cudaGetLastError();
        return SP_ERR_OOM;
    }
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(k_vc_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pairs_smem(kVcMaxBins)) !=
            cudaSuccess)
            return SP_ERR_CUDA;
        attr_set = true;
    }

    VcConst C{};
    C.n = (int)n;
    C.nbins = nbins;
    C.ntile = (int)((n + kVcTile - 1) / kVcTile);
    C.chunk = C.ntile <= 128 ? 1 : (C.ntile <= 256 ? 4 : 16);   // at most 16 (the packed histogram words)
    for (int a = 0; a < 3; ++a) {
        C.Lf[a] = (float)L[a];
        C.iLf[a] = (float)(1.0 / L[a]);
    }
    C.df = (float)delta;
    // E bounds |r_FP32 - r| for positions in [0, L): each FP32 operation rounds
    // by at most 2^-24 of a result no larger than 2 L_x (x), L_y, L_z, plus the
    // relative roundings of the squares, the approximate square root (3 ulp)
    // and the scaling.
    const double u = 5.9604644775390625e-8;
    const double E = u * (20.0 * (L[0] + L[1] + L[2]) + 16.0 * rmax);
    C.r2_hi = nextafterf((float)((rmax + 2.0 * E) * (rmax + 2.0 * E)), INFINITY);
    C.r_band = nextafterf((float)(rmax - 2.0 * E), -INFINITY);
    C.inv = (double)nbins / rmax;
    C.inv_f = (float)C.inv;
    C.eb = (float)std::min(0.5, 2.0 * E * C.inv + 8.0 * u * nbins + 4.0 * u);
    for (int a = 0; a < 3; ++a) {
        C.half[a] = (float)(L[a] * (0.5 - 64.0 * u));
        C.invL[a] = 1.0 / L[a];
    }
    C.delta = delta;
    C.kappa = kappa;
    C.rmax2 = rmax * rmax;

    KParams P{};
    P.L[0] = L[0];
    P.L[1] = L[1];
    P.L[2] = L[2];

    // blocks (I, first J of a run of `chunk` c' tiles): I covers particles
    // [512 I, 512 I + 512), so the tiles below 2 I hold no partner j > i
    std::vector<int2> tl;
    const int ni = (int)((n + 2 * kVcTile - 1) / (2 * kVcTile));
    for (int I = 0; I < ni; ++I)
        for (int J = 2 * I; J < C.ntile; J += C.chunk) tl.push_back(make_int2(I, J));
    if ((long long)tl.size() > V.tiles_cap) {
        V.tiles_cap = 0;
        V.tiles_n = 0;
        if (vc_alloc(&V.tiles, (long long)tl.size()) != cudaSuccess) {
            cudaGetLastError();
            return SP_ERR_OOM;
        }
        V.tiles_cap = (long long)tl.size();
    }
    if (V.tiles_n != (long long)tl.size() || V.tiles_for != n) {
        if (cudaMemcpyAsync(V.tiles, tl.data(), sizeof(int2) * tl.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return SP_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return SP_ERR_CUDA;
        V.tiles_n = (long long)tl.size();
        V.tiles_for = n;
    }

    const int prep_blocks = (int)std::min<long long>(kVcPrepBlocks, (n + kVcTile - 1) / kVcTile);
    unsigned int* band_n = reinterpret_cast<unsigned int*>(V.misc);
    unsigned int* umax = band_n + 1;
    int* flag = reinterpret_cast<int*>(band_n + 2);
    std::vector<unsigned long long> hs(nbins), hc(nbins);
    unsigned int misc_h[4];
    double scal_h[2];
    for (int attempt = 0; attempt < 2; ++attempt) {
        const unsigned int cap = (unsigned int)std::min<long long>(V.band_cap, 0xffffffffll);
        if (cudaMemsetAsync(V.sum, 0, sizeof(unsigned long long) * nbins, s) != cudaSuccess ||
            cudaMemsetAsync(V.cnt, 0, sizeof(unsigned long long) * nbins, s) != cudaSuccess ||
            cudaMemsetAsync(V.misc, 0, sizeof(unsigned int) * 4, s) != cudaSuccess)
            return SP_ERR_CUDA;
        k_vc_prep<<<prep_blocks, kVcTile, 0, s>>>(C, P, V.pos_n3, V.v_n3, V.p4, V.u4, V.part, umax, flag);
        k_vc_scale<<<1, 32, 0, s>>>(C.n, prep_blocks, V.part, umax, V.scal);
        cudaEventRecord(V.ev[0], s);
        k_vc_pairs<<<(unsigned)tl.size(), kVcTile, pairs_smem(nbins), s>>>(C, V.p4, V.u4, V.tiles, V.scal, V.sum,
                                                                          V.cnt, V.band, band_n, cap);
        cudaEventRecord(V.ev[1], s);
        k_vc_band<<<4 * 152, 256, 0, s>>>(C, P, V.pos_n3, V.v_n3, V.band, band_n, cap, V.scal, V.sum, V.cnt);
        if (cudaGetLastError() != cudaSuccess) return SP_ERR_CUDA;
        if (cudaMemcpyAsync(hs.data(), V.sum, sizeof(unsigned long long) * nbins, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(hc.data(), V.cnt, sizeof(unsigned long long) * nbins, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(misc_h, V.misc, sizeof(misc_h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(scal_h, V.scal, sizeof(scal_h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return SP_ERR_CUDA;
        const int bad = (int)misc_h[2];
        if (bad) {
            if (err) *err = "velocity correlation: positions must lie in [0, L) on every axis";
            return SP_ERR_INVALID_ARG;
        }
        if (misc_h[0] <= cap) break;
        // more pairs near a boundary than the list holds: grow it and run again
        const long long want = (long long)misc_h[0] + (misc_h[0] >> 2) + 1024;
        V.band_cap = 0;
        if (attempt == 1 || vc_alloc(&V.band, want) != cudaSuccess) {
            cudaGetLastError();
            if (err) *err = "velocity correlation: boundary pair list overflow";
            return SP_ERR_OOM;
        }
        V.band_cap = want;
    }
    const double S = scal_h[1];
    for (int k = 0; k < nbins; ++k) {
        if (sum_host) sum_host[k] = (double)(long long)hs[k] / S;
        if (cnt_host) cnt_host[k] = (long long)hc[k];
    }
    if (vsq_host) *vsq_host = scal_h[0];
    if (stats) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, V.ev[0], V.ev[1]);
        stats->pairs_ms = ms;
        stats->band_pairs = misc_h[0];
        stats->blocks = (long long)tl.size();
    }
    return SP_OK;
}

}  // namespace ss
