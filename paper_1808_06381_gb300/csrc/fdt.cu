// FDT-consistent thermal noise: xi = p(A) g, p the degree-K Chebyshev
// interpolant of sqrt on [1, lambda_max], so that xi has covariance ~A when g
// has covariance I (the paper draws the noise independently per particle; a
// noise correlated as A^(1/2) makes the velocities' fluctuations consistent
// with the friction matrix of Eq. algebra).  lambda_max is Gershgorin's bound
// max_i (A_ii + alpha sum_j w_ij) = max_i (2 A_ii - 1), the lower end is 1
// (A = I + alpha L_w with L_w positive semidefinite).
//
// With u = (2 A - (b + a) I) / (b - a) mapping [a, b] = [1, lambda_max] onto
// [-1, 1]: T_0 = g, T_1 = u g, T_{k+1} = 2 u T_k - T_{k-1}, and
// xi = c_0 / 2 T_0 + sum_k c_k T_k.  One kernel per degree: the sliced-layout
// SpMV of T_k, the recurrence and the accumulation of xi, per row; in FP64
// for the FP64 path, in double-float on the FP32 pipes for the mixed path.
#include <math.h>

#include "internal.cuh"

namespace ss {

namespace {

__device__ __forceinline__ double weight_at(const KParams& P, const DevBuffers& B, int e)
{
    return P.mixed ? (double)B.val32[e] + (double)B.val32lo[e] : B.val[e];
}

__device__ __forceinline__ double diag_at(const KParams& P, const DevBuffers& B, int i)
{
    return P.mixed ? (double)B.diag32[i] + (double)B.diag32lo[i] : B.diag[i];
}

// max_i (2 A_ii - 1) as the bits of a positive double (they order like integers)
__global__ void k_cheb_bound(KParams P, DevBuffers B, unsigned long long* out)
{
    double m = 1.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x)
        m = fmax(m, 2.0 * diag_at(P, B, i) - 1.0);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// One degree: tn = u(tc) (first) or 2 u(tc) - tp; y = c0h tc + ck tn (first) or y += ck tn.
__global__ void __launch_bounds__(256) k_cheb_step(KParams P, DevBuffers B, const double* __restrict__ tc,
                                                   const double* __restrict__ tp, double* __restrict__ tn,
                                                   double* __restrict__ y, double s1, double s0, double ck,
                                                   double c0h, int first)
{
    const int slot = blockIdx.x * 256 + threadIdx.x;
    if (slot >= P.nslots) return;
    const int row = B.slot_row[slot];
    if (row < 0) return;
    const int np = P.npad;
    const int e1 = B.chunk_off[(slot >> 5) + 1];
    double s[3] = {0.0, 0.0, 0.0};
    for (int e = B.chunk_off[slot >> 5] + (slot & 31); e < e1; e += 32) {
        const int j = B.col[e];
        const double w = weight_at(P, B, e);
#pragma unroll
        for (int c = 0; c < 3; ++c) s[c] = fma(w, tc[c * np + j], s[c]);
    }
    const double d = diag_at(P, B, row);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int k = c * np + row;
        const double t = tc[k];
        const double At = d * t - P.alpha * s[c];
        const double u = s1 * At - s0 * t;
        const double v = first ? u : 2.0 * u - tp[k];
        tn[k] = v;
        y[k] = first ? c0h * t + ck * v : y[k] + ck * v;
    }
}

// The same degree step for the mixed path in double-float on the FP32 pipes:
// T_k and xi as 32-byte records per row (hi float4, lo float4), the weights
// and A_ii as their double-float pairs.
__global__ void __launch_bounds__(256) k_cheb_step_df(KParams P, DevBuffers B, const float4* __restrict__ tc,
                                                      const float4* __restrict__ tp, float4* __restrict__ tn,
                                                      float4* __restrict__ y, float2 s1, float2 s0, float2 ck,
                                                      float2 c0h, int first)
{
    const int slot = blockIdx.x * 256 + threadIdx.x;
    if (slot >= P.nslots) return;
    const int row = B.slot_row[slot];
    if (row < 0) return;
    dfloat s[3];
    row_sum_df<4>(B.col, B.val32, B.val32lo, tc, B.chunk_off[slot >> 5] + (slot & 31), B.chunk_off[(slot >> 5) + 1],
                  s);
    const dfloat d{B.diag32[row], B.diag32lo[row]}, al{P.alpha_hi, P.alpha_lo};
    const dfloat S1{s1.x, s1.y}, S0{s0.x, s0.y}, CK{ck.x, ck.y}, C0{c0h.x, c0h.y};
    const float4 th = tc[2 * row], tl = tc[2 * row + 1];
    const dfloat t[3] = {{th.x, tl.x}, {th.y, tl.y}, {th.z, tl.z}};
    dfloat pv[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}, yv[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    if (!first) {
        const float4 ph = tp[2 * row], pl = tp[2 * row + 1], yh = y[2 * row], yl = y[2 * row + 1];
        pv[0] = dfloat{ph.x, pl.x};
        pv[1] = dfloat{ph.y, pl.y};
        pv[2] = dfloat{ph.z, pl.z};
        yv[0] = dfloat{yh.x, yl.x};
        yv[1] = dfloat{yh.y, yl.y};
        yv[2] = dfloat{yh.z, yl.z};
    }
    dfloat v[3], yn[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const dfloat At = df_add(df_mul(d, t[c]), df_neg(df_mul(al, s[c])));
        const dfloat u = df_add(df_mul(S1, At), df_neg(df_mul(S0, t[c])));
        v[c] = first ? u : df_add(dfloat{2.f * u.hi, 2.f * u.lo}, df_neg(pv[c]));
        yn[c] = first ? df_add(df_mul(C0, t[c]), df_mul(CK, v[c])) : df_add(yv[c], df_mul(CK, v[c]));
    }
    tn[2 * row] = make_float4(v[0].hi, v[1].hi, v[2].hi, 0.f);
    tn[2 * row + 1] = make_float4(v[0].lo, v[1].lo, v[2].lo, 0.f);
    y[2 * row] = make_float4(yn[0].hi, yn[1].hi, yn[2].hi, 0.f);
    y[2 * row + 1] = make_float4(yn[0].lo, yn[1].lo, yn[2].lo, 0.f);
}

// FP64 planes [3][npad] to double-float records and back.
__global__ void k_cheb_split(KParams P, const double* __restrict__ g, float4* __restrict__ t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const int np = P.npad;
    const dfloat a = df_split(g[i]), b = df_split(g[np + i]), c = df_split(g[2 * np + i]);
    t[2 * i] = make_float4(a.hi, b.hi, c.hi, 0.f);
    t[2 * i + 1] = make_float4(a.lo, b.lo, c.lo, 0.f);
}

__global__ void k_cheb_join(KParams P, const float4* __restrict__ y, double* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const int np = P.npad;
    const float4 h = y[2 * i], l = y[2 * i + 1];
    out[i] = (double)h.x + (double)l.x;
    out[np + i] = (double)h.y + (double)l.y;
    out[2 * np + i] = (double)h.z + (double)l.z;
}

}  // namespace

cudaError_t cheb_step_df(const KParams& P, DevBuffers& B, const float4* tc, const float4* tp, float4* tn, float4* y,
                         double s1, double s0, double ck, double c0h, bool first, cudaStream_t s)
{
    auto split = [](double x) { const float h = (float)x; return make_float2(h, (float)(x - (double)h)); };
    k_cheb_step_df<<<P.nslots / 256, 256, 0, s>>>(P, B, tc, tp, tn, y, split(s1), split(s0), split(ck), split(c0h),
                                                  first ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t cheb_split(const KParams& P, const double* g, float4* t, cudaStream_t s)
{
    k_cheb_split<<<grid_for(P.n, 256, 1 << 30), 256, 0, s>>>(P, g, t);
    return cudaGetLastError();
}

cudaError_t cheb_join(const KParams& P, const float4* y, double* out, cudaStream_t s)
{
    k_cheb_join<<<grid_for(P.n, 256, 1 << 30), 256, 0, s>>>(P, y, out);
    return cudaGetLastError();
}

cudaError_t cheb_bound(const KParams& P, DevBuffers& B, unsigned long long* out_dev, cudaStream_t s)
{
    cudaMemsetAsync(out_dev, 0, sizeof(unsigned long long), s);
    k_cheb_bound<<<grid_for(P.n, 256, 4 * 152), 256, 0, s>>>(P, B, out_dev);
    return cudaGetLastError();
}

cudaError_t cheb_step(const KParams& P, DevBuffers& B, const double* tc, const double* tp, double* tn, double* y,
                      double s1, double s0, double ck, double c0h, bool first, cudaStream_t s)
{
    k_cheb_step<<<P.nslots / 256, 256, 0, s>>>(P, B, tc, tp, tn, y, s1, s0, ck, c0h, first ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace ss
