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

// The interval's map and the interpolant's coefficients on the device (so
// that a whole step stays one graph): cs[0] = 2 / (b - a), cs[1] = (b + a) /
// (b - a), cs[2 + k] = c_k, k <= degree; csf the same as double-floats.  With
// no coupling (lambda_max = 1) p = 1: c_0 = 2, the rest 0.
__global__ void k_cheb_coeffs(const unsigned long long* __restrict__ bound, int degree, double* __restrict__ cs,
                              float2* __restrict__ csf)
{
    const double lmax = __longlong_as_double((long long)*bound);
    const bool ident = !(lmax - 1.0 > 1e-12);
    const int N = degree + 1;
    const double pi = 3.141592653589793238462643383279502884;
    auto split = [](double x) { const float h = (float)x; return make_float2(h, (float)(x - (double)h)); };
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        double acc = 0.0;
        if (!ident)
            for (int j = 0; j < N; ++j) {
                const double th = pi * (j + 0.5) / N;
                acc += sqrt(0.5 * (lmax - 1.0) * cos(th) + 0.5 * (lmax + 1.0)) * cos(k * th);
            }
        const double c = ident ? (k == 0 ? 2.0 : 0.0) : 2.0 / N * acc;
        cs[2 + k] = c;
        csf[2 + k] = split(c);
    }
    if (threadIdx.x == 0) {
        const double s1 = ident ? 0.0 : 2.0 / (lmax - 1.0), s0 = ident ? 0.0 : (lmax + 1.0) / (lmax - 1.0);
        cs[0] = s1;
        cs[1] = s0;
        csf[0] = split(s1);
        csf[1] = split(s0);
    }
}

// One degree k: tn = u(tc) (k = 1) or 2 u(tc) - tp; y = c_0/2 tc + c_1 tn (k = 1) or y += c_k tn.
__global__ void __launch_bounds__(256) k_cheb_step(KParams P, DevBuffers B, const double* __restrict__ tc,
                                                   const double* __restrict__ tp, double* __restrict__ tn,
                                                   double* __restrict__ y, const double* __restrict__ cs, int kdeg)
{
    const int first = kdeg == 1;
    const double s1 = cs[0], s0 = cs[1], ck = cs[2 + kdeg], c0h = 0.5 * cs[2];
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
                                                      float4* __restrict__ y, const float2* __restrict__ csf, int kdeg)
{
    const int first = kdeg == 1;
    const float2 s1 = csf[0], s0 = csf[1], ck = csf[2 + kdeg], c0 = csf[2];
    const float2 c0h = make_float2(0.5f * c0.x, 0.5f * c0.y);   // exact halving
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

// The normals the assembly of this step used (drawn by the pair search,
// injected by id, or drawn here as the assembly would), as FP64 planes (FP64
// path) or double-float records (mixed path).
__global__ void k_fdt_normals(KParams P, DevBuffers B, int use_inj, double* __restrict__ gp,
                              float4* __restrict__ gr)
{
    const DevState* st = B.st;
    if (st->error | st->overflow) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const int np = P.npad;
    const bool drawn = st->noise_step == st->step;
    const long long id = B.id_w[i];
    if (P.mixed) {
        dfloat g0, g1, g2;
        if (use_inj) {
            g0 = df_split(B.xi_inj[3 * id]);
            g1 = df_split(B.xi_inj[3 * id + 1]);
            g2 = df_split(B.xi_inj[3 * id + 2]);
        } else if (drawn) {
            const float2* n2 = reinterpret_cast<const float2*>(B.noise3);
            const float2 a = n2[i], b = n2[np + i], c = n2[2 * np + i];
            g0 = dfloat{a.x, a.y};
            g1 = dfloat{b.x, b.y};
            g2 = dfloat{c.x, c.y};
        } else {
            normals3_df(B.rng_tab, P.seed, (unsigned long long)st->step, (unsigned long long)id, g0, g1, g2);
        }
        gr[2 * i] = make_float4(g0.hi, g1.hi, g2.hi, 0.f);
        gr[2 * i + 1] = make_float4(g0.lo, g1.lo, g2.lo, 0.f);
    } else {
        double g0, g1, g2;
        if (use_inj) {
            g0 = B.xi_inj[3 * id];
            g1 = B.xi_inj[3 * id + 1];
            g2 = B.xi_inj[3 * id + 2];
        } else if (drawn) {
            g0 = B.noise3[i];
            g1 = B.noise3[np + i];
            g2 = B.noise3[2 * np + i];
        } else {
            normals3(P.seed, (unsigned long long)st->step, (unsigned long long)id, g0, g1, g2);
        }
        gp[i] = g0;
        gp[np + i] = g1;
        gp[2 * np + i] = g2;
    }
}

// b += (noise amplitude / zeta) (xi - g): the step's right-hand side with the
// correlated noise in place of the independent one.
__global__ void k_fdt_add(KParams P, DevBuffers B, const double* __restrict__ gp, const double* __restrict__ yp,
                          const float4* __restrict__ gr, const float4* __restrict__ yr)
{
    const DevState* st = B.st;
    if (st->error | st->overflow) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const int np = P.npad;
    if (P.mixed) {
        const dfloat amp{P.amp_z_hi, P.amp_z_lo};
        const float4 gh = gr[2 * i], gl = gr[2 * i + 1], yh = yr[2 * i], yl = yr[2 * i + 1];
        const float4 bh = B.bdf[2 * i], bl = B.bdf[2 * i + 1];
        const dfloat g[3] = {{gh.x, gl.x}, {gh.y, gl.y}, {gh.z, gl.z}};
        const dfloat y[3] = {{yh.x, yl.x}, {yh.y, yl.y}, {yh.z, yl.z}};
        const dfloat b[3] = {{bh.x, bl.x}, {bh.y, bl.y}, {bh.z, bl.z}};
        dfloat r[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) r[c] = df_add(b[c], df_mul(amp, df_add(y[c], df_neg(g[c]))));
        B.bdf[2 * i] = make_float4(r[0].hi, r[1].hi, r[2].hi, 0.f);
        B.bdf[2 * i + 1] = make_float4(r[0].lo, r[1].lo, r[2].lo, 0.f);
    } else {
        const double amp = P.noise_amp / P.zeta;
#pragma unroll
        for (int c = 0; c < 3; ++c) B.b[c * np + i] += amp * (yp[c * np + i] - gp[c * np + i]);
    }
}

}  // namespace

int enqueue_cheb(const KParams& P, DevBuffers& B, FdtBuffers& V, int degree, cudaStream_t s)
{
    const bool df = P.mixed != 0;
    cheb_bound(P, B, V.bound, s);
    cheb_coeffs(V.bound, degree, V.cs, V.csf, s);
    auto step = [&](int tc, int tp, int tn, int k) {
        if (df)
            cheb_step_df(P, B, static_cast<float4*>(V.v[tc]), tp < 0 ? nullptr : static_cast<float4*>(V.v[tp]),
                         static_cast<float4*>(V.v[tn]), static_cast<float4*>(V.v[4]), V.csf, k, s);
        else
            cheb_step(P, B, static_cast<double*>(V.v[tc]), tp < 0 ? nullptr : static_cast<double*>(V.v[tp]),
                      static_cast<double*>(V.v[tn]), static_cast<double*>(V.v[4]), V.cs, k, s);
    };
    // T_0 = g stays in v[0]; T_1 .. T_K rotate among v[1], v[2], v[3]
    step(0, -1, 1, 1);
    int prev = 0, cur = 1;
    for (int k = 2; k <= degree; ++k) {
        const int next = prev == 0 ? 2 : 6 - prev - cur;
        step(cur, prev, next, k);
        prev = cur;
        cur = next;
    }
    return 2 + degree;
}

int enqueue_fdt_noise(const KParams& P, DevBuffers& B, FdtBuffers& V, int degree, bool use_inj, cudaStream_t s)
{
    const bool df = P.mixed != 0;
    k_fdt_normals<<<grid_for(P.n, 256, 1 << 30), 256, 0, s>>>(P, B, use_inj ? 1 : 0,
                                                                 df ? nullptr : static_cast<double*>(V.v[0]),
                                                                 df ? static_cast<float4*>(V.v[0]) : nullptr);
    const int launches = enqueue_cheb(P, B, V, degree, s);
    k_fdt_add<<<grid_for(P.n, 256, 1 << 30), 256, 0, s>>>(
        P, B, df ? nullptr : static_cast<double*>(V.v[0]), df ? nullptr : static_cast<double*>(V.v[4]),
        df ? static_cast<float4*>(V.v[0]) : nullptr, df ? static_cast<float4*>(V.v[4]) : nullptr);
    return launches + 2;
}

cudaError_t cheb_step_df(const KParams& P, DevBuffers& B, const float4* tc, const float4* tp, float4* tn, float4* y,
                         const float2* csf, int k, cudaStream_t s)
{
    k_cheb_step_df<<<P.nslots / 256, 256, 0, s>>>(P, B, tc, tp, tn, y, csf, k);
    return cudaGetLastError();
}

cudaError_t cheb_coeffs(const unsigned long long* bound, int degree, double* cs, float2* csf, cudaStream_t s)
{
    k_cheb_coeffs<<<1, 128, 0, s>>>(bound, degree, cs, csf);
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
                      const double* cs, int k, cudaStream_t s)
{
    k_cheb_step<<<P.nslots / 256, 256, 0, s>>>(P, B, tc, tp, tn, y, cs, k);
    return cudaGetLastError();
}

}  // namespace ss
