// Jacobi-preconditioned conjugate gradients for Eq. algebra (arXiv 1808.06381,
// §Method: "use a sparse matrix solver"), on the GPU without host round trips.
//
// The three Cartesian components share one scalar matrix A = D - alpha W
// (D = diag, W = the truncated weights), so CG runs on (A (x) I_3) v = b and
// the step lengths are shared by the three components.  All CG scalars stay
// in device memory; each kernel's last block to finish reduces the per-block
// partial sums in a fixed order (deterministic, and no block ever waits for
// another).
//
// One iteration is two kernels.  With z = D^-1 r the search direction update
// p' = z + beta p gives A p' = A z + beta (A p), so the SpMV kernel gathers z,
// forms q' = A z + beta q and p' = z + beta p for its own rows and reduces
// p'.q' (then alpha = rho / p'.q'); the update kernel applies alpha and
// reduces r.r and r.z (then beta and the convergence test).
//
// FP64 solver: everything in FP64; z is stored by the update kernel so the
// SpMV gathers one FP64 3-vector per entry.
//
// Mixed solver: the matrix values, the Jacobi diagonal and the vectors r, p,
// q are FP32 (one float4 per row), the iteration solves for a correction d
// (FP32) of the FP64 solution x; dots accumulate in FP64.  When the FP32
// residual has dropped by the inner factor, or meets the tolerance, d is
// folded into x and the true residual b - A x is recomputed with the FP64
// matrix; the solve ends when that meets the tolerance, else the iteration
// restarts from it (residual replacement).
//
// Inside a CUDA graph the loop is a conditional WHILE node and the
// true-residual check an IF node; the kernels set both conditions.
#include <math.h>

#include "internal.cuh"

namespace ss {

constexpr int kSpmvBlock = 256;

__device__ __forceinline__ bool halted(const DevState* st)
{
    return (st->error | st->overflow | st->done) != 0;
}

__device__ __forceinline__ void set_cond(const CgLaunch& C, unsigned long long h, unsigned v)
{
    if (C.use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)h, v);
}

// Rows handled by a warp-uniform loop: group g of T lanes takes rows
// g, g + ngroups, ...; the loop bound is uniform across the warp so the
// shuffles always see every lane.
#define SS_ROW_LOOP_BEGIN(T)                                                         \
    const int lane = threadIdx.x & ((T) - 1);                                        \
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;                          \
    const int ngroups = (gridDim.x * blockDim.x) / (T);                              \
    const int warp_first_group = ((gtid >> 5) << 5) / (T);                           \
    const int group_in_warp = (threadIdx.x & 31) / (T);                              \
    for (int base = warp_first_group; base < P.n; base += ngroups) {                 \
        const int i = base + group_in_warp;                                          \
        const bool active = i < P.n;

#define SS_ROW_LOOP_END }

template <int T, class V>
__device__ __forceinline__ void group_sum3(V& s0, V& s1, V& s2)
{
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o, T);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o, T);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o, T);
    }
}

// s_a = sum_j w_ij v_a[j] over row i (FP64 planes), T lanes per row.
template <int T>
__device__ __forceinline__ void row_sum64(const int* __restrict__ row_ptr, const int* __restrict__ col,
                                          const double* __restrict__ val, const double* __restrict__ v,
                                          int np, int i, bool active, int lane, double& s0, double& s1,
                                          double& s2)
{
    s0 = s1 = s2 = 0.0;
    if (active) {
        const int end = row_ptr[i + 1];
        for (int k = row_ptr[i] + lane; k < end; k += T) {
            const int j = col[k];
            const double w = val[k];
            s0 += w * v[j];
            s1 += w * v[np + j];
            s2 += w * v[2 * np + j];
        }
    }
    group_sum3<T>(s0, s1, s2);
}

// s = sum_j w_ij dinv_j r_j over row i (FP32, float4 rows), T lanes per row.
template <int T>
__device__ __forceinline__ void row_sum32_z(const int* __restrict__ row_ptr, const int* __restrict__ col,
                                            const float* __restrict__ val, const float4* __restrict__ r,
                                            const float* __restrict__ dinv, int i, bool active, int lane,
                                            float& s0, float& s1, float& s2)
{
    s0 = s1 = s2 = 0.f;
    if (active) {
        const int end = row_ptr[i + 1];
        for (int k = row_ptr[i] + lane; k < end; k += T) {
            const int j = col[k];
            const float w = val[k] * dinv[j];
            const float4 rj = r[j];
            s0 = fmaf(w, rj.x, s0);
            s1 = fmaf(w, rj.y, s1);
            s2 = fmaf(w, rj.z, s2);
        }
    }
    group_sum3<T>(s0, s1, s2);
}

// ============================================================== FP64 solver

// r = b - A x0 (or r = b and x = 0); z = D^-1 r; p = q = 0.
template <int T>
__global__ void __launch_bounds__(kSpmvBlock) k64_init(KParams P, DevBuffers B, int from_x)
{
    DevState* st = B.st;
    if (st->error | st->overflow) return;
    const int np = P.npad;
    double bb = 0.0, rr = 0.0, rz = 0.0;
    SS_ROW_LOOP_BEGIN(T)
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    if (from_x) row_sum64<T>(B.row_ptr, B.col, B.val, B.x, np, i, active, lane, s0, s1, s2);
    if (active && lane == 0) {
        const double s[3] = {s0, s1, s2};
        const double d = B.diag[i], di = B.dinv[i];
        double rs = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int k = c * np + i;
            const double bk = B.b[k];
            double rk = bk;
            if (from_x)
                rk = bk - (d * B.x[k] - P.alpha * s[c]);
            else
                B.x[k] = 0.0;
            B.r[k] = rk;
            B.z[k] = di * rk;
            B.p[k] = 0.0;
            B.q[k] = 0.0;
            bb += bk * bk;
            rs += rk * rk;
        }
        rr += rs;
        rz += di * rs;
    }
    SS_ROW_LOOP_END
    const double v[3] = {bb, rr, rz};
    if (publish_partials<3>(v, B.partials, &st->ticket[0])) {
        double out[3];
        reduce_partials<3>(B.partials, out);
        if (threadIdx.x == 0) {
            st->bnorm2 = out[0];
            st->rr = out[1];
            st->rr_restart = out[1];
            st->rho = out[2];
            st->beta = 0.0;
            st->iter = 0;
            st->restarts = 0;
            st->check_true = 0;
            st->status = 0;
            st->zero_b = 0;
            st->done = 0;
            if (!isfinite(out[0]) || !isfinite(out[1])) {
                st->status = SP_ERR_NONFINITE;
                st->error = SP_ERR_NONFINITE;
                st->done = 1;
            } else if (out[0] == 0.0) {
                st->zero_b = 1;   // b = 0: the solution is v = 0
                st->done = 1;
                st->last_res = 0.0;
            } else if (out[1] <= P.tol2 * out[0]) {
                st->done = 1;     // the start vector already meets the tolerance (exact r)
                st->last_res = sqrt(out[1] / out[0]);
            }
        }
    }
}

// q = A z + beta q; p = z + beta p; p.q.  Last block: alpha = rho / p.q.
template <int T>
__global__ void __launch_bounds__(kSpmvBlock) k64_spmv(KParams P, DevBuffers B)
{
    DevState* st = B.st;
    if (halted(st)) return;
    const int np = P.npad;
    const double beta = st->beta;
    double pq = 0.0;
    SS_ROW_LOOP_BEGIN(T)
    double s0, s1, s2;
    row_sum64<T>(B.row_ptr, B.col, B.val, B.z, np, i, active, lane, s0, s1, s2);
    if (active && lane == 0) {
        const double s[3] = {s0, s1, s2};
        const double d = B.diag[i];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int k = c * np + i;
            const double zk = B.z[k];
            const double az = d * zk - P.alpha * s[c];
            const double qk = beta == 0.0 ? az : az + beta * B.q[k];
            const double pk = beta == 0.0 ? zk : zk + beta * B.p[k];
            B.q[k] = qk;
            B.p[k] = pk;
            pq += pk * qk;
        }
    }
    SS_ROW_LOOP_END
    const double v[1] = {pq};
    if (publish_partials<1>(v, B.partials, &st->ticket[0])) {
        double out[1];
        reduce_partials<1>(B.partials, out);
        if (threadIdx.x == 0) {
            st->pq = out[0];
            if (!(out[0] > 0.0) || !isfinite(out[0])) {
                st->status = SP_ERR_NONFINITE;
                st->error = SP_ERR_NONFINITE;
                st->done = 1;
            } else {
                st->alpha = st->rho / out[0];
            }
        }
    }
}

// Last block of an update kernel: beta, rho and the stopping test on the
// recurrence residual, which arms the true-residual check.
__device__ __forceinline__ void update_scalars(const KParams& P, DevState* st, double rr, double rz,
                                               double inner_target, const CgLaunch& C)
{
    st->iter += 1;
    st->rr = rr;
    st->beta = rz / st->rho;
    st->rho = rz;
    if (!isfinite(rr) || !isfinite(rz)) {
        st->status = SP_ERR_NONFINITE;
        st->error = SP_ERR_NONFINITE;
        st->done = 1;
    } else if (st->iter >= P.max_iter + kMaxCgRestarts + 4) {
        // the true-residual check should have ended the solve by now
        st->status = SP_ERR_NOT_CONVERGED;
        st->error = SP_ERR_NOT_CONVERGED;
        st->done = 1;
    } else if (rr <= inner_target || st->iter >= P.max_iter) {
        st->check_true = 1;
    }
    set_cond(C, C.h_check, (unsigned)(st->check_true && !st->done));
    set_cond(C, C.h_loop, st->done ? 0u : 1u);
}

// x += alpha p; r -= alpha q; z = D^-1 r; partial r.r and r.z.
__global__ void __launch_bounds__(kVecBlock) k64_update(KParams P, DevBuffers B, CgLaunch C)
{
    DevState* st = B.st;
    if (halted(st)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            set_cond(C, C.h_check, 0u);
            set_cond(C, C.h_loop, 0u);
        }
        return;
    }
    const int np = P.npad;
    const double a = st->alpha;
    double rr = 0.0, rz = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const double di = B.dinv[i];
        double rs = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int k = c * np + i;
            B.x[k] += a * B.p[k];
            const double rk = B.r[k] - a * B.q[k];
            B.r[k] = rk;
            B.z[k] = di * rk;
            rs += rk * rk;
        }
        rr += rs;
        rz += di * rs;
    }
    const double v[2] = {rr, rz};
    if (publish_partials<2>(v, B.partials, &st->ticket[0])) {
        double out[2];
        reduce_partials<2>(B.partials, out);
        if (threadIdx.x == 0) update_scalars(P, st, out[0], out[1], P.tol2 * st->bnorm2, C);
    }
}

// Last block of a true-residual kernel: accept, restart from the true
// residual (beta = 0), or give up at the iteration cap.
__device__ __forceinline__ void true_residual_scalars(const KParams& P, DevState* st, double rr,
                                                      double rz, const CgLaunch& C)
{
    st->check_true = 0;
    st->true_checks += 1;
    st->rr_true = rr;
    st->last_res = sqrt(rr / st->bnorm2);
    if (!isfinite(rr)) {
        st->status = SP_ERR_NONFINITE;
        st->error = SP_ERR_NONFINITE;
        st->done = 1;
    } else if (rr <= P.tol2 * st->bnorm2) {
        st->done = 1;
        st->status = SP_OK;
    } else if (st->iter >= P.max_iter || st->restarts >= kMaxCgRestarts + 8) {
        st->done = 1;
        st->status = SP_ERR_NOT_CONVERGED;
        st->error = SP_ERR_NOT_CONVERGED;
    } else {
        st->restarts += 1;
        st->rho = rz;
        st->beta = 0.0;
        st->rr = rr;
        st->rr_restart = rr;
    }
    set_cond(C, C.h_loop, st->done ? 0u : 1u);
}

// r = b - A x in FP64; z = D^-1 r; partial r.r and r.z.
template <int T>
__global__ void __launch_bounds__(kSpmvBlock) k64_true_residual(KParams P, DevBuffers B, int always,
                                                                CgLaunch C)
{
    DevState* st = B.st;
    if (halted(st) || (!always && !st->check_true)) return;
    const int np = P.npad;
    double rr = 0.0, rz = 0.0;
    SS_ROW_LOOP_BEGIN(T)
    double s0, s1, s2;
    row_sum64<T>(B.row_ptr, B.col, B.val, B.x, np, i, active, lane, s0, s1, s2);
    if (active && lane == 0) {
        const double s[3] = {s0, s1, s2};
        const double d = B.diag[i], di = B.dinv[i];
        double rs = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int k = c * np + i;
            const double rk = B.b[k] - (d * B.x[k] - P.alpha * s[c]);
            B.r[k] = rk;
            B.z[k] = di * rk;
            rs += rk * rk;
        }
        rr += rs;
        rz += di * rs;
    }
    SS_ROW_LOOP_END
    const double v[2] = {rr, rz};
    if (publish_partials<2>(v, B.partials, &st->ticket[0])) {
        double out[2];
        reduce_partials<2>(B.partials, out);
        if (threadIdx.x == 0) true_residual_scalars(P, st, out[0], out[1], C);
    }
}

// ============================================================= mixed solver

__device__ __forceinline__ float4 f4(float x, float y, float z) { return make_float4(x, y, z, 0.f); }

// r = b - A x0 in FP64 (or r = b and x = 0); r4 = fp32(r); d = p = q = 0.
template <int T>
__global__ void __launch_bounds__(kSpmvBlock) k32_init(KParams P, DevBuffers B, int from_x)
{
    DevState* st = B.st;
    if (st->error | st->overflow) return;
    const int np = P.npad;
    double bb = 0.0, rr = 0.0, rz = 0.0;
    SS_ROW_LOOP_BEGIN(T)
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    if (from_x) row_sum64<T>(B.row_ptr, B.col, B.val, B.x, np, i, active, lane, s0, s1, s2);
    if (active && lane == 0) {
        const double s[3] = {s0, s1, s2};
        const double d = B.diag[i];
        double rk[3];
        double rs = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int k = c * np + i;
            const double bk = B.b[k];
            rk[c] = bk;
            if (from_x)
                rk[c] = bk - (d * B.x[k] - P.alpha * s[c]);
            else
                B.x[k] = 0.0;
            bb += bk * bk;
            rs += rk[c] * rk[c];
        }
        B.r4[i] = f4((float)rk[0], (float)rk[1], (float)rk[2]);
        B.p4[i] = f4(0.f, 0.f, 0.f);
        B.q4[i] = f4(0.f, 0.f, 0.f);
        B.d4[i] = f4(0.f, 0.f, 0.f);
        rr += rs;
        rz += (double)B.dinv32[i] * rs;
    }
    SS_ROW_LOOP_END
    const double v[3] = {bb, rr, rz};
    if (publish_partials<3>(v, B.partials, &st->ticket[0])) {
        double out[3];
        reduce_partials<3>(B.partials, out);
        if (threadIdx.x == 0) {
            st->bnorm2 = out[0];
            st->rr = out[1];
            st->rr_restart = out[1];
            st->rho = out[2];
            st->beta = 0.0;
            st->iter = 0;
            st->restarts = 0;
            st->check_true = 0;
            st->status = 0;
            st->zero_b = 0;
            st->done = 0;
            if (!isfinite(out[0]) || !isfinite(out[1])) {
                st->status = SP_ERR_NONFINITE;
                st->error = SP_ERR_NONFINITE;
                st->done = 1;
            } else if (out[0] == 0.0) {
                st->zero_b = 1;
                st->done = 1;
                st->last_res = 0.0;
            } else if (out[1] <= P.tol2 * out[0]) {
                st->done = 1;
                st->last_res = sqrt(out[1] / out[0]);
            }
        }
    }
}

// FP32: z = D^-1 r gathered on the fly; q = A z + beta q; p = z + beta p; p.q in FP64.
template <int T>
__global__ void __launch_bounds__(kSpmvBlock) k32_spmv(KParams P, DevBuffers B)
{
    DevState* st = B.st;
    if (halted(st)) return;
    const float beta = (float)st->beta;
    const float alpha_e = (float)P.alpha;
    double pq = 0.0;
    SS_ROW_LOOP_BEGIN(T)
    float s0, s1, s2;
    row_sum32_z<T>(B.row_ptr, B.col, B.val32, B.r4, B.dinv32, i, active, lane, s0, s1, s2);
    if (active && lane == 0) {
        const float di = B.dinv32[i], d = B.diag32[i];
        const float4 ri = B.r4[i];
        const float z0 = di * ri.x, z1 = di * ri.y, z2 = di * ri.z;
        float q0 = fmaf(d, z0, -alpha_e * s0);
        float q1 = fmaf(d, z1, -alpha_e * s1);
        float q2 = fmaf(d, z2, -alpha_e * s2);
        float p0 = z0, p1 = z1, p2 = z2;
        if (beta != 0.f) {
            const float4 qo = B.q4[i], po = B.p4[i];
            q0 = fmaf(beta, qo.x, q0);
            q1 = fmaf(beta, qo.y, q1);
            q2 = fmaf(beta, qo.z, q2);
            p0 = fmaf(beta, po.x, p0);
            p1 = fmaf(beta, po.y, p1);
            p2 = fmaf(beta, po.z, p2);
        }
        B.q4[i] = f4(q0, q1, q2);
        B.p4[i] = f4(p0, p1, p2);
        pq += (double)(p0 * q0 + p1 * q1 + p2 * q2);
    }
    SS_ROW_LOOP_END
    const double v[1] = {pq};
    if (publish_partials<1>(v, B.partials, &st->ticket[0])) {
        double out[1];
        reduce_partials<1>(B.partials, out);
        if (threadIdx.x == 0) {
            st->pq = out[0];
            if (!(out[0] > 0.0) || !isfinite(out[0])) {
                st->status = SP_ERR_NONFINITE;
                st->error = SP_ERR_NONFINITE;
                st->done = 1;
            } else {
                st->alpha = st->rho / out[0];
            }
        }
    }
}

// FP32: d += alpha p; r -= alpha q; r.r and r.z accumulated in FP64.
__global__ void __launch_bounds__(kVecBlock) k32_update(KParams P, DevBuffers B, CgLaunch C)
{
    DevState* st = B.st;
    if (halted(st)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            set_cond(C, C.h_check, 0u);
            set_cond(C, C.h_loop, 0u);
        }
        return;
    }
    const float a = (float)st->alpha;
    double rr = 0.0, rz = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const float4 p = B.p4[i], q = B.q4[i];
        float4 d = B.d4[i], r = B.r4[i];
        d.x = fmaf(a, p.x, d.x);
        d.y = fmaf(a, p.y, d.y);
        d.z = fmaf(a, p.z, d.z);
        r.x = fmaf(-a, q.x, r.x);
        r.y = fmaf(-a, q.y, r.y);
        r.z = fmaf(-a, q.z, r.z);
        B.d4[i] = d;
        B.r4[i] = r;
        const float rs = r.x * r.x + r.y * r.y + r.z * r.z;
        rr += (double)rs;
        rz += (double)(B.dinv32[i] * rs);
    }
    const double v[2] = {rr, rz};
    if (publish_partials<2>(v, B.partials, &st->ticket[0])) {
        double out[2];
        reduce_partials<2>(B.partials, out);
        if (threadIdx.x == 0) {
            // stop the FP32 inner solve once the residual dropped by the inner
            // factor since the last restart, or meets half the tolerance
            const double target = fmax(P.inner2 * st->rr_restart, 0.25 * P.tol2 * st->bnorm2);
            update_scalars(P, st, out[0], out[1], target, C);
        }
    }
}

// x += d; d = 0 (FP64 accumulation of the FP32 correction).
__global__ void __launch_bounds__(kVecBlock) k32_fold(KParams P, DevBuffers B, int always)
{
    const DevState* st = B.st;
    if (halted(st) || (!always && !st->check_true)) return;
    const int np = P.npad;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const float4 d = B.d4[i];
        B.x[i] += (double)d.x;
        B.x[np + i] += (double)d.y;
        B.x[2 * np + i] += (double)d.z;
        B.d4[i] = f4(0.f, 0.f, 0.f);
    }
}

// r = b - A x with the FP64 matrix; r4 = fp32(r); r.r in FP64, r.z with the FP32 diagonal.
template <int T>
__global__ void __launch_bounds__(kSpmvBlock) k32_true_residual(KParams P, DevBuffers B, int always,
                                                                CgLaunch C)
{
    DevState* st = B.st;
    if (halted(st) || (!always && !st->check_true)) return;
    const int np = P.npad;
    double rr = 0.0, rz = 0.0;
    SS_ROW_LOOP_BEGIN(T)
    double s0, s1, s2;
    row_sum64<T>(B.row_ptr, B.col, B.val, B.x, np, i, active, lane, s0, s1, s2);
    if (active && lane == 0) {
        const double s[3] = {s0, s1, s2};
        const double d = B.diag[i];
        double rk[3];
        double rs = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int k = c * np + i;
            rk[c] = B.b[k] - (d * B.x[k] - P.alpha * s[c]);
            rs += rk[c] * rk[c];
        }
        B.r4[i] = f4((float)rk[0], (float)rk[1], (float)rk[2]);
        rr += rs;
        rz += (double)B.dinv32[i] * rs;
    }
    SS_ROW_LOOP_END
    const double v[2] = {rr, rz};
    if (publish_partials<2>(v, B.partials, &st->ticket[0])) {
        double out[2];
        reduce_partials<2>(B.partials, out);
        if (threadIdx.x == 0) true_residual_scalars(P, st, out[0], out[1], C);
    }
}

// ================================================================== common

// After the loop: v = 0 when b = 0, and the per-call statistics.
__global__ void k_cg_finish(KParams P, DevBuffers B)
{
    DevState* st = B.st;
    if (st->error | st->overflow) return;
    if (st->zero_b) {
        for (int k = threadIdx.x; k < 3 * P.npad; k += blockDim.x) B.x[k] = 0.0;
    }
    if (threadIdx.x == 0) {
        st->iter_sum += st->iter;
        if (st->iter > st->iter_max) st->iter_max = st->iter;
    }
}

// ------------------------------------------------------------------ launchers

constexpr int kLanes64 = 2;   // FP64: few lanes per row keep the FP64 shuffle-adds low
constexpr int kLanes32 = 4;

static int spmv_grid(const KParams& P, int T, Launch L)
{
    return grid_for((long long)P.n * T, kSpmvBlock, L.num_sms * 8);
}

static int vec_grid(const KParams& P, Launch L)
{
    return grid_for(P.n, kVecBlock, L.num_sms * 8);
}

void launch_cg_init(const KParams& P, DevBuffers& B, bool from_x, bool mixed, Launch L)
{
    if (mixed)
        k32_init<kLanes64><<<spmv_grid(P, kLanes64, L), kSpmvBlock, 0, L.stream>>>(P, B, from_x ? 1 : 0);
    else
        k64_init<kLanes64><<<spmv_grid(P, kLanes64, L), kSpmvBlock, 0, L.stream>>>(P, B, from_x ? 1 : 0);
}

void launch_cg_spmv(const KParams& P, DevBuffers& B, bool mixed, Launch L)
{
    if (mixed)
        k32_spmv<kLanes32><<<spmv_grid(P, kLanes32, L), kSpmvBlock, 0, L.stream>>>(P, B);
    else
        k64_spmv<kLanes64><<<spmv_grid(P, kLanes64, L), kSpmvBlock, 0, L.stream>>>(P, B);
}

void launch_cg_update(const KParams& P, DevBuffers& B, bool mixed, const CgLaunch& C, Launch L)
{
    if (mixed)
        k32_update<<<vec_grid(P, L), kVecBlock, 0, L.stream>>>(P, B, C);
    else
        k64_update<<<vec_grid(P, L), kVecBlock, 0, L.stream>>>(P, B, C);
}

void launch_cg_true_residual(const KParams& P, DevBuffers& B, bool mixed, bool always_check,
                             const CgLaunch& C, Launch L)
{
    if (mixed) {
        k32_fold<<<vec_grid(P, L), kVecBlock, 0, L.stream>>>(P, B, always_check ? 1 : 0);
        k32_true_residual<kLanes64><<<spmv_grid(P, kLanes64, L), kSpmvBlock, 0, L.stream>>>(
            P, B, always_check ? 1 : 0, C);
    } else {
        k64_true_residual<kLanes64><<<spmv_grid(P, kLanes64, L), kSpmvBlock, 0, L.stream>>>(
            P, B, always_check ? 1 : 0, C);
    }
}

void launch_cg_finish(const KParams& P, DevBuffers& B, bool mixed, Launch L)
{
    (void)mixed;
    k_cg_finish<<<1, 256, 0, L.stream>>>(P, B);
}

int cg_kernels_per_iteration(bool mixed)
{
    (void)mixed;
    return 2;
}

int cg_kernels_per_check(bool mixed)
{
    return mixed ? 2 : 1;
}

}  // namespace ss
