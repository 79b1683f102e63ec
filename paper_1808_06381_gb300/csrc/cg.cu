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
// The matrix is stored sliced (SELL-32-sigma256, see internal.cuh): one thread
// owns one row, a warp owns a chunk of 32 rows of nearly equal length, and
// entry k of the whole chunk is one coalesced 128-byte load of columns and of
// weights; the gathers of several entries are independent and issued together.
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
// Mixed solver: the matrix values and the vectors r, p, q, d are FP32, one
// float4 per row (r.w carries the Jacobi scale D^-1, so one 16-byte gather
// brings z_j); the iteration solves for a correction d of the FP64 solution x;
// dot products accumulate in double-float (FP32 pairs, ~44 bits).  When the
// FP32 residual has dropped by the inner factor, or meets the tolerance, d is
// folded into x and the true residual b - A x is recomputed with the FP64
// matrix; the solve ends when that meets the tolerance, else the iteration
// restarts from it (residual replacement).
//
// Inside a CUDA graph the loop is a conditional WHILE node and the
// true-residual check an IF node; the kernels set both conditions.
#include <math.h>

#include <mutex>

#include "internal.cuh"

namespace ss {

constexpr int kBlock = 256;

__device__ __forceinline__ bool halted(const DevState* st)
{
    return (st->error | st->overflow | st->done) != 0;
}

__device__ __forceinline__ void set_cond(const CgLaunch& C, unsigned long long h, unsigned v)
{
    if (C.use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)h, v);
}

// Slots handled by a grid-stride loop; nslots is a multiple of the block size,
// so every warp sees whole chunks.
#define SS_SLOT_LOOP_BEGIN                                                                       \
    for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < P.nslots;                      \
         slot += gridDim.x * blockDim.x) {                                                       \
        const int row = B.slot_row[slot];                                                        \
        const int e0 = B.chunk_off[slot >> 5] + (slot & 31);                                     \
        const int e1 = B.chunk_off[(slot >> 5) + 1];

#define SS_SLOT_LOOP_END }

// Entries of one row are processed in batches of kBatch: all column and weight
// loads of a batch are issued first, then all gathers, so one row waits for
// two memory latencies per batch instead of two per entry.  The batch count
// (the chunk's longest row / kBatch) is uniform across the warp; entries past
// the row's own length are padding (weight 0) and load nothing.
constexpr int kBatch = 6;

// s_a = sum_j w_ij v_a[j] over the entries of one row (FP64 planes).
__device__ __forceinline__ void row_sum64(const int* __restrict__ col, const double* __restrict__ val,
                                          const double* __restrict__ v, int np, int e0, int e1, bool active,
                                          double& s0, double& s1, double& s2)
{
    s0 = s1 = s2 = 0.0;
    for (int eb = e0; eb < e1; eb += 32 * kBatch) {
        int j[kBatch];
        double w[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int e = eb + 32 * u;
            j[u] = 0;
            w[u] = 0.0;
            if (active && e < e1) {
                j[u] = col[e];
                w[u] = val[e];
            }
        }
        double g0[kBatch], g1[kBatch], g2[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            g0[u] = g1[u] = g2[u] = 0.0;
            if (w[u] != 0.0) {
                g0[u] = v[j[u]];
                g1[u] = v[np + j[u]];
                g2[u] = v[2 * np + j[u]];
            }
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            s0 += w[u] * g0[u];
            s1 += w[u] * g1[u];
            s2 += w[u] * g2[u];
        }
    }
}

// s = sum_j w_ij D^-1_j r_j over the entries of one row (FP32; r.w = D^-1).
__device__ __forceinline__ void row_sum32_z(const int* __restrict__ col, const float* __restrict__ val,
                                            const float4* __restrict__ r, int e0, int e1, bool active,
                                            float& s0, float& s1, float& s2)
{
    s0 = s1 = s2 = 0.f;
    for (int eb = e0; eb < e1; eb += 32 * kBatch) {
        int j[kBatch];
        float w[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int e = eb + 32 * u;
            j[u] = 0;
            w[u] = 0.f;
            if (active && e < e1) {
                j[u] = col[e];
                w[u] = val[e];
            }
        }
        float4 g[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            g[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (w[u] != 0.f) g[u] = r[j[u]];
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const float ww = w[u] * g[u].w;
            s0 = fmaf(ww, g[u].x, s0);
            s1 = fmaf(ww, g[u].y, s1);
            s2 = fmaf(ww, g[u].z, s2);
        }
    }
}

__device__ __forceinline__ void init_scalars(const KParams& P, DevState* st, double bb, double rr, double rz)
{
    st->bnorm2 = bb;
    st->rr = rr;
    st->rr_restart = rr;
    st->rho = rz;
    st->beta = 0.0;
    st->iter = 0;
    st->restarts = 0;
    st->check_true = 0;
    st->status = 0;
    st->zero_b = 0;
    st->done = 0;
    st->res_offchip = 0;
    if (!isfinite(bb) || !isfinite(rr)) {
        st->status = SP_ERR_NONFINITE;
        st->error = SP_ERR_NONFINITE;
        st->done = 1;
    } else if (bb == 0.0) {
        st->zero_b = 1;   // b = 0: the solution is v = 0
        st->done = 1;
        st->last_res = 0.0;
    } else if (rr <= P.tol2 * bb) {
        st->done = 1;     // the start vector already meets the tolerance (exact r)
        st->last_res = sqrt(rr / bb);
    }
}

__device__ __forceinline__ void alpha_from_pq(DevState* st, double pq)
{
    st->pq = pq;
    if (!(pq > 0.0) || !isfinite(pq)) {
        st->status = SP_ERR_NONFINITE;
        st->error = SP_ERR_NONFINITE;
        st->done = 1;
    } else {
        st->alpha = st->rho / pq;
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

// ============================================================== FP64 solver

// r = b - A x0 (or r = b and x = 0); z = D^-1 r; p = q = 0.
__global__ void __launch_bounds__(kBlock) k64_init(KParams P, DevBuffers B, int from_x)
{
    DevState* st = B.st;
    if (st->error | st->overflow) return;
    const int np = P.npad;
    double bb = 0.0, rr = 0.0, rz = 0.0;
    SS_SLOT_LOOP_BEGIN
    if (row >= 0) {
        double s[3] = {0.0, 0.0, 0.0};
        if (from_x) row_sum64(B.col, B.val, B.x, np, e0, e1, true, s[0], s[1], s[2]);
        const double d = B.diag[row], di = B.dinv[row];
        double rs = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int k = c * np + row;
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
    SS_SLOT_LOOP_END
    const double v[3] = {bb, rr, rz};
    if (publish_partials<3>(v, B.partials, &st->ticket[0])) {
        double out[3];
        reduce_partials<3>(B.partials, out);
        if (threadIdx.x == 0) init_scalars(P, st, out[0], out[1], out[2]);
    }
}

// q = A z + beta q; p = z + beta p; p.q.  Last block: alpha = rho / p.q.
__global__ void __launch_bounds__(kBlock) k64_spmv(KParams P, DevBuffers B, int probe)
{
    DevState* st = B.st;
    if (!probe && halted(st)) return;
    const int np = P.npad;
    const double beta = st->beta;
    double pq = 0.0;
    SS_SLOT_LOOP_BEGIN
    if (row >= 0) {
        double s[3];
        row_sum64(B.col, B.val, B.z, np, e0, e1, true, s[0], s[1], s[2]);
        const double d = B.diag[row];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int k = c * np + row;
            const double zk = B.z[k];
            const double az = d * zk - P.alpha * s[c];
            const double qk = beta == 0.0 ? az : az + beta * B.q[k];
            const double pk = beta == 0.0 ? zk : zk + beta * B.p[k];
            B.q[k] = qk;
            B.p[k] = pk;
            pq += pk * qk;
        }
    }
    SS_SLOT_LOOP_END
    const double v[1] = {pq};
    if (publish_partials<1>(v, B.partials, &st->ticket[0])) {
        double out[1];
        reduce_partials<1>(B.partials, out);
        if (threadIdx.x == 0 && !probe) alpha_from_pq(st, out[0]);
    }
}

// x += alpha p; r -= alpha q; z = D^-1 r; partial r.r and r.z.
__global__ void __launch_bounds__(kBlock) k64_update(KParams P, DevBuffers B, CgLaunch C, int probe)
{
    DevState* st = B.st;
    if (!probe && halted(st)) {
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
        if (threadIdx.x == 0 && !probe) update_scalars(P, st, out[0], out[1], P.tol2 * st->bnorm2, C);
    }
}

// r = b - A x in FP64; z = D^-1 r; partial r.r and r.z.
__global__ void __launch_bounds__(kBlock) k64_true_residual(KParams P, DevBuffers B, int always, CgLaunch C)
{
    DevState* st = B.st;
    if (halted(st) || (!always && !st->check_true)) return;
    const int np = P.npad;
    double rr = 0.0, rz = 0.0;
    SS_SLOT_LOOP_BEGIN
    if (row >= 0) {
        double s[3];
        row_sum64(B.col, B.val, B.x, np, e0, e1, true, s[0], s[1], s[2]);
        const double d = B.diag[row], di = B.dinv[row];
        double rs = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int k = c * np + row;
            const double rk = B.b[k] - (d * B.x[k] - P.alpha * s[c]);
            B.r[k] = rk;
            B.z[k] = di * rk;
            rs += rk * rk;
        }
        rr += rs;
        rz += di * rs;
    }
    SS_SLOT_LOOP_END
    const double v[2] = {rr, rz};
    if (publish_partials<2>(v, B.partials, &st->ticket[0])) {
        double out[2];
        reduce_partials<2>(B.partials, out);
        if (threadIdx.x == 0) true_residual_scalars(P, st, out[0], out[1], C);
    }
}

// ============================================================= mixed solver

__device__ __forceinline__ float4 f4(float x, float y, float z, float w) { return make_float4(x, y, z, w); }

// x0 (FP64 planes) as the double-float records xdf of the mixed solver.
__global__ void __launch_bounds__(kBlock) k32_split_x(KParams P, DevBuffers B)
{
    if (B.st->error | B.st->overflow) return;
    const int np = P.npad;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const dfloat a = df_split(B.x[i]), b = df_split(B.x[np + i]), c = df_split(B.x[2 * np + i]);
        B.xdf[2 * i] = f4(a.hi, b.hi, c.hi, 0.f);
        B.xdf[2 * i + 1] = f4(a.lo, b.lo, c.lo, 0.f);
    }
}

// r = b - A x0 in double-float from the double-float matrix, b and x0 (or
// r = b and x = 0); r4 = (fp32(r), D^-1); d = p = q = 0.  ||b||^2 from the
// high parts of b (FP32 squares summed in FP64: the relative tolerance needs
// a few digits of it).
__global__ void __launch_bounds__(kBlock) k32_init(KParams P, DevBuffers B, int from_x)
{
    DevState* st = B.st;
    if (st->error | st->overflow) return;
    const int np = P.npad;
    double bb = 0.0, rr = 0.0, rz = 0.0;
    SS_SLOT_LOOP_BEGIN
    if (row >= 0) {
        dfloat r[3];
        if (from_x) {
            dfloat s[3];
            row_sum_df<8>(B.col, B.val32, B.val32lo, B.xdf, e0, e1, s);
            residual_df(P, B, row, s, r);
        } else {
            const float4 bh = B.bdf[2 * row], bl = B.bdf[2 * row + 1];
            r[0] = dfloat{bh.x, bl.x};
            r[1] = dfloat{bh.y, bl.y};
            r[2] = dfloat{bh.z, bl.z};
            B.xdf[2 * row] = f4(0.f, 0.f, 0.f, 0.f);
            B.xdf[2 * row + 1] = f4(0.f, 0.f, 0.f, 0.f);
        }
        const float di = B.dinv32[row];
        const float4 bh = B.bdf[2 * row];
        bb += (double)(bh.x * bh.x + bh.y * bh.y + bh.z * bh.z);
        if (!from_x) {
#pragma unroll
            for (int c = 0; c < 3; ++c) B.x[c * np + row] = 0.0;
        }
        const float rs = r[0].hi * r[0].hi + r[1].hi * r[1].hi + r[2].hi * r[2].hi;
        B.r4[row] = f4(r[0].hi, r[1].hi, r[2].hi, di);
        B.rdf[2 * row] = f4(r[0].hi, r[1].hi, r[2].hi, 0.f);
        B.rdf[2 * row + 1] = f4(r[0].lo, r[1].lo, r[2].lo, 0.f);
        B.p4[row] = f4(0.f, 0.f, 0.f, 0.f);
        B.q4[row] = f4(0.f, 0.f, 0.f, 0.f);
        B.d4[row] = f4(0.f, 0.f, 0.f, 0.f);
        rr += (double)rs;
        rz += (double)(di * rs);
    }
    SS_SLOT_LOOP_END
    const double v[3] = {bb, rr, rz};
    if (publish_partials<3>(v, B.partials, &st->ticket[0])) {
        double out[3];
        reduce_partials<3>(B.partials, out);
        if (threadIdx.x == 0) init_scalars(P, st, out[0], out[1], out[2]);
    }
}

// FP32: z_j = D^-1_j r_j gathered from r4; q = A z + beta q; p = z + beta p;
// p.q in double-float.
__global__ void __launch_bounds__(kBlock, 6) k32_spmv(KParams P, DevBuffers B, int probe)
{
    DevState* st = B.st;
    if (!probe && halted(st)) return;
    const float beta = (float)st->beta;
    const float alpha_e = (float)P.alpha;
    const int* __restrict__ col = B.col;
    const float* __restrict__ val = B.val32;
    const float4* __restrict__ r4 = B.r4;
    dfloat pq{0.f, 0.f};
    SS_SLOT_LOOP_BEGIN
    if (row >= 0) {
        float s0, s1, s2;
        row_sum32_z(col, val, r4, e0, e1, true, s0, s1, s2);
        const float4 ri = r4[row];
        const float d = B.diag32[row];
        const float z0 = ri.w * ri.x, z1 = ri.w * ri.y, z2 = ri.w * ri.z;
        float q0 = fmaf(d, z0, -alpha_e * s0);
        float q1 = fmaf(d, z1, -alpha_e * s1);
        float q2 = fmaf(d, z2, -alpha_e * s2);
        float p0 = z0, p1 = z1, p2 = z2;
        if (beta != 0.f) {
            const float4 qo = B.q4[row], po = B.p4[row];
            q0 = fmaf(beta, qo.x, q0);
            q1 = fmaf(beta, qo.y, q1);
            q2 = fmaf(beta, qo.z, q2);
            p0 = fmaf(beta, po.x, p0);
            p1 = fmaf(beta, po.y, p1);
            p2 = fmaf(beta, po.z, p2);
        }
        B.q4[row] = f4(q0, q1, q2, 0.f);
        B.p4[row] = f4(p0, p1, p2, 0.f);
        pq = df_add(pq, p0 * q0 + p1 * q1 + p2 * q2);
    }
    SS_SLOT_LOOP_END
    dfloat v[1] = {pq};
    double out[1];
    if (publish_reduce_df<1>(v, B.partials_df, &st->ticket[0], out) && threadIdx.x == 0 && !probe)
        alpha_from_pq(st, out[0]);
}

// FP32: d += alpha p; r -= alpha q; r.r and r.z in double-float.
__global__ void __launch_bounds__(kBlock) k32_update(KParams P, DevBuffers B, CgLaunch C, int probe)
{
    DevState* st = B.st;
    if (!probe && halted(st)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            set_cond(C, C.h_check, 0u);
            set_cond(C, C.h_loop, 0u);
        }
        return;
    }
    const float a = (float)st->alpha;
    dfloat rr{0.f, 0.f}, rz{0.f, 0.f};
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
        rr = df_add(rr, rs);
        rz = df_add(rz, r.w * rs);
    }
    dfloat v[2] = {rr, rz};
    double out[2];
    if (publish_reduce_df<2>(v, B.partials_df, &st->ticket[0], out) && threadIdx.x == 0 && !probe) {
        // stop the FP32 inner solve once the residual dropped by the inner
        // factor since the last restart, or meets half the tolerance
        const double target = fmax(P.inner2 * st->rr_restart, kInnerFinal2 * P.tol2 * st->bnorm2);
        update_scalars(P, st, out[0], out[1], target, C);
    }
}

// x += d; d = 0: the FP32 correction folded into the double-float x, and x
// also written in FP64 (the solution whenever the loop stops).
__global__ void __launch_bounds__(kBlock) k32_fold(KParams P, DevBuffers B, int always)
{
    const DevState* st = B.st;
    if (halted(st) || (!always && !st->check_true)) return;
    const int np = P.npad;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const float4 d = B.d4[i], xh = B.xdf[2 * i], xl = B.xdf[2 * i + 1];
        const dfloat a = df_add(dfloat{xh.x, xl.x}, d.x), b = df_add(dfloat{xh.y, xl.y}, d.y),
                     c = df_add(dfloat{xh.z, xl.z}, d.z);
        B.xdf[2 * i] = f4(a.hi, b.hi, c.hi, 0.f);
        B.xdf[2 * i + 1] = f4(a.lo, b.lo, c.lo, 0.f);
        B.x[i] = df_to_double(a);
        B.x[np + i] = df_to_double(b);
        B.x[2 * np + i] = df_to_double(c);
        B.d4[i] = f4(0.f, 0.f, 0.f, 0.f);
    }
}

// r = b - A x in double-float; r4 = (fp32(r), D^-1); r.r summed in FP64.
__global__ void __launch_bounds__(kBlock) k32_true_residual(KParams P, DevBuffers B, int always, CgLaunch C)
{
    DevState* st = B.st;
    if (halted(st) || (!always && !st->check_true)) return;
    double rr = 0.0, rz = 0.0;
    SS_SLOT_LOOP_BEGIN
    if (row >= 0) {
        dfloat s[3], r[3];
        row_sum_df<4>(B.col, B.val32, B.val32lo, B.xdf, e0, e1, s);
        residual_df(P, B, row, s, r);
        const float di = B.dinv32[row];
        const float rs = r[0].hi * r[0].hi + r[1].hi * r[1].hi + r[2].hi * r[2].hi;
        B.r4[row] = f4(r[0].hi, r[1].hi, r[2].hi, di);
        rr += (double)rs;
        rz += (double)(di * rs);
    }
    SS_SLOT_LOOP_END
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
        if (B.xdf)
            for (int k = threadIdx.x; k < 2 * P.npad; k += blockDim.x) B.xdf[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (threadIdx.x == 0) {
        st->iter_sum += st->iter;
        if (st->iter > st->iter_max) st->iter_max = st->iter;
    }
}

// ------------------------------------------------------------------ launchers

namespace {
// Resident blocks per SM of each kernel (computed once per process).
struct Occupancy {
    int k64_init, k64_spmv, k64_update, k64_true, k32_init, k32_spmv, k32_update, k32_fold, k32_true;
};
Occupancy g_occ;
std::once_flag g_occ_once;

int occ_of(const void* f)
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, kBlock, 0) != cudaSuccess || b < 1) {
        cudaGetLastError();
        b = 1;
    }
    return b;
}
}  // namespace

void cg_prepare()
{
    std::call_once(g_occ_once, [] {
        g_occ.k64_init = occ_of((const void*)k64_init);
        g_occ.k64_spmv = occ_of((const void*)k64_spmv);
        g_occ.k64_update = occ_of((const void*)k64_update);
        g_occ.k64_true = occ_of((const void*)k64_true_residual);
        g_occ.k32_init = occ_of((const void*)k32_init);
        g_occ.k32_spmv = occ_of((const void*)k32_spmv);
        g_occ.k32_update = occ_of((const void*)k32_update);
        g_occ.k32_fold = occ_of((const void*)k32_fold);
        g_occ.k32_true = occ_of((const void*)k32_true_residual);
    });
}

// One wave: at most (SMs x resident blocks), never more blocks than work.
static int wave_grid(long long threads, int occ, Launch L)
{
    long long g = (threads + kBlock - 1) / kBlock;
    const long long wave = (long long)L.num_sms * occ;
    if (g > wave) g = wave;
    if (g > kMaxPartials) g = kMaxPartials;
    return (int)(g < 1 ? 1 : g);
}

int launch_cg_init(const KParams& P, DevBuffers& B, bool from_x, bool mixed, Launch L)
{
    if (mixed) {
        if (from_x) k32_split_x<<<wave_grid(P.n, 8, L), kBlock, 0, L.stream>>>(P, B);
        k32_init<<<wave_grid(P.nslots, g_occ.k32_init, L), kBlock, 0, L.stream>>>(P, B, from_x ? 1 : 0);
        return from_x ? 2 : 1;
    }
    k64_init<<<wave_grid(P.nslots, g_occ.k64_init, L), kBlock, 0, L.stream>>>(P, B, from_x ? 1 : 0);
    return 1;
}

void launch_cg_split_x(const KParams& P, DevBuffers& B, Launch L)
{
    k32_split_x<<<wave_grid(P.n, 8, L), kBlock, 0, L.stream>>>(P, B);
}

void launch_cg_spmv(const KParams& P, DevBuffers& B, bool mixed, Launch L, int probe)
{
    if (mixed)
        k32_spmv<<<wave_grid(P.nslots, g_occ.k32_spmv, L), kBlock, 0, L.stream>>>(P, B, probe);
    else
        k64_spmv<<<wave_grid(P.nslots, g_occ.k64_spmv, L), kBlock, 0, L.stream>>>(P, B, probe);
}

void launch_cg_update(const KParams& P, DevBuffers& B, bool mixed, const CgLaunch& C, Launch L, int probe)
{
    if (mixed)
        k32_update<<<wave_grid(P.n, g_occ.k32_update, L), kBlock, 0, L.stream>>>(P, B, C, probe);
    else
        k64_update<<<wave_grid(P.n, g_occ.k64_update, L), kBlock, 0, L.stream>>>(P, B, C, probe);
}

void launch_cg_true_residual(const KParams& P, DevBuffers& B, bool mixed, bool always_check,
                             const CgLaunch& C, Launch L)
{
    if (mixed) {
        k32_fold<<<wave_grid(P.n, g_occ.k32_fold, L), kBlock, 0, L.stream>>>(P, B, always_check ? 1 : 0);
        k32_true_residual<<<wave_grid(P.nslots, g_occ.k32_true, L), kBlock, 0, L.stream>>>(
            P, B, always_check ? 1 : 0, C);
    } else {
        k64_true_residual<<<wave_grid(P.nslots, g_occ.k64_true, L), kBlock, 0, L.stream>>>(
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
