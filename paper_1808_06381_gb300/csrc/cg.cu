// Jacobi-preconditioned conjugate gradients for Eq. algebra (arXiv 1808.06381,
// §Method: "use a sparse matrix solver"), on the GPU without host round trips.
//
// The three Cartesian components share one scalar matrix A = D - alpha W
// (D = diag, W = the truncated weights), so CG runs on (A (x) I_3) v = b and
// every step length is shared by the three components.  All scalars (rho,
// alpha, beta, norms) stay in device memory; each kernel's last block to
// finish reduces the per-block partial sums in a fixed order, so results are
// deterministic and no block ever waits for another.  Inside a CUDA graph the
// iteration loop is a conditional WHILE node and the true-residual check an IF
// node; the kernels set both conditions.
//
// Per iteration: spmv  q = A p, partial p.q, last block: alpha = rho / p.q
//                update x += alpha p, r -= alpha q, partial r.r and r.D^-1 r,
//                       last block: beta, convergence test
//                [true residual r = b - A x when the recurrence says converged]
//                direction p = D^-1 r + beta p
#include <math.h>

#include "internal.cuh"

namespace ss {

constexpr int kSpmvBlock = 256;

// Off-diagonal sum s_a = sum_j w_ij v_a[j] over row i for the three planes,
// T lanes per row, reduced across the lanes with shuffles (all T lanes of the
// group end up with the sum).
template <int T>
__device__ __forceinline__ void row_weighted_sum(const int* __restrict__ row_ptr,
                                                 const int* __restrict__ col,
                                                 const double* __restrict__ val,
                                                 const double* __restrict__ v, int np, int i,
                                                 bool active, int lane, double& s0, double& s1,
                                                 double& s2)
{
    s0 = s1 = s2 = 0.0;
    if (active) {
        const int beg = row_ptr[i], end = row_ptr[i + 1];
        for (int k = beg + lane; k < end; k += T) {
            const int j = col[k];
            const double w = val[k];
            s0 += w * v[j];
            s1 += w * v[np + j];
            s2 += w * v[2 * np + j];
        }
    }
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o, T);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o, T);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o, T);
    }
}

__device__ __forceinline__ bool halted(const DevState* st)
{
    return (st->error | st->overflow | st->done) != 0;
}

// Rows handled by one warp-uniform loop: group g of T lanes takes rows
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

// r = b - A x0 (or r = b, x = 0 for a cold start); p = D^-1 r; partial
// b.b, r.r, r.D^-1 r.  Last block: initial scalars and the early exit when x0
// already meets the tolerance.
template <int T>
__global__ void __launch_bounds__(kSpmvBlock) k_cg_init(KParams P, DevBuffers B, int from_x)
{
    DevState* st = B.st;
    if (st->error | st->overflow) return;
    const int np = P.npad;
    double bb = 0.0, rr = 0.0, rz = 0.0;
    SS_ROW_LOOP_BEGIN(T)
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    if (from_x) row_weighted_sum<T>(B.row_ptr, B.col, B.val, B.x, np, i, active, lane, s0, s1, s2);
    if (active && lane == 0) {
        const double b0 = B.b[i], b1 = B.b[np + i], b2 = B.b[2 * np + i];
        double r0 = b0, r1 = b1, r2 = b2;
        if (from_x) {
            const double d = B.diag[i];
            r0 = b0 - (d * B.x[i] - P.alpha * s0);
            r1 = b1 - (d * B.x[np + i] - P.alpha * s1);
            r2 = b2 - (d * B.x[2 * np + i] - P.alpha * s2);
        } else {
            B.x[i] = 0.0;
            B.x[np + i] = 0.0;
            B.x[2 * np + i] = 0.0;
        }
        const double di = B.dinv[i];
        B.r[i] = r0;
        B.r[np + i] = r1;
        B.r[2 * np + i] = r2;
        B.p[i] = di * r0;
        B.p[np + i] = di * r1;
        B.p[2 * np + i] = di * r2;
        bb += b0 * b0 + b1 * b1 + b2 * b2;
        const double rs = r0 * r0 + r1 * r1 + r2 * r2;
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
            st->rho = out[2];
            st->beta = 0.0;
            st->iter = 0;
            st->restarts = 0;
            st->check_true = 0;
            st->status = 0;
            st->zero_b = 0;
            st->done = 0;
            st->since_replace = 0;
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

// q = A p and p.q; last block: alpha = rho / p.q.
template <int T>
__global__ void __launch_bounds__(kSpmvBlock) k_cg_spmv(KParams P, DevBuffers B)
{
    DevState* st = B.st;
    if (halted(st)) return;
    const int np = P.npad;
    double pq = 0.0;
    SS_ROW_LOOP_BEGIN(T)
    double s0, s1, s2;
    row_weighted_sum<T>(B.row_ptr, B.col, B.val, B.p, np, i, active, lane, s0, s1, s2);
    if (active && lane == 0) {
        const double d = B.diag[i];
        const double p0 = B.p[i], p1 = B.p[np + i], p2 = B.p[2 * np + i];
        const double q0 = d * p0 - P.alpha * s0;
        const double q1 = d * p1 - P.alpha * s1;
        const double q2 = d * p2 - P.alpha * s2;
        B.q[i] = q0;
        B.q[np + i] = q1;
        B.q[2 * np + i] = q2;
        pq += p0 * q0 + p1 * q1 + p2 * q2;
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

// x += alpha p; r -= alpha q; partial r.r and r.D^-1 r.  Last block: beta and
// the convergence test on the recurrence residual, which arms the
// true-residual check.
__global__ void __launch_bounds__(kVecBlock) k_cg_update(KParams P, DevBuffers B, CgLaunch C)
{
    DevState* st = B.st;
    if (halted(st)) {
        if (C.use_cond && blockIdx.x == 0 && threadIdx.x == 0)
            cudaGraphSetConditional((cudaGraphConditionalHandle)C.h_check, 0u);
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
            rs += rk * rk;
        }
        rr += rs;
        rz += di * rs;
    }
    const double v[2] = {rr, rz};
    if (publish_partials<2>(v, B.partials, &st->ticket[0])) {
        double out[2];
        reduce_partials<2>(B.partials, out);
        if (threadIdx.x == 0) {
            st->iter += 1;
            st->rr = out[0];
            st->beta = out[1] / st->rho;
            st->rho = out[1];
            if (!isfinite(out[0]) || !isfinite(out[1])) {
                st->status = SP_ERR_NONFINITE;
                st->error = SP_ERR_NONFINITE;
                st->done = 1;
            } else if (st->iter >= P.max_iter + kMaxCgRestarts + 4) {
                // the true-residual check should have ended the solve by now
                st->status = SP_ERR_NOT_CONVERGED;
                st->error = SP_ERR_NOT_CONVERGED;
                st->done = 1;
            } else if (out[0] <= P.tol2 * st->bnorm2 || st->iter >= P.max_iter) {
                st->check_true = 1;
            }
            if (C.use_cond)
                cudaGraphSetConditional((cudaGraphConditionalHandle)C.h_check,
                                        (unsigned)(st->check_true && !st->done));
        }
    }
}

// r = b - A x in FP64 with partial r.r and r.D^-1 r.  Last block: accept
// (done), or restart the recurrence from the true residual (beta = 0), or
// give up at the iteration cap.
template <int T>
__global__ void __launch_bounds__(kSpmvBlock) k_cg_true_residual(KParams P, DevBuffers B, int always)
{
    DevState* st = B.st;
    if (halted(st)) return;
    if (!always && !st->check_true) return;
    const int np = P.npad;
    double rr = 0.0, rz = 0.0;
    SS_ROW_LOOP_BEGIN(T)
    double s0, s1, s2;
    row_weighted_sum<T>(B.row_ptr, B.col, B.val, B.x, np, i, active, lane, s0, s1, s2);
    if (active && lane == 0) {
        const double d = B.diag[i];
        const double r0 = B.b[i] - (d * B.x[i] - P.alpha * s0);
        const double r1 = B.b[np + i] - (d * B.x[np + i] - P.alpha * s1);
        const double r2 = B.b[2 * np + i] - (d * B.x[2 * np + i] - P.alpha * s2);
        B.r[i] = r0;
        B.r[np + i] = r1;
        B.r[2 * np + i] = r2;
        const double rs = r0 * r0 + r1 * r1 + r2 * r2;
        rr += rs;
        rz += B.dinv[i] * rs;
    }
    SS_ROW_LOOP_END
    const double v[2] = {rr, rz};
    if (publish_partials<2>(v, B.partials, &st->ticket[0])) {
        double out[2];
        reduce_partials<2>(B.partials, out);
        if (threadIdx.x == 0) {
            st->check_true = 0;
            st->true_checks += 1;
            st->rr_true = out[0];
            st->last_res = sqrt(out[0] / st->bnorm2);
            if (!isfinite(out[0])) {
                st->status = SP_ERR_NONFINITE;
                st->error = SP_ERR_NONFINITE;
                st->done = 1;
            } else if (out[0] <= P.tol2 * st->bnorm2) {
                st->done = 1;
                st->status = SP_OK;
            } else if (st->iter >= P.max_iter || st->restarts >= kMaxCgRestarts) {
                st->done = 1;
                st->status = SP_ERR_NOT_CONVERGED;
                st->error = SP_ERR_NOT_CONVERGED;
            } else {
                st->restarts += 1;
                st->rho = out[1];
                st->beta = 0.0;
                st->rr = out[0];
            }
        }
    }
}

// p = D^-1 r + beta p; one thread then tells the WHILE node whether to go on.
__global__ void __launch_bounds__(kVecBlock) k_cg_direction(KParams P, DevBuffers B, CgLaunch C)
{
    DevState* st = B.st;
    const bool stop = halted(st) || st->iter > P.max_iter + kMaxCgRestarts + 8;
    if (!stop) {
        const int np = P.npad;
        const double beta = st->beta;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
            const double di = B.dinv[i];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int k = c * np + i;
                B.p[k] = di * B.r[k] + beta * B.p[k];
            }
        }
    }
    if (C.use_cond && blockIdx.x == 0 && threadIdx.x == 0)
        cudaGraphSetConditional((cudaGraphConditionalHandle)C.h_loop, stop ? 0u : 1u);
}

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

static int spmv_grid(const KParams& P, int T, Launch L)
{
    return grid_for(P.n, kSpmvBlock / T, L.num_sms * 8);
}

static int vec_grid(const KParams& P, Launch L)
{
    return grid_for(P.n, kVecBlock, L.num_sms * 8);
}

constexpr int kRowLanes = 4;

void launch_cg_init(const KParams& P, DevBuffers& B, bool from_x, bool mixed, Launch L)
{
    (void)mixed;
    k_cg_init<kRowLanes><<<spmv_grid(P, kRowLanes, L), kSpmvBlock, 0, L.stream>>>(P, B, from_x ? 1 : 0);
}

void launch_cg_spmv(const KParams& P, DevBuffers& B, bool mixed, Launch L)
{
    (void)mixed;
    k_cg_spmv<kRowLanes><<<spmv_grid(P, kRowLanes, L), kSpmvBlock, 0, L.stream>>>(P, B);
}

void launch_cg_update(const KParams& P, DevBuffers& B, bool mixed, const CgLaunch& C, Launch L)
{
    (void)mixed;
    k_cg_update<<<vec_grid(P, L), kVecBlock, 0, L.stream>>>(P, B, C);
}

void launch_cg_iteration_head(const KParams& P, DevBuffers& B, bool mixed, const CgLaunch& C,
                              Launch L)
{
    launch_cg_spmv(P, B, mixed, L);
    launch_cg_update(P, B, mixed, C, L);
}

void launch_cg_true_residual(const KParams& P, DevBuffers& B, bool mixed, bool always_check,
                             Launch L)
{
    (void)mixed;
    k_cg_true_residual<kRowLanes><<<spmv_grid(P, kRowLanes, L), kSpmvBlock, 0, L.stream>>>(
        P, B, always_check ? 1 : 0);
}

void launch_cg_iteration_tail(const KParams& P, DevBuffers& B, bool mixed, const CgLaunch& C,
                              Launch L)
{
    (void)mixed;
    k_cg_direction<<<vec_grid(P, L), kVecBlock, 0, L.stream>>>(P, B, C);
}

void launch_cg_finish(const KParams& P, DevBuffers& B, Launch L)
{
    k_cg_finish<<<1, 256, 0, L.stream>>>(P, B);
}

int cg_kernels_per_iteration(bool mixed)
{
    (void)mixed;
    return 3;
}

}  // namespace ss
