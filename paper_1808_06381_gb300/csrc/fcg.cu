// Flexible conjugate gradients with the learned network as a preconditioner.
//
// The solve of Eq. algebra (arXiv 1808.06381, §Method), A v = b with A = I +
// alpha L_w on each Cartesian component, by FCG(1) (Notay 2000: flexible CG
// that A-orthogonalises each new direction against the previous one only),
// in FP64.  The preconditioner may change from one iteration to the next:
// at iterations k with net_every > 0 and k % net_every == 0 it is the
// message-passing network of the learned warm start applied to the current
// residual (z = net(r), its vprev feature 0: the network maps a right-hand
// side to an approximate A^-1 of it, and a residual is a right-hand side of
// the error equation), otherwise Jacobi (z = D^-1 r).  Per iteration:
//   q = A p;  alpha = (p, r) / (p, q);  x += alpha p;  r -= alpha q;
//   z = M_k(r);  beta = -(z, q) / (p, q);  p = z + beta p.
// With Jacobi at every iteration this is Jacobi-PCG in exact arithmetic.  The
// scalars are formed on the device by the last block of each reducing kernel
// (partial sums in a fixed order); the host polls the state every 8
// iterations.  The stopping test is the recurrence residual ||r|| <= tol ||b||
// (2-norm over all 3n entries), followed by the true residual b - A x, which
// is what the solve reports.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "sim_impl.cuh"

namespace ss {

namespace {

// (A v)_i for FP64 planes v: A_ii v_i - alpha sum_j w_ij v_j over the sliced layout.
__device__ __forceinline__ void fcg_row_apply(const KParams& P, const DevBuffers& B, const double* __restrict__ v,
                                              int i, double (&out)[3])
{
    const int np = P.npad;
    const int slot = B.row_slot[i];
    const int base = B.chunk_off[slot >> 5] + (slot & 31);
    const int cnt = B.row_cnt[i];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int k = 0; k < cnt; ++k) {
        const int e = base + 32 * k;
        const int j = B.col[e];
        const double w = B.val[e];
        s0 = fma(w, v[j], s0);
        s1 = fma(w, v[np + j], s1);
        s2 = fma(w, v[2 * np + j], s2);
    }
    const double d = B.diag[i];
    out[0] = d * v[i] - P.alpha * s0;
    out[1] = d * v[np + i] - P.alpha * s1;
    out[2] = d * v[2 * np + i] - P.alpha * s2;
}

// r = b - A x; ||r||^2 (and ||b||^2 on the first call).  The last block sets
// the state: the start already meets the tolerance, or (final check) the true
// relative residual.
__global__ void k_fcg_residual(KParams P, DevBuffers B, FcgState* S, int first)
{
    const int np = P.npad;
    double v[2] = {0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        double ax[3];
        fcg_row_apply(P, B, B.x, i, ax);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double b = B.b[c * np + i];
            const double r = b - ax[c];
            B.r[c * np + i] = r;
            v[0] += r * r;
            v[1] += b * b;
        }
    }
    if (publish_partials<2>(v, B.partials, &S->ticket)) {
        double t[2];
        reduce_partials<2>(B.partials, t);
        if (threadIdx.x == 0) {
            if (first) {
                S->bb = t[1];
                S->iter = 0;
                S->status = SP_OK;
                S->done = 0;
                if (!isfinite(t[0]) || !isfinite(t[1])) {
                    S->status = SP_ERR_NONFINITE;
                    S->done = 1;
                } else if (t[0] <= P.tol2 * t[1]) {
                    S->done = 1;   // the start meets the tolerance (b = 0 included)
                }
            }
            S->rr = t[0];
            S->last_res = S->bb > 0.0 ? sqrt(t[0] / S->bb) : 0.0;
        }
    }
}

// z = D^-1 r (the Jacobi preconditioner)
__global__ void k_fcg_jacobi(KParams P, DevBuffers B, const FcgState* S)
{
    if (S->done) return;
    const int np = P.npad;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const double di = B.dinv[i];
#pragma unroll
        for (int c = 0; c < 3; ++c) B.z[c * np + i] = di * B.r[c * np + i];
    }
}

// p = z + beta p (beta = 0: the first direction)
__global__ void k_fcg_direction(KParams P, DevBuffers B, const FcgState* S, int first)
{
    if (S->done) return;
    const int np = P.npad;
    const double beta = first ? 0.0 : S->beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x)
#pragma unroll
        for (int c = 0; c < 3; ++c) B.p[c * np + i] = fma(beta, first ? 0.0 : B.p[c * np + i], B.z[c * np + i]);
}

// q = A p; (p, q) and (p, r); alpha = (p, r) / (p, q)
__global__ void k_fcg_spmv(KParams P, DevBuffers B, FcgState* S)
{
    if (S->done) return;
    const int np = P.npad;
    double v[2] = {0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        double q[3];
        fcg_row_apply(P, B, B.p, i, q);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            B.q[c * np + i] = q[c];
            const double p = B.p[c * np + i];
            v[0] += p * q[c];
            v[1] += p * B.r[c * np + i];
        }
    }
    if (publish_partials<2>(v, B.partials, &S->ticket)) {
        double t[2];
        reduce_partials<2>(B.partials, t);
        if (threadIdx.x == 0) {
            S->pq = t[0];
            if (!(t[0] > 0.0) || !isfinite(t[0]) || !isfinite(t[1])) {
                S->status = SP_ERR_NONFINITE;
                S->done = 1;
            } else {
                S->alpha = t[1] / t[0];
            }
        }
    }
}

// x += alpha p; r -= alpha q; ||r||^2 and the stopping test
__global__ void k_fcg_update(KParams P, DevBuffers B, FcgState* S)
{
    if (S->done) return;
    const int np = P.npad;
    const double a = S->alpha;
    double v[1] = {0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int k = c * np + i;
            B.x[k] = fma(a, B.p[k], B.x[k]);
            const double r = fma(-a, B.q[k], B.r[k]);
            B.r[k] = r;
            v[0] += r * r;
        }
    if (publish_partials<1>(v, B.partials, &S->ticket)) {
        double t[1];
        reduce_partials<1>(B.partials, t);
        if (threadIdx.x == 0) {
            S->rr = t[0];
            S->iter += 1;
            if (!isfinite(t[0])) {
                S->status = SP_ERR_NONFINITE;
                S->done = 1;
            } else if (t[0] <= P.tol2 * S->bb) {
                S->done = 1;
            } else if (S->iter >= P.max_iter) {
                S->status = SP_ERR_NOT_CONVERGED;
                S->done = 1;
            }
        }
    }
}

// beta = -(z, q) / (p, q): the new direction A-orthogonal to the last one
__global__ void k_fcg_beta(KParams P, DevBuffers B, FcgState* S)
{
    if (S->done) return;
    const int np = P.npad;
    double v[1] = {0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x)
#pragma unroll
        for (int c = 0; c < 3; ++c) v[0] += B.z[c * np + i] * B.q[c * np + i];
    if (publish_partials<1>(v, B.partials, &S->ticket)) {
        double t[1];
        reduce_partials<1>(B.partials, t);
        if (threadIdx.x == 0) {
            if (!isfinite(t[0])) {
                S->status = SP_ERR_NONFINITE;
                S->done = 1;
            }
            S->beta = -t[0] / S->pq;
        }
    }
}

}  // namespace

int fcg_solve(const KParams& P, DevBuffers& B, const MpBuffers* net, int net_every, FcgState* S, FcgState* S_host,
              Launch L, long long* launches)
{
    const int grid = grid_for(P.n, kVecBlock, std::min(kMaxPartials, L.num_sms * 8));
    auto precondition = [&](int k) {
        if (net && net_every > 0 && k % net_every == 0) {
            launch_mp_apply(P, B, *net, B.r, B.z, L);
            *launches += mp_infer_launches();
        } else {
            k_fcg_jacobi<<<grid, kVecBlock, 0, L.stream>>>(P, B, S);
            *launches += 1;
        }
    };
    if (cudaMemsetAsync(S, 0, sizeof(FcgState), L.stream) != cudaSuccess) return SP_ERR_CUDA;
    k_fcg_residual<<<grid, kVecBlock, 0, L.stream>>>(P, B, S, 1);
    precondition(0);
    k_fcg_direction<<<grid, kVecBlock, 0, L.stream>>>(P, B, S, 1);
    *launches += 2;
    const int chunk = 8;
    for (int k = 0; k < P.max_iter; k += chunk) {
        for (int u = 0; u < chunk; ++u) {
            k_fcg_spmv<<<grid, kVecBlock, 0, L.stream>>>(P, B, S);
            k_fcg_update<<<grid, kVecBlock, 0, L.stream>>>(P, B, S);
            precondition(k + u + 1);
            k_fcg_beta<<<grid, kVecBlock, 0, L.stream>>>(P, B, S);
            k_fcg_direction<<<grid, kVecBlock, 0, L.stream>>>(P, B, S, 0);
            *launches += 4;
        }
        if (cudaMemcpyAsync(S_host, S, sizeof(FcgState), cudaMemcpyDeviceToHost, L.stream) != cudaSuccess ||
            cudaStreamSynchronize(L.stream) != cudaSuccess)
            return SP_ERR_CUDA;
        if (S_host->done) break;
    }
    // the true residual of the final x
    const int status = S_host->status;
    k_fcg_residual<<<grid, kVecBlock, 0, L.stream>>>(P, B, S, 0);
    *launches += 1;
    if (cudaMemcpyAsync(S_host, S, sizeof(FcgState), cudaMemcpyDeviceToHost, L.stream) != cudaSuccess ||
        cudaStreamSynchronize(L.stream) != cudaSuccess)
        return SP_ERR_CUDA;
    if (cudaGetLastError() != cudaSuccess) return SP_ERR_CUDA;
    S_host->status = status;
    if (status == SP_OK && !S_host->done) S_host->status = SP_ERR_NOT_CONVERGED;
    return SP_OK;
}

}  // namespace ss
