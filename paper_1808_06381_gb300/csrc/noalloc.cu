// sp_solve_csr_noalloc: the velocity solve of Eq. algebra for callers that
// cannot allocate device memory.
//
// Some callers run where cudaMalloc is not available to them: inside a host
// framework that owns every device allocation (a fixed memory pool, a
// real-time or embedded loop that forbids allocation after start-up, or a
// library that must not touch the caller's allocator).  This entry point takes
// the system and the output from the caller and keeps its own working vectors
// (r, z, p, q, the Jacobi diagonal, the partial sums and the solver scalars)
// in one file-scope device array of fixed size, so it never allocates.
//
// Limits and sharing:
//   - at most kNoallocMaxRows rows; larger systems are rejected;
//   - the array (about 3.2 MB) lives in every device context that loads the
//     library, until the process exits;
//   - every call on a device uses the same array: calls that may overlap on
//     the GPU (other streams, other host threads) race and must be serialised
//     by the caller;
//   - the first call on a device looks up the array's device address with that
//     device current; every call reads the solver state back and synchronises
//     its stream, so no call may be made on a stream that is being captured
//     (such a call is rejected);
//   - device ordinals 0 .. 63 (one looked-up address per device).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "internal.cuh"

namespace ss {
namespace {

constexpr long long kNoallocMaxRows = 32768;
constexpr int kNaThreads = 256;
constexpr int kNaBlocks = 128;   // kNaBlocks * kNaThreads = the rows handled per grid sweep

struct NaState {
    double bnorm2, rho, alpha, beta, rr, last_res;
    int iter, done, status, check_true, restarts;
    unsigned int ticket;
};

constexpr size_t kPlane = (size_t)kNoallocMaxRows;
constexpr size_t kVecDoubles = 3 * kPlane;               // one [3][n] vector
constexpr size_t kScratchDoubles = 4 * kVecDoubles       // r, z, p, q
                                   + kPlane              // dinv
                                   + 2 * kNaBlocks;      // partial sums
constexpr size_t kScratchBytes = kScratchDoubles * sizeof(double) + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct NaPtrs {
    double *r, *z, *p, *q, *dinv, *partials;
    NaState* st;
};

NaPtrs carve(unsigned char* base)
{
    double* d = reinterpret_cast<double*>(base);
    NaPtrs s;
    s.r = d;
    s.z = d + kVecDoubles;
    s.p = d + 2 * kVecDoubles;
    s.q = d + 3 * kVecDoubles;
    s.dinv = d + 4 * kVecDoubles;
    s.partials = s.dinv + kPlane;
    s.st = reinterpret_cast<NaState*>(base + kScratchDoubles * sizeof(double));
    return s;
}

struct NaSystem {
    long long n;
    const int* row_ptr;
    const int* col;
    const double* w;
    const double* diag;
    double alpha;
    const double* b;
    double* x;
    double tol2;
    int max_iter;
};

// Sum over the block, then the last block to finish reduces the per-block sums.
template <int K>
__device__ bool na_publish(double (&v)[K], double* partials, unsigned int* ticket)
{
    __shared__ double sh[32];
    __shared__ bool last;
    for (int k = 0; k < K; ++k) {
        const double t = block_sum(v[k], sh);
        if (threadIdx.x == 0) partials[k * kNaBlocks + blockIdx.x] = t;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(partials + k * kNaBlocks + i);
        v[k] = block_sum(s, sh);
    }
    if (threadIdx.x == 0) *ticket = 0u;
    return true;
}

// (A u)_i for the three planes of a scratch vector u (plane stride kPlane): A = diag - alpha W.
__device__ __forceinline__ void na_row_apply(const NaSystem& S, const double* u, long long i, double* out3)
{
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int k = S.row_ptr[i]; k < S.row_ptr[i + 1]; ++k) {
        const long long j = S.col[k];
        const double w = S.w[k];
        s0 += w * u[j];
        s1 += w * u[kPlane + j];
        s2 += w * u[2 * kPlane + j];
    }
    const double d = S.diag[i];
    out3[0] = d * u[i] - S.alpha * s0;
    out3[1] = d * u[kPlane + i] - S.alpha * s1;
    out3[2] = d * u[2 * kPlane + i] - S.alpha * s2;
}

// Rejects a malformed CSR before anything gathers through it: row_ptr must
// start at 0 and never decrease, and every column must lie in [0, n) (a
// column in [n, kPlane) would read another call's stale entries of the shared
// array, one beyond it memory outside the array).
__global__ void k_na_validate(NaSystem S, NaPtrs W)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S.n; i += gridDim.x * blockDim.x) {
        const int b = S.row_ptr[i], e = S.row_ptr[i + 1];
        bool bad = (i == 0 && b != 0) || e < b;
        for (int k = b; k < e && !bad; ++k) {
            const int j = S.col[k];
            bad = j < 0 || (long long)j >= S.n;
        }
        if (bad) {
            W.st->status = SP_ERR_INVALID_ARG;
            W.st->done = 1;
        }
    }
}

// x = 0, r = b, z = D^-1 r, p = z; b.b and r.z.
__global__ void k_na_init(NaSystem S, NaPtrs W)
{
    if (W.st->done) return;   // rejected by k_na_validate (uniform over the grid)
    double v[2] = {0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S.n; i += gridDim.x * blockDim.x) {
        const double di = 1.0 / S.diag[i];
        W.dinv[i] = di;
        for (int c = 0; c < 3; ++c) {
            const double bk = S.b[c * S.n + i];
            S.x[c * S.n + i] = 0.0;
            W.r[c * kPlane + i] = bk;
            W.z[c * kPlane + i] = di * bk;
            W.p[c * kPlane + i] = di * bk;
            v[0] += bk * bk;
            v[1] += di * bk * bk;
        }
    }
    if (na_publish<2>(v, W.partials, &W.st->ticket) && threadIdx.x == 0) {
        NaState* st = W.st;
        st->bnorm2 = v[0];
        st->rho = v[1];
        st->rr = v[0];
        st->iter = 0;
        st->restarts = 0;
        st->check_true = 0;
        st->status = SP_OK;
        st->last_res = 0.0;
        st->done = (v[0] == 0.0) ? 1 : 0;
        if (!std::isfinite(v[0])) {
            st->status = SP_ERR_NONFINITE;
            st->done = 1;
        }
    }
}

// q = A p; p.q; alpha = rho / p.q.
__global__ void k_na_spmv(NaSystem S, NaPtrs W)
{
    NaState* st = W.st;
    if (st->done) return;
    double v[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S.n; i += gridDim.x * blockDim.x) {
        double q3[3];
        na_row_apply(S, W.p, i, q3);
        for (int c = 0; c < 3; ++c) {
            W.q[c * kPlane + i] = q3[c];
            v[0] += W.p[c * kPlane + i] * q3[c];
        }
    }
    if (na_publish<1>(v, W.partials, &st->ticket) && threadIdx.x == 0) {
        if (!(v[0] > 0.0) || !std::isfinite(v[0])) {
            st->status = SP_ERR_NONFINITE;
            st->done = 1;
        } else {
            st->alpha = st->rho / v[0];
        }
    }
}

// x += alpha p; r -= alpha q; z = D^-1 r; r.r, r.z; beta; the recurrence test.
__global__ void k_na_update(NaSystem S, NaPtrs W)
{
    NaState* st = W.st;
    if (st->done) return;
    const double a = st->alpha;
    double v[2] = {0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S.n; i += gridDim.x * blockDim.x) {
        const double di = W.dinv[i];
        for (int c = 0; c < 3; ++c) {
            S.x[c * S.n + i] += a * W.p[c * kPlane + i];
            const double rk = W.r[c * kPlane + i] - a * W.q[c * kPlane + i];
            W.r[c * kPlane + i] = rk;
            W.z[c * kPlane + i] = di * rk;
            v[0] += rk * rk;
            v[1] += di * rk * rk;
        }
    }
    if (na_publish<2>(v, W.partials, &st->ticket) && threadIdx.x == 0) {
        st->iter += 1;
        st->rr = v[0];
        st->beta = v[1] / st->rho;
        st->rho = v[1];
        if (!std::isfinite(v[0])) {
            st->status = SP_ERR_NONFINITE;
            st->done = 1;
        } else if (v[0] <= S.tol2 * st->bnorm2 || st->iter >= S.max_iter) {
            st->check_true = 1;
        }
    }
}

// When armed: r = b - A x exactly, accept or restart (beta = 0); then p = z + beta p.
__global__ void k_na_check(NaSystem S, NaPtrs W)
{
    NaState* st = W.st;
    if (st->done || !st->check_true) return;
    double v[2] = {0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S.n; i += gridDim.x * blockDim.x) {
        // A x with x in the caller's planes (plane stride n)
        double ax[3];
        const double x3[3] = {S.x[i], S.x[S.n + i], S.x[2 * S.n + i]};
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int k = S.row_ptr[i]; k < S.row_ptr[i + 1]; ++k) {
            const long long j = S.col[k];
            const double w = S.w[k];
            s0 += w * S.x[j];
            s1 += w * S.x[S.n + j];
            s2 += w * S.x[2 * S.n + j];
        }
        const double d = S.diag[i];
        ax[0] = d * x3[0] - S.alpha * s0;
        ax[1] = d * x3[1] - S.alpha * s1;
        ax[2] = d * x3[2] - S.alpha * s2;
        const double di = W.dinv[i];
        for (int c = 0; c < 3; ++c) {
            const double rk = S.b[c * S.n + i] - ax[c];
            W.r[c * kPlane + i] = rk;
            W.z[c * kPlane + i] = di * rk;
            v[0] += rk * rk;
            v[1] += di * rk * rk;
        }
    }
    if (na_publish<2>(v, W.partials, &st->ticket) && threadIdx.x == 0) {
        st->check_true = 0;
        st->last_res = st->bnorm2 > 0.0 ? sqrt(v[0] / st->bnorm2) : 0.0;
        if (v[0] <= S.tol2 * st->bnorm2) {
            st->done = 1;
        } else if (st->iter >= S.max_iter || st->restarts >= kMaxCgRestarts) {
            st->status = SP_ERR_NOT_CONVERGED;
            st->done = 1;
        } else {
            st->restarts += 1;
            st->rho = v[1];
            st->beta = 0.0;
        }
    }
}

__global__ void k_na_direction(NaSystem S, NaPtrs W)
{
    const NaState* st = W.st;
    if (st->done) return;
    const double beta = st->beta;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S.n; i += gridDim.x * blockDim.x)
        for (int c = 0; c < 3; ++c) W.p[c * kPlane + i] = W.z[c * kPlane + i] + beta * W.p[c * kPlane + i];
}

std::mutex g_na_mutex;
void* g_na_base[64] = {nullptr};

}  // namespace
}  // namespace ss

extern std::string& sp_global_error();

extern "C" int sp_solve_csr_noalloc(int32_t device, void* stream, int64_t n, const int32_t* row_ptr_dev,
                                    const int32_t* col_dev, const double* w_dev, const double* diag_dev,
                                    double alpha, const double* b_dev, double* x_dev, double tol,
                                    int32_t max_iter, sp_solve_info* info)
{
    using namespace ss;
    std::string& err = sp_global_error();
    if (n < 1 || n > kNoallocMaxRows) {
        err = "sp_solve_csr_noalloc: n must be in [1, " + std::to_string(kNoallocMaxRows) + "]";
        return SP_ERR_INVALID_ARG;
    }
    if (!row_ptr_dev || !col_dev || !w_dev || !diag_dev || !b_dev || !x_dev || !(tol > 0) || max_iter < 1 ||
        !(alpha >= 0) || device < 0 || device >= 64) {
        err = "sp_solve_csr_noalloc: null pointer or invalid tol, max_iter, alpha or device";
        return SP_ERR_INVALID_ARG;
    }
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        err = "sp_solve_csr_noalloc: no CUDA device with that ordinal";
        return SP_ERR_NO_DEVICE;
    }
    auto finish = [&](int rc, const char* what) {
        if (what) err = std::string("sp_solve_csr_noalloc: ") + what + ": " + cudaGetErrorString(cudaGetLastError());
        cudaSetDevice(prev);
        return rc;
    };
    // every call reads the solver state back and synchronises, which a stream
    // under capture does not allow (checked before anything else touches the device)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cap) != cudaSuccess)
        return finish(SP_ERR_CUDA, "cudaStreamIsCapturing");
    if (cap != cudaStreamCaptureStatusNone) {
        err = "sp_solve_csr_noalloc: the stream is being captured; this call synchronises and cannot be captured";
        cudaSetDevice(prev);
        return SP_ERR_INVALID_ARG;
    }
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_base[device]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
                return finish(SP_ERR_CUDA, "cudaGetSymbolAddress");
            g_na_base[device] = p;
        }
        base = g_na_base[device];
    }
    NaPtrs Wp = carve(static_cast<unsigned char*>(base));
    NaSystem S{n, row_ptr_dev, col_dev, w_dev, diag_dev, alpha, b_dev, x_dev, tol * tol, max_iter};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the state (and the reduction ticket) must start at zero on every call
    if (cudaMemsetAsync(Wp.st, 0, sizeof(NaState), s) != cudaSuccess) return finish(SP_ERR_CUDA, "cudaMemsetAsync");
    const int grid = (int)std::min<long long>(kNaBlocks, (n + kNaThreads - 1) / kNaThreads);
    k_na_validate<<<grid, kNaThreads, 0, s>>>(S, Wp);
    k_na_init<<<grid, kNaThreads, 0, s>>>(S, Wp);
    NaState h;
    std::memset(&h, 0, sizeof(h));
    for (int it = 0; it < max_iter + kMaxCgRestarts + 8; it += 8) {
        for (int k = 0; k < 8; ++k) {
            k_na_spmv<<<grid, kNaThreads, 0, s>>>(S, Wp);
            k_na_update<<<grid, kNaThreads, 0, s>>>(S, Wp);
            k_na_check<<<grid, kNaThreads, 0, s>>>(S, Wp);
            k_na_direction<<<grid, kNaThreads, 0, s>>>(S, Wp);
        }
        if (cudaMemcpyAsync(&h, Wp.st, sizeof(NaState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return finish(SP_ERR_CUDA, "reading the solver state");
        if (h.done) break;
    }
    int status = h.done ? h.status : SP_ERR_NOT_CONVERGED;
    if (info) {
        info->status = status;
        info->iterations = h.iter;
        info->residual = h.last_res;
        info->bnorm = std::sqrt(h.bnorm2);
        info->offchip_blocks = 0;
    }
    if (status == SP_ERR_INVALID_ARG)
        err = "sp_solve_csr_noalloc: row_ptr must start at 0 and not decrease, and every col must lie in [0, n)";
    else if (status == SP_ERR_NOT_CONVERGED)
        err = "sp_solve_csr_noalloc: not converged (max_iter reached, or the true residual stayed above tol "
              "after the restart limit)";
    else if (status != SP_OK)
        err = "sp_solve_csr_noalloc: solve failed";
    return finish(status, nullptr);
}
