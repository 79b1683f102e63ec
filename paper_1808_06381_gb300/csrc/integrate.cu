// Position update with the Lees-Edwards wrap, the pair-virial shear stress,
// and the by-id transfers used by the state-access calls (arXiv 1808.06381,
// §Method).
#include <math.h>

#include "internal.cuh"

namespace ss {

// R += v dt (first order in time, v = dR/dt).  The image offset advances first,
// delta' = delta + kappa L_y dt (mod L_x); a particle leaving through y = L_y
// re-enters at y - L_y shifted by -delta' in x (through y = 0: +delta').  The
// new state is written in the current cell order together with the ids and
// the velocities (the next step's warm start).  The last block advances the
// device's offset and step counter.
// wrap_box for a coordinate at most one box edge outside [0, L) (a step moves
// a particle by v dt, the sheared re-entry by at most L_x more) without its
// FP64 division (GB300 issues FP64 at 1/64 of the FP32 rate): the same value
// (x - L and x + L are what x - L floor(x / L) rounds to there); further out,
// wrap_box itself.
__device__ __forceinline__ double wrap_near(double x, double L)
{
    if (x >= 0.0 && x < L) return x;
    if (x >= L && x < 2.0 * L) return __dsub_rn(x, L);
    if (x < 0.0 && x >= -L) {
        const double y = __dadd_rn(x, L);
        return y < L ? y : 0.0;   // x + L rounds to L for tiny negative x: wrap_box gives 0 there
    }
    return wrap_box(x, L);
}

__global__ void __launch_bounds__(kVecBlock) k_integrate(KParams P, DevBuffers B)
{
    DevState* st = B.st;
    if (st->error | st->overflow) return;
    const int np = P.npad;
    // the advanced offset once per block: its FP64 division runs on GB300's
    // 1/64-rate FP64 pipe, and per thread it cost more than the rows' update
    __shared__ double s_dnew;
    if (threadIdx.x == 0) s_dnew = wrap_box(st->delta + P.kappa * P.L[1] * P.dt, P.L[0]);
    __syncthreads();
    const double dnew = s_dnew;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const double vx = B.x[i], vy = B.x[np + i], vz = B.x[2 * np + i];
        double x = __dadd_rn(B.pos_w[i], __dmul_rn(vx, P.dt));
        double y = __dadd_rn(B.pos_w[np + i], __dmul_rn(vy, P.dt));
        const double z = __dadd_rn(B.pos_w[2 * np + i], __dmul_rn(vz, P.dt));
        if (y < 0.0) {
            y = y + P.L[1];
            x = x + dnew;
        }
        if (y >= P.L[1]) {
            y = y - P.L[1];
            x = x - dnew;
        }
        B.pos_s[i] = wrap_near(x, P.L[0]);
        B.pos_s[np + i] = y;
        B.pos_s[2 * np + i] = wrap_near(z, P.L[2]);
        B.id_s[i] = B.id_w[i];
        B.v_s[i] = vx;
        B.v_s[np + i] = vy;
        B.v_s[2 * np + i] = vz;
    }
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&st->ticket[1], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        st->ticket[1] = 0u;
        st->delta_next = dnew;
        st->step += 1;
        st->steps_in_call += 1;
    }
}

__global__ void k_commit_step(DevBuffers B)
{
    DevState* st = B.st;
    if (st->error | st->overflow) return;
    st->delta = st->delta_next;
}

void launch_commit_step(DevBuffers& B, Launch L)
{
    k_commit_step<<<1, 1, 0, L.stream>>>(B);
}

void launch_integrate(const KParams& P, DevBuffers& B, Launch L, bool commit)
{
    k_integrate<<<grid_for(P.n, kVecBlock, L.num_sms * 8), kVecBlock, 0, L.stream>>>(P, B);
    if (commit) launch_commit_step(B, L);
}

// sigma_xy = -(1/V) sum_{i<j} y_ij f_ij,x with the pair forces of Eq. F and
// Eq. vc (times zeta): f_ij = c_ev R_ij w_ij + zeta alpha w_ij (v_j - v_i + V_ij).
// y_ij f_ij,x is symmetric in (i, j), so each row sums its whole neighbour list
// and the total is halved.  Separations come from the stored image codes and
// weights from the assembled matrix.
__global__ void __launch_bounds__(kVecBlock) k_stress(KParams P, DevBuffers B)
{
    DevState* st = B.st;
    if (st->error | st->overflow) return;
    const int np = P.npad;
    const double delta = st->delta;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const double xi = B.pos_w[i], yi = B.pos_w[np + i], zi = B.pos_w[2 * np + i];
        const double vxi = B.x[i];
        const int slot = B.row_slot[i];
        const int base = B.chunk_off[slot >> 5] + (slot & 31);
        const int cnt = B.row_cnt[i];
        for (int k = 0; k < cnt; ++k) {
            const int e = base + 32 * k;
            const int j = B.col[e];
            double dx, dy, dz;
            const double nimg = image_separation(P, delta, xi, yi, zi, B.pos_w[j], B.pos_w[np + j],
                                                 B.pos_w[2 * np + j], B.img[e], dx, dy, dz);
            const double w = B.val[e];
            const double fx = P.c_ev * dx * w + P.zeta * P.alpha * w * (B.x[j] - vxi + P.kappa * P.L[1] * nimg);
            acc += dy * fx;
        }
    }
    const double v[1] = {acc};
    if (publish_partials<1>(v, B.partials, &st->ticket[0])) {
        double out[1];
        reduce_partials<1>(B.partials, out);
        if (threadIdx.x == 0) st->stress_xy = -0.5 * out[0] / (P.L[0] * P.L[1] * P.L[2]);
    }
}

// The same sum for the mixed solver without FP64 arithmetic in the loop:
// separations from the FP32 positions and the pair's image (for box edges L
// each component is within about 5 L 2^-24 of the exact one, below 1e-5
// relative for the boxes used here), weights from the FP32 matrix, FP32
// velocities, and a double-float accumulation.  Each pair once (the entry of
// its lower row; y_ij f_ij,x is symmetric in i and j), so half the gathers.
constexpr int kStressBatch = 4;   // entries requested at a time

__global__ void __launch_bounds__(kVecBlock) k_stress32(KParams P, DevBuffers B)
{
    DevState* st = B.st;
    if (st->error | st->overflow) return;
    const int np = P.npad;
    // the step's offset in FP32 once per block (a conversion runs on GB300's slow FP64 pipe)
    __shared__ float s_deltaf;
    if (threadIdx.x == 0) s_deltaf = (float)st->delta;
    __syncthreads();
    const float deltaf = s_deltaf;
    const float c_ev = P.c_ev_f, za = P.za_f, kl = P.kly_f;
    // shifts of the image codes by selection (GB300 converts integers to
    // floats at the FP64 rate); velocities from the solver's double-float x
    auto sel = [](int k, float v) { return k == 0 ? 0.f : (k > 0 ? v : -v); };
    dfloat acc{0.f, 0.f};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const float xi = B.pos32[i], yi = B.pos32[np + i];
        const float vxi = B.xdf[2 * i].x;
        const int slot = B.row_slot[i];
        const int base = B.chunk_off[slot >> 5] + (slot & 31);
        const int cnt = B.row_cnt[i];
        float row = 0.f;
        for (int kb = 0; kb < cnt; kb += kStressBatch) {
            int j[kStressBatch], code[kStressBatch];
            float w[kStressBatch];
#pragma unroll
            for (int u = 0; u < kStressBatch; ++u) {
                const int e = base + 32 * (kb + u);
                j[u] = kb + u < cnt ? B.col[e] : i;
                code[u] = kb + u < cnt ? (int)B.img[e] : image_code(0, 0, 0);
                w[u] = kb + u < cnt ? B.val32[e] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kStressBatch; ++u) {
                if (j[u] <= i) continue;   // the pair's other entry (padding points at the row itself)
                const int a = (code[u] & 7) - 2, m = ((code[u] >> 3) & 3) - 1;
                const float ax = a == 0 ? 0.f : (a == 1 ? P.Lf[0] : (a == -1 ? -P.Lf[0] : (a == 2 ? 2.f * P.Lf[0] : -2.f * P.Lf[0])));
                const float dx = (xi - B.pos32[j[u]]) - (sel(m, deltaf) + ax);
                const float dy = (yi - B.pos32[np + j[u]]) - sel(m, P.Lf[1]);
                const float fx = c_ev * dx * w[u] + za * w[u] * (B.xdf[2 * j[u]].x - vxi + sel(m, kl));
                row = fmaf(dy, fx, row);
            }
        }
        acc = df_add(acc, row);
    }
    dfloat v[1] = {acc};
    double out[1];
    if (publish_reduce_df<1>(v, B.partials_df, &st->ticket[0], out) && threadIdx.x == 0)
        st->stress_xy = -out[0] / (P.L[0] * P.L[1] * P.L[2]);
}

void launch_stress(const KParams& P, DevBuffers& B, bool mixed, Launch L)
{
    if (mixed)
        k_stress32<<<grid_for(P.n, kVecBlock, L.num_sms * 8), kVecBlock, 0, L.stream>>>(P, B);
    else
        k_stress<<<grid_for(P.n, kVecBlock, L.num_sms * 8), kVecBlock, 0, L.stream>>>(P, B);
}

__global__ void k_scatter_by_id(const double* __restrict__ planes, int npad, const int* __restrict__ ids,
                                int n, double* __restrict__ out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const long long id = ids[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) out[3 * id + a] = planes[a * npad + k];
}

void launch_scatter_by_id(const double* planes, int npad, const int* ids, int n, double* out_n3,
                          cudaStream_t s)
{
    k_scatter_by_id<<<grid_for(n, kVecBlock, 1 << 30), kVecBlock, 0, s>>>(planes, npad, ids, n, out_n3);
}

__global__ void k_gather_by_id(const double* __restrict__ in, const int* __restrict__ ids, int n,
                               int npad, double* __restrict__ planes)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const long long id = ids[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) planes[a * npad + k] = in[3 * id + a];
}

void launch_gather_by_id(const double* in_n3, const int* ids, int n, int npad, double* planes,
                         cudaStream_t s)
{
    k_gather_by_id<<<grid_for(n, kVecBlock, 1 << 30), kVecBlock, 0, s>>>(in_n3, ids, n, npad, planes);
}

__global__ void k_gather_positions(const double* __restrict__ in, const int* __restrict__ ids, int n, int npad,
                                   double* __restrict__ planes, double L0, double L1, double L2, DevState* st)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const long long id = ids[k];
    const double x = in[3 * id], y = in[3 * id + 1], z = in[3 * id + 2];
    // the comparisons are false for NaN, so a NaN fails them too
    const bool ok = x >= 0.0 && x < L0 && y >= 0.0 && y < L1 && z >= 0.0 && z < L2;
    if (!ok) atomicCAS(&st->error, 0, (int)SP_ERR_INVALID_ARG);
    planes[k] = x;
    planes[npad + k] = y;
    planes[2 * npad + k] = z;
}

void launch_gather_positions(const double* in_n3, const int* ids, int n, int npad, double* planes,
                             const KParams& P, DevState* st, cudaStream_t s)
{
    k_gather_positions<<<grid_for(n, kVecBlock, 1 << 30), kVecBlock, 0, s>>>(in_n3, ids, n, npad, planes, P.L[0],
                                                                             P.L[1], P.L[2], st);
}

__global__ void k_reset_step_stats(DevState* st);

cudaError_t device_code_version(int* binary_version, int* ptx_version)
{
    cudaFuncAttributes a{};
    const cudaError_t e = cudaFuncGetAttributes(&a, k_reset_step_stats);
    if (e == cudaSuccess) {
        *binary_version = a.binaryVersion;
        *ptx_version = a.ptxVersion;
    }
    return e;
}

__global__ void k_reset_step_stats(DevState* st)
{
    st->iter_sum = 0;
    st->iter_max = 0;
    st->steps_in_call = 0;
    st->true_checks = 0;
}

void launch_reset_step_stats(DevState* st, cudaStream_t s)
{
    k_reset_step_stats<<<1, 1, 0, s>>>(st);
}

}  // namespace ss
