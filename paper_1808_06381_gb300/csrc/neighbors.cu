// Cell list with sheared periodic images, pair search, and the fused pair
// kernel that emits the forces of Eq. F and the friction matrix of Eq. algebra
// (arXiv 1808.06381, §Method).
//
// Rows are kept in cell order: each step re-sorts the particles by cell with a
// counting sort (histogram, exclusive scan, scatter) and orders the particles
// of a cell by id, so the order is deterministic and neighbours sit close in
// memory for the solver's gathers.
#include "internal.cuh"

namespace ss {

// ----------------------------------------------------------------- binning

__global__ void k_bin(KParams P, const double* __restrict__ pos, int* __restrict__ cell_of,
                      int* __restrict__ slot, int* __restrict__ cell_count, const DevState* st)
{
    if (st->error | st->overflow) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const int cx = cell_coord(pos[i], P.inv_cw[0], P.nc[0]);
    const int cy = cell_coord(pos[P.npad + i], P.inv_cw[1], P.nc[1]);
    const int cz = cell_coord(pos[2 * P.npad + i], P.inv_cw[2], P.nc[2]);
    const int c = (cz * P.nc[1] + cy) * P.nc[0] + cx;
    cell_of[i] = c;
    slot[i] = atomicAdd(cell_count + c, 1);
}

void launch_bin(const KParams& P, DevBuffers& B, Launch L)
{
    cudaMemsetAsync(B.cell_count, 0, sizeof(int) * (size_t)P.ncell, L.stream);
    k_bin<<<grid_for(P.n, kVecBlock, 1 << 30), kVecBlock, 0, L.stream>>>(P, B.pos_s, B.cell_of, B.slot,
                                                                            B.cell_count, B.st);
}

// ------------------------------------------------------------ exclusive scan
// out[k] = sum_{m<k} in[m] for k in [0, n]; out[n] is the total.  Three
// kernels: per-chunk sums, a one-block scan of the chunk sums, and a
// chunk-local rescan.  mode 1 also records the total as the matrix size and
// raises the overflow flag if it exceeds cap_check.

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;

__global__ void k_scan_reduce(const int* __restrict__ in, int n, int* __restrict__ bsum,
                              const DevState* st)
{
    if (st->error | st->overflow) return;
    __shared__ double sh[32];
    const int base = blockIdx.x * kScanChunk;
    long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int idx = base + k * kScanThreads + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    const double tot = block_sum((double)s, sh);
    if (threadIdx.x == 0) bsum[blockIdx.x] = (int)tot;
}

__device__ __forceinline__ int block_exclusive_scan_int(int v, int* total)
{
    __shared__ int wsum[32];
    __shared__ int wtot;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    __syncthreads();
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        int ws = lane < nw ? wsum[lane] : 0;
        int wi = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < nw) wsum[lane] = wi - ws;
        if (lane == nw - 1) wtot = wi;
    }
    __syncthreads();
    const int excl = incl - v + wsum[w];
    if (total) *total = wtot;
    __syncthreads();
    return excl;
}

__global__ void k_scan_top(int* __restrict__ bsum, int nb, int* __restrict__ out, int n,
                           long long cap_check, DevState* st, int mode)
{
    if (st->error | st->overflow) return;
    long long carry = 0;
    for (int base = 0; base < nb; base += blockDim.x) {
        const int idx = base + threadIdx.x;
        const int v = idx < nb ? bsum[idx] : 0;
        int tot;
        const int e = block_exclusive_scan_int(v, &tot);
        if (idx < nb) bsum[idx] = (int)(carry + e);
        carry += tot;
    }
    if (threadIdx.x == 0) {
        out[n] = (int)carry;
        if (mode == 1) {
            st->nnz = carry;
            if (carry > cap_check) st->overflow = 1;
        }
    }
}

__global__ void k_scan_down(const int* __restrict__ in, int* __restrict__ out, int n,
                            const int* __restrict__ bsum, const DevState* st)
{
    if (st->error | st->overflow) return;
    __shared__ int s[kScanChunk];
    const int base = blockIdx.x * kScanChunk;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int idx = base + k * kScanThreads + threadIdx.x;
        s[k * kScanThreads + threadIdx.x] = idx < n ? in[idx] : 0;
    }
    __syncthreads();
    int loc[kScanItems];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        loc[k] = sum;
        sum += s[threadIdx.x * kScanItems + k];
    }
    const int off = block_exclusive_scan_int(sum, nullptr) + bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) s[threadIdx.x * kScanItems + k] = loc[k] + off;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int idx = base + k * kScanThreads + threadIdx.x;
        if (idx < n) out[idx] = s[k * kScanThreads + threadIdx.x];
    }
}

void launch_scan(const int* in, int* out, int n, int* block_tmp, long long cap_check, DevState* st,
                 int mode, Launch L)
{
    const int nb = (n + kScanChunk - 1) / kScanChunk;
    k_scan_reduce<<<nb, kScanThreads, 0, L.stream>>>(in, n, block_tmp, st);
    k_scan_top<<<1, 1024, 0, L.stream>>>(block_tmp, nb, out, n, cap_check, st, mode);
    k_scan_down<<<nb, kScanThreads, 0, L.stream>>>(in, out, n, block_tmp, st);
}

// ------------------------------------------------- scatter, sort by id, gather

__global__ void k_scatter(int n, const int* __restrict__ cell_of, const int* __restrict__ slot,
                          const int* __restrict__ cell_start, int* __restrict__ perm,
                          const DevState* st)
{
    if (st->error | st->overflow) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    perm[cell_start[cell_of[i]] + slot[i]] = i;
}

// One thread per cell: order the cell's particles by id (the atomic slots of
// k_bin are not deterministic), then gather positions, ids and the warm-start
// velocities into the new order.
__global__ void k_sort_gather(KParams P, const int* __restrict__ cell_start, int* __restrict__ perm,
                              const int* __restrict__ id_s, const double* __restrict__ pos_s,
                              const double* __restrict__ v_s, double* __restrict__ pos_w,
                              float* __restrict__ pos32, int* __restrict__ id_w,
                              double* __restrict__ x, int warm, const DevState* st)
{
    if (st->error | st->overflow) return;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P.ncell) return;
    const int beg = cell_start[c], end = cell_start[c + 1];
    for (int k = beg + 1; k < end; ++k) {
        const int key = perm[k];
        const int kid = id_s[key];
        int j = k - 1;
        while (j >= beg && id_s[perm[j]] > kid) {
            perm[j + 1] = perm[j];
            --j;
        }
        perm[j + 1] = key;
    }
    const int np = P.npad;
    for (int k = beg; k < end; ++k) {
        const int s = perm[k];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double v = pos_s[a * np + s];
            pos_w[a * np + k] = v;
            pos32[a * np + k] = (float)v;
        }
        id_w[k] = id_s[s];
        x[k] = warm ? v_s[s] : 0.0;
        x[np + k] = warm ? v_s[np + s] : 0.0;
        x[2 * np + k] = warm ? v_s[2 * np + s] : 0.0;
    }
}

void launch_scatter_sort_gather(const KParams& P, DevBuffers& B, bool warm, Launch L)
{
    k_scatter<<<grid_for(P.n, kVecBlock, 1 << 30), kVecBlock, 0, L.stream>>>(P.n, B.cell_of, B.slot,
                                                                                B.cell_start, B.perm, B.st);
    k_sort_gather<<<grid_for(P.ncell, 128, 1 << 30), 128, 0, L.stream>>>(
        P, B.cell_start, B.perm, B.id_s, B.pos_s, B.v_s, B.pos_w, B.pos32, B.id_w, B.x, warm ? 1 : 0, B.st);
}

// Single-cell boxes (every edge below 3 r_c): keep the state order.
__global__ void k_identity_gather(KParams P, const int* __restrict__ id_s,
                                  const double* __restrict__ pos_s, const double* __restrict__ v_s,
                                  double* __restrict__ pos_w, float* __restrict__ pos32,
                                  int* __restrict__ id_w, double* __restrict__ x, int* __restrict__ perm,
                                  int warm, const DevState* st)
{
    if (st->error | st->overflow) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.n) return;
    const int np = P.npad;
    perm[k] = k;
    id_w[k] = id_s[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        pos_w[a * np + k] = pos_s[a * np + k];
        pos32[a * np + k] = (float)pos_s[a * np + k];
        x[a * np + k] = warm ? v_s[a * np + k] : 0.0;
    }
}

void launch_identity_gather(const KParams& P, DevBuffers& B, bool warm, Launch L)
{
    k_identity_gather<<<grid_for(P.n, kVecBlock, 1 << 30), kVecBlock, 0, L.stream>>>(
        P, B.id_s, B.pos_s, B.v_s, B.pos_w, B.pos32, B.id_w, B.x, B.perm, warm ? 1 : 0, B.st);
}

// ------------------------------------------------------------- pair search

// Visit every j != i with |R_ij|^2 < r_c^2 (the 5 % truncation of §Method).
// Candidate cells: the 3 x 3 x 3 block around i's cell; a row of cells that
// wraps through y = 0 or y = L_y belongs to the image displaced by -/+ delta in
// x, so its three x cells are centred on x_i +/- delta.  Axes with fewer than
// 3 cells are scanned whole (and then x is scanned whole when y is).  Every
// candidate goes through the exact predicate, so the pair set does not depend
// on the cell geometry.
template <class F>
__device__ __forceinline__ void for_each_neighbor_generic(const KParams& P, double delta,
                                                          const double* __restrict__ pos,
                                                          const int* __restrict__ cell_start, int i,
                                                          double xi, double yi, double zi, F&& visit)
{
    const int np = P.npad;
    auto scan = [&](int s0, int s1) {
        for (int j = s0; j < s1; ++j) {
            if (j == i) continue;
            double dx, dy, dz;
            const double nimg = min_image(P, delta, xi, yi, zi, pos[j], pos[np + j], pos[2 * np + j],
                                          dx, dy, dz);
            const double r2 = sq_norm_exact(dx, dy, dz);
            if (r2 < P.rc2) visit(j, dx, dy, dz, nimg, r2);
        }
    };
    if (P.ncell == 1) {
        scan(0, P.n);
        return;
    }
    const int nc0 = P.nc[0], nc1 = P.nc[1], nc2 = P.nc[2];
    const bool zall = nc2 < 3, yall = nc1 < 3, xall = (nc0 < 3) || yall;
    const int cx = cell_coord(xi, P.inv_cw[0], nc0);
    const int cy = cell_coord(yi, P.inv_cw[1], nc1);
    const int cz = cell_coord(zi, P.inv_cw[2], nc2);
    const int zlo = zall ? 0 : -1, zhi = zall ? nc2 - 1 : 1;
    const int ylo = yall ? 0 : -1, yhi = yall ? nc1 - 1 : 1;
    for (int dzc = zlo; dzc <= zhi; ++dzc) {
        int czz = zall ? dzc : cz + dzc;
        if (czz < 0) czz += nc2;
        if (czz >= nc2) czz -= nc2;
        for (int dyc = ylo; dyc <= yhi; ++dyc) {
            int cyy, m = 0;
            if (yall) {
                cyy = dyc;
            } else {
                cyy = cy + dyc;
                if (cyy < 0) {
                    cyy += nc1;
                    m = -1;
                } else if (cyy >= nc1) {
                    cyy -= nc1;
                    m = 1;
                }
            }
            const int rowbase = (czz * nc1 + cyy) * nc0;
            if (xall) {
                scan(cell_start[rowbase], cell_start[rowbase + nc0]);
                continue;
            }
            int cxc = cx;
            if (m != 0) cxc = cell_coord(wrap_box(xi - (double)m * delta, P.L[0]), P.inv_cw[0], nc0);
            const int lo = cxc - 1, hi = cxc + 1;
            if (lo < 0) {
                scan(cell_start[rowbase + nc0 - 1], cell_start[rowbase + nc0]);
                scan(cell_start[rowbase], cell_start[rowbase + hi + 1]);
            } else if (hi >= nc0) {
                scan(cell_start[rowbase + lo], cell_start[rowbase + nc0]);
                scan(cell_start[rowbase], cell_start[rowbase + 1]);
            } else {
                scan(cell_start[rowbase + lo], cell_start[rowbase + hi + 1]);
            }
        }
    }
}

__device__ __forceinline__ int floor_div(int a, int b)
{
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

// The same pair set as for_each_neighbor_generic for boxes with >= 3 cells per
// axis, with most of the FP64 work removed.  Each candidate cell is visited as
// one image of the box (integer shifts a, m, c along x, y, z), so the image
// separation R_i - (R_j + a L_x x + m (L_y y + delta x) + c L_z z) is first
// evaluated in FP32 from FP32 positions.  Its squared length differs from the
// exact one by less than the margin kept in rc2_lo / rc2_hi (bounded from the
// FP32 rounding of positions, shifts, differences and sums, for box edges up
// to L: 2^-24 (256 L r_c + 64 r_c^2)), so candidates outside the margin band
// are decided by the FP32 value, and the few inside it by the exact FP64
// predicate.  For an accepted pair the exact separation is the canonical
// minimum image with n = m and the rounded quotients equal to a and c (at most
// one image of j lies within r_c of i because every box edge is >= 3 r_c), so
// it is evaluated with those integers and the same rounded operations,
// without divisions.  FP32 arithmetic uses explicit round-to-nearest
// intrinsics so that the counting and filling passes decide identically.
template <bool NEED_D, class F>
__device__ __forceinline__ void for_each_neighbor_fast(const KParams& P, double delta,
                                                       const double* __restrict__ pos,
                                                       const float* __restrict__ pos32,
                                                       const int* __restrict__ cell_start, int i,
                                                       double xi, double yi, double zi, F&& visit)
{
    const int np = P.npad;
    const int nc0 = P.nc[0], nc1 = P.nc[1], nc2 = P.nc[2];
    const float xf = pos32[i], yf = pos32[np + i], zf = pos32[2 * np + i];
    const float deltaf = (float)delta;
    const int cx = cell_coord(xi, P.inv_cw[0], nc0);
    const int cy = cell_coord(yi, P.inv_cw[1], nc1);
    const int cz = cell_coord(zi, P.inv_cw[2], nc2);
    for (int dzc = -1; dzc <= 1; ++dzc) {
        int czz = cz + dzc, c_img = 0;
        if (czz < 0) {
            czz += nc2;
            c_img = -1;
        } else if (czz >= nc2) {
            czz -= nc2;
            c_img = 1;
        }
        const float szf = __fmul_rn((float)c_img, P.Lf[2]);
        for (int dyc = -1; dyc <= 1; ++dyc) {
            int cyy = cy + dyc, m = 0;
            if (cyy < 0) {
                cyy += nc1;
                m = -1;
            } else if (cyy >= nc1) {
                cyy -= nc1;
                m = 1;
            }
            const float syf = __fmul_rn((float)m, P.Lf[1]);
            const int cxu0 = m == 0 ? cx : (int)floor((xi - (double)m * delta) * P.inv_cw[0]);
            const int rowbase = (czz * nc1 + cyy) * nc0;
            for (int dxc = -1; dxc <= 1; ++dxc) {
                const int cxu = cxu0 + dxc;
                const int a = floor_div(cxu, nc0);
                const int c = rowbase + (cxu - a * nc0);
                const float sxf = __fadd_rn(__fmul_rn((float)m, deltaf), __fmul_rn((float)a, P.Lf[0]));
                const int j1 = cell_start[c + 1];
                for (int j = cell_start[c]; j < j1; ++j) {
                    if (j == i) continue;
                    const float dxf = __fsub_rn(__fsub_rn(xf, pos32[j]), sxf);
                    const float dyf = __fsub_rn(__fsub_rn(yf, pos32[np + j]), syf);
                    const float dzf = __fsub_rn(__fsub_rn(zf, pos32[2 * np + j]), szf);
                    const float r2f = __fadd_rn(__fadd_rn(__fmul_rn(dxf, dxf), __fmul_rn(dyf, dyf)),
                                                __fmul_rn(dzf, dzf));
                    if (r2f >= P.rc2_hi) continue;
                    if (r2f < P.rc2_lo) {
                        if (NEED_D) {
                            const double xj = pos[j], yj = pos[np + j], zj = pos[2 * np + j];
                            const double n = (double)m;
                            const double dx = __dsub_rn(__dsub_rn(__dsub_rn(xi, xj), __dmul_rn(n, delta)),
                                                        __dmul_rn(P.L[0], (double)a));
                            const double dy = __dsub_rn(__dsub_rn(yi, yj), __dmul_rn(n, P.L[1]));
                            const double dz = __dsub_rn(__dsub_rn(zi, zj), __dmul_rn(P.L[2], (double)c_img));
                            visit(j, dx, dy, dz, n, sq_norm_exact(dx, dy, dz));
                        } else {
                            visit(j, 0.0, 0.0, 0.0, 0.0, 0.0);
                        }
                    } else {
                        double dx, dy, dz;
                        const double n = min_image(P, delta, xi, yi, zi, pos[j], pos[np + j],
                                                   pos[2 * np + j], dx, dy, dz);
                        const double r2 = sq_norm_exact(dx, dy, dz);
                        if (r2 < P.rc2) visit(j, dx, dy, dz, n, r2);
                    }
                }
            }
        }
    }
}

template <bool NEED_D, class F>
__device__ __forceinline__ void for_each_neighbor(const KParams& P, double delta,
                                                  const double* __restrict__ pos,
                                                  const float* __restrict__ pos32,
                                                  const int* __restrict__ cell_start, int i,
                                                  double xi, double yi, double zi, F&& visit)
{
    if (P.fast_cells)
        for_each_neighbor_fast<NEED_D>(P, delta, pos, pos32, cell_start, i, xi, yi, zi, visit);
    else
        for_each_neighbor_generic(P, delta, pos, cell_start, i, xi, yi, zi, visit);
}

__global__ void k_nbr_count(KParams P, const double* __restrict__ pos, const float* __restrict__ pos32,
                            const int* __restrict__ cell_start, int* __restrict__ row_cnt,
                            const DevState* st)
{
    if (st->error | st->overflow) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const double delta = st->delta;
    const int np = P.npad;
    int cnt = 0;
    for_each_neighbor<false>(P, delta, pos, pos32, cell_start, i, pos[i], pos[np + i], pos[2 * np + i],
                             [&](int, double, double, double, double, double) { ++cnt; });
    row_cnt[i] = cnt;
}

void launch_nbr_count(const KParams& P, DevBuffers& B, Launch L)
{
    k_nbr_count<<<grid_for(P.n, 128, 1 << 30), 128, 0, L.stream>>>(P, B.pos_w, B.pos32, B.cell_start,
                                                                    B.row_cnt, B.st);
}

// Row i of Eq. algebra from its pair sums (§Method, Eq. F and Eq. vc):
//   A_ii = 1 + alpha sum_j w_ij
//   F_i  = noise_amp xi_i + c_ev sum_j R_ij w_ij + zeta kappa (y_i - L_y/2) x
//   b_i  = F_i / zeta + alpha kappa L_y (sum_j n_ij w_ij) x
__device__ __forceinline__ void finish_row(const KParams& P, const DevBuffers& B, int i, double yi,
                                           unsigned long long step, int use_inj, double sw,
                                           double fx, double fy, double fz, double nw)
{
    const int np = P.npad;
    const double d = 1.0 + P.alpha * sw;
    B.diag[i] = d;
    B.dinv[i] = 1.0 / d;
    B.diag32[i] = (float)d;
    B.dinv32[i] = (float)(1.0 / d);
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    if (P.noise_amp != 0.0) {
        const int id = B.id_w[i];
        if (use_inj) {
            g0 = B.xi_inj[3 * (long long)id];
            g1 = B.xi_inj[3 * (long long)id + 1];
            g2 = B.xi_inj[3 * (long long)id + 2];
        } else {
            normals3(P.seed, step, (unsigned long long)id, g0, g1, g2);
        }
    }
    double F0 = P.noise_amp * g0 + P.c_ev * fx;
    const double F1 = P.noise_amp * g1 + P.c_ev * fy;
    const double F2 = P.noise_amp * g2 + P.c_ev * fz;
    F0 += P.zeta * P.kappa * (yi - 0.5 * P.L[1]);
    B.b[i] = F0 / P.zeta + P.alpha * P.kappa * P.L[1] * nw;
    B.b[np + i] = F1 / P.zeta;
    B.b[2 * np + i] = F2 / P.zeta;
}

// Pair search writing the CSR columns; with ASSEMBLE also the weights and the
// row of Eq. algebra in the same pass.
template <bool ASSEMBLE>
__global__ void k_nbr_fill(KParams P, DevBuffers B, int use_inj)
{
    DevState* st = B.st;
    if (st->error | st->overflow) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const double delta = st->delta;
    const unsigned long long step = (unsigned long long)st->step;
    const int np = P.npad;
    const double xi = B.pos_w[i], yi = B.pos_w[np + i], zi = B.pos_w[2 * np + i];
    int k = B.row_ptr[i];
    const int kend = B.row_ptr[i + 1];
    double sw = 0.0, fx = 0.0, fy = 0.0, fz = 0.0, nw = 0.0;
    int* __restrict__ col = B.col;
    double* __restrict__ val = B.val;
    float* __restrict__ val32 = B.val32;
    for_each_neighbor<ASSEMBLE>(P, delta, B.pos_w, B.pos32, B.cell_start, i, xi, yi, zi,
                                [&](int j, double dx, double dy, double dz, double nimg, double r2) {
                                    if (k < kend) {
                                        col[k] = j;
                                        if (ASSEMBLE) {
                                            const double w = exp(-r2 / P.two_lambda2);
                                            val[k] = w;
                                            val32[k] = (float)w;
                                            sw += w;
                                            fx += dx * w;
                                            fy += dy * w;
                                            fz += dz * w;
                                            nw += nimg * w;
                                        }
                                    }
                                    ++k;
                                });
    // the counting pass and this one must agree; a mismatch is reported, never written past
    if (k != kend) atomicCAS(&st->error, 0, (int)SP_ERR_INVALID_ARG);
    if (ASSEMBLE) finish_row(P, B, i, yi, step, use_inj, sw, fx, fy, fz, nw);
}

void launch_nbr_fill(const KParams& P, DevBuffers& B, bool assemble, bool use_inj, bool mixed,
                     Launch L)
{
    (void)mixed;
    const int g = grid_for(P.n, 128, 1 << 30);
    if (assemble)
        k_nbr_fill<true><<<g, 128, 0, L.stream>>>(P, B, use_inj ? 1 : 0);
    else
        k_nbr_fill<false><<<g, 128, 0, L.stream>>>(P, B, use_inj ? 1 : 0);
}

// Assembly from an existing pair list (same arithmetic and order as the fused pass).
__global__ void k_assemble(KParams P, DevBuffers B, int use_inj)
{
    const DevState* st = B.st;
    if (st->error | st->overflow) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const double delta = st->delta;
    const unsigned long long step = (unsigned long long)st->step;
    const int np = P.npad;
    const double xi = B.pos_w[i], yi = B.pos_w[np + i], zi = B.pos_w[2 * np + i];
    double sw = 0.0, fx = 0.0, fy = 0.0, fz = 0.0, nw = 0.0;
    for (int k = B.row_ptr[i]; k < B.row_ptr[i + 1]; ++k) {
        const int j = B.col[k];
        double dx, dy, dz;
        const double nimg = min_image(P, delta, xi, yi, zi, B.pos_w[j], B.pos_w[np + j],
                                      B.pos_w[2 * np + j], dx, dy, dz);
        const double r2 = sq_norm_exact(dx, dy, dz);
        const double w = exp(-r2 / P.two_lambda2);
        B.val[k] = w;
        B.val32[k] = (float)w;
        sw += w;
        fx += dx * w;
        fy += dy * w;
        fz += dz * w;
        nw += nimg * w;
    }
    finish_row(P, B, i, yi, step, use_inj, sw, fx, fy, fz, nw);
}

void launch_assemble_only(const KParams& P, DevBuffers& B, bool use_inj, bool mixed, Launch L)
{
    (void)mixed;
    k_assemble<<<grid_for(P.n, 128, 1 << 30), 128, 0, L.stream>>>(P, B, use_inj ? 1 : 0);
}

// ------------------------------------------------------ generator utilities

// Uniform positions in the box, by id, from Philox with key (seed, 1).
__global__ void k_uniform_positions(KParams P, double* __restrict__ pos, int* __restrict__ id)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    unsigned long long c[4] = {(unsigned long long)i, 0ull, 0ull, 0ull};
    philox4x64_10(c, P.seed, 1ull);
    const double s53 = 1.0 / 9007199254740992.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double x = (double)(c[a] >> 11) * s53 * P.L[a];
        if (x >= P.L[a]) x = 0.0;
        pos[a * P.npad + i] = x;
    }
    id[i] = i;
}

void launch_uniform_positions(const KParams& P, DevBuffers& B, Launch L)
{
    k_uniform_positions<<<grid_for(P.n, kVecBlock, 1 << 30), kVecBlock, 0, L.stream>>>(P, B.pos_s,
                                                                                          B.id_s);
}

__global__ void k_philox_blocks(unsigned long long seed, unsigned long long step, long long count,
                                const long long* __restrict__ ids, unsigned long long* __restrict__ out)
{
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= count) return;
    unsigned long long c[4] = {(unsigned long long)ids[k], step, 0ull, 0ull};
    philox4x64_10(c, seed, 0ull);
#pragma unroll
    for (int a = 0; a < 4; ++a) out[4 * k + a] = c[a];
}

void launch_philox_blocks(unsigned long long seed, unsigned long long step, long long count,
                          const long long* ids, unsigned long long* out, cudaStream_t s)
{
    k_philox_blocks<<<grid_for(count, kVecBlock, 1 << 30), kVecBlock, 0, s>>>(seed, step, count, ids, out);
}

}  // namespace ss
