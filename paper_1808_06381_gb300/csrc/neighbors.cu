// Cell list with sheared periodic images, pair search, and the fused pair
// kernel that emits the forces of Eq. F and the friction matrix of Eq. algebra
// (arXiv 1808.06381, §Method).
//
// Rows are kept in cell order: each step re-sorts the particles by cell with a
// counting sort (histogram, exclusive scan, scatter) and orders the particles
// of a cell by id, so the order is deterministic.  Cells are numbered in
// tiles of 8^3 (Morton order inside a tile, cell_index), so that the rows of
// one block of the solver cover a compact region of space and neighbours sit
// close in memory for the solver's gathers.
#include <array>
#include <cmath>

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
    const int c = cell_index(P, cx, cy, cz);
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
// chunk-local rescan.  mode 2 also records the total as the padded matrix
// size and raises the overflow flag if it exceeds cap_check.

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
        if (mode == 2) {
            st->nnz_slots = carry;
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

// An input of at most TH x kScanItems in one block: its exclusive scan and
// the total (one launch instead of three; TH = 1024 covers the 8,192 chunk
// lengths of a 262,144-row sliced layout).
template <int TH>
__global__ void __launch_bounds__(TH) k_scan_single(const int* __restrict__ in, int* __restrict__ out, int n,
                                                    long long cap_check, DevState* st, int mode)
{
    if (st->error | st->overflow) return;
    __shared__ int s[TH * kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int idx = k * TH + threadIdx.x;
        s[idx] = idx < n ? in[idx] : 0;
    }
    __syncthreads();
    int loc[kScanItems];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        loc[k] = sum;
        sum += s[threadIdx.x * kScanItems + k];
    }
    int tot;
    const int off = block_exclusive_scan_int(sum, &tot);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) s[threadIdx.x * kScanItems + k] = loc[k] + off;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int idx = k * TH + threadIdx.x;
        if (idx < n) out[idx] = s[idx];
    }
    if (threadIdx.x == 0) {
        out[n] = tot;
        if (mode == 2) {
            st->nnz_slots = tot;
            if (tot > cap_check) st->overflow = 1;
        }
    }
}

int launch_scan(const int* in, int* out, int n, int* block_tmp, long long cap_check, DevState* st, int mode,
                Launch L)
{
    const int nb = (n + kScanChunk - 1) / kScanChunk;
    if (nb <= 1) {
        k_scan_single<kScanThreads><<<1, kScanThreads, 0, L.stream>>>(in, out, n, cap_check, st, mode);
        return 1;
    }
    if (n <= 1024 * kScanItems) {
        k_scan_single<1024><<<1, 1024, 0, L.stream>>>(in, out, n, cap_check, st, mode);
        return 1;
    }
    k_scan_reduce<<<nb, kScanThreads, 0, L.stream>>>(in, n, block_tmp, st);
    k_scan_top<<<1, 1024, 0, L.stream>>>(block_tmp, nb, out, n, cap_check, st, mode);
    k_scan_down<<<nb, kScanThreads, 0, L.stream>>>(in, out, n, block_tmp, st);
    return 3;
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
// k_bin are not deterministic) and record the cell of its rows.
__global__ void k_sort_cells(KParams P, const int* __restrict__ cell_start, int* __restrict__ perm,
                             const int* __restrict__ id_s, int* __restrict__ cell_w, const DevState* st)
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
    for (int k = beg; k < end; ++k) cell_w[k] = c;   // the cell of row k (the pair search reads it)
}

// One thread per row: positions (FP64 and as double-floats), id and the
// warm-start velocities of row k from its particle's row s of the state.
__global__ void k_gather_rows(KParams P, const int* __restrict__ perm, const int* __restrict__ id_s,
                              const double* __restrict__ pos_s, const double* __restrict__ v_s,
                              double* __restrict__ pos_w, float* __restrict__ pos32, float* __restrict__ pos32lo,
                              int* __restrict__ id_w, double* __restrict__ x, int warm, const DevState* st)
{
    if (st->error | st->overflow) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P.n) return;
    const int np = P.npad;
    const int s = perm[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double v = pos_s[a * np + s];
        pos_w[a * np + k] = v;
        const float vh = (float)v;
        pos32[a * np + k] = vh;
        pos32lo[a * np + k] = (float)(v - (double)vh);
    }
    id_w[k] = id_s[s];
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a * np + k] = warm ? v_s[a * np + s] : 0.0;
}

int launch_scatter_sort_gather(const KParams& P, DevBuffers& B, bool warm, Launch L)
{
    k_scatter<<<grid_for(P.n, kVecBlock, 1 << 30), kVecBlock, 0, L.stream>>>(P.n, B.cell_of, B.slot,
                                                                                B.cell_start, B.perm, B.st);
    k_sort_cells<<<grid_for(P.ncell, 128, 1 << 30), 128, 0, L.stream>>>(P, B.cell_start, B.perm, B.id_s, B.cell_of,
                                                                         B.st);
    k_gather_rows<<<grid_for(P.n, kVecBlock, 1 << 30), kVecBlock, 0, L.stream>>>(
        P, B.perm, B.id_s, B.pos_s, B.v_s, B.pos_w, B.pos32, B.pos32lo, B.id_w, B.x, warm ? 1 : 0, B.st);
    return 3;
}

// Single-cell boxes (every edge below 3 r_c): keep the state order.
__global__ void k_identity_gather(KParams P, const int* __restrict__ id_s,
                                  const double* __restrict__ pos_s, const double* __restrict__ v_s,
                                  double* __restrict__ pos_w, float* __restrict__ pos32,
                                  float* __restrict__ pos32lo, int* __restrict__ id_w, double* __restrict__ x, int* __restrict__ perm,
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
        const double v = pos_s[a * np + k];
        pos_w[a * np + k] = v;
        const float vh = (float)v;
        pos32[a * np + k] = vh;
        pos32lo[a * np + k] = (float)(v - (double)vh);
        x[a * np + k] = warm ? v_s[a * np + k] : 0.0;
    }
}

void launch_identity_gather(const KParams& P, DevBuffers& B, bool warm, Launch L)
{
    k_identity_gather<<<grid_for(P.n, kVecBlock, 1 << 30), kVecBlock, 0, L.stream>>>(
        P, B.id_s, B.pos_s, B.v_s, B.pos_w, B.pos32, B.pos32lo, B.id_w, B.x, B.perm, warm ? 1 : 0, B.st);
}

// ------------------------------------------------------------- pair search

// The exact predicate |R|^2 < r_c^2 of a candidate in the FP32 margin band,
// in FP64 at the image (code) the cell walk found.  Not inlined: the band
// holds ~0.03 candidates per row, and inlined FP64 work would be predicated
// into every candidate's path on GB300's 1/64-rate FP64 pipe.
__device__ __noinline__ bool band_pair(const KParams& P, double delta, double xi, double yi, double zi,
                                       const double* __restrict__ pos, int np, int j, unsigned char code)
{
    double dx, dy, dz;
    image_separation(P, delta, xi, yi, zi, pos[j], pos[np + j], pos[2 * np + j], code, dx, dy, dz);
    return sq_norm_exact(dx, dy, dz) < P.rc2;
}

// Canonical minimum image (min_image) that also reports the two rounded
// quotients, i.e. the image of the partner as a code.
__device__ __forceinline__ unsigned char min_image_code(const KParams& P, double delta, double xi,
                                                        double yi, double zi, double xj, double yj,
                                                        double zj, double& r2)
{
    double dx = __dsub_rn(xi, xj);
    double dy = __dsub_rn(yi, yj);
    double dz = __dsub_rn(zi, zj);
    const double n = round(__ddiv_rn(dy, P.L[1]));
    dy = __dsub_rn(dy, __dmul_rn(n, P.L[1]));
    dx = __dsub_rn(dx, __dmul_rn(n, delta));
    const double a = round(__ddiv_rn(dx, P.L[0]));
    dx = __dsub_rn(dx, __dmul_rn(P.L[0], a));
    const double c = round(__ddiv_rn(dz, P.L[2]));
    dz = __dsub_rn(dz, __dmul_rn(P.L[2], c));
    r2 = sq_norm_exact(dx, dy, dz);
    return image_code((int)a, (int)n, (int)c);
}

// Visit every j != i with |R_ij|^2 < r_c^2 (the 5 % truncation of §Method),
// passing the image code of the partner.  Candidate cells: the 3 x 3 x 3 block
// around i's cell; a row of cells that wraps through y = 0 or y = L_y belongs
// to the image displaced by -/+ delta in x, so its three x cells are centred
// on x_i +/- delta.  Axes with fewer than 3 cells are scanned whole (and then
// x is scanned whole when y is).  Every candidate goes through the exact
// predicate, so the pair set does not depend on the cell geometry.
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
            double r2;
            const unsigned char code = min_image_code(P, delta, xi, yi, zi, pos[j], pos[np + j], pos[2 * np + j], r2);
            if (r2 < P.rc2) visit(j, code);
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
    auto scan_cell = [&](int ax, int ay, int az) {
        const int c = cell_index(P, ax, ay, az);
        scan(cell_start[c], cell_start[c + 1]);
    };
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
            if (xall) {
                for (int ax = 0; ax < nc0; ++ax) scan_cell(ax, cyy, czz);
                continue;
            }
            int cxc = cx;
            if (m != 0) cxc = cell_coord(wrap_box(xi - (double)m * delta, P.L[0]), P.inv_cw[0], nc0);
            for (int dxc = -1; dxc <= 1; ++dxc) {
                int ax = cxc + dxc;
                if (ax < 0) ax += nc0;
                if (ax >= nc0) ax -= nc0;
                scan_cell(ax, cyy, czz);
            }
        }
    }
}

// The same pair set as for_each_neighbor_generic for boxes with >= 3 cells per
// axis, with almost no FP64 work.  Each candidate cell is visited as one image
// of the box (integer shifts a, m, c along x, y, z), so the image separation
// R_i - (R_j + a L_x x + m (L_y y + delta x) + c L_z z) is first evaluated in
// FP32 from FP32 positions.  Its squared length differs from the exact one by
// less than the margin kept in rc2_lo / rc2_hi (bounded from the FP32 rounding
// of positions, shifts, differences and sums, for box edges up to L:
// 2^-24 (256 L r_c + 64 r_c^2)), so candidates outside the margin band are
// decided by the FP32 value and the few inside it by the exact FP64
// predicate.  At most one image of j lies within r_c of i because every box
// edge is >= 3 r_c, so the image found here is the canonical minimum image of
// every accepted pair.  FP32 arithmetic uses explicit round-to-nearest
// intrinsics so that the counting and filling passes decide identically.
template <class F>
__device__ __forceinline__ void for_each_neighbor_fast(const KParams& P, double delta,
                                                       const double* __restrict__ pos,
                                                       const float* __restrict__ pos32,
                                                       const int* __restrict__ cell_start,
                                                       const int* __restrict__ cell_w, int i,
                                                       double xi, double yi, double zi, F&& visit)
{
    const int np = P.npad;
    const int nc0 = P.nc[0], nc1 = P.nc[1], nc2 = P.nc[2];
    const float xf = pos32[i], yf = pos32[np + i], zf = pos32[2 * np + i];
    const float deltaf = (float)delta;
    // the row's cell coordinates from its cell index (integer work; the
    // binning computed the index from the same FP64 position)
    const int ci = cell_w[i];
    const int tl = ci >> 9, lc = ci & 511;
    const int tx = tl % P.ntile[0], ty = (tl / P.ntile[0]) % P.ntile[1], tz = tl / (P.ntile[0] * P.ntile[1]);
    const int cx = 8 * tx + ((lc & 1) | ((lc >> 2) & 2) | ((lc >> 4) & 4));
    const int cy = 8 * ty + (((lc >> 1) & 1) | ((lc >> 3) & 2) | ((lc >> 5) & 4));
    const int cz = 8 * tz + (((lc >> 2) & 1) | ((lc >> 4) & 2) | ((lc >> 6) & 4));
    // x cell of x_i - m delta for the rows of cells that wrap through y (m = -1, +1):
    // FP64, so only for rows whose cell touches a y face
    int cx_m1 = cx, cx_p1 = cx;
    if (cy == 0 || cy == nc1 - 1) {
        cx_m1 = (int)floor((xi + delta) * P.inv_cw[0]);
        cx_p1 = (int)floor((xi - delta) * P.inv_cw[0]);
    }
    // image shifts by selection (no int-to-float conversions: GB300 runs them
    // at the FP64 rate); every product below is exact, as before
    auto times = [](int k, float v) { return k == 0 ? 0.f : (k > 0 ? v : -v); };
    const float L2f = 2.f * P.Lf[0];
    for (int dzc = -1; dzc <= 1; ++dzc) {
        int czz = cz + dzc, c_img = 0;
        if (czz < 0) {
            czz += nc2;
            c_img = -1;
        } else if (czz >= nc2) {
            czz -= nc2;
            c_img = 1;
        }
        const float szf = times(c_img, P.Lf[2]);
        for (int dyc = -1; dyc <= 1; ++dyc) {
            int cyy = cy + dyc, m = 0;
            if (cyy < 0) {
                cyy += nc1;
                m = -1;
            } else if (cyy >= nc1) {
                cyy -= nc1;
                m = 1;
            }
            const float syf = times(m, P.Lf[1]);
            const float mdf = times(m, deltaf);
            const int cxu0 = m == 0 ? cx : (m > 0 ? cx_p1 : cx_m1);
            for (int dxc = -1; dxc <= 1; ++dxc) {
                const int cxu = cxu0 + dxc;
                // floor(cxu / nc0) for cxu in [-2 nc0, 3 nc0)
                const int a = cxu >= 0 ? (cxu >= nc0 ? (cxu >= 2 * nc0 ? 2 : 1) : 0) : (cxu >= -nc0 ? -1 : -2);
                const int c = cell_index(P, cxu - a * nc0, cyy, czz);
                const float axf = a == 0 ? 0.f : (a == 1 ? P.Lf[0] : (a == -1 ? -P.Lf[0] : (a == 2 ? L2f : -L2f)));
                const float sxf = __fadd_rn(mdf, axf);
                const unsigned char code = image_code(a, m, c_img);
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
                        visit(j, code);
                    } else {
                        // the margin band: the exact FP64 predicate at the image the walk
                        // found, which is the canonical one of min_image_code for any |R|
                        // below L / 2 (bit-identical, without its three FP64 divisions:
                        // GB300 issues FP64 at 1/64 of the FP32 rate, and the warp waits)
                        if (band_pair(P, delta, xi, yi, zi, pos, np, j, code)) visit(j, code);
                    }
                }
            }
        }
    }
}

template <class F>
__device__ __forceinline__ void for_each_neighbor(const KParams& P, double delta,
                                                  const double* __restrict__ pos,
                                                  const float* __restrict__ pos32,
                                                  const int* __restrict__ cell_start,
                                                  const int* __restrict__ cell_w, int i,
                                                  double xi, double yi, double zi, F&& visit)
{
    if (P.fast_cells)
        for_each_neighbor_fast(P, delta, pos, pos32, cell_start, cell_w, i, xi, yi, zi, visit);
    else
        for_each_neighbor_generic(P, delta, pos, cell_start, i, xi, yi, zi, visit);
}

// The pair search of a step, run once: counts the partners of every row and
// keeps the first kCandCap of them (partner and image code, k-major so that a
// warp's stores are coalesced) for the assembly, which places them in the
// sliced layout.
__global__ void k_nbr_collect(KParams P, DevBuffers B, int draw_noise)
{
    DevState* st = B.st;
    if (st->error | st->overflow) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        st->nnz = 0;
        if (draw_noise != 2) st->noise_step = draw_noise ? st->step : -1;   // 2: drawn by k_row_normals
    }
    if (i >= P.n) return;
    if (draw_noise == 1) {   // the step's normals of this row (the assembly uses them)
        if (P.mixed) {   // double-float arithmetic; stored as (hi, lo) pairs in the same space
            dfloat g0, g1, g2;
            normals3_df(B.rng_tab, P.seed, (unsigned long long)st->step, (unsigned long long)B.id_w[i], g0, g1, g2);
            float2* n2 = reinterpret_cast<float2*>(B.noise3);
            n2[i] = make_float2(g0.hi, g0.lo);
            n2[P.npad + i] = make_float2(g1.hi, g1.lo);
            n2[2 * P.npad + i] = make_float2(g2.hi, g2.lo);
        } else {
            double g0, g1, g2;
            normals3(P.seed, (unsigned long long)st->step, (unsigned long long)B.id_w[i], g0, g1, g2);
            B.noise3[i] = g0;
            B.noise3[P.npad + i] = g1;
            B.noise3[2 * P.npad + i] = g2;
        }
    }
    const double delta = st->delta;
    const int np = P.npad;
    int cnt = 0;
    int* __restrict__ cj = B.cand_j;
    unsigned char* __restrict__ ci = B.cand_img;
    for_each_neighbor(P, delta, B.pos_w, B.pos32, B.cell_start, B.cell_of, i, B.pos_w[i], B.pos_w[np + i],
                      B.pos_w[2 * np + i], [&](int j, unsigned char code) {
                          if (cnt < kCandCap) {
                              cj[(size_t)cnt * np + i] = j;
                              ci[(size_t)cnt * np + i] = code;
                          }
                          ++cnt;
                      });
    B.row_cnt[i] = cnt;
}

// The step's normals of every row as the pair search draws them, in a kernel
// of their own (so that they can run beside the search).
__global__ void k_row_normals(KParams P, DevBuffers B)
{
    DevState* st = B.st;
    if (st->error | st->overflow) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) st->noise_step = st->step;
    if (i >= P.n) return;
    if (P.mixed) {
        dfloat g0, g1, g2;
        normals3_df(B.rng_tab, P.seed, (unsigned long long)st->step, (unsigned long long)B.id_w[i], g0, g1, g2);
        float2* n2 = reinterpret_cast<float2*>(B.noise3);
        n2[i] = make_float2(g0.hi, g0.lo);
        n2[P.npad + i] = make_float2(g1.hi, g1.lo);
        n2[2 * P.npad + i] = make_float2(g2.hi, g2.lo);
    } else {
        double g0, g1, g2;
        normals3(P.seed, (unsigned long long)st->step, (unsigned long long)B.id_w[i], g0, g1, g2);
        B.noise3[i] = g0;
        B.noise3[P.npad + i] = g1;
        B.noise3[2 * P.npad + i] = g2;
    }
}

int launch_nbr_count(const KParams& P, DevBuffers& B, bool draw_noise, Launch L, cudaStream_t side, cudaEvent_t* ev)
{
    if (draw_noise && side && ev) {   // the normals beside the search, joined before anything after it
        cudaEventRecord(ev[0], L.stream);
        cudaStreamWaitEvent(side, ev[0], 0);
        k_row_normals<<<grid_for(P.n, 256, 1 << 30), 256, 0, side>>>(P, B);
        cudaEventRecord(ev[1], side);
        k_nbr_collect<<<grid_for(P.n, 128, 1 << 30), 128, 0, L.stream>>>(P, B, 2);
        cudaStreamWaitEvent(L.stream, ev[1], 0);
        return 2;
    }
    k_nbr_collect<<<grid_for(P.n, 128, 1 << 30), 128, 0, L.stream>>>(P, B, draw_noise ? 1 : 0);
    return 1;
}

// Slices of the matrix: inside each window of 256 rows, rank the rows by
// length (longest first, ties by row) so that each chunk of 32 ranked rows has
// rows of nearly equal length; a chunk is stored column-major with the length
// of its longest row.  Also sums the entries of the matrix.
__global__ void __launch_bounds__(256) k_sell_plan(KParams P, DevBuffers B)
{
    DevState* st = B.st;
    if (st->error | st->overflow) return;
    __shared__ int cnt_s[256];
    __shared__ double sh[32];
    const int t = threadIdx.x;
    const int row = blockIdx.x * 256 + t;
    const int c = row < P.n ? B.row_cnt[row] : -1;
    cnt_s[t] = c;
    __syncthreads();
    int rank = 0;
    for (int u = 0; u < 256; ++u) {
        const int cu = cnt_s[u];
        rank += (cu > c) || (cu == c && u < t);
    }
    const int slot = blockIdx.x * 256 + rank;
    B.slot_row[slot] = row < P.n ? row : -1;
    if (row < P.n) B.row_slot[row] = slot;
    if ((rank & 31) == 0) B.chunk_len32[slot >> 5] = (c > 0 ? c : 0) * 32;
    const double tot = block_sum((double)(c > 0 ? c : 0), sh);
    if (t == 0) atomicAdd((unsigned long long*)&st->nnz, (unsigned long long)tot);
}

void launch_sell_plan(const KParams& P, DevBuffers& B, Launch L)
{
    k_sell_plan<<<P.nslots / 256, 256, 0, L.stream>>>(P, B);
}

// Row i of Eq. algebra from its pair sums (§Method, Eq. F and Eq. vc):
//   A_ii = 1 + alpha sum_j w_ij
//   F_i  = noise_amp xi_i + c_ev sum_j R_ij w_ij + zeta kappa (y_i - L_y/2) x
//   b_i  = F_i / zeta + alpha kappa L_y (sum_j n_ij w_ij) x
__device__ __forceinline__ void finish_row(const KParams& P, const DevBuffers& B, int i, double yi,
                                           unsigned long long step, int use_inj, bool drawn, double sw,
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
        } else if (drawn) {   // drawn by the pair search of this step
            g0 = B.noise3[i];
            g1 = B.noise3[np + i];
            g2 = B.noise3[2 * np + i];
        } else {
            normals3(P.seed, step, (unsigned long long)id, g0, g1, g2);
        }
    }
    double F0 = P.noise_amp * g0 + P.c_ev * fx;
    const double F1 = P.noise_amp * g1 + P.c_ev * fy;
    const double F2 = P.noise_amp * g2 + P.c_ev * fz;
    F0 += P.zeta * P.kappa * (yi - 0.5 * P.L[1]);
    const double b0 = F0 / P.zeta + P.alpha * P.kappa * P.L[1] * nw, b1 = F1 / P.zeta, b2 = F2 / P.zeta;
    B.b[i] = b0;
    B.b[np + i] = b1;
    B.b[2 * np + i] = b2;
}

// The same row of the mixed path, in double-float on the FP32 pipes from the
// double-float pair sums and normals: A_ii and b as double-floats (A_ii =
// diag32 + diag32lo, b = bdf), D^-1 in FP32 for the Jacobi iterations.
__device__ __forceinline__ void finish_row_df(const KParams& P, const DevBuffers& B, int i, dfloat yi,
                                              unsigned long long step, int use_inj, bool drawn, dfloat sw,
                                              dfloat fx, dfloat fy, dfloat fz, dfloat nw)
{
    const int np = P.npad;
    const dfloat d = df_add(dfloat{1.f, 0.f}, df_mul(dfloat{P.alpha_hi, P.alpha_lo}, sw));
    B.diag32[i] = d.hi;
    B.diag32lo[i] = d.lo;
    B.dinv32[i] = __frcp_rn(d.hi);
    dfloat g0{0.f, 0.f}, g1{0.f, 0.f}, g2{0.f, 0.f};
    if (P.noise_amp != 0.0) {
        const int id = B.id_w[i];
        if (use_inj) {
            g0 = df_split(B.xi_inj[3 * (long long)id]);
            g1 = df_split(B.xi_inj[3 * (long long)id + 1]);
            g2 = df_split(B.xi_inj[3 * (long long)id + 2]);
        } else if (drawn) {   // drawn by the pair search of this step, (hi, lo) pairs
            const float2* n2 = reinterpret_cast<const float2*>(B.noise3);
            const float2 a = n2[i], b = n2[np + i], c = n2[2 * np + i];
            g0 = dfloat{a.x, a.y};
            g1 = dfloat{b.x, b.y};
            g2 = dfloat{c.x, c.y};
        } else {
            normals3_df(B.rng_tab, P.seed, step, (unsigned long long)id, g0, g1, g2);
        }
    }
    const dfloat amp{P.amp_z_hi, P.amp_z_lo}, cev{P.cev_z_hi, P.cev_z_lo};
    dfloat b0 = df_add(df_mul(amp, g0), df_mul(cev, fx));
    const dfloat b1 = df_add(df_mul(amp, g1), df_mul(cev, fy));
    const dfloat b2 = df_add(df_mul(amp, g2), df_mul(cev, fz));
    b0 = df_add(b0, df_mul(dfloat{P.kap_hi, P.kap_lo}, df_add(yi, df_neg(dfloat{P.hly_hi, P.hly_lo}))));
    b0 = df_add(b0, df_mul(dfloat{P.akl_hi, P.akl_lo}, nw));
    B.bdf[2 * i] = make_float4(b0.hi, b1.hi, b2.hi, 0.f);
    B.bdf[2 * i + 1] = make_float4(b0.lo, b1.lo, b2.lo, 0.f);
}

// The pair weight w = exp(-|R|^2 / 2 lambda^2) of §Method for a pair within
// r_c, i.e. exp(-t) with 0 <= t < ln 20, by the table-driven method of
// P. T. P. Tang ("Table-driven implementation of the exponential function in
// IEEE floating-point arithmetic", ACM TOMS 15, 1989): 256 t = k + f with k
// the nearest integer and |f| <= 1/2, exp(-t) = E_k exp(-f / 256), E_k =
// exp(-k / 256) from a table computed on the host, and exp(-f / 256) from
// its Taylor polynomial of degree 5 (truncation below 1e-19 relative).  The
// result is within about 2 ulp of exp(-t), for 9 FP64 operations.
__device__ __forceinline__ double pair_weight(const KParams& P, const double* __restrict__ etab, double r2)
{
    constexpr double kRound = 6755399441055744.0;   // 1.5 * 2^52: adding it rounds to an integer
    constexpr double c1 = -1.0 / 256.0;
    constexpr double c2 = 1.0 / (2.0 * 65536.0);
    constexpr double c3 = -1.0 / (6.0 * 16777216.0);
    constexpr double c4 = 1.0 / (24.0 * 4294967296.0);
    constexpr double c5 = -1.0 / (120.0 * 1099511627776.0);
    const double kr = fma(r2, P.w_scale, kRound);
    const int k = __double2loint(kr);               // low word: round(256 t)
    const double kd = kr - kRound;
    if (k >= kExpTab) return exp(-r2 / P.two_lambda2);   // t >= 4: not a pair within r_c
    const double f = fma(r2, P.w_scale, -kd);       // 256 t - k, one rounding
    double q = fma(c5, f, c4);
    q = fma(q, f, c3);
    q = fma(q, f, c2);
    q = fma(q, f, c1);
    q = fma(q, f, 1.0);
    return __ldg(etab + k) * q;
}

// The double-float tables of the mixed path's normals (layout at kRngTab),
// from the host's FP64 log, cos and sin.
cudaError_t upload_rng_table(float4* rng_tab, cudaStream_t stream)
{
    static const std::array<float4, kRngTab> host = [] {
        auto df = [](double v, float& hi, float& lo) {
            hi = (float)v;
            lo = (float)(v - (double)hi);
        };
        std::array<float4, kRngTab> t{};
        for (int k = 0; k < kLnTab; ++k) {
            const double c = (double)(kLnTabBase + k) / 128.0;
            df(std::log(c), t[k].x, t[k].y);
            df(1.0 / c, t[k].z, t[k].w);
        }
        df(std::log(2.0), t[kRngConstLn].x, t[kRngConstLn].y);
        df(1.0 / 3.0, t[kRngConstLn].z, t[kRngConstLn].w);
        const double two_pi = 6.283185307179586476925286766559;
        for (int j = 0; j < kTrigTab; ++j) {
            const double a = two_pi * (double)j / (double)kTrigTab;
            df(std::cos(a), t[kRngTrig + j].x, t[kRngTrig + j].y);
            df(std::sin(a), t[kRngTrig + j].z, t[kRngTrig + j].w);
        }
        df(two_pi, t[kRngConstTrig].x, t[kRngConstTrig].y);
        df(-1.0 / 6.0, t[kRngConstTrig].z, t[kRngConstTrig].w);
        return t;
    }();
    cudaError_t e = cudaMemcpyAsync(rng_tab, host.data(), sizeof(float4) * kRngTab, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    return e;
}

cudaError_t upload_exp_table(double* exp_tab, float2* exp_tab_df, cudaStream_t stream)
{
    static const std::array<double, kExpTab> host = [] {
        std::array<double, kExpTab> t{};
        for (int k = 0; k < kExpTab; ++k) t[k] = std::exp(-(double)k / 256.0);
        return t;
    }();
    static const std::array<float2, kExpTab> host_df = [] {
        std::array<float2, kExpTab> t{};
        for (int k = 0; k < kExpTab; ++k) {
            const float hi = (float)host[k];
            t[k] = make_float2(hi, (float)(host[k] - (double)hi));
        }
        return t;
    }();
    cudaError_t e = cudaMemcpyAsync(exp_tab, host.data(), sizeof(double) * kExpTab, cudaMemcpyHostToDevice,
                                    stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(exp_tab_df, host_df.data(), sizeof(float2) * kExpTab, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    return e;
}

// The partners of row i written straight into its slots (rows with more than
// kCandCap partners), in the order of the counting search.
__device__ __noinline__ void search_row_into_slots(const KParams& P, const DevBuffers& B, int i, double delta,
                                                   int base, int cnt)
{
    const int np = P.npad;
    int k = 0;
    for_each_neighbor(P, delta, B.pos_w, B.pos32, B.cell_start, B.cell_of, i, B.pos_w[i], B.pos_w[np + i],
                      B.pos_w[2 * np + i],
                      [&](int j, unsigned char code) {
                          if (k < cnt) {
                              B.col[base + 32 * k] = j;
                              B.img[base + 32 * k] = code;
                          }
                          ++k;
                      });
    if (k != cnt) atomicCAS(&B.st->error, 0, (int)SP_ERR_INVALID_ARG);
}

// The pair weight of pair_weight() for the mixed-precision path, in
// double-float arithmetic (FP32 pipes): the same table-driven method, with
// 256 t = k + f split exactly, exp(-f/256) = 1 + g + g^2/2 + ... for
// g = -f/256 (1 + g exact as a double-float, the remaining terms, below
// 2^-19, in FP32) and E_k from the double-float table.  r2 is the squared
// separation as a double-float; the result carries about 2^-44 relative error.
__device__ __forceinline__ dfloat pair_weight_df(const KParams& P, const float2* __restrict__ etab, dfloat r2)
{
    constexpr float kRound = 12582912.f;   // 1.5 * 2^23: adding it rounds to an integer
    const dfloat t = df_mul(r2, dfloat{P.wsc_hi, P.wsc_lo});
    const float kr = __fadd_rn(t.hi, kRound);
    const int k = __float_as_int(kr) - __float_as_int(kRound);
    if (k < 0 || k >= kExpTab) {   // t >= 4: not a pair within r_c
        const double w = exp(-df_to_double(r2) / P.two_lambda2);
        const float wh = (float)w;
        return dfloat{wh, (float)(w - (double)wh)};
    }
    const dfloat f = fast_two_sum(__fsub_rn(t.hi, __fsub_rn(kr, kRound)), t.lo);   // 256 t - k
    const float gh = __fmul_rn(f.hi, -0.00390625f), gl = __fmul_rn(f.lo, -0.00390625f);   // exact
    const float tail = __fmul_rn(__fmul_rn(gh, gh),
                                 fmaf(gh, fmaf(gh, fmaf(gh, 1.f / 120.f, 1.f / 24.f), 1.f / 6.f), 0.5f));
    const dfloat one_g = two_sum(1.f, gh);
    const dfloat q = fast_two_sum(one_g.hi, __fadd_rn(one_g.lo, __fadd_rn(gl, tail)));
    const float2 e = __ldg(etab + k);
    return df_mul(dfloat{e.x, e.y}, q);
}

// Separation component R_i - R_j - shift of the minimum image, from
// double-float positions and a double-float shift.
__device__ __forceinline__ dfloat sep_df(float ih, float il, float jh, float jl, dfloat shift)
{
    const dfloat d = two_sum(ih, -jh);
    dfloat r = fast_two_sum(d.hi, __fadd_rn(d.lo, __fsub_rn(il, jl)));
    if (shift.hi != 0.f) r = df_add(r, df_neg(shift));
    return r;
}

// Assembly of Eq. algebra from the stored pairs: one thread per slot of the
// sliced layout, so the 32 rows of a warp have nearly equal lengths and read
// their entries with coalesced loads; the FP64 work runs once per entry in
// converged warps.  Separations use the entries' image codes (exact, no
// divisions): the shifts n delta and a L_x of the canonical minimum image are
// exact for |n| <= 1 and |a| <= 2 and taken by selection, and a warp whose
// current entries all pair with the central image (most warps: the rows of
// a warp are neighbours in space) skips them.  Padding entries get weight 0.
//
// DF (the mixed-precision path): the per-entry arithmetic — separations,
// |R|^2, weight, pair sums — and the row finish run in double-float on the
// FP32 pipes from the double-float positions, and the system is stored as
// double-floats only (weights val32 + val32lo, A_ii, b); it agrees with the
// FP64 assembly to ~1e-12 relative (the 2^-48 representation of the
// positions), far inside the mixed solver's tolerance.
constexpr int kAsmBatch = 4;   // partners requested at a time by the double-float assembly

template <bool DF>
__global__ void __launch_bounds__(256, 3) k_assemble_slots(KParams P, DevBuffers B, int use_inj)
{
    const DevState* st = B.st;
    if (st->error | st->overflow) return;
    const int slot = blockIdx.x * 256 + threadIdx.x;
    const int i = B.slot_row[slot];
    if (i < 0) return;
    const double delta = st->delta;
    const int np = P.npad;
    const double xi = B.pos_w[i], yi = B.pos_w[np + i], zi = B.pos_w[2 * np + i];
    const int base = B.chunk_off[slot >> 5] + (slot & 31);
    const int clen = (B.chunk_off[(slot >> 5) + 1] - B.chunk_off[slot >> 5]) >> 5;
    const int cnt = B.row_cnt[i];
    const int center = image_code(0, 0, 0);
    // partners of the row: from the search's candidates, placed into the sliced
    // layout here; a row with more than kCandCap partners is searched again
    const int* __restrict__ pj = B.cand_j + i;
    const unsigned char* __restrict__ pimg = B.cand_img + i;
    size_t pstride = (size_t)np;
    if (cnt > kCandCap) {
        search_row_into_slots(P, B, i, delta, base, cnt);
        pj = B.col + base;
        pimg = B.img + base;
        pstride = 32;
    }
    double sw = 0.0, fx = 0.0, fy = 0.0, fz = 0.0, nw = 0.0;
    dfloat dsw{0.f, 0.f}, dsx{0.f, 0.f}, dsy{0.f, 0.f}, dsz{0.f, 0.f}, dsn{0.f, 0.f};
    if (DF) {
        const float* __restrict__ ph = B.pos32;
        const float* __restrict__ pl = B.pos32lo;
        const float xih = ph[i], yih = ph[np + i], zih = ph[2 * np + i];
        const float xil = pl[i], yil = pl[np + i], zil = pl[2 * np + i];
        const float dh = (float)delta;
        const dfloat dd{dh, (float)(delta - (double)dh)};
        const dfloat Lx{P.Lf[0], P.Llo[0]}, Ly{P.Lf[1], P.Llo[1]}, Lz{P.Lf[2], P.Llo[2]};
        const dfloat zero{0.f, 0.f};
        dfloat s_w = zero, s_x = zero, s_y = zero, s_z = zero, s_n = zero;
        // partners in batches of kAsmBatch: their indices, then their positions,
        // are requested together (one latency per batch, not per partner)
        for (int k0 = 0; k0 < cnt; k0 += kAsmBatch) {
        int jb[kAsmBatch], cb[kAsmBatch];
#pragma unroll
        for (int u = 0; u < kAsmBatch; ++u) {
            const bool in = k0 + u < cnt;
            jb[u] = in ? pj[(k0 + u) * pstride] : i;
            cb[u] = in ? pimg[(k0 + u) * pstride] : center;
        }
        float pxh[kAsmBatch], pxl[kAsmBatch], pyh[kAsmBatch], pyl[kAsmBatch], pzh[kAsmBatch], pzl[kAsmBatch];
#pragma unroll
        for (int u = 0; u < kAsmBatch; ++u) {
            const int j = jb[u];
            pxh[u] = ph[j];
            pxl[u] = pl[j];
            pyh[u] = ph[np + j];
            pyl[u] = pl[np + j];
            pzh[u] = ph[2 * np + j];
            pzl[u] = pl[2 * np + j];
        }
#pragma unroll
        for (int u = 0; u < kAsmBatch; ++u) {
            const int k = k0 + u;
            if (k >= cnt) break;
            const int e = base + 32 * k;
            const int j = jb[u];
            const int code = cb[u];
            B.col[e] = j;
            B.img[e] = (unsigned char)code;
            const bool shifted = !__all_sync(__activemask(), code == center);   // warp-uniform
            dfloat shx = zero, shy = zero, shz = zero;
            int m = 0;
            if (shifted) {
                const int a = (code & 7) - 2, c = ((code >> 5) & 3) - 1;
                m = ((code >> 3) & 3) - 1;
                // a L_x + m delta as one double-float (the exact FP64 order does not matter here)
                dfloat sa = zero;
                if (a == 1 || a == -1)
                    sa = a > 0 ? Lx : df_neg(Lx);
                else if (a == 2 || a == -2)
                    sa = a > 0 ? dfloat{2.f * Lx.hi, 2.f * Lx.lo} : dfloat{-2.f * Lx.hi, -2.f * Lx.lo};
                else if (a != 0)
                    sa = df_mul(dfloat{(float)a, 0.f}, Lx);
                shx = m == 0 ? sa : df_add(sa, m > 0 ? dd : df_neg(dd));
                shy = m == 0 ? zero : (m > 0 ? Ly : df_neg(Ly));
                shz = c == 0 ? zero : (c > 0 ? Lz : df_neg(Lz));
            }
            const dfloat dx = sep_df(xih, xil, pxh[u], pxl[u], shx);
            const dfloat dy = sep_df(yih, yil, pyh[u], pyl[u], shy);
            const dfloat dz = sep_df(zih, zil, pzh[u], pzl[u], shz);
            const dfloat r2 = df_add(df_add(df_sqr(dx), df_sqr(dy)), df_sqr(dz));
            const dfloat w = pair_weight_df(P, B.exp_tab_df, r2);
            B.val32[e] = w.hi;
            B.val32lo[e] = w.lo;
            s_w = df_add(s_w, w);
            s_x = df_add(s_x, df_mul(dx, w));
            s_y = df_add(s_y, df_mul(dy, w));
            s_z = df_add(s_z, df_mul(dz, w));
            if (shifted && m != 0) s_n = df_add(s_n, m > 0 ? w : df_neg(w));
        }
        }
        dsw = s_w;
        dsx = s_x;
        dsy = s_y;
        dsz = s_z;
        dsn = s_n;
    } else {
        const double Lx = P.L[0], Ly = P.L[1], Lz = P.L[2];
        const double* __restrict__ pos = B.pos_w;
        for (int k = 0; k < cnt; ++k) {
            const int e = base + 32 * k;
            const int j = pj[k * pstride];
            const int code = pimg[k * pstride];
            B.col[e] = j;
            B.img[e] = (unsigned char)code;
            double dx = __dsub_rn(xi, pos[j]);
            double dy = __dsub_rn(yi, pos[np + j]);
            double dz = __dsub_rn(zi, pos[2 * np + j]);
            const bool shifted = !__all_sync(__activemask(), code == center);   // warp-uniform
            int m = 0;
            if (shifted) {
                const int a = (code & 7) - 2, c = ((code >> 5) & 3) - 1;
                m = ((code >> 3) & 3) - 1;
                const double sn = m == 0 ? 0.0 : (m > 0 ? delta : -delta);
                const double sa = a == 0 ? 0.0 : (a == 1 ? Lx : (a == -1 ? -Lx : __dmul_rn(Lx, (double)a)));
                const double sy = m == 0 ? 0.0 : (m > 0 ? Ly : -Ly);
                const double sz = c == 0 ? 0.0 : (c > 0 ? Lz : -Lz);
                dx = __dsub_rn(__dsub_rn(dx, sn), sa);
                dy = __dsub_rn(dy, sy);
                dz = __dsub_rn(dz, sz);
            }
            const double w = pair_weight(P, B.exp_tab, fma(dx, dx, fma(dy, dy, dz * dz)));
            B.val[e] = w;
            B.val32[e] = (float)w;
            if (B.val32lo) B.val32lo[e] = df_split(w).lo;
            sw += w;
            fx = fma(dx, w, fx);
            fy = fma(dy, w, fy);
            fz = fma(dz, w, fz);
            if (shifted) nw += m == 0 ? 0.0 : (m > 0 ? w : -w);
        }
    }
    for (int k = cnt; k < clen; ++k) {
        B.col[base + 32 * k] = i;
        B.img[base + 32 * k] = (unsigned char)center;
        B.val32[base + 32 * k] = 0.f;
        if (DF)
            B.val32lo[base + 32 * k] = 0.f;
        else
            B.val[base + 32 * k] = 0.0;
    }
    if (DF)
        finish_row_df(P, B, i, dfloat{B.pos32[np + i], B.pos32lo[np + i]}, (unsigned long long)st->step, use_inj,
                      st->noise_step == st->step, dsw, dsx, dsy, dsz, dsn);
    else
        finish_row(P, B, i, yi, (unsigned long long)st->step, use_inj, st->noise_step == st->step, sw, fx, fy, fz,
                   nw);
}

// Pair search writing the sliced columns and image codes (FP32 decisions).
__global__ void k_nbr_fill(KParams P, DevBuffers B)
{
    DevState* st = B.st;
    if (st->error | st->overflow) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const double delta = st->delta;
    const int np = P.npad;
    const double xi = B.pos_w[i], yi = B.pos_w[np + i], zi = B.pos_w[2 * np + i];
    const int slot = B.row_slot[i];
    const int base = B.chunk_off[slot >> 5] + (slot & 31);
    const int clen = (B.chunk_off[(slot >> 5) + 1] - B.chunk_off[slot >> 5]) >> 5;
    const int cnt = B.row_cnt[i];
    int k = 0;
    int* __restrict__ col = B.col;
    unsigned char* __restrict__ img = B.img;
    for_each_neighbor(P, delta, B.pos_w, B.pos32, B.cell_start, B.cell_of, i, xi, yi, zi, [&](int j, unsigned char code) {
        if (k < cnt) {
            col[base + 32 * k] = j;
            img[base + 32 * k] = code;
        }
        ++k;
    });
    // the counting pass and this one must agree; a mismatch is reported, never written past
    if (k != cnt) atomicCAS(&st->error, 0, (int)SP_ERR_INVALID_ARG);
    for (int kk = cnt; kk < clen; ++kk) {
        col[base + 32 * kk] = i;
        img[base + 32 * kk] = image_code(0, 0, 0);
    }
}

int launch_nbr_fill(const KParams& P, DevBuffers& B, bool assemble, bool use_inj, bool df, Launch L)
{
    if (assemble) {   // places the collected partners and assembles
        launch_assemble_only(P, B, use_inj, df, L);
        return 1;
    }
    k_nbr_fill<<<grid_for(P.n, 128, 1 << 30), 128, 0, L.stream>>>(P, B);
    return 1;
}

// Assembly from existing pairs (df: double-float entries, the mixed-precision path).
void launch_assemble_only(const KParams& P, DevBuffers& B, bool use_inj, bool df, Launch L)
{
    if (df)
        k_assemble_slots<true><<<P.nslots / 256, 256, 0, L.stream>>>(P, B, use_inj ? 1 : 0);
    else
        k_assemble_slots<false><<<P.nslots / 256, 256, 0, L.stream>>>(P, B, use_inj ? 1 : 0);
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

// Test hook: the normals of ids[k] at `step` as the FP64 path (df = 0) or the
// mixed path (df = 1) draws them, out[3 k + c].
__global__ void k_normals(const float4* __restrict__ tab, unsigned long long seed, unsigned long long step,
                          long long count, const long long* __restrict__ ids, double* __restrict__ out, int df)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
         k += (long long)gridDim.x * blockDim.x) {
        if (df) {
            dfloat g0, g1, g2;
            normals3_df(tab, seed, step, (unsigned long long)ids[k], g0, g1, g2);
            out[3 * k] = df_to_double(g0);
            out[3 * k + 1] = df_to_double(g1);
            out[3 * k + 2] = df_to_double(g2);
        } else {
            normals3(seed, step, (unsigned long long)ids[k], out[3 * k], out[3 * k + 1], out[3 * k + 2]);
        }
    }
}

void launch_normals(const float4* tab, unsigned long long seed, unsigned long long step, long long count,
                    const long long* ids, double* out, int df, cudaStream_t s)
{
    k_normals<<<grid_for(count, kVecBlock, 1 << 30), kVecBlock, 0, s>>>(tab, seed, step, count, ids, out, df);
}

void launch_philox_blocks(unsigned long long seed, unsigned long long step, long long count,
                          const long long* ids, unsigned long long* out, cudaStream_t s)
{
    k_philox_blocks<<<grid_for(count, kVecBlock, 1 << 30), kVecBlock, 0, s>>>(seed, step, count, ids, out);
}

}  // namespace ss
