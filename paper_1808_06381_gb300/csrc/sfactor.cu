// Inter-chain structure factor S(q) = (1/n) |sum_c exp(-i q . R_c)|^2 at q_z = 0
// (arXiv 1808.06381, Eq. Sfactor; the paper shows it in the flow-gradient
// plane as S(q_x, q_y)).
//
// Under Lees-Edwards shear the allowed wave vectors form the sheared reciprocal
// lattice q_x = 2 pi kx / L_x, q_y = 2 pi ky / L_y - gamma q_x with gamma =
// delta / L_y: in the sheared frame x' = x - gamma y (mod L_x) the density is
// periodic in (x', y) and q . R = 2 pi (kx x' / L_x + ky y / L_y).
//
// Grid mode: cloud-in-cell deposit of the particles on a G x G grid of the
// sheared frame (z summed, since q_z = 0), in 2^-32 fixed point with integer
// atomics so that the grid does not depend on the order of the deposits; a
// separable DFT of the grid for the requested modes with a precomputed twiddle
// table; division by the CIC window sinc^2(pi kx / G) sinc^2(pi ky / G).
// Direct mode: the sum over particles for every requested mode, in FP64.
#include <math.h>

#include "internal.cuh"

namespace ss {

namespace {

constexpr double kFix = 4294967296.0;   // 2^32

__global__ void k_sq_deposit(KParams P, const double* __restrict__ pos, double delta, int G,
                             unsigned long long* __restrict__ grid)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const int np = P.npad;
    const double gamma = delta / P.L[1];
    const double x = pos[i], y = pos[np + i];
    double xs = x - gamma * y;
    xs = xs - P.L[0] * floor(xs / P.L[0]);
    const double u = xs / P.L[0] * G, v = y / P.L[1] * G;
    int i0 = (int)floor(u), j0 = (int)floor(v);
    const double fu = u - i0, fv = v - j0;
    i0 = ((i0 % G) + G) % G;
    j0 = ((j0 % G) + G) % G;
    const int i1 = (i0 + 1) % G, j1 = (j0 + 1) % G;
    const unsigned long long w00 = (unsigned long long)llround((1.0 - fu) * (1.0 - fv) * kFix);
    const unsigned long long w10 = (unsigned long long)llround(fu * (1.0 - fv) * kFix);
    const unsigned long long w01 = (unsigned long long)llround((1.0 - fu) * fv * kFix);
    const unsigned long long w11 = (unsigned long long)llround(fu * fv * kFix);
    atomicAdd(grid + (size_t)j0 * G + i0, w00);
    atomicAdd(grid + (size_t)j0 * G + i1, w10);
    atomicAdd(grid + (size_t)j1 * G + i0, w01);
    atomicAdd(grid + (size_t)j1 * G + i1, w11);
}

// A[kx][gy] = sum_gx rho[gy][gx] exp(-2 pi i kx gx / G), kx = -nkx..nkx.
__global__ void k_sq_dft_x(const unsigned long long* __restrict__ grid, int G, int nkx,
                           const double2* __restrict__ tw, double2* __restrict__ A)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int nk = 2 * nkx + 1;
    if (t >= nk * G) return;
    const int kx = t / G - nkx, gy = t % G;
    double re = 0.0, im = 0.0;
    const int kk = ((kx % G) + G) % G;
    for (int gx = 0; gx < G; ++gx) {
        const double r = (double)grid[(size_t)gy * G + gx] / kFix;
        const double2 w = tw[(kk * gx) % G];   // (cos, sin) of 2 pi m / G
        re += r * w.x;
        im -= r * w.y;
    }
    A[(size_t)(kx + nkx) * G + gy] = make_double2(re, im);
}

// F[kx][ky] = sum_gy A[kx][gy] exp(-2 pi i ky gy / G), then the CIC window is
// divided out and S = |F|^2 / n, with the sheared-lattice wave vector.
__global__ void k_sq_dft_y(const double2* __restrict__ A, int G, int nkx, int nky,
                           const double2* __restrict__ tw, KParams P, double delta, double* __restrict__ S,
                           double* __restrict__ qx, double* __restrict__ qy)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int mx = 2 * nkx + 1, my = 2 * nky + 1;
    if (t >= mx * my) return;
    const int kx = t / my - nkx, ky = t % my - nky;
    const int kk = ((ky % G) + G) % G;
    double re = 0.0, im = 0.0;
    for (int gy = 0; gy < G; ++gy) {
        const double2 a = A[(size_t)(kx + nkx) * G + gy];
        const double2 w = tw[(kk * gy) % G];
        // (a.x + i a.y)(w.x - i w.y)
        re += a.x * w.x + a.y * w.y;
        im += a.y * w.x - a.x * w.y;
    }
    const double pi = 3.14159265358979323846;
    double wx = 1.0, wy = 1.0;
    if (kx != 0) {
        const double s = sin(pi * kx / G) / (pi * kx / G);
        wx = s * s;
    }
    if (ky != 0) {
        const double s = sin(pi * ky / G) / (pi * ky / G);
        wy = s * s;
    }
    const double w = wx * wy;
    S[t] = (re * re + im * im) / (w * w) / P.n;
    const double q_x = 2.0 * pi * kx / P.L[0];
    qx[t] = q_x;
    qy[t] = 2.0 * pi * ky / P.L[1] - delta / P.L[1] * q_x;
}

// Direct sum over particles for each mode (one block per mode).
__global__ void k_sq_direct(KParams P, const double* __restrict__ pos, double delta, int nkx, int nky,
                            double* __restrict__ S, double* __restrict__ qx, double* __restrict__ qy)
{
    __shared__ double sh[32];
    const int t = blockIdx.x;
    const int my = 2 * nky + 1;
    const int kx = t / my - nkx, ky = t % my - nky;
    const double pi = 3.14159265358979323846;
    const double q_x = 2.0 * pi * kx / P.L[0];
    const double q_y = 2.0 * pi * ky / P.L[1] - delta / P.L[1] * q_x;
    const int np = P.npad;
    double re = 0.0, im = 0.0;
    for (int i = threadIdx.x; i < P.n; i += blockDim.x) {
        double s, c;
        sincos(q_x * pos[i] + q_y * pos[np + i], &s, &c);
        re += c;
        im -= s;
    }
    re = block_sum(re, sh);
    __syncthreads();
    im = block_sum(im, sh);
    if (threadIdx.x == 0) {
        S[t] = (re * re + im * im) / P.n;
        qx[t] = q_x;
        qy[t] = q_y;
    }
}

}  // namespace

cudaError_t run_structure_factor(const KParams& P, const DevBuffers& B, double delta, int G, int nkx, int nky,
                                 const double* twiddle_dev, unsigned long long* grid_dev, double2* A_dev,
                                 double* S_dev, double* qx_dev, double* qy_dev, cudaStream_t s)
{
    const int m = (2 * nkx + 1) * (2 * nky + 1);
    if (G == 0) {
        k_sq_direct<<<m, 256, 0, s>>>(P, B.pos_s, delta, nkx, nky, S_dev, qx_dev, qy_dev);
        return cudaGetLastError();
    }
    cudaMemsetAsync(grid_dev, 0, sizeof(unsigned long long) * (size_t)G * G, s);
    k_sq_deposit<<<grid_for(P.n, kVecBlock, 1 << 30), kVecBlock, 0, s>>>(P, B.pos_s, delta, G, grid_dev);
    const double2* tw = reinterpret_cast<const double2*>(twiddle_dev);
    k_sq_dft_x<<<grid_for((long long)(2 * nkx + 1) * G, kVecBlock, 1 << 30), kVecBlock, 0, s>>>(grid_dev, G, nkx, tw,
                                                                                                A_dev);
    k_sq_dft_y<<<grid_for(m, kVecBlock, 1 << 30), kVecBlock, 0, s>>>(A_dev, G, nkx, nky, tw, P, delta, S_dev,
                                                                      qx_dev, qy_dev);
    return cudaGetLastError();
}

}  // namespace ss
