/*
 * CPU FP64 oracle for the coupled velocity solve of Korolkovas,
 * "Giant fluctuations in sheared viscoelastic fluids emerging in a
 * mesoscale simulation" (arXiv 1808.06381).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously correct; shares no code
 * with the CUDA library.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.
 *
 * Build: gcc -O2 -ffp-contract=off -std=c11 -fPIC -shared (no FMA contraction,
 * so every product and sum is rounded exactly as written, left to right).
 *
 * Units: the truncation radius r_c is the length unit of the inputs.  The
 * paper's unit lambda (radius of gyration) follows from the truncation rule
 * of §Method ("truncate the weights below 5 %"): exp(-r_c^2 / 2 lambda^2) =
 * 0.05, i.e. lambda^2 = r_c^2 / (2 ln 20).
 *
 * Functions and the passage each follows:
 *   or_derive            §Method: tau = lambda^2 zeta / kT; v/lambda^3 = 0.1
 *   or_min_image         §Method, "standard Lees-Edwards boundary conditions"
 *                        and the boundary correction V = kappa L_y round(y/L_y)
 *   or_neighbors_brute   §Method: weights w = exp(-R^2/2 lambda^2) truncated below 5 %
 *   or_neighbors_cells   same set as or_neighbors_brute, found with a cell list
 *                        (timing only; cross-checked against brute force)
 *   or_philox4x64_10     counter-based generator, Salmon et al., SC'11
 *   or_noise             §Method Eq. F first term: sqrt(6 zeta kT) W_c(t)
 *   or_assemble          §Method Eq. F (exvol, shear) and Eq. vc rewritten as Eq. algebra
 *   or_matvec            Eq. algebra, left-hand side
 *   or_pcg               Jacobi-preconditioned conjugate gradients on Eq. algebra
 *   or_dense_solve       Eq. algebra solved by dense Cholesky (tiny N)
 *   or_integrate         §Method: first order in time, v = dR/dt, Lees-Edwards wrap
 *   or_structure_factor  Eq. Sfactor at q_z = 0 on the sheared reciprocal lattice
 *   or_stress_xy         pair virial of the ev and friction forces (the paper defines no stress)
 *   or_velocity_correlation  §Results, Fig. vv: <v_c . v_c'> / <v_c^2> binned by |R_cc'|
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG -1
#define OR_ERR_CAPACITY -2
#define OR_ERR_NOT_CONVERGED -3
#define OR_ERR_NOT_SPD -4

typedef struct {
    int64_t n;
    double L[3];
    double rc;
    double alpha;
    double eps;
    double zeta;
    double kT;
    double kappa;   /* shear rate, in units of kT / (zeta r_c^2) */
    double dt;
    uint64_t seed;
} or_params;

typedef struct {
    double lambda2;   /* lambda^2 = r_c^2 / (2 ln 20) */
    double c_ev;      /* excluded-volume prefactor eps * (v/lambda^3) * kT / lambda^2 */
    double noise_amp; /* sqrt(2 zeta kT / dt): per Cartesian component */
    double rc2;
} or_derived;

/* §Method: lambda from the 5 % truncation; v/lambda^3 = 0.1; noise per
 * component from <W.W> = delta(t - t'), i.e. 1/3 of sqrt(6 zeta kT)^2 per axis. */
void or_derive(const or_params* p, or_derived* d)
{
    d->lambda2 = p->rc * p->rc / (2.0 * log(20.0));
    d->c_ev = p->eps * 0.1 * p->kT / d->lambda2;
    d->noise_amp = sqrt(2.0 * p->zeta * p->kT / p->dt);
    d->rc2 = p->rc * p->rc;
}

/* kappa from the paper's dimensionless kappa*tau with tau = lambda^2 zeta / kT (§Method). */
double or_kappa_from_kappa_tau(double kappa_tau, double rc, double zeta, double kT)
{
    double lambda2 = rc * rc / (2.0 * log(20.0));
    double tau = lambda2 * zeta / kT;
    return kappa_tau / tau;
}

/* Separation R_ij = R_i - R_j under the Lees-Edwards minimum image.
 * The image of j that sits n boxes up (y + n L_y) is displaced in x by n*delta;
 * n = round(y_ij / L_y) is exactly the integer of the boundary correction
 * V_ij = kappa L_y round(y_ij / L_y) x (§Method).  round() is half away from zero. */
void or_min_image(const or_params* p, double delta, const double* ri, const double* rj,
                  double* d, double* nimg)
{
    double dx = ri[0] - rj[0];
    double dy = ri[1] - rj[1];
    double dz = ri[2] - rj[2];
    double n = round(dy / p->L[1]);
    dy = dy - n * p->L[1];
    dx = dx - n * delta;
    dx = dx - p->L[0] * round(dx / p->L[0]);
    dz = dz - p->L[2] * round(dz / p->L[2]);
    d[0] = dx;
    d[1] = dy;
    d[2] = dz;
    *nimg = n;
}

static double sq_dist(const double* d)
{
    double r2 = d[0] * d[0];
    r2 = r2 + d[1] * d[1];
    r2 = r2 + d[2] * d[2];
    return r2;
}

/* All pairs i < j with |R_ij|^2 < r_c^2, i.e. w_ij > 5 % (§Method), by checking
 * every pair.  Pairs come out sorted by (i, j).  Returns OR_ERR_CAPACITY (and
 * the true count in *npairs) if cap is too small. */
int or_neighbors_brute(const or_params* p, const double* pos, double delta, int64_t cap,
                       int64_t* pairs, int64_t* npairs)
{
    or_derived dv;
    or_derive(p, &dv);
    int64_t m = 0;
    for (int64_t i = 0; i < p->n; ++i) {
        for (int64_t j = i + 1; j < p->n; ++j) {
            double d[3], nimg;
            or_min_image(p, delta, pos + 3 * i, pos + 3 * j, d, &nimg);
            if (sq_dist(d) < dv.rc2) {
                if (m < cap) {
                    pairs[2 * m] = i;
                    pairs[2 * m + 1] = j;
                }
                ++m;
            }
        }
    }
    *npairs = m;
    return m <= cap ? OR_OK : OR_ERR_CAPACITY;
}

static int cmp_pair(const void* a, const void* b)
{
    const int64_t* x = (const int64_t*)a;
    const int64_t* y = (const int64_t*)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    if (x[1] != y[1]) return x[1] < y[1] ? -1 : 1;
    return 0;
}

static int64_t wrap_cell(int64_t c, int64_t nc)
{
    c %= nc;
    return c < 0 ? c + nc : c;
}

/* The same pair set as or_neighbors_brute, found with a cell list so that
 * large systems finish in seconds.  For each particle i and each vertical
 * image m in {-1, 0, 1} of a partner j (partner image at y_j + m L_y, shifted
 * by m*delta in x), the cells that can hold such a partner are scanned with a
 * one-cell safety margin; every candidate then goes through the exact
 * predicate of or_neighbors_brute, and duplicates are dropped with a stamp.
 * Boxes with fewer than 3 cells along some axis fall back to brute force. */
int or_neighbors_cells(const or_params* p, const double* pos, double delta, int64_t cap,
                       int64_t* pairs, int64_t* npairs)
{
    or_derived dv;
    or_derive(p, &dv);
    int64_t nc[3];
    double cw[3];
    for (int k = 0; k < 3; ++k) {
        nc[k] = (int64_t)floor(p->L[k] / p->rc);
        if (nc[k] < 3) return or_neighbors_brute(p, pos, delta, cap, pairs, npairs);
        cw[k] = p->L[k] / (double)nc[k];
    }
    int64_t ncell = nc[0] * nc[1] * nc[2];
    int64_t* head = (int64_t*)malloc(sizeof(int64_t) * ncell);
    int64_t* next = (int64_t*)malloc(sizeof(int64_t) * p->n);
    int64_t* stamp = (int64_t*)malloc(sizeof(int64_t) * p->n);
    if (!head || !next || !stamp) {
        free(head); free(next); free(stamp);
        return OR_ERR_ARG;
    }
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    for (int64_t i = 0; i < p->n; ++i) stamp[i] = -1;
    for (int64_t i = p->n - 1; i >= 0; --i) {
        int64_t c3[3];
        for (int k = 0; k < 3; ++k) {
            int64_t c = (int64_t)floor(pos[3 * i + k] / cw[k]);
            if (c < 0) c = 0;
            if (c >= nc[k]) c = nc[k] - 1;
            c3[k] = c;
        }
        int64_t c = (c3[2] * nc[1] + c3[1]) * nc[0] + c3[0];
        next[i] = head[c];
        head[c] = i;
    }
    int64_t m = 0;
    for (int64_t i = 0; i < p->n; ++i) {
        const double* ri = pos + 3 * i;
        for (int img = -1; img <= 1; ++img) {
            /* partner primary position range for this vertical image */
            double yc = ri[1] - img * p->L[1];
            double xc = ri[0] - img * delta;
            int64_t ylo = (int64_t)floor((yc - p->rc) / cw[1]) - 1;
            int64_t yhi = (int64_t)floor((yc + p->rc) / cw[1]) + 1;
            if (ylo < 0) ylo = 0;
            if (yhi > nc[1] - 1) yhi = nc[1] - 1;
            if (ylo > yhi) continue;
            int64_t xlo = (int64_t)floor((xc - p->rc) / cw[0]) - 1;
            int64_t xhi = (int64_t)floor((xc + p->rc) / cw[0]) + 1;
            if (xhi - xlo + 1 > nc[0]) { xlo = 0; xhi = nc[0] - 1; }
            int64_t zlo = (int64_t)floor((ri[2] - p->rc) / cw[2]) - 1;
            int64_t zhi = (int64_t)floor((ri[2] + p->rc) / cw[2]) + 1;
            if (zhi - zlo + 1 > nc[2]) { zlo = 0; zhi = nc[2] - 1; }
            for (int64_t cz = zlo; cz <= zhi; ++cz) {
                for (int64_t cy = ylo; cy <= yhi; ++cy) {
                    for (int64_t cx = xlo; cx <= xhi; ++cx) {
                        int64_t c = (wrap_cell(cz, nc[2]) * nc[1] + cy) * nc[0] + wrap_cell(cx, nc[0]);
                        for (int64_t j = head[c]; j >= 0; j = next[j]) {
                            if (j <= i || stamp[j] == i) continue;
                            stamp[j] = i;
                            double d[3], nimg;
                            or_min_image(p, delta, ri, pos + 3 * j, d, &nimg);
                            if (sq_dist(d) < dv.rc2) {
                                if (m < cap) {
                                    pairs[2 * m] = i;
                                    pairs[2 * m + 1] = j;
                                }
                                ++m;
                            }
                        }
                    }
                }
            }
        }
    }
    free(head);
    free(next);
    free(stamp);
    *npairs = m;
    if (m > cap) return OR_ERR_CAPACITY;
    qsort(pairs, (size_t)m, 2 * sizeof(int64_t), cmp_pair);
    return OR_OK;
}

/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): ten rounds of two 64x64->128 multiplies with the
 * published multipliers and Weyl key increments. */
static void mul128(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo)
{
    unsigned __int128 r = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(r >> 64);
    *lo = (uint64_t)r;
}

void or_philox4x64_10(const uint64_t* ctr_in, const uint64_t* key_in, uint64_t* out)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint64_t k[2] = {key_in[0], key_in[1]};
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k[0] += W0;
            k[1] += W1;
        }
        uint64_t hi0, lo0, hi1, lo1;
        mul128(M0, c[0], &hi0, &lo0);
        mul128(M1, c[2], &hi1, &lo1);
        uint64_t n0 = hi1 ^ c[1] ^ k[0];
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c[3] ^ k[1];
        uint64_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Three standard normals for particle `id` at time step `step`: one Philox
 * block with key (seed, 0) and counter (id, step, 0, 0), turned into normals
 * by the Box-Muller transform (Box & Muller 1958) on 53-bit uniforms:
 * u1 in (0, 1] from words 0 and 2, u2 in [0, 1) from words 1 and 3. */
void or_normals3(uint64_t seed, uint64_t step, uint64_t id, double* xi)
{
    uint64_t ctr[4] = {id, step, 0, 0};
    uint64_t key[2] = {seed, 0};
    uint64_t o[4];
    or_philox4x64_10(ctr, key, o);
    const double two53inv = 1.0 / 9007199254740992.0;
    double u1 = (double)((o[0] >> 11) + 1) * two53inv;
    double u2 = (double)(o[1] >> 11) * two53inv;
    double u3 = (double)((o[2] >> 11) + 1) * two53inv;
    double u4 = (double)(o[3] >> 11) * two53inv;
    const double two_pi = 6.283185307179586476925286766559;
    double r1 = sqrt(-2.0 * log(u1));
    double r2 = sqrt(-2.0 * log(u3));
    xi[0] = r1 * cos(two_pi * u2);
    xi[1] = r1 * sin(two_pi * u2);
    xi[2] = r2 * cos(two_pi * u4);
}

/* Normals for particles with the given ids (xi is [n][3]). */
void or_noise(uint64_t seed, uint64_t step, int64_t n, const int64_t* ids, double* xi)
{
    for (int64_t i = 0; i < n; ++i) or_normals3(seed, step, (uint64_t)ids[i], xi + 3 * i);
}

/*
 * Assemble Eq. algebra from a pair list (§Method, Eq. F and Eq. vc):
 *
 *   F_i = noise_amp * xi_i                               (thermal noise)
 *       + c_ev * sum_j R_ij w_ij                          (Eq. exvol, R_ij = R_i - R_j)
 *       + zeta kappa (y_i - L_y/2) x                      (imposed shear)
 *   w_ij = exp(-R_ij^2 / 2 lambda^2)                      (entanglement weight)
 *   V_ij = kappa L_y n_ij x,  n_ij = round(y_ij / L_y)    (boundary correction)
 *
 *   (1 + alpha sum_j w_ij) v_i - alpha sum_j w_ij v_j = F_i / zeta + alpha sum_j V_ij w_ij
 *
 * Outputs: w[npairs] (one weight per pair), diag[n] = 1 + alpha sum_j w_ij,
 * b[n][3].  The paper's matrix shows w and F without alpha and zeta; Eq. vc
 * puts alpha on every pair term and divides F by zeta, which is what is
 * assembled here.  xi may be NULL (no noise).
 */
int or_assemble(const or_params* p, const double* pos, double delta, int64_t npairs,
                const int64_t* pairs, const double* xi, double* w, double* diag, double* b)
{
    or_derived dv;
    or_derive(p, &dv);
    int64_t n = p->n;
    double* sumw = (double*)calloc((size_t)n, sizeof(double));
    double* fev = (double*)calloc((size_t)(3 * n), sizeof(double));
    double* vw = (double*)calloc((size_t)n, sizeof(double)); /* sum_j n_ij w_ij */
    if (!sumw || !fev || !vw) {
        free(sumw); free(fev); free(vw);
        return OR_ERR_ARG;
    }
    for (int64_t k = 0; k < npairs; ++k) {
        int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
        double d[3], nimg;
        or_min_image(p, delta, pos + 3 * i, pos + 3 * j, d, &nimg);
        double r2 = sq_dist(d);
        double wij = exp(-r2 / (2.0 * dv.lambda2));
        w[k] = wij;
        sumw[i] += wij;
        sumw[j] += wij;
        for (int a = 0; a < 3; ++a) {
            fev[3 * i + a] += d[a] * wij;
            fev[3 * j + a] -= d[a] * wij;
        }
        vw[i] += nimg * wij;
        vw[j] -= nimg * wij;
    }
    for (int64_t i = 0; i < n; ++i) {
        diag[i] = 1.0 + p->alpha * sumw[i];
        double F[3];
        for (int a = 0; a < 3; ++a) {
            double noise = xi ? dv.noise_amp * xi[3 * i + a] : 0.0;
            F[a] = noise + dv.c_ev * fev[3 * i + a];
        }
        F[0] += p->zeta * p->kappa * (pos[3 * i + 1] - 0.5 * p->L[1]);
        for (int a = 0; a < 3; ++a) b[3 * i + a] = F[a] / p->zeta;
        b[3 * i + 0] += p->alpha * p->kappa * p->L[1] * vw[i];
    }
    free(sumw);
    free(fev);
    free(vw);
    return OR_OK;
}

/* y = A x for A = diag - alpha * W (Eq. algebra), acting on each of the three
 * Cartesian components (x, y are [n][3]). */
void or_matvec(int64_t n, double alpha, int64_t npairs, const int64_t* pairs, const double* w,
               const double* diag, const double* x, double* y)
{
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) y[3 * i + a] = diag[i] * x[3 * i + a];
    for (int64_t k = 0; k < npairs; ++k) {
        int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
        double c = alpha * w[k];
        for (int a = 0; a < 3; ++a) {
            y[3 * i + a] -= c * x[3 * j + a];
            y[3 * j + a] -= c * x[3 * i + a];
        }
    }
}

static double dot3n(int64_t m, const double* a, const double* b)
{
    double s = 0.0;
    for (int64_t k = 0; k < m; ++k) s += a[k] * b[k];
    return s;
}

/*
 * Jacobi-preconditioned conjugate gradients (Hestenes & Stiefel 1952) on the
 * 3n-dimensional system (A (x) I_3) v = b.  The three Cartesian components share
 * one scalar matrix, so they share the step lengths too.  Stops when the
 * recurrence residual satisfies ||r|| <= tol ||b|| (2-norm over all 3n
 * entries), then recomputes the true residual b - A x and restarts from it if
 * it does not meet tol.  x holds the start vector on entry.
 * info[0] = iterations, info[1] = final true relative residual.
 */
int or_pcg(int64_t n, double alpha, int64_t npairs, const int64_t* pairs, const double* w,
           const double* diag, const double* b, double tol, int64_t max_iter, double* x,
           double* info)
{
    int64_t m = 3 * n;
    double* r = (double*)malloc(sizeof(double) * m);
    double* z = (double*)malloc(sizeof(double) * m);
    double* pv = (double*)malloc(sizeof(double) * m);
    double* q = (double*)malloc(sizeof(double) * m);
    if (!r || !z || !pv || !q) {
        free(r); free(z); free(pv); free(q);
        return OR_ERR_ARG;
    }
    double bnorm = sqrt(dot3n(m, b, b));
    int64_t it = 0;
    int status = OR_ERR_NOT_CONVERGED;
    double rel = 0.0;
    for (int restart = 0; restart < 8; ++restart) {
        or_matvec(n, alpha, npairs, pairs, w, diag, x, q);
        for (int64_t k = 0; k < m; ++k) r[k] = b[k] - q[k];
        rel = bnorm > 0.0 ? sqrt(dot3n(m, r, r)) / bnorm : 0.0;
        if (rel <= tol) {
            status = OR_OK;
            break;
        }
        for (int64_t k = 0; k < m; ++k) z[k] = r[k] / diag[k / 3];
        for (int64_t k = 0; k < m; ++k) pv[k] = z[k];
        double rho = dot3n(m, r, z);
        while (it < max_iter) {
            or_matvec(n, alpha, npairs, pairs, w, diag, pv, q);
            double a = rho / dot3n(m, pv, q);
            for (int64_t k = 0; k < m; ++k) x[k] += a * pv[k];
            for (int64_t k = 0; k < m; ++k) r[k] -= a * q[k];
            ++it;
            if (sqrt(dot3n(m, r, r)) <= tol * bnorm) break;
            for (int64_t k = 0; k < m; ++k) z[k] = r[k] / diag[k / 3];
            double rho_new = dot3n(m, r, z);
            double beta = rho_new / rho;
            rho = rho_new;
            for (int64_t k = 0; k < m; ++k) pv[k] = z[k] + beta * pv[k];
        }
        if (it >= max_iter) {
            or_matvec(n, alpha, npairs, pairs, w, diag, x, q);
            for (int64_t k = 0; k < m; ++k) r[k] = b[k] - q[k];
            rel = bnorm > 0.0 ? sqrt(dot3n(m, r, r)) / bnorm : 0.0;
            status = rel <= tol ? OR_OK : OR_ERR_NOT_CONVERGED;
            break;
        }
    }
    info[0] = (double)it;
    info[1] = rel;
    free(r);
    free(z);
    free(pv);
    free(q);
    return status;
}

/* Eq. algebra solved directly: dense A = diag - alpha W, Cholesky A = L L^T
 * (textbook column-by-column), then forward and back substitution for the
 * three right-hand sides.  For tiny n only (n <= a few hundred). */
int or_dense_solve(int64_t n, double alpha, int64_t npairs, const int64_t* pairs, const double* w,
                   const double* diag, const double* b, double* x)
{
    double* A = (double*)calloc((size_t)(n * n), sizeof(double));
    if (!A) return OR_ERR_ARG;
    for (int64_t i = 0; i < n; ++i) A[i * n + i] = diag[i];
    for (int64_t k = 0; k < npairs; ++k) {
        int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
        A[i * n + j] -= alpha * w[k];
        A[j * n + i] -= alpha * w[k];
    }
    for (int64_t j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int64_t k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
        if (!(s > 0.0)) {
            free(A);
            return OR_ERR_NOT_SPD;
        }
        double ljj = sqrt(s);
        A[j * n + j] = ljj;
        for (int64_t i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int64_t k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / ljj;
        }
    }
    for (int a = 0; a < 3; ++a) {
        for (int64_t i = 0; i < n; ++i) {
            double t = b[3 * i + a];
            for (int64_t k = 0; k < i; ++k) t -= A[i * n + k] * x[3 * k + a];
            x[3 * i + a] = t / A[i * n + i];
        }
        for (int64_t i = n - 1; i >= 0; --i) {
            double t = x[3 * i + a];
            for (int64_t k = i + 1; k < n; ++k) t -= A[k * n + i] * x[3 * k + a];
            x[3 * i + a] = t / A[i * n + i];
        }
    }
    free(A);
    return OR_OK;
}

/* Wrap a coordinate into [0, L). */
static double wrap01(double x, double L)
{
    x = x - L * floor(x / L);
    if (x >= L) x = x - L;
    if (x < 0.0) x = 0.0;
    return x;
}

/* First-order update R += v dt (§Method: the equation of motion is first order
 * in time, v = dR/dt) followed by the Lees-Edwards wrap.  The image offset
 * advances first, delta(t+dt) = delta(t) + kappa L_y dt (mod L_x), and a
 * particle leaving through y = L_y re-enters at y - L_y shifted by -delta(t+dt)
 * in x (through y = 0: +delta(t+dt)).  Returns delta(t+dt). */
double or_integrate(const or_params* p, double* pos, const double* v, double delta)
{
    double dnew = wrap01(delta + p->kappa * p->L[1] * p->dt, p->L[0]);
    for (int64_t i = 0; i < p->n; ++i) {
        double x = pos[3 * i] + v[3 * i] * p->dt;
        double y = pos[3 * i + 1] + v[3 * i + 1] * p->dt;
        double z = pos[3 * i + 2] + v[3 * i + 2] * p->dt;
        if (y < 0.0) {
            y = y + p->L[1];
            x = x + dnew;
        }
        if (y >= p->L[1]) {
            y = y - p->L[1];
            x = x - dnew;
        }
        pos[3 * i] = wrap01(x, p->L[0]);
        pos[3 * i + 1] = y;
        pos[3 * i + 2] = wrap01(z, p->L[2]);
    }
    return dnew;
}

/* Eq. Sfactor at q_z = 0, S(q) = (1/n) |sum_c exp(-i q . R_c)|^2, by direct
 * summation.  Under Lees-Edwards the allowed wave vectors form the sheared
 * reciprocal lattice: q_x = 2 pi kx / L_x, q_y = 2 pi ky / L_y - (delta/L_y) q_x.
 * ks is [nk][2] integer pairs (kx, ky); outputs S, qx, qy of length nk. */
void or_structure_factor(const or_params* p, const double* pos, double delta, int64_t nk,
                         const int64_t* ks, double* S, double* qx, double* qy)
{
    const double two_pi = 6.283185307179586476925286766559;
    double gamma = delta / p->L[1];
    for (int64_t k = 0; k < nk; ++k) {
        double qxk = two_pi * (double)ks[2 * k] / p->L[0];
        double qyk = two_pi * (double)ks[2 * k + 1] / p->L[1] - gamma * qxk;
        double re = 0.0, im = 0.0;
        for (int64_t c = 0; c < p->n; ++c) {
            double ph = qxk * pos[3 * c] + qyk * pos[3 * c + 1];
            re += cos(ph);
            im -= sin(ph);
        }
        S[k] = (re * re + im * im) / (double)p->n;
        qx[k] = qxk;
        qy[k] = qyk;
    }
}

/* Shear stress from the pair forces.  The paper defines no stress; this is the
 * pair virial of the two pair forces of Eq. vc times zeta:
 *   f_ij = c_ev R_ij w_ij + zeta alpha w_ij (v_j - v_i + V_ij)   (force on i from j)
 *   sigma_xy = -(1/V) sum_{i<j} y_ij f_ij,x
 * (y_ij the minimum-image separation; the single-particle noise and shear
 * body forces carry no pair term). */
double or_stress_xy(const or_params* p, const double* pos, double delta, int64_t npairs,
                    const int64_t* pairs, const double* v)
{
    or_derived dv;
    or_derive(p, &dv);
    double s = 0.0;
    for (int64_t k = 0; k < npairs; ++k) {
        int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
        double d[3], nimg;
        or_min_image(p, delta, pos + 3 * i, pos + 3 * j, d, &nimg);
        double wij = exp(-sq_dist(d) / (2.0 * dv.lambda2));
        double fx = dv.c_ev * d[0] * wij
                  + p->zeta * p->alpha * wij * (v[3 * j] - v[3 * i] + p->kappa * p->L[1] * nimg);
        s += d[1] * fx;
    }
    return -s / (p->L[0] * p->L[1] * p->L[2]);
}

/* Row i alone: every j != i with |R_ij|^2 < r_c^2, by checking all particles
 * (brute force, for sampled checks of large systems).  Writes up to cap ids to
 * out in increasing j; returns the count. */
int64_t or_row_neighbors(const or_params* p, const double* pos, double delta, int64_t i, int64_t cap,
                         int64_t* out)
{
    or_derived dv;
    or_derive(p, &dv);
    int64_t m = 0;
    for (int64_t j = 0; j < p->n; ++j) {
        if (j == i) continue;
        double d[3], nimg;
        or_min_image(p, delta, pos + 3 * i, pos + 3 * j, d, &nimg);
        if (sq_dist(d) < dv.rc2) {
            if (m < cap) out[m] = j;
            ++m;
        }
    }
    return m;
}

/* Velocity cross-correlation versus distance (§Results, Fig. vv): the average
 * inter-chain velocity product <v_c . v_c'> / <v_c^2> as a function of the
 * inter-chain distance |R_cc'|.
 *   u_c = v_c - kappa (y_c - L_y/2) x   (velocity relative to the imposed flow;
 *         the Lees-Edwards image of c' moves with v_c' + kappa L_y n x, so it
 *         carries the same u; at kappa = 0, u = v)
 *   for every pair c < c' with R = the minimum-image separation and
 *   |R|^2 < rmax^2:  r = sqrt(|R|^2), k = floor(r * (nbins / rmax)) (nbins - 1
 *   where that rounds up to nbins), sum[k] += u_c . u_c', count[k] += 1
 *   vsq = (1/n) sum_c |u_c|^2;  the correlation of bin k is sum[k] / (count[k] vsq).
 * Every pair is checked (cost n^2 / 2). */
static void peculiar(const or_params* p, const double* pos, const double* v, int64_t c, double* u)
{
    u[0] = v[3 * c] - p->kappa * (pos[3 * c + 1] - 0.5 * p->L[1]);
    u[1] = v[3 * c + 1];
    u[2] = v[3 * c + 2];
}

void or_velocity_correlation(const or_params* p, const double* pos, double delta, const double* v,
                             int64_t nbins, double rmax, double* sum, int64_t* count, double* vsq)
{
    const double rmax2 = rmax * rmax;
    const double inv = (double)nbins / rmax;
    for (int64_t k = 0; k < nbins; ++k) {
        sum[k] = 0.0;
        count[k] = 0;
    }
    double s2 = 0.0;
    for (int64_t c = 0; c < p->n; ++c) {
        double uc[3];
        peculiar(p, pos, v, c, uc);
        s2 += uc[0] * uc[0] + uc[1] * uc[1] + uc[2] * uc[2];
        for (int64_t c2 = c + 1; c2 < p->n; ++c2) {
            double d[3], nimg;
            or_min_image(p, delta, pos + 3 * c, pos + 3 * c2, d, &nimg);
            double r2 = sq_dist(d);
            if (!(r2 < rmax2)) continue;
            int64_t k = (int64_t)floor(sqrt(r2) * inv);
            if (k > nbins - 1) k = nbins - 1;
            double u2[3];
            peculiar(p, pos, v, c2, u2);
            sum[k] += uc[0] * u2[0] + uc[1] * u2[1] + uc[2] * u2[2];
            count[k] += 1;
        }
    }
    *vsq = p->n > 0 ? s2 / (double)p->n : 0.0;
}
