/*
 * CPU oracle for the iterated direct-forcing immersed-boundary step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, FP64 restatement of
 * the method of Yao et al., "Particle-resolved simulations of four-way coupled
 * polydispersed, particle-laden flows" (arXiv 2109.03972).  Only the tests,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no code, header, table or constant generator with the GPU library.
 *
 * Build: cc -O2 -ffp-contract=off -fPIC -shared -o liboracle.so ibm_oracle.c -lm
 * (no FMA contraction, so each expression rounds exactly as written).
 *
 * Conventions (grid units).
 *   Grid: nx*ny*nz cells, spacing h, periodic in x, y, z.  Cell (i,j,k) has its
 *   centre at ((i+1/2)h, (j+1/2)h, (k+1/2)h); the collocated layout of Sec. 2.2
 *   (Fig. 1b).  Field arrays are [3][nz][ny][nx], x fastest.
 *   Marker l of particle p sits at X_l = x_p + r_l with r_l = (d_p/2) t_l, t_l a
 *   unit vector of the golden spiral (reading of Sec. 2.1, which fixes only the
 *   shell volume N_l dV_l and dV_l ~ h^3).  In grid units xi_l = x_p/h + a t_l
 *   with a = (d_p/2)/h.
 *   Weights: w_lc = phi(r_x) phi(r_y) phi(r_z), r = (i + 1/2) - xi (per axis),
 *   so that h^3 delta(x_c - X_l) = w_lc (Eq. 3pt-delta and its 3-D product).
 *
 * Parity status of each function is stated at the function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_PI 3.14159265358979323846

/* ------------------------------------------------------------------ kernels */

/* Three-point regularised delta, Eq. (3pt-stencil) (Roma et al.), printed form.
 * Pinned by: breakpoint values, continuity, partition of unity, zero first
 * moment, sum of squares = 1/2. */
double ora_phi3(double r)
{
    double a = fabs(r);
    if (a <= 0.5)
        return (1.0 + sqrt(-3.0 * a * a + 1.0)) / 3.0;
    if (a <= 1.5)
        return (5.0 - 3.0 * a - sqrt(-3.0 * (1.0 - a) * (1.0 - a) + 1.0)) / 6.0;
    return 0.0;
}

/* Four-point regularised delta, Eq. (4pt-stencil) (Peskin).  The printed range
 * of the first branch is garbled ("-2 <= r <= 1"); it is read as -2 <= r <= -1,
 * i.e. the symmetric |r| form below.  Pinned by: breakpoint values, even/odd
 * sums = 1/2 (Sec. 2.2.3), partition of unity, first moment 0, sum of squares
 * = 3/8. */
double ora_phi4(double r)
{
    double a = fabs(r);
    if (a <= 1.0)
        return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
    if (a <= 2.0)
        return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
    return 0.0;
}

/* d phi3 / dr, differentiated from Eq. (3pt-stencil).  Pinned by central
 * finite differences of ora_phi3 and by continuity at |r| = 1/2 and 3/2. */
double ora_dphi3(double r)
{
    double a = fabs(r), s = (r < 0.0) ? -1.0 : 1.0;
    if (a <= 0.5) {
        if (a == 0.0) return 0.0;
        return -r / sqrt(1.0 - 3.0 * a * a);
    }
    if (a <= 1.5) {
        double q = 1.0 - a;
        double root = sqrt(1.0 - 3.0 * q * q);
        /* d/da of (5 - 3a - root)/6, root' = 3q/root (q' = -1) */
        return s * (-3.0 - 3.0 * q / root) / 6.0;
    }
    return 0.0;
}

/* d phi4 / dr, differentiated from Eq. (4pt-stencil).  Pinned by central
 * finite differences of ora_phi4. */
double ora_dphi4(double r)
{
    double a = fabs(r), s = (r < 0.0) ? -1.0 : 1.0;
    if (a <= 1.0) {
        double root = sqrt(1.0 + 4.0 * a - 4.0 * a * a);
        return s * (-2.0 + (4.0 - 8.0 * a) / (2.0 * root)) / 8.0;
    }
    if (a < 2.0) {
        double root = sqrt(-7.0 + 12.0 * a - 4.0 * a * a);
        return s * (-2.0 - (12.0 - 8.0 * a) / (2.0 * root)) / 8.0;
    }
    return 0.0;
}

static double ora_phi(int width, double r) { return width == 4 ? ora_phi4(r) : ora_phi3(r); }
static double ora_dphi(int width, double r) { return width == 4 ? ora_dphi4(r) : ora_dphi3(r); }

/* ------------------------------------------------------------------ markers */

/* Marker count N_l = round(pi (d/h)^2), half away from zero (reading: the
 * paper states only N_l dV_l, Sec. 2.1, and dV_l ~ h^3; this gives 804 for
 * d = 16h, 452 for 12h, 1810 for 24h).  Pinned by those integers. */
long ora_marker_count(double d, double h)
{
    double q = d / h;
    long n = llround(ORA_PI * q * q);
    return n < 1 ? 1 : n;
}

/* Marker volume dV_l from N_l dV_l = (4/3) pi [(d/2 + h/2)^3 - (d/2 - h/2)^3]
 * (Sec. 2.1), expanded to pi (d^2 h + h^3/3) / N_l.  Pinned against the
 * printed shell-volume form. */
double ora_marker_volume(double d, double h, long nl)
{
    return ORA_PI * (d * d * h + h * h * h / 3.0) / (double)nl;
}

/* Golden-spiral unit directions t_l, l = 0..nl-1:
 *   z = 1 - (2l+1)/nl,  theta = l * pi (3 - sqrt 5),  rho = sqrt(1 - z^2),
 *   t = (rho cos theta, rho sin theta, z).
 * Reading of Sec. 2.1 (placement unspecified beyond spacing ~h).  Pinned by
 * |t| = 1, sum of z = 0 and the count/volume identities. */
void ora_marker_dirs(long nl, double *t)
{
    const double ga = ORA_PI * (3.0 - sqrt(5.0));
    for (long l = 0; l < nl; ++l) {
        double z = 1.0 - (double)(2 * l + 1) / (double)nl;
        double th = (double)l * ga;
        double rho = sqrt(1.0 - z * z);
        t[3 * l + 0] = rho * cos(th);
        t[3 * l + 1] = rho * sin(th);
        t[3 * l + 2] = z;
    }
}

/* ------------------------------------------------------------ problem state */

typedef struct {
    long n;            /* markers */
    long *pid;         /* owning particle */
    double *xi;        /* [n][3] marker position, grid units */
    double *r;         /* [n][3] arm r_l = X_l - x_p, physical units */
    double *D;         /* [n] dV_l / h^3 */
    double *Ud;        /* [n][3] desired velocity u_p + w_p x r_l (Sec. 2.1) */
} ora_markers;

static long iwrap(long i, long n) { long m = i % n; return m < 0 ? m + n : m; }

static int ora_build_markers(double h, long np, const double *x_p, const double *u_p,
                             const double *om_p, const double *d_p, ora_markers *M)
{
    long total = 0;
    for (long p = 0; p < np; ++p) total += ora_marker_count(d_p[p], h);
    M->n = total;
    M->pid = (long *)malloc(sizeof(long) * (total ? total : 1));
    M->xi = (double *)malloc(sizeof(double) * 3 * (total ? total : 1));
    M->r = (double *)malloc(sizeof(double) * 3 * (total ? total : 1));
    M->D = (double *)malloc(sizeof(double) * (total ? total : 1));
    M->Ud = (double *)malloc(sizeof(double) * 3 * (total ? total : 1));
    if (!M->pid || !M->xi || !M->r || !M->D || !M->Ud) return -1;
    long m = 0;
    for (long p = 0; p < np; ++p) {
        long nl = ora_marker_count(d_p[p], h);
        double dv = ora_marker_volume(d_p[p], h, nl);
        double *t = (double *)malloc(sizeof(double) * 3 * nl);
        if (!t) return -1;
        ora_marker_dirs(nl, t);
        double a = (0.5 * d_p[p]) / h;
        for (long l = 0; l < nl; ++l, ++m) {
            M->pid[m] = p;
            for (int c = 0; c < 3; ++c) {
                double xi_p = x_p[3 * p + c] / h;
                M->xi[3 * m + c] = xi_p + a * t[3 * l + c];
                M->r[3 * m + c] = (0.5 * d_p[p]) * t[3 * l + c];
            }
            M->D[m] = dv / (h * h * h);
            const double *w = om_p + 3 * p, *r = M->r + 3 * m;
            M->Ud[3 * m + 0] = u_p[3 * p + 0] + (w[1] * r[2] - w[2] * r[1]);
            M->Ud[3 * m + 1] = u_p[3 * p + 1] + (w[2] * r[0] - w[0] * r[2]);
            M->Ud[3 * m + 2] = u_p[3 * p + 2] + (w[0] * r[1] - w[1] * r[0]);
        }
        free(t);
    }
    return 0;
}

static void ora_free_markers(ora_markers *M)
{
    free(M->pid); free(M->xi); free(M->r); free(M->D); free(M->Ud);
}

/* Stencil of one marker along one axis: first cell index and the weights
 * (and derivative weights d/dxi) of the `width` cells.  3-point: base =
 * floor(xi), cells base-1..base+1.  4-point: base = floor(xi - 1/2), cells
 * base-1..base+2.  r = (i + 1/2) - xi. */
static long ora_axis_stencil(int width, double xi, double *w, double *dw)
{
    long first;
    if (width == 4) first = (long)floor(xi - 0.5) - 1;
    else first = (long)floor(xi) - 1;
    for (int a = 0; a < width; ++a) {
        double r = ((double)(first + a) + 0.5) - xi;
        w[a] = ora_phi(width, r);
        if (dw) dw[a] = -ora_dphi(width, r); /* d r / d xi = -1 */
    }
    return first;
}

/* Minimum-image offset r = (i + 1/2) - xi folded into [-n/2, n/2). */
static double ora_min_image(double r, long n)
{
    double L = (double)n;
    double q = r - L * floor(r / L + 0.5);
    return q;
}

/* Interpolation U_l = sum_c w_lc u_c (Sec. 2.2.2, step 1).  mode 0: stencil;
 * mode 1: brute force over every cell with minimum-image distances. */
static void ora_interp_all(int width, int mode, long nx, long ny, long nz,
                           const double *u, const ora_markers *M, double *U)
{
    const long ncell = nx * ny * nz;
    /* markers are independent: parallel over markers, results as in serial */
#pragma omp parallel for schedule(static) if (mode == 0)
    for (long m = 0; m < M->n; ++m) {
        double acc[3] = {0.0, 0.0, 0.0};
        const double *xi = M->xi + 3 * m;
        if (mode == 0) {
            double wx[4], wy[4], wz[4];
            long fx = ora_axis_stencil(width, xi[0], wx, NULL);
            long fy = ora_axis_stencil(width, xi[1], wy, NULL);
            long fz = ora_axis_stencil(width, xi[2], wz, NULL);
            for (int c = 0; c < width; ++c)
                for (int b = 0; b < width; ++b)
                    for (int a = 0; a < width; ++a) {
                        long i = iwrap(fx + a, nx), j = iwrap(fy + b, ny), k = iwrap(fz + c, nz);
                        long idx = i + nx * (j + ny * k);
                        double w = wx[a] * wy[b] * wz[c];
                        for (int q = 0; q < 3; ++q) acc[q] += w * u[q * ncell + idx];
                    }
        } else {
            for (long k = 0; k < nz; ++k)
                for (long j = 0; j < ny; ++j)
                    for (long i = 0; i < nx; ++i) {
                        double rx = ora_min_image((double)i + 0.5 - xi[0], nx);
                        double ry = ora_min_image((double)j + 0.5 - xi[1], ny);
                        double rz = ora_min_image((double)k + 0.5 - xi[2], nz);
                        double w = ora_phi(width, rx) * ora_phi(width, ry) * ora_phi(width, rz);
                        if (w == 0.0) continue;
                        long idx = i + nx * (j + ny * k);
                        for (int q = 0; q < 3; ++q) acc[q] += w * u[q * ncell + idx];
                    }
        }
        for (int q = 0; q < 3; ++q) U[3 * m + q] = acc[q];
    }
}

/* Spreading f_c = sum_l F_l w_lc D_l with D_l = dV_l/h^3 (Sec. 2.2.2, step 3:
 * f = sum F delta dV, h^3 delta = w).  f must be zeroed by the caller. */
static void ora_spread_all(int width, int mode, long nx, long ny, long nz,
                           const ora_markers *M, const double *F, double *f)
{
    const long ncell = nx * ny * nz;
    if (mode == 0) {
        /* Each thread owns a range of whole k-planes and visits every marker in
         * order, adding only to its own planes: every cell receives its
         * contributions in marker order, exactly as in the serial loop. */
#pragma omp parallel
        {
            long k0 = 0, k1 = nz;
#ifdef _OPENMP
            const int nt = omp_get_num_threads(), t = omp_get_thread_num();
            k0 = nz * t / nt;
            k1 = nz * (t + 1) / nt;
#endif
            for (long m = 0; m < M->n; ++m) {
                const double *xi = M->xi + 3 * m;
                double wx[4], wy[4], wz[4];
                long fz = ora_axis_stencil(width, xi[2], wz, NULL);
                int any = 0;
                for (int c = 0; c < width; ++c) {
                    long k = iwrap(fz + c, nz);
                    if (k >= k0 && k < k1) any = 1;
                }
                if (!any) continue;
                long fx = ora_axis_stencil(width, xi[0], wx, NULL);
                long fy = ora_axis_stencil(width, xi[1], wy, NULL);
                double g[3];
                for (int q = 0; q < 3; ++q) g[q] = F[3 * m + q] * M->D[m];
                for (int c = 0; c < width; ++c) {
                    long k = iwrap(fz + c, nz);
                    if (k < k0 || k >= k1) continue;
                    for (int b = 0; b < width; ++b)
                        for (int a = 0; a < width; ++a) {
                            long i = iwrap(fx + a, nx), j = iwrap(fy + b, ny);
                            long idx = i + nx * (j + ny * k);
                            double w = wx[a] * wy[b] * wz[c];
                            for (int q = 0; q < 3; ++q) f[q * ncell + idx] += w * g[q];
                        }
                }
            }
        }
        return;
    }
    for (long m = 0; m < M->n; ++m) {
        const double *xi = M->xi + 3 * m;
        double g[3];
        for (int q = 0; q < 3; ++q) g[q] = F[3 * m + q] * M->D[m];
        if (mode == 0) {
            double wx[4], wy[4], wz[4];
            long fx = ora_axis_stencil(width, xi[0], wx, NULL);
            long fy = ora_axis_stencil(width, xi[1], wy, NULL);
            long fz = ora_axis_stencil(width, xi[2], wz, NULL);
            for (int c = 0; c < width; ++c)
                for (int b = 0; b < width; ++b)
                    for (int a = 0; a < width; ++a) {
                        long i = iwrap(fx + a, nx), j = iwrap(fy + b, ny), k = iwrap(fz + c, nz);
                        long idx = i + nx * (j + ny * k);
                        double w = wx[a] * wy[b] * wz[c];
                        for (int q = 0; q < 3; ++q) f[q * ncell + idx] += w * g[q];
                    }
        } else {
            for (long k = 0; k < nz; ++k)
                for (long j = 0; j < ny; ++j)
                    for (long i = 0; i < nx; ++i) {
                        double rx = ora_min_image((double)i + 0.5 - xi[0], nx);
                        double ry = ora_min_image((double)j + 0.5 - xi[1], ny);
                        double rz = ora_min_image((double)k + 0.5 - xi[2], nz);
                        double w = ora_phi(width, rx) * ora_phi(width, ry) * ora_phi(width, rz);
                        if (w == 0.0) continue;
                        long idx = i + nx * (j + ny * k);
                        for (int q = 0; q < 3; ++q) f[q * ncell + idx] += w * g[q];
                    }
        }
    }
}

/* ------------------------------------------------------------ public entries */

/* Exposed single operators (used by the adjointness and brute-force pins).
 * ora_interpolate: U[n_markers][3] = W u.  ora_spread: f[3][cells] = W^T D F
 * (accumulated into f, which the caller zeroes).  Markers are generated from
 * the particles exactly as in ora_forcing_step.  Returns the marker count or
 * -1 on allocation failure. */
long ora_interpolate(int width, int mode, long nx, long ny, long nz, double h,
                     long np, const double *x_p, const double *d_p,
                     const double *u, double *U)
{
    ora_markers M;
    double *zero = (double *)calloc(3 * (size_t)(np ? np : 1), sizeof(double));
    if (!zero || ora_build_markers(h, np, x_p, zero, zero, d_p, &M)) return -1;
    if (U) ora_interp_all(width, mode, nx, ny, nz, u, &M, U);
    long n = M.n;
    ora_free_markers(&M);
    free(zero);
    return n;
}

long ora_spread(int width, int mode, long nx, long ny, long nz, double h,
                long np, const double *x_p, const double *d_p,
                const double *F, double *f)
{
    ora_markers M;
    double *zero = (double *)calloc(3 * (size_t)(np ? np : 1), sizeof(double));
    if (!zero || ora_build_markers(h, np, x_p, zero, zero, d_p, &M)) return -1;
    ora_spread_all(width, mode, nx, ny, nz, &M, F, f);
    long n = M.n;
    ora_free_markers(&M);
    free(zero);
    return n;
}

/* Marker positions (grid units) and stencil base cells, in particle-then-l
 * order.  base[m][c] = floor(xi) for the 3-point kernel (floor(xi - 1/2) for
 * width 4), NOT wrapped.  Either output may be NULL.  Returns the count. */
long ora_marker_positions(int width, double h, long np, const double *x_p, const double *d_p,
                          double *xi_out, int64_t *base_out)
{
    ora_markers M;
    double *zero = (double *)calloc(3 * (size_t)(np ? np : 1), sizeof(double));
    if (!zero || ora_build_markers(h, np, x_p, zero, zero, d_p, &M)) return -1;
    for (long m = 0; m < M.n; ++m)
        for (int c = 0; c < 3; ++c) {
            double xi = M.xi[3 * m + c];
            if (xi_out) xi_out[3 * m + c] = xi;
            if (base_out) base_out[3 * m + c] = (int64_t)floor(width == 4 ? xi - 0.5 : xi);
        }
    long n = M.n;
    ora_free_markers(&M);
    free(zero);
    return n;
}

/* Number of distinct cells touched by the union of marker stencils (a bitmap
 * over the grid).  This is the count the algorithmic-byte figures use. */
long ora_touched_count(int width, long nx, long ny, long nz, double h, long np,
                       const double *x_p, const double *d_p)
{
    ora_markers M;
    double *zero = (double *)calloc(3 * (size_t)(np ? np : 1), sizeof(double));
    unsigned char *bm = (unsigned char *)calloc((size_t)(nx * ny * nz), 1);
    if (!zero || !bm || ora_build_markers(h, np, x_p, zero, zero, d_p, &M)) return -1;
    long cnt = 0;
    for (long m = 0; m < M.n; ++m) {
        double wx[4], wy[4], wz[4];
        long fx = ora_axis_stencil(width, M.xi[3 * m + 0], wx, NULL);
        long fy = ora_axis_stencil(width, M.xi[3 * m + 1], wy, NULL);
        long fz = ora_axis_stencil(width, M.xi[3 * m + 2], wz, NULL);
        for (int c = 0; c < width; ++c)
            for (int b = 0; b < width; ++b)
                for (int a = 0; a < width; ++a) {
                    long idx = iwrap(fx + a, nx) + nx * (iwrap(fy + b, ny) + ny * iwrap(fz + c, nz));
                    if (!bm[idx]) { bm[idx] = 1; ++cnt; }
                }
    }
    ora_free_markers(&M);
    free(zero); free(bm);
    return cnt;
}

/* The outer forcing loop of Sec. 2.2.2, m = 1..n_f:
 *   1. U^{m-1}_l = sum_c w_lc u^{m-1}_c
 *   2. F^{m-1}_l = (U^d_l - U^{m-1}_l) / tau            (tau = 2 alpha_k dt)
 *   3. f^{m-1}_c = sum_l F^{m-1}_l w_lc D_l               (full-grid f)
 *   4. u^m = u^{m-1} + tau f^{m-1}
 * and the fluid-side particle loads of Eq. (basic-particle a,b), summed over
 * the iterations (reading: the paper does not say which iteration's force
 * feeds the particle; the sum is the total momentum the loop transfers):
 *   F_p += sum_l F_l dV_l,  T_p += sum_l r_l x F_l dV_l.
 * The load on the particle is -rho_f times these (Eq. basic-particle a,b).
 *
 * u      [3][nz][ny][nx], updated in place.
 * F_out, T_out  [np][3], overwritten.
 * f_tot  optional [3][cells]: sum over m of f^{m-1} (overwritten).
 * slip   optional [2]: RMS and max over markers of |U^d - W u^{n_f}| after
 *        the loop (reading of the pointwise error eps of Sec. 2.2.2).
 * mode   0 = stencil sums, 1 = brute force over every cell (tiny grids).
 * Fabs_out optional [np]: sum over m and l of |F^m_l| dV_l (the scale the
 *        load tolerances are stated against).
 * Returns 0, or -1 on allocation failure.
 * Parity: pinned by the single-marker closed form, the dense linear-algebra
 * recursion, the no-op cases and the load identities (tests). */
/* Forcing loop of Sec. 2.2.2 with some markers left out of f_IBM (Sec. 2.2.5):
 * disabled[m] != 0 (markers in particle-then-l order; NULL = none) gives
 * marker m the force F_m = 0 in every iteration, so it neither spreads nor adds
 * to the loads.  The slip is still reported over all markers. */
int ora_forcing_step_masked(int width, int mode, long nx, long ny, long nz, double h,
                            int n_forcing, double tau, long np,
                            const double *x_p, const double *u_p, const double *om_p,
                            const double *d_p, double *u, double *F_out, double *T_out,
                            double *f_tot, double *slip, double *Fabs_out,
                            const unsigned char *disabled)
{
    const long ncell = nx * ny * nz;
    ora_markers M;
    if (ora_build_markers(h, np, x_p, u_p, om_p, d_p, &M)) return -1;
    double *U = (double *)malloc(sizeof(double) * 3 * (M.n ? M.n : 1));
    double *F = (double *)malloc(sizeof(double) * 3 * (M.n ? M.n : 1));
    double *f = (double *)malloc(sizeof(double) * 3 * (size_t)ncell);
    if (!U || !F || !f) return -1;
    for (long i = 0; i < 3 * np; ++i) { F_out[i] = 0.0; T_out[i] = 0.0; }
    if (Fabs_out) for (long i = 0; i < np; ++i) Fabs_out[i] = 0.0;
    if (f_tot) memset(f_tot, 0, sizeof(double) * 3 * (size_t)ncell);
    const double h3 = h * h * h;

    for (int it = 0; it < n_forcing; ++it) {
        ora_interp_all(width, mode, nx, ny, nz, u, &M, U);
        for (long m = 0; m < M.n; ++m)
            for (int q = 0; q < 3; ++q)
                F[3 * m + q] = (disabled && disabled[m]) ? 0.0 : (M.Ud[3 * m + q] - U[3 * m + q]) / tau;
#pragma omp parallel for schedule(static)
        for (long c = 0; c < 3 * ncell; ++c) f[c] = 0.0;
        ora_spread_all(width, mode, nx, ny, nz, &M, F, f);
#pragma omp parallel for schedule(static)
        for (long c = 0; c < 3 * ncell; ++c) u[c] += tau * f[c];
        if (f_tot)
#pragma omp parallel for schedule(static)
            for (long c = 0; c < 3 * ncell; ++c) f_tot[c] += f[c];
        for (long m = 0; m < M.n; ++m) {
            long p = M.pid[m];
            double dv = M.D[m] * h3;
            const double *r = M.r + 3 * m, *Fm = F + 3 * m;
            for (int q = 0; q < 3; ++q) F_out[3 * p + q] += Fm[q] * dv;
            T_out[3 * p + 0] += (r[1] * Fm[2] - r[2] * Fm[1]) * dv;
            T_out[3 * p + 1] += (r[2] * Fm[0] - r[0] * Fm[2]) * dv;
            T_out[3 * p + 2] += (r[0] * Fm[1] - r[1] * Fm[0]) * dv;
            if (Fabs_out)
                Fabs_out[p] += sqrt(Fm[0] * Fm[0] + Fm[1] * Fm[1] + Fm[2] * Fm[2]) * dv;
        }
    }
    if (slip) {
        ora_interp_all(width, mode, nx, ny, nz, u, &M, U);
        double s2 = 0.0, mx = 0.0;
        for (long m = 0; m < M.n; ++m) {
            double e2 = 0.0;
            for (int q = 0; q < 3; ++q) {
                double e = M.Ud[3 * m + q] - U[3 * m + q];
                e2 += e * e;
            }
            s2 += e2;
            if (sqrt(e2) > mx) mx = sqrt(e2);
        }
        slip[0] = M.n ? sqrt(s2 / (double)M.n) : 0.0;
        slip[1] = mx;
    }
    free(U); free(F); free(f);
    ora_free_markers(&M);
    return 0;
}

int ora_forcing_step(int width, int mode, long nx, long ny, long nz, double h,
                     int n_forcing, double tau, long np,
                     const double *x_p, const double *u_p, const double *om_p,
                     const double *d_p, double *u, double *F_out, double *T_out,
                     double *f_tot, double *slip, double *Fabs_out)
{
    return ora_forcing_step_masked(width, mode, nx, ny, nz, h, n_forcing, tau, np, x_p, u_p, om_p, d_p, u,
                                   F_out, T_out, f_tot, slip, Fabs_out, NULL);
}

/* SplitMix64 output function (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014): the state advanced once by the
 * golden-ratio increment, then two xor-shift-multiply rounds and a final
 * xor-shift.  Used as a counter-based coin for the pair choice below. */
static uint64_t ora_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* The SplitMix64 output for state x (exported for its pin against the
 * generator's published outputs). */
uint64_t ora_splitmix64_out(uint64_t x) { return ora_splitmix64(x); }

/* Marker exclusion near contact, Sec. 2.2.5 (reading).  For every pair p < q
 * of the scene whose surface gap zeta = |x_q - x_p| - a_p - a_q (minimum
 * image) is below 2 eps_sep, one particle of the pair is chosen at random: with
 * i < j the pair's ids (ids[p], ids[q], or p, q when ids is NULL),
 * z = splitmix64(seed ^ (i << 32 | j)) and the chosen one is j if the top bit of
 * z is set, else i.  The chosen particle's markers whose distance to the other
 * particle's surface, |X_l - x_other| - a_other (minimum image), is below
 * 2 eps_sep are disabled.  All pairs by brute force, FP64, grid units.
 * disabled[n_markers] receives 0/1 (particle-then-l order); returns the marker
 * count, -1 on allocation failure.
 * Pinned by: no pair within reach leaves every marker on; the disabled set is a
 * cap facing the partner whose size matches the spherical-cap area; the choice
 * falls on either particle about equally often. */
long ora_contact_exclusion(long nx, long ny, long nz, double h, long np, const double *x_p,
                           const double *d_p, double eps_sep, uint64_t seed, const int64_t *ids,
                           unsigned char *disabled)
{
    ora_markers M;
    double *zero = (double *)calloc(3 * (size_t)(np ? np : 1), sizeof(double));
    long *first = (long *)malloc(sizeof(long) * (size_t)(np + 1));
    if (!zero || !first || ora_build_markers(h, np, x_p, zero, zero, d_p, &M)) return -1;
    first[0] = 0;
    for (long p = 0; p < np; ++p) first[p + 1] = first[p] + ora_marker_count(d_p[p], h);
    for (long m = 0; m < M.n; ++m) disabled[m] = 0;
    const long n[3] = {nx, ny, nz};
    const double lim = 2.0 * eps_sep / h;
    for (long p = 0; p < np; ++p)
        for (long q = p + 1; q < np; ++q) {
            const double ap = 0.5 * d_p[p] / h, aq = 0.5 * d_p[q] / h;
            double d2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                double dv = ora_min_image(x_p[3 * q + c] / h - x_p[3 * p + c] / h, n[c]);
                d2 += dv * dv;
            }
            if (!(sqrt(d2) - ap - aq < lim)) continue;
            uint64_t i = ids ? (uint64_t)ids[p] : (uint64_t)p, j = ids ? (uint64_t)ids[q] : (uint64_t)q;
            int swap = i > j;
            if (swap) { uint64_t t = i; i = j; j = t; }
            const int pick_j = (int)(ora_splitmix64(seed ^ ((i << 32) | j)) >> 63);
            /* pick_j chooses the particle with the larger id */
            const long e = (pick_j != swap) ? q : p, o = (e == q) ? p : q;
            const double ao = 0.5 * d_p[o] / h;
            for (long m = first[e]; m < first[e + 1]; ++m) {
                double r2 = 0.0;
                for (int c = 0; c < 3; ++c) {
                    double dv = ora_min_image(M.xi[3 * m + c] - x_p[3 * o + c] / h, n[c]);
                    r2 += dv * dv;
                }
                if (sqrt(r2) - ao < lim) disabled[m] = 1;
            }
        }
    long nm = M.n;
    ora_free_markers(&M);
    free(zero);
    free(first);
    return nm;
}

/* Fluid inertia inside each particle, Sec. 2.2.9 (midpoint quadrature with a
 * level-set volume fraction):
 *   Iu_p = sum_c alpha_c h^3 u_c,   Ir_p = sum_c alpha_c h^3 (r_c x u_c),
 *   V_p  = sum_c alpha_c h^3,
 * alpha_c = sum_m -phi_m H(-phi_m) / sum_m |phi_m| over the 8 corners m of cell
 * c, H(-phi) = 1 for phi <= 0.  Reading: phi_m is the signed distance of the
 * corner to the sphere's surface, |x_m - x_p| - d_p/2 (the printed "distance to
 * the centre" is never negative, which would make alpha vanish).  r_c is the
 * cell centre minus x_p, taken from the unwrapped cell index of the box around
 * x_p; the field value at the wrapped index.  Every cell of the box
 * floor(x_p/h - a) - 1 .. floor(x_p/h + a) + 1 per axis (a = d_p/2h) is
 * visited, by plain loops.  Iu, Ir: [np][3]; V: [np] (any may be NULL).
 * Pinned by: alpha = 1 / 0 deep inside / outside, V_p against the sphere
 * volume, a uniform field, and a rigid rotation (int r x (w x r) dV =
 * (2/5) a^2 V w). */
void ora_particle_inertia(long nx, long ny, long nz, double h, long np, const double *x_p, const double *d_p,
                          const double *u, double *Iu, double *Ir, double *V)
{
    const long ncell = nx * ny * nz;
    const long n[3] = {nx, ny, nz};
    for (long p = 0; p < np; ++p) {
        const double a = 0.5 * d_p[p] / h;
        double xi[3], su[3] = {0, 0, 0}, sr[3] = {0, 0, 0}, sv = 0.0;
        long lo[3], hi[3];
        for (int c = 0; c < 3; ++c) {
            xi[c] = x_p[3 * p + c] / h;
            lo[c] = (long)floor(xi[c] - a) - 1;
            hi[c] = (long)floor(xi[c] + a) + 1;
        }
        for (long k = lo[2]; k <= hi[2]; ++k)
            for (long j = lo[1]; j <= hi[1]; ++j)
                for (long i = lo[0]; i <= hi[0]; ++i) {
                    double num = 0.0, den = 0.0;
                    for (int m = 0; m < 8; ++m) {
                        const double cx = (double)(i + (m & 1)) - xi[0];
                        const double cy = (double)(j + ((m >> 1) & 1)) - xi[1];
                        const double cz = (double)(k + ((m >> 2) & 1)) - xi[2];
                        const double phi = sqrt(cx * cx + cy * cy + cz * cz) - a;
                        if (phi <= 0.0) num += -phi;
                        den += fabs(phi);
                    }
                    const double alpha = den > 0.0 ? num / den : 0.0;
                    if (alpha == 0.0) continue;
                    const long idx = (iwrap(k, n[2]) * ny + iwrap(j, n[1])) * nx + iwrap(i, n[0]);
                    const double uc[3] = {u[idx], u[ncell + idx], u[2 * ncell + idx]};
                    const double r[3] = {((double)i + 0.5 - xi[0]) * h, ((double)j + 0.5 - xi[1]) * h,
                                         ((double)k + 0.5 - xi[2]) * h};
                    const double w = alpha * h * h * h;
                    for (int c = 0; c < 3; ++c) su[c] += w * uc[c];
                    sr[0] += w * (r[1] * uc[2] - r[2] * uc[1]);
                    sr[1] += w * (r[2] * uc[0] - r[0] * uc[2]);
                    sr[2] += w * (r[0] * uc[1] - r[1] * uc[0]);
                    sv += w;
                }
        for (int c = 0; c < 3; ++c) {
            if (Iu) Iu[3 * p + c] = su[c];
            if (Ir) Ir[3 * p + c] = sr[c];
        }
        if (V) V[p] = sv;
    }
}

/* Number of OpenMP threads of the oracle (1 without OpenMP); n > 0 sets it.
 * The results do not depend on it. */
int ora_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Rigid-body Newton-Euler update of Eq. (basic-particle a-c) with no collision
 * force or torque (F_c = T_c = 0) and tau = 2 alpha_k dt:
 *   u_p' = u_p + tau [ rho_p rho_f / (m_p (rho_p - rho_f)) (-F_p) + g ]
 *   w_p' = w_p + tau   rho_p rho_f / (I_p (rho_p - rho_f)) (-T_p)
 *   x_p' = x_p + (tau/2)(u_p' + u_p)
 * with m_p = rho_p pi d^3 / 6 and I_p = m_p d^2 / 10 (solid sphere).  F_p, T_p
 * are the fluid-side sums of ora_forcing_step.  In place. */
void ora_newton_euler(long np, double *x_p, double *u_p, double *om_p,
                      const double *d_p, const double *rho_p, double rho_f,
                      const double *g, double tau, const double *F_p, const double *T_p)
{
    for (long p = 0; p < np; ++p) {
        double d = d_p[p];
        double m = rho_p[p] * ORA_PI * d * d * d / 6.0;
        double I = m * d * d / 10.0;
        double cf = rho_p[p] * rho_f / (m * (rho_p[p] - rho_f));
        double ct = rho_p[p] * rho_f / (I * (rho_p[p] - rho_f));
        for (int q = 0; q < 3; ++q) {
            double uold = u_p[3 * p + q];
            double unew = uold + tau * (cf * (-F_p[3 * p + q]) + g[q]);
            u_p[3 * p + q] = unew;
            om_p[3 * p + q] = om_p[3 * p + q] + tau * ct * (-T_p[3 * p + q]);
            x_p[3 * p + q] = x_p[3 * p + q] + 0.5 * tau * (unew + uold);
        }
    }
}

/* Adjoint of the forcing loop for L(u^{n_f}) (derived from the loop algebra of
 * Sec. 2.2.2; the paper has no backward pass).  With e^m = U^d - W u^{m-1} and
 * u^m = u^{m-1} + W^T D e^m, and g^m = dL/du^m (g^{n_f} = grad_u_out):
 *   g^{m-1}  = g^m - W^T D W g^m
 *   dL/dU^d_l += D_l (W g^m)_l
 *   dL/dX_l  += D_l [ (grad W g^m)_l^T e^m_l - (grad W u^{m-1})_l^T (W g^m)_l ]
 * then dL/du_p = sum_l dL/dU^d_l, dL/dw_p = sum_l r_l x dL/dU^d_l and
 * dL/dx_p = sum_l dL/dX_l (X_l = x_p + r_l; r_l does not depend on x_p).
 * grad W is taken with respect to the physical marker position (d/dX = (1/h)
 * d/dxi).  Markers and weights are recomputed from the particles.
 * u0: [3][cells] initial field (not modified).  grad_u_in [3][cells] output.
 * gU, gW, gX: [np][3] outputs.  Returns 0 or -1.
 * Parity: pinned by the dot-product test and central finite differences of
 * ora_forcing_step (tests). */
int ora_backward(int width, long nx, long ny, long nz, double h, int n_forcing,
                 long np, const double *x_p, const double *u_p, const double *om_p,
                 const double *d_p, const double *u0, const double *grad_u_out,
                 double *grad_u_in, double *gU, double *gW, double *gX)
{
    const long ncell = nx * ny * nz;
    ora_markers M;
    if (ora_build_markers(h, np, x_p, u_p, om_p, d_p, &M)) return -1;
    const long nm = M.n ? M.n : 1;
    double *us = (double *)malloc(sizeof(double) * 3 * (size_t)ncell * (size_t)(n_forcing + 1));
    double *U = (double *)malloc(sizeof(double) * 3 * nm);
    double *E = (double *)malloc(sizeof(double) * 3 * nm * (size_t)n_forcing);
    double *Wg = (double *)malloc(sizeof(double) * 3 * nm);
    double *f = (double *)malloc(sizeof(double) * 3 * (size_t)ncell);
    double *gXm = (double *)calloc(3 * nm, sizeof(double));
    double *gUd = (double *)calloc(3 * nm, sizeof(double));
    if (!us || !U || !E || !Wg || !f || !gXm || !gUd) return -1;

    /* forward replay, keeping every u^m and e^m */
    memcpy(us, u0, sizeof(double) * 3 * (size_t)ncell);
    for (int it = 0; it < n_forcing; ++it) {
        double *ucur = us + (size_t)it * 3 * ncell, *unext = ucur + 3 * ncell;
        ora_interp_all(width, 0, nx, ny, nz, ucur, &M, U);
        double *e = E + (size_t)it * 3 * nm;
        for (long m = 0; m < M.n; ++m)
            for (int q = 0; q < 3; ++q) e[3 * m + q] = M.Ud[3 * m + q] - U[3 * m + q];
        memset(f, 0, sizeof(double) * 3 * (size_t)ncell);
        ora_spread_all(width, 0, nx, ny, nz, &M, e, f);   /* W^T D e */
        for (long c = 0; c < 3 * ncell; ++c) unext[c] = ucur[c] + f[c];
    }

    memcpy(grad_u_in, grad_u_out, sizeof(double) * 3 * (size_t)ncell);
    for (int it = n_forcing - 1; it >= 0; --it) {
        const double *uprev = us + (size_t)it * 3 * ncell;   /* u^{m-1} */
        const double *e = E + (size_t)it * 3 * nm;           /* e^m */
        ora_interp_all(width, 0, nx, ny, nz, grad_u_in, &M, Wg);  /* W g^m */
        for (long m = 0; m < M.n; ++m) {
            const double *xi = M.xi + 3 * m;
            double wx[4], wy[4], wz[4], dx[4], dy[4], dz[4];
            long fx = ora_axis_stencil(width, xi[0], wx, dx);
            long fy = ora_axis_stencil(width, xi[1], wy, dy);
            long fz = ora_axis_stencil(width, xi[2], wz, dz);
            double Gg[3][3] = {{0}}, Gu[3][3] = {{0}}; /* [beta][alpha] */
            for (int c = 0; c < width; ++c)
                for (int b = 0; b < width; ++b)
                    for (int a = 0; a < width; ++a) {
                        long idx = iwrap(fx + a, nx) + nx * (iwrap(fy + b, ny) + ny * iwrap(fz + c, nz));
                        double d0 = dx[a] * wy[b] * wz[c] / h;
                        double d1 = wx[a] * dy[b] * wz[c] / h;
                        double d2 = wx[a] * wy[b] * dz[c] / h;
                        for (int q = 0; q < 3; ++q) {
                            double gv = grad_u_in[q * ncell + idx], uv = uprev[q * ncell + idx];
                            Gg[0][q] += d0 * gv; Gg[1][q] += d1 * gv; Gg[2][q] += d2 * gv;
                            Gu[0][q] += d0 * uv; Gu[1][q] += d1 * uv; Gu[2][q] += d2 * uv;
                        }
                    }
            for (int bta = 0; bta < 3; ++bta) {
                double s = 0.0;
                for (int q = 0; q < 3; ++q)
                    s += e[3 * m + q] * Gg[bta][q] - Wg[3 * m + q] * Gu[bta][q];
                gXm[3 * m + bta] += M.D[m] * s;
            }
            for (int q = 0; q < 3; ++q) gUd[3 * m + q] += M.D[m] * Wg[3 * m + q];
        }
        memset(f, 0, sizeof(double) * 3 * (size_t)ncell);
        ora_spread_all(width, 0, nx, ny, nz, &M, Wg, f);   /* W^T D W g */
        for (long c = 0; c < 3 * ncell; ++c) grad_u_in[c] -= f[c];
    }
    for (long i = 0; i < 3 * np; ++i) { gU[i] = 0.0; gW[i] = 0.0; gX[i] = 0.0; }
    for (long m = 0; m < M.n; ++m) {
        long p = M.pid[m];
        const double *r = M.r + 3 * m, *a = gUd + 3 * m;
        for (int q = 0; q < 3; ++q) { gU[3 * p + q] += a[q]; gX[3 * p + q] += gXm[3 * m + q]; }
        gW[3 * p + 0] += r[1] * a[2] - r[2] * a[1];
        gW[3 * p + 1] += r[2] * a[0] - r[0] * a[2];
        gW[3 * p + 2] += r[0] * a[1] - r[1] * a[0];
    }
    free(us); free(U); free(E); free(Wg); free(f); free(gXm); free(gUd);
    ora_free_markers(&M);
    return 0;
}
