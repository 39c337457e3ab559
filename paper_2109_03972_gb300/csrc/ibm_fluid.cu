// Collocated fractional-step fluid solver of the modified method (Sec. 2.2.3
// "Pressure-momentum coupling on a collocated grid", Sec. 2.2.4-2.2.5 and the
// steps (a)-(i) of Eq. fluid-solver) on one triply periodic grid, FP64.
//
// Kernels (one thread per cell, x fastest, grid-stride loops; the neighbours
// of a 7-point stencil come through L1/L2, so each field is read from HBM
// about once per pass):
//   k_fl_predict   step (a): u~ and the stage's convective term N(u)
//   k_fl_hrhs      right-hand side of step (e) for one component
//   k_fl_prhs      step (f) and the right-hand side of step (g): the face
//                  velocities and -div u_f* / (2 alpha dt), with per-block
//                  partial sums for its mean
//   k_fl_correct   steps (h) and (i)
//   multigrid      k_mg_smooth (red-black Gauss-Seidel), k_mg_restrict
//                  (residual averaged over the 8 children), k_mg_prolong
//                  (trilinear correction), k_mg_cg (one-CTA conjugate
//                  gradients on the coarsest level), k_mg_resid (max norm)
// Reductions are deterministic: per-block tree sums in a fixed order and a
// one-block final sum; maxima by 64-bit atomicMax on the bit patterns of
// non-negative doubles, whose order is the order of the values.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ibm_internal.h"

struct ibm_fluid {
    ibm_fluid_config cfg;
    cudaStream_t stream = nullptr;
    int n[3] = {0, 0, 0};
    long long cells = 0;
    double *nold = nullptr;     // [3][cells] convective term of the last stage
    double *rhs = nullptr;      // level-0 right-hand side
    double *f = nullptr;        // [3][cells] f_IBM of ibm_fluid_stage (lazy)
    double *red = nullptr;      // partial sums [kRedBlocks] + scalars
    unsigned long long *maxw = nullptr;  // [2]: max|b|, max|r|
    double *mean = nullptr;     // [4]: mean_f[3] (host input copy), mean of a field
    unsigned long long *hmax = nullptr;  // pinned [2]
    struct Level {
        int n[3];
        long long cells;
        double h;
        double *x, *b;          // level 0: x external, b = rhs
    };
    std::vector<Level> lv;
    double *cg = nullptr;       // r, p, q of the coarsest level
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int64_t cycles[4] = {0, 0, 0, 0};
    double resid[4] = {0, 0, 0, 0};
    std::string last_error;
};

namespace {

constexpr int kFlThreads = 256;
constexpr int kRedBlocks = 1216;      // 152 SMs x 8: fixed, so that partial sums are deterministic
constexpr int kCgThreads = 1024;
constexpr long long kCoarseMax = 32768;

// RK3 coefficients of Rai and Moin (Sec. 2.2.1)
constexpr double kAlpha[3] = {4.0 / 15.0, 1.0 / 15.0, 1.0 / 6.0};
constexpr double kGamma[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
constexpr double kZeta[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};

ibm_status fl_fail(ibm_fluid *fl, ibm_status s, const std::string &m) {
    if (fl) fl->last_error = m;
    return s;
}

ibm_status fl_cuda(ibm_fluid *fl, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return IBM_OK;
    cudaGetLastError();
    return fl_fail(fl, e == cudaErrorMemoryAllocation ? IBM_ERR_OOM : IBM_ERR_CUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

#define FK(call, what)                                          \
    do {                                                        \
        ibm_status _s = fl_cuda(fl, (call), what);              \
        if (_s != IBM_OK) return _s;                            \
    } while (0)

int grid_cells(long long n) {
    long long g = (n + kFlThreads - 1) / kFlThreads;
    return (int)std::max(1ll, std::min(g, 152ll * 32));
}

// Cell coordinates and the six periodic neighbours of linear index c.
struct Nb {
    long long xp, xm, yp, ym, zp, zm;
};

__device__ __forceinline__ Nb neighbours(long long c, int nx, int ny, int nz) {
    const long long sxy = (long long)nx * ny;
    const int i = (int)(c % nx);
    const long long t = c / nx;
    const int j = (int)(t % ny);
    const int k = (int)(t / ny);
    Nb b;
    b.xp = i == nx - 1 ? c - (nx - 1) : c + 1;
    b.xm = i == 0 ? c + (nx - 1) : c - 1;
    b.yp = j == ny - 1 ? c - (long long)(ny - 1) * nx : c + nx;
    b.ym = j == 0 ? c + (long long)(ny - 1) * nx : c - nx;
    b.zp = k == nz - 1 ? c - (long long)(nz - 1) * sxy : c + sxy;
    b.zm = k == 0 ? c + (long long)(nz - 1) * sxy : c - sxy;
    return b;
}

__device__ __forceinline__ double lap7(const double *a, long long c, const Nb &b, double ih2) {
    return (a[b.xp] + a[b.xm] + a[b.yp] + a[b.ym] + a[b.zp] + a[b.zm] - 6.0 * a[c]) * ih2;
}

__device__ __forceinline__ double dcen(const double *a, long long p, long long m, double i2h) {
    return (a[p] - a[m]) * i2h;
}

__device__ __forceinline__ void max_abs(unsigned long long *w, double v) {
    // warp maximum first, then one atomic per warp
    unsigned long long b = __double_as_longlong(fabs(v));
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long q = __shfl_xor_sync(0xffffffffu, b, o);
        b = q > b ? q : b;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(w, b);
}

// Fixed-order block sum; result valid in thread 0.
template <int T>
__device__ __forceinline__ double block_sum(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = T / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------ steps

// Step (a): u~ = u + dt (2 a nu lap u - 2 a grad P - g N(u) - z N_old); N_old <- N(u).
__global__ void __launch_bounds__(kFlThreads) k_fl_predict(int nx, int ny, int nz, double h, double nu, double a,
                                                           double g, double z, double dt, const double *__restrict__ u,
                                                           const double *__restrict__ P, double *__restrict__ nold,
                                                           double *__restrict__ ut) {
    const long long n = (long long)nx * ny * nz;
    const double ih2 = 1.0 / (h * h), i2h = 0.5 / h;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const Nb b = neighbours(c, nx, ny, nz);
        const double uc[3] = {u[c], u[n + c], u[2 * n + c]};
        const double gp[3] = {dcen(P, b.xp, b.xm, i2h), dcen(P, b.yp, b.ym, i2h), dcen(P, b.zp, b.zm, i2h)};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const double *v = u + q * n;
            const double N = uc[0] * dcen(v, b.xp, b.xm, i2h) + uc[1] * dcen(v, b.yp, b.ym, i2h) +
                             uc[2] * dcen(v, b.zp, b.zm, i2h);
            const double L = lap7(v, c, b, ih2);
            const double No = nold[q * n + c];
            ut[q * n + c] = uc[q] + dt * (2.0 * a * nu * L - 2.0 * a * gp[q] - g * N - z * No);
            nold[q * n + c] = N;
        }
    }
}

// Step (e) right-hand side of component q: b = u~_q - 2 a dt mf_q - cv lap u_q + 2 a theta dt d_q P.
__global__ void __launch_bounds__(kFlThreads) k_fl_hrhs(int nx, int ny, int nz, double h, int q, double two_a_dt,
                                                        double cv, double theta, const double *__restrict__ ut,
                                                        const double *__restrict__ u, const double *__restrict__ P,
                                                        const double *__restrict__ mf, double *__restrict__ rhs,
                                                        unsigned long long *maxb) {
    const long long n = (long long)nx * ny * nz;
    const double ih2 = 1.0 / (h * h), i2h = 0.5 / h;
    const double m = mf ? mf[q] : 0.0;
    double bmax = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const Nb b = neighbours(c, nx, ny, nz);
        const double dP = q == 0 ? dcen(P, b.xp, b.xm, i2h) : (q == 1 ? dcen(P, b.yp, b.ym, i2h) : dcen(P, b.zp, b.zm, i2h));
        const double v = ut[q * n + c] - two_a_dt * m - cv * lap7(u + q * n, c, b, ih2) + two_a_dt * theta * dP;
        rhs[c] = v;
        bmax = fmax(bmax, fabs(v));
    }
    max_abs(maxb, bmax);
}

// Step (f) and the Poisson right-hand side of step (g) for the operator -lap:
// u_f*_d = (u*_d + u*_d[+d]) / 2; b = -div u_f* / (2 a dt).  Writes per-block sums of b.
__global__ void __launch_bounds__(kFlThreads) k_fl_prhs(int nx, int ny, int nz, double h, double two_a_dt,
                                                        const double *__restrict__ us, double *__restrict__ uf,
                                                        double *__restrict__ rhs, double *__restrict__ part,
                                                        unsigned long long *maxb) {
    __shared__ double sh[kFlThreads];
    const long long n = (long long)nx * ny * nz;
    const double s = -1.0 / (two_a_dt * h);
    double acc = 0.0, bmax = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const Nb b = neighbours(c, nx, ny, nz);
        const double ux = us[c], uy = us[n + c], uz = us[2 * n + c];
        const double fx = 0.5 * (ux + us[b.xp]), fy = 0.5 * (uy + us[n + b.yp]), fz = 0.5 * (uz + us[2 * n + b.zp]);
        const double gx = 0.5 * (us[b.xm] + ux), gy = 0.5 * (us[n + b.ym] + uy), gz = 0.5 * (us[2 * n + b.zm] + uz);
        uf[c] = fx;
        uf[n + c] = fy;
        uf[2 * n + c] = fz;
        const double v = s * ((fx - gx) + (fy - gy) + (fz - gz));
        rhs[c] = v;
        acc += v;
        bmax = fmax(bmax, fabs(v));
    }
    max_abs(maxb, bmax);
    const double t = block_sum<kFlThreads>(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Per-block sums of a field (for its mean).
__global__ void __launch_bounds__(kFlThreads) k_fl_sum(long long n, const double *__restrict__ a, double *__restrict__ part) {
    __shared__ double sh[kFlThreads];
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        acc += a[c];
    const double t = block_sum<kFlThreads>(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// out = (sum of nparts partials) / n, fixed order.
__global__ void __launch_bounds__(kFlThreads) k_fl_mean_final(int nparts, const double *__restrict__ part, double n,
                                                              double *__restrict__ out) {
    __shared__ double sh[kFlThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nparts; i += kFlThreads) acc += part[i];
    const double t = block_sum<kFlThreads>(acc, sh);
    if (threadIdx.x == 0) *out = t / n;
}

__global__ void k_fl_shift(long long n, double *__restrict__ a, const double *__restrict__ m) {
    const double s = *m;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        a[c] -= s;
}

__global__ void k_fl_negate3(double *v) {
    if (threadIdx.x < 3) v[threadIdx.x] = -v[threadIdx.x];
}

// Steps (h) and (i): u = u* - 2 a dt grad phi, u_f = u_f* - 2 a dt (grad phi)_f,
// P = (1 - theta) P + theta ((phi - m) - a dt nu lap phi), m = mean phi.
__global__ void __launch_bounds__(kFlThreads) k_fl_correct(int nx, int ny, int nz, double h, double two_a_dt,
                                                           double a_dt_nu, double theta, const double *__restrict__ us,
                                                           const double *__restrict__ phi, const double *__restrict__ pm,
                                                           double *__restrict__ u, double *__restrict__ uf,
                                                           double *__restrict__ P) {
    const long long n = (long long)nx * ny * nz;
    const double ih = 1.0 / h, i2h = 0.5 / h, ih2 = 1.0 / (h * h);
    const double m = *pm;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const Nb b = neighbours(c, nx, ny, nz);
        const double p0 = phi[c];
        u[c] = us[c] - two_a_dt * dcen(phi, b.xp, b.xm, i2h);
        u[n + c] = us[n + c] - two_a_dt * dcen(phi, b.yp, b.ym, i2h);
        u[2 * n + c] = us[2 * n + c] - two_a_dt * dcen(phi, b.zp, b.zm, i2h);
        uf[c] -= two_a_dt * (phi[b.xp] - p0) * ih;
        uf[n + c] -= two_a_dt * (phi[b.yp] - p0) * ih;
        uf[2 * n + c] -= two_a_dt * (phi[b.zp] - p0) * ih;
        P[c] = (1.0 - theta) * P[c] + theta * ((p0 - m) - a_dt_nu * lap7(phi, c, b, ih2));
    }
}

// -------------------------------------------------------------- multigrid
// Operator of every level: A x = a0 x - beta (sum of the 6 neighbours - 6 x),
// beta = bcoef / h_l^2.  bs: NULL or a device scalar subtracted from b (the
// mean of the level-0 Poisson right-hand side).

// Red-black Gauss-Seidel half sweep: the cells with (i + j + k) % 2 == color.
__global__ void __launch_bounds__(kFlThreads) k_mg_smooth(int nx, int ny, int nz, double a0, double beta, int color,
                                                          double *__restrict__ x, const double *__restrict__ b,
                                                          const double *__restrict__ bs) {
    const int hx = nx >> 1;
    const long long nh = (long long)hx * ny * nz;
    const double inv = 1.0 / (a0 + 6.0 * beta);
    const double s = bs ? *bs : 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nh; t += (long long)gridDim.x * blockDim.x) {
        const int i2 = (int)(t % hx);
        const long long r = t / hx;
        const int j = (int)(r % ny);
        const int k = (int)(r / ny);
        const int i = 2 * i2 + ((j + k + color) & 1);
        const long long c = r * nx + i;
        const Nb nb = neighbours(c, nx, ny, nz);
        const double sum = x[nb.xp] + x[nb.xm] + x[nb.yp] + x[nb.ym] + x[nb.zp] + x[nb.zm];
        x[c] = (b[c] - s + beta * sum) * inv;
    }
}

// Coarse right-hand side: the fine residual averaged over the 8 children of
// each coarse cell; the maximum |r| of the fine level into *maxr.
__global__ void __launch_bounds__(kFlThreads) k_mg_restrict(int nx, int ny, int nz, double a0, double beta,
                                                            const double *__restrict__ x, const double *__restrict__ b,
                                                            const double *__restrict__ bs, double *__restrict__ bc,
                                                            unsigned long long *maxr) {
    const int cx = nx >> 1, cy = ny >> 1, cz = nz >> 1;
    const long long nc = (long long)cx * cy * cz;
    const double s = bs ? *bs : 0.0;
    double rmax = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nc; t += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(t % cx);
        const long long q = t / cx;
        const int J = (int)(q % cy);
        const int K = (int)(q / cy);
        double acc = 0.0;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const long long c = ((long long)(2 * K + (d >> 2)) * ny + (2 * J + ((d >> 1) & 1))) * nx + 2 * I + (d & 1);
            const Nb nb = neighbours(c, nx, ny, nz);
            const double xc = x[c];
            const double r = (b[c] - s) - (a0 + 6.0 * beta) * xc +
                             beta * (x[nb.xp] + x[nb.xm] + x[nb.yp] + x[nb.ym] + x[nb.zp] + x[nb.zm]);
            acc += r;
            rmax = fmax(rmax, fabs(r));
        }
        bc[t] = 0.125 * acc;
    }
    max_abs(maxr, rmax);
}

// Fine x += trilinear interpolation of the coarse correction (weights 3/4 and
// 1/4 per axis from the two nearest coarse cells, periodic).
__global__ void __launch_bounds__(kFlThreads) k_mg_prolong(int nx, int ny, int nz, const double *__restrict__ xc,
                                                           double *__restrict__ x) {
    const int cx = nx >> 1, cy = ny >> 1, cz = nz >> 1;
    const long long n = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % nx);
        const long long t = c / nx;
        const int j = (int)(t % ny);
        const int k = (int)(t / ny);
        const int I0 = i >> 1, J0 = j >> 1, K0 = k >> 1;
        const int I1 = (i & 1) ? (I0 + 1 == cx ? 0 : I0 + 1) : (I0 == 0 ? cx - 1 : I0 - 1);
        const int J1 = (j & 1) ? (J0 + 1 == cy ? 0 : J0 + 1) : (J0 == 0 ? cy - 1 : J0 - 1);
        const int K1 = (k & 1) ? (K0 + 1 == cz ? 0 : K0 + 1) : (K0 == 0 ? cz - 1 : K0 - 1);
        const long long r00 = ((long long)K0 * cy + J0) * cx, r01 = ((long long)K0 * cy + J1) * cx;
        const long long r10 = ((long long)K1 * cy + J0) * cx, r11 = ((long long)K1 * cy + J1) * cx;
        const double e = 0.421875 * xc[r00 + I0] +
                         0.140625 * (xc[r00 + I1] + xc[r01 + I0] + xc[r10 + I0]) +
                         0.046875 * (xc[r01 + I1] + xc[r10 + I1] + xc[r11 + I0]) + 0.015625 * xc[r11 + I1];
        x[c] += e;
    }
}

// Maximum |b - A x| over a level.
__global__ void __launch_bounds__(kFlThreads) k_mg_resid(int nx, int ny, int nz, double a0, double beta,
                                                         const double *__restrict__ x, const double *__restrict__ b,
                                                         const double *__restrict__ bs, unsigned long long *maxr) {
    const long long n = (long long)nx * ny * nz;
    const double s = bs ? *bs : 0.0;
    double rmax = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const Nb nb = neighbours(c, nx, ny, nz);
        const double r = (b[c] - s) - (a0 + 6.0 * beta) * x[c] +
                         beta * (x[nb.xp] + x[nb.xm] + x[nb.yp] + x[nb.ym] + x[nb.zp] + x[nb.zm]);
        rmax = fmax(rmax, fabs(r));
    }
    max_abs(maxr, rmax);
}

// Coarsest level: conjugate gradients in one CTA (n <= kCoarseMax) from the
// initial guess in x.  For the singular Poisson operator (a0 = 0) the
// right-hand side is made mean-free first and x is returned mean-free.  Stops
// at |r|_2 <= 1e-14 |r0|_2 or after maxit iterations.
__global__ void __launch_bounds__(kCgThreads) k_mg_cg(int nx, int ny, int nz, double a0, double beta,
                                                      double *__restrict__ x, const double *__restrict__ b,
                                                      double *__restrict__ r, double *__restrict__ p,
                                                      double *__restrict__ q, int maxit) {
    __shared__ double sh[kCgThreads];
    const long long n = (long long)nx * ny * nz;
    const bool singular = a0 == 0.0;
    double acc = 0.0;
    for (long long c = threadIdx.x; c < n; c += kCgThreads) acc += b[c];
    const double mb = singular ? block_sum<kCgThreads>(acc, sh) / (double)n : 0.0;
    acc = 0.0;
    for (long long c = threadIdx.x; c < n; c += kCgThreads) {
        const Nb nb = neighbours(c, nx, ny, nz);
        const double v = (b[c] - mb) - ((a0 + 6.0 * beta) * x[c] -
                                        beta * (x[nb.xp] + x[nb.xm] + x[nb.yp] + x[nb.ym] + x[nb.zp] + x[nb.zm]));
        r[c] = v;
        p[c] = v;
        acc += v * v;
    }
    double rr = block_sum<kCgThreads>(acc, sh);
    const double stop = 1e-28 * rr;
    for (int it = 0; it < maxit && rr > stop; ++it) {
        acc = 0.0;
        for (long long c = threadIdx.x; c < n; c += kCgThreads) {
            const Nb nb = neighbours(c, nx, ny, nz);
            const double v = (a0 + 6.0 * beta) * p[c] - beta * (p[nb.xp] + p[nb.xm] + p[nb.yp] + p[nb.ym] + p[nb.zp] + p[nb.zm]);
            q[c] = v;
            acc += p[c] * v;
        }
        const double pq = block_sum<kCgThreads>(acc, sh);
        if (!(pq > 0.0)) break;
        const double al = rr / pq;
        acc = 0.0;
        for (long long c = threadIdx.x; c < n; c += kCgThreads) {
            x[c] += al * p[c];
            const double v = r[c] - al * q[c];
            r[c] = v;
            acc += v * v;
        }
        const double rn = block_sum<kCgThreads>(acc, sh);
        const double be = rn / rr;
        rr = rn;
        for (long long c = threadIdx.x; c < n; c += kCgThreads) p[c] = r[c] + be * p[c];
        __syncthreads();
    }
    if (singular) {
        acc = 0.0;
        for (long long c = threadIdx.x; c < n; c += kCgThreads) acc += x[c];
        const double mx = block_sum<kCgThreads>(acc, sh) / (double)n;
        for (long long c = threadIdx.x; c < n; c += kCgThreads) x[c] -= mx;
    }
}

void vcycle(ibm_fluid *fl, size_t l, double a0, double bcoef, double *x0, const double *bs0) {
    ibm_fluid::Level &L = fl->lv[l];
    double *x = l == 0 ? x0 : L.x;
    const double *bs = l == 0 ? bs0 : nullptr;
    const double beta = bcoef / (L.h * L.h);
    cudaStream_t sm = fl->stream;
    if (l + 1 == fl->lv.size()) {
        double *r = fl->cg, *p = fl->cg + L.cells, *q = fl->cg + 2 * L.cells;
        // (a shift bs of b is a constant, which the singular solve removes anyway)
        k_mg_cg<<<1, kCgThreads, 0, sm>>>(L.n[0], L.n[1], L.n[2], a0, beta, x, L.b, r, p, q,
                                          (int)std::min(4 * L.cells + 16, 4000ll));
        return;
    }
    const int gs = grid_cells(L.cells / 2);
    for (int s = 0; s < 2; ++s)
        for (int color = 0; color < 2; ++color)
            k_mg_smooth<<<gs, kFlThreads, 0, sm>>>(L.n[0], L.n[1], L.n[2], a0, beta, color, x, L.b, bs);
    ibm_fluid::Level &C = fl->lv[l + 1];
    k_mg_restrict<<<grid_cells(C.cells), kFlThreads, 0, sm>>>(L.n[0], L.n[1], L.n[2], a0, beta, x, L.b, bs, C.b,
                                                              l == 0 ? fl->maxw + 1 : fl->maxw + 2);
    cudaMemsetAsync(C.x, 0, C.cells * sizeof(double), sm);
    vcycle(fl, l + 1, a0, bcoef, x0, bs0);
    k_mg_prolong<<<grid_cells(L.cells), kFlThreads, 0, sm>>>(L.n[0], L.n[1], L.n[2], C.x, x);
    for (int s = 0; s < 2; ++s)
        for (int color = 0; color < 2; ++color)
            k_mg_smooth<<<gs, kFlThreads, 0, sm>>>(L.n[0], L.n[1], L.n[2], a0, beta, color, x, L.b, bs);
}

double bits_to_double(unsigned long long b) {
    double d;
    std::memcpy(&d, &b, sizeof d);
    return d;
}

// Solve A x = rhs on level 0 (x holds the initial guess); fl->maxw[0] holds
// max|rhs| (written by the right-hand-side kernel).  bs: device mean of rhs or NULL.
ibm_status mg_solve(ibm_fluid *fl, double a0, double bcoef, double *x, const double *bs, int slot) {
    cudaStream_t sm = fl->stream;
    ibm_fluid::Level &L = fl->lv[0];
    const double beta = bcoef / (L.h * L.h);
    FK(cudaMemcpyAsync(fl->hmax, fl->maxw, sizeof(unsigned long long), cudaMemcpyDeviceToHost, sm), "read norm");
    FK(cudaStreamSynchronize(sm), "synchronise");
    const double bmax = bits_to_double(fl->hmax[0]);
    fl->cycles[slot] = 0;
    fl->resid[slot] = 0.0;
    if (!std::isfinite(bmax)) return fl_fail(fl, IBM_ERR_NONFINITE, "non-finite right-hand side of a fluid solve");
    if (bmax == 0.0) {
        FK(cudaMemsetAsync(x, 0, L.cells * sizeof(double), sm), "zero solution");
        return IBM_OK;
    }
    const double tol = fl->cfg.rtol * bmax;
    const bool coarse_only = fl->lv.size() == 1;
    int cyc = 0;
    double r = 0.0;
    for (cyc = 1; cyc <= fl->cfg.max_cycles; ++cyc) {
        FK(cudaMemsetAsync(fl->maxw + 1, 0, 2 * sizeof(unsigned long long), sm), "zero norm");
        vcycle(fl, 0, a0, bcoef, x, bs);
        // multigrid: the residual after this cycle's pre-smoothing (once within tol, the cycle has finished
        // the solve); a lone coarsest level: the residual after the conjugate-gradient pass
        if (coarse_only)
            k_mg_resid<<<grid_cells(L.cells), kFlThreads, 0, sm>>>(L.n[0], L.n[1], L.n[2], a0, beta, x, L.b, bs,
                                                                   fl->maxw + 1);
        FK(cudaGetLastError(), "multigrid launch");
        FK(cudaMemcpyAsync(fl->hmax + 1, fl->maxw + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost, sm),
           "read norm");
        FK(cudaStreamSynchronize(sm), "synchronise");
        r = bits_to_double(fl->hmax[1]);
        if (!std::isfinite(r)) return fl_fail(fl, IBM_ERR_NONFINITE, "non-finite residual in a fluid solve");
        if (r <= tol) break;
    }
    // final residual
    if (!coarse_only) {
        FK(cudaMemsetAsync(fl->maxw + 1, 0, sizeof(unsigned long long), sm), "zero norm");
        k_mg_resid<<<grid_cells(L.cells), kFlThreads, 0, sm>>>(L.n[0], L.n[1], L.n[2], a0, beta, x, L.b, bs,
                                                               fl->maxw + 1);
        FK(cudaMemcpyAsync(fl->hmax + 1, fl->maxw + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost, sm),
           "read norm");
        FK(cudaStreamSynchronize(sm), "synchronise");
        r = bits_to_double(fl->hmax[1]);
    }
    fl->cycles[slot] = std::min(cyc, fl->cfg.max_cycles);
    fl->resid[slot] = r / bmax;
    if (!(r <= tol))
        return fl_fail(fl, IBM_ERR_NOCONVERGE,
                       "fluid solve " + std::to_string(slot) + " stopped at relative residual " +
                           std::to_string(r / bmax) + " after " + std::to_string(fl->cycles[slot]) + " V-cycles");
    return IBM_OK;
}

void free_all(ibm_fluid *fl) {
    double *bufs[] = {fl->nold, fl->rhs, fl->f, fl->red, fl->mean, fl->cg};
    for (double *b : bufs)
        if (b) cudaFree(b);
    if (fl->maxw) cudaFree(fl->maxw);
    for (size_t l = 1; l < fl->lv.size(); ++l) {
        if (fl->lv[l].x) cudaFree(fl->lv[l].x);
        if (fl->lv[l].b) cudaFree(fl->lv[l].b);
    }
    if (fl->hmax) cudaFreeHost(fl->hmax);
    for (cudaEvent_t e : fl->ev)
        if (e) cudaEventDestroy(e);
}

bool check_fields(const ibm_fluid_fields *F) { return F && F->u && F->ut && F->uf && F->p && F->phi; }

}  // namespace

extern "C" {

ibm_status ibm_fluid_create(const ibm_fluid_config *cfg, void *cuda_stream, ibm_fluid **out) {
    if (!out) return IBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfg || cfg->nx < 2 || cfg->ny < 2 || cfg->nz < 2) return IBM_ERR_INVALID_ARG;
    if (!(cfg->h > 0.0) || !std::isfinite(cfg->h) || !(cfg->nu >= 0.0) || !std::isfinite(cfg->nu))
        return IBM_ERR_INVALID_ARG;
    if (!(cfg->theta >= 0.0 && cfg->theta <= 1.0) || cfg->rtol < 0.0 || cfg->max_cycles < 0) return IBM_ERR_INVALID_ARG;
    const long long cells = (long long)cfg->nx * cfg->ny * cfg->nz;
    if (cells > (1ll << 31) / 3) return IBM_ERR_INVALID_ARG;
    ibm_fluid *fl = new (std::nothrow) ibm_fluid;
    if (!fl) return IBM_ERR_OOM;
    fl->cfg = *cfg;
    if (fl->cfg.rtol == 0.0) fl->cfg.rtol = 1e-12;
    if (fl->cfg.max_cycles == 0) fl->cfg.max_cycles = 60;
    fl->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    fl->n[0] = cfg->nx;
    fl->n[1] = cfg->ny;
    fl->n[2] = cfg->nz;
    fl->cells = cells;
    // levels: halve while every extent is even and at least 4
    ibm_fluid::Level L0{{cfg->nx, cfg->ny, cfg->nz}, cells, cfg->h, nullptr, nullptr};
    fl->lv.push_back(L0);
    while (true) {
        const ibm_fluid::Level &p = fl->lv.back();
        if (p.n[0] % 2 || p.n[1] % 2 || p.n[2] % 2 || p.n[0] < 4 || p.n[1] < 4 || p.n[2] < 4) break;
        ibm_fluid::Level c{{p.n[0] / 2, p.n[1] / 2, p.n[2] / 2}, p.cells / 8, p.h * 2.0, nullptr, nullptr};
        fl->lv.push_back(c);
    }
    if (fl->lv.back().cells > kCoarseMax) {
        delete fl;
        return IBM_ERR_INVALID_ARG;
    }
    auto fail = [&](cudaError_t e) {
        free_all(fl);
        delete fl;
        return e == cudaErrorMemoryAllocation ? IBM_ERR_OOM : IBM_ERR_CUDA;
    };
    cudaError_t e;
    if ((e = ibm_malloc(&fl->nold, 3 * cells * sizeof(double))) != cudaSuccess) return fail(e);
    if ((e = ibm_malloc(&fl->rhs, cells * sizeof(double))) != cudaSuccess) return fail(e);
    if ((e = ibm_malloc(&fl->red, (kRedBlocks + 8) * sizeof(double))) != cudaSuccess) return fail(e);
    if ((e = ibm_malloc(&fl->mean, 8 * sizeof(double))) != cudaSuccess) return fail(e);
    if ((e = ibm_malloc(&fl->maxw, 4 * sizeof(unsigned long long))) != cudaSuccess) return fail(e);
    if ((e = ibm_malloc(&fl->cg, 3 * fl->lv.back().cells * sizeof(double))) != cudaSuccess) return fail(e);
    fl->lv[0].b = fl->rhs;
    for (size_t l = 1; l < fl->lv.size(); ++l) {
        if ((e = ibm_malloc(&fl->lv[l].x, fl->lv[l].cells * sizeof(double))) != cudaSuccess) return fail(e);
        if ((e = ibm_malloc(&fl->lv[l].b, fl->lv[l].cells * sizeof(double))) != cudaSuccess) return fail(e);
    }
    if ((e = cudaMallocHost(&fl->hmax, 4 * sizeof(unsigned long long))) != cudaSuccess) return fail(e);
    for (cudaEvent_t &ev : fl->ev)
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
    if ((e = cudaMemsetAsync(fl->nold, 0, 3 * cells * sizeof(double), fl->stream)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamSynchronize(fl->stream)) != cudaSuccess) return fail(e);
    *out = fl;
    return IBM_OK;
}

ibm_status ibm_fluid_destroy(ibm_fluid *fl) {
    if (!fl) return IBM_ERR_INVALID_ARG;
    cudaStreamSynchronize(fl->stream);
    free_all(fl);
    delete fl;
    return IBM_OK;
}

ibm_status ibm_fluid_predict(ibm_fluid *fl, int k, double dt, const ibm_fluid_fields *F) {
    if (!fl) return IBM_ERR_INVALID_ARG;
    fl->last_error.clear();
    if (k < 0 || k > 2) return fl_fail(fl, IBM_ERR_INVALID_ARG, "stage k must be 0, 1 or 2");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fl_fail(fl, IBM_ERR_INVALID_ARG, "dt must be > 0");
    if (!check_fields(F)) return fl_fail(fl, IBM_ERR_INVALID_ARG, "NULL field pointer");
    k_fl_predict<<<grid_cells(fl->cells), kFlThreads, 0, fl->stream>>>(
        fl->n[0], fl->n[1], fl->n[2], fl->cfg.h, fl->cfg.nu, kAlpha[k], kGamma[k], kZeta[k], dt, F->u, F->p,
        fl->nold, F->ut);
    FK(cudaGetLastError(), "predictor launch");
    return IBM_OK;
}

ibm_status ibm_fluid_correct(ibm_fluid *fl, int k, double dt, const ibm_fluid_fields *F, const double *mean_f,
                             int on_device) {
    if (!fl) return IBM_ERR_INVALID_ARG;
    fl->last_error.clear();
    if (k < 0 || k > 2) return fl_fail(fl, IBM_ERR_INVALID_ARG, "stage k must be 0, 1 or 2");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fl_fail(fl, IBM_ERR_INVALID_ARG, "dt must be > 0");
    if (!check_fields(F)) return fl_fail(fl, IBM_ERR_INVALID_ARG, "NULL field pointer");
    cudaStream_t sm = fl->stream;
    const long long n = fl->cells;
    const double a = kAlpha[k];
    const double two_a_dt = 2.0 * a * dt, cv = a * dt * fl->cfg.nu;
    const double *mf = nullptr;
    if (mean_f) {
        if (on_device) {
            mf = mean_f;
        } else {
            FK(cudaMemcpyAsync(fl->mean, mean_f, 3 * sizeof(double), cudaMemcpyHostToDevice, sm), "copy mean force");
            FK(cudaStreamSynchronize(sm), "synchronise");
            mf = fl->mean;
        }
    }
    const int g = grid_cells(n);
    // (e) three Helmholtz solves, each in place in ut (initial guess u~_q)
    for (int q = 0; q < 3; ++q) {
        FK(cudaMemsetAsync(fl->maxw, 0, sizeof(unsigned long long), sm), "zero norm");
        k_fl_hrhs<<<g, kFlThreads, 0, sm>>>(fl->n[0], fl->n[1], fl->n[2], fl->cfg.h, q, two_a_dt, cv, fl->cfg.theta,
                                             F->ut, F->u, F->p, mf, fl->rhs, fl->maxw);
        FK(cudaGetLastError(), "right-hand side launch");
        ibm_status st = mg_solve(fl, 1.0, cv, F->ut + q * n, nullptr, q);
        if (st != IBM_OK) return st;
    }
    // (f), (g)
    FK(cudaMemsetAsync(fl->maxw, 0, sizeof(unsigned long long), sm), "zero norm");
    k_fl_prhs<<<kRedBlocks, kFlThreads, 0, sm>>>(fl->n[0], fl->n[1], fl->n[2], fl->cfg.h, two_a_dt, F->ut, F->uf,
                                                 fl->rhs, fl->red, fl->maxw);
    k_fl_mean_final<<<1, kFlThreads, 0, sm>>>(kRedBlocks, fl->red, (double)n, fl->mean + 3);
    FK(cudaGetLastError(), "Poisson right-hand side launch");
    ibm_status st = mg_solve(fl, 0.0, 1.0, F->phi, fl->mean + 3, 3);
    if (st != IBM_OK) return st;
    // mean of phi, then (h), (i), and phi made mean-free
    k_fl_sum<<<kRedBlocks, kFlThreads, 0, sm>>>(n, F->phi, fl->red);
    k_fl_mean_final<<<1, kFlThreads, 0, sm>>>(kRedBlocks, fl->red, (double)n, fl->mean + 4);
    k_fl_correct<<<g, kFlThreads, 0, sm>>>(fl->n[0], fl->n[1], fl->n[2], fl->cfg.h, two_a_dt, a * dt * fl->cfg.nu,
                                           fl->cfg.theta, F->ut, F->phi, fl->mean + 4, F->u, F->uf, F->p);
    k_fl_shift<<<g, kFlThreads, 0, sm>>>(n, F->phi, fl->mean + 4);
    FK(cudaGetLastError(), "corrector launch");
    return IBM_OK;
}

ibm_status ibm_fluid_stage(ibm_fluid *fl, ibm_ctx *ctx, int k, double dt, const ibm_fluid_fields *F,
                           double *f_out) {
    if (!fl) return IBM_ERR_INVALID_ARG;
    ibm_status st = ibm_fluid_predict(fl, k, dt, F);
    if (st != IBM_OK) return st;
    if (!ctx || ctx->n_p == 0) return ibm_fluid_correct(fl, k, dt, F, nullptr, 0);
    const ibm_config &c = ctx->cfg;
    if (c.precision != IBM_FP64 || c.n_scenes != 1 || c.dims[0] != fl->n[0] || c.dims[1] != fl->n[1] ||
        c.dims[2] != fl->n[2] || c.h != fl->cfg.h)
        return fl_fail(fl, IBM_ERR_INVALID_ARG, "the IBM context must be FP64 with one scene of the fluid's grid");
    double *f = f_out;
    if (!f) {
        if (!fl->f) FK(ibm_malloc(&fl->f, 3 * fl->cells * sizeof(double)), "allocate f_IBM");
        f = fl->f;
    }
    // order ctx's stream after fl's, run the forcing loop and the mean force there, and come back
    FK(cudaEventRecord(fl->ev[0], fl->stream), "record event");
    FK(cudaStreamWaitEvent(ctx->stream, fl->ev[0], 0), "wait event");
    void *up[1] = {F->ut};
    void *fp[1] = {f};
    st = ibm_forcing_step(ctx, up, 2.0 * kAlpha[k] * dt, fp, nullptr);
    if (st == IBM_OK) st = ibm_mean_force(ctx, fp, fl->mean, 1);
    if (st != IBM_OK) return fl_fail(fl, st, std::string("IBM forcing: ") + ibm_last_error(ctx));
    // the grid pass returns -mean(f) (Eq. fe_IBM); the correction subtracts mean(f)
    FK(cudaEventRecord(fl->ev[1], ctx->stream), "record event");
    FK(cudaStreamWaitEvent(fl->stream, fl->ev[1], 0), "wait event");
    k_fl_negate3<<<1, 32, 0, fl->stream>>>(fl->mean);
    FK(cudaGetLastError(), "negate launch");
    return ibm_fluid_correct(fl, k, dt, F, fl->mean, 1);
}

ibm_status ibm_fluid_stats(ibm_fluid *fl, int64_t *cycles, double *resid, int *levels) {
    if (!fl) return IBM_ERR_INVALID_ARG;
    for (int i = 0; i < 4; ++i) {
        if (cycles) cycles[i] = fl->cycles[i];
        if (resid) resid[i] = fl->resid[i];
    }
    if (levels) *levels = (int)fl->lv.size();
    return IBM_OK;
}

const char *ibm_fluid_last_error(const ibm_fluid *fl) { return fl ? fl->last_error.c_str() : ""; }

}  // extern "C"
