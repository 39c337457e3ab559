// Collocated fractional-step fluid solver of the modified method (Sec. 2.2.1
// "Pressure-momentum coupling on a collocated grid"; Sec. 2.2.4, the steps
// (a)-(i) of Eq. fluid-solver) on one triply periodic grid.  The state
// and every result are FP64; the multigrid corrections inside the solves are
// FP32 (see the multigrid section).
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
//   solves         iterative refinement: k_mg_resid64 (FP64 residual, max
//                  norm, FP32 copy) and k_mg_update64 around one FP32
//                  V-cycle: k_mg_rbgs (one-pass red-black Gauss-Seidel sweep;
//                  k_mg_smooth, two half sweeps, on narrow levels),
//                  k_mg_restrict (residual averaged over the 8 children),
//                  k_mg_prolong (trilinear correction), k_mg_cg (one-CTA
//                  conjugate gradients on the coarsest level)
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
    double *rhs = nullptr;      // right-hand side of the FP64 solve
    double *f = nullptr;        // [3][cells] f_IBM of ibm_fluid_stage (lazy)
    double *red = nullptr;      // one partial sum per block of the level-0 3-D launch
    unsigned long long *maxw = nullptr;  // [2]: max|b|, max|r|
    double *mean = nullptr;     // [4]: mean_f[3] (host input copy), mean of a field
    unsigned long long *hmax = nullptr;  // pinned [2]
    struct Level {
        int n[3];
        long long cells;
        double h;
        float *x, *b;           // FP32 correction and its right-hand side (level 0: the scaled FP64 residual)
        float *x2;              // the other buffer of the fused sweeps
        bool fused;             // smoothed by k_mg_rbgs (else two k_mg_smooth half sweeps)
    };
    std::vector<Level> lv;
    float *cg = nullptr;        // r, p, q of the coarsest level
    cudaEvent_t ev[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> prof;   // pairs around finest-level smoothing launches (cfg.profile)
    size_t prof_used = 0;
    int64_t cycles[4] = {0, 0, 0, 0};
    double resid[4] = {0, 0, 0, 0};
    std::string last_error;
};

namespace {

constexpr int kFlThreads = 256;
constexpr int kCgThreads = 1024;
constexpr long long kCoarseMax = 32768;

// RK3 coefficients of the Rai and Moin scheme that Sec. 2.1 names (their published values)
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

// 3-D launch over an nx x ny x nz box: (32, 8) threads per block, x fastest;
// blocks along z loop over the planes k = blockIdx.z, + gridDim.z, ...
constexpr int kBx = 32, kBy = 8, kZBlocks = 64;
dim3 grid3(int nx, int ny, int nz) { return dim3((nx + kBx - 1) / kBx, (ny + kBy - 1) / kBy, std::min(nz, kZBlocks)); }
const dim3 kBlock3(kBx, kBy);

__device__ __forceinline__ int tid() { return threadIdx.y * blockDim.x + threadIdx.x; }

// The six periodic neighbours of cell (i, j, k) = linear index c.
struct Nb {
    long long xp, xm, yp, ym, zp, zm;
};

__device__ __forceinline__ Nb neighbours(long long c, int i, int j, int k, int nx, int ny, int nz) {
    const long long sxy = (long long)nx * ny;
    Nb b;
    b.xp = i == nx - 1 ? c - (nx - 1) : c + 1;
    b.xm = i == 0 ? c + (nx - 1) : c - 1;
    b.yp = j == ny - 1 ? c - (long long)(ny - 1) * nx : c + nx;
    b.ym = j == 0 ? c + (long long)(ny - 1) * nx : c - nx;
    b.zp = k == nz - 1 ? c - (long long)(nz - 1) * sxy : c + sxy;
    b.zm = k == 0 ? c + (long long)(nz - 1) * sxy : c - sxy;
    return b;
}

// Same from the linear index alone (32-bit division; small grids only).
__device__ __forceinline__ Nb neighbours_lin(int c, int nx, int ny, int nz) {
    const int i = c % nx, t = c / nx;
    return neighbours(c, i, t % ny, t / ny, nx, ny, nz);
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
    if ((tid() & 31) == 0) atomicMax(w, b);
}

// Fixed-order block sum over T threads; the result is returned to every thread.
template <int T>
__device__ __forceinline__ double block_sum(double v, double *sh) {
    const int t = tid();
    sh[t] = v;
    __syncthreads();
    for (int s = T / 2; s > 0; s >>= 1) {
        if (t < s) sh[t] += sh[t + s];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

#define FOR_CELLS(nx, ny, nz)                                                   \
    const int i = blockIdx.x * kBx + threadIdx.x;                               \
    const int j = blockIdx.y * kBy + threadIdx.y;                               \
    const bool active = i < nx && j < ny;                                       \
    for (int k = blockIdx.z; k < nz; k += gridDim.z)                            \
        if (active)

// ------------------------------------------------------------------ steps

// Step (a): u~ = u + dt (2 a nu lap u - 2 a grad P - g N(u) - z N_old); N_old <- N(u).
__global__ void __launch_bounds__(kFlThreads) k_fl_predict(int nx, int ny, int nz, double h, double nu, double a,
                                                           double g, double z, double dt, const double *__restrict__ u,
                                                           const double *__restrict__ P, double *__restrict__ nold,
                                                           double *__restrict__ ut) {
    const long long n = (long long)nx * ny * nz;
    const double ih2 = 1.0 / (h * h), i2h = 0.5 / h;
    FOR_CELLS(nx, ny, nz) {
        const long long c = ((long long)k * ny + j) * nx + i;
        const Nb b = neighbours(c, i, j, k, nx, ny, nz);
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
    FOR_CELLS(nx, ny, nz) {
        const long long c = ((long long)k * ny + j) * nx + i;
        const Nb b = neighbours(c, i, j, k, nx, ny, nz);
        const double dP = q == 0 ? dcen(P, b.xp, b.xm, i2h) : (q == 1 ? dcen(P, b.yp, b.ym, i2h) : dcen(P, b.zp, b.zm, i2h));
        const double v = ut[q * n + c] - two_a_dt * m - cv * lap7(u + q * n, c, b, ih2) + two_a_dt * theta * dP;
        rhs[c] = v;
        bmax = fmax(bmax, fabs(v));
    }
    max_abs(maxb, bmax);
}

// Step (f) and the Poisson right-hand side of step (g) for the operator -lap:
// u_f*_d = (u*_d + u*_d[+d]) / 2; b = -div u_f* / (2 a dt).  Writes one partial sum of b per block.
__global__ void __launch_bounds__(kFlThreads) k_fl_prhs(int nx, int ny, int nz, double h, double two_a_dt,
                                                        const double *__restrict__ us, double *__restrict__ uf,
                                                        double *__restrict__ rhs, double *__restrict__ part,
                                                        unsigned long long *maxb) {
    __shared__ double sh[kFlThreads];
    const long long n = (long long)nx * ny * nz;
    const double s = -1.0 / (two_a_dt * h);
    double acc = 0.0, bmax = 0.0;
    FOR_CELLS(nx, ny, nz) {
        const long long c = ((long long)k * ny + j) * nx + i;
        const Nb b = neighbours(c, i, j, k, nx, ny, nz);
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
    if (tid() == 0) part[((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
}

// One partial sum of a field per block (same blocks as grid3).
__global__ void __launch_bounds__(kFlThreads) k_fl_sum(int nx, int ny, int nz, const double *__restrict__ a,
                                                       double *__restrict__ part) {
    __shared__ double sh[kFlThreads];
    double acc = 0.0;
    FOR_CELLS(nx, ny, nz) acc += a[((long long)k * ny + j) * nx + i];
    const double t = block_sum<kFlThreads>(acc, sh);
    if (tid() == 0) part[((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
}

// out = (sum of nparts partials) / n, fixed order.
__global__ void __launch_bounds__(kFlThreads) k_fl_mean_final(long long nparts, const double *__restrict__ part,
                                                              double n, double *__restrict__ out) {
    __shared__ double sh[kFlThreads];
    double acc = 0.0;
    for (long long i = threadIdx.x; i < nparts; i += kFlThreads) acc += part[i];
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
    FOR_CELLS(nx, ny, nz) {
        const long long c = ((long long)k * ny + j) * nx + i;
        const Nb b = neighbours(c, i, j, k, nx, ny, nz);
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
// Each solve A x = b (level 0 in FP64) is an iterative refinement: the FP64
// residual r = b - A x of the current x, one FP32 multigrid V-cycle for the
// correction A e = r, x += e.  The FP64 residual fixes the accuracy (the
// stopping test is on it); the V-cycle only has to reduce the error by its
// usual factor, which FP32 does as well as FP64.  On this GPU FP64 arithmetic
// runs at a small fraction of the FP32 rate, so the smoothing sweeps, the
// restrictions and prolongations (most of the work) run in FP32.
// Operator of every level: A x = a0 x - beta (sum of the 6 neighbours - 6 x),
// beta = bcoef / h_l^2.

// r = ((b - bs) - A x) * rscale in FP32 (level 0); max |b - bs - A x| into *maxr.
__global__ void __launch_bounds__(kFlThreads) k_mg_resid64(int nx, int ny, int nz, double a0, double beta,
                                                           const double *__restrict__ x, const double *__restrict__ b,
                                                           const double *__restrict__ bs, double rscale,
                                                           float *__restrict__ r32, unsigned long long *maxr) {
    const double s = bs ? *bs : 0.0;
    double rmax = 0.0;
    FOR_CELLS(nx, ny, nz) {
        const long long c = ((long long)k * ny + j) * nx + i;
        const Nb nb = neighbours(c, i, j, k, nx, ny, nz);
        const double r = (b[c] - s) - (a0 + 6.0 * beta) * x[c] +
                         beta * (x[nb.xp] + x[nb.xm] + x[nb.yp] + x[nb.ym] + x[nb.zp] + x[nb.zm]);
        r32[c] = (float)(r * rscale);
        rmax = fmax(rmax, fabs(r));
    }
    max_abs(maxr, rmax);
}

// x += escale * e (level 0, FP64 += FP32 correction).
__global__ void k_mg_update64(long long n, double *__restrict__ x, const float *__restrict__ e, double escale) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        x[c] += escale * (double)e[c];
}

// Red-black Gauss-Seidel half sweep: the cells with (i + j + k) % 2 == color
// (nx even; thread i2 of a row takes cell 2 i2 or 2 i2 + 1).
template <typename T>
__global__ void __launch_bounds__(kFlThreads) k_mg_smooth(int nx, int ny, int nz, T a0, T beta, int color,
                                                          T *__restrict__ x, const T *__restrict__ b) {
    const int hx = nx >> 1;
    const T inv = T(1) / (a0 + T(6) * beta);
    const int i2 = blockIdx.x * kBx + threadIdx.x;
    const int j = blockIdx.y * kBy + threadIdx.y;
    if (i2 >= hx || j >= ny) return;
    for (int k = blockIdx.z; k < nz; k += gridDim.z) {
        const int i = 2 * i2 + ((j + k + color) & 1);
        const long long c = ((long long)k * ny + j) * nx + i;
        const Nb nb = neighbours(c, i, j, k, nx, ny, nz);
        const T sum = x[nb.xp] + x[nb.xm] + x[nb.yp] + x[nb.ym] + x[nb.zp] + x[nb.zm];
        x[c] = (b[c] + beta * sum) * inv;
    }
}

// One whole red-black Gauss-Seidel sweep (red half sweep, then black) in one
// pass, from xin to xout, bit for bit the two half sweeps of k_mg_smooth.
// A block owns a 32 x 8 tile of each plane of a chunk of kZc planes and marches
// up through it.  It stages planes of xin over the tile plus a ring of 2 cells
// (4 planes in flight) and b over the same region (2 planes), updates the red
// cells of the tile plus a ring of 1 (the red neighbours of the tile's black
// cells) from old black values, then the tile's black cells from those red
// values, and writes the tile.  Every block reads old values only (xin is
// never written during the sweep), so the result does not depend on the
// order in which blocks run.  Dimensions are even (levels that are smoothed).
constexpr int kRx = kBx + 4, kRy = kBy + 4, kRegion = kRx * kRy, kZc = 32;
template <typename T>
__global__ void __launch_bounds__(kFlThreads) k_mg_rbgs(int nx, int ny, int nz, T a0, T beta,
                                                        const T *__restrict__ xin, T *__restrict__ xout,
                                                        const T *__restrict__ b) {
    __shared__ T sx[5][kRegion];
    __shared__ T sb[3][kRegion];
    const int t = tid();
    const int X0 = blockIdx.x * kBx, Y0 = blockIdx.y * kBy;
    const int Z0 = blockIdx.z * kZc, Z1 = min(Z0 + kZc, nz);
    const int plane = nx * ny;            // cells < 2^31 (checked at creation)
    const T inv = T(1) / (a0 + T(6) * beta);
    // the (at most 2) region cells this thread stages: in-plane offsets of their periodic images
    int goff[2];
    bool have[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int e = t + r * kFlThreads;
        have[r] = e < kRegion;
        const int rx = e % kRx, ry = e / kRx;
        int gx = X0 - 2 + rx, gy = Y0 - 2 + ry;
        gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
        gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
        goff[r] = gy * nx + gx;
    }
    // red cells of a plane on the tile plus its ring of 1 (34 x 10 cells, 17 red per row): thread t < 170
    // takes row 1 + t / 17, the (t % 17)-th red cell of it; black cells of the tile (32 x 8, 16 per row):
    // thread t < 128 takes row t / 16, the (t % 16)-th black cell of it
    constexpr int kRedPerRow = (kRx - 2) / 2, kRed = kRedPerRow * (kRy - 2), kBlackPerRow = kBx / 2;
    const int red_ry = 1 + t / kRedPerRow, red_i = t % kRedPerRow;
    const int blk_ty = t / kBlackPerRow, blk_i = t % kBlackPerRow;
    auto wrapz = [&](int z) { return z < 0 ? z + nz : (z >= nz ? z - nz : z); };
    // the next plane's values are loaded into registers one iteration ahead, so
    // that their latency overlaps the current plane's updates
    T vx[2] = {T(0), T(0)}, vb[2] = {T(0), T(0)};
    auto fetch = [&](int zq) {
        const T *px = xin + wrapz(zq) * plane;
        const T *pb = b + wrapz(zq - 1) * plane;
#pragma unroll
        for (int r = 0; r < 2; ++r)
            if (have[r]) {
                vx[r] = px[goff[r]];
                if (zq >= Z0) vb[r] = pb[goff[r]];
            }
    };
    fetch(Z0 - 2);
    // ring buffers: x of plane z in sx[(z - Z0 + 2) % 5], b of plane z in sb[(z - Z0 + 1) % 3].  With five
    // and three slots a plane is overwritten only after every warp has passed the first barrier of the
    // iteration after its last use, so one barrier after the staging and one after the red cells suffice.
    for (int zp = Z0 - 2, it = 0; zp <= Z1 + 1; ++zp, ++it) {
        T *px = sx[it % 5];
#pragma unroll
        for (int r = 0; r < 2; ++r)
            if (have[r]) {
                px[t + r * kFlThreads] = vx[r];
                if (zp >= Z0) sb[(it - 2) % 3][t + r * kFlThreads] = vb[r];
            }
        if (zp + 1 <= Z1 + 1) fetch(zp + 1);
        __syncthreads();
        // red cells of plane p = zp - 1 on the tile and its ring of 1
        const int p = zp - 1;
        if (p >= Z0 - 1 && p <= Z1 && t < kRed) {
            T *cx = sx[(it + 4) % 5];
            const T *dn = sx[(it + 3) % 5], *up = sx[it % 5];
            const T *cb = sb[(it + 1) % 3];
            const int e = red_ry * kRx + 1 + ((red_ry + p + 1) & 1) + 2 * red_i;
            const T sum = cx[e + 1] + cx[e - 1] + cx[e + kRx] + cx[e - kRx] + up[e] + dn[e];
            cx[e] = (cb[e] + beta * sum) * inv;
        }
        __syncthreads();
        // black cells of plane q = zp - 2 on the tile, and the tile written out: each of the first 128
        // threads writes the black cell it updates and one red cell of the same row (final since the
        // previous iteration), so no barrier separates the update from the write
        const int q = zp - 2;
        if (q >= Z0 && q <= Z1 - 1 && t < kBx * kBy / 2) {
            T *cx = sx[(it + 3) % 5];
            const T *dn = sx[(it + 2) % 5], *up = sx[(it + 4) % 5];
            const T *cb = sb[it % 3];
            const int cb_x = ((blk_ty + q + 1) & 1) + 2 * blk_i;     // black column in the tile
            const int cr_x = ((blk_ty + q) & 1) + 2 * blk_i;         // red column in the tile
            const int e = (blk_ty + 2) * kRx + 2 + cb_x;
            const T sum = cx[e + 1] + cx[e - 1] + cx[e + kRx] + cx[e - kRx] + up[e] + dn[e];
            const T v = (cb[e] + beta * sum) * inv;
            cx[e] = v;
            if (Y0 + blk_ty < ny) {
                T *row = xout + q * plane + (Y0 + blk_ty) * nx + X0;
                if (X0 + cb_x < nx) row[cb_x] = v;
                if (X0 + cr_x < nx) row[cr_x] = cx[(blk_ty + 2) * kRx + 2 + cr_x];
            }
        }
    }
}

// Coarse right-hand side: the fine residual averaged over the 8 children of
// each coarse cell (I, J, K).
template <typename T>
__global__ void __launch_bounds__(kFlThreads) k_mg_restrict(int nx, int ny, int nz, T a0, T beta,
                                                            const T *__restrict__ x, const T *__restrict__ b,
                                                            T *__restrict__ bc) {
    const int cx = nx >> 1, cy = ny >> 1, cz = nz >> 1;
    const int I = blockIdx.x * kBx + threadIdx.x;
    const int J = blockIdx.y * kBy + threadIdx.y;
    if (I >= cx || J >= cy) return;
    for (int K = blockIdx.z; K < cz; K += gridDim.z) {
        T acc = 0;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int i = 2 * I + (d & 1), j = 2 * J + ((d >> 1) & 1), k = 2 * K + (d >> 2);
            const long long c = ((long long)k * ny + j) * nx + i;
            const Nb nb = neighbours(c, i, j, k, nx, ny, nz);
            acc += b[c] - (a0 + T(6) * beta) * x[c] +
                   beta * (x[nb.xp] + x[nb.xm] + x[nb.yp] + x[nb.ym] + x[nb.zp] + x[nb.zm]);
        }
        bc[((long long)K * cy + J) * cx + I] = T(0.125) * acc;
    }
}

// Fine x += trilinear interpolation of the coarse correction (weights 3/4 and
// 1/4 per axis from the two nearest coarse cells, periodic).
template <typename T>
__global__ void __launch_bounds__(kFlThreads) k_mg_prolong(int nx, int ny, int nz, const T *__restrict__ xc,
                                                           T *__restrict__ x) {
    const int cx = nx >> 1, cy = ny >> 1, cz = nz >> 1;
    FOR_CELLS(nx, ny, nz) {
        const long long c = ((long long)k * ny + j) * nx + i;
        const int I0 = i >> 1, J0 = j >> 1, K0 = k >> 1;
        const int I1 = (i & 1) ? (I0 + 1 == cx ? 0 : I0 + 1) : (I0 == 0 ? cx - 1 : I0 - 1);
        const int J1 = (j & 1) ? (J0 + 1 == cy ? 0 : J0 + 1) : (J0 == 0 ? cy - 1 : J0 - 1);
        const int K1 = (k & 1) ? (K0 + 1 == cz ? 0 : K0 + 1) : (K0 == 0 ? cz - 1 : K0 - 1);
        const long long r00 = ((long long)K0 * cy + J0) * cx, r01 = ((long long)K0 * cy + J1) * cx;
        const long long r10 = ((long long)K1 * cy + J0) * cx, r11 = ((long long)K1 * cy + J1) * cx;
        const T e = T(0.421875) * xc[r00 + I0] +
                    T(0.140625) * (xc[r00 + I1] + xc[r01 + I0] + xc[r10 + I0]) +
                    T(0.046875) * (xc[r01 + I1] + xc[r10 + I1] + xc[r11 + I0]) + T(0.015625) * xc[r11 + I1];
        x[c] += e;
    }
}

// Coarsest level: conjugate gradients in one CTA (n <= kCoarseMax) from x = 0,
// vectors in T, dot products accumulated in FP64.  For the singular Poisson
// operator (a0 = 0) the right-hand side is made mean-free first and x is
// returned mean-free.  Stops at |r|_2 <= tol |b|_2 or after maxit iterations.
template <typename T>
__global__ void __launch_bounds__(kCgThreads) k_mg_cg(int nx, int ny, int nz, T a0, T beta, T *__restrict__ x,
                                                      const T *__restrict__ b, T *__restrict__ r, T *__restrict__ p,
                                                      T *__restrict__ q, int maxit, double tol) {
    __shared__ double sh[kCgThreads];
    const int n = nx * ny * nz;
    const bool singular = a0 == T(0);
    double acc = 0.0;
    for (int c = threadIdx.x; c < n; c += kCgThreads) acc += (double)b[c];
    const T mb = singular ? T(block_sum<kCgThreads>(acc, sh) / (double)n) : T(0);
    acc = 0.0;
    for (int c = threadIdx.x; c < n; c += kCgThreads) {
        const T v = b[c] - mb;
        x[c] = T(0);
        r[c] = v;
        p[c] = v;
        acc += (double)v * (double)v;
    }
    double rr = block_sum<kCgThreads>(acc, sh);
    const double stop = tol * tol * rr;
    for (int it = 0; it < maxit && rr > stop; ++it) {
        acc = 0.0;
        for (int c = threadIdx.x; c < n; c += kCgThreads) {
            const Nb nb = neighbours_lin(c, nx, ny, nz);
            const T v = (a0 + T(6) * beta) * p[c] - beta * (p[nb.xp] + p[nb.xm] + p[nb.yp] + p[nb.ym] + p[nb.zp] + p[nb.zm]);
            q[c] = v;
            acc += (double)p[c] * (double)v;
        }
        const double pq = block_sum<kCgThreads>(acc, sh);
        if (!(pq > 0.0)) break;
        const T al = T(rr / pq);
        acc = 0.0;
        for (int c = threadIdx.x; c < n; c += kCgThreads) {
            x[c] += al * p[c];
            const T v = r[c] - al * q[c];
            r[c] = v;
            acc += (double)v * (double)v;
        }
        const double rn = block_sum<kCgThreads>(acc, sh);
        const T be = T(rn / rr);
        rr = rn;
        for (int c = threadIdx.x; c < n; c += kCgThreads) p[c] = r[c] + be * p[c];
        __syncthreads();
    }
    if (singular) {
        acc = 0.0;
        for (int c = threadIdx.x; c < n; c += kCgThreads) acc += (double)x[c];
        const T mx = T(block_sum<kCgThreads>(acc, sh) / (double)n);
        for (int c = threadIdx.x; c < n; c += kCgThreads) x[c] -= mx;
    }
}

// Next free event pair of the profiling pool (nullptr without cfg.profile or
// when the pool is full).
constexpr size_t kProfPairs = 4096;
cudaEvent_t *prof_pair(ibm_fluid *fl) {
    if (!fl->cfg.profile || fl->prof_used >= kProfPairs) return nullptr;
    if (fl->prof.size() < 2 * (fl->prof_used + 1)) {
        cudaEvent_t a = nullptr, b = nullptr;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
            if (a) cudaEventDestroy(a);
            cudaGetLastError();
            return nullptr;
        }
        fl->prof.push_back(a);
        fl->prof.push_back(b);
    }
    return &fl->prof[2 * fl->prof_used++];
}

// FP32 V-cycle on level l for the correction: L.x (zero on entry) from L.b.
void vcycle(ibm_fluid *fl, size_t l, double a0d, double bcoef) {
    ibm_fluid::Level &L = fl->lv[l];
    const float a0 = (float)a0d, beta = (float)(bcoef / (L.h * L.h));
    cudaStream_t sm = fl->stream;
    if (l + 1 == fl->lv.size()) {
        float *r = fl->cg, *p = fl->cg + L.cells, *q = fl->cg + 2 * L.cells;
        k_mg_cg<float><<<1, kCgThreads, 0, sm>>>(L.n[0], L.n[1], L.n[2], a0, beta, L.x, L.b, r, p, q,
                                                 (int)std::min(4 * L.cells + 16, 4000ll), 1e-6);
        return;
    }
    const dim3 gs = grid3(L.n[0] / 2, L.n[1], L.n[2]);
    const dim3 gf((L.n[0] + kBx - 1) / kBx, (L.n[1] + kBy - 1) / kBy, (L.n[2] + kZc - 1) / kZc);
    // two sweeps (x -> x2 -> x when fused)
    auto smooth = [&]() {
        for (int s = 0; s < 2; ++s) {
            cudaEvent_t *e = l == 0 ? prof_pair(fl) : nullptr;
            if (e) cudaEventRecord(e[0], sm);
            if (L.fused) {
                k_mg_rbgs<float><<<gf, kBlock3, 0, sm>>>(L.n[0], L.n[1], L.n[2], a0, beta, s == 0 ? L.x : L.x2,
                                                         s == 0 ? L.x2 : L.x, L.b);
            } else {
                for (int color = 0; color < 2; ++color)
                    k_mg_smooth<float><<<gs, kBlock3, 0, sm>>>(L.n[0], L.n[1], L.n[2], a0, beta, color, L.x, L.b);
            }
            if (e) cudaEventRecord(e[1], sm);
        }
    };
    smooth();
    ibm_fluid::Level &C = fl->lv[l + 1];
    k_mg_restrict<float><<<grid3(C.n[0], C.n[1], C.n[2]), kBlock3, 0, sm>>>(L.n[0], L.n[1], L.n[2], a0, beta, L.x,
                                                                           L.b, C.b);
    cudaMemsetAsync(C.x, 0, C.cells * sizeof(float), sm);
    vcycle(fl, l + 1, a0d, bcoef);
    k_mg_prolong<float><<<grid3(L.n[0], L.n[1], L.n[2]), kBlock3, 0, sm>>>(L.n[0], L.n[1], L.n[2], C.x, L.x);
    smooth();
}

double bits_to_double(unsigned long long b) {
    double d;
    std::memcpy(&d, &b, sizeof d);
    return d;
}

// Solve A x = rhs (FP64, level 0; x holds the initial guess) by iterative
// refinement with FP32 V-cycles; fl->maxw[0] holds max|rhs| (written by the
// right-hand-side kernel).  bs: device mean of rhs or NULL.
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
    const dim3 g3 = grid3(L.n[0], L.n[1], L.n[2]);
    double rscale = 1.0 / bmax;      // keeps the FP32 residual of order one
    double r = 0.0;
    int it = 0;
    for (;; ++it) {
        FK(cudaMemsetAsync(fl->maxw + 1, 0, sizeof(unsigned long long), sm), "zero norm");
        k_mg_resid64<<<g3, kBlock3, 0, sm>>>(L.n[0], L.n[1], L.n[2], a0, beta, x, fl->rhs, bs, rscale, L.b,
                                             fl->maxw + 1);
        FK(cudaGetLastError(), "residual launch");
        FK(cudaMemcpyAsync(fl->hmax + 1, fl->maxw + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost, sm),
           "read norm");
        FK(cudaStreamSynchronize(sm), "synchronise");
        r = bits_to_double(fl->hmax[1]);
        if (!std::isfinite(r)) return fl_fail(fl, IBM_ERR_NONFINITE, "non-finite residual in a fluid solve");
        if (r <= tol || it == fl->cfg.max_cycles) break;
        FK(cudaMemsetAsync(L.x, 0, L.cells * sizeof(float), sm), "zero correction");
        vcycle(fl, 0, a0, bcoef);
        k_mg_update64<<<grid_cells(L.cells), kFlThreads, 0, sm>>>(L.cells, x, L.x, 1.0 / rscale);
        FK(cudaGetLastError(), "multigrid launch");
        rscale = 1.0 / r;
    }
    fl->cycles[slot] = it;
    fl->resid[slot] = r / bmax;
    if (!(r <= tol))
        return fl_fail(fl, IBM_ERR_NOCONVERGE,
                       "fluid solve " + std::to_string(slot) + " stopped at relative residual " +
                           std::to_string(r / bmax) + " after " + std::to_string(it) + " V-cycles");
    return IBM_OK;
}

void free_all(ibm_fluid *fl) {
    double *bufs[] = {fl->nold, fl->rhs, fl->f, fl->red, fl->mean};
    for (double *b : bufs)
        if (b) cudaFree(b);
    if (fl->cg) cudaFree(fl->cg);
    if (fl->maxw) cudaFree(fl->maxw);
    for (size_t l = 0; l < fl->lv.size(); ++l) {
        if (fl->lv[l].x) cudaFree(fl->lv[l].x);
        if (fl->lv[l].b) cudaFree(fl->lv[l].b);
        if (fl->lv[l].x2) cudaFree(fl->lv[l].x2);
    }
    if (fl->hmax) cudaFreeHost(fl->hmax);
    for (cudaEvent_t e : fl->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : fl->prof) cudaEventDestroy(e);
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
    ibm_fluid::Level L0{{cfg->nx, cfg->ny, cfg->nz}, cells, cfg->h, nullptr, nullptr, nullptr, false};
    fl->lv.push_back(L0);
    while (true) {
        const ibm_fluid::Level &p = fl->lv.back();
        if (p.n[0] % 2 || p.n[1] % 2 || p.n[2] % 2 || p.n[0] < 4 || p.n[1] < 4 || p.n[2] < 4) break;
        ibm_fluid::Level c{{p.n[0] / 2, p.n[1] / 2, p.n[2] / 2}, p.cells / 8, p.h * 2.0, nullptr, nullptr, nullptr,
                           false};
        fl->lv.push_back(c);
    }
    // fused sweeps on the smoothed levels wide enough for a tile (the coarsest level is not smoothed)
    for (size_t l = 0; l + 1 < fl->lv.size(); ++l)
        fl->lv[l].fused = !cfg->two_pass_smoother && fl->lv[l].n[0] >= kBx && fl->lv[l].n[1] >= kBy;
    if (fl->lv.back().cells > kCoarseMax || (cfg->ny + kBy - 1) / kBy > 65535) {
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
    {
        const dim3 g3 = grid3(cfg->nx, cfg->ny, cfg->nz);
        const long long nparts = (long long)g3.x * g3.y * g3.z;
        if ((e = ibm_malloc(&fl->red, (nparts + 8) * sizeof(double))) != cudaSuccess) return fail(e);
    }
    if ((e = ibm_malloc(&fl->mean, 8 * sizeof(double))) != cudaSuccess) return fail(e);
    if ((e = ibm_malloc(&fl->maxw, 4 * sizeof(unsigned long long))) != cudaSuccess) return fail(e);
    if ((e = ibm_malloc(&fl->cg, 3 * fl->lv.back().cells * sizeof(float))) != cudaSuccess) return fail(e);
    for (size_t l = 0; l < fl->lv.size(); ++l) {
        ibm_fluid::Level &L = fl->lv[l];
        if ((e = ibm_malloc(&L.x, L.cells * sizeof(float))) != cudaSuccess) return fail(e);
        if ((e = ibm_malloc(&L.b, L.cells * sizeof(float))) != cudaSuccess) return fail(e);
        if (L.fused && (e = ibm_malloc(&L.x2, L.cells * sizeof(float))) != cudaSuccess) return fail(e);
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
    k_fl_predict<<<grid3(fl->n[0], fl->n[1], fl->n[2]), kBlock3, 0, fl->stream>>>(
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
    const dim3 g3 = grid3(fl->n[0], fl->n[1], fl->n[2]);
    const long long nparts = (long long)g3.x * g3.y * g3.z;
    // (e) three Helmholtz solves, each in place in ut (initial guess u~_q)
    for (int q = 0; q < 3; ++q) {
        FK(cudaMemsetAsync(fl->maxw, 0, sizeof(unsigned long long), sm), "zero norm");
        k_fl_hrhs<<<g3, kBlock3, 0, sm>>>(fl->n[0], fl->n[1], fl->n[2], fl->cfg.h, q, two_a_dt, cv, fl->cfg.theta,
                                             F->ut, F->u, F->p, mf, fl->rhs, fl->maxw);
        FK(cudaGetLastError(), "right-hand side launch");
        ibm_status st = mg_solve(fl, 1.0, cv, F->ut + q * n, nullptr, q);
        if (st != IBM_OK) return st;
    }
    // (f), (g)
    FK(cudaMemsetAsync(fl->maxw, 0, sizeof(unsigned long long), sm), "zero norm");
    k_fl_prhs<<<g3, kBlock3, 0, sm>>>(fl->n[0], fl->n[1], fl->n[2], fl->cfg.h, two_a_dt, F->ut, F->uf,
                                                 fl->rhs, fl->red, fl->maxw);
    k_fl_mean_final<<<1, kFlThreads, 0, sm>>>(nparts, fl->red, (double)n, fl->mean + 3);
    FK(cudaGetLastError(), "Poisson right-hand side launch");
    ibm_status st = mg_solve(fl, 0.0, 1.0, F->phi, fl->mean + 3, 3);
    if (st != IBM_OK) return st;
    // mean of phi, then (h), (i), and phi made mean-free
    k_fl_sum<<<g3, kBlock3, 0, sm>>>(fl->n[0], fl->n[1], fl->n[2], F->phi, fl->red);
    k_fl_mean_final<<<1, kFlThreads, 0, sm>>>(nparts, fl->red, (double)n, fl->mean + 4);
    k_fl_correct<<<g3, kBlock3, 0, sm>>>(fl->n[0], fl->n[1], fl->n[2], fl->cfg.h, two_a_dt, a * dt * fl->cfg.nu,
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

ibm_status ibm_fluid_kernel_timing(ibm_fluid *fl, double *total_ms, int64_t *count, int reset) {
    if (!fl) return IBM_ERR_INVALID_ARG;
    double tot = 0.0;
    if (fl->prof_used) {
        FK(cudaStreamSynchronize(fl->stream), "synchronise");
        for (size_t i = 0; i < fl->prof_used; ++i) {
            float ms = 0.f;
            FK(cudaEventElapsedTime(&ms, fl->prof[2 * i], fl->prof[2 * i + 1]), "event time");
            tot += ms;
        }
    }
    if (total_ms) *total_ms = tot;
    if (count) *count = (int64_t)fl->prof_used;
    if (reset) fl->prof_used = 0;
    return IBM_OK;
}

const char *ibm_fluid_last_error(const ibm_fluid *fl) { return fl ? fl->last_error.c_str() : ""; }

}  // extern "C"
