// ibm_forcing_step_static: the plain FP64 forcing step for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at all: hosts that hand the library a
// fixed memory budget at start-up and forbid allocations afterwards, plugins
// embedded in an application whose own allocator owns every byte of the device
// (a cudaMalloc beside it fails or fragments its pool), and time-critical loops
// that cannot afford the device-wide synchronisation of cudaFree.  This entry
// point needs no context and allocates nothing, on the device or on the host:
// its scratch (per-marker slip values, per-particle marker offsets, an error
// word) lives in one fixed-size array in this file, kStaticBytes long, which
// every GPU that loads the library holds until the process exits.
//
// The array is shared by every call: a call overwrites what the previous one
// left there (it clears what must start at zero), and two calls whose work
// overlaps on the GPU (different streams, or different host threads on the
// same device) race on it and corrupt each other's results.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>

#include "ibm_device.cuh"
#include "ibm_internal.h"

namespace {

constexpr size_t kStaticBytes = 16u << 20;          // 16 MiB of scratch per device
constexpr int kStaticMaxParticles = 65536;
constexpr int kStaticBlock = 256;
constexpr size_t kCtrlBytes = 256;                    // error word, marker total
constexpr size_t kOffBytes = ((size_t)(kStaticMaxParticles + 1) * sizeof(int) + 255) & ~(size_t)255;
constexpr size_t kStaticMaxMarkers = (kStaticBytes - kCtrlBytes - kOffBytes) / (3 * sizeof(double));

// The scratch array.  Host code must not pass this name to a kernel: in host
// code it is only a stand-in; its device address comes from
// cudaGetSymbolAddress (static_scratch_ptr below).
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

struct Scratch {
    int *err;        // [0] error bits, [1] total markers
    int *moff;       // [n_p + 1] marker offsets
    double *e;       // [markers][3] slip of the current iteration
};

__device__ __forceinline__ Scratch scratch_view(unsigned char *base) {
    Scratch s;
    s.err = reinterpret_cast<int *>(base);
    s.moff = reinterpret_cast<int *>(base + kCtrlBytes);
    s.e = reinterpret_cast<double *>(base + kCtrlBytes + kOffBytes);
    return s;
}

// Validation, marker counts N_l = round(pi (d/h)^2) and their exclusive prefix
// (one block), the marker total, and zeroed loads.  Sets error bits instead of
// running when the particle data is invalid or the markers exceed the array.
__global__ void k_static_setup(unsigned char *base, int n_p, const double *x, const double *up, const double *om,
                               const double *d, int nx, int ny, int nz, double h, double *F, double *T) {
    Scratch S = scratch_view(base);
    __shared__ long long part[kStaticBlock];
    __shared__ int bad;
    const int t = threadIdx.x;
    if (t == 0) bad = 0;
    __syncthreads();
    const int me = min(nx, min(ny, nz));
    // outputs start at zero for every particle, valid or not, so that a
    // rejected call leaves no stale rows behind
    for (int i = t; i < 3 * n_p; i += kStaticBlock) {
        F[i] = 0.0;
        T[i] = 0.0;
    }
    const int chunk = (n_p + kStaticBlock - 1) / kStaticBlock;
    const int lo = min(n_p, t * chunk), hi = min(n_p, lo + chunk);
    long long sum = 0;
    for (int p = lo; p < hi; ++p) {
        bool ok = isfinite(d[p]) && d[p] > 0.0 && d[p] / h + 4.0 <= (double)me;
        for (int c = 0; c < 3; ++c)
            ok = ok && isfinite(x[3 * p + c]) && isfinite(up[3 * p + c]) && isfinite(om[3 * p + c]);
        if (!ok) {
            atomicOr(&bad, IBM_EBIT_DIAMETER);
            continue;
        }
        const double q = d[p] / h;
        long long n = llround(IBM_PI * q * q);
        sum += n < 1 ? 1 : n;
    }
    part[t] = sum;
    __syncthreads();
    for (int o = 1; o < kStaticBlock; o <<= 1) {
        const long long v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    long long run = part[t] - sum;
    for (int p = lo; p < hi; ++p) {
        S.moff[p] = (int)min(run, (long long)INT_MAX);
        const double q = d[p] / h;
        long long n = llround(IBM_PI * q * q);
        run += n < 1 ? 1 : n;
    }
    if (t == kStaticBlock - 1) {
        const long long total = part[t];
        S.moff[n_p] = (int)min(total, (long long)INT_MAX);
        S.err[1] = (int)min(total, (long long)INT_MAX);
        int e = bad;
        if (total > (long long)kStaticMaxMarkers) e |= IBM_EBIT_OVERFLOW;
        S.err[0] = e;
    }
}

// Marker l of particle p, FP64, computed in place: golden-spiral direction
// (Sec. 2.1 reading), position xi = x_p/h + ((d/2)/h) t, its stencil base cell
// and weights (Eq. 3pt-stencil), arm r = (d/2) t and U^d = u_p + w_p x r.
struct StaticMarker {
    int b[3];
    double w[3][3];
    double r[3];
    double ud[3];
};

__device__ __forceinline__ void static_marker(int p, int l, int nl, const double *x, const double *up,
                                              const double *om, const double *d, double h, StaticMarker &M) {
    const double ga = IBM_PI * (3.0 - sqrt(5.0));
    const double z = __dsub_rn(1.0, (double)(2 * l + 1) / (double)nl);
    const double th = __dmul_rn((double)l, ga);
    const double rho = sqrt(__dsub_rn(1.0, __dmul_rn(z, z)));
    const double t[3] = {__dmul_rn(rho, cos(th)), __dmul_rn(rho, sin(th)), z};
    const double a = (0.5 * d[p]) / h;
    for (int c = 0; c < 3; ++c) {
        const double xi = __dadd_rn(x[3 * p + c] / h, __dmul_rn(a, t[c]));
        const double fb = floor(xi);
        M.b[c] = (int)fb;
        phi3_weights<double>(xi - fb, M.w[c]);
        M.r[c] = (0.5 * d[p]) * t[c];
    }
    const double *w = om + 3 * p;
    M.ud[0] = up[3 * p + 0] + (w[1] * M.r[2] - w[2] * M.r[1]);
    M.ud[1] = up[3 * p + 1] + (w[2] * M.r[0] - w[0] * M.r[2]);
    M.ud[2] = up[3 * p + 2] + (w[0] * M.r[1] - w[1] * M.r[0]);
}

__device__ __forceinline__ int static_nl(double d, double h) {
    const double q = d / h;
    const long long n = llround(IBM_PI * q * q);
    return n < 1 ? 1 : (int)n;
}

// Steps 1-2 of the outer forcing loop (Sec. 2.2.2), one block per particle:
// e = U^d - W u, kept in the scratch array; the block adds sum e D and
// sum r x e D to the particle's loads.
__global__ void __launch_bounds__(kStaticBlock) k_static_interp(unsigned char *base, int n_p, const double *x,
                                                                 const double *up, const double *om,
                                                                 const double *d, int nx, int ny, int nz,
                                                                 double h, const double *u, double *F, double *T) {
    Scratch S = scratch_view(base);
    if (S.err[0]) return;
    const long long ncell = (long long)nx * ny * nz;
    __shared__ double sh[6][kStaticBlock / 32];
    for (int p = blockIdx.x; p < n_p; p += gridDim.x) {
        const int nl = static_nl(d[p], h), moff = S.moff[p];
        const double D = IBM_PI * (d[p] * d[p] * h + h * h * h / 3.0) / (double)nl / (h * h * h);
        double acc[6] = {0, 0, 0, 0, 0, 0};
        for (int l = threadIdx.x; l < nl; l += blockDim.x) {
            StaticMarker M;
            static_marker(p, l, nl, x, up, om, d, h, M);
            double U[3] = {0, 0, 0};
            for (int cz = 0; cz < 3; ++cz)
                for (int cy = 0; cy < 3; ++cy) {
                    const long long row =
                        ((long long)wrapi(M.b[2] - 1 + cz, nz) * ny + wrapi(M.b[1] - 1 + cy, ny)) * nx;
                    for (int cx = 0; cx < 3; ++cx) {
                        const double wt = M.w[2][cz] * M.w[1][cy] * M.w[0][cx];
                        const long long idx = row + wrapi(M.b[0] - 1 + cx, nx);
                        for (int q = 0; q < 3; ++q) U[q] += wt * u[q * ncell + idx];
                    }
                }
            double e[3];
            for (int q = 0; q < 3; ++q) {
                e[q] = M.ud[q] - U[q];
                S.e[3ll * (moff + l) + q] = e[q];
            }
            acc[0] += e[0] * D;
            acc[1] += e[1] * D;
            acc[2] += e[2] * D;
            acc[3] += (M.r[1] * e[2] - M.r[2] * e[1]) * D;
            acc[4] += (M.r[2] * e[0] - M.r[0] * e[2]) * D;
            acc[5] += (M.r[0] * e[1] - M.r[1] * e[0]) * D;
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int i = 0; i < 6; ++i) {
            const double v = warp_sum(acc[i]);
            if (lane == 0) sh[i][wid] = v;
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            double v = 0.0;
            for (int w = 0; w < kStaticBlock / 32; ++w) v += sh[threadIdx.x][w];
            if (threadIdx.x < 3) F[3 * p + threadIdx.x] += v;
            else T[3 * p + threadIdx.x - 3] += v;
        }
        __syncthreads();
    }
}

// Steps 3-4 (Sec. 2.2.2): u += tau f = sum_l w D e_l, global FP64 atomics.
__global__ void __launch_bounds__(kStaticBlock) k_static_spread(unsigned char *base, int n_p, const double *x,
                                                                 const double *up, const double *om,
                                                                 const double *d, int nx, int ny, int nz,
                                                                 double h, double *u) {
    Scratch S = scratch_view(base);
    if (S.err[0]) return;
    const long long ncell = (long long)nx * ny * nz;
    for (int p = blockIdx.x; p < n_p; p += gridDim.x) {
        const int nl = static_nl(d[p], h), moff = S.moff[p];
        const double D = IBM_PI * (d[p] * d[p] * h + h * h * h / 3.0) / (double)nl / (h * h * h);
        for (int l = threadIdx.x; l < nl; l += blockDim.x) {
            StaticMarker M;
            static_marker(p, l, nl, x, up, om, d, h, M);
            double g[3];
            for (int q = 0; q < 3; ++q) g[q] = D * S.e[3ll * (moff + l) + q];
            for (int cz = 0; cz < 3; ++cz)
                for (int cy = 0; cy < 3; ++cy) {
                    const long long row =
                        ((long long)wrapi(M.b[2] - 1 + cz, nz) * ny + wrapi(M.b[1] - 1 + cy, ny)) * nx;
                    for (int cx = 0; cx < 3; ++cx) {
                        const double wt = M.w[2][cz] * M.w[1][cy] * M.w[0][cx];
                        const long long idx = row + wrapi(M.b[0] - 1 + cx, nx);
                        for (int q = 0; q < 3; ++q) atomicAdd(u + q * ncell + idx, wt * g[q]);
                    }
                }
        }
    }
}

// Loads in physical units: F_p = (h^3/tau) sum e D, T_p likewise.
__global__ void k_static_scale(unsigned char *base, int n_p, double s, double *F, double *T) {
    Scratch S = scratch_view(base);
    if (S.err[0]) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n_p; i += gridDim.x * blockDim.x) {
        F[i] *= s;
        T[i] *= s;
    }
}

// Device address of the scratch array on the current device, looked up at
// set-up: the first call on a device runs cudaGetSymbolAddress with that
// device current, later calls reuse the address.  The entries are atomic, so
// host threads calling concurrently on different devices (or racing on the
// first call of one device, which both resolve to the same address) are safe.
// cudaDeviceReset unloads the library's module on that device and makes the
// stored address stale: the entry point must not be used on a device after it
// has been reset within the same process.
constexpr int kMaxDevices = 64;
std::atomic<unsigned char *> g_scratch_ptr[kMaxDevices];

cudaError_t static_scratch_ptr(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    unsigned char *p = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        void *q = nullptr;
        e = cudaGetSymbolAddress(&q, g_static_scratch);
        if (e != cudaSuccess) return e;
        p = static_cast<unsigned char *>(q);
        g_scratch_ptr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return cudaSuccess;
}

}  // namespace

extern "C" ibm_status ibm_forcing_step_static(int nx, int ny, int nz, double h, int n_forcing, double tau, int n_p,
                                              const double *x_p, const double *u_p, const double *omega_p,
                                              const double *d_p, double *u, double *F_out, double *T_out,
                                              void *cuda_stream) {
    if (nx < 8 || ny < 8 || nz < 8 || nx > (1 << 20) || ny > (1 << 20) || nz > (1 << 20)) return IBM_ERR_INVALID_ARG;
    if (!(h > 0.0) || !std::isfinite(h) || !(tau > 0.0) || !std::isfinite(tau)) return IBM_ERR_INVALID_ARG;
    if (n_forcing < 1 || n_forcing > 64 || n_p < 0) return IBM_ERR_INVALID_ARG;
    if (n_p > kStaticMaxParticles) return IBM_ERR_CAPACITY;
    if (n_p == 0) return IBM_OK;
    if (!x_p || !u_p || !omega_p || !d_p || !u || !F_out || !T_out) return IBM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    unsigned char *base = nullptr;
    if (static_scratch_ptr(&base) != cudaSuccess) {
        cudaGetLastError();
        return IBM_ERR_CUDA;
    }
    k_static_setup<<<1, kStaticBlock, 0, st>>>(base, n_p, x_p, u_p, omega_p, d_p, nx, ny, nz, h, F_out, T_out);
    const int nb = n_p < 152 * 16 ? n_p : 152 * 16;
    for (int it = 0; it < n_forcing; ++it) {
        k_static_interp<<<nb, kStaticBlock, 0, st>>>(base, n_p, x_p, u_p, omega_p, d_p, nx, ny, nz, h, u, F_out,
                                                      T_out);
        k_static_spread<<<nb, kStaticBlock, 0, st>>>(base, n_p, x_p, u_p, omega_p, d_p, nx, ny, nz, h, u);
    }
    k_static_scale<<<(3 * n_p + 255) / 256, 256, 0, st>>>(base, n_p, h * h * h / tau, F_out, T_out);
    if (cudaGetLastError() != cudaSuccess) return IBM_ERR_CUDA;
    // report rejected sizes and invalid particle data: read the error word
    // into a host stack variable (no allocation) and wait for the stream
    int err = 0;
    if (cudaMemcpyAsync(&err, base, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return IBM_ERR_CUDA;
    }
    if (err & IBM_EBIT_OVERFLOW) return IBM_ERR_CAPACITY;
    if (err) return IBM_ERR_INVALID_ARG;
    return IBM_OK;
}
