// Particle set-up, marker templates, the plain forcing path (one thread per
// marker, global atomics; FP64 and FP32), the slip diagnostic, the particle
// loads / Newton-Euler update and the adjoint kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ibm_device.cuh"
#include "ibm_internal.h"

#define CK(call, what)                                                  \
    do {                                                                \
        ibm_status _s = ibm_cuda_check(ctx, (call), what);              \
        if (_s != IBM_OK) return _s;                                    \
    } while (0)

namespace {

constexpr int kBlock = 256;

// ------------------------------------------------------------------ set-up

// Validation and marker counts N_l = round(pi (d/h)^2) (reading of Sec. 2.1:
// N_l dV_l is the shell volume and dV_l ~ h^3).
__global__ void k_setup(int n_p, const double *x, const double *up, const double *om,
                        const double *d, const double *rho, const int32_t *scene,
                        const int32_t *dims, int n_scenes, double h, int newton_euler,
                        double rho_f, int *nl, int *max_nl, int *err) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_p; p += gridDim.x * blockDim.x) {
        bool finite = true;
        for (int c = 0; c < 3; ++c)
            finite = finite && isfinite(x[3 * p + c]) && isfinite(up[3 * p + c]) && isfinite(om[3 * p + c]);
        finite = finite && isfinite(d[p]) && (!newton_euler || isfinite(rho[p]));
        if (!finite) { set_err(err, IBM_EBIT_NONFINITE); nl[p] = 1; continue; }
        const int s = scene[p];
        if (s < 0 || s >= n_scenes) { set_err(err, IBM_EBIT_SCENE); nl[p] = 1; continue; }
        const int me = min(dims[3 * s], min(dims[3 * s + 1], dims[3 * s + 2]));
        const double q = d[p] / h;
        if (!(d[p] > 0.0) || q + 4.0 > (double)me) { set_err(err, IBM_EBIT_DIAMETER); nl[p] = 1; continue; }
        if (newton_euler && !(fabs(rho[p] / rho_f - 1.0) >= 1e-6)) set_err(err, IBM_EBIT_DENSITY);
        long long n = llround(IBM_PI * q * q);
        if (n < 1) n = 1;
        if (n > (1 << 22)) { set_err(err, IBM_EBIT_DIAMETER); n = 1; }
        nl[p] = (int)n;
        atomicMax(max_nl, (int)n);
    }
}

// Single-block exclusive scan (int in, int out with out[n] = total) and the
// 64-bit total.
__global__ void k_scan_block(const int *in, int *out, int n, long long *total) {
    __shared__ long long part[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int chunk = (n + T - 1) / T;
    const int lo = min(n, t * chunk), hi = min(n, lo + chunk);
    long long s = 0;
    for (int i = lo; i < hi; ++i) s += in[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {
        long long v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    long long run = part[t] - s;
    for (int i = lo; i < hi; ++i) {
        out[i] = (int)run;
        run += in[i];
    }
    if (t == T - 1) {
        *total = part[t];
        out[n] = (int)part[t];
    }
}

__global__ void k_flag_new_nl(int n_p, const int *nl, const int *tmpl_of_nl, int *flag) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_p; p += gridDim.x * blockDim.x) {
        const int n = nl[p];
        if (tmpl_of_nl[n] < 0) flag[n] = 1;
    }
}

// Golden-spiral unit directions of an N-marker sphere (reading of Sec. 2.1):
// z = 1 - (2l+1)/N, theta = l pi (3 - sqrt 5), rho = sqrt(1 - z^2),
// t = (rho cos theta, rho sin theta, z); rounded operation by operation.
__global__ void k_templates(const int *list_nl, const int *list_off, int n_list, double *t64,
                            float *t32) {
    const double ga = IBM_PI * (3.0 - sqrt(5.0));
    for (int k = blockIdx.y; k < n_list; k += gridDim.y) {
        const int N = list_nl[k], off = list_off[k];
        for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < N; l += gridDim.x * blockDim.x) {
            const double z = __dsub_rn(1.0, (double)(2 * l + 1) / (double)N);
            const double th = __dmul_rn((double)l, ga);
            const double rho = sqrt(__dsub_rn(1.0, __dmul_rn(z, z)));
            const double tx = __dmul_rn(rho, cos(th)), ty = __dmul_rn(rho, sin(th));
            double *o = t64 + 3ll * (off + l);
            o[0] = tx; o[1] = ty; o[2] = z;
            float *of = t32 + 3ll * (off + l);
            of[0] = (float)tx; of[1] = (float)ty; of[2] = (float)z;
        }
    }
}

__global__ void k_toff(int n_p, const int *nl, const int *tmpl_of_nl, int *toff) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_p; p += gridDim.x * blockDim.x)
        toff[p] = tmpl_of_nl[nl[p]];
}

// Per-step particle record.  dV_l = pi (d^2 h + h^3/3)/N_l (Sec. 2.1).
__global__ void k_pinfo(int n_p, const double *x, const double *up, const double *om, const double *d,
                        const int32_t *scene, const int *nl, const int *moff, const int *toff, double h,
                        PInfo *P) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_p; p += gridDim.x * blockDim.x) {
        PInfo q;
        for (int c = 0; c < 3; ++c) {
            const double xi = x[3 * p + c] / h;
            const double fb = floor(xi);
            q.xi[c] = xi;
            q.base[c] = (int)fb;
            q.fracf[c] = (float)(xi - fb);
            q.ud[c] = (float)up[3 * p + c];
            q.om[c] = (float)om[3 * p + c];
        }
        q.a = (0.5 * d[p]) / h;
        q.af = (float)q.a;
        q.nl = nl[p];
        q.moff = moff[p];
        q.toff = toff[p];
        q.scene = scene[p];
        const double dv = IBM_PI * (d[p] * d[p] * h + h * h * h / 3.0) / (double)nl[p];
        q.D64 = dv / (h * h * h);
        q.D = (float)q.D64;
        q.rphys64 = 0.5 * d[p];
        q.rphys = (float)q.rphys64;
        P[p] = q;
    }
}

// ------------------------------------------------------- marker evaluation

// K = 3: base b = floor(xi), cells b-1..b+1, Eq. (3pt-stencil).  K = 4:
// b = floor(xi - 1/2), cells b-1..b+2, the four-point kernel of Sec. 2.2.3.
template <typename T, int K = 3>
struct Stencil {
    int b[3];      // absolute (unwrapped) base cell
    T w[3][K];     // [axis][cell b-1, b, ...]
    T f[3];        // fraction: xi - b (K = 3), xi - 1/2 - b (K = 4)
};

__device__ __forceinline__ void marker_stencil(const PInfo &P, const double *t64, const float *,
                                               Stencil<double> &S) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double xi = marker_xi64(P, t64, c);
        const double fb = floor(xi);
        S.b[c] = (int)fb;
        S.f[c] = xi - fb;
        phi3_weights<double>(S.f[c], S.w[c]);
    }
}

__device__ __forceinline__ void marker_stencil(const PInfo &P, const double *t64, const float *t32,
                                               Stencil<float> &S) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float fr;
        S.b[c] = marker_split32(P, t32, t64, c, &fr);
        S.f[c] = fr;
        phi3_weights(fr, S.w[c]);
    }
}

__device__ __forceinline__ void marker_stencil(const PInfo &P, const double *t64, const float *,
                                               Stencil<double, 4> &S) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double xh = marker_xi64(P, t64, c) - 0.5;
        const double fb = floor(xh);
        S.b[c] = (int)fb;
        S.f[c] = xh - fb;
        phi4_weights<double>(S.f[c], S.w[c]);
    }
}

__device__ __forceinline__ void marker_stencil(const PInfo &P, const double *t64, const float *t32,
                                               Stencil<float, 4> &S) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float g;
        S.b[c] = marker_split32_half(P, t32, t64, c, &g);
        S.f[c] = g;
        phi4_weights<float>(g, S.w[c]);
    }
}

// Desired velocity U^d = u_p + w_p x r_l (Sec. 2.1) with r_l = (d_p/2) t_l.
__device__ __forceinline__ void marker_kinematics(const double *up, const double *om, int p,
                                                  const PInfo &P, const double *t64, const float *,
                                                  double ud[3], double r[3], double &D) {
    for (int c = 0; c < 3; ++c) r[c] = P.rphys64 * t64[c];
    const double *w = om + 3 * p;
    ud[0] = up[3 * p + 0] + (w[1] * r[2] - w[2] * r[1]);
    ud[1] = up[3 * p + 1] + (w[2] * r[0] - w[0] * r[2]);
    ud[2] = up[3 * p + 2] + (w[0] * r[1] - w[1] * r[0]);
    D = P.D64;
}

__device__ __forceinline__ void marker_kinematics(const double *, const double *, int, const PInfo &P,
                                                  const double *, const float *t32, float ud[3], float r[3],
                                                  float &D) {
    for (int c = 0; c < 3; ++c) r[c] = P.rphys * t32[c];
    ud[0] = P.ud[0] + (P.om[1] * r[2] - P.om[2] * r[1]);
    ud[1] = P.ud[1] + (P.om[2] * r[0] - P.om[0] * r[2]);
    ud[2] = P.ud[2] + (P.om[0] * r[1] - P.om[1] * r[0]);
    D = P.D;
}

struct Grid {
    int nx, ny, nz;
    long long ncell;
};

__device__ __forceinline__ Grid scene_grid(const int32_t *dims, int s) {
    Grid g;
    g.nx = dims[3 * s];
    g.ny = dims[3 * s + 1];
    g.nz = dims[3 * s + 2];
    g.ncell = (long long)g.nx * g.ny * g.nz;
    return g;
}

// Block-wide sum of NV doubles; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*sh)[32]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double s = warp_sum(v[i]);
        if (lane == 0) sh[i][wid] = s;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double s = lane < nw ? sh[i][lane] : 0.0;
            v[i] = warp_sum(s);
        }
    }
    __syncthreads();
}

// ----------------------------------------------------------- plain kernels

// Steps 1-2 of the outer forcing loop (Sec. 2.2.2): U = W u, e = U^d - U
// (F = e / tau), one block per particle, one thread per marker.  Stores e and
// adds sum e D and sum r x e D to the particle's load accumulators.
// FB (deterministic fallback): also the per-cluster maxima of |u| over the
// stencil cells, of |e| and of D (float bits in cm[3c..3c+2], atomicMax), from
// which the spreading's fixed-point scale follows.
template <typename T, bool FB = false, int K = 3>
__global__ void __launch_bounds__(kBlock) k_plain_interp(
    const PInfo *__restrict__ P, const int *__restrict__ plist, int n_list, const int *__restrict__ n_list_d,
    const double *__restrict__ t64, const float *__restrict__ t32, const double *__restrict__ up,
    const double *__restrict__ om, const int32_t *__restrict__ dims, T *const *uf, T *__restrict__ ebuf,
    double *__restrict__ cbuf, const int *__restrict__ pcl = nullptr, unsigned *cm = nullptr,
    const unsigned *__restrict__ dis = nullptr) {
    __shared__ double sh[6][32];
    __shared__ float shm[2][32];
    if (n_list_d) n_list = *n_list_d;
    for (int k = blockIdx.y; k < n_list; k += gridDim.y) {
        const int p = plist ? plist[k] : k;
        const PInfo Pp = P[p];
        const Grid g = scene_grid(dims, Pp.scene);
        const T *__restrict__ u = uf[Pp.scene];
        double acc[6] = {0, 0, 0, 0, 0, 0};
        float umax = 0.f, emax = 0.f;
        for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < Pp.nl; l += gridDim.x * blockDim.x) {
            const double *tt64 = t64 + 3ll * (Pp.toff + l);
            const float *tt32 = t32 + 3ll * (Pp.toff + l);
            Stencil<T, K> S;
            marker_stencil(Pp, tt64, tt32, S);
            T ud[3], r[3], D;
            marker_kinematics(up, om, p, Pp, tt64, tt32, ud, r, D);
            T U[3] = {T(0), T(0), T(0)};
            int ii[K];
#pragma unroll
            for (int a = 0; a < K; ++a) ii[a] = wrapi(S.b[0] - 1 + a, g.nx);
#pragma unroll
            for (int cz = 0; cz < K; ++cz) {
                const int kk = wrapi(S.b[2] - 1 + cz, g.nz);
#pragma unroll
                for (int cy = 0; cy < K; ++cy) {
                    const int jj = wrapi(S.b[1] - 1 + cy, g.ny);
                    const long long row = ((long long)kk * g.ny + jj) * g.nx;
                    const T wyz = S.w[2][cz] * S.w[1][cy];
#pragma unroll
                    for (int cx = 0; cx < K; ++cx) {
                        const T w = wyz * S.w[0][cx];
                        const long long idx = row + ii[cx];
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            const T v = u[q * g.ncell + idx];
                            U[q] += w * v;
                            if (FB) umax = fmaxf(umax, fabsf((float)v));
                        }
                    }
                }
            }
            T e[3];
            // a marker left out near contact (Sec. 2.2.5) has F = 0
            const long long mk = (long long)Pp.moff + l;
            const bool off = dis && ((dis[mk >> 5] >> (mk & 31)) & 1u);
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                e[q] = off ? T(0) : ud[q] - U[q];
                ebuf[3ll * (Pp.moff + l) + q] = e[q];
                if (FB) emax = fmaxf(emax, fabsf((float)e[q]));
            }
            const double ed[3] = {(double)(e[0] * D), (double)(e[1] * D), (double)(e[2] * D)};
            const double rd[3] = {(double)r[0], (double)r[1], (double)r[2]};
            acc[0] += ed[0];
            acc[1] += ed[1];
            acc[2] += ed[2];
            acc[3] += rd[1] * ed[2] - rd[2] * ed[1];
            acc[4] += rd[2] * ed[0] - rd[0] * ed[2];
            acc[5] += rd[0] * ed[1] - rd[1] * ed[0];
        }
        block_sum<6>(acc, sh);
        // this chunk's partial sums; the spreading kernel adds the chunks in order
        if (threadIdx.x == 0)
            for (int q = 0; q < 6; ++q) cbuf[(6ll * k) * gridDim.x + 6 * blockIdx.x + q] = acc[q];
        if (FB) {
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
            umax = warp_max(umax);
            emax = warp_max(emax);
            if (lane == 0) { shm[0][wid] = umax; shm[1][wid] = emax; }
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
                    umax = fmaxf(umax, shm[0][i]);
                    emax = fmaxf(emax, shm[1][i]);
                }
                const int c = pcl[p];
                atomicMax(cm + 3 * c, __float_as_uint(umax));
                atomicMax(cm + 3 * c + 1, __float_as_uint(emax));
                atomicMax(cm + 3 * c + 2, __float_as_uint(Pp.D));
            }
            __syncthreads();
        }
    }
}

// Fixed-point scale of a fallback cluster (deterministic mode): the largest
// power of two 2^k with (max|u| + 64 Dmax max|e|) 2^k < 2^28, as in the
// shared-memory kernel (a converted-back cell above 2^28 in magnitude sets
// IBM_EBIT_FIXEDPOINT).
__device__ __forceinline__ float fb_scale(const unsigned *cm, int c, float *inv) {
    const float range = __uint_as_float(cm[3 * c]) + 64.f * __uint_as_float(cm[3 * c + 2]) * __uint_as_float(cm[3 * c + 1]);
    int ex = 100;
    if (range > 0.f) ex = min(100, max(-100, 27 - (int)ceilf(log2f(range))));
    *inv = ldexpf(1.f, -ex);
    return ldexpf(1.f, ex);
}

// Cell (n = 0..26) of a marker's 3-point stencil, as a linear index of its scene.
__device__ __forceinline__ long long fb_cell(const Stencil<float> &st, const Grid &g, int n) {
    const int cx = n % 3, cy = (n / 3) % 3, cz = n / 9;
    return ((long long)wrapi(st.b[2] - 1 + cz, g.nz) * g.ny + wrapi(st.b[1] - 1 + cy, g.ny)) * g.nx +
           wrapi(st.b[0] - 1 + cx, g.nx);
}

// Once per step, before the fallback iterations (deterministic mode): every
// stencil cell of the fallback markers gets one owner, the first marker to set
// the cell's bit in a grid-wide bitmap; own[moff + l] is the 27-bit mask of
// the cells marker l of the particle owns.  The first conversion clears the
// bits again.
__global__ void __launch_bounds__(kBlock) k_fb_claim(const PInfo *__restrict__ P, const int *__restrict__ plist,
                                                    const int *__restrict__ n_list_d, const double *__restrict__ t64,
                                                    const float *__restrict__ t32, const int32_t *__restrict__ dims,
                                                    const long long *__restrict__ cell_off, unsigned *bits,
                                                    unsigned *__restrict__ own) {
    const int n_list = *n_list_d;
    for (int k = blockIdx.y; k < n_list; k += gridDim.y) {
        const PInfo Pp = P[plist[k]];
        const Grid g = scene_grid(dims, Pp.scene);
        for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < Pp.nl; l += gridDim.x * blockDim.x) {
            Stencil<float> st;
            marker_stencil(Pp, t64 + 3ll * (Pp.toff + l), t32 + 3ll * (Pp.toff + l), st);
            unsigned mine = 0u;
#pragma unroll
            for (int n = 0; n < 27; ++n) {
                const long long gi = cell_off[Pp.scene] + fb_cell(st, g, n);
                const unsigned bit = 1u << (gi & 31);
                if (!(atomicOr(bits + (gi >> 5), bit) & bit)) mine |= 1u << n;
            }
            own[Pp.moff + l] = mine;
        }
    }
}

// Converts the cells owned by the fallback markers (k_fb_claim) to the
// cluster's fixed point (TO) or back, each cell once.  clear != NULL: also
// zeroes the cells' bitmap words (no thread of this launch reads them).
template <bool TO>
__global__ void __launch_bounds__(kBlock) k_fb_convert(const PInfo *__restrict__ P, const int *__restrict__ plist,
                                                      const int *__restrict__ n_list_d, const double *__restrict__ t64,
                                                      const float *__restrict__ t32, const int32_t *__restrict__ dims,
                                                      const long long *__restrict__ cell_off, float *const *uf,
                                                      const int *__restrict__ pcl, const unsigned *__restrict__ cm,
                                                      const unsigned *__restrict__ own, unsigned *clear, int *err) {
    const int n_list = *n_list_d;
    for (int k = blockIdx.y; k < n_list; k += gridDim.y) {
        const int p = plist[k];
        const PInfo Pp = P[p];
        const Grid g = scene_grid(dims, Pp.scene);
        float *u = uf[Pp.scene];
        float inv;
        const float S = fb_scale(cm, pcl[p], &inv);
        for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < Pp.nl; l += gridDim.x * blockDim.x) {
            unsigned mine = own[Pp.moff + l];
            if (!mine) continue;
            Stencil<float> st;
            marker_stencil(Pp, t64 + 3ll * (Pp.toff + l), t32 + 3ll * (Pp.toff + l), st);
            while (mine) {
                const int n = __ffs(mine) - 1;
                mine &= mine - 1u;
                const long long idx = fb_cell(st, g, n);
                if (clear) clear[(cell_off[Pp.scene] + idx) >> 5] = 0u;
                for (int q = 0; q < 3; ++q) {
                    float *c = u + q * g.ncell + idx;
                    if (TO) {
                        *reinterpret_cast<int *>(c) = __float2int_rn(*c * S);
                    } else {
                        const int v = *reinterpret_cast<const int *>(c);
                        if (abs(v) > (1 << 28)) set_err(err, IBM_EBIT_FIXEDPOINT);
                        *c = (float)v * inv;
                    }
                }
            }
        }
    }
}

// Steps 3-4 (Sec. 2.2.2): u += tau f with f = sum_l F_l w D_l, i.e.
// u += scale * sum_l w D_l v_l for v = e (scale 1).  Optional f_out += that / tau.
// FB (deterministic fallback, FP32): the cells hold the cluster's fixed point
// (k_fb_convert) and the contributions are added as rounded integers.
template <typename T, bool FB = false, int K = 3>
__global__ void __launch_bounds__(kBlock) k_plain_spread(
    const PInfo *__restrict__ P, const int *__restrict__ plist, int n_list, const int *__restrict__ n_list_d,
    const double *__restrict__ t64, const float *__restrict__ t32, const int32_t *__restrict__ dims,
    const T *__restrict__ vbuf, T scale, T *const *uf, T *const *ff, T finv, const double *__restrict__ cbuf,
    double *FD, double *TD, const int *__restrict__ pcl = nullptr, const unsigned *__restrict__ cm = nullptr) {
    if (n_list_d) n_list = *n_list_d;
    for (int k = blockIdx.y; k < n_list; k += gridDim.y) {
        const int p = plist ? plist[k] : k;
        const PInfo Pp = P[p];
        const Grid g = scene_grid(dims, Pp.scene);
        T *u = uf[Pp.scene];
        T *f = ff ? ff[Pp.scene] : nullptr;
        if (cbuf && blockIdx.x == 0 && threadIdx.x < 6) {
            // the particle's loads of this iteration: its chunks' sums, in order
            double s = 0.0;
            for (int c = 0; c < (int)gridDim.x; ++c) s += cbuf[(6ll * k) * gridDim.x + 6 * c + threadIdx.x];
            if (threadIdx.x < 3) FD[3 * p + threadIdx.x] += s;
            else TD[3 * p + threadIdx.x - 3] += s;
        }
        for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < Pp.nl; l += gridDim.x * blockDim.x) {
            const double *tt64 = t64 + 3ll * (Pp.toff + l);
            const float *tt32 = t32 + 3ll * (Pp.toff + l);
            Stencil<T, K> S;
            marker_stencil(Pp, tt64, tt32, S);
            const T D = sizeof(T) == 8 ? (T)Pp.D64 : (T)Pp.D;
            T gv[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) gv[q] = scale * D * vbuf[3ll * (Pp.moff + l) + q];
            float fs = 1.f, finv_s = 0.f;
            if (FB) fs = fb_scale(cm, pcl[p], &finv_s);
            int ii[K];
#pragma unroll
            for (int a = 0; a < K; ++a) ii[a] = wrapi(S.b[0] - 1 + a, g.nx);
#pragma unroll
            for (int cz = 0; cz < K; ++cz) {
                const int kk = wrapi(S.b[2] - 1 + cz, g.nz);
#pragma unroll
                for (int cy = 0; cy < K; ++cy) {
                    const int jj = wrapi(S.b[1] - 1 + cy, g.ny);
                    const long long row = ((long long)kk * g.ny + jj) * g.nx;
                    const T wyz = S.w[2][cz] * S.w[1][cy];
#pragma unroll
                    for (int cx = 0; cx < K; ++cx) {
                        const T w = wyz * S.w[0][cx];
                        const long long idx = row + ii[cx];
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            if (FB)
                                atomicAdd(reinterpret_cast<int *>(u + q * g.ncell + idx),
                                          __float2int_rn((float)(w * gv[q]) * fs));
                            else
                                atomicAdd(u + q * g.ncell + idx, w * gv[q]);
                            if (f) atomicAdd(f + q * g.ncell + idx, w * gv[q] * finv);
                        }
                    }
                }
            }
        }
    }
}

// Slip after the loop: eps_l = |U^d - W u^{n_F}| (Sec. 2.2.2); sum of squares
// and maximum over all markers.
template <typename T, int K = 3>
__global__ void __launch_bounds__(kBlock) k_slip(const PInfo *__restrict__ P, int n_p,
                                                 const double *__restrict__ t64, const float *__restrict__ t32,
                                                 const double *__restrict__ up, const double *__restrict__ om,
                                                 const int32_t *__restrict__ dims, T *const *uf, double *acc) {
    __shared__ double sh[1][32];
    __shared__ double shm[32];
    for (int p = blockIdx.x; p < n_p; p += gridDim.x) {
        const PInfo Pp = P[p];
        const Grid g = scene_grid(dims, Pp.scene);
        const T *__restrict__ u = uf[Pp.scene];
        double s2[1] = {0.0};
        double mx = 0.0;
        for (int l = threadIdx.x; l < Pp.nl; l += blockDim.x) {
            const double *tt64 = t64 + 3ll * (Pp.toff + l);
            const float *tt32 = t32 + 3ll * (Pp.toff + l);
            Stencil<T, K> S;
            marker_stencil(Pp, tt64, tt32, S);
            T ud[3], r[3], D;
            marker_kinematics(up, om, p, Pp, tt64, tt32, ud, r, D);
            // evaluated in the path's own precision T; summed over markers in FP64
            T U[3] = {T(0), T(0), T(0)};
            for (int cz = 0; cz < K; ++cz) {
                const int kk = wrapi(S.b[2] - 1 + cz, g.nz);
                for (int cy = 0; cy < K; ++cy) {
                    const int jj = wrapi(S.b[1] - 1 + cy, g.ny);
                    const long long row = ((long long)kk * g.ny + jj) * g.nx;
                    for (int cx = 0; cx < K; ++cx) {
                        const T w = S.w[2][cz] * S.w[1][cy] * S.w[0][cx];
                        const long long idx = row + wrapi(S.b[0] - 1 + cx, g.nx);
                        for (int q = 0; q < 3; ++q) U[q] += w * u[q * g.ncell + idx];
                    }
                }
            }
            T e2 = T(0);
            for (int q = 0; q < 3; ++q) {
                const T e = ud[q] - U[q];
                e2 += e * e;
            }
            s2[0] += (double)e2;
            mx = fmax(mx, sqrt((double)e2));
        }
        mx = warp_max(mx);
        if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = mx;
        block_sum<1>(s2, sh);
        if (threadIdx.x == 0) {
            double m = 0.0;
            for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) m = fmax(m, shm[w]);
            atomicAdd(acc, s2[0]);
            atomic_max_nonneg(acc + 1, m);
        }
        __syncthreads();
    }
}

// Loads in physical units (F_p = sum F dV = (h^3/tau) sum e D) and the
// rigid-body Newton-Euler update of Eq. (basic-particle a-c), F_c = T_c = 0,
// with m_p = rho_p pi d^3/6, I_p = m_p d^2/10.
__global__ void k_finalize(int n_p, const double *FD, const double *TD, double h, double tau,
                           const double *x, const double *up, const double *om, const double *d,
                           const double *rho, int newton_euler, double rho_f, double gx, double gy,
                           double gz, double *Fo, double *To, double *xo, double *uo, double *omo) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_p; p += gridDim.x * blockDim.x) {
        const double s = h * h * h / tau;
        double F[3], T[3];
        for (int c = 0; c < 3; ++c) {
            F[c] = FD[3 * p + c] * s;
            T[c] = TD[3 * p + c] * s;
            Fo[3 * p + c] = F[c];
            To[3 * p + c] = T[c];
        }
        const double g[3] = {gx, gy, gz};
        if (newton_euler) {
            const double dd = d[p], rp = rho[p];
            const double m = rp * IBM_PI * dd * dd * dd / 6.0;
            const double I = m * dd * dd / 10.0;
            const double cf = rp * rho_f / (m * (rp - rho_f));
            const double ct = rp * rho_f / (I * (rp - rho_f));
            for (int c = 0; c < 3; ++c) {
                const double uold = up[3 * p + c];
                const double unew = uold + tau * (cf * (-F[c]) + g[c]);
                uo[3 * p + c] = unew;
                omo[3 * p + c] = om[3 * p + c] + tau * ct * (-T[c]);
                xo[3 * p + c] = x[3 * p + c] + 0.5 * tau * (unew + uold);
            }
        } else {
            for (int c = 0; c < 3; ++c) {
                uo[3 * p + c] = up[3 * p + c];
                omo[3 * p + c] = om[3 * p + c];
                xo[3 * p + c] = x[3 * p + c];
            }
        }
    }
}

template <typename T, int K = 3>
__global__ void k_marker_bases(const PInfo *__restrict__ P, int n_p, const double *t64, const float *t32,
                               int64_t *out) {
    for (int p = blockIdx.x; p < n_p; p += gridDim.x) {
        const PInfo Pp = P[p];
        for (int l = threadIdx.x; l < Pp.nl; l += blockDim.x) {
            Stencil<T, K> S;
            marker_stencil(Pp, t64 + 3ll * (Pp.toff + l), t32 + 3ll * (Pp.toff + l), S);
            for (int c = 0; c < 3; ++c) out[3ll * (Pp.moff + l) + c] = S.b[c];
        }
    }
}

// ------------------------------------------------------------ adjoint

// Forward replay of one iteration for the adjoint: e^m = U^d - W u^{m-1} and
// (grad W u^{m-1}) per marker (9 values, [beta][alpha], physical units).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_bw_fwd(const PInfo *__restrict__ P, int n_p,
                                                   const double *__restrict__ t64, const float *__restrict__ t32,
                                                   const double *__restrict__ up, const double *__restrict__ om,
                                                   const int32_t *__restrict__ dims, T *const *uf, T hinv,
                                                   T *__restrict__ e_out, T *__restrict__ gu_out) {
    for (int p = blockIdx.x; p < n_p; p += gridDim.x) {
        const PInfo Pp = P[p];
        const Grid g = scene_grid(dims, Pp.scene);
        const T *__restrict__ u = uf[Pp.scene];
        for (int l = threadIdx.x; l < Pp.nl; l += blockDim.x) {
            const double *tt64 = t64 + 3ll * (Pp.toff + l);
            const float *tt32 = t32 + 3ll * (Pp.toff + l);
            Stencil<T> S;
            marker_stencil(Pp, tt64, tt32, S);
            T dw[3][3];
            for (int c = 0; c < 3; ++c) phi3_dweights<T>(S.f[c], dw[c]);
            T ud[3], r[3], D;
            marker_kinematics(up, om, p, Pp, tt64, tt32, ud, r, D);
            T U[3] = {0, 0, 0}, G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
            for (int cz = 0; cz < 3; ++cz) {
                const int kk = wrapi(S.b[2] - 1 + cz, g.nz);
                for (int cy = 0; cy < 3; ++cy) {
                    const int jj = wrapi(S.b[1] - 1 + cy, g.ny);
                    const long long row = ((long long)kk * g.ny + jj) * g.nx;
                    for (int cx = 0; cx < 3; ++cx) {
                        const long long idx = row + wrapi(S.b[0] - 1 + cx, g.nx);
                        const T w = S.w[2][cz] * S.w[1][cy] * S.w[0][cx];
                        const T d0 = S.w[2][cz] * S.w[1][cy] * dw[0][cx] * hinv;
                        const T d1 = S.w[2][cz] * dw[1][cy] * S.w[0][cx] * hinv;
                        const T d2 = dw[2][cz] * S.w[1][cy] * S.w[0][cx] * hinv;
                        for (int q = 0; q < 3; ++q) {
                            const T v = u[q * g.ncell + idx];
                            U[q] += w * v;
                            G[0][q] += d0 * v;
                            G[1][q] += d1 * v;
                            G[2][q] += d2 * v;
                        }
                    }
                }
            }
            const long long m = Pp.moff + l;
            for (int q = 0; q < 3; ++q) e_out[3 * m + q] = ud[q] - U[q];
            for (int b = 0; b < 3; ++b)
                for (int q = 0; q < 3; ++q) gu_out[9 * m + 3 * b + q] = G[b][q];
        }
    }
}

// Adjoint of one iteration: with g = dL/du^m,
//   dL/dU^d_l += D (W g)_l,
//   dL/dX_l   += D [ (grad W g)_l^T e^m_l - (grad W u^{m-1})_l^T (W g)_l ],
// and v_l = (W g)_l is stored for g -= W^T D v.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_bw_adj(const PInfo *__restrict__ P, int n_p,
                                                   const double *__restrict__ t64, const float *__restrict__ t32,
                                                   const int32_t *__restrict__ dims, T *const *gf, T hinv,
                                                   const T *__restrict__ e_in, const T *__restrict__ gu_in,
                                                   T *__restrict__ vbuf, double *__restrict__ gmk) {
    for (int p = blockIdx.x; p < n_p; p += gridDim.x) {
        const PInfo Pp = P[p];
        const Grid g = scene_grid(dims, Pp.scene);
        const T *__restrict__ gr = gf[Pp.scene];
        for (int l = threadIdx.x; l < Pp.nl; l += blockDim.x) {
            const double *tt64 = t64 + 3ll * (Pp.toff + l);
            const float *tt32 = t32 + 3ll * (Pp.toff + l);
            Stencil<T> S;
            marker_stencil(Pp, tt64, tt32, S);
            T dw[3][3];
            for (int c = 0; c < 3; ++c) phi3_dweights<T>(S.f[c], dw[c]);
            const T D = sizeof(T) == 8 ? (T)Pp.D64 : (T)Pp.D;
            T Wg[3] = {0, 0, 0}, G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
            for (int cz = 0; cz < 3; ++cz) {
                const int kk = wrapi(S.b[2] - 1 + cz, g.nz);
                for (int cy = 0; cy < 3; ++cy) {
                    const int jj = wrapi(S.b[1] - 1 + cy, g.ny);
                    const long long row = ((long long)kk * g.ny + jj) * g.nx;
                    for (int cx = 0; cx < 3; ++cx) {
                        const long long idx = row + wrapi(S.b[0] - 1 + cx, g.nx);
                        const T w = S.w[2][cz] * S.w[1][cy] * S.w[0][cx];
                        const T d0 = S.w[2][cz] * S.w[1][cy] * dw[0][cx] * hinv;
                        const T d1 = S.w[2][cz] * dw[1][cy] * S.w[0][cx] * hinv;
                        const T d2 = dw[2][cz] * S.w[1][cy] * S.w[0][cx] * hinv;
                        for (int q = 0; q < 3; ++q) {
                            const T v = gr[q * g.ncell + idx];
                            Wg[q] += w * v;
                            G[0][q] += d0 * v;
                            G[1][q] += d1 * v;
                            G[2][q] += d2 * v;
                        }
                    }
                }
            }
            const long long m = Pp.moff + l;
            double *acc = gmk + 6 * m;
            for (int q = 0; q < 3; ++q) {
                acc[q] += (double)(D * Wg[q]);
                vbuf[3 * m + q] = Wg[q];
            }
            for (int b = 0; b < 3; ++b) {
                T s = 0;
                for (int q = 0; q < 3; ++q) s += e_in[3 * m + q] * G[b][q] - Wg[q] * gu_in[9 * m + 3 * b + q];
                acc[3 + b] += (double)(D * s);
            }
        }
    }
}

// Per-particle gradients: dL/du_p = sum dL/dU^d, dL/dw_p = sum r x dL/dU^d,
// dL/dx_p = sum dL/dX_l (FP64).
__global__ void __launch_bounds__(kBlock) k_bw_reduce(const PInfo *__restrict__ P, int n_p,
                                                      const double *__restrict__ t64, const double *gmk,
                                                      double *gU, double *gW, double *gX) {
    __shared__ double sh[9][32];
    for (int p = blockIdx.x; p < n_p; p += gridDim.x) {
        const PInfo Pp = P[p];
        double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int l = threadIdx.x; l < Pp.nl; l += blockDim.x) {
            const double *tt = t64 + 3ll * (Pp.toff + l);
            const double r[3] = {Pp.rphys64 * tt[0], Pp.rphys64 * tt[1], Pp.rphys64 * tt[2]};
            const double *a = gmk + 6ll * (Pp.moff + l);
            acc[0] += a[0]; acc[1] += a[1]; acc[2] += a[2];
            acc[3] += r[1] * a[2] - r[2] * a[1];
            acc[4] += r[2] * a[0] - r[0] * a[2];
            acc[5] += r[0] * a[1] - r[1] * a[0];
            acc[6] += a[3]; acc[7] += a[4]; acc[8] += a[5];
        }
        block_sum<9>(acc, sh);
        if (threadIdx.x == 0) {
            for (int q = 0; q < 3; ++q) {
                if (gU) gU[3 * p + q] = acc[q];
                if (gW) gW[3 * p + q] = acc[3 + q];
                if (gX) gX[3 * p + q] = acc[6 + q];
            }
        }
    }
}

int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 65535ll * 4) g = 65535ll * 4;
    return (int)g;
}

int blocks_for_particles(int n) { return std::max(1, std::min(n, 152 * 16)); }

}  // namespace

// ================================================================= host side

ibm_status ensure_field_ptrs(ibm_ctx *ctx, void *const *u_ptrs, void *const *f_out) {
    const int ns = ctx->cfg.n_scenes;
    if (!ctx->uptr_d || !ctx->fptr_d) {
        // both tables or neither: a failed second allocation releases the first
        void **ud = nullptr, **fd = nullptr;
        CK(ibm_malloc(&ud, ns * sizeof(void *)), "alloc field pointers");
        const cudaError_t e = ibm_malloc(&fd, ns * sizeof(void *));
        if (e != cudaSuccess) {
            cudaFree(ud);
            return ibm_cuda_check(ctx, e, "alloc field pointers");
        }
        if (ctx->uptr_d) cudaFree(ctx->uptr_d);
        if (ctx->fptr_d) cudaFree(ctx->fptr_d);
        ctx->uptr_d = ud;
        ctx->fptr_d = fd;
        ctx->uptr_h.assign(ns, nullptr);
        ctx->fptr_h.assign(ns, nullptr);
    }
    bool du = false, df = false;
    for (int s = 0; s < ns; ++s) {
        if (ctx->uptr_h[s] != u_ptrs[s]) du = true;
        if (f_out && ctx->fptr_h[s] != f_out[s]) df = true;
    }
    if (du) {
        ctx->uptr_h.assign(u_ptrs, u_ptrs + ns);
        CK(cudaMemcpyAsync(ctx->uptr_d, ctx->uptr_h.data(), ns * sizeof(void *), cudaMemcpyHostToDevice,
                           ctx->stream), "copy field pointers");
    }
    if (df) {
        ctx->fptr_h.assign(f_out, f_out + ns);
        CK(cudaMemcpyAsync(ctx->fptr_d, ctx->fptr_h.data(), ns * sizeof(void *), cudaMemcpyHostToDevice,
                           ctx->stream), "copy field pointers");
    }
    if (du || df) CK(cudaStreamSynchronize(ctx->stream), "sync pointer copy");
    return IBM_OK;
}

static ibm_status ensure_ebuf(ibm_ctx *ctx) {
    const long long need = 3 * std::max<long long>(ctx->n_markers, 1) * sizeof(double);
    if (ctx->ebuf_cap < need) {
        if (ctx->ebuf) cudaFree(ctx->ebuf);
        ctx->ebuf = nullptr;
        CK(ibm_malloc(&ctx->ebuf, need), "alloc marker buffer");
        ctx->ebuf_cap = need;
    }
    return IBM_OK;
}

ibm_status launch_setup_particles(ibm_ctx *ctx) {
    const int n = ctx->n_p;
    int *max_d = nullptr;
    long long *tot_d = nullptr;
    CK(ibm_malloc(&max_d, sizeof(int) + sizeof(long long) * 2), "alloc");
    tot_d = reinterpret_cast<long long *>(max_d + 2);
    CK(cudaMemsetAsync(max_d, 0, sizeof(int) + sizeof(long long) * 2, ctx->stream), "memset");
    if (n > 0)
        k_setup<<<grid_for(n, kBlock), kBlock, 0, ctx->stream>>>(
            n, ctx->x, ctx->up, ctx->om, ctx->d, ctx->rho, ctx->scene, ctx->dims_d, ctx->cfg.n_scenes,
            ctx->cfg.h, ctx->cfg.newton_euler, ctx->cfg.rho_f, ctx->nl, max_d, ctx->err_d);
    k_scan_block<<<1, 1024, 0, ctx->stream>>>(ctx->nl, ctx->moff, n, tot_d);
    int maxnl = 0;
    long long total = 0;
    CK(cudaMemcpyAsync(&maxnl, max_d, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "read max");
    CK(cudaMemcpyAsync(&total, tot_d, sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream), "read total");
    CK(cudaStreamSynchronize(ctx->stream), "sync setup");
    cudaFree(max_d);
    ibm_status s = ibm_check_err_word(ctx);
    if (s != IBM_OK) return s;
    if (total > (1ll << 31) - 1) return ibm_fail(ctx, IBM_ERR_CAPACITY, "more than 2^31 markers");
    ctx->n_markers = total;
    ctx->max_nl = maxnl;
    if (n == 0) return IBM_OK;

    // templates for marker counts not seen before
    if (maxnl >= ctx->nl_cap) {
        int cap = std::max(maxnl + 1, 2 * ctx->nl_cap);
        int *nd = nullptr;
        CK(ibm_malloc(&nd, cap * sizeof(int)), "alloc template index");
        ctx->tmpl_of_nl_h.resize(cap, -1);
        CK(cudaMemcpyAsync(nd, ctx->tmpl_of_nl_h.data(), cap * sizeof(int), cudaMemcpyHostToDevice, ctx->stream),
           "copy template index");
        if (ctx->tmpl_of_nl) cudaFree(ctx->tmpl_of_nl);
        ctx->tmpl_of_nl = nd;
        ctx->nl_cap = cap;
    }
    int *flag = nullptr;
    CK(ibm_malloc(&flag, ctx->nl_cap * sizeof(int)), "alloc flags");
    CK(cudaMemsetAsync(flag, 0, ctx->nl_cap * sizeof(int), ctx->stream), "memset flags");
    k_flag_new_nl<<<grid_for(n, kBlock), kBlock, 0, ctx->stream>>>(n, ctx->nl, ctx->tmpl_of_nl, flag);
    std::vector<int> fl(ctx->nl_cap);
    CK(cudaMemcpyAsync(fl.data(), flag, ctx->nl_cap * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
       "read flags");
    CK(cudaStreamSynchronize(ctx->stream), "sync flags");
    cudaFree(flag);
    std::vector<int> lst_nl, lst_off;
    long long used = ctx->tmpl_used;
    for (int v = 1; v < ctx->nl_cap; ++v)
        if (fl[v]) {
            lst_nl.push_back(v);
            lst_off.push_back((int)used);
            used += v;
        }
    if (!lst_nl.empty()) {
        if (used > ctx->tmpl_cap) {
            long long cap = std::max(used, 2 * ctx->tmpl_cap);
            double *n64 = nullptr;
            float *n32 = nullptr;
            CK(ibm_malloc(&n64, 3 * cap * sizeof(double)), "alloc templates");
            const cudaError_t e32 = ibm_malloc(&n32, 3 * cap * sizeof(float));
            if (e32 != cudaSuccess) {
                cudaFree(n64);
                return ibm_cuda_check(ctx, e32, "alloc templates");
            }
            if (ctx->tmpl_used) {
                CK(cudaMemcpyAsync(n64, ctx->tmpl64, 3 * ctx->tmpl_used * sizeof(double), cudaMemcpyDeviceToDevice,
                                   ctx->stream), "copy templates");
                CK(cudaMemcpyAsync(n32, ctx->tmpl32, 3 * ctx->tmpl_used * sizeof(float), cudaMemcpyDeviceToDevice,
                                   ctx->stream), "copy templates");
                CK(cudaStreamSynchronize(ctx->stream), "sync");
            }
            if (ctx->tmpl64) cudaFree(ctx->tmpl64);
            if (ctx->tmpl32) cudaFree(ctx->tmpl32);
            ctx->tmpl64 = n64;
            ctx->tmpl32 = n32;
            ctx->tmpl_cap = cap;
        }
        int *ld = nullptr;
        const int nlst = (int)lst_nl.size();
        CK(ibm_malloc(&ld, 2 * nlst * sizeof(int)), "alloc list");
        CK(cudaMemcpyAsync(ld, lst_nl.data(), nlst * sizeof(int), cudaMemcpyHostToDevice, ctx->stream), "copy");
        CK(cudaMemcpyAsync(ld + nlst, lst_off.data(), nlst * sizeof(int), cudaMemcpyHostToDevice, ctx->stream),
           "copy");
        dim3 grid((ctx->max_nl + 255) / 256, std::min(nlst, 65535));
        k_templates<<<grid, 256, 0, ctx->stream>>>(ld, ld + nlst, nlst, ctx->tmpl64, ctx->tmpl32);
        for (int i = 0; i < nlst; ++i) ctx->tmpl_of_nl_h[lst_nl[i]] = lst_off[i];
        CK(cudaMemcpyAsync(ctx->tmpl_of_nl, ctx->tmpl_of_nl_h.data(), ctx->nl_cap * sizeof(int),
                           cudaMemcpyHostToDevice, ctx->stream), "copy template index");
        CK(cudaStreamSynchronize(ctx->stream), "sync templates");
        cudaFree(ld);
        ctx->tmpl_used = used;
    }
    k_toff<<<grid_for(n, kBlock), kBlock, 0, ctx->stream>>>(n, ctx->nl, ctx->tmpl_of_nl, ctx->toff);
    return ensure_ebuf(ctx);
}

ibm_status launch_pinfo(ibm_ctx *ctx) {
    if (ctx->n_p == 0) return IBM_OK;
    k_pinfo<<<grid_for(ctx->n_p, kBlock), kBlock, 0, ctx->stream>>>(
        ctx->n_p, ctx->x, ctx->up, ctx->om, ctx->d, ctx->scene, ctx->nl, ctx->moff, ctx->toff, ctx->cfg.h,
        ctx->pinfo);
    ctx->launches += 1;
    return IBM_OK;
}

ibm_status launch_marker_bases(ibm_ctx *ctx, int64_t *base_d) {
    const int nb = blocks_for_particles(ctx->n_p);
    if (ctx->cfg.precision == IBM_FP64)
        ctx->cfg.kernel_width == 4
            ? k_marker_bases<double, 4><<<nb, kBlock, 0, ctx->stream>>>(ctx->pinfo, ctx->n_p, ctx->tmpl64,
                                                                        ctx->tmpl32, base_d)
            : k_marker_bases<double><<<nb, kBlock, 0, ctx->stream>>>(ctx->pinfo, ctx->n_p, ctx->tmpl64,
                                                                     ctx->tmpl32, base_d);
    else
        ctx->cfg.kernel_width == 4
            ? k_marker_bases<float, 4><<<nb, kBlock, 0, ctx->stream>>>(ctx->pinfo, ctx->n_p, ctx->tmpl64,
                                                                       ctx->tmpl32, base_d)
            : k_marker_bases<float><<<nb, kBlock, 0, ctx->stream>>>(ctx->pinfo, ctx->n_p, ctx->tmpl64,
                                                                    ctx->tmpl32, base_d);
    return ibm_cuda_check(ctx, cudaGetLastError(), "marker bases");
}

// Grid of the plain kernels: y = particles of the list (grid-stride), x =
// blocks sharing one particle's markers.  About 16 blocks per SM in all; a
// whole bed has enough particles for one block each, a short list (the
// clusters the shared-memory kernel cannot hold, counted on the device) splits
// each particle into chunks of kBlock markers.
static dim3 chunk_grid(const ibm_ctx *ctx, int n_list, bool count_on_device = false) {
    const int gx = count_on_device ? std::max(1, (ctx->max_nl + kBlock - 1) / kBlock) : 1;
    const int gy = std::max(1, std::min(n_list, 152 * 16 / gx));
    return dim3((unsigned)gx, (unsigned)gy);
}

// Buffers of the deterministic fallback: scene cell offsets, the grid-wide
// cell bitmap (kept zero between steps), per-cluster maxima and per-marker
// owned-cell masks.
static ibm_status fb_prepare(ibm_ctx *ctx) {
    if (!ctx->fb_bits) {
        long long off = 0;
        std::vector<long long> offs(ctx->cfg.n_scenes);
        for (int s = 0; s < ctx->cfg.n_scenes; ++s) {
            offs[s] = off;
            off += (long long)ctx->dims_h[3 * s] * ctx->dims_h[3 * s + 1] * ctx->dims_h[3 * s + 2];
        }
        const size_t words = (size_t)(off + 31) / 32 + 1;
        if (ctx->cell_off_d) cudaFree(ctx->cell_off_d);   // left by an earlier failed attempt
        ctx->cell_off_d = nullptr;
        CK(ibm_malloc(&ctx->cell_off_d, offs.size() * sizeof(long long)), "alloc scene offsets");
        CK(cudaMemcpy(ctx->cell_off_d, offs.data(), offs.size() * sizeof(long long), cudaMemcpyHostToDevice),
           "copy scene offsets");
        CK(ibm_malloc(&ctx->fb_bits, words * sizeof(unsigned)), "alloc cell bitmap");
        CK(cudaMemset(ctx->fb_bits, 0, words * sizeof(unsigned)), "zero cell bitmap");
    }
    if (ctx->fb_cm_cap < ctx->cap_p) {
        if (ctx->fb_cm) cudaFree(ctx->fb_cm);
        ctx->fb_cm = nullptr;
        ctx->fb_cm_cap = 0;
        CK(ibm_malloc(&ctx->fb_cm, 3 * (size_t)ctx->cap_p * sizeof(unsigned)), "alloc cluster maxima");
        ctx->fb_cm_cap = ctx->cap_p;
    }
    if (ctx->fb_own_cap < ctx->n_markers) {
        if (ctx->fb_own) cudaFree(ctx->fb_own);
        ctx->fb_own = nullptr;
        ctx->fb_own_cap = 0;
        CK(ibm_malloc(&ctx->fb_own, (size_t)ctx->n_markers * sizeof(unsigned)), "alloc owned-cell masks");
        ctx->fb_own_cap = ctx->n_markers;
    }
    return IBM_OK;
}

// One plain iteration over the particles in plist (all when plist == NULL).
// pcl (FP32 list only): cluster of each particle; spreading then runs in the
// deterministic fixed point of the cluster (interpolate with the maxima,
// convert the cells claimed by k_fb_claim, integer spreading, convert back);
// first: the first iteration of the step, whose conversion clears the bitmap.
// Per-(particle, chunk) load sums of the plain kernels for a list of n_list.
static ibm_status ensure_cbuf(ibm_ctx *ctx, int n_list, bool count_on_device) {
    const dim3 grid = chunk_grid(ctx, n_list, count_on_device);
    const size_t need = (size_t)std::max(1, n_list) * grid.x * 6 * sizeof(double);
    if (ctx->cbuf_cap < need) {
        if (ctx->cbuf) cudaFree(ctx->cbuf);
        ctx->cbuf = nullptr;
        ctx->cbuf_cap = 0;
        CK(ibm_malloc(&ctx->cbuf, need), "alloc chunk sums");
        ctx->cbuf_cap = need;
    }
    return IBM_OK;
}

template <typename T>
static ibm_status plain_iteration(ibm_ctx *ctx, const int *plist, int n_list, const int *n_list_d, double tau,
                                  bool with_f, const int *pcl = nullptr, bool first = false) {
    const dim3 grid = chunk_grid(ctx, n_list, n_list_d != nullptr);
    ibm_status cs = ensure_cbuf(ctx, n_list, n_list_d != nullptr);
    if (cs != IBM_OK) return cs;
    T *const *uf = reinterpret_cast<T *const *>(ctx->uptr_d);
    T *const *ff = with_f ? reinterpret_cast<T *const *>(ctx->fptr_d) : nullptr;
    if (pcl && sizeof(T) == 4) {
        float *const *u32 = reinterpret_cast<float *const *>(ctx->uptr_d);
        float *const *f32 = with_f ? reinterpret_cast<float *const *>(ctx->fptr_d) : nullptr;
        CK(cudaMemsetAsync(ctx->fb_cm, 0, 3 * (size_t)ctx->cap_p * sizeof(unsigned), ctx->stream), "zero maxima");
        k_plain_interp<float, true><<<grid, kBlock, 0, ctx->stream>>>(
            ctx->pinfo, plist, n_list, n_list_d, ctx->tmpl64, ctx->tmpl32, ctx->up, ctx->om, ctx->dims_d, u32,
            reinterpret_cast<float *>(ctx->ebuf), ctx->cbuf, pcl, ctx->fb_cm, contact_bits(ctx));
        k_fb_convert<true><<<grid, kBlock, 0, ctx->stream>>>(ctx->pinfo, plist, n_list_d, ctx->tmpl64, ctx->tmpl32,
                                                             ctx->dims_d, ctx->cell_off_d, u32, pcl, ctx->fb_cm,
                                                             ctx->fb_own, first ? ctx->fb_bits : nullptr, ctx->err_d);
        k_plain_spread<float, true><<<grid, kBlock, 0, ctx->stream>>>(
            ctx->pinfo, plist, n_list, n_list_d, ctx->tmpl64, ctx->tmpl32, ctx->dims_d,
            reinterpret_cast<const float *>(ctx->ebuf), 1.f, u32, f32, (float)(1.0 / tau), ctx->cbuf, ctx->FD,
            ctx->TD, pcl, ctx->fb_cm);
        k_fb_convert<false><<<grid, kBlock, 0, ctx->stream>>>(ctx->pinfo, plist, n_list_d, ctx->tmpl64, ctx->tmpl32,
                                                              ctx->dims_d, ctx->cell_off_d, u32, pcl, ctx->fb_cm,
                                                              ctx->fb_own, nullptr, ctx->err_d);
        ctx->launches += 4;
        return IBM_OK;
    }
    // markers left out near contact (global marker bits, so any particle list)
    const unsigned *dis = contact_bits(ctx);
    if (ctx->cfg.kernel_width == 4) {
        k_plain_interp<T, false, 4><<<grid, kBlock, 0, ctx->stream>>>(
            ctx->pinfo, plist, n_list, n_list_d, ctx->tmpl64, ctx->tmpl32, ctx->up, ctx->om, ctx->dims_d, uf,
            reinterpret_cast<T *>(ctx->ebuf), ctx->cbuf, nullptr, nullptr, dis);
        k_plain_spread<T, false, 4><<<grid, kBlock, 0, ctx->stream>>>(
            ctx->pinfo, plist, n_list, n_list_d, ctx->tmpl64, ctx->tmpl32, ctx->dims_d,
            reinterpret_cast<const T *>(ctx->ebuf), T(1), uf, ff, T(1.0 / tau), ctx->cbuf, ctx->FD, ctx->TD);
    } else {
        k_plain_interp<T><<<grid, kBlock, 0, ctx->stream>>>(ctx->pinfo, plist, n_list, n_list_d, ctx->tmpl64,
                                                            ctx->tmpl32, ctx->up, ctx->om, ctx->dims_d, uf,
                                                            reinterpret_cast<T *>(ctx->ebuf), ctx->cbuf, nullptr,
                                                            nullptr, dis);
        k_plain_spread<T><<<grid, kBlock, 0, ctx->stream>>>(ctx->pinfo, plist, n_list, n_list_d, ctx->tmpl64,
                                                            ctx->tmpl32, ctx->dims_d,
                                                            reinterpret_cast<const T *>(ctx->ebuf), T(1), uf, ff,
                                                            T(1.0 / tau), ctx->cbuf, ctx->FD, ctx->TD);
    }
    ctx->launches += 2;
    return IBM_OK;
}

// FP32 plain iterations over a particle list whose length is n_list, or, when
// n_list_d is given, the device value *n_list_d (at most n_list).  pcl != NULL:
// deterministic fixed-point spreading per cluster.
ibm_status plain_iterations_f32(ibm_ctx *ctx, const int *plist, int n_list, const int *n_list_d, double tau,
                                bool with_f, int n_it, const int *pcl) {
    if (pcl && n_it > 0) {
        // every allocation of the iterations happens before the claim: the claim
        // leaves cell bits set that only the first conversion clears, so no
        // error may return between the two
        ibm_status st = fb_prepare(ctx);
        if (st == IBM_OK) st = ensure_cbuf(ctx, n_list, n_list_d != nullptr);
        if (st != IBM_OK) return st;
        k_fb_claim<<<chunk_grid(ctx, n_list, true), kBlock, 0, ctx->stream>>>(
            ctx->pinfo, plist, n_list_d, ctx->tmpl64, ctx->tmpl32, ctx->dims_d, ctx->cell_off_d, ctx->fb_bits,
            ctx->fb_own);
        ctx->launches += 1;
    }
    for (int it = 0; it < n_it; ++it) {
        const ibm_status st = plain_iteration<float>(ctx, plist, n_list, n_list_d, tau, with_f, pcl, it == 0);
        if (st != IBM_OK) return st;
    }
    return ibm_cuda_check(ctx, cudaGetLastError(), "plain iteration");
}

ibm_status plain_forcing_step(ibm_ctx *ctx, void *const *u_ptrs, double tau, void *const *f_out) {
    ibm_status s = ensure_field_ptrs(ctx, u_ptrs, f_out);
    if (s != IBM_OK) return s;
    if (ctx->ct_enable) {
        s = contact_exclusion(ctx);
        if (s != IBM_OK) return s;
    }
    prof_begin(ctx);
    for (int it = 0; it < ctx->cfg.n_forcing; ++it) {
        s = ctx->cfg.precision == IBM_FP64 ? plain_iteration<double>(ctx, nullptr, ctx->n_p, nullptr, tau, f_out != nullptr)
                                           : plain_iteration<float>(ctx, nullptr, ctx->n_p, nullptr, tau, f_out != nullptr);
        if (s != IBM_OK) return s;
    }
    prof_end(ctx);
    return ibm_cuda_check(ctx, cudaGetLastError(), "plain forcing step");
}

ibm_status plain_slip(ibm_ctx *ctx, void *const *u_ptrs) {
    ibm_status s = ensure_field_ptrs(ctx, u_ptrs, nullptr);
    if (s != IBM_OK) return s;
    const int nb = blocks_for_particles(ctx->n_p);
    if (ctx->cfg.precision == IBM_FP64)
        ctx->cfg.kernel_width == 4
            ? k_slip<double, 4><<<nb, kBlock, 0, ctx->stream>>>(ctx->pinfo, ctx->n_p, ctx->tmpl64, ctx->tmpl32,
                                                                ctx->up, ctx->om, ctx->dims_d,
                                                                reinterpret_cast<double *const *>(ctx->uptr_d),
                                                                ctx->slip_acc)
            : k_slip<double><<<nb, kBlock, 0, ctx->stream>>>(ctx->pinfo, ctx->n_p, ctx->tmpl64, ctx->tmpl32,
                                                             ctx->up, ctx->om, ctx->dims_d,
                                                             reinterpret_cast<double *const *>(ctx->uptr_d),
                                                             ctx->slip_acc);
    else
        ctx->cfg.kernel_width == 4
            ? k_slip<float, 4><<<nb, kBlock, 0, ctx->stream>>>(ctx->pinfo, ctx->n_p, ctx->tmpl64, ctx->tmpl32,
                                                               ctx->up, ctx->om, ctx->dims_d,
                                                               reinterpret_cast<float *const *>(ctx->uptr_d),
                                                               ctx->slip_acc)
            : k_slip<float><<<nb, kBlock, 0, ctx->stream>>>(ctx->pinfo, ctx->n_p, ctx->tmpl64, ctx->tmpl32,
                                                            ctx->up, ctx->om, ctx->dims_d,
                                                            reinterpret_cast<float *const *>(ctx->uptr_d),
                                                            ctx->slip_acc);
    return ibm_cuda_check(ctx, cudaGetLastError(), "slip");
}

ibm_status finalize_particles(ibm_ctx *ctx, double tau) {
    if (ctx->n_p == 0) return IBM_OK;
    const ibm_config &c = ctx->cfg;
    k_finalize<<<grid_for(ctx->n_p, kBlock), kBlock, 0, ctx->stream>>>(
        ctx->n_p, ctx->FD, ctx->TD, c.h, tau, ctx->x, ctx->up, ctx->om, ctx->d, ctx->rho, c.newton_euler, c.rho_f,
        c.g[0], c.g[1], c.g[2], ctx->Fout, ctx->Tout, ctx->x_new, ctx->u_new, ctx->om_new);
    ctx->launches += 1;
    return ibm_cuda_check(ctx, cudaGetLastError(), "finalize");
}

template <typename T>
static ibm_status backward_impl(ibm_ctx *ctx, void *const *grad_u_out, void *const *grad_u_in, double *gU,
                                double *gOmega, double *gX) {
    const int ns = ctx->cfg.n_scenes, nf = ctx->cfg.n_forcing;
    const long long nm = std::max<long long>(ctx->n_markers, 1);
    const long long need = (long long)nf * nm;
    if (ctx->hist_cap < need) {
        if (ctx->e_hist) cudaFree(ctx->e_hist);
        if (ctx->gu_hist) cudaFree(ctx->gu_hist);
        if (ctx->gmk) cudaFree(ctx->gmk);
        ctx->e_hist = ctx->gu_hist = ctx->gmk = nullptr;
        CK(ibm_malloc(&ctx->e_hist, 3 * need * sizeof(double)), "alloc adjoint history");
        CK(ibm_malloc(&ctx->gu_hist, 9 * need * sizeof(double)), "alloc adjoint history");
        CK(ibm_malloc(&ctx->gmk, 6 * nm * sizeof(double)), "alloc adjoint accumulators");
        ctx->hist_cap = need;
    }
    ctx->bw_work.resize(ns, nullptr);
    std::vector<void *> work(ns);
    for (int s = 0; s < ns; ++s) {
        const size_t n = 3ull * ctx->dims_h[3 * s] * ctx->dims_h[3 * s + 1] * ctx->dims_h[3 * s + 2];
        if (!ctx->bw_work[s]) CK(ibm_malloc(&ctx->bw_work[s], n * sizeof(T)), "alloc adjoint work field");
        CK(cudaMemcpyAsync(ctx->bw_work[s], ctx->u0_saved[s], n * sizeof(T), cudaMemcpyDeviceToDevice, ctx->stream),
           "copy u0");
        work[s] = ctx->bw_work[s];
        if (grad_u_in[s] != grad_u_out[s])
            CK(cudaMemcpyAsync(grad_u_in[s], grad_u_out[s], n * sizeof(T), cudaMemcpyDeviceToDevice, ctx->stream),
               "copy gradient");
    }
    ibm_status st = launch_pinfo(ctx);
    if (st != IBM_OK) return st;
    const int nb = blocks_for_particles(ctx->n_p);
    const T hinv = T(1.0 / ctx->cfg.h);
    T *eh = reinterpret_cast<T *>(ctx->e_hist), *gh = reinterpret_cast<T *>(ctx->gu_hist);
    // forward replay from u^0
    st = ensure_field_ptrs(ctx, work.data(), nullptr);
    if (st != IBM_OK) return st;
    for (int it = 0; it < nf; ++it) {
        T *e_m = eh + 3 * nm * it, *g_m = gh + 9 * nm * it;
        k_bw_fwd<T><<<nb, kBlock, 0, ctx->stream>>>(ctx->pinfo, ctx->n_p, ctx->tmpl64, ctx->tmpl32, ctx->up, ctx->om,
                                                    ctx->dims_d, reinterpret_cast<T *const *>(ctx->uptr_d), hinv,
                                                    e_m, g_m);
        k_plain_spread<T><<<chunk_grid(ctx, ctx->n_p), kBlock, 0, ctx->stream>>>(
            ctx->pinfo, nullptr, ctx->n_p, nullptr, ctx->tmpl64, ctx->tmpl32, ctx->dims_d, e_m, T(1),
            reinterpret_cast<T *const *>(ctx->uptr_d), nullptr, T(0), nullptr, nullptr, nullptr);
    }
    // reverse sweep on the gradient field
    st = ensure_field_ptrs(ctx, grad_u_in, nullptr);
    if (st != IBM_OK) return st;
    CK(cudaMemsetAsync(ctx->gmk, 0, 6 * nm * sizeof(double), ctx->stream), "zero adjoint accumulators");
    for (int it = nf - 1; it >= 0; --it) {
        const T *e_m = eh + 3 * nm * it, *g_m = gh + 9 * nm * it;
        k_bw_adj<T><<<nb, kBlock, 0, ctx->stream>>>(ctx->pinfo, ctx->n_p, ctx->tmpl64, ctx->tmpl32, ctx->dims_d,
                                                    reinterpret_cast<T *const *>(ctx->uptr_d), hinv, e_m, g_m,
                                                    reinterpret_cast<T *>(ctx->ebuf), reinterpret_cast<double *>(ctx->gmk));
        k_plain_spread<T><<<chunk_grid(ctx, ctx->n_p), kBlock, 0, ctx->stream>>>(
            ctx->pinfo, nullptr, ctx->n_p, nullptr, ctx->tmpl64, ctx->tmpl32, ctx->dims_d,
            reinterpret_cast<const T *>(ctx->ebuf), T(-1), reinterpret_cast<T *const *>(ctx->uptr_d), nullptr, T(0),
            nullptr, nullptr, nullptr);
    }
    k_bw_reduce<<<nb, kBlock, 0, ctx->stream>>>(ctx->pinfo, ctx->n_p, ctx->tmpl64,
                                                reinterpret_cast<const double *>(ctx->gmk), gU, gOmega, gX);
    return ibm_cuda_check(ctx, cudaGetLastError(), "backward");
}

ibm_status plain_backward(ibm_ctx *ctx, void *const *grad_u_out, void *const *grad_u_in, double *gU,
                          double *gOmega, double *gX) {
    if (ctx->n_p == 0) return IBM_OK;
    if (ctx->cfg.precision == IBM_FP64) return backward_impl<double>(ctx, grad_u_out, grad_u_in, gU, gOmega, gX);
    return backward_impl<float>(ctx, grad_u_out, grad_u_in, gU, gOmega, gX);
}
