// Fluid inertia inside each particle, Sec. 2.2.9: midpoint quadrature over the
// cells the particle occupies, weighted by a level-set volume fraction,
//   Iu_p = sum_c alpha_c h^3 u_c,   Ir_p = sum_c alpha_c h^3 (r_c x u_c),   V_p = sum_c alpha_c h^3,
//   alpha_c = sum_m -phi_m H(-phi_m) / sum_m |phi_m|   over the 8 corners of cell c,
// with phi_m = |x_m - x_p| - d_p/2 the signed distance of corner m to the
// sphere's surface (reading: the paper calls it the distance to the centre,
// which is never negative and would make alpha vanish) and r_c the cell centre
// minus x_p.  Rate-of-change terms of the particle equations follow from two
// evaluations of these integrals (the direct form that avoids the rigid-body
// singularity at rho_p = rho_f).
//
// One block per particle.  Along a grid row (fixed y, z) the cells with
// alpha > 0, those with a corner strictly inside the sphere, lie in one x-run
// whose ends follow in closed form from the distance of the row's nearest
// corner line to the centre.  The block computes the run of every row of the
// particle's box, flattens the runs with a block-wide prefix sum, and gives
// consecutive threads consecutive cells of the flattened list, so that the
// loads of a warp cover a few contiguous row segments of u (whole 32-byte
// sectors) and no thread evaluates a cell that cannot contribute.  A thread
// finds its row from a table of the row holding every 32nd cell (no integer
// division) and keeps two cells in flight.  Each lane evaluates the four
// corners of its cell's lower x-face; the upper face comes from the next lane,
// which holds the next cell of the same row except at a row's end.  Boxes with
// more rows than the shared-memory table holds are taken in chunks of whole
// rows.  FP32 fields: per-thread sums in FP32, the block sum in FP64; FP64
// fields sum in FP64 throughout.  Per particle the result is written once,
// without atomics, so it is bit-reproducible.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "ibm_device.cuh"
#include "ibm_internal.h"

#define CK(call, what)                                                  \
    do {                                                                \
        const ibm_status ck_s = ibm_cuda_check(ctx, (call), (what));    \
        if (ck_s != IBM_OK) return ck_s;                                \
    } while (0)

namespace {

constexpr int kInBlock = 128;
constexpr int kRowCap = 768;          // rows of the run table (27 x 27 boxes of D = 24h fit)
constexpr int kRowsPerThread = kRowCap / kInBlock;
constexpr int kChunkCap = 512;        // 32-cell chunks with a start-row entry (16K cells)

// Square root and quotient of the level-set fraction: FP64 exact; FP32 the
// hardware approximations (relative error of order 2^-23, below the FP32
// rounding of phi = |x| - a itself).
__device__ __forceinline__ double lsqrt(double v) { return sqrt(v); }
__device__ __forceinline__ float lsqrt(float v) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ double ldiv(double a, double b) { return a / b; }
__device__ __forceinline__ float ldiv(float a, float b) { return __fdividef(a, b); }

template <typename T>
__global__ void __launch_bounds__(kInBlock, sizeof(T) == 4 ? 10 : 4)
    k_inertia(int n_p, const PInfo *__restrict__ P, const int32_t *__restrict__ dims, const T *const *uf, double h,
              double *__restrict__ out) {
    __shared__ int s_pre[kRowCap + 1];
    __shared__ short s_x0[kRowCap], s_iy[kRowCap], s_iz[kRowCap];
    __shared__ short s_crow[kChunkCap];
    __shared__ int s_scan[32], s_tot;
    __shared__ double sh[7][kInBlock / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int p = blockIdx.x; p < n_p; p += gridDim.x) {
        const PInfo &Pp = P[p];
        const int nx = dims[3 * Pp.scene], ny = dims[3 * Pp.scene + 1], nz = dims[3 * Pp.scene + 2];
        const long long ncell = (long long)nx * ny * nz;
        const T *__restrict__ u0 = uf[Pp.scene];
        const T *__restrict__ u1 = u0 + ncell;
        const T *__restrict__ u2 = u1 + ncell;
        const double a = Pp.a;
        int lo[3], ext[3];
        for (int c = 0; c < 3; ++c) {
            lo[c] = (int)floor(Pp.xi[c] - a) - 1;
            ext[c] = (int)floor(Pp.xi[c] + a) + 1 - lo[c] + 1;
        }
        // the box origin taken into the period once; a box is at most one period wide
        const int wx0 = wrapi(lo[0], nx), wy0 = wrapi(lo[1], ny), wz0 = wrapi(lo[2], nz);
        // cell-centre offsets relative to x_p of the box's first cell (grid units)
        const T ox = (T)((double)lo[0] + 0.5 - Pp.xi[0]);
        const T oy = (T)((double)lo[1] + 0.5 - Pp.xi[1]);
        const T oz = (T)((double)lo[2] + 0.5 - Pp.xi[2]);
        const T at = (T)a;
        T s[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
        const int nrows = ext[1] * ext[2];
        for (int r0 = 0; r0 < nrows; r0 += kRowCap) {
            const int nr = min(kRowCap, nrows - r0);
            // x-run of each row: columns whose nearest corner, ||cx| - 1/2| away in
            // x from the row's nearest corner line, can lie inside; a relative
            // margin of 1e-4 keeps the run inclusive (the corners decide)
            int len[kRowsPerThread], sum = 0;
#pragma unroll
            for (int k = 0; k < kRowsPerThread; ++k) {
                const int i = tid * kRowsPerThread + k;
                len[k] = 0;
                if (i < nr) {
                    const int r = r0 + i;
                    const int iz = r / ext[1], iy = r - iz * ext[1];   // once per row
                    const T cy = fabs(oy + (T)iy) - T(0.5), cz = fabs(oz + (T)iz) - T(0.5);
                    const T dn = at * at - cy * cy - cz * cz;
                    int x0 = 0, x1 = -1;
                    if (dn > T(-1e-4) * at * at) {
                        const T B = sqrt(fmax(dn, T(0))) + T(0.5) + T(1e-4) * at;
                        // columns with |ox + ix| < B
                        x0 = max(0, (int)floor(-B - ox) + 1);
                        x1 = min(ext[0] - 1, (int)ceil(B - ox) - 1);
                    }
                    len[k] = max(0, x1 - x0 + 1);
                    s_x0[i] = (short)x0;
                    s_iy[i] = (short)iy;
                    s_iz[i] = (short)iz;
                }
                sum += len[k];
            }
            // block-wide exclusive prefix of the run lengths
            int x = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_scan[wid] = x;
            __syncthreads();
            if (tid == 0) {
                int acc = 0;
                for (int w = 0; w < kInBlock / 32; ++w) {
                    const int v = s_scan[w];
                    s_scan[w] = acc;
                    acc += v;
                }
                s_tot = acc;
            }
            __syncthreads();
            {
                int run = s_scan[wid] + x - sum;
#pragma unroll
                for (int k = 0; k < kRowsPerThread; ++k) {
                    const int i = tid * kRowsPerThread + k;
                    if (i < nr) s_pre[i] = run;
                    run += len[k];
                }
            }
            if (tid == 0) s_pre[nr] = s_tot;
            __syncthreads();
            const int total = s_tot;
            // start row of every 32-cell chunk (the row holding cell 32k)
            const bool chunked = total <= 32 * kChunkCap;
            if (chunked)
                for (int i = tid; i < nr; i += kInBlock) {
                    const int c0 = s_pre[i], c1 = s_pre[i + 1];
                    for (int k = (c0 + 31) >> 5; 32 * k < c1; ++k) s_crow[k] = (short)i;
                }
            __syncthreads();
            // consecutive threads take consecutive cells of the runs (the cells of a
            // warp are whole 32-cell chunks); the loop bound is uniform per warp
            for (int t0 = tid; t0 < total + lane; t0 += 2 * kInBlock) {
                T al[2], cx[2], cy[2], cz[2];
                long long idx[2];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int t = t0 + j * kInBlock;
                    const bool valid = t < total;
                    int r = 0;
                    if (valid) {
                        if (chunked) {
                            r = s_crow[t >> 5];
                            while (s_pre[r + 1] <= t) ++r;
                        } else {
                            int lo_r = 0, hi_r = nr - 1;   // last row with s_pre <= t
                            while (lo_r < hi_r) {
                                const int mid = (lo_r + hi_r + 1) >> 1;
                                if (s_pre[mid] <= t) lo_r = mid;
                                else hi_r = mid - 1;
                            }
                            r = lo_r;
                        }
                    }
                    const int ix = valid ? s_x0[r] + (t - s_pre[r]) : 0;
                    const int iy = valid ? s_iy[r] : 0, iz = valid ? s_iz[r] : 0;
                    cx[j] = ox + (T)ix;
                    cy[j] = oy + (T)iy;
                    cz[j] = oz + (T)iz;
                    // signed distances of the four corners of the lower x-face
                    const T xl = cx[j] - T(0.5);
                    const T ym = cy[j] - T(0.5), yp = cy[j] + T(0.5), zm = cz[j] - T(0.5), zp = cz[j] + T(0.5);
                    const T yz[4] = {ym * ym + zm * zm, yp * yp + zm * zm, ym * ym + zp * zp, yp * yp + zp * zp};
                    T ph[8];
#pragma unroll
                    for (int k = 0; k < 4; ++k) ph[k] = lsqrt(xl * xl + yz[k]) - at;
                    // upper x-face: from the next lane when it holds the next cell of this row
                    const int rn = __shfl_down_sync(0xffffffffu, valid ? r : -1, 1);
                    const bool own = !(lane < 31 && rn == r && valid);
#pragma unroll
                    for (int k = 0; k < 4; ++k) ph[4 + k] = __shfl_down_sync(0xffffffffu, ph[k], 1);
                    if (own) {
                        const T xu = cx[j] + T(0.5);
#pragma unroll
                        for (int k = 0; k < 4; ++k) ph[4 + k] = lsqrt(xu * xu + yz[k]) - at;
                    }
                    T num = T(0), den = T(0);
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        if (ph[k] <= T(0)) num -= ph[k];
                        den += fabs(ph[k]);
                    }
                    // alpha = 1 exactly when every corner is inside (num == den)
                    al[j] = !valid || !(num > T(0)) ? T(0) : (num == den ? T(1) : ldiv(num, den));
                    int gx = wx0 + ix, gy = wy0 + iy, gz = wz0 + iz;
                    if (gx >= nx) gx -= nx;
                    if (gy >= ny) gy -= ny;
                    if (gz >= nz) gz -= nz;
                    idx[j] = ((long long)gz * ny + gy) * nx + gx;
                }
                T v[2][3];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const bool ld = al[j] != T(0);
                    v[j][0] = ld ? u0[idx[j]] : T(0);
                    v[j][1] = ld ? u1[idx[j]] : T(0);
                    v[j][2] = ld ? u2[idx[j]] : T(0);
                }
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const T w = al[j];
                    s[0] += w * v[j][0];
                    s[1] += w * v[j][1];
                    s[2] += w * v[j][2];
                    s[3] += w * (cy[j] * v[j][2] - cz[j] * v[j][1]);
                    s[4] += w * (cz[j] * v[j][0] - cx[j] * v[j][2]);
                    s[5] += w * (cx[j] * v[j][1] - cy[j] * v[j][0]);
                    s[6] += w;
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            const double v = warp_sum((double)s[k]);
            if (lane == 0) sh[k][wid] = v;
        }
        __syncthreads();
        if (tid < 7) {
            double v = 0.0;
            for (int w = 0; w < kInBlock / 32; ++w) v += sh[tid][w];
            const double h3 = h * h * h;
            // arms are in grid units: r x u carries one more factor h
            out[7ll * p + tid] = v * (tid >= 3 && tid < 6 ? h3 * h : h3);
        }
        __syncthreads();
    }
}

}  // namespace

extern "C" ibm_status ibm_particle_inertia(ibm_ctx *ctx, void *const *u_ptrs, double *Iu, double *Ir, double *V,
                                           int on_device) {
    if (!ctx || !u_ptrs) return IBM_ERR_INVALID_ARG;
    const int ns = ctx->cfg.n_scenes;
    for (int s = 0; s < ns; ++s)
        if (!u_ptrs[s]) return IBM_ERR_INVALID_ARG;
    if (ctx->n_p == 0) return IBM_OK;
    // particle records (centres in grid units, radii) of the current particles
    ibm_status st = launch_pinfo(ctx);
    if (st != IBM_OK) return st;
    if (!ctx->in_ptr) CK(ibm_malloc(&ctx->in_ptr, ns * sizeof(void *)), "alloc field pointers");
    if (ctx->in_cap < ctx->cap_p) {
        if (ctx->in_buf) cudaFree(ctx->in_buf);
        ctx->in_buf = nullptr;
        ctx->in_cap = 0;
        CK(ibm_malloc(&ctx->in_buf, 7ll * ctx->cap_p * sizeof(double)), "alloc inertia sums");
        ctx->in_cap = ctx->cap_p;
    }
    // the device pointer table is refreshed only when the pointers change (a copy
    // from pageable memory would wait for the stream); the host vector stays alive
    if (ctx->in_ptr_h.size() != (size_t)ns || !std::equal(ctx->in_ptr_h.begin(), ctx->in_ptr_h.end(), u_ptrs)) {
        ctx->in_ptr_h.assign(u_ptrs, u_ptrs + ns);
        CK(cudaMemcpyAsync(ctx->in_ptr, ctx->in_ptr_h.data(), ns * sizeof(void *), cudaMemcpyHostToDevice,
                           ctx->stream), "copy field pointers");
    }
    const int grid = std::min(ctx->n_p, 152 * 16);   // grid-stride over particles
    if (ctx->cfg.precision == IBM_FP64)
        k_inertia<double><<<grid, kInBlock, 0, ctx->stream>>>(
            ctx->n_p, ctx->pinfo, ctx->dims_d, reinterpret_cast<const double *const *>(ctx->in_ptr), ctx->cfg.h,
            ctx->in_buf);
    else
        k_inertia<float><<<grid, kInBlock, 0, ctx->stream>>>(
            ctx->n_p, ctx->pinfo, ctx->dims_d, reinterpret_cast<const float *const *>(ctx->in_ptr), ctx->cfg.h,
            ctx->in_buf);
    CK(cudaGetLastError(), "particle inertia");
    const size_t n = (size_t)ctx->n_p;
    std::vector<double> host;
    const double *src = ctx->in_buf;
    if (!on_device) {
        host.resize(7 * n);
        CK(cudaMemcpyAsync(host.data(), ctx->in_buf, 7 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
           "copy inertia sums");
        CK(cudaStreamSynchronize(ctx->stream), "particle inertia");
        for (size_t p = 0; p < n; ++p)
            for (int c = 0; c < 3; ++c) {
                if (Iu) Iu[3 * p + c] = host[7 * p + c];
                if (Ir) Ir[3 * p + c] = host[7 * p + 3 + c];
            }
        if (V)
            for (size_t p = 0; p < n; ++p) V[p] = host[7 * p + 6];
        return IBM_OK;
    }
    // device destinations: strided copies out of the [n_p][7] sums
    if (Iu) CK(cudaMemcpy2DAsync(Iu, 3 * sizeof(double), src, 7 * sizeof(double), 3 * sizeof(double), n,
                                 cudaMemcpyDeviceToDevice, ctx->stream), "copy Iu");
    if (Ir) CK(cudaMemcpy2DAsync(Ir, 3 * sizeof(double), src + 3, 7 * sizeof(double), 3 * sizeof(double), n,
                                 cudaMemcpyDeviceToDevice, ctx->stream), "copy Ir");
    if (V) CK(cudaMemcpy2DAsync(V, sizeof(double), src + 6, 7 * sizeof(double), sizeof(double), n,
                                cudaMemcpyDeviceToDevice, ctx->stream), "copy V");
    return IBM_OK;
}
