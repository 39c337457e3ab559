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
// One block per particle walks the box floor(x_p/h - a) - 1 .. floor(x_p/h + a) + 1
// per axis, one thread per cell, x fastest, so a warp reads contiguous row
// segments of u.  A cell
// whose centre lies more than sqrt(3)/2 inside (outside) the surface has all
// corners inside (outside): alpha = 1 (0, and u is not read); only the cells
// cut by the surface evaluate the eight corners.  FP32 fields: per-thread sums
// in FP32 (at most a few dozen cells each), the block sum in FP64; FP64 fields
// sum in FP64 throughout.  Per particle the result is written once, without
// atomics, so it is bit-reproducible.
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

constexpr int kInBlock = 256;

template <typename T>
__global__ void __launch_bounds__(kInBlock) k_inertia(int n_p, const PInfo *__restrict__ P,
                                                     const int32_t *__restrict__ dims, const T *const *uf, double h,
                                                     double *__restrict__ out) {
    __shared__ double sh[7][kInBlock / 32];
    for (int p = blockIdx.x; p < n_p; p += gridDim.x) {
        const PInfo &Pp = P[p];
        const int nx = dims[3 * Pp.scene], ny = dims[3 * Pp.scene + 1], nz = dims[3 * Pp.scene + 2];
        const long long ncell = (long long)nx * ny * nz;
        const T *__restrict__ u = uf[Pp.scene];
        const double a = Pp.a;
        int lo[3], ext[3];
        for (int c = 0; c < 3; ++c) {
            lo[c] = (int)floor(Pp.xi[c] - a) - 1;
            ext[c] = (int)floor(Pp.xi[c] + a) + 1 - lo[c] + 1;
        }
        // cell-centre offsets relative to x_p, per axis origin (grid units)
        const T ox = (T)((double)lo[0] + 0.5 - Pp.xi[0]);
        const T oy = (T)((double)lo[1] + 0.5 - Pp.xi[1]);
        const T oz = (T)((double)lo[2] + 0.5 - Pp.xi[2]);
        const T at = (T)a;
        const T r_in = at - (T)0.8660254037844386, r_out = at + (T)0.8660254037844386;
        const T r_in2 = r_in > T(0) ? r_in * r_in : T(-1), r_out2 = r_out * r_out;
        T s[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
        const int ncb = ext[0] * ext[1] * ext[2];
        for (int t = threadIdx.x; t < ncb; t += blockDim.x) {
            const int ix = t % ext[0], iy = (t / ext[0]) % ext[1], iz = t / (ext[0] * ext[1]);
            const T cx = ox + (T)ix, cy = oy + (T)iy, cz = oz + (T)iz;     // centre - x_p
            const T d2 = cx * cx + cy * cy + cz * cz;
            if (d2 > r_out2) continue;
            T alpha = T(1);
            if (!(d2 < r_in2)) {
                T num = T(0), den = T(0);
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const T qx = cx + ((m & 1) ? T(0.5) : T(-0.5));
                    const T qy = cy + ((m & 2) ? T(0.5) : T(-0.5));
                    const T qz = cz + ((m & 4) ? T(0.5) : T(-0.5));
                    const T phi = sqrt(qx * qx + qy * qy + qz * qz) - at;
                    if (phi <= T(0)) num -= phi;
                    den += fabs(phi);
                }
                alpha = den > T(0) ? num / den : T(0);
                if (alpha == T(0)) continue;
            }
            const long long idx = ((long long)wrapi(lo[2] + iz, nz) * ny + wrapi(lo[1] + iy, ny)) * nx +
                                  wrapi(lo[0] + ix, nx);
            const T u0 = u[idx], u1 = u[ncell + idx], u2 = u[2 * ncell + idx];
            s[0] += alpha * u0;
            s[1] += alpha * u1;
            s[2] += alpha * u2;
            s[3] += alpha * (cy * u2 - cz * u1);
            s[4] += alpha * (cz * u0 - cx * u2);
            s[5] += alpha * (cx * u1 - cy * u0);
            s[6] += alpha;
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            const double v = warp_sum((double)s[k]);
            if (lane == 0) sh[k][wid] = v;
        }
        __syncthreads();
        if (threadIdx.x < 7) {
            double v = 0.0;
            for (int w = 0; w < kInBlock / 32; ++w) v += sh[threadIdx.x][w];
            const double h3 = h * h * h;
            // arms are in grid units: r x u carries one more factor h
            out[7ll * p + threadIdx.x] = v * (threadIdx.x >= 3 && threadIdx.x < 6 ? h3 * h : h3);
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
    if (!ctx->in_ptr) CK(cudaMalloc(&ctx->in_ptr, ns * sizeof(void *)), "alloc field pointers");
    if (ctx->in_cap < ctx->cap_p) {
        if (ctx->in_buf) cudaFree(ctx->in_buf);
        ctx->in_buf = nullptr;
        ctx->in_cap = 0;
        CK(cudaMalloc(&ctx->in_buf, 7ll * ctx->cap_p * sizeof(double)), "alloc inertia sums");
        ctx->in_cap = ctx->cap_p;
    }
    // the device pointer table is refreshed only when the pointers change (a copy
    // from pageable memory would wait for the stream); the host vector stays alive
    if (ctx->in_ptr_h.size() != (size_t)ns || !std::equal(ctx->in_ptr_h.begin(), ctx->in_ptr_h.end(), u_ptrs)) {
        ctx->in_ptr_h.assign(u_ptrs, u_ptrs + ns);
        CK(cudaMemcpyAsync(ctx->in_ptr, ctx->in_ptr_h.data(), ns * sizeof(void *), cudaMemcpyHostToDevice,
                           ctx->stream), "copy field pointers");
    }
    const int grid = std::min(ctx->n_p, 152 * 16);
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
