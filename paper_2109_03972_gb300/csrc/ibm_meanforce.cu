// Mean IBM force over the grid, Sec. 2.2.4 Eq. (fe_IBM):
//   fbar = -(1 / (N_i N_j N_k)) sum_{i,j,k} f_IBM,ijk      per scene and component.
//
// One streaming pass over the force field: every scene's component array is
// cut into segments of kSeg elements; a block sums one segment at a time and
// writes its FP64 partial, and one warp per array adds the partials in a fixed
// order.  The pass reads each cell once (12 B per cell in FP32, 24 B in FP64)
// and is bound by HBM bandwidth.  FP32 fields: each thread adds 16 values in
// FP32 (four 16-byte loads in flight) before one FP64 addition, which keeps
// the FP64 pipe, far narrower than FP32 on this part, off the critical path.
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

constexpr int kMfBlock = 256;
constexpr long long kSeg = 1ll << 16;   // elements per segment, a multiple of 16

// Array a = 3 s + q (scene s, component q) starts at base[s] + q * cells[s].
template <typename T>
__global__ void __launch_bounds__(kMfBlock) k_mf_partial(const T *const *__restrict__ base,
                                                        const long long *__restrict__ cells,
                                                        const long long *__restrict__ seg_prefix, int n_arr,
                                                        double *__restrict__ partial) {
    __shared__ double s_w[kMfBlock / 32];
    const long long n_seg = seg_prefix[n_arr];
    for (long long g = blockIdx.x; g < n_seg; g += gridDim.x) {
        int lo = 0, hi = n_arr;   // largest a with seg_prefix[a] <= g
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (seg_prefix[mid] <= g) lo = mid;
            else hi = mid;
        }
        const int s = lo / 3, q = lo - 3 * s;
        const long long n = cells[s];
        const T *x = base[s] + q * n;
        const long long beg = (g - seg_prefix[lo]) * kSeg;
        const long long end = min(n, beg + kSeg);
        double acc = 0.0;
        long long tail = beg;
        if (sizeof(T) == 4 && (reinterpret_cast<uintptr_t>(x + beg) & 15) == 0) {
            const float4 *v = reinterpret_cast<const float4 *>(x + beg);
            const long long nv = (end - beg) >> 2;          // whole float4s
            const long long n4 = nv / (4 * kMfBlock) * (4 * kMfBlock);
            for (long long i = threadIdx.x; i < n4; i += 4 * kMfBlock) {
                float4 a[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) a[k] = __ldcs(v + i + k * kMfBlock);
                float t = 0.f;
#pragma unroll
                for (int k = 0; k < 4; ++k) t += (a[k].x + a[k].y) + (a[k].z + a[k].w);
                acc += (double)t;
            }
            for (long long i = n4 + threadIdx.x; i < nv; i += kMfBlock) {
                const float4 a = __ldcs(v + i);
                acc += (double)((a.x + a.y) + (a.z + a.w));
            }
            tail = beg + 4 * nv;
        }
        for (long long i = tail + threadIdx.x; i < end; i += kMfBlock) acc += (double)x[i];
        acc = warp_sum(acc);
        if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x < 32) {
            double w = threadIdx.x < kMfBlock / 32 ? s_w[threadIdx.x] : 0.0;
            w = warp_sum(w);
            if (threadIdx.x == 0) partial[g] = w;
        }
        __syncthreads();
    }
}

// One warp per array: lane j adds partials j, j + 32, ... in order, then a
// fixed shuffle tree; out[a] = -sum / cells.
__global__ void k_mf_final(const long long *__restrict__ cells, const long long *__restrict__ seg_prefix, int n_arr,
                           const double *__restrict__ partial, double *__restrict__ out) {
    const int a = blockIdx.x;
    if (a >= n_arr) return;
    double v = 0.0;
    for (long long g = seg_prefix[a] + threadIdx.x; g < seg_prefix[a + 1]; g += 32) v += partial[g];
    v = warp_sum(v);
    if (threadIdx.x == 0) out[a] = -v / (double)cells[a / 3];
}

// Segment table and scratch, built once per context (the grids are fixed at create).
ibm_status mf_prepare(ibm_ctx *ctx) {
    if (ctx->mf_seg) return IBM_OK;
    const int ns = ctx->cfg.n_scenes, n_arr = 3 * ns;
    std::vector<long long> cells(ns), prefix(n_arr + 1, 0);
    for (int s = 0; s < ns; ++s) {
        cells[s] = (long long)ctx->dims_h[3 * s] * ctx->dims_h[3 * s + 1] * ctx->dims_h[3 * s + 2];
        for (int q = 0; q < 3; ++q) prefix[3 * s + q + 1] = prefix[3 * s + q] + (cells[s] + kSeg - 1) / kSeg;
    }
    long long *seg = nullptr, *cl = nullptr;
    double *part = nullptr, *out = nullptr;
    void **ptr = nullptr;
    if (ibm_malloc(&seg, prefix.size() * sizeof(long long)) != cudaSuccess ||
        ibm_malloc(&cl, cells.size() * sizeof(long long)) != cudaSuccess ||
        ibm_malloc(&part, std::max(1ll, prefix[n_arr]) * sizeof(double)) != cudaSuccess ||
        ibm_malloc(&out, n_arr * sizeof(double)) != cudaSuccess || ibm_malloc(&ptr, ns * sizeof(void *)) != cudaSuccess) {
        cudaGetLastError();
        for (void *p : {(void *)seg, (void *)cl, (void *)part, (void *)out, (void *)ptr})
            if (p) cudaFree(p);
        return ibm_cuda_check(ctx, cudaErrorMemoryAllocation, "alloc mean-force scratch");
    }
    CK(cudaMemcpy(seg, prefix.data(), prefix.size() * sizeof(long long), cudaMemcpyHostToDevice), "copy segments");
    CK(cudaMemcpy(cl, cells.data(), cells.size() * sizeof(long long), cudaMemcpyHostToDevice), "copy cell counts");
    ctx->mf_seg = seg;
    ctx->mf_cells = cl;
    ctx->mf_part = part;
    ctx->mf_out = out;
    ctx->mf_ptr = ptr;
    ctx->mf_nseg = prefix[n_arr];
    return IBM_OK;
}

}  // namespace

extern "C" ibm_status ibm_mean_force(ibm_ctx *ctx, void *const *f_ptrs, double *fbar_out, int on_device) {
    if (!ctx || !f_ptrs || !fbar_out) return IBM_ERR_INVALID_ARG;
    const int ns = ctx->cfg.n_scenes, n_arr = 3 * ns;
    for (int s = 0; s < ns; ++s)
        if (!f_ptrs[s]) return IBM_ERR_INVALID_ARG;
    ibm_status st = mf_prepare(ctx);
    if (st != IBM_OK) return st;
    // the device pointer table is refreshed only when the pointers change (a copy
    // from pageable memory would wait for the stream); the host vector stays alive
    if (ctx->mf_ptr_h.size() != (size_t)ns || !std::equal(ctx->mf_ptr_h.begin(), ctx->mf_ptr_h.end(), f_ptrs)) {
        ctx->mf_ptr_h.assign(f_ptrs, f_ptrs + ns);
        CK(cudaMemcpyAsync(ctx->mf_ptr, ctx->mf_ptr_h.data(), ns * sizeof(void *), cudaMemcpyHostToDevice,
                           ctx->stream), "copy field pointers");
    }
    const int grid = (int)std::min<long long>(std::max(1ll, ctx->mf_nseg), 152ll * 8);
    if (ctx->cfg.precision == IBM_FP64)
        k_mf_partial<double><<<grid, kMfBlock, 0, ctx->stream>>>(reinterpret_cast<const double *const *>(ctx->mf_ptr),
                                                                ctx->mf_cells, ctx->mf_seg, n_arr, ctx->mf_part);
    else
        k_mf_partial<float><<<grid, kMfBlock, 0, ctx->stream>>>(reinterpret_cast<const float *const *>(ctx->mf_ptr),
                                                               ctx->mf_cells, ctx->mf_seg, n_arr, ctx->mf_part);
    k_mf_final<<<n_arr, 32, 0, ctx->stream>>>(ctx->mf_cells, ctx->mf_seg, n_arr, ctx->mf_part,
                                               on_device ? fbar_out : ctx->mf_out);
    st = ibm_cuda_check(ctx, cudaGetLastError(), "mean force");
    if (st != IBM_OK || on_device) return st;
    CK(cudaMemcpyAsync(fbar_out, ctx->mf_out, n_arr * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
       "copy mean force");
    return ibm_cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "mean force");
}
