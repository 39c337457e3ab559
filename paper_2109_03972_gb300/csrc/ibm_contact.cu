// Marker exclusion near contact, Sec. 2.2.5.
//
// Markers are left out of f_IBM where two particles come closer than the
// forcing can resolve: for every pair (p, q) of a scene whose surface gap
// zeta = |x_q - x_p| - a_p - a_q (minimum image) is below 2 eps_sep, one
// particle of the pair, chosen at random, loses the markers that face the
// partner.  Reading of the paper's passage (which names the pair criterion and
// the random choice but not which markers): the chosen particle's markers whose
// distance to the partner's surface, |X_l - x_o| - a_o, is below 2 eps_sep,
// i.e. the markers whose stencils reach the partner's markers' stencils.  A
// particle with many close neighbours so keeps its markers away from every
// contact.  The choice is a counter-based coin: with i < j the two particles'
// indices, z = splitmix64(seed ^ (i << 32 | j)) and the particle with index j
// is chosen when the top bit of z is set.
//
// Per step: particles are binned per scene on bins at least max(d)/h + 2 eps_sep
// wide (a pair in reach sits in the same or a neighbouring bin), one thread per
// (particle, neighbouring bin) tests the pairs in FP64 and appends the pairs in
// reach, and one block per pair marks the chosen particle's facing markers in a
// bitmap over all markers (bit moff + l).  The plain interpolation kernel then
// gives those markers e = 0 in every iteration, so they neither spread nor add
// to the loads.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "ibm_device.cuh"
#include "ibm_internal.h"

#define CK(call, what)                                                  \
    do {                                                                \
        const ibm_status ck_s = ibm_cuda_check(ctx, (call), (what));    \
        if (ck_s != IBM_OK) return ck_s;                                \
    } while (0)

namespace {

constexpr int kCtBlock = 256;

struct CtScratch {
    int n_scenes = 0, nbins = 0, cap_p = 0, cap_pairs = 0;
    double bw = 0.0;
    long long words = 0;
    int *scene_nb = nullptr, *scene_off = nullptr;   // bins per axis, first bin of each scene
    int *bin_cnt = nullptr, *bin_start = nullptr, *bin_cur = nullptr, *bin_of = nullptr, *items = nullptr;
    int *pairs = nullptr;                            // [cap_pairs][2]: chosen particle, partner
    int *cnt = nullptr;                              // [1] pairs in reach
    unsigned *bits = nullptr;                        // [words] disabled markers
};

// SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014): golden-ratio
// increment, two xor-shift-multiply rounds, a final xor-shift.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Minimum-image offset r - n floor(r / n + 1/2), in FP64 without contraction.
__device__ __forceinline__ double min_image(double r, int n) {
    const double L = (double)n;
    return __dsub_rn(r, __dmul_rn(L, floor(__dadd_rn(__ddiv_rn(r, L), 0.5))));
}

__device__ __forceinline__ int ct_bin_axis(double xi, int n, int nb) {
    const double L = (double)n;
    const double w = xi - L * floor(xi / L);            // in [0, L]
    return min(nb - 1, max(0, (int)(w * nb / L)));
}

__global__ void k_ct_bin(int n_p, const PInfo *__restrict__ P, const int32_t *__restrict__ dims,
                         const int *__restrict__ scene_nb, const int *__restrict__ scene_off, int *bin_of,
                         int *bin_cnt) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_p; p += gridDim.x * blockDim.x) {
        const PInfo &Pp = P[p];
        const int s = Pp.scene;
        int b[3];
        for (int c = 0; c < 3; ++c) b[c] = ct_bin_axis(Pp.xi[c], dims[3 * s + c], scene_nb[3 * s + c]);
        const int bin = scene_off[s] + (b[2] * scene_nb[3 * s + 1] + b[1]) * scene_nb[3 * s] + b[0];
        bin_of[p] = bin;
        atomicAdd(bin_cnt + bin, 1);
    }
}

// Exclusive scan of n counts into start[0..n] by one block: each thread scans
// a contiguous chunk, then the chunk totals are scanned by thread 0.
__global__ void k_ct_scan(const int *__restrict__ cnt, int *__restrict__ start, int n) {
    __shared__ int tot[kCtBlock + 1];
    const int per = (n + kCtBlock - 1) / kCtBlock;
    const int b0 = min(n, threadIdx.x * per), b1 = min(n, b0 + per);
    int s = 0;
    for (int i = b0; i < b1; ++i) s += cnt[i];
    tot[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int t = 0; t < kCtBlock; ++t) {
            const int v = tot[t];
            tot[t] = run;
            run += v;
        }
        tot[kCtBlock] = run;
    }
    __syncthreads();
    int run = tot[threadIdx.x];
    for (int i = b0; i < b1; ++i) {
        start[i] = run;
        run += cnt[i];
    }
    if (threadIdx.x == 0) start[n] = tot[kCtBlock];
}

__global__ void k_ct_fill(int n_p, const int *__restrict__ bin_of, const int *__restrict__ bin_start, int *bin_cur,
                          int *items) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_p; p += gridDim.x * blockDim.x) {
        const int b = bin_of[p];
        items[bin_start[b] + atomicAdd(bin_cur + b, 1)] = p;
    }
}

// One thread per (particle p, neighbouring bin): pairs p < q in reach.
__global__ void k_ct_pairs(int n_p, const PInfo *__restrict__ P, const int32_t *__restrict__ dims,
                           const int *__restrict__ scene_nb, const int *__restrict__ scene_off,
                           const int *__restrict__ bin_of, const int *__restrict__ bin_start,
                           const int *__restrict__ items, double lim, unsigned long long seed, int *pairs,
                           int cap_pairs, int *cnt, int *err) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 27ll * n_p;
         t += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(t / 27), o = (int)(t - 27ll * p);
        const PInfo &Pp = P[p];
        const int s = Pp.scene;
        const int nbx = scene_nb[3 * s], nby = scene_nb[3 * s + 1], nbz = scene_nb[3 * s + 2];
        const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
        // fewer than 3 bins along an axis: every bin of that axis once
        if ((nbx < 3 && ox + 1 >= nbx) || (nby < 3 && oy + 1 >= nby) || (nbz < 3 && oz + 1 >= nbz)) continue;
        const int b0 = bin_of[p] - scene_off[s];
        const int bx0 = b0 % nbx, by0 = (b0 / nbx) % nby, bz0 = b0 / (nbx * nby);
        const int bx = nbx >= 3 ? (bx0 + ox + nbx) % nbx : ox + 1;
        const int by = nby >= 3 ? (by0 + oy + nby) % nby : oy + 1;
        const int bz = nbz >= 3 ? (bz0 + oz + nbz) % nbz : oz + 1;
        const int b = scene_off[s] + (bz * nby + by) * nbx + bx;
        for (int i = bin_start[b]; i < bin_start[b + 1]; ++i) {
            const int q = items[i];
            if (q <= p) continue;
            const PInfo &Pq = P[q];
            double d2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                const double dv = min_image(__dsub_rn(Pq.xi[c], Pp.xi[c]), dims[3 * s + c]);
                d2 = __dadd_rn(d2, __dmul_rn(dv, dv));
            }
            if (!(__dsub_rn(__dsub_rn(sqrt(d2), Pp.a), Pq.a) < lim)) continue;
            const bool pick_q = (splitmix64(seed ^ (((unsigned long long)p << 32) | (unsigned long long)q)) >> 63) != 0;
            const int k = atomicAdd(cnt, 1);
            if (k < cap_pairs) {
                pairs[2 * k] = pick_q ? q : p;
                pairs[2 * k + 1] = pick_q ? p : q;
            } else {
                set_err(err, IBM_EBIT_OVERFLOW);
            }
        }
    }
}

// One block per pair in reach: the chosen particle's markers within lim of the
// partner's surface get their bit.  The decision is the FP64 test
// |X_l - x_o| - a_o < lim (minimum image, no contraction); an FP32 estimate
// from the FP32 directions and the pair's FP64 centre offset (error below 1e-4 h
// for particles up to a thousand cells across) settles every marker more than 1e-3 h
// from the threshold and not near a half period, and only the rest take the
// FP64 test, whose throughput on this part is a small fraction of FP32's.
__global__ void __launch_bounds__(kCtBlock) k_ct_mark(const PInfo *__restrict__ P, const double *__restrict__ t64,
                                                     const float *__restrict__ t32, const int32_t *__restrict__ dims,
                                                     const int *__restrict__ pairs, const int *__restrict__ cnt,
                                                     int cap_pairs, double lim, unsigned *bits) {
    const int n = min(*cnt, cap_pairs);
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const PInfo Pe = P[pairs[2 * k]];
        const PInfo &Po = P[pairs[2 * k + 1]];
        const double xo[3] = {Po.xi[0], Po.xi[1], Po.xi[2]};
        const double ao = Po.a;
        const int s = Pe.scene;
        float dcf[3], half[3];
        for (int c = 0; c < 3; ++c) {
            dcf[c] = (float)min_image(__dsub_rn(xo[c], Pe.xi[c]), dims[3 * s + c]);   // x_o - x_e
            half[c] = 0.5f * (float)dims[3 * s + c] - 1.0f;
        }
        const float af = (float)Pe.a, thr = (float)(ao + lim);
        for (int l = threadIdx.x; l < Pe.nl; l += blockDim.x) {
            const float *tf = t32 + 3ll * (Pe.toff + l);
            bool direct = true;
            float r2f = 0.f;
            for (int c = 0; c < 3; ++c) {
                const float v = af * tf[c] - dcf[c];                  // X_l - x_o, grid units
                direct = direct && fabsf(v) < half[c];
                r2f += v * v;
            }
            const float df = sqrtf(r2f) - thr;
            bool off;
            if (direct && df > 1e-3f) {
                off = false;
            } else if (direct && df < -1e-3f) {
                off = true;
            } else {
                const double *t = t64 + 3ll * (Pe.toff + l);
                double r2 = 0.0;
                for (int c = 0; c < 3; ++c) {
                    const double dv = min_image(__dsub_rn(marker_xi64(Pe, t, c), xo[c]), dims[3 * s + c]);
                    r2 = __dadd_rn(r2, __dmul_rn(dv, dv));
                }
                off = __dsub_rn(sqrt(r2), ao) < lim;
            }
            if (off) {
                const long long m = (long long)Pe.moff + l;
                atomicOr(bits + (m >> 5), 1u << (m & 31));
            }
        }
    }
}

ibm_status ct_alloc(ibm_ctx *ctx, CtScratch *S) {
    const int ns = ctx->cfg.n_scenes;
    const double lim = 2.0 * ctx->ct_eps / ctx->cfg.h;
    // upper bound of d/h from the largest marker count, N_l = round(pi (d/h)^2)
    const double q_max = std::sqrt((ctx->max_nl + 0.5) / M_PI) + 1e-9;
    const double bw = q_max + lim + 1e-6;
    if (S->n_scenes != ns || S->bw != bw) {
        std::vector<int> nb(3 * ns), off(ns + 1);
        long long total = 0;
        for (int s = 0; s < ns; ++s) {
            off[s] = (int)total;
            long long cells = 1;
            for (int c = 0; c < 3; ++c) {
                nb[3 * s + c] = std::max(1, (int)std::floor(ctx->dims_h[3 * s + c] / bw));
                cells *= nb[3 * s + c];
            }
            total += cells;
        }
        off[ns] = (int)total;
        if (total > (1 << 28)) return ibm_fail(ctx, IBM_ERR_CAPACITY, "too many contact bins");
        for (int **p : {&S->scene_nb, &S->scene_off, &S->bin_cnt, &S->bin_start, &S->bin_cur}) {
            if (*p) cudaFree(*p);
            *p = nullptr;
        }
        S->n_scenes = 0;
        CK(ibm_malloc(&S->scene_nb, nb.size() * sizeof(int)), "alloc contact bins");
        CK(ibm_malloc(&S->scene_off, off.size() * sizeof(int)), "alloc contact bins");
        CK(ibm_malloc(&S->bin_cnt, (total + 1) * sizeof(int)), "alloc contact bins");
        CK(ibm_malloc(&S->bin_start, (total + 1) * sizeof(int)), "alloc contact bins");
        CK(ibm_malloc(&S->bin_cur, (total + 1) * sizeof(int)), "alloc contact bins");
        CK(cudaMemcpy(S->scene_nb, nb.data(), nb.size() * sizeof(int), cudaMemcpyHostToDevice), "copy bins");
        CK(cudaMemcpy(S->scene_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice), "copy bins");
        S->nbins = (int)total;
        S->bw = bw;
        S->n_scenes = ns;
    }
    if (S->cap_p < ctx->cap_p) {
        for (int **p : {&S->bin_of, &S->items, &S->pairs, &S->cnt}) {
            if (*p) cudaFree(*p);
            *p = nullptr;
        }
        S->cap_p = 0;
        const int cap_pairs = 32 * ctx->cap_p + 64;
        CK(ibm_malloc(&S->bin_of, ctx->cap_p * sizeof(int)), "alloc contact lists");
        CK(ibm_malloc(&S->items, ctx->cap_p * sizeof(int)), "alloc contact lists");
        CK(ibm_malloc(&S->pairs, 2ll * cap_pairs * sizeof(int)), "alloc contact pairs");
        CK(ibm_malloc(&S->cnt, sizeof(int)), "alloc contact count");
        S->cap_pairs = cap_pairs;
        S->cap_p = ctx->cap_p;
    }
    const long long words = (ctx->n_markers + 31) / 32 + 1;
    if (S->words < words) {
        if (S->bits) cudaFree(S->bits);
        S->bits = nullptr;
        S->words = 0;
        CK(ibm_malloc(&S->bits, words * sizeof(unsigned)), "alloc marker bitmap");
        S->words = words;
    }
    return IBM_OK;
}

}  // namespace

ibm_status contact_exclusion(ibm_ctx *ctx) {
    CtScratch *S = reinterpret_cast<CtScratch *>(ctx->ct);
    if (!S) {
        S = new (std::nothrow) CtScratch();
        if (!S) return IBM_ERR_OOM;
        ctx->ct = S;
    }
    ibm_status st = ct_alloc(ctx, S);
    if (st != IBM_OK) return st;
    cudaStream_t sm = ctx->stream;
    const int n = ctx->n_p;
    const double lim = 2.0 * ctx->ct_eps / ctx->cfg.h;
    CK(cudaMemsetAsync(S->bits, 0, S->words * sizeof(unsigned), sm), "zero marker bitmap");
    CK(cudaMemsetAsync(S->bin_cnt, 0, (S->nbins + 1) * sizeof(int), sm), "zero contact bins");
    CK(cudaMemsetAsync(S->bin_cur, 0, (S->nbins + 1) * sizeof(int), sm), "zero contact bins");
    CK(cudaMemsetAsync(S->cnt, 0, sizeof(int), sm), "zero contact count");
    const int gb = std::max(1, std::min((n + kCtBlock - 1) / kCtBlock, 152 * 8));
    k_ct_bin<<<gb, kCtBlock, 0, sm>>>(n, ctx->pinfo, ctx->dims_d, S->scene_nb, S->scene_off, S->bin_of, S->bin_cnt);
    k_ct_scan<<<1, kCtBlock, 0, sm>>>(S->bin_cnt, S->bin_start, S->nbins);
    k_ct_fill<<<gb, kCtBlock, 0, sm>>>(n, S->bin_of, S->bin_start, S->bin_cur, S->items);
    const long long work = 27ll * n;
    const int gp = (int)std::max(1ll, std::min((work + kCtBlock - 1) / kCtBlock, 152ll * 8));
    k_ct_pairs<<<gp, kCtBlock, 0, sm>>>(n, ctx->pinfo, ctx->dims_d, S->scene_nb, S->scene_off, S->bin_of,
                                        S->bin_start, S->items, lim, (unsigned long long)ctx->ct_seed, S->pairs,
                                        S->cap_pairs, S->cnt, ctx->err_d);
    k_ct_mark<<<152 * 4, kCtBlock, 0, sm>>>(ctx->pinfo, ctx->tmpl64, ctx->tmpl32, ctx->dims_d, S->pairs, S->cnt,
                                            S->cap_pairs, lim, S->bits);
    ctx->launches += 5;
    return ibm_cuda_check(ctx, cudaGetLastError(), "contact exclusion");
}

const unsigned *contact_bits(const ibm_ctx *ctx) {
    const CtScratch *S = reinterpret_cast<const CtScratch *>(ctx->ct);
    return (ctx->ct_enable && S) ? S->bits : nullptr;
}

void contact_graph_key(const ibm_ctx *ctx, std::vector<uintptr_t> &key) {
    const CtScratch *S = reinterpret_cast<const CtScratch *>(ctx->ct);
    uint64_t eb;
    std::memcpy(&eb, &ctx->ct_eps, sizeof(eb));
    key.push_back((uintptr_t)ctx->ct_enable);
    key.push_back((uintptr_t)eb);
    key.push_back((uintptr_t)ctx->ct_seed);
    if (!S) return;
    for (const void *b : {(const void *)S->scene_nb, (const void *)S->scene_off, (const void *)S->bin_cnt,
                          (const void *)S->bin_start, (const void *)S->bin_cur, (const void *)S->bin_of,
                          (const void *)S->items, (const void *)S->pairs, (const void *)S->cnt,
                          (const void *)S->bits})
        key.push_back((uintptr_t)b);
}

void contact_free(ibm_ctx *ctx) {
    CtScratch *S = reinterpret_cast<CtScratch *>(ctx->ct);
    if (!S) return;
    for (void *p : {(void *)S->scene_nb, (void *)S->scene_off, (void *)S->bin_cnt, (void *)S->bin_start,
                    (void *)S->bin_cur, (void *)S->bin_of, (void *)S->items, (void *)S->pairs, (void *)S->cnt,
                    (void *)S->bits})
        if (p) cudaFree(p);
    delete S;
    ctx->ct = nullptr;
}

extern "C" ibm_status ibm_set_contact_exclusion(ibm_ctx *ctx, int enable, double eps_sep, uint64_t seed) {
    if (!ctx) return IBM_ERR_INVALID_ARG;
    if (enable) {
        if (ctx->cfg.requires_grad)
            return ibm_fail(ctx, IBM_ERR_INVALID_ARG, "marker exclusion has no adjoint (requires_grad)");
        if (!(eps_sep >= 0.0) || !std::isfinite(eps_sep))
            return ibm_fail(ctx, IBM_ERR_INVALID_ARG, "eps_sep must be finite and >= 0");
    }
    ctx->ct_enable = enable ? 1 : 0;
    ctx->ct_eps = eps_sep > 0.0 ? eps_sep : (ctx->cfg.kernel_width == 4 ? 2.0 : 1.5) * ctx->cfg.h;
    ctx->ct_seed = seed;
    return IBM_OK;
}

extern "C" ibm_status ibm_disabled_markers(ibm_ctx *ctx, uint32_t *bits_out, int64_t *n_disabled) {
    if (!ctx || !n_disabled) return IBM_ERR_INVALID_ARG;
    const CtScratch *S = reinterpret_cast<const CtScratch *>(ctx->ct);
    const long long words = (ctx->n_markers + 31) / 32;
    std::vector<uint32_t> h(words, 0u);
    if (ctx->ct_enable && S && S->bits && words > 0) {
        CK(cudaMemcpyAsync(h.data(), S->bits, words * sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream),
           "copy marker bitmap");
        CK(cudaStreamSynchronize(ctx->stream), "copy marker bitmap");
    }
    long long c = 0;
    for (uint32_t w : h) c += __builtin_popcount(w);
    *n_disabled = c;
    if (bits_out && words > 0) std::memcpy(bits_out, h.data(), words * sizeof(uint32_t));
    return IBM_OK;
}
