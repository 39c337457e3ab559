// Cluster path of the FP32 forcing step.
//
// Two particles interact within one forcing iteration only when a grid cell
// lies in the stencils of markers of both (the 3x3x3 supports of Eq.
// 3pt-stencil overlap).  Connected components of that relation ("clusters")
// are independent for all n_F iterations of the outer forcing loop (Sec.
// 2.2.2): no cell of one cluster is read or written by another.  So each
// cluster is processed by one CTA that
//   1. builds the exact set of touched cells (union of marker stencils) as
//      per-row bitmasks over the cluster's box, and a compact slot for each
//      touched cell (prefix sums of the masks),
//   2. gathers u at the touched cells from HBM into shared memory once,
//   3. runs all n_F iterations (interpolate -> force -> spread -> update)
//      on the shared-memory copy, with __syncthreads between the phases,
//   4. writes the touched cells back once, and the particle loads.
// HBM sees one read and one write per touched cell per step instead of one
// per iteration.  Each marker's stencil is kept as a 32-byte record (fractional
// position and the slots of its nine row runs), in shared memory when it fits
// and in an L2-resident global scratch otherwise.  A cluster that cannot be
// unwrapped along an axis of the periodic domain gets the whole period as its
// box there (rows wrap in y and z, ghost columns in x).  Clusters too large for
// one CTA's shared memory run the plain FP32 path (global atomics; in the
// deterministic mode fixed point per cluster), which touches disjoint cells
// and can therefore follow in any order.
//
// Clustering per step: particles are binned on a coarse grid, candidate pairs
// (centre distance < a_p + a_q + 3 sqrt 3, the largest distance at which two
// markers can have base cells within 2 of each other) are tested exactly
// (some marker pair with |b_l - b_l'|_inf <= 2), and joined by a lock-free
// union-find.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "ibm_device.cuh"
#include "ibm_internal.h"

#define CK(call, what)                                                  \
    do {                                                                \
        ibm_status _s = ibm_cuda_check(ctx, (call), what);              \
        if (_s != IBM_OK) return _s;                                    \
    } while (0)

namespace {

constexpr int kCapP = 32;        // particles per shared-memory batch
constexpr int kBuckets = 1024;   // work-order buckets
constexpr int kPairThreads = 128;
constexpr int kPairCap = 1024;   // near-marker list in the exact pair test
constexpr int kUnionSpin = 1 << 22;   // default bound of the union-find retries
constexpr int kSparseRows = 32768;   // box rows (y, z) of a cluster with a sparse row table

enum {
    C_NCAND = 0,
    C_NCLUST,
    C_NFB,        // particles on the fallback path
    C_WORK,       // persistent-kernel work counter
    C_NITEMS,     // clusters on the shared-memory path
    C_OVERFLOW,   // clusters that overflowed shared memory at run time
    C_MAXCELLS,
    C_TOUCHED,
    C_FBMARK,     // markers on the fallback path
    C_ONECOMP,    // clusters run one velocity component at a time
    C_NBATCH,     // shared-memory work items (batches of clusters)
    C_NBIG,       // clusters on the distributed-shared-memory path (both sizes)
    C_NBIG8,      // ... of them on 8-CTA thread-block clusters, and their work counter
    C_WORK8,
    C_NBIG16,     // ... on 16-CTA thread-block clusters, and their work counter
    C_WORK16,
    C_BIGMARK,    // markers on that path
    C_NFB2,       // particles left on the plain fallback
    C_COUNT
};

struct ClusterScratch {
    int cap_p = 0, cap_bins = 0, cap_cand = 0;
    int nbins = 0, max_nl = -1, n_scenes = 0;
    double bin_w = 0.0;
    int *scene_bin_off = nullptr, *scene_nb = nullptr;
    int *bin_cnt = nullptr, *bin_start = nullptr, *bin_cur = nullptr, *bin_items = nullptr;
    int *parent = nullptr, *cand = nullptr, *cnt = nullptr;
    long long *tot = nullptr;
    int *root_flag = nullptr, *cid = nullptr, *pcl = nullptr, *poff = nullptr;
    int *cl_np = nullptr, *cl_nm = nullptr, *cl_first = nullptr, *cl_cur = nullptr, *cl_box = nullptr;
    int *cl_plist = nullptr, *cl_bkt = nullptr;
    int *bkt_cnt = nullptr, *bkt_start = nullptr, *order = nullptr, *fb_list = nullptr;
    int *nm_ord = nullptr, *cum = nullptr, *cl_scene = nullptr;
    int *cl_path = nullptr;          // IBM_PATH_* bits of each cluster (last step)
    int2 *batches = nullptr;
    float4 *grec = nullptr;          // marker records of batches kept in global memory
    size_t grec_bytes = 0;
    int smem_bytes = 0, cap_c = 0, tpb = 0, kmax = 0, det = -1;
    // clusters too large for one SM, held in the distributed shared memory of a
    // thread-block cluster: the work list, a flag per cluster, the plain
    // fallback's remaining particles, marker records and chunk sums per slot
    int *big_list = nullptr, *big_flag = nullptr, *fb_list2 = nullptr;
    uint4 *big_rec = nullptr;
    float *big_part = nullptr;
    int *big_wl = nullptr;
    size_t big_rec_bytes = 0, big_part_bytes = 0, big_wl_bytes = 0;
    // thread-block-cluster path: configured (-1: not yet), clusters of 8 and 16 CTAs that run at once
    // (0: that size cannot run), dense cells per CTA
    int big_k = -1, big_grid8 = 0, big_grid16 = 0, big_cells = 0, big_det = -1, big_smem = 0;
    int *big_list16 = nullptr;
    // the 16-CTA launch runs beside the 8-CTA one on a stream of its own (fork and join by events)
    cudaStream_t big_side = nullptr;
    cudaEvent_t big_fork = nullptr, big_join = nullptr;
};

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ int ld_volatile(const int *p) { return *((const volatile int *)p); }

__device__ int uf_find(int *parent, int x, int spin) {
    for (int it = 0; it < spin; ++it) {
        const int p = ld_volatile(parent + x);
        if (p == x) return x;
        const int gp = ld_volatile(parent + p);
        if (gp != p) atomicCAS(parent + x, p, gp);  // path halving; parents only decrease
        x = p;
    }
    return -1;
}

__device__ bool uf_unite(int *parent, int a, int b, int spin) {
    for (int it = 0; it < spin; ++it) {
        a = uf_find(parent, a, spin);
        b = uf_find(parent, b, spin);
        if (a < 0 || b < 0) return false;
        if (a == b) return true;
        if (a > b) { const int t = a; a = b; b = t; }
        const int old = atomicCAS(parent + b, b, a);   // link the larger root under the smaller
        if (old == b) return true;
    }
    return false;
}

__device__ __forceinline__ int scene_bin(const int *scene_nb, const int *scene_bin_off, const int32_t *dims,
                                         int s, const double xi[3], int bc[3]) {
    for (int c = 0; c < 3; ++c) {
        // FP32: bins are wider than the candidate distance by a margin (1h) that
        // covers the rounding of the bin assignment
        const int n = dims[3 * s + c], nb = scene_nb[3 * s + c];
        const float f = (float)xi[c] * __frcp_rn((float)n);
        const float w = f - floorf(f);                   // wrapped into [0, 1)
        int b = (int)(w * nb);
        b = min(max(b, 0), nb - 1);
        bc[c] = b;
    }
    return scene_bin_off[s] + (bc[2] * scene_nb[3 * s + 1] + bc[1]) * scene_nb[3 * s] + bc[0];
}

// ------------------------------------------------------------- clustering

__global__ void k_bin_count(int n_p, const PInfo *P, const int *scene_nb, const int *scene_bin_off,
                            const int32_t *dims, int *bin_cnt, int *parent) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_p; p += gridDim.x * blockDim.x) {
        int bc[3];
        const int b = scene_bin(scene_nb, scene_bin_off, dims, P[p].scene, P[p].xi, bc);
        atomicAdd(bin_cnt + b, 1);
        parent[p] = p;
    }
}

__global__ void k_bin_fill(int n_p, const PInfo *P, const int *scene_nb, const int *scene_bin_off,
                           const int32_t *dims, const int *bin_start, int *bin_cur, int *bin_items) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_p; p += gridDim.x * blockDim.x) {
        int bc[3];
        const int b = scene_bin(scene_nb, scene_bin_off, dims, P[p].scene, P[p].xi, bc);
        bin_items[bin_start[b] + atomicAdd(bin_cur + b, 1)] = p;
    }
}

// Minimum-image offset of q relative to p, in whole periods (grid units).
__device__ __forceinline__ void min_image_shift(const double xp[3], const double xq[3], const int32_t *dims,
                                                int s, int sh[3]) {
    for (int c = 0; c < 3; ++c) {
        const int n = dims[3 * s + c];
        // FP32 is enough: only the nearest whole number of periods matters, and a
        // half-period tie gives the same distance either way
        sh[c] = -__float2int_rn((float)(xq[c] - xp[c]) * __frcp_rn((float)n)) * n;
    }
}

// Candidate pairs: one thread per (particle, neighbouring bin) of the 3x3x3
// bins around the particle's own (fewer where a scene has fewer bins).
__global__ void k_candidates(int n_p, const PInfo *P, const int *scene_nb, const int *scene_bin_off,
                             const int32_t *dims, const int *bin_start, const int *bin_items, int *cand,
                             int cap_cand, int *cnt) {
    const float lim = 3.0f * 1.7320508f + 1e-3f;   // margin covers the FP32 rounding of the distance
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 27ll * n_p;
         t += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(t / 27), o = (int)(t - 27ll * p);
        const PInfo &Pp = P[p];
        const int s = Pp.scene;
        const int nbx = scene_nb[3 * s], nby = scene_nb[3 * s + 1], nbz = scene_nb[3 * s + 2];
        const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
        // with fewer than 3 bins along an axis every bin is visited once
        if ((nbx < 3 && ox + 1 >= nbx) || (nby < 3 && oy + 1 >= nby) || (nbz < 3 && oz + 1 >= nbz)) continue;
        int bc[3];
        scene_bin(scene_nb, scene_bin_off, dims, s, Pp.xi, bc);
        const int bx = nbx >= 3 ? (bc[0] + ox + nbx) % nbx : ox + 1;
        const int by = nby >= 3 ? (bc[1] + oy + nby) % nby : oy + 1;
        const int bz = nbz >= 3 ? (bc[2] + oz + nbz) % nbz : oz + 1;
        const int b = scene_bin_off[s] + (bz * nby + by) * nbx + bx;
        for (int i = bin_start[b]; i < bin_start[b + 1]; ++i) {
            const int q = bin_items[i];
            if (q <= p) continue;
            const PInfo &Pq = P[q];
            int sh[3];
            min_image_shift(Pp.xi, Pq.xi, dims, s, sh);
            float d2 = 0.f;
            for (int c = 0; c < 3; ++c) {
                const float dv = (float)(Pq.xi[c] - Pp.xi[c]) + (float)sh[c];
                d2 += dv * dv;
            }
            const float r = Pp.af + Pq.af + lim;
            if (d2 < r * r) {
                const int k = atomicAdd(cnt + C_NCAND, 1);
                if (k < cap_cand) {
                    cand[2 * k] = p;
                    cand[2 * k + 1] = q;
                }
            }
        }
    }
}

// Exact test of one candidate pair: some markers l of p and l' of q with
// |b_l - b_l'|_inf <= 2 (then their 3x3x3 stencils share a cell).  Uses the
// same FP32-path base cells as the forcing kernels.  Only markers within
// a + 3 sqrt 3 + 1 of the other centre can qualify.  q's qualifying base cells
// are marked in a 32^3 bit volume around them, which is dilated by 2 along
// each axis (separable max filter on 32-bit rows), so that each qualifying
// marker of p needs one bit test.  A volume wider than 32 cells falls back to
// comparing the two lists pair by pair.
__global__ void __launch_bounds__(kPairThreads) k_pair_test(const PInfo *P, const float *t32, const double *t64,
                                                            const int32_t *dims, const int *cand, const int *cnt,
                                                            int cap_cand, int *parent, int spin, int *err) {
    __shared__ int3 qb[kPairCap];
    __shared__ unsigned vol[2][32 * 32];   // [z][y] rows of 32 x-bits
    __shared__ int nq, found, over, lo[3], hi[3];
    const int ncand = min(cnt[C_NCAND], cap_cand);
    for (int k = blockIdx.x; k < ncand; k += gridDim.x) {
        const int p = cand[2 * k], q = cand[2 * k + 1];
        const PInfo Pp = P[p], Pq = P[q];
        int sh[3];
        min_image_shift(Pp.xi, Pq.xi, dims, Pp.scene, sh);
        if (threadIdx.x == 0) {
            nq = 0; found = 0; over = 0;
            lo[0] = lo[1] = lo[2] = INT_MAX;
            hi[0] = hi[1] = hi[2] = INT_MIN;
        }
        __syncthreads();
        const float rp = (float)(Pp.a + 3.0 * 1.7320508075688772 + 1.0);
        const float rq = (float)(Pq.a + 3.0 * 1.7320508075688772 + 1.0);
        for (int l = threadIdx.x; l < Pq.nl; l += blockDim.x) {
            const float *t = t32 + 3ll * (Pq.toff + l);
            float dd = 0.f;
            for (int c = 0; c < 3; ++c) {
                const float v = (float)(Pq.xi[c] + sh[c] - Pp.xi[c]) + Pq.af * t[c];
                dd += v * v;
            }
            if (dd > rp * rp) continue;
            int b[3];
            float fr;
            for (int c = 0; c < 3; ++c) {
                b[c] = marker_split32(Pq, t, t64 + 3ll * (Pq.toff + l), c, &fr) + sh[c];
                atomicMin(&lo[c], b[c]);
                atomicMax(&hi[c], b[c]);
            }
            const int i = atomicAdd(&nq, 1);
            if (i < kPairCap) qb[i] = make_int3(b[0], b[1], b[2]);
            else over = 1;
        }
        __syncthreads();
        const int n = nq;
        if (over) {
            if (threadIdx.x == 0 && !uf_unite(parent, p, q, spin)) set_err(err, IBM_EBIT_TIMEOUT);
            __syncthreads();
            continue;
        }
        if (n == 0) {
            __syncthreads();
            continue;
        }
        const int o0 = lo[0] - 2, o1 = lo[1] - 2, o2 = lo[2] - 2;
        const bool use_vol = hi[0] - o0 < 30 && hi[1] - o1 < 30 && hi[2] - o2 < 30;
        if (use_vol) {
            for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) vol[0][i] = 0u;
            __syncthreads();
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                const int3 b = qb[j];
                atomicOr(&vol[0][(b.z - o2) * 32 + (b.y - o1)], 1u << (b.x - o0));
            }
            __syncthreads();
            for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) {
                const unsigned w = vol[0][i];
                vol[0][i] = w | (w << 1) | (w << 2) | (w >> 1) | (w >> 2);
            }
            __syncthreads();
            for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) {
                const int z = i >> 5, y = i & 31;
                unsigned w = 0u;
                for (int d = -2; d <= 2; ++d)
                    if (y + d >= 0 && y + d < 32) w |= vol[0][z * 32 + y + d];
                vol[1][i] = w;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) {
                const int z = i >> 5, y = i & 31;
                unsigned w = 0u;
                for (int d = -2; d <= 2; ++d)
                    if (z + d >= 0 && z + d < 32) w |= vol[1][(z + d) * 32 + y];
                vol[0][i] = w;
            }
            __syncthreads();
        }
        for (int l = threadIdx.x; l < Pp.nl && !found; l += blockDim.x) {
            const float *t = t32 + 3ll * (Pp.toff + l);
            float dd = 0.f;
            for (int c = 0; c < 3; ++c) {
                const float v = (float)(Pp.xi[c] - Pq.xi[c] - sh[c]) + Pp.af * t[c];
                dd += v * v;
            }
            if (dd > rq * rq) continue;
            float fr;
            const int bx = marker_split32(Pp, t, t64 + 3ll * (Pp.toff + l), 0, &fr);
            const int by = marker_split32(Pp, t, t64 + 3ll * (Pp.toff + l), 1, &fr);
            const int bz = marker_split32(Pp, t, t64 + 3ll * (Pp.toff + l), 2, &fr);
            if (use_vol) {
                // the dilated volume covers every cell within 2 of a q base
                const int x = bx - o0, y = by - o1, z = bz - o2;
                if (x >= 0 && x < 32 && y >= 0 && y < 32 && z >= 0 && z < 32 && ((vol[0][z * 32 + y] >> x) & 1u))
                    found = 1;
            } else {
                for (int j = 0; j < n; ++j) {
                    const int3 b = qb[j];
                    if (abs(b.x - bx) <= 2 && abs(b.y - by) <= 2 && abs(b.z - bz) <= 2) {
                        found = 1;
                        break;
                    }
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && found && !uf_unite(parent, p, q, spin)) set_err(err, IBM_EBIT_TIMEOUT);
        __syncthreads();
    }
}

__global__ void k_roots(int n_p, int *parent, int *root_flag, int spin, int *err) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_p; p += gridDim.x * blockDim.x) {
        const int r = uf_find(parent, p, spin);
        if (r < 0) { set_err(err, IBM_EBIT_TIMEOUT); root_flag[p] = 0; continue; }
        root_flag[p] = (r == p);
    }
}

__global__ void k_cluster_init(int n, int *cl_np, int *cl_nm, int *cl_cur, int *cl_box) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        cl_np[c] = 0;
        cl_nm[c] = 0;
        cl_cur[c] = 0;
        for (int k = 0; k < 3; ++k) {
            cl_box[12 * c + k] = INT_MAX;        // stencil box lo
            cl_box[12 * c + 3 + k] = INT_MIN;    // stencil box hi
            cl_box[12 * c + 6 + k] = INT_MAX;    // centre box lo
            cl_box[12 * c + 9 + k] = INT_MIN;    // centre box hi
        }
    }
}

// Per particle: its cluster, the whole-period shift that unwraps it next to
// the cluster's root, and the cluster's stencil box (floor(xi -+ a) -+ 1).
__global__ void k_cluster_stats(int n_p, const PInfo *P, const int32_t *dims, int *parent, const int *cid,
                                int *pcl, int *poff, int *cl_np, int *cl_nm, int *cl_box, int spin) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_p; p += gridDim.x * blockDim.x) {
        const int r = uf_find(parent, p, spin);
        const int c = cid[r < 0 ? p : r];
        pcl[p] = c;
        const PInfo &Pp = P[p];
        int sh[3];
        min_image_shift(P[r < 0 ? p : r].xi, Pp.xi, dims, Pp.scene, sh);
        atomicAdd(cl_np + c, 1);
        atomicAdd(cl_nm + c, (Pp.nl + 31) & ~31);   // padded to whole 32-marker chunks
        for (int k = 0; k < 3; ++k) {
            poff[3 * p + k] = sh[k];
            const int lo = (int)floor(Pp.xi[k] - Pp.a) - 1 + sh[k];
            const int hi = (int)floor(Pp.xi[k] + Pp.a) + 1 + sh[k];
            atomicMin(cl_box + 12 * c + k, lo);
            atomicMax(cl_box + 12 * c + 3 + k, hi);
            atomicMin(cl_box + 12 * c + 6 + k, Pp.base[k] + sh[k]);
            atomicMax(cl_box + 12 * c + 9 + k, Pp.base[k] + sh[k]);
        }
    }
}

__global__ void k_cluster_fill(int n_p, const int *pcl, const int *cl_first, int *cl_cur, int *cl_plist) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_p; p += gridDim.x * blockDim.x) {
        const int c = pcl[p];
        cl_plist[cl_first[c] + atomicAdd(cl_cur + c, 1)] = p;
    }
}

// Route each cluster: shared-memory path if it fits the CTA's capacities and
// its box is consistently unwrapped, else the plain fallback.
__global__ void k_cluster_route(const long long *n_clust_d, const PInfo *P, const int32_t *dims, const int *cl_np,
                                const int *cl_nm, const int *cl_first, const int *cl_plist, int *cl_box,
                                int cap_m, int max_rows, int *cl_bkt, int *bkt_cnt, int *fb_list, int *cl_scene,
                                int *cl_path, int *cnt) {
    const int n = (int)*n_clust_d;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const int np = cl_np[c], nm = cl_nm[c];
        const int s = P[cl_plist[cl_first[c]]].scene;
        bool ok = np <= kCapP && nm <= cap_m;
        int R = 1, wrap = 0;
        for (int k = 0; k < 3; ++k) {
            const int n_k = dims[3 * s + k];
            int ext = cl_box[12 * c + 3 + k] - cl_box[12 * c + k] + 1;
            const int cext = cl_box[12 * c + 9 + k] - cl_box[12 * c + 6 + k] + 1;
            if (!(ext <= n_k && 2 * cext < n_k)) {
                // the cluster cannot be unwrapped along this axis: its box is the
                // whole period (rows wrap in y and z; in x one ghost column each side)
                wrap |= 1 << k;
                cl_box[12 * c + k] = k == 0 ? -1 : 0;
                cl_box[12 * c + 3 + k] = k == 0 ? n_k : n_k - 1;
                ext = cl_box[12 * c + 3 + k] - cl_box[12 * c + k] + 1;
            }
            R *= (k == 0) ? (ext + 31) / 32 : ext;
        }
        // a dense row table over max_rows entries is replaced by a sparse one
        // (rows numbered in 16 bits) in the kernel
        const int nyz = (cl_box[12 * c + 4] - cl_box[12 * c + 1] + 1) * (cl_box[12 * c + 5] - cl_box[12 * c + 2] + 1);
        ok = ok && (R <= max_rows || nyz <= kSparseRows);
        // bitmask entry decode words hold y, z < 1024 and 16 words (512 cells) per row
        ok = ok && (cl_box[12 * c + 4] - cl_box[12 * c + 1]) < 1023 && (cl_box[12 * c + 5] - cl_box[12 * c + 2]) < 1023 &&
             (cl_box[12 * c + 3] - cl_box[12 * c]) < 511;
        cl_scene[c] = s | (wrap << 28);   // scene, and the wrapped axes in the top bits
        cl_path[c] = (wrap ? IBM_PATH_PERIODIC : 0) | (ok ? 0 : IBM_PATH_FALLBACK);
        if (ok) {
            const int b = min(kBuckets - 1, nm / 8);
            cl_bkt[c] = kBuckets - 1 - b;   // larger clusters first
            atomicAdd(bkt_cnt + (kBuckets - 1 - b), 1);
            atomicAdd(cnt + C_NITEMS, 1);
        } else {
            cl_bkt[c] = -1;
            const int k0 = atomicAdd(cnt + C_NFB, np);
            atomicAdd(cnt + C_FBMARK, nm);
            for (int i = 0; i < np; ++i) fb_list[k0 + i] = cl_plist[cl_first[c] + i];
        }
    }
}

__global__ void k_order_fill(const long long *n_clust_d, const int *cl_bkt, const int *bkt_start, int *bkt_cur,
                             int *order) {
    const int n = (int)*n_clust_d;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const int b = cl_bkt[c];
        if (b < 0) continue;
        order[bkt_start[b] + atomicAdd(bkt_cur + b, 1)] = c;
    }
}

// Padded marker counts in work order (zero past the end of the list).
__global__ void k_gather_nm(int n_max, const int *cnt, const int *order, const int *cl_nm, int *out) {
    const int n = cnt[C_NITEMS];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_max; i += gridDim.x * blockDim.x)
        out[i] = i < n ? cl_nm[order[i]] : 0;
}

__device__ __forceinline__ int lower_bound_int(const int *a, int n, int v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

constexpr int kCapCl = 32;      // clusters per batch

// Work items of the shared-memory kernel.  The padded marker prefix of the
// size-ordered cluster list is cut into windows of `window` markers; the
// clusters that start in one window are split greedily into batches that fit
// one CTA (kCapCl clusters, kCapP particles, `window` markers, max_rows
// row-table entries), so that small clusters share a CTA.
__global__ void k_batch_plan(const int *cnt_in, const int *cum, const int *order, const int *cl_np,
                             const int *cl_nm, const int *cl_box, int window, int max_rows, int2 *batches,
                             int *cnt) {
    const int n_items = cnt_in[C_NITEMS];
    const int nw = (cum[n_items] + window - 1) / window;
    const int cap_m3 = window;
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
        const int c0 = lower_bound_int(cum, n_items, w * window);
        const int c1 = lower_bound_int(cum, n_items, (w + 1) * window);
        int c = c0;
        while (c < c1) {
            const int start = c;
            int nb = 0, np = 0, nm = 0, R = 0;
            while (c < c1 && nb < kCapCl) {
                const int id = order[c];
                const int *box = cl_box + 12 * id;
                const int W = (box[3] - box[0] + 1 + 31) >> 5;
                const int cR = (box[4] - box[1] + 1) * (box[5] - box[2] + 1) * W;
                const int cnp = cl_np[id], cnm = cl_nm[id];
                if (nb > 0 && (np + cnp > kCapP || nm + cnm > cap_m3 || R + cR > max_rows)) break;
                np += cnp; nm += cnm; R += cR; ++nb; ++c;
            }
            batches[atomicAdd(cnt + C_NBATCH, 1)] = make_int2(start, c);
        }
    }
}

// Single-block exclusive scan (same as the set-up scan), local copy.
__global__ void k_scan1(const int *in, int *out, int n, long long *total) {
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

// --------------------------------------------------- shared-memory kernel
//
// Work items.  Clusters on the shared-memory path are ordered by size
// (largest first) and their marker counts, each particle's padded to a whole
// number of 32-marker chunks, are prefix-summed.  The prefix is cut into
// windows of the record path's marker capacity (2048 markers for 1024
// threads); the clusters that start in one window are packed into batches
// that fit one CTA's shared memory (up to kCapCl clusters, kCapP particles, a
// row-table budget and the window), so that small clusters (a single D = 12h
// sphere has 452 markers) share a CTA instead of leaving most of its threads
// idle.  A CTA takes one batch at a time from the list.

struct PS {          // particle record in shared memory
    PInfo P;
    int off[3];      // absolute base cell + off = cell relative to its cluster's box
    int mstart;      // first marker of the particle in the batch (multiple of 32)
    int gid;         // global particle index
    int cl;          // cluster within the batch
};

struct CS {          // cluster record in shared memory
    int x0, y0, z0, Bx, By, Bz, W, R;
    int row0;        // first row-table entry
    int slot0;       // first cell slot (a multiple of 4)
    int ncell;       // touched cells of the cluster
    int shift;       // padding added to the prefix slots of its rows
    int pstart;      // first particle of the cluster in the batch (before sorting)
    int first, np;   // particles in cl_plist
    int scene;
    int wrap;        // bit k: axis k is periodic in the box (whole period; x with ghost columns)
    int n[3];        // the scene's grid
    float dmax, S, invS;
    unsigned umax, emax;   // float bits (non-negative), atomicMax
};

struct KParams {
    const PInfo *P;
    const float *t32;
    const double *t64;
    const int32_t *dims;
    float *const *uf;
    float *const *ff;
    const int *order, *cl_first, *cl_np, *cl_nm, *cl_box, *cl_plist, *cl_scene, *poff;
    int *cl_path;
    const int2 *batches;
    float4 *grec;   // per CTA: 2 * TPB * KM float4 (records a, then b)
    int *cnt, *fb_list, *err;
    const unsigned *dis;   // markers left out near contact (Sec. 2.2.5): one bit per global marker, or NULL
    double *FD, *TD;
    int n_forcing, smem_bytes, max_rows;
    float finv;
};

// Block-wide exclusive scan of one int per thread; returns the prefix, and
// the total through *total (valid after the call).
template <int TPB>
__device__ __forceinline__ int block_excl_scan(int v, int *sh, int *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = lane < TPB / 32 ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < TPB / 32) sh[lane] = w;   // inclusive warp totals
    }
    __syncthreads();
    const int pre = (wid ? sh[wid - 1] : 0) + x - v;
    *total = sh[TPB / 32 - 1];
    __syncthreads();
    return pre;
}

// Box-relative base cell and fractional position of a marker (FP32 path).
// Along a periodic axis of the box the base is first taken modulo the period.
__device__ __forceinline__ void rel_base(const PS &s, const CS &cs, const float *t32, const double *t64, int l,
                                         int b[3], float f[3]) {
    const float *t = t32 + 3ll * (s.P.toff + l);
    const double *t6 = t64 + 3ll * (s.P.toff + l);
    const int wrap = cs.wrap;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int raw = marker_split32(s.P, t, t6, c, &f[c]);
        b[c] = (wrap && ((wrap >> c) & 1) ? wrapi(raw, cs.n[c]) : raw) + s.off[c];
    }
}

// Box row of stencil row (dz, dy) of a marker with box-relative base b
// (modulo the period along periodic y or z).
__device__ __forceinline__ int box_row(const CS &cs, const int b[3], int dz, int dy) {
    int y = b[1] + dy, z = b[2] + dz;
    if (cs.wrap & 2) y = wrapi(y, cs.By);
    if (cs.wrap & 4) z = wrapi(z, cs.Bz);
    return z * cs.By + y;
}

// Slots of the nine row runs of a marker's stencil.  rix (sparse row table)
// maps a box row to its compact row, nullptr for the dense table.
__device__ __forceinline__ void row_slots(const uint2 *rt, const unsigned short *rix, const CS &cs, const int b[3],
                                          int slot[9]) {
    const int x = b[0] - 1;
    const int wx = x >> 5;
    const unsigned lowmask = (1u << (x & 31)) - 1u;
    const int W = cs.W, By = cs.By;
    const bool wrap = cs.wrap != 0;
#pragma unroll
    for (int dz = 0; dz < 3; ++dz)
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            const int r = wrap ? box_row(cs, b, dz - 1, dy - 1) : (b[2] + dz - 1) * By + (b[1] + dy - 1);
            const int row = rix ? (int)rix[r] : r;
            const uint2 e = rt[row * W + wx];
            slot[dz * 3 + dy] = (int)e.y + __popc(e.x & lowmask);
        }
}

__device__ __forceinline__ void cp_async4(void *smem_ptr, const void *gmem_ptr) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_ptr);
    // no memory clobber: nothing reads the target before cp_async_wait_all
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_ptr));
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <int TPB, int KM>
__host__ __device__ constexpr int fixed_smem_bytes() {
    // particle and cluster tables, chunk sums, chunk -> particle; the row table
    // that follows starts 16-byte aligned
    return (int)(((sizeof(PS) * kCapP + sizeof(CS) * kCapCl + sizeof(float) * (TPB * KM / 32) * 6 +
                   ((TPB * KM / 32 + 15) & ~15)) + 15) & ~15);
}

struct Batch {
    int nb, np, nm, R, C;
    int gx;                      // some cluster is periodic in x (ghost columns)
    const unsigned short *rix;   // sparse row table: box row -> compact row (else nullptr)
    const unsigned short *rowid; // sparse row table: compact row -> box row
};


// Gather (LOAD) or write back the touched cells of components q0..q0+NC-1 of
// every cluster of the batch, cluster by cluster (its box and scene are
// uniform in the loop).  With the slot table s_inv (slot -> bitmask entry)
// consecutive threads take consecutive slots, i.e. consecutive cells of a row
// run, so the global accesses coalesce; without it one thread walks the set
// bits of one bitmask entry.
template <int TPB, int NC, bool LOAD>
__device__ __forceinline__ void move_cells(const KParams &prm, const Batch &bt, const CS *s_cs, const uint2 *s_row,
                                           const unsigned short *s_inv, float *s_u, int q0) {
    const int tid = threadIdx.x, C = bt.C;
    for (int j = 0; j < bt.nb; ++j) {
        const int sc0 = s_cs[j].scene;
        // box origin taken into the period once; a cell's coordinate is then the
        // origin plus at most the box extent (<= period + 2), i.e. below 3 periods
        const int x0 = wrapi(s_cs[j].x0, prm.dims[3 * sc0]), y0 = wrapi(s_cs[j].y0, prm.dims[3 * sc0 + 1]),
                  z0 = wrapi(s_cs[j].z0, prm.dims[3 * sc0 + 2]);
        const int W = s_cs[j].W, By = s_cs[j].By, row0 = s_cs[j].row0;
        const int sc = s_cs[j].scene;
        // ghost columns of a box periodic in x are copies: gathered, not written back
        const bool skip_ghosts = !LOAD && (s_cs[j].wrap & 1);
        const int Bx = s_cs[j].Bx;
        const int nx = prm.dims[3 * sc], ny = prm.dims[3 * sc + 1], nz = prm.dims[3 * sc + 2];
        const long long ncell = (long long)nx * ny * nz;
        float *u = prm.uf[sc] + (long long)q0 * ncell;
        float *f = prm.ff ? prm.ff[sc] + (long long)q0 * ncell : nullptr;
        float *su = s_u + s_cs[j].slot0;   // this cluster's slots, component q0
        // entry -> (row, word) -> (ry, rz): exact small-integer divisions in FP32
        const float rW = __frcp_rn((float)W), rBy = __frcp_rn((float)By);
        auto row_base = [&](int li, int &wx) {
            const int rc = (int)(((float)li + 0.5f) * rW);
            wx = li - rc * W;
            const int row = bt.rowid ? (int)bt.rowid[rc] : rc;
            const int rz = (int)(((float)row + 0.5f) * rBy);
            const int ry = row - rz * By;
            return ((long long)wrap_lt3(z0 + rz, nz) * ny + wrap_lt3(y0 + ry, ny)) * nx;
        };
        auto move = [&](long long g, int sl) {
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                if (LOAD) {
                    cp_async4(su + q * C + sl, u + q * ncell + g);
                } else {
                    const float v = su[q * C + sl];
                    if (f) f[q * ncell + g] = (v - u[q * ncell + g]) * prm.finv;
                    u[q * ncell + g] = v;
                }
            }
        };
        if (s_inv) {
            const int base = s_cs[j].slot0;
            for (int sl = tid; sl < s_cs[j].ncell; sl += TPB) {
                const unsigned i = s_inv[base + sl];
                const uint2 rw = s_row[i];
                int wx;
                const long long rb = row_base((int)i - row0, wx);
                const int xb = 32 * wx + (int)__fns(rw.x, 0u, base + sl - (int)rw.y + 1);
                if (skip_ghosts && (xb == 0 || xb == Bx - 1)) continue;
                move(rb + wrap_lt3(x0 + xb, nx), sl);
            }
        } else {
            for (int li = tid; li < s_cs[j].R; li += TPB) {
                unsigned mask = s_row[row0 + li].x;
                if (!mask) continue;
                int wx;
                const long long rb = row_base(li, wx);
                int sl = (int)s_row[row0 + li].y - s_cs[j].slot0;
                while (mask) {
                    const int xb = 32 * wx + __ffs(mask) - 1;
                    mask &= mask - 1u;
                    if (!(skip_ghosts && (xb == 0 || xb == Bx - 1))) move(rb + wrap_lt3(x0 + xb, nx), sl);
                    ++sl;
                }
            }
        }
    }
    if (LOAD) cp_async_wait_all();
}

// Marks the 3x3x3 stencil of a marker (box-relative base cell b) in its
// cluster's row bitmask (rows through rix for the sparse table); false if the
// stencil leaves the box (never expected: the box bounds every stencil of the
// cluster).
__device__ __forceinline__ bool in_box(const CS &cs, const int b[3]) {
    // along periodic y or z every row of the period is in the box
    return b[0] >= 1 && b[0] <= cs.Bx - 2 &&
           ((cs.wrap & 2) ? (b[1] >= 0 && b[1] < cs.By) : (b[1] >= 1 && b[1] <= cs.By - 2)) &&
           ((cs.wrap & 4) ? (b[2] >= 0 && b[2] < cs.Bz) : (b[2] >= 1 && b[2] <= cs.Bz - 2));
}

// Along periodic x, box columns 0 and Bx-1 are ghosts of the period's last
// and first column (box columns Bx-2 and 1); a stencil that reaches a ghost
// also marks its partner, so that both copies have slots.
__device__ __forceinline__ bool mark_stencil(uint2 *rt, const unsigned short *rix, const CS &cs, const int b[3]) {
    if (!cs.wrap) {
        // a box that is not periodic: plain row arithmetic
        const int Bx = cs.Bx, By = cs.By, Bz = cs.Bz, W = cs.W;
        if (b[0] < 1 || b[0] > Bx - 2 || b[1] < 1 || b[1] > By - 2 || b[2] < 1 || b[2] > Bz - 2) return false;
        const int x = b[0] - 1, wx = x >> 5, bit = x & 31;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const int r = (b[2] + dz) * By + (b[1] + dy);
                const int row = rix ? (int)rix[r] : r;
                atomicOr(&rt[row * W + wx].x, 7u << bit);
                if (bit > 29) atomicOr(&rt[row * W + wx + 1].x, 7u >> (32 - bit));
            }
        return true;
    }
    if (!in_box(cs, b)) return false;
    const int x = b[0] - 1, wx = x >> 5, bit = x & 31;
    const bool gl = (cs.wrap & 1) && b[0] == 1, gr = (cs.wrap & 1) && b[0] == cs.Bx - 2;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int r = box_row(cs, b, dz, dy);
            const int row = rix ? (int)rix[r] : r;
            atomicOr(&rt[row * cs.W + wx].x, 7u << bit);
            if (bit > 29) atomicOr(&rt[row * cs.W + wx + 1].x, 7u >> (32 - bit));
            if (gl) atomicOr(&rt[row * cs.W + ((cs.Bx - 2) >> 5)].x, 1u << ((cs.Bx - 2) & 31));
            if (gr) atomicOr(&rt[row * cs.W].x, 2u);
        }
    return true;
}

// Slot of box column x in a row's bitmask entries e (bit assumed set).
__device__ __forceinline__ int col_slot(const uint2 *e, int x) {
    const uint2 w = e[x >> 5];
    return (int)w.y + __popc(w.x & ((1u << (x & 31)) - 1u));
}

// Ghost columns of the clusters that are periodic in x: G = 0 copies the real
// cells into the ghosts (before an interpolation), G = 1 zeroes the ghosts
// (before spreading), G = 2 adds the ghosts' spread contributions to the real
// cells (after spreading; integer adds in deterministic mode, so the sum is
// exact).
template <int TPB, int NC, int G, bool DET>
__device__ __forceinline__ void ghost_pass(const Batch &bt, const CS *s_cs, const uint2 *s_row, float *s_u) {
    const int C = bt.C;
    for (int j = 0; j < bt.nb; ++j) {
        if (!(s_cs[j].wrap & 1)) continue;
        const int W = s_cs[j].W, Bx = s_cs[j].Bx, nrow = s_cs[j].R / W;
        for (int k = threadIdx.x; k < 2 * nrow; k += TPB) {
            const uint2 *e = s_row + s_cs[j].row0 + (k >> 1) * W;
            const int gx = (k & 1) ? Bx - 1 : 0, rx = (k & 1) ? 1 : Bx - 2;
            if (!((e[gx >> 5].x >> (gx & 31)) & 1u)) continue;
            const int g = col_slot(e, gx), r = col_slot(e, rx);
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                float *ug = s_u + q * C + g, *ur = s_u + q * C + r;
                if (G == 0) *ug = *ur;
                else if (G == 1) *ug = 0.f;
                else if (DET) *reinterpret_cast<int *>(ur) += *reinterpret_cast<const int *>(ug);
                else *ur += *ug;
            }
        }
    }
}

// Deterministic mode keeps the touched cells in fixed point while markers
// spread into them: value = round(u 2^k) in int32, with one power-of-two
// scale per cluster and iteration.  The scale comes from a running bound B on
// |u| over the cluster's cells: B_0 = max |u^0| (one scan after the gather),
// and before the spreading of iteration m, B_m = B_{m-1} + 64 Dmax max|e^m|,
// which bounds |u^m| as long as no cell collects more than 64 unit weights
// (Sec. 2.2.2: u^m = u^{m-1} + W^T D e^m).  2^k is the largest power of two
// with B_m 2^k < 2^28.  Integer addition wraps modulo 2^32 and is associative,
// so partial sums may wrap harmlessly; a final cell value above 2^28 in
// magnitude means the weight bound was broken (particles overlapping far more
// than non-overlapping spheres can) and sets IBM_EBIT_FIXEDPOINT on the way
// back to floating point; only a violation by more than a factor of about 15
// can wrap back into range unseen.  The
// scale depends only on the cluster, never on how clusters are batched or on
// the order of the atomic additions, so the result is bit-reproducible.
// The per-cluster slot ranges start at multiples of 4 and their padding is
// zero, so the passes use 16-byte accesses.

// B_0: max |u| over components 0..NC-1 of each cluster's cells (umax must be
// zero on entry).
template <int TPB, int NC>
__device__ __forceinline__ void det_scan(const Batch &bt, CS *s_cs, const float *s_u) {
    const int C = bt.C;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int j = 0; j < bt.nb; ++j) {
        const int n4 = (s_cs[j].ncell + 3) >> 2;
        float um = 0.f;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            const float4 *p = reinterpret_cast<const float4 *>(s_u + q * C + s_cs[j].slot0);
            for (int i = tid; i < n4; i += TPB) {
                const float4 v = p[i];
                um = fmaxf(um, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
            }
        }
        um = warp_max(um);
        if (lane == 0 && um > 0.f) atomicMax(&s_cs[j].umax, __float_as_uint(um));
    }
}

// Scale of this iteration from the bound and the iteration's max |e| (one
// thread per cluster); advances the bound and clears max |e| for the next
// iteration.
template <int TPB>
__device__ __forceinline__ void det_scale(const Batch &bt, CS *s_cs) {
    for (int j = threadIdx.x; j < bt.nb; j += TPB) {
        const float range = __uint_as_float(s_cs[j].umax) + 64.f * s_cs[j].dmax * __uint_as_float(s_cs[j].emax);
        int ex = 100;
        if (range > 0.f) ex = min(100, max(-100, 27 - (int)ceilf(log2f(range))));
        s_cs[j].S = ldexpf(1.f, ex);
        s_cs[j].invS = ldexpf(1.f, -ex);
        s_cs[j].umax = __float_as_uint(range);
        s_cs[j].emax = 0u;
    }
}

// u -> round(u S) (TO) or back, components 0..NC-1 of every cluster.
template <int TPB, int NC, bool TO>
__device__ __forceinline__ void det_convert(const Batch &bt, const CS *s_cs, float *s_u, int *err) {
    const int C = bt.C;
    const int tid = threadIdx.x;
    bool out_of_range = false;
    for (int j = 0; j < bt.nb; ++j) {
        const int n4 = (s_cs[j].ncell + 3) >> 2;
        const float S = TO ? s_cs[j].S : s_cs[j].invS;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            float4 *p = reinterpret_cast<float4 *>(s_u + q * C + s_cs[j].slot0);
            for (int i = tid; i < n4; i += TPB) {
                if (TO) {
                    const float4 v = p[i];
                    int4 r;
                    r.x = __float2int_rn(v.x * S); r.y = __float2int_rn(v.y * S);
                    r.z = __float2int_rn(v.z * S); r.w = __float2int_rn(v.w * S);
                    reinterpret_cast<int4 *>(p)[i] = r;
                } else {
                    const int4 r = reinterpret_cast<const int4 *>(p)[i];
                    constexpr int kLim = 1 << 28;
                    out_of_range |= abs(r.x) > kLim || abs(r.y) > kLim || abs(r.z) > kLim || abs(r.w) > kLim;
                    p[i] = make_float4((float)r.x * S, (float)r.y * S, (float)r.z * S, (float)r.w * S);
                }
            }
        }
    }
    if (!TO && out_of_range) set_err(err, IBM_EBIT_FIXEDPOINT);
}

// Zero the padding slots of every cluster (components 0..NC-1).
template <int TPB, int NC>
__device__ __forceinline__ void zero_padding(const Batch &bt, const CS *s_cs, float *s_u) {
    const int C = bt.C;
    for (int j = threadIdx.x; j < bt.nb; j += TPB) {
        const int s0 = s_cs[j].slot0 + s_cs[j].ncell, s1 = s_cs[j].slot0 + ((s_cs[j].ncell + 3) & ~3);
        for (int q = 0; q < NC; ++q)
            for (int i = s0; i < s1; ++i) s_u[q * C + i] = 0.f;
    }
}

// Gather components q0..q0+NC-1 of the touched cells, zero the padding and,
// in deterministic mode, start the bound of the fixed-point scale.
template <int TPB, int NC, bool DET>
__device__ __forceinline__ void load_cells(const KParams &prm, const Batch &bt, CS *s_cs, const uint2 *s_row,
                                           const unsigned short *s_inv, float *s_u, int q0) {
    for (int j = threadIdx.x; j < bt.nb; j += TPB) { s_cs[j].umax = 0u; s_cs[j].emax = 0u; }
    move_cells<TPB, NC, true>(prm, bt, s_cs, s_row, s_inv, s_u, q0);
    __syncthreads();
    zero_padding<TPB, NC>(bt, s_cs, s_u);
    __syncthreads();
    if (DET) det_scan<TPB, NC>(bt, s_cs, s_u);
}

constexpr unsigned kNoMarker = 0xffffffffu;   // record of a padding marker

// Slot i (0..8, row dz*3+dy) of a marker record: rows 0..7 packed two per
// word in rb, row 8 in the low bits of ra.w.
__device__ __forceinline__ int rec_slot(const uint4 &rb, unsigned s8, int i) {
    const unsigned wd = i < 2 ? rb.x : (i < 4 ? rb.y : (i < 6 ? rb.z : rb.w));
    return i == 8 ? (int)s8 : (int)((wd >> ((i & 1) * 16)) & 0xffffu);
}

// The outer forcing loop (Sec. 2.2.2) for components q0..q0+NC-1 of a batch,
// on its touched cells in shared memory.  Each marker's stencil is a record
// built once per step: ra[m] = (fractional position, slot of row 8), rb[m] =
// slots of rows 0..7, in shared memory when they fit there and in global
// memory (L2) otherwise, so that each iteration only recomputes the nine
// phi_3 weights.  Components are independent in the loop, so a batch too
// large for all three runs them one at a time (NC = 1).  Markers m = tid +
// k TPB, k < KR; e^m stays in registers between interpolation and spreading.
// The per-chunk load sums are taken every iteration (FP32 warp sums of 32
// markers of one particle; FP64 across chunks at the end).
template <int TPB, int KR, bool DET, int NC>
__device__ __forceinline__ void forcing_rec(const KParams &prm, const Batch &bt, const PS *s_ps, CS *s_cs,
                                            float *s_part, const unsigned char *s_chunk, const uint2 *s_row,
                                            const unsigned short *s_inv, float *s_u, const float4 *ra,
                                            const uint4 *rb, int q0) {
    int *s_ui = reinterpret_cast<int *>(s_u);
    const int tid = threadIdx.x, lane = tid & 31;
    const int C = bt.C, nm = bt.nm;
    load_cells<TPB, NC, DET>(prm, bt, s_cs, s_row, s_inv, s_u, q0);
    for (int iter = 0; iter < prm.n_forcing; ++iter) {
        if (bt.gx && iter > 0) {
            ghost_pass<TPB, NC, 0, DET>(bt, s_cs, s_row, s_u);
            __syncthreads();
        }
        float e[KR][NC];
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            const int m = tid + k * TPB;
#pragma unroll
            for (int q = 0; q < NC; ++q) e[k][q] = 0.f;
            if (m - lane >= nm) continue;   // whole warp past the end
            float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            float em = 0.f;
            const float4 a = ra[m];
            const PS &s = s_ps[s_chunk[m >> 5]];
            bool live = __float_as_uint(a.w) != kNoMarker;
            if (live && prm.dis) {
                // a marker left out near contact (Sec. 2.2.5) keeps e = 0: no force, nothing spread
                const long long mk = (long long)s.P.moff + (m - s.mstart);
                live = !((prm.dis[mk >> 5] >> (mk & 31)) & 1u);
            }
            if (live) {
                const uint4 r = rb[m];
                const unsigned s8 = __float_as_uint(a.w);
                float w[3][3];
                phi3_weights(a.x, w[0]);
                phi3_weights(a.y, w[1]);
                phi3_weights(a.z, w[2]);
                float U[NC];
#pragma unroll
                for (int q = 0; q < NC; ++q) U[q] = 0.f;
#pragma unroll
                for (int dz = 0; dz < 3; ++dz)
#pragma unroll
                    for (int dy = 0; dy < 3; ++dy) {
                        const int sl = rec_slot(r, s8, dz * 3 + dy);
                        const float wyz = w[2][dz] * w[1][dy];
                        const float a0 = wyz * w[0][0], a1 = wyz * w[0][1], a2 = wyz * w[0][2];
#pragma unroll
                        for (int q = 0; q < NC; ++q)
                            U[q] += a0 * s_u[q * C + sl] + a1 * s_u[q * C + sl + 1] + a2 * s_u[q * C + sl + 2];
                    }
                // desired velocity U^d = u_p + w_p x r_l (Sec. 2.1), from the particle record
                const float *t = prm.t32 + 3ll * (s.P.toff + (m - s.mstart));
                const float r0 = s.P.rphys * t[0], r1 = s.P.rphys * t[1], r2 = s.P.rphys * t[2];
                const float ud0 = s.P.ud[0] + (s.P.om[1] * r2 - s.P.om[2] * r1);
                const float ud1 = s.P.ud[1] + (s.P.om[2] * r0 - s.P.om[0] * r2);
                const float ud2 = s.P.ud[2] + (s.P.om[0] * r1 - s.P.om[1] * r0);
                const float D = s.P.D;
                float ed[3];
                if (NC == 3) {
                    e[k][0] = ud0 - U[0];
                    e[k][NC > 1 ? 1 : 0] = ud1 - U[NC > 1 ? 1 : 0];
                    e[k][NC > 2 ? 2 : 0] = ud2 - U[NC > 2 ? 2 : 0];
                    em = fmaxf(fabsf(e[k][0]), fmaxf(fabsf(e[k][NC > 1 ? 1 : 0]), fabsf(e[k][NC > 2 ? 2 : 0])));
                    ed[0] = e[k][0] * D; ed[1] = e[k][NC > 1 ? 1 : 0] * D; ed[2] = e[k][NC > 2 ? 2 : 0] * D;
                } else {
                    const float x = (q0 == 0 ? ud0 : (q0 == 1 ? ud1 : ud2)) - U[0];
                    e[k][0] = x;
                    em = fabsf(x);
                    ed[0] = q0 == 0 ? x * D : 0.f;
                    ed[1] = q0 == 1 ? x * D : 0.f;
                    ed[2] = q0 == 2 ? x * D : 0.f;
                }
                v[0] = ed[0]; v[1] = ed[1]; v[2] = ed[2];
                v[3] = r1 * ed[2] - r2 * ed[1];
                v[4] = r2 * ed[0] - r0 * ed[2];
                v[5] = r0 * ed[1] - r1 * ed[0];
            }
            // the 32 lanes of a warp hold markers of one particle: warp sums into
            // the chunk table (FP32 over 32 terms; FP64 across chunks at the end)
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                if (NC == 1 && ((q < 3 && q != q0) || q == 3 + q0)) continue;   // zero in this pass
                const float x = warp_sum(v[q]);
                if (lane == 0) s_part[(m >> 5) * 6 + q] += x;
            }
            if (DET) {
                const float wm = warp_max(em);
                if (lane == 0) atomicMax(&s_cs[s.cl].emax, __float_as_uint(wm));
            }
        }
        __syncthreads();
        if (DET) {
            det_scale<TPB>(bt, s_cs);
            __syncthreads();
            det_convert<TPB, NC, true>(bt, s_cs, s_u, prm.err);
            __syncthreads();
        }
        if (bt.gx) {
            ghost_pass<TPB, NC, 1, DET>(bt, s_cs, s_row, s_u);
            __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            const int m = tid + k * TPB;
            if (m >= nm) continue;
            const float4 a = ra[m];
            if (__float_as_uint(a.w) == kNoMarker) continue;
            const uint4 r = rb[m];
            const unsigned s8 = __float_as_uint(a.w);
            const PS &s = s_ps[s_chunk[m >> 5]];
            const float D = s.P.D * (DET ? s_cs[s.cl].S : 1.f);
            float g[NC];
#pragma unroll
            for (int q = 0; q < NC; ++q) g[q] = e[k][q] * D;
            float w[3][3];
            phi3_weights(a.x, w[0]);
            phi3_weights(a.y, w[1]);
            phi3_weights(a.z, w[2]);
#pragma unroll
            for (int dz = 0; dz < 3; ++dz)
#pragma unroll
                for (int dy = 0; dy < 3; ++dy) {
                    const int sl = rec_slot(r, s8, dz * 3 + dy);
                    const float wyz = w[2][dz] * w[1][dy];
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        const float c = wyz * w[0][dx];
#pragma unroll
                        for (int q = 0; q < NC; ++q) {
                            if (DET) atomicAdd(&s_ui[q * C + sl + dx], __float2int_rn(c * g[q]));
                            else atomicAdd(&s_u[q * C + sl + dx], c * g[q]);
                        }
                    }
                }
        }
        __syncthreads();
        if (bt.gx) {
            ghost_pass<TPB, NC, 2, DET>(bt, s_cs, s_row, s_u);
            __syncthreads();
        }
        if (DET) {
            det_convert<TPB, NC, false>(bt, s_cs, s_u, prm.err);
            __syncthreads();
        }
    }
    move_cells<TPB, NC, false>(prm, bt, s_cs, s_row, s_inv, s_u, q0);
}

template <class T>
__device__ __forceinline__ T *align16_to(const void *q) {
    return reinterpret_cast<T *>((reinterpret_cast<uintptr_t>(q) + 15) & ~(uintptr_t)15);
}

// Sparse row table of a batch holding one large cluster, for when the dense
// table (one entry per 32 cells of every row of the box) does not fit: the
// box rows that some stencil reaches are numbered in order (rix: box row ->
// compact row, rowid: the inverse) and only those get bitmask entries.  The
// markers' base cells come from their records.  On return s_row points to the
// compact entries and bt holds the tables; *flag is set when they do not fit.
template <int TPB>
__device__ __noinline__ void build_sparse_rows(CS *s_cs, const float4 *ra, int nm, uint2 *base, const unsigned char *dyn_end,
                                  int *s_scan, int *flag, Batch &bt, uint2 *&s_row) {
    const int tid = threadIdx.x;
    CS &cs = s_cs[0];
    const int W = cs.W, nyz = cs.By * cs.Bz;
    unsigned short *rix = reinterpret_cast<unsigned short *>(base);
    unsigned *rbits = align16_to<unsigned>(rix + nyz);
    const int nw = (nyz + 31) >> 5;
    uint2 *rows = align16_to<uint2>(rbits + nw);
    bool ok = !*flag && reinterpret_cast<const unsigned char *>(rows) + 16 <= dyn_end;   // uniform
    int nrows = 0;
    if (ok) {
        for (int i = tid; i < nw; i += TPB) rbits[i] = 0u;
        __syncthreads();
        for (int m = tid; m < nm; m += TPB) {
            const unsigned bp = __float_as_uint(ra[m].w);
            if (bp == kNoMarker) continue;
            const int b[3] = {0, (int)((bp >> 10) & 1023u), (int)(bp >> 20)};
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy) {
                    const int r = box_row(cs, b, dz, dy);
                    atomicOr(&rbits[r >> 5], 1u << (r & 31));
                }
        }
        __syncthreads();
        const int per = (nw + TPB - 1) / TPB;
        const int lo = min(nw, tid * per), hi = min(nw, lo + per);
        int sum = 0;
        for (int i = lo; i < hi; ++i) sum += __popc(rbits[i]);
        int run = block_excl_scan<TPB>(sum, s_scan, &nrows);
        unsigned short *rowid = align16_to<unsigned short>(rows + nrows * W);
        ok = reinterpret_cast<const unsigned char *>(rowid + nrows) + 16 <= dyn_end;   // uniform
        if (ok) {
            for (int i = lo; i < hi; ++i) {
                unsigned bits = rbits[i];
                while (bits) {
                    const int r = 32 * i + __ffs(bits) - 1;
                    bits &= bits - 1u;
                    rix[r] = (unsigned short)run;
                    rowid[run] = (unsigned short)r;
                    ++run;
                }
            }
            for (int i = tid; i < nrows * W; i += TPB) rows[i] = make_uint2(0u, 0u);
            __syncthreads();
            for (int m = tid; m < nm; m += TPB) {
                const unsigned bp = __float_as_uint(ra[m].w);
                if (bp == kNoMarker) continue;
                const int b[3] = {(int)(bp & 1023u), (int)((bp >> 10) & 1023u), (int)(bp >> 20)};
                mark_stencil(rows, rix, cs, b);
            }
            bt.rix = rix;
            bt.rowid = rowid;
        }
    }
    if (!ok) {
        nrows = 0;
        if (tid == 0) *flag = 1;
    }
    __syncthreads();
    bt.R = nrows * W;
    if (tid == 0) {
        cs.row0 = 0;
        cs.R = bt.R;
    }
    __syncthreads();
    s_row = rows;
}

// Persistent CTAs (MINB per SM).  KM: markers per thread of a batch (at most
// TPB KM markers, one component at a time; TPB KM / 3 with all three); KR:
// markers per thread when the records stay in shared memory.  DET =
// fixed-point spreading (int32 shared-memory atomics, bit-reproducible and
// independent of how clusters are batched).
template <int TPB, int KM, int KR, bool DET, int MINB>
__global__ void __launch_bounds__(TPB, MINB) k_cluster_forcing(KParams prm) {
    constexpr int NCH = TPB * KM / 32;   // 32-marker chunks
    extern __shared__ __align__(16) unsigned char smem[];
    PS *s_ps = reinterpret_cast<PS *>(smem);
    CS *s_cs = reinterpret_cast<CS *>(s_ps + kCapP);
    float *s_part = reinterpret_cast<float *>(s_cs + kCapCl);            // [NCH][6]
    unsigned char *s_chunk = reinterpret_cast<unsigned char *>(s_part + NCH * 6);   // [NCH] chunk -> particle
    uint2 *const s_row0 = reinterpret_cast<uint2 *>(smem + fixed_smem_bytes<TPB, KM>());   // [R] then the cells
    unsigned char *dyn_end = smem + prm.smem_bytes;
    __shared__ int s_w, s_np, s_nm, s_R, s_flag, s_scan[32], s_total;
    const int tid = threadIdx.x;
    const int n_batches = prm.cnt[C_NBATCH];

    for (;;) {
        if (tid == 0) s_w = atomicAdd(prm.cnt + C_WORK, 1);
        __syncthreads();
        const int w = s_w;
        if (w >= n_batches) break;
        {
            const int2 be = prm.batches[w];
            const int nbl = be.y - be.x;
            // cluster records, loaded in parallel; prefix sums over the batch in warp 0
            if (tid < 32) {
                int cnp = 0, cR = 0;
                if (tid < nbl) {
                    const int id = prm.order[be.x + tid];
                    const int *box = prm.cl_box + 12 * id;
                    CS &cs = s_cs[tid];
                    cs.x0 = box[0]; cs.y0 = box[1]; cs.z0 = box[2];
                    cs.Bx = box[3] - box[0] + 1; cs.By = box[4] - box[1] + 1; cs.Bz = box[5] - box[2] + 1;
                    cs.W = (cs.Bx + 31) >> 5;
                    cs.R = cs.By * cs.Bz * cs.W;
                    cs.first = prm.cl_first[id];
                    cs.np = prm.cl_np[id];
                    const int sw = prm.cl_scene[id];
                    cs.scene = sw & 0x0fffffff;
                    cs.wrap = sw >> 28;
                    cs.n[0] = prm.dims[3 * cs.scene];
                    cs.n[1] = prm.dims[3 * cs.scene + 1];
                    cs.n[2] = prm.dims[3 * cs.scene + 2];
                    cnp = cs.np;
                    cR = cs.R;
                }
                int sp = cnp, sr = cR;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int a1 = __shfl_up_sync(0xffffffffu, sp, o), a2 = __shfl_up_sync(0xffffffffu, sr, o);
                    if (tid >= o) { sp += a1; sr += a2; }
                }
                if (tid < nbl) {
                    s_cs[tid].pstart = sp - cnp;
                    s_cs[tid].row0 = sr - cR;
                }
                if (tid == 31) { s_np = sp; s_R = sr; }
                if (tid == 0) s_flag = 0;
            }
            __syncthreads();
            // batch-wide values live in shared memory (every thread writes the same
            // value), which keeps them out of the registers of the forcing loop
            __shared__ Batch s_bt;
            Batch &bt = s_bt;
            bt.nb = nbl;
            bt.np = s_np;
            bt.R = s_R;
            bt.rix = nullptr;
            bt.rowid = nullptr;
            {
                int gx = 0;
                for (int j = 0; j < nbl; ++j) gx |= s_cs[j].wrap & 1;
                bt.gx = gx;
            }
            const int np = bt.np;
            // a single cluster whose dense row table is too large gets a sparse one
            const bool sparse = bt.nb == 1 && bt.R > prm.max_rows;
            uint2 *s_row = s_row0;
            // particle table, sorted by global index (fixed marker numbering): warp 0,
            // lane i ranks its particle among the batch's (np <= 32, indices distinct)
            if (tid < 32) {
                int gid = INT_MAX, cl = 0;
                if (tid < np) {
                    int lo = 0, hi = bt.nb - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (s_cs[mid].pstart <= tid) lo = mid;
                        else hi = mid - 1;
                    }
                    cl = lo;
                    gid = prm.cl_plist[s_cs[lo].first + tid - s_cs[lo].pstart];
                }
                int rank = 0;
#pragma unroll
                for (int j = 0; j < 32; ++j) rank += __shfl_sync(0xffffffffu, gid, j) < gid;
                if (tid < np) {
                    s_ps[rank].gid = gid;
                    s_ps[rank].cl = cl;
                }
                if (tid < bt.nb) s_cs[tid].dmax = 0.f;
            }
            __syncthreads();
            if (tid < np) {
                const int p = s_ps[tid].gid;
                const CS &cs = s_cs[s_ps[tid].cl];
                s_ps[tid].P = prm.P[p];
                // periodic axes of the box take the base modulo the period instead
                s_ps[tid].off[0] = ((cs.wrap & 1) ? 0 : prm.poff[3 * p]) - cs.x0;
                s_ps[tid].off[1] = ((cs.wrap & 2) ? 0 : prm.poff[3 * p + 1]) - cs.y0;
                s_ps[tid].off[2] = ((cs.wrap & 4) ? 0 : prm.poff[3 * p + 2]) - cs.z0;
            }
            if (!sparse)
                for (int i = tid; i < bt.R; i += TPB) s_row[i].x = 0u;
            __syncthreads();
            if (tid < 32) {
                // first marker of each particle (padded to 32-marker chunks): warp scan;
                // largest D of each cluster (non-negative float bits order like ints)
                const int pad = tid < np ? (s_ps[tid].P.nl + 31) & ~31 : 0;
                int inc = pad;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, inc, o);
                    if (tid >= o) inc += y;
                }
                if (tid < np) {
                    s_ps[tid].mstart = inc - pad;
                    atomicMax(reinterpret_cast<unsigned *>(&s_cs[s_ps[tid].cl].dmax), __float_as_uint(s_ps[tid].P.D));
                }
                if (tid == 31) s_nm = inc;
            }
            __syncthreads();
            bt.nm = s_nm;
            const int nm = bt.nm;
            for (int i = tid; i < (nm >> 5) * 6; i += TPB) s_part[i] = 0.f;
            for (int i = tid; i < np; i += TPB)
                for (int ch = s_ps[i].mstart >> 5; ch < (s_ps[i].mstart + s_ps[i].P.nl + 31) >> 5; ++ch)
                    s_chunk[ch] = (unsigned char)i;
            __syncthreads();

            // 1. touched-cell bitmask of every cluster (bounds-checked), and each
            // marker's record: fractional position and packed box-relative base cell
            // (the base becomes the nine row slots after step 2).  The records go to
            // the top of shared memory when they fit there beside the row table,
            // else to this CTA's slice of a global scratch (a few hundred KB, served
            // from L2).
            const int rec_bytes = 32 * nm;
            float4 *const s_ra = reinterpret_cast<float4 *>(dyn_end - rec_bytes);
            uint4 *const s_rb = reinterpret_cast<uint4 *>(dyn_end - rec_bytes / 2);
            float4 *const g_ra = prm.grec + (size_t)blockIdx.x * (2 * TPB * KM);
            uint4 *const g_rb = reinterpret_cast<uint4 *>(g_ra + TPB * KM);
            const bool rec_smem = !sparse && nm <= TPB * KR &&
                                  reinterpret_cast<unsigned char *>(s_row + bt.R) + 16 <= dyn_end - rec_bytes;
            float4 *const ra0 = rec_smem ? s_ra : g_ra;
            for (int m = tid; m < nm; m += TPB) {
                const PS &s = s_ps[s_chunk[m >> 5]];
                const int l = m - s.mstart;
                if (l >= s.P.nl) {
                    ra0[m] = make_float4(0.f, 0.f, 0.f, __uint_as_float(kNoMarker));
                    continue;
                }
                int b[3];
                float f[3];
                const CS &cs = s_cs[s.cl];
                rel_base(s, cs, prm.t32, prm.t64, l, b, f);
                if (!sparse && !mark_stencil(s_row + cs.row0, nullptr, cs, b)) s_flag = 1;
                if (sparse && !in_box(cs, b)) s_flag = 1;
                ra0[m] = make_float4(f[0], f[1], f[2],
                                     __uint_as_float((unsigned)b[0] | ((unsigned)b[1] << 10) | ((unsigned)b[2] << 20)));
            }
            __syncthreads();
            if (sparse)
                build_sparse_rows<TPB>(s_cs, ra0, nm, s_row0, dyn_end, s_scan, &s_flag, bt, s_row);
            // 2. compact slots: exclusive prefix of the popcounts over all rows, then
            // each cluster's slots shifted to start at a multiple of 4 (so that the
            // per-cluster passes over the cells can use 16-byte accesses)
            auto slot_prefix = [&]() {
                const int per = (bt.R + TPB - 1) / TPB;
                const int lo = min(bt.R, tid * per), hi = min(bt.R, lo + per);
                int sum = 0;
                for (int i = lo; i < hi; ++i) sum += __popc(s_row[i].x);
                int total;
                int run = block_excl_scan<TPB>(sum, s_scan, &total);
                for (int i = lo; i < hi; ++i) {
                    s_row[i].y = (unsigned)run;
                    run += __popc(s_row[i].x);
                }
                __syncthreads();
                if (tid < 32) {
                    // warp 0: per-cluster padded slot offsets
                    int c0 = 0, cnt = 0;
                    if (tid < bt.nb) {
                        c0 = (int)s_row[s_cs[tid].row0].y;
                        const int c1 = tid + 1 < bt.nb ? (int)s_row[s_cs[tid + 1].row0].y : total;
                        cnt = c1 - c0;
                    }
                    const int padded = (cnt + 3) & ~3;
                    int inc = padded;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int a1 = __shfl_up_sync(0xffffffffu, inc, o);
                        if (tid >= o) inc += a1;
                    }
                    if (tid < bt.nb) {
                        s_cs[tid].slot0 = inc - padded;
                        s_cs[tid].ncell = cnt;
                        s_cs[tid].shift = (inc - padded) - c0;
                    }
                    if (tid == 31) s_total = inc;
                }
                __syncthreads();
                for (int j = 0; j < bt.nb; ++j) {
                    const unsigned sh = (unsigned)s_cs[j].shift;
                    const int r1 = s_cs[j].row0 + s_cs[j].R;
                    for (int i = s_cs[j].row0 + tid; i < r1; i += TPB)
                        if (s_row[i].x) s_row[i].y += sh;
                }
                __syncthreads();
                bt.C = s_total;
            };
            slot_prefix();
            // the row structures end before the slot table and the cells
            auto rows_end = [&]() {
                return bt.rowid ? reinterpret_cast<const void *>(bt.rowid + bt.R / s_cs[0].W)
                                : reinterpret_cast<const void *>(s_row + bt.R);
            };
            // cells go right after the row table, or after a slot -> entry table when
            // that fits too (it lets the gather/writeback run one thread per cell)
            auto align16 = [](const void *q) {
                return reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(q) + 15) & ~(uintptr_t)15);
            };
            auto cells_cap = [&]() {
                return (int)((dyn_end - reinterpret_cast<unsigned char *>(align16(rows_end()))) / 4);
            };
            if (!sparse && !rec_smem && !s_flag && bt.nb == 1 && bt.C > cells_cap()) {
                // a single large cluster whose dense row table leaves too little room:
                // rebuild it sparse from the records (in global memory) and redo the slots
                build_sparse_rows<TPB>(s_cs, ra0, nm, s_row0, dyn_end, s_scan, &s_flag, bt, s_row);
                slot_prefix();
            }
            float *const u_plain = align16(rows_end());
            const int cap_cells = cells_cap();
            const bool three = 3 * bt.C <= cap_cells && nm <= TPB * (KM / 3);
            // records stay in shared memory (below them the cells) if all fits
            const bool use_rec = rec_smem && three && 3 * bt.C + rec_bytes / 4 <= cap_cells;
            float4 *const ra = use_rec ? s_ra : g_ra;
            uint4 *const rb = use_rec ? s_rb : g_rb;
            const int need = use_rec ? 3 * bt.C + rec_bytes / 4 : (three ? 3 * bt.C : bt.C);
            if (s_flag || bt.C > cap_cells || nm > TPB * KM) {
                // does not fit even one component at a time: hand it to the plain path
                if (tid == 0) {
                    int np_fb = 0;
                    for (int j = 0; j < bt.nb; ++j) np_fb += s_cs[j].np;
                    const int k0 = atomicAdd(prm.cnt + C_NFB, np_fb);
                    atomicAdd(prm.cnt + C_FBMARK, nm);
                    atomicAdd(prm.cnt + C_OVERFLOW, bt.nb);
                    for (int i = 0; i < np; ++i) prm.fb_list[k0 + i] = s_ps[i].gid;
                }
                if (tid < bt.nb) prm.cl_path[prm.order[be.x + tid]] |= IBM_PATH_FALLBACK;
                __syncthreads();
                continue;
            }
            unsigned short *s_inv = reinterpret_cast<unsigned short *>(align16(rows_end()));
            float *const u_inv = align16(s_inv + bt.C);
            const bool use_inv = bt.R < 0xffff && (int)((dyn_end - reinterpret_cast<unsigned char *>(u_inv)) / 4) >= need;
            float *s_u = use_inv ? u_inv : u_plain;
            if (use_inv) {
                for (int i = tid; i < bt.C; i += TPB) s_inv[i] = 0xffffu;
                __syncthreads();
                for (int i = tid; i < bt.R; i += TPB) {
                    unsigned mask = s_row[i].x;
                    int sl = (int)s_row[i].y;
                    while (mask) {
                        mask &= mask - 1u;
                        s_inv[sl++] = (unsigned short)i;
                    }
                }
            } else {
                s_inv = nullptr;
            }
            // base cell -> the nine row slots of the marker's stencil (records move
            // to global memory if the cells need their shared memory)
            for (int m = tid; m < nm; m += TPB) {
                float4 a = ra0[m];
                const unsigned bp = __float_as_uint(a.w);
                if (bp != kNoMarker) {
                    const CS &cs = s_cs[s_ps[s_chunk[m >> 5]].cl];
                    const int b[3] = {(int)(bp & 1023u), (int)((bp >> 10) & 1023u), (int)(bp >> 20)};
                    int sl[9];
                    row_slots(s_row + cs.row0, bt.rix, cs, b, sl);
                    rb[m] = make_uint4((unsigned)sl[0] | ((unsigned)sl[1] << 16), (unsigned)sl[2] | ((unsigned)sl[3] << 16),
                                       (unsigned)sl[4] | ((unsigned)sl[5] << 16), (unsigned)sl[6] | ((unsigned)sl[7] << 16));
                    a.w = __uint_as_float((unsigned)sl[8]);
                }
                ra[m] = a;
            }
            __syncthreads();
            if (tid < bt.nb)
                prm.cl_path[prm.order[be.x + tid]] |= IBM_PATH_SMEM | (use_rec ? 0 : IBM_PATH_GLOBAL_RECORDS) |
                                                      (three ? 0 : IBM_PATH_ONE_COMPONENT) |
                                                      (bt.rix ? IBM_PATH_SPARSE_ROWS : 0);
            if (tid == 0) {
                int touched = 0;
                for (int j = 0; j < bt.nb; ++j) touched += s_cs[j].ncell;
                atomicMax(prm.cnt + C_MAXCELLS, touched);
                atomicAdd(prm.cnt + C_TOUCHED, touched);
                if (!three) atomicAdd(prm.cnt + C_ONECOMP, bt.nb);
            }
            __syncthreads();
            if (use_rec) {
                forcing_rec<TPB, KR, DET, 3>(prm, bt, s_ps, s_cs, s_part, s_chunk, s_row, s_inv, s_u, ra, rb, 0);
            } else if (three) {
                forcing_rec<TPB, KM / 3, DET, 3>(prm, bt, s_ps, s_cs, s_part, s_chunk, s_row, s_inv, s_u, ra, rb, 0);
            } else {
                for (int q = 0; q < 3; ++q) {
                    forcing_rec<TPB, KM, DET, 1>(prm, bt, s_ps, s_cs, s_part, s_chunk, s_row, s_inv, s_u, ra, rb, q);
                    __syncthreads();
                }
            }
            // particle loads: sums of the particle's own chunks in marker order, FP64
            for (int i = tid; i < 6 * np; i += TPB) {
                const int pi = i / 6, q = i - 6 * pi;
                const int ms = s_ps[pi].mstart, nl = s_ps[pi].P.nl;
                double sum = 0.0;
                for (int ch = ms >> 5; ch < (ms + nl + 31) >> 5; ++ch) sum += (double)s_part[ch * 6 + q];
                const int p = s_ps[pi].gid;
                if (q < 3) prm.FD[3 * p + q] = sum;
                else prm.TD[3 * p + q - 3] = sum;
            }
            __syncthreads();
        }
    }
}

int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    return (int)std::max(1ll, std::min(g, 65535ll * 8));
}

// Dynamic shared memory per CTA when minb CTAs share an SM.
static int max_dyn_smem(int minb = 1) {
    int dev = 0, optin = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const int statics = 64 * 4 + 64;   // s_item, s_flag, s_scan, s_total, s_red
    const int per_block = minb <= 1 ? optin : std::min(optin, per_sm / minb - 1024);
    return per_block - statics - 256;
}

}  // namespace

// ================================================================= host side

void cluster_free(ibm_ctx *ctx) {
    ClusterScratch *S = reinterpret_cast<ClusterScratch *>(ctx->cl);
    if (!S) return;
    int *ptrs[] = {S->scene_bin_off, S->scene_nb, S->bin_cnt, S->bin_start, S->bin_cur, S->bin_items,
                   S->parent, S->cand, S->cnt, S->root_flag, S->cid, S->pcl, S->poff, S->cl_np, S->cl_nm,
                   S->cl_first, S->cl_cur, S->cl_box, S->cl_plist, S->cl_bkt, S->bkt_cnt, S->bkt_start,
                   S->order, S->fb_list, S->nm_ord, S->cum, S->cl_scene, S->cl_path, S->big_list,
                   S->big_flag, S->fb_list2, S->big_list16};
    for (int *p : ptrs)
        if (p) cudaFree(p);
    if (S->big_rec) cudaFree(S->big_rec);
    if (S->big_part) cudaFree(S->big_part);
    if (S->big_wl) cudaFree(S->big_wl);
    if (S->big_fork) cudaEventDestroy(S->big_fork);
    if (S->big_join) cudaEventDestroy(S->big_join);
    if (S->big_side) cudaStreamDestroy(S->big_side);
    if (S->batches) cudaFree(S->batches);
    if (S->grec) cudaFree(S->grec);
    if (S->tot) cudaFree(S->tot);
    delete S;
    ctx->cl = nullptr;
}

// Replaces *p by a new device allocation of `bytes` (the old one released
// first, so that a failure leaves *p NULL rather than dangling).
template <typename T>
static cudaError_t dev_realloc(T **p, size_t bytes) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    return ibm_malloc(p, bytes);
}

static ibm_status cluster_alloc(ibm_ctx *ctx) {
    ClusterScratch *S = reinterpret_cast<ClusterScratch *>(ctx->cl);
    const int np = std::max(ctx->n_p, 1);
    const bool realloc_p = !S || S->cap_p < ctx->cap_p;
    if (!S) {
        S = new ClusterScratch();
        ctx->cl = S;
    }
    // bin layout from the largest particle: width >= 2 a_max + 3 sqrt 3 (+1)
    const double q_max = std::sqrt((ctx->max_nl + 0.5) / M_PI) + 1e-9;
    const double bw = q_max + 3.0 * std::sqrt(3.0) + 1.0;
    if (realloc_p || S->max_nl != ctx->max_nl || S->n_scenes != ctx->cfg.n_scenes) {
        std::vector<int> off(ctx->cfg.n_scenes + 1), nb(3 * ctx->cfg.n_scenes);
        long long total = 0;
        for (int s = 0; s < ctx->cfg.n_scenes; ++s) {
            off[s] = (int)total;
            long long cells = 1;
            for (int c = 0; c < 3; ++c) {
                nb[3 * s + c] = std::max(1, (int)std::floor(ctx->dims_h[3 * s + c] / bw));
                cells *= nb[3 * s + c];
            }
            total += cells;
        }
        off[ctx->cfg.n_scenes] = (int)total;
        if (total > (1 << 28)) return ibm_fail(ctx, IBM_ERR_CAPACITY, "too many particle bins");
        CK(dev_realloc(&S->scene_bin_off, off.size() * sizeof(int)), "alloc bins");
        CK(dev_realloc(&S->scene_nb, nb.size() * sizeof(int)), "alloc bins");
        CK(cudaMemcpy(S->scene_bin_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice), "copy");
        CK(cudaMemcpy(S->scene_nb, nb.data(), nb.size() * sizeof(int), cudaMemcpyHostToDevice), "copy");
        if ((int)total > S->cap_bins) {
            CK(dev_realloc(&S->bin_cnt, (total + 1) * sizeof(int)), "alloc bins");
            CK(dev_realloc(&S->bin_start, (total + 1) * sizeof(int)), "alloc bins");
            CK(dev_realloc(&S->bin_cur, (total + 1) * sizeof(int)), "alloc bins");
            S->cap_bins = (int)total;
        }
        S->nbins = (int)total;
        S->max_nl = ctx->max_nl;
        S->n_scenes = ctx->cfg.n_scenes;
        S->bin_w = bw;
    }
    if (realloc_p) {
        const int cp = std::max(ctx->cap_p, np);
        int **arrs[] = {&S->bin_items, &S->parent, &S->root_flag, &S->cid, &S->pcl, &S->cl_np, &S->cl_nm,
                        &S->cl_first, &S->cl_cur, &S->cl_plist, &S->cl_bkt, &S->order, &S->fb_list,
                        &S->nm_ord, &S->cum, &S->cl_scene, &S->cl_path, &S->big_list, &S->big_flag,
                        &S->fb_list2, &S->big_list16};
        for (int **p : arrs) CK(dev_realloc(p, (size_t)(cp + 1) * sizeof(int)), "alloc cluster scratch");
        CK(dev_realloc(&S->batches, (size_t)(cp + 1) * sizeof(int2)), "alloc batch list");
        CK(dev_realloc(&S->poff, 3 * (size_t)cp * sizeof(int)), "alloc cluster scratch");
        CK(dev_realloc(&S->cl_box, 12 * (size_t)cp * sizeof(int)), "alloc cluster scratch");
        S->cap_cand = std::max(1 << 16, 16 * cp);
        CK(dev_realloc(&S->cand, 2 * (size_t)S->cap_cand * sizeof(int)), "alloc candidates");
        if (!S->cnt) CK(ibm_malloc(&S->cnt, C_COUNT * sizeof(int)), "alloc counters");
        if (!S->tot) CK(ibm_malloc(&S->tot, 4 * sizeof(long long)), "alloc totals");
        if (!S->bkt_cnt) CK(ibm_malloc(&S->bkt_cnt, (kBuckets + 1) * sizeof(int)), "alloc buckets");
        if (!S->bkt_start) CK(ibm_malloc(&S->bkt_start, (kBuckets + 1) * sizeof(int) * 2), "alloc buckets");
        S->cap_p = cp;
    }
    return IBM_OK;
}

template <int TPB, int KM, int KR, bool DET, int MINB>
static ibm_status launch_cluster_kernel(ibm_ctx *ctx, ClusterScratch *S, KParams &prm) {
    auto kern = k_cluster_forcing<TPB, KM, KR, DET, MINB>;
    if (S->smem_bytes == 0 || S->tpb != TPB || S->det != (int)DET) {
        S->smem_bytes = max_dyn_smem(MINB) & ~15;
        S->cap_c = (S->smem_bytes - fixed_smem_bytes<TPB, KM>()) / 4;   // FP32 cell slots (all components)
        S->tpb = TPB;
        S->kmax = KM;
        S->det = (int)DET;
        CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S->smem_bytes),
           "set shared memory size");
    }
    prm.smem_bytes = S->smem_bytes;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TPB, S->smem_bytes), "occupancy");
    const int grid = std::max(1, nsm * std::max(per_sm, 1));
    const size_t grec = (size_t)grid * 2 * TPB * KM * sizeof(float4);
    if (S->grec_bytes < grec) {
        if (S->grec) cudaFree(S->grec);
        S->grec = nullptr;
        S->grec_bytes = 0;
        CK(ibm_malloc(&S->grec, grec), "alloc marker records");
        S->grec_bytes = grec;
    }
    prm.grec = S->grec;
    kern<<<grid, TPB, S->smem_bytes, ctx->stream>>>(prm);
    return ibm_cuda_check(ctx, cudaGetLastError(), "cluster kernel");
}

// marker slots per thread of the cluster kernel's recomputing path, and
// ------------------------------------------ clusters held in distributed shared memory
// A cluster whose touched cells exceed one SM's shared memory (the dense
// boxes of small periodic scenes, long chains) would otherwise run the plain
// path with global atomics.  When its stencil box fits the shared memory of a
// thread-block cluster of kBigK CTAs (one per SM), it runs here instead: the
// box is cut into z slabs, one per CTA, held densely (3 FP32 components per
// cell plus a touched-cell bit), and every CTA reaches the other slabs through
// distributed shared memory.  Per forcing iteration: interpolation of the
// CTA's share of the markers (loads from any slab), the cluster-wide fixed-
// point scale (deterministic mode: the same maxima as the plain fallback),
// the CTA's own cells converted, spreading by shared-memory atomics into any
// slab, cells converted back, with cluster barriers between the phases.  HBM
// sees each touched cell once per step, as on the one-SM path.  The work list
// is taken persistently, one cluster at a time per thread-block cluster.
// threads per CTA; marker capacity per CTA of a thread-block cluster, in units of its threads; particles
constexpr int kBigT = 1024, kBigKR = 4, kBigMaxP = 512;

struct BigParams {
    const PInfo *P;
    const float *t32;
    const double *t64;
    const int32_t *dims;
    float *const *uf;
    float *const *ff;
    int *cnt, *err;
    const int *big_list, *cl_np, *cl_first, *cl_plist, *cl_box, *cl_scene;
    int c_n, c_work;     // indices in cnt of the list's length and of its work counter
    const unsigned *dis;
    double *FD, *TD;
    uint4 *rec;          // marker records, two per marker, K * kBigT * kBigKR markers per thread-block cluster
    float *part;         // per marker: e and its load terms summed over the iterations (9 floats)
    int *wlist;          // per thread-block cluster: its markers grouped by owning CTA
    int n_forcing, cap_cells;
    float finv;
};

struct BigHdr {
    int c, np, nm, wrap;
    int lo[3], B[3], n[3];       // the box, per axis of the grid
    int perm[3], Bp[3], wp;      // local axis j is grid axis perm[j]; local axis 2 (the longest) is cut into slabs
    int slab, z0, z1, ncell;     // this CTA's slab [z0, z1) along local axis 2 and its cells
    int scene;
};

// The slab axis of a box: its longest axis (z on ties), so that the slabs are thin.
__device__ __forceinline__ int big_slab_axis(const long long B[3]) {
    int a = 2;
    if (B[0] > B[a]) a = 0;
    if (B[1] > B[a]) a = 1;
    return a;
}

__device__ __forceinline__ int big_mod(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// Box-relative cell of stencil start s (per axis) plus d, modulo the period
// along the wrapped axes (their box is the whole period).
__device__ __forceinline__ int big_ax(int s, int d, int B, bool wrapped) {
    int v = s + d;
    if (wrapped && v >= B) v -= B;
    return v;
}

template <int K, bool DET>
__global__ void __launch_bounds__(kBigT, 1) k_big_cluster(BigParams bp) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char big_dyn[];
    __shared__ BigHdr H;
    __shared__ int s_item;
    __shared__ int s_pid[kBigMaxP];
    __shared__ int s_pref[kBigMaxP + 1];
    __shared__ unsigned s_max[2][3];        // rank 0's copy: the cluster's maxima of an iteration (two buffers)
    __shared__ float s_red[3][kBigT / 32];
    __shared__ int s_own, s_cur;            // markers this CTA owns (their stencil's middle plane is in its slab)
    __shared__ int s_off[K + 1];            // offsets of every CTA's markers in the work list
    __shared__ int s_scan[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int rank = (int)cl.block_rank();
    const int slot = blockIdx.x / K;
    const int cap = bp.cap_cells;
    const int mcap = K * kBigT * kBigKR;
    float *cells = reinterpret_cast<float *>(big_dyn);
    unsigned *tb = reinterpret_cast<unsigned *>(big_dyn + 3ull * cap * sizeof(float));
    uint4 *rec = bp.rec + (size_t)slot * mcap * 2;     // two records per marker of the item
    float *eb = bp.part + (size_t)slot * mcap * 9;     // per marker: e (3) and the load terms summed over iterations (6)
    int *wl = bp.wlist + (size_t)slot * mcap;          // work list: markers grouped by owning CTA
    for (;;) {
        if (rank == 0 && tid == 0) s_item = atomicAdd(bp.cnt + bp.c_work, 1);
        cl.sync();
        const int item = *cl.map_shared_rank(&s_item, 0);
        cl.sync();   // rank 0's s_item stays valid until every CTA has read it
        if (item >= bp.cnt[bp.c_n]) break;
        // ---- header: box (whole period along wrapped axes), particles sorted by index, marker prefix
        if (tid == 0) {
            const int c = bp.big_list[item];
            H.c = c;
            H.np = bp.cl_np[c];
            H.scene = bp.cl_scene[c] & 0x0fffffff;
            H.wrap = (bp.cl_scene[c] >> 28) & 7;
            for (int k = 0; k < 3; ++k) {
                H.n[k] = bp.dims[3 * H.scene + k];
                const bool w = (H.wrap >> k) & 1;
                H.lo[k] = w ? 0 : bp.cl_box[12 * c + k];
                H.B[k] = w ? H.n[k] : bp.cl_box[12 * c + 3 + k] - bp.cl_box[12 * c + k] + 1;
            }
            const long long Bl[3] = {H.B[0], H.B[1], H.B[2]};
            const int a = big_slab_axis(Bl);
            H.perm[2] = a;
            H.perm[0] = a == 0 ? 1 : 0;
            H.perm[1] = a == 2 ? 1 : 2;
            H.wp = 0;
            for (int j = 0; j < 3; ++j) {
                H.Bp[j] = H.B[H.perm[j]];
                H.wp |= ((H.wrap >> H.perm[j]) & 1) << j;
            }
            H.slab = (H.Bp[2] + K - 1) / K;
            H.z0 = min(H.Bp[2], rank * H.slab);
            H.z1 = min(H.Bp[2], H.z0 + H.slab);
            H.ncell = (H.z1 - H.z0) * H.Bp[1] * H.Bp[0];
            s_own = 0;
            s_cur = 0;
        }
        __syncthreads();
        const int np = H.np;
        for (int i = tid; i < np; i += kBigT) s_pid[i] = bp.cl_plist[bp.cl_first[H.c] + i];
        __syncthreads();
        int my_pid = 0, my_pos = 0;
        if (tid < np) {
            my_pid = s_pid[tid];
            for (int j = 0; j < np; ++j) my_pos += s_pid[j] < my_pid;
        }
        __syncthreads();
        if (tid < np) s_pid[my_pos] = my_pid;
        __syncthreads();
        {
            // first flat marker of each particle (padded to 32-marker chunks): block scan
            const int pad = tid < np ? (bp.P[s_pid[tid]].nl + 31) & ~31 : 0;
            int total;
            const int pre = block_excl_scan<kBigT>(pad, s_scan, &total);
            if (tid < np) s_pref[tid] = pre;
            if (tid == 0) s_pref[np] = total;
        }
        if (rank == 0 && tid < 6) s_max[tid / 3][tid % 3] = 0u;
        for (int w = tid; w < (H.ncell + 31) / 32; w += kBigT) tb[w] = 0u;
        __syncthreads();
        const int nm = s_pref[np];
        const int per = (((nm >> 5) + K - 1) / K) << 5;          // flat markers set up by each CTA
        const int m0 = min(nm, rank * per), m1 = min(nm, m0 + per);
        const int B0 = H.Bp[0], B1 = H.Bp[1], B2 = H.Bp[2], slab = H.slab;
        const bool wx = H.wp & 1, wy = (H.wp >> 1) & 1, wz = (H.wp >> 2) & 1;
        // grid cell of local cell (x, y, z) of the box
        auto grid_cell = [&](int x, int y, int z) {
            int o[3];
            o[H.perm[0]] = x;
            o[H.perm[1]] = y;
            o[H.perm[2]] = z;
            return ((long long)big_mod(H.lo[2] + o[2], H.n[2]) * H.n[1] + big_mod(H.lo[1] + o[1], H.n[1])) * H.n[0] +
                   big_mod(H.lo[0] + o[0], H.n[0]);
        };
        cl.sync();   // bitmasks clear and counters zero everywhere
        // ---- records of this CTA's flat markers (box-relative stencil start, fractions), touched bits,
        // and the count of each owning CTA
        for (int m = m0 + tid; m < m1; m += kBigT) {
            int lo = 0, hi = np;   // particle of flat marker m
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_pref[mid] <= m) lo = mid;
                else hi = mid;
            }
            const int p = s_pid[lo];
            const int l = m - s_pref[lo];
            const PInfo &Pp = bp.P[p];
            bool live = l < Pp.nl;
            if (live && bp.dis) {
                const long long mk = (long long)Pp.moff + l;
                live = !((bp.dis[mk >> 5] >> (mk & 31)) & 1u);
            }
            uint4 r0 = make_uint4(0u, 0u, 0u, 0u), r1 = make_uint4(0u, 0u, 0u, 0u);
            if (live) {
                int sg[3], st[3];
                float fg[3], fr[3];
                for (int c = 0; c < 3; ++c) {
                    const int b = marker_split32(Pp, bp.t32 + 3ll * (Pp.toff + l), bp.t64 + 3ll * (Pp.toff + l), c, &fg[c]);
                    sg[c] = big_mod(b - 1 - H.lo[c], H.n[c]);
                }
                for (int j = 0; j < 3; ++j) {   // in the box's local axes
                    st[j] = sg[H.perm[j]];
                    fr[j] = fg[H.perm[j]];
                }
                r0 = make_uint4((unsigned)st[0] | ((unsigned)st[1] << 10) | ((unsigned)st[2] << 20) | (1u << 31),
                                __float_as_uint(fr[0]), __float_as_uint(fr[1]), __float_as_uint(fr[2]));
                r1 = make_uint4((unsigned)lo, (unsigned)l, (unsigned)p, 0u);
                atomicAdd(cl.map_shared_rank(&s_own, big_ax(st[2], 1, B2, wz) / slab), 1);
            }
            rec[2 * m] = r0;
            rec[2 * m + 1] = r1;
#pragma unroll
            for (int q = 3; q < 9; ++q) eb[9 * m + q] = 0.f;
        }
        cl.sync();   // records and owner counts complete
        if (tid == 0) {
            int a = 0;
            for (int r = 0; r < K; ++r) {
                s_off[r] = a;
                a += *cl.map_shared_rank(&s_own, r);
            }
            s_off[K] = a;
        }
        __syncthreads();
        // work list: each marker into its owner's range (order within a range is free: the loads are
        // summed per marker index afterwards)
        for (int m = m0 + tid; m < m1; m += kBigT) {
            const uint4 r0 = rec[2 * m];
            if (!(r0.x >> 31)) continue;
            const int owner = big_ax((int)((r0.x >> 20) & 1023u), 1, B2, wz) / slab;
            wl[s_off[owner] + atomicAdd(cl.map_shared_rank(&s_cur, owner), 1)] = m;
        }
        __threadfence();
        cl.sync();   // work lists complete
        const int w0 = s_off[rank], w1 = s_off[rank + 1];
        // touched bits, set by the owner of each marker (its own slab for the middle plane)
        for (int i = w0 + tid; i < w1; i += kBigT) {
            const uint4 r0 = rec[2 * wl[i]];
            const int st[3] = {(int)(r0.x & 1023u), (int)((r0.x >> 10) & 1023u), (int)((r0.x >> 20) & 1023u)};
            for (int cz = 0; cz < 3; ++cz) {
                const int z = big_ax(st[2], cz, B2, wz);
                const int rk = z / slab;
                unsigned *rtb = rk == rank ? tb : cl.map_shared_rank(tb, rk);
                for (int cy = 0; cy < 3; ++cy) {
                    const int y = big_ax(st[1], cy, B1, wy);
                    for (int cx = 0; cx < 3; ++cx) {
                        const int x = big_ax(st[0], cx, B0, wx);
                        const int idx = ((z - rk * slab) * B1 + y) * B0 + x;
                        atomicOr(rtb + (idx >> 5), 1u << (idx & 31));
                    }
                }
            }
        }
        cl.sync();   // touched bits complete
        // ---- gather the touched cells of this CTA's slab
        const float *const u0 = bp.uf[H.scene];
        const long long ncs = (long long)H.n[0] * H.n[1] * H.n[2];
        float ucarry = 0.f;   // max |u| over this thread's cells (deterministic mode's range)
        for (int i = tid; i < H.ncell; i += kBigT) {
            if (!((tb[i >> 5] >> (i & 31)) & 1u)) continue;
            const int x = i % B0, t = i / B0, y = t % B1, z = H.z0 + t / B1;
            const long long g = grid_cell(x, y, z);
            for (int q = 0; q < 3; ++q) {
                const float v = u0[q * ncs + g];
                cells[q * cap + i] = v;
                if (DET) ucarry = fmaxf(ucarry, fabsf(v));
            }
        }
        cl.sync();   // cells complete
        // ---- the n_F iterations; a CTA works on the markers whose stencil's middle plane it holds, so
        // most of their cells are its own (plain shared-memory accesses), the rest in the neighbour slabs
        for (int it = 0; it < bp.n_forcing; ++it) {
            float emax = 0.f, dmax = 0.f;
            for (int i = w0 + tid; i < w1; i += kBigT) {
                const int m = wl[i];
                const uint4 r0 = rec[2 * m];
                const uint4 r1 = rec[2 * m + 1];
                const PInfo &Pp = bp.P[r1.z];
                const int st[3] = {(int)(r0.x & 1023u), (int)((r0.x >> 10) & 1023u), (int)((r0.x >> 20) & 1023u)};
                float w[3][3];
                phi3_weights(__uint_as_float(r0.y), w[0]);
                phi3_weights(__uint_as_float(r0.z), w[1]);
                phi3_weights(__uint_as_float(r0.w), w[2]);
                int xs[3];
#pragma unroll
                for (int cx = 0; cx < 3; ++cx) xs[cx] = big_ax(st[0], cx, B0, wx);
                float U[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int cz = 0; cz < 3; ++cz) {
                    const int z = big_ax(st[2], cz, B2, wz);
                    const int rk = z / slab;
                    const int zb = (z - rk * slab) * B1;
                    auto row = [&](const float *rc) {
#pragma unroll
                        for (int cy = 0; cy < 3; ++cy) {
                            const float *rw = rc + (zb + big_ax(st[1], cy, B1, wy)) * B0;
                            const float wyz = w[2][cz] * w[1][cy];
#pragma unroll
                            for (int cx = 0; cx < 3; ++cx) {
                                const float ww = wyz * w[0][cx];
#pragma unroll
                                for (int q = 0; q < 3; ++q) U[q] += ww * rw[q * cap + xs[cx]];
                            }
                        }
                    };
                    if (rk == rank) row(cells);
                    else row(cl.map_shared_rank(cells, rk));
                }
                const float *t = bp.t32 + 3ll * (Pp.toff + r1.y);
                const float r[3] = {Pp.rphys * t[0], Pp.rphys * t[1], Pp.rphys * t[2]};
                const float ud[3] = {Pp.ud[0] + (Pp.om[1] * r[2] - Pp.om[2] * r[1]),
                                     Pp.ud[1] + (Pp.om[2] * r[0] - Pp.om[0] * r[2]),
                                     Pp.ud[2] + (Pp.om[0] * r[1] - Pp.om[1] * r[0])};
                const float D = Pp.D;
                float e[3];
                for (int q = 0; q < 3; ++q) {
                    e[q] = ud[q] - U[q];
                    emax = fmaxf(emax, fabsf(e[q]));
                    eb[9 * m + q] = e[q];
                }
                dmax = fmaxf(dmax, D);
                const float ed[3] = {e[0] * D, e[1] * D, e[2] * D};
                eb[9 * m + 3] += ed[0];
                eb[9 * m + 4] += ed[1];
                eb[9 * m + 5] += ed[2];
                eb[9 * m + 6] += r[1] * ed[2] - r[2] * ed[1];
                eb[9 * m + 7] += r[2] * ed[0] - r[0] * ed[2];
                eb[9 * m + 8] += r[0] * ed[1] - r[1] * ed[0];
            }
            if (DET) {
                const float umax = warp_max(ucarry);
                emax = warp_max(emax);
                dmax = warp_max(dmax);
                if (lane == 0) {
                    s_red[0][wid] = umax;
                    s_red[1][wid] = emax;
                    s_red[2][wid] = dmax;
                }
                __syncthreads();
                if (tid < 3) {
                    float mx = 0.f;
                    for (int i = 0; i < kBigT / 32; ++i) mx = fmaxf(mx, s_red[tid][i]);
                    atomicMax(cl.map_shared_rank(&s_max[it & 1][tid], 0), __float_as_uint(mx));
                }
            }
            cl.sync();   // interpolation done everywhere (and the maxima complete)
            float S = 1.f, inv = 1.f;
            if (DET) {
                const unsigned *mx = cl.map_shared_rank(&s_max[it & 1][0], 0);
                const float range = __uint_as_float(mx[0]) + 64.f * __uint_as_float(mx[2]) * __uint_as_float(mx[1]);
                int ex = 100;
                if (range > 0.f) ex = min(100, max(-100, 27 - (int)ceilf(log2f(range))));
                S = ldexpf(1.f, ex);
                inv = ldexpf(1.f, -ex);
                for (int i = tid; i < H.ncell; i += kBigT) {
                    if (!((tb[i >> 5] >> (i & 31)) & 1u)) continue;
                    for (int q = 0; q < 3; ++q) {
                        float *c = cells + q * cap + i;
                        *reinterpret_cast<int *>(c) = __float2int_rn(*c * S);
                    }
                }
                if (rank == 0 && tid < 3) s_max[(it + 1) & 1][tid] = 0u;   // the next iteration's buffer
                cl.sync();   // every slab in fixed point
            }
            // spreading: u += w D e
            for (int i = w0 + tid; i < w1; i += kBigT) {
                const int m = wl[i];
                const uint4 r0 = rec[2 * m];
                const float D = bp.P[rec[2 * m + 1].z].D;
                const int st[3] = {(int)(r0.x & 1023u), (int)((r0.x >> 10) & 1023u), (int)((r0.x >> 20) & 1023u)};
                float w[3][3];
                phi3_weights(__uint_as_float(r0.y), w[0]);
                phi3_weights(__uint_as_float(r0.z), w[1]);
                phi3_weights(__uint_as_float(r0.w), w[2]);
                const float gv[3] = {D * eb[9 * m], D * eb[9 * m + 1], D * eb[9 * m + 2]};
                int xs[3];
#pragma unroll
                for (int cx = 0; cx < 3; ++cx) xs[cx] = big_ax(st[0], cx, B0, wx);
#pragma unroll
                for (int cz = 0; cz < 3; ++cz) {
                    const int z = big_ax(st[2], cz, B2, wz);
                    const int rk = z / slab;
                    const int zb = (z - rk * slab) * B1;
                    auto row = [&](float *rc) {
#pragma unroll
                        for (int cy = 0; cy < 3; ++cy) {
                            float *rw = rc + (zb + big_ax(st[1], cy, B1, wy)) * B0;
                            const float wyz = w[2][cz] * w[1][cy];
#pragma unroll
                            for (int cx = 0; cx < 3; ++cx) {
                                const float ww = wyz * w[0][cx];
#pragma unroll
                                for (int q = 0; q < 3; ++q) {
                                    float *c = rw + q * cap + xs[cx];
                                    if (DET) atomicAdd(reinterpret_cast<int *>(c), __float2int_rn((ww * gv[q]) * S));
                                    else atomicAdd(c, ww * gv[q]);
                                }
                            }
                        }
                    };
                    if (rk == rank) row(cells);
                    else row(cl.map_shared_rank(cells, rk));
                }
            }
            cl.sync();   // spreading done everywhere
            if (DET) {
                ucarry = 0.f;
                for (int i = tid; i < H.ncell; i += kBigT) {
                    if (!((tb[i >> 5] >> (i & 31)) & 1u)) continue;
                    for (int q = 0; q < 3; ++q) {
                        float *c = cells + q * cap + i;
                        const int v = *reinterpret_cast<const int *>(c);
                        if (abs(v) > (1 << 28)) set_err(bp.err, IBM_EBIT_FIXEDPOINT);
                        const float f = (float)v * inv;
                        *c = f;
                        ucarry = fmaxf(ucarry, fabsf(f));
                    }
                }
                cl.sync();   // back in FP32 before the next interpolation
            }
        }
        // ---- write back this slab's touched cells (and f = (u^{n_F} - u^0) / tau)
        float *const uw = bp.uf[H.scene];
        float *const fw = bp.ff ? bp.ff[H.scene] : nullptr;
        for (int i = tid; i < H.ncell; i += kBigT) {
            if (!((tb[i >> 5] >> (i & 31)) & 1u)) continue;
            const int x = i % B0, t = i / B0, y = t % B1, z = H.z0 + t / B1;
            const long long g = grid_cell(x, y, z);
            for (int q = 0; q < 3; ++q) {
                const float v = cells[q * cap + i];
                if (fw) fw[q * ncs + g] = (v - uw[q * ncs + g]) * bp.finv;
                uw[q * ncs + g] = v;
            }
        }
        // ---- loads: one warp of the thread-block cluster per (particle, component): each 32-marker
        // chunk summed in FP32 by the warp, the chunks added in marker order in FP64
        __threadfence();
        cl.sync();
        for (int j = rank * (kBigT / 32) + wid; j < np * 6; j += K * (kBigT / 32)) {
            const int i = j / 6, q = j - 6 * (j / 6);
            double sum = 0.0;
            for (int c0 = s_pref[i]; c0 < s_pref[i + 1]; c0 += 32) sum += (double)warp_sum(eb[9 * (c0 + lane) + 3 + q]);
            if (lane == 0) {
                const int p = s_pid[i];
                if (q < 3) bp.FD[3 * p + q] += sum;
                else bp.TD[3 * p + q - 3] += sum;
            }
        }
        cl.sync();   // nothing of this cluster is read any more: the next one may start
    }
}

// Which fallback clusters fit a thread-block cluster (dense slabs of at most cap
// cells, at most kBigMaxP particles and K (kBigT kBigKR - 32) markers): each goes
// to the smaller size that fits and can run (8 or 16 CTAs), with a flag per
// cluster and its path bits.
__global__ void k_big_select(const long long *n_clust_d, const int32_t *dims, const int *cl_np, const int *cl_nm,
                             const int *cl_box, const int *cl_scene, int *cl_path, int use8, int use16, int cap,
                             int *list8, int *list16, int *big_flag, int *cnt) {
    const int n = (int)*n_clust_d;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        big_flag[c] = 0;
        if (!(cl_path[c] & IBM_PATH_FALLBACK)) continue;
        const int s = cl_scene[c] & 0x0fffffff, wrap = (cl_scene[c] >> 28) & 7;
        long long B[3];
        bool ok = cl_np[c] <= kBigMaxP;
        for (int k = 0; k < 3; ++k) {
            const int nk = dims[3 * s + k];
            B[k] = ((wrap >> k) & 1) ? nk : cl_box[12 * c + 3 + k] - cl_box[12 * c + k] + 1;
            ok = ok && B[k] <= nk && B[k] <= 1023;
        }
        if (!ok) continue;
        const int a = big_slab_axis(B);
        auto fits = [&](int K) {
            return cl_nm[c] <= K * (kBigT * kBigKR - 32) && (B[a] + K - 1) / K * (B[0] * B[1] * B[2] / B[a]) <= cap;
        };
        int K = 0;
        if (use8 && fits(8)) K = 8;
        else if (use16 && fits(16)) K = 16;
        if (!K) continue;
        big_flag[c] = 1;
        if (K == 8) list8[atomicAdd(cnt + C_NBIG8, 1)] = c;
        else list16[atomicAdd(cnt + C_NBIG16, 1)] = c;
        atomicAdd(cnt + C_NBIG, 1);
        atomicAdd(cnt + C_BIGMARK, cl_nm[c]);
        cl_path[c] = (cl_path[c] & ~IBM_PATH_FALLBACK) | IBM_PATH_DSMEM;
    }
}

// The plain fallback keeps the particles of the clusters that did not move to
// the thread-block-cluster path.
__global__ void k_fb_compact(const int *fb_list, const int *pcl, const int *big_flag, int *fb_list2, int *cnt) {
    const int n = cnt[C_NFB];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p = fb_list[i];
        if (!big_flag[pcl[p]]) fb_list2[atomicAdd(cnt + C_NFB2, 1)] = p;
    }
}

// Cluster size of the distributed-shared-memory path on this device (16 if a
// 16-CTA cluster of kBigT threads with the full shared memory can run, else 8,
// else 0 = path off), the dynamic shared memory and the number of clusters
// that run at once.
template <int K, bool DET>
static bool big_config(int *smem_out, int *grid) {
    auto kern = k_big_cluster<K, DET>;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int smem = (optin - (int)fa.sharedSizeBytes - 256) & ~15;
    *smem_out = smem;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (K > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(K);
    cfg.blockDim = dim3(kBigT);
    cfg.dynamicSmemBytes = (size_t)smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = K;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    *grid = n;
    return n > 0;
}

template <int K, bool DET>
static ibm_status big_launch_t(ibm_ctx *ctx, ClusterScratch *S, BigParams bp, int grid, const int *list, int c_n,
                               int c_work, cudaStream_t stream) {
    bp.big_list = list;
    bp.c_n = c_n;
    bp.c_work = c_work;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(K * grid);
    cfg.blockDim = dim3(kBigT);
    cfg.dynamicSmemBytes = (size_t)S->big_smem;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = K;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return ibm_cuda_check(ctx, cudaLaunchKernelEx(&cfg, k_big_cluster<K, DET>, bp), "thread-block-cluster kernel");
}

// Move the fallback clusters that fit a thread-block cluster to the
// distributed-shared-memory kernel; *fb_list / *fb_cnt then name what is left
// for the plain path.
static ibm_status big_clusters(ibm_ctx *ctx, ClusterScratch *S, float finv, bool with_f, bool det,
                               const int **fb_list, const int **fb_cnt) {
    *fb_list = S->fb_list;
    *fb_cnt = S->cnt + C_NFB;
    cudaStream_t sm = ctx->stream;
    if (S->big_k < 0 || S->big_det != (int)det) {
        // once per context: which thread-block-cluster sizes this device runs with the full shared memory
        int g8 = 0, g16 = 0, smem8 = 0, smem16 = 0;
        if (!(det ? big_config<8, true>(&smem8, &g8) : big_config<8, false>(&smem8, &g8))) g8 = 0;
        if (!(det ? big_config<16, true>(&smem16, &g16) : big_config<16, false>(&smem16, &g16))) g16 = 0;
        S->big_grid8 = g8;
        S->big_grid16 = g16;
        S->big_k = (g8 || g16) ? 1 : 0;
        S->big_det = (int)det;
        S->big_smem = std::min(g8 ? smem8 : INT_MAX, g16 ? smem16 : INT_MAX);
        // dense cells: 12 B and one bit each
        S->big_cells = S->big_k ? (int)(((long long)S->big_smem * 8 / 97) & ~31ll) : 0;
        if (S->big_k) {
            if (g8) CK(cudaFuncSetAttribute(det ? (const void *)k_big_cluster<8, true> : (const void *)k_big_cluster<8, false>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, S->big_smem), "shared memory");
            if (g16) CK(cudaFuncSetAttribute(det ? (const void *)k_big_cluster<16, true> : (const void *)k_big_cluster<16, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, S->big_smem), "shared memory");
        }
    }
    if (S->big_k == 0) return IBM_OK;
    const bool both = S->big_grid8 > 0 && S->big_grid16 > 0;
    if (both) {
        // each made once; one that failed before is tried again on the next step
        if (!S->big_side) {
            cudaStream_t st = nullptr;
            CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "side stream");
            S->big_side = st;
        }
        for (cudaEvent_t *ev : {&S->big_fork, &S->big_join})
            if (!*ev) {
                cudaEvent_t e = nullptr;
                CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "fork/join event");
                *ev = e;
            }
    }
    // scratch per slot: K * kBigT * kBigKR markers; the 8-CTA slots first, then the 16-CTA ones
    // (the two launches run at the same time)
    const size_t mk8 = (size_t)S->big_grid8 * 8 * kBigT * kBigKR;
    const size_t mk = mk8 + (size_t)S->big_grid16 * 16 * kBigT * kBigKR;
    const size_t rec = mk * 2 * sizeof(uint4);
    const size_t part = mk * 9 * sizeof(float);
    const size_t wl = mk * sizeof(int);
    if (S->big_rec_bytes < rec) {
        S->big_rec_bytes = 0;
        CK(dev_realloc(&S->big_rec, rec), "alloc cluster records");
        S->big_rec_bytes = rec;
    }
    if (S->big_part_bytes < part) {
        S->big_part_bytes = 0;
        CK(dev_realloc(&S->big_part, part), "alloc cluster marker sums");
        S->big_part_bytes = part;
    }
    if (S->big_wl_bytes < wl) {
        S->big_wl_bytes = 0;
        CK(dev_realloc(&S->big_wl, wl), "alloc cluster work lists");
        S->big_wl_bytes = wl;
    }
    const int n = std::max(ctx->n_p, 1);
    k_big_select<<<grid_for(n, 256), 256, 0, sm>>>(S->tot + 1, ctx->dims_d, S->cl_np, S->cl_nm, S->cl_box,
                                                   S->cl_scene, S->cl_path, S->big_grid8 > 0, S->big_grid16 > 0,
                                                   S->big_cells, S->big_list, S->big_list16, S->big_flag, S->cnt);
    k_fb_compact<<<grid_for(n, 256), 256, 0, sm>>>(S->fb_list, S->pcl, S->big_flag, S->fb_list2, S->cnt);
    BigParams bp;
    bp.P = ctx->pinfo;
    bp.t32 = ctx->tmpl32;
    bp.t64 = ctx->tmpl64;
    bp.dims = ctx->dims_d;
    bp.uf = reinterpret_cast<float *const *>(ctx->uptr_d);
    bp.ff = with_f ? reinterpret_cast<float *const *>(ctx->fptr_d) : nullptr;
    bp.cnt = S->cnt;
    bp.err = ctx->err_d;
    bp.cl_np = S->cl_np;
    bp.cl_first = S->cl_first;
    bp.cl_plist = S->cl_plist;
    bp.cl_box = S->cl_box;
    bp.cl_scene = S->cl_scene;
    bp.dis = contact_bits(ctx);
    bp.FD = ctx->FD;
    bp.TD = ctx->TD;
    bp.rec = S->big_rec;
    bp.part = S->big_part;
    bp.wlist = S->big_wl;
    bp.n_forcing = ctx->cfg.n_forcing;
    bp.cap_cells = S->big_cells;
    bp.finv = finv;
    ibm_status st = IBM_OK;
    if (S->big_grid16) {
        // the larger clusters first (they need 16 free SMs of one GPC), on the side stream when both run
        BigParams b16 = bp;
        b16.rec = S->big_rec + 2 * mk8;
        b16.part = S->big_part + 9 * mk8;
        b16.wlist = S->big_wl + mk8;
        cudaStream_t s16 = sm;
        if (both) {
            CK(cudaEventRecord(S->big_fork, sm), "fork");
            CK(cudaStreamWaitEvent(S->big_side, S->big_fork, 0), "fork wait");
            s16 = S->big_side;
        }
        st = det ? big_launch_t<16, true>(ctx, S, b16, S->big_grid16, S->big_list16, C_NBIG16, C_WORK16, s16)
                 : big_launch_t<16, false>(ctx, S, b16, S->big_grid16, S->big_list16, C_NBIG16, C_WORK16, s16);
    }
    if (st == IBM_OK && S->big_grid8)
        st = det ? big_launch_t<8, true>(ctx, S, bp, S->big_grid8, S->big_list, C_NBIG8, C_WORK8, sm)
                 : big_launch_t<8, false>(ctx, S, bp, S->big_grid8, S->big_list, C_NBIG8, C_WORK8, sm);
    if (both) {
        // join even after a failed launch, so that a stream capture stays well formed
        const cudaError_t e1 = cudaEventRecord(S->big_join, S->big_side);
        const cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(sm, S->big_join, 0) : e1;
        if (st == IBM_OK && e2 != cudaSuccess) st = ibm_cuda_check(ctx, e2, "join");
    }
    if (st != IBM_OK) return st;
    ctx->launches += 2 + (S->big_grid8 > 0) + (S->big_grid16 > 0);
    *fb_list = S->fb_list2;
    *fb_cnt = S->cnt + C_NFB2;
    return IBM_OK;
}

// markers per thread of its record path, for a block size
static int markers_per_thread(int) { return 12; }
static int records_per_thread(int) { return 2; }
static int ctas_per_sm(int tpb) { return tpb == 512 ? 2 : 1; }
static constexpr int kTuneSteps = 4;

ibm_status cluster_forcing_step(ibm_ctx *ctx, void *const *u_ptrs, double tau, void *const *f_out) {
    ibm_status st = ensure_field_ptrs(ctx, u_ptrs, f_out);
    if (st != IBM_OK) return st;
    if (ctx->ct_enable) {
        // markers left out near contact (Sec. 2.2.5): the bitmap of this step's particle set
        st = contact_exclusion(ctx);
        if (st != IBM_OK) return st;
    }
    st = cluster_alloc(ctx);
    if (st != IBM_OK) return st;
    ClusterScratch *S = reinterpret_cast<ClusterScratch *>(ctx->cl);
    const int n = ctx->n_p;
    cudaStream_t sm = ctx->stream;
    // kernel variant: fixed, or autotuned over the first steps (see ibm_config)
    const int req = ctx->cfg.threads_per_block;
    // tuning steps 0 and 1 run each variant once untimed (module load, first-use allocations of the
    // fallback buffers), steps 2 and 3 time them
    const bool tuning = req < 0 && ctx->tune_step < kTuneSteps;
    const int tpb = req > 0 ? req : (req == 0 ? 1024 : (tuning ? ((ctx->tune_step & 1) ? 512 : 1024) : ctx->tuned_tpb));
    const int cap_m = tpb * markers_per_thread(tpb);
    const int spin = ctx->wait_limit > 0 ? ctx->wait_limit : kUnionSpin;
    // row table may take at most half of the dynamic shared memory
    const int max_rows = (max_dyn_smem(ctas_per_sm(tpb)) - fixed_smem_bytes<1024, 12>()) / 16;

    CK(cudaMemsetAsync(S->cnt, 0, C_COUNT * sizeof(int), sm), "zero counters");
    CK(cudaMemsetAsync(S->bin_cnt, 0, (S->nbins + 1) * sizeof(int), sm), "zero bins");
    CK(cudaMemsetAsync(S->bin_cur, 0, (S->nbins + 1) * sizeof(int), sm), "zero bins");
    CK(cudaMemsetAsync(S->bkt_cnt, 0, (kBuckets + 1) * sizeof(int), sm), "zero buckets");
    CK(cudaMemsetAsync(S->bkt_start + kBuckets + 1, 0, (kBuckets + 1) * sizeof(int), sm), "zero buckets");
    const int gb = grid_for(n, 256);
    k_bin_count<<<gb, 256, 0, sm>>>(n, ctx->pinfo, S->scene_nb, S->scene_bin_off, ctx->dims_d, S->bin_cnt,
                                    S->parent);
    k_scan1<<<1, 1024, 0, sm>>>(S->bin_cnt, S->bin_start, S->nbins, S->tot);
    k_bin_fill<<<gb, 256, 0, sm>>>(n, ctx->pinfo, S->scene_nb, S->scene_bin_off, ctx->dims_d, S->bin_start,
                                   S->bin_cur, S->bin_items);
    k_candidates<<<grid_for(27ll * n, 256), 256, 0, sm>>>(n, ctx->pinfo, S->scene_nb, S->scene_bin_off, ctx->dims_d,
                                                         S->bin_start, S->bin_items, S->cand, S->cap_cand, S->cnt);
    k_pair_test<<<std::min(S->cap_cand, 152 * 16), kPairThreads, 0, sm>>>(
        ctx->pinfo, ctx->tmpl32, ctx->tmpl64, ctx->dims_d, S->cand, S->cnt, S->cap_cand, S->parent, spin, ctx->err_d);
    k_roots<<<gb, 256, 0, sm>>>(n, S->parent, S->root_flag, spin, ctx->err_d);
    k_scan1<<<1, 1024, 0, sm>>>(S->root_flag, S->cid, n, S->tot + 1);
    k_cluster_init<<<gb, 256, 0, sm>>>(n, S->cl_np, S->cl_nm, S->cl_cur, S->cl_box);
    k_cluster_stats<<<gb, 256, 0, sm>>>(n, ctx->pinfo, ctx->dims_d, S->parent, S->cid, S->pcl, S->poff,
                                        S->cl_np, S->cl_nm, S->cl_box, spin);
    k_scan1<<<1, 1024, 0, sm>>>(S->cl_np, S->cl_first, n, S->tot + 2);
    k_cluster_fill<<<gb, 256, 0, sm>>>(n, S->pcl, S->cl_first, S->cl_cur, S->cl_plist);
    k_cluster_route<<<gb, 256, 0, sm>>>(S->tot + 1, ctx->pinfo, ctx->dims_d, S->cl_np, S->cl_nm, S->cl_first,
                                        S->cl_plist, S->cl_box, cap_m, max_rows, S->cl_bkt, S->bkt_cnt,
                                        S->fb_list, S->cl_scene, S->cl_path, S->cnt);
    k_scan1<<<1, 1024, 0, sm>>>(S->bkt_cnt, S->bkt_start, kBuckets, S->tot + 3);
    k_order_fill<<<gb, 256, 0, sm>>>(S->tot + 1, S->cl_bkt, S->bkt_start, S->bkt_start + kBuckets + 1, S->order);
    k_gather_nm<<<gb, 256, 0, sm>>>(n, S->cnt, S->order, S->cl_nm, S->nm_ord);
    k_scan1<<<1, 1024, 0, sm>>>(S->nm_ord, S->cum, n, S->tot + 3);
    // packing window = the record path's marker capacity
    const int window = tpb * records_per_thread(tpb);
    const long long max_windows = (ctx->n_markers + 32ll * n) / window + 2;
    k_batch_plan<<<grid_for(max_windows, 128), 128, 0, sm>>>(S->cnt, S->cum, S->order, S->cl_np, S->cl_nm,
                                                            S->cl_box, window, max_rows, S->batches, S->cnt);
    ctx->launches += 16;

    KParams prm;
    prm.P = ctx->pinfo;
    prm.t32 = ctx->tmpl32;
    prm.t64 = ctx->tmpl64;
    prm.dims = ctx->dims_d;
    prm.uf = reinterpret_cast<float *const *>(ctx->uptr_d);
    prm.ff = f_out ? reinterpret_cast<float *const *>(ctx->fptr_d) : nullptr;
    prm.order = S->order;
    prm.batches = S->batches;
    prm.cl_scene = S->cl_scene;
    prm.cl_path = S->cl_path;
    prm.max_rows = max_rows;
    prm.cl_first = S->cl_first;
    prm.cl_np = S->cl_np;
    prm.cl_nm = S->cl_nm;
    prm.cl_box = S->cl_box;
    prm.cl_plist = S->cl_plist;
    prm.poff = S->poff;
    prm.cnt = S->cnt;
    prm.fb_list = S->fb_list;
    prm.err = ctx->err_d;
    prm.dis = contact_bits(ctx);
    prm.FD = ctx->FD;
    prm.TD = ctx->TD;
    prm.n_forcing = ctx->cfg.n_forcing;
    prm.finv = (float)(1.0 / tau);
    prof_begin(ctx);
    cudaEvent_t tev[2] = {nullptr, nullptr};
    if (tuning && ctx->tune_step >= 2) {
        CK(cudaEventCreate(&tev[0]), "tuning event");
        CK(cudaEventCreate(&tev[1]), "tuning event");
        CK(cudaEventRecord(tev[0], sm), "tuning event");
    }
    const bool det = ctx->cfg.spread_mode == IBM_SPREAD_DETERMINISTIC;
    if (tpb == 1024)
        st = det ? launch_cluster_kernel<1024, 12, 2, true, 1>(ctx, S, prm)
                 : launch_cluster_kernel<1024, 12, 2, false, 1>(ctx, S, prm);
    else
        st = det ? launch_cluster_kernel<512, 12, 2, true, 2>(ctx, S, prm)
                 : launch_cluster_kernel<512, 12, 2, false, 2>(ctx, S, prm);
    prof_end(ctx);
    if (st == IBM_OK) {
        ctx->launches += 1;
        // clusters that did not fit one SM: a thread-block cluster's distributed shared memory where
        // their box fits it, else plain FP32 iterations over their particles
        const int *fbl = S->fb_list, *fbn = S->cnt + C_NFB;
        st = big_clusters(ctx, S, (float)(1.0 / tau), f_out != nullptr, det, &fbl, &fbn);
        if (st == IBM_OK)
            st = plain_iterations_f32(ctx, fbl, n, fbn, tau, f_out != nullptr, ctx->cfg.n_forcing,
                                      det ? S->pcl : nullptr);
    }
    if (tev[0]) {
        // tuning step: time this variant together with the fallback work its routing leaves (host sync);
        // keep the faster after both
        float ms = 0.f;
        if (st == IBM_OK) {
            cudaEventRecord(tev[1], sm);
            cudaEventSynchronize(tev[1]);
            cudaEventElapsedTime(&ms, tev[0], tev[1]);
        }
        cudaEventDestroy(tev[0]);
        cudaEventDestroy(tev[1]);
        ctx->tune_ms[ctx->tune_step - 2] = ms;
        if (ctx->tune_step == 3) ctx->tuned_tpb = ctx->tune_ms[0] <= ctx->tune_ms[1] ? 1024 : 512;
    }
    if (tuning && st == IBM_OK) ctx->tune_step += 1;
    return st;
}

void cluster_graph_key(const ibm_ctx *ctx, std::vector<uintptr_t> &key) {
    const ClusterScratch *S = reinterpret_cast<const ClusterScratch *>(ctx->cl);
    if (!S) {
        key.push_back(0);
        return;
    }
    const void *bufs[] = {S->scene_bin_off, S->scene_nb, S->bin_cnt, S->bin_start, S->bin_cur, S->bin_items,
                          S->parent, S->cand, S->cnt, S->tot, S->root_flag, S->cid, S->pcl, S->poff, S->cl_np,
                          S->cl_nm, S->cl_first, S->cl_cur, S->cl_box, S->cl_plist, S->cl_bkt, S->bkt_cnt,
                          S->bkt_start, S->order, S->fb_list, S->nm_ord, S->cum, S->cl_scene, S->cl_path,
                          S->batches, S->grec, S->big_list, S->big_flag, S->fb_list2, S->big_rec, S->big_part,
                          S->big_wl, S->big_list16};
    for (const void *b : bufs) key.push_back((uintptr_t)b);
    const long long sizes[] = {S->cap_p, S->cap_bins, S->cap_cand, S->nbins, S->max_nl, S->n_scenes,
                               S->smem_bytes, S->tpb, S->det, (long long)S->grec_bytes, S->big_k, S->big_grid8,
                               S->big_grid16, S->big_cells};
    for (long long v : sizes) key.push_back((uintptr_t)v);
}

ibm_status cluster_stats(ibm_ctx *ctx, int64_t *stats) {
    ClusterScratch *S = reinterpret_cast<ClusterScratch *>(ctx->cl);
    if (!S) return IBM_OK;
    int c[C_COUNT];
    long long nclust = 0;
    CK(cudaMemcpyAsync(c, S->cnt, sizeof(c), cudaMemcpyDeviceToHost, ctx->stream), "read stats");
    CK(cudaMemcpyAsync(&nclust, S->tot + 1, sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream), "read stats");
    CK(cudaStreamSynchronize(ctx->stream), "sync stats");
    stats[1] = nclust;
    stats[2] = c[C_NITEMS] - c[C_OVERFLOW];
    stats[3] = c[C_FBMARK] - c[C_BIGMARK];
    stats[4] = c[C_MAXCELLS];
    stats[5] = c[C_TOUCHED];
    stats[7] = S->tpb;
    stats[8] = c[C_ONECOMP];
    stats[9] = c[C_NCAND];
    stats[10] = c[C_NBIG];
    stats[11] = c[C_BIGMARK];
    return IBM_OK;
}

ibm_status cluster_membership(ibm_ctx *ctx, int32_t *cluster_of, int32_t *path_of, int64_t *n_clusters) {
    ClusterScratch *S = reinterpret_cast<ClusterScratch *>(ctx->cl);
    if (!S) return ibm_fail(ctx, IBM_ERR_STATE, "no cluster-path forcing step yet");
    const int n = ctx->n_p;
    long long nclust = 0;
    std::vector<int> pcl(std::max(n, 1)), path;
    CK(cudaMemcpyAsync(&nclust, S->tot + 1, sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream), "read clusters");
    CK(cudaMemcpyAsync(pcl.data(), S->pcl, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
       "read clusters");
    CK(cudaStreamSynchronize(ctx->stream), "read clusters");
    path.resize(std::max(nclust, 1ll));
    CK(cudaMemcpy(path.data(), S->cl_path, (size_t)nclust * sizeof(int), cudaMemcpyDeviceToHost), "read paths");
    if (n_clusters) *n_clusters = nclust;
    for (int p = 0; p < n; ++p) {
        if (cluster_of) cluster_of[p] = pcl[p];
        if (path_of) path_of[p] = (pcl[p] >= 0 && pcl[p] < nclust) ? path[pcl[p]] : 0;
    }
    return IBM_OK;
}
