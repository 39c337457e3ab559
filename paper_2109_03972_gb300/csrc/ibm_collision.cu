// Collision models and the RK3 particle sub-steps, Sec. 2.2.6-2.2.8 (Eq.
// f_int: lubrication with the erf blend, Hertz normal contact with ACTM
// coefficients, spring-dashpot tangential contact with stick/slip) and Sec.
// 2.2.10 (n_sub sub-steps, each the three-stage predictor-corrector update of
// the particle equations under constant hydrodynamic loads).
//
// Readings of the paper (it refers to its sources for some closed forms):
//  - triply periodic boxes, no walls; pair geometry by minimum image;
//  - n = (x_q - x_p)/|x_q - x_p|, zeta_n = |x_q - x_p| - R_p - R_q, contact
//    point R_p,cp = (|x_q - x_p| + R_p - R_q)/2 from x_p along n, and
//    g_cp = (u_p + w_p x R_p,cp n) - (u_q + w_q x (-R_q,cp n));
//  - lubrication for 0 < zeta_n < eps_sep, contact for zeta_n <= 0;
//  - ACTM: the undamped Hertz impact at speed u lasts T_c when
//    k = m_eff / sqrt(u t*^5), t* = T_c (4/5)^{2/5} / (2 I_H),
//    I_H = sqrt(pi) Gamma(7/5)/Gamma(9/10) (the form of the printed k_n,crit);
//    k_n at the recorded impact speed u_in above u_in,crit (from St_crit, the
//    larger of the two particles' values), else max(k at u_in,crit, k_n,grav);
//    d_n = -2 m_eff ln(e_dry) / T_c;
//  - k_t = 2 (1 - nu)/(2 - nu) k_n, d_t as printed; stick while
//    |F_t,dp| < mu_s |F_n|, else |F_t| = mu_k |F_n|, and on slip the spring is
//    reset to the Coulomb limit (Luding) when the history advances;
//  - the spring zeta_t advances once per RK stage by 2 alpha_k dt_sub g_t at
//    the corrected state, kept in the tangent plane; it and u_in (|g_cp . n|
//    at first contact) live while the pair touches;
//  - RK3 coefficients of Rai and Moin; m_p = rho_p pi d^3/6, I_p = m_p d^2/10,
//    g' = (1 - rho_f/rho_p) g.
//
// GPU layout.  Once per call: particles binned per scene on a cell list (bins
// at least 2 R_max + eps_sep + margin wide, the items of each bin sorted by
// index), and every particle's list of the neighbours within eps_sep + margin
// (both directions, in a fixed order).  The pair state (spring, impact speed)
// lives in the entry of the pair's lower index.  Per RK stage: the collision
// loads of every particle gathered over its list in that order (no atomics,
// bit-reproducible), the predictor, the loads at the predicted state, the
// corrector, the history update per pair.  At the end: a check that no
// particle moved more than half the margin since the list was built (else
// IBM_ERR_CAPACITY: pairs could have been missed), and the pairs in contact
// kept, per particle, for the next call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
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

constexpr int kColBlock = 128;
constexpr double kPi = 3.14159265358979323846;

// Parameters of one call, derived on the host.
struct ColPrm {
    double rho_f, nu_f, mu_s, mu_k;
    double eps, zmin, lub_c, h;
    double tstar5;       // t*^5
    double ln_e;         // ln(e_dry)
    double t_c;
    double st9;          // 9 St_crit rho_f nu_f
    double kt_ratio;     // 2 (1 - nu)/(2 - nu)
    double g[3], gmag;
    double cut;          // eps_sep + margin: the neighbour-list reach beyond the surfaces
};

struct ColScratch {
    int cap_p = 0, n_scenes = 0, nbins = 0;
    long long cap_e = 0, cap_h = 0;
    int *scene_nb = nullptr, *scene_off = nullptr;
    int *bin_of = nullptr, *bin_cnt = nullptr, *bin_start = nullptr, *bin_cur = nullptr, *items = nullptr;
    int *ncnt = nullptr, *nstart = nullptr;     // neighbour counts / offsets per particle
    int *nbr = nullptr, *canon = nullptr;       // [cap_e] neighbour, canonical entry of the pair
    double *zt = nullptr, *uin = nullptr;       // [cap_e][3], [cap_e] pair state (lower index's entry)
    int *has = nullptr;                         // [cap_e] pair in contact (state valid)
    double *F0 = nullptr, *T0 = nullptr, *F1 = nullptr, *T1 = nullptr;
    double *xt = nullptr, *ut = nullptr, *wt = nullptr, *xb = nullptr, *fh = nullptr, *th = nullptr;
    long long *tot = nullptr;
    // contact history kept between calls: per particle p, its pairs (p, q > p)
    int hist_np = -1;
    int *hoff = nullptr, *hcnt = nullptr, *hq = nullptr;
    double *hz = nullptr, *hu = nullptr;
};

template <typename T>
cudaError_t dev_realloc(T **p, size_t bytes) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    return ibm_malloc(p, bytes);
}

__device__ __forceinline__ double mass(double d, double rho) { return rho * kPi * d * d * d / 6.0; }

__device__ __forceinline__ double min_img(double v, double L) { return v - L * floor(v / L + 0.5); }

__device__ __forceinline__ int bin_axis(double x, double L, int nb) {
    const double w = x - L * floor(x / L);
    return min(nb - 1, max(0, (int)(w * nb / L)));
}

// Exclusive scan of n ints into out[0..n] by one block; *total = the sum.
__global__ void k_col_scan(const int *in, int *out, int n, long long *total) {
    __shared__ long long part[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int chunk = (n + T - 1) / T;
    const int lo = min(n, t * chunk), hi = min(n, lo + chunk);
    long long s = 0;
    for (int i = lo; i < hi; ++i) s += in[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {
        const long long v = t >= o ? part[t - o] : 0;
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

__global__ void k_col_bin(int n, const double *x, const int32_t *scene, const int32_t *dims, double h,
                          const int *scene_nb, const int *scene_off, int *bin_of, int *bin_cnt) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int s = scene[p];
        int b[3];
        for (int c = 0; c < 3; ++c) b[c] = bin_axis(x[3 * p + c], dims[3 * s + c] * h, scene_nb[3 * s + c]);
        const int bin = scene_off[s] + (b[2] * scene_nb[3 * s + 1] + b[1]) * scene_nb[3 * s] + b[0];
        bin_of[p] = bin;
        atomicAdd(bin_cnt + bin, 1);
    }
}

__global__ void k_col_fill(int n, const int *bin_of, const int *bin_start, int *bin_cur, int *items) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int b = bin_of[p];
        items[bin_start[b] + atomicAdd(bin_cur + b, 1)] = p;
    }
}

// The items of every bin in ascending particle order (insertion sort; bins
// hold a handful of particles), so that the neighbour lists come out the same
// on every run.
__global__ void k_col_sort_bins(int nbins, const int *bin_start, int *items) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
        const int lo = bin_start[b], hi = bin_start[b + 1];
        for (int i = lo + 1; i < hi; ++i) {
            const int v = items[i];
            int j = i - 1;
            while (j >= lo && items[j] > v) {
                items[j + 1] = items[j];
                --j;
            }
            items[j + 1] = v;
        }
    }
}

// Neighbours of particle p within cut of its surface (COUNT: how many; else
// write them at nbr[nstart[p]...]), over the distinct neighbouring bins in a
// fixed order.
template <bool COUNT>
__global__ void k_col_list(int n, const double *x, const double *d, const int32_t *scene, const int32_t *dims,
                           double h, const int *scene_nb, const int *scene_off, const int *bin_start,
                           const int *items, double cut, int *ncnt, const int *nstart, int *nbr) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int s = scene[p];
        const int nb[3] = {scene_nb[3 * s], scene_nb[3 * s + 1], scene_nb[3 * s + 2]};
        const double L[3] = {dims[3 * s] * h, dims[3 * s + 1] * h, dims[3 * s + 2] * h};
        int b[3];
        for (int c = 0; c < 3; ++c) b[c] = bin_axis(x[3 * p + c], L[c], nb[c]);
        int k = 0, w = COUNT ? 0 : nstart[p];
        // neighbouring bin offsets per axis, each bin once when an axis has < 3 bins
        for (int oz = -1; oz <= 1; ++oz) {
            if (nb[2] < 3 && oz + 1 >= nb[2]) continue;
            const int bz = nb[2] >= 3 ? (b[2] + oz + nb[2]) % nb[2] : oz + 1;
            for (int oy = -1; oy <= 1; ++oy) {
                if (nb[1] < 3 && oy + 1 >= nb[1]) continue;
                const int by = nb[1] >= 3 ? (b[1] + oy + nb[1]) % nb[1] : oy + 1;
                for (int ox = -1; ox <= 1; ++ox) {
                    if (nb[0] < 3 && ox + 1 >= nb[0]) continue;
                    const int bx = nb[0] >= 3 ? (b[0] + ox + nb[0]) % nb[0] : ox + 1;
                    const int bin = scene_off[s] + (bz * nb[1] + by) * nb[0] + bx;
                    for (int i = bin_start[bin]; i < bin_start[bin + 1]; ++i) {
                        const int q = items[i];
                        if (q == p) continue;
                        double r2 = 0.0;
                        for (int c = 0; c < 3; ++c) {
                            const double v = min_img(x[3 * q + c] - x[3 * p + c], L[c]);
                            r2 += v * v;
                        }
                        const double lim = 0.5 * (d[p] + d[q]) + cut;
                        if (r2 < lim * lim) {
                            if (!COUNT) nbr[w] = q;
                            ++w;
                            ++k;
                        }
                    }
                }
            }
        }
        if (COUNT) ncnt[p] = k;
    }
}

// Canonical entry of every pair (the lower index's), and the state of the
// pairs that were in contact at the end of the previous call.
__global__ void k_col_canon(int n, const int *nstart, const int *nbr, int *canon, double *zt, double *uin, int *has,
                            int use_hist, const int *hoff, const int *hcnt, const int *hq, const double *hz,
                            const double *hu) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        for (int j = nstart[p]; j < nstart[p + 1]; ++j) {
            const int q = nbr[j];
            if (q > p) {
                canon[j] = j;
                has[j] = 0;
                uin[j] = -1.0;
                zt[3 * j] = zt[3 * j + 1] = zt[3 * j + 2] = 0.0;
                if (use_hist)
                    for (int k = hoff[p]; k < hoff[p] + hcnt[p]; ++k)
                        if (hq[k] == q) {
                            has[j] = 1;
                            uin[j] = hu[k];
                            for (int c = 0; c < 3; ++c) zt[3 * j + c] = hz[3 * k + c];
                        }
            } else {
                int c = -1;
                for (int k = nstart[q]; k < nstart[q + 1]; ++k)
                    if (nbr[k] == p) c = k;
                canon[j] = c;
            }
        }
    }
}

// Normal stiffness (ACTM reading, see the file header).
__device__ __forceinline__ double col_kn(const ColPrm &P, double m_eff, double uin, double rs, double ds, double ro,
                                         double dd_o, double ms, double mo) {
    const double uc = fmax(P.st9 / (rs * ds), P.st9 / (ro * dd_o));
    if (uin > uc) return m_eff / sqrt(uin * P.tstar5);
    const double kc = uc > 0.0 ? m_eff / sqrt(uc * P.tstar5) : 0.0;
    const double kg = fmax(ms * P.gmag * pow(1e-3 * 0.5 * ds, -1.5), mo * P.gmag * pow(1e-3 * 0.5 * dd_o, -1.5));
    return fmax(kc, kg);
}

// Pair geometry seen from `self` with the other particle at dv = x_o - x_s.
struct PairGeo {
    double n[3], zeta, dist, rcs, rco, gns, gn[3], gt[3];
};

__device__ __forceinline__ void col_geo(const double *dv, const double *us, const double *uo, const double *ws,
                                        const double *wo, double Rs, double Ro, PairGeo &G) {
    G.dist = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    for (int c = 0; c < 3; ++c) G.n[c] = dv[c] / G.dist;
    G.zeta = G.dist - Rs - Ro;
    G.rcs = 0.5 * (G.dist + Rs - Ro);
    G.rco = 0.5 * (G.dist + Ro - Rs);
    const double as[3] = {G.rcs * G.n[0], G.rcs * G.n[1], G.rcs * G.n[2]};
    const double ao[3] = {-G.rco * G.n[0], -G.rco * G.n[1], -G.rco * G.n[2]};
    const double cs[3] = {ws[1] * as[2] - ws[2] * as[1], ws[2] * as[0] - ws[0] * as[2], ws[0] * as[1] - ws[1] * as[0]};
    const double co[3] = {wo[1] * ao[2] - wo[2] * ao[1], wo[2] * ao[0] - wo[0] * ao[2], wo[0] * ao[1] - wo[1] * ao[0]};
    double g[3];
    for (int c = 0; c < 3; ++c) g[c] = (us[c] + cs[c]) - (uo[c] + co[c]);
    G.gns = g[0] * G.n[0] + g[1] * G.n[1] + g[2] * G.n[2];
    for (int c = 0; c < 3; ++c) {
        G.gn[c] = G.gns * G.n[c];
        G.gt[c] = g[c] - G.gn[c];
    }
}

// Force and torque on `self` from the pair (Eq. f_int and the three models).
__device__ void col_pair(const ColPrm &P, const double *dv, const double *us, const double *uo, const double *ws,
                         const double *wo, double ds, double dd_o, double rs, double ro, const double *zt,
                         double uin, double *F, double *T) {
    const double Rs = 0.5 * ds, Ro = 0.5 * dd_o;
    for (int c = 0; c < 3; ++c) F[c] = T[c] = 0.0;
    // most list entries lie beyond eps_sep: decide on the gap before the rest
    // of the geometry (the same FP64 expression as col_geo)
    if (sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]) - Rs - Ro >= P.eps) return;
    PairGeo G;
    col_geo(dv, us, uo, ws, wo, Rs, Ro, G);
    const double ms = mass(ds, rs), mo = mass(dd_o, ro);
    const double m_eff = ms * mo / (ms + mo);
    if (G.zeta > 0.0) {
        const double R_eff = Rs * Ro / (Rs + Ro);
        const double zm = G.zeta > P.zmin ? G.zeta : P.zmin;
        const double psi = 0.5 * erf(6.0 - P.lub_c * zm / P.h) + 0.5;
        const double coef = 6.0 * kPi * P.rho_f * P.nu_f * R_eff * R_eff * psi / zm;
        for (int c = 0; c < 3; ++c) F[c] = -coef * G.gn[c];
        return;
    }
    const double u_in = uin >= 0.0 ? uin : fabs(G.gns);
    const double kn = col_kn(P, m_eff, u_in, rs, ds, ro, dd_o, ms, mo);
    const double dn = -2.0 * m_eff * P.ln_e / P.t_c;
    const double ov = pow(-G.zeta, 1.5);
    double Fn[3];
    for (int c = 0; c < 3; ++c) Fn[c] = -kn * ov * G.n[c] - dn * G.gn[c];
    const double kt = P.kt_ratio * kn;
    const double dt = 2.0 * sqrt(m_eff * kt) * (-P.ln_e) / sqrt(kPi * kPi + P.ln_e * P.ln_e);
    double Fdp[3];
    for (int c = 0; c < 3; ++c) Fdp[c] = -kt * zt[c] - dt * G.gt[c];
    const double fn = sqrt(Fn[0] * Fn[0] + Fn[1] * Fn[1] + Fn[2] * Fn[2]);
    const double fdp = sqrt(Fdp[0] * Fdp[0] + Fdp[1] * Fdp[1] + Fdp[2] * Fdp[2]);
    double Ft[3];
    if (fdp < P.mu_s * fn || fdp == 0.0) {
        for (int c = 0; c < 3; ++c) Ft[c] = Fdp[c];
    } else {
        for (int c = 0; c < 3; ++c) Ft[c] = P.mu_k * fn * Fdp[c] / fdp;
    }
    for (int c = 0; c < 3; ++c) F[c] = Fn[c] + Ft[c];
    const double as[3] = {G.rcs * G.n[0], G.rcs * G.n[1], G.rcs * G.n[2]};
    T[0] = as[1] * Ft[2] - as[2] * Ft[1];
    T[1] = as[2] * Ft[0] - as[0] * Ft[2];
    T[2] = as[0] * Ft[1] - as[1] * Ft[0];
}

// Collision loads of particle p over its neighbour list, in list order.
__device__ __forceinline__ void col_loads(int p, const ColPrm &P, const double *x, const double *u,
                                          const double *om, const double *d, const double *rho,
                                          const int32_t *scene, const int32_t *dims, const int *nstart,
                                          const int *nbr, const int *canon, const double *zt, const double *uin,
                                          const int *has, double Fs[3], double Ts[3]) {
    const int s = scene[p];
    const double L[3] = {dims[3 * s] * P.h, dims[3 * s + 1] * P.h, dims[3 * s + 2] * P.h};
    for (int k = 0; k < 3; ++k) Fs[k] = Ts[k] = 0.0;
    for (int j = nstart[p]; j < nstart[p + 1]; ++j) {
        const int q = nbr[j], c = canon[j];
        double dv[3], z[3] = {0, 0, 0}, ui = -1.0;
        for (int k = 0; k < 3; ++k) dv[k] = min_img(x[3 * q + k] - x[3 * p + k], L[k]);
        if (c >= 0 && has[c]) {
            const double sgn = p < q ? 1.0 : -1.0;   // the state is stored in the lower index's frame
            for (int k = 0; k < 3; ++k) z[k] = sgn * zt[3 * c + k];
            ui = uin[c];
        }
        double F[3], T[3];
        col_pair(P, dv, u + 3 * p, u + 3 * q, om + 3 * p, om + 3 * q, d[p], d[q], rho[p], rho[q], z, ui, F, T);
        for (int k = 0; k < 3; ++k) {
            Fs[k] += F[k];
            Ts[k] += T[k];
        }
    }
}

// Collision loads of every particle at (x, u, om).
__global__ void __launch_bounds__(kColBlock) k_col_force(int n, ColPrm P, const double *x, const double *u,
                                                         const double *om, const double *d, const double *rho,
                                                         const int32_t *scene, const int32_t *dims,
                                                         const int *nstart, const int *nbr, const int *canon,
                                                         const double *zt, const double *uin, const int *has,
                                                         double *Fc, double *Tc) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        double Fs[3], Ts[3];
        col_loads(p, P, x, u, om, d, rho, scene, dims, nstart, nbr, canon, zt, uin, has, Fs, Ts);
        for (int k = 0; k < 3; ++k) {
            Fc[3 * p + k] = Fs[k];
            Tc[3 * p + k] = Ts[k];
        }
    }
}

// Half of an RK stage (Sec. 2.2.10) for every particle: the collision loads
// at (xs, us, ws) -- the state at the start of the stage for the predictor,
// the predicted state for the corrector -- then the update
//   u' = u^{k-1} + ds/m (2 alpha F_h + gamma F + zeta Fb) + 2 alpha ds g'
//   w' = w^{k-1} + ds/I (2 alpha T_h + gamma T + zeta Tb)
//   x' = x^{k-1} + alpha ds (u' + u^{k-1})
// with Fb = F_c(x^{k-2}) for the predictor and F_c(x^{k-1}) for the
// corrector.  The predictor (CORRECT = false) keeps its loads in Fa, Ta (the
// corrector's Fb) and writes (xo, uo, wo); the corrector advances (x, u, w)
// in place, which no thread of its launch reads (its loads are taken at the
// predicted state).
template <bool CORRECT>
__global__ void __launch_bounds__(kColBlock) k_col_stage(
    int n, ColPrm P, double a, double g, double z, double ds, const double *xs, const double *us, const double *ws,
    const double *d, const double *rho, const int32_t *scene, const int32_t *dims, const int *nstart,
    const int *nbr, const int *canon, const double *zt, const double *uin, const int *has, const double *Fh,
    const double *Th, double *Fa, double *Ta, const double *Fb, const double *Tb, double *x, double *u, double *w,
    double *xo, double *uo, double *wo, int *err) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        double Fs[3], Ts[3];
        col_loads(p, P, xs, us, ws, d, rho, scene, dims, nstart, nbr, canon, zt, uin, has, Fs, Ts);
        const double m = mass(d[p], rho[p]);
        if (!(m > 0.0)) {
            set_err(err, IBM_EBIT_MASS);
            continue;
        }
        const double I = m * d[p] * d[p] / 10.0;
        const double gr = 1.0 - P.rho_f / rho[p];
        for (int c = 0; c < 3; ++c) {
            const int i = 3 * p + c;
            if (!CORRECT) {
                Fa[i] = Fs[c];
                Ta[i] = Ts[c];
            }
            const double fh = Fh ? Fh[i] : 0.0, th = Th ? Th[i] : 0.0;
            const double un = u[i] + ds / m * (2.0 * a * fh + g * Fs[c] + z * Fb[i]) + 2.0 * a * ds * gr * P.g[c];
            const double wn = w[i] + ds / I * (2.0 * a * th + g * Ts[c] + z * Tb[i]);
            const double xn = x[i] + a * ds * (un + u[i]);
            if (CORRECT) {
                x[i] = xn;
                u[i] = un;
                w[i] = wn;
            } else {
                xo[i] = xn;
                uo[i] = un;
                wo[i] = wn;
            }
        }
    }
}

// History of every pair at the end of a stage of duration dts (from the
// corrected state): spring advanced in the tangent plane, impact speed at
// first contact, the Coulomb reset on slip; cleared when the pair separates.
__global__ void k_col_history(int n, ColPrm P, double dts, const double *x, const double *u, const double *om,
                              const double *d, const double *rho, const int32_t *scene, const int32_t *dims,
                              const int *nstart, const int *nbr, double *zt, double *uin, int *has) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int s = scene[p];
        const double L[3] = {dims[3 * s] * P.h, dims[3 * s + 1] * P.h, dims[3 * s + 2] * P.h};
        for (int j = nstart[p]; j < nstart[p + 1]; ++j) {
            const int q = nbr[j];
            if (q < p) continue;
            double dv[3];
            for (int k = 0; k < 3; ++k) dv[k] = min_img(x[3 * q + k] - x[3 * p + k], L[k]);
            const bool apart = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]) - 0.5 * d[p] - 0.5 * d[q] > 0.0;
            if (apart) {
                if (has[j]) {
                    has[j] = 0;
                    uin[j] = -1.0;
                    zt[3 * j] = zt[3 * j + 1] = zt[3 * j + 2] = 0.0;
                }
                continue;
            }
            PairGeo G;
            col_geo(dv, u + 3 * p, u + 3 * q, om + 3 * p, om + 3 * q, 0.5 * d[p], 0.5 * d[q], G);
            if (G.zeta > 0.0) {
                has[j] = 0;
                uin[j] = -1.0;
                zt[3 * j] = zt[3 * j + 1] = zt[3 * j + 2] = 0.0;
                continue;
            }
            double z[3] = {0, 0, 0};
            double ui = fabs(G.gns);
            if (has[j]) {
                for (int k = 0; k < 3; ++k) z[k] = zt[3 * j + k];
                ui = uin[j];
            }
            for (int k = 0; k < 3; ++k) z[k] += dts * G.gt[k];
            const double zn = z[0] * G.n[0] + z[1] * G.n[1] + z[2] * G.n[2];
            for (int k = 0; k < 3; ++k) z[k] -= zn * G.n[k];
            const double mp = mass(d[p], rho[p]), mq = mass(d[q], rho[q]);
            const double m_eff = mp * mq / (mp + mq);
            const double kn = col_kn(P, m_eff, ui, rho[p], d[p], rho[q], d[q], mp, mq);
            const double dn = -2.0 * m_eff * P.ln_e / P.t_c;
            const double ov = pow(-G.zeta, 1.5);
            double Fn[3];
            for (int k = 0; k < 3; ++k) Fn[k] = -kn * ov * G.n[k] - dn * G.gns * G.n[k];
            const double kt = P.kt_ratio * kn;
            const double dt = 2.0 * sqrt(m_eff * kt) * (-P.ln_e) / sqrt(kPi * kPi + P.ln_e * P.ln_e);
            double Fdp[3];
            for (int k = 0; k < 3; ++k) Fdp[k] = -kt * z[k] - dt * G.gt[k];
            const double fn = sqrt(Fn[0] * Fn[0] + Fn[1] * Fn[1] + Fn[2] * Fn[2]);
            const double fdp = sqrt(Fdp[0] * Fdp[0] + Fdp[1] * Fdp[1] + Fdp[2] * Fdp[2]);
            if (!(fdp < P.mu_s * fn) && fdp > 0.0)
                for (int k = 0; k < 3; ++k) z[k] = -(P.mu_k * fn * Fdp[k] / fdp + dt * G.gt[k]) / kt;
            for (int k = 0; k < 3; ++k) zt[3 * j + k] = z[k];
            uin[j] = ui;
            has[j] = 1;
        }
    }
}

// Displacement since the list was built must stay below half the margin.
__global__ void k_col_margin(int n, const double *x, const double *xb, const int32_t *scene, const int32_t *dims,
                             double h, double half_margin, int *err) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int s = scene[p];
        double r2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double v = min_img(x[3 * p + c] - xb[3 * p + c], dims[3 * s + c] * h);
            r2 += v * v;
        }
        if (!(r2 <= half_margin * half_margin)) set_err(err, IBM_EBIT_OVERFLOW);
    }
}

// Pairs in contact kept per particle for the next call (count, then fill).
template <bool COUNT>
__global__ void k_col_keep(int n, const int *nstart, const int *nbr, const double *zt, const double *uin,
                           const int *has, int *hcnt, const int *hoff, int *hq, double *hz, double *hu) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        int k = 0;
        for (int j = nstart[p]; j < nstart[p + 1]; ++j) {
            if (nbr[j] < p || !has[j]) continue;
            if (!COUNT) {
                const int o = hoff[p] + k;
                hq[o] = nbr[j];
                hu[o] = uin[j];
                for (int c = 0; c < 3; ++c) hz[3 * o + c] = zt[3 * j + c];
            }
            ++k;
        }
        if (COUNT) hcnt[p] = k;
    }
}

int grid_n(int n) { return std::max(1, std::min((n + kColBlock - 1) / kColBlock, 152 * 16)); }

ibm_status col_params(ibm_ctx *ctx, const ibm_collision_params *in, ColPrm &P, double &margin) {
    const double h = ctx->cfg.h;
    const bool four = ctx->cfg.kernel_width == 4;
    if (!(in->rho_f > 0.0) || !(in->nu_f >= 0.0) || !(in->e_dry > 0.0 && in->e_dry < 1.0) || !(in->mu_s >= 0.0) ||
        !(in->mu_k >= 0.0) || !(in->nu_poisson >= 0.0 && in->nu_poisson < 1.0) || !(in->t_c > 0.0) ||
        !(in->st_crit >= 0.0) || !(in->eps_sep >= 0.0) || !(in->zeta_min >= 0.0) || !(in->lub_c >= 0.0) ||
        !(in->pair_margin >= 0.0))
        return ibm_fail(ctx, IBM_ERR_INVALID_ARG, "collision parameters out of range");
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(in->g[c])) return ibm_fail(ctx, IBM_ERR_INVALID_ARG, "gravity must be finite");
    P.rho_f = in->rho_f;
    P.nu_f = in->nu_f;
    P.mu_s = in->mu_s;
    P.mu_k = in->mu_k;
    P.eps = in->eps_sep > 0.0 ? in->eps_sep : (four ? 2.0 : 1.5) * h;
    P.zmin = in->zeta_min > 0.0 ? in->zeta_min : 0.01 * h;
    P.lub_c = in->lub_c > 0.0 ? in->lub_c : (four ? 4.0 : 5.5);
    P.h = h;
    const double ih = std::sqrt(kPi) * std::tgamma(1.4) / std::tgamma(0.9);
    const double ts = in->t_c * std::pow(0.8, 0.4) / (2.0 * ih);
    P.tstar5 = std::pow(ts, 5.0);
    P.ln_e = std::log(in->e_dry);
    P.t_c = in->t_c;
    P.st9 = 9.0 * in->st_crit * in->rho_f * in->nu_f;
    P.kt_ratio = 2.0 * (1.0 - in->nu_poisson) / (2.0 - in->nu_poisson);
    for (int c = 0; c < 3; ++c) P.g[c] = in->g[c];
    P.gmag = std::sqrt(in->g[0] * in->g[0] + in->g[1] * in->g[1] + in->g[2] * in->g[2]);
    margin = in->pair_margin > 0.0 ? in->pair_margin : 1.5 * h;
    P.cut = P.eps + margin;
    return IBM_OK;
}

ColScratch *col_scratch(ibm_ctx *ctx) {
    if (!ctx->col) ctx->col = new (std::nothrow) ColScratch();
    return reinterpret_cast<ColScratch *>(ctx->col);
}

// Neighbour lists of the current state (and the canonical entries with the
// kept history); *n_entries receives the list length.
ibm_status col_build(ibm_ctx *ctx, ColScratch *S, const ColPrm &P, long long *n_entries) {
    const int n = ctx->n_p, ns = ctx->cfg.n_scenes;
    cudaStream_t sm = ctx->stream;
    if (S->cap_p < ctx->cap_p) {
        const size_t c = (size_t)ctx->cap_p + 1;
        S->cap_p = 0;
        CK(dev_realloc(&S->bin_of, c * sizeof(int)), "alloc collision scratch");
        CK(dev_realloc(&S->ncnt, c * sizeof(int)), "alloc collision scratch");
        CK(dev_realloc(&S->nstart, c * sizeof(int)), "alloc collision scratch");
        CK(dev_realloc(&S->items, c * sizeof(int)), "alloc collision scratch");
        CK(dev_realloc(&S->hoff, c * sizeof(int)), "alloc collision scratch");
        CK(dev_realloc(&S->hcnt, c * sizeof(int)), "alloc collision scratch");
        double **v3[] = {&S->F0, &S->T0, &S->F1, &S->T1, &S->xt, &S->ut, &S->wt, &S->xb,
                         &S->fh, &S->th};
        for (double **p : v3) CK(dev_realloc(p, 3 * c * sizeof(double)), "alloc collision scratch");
        if (!S->tot) CK(ibm_malloc(&S->tot, 4 * sizeof(long long)), "alloc collision scratch");
        S->cap_p = ctx->cap_p;
        S->hist_np = -1;
    }
    // bins of each scene at least 2 R_max + cut wide
    double dmax = 0.0;
    {
        std::vector<double> dh(n);
        CK(cudaMemcpyAsync(dh.data(), ctx->d, n * sizeof(double), cudaMemcpyDeviceToHost, sm), "read diameters");
        CK(cudaStreamSynchronize(sm), "read diameters");
        for (double v : dh) dmax = std::max(dmax, v);
    }
    const double bw = dmax + P.cut + 1e-9;
    std::vector<int> nb(3 * ns), off(ns + 1);
    long long total = 0;
    for (int s = 0; s < ns; ++s) {
        off[s] = (int)total;
        long long cells = 1;
        for (int c = 0; c < 3; ++c) {
            nb[3 * s + c] = std::max(1, (int)std::floor(ctx->dims_h[3 * s + c] * ctx->cfg.h / bw));
            cells *= nb[3 * s + c];
        }
        total += cells;
    }
    off[ns] = (int)total;
    if (total > (1 << 26)) return ibm_fail(ctx, IBM_ERR_CAPACITY, "too many collision bins");
    if (S->nbins < (int)total || S->n_scenes != ns) {
        S->nbins = 0;
        CK(dev_realloc(&S->scene_nb, nb.size() * sizeof(int)), "alloc collision bins");
        CK(dev_realloc(&S->scene_off, off.size() * sizeof(int)), "alloc collision bins");
        CK(dev_realloc(&S->bin_cnt, (total + 1) * sizeof(int)), "alloc collision bins");
        CK(dev_realloc(&S->bin_start, (total + 1) * sizeof(int)), "alloc collision bins");
        CK(dev_realloc(&S->bin_cur, (total + 1) * sizeof(int)), "alloc collision bins");
        S->nbins = (int)total;
        S->n_scenes = ns;
    }
    CK(cudaMemcpyAsync(S->scene_nb, nb.data(), nb.size() * sizeof(int), cudaMemcpyHostToDevice, sm), "copy bins");
    CK(cudaMemcpyAsync(S->scene_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice, sm), "copy bins");
    CK(cudaMemsetAsync(S->bin_cnt, 0, (total + 1) * sizeof(int), sm), "zero bins");
    CK(cudaMemsetAsync(S->bin_cur, 0, (total + 1) * sizeof(int), sm), "zero bins");
    const int gb = grid_n(n);
    const double h = ctx->cfg.h;
    k_col_bin<<<gb, kColBlock, 0, sm>>>(n, ctx->x, ctx->scene, ctx->dims_d, h, S->scene_nb, S->scene_off, S->bin_of,
                                        S->bin_cnt);
    k_col_scan<<<1, 1024, 0, sm>>>(S->bin_cnt, S->bin_start, (int)total, S->tot);
    k_col_fill<<<gb, kColBlock, 0, sm>>>(n, S->bin_of, S->bin_start, S->bin_cur, S->items);
    k_col_sort_bins<<<grid_n((int)total), kColBlock, 0, sm>>>((int)total, S->bin_start, S->items);
    k_col_list<true><<<gb, kColBlock, 0, sm>>>(n, ctx->x, ctx->d, ctx->scene, ctx->dims_d, h, S->scene_nb,
                                               S->scene_off, S->bin_start, S->items, P.cut, S->ncnt, nullptr,
                                               nullptr);
    k_col_scan<<<1, 1024, 0, sm>>>(S->ncnt, S->nstart, n, S->tot + 1);
    long long ne = 0;
    CK(cudaMemcpyAsync(&ne, S->tot + 1, sizeof(long long), cudaMemcpyDeviceToHost, sm), "read list length");
    CK(cudaStreamSynchronize(sm), "read list length");
    if (ne > INT32_MAX / 4) return ibm_fail(ctx, IBM_ERR_CAPACITY, "too many collision pairs");
    if (S->cap_e < std::max(ne, 1ll)) {
        const long long c = std::max(2 * ne, 1024ll);
        S->cap_e = 0;
        CK(dev_realloc(&S->nbr, c * sizeof(int)), "alloc neighbour lists");
        CK(dev_realloc(&S->canon, c * sizeof(int)), "alloc neighbour lists");
        CK(dev_realloc(&S->has, c * sizeof(int)), "alloc neighbour lists");
        CK(dev_realloc(&S->uin, c * sizeof(double)), "alloc neighbour lists");
        CK(dev_realloc(&S->zt, 3 * c * sizeof(double)), "alloc neighbour lists");
        S->cap_e = c;
    }
    k_col_list<false><<<gb, kColBlock, 0, sm>>>(n, ctx->x, ctx->d, ctx->scene, ctx->dims_d, h, S->scene_nb,
                                                S->scene_off, S->bin_start, S->items, P.cut, nullptr, S->nstart,
                                                S->nbr);
    const int use_hist = S->hist_np == n ? 1 : 0;
    k_col_canon<<<gb, kColBlock, 0, sm>>>(n, S->nstart, S->nbr, S->canon, S->zt, S->uin, S->has, use_hist, S->hoff,
                                          S->hcnt, S->hq, S->hz, S->hu);
    CK(cudaMemcpyAsync(S->xb, ctx->x, 3 * (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, sm), "save x");
    ctx->launches += 9;
    *n_entries = ne;
    return ibm_cuda_check(ctx, cudaGetLastError(), "collision lists");
}

// Pairs in contact kept for the next call.
ibm_status col_keep(ibm_ctx *ctx, ColScratch *S) {
    const int n = ctx->n_p;
    cudaStream_t sm = ctx->stream;
    const int gb = grid_n(n);
    k_col_keep<true><<<gb, kColBlock, 0, sm>>>(n, S->nstart, S->nbr, S->zt, S->uin, S->has, S->hcnt, nullptr,
                                               nullptr, nullptr, nullptr);
    k_col_scan<<<1, 1024, 0, sm>>>(S->hcnt, S->hoff, n, S->tot + 2);
    long long nh = 0;
    CK(cudaMemcpyAsync(&nh, S->tot + 2, sizeof(long long), cudaMemcpyDeviceToHost, sm), "read contacts");
    CK(cudaStreamSynchronize(sm), "read contacts");
    S->hist_np = -1;
    if (S->cap_h < std::max(nh, 1ll)) {
        const long long c = std::max(2 * nh, 256ll);
        S->cap_h = 0;
        CK(dev_realloc(&S->hq, c * sizeof(int)), "alloc contact history");
        CK(dev_realloc(&S->hu, c * sizeof(double)), "alloc contact history");
        CK(dev_realloc(&S->hz, 3 * c * sizeof(double)), "alloc contact history");
        S->cap_h = c;
    }
    k_col_keep<false><<<gb, kColBlock, 0, sm>>>(n, S->nstart, S->nbr, S->zt, S->uin, S->has, S->hcnt, S->hoff,
                                                S->hq, S->hz, S->hu);
    S->hist_np = n;
    ctx->launches += 3;
    return ibm_cuda_check(ctx, cudaGetLastError(), "contact history");
}

ibm_status col_upload(ibm_ctx *ctx, double *dst, const double *src, int on_device) {
    const size_t bytes = 3 * (size_t)ctx->n_p * sizeof(double);
    if (!src) return IBM_OK;
    CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream),
       "copy loads");
    return IBM_OK;
}

}  // namespace

void collision_free(ibm_ctx *ctx) {
    ColScratch *S = reinterpret_cast<ColScratch *>(ctx->col);
    if (!S) return;
    void *ptrs[] = {S->scene_nb, S->scene_off, S->bin_of, S->bin_cnt, S->bin_start, S->bin_cur, S->items, S->ncnt,
                    S->nstart, S->nbr, S->canon, S->zt, S->uin, S->has, S->F0, S->T0, S->F1, S->T1,
                    S->xt, S->ut, S->wt, S->xb, S->fh, S->th, S->tot, S->hoff, S->hcnt, S->hq, S->hz, S->hu};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete S;
    ctx->col = nullptr;
}

extern "C" ibm_status ibm_particle_substeps(ibm_ctx *ctx, const ibm_collision_params *prm, double dt, int n_sub,
                                           const double *F_h, const double *T_h, int on_device) {
    if (!ctx) return IBM_ERR_INVALID_ARG;
    ctx->last_error.clear();
    if (!prm) return ibm_fail(ctx, IBM_ERR_INVALID_ARG, "NULL collision parameters");
    if (!(dt > 0.0) || !std::isfinite(dt) || n_sub < 1 || n_sub > 100000)
        return ibm_fail(ctx, IBM_ERR_INVALID_ARG, "dt must be > 0 and 1 <= n_sub <= 100000");
    ColPrm P;
    double margin = 0.0;
    ibm_status st = col_params(ctx, prm, P, margin);
    if (st != IBM_OK) return st;
    if (ctx->n_p == 0) return IBM_OK;
    ColScratch *S = col_scratch(ctx);
    if (!S) return ibm_fail(ctx, IBM_ERR_OOM, "collision scratch");
    ctx->launches = 0;
    long long ne = 0;
    st = col_build(ctx, S, P, &ne);
    if (st != IBM_OK) return st;
    st = col_upload(ctx, S->fh, F_h, on_device);
    if (st == IBM_OK) st = col_upload(ctx, S->th, T_h, on_device);
    if (st != IBM_OK) return st;
    const double *Fh = F_h ? S->fh : nullptr, *Th = T_h ? S->th : nullptr;
    const int n = ctx->n_p, gb = grid_n(n);
    cudaStream_t sm = ctx->stream;
    const double ds = dt / n_sub;
    const double A[3] = {4.0 / 15.0, 1.0 / 15.0, 1.0 / 6.0};
    const double G[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
    const double Z[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};
    double *F0 = S->F0, *T0 = S->T0, *F1 = S->F1, *T1 = S->T1;
    for (int s = 0; s < n_sub; ++s) {
        for (int k = 0; k < 3; ++k) {
            if (k == 0) {
                CK(cudaMemsetAsync(F0, 0, 3 * (size_t)n * sizeof(double), sm), "zero loads");
                CK(cudaMemsetAsync(T0, 0, 3 * (size_t)n * sizeof(double), sm), "zero loads");
            }
            // predictor: loads at the stage's start state, kept in F1 for the corrector
            k_col_stage<false><<<gb, kColBlock, 0, sm>>>(
                n, P, A[k], G[k], Z[k], ds, ctx->x, ctx->up, ctx->om, ctx->d, ctx->rho, ctx->scene, ctx->dims_d,
                S->nstart, S->nbr, S->canon, S->zt, S->uin, S->has, Fh, Th, F1, T1, F0, T0, ctx->x, ctx->up,
                ctx->om, S->xt, S->ut, S->wt, ctx->err_d);
            // corrector: loads at the predicted state
            k_col_stage<true><<<gb, kColBlock, 0, sm>>>(
                n, P, A[k], G[k], Z[k], ds, S->xt, S->ut, S->wt, ctx->d, ctx->rho, ctx->scene, ctx->dims_d,
                S->nstart, S->nbr, S->canon, S->zt, S->uin, S->has, Fh, Th, nullptr, nullptr, F1, T1, ctx->x,
                ctx->up, ctx->om, nullptr, nullptr, nullptr, ctx->err_d);
            k_col_history<<<gb, kColBlock, 0, sm>>>(n, P, 2.0 * A[k] * ds, ctx->x, ctx->up, ctx->om, ctx->d,
                                                    ctx->rho, ctx->scene, ctx->dims_d, S->nstart, S->nbr, S->zt,
                                                    S->uin, S->has);
            std::swap(F0, F1);   // F_c(x^{k-1}) of this stage is F_c(x^{k-2}) of the next
            std::swap(T0, T1);
            ctx->launches += 3;
        }
    }
    k_col_margin<<<gb, kColBlock, 0, sm>>>(n, ctx->x, S->xb, ctx->scene, ctx->dims_d, ctx->cfg.h, 0.5 * margin,
                                           ctx->err_d);
    st = col_keep(ctx, S);
    if (st != IBM_OK) return st;
    ctx->have_step = false;   // the loads of the last forcing step no longer belong to this state
    st = ibm_check_err_word(ctx);
    if (st == IBM_ERR_CAPACITY)
        return ibm_fail(ctx, st, "a particle moved more than half the pair-list margin during the call: use a "
                                 "smaller dt or a larger pair_margin");
    return st;
}

extern "C" ibm_status ibm_collision_forces(ibm_ctx *ctx, const ibm_collision_params *prm, double *F_c, double *T_c,
                                          int on_device) {
    if (!ctx) return IBM_ERR_INVALID_ARG;
    ctx->last_error.clear();
    if (!prm) return ibm_fail(ctx, IBM_ERR_INVALID_ARG, "NULL collision parameters");
    ColPrm P;
    double margin = 0.0;
    ibm_status st = col_params(ctx, prm, P, margin);
    if (st != IBM_OK) return st;
    if (ctx->n_p == 0) return IBM_OK;
    ColScratch *S = col_scratch(ctx);
    if (!S) return ibm_fail(ctx, IBM_ERR_OOM, "collision scratch");
    long long ne = 0;
    st = col_build(ctx, S, P, &ne);
    if (st != IBM_OK) return st;
    const int n = ctx->n_p;
    k_col_force<<<grid_n(n), kColBlock, 0, ctx->stream>>>(n, P, ctx->x, ctx->up, ctx->om, ctx->d, ctx->rho,
                                                          ctx->scene, ctx->dims_d, S->nstart, S->nbr, S->canon, S->zt,
                                                          S->uin, S->has, S->F1, S->T1);
    CK(cudaGetLastError(), "collision forces");
    const size_t bytes = 3 * (size_t)n * sizeof(double);
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (F_c) CK(cudaMemcpyAsync(F_c, S->F1, bytes, k, ctx->stream), "copy collision force");
    if (T_c) CK(cudaMemcpyAsync(T_c, S->T1, bytes, k, ctx->stream), "copy collision torque");
    return on_device ? IBM_OK : ibm_check_err_word(ctx);
}

extern "C" ibm_status ibm_particle_state(ibm_ctx *ctx, double *x_p, double *u_p, double *omega_p, int on_device) {
    if (!ctx) return IBM_ERR_INVALID_ARG;
    const size_t bytes = 3 * (size_t)ctx->n_p * sizeof(double);
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (bytes) {
        if (x_p) CK(cudaMemcpyAsync(x_p, ctx->x, bytes, k, ctx->stream), "copy x");
        if (u_p) CK(cudaMemcpyAsync(u_p, ctx->up, bytes, k, ctx->stream), "copy u");
        if (omega_p) CK(cudaMemcpyAsync(omega_p, ctx->om, bytes, k, ctx->stream), "copy omega");
    }
    return on_device ? IBM_OK : ibm_check_err_word(ctx);
}

extern "C" ibm_status ibm_contact_history(ibm_ctx *ctx, int64_t *n_pairs, int32_t *p_out, int32_t *q_out,
                                         double *zeta_t, double *u_in) {
    if (!ctx || !n_pairs) return IBM_ERR_INVALID_ARG;
    ColScratch *S = reinterpret_cast<ColScratch *>(ctx->col);
    *n_pairs = 0;
    if (!S || S->hist_np != ctx->n_p || ctx->n_p == 0) return IBM_OK;
    const int n = ctx->n_p;
    std::vector<int> off(n + 1), cnt(n);
    CK(cudaMemcpyAsync(off.data(), S->hoff, (n + 1) * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "read");
    CK(cudaMemcpyAsync(cnt.data(), S->hcnt, n * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "read");
    CK(cudaStreamSynchronize(ctx->stream), "read");
    const long long nh = off[n];
    *n_pairs = nh;
    if (!p_out && !q_out && !zeta_t && !u_in) return IBM_OK;
    std::vector<int> q(std::max(nh, 1ll));
    std::vector<double> z(3 * std::max(nh, 1ll)), u(std::max(nh, 1ll));
    if (nh) {
        CK(cudaMemcpyAsync(q.data(), S->hq, nh * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "read");
        CK(cudaMemcpyAsync(z.data(), S->hz, 3 * nh * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "read");
        CK(cudaMemcpyAsync(u.data(), S->hu, nh * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "read");
        CK(cudaStreamSynchronize(ctx->stream), "read");
    }
    for (int p = 0; p < n; ++p)
        for (int k = off[p]; k < off[p] + cnt[p]; ++k) {
            if (p_out) p_out[k] = p;
            if (q_out) q_out[k] = q[k];
            if (u_in) u_in[k] = u[k];
            if (zeta_t)
                for (int c = 0; c < 3; ++c) zeta_t[3 * k + c] = z[3 * k + c];
        }
    return IBM_OK;
}
