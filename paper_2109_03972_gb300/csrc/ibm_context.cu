// C ABI: context lifetime, argument validation, particle upload and the
// dispatch of a forcing step to the plain or the cluster path.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "ibm_internal.h"

// Allocation-failure injection (ibm_debug_fail_allocation): the n-th device
// allocation after the call fails as if the device were out of memory.
static std::atomic<long long> g_fail_countdown{0};

cudaError_t ibm_dev_malloc(void **p, size_t bytes) {
    long long c = g_fail_countdown.load();
    while (c > 0) {
        if (g_fail_countdown.compare_exchange_weak(c, c - 1)) {
            if (c == 1) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMalloc(p, bytes);
}

ibm_status ibm_fail(ibm_ctx *ctx, ibm_status s, const std::string &msg) {
    if (ctx) ctx->last_error = msg;
    return s;
}

ibm_status ibm_cuda_check(ibm_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return IBM_OK;
    cudaGetLastError();
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return ibm_fail(ctx, e == cudaErrorMemoryAllocation ? IBM_ERR_OOM : IBM_ERR_CUDA, m);
}

#define CK(call, what)                                                  \
    do {                                                                \
        ibm_status _s = ibm_cuda_check(ctx, (call), what);              \
        if (_s != IBM_OK) return _s;                                    \
    } while (0)

ibm_status ibm_check_err_word(ibm_ctx *ctx) {
    CK(cudaMemcpyAsync(ctx->err_h, ctx->err_d, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
       "read error word");
    CK(cudaStreamSynchronize(ctx->stream), "synchronise");
    int e = *ctx->err_h;
    if (!e) return IBM_OK;
    CK(cudaMemsetAsync(ctx->err_d, 0, sizeof(int), ctx->stream), "clear error word");
    if (e & IBM_EBIT_NONFINITE) return ibm_fail(ctx, IBM_ERR_NONFINITE, "non-finite particle state");
    if (e & IBM_EBIT_SCENE) return ibm_fail(ctx, IBM_ERR_INVALID_ARG, "scene index out of range");
    if (e & IBM_EBIT_DIAMETER)
        return ibm_fail(ctx, IBM_ERR_INVALID_ARG,
                        "particle diameter must be > 0 and d/h + 4 <= smallest grid edge");
    if (e & IBM_EBIT_DENSITY)
        return ibm_fail(ctx, IBM_ERR_INVALID_ARG,
                        "rho_p == rho_f: the rigid-body Newton-Euler form is singular");
    if (e & IBM_EBIT_TIMEOUT) return ibm_fail(ctx, IBM_ERR_TIMEOUT, "a device-side wait timed out");
    if (e & IBM_EBIT_MASS)
        return ibm_fail(ctx, IBM_ERR_INVALID_ARG,
                        "particle sub-steps need positive densities (rho_p given to ibm_set_particles)");
    if (e & IBM_EBIT_OVERFLOW) return ibm_fail(ctx, IBM_ERR_CAPACITY, "internal scratch capacity exceeded");
    if (e & IBM_EBIT_FIXEDPOINT)
        return ibm_fail(ctx, IBM_ERR_CAPACITY,
                        "deterministic spreading left its fixed-point range (particles overlap far more than "
                        "the range allows); the velocity field of this step is not valid");
    return ibm_fail(ctx, IBM_ERR_CUDA, "internal device error");
}

template <typename T>
static ibm_status dev_alloc(ibm_ctx *ctx, T **p, size_t n) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    if (n == 0) n = 1;
    return ibm_cuda_check(ctx, ibm_malloc((void **)p, n * sizeof(T)), "cudaMalloc");
}

static const int kProfPairs = 512;

static void prof_fold(ibm_ctx *ctx) {
    // read the recorded pairs (synchronises on the last event)
    if (ctx->prof_n == 0) return;
    cudaEventSynchronize(ctx->prof_ev[2 * (ctx->prof_n - 1) + 1]);
    for (int i = 0; i < ctx->prof_n; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->prof_ev[2 * i], ctx->prof_ev[2 * i + 1]) == cudaSuccess) {
            ctx->prof_ms += ms;
            ctx->prof_count += 1;
        }
    }
    ctx->prof_n = 0;
}

void prof_begin(ibm_ctx *ctx) {
    if (!ctx->cfg.profile || ctx->prof_ev.empty() || ctx->capturing) return;
    if (ctx->prof_n == kProfPairs) prof_fold(ctx);
    cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n], ctx->stream);
}

void prof_end(ibm_ctx *ctx) {
    if (!ctx->cfg.profile || ctx->prof_ev.empty() || ctx->capturing) return;
    cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n + 1], ctx->stream);
    ctx->prof_n += 1;
}

static void free_all(ibm_ctx *ctx) {
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    ctx->graph_exec = nullptr;
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    ctx->cap_stream = nullptr;
    for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
    ctx->prof_ev.clear();
    void *ptrs[] = {ctx->dims_d, ctx->x, ctx->up, ctx->om, ctx->d, ctx->rho, ctx->scene,
                    ctx->nl, ctx->moff, ctx->toff, ctx->pinfo, ctx->tmpl64, ctx->tmpl32,
                    ctx->tmpl_of_nl, ctx->FD, ctx->TD, ctx->Fout, ctx->Tout, ctx->x_new,
                    ctx->u_new, ctx->om_new, ctx->slip_acc, ctx->ebuf, ctx->e_hist, ctx->cbuf, ctx->fb_cm, ctx->fb_bits,
                    ctx->cell_off_d, ctx->fb_own, ctx->mf_seg, ctx->mf_cells, ctx->mf_part, ctx->mf_out, ctx->mf_ptr,
                    ctx->in_ptr, ctx->in_buf, ctx->uptr_d, ctx->fptr_d,
                    ctx->gu_hist, ctx->gmk, ctx->err_d};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (void *p : ctx->u0_saved)
        if (p) cudaFree(p);
    for (void *p : ctx->bw_work)
        if (p) cudaFree(p);
    cluster_free(ctx);
    contact_free(ctx);
    collision_free(ctx);
    if (ctx->err_h) cudaFreeHost(ctx->err_h);
}

extern "C" {

const char *ibm_status_string(ibm_status s) {
    switch (s) {
        case IBM_OK: return "IBM_OK";
        case IBM_ERR_INVALID_ARG: return "IBM_ERR_INVALID_ARG";
        case IBM_ERR_CUDA: return "IBM_ERR_CUDA";
        case IBM_ERR_OOM: return "IBM_ERR_OOM";
        case IBM_ERR_CAPACITY: return "IBM_ERR_CAPACITY";
        case IBM_ERR_NONFINITE: return "IBM_ERR_NONFINITE";
        case IBM_ERR_TIMEOUT: return "IBM_ERR_TIMEOUT";
        case IBM_ERR_STATE: return "IBM_ERR_STATE";
        case IBM_ERR_NOCONVERGE: return "IBM_ERR_NOCONVERGE";
    }
    return "IBM_ERR_UNKNOWN";
}

const char *ibm_last_error(const ibm_ctx *ctx) {
    if (!ctx) return "";
    return ctx->last_error.c_str();
}

ibm_status ibm_create(const ibm_config *cfg, void *cuda_stream, ibm_ctx **out) {
    if (!out) return IBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfg || cfg->n_scenes < 1 || !cfg->dims) return IBM_ERR_INVALID_ARG;
    if (!(cfg->h > 0.0) || !std::isfinite(cfg->h)) return IBM_ERR_INVALID_ARG;
    // four-point kernel (Sec. 2.2.3): plain path, forward only
    if (cfg->kernel_width != 3 && cfg->kernel_width != 4) return IBM_ERR_INVALID_ARG;
    if (cfg->kernel_width == 4 && (cfg->spread_mode != IBM_SPREAD_PLAIN || cfg->requires_grad))
        return IBM_ERR_INVALID_ARG;
    if (cfg->n_forcing < 1 || cfg->n_forcing > 64) return IBM_ERR_INVALID_ARG;
    if (cfg->precision != IBM_FP32 && cfg->precision != IBM_FP64) return IBM_ERR_INVALID_ARG;
    if (cfg->spread_mode < 0 || cfg->spread_mode > 2) return IBM_ERR_INVALID_ARG;
    if (cfg->precision == IBM_FP64 && cfg->spread_mode != IBM_SPREAD_PLAIN) return IBM_ERR_INVALID_ARG;
    if (cfg->max_particles < 1) return IBM_ERR_INVALID_ARG;
    if (cfg->newton_euler && (!(cfg->rho_f > 0.0) || !std::isfinite(cfg->g[0]) ||
                              !std::isfinite(cfg->g[1]) || !std::isfinite(cfg->g[2])))
        return IBM_ERR_INVALID_ARG;
    if (cfg->threads_per_block != 0 && cfg->threads_per_block != -1 && cfg->threads_per_block != 512 &&
        cfg->threads_per_block != 1024)
        return IBM_ERR_INVALID_ARG;
    int min_edge = 1 << 30;
    for (int s = 0; s < cfg->n_scenes; ++s)
        for (int c = 0; c < 3; ++c) {
            int32_t n = cfg->dims[3 * s + c];
            if (n < 8 || n > (1 << 20)) return IBM_ERR_INVALID_ARG;
            min_edge = std::min(min_edge, (int)n);
        }
    ibm_ctx *ctx = new (std::nothrow) ibm_ctx();
    if (!ctx) return IBM_ERR_OOM;
    ctx->cfg = *cfg;
    ctx->dims_h.assign(cfg->dims, cfg->dims + 3 * cfg->n_scenes);
    ctx->cfg.dims = ctx->dims_h.data();
    ctx->min_edge = min_edge;
    ctx->stream = (cudaStream_t)cuda_stream;
    ibm_status s = IBM_OK;
    if ((s = dev_alloc(ctx, &ctx->dims_d, ctx->dims_h.size())) != IBM_OK ||
        (s = ibm_cuda_check(ctx, cudaMemcpy(ctx->dims_d, ctx->dims_h.data(),
                                            ctx->dims_h.size() * sizeof(int32_t),
                                            cudaMemcpyHostToDevice), "copy dims")) != IBM_OK ||
        (s = dev_alloc(ctx, &ctx->err_d, 1)) != IBM_OK ||
        (s = dev_alloc(ctx, &ctx->slip_acc, 2)) != IBM_OK ||
        (s = ibm_cuda_check(ctx, cudaMallocHost((void **)&ctx->err_h, sizeof(int)), "cudaMallocHost")) != IBM_OK ||
        (s = ibm_cuda_check(ctx, cudaMemset(ctx->err_d, 0, sizeof(int)), "memset")) != IBM_OK) {
        free_all(ctx);
        delete ctx;
        return s;
    }
    const int cp = cfg->max_particles;
    if ((s = dev_alloc(ctx, &ctx->x, 3 * (size_t)cp)) != IBM_OK ||
        (s = dev_alloc(ctx, &ctx->up, 3 * (size_t)cp)) != IBM_OK ||
        (s = dev_alloc(ctx, &ctx->om, 3 * (size_t)cp)) != IBM_OK ||
        (s = dev_alloc(ctx, &ctx->d, (size_t)cp)) != IBM_OK ||
        (s = dev_alloc(ctx, &ctx->rho, (size_t)cp)) != IBM_OK ||
        (s = dev_alloc(ctx, &ctx->scene, (size_t)cp)) != IBM_OK ||
        (s = dev_alloc(ctx, &ctx->nl, (size_t)cp)) != IBM_OK ||
        (s = dev_alloc(ctx, &ctx->moff, (size_t)cp + 1)) != IBM_OK ||
        (s = dev_alloc(ctx, &ctx->toff, (size_t)cp)) != IBM_OK ||
        (s = dev_alloc(ctx, &ctx->pinfo, (size_t)cp)) != IBM_OK ||
        (s = dev_alloc(ctx, &ctx->FD, 3 * (size_t)cp)) != IBM_OK ||
        (s = dev_alloc(ctx, &ctx->TD, 3 * (size_t)cp)) != IBM_OK ||
        (s = dev_alloc(ctx, &ctx->Fout, 3 * (size_t)cp)) != IBM_OK ||
        (s = dev_alloc(ctx, &ctx->Tout, 3 * (size_t)cp)) != IBM_OK ||
        (s = dev_alloc(ctx, &ctx->x_new, 3 * (size_t)cp)) != IBM_OK ||
        (s = dev_alloc(ctx, &ctx->u_new, 3 * (size_t)cp)) != IBM_OK ||
        (s = dev_alloc(ctx, &ctx->om_new, 3 * (size_t)cp)) != IBM_OK) {
        free_all(ctx);
        delete ctx;
        return s;
    }
    ctx->cap_p = cp;
    if (cfg->profile) {
        ctx->prof_ev.resize(2 * kProfPairs);
        for (auto &e : ctx->prof_ev) {
            if ((s = ibm_cuda_check(ctx, cudaEventCreate(&e), "cudaEventCreate")) != IBM_OK) {
                free_all(ctx);
                delete ctx;
                return s;
            }
        }
    }
    *out = ctx;
    return IBM_OK;
}

ibm_status ibm_destroy(ibm_ctx *ctx) {
    if (!ctx) return IBM_OK;
    cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
    delete ctx;
    return IBM_OK;
}

ibm_status ibm_set_particles(ibm_ctx *ctx, int n_p, const double *x_p, const double *u_p,
                             const double *omega_p, const double *d_p, const double *rho_p,
                             const int32_t *scene_of, int on_device) {
    if (!ctx) return IBM_ERR_INVALID_ARG;
    ctx->last_error.clear();
    if (n_p < 0) return ibm_fail(ctx, IBM_ERR_INVALID_ARG, "n_p < 0");
    if (n_p > ctx->cap_p) return ibm_fail(ctx, IBM_ERR_CAPACITY, "n_p exceeds max_particles");
    if (n_p > 0 && (!x_p || !u_p || !omega_p || !d_p))
        return ibm_fail(ctx, IBM_ERR_INVALID_ARG, "NULL particle array");
    if (n_p > 0 && ctx->cfg.newton_euler && !rho_p)
        return ibm_fail(ctx, IBM_ERR_INVALID_ARG, "rho_p is required with newton_euler");
    if (n_p > 0 && ctx->cfg.n_scenes > 1 && !scene_of)
        return ibm_fail(ctx, IBM_ERR_INVALID_ARG, "scene_of is required with n_scenes > 1");
    ctx->have_step = false;
    ctx->have_forward = false;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t v3 = 3 * (size_t)n_p * sizeof(double), v1 = (size_t)n_p * sizeof(double);
    ctx->n_p = n_p;
    if (n_p > 0) {
        CK(cudaMemcpyAsync(ctx->x, x_p, v3, k, ctx->stream), "copy x_p");
        CK(cudaMemcpyAsync(ctx->up, u_p, v3, k, ctx->stream), "copy u_p");
        CK(cudaMemcpyAsync(ctx->om, omega_p, v3, k, ctx->stream), "copy omega_p");
        CK(cudaMemcpyAsync(ctx->d, d_p, v1, k, ctx->stream), "copy d_p");
        if (rho_p) CK(cudaMemcpyAsync(ctx->rho, rho_p, v1, k, ctx->stream), "copy rho_p");
        else CK(cudaMemsetAsync(ctx->rho, 0, v1, ctx->stream), "zero rho");
        if (scene_of)
            CK(cudaMemcpyAsync(ctx->scene, scene_of, (size_t)n_p * sizeof(int32_t), k, ctx->stream),
               "copy scene_of");
        else CK(cudaMemsetAsync(ctx->scene, 0, (size_t)n_p * sizeof(int32_t), ctx->stream), "zero scene");
    }
    ibm_status s = launch_setup_particles(ctx);   // validation + marker counts + offsets
    if (s != IBM_OK) {
        ctx->n_p = 0;   // no step may run on a half-prepared particle set
        return s;
    }
    s = ibm_check_err_word(ctx);
    if (s != IBM_OK) {
        ctx->n_p = 0;
        return s;
    }
    return IBM_OK;
}

// One forcing step without the slip diagnostic: Sec. 2.2.2 loop, loads, and
// the Newton-Euler update.  Stream operations only (capturable into a graph
// once the buffers exist).
static ibm_status forcing_body(ibm_ctx *ctx, void *const *u_ptrs, double tau, void *const *f_out) {
    ctx->have_step = false;
    ctx->last_tau = tau;
    ctx->launches = 0;
    const size_t esz = ctx->cfg.precision == IBM_FP64 ? sizeof(double) : sizeof(float);
    if (ctx->cfg.requires_grad) {
        // keep u^0 for the backward pass
        ctx->u0_saved.resize(ctx->cfg.n_scenes, nullptr);
        for (int s = 0; s < ctx->cfg.n_scenes; ++s) {
            const size_t n = 3ull * ctx->dims_h[3 * s] * ctx->dims_h[3 * s + 1] * ctx->dims_h[3 * s + 2];
            if (!ctx->u0_saved[s]) CK(ibm_malloc(&ctx->u0_saved[s], n * esz), "alloc u0 copy");
            CK(cudaMemcpyAsync(ctx->u0_saved[s], u_ptrs[s], n * esz, cudaMemcpyDeviceToDevice, ctx->stream),
               "save u0");
        }
    }
    CK(cudaMemsetAsync(ctx->FD, 0, 3 * (size_t)std::max(ctx->n_p, 1) * sizeof(double), ctx->stream), "zero FD");
    CK(cudaMemsetAsync(ctx->TD, 0, 3 * (size_t)std::max(ctx->n_p, 1) * sizeof(double), ctx->stream), "zero TD");
    if (f_out)
        for (int s = 0; s < ctx->cfg.n_scenes; ++s) {
            const size_t n = 3ull * ctx->dims_h[3 * s] * ctx->dims_h[3 * s + 1] * ctx->dims_h[3 * s + 2];
            CK(cudaMemsetAsync(f_out[s], 0, n * esz, ctx->stream), "zero f_out");
        }
    ibm_status st = IBM_OK;
    if (ctx->n_p > 0) {
        st = launch_pinfo(ctx);
        if (st != IBM_OK) return st;
        if (ctx->cfg.spread_mode == IBM_SPREAD_PLAIN)
            st = plain_forcing_step(ctx, u_ptrs, tau, f_out);
        else
            st = cluster_forcing_step(ctx, u_ptrs, tau, f_out);
        if (st != IBM_OK) return st;
    }
    st = finalize_particles(ctx, tau);
    if (st != IBM_OK) return st;
    ctx->have_step = true;
    ctx->have_forward = ctx->cfg.requires_grad != 0;
    return IBM_OK;
}

// Key of a captured step: everything whose change would make a replay of the
// graph wrong (kernel arguments, launch shapes, buffers).
static void graph_key(const ibm_ctx *ctx, void *const *u_ptrs, double tau, void *const *f_out,
                      std::vector<uintptr_t> &key) {
    key.clear();
    for (int s = 0; s < ctx->cfg.n_scenes; ++s) {
        key.push_back((uintptr_t)u_ptrs[s]);
        key.push_back(f_out ? (uintptr_t)f_out[s] : 0);
    }
    uint64_t tb;
    memcpy(&tb, &tau, sizeof(tb));
    key.push_back((uintptr_t)tb);
    const void *bufs[] = {ctx->dims_d, ctx->x, ctx->up, ctx->om, ctx->d, ctx->rho, ctx->scene, ctx->nl, ctx->moff,
                          ctx->toff, ctx->pinfo, ctx->tmpl64, ctx->tmpl32, ctx->tmpl_of_nl, ctx->FD, ctx->TD,
                          ctx->Fout, ctx->Tout, ctx->x_new, ctx->u_new, ctx->om_new, ctx->ebuf, ctx->cbuf,
                          ctx->uptr_d, ctx->fptr_d, ctx->err_d, ctx->fb_cm, ctx->fb_bits, ctx->cell_off_d,
                          ctx->fb_own};
    for (const void *b : bufs) key.push_back((uintptr_t)b);
    const long long sizes[] = {ctx->n_p, ctx->n_markers, ctx->max_nl, ctx->cap_p, ctx->tmpl_used, ctx->tuned_tpb,
                               ctx->wait_limit};
    for (long long v : sizes) key.push_back((uintptr_t)v);
    if (ctx->cfg.spread_mode != IBM_SPREAD_PLAIN) cluster_graph_key(ctx, key);
    contact_graph_key(ctx, key);
}

// Forcing step replayed from a CUDA graph: eager while the key is new, captured
// on the next call with the same key, replayed while the key holds.
static ibm_status graph_step(ibm_ctx *ctx, void *const *u_ptrs, double tau, void *const *f_out) {
    std::vector<uintptr_t> key;
    graph_key(ctx, u_ptrs, tau, f_out, key);
    if (ctx->graph_exec && key == ctx->graph_key) {
        CK(cudaGraphLaunch(ctx->graph_exec, ctx->stream), "graph launch");
        ctx->launches = ctx->graph_launches;
        ctx->have_step = true;
        ctx->have_forward = false;
        ctx->last_tau = tau;
        return IBM_OK;
    }
    if (key != ctx->warm_key) {
        const ibm_status st = forcing_body(ctx, u_ptrs, tau, f_out);
        if (st != IBM_OK) return st;
        graph_key(ctx, u_ptrs, tau, f_out, ctx->warm_key);   // after any allocation the step made
        return ibm_cuda_check(ctx, cudaGetLastError(), "kernel launch");
    }
    // capture on a stream of our own (the legacy default stream cannot be
    // captured); the graph is launched on the context's stream
    if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking), "capture stream");
    cudaGraph_t g = nullptr;
    const cudaStream_t user = ctx->stream;
    CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    ctx->stream = ctx->cap_stream;
    ctx->capturing = true;
    const ibm_status st = forcing_body(ctx, u_ptrs, tau, f_out);
    ctx->capturing = false;
    ctx->stream = user;
    const cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &g);
    if (st != IBM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (ce != cudaSuccess) return ibm_cuda_check(ctx, ce, "end capture");
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    ctx->graph_exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        ctx->graph_exec = nullptr;
        return ibm_cuda_check(ctx, ie, "graph instantiate");
    }
    ctx->graph_key = key;
    ctx->graph_launches = ctx->launches;
    CK(cudaGraphLaunch(ctx->graph_exec, ctx->stream), "graph launch");
    return IBM_OK;
}

ibm_status ibm_forcing_step(ibm_ctx *ctx, void *const *u_ptrs, double tau, void *const *f_out,
                            double *slip_out) {
    if (!ctx) return IBM_ERR_INVALID_ARG;
    ctx->last_error.clear();
    if (!u_ptrs) return ibm_fail(ctx, IBM_ERR_INVALID_ARG, "u_ptrs is NULL");
    for (int s = 0; s < ctx->cfg.n_scenes; ++s)
        if (!u_ptrs[s]) return ibm_fail(ctx, IBM_ERR_INVALID_ARG, "NULL velocity field");
    if (f_out)
        for (int s = 0; s < ctx->cfg.n_scenes; ++s)
            if (!f_out[s]) return ibm_fail(ctx, IBM_ERR_INVALID_ARG, "NULL f_out field");
    if (!(tau > 0.0) || !std::isfinite(tau)) return ibm_fail(ctx, IBM_ERR_INVALID_ARG, "tau must be > 0");
    if (ctx->cfg.use_graph && !slip_out && !ctx->cfg.requires_grad && ctx->n_p > 0 &&
        (ctx->cfg.threads_per_block >= 0 || ctx->cfg.spread_mode == IBM_SPREAD_PLAIN || ctx->tune_step >= 4))
        return graph_step(ctx, u_ptrs, tau, f_out);
    ibm_status st = forcing_body(ctx, u_ptrs, tau, f_out);
    if (st != IBM_OK) return st;
    if (slip_out) {
        CK(cudaMemsetAsync(ctx->slip_acc, 0, 2 * sizeof(double), ctx->stream), "zero slip");
        if (ctx->n_p > 0) {
            st = plain_slip(ctx, u_ptrs);
            if (st != IBM_OK) return st;
        }
        double acc[2];
        CK(cudaMemcpyAsync(acc, ctx->slip_acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
           "read slip");
        st = ibm_check_err_word(ctx);
        if (st != IBM_OK) return st;
        slip_out[0] = ctx->n_markers ? std::sqrt(acc[0] / (double)ctx->n_markers) : 0.0;
        slip_out[1] = acc[1];
    } else {
        CK(cudaGetLastError(), "kernel launch");
    }
    return IBM_OK;
}

ibm_status ibm_particle_loads(ibm_ctx *ctx, double *F, double *T, double *x_p, double *u_p,
                              double *omega_p, int on_device) {
    if (!ctx) return IBM_ERR_INVALID_ARG;
    if (!ctx->have_step) return ibm_fail(ctx, IBM_ERR_STATE, "no forcing step since the last set_particles");
    const size_t v3 = 3 * (size_t)ctx->n_p * sizeof(double);
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (v3) {
        if (F) CK(cudaMemcpyAsync(F, ctx->Fout, v3, k, ctx->stream), "copy F");
        if (T) CK(cudaMemcpyAsync(T, ctx->Tout, v3, k, ctx->stream), "copy T");
        if (x_p) CK(cudaMemcpyAsync(x_p, ctx->x_new, v3, k, ctx->stream), "copy x");
        if (u_p) CK(cudaMemcpyAsync(u_p, ctx->u_new, v3, k, ctx->stream), "copy u");
        if (omega_p) CK(cudaMemcpyAsync(omega_p, ctx->om_new, v3, k, ctx->stream), "copy omega");
    }
    if (!on_device) return ibm_check_err_word(ctx);
    return IBM_OK;
}

ibm_status ibm_backward(ibm_ctx *ctx, void *const *grad_u_out, void *const *grad_u_in, double *gU,
                        double *gOmega, double *gX) {
    if (!ctx) return IBM_ERR_INVALID_ARG;
    ctx->last_error.clear();
    if (!ctx->cfg.requires_grad) return ibm_fail(ctx, IBM_ERR_STATE, "context created without requires_grad");
    if (!ctx->have_forward) return ibm_fail(ctx, IBM_ERR_STATE, "no forcing step to differentiate");
    if (!grad_u_out || !grad_u_in) return ibm_fail(ctx, IBM_ERR_INVALID_ARG, "NULL gradient field array");
    for (int s = 0; s < ctx->cfg.n_scenes; ++s)
        if (!grad_u_out[s] || !grad_u_in[s]) return ibm_fail(ctx, IBM_ERR_INVALID_ARG, "NULL gradient field");
    return plain_backward(ctx, grad_u_out, grad_u_in, gU, gOmega, gX);
}

ibm_status ibm_marker_bases(ibm_ctx *ctx, int64_t *base_out, int64_t *n_markers) {
    if (!ctx || !n_markers) return IBM_ERR_INVALID_ARG;
    *n_markers = ctx->n_markers;
    if (!base_out || ctx->n_markers == 0) return IBM_OK;
    int64_t *dev = nullptr;
    CK(ibm_malloc(&dev, 3 * (size_t)ctx->n_markers * sizeof(int64_t)), "alloc bases");
    ibm_status s = launch_pinfo(ctx);
    if (s == IBM_OK) s = launch_marker_bases(ctx, dev);
    if (s == IBM_OK)
        s = ibm_cuda_check(ctx, cudaMemcpyAsync(base_out, dev, 3 * (size_t)ctx->n_markers * sizeof(int64_t),
                                                cudaMemcpyDeviceToHost, ctx->stream), "copy bases");
    if (s == IBM_OK) s = ibm_check_err_word(ctx);
    cudaFree(dev);
    return s;
}

ibm_status ibm_kernel_timing(ibm_ctx *ctx, double *total_ms, int64_t *count, int reset) {
    if (!ctx) return IBM_ERR_INVALID_ARG;
    if (!ctx->cfg.profile) return ibm_fail(ctx, IBM_ERR_STATE, "context created without profile");
    prof_fold(ctx);
    if (total_ms) *total_ms = ctx->prof_ms;
    if (count) *count = ctx->prof_count;
    if (reset) {
        ctx->prof_ms = 0.0;
        ctx->prof_count = 0;
    }
    return IBM_OK;
}

ibm_status ibm_step_stats(ibm_ctx *ctx, int64_t *stats) {
    if (!ctx || !stats) return IBM_ERR_INVALID_ARG;
    ibm_status s = ibm_check_err_word(ctx);
    for (int i = 0; i < 12; ++i) stats[i] = 0;
    stats[0] = ctx->n_markers;
    stats[6] = ctx->launches;
    if (s == IBM_OK && ctx->cfg.spread_mode != IBM_SPREAD_PLAIN) s = cluster_stats(ctx, stats);
    return s;
}

ibm_status ibm_particle_clusters(ibm_ctx *ctx, int32_t *cluster_of, int32_t *path_of, int64_t *n_clusters) {
    if (!ctx) return IBM_ERR_INVALID_ARG;
    if (ctx->cfg.spread_mode == IBM_SPREAD_PLAIN)
        return ibm_fail(ctx, IBM_ERR_STATE, "PLAIN mode forms no clusters");
    if (!ctx->have_step) return ibm_fail(ctx, IBM_ERR_STATE, "no forcing step since the last set_particles");
    ibm_status s = ibm_check_err_word(ctx);
    if (s != IBM_OK) return s;
    return cluster_membership(ctx, cluster_of, path_of, n_clusters);
}

ibm_status ibm_set_wait_limit(ibm_ctx *ctx, int64_t iterations) {
    if (!ctx) return IBM_ERR_INVALID_ARG;
    if (iterations < 0 || iterations > INT32_MAX) return ibm_fail(ctx, IBM_ERR_INVALID_ARG, "wait limit out of range");
    ctx->wait_limit = (int)iterations;
    return IBM_OK;
}

ibm_status ibm_debug_fail_allocation(int64_t n) {
    if (n < 0) return IBM_ERR_INVALID_ARG;
    g_fail_countdown.store(n);
    return IBM_OK;
}

}  // extern "C"
