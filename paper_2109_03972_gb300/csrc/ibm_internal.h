// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ibm.h"

// Error bits set by kernels in ctx->err_d (never a trap).
enum : int {
    IBM_EBIT_NONFINITE = 1,
    IBM_EBIT_DIAMETER = 2,
    IBM_EBIT_SCENE = 4,
    IBM_EBIT_DENSITY = 8,
    IBM_EBIT_TIMEOUT = 16,
    IBM_EBIT_OVERFLOW = 32,   // a scratch capacity was exceeded (work skipped)
    IBM_EBIT_INTERNAL = 64,
    IBM_EBIT_FIXEDPOINT = 128,  // a deterministic-mode cell left its fixed-point range
    IBM_EBIT_MASS = 256,        // a particle without positive mass (rho_p) in the particle sub-steps
};

// Per-particle record derived from the FP64 state at every step (device).
struct PInfo {
    double xi[3];     // x_p / h  (grid units)
    double a;         // (d_p / 2) / h
    float  fracf[3];  // xi - floor(xi), float
    float  af;        // a as float
    float  ud[3];     // u_p (float)
    float  om[3];     // omega_p in grid units per time (omega * h / h = omega)
    int    base[3];   // floor(xi)
    int    nl;        // markers
    int    moff;      // first global marker index
    int    toff;      // template offset (entries)
    int    scene;
    float  D;         // dV_l / h^3
    float  rphys;     // (d_p / 2) (physical arm length)
    double D64;       // dV_l / h^3 (FP64)
    double rphys64;   // d_p / 2 (FP64)
};

struct SceneDesc {
    int n[3];
    long long off;    // unused (fields are separate pointers)
};

struct ibm_ctx {
    ibm_config cfg;
    // CUDA-graph replay of the forcing step (cfg.use_graph): the graph is
    // captured from the call after an eager one with the same key (field
    // pointers, tau, sizes and every device buffer the step touches)
    bool capturing = false;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t cap_stream = nullptr;   // capture stream (the caller's may be the legacy stream)
    std::vector<uintptr_t> graph_key, warm_key;
    int graph_launches = 0;
    // autotune of the cluster kernel variant (cfg.threads_per_block < 0):
    // step 0 warms up, steps 1 and 2 time the two variants, then the faster stays
    int tune_step = 0, tuned_tpb = 0;
    float tune_ms[2] = {0.f, 0.f};
    std::vector<int32_t> dims_h;   // [n_scenes][3]
    int32_t *dims_d = nullptr;
    int min_edge = 0;
    cudaStream_t stream = nullptr;

    int n_p = 0;
    int cap_p = 0;
    // particle state (device, FP64)
    double *x = nullptr, *up = nullptr, *om = nullptr, *d = nullptr, *rho = nullptr;
    int32_t *scene = nullptr;
    int *nl = nullptr, *moff = nullptr, *toff = nullptr;
    PInfo *pinfo = nullptr;
    long long n_markers = 0;
    int max_nl = 0;

    // marker templates (unit directions), indexed by toff
    double *tmpl64 = nullptr;
    float *tmpl32 = nullptr;
    long long tmpl_cap = 0, tmpl_used = 0;
    int *tmpl_of_nl = nullptr;     // device [nl_cap], -1 = not generated
    int nl_cap = 0;
    std::vector<int> tmpl_of_nl_h; // host mirror

    // loads / state outputs (device FP64)
    double *FD = nullptr, *TD = nullptr;     // sum e*D, sum r x e*D (per particle)
    double *cbuf = nullptr;                  // plain path: per-(particle, chunk) load sums
    size_t cbuf_cap = 0;
    // deterministic fallback: per-cluster maxima, grid-wide cell bitmap, scene cell offsets
    unsigned *fb_cm = nullptr, *fb_bits = nullptr;
    int fb_cm_cap = 0;
    long long *cell_off_d = nullptr;
    unsigned *fb_own = nullptr;      // deterministic fallback: owned stencil cells per marker
    long long fb_own_cap = 0;
    double *Fout = nullptr, *Tout = nullptr; // F_p, T_p in physical units
    double *x_new = nullptr, *u_new = nullptr, *om_new = nullptr;
    double *slip_acc = nullptr;              // [2]
    // mean force (ibm_meanforce.cu): segment table, cells per scene, partials, result, field pointers
    long long *mf_seg = nullptr, *mf_cells = nullptr;
    double *mf_part = nullptr, *mf_out = nullptr;
    void **mf_ptr = nullptr;
    long long mf_nseg = 0;
    std::vector<void *> mf_ptr_h;
    // fluid inertia inside the particles (ibm_inertia.cu): field pointer table, [cap_p][7] sums
    void **in_ptr = nullptr;
    std::vector<void *> in_ptr_h;
    double *in_buf = nullptr;
    int in_cap = 0;

    // plain-path scratch
    void *ebuf = nullptr;     // [markers][3] real
    long long ebuf_cap = 0;
    void **uptr_d = nullptr;  // device copy of the scene field pointers
    void **fptr_d = nullptr;
    std::vector<void *> uptr_h, fptr_h;
    int launches = 0;         // kernel launches of the last step

    // cluster-path scratch (see ibm_cluster.cu)
    void *cl = nullptr;

    // collision models and particle sub-steps (ibm_collision.cu)
    void *col = nullptr;

    // marker exclusion near contact (ibm_contact.cu, Sec. 2.2.5)
    void *ct = nullptr;
    int ct_enable = 0;
    double ct_eps = 0.0;
    uint64_t ct_seed = 0;

    // backward
    std::vector<void *> u0_saved;            // per scene copy of u^0
    std::vector<void *> bw_work;             // per scene work field
    void *e_hist = nullptr, *gu_hist = nullptr, *gmk = nullptr;
    long long hist_cap = 0;
    bool have_forward = false;
    double last_tau = 0.0;

    // profiling: event pairs around the main kernel of each step
    std::vector<cudaEvent_t> prof_ev;
    int prof_n = 0;           // recorded pairs since reset
    double prof_ms = 0.0;     // folded-in time of pairs already read
    long long prof_count = 0;

    // bound of the device-side retry loops (lock-free union-find of the
    // clustering); ibm_set_wait_limit, 0 = the default
    int wait_limit = 0;

    int *err_d = nullptr;
    int *err_h = nullptr;     // pinned
    bool have_step = false;
    int64_t stats[8] = {0};
    std::string last_error;
};

// Device allocations of the library all go through ibm_malloc, so that a test
// can make one of them fail on the host (ibm_debug_fail_allocation).
cudaError_t ibm_dev_malloc(void **p, size_t bytes);
template <typename T>
inline cudaError_t ibm_malloc(T **p, size_t bytes) {
    return ibm_dev_malloc(reinterpret_cast<void **>(p), bytes);
}

// helpers (ibm_context.cu)
ibm_status ibm_fail(ibm_ctx *ctx, ibm_status s, const std::string &msg);
ibm_status ibm_cuda_check(ibm_ctx *ctx, cudaError_t e, const char *what);
ibm_status ibm_check_err_word(ibm_ctx *ctx);   // synchronises

// plain path (ibm_plain.cu)
ibm_status plain_forcing_step(ibm_ctx *ctx, void *const *u_ptrs, double tau, void *const *f_out);
ibm_status plain_slip(ibm_ctx *ctx, void *const *u_ptrs);
ibm_status finalize_particles(ibm_ctx *ctx, double tau);
ibm_status plain_backward(ibm_ctx *ctx, void *const *grad_u_out, void *const *grad_u_in,
                          double *gU, double *gOmega, double *gX);
ibm_status launch_setup_particles(ibm_ctx *ctx);      // nl, validation
ibm_status launch_templates(ibm_ctx *ctx, int lo_nl, int hi_nl);
ibm_status launch_pinfo(ibm_ctx *ctx);
ibm_status launch_marker_bases(ibm_ctx *ctx, int64_t *base_d);

ibm_status ensure_field_ptrs(ibm_ctx *ctx, void *const *u_ptrs, void *const *f_out);
// marker exclusion near contact (ibm_contact.cu): per-step bitmap of the
// markers left out of f_IBM, its pointer while enabled (else NULL), graph key
// entries and teardown
ibm_status contact_exclusion(ibm_ctx *ctx);
const unsigned *contact_bits(const ibm_ctx *ctx);
void contact_graph_key(const ibm_ctx *ctx, std::vector<uintptr_t> &key);
void contact_free(ibm_ctx *ctx);
// collision models and particle sub-steps (ibm_collision.cu): teardown
void collision_free(ibm_ctx *ctx);

ibm_status plain_iterations_f32(ibm_ctx *ctx, const int *plist, int n_list, const int *n_list_d, double tau,
                                bool with_f, int n_it, const int *pcl);

// profiling (ibm_context.cu): bracket the main kernel of a step
void prof_begin(ibm_ctx *ctx);
void prof_end(ibm_ctx *ctx);

// cluster path (ibm_cluster.cu)
ibm_status cluster_forcing_step(ibm_ctx *ctx, void *const *u_ptrs, double tau, void *const *f_out);
void cluster_free(ibm_ctx *ctx);
ibm_status cluster_stats(ibm_ctx *ctx, int64_t *stats);
// each particle's cluster and its cluster's IBM_PATH_* bits in the last step
ibm_status cluster_membership(ibm_ctx *ctx, int32_t *cluster_of, int32_t *path_of, int64_t *n_clusters);
// appends the cluster path's device buffers and sizes to a graph key
void cluster_graph_key(const ibm_ctx *ctx, std::vector<uintptr_t> &key);
