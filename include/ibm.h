/*
 * ibm.h - C ABI of the GB300 immersed-boundary forcing-step library.
 *
 * The library implements the iterated direct-forcing immersed-boundary step of
 * Yao et al., "Particle-resolved simulations of four-way coupled polydispersed,
 * particle-laden flows" (arXiv 2109.03972), Sec. 2.2.2 "Outer forcing", on a
 * periodic collocated grid (Sec. 2.2, Fig. 1b) with the three-point
 * regularised delta kernel (Eq. 3pt-delta / 3pt-stencil; the four-point kernel
 * of Sec. 2.2.3 on the plain path), for spheres whose surface is represented
 * by Lagrangian markers (Sec. 2.1).  For every outer
 * forcing iteration m = 1..n_F it
 *   1. interpolates the cell-centred velocity to every marker,
 *   2. forms the marker force F = (U^d - U)/tau, U^d = u_p + w_p x r_l,
 *   3. spreads F back onto the grid over the same stencil,
 *   4. updates u += tau f,
 * and sums the fluid-side particle force and torque (Eq. basic-particle a,b).
 *
 * Conventions shared by every call
 *  - Every call returns an ibm_status; nothing aborts or exits.  After an error
 *    ibm_last_error() describes it.  Kernels never trap: device-side problems
 *    set an error word that the next synchronising call reports.
 *  - Units: positions in the same length unit as h; the grid of scene s has
 *    dims[s] = (nx, ny, nz) cells, cell (i,j,k) centred at ((i+1/2)h, ...),
 *    periodic in all three directions.  Particle centres may lie anywhere;
 *    they are taken modulo the box.
 *  - Velocity fields are caller-owned DEVICE arrays, one per scene, layout
 *    [3][nz][ny][nx] (component-major, x fastest), float (IBM_FP32) or double
 *    (IBM_FP64) according to the context's precision.
 *  - One context = one CUDA stream.  Calls on one context are not thread-safe
 *    and are ordered on that stream.  Calls that return host data synchronise
 *    the stream.
 *  - The context owns all scratch memory.  The caller owns u, f and gradient
 *    buffers and keeps ownership of every array it passes in.
 */
#ifndef IBM_H
#define IBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IBM_OK = 0,
    IBM_ERR_INVALID_ARG = 1,  /* a pointer, size or value is out of range     */
    IBM_ERR_CUDA = 2,         /* a CUDA runtime call failed                   */
    IBM_ERR_OOM = 3,          /* device or host allocation failed             */
    IBM_ERR_CAPACITY = 4,     /* more particles than max_particles            */
    IBM_ERR_NONFINITE = 5,    /* NaN/Inf in particle state                    */
    IBM_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up           */
    IBM_ERR_STATE = 7,        /* call out of order (e.g. backward w/o forward)*/
    IBM_ERR_NOCONVERGE = 8    /* an iterative solve missed its tolerance      */
} ibm_status;

/* precision */
enum { IBM_FP64 = 0, IBM_FP32 = 1 };

/* spread_mode
 *  IBM_SPREAD_CLUSTER        FP32 only.  Particles whose marker stencils share
 *                            a cell are grouped; each group's touched cells
 *                            stay in shared memory for all n_F iterations
 *                            (spreading by shared-memory atomics; the FP32
 *                            summation order is unspecified).  Groups too
 *                            large for one SM's shared memory run the plain
 *                            path with global atomics.
 *  IBM_SPREAD_DETERMINISTIC  As CLUSTER, but spreading accumulates in integer
 *                            fixed point (per group and iteration a power-of-
 *                            two scale), in shared memory and on the plain
 *                            path alike, so results are bit-reproducible.
 *                            The scale assumes that no cell collects more
 *                            than 64 unit weights (far above what non-
 *                            overlapping spheres give); heavily overlapping
 *                            particles that break it make the step report
 *                            IBM_ERR_CAPACITY at its next synchronising call.
 *  IBM_SPREAD_PLAIN          One thread per marker, global atomics into u, two
 *                            kernels per iteration.  The only mode for FP64
 *                            ("plain FP64 form"). */
enum { IBM_SPREAD_CLUSTER = 0, IBM_SPREAD_DETERMINISTIC = 1, IBM_SPREAD_PLAIN = 2 };

typedef struct {
    int n_scenes;            /* >= 1; independent periodic boxes               */
    const int32_t *dims;     /* HOST [n_scenes][3] = nx, ny, nz (each >= 8)    */
    double h;                /* grid spacing (> 0), isotropic (Sec. 2.1)       */
    int kernel_width;        /* 3: three-point kernel, Eq. (3pt-stencil);
                                4: four-point kernel of Sec. 2.2.3 (cells
                                floor(x/h - 1/2) - 1 .. + 2), PLAIN mode
                                only, no requires_grad                        */
    int n_forcing;           /* n_F >= 1 outer forcing iterations (Sec. 2.2.2) */
    int precision;           /* IBM_FP32 or IBM_FP64                           */
    int spread_mode;         /* IBM_SPREAD_*                                   */
    int newton_euler;        /* 1: apply Eq. (basic-particle a-c) after loop   */
    double rho_f;            /* fluid density (Newton-Euler only)              */
    double g[3];             /* gravity vector (Newton-Euler only)             */
    int max_particles;       /* capacity of the context                        */
    int requires_grad;       /* 1: keep what ibm_backward needs                */
    int threads_per_block;   /* cluster kernel (CLUSTER, DETERMINISTIC): 0 =
                                1024 threads, one CTA per SM; 512 = two
                                512-thread CTAs per SM; -1 = autotune: the
                                first two steps run each variant once, the
                                next two time each variant's whole step
                                (kernel and the fallback work its routing
                                leaves, with a host sync each); the faster
                                is kept for the context's lifetime          */
    int profile;             /* 1: time the main forcing kernel with CUDA events */
    int use_graph;           /* 1: ibm_forcing_step calls without slip_out (and
                                without requires_grad) are replayed from a CUDA
                                graph: a call runs eagerly while its field
                                pointers, tau, sizes or buffers are new, the
                                next call with the same ones captures the step
                                (stream capture on the context's stream, which
                                must not be captured by the caller) and later
                                ones replay it.  The results are those of the
                                eager step.                                   */
} ibm_config;

typedef struct ibm_ctx ibm_ctx;

/* Create a context.  cuda_stream is a cudaStream_t (NULL = legacy default
 * stream).  cfg->dims is copied.  On success *out owns device scratch sized for
 * cfg->max_particles; release it with ibm_destroy.
 * Errors: INVALID_ARG (bad config; kernel_width other than 3 or 4; width 4
 * with a mode other than PLAIN or with requires_grad; FP64 with a mode other
 * than PLAIN), OOM, CUDA. */
ibm_status ibm_create(const ibm_config *cfg, void *cuda_stream, ibm_ctx **out);

/* Release a context and all memory it owns.  NULL is accepted. */
ibm_status ibm_destroy(ibm_ctx *ctx);

/* Set the particle state used by the following forcing steps (Sec. 2.1: centre
 * x_p, velocity u_p, angular velocity w_p, diameter d_p, density rho_p).
 * Arrays are double, [n_p][3] or [n_p], in host memory (on_device = 0) or device
 * memory (on_device = 1); they are copied.  scene_of[n_p] (int32, same memory
 * space) gives each particle's scene and may be NULL when n_scenes == 1.
 * rho_p may be NULL when newton_euler == 0.
 * Marker set (reading of Sec. 2.1): N_l = round(pi (d_p/h)^2) markers on a
 * golden spiral of diameter d_p, each of volume dV_l = pi (d_p^2 h + h^3/3)/N_l.
 * Errors: INVALID_ARG (n_p < 0, NULL arrays, d_p <= 0 or d_p/h + 4 > the
 * smallest grid edge of its scene, scene index out of range, rho_p == rho_f
 * within 1e-6 relative with newton_euler), CAPACITY (n_p > max_particles),
 * NONFINITE (NaN/Inf anywhere), CUDA. */
ibm_status ibm_set_particles(ibm_ctx *ctx, int n_p, const double *x_p, const double *u_p,
                             const double *omega_p, const double *d_p, const double *rho_p,
                             const int32_t *scene_of, int on_device);

/* One immersed-boundary forcing step: the outer forcing loop of Sec. 2.2.2
 * (n_F iterations of interpolate -> force -> spread -> update), then the
 * fluid-side particle loads summed over the iterations, then (if enabled) the
 * rigid-body Newton-Euler update of Eq. (basic-particle a-c) with F_c = T_c = 0.
 * u_ptrs[n_scenes]: HOST array of DEVICE pointers to each scene's velocity
 *   field, updated in place (u^0 -> u^{n_F}).
 * tau = 2 alpha_k dt > 0 (the paper divides the slip by 2 alpha_k dt and
 *   multiplies the force by it, Sec. 2.2.2); u^{n_F} does not depend on tau.
 * f_out: NULL, or HOST array of DEVICE pointers (same layout/type as u) that
 *   receive the total IBM force sum_m f^m = (u^{n_F} - u^0)/tau on every cell
 *   (zero where no marker stencil reaches).
 * slip_out: NULL, or HOST double[2] receiving the RMS and the maximum over all
 *   markers of |U^d - W u^{n_F}| after the loop (the error eps of Sec. 2.2.2);
 *   requesting it synchronises the stream.
 * Asynchronous on the context's stream unless slip_out is given.
 * Errors: INVALID_ARG, STATE (no particles set), CUDA, TIMEOUT. */
ibm_status ibm_forcing_step(ibm_ctx *ctx, void *const *u_ptrs, double tau,
                            void *const *f_out, double *slip_out);

/* Fluid-side loads of the last forcing step, double [n_p][3] each:
 *   F_p = sum_m sum_l F^m_l dV_l,  T_p = sum_m sum_l r_l x F^m_l dV_l,
 * with r_l = X_l - x_p (Eq. basic-particle a,b; the load on the particle is
 * -rho_f times these).  x_p/u_p/omega_p, if non-NULL, receive the particle
 * state after the Newton-Euler update (or the unchanged state if it is off).
 * Destinations are host (on_device = 0; synchronises) or device memory.
 * Any pointer may be NULL.  Errors: STATE (no step yet), CUDA. */
ibm_status ibm_particle_loads(ibm_ctx *ctx, double *F, double *T, double *x_p, double *u_p,
                              double *omega_p, int on_device);

/* Mean IBM force of each scene over its grid, Eq. (fe_IBM) of Sec. 2.2.4:
 *   fbar_s = -(1 / (nx ny nz)) sum over all cells of f,   per component,
 * the volume-averaged forcing that a triply-periodic fluid solver removes from
 * its momentum equation.  (The paper's integral form of the same average, the
 * aperiodic pressure gradient of Sec. 2.2.4, carries the opposite sign; this
 * call returns the grid-pass form with its minus sign.)
 * f_ptrs[n_scenes]: HOST array of DEVICE pointers to force fields of the
 *   precision's type, layout [3][nz][ny][nx] (for example the f_out of
 *   ibm_forcing_step, whose cell sum equals the summed fluid-side loads F_p / h^3).
 * fbar_out: double [n_scenes][3], HOST (on_device = 0; the call synchronises
 *   the context's stream) or DEVICE memory (asynchronous).
 * One pass over every cell of the fields (12 B per cell in FP32, 24 B in FP64),
 * sums in FP64 in a fixed order, so the result is bit-reproducible; FP32 fields
 * are added in groups of at most 16 values in FP32 first.  Independent of the
 * particles; may be called before ibm_set_particles.
 * Errors: INVALID_ARG (NULL pointers), CUDA. */
ibm_status ibm_mean_force(ibm_ctx *ctx, void *const *f_ptrs, double *fbar_out, int on_device);

/* Fluid inertia inside each particle, Sec. 2.2.9 (second-order midpoint
 * quadrature with a level-set volume fraction), for the current particles:
 *   Iu_p = sum_c alpha_c h^3 u_c,   Ir_p = sum_c alpha_c h^3 (r_c x u_c),
 *   V_p  = sum_c alpha_c h^3,
 *   alpha_c = sum_m -phi_m H(-phi_m) / sum_m |phi_m|  over the 8 corners of
 *   cell c, H(-phi) = 1 for phi <= 0, phi_m = |x_m - x_p| - d_p/2 (signed
 *   distance of the corner to the sphere's surface; the paper's wording, the
 *   distance to the centre, is read as this signed distance, without which
 *   alpha would vanish); r_c = cell centre - x_p (minimum image).
 * The rate-of-change terms d/dt int u dV and d/dt int r x u dV of the particle
 * equations follow from two evaluations (the direct form, without the
 * rigid-body singularity at rho_p = rho_f).
 * u_ptrs[n_scenes]: HOST array of DEVICE pointers to the fields (the precision's
 * type, [3][nz][ny][nx]); read only.  Iu, Ir: double [n_p][3]; V: double [n_p];
 * any may be NULL; HOST (on_device = 0; synchronises) or DEVICE memory.
 * FP32 fields are summed per thread in FP32 over at most a few dozen cells and
 * per particle in FP64; the result is bit-reproducible.  With no particles set
 * the call does nothing.  Errors: INVALID_ARG (NULL u_ptrs), CUDA. */
ibm_status ibm_particle_inertia(ibm_ctx *ctx, void *const *u_ptrs, double *Iu, double *Ir, double *V,
                                int on_device);

/* Marker exclusion near contact, Sec. 2.2.5: from the next forcing step on,
 * markers are left out of f_IBM where two particles come within reach of each
 * other.  For every pair (p, q) of a scene whose surface gap
 *   zeta = |x_q - x_p| - d_p/2 - d_q/2   (minimum image)
 * is below 2 eps_sep, one particle of the pair is chosen at random and its
 * markers whose distance to the partner's surface, |X_l - x_o| - d_o/2, is
 * below 2 eps_sep get F_l = 0 in every iteration (they neither spread nor add
 * to the loads; the slip of ibm_forcing_step still covers every marker).  The
 * paper names the pair criterion and the random choice of one particle; which
 * of its markers go is this library's reading: those facing the partner within
 * the same reach.  The choice: with i < j the pair's particle indices (the
 * order of ibm_set_particles, across scenes), z = SplitMix64(seed ^ (i << 32 | j))
 * (Steele, Lea and Flood, 2014) and particle j is chosen when the top bit of
 * z is set, else particle i.
 * enable: 1 on, 0 off.  eps_sep: the threshold separation in physical units;
 *   0 takes the paper's value, 1.5 h for kernel_width 3 and 2 h for 4.
 * Every spread mode (the shared-memory cluster kernel and its plain fallback
 * skip those markers the same way); needs requires_grad = 0 (INVALID_ARG
 * otherwise: there is no adjoint of the exclusion).
 * Errors: INVALID_ARG.  A step whose pairs in reach exceed 32 per particle
 * reports CAPACITY at the next error check. */
ibm_status ibm_set_contact_exclusion(ibm_ctx *ctx, int enable, double eps_sep, uint64_t seed);

/* Markers left out by the last forcing step (ibm_set_contact_exclusion), as a
 * bitmap over markers in particle-then-l order: bit (m & 31) of word m >> 5,
 * HOST uint32[(n_markers + 31) / 32] (NULL to query the count only).
 * *n_disabled receives the number of set bits (0 while exclusion is off).
 * Synchronises.  Errors: INVALID_ARG, CUDA. */
ibm_status ibm_disabled_markers(ibm_ctx *ctx, uint32_t *bits_out, int64_t *n_disabled);

/* Backward pass of the last forcing step (requires requires_grad = 1 at
 * create).  For a loss L(u^{n_F}) with grad_u_out[s] = dL/du^{n_F} (DEVICE,
 * same layout/type as u), writes grad_u_in[s] = dL/du^0 (DEVICE, may alias
 * grad_u_out) and the FP64 particle gradients dL/du_p, dL/dw_p, dL/dx_p
 * ([n_p][3] each, DEVICE memory, any may be NULL).  The adjoint follows the
 * loop algebra of Sec. 2.2.2: spreading is the adjoint of interpolation and
 * vice versa, plus delta-kernel derivative terms for the marker positions.
 * Markers and weights are recomputed per iteration from the saved u^0.
 * Errors: STATE (requires_grad off or no forward step), INVALID_ARG, CUDA. */
ibm_status ibm_backward(ibm_ctx *ctx, void *const *grad_u_out, void *const *grad_u_in,
                        double *gU, double *gOmega, double *gX);

/* Parameters of the collision models (Sec. 2.2.6-2.2.8) for
 * ibm_particle_substeps and ibm_collision_forces, in the length and time units
 * of h and the particle state.  0 in eps_sep, zeta_min, lub_c or pair_margin
 * takes the default given. */
typedef struct {
    double rho_f;        /* fluid density (> 0)                                */
    double nu_f;         /* kinematic viscosity (>= 0; 0 turns lubrication off)*/
    double e_dry;        /* dry restitution coefficient, 0 < e_dry < 1         */
    double mu_s, mu_k;   /* static and kinetic friction coefficients           */
    double nu_poisson;   /* Poisson's ratio of the particle material           */
    double t_c;          /* collision time T_c (the paper uses 10 dt)          */
    double st_crit;      /* critical Stokes number (the paper uses 5)          */
    double eps_sep;      /* threshold separation; 0: 1.5 h (3-point), 2 h      */
    double zeta_min;     /* floor of the lubrication gap; 0: 0.01 h            */
    double lub_c;        /* C of the erf blend; 0: 5.5 (3-point), 4 (4-point)  */
    double g[3];         /* gravity                                            */
    double pair_margin;  /* neighbour-list margin beyond eps_sep; 0: 1.5 h     */
} ibm_collision_params;

/* Advance the particle state of ctx (x_p, u_p, w_p of ibm_set_particles, with
 * rho_p given) by dt under the collision models of Sec. 2.2.6-2.2.8 and
 * constant hydrodynamic loads, in n_sub sub-steps of dt/n_sub, each the
 * three-stage predictor-corrector Runge-Kutta update of Sec. 2.2.10 (the paper
 * uses 15 sub-steps).  Collision force on p (Eq. f_int), summed over its pairs
 * in the same scene, each with n from p to q (minimum image) and surface gap
 * zeta_n: for 0 < zeta_n < eps_sep the lubrication force
 * -6 pi rho_f nu_f R_eff^2 psi / max(zeta_min, zeta_n) g_n, psi =
 * erf(6 - C max(zeta_min, zeta_n)/h)/2 + 1/2; for zeta_n <= 0 the Hertz
 * contact -k_n |zeta_n|^{3/2} n - d_n g_n plus the tangential spring-dashpot
 * force capped by mu |F_n| (stick/slip), with torque R_p,cp n x F_t.  Stiffness
 * and damping follow the adaptive collision time model; where the paper cites
 * closed forms it does not print, this library's reading is used: k_n =
 * m_eff/sqrt(u_in t*^5) with t* = T_c (4/5)^{2/5}/(2 I_H), the stiffness for
 * which an undamped Hertz impact at speed u_in lasts T_c (I_H = sqrt(pi)
 * Gamma(7/5)/Gamma(9/10)), below the critical impact speed of St_crit
 * max(k_n(u_in,crit), k_n,grav); d_n = -2 m_eff ln(e_dry)/T_c; k_t =
 * 2(1-nu)/(2-nu) k_n.  No walls (periodic boxes).
 * F_h, T_h: the hydrodynamic force and torque on each particle ([n_p][3],
 * host or device per on_device, held constant over the call; NULL = 0), e.g.
 * -rho_f times the fluid-side loads of ibm_particle_loads.  The state is
 * updated in place (read it with ibm_particle_state; the next forcing step
 * uses it); the tangential springs and impact speeds of the pairs in contact
 * are kept for the next call while the particle count stays the same.
 * FP64; every sum in a fixed order (bit-reproducible).  Synchronises.
 * Errors: INVALID_ARG (parameters, dt <= 0, n_sub < 1, densities not
 * positive), CAPACITY (a particle moved more than half of pair_margin in the
 * call, so that pairs could have been missed), OOM, CUDA. */
ibm_status ibm_particle_substeps(ibm_ctx *ctx, const ibm_collision_params *prm, double dt, int n_sub,
                                 const double *F_h, const double *T_h, int on_device);

/* Collision force F_c,p and torque T_c,p of every particle (Eq. f_int) at the
 * current state with the kept contact history ([n_p][3] each, host or device;
 * either may be NULL).  Synchronises for host outputs.
 * Errors: INVALID_ARG, CAPACITY, OOM, CUDA. */
ibm_status ibm_collision_forces(ibm_ctx *ctx, const ibm_collision_params *prm, double *F_c, double *T_c,
                                int on_device);

/* Current particle state of ctx (x_p, u_p, w_p, [n_p][3] each, host or device;
 * any may be NULL).  Synchronises for host outputs.  Errors: CUDA. */
ibm_status ibm_particle_state(ibm_ctx *ctx, double *x_p, double *u_p, double *omega_p, int on_device);

/* Contact history kept by the last ibm_particle_substeps: the pairs (p, q),
 * p < q, in contact at its end, ordered by p, with the tangential spring
 * (in p's frame, double [n][3]) and the impact speed.  HOST arrays of
 * *n_pairs entries; pass NULL arrays to query the count.  Synchronises.
 * Errors: INVALID_ARG, CUDA. */
ibm_status ibm_contact_history(ibm_ctx *ctx, int64_t *n_pairs, int32_t *p, int32_t *q, double *zeta_t,
                               double *u_in);

/* Diagnostics.  Stencil base cell of every marker, in particle-then-l order,
 * as the active precision path computes it: floor(X_l/h) per axis
 * (floor(X_l/h - 1/2) for kernel_width 4), NOT wrapped
 * (int64 [n_markers][3], HOST).  *n_markers receives the count; pass base_out
 * = NULL to query it.  Synchronises.  Errors: STATE, INVALID_ARG, CUDA. */
ibm_status ibm_marker_bases(ibm_ctx *ctx, int64_t *base_out, int64_t *n_markers);

/* Diagnostics of the last forcing step (HOST int64[12], synchronises):
 * [0] markers, [1] particle clusters, [2] clusters on the shared-memory path,
 * [3] markers on the plain fallback path, [4] largest cluster held in shared
 * memory (touched cells), [5] distinct touched cells on the shared-memory
 * path, [6] kernel launches per step, [7] threads per block of the cluster
 * kernel, [8] clusters run one velocity component at a time, [9] candidate
 * particle pairs tested, [10] clusters and [11] markers on the thread-block-
 * cluster path (IBM_PATH_DSMEM).  Entries [1]-[5], [7]-[11] are 0 in PLAIN
 * mode. */
ibm_status ibm_step_stats(ibm_ctx *ctx, int64_t *stats);

/* Code paths of a particle cluster in the last forcing step, as bits of
 * ibm_particle_clusters' path_of. */
enum {
    IBM_PATH_SMEM = 1,            /* shared-memory cluster kernel                 */
    IBM_PATH_GLOBAL_RECORDS = 2,  /* ... with its marker records in global memory */
    IBM_PATH_ONE_COMPONENT = 4,   /* ... one velocity component at a time         */
    IBM_PATH_SPARSE_ROWS = 8,     /* ... with the sparse row table                */
    IBM_PATH_PERIODIC = 16,       /* the cluster's box wraps around the period    */
    IBM_PATH_FALLBACK = 32,       /* the plain path (global atomics)              */
    IBM_PATH_DSMEM = 64           /* too large for one SM: the distributed shared
                                     memory of a thread-block cluster of 8 or 16
                                     CTAs holds its box                         */
};

/* Diagnostics of the cluster modes (CLUSTER, DETERMINISTIC).  Particles whose
 * marker stencils share a grid cell, directly or through other particles, form
 * a cluster: the connected components of that relation are independent for
 * all n_F iterations of Sec. 2.2.2.  For the last forcing step, cluster_of[p]
 * receives particle p's cluster (0 .. n_clusters-1) and path_of[p] the
 * IBM_PATH_* bits of the code path its cluster took (HOST int32 [n_p] each,
 * either may be NULL); *n_clusters (may be NULL) the number of clusters.
 * Synchronises.  Errors: STATE (PLAIN mode, or no step since the last
 * ibm_set_particles), CUDA. */
ibm_status ibm_particle_clusters(ibm_ctx *ctx, int32_t *cluster_of, int32_t *path_of, int64_t *n_clusters);

/* Device time of the main forcing kernel (the shared-memory cluster kernel,
 * or the plain interpolation+spreading kernels in PLAIN mode), measured with
 * CUDA events recorded on the context's stream around each launch since the
 * last reset; requires profile = 1 at create.  *total_ms and *count receive the
 * summed time and the number of timed steps.  reset = 1 clears the record after
 * reading.  Synchronises.  Errors: STATE (profile off), CUDA. */
ibm_status ibm_kernel_timing(ibm_ctx *ctx, double *total_ms, int64_t *count, int reset);

/* One FP64 forcing step that allocates nothing (no context, no cudaMalloc or
 * cudaFree, no host allocation).  For callers that cannot allocate device
 * memory: hosts that hand the library a fixed memory budget at start-up and
 * forbid allocations afterwards, plugins inside an application whose own
 * allocator owns the device memory, and time-critical loops that cannot afford
 * the device-wide synchronisation of cudaFree.  The paper has no counterpart;
 * it is the plain FP64 form of ibm_forcing_step (one thread per marker, global
 * atomics) for a single periodic nx*ny*nz grid, with the same results up to
 * the order of floating-point additions.
 * Inputs (DEVICE, double): x_p, u_p, omega_p [n_p][3], d_p [n_p].
 * In/out (DEVICE, double): u [3][nz][ny][nx], updated in place.
 * Outputs (DEVICE, double): F_out, T_out [n_p][3], the fluid-side loads summed
 *   over the n_forcing iterations (as ibm_particle_loads).
 * Scratch: one 16 MiB array inside the library that every GPU loading the
 * library holds until exit.  Limits: n_p <= 65536 and at most 688,106 markers
 * in total (N_l = round(pi (d_p/h)^2) per particle); larger inputs return
 * IBM_ERR_CAPACITY and leave u unchanged.  Every call reuses the same array,
 * so calls whose work overlaps on the GPU (other streams, other host threads
 * on the same device) race and corrupt each other.  The first call on a device
 * does the set-up: it looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture begins.  The address stays valid until the device is
 * reset: after cudaDeviceReset the entry point must not be called on that
 * device again in the same process.  The call synchronises cuda_stream to read
 * its error word.  On an error the particle data was rejected on the device
 * (INVALID_ARG from the particle checks, CAPACITY from the marker total),
 * F_out and T_out hold zeros and u is unchanged; on an error found on the host
 * (bad sizes or pointers) nothing is written.
 * Errors: INVALID_ARG (bad sizes, NULL pointers, non-finite or oversized
 * particles: d_p/h + 4 > smallest grid edge), CAPACITY, CUDA. */
ibm_status ibm_forcing_step_static(int nx, int ny, int nz, double h, int n_forcing, double tau, int n_p,
                                   const double *x_p, const double *u_p, const double *omega_p,
                                   const double *d_p, double *u, double *F_out, double *T_out,
                                   void *cuda_stream);

/* Bound of the device-side retry loops of the cluster modes (the lock-free
 * union-find that joins particles into clusters retries a compare-and-swap
 * until it succeeds; every retry loop gives up after this many iterations and
 * the step reports IBM_ERR_TIMEOUT at its next synchronising call instead of
 * spinning on).  0 restores the default, 2^22.  Applies to the following
 * forcing steps of ctx; a step that gave up leaves its velocity field invalid,
 * the context itself stays usable.  The paper has no counterpart: it is a
 * safeguard of this library, exposed so that the give-up path can be tested.
 * Errors: INVALID_ARG (NULL ctx, iterations < 0 or > INT32_MAX). */
ibm_status ibm_set_wait_limit(ibm_ctx *ctx, int64_t iterations);

/* Test hook, process-wide: the n-th device allocation the library makes after
 * this call fails as if the device were out of memory (the call that makes it
 * returns IBM_ERR_OOM and releases what it had allocated so far); n = 0 turns
 * the hook off.  No GPU fault is involved: the allocation is refused on the
 * host before cudaMalloc.  The paper has no counterpart.
 * Errors: INVALID_ARG (n < 0). */
ibm_status ibm_debug_fail_allocation(int64_t n);

/* ------------------------------------------------------------------------
 * Collocated fractional-step fluid solver (Sec. 2.2.1 "Pressure-momentum
 * coupling on a collocated grid" and Sec. 2.2.4, the modified solver
 * Eq. fluid-solver (a)-(i)) on one triply periodic grid, FP64.  One RK3 stage
 * k (alpha_k, gamma_k, zeta_k of the Rai and Moin scheme that Sec. 2.1 names) is
 *   (a)  u~ = u + dt (2 alpha nu lap u - 2 alpha grad P - gamma N(u) - zeta N_old),
 *        N(u) = (u . grad) u (advective form, central differences), kept as
 *        the next stage's N_old;
 *   (b)-(d) the IBM forcing loop on u~ (ibm_forcing_step with tau = 2 alpha dt,
 *        which leaves u~ + 2 alpha dt f_IBM in place);
 *   (e)  (1 - alpha dt nu lap) u* = u~ - 2 alpha dt f_mean - alpha dt nu lap u
 *                                  + 2 alpha theta dt grad P     (Crank-Nicolson),
 *        f_mean the volume average of f_IBM (compatibility, Sec. 2.2.4);
 *   (f)  u_f* = I(u*): the mean of the two cells at each face;
 *   (g)  lap phi = div u_f* / (2 alpha dt)  (compact 7-point operator);
 *   (h)  u = u* - 2 alpha dt grad phi (central), u_f = u_f* - 2 alpha dt
 *        (grad phi)_f (difference across the face);
 *   (i)  P = (1 - theta) P + theta (phi - alpha dt nu lap phi).
 * The equations of (e) and (g) are solved to the relative FP64 residual rtol
 * (max norm) by iterative refinement: FP64 residual, one FP32 multigrid
 * V-cycle for the correction (two red-black Gauss-Seidel sweeps before and
 * after each coarse correction, averaging restriction, trilinear
 * prolongation, a one-CTA conjugate-gradient solve on the coarsest level),
 * FP64 update.  The Poisson right-hand side is made mean-free and phi leaves
 * each stage with zero mean.  Everything is deterministic.
 *
 * Fields are caller-owned DEVICE arrays of doubles, x fastest:
 *   u, ut, uf  [3][nz][ny][nx]; p, phi [nz][ny][nx].
 * uf[d] holds the face between cell i and cell i+1 along axis d.
 * ---------------------------------------------------------------------- */
typedef struct ibm_fluid ibm_fluid;

typedef struct {
    int nx, ny, nz;          /* periodic grid, each >= 2; halving every even
                                extent down to at most 32768 cells must be
                                possible (the coarsest multigrid level)       */
    double h;                /* grid spacing (> 0)                             */
    double nu;               /* kinematic viscosity (>= 0)                     */
    double theta;            /* 0: pressure projection, 1: pressure correction
                                (step (i)); any value in [0, 1]               */
    double rtol;             /* relative max-norm residual of each solve;
                                0 = 1e-12                                     */
    int max_cycles;          /* V-cycles (refinement steps) per solve before
                                IBM_ERR_NOCONVERGE; 0 = 60                    */
    int profile;             /* 1: time every finest-level smoothing sweep
                                with CUDA events (ibm_fluid_kernel_timing)    */
    int two_pass_smoother;   /* 1: smooth every level by two half sweeps (red,
                                then black) instead of the fused one-pass
                                sweep; the results are the same bit for bit
                                (a cross-check)                               */
} ibm_fluid_config;

typedef struct {
    double *u;      /* u^{k-1} in, u^k out                                    */
    double *ut;     /* out: u~ after ibm_fluid_predict; in: the forced u~ to
                       ibm_fluid_correct, which leaves u* in it               */
    double *uf;     /* out: face velocities u_f^k                             */
    double *p;      /* P^{k-1} in, P^k out                                    */
    double *phi;    /* in: initial guess of the Poisson solve; out: phi       */
} ibm_fluid_fields;

/* Create a solver on cuda_stream (NULL = legacy default stream).  It owns
 * the scratch: N_old (zero at creation), the FP64 right-hand side of the
 * solves and the FP32 multigrid levels, about 46 bytes per cell (70 once
 * ibm_fluid_stage keeps an f_IBM of its own).
 * Errors: INVALID_ARG (sizes, h, nu, theta, coarsest level too large),
 * OOM, CUDA. */
ibm_status ibm_fluid_create(const ibm_fluid_config *cfg, void *cuda_stream, ibm_fluid **out);
ibm_status ibm_fluid_destroy(ibm_fluid *fl);

/* Step (a) of RK3 stage k (0, 1, 2) with time step dt: writes ut and the
 * stage's convective term (kept inside fl for stage k+1; stage 0 ignores it).
 * Errors: INVALID_ARG (k, dt, NULL field), CUDA. */
ibm_status ibm_fluid_predict(ibm_fluid *fl, int k, double dt, const ibm_fluid_fields *F);

/* Steps (e)-(i) of stage k from the forced field in ut.  mean_f: NULL (no
 * IBM force), or the volume average of f_IBM per component, [3] doubles,
 * HOST memory (on_device = 0) or DEVICE memory (1).  Note that
 * ibm_mean_force returns its negation (Eq. fe_IBM).  Synchronises the stream
 * once per V-cycle (convergence test).
 * Errors: INVALID_ARG, NOCONVERGE (a solve missed rtol in max_cycles; the
 * fields then hold the last iterate), CUDA. */
ibm_status ibm_fluid_correct(ibm_fluid *fl, int k, double dt, const ibm_fluid_fields *F, const double *mean_f,
                             int on_device);

/* One whole RK3 stage k: ibm_fluid_predict, the forcing loop of ctx on ut
 * (tau = 2 alpha_k dt; ctx FP64, one scene of the same dims and h; NULL ctx
 * or no particles: no forcing), the grid-pass mean of f_IBM (ibm_mean_force),
 * and ibm_fluid_correct.  f_out: NULL (scratch inside fl), or a DEVICE
 * [3][nz][ny][nx] array that receives f_IBM.  The particle loads of the stage
 * are then available from ibm_particle_loads(ctx, ...).  ctx's stream is
 * ordered after fl's and back by events.
 * Errors: as the calls it makes (messages copied to fl). */
ibm_status ibm_fluid_stage(ibm_fluid *fl, ibm_ctx *ctx, int k, double dt, const ibm_fluid_fields *F,
                           double *f_out);

/* Solver report of the last ibm_fluid_correct: cycles[4] and resid[4] (V-cycles
 * and final relative max-norm residual of the three Helmholtz solves and the
 * Poisson solve), levels = multigrid levels.  Any pointer may be NULL. */
ibm_status ibm_fluid_stats(ibm_fluid *fl, int64_t *cycles, double *resid, int *levels);

/* With cfg.profile: total device time (ms) and count of the finest-level
 * red-black sweeps since the last reset (synchronises the stream).  Without
 * it both are 0.  Errors: INVALID_ARG, CUDA. */
ibm_status ibm_fluid_kernel_timing(ibm_fluid *fl, double *total_ms, int64_t *count, int reset);

/* Description of the last error on fl (empty string if none); never NULL. */
const char *ibm_fluid_last_error(const ibm_fluid *fl);

/* Human-readable status name; never NULL. */
const char *ibm_status_string(ibm_status s);

/* Description of the last error on ctx (empty string if none); never NULL. */
const char *ibm_last_error(const ibm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* IBM_H */
