/*
 * CPU oracle of the collision models and the RK3 particle sub-stepping of
 * Yao et al. (arXiv 2109.03972), Sec. 2.2.6-2.2.8 (Eq. f_int, the lubrication,
 * normal contact and tangential contact models) and Sec. 2.2.10 (the
 * predictor-corrector Runge-Kutta sub-steps of the particle equations).
 *
 * TEST INFRASTRUCTURE ONLY: plain FP64, every particle pair visited each time
 * (O(N^2)), no neighbour lists.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares nothing with the GPU code.
 *
 * Readings where the paper is silent or refers elsewhere:
 *  - Triply periodic boxes, no walls: the wall terms of Eq. f_int do not arise.
 *    Pair geometry uses the minimum image of x_q - x_p.
 *  - n = (x_q - x_p)/|x_q - x_p| (from p to q), zeta_n = |x_q - x_p| - R_p - R_q.
 *    The contact point lies R_p,cp = (|x_q - x_p| + R_p - R_q)/2 from x_p along
 *    n (the paper's effective radius) and R_q,cp from x_q along -n.
 *    g_cp = (u_p + w_p x R_p,cp n) - (u_q + w_q x (-R_q,cp n)), the velocity of
 *    p's surface relative to q's there; g_n = (g_cp . n) n, g_t = g_cp - g_n.
 *  - Lubrication for 0 < zeta_n < eps_sep (printed form with the erf blend),
 *    contact for zeta_n <= 0, nothing from eps_sep on.
 *  - ACTM stiffness (the paper takes the closed forms of Ray et al., not printed):
 *    the undamped Hertz impact m x'' = -k x^{3/2} at speed u lasts
 *    T = 2 I_H x_max / u with x_max = (5 m u^2 / (4 k))^{2/5} and
 *    I_H = int_0^1 (1 - s^{5/2})^{-1/2} ds = sqrt(pi) Gamma(7/5) / Gamma(9/10),
 *    so k = m_eff / sqrt(u t*^5) with t* = T_c (4/5)^{2/5} / (2 I_H) -- the form
 *    of the printed k_n,crit.  k_n = that at the impact speed u_in when
 *    u_in > u_in,crit, else max(its value at u_in,crit, k_n,grav);
 *    u_in,crit follows from St_crit with the larger of the two particles'
 *    9 rho_f nu_f / (rho d); u_in is |g_cp . n| at first contact.
 *  - d_n = -2 m_eff ln(e_dry) / T_c: the damping that gives restitution e_dry
 *    over a contact of duration T_c.
 *  - k_t = 2 (1 - nu_poi)/(2 - nu_poi) k_n (the printed ratio, dimensionless
 *    as printed, times k_n); d_t as printed with (ln e_dry)^2.
 *  - Stick when |F_t,dp| < mu_s |F_n|, else slip with |F_t| = mu_k |F_n|; on
 *    slip the spring is reset so that -k_t zeta_t - d_t g_t has magnitude
 *    mu_k |F_n| (Luding), done with the history update at the end of a stage.
 *  - zeta_t is integrated once per RK stage over its duration 2 alpha_k dt_sub
 *    from the corrected state and kept in the tangent plane; it and u_in live
 *    while the pair touches and are cleared when it separates.
 *  - RK3 coefficients of Rai and Moin: alpha = 4/15, 1/15, 1/6;
 *    gamma = 8/15, 5/12, 3/4; zeta = 0, -17/60, -5/12.
 *  - m_p = rho_p pi d^3/6, I_p = m_p d^2/10; g' = (1 - rho_f/rho_p) g (the
 *    printed rho_g read as rho_p).
 *
 * Parameter vector P: [0] rho_f [1] nu_f [2] e_dry [3] mu_s [4] mu_k
 * [5] nu_poisson [6] T_c [7] St_crit [8] eps_sep [9] zeta_min [10] C of the
 * erf blend [11..13] g [14] h.
 *
 * Pair history (canonical pairs p < q, state in p's frame): arrays hp, hq,
 * hz[3*], hu with *nh entries of capacity cap.
 *
 * Parity: pinned in the tests by the Hertz force at a given overlap, the
 * blend's limits, the stick/slip switch, pairwise momentum and angular
 * momentum balance, exact free flight under gravity, and the restitution
 * and duration of a head-on collision.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

static const double RK_A[3] = {4.0 / 15.0, 1.0 / 15.0, 1.0 / 6.0};
static const double RK_G[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
static const double RK_Z[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

double orc_tstar(double t_c)
{
    const double ih = sqrt(ORC_PI) * tgamma(1.4) / tgamma(0.9);
    return t_c * pow(0.8, 0.4) / (2.0 * ih);
}

double orc_mass(double d, double rho) { return rho * ORC_PI * d * d * d / 6.0; }

/* Minimum image of x_q - x_p in a periodic box of dims (nx, ny, nz) cells of h. */
static void min_image(const double *xp, const double *xq, const long *dims, double h, double *dv)
{
    for (int c = 0; c < 3; ++c) {
        const double L = (double)dims[c] * h;
        double v = xq[c] - xp[c];
        v -= L * floor(v / L + 0.5);
        dv[c] = v;
    }
}

/* Normal stiffness of a pair (reading above). */
double orc_kn(const double *P, double m_eff, double uin, double rho_p, double d_p, double rho_q, double d_q,
              double m_p, double m_q)
{
    const double rho_f = P[0], nu_f = P[1], st = P[7];
    const double ts = orc_tstar(P[6]);
    double uc = 9.0 * st * rho_f * nu_f / (rho_p * d_p);
    const double uc2 = 9.0 * st * rho_f * nu_f / (rho_q * d_q);
    if (uc2 > uc) uc = uc2;
    if (uin > uc) return m_eff / sqrt(uin * pow(ts, 5.0));
    double kc = uc > 0.0 ? m_eff / sqrt(uc * pow(ts, 5.0)) : 0.0;
    const double g = sqrt(P[11] * P[11] + P[12] * P[12] + P[13] * P[13]);
    double kg = m_p * g * pow(1e-3 * 0.5 * d_p, -1.5);
    const double kg2 = m_q * g * pow(1e-3 * 0.5 * d_q, -1.5);
    if (kg2 > kg) kg = kg2;
    return kc > kg ? kc : kg;
}

/* Force and torque on particle `self` from its pair with `other` (positions
 * x_self and the minimum-image offset dv = x_other - x_self); zt: the
 * tangential spring in self's frame, uin: recorded impact speed (< 0: none).
 * Returns zeta_n.  Sec. 2.2.6-2.2.8 with the readings of the file header. */
double orc_pair(const double *P, const double *dv, const double *us, const double *uo, const double *ws,
                const double *wo, double ds, double dd_o, double rs, double ro, const double *zt, double uin,
                double *F, double *T)
{
    const double h = P[14], eps = P[8];
    const double Rs = 0.5 * ds, Ro = 0.5 * dd_o;
    const double dist = sqrt(dot3(dv, dv));
    double n[3] = {dv[0] / dist, dv[1] / dist, dv[2] / dist};
    const double zeta = dist - Rs - Ro;
    for (int c = 0; c < 3; ++c) F[c] = T[c] = 0.0;
    if (zeta >= eps) return zeta;
    const double rcs = 0.5 * (dist + Rs - Ro), rco = 0.5 * (dist + Ro - Rs);
    double as[3] = {rcs * n[0], rcs * n[1], rcs * n[2]}, ao[3] = {-rco * n[0], -rco * n[1], -rco * n[2]};
    double cs[3], co[3], g[3], gn[3], gt[3];
    cross3(ws, as, cs);
    cross3(wo, ao, co);
    for (int c = 0; c < 3; ++c) g[c] = (us[c] + cs[c]) - (uo[c] + co[c]);
    const double gns = dot3(g, n);
    for (int c = 0; c < 3; ++c) {
        gn[c] = gns * n[c];
        gt[c] = g[c] - gn[c];
    }
    const double ms = orc_mass(ds, rs), mo = orc_mass(dd_o, ro);
    const double m_eff = ms * mo / (ms + mo);
    if (zeta > 0.0) {
        /* lubrication, Cox and Brenner with the erf blend */
        const double rho_f = P[0], nu_f = P[1], zmin = P[9], C = P[10];
        const double R_eff = Rs * Ro / (Rs + Ro);
        const double zm = zeta > zmin ? zeta : zmin;
        const double psi = 0.5 * erf(6.0 - C * zm / h) + 0.5;
        const double coef = 6.0 * ORC_PI * rho_f * nu_f * R_eff * R_eff * psi / zm;
        for (int c = 0; c < 3; ++c) F[c] = -coef * gn[c];
        return zeta;
    }
    /* normal contact (Hertz with ACTM coefficients) */
    const double u_in = uin >= 0.0 ? uin : fabs(gns);
    const double kn = orc_kn(P, m_eff, u_in, rs, ds, ro, dd_o, ms, mo);
    const double dn = -2.0 * m_eff * log(P[2]) / P[6];
    const double ov = pow(-zeta, 1.5);
    double Fn[3];
    for (int c = 0; c < 3; ++c) Fn[c] = -kn * ov * n[c] - dn * gn[c];
    /* tangential contact (spring-dashpot with Coulomb limit) */
    const double nu = P[5], le = log(P[2]);
    const double kt = 2.0 * (1.0 - nu) / (2.0 - nu) * kn;
    const double dt = 2.0 * sqrt(m_eff * kt) * (-le) / sqrt(ORC_PI * ORC_PI + le * le);
    double Fdp[3];
    for (int c = 0; c < 3; ++c) Fdp[c] = -kt * zt[c] - dt * gt[c];
    const double fn = sqrt(dot3(Fn, Fn)), fdp = sqrt(dot3(Fdp, Fdp));
    double Ft[3];
    if (fdp < P[3] * fn || fdp == 0.0) {
        for (int c = 0; c < 3; ++c) Ft[c] = Fdp[c];
    } else {
        for (int c = 0; c < 3; ++c) Ft[c] = P[4] * fn * Fdp[c] / fdp;
    }
    for (int c = 0; c < 3; ++c) F[c] = Fn[c] + Ft[c];
    cross3(as, Ft, T);
    return zeta;
}

static long find_pair(long nh, const long *hp, const long *hq, long p, long q)
{
    for (long i = 0; i < nh; ++i)
        if (hp[i] == p && hq[i] == q) return i;
    return -1;
}

/* Collision force F_c,p and torque T_c,p of every particle, Eq. (f_int),
 * with the pair history as given (not modified). */
void orc_collision_forces(long np, const long *dims, const int *scene, const double *P, const double *x,
                          const double *u, const double *om, const double *d, const double *rho, long nh,
                          const long *hp, const long *hq, const double *hz, const double *hu, double *Fc,
                          double *Tc)
{
    for (long p = 0; p < np; ++p) {
        double Fs[3] = {0, 0, 0}, Ts[3] = {0, 0, 0};
        for (long q = 0; q < np; ++q) {
            if (q == p || scene[q] != scene[p]) continue;
            double dv[3], F[3], T[3], zt[3] = {0, 0, 0}, uin = -1.0;
            min_image(x + 3 * p, x + 3 * q, dims + 3 * scene[p], P[14], dv);
            const long lo = p < q ? p : q, hi = p < q ? q : p;
            const long i = find_pair(nh, hp, hq, lo, hi);
            if (i >= 0) {
                const double sgn = p < q ? 1.0 : -1.0;   /* stored in the lower index's frame */
                for (int c = 0; c < 3; ++c) zt[c] = sgn * hz[3 * i + c];
                uin = hu[i];
            }
            orc_pair(P, dv, u + 3 * p, u + 3 * q, om + 3 * p, om + 3 * q, d[p], d[q], rho[p], rho[q], zt, uin, F,
                     T);
            for (int c = 0; c < 3; ++c) {
                Fs[c] += F[c];
                Ts[c] += T[c];
            }
        }
        for (int c = 0; c < 3; ++c) {
            Fc[3 * p + c] = Fs[c];
            Tc[3 * p + c] = Ts[c];
        }
    }
}

/* History update at the end of an RK stage of duration dts, from the
 * corrected state: zeta_t += dts g_t in the tangent plane, u_in recorded at
 * first contact, the Luding reset on slip; separated pairs dropped.
 * Returns 0, or -1 if the history is full. */
static int history_update(long np, const long *dims, const int *scene, const double *P, const double *x,
                          const double *u, const double *om, const double *d, const double *rho, double dts,
                          long cap, long *nh, long *hp, long *hq, double *hz, double *hu)
{
    long *np2 = malloc(sizeof(long) * (size_t)(cap > 0 ? cap : 1));
    long *nq2 = malloc(sizeof(long) * (size_t)(cap > 0 ? cap : 1));
    double *nz2 = malloc(sizeof(double) * 3 * (size_t)(cap > 0 ? cap : 1));
    double *nu2 = malloc(sizeof(double) * (size_t)(cap > 0 ? cap : 1));
    long k = 0;
    int rc = 0;
    for (long p = 0; p < np && rc == 0; ++p)
        for (long q = p + 1; q < np; ++q) {
            if (scene[q] != scene[p]) continue;
            double dv[3];
            min_image(x + 3 * p, x + 3 * q, dims + 3 * scene[p], P[14], dv);
            const double dist = sqrt(dot3(dv, dv));
            const double Rp = 0.5 * d[p], Rq = 0.5 * d[q];
            const double zeta = dist - Rp - Rq;
            if (zeta > 0.0) continue;
            if (k >= cap) { rc = -1; break; }
            double n[3] = {dv[0] / dist, dv[1] / dist, dv[2] / dist};
            const double rcp = 0.5 * (dist + Rp - Rq), rcq = 0.5 * (dist + Rq - Rp);
            double ap[3] = {rcp * n[0], rcp * n[1], rcp * n[2]}, aq[3] = {-rcq * n[0], -rcq * n[1], -rcq * n[2]};
            double cp[3], cq[3], g[3], gt[3];
            cross3(om + 3 * p, ap, cp);
            cross3(om + 3 * q, aq, cq);
            for (int c = 0; c < 3; ++c) g[c] = (u[3 * p + c] + cp[c]) - (u[3 * q + c] + cq[c]);
            const double gns = dot3(g, n);
            for (int c = 0; c < 3; ++c) gt[c] = g[c] - gns * n[c];
            const long i = find_pair(*nh, hp, hq, p, q);
            double zt[3] = {0, 0, 0};
            double uin = fabs(gns);
            if (i >= 0) {
                for (int c = 0; c < 3; ++c) zt[c] = hz[3 * i + c];
                uin = hu[i];
            }
            for (int c = 0; c < 3; ++c) zt[c] += dts * gt[c];
            const double zn = dot3(zt, n);
            for (int c = 0; c < 3; ++c) zt[c] -= zn * n[c];
            /* Luding: keep the spring on the Coulomb limit while slipping */
            const double mp = orc_mass(d[p], rho[p]), mq = orc_mass(d[q], rho[q]);
            const double m_eff = mp * mq / (mp + mq);
            const double kn = orc_kn(P, m_eff, uin, rho[p], d[p], rho[q], d[q], mp, mq);
            const double dn = -2.0 * m_eff * log(P[2]) / P[6];
            double Fn[3];
            const double ov = pow(-zeta, 1.5);
            for (int c = 0; c < 3; ++c) Fn[c] = -kn * ov * n[c] - dn * gns * n[c];
            const double nu = P[5], le = log(P[2]);
            const double kt = 2.0 * (1.0 - nu) / (2.0 - nu) * kn;
            const double dt = 2.0 * sqrt(m_eff * kt) * (-le) / sqrt(ORC_PI * ORC_PI + le * le);
            double Fdp[3];
            for (int c = 0; c < 3; ++c) Fdp[c] = -kt * zt[c] - dt * gt[c];
            const double fn = sqrt(dot3(Fn, Fn)), fdp = sqrt(dot3(Fdp, Fdp));
            if (!(fdp < P[3] * fn) && fdp > 0.0)
                for (int c = 0; c < 3; ++c) zt[c] = -(P[4] * fn * Fdp[c] / fdp + dt * gt[c]) / kt;
            np2[k] = p;
            nq2[k] = q;
            for (int c = 0; c < 3; ++c) nz2[3 * k + c] = zt[c];
            nu2[k] = uin;
            ++k;
        }
    if (rc == 0) {
        memcpy(hp, np2, sizeof(long) * (size_t)k);
        memcpy(hq, nq2, sizeof(long) * (size_t)k);
        memcpy(hz, nz2, sizeof(double) * 3 * (size_t)k);
        memcpy(hu, nu2, sizeof(double) * (size_t)k);
        *nh = k;
    }
    free(np2);
    free(nq2);
    free(nz2);
    free(nu2);
    return rc;
}

/* n_sub sub-steps of dt / n_sub, each the three-stage predictor-corrector
 * Runge-Kutta update of Sec. 2.2.10 under the constant hydrodynamic loads
 * Fh, Th (may be NULL) and the collision loads.  x, u, om updated in place;
 * history in/out.  Returns 0, or -1 (allocation or history capacity). */
int orc_particle_substeps(long np, const long *dims, const int *scene, const double *P, double dt, int n_sub,
                          const double *Fh, const double *Th, double *x, double *u, double *om, const double *d,
                          const double *rho, long cap, long *nh, long *hp, long *hq, double *hz, double *hu)
{
    const size_t v = 3 * (size_t)(np > 0 ? np : 1);
    double *F0 = calloc(v, sizeof(double)), *T0 = calloc(v, sizeof(double));
    double *F1 = calloc(v, sizeof(double)), *T1 = calloc(v, sizeof(double));
    double *F2 = calloc(v, sizeof(double)), *T2 = calloc(v, sizeof(double));
    double *xt = calloc(v, sizeof(double)), *ut = calloc(v, sizeof(double)), *wt = calloc(v, sizeof(double));
    int rc = (F0 && T0 && F1 && T1 && F2 && T2 && xt && ut && wt) ? 0 : -1;
    const double ds = dt / (double)n_sub;
    for (int s = 0; s < n_sub && rc == 0; ++s) {
        for (int k = 0; k < 3 && rc == 0; ++k) {
            const double a = RK_A[k], g = RK_G[k], z = RK_Z[k];
            orc_collision_forces(np, dims, scene, P, x, u, om, d, rho, *nh, hp, hq, hz, hu, F1, T1);
            if (k == 0)
                for (size_t i = 0; i < v; ++i) F0[i] = T0[i] = 0.0;
            for (long p = 0; p < np; ++p) {
                const double m = orc_mass(d[p], rho[p]), I = m * d[p] * d[p] / 10.0;
                const double gr = 1.0 - P[0] / rho[p];
                for (int c = 0; c < 3; ++c) {
                    const long i = 3 * p + c;
                    const double fh = Fh ? Fh[i] : 0.0, th = Th ? Th[i] : 0.0;
                    ut[i] = u[i] + ds / m * (2.0 * a * fh + g * F1[i] + z * F0[i]) + 2.0 * a * ds * gr * P[11 + c];
                    wt[i] = om[i] + ds / I * (2.0 * a * th + g * T1[i] + z * T0[i]);
                    xt[i] = x[i] + a * ds * (ut[i] + u[i]);
                }
            }
            orc_collision_forces(np, dims, scene, P, xt, ut, wt, d, rho, *nh, hp, hq, hz, hu, F2, T2);
            for (long p = 0; p < np; ++p) {
                const double m = orc_mass(d[p], rho[p]), I = m * d[p] * d[p] / 10.0;
                const double gr = 1.0 - P[0] / rho[p];
                for (int c = 0; c < 3; ++c) {
                    const long i = 3 * p + c;
                    const double fh = Fh ? Fh[i] : 0.0, th = Th ? Th[i] : 0.0;
                    const double uo = u[i];
                    u[i] = uo + ds / m * (2.0 * a * fh + g * F2[i] + z * F1[i]) + 2.0 * a * ds * gr * P[11 + c];
                    om[i] = om[i] + ds / I * (2.0 * a * th + g * T2[i] + z * T1[i]);
                    x[i] = x[i] + a * ds * (u[i] + uo);
                }
            }
            rc = history_update(np, dims, scene, P, x, u, om, d, rho, 2.0 * a * ds, cap, nh, hp, hq, hz, hu);
            memcpy(F0, F1, v * sizeof(double));
            memcpy(T0, T1, v * sizeof(double));
        }
    }
    free(F0); free(T0); free(F1); free(T1); free(F2); free(T2); free(xt); free(ut); free(wt);
    return rc;
}
