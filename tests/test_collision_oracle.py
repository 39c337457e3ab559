"""Pins of the collision oracle (Sec. 2.2.6-2.2.8, Eq. f_int) and of its RK3
particle sub-stepping (Sec. 2.2.10), CPU only.  Each pin checks the oracle
against what the physics or the paper fixes, not against its own formulas:

  * Hertz law: at rest the contact force is central, grows as overlap^{3/2}
    and acts equal and opposite on the two particles;
  * the lubrication blend: the Cox-Brenner force 6 pi rho_f nu_f R_eff^2 g_n /
    zeta well inside eps_sep, saturation below zeta_min, a continuous fade to
    almost nothing just inside eps_sep and none beyond;
  * the stick/slip switch: a small spring gives the spring-dashpot force, a
    large one the Coulomb force mu_k |F_n| opposing the spring;
  * pairwise balance: for a random jammed configuration the collision forces
    sum to zero and so do the moments about the origin (contact-point lever
    arms), whatever the history;
  * free flight: with no contact the sub-steps reproduce x0 + u0 t + 1/2 a t^2
    exactly for a constant acceleration (gravity and a hydrodynamic load);
  * head-on impact in vacuum: the contact lasts T_c (the defining property of
    the ACTM stiffness), the rebound speed approaches e_dry u_in under step
    refinement, and the scheme as printed converges at first order in the step.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O


@pytest.fixture(scope="module", autouse=True)
def _build():
    O.build()


def _P(**kw):
    return O.collision_params(**kw)


def test_hertz_force_law_at_rest():
    P = _P(nu_f=0.0)
    z3 = np.zeros(3)
    forces = []
    for ov in (0.01, 0.04, 0.09):
        dv = np.array([4.0 - ov, 0.0, 0.0])        # two D = 4 spheres overlapping by ov
        # at rest in vacuum the stiffness comes from the recorded impact speed
        Fp, Tp, zp = O.pair_force(P, dv, z3, z3, z3, z3, 4.0, 4.0, 2.0, 2.0, uin=0.5)
        Fq, Tq, zq = O.pair_force(P, -dv, z3, z3, z3, z3, 4.0, 4.0, 2.0, 2.0, uin=0.5)
        assert zp == pytest.approx(-ov) and zq == pytest.approx(-ov)
        assert Fp[0] < 0.0 and np.all(Fp[1:] == 0.0)            # pushes p away from q
        assert np.array_equal(Fq, -Fp)
        assert np.all(Tp == 0.0) and np.all(Tq == 0.0)
        forces.append(-Fp[0])
    # F proportional to overlap^{3/2}
    assert forces[1] / forces[0] == pytest.approx(4.0 ** 1.5, rel=1e-12)
    assert forces[2] / forces[0] == pytest.approx(9.0 ** 1.5, rel=1e-12)


def test_lubrication_blend_limits():
    rho_f, nu_f, h = 1.0, 0.02, 1.0
    P = _P(rho_f=rho_f, nu_f=nu_f, zeta_min=0.01)
    z3 = np.zeros(3)
    Rp, Rq = 3.0, 2.0
    R_eff = Rp * Rq / (Rp + Rq)
    gn = 0.3                                         # approach speed along n
    up, uq = np.array([gn, 0.0, 0.0]), z3

    def force(zeta):
        dv = np.array([Rp + Rq + zeta, 0.0, 0.0])
        F, T, z = O.pair_force(P, dv, up, uq, z3, z3, 2 * Rp, 2 * Rq, 2.0, 2.0)
        assert np.all(T == 0.0) and np.all(F[1:] == 0.0)
        return -F[0]

    for zeta in (0.02, 0.05, 0.1):                   # the blend is 1 to within 1e-13 here
        cox = 6 * math.pi * rho_f * nu_f * R_eff ** 2 * gn / zeta
        assert force(zeta) == pytest.approx(cox, rel=1e-12)
    assert force(0.005) == pytest.approx(force(0.01), rel=1e-14)     # saturates below zeta_min
    # continuous fade: just inside eps_sep = 1.5 h the blend is 0.5 erfc(2.25)
    near = force(1.5 - 1e-9)
    cox = 6 * math.pi * rho_f * nu_f * R_eff ** 2 * gn / 1.5
    assert near == pytest.approx(cox * 0.5 * math.erfc(2.25), rel=1e-6)
    assert near < 1e-3 * cox
    assert force(1.5) == 0.0 and force(2.0) == 0.0
    # separating particles are pulled together (the force opposes g_n)
    dv = np.array([Rp + Rq + 0.2, 0.0, 0.0])
    F, _, _ = O.pair_force(P, dv, -up, uq, z3, z3, 2 * Rp, 2 * Rq, 2.0, 2.0)
    assert F[0] > 0.0


def test_stick_slip_switch():
    P = _P(nu_f=0.0, mu_s=0.4, mu_k=0.3)
    z3 = np.zeros(3)
    dv = np.array([4.0 - 0.05, 0.0, 0.0])
    F0, _, _ = O.pair_force(P, dv, z3, z3, z3, z3, 4.0, 4.0, 2.0, 2.0, uin=0.5)
    fn = abs(F0[0])
    # tangential spring along y, particles at rest: F_t = -k_t zeta_t while sticking
    small = np.array([0.0, 1e-6, 0.0])
    Fs, Ts, _ = O.pair_force(P, dv, z3, z3, z3, z3, 4.0, 4.0, 2.0, 2.0, zt=small, uin=0.5)
    kt = -Fs[1] / small[1]
    assert kt > 0.0 and abs(Fs[1]) < 0.4 * fn
    assert Fs[1] == pytest.approx(-kt * small[1], rel=1e-12)
    Fs2, _, _ = O.pair_force(P, dv, z3, z3, z3, z3, 4.0, 4.0, 2.0, 2.0, zt=2 * small, uin=0.5)
    assert Fs2[1] == pytest.approx(2 * Fs[1], rel=1e-12)            # linear spring while sticking
    # torque of the tangential force about p's centre: lever R_p,cp n
    assert Ts[2] == pytest.approx(0.5 * (4.0 - 0.05) * Fs[1], rel=1e-12)
    # a spring beyond the static limit: Coulomb force mu_k |F_n| opposing it
    big = np.array([0.0, 10 * 0.4 * fn / kt, 0.0])
    Fb, _, _ = O.pair_force(P, dv, z3, z3, z3, z3, 4.0, 4.0, 2.0, 2.0, zt=big, uin=0.5)
    assert Fb[1] == pytest.approx(-0.3 * fn, rel=1e-12)
    assert Fb[0] == pytest.approx(F0[0], rel=1e-12)


def _jammed(seed=3, n=40, L=40):
    rng = np.random.default_rng(seed)
    x = rng.uniform(10, L - 10, size=(n, 3))
    d = rng.uniform(4.0, 8.0, size=n)
    # pull everything towards the centre so that many pairs touch or nearly touch
    c = x.mean(0)
    x = c + 0.55 * (x - c)
    u = rng.normal(0, 0.3, size=(n, 3))
    om = rng.normal(0, 0.3, size=(n, 3))
    rho = rng.uniform(1.5, 3.0, size=n)
    return (L, L, L), x, u, om, d, rho


def test_pairwise_momentum_and_moment_balance():
    dims, x, u, om, d, rho = _jammed()
    P = _P(nu_f=0.01, g=(0.0, 0.0, -0.1))
    hist = O.PairHistory()
    # run a few sub-steps so that the history holds springs of both regimes
    x1, u1, om1, hist = O.particle_substeps(P, dims, x, u, om, d, rho, 0.02, n_sub=5, hist=hist)
    assert hist.n.value > 10
    Fc, Tc = O.collision_forces(P, dims, x1, u1, om1, d, rho, hist)
    scale = np.abs(Fc).sum()
    assert scale > 0.0
    assert np.abs(Fc.sum(0)).max() <= 1e-12 * scale
    # no pair wraps the period here, so the moments about the origin balance too
    mom = np.cross(x1, Fc).sum(0) + Tc.sum(0)
    assert np.abs(mom).max() <= 1e-11 * scale * np.abs(x1).max()


def test_free_flight_is_exact():
    P = _P(g=(0.1, -0.2, -1.0), rho_f=1.0)
    d = np.array([6.0, 5.0])
    rho = np.array([2.5, 1.6])
    x0 = np.array([[10.0, 10.0, 20.0], [30.0, 30.0, 30.0]])
    u0 = np.array([[0.3, 0.1, 0.0], [-0.2, 0.0, 0.4]])
    w0 = np.array([[0.1, 0.2, 0.3], [0.0, -0.1, 0.0]])
    Fh = np.array([[0.5, 0.0, 0.0], [0.0, 0.2, -0.1]])
    Th = np.array([[0.0, 0.0, 0.7], [0.1, 0.0, 0.0]])
    t = 0.7
    x, u, w, _ = O.particle_substeps(P, (64, 64, 64), x0, u0, w0, d, rho, t, n_sub=15, F_h=Fh, T_h=Th)
    m = rho * np.pi * d ** 3 / 6
    I = m * d ** 2 / 10
    a = Fh / m[:, None] + (1 - 1.0 / rho)[:, None] * np.array([0.1, -0.2, -1.0])
    assert np.allclose(u, u0 + a * t, rtol=0, atol=1e-13)
    assert np.allclose(x, x0 + u0 * t + 0.5 * a * t * t, rtol=0, atol=1e-12)
    assert np.allclose(w, w0 + Th / I[:, None] * t, rtol=0, atol=1e-13)


def _head_on(e, dt, n_sub, t_end=0.25, t_c=0.1):
    P = _P(nu_f=0.0, e_dry=e, t_c=t_c)
    d = np.array([8.0, 8.0])
    rho = np.array([2.0, 2.0])
    x = np.array([[28.0, 32.0, 32.0], [36.05, 32.0, 32.0]])
    u = np.array([[0.5, 0.0, 0.0], [-0.5, 0.0, 0.0]])
    om = np.zeros((2, 3))
    hist = O.PairHistory(10)
    t, t0, t1 = 0.0, None, None
    for _ in range(int(round(t_end / dt))):
        x, u, om, hist = O.particle_substeps(P, (64, 64, 64), x, u, om, d, rho, dt, n_sub=n_sub, hist=hist)
        t += dt
        gap = x[1, 0] - x[0, 0] - 8.0
        if gap <= 0.0 and t0 is None:
            t0 = t
        if t0 is not None and gap > 0.0 and t1 is None:
            t1 = t
    return u[1, 0] - u[0, 0], t1 - t0


def test_head_on_impact_duration_and_restitution():
    for e in (0.97, 0.9):
        rebound, dur = _head_on(e, 0.005, 240)
        assert dur == pytest.approx(0.1, abs=0.006)          # T_c, to the outer step
        assert abs(rebound / e - 1.0) <= 0.02
    # first-order convergence of the scheme as printed (force at the predicted state)
    r1, _ = _head_on(0.9999, 0.005, 15)
    r2, _ = _head_on(0.9999, 0.005, 30)
    r4, _ = _head_on(0.9999, 0.005, 60)
    assert (1 - r1) / (1 - r2) == pytest.approx(2.0, rel=0.1)
    assert (1 - r2) / (1 - r4) == pytest.approx(2.0, rel=0.1)
