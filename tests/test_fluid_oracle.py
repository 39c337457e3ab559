"""Pins of the fluid-solver oracle (Sec. 2.2.1 and 2.2.4, Eq. fluid-solver), CPU
only.  Each pin checks the oracle against something other than its own
formulas:

  * closed forms of the stencils on trigonometric fields: the 7-point
    Laplacian of cos multiplies it by -sum 4 sin^2(kappa h/2)/h^2, a central
    difference of sin gives cos sin(kappa h)/h, and the convective term of a
    three-axis shear flow has one term per component (other wave numbers per
    axis, so a transposed axis fails);
  * brute-force loops on tiny grids: the Helmholtz and Poisson solutions
    satisfy their 7-point equations cell by cell;
  * the projection: after a stage the face velocities are discretely
    divergence-free, and a uniform flow passes through a stage unchanged;
  * the Taylor-Green vortex: decay as exp(-2 nu t), the pressure
    (cos 2x + cos 2y)/4 exp(-4 nu t), second-order convergence of the velocity
    in space (the pressure converges at least as fast), and first order in
    time on a nonlinear flow (the projection as printed is non-incremental;
    an inconsistent set of RK3 coefficients would not converge);
  * with a particle at rest in fluid at rest nothing moves, and a particle
    held in a uniform stream takes momentum out of the fluid at the rate the
    subtracted mean force puts back (the net momentum changes by less than
    1e-5 of the forcing's impulse).
"""
import itertools
import math

import numpy as np
import pytest

from oracle import fluid as F


def _grid(shape, h):
    nz, ny, nx = shape
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) * h, (np.arange(ny) + 0.5) * h, (np.arange(nx) + 0.5) * h,
                          indexing="ij")
    return x, y, z


def test_stencils_on_trigonometric_fields():
    shape, h = (8, 12, 16), 0.7
    x, y, z = _grid(shape, h)
    kx, ky, kz = 2 * math.pi * 3 / (16 * h), 2 * math.pi * 1 / (12 * h), 2 * math.pi * 2 / (8 * h)
    c = np.cos(kx * x + ky * y + kz * z)
    sym = -(4 / h ** 2) * (math.sin(kx * h / 2) ** 2 + math.sin(ky * h / 2) ** 2 + math.sin(kz * h / 2) ** 2)
    assert np.abs(F.lap(c, h) - sym * c).max() <= 1e-12 * abs(sym)
    for d, k, coord in ((0, kx, x), (1, ky, y), (2, kz, z)):
        s = np.sin(k * coord)
        assert np.abs(F.ddx(s, d, h) - np.cos(k * coord) * math.sin(k * h) / h).max() <= 1e-13


def test_convective_term_of_a_three_axis_shear():
    shape, h = (8, 12, 16), 0.5
    x, y, z = _grid(shape, h)
    kx, ky, kz = 2 * math.pi / (16 * h), 2 * 2 * math.pi / (12 * h), 2 * math.pi / (8 * h)
    u = np.stack([np.sin(ky * y), 2.0 * np.sin(kz * z), 3.0 * np.sin(kx * x)])
    N = F.convection(u, h)
    sx, sy, sz = math.sin(kx * h) / h, math.sin(ky * h) / h, math.sin(kz * h) / h
    # u_x depends on y only: N_x = u_y d_y u_x, and so on around the axes
    assert np.abs(N[0] - 2.0 * np.sin(kz * z) * np.cos(ky * y) * sy).max() <= 1e-13
    assert np.abs(N[1] - 3.0 * np.sin(kx * x) * 2.0 * np.cos(kz * z) * sz).max() <= 1e-13
    assert np.abs(N[2] - np.sin(ky * y) * 3.0 * np.cos(kx * x) * sx).max() <= 1e-13


def _lap_loops(a, h):
    nz, ny, nx = a.shape
    out = np.zeros_like(a)
    for k, j, i in itertools.product(range(nz), range(ny), range(nx)):
        s = (a[k, j, (i + 1) % nx] + a[k, j, (i - 1) % nx] + a[k, (j + 1) % ny, i] + a[k, (j - 1) % ny, i]
             + a[(k + 1) % nz, j, i] + a[(k - 1) % nz, j, i] - 6.0 * a[k, j, i])
        out[k, j, i] = s / (h * h)
    return out


def test_solvers_satisfy_their_equations_cell_by_cell():
    rng = np.random.default_rng(1)
    shape, h = (4, 6, 5), 0.3
    b = rng.normal(size=shape)
    x = F.solve_helmholtz(b, 0.04, h)
    assert np.abs(x - 0.04 * _lap_loops(x, h) - b).max() <= 1e-12 * np.abs(b).max()
    b0 = b - b.mean()
    phi = F.solve_poisson(b0, h)
    assert abs(phi.mean()) <= 1e-14
    assert np.abs(_lap_loops(phi, h) - b0).max() <= 1e-11 * np.abs(b0).max()


def _div_loops(uf, h):
    _, nz, ny, nx = uf.shape
    out = np.zeros((nz, ny, nx))
    for k, j, i in itertools.product(range(nz), range(ny), range(nx)):
        out[k, j, i] = (uf[0, k, j, i] - uf[0, k, j, (i - 1) % nx] + uf[1, k, j, i] - uf[1, k, (j - 1) % ny, i]
                        + uf[2, k, j, i] - uf[2, (k - 1) % nz, j, i]) / h
    return out


def test_stage_leaves_faces_divergence_free():
    rng = np.random.default_rng(2)
    shape, h = (6, 8, 10), 0.5
    st = F.FluidState(rng.normal(size=(3,) + shape), rng.normal(size=shape), h=h)
    for k in range(3):
        F.stage(st, k, 0.05, 0.1, theta=1.0)
        assert np.abs(_div_loops(st.uf, h)).max() <= 1e-12 * np.abs(st.uf).max() / h
    # and the cell velocities are the faces' only up to the interpolation: not divergence-free
    assert np.abs(_div_loops(F.faces(st.u), h)).max() > 1e-6


def test_uniform_flow_is_preserved():
    shape, h = (4, 6, 8), 1.0
    U = np.array([0.3, -0.2, 0.7])
    st = F.FluidState(np.broadcast_to(U[:, None, None, None], (3,) + shape), h=h)
    F.step(st, 0.1, 0.05, theta=1.0)
    assert np.abs(st.u - U[:, None, None, None]).max() <= 1e-15
    assert np.abs(st.uf - U[:, None, None, None]).max() <= 1e-15
    assert np.abs(st.P).max() <= 1e-15


def _taylor_green(n, dt, T, nu=0.1, theta=1.0):
    h = 2 * math.pi / n
    shape = (2, n, n)
    x, y, _ = _grid(shape, h)
    u = np.stack([np.sin(x) * np.cos(y), -np.cos(x) * np.sin(y), np.zeros(shape)])
    P = (np.cos(2 * x) + np.cos(2 * y)) / 4
    st = F.FluidState(u, P, h=h)
    for _ in range(int(round(T / dt))):
        F.step(st, dt, nu, theta=theta)
    decay = math.exp(-2 * nu * T)
    err_u = np.abs(st.u - u * decay).max()
    p_exact = P * decay ** 2
    err_p = np.abs((st.P - st.P.mean()) - (p_exact - p_exact.mean())).max()
    return st, err_u, err_p


def test_taylor_green_decay_pressure_and_space_order():
    _, e16, p16 = _taylor_green(16, 0.01, 0.5)
    _, e32, p32 = _taylor_green(32, 0.01, 0.5)
    assert e32 < 2e-3 and p32 < 2e-3
    assert 3.2 < e16 / e32 < 4.8                 # velocity: second order in h
    assert p16 / p32 > 3.2                       # pressure: at least second order


def _abc(n=12):
    h = 2 * math.pi / n
    shape = (n, n, n)
    x, y, z = _grid(shape, h)
    u = np.stack([np.sin(z) + 0.5 * np.cos(y), np.sin(x) + 0.5 * np.cos(z), np.sin(y) + 0.5 * np.cos(x)])
    return u, h


def test_time_order_on_a_nonlinear_flow():
    u0, h = _abc()
    T, nu = 0.4, 0.05

    def run(dt):
        st = F.FluidState(u0, h=h)
        for _ in range(int(round(T / dt))):
            F.step(st, dt, nu, theta=1.0)
        return st.u

    ref = run(0.0025)
    e1 = np.abs(run(0.04) - ref).max()
    e2 = np.abs(run(0.02) - ref).max()
    e3 = np.abs(run(0.01) - ref).max()
    # first order: with theta = 1 the pressure gradient of step (a) is taken out again in step (e), so u*
    # carries none and phi is the whole pressure (a non-incremental projection, O(dt) splitting error);
    # an inconsistent set of RK3 coefficients would not converge at all (ratio near 1)
    assert 1.8 < e1 / e2 < 2.5 and 1.8 < e2 / e3 < 2.5


def test_particle_at_rest_in_fluid_at_rest():
    shape, h = (16, 16, 16), 1.0
    st = F.FluidState(np.zeros((3,) + shape), h=h)
    parts = dict(x=np.array([[8.0, 7.5, 8.3]]), u=np.zeros((1, 3)), om=np.zeros((1, 3)), d=np.array([6.0]))
    r = F.stage(st, 0, 0.1, 0.05, particles=parts)
    assert np.abs(r["F"]).max() == 0.0
    assert np.abs(st.u).max() == 0.0 and np.abs(st.P).max() == 0.0


def test_held_particle_in_a_stream_keeps_net_momentum():
    shape, h = (16, 16, 16), 1.0
    U = np.array([0.2, 0.0, 0.0])
    st = F.FluidState(np.broadcast_to(U[:, None, None, None], (3,) + shape).copy(), h=h)
    parts = dict(x=np.array([[8.2, 7.9, 8.4]]), u=np.zeros((1, 3)), om=np.zeros((1, 3)), d=np.array([6.0]))
    mom0 = st.u.reshape(3, -1).sum(1)
    impulse = 0.0
    for k in range(3):
        r = F.stage(st, k, 0.2, 0.05, particles=parts)
        # the forcing decelerates the fluid at the markers ...
        assert r["f"][0].sum() < 0.0
        impulse += 2 * F.ALPHA[k] * 0.2 * abs(r["f"][0].sum())
    # ... and the subtracted mean force returns that momentum uniformly; what is left is the advective
    # form's own small departure from conservation
    assert impulse > 50.0
    assert np.abs(st.u.reshape(3, -1).sum(1) - mom0).max() <= 1e-5 * impulse
    assert st.u[0].min() < 0.9 * U[0]
