"""FP64 CPU oracle of the collocated fractional-step fluid solver that carries
the direct-forcing IBM (Sec. 2.2.1 and 2.2.4: the Zang et al. pressure-momentum
coupling and the modified solver, Eq. fluid-solver (a)-(i)), on a triply
periodic grid.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use this module; the GPU library never does.  It shares no
code with the library.  The IBM forcing loop it calls is the C oracle's
(``oracle.forcing_step``).

Grid: nx*ny*nz cells of spacing h, cell (i,j,k) centred at ((i+1/2)h, ...),
scalar fields [nz][ny][nx] (x fastest), vector fields [3][nz][ny][nx].  The
face value uf[d][k][j][i] sits on the face between cell i and cell i+1 along
axis d (its "upper" face).

Readings (the paper names the scheme and its order, not each stencil):
  * u.grad(u) in advective form, each derivative a central difference
    (second order on the collocated grid, step (a));
  * the Laplacian is the compact 7-point stencil, for u and for phi;
  * grad P and grad phi at cell centres are central differences; the face
    gradient (grad phi)_f is the compact difference across the face, so that
    the face correction makes div u_f vanish with the 7-point Poisson operator;
  * the interpolation I of step (f) is linear: the mean of the two cells;
  * div u_f at a cell is the sum of its face fluxes over h;
  * the forcing loop updates u~ in place to u~ + 2 alpha dt f_IBM (its f_out
    is f_IBM), so step (e)'s right-hand side is that field minus
    2 alpha dt f_mean, with f_mean the volume average of f_IBM (the aperiodic
    pressure gradient of Sec. 2.2.4, subtracted so the net forcing vanishes);
  * the implicit viscous equation of step (e) and the Poisson equation of
    step (g) are solved exactly by diagonalising the periodic 7-point
    Laplacian with the FFT (a library step); phi has zero mean;
  * theta = 0 (projection) keeps P at its initial value, theta = 1 (pressure
    correction) sets P = phi - alpha dt nu lap(phi), as printed in step (i).

Parity: pinned in tests/test_fluid_oracle.py by closed forms of the
stencils on trigonometric fields, brute-force loops on tiny grids, the
discrete divergence of the corrected face velocities, uniform-flow
preservation, the Taylor-Green vortex (decay rate, pressure, second-order
convergence in space) and first-order convergence in time on a nonlinear
flow (the projection as printed is non-incremental).
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

# the low-storage RK3 of Rai and Moin that Sec. 2.1 names: alpha_k, gamma_k, zeta_k (their published values)
ALPHA = (4.0 / 15.0, 1.0 / 15.0, 1.0 / 6.0)
GAMMA = (8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0)
ZETA = (0.0, -17.0 / 60.0, -5.0 / 12.0)


def _ax(d: int) -> int:
    """Array axis of direction d (0 = x, 1 = y, 2 = z) in a [nz][ny][nx] field."""
    return 2 - d


def shift(a, d, s):
    """a at the cell s steps along direction d (periodic): shift(a, d, 1)[i] = a[i+1]."""
    return np.roll(a, -s, axis=_ax(d))


def lap(a, h):
    """Compact 7-point Laplacian of a scalar field."""
    out = -6.0 * a
    for d in range(3):
        out = out + shift(a, d, 1) + shift(a, d, -1)
    return out / (h * h)


def ddx(a, d, h):
    """Central difference along direction d at cell centres."""
    return (shift(a, d, 1) - shift(a, d, -1)) / (2.0 * h)


def convection(u, h):
    """(u . grad) u in advective form, component c = sum_d u_d d(u_c)/dx_d."""
    return np.stack([sum(u[d] * ddx(u[c], d, h) for d in range(3)) for c in range(3)])


def faces(u):
    """Linear interpolation of the cell velocities to the faces (step (f))."""
    return np.stack([0.5 * (u[d] + shift(u[d], d, 1)) for d in range(3)])


def divergence(uf, h):
    """Net outflow of the face velocities of each cell over h."""
    return sum(uf[d] - shift(uf[d], d, -1) for d in range(3)) / h


def face_gradient(phi, d, h):
    """(grad phi)_f on the upper face along d: compact difference across it."""
    return (shift(phi, d, 1) - phi) / h


def lap_symbol(shape, h):
    """Eigenvalues of the periodic 7-point Laplacian on the FFT grid of a
    [nz][ny][nx] field: sum_d (2 cos(2 pi m_d / N_d) - 2) / h^2 (all <= 0)."""
    nz, ny, nx = shape
    lz = 2.0 * np.cos(2.0 * np.pi * np.arange(nz) / nz) - 2.0
    ly = 2.0 * np.cos(2.0 * np.pi * np.arange(ny) / ny) - 2.0
    lx = 2.0 * np.cos(2.0 * np.pi * np.arange(nx) / nx) - 2.0
    return (lz[:, None, None] + ly[None, :, None] + lx[None, None, :]) / (h * h)


def solve_helmholtz(rhs, c, h):
    """x with x - c lap(x) = rhs (c >= 0), exactly via the FFT."""
    lam = lap_symbol(rhs.shape, h)
    return np.real(np.fft.ifftn(np.fft.fftn(rhs) / (1.0 - c * lam)))


def solve_poisson(rhs, h):
    """phi with lap(phi) = rhs - mean(rhs) and mean(phi) = 0, via the FFT."""
    lam = lap_symbol(rhs.shape, h)
    R = np.fft.fftn(rhs)
    lam[0, 0, 0] = 1.0
    X = R / lam
    X[0, 0, 0] = 0.0
    return np.real(np.fft.ifftn(X))


def predictor(u, P, N_old, k, dt, nu, h):
    """Step (a): u~ = u + dt (2 alpha nu lap u - 2 alpha grad P - gamma N(u) - zeta N_old).
    Returns (u~, N(u)); N(u) is the next stage's N_old."""
    a, g, z = ALPHA[k], GAMMA[k], ZETA[k]
    N = convection(u, h)
    ut = np.empty_like(u)
    for c in range(3):
        ut[c] = u[c] + dt * (2.0 * a * nu * lap(u[c], h) - 2.0 * a * ddx(P, c, h) - g * N[c] - z * N_old[c])
    return ut, N


def corrector(ut, u_old, P, mean_f, k, dt, nu, theta, h):
    """Steps (e)-(i) from the forced field u~_F = u~ + 2 alpha dt f_IBM.
    Returns dict(u, uf, P, phi, ustar)."""
    a = ALPHA[k]
    cv = a * dt * nu
    mean_f = np.zeros(3) if mean_f is None else np.asarray(mean_f, float)
    ustar = np.empty_like(ut)
    for c in range(3):
        rhs = ut[c] - 2.0 * a * dt * mean_f[c] - cv * lap(u_old[c], h) + 2.0 * a * theta * dt * ddx(P, c, h)
        ustar[c] = solve_helmholtz(rhs, cv, h)                      # (e)
    ufs = faces(ustar)                                              # (f)
    phi = solve_poisson(divergence(ufs, h) / (2.0 * a * dt), h)     # (g)
    u = np.stack([ustar[c] - 2.0 * a * dt * ddx(phi, c, h) for c in range(3)])       # (h)
    uf = np.stack([ufs[d] - 2.0 * a * dt * face_gradient(phi, d, h) for d in range(3)])
    Pn = (1.0 - theta) * P + theta * (phi - a * dt * nu * lap(phi, h))                # (i)
    return {"u": u, "uf": uf, "P": Pn, "phi": phi, "ustar": ustar}


class FluidState:
    """u, P and the previous stage's convective term of a periodic grid."""

    def __init__(self, u, P=None, h=1.0):
        self.u = np.array(u, dtype=np.float64)
        self.P = np.zeros(self.u.shape[1:]) if P is None else np.array(P, dtype=np.float64)
        self.N_old = np.zeros_like(self.u)
        self.uf = faces(self.u)
        self.phi = np.zeros_like(self.P)
        self.h = h


def stage(st: FluidState, k, dt, nu, theta=1.0, particles=None, n_forcing=3, width=3):
    """One RK3 stage k (0, 1, 2) of the modified solver with the IBM forcing
    loop between steps (a) and (e).  particles: None or dict(x, u, om, d).
    Returns the forcing loop's dict (u, F, T, f) or None; updates st."""
    a = ALPHA[k]
    ut, N = predictor(st.u, st.P, st.N_old, k, dt, nu, st.h)
    forcing = None
    mean_f = None
    if particles is not None and len(particles["d"]) > 0:
        forcing = O.forcing_step(ut, particles["x"], particles["u"], particles["om"], particles["d"],
                                 h=st.h, n_forcing=n_forcing, tau=2.0 * a * dt, width=width,
                                 want_f=True, want_slip=False)
        ut = forcing["u"]
        mean_f = forcing["f"].reshape(3, -1).mean(axis=1)
    r = corrector(ut, st.u, st.P, mean_f, k, dt, nu, theta, st.h)
    st.u, st.uf, st.P, st.phi, st.N_old = r["u"], r["uf"], r["P"], r["phi"], N
    return forcing


def step(st: FluidState, dt, nu, theta=1.0, particles=None, n_forcing=3, width=3):
    """A full time step: the three RK3 stages, particles held fixed."""
    for k in range(3):
        stage(st, k, dt, nu, theta, particles, n_forcing, width)
