"""One coupled time step of the whole method on the GPU against the oracles:
for each RK3 stage k the fluid stage (Sec. 2.2.4, steps (a)-(i), with the IBM
forcing loop of Sec. 2.2.2 between (a) and (e)), then the particles advanced
over the stage's 2 alpha_k dt by the RK3 sub-steps of Sec. 2.2.10 under the
collision models (Sec. 2.2.6-2.2.8) and the hydrodynamic load of the stage,
F_h = -rho_f sum F dV (the fluid-side loads of the forcing loop, Eq.
basic-particle a, b), so that the next stage forces the fluid at the moved
particles.  Compared after the step: the fluid fields at the solver tolerance
(1e-8 of their scale, as in test_gpu_fluid.py) and the particle state at the
same relative tolerance (the loads inherit the fluid's error).
"""
import numpy as np
import pytest

from tests._helpers import gpu_context

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2109_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2109_03972_gb300 import ibm  # noqa: E402

TOL = 1e-8
ALPHA = (4.0 / 15.0, 1.0 / 15.0, 1.0 / 6.0)


@pytest.fixture(scope="module")
def oracles():
    from oracle import fluid as F
    from oracle import oracle as O
    O.build()
    return F, O


def _field(shape, seed):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    u = np.zeros((3,) + shape)
    for c in range(3):
        for _ in range(4):
            m = rng.integers(-2, 3, size=3)
            u[c] += 0.05 * rng.normal() * np.cos(2 * np.pi * (m[0] * i / nx + m[1] * j / ny + m[2] * k / nz)
                                                 + rng.uniform(0, 2 * np.pi))
    return u


DIMS = (32, 32, 32)
H, NU, DT, RHO_F, N_SUB = 1.0, 0.05, 0.2, 1.0, 15
G = (0.0, 0.0, -0.01)
X0 = np.array([[9.3, 10.1, 16.4], [20.2, 21.7, 15.1], [15.6, 8.4, 25.9]])
UP0 = np.array([[0.02, 0.0, -0.01], [-0.01, 0.03, 0.0], [0.0, -0.02, 0.01]])
OM0 = np.array([[0.0, 0.01, 0.0], [0.005, 0.0, 0.0], [0.0, 0.0, -0.01]])
D = np.array([8.0, 7.0, 6.0])


def _gpu_step(u0, rho, direct):
    """Fluid solver + FP64 IBM context + sub-steps on the same context.  direct: add the rate of
    change of the fluid inside each particle to F_h, T_h (Sec. 2.2.9)."""
    fl = ibm.Fluid(DIMS, h=H, nu=NU)
    Fd = ibm.FluidFields(DIMS, u0)
    ctx = gpu_context([DIMS], 3, ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN, rho_f=RHO_F, g=G)
    ctx.set_particles(X0, UP0, OM0, D, rho)
    prm = ibm.CollisionParams(rho_f=RHO_F, nu_f=NU, g=G)
    for k in range(3):
        if direct:
            i0 = ctx.particle_inertia([Fd.u], device=True)
        fl.stage(k, DT, Fd, ctx=ctx)
        loads = ctx.particle_loads(device=True)
        Fh, Th = -RHO_F * loads["F"], -RHO_F * loads["T"]
        if direct:
            i1 = ctx.particle_inertia([Fd.u], device=True)
            Fh = Fh + RHO_F * (i1["Iu"] - i0["Iu"]) / (2 * ALPHA[k] * DT)
            Th = Th + RHO_F * (i1["Ir"] - i0["Ir"]) / (2 * ALPHA[k] * DT)
        ctx.particle_substeps(prm, 2 * ALPHA[k] * DT, N_SUB, F_h=Fh.contiguous(), T_h=Th.contiguous())
    torch.cuda.synchronize()
    return Fd, ctx.particle_state()


def _oracle_step(F, O, u0, rho, direct):
    st = F.FluidState(u0, h=H)
    P = O.collision_params(rho_f=RHO_F, nu_f=NU, g=G)
    hist = O.PairHistory()
    xo, uo, wo = X0.copy(), UP0.copy(), OM0.copy()
    for k in range(3):
        if direct:
            i0 = O.particle_inertia(st.u, xo, D, h=H)
        r = F.stage(st, k, DT, NU, particles=dict(x=xo, u=uo, om=wo, d=D))
        Fh, Th = -RHO_F * r["F"], -RHO_F * r["T"]
        if direct:
            i1 = O.particle_inertia(st.u, xo, D, h=H)
            Fh = Fh + RHO_F * (i1["Iu"] - i0["Iu"]) / (2 * ALPHA[k] * DT)
            Th = Th + RHO_F * (i1["Ir"] - i0["Ir"]) / (2 * ALPHA[k] * DT)
        xo, uo, wo, hist = O.particle_substeps(P, [DIMS], xo, uo, wo, D, rho, 2 * ALPHA[k] * DT, n_sub=N_SUB,
                                               F_h=Fh, T_h=Th, hist=hist)
    return st, (xo, uo, wo)


def test_coupled_time_step_matches_oracles(oracles):
    F, O = oracles
    x, up, om = X0, UP0, OM0
    rho = np.array([1.5, 2.0, 1.8])
    u0 = _field(DIMS, 3)
    Fd, (xg, ug, wg) = _gpu_step(u0, rho, direct=False)
    st, (xo, uo, wo) = _oracle_step(F, O, u0, rho, direct=False)

    su = np.abs(st.u).max()
    assert np.abs(Fd.u.cpu().numpy() - st.u).max() <= TOL * su
    assert np.abs(Fd.uf.cpu().numpy() - st.uf).max() <= TOL * su
    # the particles moved and turned, and both sides agree
    assert np.abs(xo - x).max() > 1e-4 and np.abs(wo - om).max() > 1e-6
    assert np.abs(xg - xo).max() <= TOL * np.abs(xo).max()
    assert np.abs(ug - uo).max() <= TOL * 10 * np.abs(uo).max()
    assert np.abs(wg - wo).max() <= TOL * 10 * np.abs(wo).max()


def test_neutrally_buoyant_particles_with_the_direct_inertia_term(oracles):
    """rho_p = rho_f, where the rigid-body form of the particle equations is singular
    (m_p (1 - rho_f/rho_p) du_p/dt): the direct form of Sec. 2.2.9 instead, F_h = -rho_f sum F dV +
    rho_f d/dt int u dV (and the same for the torque), the rate of change over each RK3 stage taken
    from the fluid inertia before and after the stage at the stage's particle positions, divided by
    2 alpha_k dt.  The GPU (inertia kernel, fluid stage, sub-steps) against the same composition of
    the oracles; the rate term divides field differences by 2 alpha_k dt >= 0.027, so the particle
    velocities get 1e-6 of their scale."""
    F, O = oracles
    rho = np.full(3, RHO_F)
    u0 = _field(DIMS, 5)
    Fd, (xg, ug, wg) = _gpu_step(u0, rho, direct=True)
    st, (xo, uo, wo) = _oracle_step(F, O, u0, rho, direct=True)
    su = np.abs(st.u).max()
    assert np.abs(Fd.u.cpu().numpy() - st.u).max() <= TOL * su
    assert np.abs(xg - xo).max() <= TOL * np.abs(xo).max()
    assert np.abs(ug - uo).max() <= 1e-6 * np.abs(uo).max()
    assert np.abs(wg - wo).max() <= 1e-6 * np.abs(wo).max()
    # the inertia term matters: without it the oracle's particles end elsewhere
    _, (xn, un, wn) = _oracle_step(F, O, u0, rho, direct=False)
    assert np.abs(un - uo).max() > 1e-3 * np.abs(uo).max()
