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


def test_coupled_time_step_matches_oracles(oracles):
    F, O = oracles
    dims = (32, 32, 32)
    shape = (32, 32, 32)
    h, nu, dt, rho_f, n_sub = 1.0, 0.05, 0.2, 1.0, 15
    g = (0.0, 0.0, -0.01)
    x = np.array([[9.3, 10.1, 16.4], [20.2, 21.7, 15.1], [15.6, 8.4, 25.9]])
    up = np.array([[0.02, 0.0, -0.01], [-0.01, 0.03, 0.0], [0.0, -0.02, 0.01]])
    om = np.array([[0.0, 0.01, 0.0], [0.005, 0.0, 0.0], [0.0, 0.0, -0.01]])
    d = np.array([8.0, 7.0, 6.0])
    rho = np.array([1.5, 2.0, 1.8])
    u0 = _field(shape, 3)

    # GPU: fluid solver + FP64 IBM context + sub-steps on the same context
    fl = ibm.Fluid(dims, h=h, nu=nu)
    Fd = ibm.FluidFields(dims, u0)
    ctx = gpu_context([dims], 3, ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN, rho_f=rho_f, g=g)
    ctx.set_particles(x, up, om, d, rho)
    prm = ibm.CollisionParams(rho_f=rho_f, nu_f=nu, g=g)
    for k in range(3):
        fl.stage(k, dt, Fd, ctx=ctx)
        loads = ctx.particle_loads(device=True)
        Fh = (-rho_f * loads["F"]).contiguous()
        Th = (-rho_f * loads["T"]).contiguous()
        ctx.particle_substeps(prm, 2 * ALPHA[k] * dt, n_sub, F_h=Fh, T_h=Th)
    torch.cuda.synchronize()
    xg, ug, wg = ctx.particle_state()

    # oracles
    st = F.FluidState(u0, h=h)
    P = O.collision_params(rho_f=rho_f, nu_f=nu, g=g)
    hist = O.PairHistory()
    xo, uo, wo = x.copy(), up.copy(), om.copy()
    for k in range(3):
        r = F.stage(st, k, dt, nu, particles=dict(x=xo, u=uo, om=wo, d=d))
        xo, uo, wo, hist = O.particle_substeps(P, [dims], xo, uo, wo, d, rho, 2 * ALPHA[k] * dt, n_sub=n_sub,
                                               F_h=-rho_f * r["F"], T_h=-rho_f * r["T"], hist=hist)

    su = np.abs(st.u).max()
    assert np.abs(Fd.u.cpu().numpy() - st.u).max() <= TOL * su
    assert np.abs(Fd.uf.cpu().numpy() - st.uf).max() <= TOL * su
    # the particles moved and turned, and both sides agree
    assert np.abs(xo - x).max() > 1e-4 and np.abs(wo - om).max() > 1e-6
    assert np.abs(xg - xo).max() <= TOL * np.abs(xo).max()
    assert np.abs(ug - uo).max() <= TOL * 10 * np.abs(uo).max()
    assert np.abs(wg - wo).max() <= TOL * 10 * np.abs(wo).max()
