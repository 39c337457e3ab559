"""GPU parity of the collocated fractional-step fluid solver (Sec. 2.2.1 and 2.2.4,
steps (a)-(i) of Eq. fluid-solver) with the FP64 oracle, through the C ABI.

The oracle solves the implicit viscous step and the Poisson equation exactly
(FFT); the library by multigrid to a relative max-norm residual rtol.  The
error that leaves in a solution is at most |A^-1| |r| <= rtol max|b| /
lambda_min with lambda_min = 4 sin^2(pi / N_max) / h^2 the smallest non-zero
eigenvalue of the periodic 7-point operator, i.e. rtol * 12 / lambda_min * h^-2
relative to the solution's scale (about 1e-9 at rtol = 1e-12 on 64 cells); the
tolerance below, 1e-8 of each field's scale, covers that with a margin for the
three stages.  phi and P are compared without their means (the operator's null
space).
"""
import math

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


@pytest.fixture(scope="module")
def F_or():
    from oracle import fluid as F
    from oracle import oracle as O
    O.build()
    return F


def _smooth_random(shape, seed, modes=6, amp=1.0):
    """A random periodic field of a few low Fourier modes per component, [3][nz][ny][nx]."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = np.zeros((3,) + shape)
    for c in range(3):
        for _ in range(modes):
            m = rng.integers(-3, 4, size=3)
            ph = rng.uniform(0, 2 * np.pi)
            out[c] += amp * rng.normal() * np.cos(2 * np.pi * (m[0] * i / nx + m[1] * j / ny + m[2] * k / nz) + ph)
    return out


def _compare(fl_fields, st, what=""):
    u = fl_fields.u.cpu().numpy()
    uf = fl_fields.uf.cpu().numpy()
    P = fl_fields.p.cpu().numpy()
    phi = fl_fields.phi.cpu().numpy()
    su = max(np.abs(st.u).max(), 1e-30)
    assert np.abs(u - st.u).max() <= TOL * su, what
    assert np.abs(uf - st.uf).max() <= TOL * su, what
    sp = max(np.abs(st.phi).max(), 1e-30)
    assert abs(phi.mean()) <= 1e-12 * sp
    assert np.abs((phi - phi.mean()) - (st.phi - st.phi.mean())).max() <= TOL * sp, what
    sP = max(np.abs(st.P - st.P.mean()).max(), 1e-30)
    assert np.abs((P - P.mean()) - (st.P - st.P.mean())).max() <= TOL * sP, what


@pytest.mark.parametrize("dims,theta", [((24, 20, 16), 1.0), ((32, 32, 32), 0.0), ((16, 12, 10), 1.0)])
def test_fluid_stages_match_oracle(F_or, dims, theta):
    # (24, 20, 16): levels 24x20x16, 12x10x8, 6x5x4 (odd: conjugate gradients on 120 cells);
    # (32, 32, 32): down to 2x2x2; (16, 12, 10): 8x6x5 coarsest
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    h, nu, dt = 0.5, 0.05, 0.02
    u0 = _smooth_random(shape, 1)
    P0 = _smooth_random(shape, 2)[0]
    st = F_or.FluidState(u0, P0, h=h)
    fl = ibm.Fluid(dims, h=h, nu=nu, theta=theta)
    Fd = ibm.FluidFields(dims, u0, P0)
    for step in range(2):
        for k in range(3):
            F_or.stage(st, k, dt, nu, theta=theta)
            fl.stage(k, dt, Fd)
            torch.cuda.synchronize()
            _compare(Fd, st, f"step {step} stage {k}")
            s = fl.stats()
            assert max(s["resid"]) <= 1e-12
    assert fl.stats()["levels"] >= 2


def test_predict_and_correct_separately_with_a_mean_force(F_or):
    # the split entry points with a host and a device mean force give the composite's results
    dims = (16, 16, 16)
    shape = (16, 16, 16)
    h, nu, dt = 1.0, 0.02, 0.1
    u0 = _smooth_random(shape, 3)
    st = F_or.FluidState(u0, h=h)
    fl = ibm.Fluid(dims, h=h, nu=nu)
    Fd = ibm.FluidFields(dims, u0)
    mf = np.array([0.01, -0.02, 0.005])
    for k in range(3):
        ut, N = F_or.predictor(st.u, st.P, st.N_old, k, dt, nu, h)
        r = F_or.corrector(ut, st.u, st.P, mf, k, dt, nu, 1.0, h)
        st.u, st.uf, st.P, st.phi, st.N_old = r["u"], r["uf"], r["P"], r["phi"], N
        fl.predict(k, dt, Fd)
        torch.cuda.synchronize()
        # step (a): in the first stage only rounding (FMA contraction, summation order) separates the two;
        # later stages start from u that carries the solves' tolerance
        tol = 1e-12 if k == 0 else TOL
        assert np.abs(Fd.ut.cpu().numpy() - ut).max() <= tol * np.abs(ut).max()
        fl.correct(k, dt, Fd, mean_f=mf if k != 1 else torch.tensor(mf, device="cuda"))
        torch.cuda.synchronize()
        _compare(Fd, st, f"stage {k}")


def _particles(dims, seed, n=3, d=(6.0, 8.0)):
    rng = np.random.default_rng(seed)
    L = np.array(dims, float)
    x = rng.uniform(0.2, 0.8, size=(n, 3)) * L
    x[1] = x[0] + np.array([d[1] + 2.0, 0.5, -0.3])      # two spheres 2 h apart
    u = rng.normal(0, 0.2, size=(n, 3))
    om = rng.normal(0, 0.05, size=(n, 3))
    dp = rng.uniform(*d, size=n)
    return x % L, u, om, dp


def test_stage_with_ibm_forcing_matches_oracle(F_or):
    dims = (32, 32, 32)
    shape = (32, 32, 32)
    h, nu, dt = 1.0, 0.05, 0.2
    u0 = 0.1 * _smooth_random(shape, 4)
    x, up, om, dp = _particles(dims, 5)
    parts = dict(x=x, u=up, om=om, d=dp)
    st = F_or.FluidState(u0, h=h)
    fl = ibm.Fluid(dims, h=h, nu=nu)
    Fd = ibm.FluidFields(dims, u0)
    ctx = gpu_context([dims], len(dp), ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN)
    ctx.set_particles(x, up, om, dp)
    f_out = torch.zeros((3,) + shape, dtype=torch.float64, device="cuda")
    for k in range(3):
        r = F_or.stage(st, k, dt, nu, particles=parts)
        fl.stage(k, dt, Fd, ctx=ctx, f_out=f_out)
        torch.cuda.synchronize()
        assert np.abs(f_out.cpu().numpy() - r["f"]).max() <= 1e-9 * np.abs(r["f"]).max()
        Fg = ctx.particle_loads()["F"]
        assert np.abs(Fg - r["F"]).max() <= 1e-9 * np.abs(r["F"]).max()
        _compare(Fd, st, f"stage {k}")


def test_stage_is_bit_reproducible():
    dims = (32, 32, 64)
    u0 = _smooth_random((64, 32, 32), 7)
    out = []
    for _ in range(2):
        fl = ibm.Fluid(dims, h=1.0, nu=0.01)
        Fd = ibm.FluidFields(dims, u0)
        fl.step(0.1, Fd)
        torch.cuda.synchronize()
        out.append([t.cpu().numpy() for t in (Fd.u, Fd.uf, Fd.p, Fd.phi)])
    for a, b in zip(*out):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("dims", [(64, 48, 40), (96, 40, 66)])
def test_fused_sweeps_equal_two_half_sweeps(dims):
    # the one-pass red-black sweep (tiles with a 2-cell halo, 32-plane chunks; ragged tiles and chunks here)
    # gives the two half sweeps' results bit for bit
    nx, ny, nz = dims
    u0 = _smooth_random((nz, ny, nx), 11)
    out = []
    for two in (False, True):
        fl = ibm.Fluid(dims, h=1.0, nu=0.3, two_pass_smoother=two)
        Fd = ibm.FluidFields(dims, u0)
        for k in range(3):
            fl.stage(k, 0.2, Fd)
        torch.cuda.synchronize()
        out.append([t.cpu().numpy() for t in (Fd.u, Fd.uf, Fd.p, Fd.phi)] + [fl.stats()["cycles"]])
    for a, b in zip(*out):
        assert np.array_equal(np.asarray(a), np.asarray(b))


def test_cycle_limit_reports_noconvergence():
    dims = (64, 64, 64)
    fl = ibm.Fluid(dims, h=1.0, nu=0.01, rtol=1e-15, max_cycles=1)
    Fd = ibm.FluidFields(dims, _smooth_random((64, 64, 64), 8))
    with pytest.raises(ibm.IBMError) as e:
        fl.stage(0, 0.1, Fd)
    assert e.value.status == 8


def test_large_grid_faces_are_divergence_free_and_momentum_is_kept():
    # a 256 x 256 x 512 grid with a bed of spheres: properties that hold at any size
    dims = (256, 256, 512)
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    rng = np.random.default_rng(9)
    n = 400
    x = rng.uniform(0, 1, size=(n, 3)) * np.array(dims, float)
    up = rng.normal(0, 0.05, size=(n, 3))
    om = np.zeros((n, 3))
    dp = np.full(n, 12.0)
    u0 = torch.zeros((3,) + shape, dtype=torch.float64, device="cuda")
    u0[0] = 0.05
    fl = ibm.Fluid(dims, h=1.0, nu=0.01)
    Fd = ibm.FluidFields(dims)
    Fd.u.copy_(u0)
    ctx = gpu_context([dims], n, ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN)
    ctx.set_particles(x, up, om, dp)
    mom0 = Fd.u.sum(dim=(1, 2, 3))
    for k in range(3):
        fl.stage(k, 0.5, Fd, ctx=ctx)
    torch.cuda.synchronize()
    uf = Fd.uf
    div = (uf[0] - torch.roll(uf[0], 1, 2)) + (uf[1] - torch.roll(uf[1], 1, 1)) + (uf[2] - torch.roll(uf[2], 1, 0))
    assert div.abs().max().item() <= 1e-10 * uf.abs().max().item()
    s = fl.stats()
    assert max(s["resid"]) <= 1e-12 and max(s["cycles"]) <= 30
    # the subtracted mean force keeps the net momentum, up to the advective form's small departure
    dm = (Fd.u.sum(dim=(1, 2, 3)) - mom0).abs().max().item()
    assert dm <= 1e-6 * abs(mom0[0].item())
