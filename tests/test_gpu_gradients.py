"""Gradients on the differentiation workload: periodic 128^3 grid, 150 spheres
D = 16h, n_F = 3, loss L = 1/2 sum_cells w |u^{n_F}|^2 with w ~ U[0,1) per cell.

  * the FP64 adjoint of the library (the loop algebra of Sec. 2.2.2:
    spreading is the D-weighted transpose of interpolation, plus the
    delta-kernel derivative terms for the marker positions) against the
    oracle's FP64 adjoint;
  * central finite differences at eps = 1e-6 of the FP64 forward step through
    the torch.autograd.Function, on entries of u^0 (stencil cells of several
    particles), U_p, omega_p and x_p;
  * the FP32 gradient (FP32 forward in the deterministic cluster mode, FP32
    adjoint) against the FP64 one, norm-wise within 1e-3.
"""
import numpy as np
import pytest

from tests._helpers import f32_round, gpu_context

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2109_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2109_03972_gb300 import ibm, synth  # noqa: E402


@pytest.fixture(scope="module")
def case():
    sc = synth.workload("diff128").scenes[0]
    return sc, sc.field(), synth.loss_weights(sc.dims, 7)


@pytest.fixture(scope="module")
def oracle_mod():
    from oracle import oracle as O
    O.build()
    return O


def _gpu_grads(sc, u0, wgt, precision, mode):
    ctx = gpu_context([sc.dims], sc.n_p, precision, mode, requires_grad=True)
    ctx.set_particles(sc.x_p, sc.u_p, sc.omega_p, sc.d_p)
    dt = torch.float64 if precision == ibm.IBM_FP64 else torch.float32
    u = torch.from_numpy(u0).to(dtype=dt, device="cuda")
    ctx.forcing_step([u], 0.01)
    g = torch.from_numpy(wgt[None]).to(dtype=dt, device="cuda") * u
    gis, gU, gW, gX = ctx.backward([g])
    torch.cuda.synchronize()
    return [t.double().cpu().numpy() for t in (gis[0], gU, gW, gX)]


def test_diff128_fp64_adjoint_matches_oracle(oracle_mod, case):
    sc, u0, wgt = case
    ref_u = oracle_mod.forcing_step(u0, sc.x_p, sc.u_p, sc.omega_p, sc.d_p, n_forcing=3, tau=0.01)["u"]
    gi, gU, gW, gX = oracle_mod.backward(u0, sc.x_p, sc.u_p, sc.omega_p, sc.d_p, wgt[None] * ref_u)
    got = _gpu_grads(sc, u0, wgt, ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN)
    assert np.abs(got[0] - gi).max() <= 1e-11 * np.abs(gi).max()
    for a, b in zip(got[1:], (gU, gW, gX)):
        assert np.abs(a - b).max() <= 1e-10 * max(1.0, np.abs(b).max())


def test_diff128_finite_differences(oracle_mod, case):
    sc, u0, wgt = case
    ctx = gpu_context([sc.dims], sc.n_p, ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN, requires_grad=True)
    w = torch.from_numpy(wgt[None]).cuda()
    dev = dict(device="cuda", dtype=torch.float64)
    up = torch.tensor(sc.u_p, **dev, requires_grad=True)
    om = torch.tensor(sc.omega_p, **dev, requires_grad=True)
    xp = torch.tensor(sc.x_p, **dev, requires_grad=True)
    d = torch.tensor(sc.d_p, **dev)
    uu = torch.from_numpy(u0).cuda().requires_grad_(True)

    def field(uu, up, om, xp):
        return ibm.IBMForcing.apply(uu, up, om, xp, d, ctx, 0.01)

    out = field(uu, up, om, xp)
    (0.5 * (w * out * out).sum()).backward()
    eps = 1e-6
    # u^0 entries: stencil cells of markers of three particles (where the loop
    # couples cells), one per velocity component
    _, base = oracle_mod.marker_positions(sc.x_p, sc.d_p)
    nx, ny, nz = sc.dims
    probes_u = []
    for q, m in enumerate((10, 20000, 90000)):
        b = base[m]
        probes_u.append((q, int(b[2] % nz), int(b[1] % ny), int(b[0] % nx)))
    probes_u.append((1, 3, 5, 7))                          # a cell no stencil reaches: dL/du^0 = w u^0
    cases = [(uu, uu.grad, idx, 1e-6) for idx in probes_u]
    for t, tol in ((up, 1e-6), (om, 1e-6), (xp, 1e-5)):
        for idx in ((0, 0), (57, 1), (149, 2)):
            cases.append((t, t.grad, idx, tol))
    for t, grad, idx, tol in cases:
        with torch.no_grad():
            t[idx] += eps
            fp = field(uu, up, om, xp)
            t[idx] -= 2 * eps
            fm = field(uu, up, om, xp)
            t[idx] += eps
            # L(+) - L(-) = 1/2 sum w (u+ - u-)(u+ + u-): no cancellation in L itself
            fd = (0.5 * (w * (fp - fm) * (fp + fm)).sum()).item() / (2 * eps)
        scale = max(1.0, grad.abs().max().item())
        assert abs(fd - grad[idx].item()) <= tol * scale, (idx, fd, grad[idx].item())


def test_diff128_fp32_gradient_vs_fp64(case):
    sc, u0, wgt = case
    u0 = f32_round(u0)
    g64 = _gpu_grads(sc, u0, wgt, ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN)
    g32 = _gpu_grads(sc, u0, wgt, ibm.IBM_FP32, ibm.IBM_SPREAD_DETERMINISTIC)
    for a, b in zip(g32, g64):
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b)
