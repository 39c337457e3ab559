"""GPU parity of the grid-pass mean IBM force (Sec. 2.2.4, Eq. fe_IBM) against
the oracle's plain definition on the same fields.

Tolerances: the oracle sums in FP64.  The library adds FP32 fields in groups
of at most 16 values in FP32 (relative rounding <= 15 * 2^-24 of the group's
sum of |f|) and the groups in FP64, so
  FP32: |fbar - fbar_oracle| <= 1e-6 sum|f| / N;   FP64: <= 1e-12 sum|f| / N.
"""
import numpy as np
import pytest

from tests._helpers import gpu_context, run_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2109_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2109_03972_gb300 import ibm, synth  # noqa: E402

TOL = {ibm.IBM_FP32: 1e-6, ibm.IBM_FP64: 1e-12}


@pytest.fixture(scope="module")
def oracle_mod():
    from oracle import oracle as O
    O.build()
    return O


def _check(O, fbar, fields, prec):
    for s, f in enumerate(fields):
        f64 = f.double().cpu().numpy()
        ref = O.mean_force(f64)
        bound = TOL[prec] * np.abs(f64).sum() / f64[0].size + 1e-300
        assert np.abs(fbar[s] - ref).max() <= bound, (s, fbar[s], ref)


@pytest.mark.parametrize("prec", [ibm.IBM_FP32, ibm.IBM_FP64])
def test_mean_force_ragged_scenes(oracle_mod, prec):
    # grids whose cell counts are not multiples of 4 (component arrays off the
    # 16-byte boundary), one smaller than a segment, one spanning several
    # segments with a ragged last one
    dims = [(8, 9, 11), (33, 35, 37), (64, 64, 64), (96, 72, 41)]
    dt = torch.float64 if prec == ibm.IBM_FP64 else torch.float32
    ctx = gpu_context(dims, 1, prec, ibm.IBM_SPREAD_PLAIN)
    g = torch.Generator(device="cuda").manual_seed(7)
    fields = []
    for k, (nx, ny, nz) in enumerate(dims):
        f = torch.randn((3, nz, ny, nx), generator=g, device="cuda", dtype=torch.float64) + 0.1 * (k + 1)
        fields.append(f.to(dt))
    fbar = ctx.mean_force(fields)
    _check(oracle_mod, fbar, fields, prec)
    again = ctx.mean_force(fields)
    assert np.array_equal(fbar, again)                     # fixed summation order
    dev = ctx.mean_force(fields, device=True).cpu().numpy()
    assert np.array_equal(fbar, dev)


def test_mean_force_of_a_forcing_step(oracle_mod):
    # the f_out of a forcing step: the grid pass against the oracle's grid pass
    # of the oracle's f, and against minus the summed loads / N (the same sum
    # taken over markers instead of cells)
    sc = synth.workload("small").scenes[0]
    u0 = sc.field()
    ref = oracle_mod.forcing_step(u0, sc.x_p, sc.u_p, sc.omega_p, sc.d_p, want_f=True)
    out = run_gpu(sc, u0, ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN, want_f=True)
    f = torch.from_numpy(out["f"]).cuda()
    fbar = out["ctx"].mean_force([f])[0]
    n = f[0].numel()
    scale = np.abs(ref["f"]).sum() / n
    assert np.abs(fbar - oracle_mod.mean_force(ref["f"])).max() <= 1e-12 * scale
    assert np.abs(fbar * n + out["F"].sum(0)).max() <= 1e-12 * n * scale


def test_mean_force_full_bed(oracle_mod):
    # the bidisperse bed's grid (512 x 512 x 1024, FP32, 3.2 GB per field) with
    # the f_out of one deterministic FP32 step: the grid pass against the
    # oracle's definition on the same field, and the identity with the loads
    W = synth.workload("bidisperse")
    sc = W.scenes[0]
    ctx = ibm.Context(ibm.Config(dims=[sc.dims], n_forcing=W.n_forcing, precision=ibm.IBM_FP32,
                                 spread_mode=ibm.IBM_SPREAD_DETERMINISTIC, max_particles=sc.n_p))
    ctx.set_particles(sc.x_p, sc.u_p, sc.omega_p, sc.d_p)
    u = torch.from_numpy(sc.field().astype(np.float32)).cuda()
    f = torch.zeros_like(u)
    ctx.forcing_step([u], W.tau, f_out=[f])
    del u
    F = ctx.particle_loads()["F"]
    fbar = ctx.mean_force([f])[0]
    fh = f.cpu().numpy()
    del f
    n = fh[0].size
    ref = np.zeros(3)
    absum = 0.0
    for q in range(3):                                   # FP64 sums, slab by slab
        for z in range(0, fh.shape[1], 64):
            blk = fh[q, z:z + 64].astype(np.float64)
            ref[q] -= blk.sum()
            absum += np.abs(blk).sum()
    ref /= n
    assert np.abs(fbar - ref).max() <= 1e-6 * absum / n
    # cell sum vs marker sum: FP32 storage of the touched cells separates them
    assert np.abs(fbar * n + F.sum(0)).max() <= 1e-5 * np.abs(F).sum()
