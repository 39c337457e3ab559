"""Markers on and next to cell faces: the stencil base cell is floor(X/h)
(Eq. 3pt-stencil support, cell centres at (i + 1/2)h), and the FP32 path
computes X relative to the particle's base cell in FP32, falling back to the
FP64 position wherever the FP32 value lies within its error bound of a face.
Random placements put only a few markers in that band, so this scene puts
them there on purpose:
  * each particle's centre is shifted so that one chosen marker per axis lies
    within 1e-9 .. 3e-6 cells of a face, on either side;
  * particles of D = 8h (201 markers: marker 100 has z-direction exactly 0)
    sit at integer z, so that marker lies exactly on a face.
Bins must match the oracle bit for bit, and the step must match it at the
FP32 tolerances in every FP32 mode.
"""
import numpy as np
import pytest

from tests._helpers import f32_round, gpu_context, load_err, rel_err_u, run_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2109_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2109_03972_gb300 import ibm, synth  # noqa: E402

U_TOL32, LOAD_TOL32 = 2e-5, 1e-4


@pytest.fixture(scope="module")
def oracle_mod():
    from oracle import oracle as O
    O.build()
    return O


def _near_face_scene(O):
    dims = (64, 60, 56)
    rng = np.random.default_rng(71)
    d = np.array([16.0, 12.0, 12.0, 10.0, 10.0, 8.0, 8.0, 8.0, 8.0, 8.0, 8.0, 8.0])
    # generous gaps, so that moving a centre by less than a cell keeps them apart
    x, d = synth.rsa_spheres(dims, d, seed=73, gap=3.0)
    x = x.copy()
    for p in range(len(d)):
        nl = O.marker_count(d[p])
        t = O.marker_dirs(nl)
        a = 0.5 * d[p]
        for c in range(3):
            if d[p] == 8.0 and c == 2:
                x[p, c] = np.round(x[p, c]) % dims[c]     # marker 100: t_z = 0 exactly
                continue
            for _ in range(50):                           # keep the centre inside [0, L)
                l = rng.integers(nl)
                k = np.round(x[p, c] + a * t[l, c])
                delta = rng.uniform(1e-9, 3e-6) * rng.choice([-1.0, 1.0])
                xn = k - a * t[l, c] + delta
                if 0.0 <= xn < dims[c]:
                    x[p, c] = xn
                    break
    u_p, om, rho = synth.particle_state(len(d), 79)
    return synth.Scene(dims, x, d, u_p, om, rho, field_seed=83)


def _band(O, sc):
    xi, _ = O.marker_positions(sc.x_p, sc.d_p)
    frac = xi - np.floor(xi)
    dist = np.minimum(frac, 1.0 - frac)
    a = np.repeat(0.5 * sc.d_p, [O.marker_count(dd) for dd in sc.d_p])
    return dist, dist < 8.0 * 2.0 ** -24 * (a[:, None] + 2.0)


def test_scene_puts_markers_in_the_fp32_band(oracle_mod):
    sc = _near_face_scene(oracle_mod)
    dist, band = _band(oracle_mod, sc)
    assert band.sum() >= 2 * sc.n_p
    assert (dist == 0.0).sum() >= int((sc.d_p == 8.0).sum())


@pytest.mark.parametrize("precision", [ibm.IBM_FP32, ibm.IBM_FP64])
def test_near_face_bins_bit_exact(oracle_mod, precision):
    sc = _near_face_scene(oracle_mod)
    dist, _ = _band(oracle_mod, sc)
    assert ((dist > 0.0) & (dist < 1e-12)).sum() == 0
    mode = ibm.IBM_SPREAD_PLAIN if precision == ibm.IBM_FP64 else ibm.IBM_SPREAD_DETERMINISTIC
    ctx = gpu_context([sc.dims], sc.n_p, precision, mode)
    ctx.set_particles(sc.x_p, sc.u_p, sc.omega_p, sc.d_p)
    _, base = oracle_mod.marker_positions(sc.x_p, sc.d_p)
    assert np.array_equal(ctx.marker_bases(), base)


@pytest.mark.parametrize("mode", [ibm.IBM_SPREAD_PLAIN, ibm.IBM_SPREAD_CLUSTER, ibm.IBM_SPREAD_DETERMINISTIC])
def test_near_face_step_matches_oracle(oracle_mod, mode):
    sc = _near_face_scene(oracle_mod)
    u0 = f32_round(sc.field())
    ref = oracle_mod.forcing_step(u0, sc.x_p, sc.u_p, sc.omega_p, sc.d_p, n_forcing=3, tau=0.01)
    got = run_gpu(sc, u0, ibm.IBM_FP32, mode)
    assert rel_err_u(got["u"], ref["u"], u0) <= U_TOL32
    assert load_err(got["F"], ref["F"], ref["Fabs"]) <= LOAD_TOL32
    assert load_err(got["T"], ref["T"], 0.5 * sc.d_p * ref["Fabs"]) <= LOAD_TOL32
    if mode != ibm.IBM_SPREAD_PLAIN:
        assert got["ctx"].stats()["touched_cells"] == oracle_mod.touched_count(sc.dims, sc.x_p, sc.d_p)
