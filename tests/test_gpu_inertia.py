"""GPU parity of the fluid-inertia integrals inside each particle (Sec. 2.2.9)
against the oracle on the same fields.

Tolerances: FP64 fields 1e-12 of V_p max|u| (Iu, V) and of (d_p/2) V_p max|u|
(Ir); FP32 fields (the oracle reads the same FP32 values): per-thread FP32 sums
over at most a few dozen cells, alpha from FP32 corner distances (relative
error ~1e-6 near the surface), so 1e-5 of the same scales.
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
from paper_2109_03972_gb300 import ibm, synth  # noqa: E402

TOL = {ibm.IBM_FP64: 1e-12, ibm.IBM_FP32: 1e-5}


@pytest.fixture(scope="module")
def oracle_mod():
    from oracle import oracle as O
    O.build()
    return O


def _check(got, ref, d_p, umax, tol):
    V = math.pi * np.asarray(d_p) ** 3 / 6
    s = (V * umax)[:, None]
    assert np.all(np.abs(got["Iu"] - ref["Iu"]) <= tol * s)
    assert np.all(np.abs(got["Ir"] - ref["Ir"]) <= tol * s * 0.5 * np.asarray(d_p)[:, None])
    assert np.all(np.abs(got["V"] - ref["V"]) <= tol * V)


@pytest.mark.parametrize("prec", [ibm.IBM_FP64, ibm.IBM_FP32])
def test_inertia_matches_oracle(oracle_mod, prec):
    # two scenes (ragged edges, spheres across the periodic seams), h = 1
    rng = np.random.default_rng(5)
    scenes = [synth.make_scene((64, 56, 60), rng.choice([8.0, 12.0, 16.0], 30), 31, gap=1.0),
              synth.make_scene((45, 50, 47), rng.choice([8.0, 10.0, 20.0], 12), 32, gap=1.0)]
    dt = torch.float64 if prec == ibm.IBM_FP64 else torch.float32
    x = np.concatenate([s.x_p for s in scenes])
    d = np.concatenate([s.d_p for s in scenes])
    so = np.concatenate([np.full(s.n_p, k, np.int32) for k, s in enumerate(scenes)])
    ctx = gpu_context([s.dims for s in scenes], len(d), prec, ibm.IBM_SPREAD_PLAIN)
    ctx.set_particles(x, np.zeros_like(x), np.zeros_like(x), d, scene_of=so)
    us = [torch.from_numpy(s.field()).to(device="cuda", dtype=dt) for s in scenes]
    got = ctx.particle_inertia(us)
    again = ctx.particle_inertia(us)
    dev = ctx.particle_inertia(us, device=True)
    for k in ("Iu", "Ir", "V"):
        assert np.array_equal(got[k], again[k])                      # no atomics: reproducible
        assert np.array_equal(got[k], dev[k].cpu().numpy())
    off = 0
    for s, u in zip(scenes, us):
        uh = u.double().cpu().numpy()
        ref = oracle_mod.particle_inertia(uh, s.x_p, s.d_p)
        sl = slice(off, off + s.n_p)
        _check({k: v[sl] for k, v in got.items()}, ref, s.d_p, np.abs(uh).max(), TOL[prec])
        off += s.n_p
    s0 = scenes[0]
    a = 0.5 * s0.d_p[:, None]
    assert ((s0.x_p - a - 2 < 0) | (s0.x_p + a + 2 >= np.array(s0.dims))).any()   # some boxes wrap


def test_inertia_full_bed(oracle_mod):
    # the bidisperse bed (FP32, 512 x 512 x 1024): sampled particles against the
    # oracle on sub-boxes cut out around them (each integral only reads the
    # particle's own box), and V_p of every particle against its sphere volume
    W = synth.workload("bidisperse")
    sc = W.scenes[0]
    ctx = ibm.Context(ibm.Config(dims=[sc.dims], n_forcing=W.n_forcing, precision=ibm.IBM_FP32,
                                 spread_mode=ibm.IBM_SPREAD_DETERMINISTIC, max_particles=sc.n_p))
    ctx.set_particles(sc.x_p, sc.u_p, sc.omega_p, sc.d_p)
    u32 = sc.field().astype(np.float32)
    u = torch.from_numpy(u32).cuda()
    got = ctx.particle_inertia([u])
    del u
    V = math.pi * sc.d_p ** 3 / 6
    assert np.all(np.abs(got["V"] / V - 1) <= 2.0 / sc.d_p ** 2)
    nx, ny, nz = sc.dims
    rng = np.random.default_rng(9)
    picked = np.concatenate([rng.choice(np.nonzero(sc.d_p == dd)[0], 8, replace=False) for dd in (12.0, 24.0)])
    for p in picked:
        R = int(math.ceil(0.5 * sc.d_p[p])) + 4
        base = np.floor(sc.x_p[p]).astype(int) - R
        S = 2 * R + 1
        ix, iy, iz = ((base[c] + np.arange(S)) % n for c, n in enumerate((nx, ny, nz)))
        sub = u32[:, iz][:, :, iy][:, :, :, ix].astype(np.float64)
        ref = oracle_mod.particle_inertia(sub, (sc.x_p[p] - base)[None], sc.d_p[p:p + 1])
        _check({k: v[p:p + 1] for k, v in got.items()}, ref, sc.d_p[p:p + 1], np.abs(sub).max(),
               TOL[ibm.IBM_FP32])
