"""GPU parity of the collision models and the RK3 particle sub-steps
(Sec. 2.2.6-2.2.8, Eq. f_int; Sec. 2.2.10) with the FP64 oracle.

Scenes: spheres of 5-9 h placed by random sequential addition at zero gap in
periodic boxes (about 30% solid), moving towards the box centre with random
perturbations and random angular velocities, densities 1.5-3 rho_f, gravity:
collisions (Hertz contact with stick and slip) start and end all through the
calls, other pairs sit inside eps_sep (lubrication).  Three calls of 15
sub-steps each, the contact history carried from call to call.  Compared, at 1e-12 of their scales: positions, velocities and
angular velocities; the kept contact history (same pairs, springs, impact
speeds); the collision loads at the final state.  Also: two scenes in one
context, bit-reproducibility, exact free flight, and the margin check that
reports a particle moving too far for the neighbour list.
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
from paper_2109_03972_gb300 import ibm, synth  # noqa: E402

TOL = 1e-12


@pytest.fixture(scope="module")
def oracle_mod():
    from oracle import oracle as O
    O.build()
    return O


def _packed(dims, n, seed, dlo=5.0, dhi=9.0, converge=1.0):
    rng = np.random.default_rng(seed)
    ds = np.sort(rng.uniform(dlo, dhi, size=n))[::-1]
    x, d = synth.rsa_spheres(dims, ds, seed=seed + 1, gap=0.0)
    # velocities towards the box centre plus noise: collisions all through the calls
    c = 0.5 * np.array(dims, float)
    r = x - c
    m = d.size
    u = -converge * r / np.linalg.norm(r, axis=1)[:, None] + rng.normal(0.0, 0.1, size=(m, 3))
    om = rng.normal(0.0, 0.2, size=(m, 3))
    rho = rng.uniform(1.5, 3.0, size=m)
    return x, u, om, d, rho


PRM = dict(rho_f=1.0, nu_f=0.01, e_dry=0.9, mu_s=0.4, mu_k=0.3, nu_poisson=0.3, t_c=0.1, st_crit=5.0,
           g=(0.0, 0.0, -0.1))


def _gpu_params(**kw):
    return ibm.CollisionParams(**{**PRM, **kw})


def _oracle_params(O, **kw):
    return O.collision_params(**{**PRM, **kw})


def _run_gpu(dims_list, parts, scene_of, dt, n_sub, calls, F_h=None, T_h=None):
    x, u, om, d, rho = parts
    ctx = gpu_context(dims_list, len(d), ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN)
    ctx.set_particles(x, u, om, d, rho, scene_of=scene_of)
    prm = _gpu_params()
    for _ in range(calls):
        ctx.particle_substeps(prm, dt, n_sub, F_h=F_h, T_h=T_h)
    xs, us, ws = ctx.particle_state()
    hist = ctx.contact_history()
    Fc, Tc = ctx.collision_forces(prm)
    return xs, us, ws, hist, Fc, Tc, ctx


def _run_oracle(O, dims_list, parts, scene_of, dt, n_sub, calls, F_h=None, T_h=None):
    x, u, om, d, rho = parts
    P = _oracle_params(O)
    hist = O.PairHistory()
    for _ in range(calls):
        x, u, om, hist = O.particle_substeps(P, dims_list, x, u, om, d, rho, dt, n_sub=n_sub, F_h=F_h, T_h=T_h,
                                             hist=hist, scene=scene_of)
    Fc, Tc = O.collision_forces(P, dims_list, x, u, om, d, rho, hist, scene=scene_of)
    return x, u, om, hist, Fc, Tc


def _compare(got, ref, parts):
    xs, us, ws, (hp, hq, hz, hu), Fc, Tc, _ = got
    xo, uo, wo, hist, Fo, To = ref
    L = 64.0
    assert np.abs(xs - xo).max() <= TOL * L
    assert np.abs(us - uo).max() <= TOL * max(1.0, np.abs(uo).max())
    assert np.abs(ws - wo).max() <= TOL * max(1.0, np.abs(wo).max())
    n = hist.n.value
    assert n > 0 and hp.size == n
    order = np.lexsort((hist.q[:n], hist.p[:n]))
    assert np.array_equal(hp, hist.p[:n][order]) and np.array_equal(hq, hist.q[:n][order])
    zs = np.abs(hist.z[:n][order]).max()
    assert np.abs(hz - hist.z[:n][order]).max() <= TOL * max(zs, 1e-30) * 10
    assert np.abs(hu - hist.u[:n][order]).max() <= TOL * np.abs(hist.u[:n]).max()
    scale = np.abs(Fo).sum()
    assert np.abs(Fc - Fo).max() <= TOL * scale
    assert np.abs(Tc - To).max() <= TOL * max(np.abs(To).sum(), 1e-30)


def test_dense_scene_matches_oracle(oracle_mod):
    dims = (32, 32, 32)
    parts = _packed(dims, 70, 11)
    got = _run_gpu([dims], parts, None, 0.1, 15, 3)
    ref = _run_oracle(oracle_mod, [dims], parts, None, 0.1, 15, 3)
    hp = got[3][0]
    assert hp.size >= 2                       # pairs in contact at the end
    _compare(got, ref, parts)


def test_two_scenes_with_hydrodynamic_loads_match_oracle(oracle_mod):
    a = _packed((32, 32, 32), 70, 21)
    b = _packed((30, 34, 28), 50, 31)
    parts = tuple(np.concatenate([pa, pb]) for pa, pb in zip(a, b))
    so = np.concatenate([np.zeros(len(a[3]), np.int32), np.ones(len(b[3]), np.int32)])
    rng = np.random.default_rng(5)
    n = len(parts[3])
    Fh = rng.normal(0.0, 5.0, size=(n, 3))
    Th = rng.normal(0.0, 5.0, size=(n, 3))
    dims = [(32, 32, 32), (30, 34, 28)]
    got = _run_gpu(dims, parts, so, 0.1, 15, 3, F_h=Fh, T_h=Th)
    ref = _run_oracle(oracle_mod, dims, parts, so, 0.1, 15, 3, F_h=Fh, T_h=Th)
    _compare(got, ref, parts)


def test_substeps_are_bit_reproducible():
    dims = (32, 32, 32)
    parts = _packed(dims, 70, 11)
    a = _run_gpu([dims], parts, None, 0.1, 15, 3)
    b = _run_gpu([dims], parts, None, 0.1, 15, 3)
    for k in range(3):
        assert np.array_equal(a[k], b[k])
    assert np.array_equal(a[4], b[4]) and np.array_equal(a[3][2], b[3][2])


def test_free_flight_is_exact():
    x0 = np.array([[10.0, 12.0, 20.0], [40.0, 30.0, 30.0]])
    u0 = np.array([[0.3, 0.1, 0.0], [-0.2, 0.0, 0.4]])
    w0 = np.array([[0.1, 0.2, 0.3], [0.0, -0.1, 0.0]])
    d = np.array([6.0, 5.0])
    rho = np.array([2.5, 1.6])
    Fh = np.array([[0.5, 0.0, 0.0], [0.0, 0.2, -0.1]])
    Th = np.array([[0.0, 0.0, 0.7], [0.1, 0.0, 0.0]])
    ctx = gpu_context([(64, 64, 64)], 2, ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN)
    ctx.set_particles(x0, u0, w0, d, rho)
    ctx.particle_substeps(_gpu_params(g=(0.1, -0.2, -1.0)), 0.7, 15, F_h=Fh, T_h=Th)
    x, u, w = ctx.particle_state()
    m = rho * np.pi * d ** 3 / 6
    I = m * d ** 2 / 10
    a = Fh / m[:, None] + (1 - 1.0 / rho)[:, None] * np.array([0.1, -0.2, -1.0])
    t = 0.7
    assert np.allclose(u, u0 + a * t, rtol=0, atol=1e-13)
    assert np.allclose(x, x0 + u0 * t + 0.5 * a * t * t, rtol=0, atol=1e-12)
    assert np.allclose(w, w0 + Th / I[:, None] * t, rtol=0, atol=1e-13)


def test_margin_check_reports_fast_particles():
    dims = (32, 32, 32)
    x, u, om, d, rho = _packed(dims, 30, 41)
    u = u.copy()
    u[0] = (50.0, 0.0, 0.0)                   # 10 cells in one call of dt = 0.2
    ctx = gpu_context([dims], len(d), ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN)
    ctx.set_particles(x, u, om, d, rho)
    with pytest.raises(ibm.IBMError) as e:
        ctx.particle_substeps(_gpu_params(), 0.2, 15)
    assert e.value.status == 4
    # a wider margin lets the same call through
    ctx.set_particles(x, u, om, d, rho)
    ctx.particle_substeps(_gpu_params(pair_margin=25.0), 0.2, 15)


def test_missing_densities_are_rejected():
    ctx = gpu_context([(32, 32, 32)], 2, ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN)
    ctx.set_particles(np.array([[10.0, 10, 10], [20, 20, 20]]), np.zeros((2, 3)), np.zeros((2, 3)),
                      np.array([6.0, 6.0]))
    with pytest.raises(ibm.IBMError) as e:
        ctx.particle_substeps(_gpu_params(), 0.1, 3)
    assert e.value.status == 1


def test_larger_dense_box_matches_oracle(oracle_mod):
    # 400 spheres in a 64^3 box (about 30% solid), one call of 15 sub-steps
    dims = (64, 64, 64)
    parts = _packed(dims, 400, 51)
    got = _run_gpu([dims], parts, None, 0.1, 15, 1)
    ref = _run_oracle(oracle_mod, [dims], parts, None, 0.1, 15, 1)
    assert got[3][0].size >= 5
    _compare(got, ref, parts)
