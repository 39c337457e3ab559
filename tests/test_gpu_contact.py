"""GPU parity of marker exclusion near contact (Sec. 2.2.5) against the oracle.

The set of markers left out is index work decided by FP64 distances: both sides
compute the same distances in FP64 without contraction, so the bitmaps must
agree bit for bit, except for a marker whose distance lies within 1e-9 h of the
threshold (the marker directions come from the device's and the host's sin/cos,
which may differ in the last bit).  The forcing step with the oracle's mask then
follows the usual tolerances: FP64 1e-12 of max|u0|, FP32 2e-5 of max|u0|;
loads 1e-12 / 1e-4 of sum|F|dV.
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

SEED = 0x2109039720


@pytest.fixture(scope="module")
def oracle_mod():
    from oracle import oracle as O
    O.build()
    return O


def _dense_scene(dims=(64, 56, 60), n=40, seed=11):
    # RSA at the minimum gap of 1h: many pairs with gaps below 2 eps_sep = 3h
    rng = np.random.default_rng(seed)
    d = rng.choice([8.0, 10.0, 12.0, 14.0], n)
    return synth.make_scene(dims, d, seed, gap=1.0)


def _borderline(O, dims, x_p, d_p, width, eps=None):
    """Markers within 1e-9 of the threshold of some pair in reach (either side may decide them)."""
    xi, _ = O.marker_positions(x_p, d_p, width=width)
    counts = [O.marker_count(d) for d in d_p]
    first = np.concatenate([[0], np.cumsum(counts)])
    lim = 2 * (O.eps_sep(width) if eps is None else eps)
    L = np.array(dims, float)
    near = np.zeros(first[-1], bool)
    for p in range(len(d_p)):
        for q in range(len(d_p)):
            if p == q:
                continue
            dv = x_p[q] - x_p[p]
            dv -= L * np.floor(dv / L + 0.5)
            if np.sqrt((dv * dv).sum()) - 0.5 * (d_p[p] + d_p[q]) >= lim + 1e-9:
                continue
            r = xi[first[p]:first[p + 1]] - x_p[q]
            r -= L * np.floor(r / L + 0.5)
            dist = np.sqrt((r * r).sum(1)) - 0.5 * d_p[q]
            near[first[p]:first[p + 1]] |= np.abs(dist - lim) < 1e-9
    return near


def _run(sc, u0, prec, width=3, graph=False, steps=1, mode=ibm.IBM_SPREAD_PLAIN):
    ctx = gpu_context([sc.dims], sc.n_p, prec, mode, width=width)
    if graph:
        ctx = ibm.Context(ibm.Config(**{**ctx.cfg.__dict__, "use_graph": True}))
    ctx.set_contact_exclusion(True, 0.0, SEED)
    dt = torch.float64 if prec == ibm.IBM_FP64 else torch.float32
    ctx.set_particles(sc.x_p, sc.u_p, sc.omega_p, sc.d_p)
    out = []
    src = torch.from_numpy(u0).to(device="cuda", dtype=dt)
    u = torch.empty_like(src)                 # one buffer: graph replays need the same pointers
    for _ in range(steps):
        u.copy_(src)
        ctx.forcing_step([u], 0.01)
        mask, n = ctx.disabled_markers()
        out.append((u.double().cpu().numpy(), ctx.particle_loads(), mask, n))
    return ctx, out


def _compare_mask(O, sc, mask, width=3):
    ref = O.contact_exclusion(sc.dims, sc.x_p, sc.d_p, seed=SEED, width=width)
    diff = mask != ref
    if diff.any():
        border = _borderline(O, sc.dims, sc.x_p, sc.d_p, width)
        assert not (diff & ~border).any(), np.nonzero(diff & ~border)[0][:10]
    return ref


@pytest.mark.parametrize("prec,width", [(ibm.IBM_FP64, 3), (ibm.IBM_FP32, 3), (ibm.IBM_FP64, 4)])
def test_exclusion_matches_oracle(oracle_mod, prec, width):
    sc = _dense_scene()
    u0 = sc.field()
    ctx, [(u, loads, mask, n)] = _run(sc, u0, prec, width=width)
    ref = _compare_mask(oracle_mod, sc, mask, width)
    assert n == mask.sum() and ref.sum() > 50          # the scene has contacts
    o = oracle_mod.forcing_step(u0, sc.x_p, sc.u_p, sc.omega_p, sc.d_p, width=width, disabled=ref)
    tol_u, tol_f = (1e-12, 1e-12) if prec == ibm.IBM_FP64 else (2e-5, 1e-4)
    scale = np.abs(u0).max()
    assert np.abs(u - o["u"]).max() <= tol_u * scale
    fs = np.abs(o["Fabs"]).sum()
    assert np.abs(loads["F"] - o["F"]).max() <= tol_f * fs
    # and it differs from the step without exclusion
    plain = oracle_mod.forcing_step(u0, sc.x_p, sc.u_p, sc.omega_p, sc.d_p, width=width)
    assert np.abs(plain["u"] - o["u"]).max() > 100 * tol_u * scale


def test_exclusion_off_and_far(oracle_mod):
    # exclusion off: nothing disabled; on, but every gap >= 3h: nothing disabled
    sc = _dense_scene()
    ctx = gpu_context([sc.dims], sc.n_p, ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN)
    ctx.set_particles(sc.x_p, sc.u_p, sc.omega_p, sc.d_p)
    u = torch.from_numpy(sc.field()).cuda()
    ctx.forcing_step([u], 0.01)
    assert ctx.disabled_markers()[1] == 0
    far = synth.make_scene((64, 56, 60), np.array([10.0, 12.0, 8.0]), 5, gap=3.5)
    ctx2 = gpu_context([far.dims], far.n_p, ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN)
    ctx2.set_contact_exclusion(True, 0.0, SEED)
    ctx2.set_particles(far.x_p, far.u_p, far.omega_p, far.d_p)
    u2 = torch.from_numpy(far.field()).cuda()
    ctx2.forcing_step([u2], 0.01)
    assert ctx2.disabled_markers()[1] == 0


def test_exclusion_multi_scene_ids(oracle_mod):
    # the coin uses global particle indices: scene 1's particles follow scene 0's
    a, b = _dense_scene(seed=21), _dense_scene(dims=(48, 52, 56), n=24, seed=22)
    x = np.concatenate([a.x_p, b.x_p])
    d = np.concatenate([a.d_p, b.d_p])
    up = np.concatenate([a.u_p, b.u_p])
    om = np.concatenate([a.omega_p, b.omega_p])
    so = np.concatenate([np.zeros(a.n_p, np.int32), np.ones(b.n_p, np.int32)])
    ctx = gpu_context([a.dims, b.dims], len(d), ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN)
    ctx.set_contact_exclusion(True, 0.0, SEED)
    ctx.set_particles(x, up, om, d, scene_of=so)
    us = [torch.from_numpy(s.field()).cuda() for s in (a, b)]
    ctx.forcing_step(us, 0.01)
    mask, _ = ctx.disabled_markers()
    na = sum(oracle_mod.marker_count(v) for v in a.d_p)
    ra = oracle_mod.contact_exclusion(a.dims, a.x_p, a.d_p, seed=SEED, ids=np.arange(a.n_p))
    rb = oracle_mod.contact_exclusion(b.dims, b.x_p, b.d_p, seed=SEED, ids=a.n_p + np.arange(b.n_p))
    assert np.array_equal(mask[:na], ra) and np.array_equal(mask[na:], rb)
    assert ra.any() and rb.any()


@pytest.mark.parametrize("mode", [ibm.IBM_SPREAD_CLUSTER, ibm.IBM_SPREAD_DETERMINISTIC])
def test_exclusion_on_the_cluster_kernel_matches_oracle(oracle_mod, mode):
    # the shared-memory cluster kernel (and its plain fallback) leave the same markers out
    sc = _dense_scene()
    u0 = sc.field()
    ctx, [(u, loads, mask, n)] = _run(sc, u0, ibm.IBM_FP32, mode=mode)
    ref = _compare_mask(oracle_mod, sc, mask)
    assert ref.sum() > 50
    st = ctx.stats()
    assert st["clusters_smem"] > 0                      # the step ran the shared-memory kernel
    o = oracle_mod.forcing_step(u0, sc.x_p, sc.u_p, sc.omega_p, sc.d_p, disabled=ref)
    scale = np.abs(u0).max()
    assert np.abs(u - o["u"]).max() <= 2e-5 * scale
    assert np.abs(loads["F"] - o["F"]).max() <= 1e-4 * np.abs(o["Fabs"]).sum()
    plain = oracle_mod.forcing_step(u0, sc.x_p, sc.u_p, sc.omega_p, sc.d_p)
    assert np.abs(plain["u"] - o["u"]).max() > 100 * 2e-5 * scale


def test_exclusion_on_an_oversized_cluster_and_graph(oracle_mod):
    # a dense 48^3 box of the batched workload (27 spheres, one cluster of about 17,700 markers) runs its
    # big cluster off the one-SM kernel (a thread-block cluster); the step replayed from a graph
    sc = synth.workload("batched").scenes[123]
    u0 = sc.field()
    ctx, out = _run(sc, u0, ibm.IBM_FP32, mode=ibm.IBM_SPREAD_DETERMINISTIC, graph=True, steps=3)
    st = ctx.stats()
    assert st["markers_dsmem"] + st["markers_fallback"] > 0
    u, loads, mask, n = out[0]
    ref = _compare_mask(oracle_mod, sc, mask)
    o = oracle_mod.forcing_step(u0, sc.x_p, sc.u_p, sc.omega_p, sc.d_p, disabled=ref)
    assert np.abs(u - o["u"]).max() <= 2e-5 * np.abs(u0).max()
    for u2, _, m2, _ in out[1:]:
        assert np.array_equal(m2, mask) and np.array_equal(u2, u)   # deterministic mode: bit for bit


def test_exclusion_graph_replay_and_config_errors(oracle_mod):
    sc = _dense_scene()
    u0 = sc.field()
    _, out = _run(sc, u0, ibm.IBM_FP64, graph=True, steps=3)
    ref = _compare_mask(oracle_mod, sc, out[0][2])
    for u, loads, mask, n in out[1:]:
        assert np.array_equal(mask, out[0][2])
        assert np.abs(u - out[0][0]).max() <= 1e-12 * np.abs(u0).max()
    assert ref.any()
    c = gpu_context([sc.dims], sc.n_p, ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN, requires_grad=True)
    with pytest.raises(ibm.IBMError):
        c.set_contact_exclusion(True)
    c = gpu_context([sc.dims], sc.n_p, ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN)
    with pytest.raises(ibm.IBMError):
        c.set_contact_exclusion(True, -1.0)


def test_exclusion_full_bed(oracle_mod):
    # the bidisperse bed (13,500 spheres, 8.1M markers), FP32 plain path: the
    # whole bitmap against the oracle's brute force over all pairs
    W = synth.workload("bidisperse")
    sc = W.scenes[0]
    ctx = ibm.Context(ibm.Config(dims=[sc.dims], n_forcing=W.n_forcing, precision=ibm.IBM_FP32,
                                 spread_mode=ibm.IBM_SPREAD_PLAIN, max_particles=sc.n_p))
    ctx.set_contact_exclusion(True, 0.0, SEED)
    ctx.set_particles(sc.x_p, sc.u_p, sc.omega_p, sc.d_p)
    u = torch.from_numpy(sc.field().astype(np.float32)).cuda()
    ctx.forcing_step([u], W.tau)
    del u
    mask, n = ctx.disabled_markers()
    ref = oracle_mod.contact_exclusion(sc.dims, sc.x_p, sc.d_p, seed=SEED)
    assert ref.sum() > 1000
    diff = np.nonzero(mask != ref)[0]
    assert diff.size <= 4, diff[:10]          # at most a few borderline markers
