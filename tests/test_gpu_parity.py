"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances:
  FP64 path : |u - u_oracle|_inf <= 1e-12 |u0|_inf; loads <= 1e-12 sum|F|dV
              (the two differ only in the order of the additions).
  FP32 paths: |u - u_oracle|_inf <= 2e-5 |u0|_inf; force <= 1e-4 sum|F|dV,
              torque <= 1e-4 (d/2) sum|F|dV; slip RMS <= 1e-3 relative.
              Each cell is u0 plus n_F spreads of about 30 FP32 products and
              each interpolated velocity a 27-term FP32 sum, so the rounding
              stays near 3 * 27 * 2^-24 ~ 5e-6 of the field scale; the loads
              add FP32 products in 32-marker chunks before the FP64 sums.
  Stencil base cells: bit-exact.
"""
import math

import numpy as np
import pytest

from tests._helpers import f32_round, load_err, rel_err_u, run_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2109_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2109_03972_gb300 import ibm, synth  # noqa: E402

FP32_MODES = [ibm.IBM_SPREAD_PLAIN, ibm.IBM_SPREAD_CLUSTER, ibm.IBM_SPREAD_DETERMINISTIC]
U_TOL32, LOAD_TOL32, SLIP_TOL32 = 2e-5, 1e-4, 1e-3


def _scene(name):
    return synth.workload(name).scenes[0]


def _chain_scene():
    # Spheres at the minimum gap of 1h in a chain that crosses the periodic seam:
    # one particle cluster whose stencils overlap everywhere.
    dims = (48, 40, 44)
    d = np.array([10.0, 12.0, 9.0, 11.0, 10.0])
    x = np.array([[5.2, 20.3, 22.1]])
    pts = [x[0]]
    rng = np.random.default_rng(4)
    for i in range(1, len(d)):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        pts.append(pts[-1] + v * (0.5 * (d[i] + d[i - 1]) + 1.0))
    x = np.array(pts) % np.array(dims)
    u_p, om, rho = synth.particle_state(len(d), 9)
    return synth.Scene(dims, x, d, u_p, om, rho, field_seed=17)


SCENES = {"small": lambda: _scene("small"), "single64": lambda: _scene("single64"), "chain": _chain_scene}


@pytest.fixture(scope="module")
def oracle_mod():
    from oracle import oracle as O
    O.build()
    return O


def _oracle_run(O, sc, u0, nf=3, tau=0.01, want_f=False):
    return O.forcing_step(u0, sc.x_p, sc.u_p, sc.omega_p, sc.d_p, n_forcing=nf, tau=tau, want_f=want_f)


@pytest.mark.parametrize("name", ["small", "single64", "chain"])
def test_fp64_plain_matches_oracle(oracle_mod, name):
    sc = SCENES[name]()
    u0 = sc.field()
    ref = _oracle_run(oracle_mod, sc, u0, want_f=True)
    got = run_gpu(sc, u0, ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN, want_f=True)
    assert rel_err_u(got["u"], ref["u"], u0) <= 1e-12
    assert load_err(got["F"], ref["F"], ref["Fabs"]) <= 1e-12
    assert load_err(got["T"], ref["T"], 0.5 * sc.d_p * ref["Fabs"]) <= 1e-12
    assert np.abs(got["f"] - ref["f"]).max() <= 1e-12 * np.abs(u0).max() / 0.01
    assert got["slip"][0] == pytest.approx(ref["slip"][0], rel=1e-10)
    assert got["slip"][1] == pytest.approx(ref["slip"][1], rel=1e-10)


@pytest.mark.parametrize("mode", FP32_MODES)
@pytest.mark.parametrize("name", ["small", "single64", "chain"])
def test_fp32_matches_oracle(oracle_mod, name, mode):
    sc = SCENES[name]()
    u0 = f32_round(sc.field())
    ref = _oracle_run(oracle_mod, sc, u0, want_f=True)
    got = run_gpu(sc, u0, ibm.IBM_FP32, mode, want_f=True)
    assert rel_err_u(got["u"], ref["u"], u0) <= U_TOL32
    assert load_err(got["F"], ref["F"], ref["Fabs"]) <= LOAD_TOL32
    assert load_err(got["T"], ref["T"], 0.5 * sc.d_p * ref["Fabs"]) <= LOAD_TOL32
    assert np.abs(got["f"] - ref["f"]).max() <= U_TOL32 * np.abs(u0).max() / 0.01
    assert got["slip"][0] == pytest.approx(ref["slip"][0], rel=SLIP_TOL32)


@pytest.mark.parametrize("precision", [ibm.IBM_FP64, ibm.IBM_FP32])
@pytest.mark.parametrize("name", ["small", "single64", "chain"])
def test_bins_bit_exact(oracle_mod, name, precision):
    sc = SCENES[name]()
    mode = ibm.IBM_SPREAD_PLAIN if precision == ibm.IBM_FP64 else ibm.IBM_SPREAD_CLUSTER
    from tests._helpers import gpu_context
    ctx = gpu_context([sc.dims], sc.n_p, precision, mode)
    ctx.set_particles(sc.x_p, sc.u_p, sc.omega_p, sc.d_p)
    got = ctx.marker_bases()
    xi, base = oracle_mod.marker_positions(sc.x_p, sc.d_p)
    ties = np.abs(xi - np.round(xi)) < 1e-9
    assert ties.sum() == 0
    assert np.array_equal(got, base)


def test_newton_euler_matches_oracle(oracle_mod):
    sc = _scene("small")
    u0 = sc.field()
    g = (0.0, 0.0, -1e-3)
    ref = _oracle_run(oracle_mod, sc, u0)
    x, u, w = oracle_mod.newton_euler(sc.x_p, sc.u_p, sc.omega_p, sc.d_p, sc.rho_p, 1.0, g, 0.01,
                                      ref["F"], ref["T"])
    got = run_gpu(sc, u0, ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN, newton_euler=True)
    assert np.allclose(got["u_p"], u, rtol=1e-11, atol=1e-13)
    assert np.allclose(got["omega_p"], w, rtol=1e-11, atol=1e-13)
    assert np.allclose(got["x_p"], x, rtol=1e-13, atol=1e-12)
    got32 = run_gpu(sc, f32_round(u0), ibm.IBM_FP32, ibm.IBM_SPREAD_CLUSTER, newton_euler=True)
    ref32 = _oracle_run(oracle_mod, sc, f32_round(u0))
    x, u, w = oracle_mod.newton_euler(sc.x_p, sc.u_p, sc.omega_p, sc.d_p, sc.rho_p, 1.0, g, 0.01,
                                      ref32["F"], ref32["T"])
    scale = np.abs(u - sc.u_p).max()
    assert np.abs(got32["u_p"] - u).max() <= LOAD_TOL32 * 10 * scale


def test_empty_particle_set():
    from tests._helpers import gpu_context
    ctx = gpu_context([(32, 32, 32)], 4, ibm.IBM_FP32, ibm.IBM_SPREAD_CLUSTER)
    ctx.set_particles(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0))
    u = torch.randn(3, 32, 32, 32, device="cuda")
    u0 = u.clone()
    slip = ctx.forcing_step([u], 0.01, want_slip=True)
    assert torch.equal(u, u0)
    assert slip == (0.0, 0.0)


@pytest.mark.parametrize("mode", FP32_MODES)
def test_multi_scene_matches_oracle(oracle_mod, mode):
    # Three independent periodic scenes of different sizes in one context.
    W = synth.workload("batched")
    scenes = [s for s in W.scenes[:40] if s.n_p > 0][:3]
    from tests._helpers import gpu_context
    n = sum(s.n_p for s in scenes)
    ctx = gpu_context([s.dims for s in scenes], n, ibm.IBM_FP32, mode)
    x = np.concatenate([s.x_p for s in scenes])
    up = np.concatenate([s.u_p for s in scenes])
    om = np.concatenate([s.omega_p for s in scenes])
    d = np.concatenate([s.d_p for s in scenes])
    so = np.concatenate([np.full(s.n_p, i, dtype=np.int32) for i, s in enumerate(scenes)])
    u0s = [f32_round(s.field()) for s in scenes]
    us = [torch.from_numpy(a).float().cuda() for a in u0s]
    ctx.set_particles(x, up, om, d, scene_of=so)
    ctx.forcing_step(us, 0.01)
    loads = ctx.particle_loads()
    off = 0
    for s, u0, u in zip(scenes, u0s, us):
        ref = _oracle_run(oracle_mod, s, u0)
        assert rel_err_u(u.double().cpu().numpy(), ref["u"], u0) <= U_TOL32
        sl = slice(off, off + s.n_p)
        assert load_err(loads["F"][sl], ref["F"], ref["Fabs"]) <= LOAD_TOL32
        off += s.n_p


def test_invalid_arguments_are_reported():
    from tests._helpers import gpu_context
    ctx = gpu_context([(32, 32, 32)], 2, ibm.IBM_FP32, ibm.IBM_SPREAD_CLUSTER)
    good = dict(x_p=np.array([[16.0, 16.0, 16.0]]), u_p=np.zeros((1, 3)), omega_p=np.zeros((1, 3)),
                d_p=np.array([8.0]))
    with pytest.raises(ibm.IBMError) as e:
        ctx.set_particles(**{**good, "x_p": np.array([[np.nan, 1.0, 1.0]])})
    assert e.value.status == 5
    with pytest.raises(ibm.IBMError) as e:
        ctx.set_particles(**{**good, "d_p": np.array([29.0])})
    assert e.value.status == 1
    with pytest.raises(ibm.IBMError) as e:
        ctx.set_particles(**{**good, "d_p": np.array([-1.0])})
    assert e.value.status == 1
    with pytest.raises(ibm.IBMError) as e:
        ctx.set_particles(np.zeros((3, 3)), np.zeros((3, 3)), np.zeros((3, 3)), np.full(3, 8.0))
    assert e.value.status == 4
    with pytest.raises(ibm.IBMError) as e:
        ctx.particle_loads()
    assert e.value.status == 7
    with pytest.raises(ibm.IBMError) as e:
        ctx.backward([torch.zeros(3, 32, 32, 32, device="cuda")])
    assert e.value.status == 7
    ctx.set_particles(**good)
    with pytest.raises(ibm.IBMError) as e:
        ctx.forcing_step([torch.zeros(3, 32, 32, 32, device="cuda")], -1.0)
    assert e.value.status == 1
    ne = gpu_context([(32, 32, 32)], 2, ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN, newton_euler=True)
    with pytest.raises(ibm.IBMError) as e:
        ne.set_particles(**good, rho_p=np.array([1.0]))
    assert e.value.status == 1


def _grad_case():
    sc = _scene("small")
    rng = np.random.default_rng(5)
    wgt = rng.uniform(0, 1, size=(sc.dims[2], sc.dims[1], sc.dims[0]))
    return sc, sc.field(), wgt


def test_backward_fp64_matches_oracle(oracle_mod):
    sc, u0, wgt = _grad_case()
    ref_u = _oracle_run(oracle_mod, sc, u0)["u"]
    go = wgt[None] * ref_u
    gi, gU, gW, gX = oracle_mod.backward(u0, sc.x_p, sc.u_p, sc.omega_p, sc.d_p, go)
    from tests._helpers import gpu_context
    ctx = gpu_context([sc.dims], sc.n_p, ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN, requires_grad=True)
    ctx.set_particles(sc.x_p, sc.u_p, sc.omega_p, sc.d_p)
    u = torch.from_numpy(u0).cuda()
    ctx.forcing_step([u], 0.01)
    g = torch.from_numpy(wgt[None]).cuda() * u
    gis, tU, tW, tX = ctx.backward([g])
    torch.cuda.synchronize()
    assert np.abs(gis[0].cpu().numpy() - gi).max() <= 1e-11 * np.abs(gi).max()
    for a, b in ((tU, gU), (tW, gW), (tX, gX)):
        assert np.abs(a.cpu().numpy() - b).max() <= 1e-10 * max(1.0, np.abs(b).max())


def test_backward_fp32_vs_fp64():
    sc, u0, wgt = _grad_case()
    from tests._helpers import gpu_context
    res = {}
    for prec, mode in ((ibm.IBM_FP64, ibm.IBM_SPREAD_PLAIN), (ibm.IBM_FP32, ibm.IBM_SPREAD_CLUSTER)):
        ctx = gpu_context([sc.dims], sc.n_p, prec, mode, requires_grad=True)
        ctx.set_particles(sc.x_p, sc.u_p, sc.omega_p, sc.d_p)
        dt = torch.float64 if prec == ibm.IBM_FP64 else torch.float32
        u = torch.from_numpy(f32_round(u0)).to(dtype=dt, device="cuda")
        ctx.forcing_step([u], 0.01)
        g = torch.from_numpy(wgt[None]).to(dtype=dt, device="cuda") * u
        res[prec] = [t.double().cpu().numpy() if hasattr(t, "cpu") else t
                     for t in (lambda r: [r[0][0], r[1], r[2], r[3]])(ctx.backward([g]))]
    for a, b in zip(res[ibm.IBM_FP32], res[ibm.IBM_FP64]):
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b)


def test_autograd_function_fd():
    # torch.autograd.Function over the hand-written adjoint, FP64 central FD at eps = 1e-6.
    sc, u0, wgt = _grad_case()
    from tests._helpers import gpu_context
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
    L = 0.5 * (w * out * out).sum()
    L.backward()
    eps = 1e-6
    for t, grad in ((up, up.grad), (om, om.grad), (xp, xp.grad)):
        for (p, c) in ((0, 0), (1, 2), (3, 1)):
            with torch.no_grad():
                t[p, c] += eps
                up_f = field(uu, up, om, xp)
                t[p, c] -= 2 * eps
                um_f = field(uu, up, om, xp)
                t[p, c] += eps
                # L(+) - L(-) = 1/2 sum w (u+ - u-)(u+ + u-): no cancellation in L itself
                fd = (0.5 * (w * (up_f - um_f) * (up_f + um_f)).sum()).item() / (2 * eps)
            tol = 1e-5 if t is xp else 1e-6
            assert abs(fd - grad[p, c].item()) <= tol * max(1.0, grad.abs().max().item())


def _big_chain_scene():
    # Four D=24 spheres at the minimum gap: one cluster of ~29K touched cells and
    # 7240 markers, too large to hold all three velocity components in shared
    # memory, so the kernel runs the components one at a time.
    dims = (128, 120, 112)
    d = np.array([24.0, 24.0, 24.0, 24.0])
    pts = [np.array([30.3, 60.7, 55.2])]
    for v in ([1.0, 0.0, 0.0], [0.6, 0.8, 0.0], [0.0, 0.6, 0.8]):
        pts.append(pts[-1] + np.array(v) * 25.0)
    u_p, om, rho = synth.particle_state(4, 21)
    return synth.Scene(dims, np.array(pts), d, u_p, om, rho, field_seed=23)


@pytest.mark.parametrize("mode", [ibm.IBM_SPREAD_CLUSTER, ibm.IBM_SPREAD_DETERMINISTIC])
def test_large_cluster_one_component_path(oracle_mod, mode):
    sc = _big_chain_scene()
    u0 = f32_round(sc.field())
    ref = _oracle_run(oracle_mod, sc, u0)
    got = run_gpu(sc, u0, ibm.IBM_FP32, mode)
    st = got["ctx"].stats()
    assert st["clusters"] == 1 and st["markers_fallback"] == 0
    assert rel_err_u(got["u"], ref["u"], u0) <= U_TOL32
    assert load_err(got["F"], ref["F"], ref["Fabs"]) <= LOAD_TOL32
    assert load_err(got["T"], ref["T"], 0.5 * sc.d_p * ref["Fabs"]) <= LOAD_TOL32


def _diagonal_chain_scene():
    # Fourteen D=12 spheres at the minimum gap along the (0, 1, 1) diagonal: one
    # cluster whose box has ~136 x 136 rows, too many for a dense row table
    # beside its cells, so the kernel numbers only the rows its stencils reach.
    dims = (40, 256, 256)
    n = 14
    d = np.full(n, 12.0)
    step = np.array([0.0, 1.0, 1.0]) / np.sqrt(2.0) * 13.0
    x = np.array([20.3, 30.1, 28.7]) + np.arange(n)[:, None] * step
    u_p, om, rho = synth.particle_state(n, 31)
    return synth.Scene(dims, x, d, u_p, om, rho, field_seed=37)


@pytest.mark.parametrize("mode", [ibm.IBM_SPREAD_CLUSTER, ibm.IBM_SPREAD_DETERMINISTIC])
def test_elongated_cluster_sparse_rows(oracle_mod, mode):
    sc = _diagonal_chain_scene()
    # dense table: (x words) * (y rows) * (z rows) of the stencil box, far above
    # what fits in shared memory beside the cells
    ext = np.floor(sc.x_p + 0.5 * sc.d_p[:, None]).max(0) - np.floor(sc.x_p - 0.5 * sc.d_p[:, None]).min(0) + 3
    assert ((ext[0] + 31) // 32) * ext[1] * ext[2] > 16000
    u0 = f32_round(sc.field())
    ref = _oracle_run(oracle_mod, sc, u0)
    got = run_gpu(sc, u0, ibm.IBM_FP32, mode)
    st = got["ctx"].stats()
    assert st["clusters"] == 1 and st["markers_fallback"] == 0
    assert st["touched_cells"] == oracle_mod.touched_count(sc.dims, sc.x_p, sc.d_p)
    assert rel_err_u(got["u"], ref["u"], u0) <= U_TOL32
    assert load_err(got["F"], ref["F"], ref["Fabs"]) <= LOAD_TOL32
    assert load_err(got["T"], ref["T"], 0.5 * sc.d_p * ref["Fabs"]) <= LOAD_TOL32


@pytest.mark.parametrize("name", ["small", "single64", "chain"])
def test_touched_cells_match_oracle(oracle_mod, name):
    sc = SCENES[name]()
    got = run_gpu(sc, f32_round(sc.field()), ibm.IBM_FP32, ibm.IBM_SPREAD_DETERMINISTIC, want_slip=False)
    st = got["ctx"].stats()
    assert st["markers_fallback"] == 0
    assert st["touched_cells"] == oracle_mod.touched_count(sc.dims, sc.x_p, sc.d_p)


@pytest.mark.parametrize("name", ["small", "chain"])
def test_deterministic_mode_is_bit_reproducible(name):
    sc = SCENES[name]()
    u0 = f32_round(sc.field())
    a = run_gpu(sc, u0, ibm.IBM_FP32, ibm.IBM_SPREAD_DETERMINISTIC)
    for _ in range(2):
        b = run_gpu(sc, u0, ibm.IBM_FP32, ibm.IBM_SPREAD_DETERMINISTIC)
        assert np.array_equal(a["u"], b["u"])
        assert np.array_equal(a["F"], b["F"]) and np.array_equal(a["T"], b["T"])


def test_deterministic_fallback_is_bit_reproducible_and_matches_oracle(oracle_mod):
    # 150 spheres in 128^3: one cluster is too large for a CTA and runs a thread-block
    # cluster or the plain path, whose deterministic modes spread in per-cluster
    # integer fixed point
    sc = synth.workload("diff128").scenes[0]
    u0 = f32_round(sc.field())
    a = run_gpu(sc, u0, ibm.IBM_FP32, ibm.IBM_SPREAD_DETERMINISTIC)
    st = a["ctx"].stats()
    assert st["markers_fallback"] + st["markers_dsmem"] > 0     # off the one-SM kernel
    ref = _oracle_run(oracle_mod, sc, u0)
    assert rel_err_u(a["u"], ref["u"], u0) <= U_TOL32
    assert load_err(a["F"], ref["F"], ref["Fabs"]) <= LOAD_TOL32
    assert load_err(a["T"], ref["T"], 0.5 * sc.d_p * ref["Fabs"]) <= LOAD_TOL32
    for _ in range(2):
        b = run_gpu(sc, u0, ibm.IBM_FP32, ibm.IBM_SPREAD_DETERMINISTIC)
        assert np.array_equal(a["u"], b["u"])
        assert np.array_equal(a["F"], b["F"]) and np.array_equal(a["T"], b["T"])


def _ring_scene(axis):
    # four D=10 spheres at the minimum gap spaced 11 cells apart along one axis of
    # a 44-cell period: a cluster that closes on itself across the seam
    dims = [36, 40, 38]
    dims[axis] = 44
    x = np.tile(np.array([17.3, 19.6, 18.2]), (4, 1))
    x[:, axis] = 3.7 + 11.0 * np.arange(4)
    u_p, om, rho = synth.particle_state(4, 41 + axis)
    return synth.Scene(tuple(dims), x, np.full(4, 10.0), u_p, om, rho, field_seed=43 + axis)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("mode", [ibm.IBM_SPREAD_CLUSTER, ibm.IBM_SPREAD_DETERMINISTIC])
def test_periodic_cluster_in_shared_memory(oracle_mod, axis, mode):
    # the ring cannot be unwrapped: its box is the whole period along that axis
    # (ghost columns in x), and it must still run in the shared-memory kernel
    sc = _ring_scene(axis)
    u0 = f32_round(sc.field())
    ref = _oracle_run(oracle_mod, sc, u0)
    got = run_gpu(sc, u0, ibm.IBM_FP32, mode)
    st = got["ctx"].stats()
    assert st["clusters"] == 1 and st["markers_fallback"] == 0
    assert rel_err_u(got["u"], ref["u"], u0) <= U_TOL32
    assert load_err(got["F"], ref["F"], ref["Fabs"]) <= LOAD_TOL32
    assert load_err(got["T"], ref["T"], 0.5 * sc.d_p * ref["Fabs"]) <= LOAD_TOL32
    if mode == ibm.IBM_SPREAD_DETERMINISTIC:
        again = run_gpu(sc, u0, ibm.IBM_FP32, mode)
        assert np.array_equal(got["u"], again["u"])


@pytest.mark.parametrize("k", [2, 8])
def test_dense_small_box_matches_oracle(oracle_mod, k):
    # dense 32^3 scenes of the batched workload: clusters wrap in several axes
    sc = synth.workload("batched", n_scenes=k + 1).scenes[k]
    u0 = f32_round(sc.field())
    ref = _oracle_run(oracle_mod, sc, u0)
    got = run_gpu(sc, u0, ibm.IBM_FP32, ibm.IBM_SPREAD_DETERMINISTIC)
    assert got["ctx"].stats()["markers_fallback"] == 0
    assert rel_err_u(got["u"], ref["u"], u0) <= U_TOL32
    assert load_err(got["F"], ref["F"], ref["Fabs"]) <= LOAD_TOL32


@pytest.mark.parametrize("name", ["small", "single64", "chain"])
@pytest.mark.parametrize("precision", [ibm.IBM_FP64, ibm.IBM_FP32])
def test_four_point_kernel_matches_oracle(oracle_mod, name, precision):
    # the four-point kernel of Sec. 2.2.3 on the plain path: bins bit-exact,
    # FP64 at 1e-12, FP32 at the FP32 tolerances
    sc = SCENES[name]()
    from tests._helpers import gpu_context
    ctx = gpu_context([sc.dims], sc.n_p, precision, ibm.IBM_SPREAD_PLAIN, width=4)
    ctx.set_particles(sc.x_p, sc.u_p, sc.omega_p, sc.d_p)
    xi, base = oracle_mod.marker_positions(sc.x_p, sc.d_p, width=4)
    assert np.array_equal(ctx.marker_bases(), base)
    u0 = sc.field() if precision == ibm.IBM_FP64 else f32_round(sc.field())
    ref = oracle_mod.forcing_step(u0, sc.x_p, sc.u_p, sc.omega_p, sc.d_p, n_forcing=3, tau=0.01, width=4)
    got = run_gpu(sc, u0, precision, ibm.IBM_SPREAD_PLAIN, width=4)
    tu, tl = (1e-12, 1e-12) if precision == ibm.IBM_FP64 else (U_TOL32, LOAD_TOL32)
    assert rel_err_u(got["u"], ref["u"], u0) <= tu
    assert load_err(got["F"], ref["F"], ref["Fabs"]) <= tl
    assert load_err(got["T"], ref["T"], 0.5 * sc.d_p * ref["Fabs"]) <= tl
    assert got["slip"][0] == pytest.approx(ref["slip"][0], rel=1e-10 if precision == ibm.IBM_FP64 else SLIP_TOL32)


@pytest.mark.parametrize("name", ["small", "chain"])
def test_two_ctas_per_sm_variant_matches_oracle(oracle_mod, name):
    # the 512-thread variant (two CTAs per SM, half the shared memory each)
    sc = SCENES[name]()
    u0 = f32_round(sc.field())
    ref = _oracle_run(oracle_mod, sc, u0)
    got = run_gpu(sc, u0, ibm.IBM_FP32, ibm.IBM_SPREAD_DETERMINISTIC, tpb=512)
    assert got["ctx"].stats()["threads_per_block"] == 512
    assert rel_err_u(got["u"], ref["u"], u0) <= U_TOL32
    assert load_err(got["F"], ref["F"], ref["Fabs"]) <= LOAD_TOL32
    assert load_err(got["T"], ref["T"], 0.5 * sc.d_p * ref["Fabs"]) <= LOAD_TOL32
