"""Failure handling of the library, exercised without faulting the GPU.

  * bounded device-side retries: the lock-free union-find of the clustering
    gives up after ibm_set_wait_limit iterations; with a limit of 1 a scene
    with a multi-particle cluster must report IBM_ERR_TIMEOUT at the next
    synchronising call, and the same context must then run a normal step that
    matches the oracle;
  * allocation failures: the test hook ibm_debug_fail_allocation refuses the
    n-th device allocation on the host; every call that allocates must return
    IBM_ERR_OOM for every n, the same context must work once the hook is off,
    and no device memory may be left behind;
  * the fixed-point range of deterministic spreading: far more overlap than
    non-overlapping spheres can produce (hundreds of coincident spheres) must
    be reported as IBM_ERR_CAPACITY instead of wrapping silently, while a
    moderate overlap (a shared-memory cluster) stays within range and matches
    the oracle.
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

IBM_ERR_OOM, IBM_ERR_CAPACITY, IBM_ERR_TIMEOUT = 3, 4, 6
U_TOL32, LOAD_TOL32 = 2e-5, 1e-4


@pytest.fixture(scope="module")
def oracle_mod():
    from oracle import oracle as O
    O.build()
    return O


def _chain():
    # five spheres at the minimum gap: one cluster, four unions
    dims = (48, 40, 44)
    d = np.array([10.0, 12.0, 9.0, 11.0, 10.0])
    pts = [np.array([12.2, 20.3, 22.1])]
    for i in range(1, len(d)):
        pts.append(pts[-1] + np.array([1.0, 0.0, 0.0]) * (0.5 * (d[i] + d[i - 1]) + 1.0))
    u_p, om, rho = synth.particle_state(len(d), 9)
    return synth.Scene(dims, np.array(pts) % np.array(dims), d, u_p, om, rho, field_seed=17)


@pytest.mark.parametrize("mode", [ibm.IBM_SPREAD_CLUSTER, ibm.IBM_SPREAD_DETERMINISTIC])
def test_union_find_wait_limit_reports_timeout_and_recovers(oracle_mod, mode):
    sc = _chain()
    u0 = f32_round(sc.field())
    ctx = gpu_context([sc.dims], sc.n_p, ibm.IBM_FP32, mode)
    ctx.set_particles(sc.x_p, sc.u_p, sc.omega_p, sc.d_p)
    ctx.set_wait_limit(1)
    u = torch.from_numpy(u0).float().cuda()
    with pytest.raises(ibm.IBMError) as e:
        ctx.forcing_step([u], 0.01, want_slip=True)
    assert e.value.status == IBM_ERR_TIMEOUT
    ctx.set_wait_limit(0)
    u = torch.from_numpy(u0).float().cuda()
    ctx.forcing_step([u], 0.01, want_slip=True)
    loads = ctx.particle_loads()
    ref = oracle_mod.forcing_step(u0, sc.x_p, sc.u_p, sc.omega_p, sc.d_p, n_forcing=3, tau=0.01)
    assert ctx.stats()["clusters"] == 1
    assert rel_err_u(u.double().cpu().numpy(), ref["u"], u0) <= U_TOL32
    assert load_err(loads["F"], ref["F"], ref["Fabs"]) <= LOAD_TOL32
    with pytest.raises(ibm.IBMError) as e:
        ctx.set_wait_limit(-1)
    assert e.value.status == 1


def _steps(ctx, sc, u0):
    ctx.set_particles(sc.x_p, sc.u_p, sc.omega_p, sc.d_p)
    u = torch.from_numpy(u0).float().cuda()
    ctx.forcing_step([u], 0.01, want_slip=True)
    return u, ctx.particle_loads()


def _fail_sweep(sc, u0, mode, ref_u):
    """Refuse the n-th allocation for n = 1, 2, ... until a whole create + set +
    step sequence gets through; returns how many positions were tried."""
    seen_ok, n = False, 0
    while not seen_ok:
        n += 1
        assert n < 200
        ibm.debug_fail_allocation(n)
        ctx = None
        try:
            ctx = gpu_context([sc.dims], sc.n_p, ibm.IBM_FP32, mode)
            _steps(ctx, sc, u0)
            seen_ok = True                  # the n-th allocation was never reached
        except ibm.IBMError as err:
            assert err.status == IBM_ERR_OOM, (n, err)
        ibm.debug_fail_allocation(0)
        if ctx is not None:
            # the same context recovers once allocations succeed again
            u, loads = _steps(ctx, sc, u0)
            u = u.cpu().numpy()
            if mode == ibm.IBM_SPREAD_DETERMINISTIC:
                assert np.array_equal(u, ref_u), n     # bit-reproducible, even after a failed step
            assert rel_err_u(u.astype(np.float64), ref_u.astype(np.float64), u0) <= U_TOL32
            ctx.close()
    return n


@pytest.mark.parametrize("mode", [ibm.IBM_SPREAD_DETERMINISTIC, ibm.IBM_SPREAD_PLAIN])
def test_every_failed_allocation_returns_oom(mode):
    # diff128 in deterministic mode has a fallback cluster: the cluster path,
    # the plain fallback and its fixed-point buffers all allocate
    sc = synth.workload("diff128").scenes[0]
    u0 = f32_round(sc.field())
    ctx = gpu_context([sc.dims], sc.n_p, ibm.IBM_FP32, mode)
    ref_u, _ = _steps(ctx, sc, u0)
    ref_u = ref_u.cpu().numpy()
    ctx.close()

    def free_bytes():
        torch.cuda.synchronize()
        torch.cuda.empty_cache()        # torch's cached blocks are not the library's
        return torch.cuda.mem_get_info()[0]

    # the first sweep may load code and reserve memory once; a second identical
    # sweep must not take any more device memory (no leak on any failure path)
    n = _fail_sweep(sc, u0, mode, ref_u)
    assert n > 10
    free1 = free_bytes()
    assert _fail_sweep(sc, u0, mode, ref_u) == n
    assert abs(free_bytes() - free1) <= 4 << 20


def _coincident(n, d=4.0, dims=(32, 32, 32)):
    rng = np.random.default_rng(5)
    x = np.array([16.3, 15.7, 16.1]) + rng.uniform(-1e-3, 1e-3, size=(n, 3))
    z = np.zeros((n, 3))
    return synth.Scene(dims, x, np.full(n, d), z, z.copy(), np.full(n, 1.3), field_seed=3)


def test_moderate_overlap_stays_in_fixed_point_range(oracle_mod):
    # 16 coincident spheres: one shared-memory cluster, about 12 unit weights per
    # cell (a sphere gives at most about 1); the loop diverges (W W^T D has
    # eigenvalues far above 2), so errors are judged against the result's scale
    sc = _coincident(16)
    u0 = np.full((3, 32, 32, 32), 5.0)
    ref = oracle_mod.forcing_step(u0, sc.x_p, sc.u_p, sc.omega_p, sc.d_p, n_forcing=3, tau=0.01)
    got = run_gpu(sc, u0, ibm.IBM_FP32, ibm.IBM_SPREAD_DETERMINISTIC)
    assert got["ctx"].stats()["markers_fallback"] == 0
    scale = np.abs(ref["u"]).max()
    assert np.abs(got["u"] - ref["u"]).max() <= U_TOL32 * scale
    assert load_err(got["F"], ref["F"], ref["Fabs"]) <= LOAD_TOL32


def test_overlap_beyond_range_on_the_thread_block_cluster_path():
    # 320 coincident spheres (20,480 markers: too many for one SM, not for a thread-block cluster): the
    # distributed-shared-memory kernel's conversion reports the range too
    sc = _coincident(320)
    u0 = np.full((3, 32, 32, 32), 5.0)
    ctx = gpu_context([sc.dims], sc.n_p, ibm.IBM_FP32, ibm.IBM_SPREAD_DETERMINISTIC)
    ctx.set_particles(sc.x_p, sc.u_p, sc.omega_p, sc.d_p)
    u = torch.from_numpy(u0).float().cuda()
    with pytest.raises(ibm.IBMError) as e:
        ctx.forcing_step([u], 0.01, want_slip=True)
    assert e.value.status == IBM_ERR_CAPACITY
    assert ctx.stats()["markers_dsmem"] > 0


def test_extreme_overlap_reports_fixed_point_range(oracle_mod):
    # 520 coincident spheres (more particles than a thread-block cluster takes: the plain fallback): about
    # 400 unit weights per cell, six times the bound the fixed-point scale assumes; deterministic mode must
    # say so rather than return wrapped integers, and the context must run a valid scene afterwards; the
    # FP32 atomic mode has no such range
    sc = _coincident(520)
    u0 = np.full((3, 32, 32, 32), 5.0)
    ctx = gpu_context([sc.dims], sc.n_p, ibm.IBM_FP32, ibm.IBM_SPREAD_DETERMINISTIC)
    ctx.set_particles(sc.x_p, sc.u_p, sc.omega_p, sc.d_p)
    u = torch.from_numpy(u0).float().cuda()
    with pytest.raises(ibm.IBMError) as e:
        ctx.forcing_step([u], 0.01, want_slip=True)
    assert e.value.status == IBM_ERR_CAPACITY
    one = synth.Scene(sc.dims, np.array([[15.2, 16.9, 14.4]]), np.array([12.0]), np.array([[0.1, 0.0, -0.1]]),
                      np.zeros((1, 3)), np.array([1.3]), field_seed=8)
    uu = f32_round(one.field())
    got_u, loads = _steps(ctx, one, uu)
    ref = oracle_mod.forcing_step(uu, one.x_p, one.u_p, one.omega_p, one.d_p, n_forcing=3, tau=0.01)
    assert rel_err_u(got_u.double().cpu().numpy(), ref["u"], uu) <= U_TOL32
    ref = oracle_mod.forcing_step(u0, sc.x_p, sc.u_p, sc.omega_p, sc.d_p, n_forcing=1, tau=0.01)
    got = run_gpu(sc, u0, ibm.IBM_FP32, ibm.IBM_SPREAD_CLUSTER, nf=1)
    assert np.abs(got["u"] - ref["u"]).max() <= U_TOL32 * np.abs(ref["u"]).max()
