"""GPU test of ibm_forcing_step_static, the entry point that allocates nothing.

It serves callers that cannot allocate device memory: a host that hands the
library a fixed memory budget at start-up, an application whose own allocator
owns the device, loops that cannot afford cudaFree's device-wide
synchronisation.  Its scratch is a fixed array inside the library.  Checked
through the C ABI against the context-based FP64 plain path (ibm_forcing_step)
on two calls in a row, at the FP64 tolerance of the other parity tests; a call
after the first must leave the device's free memory unchanged; sizes beyond the
array are rejected.  Named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2109_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2109_03972_gb300 import ibm, synth  # noqa: E402

IBM_ERR_CAPACITY = 4


def _lib():
    L = ibm.load_library()
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.ibm_forcing_step_static.argtypes = [i, i, i, d, i, d, i, vp, vp, vp, vp, vp, vp, vp, vp]
    L.ibm_forcing_step_static.restype = i
    return L


def _static_step(L, dims, x, up, om, d, u, F, T, nf=3, tau=0.01):
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.ibm_forcing_step_static(dims[0], dims[1], dims[2], 1.0, nf, tau, int(d.shape[0]), p(x), p(up),
                                     p(om), p(d), p(u), p(F), p(T), stream)


def test_static_step_matches_context_step_twice():
    L = _lib()
    sc = synth.workload("small").scenes[0]
    u0 = sc.field()
    dev = dict(device="cuda", dtype=torch.float64)
    ua = torch.tensor(u0, **dev)
    ub = ua.clone()
    ctx = ibm.Context(ibm.Config(dims=[sc.dims], precision=ibm.IBM_FP64, spread_mode=ibm.IBM_SPREAD_PLAIN,
                                 max_particles=sc.n_p))
    ctx.set_particles(sc.x_p, sc.u_p, sc.omega_p, sc.d_p)
    x, up, om, d = (torch.tensor(a, **dev).contiguous() for a in (sc.x_p, sc.u_p, sc.omega_p, sc.d_p))
    F = torch.empty((sc.n_p, 3), **dev)
    T = torch.empty((sc.n_p, 3), **dev)
    scale = np.abs(u0).max()
    for call in range(2):
        ctx.forcing_step([ua], 0.01)
        ref = ctx.particle_loads()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert _static_step(L, sc.dims, x, up, om, d, ub, F, T) == 0
        torch.cuda.synchronize()
        if call > 0:
            # after the first call (which looks up the scratch address and loads
            # the kernels) a call takes no device memory at all
            assert torch.cuda.mem_get_info()[0] == free0
        assert (ua - ub).abs().max().item() <= 1e-12 * scale
        Fs, Ts = F.cpu().numpy(), T.cpu().numpy()
        fs = np.abs(ref["F"]).max()
        assert np.abs(Fs - ref["F"]).max() <= 1e-12 * fs
        assert np.abs(Ts - ref["T"]).max() <= 1e-12 * np.abs(ref["T"]).max()


def test_static_step_rejects_sizes_beyond_its_array():
    L = _lib()
    dims = (64, 64, 64)
    rng = np.random.default_rng(3)
    n = 900                       # 900 spheres of 804 markers: 723,600 > 688,106
    dev = dict(device="cuda", dtype=torch.float64)
    x = torch.tensor(rng.uniform(0, 64, size=(n, 3)), **dev)
    up = torch.zeros((n, 3), **dev)
    om = torch.zeros((n, 3), **dev)
    d = torch.full((n,), 16.0, **dev)
    u = torch.randn((3, 64, 64, 64), **dev)
    u0 = u.clone()
    F = torch.full((n, 3), 7.0, **dev)
    T = torch.full((n, 3), 7.0, **dev)
    assert _static_step(L, dims, x, up, om, d, u, F, T) == IBM_ERR_CAPACITY
    torch.cuda.synchronize()
    assert torch.equal(u, u0)
    # a rejected call leaves zeros in the loads, not the caller's old values
    assert torch.count_nonzero(F).item() == 0 and torch.count_nonzero(T).item() == 0
    big = 65537
    xb = torch.zeros((big, 3), **dev)
    db = torch.full((big,), 8.0, **dev)
    assert _static_step(L, dims, xb, xb, xb, db, u, torch.empty((big, 3), **dev),
                        torch.empty((big, 3), **dev)) == IBM_ERR_CAPACITY
