"""CPU checks of the C-ABI library: it builds, loads, and exports every entry
point that include/ibm.h declares.  No compute call (no GPU here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ibm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(ibm_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ibm_create", "ibm_destroy", "ibm_set_particles", "ibm_forcing_step",
              "ibm_particle_loads", "ibm_backward", "ibm_mean_force", "ibm_set_contact_exclusion",
              "ibm_disabled_markers", "ibm_particle_inertia"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2109_03972_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n


def test_status_strings_without_gpu():
    from paper_2109_03972_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.ibm_status_string.restype = ctypes.c_char_p
    assert lib.ibm_status_string(0) == b"IBM_OK"
    assert lib.ibm_status_string(6) == b"IBM_ERR_TIMEOUT"
    lib.ibm_last_error.restype = ctypes.c_char_p
    assert lib.ibm_last_error(None) == b""


def test_create_rejects_bad_config_without_touching_gpu():
    # Invalid configurations are rejected before any CUDA call.
    from paper_2109_03972_gb300 import build, ibm
    L = ibm.load_library(build.build())
    dims = (ctypes.c_int32 * 3)(32, 32, 32)
    for bad in ({"h": -1.0}, {"kernel_width": 5}, {"n_forcing": 0}, {"precision": 9},
                {"max_particles": 0}, {"precision": ibm.IBM_FP64, "spread_mode": ibm.IBM_SPREAD_CLUSTER},
                {"threads_per_block": 256}, {"threads_per_block": -2},
                {"kernel_width": 4, "spread_mode": ibm.IBM_SPREAD_DETERMINISTIC},
                {"kernel_width": 4, "requires_grad": 1}):
        c = ibm._Config()
        c.n_scenes, c.dims, c.h, c.kernel_width, c.n_forcing = 1, dims, 1.0, 3, 3
        c.precision, c.spread_mode, c.max_particles = ibm.IBM_FP32, ibm.IBM_SPREAD_PLAIN, 4
        for k, v in bad.items():
            setattr(c, k, v)
        out = ctypes.c_void_p()
        assert L.ibm_create(ctypes.byref(c), None, ctypes.byref(out)) == 1
    # dims below 8 cells
    c = ibm._Config()
    small = (ctypes.c_int32 * 3)(4, 32, 32)
    c.n_scenes, c.dims, c.h, c.kernel_width, c.n_forcing = 1, small, 1.0, 3, 3
    c.precision, c.spread_mode, c.max_particles = ibm.IBM_FP32, ibm.IBM_SPREAD_PLAIN, 4
    assert L.ibm_create(ctypes.byref(c), None, ctypes.byref(ctypes.c_void_p())) == 1


def test_new_entry_points_reject_null_without_touching_gpu():
    # NULL context or NULL required pointers return IBM_ERR_INVALID_ARG (1)
    # before any CUDA call.
    from paper_2109_03972_gb300 import build, ibm
    L = ibm.load_library(build.build())
    n = ctypes.c_int64()
    fbar = (ctypes.c_double * 3)()
    assert L.ibm_mean_force(None, None, fbar, 0) == 1
    assert L.ibm_set_contact_exclusion(None, 1, 0.0, 0) == 1
    assert L.ibm_disabled_markers(None, None, ctypes.byref(n)) == 1
    assert L.ibm_particle_inertia(None, None, None, None, None, 0) == 1


def test_fluid_solver_rejects_bad_config_without_touching_gpu():
    # the fluid solver checks sizes, h, nu, theta and the coarsest multigrid level before any CUDA call
    from paper_2109_03972_gb300 import build, ibm
    L = ibm.load_library(build.build())
    good = dict(nx=32, ny=32, nz=64, h=1.0, nu=0.01, theta=1.0, rtol=0.0, max_cycles=0, profile=0, two_pass_smoother=0)
    for bad in ({"nx": 1}, {"h": 0.0}, {"nu": -1.0}, {"theta": 1.5}, {"rtol": -1.0}, {"max_cycles": -1},
                {"nx": 33, "ny": 33, "nz": 33},        # odd: one level of 35937 cells > 32768
                {"nx": 2 ** 14, "ny": 2 ** 14, "nz": 4}):  # beyond the index range
        c = ibm._FluidConfig(**{**good, **bad})
        out = ctypes.c_void_p()
        assert L.ibm_fluid_create(ctypes.byref(c), None, ctypes.byref(out)) == 1, bad
        assert not out.value
    assert L.ibm_fluid_predict(None, 0, 0.1, None) == 1
    assert L.ibm_fluid_correct(None, 0, 0.1, None, None, 0) == 1
    assert L.ibm_fluid_stage(None, None, 0, 0.1, None, None) == 1
    assert L.ibm_fluid_stats(None, None, None, None) == 1
    assert L.ibm_fluid_kernel_timing(None, None, None, 0) == 1
    assert L.ibm_fluid_destroy(None) == 1
    assert L.ibm_fluid_last_error(None) == b""
    assert L.ibm_status_string(8) == b"IBM_ERR_NOCONVERGE"


def test_binding_fails_loudly_without_the_library(tmp_path):
    # no CPU fallback: a missing libibm.so is an ImportError, in a fresh process
    import subprocess
    import sys
    code = ("import paper_2109_03972_gb300.ibm as m\n"
            "m._lib = None\n"
            "try:\n"
            "    m.load_library(%r)\n"
            "except ImportError:\n"
            "    print('raised')\n") % str(tmp_path / "libibm.so")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, timeout=300)
    assert r.returncode == 0 and "raised" in r.stdout, r.stderr[-1000:]
