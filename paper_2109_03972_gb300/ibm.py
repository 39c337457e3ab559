"""Thin Python binding of the C ABI in ``include/ibm.h``.

Argument marshalling only: every step of the forcing loop runs in the CUDA
kernels of ``libibm.so``.  PyTorch supplies device memory and the stream.  If
the library is missing this module raises on import: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libibm.so")

IBM_FP64, IBM_FP32 = 0, 1
IBM_SPREAD_CLUSTER, IBM_SPREAD_DETERMINISTIC, IBM_SPREAD_PLAIN = 0, 1, 2
IBM_PATH_SMEM, IBM_PATH_GLOBAL_RECORDS, IBM_PATH_ONE_COMPONENT = 1, 2, 4
IBM_PATH_SPARSE_ROWS, IBM_PATH_PERIODIC, IBM_PATH_FALLBACK, IBM_PATH_DSMEM = 8, 16, 32, 64

STATUS = {0: "IBM_OK", 1: "IBM_ERR_INVALID_ARG", 2: "IBM_ERR_CUDA", 3: "IBM_ERR_OOM",
          4: "IBM_ERR_CAPACITY", 5: "IBM_ERR_NONFINITE", 6: "IBM_ERR_TIMEOUT", 7: "IBM_ERR_STATE",
          8: "IBM_ERR_NOCONVERGE"}

EXPORTED = ["ibm_create", "ibm_destroy", "ibm_set_particles", "ibm_forcing_step",
            "ibm_particle_loads", "ibm_backward", "ibm_marker_bases", "ibm_step_stats",
            "ibm_kernel_timing", "ibm_status_string", "ibm_last_error"]


class IBMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Config(ctypes.Structure):
    _fields_ = [("n_scenes", ctypes.c_int), ("dims", ctypes.POINTER(ctypes.c_int32)),
                ("h", ctypes.c_double), ("kernel_width", ctypes.c_int), ("n_forcing", ctypes.c_int),
                ("precision", ctypes.c_int), ("spread_mode", ctypes.c_int),
                ("newton_euler", ctypes.c_int), ("rho_f", ctypes.c_double),
                ("g", ctypes.c_double * 3), ("max_particles", ctypes.c_int),
                ("requires_grad", ctypes.c_int), ("threads_per_block", ctypes.c_int),
                ("profile", ctypes.c_int), ("use_graph", ctypes.c_int)]


class _CollisionParams(ctypes.Structure):
    _fields_ = [("rho_f", ctypes.c_double), ("nu_f", ctypes.c_double), ("e_dry", ctypes.c_double),
                ("mu_s", ctypes.c_double), ("mu_k", ctypes.c_double), ("nu_poisson", ctypes.c_double),
                ("t_c", ctypes.c_double), ("st_crit", ctypes.c_double), ("eps_sep", ctypes.c_double),
                ("zeta_min", ctypes.c_double), ("lub_c", ctypes.c_double), ("g", ctypes.c_double * 3),
                ("pair_margin", ctypes.c_double)]


class _FluidConfig(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("h", ctypes.c_double),
                ("nu", ctypes.c_double), ("theta", ctypes.c_double), ("rtol", ctypes.c_double),
                ("max_cycles", ctypes.c_int), ("profile", ctypes.c_int), ("two_pass_smoother", ctypes.c_int)]


class _FluidFields(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("ut", ctypes.c_void_p), ("uf", ctypes.c_void_p), ("p", ctypes.c_void_p),
                ("phi", ctypes.c_void_p)]


@dataclass
class CollisionParams:
    """Collision models of Sec. 2.2.6-2.2.8 (0 in eps_sep, zeta_min, lub_c,
    pair_margin takes the library's default)."""
    rho_f: float = 1.0
    nu_f: float = 0.01
    e_dry: float = 0.97
    mu_s: float = 0.4
    mu_k: float = 0.3
    nu_poisson: float = 0.3
    t_c: float = 0.1
    st_crit: float = 5.0
    eps_sep: float = 0.0
    zeta_min: float = 0.0
    lub_c: float = 0.0
    g: tuple = (0.0, 0.0, 0.0)
    pair_margin: float = 0.0

    def _c(self):
        c = _CollisionParams()
        for k in ("rho_f", "nu_f", "e_dry", "mu_s", "mu_k", "nu_poisson", "t_c", "st_crit", "eps_sep",
                  "zeta_min", "lub_c", "pair_margin"):
            setattr(c, k, float(getattr(self, k)))
        c.g = (ctypes.c_double * 3)(*[float(v) for v in self.g])
        return c


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libibm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libibm.so not found at {path}; build it with "
                          "paper_2109_03972_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.ibm_create.argtypes = [ctypes.POINTER(_Config), vp, ctypes.POINTER(vp)]
    L.ibm_destroy.argtypes = [vp]
    L.ibm_set_particles.argtypes = [vp, i, vp, vp, vp, vp, vp, vp, i]
    L.ibm_forcing_step.argtypes = [vp, vp, d, vp, vp]
    L.ibm_particle_loads.argtypes = [vp, vp, vp, vp, vp, vp, i]
    L.ibm_backward.argtypes = [vp, vp, vp, vp, vp, vp]
    L.ibm_mean_force.argtypes = [vp, vp, vp, i]
    L.ibm_particle_inertia.argtypes = [vp, vp, vp, vp, vp, i]
    L.ibm_set_contact_exclusion.argtypes = [vp, i, d, ctypes.c_uint64]
    L.ibm_disabled_markers.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int64)]
    L.ibm_marker_bases.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int64)]
    L.ibm_step_stats.argtypes = [vp, vp]
    L.ibm_particle_clusters.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_int64)]
    L.ibm_particle_clusters.restype = i
    L.ibm_particle_substeps.argtypes = [vp, ctypes.POINTER(_CollisionParams), d, i, vp, vp, i]
    L.ibm_particle_substeps.restype = i
    L.ibm_collision_forces.argtypes = [vp, ctypes.POINTER(_CollisionParams), vp, vp, i]
    L.ibm_collision_forces.restype = i
    L.ibm_particle_state.argtypes = [vp, vp, vp, vp, i]
    L.ibm_particle_state.restype = i
    L.ibm_contact_history.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), vp, vp, vp, vp]
    L.ibm_contact_history.restype = i
    L.ibm_set_wait_limit.argtypes = [vp, ctypes.c_int64]
    L.ibm_set_wait_limit.restype = i
    L.ibm_debug_fail_allocation.argtypes = [ctypes.c_int64]
    L.ibm_debug_fail_allocation.restype = i
    L.ibm_kernel_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), i]
    L.ibm_fluid_create.argtypes = [ctypes.POINTER(_FluidConfig), vp, ctypes.POINTER(vp)]
    L.ibm_fluid_create.restype = i
    L.ibm_fluid_destroy.argtypes = [vp]
    L.ibm_fluid_destroy.restype = i
    L.ibm_fluid_predict.argtypes = [vp, i, d, ctypes.POINTER(_FluidFields)]
    L.ibm_fluid_predict.restype = i
    L.ibm_fluid_correct.argtypes = [vp, i, d, ctypes.POINTER(_FluidFields), vp, i]
    L.ibm_fluid_correct.restype = i
    L.ibm_fluid_stage.argtypes = [vp, vp, i, d, ctypes.POINTER(_FluidFields), vp]
    L.ibm_fluid_stage.restype = i
    L.ibm_fluid_stats.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_int)]
    L.ibm_fluid_stats.restype = i
    L.ibm_fluid_kernel_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), i]
    L.ibm_fluid_kernel_timing.restype = i
    L.ibm_fluid_last_error.argtypes = [vp]
    L.ibm_fluid_last_error.restype = ctypes.c_char_p
    L.ibm_status_string.argtypes = [i]
    L.ibm_status_string.restype = ctypes.c_char_p
    L.ibm_last_error.argtypes = [vp]
    L.ibm_last_error.restype = ctypes.c_char_p
    for n in EXPORTED[:9]:
        getattr(L, n).restype = i
    _lib = L
    return L


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return ctypes.c_void_p(t.data_ptr())
    return t.ctypes.data_as(ctypes.c_void_p)


def _ptr_array(ts):
    arr = (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])
    return arr


@dataclass
class Config:
    dims: list                       # [(nx, ny, nz), ...] one per scene
    h: float = 1.0
    n_forcing: int = 3
    precision: int = IBM_FP32
    spread_mode: int = IBM_SPREAD_CLUSTER
    newton_euler: bool = False
    rho_f: float = 1.0
    g: tuple = (0.0, 0.0, 0.0)
    max_particles: int = 1
    requires_grad: bool = False
    kernel_width: int = 3
    threads_per_block: int = 0        # 0: 1024 threads; 512; -1: autotune
    profile: bool = False
    use_graph: bool = False
    extra: dict = field(default_factory=dict)


class Context:
    """Owns one ibm_ctx on a CUDA stream (torch's current stream by default)."""

    def __init__(self, cfg: Config, stream: torch.cuda.Stream | None = None):
        self.L = load_library()
        self.cfg = cfg
        self.stream = stream or torch.cuda.current_stream()
        dims = np.ascontiguousarray(np.asarray(cfg.dims, dtype=np.int32).reshape(-1, 3))
        self._dims = dims
        c = _Config()
        c.n_scenes = dims.shape[0]
        c.dims = dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        c.h = cfg.h
        c.kernel_width = cfg.kernel_width
        c.n_forcing = cfg.n_forcing
        c.precision = cfg.precision
        c.spread_mode = cfg.spread_mode
        c.newton_euler = int(cfg.newton_euler)
        c.rho_f = cfg.rho_f
        c.g = (ctypes.c_double * 3)(*cfg.g)
        c.max_particles = cfg.max_particles
        c.requires_grad = int(cfg.requires_grad)
        c.threads_per_block = cfg.threads_per_block
        c.profile = int(cfg.profile)
        c.use_graph = int(cfg.use_graph)
        h = ctypes.c_void_p()
        st = self.L.ibm_create(ctypes.byref(c), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != 0:
            raise IBMError(st, "ibm_create rejected the configuration")
        self.h = h
        self.n_p = 0
        self.dtype = torch.float64 if cfg.precision == IBM_FP64 else torch.float32

    def _check(self, st):
        if st != 0:
            raise IBMError(st, self.L.ibm_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.ibm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_particles(self, x_p, u_p, omega_p, d_p, rho_p=None, scene_of=None):
        """Arrays: numpy (host) or torch tensors (device), float64."""
        on_dev = isinstance(x_p, torch.Tensor) and x_p.is_cuda
        conv = (lambda a: a.contiguous()) if on_dev else (lambda a: np.ascontiguousarray(a, dtype=np.float64))
        arrs = [conv(a) for a in (x_p, u_p, omega_p, d_p)]
        rho = None if rho_p is None else conv(rho_p)
        sc = None
        if scene_of is not None:
            sc = scene_of.contiguous() if on_dev else np.ascontiguousarray(scene_of, dtype=np.int32)
        n = int(arrs[3].shape[0])
        self._keep = (arrs, rho, sc)
        self._check(self.L.ibm_set_particles(self.h, n, *[_ptr(a) for a in arrs], _ptr(rho), _ptr(sc),
                                             int(on_dev)))
        self.n_p = n

    def forcing_step(self, u_fields, tau, f_out=None, want_slip=False):
        u_fields = list(u_fields) if isinstance(u_fields, (list, tuple)) else [u_fields]
        up = _ptr_array(u_fields)
        fp = _ptr_array(list(f_out)) if f_out is not None else None
        slip = (ctypes.c_double * 2)() if want_slip else None
        self._check(self.L.ibm_forcing_step(self.h, up, float(tau), fp, slip))
        return (slip[0], slip[1]) if want_slip else None

    def particle_loads(self, device=False):
        n = self.n_p
        if device:
            out = [torch.empty((n, 3), dtype=torch.float64, device="cuda") for _ in range(5)]
        else:
            out = [np.empty((n, 3)) for _ in range(5)]
        self._check(self.L.ibm_particle_loads(self.h, *[_ptr(o) for o in out], int(device)))
        keys = ("F", "T", "x_p", "u_p", "omega_p")
        return dict(zip(keys, out))

    def mean_force(self, f_fields, device=False):
        """Mean IBM force per scene over its grid, Eq. (fe_IBM): [n_scenes][3] FP64."""
        f_fields = list(f_fields) if isinstance(f_fields, (list, tuple)) else [f_fields]
        n = len(self._dims)
        out = torch.empty((n, 3), dtype=torch.float64, device="cuda") if device else np.empty((n, 3))
        self._check(self.L.ibm_mean_force(self.h, _ptr_array(f_fields), _ptr(out), int(device)))
        return out

    def particle_inertia(self, u_fields, device=False):
        """Fluid inertia inside each particle (Sec. 2.2.9): dict(Iu [n,3], Ir [n,3], V [n]), FP64."""
        u_fields = list(u_fields) if isinstance(u_fields, (list, tuple)) else [u_fields]
        n = self.n_p
        if device:
            out = [torch.empty(s, dtype=torch.float64, device="cuda") for s in ((n, 3), (n, 3), (n,))]
        else:
            out = [np.empty(s) for s in ((n, 3), (n, 3), (n,))]
        self._check(self.L.ibm_particle_inertia(self.h, _ptr_array(u_fields), *[_ptr(o) for o in out],
                                                int(device)))
        return dict(zip(("Iu", "Ir", "V"), out))

    def set_contact_exclusion(self, enable=True, eps_sep=0.0, seed=0):
        """Leave markers out of f_IBM near contact (Sec. 2.2.5); eps_sep = 0: the paper's value."""
        self._check(self.L.ibm_set_contact_exclusion(self.h, int(enable), float(eps_sep),
                                                     int(seed) & (2 ** 64 - 1)))

    def disabled_markers(self):
        """Markers left out by the last step: bool [n_markers], particle-then-l order."""
        n = ctypes.c_int64()
        words = np.zeros(max(1, (int(self.stats()["markers"]) + 31) // 32), dtype=np.uint32)
        self._check(self.L.ibm_disabled_markers(self.h, _ptr(words), ctypes.byref(n)))
        bits = np.unpackbits(words.view(np.uint8), bitorder="little").astype(bool)
        return bits[:int(self.stats()["markers"])], int(n.value)

    def backward(self, grad_u_out, grad_u_in=None):
        gos = list(grad_u_out) if isinstance(grad_u_out, (list, tuple)) else [grad_u_out]
        gis = [torch.empty_like(g) for g in gos] if grad_u_in is None else list(grad_u_in)
        gU, gW, gX = (torch.empty((self.n_p, 3), dtype=torch.float64, device="cuda") for _ in range(3))
        self._check(self.L.ibm_backward(self.h, _ptr_array(gos), _ptr_array(gis), _ptr(gU), _ptr(gW), _ptr(gX)))
        return gis, gU, gW, gX

    def marker_bases(self):
        n = ctypes.c_int64()
        self._check(self.L.ibm_marker_bases(self.h, None, ctypes.byref(n)))
        out = np.empty((n.value, 3), dtype=np.int64)
        self._check(self.L.ibm_marker_bases(self.h, _ptr(out), ctypes.byref(n)))
        return out

    def kernel_timing(self, reset=True):
        ms, n = ctypes.c_double(), ctypes.c_int64()
        self._check(self.L.ibm_kernel_timing(self.h, ctypes.byref(ms), ctypes.byref(n), int(reset)))
        return ms.value, n.value

    def particle_substeps(self, prm, dt, n_sub=15, F_h=None, T_h=None):
        """Advance the particle state by dt under the collision models and the
        constant hydrodynamic loads F_h, T_h (numpy [n_p, 3] or device tensors)."""
        on_dev = isinstance(F_h, torch.Tensor) or isinstance(T_h, torch.Tensor)
        conv = (lambda a: a.contiguous()) if on_dev else (
            lambda a: np.ascontiguousarray(a, dtype=np.float64))
        Fh = None if F_h is None else conv(F_h)
        Th = None if T_h is None else conv(T_h)
        c = prm._c()
        self._check(self.L.ibm_particle_substeps(self.h, ctypes.byref(c), float(dt), int(n_sub), _ptr(Fh),
                                                 _ptr(Th), int(on_dev)))

    def collision_forces(self, prm):
        n = self.n_p
        F, T = np.zeros((n, 3)), np.zeros((n, 3))
        c = prm._c()
        self._check(self.L.ibm_collision_forces(self.h, ctypes.byref(c), _ptr(F), _ptr(T), 0))
        return F, T

    def particle_state(self):
        n = self.n_p
        x, u, w = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
        self._check(self.L.ibm_particle_state(self.h, _ptr(x), _ptr(u), _ptr(w), 0))
        return x, u, w

    def contact_history(self):
        nc = ctypes.c_int64()
        self._check(self.L.ibm_contact_history(self.h, ctypes.byref(nc), None, None, None, None))
        m = int(nc.value)
        p, q = np.zeros(max(m, 1), dtype=np.int32), np.zeros(max(m, 1), dtype=np.int32)
        z, u = np.zeros((max(m, 1), 3)), np.zeros(max(m, 1))
        self._check(self.L.ibm_contact_history(self.h, ctypes.byref(nc), _ptr(p), _ptr(q), _ptr(z), _ptr(u)))
        return p[:m], q[:m], z[:m], u[:m]

    def set_wait_limit(self, iterations=0):
        """Bound of the device-side retry loops of the cluster modes (0 = default)."""
        self._check(self.L.ibm_set_wait_limit(self.h, int(iterations)))

    def particle_clusters(self):
        """Each particle's cluster and its cluster's IBM_PATH_* bits in the last step."""
        n = self.n_p
        cl = np.zeros(max(n, 1), dtype=np.int32)
        path = np.zeros(max(n, 1), dtype=np.int32)
        nc = ctypes.c_int64()
        self._check(self.L.ibm_particle_clusters(self.h, _ptr(cl), _ptr(path), ctypes.byref(nc)))
        return cl[:n], path[:n], int(nc.value)

    def stats(self):
        out = np.zeros(12, dtype=np.int64)
        self._check(self.L.ibm_step_stats(self.h, _ptr(out)))
        keys = ("markers", "clusters", "clusters_smem", "markers_fallback", "largest_cluster_cells",
                "touched_cells", "launches", "threads_per_block", "clusters_one_component", "candidate_pairs",
                "clusters_dsmem", "markers_dsmem")
        return dict(zip(keys, (int(v) for v in out)))


class FluidFields:
    """Device state of one periodic grid: u, ut, uf [3, nz, ny, nx], p, phi [nz, ny, nx], float64."""

    def __init__(self, dims, u=None, p=None, device="cuda"):
        nx, ny, nz = dims
        z = lambda *s: torch.zeros(s, dtype=torch.float64, device=device)
        self.u = z(3, nz, ny, nx) if u is None else torch.as_tensor(u, dtype=torch.float64, device=device).clone()
        self.ut = z(3, nz, ny, nx)
        self.uf = z(3, nz, ny, nx)
        self.p = z(nz, ny, nx) if p is None else torch.as_tensor(p, dtype=torch.float64, device=device).clone()
        self.phi = z(nz, ny, nx)
        for t in (self.u, self.ut, self.uf, self.p, self.phi):
            assert t.is_contiguous()

    def _c(self):
        return _FluidFields(*[t.data_ptr() for t in (self.u, self.ut, self.uf, self.p, self.phi)])


class Fluid:
    """ibm_fluid: the collocated fractional-step solver of Sec. 2.2.1 and 2.2.4 on
    one periodic grid (FP64), on a CUDA stream (torch's current by default)."""

    def __init__(self, dims, h=1.0, nu=0.01, theta=1.0, rtol=0.0, max_cycles=0, profile=False,
                 two_pass_smoother=False, stream=None):
        self.L = load_library()
        self.dims = tuple(int(v) for v in dims)
        self.stream = stream or torch.cuda.current_stream()
        c = _FluidConfig(*self.dims, float(h), float(nu), float(theta), float(rtol), int(max_cycles), int(profile),
                         int(two_pass_smoother))
        hnd = ctypes.c_void_p()
        st = self.L.ibm_fluid_create(ctypes.byref(c), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(hnd))
        if st != 0:
            raise IBMError(st, "ibm_fluid_create rejected the configuration")
        self.h = hnd

    def _check(self, st):
        if st != 0:
            raise IBMError(st, self.L.ibm_fluid_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.ibm_fluid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def predict(self, k, dt, F: FluidFields):
        c = F._c()
        self._check(self.L.ibm_fluid_predict(self.h, int(k), float(dt), ctypes.byref(c)))

    def correct(self, k, dt, F: FluidFields, mean_f=None):
        """mean_f: None, a host sequence of 3 floats, or a device float64 tensor of 3."""
        c = F._c()
        if mean_f is None:
            ptr, dev = None, 0
        elif isinstance(mean_f, torch.Tensor) and mean_f.is_cuda:
            keep = mean_f.contiguous()
            ptr, dev = ctypes.c_void_p(keep.data_ptr()), 1
        else:
            keep = (ctypes.c_double * 3)(*[float(v) for v in mean_f])
            ptr, dev = ctypes.cast(keep, ctypes.c_void_p), 0
        self._check(self.L.ibm_fluid_correct(self.h, int(k), float(dt), ctypes.byref(c), ptr, dev))

    def stage(self, k, dt, F: FluidFields, ctx: "Context | None" = None, f_out=None):
        c = F._c()
        self._check(self.L.ibm_fluid_stage(self.h, ctx.h if ctx is not None else None, int(k), float(dt),
                                           ctypes.byref(c), _ptr(f_out)))

    def step(self, dt, F: FluidFields, ctx: "Context | None" = None):
        for k in range(3):
            self.stage(k, dt, F, ctx)

    def kernel_timing(self, reset=True):
        """(total ms, launches) of the finest-level smoothing launches (profile=True)."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        self._check(self.L.ibm_fluid_kernel_timing(self.h, ctypes.byref(ms), ctypes.byref(n), int(reset)))
        return ms.value, n.value

    def stats(self):
        cyc = (ctypes.c_int64 * 4)()
        res = (ctypes.c_double * 4)()
        lv = ctypes.c_int()
        self._check(self.L.ibm_fluid_stats(self.h, cyc, res, ctypes.byref(lv)))
        return {"cycles": list(cyc), "resid": list(res), "levels": lv.value}


def debug_fail_allocation(n):
    """Test hook: the n-th device allocation of the library from now on fails (0 = off)."""
    st = load_library().ibm_debug_fail_allocation(int(n))
    if st != 0:
        raise IBMError(st, "ibm_debug_fail_allocation")


class IBMForcing(torch.autograd.Function):
    """u^{n_F} = IBM forcing loop(u^0; U_p, omega_p, x_p) with the hand-written adjoint.

    ``ctx_obj`` must be a Context created with requires_grad=True.  Gradients flow to
    u0 (all scenes' fields concatenated is not supported: one scene) and to the FP64
    particle tensors u_p, omega_p, x_p (device, [n_p, 3]).
    """

    @staticmethod
    def forward(ctx, u0, u_p, omega_p, x_p, d_p, ibm_ctx, tau):
        ibm_ctx.set_particles(x_p.detach().contiguous(), u_p.detach().contiguous(),
                              omega_p.detach().contiguous(), d_p.detach().contiguous())
        u = u0.detach().clone()
        ibm_ctx.forcing_step([u], tau)
        ctx.ibm_ctx = ibm_ctx
        return u

    @staticmethod
    def backward(ctx, grad_u):
        gis, gU, gW, gX = ctx.ibm_ctx.backward([grad_u.contiguous()])
        return gis[0], gU, gW, gX, None, None, None
