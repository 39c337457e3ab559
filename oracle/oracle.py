"""ctypes binding of the FP64 CPU oracle (``ibm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg load this module; the GPU library never does.  It builds
``liboracle.so`` next to the C source with plain ``cc -O2 -ffp-contract=off``
and OpenMP (interpolation over markers, spreading over owned z-slabs; the
results do not depend on the thread count).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ibm_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.c_double
_l = ctypes.c_long
_i = ctypes.c_int
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile liboracle.so if missing or older than its source."""
    with _lock:
        if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
            tmp = LIB + f".{os.getpid()}.tmp"
            cc = os.environ.get("CC", "cc")
            subprocess.check_call([cc, "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                                   "-o", tmp, SRC, "-lm"])
            os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        for name in ("ora_phi3", "ora_phi4", "ora_dphi3", "ora_dphi4"):
            f = getattr(L, name)
            f.restype, f.argtypes = _d, [_d]
        L.ora_marker_count.restype, L.ora_marker_count.argtypes = _l, [_d, _d]
        L.ora_marker_volume.restype, L.ora_marker_volume.argtypes = _d, [_d, _d, _l]
        L.ora_marker_dirs.restype, L.ora_marker_dirs.argtypes = None, [_l, _p]
        L.ora_interpolate.restype = _l
        L.ora_interpolate.argtypes = [_i, _i, _l, _l, _l, _d, _l, _p, _p, _p, _p]
        L.ora_spread.restype = _l
        L.ora_spread.argtypes = [_i, _i, _l, _l, _l, _d, _l, _p, _p, _p, _p]
        L.ora_threads.restype, L.ora_threads.argtypes = _i, [_i]
        L.ora_marker_positions.restype = _l
        L.ora_marker_positions.argtypes = [_i, _d, _l, _p, _p, _p, _p]
        L.ora_touched_count.restype = _l
        L.ora_touched_count.argtypes = [_i, _l, _l, _l, _d, _l, _p, _p]
        L.ora_forcing_step.restype = _i
        L.ora_forcing_step.argtypes = [_i, _i, _l, _l, _l, _d, _i, _d, _l,
                                       _p, _p, _p, _p, _p, _p, _p, _p, _p, _p]
        L.ora_forcing_step_masked.restype = _i
        L.ora_forcing_step_masked.argtypes = L.ora_forcing_step.argtypes + [_p]
        L.ora_splitmix64_out.restype, L.ora_splitmix64_out.argtypes = ctypes.c_uint64, [ctypes.c_uint64]
        L.ora_contact_exclusion.restype = _l
        L.ora_contact_exclusion.argtypes = [_l, _l, _l, _d, _l, _p, _p, _d, ctypes.c_uint64, _p, _p]
        L.ora_particle_inertia.restype = None
        L.ora_particle_inertia.argtypes = [_l, _l, _l, _d, _l, _p, _p, _p, _p, _p, _p]
        L.ora_newton_euler.restype = None
        L.ora_newton_euler.argtypes = [_l, _p, _p, _p, _p, _p, _d, _p, _d, _p, _p]
        L.ora_backward.restype = _i
        L.ora_backward.argtypes = [_i, _l, _l, _l, _d, _i, _l, _p, _p, _p, _p,
                                   _p, _p, _p, _p, _p, _p]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def phi3(r): return lib().ora_phi3(float(r))
def phi4(r): return lib().ora_phi4(float(r))
def dphi3(r): return lib().ora_dphi3(float(r))
def dphi4(r): return lib().ora_dphi4(float(r))


def marker_count(d, h=1.0) -> int:
    return int(lib().ora_marker_count(float(d), float(h)))


def marker_volume(d, h=1.0, nl=None) -> float:
    nl = marker_count(d, h) if nl is None else nl
    return float(lib().ora_marker_volume(float(d), float(h), int(nl)))


def marker_dirs(nl) -> np.ndarray:
    t = np.empty((nl, 3))
    lib().ora_marker_dirs(int(nl), _ptr(t))
    return t


def total_markers(d_p, h=1.0) -> int:
    return int(sum(marker_count(d, h) for d in np.asarray(d_p).ravel()))


def interpolate(u, x_p, d_p, h=1.0, width=3, brute=False):
    """U [n_markers, 3] = W u."""
    u = _f64(u)
    nz, ny, nx = u.shape[1:]
    x_p, d_p = _f64(x_p, (-1, 3)), _f64(d_p, (-1,))
    U = np.zeros((total_markers(d_p, h), 3))
    lib().ora_interpolate(width, int(brute), nx, ny, nz, h, d_p.size, _ptr(x_p), _ptr(d_p),
                          _ptr(u), _ptr(U))
    return U


def spread(F, dims, x_p, d_p, h=1.0, width=3, brute=False):
    """f [3, nz, ny, nx] = W^T D F."""
    nx, ny, nz = dims
    x_p, d_p = _f64(x_p, (-1, 3)), _f64(d_p, (-1,))
    F = _f64(F, (-1, 3))
    f = np.zeros((3, nz, ny, nx))
    lib().ora_spread(width, int(brute), nx, ny, nz, h, d_p.size, _ptr(x_p), _ptr(d_p),
                     _ptr(F), _ptr(f))
    return f


def threads(n: int = 0) -> int:
    """OpenMP threads of the oracle; n > 0 sets the count.  Returns the count."""
    return int(lib().ora_threads(int(n)))


def marker_positions(x_p, d_p, h=1.0, width=3):
    """(xi [n,3] grid-unit positions, base [n,3] int64 unwrapped stencil base cells)."""
    x_p, d_p = _f64(x_p, (-1, 3)), _f64(d_p, (-1,))
    n = total_markers(d_p, h)
    xi = np.empty((n, 3))
    base = np.empty((n, 3), dtype=np.int64)
    lib().ora_marker_positions(width, h, d_p.size, _ptr(x_p), _ptr(d_p), _ptr(xi), _ptr(base))
    return xi, base


def touched_count(dims, x_p, d_p, h=1.0, width=3) -> int:
    nx, ny, nz = dims
    x_p, d_p = _f64(x_p, (-1, 3)), _f64(d_p, (-1,))
    return int(lib().ora_touched_count(width, nx, ny, nz, h, d_p.size, _ptr(x_p), _ptr(d_p)))


def forcing_step(u, x_p, u_p, om_p, d_p, h=1.0, n_forcing=3, tau=0.01, width=3,
                 brute=False, want_f=False, want_slip=True, disabled=None):
    """Run the forcing loop on a copy of u.  Returns dict(u, F, T, f, slip).
    disabled: optional per-marker 0/1 array (markers left out of f_IBM)."""
    u = _f64(u).copy()
    nz, ny, nx = u.shape[1:]
    x_p, u_p, om_p = (_f64(a, (-1, 3)) for a in (x_p, u_p, om_p))
    d_p = _f64(d_p, (-1,))
    np_ = d_p.size
    F = np.zeros((np_, 3))
    T = np.zeros((np_, 3))
    f = np.zeros_like(u) if want_f else None
    slip = np.zeros(2) if want_slip else None
    Fabs = np.zeros(np_)
    mask = None if disabled is None else np.ascontiguousarray(disabled, dtype=np.uint8)
    rc = lib().ora_forcing_step_masked(width, int(brute), nx, ny, nz, h, n_forcing, tau, np_,
                                       _ptr(x_p), _ptr(u_p), _ptr(om_p), _ptr(d_p), _ptr(u),
                                       _ptr(F), _ptr(T), _ptr(f), _ptr(slip), _ptr(Fabs), _ptr(mask))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return {"u": u, "F": F, "T": T, "f": f, "slip": slip, "Fabs": Fabs}


def newton_euler(x_p, u_p, om_p, d_p, rho_p, rho_f, g, tau, F, T):
    x, u, w = (_f64(a, (-1, 3)).copy() for a in (x_p, u_p, om_p))
    d_p, rho_p = _f64(d_p, (-1,)), _f64(rho_p, (-1,))
    g = _f64(g, (3,))
    F, T = _f64(F, (-1, 3)), _f64(T, (-1, 3))
    lib().ora_newton_euler(d_p.size, _ptr(x), _ptr(u), _ptr(w), _ptr(d_p), _ptr(rho_p),
                           float(rho_f), _ptr(g), float(tau), _ptr(F), _ptr(T))
    return x, u, w


def backward(u0, x_p, u_p, om_p, d_p, grad_u_out, h=1.0, n_forcing=3, width=3):
    """Gradients of L(u^{n_f}) given dL/du^{n_f}: (grad_u0, gU, gW, gX)."""
    u0 = _f64(u0)
    nz, ny, nx = u0.shape[1:]
    x_p, u_p, om_p = (_f64(a, (-1, 3)) for a in (x_p, u_p, om_p))
    d_p = _f64(d_p, (-1,))
    go = _f64(grad_u_out)
    gi = np.zeros_like(u0)
    n = d_p.size
    gU, gW, gX = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
    rc = lib().ora_backward(width, nx, ny, nz, h, n_forcing, n, _ptr(x_p), _ptr(u_p),
                            _ptr(om_p), _ptr(d_p), _ptr(u0), _ptr(go), _ptr(gi),
                            _ptr(gU), _ptr(gW), _ptr(gX))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return gi, gU, gW, gX


def mean_force(f) -> np.ndarray:
    """Grid-pass mean IBM force, Sec. 2.2.5 Eq. (fe_IBM): the negated average
    of f_IBM over all N_i N_j N_k cells, per component.  f: [3][nz][ny][nx]."""
    f = _f64(f)
    return -f.reshape(3, -1).sum(axis=1) / float(f[0].size)


def eps_sep(width=3, h=1.0) -> float:
    """Threshold separation of Sec. 2.2.6: 1.5h for the three-point kernel, 2h for four."""
    return (2.0 if width == 4 else 1.5) * h


def contact_exclusion(dims, x_p, d_p, h=1.0, eps=None, seed=0, ids=None, width=3) -> np.ndarray:
    """Markers left out of f_IBM near contact (Sec. 2.2.6, reading in
    ora_contact_exclusion): bool [n_markers], particle-then-l order."""
    nx, ny, nz = dims
    x_p = _f64(x_p, (-1, 3))
    d_p = _f64(d_p, (-1,))
    n = total_markers(d_p, h)
    out = np.zeros(n, dtype=np.uint8)
    idv = None if ids is None else np.ascontiguousarray(ids, dtype=np.int64)
    e = eps_sep(width, h) if eps is None else float(eps)
    got = lib().ora_contact_exclusion(nx, ny, nz, h, d_p.size, _ptr(x_p), _ptr(d_p), e, int(seed) & (2**64 - 1),
                                      _ptr(idv), _ptr(out))
    if got != n:
        raise MemoryError("oracle allocation failed")
    return out.astype(bool)


def particle_inertia(u, x_p, d_p, h=1.0):
    """Fluid inertia inside each particle, Sec. 2.2.9: dict(Iu [n,3], Ir [n,3], V [n])
    (reading and quadrature in ora_particle_inertia)."""
    u = _f64(u)
    nz, ny, nx = u.shape[1:]
    x_p, d_p = _f64(x_p, (-1, 3)), _f64(d_p, (-1,))
    n = d_p.size
    Iu, Ir, V = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
    lib().ora_particle_inertia(nx, ny, nz, h, n, _ptr(x_p), _ptr(d_p), _ptr(u), _ptr(Iu), _ptr(Ir), _ptr(V))
    return {"Iu": Iu, "Ir": Ir, "V": V}


def splitmix64(x: int) -> int:
    """SplitMix64 output for state x (the counter-based coin of the pair choice)."""
    return int(lib().ora_splitmix64_out(int(x) & (2**64 - 1)))
