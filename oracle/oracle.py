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
SRC_COLLISION = os.path.join(HERE, "ibm_collision_oracle.c")
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
        newest = max(os.path.getmtime(SRC), os.path.getmtime(SRC_COLLISION))
        if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
            tmp = LIB + f".{os.getpid()}.tmp"
            cc = os.environ.get("CC", "cc")
            subprocess.check_call([cc, "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                                   "-o", tmp, SRC, SRC_COLLISION, "-lm"])
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
        L.orc_tstar.restype, L.orc_tstar.argtypes = _d, [_d]
        L.orc_kn.restype, L.orc_kn.argtypes = _d, [_p, _d, _d, _d, _d, _d, _d, _d, _d]
        L.orc_pair.restype = _d
        L.orc_pair.argtypes = [_p, _p, _p, _p, _p, _p, _d, _d, _d, _d, _p, _d, _p, _p]
        L.orc_collision_forces.restype = None
        L.orc_collision_forces.argtypes = [_l, _p, _p, _p, _p, _p, _p, _p, _p, _l, _p, _p, _p, _p, _p, _p]
        L.orc_particle_substeps.restype = _i
        L.orc_particle_substeps.argtypes = [_l, _p, _p, _p, _d, _i, _p, _p, _p, _p, _p, _p, _p, _l, _p, _p, _p,
                                            _p, _p]
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
    """Grid-pass mean IBM force, Sec. 2.2.4 Eq. (fe_IBM): the negated average
    of f_IBM over all N_i N_j N_k cells, per component.  f: [3][nz][ny][nx]."""
    f = _f64(f)
    return -f.reshape(3, -1).sum(axis=1) / float(f[0].size)


def eps_sep(width=3, h=1.0) -> float:
    """Threshold separation of Sec. 2.2.4: 1.5h for the three-point kernel, 2h for four."""
    return (2.0 if width == 4 else 1.5) * h


def contact_exclusion(dims, x_p, d_p, h=1.0, eps=None, seed=0, ids=None, width=3) -> np.ndarray:
    """Markers left out of f_IBM near contact (Sec. 2.2.5, reading in
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


# ---------------------------------------------------------------- collisions

COLLISION_DEFAULTS = dict(rho_f=1.0, nu_f=0.01, e_dry=0.97, mu_s=0.4, mu_k=0.3, nu_poisson=0.3, t_c=0.1,
                          st_crit=5.0, eps_sep=None, zeta_min=None, lub_c=5.5, g=(0.0, 0.0, 0.0))


def collision_params(h=1.0, **kw):
    """Parameter vector of the collision oracle (ibm_collision_oracle.c):
    eps_sep defaults to 1.5 h, zeta_min to 0.01 h."""
    c = {**COLLISION_DEFAULTS, **kw}
    eps = 1.5 * h if c["eps_sep"] is None else c["eps_sep"]
    zmin = 0.01 * h if c["zeta_min"] is None else c["zeta_min"]
    g = list(c["g"])
    return np.array([c["rho_f"], c["nu_f"], c["e_dry"], c["mu_s"], c["mu_k"], c["nu_poisson"], c["t_c"],
                     c["st_crit"], eps, zmin, c["lub_c"], g[0], g[1], g[2], h], dtype=np.float64)


def collision_tstar(t_c):
    return float(lib().orc_tstar(float(t_c)))


def pair_force(P, dv, u_s, u_o, w_s, w_o, d_s, d_o, rho_s, rho_o, zt=(0.0, 0.0, 0.0), uin=-1.0):
    """Force and torque on `self` from one pair (dv = x_other - x_self); returns (F, T, zeta_n)."""
    F, T = np.zeros(3), np.zeros(3)
    args = [_f64(a, (3,)) for a in (dv, u_s, u_o, w_s, w_o)]
    zt = _f64(zt, (3,))
    z = lib().orc_pair(_ptr(P), *[_ptr(a) for a in args], float(d_s), float(d_o), float(rho_s), float(rho_o),
                       _ptr(zt), float(uin), _ptr(F), _ptr(T))
    return F, T, z


class PairHistory:
    """Contact history of the oracle: canonical pairs p < q with the tangential
    spring (in p's frame) and the impact speed."""

    def __init__(self, cap=100000):
        self.cap = cap
        self.n = ctypes.c_long(0)
        self.p = np.zeros(cap, dtype=np.int64)
        self.q = np.zeros(cap, dtype=np.int64)
        self.z = np.zeros((cap, 3))
        self.u = np.zeros(cap)

    def arrays(self):
        return self.p, self.q, self.z, self.u


def _scene_arrays(dims, scene, n):
    dims = np.ascontiguousarray(np.asarray(dims, dtype=np.int64).reshape(-1, 3))
    sc = np.zeros(n, dtype=np.int32) if scene is None else np.ascontiguousarray(scene, dtype=np.int32)
    return dims, sc


def collision_forces(P, dims, x, u, om, d, rho, hist=None, scene=None):
    """F_c,p and T_c,p of every particle (Eq. f_int), history as given."""
    x, u, om = (_f64(a, (-1, 3)) for a in (x, u, om))
    d, rho = _f64(d, (-1,)), _f64(rho, (-1,))
    n = d.size
    dims, sc = _scene_arrays(dims, scene, n)
    hist = hist or PairHistory(1)
    Fc, Tc = np.zeros((n, 3)), np.zeros((n, 3))
    lib().orc_collision_forces(n, _ptr(dims), _ptr(sc), _ptr(P), _ptr(x), _ptr(u), _ptr(om), _ptr(d), _ptr(rho),
                               hist.n.value, *[_ptr(a) for a in hist.arrays()], _ptr(Fc), _ptr(Tc))
    return Fc, Tc


def particle_substeps(P, dims, x, u, om, d, rho, dt, n_sub=15, F_h=None, T_h=None, hist=None, scene=None):
    """RK3 predictor-corrector sub-steps of Sec. 2.2.10 (oracle); returns
    (x, u, om, hist) with the state advanced by dt."""
    x, u, om = (_f64(a, (-1, 3)).copy() for a in (x, u, om))
    d, rho = _f64(d, (-1,)), _f64(rho, (-1,))
    n = d.size
    dims, sc = _scene_arrays(dims, scene, n)
    hist = hist or PairHistory()
    Fh = None if F_h is None else _f64(F_h, (-1, 3))
    Th = None if T_h is None else _f64(T_h, (-1, 3))
    rc = lib().orc_particle_substeps(n, _ptr(dims), _ptr(sc), _ptr(P), float(dt), int(n_sub), _ptr(Fh), _ptr(Th),
                                     _ptr(x), _ptr(u), _ptr(om), _ptr(d), _ptr(rho), hist.cap,
                                     ctypes.byref(hist.n), *[_ptr(a) for a in hist.arrays()])
    if rc != 0:
        raise MemoryError("oracle collision history full")
    return x, u, om, hist
