"""Seeded synthetic inputs for the immersed-boundary forcing step.

This module only draws inputs: a periodic random-Fourier velocity field,
non-overlapping sphere placements (random sequential addition), particle
velocities and loss weights.  It contains none of the forcing-step arithmetic
(no delta kernel, no markers, no interpolation or spreading), so both the GPU
library's tests/benchmarks and the CPU oracle can consume the same inputs.

Workload shapes follow the particle beds of the paper (Sec. 3.5-3.6: mono- and
bidisperse fluidised beds with d_p/h of order 10-25 on periodic grids); the
concrete sizes are the synthetic stand-ins named in each ``workload()`` entry.
All generators use numpy's PCG64 (``default_rng(seed)``).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * math.pi


def fourier_wavevectors(kmax2: int = 16) -> np.ndarray:
    """Every integer wavevector k with 1 <= |k|^2 <= kmax2, lexicographic (kx, ky, kz)."""
    kmax = int(math.isqrt(kmax2))
    ks = []
    for kx in range(-kmax, kmax + 1):
        for ky in range(-kmax, kmax + 1):
            for kz in range(-kmax, kmax + 1):
                k2 = kx * kx + ky * ky + kz * kz
                if 1 <= k2 <= kmax2:
                    ks.append((kx, ky, kz))
    return np.asarray(ks, dtype=np.int64)


def fourier_field(dims, seed: int, h: float = 1.0, kmax2: int = 16) -> np.ndarray:
    """Periodic random-Fourier velocity field, float64, layout [3][nz][ny][nx] (x fastest).

    Per component c: u_c(x) = sum_k cos(2*pi*(kx*x/Lx + ky*y/Ly + kz*z/Lz) + phi_{k,c})
    over all integer k with 1 <= |k|^2 <= kmax2 (unit amplitude per mode), phases
    uniform on [0, 2*pi), evaluated at cell centres x = (i + 1/2) h.
    The sum is evaluated separably (z, then y, then a real matmul over x), which is
    exact up to rounding.
    """
    nx, ny, nz = (int(d) for d in dims)
    rng = np.random.default_rng(seed)
    ks = fourier_wavevectors(kmax2)
    nk = ks.shape[0]
    phases = rng.uniform(0.0, TWO_PI, size=(3, nk))
    kmax = int(math.isqrt(kmax2))
    nkk = 2 * kmax + 1

    def modes(n, L):
        pos = (np.arange(n, dtype=np.float64) + 0.5) * h
        kk = np.arange(-kmax, kmax + 1, dtype=np.float64)
        return np.exp(1j * TWO_PI * np.outer(kk, pos) / L)  # [nkk, n]

    Ex, Ey, Ez = modes(nx, nx * h), modes(ny, ny * h), modes(nz, nz * h)
    out = np.empty((3, nz, ny, nx), dtype=np.float64)
    for c in range(3):
        coef = np.zeros((nkk, nkk, nkk), dtype=np.complex128)
        coef[ks[:, 0] + kmax, ks[:, 1] + kmax, ks[:, 2] + kmax] = np.exp(1j * phases[c])
        G = np.einsum("abc,cz->abz", coef, Ez)           # [kx, ky, z]
        H = np.einsum("abz,by->azy", G, Ey)              # [kx, z, y]
        Hr = H.reshape(nkk, nz * ny)
        # u = Re(sum_kx H[kx] Ex[kx]) = Re(H)^T Re(Ex) - Im(H)^T Im(Ex)
        A = np.concatenate([Hr.real, -Hr.imag], axis=0).T  # [nz*ny, 2*nkk]
        B = np.concatenate([Ex.real, Ex.imag], axis=0)       # [2*nkk, nx]
        out[c] = (A @ B).reshape(nz, ny, nx)
    return out


def rsa_spheres(dims, diameters, seed: int, gap: float = 1.0, h: float = 1.0,
                max_attempts: int = 1000):
    """Random sequential addition of spheres in a periodic box.

    Spheres are placed in the order given (callers pass large spheres first).
    Centres are uniform on [0, L); a candidate is rejected if its surface-to-surface
    distance (periodic minimum image) to any placed sphere is below ``gap``.
    A sphere that fails ``max_attempts`` draws is dropped.
    Returns (centres [n,3] float64, kept diameters [n] float64).
    """
    L = np.array([dims[0] * h, dims[1] * h, dims[2] * h], dtype=np.float64)
    diameters = np.asarray(diameters, dtype=np.float64)
    rng = np.random.default_rng(seed)
    if diameters.size == 0:
        return np.zeros((0, 3)), diameters
    cs = float(diameters.max() + gap)
    ncell = np.maximum((L // cs).astype(np.int64), 1)
    csz = L / ncell
    buckets: dict = {}
    centres, kept = [], []
    for d in diameters:
        for _ in range(max_attempts):
            x = rng.uniform(0.0, 1.0, size=3) * L
            ci = np.minimum((x // csz).astype(np.int64), ncell - 1)
            # neighbouring buckets, each once (boxes with fewer than 3 buckets per axis
            # would otherwise list the same bucket several times)
            keys = {((int(ci[0]) + ox) % int(ncell[0]), (int(ci[1]) + oy) % int(ncell[1]),
                     (int(ci[2]) + oz) % int(ncell[2]))
                    for ox in (-1, 0, 1) for oy in (-1, 0, 1) for oz in (-1, 0, 1)}
            ok = True
            for key in keys:
                for j in buckets.get(key, ()):
                    dv = x - centres[j]
                    dv -= L * np.round(dv / L)
                    if math.sqrt(float(dv @ dv)) < 0.5 * (d + kept[j]) + gap:
                        ok = False
                        break
                if not ok:
                    break
            if ok:
                key = (int(ci[0]), int(ci[1]), int(ci[2]))
                buckets.setdefault(key, []).append(len(centres))
                centres.append(x)
                kept.append(float(d))
                break
    return np.asarray(centres, dtype=np.float64).reshape(-1, 3), np.asarray(kept)


@dataclass
class Scene:
    dims: tuple                      # (nx, ny, nz)
    x_p: np.ndarray                  # [n,3] float64 centres
    d_p: np.ndarray                  # [n] float64 diameters
    u_p: np.ndarray                  # [n,3]
    omega_p: np.ndarray              # [n,3]
    rho_p: np.ndarray                # [n]
    field_seed: int
    h: float = 1.0

    @property
    def n_p(self) -> int:
        return int(self.x_p.shape[0])

    def field(self) -> np.ndarray:
        return fourier_field(self.dims, self.field_seed, self.h)


@dataclass
class Workload:
    name: str
    scenes: list
    n_forcing: int = 3
    tau: float = 0.01
    rho_f: float = 1.0
    g: tuple = (0.0, 0.0, -1.0e-3)
    meta: dict = field(default_factory=dict)


def particle_state(n, seed, rho_ratio=1.3, vel_std=0.1):
    """U_p, omega_p ~ N(0, vel_std) per component; rho_p = rho_ratio (rho_f = 1)."""
    rng = np.random.default_rng(seed)
    u_p = rng.normal(0.0, vel_std, size=(n, 3))
    om = rng.normal(0.0, vel_std, size=(n, 3))
    return u_p, om, np.full(n, rho_ratio, dtype=np.float64)


def make_scene(dims, diameters, seed, gap=1.0, h=1.0, max_attempts=1000):
    x_p, d_p = rsa_spheres(dims, diameters, seed=seed, gap=gap, h=h,
                           max_attempts=max_attempts)
    u_p, om, rho = particle_state(x_p.shape[0], seed + 1)
    return Scene(tuple(int(v) for v in dims), x_p, d_p, u_p, om, rho,
                 field_seed=seed + 2, h=h)


def workload(name: str, seed: int = 2109, n_scenes: int = 512) -> Workload:
    """The named synthetic workloads (all periodic, h = 1, n_F = 3, tau = 0.01).

    single64   : 64^3 grid, one sphere D=16 at a random position (~804 markers)
    mono       : 256x256x512, 2000 spheres D=16, gap >= 1h (~12.8% solid)
    bidisperse : 512x512x1024, 1500 spheres D=24 then 12000 spheres D=12, gap >= 1h
    batched    : 512 scenes, edge in {32,48,64,96,128}, n in U{1..40}, D ~ U[8,20]
                 (the first n_scenes of them; the draws do not depend on n_scenes)
    diff128    : 128^3, 150 spheres D=16 (differentiation workload)
    small      : 40x36x44, 6 spheres D in {6,8,10} (fast parity case, ragged dims)
    """
    if name == "single64":
        return Workload(name, [make_scene((64, 64, 64), [16.0], seed)])
    if name == "mono":
        return Workload(name, [make_scene((256, 256, 512), [16.0] * 2000, seed)])
    if name == "bidisperse":
        ds = [24.0] * 1500 + [12.0] * 12000
        return Workload(name, [make_scene((512, 512, 1024), ds, seed)])
    if name == "diff128":
        return Workload(name, [make_scene((128, 128, 128), [16.0] * 150, seed)])
    if name == "small":
        return Workload(name, [make_scene((40, 36, 44), [10.0, 8.0, 8.0, 6.0, 6.0, 6.0], seed)])
    if name == "batched":
        rng = np.random.default_rng(seed)
        edges = rng.choice([32, 48, 64, 96, 128], size=512)
        counts = rng.integers(1, 41, size=512)
        scenes = []
        for s in range(min(512, n_scenes)):
            ds = np.sort(rng.uniform(8.0, 20.0, size=int(counts[s])))[::-1]
            e = int(edges[s])
            scenes.append(make_scene((e, e, e), ds, seed + 7 * s + 11))
        return Workload(name, scenes)
    raise KeyError(name)


def loss_weights(dims, seed: int) -> np.ndarray:
    """Loss weight field w ~ U[0, 1) per cell, layout [nz][ny][nx]."""
    nx, ny, nz = dims
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=(nz, ny, nx))
