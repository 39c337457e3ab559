"""CPU checks of the seeded synthetic inputs: the recipes of the workloads
(sizes, counts, gaps, solid fractions, velocity statistics) and the
random-Fourier field, against independent evaluations."""
import math

import numpy as np
import pytest

from paper_2109_03972_gb300 import synth

spatial = pytest.importorskip("scipy.spatial")


def _marker_count(d):
    return int(round(math.pi * d * d))          # N_l = round(pi (d/h)^2), h = 1


def _min_gap(sc):
    """Smallest surface gap over all pairs (minimum image), by a periodic k-d tree."""
    L = np.array(sc.dims, float)
    tree = spatial.cKDTree(np.mod(sc.x_p, L), boxsize=L)
    reach = 2 * sc.d_p.max() + 2.0
    pairs = tree.query_pairs(0.5 * reach + 0.5 * sc.d_p.max(), output_type="ndarray")
    if len(pairs) == 0:
        return np.inf
    dv = sc.x_p[pairs[:, 1]] - sc.x_p[pairs[:, 0]]
    dv -= L * np.round(dv / L)
    gap = np.sqrt((dv * dv).sum(1)) - 0.5 * (sc.d_p[pairs[:, 0]] + sc.d_p[pairs[:, 1]])
    return gap.min()


def test_fourier_field_matches_direct_sum():
    # the separable evaluation against the plain sum of cosines at sampled cells
    dims, seed = (20, 18, 22), 5
    u = synth.fourier_field(dims, seed)
    ks = synth.fourier_wavevectors(16)
    assert len(ks) == 256                        # every integer k with 1 <= |k|^2 <= 16
    ph = np.random.default_rng(seed).uniform(0.0, 2 * math.pi, size=(3, len(ks)))
    rng = np.random.default_rng(1)
    L = np.array(dims, float)
    for _ in range(20):
        i, j, k = (int(rng.integers(0, n)) for n in dims)
        x = (np.array([i, j, k]) + 0.5) / L
        for c in range(3):
            ref = np.cos(2 * math.pi * (ks @ x) + ph[c]).sum()
            assert abs(u[c, k, j, i] - ref) < 1e-10


def test_fourier_field_moments():
    # on a grid that resolves every mode: zero mean, and (Parseval) mean square
    # 256 / 2 plus the cross terms of the modes k and -k, whose phases are
    # independent: sum over pairs of cos(phi_k + phi_-k)
    seed = 9
    u = synth.fourier_field((32, 32, 32), seed)
    ks = synth.fourier_wavevectors(16)
    ph = np.random.default_rng(seed).uniform(0.0, 2 * math.pi, size=(3, len(ks)))
    index = {tuple(k): n for n, k in enumerate(ks)}
    for c in range(3):
        cross = sum(math.cos(ph[c, n] + ph[c, index[tuple(-k)]]) for n, k in enumerate(ks) if tuple(k) > tuple(-k))
        assert abs(u[c].mean()) < 1e-10
        assert abs((u[c] ** 2).mean() - (128.0 + cross)) < 1e-8


def test_bidisperse_bed_recipe():
    W = synth.workload("bidisperse")
    sc = W.scenes[0]
    assert sc.dims == (512, 512, 1024) and W.n_forcing == 3 and W.tau == 0.01
    assert (sc.d_p == 24.0).sum() == 1500 and (sc.d_p == 12.0).sum() == 12000
    assert np.all(sc.d_p[:1500] == 24.0)         # large spheres placed first
    assert sum(_marker_count(d) for d in sc.d_p) == 8139000
    assert _min_gap(sc) >= 1.0 - 1e-9
    solid = (math.pi / 6 * sc.d_p ** 3).sum() / np.prod(sc.dims)
    assert abs(solid - 0.081) < 0.001
    for a in (sc.u_p, sc.omega_p):
        assert abs(a.std() - 0.1) < 0.005 and abs(a.mean()) < 0.005


def test_monodisperse_bed_recipe():
    sc = synth.workload("mono").scenes[0]
    assert sc.dims == (256, 256, 512) and sc.n_p == 2000 and np.all(sc.d_p == 16.0)
    assert _min_gap(sc) >= 1.0 - 1e-9
    solid = (math.pi / 6 * sc.d_p ** 3).sum() / np.prod(sc.dims)
    assert abs(solid - 0.128) < 0.001


def test_batched_scenes_recipe_and_prefix_stability():
    # the draws do not depend on how many scenes are taken
    a = synth.workload("batched", n_scenes=12)
    b = synth.workload("batched", n_scenes=20)
    assert len(a.scenes) == 12 and len(b.scenes) == 20
    for s, t in zip(a.scenes, b.scenes):
        assert s.dims == t.dims and np.array_equal(s.x_p, t.x_p) and np.array_equal(s.d_p, t.d_p)
    for sc in b.scenes:
        assert sc.dims[0] == sc.dims[1] == sc.dims[2] and sc.dims[0] in (32, 48, 64, 96, 128)
        assert 1 <= sc.n_p <= 40
        assert np.all((sc.d_p >= 8.0) & (sc.d_p <= 20.0))
        assert _min_gap(sc) >= 1.0 - 1e-9


def test_seeds_fix_everything():
    a, b = synth.workload("diff128"), synth.workload("diff128")
    c = synth.workload("diff128", seed=7)
    sa, sb, sc = a.scenes[0], b.scenes[0], c.scenes[0]
    assert np.array_equal(sa.x_p, sb.x_p) and np.array_equal(sa.u_p, sb.u_p)
    assert np.array_equal(sa.field()[:, :4], sb.field()[:, :4])
    assert not np.array_equal(sa.x_p, sc.x_p)
