"""GPU tests of the batched-scene machinery: CUDA-graph replay of the forcing
step and the autotuned kernel variant, through the C ABI."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2109_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2109_03972_gb300 import ibm, synth  # noqa: E402
from _helpers import f32_round  # noqa: E402


def _scenes(n=12):
    # the first scenes of the batched workload (uneven edges, particle counts and diameters)
    return synth.workload("batched", n_scenes=n).scenes


def _context(scenes, **kw):
    cfg = ibm.Config(dims=[sc.dims for sc in scenes], n_forcing=3, precision=ibm.IBM_FP32,
                     spread_mode=ibm.IBM_SPREAD_DETERMINISTIC, max_particles=sum(sc.n_p for sc in scenes), **kw)
    ctx = ibm.Context(cfg)
    x = np.concatenate([sc.x_p for sc in scenes])
    up = np.concatenate([sc.u_p for sc in scenes])
    om = np.concatenate([sc.omega_p for sc in scenes])
    d = np.concatenate([sc.d_p for sc in scenes])
    rho = np.concatenate([sc.rho_p for sc in scenes])
    sid = np.concatenate([np.full(sc.n_p, i, np.int32) for i, sc in enumerate(scenes)])
    ctx.set_particles(x, up, om, d, rho, scene_of=sid)
    return ctx


def _fields(scenes):
    return [torch.from_numpy(f32_round(sc.field())).cuda().float().contiguous() for sc in scenes]


def _steps_agree(scenes, n_steps, exact, **kw):
    ua, ub = _fields(scenes), _fields(scenes)
    eager = _context(scenes)
    other = _context(scenes, **kw)
    for step in range(n_steps):   # eager, capture + replay, replays
        eager.forcing_step(ua, 0.01)
        other.forcing_step(ub, 0.01)
        torch.cuda.synchronize()
        for a, b in zip(ua, ub):
            if exact:
                assert torch.equal(a, b), step
            else:
                assert (a - b).abs().max().item() <= 2e-5 * a.abs().max().item(), step
        la, lb = eager.particle_loads(), other.particle_loads()
        if exact:
            assert np.array_equal(la["F"], lb["F"]) and np.array_equal(la["T"], lb["T"])
        else:
            assert np.abs(la["F"] - lb["F"]).max() <= 1e-4 * np.abs(la["F"]).sum(1).max()
    return eager, other


def test_graph_replay_is_bitwise_the_eager_step():
    # deterministic mode is bit-reproducible (the shared-memory kernel and the
    # fixed-point fallback alike), so the replayed graph must give the eager bits
    scenes = [synth.workload(n).scenes[0] for n in ("small", "single64", "diff128")]
    eager, graph = _steps_agree(scenes, 5, True, use_graph=True)
    assert eager.stats()["markers_fallback"] > 0
    assert graph.stats()["launches"] == eager.stats()["launches"]


def test_graph_replay_on_batched_scenes():
    # small dense periodic boxes, many clusters on the fallback path
    _steps_agree(_scenes(), 5, True, use_graph=True)


def test_autotuned_variant_matches_fixed_variant():
    scenes = _scenes()
    ua, ub = _fields(scenes), _fields(scenes)
    fixed = _context(scenes)
    tuned = _context(scenes, threads_per_block=-1, use_graph=True)
    for _ in range(7):                        # 4 tuning steps, a capture, two replays
        fixed.forcing_step(ua, 0.01)
        tuned.forcing_step(ub, 0.01)
        torch.cuda.synchronize()
        for a, b in zip(ua, ub):
            scale = a.abs().max().item()
            assert (a - b).abs().max().item() <= 2e-5 * scale
    assert tuned.stats()["threads_per_block"] in (512, 1024)


def test_graph_follows_new_particle_sets():
    # a new particle set (other count, other buffers) must not replay the old
    # graph: the step runs eagerly, is captured again, and matches the eager context
    a = [synth.workload("small").scenes[0]]
    b = [synth.workload("single64").scenes[0]]
    dims = [a[0].dims]
    cfg = dict(dims=dims, n_forcing=3, precision=ibm.IBM_FP32, spread_mode=ibm.IBM_SPREAD_DETERMINISTIC,
               max_particles=max(a[0].n_p, b[0].n_p) + 4)
    eager, graph = ibm.Context(ibm.Config(**cfg)), ibm.Context(ibm.Config(**cfg, use_graph=True))
    ua, ub = _fields(a), _fields(a)
    for scenes in (a, b, a):
        sc = scenes[0]
        x = sc.x_p % np.array(dims[0])            # positions inside the first scene's box
        for ctx in (eager, graph):
            ctx.set_particles(x, sc.u_p, sc.omega_p, sc.d_p)
        for _ in range(4):
            eager.forcing_step(ua, 0.01)
            graph.forcing_step(ub, 0.01)
            torch.cuda.synchronize()
            assert torch.equal(ua[0], ub[0])
            assert np.array_equal(eager.particle_loads()["F"], graph.particle_loads()["F"])
