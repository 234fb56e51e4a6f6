"""One persistent launch per step (gx_config.fused_step): the masked resets,
the physics and the rendering of a step in one cooperative launch, separated
by grid-wide barriers.  It runs the same per-environment code as the separate
kernels, so its results must equal theirs bit for bit, step after step, with
resets in between, graph replay, the paper's heuristics, the broad-phase,
more objects than fit the shared-memory staging, and the autotuner; and they
must match the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2306_07552_b300 import inputs as I
from tests.parity import Tally, check_image, check_step

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROBOT = I.fetch_like_robot()
KEYS = ["depth", "rgb", "pose", "obj_pos", "held", "contact_mask", "contact_flags", "event",
        "reward", "task_obs", "success"]


@pytest.fixture(scope="module")
def rooms():
    from paper_2306_07552_b300 import build, gx
    build.build()
    scenes = [I.room_scene(1000, 2000), I.room_scene(1001, 6000), I.room_scene(1002, 1000)]
    ss = gx.SceneSet(scenes)
    yield gx, scenes, ss
    ss.close()


def _pair(gx, ss, n, fused_kw=None, **kw):
    a = gx.Sim(ss, ROBOT, n, fused_step=True, **{**kw, **(fused_kw or {})})
    b = gx.Sim(ss, ROBOT, n, **kw)
    a.reset()
    b.reset()
    return a, b


def _compare(a, b, steps, n, seed, p_reset=0.2, stream=None):
    acts = I.make_actions(steps, n, "gaussian", seed=seed)
    rng = np.random.default_rng(seed)
    x = torch.empty((n, 11), dtype=torch.float32, device="cuda")
    m = torch.empty((n,), dtype=torch.uint8, device="cuda")
    for t in range(steps):
        x.copy_(torch.from_numpy(acts[t]))
        m.copy_(torch.from_numpy((rng.random(n) < p_reset).astype(np.uint8)))
        oa = a.step_reset(m, x, stream=stream)
        ob = b.step_reset(m, x, stream=stream)
        torch.cuda.synchronize()
        for k in KEYS:
            assert torch.equal(oa[k], ob[k]), (t, k)
    sa, sb = a.state_arrays(), b.state_arrays()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k


def test_fused_equals_separate_launches_with_resets_and_graphs(rooms):
    gx, scenes, ss = rooms
    n = 300
    es = np.arange(n) % 3
    kw = dict(img=(64, 64), n_objects=16, seed=4, env_scene=es)
    a, b = _pair(gx, ss, n, **kw)
    _compare(a, b, 10, n, seed=5)
    a.close()
    b.close()
    # graph replay of the fused launch (on a side stream) against plain launches
    a, b = _pair(gx, ss, n, fused_kw=dict(use_graph=True), **kw)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        _compare(a, b, 8, n, seed=6, stream=stream)
    a.close()
    b.close()


def test_fused_with_heuristics_broadphase_and_many_objects(rooms):
    gx, scenes, ss = rooms
    # heuristics and the broad-phase, 40 objects
    n = 96
    kw = dict(img=(64, 64), n_objects=40, seed=7, heuristics=3, broadphase=True,
              render_robot=True)
    a, b = _pair(gx, ss, n, **kw)
    _compare(a, b, 8, n, seed=8)
    a.close()
    b.close()
    # more objects than the shared-memory staging holds (global scratch)
    n = 12
    kw = dict(img=(32, 32), n_objects=200, obj_radius=(0.03, 0.035), seed=9)
    a, b = _pair(gx, ss, n, **kw)
    _compare(a, b, 5, n, seed=10, p_reset=0.3)
    a.close()
    b.close()


def test_fused_matches_the_oracle_and_autotunes(rooms):
    gx, scenes, ss = rooms
    n, M, W = 32, 10, 64
    sim = gx.Sim(ss, ROBOT, n, img=(W, W), n_objects=M, seed=11, env_scene=np.zeros(n, np.int32),
                 fused_step=True)
    sim.reset()
    orc = O.Oracle(ROBOT, scenes[0], I.icosahedron(), I.object_colors(256))
    acts = I.make_actions(6, n, "uniform", seed=12)
    tally = Tally()
    for t in range(6):
        before = {k: v.copy() for k, v in sim.state_arrays().items()}
        out = sim.step(torch.from_numpy(acts[t]).cuda())
        torch.cuda.synchronize()
        after = sim.state_arrays()
        check_step(orc, before, after, out, acts[t], range(n), M, tally)
        for e in (0, 13, 31):
            check_image(orc, after, out, e, W, W, M, tally)
    print(tally)
    assert tally.envs - tally.near_band_flips >= 0.95 * tally.envs and tally.pixels > 0
    best = sim.autotune(torch.from_numpy(acts[0]).cuda(), steps=2)
    assert best["ms_per_step"] > 0
    assert sim.device_error() == 0
    sim.close()


def test_fused_refused_with_neural_sdf_or_boxes(rooms):
    gx, scenes, ss = rooms
    for kw in (dict(sdf_mode=1), dict(object_boxes=True)):
        with pytest.raises(gx.GxError):
            gx.Sim(ss, ROBOT, 4, img=(32, 32), n_objects=4, fused_step=True, **kw)
