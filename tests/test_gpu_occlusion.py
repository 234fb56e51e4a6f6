"""Occlusion culling of clusters (gx_config.occlusion_cull): a cluster or an
object is skipped only when it lies strictly behind the depth bound of every
8x8 tile its screen rectangle touches, so the images must equal those of the
unculled rasteriser bit for bit -- step after step, with resets, graph replay,
the counting variant of the kernel and the autotuner -- while many clusters
are in fact skipped; and they must match the FP64 oracle."""
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
def apartments():
    from paper_2306_07552_b300 import build, gx
    build.build()
    w = I.WORKLOADS["uneven8192"]
    scenes = I.make_scenes(w, only=[0, 7, 21])
    ss = gx.SceneSet(scenes)
    yield gx, scenes, ss
    ss.close()


def _run_pair(gx, ss, n, steps, act_seed, a_kw, b_kw, **kw):
    a = gx.Sim(ss, ROBOT, n, **kw, **a_kw)
    b = gx.Sim(ss, ROBOT, n, **kw, **b_kw)
    a.reset()
    b.reset()
    acts = I.make_actions(steps, n, "gauss0.5", seed=act_seed)
    rng = np.random.default_rng(act_seed)
    x = torch.empty((n, 11), dtype=torch.float32, device="cuda")
    m = torch.empty((n,), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for t in range(steps):
            x.copy_(torch.from_numpy(acts[t]))
            m.copy_(torch.from_numpy((rng.random(n) < 0.1).astype(np.uint8)))
            oa = a.step_reset(m, x, stream=stream)
            ob = b.step_reset(m, x, stream=stream)
            torch.cuda.synchronize()
            for k in KEYS:
                assert torch.equal(oa[k], ob[k]), (t, k)
    return a, b


def test_occlusion_culling_leaves_images_unchanged(apartments):
    gx, scenes, ss = apartments
    n = 192
    es = np.arange(n) % 3
    kw = dict(img=(128, 128), n_objects=40, seed=3, env_scene=es)
    # graph-replayed culled context against the plain one
    a, b = _run_pair(gx, ss, n, 12, 4, dict(occlusion_cull=True, use_graph=True), {}, **kw)
    a.close()
    b.close()
    # the counting variant: identical images too, and clusters really skipped
    a, b = _run_pair(gx, ss, n, 6, 5, dict(occlusion_cull=True, profile=2), dict(profile=2), **kw)
    ca, cb = a.raster_counters(), b.raster_counters()
    print("culled:", {k: ca[k] / (6 * n) for k in ("clusters_drawn", "clusters_occluded",
                                                    "tris_seen", "fragments")},
          "plain:", {k: cb[k] / (6 * n) for k in ("clusters_drawn", "tris_seen", "fragments")})
    assert ca["clusters_occluded"] > 0.1 * ca["clusters_drawn"]
    assert ca["clusters_drawn"] < 0.9 * cb["clusters_drawn"]
    assert ca["fragments"] < cb["fragments"]
    a.close()
    b.close()
    # FP16 depth and a 256 x 192 image (more tiles than 128 x 128 has)
    kw2 = dict(img=(256, 192), n_objects=12, seed=6, env_scene=np.arange(24) % 3, depth_fp16=True)
    a, b = _run_pair(gx, ss, 24, 5, 7, dict(occlusion_cull=True), {}, **kw2)
    a.close()
    b.close()


def test_occlusion_culling_matches_the_oracle_and_autotunes(apartments):
    gx, scenes, ss = apartments
    n, M, W = 24, 20, 128
    sim = gx.Sim(ss, ROBOT, n, img=(W, W), n_objects=M, seed=9,
                 env_scene=np.zeros(n, np.int32), occlusion_cull=True)
    sim.reset()
    orc = O.Oracle(ROBOT, scenes[0], I.icosahedron(), I.object_colors(256))
    acts = I.make_actions(5, n, "gauss0.5", seed=10)
    tally = Tally()
    for t in range(5):
        before = {k: v.copy() for k, v in sim.state_arrays().items()}
        out = sim.step(torch.from_numpy(acts[t]).cuda())
        torch.cuda.synchronize()
        after = sim.state_arrays()
        check_step(orc, before, after, out, acts[t], range(n), M, tally)
        for e in (0, 11, 23):
            check_image(orc, after, out, e, W, W, M, tally)
    print(tally)
    assert tally.pixels > 0
    best = sim.autotune(torch.from_numpy(acts[0]).cuda(), steps=2)
    print("autotune:", best)
    assert best["occlusion_cull"] in (0, 1)
    assert sim.device_error() == 0
    sim.close()


def test_occlusion_culling_refused_with_fused_step_or_boxes(apartments):
    gx, scenes, ss = apartments
    for kw in (dict(fused_step=True), dict(object_boxes=True)):
        with pytest.raises(gx.GxError):
            gx.Sim(ss, ROBOT, 4, img=(32, 32), n_objects=4, occlusion_cull=True, **kw)
