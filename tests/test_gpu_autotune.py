"""The rasteriser's work order and the autotuner: every candidate setting must
render the same images (coverage and winners do not depend on the order in
which environments are drawn or on which path rasterises a triangle), and the
autotuner must leave the state as it found it."""
import numpy as np
import pytest

from paper_2306_07552_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROBOT = I.fetch_like_robot()
KEYS = ["depth", "rgb", "pose", "obj_pos", "held", "contact_mask", "contact_flags", "event"]


@pytest.fixture(scope="module")
def uneven():
    from paper_2306_07552_b300 import build, gx
    build.build()
    # scenes of very different size: the costliest-first order is on by default
    scenes = [I.room_scene(1000, 1000), I.room_scene(1001, 12000), I.room_scene(1002, 4000)]
    ss = gx.SceneSet(scenes)
    yield gx, ss
    ss.close()


def test_autotune_restores_state_and_changes_no_result(uneven):
    gx, ss = uneven
    n = 300
    es = np.arange(n) % 3
    kw = dict(img=(64, 64), n_objects=16, seed=4, env_scene=es)
    a = gx.Sim(ss, ROBOT, n, **kw)
    b = gx.Sim(ss, ROBOT, n, **kw)
    a.reset()
    b.reset()
    acts = I.make_actions(12, n, "gaussian", seed=5)
    for t in range(4):
        x = torch.from_numpy(acts[t]).cuda()
        a.step(x)
        b.step(x)
    torch.cuda.synchronize()
    before = {k: v.copy() for k, v in b.state_arrays().items()}
    best = b.autotune(torch.from_numpy(acts[4]).cuda(), steps=2)
    torch.cuda.synchronize()
    print("autotune:", best)
    after = b.state_arrays()
    for k in before:
        assert np.array_equal(before[k], after[k]), k
    assert best["ms_per_step"] > 0 and best["raster_ctas"] > 0
    for t in range(4, 12):
        x = torch.from_numpy(acts[t]).cuda()
        oa, ob = a.step(x), b.step(x)
        torch.cuda.synchronize()
        for k in KEYS:
            assert torch.equal(oa[k], ob[k]), (t, k)
    a.close()
    b.close()
