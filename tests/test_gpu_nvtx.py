"""Profile bit 3 (NVTX ranges around the step's calls and kernel enqueues):
without a profiler attached the ranges cost nothing visible and change no
result; the step gives the same bytes as without them."""
import numpy as np
import pytest

from paper_2306_07552_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROBOT = I.fetch_like_robot()


@pytest.mark.parametrize("sdf_mode", [0, 1])
def test_nvtx_ranges_change_nothing(sdf_mode):
    from paper_2306_07552_b300 import build, gx
    build.build()
    scenes = [I.room_scene(1000, 2000), I.room_scene(1001, 2000)]
    ss = gx.SceneSet(scenes)
    for k in range(2):
        ss.nsdf_set_weights(k, I.fourier_matrix(7), I.nsdf_init(7 + k))
    n = 64
    kw = dict(img=(64, 64), n_objects=10, seed=2, sdf_mode=sdf_mode, env_scene=np.arange(n) % 2)
    a = gx.Sim(ss, ROBOT, n, **kw)
    b = gx.Sim(ss, ROBOT, n, profile=8, **kw)
    a.reset()
    b.reset()
    acts = I.make_actions(5, n, "uniform", seed=3)
    for t in range(5):
        x = torch.from_numpy(acts[t]).cuda()
        oa, ob = a.step(x), b.step(x)
        torch.cuda.synchronize()
        for k in ("depth", "rgb", "pose", "contact_mask", "event"):
            assert torch.equal(oa[k], ob[k]), (t, k)
    assert a.device_error() == 0 and b.device_error() == 0
    a.close()
    b.close()
    ss.close()
