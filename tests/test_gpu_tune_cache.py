"""Autotuning results kept in a JSON cache keyed by the configuration, the
scene set and the GPU: a second context with the same key takes the stored
rasteriser setting without timing candidates (gx_apply_tune) and renders the
same images; another configuration misses and adds its own entry; settings
that do not fit a context are refused with GX_EINVAL."""
import json

import numpy as np
import pytest

from paper_2306_07552_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROBOT = I.fetch_like_robot()
GX_EINVAL = 1


def test_tuning_cache_hit_miss_and_refusals(tmp_path):
    from paper_2306_07552_b300 import build, gx
    build.build()
    scenes = I.make_scenes(I.WORKLOADS["apartments4096"], only=[0, 1])
    ss = gx.SceneSet(scenes)
    cache = str(tmp_path / "tune.json")
    kw = dict(img=(128, 128), n_objects=20, seed=4)
    n = 512
    acts = torch.from_numpy(I.make_actions(1, n, "gauss0.5", seed=1)[0]).cuda()
    a = gx.Sim(ss, ROBOT, n, **kw)
    a.reset()
    ra = a.autotune(acts, steps=2, cache=cache)
    assert "cached" not in ra
    table = json.load(open(cache))
    assert list(table) == [a.tune_key()]
    b = gx.Sim(ss, ROBOT, n, **kw)
    b.reset()
    rb = b.autotune(acts, steps=2, cache=cache)
    assert rb.get("cached") is True
    assert {k: rb[k] for k in ra} == ra
    # the same steps from the same state render the same images under both
    oa, ob = a.step(acts), b.step(acts)
    torch.cuda.synchronize()
    for k in ("depth", "rgb", "pose", "contact_mask"):
        assert torch.equal(oa[k], ob[k]), k
    # another batch size is another key: tuned and stored beside the first
    c = gx.Sim(ss, ROBOT, 256, **kw)
    c.reset()
    rc = c.autotune(acts[:256], steps=2, cache=cache)
    assert "cached" not in rc
    assert len(json.load(open(cache))) == 2
    # settings that do not fit the context
    for bad in (dict(ra, raster_warps=5), dict(ra, raster_ctas=10**6), dict(ra, raster_ctas=0),
                dict(ra, occlusion_cull=1), dict(ra, order_costliest_first=2),
                dict(ra, small_tri_px=-1)):
        with pytest.raises(gx.GxError) as ei:
            a.apply_tune(bad)
        assert ei.value.status == GX_EINVAL
    a.apply_tune(ra)
    out = a.step(acts)
    torch.cuda.synchronize()
    assert np.isfinite(out["depth"].float().cpu().numpy()).all()
    assert a.device_error() == 0 and b.device_error() == 0 and c.device_error() == 0
    for s in (a, b, c):
        s.close()
    ss.close()
