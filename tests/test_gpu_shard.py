"""A batch split into shards (one context per shard, as one per GPU) evolves
exactly like one context over the whole batch: each shard context holds only
the scenes its environments use and draws its resets from the global
environment indices (gx_config.env_offset), so states and outputs agree bit
for bit, environment by environment.  Both sides run on the one GPU here;
across GPUs nothing else changes (no data is exchanged)."""
import dataclasses

import numpy as np
import pytest

from paper_2306_07552_b300 import inputs as I
from paper_2306_07552_b300 import shard

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROBOT = I.fetch_like_robot()
KEYS = ["depth", "rgb", "pose", "obj_pos", "held", "contact_mask", "contact_flags", "event",
        "reward", "task_obs", "success"]


def test_two_shards_equal_the_whole_batch():
    from paper_2306_07552_b300 import build, gx
    build.build()
    w = dataclasses.replace(I.WORKLOADS["room16"], n_envs=96, n_scenes=3, tri_range=(1500, 1500))
    n, steps = w.n_envs, 8
    kw = dict(img=(64, 64), n_objects=w.n_objects, obj_radius=w.obj_radius, seed=w.reset_seed)
    full_set = gx.SceneSet(I.make_scenes(w))
    full = gx.Sim(full_set, ROBOT, n, **kw)
    plans = [shard.plan(n, w.n_scenes, 2, r) for r in range(2)]
    sets = [gx.SceneSet(I.make_scenes(w, only=p.scenes)) for p in plans]
    parts = [gx.Sim(s, ROBOT, p.count, env_scene=p.env_scene, env_offset=p.first, **kw)
             for s, p in zip(sets, plans)]
    assert plans[0].scenes == (0, 1) and plans[1].scenes == (1, 2)
    acts = I.make_actions(steps, n, "uniform", seed=3)
    rng = np.random.default_rng(5)
    full.reset()
    for s in parts:
        s.reset()
    for t in range(steps):
        if t == 4:   # a masked reset in the middle: same environments on both sides
            m = (rng.random(n) < 0.3).astype(np.uint8)
            full.reset(torch.from_numpy(m).cuda())
            for s, p in zip(parts, plans):
                s.reset(torch.from_numpy(np.ascontiguousarray(m[p.first:p.first + p.count])).cuda())
        of = full.step(torch.from_numpy(acts[t]).cuda())
        ops = [s.step(torch.from_numpy(np.ascontiguousarray(acts[t, p.first:p.first + p.count]))
                      .cuda()) for s, p in zip(parts, plans)]
        torch.cuda.synchronize()
        for k in KEYS:
            whole = of[k]
            joined = torch.cat([o[k] for o in ops])
            assert torch.equal(whole, joined), (t, k)
    sf = full.state_arrays()
    for s, p in zip(parts, plans):
        sp = s.state_arrays()
        for k, v in sp.items():
            ref = sf[k]
            sl = (ref[:, p.first:p.first + p.count] if k in ("q", "c_off", "p_pre", "r_off")
                  else ref[p.first:p.first + p.count])
            assert np.array_equal(v, sl), k
    # the reset draws really depend on the global index: the second shard
    # without its offset places objects differently
    wrong = gx.Sim(sets[1], ROBOT, plans[1].count, env_scene=plans[1].env_scene, **kw)
    wrong.reset()
    torch.cuda.synchronize()
    fresh = gx.Sim(sets[1], ROBOT, plans[1].count, env_scene=plans[1].env_scene,
                   env_offset=plans[1].first, **kw)
    fresh.reset()
    torch.cuda.synchronize()
    assert not np.array_equal(wrong.state_arrays()["obj"], fresh.state_arrays()["obj"])
    for s in (*parts, full, wrong, fresh):
        s.close()
    for s in (*sets, full_set):
        s.close()
