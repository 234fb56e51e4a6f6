"""Property tests of the CUDA step on small random batches (hypothesis, GPU).

The same invariants as the oracle's property tests, on the GPU's outputs
through the C ABI, over random batch sizes, object counts, image sizes, reset
seeds and actions (beyond [-1, 1] too): joints within their limits and the
yaw within (-pi, pi] after every step; a step with a contact (contact mask
non-zero and no sliding) leaves base and joints as they were; depth is 0 or
at least the near plane; the device error word stays clear."""
import functools
import math

import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import HealthCheck, given, settings, strategies as st  # noqa: E402

from paper_2306_07552_b300 import inputs as I  # noqa: E402

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROBOT = I.fetch_like_robot()


@functools.lru_cache(maxsize=1)
def _set():
    from paper_2306_07552_b300 import build, gx
    build.build()
    scenes = [I.room_scene(1000 + k, 1500, n_furniture=8) for k in range(3)]
    return gx, gx.SceneSet(scenes), len(scenes)


@settings(max_examples=15, deadline=None, suppress_health_check=[HealthCheck.too_slow])
@given(n=st.integers(1, 64), M=st.integers(0, 12), side=st.sampled_from([32, 64, 96, 128]),
       fp16=st.booleans(), seed=st.integers(0, 2**31 - 1), steps=st.integers(1, 6),
       act_seed=st.integers(0, 2**31 - 1), store=st.integers(0, 1))
def test_gpu_step_invariants(n, M, side, fp16, seed, steps, act_seed, store):
    gx, ss, n_scenes = _set()
    es = np.random.default_rng(seed).integers(0, n_scenes, n).astype(np.int32)
    sim = gx.Sim(ss, ROBOT, n, img=(side, side), depth_fp16=fp16, n_objects=M, seed=seed,
                 env_scene=es, static_store=store)
    sim.reset()
    acts = np.random.default_rng(act_seed).uniform(-1.5, 1.5, (steps, n, 11)).astype(np.float32)
    qmin = np.asarray(ROBOT.q_min, np.float32)[:, None]
    qmax = np.asarray(ROBOT.q_max, np.float32)[:, None]
    for t in range(steps):
        before = sim.state_arrays()
        out = sim.step(torch.from_numpy(acts[t]).cuda())
        torch.cuda.synchronize()
        after = sim.state_arrays()
        assert np.all(after["q"] >= qmin) and np.all(after["q"] <= qmax)
        assert np.all(after["yaw"] > -math.pi) and np.all(after["yaw"] <= math.pi)
        hit = out["contact_mask"].cpu().numpy() != 0
        for k in ("base_x", "base_z", "yaw"):
            assert np.array_equal(after[k][hit], before[k][hit])
        assert np.array_equal(after["q"][:, hit], before["q"][:, hit])
        d = out["depth"].float().cpu().numpy()
        assert np.all((d == 0) | (d >= np.float32(ROBOT.cam_near) * (1 - 1e-3)))
    assert sim.device_error() == 0
    sim.close()
