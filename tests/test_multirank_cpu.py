"""The multi-GPU path on CPU: two gloo ranks.

Environments are independent, so one batch splits into contiguous shards,
one per rank, with no collective on the data path: rank g takes environments
[g*N/G, (g+1)*N/G), loads only the scenes they use and draws its resets from
the global environment indices.  Each rank here runs the FP64 oracle on its
own shard (a stand-in for its GPU context: the shard arithmetic, the scene
subset and the counter sum are the host logic under test); the result must
equal one run over the whole batch, environment by environment.  The timed
region's max over ranks and the whole-job value are checked too.
"""
import dataclasses
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2306_07552_b300 import inputs as I
from paper_2306_07552_b300 import shard

N_GLOBAL, N_SCENES, STEPS = 8, 4, 3
W = dataclasses.replace(I.WORKLOADS["room16"], name="room8x4", n_envs=N_GLOBAL,
                        n_scenes=N_SCENES, tri_range=(600, 600))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _run_envs(first, count, scene_ids, local_map):
    """Oracle reset + STEPS steps for global environments [first, first+count);
    returns per-env final state rows and the shard's counters."""
    import oracle as O
    robot = I.fetch_like_robot()
    scenes = I.make_scenes(W, only=scene_ids)
    orcs = [O.Oracle(robot, sc) for sc in scenes]
    acts = I.make_actions(STEPS, N_GLOBAL, W.action_dist, seed=W.action_seed)
    rows, cnt = {}, {"contacts": 0.0, "reward": 0.0, "grasps": 0.0, "env_steps": 0.0}
    for k in range(count):
        e = first + k
        orc = orcs[int(local_map[k])]
        st = O.Oracle.make_state((0, 0, 0), np.zeros(7))
        orc.reset(st, W.reset_seed, e, W.n_objects, *W.obj_radius)
        for t in range(STEPS):
            o = orc.step(st, acts[t, e])
            cnt["contacts"] += float(o.contact_mask != 0)
            cnt["reward"] += float(o.reward)
            cnt["grasps"] += float(o.event == 1)
            cnt["env_steps"] += 1.0
        rows[e] = np.array([*st.base, *st.q, st.held,
                            *O.Oracle.state_objs(st).ravel()], np.float64)
    return rows, cnt


def _shard_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = shard.plan(N_GLOBAL, N_SCENES, world, rank)
    rows, cnt = _run_envs(p.first, p.count, p.scenes, p.env_scene)
    total = shard.sum_counters(dist, cnt)
    ms_local = [100.0, 250.0][rank]          # rank 1 is the slow one
    value, ms = bench.job_value(dist, p.count, 50, ms_local)
    q.put((rank, p, rows, total, value, ms))
    dist.destroy_process_group()


def test_env_range_partitions_the_batch():
    for n in (8, 9, 16384, 16385):
        for world in (1, 2, 3, 8):
            spans = [shard.env_range(n, world, r) for r in range(world)]
            assert spans[0][0] == 0
            for (f0, c0), (f1, _) in zip(spans, spans[1:]):
                assert f0 + c0 == f1                      # contiguous, no gap or overlap
            assert sum(c for _, c in spans) == n
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1
    with pytest.raises(ValueError):
        shard.env_range(4, 2, 2)


def test_plan_loads_only_the_scenes_its_envs_use():
    gmap = I.env_scene_map(16384, 64)
    p0, p1 = (shard.plan(16384, 64, 2, r) for r in range(2))
    assert (p0.first, p0.count, p1.first, p1.count) == (0, 8192, 8192, 8192)
    assert p0.scenes == tuple(range(32)) and p1.scenes == tuple(range(32, 64))
    assert not set(p0.scenes) & set(p1.scenes)
    for p in (p0, p1):
        assert np.array_equal(np.asarray(p.scenes)[p.env_scene], gmap[p.first:p.first + p.count])
    # a caller's own map: rank 0 holds just the scenes its environments name
    m = np.array([3, 3, 1, 0, 2, 2, 2, 2])
    q0 = shard.plan(8, 4, 2, 0, m)
    assert q0.scenes == (0, 1, 3) and list(q0.env_scene) == [2, 2, 1, 0]


def test_two_ranks_equal_one_run_over_the_whole_batch():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort(key=lambda x: x[0])
    # the single-rank run over all environments
    full_rows, full_cnt = _run_envs(0, N_GLOBAL, tuple(range(N_SCENES)),
                                    I.env_scene_map(N_GLOBAL, N_SCENES))
    seen = {}
    for rank, p, rows, total, value, ms in out:
        assert set(rows) == set(range(p.first, p.first + p.count))
        # rank 0's environments use scenes 0 and 1 only; rank 1's 2 and 3
        assert p.scenes == ((0, 1) if rank == 0 else (2, 3))
        for e, r in rows.items():
            assert np.array_equal(r, full_rows[e]), e      # bit-identical evolution
        seen.update(rows)
        assert total == pytest.approx(full_cnt, rel=0, abs=1e-9)   # host-side sum
        assert ms == 250.0                                 # max over ranks
        assert value == pytest.approx(2 * p.count * 50 / 0.250)   # whole job
    assert sorted(seen) == list(range(N_GLOBAL))
    assert full_cnt["env_steps"] == N_GLOBAL * STEPS
