"""The box store (gx_config.static_store 1): distance-grid nodes recomputed in
FP32 from the scene's solid boxes over per-cell candidate lists, instead of
read from the dense FP32 grid.

What the paper and the definitions fix: a node's value is the signed distance
of the union of boxes (the grid's definition, appendix "Additional
Collision-Detection Details"; the oracle evaluates it in FP64 over every box).
So the store is checked node by node against the oracle -- every node of a
room, a random half million of an apartment with 118 boxes -- within the FP32
bound derived for it (about 4e-6 m at coordinates below 16 m, tested at
1e-5 m), far inside the 1e-4 m near band of the decision tests.  A candidate
list that missed the nearest box would show an error of centimetres.  Then
the whole step with the store runs in lockstep against the oracle (resets,
grasps, releases, the sliding and placing heuristics), and the neural form
runs on a scene set that holds no dense grid at all.
"""
import numpy as np
import pytest

import oracle as O
from paper_2306_07552_b300 import inputs as I
from tests.parity import Tally, check_image, check_step

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROBOT = I.fetch_like_robot()
NODE_TOL = 1e-5      # box store (FP32 from the boxes) vs the oracle's FP64 node
MARGIN = 0.02
NEAR_BAND = 1e-4


def _gx():
    from paper_2306_07552_b300 import build, gx
    build.build()
    return gx


def _node_pts(scene, ijk):
    o = scene.grid_origin.astype(np.float64)
    return (o + ijk * np.float64(scene.grid_h)).astype(np.float32)


def _compare_nodes(gx, ss, k, scene, ijk):
    orc = O.Oracle(ROBOT, scene)
    want = np.array([orc.grid_node(*t) for t in ijk])
    pts = torch.from_numpy(_node_pts(scene, ijk)).cuda()
    got1 = ss.static_distance(k, pts, store=1).cpu().numpy().astype(np.float64)
    got0 = ss.static_distance(k, pts, store=0).cpu().numpy().astype(np.float64)
    e1, e0 = np.abs(got1 - want), np.abs(got0 - want)
    print(f"scene {k}: {len(ijk)} nodes, box store max |err| {e1.max():.2e} (median "
          f"{np.median(e1):.1e}), dense grid {e0.max():.2e}")
    assert np.all(np.isfinite(got1))
    assert e1.max() <= NODE_TOL
    assert e0.max() <= NODE_TOL
    return e1


def test_box_store_nodes_match_oracle():
    gx = _gx()
    room = I.room_scene(1000, 2000)                      # 5 cm lattice: every node
    w = I.WORKLOADS["uneven16384_nsdf"]
    apt = I.make_scenes(w, only=[3])[0]                  # 118 boxes, 2 cm lattice
    ss = gx.SceneSet([room, apt])
    nx, ny, nz = [int(v) for v in room.grid_dims]
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    all_room = np.stack([i.ravel(), j.ravel(), k.ravel()], 1)
    _compare_nodes(gx, ss, 0, room, all_room)
    rng = np.random.default_rng(5)
    dims = apt.grid_dims.astype(np.int64)
    ijk = rng.integers(0, dims, (500_000, 3))
    _compare_nodes(gx, ss, 1, apt, ijk)
    # between nodes: the trilinear value against the oracle's FP64 query
    lo = apt.grid_origin.astype(np.float64)
    hi = lo + (dims - 1) * np.float64(apt.grid_h)
    pts = rng.uniform(lo, hi, (200_000, 3)).astype(np.float32)
    orc = O.Oracle(ROBOT, apt)
    want = np.array([orc.grid_query(p)[1] for p in pts.astype(np.float64)])
    got = ss.static_distance(1, torch.from_numpy(pts).cuda(), store=1).cpu().numpy()
    err = np.abs(got - want)
    print(f"points: box store max |err| {np.nanmax(err):.2e}")
    assert np.nanmax(err) <= NODE_TOL
    ss.close()


def test_box_store_bytes_and_set_without_dense_grids():
    gx = _gx()
    w = I.WORKLOADS["uneven16384_nsdf"]
    scenes = I.make_scenes(w, only=[0, 1, 2, 3])
    free0, _ = torch.cuda.mem_get_info()
    full = gx.SceneSet(scenes)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    lean = gx.SceneSet(scenes, dense_grid=False, column_grid=False)
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    dense_total = store_total = 0
    for k, sc in enumerate(scenes):
        b = full.scene_bytes(k)
        bl = lean.scene_bytes(k)
        nodes = int(np.prod(sc.grid_dims))
        assert b["dense_grid"] == 4 * nodes and bl["dense_grid"] == 0 and bl["column_grid"] == 0
        assert b["box_store"] == bl["box_store"] > 0
        print(f"scene {k}: dense grid {b['dense_grid'] / 1e6:.1f} MB, box store "
              f"{b['box_store'] / 1e3:.1f} KB ({b['box_store'] / b['dense_grid']:.3%}), column "
              f"grid {b['column_grid'] / 1e6:.1f} MB, render {b['render'] / 1e6:.2f} MB")
        assert b["box_store"] <= 0.01 * b["dense_grid"]
        dense_total += b["dense_grid"]
        store_total += b["box_store"]
    used_full, used_lean = free0 - free1, free1 - free2
    print(f"device memory taken: with dense grids {used_full / 1e6:.1f} MB, without "
          f"{used_lean / 1e6:.1f} MB")
    # the set without dense grids really leaves them out (allocation granularity aside)
    assert used_lean <= 0.1 * used_full
    # a context that asks for the dense grid of a set without one is refused
    with pytest.raises(gx.GxError):
        gx.Sim(lean, ROBOT, 8, img=(64, 64), n_objects=4)
    with pytest.raises(gx.GxError):
        gx.Sim(lean, ROBOT, 8, img=(64, 64), n_objects=4, static_store=1, sdf_mode=2)
    full.close()
    lean.close()


def test_box_store_step_matches_dense_step_and_oracle():
    """The same batch stepped with either store: identical results (the node
    values differ by a few 1e-6 m, so a decision can only flip within that of
    its threshold), and the box-store step in lockstep with the oracle."""
    gx = _gx()
    w = I.WORKLOADS["apartments4096"]
    scenes = I.make_scenes(w, only=[0, 1])
    ss = gx.SceneSet(scenes)
    orcs = [O.Oracle(ROBOT, sc, I.icosahedron(), I.object_colors(256)) for sc in scenes]
    n, M, T = 256, 40, 40
    es = np.arange(n) % 2
    kw = dict(img=(64, 64), n_objects=M, seed=3, env_scene=es)
    a = gx.Sim(ss, ROBOT, n, **kw)
    b = gx.Sim(ss, ROBOT, n, static_store=1, **kw)
    a.reset()
    b.reset()
    sa, sb = a.state_arrays(), b.state_arrays()
    for key in sa:
        assert np.array_equal(sa[key], sb[key]), key
    acts = I.make_actions(T, n, "gauss0.5", seed=2)
    tally = Tally()
    differ = 0
    for t in range(T):
        before = {k: v.copy() for k, v in b.state_arrays().items()}
        x = torch.from_numpy(acts[t]).cuda()
        oa, ob = a.step(x), b.step(x)
        torch.cuda.synchronize()
        same = all(torch.equal(oa[k], ob[k]) for k in
                   ["pose", "obj_pos", "held", "contact_mask", "contact_flags", "event"])
        differ += 0 if same else 1
        if same:
            assert torch.equal(oa["depth"], ob["depth"]) and torch.equal(oa["rgb"], ob["rgb"])
        after = b.state_arrays()
        for k in range(2):
            check_step(orcs[k], before, after, ob, acts[t], np.flatnonzero(es == k), M, tally)
        if t % 10 == 9:
            for e in (0, 1):
                check_image(orcs[e], after, ob, e, 64, 64, M, tally)
        if not same:  # continue both from the same state
            a.load_state(b.save_state())
    print(tally, f"steps whose outputs differ between the stores: {differ} of {T}")
    assert differ <= 1
    assert tally.near_band <= 0.02 * tally.envs
    assert a.device_error() == 0 and b.device_error() == 0
    a.close()
    b.close()
    ss.close()


def test_box_store_heuristics_match_oracle():
    """Sliding reads the grid's horizontal gradient and the placing jitter
    re-casts objects down: both through the box store, against orc_step_ex."""
    gx = _gx()
    scene = I.room_scene(1000, 2000)
    ss = gx.SceneSet([scene], dense_grid=False, column_grid=False)
    orc = O.Oracle(ROBOT, scene, I.icosahedron(), I.object_colors(256))
    n, M, seed = 64, 10, 21
    sim = gx.Sim(ss, ROBOT, n, img=(64, 64), n_objects=M, seed=seed, heuristics=3,
                 static_store=1)
    sim.reset()
    acts = I.make_actions(40, n, "uniform", seed=4)
    tally = Tally()
    fn = lambda st, a, e: orc.step_ex(st, a, slide=True, place_jitter=True, seed=seed, env=e)  # noqa
    slid = 0
    for t in range(len(acts)):
        before = {k: v.copy() for k, v in sim.state_arrays().items()}
        out = sim.step(torch.from_numpy(acts[t]).cuda())
        torch.cuda.synchronize()
        after = sim.state_arrays()
        check_step(orc, before, after, out, acts[t], range(n), M, tally, step_fn=fn)
        slid += int(((out["contact_flags"].cpu().numpy() & 8) != 0).sum())
    print(tally, f"slides {slid}")
    assert slid >= 20
    assert tally.near_band <= 0.05 * tally.envs
    assert sim.device_error() == 0
    sim.close()
    ss.close()


def test_neural_form_without_dense_grid():
    """The neural SDF with the box store as its exact fallback, on a scene set
    created without dense (or column) grids: networks trained on the store's
    distances, the step's decisions against the grid-only rule (<= 0.1%), the
    rule against the oracle, and the bytes each scene keeps on the device."""
    gx = _gx()
    scenes = [I.room_scene(1000, 2000), I.room_scene(1001, 2000)]
    ss = gx.SceneSet(scenes, dense_grid=False, column_grid=False)
    for k in range(2):
        ss.nsdf_set_weights(k, I.fourier_matrix(7), I.nsdf_init(7))
        losses = ss.nsdf_train(k, n_samples=4_000_000, batch=65536, steps=1500, lr=1e-3, seed=11)
        assert np.isfinite(losses).all()
    for k, sc in enumerate(scenes):
        b = ss.scene_bytes(k)
        dense = 4 * int(np.prod(sc.grid_dims))
        resident = b["box_store"] + b["nsdf_weights"]
        print(f"scene {k}: static bytes of the neural form {resident / 1e3:.1f} KB "
              f"(weights {b['nsdf_weights'] / 1e3:.1f} KB + box store "
              f"{b['box_store'] / 1e3:.1f} KB) vs the dense grid's {dense / 1e6:.2f} MB")
        assert b["dense_grid"] == 0 and b["box_store"] <= 0.1 * dense
    n, M, T = 512, 40, 60
    es = np.arange(n) % 2
    sim = gx.Sim(ss, ROBOT, n, img=(64, 64), n_objects=M, seed=8, sdf_mode=1, sdf_margin=MARGIN,
                 profile=4, static_store=1, env_scene=es)
    sim.reset()
    orcs = [O.Oracle(ROBOT, sc, I.icosahedron(), I.object_colors(256)) for sc in scenes]
    acts = I.make_actions(T, n, "gaussian", seed=9)
    tallies = [Tally(), Tally()]

    def rule(k, pred):
        def f(st, action, env):
            c, r, act = orcs[k].candidate_spheres(st, action)
            d = np.full(31, -1e9)
            idx = np.flatnonzero(act)
            d[idx] = pred[env, idx]
            return orcs[k].step_nsdf(st, action, d, MARGIN, NEAR_BAND)
        return f

    for t in range(T):
        check = t % 6 == 0
        before = {k: v.copy() for k, v in sim.state_arrays().items()} if check else None
        out = sim.step(torch.from_numpy(acts[t]).cuda())
        if check:
            torch.cuda.synchronize()
            after = sim.state_arrays()
            pred = sim.nsdf_step_predictions().astype(np.float64)
            for k in range(2):
                check_step(orcs[k], before, after, out, acts[t], np.flatnonzero(es == k)[:64], M,
                           tallies[k], step_fn=rule(k, pred))
    c = sim.nsdf_counters()
    rate = c["disagree"] / c["tests"]
    print(tallies, f"grid fallbacks {c['grid_fallbacks'] / c['tests']:.2%}, decisions "
          f"differing from the grid-only rule {rate:.4%}")
    assert c["tests"] >= n * T * 30
    assert rate <= 1e-3
    assert c["grid_fallbacks"] / c["tests"] <= 0.2
    assert sum(tl.envs for tl in tallies) >= 0.8 * 10 * 128
    assert sim.device_error() == 0
    sim.close()
    ss.close()
