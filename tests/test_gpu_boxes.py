"""The oriented-box object model (appendix "Additional Collision-Detection
Details") against the FP64 oracle, lockstep: resets that place boxes on
support tops, steps whose robot spheres meet boxes, grasps that carry a box
as eight spheres turning with the tool, releases that stand it upright on the
highest landing of its bottom spheres or restore it, and the images of boxes
resting and carried.  Same tolerances as the sphere model.  Run on the dense
grid and on the box store (a scene set without its dense grid)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2306_07552_b300 import inputs as I
from tests.parity import Tally, check_image, check_step, oracle_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROBOT = I.fetch_like_robot()


@pytest.fixture(scope="module")
def room():
    from paper_2306_07552_b300 import build, gx
    build.build()
    scene = I.room_scene(1000, 2000)
    ss = gx.SceneSet([scene])
    # the same scene without its dense grid: the box store serves every static test
    lean = gx.SceneSet([scene], dense_grid=False, column_grid=False)
    orc = O.Oracle(ROBOT, scene, I.unit_cube(), I.object_colors(256))
    yield gx, scene, {0: ss, 1: lean}, orc
    ss.close()
    lean.close()


def _check_resets(sim, orc, before, M, seed, rho):
    s = sim.state_arrays()
    checked = flips = 0
    for e in range(sim.n):
        st = oracle_state(before, e, M, boxes=True)
        r = orc.reset(st, seed, e, M, *rho)
        placed = (np.allclose(s["obj"][e, :M], O.Oracle.state_objs(st), atol=1e-5)
                  and np.allclose(s["box"][e, :M, :3], O.Oracle.state_boxes(st)[:, :3], atol=1e-6)
                  and abs(s["base_x"][e] - st.base[0]) < 1e-5
                  and abs(s["base_z"][e] - st.base[1]) < 1e-5)
        if r.near_band and not placed:
            flips += 1
            continue
        assert placed, e
        yaw_g, yaw_o = s["box"][e, :M, 3], O.Oracle.state_boxes(st)[:, 3]
        d = np.abs((yaw_g - yaw_o + math.pi) % (2 * math.pi) - math.pi)
        assert np.all(d < 1e-5), e
        assert s["held"][e] == -1 and s["episode"][e] == st.episode
        want = [*st.goal, *st.obj_start, *st.prev_a, st.prev_d, st.prev_e]
        assert np.allclose(s["task"][e, :15], want, atol=1e-5), e
        checked += 1
    return checked, flips


def _lockstep(sim, orc, acts, M, W, tally, image_envs):
    for t in range(len(acts)):
        before = {k: v.copy() for k, v in sim.state_arrays().items()}
        out = sim.step(torch.from_numpy(acts[t]).cuda())
        torch.cuda.synchronize()
        after = sim.state_arrays()
        check_step(orc, before, after, out, acts[t], range(sim.n), M, tally, boxes=True)
        for e in image_envs(t):
            check_image(orc, after, out, e, W, W, M, tally, boxes=True)


# warps 0: the default rasteriser shape for box objects (7 warps per CTA); 8: the other one
@pytest.mark.parametrize("store,warps", [(0, 0), (1, 0), (0, 8)])
def test_box_resets_and_random_steps(room, store, warps):
    gx, scene, sets, orc = room
    n, M, W = 48, 12, 64
    rho = (0.03, 0.06)
    sim = gx.Sim(sets[store], ROBOT, n, img=(W, W), n_objects=M, obj_radius=rho, seed=5,
                 object_boxes=True, static_store=store, raster_warps=warps)
    before = {k: v.copy() for k, v in sim.state_arrays().items()}
    sim.reset()
    torch.cuda.synchronize()
    checked, flips = _check_resets(sim, orc, before, M, 5, rho)
    print(f"resets checked {checked}, near-band flips {flips}")
    assert checked >= n - 2
    acts = I.make_actions(12, n, "uniform", seed=8)
    tally = Tally()
    _lockstep(sim, orc, acts, M, W, tally, lambda t: [0, 17, 40] if t % 4 == 0 else [])
    print(tally)
    print(tally.report())
    assert tally.envs - tally.near_band_flips >= 0.95 * tally.envs
    assert tally.contacts > 0 and tally.pixels > 0
    # a masked reset in the middle
    mask = np.zeros(n, np.uint8)
    mask[::3] = 1
    before = {k: v.copy() for k, v in sim.state_arrays().items()}
    sim.reset(torch.from_numpy(mask).cuda())
    torch.cuda.synchronize()
    s = sim.state_arrays()
    for e in np.flatnonzero(mask == 0):
        assert np.array_equal(s["obj"][e], before["obj"][e])
    sim.close()


def _box_at_tip(sim, orc, M):
    """Box 0 of every env just below the suction tip, upright, a random yaw;
    in odd envs a wide, low box 1 on the floor under it, in the way of a
    landing (the static grid does not know about boxes)."""
    buf = sim.save_state().copy()
    s = sim.state_arrays(buf)
    rng = np.random.default_rng(4)
    clear = float(np.float32(ROBOT.rest_clearance))
    for e in range(sim.n):
        _, ee, _ = orc.fk((s["base_x"][e], s["base_z"][e], s["yaw"][e]), s["q"][:, e])
        t = ee[9:]
        h = rng.uniform(0.03, 0.05, 3)
        s["box"][e, 0] = [*h, rng.uniform(-math.pi, math.pi)]
        s["obj"][e, 0] = [t[0], t[1] - h[1] - 0.01, t[2], np.linalg.norm(h)]
        if e % 2:
            h1 = np.array([0.35, 0.05, 0.35])
            s["box"][e, 1] = [*h1, 0.0]
            s["obj"][e, 1] = [t[0], 0.0 + h1[1] + clear, t[2], np.linalg.norm(h1)]
    sim.load_state(buf)


@pytest.mark.parametrize("store", [0, 1])
def test_box_grasp_carry_release(room, store):
    gx, scene, sets, orc = room
    n, M, W = 32, 8, 64
    sim = gx.Sim(sets[store], ROBOT, n, img=(W, W), n_objects=M, obj_radius=(0.03, 0.06),
                 seed=9, object_boxes=True, static_store=store)
    sim.reset()
    torch.cuda.synchronize()
    _box_at_tip(sim, orc, M)
    rng = np.random.default_rng(2)
    T = 9
    acts = np.zeros((T, n, 11), np.float32)
    acts[:, :, 2:9] = rng.uniform(-1, 1, (T, n, 7)) * 0.5
    acts[:, :, 0] = rng.uniform(-1, 1, (T, n)) * 0.3
    acts[:6, 0::2, 9] = 1.0  # even envs: grasp, carry five steps, release
    acts[:1, 1::2, 9] = 1.0  # odd envs: grasp, release at once over box 1
    tally = Tally()
    _lockstep(sim, orc, acts, M, W, tally, lambda t: [0, 5, 11] if t in (0, 1, 3, 6) else [])
    print(tally)
    print(tally.report())
    assert tally.events.get(1, 0) >= 24
    assert tally.events.get(3, 0) >= 10      # landed upright
    assert tally.events.get(4, 0) >= 5       # restored: the landing overlapped box 1
    assert tally.envs - tally.near_band_flips >= 0.95 * tally.envs
    sim.close()


def test_box_configurations_refused(room):
    gx, scene, sets, orc = room
    ss = sets[0]
    for kw in (dict(heuristics=1), dict(broadphase=True), dict(render_robot=True),
               dict(sdf_mode=2), dict(raster_warps=6), dict(raster_warps=12)):
        with pytest.raises(gx.GxError):
            gx.Sim(ss, ROBOT, 4, img=(32, 32), n_objects=4, object_boxes=True, **kw)
