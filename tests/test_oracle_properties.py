"""Property tests of the oracle on small random rooms (hypothesis, CPU).

Invariants the method fixes whatever the inputs (Sec. 3.2: any contact
rejects all robot motion; a grasped object moves rigidly with the tool; the
joint limits hold; Sec. 3.1: depth is a forward distance beyond the near
plane or 0): over random scenes, object counts, reset seeds and action
sequences -- actions drawn beyond [-1, 1] too, which the step clips -- after
every step
  - the joints lie within their limits and the yaw within (-pi, pi];
  - a step that was not reverted leaves every robot sphere clear of the
    static scene (grid distance >= radius) and of every resting object it was
    tested against, and the held object clear of the scene;
  - a reverted step leaves the base and the joints as they were;
  - an object held before and after the step sits where the tool frame carries
    its fixed offset;
and every rendered pixel's depth is 0 or at least the near plane.
"""
import functools
import math

import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle as O  # noqa: E402
from paper_2306_07552_b300 import inputs as I  # noqa: E402

ROBOT = I.fetch_like_robot()
SLACK = 1e-9


@functools.lru_cache(maxsize=8)
def _room(seed):
    scene = I.room_scene(seed, 600, n_furniture=6)
    return scene, O.Oracle(ROBOT, scene, I.icosahedron(), I.object_colors(256))


def _state_tuple(s):
    return (np.array(s.base[:]), np.array(s.q[:]), int(s.held),
            O.Oracle.state_objs(s).copy())


def _check_step(orc, before, s, out, action):
    base0, q0, held0, objs0 = before
    base1, q1 = np.array(s.base[:]), np.array(s.q[:])
    assert np.all(q1 >= np.array(ROBOT.q_min) - 1e-12)
    assert np.all(q1 <= np.array(ROBOT.q_max) + 1e-12)
    assert -math.pi < base1[2] <= math.pi
    if out.reverted:
        assert np.array_equal(base1, base0) and np.array_equal(q1, q0)
        return
    # accepted: every robot sphere clear of the scene and of the resting objects
    cs = orc.sphere_centres(base1, q1)
    radii = np.asarray(ROBOT.sphere_radius, np.float64)
    for c, r in zip(cs, radii):
        inside, d, _ = orc.grid_query(c)
        assert inside and d >= r - SLACK, (c, r, d)
        for j, o in enumerate(objs0):
            if j == held0:
                continue
            assert np.linalg.norm(c - o[:3]) >= r + o[3] - SLACK, (j, c, o)
    if held0 >= 0 and int(s.held) == held0:
        # the carried object: rigid with the tool tip, clear of the scene
        _, ee, _ = orc.fk(base1, q1)
        R, t = ee[:9].reshape(3, 3), ee[9:]
        p = t + R @ np.array(s.c_off[:])
        obj = O.Oracle.state_objs(s)[held0]
        assert np.allclose(obj[:3], p, atol=1e-9), (obj, p)
        inside, d, _ = orc.grid_query(obj[:3])
        assert inside and d >= obj[3] - SLACK


@settings(max_examples=30, deadline=None)
@given(scene_seed=st.integers(1000, 1005), n_obj=st.integers(0, 8),
       reset_seed=st.integers(0, 2**31 - 1),
       actions=st.lists(st.lists(st.floats(-1.5, 1.5, allow_nan=False), min_size=11,
                                 max_size=11), min_size=1, max_size=8))
def test_step_invariants(scene_seed, n_obj, reset_seed, actions):
    scene, orc = _room(scene_seed)
    s = O.Oracle.make_state((0, 0, 0), np.zeros(7))
    orc.reset(s, reset_seed, 0, n_obj, 0.03, 0.06)
    for a in actions:
        before = _state_tuple(s)
        out = orc.step(s, np.asarray(a, np.float32))
        _check_step(orc, before, s, out, a)


@settings(max_examples=30, deadline=None)
@given(scene_seed=st.integers(1000, 1005), reset_seed=st.integers(0, 2**31 - 1),
       grasp_steps=st.integers(1, 4), moves=st.lists(
           st.lists(st.floats(-1.0, 1.0, allow_nan=False), min_size=9, max_size=9),
           min_size=1, max_size=5))
def test_grasped_object_moves_rigidly(scene_seed, reset_seed, grasp_steps, moves):
    """An object put at the suction tip is grasped and then carried rigidly by
    every accepted move until the grasp action drops."""
    scene, orc = _room(scene_seed)
    s = O.Oracle.make_state((0, 0, 0), np.zeros(7))
    orc.reset(s, reset_seed, 0, 4, 0.03, 0.06)
    _, ee, _ = orc.fk(np.array(s.base[:]), np.array(s.q[:]))
    p = ee[9:] + ee[:9].reshape(3, 3) @ np.array([0.05, 0.0, 0.0])
    s.obj[0][:] = [p[0], p[1], p[2], 0.035]
    grasp = np.zeros(11, np.float32)
    grasp[9] = 1.0
    out = orc.step(s, grasp)
    if int(s.held) != 0:           # the tip sphere met another object first, or contact
        return
    for m in moves:
        a = np.zeros(11, np.float32)
        a[:9] = m
        a[9] = 1.0                 # keep holding
        before = _state_tuple(s)
        out = orc.step(s, a)
        _check_step(orc, before, s, out, a)
        assert int(s.held) == 0


@settings(max_examples=12, deadline=None)
@given(scene_seed=st.integers(1000, 1005), reset_seed=st.integers(0, 2**31 - 1),
       n_obj=st.integers(0, 8))
def test_depth_is_zero_or_beyond_near(scene_seed, reset_seed, n_obj):
    scene, orc = _room(scene_seed)
    s = O.Oracle.make_state((0, 0, 0), np.zeros(7))
    orc.reset(s, reset_seed, 0, n_obj, 0.03, 0.06)
    depth = orc.render(s, 32, 32)[0]
    assert np.all((depth == 0) | (depth >= ROBOT.cam_near - 1e-12))
    assert np.any(depth > 0)
