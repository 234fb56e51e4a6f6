"""Pins the oracle's versions of the paper's two heuristics (appendix
"Description of Heuristics": sliding the base out of a penetration, and
jittering a dropped object to a free resting place) and the grid gradient
they use, against closed forms and brute force."""
import numpy as np
import pytest

import oracle as O
from paper_2306_07552_b300 import inputs as I

from test_oracle_pins import FLOOR, ROBOT, _act, _state, _tip, oracle_for, scene_from_boxes


def test_grid_gradient_of_linear_fields_is_exact():
    sc = scene_from_boxes([FLOOR], (-1, -0.3, -1), (1, 1.5, 1), h=0.05)
    orc = oracle_for(sc)
    inside, g = orc.grid_gradient([0.123, 0.456, -0.321])
    assert inside and np.allclose(g, [0, 1, 0], atol=1e-12)       # d = y
    wall = [0.8, -1.0, -5.0, 3.0, 3.0, 5.0]                        # face at x = 0.8
    sc = scene_from_boxes([wall], (-1, -0.3, -1), (1, 1.5, 1), h=0.05)
    orc = oracle_for(sc)
    inside, g = orc.grid_gradient([0.4, 0.7, 0.2])
    assert inside and np.allclose(g, [-1, 0, 0], atol=1e-12)      # d = 0.8 - x
    assert not orc.grid_gradient([1.5, 0.7, 0.2])[0]


def test_grid_gradient_matches_differences_inside_a_cell():
    table = [0.3, 0.0, -0.5, 1.5, 0.75, 0.5]
    sc = scene_from_boxes([FLOOR, table], (-2, -0.3, -2), (2, 2.5, 2), h=0.05)
    orc = oracle_for(sc)
    rng = np.random.default_rng(2)
    for _ in range(20):
        # a point and a step that stay inside one lattice cell
        cell = rng.integers(5, 60, 3)
        c = sc.grid_origin + (cell + rng.uniform(0.3, 0.7, 3)) * sc.grid_h
        _, g = orc.grid_gradient(c)
        eps = 1e-3 * sc.grid_h
        for a in range(3):
            e = np.zeros(3)
            e[a] = eps
            fd = (orc.grid_query(c + e)[1] - orc.grid_query(c - e)[1]) / (2 * eps)
            assert g[a] == pytest.approx(fd, abs=1e-8)


def test_sliding_backs_off_a_wall_along_its_normal():
    wall = [0.45, -1.0, -5.0, 3.0, 3.0, 5.0]          # face at x = 0.45
    sc = scene_from_boxes([FLOOR, wall], (-2, -0.3, -2), (1.5, 2.5, 2), h=0.05)
    orc = oracle_for(sc)
    step = float(np.float32(ROBOT.base_step))
    cand_x = 0.2 + step
    cand = orc.sphere_centres([cand_x, 0.0, 0.0], ROBOT.q_rest)
    xw = float(np.float32(0.45))                       # box coordinates are FP32 inputs
    pen = [r - (xw - c[0]) for c, r in zip(cand, ROBOT.sphere_radius)]
    assert max(pen) > 0                                 # the move penetrates the wall
    # without sliding the robot does not move
    st = _state(orc, base=(0.2, 0, 0))
    out = orc.step_ex(st, _act(fwd=1.0))
    assert out.reverted and st.base[0] == 0.2
    # with sliding: one jitter of (deepest penetration + 1 mm) along -x
    st = _state(orc, base=(0.2, 0, 0))
    out = orc.step_ex(st, _act(fwd=1.0), slide=True)
    assert not out.reverted and out.flags & 8 and out.flags & 1
    # (the grid stores the distances in FP32: ~1e-8)
    assert st.base[0] == pytest.approx(cand_x - max(pen) - 0.001, abs=1e-7)
    assert abs(st.base[1]) < 1e-12 and st.base[2] == 0.0
    # the slid pose is contact-free
    probe = O.Oracle.make_state(list(st.base), list(st.q))
    assert orc.step(probe, np.zeros(11, np.float32)).contact_mask == 0


def test_sliding_off_reproduces_the_plain_step_and_slid_poses_are_free():
    post = [-0.5, 0.0, -0.1, -0.3, 1.0, 0.1]
    sc = scene_from_boxes([FLOOR, post], (-2, -0.3, -2), (2, 2.5, 2), h=0.02)
    orc = oracle_for(sc)
    acts = I.make_actions(40, 1, "uniform", seed=12)[:, 0]
    a, b, c = _state(orc), _state(orc), _state(orc)
    slid = 0
    for t in range(40):
        oa, ob = orc.step(a, acts[t]), orc.step_ex(b, acts[t])
        assert (oa.contact_mask, oa.flags, list(a.base)) == (ob.contact_mask, ob.flags, list(b.base))
        oc = orc.step_ex(c, acts[t], slide=True)
        if oc.flags & 8:
            slid += 1
            probe = O.Oracle.make_state(list(c.base), list(c.q))
            assert orc.step(probe, np.zeros(11, np.float32)).contact_mask == 0
    assert slid > 0


def _drop_setup(scene_boxes, lo, hi, others):
    sc = scene_from_boxes(scene_boxes, lo, hi, h=0.02)
    orc = oracle_for(sc)
    tip = _tip(orc, (0, 0, 0), ROBOT.q_rest.astype(np.float64))[9:]
    start = tip + [0.0, 0.0, 0.06]
    objs = np.array([[*start, 0.04], *others(start)])
    st = _state(orc, objs=objs)
    assert orc.step(st, _act(grasp=1.0)).event == 1
    return orc, st, start


def test_placement_jitter_lands_clear_of_the_object_below():
    clear = float(np.float32(ROBOT.rest_clearance))
    rho = 0.04
    orc, st, start = _drop_setup([FLOOR], (-2, -0.3, -2), (2, 2.5, 2),
                                 lambda s: [[s[0], 0.03 + clear, s[2], 0.03]])
    out = orc.step_ex(st, _act(grasp=0.0), place_jitter=True, seed=3, env=5)
    assert out.event == 5 and st.held == -1
    p = O.Oracle.state_objs(st)
    assert p[0, 1] == pytest.approx(rho + clear, abs=1e-12)         # on the floor
    assert np.linalg.norm(p[0, :3] - p[1, :3]) >= rho + 0.03         # clear of the other
    r = np.hypot(p[0, 0] - start[0], p[0, 2] - start[2])
    assert r <= 6 * 2 * rho + 1e-12
    # the same draw again is the same landing; another environment draws anew
    orc2, st2, _ = _drop_setup([FLOOR], (-2, -0.3, -2), (2, 2.5, 2),
                               lambda s: [[s[0], 0.03 + clear, s[2], 0.03]])
    orc2.step_ex(st2, _act(grasp=0.0), place_jitter=True, seed=3, env=5)
    assert np.array_equal(O.Oracle.state_objs(st2), p)
    orc3, st3, _ = _drop_setup([FLOOR], (-2, -0.3, -2), (2, 2.5, 2),
                               lambda s: [[s[0], 0.03 + clear, s[2], 0.03]])
    orc3.step_ex(st3, _act(grasp=0.0), place_jitter=True, seed=3, env=6)
    assert not np.array_equal(O.Oracle.state_objs(st3), p)
    # without the heuristic the drop is restored
    orc4, st4, _ = _drop_setup([FLOOR], (-2, -0.3, -2), (2, 2.5, 2),
                               lambda s: [[s[0], 0.03 + clear, s[2], 0.03]])
    assert orc4.step_ex(st4, _act(grasp=0.0)).event == 4


def test_placement_jitter_restores_when_nothing_is_below():
    # no floor anywhere: every cast fails, six jitters, then the object goes back
    high = [-5.0, 3.0, -5.0, 5.0, 3.5, 5.0]
    orc, st, start = _drop_setup([high], (-2, -0.3, -2), (2, 2.5, 2), lambda s: [])
    out = orc.step_ex(st, _act(grasp=0.0), place_jitter=True, seed=3, env=1)
    assert out.event == 4
    assert np.allclose(O.Oracle.state_objs(st)[0, :3], start, atol=1e-12)
