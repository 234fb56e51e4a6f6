"""Pins the oracle's rearrangement-task epilogue (App. "Additional Task
Details": the reward equation; Sec. 4.1: egomotion observations) to closed
forms built from the pinned forward kinematics."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2306_07552_b300 import inputs as I

from test_oracle_pins import FLOOR, ROBOT, _act, _state, _tip, oracle_for, scene_from_boxes

OPEN = scene_from_boxes([FLOOR], (-5, -0.3, -5), (5, 2.5, 5), h=0.05,
                        supports=[[0.5, -0.5, 1.5, 0.5, 0.0]])


def _task(goal, start, prev_a=np.zeros(7), prev_d=0.0, prev_e=0.0):
    return [*goal, *start, *prev_a, prev_d, prev_e, 0.0]


def _dist(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)))


def test_joint_action_change_and_distance_terms():
    orc = oracle_for(OPEN)
    target = np.array([1.5, 0.04, 1.0, 0.04])
    goal = np.array([2.0, 0.04, -1.0])
    q = ROBOT.q_rest.astype(np.float64)
    tip0 = _tip(orc, (0, 0, 0), q)[9:]
    d0, e0 = _dist(tip0, target[:3]), _dist(target[:3], goal)
    prev_a = np.array([0.1, -0.2, 0, 0, 0.3, 0, 0])
    st = O.Oracle.make_state((0, 0, 0), q, objs=[target],
                             task=_task(goal, target[:3], prev_a, d0, e0))
    a = np.zeros(11, np.float32)
    a[2:9] = [0.5, 0.5, -0.5, 0.0, 0.25, 0.0, -1.0]
    out = orc.step(st, a)
    assert not out.reverted
    af = a[2:9].astype(np.float64)
    C = float(np.sum((af - prev_a) ** 2))
    d1 = _dist(out.ee, target[:3])
    assert out.reward == pytest.approx((d0 - d1) + (e0 - e0) - 0.001 * C, abs=1e-12)
    assert st.prev_d == pytest.approx(d1, abs=1e-15) and list(st.prev_a) == list(af)


def test_pick_bonus_only_for_the_target():
    orc = oracle_for(OPEN)
    q = ROBOT.q_rest.astype(np.float64)
    tip = _tip(orc, (0, 0, 0), q)[9:]
    goal = [3.0, 0.04, 0.0]
    for target_first in (True, False):
        near = [*tip, 0.02]
        far = [3.0, 0.04, 3.0, 0.04]
        objs = [near, far] if target_first else [far, near]
        d0 = _dist(tip, objs[0][:3])
        st = O.Oracle.make_state((0, 0, 0), q, objs=objs,
                                 task=_task(goal, objs[0][:3], prev_d=d0,
                                            prev_e=_dist(objs[0][:3], goal)))
        out = orc.step(st, _act(grasp=1.0))
        assert out.event == 1
        base = out.reward - (d0 - _dist(out.ee, O.Oracle.state_objs(st)[0, :3]))
        assert base == pytest.approx(5.0 if target_first else 0.0, abs=1e-12)


def test_success_needs_stop_release_and_15_cm():
    orc = oracle_for(OPEN)
    q = ROBOT.q_rest.astype(np.float64)
    for gap, hold, stop, expect in [(0.10, False, 1.0, 1), (0.20, False, 1.0, 0),
                                    (0.10, True, 1.0, 0), (0.10, False, 0.0, 0)]:
        target = [1.0, 0.04, 1.0, 0.04]
        goal = [1.0 + gap, 0.04, 1.0]
        kw = dict(objs=[target], task=_task(goal, target[:3], prev_d=1.0, prev_e=gap))
        if hold:
            tip = _tip(orc, (0, 0, 0), q)
            R, t = tip[:9].reshape(3, 3), tip[9:]
            target = [*t, 0.04]
            goal = [t[0] + gap, t[1], t[2]]
            kw = dict(objs=[target], held=0, task=_task(goal, target[:3], prev_d=0.0,
                                                         prev_e=gap))
        st = O.Oracle.make_state((0, 0, 0), q, **kw)
        a = np.zeros(11, np.float32)
        a[10] = stop
        a[9] = 1.0 if hold else 0.0
        out = orc.step(st, a)
        assert out.success == expect, (gap, hold, stop)
        if expect:
            d1 = _dist(out.ee, target[:3])
            assert out.reward == pytest.approx(10.0 + (1.0 - d1), abs=1e-12)


def test_observations_are_in_the_base_frame():
    orc = oracle_for(OPEN)
    yaw = math.pi / 2                         # forward = R_y(yaw) (1, 0, 0) = (0, 0, -1)
    start, goal = [1.0, 0.5, 2.0], [0.0, 0.3, 1.0]
    st = O.Oracle.make_state((1.0, 3.0, yaw), ROBOT.q_rest, objs=[[*start, 0.04]],
                             task=_task(goal, start))
    out = orc.step(st, np.zeros(11, np.float32))
    tip = np.array(out.ee)
    c, s = math.cos(yaw), math.sin(yaw)
    RT = np.array([[c, 0, -s], [0, 1, 0], [s, 0, c]])
    base = np.array([1.0, 0.0, 3.0])
    want = np.concatenate([RT @ (np.array(start) - base), RT @ (np.array(goal) - base),
                           RT @ (np.array(start) - tip), RT @ (np.array(goal) - tip)])
    assert np.allclose(list(out.task_obs), want, atol=1e-12)
    # start 1 m ahead-left of a base facing -z: x_local = forward distance
    assert out.task_obs[0] == pytest.approx(1.0, abs=1e-12)    # -(z - 3) = 1 forward


def test_reset_puts_the_goal_on_a_support_top():
    sc = scene_from_boxes([FLOOR, [0.5, 0.0, -0.5, 1.5, 0.75, 0.5]], (-2, -0.3, -2), (2, 2.5, 2),
                          h=0.05, supports=[[0.5, -0.5, 1.5, 0.5, 0.75]], spawn=[-1.5, -1.5, -0.5, 1.5])
    orc = oracle_for(sc)
    clear = float(np.float32(ROBOT.rest_clearance))
    for env in range(6):
        st = O.Oracle.make_state((0, 0, 0), np.zeros(7))
        orc.reset(st, 9, env, 4, 0.03, 0.06)
        rho = st.obj[0][3]
        assert 0.5 + rho <= st.goal[0] <= 1.5 - rho and -0.5 + rho <= st.goal[2] <= 0.5 - rho
        assert st.goal[1] == pytest.approx(0.75 + rho + clear, abs=1e-12)
        assert list(st.obj_start) == list(st.obj[0])[:3]
        tip = _tip(orc, list(st.base), list(st.q))[9:]
        assert st.prev_d == pytest.approx(_dist(tip, st.obj_start), abs=1e-12)
        assert st.prev_e == pytest.approx(_dist(st.obj_start, st.goal), abs=1e-12)
        assert list(st.prev_a) == [0.0] * 7
