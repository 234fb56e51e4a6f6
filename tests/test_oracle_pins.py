"""Pins the FP64 oracle to facts that do not come from the oracle itself:
published known-answer vectors, closed-form distances and depths,
hand-computed kinematic poses, brute-force enumeration on tiny inputs and
invariants of the method.  Each check is chosen so that a plausible slip in
the oracle (a dropped term, a wrong sign or index, a transposed operand)
fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2306_07552_b300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ROBOT = I.fetch_like_robot()


def scene_from_boxes(boxes, lo, hi, h=0.05, supports=None, rgb=None, spawn=None, tris=None):
    """Tiny hand-built scene: the listed solid boxes, a lattice over [lo, hi]."""
    boxes = np.array(boxes, np.float32).reshape(-1, 6)
    origin = np.array(lo, np.float32)
    dims = (np.ceil((np.array(hi) - np.array(lo)) / h).astype(np.int32) + 1)
    if tris is None:
        verts = np.zeros((3, 3), np.float32)
        tr = np.zeros((0, 3), np.int32)
        trgb = np.zeros(0, np.uint32)
    else:
        verts, tr, trgb = tris
    return I.Scene(boxes=boxes, box_rgb=np.zeros(len(boxes), np.uint32), verts=verts, tris=tr,
                   tri_rgb=trgb,
                   supports=np.array(supports if supports is not None else [[0, 0, 1, 1, 0]],
                                     np.float32),
                   grid_origin=origin, grid_h=float(np.float32(h)), grid_dims=dims,
                   spawn=np.array(spawn if spawn is not None else [-1, -1, 1, 1], np.float32))


FLOOR = [-20, -1, -20, 20, 0, 20]   # a floor slab whose top is y = 0


def oracle_for(scene, robot=ROBOT):
    return O.Oracle(robot, scene, I.icosahedron(), I.object_colors(256))


# ---------------------------------------------------------------- Philox

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert list(out) == v[6:10]


# ------------------------------------------------------- distance grid

def test_box_sdf_closed_forms():
    box = [0, 0, 0, 2, 1, 4]
    # above the top face: the height above it
    assert O.box_sdf([1.0, 3.5, 2.0], box) == pytest.approx(2.5, abs=1e-15)
    # beside a face: the gap to it
    assert O.box_sdf([-0.75, 0.5, 1.0], box) == pytest.approx(0.75, abs=1e-15)
    # outside a corner: Euclidean distance to that corner
    p = [2.3, 1.4, 4.5]
    assert O.box_sdf(p, box) == pytest.approx(math.dist(p, [2, 1, 4]), abs=1e-15)
    # outside an edge (x and y out, z within): distance to the edge line
    assert O.box_sdf([-0.3, 1.4, 2.0], box) == pytest.approx(0.5, abs=1e-15)
    # inside: minus the distance to the nearest face
    assert O.box_sdf([1.0, 0.8, 2.0], box) == pytest.approx(-0.2, abs=1e-15)
    assert O.box_sdf([0.1, 0.5, 2.0], box) == pytest.approx(-0.1, abs=1e-15)


def test_grid_nodes_are_min_over_boxes():
    boxes = [FLOOR, [0.5, 0, 0.5, 1.0, 0.8, 1.2], [-1.0, 0, -0.2, -0.6, 1.5, 0.3]]
    sc = scene_from_boxes(boxes, (-1.5, -0.2, -1.5), (1.5, 2.0, 1.5), h=0.05)
    orc = oracle_for(sc)
    rng = np.random.default_rng(3)
    for _ in range(50):
        i, j, k = (int(rng.integers(0, d)) for d in sc.grid_dims)
        p = sc.grid_origin.astype(np.float64) + np.array([i, j, k]) * float(sc.grid_h)
        # expected: distance to the union written independently of box_sdf
        expect = min(_sdf_box_numpy(p, b) for b in boxes)
        assert orc.grid_node(i, j, k) == pytest.approx(expect, abs=1e-12)


def _sdf_box_numpy(p, b):
    lo, hi = np.array(b[:3], np.float64), np.array(b[3:], np.float64)
    lo, hi = lo.astype(np.float32).astype(np.float64), hi.astype(np.float32).astype(np.float64)
    closest = np.clip(p, lo, hi)
    if np.any(closest != p):
        return float(np.linalg.norm(p - closest))
    return -float(np.min(np.concatenate([p - lo, hi - p])))


def test_trilinear_reproduces_linear_field():
    # floor only: d = y exactly over the slab interior, so interpolation of
    # node values must give y at any point inside the lattice
    sc = scene_from_boxes([FLOOR], (-1, -0.3, -1), (1, 2.0, 1), h=0.05)
    orc = oracle_for(sc)
    rng = np.random.default_rng(1)
    for _ in range(200):
        c = rng.uniform([-0.99, 0.01, -0.99], [0.99, 1.99, 0.99])
        inside, d, edge = orc.grid_query(c)
        assert inside
        assert d == pytest.approx(c[1], abs=1e-12)
    inside, d, edge = orc.grid_query([0.0, 2.5, 0.0])
    assert not inside and edge < 0


# ------------------------------------------------------ kinematics

def _rot(axis, a):
    c, s = math.cos(a), math.sin(a)
    if axis == 0:
        return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
    if axis == 1:
        return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])


def test_fk_zero_pose_is_chain_sum():
    orc = oracle_for(scene_from_boxes([FLOOR], (-2, -0.2, -2), (2, 2, 2)))
    links, ee, cam = orc.fk([0.0, 0.0, 0.0], np.zeros(7))
    off = ROBOT.link_offset.astype(np.float64)
    acc = np.zeros(3)
    for k in range(7):
        acc = acc + off[k]
        assert np.allclose(links[k + 1][9:], acc, atol=1e-12)
        assert np.allclose(links[k + 1][:9].reshape(3, 3), np.eye(3), atol=1e-12)
    assert np.allclose(ee[9:], acc + off[7], atol=1e-12)
    # base yaw only rotates the chain about +y and moves it with the base
    th = 0.7
    links2, ee2, _ = orc.fk([1.5, -2.0, th], np.zeros(7))
    expect = np.array([1.5, 0, -2.0]) + _rot(1, th) @ (acc + off[7])
    assert np.allclose(ee2[9:], expect, atol=1e-12)


@pytest.mark.parametrize("joint", range(7))
@pytest.mark.parametrize("ang", [math.pi / 2, -math.pi / 2])
def test_fk_single_joint_quarter_turns(joint, ang):
    orc = oracle_for(scene_from_boxes([FLOOR], (-2, -0.2, -2), (2, 2, 2)))
    q = np.zeros(7)
    q[joint] = ang
    _, ee, _ = orc.fk([0.0, 0.0, 0.0], q)
    off = ROBOT.link_offset.astype(np.float64)
    before = off[:joint + 1].sum(0)
    after = off[joint + 1:].sum(0)   # links after the joint plus the tool tip
    # quarter-turn matrices written out by hand
    c, s = 0.0, float(np.sign(ang))
    R = {0: [[1, 0, 0], [0, c, -s], [0, s, c]], 1: [[c, 0, s], [0, 1, 0], [-s, 0, c]],
         2: [[c, -s, 0], [s, c, 0], [0, 0, 1]]}[int(ROBOT.link_axis[joint])]
    assert np.allclose(ee[9:], before + np.array(R) @ after, atol=1e-12)


def test_fk_frames_orthonormal():
    orc = oracle_for(scene_from_boxes([FLOOR], (-2, -0.2, -2), (2, 2, 2)))
    rng = np.random.default_rng(0)
    for _ in range(20):
        q = rng.uniform(-2.5, 2.5, 7)
        links, ee, cam = orc.fk([rng.uniform(-3, 3), rng.uniform(-3, 3), rng.uniform(-3, 3)], q)
        for F in list(links) + [ee, cam]:
            R = F[:9].reshape(3, 3)
            assert np.allclose(R.T @ R, np.eye(3), atol=1e-12)
            assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-12)


def test_camera_mount_axes():
    orc = oracle_for(scene_from_boxes([FLOOR], (-2, -0.2, -2), (2, 2, 2)))
    _, _, cam = orc.fk([0.0, 0.0, 0.0], np.zeros(7))
    R = cam[:9].reshape(3, 3)
    p = ROBOT.cam_pitch
    assert np.allclose(R[:, 2], [math.cos(p), math.sin(p), 0], atol=1e-7)   # forward
    assert np.allclose(R[:, 0], [0, 0, -1], atol=1e-12)                     # right
    assert np.allclose(cam[9:], ROBOT.cam_pos, atol=1e-12)


# ------------------------------------------------------- action decoding

def _state(orc, base=(0, 0, 0), q=None, objs=None, held=-1, c_off=(0, 0, 0), p_pre=(0, 0, 0)):
    return O.Oracle.make_state(base, ROBOT.q_rest if q is None else q, held, c_off, p_pre, objs)


def _act(**kw):
    a = np.zeros(11, np.float32)
    for k, v in kw.items():
        a[{"fwd": 0, "rot": 1, "grasp": 9, "stop": 10}[k] if not k.startswith("q") else
          2 + int(k[1:])] = v
    return a


OPEN = scene_from_boxes([FLOOR], (-5, -0.3, -5), (5, 2.5, 5), h=0.05)


def test_base_translation_and_turn_directions():
    # the robot table is an FP32 input: 10 cm and 5 degrees as float32 values
    step = float(np.float32(ROBOT.base_step))
    turn = float(np.float32(ROBOT.base_turn))
    assert step == pytest.approx(0.10, abs=1e-8) and turn == pytest.approx(math.radians(5), abs=1e-8)
    orc = oracle_for(OPEN)
    st = _state(orc, base=(0, 0, 0))
    orc.step(st, _act(fwd=1.0))
    assert list(st.base) == pytest.approx([step, 0.0, 0.0], abs=1e-15)
    st = _state(orc, base=(0, 0, math.pi / 2))
    orc.step(st, _act(fwd=1.0))          # heading +90 deg faces -z
    assert list(st.base)[:2] == pytest.approx([0.0, -step], abs=1e-15)
    st = _state(orc, base=(0, 0, 0))
    orc.step(st, _act(rot=1.0))          # clockwise seen from above
    assert st.base[2] == pytest.approx(-turn, abs=1e-15)
    # translation uses the pre-step heading
    st = _state(orc, base=(0, 0, 0))
    orc.step(st, _act(fwd=0.5, rot=-1.0))
    assert list(st.base) == pytest.approx([0.5 * step, 0.0, turn], abs=1e-15)
    # yaw stays in (-pi, pi]
    st = _state(orc, base=(0, 0, math.pi - 0.01))
    orc.step(st, _act(rot=-1.0))
    assert -math.pi < st.base[2] <= math.pi
    assert st.base[2] == pytest.approx(math.pi - 0.01 + turn - 2 * math.pi, abs=1e-12)


def test_joint_limit_clamp_and_action_clip():
    orc = oracle_for(OPEN)
    q = np.array(ROBOT.q_rest, np.float64)
    q[0] = 2.45
    st = _state(orc, q=q)
    orc.step(st, _act(q0=1.0))
    assert st.q[0] == 2.5                      # clamped exactly to the limit
    st = _state(orc, q=q)
    orc.step(st, _act(q0=0.3))
    assert st.q[0] == pytest.approx(2.45 + float(np.float32(0.3)) * float(np.float32(0.1)), abs=1e-15)
    st = _state(orc, q=q)
    orc.step(st, _act(q0=7.0))                 # actions are clipped to [-1, 1]
    assert st.q[0] == 2.5
    q[2] = -2.45
    st = _state(orc, q=q)
    orc.step(st, _act(q2=-1.0))
    assert st.q[2] == -2.5


def test_non_finite_actions_count_as_zero():
    orc = oracle_for(OPEN)
    st = _state(orc)
    a = _act(fwd=np.nan, rot=np.inf)
    orc.step(st, a)
    assert list(st.base) == [0.0, 0.0, 0.0]


# ------------------------------------------------------- collision

def _brute_mask(centres, radii, objs, static_d=None):
    mask = 0
    for i, (c, r) in enumerate(zip(centres, radii)):
        hit = False
        for o in objs:
            if np.sqrt(((c - o[:3]) ** 2).sum()) < r + o[3]:
                hit = True
        if static_d is not None and static_d[i] < r:
            hit = True
        if hit:
            mask |= 1 << i
    return mask


def test_object_contacts_match_brute_force():
    orc = oracle_for(OPEN)
    rng = np.random.default_rng(5)
    radii = ROBOT.sphere_radius.astype(np.float64)
    n_hit = 0
    for trial in range(40):
        base = (0.0, 0.0, float(rng.uniform(-3, 3)))
        q = ROBOT.q_rest.astype(np.float64)
        centres = orc.sphere_centres(base, q)
        objs = []
        for j in range(6):
            i = int(rng.integers(0, 30))
            rho = float(rng.uniform(0.03, 0.06))
            dirn = rng.normal(size=3)
            dirn /= np.linalg.norm(dirn)
            gap = float(rng.choice([-0.01, 0.01]))
            objs.append(np.r_[centres[i] + dirn * (radii[i] + rho + gap), rho])
        objs = np.array(objs)
        st = _state(orc, base=base, q=q, objs=objs)
        out = orc.step(st, np.zeros(11, np.float32))
        expect = _brute_mask(centres, radii, objs)
        assert out.contact_mask == expect
        assert bool(out.flags & 2) == (expect != 0)
        assert bool(out.reverted) == (expect != 0)
        n_hit += expect != 0
    assert n_hit > 5


def test_static_contact_reverts_all_motion():
    # a post just behind the base: backing up drives a base sphere into it
    post = [-0.5, 0.0, -0.1, -0.3, 1.0, 0.1]
    sc = scene_from_boxes([FLOOR, post], (-2, -0.3, -2), (2, 2.5, 2), h=0.02)
    orc = oracle_for(sc)
    st = _state(orc)
    assert orc.step(st, np.zeros(11, np.float32)).contact_mask == 0
    before = (list(st.base), list(st.q))
    out = orc.step(st, _act(fwd=-1.0, q1=0.5))
    assert out.reverted and out.flags & 1
    assert (list(st.base), list(st.q)) == before     # base AND arm held back
    # which spheres: brute force against the exact box distance
    cq = np.array(before[1])
    cq[1] += float(np.float32(0.5)) * float(np.float32(ROBOT.dq_max))
    cand = orc.sphere_centres([-float(np.float32(ROBOT.base_step)), 0.0, 0.0], cq)
    d = [min(_sdf_box_numpy(c, FLOOR), _sdf_box_numpy(c, post)) for c in cand]
    assert out.contact_mask == _brute_mask(cand, ROBOT.sphere_radius, [], d)


def test_leaving_the_grid_is_contact():
    sc = scene_from_boxes([FLOOR], (-1, -0.3, -1), (1.0, 2.5, 1.0), h=0.05)
    orc = oracle_for(sc)
    st = _state(orc, base=(0.45, 0, 0))
    out = orc.step(st, _act(fwd=1.0))   # front base spheres cross x = 1
    assert out.reverted and out.flags & 1


# ------------------------------------------------------- grasp and release

def _tip(orc, base, q):
    _, ee, _ = orc.fk(base, q)
    return ee


def test_grasp_attach_rigid_offset_and_nearest_rule():
    orc = oracle_for(OPEN)
    q = ROBOT.q_rest.astype(np.float64)
    ee = _tip(orc, (0, 0, 0), q)
    tip = ee[9:]
    # two objects overlap the suction sphere; the one with the smaller
    # surface distance wins even though its centre is farther away
    objs = np.array([[*(tip + [0.0, 0.0, 0.05]), 0.03],
                     [*(tip + [0.0, 0.0, -0.06]), 0.045],
                     [3.0, 0.5, 3.0, 0.04]])
    st = _state(orc, objs=objs)
    out = orc.step(st, _act(grasp=1.0))
    assert out.event == 1 and st.held == 1
    # carried rigidly: p = T_ee c_off after arbitrary motion, fixed tip distance
    d0 = np.linalg.norm(objs[1, :3] - tip)
    rng = np.random.default_rng(2)
    for _ in range(10):
        a = rng.uniform(-1, 1, 11).astype(np.float32)
        a[9] = 1.0
        out = orc.step(st, a)
        _, ee, _ = orc.fk(list(st.base), list(st.q))
        R, t = ee[:9].reshape(3, 3), ee[9:]
        p = np.array([st.obj[1][a_] for a_ in range(3)])
        assert np.allclose(p, R @ np.array(list(st.c_off)) + t, atol=1e-12)
        assert np.linalg.norm(p - t) == pytest.approx(d0, abs=1e-12)
    # a miss when nothing overlaps
    st = _state(orc, objs=objs[2:])
    assert orc.step(st, _act(grasp=1.0)).event == 2 and st.held == -1


def test_snap_lands_on_floor_and_table_exactly():
    table = [0.5, 0.0, -0.5, 1.5, 0.75, 0.5]
    sc = scene_from_boxes([FLOOR, table], (-2, -0.3, -2), (2, 2.5, 2), h=0.02)
    orc = oracle_for(sc)
    tgt = 0.04 + ROBOT.rest_clearance
    y, ok, nb = orc.snap([-1.0, 1.4, 0.3], tgt)
    assert ok and y == pytest.approx(tgt, abs=1e-12)
    y, ok, nb = orc.snap([1.0, 1.4, 0.1], tgt)
    assert ok and y == pytest.approx(0.75 + tgt, abs=1e-12)
    # already resting: stays put
    y, ok, nb = orc.snap([1.0, 0.75 + tgt, 0.1], tgt)
    assert ok and y == pytest.approx(0.75 + tgt, abs=1e-12)


def test_release_lands_or_restores():
    table = [0.3, 0.0, -0.5, 1.5, 0.75, 0.5]
    sc = scene_from_boxes([FLOOR, table], (-2, -0.3, -2), (2, 2.5, 2), h=0.02)
    orc = oracle_for(sc)
    q = ROBOT.q_rest.astype(np.float64)
    tip = _tip(orc, (0, 0, 0), q)[9:]
    rho = 0.04
    start = tip + [0.0, 0.0, 0.06]
    objs = np.array([[*start, rho], [-1.5, 0.5, -1.5, 0.03]])
    st = _state(orc, objs=objs)
    assert orc.step(st, _act(grasp=1.0)).event == 1
    out = orc.step(st, _act(grasp=0.0))
    assert out.event == 3 and st.held == -1
    p = O.Oracle.state_objs(st)[0]
    assert p[0] == pytest.approx(start[0], abs=1e-12)
    assert p[2] == pytest.approx(start[2], abs=1e-12)
    clear = float(np.float32(ROBOT.rest_clearance))   # an FP32 input
    below_floor = 0.0 + rho + clear
    on_table = 0.75 + rho + clear
    assert p[1] == pytest.approx(on_table if 0.3 <= start[0] <= 1.5 else below_floor, abs=1e-12)
    # an object already resting where it would land -> restore p_pre
    land = np.array([start[0], p[1], start[2]])
    objs = np.array([[*start, rho], [*land, 0.03]])
    st = _state(orc, objs=objs)
    orc.step(st, _act(grasp=1.0))
    out = orc.step(st, _act(grasp=0.0))
    assert out.event == 4
    assert np.allclose(O.Oracle.state_objs(st)[0, :3], start, atol=1e-12)


# ------------------------------------------------------- reset

def test_reset_places_objects_on_supports_and_robot_free():
    sc = I.room_scene(1000, 2000)
    orc = oracle_for(sc)
    st = _state(orc)
    out = orc.reset(st, seed=1, env=3, n_obj=10, rho_min=0.03, rho_max=0.06)
    assert out.failed == 0
    objs = O.Oracle.state_objs(st)
    for o in objs:
        on = [s for s in sc.supports
              if s[0] + o[3] - 1e-9 <= o[0] <= s[2] - o[3] + 1e-9
              and s[1] + o[3] - 1e-9 <= o[2] <= s[3] - o[3] + 1e-9
              and abs(o[1] - (s[4] + o[3] + ROBOT.rest_clearance)) < 1e-6]
        assert on, o
        assert 0.03 <= o[3] < 0.06
    for a in range(len(objs)):
        for b in range(a):
            assert np.linalg.norm(objs[a, :3] - objs[b, :3]) >= objs[a, 3] + objs[b, 3]
    # robot free: a zero action is accepted
    assert orc.step(st, np.zeros(11, np.float32)).contact_mask == 0
    assert list(st.q) == pytest.approx(list(ROBOT.q_rest), abs=1e-7)
    # deterministic per (seed, env, episode); a new episode moves things
    st2 = _state(orc)
    orc.reset(st2, seed=1, env=3, n_obj=10, rho_min=0.03, rho_max=0.06)
    assert np.array_equal(O.Oracle.state_objs(st2), objs)
    orc.reset(st2, seed=1, env=3, n_obj=10, rho_min=0.03, rho_max=0.06)
    assert not np.array_equal(O.Oracle.state_objs(st2), objs)


# ------------------------------------------------------- rendering

def _quad_scene(corners, rgb=0x123456):
    v = np.array(corners, np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    return scene_from_boxes([FLOOR], (-5, -1.5, -5), (5, 3, 5), h=0.1,
                            tris=(v, t, np.array([rgb, rgb], np.uint32)))


def _camera(orc, base=(0, 0, 0)):
    _, _, cam = orc.fk(base, ROBOT.q_rest)
    return cam[:9].reshape(3, 3), cam[9:]


def test_depth_of_fronto_parallel_quad():
    W = H = 64
    orc0 = oracle_for(OPEN)
    R, eye = _camera(orc0)
    D = 2.0
    right, up, fwd = R[:, 0], R[:, 1], R[:, 2]
    # quad spanning camera-space x in [-0.5, 0.3], y in [-0.4, 0.6] at z = D,
    # wound so its normal faces the camera
    cs = [eye + fwd * D + right * x + up * y for (x, y) in
          [(-0.5, -0.4), (-0.5, 0.6), (0.3, 0.6), (0.3, -0.4)]]
    sc = _quad_scene(cs)
    orc = oracle_for(sc)
    st = O.Oracle.make_state((0, 0, 0), ROBOT.q_rest)
    depth, rgb, amb, win, stats = orc.render(st, W, H)
    f, c = W / 2, W / 2
    u = np.arange(W) + 0.5
    v = np.arange(H) + 0.5
    inu = (u > c + f * -0.5 / D) & (u < c + f * 0.3 / D)
    inv = (v > c - f * 0.6 / D) & (v < c - f * -0.4 / D)
    cover = inv[:, None] & inu[None, :]
    # float32 vertex storage moves the corners by ~1e-7 m: no pixel centre
    # of this layout lies that close to an edge
    assert cover.sum() == int(inu.sum()) * int(inv.sum()) == (depth > 0).sum()
    assert np.all(depth[cover] == pytest.approx(D, abs=2e-6))
    assert np.all(rgb[cover] == 0x123456) and np.all(rgb[~cover] == 0)


def test_depth_of_tilted_quad_matches_plane():
    W = H = 64
    orc0 = oracle_for(OPEN)
    R, eye = _camera(orc0)
    right, up, fwd = R[:, 0], R[:, 1], R[:, 2]
    # plane through eye + D fwd, tilted about the camera y axis: z = D + k x
    D, k = 2.0, 0.6
    cs = [eye + right * x + up * y + fwd * (D + k * x) for (x, y) in
          [(-0.8, -0.7), (-0.8, 0.7), (0.8, 0.7), (0.8, -0.7)]]
    sc = _quad_scene(cs)
    orc = oracle_for(sc)
    st = O.Oracle.make_state((0, 0, 0), ROBOT.q_rest)
    depth, rgb, amb, win, _ = orc.render(st, W, H)
    f, c = W / 2, W / 2
    jj, ii = np.nonzero(depth > 0)
    assert len(ii) > 500
    # along the ray x = z (u - c)/f:  z = D + k z (u - c)/f  ->  z = D / (1 - k (u - c)/f)
    expect = D / (1 - k * ((ii + 0.5) - c) / f)
    assert np.allclose(depth[jj, ii], expect, rtol=1e-6)


def _bruteforce_raycast(verts, tris, R, eye, W, H, near):
    """Pixel-major FP64 Moller-Trumbore over every front-facing triangle."""
    f, c = W / 2, W / 2
    best = np.full((H, W), np.inf)
    who = np.full((H, W), -1)
    u = (np.arange(W) + 0.5 - c) / f
    v = -(np.arange(H) + 0.5 - c) / f
    dc = np.stack(np.broadcast_arrays(u[None, :], v[:, None], np.ones((1, 1))), -1)
    Dw = dc @ R.T                      # world ray directions, camera z = 1
    for t, (a, b, cc) in enumerate(tris):
        A, B, Cc = (verts[i].astype(np.float64) for i in (a, b, cc))
        e1, e2 = B - A, Cc - A
        if not np.dot(np.cross(e1, e2), A - eye) < 0:
            continue                   # back-facing
        pvec = np.cross(Dw, e2)
        det = pvec @ e1
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / det
            tvec = eye - A
            uu = (pvec @ tvec) * inv
            qvec = np.cross(tvec, e1)
            vv = (Dw @ qvec) * inv
            tt = (qvec @ e2) * inv
        hit = (uu > 0) & (vv > 0) & (uu + vv < 1) & (tt >= near)
        upd = hit & (tt < best)
        best[upd] = tt[upd]
        who[upd] = t
    return np.where(np.isfinite(best), best, 0.0), who


def test_raster_equals_bruteforce_raycast_on_tiny_scene():
    sc = I.room_scene(7, tri_target=300, n_furniture=4, size=4.0, grid_h=0.1)
    orc = oracle_for(sc)
    W = H = 32
    rng = np.random.default_rng(11)
    checked = 0
    for trial in range(4):
        base = (float(rng.uniform(1, 3)), float(rng.uniform(1, 3)), float(rng.uniform(-3, 3)))
        st = O.Oracle.make_state(base, ROBOT.q_rest)
        depth, rgb, amb, win, _ = orc.render(st, W, H)
        _, _, cam = orc.fk(base, ROBOT.q_rest)
        R, eye = cam[:9].reshape(3, 3), cam[9:]
        bd, bw = _bruteforce_raycast(sc.verts, sc.tris, R, eye, W, H, ROBOT.cam_near)
        ok = ~amb
        assert ok.mean() > 0.9
        assert np.array_equal(bw[ok], win[ok])
        assert np.allclose(bd[ok], depth[ok], rtol=1e-12, atol=0)
        checked += ok.sum()
    assert checked > 3000


def test_near_plane_clips_and_objects_render():
    # an object straight ahead renders as its flat colour with depth >= near
    orc0 = oracle_for(OPEN)
    R, eye = _camera(orc0)
    p = eye + R[:, 2] * 0.5
    objs = np.array([[*p, 0.06]])
    orc = oracle_for(OPEN)
    st = O.Oracle.make_state((0, 0, 0), ROBOT.q_rest, objs=objs)
    depth, rgb, amb, win, _ = orc.render(st, 32, 32)
    centre = rgb[15:17, 15:17]
    assert np.all(centre == I.object_colors(256)[0])
    assert np.all(depth[depth > 0] >= ROBOT.cam_near)
    # the icosahedron is inscribed in the sphere: its surface lies between the
    # inradius (0.7947 of the circumradius) and the circumradius from the centre
    assert 0.5 - 0.06 <= depth[16, 16] <= 0.5 - 0.06 * 0.7946
    # an object straddling the near plane is cut by it: nothing nearer than near
    objs = np.array([[*(eye + R[:, 2] * 0.06), 0.05]])
    st = O.Oracle.make_state((0, 0, 0), ROBOT.q_rest, objs=objs)
    depth, rgb, amb, win, _ = orc.render(st, 32, 32)
    assert np.all(depth[depth > 0] >= ROBOT.cam_near - 1e-12)


# ------------------------------------------------------- neural SDF MLP

def _rand_mlp(rng, F=4, widths=(16, 16), scale=0.5):
    dims = [2 * F, *widths, 1]
    Ws = [rng.normal(0, scale, (dims[i + 1], dims[i])) for i in range(len(dims) - 1)]
    bs = [rng.normal(0, 0.1, dims[i + 1]) for i in range(len(dims) - 1)]
    return O.MLP64(rng.normal(0, 1, (F, 3)), Ws, bs)


def test_mlp_one_layer_closed_form_gradient():
    rng = np.random.default_rng(0)
    F = 5
    B = rng.normal(0, 1, (F, 3))
    W = rng.normal(0, 1, (1, 2 * F))
    b = rng.normal(0, 1, 1)
    m = O.MLP64(B, [W], [b])
    X = rng.uniform(-1, 1, (7, 3))
    y = rng.uniform(-0.5, 0.5, 7)
    ph = 2 * np.pi * X @ B.T
    gam = np.concatenate([np.sin(ph), np.cos(ph)], 1)
    pred = gam @ W[0] + b[0]
    assert np.allclose(m.forward(X), pred, atol=1e-13)
    loss, gW, gb = m.loss_grad(X, y, -10, 10)
    sg = np.sign(pred - y) / len(X)
    assert loss == pytest.approx(np.abs(pred - y).mean(), abs=1e-14)
    assert np.allclose(gW[0][0], sg @ gam, atol=1e-13)
    assert gb[0][0] == pytest.approx(sg.sum(), abs=1e-14)


def test_mlp_gradient_matches_central_differences():
    rng = np.random.default_rng(4)
    m = _rand_mlp(rng)
    X = rng.uniform(-1, 1, (5, 3))
    y = m.forward(X) - 3.0          # all residuals positive: loss is smooth here
    loss, gW, gb = m.loss_grad(X, y, -100, 100)
    h = 1e-6
    for l in range(len(m.Ws)):
        for (r, c) in [(0, 0), (m.Ws[l].shape[0] - 1, m.Ws[l].shape[1] - 1), (0, m.Ws[l].shape[1] // 2)]:
            old = m.Ws[l][r, c]
            m.Ws[l][r, c] = old + h
            lp = m.loss_grad(X, y, -100, 100)[0]
            m.Ws[l][r, c] = old - h
            lm = m.loss_grad(X, y, -100, 100)[0]
            m.Ws[l][r, c] = old
            assert gW[l][r, c] == pytest.approx((lp - lm) / (2 * h), abs=1e-8)
        old = m.bs[l][0]
        m.bs[l][0] = old + h
        lp = m.loss_grad(X, y, -100, 100)[0]
        m.bs[l][0] = old - h
        lm = m.loss_grad(X, y, -100, 100)[0]
        m.bs[l][0] = old
        assert gb[l][0] == pytest.approx((lp - lm) / (2 * h), abs=1e-8)


def test_mlp_label_clamp():
    rng = np.random.default_rng(1)
    m = _rand_mlp(rng)
    X = rng.uniform(-1, 1, (4, 3))
    pred = m.forward(X)
    y = np.array([5.0, -5.0, 5.0, -5.0])
    loss, _, _ = m.loss_grad(X, y, -0.2, 1.0)
    assert loss == pytest.approx(np.abs(pred - np.clip(y, -0.2, 1.0)).mean(), abs=1e-14)


# ------------------------------------------------------- invariants

def test_invariants_over_random_rollouts():
    """Accepted poses are contact-free, joints stay in limits, a held object
    stays rigidly attached, depth is 0 or >= near."""
    sc = I.room_scene(1001, 1500)
    orc = oracle_for(sc)
    rng = np.random.default_rng(9)
    acts = I.make_actions(60, 1, "uniform", seed=9)[:, 0]
    st = _state(orc)
    orc.reset(st, seed=5, env=0, n_obj=10, rho_min=0.03, rho_max=0.06)
    for t in range(60):
        prev = (list(st.base), list(st.q))
        out = orc.step(st, acts[t])
        assert all(ROBOT.q_min[k] <= st.q[k] <= ROBOT.q_max[k] for k in range(7))
        if out.reverted:
            assert (list(st.base), list(st.q)) == prev
        elif out.near_band == 0:
            # the accepted pose is contact-free: standing still reports no contact
            probe = O.Oracle.make_state(list(st.base), list(st.q), st.held, list(st.c_off),
                                        list(st.p_pre), O.Oracle.state_objs(st))
            a0 = np.zeros(11, np.float32)
            a0[9] = 1.0 if st.held >= 0 else 0.0
            assert orc.step(probe, a0).contact_mask == 0
        if t % 20 == 0:
            depth, _, _, _, _ = orc.render(st, 32, 32)
            assert np.all((depth == 0) | (depth >= ROBOT.cam_near))


def test_robot_body_renders_as_instanced_spheres():
    """With robot colours given, the robot's collision spheres render like
    the objects: every pixel they win carries its sphere's colour, pixels
    elsewhere are unchanged, and the arm in front of the head camera shows."""
    sc = scene_from_boxes([FLOOR], (-3, -0.3, -3), (3, 2.5, 3), h=0.05)
    rc = I.robot_colors(ROBOT)
    plain = O.Oracle(ROBOT, sc, I.icosahedron(), I.object_colors(256))
    body = O.Oracle(ROBOT, sc, I.icosahedron(), I.object_colors(256), robot_rgb=rc)
    st = O.Oracle.make_state((0, 0, 0), ROBOT.q_rest)
    d0, c0, a0, w0, _ = plain.render(st, 64, 64)
    d1, c1, a1, w1, _ = body.render(st, 64, 64)
    n_tris, nt = len(sc.tris), len(I.icosahedron()[1])
    rob = w1 >= n_tris + O.MAX_OBJ * nt
    assert rob.sum() > 20                                  # the arm is in view
    sphere = (w1[rob] - n_tris) // nt - O.MAX_OBJ
    assert np.array_equal(c1[rob], rc[sphere])
    assert np.all(d1[rob] <= np.where(d0[rob] > 0, d0[rob], np.inf) + 1e-12)
    same = ~rob & ~a0 & ~a1
    assert np.array_equal(c1[same], c0[same]) and np.allclose(d1[same], d0[same])
