"""Pins the oracle's oriented-box object model (appendix "Additional
Collision-Detection Details": resting objects are oriented boxes, a grasped
object is a set of spheres) to facts that do not come from the oracle: closed
forms of the distance to a box in its own frame, brute-force overlap of two
box footprints, the geometry of the carried sphere set, exact landing heights
on a floor and a table top, the rigid carry, and the analytic depth of a box
face in the oracle's image."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2306_07552_b300 import inputs as I

from test_oracle_pins import FLOOR, ROBOT, _act, scene_from_boxes

CLEAR = float(np.float32(ROBOT.rest_clearance))   # an FP32 input


def box_oracle(scene):
    return O.Oracle(ROBOT, scene, I.unit_cube(), I.object_colors(256))


def box_state(objs, boxes, base=(0, 0, 0), q=None, held=-1, c_off=(0, 0, 0), p_pre=(0, 0, 0),
              r_off=None):
    objs = np.asarray(objs, np.float64).reshape(-1, 4).copy()
    boxes = np.asarray(boxes, np.float64).reshape(-1, 4)
    objs[:, 3] = np.linalg.norm(boxes[:, :3], axis=1)     # bounding radius
    return O.Oracle.make_state(base, ROBOT.q_rest if q is None else q, held, c_off, p_pre, objs,
                               boxes=boxes, r_off=r_off)


def ry(yaw):
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])


def test_box_distance_closed_forms_in_the_box_frame():
    h = np.array([0.2, 0.1, 0.05])
    for yaw in (0.0, 0.7, -2.3):
        R = ry(yaw)
        p = np.array([1.0, 0.5, -2.0])
        st = box_state([[*p, 0]], [[*h, yaw]])
        world = lambda q: p + R @ np.asarray(q, np.float64)  # noqa: E731
        # beside the +x face: the gap along the box's own x axis
        assert O.box_distance(st, 0, world([0.2 + 0.03, 0.02, -0.01])) == pytest.approx(0.03, abs=1e-14)
        # over the top face
        assert O.box_distance(st, 0, world([0.1, 0.1 + 0.4, 0.0])) == pytest.approx(0.4, abs=1e-14)
        # outside a corner: Euclidean distance to that corner
        q = np.array([0.25, -0.13, 0.09])
        assert O.box_distance(st, 0, world(q)) == pytest.approx(
            np.linalg.norm(q - [0.2, -0.1, 0.05]), abs=1e-14)
        # inside: minus the distance to the nearest face (z, 0.05 - 0.01)
        assert O.box_distance(st, 0, world([0.05, 0.0, 0.01])) == pytest.approx(-0.04, abs=1e-14)
        # a world axis step is not a box axis step when the box is turned
        if yaw != 0.0:
            assert O.box_distance(st, 0, p + [0.23, 0, 0]) != pytest.approx(0.03, abs=1e-6)


def _footprint_overlap_brute(pa, ba, pb, bb, n=240):
    """Sample box a's footprint densely and test the samples against box b
    (in b's frame); vertical intervals by hand."""
    if abs(pa[1] - pb[1]) >= ba[1] + bb[1]:
        return False
    u = np.linspace(-1, 1, n)
    X, Z = np.meshgrid(u * ba[0], u * ba[2])
    Ra, Rb = ry(ba[3]), ry(bb[3])
    pts = np.stack([X.ravel(), np.zeros(X.size), Z.ravel()], 1) @ Ra.T + pa
    qb = (pts - pb) @ Rb                 # R_b^T (p - p_b), row by row
    return bool(np.any((np.abs(qb[:, 0]) < bb[0]) & (np.abs(qb[:, 2]) < bb[2])))


def test_box_overlap_matches_brute_force():
    rng = np.random.default_rng(3)
    agree = checked = 0
    for _ in range(400):
        ba = [*rng.uniform(0.03, 0.12, 3), rng.uniform(-math.pi, math.pi)]
        bb = [*rng.uniform(0.03, 0.12, 3), rng.uniform(-math.pi, math.pi)]
        pa = np.array([0.0, 0.0, 0.0])
        pb = np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.2, 0.2), rng.uniform(-0.3, 0.3)])
        got, nb = O.boxes_overlap(pa, ba, pb, bb)
        # footprints that nearly touch are left out (sampling resolution)
        d = np.linalg.norm(pb[[0, 2]] - pa[[0, 2]])
        if nb:
            continue
        brute = _footprint_overlap_brute(pa, ba, pb, bb)
        brute_rev = _footprint_overlap_brute(pb, bb, pa, ba)
        if brute != brute_rev:           # a sliver the samples straddle: unresolved
            continue
        checked += 1
        agree += got == brute
        assert got == brute, (pa, ba, pb, bb, d)
    assert checked > 300
    # touching faces do not overlap; a hair closer they do
    b = [0.1, 0.1, 0.1, 0.0]
    assert not O.boxes_overlap([0, 0, 0], b, [0.2, 0, 0], b)[0]
    assert O.boxes_overlap([0, 0, 0], b, [0.2 - 1e-3, 0, 0], b)[0]
    # stacked boxes do not overlap; interpenetrating vertically they do
    assert not O.boxes_overlap([0, 0, 0], b, [0.05, 0.2, 0], b)[0]
    assert O.boxes_overlap([0, 0, 0], b, [0.05, 0.19, 0], b)[0]
    # a square turned by 45 degrees reaches sqrt(2) h along the diagonal
    t = [0.1, 0.1, 0.1, math.pi / 4]
    assert O.boxes_overlap([0, 0, 0], t, [0.1 * math.sqrt(2) + 0.1 - 1e-3, 0, 0], b)[0]
    assert not O.boxes_overlap([0, 0, 0], t, [0.1 * math.sqrt(2) + 0.1 + 1e-3, 0, 0], b)[0]


def test_carried_sphere_set_geometry():
    h = np.array([0.05, 0.03, 0.04])
    c, s = O.box_spheres(h)
    assert s == 0.03
    # eight inset corners, each sphere inside the box and touching its three
    # nearest faces (or the face pair along the thinnest axis)
    assert np.allclose(np.abs(c), [0.02, 0.0, 0.01], atol=1e-15)
    assert len({tuple(np.sign(x) for x in row[[0, 2]]) for row in c}) == 4   # four columns
    for k in range(8):
        assert np.all(np.abs(c[k]) + s <= h + 1e-15)
    # a cube collapses to one sphere at its centre, the inscribed ball
    c, s = O.box_spheres([0.04, 0.04, 0.04])
    assert s == 0.04 and np.all(c == 0)


def test_box_contact_bit_follows_the_exact_distance():
    scene = scene_from_boxes([FLOOR], (-5, -0.3, -5), (5, 2.5, 5), h=0.05)
    orc = box_oracle(scene)
    cs = orc.sphere_centres((0, 0, 0), ROBOT.q_rest.astype(np.float64))
    i = int(np.argmax(cs[:, 1]))         # the highest robot sphere, clear of the floor
    r = float(np.float32(ROBOT.sphere_radius[i]))
    h = np.array([0.1, 0.08, 0.06])
    for yaw in (0.0, 0.9):
        R = ry(yaw)
        for gap, hit in ((1e-3, False), (-1e-3, True)):
            # the box's +x face sits r + gap from the sphere centre
            p = cs[i] - R @ np.array([h[0] + r + gap, 0.0, 0.0])
            st = box_state([[*p, 0]], [[*h, yaw]])
            out = orc.step(st, _act())
            assert bool(out.contact_mask >> i & 1) == hit
            assert bool(out.flags & 2) == hit and (out.reverted == hit)


def test_grasp_carries_the_box_rigidly_and_release_lands_upright():
    table = [0.3, 0.0, -0.5, 1.5, 0.75, 0.5]
    scene = scene_from_boxes([FLOOR, table], (-2, -0.3, -2), (2, 2.5, 2), h=0.02)
    orc = box_oracle(scene)
    q = ROBOT.q_rest.astype(np.float64)
    _, ee, _ = orc.fk((0, 0, 0), q)
    tip = ee[9:]
    h = np.array([0.05, 0.04, 0.03])
    yaw = 0.6
    # the box's centre 5 cm below the tip: its top face 1 cm below the tip,
    # inside the 3 cm suction sphere; a second box farther away
    p0 = tip - [0, 0.05, 0]
    st = box_state([[*p0, 0], [1.0, 0.8, 0.3, 0]], [[*h, yaw], [0.05, 0.05, 0.05, 0.0]])
    out = orc.step(st, _act(grasp=1.0))
    assert out.event == 1 and st.held == 0
    Re = ee[:9].reshape(3, 3)
    Roff = np.array(list(st.r_off)).reshape(3, 3)
    assert np.allclose(Re @ Roff, ry(yaw), atol=1e-12)
    rng = np.random.default_rng(5)
    for _ in range(8):
        a = rng.uniform(-1, 1, 11).astype(np.float32)
        a[9] = 1.0
        orc.step(st, a)
        _, ee, _ = orc.fk(list(st.base), list(st.q))
        R, t = ee[:9].reshape(3, 3), ee[9:]
        p = O.Oracle.state_objs(st)[0, :3]
        assert np.allclose(p, R @ np.array(list(st.c_off)) + t, atol=1e-12)
        Rw = R @ np.array(list(st.r_off)).reshape(3, 3)
        assert np.allclose(Rw.T @ Rw, np.eye(3), atol=1e-12)      # still a rotation
    # release over the floor: upright about the current heading, resting at
    # floor + hy + clearance exactly (the bottom spheres land at s + clearance)
    Rw = R @ np.array(list(st.r_off)).reshape(3, 3)
    heading = math.atan2(-Rw[2, 0], Rw[0, 0])
    p = O.Oracle.state_objs(st)[0, :3].copy()
    out = orc.step(st, _act(grasp=0.0))
    assert st.held == -1
    land = O.Oracle.state_objs(st)[0]
    box = O.Oracle.state_boxes(st)[0]
    if out.event == 3:
        assert box[3] == pytest.approx(heading, abs=1e-12)
        assert land[0] == pytest.approx(p[0], abs=1e-12) and land[2] == pytest.approx(p[2], abs=1e-12)
        on_table = 0.3 - 0.1 < p[0] < 1.5 + 0.1 and abs(p[2]) < 0.6
        if not on_table:
            assert land[1] == pytest.approx(0.0 + h[1] + CLEAR, abs=1e-12)
    else:
        assert out.event == 4 and np.allclose(land[:3], p0, atol=1e-12)


def test_release_on_a_table_and_restore_on_overlap():
    table = [-1.0, 0.0, -1.0, 1.0, 0.75, 1.0]
    scene = scene_from_boxes([FLOOR, table], (-2, -0.3, -2), (2, 2.5, 2), h=0.02)
    orc = box_oracle(scene)
    q = ROBOT.q_rest.astype(np.float64)
    _, ee, _ = orc.fk((0, 0, 0), q)
    Re, tip = ee[:9].reshape(3, 3), ee[9:]
    h = np.array([0.06, 0.05, 0.04])
    p = tip - [0, 0.06, 0]
    # held already: tool-frame offset and rotation of an upright box, yaw 0.3
    c_off = Re.T @ (p - tip)
    r_off = Re.T @ ry(0.3)
    st = box_state([[*p, 0]], [[*h, 0.3]], held=0, c_off=c_off, p_pre=[1.5, 0.8, 1.5],
                   r_off=r_off)
    if p[1] - h[1] > 0.75 and abs(p[0]) < 0.9 and abs(p[2]) < 0.9:
        out = orc.step(st, _act(grasp=0.0))
        assert out.event == 3
        land = O.Oracle.state_objs(st)[0]
        assert land[1] == pytest.approx(0.75 + h[1] + CLEAR, abs=1e-12)
        assert O.Oracle.state_boxes(st)[0][3] == pytest.approx(0.3, abs=1e-12)
        # a box already resting where this one would land: back to p_pre
        st = box_state([[*p, 0], [land[0] + 0.05, land[1], land[2], 0]],
                       [[*h, 0.3], [0.05, 0.05, 0.05, 1.0]], held=0, c_off=c_off,
                       p_pre=[1.5, 0.8, 1.5], r_off=r_off)
        out = orc.step(st, _act(grasp=0.0))
        assert out.event == 4
        assert np.allclose(O.Oracle.state_objs(st)[0, :3], [1.5, 0.8, 1.5], atol=1e-12)
    else:   # the robot's rest pose must hold the tip above the table for this pin
        pytest.fail("tool tip not above the table in the rest pose")


def test_reset_places_boxes_upright_on_supports_without_overlap():
    tables = [[0.5, 0.0, -1.5, 1.7, 0.7, -0.3], [-1.8, 0.0, 0.4, -0.4, 0.9, 1.6]]
    sup = [[0.5, -1.5, 1.7, -0.3, 0.7], [-1.8, 0.4, -0.4, 1.6, 0.9]]
    sup32 = np.asarray(sup, np.float32).astype(np.float64)   # as the scene stores them
    scene = scene_from_boxes([FLOOR, *tables], (-2.5, -0.3, -2.5), (2.5, 2.5, 2.5), h=0.02,
                             supports=sup, spawn=[-2, -2, 2, 2])
    orc = box_oracle(scene)
    for env in range(6):
        st = box_state(np.zeros((0, 4)), np.zeros((0, 4)))
        st.boxes = 1
        out = orc.reset(st, 7, env, 12, 0.03, 0.06)
        P, B = O.Oracle.state_objs(st), O.Oracle.state_boxes(st)
        assert len(P) == 12
        for j in range(12):
            hx, hy, hz, yaw = B[j]
            assert 0.03 <= min(hx, hy, hz) and max(hx, hy, hz) < 0.06
            assert P[j, 3] == pytest.approx(math.sqrt(hx * hx + hy * hy + hz * hz), abs=1e-15)
            # on one support's top, its turned footprint inside the top
            on = [k for k, s in enumerate(sup32) if abs(P[j, 1] - (s[4] + hy + CLEAR)) < 1e-12]
            assert on, j
            s = sup32[on[0]]
            corners = [P[j, [0, 2]] + (ry(yaw) @ [sx * hx, 0, sz * hz])[[0, 2]]
                       for sx in (-1, 1) for sz in (-1, 1)]
            for cx, cz in corners:
                assert s[0] - 1e-12 <= cx <= s[2] + 1e-12 and s[1] - 1e-12 <= cz <= s[3] + 1e-12
            if out.failed == 0:
                for k in range(j):
                    assert not _footprint_overlap_brute(P[j, :3], B[j], P[k, :3], B[k])


def test_box_face_depth_in_the_oracle_image():
    scene = scene_from_boxes([FLOOR], (-5, -0.3, -5), (5, 2.5, 5), h=0.05)
    orc = box_oracle(scene)
    base = (0.0, 0.0, 0.3)
    q = ROBOT.q_rest.astype(np.float64)
    _, _, cam = orc.fk(base, q)
    R, eye = cam[:9].reshape(3, 3), cam[9:]
    W = H = 64
    # a large box whose -x face is the plane x = eye_x + 1.5 (world), turned
    # by the base yaw so that face is square to the camera's heading
    yaw = base[2]
    hx = 0.5
    centre = eye + ry(yaw) @ [1.5 + hx, 0.0, 0.0]
    st = box_state([[*centre, 0]], [[hx, 2.5, 1.2, yaw]], base=base, q=q)
    depth, rgb, amb, win, _ = orc.render(st, W, H)
    n = ry(yaw) @ [1.0, 0, 0]            # the face's outward normal is -n
    checked = 0
    for j in (20, 32, 44):
        for i in (20, 32, 44):
            d = R @ [(i + 0.5 - W / 2) / (W / 2), -(j + 0.5 - H / 2) / (W / 2), 1.0]
            t = 1.5 / float(n @ d)        # ray eye + t d meets the face plane
            if not amb[j, i]:
                assert depth[j, i] == pytest.approx(t, rel=1e-12)
                assert rgb[j, i] == I.object_colors(256)[0]
                checked += 1
    assert checked >= 8
