"""Pins the oracle's column grid (appendix "Additional Collision-Detection
Details": per working-set radius, vertical columns 3 cm apart holding the
free spans of a sphere centre's height) to closed forms and brute force."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2306_07552_b300 import inputs as I

from test_oracle_pins import FLOOR, ROBOT, _act, _state, oracle_for, scene_from_boxes

CEIL = [-20, 2.5, -20, 20, 2.7, 20]          # ceiling slab, underside y = 2.5
R = [0.015, 0.05, 0.12]
f32 = lambda v: float(np.float32(v))         # noqa: E731 -- box coordinates are FP32 inputs


def _room(*boxes):
    sc = scene_from_boxes([FLOOR, CEIL, *boxes], (-1.5, -0.2, -1.5), (1.5, 2.6, 1.5), h=0.05)
    return sc, oracle_for(sc)


def test_radius_index_takes_the_smallest_working_radius_not_below():
    L = O.lib()
    assert [L.orc_column_radius_index(r) for r in (0.01, 0.015, 0.03, 0.05, 0.06, 0.1, 0.2)] == \
        [0, 0, 1, 1, 2, 2, 2]
    assert L.orc_column_radius_index(f32(0.05)) == 1      # FP32 radius just above 0.05


def test_open_floor_has_one_span_per_radius():
    sc, orc = _room()
    for ri in range(3):
        sp = orc.column_spans(ri, 40, 40)
        assert sp.shape == (1, 2)
        assert sp[0] == pytest.approx([0.0 + R[ri], f32(2.5) - R[ri]], abs=1e-12)


def test_table_splits_the_column_into_two_layers():
    top = [-0.6, 0.7, -0.6, 0.6, 0.75, 0.6]
    sc, orc = _room(top)
    dims = orc.column_dims()
    i = k = 50                          # x = z = origin + 1.5 m = 0: under the table centre
    assert sc.grid_origin[0] + i * 0.03 == pytest.approx(0.0, abs=1e-6)
    for ri in range(3):
        sp = orc.column_spans(ri, i, k)
        assert sp == pytest.approx(np.array([[R[ri], f32(0.7) - R[ri]],
                                             [f32(0.75) + R[ri], f32(2.5) - R[ri]]]), abs=1e-9)
    assert dims == (101, 101)


def test_span_end_beside_a_box_edge_is_the_sphere_touching_the_corner():
    block = [0.3, 0.0, -2.0, 2.0, 1.0, 2.0]       # x >= 0.3 blocked up to y = 1
    sc, orc = _room(block)
    i = int(np.floor((0.3 - sc.grid_origin[0]) / 0.03 - 1e-6))   # last column before x = 0.3
    x = sc.grid_origin[0] + i * 0.03
    dxz = f32(0.3) - x
    assert 0 < dxz < 0.05
    sp = orc.column_spans(1, i, 40)
    e = math.sqrt(0.05 ** 2 - dxz ** 2)
    assert sp[0] == pytest.approx([f32(1.0) + e, f32(2.5) - 0.05], abs=1e-9)


def test_column_spans_match_brute_force_sphere_box_distances():
    boxes = [[-0.6, 0.7, -0.6, 0.6, 0.75, 0.6], [-0.55, 0.0, -0.55, -0.5, 0.7, -0.5],
             [0.4, 0.0, 0.2, 1.2, 1.8, 0.5], [-1.0, 0.4, 0.8, -0.2, 0.45, 1.2]]
    sc, orc = _room(*boxes)
    allb = [FLOOR, CEIL, *boxes]
    rng = np.random.default_rng(5)
    dims = orc.column_dims()
    for _ in range(300):
        ri = int(rng.integers(0, 3))
        i, k = int(rng.integers(0, dims[0])), int(rng.integers(0, dims[1]))
        x, z = sc.grid_origin[0] + i * 0.03, sc.grid_origin[2] + k * 0.03
        sp = orc.column_spans(ri, i, k)
        for y in rng.uniform(-0.1, 2.6, 8):
            p = np.array([x, y, z])
            hit = any(O.box_sdf(p, np.array(b, np.float32)) < R[ri] for b in allb)
            ylo, yhi = sc.grid_origin[1], sc.grid_origin[1] + (sc.grid_dims[1] - 1) * sc.grid_h
            hit = hit or not (ylo <= y <= yhi)
            free = any(a <= y <= b for a, b in sp)
            margin = min([abs(y - v) for v in sp.ravel()] + [1.0])
            if margin > 1e-9:
                assert free == (not hit), (ri, i, k, y, sp)


def test_query_uses_the_nearest_column_and_inflated_radius():
    wall = [0.5, 0.0, -2.0, 2.0, 2.5, 2.0]        # face at x = 0.5
    sc, orc = _room(wall)
    # r = 0.1 -> column radius 0.12: a centre 0.11 from the wall is in contact
    # on the column grid although the distance grid says free
    c = [f32(0.5) - 0.11, 1.0, 0.0]
    assert orc.column_contact(c, 0.1)[0]
    inside, d, _ = orc.grid_query(c)
    assert inside and d > 0.1
    # nearest column: 1.4 cm vs 1.6 cm past a column centre
    i = int(round((0.0 - sc.grid_origin[0]) / 0.03))
    x0 = sc.grid_origin[0] + i * 0.03
    lo_i = orc.column_spans(1, i, 40)
    lo_n = orc.column_spans(1, i + 1, 40)
    assert lo_i.shape == lo_n.shape == (1, 2)
    hit_a, nb_a = orc.column_contact([x0 + 0.014, 1.0, sc.grid_origin[2] + 40 * 0.03], 0.05)
    assert not hit_a and nb_a == 0
    # outside the columns' extent: contact
    assert orc.column_contact([sc.grid_origin[0] - 0.05, 1.0, 0.0], 0.05)[0]


def test_smaller_sphere_rests_on_the_floor_as_with_its_own_radius():
    sc, orc = _room()
    x = sc.grid_origin[0] + 40 * 0.03
    for r in (0.03, 0.1, f32(0.1)):
        # spans for R >= r widened by R - r: a sphere resting above the floor
        # is free exactly when its centre is at least r high
        assert not orc.column_contact([x, r + 1e-3, x], r)[0]
        assert orc.column_contact([x, r - 1e-3, x], r)[0]


def test_step_on_the_column_grid():
    wall = [0.45, -1.0, -5.0, 3.0, 3.0, 5.0]
    sc = scene_from_boxes([FLOOR, wall], (-2, -0.3, -2), (1.5, 2.5, 2), h=0.05)
    orc = oracle_for(sc)
    # standing still 0.2 m from the wall: base spheres r = 0.1 -> 0.12 columns
    cand = orc.sphere_centres([0.2, 0.0, 0.0], ROBOT.q_rest)
    expect = 0
    for i, (c, r) in enumerate(zip(cand, ROBOT.sphere_radius)):
        if orc.column_contact(c, r)[0]:
            expect |= 1 << i
    out = orc.step_ex(_state(orc, base=(0.2, 0, 0)), np.zeros(11, np.float32), column=True)
    assert out.contact_mask == expect
    out2 = orc.step_ex(_state(orc, base=(0.2, 0, 0)), np.zeros(11, np.float32))
    assert (out2.contact_mask & ~expect) == 0        # the column grid is conservative here
