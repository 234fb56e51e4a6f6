"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This module only *creates inputs*: the robot description, procedural scenes
(solid boxes plus the triangle soup that renders them), the instanced object
mesh, object colours and action sequences.  It holds none of the method's
arithmetic (no kinematics, no distance field, no collision, no rendering), so
both sides of every parity test can consume it without sharing code.

The synthetic scenes stand in for the ReplicaCAD apartments, YCB objects and
Rearrange-Easy episodes the paper trains on (Sec. 4.1), which are not
available here.  They keep the paper's shapes: apartment-scale indoor scenes
with furniture, tens of free objects per environment, a 128x128 90-degree
head camera (Sec. 4.1) and 11-dimensional actions in [-1, 1] (App. A).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# Robot: a Fetch-like mobile manipulator in round numbers.
#
# The paper approximates each articulated link with hand-authored spheres
# (App. "Additional Collision-Detection Details") but does not list them.
# This table is our own Fetch-like choice: SE(2) base, 7 revolute joints with
# axes alternating yaw / pitch / roll, 30 collision spheres of radius 3-10 cm.
# Frames: link k's frame sits at joint k; sphere centres are in that frame.
# Axis codes: 0 = x, 1 = y, 2 = z.
# --------------------------------------------------------------------------

N_JOINTS = 7
N_ACTIONS = 11  # fwd, rot, 7 joint deltas, grasp, stop (Sec. 4.1, App. A)


@dataclass
class Robot:
    link_offset: np.ndarray  # [8][3]  o_1..o_7 and the tool tip offset
    link_axis: np.ndarray    # [7] int32
    q_min: np.ndarray        # [7]
    q_max: np.ndarray        # [7]
    q_rest: np.ndarray       # [7]
    dq_max: float            # rad per step at |a| = 1
    base_step: float         # m per step at |a| = 1 (App. A: 10 cm)
    base_turn: float         # rad per step at |a| = 1 (App. A: 5 degrees)
    sphere_link: np.ndarray  # [S] int32, 0 = base, k = link k
    sphere_pos: np.ndarray   # [S][3]
    sphere_radius: np.ndarray  # [S]
    cam_pos: np.ndarray      # [3] head camera position in the base frame
    cam_pitch: float         # rad, negative looks down
    cam_near: float          # near plane (m)
    grasp_radius: float      # suction sphere at the tool tip (Sec. 3.2: 3 cm)
    rest_clearance: float    # resting objects float this far above contact


def fetch_like_robot() -> Robot:
    f32 = np.float32
    link_offset = np.array([
        [0.12, 0.72, 0.00],   # shoulder pan  (axis y)
        [0.12, 0.00, 0.00],   # shoulder lift (axis z)
        [0.20, 0.00, 0.00],   # upper-arm roll (axis x)
        [0.15, 0.00, 0.00],   # elbow flex    (axis z)
        [0.14, 0.00, 0.00],   # forearm roll  (axis x)
        [0.15, 0.00, 0.00],   # wrist flex    (axis z)
        [0.14, 0.00, 0.00],   # wrist roll    (axis x)
        [0.16, 0.00, 0.00],   # tool tip (suction cup) in link-7 frame
    ], dtype=f32)
    link_axis = np.array([1, 2, 0, 2, 0, 2, 0], dtype=np.int32)
    spheres = []
    # base ring: 6 spheres of 10 cm, 2 cm above the floor
    for k in range(6):
        a = k * math.pi / 3.0
        spheres.append((0, (0.17 * math.cos(a), 0.12, 0.17 * math.sin(a)), 0.10))
    spheres += [
        (0, (-0.05, 0.35, 0.0), 0.10),   # torso
        (0, (-0.05, 0.55, 0.0), 0.10),
        (0, (-0.05, 0.75, 0.0), 0.10),
        (0, (0.06, 1.08, 0.0), 0.10),    # head (holds the camera)
        (1, (0.00, 0.00, 0.0), 0.07),    # shoulder
        (1, (0.06, 0.00, 0.0), 0.06),
        (2, (0.04, 0.00, 0.0), 0.06),    # upper arm
        (2, (0.10, 0.00, 0.0), 0.055),
        (2, (0.16, 0.00, 0.0), 0.055),
        (3, (0.05, 0.00, 0.0), 0.055),
        (3, (0.11, 0.00, 0.0), 0.05),
        (4, (0.00, 0.00, 0.0), 0.055),   # elbow / forearm
        (4, (0.06, 0.00, 0.0), 0.05),
        (4, (0.12, 0.00, 0.0), 0.05),
        (5, (0.05, 0.00, 0.0), 0.045),
        (5, (0.11, 0.00, 0.0), 0.045),
        (6, (0.00, 0.00, 0.0), 0.045),   # wrist
        (6, (0.06, 0.00, 0.0), 0.04),
        (6, (0.12, 0.00, 0.0), 0.04),
        (7, (0.02, 0.00, 0.0), 0.04),    # gripper body, ends 6 cm short of the tip
        (7, (0.07, 0.00, 0.0), 0.035),
        (7, (0.08, 0.03, 0.0), 0.03),
        (7, (0.08, -0.03, 0.0), 0.03),
        (7, (0.10, 0.00, 0.0), 0.03),
    ]
    assert len(spheres) == 30
    return Robot(
        link_offset=link_offset,
        link_axis=link_axis,
        q_min=np.full(7, -2.5, f32),
        q_max=np.full(7, 2.5, f32),
        q_rest=np.array([0.0, -1.3, 0.0, 2.2, 0.0, 1.2, 0.0], f32),
        dq_max=0.1,
        base_step=0.10,
        base_turn=5.0 * math.pi / 180.0,
        sphere_link=np.array([s[0] for s in spheres], np.int32),
        sphere_pos=np.array([s[1] for s in spheres], f32),
        sphere_radius=np.array([s[2] for s in spheres], f32),
        cam_pos=np.array([0.08, 1.10, 0.0], f32),
        cam_pitch=-0.35,
        cam_near=0.05,
        grasp_radius=0.03,
        rest_clearance=0.001,
    )


# --------------------------------------------------------------------------
# Instanced object mesh: free objects render as icosahedra inscribed in their
# collision sphere (unit circumradius, scaled by the object radius).
# --------------------------------------------------------------------------

def icosahedron() -> tuple[np.ndarray, np.ndarray]:
    p = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([
        [-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
        [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
        [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1],
    ], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ], dtype=np.int32)
    # make every face wind counter-clockwise seen from outside
    for t in range(len(f)):
        a, b, c = v[f[t]]
        if np.dot(np.cross(b - a, c - a), a + b + c) < 0:
            f[t] = f[t][[0, 2, 1]]
    return v.astype(np.float32), f


def unit_cube() -> tuple[np.ndarray, np.ndarray]:
    """The box objects' instance mesh: corners (+-1, +-1, +-1), corner k
    having the signs of bits 0 (x), 1 (y), 2 (z) of k (clear = minus); two
    triangles per face, counter-clockwise seen from outside."""
    v = np.array([[1.0 if (k >> a) & 1 else -1.0 for a in range(3)] for k in range(8)])
    f = np.array([[0, 4, 6], [0, 6, 2], [1, 3, 7], [1, 7, 5], [0, 1, 5], [0, 5, 4],
                  [2, 6, 7], [2, 7, 3], [0, 2, 3], [0, 3, 1], [4, 5, 7], [4, 7, 6]], np.int32)
    return v.astype(np.float32), f


def robot_colors(robot: "Robot") -> np.ndarray:
    """Flat colour of each robot collision sphere when the robot body is
    rendered: grey shades by link (base darkest)."""
    link = np.asarray(robot.sphere_link, np.int64)
    g = (0x50 + 0x12 * link).astype(np.uint32)
    return ((g << 16) | (g << 8) | (g + 0x10)).astype(np.uint32)


def object_colors(m: int, seed: int = 77) -> np.ndarray:
    rng = np.random.default_rng(seed)
    hues = (np.arange(m) * 0.61803398875 + rng.random()) % 1.0
    out = np.zeros(m, np.uint32)
    for j, h in enumerate(hues):
        r, g, b = _hsv(h, 0.75, 0.95)
        out[j] = (r << 16) | (g << 8) | b
    return out


def _hsv(h, s, v):
    i = int(h * 6.0) % 6
    f = h * 6.0 - int(h * 6.0)
    p, q, t = v * (1 - s), v * (1 - f * s), v * (1 - (1 - f) * s)
    r, g, b = [(v, t, p), (q, v, p), (p, v, t), (p, q, v), (t, p, v), (v, p, q)][i]
    return int(r * 255), int(g * 255), int(b * 255)


# --------------------------------------------------------------------------
# Procedural scenes.  A scene is a union of axis-aligned solid boxes (the
# static geometry the distance grid is built from), the tessellated triangle
# soup that renders those boxes, flat per-triangle colours, the support
# rectangles objects are placed on, the distance-grid lattice and the region
# the robot base is spawned in.
# --------------------------------------------------------------------------

@dataclass
class Scene:
    boxes: np.ndarray        # [B][6] f32 min xyz, max xyz
    box_rgb: np.ndarray      # [B] u32
    verts: np.ndarray        # [V][3] f32
    tris: np.ndarray         # [T][3] i32 (counter-clockwise seen from outside)
    tri_rgb: np.ndarray      # [T] u32 0xRRGGBB
    supports: np.ndarray     # [P][5] f32 x0, z0, x1, z1, top_y
    grid_origin: np.ndarray  # [3] f32
    grid_h: float
    grid_dims: np.ndarray    # [3] i32 nx, ny, nz
    spawn: np.ndarray        # [4] f32 x0, z0, x1, z1
    meta: dict = field(default_factory=dict)

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])


class _Builder:
    def __init__(self, rng: np.random.Generator):
        self.rng = rng
        self.boxes: list[tuple] = []
        self.rgb: list[int] = []
        self.hidden: list[tuple] = []   # faces never rendered: (box index, face id)
        self.supports: list[tuple] = []

    def box(self, lo, hi, rgb, skip_faces=()):
        lo = [float(x) for x in lo]
        hi = [float(x) for x in hi]
        assert all(h > l for l, h in zip(lo, hi)), (lo, hi)
        self.boxes.append((*lo, *hi))
        self.rgb.append(int(rgb))
        for f in skip_faces:
            self.hidden.append((len(self.boxes) - 1, f))
        return len(self.boxes) - 1

    def jitter(self, rgb, amt=18):
        r, g, b = (rgb >> 16) & 255, (rgb >> 8) & 255, rgb & 255
        d = self.rng.integers(-amt, amt + 1, 3)
        r, g, b = [int(np.clip(c + dc, 0, 255)) for c, dc in zip((r, g, b), d)]
        return (r << 16) | (g << 8) | b


# face ids: 0 -x, 1 +x, 2 -y, 3 +y, 4 -z, 5 +z
_FACE_SHADE = [0.80, 0.80, 0.55, 1.00, 0.90, 0.90]


def _face_quads(b, face):
    """(origin, edge_a, edge_b) of a box face with edge_a x edge_b outward."""
    x0, y0, z0, x1, y1, z1 = b
    if face == 0:   # -x: a = +z, b = +y -> a x b = -x
        return (x0, y0, z0), (0, 0, z1 - z0), (0, y1 - y0, 0)
    if face == 1:   # +x: a = +y, b = +z -> +x
        return (x1, y0, z0), (0, y1 - y0, 0), (0, 0, z1 - z0)
    if face == 2:   # -y: a = +x, b = +z -> x cross z = -y
        return (x0, y0, z0), (x1 - x0, 0, 0), (0, 0, z1 - z0)
    if face == 3:   # +y: a = +z, b = +x -> z cross x = +y
        return (x0, y1, z0), (0, 0, z1 - z0), (x1 - x0, 0, 0)
    if face == 4:   # -z: a = +y, b = +x -> y cross x = -z
        return (x0, y0, z0), (0, y1 - y0, 0), (x1 - x0, 0, 0)
    return (x0, y0, z1), (x1 - x0, 0, 0), (0, y1 - y0, 0)  # +z: x cross y = +z


def _shade(rgb, s):
    r, g, b = (rgb >> 16) & 255, (rgb >> 8) & 255, rgb & 255
    return (int(r * s) << 16) | (int(g * s) << 8) | int(b * s)


def _tessellate(boxes, rgbs, hidden, cell):
    hidden = set(hidden)
    faces = []
    for bi, b in enumerate(boxes):
        for f in range(6):
            if (bi, f) in hidden:
                continue
            o, a, bb = _face_quads(b, f)
            la, lb = math.sqrt(sum(x * x for x in a)), math.sqrt(sum(x * x for x in bb))
            nu, nv = max(1, math.ceil(la / cell - 1e-9)), max(1, math.ceil(lb / cell - 1e-9))
            faces.append((bi, f, o, a, bb, nu, nv))
    return faces


def _count(faces):
    return sum(2 * f[5] * f[6] for f in faces)


def _emit(faces, rgbs):
    verts, tris, cols = [], [], []
    base = 0
    for (bi, f, o, a, bb, nu, nv) in faces:
        o, a, bb = np.array(o), np.array(a), np.array(bb)
        iu, iv = np.meshgrid(np.arange(nu + 1), np.arange(nv + 1), indexing="ij")
        pts = o + (iu[..., None] / nu) * a + (iv[..., None] / nv) * bb
        verts.append(pts.reshape(-1, 3))
        idx = np.arange((nu + 1) * (nv + 1)).reshape(nu + 1, nv + 1) + base
        p00, p10 = idx[:-1, :-1], idx[1:, :-1]
        p11, p01 = idx[1:, 1:], idx[:-1, 1:]
        t1 = np.stack([p00, p10, p11], -1).reshape(-1, 3)
        t2 = np.stack([p00, p11, p01], -1).reshape(-1, 3)
        tt = np.stack([t1, t2], 1).reshape(-1, 3)
        tris.append(tt)
        cols.append(np.full(len(tt), _shade(rgbs[bi], _FACE_SHADE[f]), np.uint32))
        base += (nu + 1) * (nv + 1)
    return (np.concatenate(verts).astype(np.float32), np.concatenate(tris).astype(np.int32),
            np.concatenate(cols))


def _finish(bld: _Builder, tri_target: int, lo, hi, grid_h, spawn, meta) -> Scene:
    boxes = bld.boxes
    # pick the quad size whose tessellation lands closest to the target count
    a, b = 0.005, 20.0
    for _ in range(60):
        mid = math.sqrt(a * b)
        if _count(_tessellate(boxes, bld.rgb, bld.hidden, mid)) > tri_target:
            a = mid
        else:
            b = mid
    faces = _tessellate(boxes, bld.rgb, bld.hidden, b)
    verts, tris, cols = _emit(faces, bld.rgb)
    pad = 0.2
    origin = np.array([lo[0] - pad, lo[1] - pad, lo[2] - pad], np.float32)
    ext = np.array([hi[0] - lo[0] + 2 * pad, hi[1] - lo[1] + 2 * pad, hi[2] - lo[2] + 2 * pad])
    dims = np.ceil(ext / grid_h).astype(np.int32) + 1
    meta = dict(meta, quad_size=b)
    return Scene(
        boxes=np.array(boxes, np.float32),
        box_rgb=np.array(bld.rgb, np.uint32),
        verts=verts, tris=tris, tri_rgb=cols,
        supports=np.array(bld.supports, np.float32).reshape(-1, 5),
        grid_origin=origin, grid_h=float(np.float32(grid_h)), grid_dims=dims,
        spawn=np.array(spawn, np.float32), meta=meta,
    )


_WALL = 0xD8D2C4
_FLOOR = 0x9A7B56
_CEIL = 0xF0F0EC
_FURN = [0x7A4E2D, 0x5C6E7F, 0x8C8C6E, 0x9E3B33, 0x3F6B4A, 0xB59A6A, 0x44475A]


def _shell(bld, x1, z1, height=2.7, t=0.1):
    """Floor slab, ceiling slab and the four outer walls of [0,x1]x[0,z1]."""
    bld.box((-t, -t, -t), (x1 + t, 0.0, z1 + t), bld.jitter(_FLOOR), skip_faces=(2,))
    bld.box((-t, height, -t), (x1 + t, height + t, z1 + t), _CEIL, skip_faces=(3,))
    w = bld.jitter(_WALL, 6)
    bld.box((-t, 0, -t), (0, height, z1 + t), w)
    bld.box((x1, 0, -t), (x1 + t, height, z1 + t), w)
    bld.box((0, 0, -t), (x1, height, 0), w)
    bld.box((0, 0, z1), (x1, height, z1 + t), w)


def _overlaps(r, placed, gap):
    for q in placed:
        if r[0] < q[2] + gap and q[0] < r[2] + gap and r[1] < q[3] + gap and q[1] < r[3] + gap:
            return True
    return False


def _furniture(bld, kind, x0, z0, x1, z1):
    """Adds one piece over the footprint [x0,x1]x[z0,z1]; returns nothing."""
    rng = bld.rng
    col = bld.jitter(_FURN[rng.integers(len(_FURN))])
    if kind == "table":
        top = float(rng.uniform(0.70, 0.78))
        th = 0.04
        bld.box((x0, top - th, z0), (x1, top, z1), col)
        leg = 0.05
        for (lx, lz) in ((x0, z0), (x1 - leg, z0), (x0, z1 - leg), (x1 - leg, z1 - leg)):
            bld.box((lx, 0.0, lz), (lx + leg, top - th, lz + leg), col, skip_faces=(2,))
        bld.supports.append((x0, z0, x1, z1, top))
    elif kind == "cabinet":
        top = float(rng.uniform(0.45, 0.95))
        bld.box((x0, 0.0, z0), (x1, top, z1), col, skip_faces=(2,))
        bld.supports.append((x0, z0, x1, z1, top))
    elif kind == "shelf":
        height = float(rng.uniform(1.2, 1.9))
        t = 0.03
        nb = int(rng.integers(3, 5))
        alongx = (x1 - x0) >= (z1 - z0)
        if alongx:
            bld.box((x0, 0.0, z0), (x0 + t, height, z1), col, skip_faces=(2,))
            bld.box((x1 - t, 0.0, z0), (x1, height, z1), col, skip_faces=(2,))
            bld.box((x0 + t, 0.0, z1 - t), (x1 - t, height, z1), col, skip_faces=(2,))
            ix0, ix1, iz0, iz1 = x0 + t, x1 - t, z0, z1 - t
        else:
            bld.box((x0, 0.0, z0), (x1, height, z0 + t), col, skip_faces=(2,))
            bld.box((x0, 0.0, z1 - t), (x1, height, z1), col, skip_faces=(2,))
            bld.box((x1 - t, 0.0, z0 + t), (x1, height, z1 - t), col, skip_faces=(2,))
            ix0, ix1, iz0, iz1 = x0, x1 - t, z0 + t, z1 - t
        for k in range(nb):
            y = 0.08 + k * (height - 0.08) / nb
            bld.box((ix0, y, iz0), (ix1, y + t, iz1), col)
            bld.supports.append((ix0, iz0, ix1, iz1, y + t))
        bld.box((ix0, height - t, iz0), (ix1, height, iz1), col)
        bld.supports.append((ix0, iz0, ix1, iz1, height))
    elif kind == "sofa":
        seat = float(rng.uniform(0.40, 0.48))
        bld.box((x0, 0.0, z0), (x1, seat, z1), col, skip_faces=(2,))
        bld.supports.append((x0, z0, x1, z1, seat))
    else:  # bed / block
        top = float(rng.uniform(0.35, 0.60))
        bld.box((x0, 0.0, z0), (x1, top, z1), col, skip_faces=(2,))
        bld.supports.append((x0, z0, x1, z1, top))


_SIZES = {
    "table": ((0.8, 1.6), (0.6, 1.0)),
    "cabinet": ((0.5, 1.2), (0.4, 0.6)),
    "shelf": ((0.7, 1.2), (0.35, 0.45)),
    "sofa": ((1.4, 2.2), (0.8, 1.0)),
    "bed": ((1.4, 2.0), (1.9, 2.1)),
}


def _furnish(bld, rx0, rz0, rx1, rz1, n_pieces, keepout):
    rng = bld.rng
    placed = list(keepout)
    kinds = ["table", "cabinet", "shelf", "sofa", "bed"]
    probs = [0.35, 0.25, 0.2, 0.1, 0.1]
    for _ in range(n_pieces):
        for _try in range(40):
            kind = kinds[rng.choice(len(kinds), p=probs)]
            (wa, wb), (da, db) = _SIZES[kind]
            w, d = float(rng.uniform(wa, wb)), float(rng.uniform(da, db))
            if rng.random() < 0.5:
                w, d = d, w
            m = 0.05
            if rx1 - rx0 - 2 * m < w or rz1 - rz0 - 2 * m < d:
                continue
            x0 = float(rng.uniform(rx0 + m, rx1 - m - w))
            z0 = float(rng.uniform(rz0 + m, rz1 - m - d))
            r = (x0, z0, x0 + w, z0 + d)
            if _overlaps(r, placed, 0.6):
                continue
            placed.append(r)
            _furniture(bld, kind, *r)
            break


def room_scene(seed: int, tri_target: int = 2000, n_furniture: int = 12,
               size: float = 6.0, grid_h: float = 0.05) -> Scene:
    """One axis-aligned room with box furniture pieces on the floor."""
    rng = np.random.default_rng(seed)
    bld = _Builder(rng)
    height = 2.7
    _shell(bld, size, size, height)
    placed = []
    n = 0
    while n < n_furniture:
        w, d = float(rng.uniform(0.4, 1.4)), float(rng.uniform(0.4, 1.0))
        hgt = float(rng.uniform(0.4, 1.1))
        x0, z0 = float(rng.uniform(0.05, size - 0.05 - w)), float(rng.uniform(0.05, size - 0.05 - d))
        r = (x0, z0, x0 + w, z0 + d)
        if _overlaps(r, placed, 0.5):
            continue
        placed.append(r)
        bld.box((x0, 0.0, z0), (x0 + w, hgt, z0 + d), bld.jitter(_FURN[n % len(_FURN)]),
                skip_faces=(2,))
        bld.supports.append((x0, z0, x0 + w, z0 + d, hgt))
        n += 1
    return _finish(bld, tri_target, (-0.1, -0.1, -0.1), (size + 0.1, height + 0.1, size + 0.1),
                   grid_h, (0.3, 0.3, size - 0.3, size - 0.3), dict(kind="room", seed=seed))


def apartment_scene(seed: int, tri_target: int, grid_h: float = 0.02) -> Scene:
    """An apartment of 3-6 rooms (3-5 m each, 2.7 m ceiling, 0.1 m walls,
    1 m doors) laid out on a rows x cols grid, furnished room by room."""
    rng = np.random.default_rng(seed)
    bld = _Builder(rng)
    height, t = 2.7, 0.1
    n_rooms = int(rng.integers(3, 7))
    rows = 1 if n_rooms == 3 else 2
    cols = {3: 3, 4: 2, 5: 3, 6: 3}[n_rooms]
    widths = rng.uniform(3.0, 5.0, cols)
    depths = rng.uniform(3.0, 5.0, rows)
    xs = np.concatenate([[0.0], np.cumsum(widths)])
    zs = np.concatenate([[0.0], np.cumsum(depths)])
    X, Z = float(xs[-1]), float(zs[-1])
    _shell(bld, X, Z, height, t)
    merged = (n_rooms == 5)   # the last two cells of the second row form one room
    wall = bld.jitter(_WALL, 6)
    door_w, door_h = 1.0, 2.1
    doors = []

    def wall_with_door(axis, pos, a0, a1):
        # interior wall at x = pos (axis 'x') or z = pos spanning [a0, a1]
        c = float(rng.uniform(a0 + 0.3 + door_w / 2, a1 - 0.3 - door_w / 2))
        d0, d1 = c - door_w / 2, c + door_w / 2
        if axis == "x":
            bld.box((pos - t / 2, 0, a0), (pos + t / 2, height, d0), wall)
            bld.box((pos - t / 2, 0, d1), (pos + t / 2, height, a1), wall)
            bld.box((pos - t / 2, door_h, d0), (pos + t / 2, height, d1), wall)
            doors.append((pos - 0.8, d0 - 0.1, pos + 0.8, d1 + 0.1))
        else:
            bld.box((a0, 0, pos - t / 2), (d0, height, pos + t / 2), wall)
            bld.box((d1, 0, pos - t / 2), (a1, height, pos + t / 2), wall)
            bld.box((d0, door_h, pos - t / 2), (d1, height, pos + t / 2), wall)
            doors.append((d0 - 0.1, pos - 0.8, d1 + 0.1, pos + 0.8))

    for r in range(rows):
        for c in range(1, cols):
            if merged and r == 1 and c == cols - 1:
                continue
            wall_with_door("x", float(xs[c]), float(zs[r]), float(zs[r + 1]))
    for r in range(1, rows):
        for c in range(cols):
            wall_with_door("z", float(zs[r]), float(xs[c]), float(xs[c + 1]))

    cells = [(r, c) for r in range(rows) for c in range(cols)]
    if merged:
        cells = [rc for rc in cells if rc != (1, cols - 1)]
    for (r, c) in cells:
        x0, x1 = float(xs[c]) + t / 2, float(xs[c + 1]) - t / 2
        if merged and r == 1 and c == cols - 2:
            x1 = float(xs[cols]) - t / 2
        z0, z1 = float(zs[r]) + t / 2, float(zs[r + 1]) - t / 2
        _furnish(bld, x0, z0, x1, z1, int(rng.integers(3, 7)), doors)
    return _finish(bld, tri_target, (-t, -t, -t), (X + t, height + t, Z + t), grid_h,
                   (0.3, 0.3, X - 0.3, Z - 0.3),
                   dict(kind="apartment", seed=seed, rooms=n_rooms))


# --------------------------------------------------------------------------
# Workloads.  Each names its sizes; the parity tests and the bench build the
# same objects from these recipes.
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    n_envs: int
    n_scenes: int
    scene_kind: str          # "room" | "apartment"
    tri_range: tuple         # (min, max)
    tri_dist: str            # "fixed" | "uniform" | "loguniform"
    grid_h: float
    n_objects: int
    obj_radius: tuple
    img: int
    depth_fp16: bool
    rgb: bool
    steps: int
    action_dist: str         # "uniform" | "gauss0.5"
    reset_every: int         # episode length (0 = never)
    reset_prob: float        # per-env Bernoulli reset probability per step
    scene_seed: int
    reset_seed: int = 1
    action_seed: int = 0
    sdf: str = "grid"        # static test: "grid" | "neural" (neural SDF, grid below margin)
                             # | "column" (the paper's column grid)
    sdf_margin: float = 0.02
    nsdf_samples: int = 10_000_000
    nsdf_steps: int = 2000   # Adam steps per scene, batch 65,536
    nsdf_seed: int = 7
    objects: str = "spheres"  # "spheres" | "boxes" (upright oriented boxes, carried as
                              # eight spheres; half extents in obj_radius per axis)


WORKLOADS = {
    "room16": Workload("room16", 16, 1, "room", (2000, 2000), "fixed", 0.05, 10, (0.03, 0.06),
                       64, False, True, 20, "uniform", 0, 0.0, 1000),
    "apartments4096": Workload("apartments4096", 4096, 16, "apartment", (20000, 60000), "uniform",
                               0.02, 40, (0.03, 0.06), 128, False, True, 500, "gauss0.5", 200,
                               0.0, 1000),
    "uneven8192": Workload("uneven8192", 8192, 64, "apartment", (5000, 150000), "loguniform",
                           0.02, 40, (0.03, 0.06), 128, True, False, 500, "gauss0.5", 0, 0.005,
                           2000),
    "apartments4096_nsdf": Workload("apartments4096_nsdf", 4096, 16, "apartment", (20000, 60000),
                                    "uniform", 0.02, 40, (0.03, 0.06), 128, False, True, 500,
                                    "gauss0.5", 200, 0.0, 1000, sdf="neural"),
    "apartments4096_obj200": Workload("apartments4096_obj200", 4096, 16, "apartment",
                                      (20000, 60000), "uniform", 0.02, 200, (0.03, 0.06), 128,
                                      False, True, 500, "gauss0.5", 200, 0.0, 1000),
    "apartments4096_boxes": Workload("apartments4096_boxes", 4096, 16, "apartment",
                                     (20000, 60000), "uniform", 0.02, 40, (0.03, 0.06), 128,
                                     False, True, 500, "gauss0.5", 200, 0.0, 1000,
                                     objects="boxes"),
    "apartments4096_column": Workload("apartments4096_column", 4096, 16, "apartment",
                                      (20000, 60000), "uniform", 0.02, 40, (0.03, 0.06), 128,
                                      False, True, 500, "gauss0.5", 200, 0.0, 1000, sdf="column"),
    "uneven16384_nsdf": Workload("uneven16384_nsdf", 16384, 64, "apartment", (5000, 150000),
                                 "loguniform", 0.02, 40, (0.03, 0.06), 128, True, True, 1000,
                                 "gauss0.5", 0, 0.005, 2000, sdf="neural"),
}


def scene_tri_targets(w: Workload) -> list[int]:
    rng = np.random.default_rng(w.scene_seed)
    lo, hi = w.tri_range
    if w.tri_dist == "fixed":
        return [lo] * w.n_scenes
    if w.tri_dist == "uniform":
        return [int(x) for x in rng.uniform(lo, hi, w.n_scenes)]
    return [int(x) for x in np.exp(rng.uniform(math.log(lo), math.log(hi), w.n_scenes))]


def make_scenes(w: Workload, only=None) -> list[Scene]:
    """The workload's scenes in index order, or only the global indices in
    `only` (in that order): each scene depends on its own seed alone."""
    targets = scene_tri_targets(w)
    out = []
    for s in (range(w.n_scenes) if only is None else only):
        if w.scene_kind == "room":
            out.append(room_scene(w.scene_seed + s, targets[s], grid_h=w.grid_h))
        else:
            out.append(apartment_scene(w.scene_seed + s, targets[s], grid_h=w.grid_h))
    return out


def make_actions(n_steps: int, n_envs: int, dist: str, seed: int = 0) -> np.ndarray:
    """Synthetic actions [T][N][11] f32 in [-1, 1] (App. A ranges)."""
    rng = np.random.default_rng(seed)
    if dist == "uniform":
        a = rng.uniform(-1.0, 1.0, (n_steps, n_envs, N_ACTIONS))
    else:
        a = np.clip(rng.normal(0.0, 0.5, (n_steps, n_envs, N_ACTIONS)), -1.0, 1.0)
    return a.astype(np.float32)


def fourier_matrix(seed: int = 7, n_freq: int = 32, sigma: float = 0.25) -> np.ndarray:
    """Fourier feature frequencies B [n_freq][3] ~ N(0, sigma^2), in cycles per
    metre, for the neural SDF's features.  sigma = 0.25 / m: with 2 / m the
    ReLU network stays at the constant predictor's loss; 0.25, 0.5 and 1 / m
    reach 1.3, 1.7 and 3.3 cm mean error in 1,500 Adam steps (batch 8,192)."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, sigma, (n_freq, 3)).astype(np.float32)


def nsdf_init(seed: int = 7) -> np.ndarray:
    """Initial neural-SDF parameters (He-normal weights, zero biases) in the
    C ABI's flat layout: W1 [128][64], b1, W2..W4 [128][128] with biases,
    W5 [128], b5."""
    rng = np.random.default_rng(seed + 1)
    parts = []
    for fan_in, fan_out in [(64, 128), (128, 128), (128, 128), (128, 128)]:
        parts.append(rng.normal(0.0, math.sqrt(2.0 / fan_in), fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    parts.append(rng.normal(0.0, math.sqrt(1.0 / 128), 128))
    parts.append(np.zeros(1))
    return np.concatenate(parts).astype(np.float32)


def env_scene_map(n_envs: int, n_scenes: int) -> np.ndarray:
    """Contiguous blocks: env i uses scene floor(i * S / N)."""
    return (np.arange(n_envs, dtype=np.int64) * n_scenes // n_envs).astype(np.int32)
