"""ctypes binding of the FP64 CPU oracle (oracle/gx_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the bench's CPU
baseline leg use it to check and time the CUDA path.  It shares no code with
the CUDA path and never imports it; both consume the same seeded inputs from
``paper_2306_07552_b300.inputs``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libgx_oracle.so")
MAX_OBJ = 256
BAND = 1e-4


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "gx_oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "gx_oracle.h"))):
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-Wall", "-fPIC", "-shared", "-o", _SO,
                               src, "-lm"])
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


f32p = C.POINTER(C.c_float)
f64p = C.POINTER(C.c_double)
i32p = C.POINTER(C.c_int32)
u32p = C.POINTER(C.c_uint32)
u8p = C.POINTER(C.c_uint8)


class Robot_c(C.Structure):
    _fields_ = [("link_offset", f32p), ("link_axis", i32p), ("q_min", f32p), ("q_max", f32p),
                ("q_rest", f32p), ("dq_max", C.c_float), ("base_step", C.c_float),
                ("base_turn", C.c_float), ("n_spheres", C.c_int32), ("sphere_link", i32p),
                ("sphere_pos", f32p), ("sphere_radius", f32p), ("cam_pos", f32p),
                ("cam_pitch", C.c_float), ("cam_near", C.c_float), ("grasp_radius", C.c_float),
                ("rest_clearance", C.c_float)]


class Scene_c(C.Structure):
    _fields_ = [("n_boxes", C.c_int32), ("boxes", f32p), ("n_verts", C.c_int32), ("verts", f32p),
                ("n_tris", C.c_int32), ("tris", i32p), ("tri_rgb", u32p),
                ("n_supports", C.c_int32), ("supports", f32p), ("grid_origin", C.c_float * 3),
                ("grid_h", C.c_float), ("grid_dims", C.c_int32 * 3), ("spawn", C.c_float * 4)]


class ObjMesh_c(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("verts", f32p), ("n_tris", C.c_int32), ("tris", i32p),
                ("obj_rgb", u32p), ("robot_rgb", u32p)]


class State_c(C.Structure):
    _fields_ = [("base", C.c_double * 3), ("q", C.c_double * 7), ("held", C.c_int32),
                ("c_off", C.c_double * 3), ("p_pre", C.c_double * 3), ("n_obj", C.c_int32),
                ("obj", (C.c_double * 4) * MAX_OBJ), ("step_count", C.c_int32),
                ("episode", C.c_int32), ("goal", C.c_double * 3), ("obj_start", C.c_double * 3),
                ("prev_a", C.c_double * 7), ("prev_d", C.c_double), ("prev_e", C.c_double),
                ("boxes", C.c_int32), ("box", (C.c_double * 4) * MAX_OBJ),
                ("r_off", C.c_double * 9)]


class StepOut_c(C.Structure):
    _fields_ = [("contact_mask", C.c_uint32), ("flags", C.c_uint8), ("event", C.c_uint8),
                ("reverted", C.c_uint8), ("pad", C.c_uint8), ("near_band", C.c_int32),
                ("ee", C.c_double * 3), ("cam_R", C.c_double * 9), ("cam_t", C.c_double * 3),
                ("reward", C.c_double), ("task_obs", C.c_double * 12), ("success", C.c_uint8),
                ("pad2", C.c_uint8 * 7)]


class ResetOut_c(C.Structure):
    _fields_ = [("near_band", C.c_int32), ("failed", C.c_int32)]


class RenderStats_c(C.Structure):
    _fields_ = [("tris_setup", C.c_int64), ("frags_covered", C.c_int64),
                ("ambiguous", C.c_int64), ("overflow", C.c_int64)]


class StepOpts_c(C.Structure):
    _fields_ = [("dhat", f64p), ("margin", C.c_double), ("band", C.c_double),
                ("slide", C.c_int32), ("place_jitter", C.c_int32), ("seed", C.c_uint64),
                ("env", C.c_int32), ("column", C.c_int32)]


def _declare(L):
    P = C.POINTER
    L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
    L.orc_box_sdf.argtypes = [f64p, f32p]
    L.orc_box_sdf.restype = C.c_double
    L.orc_grid_node.argtypes = [P(Scene_c), C.c_int, C.c_int, C.c_int]
    L.orc_grid_node.restype = C.c_double
    L.orc_grid_query.argtypes = [P(Scene_c), f64p, f64p, f64p]
    L.orc_grid_query.restype = C.c_int
    L.orc_fk.argtypes = [P(Robot_c), f64p, f64p, f64p, f64p, f64p]
    L.orc_sphere_centres.argtypes = [P(Robot_c), f64p, f64p, f64p]
    L.orc_step.argtypes = [P(Robot_c), P(Scene_c), P(State_c), f32p, P(StepOut_c)]
    L.orc_step_ex.argtypes = [P(Robot_c), P(Scene_c), P(State_c), f32p, P(StepOpts_c), P(StepOut_c)]
    L.orc_grid_gradient.argtypes = [P(Scene_c), f64p, f64p]
    L.orc_column_radius_index.argtypes = [C.c_double]
    L.orc_column_radius_index.restype = C.c_int
    L.orc_column_dims.argtypes = [P(Scene_c), i32p]
    L.orc_column_spans.argtypes = [P(Scene_c), C.c_int, C.c_int, C.c_int, f64p, C.c_int]
    L.orc_column_spans.restype = C.c_int
    L.orc_column_contact.argtypes = [P(Scene_c), f64p, C.c_double, P(C.c_int)]
    L.orc_column_contact.restype = C.c_int
    L.orc_grid_gradient.restype = C.c_int
    L.orc_step_nsdf.argtypes = [P(Robot_c), P(Scene_c), P(State_c), f32p, f64p, C.c_double,
                                C.c_double, P(StepOut_c)]
    L.orc_candidate_spheres.argtypes = [P(Robot_c), P(State_c), f32p, f64p, f64p, i32p]
    L.orc_reset.argtypes = [P(Robot_c), P(Scene_c), P(State_c), C.c_uint64, C.c_int32, C.c_int32,
                            C.c_float, C.c_float, P(ResetOut_c)]
    L.orc_snap.argtypes = [P(Scene_c), f64p, C.c_double, P(C.c_int), P(C.c_int)]
    L.orc_snap.restype = C.c_double
    L.orc_render.argtypes = [P(Robot_c), P(Scene_c), P(ObjMesh_c), P(State_c), C.c_int32,
                             C.c_int32, C.c_double, C.c_double, C.c_double, f64p, u32p, u8p,
                             i32p, P(RenderStats_c)]
    L.orc_render_cos.argtypes = L.orc_render.argtypes + [f64p]
    L.orc_nsdf_sample.argtypes = [P(Scene_c), C.c_uint64, C.c_uint32, C.c_uint32, C.c_double,
                                  f64p, f64p, P(C.c_int)]
    L.orc_nsdf_sample.restype = C.c_int
    L.orc_mlp_set_bf16_operands.argtypes = [C.c_int]
    L.orc_mlp_forward.argtypes = [f64p, C.c_int, P(f64p), P(f64p), i32p, C.c_int, f64p, f64p]
    L.orc_mlp_forward.restype = C.c_double
    L.orc_mlp_loss_grad.argtypes = [f64p, C.c_int, P(f64p), P(f64p), i32p, C.c_int, f64p, f64p,
                                    C.c_int, C.c_double, C.c_double, P(f64p), P(f64p)]
    L.orc_mlp_loss_grad.restype = C.c_double
    L.orc_mlp_rounding_bound.argtypes = [f64p, C.c_int, P(f64p), P(f64p), i32p, C.c_int, f64p,
                                         C.c_double, f64p]
    L.orc_mlp_rounding_bound.restype = C.c_double
    L.orc_box_distance.argtypes = [P(State_c), C.c_int, f64p]
    L.orc_box_distance.restype = C.c_double
    L.orc_box_spheres.argtypes = [f64p, f64p]
    L.orc_box_spheres.restype = C.c_double
    L.orc_boxes_overlap.argtypes = [f64p, f64p, f64p, f64p, P(C.c_int)]
    L.orc_boxes_overlap.restype = C.c_int


def _p(a, t):
    return a.ctypes.data_as(t)


class Oracle:
    """FP64 oracle bound to one robot, one scene and the instanced object mesh
    (the icosahedron for sphere objects, the unit cube for box objects)."""

    # rasteriser ambiguity band (1/64 px), relative depth tolerance and the
    # smallest |cos| of a hit that is not flagged as grazing
    EPS_PX = 1.0 / 64.0
    TOL_REL = 1e-5
    COS_MIN = 0.05

    def __init__(self, robot, scene, obj_mesh=None, obj_rgb=None, robot_rgb=None):
        self._keep = []
        k = self._keep.append
        r = robot
        arrs = dict(link_offset=np.ascontiguousarray(r.link_offset, np.float32),
                    link_axis=np.ascontiguousarray(r.link_axis, np.int32),
                    q_min=np.ascontiguousarray(r.q_min, np.float32),
                    q_max=np.ascontiguousarray(r.q_max, np.float32),
                    q_rest=np.ascontiguousarray(r.q_rest, np.float32),
                    sphere_link=np.ascontiguousarray(r.sphere_link, np.int32),
                    sphere_pos=np.ascontiguousarray(r.sphere_pos, np.float32),
                    sphere_radius=np.ascontiguousarray(r.sphere_radius, np.float32),
                    cam_pos=np.ascontiguousarray(r.cam_pos, np.float32))
        for v in arrs.values():
            k(v)
        self.robot = Robot_c(
            _p(arrs["link_offset"], f32p), _p(arrs["link_axis"], i32p), _p(arrs["q_min"], f32p),
            _p(arrs["q_max"], f32p), _p(arrs["q_rest"], f32p), r.dq_max, r.base_step,
            r.base_turn, len(r.sphere_radius), _p(arrs["sphere_link"], i32p),
            _p(arrs["sphere_pos"], f32p), _p(arrs["sphere_radius"], f32p),
            _p(arrs["cam_pos"], f32p), r.cam_pitch, r.cam_near, r.grasp_radius, r.rest_clearance)
        s = scene
        sa = dict(boxes=np.ascontiguousarray(s.boxes, np.float32),
                  verts=np.ascontiguousarray(s.verts, np.float32),
                  tris=np.ascontiguousarray(s.tris, np.int32),
                  tri_rgb=np.ascontiguousarray(s.tri_rgb, np.uint32),
                  supports=np.ascontiguousarray(s.supports, np.float32))
        for v in sa.values():
            k(v)
        self.scene = Scene_c(len(sa["boxes"]), _p(sa["boxes"], f32p), len(sa["verts"]),
                             _p(sa["verts"], f32p), len(sa["tris"]), _p(sa["tris"], i32p),
                             _p(sa["tri_rgb"], u32p), len(sa["supports"]),
                             _p(sa["supports"], f32p),
                             (C.c_float * 3)(*[float(x) for x in s.grid_origin]), s.grid_h,
                             (C.c_int32 * 3)(*[int(x) for x in s.grid_dims]),
                             (C.c_float * 4)(*[float(x) for x in s.spawn]))
        if obj_mesh is not None:
            mv = np.ascontiguousarray(obj_mesh[0], np.float32)
            mt = np.ascontiguousarray(obj_mesh[1], np.int32)
            rgb = np.zeros(MAX_OBJ, np.uint32)
            if obj_rgb is not None:
                rgb[:len(obj_rgb)] = obj_rgb
            for v in (mv, mt, rgb):
                k(v)
            rr = None
            if robot_rgb is not None:
                rr = np.zeros(32, np.uint32)
                rr[:len(robot_rgb)] = robot_rgb
                k(rr)
            self.objmesh = ObjMesh_c(len(mv), _p(mv, f32p), len(mt), _p(mt, i32p), _p(rgb, u32p),
                                     _p(rr, u32p) if rr is not None else None)
        else:
            self.objmesh = None
        self.L = lib()

    # ---------------------------------------------------------------- state
    @staticmethod
    def make_state(base, q, held=-1, c_off=(0, 0, 0), p_pre=(0, 0, 0), objs=None,
                   step_count=0, episode=0, task=None, boxes=None, r_off=None):
        """task: [16] goal xyz, target start xyz, previous joint actions [7],
        previous tip-target and target-goal distances (the GPU's layout).
        boxes: [n][4] half extents and yaw per object (the oriented-box object
        model; None: spheres); r_off: [9] the held box's rotation in the
        tool frame, row-major."""
        st = State_c()
        st.base[:] = [float(x) for x in base]
        st.q[:] = [float(x) for x in q]
        st.held = int(held)
        st.c_off[:] = [float(x) for x in c_off]
        st.p_pre[:] = [float(x) for x in p_pre]
        objs = np.zeros((0, 4)) if objs is None else np.asarray(objs, np.float64)
        st.n_obj = len(objs)
        for j in range(len(objs)):
            st.obj[j][:] = [float(x) for x in objs[j]]
        st.step_count = int(step_count)
        st.episode = int(episode)
        if task is not None:
            t = [float(x) for x in task]
            st.goal[:] = t[0:3]
            st.obj_start[:] = t[3:6]
            st.prev_a[:] = t[6:13]
            st.prev_d, st.prev_e = t[13], t[14]
        if boxes is not None:
            st.boxes = 1
            bx = np.asarray(boxes, np.float64)
            for j in range(len(bx)):
                st.box[j][:] = [float(x) for x in bx[j]]
            if r_off is not None:
                st.r_off[:] = [float(x) for x in np.ravel(r_off)]
        return st

    @staticmethod
    def state_boxes(st):
        return np.array([[st.box[j][a] for a in range(4)] for j in range(st.n_obj)]).reshape(-1, 4)

    @staticmethod
    def state_objs(st):
        return np.array([[st.obj[j][a] for a in range(4)] for j in range(st.n_obj)]).reshape(-1, 4)

    # ------------------------------------------------------------ functions
    def step(self, st, action):
        a = np.ascontiguousarray(action, np.float32)
        out = StepOut_c()
        self.L.orc_step(C.byref(self.robot), C.byref(self.scene), C.byref(st), _p(a, f32p),
                        C.byref(out))
        return out

    def step_ex(self, st, action, slide=False, place_jitter=False, seed=0, env=0, dhat=None,
                margin=0.0, band=0.0, column=False):
        """One step with the paper's heuristics switched on as asked."""
        a = np.ascontiguousarray(action, np.float32)
        o = StepOpts_c()
        d = None
        if dhat is not None:
            d = np.ascontiguousarray(dhat, np.float64)
            o.dhat = _p(d, f64p)
        o.margin, o.band = float(margin), float(band)
        o.slide, o.place_jitter = int(slide), int(place_jitter)
        o.seed, o.env = int(seed), int(env)
        o.column = int(column)
        out = StepOut_c()
        self.L.orc_step_ex(C.byref(self.robot), C.byref(self.scene), C.byref(st), _p(a, f32p),
                           C.byref(o), C.byref(out))
        return out

    def column_spans(self, ri, i, k):
        sp = np.zeros((64, 2))
        n = self.L.orc_column_spans(C.byref(self.scene), int(ri), int(i), int(k), _p(sp, f64p), 64)
        return sp[:n]

    def column_dims(self):
        d = np.zeros(2, np.int32)
        self.L.orc_column_dims(C.byref(self.scene), _p(d, i32p))
        return tuple(int(x) for x in d)

    def column_contact(self, c, r):
        cc = np.ascontiguousarray(c, np.float64)
        nb = C.c_int()
        hit = self.L.orc_column_contact(C.byref(self.scene), _p(cc, f64p), float(r), C.byref(nb))
        return bool(hit), nb.value

    def grid_gradient(self, c):
        cc = np.ascontiguousarray(c, np.float64)
        g = np.zeros(3)
        inside = self.L.orc_grid_gradient(C.byref(self.scene), _p(cc, f64p), _p(g, f64p))
        return bool(inside), g

    def candidate_spheres(self, st, action):
        """Centres [31][3], radii [31] and the active mask of the proposed pose."""
        a = np.ascontiguousarray(action, np.float32)
        c = np.zeros((31, 3))
        r = np.zeros(31)
        act = np.zeros(31, np.int32)
        self.L.orc_candidate_spheres(C.byref(self.robot), C.byref(st), _p(a, f32p), _p(c, f64p),
                                     _p(r, f64p), _p(act, i32p))
        return c, r, act.astype(bool)

    def step_nsdf(self, st, action, dhat, margin, band):
        """One step with the neural-SDF static test (dhat [31] predictions)."""
        a = np.ascontiguousarray(action, np.float32)
        d = np.ascontiguousarray(dhat, np.float64)
        out = StepOut_c()
        self.L.orc_step_nsdf(C.byref(self.robot), C.byref(self.scene), C.byref(st), _p(a, f32p),
                             _p(d, f64p), float(margin), float(band), C.byref(out))
        return out

    def reset(self, st, seed, env, n_obj, rho_min, rho_max):
        out = ResetOut_c()
        self.L.orc_reset(C.byref(self.robot), C.byref(self.scene), C.byref(st), int(seed),
                         int(env), int(n_obj), float(rho_min), float(rho_max), C.byref(out))
        return out

    def fk(self, base, q):
        b = np.ascontiguousarray(base, np.float64)
        qq = np.ascontiguousarray(q, np.float64)
        links = np.zeros((8, 12))
        ee = np.zeros(12)
        cam = np.zeros(12)
        self.L.orc_fk(C.byref(self.robot), _p(b, f64p), _p(qq, f64p), _p(links, f64p),
                      _p(ee, f64p), _p(cam, f64p))
        return links, ee, cam

    def sphere_centres(self, base, q):
        b = np.ascontiguousarray(base, np.float64)
        qq = np.ascontiguousarray(q, np.float64)
        out = np.zeros((self.robot.n_spheres, 3))
        self.L.orc_sphere_centres(C.byref(self.robot), _p(b, f64p), _p(qq, f64p),
                                  _p(out, f64p))
        return out

    def grid_node(self, i, j, k):
        return self.L.orc_grid_node(C.byref(self.scene), int(i), int(j), int(k))

    def grid_query(self, c):
        cc = np.ascontiguousarray(c, np.float64)
        d = C.c_double()
        e = C.c_double()
        inside = self.L.orc_grid_query(C.byref(self.scene), _p(cc, f64p), C.byref(d), C.byref(e))
        return bool(inside), d.value, e.value

    def snap(self, p, target):
        pp = np.ascontiguousarray(p, np.float64)
        ok = C.c_int()
        nb = C.c_int()
        y = self.L.orc_snap(C.byref(self.scene), _p(pp, f64p), float(target), C.byref(ok),
                            C.byref(nb))
        return y, bool(ok.value), nb.value

    def nsdf_samples(self, seed, scene, idx, band=0.1):
        """Training samples idx (neural SDF): points [n][3], labels, draw used, near-band draws."""
        idx = np.atleast_1d(np.asarray(idx, np.int64))
        P = np.zeros((len(idx), 3))
        d = np.zeros(len(idx))
        t = np.zeros(len(idx), np.int32)
        nb = np.zeros(len(idx), np.int32)
        p3 = np.zeros(3)
        dd = C.c_double()
        nbb = C.c_int()
        for k, i in enumerate(idx):
            t[k] = self.L.orc_nsdf_sample(C.byref(self.scene), int(seed), int(scene), int(i),
                                          float(band), _p(p3, f64p), C.byref(dd), C.byref(nbb))
            P[k] = p3
            d[k] = dd.value
            nb[k] = nbb.value
        return P, d, t, nb

    def render(self, st, W, H, eps_px=None, tol_rel=None, cos_min=None, cos_out=None):
        n = W * H
        depth = np.zeros(n)
        rgb = np.zeros(n, np.uint32)
        amb = np.zeros(n, np.uint8)
        win = np.zeros(n, np.int32)
        stats = RenderStats_c()
        cs = np.ones(n)
        self.L.orc_render_cos(C.byref(self.robot), C.byref(self.scene), C.byref(self.objmesh),
                              C.byref(st), W, H, self.EPS_PX if eps_px is None else eps_px,
                              self.TOL_REL if tol_rel is None else tol_rel,
                              self.COS_MIN if cos_min is None else cos_min, _p(depth, f64p),
                              _p(rgb, u32p), _p(amb, u8p), _p(win, i32p), C.byref(stats),
                              _p(cs, f64p))
        if cos_out is not None:
            cos_out[...] = cs.reshape(H, W)
        return (depth.reshape(H, W), rgb.reshape(H, W), amb.reshape(H, W).astype(bool),
                win.reshape(H, W), stats)


def box_distance(st, j, c):
    """Exact signed distance from c to resting box j of state st."""
    cc = np.ascontiguousarray(c, np.float64)
    return lib().orc_box_distance(C.byref(st), int(j), _p(cc, f64p))


def box_spheres(h):
    """The eight carried spheres of a box with half extents h: centres in
    its frame [8][3] and their radius."""
    hh = np.ascontiguousarray(h, np.float64)
    out = np.zeros((8, 3))
    s = lib().orc_box_spheres(_p(hh, f64p), _p(out, f64p))
    return out, s


def boxes_overlap(pa, ba, pb, bb):
    """Overlap of two upright boxes (centres p, (hx, hy, hz, yaw)) and the
    near-band count of the decision."""
    a = [np.ascontiguousarray(x, np.float64) for x in (pa, ba, pb, bb)]
    nb = C.c_int(0)
    r = lib().orc_boxes_overlap(*[_p(x, f64p) for x in a], C.byref(nb))
    return bool(r), nb.value


def philox4x32_10(ctr, key):
    L = lib()
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    L.orc_philox4x32_10(_p(c, u32p), _p(k, u32p), _p(o, u32p))
    return o


def box_sdf(p, box):
    L = lib()
    pp = np.ascontiguousarray(p, np.float64)
    b = np.ascontiguousarray(box, np.float32)
    return L.orc_box_sdf(_p(pp, f64p), _p(b, f32p))


class MLP64:
    """FP64 Fourier-feature MLP used to check the neural-SDF kernels.
    bf16_operands=True rounds what the tensor cores consume to BF16."""

    def __init__(self, B, Ws, bs, bf16_operands=False):
        self.bf16 = bool(bf16_operands)
        self.B = np.ascontiguousarray(B, np.float64)
        self.Ws = [np.ascontiguousarray(w, np.float64) for w in Ws]
        self.bs = [np.ascontiguousarray(b, np.float64) for b in bs]
        self.dims = np.array([self.Ws[0].shape[1]] + [w.shape[0] for w in self.Ws], np.int32)
        self.F = self.B.shape[0]
        assert self.dims[0] == 2 * self.F
        self._wp = (f64p * len(self.Ws))(*[_p(w, f64p) for w in self.Ws])
        self._bp = (f64p * len(self.bs))(*[_p(b, f64p) for b in self.bs])

    def forward(self, X):
        X = np.ascontiguousarray(np.atleast_2d(X), np.float64)
        L = lib()
        L.orc_mlp_set_bf16_operands(int(self.bf16))
        out = np.zeros(len(X))
        for i in range(len(X)):
            out[i] = L.orc_mlp_forward(_p(self.B, f64p), self.F, self._wp, self._bp,
                                       _p(self.dims, i32p), len(self.Ws), _p(X[i], f64p), None)
        return out

    def rounding_bound(self, X, feat_err=4e-7, terms=False):
        """Plain FP64 outputs (nothing rounded) and, per point, the first-order
        bound on how far a kernel that rounds features and hidden activations
        to BF16 and sums in FP32 can be from them (orc_mlp_rounding_bound);
        terms=True also returns its [n][4] operand, feature and FP32 parts and
        the operand part's standard deviation for independent roundings."""
        X = np.ascontiguousarray(np.atleast_2d(X), np.float64)
        L = lib()
        out = np.zeros(len(X))
        parts = np.zeros((len(X), 4))
        for i in range(len(X)):
            out[i] = L.orc_mlp_rounding_bound(_p(self.B, f64p), self.F, self._wp, self._bp,
                                              _p(self.dims, i32p), len(self.Ws), _p(X[i], f64p),
                                              float(feat_err), _p(parts[i], f64p))
        bnd = parts[:, :3].sum(axis=1)
        return (out, bnd, parts) if terms else (out, bnd)

    def loss_grad(self, X, y, lo, hi):
        X = np.ascontiguousarray(X, np.float64)
        y = np.ascontiguousarray(y, np.float64)
        gW = [np.zeros_like(w) for w in self.Ws]
        gb = [np.zeros_like(b) for b in self.bs]
        gwp = (f64p * len(gW))(*[_p(w, f64p) for w in gW])
        gbp = (f64p * len(gb))(*[_p(b, f64p) for b in gb])
        lib().orc_mlp_set_bf16_operands(int(self.bf16))
        loss = lib().orc_mlp_loss_grad(_p(self.B, f64p), self.F, self._wp, self._bp,
                                       _p(self.dims, i32p), len(self.Ws), _p(X, f64p),
                                       _p(y, f64p), len(X), lo, hi, gwp, gbp)
        return loss, gW, gb


# ------------------------------------------------------------------ training
# Adam (Kingma and Ba, ICLR 2015, Algorithm 1) and a cosine learning-rate
# decay, in FP64, for checking the neural-SDF optimiser step.

def cosine_lr(lr0, t, T):
    """Learning rate of step t (0-based) of T: lr0 (1 + cos(pi t / T)) / 2."""
    return lr0 * 0.5 * (1.0 + np.cos(np.pi * t / T))


def adam_step(p, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t (1-based): returns new (p, m, v)."""
    g = np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return np.asarray(p, np.float64) - lr * mhat / (np.sqrt(vhat) + eps), m, v
