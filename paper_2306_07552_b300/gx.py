"""Python binding of the gx C ABI (include/gx.h): argument marshalling only.

Every step of the environment update runs in the CUDA kernels of libgx.so;
this module builds the C structs, allocates caller-owned output tensors with
PyTorch (device memory and streams are all PyTorch is used for) and forwards
calls.  There is no CPU fallback: without the library or a CUDA device the
constructors raise.
"""
from __future__ import annotations

import ctypes as C
import hashlib
import json
import os

import numpy as np

from . import inputs as _inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "libgx.so")

GX_OK, GX_EINVAL, GX_ENOMEM, GX_ECUDA, GX_EDEVICE, GX_ESTATE = range(6)
GX_DEV_NONFINITE_ACTION = 0x1
GX_DEV_PLACEMENT_FAILED = 0x2
GX_NOALLOC_WAIT_TIMEOUT = 0x100
GX_NOALLOC_BAD_SCENE = 0x200
MAX_OBJECTS = 256
STATE_ARRAYS = 13
MAX_SPHERES = 31

SYMBOLS = ["gx_scene_set_create", "gx_scene_set_destroy", "gx_create", "gx_destroy", "gx_reset",
           "gx_step", "gx_step_reset", "gx_step_host", "gx_sync", "gx_device_error", "gx_state_bytes",
           "gx_save_state", "gx_load_state", "gx_state_layout", "gx_phase_times",
           "gx_raster_counters", "gx_render_noalloc", "gx_render_noalloc_error",
           "gx_nsdf_set_weights",
           "gx_nsdf_get_weights", "gx_nsdf_query", "gx_nsdf_get_master", "gx_nsdf_samples",
           "gx_nsdf_grad",
           "gx_nsdf_train", "gx_nsdf_counters", "gx_nsdf_step_predictions", "gx_autotune",
           "gx_column_info", "gx_column_spans", "gx_device_outputs", "gx_last_error",
           "gx_scene_set_create_ex", "gx_scene_bytes", "gx_static_distance",
           "gx_box_store_lists", "gx_set_device_memory_cap", "gx_device_memory_in_use",
           "gx_apply_tune", "gx_nsdf_train_steps", "gx_step_counters"]
NSDF_PARAMS = 57985
STEP_COUNTERS = ["contacts", "grasps", "grasp_misses", "landed", "restored", "near_static",
                 "near_pairs", "slides"]
NSDF_FREQ = 32
RASTER_COUNTERS = ["clusters_tested", "clusters_drawn", "tris_seen", "tris_front", "tris_expand",
                   "expand_pixels", "tris_warp", "warp_blocks", "tris_clipped", "fragments", "wait_polls",
                   "expand_trips", "rounds", "expand_slots", "clusters_occluded"]

f32p = C.POINTER(C.c_float)
i32p = C.POINTER(C.c_int32)
u32p = C.POINTER(C.c_uint32)
u8p = C.POINTER(C.c_uint8)


class GxRobot(C.Structure):
    _fields_ = [("link_offset", (C.c_float * 3) * 8), ("link_axis", C.c_int32 * 7),
                ("q_min", C.c_float * 7), ("q_max", C.c_float * 7), ("q_rest", C.c_float * 7),
                ("dq_max", C.c_float), ("base_step", C.c_float), ("base_turn", C.c_float),
                ("n_spheres", C.c_int32), ("sphere_link", C.c_int32 * MAX_SPHERES),
                ("sphere_pos", (C.c_float * 3) * MAX_SPHERES),
                ("sphere_radius", C.c_float * MAX_SPHERES), ("cam_pos", C.c_float * 3),
                ("cam_pitch", C.c_float), ("cam_near", C.c_float), ("grasp_radius", C.c_float),
                ("rest_clearance", C.c_float)]


class GxSceneDesc(C.Structure):
    _fields_ = [("n_boxes", C.c_int32), ("boxes", f32p), ("n_verts", C.c_int32), ("verts", f32p),
                ("n_tris", C.c_int32), ("tris", i32p), ("tri_rgb", u32p),
                ("n_supports", C.c_int32), ("supports", f32p), ("grid_origin", C.c_float * 3),
                ("grid_h", C.c_float), ("grid_dims", C.c_int32 * 3), ("spawn", C.c_float * 4)]


class GxObjectMesh(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("verts", f32p), ("n_tris", C.c_int32), ("tris", i32p),
                ("obj_rgb", C.c_uint32 * MAX_OBJECTS), ("robot_rgb", C.c_uint32 * 32)]


class GxConfig(C.Structure):
    _fields_ = [("n_envs", C.c_int32), ("img_w", C.c_int32), ("img_h", C.c_int32),
                ("depth_fp16", C.c_int32), ("render_rgb", C.c_int32), ("n_objects", C.c_int32),
                ("obj_radius_min", C.c_float), ("obj_radius_max", C.c_float),
                ("seed", C.c_uint64), ("env_scene", i32p),
                ("small_tri_px", C.c_int32), ("use_graph", C.c_int32), ("profile", C.c_int32),
                ("sdf_mode", C.c_int32), ("sdf_margin", C.c_float), ("broadphase", C.c_int32),
                ("render_robot", C.c_int32), ("heuristics", C.c_int32),
                ("raster_order", C.c_int32), ("env_offset", C.c_int32),
                ("object_boxes", C.c_int32), ("raster_warps", C.c_int32),
                ("occlusion_cull", C.c_int32), ("fused_step", C.c_int32),
                ("static_store", C.c_int32)]


class GxSceneOptions(C.Structure):
    _fields_ = [("dense_grid", C.c_int32), ("column_grid", C.c_int32)]


OUTPUT_KEYS = ["depth", "rgb", "pose", "obj_pos", "held", "contact_mask", "contact_flags", "event",
               "reward", "task_obs", "success"]


class GxOutputs(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in OUTPUT_KEYS]


class GxTrainParams(C.Structure):
    _fields_ = [("n_samples", C.c_int64), ("batch", C.c_int32), ("steps", C.c_int32),
                ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("clamp_lo", C.c_float), ("clamp_hi", C.c_float),
                ("near_band", C.c_float), ("seed", C.c_uint64)]


class GxTuneResult(C.Structure):
    _fields_ = [("small_tri_px", C.c_int32), ("order_costliest_first", C.c_int32),
                ("raster_ctas", C.c_int32), ("ms_per_step", C.c_float),
                ("raster_warps", C.c_int32), ("occlusion_cull", C.c_int32)]


class GxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"gx status {status}: {msg}")
        self.status = status


_lib = None


def lib():
    """Loads libgx.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(SO_PATH):
            raise RuntimeError(f"{SO_PATH} is missing: run paper_2306_07552_b300.build.build()")
        L = C.CDLL(SO_PATH)
        P = C.POINTER
        vp = C.c_void_p
        L.gx_scene_set_create.argtypes = [P(GxSceneDesc), C.c_int32, P(GxObjectMesh), P(vp)]
        L.gx_scene_set_create_ex.argtypes = [P(GxSceneDesc), C.c_int32, P(GxObjectMesh),
                                             P(GxSceneOptions), P(vp)]
        L.gx_scene_bytes.argtypes = [vp, C.c_int32, C.POINTER(C.c_uint64)]
        L.gx_static_distance.argtypes = [vp, C.c_int32, C.c_int32, vp, C.c_int32, vp, vp]
        L.gx_box_store_lists.argtypes = [P(GxSceneDesc), C.POINTER(C.c_int32), vp, vp,
                                         C.POINTER(C.c_uint64)]
        L.gx_scene_set_destroy.argtypes = [vp]
        L.gx_create.argtypes = [vp, P(GxRobot), P(GxConfig), P(vp)]
        L.gx_destroy.argtypes = [vp]
        L.gx_destroy.restype = None
        L.gx_reset.argtypes = [vp, vp, vp]
        L.gx_step.argtypes = [vp, vp, P(GxOutputs), vp]
        L.gx_step_reset.argtypes = [vp, vp, vp, P(GxOutputs), vp]
        L.gx_step_host.argtypes = [vp, vp, P(GxOutputs), vp]
        L.gx_sync.argtypes = [vp]
        L.gx_device_error.argtypes = [vp]
        L.gx_device_error.restype = C.c_uint32
        L.gx_state_bytes.argtypes = [vp]
        L.gx_state_bytes.restype = C.c_size_t
        L.gx_save_state.argtypes = [vp, vp, C.c_size_t]
        L.gx_load_state.argtypes = [vp, vp, C.c_size_t]
        L.gx_state_layout.argtypes = [vp, P(C.c_size_t)]
        L.gx_phase_times.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
        L.gx_raster_counters.argtypes = [vp, C.POINTER(C.c_int64), C.c_int32]
        L.gx_step_counters.argtypes = [vp, C.POINTER(C.c_int64), C.c_int32]
        L.gx_render_noalloc.argtypes = [vp, C.c_int32, vp, vp, vp, C.c_int32, C.c_int32,
                                        C.c_int32, C.c_float, vp, C.c_int32, vp, vp]
        L.gx_render_noalloc_error.argtypes = [C.POINTER(C.c_uint32)]
        L.gx_nsdf_set_weights.argtypes = [vp, C.c_int32, vp, vp]
        L.gx_nsdf_get_weights.argtypes = [vp, C.c_int32, vp, vp, vp]
        L.gx_nsdf_query.argtypes = [vp, C.c_int32, vp, C.c_int32, vp, vp]
        L.gx_nsdf_get_master.argtypes = [vp, C.c_int32, vp]
        L.gx_nsdf_samples.argtypes = [vp, C.c_int32, C.c_uint64, C.c_int64, C.c_int64, C.c_float,
                                      vp, vp, vp]
        L.gx_nsdf_grad.argtypes = [vp, C.c_int32, vp, vp, C.c_int32, C.c_float, C.c_float, vp, vp,
                                   vp]
        L.gx_nsdf_counters.argtypes = [vp, C.POINTER(C.c_int64)]
        L.gx_nsdf_step_predictions.argtypes = [vp, C.POINTER(C.c_float), C.c_size_t]
        L.gx_device_outputs.argtypes = [vp, P(GxOutputs)]
        L.gx_column_info.argtypes = [vp, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_uint64)]
        L.gx_column_spans.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, vp, C.c_int32]
        L.gx_column_spans.restype = C.c_int32
        L.gx_autotune.argtypes = [vp, vp, P(GxOutputs), C.c_int32, P(GxTuneResult), vp]
        L.gx_apply_tune.argtypes = [vp, P(GxTuneResult)]
        L.gx_nsdf_train.argtypes = [vp, C.c_int32, C.POINTER(GxTrainParams), vp, vp]
        L.gx_nsdf_train_steps.argtypes = [vp, C.c_int32, C.POINTER(GxTrainParams), C.c_int32,
                                          C.c_int32, vp, vp, vp, vp]
        L.gx_set_device_memory_cap.argtypes = [C.c_uint64]
        L.gx_set_device_memory_cap.restype = None
        L.gx_device_memory_in_use.argtypes = []
        L.gx_device_memory_in_use.restype = C.c_uint64
        L.gx_last_error.argtypes = [vp]
        L.gx_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(status, ctx=None):
    if status != GX_OK:
        msg = lib().gx_last_error(ctx).decode(errors="replace")
        raise GxError(status, msg)


def robot_struct(r: _inputs.Robot) -> GxRobot:
    g = GxRobot()
    for k in range(8):
        g.link_offset[k][:] = [float(x) for x in r.link_offset[k]]
    g.link_axis[:] = [int(x) for x in r.link_axis]
    g.q_min[:] = [float(x) for x in r.q_min]
    g.q_max[:] = [float(x) for x in r.q_max]
    g.q_rest[:] = [float(x) for x in r.q_rest]
    g.dq_max, g.base_step, g.base_turn = r.dq_max, r.base_step, r.base_turn
    S = len(r.sphere_radius)
    g.n_spheres = S
    for i in range(S):
        g.sphere_link[i] = int(r.sphere_link[i])
        g.sphere_pos[i][:] = [float(x) for x in r.sphere_pos[i]]
        g.sphere_radius[i] = float(r.sphere_radius[i])
    g.cam_pos[:] = [float(x) for x in r.cam_pos]
    g.cam_pitch, g.cam_near = r.cam_pitch, r.cam_near
    g.grasp_radius, g.rest_clearance = r.grasp_radius, r.rest_clearance
    return g


def scene_desc(s, keep):
    """The C description of one scene (arrays kept alive in `keep`)."""
    arrs = [np.ascontiguousarray(s.boxes, np.float32), np.ascontiguousarray(s.verts, np.float32),
            np.ascontiguousarray(s.tris, np.int32), np.ascontiguousarray(s.tri_rgb, np.uint32),
            np.ascontiguousarray(s.supports, np.float32)]
    keep += arrs
    b, v, t, c, sp = arrs
    d = GxSceneDesc()
    d.n_boxes, d.boxes = len(b), b.ctypes.data_as(f32p)
    d.n_verts, d.verts = len(v), v.ctypes.data_as(f32p)
    d.n_tris, d.tris, d.tri_rgb = len(t), t.ctypes.data_as(i32p), c.ctypes.data_as(u32p)
    d.n_supports, d.supports = len(sp), sp.ctypes.data_as(f32p)
    d.grid_origin[:] = [float(x) for x in s.grid_origin]
    d.grid_h = float(s.grid_h)
    d.grid_dims[:] = [int(x) for x in s.grid_dims]
    d.spawn[:] = [float(x) for x in s.spawn]
    return d


def set_device_memory_cap(nbytes):
    """Caps the device bytes the library may hold (0: no cap)."""
    lib().gx_set_device_memory_cap(int(nbytes))


def device_memory_in_use():
    """Device bytes the library holds now."""
    return int(lib().gx_device_memory_in_use())


def box_store_lists(scene):
    """The box store's candidate lists of one scene, built on the host (no
    device needed): (dims [3], offsets [cells + 1], box ids)."""
    keep = []
    d = scene_desc(scene, keep)
    dims = (C.c_int32 * 3)()
    n = C.c_uint64()
    _check(lib().gx_box_store_lists(C.byref(d), dims, None, None, C.byref(n)))
    cells = dims[0] * dims[1] * dims[2]
    off = np.zeros(cells + 1, np.uint32)
    ids = np.zeros(max(n.value, 1), np.uint16)
    _check(lib().gx_box_store_lists(C.byref(d), dims, off.ctypes.data, ids.ctypes.data,
                                    C.byref(n)))
    return np.array(list(dims)), off, ids[:n.value]


class SceneSet:
    """Device copies of a list of scenes (grid, clusters, supports)."""

    def __init__(self, scenes, obj_mesh=None, obj_rgb=None, robot_rgb=None, dense_grid=True,
                 column_grid=True):
        self._keep = []
        n = len(scenes)
        descs = (GxSceneDesc * n)()
        sig = hashlib.sha1()
        for i, s in enumerate(scenes):
            descs[i] = scene_desc(s, self._keep)
            for a in (s.boxes, s.verts, s.tris, s.grid_dims):
                sig.update(np.ascontiguousarray(a).tobytes())
        self.signature = sig.hexdigest()   # identifies the scenes (tuning cache keys)
        mv, mt = obj_mesh if obj_mesh is not None else _inputs.icosahedron()
        mv = np.ascontiguousarray(mv, np.float32)
        mt = np.ascontiguousarray(mt, np.int32)
        self._keep += [mv, mt]
        m = GxObjectMesh()
        m.n_verts, m.verts = len(mv), mv.ctypes.data_as(f32p)
        m.n_tris, m.tris = len(mt), mt.ctypes.data_as(i32p)
        rgb = _inputs.object_colors(MAX_OBJECTS) if obj_rgb is None else obj_rgb
        m.obj_rgb[:] = [int(x) for x in np.asarray(rgb, np.uint32)[:MAX_OBJECTS]]
        rr = np.zeros(32, np.uint32)
        rc = _inputs.robot_colors(_inputs.fetch_like_robot()) if robot_rgb is None else robot_rgb
        rr[:len(rc)] = np.asarray(rc, np.uint32)[:32]
        m.robot_rgb[:] = [int(x) for x in rr]
        self.n_obj_tris = len(mt)
        self.handle = C.c_void_p()
        opt = GxSceneOptions()
        opt.dense_grid, opt.column_grid = int(dense_grid), int(column_grid)
        _check(lib().gx_scene_set_create_ex(descs, n, C.byref(m), C.byref(opt),
                                            C.byref(self.handle)))
        self._keep = []   # the library copied everything
        self.n = n

    def scene_bytes(self, scene):
        """Device bytes of a scene's structures: dict dense_grid, box_store,
        column_grid, render, nsdf_weights, nsdf_master."""
        b = (C.c_uint64 * 6)()
        _check(lib().gx_scene_bytes(self.handle, scene, b))
        keys = ["dense_grid", "box_store", "column_grid", "render", "nsdf_weights", "nsdf_master"]
        return {k: int(v) for k, v in zip(keys, b)}

    def static_distance(self, scene, pts, store, stream=None):
        """Trilinear static distance at device points pts [n][3] (NaN outside
        the lattice box), node values from store 0 (dense grid) or 1 (box store)."""
        import torch
        out = torch.empty(pts.shape[0], dtype=torch.float32, device=pts.device)
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(lib().gx_static_distance(self.handle, scene, int(store), C.c_void_p(pts.data_ptr()),
                                        int(pts.shape[0]), C.c_void_p(out.data_ptr()),
                                        C.c_void_p(s.cuda_stream)))
        return out

    # -------------------------------------------------------- neural SDF
    def nsdf_set_weights(self, scene, fourier_B, params):
        B = np.ascontiguousarray(fourier_B, np.float32)
        P = np.ascontiguousarray(params, np.float32)
        assert B.shape == (NSDF_FREQ, 3) and P.shape == (NSDF_PARAMS,)
        _check(lib().gx_nsdf_set_weights(self.handle, scene, B.ctypes.data, P.ctypes.data))

    def nsdf_get_weights(self, scene):
        """(B, params, centre) as the kernels use them."""
        B = np.zeros((NSDF_FREQ, 3), np.float32)
        P = np.zeros(NSDF_PARAMS, np.float32)
        c = np.zeros(3, np.float32)
        _check(lib().gx_nsdf_get_weights(self.handle, scene, B.ctypes.data, P.ctypes.data,
                                         c.ctypes.data))
        return B, P, c

    def nsdf_get_master(self, scene):
        """FP32 master parameters (training's copy)."""
        P = np.zeros(NSDF_PARAMS, np.float32)
        _check(lib().gx_nsdf_get_master(self.handle, scene, P.ctypes.data))
        return P

    def nsdf_query(self, scene, pts, out, stream=None):
        """pts: CUDA float32 [n][3]; out: CUDA float32 [n]."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(lib().gx_nsdf_query(self.handle, scene, C.c_void_p(pts.data_ptr()),
                                   int(pts.shape[0]), C.c_void_p(out.data_ptr()),
                                   C.c_void_p(s.cuda_stream)))
        return out

    def column_info(self, scene):
        """(columns along x, columns along z), device bytes of a scene's column grid."""
        d = (C.c_int32 * 2)()
        b = C.c_uint64()
        _check(lib().gx_column_info(self.handle, scene, d, C.byref(b)))
        return (d[0], d[1]), b.value

    def column_spans(self, scene, ri, i, k):
        sp = np.zeros((64, 2), np.float32)
        n = lib().gx_column_spans(self.handle, scene, ri, i, k, sp.ctypes.data, 64)
        if n < 0:
            raise ValueError("bad column")
        return sp[:min(n, 64)]

    def nsdf_samples(self, scene, seed, first, n, near_band=0.1, stream=None):
        """Training samples [first, first + n): (CUDA [n][3] points, CUDA [n] labels)."""
        import torch
        pts = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        d = torch.empty(n, dtype=torch.float32, device="cuda")
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(lib().gx_nsdf_samples(self.handle, scene, int(seed), int(first), int(n),
                                     float(near_band), C.c_void_p(pts.data_ptr()),
                                     C.c_void_p(d.data_ptr()), C.c_void_p(s.cuda_stream)))
        return pts, d

    def nsdf_grad(self, scene, pts, labels, clamp_lo=-0.2, clamp_hi=1.0, stream=None):
        """(gradient CUDA [NSDF_PARAMS], loss) of the mean clamped L1 loss."""
        import torch
        g = torch.empty(NSDF_PARAMS, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(lib().gx_nsdf_grad(self.handle, scene, C.c_void_p(pts.data_ptr()),
                                  C.c_void_p(labels.data_ptr()), int(pts.shape[0]),
                                  float(clamp_lo), float(clamp_hi), C.c_void_p(g.data_ptr()),
                                  C.c_void_p(loss.data_ptr()), C.c_void_p(s.cuda_stream)))
        return g, float(loss.item())

    def nsdf_train(self, scene, n_samples=10_000_000, batch=65536, steps=1000, lr=1e-3,
                   beta1=0.9, beta2=0.999, eps=1e-8, clamp_lo=-0.2, clamp_hi=1.0,
                   near_band=0.1, seed=7, stream=None):
        """Adam training from the current weights; returns the per-step losses."""
        import torch
        tp = GxTrainParams(n_samples, batch, steps, lr, beta1, beta2, eps, clamp_lo, clamp_hi,
                           near_band, seed)
        losses = np.zeros(max(steps, 1), np.float32)
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(lib().gx_nsdf_train(self.handle, scene, C.byref(tp), losses.ctypes.data,
                                   C.c_void_p(s.cuda_stream)))
        return losses[:steps]

    def nsdf_train_steps(self, scene, first_step, n_steps, moments=None, n_samples=10_000_000,
                         batch=65536, steps=1000, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                         clamp_lo=-0.2, clamp_hi=1.0, near_band=0.1, seed=7, stream=None):
        """Steps first_step .. first_step + n_steps - 1 of the run of `steps`
        steps, from the current weights and `moments` ([2][GX_NSDF_PARAMS]
        float32, None: zero); returns (losses, moments after the last step)."""
        import torch
        tp = GxTrainParams(n_samples, batch, steps, lr, beta1, beta2, eps, clamp_lo, clamp_hi,
                           near_band, seed)
        losses = np.zeros(max(n_steps, 1), np.float32)
        m_out = np.zeros((2, NSDF_PARAMS), np.float32)
        m_in = None if moments is None else np.ascontiguousarray(moments, np.float32)
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(lib().gx_nsdf_train_steps(self.handle, scene, C.byref(tp), int(first_step),
                                         int(n_steps),
                                         m_in.ctypes.data if m_in is not None else None,
                                         m_out.ctypes.data, losses.ctypes.data,
                                         C.c_void_p(s.cuda_stream)))
        return losses[:n_steps], m_out

    def close(self):
        if self.handle:
            lib().gx_scene_set_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


STATE_FIELDS = ["base_x", "base_z", "yaw", "q", "held", "c_off", "p_pre", "obj", "step", "episode"]


class Sim:
    """A batch of environments stepped by libgx on the current CUDA device."""

    def __init__(self, scene_set: SceneSet, robot: _inputs.Robot, n_envs: int, img=(128, 128),
                 depth_fp16=False, render_rgb=True, n_objects=40, obj_radius=(0.03, 0.06),
                 seed=1, env_scene=None, small_tri_px=0, use_graph=False,
                 profile=0, sdf_mode=0, sdf_margin=0.02, heuristics=0, render_robot=False,
                 broadphase=False, raster_order=0, env_offset=0, object_boxes=False,
                 fused_step=False, raster_warps=0, occlusion_cull=False, static_store=0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("gx needs a CUDA device; there is no CPU fallback")
        self.torch = torch
        self.scene_set = scene_set
        self.n, self.W, self.H, self.M = n_envs, img[0], img[1], n_objects
        self.depth_fp16, self.render_rgb = bool(depth_fp16), bool(render_rgb)
        cfg = GxConfig()
        cfg.n_envs, cfg.img_w, cfg.img_h = n_envs, img[0], img[1]
        cfg.depth_fp16, cfg.render_rgb, cfg.n_objects = int(depth_fp16), int(render_rgb), n_objects
        cfg.obj_radius_min, cfg.obj_radius_max = obj_radius
        cfg.seed = seed
        es = None
        if env_scene is not None:
            es = np.ascontiguousarray(env_scene, np.int32)
            cfg.env_scene = es.ctypes.data_as(i32p)
        cfg.small_tri_px, cfg.use_graph = small_tri_px, int(use_graph)
        cfg.profile = int(profile)
        cfg.sdf_mode, cfg.sdf_margin = int(sdf_mode), float(sdf_margin)
        cfg.heuristics = int(heuristics)
        cfg.render_robot = int(render_robot)
        cfg.broadphase = int(broadphase)
        cfg.raster_order = int(raster_order)
        cfg.env_offset = int(env_offset)
        cfg.object_boxes = int(object_boxes)
        cfg.fused_step = int(fused_step)
        cfg.raster_warps = int(raster_warps)
        cfg.occlusion_cull = int(occlusion_cull)
        cfg.static_store = int(static_store)
        self.object_boxes = bool(object_boxes)
        self._key_fields = dict(
            n_envs=n_envs, img=list(img), depth_fp16=bool(depth_fp16), render_rgb=bool(render_rgb),
            n_objects=n_objects, obj_radius=[float(x) for x in obj_radius],
            env_scene=(hashlib.sha1(es.tobytes()).hexdigest() if es is not None else None),
            sdf_mode=int(sdf_mode), static_store=int(static_store), heuristics=int(heuristics),
            render_robot=bool(render_robot), broadphase=bool(broadphase),
            object_boxes=bool(object_boxes), fused_step=bool(fused_step),
            raster_warps=int(raster_warps), occlusion_cull=bool(occlusion_cull),
            scenes=scene_set.signature)
        self.robot_c = robot_struct(robot)
        self.handle = C.c_void_p()
        _check(lib().gx_create(scene_set.handle, C.byref(self.robot_c), C.byref(cfg),
                               C.byref(self.handle)))
        dev = torch.device("cuda")
        self.out = dict(
            depth=torch.zeros((n_envs, img[1], img[0]),
                              dtype=torch.float16 if depth_fp16 else torch.float32, device=dev),
            rgb=torch.zeros((n_envs, img[1], img[0], 3), dtype=torch.uint8, device=dev)
            if render_rgb else None,
            pose=torch.zeros((n_envs, 16), dtype=torch.float32, device=dev),
            obj_pos=torch.zeros((n_envs, max(n_objects, 1), 4), dtype=torch.float32, device=dev),
            held=torch.zeros(n_envs, dtype=torch.int32, device=dev),
            contact_mask=torch.zeros(n_envs, dtype=torch.int32, device=dev),
            contact_flags=torch.zeros(n_envs, dtype=torch.uint8, device=dev),
            event=torch.zeros(n_envs, dtype=torch.uint8, device=dev),
            reward=torch.zeros(n_envs, dtype=torch.float32, device=dev),
            task_obs=torch.zeros((n_envs, 12), dtype=torch.float32, device=dev),
            success=torch.zeros(n_envs, dtype=torch.uint8, device=dev),
        )
        self._outs = self._outputs_struct(self.out)

    @staticmethod
    def _outputs_struct(d):
        o = GxOutputs()
        for k in OUTPUT_KEYS:
            v = d.get(k)
            setattr(o, k, None if v is None else (v.data_ptr() if hasattr(v, "data_ptr")
                                                  else v.ctypes.data))
        return o

    def _stream(self, stream):
        s = stream if stream is not None else self.torch.cuda.current_stream()
        return C.c_void_p(s.cuda_stream)

    def reset(self, mask=None, stream=None):
        ptr = None if mask is None else C.c_void_p(mask.data_ptr())
        _check(lib().gx_reset(self.handle, ptr, self._stream(stream)), self.handle)

    def step(self, actions, stream=None):
        """actions: CUDA float32 tensor [n][11]; returns the output tensors."""
        assert actions.is_cuda and actions.dtype == self.torch.float32 and actions.is_contiguous()
        assert tuple(actions.shape) == (self.n, 11)
        _check(lib().gx_step(self.handle, C.c_void_p(actions.data_ptr()), C.byref(self._outs),
                             self._stream(stream)), self.handle)
        return self.out

    def step_reset(self, mask, actions, stream=None):
        """Resets the environments whose mask byte is set (CUDA uint8 [n], or
        None), then steps every environment: one launch with fused_step."""
        assert actions.is_cuda and actions.dtype == self.torch.float32 and actions.is_contiguous()
        assert tuple(actions.shape) == (self.n, 11)
        mp = None if mask is None else C.c_void_p(mask.data_ptr())
        _check(lib().gx_step_reset(self.handle, mp, C.c_void_p(actions.data_ptr()),
                                   C.byref(self._outs), self._stream(stream)), self.handle)
        return self.out

    def host_outputs(self, pinned=True):
        """Host buffers (pinned torch tensors) matching the outputs of step()."""
        t = self.torch
        d = {k: (None if v is None else t.empty(v.shape, dtype=v.dtype, pin_memory=pinned))
             for k, v in self.out.items()}
        return d

    def step_host(self, actions_host, host_out, stream=None):
        """Same step with host actions: copies them in, steps, copies back the
        host buffers given (None entries stay on the device, see
        device_outputs); returns when the host buffers hold the results."""
        o = self._outputs_struct(host_out)
        ptr = actions_host.data_ptr() if hasattr(actions_host, "data_ptr") else actions_host.ctypes.data
        _check(lib().gx_step_host(self.handle, C.c_void_p(ptr), C.byref(o), self._stream(stream)),
               self.handle)
        return host_out

    def device_outputs(self):
        """Device pointers of the outputs step_host left on the device."""
        o = GxOutputs()
        _check(lib().gx_device_outputs(self.handle, C.byref(o)), self.handle)
        return {k: getattr(o, k) for k in OUTPUT_KEYS}

    def phase_times(self):
        """(ms, launches) per kernel since the last call: physics, raster, reset,
        neural-SDF queries."""
        ms = (C.c_double * 4)()
        n = (C.c_int64 * 4)()
        _check(lib().gx_phase_times(self.handle, ms, n), self.handle)
        return list(ms), list(n)

    def raster_counters(self):
        """Rasteriser work counters since the last call (profile bit 1 only)."""
        v = (C.c_int64 * len(RASTER_COUNTERS))()
        _check(lib().gx_raster_counters(self.handle, v, len(RASTER_COUNTERS)), self.handle)
        return dict(zip(RASTER_COUNTERS, list(v)))

    def tune_key(self):
        """The autotuning cache key of this context: its configuration, its
        scene set's scenes and the GPU (name and SM count)."""
        props = self.torch.cuda.get_device_properties(self.torch.cuda.current_device())
        return json.dumps(dict(self._key_fields, gpu=props.name,
                               sms=props.multi_processor_count), sort_keys=True)

    def apply_tune(self, setting):
        """Applies a setting returned by autotune (no timing)."""
        r = GxTuneResult(int(setting["small_tri_px"]), int(setting["order_costliest_first"]),
                         int(setting["raster_ctas"]), float(setting.get("ms_per_step", 0.0)),
                         int(setting["raster_warps"]), int(setting["occlusion_cull"]))
        _check(lib().gx_apply_tune(self.handle, C.byref(r)), self.handle)

    def autotune(self, actions, steps=5, stream=None, cache=None):
        """Picks the fastest rasteriser setting on this batch's own state
        (state restored afterwards); returns the chosen setting.  cache: path
        of a JSON file of earlier results keyed by tune_key(); a hit applies
        the stored setting without timing (returned with "cached": True), a
        miss tunes and adds its result to the file."""
        key = self.tune_key() if cache is not None else None
        if key is not None and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
            if key in table:
                self.apply_tune(table[key])
                return dict(table[key], cached=True)
        r = GxTuneResult()
        _check(lib().gx_autotune(self.handle, C.c_void_p(actions.data_ptr()),
                                 C.byref(self._outs), int(steps), C.byref(r),
                                 self._stream(stream)), self.handle)
        best = {"small_tri_px": r.small_tri_px, "order_costliest_first": r.order_costliest_first,
                "raster_ctas": r.raster_ctas, "raster_warps": r.raster_warps,
                "occlusion_cull": r.occlusion_cull, "ms_per_step": r.ms_per_step}
        if key is not None:
            table = {}
            if os.path.exists(cache):
                with open(cache) as f:
                    table = json.load(f)
            table[key] = best
            tmp = f"{cache}.{os.getpid()}.tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return best

    def step_counters(self):
        """Step event counters since the last call (profile bit 4 only)."""
        v = (C.c_int64 * len(STEP_COUNTERS))()
        _check(lib().gx_step_counters(self.handle, v, len(STEP_COUNTERS)), self.handle)
        return dict(zip(STEP_COUNTERS, list(v)))

    def nsdf_counters(self):
        """Neural-SDF decision counters since the last call (profile bit 2 only)."""
        v = (C.c_int64 * 4)()
        _check(lib().gx_nsdf_counters(self.handle, v), self.handle)
        return dict(zip(["tests", "grid_fallbacks", "disagree", "env_disagree"], list(v)))

    def nsdf_step_predictions(self):
        """The network's predictions the last step's static test used, [n][32]
        (sdf_mode 1; slot s < 30 robot sphere s, 30 the held object)."""
        out = np.empty((self.n, 32), np.float32)
        _check(lib().gx_nsdf_step_predictions(
            self.handle, out.ctypes.data_as(C.POINTER(C.c_float)), out.size), self.handle)
        return out

    def sync(self):
        _check(lib().gx_sync(self.handle), self.handle)

    def device_error(self):
        return int(lib().gx_device_error(self.handle))

    # ------------------------------------------------------------- state
    def state_bytes(self):
        return int(lib().gx_state_bytes(self.handle))

    def save_state(self) -> np.ndarray:
        buf = np.zeros(self.state_bytes(), np.uint8)
        _check(lib().gx_save_state(self.handle, buf.ctypes.data, buf.nbytes), self.handle)
        return buf

    def load_state(self, buf: np.ndarray):
        buf = np.ascontiguousarray(buf, np.uint8)
        _check(lib().gx_load_state(self.handle, buf.ctypes.data, buf.nbytes), self.handle)

    def layout(self):
        offs = (C.c_size_t * STATE_ARRAYS)()
        _check(lib().gx_state_layout(self.handle, offs), self.handle)
        return list(offs)

    def state_arrays(self, buf=None):
        """Views of a saved state blob as named numpy arrays."""
        buf = self.save_state() if buf is None else buf
        o = self.layout()
        n, M = self.n, max(self.M, 1)

        def arr(k, dt, shape):
            cnt = int(np.prod(shape))
            return np.frombuffer(buf, dt, cnt, o[k]).reshape(shape)

        return dict(base_x=arr(0, np.float32, (n,)), base_z=arr(1, np.float32, (n,)),
                    yaw=arr(2, np.float32, (n,)), q=arr(3, np.float32, (7, n)),
                    held=arr(4, np.int32, (n,)), c_off=arr(5, np.float32, (3, n)),
                    p_pre=arr(6, np.float32, (3, n)), obj=arr(7, np.float32, (n, M, 4)),
                    step=arr(8, np.int32, (n,)), episode=arr(9, np.int32, (n,)),
                    task=arr(10, np.float32, (n, 16)), box=arr(11, np.float32, (n, M, 4)),
                    r_off=arr(12, np.float32, (9, n)))

    def close(self):
        if self.handle:
            lib().gx_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
