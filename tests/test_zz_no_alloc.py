"""gx_render_noalloc: rendering for callers that cannot allocate device memory
when they need images (allocation-free sections of real-time or serving
code, hosts that only allocate at start-up).  It renders with a fixed scratch
array inside the library, so its images must agree with those of the regular
step, which renders with framebuffer slots its context allocated, and with
the FP64 oracle's images of the same state.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_2306_07552_b300 import inputs as I
from tests.parity import DEPTH_REL, oracle_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROBOT = I.fetch_like_robot()


def _camera_rows(orc, st_arrays, n):
    """Camera-to-world poses in the library's layout, from the FP64 oracle's
    kinematics of the GPU state, rounded to float32."""
    cam = np.zeros((n, 12), np.float32)
    for e in range(n):
        _, _, c = orc.fk((st_arrays["base_x"][e], st_arrays["base_z"][e], st_arrays["yaw"][e]),
                         st_arrays["q"][:, e])
        cam[e] = c.astype(np.float32)
    return cam


def test_render_noalloc_matches_step_on_two_calls():
    from paper_2306_07552_b300 import build, gx
    build.build()
    L = gx.lib()
    scene = I.room_scene(1000, 2000)
    ss = gx.SceneSet([scene])
    n, M, W = 16, 10, 64
    sim = gx.Sim(ss, ROBOT, n, img=(W, W), n_objects=M, obj_radius=(0.03, 0.06), seed=21)
    sim.reset()
    orc = O.Oracle(ROBOT, scene, I.icosahedron(), I.object_colors(256))
    env_scene = torch.zeros(n, dtype=torch.int32, device="cuda")
    depth = torch.empty((n, W, W), dtype=torch.float32, device="cuda")
    rgb = torch.empty((n, W, W, 3), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    acts = I.make_actions(2, n, "uniform", seed=13)
    checked = 0
    for call in range(2):
        out = sim.step(torch.from_numpy(acts[call]).cuda())
        torch.cuda.synchronize()
        st = sim.state_arrays()
        cam = torch.from_numpy(_camera_rows(orc, st, n)).cuda()
        obj = torch.from_numpy(np.ascontiguousarray(st["obj"][:, :M])).cuda()
        depth.fill_(-1.0)
        rgb.fill_(7)
        status = L.gx_render_noalloc(ss.handle, n, C.c_void_p(env_scene.data_ptr()),
                                     C.c_void_p(cam.data_ptr()), C.c_void_p(obj.data_ptr()), M,
                                     W, W, ROBOT.cam_near, C.c_void_p(depth.data_ptr()), 0,
                                     C.c_void_p(rgb.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert status == gx.GX_OK, L.gx_last_error(None)
        torch.cuda.synchronize()
        nd, ng = depth.cpu().numpy().astype(np.float64), rgb.cpu().numpy()
        sd, sg = out["depth"].cpu().numpy().astype(np.float64), out["rgb"].cpu().numpy()
        for e in range(n):
            # pixels the oracle does not flag as ambiguous for this state:
            # coverage and colour exact, depth within the parity tolerance
            _, _, amb, _, _ = orc.render(oracle_state(st, e, M), W, W)
            ok = ~amb
            assert np.array_equal(nd[e][ok] > 0, sd[e][ok] > 0)
            assert np.array_equal(ng[e][ok], sg[e][ok])
            cov = ok & (sd[e] > 0)
            assert np.all(np.abs(nd[e][cov] - sd[e][cov]) <= DEPTH_REL * sd[e][cov])
            checked += int(ok.sum())
    assert checked > 0.9 * 2 * n * W * W
    # sizes beyond the fixed scratch are refused before any work
    status = L.gx_render_noalloc(ss.handle, n, C.c_void_p(env_scene.data_ptr()),
                                 C.c_void_p(cam.data_ptr()), C.c_void_p(obj.data_ptr()), M, 512,
                                 512, ROBOT.cam_near, C.c_void_p(depth.data_ptr()), 0, None,
                                 C.c_void_p(stream.cuda_stream))
    assert status == gx.GX_EINVAL
    assert b"256" in L.gx_last_error(None)
    sim.close()
    ss.close()


def _render(L, gx, ss, n, env_scene, cam, obj, M, W, depth, fp16, rgb, stream):
    return L.gx_render_noalloc(ss.handle, n, C.c_void_p(env_scene.data_ptr()),
                               C.c_void_p(cam.data_ptr()), C.c_void_p(obj.data_ptr()), M, W, W,
                               ROBOT.cam_near, C.c_void_p(depth.data_ptr()), fp16,
                               C.c_void_p(rgb.data_ptr()) if rgb is not None else None,
                               C.c_void_p(stream.cuda_stream))


def _check_vs_oracle(orc, st, e, M, W, nd, ng, fp16=False):
    """Unambiguous pixels: coverage and colour equal the oracle's, depth
    within 1e-5 relative (FP32) or half an FP16 ulp + 1e-5 relative."""
    depth, rgb, amb, _, _ = orc.render(oracle_state(st, e, M), W, W)
    ok = ~amb
    assert np.array_equal(nd[ok] > 0, depth[ok] > 0)
    if ng is not None:
        g = ng.astype(np.uint32)
        assert np.array_equal(((g[..., 0] << 16) | (g[..., 1] << 8) | g[..., 2])[ok], rgb[ok])
    cov = ok & (depth > 0)
    lim = DEPTH_REL * depth[cov]
    if fp16:
        lim = lim + 0.5 * np.spacing(depth[cov].astype(np.float16)).astype(np.float64)
    assert np.all(np.abs(nd[cov] - depth[cov]) <= lim)
    return int(ok.sum())


def test_render_noalloc_many_envs_per_slot_fp16_and_bad_scene():
    """256x256 images leave room for 32 framebuffer slots in the fixed scratch,
    so with 64 environments CTAs render several environments each; then the
    same images with FP16 depth; then scene indices outside the set, which
    the kernel refuses (empty images, error bit read back by
    gx_render_noalloc_error) while the other environments render as before."""
    from paper_2306_07552_b300 import build, gx
    build.build()
    L = gx.lib()
    scene = I.room_scene(1000, 2000)
    ss = gx.SceneSet([scene])
    n, M, W = 64, 10, 256
    sim = gx.Sim(ss, ROBOT, n, img=(W, W), n_objects=M, obj_radius=(0.03, 0.06), seed=23)
    sim.reset()
    orc = O.Oracle(ROBOT, scene, I.icosahedron(), I.object_colors(256))
    acts = I.make_actions(1, n, "uniform", seed=17)
    out = sim.step(torch.from_numpy(acts[0]).cuda())
    torch.cuda.synchronize()
    st = sim.state_arrays()
    cam = torch.from_numpy(_camera_rows(orc, st, n)).cuda()
    obj = torch.from_numpy(np.ascontiguousarray(st["obj"][:, :M])).cuda()
    env_scene = torch.zeros(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    assert L.gx_render_noalloc_error(None) in (gx.GX_OK, gx.GX_EDEVICE)  # start clean

    depth = torch.full((n, W, W), -1.0, dtype=torch.float32, device="cuda")
    rgb = torch.full((n, W, W, 3), 7, dtype=torch.uint8, device="cuda")
    assert _render(L, gx, ss, n, env_scene, cam, obj, M, W, depth, 0, rgb, stream) == gx.GX_OK
    bits = C.c_uint32(99)
    assert L.gx_render_noalloc_error(C.byref(bits)) == gx.GX_OK and bits.value == 0
    nd, ng = depth.cpu().numpy().astype(np.float64), rgb.cpu().numpy()
    sd, sg = out["depth"].cpu().numpy().astype(np.float64), out["rgb"].cpu().numpy()
    checked = 0
    for e in range(n):
        # the regular step's images of the same state (its camera from FP32
        # kinematics): coverage and colour agree except along silhouettes
        same = (nd[e] > 0) == (sd[e] > 0)
        assert same.mean() > 0.995, (e, same.mean())
        both = (nd[e] > 0) & (sd[e] > 0) & np.all(ng[e] == sg[e], axis=-1)
        close = np.abs(nd[e][both] - sd[e][both]) <= DEPTH_REL * sd[e][both]
        assert close.mean() > 0.999, (e, close.mean())
    for e in range(0, n, 8):
        checked += _check_vs_oracle(orc, st, e, M, W, nd[e], ng[e])
    assert checked > 0.9 * 8 * W * W

    # FP16 depth through the same scratch
    d16 = torch.full((n, W, W), -1.0, dtype=torch.float16, device="cuda")
    assert _render(L, gx, ss, n, env_scene, cam, obj, M, W, d16, 1, None, stream) == gx.GX_OK
    n16 = d16.float().cpu().numpy().astype(np.float64)
    assert np.array_equal(n16 > 0, nd > 0)
    assert np.array_equal(n16, nd.astype(np.float16).astype(np.float64))
    for e in range(3, n, 16):
        _check_vs_oracle(orc, st, e, M, W, n16[e], None, fp16=True)

    # scene indices outside [0, 1): those environments come back empty
    bad = [5, 22, 63]
    es = np.zeros(n, np.int32)
    es[bad] = [1, -1, 1 << 20]
    env_bad = torch.from_numpy(es).cuda()
    depth.fill_(-1.0)
    rgb.fill_(7)
    assert _render(L, gx, ss, n, env_bad, cam, obj, M, W, depth, 0, rgb, stream) == gx.GX_OK
    assert L.gx_render_noalloc_error(C.byref(bits)) == gx.GX_EDEVICE
    assert bits.value & gx.GX_NOALLOC_BAD_SCENE
    assert b"scene index" in L.gx_last_error(None)
    bd, bg = depth.cpu().numpy().astype(np.float64), rgb.cpu().numpy()
    good = np.setdiff1d(np.arange(n), bad)
    assert np.all(bd[bad] == 0) and np.all(bg[bad] == 0)
    assert np.array_equal(bd[good], nd[good]) and np.array_equal(bg[good], ng[good])
    # the word was cleared by the query
    assert L.gx_render_noalloc_error(C.byref(bits)) == gx.GX_OK and bits.value == 0
    sim.close()
    ss.close()
