"""gx_render_noalloc: rendering for callers that cannot allocate device memory
when they need images (allocation-free sections of real-time or serving
code, hosts that only allocate at start-up).  It renders with a fixed scratch
array inside the library, so its images must agree with those of the regular
step, which renders with framebuffer slots its context allocated.

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
