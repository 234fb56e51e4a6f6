"""Every rasteriser setting the autotuner may pick renders the oracle's images.

The autotuner chooses among expansion limits small_tri_px in {0, 256, 96, 48}
(triangles whose clipped bounding box exceeds the limit are scanned by a whole
warp over 8x4 blocks with int64 edge functions instead of being expanded
pixel by pixel), two work orders (index order, costliest scene first) and
four CTA shapes (8 warps, three CTAs per SM; 12 warps, two per SM; 6 or 7
warps, four per SM).
Each candidate is checked against the FP64 oracle's images of the same
state, pixel by pixel, on views forced close to walls so that the block-scan
path draws many large triangles per view (coarsely tessellated walls a
few tenths of a metre from the camera).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2306_07552_b300 import inputs as I
from tests.parity import Tally, check_image, oracle_image

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROBOT = I.fetch_like_robot()
SIZE = 6.0   # room_scene interior: x and z in [0, 6]


def near_wall_poses(n, seed):
    """Base poses 0.35-0.85 m from one of the four walls, facing it within
    +-0.6 rad (forward = (cos yaw, 0, -sin yaw))."""
    rng = np.random.default_rng(seed)
    x = np.zeros(n, np.float32)
    z = np.zeros(n, np.float32)
    yaw = np.zeros(n, np.float32)
    for e in range(n):
        d = 0.35 + 0.5 * rng.random()
        lat = 1.0 + 4.0 * rng.random()
        k = e % 4
        if k == 0:
            x[e], z[e], face = SIZE - d, lat, 0.0            # wall x = 6
        elif k == 1:
            x[e], z[e], face = d, lat, math.pi               # wall x = 0
        elif k == 2:
            x[e], z[e], face = lat, d, math.pi / 2           # wall z = 0
        else:
            x[e], z[e], face = lat, SIZE - d, -math.pi / 2   # wall z = 6
        a = face + rng.uniform(-0.6, 0.6)
        yaw[e] = math.atan2(math.sin(a), math.cos(a))
    return x, z, yaw


def test_every_autotune_candidate_renders_the_oracle_images():
    from paper_2306_07552_b300 import build, gx
    build.build()
    # coarse walls (few, very large triangles) and a fine room whose
    # 15-20 cm wall triangles cover a few hundred pixels each at these
    # distances
    scenes = [I.room_scene(1000, 600), I.room_scene(1001, 12000)]
    ss = gx.SceneSet(scenes)
    orcs = [O.Oracle(ROBOT, sc, I.icosahedron(), I.object_colors(256)) for sc in scenes]
    n, M, W = 48, 10, 128
    env_scene = np.repeat(np.arange(2), n // 2).astype(np.int32)
    kw = dict(img=(W, W), n_objects=M, obj_radius=(0.03, 0.06), seed=31, env_scene=env_scene)
    base = gx.Sim(ss, ROBOT, n, **kw)
    base.reset()
    torch.cuda.synchronize()
    blob = base.save_state()
    arrs = base.state_arrays(blob)
    arrs["base_x"][:], arrs["base_z"][:], arrs["yaw"][:] = near_wall_poses(n, 7)
    base.close()
    still = torch.zeros((n, 11), dtype=torch.float32, device="cuda")   # stand still

    # how often the block-scan path runs under the smallest limit
    counting = gx.Sim(ss, ROBOT, n, small_tri_px=48, profile=2, **kw)
    counting.load_state(blob)
    counting.step(still)
    c = counting.raster_counters()
    counting.close()
    per_view = c["tris_warp"] / n
    print("warp-scanned triangles per view at small_tri_px=48:", per_view,
          "expanded:", c["tris_expand"] / n)
    assert per_view >= 60

    refs, after0, tally = None, None, Tally()
    cands = [(px, order, 8) for px in (0, 256, 96, 48) for order in (1, 2)]
    cands += [(px, 2, 12) for px in (0, 48)]     # the 12-warp CTA shape
    cands += [(px, o, 6) for px in (0, 48) for o in (1, 2)]   # the 6-warp CTA shape
    cands += [(px, o, 7) for px in (0, 48) for o in (1, 2)]   # the 7-warp CTA shape
    for px, order, warps in cands:
        sim = gx.Sim(ss, ROBOT, n, small_tri_px=px, raster_order=order, raster_warps=warps,
                     **kw)
        sim.load_state(blob)
        out = sim.step(still)
        torch.cuda.synchronize()
        after = sim.state_arrays()
        if refs is None:
            after0 = {k: v.copy() for k, v in after.items()}
            refs = [oracle_image(orcs[env_scene[e]], after0, e, W, W, M) for e in range(n)]
        for k in after0:
            assert np.array_equal(after[k], after0[k]), (px, order, warps, k)
        for e in range(n):
            check_image(orcs[env_scene[e]], after0, out, e, W, W, M, tally, ref=refs[e])
        sim.close()
    print(tally)
    print(tally.report())
    assert tally.pixels > 0.9 * len(cands) * n * W * W
    ss.close()
