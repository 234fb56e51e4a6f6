"""Step event counters (profile bit 4, gx_step_counters): the event counts
equal what the step's own outputs show, step after step (contact masks,
grasp events, sliding flags); the near-threshold counts agree with the same
tests recomputed in FP64 by the oracle from the step's state and actions (the
candidate sphere centres, grid distances and object distances); counting
changes no result."""
import numpy as np
import pytest

import oracle as O
from paper_2306_07552_b300 import inputs as I
from tests.parity import oracle_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROBOT = I.fetch_like_robot()
BAND = 1e-4


def test_step_counters_match_outputs_and_oracle():
    from paper_2306_07552_b300 import build, gx
    build.build()
    scene = I.room_scene(1000, 2000)
    ss = gx.SceneSet([scene])
    orc = O.Oracle(ROBOT, scene, I.icosahedron(), I.object_colors(256))
    n, M, T = 64, 10, 25
    kw = dict(img=(64, 64), n_objects=M, seed=6, heuristics=1)
    a = gx.Sim(ss, ROBOT, n, profile=16, **kw)
    b = gx.Sim(ss, ROBOT, n, **kw)
    a.reset()
    b.reset()
    a.step_counters()                      # the resets count nothing; start clean
    acts = I.make_actions(T, n, "uniform", seed=7)
    want = dict.fromkeys(gx.STEP_COUNTERS, 0)
    near_s = near_o = 0
    for t in range(T):
        before = a.state_arrays()
        x = torch.from_numpy(acts[t]).cuda()
        oa, ob = a.step(x), b.step(x)
        torch.cuda.synchronize()
        for k in ("depth", "pose", "obj_pos", "contact_mask", "contact_flags", "event"):
            assert torch.equal(oa[k], ob[k]), (t, k)
        mask = oa["contact_mask"].cpu().numpy()
        ev = oa["event"].cpu().numpy()
        fl = oa["contact_flags"].cpu().numpy()
        want["contacts"] += int((mask != 0).sum())
        want["grasps"] += int((ev == 1).sum())
        want["grasp_misses"] += int((ev == 2).sum())
        want["landed"] += int(((ev == 3) | (ev == 5)).sum())
        want["restored"] += int((ev == 4).sum())
        want["slides"] += int(((fl & 8) != 0).sum())
        # the near-threshold tests recomputed in FP64 at the candidate pose
        for e in range(n):
            st = oracle_state(before, e, M)
            c, r, act = orc.candidate_spheres(st, acts[t, e])
            objs = O.Oracle.state_objs(st)
            held = int(st.held)
            for i in np.flatnonzero(act):
                inside, d, _ = orc.grid_query(c[i])
                near_s += int(inside and abs(d - r[i]) < BAND)
                dist = np.linalg.norm(objs[:, :3] - c[i], axis=1) - (r[i] + objs[:, 3])
                if held >= 0:
                    dist[held] = np.inf
                near_o += int(np.any(np.abs(dist) < BAND))
    got = a.step_counters()
    print(got, f"oracle near static {near_s}, near pairs {near_o}")
    for k in ("contacts", "grasps", "grasp_misses", "landed", "restored", "slides"):
        assert got[k] == want[k], k
    assert got["contacts"] > 0 and got["slides"] > 0 and got["grasp_misses"] > 0
    for g, o in ((got["near_static"], near_s), (got["near_pairs"], near_o)):
        assert abs(g - o) <= max(2, 0.05 * o), (g, o)
    with pytest.raises(gx.GxError):
        b.step_counters()                  # a context that does not count
    a.close()
    b.close()
    ss.close()
