"""The object broad-phase (four offset regular grids per environment) on the
GPU: with 200 objects per environment the step must give exactly the
brute-force results -- against the oracle in lockstep, and bit for bit
against the same context without the broad-phase, through grasps, releases
(which move objects between cells) and a state reload (which rebuilds the
cells)."""
import numpy as np
import pytest

import oracle as O
from paper_2306_07552_b300 import inputs as I
from tests.parity import Tally, check_step

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROBOT = I.fetch_like_robot()
KEYS = ["depth", "rgb", "pose", "obj_pos", "held", "contact_mask", "contact_flags", "event",
        "reward", "task_obs", "success"]


@pytest.fixture(scope="module")
def apartment():
    from paper_2306_07552_b300 import build, gx
    build.build()
    scene = I.apartment_scene(1005, 25000)
    ss = gx.SceneSet([scene])
    orc = O.Oracle(ROBOT, scene, I.icosahedron(), I.object_colors(256))
    yield gx, scene, ss, orc
    ss.close()


def _actions(T, n, seed):
    a = I.make_actions(T, n, "uniform", seed=seed)
    a[:, :, 9] = np.where(np.arange(T)[:, None] % 6 < 3, 1.0, 0.0)   # grasp 3, release 3
    return a


def test_broadphase_matches_oracle_with_200_objects(apartment):
    gx, scene, ss, orc = apartment
    n, M = 64, 200
    sim = gx.Sim(ss, ROBOT, n, img=(64, 64), n_objects=M, seed=12, broadphase=True,
                 heuristics=2)
    sim.reset()
    acts = _actions(24, n, 3)
    tally = Tally()
    fn = lambda st, a, e: orc.step_ex(st, a, place_jitter=True, seed=12, env=e)  # noqa: E731
    for t in range(len(acts)):
        before = {k: v.copy() for k, v in sim.state_arrays().items()}
        out = sim.step(torch.from_numpy(acts[t]).cuda())
        torch.cuda.synchronize()
        after = sim.state_arrays()
        check_step(orc, before, after, out, acts[t], range(n), M, tally, step_fn=fn)
    print(tally)
    assert tally.contacts > 0 and tally.near_band <= 0.1 * tally.envs
    assert sim.device_error() == 0
    sim.close()


def test_broadphase_is_bit_identical_to_brute_force(apartment):
    gx, scene, ss, orc = apartment
    n, M = 256, 200
    kw = dict(img=(64, 64), n_objects=M, seed=13, heuristics=3)
    a = gx.Sim(ss, ROBOT, n, **kw)
    b = gx.Sim(ss, ROBOT, n, broadphase=True, **kw)
    a.reset()
    b.reset()
    # object 0 of every env just in front of the tool tip (loading the state
    # rebuilds b's cells), so the grasp-carry-release script moves objects
    st = a.state_arrays()
    buf = a.save_state().copy()
    o = a.layout()
    obj = np.frombuffer(buf, np.float32, n * M * 4, o[7]).reshape(n, M, 4).copy()
    for e in range(n):
        _, ee, _ = orc.fk((st["base_x"][e], st["base_z"][e], st["yaw"][e]), st["q"][:, e])
        R, tt = ee[:9].reshape(3, 3), ee[9:]
        obj[e, 0, :3] = tt + R @ np.array([0.05, 0.0, 0.0])
        obj[e, 0, 3] = 0.035
    buf[o[7]:o[7] + obj.nbytes] = obj.view(np.uint8).ravel()
    a.load_state(buf)
    b.load_state(buf)
    acts = _actions(30, n, 4)
    acts[:, :, 2:9] *= 0.5
    moved = 0
    for t in range(30):
        if t == 15:   # a reload rebuilds the cells from the saved objects
            s = b.save_state()
            b.load_state(s)
        x = torch.from_numpy(acts[t]).cuda()
        oa, ob = a.step(x), b.step(x)
        torch.cuda.synchronize()
        moved += int(((oa["event"] == 3) | (oa["event"] == 5)).sum())
        for k in KEYS:
            assert torch.equal(oa[k], ob[k]), (t, k)
    print(f"objects moved by releases: {moved}")
    assert moved > 20
    a.close()
    b.close()
