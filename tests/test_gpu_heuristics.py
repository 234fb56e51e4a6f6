"""The paper's sliding and object-placing heuristics (appendix "Description of
Heuristics") on the GPU against the oracle's orc_step_ex, in lockstep: every
environment, every step, bit-exact discrete results outside the near band."""
import numpy as np
import pytest

import oracle as O
from paper_2306_07552_b300 import inputs as I
from tests.parity import Tally, check_image, check_step

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROBOT = I.fetch_like_robot()


@pytest.fixture(scope="module")
def room():
    from paper_2306_07552_b300 import build, gx
    build.build()
    scene = I.room_scene(1000, 2000)
    ss = gx.SceneSet([scene])
    orc = O.Oracle(ROBOT, scene, I.icosahedron(), I.object_colors(256))
    yield gx, scene, ss, orc
    ss.close()


def _lockstep(sim, orc, acts, M, seed, tally, img_envs=()):
    slid = 0
    fn = lambda st, a, e: orc.step_ex(st, a, slide=True, place_jitter=True, seed=seed, env=e)  # noqa
    for t in range(len(acts)):
        before = {k: v.copy() for k, v in sim.state_arrays().items()}
        out = sim.step(torch.from_numpy(acts[t]).cuda())
        torch.cuda.synchronize()
        after = sim.state_arrays()
        check_step(orc, before, after, out, acts[t], range(sim.n), M, tally, step_fn=fn)
        slid += int(((out["contact_flags"].cpu().numpy() & 8) != 0).sum())
        for e in img_envs:
            check_image(orc, after, out, e, sim.W, sim.H, M, tally)
    return slid


def test_sliding_matches_oracle(room):
    gx, scene, ss, orc = room
    n, M, seed = 64, 10, 21
    sim = gx.Sim(ss, ROBOT, n, img=(64, 64), n_objects=M, seed=seed, heuristics=3)
    sim.reset()
    acts = I.make_actions(40, n, "uniform", seed=4)
    tally = Tally()
    slid = _lockstep(sim, orc, acts, M, seed, tally, img_envs=(0, 7))
    print(tally, f"slides {slid}")
    assert slid >= 20                                   # the heuristic really ran
    assert tally.near_band <= 0.05 * tally.envs
    assert sim.device_error() == 0
    sim.close()


def test_placing_jitter_matches_oracle(room):
    gx, scene, ss, orc = room
    n, M, seed = 32, 10, 22
    sim = gx.Sim(ss, ROBOT, n, img=(64, 64), n_objects=M, seed=seed, heuristics=3)
    sim.reset()
    # object 0 just in front of the tip, object 1 (smaller, 1 cm aside)
    # resting on the floor below it: releasing object 0 in place lands on
    # object 1; a jitter of 2 rho then clears it by 5 mm or more
    s = sim.state_arrays()
    buf = sim.save_state().copy()
    o = sim.layout()
    obj = np.frombuffer(buf, np.float32, n * M * 4, o[7]).reshape(n, M, 4).copy()
    clear = float(np.float32(ROBOT.rest_clearance))
    for e in range(n):
        _, ee, _ = orc.fk((s["base_x"][e], s["base_z"][e], s["yaw"][e]), s["q"][:, e])
        R, t = ee[:9].reshape(3, 3), ee[9:]
        p = t + R @ np.array([0.05, 0.0, 0.0])
        obj[e, 0] = [*p, 0.035]
        obj[e, 1] = [p[0] + 0.01, 0.03 + clear, p[2], 0.03]
    buf[o[7]:o[7] + obj.nbytes] = obj.view(np.uint8).ravel()
    sim.load_state(buf)
    acts = np.zeros((4, n, 11), np.float32)
    acts[:2, :, 9] = 1.0                                # grasp, hold, release, rest
    tally = Tally()
    _lockstep(sim, orc, acts, M, seed, tally)
    print(tally)
    assert tally.events.get(1, 0) >= n // 2
    assert tally.events.get(5, 0) >= n // 4             # jittered landings
    sim.close()
