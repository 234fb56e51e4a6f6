"""The column grid on the GPU (sdf_mode 2) against the oracle: the spans the
GPU builds (FP64, stored in FP32) and the step's decisions in lockstep."""
import numpy as np
import pytest

import oracle as O
from paper_2306_07552_b300 import inputs as I
from tests.parity import Tally, check_step

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROBOT = I.fetch_like_robot()


@pytest.fixture(scope="module")
def scenes():
    from paper_2306_07552_b300 import build, gx
    build.build()
    sc = [I.room_scene(1000, 2000), I.apartment_scene(1003, 20000)]
    ss = gx.SceneSet(sc)
    orcs = [O.Oracle(ROBOT, s, I.icosahedron(), I.object_colors(256)) for s in sc]
    yield gx, sc, ss, orcs
    ss.close()


def test_column_spans_match_oracle(scenes):
    gx, sc, ss, orcs = scenes
    rng = np.random.default_rng(3)
    for s in range(2):
        dims, nbytes = ss.column_info(s)
        assert dims == orcs[s].column_dims()
        print(f"scene {s}: columns {dims}, {nbytes / 1e6:.1f} MB")
        for _ in range(400):
            ri = int(rng.integers(0, 3))
            i, k = int(rng.integers(0, dims[0])), int(rng.integers(0, dims[1]))
            g = ss.column_spans(s, ri, i, k).astype(np.float64)
            o = orcs[s].column_spans(ri, i, k)
            assert g.shape == o.shape, (s, ri, i, k, g, o)
            assert np.allclose(g, o, rtol=0, atol=1e-6 * (1 + np.abs(o)))


def test_column_step_matches_oracle(scenes):
    gx, sc, ss, orcs = scenes
    n, M, seed = 64, 10, 31
    es = np.arange(n) % 2
    sim = gx.Sim(ss, ROBOT, n, img=(64, 64), n_objects=M, seed=seed, env_scene=es, sdf_mode=2)
    sim.reset()
    acts = I.make_actions(30, n, "uniform", seed=8)
    tallies = [Tally(), Tally()]
    for t in range(30):
        before = {k: v.copy() for k, v in sim.state_arrays().items()}
        out = sim.step(torch.from_numpy(acts[t]).cuda())
        torch.cuda.synchronize()
        after = sim.state_arrays()
        for s in range(2):
            fn = lambda st, a, e, s=s: orcs[s].step_ex(st, a, column=True)  # noqa: E731
            check_step(orcs[s], before, after, out, acts[t], np.flatnonzero(es == s), M,
                       tallies[s], step_fn=fn)
    print(tallies)
    for tl in tallies:
        assert tl.near_band <= 0.1 * tl.envs and tl.contacts > 0
    sim.close()
