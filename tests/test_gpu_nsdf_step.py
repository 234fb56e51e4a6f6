"""The neural SDF inside the step (sdf_mode 1) against the FP64 oracle.

The oracle applies the same rule (orc_step_nsdf): outside the lattice box is
contact, a predicted clearance d - r of at least the margin is free, else the
grid decides.  The check is split in two.  The rule: the oracle takes the
predictions the GPU's step used (gx_nsdf_step_predictions) and must reach the
same decisions, near band 1e-4 m as everywhere.  The network: those
predictions, at the oracle's own sphere centres (weights drawn here, W1..W4
rounded to BF16 with PyTorch), against
  - the plain FP64 MLP (nothing but the weights rounded): every prediction
    within the oracle's first-order rounding bound of the BF16-operand
    network (orc_mlp_rounding_bound), and within 6 standard deviations of
    independent roundings (a wrong row would stand out by far more); the
    margin decisions (d - r >= margin) that differ from the plain network's
    are counted;
  - the oracle's BF16-operand mode, which rounds at the kernels' points: the
    median error is the FP32 sums alone (~1e-7).
"""
import numpy as np
import pytest

import oracle as O
from paper_2306_07552_b300 import inputs as I
from tests.parity import Tally, check_step

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROBOT = I.fetch_like_robot()
MARGIN = 0.02
NEAR_BAND = 1e-4


def network_errors(errs, refs):
    """Prediction error of the step's network against the oracle MLP in its
    BF16-operand mode: the same rounding points, so the median is the FP32
    sums alone."""
    err, ref = np.concatenate(errs), np.concatenate(refs)
    scale = 1 + np.abs(ref).mean()
    print(f"step predictions vs oracle MLP (BF16 operands): median {np.median(err):.2e}, "
          f"p99 {np.quantile(err, .99):.2e}, max {err.max():.2e} over {err.size}")
    assert np.median(err) < 1e-5 * scale


def plain_errors(errs, bounds, sigmas, flips, n_decisions, label):
    """Predictions against the plain FP64 network: each within its rounding
    bound and within 6 standard deviations of independent roundings."""
    err, bnd, sig = np.concatenate(errs), np.concatenate(bounds), np.concatenate(sigmas)
    z = err / sig
    print(f"{label}: |gpu - plain FP64| median {np.median(err):.2e}, max {err.max():.2e}; "
          f"bound median {np.median(bnd):.2e}, max {bnd.max():.2e}; err/bound max "
          f"{(err / bnd).max():.3f}; in deviations: rms {np.sqrt(np.mean(z ** 2)):.2f}, max "
          f"{z.max():.2f}; margin decisions differing {flips} of {n_decisions}")
    assert np.all(err <= bnd)
    assert z.max() <= 6.0
    return err, bnd


def plain_mlp(B, P):
    """The plain FP64 network with the weights the kernels hold (W1..W4 in
    BF16), nothing else rounded."""
    m = oracle_mlp(B, P)
    return O.MLP64(m.B, m.Ws, m.bs, bf16_operands=False)


def _bf16(a):
    return torch.as_tensor(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def oracle_mlp(B, P):
    """FP64 MLP with the weights a BF16 kernel holds: W1..W4 rounded by
    PyTorch, biases and the output row as given."""
    sizes = [(128, 64), (128, 128), (128, 128), (128, 128), (1, 128)]
    Ws, bs, o = [], [], 0
    for l, (n_out, n_in) in enumerate(sizes):
        W = np.asarray(P[o:o + n_in * n_out], np.float32).reshape(n_out, n_in)
        Ws.append(_bf16(W) if l < 4 else W.astype(np.float64))
        o += n_in * n_out
        bs.append(np.asarray(P[o:o + n_out], np.float64))
        o += n_out
    return O.MLP64(np.asarray(B, np.float64), Ws, bs, bf16_operands=True)


def grid_centre(scene):
    return scene.grid_origin.astype(np.float64) + 0.5 * (scene.grid_dims - 1) * np.float64(
        scene.grid_h)


@pytest.fixture(scope="module")
def two_rooms():
    from paper_2306_07552_b300 import build, gx
    build.build()
    scenes = [I.room_scene(1000, 2000), I.room_scene(1001, 2000)]
    ss = gx.SceneSet(scenes)
    B = I.fourier_matrix(7)
    Ps = []
    for k in range(2):
        P = I.nsdf_init(7 + k)
        P[-1] = 0.3 + 0.2 * k          # output bias: a mix of trusted and checked spheres
        ss.nsdf_set_weights(k, B, P)
        Ps.append(P)
    orcs = [O.Oracle(ROBOT, sc, I.icosahedron(), I.object_colors(256)) for sc in scenes]
    yield gx, scenes, ss, orcs, B, Ps
    ss.close()


def test_huge_margin_reproduces_the_grid_step(two_rooms):
    """Every sphere falls back to the grid: the neural mode must give the
    grid mode's results bit for bit (also through graph replay)."""
    gx, scenes, ss, orcs, B, Ps = two_rooms
    n, M = 96, 12
    es = np.arange(n) % 2                                     # interleaved scenes
    kw = dict(img=(64, 64), n_objects=M, seed=3, env_scene=es)
    a = gx.Sim(ss, ROBOT, n, **kw)
    b = gx.Sim(ss, ROBOT, n, sdf_mode=1, sdf_margin=1e6, use_graph=True, **kw)
    a.reset()
    b.reset()
    acts = I.make_actions(25, n, "gaussian", seed=2)
    for t in range(25):
        x = torch.from_numpy(acts[t]).cuda()
        oa, ob = a.step(x), b.step(x)
        torch.cuda.synchronize()
        for k in ["depth", "rgb", "pose", "obj_pos", "held", "contact_mask", "contact_flags",
                  "event"]:
            assert torch.equal(oa[k], ob[k]), (t, k)
    a.close()
    b.close()


def test_neural_step_is_deterministic(two_rooms):
    """Two contexts in neural mode, one replaying a CUDA graph: identical
    results step after step."""
    gx, scenes, ss, orcs, B, Ps = two_rooms
    n, M = 96, 12
    es = np.arange(n) % 2
    kw = dict(img=(64, 64), n_objects=M, seed=3, env_scene=es, sdf_mode=1, sdf_margin=MARGIN)
    a = gx.Sim(ss, ROBOT, n, **kw)
    b = gx.Sim(ss, ROBOT, n, use_graph=True, **kw)
    a.reset()
    b.reset()
    acts = I.make_actions(20, n, "gaussian", seed=4)
    stream = torch.cuda.Stream()
    x = torch.empty((n, 11), dtype=torch.float32, device="cuda")
    for t in range(20):
        with torch.cuda.stream(stream):
            x.copy_(torch.from_numpy(acts[t]))
            oa, ob = a.step(x, stream=stream), b.step(x, stream=stream)
        torch.cuda.synchronize()
        for k in ["depth", "rgb", "pose", "obj_pos", "held", "contact_mask", "contact_flags",
                  "event", "reward"]:
            assert torch.equal(oa[k], ob[k]), (t, k)
        assert np.array_equal(a.nsdf_step_predictions(), b.nsdf_step_predictions(), equal_nan=True)
    a.close()
    b.close()


def test_neural_rule_matches_oracle(two_rooms):
    gx, scenes, ss, orcs, B, Ps = two_rooms
    n, M, T = 64, 12, 30
    es = np.arange(n) % 2
    sim = gx.Sim(ss, ROBOT, n, img=(64, 64), n_objects=M, seed=5, env_scene=es, sdf_mode=1,
                 sdf_margin=MARGIN, profile=4)
    sim.reset()
    mlps = [oracle_mlp(B, P) for P in Ps]
    plains = [plain_mlp(B, P) for P in Ps]
    cents = [grid_centre(sc) for sc in scenes]
    acts = I.make_actions(T, n, "gaussian", seed=6)
    tallies = [Tally(), Tally()]
    trusted = 0
    errs, refs = [], []
    perrs, pbounds, psig = [], [], []
    flips = decisions = 0

    def step_fn_for(k, pred):
        def f(st, action, env):
            nonlocal trusted, flips, decisions
            c, r, act = orcs[k].candidate_spheres(st, action)
            d = np.full(31, -1e9)
            idx = np.flatnonzero(act)
            d[idx] = pred[env, idx]
            assert np.all(np.isfinite(d[idx])), env
            ref = mlps[k].forward(c[idx] - cents[k])
            errs.append(np.abs(d[idx] - ref))
            refs.append(ref)
            plain, bnd, parts = plains[k].rounding_bound(c[idx] - cents[k], terms=True)
            perrs.append(np.abs(d[idx] - plain))
            pbounds.append(bnd)
            psig.append(parts[:, 3])
            flips += int(np.sum((d[idx] - r[idx] >= MARGIN) != (plain - r[idx] >= MARGIN)))
            decisions += len(idx)
            trusted += int(np.sum(d[idx] - r[idx] >= MARGIN))
            return orcs[k].step_nsdf(st, action, d, MARGIN, NEAR_BAND)
        return f

    for t in range(T):
        before = {k: v.copy() for k, v in sim.state_arrays().items()}
        out = sim.step(torch.from_numpy(acts[t]).cuda())
        torch.cuda.synchronize()
        after = sim.state_arrays()
        pred = sim.nsdf_step_predictions().astype(np.float64)
        for k in range(2):
            check_step(orcs[k], before, after, out, acts[t], np.flatnonzero(es == k), M,
                       tallies[k], step_fn=step_fn_for(k, pred))
    cnt = sim.nsdf_counters()
    print(tallies, f"trusted predictions {trusted}", cnt)
    network_errors(errs, refs)
    plain_errors(perrs, pbounds, psig, flips, decisions, "step predictions (random weights)")
    checked = sum(tl.envs - tl.near_band_flips for tl in tallies)
    assert checked >= 0.9 * n * T
    assert trusted > 0 and cnt["grid_fallbacks"] > 0     # both branches exercised
    assert cnt["tests"] >= n * T * 30
    sim.close()


def test_trained_network_agrees_with_the_grid(two_rooms):
    """Networks trained on each scene: the step's decisions against the
    grid-only rule (the grid is the reference), and what the network gains over
    the method without it: most static tests are decided by 116 KB of weights
    instead of gathers into the scene's distance grid."""
    gx, scenes, ss, orcs, B, Ps = two_rooms
    for k in range(2):
        ss.nsdf_set_weights(k, B, I.nsdf_init(7))
        losses = ss.nsdf_train(k, n_samples=4_000_000, batch=65536, steps=1500, lr=1e-3, seed=11)
        assert np.isfinite(losses).all()
    n, M, T = 512, 40, 60
    sim = gx.Sim(ss, ROBOT, n, img=(64, 64), n_objects=M, seed=8, sdf_mode=1,
                 sdf_margin=MARGIN, profile=4)
    sim.reset()
    acts = I.make_actions(T, n, "gaussian", seed=9)
    for t in range(T):
        sim.step(torch.from_numpy(acts[t]).cuda())
    c = sim.nsdf_counters()
    rate = c["disagree"] / c["tests"]
    env_rate = c["env_disagree"] / (n * T)
    print(f"static tests {c['tests']}, grid fallbacks {c['grid_fallbacks'] / c['tests']:.3%}, "
          f"decisions differing from the grid {rate:.4%}, env-steps differing {env_rate:.4%}")
    assert c["tests"] >= n * T * 30
    assert rate <= 1e-3
    # the gain: at least 80% of the static tests never touch the grid
    grid_share = c["grid_fallbacks"] / c["tests"]
    grid_bytes = int(np.prod(scenes[0].grid_dims)) * 4
    print(f"grid consulted for {grid_share:.2%} of the tests; network {gx.NSDF_PARAMS * 2} B of "
          f"BF16 weights vs a {grid_bytes / 1e6:.1f} MB distance grid")
    assert grid_share <= 0.2
    sim.close()
    # the trained networks' queries against the plain FP64 network: within
    # the rounding bound, and how many margin decisions (for the robot's
    # radii) the BF16 rounding changes
    radii = np.unique(np.asarray(ROBOT.sphere_radius, np.float64))
    for k in range(2):
        Bq, Pq, centre = ss.nsdf_get_weights(k)
        plain = plain_mlp(Bq, Pq)
        rng = np.random.default_rng(20 + k)
        lo = scenes[k].grid_origin.astype(np.float64)
        hi = lo + (scenes[k].grid_dims - 1) * np.float64(scenes[k].grid_h)
        pts = rng.uniform(lo, hi, (4096, 3)).astype(np.float32)
        out = torch.empty(len(pts), dtype=torch.float32, device="cuda")
        ss.nsdf_query(k, torch.from_numpy(pts).cuda(), out)
        torch.cuda.synchronize()
        gpu = out.cpu().numpy().astype(np.float64)
        ref, bnd, parts = plain.rounding_bound(pts.astype(np.float64) - centre, terms=True)
        fl = sum(int(np.sum((gpu - r >= MARGIN) != (ref - r >= MARGIN))) for r in radii)
        err, _ = plain_errors([np.abs(gpu - ref)], [bnd], [parts[:, 3]], fl,
                              len(pts) * len(radii), f"trained network, scene {k}")
        # the worst-case first-order bound (every rounding aligned) is loose,
        # a few centimetres; the errors are sums of many independent
        # roundings and stay within 6 deviations (asserted above): under half
        # the 2 cm margin, with few margin decisions changed by rounding
        assert err.max() < 0.5 * MARGIN
        assert fl <= 0.01 * len(pts) * len(radii)
    # restore the random weights the other tests use
    for k in range(2):
        ss.nsdf_set_weights(k, B, Ps[k])
