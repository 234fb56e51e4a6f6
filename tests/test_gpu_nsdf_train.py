"""Neural-SDF training on the tensor cores against the FP64 oracle: the sample
stream, the loss gradient (forward, backward-data and weight-gradient
kernels), the Adam update, and a short training run checked against the grid.

Gradient tolerance.  Both sides round the same operands to BF16 (features,
hidden activations, hidden-layer gradients); the kernels sum in FP32 where
the oracle sums in FP64, and their features (hardware sin and cos of a phase
reduced exactly to a fraction of a turn) are good to 4e-7.  A value within
that distance of a BF16 rounding boundary can round the other way: with BF16
steps of 2^-8 relative this happens to ~2e-4 of the features and ~3e-5 of the
hidden values, each time moving that operand by one step.
Over the ~5e5 rounded operands of a 1000-sample batch a few tens flip; the
per-layer gradient then differs by well under 1e-3 relative (L2), and the
loss (a mean of |prediction - label|) by ~1e-5 relative.  Asserted: 2e-3
per layer, mean elementwise error 1e-3 of the mean magnitude, loss 1e-4.
"""
import numpy as np
import pytest

import oracle as O
from paper_2306_07552_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAYER_SIZES = [(128, 64), (128, 128), (128, 128), (128, 128), (1, 128)]


def split_params(P):
    Ws, bs, o = [], [], 0
    for n_out, n_in in LAYER_SIZES:
        Ws.append(np.asarray(P[o:o + n_in * n_out], np.float64).reshape(n_out, n_in))
        o += n_in * n_out
        bs.append(np.asarray(P[o:o + n_out], np.float64))
        o += n_out
    assert o == len(P)
    return Ws, bs


def flat(Ws, bs):
    return np.concatenate([np.concatenate([w.ravel(), b]) for w, b in zip(Ws, bs)])


@pytest.fixture(scope="module")
def setup():
    from paper_2306_07552_b300 import build, gx
    build.build()
    scene = I.room_scene(1000, 2000)
    ss = gx.SceneSet([scene])
    B = I.fourier_matrix(7)
    P0 = I.nsdf_init(7)
    rng = np.random.default_rng(3)
    P0 = P0 + rng.normal(0, 0.02, P0.shape).astype(np.float32)
    ss.nsdf_set_weights(0, B, P0)
    orc = O.Oracle(I.fetch_like_robot(), scene, I.icosahedron(), I.object_colors(256))
    yield gx, scene, ss, orc, B, P0
    ss.close()


def test_samples_match_oracle(setup):
    gx, scene, ss, orc, B, P0 = setup
    for first, n in [(0, 3000), (4_000_000_001, 600)]:
        pts, d = ss.nsdf_samples(0, seed=123, first=first, n=n, near_band=0.1)
        torch.cuda.synchronize()
        P = pts.cpu().numpy().astype(np.float64)
        D = d.cpu().numpy().astype(np.float64)
        Po, Do, t, nb = orc.nsdf_samples(123, 0, np.arange(first, first + n), 0.1)
        clean = nb == 0
        dp = np.abs(P - Po).max(1)
        print(f"first={first}: {clean.sum()}/{n} without near-band draws, max |dp| "
              f"{dp[clean].max():.2e}, draws used mean {t.mean():.2f}")
        assert clean.mean() > 0.95
        assert np.all(dp[clean] < 1e-5)          # the same draw, FP32-rounded
        # every label is the grid distance at the GPU's own point
        ref = np.array([orc.grid_query(p)[1] for p in P])
        assert np.abs(D - ref).max() < 2e-5
        acc = (np.arange(first, first + n) % 2 == 1) & (t < 63)
        assert np.all(np.abs(D[acc & clean]) < 0.1)


@pytest.mark.parametrize("n", [300, 1000, 20000])
def test_gradient_matches_oracle(setup, n):
    gx, scene, ss, orc, B, P0 = setup
    ss.nsdf_set_weights(0, B, P0)
    pts, lab = ss.nsdf_samples(0, seed=5, first=0, n=n)
    g, loss = ss.nsdf_grad(0, pts, lab, -0.2, 1.0)
    torch.cuda.synchronize()
    g = g.cpu().numpy().astype(np.float64)
    Bq, Pq, c = ss.nsdf_get_weights(0)
    Ws, bs = split_params(Pq)
    m = O.MLP64(Bq, Ws, bs, bf16_operands=True)
    X = pts.cpu().numpy().astype(np.float64) - c.astype(np.float64)
    y = lab.cpu().numpy().astype(np.float64)
    loss_o, gW, gb = m.loss_grad(X, y, -0.2, 1.0)
    assert loss == pytest.approx(loss_o, rel=1e-4)
    ref = flat(gW, gb)
    o = 0
    for l, (n_out, n_in) in enumerate(LAYER_SIZES):
        k = n_out * n_in + n_out
        a, b = g[o:o + k], ref[o:o + k]
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        print(f"n={n} layer {l + 1}: |g| {np.linalg.norm(b):.3e} rel L2 err {rel:.2e} "
              f"max abs {np.abs(a - b).max():.2e}")
        assert rel < 2e-3
        assert np.mean(np.abs(a - b)) < 1e-3 * np.mean(np.abs(b)) + 1e-12
        o += k


def test_adam_steps_match_oracle(setup):
    gx, scene, ss, orc, B, P0 = setup
    lr, N, bs_ = 1e-3, 8192, 4096
    ss.nsdf_set_weights(0, B, P0)
    pts, lab = ss.nsdf_samples(0, seed=9, first=0, n=N)
    g0, _ = ss.nsdf_grad(0, pts[:bs_], lab[:bs_])
    g0 = g0.cpu().numpy().astype(np.float64)
    ss.nsdf_train(0, n_samples=N, batch=bs_, steps=1, lr=lr, seed=9)
    m1 = ss.nsdf_get_master(0).astype(np.float64)
    p1, mo, vo = O.adam_step(P0.astype(np.float64), 0.0, 0.0, g0, 1, O.cosine_lr(lr, 0, 1))
    e1 = np.abs(m1 - p1)
    print(f"one step: max |gpu - oracle| {e1.max():.2e}; moved {np.abs(m1 - P0).mean():.2e}")
    assert e1.max() < 1e-6
    assert np.abs(m1 - P0).mean() > 0.5 * lr          # Adam's first step has size ~lr
    # second step: gradient at the first step's weights on the second batch
    ss.nsdf_set_weights(0, B, p1.astype(np.float32))
    g1, _ = ss.nsdf_grad(0, pts[bs_:], lab[bs_:])
    g1 = g1.cpu().numpy().astype(np.float64)
    p1b, m_1, v_1 = O.adam_step(P0.astype(np.float64), 0.0, 0.0, g0, 1, O.cosine_lr(lr, 0, 2))
    p2, _, _ = O.adam_step(p1b, m_1, v_1, g1, 2, O.cosine_lr(lr, 1, 2))
    ss.nsdf_set_weights(0, B, P0)
    ss.nsdf_train(0, n_samples=N, batch=bs_, steps=2, lr=lr, seed=9)
    m2 = ss.nsdf_get_master(0).astype(np.float64)
    e2 = np.abs(m2 - p2)
    print(f"two steps: max |gpu - oracle| {e2.max():.2e}, median {np.median(e2):.2e}")
    assert np.median(e2) < 1e-7
    assert e2.max() < 2e-5


def test_training_fits_the_grid(setup):
    gx, scene, ss, orc, B, P0 = setup
    import time
    ss.nsdf_set_weights(0, B, I.nsdf_init(7))
    t0 = time.perf_counter()
    losses = ss.nsdf_train(0, n_samples=2_000_000, batch=65536, steps=400, lr=1e-3, seed=3)
    dt = time.perf_counter() - t0
    assert np.all(np.isfinite(losses))
    print(f"loss first {losses[0]:.4f} last {losses[-20:].mean():.4f}; 400 steps in {dt:.3f} s "
          f"(samples and workspace included)")
    assert losses[-20:].mean() < 0.5 * losses[0]
    # held out: a different sample stream, compared with the FP64 grid
    pts, _ = ss.nsdf_samples(0, seed=99, first=0, n=4000)
    out = torch.empty(4000, dtype=torch.float32, device="cuda")
    ss.nsdf_query(0, pts, out)
    torch.cuda.synchronize()
    P = pts.cpu().numpy().astype(np.float64)
    ref = np.clip(np.array([orc.grid_query(p)[1] for p in P]), -0.2, 1.0)
    err = np.abs(out.cpu().numpy() - ref)
    near = np.abs(ref) < 0.1
    print(f"held-out |d_hat - d_grid|: mean {err.mean():.4f} m, near-surface mean "
          f"{err[near].mean():.4f} m, p99 {np.quantile(err, 0.99):.4f} m")
    # far better than the best constant (the median label)
    assert err.mean() < 0.3 * np.abs(ref - np.median(ref)).mean()


def test_training_resumes_bit_exactly(setup):
    """A training run split in two, its FP32 master parameters and Adam
    moments checkpointed to the host in between and restored (as another
    process would), ends with the same parameters bit for bit as the run in
    one call, and the same per-step losses."""
    gx, scene, ss, orc, B, P0 = setup
    kw = dict(n_samples=300_000, batch=16384, steps=30, lr=1e-3, seed=5)
    ss.nsdf_set_weights(0, B, P0)
    full = ss.nsdf_train(0, **kw)
    m_full = ss.nsdf_get_master(0)
    ss.nsdf_set_weights(0, B, P0)
    l1, mom = ss.nsdf_train_steps(0, 0, 12, None, **kw)
    ckpt_params, ckpt_moments = ss.nsdf_get_master(0).copy(), mom.copy()
    # "another process": fresh weights, then the checkpoint restored
    ss.nsdf_set_weights(0, B, I.nsdf_init(11))
    ss.nsdf_set_weights(0, B, ckpt_params)
    l2, mom2 = ss.nsdf_train_steps(0, 12, 18, ckpt_moments, **kw)
    m_split = ss.nsdf_get_master(0)
    assert np.array_equal(m_split, m_full)
    assert np.array_equal(np.concatenate([l1, l2]), full)
    assert np.all(np.isfinite(mom2)) and np.any(mom2[1] > 0)
    with pytest.raises(gx.GxError):
        ss.nsdf_train_steps(0, 25, 10, None, **kw)        # past the run's 30 steps
    ss.nsdf_set_weights(0, B, P0)
