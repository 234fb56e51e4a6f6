"""Neural SDF on the tensor cores against the FP64 oracle MLP.

The oracle runs the same network with the weights the kernels use (BF16
values widened) and, in its BF16-operand mode, rounds features and hidden
activations to BF16 where the kernels do; its sums are FP64.  Against the
plain FP64 network (nothing but the weights rounded) the kernels must stay
within the oracle's first-order bound of that rounding.
"""
import numpy as np
import pytest

import oracle as O
from paper_2306_07552_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def split_params(P):
    """Flat C-ABI parameter vector -> (Ws, bs) per layer."""
    dims = [64, 128, 128, 128, 128, 1]
    Ws, bs, o = [], [], 0
    for l in range(5):
        n_in, n_out = dims[l], dims[l + 1]
        Ws.append(P[o:o + n_in * n_out].reshape(n_out, n_in).astype(np.float64))
        o += n_in * n_out
        bs.append(P[o:o + n_out].astype(np.float64))
        o += n_out
    assert o == len(P)
    return Ws, bs


@pytest.fixture(scope="module")
def nsdf_scene():
    from paper_2306_07552_b300 import build, gx
    build.build()
    scene = I.room_scene(1000, 2000)
    ss = gx.SceneSet([scene])
    B = I.fourier_matrix(7)
    P = I.nsdf_init(7)
    rng = np.random.default_rng(3)
    P = P + rng.normal(0, 0.05, P.shape).astype(np.float32)   # non-zero biases too
    ss.nsdf_set_weights(0, B, P)
    yield gx, scene, ss
    ss.close()


def _points(scene, n, seed):
    rng = np.random.default_rng(seed)
    lo = scene.grid_origin.astype(np.float64)
    hi = lo + (scene.grid_dims - 1) * scene.grid_h
    return rng.uniform(lo, hi, (n, 3)).astype(np.float32)


def test_query_matches_oracle(nsdf_scene):
    gx, scene, ss = nsdf_scene
    Bq, Pq, centre = ss.nsdf_get_weights(0)
    # the stored weights are the given ones rounded to BF16 (W1..W4) or exact
    Ws, bs = split_params(Pq.astype(np.float64))
    n = 3 * 128 + 77                                  # several tiles + a ragged tail
    pts = _points(scene, n, 11)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    ss.nsdf_query(0, torch.from_numpy(pts).cuda(), out)
    torch.cuda.synchronize()
    gpu = out.cpu().numpy().astype(np.float64)
    rel = pts.astype(np.float64) - centre.astype(np.float64)
    ref = O.MLP64(Bq, Ws, bs, bf16_operands=True).forward(rel)
    exact = O.MLP64(Bq, Ws, bs, bf16_operands=False).forward(rel)
    err = np.abs(gpu - ref)
    print(f"max |gpu - oracle(bf16 operands)| = {err.max():.3e}, p99 {np.quantile(err, .99):.3e}, "
          f"median {np.median(err):.3e}; vs unrounded FP64: max {np.abs(gpu - exact).max():.3e}; "
          f"output scale {np.abs(ref).mean():.3e}")
    assert np.all(np.isfinite(gpu))
    assert np.median(err) < 1e-5 * (1 + np.abs(ref).mean())
    # against the plain FP64 network (BF16 weights, nothing else rounded):
    # within the first-order rounding bound of the BF16-operand kernel and
    # within 6 standard deviations of independent roundings
    plain, bnd, parts = O.MLP64(Bq, Ws, bs).rounding_bound(rel, terms=True)
    perr = np.abs(gpu - plain)
    z = perr / parts[:, 3]
    print(f"vs plain FP64: max {perr.max():.3e}, bound median {np.median(bnd):.3e}, "
          f"err/bound max {(perr / bnd).max():.3f}, deviations rms "
          f"{np.sqrt(np.mean(z ** 2)):.2f} max {z.max():.2f}")
    assert np.all(perr <= bnd)
    assert z.max() <= 6.0


def test_query_is_deterministic(nsdf_scene):
    """Same points, same bits: several launches, and the points in another
    order (tiles are independent, so a row's value cannot depend on them)."""
    gx, scene, ss = nsdf_scene
    n = 5 * 128 + 3
    pts = torch.from_numpy(_points(scene, n, 12)).cuda()
    outs = []
    for _ in range(3):
        o = torch.empty(n, dtype=torch.float32, device="cuda")
        ss.nsdf_query(0, pts, o)
        outs.append(o)
    perm = torch.randperm(n, generator=torch.Generator().manual_seed(0)).cuda()
    o = torch.empty(n, dtype=torch.float32, device="cuda")
    ss.nsdf_query(0, pts[perm].contiguous(), o)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    assert torch.equal(outs[0][perm], o)


def test_weights_round_trip_bf16(nsdf_scene):
    gx, scene, ss = nsdf_scene
    B, P, c = ss.nsdf_get_weights(0)
    P0 = I.nsdf_init(7) + np.random.default_rng(3).normal(0, 0.05, P.shape).astype(np.float32)
    Ws0, bs0 = split_params(P0)
    Ws, bs = split_params(P)
    for l in range(4):
        # W1..W4 are the nearest BF16 values: within half a BF16 ulp
        assert np.all(np.abs(Ws[l] - Ws0[l]) <= np.abs(Ws0[l]) * 2.0 ** -8 + 1e-30)
        assert np.array_equal(bs[l], bs0[l])
    assert np.array_equal(Ws[4], Ws0[4]) and np.array_equal(bs[4], bs0[4])
    assert np.array_equal(B, I.fourier_matrix(7))
