"""Pins the oracle's neural-SDF training pieces (the workload's learned part,
not in the paper) to facts that do not come from the oracle: a planar field
whose distance is known in closed form, acceptance rates that follow from the
geometry, Adam's published invariances (Kingma and Ba, ICLR 2015, Sec. 2.1)
and PyTorch's own BF16 rounding and autograd for the BF16-operand mode."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2306_07552_b300 import inputs as I

from test_oracle_pins import FLOOR, oracle_for, scene_from_boxes

BAND = 0.1


@pytest.fixture(scope="module")
def floor_oracle():
    # a floor slab (top y = 0) under a 2 x 2 x 2 m lattice from y = -0.5
    sc = scene_from_boxes([FLOOR], (-1, -0.5, -1), (1, 1.5, 1), h=0.05)
    return sc, oracle_for(sc)


def test_samples_lie_in_the_lattice_box_with_planar_labels(floor_oracle):
    sc, orc = floor_oracle
    P, d, t, nb = orc.nsdf_samples(seed=11, scene=3, idx=np.arange(400), band=BAND)
    lo = sc.grid_origin.astype(np.float64)
    hi = lo + (sc.grid_dims - 1) * np.float64(sc.grid_h)
    assert np.all(P >= lo) and np.all(P < hi)
    # the floor's distance field is d = y in this box (nearest face is the top)
    assert np.allclose(d, P[:, 1], atol=1e-12)
    assert np.all(t[0::2] == 0)                    # even samples: one uniform draw


def test_near_surface_half_accepts_inside_the_band(floor_oracle):
    _, orc = floor_oracle
    idx = np.arange(1, 1601, 2)
    P, d, t, nb = orc.nsdf_samples(seed=5, scene=0, idx=idx, band=BAND)
    acc = t < 63
    assert np.all(np.abs(d[acc]) < BAND)
    # P(|y| < 0.1) over a 2 m tall box is 0.1: draws until acceptance are
    # geometric with mean 10
    assert 8.5 < (t + 1).mean() < 11.5
    # accepted heights are uniform in (-0.1, 0.1)
    assert abs(P[acc, 1].mean()) < 0.01


def test_uniform_half_is_uniform(floor_oracle):
    _, orc = floor_oracle
    P, d, t, nb = orc.nsdf_samples(seed=7, scene=1, idx=np.arange(0, 4000, 2), band=BAND)
    # box y in [-0.5, 1.5): mean 0.5, a quarter below the floor
    assert abs(P[:, 1].mean() - 0.5) < 0.04
    assert abs((P[:, 1] < 0).mean() - 0.25) < 0.03
    assert abs(P[:, 0].mean()) < 0.04 and abs(P[:, 2].mean()) < 0.04


def test_samples_are_counter_based(floor_oracle):
    _, orc = floor_oracle
    a = orc.nsdf_samples(seed=9, scene=2, idx=[10, 11, 12])[0]
    b = orc.nsdf_samples(seed=9, scene=2, idx=[12, 11, 10])[0]
    assert np.array_equal(a, b[::-1])
    c = orc.nsdf_samples(seed=10, scene=2, idx=[10, 11, 12])[0]
    e = orc.nsdf_samples(seed=9, scene=4, idx=[10, 11, 12])[0]
    assert not np.allclose(a, c) and not np.allclose(a, e)


# ------------------------------------------------------------------ Adam

def test_adam_first_step_has_size_lr():
    g = np.array([3.0, -1e-3, 250.0, -7.0])
    p, m, v = O.adam_step(np.zeros(4), np.zeros(4), np.zeros(4), g, t=1, lr=0.01)
    assert np.allclose(p, -0.01 * np.sign(g), rtol=1e-4)


def test_adam_is_invariant_to_gradient_scale():
    rng = np.random.default_rng(0)
    p0 = rng.normal(size=8)
    state_a = (p0, np.zeros(8), np.zeros(8))
    state_b = (p0, np.zeros(8), np.zeros(8))
    for t in range(1, 20):
        g = rng.normal(size=8)
        state_a = O.adam_step(*state_a, g, t, 1e-3)
        state_b = O.adam_step(*state_b, 1000.0 * g, t, 1e-3)
    assert np.allclose(state_a[0], state_b[0], rtol=0, atol=1e-9)


def test_adam_constant_gradient_moves_lr_per_step():
    s = (np.zeros(3), np.zeros(3), np.zeros(3))
    g = np.array([0.5, -2.0, 1e-2])
    for t in range(1, 51):
        s = O.adam_step(*s, g, t, 1e-3)
    assert np.allclose(s[0], -50 * 1e-3 * np.sign(g), rtol=1e-5)


def test_adam_minimises_a_quadratic():
    a = np.array([1.0, 10.0, 0.1])
    s = (np.array([1.0, -1.0, 2.0]), np.zeros(3), np.zeros(3))
    for t in range(1, 3001):
        s = O.adam_step(*s, a * s[0], t, O.cosine_lr(0.05, t - 1, 3000))
    assert np.all(np.abs(s[0]) < 1e-2)


def test_cosine_schedule_end_points():
    assert O.cosine_lr(1e-3, 0, 100) == pytest.approx(1e-3)
    assert O.cosine_lr(1e-3, 50, 100) == pytest.approx(5e-4)
    assert O.cosine_lr(1e-3, 100, 100) == pytest.approx(0.0, abs=1e-18)
    lrs = [O.cosine_lr(1e-3, t, 100) for t in range(101)]
    assert all(b <= a for a, b in zip(lrs, lrs[1:]))


# ------------------------------------------------------ BF16 operand mode

def _bf16(x):
    return torch.as_tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64)


def test_bf16_operand_mode_matches_torch_rounding_and_autograd():
    """Forward and gradients of the BF16-operand mode against PyTorch: FP64
    arithmetic, PyTorch's BF16 rounding of features and hidden activations
    (straight-through in backward) and of each hidden layer's gradient."""
    rng = np.random.default_rng(3)
    F, widths = 6, (24, 20, 16)
    dims = [2 * F, *widths, 1]
    Ws = [rng.normal(0, 0.4, (dims[i + 1], dims[i])) for i in range(len(dims) - 1)]
    bs = [rng.normal(0, 0.1, dims[i + 1]) for i in range(len(dims) - 1)]
    B = rng.normal(0, 1, (F, 3))
    X = rng.uniform(-1, 1, (9, 3))
    y = rng.uniform(-0.3, 1.2, 9)
    m = O.MLP64(B, Ws, bs, bf16_operands=True)

    Wt = [torch.tensor(w, requires_grad=True) for w in Ws]
    bt = [torch.tensor(b, requires_grad=True) for b in bs]
    ph = 2 * math.pi * torch.tensor(X) @ torch.tensor(B).T
    h = torch.cat([torch.sin(ph), torch.cos(ph)], 1)
    h = h + (_bf16(h.detach()) - h).detach()
    for l in range(len(Ws)):
        z = h @ Wt[l].T + bt[l]
        if l == len(Ws) - 1:
            h = z
            break
        z.register_hook(lambda g: _bf16(g))
        a = torch.relu(z)
        h = a + (_bf16(a.detach()) - a).detach()
    pred = h[:, 0]
    assert np.allclose(m.forward(X), pred.detach().numpy(), rtol=0, atol=1e-12)
    t = torch.clamp(torch.tensor(y), -0.2, 1.0)
    loss_t = torch.abs(pred - t).mean()
    loss_t.backward()
    loss, gW, gb = m.loss_grad(X, y, -0.2, 1.0)
    assert loss == pytest.approx(loss_t.item(), abs=1e-13)
    for l in range(len(Ws)):
        assert np.allclose(gW[l], Wt[l].grad.numpy(), rtol=0, atol=1e-12)
        assert np.allclose(gb[l], bt[l].grad.numpy(), rtol=0, atol=1e-12)
    # rounding is really applied: the FP64 mode differs
    assert not np.allclose(O.MLP64(B, Ws, bs).forward(X), m.forward(X), rtol=0, atol=1e-9)


# ------------------------------------------- neural static test in the step

from test_oracle_pins import _act, _state  # noqa: E402

POST = [-0.5, 0.0, -0.1, -0.3, 1.0, 0.1]


def _post_oracle():
    sc = scene_from_boxes([FLOOR, POST], (-2, -0.3, -2), (2, 2.5, 2), h=0.02)
    return oracle_for(sc)


def test_candidate_spheres_are_the_proposed_pose():
    orc = _post_oracle()
    st = _state(orc, base=(0.2, 0.1, 0.3))
    c, r, act = orc.candidate_spheres(st, np.zeros(11, np.float32))
    n = len(I.fetch_like_robot().sphere_radius)
    assert np.allclose(c[:n], orc.sphere_centres([0.2, 0.1, 0.3], I.fetch_like_robot().q_rest),
                       atol=1e-12)
    assert np.array_equal(act[:n], np.ones(n, bool)) and not act[30]
    # a held object rides at T_ee c_off
    st = _state(orc, objs=[[0.5, 0.5, 0.0, 0.04]], held=0, c_off=(0.01, 0.02, 0.03))
    c, r, act = orc.candidate_spheres(st, np.zeros(11, np.float32))
    _, ee, _ = orc.fk((0, 0, 0), I.fetch_like_robot().q_rest)
    assert act[30] and r[30] == pytest.approx(0.04)
    R, t = ee[:9].reshape(3, 3), ee[9:]
    assert np.allclose(c[30], R @ [0.01, 0.02, 0.03] + t, atol=1e-12)


def test_neural_rule_reduces_to_grid_when_every_prediction_is_close():
    orc = _post_oracle()
    acts = I.make_actions(40, 1, "uniform", seed=4)[:, 0]
    sa, sb = _state(orc), _state(orc)
    for t in range(40):
        oa = orc.step(sa, acts[t])
        ob = orc.step_nsdf(sb, acts[t], np.full(31, -1e9), 0.02, 1e-3)
        assert (oa.contact_mask, oa.flags, oa.event) == (ob.contact_mask, ob.flags, ob.event)
        assert list(sa.base) == list(sb.base) and list(sa.q) == list(sb.q)


def test_neural_rule_trusts_a_large_clearance_but_not_the_box_edge():
    orc = _post_oracle()
    st = _state(orc)
    back = _act(fwd=-1.0, q1=0.5)           # drives a base sphere into the post
    assert orc.step(_state(orc), back).flags & 1
    out = orc.step_nsdf(st, back, np.full(31, 1e9), 0.02, 1e-3)
    assert out.contact_mask == 0 and not out.reverted
    # outside the lattice box stays contact whatever the prediction
    sc = scene_from_boxes([FLOOR], (-1, -0.3, -1), (1.0, 2.5, 1.0), h=0.05)
    o2 = oracle_for(sc)
    out = o2.step_nsdf(_state(o2, base=(0.45, 0, 0)), _act(fwd=1.0), np.full(31, 1e9), 0.02, 1e-3)
    assert out.reverted and out.flags & 1


def test_neural_rule_margin_is_inclusive_and_banded():
    orc = _post_oracle()
    back = _act(fwd=-1.0, q1=0.5)
    c, r, act = orc.candidate_spheres(_state(orc), back)
    hit = orc.step(_state(orc), back).contact_mask
    i = int(np.flatnonzero([(hit >> k) & 1 for k in range(31)])[0])
    d = np.full(31, 1e9)
    d[i] = r[i] + 0.02                       # clearance exactly the margin: trusted
    assert orc.step_nsdf(_state(orc), back, d, 0.02, 1e-3).contact_mask & (1 << i) == 0
    d[i] = np.nextafter(r[i] + 0.02, 0)      # just below: the grid decides
    out = orc.step_nsdf(_state(orc), back, d, 0.02, 1e-3)
    assert out.contact_mask & (1 << i) and out.near_band >= 1


# ---------------------------------------------------------------------------
# The rounding-error bound of the BF16-operand network (orc_mlp_rounding_bound)
# ---------------------------------------------------------------------------
UB, UF = 2.0 ** -8, 2.0 ** -24


def _random_net(seed, dims=(64, 128, 128, 128, 128, 1), bias=0.05):
    rng = np.random.default_rng(seed)
    B = rng.normal(0, 0.5, (dims[0] // 2, 3))
    Ws = [rng.normal(0, math.sqrt(2.0 / dims[l]), (dims[l + 1], dims[l]))
          for l in range(len(dims) - 1)]
    bs = [rng.normal(0, bias, dims[l + 1]) for l in range(len(dims) - 1)]
    return B, Ws, bs


def _numpy_forward(B, Ws, bs, x, bump=None):
    """Plain FP64 forward written out with numpy; bump(l, a) may perturb the
    operand a_l (layer l's input) before it is used."""
    ph = 2 * np.pi * (B @ x)
    a = np.concatenate([np.sin(ph), np.cos(ph)])
    for l, (W, b) in enumerate(zip(Ws, bs)):
        if bump is not None:
            a = bump(l, a)
        z = W @ a + b
        a = z if l == len(Ws) - 1 else np.maximum(z, 0.0)
    return float(a[0])


def test_rounding_bound_of_one_linear_layer_is_its_closed_form():
    # d = w . gamma(x) + b: the operand term is u_b sum |w_i gamma_i|, the
    # feature term feat_err (1 + u_b) sum |w_i|, the FP32 sum 2 K u_f sum
    # |w_i gamma_i| and the bias add u_f (|d| + |b|)
    B, Ws, bs = _random_net(3, dims=(16, 1))
    x = np.array([0.3, -1.2, 0.7])
    ph = 2 * np.pi * (B @ x)
    gam = np.concatenate([np.sin(ph), np.cos(ph)])
    w, b = Ws[0][0], bs[0][0]
    d = float(w @ gam + b)
    want = (UB * np.abs(w * gam).sum() + 4e-7 * (1 + UB) * np.abs(w).sum()
            + 2 * 16 * UF * np.abs(w * gam).sum() + UF * (abs(d) + abs(b)))
    out, bnd = O.MLP64(B, Ws, bs).rounding_bound(x[None], feat_err=4e-7)
    assert out[0] == pytest.approx(d, rel=1e-13)
    assert bnd[0] == pytest.approx(want, rel=1e-12)


def test_rounding_bound_operand_term_is_the_worst_case_first_order_shift():
    # perturb every operand a_{l,i} by h |a_{l,i}| in the direction that
    # raises d (the sign of a central finite difference): d moves by
    # h sum |dd/da_{l,i}| |a_{l,i}| to first order, which is the bound's
    # operand term with u_b = h (the FP32 sums add a few per cent on top)
    B, Ws, bs = _random_net(5)
    for x in (np.array([0.1, 0.9, -0.4]), np.array([-1.3, 0.2, 0.6])):
        base = _numpy_forward(B, Ws, bs, x)
        # operands of the plain network at x
        ops = []
        _numpy_forward(B, Ws, bs, x, bump=lambda l, a: (ops.append(a.copy()), a)[1])
        signs = []
        for l, a in enumerate(ops):
            s = np.zeros_like(a)
            for i in range(len(a)):
                if a[i] == 0.0:
                    continue
                e = 1e-6
                def up(k, v, i=i, l=l, e=e):
                    if k == l:
                        v = v.copy()
                        v[i] += e
                    return v
                def dn(k, v, i=i, l=l, e=e):
                    if k == l:
                        v = v.copy()
                        v[i] -= e
                    return v
                s[i] = np.sign(_numpy_forward(B, Ws, bs, x, up) - _numpy_forward(B, Ws, bs, x, dn))
            signs.append(s)
        h = 1e-5
        shifted = _numpy_forward(B, Ws, bs, x,
                                 bump=lambda l, a: a + h * signs[l] * np.abs(ops[l]))
        first_order = (shifted - base) / h * UB
        _, bnd, parts = O.MLP64(B, Ws, bs).rounding_bound(x[None], feat_err=0.0, terms=True)
        assert first_order > 0
        assert parts[0, 0] == pytest.approx(first_order, rel=2e-3)
        assert parts[0, 1] == 0.0 and 0 < parts[0, 2] < 0.1 * parts[0, 0]


def test_rounding_bound_covers_the_bf16_operand_mode():
    # the oracle's BF16-operand mode rounds exactly the operands the bound
    # accounts for (its sums stay FP64): it must lie within the bound, and
    # the bound must not be vacuous
    B, Ws, bs = _random_net(9)
    rng = np.random.default_rng(4)
    X = rng.uniform(-2, 2, (300, 3))
    plain, bnd, parts = O.MLP64(B, Ws, bs).rounding_bound(X, feat_err=0.0, terms=True)
    assert np.allclose(plain, O.MLP64(B, Ws, bs).forward(X), rtol=1e-12, atol=1e-12)
    rounded = O.MLP64(B, Ws, bs, bf16_operands=True).forward(X)
    err = np.abs(rounded - plain)
    ratio = err / bnd
    z = err / parts[:, 3]
    print(f"|bf16 - plain| / bound: median {np.median(ratio):.3f}, max {ratio.max():.3f}; "
          f"bound median {np.median(bnd):.2e}; in standard deviations: median "
          f"{np.median(z):.2f}, max {z.max():.2f}")
    assert np.all(err <= bnd)
    assert ratio.max() > 0.05
    # independent roundings: the errors spread like the stated deviation
    assert 0.3 < np.sqrt(np.mean(z ** 2)) < 3.0
