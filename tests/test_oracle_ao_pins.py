"""Pins of the learned-AO oracle (aomlp.c, aotrain.py) to facts other than itself.

The surrogate is not in the paper; what fixes it is the model definition
(reading L1): bfloat16 rounding (checked against PyTorch's conversion),
the feature layout (hand-built grids with closed-form inputs), networks whose
every intermediate is exact (checked against a float64 PyTorch evaluation),
one network that shows where the neighbourhood sum is rounded, the chain rule
(central finite differences) and Adam (checked against torch.optim.Adam).
None needs a GPU.
"""
import math

import numpy as np
import pytest
import torch

from oracle import aotrain as T


def _torch_bf16(x):
    return torch.tensor(np.asarray(x, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def test_bf16_rounding_matches_torch(orc):
    rng = np.random.default_rng(1)
    vals = rng.standard_normal(4000).astype(np.float32) * np.float32(10.0) ** rng.integers(-6, 6, 4000)
    # exact ties between two bfloat16 neighbours (even and odd last kept bit)
    base = np.array([1.0, 1.0078125, 3.0, -5.5, 1e-3], np.float32)
    ties = (base.view(np.uint32) + np.uint32(0x8000)).view(np.float32)
    vals = np.concatenate([vals, ties, np.array([0.0, -0.0, 1e30, -1e-30], np.float32)])
    want = _torch_bf16(vals)
    assert np.array_equal(T.bf16(vals), want)
    assert np.array_equal(np.array([orc.bf16(float(v)) for v in vals]), want)


def test_tangent_sign_and_zero(orc):
    assert np.allclose(orc.ao_tangent([0, 0, 0], [0, -3, 4]), [0.0, 0.6, -0.8], atol=1e-15)
    assert np.allclose(orc.ao_tangent([1, 1, 1], [-1, 1, 1]), [1.0, 0.0, 0.0], atol=1e-15)
    assert np.array_equal(orc.ao_tangent([1, 2, 3], [1, 2, 3]), [0.0, 0.0, 0.0])


def _dens_levels(dims0, fill=0.0):
    d0 = np.full(dims0[::-1], fill)
    d1 = np.full([(n + 1) // 2 for n in dims0][::-1], fill)
    d2 = np.full([(n + 3) // 4 for n in dims0][::-1], fill)
    return [d0, d1, d2]


def test_features_single_cell_per_level_closed_form(orc):
    """Grid 12 x 10 x 9 (x, y, z), hit voxel (5, 3, 6) at p = (5.25, 3.5, 6.75).
    One non-empty cell per level: level 0 (6, 4, 5) is the neighbour
    (1, 1, -1) -> slot (dz+2)*25 + (dy+2)*5 + (dx+2) = 43; level 1: the voxel
    lies in cell (2, 1, 3) and (0, 2, 4) is (-2, 1, 1) -> 75 + 15 + 0 = 90;
    level 2: cell (1, 0, 1) and (1, 0, 1) itself -> slot 62. Input value
    log1p(8 dens / 8^l). Offsets: p / 2^l - floor(v / 2^l) - 1/2."""
    d = _dens_levels((12, 10, 9))
    d[0][5, 4, 6] = 0.5
    d[1][4, 2, 0] = 3.0
    d[2][1, 0, 1] = 20.0
    lod = orc.HandLod(d)
    v = (5, 3, 6)
    vox = v[0] + 12 * (v[1] + 10 * v[2])
    t, n, p = [0.6, 0.0, -0.8], [0.0, 1.0, 0.0], [5.25, 3.5, 6.75]
    x = orc.ao_features(lod, vox, t, n, p)
    want = np.zeros(400)
    want[0:3], want[3:6] = t, n
    want[6:9] = [0.25 - 0.5, 0.5 - 0.5, 0.75 - 0.5]
    want[9:12] = [5.25 / 2 - 2 - 0.5, 3.5 / 2 - 1 - 0.5, 6.75 / 2 - 3 - 0.5]
    want[12:15] = [5.25 / 4 - 1 - 0.5, 3.5 / 4 - 0 - 0.5, 6.75 / 4 - 1 - 0.5]
    want[16 + 43] = math.log1p(8 * 0.5)
    want[16 + 125 + 90] = math.log1p(8 * 3.0 / 8)
    want[16 + 250 + 62] = math.log1p(8 * 20.0 / 64)
    assert np.allclose(x, want, rtol=0, atol=1e-15)
    assert np.count_nonzero(x[16:]) == 3


def test_features_grid_corner_zero_outside(orc):
    """Uniform density; at the corner voxel only offsets 0..2 on each axis are
    inside at every level: 27 non-zero slots per level, dx, dy, dz >= 0."""
    d = _dens_levels((20, 20, 20), 1.0)
    lod = orc.HandLod(d)
    x = orc.ao_features(lod, 0, [0, 0, 1.0], [1.0, 0, 0], [0.5, 0.5, 0.5])
    for l in range(3):
        nb = x[16 + 125 * l:16 + 125 * (l + 1)].reshape(5, 5, 5)     # [dz][dy][dx]
        assert np.all(nb[2:, 2:, 2:] == math.log1p(8.0 / 8 ** l))
        nb = nb.copy()
        nb[2:, 2:, 2:] = 0.0
        assert not nb.any()
    assert np.all(x[391:] == 0.0) and x[15] == 0.0
    with pytest.raises(ValueError):
        orc.ao_features(orc.HandLod(d[:2]), 0, [0, 0, 1.0], [1.0, 0, 0], [0.5, 0.5, 0.5])


def _params():
    return np.zeros(T.NPARAM, np.float32)


def test_mlp_zero_weights_is_sigmoid_of_output_bias(orc):
    p = _params()
    p[T.OB4] = 0.75
    x = np.random.default_rng(2).standard_normal(400)
    assert orc.ao_mlp(p, x) == 1.0 / (1.0 + math.exp(-0.75))


def _sparse(rng, rows, cols, nnz, scale):
    w = np.zeros((rows, cols))
    for r in range(rows):
        w[r, rng.choice(cols, nnz, replace=False)] = rng.choice([-1.0, 1.0], nnz) * scale
    return w


def test_mlp_exact_network_matches_torch(orc):
    """Sparse weights in {-1, 0, 1} times powers of two, inputs in {0, 1/2, 1}:
    every sum and activation is a short binary fraction, exact in bfloat16, so
    all roundings are identities and the model equals a float64 PyTorch MLP."""
    rng = np.random.default_rng(3)
    p = _params()
    p[T.OW1:T.OB1] = _sparse(rng, T.NH, T.NIN, 8, 1.0).reshape(-1)
    p[T.OW1:T.OB1].reshape(T.NH, T.NIN)[:, 15] = 0.0
    p[T.OW1:T.OB1].reshape(T.NH, T.NIN)[:, 391:] = 0.0
    p[T.OB1:T.OW2] = rng.integers(-2, 3, T.NH) / 2.0
    p[T.OW2:T.OB2] = _sparse(rng, T.NH, T.NH, 4, 1 / 8).reshape(-1)
    p[T.OB2:T.OW3] = rng.integers(-2, 3, T.NH) / 16.0
    p[T.OW3:T.OB3] = _sparse(rng, T.NH, T.NH, 4, 1 / 4).reshape(-1)
    p[T.OB3:T.OW4] = rng.integers(-2, 3, T.NH) / 64.0
    p[T.OW4:T.OB4] = _sparse(rng, 1, T.NH, 8, 1 / 2).reshape(-1)
    p[T.OB4] = 0.25
    x = np.zeros(400)
    x[:15] = rng.integers(-2, 3, 15) / 2.0
    x[16:391] = rng.integers(0, 3, 375) / 2.0
    W1, b1, W2, b2, W3, b3, W4, b4 = [torch.tensor(np.asarray(a, np.float64)) for a in T.unpack(p)]
    h = torch.tensor(x)
    h = torch.relu(torch.nn.functional.linear(h, W1, b1))
    h = torch.relu(torch.nn.functional.linear(h, W2, b2))
    h = torch.relu(torch.nn.functional.linear(h, W3, b3))
    want = torch.sigmoid(h @ W4 + b4).item()
    # the exactness premise: every intermediate is a bfloat16 value, and not all are zero
    f = T.forward(p, x[None, :], rnd=False)
    for k in ("Z1", "Z2", "Z3"):
        assert np.array_equal(T.bf16(f[k]), f[k]) and (f[k] > 0).sum() >= 8
    assert abs(want - 1.0 / (1.0 + math.exp(-0.25))) > 1e-3
    assert orc.ao_mlp(p, x) == pytest.approx(want, rel=1e-15)
    assert T.forward(p, x[None, :])["y"][0] == pytest.approx(want, rel=1e-15)


def test_mlp_rounds_the_neighbourhood_sum_before_the_direction(orc):
    """Per-voxel inputs 256 and 1 with unit weights sum to 257, which is
    stored as bfloat16 256; adding the per-hit part 0.5 gives 256.5 -> 256.
    Without that rounding the unit would be bfloat16(257.5) = 258. Then
    h2 = h1 / 256, h3 = h2, output = sigmoid(h3 - 1): 1/2 exactly (the other
    order would give sigmoid(2/256))."""
    p = _params()
    p[T.OW1 + 0] = 1.0          # W1[0][0] (per hit)
    p[T.OW1 + 16] = 1.0         # W1[0][16] (per voxel)
    p[T.OW1 + 17] = 1.0         # W1[0][17]
    p[T.OW2] = 1.0 / 256.0      # W2[0][0]
    p[T.OW3] = 1.0              # W3[0][0]
    p[T.OW4] = 1.0              # W4[0]
    p[T.OB4] = -1.0
    x = np.zeros(400)
    x[0], x[16], x[17] = 0.5, 256.0, 1.0
    assert orc.ao_mlp(p, x) == 0.5


def test_mlp_rounds_each_hidden_activation(orc):
    """One path through layers 2 and 3: h1 = 1; z2 = 1 + 2^-9 -> h2 = 1;
    z3 = (1 + 2^-7) h2 + 0.003 = 1.0108... -> h3 = 1 + 2^-7; output =
    sigmoid(h3 - 1) = sigmoid(2^-7). Keeping z2 unrounded would give
    h3 = 1 + 2^-6; keeping z3 unrounded, sigmoid(0.0108...)."""
    p = _params()
    p[T.OW1 + 20] = 1.0
    p[T.OW2] = 1.0
    p[T.OB2] = 2.0 ** -9
    p[T.OW3] = 1.0 + 2.0 ** -7
    p[T.OB3] = 0.003
    p[T.OW4] = 1.0
    p[T.OB4] = -1.0
    x = np.zeros(400)
    x[20] = 1.0
    want = 1.0 / (1.0 + math.exp(-(2.0 ** -7)))
    assert orc.ao_mlp(p, x) == want
    assert T.forward(p, x[None, :])["y"][0] == pytest.approx(want, rel=1e-15)


def test_training_gradient_is_the_derivative(orc):
    """With the roundings off, the analytic gradient equals central finite
    differences of the float64 loss, in every parameter block."""
    rng = np.random.default_rng(4)
    p = (rng.standard_normal(T.NPARAM) * 0.2).astype(np.float64)
    X = rng.standard_normal((12, 400))
    t = rng.uniform(0.0, 1.0, 12)
    _, g = T.loss_and_grad(p, X, t, rnd=False)
    blocks = [(T.OW1, T.OB1), (T.OB1, T.OW2), (T.OW2, T.OB2), (T.OB2, T.OW3), (T.OW3, T.OB3),
              (T.OB3, T.OW4), (T.OW4, T.OB4), (T.OB4, T.NPARAM)]
    h = 1e-6
    for lo, hi in blocks:
        for i in rng.choice(np.arange(lo, hi), size=min(6, hi - lo), replace=False):
            pp, pm = p.copy(), p.copy()
            pp[i] += h
            pm[i] -= h
            fd = (T.loss(pp, X, t, rnd=False) - T.loss(pm, X, t, rnd=False)) / (2 * h)
            assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-10), (lo, i)


class _Q(torch.autograd.Function):
    """bfloat16 rounding forward, identity backward (straight-through)."""

    @staticmethod
    def forward(ctx, x):
        return x.to(torch.float32).to(torch.bfloat16).to(torch.float64)

    @staticmethod
    def backward(ctx, g):
        return g


class _QG(torch.autograd.Function):
    """Identity forward, bfloat16 rounding of the gradient backward."""

    @staticmethod
    def forward(ctx, x):
        return x.clone()

    @staticmethod
    def backward(ctx, g):
        return g.to(torch.float32).to(torch.bfloat16).to(torch.float64)


def test_rounded_gradient_matches_torch_autograd():
    """The bfloat16 training step written as a PyTorch float64 graph: rounded
    operands (straight-through), hidden-layer gradients rounded where they
    enter the products (and not for the biases); torch's autograd then gives
    the gradient the oracle computes by hand."""
    rng = np.random.default_rng(5)
    p = rng.standard_normal(T.NPARAM) * 0.1
    X = np.abs(rng.standard_normal((32, 400)))
    t = rng.uniform(0.0, 1.0, 32)
    tp = torch.tensor(p, requires_grad=True)
    W1, b1 = tp[T.OW1:T.OB1].reshape(64, 400), tp[T.OB1:T.OW2]
    W2, b2 = tp[T.OW2:T.OB2].reshape(64, 64), tp[T.OB2:T.OW3]
    W3, b3 = tp[T.OW3:T.OB3].reshape(64, 64), tp[T.OB3:T.OW4]
    W4, b4 = tp[T.OW4:T.OB4], tp[T.OB4]
    q, qg = _Q.apply, _QG.apply
    h = q(torch.tensor(X))
    for W, b in ((W1, b1), (W2, b2), (W3, b3)):
        h = q(torch.relu(qg(h @ q(W).T) + b))
    y = torch.sigmoid(h @ q(W4) + b4)
    loss = torch.mean((y - torch.tensor(t)) ** 2)
    loss.backward()
    l_orc, g_orc = T.loss_and_grad(p, X, t, rnd=True)
    assert l_orc == pytest.approx(loss.item(), rel=1e-13)
    g_t = tp.grad.numpy()
    assert np.allclose(g_orc, g_t, rtol=1e-10, atol=1e-14 * np.abs(g_t).max())
    # and the rounding matters: the exact gradient differs
    _, g_exact = T.loss_and_grad(p, X, t, rnd=False)
    assert not np.allclose(g_exact, g_t, rtol=1e-6, atol=0)


def test_adam_matches_torch():
    rng = np.random.default_rng(6)
    p0 = rng.standard_normal(50)
    tp = torch.tensor(p0.copy(), requires_grad=True)
    opt = torch.optim.Adam([tp], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for step in range(1, 5):
        g = rng.standard_normal(50)
        tp.grad = torch.tensor(g)
        opt.step()
        p, m, v = T.adam(p, g, m, v, step, 3e-3)
        assert np.allclose(p, tp.detach().numpy(), rtol=0, atol=1e-14)
