"""Pins for the FP64 reference of the learned indicator: gradients against central finite
differences, loss against the direct formula, Adam against a hand-evaluated first step,
feature invariances (affine rescaling of the state) and the harvest label definition."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1904_11147_gb300 import workloads as W


def _data(F=12, B=40, seed=0):
    rng = np.random.default_rng(seed)
    p = mlp.init_params(F, rng)
    for k in p:
        p[k] = p[k] + 0.05 * rng.normal(size=np.shape(p[k]))  # non-zero biases
    X = rng.normal(size=(B, F))
    y = (rng.uniform(size=B) < 0.3).astype(float)
    return p, X, y


def test_gradients_match_finite_differences():
    p, X, y = _data()
    g = mlp.grads(p, X, y, pw=3.0)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(p, X, y, 3.0)
            flat[idx] = old - h
            lm = mlp.loss(p, X, y, 3.0)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(g[k].reshape(-1)[idx] - fd) <= 1e-7 + 1e-6 * abs(fd), (k, idx)


def test_loss_matches_direct_formula():
    p, X, y = _data(seed=1)
    z, _ = mlp.forward(p, X)
    sig = 1 / (1 + np.exp(-z))
    ref = -np.mean(2.5 * y * np.log(sig) + (1 - y) * np.log(1 - sig))
    assert abs(mlp.loss(p, X, y, 2.5) - ref) < 1e-12


def test_adam_first_step_is_lr_times_sign():
    """With zero moments, the bias-corrected first Adam step is lr * g / (|g| + eps)."""
    p, X, y = _data(seed=2)
    g = mlp.grads(p, X, y, 1.0)
    p0 = {k: v.copy() for k, v in p.items()}
    mlp.adam_step(p, g, {}, lr=1e-3)
    for k in p:
        np.testing.assert_allclose(p0[k] - p[k], 1e-3 * g[k] / (np.abs(g[k]) + 1e-8), rtol=1e-10, atol=1e-15)


@pytest.mark.parametrize("dim,pde,N", [(1, 0, 2), (1, 1, 3), (2, 0, 2), (2, 1, 2)])
def test_features_are_invariant_to_affine_rescaling(dim, pde, N):
    """Adding a constant state and multiplying all modes by a positive factor leaves the
    features unchanged (means enter as differences, everything is divided by s_v)."""
    nx, ny = (20, 1) if dim == 1 else (7, 6)
    m = oracle.Mesh(dim, pde, N, nx, ny, bc=oracle.BC_OUTFLOW)
    rng = np.random.default_rng(3)
    u = W.random_modes(dim, pde, N, nx * ny, rng, smooth=0.1)
    f0 = mlp.features(m, u)
    assert f0.shape == (nx * ny, mlp.n_features(dim, pde, N))
    u2 = 3.0 * u
    u2[:, :, 0] += 1.7
    np.testing.assert_allclose(mlp.features(m, u2), f0, rtol=1e-10, atol=1e-12)
    # the mean differences and the cell's own higher modes are bounded by the scale s_v
    V = 1 if pde == 0 else (3 if dim == 1 else 4)
    NP = N + 1 if dim == 1 else (N + 1) * (N + 2) // 2
    nb = 2 if dim == 1 else 4
    per_v = nb + (nb + 1) * (NP - 1)
    for v in range(V):
        own = f0[:, v * per_v: v * per_v + nb + NP - 1]
        assert np.abs(own).max() <= 1.0 + 1e-12


def test_harvest_label_definition():
    """A step profile: the cell whose slope overshoots is flagged and changed (label 1);
    a flat region is neither flagged nor labelled."""
    K = 12
    m = oracle.Mesh(1, 0, 2, K, box=(0, 1, 0, 1), bc=oracle.BC_OUTFLOW)
    u = np.zeros((K, 1, 3))
    u[:6, 0, 0] = math.sqrt(2)
    u[5, 0, 1] = -0.4
    fl, lab, change = mlp.labels(m, u)
    assert fl[5] == 1 and lab[5] == 1
    assert fl[0] == 0 and lab[0] == 0
    assert np.all(lab <= fl) and change[5] > 1e-3 and change[0] == 0
