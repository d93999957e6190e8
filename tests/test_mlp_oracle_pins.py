"""Pins for the FP64 reference of the proposal network and its features.

The backward formulas are pinned by central finite differences of the FP64
loss (plain network, no bf16 rounding); the bf16 rounding helper against
exactly representable values and ties; the patch features against closed
forms on a linear ramp, where the interpolated gradient is the field's."""
import math

import numpy as np
import pytest

from oracle import mlp


def _rand_params(seed, scale=0.2):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, scale, mlp.N_PARAMS)
    p[~mlp.trainable_mask()] = 0.0
    return p


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = _rand_params(1)
    X = np.zeros((6, mlp.K_PAD))
    X[:, :mlp.K_IN] = rng.normal(0, 1, (6, mlp.K_IN))
    T = rng.normal(0, 1.5, (6, 4))
    T[2, 3] = np.nan                          # an ignored row
    loss, g = mlp.loss_and_grads(p, X, T, bf16=False)
    idx = np.concatenate([rng.choice(np.arange(mlp.OFF_W1, mlp.OFF_B1)[mlp.trainable_mask()[mlp.OFF_W1:mlp.OFF_B1]], 12),
                          rng.choice(np.arange(mlp.OFF_B1, mlp.OFF_W2), 4),
                          rng.choice(np.arange(mlp.OFF_W2, mlp.OFF_B2), 8),
                          rng.choice(np.arange(mlp.OFF_B2, mlp.OFF_W3), 4),
                          np.arange(mlp.OFF_W3, mlp.OFF_W3 + 4 * mlp.H, 37),
                          np.arange(mlp.OFF_B3, mlp.OFF_B3 + 4)])
    eps = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (mlp.loss_and_grads(pp, X, T, bf16=False)[0] - mlp.loss_and_grads(pm, X, T, bf16=False)[0]) / (2 * eps)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-8), i


def test_huber_regions():
    p = np.zeros(mlp.N_PARAMS)
    p[mlp.OFF_B3:mlp.OFF_B3 + 4] = [0.5, -3.0, 0.0, 2.0]
    X = np.zeros((1, mlp.K_PAD))
    T = np.zeros((1, 4))
    loss, g = mlp.loss_and_grads(p, X, T, bf16=False)
    assert loss == pytest.approx(0.5 * 0.25 + (3.0 - 0.5) + 0.0 + (2.0 - 0.5))
    np.testing.assert_allclose(g[mlp.OFF_B3:mlp.OFF_B3 + 4], [0.5, -1.0, 0.0, 1.0])


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 1e-3])
    r = mlp.bf16_round(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # tie -> even
    assert r[2] == 1.0 + 2 ** -7            # representable
    assert r[3] == 1.0 + 2 ** -6            # tie -> even (up)
    assert r[4] == -2.5
    assert abs(r[5] - 1e-3) <= 2 ** -9 * 1e-3


def test_features_on_a_linear_ramp():
    # D_r = a + g . r, D_e = D_r - delta: the gradient magnitude is |g| everywhere
    # and channel 0 at patch voxel p is (D_e(p) - D_r(v)) / dD = (g . (p - v) - delta) / dD.
    shape, sp = (9, 10, 11), (2.0, 1.25, 1.5)
    grad = np.array([0.004, 0.009, -0.006])
    coords = np.meshgrid(*[np.arange(n) * h for n, h in zip(shape, sp)], indexing="ij")
    ref = 0.6 + sum(g_ * c for g_, c in zip(grad, coords))
    ev = ref - 0.0125
    dd, dta = 0.02, 3.0
    v = np.ravel_multi_index((4, 5, 5), shape)
    f = mlp.features(ref, ev, sp, dd, dta, [v], dose_norm=1.0)[0]
    gm = math.sqrt(float((grad ** 2).sum())) * dta / dd
    np.testing.assert_allclose(f[125:250], gm, rtol=1e-12)
    np.testing.assert_allclose(f[250:375], gm, rtol=1e-12)
    for pi in (0, 62, 124):
        o = np.array([pi // 25 - 2, (pi // 5) % 5 - 2, pi % 5 - 2])      # z, y, x
        want = (float((grad * o * np.array(sp)).sum()) - 0.0125) / dd
        assert f[pi] == pytest.approx(want, rel=1e-10)
    assert np.all(f[375:] == 0)
