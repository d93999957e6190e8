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


def _corner_features(field, ev, sp, dd, dta, corner):
    v = np.ravel_multi_index(corner, field.shape)
    return mlp.features(field, ev, sp, dd, dta, [v], dose_norm=1.0)[0]


def test_edge_gradient_is_one_sided_on_a_quadratic_field():
    # D = c x^2 along x only (array axis 2).  Central differences give 2 c x
    # exactly inside; the one-sided differences at the two grid edges give
    # c h (first node) and c (2n - 3) h (last node).  A patch around the
    # voxel at the corner x = 0 sees x = 0, 1, 2 (positions -2, -1 are outside
    # the grid); a patch around the last node sees n-3 .. n-1.
    shape, sp = (6, 7, 9), (1.5, 2.0, 1.25)
    h, c, n = sp[2], 0.003, shape[2]
    x = np.arange(n) * h
    ref = np.broadcast_to(0.2 + c * x * x, shape).copy()
    ev = ref.copy()
    dd, dta = 0.02, 2.5
    scale = dta / dd                                   # |grad| * dta / dD with dD = dd * 1
    want = {0: c * h, n - 1: c * (2 * n - 3) * h}
    want.update({i: 2 * c * i * h for i in range(1, n - 1)})
    for corner_x in (0, n - 1):
        f = _corner_features(ref, ev, sp, dd, dta, (3, 3, corner_x))
        for pi in range(125):
            ox, oy, oz = pi % 5 - 2, (pi // 5) % 5 - 2, pi // 25 - 2
            px = corner_x + ox
            if not 0 <= px < n:
                continue
            assert 0 <= 3 + oy < shape[1] and 0 <= 3 + oz < shape[0]
            g = want[px] * scale
            assert f[125 + pi] == pytest.approx(g, rel=1e-12), (corner_x, pi)
            assert f[250 + pi] == pytest.approx(g, rel=1e-12), (corner_x, pi)


def test_patch_entries_outside_the_grid_are_zero():
    # Voxel at the grid corner (0, 0, 0): of the 5^3 patch positions only the
    # 3^3 with every offset >= 0 lie inside the grid; the other 98 are zero in
    # all three channels, while the inside ones are not (a ramp with a dose
    # offset keeps every inside value away from zero).
    shape, sp = (5, 6, 7), (2.0, 2.0, 2.0)
    coords = np.meshgrid(*[np.arange(k) * h for k, h in zip(shape, sp)], indexing="ij")
    ref = 0.5 + 0.01 * coords[0] + 0.02 * coords[1] + 0.015 * coords[2]
    ev = ref + 0.004
    f = _corner_features(ref, ev, sp, 0.02, 3.0, (0, 0, 0))
    inside = np.zeros(125, dtype=bool)
    for pi in range(125):
        ox, oy, oz = pi % 5 - 2, (pi // 5) % 5 - 2, pi // 25 - 2
        inside[pi] = ox >= 0 and oy >= 0 and oz >= 0
    assert inside.sum() == 27
    for ch in range(3):
        blk = f[125 * ch:125 * (ch + 1)]
        assert np.all(blk[~inside] == 0.0), ch
        assert np.all(blk[inside] != 0.0), ch
    # the dose channel inside: (D_e(p) - D_r(v)) / dD, v at the origin
    p_idx = [pi for pi in range(125) if inside[pi]]
    for pi in p_idx:
        o = (pi // 25 - 2, (pi // 5) % 5 - 2, pi % 5 - 2)             # z, y, x
        want = (ev[o] - ref[0, 0, 0]) / 0.02                       # dD = 0.02 * D_norm, D_norm = 1
        assert f[pi] == pytest.approx(want, rel=1e-12)


def test_features_are_clamped():
    # Channel 0 saturates at +-16 (a dose difference of +-0.5 at dD = 0.01);
    # channels 1 and 2 saturate at 32 (slope 0.05 / mm * 3 mm / 0.003 = 50).
    shape, sp = (5, 5, 6), (1.0, 1.0, 1.0)
    x = np.arange(shape[2]) * sp[2]
    ref = np.broadcast_to(0.4 + 0.05 * x, shape).copy()
    for delta, want0 in ((0.5, 16.0), (-0.5, -16.0)):
        ev = ref + delta
        f = _corner_features(ref, ev, sp, 0.01, 3.0, (2, 2, 2))
        assert np.all(f[:125] == want0)                  # every patch voxel is inside
    f = _corner_features(ref, ref.copy(), sp, 0.003, 3.0, (2, 2, 2))
    assert np.all(f[125:375] == 32.0)
    # just below the clamp the value passes through unchanged
    f = _corner_features(ref, ref.copy(), sp, 0.006, 3.0, (2, 2, 2))
    np.testing.assert_allclose(f[125:375], 0.05 * 3.0 / 0.006, rtol=1e-12)


def test_2d_features_use_the_first_25_of_each_channel():
    # A 2D grid uses the 5x5 patch at patch indices 0..24 of each channel
    # (x fastest, then y); indices 25..124 of every channel stay zero.
    shape, sp = (9, 8), (1.5, 1.0)
    yy, xx = np.meshgrid(np.arange(shape[0]) * sp[0], np.arange(shape[1]) * sp[1], indexing="ij")
    gy, gx = 0.004, -0.007
    ref = 0.6 + gy * yy + gx * xx
    ev = ref - 0.01
    dd, dta = 0.02, 3.0
    v = np.ravel_multi_index((4, 4), shape)
    f = mlp.features(ref, ev, sp, dd, dta, [v], dose_norm=1.0)[0]
    gm = math.hypot(gy, gx) * dta / dd
    for ch in range(3):
        blk = f[125 * ch:125 * (ch + 1)]
        assert np.all(blk[25:] == 0.0), ch
    np.testing.assert_allclose(f[125:150], gm, rtol=1e-12)
    np.testing.assert_allclose(f[250:275], gm, rtol=1e-12)
    for pi in range(25):
        ox, oy = pi % 5 - 2, pi // 5 - 2
        want = (gy * oy * sp[0] + gx * ox * sp[1] - 0.01) / dd
        assert f[pi] == pytest.approx(want, rel=1e-10, abs=1e-12)
