"""Element-wise error bounds for the proposal network's GPU kernels against
the FP64 reference (oracle/mlp.py), test infrastructure.

The GPU network rounds to bfloat16 at the same points as the reference
(weights, H1, H2, dZ2, dZ1) and accumulates products of bf16 operands in
FP32.  When both sides start from the same bf16 operands, an FP32 sum of K
products differs from the exact sum by at most ACC * sum |term| (a
probabilistic bound that holds for any summation order).  A bf16 rounding R (with or
without a ReLU in front) is monotone, so if the GPU's argument lies within e
of the reference's z, the GPU's rounded value lies between R(z - e) and
R(z + e): most elements then round to the same bf16 number as the reference
and carry no error at all, and the few whose argument sits within e of a
rounding boundary differ by one bf16 step.  A ReLU mask (backward) can only
differ where |z| <= e.  The functions below carry these per-element bounds
through the layers in FP64, from the reference's own intermediates, so that
every GPU output and gradient element is held to its own bound instead of to
a norm over a whole block.  Where that bound is loose (the first layer's
gradient, behind two rounding points of the backward pass), every row and
column of the block is also held to 2 % of its own norm.
"""
from __future__ import annotations

import numpy as np

from oracle import mlp

# FP32 accumulation error per unit of sum |term|: the probabilistic bound
# lambda sqrt(K) u on a sum of K rounded terms (u = 2^-24), with lambda ~ 8
# for the K <= 384 features and M <= 1024 rows summed here.  (The worst-case
# K u would put almost every bf16 value on a rounding boundary and bound
# nothing.)
ACC = 2.0 ** -16


def _r(v):
    return mlp.bf16_round(v)


def _relu_round_spread(z, e):
    """max |R(z') - R(z)| over |z' - z| <= e, R = bf16(relu(.))."""
    hi = _r(np.maximum(z + e, 0.0))
    lo = _r(np.maximum(z - e, 0.0))
    return hi - lo


def _masked_round_spread(g, e_g, z, e_z):
    """Bound on |bf16(g' [z' > 0]) - bf16(g [z > 0])| for |g' - g| <= e_g,
    |z' - z| <= e_z."""
    hi, lo = _r(g + e_g), _r(g - e_g)
    same_mask = np.abs(z) > e_z
    spread = hi - lo
    flip = np.maximum(np.abs(hi), np.abs(lo)) + spread
    return np.where(same_mask, np.where(z > 0, spread, 0.0), flip)


def forward_bounds(p, X):
    """Reference forward (bf16 rounding points) and per-element bounds on
    |gpu - ref| of z1, h1, z2, h2 and y.  X must hold bf16 values."""
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p)
    X = np.asarray(X, dtype=np.float64)
    f = mlp.forward(p, X, bf16=True)
    W1b, W2b, W3b = np.abs(_r(W1)), np.abs(_r(W2)), np.abs(_r(W3))
    e_z1 = ACC * (np.abs(X) @ W1b.T + np.abs(b1))
    e_h1 = _relu_round_spread(f["z1"], e_z1)
    e_z2 = e_h1 @ W2b.T + ACC * (np.abs(f["h1"]) @ W2b.T + np.abs(b2))
    e_h2 = _relu_round_spread(f["z2"], e_z2)
    e_y = (e_h2 @ W3b.T + ACC * (np.abs(f["h2"]) @ W3b.T + np.abs(b3)))[:, :mlp.OUT]
    return f, {"z1": e_z1, "h1": e_h1, "z2": e_z2, "h2": e_h2, "y": e_y}


def backward_bounds(p, X, T):
    """Reference loss and gradients with per-element bounds on the GPU's.
    Returns (loss, grads (flat), loss bound, grad bounds (flat))."""
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    M = X.shape[0]
    loss, g = mlp.loss_and_grads(p, X, T, bf16=True)
    f, e = forward_bounds(p, X)
    valid = np.isfinite(T[:, 3])
    res = np.where(valid[:, None], f["y"] - np.nan_to_num(T), 0.0)
    dy = np.where(np.abs(res) <= 1.0, res, np.sign(res)) / M
    e_dy = np.where(valid[:, None], e["y"], 0.0) / M                  # Huber' is 1-Lipschitz
    e_loss = float(e_dy.sum()) + ACC * abs(loss)
    ady, ah1, ah2, aX = np.abs(dy), np.abs(f["h1"]), np.abs(f["h2"]), np.abs(X)
    eb = np.zeros(mlp.N_PARAMS)

    # output layer: dY^T H2, and dZ2 = bf16((dY W3) * [Z2 > 0]) with FP32 W3
    eW3 = np.zeros((mlp.OUT_PAD, mlp.H))
    eW3[:mlp.OUT] = ady.T @ e["h2"] + e_dy.T @ ah2 + e_dy.T @ e["h2"] + ACC * (ady.T @ ah2)
    eb3 = np.zeros(mlp.OUT_PAD)
    eb3[:mlp.OUT] = e_dy.sum(0) + ACC * ady.sum(0)
    aW3 = np.abs(W3[:mlp.OUT])
    g2 = dy @ W3[:mlp.OUT]
    e_g2 = e_dy @ aW3 + ACC * (ady @ aW3)
    dz2 = _r(g2 * (f["z2"] > 0))
    e_dz2 = _masked_round_spread(g2, e_g2, f["z2"], e["z2"])
    adz2 = np.abs(dz2)
    eW2 = e_dz2.T @ ah1 + adz2.T @ e["h1"] + e_dz2.T @ e["h1"] + ACC * (adz2.T @ ah1)
    eb2 = e_dz2.sum(0) + ACC * adz2.sum(0)
    # hidden layer: dZ1 = bf16((dZ2 bf16(W2)) * [Z1 > 0]), then dZ1^T X
    aW2b = np.abs(_r(W2))
    g1 = dz2 @ _r(W2)
    e_g1 = e_dz2 @ aW2b + ACC * (adz2 @ aW2b)
    dz1 = _r(g1 * (f["z1"] > 0))
    e_dz1 = _masked_round_spread(g1, e_g1, f["z1"], e["z1"])
    adz1 = np.abs(dz1)
    eW1 = e_dz1.T @ aX + ACC * (adz1.T @ aX)
    eb1 = e_dz1.sum(0) + ACC * adz1.sum(0)

    eb[mlp.OFF_W1:mlp.OFF_B1] = eW1.ravel()
    eb[mlp.OFF_B1:mlp.OFF_W2] = eb1
    eb[mlp.OFF_W2:mlp.OFF_B2] = eW2.ravel()
    eb[mlp.OFF_B2:mlp.OFF_W3] = eb2
    eb[mlp.OFF_W3:mlp.OFF_B3] = eW3.ravel()
    eb[mlp.OFF_B3:mlp.N_PARAMS] = eb3
    return loss, g, e_loss, eb


BLOCKS = [("W1", mlp.OFF_W1, mlp.OFF_B1), ("b1", mlp.OFF_B1, mlp.OFF_W2),
          ("W2", mlp.OFF_W2, mlp.OFF_B2), ("b2", mlp.OFF_B2, mlp.OFF_W3),
          ("W3", mlp.OFF_W3, mlp.OFF_B3), ("b3", mlp.OFF_B3, mlp.N_PARAMS)]


def check(got, want, bound, what, floor=1e-12):
    """Every element within its bound (plus a tiny absolute floor)."""
    got = np.asarray(got, dtype=np.float64)
    err = np.abs(got - want)
    lim = bound + floor
    bad = np.nonzero(~(err <= lim))
    if bad[0].size:
        i = tuple(b[0] for b in bad)
        raise AssertionError(f"{what}: {bad[0].size} element(s) outside the bound, first at {i}: "
                             f"got {got[i]!r}, want {want[i]!r}, bound {lim[i]!r}")


def check_lines(got, want, shape, what, rtol=2e-2, floor=1e-9):
    """Each row and each column of a gradient block within rtol of the
    reference in relative norm: a wrong row or column cannot hide behind the
    rest of a large block."""
    G = np.asarray(got, dtype=np.float64).reshape(shape)
    W = np.asarray(want, dtype=np.float64).reshape(shape)
    for axis, name in ((1, "row"), (0, "column")):
        err = np.sqrt(((G - W) ** 2).sum(axis))
        ref = np.sqrt((W ** 2).sum(axis))
        bad = np.nonzero(~(err <= rtol * ref + floor))[0]
        if bad.size:
            raise AssertionError(f"{what}: {name} {bad[0]} off by {err[bad[0]]:.3e} "
                                 f"(norm {ref[bad[0]]:.3e})")


SHAPES = {"W1": (mlp.H, mlp.K_PAD), "b1": (1, mlp.H), "W2": (mlp.H, mlp.H), "b2": (1, mlp.H),
          "W3": (mlp.OUT_PAD, mlp.H), "b3": (1, mlp.OUT_PAD)}


def check_grads(got, want, bound):
    """Every gradient element within its bound, and every row and column of
    every block within 2 % in norm."""
    for name, a, b in BLOCKS:
        check(got[a:b], want[a:b], bound[a:b], name)
        check_lines(got[a:b], want[a:b], SHAPES[name], name)


def emulate_fp32(p, X, T=None):
    """An independent FP32 evaluation of the same network (bf16 rounding at
    the same points, FP32 sums in a different order): a stand-in for the GPU
    kernels on which the bounds can be checked without a GPU."""
    W1, b1, W2, b2, W3, b3 = [np.asarray(a, dtype=np.float32) for a in mlp.unpack(p)]
    r = lambda a: mlp.bf16_round(np.asarray(a, dtype=np.float32)).astype(np.float32)
    X = np.asarray(X, dtype=np.float32)
    # reversed K order: a different accumulation order than the reference
    z1 = (X[:, ::-1] @ r(W1)[:, ::-1].T) + b1
    h1 = r(np.maximum(z1, 0))
    z2 = (h1[:, ::-1] @ r(W2)[:, ::-1].T) + b2
    h2 = r(np.maximum(z2, 0))
    y = (h2 @ r(W3).T + b3)[:, :mlp.OUT]
    if T is None:
        return y
    T = np.asarray(T, dtype=np.float32)
    M = X.shape[0]
    valid = np.isfinite(T[:, 3])
    res = np.where(valid[:, None], y - np.nan_to_num(T), 0).astype(np.float32)
    a = np.abs(res)
    loss = float(np.where(a <= 1, 0.5 * res * res, a - 0.5).sum(dtype=np.float32) / M)
    dy = (np.where(a <= 1, res, np.sign(res)) / M).astype(np.float32)
    g = np.zeros(mlp.N_PARAMS, np.float32)
    gW3 = np.zeros((mlp.OUT_PAD, mlp.H), np.float32)
    gW3[:mlp.OUT] = dy.T @ h2
    dz2 = r((dy @ W3[:mlp.OUT]) * (z2 > 0))
    dz1 = r((dz2 @ r(W2)) * (z1 > 0))
    g[mlp.OFF_W1:mlp.OFF_B1] = (dz1.T @ X).ravel()
    g[mlp.OFF_B1:mlp.OFF_W2] = dz1.sum(0)
    g[mlp.OFF_W2:mlp.OFF_B2] = (dz2.T @ h1).ravel()
    g[mlp.OFF_B2:mlp.OFF_W3] = dz2.sum(0)
    g[mlp.OFF_W3:mlp.OFF_B3] = gW3.ravel()
    g[mlp.OFF_B3:mlp.OFF_B3 + mlp.OUT] = dy.sum(0)
    return y, loss, g
