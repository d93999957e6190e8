"""FP64 CPU reference of the proposal network and its patch features.

TEST INFRASTRUCTURE ONLY (tests and the benchmark's checks).  Plain numpy
matrix products in float64.  The network is defined with BF16 weights and
BF16 activations; with ``bf16=True`` this reference rounds at exactly those
points (W1/W2/W3 to bf16 for the products, H1/H2 after the ReLU, the
backward intermediates dZ2/dZ1 before their products), so a correct GPU
implementation differs from it only by FP32 accumulation order.  With
``bf16=False`` it is the plain FP64 network, used to pin the backward
formulas by finite differences.

Network: x (384: 375 features + zero padding) -> z1 = W1 x + b1 -> h1 =
relu(z1) -> z2 = W2 h1 + b2 -> h2 = relu(z2) -> y = W3 h2 + b3 (4 outputs).
Loss: Huber (delta 1) summed over the 4 outputs, averaged over all M rows;
rows whose last target is NaN contribute nothing.
"""
from __future__ import annotations

import numpy as np

K_IN, K_PAD, H, OUT, OUT_PAD = 375, 384, 128, 4, 8
OFF_W1 = 0
OFF_B1 = OFF_W1 + H * K_PAD
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + OUT_PAD * H
N_PARAMS = OFF_B3 + OUT_PAD


def bf16_round(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = rounded.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def unpack(p: np.ndarray):
    p = np.asarray(p, dtype=np.float64)
    return (p[OFF_W1:OFF_B1].reshape(H, K_PAD), p[OFF_B1:OFF_W2], p[OFF_W2:OFF_B2].reshape(H, H),
            p[OFF_B2:OFF_W3], p[OFF_W3:OFF_B3].reshape(OUT_PAD, H), p[OFF_B3:N_PARAMS])


def forward(p, X, bf16: bool = True):
    W1, b1, W2, b2, W3, b3 = unpack(p)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ r(W1).T + b1
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ r(W2).T + b2
    h2 = r(np.maximum(z2, 0.0))
    y = h2 @ r(W3).T + b3
    return {"z1": z1, "h1": h1, "z2": z2, "h2": h2, "y": y[:, :OUT]}


def loss_and_grads(p, X, T, bf16: bool = True):
    """Mean Huber loss and the gradient of every parameter (flat, N_PARAMS)."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    M = X.shape[0]
    f = forward(p, X, bf16)
    valid = np.isfinite(T[:, 3])
    res = np.where(valid[:, None], f["y"] - np.nan_to_num(T), 0.0)
    a = np.abs(res)
    loss = np.where(a <= 1.0, 0.5 * res * res, a - 0.5).sum() / M
    dy = np.where(a <= 1.0, res, np.sign(res)) / M                  # M x 4
    g = np.zeros(N_PARAMS)
    gW3 = np.zeros((OUT_PAD, H))
    gW3[:OUT] = dy.T @ f["h2"]
    gb3 = np.zeros(OUT_PAD)
    gb3[:OUT] = dy.sum(0)
    dz2 = r((dy @ W3[:OUT]) * (f["z2"] > 0))
    gW2 = dz2.T @ f["h1"]
    gb2 = dz2.sum(0)
    dz1 = r((dz2 @ r(W2)) * (f["z1"] > 0))
    gW1 = dz1.T @ X
    gb1 = dz1.sum(0)
    g[OFF_W1:OFF_B1] = gW1.ravel()
    g[OFF_B1:OFF_W2] = gb1
    g[OFF_W2:OFF_B2] = gW2.ravel()
    g[OFF_B2:OFF_W3] = gb2
    g[OFF_W3:OFF_B3] = gW3.ravel()
    g[OFF_B3:N_PARAMS] = gb3
    return loss, g


def trainable_mask() -> np.ndarray:
    k = np.ones(N_PARAMS, dtype=bool)
    k[OFF_W1:OFF_B1].reshape(H, K_PAD)[:, K_IN:] = False
    k[OFF_W3:OFF_B3].reshape(OUT_PAD, H)[OUT:] = False
    k[OFF_B3 + OUT:N_PARAMS] = False
    return k


# ---------------------------------------------------------------------------
# Patch features
# ---------------------------------------------------------------------------

def _grad_norm(D: np.ndarray, spacing, dta) -> np.ndarray:
    """|grad D| * dta per grid point: central differences inside, one-sided
    at the grid edge (axes in array order, spacing in the same order)."""
    g2 = np.zeros(D.shape)
    for ax, h in enumerate(spacing):
        d = np.zeros(D.shape)
        sl = lambda a, b: tuple(slice(a, b) if i == ax else slice(None) for i in range(D.ndim))
        d[sl(1, -1)] = (D[sl(2, None)] - D[sl(None, -2)]) / (2.0 * h)
        d[sl(0, 1)] = (D[sl(1, 2)] - D[sl(0, 1)]) / h
        d[sl(-1, None)] = (D[sl(-1, None)] - D[sl(-2, -1)]) / h
        g2 += d * d
    return np.sqrt(g2) * dta


def features(ref, ev, spacing, dd_frac, dta, voxels, local=False, dose_norm=0.0) -> np.ndarray:
    """Features of flat voxel indices `voxels` (FP64, before rounding):
    channel-major over the 5^n patch (x fastest), 375 values, zero-padded to
    384; see the definition in the kernels' documentation."""
    ref = np.asarray(ref, dtype=np.float64)
    ev = np.asarray(ev, dtype=np.float64)
    nd = ref.ndim
    dn = dose_norm if dose_norm > 0 else float(ref.max())
    ge = _grad_norm(ev, spacing, dta)
    gr = _grad_norm(ref, spacing, dta)
    out = np.zeros((len(voxels), K_PAD))
    shape = ref.shape
    for row, v in enumerate(voxels):
        idx = np.unravel_index(int(v), shape)
        dr = ref[idx]
        dD = dd_frac * (dr if local else dn)
        inv = 1.0 / dD
        for pi in range(125):
            o = (pi % 5 - 2, (pi // 5) % 5 - 2, pi // 25 - 2)          # x, y, z
            if nd == 2 and o[2] != -2:
                continue
            offs = o[:nd][::-1]                                     # array order
            p = tuple(i + d for i, d in zip(idx, offs))
            if any(c < 0 or c >= n for c, n in zip(p, shape)):
                continue
            out[row, pi] = np.clip((ev[p] - dr) * inv, -16.0, 16.0)
            out[row, 125 + pi] = min(ge[p] * inv, 32.0)
            out[row, 250 + pi] = min(gr[p] * inv, 32.0)
    return out
