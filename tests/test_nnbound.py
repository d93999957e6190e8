"""CPU checks of the element-wise bounds the network's GPU tests use: an
independent FP32 evaluation of the network (different accumulation order,
bf16 rounding at the same points) stays inside them, and the plausible
mistakes a kernel could make (a zeroed, swapped or sign-flipped row or
column of a gradient block, swapped outputs) fall outside them."""
import numpy as np
import pytest

from oracle import mlp
from tests import _nnbound as nb


def _case(seed, M=300):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.08, mlp.N_PARAMS)
    p[~mlp.trainable_mask()] = 0.0
    X = np.zeros((M, mlp.K_PAD), np.float32)
    X[:, :mlp.K_IN] = rng.normal(0, 1.5, (M, mlp.K_IN))
    X = mlp.bf16_round(X)
    T = rng.normal(0, 1, (M, 4))
    T[::17, 3] = np.nan
    return p, X, T


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fp32_emulation_is_inside_the_bounds(seed):
    p, X, T = _case(seed)
    f, e = nb.forward_bounds(p, X)
    y = nb.emulate_fp32(p, X)
    nb.check(y, f["y"], e["y"], "forward")
    loss, g, e_loss, eg = nb.backward_bounds(p, X, T)
    y2, loss32, g32 = nb.emulate_fp32(p, X, T)
    assert abs(loss32 - loss) <= e_loss + 1e-7
    nb.check_grads(g32, g, eg)


def test_bounds_catch_row_and_column_mistakes():
    p, X, T = _case(5)
    loss, g, e_loss, eg = nb.backward_bounds(p, X, T)
    shapes = {"W1": (mlp.H, mlp.K_PAD), "W2": (mlp.H, mlp.H), "W3": (mlp.OUT_PAD, mlp.H)}
    for name, a, b in nb.BLOCKS:
        if name not in shapes:
            continue
        G = g[a:b].reshape(shapes[name])
        E = eg[a:b].reshape(shapes[name])
        rows = 4 if name == "W3" else mlp.H
        cols = mlp.K_IN if name == "W1" else mlp.H
        for mistake in ("zero_row", "swap_rows", "neg_col", "zero_col"):
            bad = G.copy()
            if mistake == "zero_row":
                bad[1] = 0.0
            elif mistake == "swap_rows":
                bad[[0, rows - 1]] = bad[[rows - 1, 0]]
            elif mistake == "neg_col":
                bad[:rows, 3] = -bad[:rows, 3]
            else:
                bad[:rows, cols - 1] = 0.0
            gbad = g.copy()
            gbad[a:b] = bad.ravel()
            with pytest.raises(AssertionError):
                nb.check_grads(gbad, g, eg)
    f, e = nb.forward_bounds(p, X)
    with pytest.raises(AssertionError):
        nb.check(f["y"][:, [1, 0, 2, 3]], f["y"], e["y"], "swapped outputs")
