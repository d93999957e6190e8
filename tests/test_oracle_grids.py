"""Pins of the oracle for reference and evaluation doses on different grids
(each grid with its own shape, spacing and origin).  CPU only.

The oracle takes Eq. 1 literally (minimum over the evaluation surface, the
Freudenthal interpolant of the evaluation grid), so it is checked against:
  - the pinned coincident-grid oracle when both grids are the same;
  - brute force over every simplex of a tiny evaluation grid, for reference
    points inside and outside the evaluation grid;
  - the closed form for a linear dose field (the interpolant of a linear
    field is the field, so gamma is the distance to a hyperplane);
  - invariance under a common translation of both grids and under scaling
    every length (spacings, origins and DTA) together.
"""
import numpy as np
import pytest

import oracle
from tests._brute import closed_simplex_distance, freudenthal_simplices

f32 = lambda x: float(np.float32(x))


def _positions(shape, spacing, origin):
    """Physical positions (x, y[, z]) of every node of a (z, y, x) grid."""
    axes = [o + np.arange(n) * h for n, h, o in zip(shape, spacing, origin)]
    g = np.meshgrid(*axes, indexing="ij")
    return np.stack(g[::-1], axis=-1).reshape(-1, len(shape))


def _brute(ref, rsp, ro, ev, esp, eo, dd, dta, local=False, cutoff=0.0):
    """Minimum over every simplex of the evaluation grid."""
    n = ref.ndim
    dnorm = float(ref.max())
    X = _positions(ref.shape, rsp, ro) / dta
    r = ref.astype(np.float64).ravel()
    dD = dd * (r if local else np.full_like(r, dnorm))
    mask = np.float32(r) >= np.float32(f32(cutoff) * np.float32(dnorm))
    if local:
        mask &= r > 0
    E = _positions(ev.shape, esp, eo) / dta
    e = ev.astype(np.float64).ravel()
    S = freudenthal_simplices(ev.shape)                      # (s, n + 1) flat ids
    out = np.full(r.shape, np.nan)
    for v in np.nonzero(mask)[0]:
        W = np.concatenate([E[S], (e[S] / dD[v])[..., None]], axis=-1)
        P = np.concatenate([X[v], [r[v] / dD[v]]])[None]
        out[v] = closed_simplex_distance(W, P).min()
    return out.reshape(ref.shape)


def _grids(ref, rsp, ro, ev, esp, eo, dd, dta, **kw):
    return oracle.gamma_grids(ref, rsp, ro, ev, esp, eo, f32(dd), f32(dta), **kw)


@pytest.mark.parametrize("local", [False, True])
@pytest.mark.parametrize("nd", [2, 3])
def test_coincident_grids_equal_the_pinned_oracle(nd, local):
    rng = np.random.default_rng(40 + nd)
    shape = (9, 11) if nd == 2 else (6, 7, 8)
    sp = (1.5, 1.0) if nd == 2 else (2.0, 1.5, 1.0)
    ref = rng.uniform(0.2, 1.0, shape).astype(np.float32)
    ev = (ref + rng.normal(0, 0.05, shape)).astype(np.float32)
    want = oracle.gamma(ref, ev, sp, f32(0.03), f32(2.0), local=local, cutoff_frac=f32(0.25))
    got = _grids(ref, sp, (0.0,) * nd, ev, sp, (0.0,) * nd, 0.03, 2.0, local=local,
                 cutoff_frac=f32(0.25))
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    assert np.max(np.abs(got[ok] - want[ok])) < 1e-12


@pytest.mark.parametrize("nd", [2, 3])
def test_against_brute_force_inside_and_outside(nd):
    rng = np.random.default_rng(50 + nd)
    if nd == 2:
        ev = rng.uniform(0.0, 1.0, (5, 6)).astype(np.float32)
        esp, eo = (1.3, 0.9), (0.4, -0.7)
        ref = rng.uniform(0.3, 1.0, (7, 8)).astype(np.float32)
        rsp, ro = (0.8, 0.75), (-1.0, -1.5)                  # reaches outside the eval grid
    else:
        ev = rng.uniform(0.0, 1.0, (4, 4, 5)).astype(np.float32)
        esp, eo = (1.2, 1.0, 0.9), (0.3, -0.2, 0.5)
        ref = rng.uniform(0.3, 1.0, (5, 5, 5)).astype(np.float32)
        rsp, ro = (1.0, 0.85, 0.95), (-0.8, -0.6, -0.4)
    for local in (False, True):
        want = _brute(ref, rsp, ro, ev, esp, eo, f32(0.1), f32(1.0), local=local)
        got = _grids(ref, rsp, ro, ev, esp, eo, 0.1, 1.0, local=local)
        assert np.array_equal(np.isnan(got), np.isnan(want))
        ok = ~np.isnan(want)
        assert np.max(np.abs(got[ok] - want[ok])) < 1e-9


@pytest.mark.parametrize("nd", [2, 3])
def test_linear_field_closed_form(nd):
    # D(x) = a + g . x on both grids (the reference lowered by delta): the
    # surface is the hyperplane, so gamma = delta/dD / sqrt(1 + |g dta/dD|^2)
    # wherever the foot of the perpendicular lies inside the evaluation grid.
    g = np.array([0.02, -0.015, 0.01][:nd])
    a, delta, dta, dd = 1.0, 0.02, 3.0, 0.03
    if nd == 2:
        eshape, esp, eo = (30, 28), (1.1, 1.3), (-2.0, -1.0)
        rshape, rsp, ro = (12, 12), (1.7, 1.6), (8.0, 7.5)
    else:
        eshape, esp, eo = (16, 18, 17), (1.4, 1.2, 1.3), (-1.0, -2.0, -1.5)
        rshape, rsp, ro = (6, 6, 6), (1.6, 1.5, 1.7), (6.0, 7.0, 6.5)
    E = _positions(eshape, esp, eo)
    R = _positions(rshape, rsp, ro)
    ev = (a + E @ g).reshape(eshape).astype(np.float32)
    ref = (a + R @ g - delta).reshape(rshape).astype(np.float32)
    got = _grids(ref, rsp, ro, ev, esp, eo, dd, dta, dose_norm=1.0)
    # the closed form with the float32 doses actually stored
    dD = f32(dd) * 1.0
    resid = (a + R @ g - ref.ravel().astype(np.float64))       # D_e(x_r) - D_r
    gn = np.linalg.norm(g) * f32(dta) / dD
    want = np.abs(resid) / dD / np.sqrt(1.0 + gn * gn)
    # float32 storage of the evaluation doses perturbs the plane by <= 1 ulp
    assert np.max(np.abs(got.ravel() - want)) < 2e-5


def test_common_translation_and_scaling_are_invariant():
    rng = np.random.default_rng(60)
    ev = rng.uniform(0.0, 1.0, (5, 6, 7)).astype(np.float32)
    ref = rng.uniform(0.3, 1.0, (4, 5, 5)).astype(np.float32)
    esp, eo = (1.2, 1.0, 0.9), (0.3, -0.2, 0.5)
    rsp, ro = (1.1, 0.85, 0.95), (0.2, 0.1, 0.4)
    base = _grids(ref, rsp, ro, ev, esp, eo, 0.05, 1.5)
    t = np.array([7.25, -3.5, 11.0])
    moved = _grids(ref, rsp, tuple(np.add(ro, t)), ev, esp, tuple(np.add(eo, t)), 0.05, 1.5)
    assert np.max(np.abs(moved - base)) < 1e-9
    s = 2.0                                                    # exact in binary
    scaled = _grids(ref, tuple(np.multiply(rsp, s)), tuple(np.multiply(ro, s)), ev,
                    tuple(np.multiply(esp, s)), tuple(np.multiply(eo, s)), 0.05, 3.0)
    assert np.max(np.abs(scaled - base)) < 1e-9
