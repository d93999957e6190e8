"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle (oracle/gamma_oracle.c) against something other
than itself: KKT enumeration, exhaustive search, fine-grid brute force,
closed forms, 1D polylines, invariants and hand-derived golden values.  A
dropped term, a wrong sign or index, or a transposed operand in the oracle
fails at least one of them.
"""
import glob
import math
import os

import numpy as np
import pytest

import oracle
import synth
from tests import _brute as brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def smooth_field(shape, seed, lo=0.2, hi=1.0, blur=1.5):
    from scipy import ndimage
    rng = np.random.default_rng(seed)
    f = ndimage.gaussian_filter(rng.standard_normal(shape), blur, mode="reflect")
    f = (f - f.min()) / (f.max() - f.min())
    return (lo + (hi - lo) * f).astype(np.float32)


# --------------------------------------------------------------------------
# Point-to-simplex distance (Section 2.1 normal equations + Ju recursion)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("K", [2, 3, 4])
def test_simplex_distance_matches_kkt_enumeration(K):
    rng = np.random.default_rng(K)
    for nv in range(1, K + 2):
        for trial in range(60):
            W = rng.normal(size=(nv, K)) * rng.uniform(0.1, 3.0)
            if trial % 3 == 0:
                W[:, -1] *= 40.0          # steep dose axis, as at 1 % criteria
            P = rng.normal(size=K) * 2.0
            want = brute.closed_simplex_distance(W[None], P[None])[0, 0]
            got = oracle.simplex_distance(W, P)
            assert got == pytest.approx(want, rel=1e-10, abs=1e-12), (nv, trial)


def test_simplex_distance_upper_bounded_by_samples():
    # Every point of the simplex is at least as far as the reported distance,
    # and dense samples come close to it.
    rng = np.random.default_rng(11)
    for _ in range(40):
        W = rng.normal(size=(4, 4))
        P = rng.normal(size=4) * 1.5
        d = oracle.simplex_distance(W, P)
        lam = rng.dirichlet(np.ones(4) * 0.3, size=200000)
        samples = lam @ W
        ds = np.sqrt(((samples - P) ** 2).sum(-1))
        assert ds.min() >= d - 1e-12
        assert ds.min() <= d + 0.05


def test_simplex_distance_inside_is_zero_and_vertex_case():
    W = np.array([[0, 0, 0.0], [1, 0, 0.0], [0, 1, 0.0]])
    assert oracle.simplex_distance(W, np.array([0.2, 0.2, 0.0])) == pytest.approx(0, abs=1e-15)
    assert oracle.simplex_distance(W, np.array([0.2, 0.2, 0.5])) == pytest.approx(0.5)
    # beyond the vertex (1, 0): nearest point is the vertex itself
    assert oracle.simplex_distance(W, np.array([2.0, -1.0, 0.0])) == pytest.approx(math.sqrt(2))


# --------------------------------------------------------------------------
# Table and early exit (Algorithm A1 steps 2-4) vs exhaustive search
# --------------------------------------------------------------------------

def test_cell_table_sorted_and_complete():
    shape, spacing, dta, R = (9, 11, 10), (2.5, 2.0, 1.5), 3.0, 2.7
    offs, keys = oracle.cell_table(3, shape, spacing, dta, R)
    # brute force: every offset whose cube fits some voxel, key < R
    want = []
    hz, hy, hx = spacing
    gap = lambda i: i if i >= 0 else -i - 1
    for k in range(-(shape[0] - 1), shape[0] - 1):
        for j in range(-(shape[1] - 1), shape[1] - 1):
            for i in range(-(shape[2] - 1), shape[2] - 1):
                key = math.sqrt((gap(i) * hx) ** 2 + (gap(j) * hy) ** 2 + (gap(k) * hz) ** 2) / dta
                if key < R:
                    want.append((key, k, j, i))
    want.sort()
    assert len(want) == len(keys)
    np.testing.assert_allclose(keys, [w[0] for w in want], rtol=0, atol=1e-14)
    assert np.all(np.diff(keys) >= 0)
    got = sorted(zip(np.round(keys, 12), offs[:, 2], offs[:, 1], offs[:, 0]))
    assert got == sorted((round(w[0], 12), w[1], w[2], w[3]) for w in want)


@pytest.mark.parametrize("local", [False, True])
@pytest.mark.parametrize("cap", [1 << 22, 3])
def test_pruned_search_equals_exhaustive_2d(local, cap):
    ref = smooth_field((11, 12), 1)
    ev = smooth_field((11, 12), 2, lo=0.1, hi=1.1)
    sp = (1.5, 1.0)
    want = brute.exhaustive_gamma(ref, ev, sp, 0.03, 2.0, local=local, cutoff_frac=0.1)
    got = oracle.gamma(ref, ev, sp, 0.03, 2.0, local=local, cutoff_frac=0.1, table_cap=cap)
    np.testing.assert_array_equal(np.isnan(got), np.isnan(want))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-10, equal_nan=True)


@pytest.mark.parametrize("local,cap", [(False, 1 << 22), (True, 1 << 22), (False, 7)])
def test_pruned_search_equals_exhaustive_3d(local, cap):
    ref = smooth_field((5, 6, 5), 3)
    ev = smooth_field((5, 6, 5), 4, lo=0.15, hi=1.05)
    sp = (2.5, 2.0, 1.5)
    want = brute.exhaustive_gamma(ref, ev, sp, 0.03, 3.0, local=local, cutoff_frac=0.1)
    got = oracle.gamma(ref, ev, sp, 0.03, 3.0, local=local, cutoff_frac=0.1, table_cap=cap)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-10, equal_nan=True)


def test_idx_subset_matches_full_grid():
    p = synth.workload("imrt_small")
    full = oracle.gamma_pair(p)
    rng = np.random.default_rng(0)
    idx = rng.choice(full.size, 500, replace=False)
    part = oracle.gamma_pair(p, idx=idx)
    np.testing.assert_array_equal(part, full.ravel()[idx])


# --------------------------------------------------------------------------
# Fine-grid brute force on the same interpolant
# --------------------------------------------------------------------------

def test_fine_grid_bound_2d():
    ref = smooth_field((10, 9), 5)
    ev = smooth_field((10, 9), 6, lo=0.1, hi=1.0)
    sp, dd, dta = (1.2, 1.0), 0.05, 2.0
    g = oracle.gamma(ref, ev, sp, dd, dta)
    gf, slack = brute.fine_grid_gamma(ref, ev, sp, dd, dta, factor=20)
    assert np.all(g <= gf + 1e-12)
    assert np.all(gf <= g + slack + 1e-12)
    assert np.max(gf - g) < 0.05


def test_fine_grid_bound_3d():
    ref = smooth_field((4, 5, 4), 7)
    ev = smooth_field((4, 5, 4), 8, lo=0.1, hi=1.0)
    sp, dd, dta = (2.0, 1.5, 1.0), 0.08, 2.5
    g = oracle.gamma(ref, ev, sp, dd, dta)
    gf, slack = brute.fine_grid_gamma(ref, ev, sp, dd, dta, factor=10)
    assert np.all(g <= gf + 1e-12)
    assert np.all(gf <= g + slack + 1e-12)


# --------------------------------------------------------------------------
# Closed forms
# --------------------------------------------------------------------------

def test_identical_doses_give_zero():
    p = synth.workload("imrt_small")
    g = oracle.gamma(p.ref, p.ref, p.spacing, 0.03, 3.0, cutoff_frac=0.1)
    ev = ~np.isnan(g)
    assert ev.sum() > 100
    assert np.all(g[ev] == 0.0)


@pytest.mark.parametrize("ndim", [2, 3])
def test_flat_field_shift(ndim):
    shape = (6, 7) if ndim == 2 else (5, 6, 7)
    sp = (1.0, 2.0) if ndim == 2 else (2.5, 1.0, 2.0)
    ref = np.full(shape, 0.5, np.float32)
    delta = np.float32(0.0625)          # exactly representable
    ev = ref + delta
    g = oracle.gamma(ref, ev, sp, 0.02, 3.0, dose_norm=1.0)
    np.testing.assert_allclose(g, float(delta) / 0.02, rtol=1e-13)


@pytest.mark.parametrize("ndim", [2, 3])
def test_linear_ramp_closed_form(ndim):
    # D_r = a + grad . r, D_e(r) = D_r(r) - delta: the interpolant of a linear
    # field is the field, so gamma is the distance to a hyperplane:
    # |delta/dD| / sqrt(1 + |grad * dta / dD|^2).
    shape = (14, 15) if ndim == 2 else (9, 10, 11)
    sp = (1.0, 1.5) if ndim == 2 else (2.0, 1.25, 1.5)
    grad = np.array([0.011, -0.007] if ndim == 2 else [0.004, 0.009, -0.006])  # per mm, axis order
    coords = np.meshgrid(*[np.arange(n) * h for n, h in zip(shape, sp)], indexing="ij")
    ramp = 0.6 + sum(g_ * c for g_, c in zip(grad, coords))
    ref = ramp.astype(np.float32)
    delta = 0.0125
    ev = (ramp - delta).astype(np.float32)
    # use the float32-rounded difference actually stored
    dd, dta = 0.02, 3.0
    dD = dd * 1.0
    g = oracle.gamma(ref, ev, sp, dd, dta, dose_norm=1.0)
    want_scale = 1.0 / math.sqrt(1.0 + float(np.sum((grad * dta / dD) ** 2)))
    inner = tuple(slice(3, -3) for _ in shape)
    diff = (ref.astype(np.float64) - ev.astype(np.float64))[inner] / dD
    # f32 rounding of the stored doses perturbs the field by ~1e-8; allow it
    np.testing.assert_allclose(g[inner], np.abs(diff) * want_scale, rtol=0, atol=5e-6)
    np.testing.assert_allclose(g[inner], delta / dD * want_scale, rtol=0, atol=5e-6)


# --------------------------------------------------------------------------
# 1D profiles: the surface cross-section is the polyline through the samples
# --------------------------------------------------------------------------

@pytest.mark.parametrize("axis", [0, 1, 2])
def test_one_dimensional_profile_matches_polyline(axis):
    rng = np.random.default_rng(40 + axis)
    n = 23
    xs = np.arange(n)
    prof_r = 0.5 + 0.4 * np.sin(xs / 3.1) + rng.normal(0, 0.01, n)
    prof_e = 0.5 + 0.42 * np.sin((xs - 0.6) / 3.1) + rng.normal(0, 0.01, n)
    shape = [4, 5, 6]
    shape[axis] = n
    sp = [1.5, 2.0, 2.5]
    expand = [None, None, None]
    expand[axis] = slice(None)
    ref = np.broadcast_to(prof_r.astype(np.float32)[tuple(expand)], shape).copy()
    ev = np.broadcast_to(prof_e.astype(np.float32)[tuple(expand)], shape).copy()
    dd, dta = 0.03, 3.0
    g = oracle.gamma(ref, ev, sp, dd, dta, dose_norm=1.0)
    want = brute.polyline_gamma_1d(prof_r.astype(np.float32).astype(np.float64),
                                   prof_e.astype(np.float32).astype(np.float64),
                                   sp[axis], dd, dta)
    got = np.moveaxis(g, axis, 0)
    for idx in np.ndindex(got.shape[1:]):
        np.testing.assert_allclose(got[(slice(None),) + idx], want, rtol=0, atol=1e-11)


# --------------------------------------------------------------------------
# Invariants
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def small3d():
    p = synth.make_pair_3d(shape=(10, 14, 12), spacing=(2.5, 2.5, 2.5), seed=9,
                           shift_mm=(0.5, 0.0, 1.5), scale=1.04)
    g = oracle.gamma(p.ref, p.eval, p.spacing, 0.03, 3.0, cutoff_frac=0.1)
    return p, g


def test_scaling_spacing_and_dta_together(small3d):
    p, g = small3d
    s = 2.5
    g2 = oracle.gamma(p.ref, p.eval, tuple(h * s for h in p.spacing), 0.03, 3.0 * s, cutoff_frac=0.1)
    np.testing.assert_allclose(g2, g, rtol=1e-12, atol=1e-13, equal_nan=True)


def test_scaling_doses_and_norm_together_global(small3d):
    p, g = small3d
    s = np.float32(4.0)      # power of two: the float32 doses scale exactly
    dn = float(p.ref.max())
    g2 = oracle.gamma(p.ref * s, p.eval * s, p.spacing, 0.03, 3.0, cutoff_frac=0.1,
                      dose_norm=dn * float(s))
    np.testing.assert_allclose(g2, g, rtol=1e-12, atol=1e-13, equal_nan=True)


@pytest.mark.parametrize("perm", [(0, 2, 1), (1, 0, 2), (2, 1, 0), (1, 2, 0)])
def test_axis_permutation(small3d, perm):
    p, g = small3d
    sp = tuple(np.array(p.spacing)[list(perm)])
    ref = np.ascontiguousarray(p.ref.transpose(perm))
    ev = np.ascontiguousarray(p.eval.transpose(perm))
    g2 = oracle.gamma(ref, ev, sp, 0.03, 3.0, cutoff_frac=0.1, dose_norm=float(p.ref.max()))
    np.testing.assert_allclose(g2, g.transpose(perm), rtol=1e-12, atol=1e-13, equal_nan=True)


def test_bounds_zero_gamma0_and_discrete(small3d):
    p, g = small3d
    dD = 0.03 * float(p.ref.max())
    g0 = np.abs(p.eval.astype(np.float64) - p.ref) / dD
    ok = ~np.isnan(g)
    assert np.all(g[ok] >= 0)
    assert np.all(g[ok] <= g0[ok] + 1e-15)
    gd = brute.discrete_gamma(p.ref, p.eval, p.spacing, 0.03, 3.0, cutoff_frac=0.1)
    assert np.all(g[ok] <= gd[ok] + 1e-12)
    assert np.mean(g[ok] < gd[ok] - 1e-6) > 0.1     # interpolation does help


def test_crop_locality():
    # Whole-voxel translation/cropping leaves gamma unchanged wherever the
    # search ball fits in the crop.
    p = synth.make_pair_3d(shape=(18, 22, 20), spacing=(2.5, 2.5, 2.5), seed=9,
                           shift_mm=(0.5, 0.0, 1.5), scale=1.04)
    dn = float(p.ref.max())
    g = oracle.gamma(p.ref, p.eval, p.spacing, 0.03, 3.0, cutoff_frac=0.1, dose_norm=dn)
    c = 4
    sub = (slice(c, -c),) * 3
    g2 = oracle.gamma(np.ascontiguousarray(p.ref[sub]), np.ascontiguousarray(p.eval[sub]),
                      p.spacing, 0.03, 3.0, cutoff_frac=0.1, dose_norm=dn)
    ref_c = g[sub]
    zz, yy, xx = np.indices(ref_c.shape)
    edge = np.minimum.reduce([zz, yy, xx, ref_c.shape[0] - 1 - zz, ref_c.shape[1] - 1 - yy,
                              ref_c.shape[2] - 1 - xx]) * 2.5
    inner = np.nan_to_num(ref_c, nan=1e9) * 3.0 + 2.5 * math.sqrt(3) < edge
    assert inner.sum() > 20
    np.testing.assert_allclose(g2[inner], ref_c[inner], rtol=1e-12, atol=1e-13)
    np.testing.assert_array_equal(np.isnan(g2), np.isnan(ref_c))


def test_two_identical_slices_equal_2d():
    p = synth.make_pair_2d(shape=(20, 18), seed=4)
    g2d = oracle.gamma(p.ref, p.eval, p.spacing, 0.03, 3.0, cutoff_frac=0.1)
    ref3 = np.stack([p.ref, p.ref])
    ev3 = np.stack([p.eval, p.eval])
    g3 = oracle.gamma(ref3, ev3, (2.0,) + p.spacing, 0.03, 3.0, cutoff_frac=0.1)
    np.testing.assert_allclose(g3[0], g2d, rtol=1e-12, atol=1e-14, equal_nan=True)
    np.testing.assert_allclose(g3[1], g2d, rtol=1e-12, atol=1e-14, equal_nan=True)


def test_local_mode_is_global_with_voxel_norm():
    # Local criterion: dD(v) = dd * D_r(v).  Voxel by voxel this is the global
    # criterion with dose_norm = D_r(v).
    p = synth.make_pair_2d(shape=(16, 16), seed=2)
    gl = oracle.gamma(p.ref, p.eval, p.spacing, 0.02, 2.0, local=True, cutoff_frac=0.2)
    rng = np.random.default_rng(1)
    cand = np.nonzero(~np.isnan(gl.ravel()))[0]
    for v in rng.choice(cand, 12, replace=False):
        gg = oracle.gamma(p.ref, p.eval, p.spacing, 0.02, 2.0, cutoff_frac=0.0,
                          dose_norm=float(p.ref.ravel()[v]), idx=np.array([v]))
        assert gg[0] == pytest.approx(gl.ravel()[v], rel=1e-12)


def test_cutoff_mask():
    p = synth.workload("plane_128")
    g = oracle.gamma_pair(p)
    thr = 0.1 * float(p.ref.max())
    np.testing.assert_array_equal(np.isnan(g), p.ref < thr)


def test_bad_shapes_rejected():
    with pytest.raises(ValueError):
        oracle.gamma(np.ones((1, 5), np.float32), np.ones((1, 5), np.float32), (1, 1), 0.03, 3)
    with pytest.raises(ValueError):
        oracle.gamma(np.full((4, 4), np.nan, np.float32), np.ones((4, 4), np.float32),
                     (1, 1), 0.03, 3)


# --------------------------------------------------------------------------
# Hand-derived golden values
# --------------------------------------------------------------------------

@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "freudenthal_*.txt"))))
def test_golden_fixtures(path):
    ref, ev, sp, crit, expect = brute.read_golden(path)
    g = oracle.gamma(ref, ev, sp, **crit)
    # the exhaustive brute force agrees with the hand derivation too
    gb = brute.exhaustive_gamma(ref, ev, sp, crit["dd_frac"], crit["dta_mm"],
                                cutoff_frac=crit["cutoff_frac"], dose_norm=crit["dose_norm"])
    for flat, want, expr in expect:
        assert g.ravel()[flat] == pytest.approx(want, rel=1e-13), expr
        assert gb.ravel()[flat] == pytest.approx(want, rel=1e-12), expr
