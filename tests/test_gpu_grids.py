"""Reference and evaluation doses on different grids: the CUDA path against the
oracle (element by element), on planes and volumes, with the reference grid
reaching outside the evaluation grid, in global and local mode, past a
truncated cell table, and the identical-geometry case against the
coincident-grid search."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4
f32 = lambda x: float(np.float32(x))


def _crit(g, c):
    return g.criteria(c.dd_frac, c.dta_mm, c.local, c.cutoff_frac, c.dose_norm)


def gpu_grids(ref, rsp, ro, ev, esp, eo, crit, options=None):
    import paper_1012_1900_gb300 as g
    nd = ref.ndim
    pad = (lambda v, x: v if nd == 3 else (x,) + tuple(v))
    r = torch.from_numpy(np.ascontiguousarray(ref, dtype=np.float32)).cuda()
    e = torch.from_numpy(np.ascontiguousarray(ev, dtype=np.float32)).cuda()
    out = torch.full_like(r, -7.0)
    h = g.gamma_create_grids(r, e, nd, pad(ref.shape, 1), pad(rsp, 1.0), pad(ro, 0.0),
                             pad(ev.shape, 1), pad(esp, 1.0), pad(eo, 0.0), _crit(g, crit))
    try:
        for k, v in (options or {}).items():
            g.gamma_set_option(h, k, v)
        g.gamma_run(h, out)
        counts = g.gamma_pass_rate(h)
        st = g.gamma_get_stats(h)
    finally:
        g.gamma_destroy(h)
    return out.cpu().numpy().astype(np.float64), counts, st


def oracle_grids(ref, rsp, ro, ev, esp, eo, crit):
    return oracle.gamma_grids(ref, rsp, ro, ev, esp, eo, f32(crit.dd_frac), f32(crit.dta_mm),
                              local=crit.local, cutoff_frac=f32(crit.cutoff_frac),
                              dose_norm=f32(crit.dose_norm))


def check(got, want, counts):
    assert np.array_equal(np.isnan(got), np.isnan(want)), "evaluated masks differ"
    ok = ~np.isnan(want)
    err = np.abs(got[ok] - want[ok])
    assert err.max() <= TOL, f"max |dgamma| = {err.max():.3e}"
    n_eval, n_pass = counts[1], counts[2]
    assert n_eval == int(ok.sum())
    edge = np.abs(want[ok] - 1.0) < 1e-4
    assert abs(n_pass - int((want[ok] <= 1.0).sum())) <= int(edge.sum())


def _volume_pair(seed, shape=(20, 24, 22)):
    return synth.make_pair_3d(shape=shape, spacing=(2.5, 2.5, 2.5), seed=seed,
                              shift_mm=(0.5, -1.0, 1.5), scale=1.03)


@pytest.mark.parametrize("walk", [0, 3], ids=["lane_walk", "warp_cells"])
@pytest.mark.parametrize("local", [False, True])
def test_volume_on_a_finer_shifted_grid(local, walk):
    # evaluation at 2.5 mm, reference resampled at 1.7 mm from another origin
    p = _volume_pair(31)
    ev = p.eval
    esp, eo = (2.5, 2.5, 2.5), (0.0, 0.0, 0.0)
    rshape, rsp, ro = (26, 30, 28), (1.7, 1.75, 1.8), (1.1, 2.3, 0.7)
    # reference doses: the evaluation generator's clean field sampled on the
    # reference grid (nearest evaluation node, then perturbed)
    rng = np.random.default_rng(5)
    zz, yy, xx = np.meshgrid(*[np.clip(np.rint((o + np.arange(n) * h) / 2.5).astype(int), 0, s - 1)
                               for n, h, o, s in zip(rshape, rsp, ro, ev.shape)], indexing="ij")
    ref = (p.ref[zz, yy, xx] * (1 + rng.normal(0, 0.01, rshape))).astype(np.float32)
    crit = synth.Criteria(0.02, 2.0, local=local)
    got, counts, _ = gpu_grids(ref, rsp, ro, ev, esp, eo, crit, {"walk": walk})
    want = oracle_grids(ref, rsp, ro, ev, esp, eo, crit)
    check(got, want, counts)


@pytest.mark.parametrize("walk", [0, 3], ids=["lane_walk", "warp_cells"])
def test_plane_reaching_outside_the_evaluation_grid(walk):
    rng = np.random.default_rng(7)
    p = synth.make_pair_2d(shape=(48, 52), spacing=(1.0, 1.0), seed=7, shift_mm=(0.6, -0.4))
    ev = p.eval
    esp, eo = (1.0, 1.0), (0.0, 0.0)
    rshape, rsp, ro = (40, 44), (1.3, 1.25), (-4.0, -3.5)   # beyond the evaluation edges
    yy, xx = np.meshgrid(*[np.clip(np.rint((o + np.arange(n) * h)).astype(int), 0, s - 1)
                           for n, h, o, s in zip(rshape, rsp, ro, ev.shape)], indexing="ij")
    ref = (p.ref[yy, xx] * (1 + rng.normal(0, 0.01, rshape))).astype(np.float32)
    crit = synth.Criteria(0.03, 3.0)
    got, counts, _ = gpu_grids(ref, rsp, ro, ev, esp, eo, crit, {"walk": walk})
    want = oracle_grids(ref, rsp, ro, ev, esp, eo, crit)
    check(got, want, counts)


@pytest.mark.parametrize("walk", [0, 3], ids=["lane_walk", "warp_cells"])
def test_truncated_table_box_scan(walk):
    p = _volume_pair(33, shape=(12, 14, 13))
    ev = p.eval
    rshape, rsp, ro = (10, 12, 11), (2.9, 2.8, 3.1), (0.4, -0.3, 0.9)
    rng = np.random.default_rng(9)
    ref = (rng.uniform(0.2, 1.0, rshape) * float(ev.max())).astype(np.float32)
    crit = synth.Criteria(0.01, 1.0, local=True)
    got, counts, st = gpu_grids(ref, rsp, ro, ev, (2.5, 2.5, 2.5), (0.0, 0.0, 0.0), crit,
                                {"table_cap": 32, "walk": walk})
    assert st["overflow_voxels"] > 0
    want = oracle_grids(ref, rsp, ro, ev, (2.5, 2.5, 2.5), (0.0, 0.0, 0.0), crit)
    check(got, want, counts)


def test_identical_geometry_is_the_coincident_search():
    import paper_1012_1900_gb300 as g
    p = synth.workload("imrt_small")
    crit = p.criteria
    sp, o = p.spacing, (0.0, 0.0, 0.0)
    got, counts, _ = gpu_grids(p.ref, sp, o, p.eval, sp, o, crit)
    want = oracle.gamma(p.ref, p.eval, sp, f32(crit.dd_frac), f32(crit.dta_mm),
                        cutoff_frac=f32(crit.cutoff_frac))
    check(got, want, counts)
    # a slightly moved origin takes the two-grid path and must agree with the oracle too
    o2 = (0.0, 0.0, 1e-3)
    got2, counts2, _ = gpu_grids(p.ref, sp, o, p.eval, sp, o2, crit)
    want2 = oracle_grids(p.ref, sp, o, p.eval, sp, o2, crit)
    check(got2, want2, counts2)


@pytest.mark.parametrize("fp64_all", [False, True], ids=["fp32", "fp64_every_cell"])
def test_warp_evaluated_grid_walk_is_bitwise_the_lane_walk(fp64_all):
    # walk = 3 evaluates each cell with the lane walk's arithmetic (with the
    # FP64 redo forced on every cell, every voxel goes to the 32-lane re-search)
    p = _volume_pair(35, shape=(24, 26, 28))
    ev = p.eval
    rshape, rsp, ro = (30, 34, 36), (1.9, 1.8, 1.7), (0.35, 0.6, -0.2)
    rng = np.random.default_rng(11)
    zz, yy, xx = np.meshgrid(*[np.clip(np.rint((o + np.arange(n) * h) / 2.5).astype(int), 0, s - 1)
                               for n, h, o, s in zip(rshape, rsp, ro, ev.shape)], indexing="ij")
    ref = (p.ref[zz, yy, xx] * (1 + rng.normal(0, 0.01, rshape))).astype(np.float32)
    crit = synth.Criteria(0.02, 2.0)
    extra = {"fp64_tau_exp10": 1} if fp64_all else {}
    a, ca, sa = gpu_grids(ref, rsp, ro, ev, (2.5, 2.5, 2.5), (0.0, 0.0, 0.0), crit,
                          {"walk": 0, "lanes_per_voxel": 8, **extra})
    b, cb, sb = gpu_grids(ref, rsp, ro, ev, (2.5, 2.5, 2.5), (0.0, 0.0, 0.0), crit, {"walk": 3, **extra})
    np.testing.assert_array_equal(a, b)
    assert ca == cb
    if fp64_all:
        assert sb["fp64_cells"] > 0
