"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bar: |gamma_gpu - gamma_oracle| <= 1e-4 absolute on every evaluated voxel,
identical evaluated masks (NaN pattern), and identical pass/fail (gamma <= 1)
except where |gamma_oracle - 1| < 1e-4.  Small grids are compared in full;
the full-size workloads are compared on sampled voxels the oracle computes
one by one, plus properties that hold at any size.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from tests import _brute as brute

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-4
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def f32(x):
    return float(np.float32(x))


def _geom(ref, spacing):
    if ref.ndim == 2:
        return 2, (1,) + ref.shape, (1.0,) + tuple(spacing)
    return 3, ref.shape, tuple(spacing)


def gpu_gamma(ref, ev, spacing, crit, options=None, runs=1):
    import paper_1012_1900_gb300 as g
    ndim, shape, sp = _geom(ref, spacing)
    r = torch.from_numpy(np.ascontiguousarray(ref, dtype=np.float32)).cuda()
    e = torch.from_numpy(np.ascontiguousarray(ev, dtype=np.float32)).cuda()
    out = torch.full_like(r, -7.0)
    h = g.gamma_create(r, e, ndim, shape, sp,
                       g.criteria(crit.dd_frac, crit.dta_mm, crit.local, crit.cutoff_frac,
                                  crit.dose_norm))
    try:
        for k, v in (options or {}).items():
            g.gamma_set_option(h, k, v)
        outs = []
        for _ in range(runs):
            g.gamma_run(h, out)
            counts = g.gamma_pass_rate(h)
            outs.append(out.cpu().numpy().astype(np.float64))
        st = g.gamma_get_stats(h)
    finally:
        g.gamma_destroy(h)
    return (outs[0] if runs == 1 else outs), counts, st


def oracle_gamma(ref, ev, spacing, crit, idx=None, **kw):
    return oracle.gamma(ref, ev, spacing, f32(crit.dd_frac), f32(crit.dta_mm), local=crit.local,
                        cutoff_frac=f32(crit.cutoff_frac), dose_norm=f32(crit.dose_norm),
                        idx=idx, **kw)


def assert_parity(got, want, counts=None):
    assert np.array_equal(np.isnan(got), np.isnan(want)), "evaluated masks differ"
    ok = ~np.isnan(want)
    if not ok.any():
        return 0.0
    err = np.abs(got[ok] - want[ok])
    worst = float(err.max())
    assert worst <= TOL, f"max |dgamma| = {worst:.3e} at {np.argmax(err)}"
    band = np.abs(want[ok] - 1.0) < TOL
    assert np.array_equal((got[ok] <= 1.0)[~band], (want[ok] <= 1.0)[~band]), "pass/fail differs"
    if counts is not None:
        rate, n_eval, n_pass = counts
        gg = got[~np.isnan(got)]
        assert n_eval == gg.size
        assert n_pass == int((gg <= 1.0).sum())
    return worst


# --------------------------------------------------------------------------
# Small grids, compared in full
# --------------------------------------------------------------------------

def test_plane_128_full():
    p = synth.workload("plane_128")
    got, counts, st = gpu_gamma(p.ref, p.eval, p.spacing, p.criteria)
    want = oracle_gamma(p.ref, p.eval, p.spacing, p.criteria)
    assert_parity(got, want, counts)
    assert st["n_eval"] > 1000


@pytest.mark.parametrize("blocks", [1, 2, 3, 4])
def test_plane_larger_than_one_tile_per_block(blocks):
    # More 32x8 tiles than persistent blocks: every block stages tiles into
    # both of its shared-memory buffers (the second one must stay aligned for
    # the tensor copy).
    p = synth.make_pair_2d(shape=(512, 640), spacing=(1.0, 1.0), seed=13, shift_mm=(0.5, 1.2),
                           scale=1.03)
    crit = synth.Criteria(0.02, 2.0)
    got, counts, _ = gpu_gamma(p.ref, p.eval, p.spacing, crit, {"shell_blocks_per_sm": blocks})
    want = oracle_gamma(p.ref, p.eval, p.spacing, crit)
    assert_parity(got, want, counts)


@pytest.mark.parametrize("blocks", [1, 2, 3, 4])
def test_volume_every_shell_register_budget(blocks):
    # 3D, 768 tiles of 32x4x2 voxels: more tiles than persistent blocks at
    # every budget (the 3- and 4-block variants run with register spills).
    p = synth.make_pair_3d(shape=(48, 64, 64), spacing=(2.5, 2.0, 2.0), seed=17,
                           shift_mm=(0.5, -1.0, 1.5), scale=1.02)
    crit = synth.Criteria(0.02, 2.0)
    got, counts, _ = gpu_gamma(p.ref, p.eval, p.spacing, crit, {"shell_blocks_per_sm": blocks})
    want = oracle_gamma(p.ref, p.eval, p.spacing, crit)
    assert_parity(got, want, counts)


@pytest.mark.parametrize("local", [False, True])
def test_plane_ragged(local):
    p = synth.make_pair_2d(shape=(37, 53), spacing=(1.25, 0.8), seed=11, shift_mm=(0.4, -1.1),
                           scale=0.97, noise_sd=0.01)
    crit = synth.Criteria(0.02, 2.0, local=local, cutoff_frac=0.2)
    got, counts, _ = gpu_gamma(p.ref, p.eval, p.spacing, crit)
    want = oracle_gamma(p.ref, p.eval, p.spacing, crit)
    assert_parity(got, want, counts)


CRITS = [synth.Criteria(0.03, 3.0), synth.Criteria(0.02, 2.0), synth.Criteria(0.01, 1.0, local=True),
         synth.Criteria(0.01, 3.0), synth.Criteria(0.03, 1.0, cutoff_frac=0.0)]


@pytest.mark.parametrize("crit", CRITS, ids=lambda c: c.label.replace("/", "_").replace(" ", "_"))
def test_volume_small_full(crit):
    p = synth.workload("imrt_small")
    got, counts, st = gpu_gamma(p.ref, p.eval, p.spacing, crit)
    want = oracle_gamma(p.ref, p.eval, p.spacing, crit)
    assert_parity(got, want, counts)


def test_volume_ragged_anisotropic():
    p = synth.make_pair_3d(shape=(19, 33, 29), spacing=(3.0, 2.0, 1.5), seed=21,
                           shift_mm=(1.0, -0.5, 2.0), scale=1.05)
    crit = synth.Criteria(0.02, 2.0, cutoff_frac=0.05)
    got, counts, _ = gpu_gamma(p.ref, p.eval, p.spacing, crit)
    want = oracle_gamma(p.ref, p.eval, p.spacing, crit)
    assert_parity(got, want, counts)


@pytest.mark.parametrize("lanes", [2, 4, 8, 16, 32])
@pytest.mark.parametrize("sort_tail,tail_blocks", [(0, 1), (1, 2), (1, 1), (1, 3), (0, 3)])
def test_launch_shapes_agree(lanes, sort_tail, tail_blocks):
    p = synth.workload("imrt_small")
    crit = synth.Criteria(0.01, 1.0, local=True)
    got, counts, _ = gpu_gamma(p.ref, p.eval, p.spacing, crit,
                               {"walk": 0, "lanes_per_voxel": lanes, "sort_tail": sort_tail,
                                "tail_blocks_per_sm": tail_blocks})
    want = oracle_gamma(p.ref, p.eval, p.spacing, crit)
    assert_parity(got, want, counts)


@pytest.mark.parametrize("walk", [0, 3])
@pytest.mark.parametrize("ndim", [2, 3])
def test_truncated_table_box_scan(ndim, walk):
    # A tiny table forces most voxels past its end, into the box scan (for
    # walk = 3, in its finishing pass).
    if ndim == 2:
        p = synth.make_pair_2d(shape=(30, 26), seed=5, shift_mm=(2.0, 1.0), scale=1.06)
    else:
        p = synth.make_pair_3d(shape=(14, 18, 16), spacing=(2.0, 2.0, 2.0), seed=6,
                               shift_mm=(1.0, 2.0, 2.5), scale=1.06)
    crit = synth.Criteria(0.01, 1.0, local=True)
    got, counts, st = gpu_gamma(p.ref, p.eval, p.spacing, crit, {"table_cap": 16, "walk": walk})
    assert st["overflow_voxels"] > 0
    want = oracle_gamma(p.ref, p.eval, p.spacing, crit)
    assert_parity(got, want, counts)


@pytest.mark.parametrize("case", ["plane_128", "volume_local", "volume_ragged", "truncated_3d",
                                  "truncated_2d", "unsorted"])
@pytest.mark.parametrize("blocks", [1, 3])
@pytest.mark.parametrize("walk", [1, 2, 3], ids=["tiles", "rows", "warp_cells"])
def test_staged_walks(case, blocks, walk):
    # Options walk = 1 / 2: the queued voxels walked tile by tile or warp row
    # by warp row from a TMA-staged halo box (cells beyond the box read global
    # memory; a tiny table sends voxels into the box scan; "unsorted" takes the
    # tiles or rows in discovery order).  walk = 3: voxel by voxel, one lane
    # each, the surviving cells evaluated by the whole warp.
    opts = {"walk": walk, "tail_blocks_per_sm": blocks}
    if case == "plane_128":
        p, crit = synth.workload("plane_128"), synth.Criteria(0.03, 3.0)
    elif case in ("volume_local", "unsorted"):
        p, crit = synth.workload("imrt_small"), synth.Criteria(0.01, 1.0, local=True)
        if case == "unsorted":
            opts["sort_tail"] = 0
    elif case == "volume_ragged":
        p = synth.make_pair_3d(shape=(19, 33, 29), spacing=(3.0, 2.0, 1.5), seed=21,
                               shift_mm=(1.0, -0.5, 2.0), scale=1.05)
        crit = synth.Criteria(0.02, 2.0, cutoff_frac=0.05)
    elif case == "truncated_3d":
        p = synth.make_pair_3d(shape=(14, 18, 16), spacing=(2.0, 2.0, 2.0), seed=6,
                               shift_mm=(1.0, 2.0, 2.5), scale=1.06)
        crit = synth.Criteria(0.01, 1.0, local=True)
        opts["table_cap"] = 16
    else:
        p = synth.make_pair_2d(shape=(30, 26), seed=5, shift_mm=(2.0, 1.0), scale=1.06)
        crit = synth.Criteria(0.01, 1.0, local=True)
        opts["table_cap"] = 16
    got, counts, st = gpu_gamma(p.ref, p.eval, p.spacing, crit, opts, runs=2)
    if case.startswith("truncated"):
        assert st["overflow_voxels"] > 0
    want = oracle_gamma(p.ref, p.eval, p.spacing, crit)
    for g_ in got:                                   # a direct run, then the graph replay
        assert_parity(g_, want, counts)


@pytest.mark.parametrize("crit", [(0.03, 3.0, False), (0.01, 1.0, True)], ids=["3-3", "1-1-local"])
@pytest.mark.parametrize("groups", [(0, 32, 32), (32, 0, 32), (32, 32, 0), (9, 32, 32), (32, 32, 32),
                                    (5, 9, 13)],
                         ids=["all4", "all8", "all32", "default", "none", "tiers"])
@pytest.mark.parametrize("blocks", [1, 2, 3, 4])
def test_warp_evaluated_walk_is_bitwise_the_voxel_walk(crit, groups, blocks):
    # walk = 3 evaluates every cell with the same arithmetic as walk = 0 and
    # reaches the same minimising cell, so the two maps agree bit for bit,
    # whichever voxels walk four, eight or 32 lanes each (a threshold of 0:
    # all of them; 32: none) and at every register budget
    p = synth.workload("imrt_small")
    c = synth.Criteria(crit[0], crit[1], local=crit[2])
    a, ca, sa = gpu_gamma(p.ref, p.eval, p.spacing, c, {"walk": 0, "lanes_per_voxel": 2, "stats": 1})
    b, cb, sb = gpu_gamma(p.ref, p.eval, p.spacing, c, {"walk": 3, "stats": 1, "group_bucket": groups[0],
                                                      "group8_bucket": groups[1],
                                                      "group32_bucket": groups[2],
                                                      "tail_blocks_per_sm": blocks})
    np.testing.assert_array_equal(a, b)
    assert ca == cb
    assert sb["tail_voxels"] == sa["tail_voxels"] > 0
    assert sb["cells_visited"] > 0 and sb["cells_keyed"] > 0


@pytest.mark.parametrize("design", [1, 2])
@pytest.mark.parametrize("face_eval", [0, 1])
@pytest.mark.parametrize("ndim", [2, 3])
def test_paper_design_ablation(design, face_eval, ndim):
    # The paper's own GPU design (one thread per voxel, DD-sorted or not; all
    # faces in closed form or Ju's recursion) must give the same map.
    if ndim == 2:
        p = synth.make_pair_2d(shape=(61, 47), spacing=(1.0, 1.25), seed=21, shift_mm=(0.9, -1.3),
                               scale=1.03, noise_sd=0.01)
        crit = synth.Criteria(0.02, 2.0)
    else:
        p = synth.workload("imrt_small")
        crit = synth.Criteria(0.01, 1.0, local=True)
    got, counts, _ = gpu_gamma(p.ref, p.eval, p.spacing, crit, {"design": design, "face_eval": face_eval})
    want = oracle_gamma(p.ref, p.eval, p.spacing, crit)
    assert_parity(got, want, counts)


@pytest.mark.parametrize("face_eval", [0, 1])
def test_paper_design_truncated_table(face_eval):
    p = synth.make_pair_3d(shape=(14, 18, 16), spacing=(2.0, 2.0, 2.0), seed=6,
                           shift_mm=(1.0, 2.0, 2.5), scale=1.06)
    crit = synth.Criteria(0.01, 1.0, local=True)
    got, counts, st = gpu_gamma(p.ref, p.eval, p.spacing, crit,
                                {"table_cap": 16, "design": 1, "face_eval": face_eval})
    assert st["overflow_voxels"] > 0
    want = oracle_gamma(p.ref, p.eval, p.spacing, crit)
    assert_parity(got, want, counts)


@pytest.mark.parametrize("walk", [0, 3])
def test_fp64_redo_paths(walk):
    # walk = 3 leaves voxels with a near-singular cell to its finishing pass
    p = synth.workload("imrt_small")
    crit = synth.Criteria(0.01, 1.0, local=True)
    want = oracle_gamma(p.ref, p.eval, p.spacing, crit)
    g_off, c_off, s_off = gpu_gamma(p.ref, p.eval, p.spacing, crit, {"fp64_tau_exp10": 0, "walk": walk})
    g_all, c_all, s_all = gpu_gamma(p.ref, p.eval, p.spacing, crit, {"fp64_tau_exp10": 1, "walk": walk})
    assert s_off["fp64_cells"] == 0
    assert s_all["fp64_cells"] > 0
    assert_parity(g_off, want, c_off)
    e_all = assert_parity(g_all, want, c_all)
    assert e_all <= 1e-5
    if walk == 3:
        g0, c0, _ = gpu_gamma(p.ref, p.eval, p.spacing, crit, {"fp64_tau_exp10": 1, "walk": 0})
        np.testing.assert_array_equal(g_all, g0)
        assert c_all == c0


def test_identical_doses_zero_and_flat_shift():
    p = synth.workload("imrt_small")
    crit = synth.Criteria(0.03, 3.0)
    got, counts, _ = gpu_gamma(p.ref, p.ref, p.spacing, crit)
    ok = ~np.isnan(got)
    assert ok.sum() > 100 and np.all(got[ok] == 0.0)
    ref = np.full((9, 10, 11), 0.5, np.float32)
    ev = ref + np.float32(0.0625)
    crit = synth.Criteria(0.02, 3.0, dose_norm=1.0, cutoff_frac=0.0)
    got, counts, _ = gpu_gamma(ref, ev, (2.5, 1.0, 2.0), crit)
    np.testing.assert_allclose(got, 0.0625 / f32(0.02), rtol=2e-6)


def test_linear_ramp_closed_form():
    shape, sp = (12, 13, 14), (2.0, 1.25, 1.5)
    grad = np.array([0.004, 0.009, -0.006])
    coords = np.meshgrid(*[np.arange(n) * h for n, h in zip(shape, sp)], indexing="ij")
    ramp = 0.6 + sum(g_ * c for g_, c in zip(grad, coords))
    ref = ramp.astype(np.float32)
    ev = (ramp - 0.0125).astype(np.float32)
    crit = synth.Criteria(0.02, 3.0, dose_norm=1.0, cutoff_frac=0.0)
    got, _, _ = gpu_gamma(ref, ev, sp, crit)
    dD = f32(0.02)
    want = 0.0125 / dD / np.sqrt(1.0 + np.sum((grad * 3.0 / dD) ** 2))
    inner = tuple(slice(3, -3) for _ in shape)
    np.testing.assert_allclose(got[inner], want, atol=2e-5)


@pytest.mark.parametrize("name", ["freudenthal_corner_2d.txt", "freudenthal_corner_3d.txt"])
def test_tiny_golden_grids(name):
    ref, ev, sp, c, expect = brute.read_golden(os.path.join(GOLDEN, name))
    crit = synth.Criteria(c["dd_frac"], c["dta_mm"], cutoff_frac=c["cutoff_frac"],
                          dose_norm=c["dose_norm"])
    got, _, _ = gpu_gamma(ref, ev, sp, crit)
    for flat, value, expr in expect:
        assert abs(got.ravel()[flat] - value) <= 1e-6, expr


@pytest.mark.parametrize("where", [(3, 4, 5), (0, 0, 0), (-1, -1, -1), (-1, 0, -1)])
@pytest.mark.parametrize("which,value", [("eval", np.nan), ("eval", np.inf), ("ref", np.nan),
                                         ("ref", -np.inf)])
def test_non_finite_input_reported(where, which, value):
    # The reference dose is checked by the dose-norm pass, the evaluation dose
    # by the shell (every value is the centre of one tile voxel), corners too.
    import paper_1012_1900_gb300 as g
    p = synth.workload("imrt_small")
    ref, ev = p.ref.copy(), p.eval.copy()
    (ev if which == "eval" else ref)[where] = value
    with pytest.raises(g.GammaError) as e:
        gpu_gamma(ref, ev, p.spacing, p.criteria)
    assert e.value.code == -3


@pytest.mark.parametrize("which", ["eval", "ref"])
def test_non_finite_input_reported_on_host_runs(which):
    import paper_1012_1900_gb300 as g
    p = synth.workload("imrt_small")
    ref, ev = p.ref.copy(), p.eval.copy()
    (ev if which == "eval" else ref)[-1, 7, 0] = np.nan
    crit = p.criteria
    h = g.gamma_create(None, None, 3, p.ref.shape, p.spacing,
                       g.criteria(crit.dd_frac, crit.dta_mm, cutoff_frac=crit.cutoff_frac))
    try:
        for pipe in (4, 0):
            g.gamma_set_option(h, "pipeline", pipe)
            r = torch.from_numpy(ref).pin_memory()
            e = torch.from_numpy(ev).pin_memory()
            o = torch.empty_like(r).pin_memory()
            g.gamma_run_host(h, r, e, o)
            with pytest.raises(g.GammaError) as err:
                g.gamma_pass_rate(h)
            assert err.value.code == -3
    finally:
        g.gamma_destroy(h)


def test_repeat_runs_identical_and_counters_reset():
    p = synth.workload("imrt_small")
    outs, counts, st = gpu_gamma(p.ref, p.eval, p.spacing, synth.Criteria(0.02, 2.0), runs=3)
    assert np.array_equal(outs[0], outs[1], equal_nan=True)
    assert np.array_equal(outs[0], outs[2], equal_nan=True)
    assert counts[1] == int((~np.isnan(outs[2])).sum())


@pytest.mark.parametrize("name", ["imrt_small", "plane_128"])
@pytest.mark.parametrize("mode", ["pipelined", "one_slab", "eight_slabs", "in_order", "pageable"])
def test_run_host_matches_device_run(name, mode):
    # Pinned buffers take the overlapped path (z slabs of the evaluation dose,
    # map copied out during the table walk, queued voxels patched through the
    # mapped address); option "pipeline" = 0 and pageable arrays run in order.
    # Every path must give the device run's map bit for bit, on every run.
    import paper_1012_1900_gb300 as g
    p = synth.workload(name)
    crit = synth.Criteria(0.03, 3.0)
    dev_out, dev_counts, _ = gpu_gamma(p.ref, p.eval, p.spacing, crit)
    ndim, shape, sp = _geom(p.ref, p.spacing)
    h = g.gamma_create(None, None, ndim, shape, sp,
                       g.criteria(crit.dd_frac, crit.dta_mm, cutoff_frac=crit.cutoff_frac))
    try:
        slabs = {"in_order": 0, "one_slab": 1, "eight_slabs": 8}
        if mode in slabs:
            g.gamma_set_option(h, "pipeline", slabs[mode])
        if mode == "pageable":
            ref, ev = np.ascontiguousarray(p.ref), np.ascontiguousarray(p.eval)
            out = np.empty_like(ref)
            view = lambda: out
        else:
            ref = torch.from_numpy(p.ref).pin_memory()
            ev = torch.from_numpy(p.eval).pin_memory()
            out = torch.empty_like(ref).pin_memory()
            view = lambda: out.numpy()
        for _ in range(3):
            view()[...] = -7.0
            g.gamma_run_host(h, ref, ev, out)
            counts = g.gamma_pass_rate(h)
            assert np.array_equal(view().astype(np.float64).reshape(dev_out.shape), dev_out,
                                  equal_nan=True)
            assert counts == dev_counts
    finally:
        g.gamma_destroy(h)


@pytest.mark.parametrize("pct", [5, 100, 2000])
def test_queue_parts_chosen_from_the_queue(pct):
    # group_bucket -1: the walk picks its 4-, 8- and 32-lane parts from the
    # queue; only the lanes per voxel change, so the map is the default one
    p = synth.workload("imrt_small")
    crit = synth.Criteria(0.01, 1.0, local=True)
    base, _, _ = gpu_gamma(p.ref, p.eval, p.spacing, crit)
    got, counts, _ = gpu_gamma(p.ref, p.eval, p.spacing, crit, {"group_bucket": -1, "group_auto_pct": pct})
    np.testing.assert_array_equal(got, base)
    assert_parity(got, oracle_gamma(p.ref, p.eval, p.spacing, crit), counts)


def test_stats_mode_counts_cells():
    p = synth.workload("imrt_small")
    crit = synth.Criteria(0.01, 1.0, local=True)
    _, _, st = gpu_gamma(p.ref, p.eval, p.spacing, crit, {"stats": 1})
    assert st["tail_voxels"] > 0
    assert st["cells_visited"] > 0 and st["cells_pruned"] > 0
    # keyed cells whose corner falls outside the grid are neither visited nor pruned
    assert st["cells_keyed"] >= st["cells_visited"] + st["cells_pruned"]
    # the default walk's lane slots: whole warp steps, and every keyed cell takes one
    assert st["lane_slot_steps"] > 0 and st["lane_slot_steps"] % 32 == 0
    assert st["lane_slot_steps"] >= st["cells_keyed"]
    _, _, st0 = gpu_gamma(p.ref, p.eval, p.spacing, crit, {"stats": 1, "walk": 0})
    assert st0["lane_slot_steps"] == 0 and st0["cells_keyed"] > 0


# --------------------------------------------------------------------------
# Full-size workloads: sampled voxels + properties at any size
# --------------------------------------------------------------------------

def _sample(got, n, seed):
    rng = np.random.default_rng(seed)
    ev = np.nonzero(~np.isnan(got.ravel()))[0]
    pick = rng.choice(ev, min(n, ev.size), replace=False)
    # always include the largest gammas (the longest searches)
    top = ev[np.argsort(got.ravel()[ev])[-200:]]
    return np.unique(np.concatenate([pick, top]))


def _full_size_check(p, crit, n_sample, table_cap=1 << 22):
    got, counts, st = gpu_gamma(p.ref, p.eval, p.spacing, crit)
    ok = ~np.isnan(got)
    # mask from the cutoff rule, in float32 as specified
    dn = np.float32(crit.dose_norm) if crit.dose_norm > 0 else p.ref.max()
    thr = np.float32(np.float32(crit.cutoff_frac) * dn)
    mask = p.ref >= thr
    if crit.local:
        mask &= p.ref > 0
    assert np.array_equal(ok, mask)
    # 0 <= gamma <= gamma0 everywhere
    dD = np.broadcast_to(np.float32(crit.dd_frac) * (p.ref if crit.local else dn),
                         p.ref.shape).astype(np.float64)
    g0 = np.abs(p.eval.astype(np.float64) - p.ref)[ok] / dD[ok]
    assert np.all(got[ok] >= 0)
    assert np.all(got[ok] <= g0 * (1 + 1e-6) + 1e-6)
    idx = _sample(got, n_sample, 7)
    want = oracle_gamma(p.ref, p.eval, p.spacing, crit, idx=idx, table_cap=table_cap)
    worst = assert_parity(got.ravel()[idx], want)
    rate, n_eval, n_pass = counts
    assert n_eval == int(ok.sum()) and n_pass == int((got[ok] <= 1).sum())
    return worst, st


def test_imrt_160_3pct3mm_sampled():
    p = synth.workload("imrt_160")
    worst, st = _full_size_check(p, p.criteria, 20000)
    assert st["tail_voxels"] > 0


def test_imrt_160_2pct2mm_sampled():
    p = synth.workload("imrt_160_2mm2pct")
    _full_size_check(p, p.criteria, 20000)


def test_imrt_320_local_sampled():
    p = synth.workload("imrt_320_local")
    _full_size_check(p, p.criteria, 4000, table_cap=1 << 20)


def test_fp32_peak_probe_confirms_the_derived_peak():
    # The search's roofline is quoted against SMs x 128 FP32 lanes x 2 FLOP x
    # clock; a measured FMA loop must land below that at the 2070 MHz maximum
    # clock (it cannot beat the lanes) and not far below it.
    import paper_1012_1900_gb300 as g
    r = g.gamma_measure_fp32_peak()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    derived = n_sm * 128 * 2 * 2070e6 / 1e12
    assert 0.5 * derived < r["tflops"] < 1.02 * derived, (r, derived)
    assert r["ms"] > 0.1


def test_slab_gate_timeout_is_reported_and_the_next_run_recovers():
    # Failure made on the host: the readiness flag of one evaluation-dose slab
    # is never written, so the gated shell's bounded wait gives up.  The run
    # must report GAMMA_ERR_TIMEOUT (not hang or fault), and the same handle's
    # next run must be exact again.
    import paper_1012_1900_gb300 as g
    p = synth.workload("imrt_small")
    crit = synth.Criteria(0.03, 3.0)
    dev_out, dev_counts, _ = gpu_gamma(p.ref, p.eval, p.spacing, crit)
    h = g.gamma_create(None, None, 3, p.ref.shape, p.spacing,
                       g.criteria(crit.dd_frac, crit.dta_mm, cutoff_frac=crit.cutoff_frac))
    try:
        ref = torch.from_numpy(p.ref).pin_memory()
        ev = torch.from_numpy(p.eval).pin_memory()
        out = torch.empty_like(ref).pin_memory()
        g.gamma_set_option(h, "timing", 1)
        g.gamma_set_option(h, "pipeline", 4)
        g.gamma_run_host(h, ref, ev, out)
        g.gamma_pass_rate(h)
        if g.gamma_get_timings(h)["overlapped"] != 2:
            pytest.skip("the slab gate is not available on this device")
        g.gamma_set_option(h, "drop_slab_flag", 2)
        g.gamma_run_host(h, ref, ev, out)
        with pytest.raises(g.GammaError) as err:
            g.gamma_pass_rate(h)
        assert err.value.code == -6                      # GAMMA_ERR_TIMEOUT
        g.gamma_set_option(h, "drop_slab_flag", 0)
        out.numpy()[...] = -7.0
        g.gamma_run_host(h, ref, ev, out)
        assert g.gamma_pass_rate(h) == dev_counts
        assert np.array_equal(out.numpy().astype(np.float64), dev_out, equal_nan=True)
    finally:
        g.gamma_destroy(h)


def test_graph_replay_matches_direct_launches():
    # Single-pair runs are captured once the same output has been run twice
    # with no option change between, then replayed.  Replays, a recapture after
    # an option change and a new output tensor must all give the direct map.
    import paper_1012_1900_gb300 as g
    p = synth.workload("imrt_small")
    c = synth.Criteria(0.02, 2.0)
    ndim, shape, sp = _geom(p.ref, p.spacing)
    r = torch.from_numpy(p.ref).cuda()
    e = torch.from_numpy(p.eval).cuda()
    crit = g.criteria(c.dd_frac, c.dta_mm, cutoff_frac=c.cutoff_frac)
    h0 = g.gamma_create(r, e, ndim, shape, sp, crit)
    h = g.gamma_create(r, e, ndim, shape, sp, crit)
    try:
        g.gamma_set_option(h0, "graph", 0)
        ref_out = torch.empty_like(r)
        g.gamma_run(h0, ref_out)
        want = ref_out.cpu().numpy()
        want_counts = g.gamma_pass_rate(h0)
        out = torch.empty_like(r)
        for k in range(6):
            if k == 3:                                  # drops the captured graph
                for hh in (h, h0):
                    g.gamma_set_option(hh, "lanes_per_voxel", 16)
                g.gamma_run(h0, ref_out)
                want = ref_out.cpu().numpy()
                want_counts = g.gamma_pass_rate(h0)
            out.fill_(-7.0)
            g.gamma_run(h, out)
            assert g.gamma_pass_rate(h) == want_counts
            assert np.array_equal(out.cpu().numpy(), want, equal_nan=True)
        other = torch.full_like(r, -7.0)
        g.gamma_run(h, other)
        g.gamma_run(h, other)
        assert np.array_equal(other.cpu().numpy(), want, equal_nan=True)
    finally:
        g.gamma_destroy(h0)
        g.gamma_destroy(h)


def test_imrt_320_global_sampled():
    p = synth.workload("imrt_320_global")
    _full_size_check(p, p.criteria, 6000)


def test_plane_128_host_run_matches_oracle():
    # The 2D workload through the overlapped host-buffer path, in full.
    import paper_1012_1900_gb300 as g
    p = synth.workload("plane_128")
    c = p.criteria
    ndim, shape, sp = _geom(p.ref, p.spacing)
    h = g.gamma_create(None, None, ndim, shape, sp,
                       g.criteria(c.dd_frac, c.dta_mm, cutoff_frac=c.cutoff_frac))
    try:
        r = torch.from_numpy(p.ref).pin_memory()
        e = torch.from_numpy(p.eval).pin_memory()
        o = torch.empty_like(r).pin_memory()
        g.gamma_run_host(h, r, e, o)
        counts = g.gamma_pass_rate(h)
    finally:
        g.gamma_destroy(h)
    want = oracle_gamma(p.ref, p.eval, p.spacing, c)
    assert_parity(o.numpy().astype(np.float64), want, counts)
