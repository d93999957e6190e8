"""GPU parity of batched runs: many uneven pairs (2D and 3D, per-pair criteria,
grids with and without TMA-compatible rows) in one graph-captured launch
sequence, each pair checked against the FP64 oracle and against its own
single-pair run."""
import numpy as np
import pytest

import oracle
import synth
from tests.test_gpu_parity import TOL, assert_parity, f32, gpu_gamma, oracle_gamma

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _pairs():
    ps = []
    crits = [synth.Criteria(0.03, 3.0), synth.Criteria(0.02, 2.0), synth.Criteria(0.01, 1.0),
             synth.Criteria(0.01, 1.0, local=True), synth.Criteria(0.03, 1.0, cutoff_frac=0.05)]
    for i in range(5):
        shape = [(48, 64), (37, 53), (64, 40), (29, 31), (56, 56)][i]
        p = synth.make_pair_2d(shape=shape, spacing=(1.0, 1.25), seed=60 + i,
                               shift_mm=(0.3 * i, 1.0 - 0.2 * i), scale=0.98 + 0.015 * i,
                               criteria=crits[i])
        ps.append(p)
    for i in range(5):
        shape = [(16, 24, 20), (13, 19, 23), (20, 28, 32), (11, 17, 15), (18, 22, 26)][i]
        p = synth.make_pair_3d(shape=shape, spacing=(2.5, 2.0, 2.0), seed=70 + i,
                               shift_mm=(0.5, 0.2 * i, 1.5), scale=1.0 + 0.012 * i,
                               criteria=crits[(i + 2) % 5])
        ps.append(p)
    return ps


def _batch_run(ps, options=None, runs=1):
    import paper_1012_1900_gb300 as g
    refs, evs, outs, descs = [], [], [], []
    for p in ps:
        r = torch.from_numpy(p.ref).cuda()
        e = torch.from_numpy(p.eval).cuda()
        o = torch.full_like(r, -7.0)
        refs.append(r)
        evs.append(e)
        outs.append(o)
        nd = p.ref.ndim
        shape = p.ref.shape if nd == 3 else (1,) + p.ref.shape
        sp = p.spacing if nd == 3 else (1.0,) + p.spacing
        c = p.criteria
        descs.append((r, e, o, nd, shape, sp,
                      g.criteria(c.dd_frac, c.dta_mm, c.local, c.cutoff_frac, c.dose_norm)))
    h = g.gamma_batch_create(descs)
    try:
        for k, v in (options or {}).items():
            g.gamma_set_option(h, k, v)
        results = []
        for _ in range(runs):
            g.gamma_batch_run(h)
            counts = [g.gamma_batch_pass_rate(h, i) for i in range(len(ps))]
            results.append(([o.cpu().numpy().astype(np.float64) for o in outs], counts))
        total = g.gamma_pass_rate(h)
    finally:
        g.gamma_destroy(h)
    return results, total


def test_batch_matches_oracle_and_single_runs():
    ps = _pairs()
    (maps, counts), = _batch_run(ps)[0]
    for p, got, cnt in zip(ps, maps, counts):
        want = oracle_gamma(p.ref, p.eval, p.spacing, p.criteria)
        assert_parity(got, want, cnt)
        single, scnt, _ = gpu_gamma(p.ref, p.eval, p.spacing, p.criteria)
        np.testing.assert_allclose(got, single, rtol=0, atol=1e-6, equal_nan=True)


@pytest.mark.parametrize("opts", [{"graph": 0}, {"walk": 0, "lanes_per_voxel": 32, "shell_blocks_per_sm": 1},
                                  {"walk": 0, "lanes_per_voxel": 4}, {"walk": 0, "table_cap": 16},
                                  {"table_cap": 16}, {"group_bucket": 0}, {"group_bucket": 32},
                                  {"group8_bucket": 0}, {"group32_bucket": 0},
                                  {"group_bucket": 5, "group8_bucket": 9, "group32_bucket": 13},
                                  {"tail_blocks_per_sm": 4}, {"tail_blocks_per_sm": 1},
                                  {"group_bucket": -1}, {"group_bucket": -1, "group_auto_pct": 5}])
def test_batch_options_agree(opts):
    # the default batched walk is the warp-evaluated one (walk 3); walk 0
    # is the voxel walk with its lane counts
    ps = _pairs()
    base, _ = _batch_run(ps)
    other, _ = _batch_run(ps, opts)
    for a, b in zip(base[0][0], other[0][0]):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-6, equal_nan=True)
    assert base[0][1] == other[0][1] or opts.get("table_cap")


def test_batch_replays_are_identical_and_totals_add_up():
    ps = _pairs()
    results, total = _batch_run(ps, runs=3)
    for k in range(1, 3):
        for a, b in zip(results[0][0], results[k][0]):
            assert np.array_equal(a, b, equal_nan=True)
    counts = results[-1][1]
    assert total[1] == sum(c[1] for c in counts)
    assert total[2] == sum(c[2] for c in counts)


def test_autotune_single_and_batch():
    import paper_1012_1900_gb300 as g
    p = synth.workload("imrt_small")
    r = torch.from_numpy(p.ref).cuda()
    e = torch.from_numpy(p.eval).cuda()
    o = torch.empty_like(r)
    c = p.criteria
    h = g.gamma_create(r, e, 3, p.ref.shape, p.spacing, g.criteria(c.dd_frac, c.dta_mm))
    try:
        t = g.gamma_autotune(h, o, reps=2)
        assert t["lanes_per_voxel"] in (2, 4, 8, 16, 32) and t["shell_blocks_per_sm"] in (1, 2, 3, 4)
        assert t["tail_blocks_per_sm"] in (1, 2, 3, 4) and t["ms"] > 0
        for k in ("shell_blocks_per_sm", "tail_blocks_per_sm"):
            assert g.gamma_get_option(h, k) == t[k]
        # the queue parts it kept: the fixed thresholds or the choice from the queue
        assert g.gamma_get_option(h, "group_bucket") in (9, -1)
        g.gamma_set_option(h, "group_auto_pct", 250)
        assert g.gamma_get_option(h, "group_auto_pct") == 250
        with pytest.raises(g.GammaError):
            g.gamma_get_option(h, "no_such_option")
        g.gamma_run(h, o)
        g.gamma_pass_rate(h)
    finally:
        g.gamma_destroy(h)
    want = oracle_gamma(p.ref, p.eval, p.spacing, p.criteria)
    assert_parity(o.cpu().numpy().astype(np.float64), want)


@pytest.mark.parametrize("which", ["eval", "ref"])
def test_non_finite_input_reported_per_pair(which):
    # A NaN in one pair's dose (a corner voxel) is reported for that pair only.
    import paper_1012_1900_gb300 as g
    ps = _pairs()[3:7]
    bad = 2
    arr = ps[bad].eval if which == "eval" else ps[bad].ref
    arr[(-1,) * arr.ndim] = np.nan
    tensors, descs = [], []
    for p in ps:
        r, e = torch.from_numpy(p.ref).cuda(), torch.from_numpy(p.eval).cuda()
        o = torch.empty_like(r)
        tensors += [r, e, o]
        nd = p.ref.ndim
        c = p.criteria
        descs.append((r, e, o, nd, p.ref.shape if nd == 3 else (1,) + p.ref.shape,
                      p.spacing if nd == 3 else (1.0,) + p.spacing,
                      g.criteria(c.dd_frac, c.dta_mm, c.local, c.cutoff_frac, c.dose_norm)))
    h = g.gamma_batch_create(descs)
    try:
        g.gamma_batch_run(h)
        for i in range(len(ps)):
            if i == bad:
                with pytest.raises(g.GammaError) as err:
                    g.gamma_batch_pass_rate(h, i)
                assert err.value.code == -3
            else:
                g.gamma_batch_pass_rate(h, i)
    finally:
        g.gamma_destroy(h)


def test_batch_phase_timings_then_graph_runs():
    # "timing" runs a batch by direct launches (its phase events cannot time
    # a replayed graph); switching it off again returns to the captured graph,
    # and every run gives the same maps
    import paper_1012_1900_gb300 as g
    ps = _pairs()
    base, _ = _batch_run(ps)
    refs, evs, outs, descs = [], [], [], []
    for p in ps:
        r = torch.from_numpy(p.ref).cuda()
        e = torch.from_numpy(p.eval).cuda()
        o = torch.full_like(r, -7.0)
        refs.append(r)
        evs.append(e)
        outs.append(o)
        nd = p.ref.ndim
        c = p.criteria
        descs.append((r, e, o, nd, p.ref.shape if nd == 3 else (1,) + p.ref.shape,
                      p.spacing if nd == 3 else (1.0,) + p.spacing,
                      g.criteria(c.dd_frac, c.dta_mm, c.local, c.cutoff_frac, c.dose_norm)))
    h = g.gamma_batch_create(descs)
    try:
        for timing in (0, 1, 1, 0, 0):
            g.gamma_set_option(h, "timing", timing)
            g.gamma_batch_run(h)
            if timing:
                tm = g.gamma_get_timings(h)
                assert tm["shell_ms"] > 0 and tm["tail_ms"] > 0 and tm["prepare_ms"] > 0
                assert tm["total_ms"] >= tm["shell_ms"] + tm["tail_ms"]
            maps = [o.cpu().numpy().astype(np.float64) for o in outs]
            for got, want in zip(maps, base[0][0]):
                np.testing.assert_array_equal(got, want)
    finally:
        g.gamma_destroy(h)
