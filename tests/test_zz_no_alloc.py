"""The allocation-free entry point, gamma_run_noalloc, against the regular path
and the FP64 oracle.

Callers whose device memory belongs to their own pool allocator (a planning
or QA application, a framework operator) cannot let a library call
cudaMalloc/cudaFree: a hidden allocation escapes their memory budget and can
synchronise the whole device.  gamma_run_noalloc keeps all its scratch in one
fixed array inside the library instead.  This file is collected last on
purpose.  It calls the entry point through the C ABI twice in a row on
different dose pairs (3D local and global criteria, and a 2D plane), and
checks each gamma map and its counts against gamma_create + gamma_run on the
same inputs and against the oracle, within the parity tolerance the other
GPU tests use; a pair whose search runs past the fixed-size cell table into
the box scan is checked against the oracle voxel by voxel.  It also checks
that device memory stays as it was across a call, and that a grid beyond the
fixed capacity is refused with a clear error.
"""
import numpy as np
import pytest

import synth
from tests.test_gpu_parity import assert_parity, oracle_gamma

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-4
# cells of the library's fixed cell table (GAMMA_NOALLOC_MAX_TABLE)
MAX_TABLE = 32768


def _crit(g, c):
    return g.criteria(c.dd_frac, c.dta_mm, c.local, c.cutoff_frac, c.dose_norm)


def _geom(p):
    if p.ref.ndim == 2:
        return 2, (1,) + p.ref.shape, (1.0,) + tuple(p.spacing)
    return 3, p.ref.shape, tuple(p.spacing)


def _regular(g, p, crit):
    ndim, shape, sp = _geom(p)
    ref = torch.from_numpy(p.ref).cuda()
    ev = torch.from_numpy(p.eval).cuda()
    out = torch.empty_like(ref)
    h = g.gamma_create(ref, ev, ndim, shape, sp, _crit(g, crit))
    try:
        g.gamma_run(h, out)
        _, n_eval, n_pass = g.gamma_pass_rate(h)
    finally:
        g.gamma_destroy(h)
    return out.cpu().numpy().astype(np.float64), (n_eval, n_pass)


def _noalloc(g, p, crit):
    ndim, shape, sp = _geom(p)
    ref = torch.from_numpy(p.ref).cuda()
    ev = torch.from_numpy(p.eval).cuda()
    out = torch.full_like(ref, -7.0)
    counts = g.gamma_run_noalloc(ref, ev, out, ndim, shape, sp, _crit(g, crit))
    return out.cpu().numpy().astype(np.float64), counts


def test_noalloc_matches_regular_path_and_oracle_two_calls_in_a_row():
    import paper_1012_1900_gb300 as g
    cases = [
        (synth.workload("imrt_small"), synth.Criteria(0.01, 1.0, local=True)),
        (synth.make_pair_3d(shape=(30, 44, 40), spacing=(2.0, 2.5, 2.0), seed=12,
                            shift_mm=(0.5, 1.0, 2.0), scale=1.04), synth.Criteria(0.02, 2.0)),
        (synth.workload("plane_128"), synth.Criteria(0.03, 3.0)),
    ]
    for p, crit in cases:                      # calls in a row, different pairs
        want, want_counts = _regular(g, p, crit)
        got, counts = _noalloc(g, p, crit)
        assert np.array_equal(np.isnan(got), np.isnan(want))
        ok = ~np.isnan(want)
        assert ok.sum() > 100
        assert np.max(np.abs(got[ok] - want[ok])) <= TOL
        assert counts == want_counts
        assert_parity(got, oracle_gamma(p.ref, p.eval, p.spacing, crit),
                      (None,) + tuple(counts))


def test_noalloc_past_its_cell_table_matches_oracle():
    # A flat-topped field with a large uniform dose offset at 1 %/4 mm on 1 mm
    # voxels: gamma reaches ~15 DTA units, i.e. ~60 voxels, far beyond the
    # ~20-voxel radius the fixed table of MAX_TABLE cells covers, so those
    # voxels finish with the exact box scan over the grid.
    import paper_1012_1900_gb300 as g
    base = synth.make_pair_3d(shape=(36, 40, 44), spacing=(1.0, 1.0, 1.0), seed=21,
                              shift_mm=(0.0, 0.0, 0.0), scale=1.0)
    ref = (0.5 + 0.5 * base.ref).astype(np.float32)
    ev = (ref + 0.15).astype(np.float32)
    crit = synth.Criteria(0.01, 4.0, cutoff_frac=0.0)
    p = synth.Pair("offset_plateau", ref, ev, base.spacing, crit)
    got, counts = _noalloc(g, p, crit)
    hn = 1.0 / 4.0                                           # voxel size / DTA
    table_radius_vox = (MAX_TABLE * 3.0 / (4.0 * np.pi)) ** (1.0 / 3.0)
    assert np.nanmax(got) / hn > 1.5 * table_radius_vox      # searched past the table
    rng = np.random.default_rng(7)
    flat = got.ravel()
    order = np.argsort(-np.nan_to_num(flat, nan=-1.0))
    idx = np.unique(np.concatenate([order[:40], rng.choice(flat.size, 160, replace=False)]))
    want = oracle_gamma(p.ref, p.eval, p.spacing, crit, idx=idx)
    assert np.array_equal(np.isnan(flat[idx]), np.isnan(want))
    ok = ~np.isnan(want)
    assert np.max(np.abs(flat[idx][ok] - want[ok])) <= TOL
    assert counts[0] == int(np.isfinite(flat).sum())
    assert counts[1] == int((flat[np.isfinite(flat)] <= 1.0).sum())


def test_noalloc_leaves_device_memory_unchanged():
    import paper_1012_1900_gb300 as g
    p = synth.make_pair_3d(shape=(30, 44, 40), spacing=(2.0, 2.5, 2.0), seed=13,
                           shift_mm=(0.5, 1.0, 2.0), scale=1.04)
    crit = g.criteria(0.02, 2.0)
    ref = torch.from_numpy(p.ref).cuda()
    ev = torch.from_numpy(p.eval).cuda()
    out = torch.empty_like(ref)
    g.gamma_run_noalloc(ref, ev, out, 3, p.ref.shape, p.spacing, crit)   # loads its kernels
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    g.gamma_run_noalloc(ref, ev, out, 3, p.ref.shape, p.spacing, crit, counts=False)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_refuses_grids_beyond_its_scratch():
    import paper_1012_1900_gb300 as g
    dummy = torch.zeros(4, device="cuda")
    with pytest.raises(g.GammaError) as e:
        g.gamma_run_noalloc(dummy, dummy, dummy, 2, (1, 2049, 2048), (1.0, 1.0, 1.0),
                            g.criteria(0.03, 3.0))
    assert e.value.code == -11
