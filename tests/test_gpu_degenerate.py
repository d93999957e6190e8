"""Degenerate criteria on the GPU: global criteria need a positive dose norm.

Global Delta D is dd_frac * D_norm (D_norm = the reference maximum unless
given).  A reference with no positive dose and no norm given leaves Delta D
at zero; the oracle refuses such input, and the library evaluates no voxel
(every gamma NaN) and reports GAMMA_ERR_DOSE_NORM from the pass rate, on
every path (coincident grids with each walk, the paper's design, batches,
two grids, the allocation-free call).  The same handle then runs a valid
pair exactly.  A norm given by the caller, or local criteria, need no
positive reference dose.
"""
import numpy as np
import pytest

import synth
from tests.test_gpu_parity import assert_parity, f32, gpu_gamma, oracle_gamma

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DOSE_NORM = -12


def _pair():
    return synth.make_pair_3d(shape=(14, 18, 20), spacing=(2.5, 2.5, 2.5), seed=41,
                              shift_mm=(0.0, 1.0, 1.5), scale=1.03)


def _crit(g, c):
    return g.criteria(c.dd_frac, c.dta_mm, c.local, c.cutoff_frac, c.dose_norm)


@pytest.mark.parametrize("opts", [{}, {"walk": 0}, {"walk": 1}, {"design": 1}, {"graph": 0}],
                         ids=["default", "voxel_walk", "tile_walk", "paper_design", "no_graph"])
def test_zero_reference_under_global_criteria_evaluates_nothing(opts):
    import paper_1012_1900_gb300 as g
    p = _pair()
    zero = np.zeros_like(p.ref)
    crit = synth.Criteria(0.03, 3.0)
    r = torch.from_numpy(zero).cuda()
    e = torch.from_numpy(p.eval).cuda()
    out = torch.full_like(r, -7.0)
    h = g.gamma_create(r, e, 3, p.ref.shape, p.spacing, _crit(g, crit))
    try:
        for k, v in opts.items():
            g.gamma_set_option(h, k, v)
        for _ in range(3):                     # direct launches, then graph capture and replay
            out.fill_(-7.0)
            g.gamma_run(h, out)
            with pytest.raises(g.GammaError) as err:
                g.gamma_pass_rate(h)
            assert err.value.code == DOSE_NORM
            assert np.all(np.isnan(out.cpu().numpy()))
        # the same handle on a valid reference is exact again
        r2 = torch.from_numpy(p.ref).cuda()
        g.gamma_set_inputs(h, r2, e)
        g.gamma_run(h, out)
        counts = g.gamma_pass_rate(h)
        got = out.cpu().numpy().astype(np.float64)
    finally:
        g.gamma_destroy(h)
    assert_parity(got, oracle_gamma(p.ref, p.eval, p.spacing, crit), counts)


def test_zero_reference_with_a_given_norm_or_local_criteria():
    p = _pair()
    zero = np.zeros_like(p.ref)
    # a norm given by the caller: every voxel (cutoff 0) is evaluated, gamma
    # = the oracle's
    crit = synth.Criteria(0.03, 3.0, dose_norm=1.0, cutoff_frac=0.0)
    got, counts, _ = gpu_gamma(zero, p.eval, p.spacing, crit)
    assert counts[1] == zero.size
    assert_parity(got, oracle_gamma(zero, p.eval, p.spacing, crit), counts)
    # local criteria evaluate only voxels with a positive reference dose: none
    crit = synth.Criteria(0.03, 3.0, local=True)
    got, counts, _ = gpu_gamma(zero, p.eval, p.spacing, crit)
    assert counts[1] == 0 and np.all(np.isnan(got))


def test_batch_reports_the_pair_without_a_dose_norm():
    import paper_1012_1900_gb300 as g
    p = _pair()
    q = synth.make_pair_2d(shape=(40, 36), spacing=(1.0, 1.0), seed=42, shift_mm=(0.5, 0.7),
                           scale=1.02, noise_sd=0.005)
    crit = synth.Criteria(0.03, 3.0)
    keep, descs = [], []
    for ref, ev, nd, shape, sp in ((p.ref, p.eval, 3, p.ref.shape, p.spacing),
                                   (np.zeros_like(p.ref), p.eval, 3, p.ref.shape, p.spacing),
                                   (q.ref, q.eval, 2, (1,) + q.ref.shape, (1.0,) + q.spacing)):
        r = torch.from_numpy(np.ascontiguousarray(ref)).cuda()
        e = torch.from_numpy(np.ascontiguousarray(ev)).cuda()
        o = torch.full_like(r, -7.0)
        keep += [r, e, o]
        descs.append((r, e, o, nd, shape, sp, _crit(g, crit)))
    hb = g.gamma_batch_create(descs)
    try:
        for _ in range(2):
            g.gamma_batch_run(hb)
            with pytest.raises(g.GammaError) as err:
                g.gamma_batch_pass_rate(hb, 1)
            assert err.value.code == DOSE_NORM
            with pytest.raises(g.GammaError) as err:
                g.gamma_pass_rate(hb)
            assert err.value.code == DOSE_NORM
            c0 = g.gamma_batch_pass_rate(hb, 0)
            c2 = g.gamma_batch_pass_rate(hb, 2)
        maps = [d[2].cpu().numpy().astype(np.float64) for d in descs]
    finally:
        g.gamma_destroy(hb)
    assert np.all(np.isnan(maps[1]))
    assert_parity(maps[0], oracle_gamma(p.ref, p.eval, p.spacing, crit), c0)
    assert_parity(maps[2], oracle_gamma(q.ref, q.eval, q.spacing, crit), c2)


def test_two_grids_and_noalloc_report_a_missing_dose_norm():
    import paper_1012_1900_gb300 as g
    p = _pair()
    zero = torch.zeros(p.ref.shape, dtype=torch.float32, device="cuda")
    e = torch.from_numpy(p.eval).cuda()
    out = torch.full_like(zero, -7.0)
    crit = _crit(g, synth.Criteria(0.03, 3.0))
    h = g.gamma_create_grids(zero, e, 3, p.ref.shape, p.spacing, (0.0, 0.0, 0.0),
                             p.eval.shape, p.spacing, (0.0, 0.0, 1.0), crit)
    try:
        g.gamma_run(h, out)
        with pytest.raises(g.GammaError) as err:
            g.gamma_pass_rate(h)
        assert err.value.code == DOSE_NORM
    finally:
        g.gamma_destroy(h)
    assert torch.isnan(out).all()
    out.fill_(-7.0)
    with pytest.raises(g.GammaError) as err:
        g.gamma_run_noalloc(zero, e, out, 3, p.ref.shape, p.spacing, crit)
    assert err.value.code == DOSE_NORM
    assert torch.isnan(out).all()
