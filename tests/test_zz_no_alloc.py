"""The allocation-free entry point, gamma_run_noalloc, against the regular path.

Callers whose device memory belongs to their own pool allocator (a planning
or QA application, a framework operator) cannot let a library call
cudaMalloc/cudaFree; gamma_run_noalloc keeps all its scratch in one fixed
array inside the library instead.  This file is collected last on purpose.
It calls the entry point through the C ABI twice in a row, on two different
dose pairs, and checks each gamma map and its counts against
gamma_create + gamma_run on the same inputs, within the parity tolerance
the other GPU tests use.  It also checks that a grid beyond the fixed
capacity is refused with a clear error.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-4


def _crit(g, c):
    return g.criteria(c.dd_frac, c.dta_mm, c.local, c.cutoff_frac, c.dose_norm)


def _regular(g, p, crit):
    ref = torch.from_numpy(p.ref).cuda()
    ev = torch.from_numpy(p.eval).cuda()
    out = torch.empty_like(ref)
    h = g.gamma_create(ref, ev, 3, p.ref.shape, p.spacing, _crit(g, crit))
    try:
        g.gamma_run(h, out)
        _, n_eval, n_pass = g.gamma_pass_rate(h)
    finally:
        g.gamma_destroy(h)
    return out.cpu().numpy().astype(np.float64), (n_eval, n_pass)


def test_noalloc_matches_regular_path_two_calls_in_a_row():
    import paper_1012_1900_gb300 as g
    cases = [
        (synth.workload("imrt_small"), synth.Criteria(0.01, 1.0, local=True)),
        (synth.make_pair_3d(shape=(30, 44, 40), spacing=(2.0, 2.5, 2.0), seed=12,
                            shift_mm=(0.5, 1.0, 2.0), scale=1.04), synth.Criteria(0.02, 2.0)),
    ]
    for p, crit in cases:                      # two calls in a row, different pairs
        want, want_counts = _regular(g, p, crit)
        ref = torch.from_numpy(p.ref).cuda()
        ev = torch.from_numpy(p.eval).cuda()
        out = torch.full_like(ref, -7.0)
        counts = g.gamma_run_noalloc(ref, ev, out, 3, p.ref.shape, p.spacing, _crit(g, crit))
        got = out.cpu().numpy().astype(np.float64)
        assert np.array_equal(np.isnan(got), np.isnan(want))
        ok = ~np.isnan(want)
        assert ok.sum() > 100
        assert np.max(np.abs(got[ok] - want[ok])) <= TOL
        assert counts == want_counts


def test_noalloc_refuses_grids_beyond_its_scratch():
    import paper_1012_1900_gb300 as g
    dummy = torch.zeros(4, device="cuda")
    with pytest.raises(g.GammaError) as e:
        g.gamma_run_noalloc(dummy, dummy, dummy, 2, (1, 2049, 2048), (1.0, 1.0, 1.0),
                            g.criteria(0.03, 3.0))
    assert e.value.code == -11
