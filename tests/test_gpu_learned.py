"""GPU checks of the learned proposal: the network's forward and backward
against the FP64 reference with the same bf16 rounding points, features
against their FP64 definition, labels as true nearest surface points,
training that lowers the loss, and runs with a model attached that stay
exactly equal to runs without it."""
import math
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import mlp
from tests import _brute as brute
from tests import _nnbound as nb
from tests.test_gpu_parity import assert_parity, f32, gpu_gamma, oracle_gamma

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _bf16_rows(rng, M):
    X = np.zeros((M, mlp.K_PAD), np.float32)
    X[:, :mlp.K_IN] = rng.normal(0, 1.5, (M, mlp.K_IN))
    Xb = torch.from_numpy(X).to(torch.bfloat16).cuda()
    return Xb, Xb.float().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("M", [300, 1500])
def test_forward_and_backward_match_reference(M):
    # Element by element: every output and every gradient entry within the
    # bound propagated from the bf16 rounding points and FP32 sums
    # (tests/_nnbound.py), and every row and column of each gradient block
    # within 2 % of its own norm.  300 rows: ragged against the 128-row tiles
    # and against the 8-row padding of the batch-contiguous operands; 1,500
    # rows: the weight gradients split their batch sum over blocks.
    import paper_1012_1900_gb300 as g
    rng = np.random.default_rng(3)
    m = g.gamma_model_create(7)
    try:
        Xb, Xq = _bf16_rows(rng, M)
        T = rng.normal(0, 1, (M, 4)).astype(np.float32)
        T[::17, 3] = np.nan
        Tt = torch.from_numpy(T).cuda()
        p = g.gamma_model_get_params(m).astype(np.float64)
        Y = torch.empty((M, 4), device="cuda")
        g.gamma_model_forward(m, Xb, Y)
        f, e = nb.forward_bounds(p, Xq)
        nb.check(Y.cpu().numpy(), f["y"], e["y"], "forward")
        loss = g.gamma_model_backward(m, Xb, Tt)
        want_loss, want_g, e_loss, e_g = nb.backward_bounds(p, Xq, T)
        assert abs(loss - want_loss) <= e_loss + 1e-7
        got_g = g.gamma_model_get_params(m, which=1).astype(np.float64)
        nb.check_grads(got_g, want_g, e_g)
        assert np.all(got_g[~mlp.trainable_mask()] == 0)
    finally:
        g.gamma_model_destroy(m)


@pytest.mark.parametrize("M", [1, 300, 40000])
def test_tensor_core_inference_matches_reference(M):
    # The search's inference kernel (tcgen05 MMAs, TMEM accumulators) against
    # the FP64 network with the same BF16 rounding points, element by element.
    # 300 rows leave a ragged last tile; 40,000 rows give every block several
    # tiles, so the barrier phases carry over between tiles.
    import paper_1012_1900_gb300 as g
    rng = np.random.default_rng(5 + M)
    m = g.gamma_model_create(21)
    try:
        Xb, Xq = _bf16_rows(rng, M)
        p = g.gamma_model_get_params(m).astype(np.float64)
        Y = torch.full((M, 4), float("nan"), device="cuda")
        g.gamma_model_infer(m, Xb, Y)
        got = Y.cpu().numpy().astype(np.float64)
        f, e = nb.forward_bounds(p, Xq)
        assert np.all(np.isfinite(got))
        nb.check(got, f["y"], e["y"], "tensor-core inference")
        Y2 = torch.empty((M, 4), device="cuda")
        g.gamma_model_forward(m, Xb, Y2)                 # the training kernels agree
        nb.check(Y2.cpu().numpy(), f["y"], e["y"], "training forward")
    finally:
        g.gamma_model_destroy(m)


def test_adam_step_and_save_load(tmp_path):
    import paper_1012_1900_gb300 as g
    rng = np.random.default_rng(4)
    m = g.gamma_model_create(11)
    m2 = g.gamma_model_create(12)
    try:
        X = torch.from_numpy(rng.normal(0, 1, (128, mlp.K_PAD)).astype(np.float32)).to(torch.bfloat16).cuda()
        T = torch.from_numpy(rng.normal(0, 1, (128, 4)).astype(np.float32)).cuda()
        p0 = g.gamma_model_get_params(m).astype(np.float64)
        g.gamma_model_backward(m, X, T)
        gr = g.gamma_model_get_params(m, which=1).astype(np.float64)
        g.gamma_model_train_step(m, X, T, 1e-3)
        p1 = g.gamma_model_get_params(m).astype(np.float64)
        # first Adam step: update = lr * g / (|g| + eps) elementwise (eps = 1e-8)
        k = mlp.trainable_mask() & (np.abs(gr) > 1e-7)
        want = 1e-3 * gr[k] / (np.abs(gr[k]) + 1e-8)
        np.testing.assert_allclose((p0 - p1)[k], want, rtol=2e-3, atol=1e-7)
        assert np.all(p1[~mlp.trainable_mask()] == 0)
        path = os.path.join(tmp_path, "m.gmlp")
        g.gamma_model_save(m, path)
        g.gamma_model_load(m2, path)
        assert np.array_equal(g.gamma_model_get_params(m2), g.gamma_model_get_params(m))
    finally:
        g.gamma_model_destroy(m)
        g.gamma_model_destroy(m2)


def _handle(g, p):
    r = torch.from_numpy(p.ref).cuda()
    e = torch.from_numpy(p.eval).cuda()
    c = p.criteria
    h = g.gamma_create(r, e, 3, p.ref.shape, p.spacing,
                       g.criteria(c.dd_frac, c.dta_mm, c.local, c.cutoff_frac, c.dose_norm))
    return h, r, e


@pytest.mark.parametrize("volumes", [False, True], ids=["no_model", "model_attached"])
def test_features_match_definition(volumes):
    # The features of listed voxels, with and without a model attached to the
    # handle (the seeding pass computes the same features for its rows).
    import paper_1012_1900_gb300 as g
    p = synth.workload("imrt_small")
    h, r, e = _handle(g, p)
    m = g.gamma_model_create(3) if volumes else None
    try:
        if volumes:
            g.gamma_set_model(h, m)
        out = torch.empty_like(r)
        g.gamma_run(h, out)
        g.gamma_pass_rate(h)
        rng = np.random.default_rng(0)
        ok = np.nonzero(np.isfinite(out.cpu().numpy().ravel()))[0]
        vox = rng.choice(ok, 40, replace=False).astype(np.int32)
        X = torch.empty((vox.size, 384), dtype=torch.bfloat16, device="cuda")
        g.gamma_features(h, torch.from_numpy(vox).cuda(), X)
        got = X.float().cpu().numpy().astype(np.float64)
    finally:
        g.gamma_destroy(h)
        g.gamma_model_destroy(m)
    c = p.criteria
    want = mlp.bf16_round(mlp.features(p.ref.astype(np.float64), p.eval.astype(np.float64), p.spacing,
                                       f32(c.dd_frac), f32(c.dta_mm), vox))
    assert np.all(np.abs(got - want) <= 2 ** -7 * np.abs(want) + 1e-6)


def test_features_at_grid_edges_and_saturation():
    # The corners, edges and faces of the grid (patches that leave it, one-
    # sided gradients) and a steep pair whose features saturate (dose channel
    # at +-16, gradient channels at 32), element by element against the FP64
    # definition with the same bf16 rounding.
    import paper_1012_1900_gb300 as g
    base = synth.workload("imrt_small")
    steep = synth.Pair("steep", base.ref, (1.25 * base.ref).astype(np.float32), base.spacing,
                       synth.Criteria(0.003, 3.0, cutoff_frac=0.0))
    for p in (synth.Pair(base.name, base.ref, base.eval, base.spacing,
                         synth.Criteria(0.03, 3.0, cutoff_frac=0.0)), steep):
        nz, ny, nx = p.ref.shape
        pts = [(z, y, x) for z in (0, 1, nz - 1) for y in (0, ny - 2, ny - 1) for x in (0, 1, nx - 1)]
        pts += [(nz // 2, ny // 2, x) for x in range(nx)]
        vox = np.array([np.ravel_multi_index(q, p.ref.shape) for q in pts], dtype=np.int32)
        h, r, e = _handle(g, p)
        try:
            out = torch.empty_like(r)
            g.gamma_run(h, out)                       # the dose norm the features use
            g.gamma_pass_rate(h)
            X = torch.empty((vox.size, 384), dtype=torch.bfloat16, device="cuda")
            g.gamma_features(h, torch.from_numpy(vox).cuda(), X)
            got = X.float().cpu().numpy().astype(np.float64)
        finally:
            g.gamma_destroy(h)
        c = p.criteria
        want = mlp.bf16_round(mlp.features(p.ref.astype(np.float64), p.eval.astype(np.float64),
                                           p.spacing, f32(c.dd_frac), f32(c.dta_mm), vox))
        assert np.all(np.abs(got - want) <= 2 ** -7 * np.abs(want) + 1e-6), p.name
        if p.name == "steep":
            assert (np.abs(want[:, :125]) == 16.0).any() and (want[:, 125:375] == 32.0).any()


def test_labels_are_nearest_surface_points():
    import paper_1012_1900_gb300 as g
    p = synth.workload("imrt_small")
    crit = synth.Criteria(0.01, 1.0, local=True)
    p = synth.Pair(p.name, p.ref, p.eval, p.spacing, crit)
    h, r, e = _handle(g, p)
    try:
        out = torch.empty_like(r)
        g.gamma_run(h, out)
        g.gamma_pass_rate(h)
        gm = out.cpu().numpy().ravel().astype(np.float64)
        ok = np.nonzero(np.isfinite(gm) & (gm > 0.9))[0]
        rng = np.random.default_rng(1)
        vox = rng.choice(ok, min(60, ok.size), replace=False).astype(np.int32)
        T = torch.empty((vox.size, 4), device="cuda")
        g.gamma_labels(h, out, torch.from_numpy(vox).cuda(), T)
        T = T.cpu().numpy().astype(np.float64)
    finally:
        g.gamma_destroy(h)
    want = oracle_gamma(p.ref, p.eval, p.spacing, crit, idx=vox)
    hn = np.array(p.spacing[::-1]) / crit.dta_mm                  # x, y, z
    shape = p.ref.shape
    for row, v in enumerate(vox):
        z, y, x = np.unravel_index(v, shape)
        off = T[row, :3] / hn                                        # voxel units (x, y, z)
        pos = np.array([x, y, z]) + off
        de = brute.freudenthal_interpolate(p.eval, pos[None, :])[0]
        dr = float(p.ref.ravel()[v])
        dD = f32(crit.dd_frac) * dr
        dist = math.sqrt(float((T[row, :3] ** 2).sum()) + ((de - dr) / dD) ** 2)
        assert dist == pytest.approx(want[row], abs=2e-4), row
        assert T[row, 3] == pytest.approx(math.log(want[row] + 1e-3), abs=1e-4)


def test_training_lowers_the_loss():
    import paper_1012_1900_gb300 as g
    from paper_1012_1900_gb300 import train
    pairs = [synth.make_pair_3d(shape=(30, 40, 40), spacing=(2.0, 2.0, 2.0), seed=1000 + i,
                                shift_mm=(0.0, 1.0 + i, 2.0), scale=1.0 + 0.02 * i,
                                criteria=synth.Criteria(0.02, 2.0)) for i in range(3)]
    X, T = train.build_dataset(pairs, 3000, seed=0)
    assert X.shape[0] > 1000
    m = g.gamma_model_create(5)
    try:
        losses = train.train(m, X, T, steps=300, batch=1024, lr=3e-3)
    finally:
        g.gamma_model_destroy(m)
    first = float(np.mean(losses[:10]))
    last = float(np.mean(losses[-10:]))
    assert last < 0.5 * first, (first, last)


@pytest.mark.parametrize("gate", [0, 9, 31])
@pytest.mark.parametrize("crit", [synth.Criteria(0.02, 2.0), synth.Criteria(0.01, 1.0, local=True)],
                         ids=["2pct2mm", "1pct1mm_local"])
def test_runs_with_a_model_stay_exact(crit, gate):
    # gate: the seeding pass takes only queued voxels of cost bucket >= gate
    # (0: all of them); the search stays exact whichever voxels are seeded.
    import paper_1012_1900_gb300 as g
    p = synth.make_pair_3d(shape=(24, 36, 32), spacing=(2.0, 2.0, 2.0), seed=2001,
                           shift_mm=(0.5, 1.5, 2.5), scale=1.04, criteria=crit)
    plain, pc, _ = gpu_gamma(p.ref, p.eval, p.spacing, crit)
    m = g.gamma_model_create(9)                 # untrained: any proposal must be safe
    h, r, e = _handle(g, p)
    try:
        g.gamma_set_model(h, m)
        g.gamma_set_option(h, "seed_min_bucket", gate)
        out = torch.empty_like(r)
        g.gamma_run(h, out)
        counts = g.gamma_pass_rate(h)
        st = g.gamma_get_stats(h)
        got = out.cpu().numpy().astype(np.float64)
    finally:
        g.gamma_destroy(h)
        g.gamma_model_destroy(m)
    if gate == 0:
        assert st["seeded"] == st["tail_voxels"] > 0
    else:
        assert st["seeded"] < st["tail_voxels"]
    np.testing.assert_allclose(got, plain, rtol=0, atol=1e-6, equal_nan=True)
    want = oracle_gamma(p.ref, p.eval, p.spacing, crit)
    assert_parity(got, want, counts)
