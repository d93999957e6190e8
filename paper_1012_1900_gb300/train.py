"""Training data and training loop of the proposal network.

Orchestration only: labels come from the exact GPU search (gamma_run then
gamma_labels), features from gamma_features, and every forward, backward and
optimiser step runs in the library's kernels (gamma_model_train_step).

Samples are drawn where the network is used: voxels whose gamma exceeds the
first non-zero cell key (the ones the search queues past the key-0 cells),
plus a quarter of uniformly drawn evaluated voxels.
"""
from __future__ import annotations

import math
from typing import Iterable, List, Tuple

import numpy as np

import paper_1012_1900_gb300 as g


def _crit(c):
    return g.criteria(c.dd_frac, c.dta_mm, c.local, c.cutoff_frac, c.dose_norm)


def pair_samples(pair, n: int, rng: np.random.Generator, device="cuda"):
    """(X bf16 [m, 384], T float32 [m, 4]) for up to n voxels of one pair."""
    import torch
    ref = torch.from_numpy(pair.ref).to(device)
    ev = torch.from_numpy(pair.eval).to(device)
    out = torch.empty_like(ref)
    nd = pair.ref.ndim
    shape = pair.ref.shape if nd == 3 else (1,) + pair.ref.shape
    sp = pair.spacing if nd == 3 else (1.0,) + pair.spacing
    h = g.gamma_create(ref, ev, nd, shape, sp, _crit(pair.criteria))
    try:
        g.gamma_run(h, out)
        g.gamma_pass_rate(h)
        gm = out.cpu().numpy().ravel()
        ok = np.isfinite(gm)
        k1 = min(pair.spacing) / pair.criteria.dta_mm
        far = np.nonzero(ok & (gm > k1))[0]
        anyv = np.nonzero(ok)[0]
        if anyv.size == 0:
            return None
        n_far = min(far.size, (3 * n) // 4)
        pick = [rng.choice(far, n_far, replace=False)] if n_far else []
        pick.append(rng.choice(anyv, min(anyv.size, n - n_far), replace=False))
        vox = np.unique(np.concatenate(pick)).astype(np.int32)
        vt = torch.from_numpy(vox).to(device)
        X = torch.empty((vox.size, 384), dtype=torch.bfloat16, device=device)
        T = torch.empty((vox.size, 4), dtype=torch.float32, device=device)
        g.gamma_features(h, vt, X)
        g.gamma_labels(h, out, vt, T)
        torch.cuda.synchronize()
    finally:
        g.gamma_destroy(h)
    keep = torch.isfinite(T[:, 3])
    return X[keep].contiguous(), T[keep].contiguous()


def build_dataset(pairs: Iterable, per_pair: int, seed: int = 0):
    import torch
    rng = np.random.default_rng(seed)
    xs: List = []
    ts: List = []
    for p in pairs:
        s = pair_samples(p, per_pair, rng)
        if s is not None:
            xs.append(s[0])
            ts.append(s[1])
    return torch.cat(xs), torch.cat(ts)


def train(model: int, X, T, steps: int, batch: int = 8192, lr: float = 2e-3, seed: int = 0,
          log_every: int = 0) -> List[float]:
    """Minibatch Adam on (X, T); returns the loss of every step.  The
    learning rate follows a cosine decay to 5 % of lr."""
    import torch
    gen = torch.Generator(device=X.device)
    gen.manual_seed(seed)
    n = X.shape[0]
    losses = []
    for s in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), device=X.device, generator=gen)
        xb = X[idx].contiguous()
        tb = T[idx].contiguous()
        rate = lr * (0.05 + 0.95 * 0.5 * (1 + math.cos(math.pi * s / max(1, steps))))
        loss = g.gamma_model_train_step(model, xb, tb, rate)
        losses.append(loss)
        if log_every and s % log_every == 0:
            print(f"step {s}: loss {loss:.4f}", flush=True)
    return losses


def _gen_training_pair(args):
    import synth
    i, shape = args
    return synth.training_pair(i, shape=shape)


def main(argv=None) -> None:
    """Train the proposal network on the learned-proposal recipe (synthetic
    3D pairs at 2 mm, 2 %/2 mm global, shift U[0, 4] mm, scale U[0.95, 1.05],
    labelled by the exact GPU search) and save it:

        python -m paper_1012_1900_gb300.train --pairs 200 --steps 3000 --out model.gmlp
    """
    import argparse
    import multiprocessing as mp
    import os
    import sys
    import time

    import torch

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--pairs", type=int, default=200)
    ap.add_argument("--shape", type=int, nargs=3, default=(150, 200, 200), metavar=("NZ", "NY", "NX"))
    ap.add_argument("--per-pair", type=int, default=4096, help="training rows drawn per pair")
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=1234)
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    t0 = time.perf_counter()
    m = g.gamma_model_create(a.seed)
    try:
        xs, ts = [], []
        jobs = [(i, tuple(a.shape)) for i in range(a.pairs)]
        with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
            for k in range(0, len(jobs), 16):
                chunk = pool.map(_gen_training_pair, jobs[k:k + 16])
                X, T = build_dataset(chunk, a.per_pair, seed=k)
                xs.append(X)
                ts.append(T)
        X, T = torch.cat(xs), torch.cat(ts)
        losses = train(m, X, T, steps=a.steps, batch=a.batch, lr=a.lr)
        g.gamma_model_save(m, a.out)
    finally:
        g.gamma_model_destroy(m)
    print(f"trained on {X.shape[0]} rows from {a.pairs} pairs in {time.perf_counter() - t0:.1f} s; "
          f"loss {np.mean(losses[:10]):.4f} -> {np.mean(losses[-50:]):.4f}; saved {a.out}", flush=True)


if __name__ == "__main__":
    main()
