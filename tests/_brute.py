"""Independent brute-force gamma routines used to pin the oracle.

None of this calls the oracle or the CUDA path.  They restate the definition
(Eq. 1, Section 2.1: minimum normalised dose-distance to the evaluation
surface) in the most direct way available at tiny sizes:

* closed-simplex distance by KKT enumeration: the nearest point of a simplex
  lies in the relative interior of exactly one sub-face, where it equals the
  orthogonal projection onto that sub-face's affine hull; so the distance is
  the minimum, over all sub-faces whose projection has non-negative
  barycentric weights, of the projection distance;
* exhaustive gamma: minimum over every simplex of the grid, no table, no
  radius, no early exit;
* fine-grid gamma: the piecewise-linear (Freudenthal) interpolant sampled on a
  grid `f` times finer, minimum over the samples (an upper bound);
* 1D polylines: a profile that varies along one axis only has, over every
  triangulation, the polyline through its samples as its surface cross-section.
"""
from __future__ import annotations

import itertools
from typing import Sequence

import numpy as np


def normalised_nodes(shape, spacing, dta):
    """Normalised spatial coordinates (x/dta, y/dta[, z/dta]) of every node, in
    the axis order (x, y[, z]), as an array (..., n)."""
    axes = [np.arange(n) * h / dta for n, h in zip(shape, spacing)]
    grids = np.meshgrid(*axes, indexing="ij")          # (z, y, x) order
    return np.stack(grids[::-1], axis=-1)               # last dim: x, y, z


def freudenthal_simplices(shape):
    """Vertex flat-indices of every simplex of the Freudenthal triangulation
    of a grid with the given (z, y, x) / (y, x) shape: (S, n + 1) ints."""
    n = len(shape)
    strides = np.cumprod((1,) + tuple(shape[::-1]))[:-1]   # strides of x, y, z
    corners = itertools.product(*[range(s - 1) for s in shape[::-1]])  # x, y, z
    out = []
    for c in corners:
        base = int(np.dot(c, strides))
        for perm in itertools.permutations(range(n)):
            v = [base]
            cur = base
            for ax in perm:
                cur += int(strides[ax])
                v.append(cur)
            out.append(v)
    return np.array(out, dtype=np.int64)


def closed_simplex_distance(W: np.ndarray, P: np.ndarray) -> np.ndarray:
    """Distances from points P (V, K) to closed simplices W (S, nv, K) by KKT
    enumeration over every sub-face.  Returns (V, S)."""
    Vn = P.shape[0]
    S, nv, K = W.shape
    best = np.full((Vn, S), np.inf)
    for r in range(1, nv + 1):
        for sub in itertools.combinations(range(nv), r):
            base = W[:, sub[0], :]                          # (S, K)
            b = P[:, None, :] - base[None, :, :]            # (V, S, K)
            if r == 1:
                best = np.minimum(best, np.sqrt((b * b).sum(-1)))
                continue
            E = W[:, list(sub[1:]), :] - base[:, None, :]   # (S, m, K)
            G = np.einsum("smk,snk->smn", E, E)
            Ginv = np.linalg.inv(G)
            rhs = np.einsum("smk,vsk->vsm", E, b)
            mu = np.einsum("smn,vsn->vsm", Ginv, rhs)       # (V, S, m)
            w0 = 1.0 - mu.sum(-1)
            ok = (mu >= -1e-13).all(-1) & (w0 >= -1e-13)
            res = b - np.einsum("vsm,smk->vsk", mu, E)
            d = np.sqrt((res * res).sum(-1))
            best = np.minimum(best, np.where(ok, d, np.inf))
    return best


def _resolve(ref, dd_frac, local, cutoff_frac, dose_norm):
    dnorm = dose_norm if dose_norm > 0 else float(ref.max())
    r = ref.astype(np.float64).ravel()
    dD = dd_frac * (r if local else np.full_like(r, dnorm))
    mask = r >= cutoff_frac * dnorm
    if local:
        mask &= r > 0
    return dD, mask


def exhaustive_gamma(ref, ev, spacing, dd_frac, dta, local=False, cutoff_frac=0.0,
                     dose_norm=0.0, chunk=64):
    """Minimum over every simplex of the grid (closed-simplex distances)."""
    shape = ref.shape
    n = ref.ndim
    nodes = normalised_nodes(shape, spacing, dta).reshape(-1, n)
    e = ev.astype(np.float64).ravel()
    r = ref.astype(np.float64).ravel()
    dD, mask = _resolve(ref, dd_frac, local, cutoff_frac, dose_norm)
    simp = freudenthal_simplices(shape)
    out = np.full(r.size, np.nan)
    vox = np.nonzero(mask)[0]
    for s in range(0, vox.size, chunk):
        vv = vox[s:s + chunk]
        # dose scale differs per voxel in local mode: group by unique dD
        for scale in np.unique(dD[vv]):
            sel = vv[dD[vv] == scale]
            W = np.concatenate([nodes[simp], (e[simp] / scale)[..., None]], axis=-1)
            P = np.concatenate([nodes[sel], (r[sel] / scale)[:, None]], axis=-1)
            out[sel] = closed_simplex_distance(W, P).min(axis=1)
    return out.reshape(shape)


def freudenthal_interpolate(ev: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Evaluate the Freudenthal piecewise-linear interpolant of ev at points X
    given in voxel units, X[..., d] along axis d of (x, y[, z])."""
    shape_xyz = ev.shape[::-1]
    n = len(shape_xyz)
    flat = ev.astype(np.float64).ravel()
    strides = np.cumprod((1,) + tuple(shape_xyz))[:-1]
    base = np.floor(X).astype(np.int64)
    for d in range(n):
        base[..., d] = np.clip(base[..., d], 0, shape_xyz[d] - 2)
    t = X - base
    order = np.argsort(-t, axis=-1, kind="stable")
    lin = (base * strides).sum(-1)
    val = flat[lin].copy()
    prev = val.copy()
    cur = lin.copy()
    for i in range(n):
        ax = order[..., i]
        cur = cur + strides[ax]
        nxt = flat[cur]
        ti = np.take_along_axis(t, ax[..., None], axis=-1)[..., 0]
        val += ti * (nxt - prev)
        prev = nxt
    return val


def fine_grid_gamma(ref, ev, spacing, dd_frac, dta, factor, local=False, cutoff_frac=0.0,
                    dose_norm=0.0):
    """Minimum over samples of the interpolant on a `factor`-times finer grid.
    Returns (gamma_fine, slack) where slack bounds gamma_fine - gamma_exact:
    half the fine-cell diagonal times sqrt(1 + L^2), L the largest normalised
    slope of the interpolant."""
    shape = ref.shape
    n = ref.ndim
    sp_xyz = np.array(spacing[::-1], dtype=np.float64)
    fine_axes = [np.linspace(0, s - 1, (s - 1) * factor + 1) for s in shape[::-1]]
    Xf = np.stack(np.meshgrid(*fine_axes, indexing="ij"), axis=-1).reshape(-1, n)
    Df = freudenthal_interpolate(ev, Xf)
    Pf = Xf * sp_xyz / dta
    r = ref.astype(np.float64).ravel()
    dD, mask = _resolve(ref, dd_frac, local, cutoff_frac, dose_norm)
    nodes = normalised_nodes(shape, spacing, dta).reshape(-1, n)
    out = np.full(r.size, np.nan)
    # largest slope: over every simplex, gradient along its chain steps
    simp = freudenthal_simplices(shape)
    e = ev.astype(np.float64).ravel()
    steps = np.diff(e[simp], axis=1)                       # (S, n) dose steps
    # step i moves along one axis; its normalised length is h_axis / dta
    strides = np.cumprod((1,) + tuple(shape[::-1]))[:-1]
    hop = np.diff(simp, axis=1)                            # stride taken
    hstep = np.zeros_like(steps)
    for d in range(n):
        hstep[hop == strides[d]] = sp_xyz[d] / dta
    grad2 = ((steps / hstep) ** 2).sum(-1).max()
    delta = 0.5 * np.sqrt(((sp_xyz / factor / dta) ** 2).sum())
    slack = np.full(r.size, np.nan)
    for v in np.nonzero(mask)[0]:
        dd = dD[v]
        d2 = ((Pf - nodes[v]) ** 2).sum(-1) + ((Df - r[v]) / dd) ** 2
        out[v] = np.sqrt(d2.min())
        slack[v] = delta * np.sqrt(1.0 + grad2 / dd ** 2)
    return out.reshape(shape), slack.reshape(shape)


def polyline_gamma_1d(ref_profile, ev_profile, h, dd, dta):
    """Gamma of a 1D problem: distance in (x/dta, D/dd) from each reference
    sample to the polyline through the evaluation samples."""
    x = np.arange(len(ev_profile)) * h / dta
    A = np.stack([x[:-1], ev_profile[:-1] / dd], -1)
    B = np.stack([x[1:], ev_profile[1:] / dd], -1)
    P = np.stack([x, ref_profile / dd], -1)
    AB = B - A
    t = np.einsum("vk,sk->vs", P, AB) - (A * AB).sum(-1)[None]
    t = np.clip(t / (AB * AB).sum(-1)[None], 0.0, 1.0)
    Q = A[None] + t[..., None] * AB[None]
    return np.sqrt(((P[:, None] - Q) ** 2).sum(-1)).min(1)


def discrete_gamma(ref, ev, spacing, dd_frac, dta, local=False, cutoff_frac=0.0,
                   dose_norm=0.0):
    """Low et al. 1998 discrete gamma: minimum over evaluation grid nodes only."""
    n = ref.ndim
    nodes = normalised_nodes(ref.shape, spacing, dta).reshape(-1, n)
    r = ref.astype(np.float64).ravel()
    e = ev.astype(np.float64).ravel()
    dD, mask = _resolve(ref, dd_frac, local, cutoff_frac, dose_norm)
    out = np.full(r.size, np.nan)
    for v in np.nonzero(mask)[0]:
        d2 = ((nodes - nodes[v]) ** 2).sum(-1) + ((e - r[v]) / dD[v]) ** 2
        out[v] = np.sqrt(d2.min())
    return out.reshape(ref.shape)


def read_golden(path: str):
    """Parse a tests/golden/*.txt fixture."""
    fields = {}
    expect = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            if key == "expect":
                expect.append((int(vals[0]), float(vals[1]), vals[2]))
            else:
                fields[key] = vals
    ndim = int(fields["ndim"][0])
    shape = tuple(int(v) for v in fields["shape"])
    if ndim == 2:
        shape = shape[1:]
    spacing = tuple(float(v) for v in fields["spacing"])[-ndim:]
    ref = np.array([float(v) for v in fields["ref"]], dtype=np.float32).reshape(shape)
    ev = np.array([float(v) for v in fields["eval"]], dtype=np.float32).reshape(shape)
    crit = dict(dd_frac=float(fields["dd_frac"][0]), dta_mm=float(fields["dta_mm"][0]),
                dose_norm=float(fields["dose_norm"][0]),
                cutoff_frac=float(fields["cutoff_frac"][0]))
    return ref, ev, spacing, crit, expect
