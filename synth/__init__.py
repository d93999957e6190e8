"""Seeded synthetic dose pairs shaped like the paper's IMRT test data.

The paper evaluates on eight clinical IMRT pairs (Monte Carlo reference,
pencil-beam evaluation; Section 3.1), which are not available.  These
generators stand in for them with analytic phantoms of the same shape and
dose structure.  Because each phantom is an analytic function of position, an
evaluation dose "shifted by s" is the same function evaluated at x - s, with no
resampling error.

This module holds no gamma arithmetic: it only produces (reference,
evaluation) float32 arrays.  Both the CUDA path's tests and the CPU oracle's
tests take their inputs from here.

Conventions: arrays are C-ordered (z, y, x); 2D planes are (y, x).  Spacings
are given in the same axis order, in millimetres.  Voxel centres sit at
index * spacing, so the physical box of an axis with n voxels of size h is
[-h/2, (n - 1/2) h].
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Sequence, Tuple

import numpy as np
from scipy import ndimage, special

__all__ = [
    "Criteria", "Pair", "blob_phantom_2d", "beam_phantom_3d", "make_pair_2d",
    "make_pair_3d", "workload", "batch_pair", "batch_pairs", "training_pair", "test_pair",
    "random_field",
]


@dataclasses.dataclass(frozen=True)
class Criteria:
    """Gamma criteria: dose difference as a fraction, DTA in mm."""
    dd_frac: float
    dta_mm: float
    local: bool = False
    cutoff_frac: float = 0.10
    dose_norm: float = 0.0   # <= 0: use max of the reference dose

    @property
    def label(self) -> str:
        mode = "local" if self.local else "global"
        return f"{self.dd_frac * 100:g}%/{self.dta_mm:g}mm {mode}"


@dataclasses.dataclass
class Pair:
    """One reference/evaluation dose pair on a shared grid."""
    name: str
    ref: np.ndarray          # float32, (nz, ny, nx) or (ny, nx)
    eval: np.ndarray         # float32, same shape
    spacing: Tuple[float, ...]   # mm, same axis order as the arrays
    criteria: Criteria

    @property
    def ndim(self) -> int:
        return self.ref.ndim

    @property
    def nvox(self) -> int:
        return int(self.ref.size)


def _axes(shape: Sequence[int], spacing: Sequence[float]) -> List[np.ndarray]:
    return [np.arange(n, dtype=np.float64) * h for n, h in zip(shape, spacing)]


# ---------------------------------------------------------------------------
# 2D: sum of Gaussian blobs
# ---------------------------------------------------------------------------

def blob_phantom_2d(shape: Sequence[int], spacing: Sequence[float], seed: int,
                    n_blobs: int = 6) -> Callable[[np.ndarray, np.ndarray], np.ndarray]:
    """Return D(y, x): n_blobs isotropic Gaussians, centres U[0.2, 0.8] of the
    extent, sigma U[8, 25] mm, amplitude U[0.3, 1], scaled so that the
    maximum over the grid is 1."""
    rng = np.random.default_rng(seed)
    ext = np.array([n * h for n, h in zip(shape, spacing)], dtype=np.float64)
    centres = rng.uniform(0.2, 0.8, size=(n_blobs, 2)) * ext
    sigmas = rng.uniform(8.0, 25.0, size=n_blobs)
    amps = rng.uniform(0.3, 1.0, size=n_blobs)

    def raw(yy: np.ndarray, xx: np.ndarray) -> np.ndarray:
        out = np.zeros(np.broadcast(yy, xx).shape, dtype=np.float64)
        for (cy, cx), s, a in zip(centres, sigmas, amps):
            out += a * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2.0 * s * s))
        return out

    y, x = _axes(shape, spacing)
    norm = raw(y[:, None], x[None, :]).max()

    def dose(yy: np.ndarray, xx: np.ndarray) -> np.ndarray:
        return raw(yy, xx) / norm

    return dose


def make_pair_2d(shape=(128, 128), spacing=(1.0, 1.0), seed: int = 0,
                 shift_mm=(0.0, 0.7), scale: float = 1.02,
                 noise_sd: float = 0.005,
                 criteria: Criteria = Criteria(0.03, 3.0),
                 name: str = "") -> Pair:
    """2D pair: reference blobs; evaluation = scale * D(r - shift) + white
    noise N(0, noise_sd^2) per pixel.  shift_mm is (dy, dx)."""
    dose = blob_phantom_2d(shape, spacing, seed)
    y, x = _axes(shape, spacing)
    yy, xx = y[:, None], x[None, :]
    ref = dose(yy, xx)
    ev = scale * dose(yy - shift_mm[0], xx - shift_mm[1])
    rng = np.random.default_rng(seed + 7919)
    if noise_sd > 0:
        ev = ev + rng.normal(0.0, noise_sd, size=ev.shape)
    return Pair(name or f"2d_{shape[0]}x{shape[1]}_s{seed}",
                np.ascontiguousarray(ref, dtype=np.float32),
                np.ascontiguousarray(ev, dtype=np.float32), tuple(float(h) for h in spacing),
                criteria)


# ---------------------------------------------------------------------------
# 3D: coplanar IMRT-like beams
# ---------------------------------------------------------------------------

def beam_phantom_3d(shape: Sequence[int], spacing: Sequence[float], seed: int,
                    n_beams: int = 7, mu_per_mm: float = 0.005,
                    n_beamlets: int = 10, field_frac: float = 0.4,
                    penumbra_sigma_mm: float = 3.0):
    """Return D(z, y, x) for n_beams coplanar beams about the z axis through
    the box centre, gantry angles 2 pi k / n_beams.  Each beam is
    exp(-mu * depth) * F(u, z), depth measured along the beam from where it
    enters the box, F an n_beamlets x n_beamlets fluence map with weights
    U[0.2, 1] over a square field field_frac of the transverse extents,
    blurred by a Gaussian penumbra (closed form: differences of normal CDFs).
    The sum is scaled so that its maximum over the grid is 1.

    The returned callable takes a shift (dz, dy, dx) in mm and returns the
    dose sampled at every grid point r - shift, as a float64 (nz, ny, nx)
    array."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    hz, hy, hx = spacing
    lo = np.array([-hz / 2, -hy / 2, -hx / 2])
    hi = np.array([(nz - 0.5) * hz, (ny - 0.5) * hy, (nx - 0.5) * hx])
    centre = (lo + hi) / 2.0
    w_u = field_frac * max(hi[1] - lo[1], hi[2] - lo[2])
    w_z = field_frac * (hi[0] - lo[0])
    u_edges = np.linspace(-w_u / 2, w_u / 2, n_beamlets + 1)
    z_edges = np.linspace(-w_z / 2, w_z / 2, n_beamlets + 1)
    weights = rng.uniform(0.2, 1.0, size=(n_beams, n_beamlets, n_beamlets))
    sig = penumbra_sigma_mm

    def raw(shift) -> np.ndarray:
        sz, sy, sx = shift
        z = np.arange(nz) * hz - sz - centre[0]
        y = np.arange(ny) * hy - sy
        x = np.arange(nx) * hx - sx
        yy, xx = np.meshgrid(y, x, indexing="ij")      # absolute coords
        # beamlet profiles along z: (n_beamlets, nz)
        cz = special.ndtr((z[None, :] - z_edges[:-1, None]) / sig) - \
            special.ndtr((z[None, :] - z_edges[1:, None]) / sig)
        total = np.zeros((ny * nx, nz), dtype=np.float64)
        for k in range(n_beams):
            th = 2.0 * math.pi * k / n_beams
            dy_, dx_ = math.sin(th), math.cos(th)       # beam direction
            # distance travelled back along the beam to the box boundary
            tx = np.where(dx_ > 1e-12, (xx - lo[2]) / max(dx_, 1e-12),
                          np.where(dx_ < -1e-12, (hi[2] - xx) / max(-dx_, 1e-12), np.inf))
            ty = np.where(dy_ > 1e-12, (yy - lo[1]) / max(dy_, 1e-12),
                          np.where(dy_ < -1e-12, (hi[1] - yy) / max(-dy_, 1e-12), np.inf))
            depth = np.maximum(np.minimum(tx, ty), 0.0)
            u = (yy - centre[1]) * dx_ - (xx - centre[2]) * dy_
            cu = special.ndtr((u[..., None] - u_edges[:-1]) / sig) - \
                special.ndtr((u[..., None] - u_edges[1:]) / sig)   # (ny, nx, nb)
            bz = weights[k] @ cz                       # (nb_u, nz): sum_j w_ij c_j(z)
            att = np.exp(-mu_per_mm * depth)
            total += (att[..., None] * cu).reshape(ny * nx, n_beamlets) @ bz
        return total.reshape(ny, nx, nz).transpose(2, 0, 1)

    norm = raw((0.0, 0.0, 0.0)).max()

    def dose(shift=(0.0, 0.0, 0.0)) -> np.ndarray:
        return raw(shift) / norm

    return dose


def random_field(shape: Sequence[int], spacing: Sequence[float], seed: int,
                 sigma_mm: float, sd: float) -> np.ndarray:
    """White noise blurred by a Gaussian of sigma_mm, rescaled to std sd."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal(size=tuple(shape))
    sm = ndimage.gaussian_filter(white, sigma=[sigma_mm / h for h in spacing],
                                 mode="reflect")
    s = sm.std()
    return sm * (sd / s) if s > 0 else sm


def make_pair_3d(shape=(120, 160, 160), spacing=(2.5, 2.5, 2.5), seed: int = 0,
                 shift_mm=(0.0, 0.0, 1.5), scale: float = 1.03,
                 noise_sd: float = 0.01, noise_sigma_mm: float = 10.0,
                 criteria: Criteria = Criteria(0.03, 3.0),
                 name: str = "") -> Pair:
    """3D pair: reference = beam phantom; evaluation = scale * D(r - shift)
    + smooth noise (Gaussian random field, sigma noise_sigma_mm, std
    noise_sd).  shift_mm is (dz, dy, dx)."""
    dose = beam_phantom_3d(shape, spacing, seed)
    ref = dose((0.0, 0.0, 0.0))
    ev = scale * dose(tuple(shift_mm))
    if noise_sd > 0:
        ev = ev + random_field(shape, spacing, seed + 104729, noise_sigma_mm, noise_sd)
    tag = "x".join(str(s) for s in shape[::-1])
    return Pair(name or f"3d_{tag}_s{seed}", np.ascontiguousarray(ref, dtype=np.float32),
                np.ascontiguousarray(ev, dtype=np.float32), tuple(float(h) for h in spacing),
                criteria)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

def workload(name: str, criteria: Criteria | None = None) -> Pair:
    """The named single-pair workloads.

    plane_128     2D 128x128, 1 mm, blobs; eval 1.02 * D(x - 0.7 mm) + N(0, .005^2);
                  3%/3 mm global, 10 % cutoff, seed 0.
    imrt_160      3D 160x160x120 at 2.5 mm, 7 beams; eval 1.03 * D(x - 1.5 mm) +
                  smooth noise sd 0.01; 3%/3 mm global (2%/2 mm with seed 1).
    imrt_320      3D 320x320x240 at 1.25 mm; shift 3 mm, scale 1.05;
                  1%/1 mm local (or 3%/3 mm global).
    Small variants (for quick tests) keep the generator and shrink the grid.
    """
    if name == "plane_128":
        return make_pair_2d(criteria=criteria or Criteria(0.03, 3.0), name=name)
    if name == "imrt_160":
        return make_pair_3d(criteria=criteria or Criteria(0.03, 3.0), name=name)
    if name == "imrt_160_2mm2pct":
        return make_pair_3d(seed=1, criteria=criteria or Criteria(0.02, 2.0), name=name)
    if name == "imrt_320_local":
        return make_pair_3d(shape=(240, 320, 320), spacing=(1.25, 1.25, 1.25),
                            shift_mm=(0.0, 0.0, 3.0), scale=1.05,
                            criteria=criteria or Criteria(0.01, 1.0, local=True), name=name)
    if name == "imrt_320_global":
        return make_pair_3d(shape=(240, 320, 320), spacing=(1.25, 1.25, 1.25),
                            shift_mm=(0.0, 0.0, 3.0), scale=1.05,
                            criteria=criteria or Criteria(0.03, 3.0), name=name)
    if name == "imrt_small":
        return make_pair_3d(shape=(24, 40, 36), spacing=(2.5, 2.5, 2.5), seed=5,
                            criteria=criteria or Criteria(0.03, 3.0), name=name)
    raise KeyError(name)


_CRIT_SET = (Criteria(0.01, 1.0), Criteria(0.02, 2.0), Criteria(0.03, 3.0))


def batch_pair(i: int, n2d: int = 32, base_seed: int = 3000,
               max_shape=(150, 200, 200), min_shape=(64, 64, 64)) -> Pair:
    """Pair i of the uneven batch: pairs 0..n2d-1 are planes 256x256 at 1 mm,
    the others volumes at 2 mm with shapes log-uniform between min_shape and
    max_shape; per pair a shift U[0, 3] mm in a random direction, scale
    U[0.97, 1.05] and criteria drawn from {1%/1 mm, 2%/2 mm, 3%/3 mm}
    (global, 10 % cutoff)."""
    seed = base_seed + i
    rng = np.random.default_rng(seed + 55555)
    crit = _CRIT_SET[int(rng.integers(0, 3))]
    mag = rng.uniform(0.0, 3.0)
    scale = float(rng.uniform(0.97, 1.05))
    if i < n2d:
        ang = rng.uniform(0, 2 * math.pi)
        shift = (mag * math.sin(ang), mag * math.cos(ang))
        return make_pair_2d(shape=(256, 256), spacing=(1.0, 1.0), seed=seed, shift_mm=shift,
                            scale=scale, criteria=crit, name=f"batch{i:02d}_2d")
    v = rng.normal(size=3)
    v /= np.linalg.norm(v)
    t = rng.uniform(0.0, 1.0)
    shp = tuple(int(round(math.exp(math.log(a) + t * (math.log(b) - math.log(a)))))
                for a, b in zip(min_shape, max_shape))
    return make_pair_3d(shape=shp, spacing=(2.0, 2.0, 2.0), seed=seed, shift_mm=tuple(mag * v),
                        scale=scale, criteria=crit, name=f"batch{i:02d}_3d")


def batch_pairs(n2d: int = 32, n3d: int = 32, base_seed: int = 3000) -> List[Pair]:
    """The uneven batch: n2d planes and n3d volumes (see batch_pair)."""
    return [batch_pair(i, n2d=n2d, base_seed=base_seed) for i in range(n2d + n3d)]


def training_pair(i: int, shape=(150, 200, 200), crit: Criteria = Criteria(0.02, 2.0)) -> Pair:
    """Training pair i (seed 1000 + i): 2 mm voxels, shift U[0, 4] mm in a
    random direction, scale U[0.95, 1.05]."""
    seed = 1000 + i
    return _learned_pair(seed, shape, crit, f"train{i:03d}")


def test_pair(i: int, shape=(150, 200, 200), crit: Criteria = Criteria(0.02, 2.0)) -> Pair:
    """Held-out pair i (seed 2000 + i), same recipe as training_pair."""
    seed = 2000 + i
    return _learned_pair(seed, shape, crit, f"test{i:02d}")


def _learned_pair(seed: int, shape, crit: Criteria, name: str) -> Pair:
    rng = np.random.default_rng(seed + 424242)
    v = rng.normal(size=3)
    v /= np.linalg.norm(v)
    mag = rng.uniform(0.0, 4.0)
    scale = float(rng.uniform(0.95, 1.05))
    return make_pair_3d(shape=shape, spacing=(2.0, 2.0, 2.0), seed=seed,
                        shift_mm=tuple(mag * v), scale=scale, criteria=crit, name=name)
