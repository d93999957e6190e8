"""GB300 gamma-index library: thin ctypes binding of libgamma_gb300.so.

Every function here has the name of the C entry point it wraps (see
include/gamma.h) and only marshals arguments: torch tensors become device
pointers and CUDA stream handles, status codes become exceptions.  All
gamma arithmetic runs in the library's CUDA kernels; there is no CPU path.
If the library has not been built, importing this package raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

from . import _build

__all__ = [
    "GammaError", "gamma_criteria", "gamma_stats", "gamma_create", "gamma_set_inputs",
    "gamma_run", "gamma_run_host", "gamma_pass_rate", "gamma_get_stats", "gamma_get_timings",
    "gamma_set_option",
    "gamma_run_noalloc", "gamma_batch_create", "gamma_batch_run", "gamma_batch_pass_rate",
    "gamma_batch_get_stats", "gamma_create_grids", "gamma_autotune", "gamma_pair_desc", "gamma_destroy",
    "gamma_model_create", "gamma_model_destroy", "gamma_model_num_params", "gamma_model_get_params",
    "gamma_model_set_params", "gamma_model_forward", "gamma_model_infer", "gamma_model_backward",
    "gamma_model_train_step", "gamma_model_save", "gamma_model_load", "gamma_features",
    "gamma_labels", "gamma_set_model", "gamma_load_model", "gamma_measure_fp32_peak", "gamma_strerror",
    "gamma_version", "library_path",
    "criteria",
    "GLOBAL", "LOCAL",
]

GLOBAL, LOCAL = 0, 1


class gamma_criteria(ctypes.Structure):
    _fields_ = [("dd_frac", ctypes.c_float), ("dta_mm", ctypes.c_float), ("mode", ctypes.c_int),
                ("cutoff_frac", ctypes.c_float), ("dose_norm", ctypes.c_float)]


class gamma_stats(ctypes.Structure):
    _fields_ = [("n_voxels", ctypes.c_int64), ("n_eval", ctypes.c_int64),
                ("n_pass", ctypes.c_int64), ("tail_voxels", ctypes.c_int64),
                ("overflow_voxels", ctypes.c_int64), ("fp64_cells", ctypes.c_int64),
                ("seeded", ctypes.c_int64), ("seed_improved", ctypes.c_int64),
                ("cells_keyed", ctypes.c_int64), ("cells_visited", ctypes.c_int64),
                ("cells_pruned", ctypes.c_int64), ("d_norm", ctypes.c_double),
                ("r_max", ctypes.c_double), ("table_entries", ctypes.c_int64),
                ("table_radius", ctypes.c_double), ("flags", ctypes.c_uint32),
                ("lane_slot_steps", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gamma_timings(ctypes.Structure):
    _fields_ = [(k, ctypes.c_float) for k in ("h2d_ms", "prepare_ms", "shell_ms", "order_ms",
                                              "tail_ms", "d2h_ms", "total_ms")] + \
        [("overlapped", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gamma_pair_desc(ctypes.Structure):
    _fields_ = [("ref_dev", ctypes.c_void_p), ("eval_dev", ctypes.c_void_p),
                ("gamma_out_dev", ctypes.c_void_p), ("ndim", ctypes.c_int),
                ("shape", ctypes.c_int64 * 3), ("spacing_mm", ctypes.c_float * 3),
                ("crit", gamma_criteria)]


class GammaError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.gamma_strerror(code).decode()
        if code == -7:
            msg += ": " + _lib.gamma_last_cuda_error().decode()
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


def library_path() -> str:
    return _build.LIB


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
    f32p = ctypes.POINTER(ctypes.c_float)
    lib.gamma_create.argtypes = [ctypes.POINTER(vp), vp, vp, ctypes.c_int, i64p, f32p,
                                 ctypes.POINTER(gamma_criteria)]
    lib.gamma_create_grids.argtypes = [ctypes.POINTER(vp), vp, vp, ctypes.c_int, i64p, f32p, f32p,
                                       i64p, f32p, f32p, ctypes.POINTER(gamma_criteria)]
    lib.gamma_set_inputs.argtypes = [vp, vp, vp]
    lib.gamma_run.argtypes = [vp, vp, vp]
    lib.gamma_run_host.argtypes = [vp, vp, vp, vp, vp]
    lib.gamma_pass_rate.argtypes = [vp, ctypes.POINTER(ctypes.c_double), i64p, i64p]
    lib.gamma_get_stats.argtypes = [vp, ctypes.POINTER(gamma_stats)]
    lib.gamma_get_timings.argtypes = [vp, ctypes.POINTER(gamma_timings)]
    lib.gamma_set_option.argtypes = [vp, ctypes.c_char_p, ctypes.c_int64]
    lib.gamma_get_option.argtypes = [vp, ctypes.c_char_p, i64p]
    lib.gamma_run_noalloc.argtypes = [vp, vp, vp, ctypes.c_int, i64p, f32p,
                                      ctypes.POINTER(gamma_criteria), vp, i64p, i64p]
    lib.gamma_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int,
                                       ctypes.POINTER(gamma_pair_desc)]
    lib.gamma_batch_run.argtypes = [vp, vp]
    lib.gamma_batch_pass_rate.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                          i64p, i64p]
    lib.gamma_batch_get_stats.argtypes = [vp, ctypes.c_int, ctypes.POINTER(gamma_stats)]
    lib.gamma_autotune.argtypes = [vp, vp, vp, ctypes.c_int, i64p, i64p, i64p,
                                   ctypes.POINTER(ctypes.c_float)]
    lib.gamma_model_create.argtypes = [ctypes.POINTER(vp), ctypes.c_uint64]
    lib.gamma_model_destroy.argtypes = [vp]
    lib.gamma_model_destroy.restype = None
    lib.gamma_model_num_params.restype = ctypes.c_int64
    lib.gamma_model_get_params.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int]
    lib.gamma_model_set_params.argtypes = [vp, vp, ctypes.c_int64]
    lib.gamma_model_forward.argtypes = [vp, vp, ctypes.c_int64, vp, vp]
    lib.gamma_model_infer.argtypes = [vp, vp, ctypes.c_int64, vp, vp]
    lib.gamma_model_backward.argtypes = [vp, vp, vp, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_float), vp]
    lib.gamma_model_train_step.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.c_float,
                                           ctypes.POINTER(ctypes.c_float), vp]
    lib.gamma_model_save.argtypes = [vp, ctypes.c_char_p]
    lib.gamma_model_load.argtypes = [vp, ctypes.c_char_p]
    lib.gamma_features.argtypes = [vp, vp, ctypes.c_int64, vp, vp]
    lib.gamma_labels.argtypes = [vp, vp, vp, ctypes.c_int64, vp, vp]
    lib.gamma_set_model.argtypes = [vp, vp]
    lib.gamma_load_model.argtypes = [vp, ctypes.c_char_p]
    lib.gamma_destroy.argtypes = [vp]
    lib.gamma_destroy.restype = None
    lib.gamma_measure_fp32_peak.argtypes = [ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double), vp]
    lib.gamma_strerror.argtypes = [ctypes.c_int]
    lib.gamma_strerror.restype = ctypes.c_char_p
    lib.gamma_last_cuda_error.restype = ctypes.c_char_p
    lib.gamma_version.restype = ctypes.c_char_p
    return lib


_lib = _load()


def _check(rc: int, where: str):
    if rc != 0:
        raise GammaError(rc, where)


def _dev_ptr(t) -> int:
    """Device pointer of a contiguous float32 CUDA tensor (or an int)."""
    if t is None:
        return 0
    if isinstance(t, int):
        return t
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"expected a torch.Tensor, got {type(t).__name__}")
    if t.device.type != "cuda" or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("expected a contiguous float32 CUDA tensor, got "
                         f"device={t.device} dtype={t.dtype} contiguous={t.is_contiguous()}")
    return t.data_ptr()


def _stream_ptr(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def criteria(dd_frac: float, dta_mm: float, local: bool = False, cutoff_frac: float = 0.10,
             dose_norm: float = 0.0) -> gamma_criteria:
    return gamma_criteria(dd_frac, dta_mm, LOCAL if local else GLOBAL, cutoff_frac, dose_norm)


def gamma_create(ref_dev, eval_dev, ndim: int, shape: Sequence[int], spacing_mm: Sequence[float],
                 crit: gamma_criteria) -> int:
    """Create a handle.  ref_dev/eval_dev: float32 CUDA tensors (or None for a
    handle that owns its device buffers).  shape/spacing in (z, y, x) order,
    shape[0] = 1 for 2D.  Returns the handle (an int)."""
    h = ctypes.c_void_p()
    shp = (ctypes.c_int64 * 3)(*[int(s) for s in shape])
    sp = (ctypes.c_float * 3)(*[float(s) for s in spacing_mm])
    _check(_lib.gamma_create(ctypes.byref(h), _dev_ptr(ref_dev), _dev_ptr(eval_dev), int(ndim),
                             shp, sp, ctypes.byref(crit)), "gamma_create")
    return h.value


def gamma_create_grids(ref_dev, eval_dev, ndim: int, ref_shape: Sequence[int],
                       ref_spacing_mm: Sequence[float], ref_origin_mm: Sequence[float],
                       eval_shape: Sequence[int], eval_spacing_mm: Sequence[float],
                       eval_origin_mm: Sequence[float], crit: gamma_criteria) -> int:
    """Handle for doses on two different grids (float32 CUDA tensors); every
    shape / spacing / origin in (z, y, x) order, 1 / 1.0 / 0.0 first for 2D."""
    h = ctypes.c_void_p()
    i3 = lambda v: (ctypes.c_int64 * 3)(*[int(s) for s in v])
    f3 = lambda v: (ctypes.c_float * 3)(*[float(s) for s in v])
    _check(_lib.gamma_create_grids(ctypes.byref(h), _dev_ptr(ref_dev), _dev_ptr(eval_dev),
                                   int(ndim), i3(ref_shape), f3(ref_spacing_mm),
                                   f3(ref_origin_mm), i3(eval_shape), f3(eval_spacing_mm),
                                   f3(eval_origin_mm), ctypes.byref(crit)), "gamma_create_grids")
    return h.value


def gamma_set_inputs(h: int, ref_dev, eval_dev) -> None:
    _check(_lib.gamma_set_inputs(h, _dev_ptr(ref_dev), _dev_ptr(eval_dev)), "gamma_set_inputs")


def gamma_run(h: int, gamma_out_dev, stream=None) -> None:
    _check(_lib.gamma_run(h, _dev_ptr(gamma_out_dev), _stream_ptr(stream)), "gamma_run")


def gamma_run_host(h: int, ref_host, eval_host, gamma_out_host, stream=None) -> None:
    """Host-buffer run; arguments are CPU float32 tensors or numpy arrays
    (pinned tensors give asynchronous copies)."""
    def hp(a):
        if hasattr(a, "data_ptr"):
            if a.is_cuda or not a.is_contiguous():
                raise ValueError("expected a contiguous CPU tensor")
            return a.data_ptr()
        if not a.flags["C_CONTIGUOUS"] or a.dtype.name != "float32":
            raise ValueError("expected a C-contiguous float32 array")
        return a.ctypes.data
    _check(_lib.gamma_run_host(h, hp(ref_host), hp(eval_host), hp(gamma_out_host),
                               _stream_ptr(stream)), "gamma_run_host")


def gamma_measure_fp32_peak(stream=None) -> dict:
    """Measured FP32 FMA throughput of the current device (TFLOP/s) and the
    time of the timed launch (ms)."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(_lib.gamma_measure_fp32_peak(ctypes.byref(t), ctypes.byref(ms), _stream_ptr(stream)),
           "gamma_measure_fp32_peak")
    return {"tflops": t.value, "ms": ms.value}


def gamma_pass_rate(h: int):
    """(rate, n_eval, n_pass) of the last run (synchronises its stream)."""
    rate = ctypes.c_double()
    ne, npass = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.gamma_pass_rate(h, ctypes.byref(rate), ctypes.byref(ne), ctypes.byref(npass)),
           "gamma_pass_rate")
    return rate.value, ne.value, npass.value


def gamma_get_stats(h: int) -> dict:
    st = gamma_stats()
    _check(_lib.gamma_get_stats(h, ctypes.byref(st)), "gamma_get_stats")
    return st.as_dict()


def gamma_get_timings(h: int) -> dict:
    """Per-phase device times (ms) of the last run (option "timing" must be 1)."""
    t = gamma_timings()
    _check(_lib.gamma_get_timings(h, ctypes.byref(t)), "gamma_get_timings")
    return t.as_dict()


def gamma_set_option(h: int, key: str, value: int) -> None:
    _check(_lib.gamma_set_option(h, key.encode(), int(value)), f"gamma_set_option({key})")


def gamma_get_option(h: int, key: str) -> int:
    v = ctypes.c_int64()
    _check(_lib.gamma_get_option(h, key.encode(), ctypes.byref(v)), f"gamma_get_option({key})")
    return v.value


def gamma_run_noalloc(ref_dev, eval_dev, gamma_out_dev, ndim: int, shape: Sequence[int],
                      spacing_mm: Sequence[float], crit: gamma_criteria, stream=None,
                      counts: bool = True):
    """One gamma map with no allocation (the library's fixed scratch array).
    Returns (n_eval, n_pass) when counts is true (synchronises), else None."""
    shp = (ctypes.c_int64 * 3)(*[int(s) for s in shape])
    sp = (ctypes.c_float * 3)(*[float(s) for s in spacing_mm])
    ne, npass = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.gamma_run_noalloc(_dev_ptr(ref_dev), _dev_ptr(eval_dev), _dev_ptr(gamma_out_dev),
                                  int(ndim), shp, sp, ctypes.byref(crit), _stream_ptr(stream),
                                  ctypes.byref(ne) if counts else None,
                                  ctypes.byref(npass) if counts else None), "gamma_run_noalloc")
    return (ne.value, npass.value) if counts else None


def gamma_batch_create(pairs) -> int:
    """Batch handle over a list of (ref_dev, eval_dev, gamma_out_dev, ndim, shape,
    spacing_mm, crit) tuples; tensors are float32 CUDA tensors, shape/spacing
    in (z, y, x) order with shape[0] = 1 for 2D."""
    arr = (gamma_pair_desc * len(pairs))()
    for d, (ref, ev, out, ndim, shape, spacing, crit) in zip(arr, pairs):
        d.ref_dev, d.eval_dev, d.gamma_out_dev = _dev_ptr(ref), _dev_ptr(ev), _dev_ptr(out)
        d.ndim = int(ndim)
        d.shape = (ctypes.c_int64 * 3)(*[int(v) for v in shape])
        d.spacing_mm = (ctypes.c_float * 3)(*[float(v) for v in spacing])
        d.crit = crit
    h = ctypes.c_void_p()
    _check(_lib.gamma_batch_create(ctypes.byref(h), len(pairs), arr), "gamma_batch_create")
    return h.value


def gamma_batch_run(h: int, stream=None) -> None:
    _check(_lib.gamma_batch_run(h, _stream_ptr(stream)), "gamma_batch_run")


def gamma_batch_pass_rate(h: int, pair: int):
    rate = ctypes.c_double()
    ne, npass = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.gamma_batch_pass_rate(h, int(pair), ctypes.byref(rate), ctypes.byref(ne),
                                      ctypes.byref(npass)), "gamma_batch_pass_rate")
    return rate.value, ne.value, npass.value


def gamma_batch_get_stats(h: int, pair: int) -> dict:
    st = gamma_stats()
    _check(_lib.gamma_batch_get_stats(h, int(pair), ctypes.byref(st)), "gamma_batch_get_stats")
    return st.as_dict()


def gamma_autotune(h: int, gamma_out_dev=None, stream=None, reps: int = 3):
    """Time every (lanes_per_voxel, shell_blocks_per_sm, tail_blocks_per_sm)
    choice, keep the fastest; returns a dict of the three and the time (ms)."""
    lanes, blocks, tblocks = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    ms = ctypes.c_float()
    _check(_lib.gamma_autotune(h, _dev_ptr(gamma_out_dev), _stream_ptr(stream), int(reps),
                               ctypes.byref(lanes), ctypes.byref(blocks), ctypes.byref(tblocks),
                               ctypes.byref(ms)),
           "gamma_autotune")
    return {"lanes_per_voxel": lanes.value, "shell_blocks_per_sm": blocks.value,
            "tail_blocks_per_sm": tblocks.value, "ms": ms.value}


# ---- learned proposal ----

def _raw_ptr(t) -> int:
    """Device pointer of any contiguous CUDA tensor (bf16, float32, int32...)."""
    import torch
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def gamma_model_create(seed: int = 0) -> int:
    m = ctypes.c_void_p()
    _check(_lib.gamma_model_create(ctypes.byref(m), int(seed)), "gamma_model_create")
    return m.value


def gamma_model_destroy(m: Optional[int]) -> None:
    if m:
        _lib.gamma_model_destroy(m)


def gamma_model_num_params() -> int:
    return int(_lib.gamma_model_num_params())


def gamma_model_get_params(m: int, which: int = 0):
    import numpy as np
    n = gamma_model_num_params()
    out = np.empty(n, dtype=np.float32)
    _check(_lib.gamma_model_get_params(m, out.ctypes.data, n, int(which)), "gamma_model_get_params")
    return out


def gamma_model_set_params(m: int, params) -> None:
    import numpy as np
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(_lib.gamma_model_set_params(m, p.ctypes.data, p.size), "gamma_model_set_params")


def gamma_model_forward(m: int, X_bf16, Y, stream=None) -> None:
    _check(_lib.gamma_model_forward(m, _raw_ptr(X_bf16), int(X_bf16.shape[0]), _raw_ptr(Y),
                                    _stream_ptr(stream)), "gamma_model_forward")


def gamma_model_infer(m: int, X_bf16, Y, stream=None) -> None:
    """Network outputs with the tensor-core inference kernel of the search."""
    _check(_lib.gamma_model_infer(m, _raw_ptr(X_bf16), int(X_bf16.shape[0]), _raw_ptr(Y),
                                  _stream_ptr(stream)), "gamma_model_infer")


def gamma_model_backward(m: int, X_bf16, T, stream=None) -> float:
    loss = ctypes.c_float()
    _check(_lib.gamma_model_backward(m, _raw_ptr(X_bf16), _raw_ptr(T), int(X_bf16.shape[0]),
                                     ctypes.byref(loss), _stream_ptr(stream)),
           "gamma_model_backward")
    return loss.value


def gamma_model_train_step(m: int, X_bf16, T, lr: float, stream=None, want_loss: bool = True):
    loss = ctypes.c_float()
    _check(_lib.gamma_model_train_step(m, _raw_ptr(X_bf16), _raw_ptr(T), int(X_bf16.shape[0]),
                                       float(lr), ctypes.byref(loss) if want_loss else None,
                                       _stream_ptr(stream)), "gamma_model_train_step")
    return loss.value if want_loss else None


def gamma_model_save(m: int, path: str) -> None:
    _check(_lib.gamma_model_save(m, str(path).encode()), "gamma_model_save")


def gamma_model_load(m: int, path: str) -> None:
    _check(_lib.gamma_model_load(m, str(path).encode()), "gamma_model_load")


def gamma_features(h: int, voxels, X_bf16, stream=None) -> None:
    _check(_lib.gamma_features(h, _raw_ptr(voxels), int(voxels.numel()), _raw_ptr(X_bf16),
                               _stream_ptr(stream)), "gamma_features")


def gamma_labels(h: int, gamma_map, voxels, targets, stream=None) -> None:
    _check(_lib.gamma_labels(h, _dev_ptr(gamma_map), _raw_ptr(voxels), int(voxels.numel()),
                             _raw_ptr(targets), _stream_ptr(stream)), "gamma_labels")


def gamma_set_model(h: int, m: Optional[int]) -> None:
    _check(_lib.gamma_set_model(h, m or 0), "gamma_set_model")


def gamma_load_model(h: int, path: str) -> None:
    _check(_lib.gamma_load_model(h, str(path).encode()), "gamma_load_model")


def gamma_destroy(h: Optional[int]) -> None:
    if h:
        _lib.gamma_destroy(h)


def gamma_strerror(code: int) -> str:
    return _lib.gamma_strerror(code).decode()


def gamma_version() -> str:
    return _lib.gamma_version().decode()
