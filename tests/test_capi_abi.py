"""Host-only checks of the C ABI: the library builds, loads and exports every
function that include/*.h declares; argument validation needs no GPU; the
product path and the oracle never import each other."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(hdr).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(gamma_\w+)\s*\(", src, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_gb", os.path.join(ROOT, "paper_1012_1900_gb300", "_build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    path = mod.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("gamma_create", "gamma_run", "gamma_pass_rate", "gamma_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_version_without_gpu(lib):
    lib.gamma_strerror.restype = ctypes.c_char_p
    lib.gamma_version.restype = ctypes.c_char_p
    assert lib.gamma_strerror(0) == b"ok"
    assert lib.gamma_strerror(-2) == b"invalid shape"
    assert b"dose norm" in lib.gamma_strerror(-12)
    assert b"sm_103a" in lib.gamma_version()


def test_argument_validation_without_gpu():
    import paper_1012_1900_gb300 as g
    crit = g.criteria(0.03, 3.0)
    with pytest.raises(g.GammaError) as e:
        g.gamma_create(None, None, 4, (2, 2, 2), (1, 1, 1), crit)
    assert e.value.code == -2
    with pytest.raises(g.GammaError) as e:
        g.gamma_create(None, None, 3, (1, 4, 4), (1, 1, 1), crit)
    assert e.value.code == -2
    with pytest.raises(g.GammaError) as e:
        g.gamma_create(None, None, 3, (4, 4, 4), (1, 0, 1), crit)
    assert e.value.code == -1
    with pytest.raises(g.GammaError) as e:
        g.gamma_create(None, None, 3, (4, 4, 4), (1, 1, 1), g.criteria(0.0, 3.0))
    assert e.value.code == -1
    with pytest.raises(g.GammaError) as e:
        g.gamma_create(None, None, 2, (2, 4, 4), (1, 1, 1), crit)
    assert e.value.code == -2


def _imports(path):
    src = open(path).read()
    return set(re.findall(r"^\s*(?:from|import)\s+([\w\.]+)", src, flags=re.M))


def test_product_and_oracle_are_independent():
    for f in glob.glob(os.path.join(ROOT, "paper_1012_1900_gb300", "**", "*.py"), recursive=True):
        assert not any(m.split(".")[0] == "oracle" for m in _imports(f)), f
    for f in glob.glob(os.path.join(ROOT, "paper_1012_1900_gb300", "csrc", "*")):
        incs = re.findall(r'#include\s+[<"]([^>"]+)', open(f).read())
        assert not any("oracle" in i for i in incs), f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        assert not any(m.split(".")[0] in ("paper_1012_1900_gb300", "synth") for m in _imports(f)), f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.c")):
        incs = re.findall(r'#include\s+[<"]([^>"]+)', open(f).read())
        assert all(i in ("math.h", "stdint.h", "stdlib.h", "string.h", "omp.h") for i in incs), incs


def test_more_argument_validation_without_gpu(lib):
    # Entry points that must reject bad arguments before touching a device.
    import ctypes
    INVALID = -1
    assert lib.gamma_measure_fp32_peak(None, None, None) == INVALID
    assert lib.gamma_set_option(None, b"pipeline", 1) == INVALID
    v = ctypes.c_int64()
    assert lib.gamma_get_option(None, b"walk", ctypes.byref(v)) == INVALID
    assert lib.gamma_run_host(None, None, None, None, None) == INVALID
    assert lib.gamma_run(None, None, None) == INVALID
    assert lib.gamma_pass_rate(None, None, None, None) == INVALID
    out = ctypes.c_void_p()
    assert lib.gamma_batch_create(ctypes.byref(out), 0, None) == INVALID
    assert lib.gamma_batch_create(ctypes.byref(out), 70000, None) == INVALID
