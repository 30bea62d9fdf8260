"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point declared in include/sog.h; the binding fails loudly without it."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sog.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(sog_[a-z_]+)\s*\(", src)
    return sorted(set(n for n in names if n != "sog_status"))


def test_header_declares_the_documented_entry_points():
    names = declared_functions()
    for n in ("sog_plan_create", "sog_eval", "sog_plan_destroy", "sog_select_params",
              "sog_eval_host", "sog_plan_check", "sog_eval_components"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2412_04595_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    for n in declared_functions():
        assert hasattr(lib, n), n


@pytest.mark.parametrize("window", ["es", "kb", "gauss"])
def test_select_params_through_the_abi_without_gpu(oracle_mod, window):
    """sog_select_params is host-only: callable here and equal to the
    oracle's own selection (Sec. 4.3) for the benchmark configuration, for
    each window."""
    from paper_2412_04595_gb300 import _build, binding
    _build.build()
    code = {"es": binding.SOG_WIN_ES, "kb": binding.SOG_WIN_KB, "gauss": binding.SOG_WIN_GAUSS}
    a = binding.sog_select_params(100000, 100.0, 100.0, 100.0, 1e-6, window=code[window], n_nb=120)
    b = oracle_mod.select_params(100000, 100.0, 100.0, 100.0, 1e-6, n_nb=120, window=window)
    assert a["window"] == window and a["long_direct"] == b["long_direct"]
    for k in ("M", "m", "I", "P_win", "I_long", "P_cheb"):
        assert tuple(map(int, __import__("numpy").atleast_1d(a[k]))) == \
            tuple(map(int, __import__("numpy").atleast_1d(b[k]))), k
    for k in ("rc", "sigma", "hz", "shape"):
        assert abs(a[k] - b[k]) <= 1e-13 * abs(b[k])


def test_argument_errors_are_reported():
    from paper_2412_04595_gb300 import binding
    with pytest.raises(binding.SogError):
        binding.sog_select_params(1, 10.0, 10.0, 10.0, 1e-6)
    with pytest.raises(binding.SogError):
        binding.sog_select_params(100, 10.0, 10.0, 10.0, 0.0)


def test_tune_cutoff_argument_errors_without_device_work():
    """sog_tune_cutoff checks its arguments before any CUDA call: no
    candidates, too many, a non-positive candidate, NULL inputs, bad reps."""
    from paper_2412_04595_gb300 import _build, binding
    lib = ctypes.CDLL(_build.build())
    f = lib.sog_tune_cutoff
    d, i32, vp = ctypes.c_double, ctypes.c_int32, ctypes.c_void_p
    f.argtypes = [ctypes.c_int64, d, d, d, d, vp, vp, vp, ctypes.POINTER(d), i32, i32,
                  ctypes.POINTER(d), ctypes.POINTER(ctypes.c_float), vp]
    best = d(0.0)
    dummy = vp(16)  # never dereferenced: every call below fails its argument checks
    def call(cands, n, reps=3, q=dummy, r=dummy):
        arr = (d * max(1, len(cands)))(*cands)
        return f(1000, 10.0, 10.0, 10.0, 1e-6, None, q, r, arr, n, reps, ctypes.byref(best),
                 None, None)
    assert call([120.0], 0) == 1  # SOG_ERR_ARG
    assert call([120.0] * 33, 33) == 1  # SOG_ERR_ARG
    assert call([120.0, -1.0], 2) == 1  # SOG_ERR_ARG
    assert call([120.0], 1, reps=0) == 1  # SOG_ERR_ARG
    assert call([120.0], 1, q=None) == 1  # SOG_ERR_ARG


def test_binding_fails_loudly_without_library(monkeypatch):
    from paper_2412_04595_gb300 import _build, binding
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(_build, "LIB", os.path.join(ROOT, "no_such_dir", "libsog.so"))
    with pytest.raises(RuntimeError, match="not built"):
        binding.load()


@pytest.mark.parametrize("N,L,tol", [
    (1000, (10.0, 10.0, 10.0), 1e-6),
    (100000, (100.0, 100.0, 100.0), 1e-4),
    (1000000, (1000.0, 1000.0, 10.0), 1e-6),
    (1000000, (50.0, 50.0, 2000.0), 1e-6),
    (4000000, (400.0, 400.0, 100.0), 1e-5),
    (20000, (37.0, 41.0, 9.0), 1e-6),
    (5000, (12.0, 12.0, 80.0), 1e-5),
])
def test_library_selection_equals_the_oracle_on_every_workload(oracle_mod, N, L, tol):
    """The host selection of the library and the oracle's selection agree
    on the workloads of the benchmark and on off-cube boxes: same integers,
    same reals to rounding, same choice between Algorithms 2 and 3."""
    from paper_2412_04595_gb300 import _build, binding
    _build.build()
    a = binding.sog_select_params(N, *L, tol)
    b = oracle_mod.select_params(N, *L, tol)
    for k in ("M", "m", "I", "P_win", "I_long", "P_long", "P_cheb", "long_direct"):
        assert tuple(np.atleast_1d(a[k]).astype(int)) == tuple(np.atleast_1d(b[k]).astype(int)), k
    for k in ("rc", "sigma", "hz", "shape", "shape_long"):
        assert abs(a[k] - b[k]) <= 1e-12 * max(abs(b[k]), 1e-300), k
