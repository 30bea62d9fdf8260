"""Loader for the oracle's C sums (``sog_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``oracle`` and nothing in the product
path.  The shared object is built with gcc (OpenMP when available) next to
the source on first use, or ahead of time by ``build_oracle()``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sog_oracle.c")
_LIB = os.path.join(_HERE, "_sog_oracle.so")
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile ``sog_oracle.c`` into ``_sog_oracle.so`` (gcc -O2 -fopenmp)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(cmd, check=True, capture_output=True)
    except subprocess.CalledProcessError:
        cmd.remove("-fopenmp")
        subprocess.run(cmd, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build_oracle()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int64)
        ci, cd = ctypes.c_int, ctypes.c_double
        L.oracle_ewald2d.argtypes = [ci, dp, ip, ci, dp, dp, cd, cd, cd, cd, cd, dp, dp]
        L.oracle_brute_images.argtypes = [ci, dp, ip, ci, dp, dp, cd, cd, ci, dp]
        L.oracle_near.argtypes = [ci, dp, ip, ci, dp, dp, cd, cd, cd, ci, dp, dp, dp, dp]
        L.oracle_gauss_images.argtypes = [ci, dp, ci, dp, dp, cd, cd, ci, dp, dp, dp, dp]
        L.oracle_num_threads.restype = ci
        for f in (L.oracle_ewald2d, L.oracle_brute_images, L.oracle_near,
                  L.oracle_gauss_images):
            f.restype = None
        _lib = L
    return _lib


def dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def iptr(a: np.ndarray):
    assert a.dtype == np.int64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def num_threads() -> int:
    return int(lib().oracle_num_threads())
