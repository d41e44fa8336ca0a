"""Loader for the oracle's C core (``ckks_oracle.c``).

TEST INFRASTRUCTURE ONLY: the oracle is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``; the
product library never loads it.

The shared object is built with plain ``gcc -O2 -fopenmp`` into
``oracle/_build/``.  ``build()`` is called by ``__graft_entry__.build()`` and,
if the library is missing, on first import.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ckks_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_OUT = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C core; returns the path of the shared object."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


_u64p = ctypes.POINTER(ctypes.c_uint64)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.orc_is_prime.argtypes = [ctypes.c_uint64]
            L.orc_is_prime.restype = ctypes.c_int
            for f in ("orc_powmod", "orc_mulmod"):
                getattr(L, f).argtypes = [ctypes.c_uint64] * 3
                getattr(L, f).restype = ctypes.c_uint64
            L.orc_invmod.argtypes = [ctypes.c_uint64] * 2
            L.orc_invmod.restype = ctypes.c_uint64
            L.orc_root_of_unity.argtypes = [ctypes.c_uint64] * 2
            L.orc_root_of_unity.restype = ctypes.c_uint64
            L.orc_nega_forward.argtypes = [_u64p, ctypes.c_size_t, ctypes.c_uint64]
            L.orc_nega_inverse.argtypes = [_u64p, ctypes.c_size_t, ctypes.c_uint64]
            L.orc_base_conv_rounded.argtypes = [_u64p, ctypes.c_size_t, _u64p, ctypes.c_int, _u64p, ctypes.c_int, _u64p]
            L.orc_seeded_key_a.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, _u64p, ctypes.c_int, ctypes.c_size_t, _u64p]
            L.orc_polymul_schoolbook.argtypes = [_u64p, _u64p, _u64p, ctypes.c_size_t, ctypes.c_uint64]
            L.orc_ring_mac.argtypes = [_u64p, ctypes.c_size_t, _u64p, ctypes.c_size_t, ctypes.c_int,
                                       _u64p, ctypes.c_int, ctypes.c_size_t, _u64p]
            L.orc_mul_scalar.argtypes = [_u64p, _u64p, _u64p, ctypes.c_int, ctypes.c_size_t, _u64p]
            L.orc_mul_pointwise.argtypes = [_u64p, _u64p, _u64p, ctypes.c_int, ctypes.c_size_t, _u64p]
            L.orc_fast_base_conv.argtypes = [_u64p, ctypes.c_size_t, _u64p, ctypes.c_int,
                                             _u64p, ctypes.c_int, _u64p]
            L.orc_fast_base_conv_centered.argtypes = [_u64p, ctypes.c_size_t, _u64p, ctypes.c_int,
                                                      _u64p, ctypes.c_int, _u64p]
            _lib = L
    return _lib


def ptr(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"], (a.dtype, a.flags)
    return a.ctypes.data_as(_u64p)


def u64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))
