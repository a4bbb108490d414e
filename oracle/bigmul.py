"""ctypes front end of ``oracle/bigmul.c`` (test infrastructure only).

Exact full product of little-endian uint64 limb arrays and the low / high
products by their definitions (Section 1 of the paper):
  low  product: w = uv mod 2^n;
  high product: any 0 <= w <= 2^n with |uv - 2^n w| < 2^n, i.e. w = floor(uv/2^n),
                or floor(uv/2^n) + 1 when uv mod 2^n != 0.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bigmul.c")
_LIB = os.path.join(_HERE, "liboracle_bigmul.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile bigmul.c into a shared library next to it (plain gcc, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", _LIB, _SRC])
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            p64 = ctypes.POINTER(ctypes.c_uint64)
            lib.oracle_mul_full.argtypes = [p64, p64, p64, ctypes.c_size_t, ctypes.c_int]
            lib.oracle_mul_lo.argtypes = [p64, p64, p64, ctypes.c_uint64, ctypes.c_int]
            lib.oracle_mul_hi_floor.argtypes = [p64, ctypes.POINTER(ctypes.c_int), p64, p64,
                                                ctypes.c_uint64, ctypes.c_int]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def limbs_for(n_bits: int) -> int:
    return (n_bits + 63) // 64


def mul_full(u: np.ndarray, v: np.ndarray, par_depth: int = 0) -> np.ndarray:
    """Exact product u*v of two equal-length limb arrays -> 2*len(u) limbs."""
    u = np.ascontiguousarray(u, dtype=np.uint64)
    v = np.ascontiguousarray(v, dtype=np.uint64)
    assert u.shape == v.shape and u.ndim == 1
    out = np.zeros(2 * u.size, dtype=np.uint64)
    if u.size:
        _load().oracle_mul_full(_ptr(out), _ptr(u), _ptr(v), u.size, par_depth)
    return out


def mul_lo(u: np.ndarray, v: np.ndarray, n_bits: int, par_depth: int = 0) -> np.ndarray:
    """Low product uv mod 2^n (Section 1) -> ceil(n/64) limbs."""
    u = np.ascontiguousarray(u, dtype=np.uint64)
    v = np.ascontiguousarray(v, dtype=np.uint64)
    assert u.size == v.size == limbs_for(n_bits)
    out = np.zeros(limbs_for(n_bits), dtype=np.uint64)
    _load().oracle_mul_lo(_ptr(out), _ptr(u), _ptr(v), n_bits, par_depth)
    return out


def mul_hi_floor(u: np.ndarray, v: np.ndarray, n_bits: int, par_depth: int = 0):
    """(q, q_plus_one_ok): q = floor(uv / 2^n) as floor(n/64)+1 limbs, and whether
    q + 1 is also an admissible high product (Section 1: |uv - 2^n w| < 2^n)."""
    u = np.ascontiguousarray(u, dtype=np.uint64)
    v = np.ascontiguousarray(v, dtype=np.uint64)
    assert u.size == v.size == limbs_for(n_bits)
    out = np.zeros(n_bits // 64 + 1, dtype=np.uint64)
    nz = ctypes.c_int(0)
    _load().oracle_mul_hi_floor(_ptr(out), ctypes.byref(nz), _ptr(u), _ptr(v), n_bits, par_depth)
    return out, bool(nz.value)


# ---- conversions between limb arrays and Python integers (used by tests) ----

def to_int(limbs: np.ndarray) -> int:
    return int.from_bytes(np.ascontiguousarray(limbs, dtype="<u8").tobytes(), "little")


def from_int(x: int, nlimbs: int) -> np.ndarray:
    assert 0 <= x < (1 << (64 * nlimbs))
    return np.frombuffer(x.to_bytes(8 * nlimbs, "little"), dtype="<u8").astype(np.uint64)
