"""Oracle for exact string matching -- TEST INFRASTRUCTURE ONLY.

Plain C (``oracle.c``) wrapped with ctypes. Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package. It shares no code with the CUDA library and the library never
calls it.

What each function follows (Tarhio, Holub, Giaquinta, "Technology Beats
Algorithms (in Exact String Matching)"):

* ``naive_count`` / ``naive_report`` -- Algorithm 1 (Sec. 2.1), 0-based,
  the reporting version emitting position i where Algorithm 1 counts.
* ``memcmp_count`` / ``kmp_count`` -- independent cross-checks (brute force
  and the Knuth-Morris-Pratt automaton cited in Sec. 1).
* ``histogram`` -- symbol frequencies of the searched text (Sec. 2.2).
* ``order_freq`` -- Sec. 2.2 / Algorithm 3: positions by increasing symbol
  frequency, ties by ascending position.
* ``order_h`` / ``order_hs`` -- the fixed orders of Sec. 2.4.
* ``batch_count`` -- Algorithm 1 over each (text, pattern) pair of a batch.
* ``count_threads`` / ``report_threads`` -- Algorithm 1 on start ranges split
  across host threads, for the CPU baseline and large inputs.

Every function is pinned by ``tests/test_oracle.py`` against values the paper
prints (Fig. 1), closed forms, brute force on tiny inputs and invariants.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build", platform.machine())
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/<machine>/liboracle.so with gcc."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    u8p, u64p, u32p = C.POINTER(C.c_uint8), C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)
    i64p, i32p = C.POINTER(C.c_int64), C.POINTER(C.c_int32)
    u64 = C.c_uint64
    for name in ("oracle_naive_count", "oracle_memcmp_count", "oracle_kmp_count"):
        f = getattr(lib, name)
        f.argtypes = [u8p, u64, u8p, u64]
        f.restype = u64
    lib.oracle_naive_report.argtypes = [u8p, u64, u8p, u64, u64p, u64]
    lib.oracle_naive_report.restype = u64
    lib.oracle_histogram.argtypes = [u8p, u64, u64p]
    lib.oracle_histogram.restype = None
    lib.oracle_order_freq.argtypes = [u8p, C.c_uint32, u64p, u32p]
    lib.oracle_order_freq.restype = C.c_int
    lib.oracle_order_h.argtypes = [C.c_uint32, u32p]
    lib.oracle_order_h.restype = C.c_int
    lib.oracle_order_hs.argtypes = [u8p, C.c_uint32, u32p]
    lib.oracle_order_hs.restype = C.c_int
    lib.oracle_batch_count.argtypes = [u8p, i64p, C.c_uint32, u8p, i64p, i32p, C.c_uint32, i64p]
    lib.oracle_batch_count.restype = C.c_int
    lib.oracle_count_threads.argtypes = [u8p, u64, u8p, u64, C.c_int]
    lib.oracle_count_threads.restype = u64
    lib.oracle_report_threads.argtypes = [u8p, u64, u8p, u64, u64p, u64, C.c_int]
    lib.oracle_report_threads.restype = u64
    return lib


def _u8(x) -> np.ndarray:
    if isinstance(x, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(x), dtype=np.uint8)
    a = np.ascontiguousarray(x)
    if a.dtype != np.uint8:
        raise TypeError("byte arrays must be uint8")
    return a


def _ptr(a: np.ndarray, ct):
    # a zero-length array still needs a valid pointer
    if a.size == 0:
        a = np.zeros(1, dtype=a.dtype)
    return a.ctypes.data_as(C.POINTER(ct)), a


class Oracle:
    """The oracle's functions bound to one compiled copy of oracle.c."""

    def __init__(self, lib_path: str):
        self.path = lib_path
        self._lib = _bind(C.CDLL(lib_path))

    def naive_count(self, p, t) -> int:
        p, t = _u8(p), _u8(t)
        (pp, _k1), (tp, _k2) = _ptr(p, C.c_uint8), _ptr(t, C.c_uint8)
        return int(self._lib.oracle_naive_count(pp, p.size, tp, t.size))

    def naive_report(self, p, t, cap: int | None = None) -> tuple[np.ndarray, int]:
        """Return (positions, count); at most ``cap`` positions (default: all)."""
        p, t = _u8(p), _u8(t)
        if cap is None:
            cap = max(t.size - p.size + 1, 0) if p.size else t.size + 1
        out = np.zeros(max(cap, 1), dtype=np.uint64)
        (pp, _k1), (tp, _k2) = _ptr(p, C.c_uint8), _ptr(t, C.c_uint8)
        c = int(self._lib.oracle_naive_report(pp, p.size, tp, t.size,
                                            out.ctypes.data_as(C.POINTER(C.c_uint64)), cap))
        return out[: min(c, cap)].copy(), c

    def memcmp_count(self, p, t) -> int:
        p, t = _u8(p), _u8(t)
        (pp, _k1), (tp, _k2) = _ptr(p, C.c_uint8), _ptr(t, C.c_uint8)
        return int(self._lib.oracle_memcmp_count(pp, p.size, tp, t.size))

    def kmp_count(self, p, t) -> int:
        p, t = _u8(p), _u8(t)
        (pp, _k1), (tp, _k2) = _ptr(p, C.c_uint8), _ptr(t, C.c_uint8)
        return int(self._lib.oracle_kmp_count(pp, p.size, tp, t.size))

    def histogram(self, t) -> np.ndarray:
        t = _u8(t)
        h = np.zeros(256, dtype=np.uint64)
        tp, _k = _ptr(t, C.c_uint8)
        self._lib.oracle_histogram(tp, t.size, h.ctypes.data_as(C.POINTER(C.c_uint64)))
        return h

    def order_freq(self, p, hist) -> np.ndarray:
        p = _u8(p)
        h = np.ascontiguousarray(hist, dtype=np.uint64)
        pi = np.zeros(max(p.size, 1), dtype=np.uint32)
        pp, _k = _ptr(p, C.c_uint8)
        if self._lib.oracle_order_freq(pp, p.size, h.ctypes.data_as(C.POINTER(C.c_uint64)),
                                     pi.ctypes.data_as(C.POINTER(C.c_uint32))) != 0:
            raise MemoryError
        return pi[: p.size].copy()

    def order_h(self, m: int) -> np.ndarray:
        pi = np.zeros(max(m, 1), dtype=np.uint32)
        if self._lib.oracle_order_h(m, pi.ctypes.data_as(C.POINTER(C.c_uint32))) != 0:
            raise MemoryError
        return pi[:m].copy()

    def order_hs(self, p) -> np.ndarray:
        p = _u8(p)
        pi = np.zeros(max(p.size, 1), dtype=np.uint32)
        pp, _k = _ptr(p, C.c_uint8)
        if self._lib.oracle_order_hs(pp, p.size, pi.ctypes.data_as(C.POINTER(C.c_uint32))) != 0:
            raise MemoryError
        return pi[: p.size].copy()

    def batch_count(self, texts: np.ndarray, text_off: np.ndarray, pats: np.ndarray,
                    pat_off: np.ndarray, pat_text: np.ndarray) -> np.ndarray:
        texts, pats = _u8(texts), _u8(pats)
        text_off = np.ascontiguousarray(text_off, dtype=np.int64)
        pat_off = np.ascontiguousarray(pat_off, dtype=np.int64)
        pat_text = np.ascontiguousarray(pat_text, dtype=np.int32)
        npats = pat_text.size
        out = np.zeros(max(npats, 1), dtype=np.int64)
        tp, _k1 = _ptr(texts, C.c_uint8)
        pp, _k2 = _ptr(pats, C.c_uint8)
        rc = self._lib.oracle_batch_count(tp, text_off.ctypes.data_as(C.POINTER(C.c_int64)),
                                        text_off.size - 1, pp,
                                        pat_off.ctypes.data_as(C.POINTER(C.c_int64)),
                                        pat_text.ctypes.data_as(C.POINTER(C.c_int32)),
                                        npats, out.ctypes.data_as(C.POINTER(C.c_int64)))
        if rc != 0:
            raise ValueError("pattern refers to a missing text")
        return out[:npats].copy()

    def count_threads(self, p, t, threads: int | None = None) -> int:
        p, t = _u8(p), _u8(t)
        threads = threads or os.cpu_count() or 1
        (pp, _k1), (tp, _k2) = _ptr(p, C.c_uint8), _ptr(t, C.c_uint8)
        return int(self._lib.oracle_count_threads(pp, p.size, tp, t.size, threads))

    def report_threads(self, p, t, cap: int, threads: int | None = None) -> tuple[np.ndarray, int]:
        p, t = _u8(p), _u8(t)
        threads = threads or os.cpu_count() or 1
        out = np.zeros(max(cap, 1), dtype=np.uint64)
        (pp, _k1), (tp, _k2) = _ptr(p, C.c_uint8), _ptr(t, C.c_uint8)
        c = int(self._lib.oracle_report_threads(pp, p.size, tp, t.size,
                                              out.ctypes.data_as(C.POINTER(C.c_uint64)), cap, threads))
        return out[: min(c, cap)].copy(), c


_default: Oracle | None = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


def __getattr__(name):
    # module-level access to the default instance: oracle.naive_count(...)
    if name.startswith("_"):
        raise AttributeError(name)
    return getattr(default(), name)

