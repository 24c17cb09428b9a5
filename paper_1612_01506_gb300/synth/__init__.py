"""Seeded synthetic texts and patterns (input generation only).

The paper's corpora (bible.txt, a Czech novel, E.coli, a protein file) are not
available, so inputs are synthetic stand-ins with the same alphabet sizes and
structure:

* ``uniform(n, sigma)`` -- i.i.d. symbols over a fixed alphabet: sigma=2
  ``"01"``, 4 ``"ACGT"`` (stand-in for E.coli), 20 the amino-acid letters
  (stand-in for the protein file), 64 the base64 alphabet, 256 all bytes.
* ``markov95(n)`` -- English-like text over the 95 printable ASCII bytes with
  Zipf(s=1) stationary frequencies (space the most frequent), first-order
  Markov correlation between neighbours (stand-in for bible.txt and the
  Czech novel).
* ``sample_patterns`` -- patterns copied from the text at seeded offsets
  ("picked randomly from the text", Sec. 2.3 of the paper).

Generation is in C (``synth.c``, counter-based SplitMix64, threaded) and
holds no matching arithmetic. Both the oracle and the CUDA library receive
the same bytes from here.
"""
from __future__ import annotations

import ctypes as C
import hashlib
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_OUT_DIR = os.path.join(os.path.dirname(_HERE), "_build", platform.machine())
_LIB_PATH = os.path.join(_OUT_DIR, "libsynth.so")
_lib = None

ALPHABETS: dict[int, bytes] = {
    2: b"01",
    4: b"ACGT",
    20: b"ACDEFGHIKLMNPQRSTVWY",
    64: b"ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz0123456789+/",
    256: bytes(range(256)),
}
MARKOV95 = bytes(range(0x20, 0x7F))


def build(force: bool = False) -> str:
    """Compile synth.c into the package's _build/libsynth.so with gcc."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        u64 = C.c_uint64
        lib.synth_draw.argtypes = [u64, u64, u64]
        lib.synth_draw.restype = u64
        lib.synth_below.argtypes = [C.POINTER(u64), u64, u64, u64, u64]
        lib.synth_below.restype = None
        lib.synth_uniform.argtypes = [C.c_void_p, u64, C.c_char_p, C.c_uint32, u64, u64, C.c_int]
        lib.synth_uniform.restype = C.c_int
        lib.synth_markov95.argtypes = [C.c_void_p, u64, u64, u64, C.c_int]
        lib.synth_markov95.restype = C.c_int
        lib.synth_markov95_weights.argtypes = [C.POINTER(u64), u64]
        lib.synth_markov95_weights.restype = None
        _lib = lib
    return _lib


def _threads(threads):
    return int(threads or min(os.cpu_count() or 1, 64))


def stream_id(*parts) -> int:
    """A stable 64-bit stream id from any printable description of a case."""
    h = hashlib.blake2b(repr(parts).encode(), digest_size=8).digest()
    return int.from_bytes(h, "little")


def draw(seed: int, stream: int, index: int) -> int:
    return int(_load().synth_draw(seed, stream, index))


def below(k: int, bound: int, seed: int, stream: int) -> np.ndarray:
    """k counter-based integers uniform in [0, bound)."""
    out = np.zeros(max(k, 1), dtype=np.uint64)
    _load().synth_below(out.ctypes.data_as(C.POINTER(C.c_uint64)), k, bound, seed, stream)
    return out[:k]


def uniform(n: int, sigma: int, seed: int = 0, stream: int = 0, threads=None,
            alphabet: bytes | None = None, out: np.ndarray | None = None) -> np.ndarray:
    alpha = alphabet if alphabet is not None else ALPHABETS[sigma]
    if len(alpha) != sigma:
        raise ValueError("alphabet length must equal sigma")
    buf = out if out is not None else np.empty(max(n, 1), dtype=np.uint8)
    if n:
        rc = _load().synth_uniform(buf.ctypes.data, n, alpha, sigma, seed, stream, _threads(threads))
        if rc != 0:
            raise ValueError("synth_uniform failed")
    return buf[:n]


def markov95(n: int, seed: int = 0, stream: int = 0, threads=None,
             out: np.ndarray | None = None) -> np.ndarray:
    buf = out if out is not None else np.empty(max(n, 1), dtype=np.uint8)
    if n:
        _load().synth_markov95(buf.ctypes.data, n, seed, stream, _threads(threads))
    return buf[:n]


def markov95_weights(seed: int = 0) -> np.ndarray:
    w = np.zeros(256, dtype=np.uint64)
    _load().synth_markov95_weights(w.ctypes.data_as(C.POINTER(C.c_uint64)), seed)
    return w


def text(kind: str | int, n: int, seed: int = 0, stream: int = 0, threads=None,
         out: np.ndarray | None = None) -> np.ndarray:
    """kind: an alphabet size (2, 4, 20, 64, 256) or "markov95"."""
    if kind in ("markov95", 95):
        return markov95(n, seed, stream, threads, out=out)
    return uniform(n, int(kind), seed, stream, threads, out=out)


def alphabet_of(kind: str | int) -> bytes:
    return MARKOV95 if kind in ("markov95", 95) else ALPHABETS[int(kind)]


def sample_offsets(n: int, m: int, k: int, seed: int, stream: int) -> np.ndarray:
    if m > n:
        raise ValueError("pattern longer than text")
    return below(k, n - m + 1, seed, stream)


def sample_patterns(t: np.ndarray, m: int, k: int, seed: int = 0, stream: int = 0) -> list[bytes]:
    """k patterns of length m copied from t at seeded offsets."""
    offs = sample_offsets(t.size, m, k, seed, stream)
    return [t[int(o): int(o) + m].tobytes() for o in offs]


def random_patterns(alphabet: bytes, m: int, k: int, seed: int = 0, stream: int = 0) -> list[bytes]:
    """k patterns of length m with i.i.d. symbols over ``alphabet``."""
    a = np.frombuffer(alphabet, dtype=np.uint8)
    idx = below(k * m, len(alphabet), seed, stream).reshape(k, m) if k * m else np.zeros((k, m), np.uint64)
    return [a[row.astype(np.int64)].tobytes() for row in idx]
