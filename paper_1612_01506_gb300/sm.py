"""Python binding of the C ABI in include/sm.h (ctypes; argument marshalling only).

Every function here has the name of the C entry point it calls. Device
buffers are torch CUDA tensors (``uint8`` texts; counts, positions
and histograms are 64-bit tensors, int64 by default, holding the ABI's
uint64 values); the stream is torch's current stream unless one is given. There is
no CPU fallback: if ``libsm.so`` is missing the first call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB as _LIB_PATH

SM_OK, SM_EINVAL, SM_ENOMEM, SM_ECUDA, SM_ETRUNC, SM_ETIMEOUT, SM_ENOTSUP = range(7)
SM_MAX_M = 4096
SM_TILE_STARTS = 16384
SM_ORDER_H, SM_ORDER_HS = 1, 2
SM_KNOB_STAGES, SM_KNOB_GRID, SM_KNOB_SPIN_NS, SM_KNOB_TEST_SKIP_COPY = 1, 2, 3, 4
SM_NOALLOC_MAX_STARTS = 16384 * 16384
SM_NOALLOC_TIMEOUT = (1 << 64) - 1   # *d_count after an expired bounded wait (int64 view: -1)

# Every symbol the header declares (checked against include/sm.h by the tests).
EXPORTS = ("sm_create", "sm_destroy", "sm_last_error", "sm_status_string", "sm_sync", "sm_set_knob",
           "sm_histogram", "sm_order", "sm_order_fixed", "sm_count", "sm_count_ex", "sm_report",
           "sm_report_ex", "sm_report_noalloc", "sm_batch_create", "sm_batch_count", "sm_batch_report",
           "sm_batch_tune", "sm_batch_destroy", "sm_count_batch", "sm_stepper_create", "sm_stepper_chunks", "sm_stepper_admit",
           "sm_stepper_step", "sm_stepper_steps", "sm_stepper_retire", "sm_stepper_report", "sm_stepper_destroy",
           "sm_tune_bucket", "sm_tune_set", "sm_tune_get", "sm_tune_search")
SM_TUNE_M_BUCKETS, SM_TUNE_SIGMA_BUCKETS = 13, 5


class SmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


SM_SEARCH_BYTES = 1


class BatchTuning(C.Structure):
    _fields_ = [("cand_freq", C.c_float), ("cand_min", C.c_uint32), ("stages", C.c_uint32), ("ms", C.c_float)]


class Tuning(C.Structure):
    _fields_ = [("peel", C.c_uint32), ("stages", C.c_uint32), ("ctas_per_sm", C.c_uint32), ("ms", C.c_float)]


class SearchOpts(C.Structure):
    _fields_ = [("peel", C.c_uint32), ("flags", C.c_uint32), ("h_hist256", C.POINTER(C.c_uint64))]


_lib = None


def library_path() -> str:
    """The CUDA library in use: $SM_LIBRARY if set, else the in-tree build."""
    return os.environ.get("SM_LIBRARY") or _LIB_PATH


def load():
    """Load libsm.so (built by ``__graft_entry__.build()``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = C.CDLL(path)
    vp, u8p, u32p, u64p = C.c_void_p, C.POINTER(C.c_uint8), C.POINTER(C.c_uint32), C.POINTER(C.c_uint64)
    st, u32, u64 = C.c_int, C.c_uint32, C.c_uint64
    sig = {
        "sm_create": (st, [C.POINTER(vp), C.c_int]),
        "sm_destroy": (None, [vp]),
        "sm_last_error": (C.c_char_p, []),
        "sm_status_string": (C.c_char_p, [st]),
        "sm_sync": (st, [vp, vp]),
        "sm_set_knob": (st, [vp, C.c_int, C.c_int64]),
        "sm_histogram": (st, [vp, vp, u64, vp, vp]),
        "sm_order": (st, [u8p, u32, u64p, u32p]),
        "sm_order_fixed": (st, [u8p, u32, C.c_int, u32p]),
        "sm_count": (st, [vp, vp, u64, u8p, u32, u32p, vp, vp]),
        "sm_count_ex": (st, [vp, vp, u64, u8p, u32, u32p, C.POINTER(SearchOpts), vp, vp]),
        "sm_report": (st, [vp, vp, u64, u8p, u32, u32p, vp, u64, vp, vp]),
        "sm_report_ex": (st, [vp, vp, u64, u8p, u32, u32p, C.POINTER(SearchOpts), vp, u64, vp, vp]),
        "sm_report_noalloc": (st, [vp, u64, u8p, u32, u32p, vp, u64, vp, vp]),
        "sm_batch_create": (st, [vp, vp, C.POINTER(C.c_int64), u32, u8p, C.POINTER(C.c_int64),
                                 C.POINTER(C.c_int32), u32, C.POINTER(vp), vp]),
        "sm_batch_count": (st, [vp, vp, vp]),
        "sm_batch_report": (st, [vp, vp, vp, vp, vp]),
        "sm_batch_tune": (st, [vp, u32, C.POINTER(BatchTuning), vp]),
        "sm_batch_destroy": (None, [vp]),
        "sm_count_batch": (st, [vp, vp, vp, u32, vp, vp, vp, u32, vp, vp, vp, vp]),
        "sm_tune_bucket": (st, [u64p, u32, u32p, u32p]),
        "sm_tune_set": (st, [vp, u32, u32, C.POINTER(Tuning)]),
        "sm_tune_get": (st, [vp, u32, u32, C.POINTER(Tuning)]),
        "sm_tune_search": (st, [vp, vp, u64, u64p, u8p, C.POINTER(C.c_int64), u32, u32, C.POINTER(Tuning), vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    _lib = lib
    return lib


def _status_name(s: int) -> str:
    names = ["SM_OK", "SM_EINVAL", "SM_ENOMEM", "SM_ECUDA", "SM_ETRUNC", "SM_ETIMEOUT", "SM_ENOTSUP"]
    return names[s] if 0 <= s < len(names) else f"status {s}"


def _check(status: int):
    if status != SM_OK:
        raise SmError(status, load().sm_last_error().decode(errors="replace"))


def _bytes(x) -> np.ndarray:
    if isinstance(x, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(x), dtype=np.uint8)
    a = np.ascontiguousarray(x)
    if a.dtype != np.uint8:
        raise TypeError("patterns must be bytes or uint8 arrays")
    return a


def _u8p(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_uint8)) if a.size else C.cast(C.c_char_p(b"\0"), C.POINTER(C.c_uint8))


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


_WORD64 = ("torch.int64", "torch.uint64")


def _dev_ptr(t, dtypes=None) -> int:
    if t is None:
        return 0
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device buffers must be contiguous CUDA tensors")
    if dtypes and str(t.dtype) not in dtypes:
        raise TypeError(f"expected one of {dtypes}, got {t.dtype}")
    return t.data_ptr()


class Ctx:
    """Owns an sm_ctx*; destroyed with the object."""

    def __init__(self, handle: int, device: int):
        self.handle, self.device = handle, device

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.sm_destroy(h)


def sm_create(device: int = 0) -> Ctx:
    h = C.c_void_p()
    _check(load().sm_create(C.byref(h), device))
    return Ctx(h.value, device)


def sm_sync(ctx: Ctx, stream=None) -> int:
    """Wait for the stream; return the deferred status (SM_OK, SM_ETRUNC, SM_ETIMEOUT)."""
    s = load().sm_sync(ctx.handle, _stream(stream))
    if s not in (SM_OK, SM_ETRUNC, SM_ETIMEOUT):
        _check(s)
    return s


def sm_set_knob(ctx: Ctx, knob: int, value: int):
    _check(load().sm_set_knob(ctx.handle, knob, value))


def sm_histogram(ctx: Ctx, text, out=None, stream=None):
    import torch
    if out is None:
        out = torch.empty(256, dtype=torch.int64, device=text.device)
    _check(load().sm_histogram(ctx.handle, _dev_ptr(text, ("torch.uint8",)), text.numel(),
                               _dev_ptr(out, _WORD64), _stream(stream)))
    return out


def sm_order(pattern, hist) -> np.ndarray:
    p = _bytes(pattern)
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    if h.size != 256:
        raise ValueError("histogram must have 256 entries")
    pi = np.zeros(max(p.size, 1), dtype=np.uint32)
    _check(load().sm_order(_u8p(p), p.size, h.ctypes.data_as(C.POINTER(C.c_uint64)),
                           pi.ctypes.data_as(C.POINTER(C.c_uint32))))
    return pi[: p.size]


def sm_order_fixed(pattern, mode: int) -> np.ndarray:
    p = _bytes(pattern)
    pi = np.zeros(max(p.size, 1), dtype=np.uint32)
    _check(load().sm_order_fixed(_u8p(p), p.size, mode, pi.ctypes.data_as(C.POINTER(C.c_uint32))))
    return pi[: p.size]


def _opts(peel: int, hist, bytes_only: bool = False):
    if not peel and hist is None and not bytes_only:
        return None, None
    h = None if hist is None else np.ascontiguousarray(hist, dtype=np.uint64)
    o = SearchOpts(peel, SM_SEARCH_BYTES if bytes_only else 0,
                   h.ctypes.data_as(C.POINTER(C.c_uint64)) if h is not None else None)
    return o, h


def _pi(pi, m):
    if pi is None:
        return None, None
    a = np.ascontiguousarray(pi, dtype=np.uint32)
    if a.size != m:
        raise ValueError("order must have m entries")
    return a.ctypes.data_as(C.POINTER(C.c_uint32)), a


def sm_count(ctx: Ctx, text, pattern, pi=None, out=None, stream=None, peel: int = 0, hist=None,
             bytes_only: bool = False):
    """Enqueue a count; returns the 1-element int64 device tensor it writes.
    bytes_only: compare bytes even where the 2-bit codes of a text of at most
    four symbols apply (SM_SEARCH_BYTES)."""
    import torch
    p = _bytes(pattern)
    if out is None:
        out = torch.empty(1, dtype=torch.int64, device=text.device)
    pip, _keep_pi = _pi(pi, p.size)
    o, _keep_h = _opts(peel, hist, bytes_only)
    lib = load()
    if o is None:
        st = lib.sm_count(ctx.handle, _dev_ptr(text, ("torch.uint8",)), text.numel(), _u8p(p), p.size, pip,
                          _dev_ptr(out, _WORD64), _stream(stream))
    else:
        st = lib.sm_count_ex(ctx.handle, _dev_ptr(text, ("torch.uint8",)), text.numel(), _u8p(p), p.size, pip,
                             C.byref(o), _dev_ptr(out, _WORD64), _stream(stream))
    _check(st)
    return out


def sm_report(ctx: Ctx, text, pattern, cap: int, pi=None, out_pos=None, out_count=None, stream=None,
              peel: int = 0, hist=None, bytes_only: bool = False):
    """Enqueue a report; returns (positions int64[cap], count int64[1]) device tensors."""
    import torch
    p = _bytes(pattern)
    if out_pos is None:
        out_pos = torch.empty(max(cap, 1), dtype=torch.int64, device=text.device)
    if out_count is None:
        out_count = torch.empty(1, dtype=torch.int64, device=text.device)
    pip, _keep_pi = _pi(pi, p.size)
    o, _keep_h = _opts(peel, hist, bytes_only)
    lib = load()
    if o is None:
        st = lib.sm_report(ctx.handle, _dev_ptr(text, ("torch.uint8",)), text.numel(), _u8p(p), p.size, pip,
                           _dev_ptr(out_pos, _WORD64), cap, _dev_ptr(out_count, _WORD64), _stream(stream))
    else:
        st = lib.sm_report_ex(ctx.handle, _dev_ptr(text, ("torch.uint8",)), text.numel(), _u8p(p), p.size, pip,
                              C.byref(o), _dev_ptr(out_pos, _WORD64), cap, _dev_ptr(out_count, _WORD64), _stream(stream))
    _check(st)
    return out_pos, out_count


def sm_report_noalloc(text, pattern, cap: int, out_pos, out_count, pi=None, stream=None) -> int:
    """Enqueue sm_report_noalloc into caller-provided buffers; returns the status.

    The C call allocates nothing; the caller passes the position buffer
    (at least ``cap`` 64-bit entries) and the 1-entry count buffer.
    """
    p = _bytes(pattern)
    pip, _keep_pi = _pi(pi, p.size)
    return load().sm_report_noalloc(_dev_ptr(text, ("torch.uint8",)), text.numel(), _u8p(p), p.size, pip,
                                    _dev_ptr(out_pos, _WORD64), cap, _dev_ptr(out_count, _WORD64),
                                    _stream(stream))


class Batch:
    """A planned batch (sm_batch*); destroyed with the object. Keeps the texts alive."""

    def __init__(self, handle: int, texts, npats: int):
        self.handle, self.texts, self.npats = handle, texts, npats

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.sm_batch_destroy(h)


def sm_batch_create(ctx: Ctx, texts, text_off, patterns: list, pat_text, stream=None) -> Batch:
    """Plan a batch: texts is one packed uint8 CUDA tensor with host offsets
    text_off (ntexts + 1); patterns a list of bytes, pattern k searched in
    text pat_text[k]."""
    toff = np.ascontiguousarray(text_off, dtype=np.int64)
    pt = np.ascontiguousarray(pat_text, dtype=np.int32)
    flat = np.frombuffer(b"".join(bytes(p) for p in patterns), dtype=np.uint8) if patterns else np.zeros(0, np.uint8)
    poff = np.zeros(len(patterns) + 1, dtype=np.int64)
    if patterns:
        poff[1:] = np.cumsum([len(p) for p in patterns])
    h = C.c_void_p()
    _check(load().sm_batch_create(ctx.handle, _dev_ptr(texts, ("torch.uint8",)), toff.ctypes.data_as(C.POINTER(C.c_int64)),
                                  toff.size - 1, _u8p(flat), poff.ctypes.data_as(C.POINTER(C.c_int64)),
                                  pt.ctypes.data_as(C.POINTER(C.c_int32)), len(patterns), C.byref(h), _stream(stream)))
    return Batch(h.value, texts, len(patterns))


def sm_batch_count(batch: Batch, out=None, stream=None):
    """Enqueue the batch; returns the int64 device tensor of counts (one per pattern)."""
    import torch
    if out is None:
        out = torch.empty(max(batch.npats, 1), dtype=torch.int64, device=batch.texts.device)
    _check(load().sm_batch_count(batch.handle, _dev_ptr(out, _WORD64), _stream(stream)))
    return out


def sm_batch_report(batch: Batch, d_pos_off, d_pos=None, out=None, stream=None):
    """Enqueue the batched report: positions of pattern k, ascending, into
    d_pos[d_pos_off[k] .. d_pos_off[k+1]) (d_pos_off: int64 CUDA tensor,
    npats + 1 entries; d_pos allocated when None). Returns (counts, d_pos)."""
    import torch
    if out is None:
        out = torch.empty(max(batch.npats, 1), dtype=torch.int64, device=batch.texts.device)
    if d_pos is None:
        d_pos = torch.empty(max(int(d_pos_off[-1].item()), 1), dtype=torch.int64, device=batch.texts.device)
    _check(load().sm_batch_report(batch.handle, _dev_ptr(out, _WORD64), _dev_ptr(d_pos, _WORD64),
                                  _dev_ptr(d_pos_off, _WORD64), _stream(stream)))
    return out, d_pos


def sm_batch_tune(batch: Batch, reps: int = 2, stream=None) -> dict:
    """Run the batch's autotuner; returns the chosen plan parameters and its ms per count."""
    t = BatchTuning()
    _check(load().sm_batch_tune(batch.handle, reps, C.byref(t), _stream(stream)))
    return {"cand_freq": round(t.cand_freq, 4), "cand_min": t.cand_min, "stages": t.stages, "ms": t.ms}


def sm_count_batch(ctx: Ctx, texts, d_text_off, d_pats, d_pat_off, d_pat_text, d_counts, d_pos=None,
                   d_pos_off=None, stream=None):
    """The one-shot batch call with device-resident metadata (all CUDA tensors)."""
    _check(load().sm_count_batch(ctx.handle, _dev_ptr(texts, ("torch.uint8",)), _dev_ptr(d_text_off, _WORD64),
                                 d_text_off.numel() - 1, _dev_ptr(d_pats, ("torch.uint8",)),
                                 _dev_ptr(d_pat_off, _WORD64), _dev_ptr(d_pat_text, ("torch.int32",)),
                                 d_pat_text.numel(), _dev_ptr(d_counts, _WORD64),
                                 _dev_ptr(d_pos, _WORD64) if d_pos is not None else None,
                                 _dev_ptr(d_pos_off, _WORD64) if d_pos_off is not None else None, _stream(stream)))
    return d_counts


# ------------------------------------------------------------------ tuning

def _tuning_dict(t: Tuning) -> dict:
    return {"peel": t.peel, "stages": t.stages, "ctas_per_sm": t.ctas_per_sm, "ms": round(float(t.ms), 6)}


def sm_tune_bucket(hist, m: int) -> tuple[int, int]:
    """(m bucket, sigma bucket) of a search for a pattern of length m in a text with this histogram."""
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    mb, sb = C.c_uint32(), C.c_uint32()
    _check(load().sm_tune_bucket(h.ctypes.data_as(C.POINTER(C.c_uint64)), m, C.byref(mb), C.byref(sb)))
    return mb.value, sb.value


def sm_tune_set(ctx: Ctx, m_bucket: int, sigma_bucket: int, plan: dict | None):
    """Install a plan ({"peel", "stages", "ctas_per_sm"}; None clears) for a bucket."""
    t = None if plan is None else Tuning(int(plan.get("peel", 0)), int(plan.get("stages", 0)),
                                         int(plan.get("ctas_per_sm", 0)), float(plan.get("ms", 0.0)))
    _check(load().sm_tune_set(ctx.handle, m_bucket, sigma_bucket, C.byref(t) if t is not None else None))


def sm_tune_get(ctx: Ctx, m_bucket: int, sigma_bucket: int) -> dict:
    t = Tuning()
    _check(load().sm_tune_get(ctx.handle, m_bucket, sigma_bucket, C.byref(t)))
    return _tuning_dict(t)


def sm_tune_search(ctx: Ctx, text, hist, patterns: list, reps: int = 3, stream=None) -> dict:
    """Autotune the bucket of `patterns` (one m bucket) on `text`; installs and returns the best plan."""
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    flat = np.frombuffer(b"".join(bytes(p) for p in patterns), dtype=np.uint8)
    off = np.zeros(len(patterns) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(p) for p in patterns])
    t = Tuning()
    _check(load().sm_tune_search(ctx.handle, _dev_ptr(text, ("torch.uint8",)), text.numel(),
                                 h.ctypes.data_as(C.POINTER(C.c_uint64)), _u8p(flat),
                                 off.ctypes.data_as(C.POINTER(C.c_int64)), len(patterns), reps, C.byref(t),
                                 _stream(stream)))
    return _tuning_dict(t)
