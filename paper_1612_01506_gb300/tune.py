"""Autotuned plans of the single-pattern scan, kept in a JSON cache.

Sec. 2.3 of the paper leaves the peeling factor r to tuning; on the GPU the
pipeline depth and the CTAs per SM also change the speed of a search, never
its result. ``autotune`` measures, for each (m bucket, sigma bucket) of a text
and a set of pattern lengths, the plan that ``sm_tune_search`` finds fastest
(peel, stages, CTAs per SM) and installs it in the context; ``save`` merges
the plans into a JSON file under the GPU's name and ``load`` installs them in
a new context, so that later processes on the same kind of GPU start tuned.

The cache file (``$SM_TUNE_CACHE``, else
``~/.cache/paper_1612_01506_gb300/tune.json``) maps a GPU key to a list of
entries ``{"m_bucket", "sigma_bucket", "peel", "stages", "ctas_per_sm",
"ms"}``; fields 0 keep the library's defaults.
"""
from __future__ import annotations

import json
import os

from . import sm, synth

FIELDS = ("peel", "stages", "ctas_per_sm")


def cache_path() -> str:
    return os.environ.get("SM_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache",
                                                           "paper_1612_01506_gb300", "tune.json")


def gpu_key(device: int = 0) -> str:
    import torch
    p = torch.cuda.get_device_properties(device)
    return f"{p.name} ({p.multi_processor_count} SMs)"


def read_entries(path: str, key: str) -> list[dict]:
    """The entries stored for `key` (empty when the file or key is missing)."""
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return []
    out = []
    for e in data.get(key, []):
        try:
            out.append({"m_bucket": int(e["m_bucket"]), "sigma_bucket": int(e["sigma_bucket"]),
                        **{k: int(e.get(k, 0)) for k in FIELDS}, "ms": float(e.get("ms", 0.0))})
        except (KeyError, TypeError, ValueError):
            continue
    return out


def write_entries(path: str, key: str, entries: list[dict]) -> None:
    """Merge `entries` into the file under `key` (a bucket's new entry replaces its old one)."""
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {}
    merged = {(e["m_bucket"], e["sigma_bucket"]): e for e in read_entries(path, key)}
    for e in entries:
        merged[(e["m_bucket"], e["sigma_bucket"])] = dict(e)
    data[key] = [merged[k] for k in sorted(merged)]
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def install(ctx, entries: list[dict]) -> int:
    """Install plans in a context; returns how many."""
    for e in entries:
        sm.sm_tune_set(ctx, e["m_bucket"], e["sigma_bucket"], e)
    return len(entries)


def load(ctx, path: str | None = None, device: int | None = None) -> int:
    """Install the cached plans of this GPU in `ctx`; returns how many."""
    return install(ctx, read_entries(path or cache_path(), gpu_key(ctx.device if device is None else device)))


def save(entries: list[dict], path: str | None = None, device: int = 0) -> str:
    path = path or cache_path()
    write_entries(path, gpu_key(device), entries)
    return path


def autotune(ctx, text, hist, host_text, ms, patterns: int = 8, reps: int = 3, seed: int = 1) -> list[dict]:
    """Tune the buckets of pattern lengths `ms` on the device text `text`
    (host copy `host_text`, histogram `hist`): `patterns` patterns per length
    copied from the text at seeded offsets, one sm_tune_search per length.
    Returns the entries (also installed in ctx)."""
    out = []
    for m in ms:
        pats = synth.sample_patterns(host_text, m, patterns, seed=seed, stream=synth.stream_id("tune", m))
        plan = sm.sm_tune_search(ctx, text, hist, pats, reps=reps)
        mb, sb = sm.sm_tune_bucket(hist, m)
        out.append({"m_bucket": mb, "sigma_bucket": sb, **{k: plan[k] for k in FIELDS}, "ms": plan["ms"]})
    return out
