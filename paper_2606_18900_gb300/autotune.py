"""Launch-configuration autotuner.

Times a decode call (whole-file or batch) under a small grid of launch
configurations of the library — persistent CTAs (wavefront width), working
warps per CTA, and shared-memory staging bytes per warp (staging depth) — and
keeps the fastest. Results are cached in a JSON file keyed by the GPU name
and a caller-given workload key, so a later run applies the cached choice
without re-timing. Timing uses CUDA events on the call's stream.
"""
from __future__ import annotations

import json
import os
import threading

_lock = threading.Lock()
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "aceapex_autotune.json")


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def candidates(max_ctas: int):
    out = []
    for frac in (1.0, 0.75, 0.5):
        for warps in (32, 24, 16):
            for stage in (3072, 1024):
                out.append((max(1, int(max_ctas * frac)), warps, stage))
    return out


def tune(handle, run, *, key: str, reps: int = 3, cache_path: str | None = None, retune: bool = False,
         stream=None, cands=None):
    """Pick and apply the fastest launch configuration for ``run()``.

    handle: the Archive whose launch knobs ``run`` uses (for batches, the
    first archive). run: issues one decode on ``stream``. Returns
    (config dict, table of (config, ms)).
    """
    import torch

    cache_path = cache_path or DEFAULT_CACHE
    gpu = torch.cuda.get_device_name(handle.device)
    full_key = f"{gpu}|{key}"
    with _lock:
        cache = _load(cache_path)
    if not retune and full_key in cache:
        c = cache[full_key]
        handle.set_launch(c["ctas"], c["warps_per_cta"], c["stage_bytes"])
        return c, []
    handle.set_launch()
    max_ctas = handle.get_launch()["max_ctas"]
    table = []
    s = stream or torch.cuda.current_stream()
    for ctas, warps, stage in (cands or candidates(max_ctas)):
        handle.set_launch(ctas, warps, stage)
        run()
        handle.check(s)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        for _ in range(reps):
            run()
        b.record(s)
        b.synchronize()
        handle.check(s)
        table.append(({"ctas": ctas, "warps_per_cta": warps, "stage_bytes": stage}, a.elapsed_time(b) / reps))
    best, ms = min(table, key=lambda t: t[1])
    handle.set_launch(best["ctas"], best["warps_per_cta"], best["stage_bytes"])
    rec = dict(best, ms=ms)
    with _lock:
        cache = _load(cache_path)
        cache[full_key] = rec
        _store(cache_path, cache)
    return rec, table
