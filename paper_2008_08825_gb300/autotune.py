"""Autotuner for the launch shapes of the solver (times candidates on the GPU,
caches the winner per device and workload class in a JSON file).

Tunables:
  * batched persistent kernel: resident CTAs per SM (1 or 2) -- one CTA per
    SM gives the largest instances the whole FP64 pipe of their SM, two hide
    more latency; the best choice depends on the size mix of the batch;
  * mixed form: the m*n*k threshold above which complex products use the
    split-operand tensor-core engine instead of the FP64 FMA engine.

Every candidate is timed with CUDA events on the current stream after one
untimed run; the cache key contains the device name, the library's workload
class (size bucket) and the tunable's name.
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

from . import bse

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("BSE_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "bse_gb300", "autotune.json"))


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, value) -> None:
    with _lock:
        d = _load()
        d[key] = value
        path = cache_path()
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def _device_key() -> str:
    return torch.cuda.get_device_name().replace(" ", "_")


def _time(fn, reps: int = 1) -> float:
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def batch_class(sizes) -> str:
    """Workload class of a batch: count bucket and largest-size bucket (powers of 2)."""
    sizes = list(sizes)
    return f"c{2 ** math.ceil(math.log2(max(len(sizes), 1)))}_nmax{2 ** math.ceil(math.log2(max(sizes)))}"


def tune_batched(batch: "bse.Batch", handle: "bse.Handle", force: bool = False) -> dict:
    """Pick the CTAs-per-SM density for `batch` and apply it to `handle`."""
    key = f"{_device_key()}/batched/{batch_class(batch.n)}/k{batch.k}"
    cached = None if force else _load().get(key)
    if cached is None:
        times = {}
        for cps in (1, 2):
            handle.set_batch_ctas_per_sm(cps)
            times[cps] = _time(lambda: batch.run(handle=handle))
        best = min(times, key=times.get)
        cached = {"ctas_per_sm": best, "ms": {str(k): v for k, v in times.items()}}
        _store(key, cached)
    handle.set_batch_ctas_per_sm(cached["ctas_per_sm"])
    return cached


def tune_tc_threshold(A: torch.Tensor, B: torch.Tensor, method: str, handle: "bse.Handle",
                      candidates=(1 << 18, 1 << 21, 1 << 24, 1 << 27), force: bool = False) -> dict:
    """Pick the tensor-core product threshold of the mixed form for this size."""
    n = A.shape[0]
    key = f"{_device_key()}/tc_min_mnk/{method}/n{2 ** math.ceil(math.log2(max(n, 1)))}"
    cached = None if force else _load().get(key)
    if cached is None:
        times = {}
        for c in candidates:
            handle.set_tc_min_mnk(c)
            times[c] = _time(lambda: bse.solve(A, B, method=method, precision="mixed", handle=handle))
        best = min(times, key=times.get)
        cached = {"tc_min_mnk": best, "ms": {str(k): v for k, v in times.items()}}
        _store(key, cached)
    handle.set_tc_min_mnk(cached["tc_min_mnk"])
    return cached
