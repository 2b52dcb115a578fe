"""Autotuner for the launch shapes of the solver (times candidates on the GPU,
caches the winner per device and workload class in a JSON file).

Tunables:
  * Householder tridiagonalisation: row tiles per work item of its
    matrix-vector kernel (granularity of the per-column work queue);
  * back-transformations: the split-K cap of their thin V^H Z products;
  * mixed form: the m*n*k threshold above which complex products use the
    split-operand tensor-core engine instead of the FP64 FMA engine;
  * batched solves: the team size (CTAs of one cluster per large instance)
    and the size from which instances get a team;
  * batched persistent kernel without teams: resident CTAs per SM (1 or 2).

Every candidate is timed with CUDA events on the current stream after one
untimed run; the cache key contains the device name, the workload class
(size bucket) and the tunable's name.  A table tuned on a GB300 ships with
the package (tuned_gb300.json); the user cache (BSE_AUTOTUNE_CACHE or
~/.cache/bse_gb300/autotune.json) takes precedence over it.  The tile shapes
of the GEMM engines and the tensor-core kernel's stage ring are compile-time
constants of their kernels and are not tuned here.

    python -m paper_2008_08825_gb300.autotune --n 8192 --out tuned.json
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


SHIPPED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_gb300.json")


_files: dict = {}  # path -> (mtime, contents)


def _load(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        mt = os.path.getmtime(path)
        hit = _files.get(path)
        if hit and hit[0] == mt:
            return hit[1]
        with open(path) as f:
            d = json.load(f)
        _files[path] = (mt, d)
        return d
    except (OSError, ValueError):
        return {}


def lookup(key: str):
    """The cached choice for `key`: the user cache first, then the shipped table."""
    v = _load().get(key)
    return v if v is not None else _load(SHIPPED).get(key)


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


def size_bucket(n: int) -> int:
    return 2 ** math.ceil(math.log2(max(int(n), 1)))


def _launch_key(n: int, precision: str) -> str:
    return f"{_device_key()}/launch/n{size_bucket(n)}/{precision}"


def tune_launch_shapes(A: torch.Tensor, B: torch.Tensor, handle: "bse.Handle", precision: str = "fp64",
                       hemv_candidates=(2, 4, 8, 16), splitk_candidates=(1, 2, 4, 8), force: bool = False) -> dict:
    """Pick the matvec work-item size (timed on eigenvalues-only Alg. 2 solves,
    which the reduction dominates) and then the split-K cap (timed on Alg. 2
    solves with vectors, where the back-transformation runs) for this size
    and precision; apply both to `handle`."""
    n = A.shape[0]
    key = _launch_key(n, precision)
    cached = None if force else _load().get(key)
    if cached is None:
        t_h = {}
        for c in hemv_candidates:
            handle.set_launch_shapes(c, 0)
            t_h[c] = _time(lambda: bse.solve(A, B, method="chol", precision=precision, vectors=False, handle=handle))
        best_h = min(t_h, key=t_h.get)
        t_s = {}
        for c in splitk_candidates:
            handle.set_launch_shapes(best_h, c)
            t_s[c] = _time(lambda: bse.solve(A, B, method="chol", precision=precision, handle=handle))
        best_s = min(t_s, key=t_s.get)
        cached = {"hemv_item_tiles": best_h, "splitk_max": best_s,
                  "ms_values_only_by_hemv_item_tiles": {str(k): v for k, v in t_h.items()},
                  "ms_with_vectors_by_splitk_max": {str(k): v for k, v in t_s.items()}}
        _store(key, cached)
    handle.set_launch_shapes(cached["hemv_item_tiles"], cached["splitk_max"])
    return cached


def tune_batched_teams(batch: "bse.Batch", handle: "bse.Handle",
                       candidates=((1, 448), (2, 448), (4, 320), (4, 448), (4, 640), (8, 640)),
                       force: bool = False) -> dict:
    """Pick the team size and threshold of a batched solve for this method and batch class."""
    key = f"{_device_key()}/batched_team/{batch.method}/{batch_class(batch.n)}/k{batch.k}"
    cached = None if force else _load().get(key)
    if cached is None:
        times = {}
        for team, min_n in candidates:
            handle.set_batch_team(team, min_n)
            times[f"{team}/{min_n}"] = _time(lambda: batch.run(handle=handle))
        best = min(times, key=times.get)
        team, min_n = (int(x) for x in best.split("/"))
        cached = {"team": team, "min_n": min_n, "ms": times}
        _store(key, cached)
    handle.set_batch_team(cached["team"], cached["min_n"])
    return cached


def apply_tuned(handle: "bse.Handle", n: int, precision: str = "fp64") -> dict:
    """Apply the cached launch shapes for size n (user cache, else the shipped
    table) to `handle`; returns what was applied ({} when nothing is cached)."""
    cached = lookup(_launch_key(n, precision))
    if not cached:
        return {}
    handle.set_launch_shapes(cached["hemv_item_tiles"], cached["splitk_max"])
    out = {"hemv_item_tiles": cached["hemv_item_tiles"], "splitk_max": cached["splitk_max"]}
    tc = lookup(f"{_device_key()}/tc_min_mnk/chol/n{size_bucket(n)}") if precision == "mixed" else None
    if tc:
        handle.set_tc_min_mnk(tc["tc_min_mnk"])
        out["tc_min_mnk"] = tc["tc_min_mnk"]
    return out


def apply_tuned_batched(handle: "bse.Handle", batch: "bse.Batch") -> dict:
    cached = lookup(f"{_device_key()}/batched_team/{batch.method}/{batch_class(batch.n)}/k{batch.k}")
    if not cached:
        return {}
    handle.set_batch_team(cached["team"], cached["min_n"])
    return {"team": cached["team"], "min_n": cached["min_n"]}


def main():
    """Tune on this GPU for the n = 8192 workload (both precisions) and the
    512-instance batched workload; write the table to --out."""
    import argparse

    from . import inputs

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--out", default=None, help="write the tuned entries here (default: the user cache)")
    args = ap.parse_args()
    if args.out:
        os.environ["BSE_AUTOTUNE_CACHE"] = args.out
    dev = torch.device("cuda", 0)
    A, B = inputs.base(args.n, 0)
    At, Bt = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    del A, B
    h = bse.Handle()
    for prec in ("fp64", "mixed"):
        print(prec, tune_launch_shapes(At, Bt, h, precision=prec, force=True), flush=True)
    print("tc", tune_tc_threshold(At, Bt, "chol", h, candidates=(1 << 21, 1 << 24, 1 << 27), force=True), flush=True)
    del At, Bt
    torch.cuda.empty_cache()
    sizes = inputs.batched_sizes()
    inst = []
    for i in range(len(sizes)):
        A, B = inputs.base(int(sizes[i]), seed=i)
        inst.append((torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)))
    for method in ("chol", "svd"):
        bt = bse.Batch(inst, k=32, method=method)
        print("teams", method, tune_batched_teams(bt, h, force=True), flush=True)


if __name__ == "__main__":
    main()
