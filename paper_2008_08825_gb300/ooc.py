"""Out-of-core planning for one large solve (n beyond what HBM holds).

At n = 1e5, the size the paper's Section 4 names for real exciton problems,
one complex128 n x n matrix is 160 GB: A and B alone exceed a GB300's HBM
(~280 GB usable) once the Cholesky factor and the congruence product are
added, so the matrices live in host memory (Grace LPDDR5X, reached over
NVLink-C2C) and move to the GPU tile by tile.  This module plans that
movement for the BLAS3 stages of Alg. 2 -- the tiled Cholesky factorisation
of A - B and the congruence M = L^H (A + B) L -- under a device-memory
budget, and checks a plan by executing it on the CPU with numpy tiles.

Model
  * Matrices are split into nb x nb tiles; Hermitian matrices keep their
    lower tiles only.  A tile is named (matrix, i, j).
  * ``cholesky_tasks`` and ``congruence_tasks`` list the tile tasks in the
    order of the right-looking tile algorithms (every task reads and writes
    whole tiles; a task's inputs and outputs must be resident on the device).
  * ``plan`` turns a task list into device operations -- LOAD (host to
    device), ALLOC (a new zero tile, no transfer), COMPUTE, STORE (device to
    host, only for tiles modified since their load), FREE -- keeping at most
    ``budget`` tiles resident.  The victim of an eviction is the resident tile
    whose next use lies farthest in the future (Belady's rule; the task list
    is known in advance), so the plan's transfer volume is the minimum for
    that task order and budget.
  * ``simulate`` executes a plan with numpy tiles, asserting residency and
    the budget at every step; ``estimate`` converts a plan into transfer
    bytes and a time bound from a copy bandwidth and a compute rate.

The Householder reduction of M is not a tile algorithm in its one-stage form
(every column needs a matrix-vector product with the whole trailing matrix);
out of core it needs the two-stage reduction (band reduction in tiles, then
bulge chasing on the band, which fits in HBM), which the library does not
have.  This module covers the stages that are tile algorithms already.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

Tile = tuple  # (matrix name, i, j)


@dataclass
class Task:
    kind: str              # POTRF, TRSM, HERK, GEMM, ...
    reads: tuple           # tiles read (not modified)
    writes: tuple          # tiles modified (read and written, or created when `fresh`)
    flops: float           # real flops
    fresh: tuple = ()      # tiles of `writes` that the task creates (start at zero)
    args: dict = field(default_factory=dict)


def _herk_flops(nb):
    return 4.0 * nb ** 3  # complex nb x nb x nb, half the output (x 8 / 2)


def _gemm_flops(nb):
    return 8.0 * nb ** 3


def cholesky_tasks(nt: int, nb: int, mat: str = "L") -> list:
    """Right-looking tile Cholesky of the Hermitian matrix `mat` (lower tiles),
    in place: L L^H = mat (Alg. 2 step 1 at tile granularity)."""
    tasks = []
    for k in range(nt):
        tasks.append(Task("POTRF", (), ((mat, k, k),), 8.0 * nb ** 3 / 6.0, args={"k": k}))
        for i in range(k + 1, nt):
            tasks.append(Task("TRSM", ((mat, k, k),), ((mat, i, k),), 4.0 * nb ** 3, args={"i": i, "k": k}))
        for i in range(k + 1, nt):
            tasks.append(Task("HERK", ((mat, i, k),), ((mat, i, i),), _herk_flops(nb), args={"i": i, "k": k}))
            for j in range(k + 1, i):
                tasks.append(Task("GEMM", ((mat, i, k), (mat, j, k)), ((mat, i, j),), _gemm_flops(nb),
                                  args={"i": i, "j": j, "k": k}))
    return tasks


def congruence_tasks(nt: int, nb: int, m1: str = "M1", fac: str = "L", w: str = "W", out: str = "M") -> list:
    """W = M1 L (M1 Hermitian, lower tiles; L lower triangular), then the lower
    tiles of M = L^H W (Alg. 2 step 2 at tile granularity)."""
    tasks = []
    for j in range(nt):
        for i in range(nt):
            for k in range(j, nt):  # L(k, j) = 0 for k < j
                a = (m1, i, k) if i >= k else (m1, k, i)  # the stored lower tile, transposed when i < k
                tasks.append(Task("WGEMM", (a, (fac, k, j)), ((w, i, j),), _gemm_flops(nb),
                                  fresh=((w, i, j),) if k == j else (), args={"i": i, "j": j, "k": k}))
    for j in range(nt):
        for i in range(j, nt):
            for k in range(i, nt):  # L(k, i) = 0 for k < i
                tasks.append(Task("MGEMM", ((fac, k, i), (w, k, j)), ((out, i, j),), _gemm_flops(nb),
                                  fresh=((out, i, j),) if k == i else (), args={"i": i, "j": j, "k": k}))
    return tasks


@dataclass
class Op:
    kind: str      # LOAD, ALLOC, COMPUTE, STORE, FREE
    tile: Tile = None
    task: int = -1


def plan(tasks: list, budget: int, keep: set | None = None) -> list:
    """Device operations executing `tasks` with at most `budget` resident tiles.
    Tiles in `keep` (results) are stored to the host at the end when dirty."""
    need = max(len(set(t.reads) | set(t.writes)) for t in tasks)
    if budget < need:
        raise ValueError(f"budget {budget} tiles is below the {need} one task needs")
    uses = {}
    for idx, t in enumerate(tasks):
        for tile in set(t.reads) | set(t.writes):
            uses.setdefault(tile, []).append(idx)
    ptr = {tile: 0 for tile in uses}
    resident, dirty, on_host = set(), set(), set()
    created = {tile for t in tasks for tile in t.fresh}  # every other tile starts on the host
    ops = []

    def next_use(tile, now):
        lst = uses[tile]
        p = ptr[tile]
        while p < len(lst) and lst[p] < now:
            p += 1
        ptr[tile] = p
        return lst[p] if p < len(lst) else float("inf")

    def evict(now, protect):
        victim = max((x for x in resident if x not in protect), key=lambda x: next_use(x, now))
        if victim in dirty:
            ops.append(Op("STORE", victim))
            dirty.discard(victim)
            on_host.add(victim)
        ops.append(Op("FREE", victim))
        resident.discard(victim)

    for idx, t in enumerate(tasks):
        want = list(dict.fromkeys(t.reads + t.writes))
        protect = set(want)
        for tile in want:
            if tile in resident:
                continue
            while len(resident) >= budget:
                evict(idx, protect)
            if tile in t.fresh and tile not in on_host:
                ops.append(Op("ALLOC", tile))
            elif tile in created and tile not in on_host:
                raise ValueError(f"task {idx} reads {tile} before it is created")
            else:
                ops.append(Op("LOAD", tile))
            resident.add(tile)
        ops.append(Op("COMPUTE", task=idx))
        dirty.update(t.writes)
        # tiles with no further use leave at once (results go back to the host)
        for tile in want:
            if next_use(tile, idx + 1) == float("inf"):
                if tile in dirty and (keep is None or tile[0] in keep):
                    ops.append(Op("STORE", tile))
                    on_host.add(tile)
                dirty.discard(tile)
                ops.append(Op("FREE", tile))
                resident.discard(tile)
    for tile in sorted(resident):
        if tile in dirty and (keep is None or tile[0] in keep):
            ops.append(Op("STORE", tile))
        ops.append(Op("FREE", tile))
    return ops


def _run_task(t: Task, dev: dict):
    a = t.args
    if t.kind == "POTRF":
        (tile,) = t.writes
        dev[tile] = np.linalg.cholesky(np.tril(dev[tile]) + np.tril(dev[tile], -1).conj().T)
    elif t.kind == "TRSM":
        (lkk,), (tile,) = t.reads, t.writes
        dev[tile] = np.linalg.solve(dev[lkk].conj(), dev[tile].T).T  # X L^H = A  <=>  conj(L) X^T = A^T
    elif t.kind == "HERK":
        (aik,), (tile,) = t.reads, t.writes
        dev[tile] = dev[tile] - np.tril(dev[aik] @ dev[aik].conj().T)
    elif t.kind == "GEMM":
        (aik, ajk), (tile,) = t.reads, t.writes
        dev[tile] = dev[tile] - dev[aik] @ dev[ajk].conj().T
    elif t.kind == "WGEMM":
        (m1, lkj), (tile,) = t.reads, t.writes
        i, k = a["i"], a["k"]
        blk = dev[m1]
        if i == k:
            blk = np.tril(blk) + np.tril(blk, -1).conj().T
        elif i < k:
            blk = blk.conj().T
        dev[tile] = dev[tile] + blk @ dev[lkj]
    elif t.kind == "MGEMM":
        (lki, wkj), (tile,) = t.reads, t.writes
        dev[tile] = dev[tile] + dev[lki].conj().T @ dev[wkj]
    else:
        raise ValueError(t.kind)


def simulate(tasks: list, ops: list, host: dict, budget: int, nb: int) -> dict:
    """Execute `ops` with numpy tiles: `host` maps tiles to arrays (updated in
    place by STOREs).  Asserts that every task finds its tiles resident and
    that at most `budget` tiles are resident.  Returns transfer statistics."""
    dev = {}
    stats = {"load": 0, "store": 0, "alloc": 0, "peak": 0}
    for op in ops:
        if op.kind == "LOAD":
            assert op.tile not in dev
            dev[op.tile] = host[op.tile].copy()
            stats["load"] += 1
        elif op.kind == "ALLOC":
            assert op.tile not in dev
            dev[op.tile] = np.zeros((nb, nb), dtype=np.complex128)
            stats["alloc"] += 1
        elif op.kind == "STORE":
            host[op.tile] = dev[op.tile].copy()
            stats["store"] += 1
        elif op.kind == "FREE":
            del dev[op.tile]
        elif op.kind == "COMPUTE":
            t = tasks[op.task]
            for tile in t.reads + t.writes:
                assert tile in dev, (t.kind, tile)
            _run_task(t, dev)
        stats["peak"] = max(stats["peak"], len(dev))
        assert len(dev) <= budget
    assert not dev, "tiles left on the device"
    return stats


def estimate(tasks: list, ops: list, nb: int, copy_gbs: float = 900.0, tflops: float = 1.19) -> dict:
    """Transfer bytes and a time bound of a plan: copies at `copy_gbs` (one
    direction of NVLink-C2C) and compute at `tflops` (the FP64 engine's
    measured rate); with the copies of the next tiles overlapped with the
    current task, the time is at least the larger of the two sums."""
    tile_bytes = 16.0 * nb * nb
    nload = sum(1 for o in ops if o.kind == "LOAD")
    nstore = sum(1 for o in ops if o.kind == "STORE")
    flops = sum(t.flops for t in tasks)
    t_copy = (nload + nstore) * tile_bytes / (copy_gbs * 1e9)
    t_comp = flops / (tflops * 1e12)
    return {"tile_bytes": tile_bytes, "loads": nload, "stores": nstore,
            "bytes_moved": (nload + nstore) * tile_bytes, "flops": flops,
            "copy_s": t_copy, "compute_s": t_comp, "time_lower_bound_s": max(t_copy, t_comp),
            "compute_bound": t_comp >= t_copy}


def tiles_of(M: np.ndarray, nb: int, name: str, lower: bool = True) -> dict:
    nt = M.shape[0] // nb
    out = {}
    for i in range(nt):
        for j in range(nt):
            if lower and j > i:
                continue
            out[(name, i, j)] = np.array(M[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb], dtype=np.complex128)
    return out


def assemble(host: dict, name: str, nt: int, nb: int, lower: bool = True) -> np.ndarray:
    M = np.zeros((nt * nb, nt * nb), dtype=np.complex128)
    for i in range(nt):
        for j in range(nt):
            if lower and j > i:
                continue
            M[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb] = host[(name, i, j)]
    return M
