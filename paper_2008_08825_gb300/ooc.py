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

``run_device`` executes a plan on the GPU through the library's tile
executor (bse_ooc_run): copies on a copy stream, tile tasks on the FP64 GEMM
engine and the blocked Cholesky, the two overlapped through per-slot events.
``alg2_stage_tasks`` lists the whole BLAS3 part of Alg. 2 (forming A - B and
A + B from tiles of A and B, the Cholesky factorisation and the congruence).

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


def form_tasks(nt: int, a: str = "A", b: str = "B", plus: str = "M1", minus: str = "L") -> list:
    """Lower tiles of A + B and A - B from the lower tiles of A and B (the
    sums of Alg. 2 before step 1); the outputs are created by the tasks."""
    tasks = []
    for j in range(nt):
        for i in range(j, nt):
            for kind, out in (("FORM_SUM", plus), ("FORM_DIFF", minus)):
                tasks.append(Task(kind, ((a, i, j), (b, i, j)), ((out, i, j),), 0.0, fresh=((out, i, j),),
                                  args={"i": i, "j": j}))
    return tasks


def alg2_stage_tasks(nt: int, nb: int) -> list:
    """Alg. 2's tile stages in order: M1 = A + B and L := A - B (lower
    tiles), L L^H = A - B in place, W = M1 L, M = L^H W (lower tiles)."""
    return form_tasks(nt) + cholesky_tasks(nt, nb, "L") + congruence_tasks(nt, nb, m1="M1", fac="L", w="W", out="M")


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
                # L(j, j) is lower triangular: half the multiply-adds
                tasks.append(Task("WGEMM", (a, (fac, k, j)), ((w, i, j),), _gemm_flops(nb) / (2 if k == j else 1),
                                  fresh=((w, i, j),) if k == j else (), args={"i": i, "j": j, "k": k}))
    for j in range(nt):
        for i in range(j, nt):
            for k in range(i, nt):  # L(k, i) = 0 for k < i
                tasks.append(Task("MGEMM", ((fac, k, i), (w, k, j)), ((out, i, j),),
                                  _gemm_flops(nb) / (2 if k == i else 1),
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
    if t.kind in ("FORM_SUM", "FORM_DIFF"):
        (x, y), (tile,) = t.reads, t.writes
        dev[tile] = dev[x] + dev[y] if t.kind == "FORM_SUM" else dev[x] - dev[y]
    elif t.kind == "POTRF":
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


# ---------------------------------------------------------------------------
# GPU execution through the library's tile executor

OP_KINDS = {"LOAD": 0, "ALLOC": 1, "COMPUTE": 2, "STORE": 3, "FREE": 4}
TASK_KINDS = {"FORM_SUM": 0, "FORM_DIFF": 1, "POTRF": 2, "TRSM": 3, "HERK": 4, "GEMM": 5, "WGEMM": 6, "MGEMM": 6}
IN0_CONJT, IN0_HERM, IN0_LOWER, IN1_LOWER = 1, 2, 4, 8


def encode(tasks: list, ops: list):
    """Tile names, executor tasks (kind, out, in0, in1, flags) and executor
    ops (kind, arg) for a task list and its plan."""
    names = []
    index = {}

    def tid(tile):
        if tile not in index:
            index[tile] = len(names)
            names.append(tile)
        return index[tile]

    enc = []
    for t in tasks:
        a = t.args
        flags = 0
        ins = list(t.reads)
        if t.kind == "POTRF":
            flags = a["k"] << 8
        elif t.kind == "WGEMM":  # W(i, j) += op(M1 tile) L(k, j)
            i, j, k = a["i"], a["j"], a["k"]
            flags = IN0_HERM if i == k else (IN0_CONJT if i < k else 0)
            if k == j:
                flags |= IN1_LOWER
        elif t.kind == "MGEMM":  # M(i, j) += L(k, i)^H W(k, j)
            flags = IN0_CONJT | (IN0_LOWER if a["k"] == a["i"] else 0)
        elif t.kind == "TRSM":
            ins = [t.reads[0]]
        (out,) = t.writes
        in0 = tid(ins[0]) if len(ins) > 0 else -1
        in1 = tid(ins[1]) if len(ins) > 1 else -1
        enc.append((TASK_KINDS[t.kind], tid(out), in0, in1, flags))
    eops = []
    for op in ops:
        if op.kind == "COMPUTE":
            eops.append((OP_KINDS["COMPUTE"], op.task))
        else:
            eops.append((OP_KINDS[op.kind], tid(op.tile)))
    return names, enc, eops


class DevicePlan:
    """The BLAS3 stages of Alg. 2 planned for the GPU executor: A and B (n x n
    Hermitian, lower triangles read, n a multiple of nb) in host tiles, at
    most `budget` device tiles.  run() executes the plan (repeatable: the
    input tiles are only read, every other tile is recreated); results()
    gives L (L L^H = A - B) and M = L^H (A + B) L as dense lower triangles."""

    def __init__(self, A: np.ndarray, B: np.ndarray, nb: int, budget: int, pinned: bool = True):
        import torch

        n = A.shape[0]
        if n % nb:
            raise ValueError("n must be a multiple of nb")
        self.n, self.nb, self.nt, self.budget = n, nb, n // nb, budget
        self.tasks = alg2_stage_tasks(self.nt, nb)
        self.ops = plan(self.tasks, budget, keep={"L", "M"})
        self.names, self.enc, self.eops = encode(self.tasks, self.ops)
        self.host = []
        for name, i, j in self.names:
            t = torch.empty((nb, nb), dtype=torch.complex128, pin_memory=pinned)
            if name in ("A", "B"):
                src = A if name == "A" else B
                # column-major tile: the row-major tensor holds the tile's transpose
                t.copy_(torch.from_numpy(np.ascontiguousarray(src[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb].T)))
            self.host.append(t)
        est = estimate(self.tasks, self.ops, nb)
        self.stats = {"loads": est["loads"], "stores": est["stores"], "tiles": len(self.names),
                      "bytes_moved": est["bytes_moved"], "flops": est["flops"]}

    def run(self, handle=None, stream=None) -> None:
        from . import bse

        bse.ooc_run(self.nb, self.host, self.eops, self.enc, self.budget, handle=handle, stream=stream)

    def results(self):
        n, nb, nt = self.n, self.nb, self.nt
        index = {name: q for q, name in enumerate(self.names)}
        out = []
        for mat in ("L", "M"):
            Mx = np.zeros((n, n), dtype=np.complex128)
            for i in range(nt):
                for j in range(i + 1):
                    Mx[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb] = self.host[index[(mat, i, j)]].numpy().T
            out.append(np.tril(Mx))
        return out[0], out[1]


def run_device(A: np.ndarray, B: np.ndarray, nb: int, budget: int, handle=None, pinned: bool = True):
    """One GPU execution of the BLAS3 stages of Alg. 2 out of core (see
    DevicePlan): returns (L, M, statistics of the plan)."""
    p = DevicePlan(A, B, nb, budget, pinned)
    p.run(handle)
    L, M = p.results()
    return L, M, p.stats
