"""Multi-rank host logic: bank shards, tail gathering, per-lag maxima
merged across shards, failed-rank re-queue.

Every (segment, template) correlation is independent (the paper's partition
of the bank into groups W_alpha and the data into blocks Y_beta, Sec. 3.1),
so N ranks split a bank into contiguous row ranges, search their own range
with no collective on the data path, and rank 0 concatenates the tails.  If
a rank fails, the ranges it had not finished are re-queued to the ranks that
are still alive.  The compute step is a callable, so the same logic drives
GPU ranks (libbege) and CPU ranks in tests.
"""
from __future__ import annotations

import numpy as np


def shard_ranges(count: int, world: int) -> list[tuple[int, int]]:
    """Contiguous [begin, end) row ranges, sizes differing by at most one."""
    if world < 1:
        raise ValueError("world must be >= 1")
    base, extra = divmod(count, world)
    out, k = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((k, k + n))
        k += n
    return out


def merge_tails(parts: list[np.ndarray]) -> np.ndarray:
    """Concatenate per-rank tail records and order them by (tmpl, lag)."""
    parts = [p for p in parts if p is not None and len(p)]
    if not parts:
        return np.empty(0, dtype=[("tmpl", np.uint32), ("lag", np.uint32), ("value", np.float32)])
    t = np.concatenate(parts)
    return np.sort(t, order=["tmpl", "lag"])


def projection_key(snr: np.ndarray, tmpl: np.ndarray) -> np.ndarray:
    """Per-lag maximum (Eq. Ak over a shard of the bank) as one int64 key
    per lag, the device's ordering: (FP32 bits of rho/sigma) << 32 |
    ~template, 0 where no template hit.  The kept values are above kappa > 0,
    so their bits order like the values and stay below 2^63; equal values
    keep the smaller template."""
    snr = np.asarray(snr, dtype=np.float32)
    tmpl = np.asarray(tmpl, dtype=np.int32)
    hit = tmpl >= 0
    if np.any(snr[hit] <= 0):
        raise ValueError("a kept per-lag maximum must be positive")
    bits = snr.view(np.uint32).astype(np.int64)
    low = (~tmpl.astype(np.uint32)).astype(np.int64)
    return np.where(hit, (bits << 32) | low, 0)


def projection_from_key(key: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Inverse of projection_key: (snr FP32, template int32, -1 = no hit)."""
    key = np.asarray(key, dtype=np.int64)
    snr = (key >> 32).astype(np.uint32).view(np.float32).copy()
    tmpl = (~(key & 0xFFFFFFFF).astype(np.uint32)).astype(np.int32)
    none = key == 0
    snr[none], tmpl[none] = 0.0, -1
    return snr, tmpl


def merge_projections(parts: list[tuple[np.ndarray, np.ndarray]]):
    """Element-wise maximum of per-shard projections of one segment's N
    lags (the one exchange the per-lag maximum needs when the bank is
    split): the largest rho/sigma per lag over all shards, ties to the
    smaller template."""
    if not parts:
        raise ValueError("no projections to merge")
    key = projection_key(*parts[0])
    for p in parts[1:]:
        key = np.maximum(key, projection_key(*p))
    return projection_from_key(key)


def all_reduce_projection(dist, snr: np.ndarray, tmpl: np.ndarray):
    """merge_projections across the ranks of ``dist``: one all_reduce(MAX)
    of the N int64 keys in host memory (gloo), the result on every rank."""
    import torch
    key = torch.from_numpy(projection_key(snr, tmpl))
    dist.all_reduce(key, op=dist.ReduceOp.MAX)
    return projection_from_key(key.numpy())


def run_sharded(dist, compute, count: int, chunk: int, fail_rank: int | None = None,
                fail_after: int = 0):
    """Search rows [0, count) over all ranks of ``dist`` (an initialised
    torch.distributed module) in chunks of ``chunk`` rows.

    ``compute(k0, k1)`` returns this rank's tail records for rows [k0, k1),
    or a pair (records, (snr, tmpl)) with the chunk's per-lag maximum
    (Eq. Ak over those rows, as bege_fetch_max returns it).  Chunks are
    dealt round-robin; after every round the ranks exchange (on the host,
    via all_gather_object) which chunks they finished.  A rank that raises
    is treated as failed: it reports no more progress, and its unfinished
    chunks are dealt again to the survivors.  ``fail_rank`` / ``fail_after``
    make that rank fail after that many chunks (fault injection for tests).
    Returns the merged tails on rank 0 (None elsewhere) and the set of ranks
    that failed; with projections, also the merged per-lag maximum over the
    whole bank (every rank), from one all_reduce(MAX) of the packed keys.
    """
    rank, world = dist.get_rank(), dist.get_world_size()
    pending = [(k, min(k + chunk, count)) for k in range(0, count, chunk)]
    alive = list(range(world))
    failed: set[int] = set()
    mine: list[np.ndarray] = []
    proj_key = None  # this rank's per-lag maximum over its finished chunks
    done_here = 0
    dead = False
    while pending:
        # deal the pending chunks round-robin over the live ranks
        assign = {r: [] for r in alive}
        for i, c in enumerate(pending):
            assign[alive[i % len(alive)]].append(c)
        finished, crashed = [], False
        if not dead and rank in assign:
            for c in assign[rank]:
                try:
                    if fail_rank == rank and done_here >= fail_after:
                        raise RuntimeError(f"rank {rank} failed (injected)")
                    res = compute(*c)
                    if isinstance(res, tuple):
                        res, (snr, tmpl) = res
                        key = projection_key(snr, tmpl)
                        proj_key = key if proj_key is None else np.maximum(proj_key, key)
                    mine.append(res)
                    finished.append(c)
                    done_here += 1
                except RuntimeError:
                    crashed = dead = True
                    break
        reports = [None] * world
        dist.all_gather_object(reports, {"finished": finished, "crashed": crashed})
        for r, rep in enumerate(reports):
            if rep["crashed"]:
                failed.add(r)
        done = {c for rep in reports for c in rep["finished"]}
        pending = [c for c in pending if c not in done]
        alive = [r for r in alive if r not in failed]
        if not alive:
            raise RuntimeError("every rank failed")
    gathered = [None] * world
    dist.all_gather_object(gathered, merge_tails(mine))
    tails = merge_tails(gathered) if rank == 0 else None
    # projections: every rank learns the length, ranks without a finished
    # chunk contribute zeros (no hit), then one MAX reduction of the keys
    lengths = [None] * world
    dist.all_gather_object(lengths, None if proj_key is None else len(proj_key))
    n = max((x for x in lengths if x is not None), default=None)
    if n is None:
        return tails, failed
    import torch
    key = torch.from_numpy(proj_key if proj_key is not None else np.zeros(n, np.int64))
    dist.all_reduce(key, op=dist.ReduceOp.MAX)
    return tails, failed, projection_from_key(key.numpy())
