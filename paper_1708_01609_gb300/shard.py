"""Multi-rank host logic: bank shards, tail gathering, per-lag maxima
merged across shards, failed-rank re-queue.

Every (segment, template) correlation is independent (the paper's partition
of the bank into groups W_alpha and the data into blocks Y_beta, Sec. 3.1),
so N ranks split a bank into contiguous row ranges, search their own range
with no collective on the data path, and rank 0 concatenates the tails.  If
a rank fails, the ranges it had not finished are re-queued to the ranks that
are still alive.  The compute step is a callable, so the same logic drives
GPU ranks (``LibbegeShard``: libbege on the rank's own device, holding only
the rank's own rows of the bank) and CPU ranks in tests.
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


def deal(pending: list, alive: list[int]) -> dict:
    """Deal the pending chunks (in row order) to the live ranks as
    contiguous runs whose lengths differ by at most one, so that in the
    first round each rank gets one contiguous range of the bank."""
    return {r: pending[a:b]
            for r, (a, b) in zip(alive, shard_ranges(len(pending), len(alive)))}


def first_range(count: int, chunk: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [begin, end) that ``run_sharded`` deals to ``rank`` in its first
    round (all ranks alive): the rank's resident shard of the bank."""
    pending = [(k, min(k + chunk, count)) for k in range(0, count, chunk)]
    mine = deal(pending, list(range(world)))[rank]
    return (mine[0][0], mine[-1][1]) if mine else (0, 0)


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
    dealt as contiguous runs (``deal``); after every round the ranks
    exchange (on the host, via all_gather_object) which chunks they
    finished.  A rank that raises
    is treated as failed: it reports no more progress, and its unfinished
    chunks are dealt again to the survivors.  ``fail_rank`` / ``fail_after``
    make that rank fail after that many chunks (fault injection for tests).
    In the first round rank r gets the contiguous rows ``first_range``
    gives; re-dealt chunks go to the survivors as contiguous runs too.
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
        assign = deal(pending, alive)
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


class LibbegeShard:
    """The compute step of ``run_sharded`` on a GPU rank: libbege searches
    of one segment against rows [k0, k1) of a chirp bank.

    The rank defines only its own rows ``own`` = [b0, b1) of the bank on the
    device (its shard, resident for the whole search); a chunk outside them
    -- one re-dealt from a failed rank -- is defined for that chunk alone and
    released after it.  Every row runs the same kernels whatever bank it
    sits in, so the gathered tails, sigma and per-lag maxima equal a
    single-process search of the whole bank bitwise.  Records and
    projections carry bank-wide template indices.

    ctx: a binding.Context; seg: its segment handle; params: (K, 2) array of
    (f0, fdot) for the whole bank; project: also return each chunk's per-lag
    maximum (bege_correlate_max / bege_fetch_max).  A chunk whose tails
    overflow the context's tail capacity raises RuntimeError (so
    ``run_sharded`` treats the rank as failed rather than lose records).
    """

    def __init__(self, ctx, seg: int, n: int, params: np.ndarray, own: tuple[int, int],
                 kappa: float, tau: float = 1.0, taper_frac: float = 0.05,
                 project: bool = False, stream: int = 0):
        self.ctx, self.seg, self.n = ctx, seg, n
        self.params, self.kappa = np.asarray(params, dtype=np.float64), kappa
        self.tau, self.taper, self.project, self.stream = tau, taper_frac, project, stream
        self.own = own
        self.bank = None
        if own[1] > own[0]:
            self.bank = ctx.bege_define_bank(self.params[own[0]:own[1]], tau=tau,
                                             taper_frac=taper_frac, stream=stream)
        self.sigma = {}   # chunk (k0, k1) -> sigma of its rows

    def __call__(self, k0: int, k1: int):
        ctx = self.ctx
        if self.bank is not None and self.own[0] <= k0 and k1 <= self.own[1]:
            bank, base, temp = self.bank, self.own[0], False
        else:
            bank = ctx.bege_define_bank(self.params[k0:k1], tau=self.tau,
                                        taper_frac=self.taper, stream=self.stream)
            base, temp = k0, True
        try:
            if self.project:
                job = ctx.bege_correlate_max(self.seg, bank, k0 - base, k1 - base, self.kappa,
                                             self.stream)
            else:
                job = ctx.bege_correlate(self.seg, bank, k0 - base, k1 - base, self.kappa,
                                         self.stream)
            recs, total = ctx.bege_fetch_tails(job)
            if total != len(recs):
                ctx.bege_release(job)
                raise RuntimeError(f"rows [{k0}, {k1}): {total} tails overflow the capacity")
            recs = recs.copy()
            recs["tmpl"] += np.uint32(base)
            self.sigma[(k0, k1)] = ctx.bege_get_sigma(job, k1 - k0)
            proj = None
            if self.project:
                snr, tmpl = ctx.bege_fetch_max(job, self.n)
                tmpl = np.where(tmpl >= 0, tmpl + base, -1).astype(np.int32)
                proj = (snr, tmpl)
            ctx.bege_release(job)
        finally:
            if temp:
                ctx.bege_release(bank)
        return recs if proj is None else (recs, proj)
