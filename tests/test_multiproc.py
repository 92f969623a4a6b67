"""Multi-rank path on CPU: world_size-2 gloo ranks shard a bank, search their
ranges with the oracle as the compute step, and rank 0 gathers the tails;
a rank that fails part-way has its unfinished ranges re-queued.  Also the
max-over-ranks timing rule of bench.py."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1708_01609_gb300 import shard


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def small_problem():
    import oracle as O
    import synthetic as S
    y = S.band_limited_noise(2048, 3)
    bank = S.random_samples_bank(23, 300, 4).astype(np.float64)
    return y, bank, O


def worker(rank, world, port, fail_rank, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    y, bank, O = small_problem()

    def compute(k0, k1):
        t = O.search(y, bank[k0:k1], 3.0, k0=k0)["tails"]
        out = np.empty(len(t), dtype=[("tmpl", np.uint32), ("lag", np.uint32),
                                      ("value", np.float32)])
        out["tmpl"], out["lag"], out["value"] = t["tmpl"], t["lag"], t["value"]
        return out

    tails, failed = shard.run_sharded(dist, compute, len(bank), 4, fail_rank=fail_rank,
                                      fail_after=1)
    # the timing rule of bench.py: every rank's time, the max reported
    import torch
    t = torch.tensor([10.0 + rank])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        np.save(os.path.join(out_dir, "tails.npy"), tails)
        np.save(os.path.join(out_dir, "meta.npy"), np.array([t.item(), len(failed)]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("fail_rank", [None, 1])
def test_two_gloo_ranks_shard_and_gather(tmp_path, fail_rank):
    world = 2
    mp.start_processes(worker, args=(world, free_port(), fail_rank, str(tmp_path)),
                       nprocs=world, start_method="spawn")
    tails = np.load(tmp_path / "tails.npy")
    tmax, nfailed = np.load(tmp_path / "meta.npy")
    y, bank, O = small_problem()
    ref = O.search(y, bank, 3.0)["tails"]
    assert tails["tmpl"].tolist() == ref["tmpl"].tolist()
    assert tails["lag"].tolist() == ref["lag"].tolist()
    assert np.allclose(tails["value"], ref["value"], rtol=1e-6)
    assert tmax == 11.0
    assert nfailed == (0 if fail_rank is None else 1)


def test_shard_ranges_cover_bank():
    for count in [0, 1, 7, 1 << 20]:
        for world in [1, 2, 3, 8]:
            r = shard.shard_ranges(count, world)
            assert r[0][0] == 0 and r[-1][1] == count
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            sizes = [b - a for a, b in r]
            assert max(sizes) - min(sizes) <= 1


def projection_worker(rank, world, port, out_dir):
    """Each rank projects its own shard of the bank (the oracle's per-lag
    maximum, Eq. Ak over rows [k0, k1)); the shards meet in one host
    all_reduce(MAX) of the packed keys."""
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    y, bank, O = small_problem()
    k0, k1 = shard.shard_ranges(len(bank), world)[rank]
    rho = np.stack([O.correlate_fft(w, y) for w in bank[k0:k1]])
    sig = np.array([O.sigma_rms(r) for r in rho])
    snr, tmpl = O.max_projection(rho, sig, 2.5, k0=k0)
    m_snr, m_tmpl = shard.all_reduce_projection(dist, snr, tmpl)
    if rank == 0:
        np.save(os.path.join(out_dir, "proj.npy"), np.stack([m_snr, m_tmpl.astype(np.float32)]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_merge_projections(tmp_path):
    world = 2
    mp.start_processes(projection_worker, args=(world, free_port(), str(tmp_path)),
                       nprocs=world, start_method="spawn")
    m_snr, m_tmpl = np.load(tmp_path / "proj.npy")
    y, bank, O = small_problem()
    rho = np.stack([O.correlate_fft(w, y) for w in bank])
    sig = np.array([O.sigma_rms(r) for r in rho])
    snr, tmpl = O.max_projection(rho, sig, 2.5)
    assert np.sum(tmpl >= 0) > 20 and len(np.unique(tmpl[tmpl >= 0])) > 1
    assert np.array_equal(m_tmpl.astype(np.int32), tmpl)
    assert np.array_equal(m_snr, snr.astype(np.float32))


def test_merge_projections_keeps_max_and_smaller_template_on_ties():
    a_snr = np.array([0.0, 5.0, 6.0, 7.0], np.float32)
    a_tm = np.array([-1, 3, 4, 9], np.int32)
    b_snr = np.array([5.5, 0.0, 6.5, 7.0], np.float32)
    b_tm = np.array([12, -1, 20, 2], np.int32)
    snr, tm = shard.merge_projections([(a_snr, a_tm), (b_snr, b_tm)])
    assert snr.tolist() == [5.5, 5.0, 6.5, 7.0]
    assert tm.tolist() == [12, 3, 20, 2]
    s1, t1 = shard.merge_projections([(a_snr, a_tm)])
    assert np.array_equal(s1, a_snr) and np.array_equal(t1, a_tm)
    with pytest.raises(ValueError):
        shard.merge_projections([(np.array([-1.0], np.float32), np.array([0], np.int32))])


def sharded_max_worker(rank, world, port, fail_rank, out_dir):
    """run_sharded with per-chunk projections: chunks of the bank searched
    by the oracle (tails and the per-lag maximum of the chunk's rows), a
    rank failing after one chunk, the projection merged over every chunk."""
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    y, bank, O = small_problem()

    def compute(k0, k1):
        res = O.search(y, bank[k0:k1], 2.5, k0=k0, return_rho=True)
        t = res["tails"]
        out = np.empty(len(t), dtype=[("tmpl", np.uint32), ("lag", np.uint32),
                                      ("value", np.float32)])
        out["tmpl"], out["lag"], out["value"] = t["tmpl"], t["lag"], t["value"]
        return out, O.max_projection(res["rho"], res["sigma"], 2.5, k0=k0)

    tails, failed, (snr, tmpl) = shard.run_sharded(dist, compute, len(bank), 3,
                                                   fail_rank=fail_rank, fail_after=1)
    if rank == 0:
        np.save(os.path.join(out_dir, "proj2.npy"), np.stack([snr, tmpl.astype(np.float32)]))
        np.save(os.path.join(out_dir, "meta2.npy"), np.array([len(tails), len(failed)]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("fail_rank", [None, 1])
def test_sharded_search_merges_projections(tmp_path, fail_rank):
    world = 2
    mp.start_processes(sharded_max_worker, args=(world, free_port(), fail_rank, str(tmp_path)),
                       nprocs=world, start_method="spawn")
    m_snr, m_tmpl = np.load(tmp_path / "proj2.npy")
    n_tails, n_failed = np.load(tmp_path / "meta2.npy")
    y, bank, O = small_problem()
    res = O.search(y, bank, 2.5, return_rho=True)
    snr, tmpl = O.max_projection(res["rho"], res["sigma"], 2.5)
    assert np.sum(tmpl >= 0) > 20
    assert np.array_equal(m_tmpl.astype(np.int32), tmpl)
    assert np.array_equal(m_snr, snr.astype(np.float32))
    assert n_tails == len(res["tails"])
    assert n_failed == (0 if fail_rank is None else 1)


def test_deal_gives_contiguous_runs():
    pending = [(k, min(k + 3, 20)) for k in range(0, 20, 3)]   # 7 chunks
    a = shard.deal(pending, [0, 1])
    assert a[0] == pending[:4] and a[1] == pending[4:]
    b = shard.deal(pending[2:], [1])
    assert b[1] == pending[2:]
    assert shard.first_range(20, 3, 2, 0) == (0, 12)
    assert shard.first_range(20, 3, 2, 1) == (12, 20)
    assert shard.first_range(2, 3, 2, 1) == (0, 0)
    # every row is dealt exactly once
    for count, chunk, world in [(65536, 8192, 2), (1000, 7, 3), (5, 10, 4)]:
        got = [shard.first_range(count, chunk, world, r) for r in range(world)]
        cover = sorted(x for x in got if x[1] > x[0])
        assert cover[0][0] == 0 and cover[-1][1] == count
        assert all(p[1] == q[0] for p, q in zip(cover, cover[1:]))
