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
