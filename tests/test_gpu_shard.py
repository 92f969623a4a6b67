"""The bank-sharded search through libbege (the paper's partition of the
bank into independent groups, Sec. 3.1): two gloo ranks, each with its own
context on the same GPU and only its own half of a 2^16-chirp bank resident,
search one N = 2^16 segment with ``shard.run_sharded`` and ``LibbegeShard``.
The gathered tails, the sigma of every row and the merged per-lag maximum
equal a single-process search of the whole bank bitwise, also when rank 1
fails after its first chunk and rank 0 takes over its remaining chunks
(defining those rows on demand).  The ranks exchange only host data; their
kernels never wait on each other."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

KAPPA = 5.5
CHUNK = 8192


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def problem():
    import synthetic as S
    params = S.grid_paper(64, 1024)                  # 65536 in-band chirps
    seg = S.make_segment(1 << 16, params, 8, 4711)
    return seg, params


def worker(rank, world, port, fail_rank, out_dir):
    import torch.distributed as dist

    from paper_1708_01609_gb300 import binding, build, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    build()
    seg_data, params = problem()
    ctx = binding.Context(0, tail_capacity=1 << 22)
    seg = ctx.bege_load_segment(seg_data.y)
    own = shard.first_range(len(params), CHUNK, world, rank)
    comp = shard.LibbegeShard(ctx, seg, seg_data.n, params, own, KAPPA, project=True)
    resident = ctx.bege_device_bytes()
    tails, failed, (snr, tmpl) = shard.run_sharded(dist, comp, len(params), CHUNK,
                                                   fail_rank=fail_rank, fail_after=1)
    sigmas = [None] * world
    dist.all_gather_object(sigmas, comp.sigma)
    owns = [None] * world
    dist.all_gather_object(owns, (own, resident))
    if rank == 0:
        sig = np.full(len(params), np.nan, np.float32)
        for part in sigmas:
            for (k0, k1), v in part.items():
                sig[k0:k1] = v
        np.save(os.path.join(out_dir, "tails.npy"), tails)
        np.save(os.path.join(out_dir, "sigma.npy"), sig)
        np.save(os.path.join(out_dir, "proj.npy"), np.stack([snr.view(np.int32), tmpl]))
        np.save(os.path.join(out_dir, "meta.npy"),
                np.array([len(failed)] + [x for (a, b), r in owns for x in (a, b, r)],
                         np.int64))
    ctx.close()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("fail_rank", [None, 1], ids=["clean", "rank1_fails"])
def test_sharded_search_equals_single_process(tmp_path, fail_rank):
    from gpu_helpers import make_ctx
    world = 2
    mp.start_processes(worker, args=(world, free_port(), fail_rank, str(tmp_path)),
                       nprocs=world, start_method="spawn")
    tails = np.load(tmp_path / "tails.npy")
    sig = np.load(tmp_path / "sigma.npy")
    proj = np.load(tmp_path / "proj.npy")
    meta = np.load(tmp_path / "meta.npy")
    seg_data, params = problem()
    count = len(params)
    # each rank held only its own half of the bank
    assert meta[0] == (0 if fail_rank is None else 1)
    assert (meta[1], meta[2]) == (0, count // 2) and (meta[4], meta[5]) == (count // 2, count)
    bank_bytes = (count // 2) * 4096 * 4
    assert bank_bytes <= meta[3] < 2 * bank_bytes and bank_bytes <= meta[6] < 2 * bank_bytes
    # the single-process search of the whole bank
    ctx = make_ctx(tail_capacity=1 << 24)
    seg = ctx.bege_load_segment(seg_data.y)
    bid = ctx.bege_define_bank(params)
    job = ctx.bege_correlate_max(seg, bid, 0, count, KAPPA)
    ref, total = ctx.bege_fetch_tails(job, sort=True)
    ref_sig = ctx.bege_get_sigma(job, count)
    snr, tmpl = ctx.bege_fetch_max(job, seg_data.n)
    ctx.close()
    assert total == len(ref) > 1000
    assert np.array_equal(tails, ref)
    assert np.array_equal(sig.view(np.uint32), ref_sig.view(np.uint32))
    assert np.array_equal(proj[0], snr.view(np.int32)) and np.array_equal(proj[1], tmpl)
    got = set(zip(tails["tmpl"].tolist(), tails["lag"].tolist()))
    assert all((k, lag) in got for k, lag, _ in seg_data.injections)
