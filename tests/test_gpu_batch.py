"""Batching form: many segments of uneven length, each against its own bank
range, in one persistent launch inside a CUDA graph.  The batch must give
the same sigma and tails as the single-segment launches (same per-template
arithmetic), every plan must agree, and sampled templates must match the
oracle."""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_helpers import compare_tails, make_ctx, oracle_rho

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx(tail_capacity=1 << 22)
    yield c
    c.close()


@pytest.fixture(scope="module")
def small_batch(ctx):
    entries, grids = S.batch_case(seed=2, n_segments=10, n_inject=2, sub_bank=(40, 300),
                                  n_fdot=64, n_f0=64)
    banks = {tau: ctx.bege_define_bank(grids[tau], tau=tau, taper_frac=0.05) for tau in grids}
    spec = [(e.seg.y, banks[e.tau], e.k0, e.k1, 5.0) for e in entries]
    bid = ctx.bege_batch_create(spec)
    return entries, grids, banks, bid


def single_segment(ctx, e, bank, kappa=5.0):
    n = e.seg.n
    ctx.bege_set_config(n, 2, 256)
    seg = ctx.bege_load_segment(e.seg.y)
    job = ctx.bege_correlate(seg, bank, e.k0, e.k1, kappa)
    recs, total = ctx.bege_fetch_tails(job)
    sig = ctx.bege_get_sigma(job, e.k1 - e.k0)
    ctx.bege_release(job)
    ctx.bege_release(seg)
    return np.sort(recs, order=["tmpl", "lag"]), sig


def test_batch_matches_single_launches(ctx, small_batch):
    entries, grids, banks, bid = small_batch
    assert {e.seg.n for e in entries} >= {1 << 14, 1 << 17}
    for plan in (0, 1):
        ctx.bege_batch_set_plan(bid, plan, 64, 1)
        ctx.bege_batch_run(bid)
        for i, e in enumerate(entries):
            recs, total = ctx.bege_batch_fetch_tails(bid, i)
            assert total == len(recs)
            sig = ctx.bege_batch_get_sigma(bid, i, e.k1 - e.k0)
            ref_recs, ref_sig = single_segment(ctx, e, banks[e.tau])
            assert np.array_equal(sig, ref_sig), (plan, i)
            assert np.array_equal(np.sort(recs, order=["tmpl", "lag"]), ref_recs), (plan, i)


def test_batch_sampled_oracle(ctx, small_batch):
    entries, grids, banks, bid = small_batch
    ctx.bege_batch_set_plan(bid, 0, 128, 0)
    ctx.bege_batch_run(bid)
    for i, e in enumerate(entries[:4]):
        recs, _ = ctx.bege_batch_fetch_tails(bid, i)
        sig = ctx.bege_batch_get_sigma(bid, i, e.k1 - e.k0)
        rows = sorted({e.k0, e.k1 - 1} | {k for k, _, _ in e.seg.injections})
        length = int(round(e.tau * 4096))
        bank = O.chirp_bank(grids[e.tau][rows], 4096.0, length, 0.05)
        rho, osig = oracle_rho(e.seg.y, bank)
        assert np.all(np.abs(sig[np.array(rows) - e.k0] / osig - 1) <= 1e-6)
        compare_tails(recs, {k: (rho[j], osig[j]) for j, k in enumerate(rows)}, 5.0,
                      tmpl_subset=set(rows))
        keys = set(zip(recs["tmpl"].tolist(), recs["lag"].tolist()))
        for k, lag, _ in e.seg.injections:
            assert (k, lag) in keys


def test_batch_autotune_keeps_results(ctx, small_batch):
    entries, grids, banks, bid = small_batch
    ctx.bege_batch_set_plan(bid, 0, 256, 0)
    ctx.bege_batch_run(bid)
    before = [ctx.bege_batch_get_sigma(bid, i, e.k1 - e.k0) for i, e in enumerate(entries)]
    ms = ctx.bege_batch_autotune(bid, reps=1)
    assert ms > 0
    plan, chunk, order = ctx.bege_batch_get_plan(bid)
    assert plan in (0, 1) and chunk >= 1 and order in (0, 1)
    ctx.bege_batch_run(bid)
    assert ctx.bege_batch_elapsed_ms(bid) > 0
    for i, e in enumerate(entries):
        assert np.array_equal(ctx.bege_batch_get_sigma(bid, i, e.k1 - e.k0), before[i])


def test_batch_rejects_unsupported_entries(ctx):
    from paper_1708_01609_gb300.binding import BegeError
    bank = ctx.bege_define_bank(S.grid_small()[:4], tau=1.0)
    long_bank = ctx.bege_define_bank_samples(np.ones((2, 8192), np.float32))
    y = S.band_limited_noise(1 << 13, 1)
    with pytest.raises(BegeError):
        ctx.bege_batch_create([(y, bank, 0, 4, 5.0)])                 # N = 2^13
    y = S.band_limited_noise(1 << 15, 1)
    with pytest.raises(BegeError):
        ctx.bege_batch_create([(y, long_bank, 0, 2, 5.0)])            # L > 4096
    with pytest.raises(BegeError):
        ctx.bege_batch_create([(y, bank, 0, 5, 5.0)])                 # rows outside bank
    ctx.bege_release(bank)
    ctx.bege_release(long_bank)
