"""Serving form: continuous batching over a resident bank.  Each request's
result is the same alone and in a mix of concurrent requests (bitwise: every
template runs the same kernel arithmetic), equals the regular entry points,
matches the FP64 oracle on sampled templates, and requests queue under a
small HBM budget instead of failing."""
import time

import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_helpers import compare_tails, make_ctx, oracle_rho

pytestmark = pytest.mark.gpu

KAPPA = 4.5


@pytest.fixture(scope="module", params=[0, 1], ids=["fp32", "bf16x3"])
def served(request):
    """A context of the given precision (FP32 path, or the BF16x3 precision
    form) with a resident bank."""
    ctx = make_ctx(tail_capacity=1 << 20, precision=request.param)
    params = S.grid_paper(64, 96)                     # 6144 in-band chirps
    bank = ctx.bege_define_bank(params, tau=1.0)
    yield ctx, params, bank, request.param
    ctx.close()


def result(ctx, sv, rid, count):
    assert ctx.bege_serve_wait(sv, rid, 120000)
    recs, total = ctx.bege_serve_fetch_tails(sv, rid)
    assert total == len(recs)
    return np.sort(recs, order=["tmpl", "lag"]), ctx.bege_serve_get_sigma(sv, rid, count)


def test_alone_equals_in_the_mix_and_regular_path(served):
    ctx, params, bank, _ = served
    count = len(params)
    reqs = S.serving_stream(9, seed=5, n_inject=2, params=params)
    sv = ctx.bege_serve_create(bank, KAPPA, streams=3, slice_templates=1000)
    # each request alone
    alone = []
    for a in reqs:
        rid = ctx.bege_serve_submit(sv, a.y, a.channel)
        alone.append(result(ctx, sv, rid, count))
    # all of them at once: their slices interleave on three streams
    ids = [ctx.bege_serve_submit(sv, a.y, a.channel) for a in reqs]
    infos = []
    for a, rid, (ra, sa) in zip(reqs, ids, alone):
        rm, sm = result(ctx, sv, rid, count)
        assert np.array_equal(sm, sa)
        assert np.array_equal(rm, ra)
        infos.append(ctx.bege_serve_info_get(sv, rid))
    # the mixed requests really overlapped: later ones were admitted before
    # earlier ones finished
    assert any(infos[i + 1]["t_admit"] < infos[i]["t_done"] for i in range(len(infos) - 1))
    ctx.bege_serve_destroy(sv)
    # the regular entry points give the same numbers
    for a, (ra, sa) in list(zip(reqs, alone))[:3]:
        seg = ctx.bege_load_segment(a.y)
        job = ctx.bege_correlate(seg, bank, 0, count, KAPPA)
        rr, _ = ctx.bege_fetch_tails(job)
        assert np.array_equal(ctx.bege_get_sigma(job, count), sa)
        assert np.array_equal(np.sort(rr, order=["tmpl", "lag"]), ra)
        ctx.bege_release(job)
        ctx.bege_release(seg)


def test_served_requests_match_oracle(served):
    """Three requests of 8, 16 and 32 s from the two channels, each with two
    injected chirps of the bank, served together (their slices interleave on
    three streams): every request's sigma and tails on a sample of templates
    (every injected template with its neighbours in f0 and fdot, and 16
    random ones) against the FP64 oracle.  Bars as for the regular path:
    sigma within 1e-6 relative (1e-5 for the precision form), tail values
    within 1e-5 sigma (2e-3 sigma), tail sets identical away from the
    threshold."""
    ctx, params, bank, prec = served
    count, n_f0 = len(params), 96
    tol, sig_tol = (1e-5, 1e-6) if prec == 0 else (2e-3, 1e-5)
    segs = [(c, S.make_segment(n, params, 2, 300 + i))
            for i, (c, n) in enumerate([(0, 1 << 15), (1, 1 << 16), (0, 1 << 17)])]
    sv = ctx.bege_serve_create(bank, KAPPA, streams=3, slice_templates=1000)
    ids = [ctx.bege_serve_submit(sv, seg.y, c) for c, seg in segs]
    served_out = [result(ctx, sv, rid, count) for rid in ids]
    infos = [ctx.bege_serve_info_get(sv, rid) for rid in ids]
    ctx.bege_serve_destroy(sv)
    assert [i["n"] for i in infos] == [1 << 15, 1 << 16, 1 << 17]
    rng = np.random.Generator(np.random.PCG64(77))
    for (c, seg), (recs, sig) in zip(segs, served_out):
        sample = set(rng.choice(count, 16, replace=False).tolist())
        for k, _, _ in seg.injections:
            for d in (0, -1, 1, -n_f0, n_f0):
                if 0 <= k + d < count:
                    sample.add(k + d)
        sample = sorted(sample)
        bank64 = O.chirp_bank(params[sample], 4096.0, 4096, 0.05)
        rho, osig = oracle_rho(seg.y, bank64)
        assert np.all(np.abs(sig[sample] / osig - 1) <= sig_tol)
        res = compare_tails(recs, {k: (rho[i], osig[i]) for i, k in enumerate(sample)},
                            KAPPA, tmpl_subset=sample, tol=tol)
        assert res["matched"] > 0
        got = set(zip(recs["tmpl"].tolist(), recs["lag"].tolist()))
        for k, lag, _ in seg.injections:
            assert (k, lag) in got, (seg.n, k, lag)


def test_budget_admission_queues_requests(served):
    ctx, params, bank, _ = served
    count = len(params)
    reqs = S.serving_stream(6, seed=8)
    # room for one 32 s segment's spectrum at a time
    budget = (1 << 17) * 4 + (1 << 16) * 24 + 64
    sv = ctx.bege_serve_create(bank, KAPPA, streams=2, slice_templates=2048,
                               hbm_budget_bytes=budget)
    ids = [ctx.bege_serve_submit(sv, a.y, a.channel) for a in reqs]
    for rid in ids:
        assert ctx.bege_serve_wait(sv, rid, 120000)
    infos = [ctx.bege_serve_info_get(sv, rid) for rid in ids]
    assert all(i["state"] == 2 for i in infos)

    def held(n):  # spectrum + coefficients + staged strain of a segment
        return 16 * n + 8

    # at every admission the requests admitted and not yet done fit the budget
    for i in infos:
        live = [j for j in infos if j["t_admit"] <= i["t_admit"] < j["t_done"]]
        assert sum(held(j["n"]) for j in live) <= budget
    # and the budget did make requests wait: some admission followed a completion
    assert any(i["t_admit"] > i["t_submit"] + 1e-3 for i in infos)
    ctx.bege_serve_destroy(sv)


def test_request_larger_than_budget_fails():
    from paper_1708_01609_gb300.binding import BegeError
    ctx = make_ctx()
    bank = ctx.bege_define_bank(S.grid_small()[:8])
    sv = ctx.bege_serve_create(bank, KAPPA, hbm_budget_bytes=1 << 16)
    rid = ctx.bege_serve_submit(sv, S.band_limited_noise(1 << 15, 3))
    with pytest.raises(BegeError) as e:
        ctx.bege_serve_wait(sv, rid, 60000)
    assert e.value.code == -3
    assert ctx.bege_serve_info_get(sv, rid)["state"] == 3
    ctx.bege_serve_destroy(sv)
    ctx.close()


def test_destroy_with_work_in_flight():
    """Destroying a busy server drains the slices in flight and releases every
    segment: only the pooled slice buffers (at most a few) remain."""
    ctx = make_ctx(tail_capacity=1 << 16)
    bank = ctx.bege_define_bank(S.grid_paper(32, 64))
    before = ctx.bege_device_bytes()
    sv = ctx.bege_serve_create(bank, KAPPA, streams=2, slice_templates=256)
    for a in S.serving_stream(5, seed=11):
        ctx.bege_serve_submit(sv, a.y, a.channel)
    time.sleep(0.01)
    ctx.bege_serve_destroy(sv)
    assert ctx.bege_device_bytes() - before < (8 << 20)
    ctx.close()
