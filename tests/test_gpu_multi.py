"""Several segments of one length in one launch (the paper's block of
segments per template, Sec. 3.2): every segment's tails and sigma equal,
bitwise, those of a single search of that segment."""
import numpy as np
import pytest

import synthetic as S
from gpu_helpers import make_ctx

pytestmark = pytest.mark.gpu


def _sorted(recs):
    return recs[np.lexsort((recs["lag"], recs["tmpl"]))]


@pytest.fixture(scope="module")
def mctx():
    c = make_ctx(tail_capacity=1 << 22)
    _, params = S.paper_case(seed=2017)
    bank = c.bege_define_bank(params[:: 128], tau=1.0, taper_frac=0.05)   # 8192 chirps
    yield c, bank, params[:: 128]
    c.close()


@pytest.mark.parametrize("lg,m", [(16, 1), (16, 3), (16, 8), (14, 2), (17, 2)])
def test_multi_equals_single_searches(mctx, lg, m):
    ctx, bank, params = mctx
    n = 1 << lg
    kappa = 5.0
    segs = []
    for i in range(m):
        y = S.band_limited_noise(n, 500 + 10 * lg + i).astype(np.float64)
        f0, fd = params[(37 * i + 11) % len(params)]
        y = S.inject(y, S.chirp_signal(f0, fd, 4096), (1000 + 777 * i) % (n - 4096),
                     15.0 * S.expected_filter_rms(n))
        segs.append(ctx.bege_load_segment(y))
    k0, k1 = 5, len(params) - 3
    jobs = ctx.bege_correlate_multi(segs, bank, k0, k1, kappa)
    assert len(jobs) == m
    for seg, job in zip(segs, jobs):
        got, total = ctx.bege_fetch_tails(job)
        sig = ctx.bege_get_sigma(job, k1 - k0)
        ref_job = ctx.bege_correlate(seg, bank, k0, k1, kappa)
        ref, ref_total = ctx.bege_fetch_tails(ref_job)
        assert total == ref_total > 0
        assert np.array_equal(sig, ctx.bege_get_sigma(ref_job, k1 - k0))
        assert np.array_equal(_sorted(got), _sorted(ref))
        ctx.bege_release(ref_job)
        ctx.bege_release(job)
    for sg in segs:
        ctx.bege_release(sg)


def test_multi_rejects_bad_arguments(mctx):
    from paper_1708_01609_gb300.binding import BegeError
    ctx, bank, params = mctx
    a = ctx.bege_load_segment(S.band_limited_noise(1 << 16, 1))
    b = ctx.bege_load_segment(S.band_limited_noise(1 << 15, 2))
    with pytest.raises(BegeError):
        ctx.bege_correlate_multi([a, b], bank, 0, 10, 5.0)          # two lengths
    with pytest.raises(BegeError):
        ctx.bege_correlate_multi([a] * 9, bank, 0, 10, 5.0)         # more than 8
    with pytest.raises(BegeError):
        ctx.bege_correlate_multi([], bank, 0, 10, 5.0)
    long_bank = ctx.bege_define_bank_samples(np.ones((2, 5000), np.float32))
    with pytest.raises(BegeError):
        ctx.bege_correlate_multi([a], long_bank, 0, 2, 5.0)         # template > 4096
    for h in (a, b, long_bank):
        ctx.bege_release(h)
    tc = make_ctx(precision=1)
    seg = tc.bege_load_segment(S.band_limited_noise(1 << 16, 3))
    tb = tc.bege_define_bank(params[:16])
    with pytest.raises(BegeError):
        tc.bege_correlate_multi([seg], tb, 0, 16, 5.0)               # FP32 contexts only
    tc.close()
