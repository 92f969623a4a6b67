"""bege_search_noalloc: the entry point for callers that may not allocate
device memory (their device memory belongs to an allocator of their own, for
example a framework's pool or an arena reserved at start-up).

The caller allocates every input and output here (with torch, standing in
for the caller's own allocator) and the library uses only its fixed scratch
array.  Three calls in a row, with different segment lengths (2^16 and 2^14
split into columns; 2^11 a single column, whose twiddle tables only this
call's table kernel writes), must agree with the regular entry points (load
segment, define bank, correlate, fetch) within the tolerances of the other
GPU tests: sigma within 1e-6 relative, tail values within 1e-5 sigma, tail
sets identical away from the threshold.  The first call is also checked
against the FP64 oracle with the same rule.

This file is named to be collected last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_helpers import NEAR, TOL_FP32, compare_tails, make_ctx

pytestmark = pytest.mark.gpu


def regular_search(ctx, y, bank, k0, k1, kappa):
    seg = ctx.bege_load_segment(y)
    bid = ctx.bege_define_bank_samples(bank)
    job = ctx.bege_correlate(seg, bid, k0, k1, kappa)
    recs, total = ctx.bege_fetch_tails(job)
    sig = ctx.bege_get_sigma(job, k1 - k0)
    for h in (job, bid, seg):
        ctx.bege_release(h)
    return recs, total, sig


def noalloc_search(y, bank, k0, k1, kappa, cap):
    import torch

    from paper_1708_01609_gb300 import binding
    y_d = torch.from_numpy(y).cuda()
    bank_d = torch.from_numpy(bank).cuda()
    sig_d = torch.zeros(k1 - k0, dtype=torch.float32, device="cuda")
    tails_d = torch.zeros(cap * binding.TAIL_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    cnt_d = torch.zeros(1, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    binding.bege_search_noalloc(y_d.data_ptr(), len(y), bank_d.data_ptr(), bank.shape[1], k0, k1,
                                kappa, sig_d.data_ptr(), tails_d.data_ptr(), cap,
                                cnt_d.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    total = int(cnt_d.item())
    recs = tails_d.cpu().numpy().view(binding.TAIL_DTYPE)[: min(total, cap)]
    return recs, total, sig_d.cpu().numpy()


def case(n, count, length, seed):
    bank = S.random_samples_bank(count, length, seed)
    y = S.band_limited_noise(n, seed + 1).astype(np.float64)
    w = bank[5].astype(np.float64)
    w /= np.linalg.norm(w)
    y[(1234 + np.arange(length)) % n] += 15.0 * w     # one strong injection of row 5
    return y.astype(np.float32), bank


def test_noalloc_matches_regular_entry_points_two_calls():
    from paper_1708_01609_gb300.binding import BegeError, bege_search_noalloc
    ctx = make_ctx(tail_capacity=1 << 20)
    calls = [(1 << 16, 24, 4096, 0, 24, 4.5, 11), (1 << 14, 40, 2048, 3, 40, 4.5, 12),
             (1 << 11, 16, 512, 2, 16, 4.0, 13)]
    for i, (n, count, length, k0, k1, kappa, seed) in enumerate(calls):
        y, bank = case(n, count, length, seed)
        got, got_total, got_sig = noalloc_search(y, bank, k0, k1, kappa, cap=1 << 16)
        if i == 0:
            # the same call against the FP64 oracle
            ref_o = O.search(y, bank[k0:k1].astype(np.float64), np.inf, k0=k0, batch=8,
                             return_rho=True)
            assert np.all(np.abs(got_sig / ref_o["sigma"] - 1) <= 1e-6)
            compare_tails(got, {k0 + r: (ref_o["rho"][r], ref_o["sigma"][r])
                                for r in range(k1 - k0)}, kappa)
        ref, ref_total, ref_sig = regular_search(ctx, y, bank, k0, k1, kappa)
        assert got_total == len(got) and ref_total == len(ref) and got_total > 0
        assert np.all(np.abs(got_sig / ref_sig - 1) <= 1e-6)
        a = {(int(r["tmpl"]), int(r["lag"])): float(r["value"]) for r in got}
        b = {(int(r["tmpl"]), int(r["lag"])): float(r["value"]) for r in ref}
        for key in set(a) | set(b):
            sig = float(ref_sig[key[0] - k0])
            if key in a and key in b:
                assert abs(a[key] - b[key]) <= TOL_FP32 * sig
            else:
                v = a.get(key, b.get(key))
                assert abs(abs(v) - kappa * sig) <= NEAR * sig, key
        assert (5, 1234) in a
    # sizes beyond the scratch array are refused with a clear error
    with pytest.raises(BegeError) as err:
        bege_search_noalloc(1 << 20, 1 << 17, 1 << 20, 4096, 0, 1, 5.0, 1 << 20, 1 << 20, 1,
                            1 << 20)
    assert err.value.code == -1 and "2^16" in str(err.value)
    # so are output buffers that the kernels' 4-byte stores could not use
    for sig_p, tails_p in ((1 << 20, (1 << 20) + 2), ((1 << 20) + 1, 1 << 20)):
        with pytest.raises(BegeError) as err:
            bege_search_noalloc(1 << 20, 1 << 14, 1 << 20, 4096, 0, 1, 5.0, sig_p, tails_p, 1,
                                1 << 20)
        assert err.value.code == -1 and "misaligned" in str(err.value)
    ctx.close()
