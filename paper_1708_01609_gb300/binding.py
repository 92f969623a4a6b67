"""ctypes binding of libbege (include/bege.h): argument marshalling only.

Every function here forwards to the C ABI of the same name; all arithmetic of
the search runs in the library's CUDA kernels.  Importing this module fails
loudly when the compiled library is missing: there is no CPU fallback.

Streams are passed as integers (a cudaStream_t, e.g.
``torch.cuda.current_stream().cuda_stream``); 0 is the legacy default stream.
Device pointers (``bege_load_segment_device``) are integers too, e.g.
``tensor.data_ptr()``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbege.so")

BEGE_OK = 0
BEGE_EINVAL = -1
BEGE_ENOMEM = -2
BEGE_EBUDGET = -3
BEGE_EOVERFLOW = -4
BEGE_ENOTREADY = -5
BEGE_ETIMEDOUT = -6
BEGE_ECUDA = -7

STATUS_NAMES = {0: "BEGE_OK", -1: "BEGE_EINVAL", -2: "BEGE_ENOMEM", -3: "BEGE_EBUDGET",
                -4: "BEGE_EOVERFLOW", -5: "BEGE_ENOTREADY", -6: "BEGE_ETIMEDOUT",
                -7: "BEGE_ECUDA"}

TAIL_DTYPE = np.dtype([("tmpl", np.uint32), ("lag", np.uint32), ("value", np.float32)])


class bege_config(ctypes.Structure):
    _fields_ = [("fs", ctypes.c_double), ("hbm_budget_bytes", ctypes.c_uint64),
                ("tail_capacity", ctypes.c_uint64), ("precision", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class bege_chirp(ctypes.Structure):
    _fields_ = [("f0", ctypes.c_double), ("fdot", ctypes.c_double)]


class bege_batch_entry(ctypes.Structure):
    _fields_ = [("strain", ctypes.c_void_p), ("n", ctypes.c_int64), ("bank_id", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("k_begin", ctypes.c_int64), ("k_end", ctypes.c_int64),
                ("kappa", ctypes.c_float), ("reserved2", ctypes.c_float)]


class bege_serve_config(ctypes.Structure):
    _fields_ = [("bank_id", ctypes.c_int32), ("streams", ctypes.c_int32),
                ("slice_templates", ctypes.c_int64), ("kappa", ctypes.c_float),
                ("reserved", ctypes.c_float), ("hbm_budget_bytes", ctypes.c_uint64)]


class bege_serve_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("channel", ctypes.c_int32), ("n", ctypes.c_int64),
                ("n_tails", ctypes.c_int64), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("gpu_ms", ctypes.c_double)]


class bege_search_opts(ctypes.Structure):
    _fields_ = [("kappa", ctypes.c_float), ("kappa_hi", ctypes.c_float),
                ("linear", ctypes.c_int32), ("project", ctypes.c_int32)]


class bege_tail(ctypes.Structure):
    _fields_ = [("tmpl", ctypes.c_uint32), ("lag", ctypes.c_uint32), ("value", ctypes.c_float)]


assert ctypes.sizeof(bege_tail) == TAIL_DTYPE.itemsize == 12

# name -> (restype, argtypes); every symbol declared in include/bege.h
_VP = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_PI32 = ctypes.POINTER(ctypes.c_int32)
_PI64 = ctypes.POINTER(ctypes.c_int64)
SIGNATURES = {
    "bege_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(bege_config)]),
    "bege_destroy": (ctypes.c_int, [_VP]),
    "bege_load_segment": (ctypes.c_int, [_VP, _VP, _I64, _I32, _VP, _PI32]),
    "bege_load_segment_device": (ctypes.c_int, [_VP, _VP, _I64, _I32, _VP, _PI32]),
    "bege_define_bank": (ctypes.c_int, [_VP, _VP, _I64, ctypes.c_double, ctypes.c_double, _VP,
                                        _PI32]),
    "bege_define_bank_symmetric": (ctypes.c_int, [_VP, _VP, _I64, ctypes.c_double, ctypes.c_double,
                                                  _VP, _PI32]),
    "bege_define_bank_samples": (ctypes.c_int, [_VP, _VP, _I64, _I64, _VP, _PI32]),
    "bege_correlate": (ctypes.c_int, [_VP, _I32, _I32, _I64, _I64, ctypes.c_float, _VP, _PI32]),
    "bege_correlate_max": (ctypes.c_int, [_VP, _I32, _I32, _I64, _I64, ctypes.c_float, _VP, _PI32]),
    "bege_correlate_multi": (ctypes.c_int, [_VP, _VP, _I32, _I32, _I64, _I64, ctypes.c_float, _VP,
                                            _VP]),
    "bege_fetch_max": (ctypes.c_int, [_VP, _I32, _VP, _VP, _I64]),
    "bege_correlate_band": (ctypes.c_int, [_VP, _I32, _I32, _I64, _I64, ctypes.c_float,
                                           ctypes.c_float, _VP, _PI32]),
    "bege_correlate_ex": (ctypes.c_int, [_VP, _I32, _I32, _I64, _I64,
                                         ctypes.POINTER(bege_search_opts), _VP, _PI32]),
    "bege_fetch_tails": (ctypes.c_int, [_VP, _I32, _VP, _I64, _PI64, _PI64]),
    "bege_sort_tails": (ctypes.c_int, [_VP, _I64]),
    "bege_query": (ctypes.c_int, [_VP, _I32]),
    "bege_job_kernel_ms": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(ctypes.c_float)]),
    "bege_get_sigma": (ctypes.c_int, [_VP, _I32, _VP, _I64]),
    "bege_dump_correlation": (ctypes.c_int, [_VP, _I32, _I32, _I64, _I64, _VP, _VP]),
    "bege_get_segment_spectrum": (ctypes.c_int, [_VP, _I32, _VP]),
    "bege_get_bank_samples": (ctypes.c_int, [_VP, _I32, _I64, _I64, _VP]),
    "bege_segment_length": (_I64, [_VP, _I32]),
    "bege_bank_length": (_I64, [_VP, _I32]),
    "bege_device_bytes": (ctypes.c_uint64, [_VP]),
    "bege_list_configs": (ctypes.c_int, [_VP, _I64, _PI32, _I32, _PI32]),
    "bege_set_config": (ctypes.c_int, [_VP, _I64, _I32, _I32]),
    "bege_get_config": (ctypes.c_int, [_VP, _I64, _PI32, _PI32]),
    "bege_autotune": (ctypes.c_int, [_VP, _I32, _I32, _I64, _I64, _I32, _VP,
                                     ctypes.POINTER(ctypes.c_float)]),
    "bege_batch_create": (ctypes.c_int, [_VP, _VP, _I32, ctypes.c_uint64, _VP, _PI32]),
    "bege_batch_run": (ctypes.c_int, [_VP, _I32, _VP]),
    "bege_batch_elapsed_ms": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(ctypes.c_float)]),
    "bege_batch_fetch_tails": (ctypes.c_int, [_VP, _I32, _I32, _VP, _I64, _PI64, _PI64]),
    "bege_batch_get_sigma": (ctypes.c_int, [_VP, _I32, _I32, _VP, _I64]),
    "bege_batch_set_plan": (ctypes.c_int, [_VP, _I32, _I32, _I64, _I32]),
    "bege_batch_get_plan": (ctypes.c_int, [_VP, _I32, _PI32, _PI64, _PI32]),
    "bege_batch_autotune": (ctypes.c_int, [_VP, _I32, _I32, _VP, ctypes.POINTER(ctypes.c_float)]),
    "bege_search_noalloc": (ctypes.c_int, [_VP, _I64, _VP, _I64, _I64, _I64, ctypes.c_float, _VP,
                                           _VP, ctypes.c_uint64, _VP, _VP]),
    "bege_serve_create": (ctypes.c_int, [_VP, ctypes.POINTER(bege_serve_config), _PI32]),
    "bege_serve_submit": (ctypes.c_int, [_VP, _I32, _VP, _I64, _I32, _PI64]),
    "bege_serve_wait": (ctypes.c_int, [_VP, _I32, _I64, _I32]),
    "bege_serve_info_get": (ctypes.c_int, [_VP, _I32, _I64, ctypes.POINTER(bege_serve_info)]),
    "bege_serve_fetch_tails": (ctypes.c_int, [_VP, _I32, _I64, _VP, _I64, _PI64, _PI64]),
    "bege_serve_get_sigma": (ctypes.c_int, [_VP, _I32, _I64, _VP, _I64]),
    "bege_serve_forget": (ctypes.c_int, [_VP, _I32, _I64]),
    "bege_serve_destroy": (ctypes.c_int, [_VP, _I32]),
    "bege_release": (ctypes.c_int, [_VP, _I32]),
    "bege_last_error": (ctypes.c_char_p, [_VP]),
    "bege_version": (ctypes.c_char_p, []),
}

_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libbege.so (built by ``paper_1708_01609_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libbege.so not built at {path}; run paper_1708_01609_gb300.build")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class BegeError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _check(code: int, where: str, ok=(BEGE_OK,)) -> int:
    if code not in ok:
        msg = load_library().bege_last_error(None)
        raise BegeError(code, where, msg.decode() if msg else "")
    return code


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class Context:
    """One libbege context on one CUDA device (method names follow bege.h)."""

    def __init__(self, device: int = 0, fs: float = 4096.0, hbm_budget_bytes: int = 0,
                 tail_capacity: int = 1 << 20, precision: int = 0):
        self.lib = load_library()
        cfg = bege_config(fs, hbm_budget_bytes, tail_capacity, precision, 0)
        h = _VP()
        _check(self.lib.bege_create(ctypes.byref(h), device, ctypes.byref(cfg)), "bege_create")
        self.h = h
        self.fs = fs

    def close(self):
        if getattr(self, "h", None):
            _check(self.lib.bege_destroy(self.h), "bege_destroy")
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- segments ---------------------------------------------------------
    def bege_load_segment(self, strain: np.ndarray, channel: int = 0, stream: int = 0) -> int:
        y = np.ascontiguousarray(strain, dtype=np.float32)
        sid = _I32()
        _check(self.lib.bege_load_segment(self.h, _ptr(y), len(y), channel, stream,
                                          ctypes.byref(sid)), "bege_load_segment")
        return sid.value

    def bege_load_segment_device(self, ptr: int, n: int, channel: int = 0, stream: int = 0) -> int:
        sid = _I32()
        _check(self.lib.bege_load_segment_device(self.h, ptr, n, channel, stream,
                                                 ctypes.byref(sid)), "bege_load_segment_device")
        return sid.value

    # -- banks ------------------------------------------------------------
    def bege_define_bank(self, params: np.ndarray, tau: float = 1.0, taper_frac: float = 0.05,
                         stream: int = 0, symmetric: bool = False) -> int:
        """symmetric: bege_define_bank_symmetric (chirps forward + backward in time)."""
        p = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 2)
        bid = _I32()
        fn = self.lib.bege_define_bank_symmetric if symmetric else self.lib.bege_define_bank
        _check(fn(self.h, _ptr(p), len(p), tau, taper_frac, stream, ctypes.byref(bid)),
               "bege_define_bank_symmetric" if symmetric else "bege_define_bank")
        return bid.value

    def bege_define_bank_samples(self, samples: np.ndarray, stream: int = 0) -> int:
        w = np.ascontiguousarray(samples, dtype=np.float32)
        if w.ndim != 2:
            raise ValueError("samples must be (count, length)")
        bid = _I32()
        _check(self.lib.bege_define_bank_samples(self.h, _ptr(w), w.shape[0], w.shape[1], stream,
                                                 ctypes.byref(bid)), "bege_define_bank_samples")
        return bid.value

    # -- search -----------------------------------------------------------
    def bege_correlate(self, seg: int, bank: int, k_begin: int, k_end: int, kappa: float,
                       stream: int = 0) -> int:
        jid = _I32()
        _check(self.lib.bege_correlate(self.h, seg, bank, k_begin, k_end, kappa, stream,
                                       ctypes.byref(jid)), "bege_correlate")
        return jid.value

    def bege_correlate_multi(self, segs, bank: int, k_begin: int, k_end: int, kappa: float,
                             stream: int = 0) -> list[int]:
        """One launch for several segments of one length; a job per segment."""
        ids = np.ascontiguousarray(segs, dtype=np.int32)
        out = np.empty(len(ids), dtype=np.int32)
        _check(self.lib.bege_correlate_multi(self.h, _ptr(ids), len(ids), bank, k_begin, k_end,
                                             kappa, stream, _ptr(out)), "bege_correlate_multi")
        return out.tolist()

    def bege_correlate_max(self, seg: int, bank: int, k_begin: int, k_end: int, kappa: float,
                           stream: int = 0) -> int:
        jid = _I32()
        _check(self.lib.bege_correlate_max(self.h, seg, bank, k_begin, k_end, kappa, stream,
                                           ctypes.byref(jid)), "bege_correlate_max")
        return jid.value

    def bege_correlate_band(self, seg: int, bank: int, k_begin: int, k_end: int, kappa_lo: float,
                            kappa_hi: float, stream: int = 0) -> int:
        jid = _I32()
        _check(self.lib.bege_correlate_band(self.h, seg, bank, k_begin, k_end, kappa_lo, kappa_hi,
                                            stream, ctypes.byref(jid)), "bege_correlate_band")
        return jid.value

    def bege_correlate_ex(self, seg: int, bank: int, k_begin: int, k_end: int, kappa: float,
                          kappa_hi: float = 0.0, linear: bool = False, project: bool = False,
                          stream: int = 0) -> int:
        """The search with the epilogue options combined: band upper end
        kappa_hi (0 = none), overlap-save lag mask (linear) and per-lag
        maximum (project; fetch it with bege_fetch_max)."""
        o = bege_search_opts(kappa, kappa_hi, int(linear), int(project))
        jid = _I32()
        _check(self.lib.bege_correlate_ex(self.h, seg, bank, k_begin, k_end, ctypes.byref(o),
                                          stream, ctypes.byref(jid)), "bege_correlate_ex")
        return jid.value

    def bege_fetch_max(self, job: int, n: int):
        """Returns (snr FP32 array, template int32 array) of n = N lags."""
        snr = np.empty(n, dtype=np.float32)
        tmpl = np.empty(n, dtype=np.int32)
        _check(self.lib.bege_fetch_max(self.h, job, _ptr(snr), _ptr(tmpl), n), "bege_fetch_max")
        return snr, tmpl

    def bege_fetch_tails(self, job: int, capacity: int | None = None, out: np.ndarray | None = None,
                         sort: bool = False):
        """Returns (records as TAIL_DTYPE array, n_total).

        With neither ``capacity`` nor ``out`` the true count is queried first
        and a buffer of that size is used.  ``sort``: records in (template,
        lag) order (bege_sort_tails) instead of device completion order."""
        nw, nt = _I64(), _I64()
        if out is None:
            if capacity is None:
                _check(self.lib.bege_fetch_tails(self.h, job, None, 0, ctypes.byref(nw),
                                                 ctypes.byref(nt)), "bege_fetch_tails",
                       ok=(BEGE_OK, BEGE_EOVERFLOW))
                capacity = nt.value
            out = np.empty(capacity, dtype=TAIL_DTYPE)
        _check(self.lib.bege_fetch_tails(self.h, job, _ptr(out), len(out), ctypes.byref(nw),
                                         ctypes.byref(nt)), "bege_fetch_tails",
               ok=(BEGE_OK, BEGE_EOVERFLOW))
        recs = out[: nw.value]
        if sort:
            bege_sort_tails(recs)
        return recs, nt.value

    def bege_query(self, job: int) -> bool:
        return _check(self.lib.bege_query(self.h, job), "bege_query",
                      ok=(BEGE_OK, BEGE_ENOTREADY)) == BEGE_OK

    def bege_job_kernel_ms(self, job: int) -> float:
        ms = ctypes.c_float()
        _check(self.lib.bege_job_kernel_ms(self.h, job, ctypes.byref(ms)), "bege_job_kernel_ms")
        return float(ms.value)

    def bege_get_sigma(self, job: int, count: int) -> np.ndarray:
        out = np.empty(count, dtype=np.float32)
        _check(self.lib.bege_get_sigma(self.h, job, _ptr(out), count), "bege_get_sigma")
        return out

    def bege_dump_correlation(self, seg: int, bank: int, k_begin: int, k_end: int,
                              stream: int = 0) -> np.ndarray:
        n = self.lib.bege_segment_length(self.h, seg)
        out = np.empty((k_end - k_begin, n), dtype=np.float32)
        _check(self.lib.bege_dump_correlation(self.h, seg, bank, k_begin, k_end, _ptr(out),
                                              stream), "bege_dump_correlation")
        return out

    def bege_get_segment_spectrum(self, seg: int) -> np.ndarray:
        n = self.lib.bege_segment_length(self.h, seg)
        out = np.empty(n + 2, dtype=np.float32)
        _check(self.lib.bege_get_segment_spectrum(self.h, seg, _ptr(out)),
               "bege_get_segment_spectrum")
        return out[0::2].astype(np.float64) + 1j * out[1::2]

    def bege_get_bank_samples(self, bank: int, k_begin: int, k_end: int) -> np.ndarray:
        length = self.lib.bege_bank_length(self.h, bank)
        out = np.empty((k_end - k_begin, length), dtype=np.float32)
        _check(self.lib.bege_get_bank_samples(self.h, bank, k_begin, k_end, _ptr(out)),
               "bege_get_bank_samples")
        return out

    def bege_list_configs(self, n: int) -> list[tuple[int, int]]:
        buf = (ctypes.c_int32 * 32)()
        cnt = _I32()
        _check(self.lib.bege_list_configs(self.h, n, buf, 16, ctypes.byref(cnt)),
               "bege_list_configs")
        return [(buf[2 * i], buf[2 * i + 1]) for i in range(min(cnt.value, 16))]

    def bege_set_config(self, n: int, nc: int, threads: int) -> None:
        _check(self.lib.bege_set_config(self.h, n, nc, threads), "bege_set_config")

    def bege_get_config(self, n: int) -> tuple[int, int]:
        a, b = _I32(), _I32()
        _check(self.lib.bege_get_config(self.h, n, ctypes.byref(a), ctypes.byref(b)),
               "bege_get_config")
        return a.value, b.value

    def bege_autotune(self, seg: int, bank: int, k_begin: int, k_end: int, reps: int = 3,
                      stream: int = 0) -> float:
        ms = ctypes.c_float()
        _check(self.lib.bege_autotune(self.h, seg, bank, k_begin, k_end, reps, stream,
                                      ctypes.byref(ms)), "bege_autotune")
        return float(ms.value)

    # -- batching form ----------------------------------------------------
    def bege_batch_create(self, entries, tail_capacity: int = 0, stream: int = 0) -> int:
        """entries: list of (strain FP32 array, bank_id, k_begin, k_end, kappa)."""
        keep = [np.ascontiguousarray(e[0], dtype=np.float32) for e in entries]
        arr = (bege_batch_entry * len(entries))()
        for i, (e, y) in enumerate(zip(entries, keep)):
            arr[i] = bege_batch_entry(y.ctypes.data, len(y), e[1], 0, e[2], e[3], e[4], 0.0)
        bid = _I32()
        _check(self.lib.bege_batch_create(self.h, arr, len(entries), tail_capacity, stream,
                                          ctypes.byref(bid)), "bege_batch_create")
        return bid.value

    def bege_batch_run(self, batch: int, stream: int = 0) -> None:
        _check(self.lib.bege_batch_run(self.h, batch, stream), "bege_batch_run")

    def bege_batch_elapsed_ms(self, batch: int) -> float:
        ms = ctypes.c_float()
        _check(self.lib.bege_batch_elapsed_ms(self.h, batch, ctypes.byref(ms)),
               "bege_batch_elapsed_ms")
        return float(ms.value)

    def bege_batch_fetch_tails(self, batch: int, entry: int, capacity: int | None = None):
        nw, nt = _I64(), _I64()
        if capacity is None:
            _check(self.lib.bege_batch_fetch_tails(self.h, batch, entry, None, 0, ctypes.byref(nw),
                                                   ctypes.byref(nt)), "bege_batch_fetch_tails",
                   ok=(BEGE_OK, BEGE_EOVERFLOW))
            capacity = nt.value
        out = np.empty(capacity, dtype=TAIL_DTYPE)
        _check(self.lib.bege_batch_fetch_tails(self.h, batch, entry, _ptr(out), capacity,
                                               ctypes.byref(nw), ctypes.byref(nt)),
               "bege_batch_fetch_tails", ok=(BEGE_OK, BEGE_EOVERFLOW))
        return out[: nw.value], nt.value

    def bege_batch_get_sigma(self, batch: int, entry: int, count: int) -> np.ndarray:
        out = np.empty(count, dtype=np.float32)
        _check(self.lib.bege_batch_get_sigma(self.h, batch, entry, _ptr(out), count),
               "bege_batch_get_sigma")
        return out

    def bege_batch_set_plan(self, batch: int, plan: int, chunk: int = 256, order: int = 0):
        _check(self.lib.bege_batch_set_plan(self.h, batch, plan, chunk, order),
               "bege_batch_set_plan")

    def bege_batch_get_plan(self, batch: int) -> tuple[int, int, int]:
        p, c, o = _I32(), _I64(), _I32()
        _check(self.lib.bege_batch_get_plan(self.h, batch, ctypes.byref(p), ctypes.byref(c),
                                            ctypes.byref(o)), "bege_batch_get_plan")
        return p.value, c.value, o.value

    def bege_batch_autotune(self, batch: int, reps: int = 2, stream: int = 0) -> float:
        ms = ctypes.c_float()
        _check(self.lib.bege_batch_autotune(self.h, batch, reps, stream, ctypes.byref(ms)),
               "bege_batch_autotune")
        return float(ms.value)

    # -- serving form ------------------------------------------------------
    def bege_serve_create(self, bank: int, kappa: float, streams: int = 0,
                          slice_templates: int = 0, hbm_budget_bytes: int = 0) -> int:
        cfg = bege_serve_config(bank, streams, slice_templates, kappa, 0.0, hbm_budget_bytes)
        sid = _I32()
        _check(self.lib.bege_serve_create(self.h, ctypes.byref(cfg), ctypes.byref(sid)),
               "bege_serve_create")
        return sid.value

    def bege_serve_submit(self, server: int, strain: np.ndarray, channel: int = 0) -> int:
        y = np.ascontiguousarray(strain, dtype=np.float32)
        rid = _I64()
        _check(self.lib.bege_serve_submit(self.h, server, _ptr(y), len(y), channel,
                                          ctypes.byref(rid)), "bege_serve_submit")
        return rid.value

    def bege_serve_wait(self, server: int, request: int, timeout_ms: int = -1) -> bool:
        rc = _check(self.lib.bege_serve_wait(self.h, server, request, timeout_ms),
                    "bege_serve_wait", ok=(BEGE_OK, BEGE_ETIMEDOUT))
        return rc == BEGE_OK

    def bege_serve_info_get(self, server: int, request: int) -> dict:
        info = bege_serve_info()
        _check(self.lib.bege_serve_info_get(self.h, server, request, ctypes.byref(info)),
               "bege_serve_info_get")
        return {f: getattr(info, f) for f, _ in bege_serve_info._fields_}

    def bege_serve_fetch_tails(self, server: int, request: int):
        nw, nt = _I64(), _I64()
        _check(self.lib.bege_serve_fetch_tails(self.h, server, request, None, 0, ctypes.byref(nw),
                                               ctypes.byref(nt)), "bege_serve_fetch_tails",
               ok=(BEGE_OK, BEGE_EOVERFLOW))
        out = np.empty(nt.value, dtype=TAIL_DTYPE)
        _check(self.lib.bege_serve_fetch_tails(self.h, server, request, _ptr(out), len(out),
                                               ctypes.byref(nw), ctypes.byref(nt)),
               "bege_serve_fetch_tails", ok=(BEGE_OK, BEGE_EOVERFLOW))
        return out[: nw.value], nt.value

    def bege_serve_get_sigma(self, server: int, request: int, count: int) -> np.ndarray:
        out = np.empty(count, dtype=np.float32)
        _check(self.lib.bege_serve_get_sigma(self.h, server, request, _ptr(out), count),
               "bege_serve_get_sigma")
        return out

    def bege_serve_forget(self, server: int, request: int) -> None:
        _check(self.lib.bege_serve_forget(self.h, server, request), "bege_serve_forget")

    def bege_serve_destroy(self, server: int) -> None:
        _check(self.lib.bege_serve_destroy(self.h, server), "bege_serve_destroy")

    def bege_release(self, handle: int) -> None:
        _check(self.lib.bege_release(self.h, handle), "bege_release")

    def bege_device_bytes(self) -> int:
        return int(self.lib.bege_device_bytes(self.h))


def bege_search_noalloc(strain_dev: int, n: int, bank_dev: int, ld: int, k_begin: int,
                        k_end: int, kappa: float, sigma_dev: int, tails_dev: int,
                        tail_capacity: int, tail_count_dev: int, stream: int = 0) -> None:
    """Search of one segment that allocates no device memory: every pointer is
    a device address owned by the caller (see include/bege.h)."""
    lib = load_library()
    _check(lib.bege_search_noalloc(strain_dev, n, bank_dev, ld, k_begin, k_end, kappa,
                                   sigma_dev, tails_dev, tail_capacity, tail_count_dev, stream),
           "bege_search_noalloc")


def bege_sort_tails(recs: np.ndarray) -> np.ndarray:
    """Sort TAIL_DTYPE records in place by (template, lag); returns them."""
    if recs.dtype != TAIL_DTYPE or not recs.flags.c_contiguous:
        raise ValueError("records must be a contiguous TAIL_DTYPE array")
    _check(load_library().bege_sort_tails(_ptr(recs) if len(recs) else None, len(recs)),
           "bege_sort_tails")
    return recs


def bege_version() -> str:
    return load_library().bege_version().decode()
