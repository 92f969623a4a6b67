"""The C-ABI library builds, loads and exports every symbol of include/bege.h.

CPU-only: no compute call is made.  bege_create is the one call exercised,
and on a machine without a usable GPU it must fail loudly (BEGE_ECUDA), not
fall back to the CPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bege.h")


def declared_symbols():
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bege_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1708_01609_gb300 import build
    path = build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["bege_create", "bege_load_segment", "bege_define_bank", "bege_correlate",
                 "bege_fetch_tails", "bege_get_sigma", "bege_release", "bege_last_error"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1708_01609_gb300 import binding
    assert set(binding.SIGNATURES) == set(declared_symbols())


def test_struct_layouts_match_header():
    from paper_1708_01609_gb300 import binding
    assert ctypes.sizeof(binding.bege_tail) == 12
    assert ctypes.sizeof(binding.bege_chirp) == 16
    assert ctypes.sizeof(binding.bege_config) == 32


def test_version_string(lib):
    lib.bege_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.bege_version()


def test_create_without_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.bege_create(ctypes.byref(h), 0, None)
    assert rc == -7  # BEGE_ECUDA
    lib.bege_last_error.restype = ctypes.c_char_p
    assert lib.bege_last_error(None)


def test_null_arguments_rejected(lib):
    # argument validation happens before any CUDA call
    assert lib.bege_create(None, 0, None) == -1
    assert lib.bege_destroy(None) == -1
    assert lib.bege_release(None, 1) == -1


def test_sort_tails_orders_by_template_then_lag():
    """bege_sort_tails is host-only: records in (template, lag) order, values
    carried along, the empty array accepted and a bad array rejected."""
    import numpy as np
    from paper_1708_01609_gb300 import binding
    g = np.random.default_rng(3)
    pairs = np.unique(g.integers(0, 1 << 20, (5000, 2)).astype(np.uint32), axis=0)
    pairs = pairs[g.permutation(len(pairs))]
    recs = np.empty(len(pairs), dtype=binding.TAIL_DTYPE)
    recs["tmpl"], recs["lag"] = pairs[:, 0], pairs[:, 1]
    recs["value"] = (pairs[:, 0].astype(np.float64) - pairs[:, 1]).astype(np.float32)
    want = recs[np.lexsort((recs["lag"], recs["tmpl"]))].copy()
    got = binding.bege_sort_tails(recs)
    assert np.array_equal(got, want)
    binding.bege_sort_tails(np.empty(0, dtype=binding.TAIL_DTYPE))
    lib = binding.load_library()
    assert lib.bege_sort_tails(None, 5) == binding.BEGE_EINVAL
    assert lib.bege_sort_tails(None, -1) == binding.BEGE_EINVAL


STRUCTS = ["bege_config", "bege_chirp", "bege_tail", "bege_search_opts", "bege_batch_entry",
           "bege_serve_config", "bege_serve_info"]


def test_header_is_c_and_binding_layouts_match(tmp_path):
    """The header compiles as plain C11 (gcc, -Wall -Werror), and every
    struct's size and field offsets in C equal the ctypes binding's."""
    import shutil
    import subprocess
    from paper_1708_01609_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bege.h"', "int main(void) {"]
    for name in STRUCTS:
        st = getattr(binding, name)
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-I",
                        os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for line in out.splitlines():
        name, key, value = line.split()
        got[(name, key)] = int(value)
    for name in STRUCTS:
        st = getattr(binding, name)
        assert got[(name, "size")] == ctypes.sizeof(st), name
        for field, _ in st._fields_:
            assert got[(name, field)] == getattr(st, field).offset, (name, field)
