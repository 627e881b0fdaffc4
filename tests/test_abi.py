"""The C-ABI library: it loads, exports every declared entry point, and its
host-side argument checks and segment arithmetic behave (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_1407_6915_gb300 as fs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b((?:fftseg|fftsrv)_\w+)\s*\(", text, flags=re.M):
                names.add(m.group(1))
    return names


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1407_6915_gb300 import build
    build.build()


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert {"fftseg_plan_create", "fftseg_exec", "fftseg_stream", "fftsrv_submit", "fftsrv_poll"} <= names
    L = ctypes.CDLL(fs.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def _create(n, batch=1, direction=fs.FORWARD, norm=fs.NORM_NONE, prec=fs.PREC_FP32, out=fs.OUT_COMPLEX):
    h = ctypes.c_void_p()
    rc = fs.lib().fftseg_plan_create(ctypes.byref(h), n, batch, direction, norm, prec, out, 0)
    return rc, h


@pytest.mark.parametrize("n", [0, 1, (1 << 23) + 1, (1 << 24) + 1, 1 << 25])
def test_plan_rejects_bad_lengths(n):
    # powers of two up to 2^24, other lengths (Bluestein) up to 2^23
    rc, h = _create(n)
    assert rc == fs.E_UNSUPPORTED and not h.value
    assert "outside" in fs.last_error()


def test_other_lengths_are_fp32_only():
    rc, h = _create(1000, prec=fs.PREC_TC_FP16)
    assert rc == fs.E_UNSUPPORTED and not h.value


@pytest.mark.parametrize("kw", [dict(batch=0), dict(direction=0), dict(direction=2), dict(norm=7),
                                dict(prec=9), dict(out=3)])
def test_plan_rejects_bad_arguments(kw):
    rc, h = _create(1024, **kw)
    assert rc == fs.E_INVALID and not h.value and fs.last_error()


def test_null_arguments_are_errors_not_crashes():
    L = fs.lib()
    assert L.fftseg_plan_create(None, 1024, 1, -1, 0, 0, 0, 0) == fs.E_INVALID
    assert L.fftseg_exec(None, None, None, None) == fs.E_INVALID
    assert L.fftseg_exec_n(None, None, None, 1, None) == fs.E_INVALID
    assert L.fftseg_plan_destroy(None) == fs.E_INVALID
    committed = ctypes.c_int64(-1)
    assert L.fftseg_stream(None, None, None, None, None, 0, 0, 0, ctypes.byref(committed)) == fs.E_INVALID
    assert L.fftseg_plan_info(None, None) == fs.E_INVALID
    assert L.fftseg_stream_phases(None, None) == fs.E_INVALID
    assert L.fftseg_exec_host(None, 0, None, None, 1, 0) == fs.E_INVALID
    assert L.fftseg_autotune(1024, 1, 0, 0, None, None) == fs.E_INVALID
    flags = ctypes.c_uint(0)
    assert L.fftseg_autotune(1000, 1, 0, 0, ctypes.byref(flags), None) == fs.E_UNSUPPORTED
    assert L.fftseg_autotune(1024, 0, 0, 0, ctypes.byref(flags), None) == fs.E_INVALID
    assert isinstance(fs.launch_count(), int)


def test_binding_constants_match_the_header():
    text = open(os.path.join(ROOT, "include", "fftseg.h")).read()
    defines = {m.group(1): int(m.group(2), 16) for m in
               re.finditer(r"#define\s+FFTSEG_((?:FLAG|FILE)_\w+)\s+(0x[0-9a-fA-F]+)u", text)}
    assert defines, "no flag defines found"
    for name, value in defines.items():
        assert getattr(fs, name) == value, name
    for name in ("OK", "E_INVALID", "E_NOMEM", "E_CUDA", "E_IO", "E_PARTIAL", "E_TIMEOUT", "E_UNSUPPORTED"):
        m = re.search(r"FFTSEG_%s\s*=\s*(-?\d+)" % name, text)
        assert m and int(m.group(1)) == getattr(fs, name), name
    assert fs.FLAG_CLUSTER_LOG2(3) == 3 << 8


def test_paper_record_arithmetic():
    # Sec. III: 1024-point single-precision records are 4096 bytes; a 1 TB file
    # holds 268,435,456 of them; 512 MB blocks give 2,048 map tasks.
    g = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "paper_record_arithmetic.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            g[k] = int(v)
    n, sb = g["fft_size"], g["sample_bytes"]
    assert fs.segment_offset(1, n, sb) == g["record_bytes"]
    assert fs.segment_count(g["file_bytes"], n, sb) == (g["records_per_file"], 0)
    assert fs.segment_count(g["file_bytes"], g["block_bytes"] // sb, sb) == (g["blocks_per_file"], 0)
    # the library's own sample is complex64 (8 bytes): segment s starts at s*n*8
    assert fs.segment_offset(5, 1024) == 5 * 8192
    assert fs.segment_count(3 * 8192 + 100, 1024) == (3, 100)
