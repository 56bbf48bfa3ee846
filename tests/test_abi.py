"""The C-ABI library loads and exports every symbol include/pivco.h declares
(CPU only: no compute call is made here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pivco.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pivco_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2606_05765_gb300 import build as B
    path = B.build()
    return path


def test_header_declares_calls():
    names = declared_functions()
    for core in ["pivco_histogram", "pivco_code_lengths", "pivco_build_layout", "pivco_encode_blocks",
                 "pivco_decode_blocks", "pivco_ans_encode_blocks", "pivco_exclusive_scan"]:
        assert core in names


def test_library_exports_every_declared_symbol(built_lib):
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pivco_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_reports(built_lib):
    import paper_2606_05765_gb300 as P
    assert "PVC1" in P.version()
    assert P.layout_bytes() >= 4096
    assert P.scan_workspace_size(1000) >= 16
    assert P.decode_plan_bytes(10) % 256 == 0


def test_ans_tables_match_oracle(built_lib, oracle):
    """The library's own static ANS tables equal the oracle's (Sec. 5.2)."""
    import numpy as np
    import paper_2606_05765_gb300 as P
    fq, cf = P.ans_tables()
    for t in range(50, 100):
        assert fq[t - 50] == oracle.fse_h_q16(t)
        assert np.array_equal(cf[t - 50], oracle.ans_class_freqs(t))


def test_host_argument_errors(built_lib):
    """Host-side argument checks return an error without touching the GPU."""
    import ctypes as C
    import paper_2606_05765_gb300 as P
    L = P.lib()
    assert L.pivco_code_lengths(None, 1, 0, None, None, None) == P.ERR_INVALID_ARG
    assert L.pivco_code_lengths(None, 1, 16, None, None, None) == P.ERR_INVALID_ARG
    assert L.pivco_histogram(None, None, -1, None, None) == P.ERR_INVALID_ARG
    bad = P.params()
    bad.ans_skew_den = 0
    assert L.pivco_build_layout(None, None, 0, C.byref(bad), None, None, None, None) == P.ERR_INVALID_ARG
    assert L.pivco_decode_blocks(None, None, -1, None, None, None, 0, None, None) == P.ERR_INVALID_ARG


def test_tuning_validation(built_lib):
    """Host-side checks of the decode tuning (no device work)."""
    import paper_2606_05765_gb300 as P
    try:
        for bad in [(65536, 512, 0), (65536, 100, 0), (100, 128, 0), (65536, 128, 33), ((1 << 20) + 128, 128, 0)]:
            with pytest.raises(P.PivcoError):
                P.set_tuning(*bad)
        P.set_tuning(16384, 256, 2)
        t = P.get_tuning()
        assert (t.tile_max, t.dir_bits, t.ctas_per_sm) == (16384, 256, 2)
    finally:
        P.set_tuning()
    t = P.get_tuning()
    assert (t.tile_max, t.dir_bits, t.ctas_per_sm) == (1 << 20, 128, 0)


def test_host_codec_and_plan_argument_errors(built_lib):
    """The host-buffer codec and the one-launch plan reject bad arguments on
    the host, before any CUDA call (so this runs without a GPU)."""
    import ctypes as C
    import numpy as np
    import paper_2606_05765_gb300 as P
    L = P.lib()
    prm = P.params()
    off = np.array([0, 10, 30], np.uint64)
    h = C.c_void_p()
    p_off = C.c_void_p(off.ctypes.data)
    assert L.pivco_host_codec_create(p_off, 2, C.byref(prm), 0, C.byref(h)) == P.ERR_INVALID_ARG   # no pieces
    assert L.pivco_host_codec_create(p_off, -1, C.byref(prm), 4, C.byref(h)) == P.ERR_INVALID_ARG
    assert L.pivco_host_codec_create(None, 2, C.byref(prm), 4, C.byref(h)) == P.ERR_INVALID_ARG
    assert L.pivco_host_codec_create(p_off, 2, None, 4, C.byref(h)) == P.ERR_INVALID_ARG
    bad_off = np.array([0, 10, 5], np.uint64)                                                   # decreasing
    assert L.pivco_host_codec_create(C.c_void_p(bad_off.ctypes.data), 2, C.byref(prm), 4, C.byref(h)) == \
        P.ERR_INVALID_ARG
    shifted = np.array([3, 10, 30], np.uint64)                                                  # must start at 0
    assert L.pivco_host_codec_create(C.c_void_p(shifted.ctypes.data), 2, C.byref(prm), 4, C.byref(h)) == \
        P.ERR_INVALID_ARG
    bad = P.params()
    bad.max_len = 16
    assert L.pivco_host_codec_create(p_off, 2, C.byref(bad), 4, C.byref(h)) == P.ERR_INVALID_ARG
    assert not h.value
    assert L.pivco_host_compress(None, None, None, 0, None, None) == P.ERR_INVALID_ARG
    assert L.pivco_host_decompress(None, None, None, None, None) == P.ERR_INVALID_ARG
    assert L.pivco_host_codec_destroy(None) == P.ERR_INVALID_ARG
    assert L.pivco_host_codec_comp_capacity(None) == 0
    # the plan: missing buffers, bad parameters, a layout buffer off a 16-byte boundary
    assert L.pivco_plan_blocks(None, None, 1, C.byref(prm), None, None, None, None, None, None, None) == \
        P.ERR_INVALID_ARG
    assert L.pivco_plan_blocks(None, None, 0, C.byref(bad), None, None, None, None, None, None, None) == \
        P.ERR_INVALID_ARG
    fake = C.c_void_p(0x1000)
    odd = C.c_void_p(0x1008)
    assert L.pivco_plan_blocks(fake, fake, 1, C.byref(prm), fake, fake, fake, odd, fake, fake, None) == \
        P.ERR_INVALID_ARG
    assert L.pivco_encode_blocks(fake, fake, 1, odd, fake, fake, fake, fake, None) == P.ERR_INVALID_ARG
