"""The C-ABI library: builds, loads without a GPU, exports every symbol that
include/xc.h declares, validates arguments on the host, and its triangular
block map (Sec. 4.2) round-trips exactly."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1107_4264_gb300 import build as engine_build
from paper_1107_4264_gb300 import xc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    engine_build.build()
    return xc.load()


def declared_functions():
    with open(os.path.join(ROOT, "include", "xc.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(xc_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(xc.EXPORTS) == names


def test_version_and_status_strings(lib):
    assert "sm_103a" in xc.xc_version()
    assert xc.status_string(xc.XC_OK) == "XC_OK"
    assert xc.status_string(xc.XC_ERR_TIMEOUT) == "XC_ERR_TIMEOUT"


@pytest.mark.parametrize("args,status", [
    ((0, 2, 8, 256, xc.XC_CI8), xc.XC_ERR_INVALID_ARG),
    ((16, 3, 8, 256, xc.XC_CI8), xc.XC_ERR_INVALID_ARG),
    ((16, 2, 0, 256, xc.XC_CI8), xc.XC_ERR_INVALID_ARG),
    ((16, 2, 8, 0, xc.XC_CI8), xc.XC_ERR_INVALID_ARG),
    ((16, 2, 8, 256, 7), xc.XC_ERR_INVALID_ARG),
    ((16, 2, 8, xc.XC_CI8_MAX_NTIME + 1, xc.XC_CI8), xc.XC_ERR_OVERFLOW_RISK),
    ((16, 2, 70000, 256, xc.XC_CI8), xc.XC_ERR_UNSUPPORTED),
])
def test_create_rejects_bad_arguments(lib, args, status):
    h = lib.xc_create(*args)
    assert not h
    assert lib.xc_last_error() == status
    assert lib.xc_last_error_message()


def test_null_handle_calls(lib):
    assert lib.xc_correlate(None, None, None, None) == xc.XC_ERR_INVALID_ARG
    assert lib.xc_correlate_stream(None, None, 1, None, None, None) == xc.XC_ERR_INVALID_ARG
    assert lib.xc_set_option(None, xc.XC_OPT_ENGINE, 0) == xc.XC_ERR_INVALID_ARG
    assert lib.xc_synchronize(None, None) == xc.XC_ERR_INVALID_ARG
    assert lib.xc_correlate_backward(None, None, None, None, None) == xc.XC_ERR_INVALID_ARG
    assert lib.xc_input_bytes(None) == 0
    lib.xc_destroy(None)  # NULL-safe


# Fake, 16-byte aligned addresses: every case below is rejected by the host-side
# argument checks before any device call, so nothing is dereferenced.
_IN, _OUT, _TAPS = 0x10000, 0x20000, 0x30000


@pytest.mark.parametrize("args,status", [
    ((None, xc.XC_CI8, 4, 2, 64, 8, 1.0, _OUT, xc.XC_CF16, None), xc.XC_ERR_INVALID_ARG),
    ((_IN, xc.XC_CI8, 4, 2, 64, 8, 1.0, None, xc.XC_CF16, None), xc.XC_ERR_INVALID_ARG),
    ((_IN, xc.XC_CI8, 0, 2, 64, 8, 1.0, _OUT, xc.XC_CF16, None), xc.XC_ERR_INVALID_ARG),
    ((_IN, xc.XC_CI8, 4, 3, 64, 8, 1.0, _OUT, xc.XC_CF16, None), xc.XC_ERR_INVALID_ARG),
    ((_IN, xc.XC_CI8, 4, 2, 64, 0, 1.0, _OUT, xc.XC_CF16, None), xc.XC_ERR_INVALID_ARG),
    ((_IN, 9, 4, 2, 64, 8, 1.0, _OUT, xc.XC_CF16, None), xc.XC_ERR_INVALID_ARG),
    ((_IN, xc.XC_CI8, 4, 2, 64, 8, 1.0, _OUT, 9, None), xc.XC_ERR_INVALID_ARG),
    ((_IN, xc.XC_CI8, 4, 2, 48, 8, 1.0, _OUT, xc.XC_CF16, None), xc.XC_ERR_UNSUPPORTED),
    ((_IN, xc.XC_CI8, 4, 2, 8, 8, 1.0, _OUT, xc.XC_CF16, None), xc.XC_ERR_UNSUPPORTED),
    ((_IN, xc.XC_CI8, 4, 2, 8192, 8, 1.0, _OUT, xc.XC_CF16, None), xc.XC_ERR_UNSUPPORTED),
    ((_IN, xc.XC_CI8, 2 ** 22, 2, 4096, 1, 1.0, _OUT, xc.XC_CF16, None), xc.XC_ERR_UNSUPPORTED),
    ((_IN + 4, xc.XC_CI8, 4, 2, 64, 8, 1.0, _OUT, xc.XC_CF16, None), xc.XC_ERR_ALIGNMENT),
    ((_IN, xc.XC_CI8, 4, 2, 64, 8, 1.0, _OUT + 8, xc.XC_CF16, None), xc.XC_ERR_ALIGNMENT),
], ids=["null_in", "null_out", "no_station", "npol3", "no_block", "in_type", "out_type",
        "nchan48", "nchan8", "nchan8192", "too_many_inputs", "in_misaligned", "out_misaligned"])
def test_channelize_rejects_bad_arguments(lib, args, status):
    assert lib.xc_channelize(*args) == status
    assert lib.xc_last_error() == status
    assert lib.xc_last_error_message()


@pytest.mark.parametrize("taps,ntaps,nblock,status", [
    (None, 4, 8, xc.XC_ERR_INVALID_ARG),    # no taps
    (_TAPS, 0, 8, xc.XC_ERR_INVALID_ARG),   # no tap
    (_TAPS, 9, 8, xc.XC_ERR_INVALID_ARG),   # more taps than blocks
    (_TAPS, 65, 100, xc.XC_ERR_INVALID_ARG),  # above 64 taps
    (_TAPS + 4, 4, 8, xc.XC_ERR_ALIGNMENT),
], ids=["null_taps", "zero_taps", "taps_gt_blocks", "taps_gt_64", "taps_misaligned"])
def test_channelize_pfb_rejects_bad_arguments(lib, taps, ntaps, nblock, status):
    st = lib.xc_channelize_pfb(_IN, xc.XC_CI8, 4, 2, 64, nblock, taps, ntaps, 1.0, _OUT,
                               xc.XC_CF16, None)
    assert st == status
    assert lib.xc_last_error() == status


def test_channels_packed_rule(lib):
    """The packing decision: k = the largest divisor of F with k n <= 128 for
    n = N P <= 64 inputs, else 1 (restated here from its documentation)."""
    def rule(N, P, F):
        n = N * P
        if n > 64:
            return 1
        return max(k for k in range(1, 128 // n + 1) if F % k == 0)
    for N in (1, 2, 3, 5, 8, 16, 24, 32, 33, 64, 200):
        for P in (1, 2):
            for F in (1, 2, 3, 7, 8, 12, 60, 64, 1024, 65535, 65528):
                assert lib.xc_channels_packed(N, P, F) == rule(N, P, F), (N, P, F)
    assert lib.xc_channels_packed(16, 2, 1024) == 4
    assert lib.xc_channels_packed(256, 2, 1024) == 1
    assert lib.xc_channels_packed(0, 2, 8) == 0
    # sizes xc_create rejects give 0: npol outside {1, 2}, more than 2^30 rows
    for P in (0, 3, 4, -1):
        assert lib.xc_channels_packed(16, P, 8) == 0, P
    assert lib.xc_channels_packed(2 ** 28, 2, 8) == 1  # 2^30 rows: accepted
    assert lib.xc_channels_packed(2 ** 28 + 1, 2, 8) == 0
    assert lib.xc_channels_packed(2 ** 31 - 1, 2, 8) == 0  # 2 P N would overflow int


def test_small_engine_channels_rule(lib):
    """The small-array engine's reach: 128 / W channels per tile for
    W = 2 N P in {16, 32, 64, 128}, one channel of two tiles for W = 256,
    else 0 (restated from its documentation)."""
    for N in range(0, 160):
        for P in (-1, 0, 1, 2, 3):
            W = 2 * N * P
            want = (128 // W if W <= 128 else 1) if P in (1, 2) and W in (16, 32, 64, 128, 256) else 0
            assert lib.xc_small_engine_channels(N, P) == want, (N, P)
    assert lib.xc_small_engine_channels(16, 2) == 2
    assert lib.xc_small_engine_channels(64, 2) == 1 and lib.xc_small_engine_channels(128, 1) == 1
    assert lib.xc_small_engine_channels(2 ** 31 - 1, 2) == 0


def test_tri_map_round_trip_exhaustive(lib):
    # every block of the lower triangle up to 4000 block rows (8e6 blocks)
    n = 4000
    by = np.repeat(np.arange(n, dtype=np.int64), np.arange(1, n + 1))
    bx = np.arange(len(by), dtype=np.int64) - by * (by + 1) // 2
    g = np.arange(len(by), dtype=np.int64)
    assert (bx >= 0).all() and (bx <= by).all()
    # forward map through the library on a sample, inverse on a dense prefix
    for i in list(range(0, 20000)) + list(range(len(g) - 2000, len(g))):
        assert lib.xc_tri_index(int(bx[i]), int(by[i])) == g[i]
        assert xc.xc_tri_coords(int(g[i])) == (int(bx[i]), int(by[i]))


def test_tri_map_boundaries(lib):
    # first and last block of every row near 2^31 blocks, where a float
    # square root without the integer correction can pick the wrong row
    for y in list(range(0, 200)) + [65535, 65536, 92681, 92682, 2 ** 20, 3_000_000]:
        first = y * (y + 1) // 2
        assert xc.xc_tri_coords(first) == (0, y)
        assert xc.xc_tri_coords(first + y) == (y, y)
        if y:
            assert xc.xc_tri_coords(first - 1) == (y - 1, y - 1)
