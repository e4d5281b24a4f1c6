"""CPU checks of the batch tuner's cache: the key that names a batch and the
lookup of a tuning file (host-side helpers of the C ABI, no device work)."""
import pytest

from paper_1107_4264_gb300 import build as engine_build
from paper_1107_4264_gb300 import xc


@pytest.fixture(scope="module")
def lib():
    engine_build.build()
    return xc.load()


def test_key_names_sizes_order_npol_dtype_and_version(lib):
    k = xc.xc_batch_cache_key([32, 1024], [64, 96], [256, 8192], 2, xc.XC_CI8)
    assert k.startswith(xc.xc_version() + "|")
    assert k.endswith("|npol=2|dtype=0|32:64:256,1024:96:8192")
    # every field changes the key; subarray order matters (it is the batch's own order)
    others = [xc.xc_batch_cache_key([1024, 32], [96, 64], [8192, 256], 2, xc.XC_CI8),
              xc.xc_batch_cache_key([32, 1024], [64, 96], [256, 8192], 1, xc.XC_CI8),
              xc.xc_batch_cache_key([32, 1024], [64, 96], [256, 8193], 2, xc.XC_CI8),
              xc.xc_batch_cache_key([32, 1024], [64, 96], [256, 8192], 2, xc.XC_CF16)]
    assert len(set(others + [k])) == 5


def test_key_rejects_bad_arguments(lib):
    import ctypes
    arr = ctypes.c_int * 1
    buf = ctypes.create_string_buffer(8)
    # too small a buffer, no subarray, too many subarrays
    assert lib.xc_batch_cache_key(1, arr(16), arr(8), arr(64), 2, 0, buf, 8) == -1
    assert lib.xc_batch_cache_key(0, arr(16), arr(8), arr(64), 2, 0, buf, 8) == -1
    big = ctypes.c_int * 9
    assert lib.xc_batch_cache_key(9, big(*[1] * 9), big(*[1] * 9), big(*[1] * 9), 2, 0,
                                  ctypes.create_string_buffer(512), 512) == -1


def test_lookup_last_line_of_the_key_wins(lib, tmp_path):
    key = xc.xc_batch_cache_key([64, 200], [8, 16], [512, 1000], 2, xc.XC_CI8)
    other = xc.xc_batch_cache_key([64, 201], [8, 16], [512, 1000], 2, xc.XC_CI8)
    path = tmp_path / "tune.txt"
    assert xc.xc_batch_cache_lookup(str(path), key) == -1  # no file
    path.write_text("\n".join([
        "%s\t%d\t%.3f" % (key, 5, 1.25),
        "%s\t%d\t%.3f" % (other, 7, 0.5),
        "garbage line",
        "%sX\t%d\t1.0" % (key, 9),             # a longer key is another key
        "%s\t%d\t1.0" % (key, 99),             # candidate out of range: ignored
        "%s\t%d\t%.3f" % (key, 14, 1.1),
    ]) + "\n")
    assert xc.xc_batch_cache_lookup(str(path), key) == 14
    assert xc.xc_batch_cache_lookup(str(path), other) == 7
    assert xc.xc_batch_cache_lookup(str(path), "no such key") == -1
