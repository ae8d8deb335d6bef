"""libhd.so builds for sm_103a, loads without a GPU, exports every function
that include/hd.h declares, and rejects bad arguments on the host before any
CUDA call."""
import ctypes
import shutil

import numpy as np

import pytest

from paper_1412_6862_gb300 import build as hd_build
from paper_1412_6862_gb300 import hd


@pytest.fixture(scope="module")
def lib():
    if shutil.which(hd_build.nvcc()) is None and not hd_build.up_to_date():
        pytest.skip("nvcc not available and libhd.so not built")
    hd_build.build()
    return hd.lib()


def test_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(hd.LIB_PATH)
    names = hd.header_functions()
    assert "hd_decode" in names
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, f"declared in include/hd.h but not exported: {missing}"
    # the binding describes every declared function and nothing else
    assert sorted(hd.SIGNATURES) == names


def test_variant_counts_host_only(lib):
    for n in (7, 15, 31, 63, 127, 255):
        for syn in (0, 1, 2):
            assert hd.hd_variant_count(n, syn) >= 1
    assert hd.lib().hd_variant_count(8, 0, None) in (hd.HD_ERR_NULL, hd.HD_ERR_INVALID_N)


def test_status_strings(lib):
    for code in range(9):
        assert hd.status_string(code).startswith("HD_")
    assert hd.hd_version() >= 100


def test_host_side_validation(lib):
    # invalid n
    assert hd.hd_decode(16, 8 * 4, 8, 4, 16, None, 0, None, None) == hd.HD_ERR_INVALID_N
    assert hd.hd_decode(16, 511, 511, 1, 16, None, 0, None, None) == hd.HD_ERR_INVALID_N
    # in_bits != n * num_codewords
    assert hd.hd_decode(16, 7 * 4 + 1, 7, 4, 16, None, 0, None, None) == hd.HD_ERR_SIZE
    # null pointers
    assert hd.hd_decode(None, 7 * 4, 7, 4, 16, None, 0, None, None) == hd.HD_ERR_NULL
    assert hd.hd_decode(16, 7 * 4, 7, 4, None, None, 0, None, None) == hd.HD_ERR_NULL
    assert hd.hd_decode(16, 7 * 4, 7, 4, 16, None, hd.SYN_U8, None, None) == hd.HD_ERR_NULL
    # alignment
    assert hd.hd_decode(20, 7 * 4, 7, 4, 16, None, 0, None, None) == hd.HD_ERR_ALIGN
    assert hd.hd_decode(16, 7 * 4, 7, 4, 24, None, 0, None, None) == hd.HD_ERR_ALIGN
    # bad syndrome type
    assert hd.hd_decode(16, 7 * 4, 7, 4, 16, None, 7, None, None) == hd.HD_ERR_INVALID_ARG
    # zero codewords without err_count touches nothing
    assert hd.hd_decode(None, 0, 7, 0, None, None, 0, None, None) == hd.HD_OK
    assert hd.hd_encode(16, 9, 4, 16, None) == hd.HD_ERR_INVALID_N
    assert hd.hd_encode(None, 7, 4, 16, None) == hd.HD_ERR_NULL
    assert hd.hd_encode(20, 7, 4, 16, None) == hd.HD_ERR_ALIGN


def test_no_launches_counted_for_rejected_calls(lib):
    before = hd.hd_launch_count()
    hd.hd_decode(16, 7 * 4 + 1, 7, 4, 16, None, 0, None, None)
    assert hd.hd_launch_count() == before


def test_plan_validation_host_only(lib):
    import ctypes
    bad_n = hd.packet_table([(16, 16, None, 10, 8, 0)])
    plan = ctypes.c_void_p()
    assert hd.lib().hd_plan_create(bad_n, 1, ctypes.byref(plan)) == hd.HD_ERR_INVALID_N
    misaligned = hd.packet_table([(16, 16, None, 10, 7, 0), (20, 16, None, 10, 7, 0)])
    assert hd.lib().hd_plan_create(misaligned, 2, ctypes.byref(plan)) == hd.HD_ERR_ALIGN
    null_in = hd.packet_table([(None, 16, None, 10, 15, 0)])
    assert hd.lib().hd_plan_create(null_in, 1, ctypes.byref(plan)) == hd.HD_ERR_NULL
    null_syn = hd.packet_table([(16, 16, None, 10, 15, 1)])
    assert hd.lib().hd_plan_create(null_syn, 1, ctypes.byref(plan)) == hd.HD_ERR_NULL
    assert hd.lib().hd_plan_create(None, 3, ctypes.byref(plan)) == hd.HD_ERR_NULL
    assert hd.lib().hd_decode_batch(bad_n, 1, None, None) == hd.HD_ERR_INVALID_N


def test_host_decode_validation_host_only(lib):
    import numpy as np
    z = np.zeros(8, np.uint32)
    assert hd.hd_decode_host(z.ctypes.data, 15 * 4, 14, 4, z.ctypes.data, None, 0, 0, 0)[0] == hd.HD_ERR_INVALID_N
    assert hd.hd_decode_host(z.ctypes.data, 15 * 4 + 1, 15, 4, z.ctypes.data, None, 0, 0, 0)[0] == hd.HD_ERR_SIZE
    assert hd.hd_decode_host(z.ctypes.data, 15 * 4, 15, 4, z.ctypes.data, None, 0, 100, 0)[0] == hd.HD_ERR_INVALID_ARG
    assert hd.hd_decode_host(z.ctypes.data, 15 * 4, 15, 4, z.ctypes.data, None, 0, 128, 9)[0] == hd.HD_ERR_INVALID_ARG
    assert hd.hd_decode_host(None, 15 * 4, 15, 4, z.ctypes.data, None, 0, 0, 0)[0] == hd.HD_ERR_NULL
    assert hd.hd_decode_host(z.ctypes.data, 15 * 4, 15, 4, z.ctypes.data, None, 1, 0, 0)[0] == hd.HD_ERR_NULL


def test_short_params_host_only(lib, oracle_mod):
    for n in list(range(3, 600)) + [1611, 8013, 16383, 16384, 32767]:
        assert hd.hd_short_params(n) == oracle_mod.short_params(n)
    for bad in (0, 1, 2, 32768, 1 << 20):
        with pytest.raises(hd.HDError):
            hd.hd_short_params(bad)


def test_segment_params_match_the_splitter_rule(lib, oracle_mod):
    """Sec. II: a packet of M bytes cut into t segments; each segment carries
    k = ceil(8M/t) data bits and the fewest checksum bits r with
    2^r >= k + r + 1 (brute force here), so n = k + r is a shortened length."""
    for M in list(range(1, 80)) + [400, 800, 1200, 1600, 2000, 4000]:
        for t in range(1, 9):
            if t > 8 * M:
                continue
            k = -(-8 * M // t)
            r = next(r for r in range(1, 40) if 2 ** r >= k + r + 1)
            if k + r < 3 or k + r > 32767:
                continue
            n, kk, rr = hd.hd_segment_params(M, t)
            assert (n, kk, rr) == (k + r, k, r), (M, t)
            assert oracle_mod.short_params(n) == (r, k)
    assert lib.hd_segment_params(100, 0, None, None, None) == hd.HD_ERR_INVALID_ARG
    assert lib.hd_segment_params(1, 9, None, None, None) == hd.HD_ERR_INVALID_ARG
    assert lib.hd_segment_params(5000, 1, None, None, None) == hd.HD_ERR_SIZE


def test_short_host_side_validation(lib):
    assert hd.hd_decode_short(16, 2 * 4, 2, 4, 16, None, 0, None, None, None) == hd.HD_ERR_INVALID_N
    assert hd.hd_decode_short(16, 32768, 32768, 1, 16, None, 0, None, None, None) == hd.HD_ERR_INVALID_N
    assert hd.hd_decode_short(16, 11 * 4 + 1, 11, 4, 16, None, 0, None, None, None) == hd.HD_ERR_SIZE
    assert hd.hd_decode_short(None, 11 * 4, 11, 4, 16, None, 0, None, None, None) == hd.HD_ERR_NULL
    assert hd.hd_decode_short(16, 11 * 4, 11, 4, None, None, 0, None, None, None) == hd.HD_ERR_NULL
    assert hd.hd_decode_short(16, 11 * 4, 11, 4, 16, None, hd.SYN_U16, None, None, None) == hd.HD_ERR_NULL
    assert hd.hd_decode_short(20, 11 * 4, 11, 4, 16, None, 0, None, None, None) == hd.HD_ERR_ALIGN
    assert hd.hd_decode_short(16, 11 * 4, 11, 4, 24, None, 0, None, None, None) == hd.HD_ERR_ALIGN
    assert hd.hd_decode_short(16, 300 * 4, 300, 4, 16, 32, hd.SYN_U8, None, None, None) == hd.HD_ERR_INVALID_ARG
    assert hd.hd_decode_short(16, 11 * 4, 11, 4, 16, 32, 5, None, None, None) == hd.HD_ERR_INVALID_ARG
    assert hd.hd_decode_short(None, 0, 11, 0, None, None, 0, None, None, None) == hd.HD_OK
    assert hd.hd_encode_short(16, 2, 4, 16, None) == hd.HD_ERR_INVALID_N
    assert hd.hd_encode_short(None, 11, 4, 16, None) == hd.HD_ERR_NULL
    assert hd.hd_encode_short(16, 11, 4, 20, None) == hd.HD_ERR_ALIGN
    assert hd.hd_short_variant_count() >= 1
    assert lib.hd_short_variant_select(hd.hd_short_variant_count()) == hd.HD_ERR_INVALID_ARG


def test_secded_host_side_validation(lib):
    assert hd.hd_decode_secded(16, 10 * 4, 9, 4, 16, None, 0, None, None, None) == hd.HD_ERR_INVALID_N
    assert hd.hd_decode_secded(16, 7 * 4, 7, 4, 16, None, 0, None, None, None) == hd.HD_ERR_SIZE  # needs 8 * 4
    assert hd.hd_decode_secded(None, 8 * 4, 7, 4, 16, None, 0, None, None, None) == hd.HD_ERR_NULL
    assert hd.hd_decode_secded(16, 8 * 4, 7, 4, None, None, 0, None, None, None) == hd.HD_ERR_NULL
    assert hd.hd_decode_secded(20, 8 * 4, 7, 4, 16, None, 0, None, None, None) == hd.HD_ERR_ALIGN
    assert hd.hd_decode_secded(16, 256 * 4, 255, 4, 16, 32, hd.SYN_U8, None, None, None) == hd.HD_ERR_INVALID_ARG
    assert hd.hd_decode_secded(16, 128 * 4, 127, 4, 16, None, hd.SYN_U8, None, None, None) == hd.HD_ERR_NULL
    assert hd.hd_decode_secded(None, 0, 63, 0, None, None, 0, None, None, None) == hd.HD_OK
    assert hd.hd_encode_secded(16, 9, 4, 16, None) == hd.HD_ERR_INVALID_N
    assert hd.hd_encode_secded(None, 7, 4, 16, None) == hd.HD_ERR_NULL


def test_host_batch_validation_host_only(lib):
    z = np.zeros(64, np.uint32)
    good = (z.ctypes.data, 15, 4, z.ctypes.data, None, 0)
    assert hd.hd_decode_host_batch([])[0] == hd.HD_OK
    assert hd.hd_decode_host_batch([good, (z.ctypes.data, 14, 4, z.ctypes.data, None, 0)])[0] == hd.HD_ERR_INVALID_N
    assert hd.hd_decode_host_batch([good], 100, 0)[0] == hd.HD_ERR_INVALID_ARG
    assert hd.hd_decode_host_batch([good], 0, 9)[0] == hd.HD_ERR_INVALID_ARG
    assert hd.hd_decode_host_batch([(None, 15, 4, z.ctypes.data, None, 0)])[0] == hd.HD_ERR_NULL
    assert hd.hd_decode_host_batch([(z.ctypes.data, 15, 4, z.ctypes.data, None, 1)])[0] == hd.HD_ERR_NULL
    assert lib.hd_decode_host_batch(None, 1, 0, 0) == hd.HD_ERR_NULL


def _tiles_model(n, N):
    # the batch plan's cut: whole chunks grouped into full tiles, then tails of
    # at most 1024 codewords (n = 3 is all tail)
    chunk = {3: 1024, 7: 1024, 15: 1024, 31: 1024, 63: 512, 127: 256, 255: 128}[n]
    per = {7: 4, 15: 2}.get(n, 1)
    full = 0 if n == 3 else N // chunk
    return -(-full // per) + -(-(N - full * chunk) // 1024)


def test_batch_tiles_host_only(lib):
    rng = np.random.default_rng(5)
    codes = (3, 7, 15, 31, 63, 127, 255)
    for trial in range(40):
        P = int(rng.integers(0, 50))
        rows = [(16, 16, None, int(rng.integers(0, 1 << int(rng.integers(0, 22)))), int(rng.choice(codes)), 0)
                for _ in range(P)]
        expected = sum(_tiles_model(n, N) for (_, _, _, N, n, _) in rows)
        assert hd.hd_batch_tiles(hd.packet_table(rows), P) == expected
    # worked cases: one chunk fewer or more changes the count as the rule says
    assert hd.hd_batch_tiles(hd.packet_table([(16, 16, None, 128 * 60, 255, 0)]), 1) == 60
    assert hd.hd_batch_tiles(hd.packet_table([(16, 16, None, 128 * 60 + 1, 255, 0)]), 1) == 61
    assert hd.hd_batch_tiles(hd.packet_table([(16, 16, None, 4096 * 3, 7, 0)]), 1) == 3
    assert hd.hd_batch_tiles(hd.packet_table([(16, 16, None, 0, 15, 0)]), 1) == 0
    import ctypes
    t = ctypes.c_uint64(0)
    assert hd.lib().hd_batch_tiles(hd.packet_table([(16, 16, None, 10, 8, 0)]), 1, ctypes.byref(t)) == \
        hd.HD_ERR_INVALID_N
    assert hd.lib().hd_batch_tiles(hd.packet_table([(16, 16, None, 10, 7, 3)]), 1, ctypes.byref(t)) == \
        hd.HD_ERR_INVALID_ARG
    assert hd.lib().hd_batch_tiles(hd.packet_table([(16, 16, None, (1 << 40) + 1, 7, 0)]), 1, ctypes.byref(t)) == \
        hd.HD_ERR_SIZE
    assert hd.lib().hd_batch_tiles(None, 2, ctypes.byref(t)) == hd.HD_ERR_NULL


def test_max_ctas_host_only(lib):
    assert hd.hd_get_max_ctas() == 0
    try:
        hd.hd_set_max_ctas(3)
        assert hd.hd_get_max_ctas() == 3
    finally:
        hd.hd_set_max_ctas(0)
    assert hd.hd_get_max_ctas() == 0


def test_secded_variants_host_only(lib):
    for n in (7, 15, 31, 63, 127, 255):
        for syn in (0, 1, 2):
            if syn == 1 and n == 255:
                continue
            # at least one arithmetic configuration, plus table ones for n = 7 and 15
            c = hd.hd_secded_variant_count(n, syn)
            infos = [hd.hd_secded_variant_info_get(n, syn, i) for i in range(c)]
            assert any(not i["table_lookup"] for i in infos)
            assert any(i["table_lookup"] for i in infos) == (n in (7, 15))
    assert hd.lib().hd_secded_variant_count(9, 0, None) in (hd.HD_ERR_NULL, hd.HD_ERR_INVALID_N)
    assert hd.lib().hd_secded_variant_select(9, 0, 0) == hd.HD_ERR_INVALID_N


def test_decode_streams_validation_host_only(lib):
    # rejected on the host before any device work; the pointers are never used
    assert hd.hd_decode_streams(None, 2, None) == hd.HD_ERR_NULL
    assert hd.hd_decode_streams(None, 0, None) == hd.HD_OK
    many = hd.stream_jobs([(16, 7, 32, 16, None, 0, None)] * 33)
    assert hd.hd_decode_streams(many, 33, None) == hd.HD_ERR_CAPACITY
    bad_n = hd.stream_jobs([(16, 7, 32, 16, None, 0, None), (16, 9, 32, 16, None, 0, None)])
    assert hd.hd_decode_streams(bad_n, 2, None) == hd.HD_ERR_INVALID_N
    unaligned = hd.stream_jobs([(20, 7, 32, 16, None, 0, None)])
    assert hd.hd_decode_streams(unaligned, 1, None) == hd.HD_ERR_ALIGN
    no_syn = hd.stream_jobs([(16, 7, 32, 16, None, 0, None)])
    no_syn[0].syn_type = hd.SYN_U8  # a syndrome type without a buffer
    assert hd.hd_decode_streams(no_syn, 1, None) == hd.HD_ERR_NULL
