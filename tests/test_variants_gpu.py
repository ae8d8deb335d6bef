"""Every compiled configuration of the streaming decoder (codewords per
thread, threads, stages, in-place output) is bit-exact against the oracle, and
the autotuner picks one of them without changing any result."""
import numpy as np
import pytest

import oracle
from paper_1412_6862_gb300 import hd
from tests import gpu_cases as gc

pytestmark = pytest.mark.gpu

ALL_N = [7, 15, 31, 63, 127, 255]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_6862_gb300 import build
    build.build()
    hd.lib()
    yield
    for n in ALL_N:
        for syn in (0, 1, 2):
            hd.hd_variant_select(n, syn, -1)


def _cases():
    out = []
    for n in ALL_N:
        for syn in (hd.SYN_NONE, hd.SYN_U8, hd.SYN_U16):
            out.append((n, syn))
    return out


@pytest.mark.parametrize("n,syn", _cases())
def test_every_variant_matches_oracle(n, syn):
    import torch
    cnt = hd.hd_variant_count(n, syn)
    assert cnt >= 1
    infos = [hd.hd_variant_info_get(n, syn, i) for i in range(cnt)]
    # several chunks of the largest configuration plus a ragged tail
    N = 3 * max(i["chunk_codewords"] for i in infos) + 1237
    stream, _, _ = gc.received_stream(n, N, seed=n * 7 + syn, p1=0.2, p2=0.02)
    exp = gc.expected(stream, n, N, syn)
    d_in = gc.to_device(stream)
    try:
        for i, info in enumerate(infos):
            assert info["blocks_per_sm"] >= 1, info
            hd.hd_variant_select(n, syn, i)
            assert hd.hd_variant_current(n, syn)["index"] == i
            got = hd.decode(d_in, n, N, syn_type=syn)
            torch.cuda.synchronize()
            try:
                gc.assert_same(got, exp, n, N, syn)
            except AssertionError as e:
                raise AssertionError(f"variant {info}: {e}") from None
    finally:
        hd.hd_variant_select(n, syn, -1)
    assert hd.hd_device_status() == 0


@pytest.mark.parametrize("n", [15, 63, 255])
def test_autotune_picks_a_variant_and_keeps_results(n):
    import torch
    syn = hd.SYN_U8 if n < 255 else hd.SYN_U16
    info = hd.hd_autotune(n, syn, 1 << 20, reps=3)
    assert info["measured_us"] > 0 and info["n"] == n
    assert hd.hd_variant_current(n, syn)["index"] == info["index"]
    N = 200000
    stream, _, _ = gc.received_stream(n, N, seed=3)
    exp = gc.expected(stream, n, N, syn)
    got = hd.decode(gc.to_device(stream), n, N, syn_type=syn)
    torch.cuda.synchronize()
    gc.assert_same(got, exp, n, N, syn)
    hd.hd_variant_select(n, syn, -1)
