"""hd_decode_batch_noalloc, the batched decode that allocates nothing, against
the allocating entry point hd_decode_batch and against the CPU oracle.

Some callers cannot allocate device memory: a process that budgets all device
memory up front, an application whose allocator hooks forbid allocations from
inside libraries, or a latency-critical receive path where an allocation could
stall or fail.  For them the library keeps the batch tile table in a fixed 1 MiB
device array.  These tests check that two calls in a row give bit-exactly the
data bits, syndromes and error counts of hd_decode_batch and of the oracle,
and that batches beyond the array's limits are refused.

The file name sorts last, so a run that stops at the first failure has already
run every other test.
"""
import numpy as np
import pytest

import oracle
from paper_1412_6862_gb300 import hd, synth
from tests import gpu_cases as gc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_6862_gb300 import build
    build.build()
    hd.lib()


def _packets(num, seed):
    """Mixed-n packets with mixed lengths and syndrome types, plus a second set
    of output buffers for the reference decode, and the oracle's decode of
    every packet."""
    import torch
    lengths = (3, 7, 15, 31, 63, 127, 255)
    ns = synth.below(seed, 21, 0, num, len(lengths))
    lens = synth.below(seed, 22, 0, num, 30000)
    stypes = synth.below(seed, 23, 0, num, 3)
    mine, ref, want = [], [], []
    for j in range(num):
        n = lengths[int(ns[j])]
        N = 0 if j % 31 == 7 else int(lens[j])
        st = int(stypes[j])
        m, k = hd.code_params(n)
        stream, _, _ = gc.received_stream(n, N, seed=seed * 100 + j, p1=0.1, p2=0.02)
        want.append(oracle.decode(stream, n, N, syn_type=st) if N else
                    (np.zeros(0, np.uint32), np.zeros(0, np.uint8 if st == 1 else np.uint16) if st else None, 0))
        d_in = gc.to_device(stream)
        for dst in (mine, ref):
            out = torch.full((max(1, hd.words_for(N * k)),), -1, dtype=torch.int32, device="cuda")
            syn = None
            if st != hd.SYN_NONE:
                syn = torch.full((max(1, N),), 0x3C, dtype=torch.uint8 if st == 1 else torch.int16, device="cuda")
            dst.append((d_in, out, syn, N, n, st))
    return mine, ref, want


def _table(pkts):
    return hd.packet_table([(hd._ptr(a), hd._ptr(b), hd._ptr(c), N, n, st) for a, b, c, N, n, st in pkts])


def _host(pkts, err):
    res = []
    for (d_in, out, syn, N, n, st) in pkts:
        m, k = hd.code_params(n)
        o = gc.host_u32(out)[:hd.words_for(N * k)]
        s = None if syn is None else syn.cpu().numpy()[:N]
        res.append((o, s))
    return res, err.cpu().numpy().copy()


def test_noalloc_matches_allocating_batch_two_calls():
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    mine, ref, want = _packets(150, seed=3)
    num = len(mine)
    err_ref = torch.full((num,), 9, dtype=torch.int64, device="cuda")
    assert hd.hd_decode_batch(_table(ref), num, err_ref.data_ptr(), stream) == hd.HD_OK
    torch.cuda.synchronize()
    expect, expect_err = _host(ref, err_ref)
    assert expect_err.sum() > 0

    table = _table(mine)
    assert hd.hd_batch_tiles(table, num) > 2 * 480  # several upload launches of the tile table
    err = torch.empty(num, dtype=torch.int64, device="cuda")
    for call in range(2):
        for (_, out, syn, _, _, _) in mine:  # stale results must not mask a failure
            out.fill_(-1)
            if syn is not None:
                syn.fill_(0x3C)
        err.fill_(123)
        assert hd.hd_decode_batch_noalloc(table, num, err.data_ptr(), stream) == hd.HD_OK
        torch.cuda.synchronize()
        got, got_err = _host(mine, err)
        assert np.array_equal(got_err, expect_err), f"call {call}: error counts differ"
        for j, ((go, gs), (eo, es), (wo, ws, we)) in enumerate(zip(got, expect, want)):
            assert np.array_equal(go, eo), f"call {call}, packet {j}: data bits differ"
            assert np.array_equal(go, wo), f"call {call}, packet {j}: data bits differ from the oracle"
            assert got_err[j] == we, f"call {call}, packet {j}: error count differs from the oracle"
            if es is not None:
                assert np.array_equal(gs, es), f"call {call}, packet {j}: syndromes differ"
                gs_typed = gs.view(np.uint16) if gs.dtype != np.uint8 else gs
                assert np.array_equal(gs_typed, ws), f"call {call}, packet {j}: syndromes differ from the oracle"
    assert hd.hd_device_status() == 0


def test_noalloc_refuses_batches_beyond_its_array():
    # rejected on the host before any device work; the pointers are never used
    too_many_packets = hd.packet_table([(16, 16, None, 1, 7, 0)] * 4097)
    assert hd.hd_decode_batch_noalloc(too_many_packets, 4097, None, None) == hd.HD_ERR_CAPACITY
    # n = 7 packs four 1024-codeword chunks per tile; the array holds 16,380 tiles
    too_many_tiles = hd.packet_table([(16, 16, None, 4096 * 16381, 7, 0)])
    assert hd.hd_decode_batch_noalloc(too_many_tiles, 1, None, None) == hd.HD_ERR_CAPACITY
    bad_n = hd.packet_table([(16, 16, None, 10, 9, 0)])
    assert hd.hd_decode_batch_noalloc(bad_n, 1, None, None) == hd.HD_ERR_INVALID_N
