"""GPU parity: libhd's decoder against the CPU oracle, bit-exact on data bits,
syndromes and err_count, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1412_6862_gb300 import hd
from tests import gpu_cases as gc

pytestmark = pytest.mark.gpu

ALL_N = [3, 7, 15, 31, 63, 127, 255]
SYN = {"none": hd.SYN_NONE, "u8": hd.SYN_U8, "u16": hd.SYN_U16}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_6862_gb300 import build
    build.build()
    hd.lib()


def run_case(n, N, syn_type, seed=0, p1=0.1, p2=0.01):
    import torch
    stream, _, _ = gc.received_stream(n, N, seed=seed, p1=p1, p2=p2)
    exp = gc.expected(stream, n, N, syn_type)
    d_in = gc.to_device(stream)
    got = hd.decode(d_in, n, N, syn_type=syn_type)
    torch.cuda.synchronize()
    gc.assert_same(got, exp, n, N, syn_type)
    return got


# Sizes that span several streaming chunks (32*T codewords, T up to 256)
# plus ragged tails that end inside a warp tile and inside a word.
@pytest.mark.parametrize("n", ALL_N)
@pytest.mark.parametrize("N", [1, 31, 33, 1000, 3 * 8192 + 1234, 70001])
def test_parity_small(n, N):
    run_case(n, N, hd.SYN_U8 if n < 127 else hd.SYN_U16, seed=N)


@pytest.mark.parametrize("n", ALL_N)
@pytest.mark.parametrize("syn", ["none", "u8", "u16"])
def test_parity_syndrome_types(n, syn):
    run_case(n, 5 * 8192 + 77, SYN[syn], seed=n)


@pytest.mark.parametrize("n", [15, 31, 63])
@pytest.mark.parametrize("p1", [0.01, 0.1, 0.5])
def test_parity_error_rates(n, p1):
    """The single-n sweep's error rates, with 2-bit errors (miscorrection)."""
    run_case(n, 200003, hd.SYN_U8, seed=int(p1 * 100), p1=p1, p2=0.01)


def test_zero_codewords_zeroes_err_count():
    import torch
    err = torch.full((1,), 12345, dtype=torch.int64, device="cuda")
    rc = hd.hd_decode(None, 0, 15, 0, None, None, hd.SYN_NONE, err.data_ptr(),
                      torch.cuda.current_stream().cuda_stream)
    assert rc == hd.HD_OK
    assert int(err.item()) == 0


def test_err_count_overwritten_not_accumulated():
    import torch
    n, N = 31, 50000
    stream, _, ev = gc.received_stream(n, N, seed=4)
    d_in = gc.to_device(stream)
    err = torch.full((1,), 999, dtype=torch.int64, device="cuda")
    for _ in range(2):
        hd.decode(d_in, n, N, err_count=err)
    assert int(err.item()) == ev.num_events


def test_output_pad_bits_zero_and_no_overrun():
    """The last output word's pad bits are 0 and nothing past it is written."""
    import torch
    for n in ALL_N:
        k = n - gc.M_OF[n]
        N = 8192 * 2 + 3
        stream, _, _ = gc.received_stream(n, N, seed=n)
        nw = (N * k + 31) // 32
        out = torch.full((nw + 8,), -1, dtype=torch.int32, device="cuda")
        hd.decode(gc.to_device(stream), n, N, out=out)
        o = gc.host_u32(out)
        tail = (N * k) % 32
        if tail:
            assert int(o[nw - 1]) >> tail == 0
        assert (o[nw:] == 0xFFFFFFFF).all()


def test_input_pad_bits_ignored():
    import torch
    n, N = 15, 8192 + 5
    stream, _, _ = gc.received_stream(n, N, seed=1)
    dirty = stream.copy()
    if (N * n) % 32:
        dirty[-1] |= np.uint32((0xFFFFFFFF << ((N * n) % 32)) & 0xFFFFFFFF)
    a = hd.decode(gc.to_device(stream), n, N)
    b = hd.decode(gc.to_device(dirty), n, N)
    torch.cuda.synchronize()
    assert np.array_equal(gc.host_u32(a[0]), gc.host_u32(b[0]))


@pytest.mark.parametrize("n", ALL_N)
def test_encoder_matches_oracle(n):
    import torch
    for N in (1, 33, 8192 * 3 + 7):
        k = n - gc.M_OF[n]
        from paper_1412_6862_gb300 import synth
        data = synth.random_words(7, N * k)
        exp = oracle.encode(data, n, N)
        got = hd.encode(gc.to_device(data), n, N)
        torch.cuda.synchronize()
        assert np.array_equal(gc.host_u32(got)[:exp.size], exp), (n, N)


def test_device_status_clean():
    assert hd.hd_device_status() == 0


# Full sizes of the benchmark workloads, in the launch configuration the
# benchmark times, compared element by element with the threaded oracle.
FULL = [(7, 1 << 20, hd.SYN_U8), (15, 1 << 24, hd.SYN_U8), (31, 1 << 24, hd.SYN_U8),
        (63, 1 << 24, hd.SYN_U8), (127, 1 << 22, hd.SYN_U16), (255, 1 << 22, hd.SYN_U16)]


@pytest.mark.parametrize("n,N,syn", FULL)
def test_parity_full_size(n, N, syn):
    p1, p2 = {7: (0.1, 0.0), 127: (0.05, 0.005), 255: (0.05, 0.005)}.get(n, (0.1, 0.01))
    run_case(n, N, syn, seed=0, p1=p1, p2=p2)


def _streams_case(seed):
    import torch
    specs = [(63, 3 * 8192 + 5, hd.SYN_U8), (15, 70001, hd.SYN_U8), (255, 9001, hd.SYN_U16), (7, 1, hd.SYN_NONE),
             (31, 50000, hd.SYN_U16), (127, 4099, hd.SYN_U8), (3, 777, hd.SYN_U8), (31, 0, hd.SYN_U8)]
    jobs, bufs, exp = [], [], []
    for i, (n, N, st) in enumerate(specs):
        m, k = hd.code_params(n)
        stream, _, _ = gc.received_stream(n, N, seed=seed + i, p1=0.2, p2=0.02)
        exp.append(gc.expected(stream, n, N, st) if N else (np.zeros(0, np.uint32), None, 0))
        d_in = gc.to_device(stream)
        out = torch.full((max(1, hd.words_for(N * k)),), -1, dtype=torch.int32, device="cuda")
        syn = None if st == hd.SYN_NONE else torch.full((max(1, N),), 0x55, dtype=torch.uint8 if st == 1 else
                                                         torch.int16, device="cuda")
        err = torch.full((1,), 999, dtype=torch.int64, device="cuda")
        bufs.append((d_in, out, syn, err, n, N, st))
        jobs.append((d_in.data_ptr(), n, N, out.data_ptr(), None if syn is None else syn.data_ptr(), st,
                     err.data_ptr()))
    return hd.stream_jobs(jobs), bufs, exp


def _streams_check(bufs, exp):
    for (d_in, out, syn, err, n, N, st), (eo, es, ee) in zip(bufs, exp):
        if N == 0:
            assert int(err.item()) == 0
            continue
        gc.assert_same((out, syn, err), (eo, es, ee), n, N, st)


def test_decode_streams_matches_oracle_directly_and_in_a_graph():
    """Several streams of different n decoded concurrently (hd_decode_streams):
    every element equals the oracle's, called directly and replayed from a
    captured CUDA graph."""
    import torch
    jobs, bufs, exp = _streams_case(seed=500)
    rc = hd.hd_decode_streams(jobs, len(bufs), torch.cuda.current_stream().cuda_stream)
    assert rc == hd.HD_OK
    torch.cuda.synchronize()
    _streams_check(bufs, exp)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        assert hd.hd_decode_streams(jobs, len(bufs), s.cuda_stream) == hd.HD_OK
    for _ in range(2):
        for (d_in, out, syn, err, n, N, st) in bufs:
            out.fill_(-1)
            err.fill_(12345)
        g.replay()
        torch.cuda.synchronize()
        _streams_check(bufs, exp)
    assert hd.hd_device_status() == 0
