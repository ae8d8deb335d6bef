"""Shortened codes on the GPU (hd_decode_short / hd_encode_short) against the
oracle, bit-exact: data bits, syndromes, the count of nonzero syndromes and
the count of detected (syndrome past n) segments.

Lengths cover the per-lane kernel (k < 64), the tiled kernel (k >= 64) and
the boundary between them, every full length, powers of two and their
neighbours, the paper's segment lengths (packets of 400..2000 bytes cut into
2..6 segments, Sec. IV-A) and the longest supported segment; stream lengths
span several tiles with ragged tails."""
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


def _received(n, N, seed, p1=0.3, p2=0.2):
    r, k = oracle.short_params(n)
    data = synth.random_words(seed, N * k)
    stream = oracle.encode_short(data, n, N) if N else np.zeros(0, np.uint32)
    ev = synth.error_events(seed + 7, n, N, p1=p1, p2=p2)
    synth.apply_errors(stream, ev)
    return stream, data, ev


def _check(n, N, syn_type, seed=0, p1=0.3, p2=0.2):
    import torch
    r, k = oracle.short_params(n)
    rx, _, ev = _received(n, N, seed, p1, p2)
    d_in = gc.to_device(rx, pad_words=4)
    out = torch.full((max(4, hd.words_for(N * k)),), -1, dtype=torch.int32, device="cuda")
    syn = None
    if syn_type != hd.SYN_NONE:
        syn = torch.full((max(16, N),), 0x77, dtype=torch.uint8 if syn_type == hd.SYN_U8 else torch.int16,
                         device="cuda")
    counts = torch.full((2,), 12345, dtype=torch.int64, device="cuda")
    hd.decode_short(d_in, n, N, syn_type, out=out, syndromes=syn, counts=counts)
    torch.cuda.synchronize()
    eo, es, ee, ed = oracle.decode_short(rx, n, N, syn_type if syn_type != hd.SYN_NONE else oracle.SYN_U16,
                                         threads=8)
    nw = hd.words_for(N * k)
    got = gc.host_u32(out)[:nw]
    if not np.array_equal(got, eo[:nw]):
        bad = np.nonzero(got != eo[:nw])[0]
        raise AssertionError(f"n={n} N={N}: {bad.size} output words differ, first {bad[0]} "
                             f"(gpu {got[bad[0]]:#010x} oracle {eo[bad[0]]:#010x})")
    if syn is not None:
        sg = syn.cpu().numpy()[:N]
        if syn_type == hd.SYN_U16:
            sg = sg.view(np.uint16)
        assert np.array_equal(sg, es[:N].astype(sg.dtype)), f"n={n} N={N}: syndromes differ"
    c = counts.cpu().numpy()
    assert (int(c[0]), int(c[1])) == (ee, ed), (n, N, c, ee, ed)
    assert hd.hd_device_status() == 0
    return ee, ed


CASES = [
    (3, 1000), (4, 777), (5, 1000), (6, 999), (11, 4099), (12, 3000), (20, 2000), (31, 1111), (33, 1500),
    (50, 999), (64, 1234), (70, 1000), (71, 1000), (72, 999), (100, 3001), (127, 2049), (128, 1500),
    (200, 1500), (255, 1025), (256, 1000), (300, 999), (545, 3000), (1078, 1000), (1611, 777), (2000, 500),
    (4095, 300), (4096, 300), (4097, 301), (8013, 300), (16383, 50), (16384, 41), (32767, 40),
]


@pytest.mark.parametrize("n,N", CASES)
def test_decode_short_u16(n, N):
    _check(n, N, hd.SYN_U16, seed=n)


@pytest.mark.parametrize("n,N", [c for c in CASES if c[0] <= 255])
def test_decode_short_u8(n, N):
    _check(n, N, hd.SYN_U8, seed=n + 1)


@pytest.mark.parametrize("n,N", [(11, 999), (545, 1001), (8013, 77)])
def test_decode_short_no_syndromes(n, N):
    _check(n, N, hd.SYN_NONE, seed=n + 2)


def test_detected_segments_are_counted():
    # every codeword carries two errors: many syndromes name no position
    ee, ed = _check(100, 2000, hd.SYN_U16, seed=5, p1=0.0, p2=1.0)
    assert ee == 2000 and 0 < ed < 2000


@pytest.mark.parametrize("n,N", [(71, 523), (545, 523), (1078, 77), (2000, 40), (8013, 523), (32767, 37)])
def test_every_tile_configuration_agrees(n, N):
    try:
        for v in range(hd.hd_short_variant_count()):
            hd.hd_short_variant_select(v)
            _check(n, N, hd.SYN_U16, seed=100 + v)
    finally:
        hd.hd_short_variant_select(-1)


@pytest.mark.parametrize("n,N", [(3, 100), (11, 777), (71, 300), (545, 301), (1611, 99), (8013, 33),
                                 (32767, 5), (127, 640), (256, 3)])
def test_encode_short_matches_oracle(n, N):
    import torch
    r, k = oracle.short_params(n)
    data = synth.random_words(n + 9, N * k)
    d = gc.to_device(data, pad_words=4)
    out = torch.full((hd.words_for(N * n) + 4,), -1, dtype=torch.int32, device="cuda")
    hd.encode_short(d, n, N, out=out)
    torch.cuda.synchronize()
    want = oracle.encode_short(data, n, N)
    assert np.array_equal(gc.host_u32(out)[:want.size], want)


@pytest.mark.parametrize("n,N", [(63, 4099), (127, 2049), (255, 1025)])
def test_full_lengths_match_hd_decode(n, N):
    stream, _, _ = gc.received_stream(n, N, seed=n, p1=0.2, p2=0.05)
    d = gc.to_device(stream, pad_words=4)
    o1, s1, e1 = hd.decode(d, n, N, hd.SYN_U16)
    o2, s2, c2 = hd.decode_short(d, n, N, hd.SYN_U16)
    m, k = hd.code_params(n)
    nw = hd.words_for(N * k)
    assert np.array_equal(gc.host_u32(o1)[:nw], gc.host_u32(o2)[:nw])
    assert np.array_equal(s1.cpu().numpy()[:N], s2.cpu().numpy()[:N])
    assert int(e1.item()) == int(c2[0].item()) and int(c2[1].item()) == 0


def test_zero_and_single_segments():
    import torch
    counts = torch.full((2,), 7, dtype=torch.int64, device="cuda")
    hd.check(hd.hd_decode_short(None, 0, 545, 0, None, None, 0, counts.data_ptr(), counts.data_ptr() + 8,
                                torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert counts.cpu().tolist() == [0, 0]
    for n in (11, 71, 8013, 32767):
        _check(n, 1, hd.SYN_U16, seed=3, p1=1.0, p2=0.0)


# The paper's workload grid: packets of M bytes cut into t segments (Sec. IV-A).
GRID = [(M, t) for M in (400, 800, 1200, 1600, 2000) for t in (2, 3, 4, 5, 6)]


@pytest.mark.parametrize("M,t", GRID)
def test_paper_grid_small(M, t):
    n, k, r = hd.hd_segment_params(M, t)
    _check(n, 37 * t, hd.SYN_U16, seed=M + t, p1=0.1, p2=0.02)


@pytest.mark.parametrize("M,t", [(2000, 2), (400, 6), (1200, 4)])
def test_paper_grid_full_size(M, t):
    """About 256 MB of segments of one (M, t), decoded in the launch
    configuration the benchmark times; every data bit, syndrome and both
    counts against the threaded oracle, and the counts against the injected
    channel events (every event gives a nonzero syndrome; a double error is
    detected iff p XOR q > n).  Inputs: the oracle encoder and the
    generator's errors."""
    import os
    import torch
    n, k, r = hd.hd_segment_params(M, t)
    N = (256 << 23) // n  # ~256 MB of input
    data = synth.random_words(M * 10 + t, N * k)
    rx = gc.oracle_encode_parallel(oracle.encode_short, data, n, N, k, n)
    ev = synth.error_events(M * 10 + t, n, N, p1=0.05, p2=0.005)
    synth.apply_errors(rx, ev)
    d_in = gc.to_device(rx, pad_words=4)
    out, syn, counts = hd.decode_short(d_in, n, N, hd.SYN_U16)
    torch.cuda.synchronize()
    c = counts.cpu().numpy()
    dbl = (ev.double_p ^ ev.double_q) > n
    assert int(c[0]) == ev.single_cw.size + ev.double_cw.size
    assert int(c[1]) == int(dbl.sum())
    eo, es, ee, ed = oracle.decode_short(rx, n, N, oracle.SYN_U16, threads=os.cpu_count() or 8)
    nw = hd.words_for(N * k)
    got = gc.host_u32(out)[:nw]
    if not np.array_equal(got, eo[:nw]):
        bad = np.nonzero(got != eo[:nw])[0]
        raise AssertionError(f"(M, t) = ({M}, {t}): {bad.size} output words differ, first {bad[0]}")
    assert np.array_equal(syn.cpu().numpy().view(np.uint16)[:N], es[:N])
    assert (int(c[0]), int(c[1])) == (ee, ed)
    assert hd.hd_device_status() == 0


def test_alternating_lengths():
    # the shared-memory need of the tiled kernel depends on n; a long length after a
    # shorter one must still launch (and give the same bits)
    for n in (8013, 300, 4096, 8013, 71, 32767, 545):
        _check(n, 97 if n < 10000 else 9, hd.SYN_U16, seed=n + 31)


def test_autotune_keeps_parity():
    try:
        for n in (2679, 544, 8013):
            v = hd.hd_short_autotune(n, 20000, 2)
            assert 0 <= v < hd.hd_short_variant_count()
            _check(n, 777 if n < 5000 else 200, hd.SYN_U16, seed=n + 5)
        assert hd.hd_short_autotune(33, 1000, 1) == -1  # k < 64: a single kernel
    finally:
        hd.hd_short_variant_select(-1)


@pytest.mark.parametrize("n", [33, 545, 2679, 32767])
def test_plan_matches_oracle_and_runs_inside_a_capture(n):
    """hd_decode_short_plan: bit-exact against the oracle, directly and when
    recorded in a CUDA graph and replayed (the plan allocates nothing and
    synchronises nothing, so the decode can be captured)."""
    import torch
    r, k = oracle.short_params(n)
    N = 4001 if n < 10000 else 77
    rx, _, _ = _received(n, N, seed=n + 61, p1=0.3, p2=0.2)
    eo, es, ee, ed = oracle.decode_short(rx, n, N, oracle.SYN_U16, threads=8)
    d_in = gc.to_device(rx, pad_words=4)
    nw = hd.words_for(N * k)
    plan = hd.ShortPlan(n)
    try:
        def check(out, syn, counts):
            assert np.array_equal(gc.host_u32(out)[:nw], eo[:nw])
            assert np.array_equal(syn.cpu().numpy()[:N].view(np.uint16), es[:N])
            assert tuple(int(x) for x in counts.cpu().numpy()) == (ee, ed)

        out, syn, counts = plan.decode(d_in, N, hd.SYN_U16)
        torch.cuda.synchronize()
        check(out, syn, counts)
        out.fill_(-1)
        syn.fill_(0x55)
        counts.fill_(9)
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            plan.decode(d_in, N, hd.SYN_U16, out=out, syndromes=syn, counts=counts, cuda_stream=s)
        for _ in range(2):
            out.fill_(-1)
            g.replay()
            torch.cuda.synchronize()
            check(out, syn, counts)
    finally:
        plan.close()
    assert hd.hd_device_status() == 0


def test_cached_path_refuses_a_new_length_inside_a_capture():
    """hd_decode_short builds a length's table on first use, which cannot
    happen inside a stream capture: the call is refused and nothing is
    enqueued (the capture stays valid)."""
    import torch
    n = 4093  # a length no other test decodes
    r, k = oracle.short_params(n)
    N = 64
    rx, _, _ = _received(n, N, seed=3)
    d_in = gc.to_device(rx, pad_words=4)
    out = torch.empty(hd.words_for(N * k) + 4, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rc = hd.hd_decode_short(d_in.data_ptr(), n * N, n, N, out.data_ptr(), None, hd.SYN_NONE, None, None,
                                s.cuda_stream)
    assert rc == hd.HD_ERR_INVALID_ARG
    del g
    _check(n, N, hd.SYN_U16, seed=3)  # outside a capture the same length decodes
