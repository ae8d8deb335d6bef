"""SECDED on the GPU (hd_decode_secded / hd_encode_secded) against the oracle,
bit-exact: data bits, syndromes (s | P << m), the count of nonzero syndromes
and the count of detected double errors.  Stream lengths cover whole chunks of
the streaming kernel plus ragged tails, tails alone, and the full benchmark
size; the error mix includes single errors at every position (the overall
parity bit included), double and triple errors."""
import numpy as np
import pytest

import oracle
from paper_1412_6862_gb300 import hd, synth
from tests import gpu_cases as gc

pytestmark = pytest.mark.gpu

ALL_N = [3, 7, 15, 31, 63, 127, 255]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_6862_gb300 import build
    build.build()
    hd.lib()


def _received(n, N, seed, p1, p2, p3=0.0):
    m, k = hd.code_params(n)
    data = synth.random_words(seed, N * k)
    st = oracle.encode_secded(data, n, N) if N else np.zeros(0, np.uint32)
    ev = synth.error_events(seed + 3, n + 1, N, p1=p1, p2=p2)  # event position e = codeword position e - 1
    synth.apply_errors(st, ev)
    if p3 > 0 and N:
        # a third flip on some double-error codewords (miscorrected by design)
        pick = ev.double_cw[synth.below(seed, 91, 0, ev.double_cw.size, 100) < int(p3 * 100)]
        pos = synth.below(seed, 92, 0, pick.size, n + 1)
        clash = (pos == ev.double_p[np.isin(ev.double_cw, pick)] - 1) | (pos == ev.double_q[np.isin(ev.double_cw, pick)] - 1)
        pick, pos = pick[~clash], pos[~clash]
        synth.flip_bits(st, pick * (n + 1) + pos)
    return st


def _check(n, N, syn_type, seed=0, p1=0.2, p2=0.05, p3=0.0):
    import torch
    m, k = hd.code_params(n)
    rx = _received(n, N, seed, p1, p2, p3)
    d_in = gc.to_device(rx, pad_words=4)
    out = torch.full((max(4, hd.words_for(N * k)),), -1, dtype=torch.int32, device="cuda")
    syn = None
    if syn_type != hd.SYN_NONE:
        syn = torch.full((max(16, N),), 0x55, dtype=torch.uint8 if syn_type == hd.SYN_U8 else torch.int16,
                         device="cuda")
    counts = torch.full((2,), 777, dtype=torch.int64, device="cuda")
    hd.decode_secded(d_in, n, N, syn_type, out=out, syndromes=syn, counts=counts)
    torch.cuda.synchronize()
    eo, es, ee, ed = oracle.decode_secded(rx, n, N, syn_type if syn_type != hd.SYN_NONE else oracle.SYN_U16,
                                          threads=8)
    nw = hd.words_for(N * k)
    got = gc.host_u32(out)[:nw]
    if not np.array_equal(got, eo[:nw]):
        bad = np.nonzero(got != eo[:nw])[0]
        raise AssertionError(f"n={n} N={N}: {bad.size} output words differ, first {bad[0]}")
    if syn is not None:
        sg = syn.cpu().numpy()[:N]
        if syn_type == hd.SYN_U16:
            sg = sg.view(np.uint16)
        assert np.array_equal(sg, es[:N].astype(sg.dtype)), f"n={n}: syndromes differ"
    c = counts.cpu().numpy()
    assert (int(c[0]), int(c[1])) == (ee, ed), (n, N, c, ee, ed)
    assert hd.hd_device_status() == 0
    return ee, ed


@pytest.mark.parametrize("n", ALL_N)
@pytest.mark.parametrize("N", [1, 31, 1000, 4096 * 3 + 77, 100003])
def test_secded_u16(n, N):
    _check(n, N, hd.SYN_U16, seed=n * 7 + N)


@pytest.mark.parametrize("n", [3, 7, 15, 31, 63, 127])
def test_secded_u8_and_none(n):
    _check(n, 50000 + n, hd.SYN_U8, seed=n + 1)
    _check(n, 40000 + n, hd.SYN_NONE, seed=n + 2)


@pytest.mark.parametrize("n", [15, 63, 255])
def test_secded_triple_errors_are_miscorrected_like_the_oracle(n):
    ee, ed = _check(n, 30000, hd.SYN_U16, seed=n + 9, p1=0.1, p2=0.3, p3=0.5)
    assert ed > 0


@pytest.mark.parametrize("n", ALL_N)
def test_secded_encoder_matches_oracle(n):
    import torch
    m, k = hd.code_params(n)
    N = 7777
    data = synth.random_words(n + 17, N * k)
    d = gc.to_device(data, pad_words=4)
    out = torch.full((hd.words_for(N * (n + 1)) + 4,), -1, dtype=torch.int32, device="cuda")
    hd.encode_secded(d, n, N, out=out)
    torch.cuda.synchronize()
    want = oracle.encode_secded(data, n, N)
    assert np.array_equal(gc.host_u32(out)[:want.size], want)


# The SECDED benchmark workload at full size: 2^24 codewords for n <= 63, 2^22
# above, p1 = 0.05 and p2 = 0.005 over the n + 1 bits, u16 syndromes.
FULL_SECDED = [(7, 1 << 24), (15, 1 << 24), (31, 1 << 24), (63, 1 << 24), (127, 1 << 22), (255, 1 << 22)]


@pytest.mark.parametrize("n,N", FULL_SECDED)
def test_secded_full_size(n, N):
    """Full-size streams in the launch configuration the benchmark times;
    every data bit, every syndrome and both counts against the threaded
    oracle, and the counts against the injected channel events (every event
    gives a nonzero syndrome, exactly the doubles are detected).  Inputs:
    the oracle encoder and the generator's errors."""
    import os
    import torch
    m, k = hd.code_params(n)
    data = synth.random_words(n + 5, N * k)
    rx = gc.oracle_encode_parallel(oracle.encode_secded, data, n, N, k, n + 1)
    ev = synth.error_events(n + 5, n + 1, N, p1=0.05, p2=0.005)
    synth.apply_errors(rx, ev)
    d_in = gc.to_device(rx, pad_words=4)
    out, syn, counts = hd.decode_secded(d_in, n, N, hd.SYN_U16)
    torch.cuda.synchronize()
    c = counts.cpu().numpy()
    assert int(c[0]) == ev.single_cw.size + ev.double_cw.size
    assert int(c[1]) == ev.double_cw.size
    eo, es, ee, ed = oracle.decode_secded(rx, n, N, oracle.SYN_U16, threads=os.cpu_count() or 8)
    nw = hd.words_for(N * k)
    got = gc.host_u32(out)[:nw]
    if not np.array_equal(got, eo[:nw]):
        bad = np.nonzero(got != eo[:nw])[0]
        raise AssertionError(f"n={n}: {bad.size} output words differ, first {bad[0]}")
    assert np.array_equal(syn.cpu().numpy().view(np.uint16)[:N], es[:N])
    assert (int(c[0]), int(c[1])) == (ee, ed)
    assert hd.hd_device_status() == 0
