"""Pins for the CPU oracle, checked against what the paper and the mathematics
fix rather than against the oracle itself:

* the index sets printed in Sec. III-A (golden fixture);
* a hand-worked (7,4) codeword (closed form below);
* brute force over every message and every single and double error for n = 7
  and n = 15, with expectations built from the error pattern, not from a decode;
* the parity-check-matrix form H r^T for every supported n;
* code properties: minimum distance 3, the perfect-code property, linearity.
"""
import os

import numpy as np
import pytest

from paper_1412_6862_gb300 import synth
from tests import np_ref

ALL_N = [3, 7, 15, 31, 63, 127, 255]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_index_sets():
    sets = {}
    with open(os.path.join(GOLDEN, "index_sets_sec3a.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, vals = line.split(":")
            sets[int(name.strip()[1:])] = [int(v) for v in vals.split()]
    return sets


def test_index_sets_match_paper(oracle_mod):
    """Sec. III-A: with 4 checksum bits over positions 1..11, checksum bit j covers
    exactly the printed I_j.  A single 1 at position p must give syndrome p, and
    for any word supported on positions 1..11 syndrome bit j must be the XOR of
    the bits at the positions of I_j."""
    sets = _read_index_sets()
    n, N = 15, 11
    stream = np.zeros((N * n + 31) // 32, np.uint32)
    for i, p in enumerate(range(1, 12)):
        np_ref_bits = i * n + p - 1
        stream[np_ref_bits >> 5] |= np.uint32(1 << (np_ref_bits & 31))
    _, syn, err = oracle_mod.decode(stream, n, N)
    assert list(syn) == list(range(1, 12))
    assert err == N
    for j, members in sets.items():
        for p in range(1, 12):
            assert ((int(syn[p - 1]) >> j) & 1) == (1 if p in members else 0), (j, p)
    # random words supported on positions 1..11
    rng_words = synth.random_words(5, 400 * n)
    bits = np_ref.words_to_bits(rng_words, 400 * n).reshape(400, n).copy()
    bits[:, 11:] = 0
    w = np_ref.bits_to_words(bits.reshape(-1))
    _, syn, _ = oracle_mod.decode(w, n, 400)
    for j, members in sets.items():
        expect = np.bitwise_xor.reduce(bits[:, [p - 1 for p in members]], axis=1)
        assert np.array_equal((syn.astype(np.int64) >> j) & 1, expect), j


def test_worked_example_7_4(oracle_mod):
    """Data d1..d4 = 1,0,1,1 sits at positions 3,5,6,7.  Even parity gives
    position 1 = d1^d2^d4 = 0, position 2 = d1^d3^d4 = 1, position 4 = d2^d3^d4 = 0,
    so positions 1..7 read 0 1 1 0 0 1 1, i.e. 0x66 LSB first; the data word
    LSB first is 0b1101 = 0xD.  Flipping position 5 gives 0x76 and syndrome 5."""
    data = np.array([0xD], np.uint32)
    cw = oracle_mod.encode(data, 7, 1)
    assert int(cw[0]) == 0x66
    out, syn, err = oracle_mod.decode(np.array([0x66], np.uint32), 7, 1)
    assert (int(out[0]), int(syn[0]), err) == (0xD, 0, 0)
    out, syn, err = oracle_mod.decode(np.array([0x76], np.uint32), 7, 1)
    assert (int(out[0]), int(syn[0]), err) == (0xD, 5, 1)


def _all_messages(k):
    msgs = np.arange(1 << k, dtype=np.int64)
    return ((msgs[:, None] >> np.arange(k)[None, :]) & 1).astype(np.uint8)


@pytest.mark.parametrize("n", [7, 15])
def test_bruteforce_single_and_double_errors(oracle_mod, n):
    m = np_ref.m_of(n)
    k = n - m
    M = _all_messages(k)                                      # 2^k x k
    data_words = np_ref.bits_to_words(M.reshape(-1))
    cw = oracle_mod.encode(data_words, n, M.shape[0])
    C = np_ref.codeword_matrix(cw, n, M.shape[0])
    H = np_ref.parity_check_matrix(n)
    # every encoder output satisfies H c^T = 0 and carries the message at the data positions
    assert not ((C.astype(np.int64) @ H.T) & 1).any()
    dpos = np_ref.data_positions(n)
    assert np.array_equal(C[:, dpos - 1], M)

    patterns = [()] + [(p,) for p in range(1, n + 1)] + \
               [(p, q) for p in range(1, n + 1) for q in range(p + 1, n + 1)]
    P = len(patterns)
    R = np.repeat(C, P, axis=0)                               # (2^k * P) x n
    exp_s = np.zeros(R.shape[0], np.int64)
    exp_D = np.repeat(M, P, axis=0).copy()
    pos_to_data = {int(p): i for i, p in enumerate(dpos)}
    for t, pat in enumerate(patterns):
        rows = slice(t, None, P)
        s = 0
        for p in pat:
            R[rows, p - 1] ^= 1
            s ^= p
        exp_s[rows] = s
        # a plain SEC decoder flips position s: the data bits at p, q and s are wrong
        # or right according to the flip count per position
        flips = {}
        for p in list(pat) + ([s] if s else []):
            flips[p] = flips.get(p, 0) ^ 1
        for p, f in flips.items():
            if f and p in pos_to_data:
                exp_D[rows, pos_to_data[p]] ^= 1
    stream = np_ref.bits_to_words(R.reshape(-1))
    out, syn, err = oracle_mod.decode(stream, n, R.shape[0])
    assert np.array_equal(syn.astype(np.int64), exp_s)
    assert err == int((exp_s != 0).sum()) == (1 << k) * (P - 1)
    D = np_ref.words_to_bits(out, R.shape[0] * k).reshape(-1, k)
    assert np.array_equal(D, exp_D)
    # single errors are corrected exactly
    single_rows = np.concatenate([np.arange(t, R.shape[0], P) for t in range(1, n + 1)])
    assert np.array_equal(D[single_rows], np.repeat(M, P, axis=0)[single_rows])


@pytest.mark.parametrize("n", [7, 15])
def test_minimum_distance_three(oracle_mod, n):
    k = n - np_ref.m_of(n)
    M = _all_messages(k)
    cw = oracle_mod.encode(np_ref.bits_to_words(M.reshape(-1)), n, M.shape[0])
    C = np_ref.codeword_matrix(cw, n, M.shape[0])
    vals = (C.astype(np.int64) << np.arange(n)[None, :]).sum(axis=1)
    assert np.unique(vals).size == 1 << k
    x = vals[:, None] ^ vals[None, :]
    w = np.zeros_like(x)
    for b in range(n):
        w += (x >> b) & 1
    np.fill_diagonal(w, 99)
    assert w.min() == 3


@pytest.mark.parametrize("n", ALL_N)
def test_syndrome_equals_parity_check(oracle_mod, n):
    N = 3000
    stream = synth.random_words(11 + n, N * n)
    _, syn, err = oracle_mod.decode(stream, n, N, syn_type=oracle_mod.SYN_U16)
    s_ref = np_ref.syndromes(stream, n, N)
    assert np.array_equal(syn.astype(np.int64), s_ref)
    assert err == int((s_ref != 0).sum())
    words, s2, e2 = np_ref.decode(stream, n, N)
    out, _, _ = oracle_mod.decode(stream, n, N)
    assert np.array_equal(out, words)


@pytest.mark.parametrize("n", ALL_N)
def test_perfect_code_property(oracle_mod, n):
    """Every received word lies within distance 1 of exactly one codeword: the
    re-encoded decoded data differs from the received word exactly at position s
    (nowhere when s = 0)."""
    N = 2000
    m = np_ref.m_of(n)
    k = n - m
    stream = synth.random_words(100 + n, N * n)
    out, syn, _ = oracle_mod.decode(stream, n, N, syn_type=oracle_mod.SYN_U16)
    re = oracle_mod.encode(out, n, N)
    diff = np_ref.codeword_matrix(re ^ stream, n, N)
    exp = np.zeros((N, n), np.uint8)
    nz = np.nonzero(syn)[0]
    exp[nz, syn[nz].astype(np.int64) - 1] = 1
    assert np.array_equal(diff, exp)


@pytest.mark.parametrize("n", ALL_N)
def test_syndrome_linearity(oracle_mod, n):
    N = 1000
    a = synth.random_words(1, N * n)
    b = synth.random_words(2, N * n)
    _, sa, _ = oracle_mod.decode(a, n, N, syn_type=oracle_mod.SYN_U16)
    _, sb, _ = oracle_mod.decode(b, n, N, syn_type=oracle_mod.SYN_U16)
    _, sab, _ = oracle_mod.decode(a ^ b, n, N, syn_type=oracle_mod.SYN_U16)
    assert np.array_equal(sab, sa ^ sb)


@pytest.mark.parametrize("n", ALL_N)
def test_err_count_equals_injected_events(oracle_mod, n):
    N = 5000
    m = np_ref.m_of(n)
    k = n - m
    data = synth.random_words(0, N * k)
    cw = oracle_mod.encode(data, n, N)
    ev = synth.error_events(0, n, N, p1=0.1, p2=0.05)
    synth.apply_errors(cw, ev)
    out, syn, err = oracle_mod.decode(cw, n, N)
    assert err == ev.num_events
    # single-error codewords decode to the original message
    D = np_ref.words_to_bits(out, N * k).reshape(N, k)
    D0 = np_ref.words_to_bits(data, N * k).reshape(N, k)
    clean = np.ones(N, bool)
    clean[ev.double_cw] = False
    assert np.array_equal(D[clean], D0[clean])
    assert np.array_equal(syn[ev.single_cw].astype(np.int64), ev.single_pos)
    assert np.array_equal(syn[ev.double_cw].astype(np.int64), ev.double_p ^ ev.double_q)


@pytest.mark.parametrize("n", ALL_N)
def test_pad_bits_zero_and_edge_sizes(oracle_mod, n):
    k = n - np_ref.m_of(n)
    for N in (1, 2, 31, 33):
        stream = synth.random_words(9, N * n)
        stream_dirty = stream.copy()
        if (N * n) % 32:
            stream_dirty[-1] |= np.uint32(0xFFFFFFFF << ((N * n) % 32) & 0xFFFFFFFF)
        out, syn, err = oracle_mod.decode(stream_dirty, n, N)
        out2, syn2, err2 = oracle_mod.decode(stream, n, N)
        assert np.array_equal(out, out2) and err == err2  # input pad bits are ignored
        tail = (N * k) % 32
        if tail:
            assert int(out[-1]) >> tail == 0
    out, syn, err = oracle_mod.decode(np.zeros(1, np.uint32), n, 0)
    assert err == 0


def test_argument_errors(oracle_mod):
    z = np.zeros(64, np.uint32)
    assert oracle_mod.decode_rc(z, 8 * 10, 8, 10) == 1      # n not 2^m - 1
    assert oracle_mod.decode_rc(z, 511 * 1, 511, 1) == 1    # m > 8
    assert oracle_mod.decode_rc(z, 7 * 10 + 1, 7, 10) == 3  # in_bits != n * N
    assert oracle_mod.decode_rc(z, 7 * 10, 7, 10) == 0


@pytest.mark.parametrize("n", [15, 63, 255])
def test_threaded_equals_serial(oracle_mod, n):
    N = 4099
    k = n - np_ref.m_of(n)
    stream = synth.random_words(3, N * n)
    out, syn, err = oracle_mod.decode(stream, n, N)
    out_t = np.zeros_like(out)
    syn_t = np.zeros_like(syn)
    err_t = oracle_mod.decode_threaded(stream, n, N, oracle_mod.SYN_U8, 4, out_t, syn_t)
    assert err_t == err and np.array_equal(out_t, out) and np.array_equal(syn_t, syn)
