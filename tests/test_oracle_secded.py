"""Pins for the oracle's SECDED decoder (extended Hamming: a full-length code
plus an overall parity bit at position 0; not in the paper, an extension of its
single-error decoder that detects double errors instead of miscorrecting them).
Checked against what the mathematics fixes:

* brute force over every message for n = 7 and 15: encoder outputs satisfy the
  parity-check equations and even overall parity, the code has minimum
  distance 4, every single error (position 0 included) is corrected, every
  double error is detected and left as received, triple errors are
  miscorrected exactly as s = p ^ q ^ r with P = 1 prescribes;
* the relation to the independently pinned single-error decoder: a codeword
  with odd overall parity decodes exactly like the plain code on positions
  1..n, one with even parity and s != 0 is left as received;
* the parity-check-matrix form on random words of every length.
"""
import itertools

import numpy as np
import pytest

from paper_1412_6862_gb300 import synth
from tests import np_ref
from tests import test_oracle as full_pins

M_OF = {3: 2, 7: 3, 15: 4, 31: 5, 63: 6, 127: 7, 255: 8}


def _bits(words, nbits):
    return np_ref.words_to_bits(words, nbits)


@pytest.mark.parametrize("n", [7, 15])
def test_secded_bruteforce(oracle_mod, n):
    m = M_OF[n]
    k = n - m
    L = n + 1
    M = 1 << k
    msg = ((np.arange(M)[:, None] >> np.arange(k)[None, :]) & 1).astype(np.uint8)
    stream = oracle_mod.encode_secded(np_ref.bits_to_words(msg.reshape(-1)), n, M)
    C = _bits(stream, M * L).reshape(M, L)
    dpos = np_ref.data_positions(n)
    assert np.array_equal(C[:, dpos], msg)
    H = np_ref.parity_check_matrix(n)
    assert ((C[:, 1:].astype(np.int64) @ H.T) % 2 == 0).all()
    assert (C.sum(axis=1) % 2 == 0).all()
    w = C.sum(axis=1)
    assert w[0] == 0 and (w[1:] >= 4).all() and (w[1:] == 4).any()
    pick = np.arange(M) if M <= 64 else synth.below(4, n, 0, 64, M)
    sub = C[pick]
    P = len(pick)

    def dec(R):
        return oracle_mod.decode_secded(np_ref.bits_to_words(R.reshape(-1)), n, P)

    out, syn, errs, det = dec(sub)
    assert (syn == 0).all() and errs == 0 and det == 0
    assert np.array_equal(_bits(out, P * k).reshape(P, k), msg[pick])
    for p in range(L):
        R = sub.copy()
        R[:, p] ^= 1
        out, syn, errs, det = dec(R)
        assert (syn == (p | (1 << m))).all() and errs == P and det == 0, p
        assert np.array_equal(_bits(out, P * k).reshape(P, k), msg[pick]), p
    for p, q in itertools.combinations(range(L), 2):
        R = sub.copy()
        R[:, [p, q]] ^= 1
        out, syn, errs, det = dec(R)
        assert (syn == (p ^ q)).all() and errs == P and det == P, (p, q)
        assert np.array_equal(_bits(out, P * k).reshape(P, k), R[:, dpos]), (p, q)
    for p, q, r in list(itertools.combinations(range(L), 3))[::7]:
        R = sub.copy()
        R[:, [p, q, r]] ^= 1
        out, syn, errs, det = dec(R)
        s = p ^ q ^ r
        assert (syn == (s | (1 << m))).all() and det == 0
        E = R.copy()
        E[:, s] ^= 1
        assert np.array_equal(_bits(out, P * k).reshape(P, k), E[:, dpos]), (p, q, r)


@pytest.mark.parametrize("n", full_pins.ALL_N)
def test_secded_relation_to_single_error_decoder(oracle_mod, n):
    m = M_OF[n]
    k = n - m
    L = n + 1
    N = 500
    rnd = synth.random_words(31 + n, N * L)
    out, syn, errs, det = oracle_mod.decode_secded(rnd, n, N)
    R = _bits(rnd, N * L).reshape(N, L)
    plain = np_ref.bits_to_words(R[:, 1:].reshape(-1))
    pout, psyn, perr = oracle_mod.decode(plain, n, N, oracle_mod.SYN_U16)
    par = R.sum(axis=1) % 2
    got = _bits(out, N * k).reshape(N, k)
    single = _bits(pout, N * k).reshape(N, k)
    assert np.array_equal(syn.astype(np.int64), psyn.astype(np.int64) | (par.astype(np.int64) << m))
    odd = par == 1
    assert np.array_equal(got[odd], single[odd])
    even = ~odd
    assert np.array_equal(got[even], R[even][:, np_ref.data_positions(n)])
    assert errs == int(((psyn != 0) | odd).sum())
    assert det == int(((psyn != 0) & even).sum())


@pytest.mark.parametrize("n", [31, 63, 127, 255])
def test_secded_matrix_form(oracle_mod, n):
    m = M_OF[n]
    L = n + 1
    N = 300
    rnd = synth.random_words(57 + n, N * L)
    _, syn, _, _ = oracle_mod.decode_secded(rnd, n, N)
    R = _bits(rnd, N * L).reshape(N, L).astype(np.int64)
    H = np_ref.parity_check_matrix(n)
    S = (R[:, 1:] @ H.T) % 2
    s = (S << np.arange(m)[None, :]).sum(axis=1)
    assert np.array_equal(syn.astype(np.int64), s | ((R.sum(axis=1) % 2) << m))


def test_secded_injected_events(oracle_mod):
    # with at most two flips per codeword every event is seen: singles corrected, doubles detected
    n, N = 63, 4000
    k = n - 6
    data = synth.random_words(3, N * k)
    st = oracle_mod.encode_secded(data, n, N)
    # events over the n + 1 bits of each codeword (event position e is codeword position e - 1)
    ev = synth.error_events(8, n + 1, N, p1=0.2, p2=0.1)
    rx = st.copy()
    synth.apply_errors(rx, ev)
    out, syn, errs, det = oracle_mod.decode_secded(rx, n, N)
    assert errs == ev.single_cw.size + ev.double_cw.size
    assert det == ev.double_cw.size
    got = _bits(out, N * k).reshape(N, k)
    want = _bits(data, N * k).reshape(N, k)
    ok = np.setdiff1d(np.arange(N), ev.double_cw)
    assert np.array_equal(got[ok], want[ok])
