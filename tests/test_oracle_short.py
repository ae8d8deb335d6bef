"""Pins for the oracle's shortened codes (segments of any length n, Sec. II and
Sec. IV-A: a packet of M bytes is split into t segments, each protected by its
own checksum bits), checked against what the paper and the mathematics fix:

* the index sets printed in Sec. III-A, which describe exactly the shortened
  code with 11 positions and 4 checksum bits (golden fixture);
* brute force over every message and every single and double error for small
  n, with expectations built from the error pattern, not from a decode;
* the shortening identity: a codeword of length n is a full-length codeword of
  length 2^r - 1 whose positions past n are zero, so the pinned full-length
  decoder gives the same data bits and syndromes (and a syndrome past n is the
  detected-uncorrectable case);
* the parity-check-matrix form on long segments (n up to 32767);
* the full-length lengths reduce to the full-length decoder.
"""
import itertools

import numpy as np
import pytest

from paper_1412_6862_gb300 import synth
from tests import np_ref
from tests import test_oracle as full_pins


def _bits(words, nbits):
    return np_ref.words_to_bits(words, nbits)


def test_short_params_are_minimal(oracle_mod):
    for n in list(range(3, 300)) + [545, 1611, 8013, 16383, 16384, 32767]:
        r, k = oracle_mod.short_params(n)
        assert (1 << r) >= n + 1 and (1 << (r - 1)) < n + 1, n
        # r checksum positions 1, 2, ..., 2^(r-1) all lie inside the codeword
        assert sum(1 for j in range(20) if (1 << j) <= n) == r
        assert k == n - r
    for bad in (0, 1, 2, 65536):
        with pytest.raises(ValueError):
            oracle_mod.short_params(bad)


def test_short_index_sets_match_paper(oracle_mod):
    """Sec. III-A lists I_0..I_3 over positions 1..11: a single error at
    position p must set exactly the syndrome bits j with p in I_j, and be
    corrected."""
    sets = full_pins._read_index_sets()
    n = 11
    r, k = oracle_mod.short_params(n)
    assert r == len(sets) == 4
    msgs = synth.random_words(5, 64 * k)
    stream = oracle_mod.encode_short(msgs, n, 64)
    for p in range(1, n + 1):
        want = sum(1 << j for j, ids in sets.items() if p in ids)
        bits = _bits(stream, 64 * n).copy()
        bits[np.arange(64) * n + p - 1] ^= 1
        out, syn, errs, detected = oracle_mod.decode_short(np_ref.bits_to_words(bits), n, 64)
        assert (syn == want).all(), p
        assert errs == 64 and detected == 0
        assert np.array_equal(_bits(out, 64 * k), _bits(msgs, 64 * k))


@pytest.mark.parametrize("n", [3, 5, 6, 9, 10, 11, 12, 13, 14, 17, 20])
def test_short_bruteforce(oracle_mod, n):
    """Every message of length k: encoding lands in the null space of the
    parity-check matrix, the message sits at the non-power-of-two positions,
    the code has minimum distance 3; every single error is corrected; every
    double error gives syndrome p XOR q, which is miscorrected when it names a
    position and flagged as detected otherwise."""
    r, k = oracle_mod.short_params(n)
    M = 1 << k
    msg_bits = ((np.arange(M)[:, None] >> np.arange(k)[None, :]) & 1).astype(np.uint8)
    data = np_ref.bits_to_words(msg_bits.reshape(-1))
    stream = oracle_mod.encode_short(data, n, M)
    C = _bits(stream, M * n).reshape(M, n)
    dpos = np_ref.data_positions(n) - 1
    assert np.array_equal(C[:, dpos], msg_bits)
    assert (np_ref.short_syndromes(stream, n, M) == 0).all()
    w = C.sum(axis=1)
    assert w[0] == 0 and (w[1:] >= 3).all() and (w[1:] == 3).any()
    assert len({row.tobytes() for row in C}) == M
    # single errors on a sample of messages (all of them for small k)
    pick = np.arange(M) if M <= 256 else synth.below(9, n, 0, 256, M)
    sub = C[pick]
    for p in range(1, n + 1):
        R = sub.copy()
        R[:, p - 1] ^= 1
        out, syn, errs, detected = oracle_mod.decode_short(np_ref.bits_to_words(R.reshape(-1)), n, len(pick))
        assert (syn == p).all() and errs == len(pick) and detected == 0
        assert np.array_equal(_bits(out, len(pick) * k).reshape(-1, k), msg_bits[pick])
    # every double error
    for p, q in itertools.combinations(range(1, n + 1), 2):
        R = sub.copy()
        R[:, [p - 1, q - 1]] ^= 1
        out, syn, errs, detected = oracle_mod.decode_short(np_ref.bits_to_words(R.reshape(-1)), n, len(pick))
        s = p ^ q
        assert (syn == s).all()
        assert errs == len(pick)
        E = R.copy()
        if s <= n:
            E[:, s - 1] ^= 1
            assert detected == 0
        else:
            assert detected == len(pick)
        assert np.array_equal(_bits(out, len(pick) * k).reshape(-1, k), E[:, dpos])


@pytest.mark.parametrize("n", [3, 4, 11, 12, 20, 33, 40, 64, 65, 100, 128, 200, 254])
def test_short_equals_zero_padded_full_length(oracle_mod, n):
    """Shortening: pad each length-n codeword with zeros at positions n+1..2^r-1
    and decode it with the (independently pinned) full-length decoder.  Data
    bits at positions <= n and syndromes agree; a syndrome past n makes the
    full-length decoder flip a padding position, the shortened one flags it."""
    r, k = oracle_mod.short_params(n)
    Nf = (1 << r) - 1
    mf = r
    kf = Nf - mf
    N = 400
    rnd = synth.random_words(11 + n, N * n)
    out, syn, errs, detected = oracle_mod.decode_short(rnd, n, N)
    R = _bits(rnd, N * n).reshape(N, n)
    P = np.zeros((N, Nf), np.uint8)
    P[:, :n] = R
    fout, fsyn, ferr = oracle_mod.decode(np_ref.bits_to_words(P.reshape(-1)), Nf, N, oracle_mod.SYN_U16)
    assert np.array_equal(syn.astype(np.int64), fsyn.astype(np.int64))
    assert errs == ferr
    assert detected == int((fsyn > n).sum())
    # data positions <= n are the first k data positions of the full code
    assert np.array_equal(_bits(out, N * k).reshape(N, k), _bits(fout, N * kf).reshape(N, kf)[:, :k])


@pytest.mark.parametrize("n", [71, 545, 1611, 8013, 32767])
def test_short_matrix_form_long(oracle_mod, n):
    """Long segments (the paper's packets of 400..2000 bytes split into 2..6
    segments have n of about 550..8000): the oracle agrees with the
    parity-check-matrix decode on encoded words with injected errors."""
    r, k = oracle_mod.short_params(n)
    N = 40 if n < 10000 else 24
    data = synth.random_words(13 + n, N * k)
    stream = oracle_mod.encode_short(data, n, N)
    ev = synth.error_events(17, n, N, 0.5, 0.2)
    rx = stream.copy()
    synth.apply_errors(rx, ev)
    out, syn, errs, detected = oracle_mod.decode_short(rx, n, N, threads=4)
    eout, esyn, ecor, edet = np_ref.short_decode(rx, n, N)
    assert np.array_equal(syn.astype(np.int64), esyn)
    assert (errs, detected) == (ecor, edet)
    assert np.array_equal(out, eout)
    # single-error codewords come back as the message
    assert ev.single_cw.size and ev.double_cw.size
    got = _bits(out, N * k).reshape(N, k)
    want = _bits(data, N * k).reshape(N, k)
    assert np.array_equal(got[ev.single_cw], want[ev.single_cw])
    clean = np.setdiff1d(np.arange(N), np.concatenate([ev.single_cw, ev.double_cw]))
    assert np.array_equal(got[clean], want[clean])


@pytest.mark.parametrize("n", full_pins.ALL_N)
def test_short_full_lengths_reduce_to_full_decoder(oracle_mod, n):
    N = 300
    rnd = synth.random_words(19 + n, N * n)
    out, syn, errs, detected = oracle_mod.decode_short(rnd, n, N)
    fout, fsyn, ferr = oracle_mod.decode(rnd, n, N, oracle_mod.SYN_U16)
    assert np.array_equal(out, fout) and np.array_equal(syn, fsyn)
    assert errs == ferr and detected == 0
