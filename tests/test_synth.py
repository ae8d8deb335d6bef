"""The seeded input generator: SplitMix64 against its published outputs, layout,
reproducibility of sub-ranges, and the error and packet distributions."""
import math

import numpy as np

from paper_1412_6862_gb300 import synth

# First outputs of SplitMix64 seeded with 0 (Steele, Lea and Flood, OOPSLA 2014;
# the widely reproduced reference sequence).
SPLITMIX64_SEED0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]


def test_splitmix64_published_sequence():
    idx = np.arange(1, 5, dtype=np.uint64)
    with np.errstate(over="ignore"):
        out = synth._mix(idx * synth.GOLDEN)
    assert [int(v) for v in out] == SPLITMIX64_SEED0


def test_draws_are_counter_based():
    a = synth.draws(7, synth.TAG_DATA, 0, 1000)
    b = synth.draws(7, synth.TAG_DATA, 500, 500)
    assert np.array_equal(a[500:], b)
    assert not np.array_equal(a, synth.draws(8, synth.TAG_DATA, 0, 1000))
    assert not np.array_equal(a, synth.draws(7, synth.TAG_ERR_KIND, 0, 1000))


def test_random_words_pad_and_balance():
    w = synth.random_words(0, 32 * 1000 + 5)
    assert w.dtype == np.uint32 and w.size == 1001
    assert int(w[-1]) >> 5 == 0
    ones = sum(bin(int(x)).count("1") for x in w[:-1])
    assert abs(ones / (32 * 1000) - 0.5) < 0.01


def test_error_events_distribution_and_subrange():
    n, N = 31, 200000
    ev = synth.error_events(3, n, N, p1=0.1, p2=0.01)
    assert abs(ev.single_cw.size / N - 0.1) < 0.005
    assert abs(ev.double_cw.size / N - 0.01) < 0.002
    assert ev.single_pos.min() >= 1 and ev.single_pos.max() <= n
    assert (ev.double_p != ev.double_q).all()
    assert ev.double_q.min() >= 1 and ev.double_q.max() <= n
    assert np.intersect1d(ev.single_cw, ev.double_cw).size == 0
    # uniform positions
    counts = np.bincount(ev.single_pos, minlength=n + 1)[1:]
    assert counts.min() > 0.8 * counts.mean()
    sub = synth.error_events(3, n, 1000, p1=0.1, p2=0.01, first_codeword=5000)
    sel = (ev.single_cw >= 5000) & (ev.single_cw < 6000)
    assert np.array_equal(sub.single_cw, ev.single_cw[sel])
    assert np.array_equal(sub.single_pos, ev.single_pos[sel])


def test_apply_errors_flips_exact_bits():
    n, N = 15, 100
    w = np.zeros((N * n + 31) // 32, np.uint32)
    ev = synth.error_events(1, n, N, p1=0.3, p2=0.2)
    synth.apply_errors(w, ev)
    bits = np.unpackbits(w.view(np.uint8), bitorder="little")
    assert bits.sum() == ev.single_cw.size + 2 * ev.double_cw.size
    for c, p in zip(ev.single_cw, ev.single_pos):
        assert bits[c * n + p - 1] == 1


def test_packet_table_shape():
    pk = synth.packet_table(0, 10000)
    ns = np.array([p.n for p in pk])
    assert set(ns) == set(synth.CODE_LENGTHS)
    bits = np.array([p.n * p.num_codewords for p in pk], dtype=np.float64)
    assert (np.array([p.num_codewords for p in pk]) >= 1).all()
    assert bits.max() <= 4 * 1024 * 1024 + 255
    # log-uniform: the median of log(bits) sits near the middle of [log 64, log 4Mi]
    mid = 0.5 * (math.log(64) + math.log(4 * 1024 * 1024))
    assert abs(np.median(np.log(np.maximum(bits, 64))) - mid) < 0.3


def test_poisson_arrivals_rate():
    t = synth.poisson_arrivals(0, 100000, 1e5)
    assert abs(t[-1] - 1.0) < 0.02
    assert (np.diff(t) > 0).all()
