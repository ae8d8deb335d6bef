"""Seeded synthetic inputs for the Hamming decoder: random bits, channel errors,
packet tables and arrival times.

This module holds no Hamming arithmetic. It draws random numbers and flips bits
at given stream positions; building codewords from data bits (the encoder) and
decoding them happen elsewhere. Both the CPU oracle's tests and the GPU path's
tests and benchmark draw their inputs from here, so the two sides see identical
bits without sharing any code that computes a syndrome or moves a data bit.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw ``i`` of stream ``tag`` under ``seed`` is the SplitMix64
finaliser applied to ``key(seed, tag) + (i + 1) * GOLDEN``.  Everything is
vectorised numpy on uint64 and gives the same bits on x86-64 and aarch64.

Bit layout shared by every producer and consumer in this repository: stream bit
``b`` is bit ``b % 32`` of uint32 word ``b // 32`` (LSB first).  Codeword ``i``
of length ``n`` occupies stream bits ``[i*n, (i+1)*n)``; its position ``p``
(1-indexed, p = 1..n) is stream bit ``i*n + p - 1``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream tags keep the draws for different purposes independent.
TAG_DATA = 1
TAG_ERR_KIND = 2
TAG_ERR_POS1 = 3
TAG_ERR_POS2 = 4
TAG_PKT_N = 5
TAG_PKT_LEN = 6
TAG_ARRIVAL = 7


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser (the published constants 30/27/31)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _key(seed: int, tag: int) -> np.uint64:
    k = np.array([(int(seed) & 0xFFFFFFFFFFFFFFFF) ^ ((int(tag) * 0xD1B54A32D192ED03) & 0xFFFFFFFFFFFFFFFF)],
                 dtype=np.uint64)
    return _mix(k)[0]


def draws(seed: int, tag: int, start: int, count: int) -> np.ndarray:
    """``count`` uint64 draws of stream ``tag`` starting at counter ``start``."""
    idx = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(_key(seed, tag) + (idx + np.uint64(1)) * GOLDEN)


def uniform01(seed: int, tag: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each draw."""
    return (draws(seed, tag, start, count) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def below(seed: int, tag: int, start: int, count: int, bound: int) -> np.ndarray:
    """Integers uniform in [0, bound) by the multiply-shift map of a 32-bit draw."""
    hi = draws(seed, tag, start, count) >> np.uint64(32)
    return ((hi * np.uint64(bound)) >> np.uint64(32)).astype(np.int64)


def random_words(seed: int, num_bits: int, tag: int = TAG_DATA) -> np.ndarray:
    """``ceil(num_bits/32)`` uint32 words of uniform random bits; pad bits are 0."""
    nwords = (int(num_bits) + 31) // 32
    n64 = (nwords + 1) // 2
    w = draws(seed, tag, 0, n64).view(np.uint32)[:nwords].copy()  # little-endian halves
    tail = int(num_bits) % 32
    if nwords and tail:
        w[-1] &= np.uint32((1 << tail) - 1)
    return w


@dataclass
class ErrorEvents:
    """Channel errors for one stream of ``num_codewords`` codewords of length ``n``.

    ``single_cw[j]`` gets one flip at position ``single_pos[j]``; ``double_cw[j]``
    gets flips at the two distinct positions ``double_p[j]`` and ``double_q[j]``.
    Positions are 1-indexed.
    """

    n: int
    num_codewords: int
    single_cw: np.ndarray
    single_pos: np.ndarray
    double_cw: np.ndarray
    double_p: np.ndarray
    double_q: np.ndarray

    @property
    def num_events(self) -> int:
        return int(self.single_cw.size + self.double_cw.size)

    def stream_bits(self) -> np.ndarray:
        """Every flipped stream bit index (int64)."""
        n = np.int64(self.n)
        parts = [self.single_cw * n + self.single_pos - 1,
                 self.double_cw * n + self.double_p - 1,
                 self.double_cw * n + self.double_q - 1]
        return np.concatenate(parts).astype(np.int64)


def error_events(seed: int, n: int, num_codewords: int, p1: float, p2: float = 0.0,
                 first_codeword: int = 0) -> ErrorEvents:
    """Per codeword, mutually exclusive: with probability p2 two distinct uniform
    positions flip, else with probability p1 one uniform position flips, else
    nothing.  Draws are keyed by the absolute codeword index, so a sub-range
    reproduces exactly the events of the full stream."""
    N = int(num_codewords)
    u = uniform01(seed, TAG_ERR_KIND, first_codeword, N)
    pos1 = below(seed, TAG_ERR_POS1, first_codeword, N, n) + 1
    pos2 = below(seed, TAG_ERR_POS2, first_codeword, N, max(n - 1, 1)) + 1
    pos2 = np.where(pos2 >= pos1, pos2 + 1, pos2)  # distinct from pos1
    cw = np.arange(first_codeword, first_codeword + N, dtype=np.int64)
    dbl = u < p2
    sgl = (~dbl) & (u < p2 + p1)
    return ErrorEvents(n=n, num_codewords=N,
                       single_cw=cw[sgl], single_pos=pos1[sgl],
                       double_cw=cw[dbl], double_p=pos1[dbl], double_q=pos2[dbl])


def flip_bits(words: np.ndarray, bit_index: np.ndarray, base_bit: int = 0) -> None:
    """XOR-in a 1 at each stream bit ``bit_index - base_bit`` of ``words`` (in place)."""
    b = np.asarray(bit_index, dtype=np.int64) - np.int64(base_bit)
    if b.size == 0:
        return
    np.bitwise_xor.at(words, b >> 5, (np.uint32(1) << (b & 31).astype(np.uint32)))


def apply_errors(words: np.ndarray, ev: ErrorEvents, first_codeword: int = 0) -> None:
    """Flip the event bits of ``ev`` in a stream that starts at codeword ``first_codeword``."""
    flip_bits(words, ev.stream_bits(), base_bit=first_codeword * ev.n)


# ---------------------------------------------------------------------------
# Workload tables for the batched and serving configurations
# ---------------------------------------------------------------------------
CODE_LENGTHS = (7, 15, 31, 63, 127, 255)


@dataclass
class PacketSpec:
    n: int
    num_codewords: int


def packet_table(seed: int, num_packets: int, min_bits: int = 64, max_bits: int = 4 * 1024 * 1024,
                 lengths=CODE_LENGTHS) -> list[PacketSpec]:
    """Packets with n uniform over ``lengths`` and a bit length log-uniform on
    [min_bits, max_bits], rounded to the nearest whole number of codewords (at least 1)."""
    nsel = below(seed, TAG_PKT_N, 0, num_packets, len(lengths))
    u = uniform01(seed, TAG_PKT_LEN, 0, num_packets)
    lo, hi = math.log(min_bits), math.log(max_bits)
    L = np.exp(lo + u * (hi - lo))
    out = []
    for j in range(num_packets):
        n = lengths[int(nsel[j])]
        out.append(PacketSpec(n=n, num_codewords=max(1, int(round(L[j] / n)))))
    return out


def poisson_arrivals(seed: int, count: int, rate_per_s: float) -> np.ndarray:
    """Arrival times in seconds (cumulative exponential gaps) of a Poisson process."""
    u = uniform01(seed, TAG_ARRIVAL, 0, count)
    gaps = -np.log1p(-u) / float(rate_per_s)
    return np.cumsum(gaps)
