"""Independent numpy formulations used by the tests to pin the oracle.

These restate the code through its parity-check matrix H (column p holds the
binary expansion of p, so H c^T is the checksum vector of Sec. III-A) and
through plain bit-array indexing, a different formulation from the oracle's
per-bit XOR-of-positions loop.  They are test helpers only.
"""
import numpy as np


def m_of(n: int) -> int:
    m = (n + 1).bit_length() - 1
    assert (1 << m) - 1 == n, n
    return m


def parity_check_matrix(n: int) -> np.ndarray:
    """m x n matrix over GF(2): H[j, p-1] = bit j of p."""
    m = m_of(n)
    p = np.arange(1, n + 1)
    return ((p[None, :] >> np.arange(m)[:, None]) & 1).astype(np.int64)


def data_positions(n: int) -> np.ndarray:
    """Non-power-of-two positions 1..n in increasing order."""
    p = np.arange(1, n + 1)
    return p[(p & (p - 1)) != 0]


def words_to_bits(words: np.ndarray, nbits: int) -> np.ndarray:
    """LSB-first unpack of uint32 words into a uint8 bit array of length nbits."""
    b = np.unpackbits(np.ascontiguousarray(words, dtype="<u4").view(np.uint8), bitorder="little")
    return b[:nbits]


def bits_to_words(bits: np.ndarray) -> np.ndarray:
    nb = bits.size
    pad = (-nb) % 32
    b = np.concatenate([bits.astype(np.uint8), np.zeros(pad, np.uint8)])
    return np.packbits(b, bitorder="little").view("<u4").astype(np.uint32)


def codeword_matrix(stream: np.ndarray, n: int, N: int) -> np.ndarray:
    """N x n bit matrix; column p-1 is position p."""
    return words_to_bits(stream, N * n).reshape(N, n)


def syndromes(stream: np.ndarray, n: int, N: int) -> np.ndarray:
    """Checksum vectors as integers: sum_j 2^j (H r^T)_j mod 2."""
    H = parity_check_matrix(n)
    R = codeword_matrix(stream, n, N).astype(np.int64)
    S = (R @ H.T) & 1
    return (S << np.arange(H.shape[0])[None, :]).sum(axis=1)


def decode(stream: np.ndarray, n: int, N: int):
    """Matrix-form single-error-correcting decode: (data words, syndromes, err_count)."""
    R = codeword_matrix(stream, n, N).copy()
    s = syndromes(stream, n, N)
    rows = np.nonzero(s)[0]
    R[rows, s[rows] - 1] ^= 1
    D = R[:, data_positions(n) - 1]
    return bits_to_words(D.reshape(-1)), s, int(rows.size)


# -- shortened codes: any length n, r = the smallest count with 2^r >= n + 1 --
def short_r(n: int) -> int:
    r = 0
    while (1 << r) < n + 1:
        r += 1
    return r


def short_parity_check_matrix(n: int) -> np.ndarray:
    """r x n matrix over GF(2): column p-1 holds the binary expansion of p."""
    r = short_r(n)
    p = np.arange(1, n + 1)
    return ((p[None, :] >> np.arange(r)[:, None]) & 1).astype(np.int64)


def short_syndromes(stream: np.ndarray, n: int, N: int) -> np.ndarray:
    H = short_parity_check_matrix(n)
    R = codeword_matrix(stream, n, N).astype(np.int64)
    S = (R @ H.T) & 1
    return (S << np.arange(H.shape[0])[None, :]).sum(axis=1)


def short_decode(stream: np.ndarray, n: int, N: int):
    """Matrix-form decode of a shortened code: a syndrome s <= n flips position
    s, a larger one flips nothing.  Returns (data words, syndromes, err_count,
    detected) with err_count = nonzero syndromes, detected = syndromes > n."""
    R = codeword_matrix(stream, n, N).copy()
    s = short_syndromes(stream, n, N)
    fix = np.nonzero((s != 0) & (s <= n))[0]
    R[fix, s[fix] - 1] ^= 1
    D = R[:, data_positions(n) - 1]
    return bits_to_words(D.reshape(-1)), s, int(np.count_nonzero(s)), int(np.count_nonzero(s > n))
