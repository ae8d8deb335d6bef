"""CPU oracle for the Hamming decoder -- TEST INFRASTRUCTURE ONLY.

A bit-by-bit C restatement of the paper's decoder (``hd_oracle.c``) behind
ctypes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package; the decoder product never does.

The shared library is compiled here with the system C compiler (plain C99, no
target-specific flags, so it builds the same on x86-64 and aarch64).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hd_oracle.c")
LIB_PATH = os.path.join(_HERE, "libhd_oracle.so")

SYN_NONE, SYN_U8, SYN_U16 = 0, 1, 2
_lock = threading.Lock()


def build(force: bool = False, src: str = _SRC, out: str = LIB_PATH) -> str:
    """Compile ``hd_oracle.c`` into ``libhd_oracle.so`` (skipped when up to date)."""
    with _lock:
        if (not force and os.path.exists(out)
                and os.path.getmtime(out) >= os.path.getmtime(src)):
            return out
        tmp = out + f".tmp{os.getpid()}"
        cc = os.environ.get("CC", "gcc")
        subprocess.check_call([cc, "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, out)
        return out


def _u32p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def words_for(bits: int) -> int:
    return (int(bits) + 31) // 32


class Oracle:
    """ctypes front end of one build of the oracle library."""

    SYN_NONE, SYN_U8, SYN_U16 = SYN_NONE, SYN_U8, SYN_U16

    def __init__(self, path: str):
        L = ctypes.CDLL(path)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.hd_ref_num_checksum_bits.argtypes = [ctypes.c_uint32]
        L.hd_ref_num_checksum_bits.restype = ctypes.c_int
        L.hd_ref_decode_range.argtypes = [u32p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                          u32p, ctypes.c_void_p, ctypes.c_int, u64p]
        L.hd_ref_decode_range.restype = ctypes.c_int
        L.hd_ref_decode.argtypes = [u32p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                    u32p, ctypes.c_void_p, ctypes.c_int, u64p]
        L.hd_ref_decode.restype = ctypes.c_int
        L.hd_ref_encode.argtypes = [u32p, ctypes.c_uint32, ctypes.c_uint64, u32p]
        L.hd_ref_encode.restype = ctypes.c_int
        L.hd_ref_short_checksum_bits.argtypes = [ctypes.c_uint32]
        L.hd_ref_short_checksum_bits.restype = ctypes.c_int
        L.hd_ref_decode_short.argtypes = [u32p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, u32p,
                                          ctypes.c_void_p, ctypes.c_int, u64p, u64p]
        L.hd_ref_decode_short.restype = ctypes.c_int
        L.hd_ref_decode_short_range.argtypes = [u32p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, u32p,
                                                ctypes.c_void_p, ctypes.c_int, u64p, u64p]
        L.hd_ref_decode_short_range.restype = ctypes.c_int
        L.hd_ref_encode_short.argtypes = [u32p, ctypes.c_uint32, ctypes.c_uint64, u32p]
        L.hd_ref_encode_short.restype = ctypes.c_int
        L.hd_ref_decode_secded.argtypes = [u32p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, u32p,
                                           ctypes.c_void_p, ctypes.c_int, u64p, u64p]
        L.hd_ref_decode_secded.restype = ctypes.c_int
        L.hd_ref_decode_secded_range.argtypes = [u32p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, u32p,
                                                 ctypes.c_void_p, ctypes.c_int, u64p, u64p]
        L.hd_ref_decode_secded_range.restype = ctypes.c_int
        L.hd_ref_encode_secded.argtypes = [u32p, ctypes.c_uint32, ctypes.c_uint64, u32p]
        L.hd_ref_encode_secded.restype = ctypes.c_int
        self.lib = L
        self.path = path

    def num_checksum_bits(self, n: int) -> int:
        return self.lib.hd_ref_num_checksum_bits(n)

    def params(self, n: int) -> tuple[int, int]:
        """(m, k) of the full-length code of length n."""
        m = self.num_checksum_bits(n)
        if m == 0:
            raise ValueError(f"unsupported code length n={n}")
        return m, n - m

    def encode(self, data_words: np.ndarray, n: int, num_codewords: int) -> np.ndarray:
        """Encode ``num_codewords`` messages of k bits each (packed LSB first)."""
        m, k = self.params(n)
        data = np.ascontiguousarray(data_words, dtype=np.uint32)
        if data.size < words_for(num_codewords * k):
            raise ValueError("data buffer too small")
        out = np.zeros(max(1, words_for(num_codewords * n)), dtype=np.uint32)
        rc = self.lib.hd_ref_encode(_u32p(data), n, num_codewords, _u32p(out))
        if rc != 0:
            raise RuntimeError(f"hd_ref_encode failed: {rc}")
        return out[:words_for(num_codewords * n)]

    def decode(self, stream: np.ndarray, n: int, num_codewords: int, syn_type: int = SYN_U8,
               in_bits: int | None = None):
        """Decode a whole stream.  Returns (data words, syndromes or None, err_count)."""
        m, k = self.params(n)
        s = np.ascontiguousarray(stream, dtype=np.uint32)
        out = np.zeros(max(1, words_for(num_codewords * k)), dtype=np.uint32)
        syn = None
        if syn_type == SYN_U8:
            syn = np.zeros(max(1, num_codewords), dtype=np.uint8)
        elif syn_type == SYN_U16:
            syn = np.zeros(max(1, num_codewords), dtype=np.uint16)
        err = ctypes.c_uint64(0)
        bits = n * num_codewords if in_bits is None else in_bits
        rc = self.lib.hd_ref_decode(_u32p(s), bits, n, num_codewords, _u32p(out),
                                    None if syn is None else syn.ctypes.data_as(ctypes.c_void_p),
                                    syn_type, ctypes.byref(err))
        if rc != 0:
            raise RuntimeError(f"hd_ref_decode failed: {rc}")
        out = out[:words_for(num_codewords * k)]
        if syn is not None:
            syn = syn[:num_codewords]
        return out, syn, int(err.value)

    def decode_rc(self, stream: np.ndarray, in_bits: int, n: int, num_codewords: int) -> int:
        """Status code of a whole-stream decode (for argument-check tests)."""
        k = max(0, n - max(self.num_checksum_bits(n), 0))
        s = np.ascontiguousarray(stream, dtype=np.uint32)
        out = np.zeros(max(1, words_for(num_codewords * k)), dtype=np.uint32)
        err = ctypes.c_uint64(0)
        return self.lib.hd_ref_decode(_u32p(s), in_bits, n, num_codewords, _u32p(out), None,
                                      SYN_NONE, ctypes.byref(err))

    # -- shortened codes (any length n >= 3) --------------------------------
    def short_params(self, n: int) -> tuple[int, int]:
        """(r, k) of the shortened code of length n."""
        r = self.lib.hd_ref_short_checksum_bits(n)
        if r == 0:
            raise ValueError(f"unsupported shortened length n={n}")
        return r, n - r

    def encode_short(self, data_words: np.ndarray, n: int, num_codewords: int) -> np.ndarray:
        r, k = self.short_params(n)
        data = np.ascontiguousarray(data_words, dtype=np.uint32)
        if data.size < words_for(num_codewords * k):
            raise ValueError("data buffer too small")
        out = np.zeros(max(1, words_for(num_codewords * n)), dtype=np.uint32)
        rc = self.lib.hd_ref_encode_short(_u32p(data), n, num_codewords, _u32p(out))
        if rc != 0:
            raise RuntimeError(f"hd_ref_encode_short failed: {rc}")
        return out[:words_for(num_codewords * n)]

    def decode_short(self, stream: np.ndarray, n: int, num_codewords: int, syn_type: int = SYN_U16,
                     threads: int = 1):
        """Decode a shortened-code stream: (data words, syndromes, err_count, detected);
        err_count counts nonzero syndromes, detected those past n."""
        r, k = self.short_params(n)
        s = np.ascontiguousarray(stream, dtype=np.uint32)
        out = np.zeros(max(1, words_for(num_codewords * k)), dtype=np.uint32)
        syn = None
        if syn_type == SYN_U8:
            syn = np.zeros(max(1, num_codewords), dtype=np.uint8)
        elif syn_type == SYN_U16:
            syn = np.zeros(max(1, num_codewords), dtype=np.uint16)
        synp = None if syn is None else syn.ctypes.data_as(ctypes.c_void_p)
        if threads <= 1 or num_codewords < 64:
            ce, de = ctypes.c_uint64(0), ctypes.c_uint64(0)
            rc = self.lib.hd_ref_decode_short(_u32p(s), n * num_codewords, n, num_codewords, _u32p(out), synp,
                                              syn_type, ctypes.byref(ce), ctypes.byref(de))
            if rc != 0:
                raise RuntimeError(f"hd_ref_decode_short failed: {rc}")
            c, d = int(ce.value), int(de.value)
        else:
            per = max(32, ((num_codewords + threads - 1) // threads + 31) // 32 * 32)
            ranges = [(a, min(per, num_codewords - a)) for a in range(0, num_codewords, per)]

            def run(rg):
                ce, de = ctypes.c_uint64(0), ctypes.c_uint64(0)
                rc = self.lib.hd_ref_decode_short_range(_u32p(s), n, rg[0], rg[1], _u32p(out), synp, syn_type,
                                                        ctypes.byref(ce), ctypes.byref(de))
                if rc != 0:
                    raise RuntimeError(f"hd_ref_decode_short_range failed: {rc}")
                return int(ce.value), int(de.value)

            with ThreadPoolExecutor(max_workers=threads) as ex:
                res = list(ex.map(run, ranges))
            c, d = sum(x[0] for x in res), sum(x[1] for x in res)
        out = out[:words_for(num_codewords * k)]
        if syn is not None:
            syn = syn[:num_codewords]
        return out, syn, c, d

    # -- SECDED: full-length code plus an overall parity bit at position 0 ---
    def encode_secded(self, data_words: np.ndarray, n: int, num_codewords: int) -> np.ndarray:
        m = self.lib.hd_ref_num_checksum_bits(n)
        if m == 0:
            raise ValueError(f"unsupported n={n}")
        k = n - m
        data = np.ascontiguousarray(data_words, dtype=np.uint32)
        if data.size < words_for(num_codewords * k):
            raise ValueError("data buffer too small")
        out = np.zeros(max(1, words_for(num_codewords * (n + 1))), dtype=np.uint32)
        rc = self.lib.hd_ref_encode_secded(_u32p(data), n, num_codewords, _u32p(out))
        if rc != 0:
            raise RuntimeError(f"hd_ref_encode_secded failed: {rc}")
        return out[:words_for(num_codewords * (n + 1))]

    def decode_secded(self, stream: np.ndarray, n: int, num_codewords: int, syn_type: int = SYN_U16,
                      threads: int = 1):
        """Decode an extended-Hamming stream: (data words, syndromes, err_count, detected).
        Syndrome values are s | P << m."""
        m = self.lib.hd_ref_num_checksum_bits(n)
        if m == 0:
            raise ValueError(f"unsupported n={n}")
        k = n - m
        s = np.ascontiguousarray(stream, dtype=np.uint32)
        out = np.zeros(max(1, words_for(num_codewords * k)), dtype=np.uint32)
        syn = None
        if syn_type == SYN_U8:
            syn = np.zeros(max(1, num_codewords), dtype=np.uint8)
        elif syn_type == SYN_U16:
            syn = np.zeros(max(1, num_codewords), dtype=np.uint16)
        synp = None if syn is None else syn.ctypes.data_as(ctypes.c_void_p)
        if threads <= 1 or num_codewords < 64:
            ce, de = ctypes.c_uint64(0), ctypes.c_uint64(0)
            rc = self.lib.hd_ref_decode_secded(_u32p(s), (n + 1) * num_codewords, n, num_codewords, _u32p(out),
                                               synp, syn_type, ctypes.byref(ce), ctypes.byref(de))
            if rc != 0:
                raise RuntimeError(f"hd_ref_decode_secded failed: {rc}")
            c, d = int(ce.value), int(de.value)
        else:
            per = max(32, ((num_codewords + threads - 1) // threads + 31) // 32 * 32)
            ranges = [(a, min(per, num_codewords - a)) for a in range(0, num_codewords, per)]

            def run(rg):
                ce, de = ctypes.c_uint64(0), ctypes.c_uint64(0)
                rc = self.lib.hd_ref_decode_secded_range(_u32p(s), n, rg[0], rg[1], _u32p(out), synp, syn_type,
                                                         ctypes.byref(ce), ctypes.byref(de))
                if rc != 0:
                    raise RuntimeError(f"hd_ref_decode_secded_range failed: {rc}")
                return int(ce.value), int(de.value)

            with ThreadPoolExecutor(max_workers=threads) as ex:
                res = list(ex.map(run, ranges))
            c, d = sum(x[0] for x in res), sum(x[1] for x in res)
        out = out[:words_for(num_codewords * k)]
        if syn is not None:
            syn = syn[:num_codewords]
        return out, syn, c, d

    def decode_threaded(self, stream: np.ndarray, n: int, num_codewords: int, syn_type: int,
                        threads: int, out: np.ndarray, syn: np.ndarray | None) -> int:
        """Decode with ``threads`` host threads over 32-codeword-aligned ranges.

        The C calls release the GIL, so the ranges run in parallel.  Range
        starts are multiples of 32 codewords, so every range starts on an output
        word boundary and no two threads write the same word.  Returns
        err_count; the output pad bits are not touched (callers pass a zeroed
        buffer)."""
        L = self.lib
        s = np.ascontiguousarray(stream, dtype=np.uint32)
        per = max(32, ((num_codewords + threads - 1) // threads + 31) // 32 * 32)
        ranges = [(a, min(per, num_codewords - a)) for a in range(0, num_codewords, per)]
        synp = None if syn is None else syn.ctypes.data_as(ctypes.c_void_p)

        def run(r):
            e = ctypes.c_uint64(0)
            rc = L.hd_ref_decode_range(_u32p(s), n, r[0], r[1], _u32p(out), synp, syn_type,
                                       ctypes.byref(e))
            if rc != 0:
                raise RuntimeError(f"hd_ref_decode_range failed: {rc}")
            return int(e.value)

        with ThreadPoolExecutor(max_workers=threads) as ex:
            return sum(ex.map(run, ranges))


_default = None


def default() -> Oracle:
    """The oracle built from this directory's source."""
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


def params(n):
    return default().params(n)


def num_checksum_bits(n):
    return default().num_checksum_bits(n)


def encode(data_words, n, num_codewords):
    return default().encode(data_words, n, num_codewords)


def decode(stream, n, num_codewords, syn_type=SYN_U8, in_bits=None):
    return default().decode(stream, n, num_codewords, syn_type, in_bits)


def decode_rc(stream, in_bits, n, num_codewords):
    return default().decode_rc(stream, in_bits, n, num_codewords)


def decode_threaded(stream, n, num_codewords, syn_type, threads, out, syn):
    return default().decode_threaded(stream, n, num_codewords, syn_type, threads, out, syn)


def short_params(n):
    return default().short_params(n)


def encode_short(data_words, n, num_codewords):
    return default().encode_short(data_words, n, num_codewords)


def decode_short(stream, n, num_codewords, syn_type=SYN_U16, threads=1):
    return default().decode_short(stream, n, num_codewords, syn_type, threads)


def encode_secded(data_words, n, num_codewords):
    return default().encode_secded(data_words, n, num_codewords)


def decode_secded(stream, n, num_codewords, syn_type=SYN_U16, threads=1):
    return default().decode_secded(stream, n, num_codewords, syn_type, threads)
