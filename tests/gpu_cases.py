"""Shared helpers of the GPU parity tests: seeded inputs built on the CPU with
the oracle's encoder and the generator's channel errors, expected values from
the oracle, and bit-exact comparison of the GPU outputs."""
import numpy as np

import oracle
from paper_1412_6862_gb300 import synth

M_OF = {3: 2, 7: 3, 15: 4, 31: 5, 63: 6, 127: 7, 255: 8}


def received_stream(n: int, N: int, seed: int = 0, p1: float = 0.1, p2: float = 0.01):
    """Encoded random data with channel errors: (stream words, data words, events)."""
    k = n - M_OF[n]
    data = synth.random_words(seed, N * k)
    stream = oracle.encode(data, n, N) if N else np.zeros(0, np.uint32)
    ev = synth.error_events(seed, n, N, p1=p1, p2=p2)
    synth.apply_errors(stream, ev)
    return stream, data, ev


def expected(stream, n, N, syn_type, threads: int = 8):
    """Oracle decode (threaded for large N): (out words, syndromes, err_count)."""
    k = n - M_OF[n]
    if N < 200000:
        return oracle.decode(stream, n, N, syn_type=syn_type)
    out = np.zeros((N * k + 31) // 32, np.uint32)
    syn = None
    if syn_type == oracle.SYN_U8:
        syn = np.zeros(N, np.uint8)
    elif syn_type == oracle.SYN_U16:
        syn = np.zeros(N, np.uint16)
    err = oracle.decode_threaded(stream, n, N, syn_type, threads, out, syn)
    return out, syn, err


def oracle_encode_parallel(encode, data: np.ndarray, n: int, N: int, k: int, L: int, threads: int = 0):
    """The oracle encoder ``encode(data_words, n, count)`` over N codewords of
    L bits (k data bits each), in host threads over ranges of whole 32-codeword
    groups: every range starts on a word boundary of both the data and the
    stream, so the ranges' words never overlap."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    threads = threads or (os.cpu_count() or 4)
    per = max(32, ((N + threads - 1) // threads + 31) // 32 * 32)
    out = np.zeros((N * L + 31) // 32, np.uint32)

    def part(i0):
        c = min(per, N - i0)
        w = encode(data[i0 * k // 32:(i0 * k + c * k + 31) // 32], n, c)
        o = i0 * L // 32
        out[o:o + w.size] = w

    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(part, range(0, N, per)))
    return out


def to_device(words: np.ndarray, pad_words: int = 0):
    import torch
    a = np.zeros(max(1, words.size + pad_words), np.uint32)
    a[:words.size] = words
    return torch.from_numpy(a.view(np.int32)).cuda()


def host_u32(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def assert_same(gpu, exp, n, N, syn_type):
    out_g, syn_g, err_g = gpu
    out_e, syn_e, err_e = exp
    k = n - M_OF[n]
    nw = (N * k + 31) // 32
    og = host_u32(out_g)[:nw]
    if not np.array_equal(og, out_e[:nw]):
        bad = np.nonzero(og != out_e[:nw])[0]
        raise AssertionError(f"n={n} N={N}: {bad.size} output words differ, first at word {bad[0]} "
                             f"(gpu {og[bad[0]]:#010x} oracle {out_e[bad[0]]:#010x})")
    if syn_type != oracle.SYN_NONE:
        sg = syn_g.cpu().numpy()[:N]
        if syn_type == oracle.SYN_U16:
            sg = sg.view(np.uint16)
        if not np.array_equal(sg, syn_e[:N]):
            bad = np.nonzero(sg != syn_e[:N])[0]
            raise AssertionError(f"n={n} N={N}: {bad.size} syndromes differ, first at {bad[0]}")
    assert int(err_g.item()) == err_e, (n, N, int(err_g.item()), err_e)
