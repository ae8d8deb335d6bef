"""Batched mixed-n decode (plan and one-shot) against the oracle, packet by
packet, in every batch-kernel configuration."""
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


def make_batch(num_packets, seed, max_cw=40000, lengths=(3, 7, 15, 31, 63, 127, 255)):
    """Packets with mixed n, lengths from 0 (a few) to max_cw codewords, mixed
    syndrome types (including none), each in its own device tensors."""
    import torch
    ns = synth.below(seed, 11, 0, num_packets, len(lengths))
    lens = synth.below(seed, 12, 0, num_packets, max_cw + 1)
    logs = synth.uniform01(seed, 13, 0, num_packets)
    stypes = synth.below(seed, 14, 0, num_packets, 3)
    pkts, exp = [], []
    for j in range(num_packets):
        n = lengths[int(ns[j])]
        N = int(lens[j] ** logs[j]) if j % 7 else int(lens[j])  # skew toward short packets
        if j % 29 == 5:
            N = 0
        st = int(stypes[j])
        if n == 255 and st == 1:
            st = 2 if j % 2 else 1
        stream, _, _ = gc.received_stream(n, N, seed=seed * 1000 + j, p1=0.1, p2=0.02)
        e = gc.expected(stream, n, N, st) if N else (np.zeros(0, np.uint32), None, 0)
        m, k = hd.code_params(n)
        d_in = gc.to_device(stream)
        out = torch.full((max(1, hd.words_for(N * k)),), -1, dtype=torch.int32, device="cuda")
        syn = None
        if st != hd.SYN_NONE:
            syn = torch.full((max(1, N),), 0x5A, dtype=torch.uint8 if st == 1 else torch.int16, device="cuda")
        pkts.append((d_in, out, syn, N, n, st))
        exp.append(e)
    return pkts, exp


def check_batch(pkts, exp, err):
    e_h = err.cpu().numpy()
    for j, ((d_in, out, syn, N, n, st), (eo, es, ee)) in enumerate(zip(pkts, exp)):
        if N == 0:
            assert e_h[j] == 0
            continue
        gc.assert_same((out, syn, err[j:j + 1]), (eo, es, ee), n, N, st)


def test_plan_matches_oracle_all_variants():
    import torch
    pkts, exp = make_batch(120, seed=1)
    plan = hd.Plan(pkts)
    info = plan.info()
    assert info["num_packets"] == 120 and info["num_tiles"] >= info["full_tiles"] > 0
    err = torch.full((120,), 77, dtype=torch.int64, device="cuda")
    for v in range(info["num_variants"]):
        plan.select(v)
        for _ in range(2):  # first launch records the graph, the second replays it
            for d_in, out, syn, N, n, st in pkts:
                out.fill_(-1)
            plan.launch(err)
            torch.cuda.synchronize()
            check_batch(pkts, exp, err)
    plan.close()
    assert hd.hd_device_status() == 0


def test_one_shot_batch_matches_oracle():
    import torch
    pkts, exp = make_batch(60, seed=2)
    table = hd.packet_table([(hd._ptr(a), hd._ptr(b), hd._ptr(c), N, n, st) for a, b, c, N, n, st in pkts])
    err = torch.full((60,), 5, dtype=torch.int64, device="cuda")
    rc = hd.hd_decode_batch(table, 60, err.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == hd.HD_OK
    torch.cuda.synchronize()
    check_batch(pkts, exp, err)


def test_plan_autotune_and_long_packets():
    import torch
    # few long packets of every n: many full tiles per packet, ragged tails
    pkts, exp = [], []
    for j, n in enumerate((7, 15, 31, 63, 127, 255)):
        N = 150000 + 37 * j
        st = hd.SYN_U16 if n >= 127 else hd.SYN_U8
        stream, _, _ = gc.received_stream(n, N, seed=50 + j)
        exp.append(gc.expected(stream, n, N, st))
        m, k = hd.code_params(n)
        out = torch.empty(hd.words_for(N * k), dtype=torch.int32, device="cuda")
        syn = torch.empty(N, dtype=torch.uint8 if st == 1 else torch.int16, device="cuda")
        pkts.append((gc.to_device(stream), out, syn, N, n, st))
    plan = hd.Plan(pkts)
    info = plan.autotune(reps=2)
    assert info["measured_us"] > 0
    err = torch.empty(len(pkts), dtype=torch.int64, device="cuda")
    plan.launch(err)
    torch.cuda.synchronize()
    check_batch(pkts, exp, err)
    plan.close()


def test_batched_config_full_size():
    """The batched benchmark configuration at full size (10,000 packets, n
    uniform over six codes, log-uniform lengths up to 4 Mbit), every packet
    compared with the oracle.  Inputs: oracle encoder + generator errors."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    import torch
    specs = synth.packet_table(0, 10000)

    def make(j):
        sp = specs[j]
        m, k = hd.code_params(sp.n)
        data = synth.random_words(j, sp.num_codewords * k)
        s = oracle.encode(data, sp.n, sp.num_codewords)
        synth.apply_errors(s, synth.error_events(j, sp.n, sp.num_codewords, p1=0.05))
        return s, oracle.decode(s, sp.n, sp.num_codewords, syn_type=oracle.SYN_U8)

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        made = list(ex.map(make, range(len(specs))))
    # arenas with 16-byte aligned packets
    offs_in, offs_out, offs_syn, tin, tout, tsyn = [], [], [], 0, 0, 0
    for sp, (s, _) in zip(specs, made):
        m, k = hd.code_params(sp.n)
        offs_in.append(tin)
        offs_out.append(tout)
        offs_syn.append(tsyn)
        tin += (s.size + 3) // 4 * 4
        tout += (hd.words_for(sp.num_codewords * k) + 3) // 4 * 4
        tsyn += (sp.num_codewords + 15) // 16 * 16
    h_in = np.zeros(tin, np.uint32)
    for o, (s, _) in zip(offs_in, made):
        h_in[o:o + s.size] = s
    d_in = torch.from_numpy(h_in.view(np.int32)).cuda()
    d_out = torch.full((tout,), -1, dtype=torch.int32, device="cuda")
    d_syn = torch.full((tsyn,), 0xEE, dtype=torch.uint8, device="cuda")
    rows = [(d_in.data_ptr() + 4 * oi, d_out.data_ptr() + 4 * oo, d_syn.data_ptr() + osy, sp.num_codewords, sp.n,
             hd.SYN_U8) for sp, oi, oo, osy in zip(specs, offs_in, offs_out, offs_syn)]
    table = hd.packet_table(rows)
    plan = hd.hd_plan_create(table, len(rows))
    err = torch.empty(len(rows), dtype=torch.int64, device="cuda")
    try:
        # every configuration the autotuner can pick, at this size
        for v in range(hd.hd_plan_get_info(plan)["num_variants"]):
            hd.hd_plan_select(plan, v)
            d_out.fill_(-1)
            d_syn.fill_(0xEE)
            err.fill_(-1)
            assert hd.hd_plan_launch(plan, err.data_ptr(), torch.cuda.current_stream().cuda_stream) == hd.HD_OK
            torch.cuda.synchronize()
            o_h = d_out.cpu().numpy().view(np.uint32)
            s_h = d_syn.cpu().numpy()
            e_h = err.cpu().numpy()
            for j, (sp, (s, (eo, es, ee))) in enumerate(zip(specs, made)):
                m, k = hd.code_params(sp.n)
                nw = hd.words_for(sp.num_codewords * k)
                assert np.array_equal(o_h[offs_out[j]:offs_out[j] + nw], eo[:nw]), \
                    f"configuration {v}, packet {j} (n={sp.n}) data bits"
                assert np.array_equal(s_h[offs_syn[j]:offs_syn[j] + sp.num_codewords], es), \
                    f"configuration {v}, packet {j} syndromes"
                assert e_h[j] == ee, f"configuration {v}, packet {j} err_count"
    finally:
        hd.hd_plan_destroy(plan)
    assert hd.hd_device_status() == 0
