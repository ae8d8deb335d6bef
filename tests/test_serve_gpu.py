"""Serving loop (continuous batching): every packet's result through the
server, mixed with others in waves, is bit-identical to decoding it alone."""
import numpy as np
import pytest

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


def _mixed(num, seed):
    import torch
    lengths = (3, 7, 15, 31, 63, 127, 255)
    ns = synth.below(seed, 31, 0, num, len(lengths))
    lens = synth.below(seed, 32, 0, num, 20000)
    sts = synth.below(seed, 33, 0, num, 3)
    pk = []
    for j in range(num):
        n, N, st = lengths[int(ns[j])], int(lens[j]) + 1, int(sts[j])
        m, k = hd.code_params(n)
        stream, _, _ = gc.received_stream(n, N, seed=seed * 1000 + j, p1=0.1, p2=0.02)
        d_in = gc.to_device(stream)
        alone = hd.decode(d_in, n, N, syn_type=st)
        out = torch.full((hd.words_for(N * k),), -1, dtype=torch.int32, device="cuda")
        syn = None if st == 0 else torch.full((N,), 0x77, dtype=torch.uint8 if st == 1 else torch.int16,
                                              device="cuda")
        pk.append(dict(n=n, N=N, st=st, d_in=d_in, alone=alone, out=out, syn=syn))
    torch.cuda.synchronize()
    return pk


def _same(p, err_count):
    ao, asyn, aerr = p["alone"]
    assert np.array_equal(gc.host_u32(p["out"]), gc.host_u32(ao)[:p["out"].numel()])
    if p["st"] != 0:
        assert np.array_equal(p["syn"].cpu().numpy(), asyn.cpu().numpy()[:p["N"]])
    assert err_count == int(aerr.item())


def test_trace_results_identical_alone_and_in_the_mix():
    num = 400
    pk = _mixed(num, seed=7)
    table = hd.packet_table([(p["d_in"].data_ptr(), p["out"].data_ptr(),
                              None if p["syn"] is None else p["syn"].data_ptr(), p["N"], p["n"], p["st"]) for p in pk])
    arrivals = synth.poisson_arrivals(1, num, 2e5)  # dense enough that waves mix packets
    cfg = hd.server_config(max_waves=4, max_wave_packets=64, max_wave_tiles=8192, queue_capacity=1024)
    comps, stats = hd.hd_serve_trace(cfg, table, arrivals, num)
    assert stats["completed"] == num and stats["waves"] >= 2
    assert stats["mean_wave_packets"] > 1.0, "the trace should mix packets in waves"
    for j, p in enumerate(pk):
        assert comps[j].tag == j and comps[j].status == hd.HD_OK
        assert comps[j].t_done_ns >= comps[j].t_admit_ns >= comps[j].t_submit_ns
        _same(p, comps[j].err_count)
    assert stats["p99_latency_us"] >= stats["p50_latency_us"] > 0


def test_server_submit_poll_drain_and_budget():
    pk = _mixed(60, seed=8)
    cost = [(p["N"] * p["n"] + 7) // 8 + (p["N"] * hd.code_params(p["n"])[1] + 7) // 8 + 2 * p["N"] for p in pk]
    budget = 2 * max(cost)  # room for about two packets at a time: admission must wait for completions
    srv = hd.Server(hd.server_config(max_waves=2, max_wave_packets=8, max_wave_tiles=4096, queue_capacity=256,
                                     mem_cap_bytes=budget))
    for j, p in enumerate(pk):
        rc = srv.submit(p["d_in"].data_ptr(), p["out"].data_ptr(), 0 if p["syn"] is None else p["syn"].data_ptr(),
                        p["N"], p["n"], p["st"], 1000 + j)
        assert rc == hd.HD_OK
    assert srv.drain(60.0) == hd.HD_OK
    rc, comps = srv.poll(1000)
    assert rc == hd.HD_OK and len(comps) == len(pk)
    st = srv.stats()
    assert st["max_resident_bytes"] <= budget  # the admission budget held
    for c in comps:
        _same(pk[c.tag - 1000], c.err_count)
    # a packet larger than the whole budget is refused up front
    big = pk[0]
    huge_N = budget * 8  # far beyond the budget in bytes
    assert srv.submit(big["d_in"].data_ptr(), big["out"].data_ptr(), 0, huge_N, 7, 0, 1) == hd.HD_ERR_CAPACITY
    assert srv.submit(big["d_in"].data_ptr(), big["out"].data_ptr(), 0, 10, 8, 0, 1) == hd.HD_ERR_INVALID_N
    srv.close()


def test_drain_waits_for_every_admitted_packet():
    # admission moves requests out of the queue and marks their wave busy atomically, so a
    # drain that returns HD_OK has every completion ready to poll (repeated to give a race
    # between admission and drain many chances)
    pk = _mixed(24, seed=13)
    for rep in range(25):
        srv = hd.Server(hd.server_config(max_waves=3, max_wave_packets=4, max_wave_tiles=4096, queue_capacity=256,
                                         mem_cap_bytes=1 << 34))
        try:
            for j, p in enumerate(pk):
                assert srv.submit(p["d_in"].data_ptr(), p["out"].data_ptr(),
                                  0 if p["syn"] is None else p["syn"].data_ptr(), p["N"], p["n"], p["st"],
                                  j) == hd.HD_OK
            assert srv.drain(60.0) == hd.HD_OK
            rc, comps = srv.poll(1000)
            assert rc == hd.HD_OK and len(comps) == len(pk), (rep, len(comps))
        finally:
            srv.close()


def test_wave_tile_limit_counts_short_chunks_exactly():
    # n = 255 packets of 7,680 codewords are exactly 60 tiles each (half-warp
    # chunks of 128 codewords), so a 64-tile wave holds one of them: admission
    # must count the tiles as the batch plan cuts them, never two per wave
    import torch
    n, N = 255, 128 * 60
    m, k = hd.code_params(n)
    pk = []
    for j in range(4):
        stream, _, _ = gc.received_stream(n, N, seed=900 + j, p1=0.1, p2=0.02)
        d_in = gc.to_device(stream)
        alone = hd.decode(d_in, n, N, syn_type=hd.SYN_U16)
        out = torch.full((hd.words_for(N * k),), -1, dtype=torch.int32, device="cuda")
        syn = torch.full((N,), 0x77, dtype=torch.int16, device="cuda")
        pk.append(dict(n=n, N=N, st=hd.SYN_U16, d_in=d_in, alone=alone, out=out, syn=syn))
    torch.cuda.synchronize()
    srv = hd.Server(hd.server_config(max_waves=2, max_wave_packets=8, max_wave_tiles=64, queue_capacity=16))
    for j, p in enumerate(pk):
        assert srv.submit(p["d_in"].data_ptr(), p["out"].data_ptr(), p["syn"].data_ptr(), N, n, p["st"], j) == hd.HD_OK
    assert srv.drain(60.0) == hd.HD_OK
    rc, comps = srv.poll(16)
    assert rc == hd.HD_OK and len(comps) == len(pk)
    assert srv.stats()["waves"] >= len(pk)  # one packet per wave
    for c in comps:
        assert c.status == hd.HD_OK
        _same(pk[c.tag], c.err_count)
    srv.close()
