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


def _host_mixed(num, seed):
    """Packets in pinned host memory (mixed n, lengths and syndrome types) and
    the oracle's decode of each."""
    import torch
    import oracle
    lengths = (3, 7, 15, 31, 63, 127, 255)
    ns = synth.below(seed, 41, 0, num, len(lengths))
    lens = synth.below(seed, 42, 0, num, 20000)
    sts = synth.below(seed, 43, 0, num, 3)
    pk = []
    for j in range(num):
        n, N, st = lengths[int(ns[j])], int(lens[j]) + 1, int(sts[j])
        m, k = hd.code_params(n)
        stream, _, _ = gc.received_stream(n, N, seed=seed * 1000 + j, p1=0.1, p2=0.02)
        h_in = torch.from_numpy(stream.view(np.int32).copy()).pin_memory()
        out = torch.full((hd.words_for(N * k),), -1, dtype=torch.int32).pin_memory()
        syn = None if st == 0 else torch.full((N,), 0x77, dtype=torch.uint8 if st == 1 else torch.int16).pin_memory()
        want = oracle.decode(stream, n, N, syn_type=st)
        pk.append(dict(n=n, N=N, st=st, h_in=h_in, out=out, syn=syn, want=want))
    return pk


def _host_row(p):
    return (p["h_in"].data_ptr(), p["out"].data_ptr(), None if p["syn"] is None else p["syn"].data_ptr(), p["N"],
            p["n"], p["st"])


def _matches_oracle(p, err_count):
    eo, es, ee = p["want"]
    assert np.array_equal(p["out"].numpy().view(np.uint32), eo), "data bits differ from the oracle"
    if p["st"] != 0:
        got = p["syn"].numpy()
        assert np.array_equal(got.view(np.uint16) if p["st"] == 2 else got, es), "syndromes differ from the oracle"
    assert err_count == ee


def _reset(pk):
    for p in pk:
        p["out"].fill_(-1)
        if p["syn"] is not None:
            p["syn"].fill_(0x77)


def test_host_packets_match_the_oracle_alone_and_in_the_mix():
    """Packets submitted from pinned host memory: gathered into the slot's
    staging, decoded and scattered back.  Each result equals the oracle's,
    whether the packet is served in a wave of its own or mixed with others."""
    num = 160
    pk = _host_mixed(num, seed=21)
    table = hd.packet_table([_host_row(p) for p in pk])
    # in the mix: dense arrivals, up to 64 packets per wave, four slots
    arrivals = synth.poisson_arrivals(3, num, 2e5)
    cfg = hd.server_config(max_waves=4, max_wave_packets=64, max_wave_tiles=8192, queue_capacity=1024,
                           host_staging_bytes=32 << 20)
    comps, stats = hd.hd_serve_trace(cfg, table, arrivals, num, host=True)
    assert stats["completed"] == num and stats["mean_wave_packets"] > 1.0
    assert stats["host_waves"] == stats["waves"] > 0
    assert stats["mean_t_in_us"] > 0 and stats["mean_t_decode_us"] > 0 and stats["mean_t_out_us"] > 0
    for j, p in enumerate(pk):
        assert comps[j].tag == j and comps[j].status == hd.HD_OK
        _matches_oracle(p, comps[j].err_count)
    # alone: one packet per wave, each drained before the next is submitted
    _reset(pk)
    srv = hd.Server(hd.server_config(max_waves=2, max_wave_packets=1, max_wave_tiles=8192, queue_capacity=16,
                                     host_staging_bytes=32 << 20))
    try:
        for j, p in enumerate(pk):
            a, b, c, N, n, st = _host_row(p)
            assert srv.submit_host(a, b, c or 0, N, n, st, j) == hd.HD_OK
            assert srv.drain(60.0) == hd.HD_OK
            rc, cs = srv.poll(4)
            assert rc == hd.HD_OK and len(cs) == 1 and cs[0].tag == j and cs[0].status == hd.HD_OK
            _matches_oracle(p, cs[0].err_count)
        assert srv.stats()["waves"] == num
    finally:
        srv.close()
    assert hd.hd_device_status() == 0


def test_mixed_device_and_host_packets_in_one_server():
    import torch
    dev_pk = _mixed(40, seed=22)
    host_pk = _host_mixed(40, seed=23)
    srv = hd.Server(hd.server_config(max_waves=3, max_wave_packets=16, max_wave_tiles=8192, queue_capacity=256,
                                     host_staging_bytes=16 << 20))
    try:
        for j in range(40):
            p = dev_pk[j]
            assert srv.submit(p["d_in"].data_ptr(), p["out"].data_ptr(), 0 if p["syn"] is None else
                              p["syn"].data_ptr(), p["N"], p["n"], p["st"], j) == hd.HD_OK
            a, b, c, N, n, st = _host_row(host_pk[j])
            assert srv.submit_host(a, b, c or 0, N, n, st, 100 + j) == hd.HD_OK
        assert srv.drain(60.0) == hd.HD_OK
        rc, comps = srv.poll(1000)
        assert rc == hd.HD_OK and len(comps) == 80
        torch.cuda.synchronize()
        for c in comps:
            assert c.status == hd.HD_OK
            if c.tag < 100:
                _same(dev_pk[c.tag], c.err_count)
            else:
                _matches_oracle(host_pk[c.tag - 100], c.err_count)
    finally:
        srv.close()


def test_host_submission_refuses_unpinned_or_unstaged_buffers():
    import torch
    p = _host_mixed(1, seed=24)[0]
    a, b, c, N, n, st = _host_row(p)
    srv = hd.Server(hd.server_config(max_waves=1, max_wave_packets=4, max_wave_tiles=4096, queue_capacity=16))
    try:  # no host staging configured
        assert srv.submit_host(a, b, c or 0, N, n, st, 0) == hd.HD_ERR_INVALID_ARG
    finally:
        srv.close()
    srv = hd.Server(hd.server_config(max_waves=1, max_wave_packets=4, max_wave_tiles=4096, queue_capacity=16,
                                     host_staging_bytes=1 << 20))
    try:
        pageable = np.zeros(N * n // 32 + 8, np.uint32)
        assert srv.submit_host(int(pageable.ctypes.data), b, c or 0, N, n, st, 0) == hd.HD_ERR_INVALID_ARG
        dev = torch.zeros(N * n // 32 + 8, dtype=torch.int32, device="cuda")
        assert srv.submit_host(dev.data_ptr(), b, c or 0, N, n, st, 0) == hd.HD_ERR_INVALID_ARG
        big = torch.zeros(1 << 19, dtype=torch.int32).pin_memory()  # 2 MB > 1 MB of staging
        assert srv.submit_host(big.data_ptr(), big.data_ptr(), 0, (1 << 24) // 7, 7, 0, 0) == hd.HD_ERR_CAPACITY
        assert srv.submit_host(a, b, c or 0, N, n, st, 7) == hd.HD_OK
        assert srv.drain(60.0) == hd.HD_OK
        rc, cs = srv.poll(4)
        assert rc == hd.HD_OK and len(cs) == 1
        _matches_oracle(p, cs[0].err_count)
    finally:
        srv.close()


def test_injected_launch_failure_fails_its_packets_and_the_server():
    """A wave launch that fails (injected on the host: nothing of that wave is
    enqueued) completes its packets with HD_ERR_CUDA at once, the server keeps
    the error and completes every waiting packet with it; a new server on the
    same device then serves the same packets correctly."""
    import time
    pk = _mixed(30, seed=25)
    srv = hd.Server(hd.server_config(max_waves=2, max_wave_packets=4, max_wave_tiles=4096, queue_capacity=256))
    try:
        srv.inject_launch_failures(1)
        accepted = 0
        for j, p in enumerate(pk):
            rc = srv.submit(p["d_in"].data_ptr(), p["out"].data_ptr(), 0 if p["syn"] is None else p["syn"].data_ptr(),
                            p["N"], p["n"], p["st"], j)
            assert rc in (hd.HD_OK, hd.HD_ERR_CUDA)
            accepted += rc == hd.HD_OK
        comps, t0 = [], time.time()
        while len(comps) < accepted and time.time() - t0 < 30:
            rc, cs = srv.poll(1000)
            comps += cs
        assert len(comps) == accepted
        assert rc == hd.HD_ERR_CUDA
        assert all(c.status == hd.HD_ERR_CUDA for c in comps[:1])  # at least the failed wave's packets
        bad = [c for c in comps if c.status != hd.HD_OK]
        assert bad, "the injected failure must reach the packets of its wave"
        assert all(c.status == hd.HD_ERR_CUDA and c.err_count == 0 for c in bad)
        assert srv.drain(1.0) == hd.HD_ERR_CUDA
        assert srv.submit(pk[0]["d_in"].data_ptr(), pk[0]["out"].data_ptr(), 0, pk[0]["N"], pk[0]["n"], 0,
                          99) == hd.HD_ERR_CUDA
        st = srv.stats()
        assert st["completed"] == st["submitted"] == accepted
    finally:
        srv.close()
    srv = hd.Server(hd.server_config(max_waves=2, max_wave_packets=4, max_wave_tiles=4096, queue_capacity=256))
    try:
        for j, p in enumerate(pk):
            assert srv.submit(p["d_in"].data_ptr(), p["out"].data_ptr(), 0 if p["syn"] is None else
                              p["syn"].data_ptr(), p["N"], p["n"], p["st"], j) == hd.HD_OK
        assert srv.drain(60.0) == hd.HD_OK
        rc, comps = srv.poll(1000)
        assert rc == hd.HD_OK and len(comps) == len(pk)
        for c in comps:
            assert c.status == hd.HD_OK
            _same(pk[c.tag], c.err_count)
    finally:
        srv.close()
    assert hd.hd_device_status() == 0
