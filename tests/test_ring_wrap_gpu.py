"""Every compiled kernel configuration, with every warp walking many chunks.

The persistent decoders size their grid to the device (SMs x resident CTAs),
so on inputs small enough for the CPU oracle each warp would see at most one
chunk or tile and its staging ring would never wrap: the mbarrier phase flip,
the in-place refill one iteration behind and the claim pipeline of the batch
kernel would go untested.  hd_set_max_ctas() caps the grid instead, and each
case below sizes its input so that every warp of the configuration under
test runs at least S + 2 iterations, then compares every output element with
the oracle: the streaming decoder (arithmetic and decode-table
configurations, every syndrome type), the SECDED decoder (every
configuration), the batch kernel (every configuration) and the shortened-code
tiled kernel (every configuration, each table placement)."""
import numpy as np
import pytest

import oracle
from paper_1412_6862_gb300 import hd, synth
from tests import gpu_cases as gc

pytestmark = pytest.mark.gpu

CAP = 2          # CTAs per launch while these tests run
EXTRA_ITERS = 3  # iterations per warp beyond the S stages of its ring


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_6862_gb300 import build
    build.build()
    hd.lib()
    yield
    hd.hd_set_max_ctas(0)


@pytest.fixture(autouse=True)
def _cap():
    hd.hd_set_max_ctas(CAP)
    yield
    hd.hd_set_max_ctas(0)


def _wrap_size(infos):
    """Codewords that give every warp of every configuration S + EXTRA_ITERS
    chunks, plus a ragged tail that ends inside a tile and inside a word."""
    need = max((i["stages"] + EXTRA_ITERS) * (i["threads"] // 32) * CAP * i["chunk_codewords"] for i in infos)
    return need + 1237


def _iters(info, N):
    warps = CAP * (info["threads"] // 32)
    return (N // info["chunk_codewords"]) // warps


@pytest.mark.parametrize("n", [7, 15, 31, 63, 127, 255])
@pytest.mark.parametrize("syn", [hd.SYN_NONE, hd.SYN_U8, hd.SYN_U16])
def test_streaming_configurations_wrap_their_rings(n, syn):
    import torch
    cnt = hd.hd_variant_count(n, syn)
    infos = [hd.hd_variant_info_get(n, syn, i) for i in range(cnt)]
    N = _wrap_size(infos)
    stream, _, _ = gc.received_stream(n, N, seed=900 + n * 3 + syn, p1=0.2, p2=0.02)
    exp = gc.expected(stream, n, N, syn)
    d_in = gc.to_device(stream)
    try:
        for i, info in enumerate(infos):
            assert _iters(info, N) >= info["stages"] + 2, info
            hd.hd_variant_select(n, syn, i)
            got = hd.decode(d_in, n, N, syn_type=syn)
            torch.cuda.synchronize()
            try:
                gc.assert_same(got, exp, n, N, syn)
            except AssertionError as e:
                raise AssertionError(f"configuration {info}: {e}") from None
    finally:
        hd.hd_variant_select(n, syn, -1)
    assert hd.hd_device_status() == 0


def _secded_received(n, N, seed):
    m, k = hd.code_params(n)
    data = synth.random_words(seed, N * k)
    st = oracle.encode_secded(data, n, N)
    synth.apply_errors(st, synth.error_events(seed + 3, n + 1, N, p1=0.2, p2=0.05))
    return st


# u8 SECDED syndromes hold n <= 127 (s | P << m takes m + 1 bits)
_SECDED_CASES = [(n, syn) for n in (7, 15, 31, 63, 127, 255) for syn in (hd.SYN_NONE, hd.SYN_U8, hd.SYN_U16)
                 if not (syn == hd.SYN_U8 and n == 255)]


@pytest.mark.parametrize("n,syn", _SECDED_CASES)
def test_secded_configurations_wrap_their_rings(n, syn):
    import torch
    m, k = hd.code_params(n)
    cnt = hd.hd_secded_variant_count(n, syn)
    assert cnt >= 1
    infos = [hd.hd_secded_variant_info_get(n, syn, i) for i in range(cnt)]
    assert any(i["table_lookup"] for i in infos) == (n in (7, 15))
    N = _wrap_size(infos)
    rx = _secded_received(n, N, seed=700 + n + syn)
    eo, es, ee, ed = oracle.decode_secded(rx, n, N, syn if syn != hd.SYN_NONE else oracle.SYN_U16, threads=8)
    d_in = gc.to_device(rx, pad_words=4)
    nw = hd.words_for(N * k)
    try:
        for i, info in enumerate(infos):
            assert _iters(info, N) >= info["stages"] + 2, info
            hd.hd_secded_variant_select(n, syn, i)
            out = torch.full((nw + 4,), -1, dtype=torch.int32, device="cuda")
            sy = None
            if syn != hd.SYN_NONE:
                sy = torch.full((N + 16,), 0x55, dtype=torch.uint8 if syn == hd.SYN_U8 else torch.int16,
                                device="cuda")
            counts = torch.full((2,), 777, dtype=torch.int64, device="cuda")
            hd.decode_secded(d_in, n, N, syn, out=out, syndromes=sy, counts=counts)
            torch.cuda.synchronize()
            got = gc.host_u32(out)[:nw]
            assert np.array_equal(got, eo[:nw]), f"configuration {info}: data bits differ"
            if sy is not None:
                sg = sy.cpu().numpy()[:N]
                if syn == hd.SYN_U16:
                    sg = sg.view(np.uint16)
                assert np.array_equal(sg, es[:N].astype(sg.dtype)), f"configuration {info}: syndromes differ"
            c = counts.cpu().numpy()
            assert (int(c[0]), int(c[1])) == (ee, ed), f"configuration {info}: counts {c} vs {(ee, ed)}"
    finally:
        hd.hd_secded_variant_select(n, syn, -1)
    assert hd.hd_device_status() == 0


def test_batch_configurations_wrap_their_rings():
    """Every batch-kernel configuration on two CTAs: each warp claims and
    decodes dozens of tiles (full tiles of every n, ragged tails, n = 3)."""
    import torch
    from tests.test_batch_gpu import check_batch, make_batch
    pkts, exp = make_batch(90, seed=41, max_cw=60000)
    table = hd.packet_table([(hd._ptr(a), hd._ptr(b), hd._ptr(c), N, n, st) for a, b, c, N, n, st in pkts])
    tiles = hd.hd_batch_tiles(table, len(pkts))
    plan = hd.Plan(pkts)
    info = plan.info()
    err = torch.full((len(pkts),), 77, dtype=torch.int64, device="cuda")
    try:
        for v in range(info["num_variants"]):
            plan.select(v)
            vi = plan.info()
            # claims are dynamic: on average a warp decodes tiles / (CTAs * warps) tiles
            assert tiles // (CAP * vi["warps_per_cta"]) >= 4 * (vi["stages"] + 2), (tiles, vi)
            for d_in, out, syn, N, n, st in pkts:
                out.fill_(-1)
            plan.launch(err)
            torch.cuda.synchronize()
            try:
                check_batch(pkts, exp, err)
            except AssertionError as e:
                raise AssertionError(f"batch configuration {vi}: {e}") from None
    finally:
        plan.close()
    assert hd.hd_device_status() == 0


def test_stream_group_configuration_wraps_its_rings():
    """The batch plan's stream-group configuration (its last) on two CTAs per
    kernel: every (n, syndrome type) group holds over 300 whole chunks, so that
    each warp of the widest group kernel (18 warps) walks at least eight items
    of its range; packets of one group sit apart in the table and mix lengths
    of many chunks, one chunk, less than a chunk and none, so that runs, the
    run window and the rest's tiles are all exercised."""
    import torch
    from tests.test_batch_gpu import check_batch
    groups = [(n, st) for n in (7, 15, 31, 63, 127, 255) for st in (hd.SYN_NONE, hd.SYN_U8, hd.SYN_U16)]
    # packet lengths in chunks of the group's kernel (1024 codewords up to
    # n = 63, 256 above): 302 whole chunks per group in all
    shapes = (lambda c: 100 * c + 17, lambda c: c, lambda c: c - 1, lambda c: 5, lambda c: 60 * c,
              lambda c: 139 * c + c // 2, lambda c: 0, lambda c: 2 * c + 1)
    specs = [(n, st, shape(1024 if n <= 63 else 256)) for shape in shapes for n, st in groups]
    pkts, exp = [], []
    for j, (n, st, N) in enumerate(specs):
        stream, _, _ = gc.received_stream(n, N, seed=9100 + j, p1=0.1, p2=0.02)
        e = gc.expected(stream, n, N, st) if N else (np.zeros(0, np.uint32), None, 0)
        m, k = hd.code_params(n)
        out = torch.full((max(1, hd.words_for(N * k)),), -1, dtype=torch.int32, device="cuda")
        syn = None
        if st != hd.SYN_NONE:
            syn = torch.full((max(1, N),), 0x5A, dtype=torch.uint8 if st == 1 else torch.int16, device="cuda")
        pkts.append((gc.to_device(stream), out, syn, N, n, st))
        exp.append(e)
    plan = hd.Plan(pkts)
    err = torch.full((len(pkts),), 77, dtype=torch.int64, device="cuda")
    try:
        info = plan.info()
        plan.select(info["num_variants"] - 1)
        for rep in range(2):  # the recorded graph, then its replay
            for d_in, out, syn, N, n, st in pkts:
                out.fill_(-1)
            plan.launch(err)
            torch.cuda.synchronize()
            check_batch(pkts, exp, err)
    finally:
        plan.close()
    assert hd.hd_device_status() == 0


@pytest.mark.parametrize("n", [545, 2679, 8013, 32767])
def test_shortened_configurations_wrap_their_rings(n):
    """Every tiled shortened-code configuration on two CTAs (warps <= 16,
    stages <= 4, stages of at most 8 KB: 4 MB of input gives every warp more
    than 30 tiles); the lengths cover the three table placements (split
    tables for k < 1280, the table in shared memory, in global memory)."""
    import torch
    r, k = oracle.short_params(n)
    N = max(64, (32 << 20) // n)
    data = synth.random_words(n + 1, N * k)
    rx = oracle.encode_short(data, n, N)
    synth.apply_errors(rx, synth.error_events(n + 8, n, N, p1=0.3, p2=0.2))
    eo, es, ee, ed = oracle.decode_short(rx, n, N, oracle.SYN_U16, threads=8)
    d_in = gc.to_device(rx, pad_words=4)
    nw = hd.words_for(N * k)
    try:
        for v in range(hd.hd_short_variant_count()):
            hd.hd_short_variant_select(v)
            out = torch.full((nw + 4,), -1, dtype=torch.int32, device="cuda")
            sy = torch.full((N + 16,), 0x77, dtype=torch.int16, device="cuda")
            counts = torch.full((2,), 12345, dtype=torch.int64, device="cuda")
            hd.decode_short(d_in, n, N, hd.SYN_U16, out=out, syndromes=sy, counts=counts)
            torch.cuda.synchronize()
            got = gc.host_u32(out)[:nw]
            if not np.array_equal(got, eo[:nw]):
                bad = np.nonzero(got != eo[:nw])[0]
                raise AssertionError(f"configuration {v}: {bad.size} words differ, first {bad[0]}")
            assert np.array_equal(sy.cpu().numpy()[:N].view(np.uint16), es[:N]), f"configuration {v}: syndromes"
            c = counts.cpu().numpy()
            assert (int(c[0]), int(c[1])) == (ee, ed), f"configuration {v}: counts"
    finally:
        hd.hd_short_variant_select(-1)
    assert hd.hd_device_status() == 0


def test_cap_is_reported_and_cleared():
    assert hd.hd_get_max_ctas() == CAP
    hd.hd_set_max_ctas(0)
    assert hd.hd_get_max_ctas() == 0
