"""hd_decode_host: host buffers in and out, chunked transfers overlapped with
decoding; bit-exact against the oracle for pinned and pageable buffers."""
import numpy as np
import pytest

import oracle
from paper_1412_6862_gb300 import hd
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


@pytest.mark.parametrize("n", [7, 15, 63, 255])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_pipeline_matches_oracle(n, pinned):
    import torch
    N = 5 * 4096 + 333
    syn = hd.SYN_U16 if n == 255 else hd.SYN_U8
    stream, _, _ = gc.received_stream(n, N, seed=n + pinned, p1=0.2, p2=0.02)
    exp_out, exp_syn, exp_err = gc.expected(stream, n, N, syn)
    m, k = hd.code_params(n)
    if pinned:
        src = torch.from_numpy(stream.view(np.int32).copy()).pin_memory()
        out = torch.zeros(hd.words_for(N * k), dtype=torch.int32).pin_memory()
        sy = torch.zeros(N, dtype=torch.uint8 if syn == 1 else torch.int16).pin_memory()
    else:
        src, out = stream.copy(), np.zeros(hd.words_for(N * k), np.uint32)
        sy = np.zeros(N, np.uint8 if syn == 1 else np.uint16)
    for chunk, depth in ((4096, 3), (0, 0), (128, 8)):
        o, s, e = hd.decode_host(src, n, N, syn_type=syn, out=out, syndromes=sy, chunk_codewords=chunk, depth=depth)
        on = o.numpy().view(np.uint32) if hasattr(o, "numpy") else o
        sn = s.numpy() if hasattr(s, "numpy") else s
        if syn == hd.SYN_U16:
            sn = sn.view(np.uint16)
        assert np.array_equal(on[:exp_out.size], exp_out), (chunk, depth)
        assert np.array_equal(sn[:N], exp_syn), (chunk, depth)
        assert e == exp_err


def test_host_pipeline_zero_and_errors():
    z = np.zeros(4, np.uint32)
    assert hd.decode_host(z, 15, 0, syn_type=hd.SYN_NONE)[2] == 0
    rc, _ = hd.hd_decode_host(z.ctypes.data, 15 * 4, 15, 4, z.ctypes.data, None, 0, 100, 2)  # chunk not % 128
    assert rc == hd.HD_ERR_INVALID_ARG


@pytest.mark.parametrize("chunk,depth", [(0, 0), (128, 8), (4096, 3), (1 << 14, 2)])
def test_host_batch_matches_oracle(chunk, depth):
    """Several streams in one pipeline (ramped first and last chunks, chunks of
    different jobs interleaved on the rotating streams): every job bit-exact."""
    import torch
    jobs_spec = [(15, 3 * 4096 + 77, hd.SYN_U8), (63, 0, hd.SYN_U8), (31, 2 * 4096 + 1, hd.SYN_NONE),
                 (255, 5000, hd.SYN_U16), (7, 129, hd.SYN_U8)]
    jobs, keep, expect = [], [], []
    for j, (n, N, syn) in enumerate(jobs_spec):
        m, k = hd.code_params(n)
        stream, _, _ = gc.received_stream(n, N, seed=50 + j, p1=0.2, p2=0.02)
        expect.append(gc.expected(stream, n, N, syn if syn != hd.SYN_NONE else hd.SYN_U8))
        src = torch.from_numpy(np.concatenate([stream, np.zeros(4, np.uint32)]).view(np.int32)).pin_memory()
        out = torch.full((hd.words_for(N * k) + 4,), -1, dtype=torch.int32).pin_memory()
        sy = None if syn == hd.SYN_NONE else torch.full((N + 16,), 0x3C, dtype=torch.uint8 if syn == 1 else torch.int16).pin_memory()
        keep.append((src, out, sy))
        jobs.append((src.data_ptr(), n, N, out.data_ptr(), None if sy is None else sy.data_ptr(), syn))
    rc, errs = hd.hd_decode_host_batch(jobs, chunk, depth)
    assert rc == hd.HD_OK
    for j, ((n, N, syn), (src, out, sy), (eo, es, ee)) in enumerate(zip(jobs_spec, keep, expect)):
        m, k = hd.code_params(n)
        nw = hd.words_for(N * k)
        assert np.array_equal(out.numpy().view(np.uint32)[:nw], eo[:nw]), (j, chunk, depth)
        if sy is not None:
            sn = sy.numpy()[:N]
            if syn == hd.SYN_U16:
                sn = sn.view(np.uint16)
            assert np.array_equal(sn, es[:N]), (j, chunk)
        assert errs[j] == ee, (j, errs[j], ee)
