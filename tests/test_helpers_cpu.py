"""The test helpers that build large inputs on the host: the threaded oracle
encoder gives exactly the single-call oracle encoder's stream."""
import numpy as np
import pytest

import oracle
from paper_1412_6862_gb300 import synth
from tests import gpu_cases as gc


@pytest.mark.parametrize("kind,n", [("plain", 31), ("plain", 255), ("secded", 15), ("secded", 127),
                                    ("short", 545), ("short", 2679)])
@pytest.mark.parametrize("N", [1, 33, 64 * 97 + 5])
def test_parallel_oracle_encoder_equals_single_call(oracle_mod, kind, n, N):
    if kind == "plain":
        m, k = oracle.params(n)
        enc, L = oracle.encode, n
    elif kind == "secded":
        m, k = oracle.params(n)
        enc, L = oracle.encode_secded, n + 1
    else:
        r, k = oracle.short_params(n)
        enc, L = oracle.encode_short, n
    data = synth.random_words(n + N, N * k)
    want = enc(data, n, N)
    got = gc.oracle_encode_parallel(enc, data, n, N, k, L, threads=5)
    assert np.array_equal(got, want)
