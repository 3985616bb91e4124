"""The allocation-free histogram entry point (raduls_histogram_static).

It exists for callers that cannot let a library allocate device memory (an
application whose memory is all reserved by its own allocator, a
latency-critical loop that cannot take cudaMalloc's synchronisation, code
inside a stream capture).  Its result must equal the allocating entry point's,
exactly (integer counts), on two calls in a row: the second call reuses the
library's fixed scratch array, whose contents the first call left behind.
This file is collected last, so a run that stops at its first failure has run
every other test before it.  The static entry point reports argument and
launch errors through its return code only (it records no device-side
status), so the comparison of the two results is the whole check.
"""
from __future__ import annotations

import numpy as np
import pytest

import datagen
from gpu_util import lib, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib()


def test_static_histogram_equals_allocating_one_on_two_calls():
    import torch
    p = lib()
    cases = [(3 * 16384 + 777, 16, 8, 7), (70001, 32, 16, 12), (5000, 8, 8, 0), (1, 24, 16, 15)]
    for call in range(2):
        for n, rec, key, digit in cases:
            recs = datagen.random_records(n, rec, key, n + call, alphabet=None if call else 5)
            d = to_dev(recs)
            want = torch.zeros(256, dtype=torch.int64, device="cuda")
            got = torch.full((256,), -1, dtype=torch.int64, device="cuda")
            p.raduls_histogram(d, n, rec, key, digit, want)
            p.raduls_histogram_static(d, n, rec, key, digit, got)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(got.cpu().numpy(), want.cpu().numpy(),
                                          err_msg=f"call {call}, n={n}, rec={rec}, key={key}, digit={digit}")


def test_static_histogram_rejects_sizes_beyond_its_scratch():
    import torch
    p = lib()
    d = to_dev(datagen.random_records(16, 16, 8, 1))
    h = torch.zeros(256, dtype=torch.int64, device="cuda")
    rc = p.load().raduls_histogram_static(d.data_ptr(), 1 << 33, 16, 8, 7, h.data_ptr(), None)
    assert rc == 3   # RADULS_ERR_UNSUPPORTED, nothing launched
