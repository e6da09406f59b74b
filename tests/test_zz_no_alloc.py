"""ffgpu_fgemm_noalloc, the entry point for callers that cannot allocate
device memory (their framework owns it, or an allocation's synchronisation or
failure is not acceptable on their path).  It must give exactly what
ffgpu_fgemm gives.  This file sorts last so that a run stopping at the first
failure has already run every other test; it also passes on its own in a fresh
process (the first call looks up the static scratch on the device)."""
import numpy as np
import pytest
import torch

import paper_cs_0601133_gb300 as ff
from paper_cs_0601133_gb300 import workloads as W
from tests.gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu


def _call(fn, A, B, C, p, alpha, beta):
    m, k = A.shape
    n = B.shape[1]
    stream = torch.cuda.current_stream().cuda_stream
    return fn(m, n, k, p, alpha, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), beta,
              C.data_ptr(), C.stride(0), stream)


@pytest.mark.parametrize("p", [251, 65521, 2147483647])
def test_noalloc_matches_fgemm_on_two_calls_in_a_row(p):
    rng = W.rng_for("smoke", 99, p)
    shapes = [(300, 700, 260), (513, 1000, 129)]     # (m, k, n): two different problems in a row
    for m, k, n in shapes:
        A = W.uniform_words(rng, (m, k))
        B = W.uniform_words(rng, (k, n))
        C = W.uniform_words(rng, (m, n))
        alpha, beta = int(rng.integers(0, p)), int(rng.integers(0, p))
        dA, dB = to_dev(A), to_dev(B)
        ref_C, got_C = to_dev(C), to_dev(C)
        assert _call(ff.fgemm_ptr, dA, dB, ref_C, p, alpha, beta) == 0
        assert _call(ff.fgemm_noalloc_ptr, dA, dB, got_C, p, alpha, beta) == 0
        torch.cuda.synchronize()
        # exact arithmetic: the tolerance of every parity test here is zero
        assert np.array_equal(from_dev(got_C), from_dev(ref_C))


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    # 4096^3 at p < 2^31 needs ~330 MB of planes: more than the static array
    dA = torch.zeros((4096, 4096), dtype=torch.int32, device="cuda")
    dC = torch.zeros((4096, 4096), dtype=torch.int32, device="cuda")
    rc = _call(ff.fgemm_noalloc_ptr, dA, dA, dC, 2147483647, 1, 0)
    assert rc == -3  # FFGPU_ERR_NOMEM, nothing enqueued
