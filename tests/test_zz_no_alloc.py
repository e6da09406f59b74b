"""ffgpu_fgemm_noalloc, the entry point for callers that cannot allocate
device memory: a framework that owns every byte of it and hands out only
pre-sized buffers, a latency-critical path that cannot take an allocation's
synchronisation or failure, or a process that has already reserved the whole
device.  It must give exactly what ffgpu_fgemm gives, and what the oracle
gives, on both of its routes: the CUDA-core kernel for small products (only
its k-split partial sums live in the static scratch) and the tensor-core route
(channel planes, residue slots and error word all in the static scratch, at
most 32 persistent CTAs).

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process (the first
call looks up the static scratch on the device)."""
import numpy as np
import pytest
import torch

import oracle
import paper_cs_0601133_gb300 as ff
from paper_cs_0601133_gb300 import workloads as W
from tests.gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu

SCRATCH = 64 * 1024 * 1024      # FFGPU_NOALLOC_SCRATCH_BYTES


def _call(fn, A, B, C, p, alpha, beta, stream=None):
    m, k = A.shape
    n = B.shape[1]
    s = (stream or torch.cuda.current_stream()).cuda_stream
    return fn(m, n, k, p, alpha, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), beta,
              C.data_ptr(), C.stride(0), s)


@pytest.fixture
def threshold():
    """Restores the CUDA-core threshold after a test that changes it."""
    old = ff.get_small_threshold()
    yield
    ff.set_small_threshold(old)


def _problem(rng, m, k, n, p):
    A = W.uniform_words(rng, (m, k))
    B = W.uniform_words(rng, (k, n))
    C = W.uniform_words(rng, (m, n))
    alpha, beta = int(rng.integers(0, p)), int(rng.integers(0, p))
    return A, B, C, alpha, beta


def _both(A, B, C, p, alpha, beta):
    """C from ffgpu_fgemm and from ffgpu_fgemm_noalloc, same inputs."""
    dA, dB = to_dev(A), to_dev(B)
    ref_C, got_C = to_dev(C), to_dev(C)
    assert _call(ff.fgemm_ptr, dA, dB, ref_C, p, alpha, beta) == 0
    assert _call(ff.fgemm_noalloc_ptr, dA, dB, got_C, p, alpha, beta) == 0
    torch.cuda.synchronize()
    return from_dev(got_C), from_dev(ref_C)


# (m, k, n) pairs run back to back: CUDA-core products (at most 2^27
# multiply-adds), then tensor-core products with the default threshold
# (1024^3 and a ragged 1100 x 700 x 900 are above 2^27).
CORE_SHAPES = [(300, 700, 260), (513, 1000, 129)]
TENSOR_SHAPES = [(1024, 1024, 1024), (1100, 700, 900)]


@pytest.mark.parametrize("p", [251, 65521, 2147483647])
@pytest.mark.parametrize("shapes", [CORE_SHAPES, TENSOR_SHAPES], ids=["cuda_cores", "tensor_cores"])
def test_noalloc_matches_fgemm_and_oracle_on_two_calls_in_a_row(p, shapes):
    rng = W.rng_for("smoke", 99, p, shapes[0][0])
    for m, k, n in shapes:
        A, B, C, alpha, beta = _problem(rng, m, k, n, p)
        got, ref = _both(A, B, C, p, alpha, beta)
        # exact arithmetic: the tolerance of every parity test here is zero
        assert np.array_equal(got, ref)
        assert np.array_equal(got, oracle.fgemm(A, B, p, alpha, beta, C))


@pytest.mark.parametrize("p", [65521, 2147483647])
def test_noalloc_tensor_cores_for_small_products(p, threshold):
    """With the CUDA-core threshold at 0 every product takes the tensor-core
    route, the small ones included: one tile, several tiles, a ragged edge."""
    ff.set_small_threshold(0)
    rng = W.rng_for("smoke", 98, p)
    for m, k, n in [(300, 700, 260), (129, 65, 257), (513, 1000, 129)]:
        A, B, C, alpha, beta = _problem(rng, m, k, n, p)
        got, ref = _both(A, B, C, p, alpha, beta)
        assert np.array_equal(got, ref)
        assert np.array_equal(got, oracle.fgemm(A, B, p, alpha, beta, C))


def _tensor_scratch_bytes(m, n, k, channels):
    """Scratch of the tensor-core route: 32 CTAs x 2 residue slots of
    channels x 128 x 256 bytes, then the bf16 planes of A and B (k padded to
    64), each part 256-byte aligned, after the 256-byte error word."""
    a256 = lambda x: (x + 255) // 256 * 256
    kp = (k + 63) // 64 * 64
    return 256 + a256(32 * 2 * channels * 128 * 256) + a256(channels * m * kp * 2) + a256(channels * n * kp * 2)


def test_noalloc_just_under_the_limit_then_a_smaller_problem():
    """The largest k that fits at m = n = 1024, p = 2^31 - 1 (k = 1088: 97 %
    of the array), then a smaller problem in the same array: stale planes or
    digits of the first call must not reach the second's result.  One more
    64-column block of k no longer fits and is refused."""
    p = 2147483647
    m = n = 1024
    k = 1088
    ch = ff.fgemm_plan(m, n, k, p)["channels"]
    assert _tensor_scratch_bytes(m, n, k, ch) <= SCRATCH < _tensor_scratch_bytes(m, n, k + 1, ch)
    assert _tensor_scratch_bytes(m, n, k, ch) >= 0.95 * SCRATCH
    rng = W.rng_for("smoke", 97)
    for mm, kk, nn in [(m, k, n), (700, 600, 520)]:
        A, B, C, alpha, beta = _problem(rng, mm, kk, nn, p)
        got, ref = _both(A, B, C, p, alpha, beta)
        assert np.array_equal(got, ref)
        assert np.array_equal(got, oracle.fgemm(A, B, p, alpha, beta, C))
    dA = torch.zeros((m, k + 1), dtype=torch.int32, device="cuda")
    dB = torch.zeros((k + 1, n), dtype=torch.int32, device="cuda")
    dC = torch.zeros((m, n), dtype=torch.int32, device="cuda")
    assert _call(ff.fgemm_noalloc_ptr, dA, dB, dC, p, 1, 0) == -3   # FFGPU_ERR_NOMEM


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    # 4096^3 at p < 2^31 needs ~330 MB of planes: more than the static array
    dA = torch.zeros((4096, 4096), dtype=torch.int32, device="cuda")
    dC = torch.zeros((4096, 4096), dtype=torch.int32, device="cuda")
    rc = _call(ff.fgemm_noalloc_ptr, dA, dA, dC, 2147483647, 1, 0)
    assert rc == -3  # FFGPU_ERR_NOMEM, nothing enqueued


def test_noalloc_skinny_small_product_fits():
    """A valid CUDA-core product with a long inner dimension (64 x 32768 x 64)
    needs only its partial sums, not the planes a tensor-core launch would."""
    p = 2147483647
    rng = W.rng_for("smoke", 96)
    A, B, C, alpha, beta = _problem(rng, 64, 32768, 64, p)
    got, ref = _both(A, B, C, p, alpha, beta)
    assert np.array_equal(got, ref)
    assert np.array_equal(got, oracle.fgemm(A, B, p, alpha, beta, C))


def test_noalloc_allocates_nothing():
    """After a first call of each shape (which loads the kernels it uses), calls
    on a fresh stream change neither the device's free memory nor torch's
    caching allocator: a regular entry point on a new stream would grow a new
    workspace pool there."""
    p = 2147483647
    rng = W.rng_for("smoke", 95)
    probs = [_problem(rng, m, k, n, p) for m, k, n in [(1024, 1024, 1024), (300, 700, 260)]]
    dev = []
    for A, B, C, alpha, beta in probs:
        dA, dB, dC = to_dev(A), to_dev(B), to_dev(C)
        assert _call(ff.fgemm_noalloc_ptr, dA, dB, dC, p, alpha, beta) == 0
        dev.append((dA, dB, dC, alpha, beta))
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(2):
        for dA, dB, dC, alpha, beta in dev:
            assert _call(ff.fgemm_noalloc_ptr, dA, dB, dC, p, alpha, beta, stream=s) == 0
    s.synchronize()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
