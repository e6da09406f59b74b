"""Failure detection on the GPU without a fault: a bounded wait runs out on a
barrier nothing completes, the kernel reports it through the device error
word, and the context keeps working (section 5 of the design: every wait in
the library's kernels is bounded)."""
import numpy as np
import pytest
import torch

import oracle
import paper_cs_0601133_gb300 as ff
from paper_cs_0601133_gb300 import workloads as W
from tests.gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu


def test_wait_timeout_is_reported_and_context_survives():
    assert ff.last_device_error() == 0
    ff.selftest_wait_timeout(2_000_000)           # ~1 ms of SM clock
    assert ff.last_device_error() == -5           # FFGPU_ERR_TIMEOUT
    assert ff.last_device_error() == 0            # the record is cleared once read
    # the device still computes correctly afterwards
    p = 65521
    rng = W.rng_for("smoke", 31)
    A = W.uniform_residues(rng, (200, 300), p)
    B = W.uniform_residues(rng, (300, 150), p)
    dC = to_dev(np.zeros((200, 150), np.uint32))
    ff.fgemm(to_dev(A), to_dev(B), p, 1, 0, dC)
    torch.cuda.synchronize()
    assert ff.last_device_error() == 0
    assert np.array_equal(from_dev(dC), oracle.fgemm(A, B, p))


def test_selftest_rejects_bad_limits():
    with pytest.raises(ff.FFGPUError):
        ff.selftest_wait_timeout(0)


def test_injected_allocation_failure_and_recovery(monkeypatch):
    """A workspace allocation that fails (injected on the host) surfaces as
    FFGPU_ERR_NOMEM with nothing launched, and the same call on the same
    stream succeeds once allocation works again."""
    p = 65521
    rng = W.rng_for("smoke", 32)
    A = W.uniform_residues(rng, (512, 700), p)   # 2.2e8 multiply-adds: the tensor-core
    B = W.uniform_residues(rng, (700, 600), p)   # route, which needs a workspace
    dA, dB = to_dev(A), to_dev(B)
    dC = to_dev(np.full((512, 600), 7, np.uint32))
    s = torch.cuda.Stream()                       # its workspace pool is still empty
    monkeypatch.setenv("FFGPU_INJECT_ALLOC_FAIL", "1")
    with pytest.raises(ff.FFGPUError) as e:
        ff.fgemm(dA, dB, p, 1, 0, dC, stream=s)
    assert e.value.status == -3                   # FFGPU_ERR_NOMEM
    s.synchronize()
    assert (from_dev(dC) == 7).all()              # C untouched
    monkeypatch.delenv("FFGPU_INJECT_ALLOC_FAIL")
    ff.fgemm(dA, dB, p, 1, 0, dC, stream=s)
    s.synchronize()
    assert ff.last_device_error() == 0
    assert np.array_equal(from_dev(dC), oracle.fgemm(A, B, p))
