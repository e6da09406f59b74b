"""The warp-level MMA peak probe (the int8 reference point beside the bf16
tensor-core roofline): every kind runs and reports a positive rate, and the
rates are ordered as the units are (int8 and bf16 far above FP64)."""
import pytest

import paper_cs_0601133_gb300 as ff

pytestmark = pytest.mark.gpu


def test_probe_rates():
    r = {k: ff.peak_probe(k, iters) for k, iters in (("int8", 20000), ("bf16", 20000), ("fp64", 2000))}
    assert all(v > 0 for v in r.values())
    assert r["int8"] > 5 * r["fp64"] and r["bf16"] > 5 * r["fp64"]


def test_probe_rejects_bad_arguments():
    import ctypes
    out = ctypes.c_double(0.0)
    for kind, iters in ((3, 10), (0, 0), (0, 2 ** 25)):
        assert ff.lib().ffgpu_peak_probe(kind, iters, ctypes.byref(out), None) == -1
