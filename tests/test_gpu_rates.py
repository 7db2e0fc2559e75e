"""gl_unit_rates: the pipe throughputs behind the roofline, measured on the
device in operations per SM per SM clock. The FP32 rates cannot exceed the
128 lanes an SM has, paired instructions give the same lane throughput as
scalar ones (two pipe cycles each), and the MUFU rate is a small fraction of
the FP32 rate. A NULL output is refused before any device work."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_30633_b300 import build
    build.build()
    import paper_2606_30633_b300 as g
    return g


def test_rates_are_physical(gl):
    r = gl.unit_rates()
    assert 96.0 <= r["fp32"] <= 128.0, r
    assert 96.0 <= r["fp32x2"] <= 128.0, r
    assert abs(r["fp32"] - r["fp32x2"]) <= 0.1 * r["fp32"], r
    assert 4.0 <= r["mufu"] <= 0.5 * r["fp32"], r


def test_null_output_is_rejected(gl):
    lib = gl.load()
    v = ctypes.c_double()
    assert lib.gl_unit_rates(None, ctypes.addressof(v), ctypes.addressof(v)) == gl.GL_EINVAL
