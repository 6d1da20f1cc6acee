"""The tensor-rate microbenchmarks that serve as the heavy product's roofline
denominators run to completion and give rates of the right magnitude for a
GB300 (dense FP8 nominally 4.5 PFLOP/s; legacy INT8 mma.sync far lower)."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_tensor_peaks_are_plausible():
    import torch
    from paper_2002_12459_gb300 import build, jp
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for the -m gpu tests")
    ctx = jp.Context(0)
    try:
        p = ctx.measure_peaks()
    finally:
        ctx.close()
    assert 1000.0 < p["fp8_tcgen05_tflops"] < 6000.0, p
    assert 10.0 < p["int8_mma_sync_tflops"] < p["fp8_tcgen05_tflops"], p
