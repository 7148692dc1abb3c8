"""The FP64 FMA issue-rate probe behind the roofline denominator of the FP64 kernels (dgasm_probe_fp64; no
paper counterpart).  The nominal FP64 rate of this part is 1/64 of its FP32 rate, 2 FMA per clock per SM; the
probe must report a rate at most that (a higher one would mean the probe does not measure FP64 FMAs) and not
far below it, and a GPU-wide rate consistent with the per-SM rate at a clock between 1 and 2.1 GHz."""
import pytest

from tests.helpers import have_gpu

pytestmark = pytest.mark.gpu

if have_gpu():
    import torch
    from paper_1903_11357_gb300 import dgasm as dg


def test_probe_fp64_rate_is_plausible():
    nsm, rate, tflops = dg.probe_fp64()
    assert nsm == torch.cuda.get_device_properties(0).multi_processor_count
    assert 1.0 <= rate <= 2.0 + 1e-6, rate
    clock_ghz = tflops * 1e12 / (2.0 * rate * nsm) / 1e9
    assert 1.0 <= clock_ghz <= 2.1, clock_ghz
