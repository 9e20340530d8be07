"""The throughput probes behind the roofline: FP64 FMA chains and FP64
tensor-core (DMMA) chains both report a positive, finite rate, and the FMA
rate stays below the derived peak of 2 DFMA per clock per SM at the maximum
SM clock (a probe far above it would not be doing its work)."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_fp64_probes_report_plausible_rates():
    import torch

    from paper_2603_03639_gb300.tnrc import measure_dmma_peak, measure_fp64_peak
    props = torch.cuda.get_device_properties(0)
    buf = torch.empty(4 * 256 * props.multi_processor_count, dtype=torch.float64, device="cuda")
    fma = measure_fp64_peak(buf.data_ptr(), buf.numel() * 8)
    dmma = measure_dmma_peak(buf.data_ptr(), buf.numel() * 8)
    assert math.isfinite(fma) and math.isfinite(dmma)
    assert fma > 100.0 and dmma > 100.0                     # GFLOP/s
    derived = 4.0 * props.multi_processor_count * 2.2       # 2 DFMA x 2 flops per clock, clocks <= 2.2 GHz
    assert fma < 1.05 * derived
    print("FP64 FMA %.1f GFLOP/s, DMMA %.1f GFLOP/s" % (fma, dmma))
