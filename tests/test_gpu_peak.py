"""The bench-only FMA-rate probe (libps_bench.so) that the FP64 step's ALU
roofline is held against."""
import os
import sys

import pytest
import torch

from paper_2002_08642_gb300 import build as pbuild

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

pytestmark = pytest.mark.gpu


def test_fma_peak_is_plausible():
    pbuild.build()
    s = torch.cuda.current_stream().cuda_stream
    f64 = bench.fma_peak(1, 2000, s)
    f32 = bench.fma_peak(0, 20000, s)
    print("FMA rate: FP64 %.3f TFLOP/s, FP32 %.1f TFLOP/s" % (f64 / 1e12, f32 / 1e12))
    # below the nominal 2 x 128 lanes x 152 SMs x 2.07 GHz = 80.5 TFLOP/s FP32
    assert 1e10 < f64 < f32 < 8.2e13
    with pytest.raises(RuntimeError):
        bench.fma_peak(7, 10, s)
