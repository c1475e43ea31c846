"""The device-limit probes behind the rooflines' denominators: measured FP64 / FP32 FMA throughput and
copy bandwidths in plausible ranges for a GB300 (FP64 about 1.2 TFLOP/s, FP32 tens of TFLOP/s, an
L2-resident copy faster than one through HBM)."""

import pytest

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def test_fma_and_copy_probes():
    require_gpu()
    from paper_0910_0262_gb300 import qcd as Q
    fp64 = Q.qcd_probe_fma_peak(64)
    fp32 = Q.qcd_probe_fma_peak(32)
    assert 0.2 < fp64 < 100.0, fp64
    assert fp32 > 5 * fp64, (fp32, fp64)
    l2 = Q.qcd_probe_copy_bandwidth(24 << 20, 5)
    hbm = Q.qcd_probe_copy_bandwidth(1 << 30, 3)
    assert 1000.0 < hbm < 20000.0, hbm
    assert l2 > hbm, (l2, hbm)


def test_probe_argument_errors():
    require_gpu()
    from paper_0910_0262_gb300 import qcd as Q
    with pytest.raises(Q.QCDError):
        Q.qcd_probe_fma_peak(16)
    with pytest.raises(Q.QCDError):
        Q.qcd_probe_copy_bandwidth(15, 1)
