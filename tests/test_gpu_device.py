"""Device facts of the built library on the GPU: the engine kernel is sm_103a code (the
CUDA runtime's kernel attributes, not the binary), and the FP32 probe measures a
throughput in the range the SM count and clock allow."""
import pytest

from paper_2307_11447_gb300 import lib as h4d

pytestmark = pytest.mark.gpu


def test_engine_kernel_is_sm103_code():
    sms, binary, ptx = h4d.h4d_device_info()
    assert binary == 103, binary
    assert ptx >= 100 and sms > 0


def test_fp32_probe_is_within_the_nominal_peak():
    sms, _, _ = h4d.h4d_device_info()
    tflops, secs = h4d.h4d_measure_fp32_peak()
    nominal = sms * 128 * 2 * 2.07e9 / 1e12  # 128 FP32 lanes per SM at the 2070 MHz maximum clock
    print(f"\nFP32 FMA-chain probe {tflops:.1f} TFLOP/s in {secs * 1e3:.1f} ms; nominal {nominal:.1f}")
    assert 0.5 * nominal < tflops <= 1.02 * nominal
