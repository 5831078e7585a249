"""The measured-peak entry points used by the roofline (ceedbp_fma_peak, ceedbp_mma_peak):
finite positive rates, the device's SM count, and argument errors reported as statuses."""
import ctypes

import pytest
import torch

import paper_2004_06722_gb300 as pkg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    pkg.load_library()


def test_fma_peaks():
    f64, sms = pkg.fma_peak(True)
    f32, sms32 = pkg.fma_peak(False)
    assert sms == sms32 == torch.cuda.get_device_properties(0).multi_processor_count
    assert 0.0 < f64 < f32 < 1e4
    print(f"FMA peaks: FP64 {f64:.3f} TFLOP/s, FP32 {f32:.1f} TFLOP/s on {sms} SMs")


def test_mma_peaks():
    rates = [pkg.mma_peak(k) for k in range(3)]
    assert all(0.0 < r < 1e5 for r in rates)
    print("mma.sync peaks (TFLOP/s): FP64 m8n8k4 %.3f, TF32 m16n8k8 %.1f, BF16 m16n8k16 %.1f" % tuple(rates))


def test_peak_argument_errors():
    lib = pkg.load_library()
    assert lib.ceedbp_mma_peak(3, ctypes.byref(ctypes.c_double())) == pkg.EINVAL
    assert lib.ceedbp_mma_peak(0, None) == pkg.EINVAL
    assert lib.ceedbp_fma_peak(1, None, None) == pkg.EINVAL
