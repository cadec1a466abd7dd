"""The measured arithmetic peaks (tddft_testing_peak) that serve as roofline
denominators: FP32 FMA throughput of the CUDA cores and TF32 throughput of the
tcgen05 tensor cores. Checked for plausibility against the device's nominal
figures (148 SMs x 128 FP32 lanes x 2 flops x ~2 GHz = 77 TFLOP/s; TF32 dense
about 1.1 PFLOP/s): a measurement far outside means the kernel did not do the
work it counts."""
import pytest

from paper_2309_03513_b300 import tddft as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    return _t


def test_fp32_fma_peak(torch):
    r = T.measure_peak(0)
    assert 20.0 < r["tflops"] < 120.0, r


def test_tf32_tensor_peak(torch):
    r = T.measure_peak(1)
    assert 200.0 < r["tflops"] < 2500.0, r


def test_peak_rejects_unknown_kind(torch):
    with pytest.raises(T.TddftError):
        T.measure_peak(2)
