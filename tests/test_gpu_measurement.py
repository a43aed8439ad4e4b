"""The FMA-rate microbenchmark behind the roofline denominators: plausible rates on the GPU (the FP64
pipe is 1/64 of the FP32 one on this part) and host-side rejection of bad arguments."""
import pytest

torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_fma_rates_are_plausible():
    from paper_2404_16245_gb300 import shgo
    f64, ms64 = shgo.shgo_measure_fma_rate(shgo.SHGO_PREC_FP64, 256)
    f32, ms32 = shgo.shgo_measure_fma_rate(shgo.SHGO_PREC_FP32_BULK, 16384)
    assert ms64 > 0 and ms32 > 0
    # nominal at 2.07 GHz: 1.26 TFLOP/s FP64, 80.6 TFLOP/s FP32; clocks may sit lower under a power cap
    assert 0.3e12 < f64 < 1.5e12, f64
    assert 20e12 < f32 < 95e12, f32
    assert 20 < f32 / f64 < 200


def test_fma_rate_rejects_bad_arguments_before_gpu_work():
    shgo = pytest.importorskip("paper_2404_16245_gb300.shgo", reason="libshgo.so not built")
    with pytest.raises(shgo.ShgoError) as e:
        shgo.shgo_measure_fma_rate(shgo.SHGO_PREC_FP64, 0, stream=0)
    assert e.value.status == 1
    with pytest.raises(shgo.ShgoError) as e:
        shgo.shgo_measure_fma_rate(7, 10, stream=0)
    assert e.value.status == 1
