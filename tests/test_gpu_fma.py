"""The FMA-rate microbenchmark (amr_fma_rate), the measured denominator of
the arithmetic-bound rooflines: FP64 within reach of GB300's FP64 pipe
(152 SMs x 2 FMA per clock: 1.26 TFLOP/s at the 2070 MHz maximum clock),
FP32 far above it (the FP64 rate is 1/64 of FP32 on this part)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2607_20704_gb300 import amr, build
    build.build()
    amr.load()


def test_rates_are_plausible():
    from paper_2607_20704_gb300 import amr
    f64 = amr.fma_rate(0, 8)
    f32 = amr.fma_rate(0, 4)
    assert 0.2e12 < f64 < 1.6e12, f64
    assert f32 > 16 * f64, (f32, f64)


def test_bad_precision_is_refused():
    from paper_2607_20704_gb300 import amr
    with pytest.raises(amr.AmrError) as e:
        amr.fma_rate(0, 2)
    assert e.value.status == amr.AMR_EINVAL
