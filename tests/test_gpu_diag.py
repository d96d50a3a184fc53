"""Roofline denominators measured by the library (include/mg_diag.h)."""
import pytest

torch = pytest.importorskip("torch")

from paper_2303_18244_gb300 import mg  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_peaks_are_measured_and_ordered():
    """FP64 FMA < FP32 FMA < FP16 tensor-core MMA, each within a factor of
    the GB300 figures (FP32 about 2 x 128 lanes x 152 SMs x clock; dense FP16
    tensor about 2.25 PFLOP/s nominal)."""
    fp32 = mg.diag_fma_peak(0) / 1e3
    fp64 = mg.diag_fma_peak(1) / 1e3
    mma = mg.diag_mma_peak()
    assert 0.1 < fp64 < fp32 < mma
    assert 20 < fp32 < 200
    assert 300 < mma < 3000
