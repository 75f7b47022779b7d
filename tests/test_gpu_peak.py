"""wf_alu_peak: the measured FMA throughput used as the ALU roofline of the
FP64 path must be positive, finite, and ordered as the hardware is (FP32 FMA
well above FP64 FMA)."""
import math

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1810_00503_gb300 import wf  # noqa: E402
from tests.helpers import ensure_lib  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    ensure_lib()


def test_alu_peaks_are_plausible():
    f32 = wf.alu_peak("f32")
    f64 = wf.alu_peak("f64")
    assert math.isfinite(f32) and math.isfinite(f64)
    assert f32 > 1e12 and f64 > 1e10
    assert f32 > 4 * f64


def test_alu_peak_rejects_bad_dtype():
    import ctypes
    v = ctypes.c_double()
    assert wf.lib().wf_alu_peak(7, ctypes.byref(v)) == 1  # WF_EINVAL
