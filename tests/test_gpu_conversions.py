"""The FP32 form converts between float and double with integer instructions
(the hardware conversion runs on the narrow FP64 pipe of this GPU).  These
conversions must agree bit for bit with the hardware's round-to-nearest-even
conversion on every input in the normal FP32 range, and flush inputs below it
to signed zero."""
import pytest

from paper_2604_02125_gb300 import crkfr


@pytest.mark.gpu
@pytest.mark.parametrize("seed", [2604021255, 7])
def test_integer_conversions_match_hardware(seed):
    assert crkfr.check_conversions(n=1 << 24, seed=seed) == 0


@pytest.mark.gpu
def test_conversion_check_rejects_bad_arguments():
    with pytest.raises(crkfr.CrError):
        crkfr.check_conversions(n=-1)
