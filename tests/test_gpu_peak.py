"""wpm_int_peak, the measured integer throughput behind the search kernels' roofline: its
figures lie between a single SM's issue rate and the nominal all-SM INT32 rate with some
headroom (2 instructions a step, 8 chains, every SM), a longer run measures the same rate,
and bad arguments are refused."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2301_00806_gb300 import wpm
    wpm.lib()
    return wpm


def test_int_peak_is_plausible_and_stable(W):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    clock_hz = 2.5e9  # above any GB300 SM clock
    nominal = sms * 128 * clock_hz
    for op in (0, 1):
        a, ms_a = W.int_peak(op, 1 << 14)
        b, ms_b = W.int_peak(op, 1 << 16)
        assert 1e11 < a < 1.2 * nominal and 1e11 < b < 1.2 * nominal
        assert ms_b > 2 * ms_a            # four times the work takes longer
        assert abs(a - b) / b < 0.25      # and runs at about the same rate


def test_int_peak_rejects_bad_arguments(W):
    for op, iters in ((2, 1024), (0, 0), (-1, 1024)):
        with pytest.raises(W.WpmError) as e:
            W.int_peak(op, iters)
        assert e.value.code == W.ERR_INPUT
