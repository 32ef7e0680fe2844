"""The integer-pipe throughput probe used for the roofline context."""
import ctypes

import pytest

from paper_2303_14335_gb300 import mpld

pytestmark = pytest.mark.gpu


def test_int_pipe_probe_reports_positive_rates():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fn = mpld.probe_library().mpld_probe_int_peak
    out = (ctypes.c_double * 2)()
    assert fn(1 << 12, out) == 0
    # more than one op per SM per clock, less than 1,024 per SM per clock
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for v in out:
        assert sms * 1.0 * 0.5 < v < sms * 1024 * 2.2
    assert fn(4, out) == mpld.MPLD_E_INVALID
