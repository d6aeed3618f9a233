"""The FP64 issue-rate probes that bench.py reports beside the derived peak:
every form gives a positive rate, the register-operand DFMA chain (the pipe's
peak, mhd_probe_fp64) is the fastest form, and it lies within a few percent
of 148 SMs x 2 DFMA per clock x 2 flops at the device's clock range."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mhd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_20337_b300 import mhd as M
    M.lib()
    return M


def test_fp64_forms(mhd):
    import torch
    rates = mhd.probe_fp64_forms()
    assert set(rates) == set(mhd.FP64_FORMS)
    for k, v in rates.items():
        assert v > 0.0, k
    for k, v in rates.items():
        assert rates["dfma"] >= 0.99 * v, (k, rates)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    upper = sms * 2 * 2 * 2.2  # GFLOP/s at a 2.2 GHz clock, above any B300 boost clock
    assert rates["dfma"] <= upper
    single = mhd.probe_fp64_gflops()
    assert abs(single - rates["dfma"]) <= 0.05 * rates["dfma"]
