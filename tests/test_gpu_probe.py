"""ALU throughput probes (measurement support for the roofline's ALU term)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")


def test_probe_rates_are_physical():
    import torch

    from paper_2512_09664_b300 import measure as B
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # an upper bound no probe can pass: every FP32 lane busy every cycle at 2.2 GHz
    ceiling = sms * 128 * 2.2e9
    fma = B.alu_probe("fma", iters=2048, reps=2)
    assert 0.3 * ceiling < fma <= ceiling
    erfc = B.alu_probe("erfc", iters=256, reps=2)
    ex2 = B.alu_probe("ex2", iters=1024, reps=2)
    umulhi = B.alu_probe("umulhi", iters=1024, reps=2)
    # erfcf is a sequence of FP32 operations; the exponential runs on the
    # special-function units (a quarter of the FP32 lanes or fewer)
    assert 0.0 < erfc < fma / 4
    assert 0.0 < ex2 <= fma / 2
    assert 0.0 < umulhi <= fma
    n = B.lib().synthpix_alu_probe_threads()
    assert n == sms * 2048
