"""The FP64 fused-multiply-add probe behind the bench's measured FP64 roofline (GPU).

Each thread runs 8 chains x <- x m + c for `steps` steps from
x0 = 1e-3 ((tid + k) mod 64); the stored value is the sum of the chains.  The
chain has the closed form x_n = q + (x0 - q) m^n with q = c / (1 - m), so the
output shows that every step ran (a probe that skipped work would report a
rate it never reached), and the flop count is 2 x 8 x steps per thread.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cola():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_00850_gb300 as cola
    from paper_2302_00850_gb300 import build

    build.build()
    return cola


def test_probe_computes_its_chains(cola):
    import torch

    blocks, threads, steps = 3, 64, 400
    out = torch.zeros(blocks * threads, dtype=torch.float64, device="cuda")
    flop = cola.api.probe_fp64_fma(out, blocks, threads, steps)
    torch.cuda.synchronize()
    assert flop == 2 * 8 * steps * threads * blocks
    m, c = 0.999999, 1e-7
    q = c / (1.0 - m)
    tid = np.arange(blocks * threads)
    want = np.zeros(blocks * threads)
    for k in range(8):
        x0 = 1e-3 * ((tid + k) % 64)
        want += q + (x0 - q) * m ** steps
    got = out.cpu().numpy()
    assert np.max(np.abs(got - want)) < 1e-12


def test_probe_rate_is_plausible(cola):
    """The measured rate lies between a tenth of and just above the derived
    FP64 peak of the part (unit counts x clock), as a timed probe must."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks, threads, steps = 8 * sms, 256, 4096
    out = torch.empty(blocks * threads, dtype=torch.float64, device="cuda")
    cola.api.probe_fp64_fma(out, blocks, threads, steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    flop = cola.api.probe_fp64_fma(out, blocks, threads, steps)
    e1.record()
    torch.cuda.synchronize()
    tflops = flop / (e0.elapsed_time(e1) * 1e-3) / 1e12
    derived = sms * 2 * 2 * 2.07e9 / 1e12  # 2 DFMA per SM per cycle, 2 flop, maximum clock
    assert 0.1 * derived < tflops < 1.05 * derived, (tflops, derived)
