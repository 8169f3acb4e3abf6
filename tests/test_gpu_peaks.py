"""The peak-throughput probes (ut_peak_probe) behind the compositing kernels' roofline
fractions: each probe computes what it states (its chains against a host replay) and its
measured rate lies between a third of the nominal figure and just above it, so the
denominators the benchmark divides by are neither inflated nor empty."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2412_12507_gb300 import abi  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2412_12507_gb300 import build
    build.build()
    return abi.lib()


def _run(L, kind, blocks, threads, iters):
    out = torch.zeros(blocks * threads, dtype=torch.float32, device="cuda")
    st = L.ut_peak_probe(kind, blocks, threads, iters, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == abi.UT_OK
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_fma_probe_computes_its_chains(L):
    blocks, threads, iters = 2, 64, 7
    got = _run(L, abi.UT_PROBE_FMA, blocks, threads, iters)
    t = np.tile(np.arange(threads), blocks)
    a, b = np.float32(0.999), np.float32(1e-3)
    s = np.zeros(blocks * threads, np.float32)
    for j in range(8):
        x = (np.float32(1e-3) * t.astype(np.float32) + np.float32(j)).astype(np.float32)
        for _ in range(iters):  # one rounding per fused multiply-add (the FP64 product is exact)
            x = (x.astype(np.float64) * np.float64(a) + np.float64(b)).astype(np.float32)
        s = (s + x).astype(np.float32)
    np.testing.assert_allclose(got, s, rtol=2e-7, atol=0)


def test_ex2_probe_computes_its_chains(L):
    blocks, threads, iters = 1, 96, 5
    got = _run(L, abi.UT_PROBE_EX2, blocks, threads, iters)
    t = np.arange(threads, dtype=np.float64)
    s = np.zeros(threads)
    for j in range(8):
        x = np.float32(1e-3) * t.astype(np.float32) + np.float32(0.1) * np.float32(j)
        x = x.astype(np.float64)
        for _ in range(iters):
            x = 2.0 ** (-x)
        s += x
    np.testing.assert_allclose(got, s, rtol=1e-5)


def test_fma_probe_rate_is_plausible(L):
    """8 blocks of 256 per SM, 40000 iterations: the measured FP32 rate is between a third of and
    10 % above 128 lanes x 2 flop x 2.1 GHz per SM (the top boost clock of this part)."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks, threads, iters = sms * 8, 256, 40000
    out = torch.empty(blocks * threads, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream()
    launch = lambda: L.ut_peak_probe(abi.UT_PROBE_FMA, blocks, threads, iters, out.data_ptr(), s.cuda_stream)  # noqa: E731
    assert launch() == abi.UT_OK
    torch.cuda.synchronize()
    ts = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        launch()
        e1.record(s)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    rate = blocks * threads * iters * 8 * 2.0 / (min(ts) / 1e3)
    nominal = sms * 128 * 2 * 2.1e9
    assert nominal / 3 < rate < 1.1 * nominal, (rate, nominal)
    assert np.all(np.isfinite(out.cpu().numpy()))
