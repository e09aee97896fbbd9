"""The measured pipe rates (C ABI sbio_measure_peaks), the roofline
denominators of the far and near kernels: each rate lies below what the
multiprocessor count and the measured clock allow for its pipe (128 FP32
lanes, at most 64 FP64 lanes and 32 MUFU lanes per SM per clock) and above a
tenth of it."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as G

    G.build()
    import paper_2506_20809_gb300.sbio as S

    return S


def test_measured_peaks_are_plausible(S):
    pk = S.sbio_measure_peaks(0)
    assert pk["sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    ghz = pk["sm_clock_mhz"] / 1e3
    assert 0.3 < ghz < 3.0
    fp32 = pk["sms"] * 128 * 2 * ghz / 1e3          # TFLOP/s at the measured clock
    for key in ("fp32_ffma_tflops", "fp32_ffma2_tflops"):
        assert 0.1 * fp32 < pk[key] < 1.05 * fp32, (key, pk[key], fp32)
    assert 0 < pk["rsqrt_per_s"] < 1.05 * pk["sms"] * 32 * ghz * 1e9
    assert 0 < pk["fp64_dfma_tflops"] < 1.05 * pk["sms"] * 64 * 2 * ghz / 1e3
    # the pair mix can go no faster than its FP32 share allows (11 f32x2 per 2 pairs)
    assert 0 < pk["pairmix_pairs_per_s"] < 1.05 * pk["fp32_ffma2_tflops"] * 1e12 / 22.0
    # fed from shared memory the pair cannot be faster than from registers
    assert 0 < pk["pairsmem_pairs_per_s"] < 1.05 * pk["pairmix_pairs_per_s"]
