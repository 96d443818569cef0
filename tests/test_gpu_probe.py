"""The FP64 FMA probe (include/exa_probe.h) that gives the FP64 roofline its measured peak."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_fp64_fma_probe_is_plausible():
    """The measured rate lies between a tenth and twice the rate derived from the unit counts
    (2 FP64 operations per clock per SM at the maximum clock), and repeats within 10 %."""
    from paper_2608_16265_gb300 import binding as B
    props = torch.cuda.get_device_properties(0)
    a = B.exa_probe_fp64_fma(0, 100.0)
    b = B.exa_probe_fp64_fma(0, 100.0)
    assert a["sms"] == props.multi_processor_count
    derived = 2 * a["sms"] * 2.07e9
    assert 0.1 * derived < a["dfma_per_s"] < 2.0 * derived, a
    assert abs(a["dfma_per_s"] - b["dfma_per_s"]) <= 0.1 * max(a["dfma_per_s"], b["dfma_per_s"])
    assert 50.0 <= a["ms"] <= 400.0
    with pytest.raises(B.ExaError):
        B.exa_probe_fp64_fma(999, 100.0)


def test_host_link_probe_is_plausible():
    """Both directions of the host link measure between 10 GB/s and 2 TB/s."""
    from paper_2608_16265_gb300 import binding as B
    r = B.exa_probe_host_link(0, 256 << 20)
    for k in ("h2d_bytes_per_s", "d2h_bytes_per_s"):
        assert 1e10 < r[k] < 2e12, r
