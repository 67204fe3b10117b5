"""The measurement helpers the benchmark's roofline uses (GPU)."""
import pytest

torch = pytest.importorskip("torch")

from paper_2605_00038_gb300 import lbp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def test_smem_probe_reports_plausible_bandwidth():
    """The shared-memory probe loads 2 x SMs x 1024 threads x trips x 8 x 16
    bytes; its rate must lie between a tenth of and twice the nominal
    152 SMs x 128 B/clock x 2.07 GHz (40.3 TB/s)."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    b, ms = lbp.lbp_probe_smem(512)
    assert b == 2 * sms * 1024 * 512 * 8 * 16
    assert ms > 0
    bps = b / (ms / 1e3)
    assert 4.0e12 < bps < 80.0e12, bps
    with pytest.raises(lbp.LbpError):
        lbp.lbp_probe_smem(0)
