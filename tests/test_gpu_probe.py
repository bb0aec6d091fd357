"""The memory-level probes that give the annealer's roofline its denominators
(satpila_probe_read / satpila_probe_smem): plausible, ordered rates."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1411_4622_gb300 import api as a
    from paper_1411_4622_gb300 import build

    build.build()
    torch.cuda.set_device(0)
    return a


def test_probe_rates_are_ordered(api):
    l2 = torch.ones(64 << 20, dtype=torch.uint8, device="cuda")
    big = torch.ones(2 << 30, dtype=torch.uint8, device="cuda")
    l2_stream = api.probe_read(l2, api.PROBE_STREAM, loads=1 << 28)
    l2_sector = api.probe_read(l2, api.PROBE_SECTOR, loads=1 << 26)
    hbm_stream = api.probe_read(big, api.PROBE_STREAM, loads=1 << 27)
    hbm_sector = api.probe_read(big, api.PROBE_SECTOR, loads=1 << 25, region_bytes=1 << 20)
    smem = api.probe_smem(0, loads=1 << 30)
    smem_rand = api.probe_smem(1, loads=1 << 29)
    # every rate positive and below a physical bound (100 TB/s)
    for r in (l2_stream, l2_sector, hbm_stream, hbm_sector, smem, smem_rand):
        assert 0 < r < 1e5
    # a buffer 16x larger than L2 streams slower than one inside it, and a
    # scattered sector gather from HBM is slower than streaming it
    assert hbm_stream < l2_stream
    assert hbm_sector < hbm_stream
    # scattered words meet bank conflicts
    assert smem_rand < smem


def test_probe_rejects_bad_arguments(api):
    import numpy as np

    with pytest.raises(api.SatpilaError):
        api.probe_read(torch.ones(1024, dtype=torch.uint8, device="cuda"), api.PROBE_STREAM)  # < 4096 B
    with pytest.raises(api.SatpilaError):
        api.probe_read(torch.ones(8192, dtype=torch.uint8, device="cuda"), 7)
    with pytest.raises(TypeError):
        api.probe_read(np.ones(8192, np.uint8), api.PROBE_STREAM)  # host arrays have no numel
