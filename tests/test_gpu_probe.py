"""The random-sector probe behind the shard roofline touches exactly the
sectors its definition names (sbf_probe_sectors: sector i of a run is
floor(mix64(seed + i) * n_sectors / 2^64))."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

M64 = (1 << 64) - 1


def _mix64(x: int) -> int:
    x ^= x >> 30
    x = (x * 0xBF58476D1CE4E5B9) & M64
    x ^= x >> 27
    x = (x * 0x94D049BB133111EB) & M64
    return x ^ (x >> 31)


@pytest.fixture(scope="module")
def torch_dev():
    import torch

    from paper_2606_24417_gb300 import build_lib

    build_lib.build()
    return torch, torch.device("cuda", 0)


@pytest.mark.parametrize("sector_bytes", [32, 64])
def test_rmw_sets_the_defined_bits(torch_dev, sector_bytes):
    from paper_2606_24417_gb300.sbf import probe_sectors

    torch, dev = torch_dev
    n_sectors, n, seed = 1000, 5000, 7
    buf = torch.zeros(n_sectors * sector_bytes, dtype=torch.uint8, device=dev)
    probe_sectors(buf, sector_bytes, n, seed=seed, rmw=True)
    torch.cuda.synchronize()
    got = buf.cpu().numpy().view(np.uint64)
    W = sector_bytes // 8
    want = np.zeros(n_sectors * W, dtype=np.uint64)
    for i in range(n):
        h = _mix64((seed + i) & M64)
        x = (h * n_sectors) >> 64
        for part in range(W):
            want[x * W + part] |= np.uint64(1 << ((h >> (6 * part)) & 63))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("sector_bytes", [32, 64])
def test_gather_runs_and_leaves_the_buffer(torch_dev, sector_bytes):
    from paper_2606_24417_gb300.sbf import probe_sectors

    torch, dev = torch_dev
    buf = torch.arange(1 << 20, dtype=torch.int64, device=dev)
    before = buf.clone()
    sink = torch.zeros(1, dtype=torch.int64, device=dev)
    probe_sectors(buf, sector_bytes, 1 << 22, seed=3, sink=sink)
    probe_sectors(buf, sector_bytes, 0, seed=3, sink=sink)  # n = 0: nothing launched
    torch.cuda.synchronize()
    assert torch.equal(buf, before)
    assert int(sink.item()) <= 1 << 22
