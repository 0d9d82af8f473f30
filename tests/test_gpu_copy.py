"""mihs_copy_to_device: pinned, aligned host memory read by the SMs; pageable,
unaligned and tail bytes through cudaMemcpyAsync.  mihs_copy_to_device_dma:
a copy engine for all of it.  Byte-exact in every case."""
import pytest
import torch

from paper_1912_03514_gb300 import mihs
from paper_1912_03514_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.mark.parametrize("numel", [1, 3, 4, 1001, 4096, 1 << 20, (1 << 22) + 5])
@pytest.mark.parametrize("pinned", [True, False])
def test_copy_to_device_is_exact(numel, pinned):
    src = W.randn((numel,), 7 + numel)
    if pinned:
        src = src.pin_memory()
    dst = torch.full((numel,), float("nan"), device=DEV)
    c0 = mihs.launch_count()
    mihs.copy_to_device(dst, src)
    torch.cuda.synchronize()
    assert torch.equal(dst.cpu(), src)
    # the SM path runs a kernel whenever at least 16 aligned bytes come from pinned memory
    assert (mihs.launch_count() > c0) == (pinned and numel >= 4)


def test_copy_unaligned_offsets_and_views():
    base = W.randn((4099,), 3).pin_memory()
    for off in (1, 2, 3):
        src = base[off:off + 4000]
        dst = torch.empty(4000, device=DEV)
        mihs.copy_to_device(dst, src)
        torch.cuda.synchronize()
        assert torch.equal(dst.cpu(), src)
    dst = torch.empty(4000, device=DEV)
    out = torch.empty(4004, device=DEV)
    mihs.copy_to_device(out[1:4001], base[:4000])  # unaligned destination
    torch.cuda.synchronize()
    assert torch.equal(out[1:4001].cpu(), base[:4000])


def test_copy_concurrent_streams():
    srcs = [W.randn((1 << 22,), 40 + k).pin_memory() for k in range(3)]
    dsts = [torch.empty(1 << 22, device=DEV) for _ in range(3)]
    streams = [torch.cuda.Stream() for _ in range(3)]
    for s_, src, dst in zip(streams, srcs, dsts):
        mihs.copy_to_device(dst, src, stream=s_)
    torch.cuda.synchronize()
    for src, dst in zip(srcs, dsts):
        assert torch.equal(dst.cpu(), src)


def test_copy_rejects_bad_arguments():
    with pytest.raises(ValueError):
        mihs.copy_to_device(torch.empty(4, device=DEV), torch.empty(5))
    with pytest.raises(ValueError):
        mihs.copy_to_device(torch.empty(4), torch.empty(4))
    with pytest.raises(mihs.MihsError):  # destination on the host
        mihs._check(mihs.lib().mihs_copy_to_device(torch.empty(4).data_ptr(), torch.empty(4).data_ptr(), 16, None))


@pytest.mark.parametrize("numel", [1, 1001, (1 << 22) + 5])
@pytest.mark.parametrize("pinned", [True, False])
def test_copy_engine_form_is_exact_and_launches_nothing(numel, pinned):
    src = W.randn((numel,), 70 + numel)
    if pinned:
        src = src.pin_memory()
    dst = torch.full((numel,), float("nan"), device=DEV)
    c0 = mihs.launch_count()
    mihs.copy_to_device(dst, src, engine="dma")
    torch.cuda.synchronize()
    assert torch.equal(dst.cpu(), src)
    assert mihs.launch_count() == c0
    with pytest.raises(ValueError):
        mihs.copy_to_device(dst, src, engine="tma")
    with pytest.raises(mihs.MihsError):  # destination on the host
        mihs._check(mihs.lib().mihs_copy_to_device_dma(torch.empty(4).data_ptr(), src.data_ptr(), 4, None))
