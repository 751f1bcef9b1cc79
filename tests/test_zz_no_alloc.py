"""md_partition_noalloc: the partition entry point for callers that cannot
allocate device memory while they run.  It must give the same bounds as
md_partition (which allocates its scan scratch), call after call, although
every call reuses the same fixed scratch array.  Kept in a file of its own
that pytest collects last."""
import numpy as np
import pytest

from paper_1611_00075_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def md():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_00075_gb300 import build
    build.build()
    from paper_1611_00075_gb300 import md as _md
    torch.cuda.set_device(0)
    _md.lib()
    return _md


def costs(seed, ncells):
    c = (inputs.splitmix64(seed, ncells) % 50000).astype(np.int64)
    c[inputs.splitmix64(seed + 1, ncells // 4 + 1) % ncells] = 0
    return torch.from_numpy(c).cuda()


def test_noalloc_matches_allocating_partition_twice_in_a_row(md):
    # two different calls back to back: the second one runs on whatever the
    # first left in the shared scratch, and must still be exact
    for seed, ncells, nparts in ((901, 857375, 4864), (902, 1000, 7)):
        c = costs(seed, ncells)
        ref = torch.empty(nparts + 1, dtype=torch.int64, device="cuda")
        got = torch.full((nparts + 1,), -1, dtype=torch.int64, device="cuda")
        md.md_partition(c, nparts, ref)
        md.md_partition_noalloc(c, nparts, got)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), (seed, ncells, nparts)


def test_noalloc_rejects_sizes_beyond_its_scratch(md):
    c = torch.zeros((1 << 20) + 1, dtype=torch.int64, device="cuda")
    b = torch.empty(9, dtype=torch.int64, device="cuda")
    with pytest.raises(md.MDError) as e:
        md.md_partition_noalloc(c, 8, b)
    assert e.value.status == md.MD_ERR_INVALID
    assert "scratch limit" in str(e.value)


def test_noalloc_at_its_exact_size_limit(md):
    # 2^20 cells fill the scratch to its last tile sum; an awkward part count
    for seed, nparts in ((903, 4861), (904, 3)):
        c = costs(seed, 1 << 20)
        ref = torch.empty(nparts + 1, dtype=torch.int64, device="cuda")
        got = torch.full((nparts + 1,), -1, dtype=torch.int64, device="cuda")
        md.md_partition(c, nparts, ref)
        md.md_partition_noalloc(c, nparts, got)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), (seed, nparts)


def test_noalloc_inside_a_captured_graph(md):
    """After one call on the device, md_partition_noalloc is captured into a
    CUDA graph on a side stream; replays with new costs copied into the
    captured input give md_partition's bounds."""
    ncells, nparts = 300000, 1001
    c = costs(905, ncells)
    got = torch.full((nparts + 1,), -1, dtype=torch.int64, device="cuda")
    md.md_partition_noalloc(c, nparts, got)  # the first call on the device
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        md.md_partition_noalloc(c, nparts, got, stream=side)
    for seed in (906, 907):
        c.copy_(costs(seed, ncells))
        got.fill_(-1)
        g.replay()
        ref = torch.empty(nparts + 1, dtype=torch.int64, device="cuda")
        md.md_partition(c, nparts, ref)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), seed
