"""The allocation-free partial Gramian, for callers that cannot allocate.

Such callers (device memory owned by another allocator, or a latency-bound
loop that must not call cudaMalloc / cudaFree) use
ials_partial_gramian_noalloc, which keeps its split-K partials in a fixed
device array.  This file is collected last so that a failure here cannot stop
the other GPU tests from running first.  It checks the new entry point against
the allocating one, through the C ABI, on two calls in a row (the fixed array
keeps the previous call's contents, which must not leak into the next result).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_14044_gb300 import _abi, build
    build.build()
    return _abi


def test_noalloc_gramian_matches_allocating_entry_point_twice(abi):
    import torch
    rng = np.random.default_rng(21)
    cases = [(20011, 128, 32, 32), (136000, 128, 96, 32), (777, 16, 8, 8), (41000, 1024, 128, 128),
             (3000, 1100, 100, 1000)]  # the last needs fewer row ranges to fit the scratch
    stream = torch.cuda.current_stream()
    for n, d, p0, bs in cases:
        X = torch.from_numpy(rng.normal(0, 1, (n, d)).astype(np.float32)).cuda()
        ref = torch.empty((d, bs), dtype=torch.float32, device="cuda")
        abi.ials_partial_gramian(X, n, d, p0, bs, ref, stream)
        want = ref.cpu().numpy()
        scale = np.abs(want).max()
        for _ in range(2):  # the second call reuses the scratch the first one filled
            G = torch.full((d, bs), float("nan"), dtype=torch.float32, device="cuda")
            abi.ials_partial_gramian_noalloc(X, n, d, p0, bs, G, stream)
            torch.cuda.synchronize()
            got = G.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert np.abs(got - want).max() <= 1e-5 * scale, (n, d, bs)


def test_noalloc_gramian_rejects_oversized_problem(abi):
    import torch
    X = torch.zeros((4, 4096), dtype=torch.float32, device="cuda")
    G = torch.zeros((4096, 1024), dtype=torch.float32, device="cuda")
    with pytest.raises(abi.IalsError) as ei:
        abi.ials_partial_gramian_noalloc(X, 4, 4096, 0, 1024, G)
    assert ei.value.status == abi.EINVAL
    assert "scratch" in abi.ials_last_error()


def test_noalloc_gramian_rejects_host_arrays(abi):
    import torch
    n, d, bs = 64, 16, 8
    Xh = np.ones((n, d), np.float32)
    Gh = np.zeros((d, bs), np.float32)
    Xd = torch.ones((n, d), dtype=torch.float32, device="cuda")
    Gd = torch.zeros((d, bs), dtype=torch.float32, device="cuda")
    for X, G in ((Xh, Gd), (Xd, Gh), (Xh, Gh)):
        with pytest.raises(abi.IalsError) as ei:
            abi.ials_partial_gramian_noalloc(X, n, d, 0, bs, G)
        assert ei.value.status == abi.EINVAL
        assert "device" in abi.ials_last_error()


def test_noalloc_gramian_allocates_no_device_memory(abi):
    """After the first call (which looks up the fixed array's address), further
    calls leave both the driver's free-memory count and torch's allocator as they were."""
    import torch
    n, d, bs = 50000, 256, 64
    X = torch.randn((n, d), dtype=torch.float32, device="cuda")
    G = torch.empty((d, bs), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    abi.ials_partial_gramian_noalloc(X, n, d, 0, bs, G, stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    for p0 in (0, 64, 128, 192):
        abi.ials_partial_gramian_noalloc(X, n, d, p0, bs, G, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0
    for key in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
        assert stats1.get(key, 0) == stats0.get(key, 0), key
