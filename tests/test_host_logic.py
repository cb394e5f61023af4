"""Host-side logic that needs no GPU: the autotuner's admissible block sizes,
the benchmark's DRAM-traffic record and its fold-in request generator."""
import numpy as np

import bench
from paper_2110_14044_gb300 import _abi, autotune


def test_admissible_block_sizes():
    fp32, bf16 = _abi.PREC_FP32, _abi.PREC_BF16
    # b must divide d and not exceed it (contiguous blocks [k b, (k+1) b))
    assert autotune.admissible(128, 32, fp32)
    assert autotune.admissible(128, 128, fp32)   # b = d: Algorithm 1
    assert autotune.admissible(128, 1, fp32)     # b = 1: Algorithm 2
    assert not autotune.admissible(64, 128, fp32)
    assert not autotune.admissible(48, 32, fp32)
    assert not autotune.admissible(96, 3, fp32)  # not a supported kernel width
    # the BF16 pattern runs on 16-row tensor-core tiles
    assert autotune.admissible(128, 16, bf16) and autotune.admissible(1024, 128, bf16)
    assert not autotune.admissible(128, 8, bf16)
    assert [b for b in autotune.CANDIDATES if autotune.admissible(64, b, fp32)] == [1, 2, 4, 8, 16, 32, 64]
    assert autotune.admissible(512, 256, fp32) and not autotune.admissible(512, 256, bf16)
    # b = d above 256 (iALS, FP32 only): d a multiple of 64 up to 1024
    assert autotune.admissible(512, 512, fp32) and autotune.admissible(1024, 1024, fp32)
    assert autotune.admissible(320, 320, fp32) and not autotune.admissible(2048, 2048, fp32)
    assert not autotune.admissible(512, 512, bf16) and not autotune.admissible(1024, 512, fp32)
    assert [b for b in autotune.CANDIDATES if autotune.admissible(64, b, bf16)] == [16, 32, 64]


def test_traffic_record_applies_only_to_its_workload_and_sources(monkeypatch):
    rec = dict(bench.NCU_TRAFFIC[("sparse", "bf16")])
    wl = rec["workload"]
    current = bench.sources_hash(rec["sources"])
    rec["sha256_16"] = current
    monkeypatch.setitem(bench.NCU_TRAFFIC, ("sparse", "bf16"), rec)
    assert bench.measured_traffic("sparse", "bf16", wl) == rec["bytes_per_launch"]
    # another workload (or the same one at another d or b) gets no traffic figure
    assert bench.measured_traffic("sparse", "bf16", ("msd_570k", 1024, 32)) is None
    assert bench.measured_traffic("sparse", "bf16", (wl[0], wl[1], 16)) is None
    # nor does a kernel whose sources changed since the capture
    rec2 = dict(rec, sha256_16="0" * 16)
    monkeypatch.setitem(bench.NCU_TRAFFIC, ("sparse", "bf16"), rec2)
    assert bench.measured_traffic("sparse", "bf16", wl) is None
    assert bench.measured_traffic("gram", "bf16", wl) is None


def test_foldin_requests_follow_the_recipe():
    rng = np.random.default_rng(3)
    n_items = 41000
    p = np.arange(1, n_items + 1, dtype=np.float64) ** -1.0
    cdf = np.cumsum(p / p.sum())
    cdf[-1] = 1.0
    reqs = bench.foldin_requests(rng, n_items, 400, cdf)
    lens = np.array([r.size for r in reqs])
    assert lens.min() >= 1 and lens.max() <= 5000
    for r in reqs:
        assert r.dtype == np.int32
        assert np.unique(r).size == r.size          # distinct items per history
        assert r.min() >= 0 and r.max() < n_items
    # log-uniform on [1, 5000]: the median length is near sqrt(5000) ~ 71
    assert 30 < np.median(lens) < 150
    # Zipf popularity: item 0 (the most popular here) is in far more histories than item 40,000
    counts = np.bincount(np.concatenate(reqs), minlength=n_items)
    assert counts[0] > 10 * max(1, counts[40000])


def test_launch_count_per_epoch_matches_the_kernel_structure():
    """ML20M shape, d = 128, b = 32 (4 blocks, both sides split long rows): the
    ncu launch list of a BF16 epoch holds 65 kernels (sparse, split solve,
    split residual, retry, tcgen05 Gramian, its reduction, G transpose-split
    and tcgen05 row terms 8 each, one residual recompute)."""
    steps = 3
    marks = {"residual": 1, "gram": 8, "rowterm": 8, "sparse": 8, "split_solve": 8,
             "split_resid": 8, "retry": 8, "objective": 0}
    kern = {k: (1.0, c * steps) for k, c in marks.items()}
    assert bench.launches_per_epoch(kern, steps, True, 32) == 65
    # FP32: Gramian tile + reduction, one row-term kernel
    assert bench.launches_per_epoch(kern, steps, False, 32) == 57
    # BF16 at b = 128 = d: one block, 4 slabs of 32 columns per Gramian and row term
    marks1 = dict(marks, gram=2, rowterm=2, sparse=2, split_solve=2, split_resid=2, retry=2)
    kern1 = {k: (1.0, c) for k, c in marks1.items()}
    assert bench.launches_per_epoch(kern1, 1, True, 128) == 1 + 2 * 8 + 2 * 8 + 4 * 2
