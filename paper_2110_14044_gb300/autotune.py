"""Block-size autotuner.

The block size b of iALS++ changes the work per epoch (the sparse statistics
grow with b^2 per interaction, the solves with b^3 per row, the number of
passes over S with d / b) but not the quality of the model (Section 5.2.2, Fig.
2: final quality is flat in b).  The candidates run from b = 1 (iCD, Alg. 2)
to b = d (iALS, Alg. 1) where d allows.  It is therefore a system parameter: this
module times one epoch of the library for every admissible b on the given
workload and returns the fastest, together with the measured table.

The work decomposition is tuned the same way: with b fixed, `autotune` also
times the split length (rows longer than it are cut into chunks whose
statistics are summed in chunk order), which sets the load balance of the
persistent sparse launch on skewed histories.

Timing uses CUDA events on the context's stream around a CUDA-graph epoch,
after one warm-up epoch (which also captures the graph).
"""
from __future__ import annotations

import numpy as np

from . import _abi

CANDIDATES = (1, 2, 4, 8, 16, 32, 64, 128, 256)  # b = 1 is iCD (Alg. 2); b = d is iALS (Alg. 1)
SPLIT_CANDIDATES = (0, 512, 2048, 8192)  # 0: the library's choice from nnz


def admissible(d: int, b: int, precision: int) -> bool:
    if d % b != 0 or b > d:
        return False
    if precision == _abi.PREC_BF16:
        return b in (16, 32, 64, 128) and d % 8 == 0
    if b == d and 256 < d <= 1024 and d % 64 == 0:  # iALS (Algorithm 1) at large d
        return True
    return b in (1, 2, 4, 8, 16, 32, 64, 128, 256)


def time_epoch(data, d, b, alpha0, lam, nu=0.0, precision=_abi.PREC_FP32, epochs=2, W0=None,
               H0=None, seed=0, split_len=0, stream=None):
    """Seconds per graph-replayed epoch of one configuration (one warm-up epoch first)."""
    import torch

    from . import Model
    stream = stream if stream is not None else torch.cuda.Stream()
    m = Model(data, d, b, alpha0, lam, nu, precision=precision, graph=True, stream=stream,
              seed=seed, W0=W0, H0=H0, split_len=split_len)
    try:
        m.epoch(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        m.epoch(epochs)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / epochs
    finally:
        m.close()


def autotune_block_size(data, d, alpha0, lam, nu=0.0, precision=_abi.PREC_FP32,
                        candidates=CANDIDATES, epochs=2, W0=None, H0=None, seed=0, stream=None):
    """Return (best_b, table) with table[b] = seconds per epoch."""
    table = {}
    for b in candidates:
        if not admissible(d, b, precision):
            continue
        table[b] = time_epoch(data, d, b, alpha0, lam, nu, precision, epochs, W0, H0, seed,
                              stream=stream)
    if not table:
        raise ValueError(f"no admissible block size for d={d}")
    best = min(table, key=table.get)
    return best, table


def autotune(data, d, alpha0, lam, nu=0.0, precision=_abi.PREC_FP32, candidates=CANDIDATES,
             split_candidates=SPLIT_CANDIDATES, epochs=2, W0=None, H0=None, seed=0, stream=None):
    """Tune b, then the split length at that b.

    Returns {"b": best b, "split_len": best split length (0 = library choice),
    "epoch_s_by_b": {b: s}, "epoch_s_by_split_len": {split_len: s}, "epoch_s": s}."""
    best_b, by_b = autotune_block_size(data, d, alpha0, lam, nu, precision, candidates, epochs,
                                       W0, H0, seed, stream)
    by_split = {0: by_b[best_b]}
    for sl in split_candidates:
        if sl not in by_split:
            by_split[sl] = time_epoch(data, d, best_b, alpha0, lam, nu, precision, epochs, W0, H0,
                                      seed, sl, stream)
    best_sl = min(by_split, key=by_split.get)
    return {"b": best_b, "split_len": best_sl, "epoch_s_by_b": by_b,
            "epoch_s_by_split_len": by_split, "epoch_s": by_split[best_sl]}
