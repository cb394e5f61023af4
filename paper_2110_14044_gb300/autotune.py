"""Block-size autotuner.

The block size b of iALS++ changes the work per epoch (the sparse statistics
grow with b^2 per interaction, the solves with b^3 per row, the number of
passes over S with d / b) but not the quality of the model (Section 5.2.2, Fig.
2: final quality is flat in b).  The candidates run from b = 1 (iCD, Alg. 2)
to b = d (iALS, Alg. 1) where d allows.  It is therefore a system parameter: this
module times one epoch of the library for every admissible b on the given
workload and returns the fastest, together with the measured table.

Timing uses CUDA events on the context's stream around a CUDA-graph epoch,
after one warm-up epoch (which also captures the graph).
"""
from __future__ import annotations

import numpy as np

from . import _abi

CANDIDATES = (1, 2, 4, 8, 16, 32, 64, 128, 256)  # b = 1 is iCD (Alg. 2); b = d is iALS (Alg. 1)


def admissible(d: int, b: int, precision: int) -> bool:
    if d % b != 0 or b > d:
        return False
    if precision == _abi.PREC_BF16:
        return b in (16, 32, 64, 128) and d % 8 == 0
    return b in (1, 2, 4, 8, 16, 32, 64, 128, 256)


def autotune_block_size(data, d, alpha0, lam, nu=0.0, precision=_abi.PREC_FP32,
                        candidates=CANDIDATES, epochs=2, W0=None, H0=None, seed=0):
    """Return (best_b, table) with table[b] = seconds per epoch."""
    import torch

    from . import Model
    stream = torch.cuda.Stream()
    table = {}
    for b in candidates:
        if not admissible(d, b, precision):
            continue
        m = Model(data, d, b, alpha0, lam, nu, precision=precision, graph=True, stream=stream,
                  seed=seed, W0=W0, H0=H0)
        m.epoch(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        m.epoch(epochs)
        e1.record(stream)
        torch.cuda.synchronize()
        table[b] = e0.elapsed_time(e1) / 1e3 / epochs
        m.close()
    if not table:
        raise ValueError(f"no admissible block size for d={d}")
    best = min(table, key=table.get)
    return best, table
