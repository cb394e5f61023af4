"""Write msd_subsample_trace.json: the FP64 oracle's objective per epoch on the
1% user subsample of the MSD-shaped workload (d = 1024, b = 128, 8 epochs of
Algorithm 3), so that the GPU path can be compared with it epoch by epoch
without re-running the oracle (tens of minutes of host time).

Inputs come from the seeded generator alone; every stored number comes from
the oracle.  The file also holds a fingerprint of the inputs (CSR and initial
factors), so a reader can tell whether it regenerated the same problem.

    python tests/golden/make_msd_subsample_trace.py [--threads N]
"""
import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2110_14044_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "msd_subsample_trace.json")


def subsample():
    """The MSD-shaped preset at 1/100 of its users and positives, all items."""
    cfg = synth.PRESETS["msd_570k"]
    return synth.preset("msd_570k", seed=0, n_users=cfg["n_users"] // 100, nnz=cfg["nnz"] // 100)


def fingerprint(prob):
    h = hashlib.sha256()
    for a in (prob.data.u_indptr, prob.data.u_items, prob.W0, prob.H0):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--epochs", type=int, default=8)
    args = ap.parse_args()
    prob = subsample()
    P = oracle.Problem.from_data(prob.data, prob.d, prob.b, prob.alpha0, prob.lam, prob.nu,
                                 n_threads=args.threads or None)
    rec = {
        "about": "FP64 oracle (Algorithm 3) on the 1% user subsample of the MSD-shaped workload; "
                 "objective L(W,H) of Eq. 2 before and after each epoch. Written by "
                 "tests/golden/make_msd_subsample_trace.py from the seeded generator and oracle/ only.",
        "cite": "Algorithm 3; Eq. 2; Table 2 (MSD alpha0, lambda)",
        "problem": {"n_users": prob.data.n_users, "n_items": prob.data.n_items, "nnz": int(prob.data.nnz),
                    "d": prob.d, "b": prob.b, "alpha0": prob.alpha0, "lambda": prob.lam, "nu": prob.nu,
                    "seed": 0},
        "inputs_sha256_16": fingerprint(prob),
        "threads": P.n_threads,
        "objective_before": float(oracle.objective(P, prob.W0, prob.H0)),
        "objective_after_epoch": [],
        "seconds_per_epoch": [],
    }
    W, H = prob.W0, prob.H0
    for e in range(args.epochs):
        t0 = time.perf_counter()
        # one epoch per call (each call recomputes yhat first, as every epoch of
        # Algorithm 3 does, so this equals one multi-epoch run); the objective
        # once per epoch rather than after every half-step
        W, H, _, _, st = oracle.ialspp(P, 1, W, H)
        if st != 0:
            raise SystemExit(f"oracle status {st} in epoch {e + 1}")
        obj = float(oracle.objective(P, W, H))
        rec["objective_after_epoch"].append(obj)
        rec["seconds_per_epoch"].append(round(time.perf_counter() - t0, 1))
        print(f"epoch {e + 1}: L = {obj:.12g} ({rec['seconds_per_epoch'][-1]} s)", flush=True)
        with open(OUT + ".partial", "w") as f:
            json.dump(rec, f, indent=1)
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    os.remove(OUT + ".partial")


if __name__ == "__main__":
    main()
