"""Write the FP64 oracle's objective trace (Algorithm 3, Eq. 2 after every
epoch) for one of the stored cases, so that GPU tests can compare the CUDA
path with it epoch by epoch without re-running the oracle (minutes to tens of
minutes of host time).

Cases (inputs from the seeded generator alone; every stored number comes from
the oracle):

  msd_sub_b128   the 1% user subsample of the MSD-shaped workload (5,700 x
                 41,000, 340,000 positives), d = 1024, b = 128, 8 epochs
                 -> msd_subsample_trace.json
  msd_sub_b32    the same subsample at b = 32, 8 epochs
                 -> msd_subsample_b32_trace.json
  ml20m_b32      the whole ML20M-shaped workload (136,000 x 20,000, 10M
                 positives), d = 128, b = 32, 16 epochs -> ml20m_trace.json

Each file also holds a fingerprint of the inputs (CSR and initial factors), so
a reader can tell whether it regenerated the same problem.

    python tests/golden/make_oracle_trace.py CASE [--threads N]
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


def msd_subsample(b):
    """The MSD-shaped preset at 1/100 of its users and positives, all items."""
    cfg = synth.PRESETS["msd_570k"]
    return synth.preset("msd_570k", seed=0, n_users=cfg["n_users"] // 100, nnz=cfg["nnz"] // 100, b=b)


CASES = {
    "msd_sub_b128": dict(make=lambda: msd_subsample(128), epochs=8, out="msd_subsample_trace.json",
                         about="the 1% user subsample of the MSD-shaped workload",
                         cite="Algorithm 3; Eq. 2; Table 2 (MSD alpha0, lambda)"),
    "msd_sub_b32": dict(make=lambda: msd_subsample(32), epochs=8, out="msd_subsample_b32_trace.json",
                        about="the 1% user subsample of the MSD-shaped workload, b = 32",
                        cite="Algorithm 3; Eq. 2; Table 2 (MSD alpha0, lambda)"),
    "ml20m_b32": dict(make=lambda: synth.preset("ml20m_136k", seed=0), epochs=16, out="ml20m_trace.json",
                      about="the whole ML20M-shaped workload",
                      cite="Algorithm 3; Eq. 2; Table 2 (ML20M shape)"),
}


def fingerprint(prob):
    h = hashlib.sha256()
    for a in (prob.data.u_indptr, prob.data.u_items, prob.W0, prob.H0):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=sorted(CASES))
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--epochs", type=int, default=0)
    args = ap.parse_args()
    case = CASES[args.case]
    epochs = args.epochs or case["epochs"]
    out = os.path.join(HERE, case["out"])
    prob = case["make"]()
    P = oracle.Problem.from_data(prob.data, prob.d, prob.b, prob.alpha0, prob.lam, prob.nu,
                                 n_threads=args.threads or None)
    rec = {
        "about": f"FP64 oracle (Algorithm 3) on {case['about']}; objective L(W,H) of Eq. 2 before "
                 f"and after each epoch. Written by tests/golden/make_oracle_trace.py "
                 f"{args.case} from the seeded generator and oracle/ only.",
        "cite": case["cite"],
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
    for e in range(epochs):
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
        with open(out + ".partial", "w") as f:
            json.dump(rec, f, indent=1)
    with open(out, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    os.remove(out + ".partial")


if __name__ == "__main__":
    main()
