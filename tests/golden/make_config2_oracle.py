"""Writes config2_oracle.json: the FP64 oracle's sequential per-entry SGD (Alg. 1 with one
worker) on the paper-scale synthetic problem (4,500 x 15,000 x 5, 27M training entries,
core 10 x 10 x 5, 300,000-edge gene network), test RMSE after each of 10 epochs.

Calls only oracle/ and snect_synth/.  About 10-15 minutes on one core.
Usage: python tests/golden/make_config2_oracle.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import snect_synth as S  # noqa: E402


def main():
    p = S.config2()
    P = oracle.Params(p.G0, p.U0)
    out = {"workload": "config2 (seed 2): 4500x15000x5, 27M train / 3M test, core 10x10x5, lam 0.01, "
                       "lam_g 0.1, lr 0.01, sequential per-entry SGD + network pass per epoch",
           "rmse_test_init": oracle.rmse(P, p.test_idx, p.test_val), "rmse_test": [], "rmse_train": [],
           "seconds_per_epoch": []}
    for ep in range(p.epochs):
        t0 = time.time()
        oracle.sgd_epoch(p.I, P, p.lam, p.lam_g, p.lr, p.idx, p.val, p.edges, p.w)
        out["seconds_per_epoch"].append(time.time() - t0)
        out["rmse_test"].append(oracle.rmse(P, p.test_idx, p.test_val))
        out["rmse_train"].append(oracle.rmse(P, p.idx, p.val))
        print(ep + 1, out["rmse_test"][-1], out["seconds_per_epoch"][-1], flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "config2_oracle.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
