"""Train the classifier and the ln K initializer (Sec. 4) on the GPU with the
library's own kernels, on plain-method flashes of the 10-pseudo-component
workload (T in [250, 450] K, P in [2, 15] MPa, z ~ Dirichlet(1)), and write
the checkpoint used by the learned form.

    python -m paper_2205_03090_gb300.train_nn [--n 1000000] [--epochs 100] [--patience 12]
        [--stage2-epochs 10] [--calib-n 500000] [--out PATH]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "weights", "nc10_2phase")
TRAIN_SEED = 101  # conditions drawn apart from the benchmark's (seed 4)
CALIB_SEED = 103  # held-out mixtures for the thresholds


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--epochs", type=int, default=100)
    ap.add_argument("--patience", type=int, default=12)
    ap.add_argument("--stage2-epochs", type=int, default=10)
    ap.add_argument("--calib-n", type=int, default=500_000)
    ap.add_argument("--out", default=DEFAULT_OUT)
    args = ap.parse_args(argv)
    import torch
    from . import build, nn, ptflash, workloads as wl
    build.build()
    w = wl.WORKLOADS["nc10_2phase_1e7"]
    comp = wl.pseudo_components(w["nc"], w["comp_seed"])
    cond = wl.conditions(w["nc"], args.n, TRAIN_SEED, w["T_range"], w["P_range"], w["alpha"])
    fl = ptflash.Flash(comp.Tc, comp.Pc, comp.omega, comp.kij, n_max=args.n)
    t0 = time.time()
    cfg = nn.TrainConfig(epochs=args.epochs, patience=args.patience, stage2_epochs=args.stage2_epochs)
    logs = nn.train_both(fl, cond, cfg, log_fn=print)
    dt = time.time() - t0
    cal = wl.conditions(w["nc"], args.calib_n, CALIB_SEED, w["T_range"], w["P_range"], w["alpha"])
    thr = nn.calibrate_thresholds(fl, cal, log_fn=print)
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    meta = {"workload": "nc10 pseudo-components, T 250-450 K, P 2-15 MPa, z ~ Dirichlet(1)",
            "train_samples": args.n, "train_seed": TRAIN_SEED, "seconds": dt,
            "classifier": {"best_epoch": logs[0].best_epoch, "test_bce": logs[0].test_loss,
                           "test_accuracy": logs[0].test_acc},
            "initializer": {"best_epoch": logs[1].best_epoch, "test_mae_lnK_sum": logs[1].test_loss,
                            "test_mae_lnK_per_component": logs[1].test_loss / w["nc"]},
            "thresholds": thr, "calib_seed": CALIB_SEED}
    if "stage2" in logs:
        s2 = logs["stage2"]
        meta["initializer"]["stage2"] = {"epochs_run": len(s2.epochs), "best_epoch": s2.best_epoch,
                                         "test_loss": s2.test_loss, "test_mae_theta": s2.test_acc,
                                         "test_mae_lnK_sum": s2.test_mae_lnK,
                                         "test_mae_lnK_per_component": s2.test_mae_lnK / w["nc"]}
    nn.save(fl, args.out, meta)
    print(json.dumps(meta))
    fl.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
