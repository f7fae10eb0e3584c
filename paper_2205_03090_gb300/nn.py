"""Learned form of the flash (Sec. 4): training and use of the stability
classifier and the ln K initializer through the C ABI.

Every forward, backward and Adam step runs in the CUDA library; this module
only builds datasets with the plain GPU flash, splits them 70/15/15
(Sec. 4.1.2), drives the triangular cyclic learning rate and early stopping
(Sec. 4.1.2: Adam, batch 512, CLR, early stopping) and stores checkpoints.
"""
from __future__ import annotations

import json
import os
import time
from dataclasses import dataclass, field

import numpy as np

from . import ptflash, workloads as wl

CLASSIFIER, INITIALIZER = 0, 1
HIDDEN = {CLASSIFIER: 64, INITIALIZER: 128}


@dataclass
class TrainConfig:
    epochs: int = 30
    batch: int = 512
    lr_min: float = 1e-4
    lr_max: float = 3e-3
    half_cycle_epochs: int = 2      # triangular CLR: steps per half cycle = this x steps per epoch
    patience: int = 6               # early stopping on the validation loss
    seed: int = 7


@dataclass
class TrainLog:
    epochs: list = field(default_factory=list)  # (epoch, train_loss, val_loss, val_acc, lr_end, seconds)
    best_epoch: int = -1
    test_loss: float = float("nan")
    test_acc: float = float("nan")


def clr(step: np.ndarray, half: int, lo: float, hi: float) -> np.ndarray:
    """Triangular cyclic learning rate (Smith 2017): linear lo -> hi -> lo
    over 2 * half steps."""
    c = np.abs((step / half) % 2.0 - 1.0)
    return (lo + (hi - lo) * (1.0 - c)).astype(np.float32)


def feature_stats(P, T, z):
    """Mean and standard deviation of the features (z_1..z_nc, P, T)."""
    v = np.concatenate([z, P[None, :], T[None, :]], axis=0)
    return v.mean(axis=1).astype(np.float32), np.maximum(v.std(axis=1), 1e-12).astype(np.float32)


def make_dataset(fl: ptflash.Flash, cond: wl.Conditions, device="cuda"):
    """Plain-method labels for the conditions (the plain GPU flash):
    stable flag (nphase == 1) and ln K of the two-phase mixtures."""
    import torch
    P = torch.tensor(cond.P, device=device)
    T = torch.tensor(cond.T, device=device)
    z = torch.tensor(cond.z, device=device).contiguous()
    out = fl.ptflash_flash(P, T, z)
    torch.cuda.synchronize()
    return P, T, z, out


def split_indices(n: int, seed: int):
    g = np.random.Generator(np.random.PCG64(seed))
    p = g.permutation(n)
    a, b = int(0.7 * n), int(0.85 * n)
    return p[:a], p[a:b], p[b:]


def train_network(fl: ptflash.Flash, which: int, X, Y, idx_train, idx_val, idx_test, cfg: TrainConfig,
                  log_fn=None) -> TrainLog:
    """Train one network in place (its parameters and scaler must be set).
    X [din, n], Y [dout, n] device float32 tensors over the whole dataset."""
    import torch
    dev = X.device
    Xtr, Ytr = X[:, idx_train].contiguous(), Y[:, idx_train].contiguous()
    Xva, Yva = X[:, idx_val].contiguous(), Y[:, idx_val].contiguous()
    Xte, Yte = X[:, idx_test].contiguous(), Y[:, idx_test].contiguous()
    ntr = Xtr.shape[1]
    steps = ntr // cfg.batch
    half = cfg.half_cycle_epochs * steps
    nparam = ptflash.load().ptflash_nn_param_count(X.shape[0], HIDDEN[which], Y.shape[0])
    best, best_val, bad = None, float("inf"), 0
    log = TrainLog()
    loss_dev = torch.zeros(steps, dtype=torch.float32, device=dev)
    for ep in range(cfg.epochs):
        t0 = time.time()
        perm = torch.tensor(wl.epoch_permutation(ntr, cfg.seed, ep)[: steps * cfg.batch], device=dev)
        lr = clr(np.arange(ep * steps, (ep + 1) * steps), half, cfg.lr_min, cfg.lr_max)
        loss_dev.zero_()
        fl.ptflash_nn_train_steps(which, Xtr, Ytr, perm, steps, cfg.batch, lr, loss=loss_dev)
        tl = float(loss_dev.mean().item())
        vl, va = fl.ptflash_nn_eval(which, Xva, Yva)
        log.epochs.append((ep, tl, vl, va, float(lr[-1]), time.time() - t0))
        if log_fn:
            log_fn(f"net {which} epoch {ep} train {tl:.5f} val {vl:.5f} acc {va:.5f} ({time.time() - t0:.1f}s)")
        if vl < best_val - 1e-7:
            best_val, bad, log.best_epoch = vl, 0, ep
            best = fl.ptflash_nn_get(which, nparam)
        else:
            bad += 1
            if bad >= cfg.patience:
                break
    mean, std = fl._nn_scaler[which]
    fl.ptflash_nn_set(which, HIDDEN[which], best, mean, std)
    log.test_loss, log.test_acc = fl.ptflash_nn_eval(which, Xte, Yte)
    return log


def train_both(fl: ptflash.Flash, cond: wl.Conditions, cfg: TrainConfig = TrainConfig(), log_fn=None):
    """Generate plain-method labels for `cond`, then train the classifier on
    all samples and the initializer on the two-phase ones (Sec. 4)."""
    import torch
    nc = fl.nc
    P, T, z, out = make_dataset(fl, cond)
    nphase = out.nphase
    mean, std = feature_stats(cond.P, cond.T, cond.z)
    fl._nn_scaler = {}
    logs = {}
    for which in (CLASSIFIER, INITIALIZER):
        dout = 1 if which == CLASSIFIER else nc
        theta = wl.mlp_init(nc + 2, HIDDEN[which], dout, cfg.seed + which)
        fl.ptflash_nn_set(which, HIDDEN[which], theta, mean, std)
        fl._nn_scaler[which] = (mean, std)
    X = torch.empty(nc + 2, cond.n, dtype=torch.float32, device=P.device)
    fl.ptflash_nn_features(CLASSIFIER, P, T, z, X)
    # classifier on every sample: y = 1 stable (single phase)
    Yc = (nphase == 1).to(torch.float32)[None, :].contiguous()
    tr, va, te = split_indices(cond.n, cfg.seed)
    logs[CLASSIFIER] = train_network(fl, CLASSIFIER, X, Yc, torch.tensor(tr, device=P.device),
                                     torch.tensor(va, device=P.device), torch.tensor(te, device=P.device), cfg,
                                     log_fn)
    # initializer on the two-phase samples: ln K targets
    two = torch.nonzero(nphase == 2).flatten()
    X2 = X[:, two].contiguous()
    Y2 = torch.log(out.K[:, two]).to(torch.float32).contiguous()
    tr, va, te = split_indices(int(two.shape[0]), cfg.seed + 1)
    logs[INITIALIZER] = train_network(fl, INITIALIZER, X2, Y2, torch.tensor(tr, device=P.device),
                                      torch.tensor(va, device=P.device), torch.tensor(te, device=P.device), cfg,
                                      log_fn)
    return logs


def save(fl: ptflash.Flash, path: str, meta: dict | None = None):
    """Checkpoint: one flat float32 file (classifier then initializer
    parameters, then both scalers) and a JSON header beside it."""
    nc = fl.nc
    parts, header = [], {"nc": nc, "nets": []}
    for which in (CLASSIFIER, INITIALIZER):
        dout = 1 if which == CLASSIFIER else nc
        cnt = ptflash.load().ptflash_nn_param_count(nc + 2, HIDDEN[which], dout)
        th = fl.ptflash_nn_get(which, cnt)
        mean, std = fl._nn_scaler[which]
        parts += [th, mean, std]
        header["nets"].append({"which": which, "hidden": HIDDEN[which], "dout": dout, "count": int(cnt)})
    header.update(meta or {})
    np.concatenate(parts).astype(np.float32).tofile(path + ".bin")
    with open(path + ".json", "w") as f:
        json.dump(header, f, indent=1)


def load_checkpoint(fl: ptflash.Flash, path: str):
    with open(path + ".json") as f:
        header = json.load(f)
    if header["nc"] != fl.nc:
        raise ValueError("checkpoint was trained for a different number of components")
    flat = np.fromfile(path + ".bin", dtype=np.float32)
    k, d = 0, fl.nc + 2
    fl._nn_scaler = {}
    for net in header["nets"]:
        th = flat[k:k + net["count"]]
        k += net["count"]
        mean, std = flat[k:k + d], flat[k + d:k + 2 * d]
        k += 2 * d
        fl.ptflash_nn_set(net["which"], net["hidden"], th, mean, std)
        fl._nn_scaler[net["which"]] = (mean, std)
    return header


def exists(path: str) -> bool:
    return os.path.exists(path + ".json") and os.path.exists(path + ".bin")
