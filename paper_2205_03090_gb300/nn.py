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
# (arch, hidden) per network.  DEFAULT_NETS: 3-hidden-layer networks of 64 and
# 128 units.  PAPER_NETS: the paper's classifier (3 x 32, Sec. 4.1.1) and
# initializer (a hidden layer, 3 residual blocks, wide output; 64 units,
# Sec. 4.2.1).
DEFAULT_NETS = {CLASSIFIER: (0, 64), INITIALIZER: (0, 128)}
PAPER_NETS = {CLASSIFIER: (0, 32), INITIALIZER: (1, 64)}


@dataclass
class TrainConfig:
    epochs: int = 30
    batch: int = 512
    lr_min: float = 1e-4
    lr_max: float = 3e-3
    half_cycle_epochs: int = 2      # triangular CLR: steps per half cycle = this x steps per epoch
    patience: int = 6               # early stopping on the validation loss
    seed: int = 7
    nets: dict = field(default_factory=lambda: dict(DEFAULT_NETS))
    stage2_epochs: int = 0          # initializer second stage: + |theta - theta_hat| (Sec. 4.2.2)
    stage2_lr: float = 1e-5
    stage2_weight: float = 1.0


@dataclass
class TrainLog:
    epochs: list = field(default_factory=list)  # (epoch, train_loss, val_loss, val_acc, lr_end, seconds)
    best_epoch: int = -1
    test_loss: float = float("nan")
    test_acc: float = float("nan")
    test_mae_lnK: float = float("nan")


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


def dout_of(fl, which):
    return 1 if which == CLASSIFIER else fl.nc


def train_network(fl: ptflash.Flash, which: int, X, Y, idx_train, idx_val, idx_test, cfg: TrainConfig,
                  log_fn=None, epochs=None, constant_lr=False) -> TrainLog:
    """Train one network in place (its parameters and scaler must be set).
    X [din, n], Y [rows, n] device float32 tensors over the whole dataset
    (rows: the loss's target rows).  CLR between lr_min and lr_max, or the
    constant stage2_lr with constant_lr."""
    import torch
    dev = X.device
    Xtr, Ytr = X[:, idx_train].contiguous(), Y[:, idx_train].contiguous()
    Xva, Yva = X[:, idx_val].contiguous(), Y[:, idx_val].contiguous()
    Xte, Yte = X[:, idx_test].contiguous(), Y[:, idx_test].contiguous()
    ntr = Xtr.shape[1]
    steps = ntr // cfg.batch
    half = cfg.half_cycle_epochs * steps
    arch, hid = cfg.nets[which]
    nparam = ptflash.load().ptflash_nn_param_count_arch(arch, X.shape[0], hid, dout_of(fl, which))
    best, best_val, bad = None, float("inf"), 0
    log = TrainLog()
    loss_dev = torch.zeros(steps, dtype=torch.float32, device=dev)
    for ep in range(cfg.epochs if epochs is None else epochs):
        t0 = time.time()
        perm = torch.tensor(wl.epoch_permutation(ntr, cfg.seed, ep)[: steps * cfg.batch], device=dev)
        lr = (np.full(steps, cfg.stage2_lr, np.float32) if constant_lr else
              clr(np.arange(ep * steps, (ep + 1) * steps), half, cfg.lr_min, cfg.lr_max))
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
    if best is not None:
        fl.ptflash_nn_set(which, hid, best, mean, std, arch=arch)
    log.test_loss, log.test_acc = fl.ptflash_nn_eval(which, Xte, Yte)
    return log


def train_both(fl: ptflash.Flash, cond: wl.Conditions, cfg: TrainConfig = TrainConfig(), log_fn=None):
    """Generate plain-method labels for `cond`, then train the classifier on
    all samples and the initializer on the two-phase ones (Sec. 4); with
    cfg.stage2_epochs, a second initializer stage adds the |theta -
    theta_hat| term at the constant rate stage2_lr (Sec. 4.2.2)."""
    import torch
    nc = fl.nc
    P, T, z, out = make_dataset(fl, cond)
    nphase = out.nphase
    mean, std = feature_stats(cond.P, cond.T, cond.z)
    fl._nn_scaler = {}
    fl._nn_arch = {}
    logs = {}
    for which in (CLASSIFIER, INITIALIZER):
        arch, hid = cfg.nets[which]
        theta = init_params(nc + 2, hid, dout_of(fl, which), cfg.seed + which, arch)
        fl.ptflash_nn_set(which, hid, theta, mean, std, arch=arch)
        fl._nn_scaler[which] = (mean, std)
        fl._nn_arch[which] = (arch, hid)
    fl.ptflash_nn_set_theta_loss(INITIALIZER, 0.0)
    X = torch.empty(nc + 2, cond.n, dtype=torch.float32, device=P.device)
    fl.ptflash_nn_features(CLASSIFIER, P, T, z, X)
    # classifier on every sample: y = 1 stable (single phase)
    Yc = (nphase == 1).to(torch.float32)[None, :].contiguous()
    tr, va, te = split_indices(cond.n, cfg.seed)
    dev = P.device
    logs[CLASSIFIER] = train_network(fl, CLASSIFIER, X, Yc, torch.tensor(tr, device=dev),
                                     torch.tensor(va, device=dev), torch.tensor(te, device=dev), cfg, log_fn)
    # initializer on the two-phase samples: ln K targets
    two = torch.nonzero(nphase == 2).flatten()
    X2 = X[:, two].contiguous()
    Y2 = torch.log(out.K[:, two]).to(torch.float32).contiguous()
    tr, va, te = split_indices(int(two.shape[0]), cfg.seed + 1)
    ti, vi, tei = (torch.tensor(a, device=dev) for a in (tr, va, te))
    logs[INITIALIZER] = train_network(fl, INITIALIZER, X2, Y2, ti, vi, tei, cfg, log_fn)
    if cfg.stage2_epochs > 0:
        # second stage: targets [ln K; theta; z], loss mae(ln K) + w mae(theta)
        Y3 = torch.cat([Y2, out.beta[two][None, :].to(torch.float32), z[:, two].to(torch.float32)], 0).contiguous()
        fl.ptflash_nn_set_theta_loss(INITIALIZER, cfg.stage2_weight)
        logs["stage2"] = train_network(fl, INITIALIZER, X2, Y3, ti, vi, tei, cfg, log_fn, epochs=cfg.stage2_epochs,
                                       constant_lr=True)
        # first-stage loss on the test set, for comparison
        fl.ptflash_nn_set_theta_loss(INITIALIZER, 0.0)
        logs["stage2"].test_mae_lnK = fl.ptflash_nn_eval(INITIALIZER, X2[:, tei].contiguous(), Y2[:, tei].contiguous())[0]
    return logs


def calibrate_thresholds(fl: ptflash.Flash, cond: wl.Conditions, margin_logit: float = 1.0, log_fn=None):
    """Thresholds p_l <= p_r of the learned form from held-out mixtures
    (Sec. 5.2 chooses them so that no misclassification occurs), with the
    plain GPU flash as the reference:

    * p_r: above the classifier probability of every mixture that the
      learned form with p_l = 0 and p_r = 1/2 reports stable (NN_STABLE, so
      its tpd trials did not catch it) while the plain flash finds two phases;
    * p_l: below the probability of every mixture that the learned form with
      p_l = 1/2 and p_r = 1 keeps from a network-started split (NN_UNSTABLE,
      accepted by the judge) while the plain flash disagrees (phase count, or
      beta, x or y by more than 1e-8).

    Each bound is widened by margin_logit in logit space and is at least as
    strict as the paper's 0.02 / 0.98.  Returns a dict with p_l, p_r and the
    fraction of the held-out mixtures the networks then decide."""
    import torch
    P = torch.tensor(cond.P, device="cuda")
    T = torch.tensor(cond.T, device="cuda")
    z = torch.tensor(cond.z, device="cuda").contiguous()
    plain = fl.ptflash_flash(P, T, z)
    logit = torch.empty(1, cond.n, dtype=torch.float32, device="cuda")
    fl.ptflash_nn_infer(CLASSIFIER, P, T, z, logit)
    hi = fl.ptflash_flash(P, T, z, use_nn=True, p_l=0.0, p_r=0.5)
    lo = fl.ptflash_flash(P, T, z, use_nn=True, p_l=0.5, p_r=1.0)
    torch.cuda.synchronize()
    lg = logit[0].double().cpu().numpy()
    pn = plain.nphase.cpu().numpy()
    bad_r = ((hi.status.cpu().numpy() & ptflash.PTF_ST_NN_STABLE) != 0) & (pn == 2)
    lst = lo.status.cpu().numpy()
    kept = ((lst & ptflash.PTF_ST_NN_UNSTABLE) != 0) & ((lst & ptflash.PTF_ST_NN_REJECTED) == 0)
    dv = torch.maximum((lo.beta - plain.beta).abs(),
                       torch.maximum((lo.x - plain.x).abs().amax(0), (lo.y - plain.y).abs().amax(0))).cpu().numpy()
    bad_l = kept & ((lo.nphase.cpu().numpy() != pn) | (dv > 1e-8))
    sig = lambda v: float(1.0 / (1.0 + np.exp(-v)))
    p_r = max(0.98, sig(lg[bad_r].max() + margin_logit)) if bad_r.any() else 0.98
    p_l = min(0.02, sig(lg[bad_l].min() - margin_logit)) if bad_l.any() else 0.02
    p = 1.0 / (1.0 + np.exp(-lg))
    decided = float(((p >= p_r) | (p <= p_l)).mean())
    res = {"p_l": p_l, "p_r": p_r, "held_out": int(cond.n), "margin_logit": margin_logit,
           "errors_above_half": int(bad_r.sum()), "errors_below_half": int(bad_l.sum()),
           "decided_frac": decided, "rejected_frac_below_half": float(((lst & ptflash.PTF_ST_NN_REJECTED) != 0).mean())}
    if log_fn:
        log_fn(f"calibration: {res}")
    return res


def init_params(din, hid, dout, seed, arch=0):
    """Seeded Glorot-uniform weights and zero biases for either architecture."""
    return wl.mlp_init(din, hid, dout, seed, arch)


def save(fl: ptflash.Flash, path: str, meta: dict | None = None):
    """Checkpoint: one flat float32 file (classifier then initializer
    parameters, then both scalers) and a JSON header beside it."""
    nc = fl.nc
    parts, header = [], {"nc": nc, "nets": []}
    arch_of = getattr(fl, "_nn_arch", {w: DEFAULT_NETS[w] for w in (CLASSIFIER, INITIALIZER)})
    for which in (CLASSIFIER, INITIALIZER):
        arch, hid = arch_of[which]
        dout = dout_of(fl, which)
        cnt = ptflash.load().ptflash_nn_param_count_arch(arch, nc + 2, hid, dout)
        th = fl.ptflash_nn_get(which, cnt)
        mean, std = fl._nn_scaler[which]
        parts += [th, mean, std]
        header["nets"].append({"which": which, "arch": arch, "hidden": hid, "dout": dout, "count": int(cnt)})
    header.update(meta or {})
    np.concatenate(parts).astype(np.float32).tofile(path + ".bin")
    with open(path + ".json", "w") as f:
        json.dump(header, f, indent=1)


def thresholds(header: dict):
    """The learned form's (p_l, p_r) stored with a checkpoint, else the
    paper's 0.02 / 0.98."""
    t = header.get("thresholds") or {}
    return float(t.get("p_l", 0.02)), float(t.get("p_r", 0.98))


def load_checkpoint(fl: ptflash.Flash, path: str):
    with open(path + ".json") as f:
        header = json.load(f)
    if header["nc"] != fl.nc:
        raise ValueError("checkpoint was trained for a different number of components")
    flat = np.fromfile(path + ".bin", dtype=np.float32)
    k, d = 0, fl.nc + 2
    fl._nn_scaler = {}
    fl._nn_arch = {}
    for net in header["nets"]:
        th = flat[k:k + net["count"]]
        k += net["count"]
        mean, std = flat[k:k + d], flat[k + d:k + 2 * d]
        k += 2 * d
        arch = net.get("arch", 0)
        fl.ptflash_nn_set(net["which"], net["hidden"], th, mean, std, arch=arch)
        fl._nn_scaler[net["which"]] = (mean, std)
        fl._nn_arch[net["which"]] = (arch, net["hidden"])
    return header


def exists(path: str) -> bool:
    return os.path.exists(path + ".json") and os.path.exists(path + ".bin")
