#!/usr/bin/env python
"""Benchmark of the batched isothermal two-phase flash on GB300.

Metric: oracle-matching flashes per second on the 8-pseudo-component,
1e6-mixture workload (z ~ Dirichlet(0.5)), FP64, inputs resident in HBM.
A "step" is one ptflash_flash call over the whole batch (all stages: prep
and precheck, stability SS / trust region, decision, split SS / trust
region).  value = mixtures x (fraction matching the CPU oracle on a sampled
subset) / step time, summed over ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank flashes its own 1e6 mixtures (weak
scaling, no collective on the data path); the step time is the max over
ranks.  --impl reference times the CPU oracle (the method as plain C on the
host cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "flashes/sec on 1 GB300 (n_c=8, 1e6 mixtures, |Δβ|≤1e-8), plain vs batched+learned"
WORKLOAD = "nc8_1e6"
WORKLOAD_DESC = ("8 SRK pseudo-components (Tc~U(150,650) K sorted, Pc~U(2,5) MPa, omega~U(0,0.5), "
                 "k_ij~U(0,0.1)), 1e6 mixtures, T~U(200,600) K, P~U(0.1,20) MPa, z~Dirichlet(0.5)")
SMS = 152
FP64_FMA_PER_CLK_PER_SM = 2  # GB300 FP64 units (recipe: 1.25 TFLOP/s at 2.07 GHz)
OP_KINDS = ("div", "sqrt", "exp", "log")  # counted apart from the plain flops by the oracle
TOL = 1e-8
LIB_STAGES = ("prep_precheck", "stab_ss", "stab_tr", "stab_decide", "split_ss", "split_tr")
ORACLE_STAGE = {"prep_precheck": 0, "stab_ss": 1, "stab_tr": 2, "split_ss": 3, "split_tr": 4}
KERNELS_PER_STEP = 14  # prep, 2 precheck, 2 stability SS, stability TR, decide, 4 split SS (two parts, FP32 + FP64),
                       # queue order, split TR, counter fold
LEARNED_WORKLOAD = "nc10_2phase_1e7"
LEARNED_DESC = ("10 SRK pseudo-components drawn as above, 1e7 mixtures, T~U(250,450) K, P~U(2,15) MPa, "
                "z~Dirichlet(1); classifier 3x64 SiLU and ln K initializer 3x128 SiLU (BF16/FP32), "
                "p_l=0.02, p_r=0.98")


# DRAM bytes per unit of work of a kernel, from one ncu capture of
# dram__bytes_read.sum + dram__bytes_write.sum (profiles/ncu_split_tr_nc8_3e5.md:
# k_split_tr on 3e5 mixtures, 70,791 split trust-region mixtures, 857.7 MB);
# the bench scales it by this run's units.  Only valid for the kernel as
# captured: set to {} when the kernel changes until it is captured again.
TRAFFIC_PER_UNIT = {"split_tr": (857.706e6 / 70791, "split trust-region mixtures", lambda q: q["split_tr"])}


def measured_hbm_gbs():
    """The measured HBM copy bandwidth of this machine's GPUs (MEASURED_PEAKS.json),
    else the recipe's 6.8 TB/s fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def rank_conditions(w: dict, n: int, rank: int):
    """This rank's shard of the workload: the same distribution, its own seed
    (weak scaling: every rank flashes n mixtures of its own)."""
    from paper_2205_03090_gb300 import workloads as wl
    return wl.conditions(w["nc"], n, w["cond_seed"] + 1000 * rank, w["T_range"], w["P_range"], w["alpha"])


def job_ms(ms: float, dist, device) -> float:
    """The job's time per step: the maximum over ranks (every rank's value
    when there is one rank)."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(n_per_rank: int, ws: int, frac: float, ms: float) -> float:
    """Whole-job throughput: oracle-matching flashes of all ranks per second
    (NaN without an oracle-matching fraction: a diagnostic run)."""
    return ws * n_per_rank * frac / (ms / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


UNEVEN_DESC = ("uneven batch: 64 fluid systems, nc ~ U{3..16} each with its own pseudo-components (drawn as above), "
               "62,500 mixtures each (4e6), T~U(200,600) K, P~U(0.1,20) MPa, z~Dirichlet(1); one CUDA graph launch, "
               "persistent-kernel grids tuned per nc")


def uneven_leg(args, rank, dev, flush, stream):
    """The uneven batch through ptflash_batch_flash: tuned once (untimed),
    then one graph launch per step; checked against the oracle on a sample of
    every system."""
    import torch
    from paper_2205_03090_gb300 import ptflash, workloads as wl
    systems = wl.uneven_systems(seed=2 + 1000 * rank)
    b = ptflash.Batch([(c.Tc, c.Pc, c.omega, c.kij) for c, _ in systems], [cd.n for _, cd in systems])
    P, T, z = b.pack([(cd.P, cd.T, cd.z) for _, cd in systems], device=dev)
    out = b.alloc_outputs(dev)
    t0 = time.perf_counter()
    bps, group_ms = b.ptflash_batch_tune(P, T, z, out)
    tune_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        b.ptflash_batch_flash(P, T, z, out=out, stream=stream)
    ms = []
    for _ in range(max(1, args.steps)):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        b.ptflash_batch_flash(P, T, z, out=out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    info = b.ptflash_batch_info()
    frac, sample = float("nan"), 0
    if rank == 0 and args.cpu_sample > 0:
        rng = np.random.default_rng(17)
        ok = []
        for k, (comp, cond) in enumerate(systems):
            g = b.unpack(out, k)
            idx = np.sort(rng.choice(cond.n, 32, replace=False))
            o, _, s = run_oracle_sample(comp, cond, idx)
            ok.append(match_fraction(s, comp, cond, idx, o, g) * len(idx))
            sample += len(idx)
        frac = float(np.sum(ok) / sample)
    b.close()
    t = float(np.mean(ms))
    return {"workload": UNEVEN_DESC, "n": info["mixtures"], "ms_per_step": t,
            "value": info["mixtures"] * (frac if frac == frac else 1.0) / (t / 1e3), "unit": "flashes/s",
            "oracle_match": {"frac": frac, "sample": sample, "tol": TOL},
            "graph": {"groups": info["groups"], "nodes": info["graph_nodes"], "launches_per_step": 1},
            "tuned_blocks_per_sm": {str(k): v for k, v in bps.items()},
            "tuned_group_ms_alone": {str(k): round(v, 3) for k, v in group_ms.items()},
            "tune_seconds": round(tune_s, 2)}


ADJOINT_DESC = ("differentiation: 10 SRK pseudo-components drawn as above, 1e6 mixtures, T~U(250,450) K, "
                "P~U(2,15) MPa, z~Dirichlet(1); FP64 flash + implicit-function-theorem adjoint of (beta, x, y) "
                "w.r.t. (P, T, z) for a random output functional")


def adjoint_leg(args, rank, dev, flush, stream):
    """Forward flash plus one adjoint launch on the 10-component workload;
    the vector-Jacobian products checked against the oracle's forward
    Jacobian on a sample."""
    import torch
    from paper_2205_03090_gb300 import ptflash, workloads as wl
    w = wl.WORKLOADS["nc10_2phase_1e6"]
    comp = wl.pseudo_components(w["nc"], w["comp_seed"])
    n = w["n"]
    cond = wl.conditions(w["nc"], n, w["cond_seed"] + 1000 * rank, w["T_range"], w["P_range"], w["alpha"])
    fl = ptflash.Flash(comp.Tc, comp.Pc, comp.omega, comp.kij, n_max=n)
    P = torch.tensor(cond.P, device=dev)
    T = torch.tensor(cond.T, device=dev)
    z = torch.tensor(cond.z, device=dev).contiguous()
    rng = np.random.default_rng(23)
    wb, wx, wy = (torch.tensor(a, device=dev) for a in (rng.normal(size=n), rng.normal(size=(w["nc"], n)),
                                                        rng.normal(size=(w["nc"], n))))
    res = fl.alloc_outputs(n, dev)
    fwd_ms, adj_ms = [], []
    for it in range(args.warmup + max(1, args.steps)):
        flush.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        e[0].record(stream)
        fl.ptflash_flash(P, T, z, out=res, stream=stream)
        e[1].record(stream)
        gP, gT, gz, ast = fl.ptflash_flash_adjoint(P, T, z, res, wb, wx, wy, stream=stream)
        e[2].record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            fwd_ms.append(e[0].elapsed_time(e[1]))
            adj_ms.append(e[1].elapsed_time(e[2]))
    frac, sample = float("nan"), 0
    if rank == 0 and args.cpu_sample > 0:
        import oracle
        sample = 2000
        idx = np.sort(rng.choice(n, sample, replace=False))
        s = oracle.System(comp.Tc, comp.Pc, comp.omega, comp.kij)
        g = {k: getattr(res, k).cpu().numpy()[..., idx] for k in ("nphase", "beta", "x", "y")}
        Jo, ok = oracle.flash_jacobian(s, cond.P[idx], cond.T[idx], np.ascontiguousarray(cond.z[:, idx]), g)
        wv = np.concatenate([wb.cpu().numpy()[None], wx.cpu().numpy(), wy.cpu().numpy()], 0)[:, idx].T
        vjp = np.einsum("nr,nrc->nc", wv, Jo)
        got = np.concatenate([gP.cpu().numpy()[idx, None], gT.cpu().numpy()[idx, None],
                              gz.cpu().numpy()[:, idx].T], 1)
        scale = np.maximum(np.einsum("nr,nrc->nc", np.abs(wv), np.abs(Jo)), 1e-300)
        err = (np.abs(got - vjp) / scale).max(axis=1)
        frac = float(((err <= 1e-8) & (ok == 0)).mean())
    counts = np.bincount(ast.cpu().numpy(), minlength=3)
    fl.close()
    f, a = float(np.mean(fwd_ms)), float(np.mean(adj_ms))
    return {"workload": ADJOINT_DESC, "n": n, "forward_ms": f, "adjoint_ms": a,
            "value": n / ((f + a) / 1e3), "unit": "flashes with gradient/s",
            "adjoint_only_value": n / (a / 1e3),
            "oracle_match": {"frac": frac, "sample": sample, "tol": "1e-8 relative to |w|.|J| per input"},
            "astatus": {"two_phase": int(counts[0]), "single_phase": int(counts[1]), "singular": int(counts[2])}}


# Paper Table 4 (9 components, 1e6 mixtures, RTX 3080): per-stage counts; context only.
PAPER_TABLE4 = {"precheck_unstable_frac": 0.3744, "stab": 625645, "stab_tr_vapour": 130715, "stab_tr_liquid": 90179,
                "split": 413442, "split_ss_converged_frac": 0.4588, "split_tr": 223741, "max_stab_tr_iters": 18,
                "max_split_tr_iters": 13, "total_s": 3.0346}
CASES = (("c2", 10_000_000), ("c4", 5_000_000), ("c9", 1_000_000))  # the paper's largest n per case (Sec. 5.1)


def cases_leg(args, rank, dev, flush, stream):
    """The paper's three case studies (Sec. 2.3) at the paper's largest batch
    sizes: flashes/s, stage counts (Table 4's rows for the 9-component
    fluid) and a sampled oracle check."""
    import torch
    from paper_2205_03090_gb300 import ptflash, workloads as wl
    out_all = {}
    for case, n in CASES:
        n = max(1, int(n * args.cases_scale))
        comp, cond, ft = wl.paper_case(case, n, 100 + rank)
        fl = ptflash.Flash(comp.Tc, comp.Pc, comp.omega, comp.kij, n_max=n)
        P = torch.tensor(cond.P, device=dev)
        T = torch.tensor(cond.T, device=dev)
        z = torch.tensor(cond.z, device=dev).contiguous()
        out = fl.alloc_outputs(n, dev)
        ms = []
        for it in range(args.warmup + max(1, args.steps)):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            fl.ptflash_flash(P, T, z, out=out, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if it >= args.warmup:
                ms.append(e0.elapsed_time(e1))
        q = fl.ptflash_last_counts()
        g = {k: getattr(out, k).cpu().numpy() for k in ("nphase", "beta", "x", "y", "status", "iters")}
        st, it = g["status"], g["iters"]
        stats = {"precheck_unstable_frac": float((st & 1).mean()), "stab": q["stab"], "stab_tr_items": q["stab_tr"],
                 "split": q["split"], "split_ss_converged_frac": 1.0 - q["split_tr"] / max(1, q["split"]),
                 "split_tr": q["split_tr"], "max_stab_tr_iters": int(((it >> 24) & 0xff).max()),
                 "max_split_tr_iters": int(((it >> 8) & 0xff).max()), "two_phase_frac": float((g["nphase"] == 2).mean()),
                 "maxiter": int(((st & 16) != 0).sum())}
        frac, sample = float("nan"), 0
        if rank == 0 and args.cpu_sample > 0:
            rng = np.random.default_rng(29)
            sample = min(n, 5000)
            idx = np.sort(rng.choice(n, sample, replace=False))
            o, _, s = run_oracle_sample(comp, cond, idx)
            frac = match_fraction(s, comp, cond, idx, o, g)
        fl.close()
        t = float(np.mean(ms))
        out_all[case] = {"components": list(wl.PAPER_CASES[case]["names"]), "n": n, "ms_per_step": t,
                         "value": n * (frac if frac == frac else 1.0) / (t / 1e3), "unit": "flashes/s",
                         "oracle_match": {"frac": frac, "sample": sample, "tol": TOL}, "stages": stats}
    out_all["paper_table4_context"] = PAPER_TABLE4
    return out_all


# Paper Table 5 (NN-PTFlash, 9 components, 1e6 mixtures, RTX 3080); context only.
PAPER_TABLE5 = {"classifier_decided_frac": 0.9942, "stab": 5818, "split": 413442, "split_ss_converged_frac": 0.674,
                "split_tr": 134786, "speedup_vs_plain_gpu": 2.2}


def paper_learned_leg(args, rank, dev, flush, stream):
    """The paper's networks (classifier 3 x 32, residual + wide initializer)
    on the 9-component case study: plain vs learned form on the same 1e6
    mixtures, stage counts beside Table 5, sampled oracle check.  Trains the
    networks first if the checkpoint is missing."""
    import torch
    from paper_2205_03090_gb300 import nn, ptflash, workloads as wl
    from paper_2205_03090_gb300 import train_paper_nn
    if not nn.exists(train_paper_nn.DEFAULT_OUT):
        train_paper_nn.main([])
    n = max(1, int(1_000_000 * args.cases_scale))
    comp, cond, ft = wl.paper_case("c9", n, 300 + rank)
    fl = ptflash.Flash(comp.Tc, comp.Pc, comp.omega, comp.kij, n_max=n)
    meta = nn.load_checkpoint(fl, train_paper_nn.DEFAULT_OUT)
    p_l, p_r = nn.thresholds(meta)
    P = torch.tensor(cond.P, device=dev)
    T = torch.tensor(cond.T, device=dev)
    z = torch.tensor(cond.z, device=dev).contiguous()
    out = fl.alloc_outputs(n, dev)
    res = {}
    for form in ("plain", "learned"):
        use = form == "learned"
        ms = []
        for it in range(args.warmup + max(1, args.steps)):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            fl.ptflash_flash(P, T, z, out=out, use_nn=use, p_l=p_l, p_r=p_r, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if it >= args.warmup:
                ms.append(e0.elapsed_time(e1))
        q = fl.ptflash_last_counts()
        st = out.status.cpu().numpy()
        res[form] = {"ms_per_step": float(np.mean(ms)), "queues": q,
                     "split_ss_converged_frac": 1.0 - q["split_tr"] / max(1, q["split"])}
        if use:
            res[form]["classifier_decided_frac"] = float(((st & (128 | 256)) != 0).mean())
            res[form]["rejected_frac"] = float(((st & 1024) != 0).mean())
            g = {k: getattr(out, k).cpu().numpy() for k in ("nphase", "beta", "x", "y", "status")}
    frac, sample = float("nan"), 0
    if rank == 0 and args.cpu_sample > 0:
        rng = np.random.default_rng(31)
        sample = min(n, 20000)
        idx = np.sort(rng.choice(n, sample, replace=False))
        o, _, s = run_oracle_sample(comp, cond, idx)
        frac = match_fraction(s, comp, cond, idx, o, g)
    fl.close()
    lv = n * (frac if frac == frac else 1.0) / (res["learned"]["ms_per_step"] / 1e3)
    return {"workload": "paper case study, 9 components, four fluid types, 1e6 mixtures", "n": n,
            "value": lv, "unit": "flashes/s", "ms_per_step": res["learned"]["ms_per_step"],
            "plain_ms_per_step": res["plain"]["ms_per_step"],
            "speedup_vs_plain": res["plain"]["ms_per_step"] / res["learned"]["ms_per_step"],
            "oracle_match": {"frac": frac, "sample": sample, "tol": TOL}, "plain": res["plain"],
            "learned": res["learned"], "networks": {k: meta.get(k) for k in ("classifier", "initializer")},
            "thresholds": {"p_l": p_l, "p_r": p_r},
            "paper_table5_context": PAPER_TABLE5}


def run_oracle_sample(comp, cond, idx, nthreads=None):
    import oracle
    s = oracle.System(comp.Tc, comp.Pc, comp.omega, comp.kij)
    P, T, z = cond.P[idx], cond.T[idx], np.ascontiguousarray(cond.z[:, idx])
    t0 = time.perf_counter()
    o = oracle.flash(s, P, T, z, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return o, dt, s


def match_fraction(s, comp, cond, idx, o, g, misses=None):
    """Fraction of sampled flashes matching the oracle (label exact where the
    oracle's fully converged |min tpd| > 1e-8; beta, x, y within 1e-8 where
    both are two-phase).  misses (a list), if given, receives up to 20
    records of the mismatches: index, both statuses, phase counts, |dbeta|."""
    import oracle
    gn, gb = g["nphase"][idx], g["beta"][idx]
    gx, gy = g["x"][:, idx], g["y"][:, idx]
    ok = np.ones(len(idx), bool)
    both = (gn == 2) & (o["nphase"] == 2)
    ok &= ~(both & ((np.abs(gb - o["beta"]) > TOL) | (np.abs(gx - o["x"]).max(0) > TOL) |
                    (np.abs(gy - o["y"]).max(0) > TOL)))
    diff = np.nonzero(gn != o["nphase"])[0]
    if len(diff):
        tp = oracle.tpd_min(s, cond.P[idx][diff], cond.T[idx][diff], np.ascontiguousarray(cond.z[:, idx][:, diff]))
        ok[diff[np.abs(tp) > 1e-8]] = False
    if misses is not None:
        for k in np.nonzero(~ok)[0][:20]:
            misses.append({"mixture": int(idx[k]), "status": int(g["status"][idx[k]]), "status_oracle": int(o["status"][k]),
                           "nphase": int(gn[k]), "nphase_oracle": int(o["nphase"][k]),
                           "dbeta": float(abs(gb[k] - o["beta"][k]))})
    return float(ok.mean())


def reference_arm(args, ws, rank):
    """CPU oracle on the host cores, a bounded sample per step."""
    if rank != 0:
        return 0
    import oracle
    from paper_2205_03090_gb300 import workloads as wl
    oracle.build()
    comp, cond = wl.workload(WORKLOAD)
    cores = oracle.default_threads()
    sample = args.ref_sample
    rng = np.random.default_rng(7)
    for _ in range(args.warmup):
        run_oracle_sample(comp, cond, np.sort(rng.choice(cond.n, min(2000, sample), replace=False)))
    times = []
    for k in range(args.steps):
        idx = np.sort(rng.choice(cond.n, sample, replace=False))
        _, dt, _ = run_oracle_sample(comp, cond, idx)
        times.append(dt)
    ms = 1e3 * float(np.mean(times))
    value = sample / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "flashes/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "n": int(cond.n), "nc": int(comp.nc),
                       "step": f"{sample} sampled mixtures on the host cores"},
            "cpu_baseline": {"value": value, "unit": "flashes/s", "cores": cores, "kind": "oracle",
                             "sample": f"{sample} random mixtures of the 1e6-mixture workload per step"},
            "e2e": {"value": value, "unit": "flashes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def ours_arm(args, ws, rank, local):
    import torch
    from paper_2205_03090_gb300 import build, ptflash, workloads as wl
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    build.build()
    w = dict(wl.WORKLOADS[WORKLOAD])
    comp = wl.pseudo_components(w["nc"], w["comp_seed"])
    n_mix = args.n or w["n"]
    cond = rank_conditions(w, n_mix, rank)
    n, nc = cond.n, comp.nc
    fl = ptflash.Flash(comp.Tc, comp.Pc, comp.omega, comp.kij, n_max=n)
    P = torch.tensor(cond.P, device=dev)
    T = torch.tensor(cond.T, device=dev)
    z = torch.tensor(cond.z, device=dev).contiguous()
    out = fl.alloc_outputs(n, dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream()

    def step():
        fl.ptflash_flash(P, T, z, out=out, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # FP64 FMA probe of this GPU right after the timed steps (same clock record)
    probe_tf, probe_ms = ptflash.fp64_fma_rate(6000)
    clk = clocks.stop()
    # Stage times: further steps with the library's per-stage events, which
    # run the stages one after another (in the timed steps the split SS of the
    # precheck-routed mixtures overlaps the stability stages).
    fl.ptflash_set_profiling(True)
    stage_ms = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        step()
        stage_ms.append(fl.ptflash_last_stage_ms())
    fl.ptflash_set_profiling(False)
    ms = job_ms(float(np.mean(step_ms)), dist, dev)
    counts = fl.ptflash_last_counts()
    g = {k: getattr(out, k).cpu().numpy() for k in ("nphase", "beta", "x", "y", "status")}

    # end to end through the host-buffer entry point (H2D + flash + D2H each step)
    Ph, Th, zh = (torch.tensor(a).pin_memory() for a in (cond.P, cond.T, cond.z))
    hout = ptflash.FlashResult(torch.empty(n, dtype=torch.int32).pin_memory(),
                               torch.empty(n, dtype=torch.float64).pin_memory(),
                               *(torch.empty(nc, n, dtype=torch.float64).pin_memory() for _ in range(3)),
                               torch.empty(n, dtype=torch.int32).pin_memory(),
                               torch.empty(n, dtype=torch.int32).pin_memory())
    fl.ptflash_flash_host(Ph, Th, zh, out=hout, stream=stream)
    e2e = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fl.ptflash_flash_host(Ph, Th, zh, out=hout, stream=stream)
        e2e.append(time.perf_counter() - t0)
    e2e_s = float(np.mean(e2e))
    if dist:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    h2d = n * (2 + nc) * 8
    d2h = n * (4 + 8 + 3 * nc * 8 + 4 + 4)

    learned = learned_leg(args, rank, dev, flush, stream) if args.learned_n > 0 else None
    uneven = uneven_leg(args, rank, dev, flush, stream) if args.uneven else None
    adjoint = adjoint_leg(args, rank, dev, flush, stream) if args.adjoint else None
    cases = cases_leg(args, rank, dev, flush, stream) if args.cases else None
    paper_learned = paper_learned_leg(args, rank, dev, flush, stream) if args.paper_nn else None

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    # CPU baseline (the oracle as it stands) on a bounded sample, which also
    # gives the oracle-matching fraction and the algorithmic FP64 work
    # (--cpu-sample 0 skips it: diagnostic runs only, no valid value)
    sample = min(n, args.cpu_sample)
    if sample > 0:
        rng = np.random.default_rng(11)
        idx = np.sort(rng.choice(n, sample, replace=False))
        o, cpu_dt, s = run_oracle_sample(comp, cond, idx)
        import oracle as _or
        cores = _or.default_threads()
        misses = []
        frac = match_fraction(s, comp, cond, idx, o, g, misses)
        ops_per_flash = o["ops"] / sample  # [oracle stage, kind]
    else:
        cpu_dt, cores, frac, ops_per_flash, misses = float("nan"), 0, float("nan"), np.full((5, 5), np.nan), []

    mean_stage = {k: float(np.mean([d[k] for d in stage_ms])) for k in LIB_STAGES}
    dom = max(mean_stage, key=mean_stage.get)
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
    peak = SMS * FP64_FMA_PER_CLK_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    if dom in ORACLE_STAGE:
        q = ORACLE_STAGE[dom]
        work = float(ops_per_flash[q, 0] * n)  # plain FP64 flops: add, multiply 1, FMA 2
        special = {k: float(ops_per_flash[q, 1 + j] * n) for j, k in enumerate(OP_KINDS)}
        achieved = work / (mean_stage[dom] / 1e3) / 1e12
    else:
        work, special, achieved = None, None, None
    step_ops = {k: float(ops_per_flash[:, j].sum() * n) for j, k in enumerate(("flops",) + OP_KINDS)}
    hbm_peak = measured_hbm_gbs()
    traffic, traffic_src = None, None
    if dom in TRAFFIC_PER_UNIT:
        per, unit, count = TRAFFIC_PER_UNIT[dom]
        traffic = per * count(counts)
        traffic_src = (f"ncu dram bytes of k_{dom} on a 3e5-mixture case, {per:.0f} B per {unit[:-1]}, "
                       f"x {count(counts)} {unit} of this launch")
    value = job_value(n, ws, frac, ms)
    line = {
        "metric": METRIC, "value": value, "unit": "flashes/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "n": n, "nc": nc, "form": "plain", "parallelism": f"replicas{ws}",
                   "l2": "flushed between steps (512 MB write); inputs resident in HBM"},
        "oracle_match": {"frac": frac, "sample": sample, "tol": TOL, "misses": misses},
        "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "traffic_source": traffic_src,
                     "peak_source": f"152 SMs x 2 FP64 FMA/clk x 2 flop x {sm_mhz:.0f} MHz (sampled median), "
                                    f"the unit-count peak (MEASURED_PEAKS.json has no FP64 figure); the FP64 FMA "
                                    f"probe (ptflash_fp64_fma_rate, profiles/fp64_fma_probe.md) measured "
                                    f"{probe_tf:.3f} TFLOP/s on this GPU after the timed steps: frac_of_probe",
                     "peak_probe": probe_tf, "frac_of_probe": (achieved / probe_tf) if achieved else None,
                     "fp64_ops": work, "transcendental_ops": special,
                     "ops_note": "oracle-counted algorithmic work of the dominant stage per launch: fp64_ops are "
                                 "plain flops (add, multiply 1, FMA 2); divisions, square roots, exponentials and "
                                 "logarithms are counted apart (each costs many FP64 pipe slots on the GPU)",
                     "step_ops": step_ops,
                     "hbm_algorithmic_bytes_per_step": h2d + d2h,
                     "hbm_achieved_gbs": (h2d + d2h) / (ms / 1e3) / 1e9,
                     "hbm_peak_gbs": hbm_peak,
                     "hbm_frac": ((h2d + d2h) / (ms / 1e3) / 1e9 / hbm_peak) if hbm_peak else None},
        "stage_ms": mean_stage,
        "stage_ms_note": "separate steps after the timed ones, stages one after another with per-stage CUDA events; "
                         "the timed steps overlap the precheck-routed split SS with the stability stages",
        "queues": counts,
        "cpu_baseline": {"value": sample / cpu_dt, "unit": "flashes/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sample} random mixtures of the workload, {cpu_dt:.1f} s on {cores} threads"},
        "e2e": {"value": ws * n * frac / e2e_s, "unit": "flashes/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": KERNELS_PER_STEP * args.steps,
        "clocks": clk,
        "learned": learned,
        "uneven": uneven,
        "adjoint": adjoint,
        "paper_cases": cases,
        "paper_learned": paper_learned,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def learned_leg(args, rank, dev, flush, stream):
    """Plain vs learned form (Sec. 4) on the 10-component workload: the same
    inputs timed through both, the learned result checked against the
    oracle on a sample.  Uses the committed checkpoint, training one first if
    there is none."""
    import torch
    from paper_2205_03090_gb300 import nn, ptflash, workloads as wl
    from paper_2205_03090_gb300 import train_nn
    w = dict(wl.WORKLOADS[LEARNED_WORKLOAD])
    comp = wl.pseudo_components(w["nc"], w["comp_seed"])
    n = args.learned_n
    cond = wl.conditions(w["nc"], n, w["cond_seed"] + 1000 * rank, w["T_range"], w["P_range"], w["alpha"])
    if not nn.exists(train_nn.DEFAULT_OUT):
        train_nn.main([])
    fl = ptflash.Flash(comp.Tc, comp.Pc, comp.omega, comp.kij, n_max=n)
    meta = nn.load_checkpoint(fl, train_nn.DEFAULT_OUT)
    p_l, p_r = nn.thresholds(meta)
    P = torch.tensor(cond.P, device=dev)
    T = torch.tensor(cond.T, device=dev)
    z = torch.tensor(cond.z, device=dev).contiguous()
    out = fl.alloc_outputs(n, dev)
    res = {}
    for form in ("plain", "learned"):
        use = form == "learned"
        for _ in range(max(1, args.warmup - 1)):
            fl.ptflash_flash(P, T, z, out=out, use_nn=use, p_l=p_l, p_r=p_r, stream=stream)
        ms = []
        for _ in range(max(1, args.steps)):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            fl.ptflash_flash(P, T, z, out=out, use_nn=use, p_l=p_l, p_r=p_r, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        res[form] = {"ms_per_step": float(np.mean(ms)), "queues": fl.ptflash_last_counts()}
        if use:
            g = {k: getattr(out, k).cpu().numpy() for k in ("nphase", "beta", "x", "y", "status")}
            st = g["status"]
            res[form]["routes"] = {"nn_stable": float(((st & 128) != 0).mean()),
                                   "nn_unstable": float(((st & 256) != 0).mean()),
                                   "rejected": float(((st & 1024) != 0).mean())}
    frac, sample, misses = float("nan"), 0, []
    if rank == 0 and args.cpu_sample > 0:
        rng = np.random.default_rng(13)
        sample = min(n, max(40_000, args.cpu_sample // 5))
        idx = np.sort(rng.choice(n, sample, replace=False))
        o, _, s = run_oracle_sample(comp, cond, idx)
        frac = match_fraction(s, comp, cond, idx, o, g, misses)
    fl.close()
    learned_v = n * (frac if frac == frac else 1.0) / (res["learned"]["ms_per_step"] / 1e3)
    return {"workload": LEARNED_DESC, "n": n, "ms_per_step": res["learned"]["ms_per_step"],
            "value": learned_v, "unit": "flashes/s",
            "plain_ms_per_step": res["plain"]["ms_per_step"],
            "plain_value": n / (res["plain"]["ms_per_step"] / 1e3),
            "speedup_vs_plain": res["plain"]["ms_per_step"] / res["learned"]["ms_per_step"],
            "oracle_match": {"frac": frac, "sample": sample, "tol": TOL, "misses": misses},
            "queues_plain": res["plain"]["queues"], "queues_learned": res["learned"]["queues"],
            "routes": res["learned"]["routes"], "thresholds": {"p_l": p_l, "p_r": p_r},
            "networks": {k: meta.get(k) for k in ("classifier", "initializer", "train_samples")}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-sample", type=int, default=200_000)
    ap.add_argument("--ref-sample", type=int, default=20_000)
    ap.add_argument("--n", type=int, default=0, help="mixtures per rank (default: the workload's 1e6)")
    ap.add_argument("--learned-n", type=int, default=10_000_000,
                    help="mixtures of the learned-form leg (0 skips it)")
    ap.add_argument("--uneven", type=int, default=1, help="run the uneven-batch leg (0 skips it)")
    ap.add_argument("--adjoint", type=int, default=1, help="run the flash + adjoint leg (0 skips it)")
    ap.add_argument("--cases", type=int, default=1, help="run the paper case-study leg (0 skips it)")
    ap.add_argument("--cases-scale", type=float, default=1.0, help="fraction of the case-study batch sizes")
    ap.add_argument("--paper-nn", type=int, default=1, help="run the paper-network leg on the 9-component case")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return reference_arm(args, ws, rank)
    return ours_arm(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
