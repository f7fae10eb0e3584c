"""Decisions at their margins, options and failure forms, on the GPU through
the C ABI.

* The cubic's root count and root choice (Appendix A, reading R6), which the
  kernels may take in FP32 only where an error bound proves FP64 agrees:
  points whose critical values or gbar differences lie in [1e-6, 1e-3] of the
  switch, compared root by root with the oracle (ptflash_phase_eos).
* The precheck's Rachford-Rice route (Sec. 2.2.3), whose first two
  evaluations run in FP32: mixtures whose theta after the first or second
  evaluation lies within 1e-7..1e-4 of 0 or 1 take the oracle's route and
  reach its result.
* Iteration caps and tolerances of ptflash_options: a cap of 1 gives MAXITER
  statuses; invalid options are rejected.
* Non-finite inputs injected on the host (NaN or infinite P, T, z) come back
  single-phase with the NONFINITE status, without disturbing the rest of the
  batch.
"""
import numpy as np
import pytest

from paper_2205_03090_gb300 import workloads as wl
import eos_margins
import precheck_margins
from test_gpu_parity import _assert_parity, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ptf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2205_03090_gb300 import build, ptflash
    build.build()
    ptflash.load()
    return ptflash


def _dev(*arrs):
    import torch
    return [torch.tensor(np.ascontiguousarray(a), device="cuda") for a in arrs]


@pytest.mark.parametrize("nc,seed", [(2, 5), (4, 2), (8, 0)])
def test_eos_root_count_and_choice_at_margins(ptf, oracle_mod, nc, seed):
    import torch
    comp = wl.pseudo_components(nc, seed)
    s = oracle_mod.System(comp.Tc, comp.Pc, comp.omega, comp.kij)
    P, T, c, kind = eos_margins.margin_cases(oracle_mod, s, 100 + seed)
    assert (kind == 0).sum() >= 50 and (kind == 1).sum() >= 20
    fl = ptf.Flash(comp.Tc, comp.Pc, comp.omega, comp.kij, n_max=4096)
    Zg, lg = fl.ptflash_phase_eos(*_dev(P, T, c))
    torch.cuda.synchronize()
    Zg, lg = Zg.cpu().numpy(), lg.cpu().numpy()
    worst_gap, dense = np.inf, 1.0
    for k in range(len(P)):
        Zo, lo, _, AB = oracle_mod.eos(s, P[k], T[k], c[:, k], with_jac=True)
        roots = oracle_mod.cubic_roots(*AB)
        roots = roots[roots > AB[1]]
        # the same root: closer to the oracle's choice than to any other admissible root
        others = np.abs(roots - Zo)
        gap = others[others > 0].min() if (others > 0).any() else np.inf
        worst_gap = min(worst_gap, gap)
        dense = min(dense, (roots.min() - AB[1]) / roots.min())
        assert abs(Zg[k] - Zo) <= 1e-10 * Zo, (k, kind[k], P[k], T[k], Zg[k], Zo, roots)
        assert np.abs(lg[:, k] - lo).max() <= 1e-9, (k, kind[k], np.abs(lg[:, k] - lo).max())
    print(f"nc {nc}: {len(P)} margin points ({(kind == 0).sum()} root count, {(kind == 1).sum()} root choice), "
          f"closest other root {worst_gap:.2e}, smallest (Z_l - B)/Z_l {dense:.3f}")
    fl.close()


@pytest.mark.parametrize("nc,seed", [(3, 0), (8, 0)])
def test_precheck_routes_at_theta_margins(ptf, oracle_mod, nc, seed):
    import torch
    comp = wl.pseudo_components(nc, seed)
    s = oracle_mod.System(comp.Tc, comp.Pc, comp.omega, comp.kij)
    P, T, z, which = precheck_margins.margin_mixtures(oracle_mod, s, 200 + seed)
    assert (which == 1).sum() >= 20 and (which == 2).sum() >= 20
    fl = ptf.Flash(comp.Tc, comp.Pc, comp.omega, comp.kij, n_max=4096)
    out = fl.ptflash_flash(*_dev(P, T, z))
    torch.cuda.synchronize()
    g = {k: getattr(out, k).cpu().numpy() for k in ("nphase", "beta", "x", "y", "status")}
    cond = wl.Conditions(P=P, T=T, z=z)
    r = compare(oracle_mod, comp, cond, g)
    print(f"nc {nc}: {len(P)} margin mixtures", {k: v for k, v in r.items() if k != "bad_idx"})
    _assert_parity(r, max_capped_frac=0.0)
    fl.close()


def test_forced_caps_give_maxiter_and_bad_options_are_rejected(ptf):
    import torch
    comp, cond = wl.workload("nc8_1e6", 20000)
    fl = ptf.Flash(comp.Tc, comp.Pc, comp.omega, comp.kij, n_max=1 << 15)
    P, T, z = _dev(cond.P, cond.T, cond.z)
    base = fl.ptflash_flash(P, T, z)
    torch.cuda.synchronize()
    bst, bit = base.status.cpu().numpy(), base.iters.cpu().numpy()
    split_tr = (bst & 8) != 0
    assert split_tr.sum() > 100 and ((bst & 16) != 0).sum() == 0
    # one split trust-region iteration: every run that needs more stops at the cap
    one = fl.ptflash_flash(P, T, z, max_tr_split=1, max_polish=1)
    torch.cuda.synchronize()
    st, it = one.status.cpu().numpy(), one.iters.cpu().numpy()
    # the split TR field counts trust-region iterations and Newton steps: runs
    # that took more than one of each cannot converge under these caps
    need_more = split_tr & (((bit >> 8) & 255) > 2)
    assert need_more.sum() > 100
    assert np.all((st[need_more] & 16) != 0)
    assert np.all(((it[split_tr] >> 8) & 255) <= 2)  # one TR iteration + at most one Newton step
    # mixtures that never reach the split trust region are untouched
    same = ~split_tr
    np.testing.assert_array_equal(one.nphase.cpu().numpy()[same], base.nphase.cpu().numpy()[same])
    np.testing.assert_array_equal(one.beta.cpu().numpy()[same], base.beta.cpu().numpy()[same])
    # stability trust region capped at one iteration per trial
    one_s = fl.ptflash_flash(P, T, z, max_tr_stab=1)
    torch.cuda.synchronize()
    st_s, it_s = one_s.status.cpu().numpy(), one_s.iters.cpu().numpy()
    stab_tr_runs = ((bit >> 24) & 255) > 2  # more than one iteration in a trial at least
    assert stab_tr_runs.sum() > 10
    assert np.all(((it_s >> 24) & 255) <= 2)
    assert np.any((st_s[stab_tr_runs] & 16) != 0)
    # a tighter fugacity tolerance is met where runs converge
    tight = fl.ptflash_flash(P, T, z, tol_fug=1e-12)
    torch.cuda.synchronize()
    assert ((tight.status.cpu().numpy() & 16) != 0).mean() < 0.01
    for bad in (dict(max_tr_split=-1), dict(max_ss_stab=201), dict(tol_fug=-1.0), dict(tol_stab=float("nan"))):
        with pytest.raises(ptf.PtflashError):
            fl.ptflash_flash(P, T, z, **bad)
    fl.close()


def test_nonfinite_inputs_are_flagged_without_fault(ptf):
    import torch
    comp, cond = wl.workload("nc8_1e6", 4096)
    fl = ptf.Flash(comp.Tc, comp.Pc, comp.omega, comp.kij, n_max=1 << 13)
    clean = fl.ptflash_flash(*_dev(cond.P, cond.T, cond.z))
    torch.cuda.synchronize()
    P, T, z = cond.P.copy(), cond.T.copy(), cond.z.copy()
    rng = np.random.default_rng(9)
    bad = np.sort(rng.choice(cond.n, 60, replace=False))
    kinds = [("P", np.nan), ("T", np.nan), ("z", np.nan), ("P", np.inf), ("T", -np.inf), ("z", np.inf)]
    for j, k in enumerate(bad):
        name, v = kinds[j % len(kinds)]
        if name == "P":
            P[k] = v
        elif name == "T":
            T[k] = v
        else:
            z[j % comp.nc, k] = v
    out = fl.ptflash_flash(*_dev(P, T, z))
    torch.cuda.synchronize()
    st, nph = out.status.cpu().numpy(), out.nphase.cpu().numpy()
    assert np.all((st[bad] & 64) != 0), st[bad]
    assert np.all(nph[bad] == 1)
    good = np.setdiff1d(np.arange(cond.n), bad)
    for key in ("nphase", "status", "beta", "x", "y", "K"):
        a = getattr(out, key).cpu().numpy()[..., good]
        b = getattr(clean, key).cpu().numpy()[..., good]
        np.testing.assert_array_equal(a, b)
    fl.close()


def test_fp64_probe(ptf):
    """The FP64 FMA probe runs and reports a rate in the range this class of
    GPU can reach (above 0.3 and below 3 TFLOP/s)."""
    tf, ms = ptf.fp64_fma_rate(2000)
    print(f"fp64 fma rate {tf:.3f} TFLOP/s over {ms:.2f} ms")
    assert 0.3 < tf < 3.0 and ms > 0
