"""Trust-region runs with several lanes each give the one-lane results bit for bit.

The split trust region runs one lane per mixture while its queue lasts and,
in the drain, G lanes per mixture (one per component).  The option tr_lanes
forces one lane throughout (1) or G lanes throughout (2).  Every output of
every mixture must be identical, bit for bit, in the three modes: the
several-lanes code performs the one-lane operations in the same order, so any
difference is a bug in it.  Mode 2 runs every split trust-region mixture
through the several-lanes code, so it checks that code on all of them.
"""
import numpy as np
import pytest

from paper_2205_03090_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FIELDS = ("nphase", "beta", "x", "y", "K", "status", "iters")


@pytest.fixture(scope="module")
def ptf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2205_03090_gb300 import build, ptflash
    build.build()
    ptflash.load()
    return ptflash


def _run(ptf, comp, cond, **opts):
    import torch
    fl = ptf.Flash(comp.Tc, comp.Pc, comp.omega, comp.kij, n_max=cond.n)
    P, T, z = (torch.tensor(cond.P, device="cuda"), torch.tensor(cond.T, device="cuda"),
               torch.tensor(cond.z, device="cuda").contiguous())
    out = fl.ptflash_flash(P, T, z, **opts)
    torch.cuda.synchronize()
    res = {k: getattr(out, k).cpu().numpy() for k in FIELDS}
    res["counts"] = fl.ptflash_last_counts()
    fl.close()
    return res


def _same_bits(a, b):
    if a.dtype == np.float64:
        return np.array_equal(a.view(np.int64), b.view(np.int64))
    return np.array_equal(a, b)


def _cases():
    c9_comp, c9_cond, _ = wl.paper_case("c9", 60_000, seed=5)
    return [
        ("nc8", *wl.workload("nc8_1e6", n=150_000)),
        ("c9", c9_comp, c9_cond),
        ("nc5", wl.pseudo_components(5, 7), wl.conditions(5, 60_000, 7, alpha=0.5)),
        ("nc12", wl.pseudo_components(12, 8), wl.conditions(12, 40_000, 8, alpha=0.5)),
        ("nc16", wl.pseudo_components(16, 9), wl.conditions(16, 20_000, 9, alpha=0.5)),
        ("nc3", *wl.workload("nc3_1e4")),
    ]


@pytest.mark.parametrize("case", range(6))
def test_tr_lanes_bit_identical(ptf, case):
    name, comp, cond = _cases()[case]
    one = _run(ptf, comp, cond, tr_lanes=1)
    assert one["counts"]["split_tr"] > 0, f"{name}: no split trust-region run to compare"
    for mode in (0, 2):
        r = _run(ptf, comp, cond, tr_lanes=mode)
        for k in FIELDS:
            if not _same_bits(one[k], r[k]):
                a, b = one[k], r[k]
                bad = np.nonzero((a != b).reshape(-1, cond.n).any(axis=0) if a.ndim > 1 else a != b)[0]
                raise AssertionError(f"{name}, tr_lanes={mode}: {k} differs from one lane per run on "
                                     f"{len(bad)} mixtures, first {bad[:5].tolist()}, status "
                                     f"{one['status'][bad[:5]].tolist()} vs {r['status'][bad[:5]].tolist()}")
        assert one["counts"] == r["counts"]


def test_tr_lanes_invalid(ptf):
    comp, cond = wl.workload("nc3_1e4", n=64)
    with pytest.raises(ptf.PtflashError):
        _run(ptf, comp, cond, tr_lanes=3)
    with pytest.raises(ptf.PtflashError):
        _run(ptf, comp, cond, tr_lanes=-1)
