"""Uneven batches (many fluid systems of different nc in one graph launch)
through the C ABI, against the CPU oracle system by system.

The method per mixture is the plain flash of Sec. 2.2.3; a batch only gives
each mixture its own system's component data, so every system's results must
meet the same parity bar as a single-system flash, and equal the
single-system entry point's results.
"""
import numpy as np
import pytest

from paper_2205_03090_gb300 import workloads as wl
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


def _systems_small():
    # every nc from 2 to 16 once (nc = 2 outside the uneven workload's range),
    # ragged sizes, one empty system, two systems sharing nc = 8
    ncs = list(range(2, 17)) + [8]
    g = np.random.Generator(np.random.PCG64(41))
    ns = [int(v) for v in g.integers(200, 1500, len(ncs))]
    ns[5] = 0
    out = []
    for s, (nc, n) in enumerate(zip(ncs, ns)):
        out.append((wl.pseudo_components(nc, [41, s, 0]), wl.conditions(nc, n, [41, s, 1])))
    return out


def _batch(ptf, systems):
    b = ptf.Batch([(c.Tc, c.Pc, c.omega, c.kij) for c, _ in systems], [cd.n for _, cd in systems])
    P, T, z = b.pack([(cd.P, cd.T, cd.z) for _, cd in systems])
    return b, P, T, z


def test_batch_parity_every_nc(ptf, oracle_mod):
    import torch
    systems = _systems_small()
    b, P, T, z = _batch(ptf, systems)
    out = b.ptflash_batch_flash(P, T, z)
    torch.cuda.synchronize()
    info = b.ptflash_batch_info()
    assert info["groups"] == len({c.nc for c, cd in systems if cd.n > 0})
    assert info["mixtures"] == sum(cd.n for _, cd in systems)
    assert info["graph_nodes"] >= 13 * info["groups"]  # memset, gather, 10 pipeline kernels, scatter
    for s, (comp, cond) in enumerate(systems):
        if cond.n == 0:
            continue
        g = b.unpack(out, s)
        r = compare(oracle_mod, comp, cond, g)
        print("system", s, "nc", comp.nc, {k: v for k, v in r.items() if k != "bad_idx"})
        _assert_parity(r, max_capped_frac=1e-3)
    b.close()


def test_batch_equals_single_system_path(ptf):
    """The per-mixture component tables give the single-system results."""
    import torch
    systems = _systems_small()
    b, P, T, z = _batch(ptf, systems)
    out = b.ptflash_batch_flash(P, T, z)
    torch.cuda.synchronize()
    for s in (0, 6, 9, 14, 15):
        comp, cond = systems[s]
        fl = ptf.Flash(comp.Tc, comp.Pc, comp.omega, comp.kij, n_max=4096)
        d = [torch.tensor(a, device="cuda") for a in (cond.P, cond.T, cond.z)]
        one = fl.ptflash_flash(d[0], d[1], d[2].contiguous())
        torch.cuda.synchronize()
        g = b.unpack(out, s)
        assert np.array_equal(g["nphase"], one.nphase.cpu().numpy())
        assert np.array_equal(g["status"], one.status.cpu().numpy())
        assert np.abs(g["beta"] - one.beta.cpu().numpy()).max() <= 1e-13
        assert np.abs(g["x"] - one.x.cpu().numpy()).max() <= 1e-13
        fl.close()
    b.close()


def test_batch_recapture_and_tune(ptf):
    """New output pointers re-capture the graph; tuning keeps the results."""
    import torch
    systems = _systems_small()
    b, P, T, z = _batch(ptf, systems)
    o1 = b.ptflash_batch_flash(P, T, z)
    o2 = b.ptflash_batch_flash(P, T, z)  # fresh outputs: new pointers, new capture
    torch.cuda.synchronize()
    assert torch.equal(o1.nphase, o2.nphase) and torch.equal(o1.beta, o2.beta)
    bps, ms = b.ptflash_batch_tune(P, T, z)
    assert set(bps) == set(int(k) for k, m in zip(b.nc, b.n) if m > 0)
    assert all(v in (0, 1, 2, 3, 4) for v in bps.values())
    assert all(t > 0 for t in ms.values())
    o3 = b.ptflash_batch_flash(P, T, z)
    torch.cuda.synchronize()
    assert torch.equal(o1.nphase, o3.nphase) and torch.equal(o1.status, o3.status)
    assert (o1.beta - o3.beta).abs().max().item() <= 1e-13
    b.close()


def test_batch_full_size_sampled(ptf, oracle_mod):
    """64 systems, nc ~ U{3..16}, 62,500 mixtures each (4e6, one graph
    launch): 40 sampled mixtures per system against the oracle."""
    import torch
    systems = wl.uneven_systems()
    b, P, T, z = _batch(ptf, systems)
    b.ptflash_batch_tune(P, T, z)
    out = b.ptflash_batch_flash(P, T, z)
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    bad = 0
    for s, (comp, cond) in enumerate(systems):
        g = b.unpack(out, s)
        idx = np.sort(rng.choice(cond.n, 40, replace=False))
        r = compare(oracle_mod, comp, cond, g, idx=idx, fug_checks=40)
        assert r["label_bad"] == 0, (s, r)
        assert r["mass_balance"] < 1e-12 and r["max_fug"] <= 1e-10, (s, r)
        bad += r["val_bad"]
    assert bad <= 2, bad
    b.close()


def test_batch_invalid_arguments(ptf):
    c = wl.pseudo_components(4, 0)
    with pytest.raises(ptf.PtflashError):  # nc = 17
        c17 = wl.pseudo_components(17, 0)
        ptf.Batch([(c17.Tc, c17.Pc, c17.omega, c17.kij)], [10])
    k = c.kij.copy()
    k[0, 1] += 0.01  # not symmetric
    with pytest.raises(ptf.PtflashError):
        ptf.Batch([(c.Tc, c.Pc, c.omega, k)], [10])
    with pytest.raises(ptf.PtflashError):
        ptf.Batch([(c.Tc, c.Pc, c.omega, c.kij)], [-1])
    b = ptf.Batch([(c.Tc, c.Pc, c.omega, c.kij)], [0])  # an empty batch flashes nothing
    import torch
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    b.ptflash_batch_flash(e, e, e)
    b.close()
