"""The paper's three case studies (Sec. 2.3; Table 1 components, LHS and
Eq. sampling inputs) through the GPU flash, against the oracle mixture by
mixture: CH4/C6H14, C1-C4, and the 9-component fluid with four reservoir
fluid types equally represented."""
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


@pytest.mark.parametrize("case,n", [("c2", 20000), ("c4", 20000), ("c9", 20000)])
def test_case_study_parity(ptf, oracle_mod, case, n):
    import torch
    comp, cond, ft = wl.paper_case(case, n, 11)
    fl = ptf.Flash(comp.Tc, comp.Pc, comp.omega, comp.kij, n_max=n)
    P, T, z = (torch.tensor(a, device="cuda") for a in (cond.P, cond.T, cond.z))
    out = fl.ptflash_flash(P, T, z.contiguous())
    torch.cuda.synchronize()
    g = {k: getattr(out, k).cpu().numpy() for k in ("nphase", "beta", "x", "y", "status")}
    r = compare(oracle_mod, comp, cond, g)
    print(case, {k: v for k, v in r.items() if k != "bad_idx"}, "two-phase", float((g["nphase"] == 2).mean()))
    _assert_parity(r, max_capped_frac=1e-3)
    if ft is not None:  # every fluid type reaches both phase counts
        for t in range(4):
            assert set(np.unique(g["nphase"][ft == t])) <= {1, 2}
    fl.close()
