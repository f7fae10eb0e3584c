"""The paper's case-study inputs (Sec. 2.3-2.4): Latin hypercube strata,
Table 2 composition ranges, equal representation of the fluid types, and the
Dirichlet(1) marginals of the whole-simplex cases."""
import numpy as np

from paper_2205_03090_gb300 import workloads as wl


def test_lhs_one_point_per_stratum():
    g = np.random.Generator(np.random.PCG64(0))
    u = wl.lhs_uniform(g, 1000, 5)
    for j in range(5):
        assert np.array_equal(np.sort(np.floor(u[:, j] * 1000).astype(int)), np.arange(1000))


def test_whole_simplex_cases():
    for case, nc in (("c2", 2), ("c4", 4)):
        comp, cond, ft = wl.paper_case(case, 20000, 3)
        assert comp.nc == nc and ft is None
        assert cond.P.min() >= 0.1 and cond.P.max() <= 10.0 and cond.T.min() >= 200.0 and cond.T.max() <= 500.0
        assert np.allclose(cond.z.sum(axis=0), 1.0)
        # Dirichlet(1, ..., 1): every marginal has mean 1/nc and variance (nc - 1)/(nc^2 (nc + 1))
        assert np.allclose(cond.z.mean(axis=1), 1.0 / nc, atol=0.01)
        assert np.allclose(cond.z.var(axis=1), (nc - 1) / (nc * nc * (nc + 1)), rtol=0.05)


def test_nine_component_fluid_types():
    comp, cond, ft = wl.paper_case("c9", 8000, 5)
    assert comp.nc == 9 and np.array_equal(np.bincount(ft), [2000] * 4)
    assert cond.P.min() >= 5.0 and cond.P.max() <= 25.0 and cond.T.min() >= 200.0 and cond.T.max() <= 600.0
    # only the CH4-CO2 interaction is non-zero (Sec. 2.3)
    k = comp.kij.copy()
    assert k[0, 7] == k[7, 0] == 0.0882
    k[0, 7] = k[7, 0] = 0.0
    assert not k.any()
    for t, name in enumerate(wl.PAPER_TABLE2):
        lo = np.array([r[0] for r in wl.PAPER_TABLE2[name]])
        hi = np.array([r[1] for r in wl.PAPER_TABLE2[name]])
        z = cond.z[:, ft == t].T
        assert np.all(z >= lo - 1e-11) and np.all(z <= hi + 1e-11), name
