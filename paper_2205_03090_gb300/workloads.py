"""Seeded synthetic inputs for the flash workloads.

This module draws random numbers only; it holds none of the method's
arithmetic, so both the CUDA path and the CPU oracle can be fed from it.
Every draw uses NumPy ``Generator(PCG64(seed))``.

Workloads (sizes named by what they are):
  * ``nc3_1e4``  -- 3 pseudo-components, 1e4 mixtures, z ~ Dirichlet(1)
  * ``nc8_1e6``  -- 8 pseudo-components, 1e6 mixtures, z ~ Dirichlet(0.5)
  * ``nc10_2phase_1e6`` -- 10 pseudo-components, T in [250, 450] K,
    P in [2, 15] MPa, z ~ Dirichlet(1) (two-phase-biased conditions)
  * ``uneven_systems()`` -- 64 fluid systems with nc ~ U{3..16}, each its
    own pseudo-components, 62,500 mixtures each (4e6 in all)
Pseudo-components: Tc ~ U(150, 650) K sorted ascending, Pc ~ U(2, 5) MPa,
omega ~ U(0, 0.5), symmetric k_ij ~ U(0, 0.1) with zero diagonal.  The paper's
own case-study data are synthetic too (Sec. 2.4: LHS + Dirichlet draws);
these draws stand in for them.  Compositions are floored at 1e-12 and
renormalised so that ln z stays finite for both implementations.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

Z_FLOOR = 1e-12


@dataclass
class Components:
    Tc: np.ndarray      # [nc] K
    Pc: np.ndarray      # [nc] MPa
    omega: np.ndarray   # [nc]
    kij: np.ndarray     # [nc, nc] symmetric, zero diagonal

    @property
    def nc(self) -> int:
        return int(self.Tc.shape[0])


@dataclass
class Conditions:
    P: np.ndarray   # [n] MPa
    T: np.ndarray   # [n] K
    z: np.ndarray   # [nc, n] component-major, columns sum to 1

    @property
    def n(self) -> int:
        return int(self.P.shape[0])


def pseudo_components(nc: int, seed: int) -> Components:
    g = np.random.Generator(np.random.PCG64(seed))
    Tc = np.sort(g.uniform(150.0, 650.0, nc))
    Pc = g.uniform(2.0, 5.0, nc)
    om = g.uniform(0.0, 0.5, nc)
    k = g.uniform(0.0, 0.1, (nc, nc))
    k = np.triu(k, 1)
    k = k + k.T
    return Components(Tc, Pc, om, k)


def dirichlet(g: np.random.Generator, alpha: float, nc: int, n: int) -> np.ndarray:
    z = g.dirichlet(np.full(nc, alpha), size=n).T.copy()  # [nc, n]
    z = np.maximum(z, Z_FLOOR)
    z /= z.sum(axis=0, keepdims=True)
    return np.ascontiguousarray(z)


def conditions(nc: int, n: int, seed: int, T_range=(200.0, 600.0), P_range=(0.1, 20.0),
               alpha: float = 1.0) -> Conditions:
    g = np.random.Generator(np.random.PCG64(seed))
    T = g.uniform(T_range[0], T_range[1], n)
    P = g.uniform(P_range[0], P_range[1], n)
    z = dirichlet(g, alpha, nc, n)
    return Conditions(P, T, z)


# Named workloads: (nc, n, component seed, condition seed, T range, P range, alpha)
WORKLOADS = {
    "nc3_1e4": dict(nc=3, n=10_000, comp_seed=0, cond_seed=0, T_range=(200.0, 600.0), P_range=(0.1, 20.0),
                    alpha=1.0),
    "nc8_1e6": dict(nc=8, n=1_000_000, comp_seed=0, cond_seed=1, T_range=(200.0, 600.0), P_range=(0.1, 20.0),
                    alpha=0.5),
    "nc10_2phase_1e6": dict(nc=10, n=1_000_000, comp_seed=0, cond_seed=3, T_range=(250.0, 450.0),
                            P_range=(2.0, 15.0), alpha=1.0),
    "nc10_2phase_1e7": dict(nc=10, n=10_000_000, comp_seed=0, cond_seed=4, T_range=(250.0, 450.0),
                            P_range=(2.0, 15.0), alpha=1.0),
}


def workload(name: str, n: int | None = None):
    """Components and conditions of a named workload (optionally the first
    ``n`` mixtures of a fresh draw of size n with the same seed)."""
    w = WORKLOADS[name]
    comp = pseudo_components(w["nc"], w["comp_seed"])
    cond = conditions(w["nc"], n if n is not None else w["n"], w["cond_seed"], w["T_range"], w["P_range"],
                      w["alpha"])
    return comp, cond


def uneven_systems(n_sys: int = 64, n_per: int = 62_500, seed: int = 2, nc_range=(3, 16), n_list=None):
    """Uneven batch: n_sys fluid systems with nc ~ U{nc_range} each, every
    system its own pseudo-components (drawn as above, seed [seed, s, 0]) and
    conditions T ~ U(200, 600) K, P ~ U(0.1, 20) MPa, z ~ Dirichlet(1) (seed
    [seed, s, 1]); n_per mixtures per system unless n_list gives them.
    Returns a list of (Components, Conditions)."""
    g = np.random.Generator(np.random.PCG64(seed))
    ncs = g.integers(nc_range[0], nc_range[1] + 1, n_sys)
    out = []
    for s in range(n_sys):
        n = int(n_list[s]) if n_list is not None else n_per
        comp = pseudo_components(int(ncs[s]), [seed, s, 0])
        cond = conditions(int(ncs[s]), n, [seed, s, 1])
        out.append((comp, cond))
    return out


# Paper Table 1 (Sec. 2.3): Pc [MPa], Tc [K], omega of the nine components;
# the only nonzero BIP is CH4-CO2 = 0.0882.
PAPER_TABLE1 = dict(
    names=["CH4", "C2H6", "C3H8", "nC4H10", "nC5H12", "C6H14", "C7H16+", "CO2", "N2"],
    Pc=[4.6, 4.875, 4.268, 3.796, 3.3332, 2.9688, 2.622, 7.382, 3.3944],
    Tc=[190.55, 305.43, 369.82, 425.16, 467.15, 507.4, 604.5, 304.19, 126.25],
    omega=[0.0111, 0.097, 0.1536, 0.2008, 0.2635, 0.296, 0.3565, 0.225, 0.039],
)


def paper_components(names) -> Components:
    t = PAPER_TABLE1
    idx = [t["names"].index(s) for s in names]
    Tc = np.array([t["Tc"][i] for i in idx])
    Pc = np.array([t["Pc"][i] for i in idx])
    om = np.array([t["omega"][i] for i in idx])
    k = np.zeros((len(idx), len(idx)))
    if "CH4" in names and "CO2" in names:
        a, b = names.index("CH4"), names.index("CO2")
        k[a, b] = k[b, a] = 0.0882
    return Components(Tc, Pc, om, k)


# Paper Table 2 (Sec. 2.3): composition ranges (mole fractions) of the four
# reservoir fluid types, in the component order of Table 1.
PAPER_TABLE2 = {
    "wet_gas":        [(0.80, 1.00), (0.02, 0.07), (0.0, 0.03), (0.0, 0.02), (0.0, 0.02), (0.0, 0.02), (0.0, 0.01),
                       (0.0, 0.02), (0.0, 0.005)],
    "gas_condensate": [(0.60, 0.80), (0.05, 0.10), (0.0, 0.04), (0.0, 0.03), (0.0, 0.02), (0.0, 0.02), (0.05, 0.10),
                       (0.0, 0.035), (0.0, 0.005)],
    "volatile_oil":   [(0.50, 0.70), (0.06, 0.10), (0.0, 0.045), (0.0, 0.03), (0.0, 0.02), (0.0, 0.02), (0.10, 0.30),
                       (0.0, 0.02), (0.0, 0.005)],
    "black_oil":      [(0.20, 0.40), (0.03, 0.06), (0.0, 0.015), (0.0, 0.015), (0.0, 0.01), (0.0, 0.02),
                       (0.45, 0.65), (0.0, 0.001), (0.0, 0.005)],
}
# Paper Table 3 (Sec. 2.4): Dirichlet concentrations per fluid type,
# (alpha_CH4, alpha_C2H6, alpha_C7H16+); 1 for the other components.
PAPER_TABLE3 = {"wet_gas": (100.0, 5.0, 1.0), "gas_condensate": (40.0, 5.0, 5.0), "volatile_oil": (55.0, 8.0, 20.0),
                "black_oil": (25.0, 4.0, 40.0)}
# The three case studies (Sec. 2.3): components and P [MPa], T [K] ranges.
PAPER_CASES = {
    "c2": dict(names=["CH4", "C6H14"], P=(0.1, 10.0), T=(200.0, 500.0)),
    "c4": dict(names=["CH4", "C2H6", "C3H8", "nC4H10"], P=(0.1, 10.0), T=(200.0, 500.0)),
    "c9": dict(names=list(PAPER_TABLE1["names"]), P=(5.0, 25.0), T=(200.0, 600.0)),
}


def lhs_uniform(g: np.random.Generator, n: int, d: int) -> np.ndarray:
    """Latin hypercube sample of U(0,1)^d (McKay et al.): in every dimension
    each of the n strata [k/n, (k+1)/n) holds exactly one point."""
    u = np.empty((n, d))
    for j in range(d):
        u[:, j] = (g.permutation(n) + g.uniform(size=n)) / n
    return u


def _dirichlet_from_uniform(u: np.ndarray, alpha: np.ndarray) -> np.ndarray:
    """Eq. sampling: y_i = Gamma(alpha_i, 1).ppf(u_i), z = y / sum y.
    Returns z [n, nc].  Gamma(1, 1).ppf(u) = -ln(1 - u) in closed form."""
    y = np.empty_like(u)
    one = alpha == 1.0
    y[:, one] = -np.log1p(-u[:, one])
    if (~one).any():
        from scipy.special import gammaincinv
        y[:, ~one] = gammaincinv(alpha[None, ~one], u[:, ~one])
    return y / y.sum(axis=1, keepdims=True)


def paper_case(case: str, n: int, seed: int = 0):
    """Inputs of a paper case study (Sec. 2.3-2.4).
    c2, c4: LHS samples of (P, T, u) with P, T scaled to the case's ranges and
    z from Eq. sampling with alpha = 1 (the whole simplex).
    c9: the four fluid types of Table 2 equally represented; each type's z is
    Dirichlet with its Table 3 alpha, kept only if every component lies in
    the type's range.  The acceptance rates are low (black oil ~0.1 %, gas
    condensate ~1 %), so the candidates come from Gamma(alpha_i, 1) draws
    (the same accepted distribution as Gamma.ppf of LHS uniforms, whose
    stratification the rejection would undo) and P, T keep their LHS strata.
    Returns (Components, Conditions, fluid type index per mixture or None)."""
    c = PAPER_CASES[case]
    comp = paper_components(c["names"])
    nc = comp.nc
    g = np.random.Generator(np.random.PCG64(seed))
    if case != "c9":
        u = lhs_uniform(g, n, 2 + nc)
        P = c["P"][0] + (c["P"][1] - c["P"][0]) * u[:, 0]
        T = c["T"][0] + (c["T"][1] - c["T"][0]) * u[:, 1]
        z = _dirichlet_from_uniform(u[:, 2:], np.ones(nc))
        z = np.maximum(z, Z_FLOOR)
        z /= z.sum(axis=1, keepdims=True)
        return comp, Conditions(P, T, np.ascontiguousarray(z.T)), None
    types = list(PAPER_TABLE2)
    per = [n // 4 + (1 if k < n % 4 else 0) for k in range(4)]
    Ps, Ts, zs, ft = [], [], [], []
    for k, name in enumerate(types):
        a1, a2, a7 = PAPER_TABLE3[name]
        alpha = np.ones(nc)
        alpha[0], alpha[1], alpha[6] = a1, a2, a7
        lo = np.array([r[0] for r in PAPER_TABLE2[name]])
        hi = np.array([r[1] for r in PAPER_TABLE2[name]])
        # the ranges checked on the shrinking candidate set, narrowest first
        order = np.argsort(hi - lo)
        acc, got = [], 0
        while got < per[k]:
            m = 1 << 20
            y = np.empty((nc, m))
            for i in range(nc):
                y[i] = g.standard_exponential(m) if alpha[i] == 1.0 else g.standard_gamma(alpha[i], m)
            S = y.sum(axis=0)
            keep = np.arange(m)
            for i in order:
                zi = y[i, keep] / S[keep]
                keep = keep[(zi >= lo[i]) & (zi <= hi[i])]
            z = (y[:, keep] / S[keep]).T[:per[k] - got]
            acc.append(z)
            got += len(z)
        u = lhs_uniform(g, per[k], 2)
        Ps.append(c["P"][0] + (c["P"][1] - c["P"][0]) * u[:, 0])
        Ts.append(c["T"][0] + (c["T"][1] - c["T"][0]) * u[:, 1])
        zs.append(np.concatenate(acc))
        ft.append(np.full(per[k], k, np.int32))
    z = np.concatenate(zs)
    z = np.maximum(z, Z_FLOOR)
    z /= z.sum(axis=1, keepdims=True)
    return comp, Conditions(np.concatenate(Ps), np.concatenate(Ts), np.ascontiguousarray(z.T)), np.concatenate(ft)


def mlp_init(din: int, hidden: int, dout: int, seed: int, arch: int = 0) -> np.ndarray:
    """Initial network parameters drawn from seeded Glorot-uniform
    distributions (weights) with zero biases, in the flat order W_0, b_0,
    W_1, b_1, ... (each W row-major [out, in]).  arch 0: three hidden layers;
    arch 1: a hidden layer, six residual-block layers, output on [u; h]."""
    g = np.random.Generator(np.random.PCG64(seed))
    parts = []
    shapes = ([(hidden, din)] + [(hidden, hidden)] * 6 + [(dout, din + hidden)] if arch == 1 else
              [(hidden, din), (hidden, hidden), (hidden, hidden), (dout, hidden)])
    for o, i in shapes:
        lim = np.sqrt(6.0 / (i + o))
        parts.append(g.uniform(-lim, lim, o * i))
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


def epoch_permutation(n: int, seed: int, epoch: int) -> np.ndarray:
    """Seeded shuffle of n training samples for one epoch."""
    g = np.random.Generator(np.random.PCG64([seed, epoch]))
    return g.permutation(n).astype(np.int32)
