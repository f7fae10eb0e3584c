"""Seeded phase-EOS cases at the margins of the cubic's two decisions, built
from the oracle alone (test infrastructure):

* root count: pressures where f(Z) = Z^3 - Z^2 + r1 Z - r0 (Appendix A, Eq.
  cubic_Z) has a critical value f(zm) or f(zp) of size in [1e-6, 1e-3], on
  both sides of zero (one real root, or three with two close together);
* root choice: pressures with three admissible roots whose residual Gibbs
  energies gbar(Z) = Z - 1 - ln(Z - B) - (A/B) ln(1 + B/Z) (reading R6)
  differ by [1e-6, 1e-3], on both sides of the switch (the saturation line
  of a pure-like feed), including dense liquid roots close to B.

A and B scale with P at fixed T and composition, so each case is found by
bisection on P after one oracle evaluation at P = 1.
"""
import numpy as np

TARGETS = (1e-6, 1e-5, 1e-4, 1e-3)


def _ab(oracle_mod, s, T, c):
    _, _, _, AB = oracle_mod.eos(s, 1.0, T, c, with_jac=True)
    return AB[0], AB[1]


def _crit(a, b, P):
    A, B = a * P, b * P
    r1, r0 = A - B - B * B, A * B
    dc = 4.0 - 12.0 * r1
    if dc <= 0.0:
        return None
    sq = np.sqrt(dc)
    f = lambda z: ((z - 1.0) * z + r1) * z - r0
    return f((2.0 - sq) / 6.0), f((2.0 + sq) / 6.0)


def _gbar(Z, A, B):
    return Z - 1.0 - np.log(Z - B) - (A / B) * np.log1p(B / Z)


def _dg(oracle_mod, a, b, P):
    A, B = a * P, b * P
    r = oracle_mod.cubic_roots(A, B)
    r = r[r > B]
    if len(r) < 3:
        return None
    return _gbar(r.min(), A, B) - _gbar(r.max(), A, B)


def _bisect(fun, lo, hi, target, iters=200):
    """P in [lo, hi] with fun(P) = target, fun - target changing sign."""
    flo = fun(lo) - target
    for _ in range(iters):
        mid = np.sqrt(lo * hi)
        fm = fun(mid) - target
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
        if hi / lo - 1.0 < 1e-15:
            break
    return np.sqrt(lo * hi)


def _around(fun, P0, P1, out):
    """fun changes sign on [P0, P1]: append the pressures where |fun| equals
    each target on both sides of the zero."""
    Pz = _bisect(fun, P0, P1, 0.0)
    for side in (P0, P1):
        for t in TARGETS:
            v = fun(side)
            if v is None or abs(v) < t:
                continue
            lo, hi = (side, Pz) if side < Pz else (Pz, side)
            out.append(_bisect(fun, lo, hi, np.sign(v) * t))


def margin_cases(oracle_mod, s, seed, n_draws=30):
    """(P, T, c[nc, n], kind) arrays; kind 0 root count, 1 root choice."""
    rng = np.random.default_rng(seed)
    nc = s.nc
    Ps, Ts, cs, kinds = [], [], [], []
    for _ in range(n_draws):
        T = rng.uniform(0.35, 1.0) * rng.uniform(s.Tc.min(), s.Tc.max())
        c = rng.dirichlet(np.full(nc, 0.3))
        c = np.maximum(c, 1e-12)
        c /= c.sum()
        a, b = _ab(oracle_mod, s, T, c)
        grid = np.logspace(-3, 3, 1500)
        for j in (0, 1):
            f = lambda P, j=j: (lambda v: None if v is None else v[j])(_crit(a, b, P))
            v = [f(P) for P in grid]
            for k in range(len(grid) - 1):
                if v[k] is not None and v[k + 1] is not None and (v[k] > 0) != (v[k + 1] > 0):
                    got = []
                    _around(lambda P: f(P) if f(P) is not None else 0.0, grid[k], grid[k + 1], got)
                    for P in got:
                        Ps.append(P), Ts.append(T), cs.append(c), kinds.append(0)
        g = lambda P: _dg(oracle_mod, a, b, P)
        v = [g(P) for P in grid]
        for k in range(len(grid) - 1):
            if v[k] is not None and v[k + 1] is not None and (v[k] > 0) != (v[k + 1] > 0):
                got = []
                _around(lambda P: g(P) if g(P) is not None else 0.0, grid[k], grid[k + 1], got)
                for P in got:
                    Ps.append(P), Ts.append(T), cs.append(c), kinds.append(1)
    return np.array(Ps), np.array(Ts), np.ascontiguousarray(np.array(cs).T), np.array(kinds)
