"""Seeded mixtures whose precheck Rachford-Rice root (Sec. 2.2.3, reading R11:
three SS evaluations from Wilson K) lies just inside or outside (0, 1), built
from the oracle's primitives alone (test infrastructure).

Along a composition path z(s) = (1 - s) z_a + s z_b between a heavy-rich and
a light-rich feed, theta_1(s) (the root for Wilson K) and theta_2(s) (the root
after one SS update, ln K_2 = ln phi^L(x_1) - ln phi^V(y_1)) vary
continuously; bisection on s puts them at 0 or 1 plus or minus each target.
"""
import numpy as np

TARGETS = (1e-7, 1e-6, 1e-5, 1e-4)


def _thetas(oracle_mod, s, P, T, z, lnKw):
    th1 = oracle_mod.rr(z, np.exp(lnKw))
    if th1 is None:
        return None, None
    if not (0.0 < th1 < 1.0):
        return th1, None
    K = np.exp(lnKw)
    x = z / (1.0 + th1 * (K - 1.0))
    y = K * x
    try:
        _, lx = oracle_mod.eos(s, P, T, x)
        _, ly = oracle_mod.eos(s, P, T, y)
    except ValueError:
        return th1, None
    return th1, oracle_mod.rr(z, np.exp(lx - ly))


def _bisect(fun, lo, hi, target, iters=100):
    flo = fun(lo) - target
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        fm = fun(mid) - target
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


def margin_mixtures(oracle_mod, s, seed, n_paths=12, P_range=(0.1, 20.0), T_range=(200.0, 600.0)):
    """(P, T, z[nc, n], which) with which = 1 or 2: the evaluation whose theta
    sits at the margin."""
    rng = np.random.default_rng(seed)
    nc = s.nc
    out = []
    for _ in range(n_paths):
        P, T = rng.uniform(*P_range), rng.uniform(*T_range)
        lnKw = oracle_mod.wilson(s, P, T)
        light = lnKw > np.median(lnKw)
        za = np.where(light, 0.02, 1.0) * rng.dirichlet(np.ones(nc))
        zb = np.where(light, 1.0, 0.02) * rng.dirichlet(np.ones(nc))
        za, zb = za / za.sum(), zb / zb.sum()
        zs = lambda t: (1.0 - t) * za + t * zb
        grid = np.linspace(0.0, 1.0, 161)
        th = [_thetas(oracle_mod, s, P, T, zs(t), lnKw) for t in grid]
        for which in (1, 2):
            def f(t, which=which):
                v = _thetas(oracle_mod, s, P, T, zs(t), lnKw)[which - 1]
                return np.nan if v is None else v
            for k in range(len(grid) - 1):
                a, b = th[k][which - 1], th[k + 1][which - 1]
                if a is None or b is None:
                    continue
                for edge in (0.0, 1.0):
                    if (a - edge) * (b - edge) < 0:
                        for t in TARGETS:
                            for sgn in (-1.0, 1.0):
                                tt = _bisect(f, grid[k], grid[k + 1], edge + sgn * t)
                                v = f(tt)
                                if np.isfinite(v) and abs(v - (edge + sgn * t)) < 0.5 * t:
                                    out.append((P, T, zs(tt), which))
    P = np.array([o[0] for o in out])
    T = np.array([o[1] for o in out])
    z = np.maximum(np.array([o[2] for o in out]).T, 1e-12)  # the workloads' floor (finite ln z in FP32 too)
    z = np.ascontiguousarray(z / z.sum(axis=0, keepdims=True))
    return P, T, z, np.array([o[3] for o in out])
