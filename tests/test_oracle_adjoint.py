"""Pins of the oracle's sensitivities of the converged flash (the
implicit-function-theorem idea of Sec. 4.2.2 applied to the whole
equilibrium of Eq. eq_cond), each against something other than the formula
itself: finite differences of the oracle's ln phi and of its whole flash, the
phase rule and lever rule of a binary, and exact invariants (degree-0
homogeneity in the feed, normalised phases, the differentiated material
balance of Eq. material_balance)."""
import numpy as np
import pytest

from paper_2205_03090_gb300 import workloads as wl


def _sys(oracle_mod, comp):
    return oracle_mod.System(comp.Tc, comp.Pc, comp.omega, comp.kij)


@pytest.mark.parametrize("nc,seed", [(3, 0), (8, 1)])
def test_dlnphi_dPT_matches_finite_differences(oracle_mod, nc, seed):
    comp = wl.pseudo_components(nc, seed)
    s = _sys(oracle_mod, comp)
    cond = wl.conditions(nc, 12, 50 + seed)
    for k in range(cond.n):
        P, T, c = cond.P[k], cond.T[k], cond.z[:, k]
        dP, dT = oracle_mod.dlnphi_dPT(s, P, T, c)
        for which, (val, an) in enumerate(((P, dP), (T, dT))):
            h = 1e-6 * val
            args_p = [P + h, T] if which == 0 else [P, T + h]
            args_m = [P - h, T] if which == 0 else [P, T - h]
            Zp, lp = oracle_mod.eos(s, *args_p, c)
            Zm, lm = oracle_mod.eos(s, *args_m, c)
            Z0, _ = oracle_mod.eos(s, P, T, c)
            if abs(Zp - Zm) > 0.1 * Z0:  # the chosen root switched branch between the two points
                continue
            fd = (lp - lm) / (2 * h)
            assert np.abs(fd - an).max() <= 1e-6 * max(1.0, np.abs(an).max()) + 1e-9, (k, which, fd, an)


def _flash_fd(oracle_mod, s, P, T, z, nc):
    """Central differences (relative step 1e-6) of the oracle's whole flash;
    a perturbed feed is renormalised (the result depends on z / sum z)."""
    def f(P_, T_, z_):
        zz = (z_ / z_.sum()).reshape(nc, 1)
        r = oracle_mod.flash(s, np.array([P_]), np.array([T_]), zz, nthreads=1)
        return np.concatenate([r["beta"], r["x"][:, 0], r["y"][:, 0]]), r["nphase"][0]
    fd = np.zeros((1 + 2 * nc, nc + 2))
    for col in range(nc + 2):
        h = 1e-6 * ([P, T][col] if col < 2 else z[col - 2])
        ap, am = [P, T, z.copy()], [P, T, z.copy()]
        if col < 2:
            ap[col] += h
            am[col] -= h
        else:
            ap[2][col - 2] += h
            am[2][col - 2] -= h
        fp, np_ = f(*ap)
        fm, nm = f(*am)
        if np_ != 2 or nm != 2:
            return None
        fd[:, col] = (fp - fm) / (2 * h)
    return fd


@pytest.mark.parametrize("name,nc_sample", [("nc3_1e4", 12), ("nc10_2phase_1e6", 8)])
def test_flash_jacobian_matches_finite_differences(oracle_mod, name, nc_sample):
    comp, cond = wl.workload(name, 400)
    s = _sys(oracle_mod, comp)
    o = oracle_mod.flash(s, cond.P, cond.T, cond.z)
    jac, ok = oracle_mod.flash_jacobian(s, cond.P, cond.T, cond.z, o)
    # converged two-phase mixtures away from the critical region
    two = np.nonzero((o["nphase"] == 2) & ((o["status"] & 16) == 0) &
                     (np.abs(np.log(o["K"])).max(axis=0) > 0.3))[0][:nc_sample]
    assert len(two) >= nc_sample // 2
    errs = []
    for k in two:
        fd = _flash_fd(oracle_mod, s, cond.P[k], cond.T[k], cond.z[:, k].copy(), comp.nc)
        if fd is None:
            continue
        assert ok[k] == 0
        # column-wise relative error (P, T and z columns have different units)
        scale = np.maximum(np.abs(jac[k]).max(axis=0), 1e-12)
        errs.append((np.abs(fd - jac[k]).max(axis=0) / scale).max())
    errs = np.array(errs)
    print(name, "FD rel errors: median", np.median(errs), "max", errs.max())
    assert np.median(errs) < 1e-6 and errs.max() < 1e-4


def test_binary_phase_rule_and_lever_rule(oracle_mod):
    """Two components at fixed P, T: x and y do not depend on the feed inside
    the envelope (phase rule), and beta = (z_1 - x_1)/(y_1 - x_1) (lever rule)."""
    comp = wl.pseudo_components(2, 1)  # Tc 406 K and 625 K: a wide two-phase region
    s = _sys(oracle_mod, comp)
    cond = wl.conditions(2, 5000, 7, T_range=(150.0, 350.0), P_range=(0.5, 8.0))
    o = oracle_mod.flash(s, cond.P, cond.T, cond.z)
    jac, ok = oracle_mod.flash_jacobian(s, cond.P, cond.T, cond.z, o)
    two = np.nonzero((o["nphase"] == 2) & ((o["status"] & 16) == 0))[0]
    assert len(two) > 20
    for k in two[:50]:
        J = jac[k]
        assert np.abs(J[1:, 2:]).max() <= 1e-9 * max(1.0, np.abs(J).max()), J
        x1, y1, z = o["x"][0, k], o["y"][0, k], cond.z[:, k]
        S = z.sum()
        lever = np.array([(1.0 - z[0] / S) / S, (0.0 - z[0] / S) / S]) / (y1 - x1)
        assert np.allclose(J[0, 2:], lever, rtol=1e-8, atol=1e-12), (J[0, 2:], lever)


def test_single_phase_and_invariants(oracle_mod):
    comp, cond = wl.workload("nc10_2phase_1e6", 300)
    nc = comp.nc
    s = _sys(oracle_mod, comp)
    o = oracle_mod.flash(s, cond.P, cond.T, cond.z)
    jac, ok = oracle_mod.flash_jacobian(s, cond.P, cond.T, cond.z, o)
    one = np.nonzero(o["nphase"] == 1)[0]
    assert len(one) > 5
    for k in one:
        J, z = jac[k], cond.z[:, k]
        expect = np.eye(nc) - z[:, None]
        assert np.abs(J[0]).max() == 0.0 and np.abs(J[1:, :2]).max() == 0.0
        assert np.allclose(J[1:1 + nc, 2:], expect, atol=1e-15) and np.allclose(J[1 + nc:, 2:], expect, atol=1e-15)
    two = np.nonzero((o["nphase"] == 2) & (ok == 0))[0]
    assert len(two) > 50
    for k in two:
        J, z, b = jac[k], cond.z[:, k], o["beta"][k]
        x, y = o["x"][:, k], o["y"][:, k]
        sc = max(1.0, np.abs(J).max())
        # degree-0 homogeneity in the feed: the z columns annihilate z
        assert np.abs(J[:, 2:] @ z).max() <= 1e-9 * sc
        # x and y stay normalised
        assert np.abs(J[1:1 + nc].sum(axis=0)).max() <= 1e-9 * sc
        assert np.abs(J[1 + nc:].sum(axis=0)).max() <= 1e-9 * sc
        # differentiated material balance: (1 - beta) x + beta y = z / sum z
        dmb = (1 - b) * J[1:1 + nc] + b * J[1 + nc:] + np.outer(y - x, J[0])
        expect = np.zeros((nc, nc + 2))
        expect[:, 2:] = np.eye(nc) - z[:, None] / z.sum()
        assert np.abs(dmb - expect).max() <= 1e-9 * sc, np.abs(dmb - expect).max()
