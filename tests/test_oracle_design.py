"""Pins of the oracle's design loop: density filter (Sec. 2.3), SIMP and the
sensitivity chain (Eq. sens) by finite differences, the OC update against an
exact breakpoint solver, and Alg. 1 against a hand trace."""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import design, fem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_filter_taps():
    assert len(design.filter_offsets(1.5)) == 19
    assert len(design.filter_offsets(2.0)) == 27
    assert len(design.filter_offsets(1.0)) == 1


@pytest.mark.parametrize("rmin", [1.5, 2.0, 2.5])
def test_filter_brute_force_dense(rmin):
    """W built element pair by element pair from minimum-image centroid
    distances."""
    n = 7
    N = n ** 3
    coords = np.array([(x, y, z) for z in range(n) for y in range(n) for x in range(n)])
    W = np.zeros((N, N))
    for e in range(N):
        d = coords - coords[e]
        d = (d + n // 2) % n - n // 2           # minimum image (n odd)
        dist = np.sqrt((d * d).sum(axis=1))
        w = np.where(dist < rmin, rmin - dist, 0.0)
        W[e] = w / w.sum()
    rng = np.random.default_rng(0)
    rho = rng.uniform(size=N)
    assert np.allclose(design.density_filter(n, rho, rmin), W @ rho, atol=1e-14)
    s = rng.standard_normal(N)
    assert np.allclose(design.density_filter_transpose(n, s, rmin), W.T @ s, atol=1e-14)


def test_filter_mean_and_constants():
    n = 8
    rng = np.random.default_rng(1)
    rho = rng.uniform(size=n ** 3)
    rf = design.density_filter(n, rho, 2.0)
    assert abs(rf.mean() - rho.mean()) < 1e-14
    assert np.allclose(design.density_filter(n, np.full(n ** 3, 0.3), 1.5), 0.3, atol=1e-15)
    # W is symmetric on the periodic grid
    s = rng.standard_normal(n ** 3)
    assert np.allclose(design.density_filter_transpose(n, s, 1.5),
                       design.density_filter(n, s, 1.5), atol=1e-14)


def test_simp_derivative_fd():
    x = np.linspace(0.05, 0.95, 13)
    h = 1e-6
    fd = (design.simp(x + h, 3, 1, 1e-3) - design.simp(x - h, 3, 1, 1e-3)) / (2 * h)
    assert np.allclose(fd, design.simp_derivative(x, 3, 1, 1e-3), rtol=1e-8)
    assert np.allclose(design.simp(np.array([0.0, 1.0]), 3, 1, 1e-3), [1e-3, 1.0])


def _chain(n, rho, target, kind, rmin=1.5):
    rf = design.density_filter(n, rho, rmin)
    k = design.simp(rf, 3.0, 1.0, 1e-3)
    h = fem.homogenize(n, k, tol=1e-14)
    g, dg = design.objective(h["kappa"], target, kind)
    return g, dg, rf, h


@pytest.mark.parametrize("kind", ["mse", "fracmse", "l1"])
def test_sensitivity_matches_central_differences(kind):
    n = 4
    rng = np.random.default_rng(5)
    rho = rng.uniform(0.2, 0.8, n ** 3)
    target = (0.3, 0.2, 0.1, 0.1, 0.05, 0.05)
    g, dg, rf, h = _chain(n, rho, target, kind)
    _, s = design.sensitivity(n, rf, h["E"], dg, 3.0, 1.0, 1e-3, 1.5)
    step = 1e-6
    for j in rng.choice(n ** 3, size=6, replace=False):
        rp, rm = rho.copy(), rho.copy()
        rp[j] += step
        rm[j] -= step
        fd = (_chain(n, rp, target, kind)[0] - _chain(n, rm, target, kind)[0]) / (2 * step)
        assert abs(fd - s[j]) <= 1e-5 * np.max(np.abs(s)), (j, fd, s[j])


def test_kappa_component_sensitivity_fd():
    n = 5
    rng = np.random.default_rng(6)
    rho = rng.uniform(0.2, 0.8, n ** 3)
    _, _, rf, h = _chain(n, rho, (0,) * 6, "mse", rmin=2.0)
    step = 1e-6
    j = 37
    for c in range(6):
        unit = np.zeros(6)
        unit[c] = 1.0
        _, s = design.sensitivity(n, rf, h["E"], unit, 3.0, 1.0, 1e-3, 2.0)
        rp, rm = rho.copy(), rho.copy()
        rp[j] += step
        rm[j] -= step
        kp = _chain(n, rp, (0,) * 6, "mse", rmin=2.0)[3]["kappa"][c]
        km = _chain(n, rm, (0,) * 6, "mse", rmin=2.0)[3]["kappa"][c]
        fd = (kp - km) / (2 * step)
        assert abs(fd - s[j]) <= 1e-5 * np.max(np.abs(s)) + 1e-13


def _oc_exact(rho, s, vstar, move, damp, rho_min):
    """Exact OC solution: with mu = lambda^-eta the volume is piecewise linear
    in mu with breakpoints lo/c and hi/c; sort them and solve on the segment."""
    lo = np.maximum(rho_min, rho - move)
    hi = np.minimum(1.0, rho + move)
    B = np.maximum(0.0, -s)
    c = rho * B ** damp
    grow = c > 0
    N = rho.size
    full = np.where(grow, hi, lo)
    if full.sum() <= vstar * N:
        return full
    if lo.sum() > vstar * N:
        return lo
    bps = np.sort(np.concatenate([lo[grow] / c[grow], hi[grow] / c[grow]]))

    def vol(mu):
        return np.where(grow, np.clip(c * mu, lo, hi), lo).sum()

    target = vstar * N
    vals = np.array([vol(m) for m in bps])
    k = np.searchsorted(vals, target, side="right")   # vals[k-1] <= target < vals[k]
    a, b = bps[k - 1], bps[k]
    va, vb = vals[k - 1], vals[k]
    mu = a + (target - va) * (b - a) / (vb - va)
    return np.where(grow, np.clip(c * mu, lo, hi), lo)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_oc_against_exact_breakpoint_solution(seed):
    rng = np.random.default_rng(seed)
    N = 300
    rho = rng.uniform(0.0, 1.0, N)
    s = rng.standard_normal(N) * 10.0 ** rng.uniform(-3, 1, N)
    if seed < 2:
        s = -np.abs(s) * (rng.uniform(size=N) < 0.8) + np.abs(s) * 0.01
    vstar = float(rho.mean() + rng.uniform(-0.03, 0.0))
    new, lam = design.oc_update(rho, s, vstar, 0.05, 0.5, 1e-3)
    ref = _oc_exact(rho, s, vstar, 0.05, 0.5, 1e-3)
    assert np.max(np.abs(new - ref)) < 1e-9
    lo = np.maximum(1e-3, rho - 0.05)
    hi = np.minimum(1.0, rho + 0.05)
    assert np.all(new >= lo - 1e-15) and np.all(new <= hi + 1e-15)
    assert new.mean() <= vstar + 1e-12
    full = np.where(s < 0, hi, lo).mean()
    active = full > vstar and lo.mean() <= vstar
    if seed < 2:
        assert active
    if active:
        assert abs(new.mean() - vstar) < 1e-9


def test_oc_zero_density_stays_at_lower_bound():
    """rho = 0 gives a zero update factor for every lambda, so the element
    takes its lower bound even when the constraint is inactive."""
    rho = np.array([0.0, 0.5])
    s = np.array([-1.0, -1.0])
    new, lam = design.oc_update(rho, s, 1.0, 0.05, 0.5, 1e-3)
    assert lam == 0.0
    assert np.allclose(new, [1e-3, 0.55])


def test_oc_inactive_and_infeasible():
    rho = np.array([0.2, 0.5, 0.9, 0.0005])
    s = np.array([-1.0, 2.0, -0.5, -3.0])
    new, lam = design.oc_update(rho, s, 1.0, 0.05, 0.5, 1e-3)
    assert lam == 0.0
    assert np.allclose(new, [0.25, 0.45, 0.95, 0.0505])
    new, lam = design.oc_update(rho, s, 0.0, 0.05, 0.5, 1e-3)
    assert math.isinf(lam)
    assert np.allclose(new, [0.15, 0.45, 0.85, 1e-3])


def test_oc_volume_monotone_in_lambda():
    rng = np.random.default_rng(9)
    rho = rng.uniform(0, 1, 200)
    s = -np.abs(rng.standard_normal(200))
    lo = np.maximum(1e-3, rho - 0.05)
    hi = np.minimum(1.0, rho + 0.05)
    vols = [np.clip(rho * (-s / lam) ** 0.5, lo, hi).mean() for lam in np.logspace(-4, 4, 50)]
    assert np.all(np.diff(vols) <= 1e-15)


def test_governor_hand_trace():
    rows = []
    with open(os.path.join(GOLDEN, "governor_trace.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    gov = design.Governor()
    for g, low, vol, vstar, df, count in rows:
        gov.update(g, low, vol)
        assert abs(gov.vstar - vstar) < 1e-14, (g, gov.vstar, vstar)
        assert abs(gov.df - df) < 1e-14
        assert gov.count == int(count)


def test_objectives():
    kap = np.array([0.29, 0.21, 0.1, 0.0, 0.05, 0.06])
    tgt = np.array([0.3, 0.2, 0.1, 0.1, 0.05, 0.05])
    g, dg = design.objective(kap, tgt, "mse")
    assert abs(g - (0.01 ** 2 + 0.01 ** 2 + 0.1 ** 2 + 0.01 ** 2)) < 1e-15
    g, dg = design.objective(kap, tgt, "l1")
    assert abs(g - 0.13) < 1e-15 and dg[2] == 0.0 and dg[4] == 0.0
    g, _ = design.objective(kap, tgt, "fracmse")
    want = (0.29 / 0.3 - 1) ** 2 + (0.21 / 0.2 - 1) ** 2 + 1.0 + (0.06 / 0.05 - 1) ** 2
    assert abs(g - want) < 1e-14


def test_central_symmetry_pairs():
    n = 4
    a = np.arange(n ** 3, dtype=float)
    sym = design.central_symmetrize(n, a)
    # (x,y,z) and (n-1-x, n-1-y, n-1-z) have indices e and N-1-e
    assert np.allclose(sym, sym[::-1])
    assert np.allclose(sym, (n ** 3 - 1) / 2)


def test_design_steps_keep_bounds():
    n = 4
    rho0 = 0.3 + np.random.default_rng(0).uniform(-0.05, 0.05, n ** 3)
    p = design.DesignParams(n=n, kappa_target=(0.1, 0.1, 0.1, 0, 0, 0), rmin=1.5)
    d = design.Design(p, rho0)
    prev = d.rho.copy()
    for _ in range(4):
        info = d.step()
        assert np.all(d.rho >= np.maximum(1e-3, prev - 0.05) - 1e-15)
        assert np.all(d.rho <= np.minimum(1.0, prev + 0.05) + 1e-15)
        assert d.rho.mean() <= info["vstar"] + 1e-12
        prev = d.rho.copy()
    # the target is above the initial conductivity: every element grows
    assert info["kappa"][0] > 0.03
