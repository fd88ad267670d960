"""FP64 design loop of the paper: filter, SIMP, objective, sensitivity, OC
update with the adaptive volume bound.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Readings of points where the paper is silent or garbled:

* Filter weight (Sec. 2.3): d_e(x_i, r) = max(0, r - |x_i - x_e|) over voxel
  centroids at minimum-image periodic distance, neighbourhood |x_i - x_e| < r,
  unit voxel volumes.
* SIMP (Sec. 2.2): k_e = k_min + rho~_e^p (k_0 - k_min).
* Sensitivity (Eq. sens): exact derivative of the discrete Eq. homo,
  d kappa_ij / d rho~_e = (1/|Omega|) p rho~_e^(p-1) (k_0 - k_min) E_ij,e
  (the paper's printed formula writes kappa^0 for (k_0 - k_min), adds a
  spurious sum over e and drops K^0); then the chain rule through the filter,
  dg/drho = W^T dg/drho~ (no extra sensitivity filter).
* OC (Sec. 3.3, OCOptimizer(min_density, stepLimit, dampExponent)):
  rho_new = clamp(rho * (max(0, -dg/drho) / lambda)^eta, max(rho_min, rho - m),
  min(1, rho + m)); lambda solves mean(rho_new) = V* by bisection.  If the
  volume with every growing element at its upper bound is already <= V* the
  constraint is inactive and that limit is taken; if even the all-lower-bound
  volume exceeds V*, every element takes its lower bound.
* Alg. 1 thresholds: bound = 1e-4, is_small(dg) = |dg| < 1e-3 g,
  is_big(g) = g > bound, is_small(V - V*) = |V - V*| < 1e-2, gap = 0 before
  its first assignment, lowBound = mean(rho~^p), V* clamped to [0, 1].

Parity: pinned -- filter (mean preservation, adjointness, brute force),
sensitivity (central finite differences through the whole chain), OC
(brute-force exact lambda from sorted breakpoints, bound and volume
invariants), Alg. 1 (hand-traced scripted sequences).  See
tests/test_oracle_design.py.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

from . import fem


# ----------------------------------------------------------------------------
# Density filter (Sec. 2.3)
# ----------------------------------------------------------------------------

def filter_offsets(rmin: float):
    """List of (dx, dy, dz, w) with w = r - |o| > 0 for |o| < r."""
    R = int(math.ceil(rmin))
    out = []
    for dz in range(-R, R + 1):
        for dy in range(-R, R + 1):
            for dx in range(-R, R + 1):
                d = math.sqrt(dx * dx + dy * dy + dz * dz)
                if d < rmin:
                    out.append((dx, dy, dz, rmin - d))
    return out


def _index(n: int, x, y, z):
    return (x % n) + n * ((y % n) + n * (z % n))


def density_filter(n: int, rho: np.ndarray, rmin: float) -> np.ndarray:
    """rho~_e = sum_i d_e(x_i, r) v_i rho_i / sum_i d_e(x_i, r) v_i over the
    periodic neighbourhood N_e (Sec. 2.3), v_i = 1."""
    offs = filter_offsets(rmin)
    wsum = sum(w for (_, _, _, w) in offs)
    r = np.arange(n)
    Z, Y, X = np.meshgrid(r, r, r, indexing="ij")
    X, Y, Z = X.ravel(), Y.ravel(), Z.ravel()
    out = np.zeros(n ** 3)
    for dx, dy, dz, w in offs:
        out += w * rho[_index(n, X + dx, Y + dy, Z + dz)]
    return out / wsum


def density_filter_transpose(n: int, s: np.ndarray, rmin: float) -> np.ndarray:
    """W^T s, written as the scatter of each element's value to the
    neighbours it was gathered from: (W^T s)_i = sum_e W_ei s_e."""
    offs = filter_offsets(rmin)
    wsum = sum(w for (_, _, _, w) in offs)
    r = np.arange(n)
    Z, Y, X = np.meshgrid(r, r, r, indexing="ij")
    X, Y, Z = X.ravel(), Y.ravel(), Z.ravel()
    out = np.zeros(n ** 3)
    for dx, dy, dz, w in offs:
        np.add.at(out, _index(n, X + dx, Y + dy, Z + dz), w * s)
    return out / wsum


# ----------------------------------------------------------------------------
# SIMP (Sec. 2.2)
# ----------------------------------------------------------------------------

def simp(rho_f: np.ndarray, penal: float, k_solid: float, k_void: float) -> np.ndarray:
    return k_void + rho_f ** penal * (k_solid - k_void)


def simp_derivative(rho_f: np.ndarray, penal: float, k_solid: float, k_void: float) -> np.ndarray:
    return penal * rho_f ** (penal - 1.0) * (k_solid - k_void)


# ----------------------------------------------------------------------------
# Objectives (Eq. mse, Eq. fracmse, Eq. l1) on the 6-vector of Eq. rep
# ----------------------------------------------------------------------------

def objective(kappa, target, kind: str = "mse"):
    """Returns (g, dg/dkappa_c) for c over the six components of Eq. rep.

    fracmse divides by the target component; a zero target component is
    scored by its plain squared error (the paper's formula is undefined
    there).  l1 uses d|a|/da = 0 at a = 0 (Sec. 4.4)."""
    kappa = np.asarray(kappa, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    if kind == "mse":
        d = kappa - target
        return float((d * d).sum()), 2.0 * d
    if kind == "fracmse":
        g, dg = 0.0, np.zeros(6)
        for c in range(6):
            if target[c] != 0.0:
                a = kappa[c] / target[c] - 1.0
                g += a * a
                dg[c] = 2.0 * a / target[c]
            else:
                g += kappa[c] ** 2
                dg[c] = 2.0 * kappa[c]
        return float(g), dg
    if kind == "l1":
        d = kappa - target
        return float(np.abs(d).sum()), np.sign(d)
    raise ValueError(kind)


# ----------------------------------------------------------------------------
# Sensitivity (Eq. sens with the chain rule of Sec. 2.3)
# ----------------------------------------------------------------------------

def sensitivity(n: int, rho_f: np.ndarray, E: np.ndarray, dg_dkappa: np.ndarray,
                penal: float, k_solid: float, k_void: float, rmin: float):
    """dg/drho = W^T [ sum_c dg/dkappa_c * d kappa_c / d rho~ ] with
    d kappa_c / d rho~_e = (1/|Omega|) k'(rho~_e) E[c, e].
    Returns (dg/drho~, dg/drho)."""
    N = n ** 3
    dk = simp_derivative(rho_f, penal, k_solid, k_void)
    s_f = (dg_dkappa[:, None] * E).sum(axis=0) * dk / N
    return s_f, density_filter_transpose(n, s_f, rmin)


def central_symmetrize(n: int, a: np.ndarray) -> np.ndarray:
    """Average of each element with its point-symmetric partner about the
    cell centre, (x, y, z) <-> (n-1-x, n-1-y, n-1-z) (Sec. 4.1)."""
    return 0.5 * (a + a[::-1])


# ----------------------------------------------------------------------------
# OC update (Sec. 3.3)
# ----------------------------------------------------------------------------

def oc_update(rho: np.ndarray, s: np.ndarray, vstar: float, move: float, damp: float,
              rho_min: float, rel_tol: float = 1e-14, max_bisect: int = 400):
    """Optimality-criteria step.  Returns (rho_new, lambda); lambda = 0 marks
    the inactive-constraint limit and +inf the all-lower-bound case."""
    lo = np.maximum(rho_min, rho - move)
    hi = np.minimum(1.0, rho + move)
    B = np.maximum(0.0, -s)

    def new(lam):
        return np.clip(rho * (B / lam) ** damp, lo, hi)

    grow = (B > 0.0) & (rho > 0.0)       # elements whose update factor is non-zero
    v_full = np.where(grow, hi, lo).mean()
    if v_full <= vstar:
        return np.where(grow, hi, lo), 0.0
    if lo.mean() > vstar:
        return lo.copy(), math.inf
    c = rho[grow] * B[grow] ** damp
    # every breakpoint of lambda -> mean(new(lambda)) lies in [lam_a, lam_b]
    lam_a = float(np.min((c / hi[grow]) ** (1.0 / damp)))
    lam_b = float(np.max((c / lo[grow]) ** (1.0 / damp)))
    lam_a *= 0.5
    lam_b *= 2.0
    for _ in range(max_bisect):
        if lam_b - lam_a <= rel_tol * lam_b:
            break
        mid = math.sqrt(lam_a * lam_b)
        if mid <= lam_a or mid >= lam_b:
            break
        if new(mid).mean() > vstar:
            lam_a = mid
        else:
            lam_b = mid
    return new(lam_b), lam_b


# ----------------------------------------------------------------------------
# Adaptive volume bound (Alg. 1)
# ----------------------------------------------------------------------------

@dataclass
class Governor:
    bound: float = 1e-4
    small_rel: float = 1e-3
    vol_tol: float = 1e-2
    df: float = 1.0
    vstar: float = 1.0
    count: int = 0
    g_prev: float = 1.0
    gap: float = 0.0

    def update(self, g: float, low_bound: float, vol: float) -> float:
        """One pass of the loop body of Alg. 1 after InvHomo() produced g."""
        if g <= self.bound:
            self.gap = self.vstar - low_bound
            self.vstar = self.vstar - self.gap * self.df
            self.df = 0.8 * self.df
        cond1 = abs(self.g_prev - g) < self.small_rel * g
        cond2 = g > self.bound
        cond3 = abs(vol - self.vstar) < self.vol_tol
        if cond1 and cond2 and cond3:
            self.count += 1
        else:
            self.count = 0
        if self.count >= 5:
            self.vstar = self.vstar + 0.3 * self.gap * self.df
            self.count = 0
        self.vstar = min(1.0, max(0.0, self.vstar))
        self.g_prev = g
        return self.vstar


# ----------------------------------------------------------------------------
# One design iteration (Alg. 2 with the loop of Sec. 3.4, model of Eq. model3)
# ----------------------------------------------------------------------------

@dataclass
class DesignParams:
    n: int
    kappa_target: tuple
    penal: float = 3.0
    rmin: float = 1.5
    k_solid: float = 1.0
    k_void: float = 1e-3
    move: float = 0.05
    damp: float = 0.5
    rho_min: float = 1e-3
    cg_tol: float = 1e-12
    governor: bool = True
    fixed_volume: float = 1.0
    objective: str = "mse"
    symmetry: bool = False
    warm_start: bool = True
    optimizer: str = "oc"       # "oc": Eq. model3 / model1 by OC; "mma": Eq. model2 by MMA (oracle.mma)
    mma_eps: float = 1e-4       # eps of Eq. model2's constraint g <= eps
    mma_move: float = 0.5
    mma_c: float = 1000.0
    mma_d: float = 1.0


class Design:
    """State of the oracle's design loop: rho, the previous solution (warm
    start) and the Alg. 1 governor."""

    def __init__(self, params: DesignParams, rho0: np.ndarray):
        self.p = params
        self.rho = np.asarray(rho0, dtype=np.float64).copy()
        self.chi = None
        self.gov = Governor()
        if not params.governor:
            self.gov.vstar = params.fixed_volume
        self.iteration = 0
        self.mma = None
        if params.optimizer == "mma":
            from .mma import MmaState
            self.mma = MmaState(self.rho)

    def step(self):
        p = self.p
        n = p.n
        rho_f = density_filter(n, self.rho, p.rmin)
        k = simp(rho_f, p.penal, p.k_solid, p.k_void)
        h = fem.homogenize(n, k, tol=p.cg_tol,
                           chi0=self.chi if p.warm_start else None)
        self.chi = h["chi"]
        kappa = h["kappa"]
        g, dg = objective(kappa, p.kappa_target, p.objective)
        _, s = sensitivity(n, rho_f, h["E"], dg, p.penal, p.k_solid, p.k_void, p.rmin)
        low_bound = float((rho_f ** p.penal).mean())
        vol = float(self.rho.mean())
        if p.optimizer == "mma":
            vstar = 0.0
        elif p.governor:
            vstar = self.gov.update(g, low_bound, vol)
        else:
            vstar = p.fixed_volume
        rho = self.rho
        if p.symmetry:
            rho = central_symmetrize(n, rho)
            s = central_symmetrize(n, s)
        if p.optimizer == "mma":
            # Eq. model2: f0 = V = mean(rho~), df0/drho = W^T (1/N); f1 = g - eps
            N = rho.size
            df0 = density_filter_transpose(n, np.full(N, 1.0 / N), p.rmin)
            rho_new, lam = self.mma.step(rho, df0, g - p.mma_eps, s, move=p.mma_move, c=p.mma_c, d=p.mma_d)
        else:
            rho_new, lam = oc_update(rho, s, vstar, p.move, p.damp, p.rho_min)
        self.rho = rho_new
        self.iteration += 1
        return dict(g=g, kappa=kappa, vstar=vstar, lam=lam, mean_rho=vol,
                    mean_rhop=low_bound, iters=h["iters"], resid=h["resid"],
                    rho_f=rho_f, s=s, k=k)
