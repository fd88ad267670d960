"""Method of Moving Asymptotes for the paper's model 2 (Sec. 2.3, Eq. model2):

    min_rho V(rho)  s.t.  K(rho) T = f,  g(kappa^H(rho), kappa*) <= eps,  0 <= rho <= 1,

which the paper solves with MMA (Svanberg 1987) through its class
MMAOptimizer(nconstraint, nvar, a0, a, c, d) (Sec. 3.3) and reports with g
below 1e-4 (Sec. 5, "Different solvers").

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper names the method and the constructor's parameters but prints no
formulas, so this module follows Svanberg's published method; the readings:

* Standard form with one constraint (m = 1): minimise
  f0(x) + a0 z + c y + d y^2 / 2 subject to f1(x) - a z - y <= 0,
  xmin <= x <= xmax, y >= 0, z >= 0, with a = 0 (so z = 0 at the optimum and
  a0 plays no part), c = 1000, d = 1.
* Moving asymptotes: in the first two iterations L = x - s0 (xmax - xmin),
  U = x + s0 (xmax - xmin) with s0 = 0.5; afterwards, per variable,
  gamma = 1.2 where x^k - x^(k-1) and x^(k-1) - x^(k-2) have the same sign,
  0.7 where they have opposite signs and 1 where either is zero, and
  L = x - gamma (x^(k-1) - L^(k-1)), U = x + gamma (U^(k-1) - x^(k-1)),
  each kept between 0.01 and 10 times (xmax - xmin) away from x.
* Move limits: alpha = max(xmin, L + 0.1 (x - L), x - move (xmax - xmin)),
  beta = min(xmax, U - 0.1 (U - x), x + move (xmax - xmin)), move = 0.5.
* Convex separable approximation of f_i at x^k:
  p_ij = (U_j - x_j)^2 (1.001 (df_i/dx_j)^+ + 0.001 (df_i/dx_j)^- + 1e-5 / (xmax_j - xmin_j)),
  q_ij = (x_j - L_j)^2 (0.001 (df_i/dx_j)^+ + 1.001 (df_i/dx_j)^- + 1e-5 / (xmax_j - xmin_j)),
  f~_i(x) = r_i + sum_j (p_ij / (U_j - x_j) + q_ij / (x_j - L_j)), with r_i
  chosen so that f~_i(x^k) = f_i(x^k); then df~_i/dx_j = df_i/dx_j at x^k.
* Subproblem through its dual in the one multiplier lambda >= 0: for fixed
  lambda each x_j minimises (p_0j + lambda p_1j) / (U_j - x) +
  (q_0j + lambda q_1j) / (x - L_j) over [alpha_j, beta_j], i.e. the clamp of
  (sqrt(P) L_j + sqrt(Q) U_j) / (sqrt(P) + sqrt(Q)); y = max(0, (lambda - c) / d).
  The dual derivative phi(lambda) = f~_1(x(lambda)) - y(lambda) is
  non-increasing: lambda* = 0 when phi(0) <= 0, else its root.
* Model 2 (Eq. model2): x = rho, f0 = V(rho) = mean of the filtered density
  (equal to mean(rho): the periodic filter preserves the mean),
  df0/drho = W^T (1/N) = 1/N, f1 = g - eps with eps = 1e-4, df1/drho = dg/drho.

Parity: pinned -- the approximation's value and gradient at x^k (finite
differences), the subproblem's solution against a general constrained
solver on small problems in every regime (inactive, active, infeasible),
an analytic problem whose optimum is known in closed form, and a
hand-traced asymptote sequence.  See tests/test_oracle_mma.py.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq

ASYINIT = 0.5
ASYINCR = 1.2
ASYDECR = 0.7
ALBEFA = 0.1
MOVE = 0.5
RAA0 = 1e-5


def asymptotes(k: int, x, x1, x2, L_old, U_old, xmin, xmax, s0: float = ASYINIT):
    """Asymptotes of iteration k (0-based) from the two previous iterates."""
    span = xmax - xmin
    if k < 2:
        return x - s0 * span, x + s0 * span
    t = (x - x1) * (x1 - x2)
    gamma = np.where(t > 0, ASYINCR, np.where(t < 0, ASYDECR, 1.0))
    L = x - gamma * (x1 - L_old)
    U = x + gamma * (U_old - x1)
    L = np.minimum(np.maximum(L, x - 10.0 * span), x - 0.01 * span)
    U = np.maximum(np.minimum(U, x + 10.0 * span), x + 0.01 * span)
    return L, U


def move_limits(x, L, U, xmin, xmax, move: float = MOVE):
    span = xmax - xmin
    alpha = np.maximum(np.maximum(xmin, L + ALBEFA * (x - L)), x - move * span)
    beta = np.minimum(np.minimum(xmax, U - ALBEFA * (U - x)), x + move * span)
    return alpha, beta


def approximation(x, L, U, df, xmin, xmax):
    """(p, q) of one function's convex separable approximation at x."""
    pos = np.maximum(df, 0.0)
    neg = np.maximum(-df, 0.0)
    reg = RAA0 / (xmax - xmin)
    p = (U - x) ** 2 * (1.001 * pos + 0.001 * neg + reg)
    q = (x - L) ** 2 * (0.001 * pos + 1.001 * neg + reg)
    return p, q


def approx_value(xv, p, q, L, U, r):
    """f~(xv) = r + sum_j p_j / (U_j - xv_j) + q_j / (xv_j - L_j)."""
    return r + float(np.sum(p / (U - xv) + q / (xv - L)))


def x_of_lambda(lam, p0, q0, p1, q1, L, U, alpha, beta):
    P = p0 + lam * p1
    Q = q0 + lam * q1
    sp, sq = np.sqrt(P), np.sqrt(Q)
    x = (sp * L + sq * U) / (sp + sq)
    return np.minimum(np.maximum(x, alpha), beta)


def solve_subproblem(p0, q0, p1, q1, r1, L, U, alpha, beta, c: float = 1000.0, d: float = 1.0):
    """(x, lambda, y) of the MMA subproblem with one constraint and a = 0."""
    def phi(lam):
        xl = x_of_lambda(lam, p0, q0, p1, q1, L, U, alpha, beta)
        y = max(0.0, (lam - c) / d)
        return approx_value(xl, p1, q1, L, U, r1) - y

    if phi(0.0) <= 0.0:
        lam = 0.0
    else:
        # f~_1 on the box is at most the sum of its endpoint maxima, so phi < 0
        # beyond c + d * (that bound)
        fmax = r1 + float(np.sum(np.maximum(p1 / (U - alpha) + q1 / (alpha - L),
                                            p1 / (U - beta) + q1 / (beta - L))))
        hi = c + d * max(fmax, 0.0) + 1.0
        lam = brentq(phi, 0.0, hi, xtol=1e-15 * hi, rtol=4 * np.finfo(float).eps, maxiter=500)
    x = x_of_lambda(lam, p0, q0, p1, q1, L, U, alpha, beta)
    return x, lam, max(0.0, (lam - c) / d)


def mma_update(k: int, x, x1, x2, L_old, U_old, df0, f1: float, df1, xmin=0.0, xmax=1.0,
               move: float = MOVE, c: float = 1000.0, d: float = 1.0):
    """One MMA iteration with one constraint f1(x) <= 0.  Returns
    (x_new, L, U, lambda); the caller shifts x2 <- x1 <- x."""
    x = np.asarray(x, dtype=np.float64)
    xmin = np.broadcast_to(np.asarray(xmin, dtype=np.float64), x.shape)
    xmax = np.broadcast_to(np.asarray(xmax, dtype=np.float64), x.shape)
    L, U = asymptotes(k, x, x1, x2, L_old, U_old, xmin, xmax)
    alpha, beta = move_limits(x, L, U, xmin, xmax, move)
    df0 = np.broadcast_to(np.asarray(df0, dtype=np.float64), x.shape)
    p0, q0 = approximation(x, L, U, df0, xmin, xmax)
    p1, q1 = approximation(x, L, U, df1, xmin, xmax)
    r1 = f1 - float(np.sum(p1 / (U - x) + q1 / (x - L)))
    xn, lam, _ = solve_subproblem(p0, q0, p1, q1, r1, L, U, alpha, beta, c, d)
    return xn, L, U, lam


class MmaState:
    """The iterates and asymptotes MMA carries between iterations."""

    def __init__(self, x0):
        x0 = np.asarray(x0, dtype=np.float64)
        self.k = 0
        self.x1 = x0.copy()
        self.x2 = x0.copy()
        self.L = np.zeros_like(x0)
        self.U = np.ones_like(x0)

    def step(self, x, df0, f1, df1, **kw):
        xn, L, U, lam = mma_update(self.k, x, self.x1, self.x2, self.L, self.U, df0, f1, df1, **kw)
        self.x2 = self.x1
        self.x1 = np.asarray(x, dtype=np.float64).copy()
        self.L, self.U = L, U
        self.k += 1
        return xn, lam
