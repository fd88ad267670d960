"""Pins of the oracle's MMA (oracle/mma.py) against what the method fixes:
the approximation reproduces the value and gradient at the expansion point,
the subproblem's solution is the constrained optimum a general solver finds,
the iteration reaches a closed-form optimum, and the asymptote rule matches
a hand trace."""
import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import mma


def _setup(seed, n=8, k=0):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.2, 0.8, n)
    xmin, xmax = np.zeros(n), np.ones(n)
    x1 = np.clip(x + rng.uniform(-0.1, 0.1, n), 0, 1)
    x2 = np.clip(x1 + rng.uniform(-0.1, 0.1, n), 0, 1)
    L0, U0 = x1 - rng.uniform(0.1, 0.5, n), x1 + rng.uniform(0.1, 0.5, n)
    L, U = mma.asymptotes(k, x, x1, x2, L0, U0, xmin, xmax)
    return rng, x, L, U, xmin, xmax


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("k", [0, 3])
def test_approximation_matches_value_and_gradient(seed, k):
    """f~(x^k) = f(x^k) and grad f~(x^k) = grad f(x^k), the gradient by
    central differences of the approximation itself, for gradients of both
    signs (a swapped p / q or a misplaced 1.001 fails this)."""
    rng, x, L, U, xmin, xmax = _setup(seed, k=k)
    df = rng.standard_normal(x.size) * 10.0 ** rng.uniform(-3, 1, x.size)
    f = 0.37
    p, q = mma.approximation(x, L, U, df, xmin, xmax)
    r = f - np.sum(p / (U - x) + q / (x - L))
    assert abs(mma.approx_value(x, p, q, L, U, r) - f) <= 1e-13
    h = 1e-6
    for j in range(x.size):
        e = np.zeros_like(x)
        e[j] = h
        fd = (mma.approx_value(x + e, p, q, L, U, r) - mma.approx_value(x - e, p, q, L, U, r)) / (2 * h)
        assert abs(fd - df[j]) <= 1e-6 * max(1.0, abs(df[j])), (j, fd, df[j])
    # convex on (L, U): second derivative 2p/(U-x)^3 + 2q/(x-L)^3 > 0
    assert np.all(2 * p / (U - x) ** 3 + 2 * q / (x - L) ** 3 > 0)


def _subproblem(seed, f1):
    rng, x, L, U, xmin, xmax = _setup(seed, k=3)
    alpha, beta = mma.move_limits(x, L, U, xmin, xmax)
    df0 = np.full(x.size, 1.0 / x.size)
    df1 = rng.standard_normal(x.size)
    p0, q0 = mma.approximation(x, L, U, df0, xmin, xmax)
    p1, q1 = mma.approximation(x, L, U, df1, xmin, xmax)
    r1 = f1 - np.sum(p1 / (U - x) + q1 / (x - L))
    return x, L, U, alpha, beta, p0, q0, p1, q1, r1


@pytest.mark.parametrize("seed", [4, 5, 6])
@pytest.mark.parametrize("regime,f1", [("inactive", -1e6), ("active", 0.05), ("infeasible", 1e4)])
@pytest.mark.parametrize("d", [1.0, 2.5])
def test_subproblem_is_the_constrained_optimum(seed, regime, f1, d):
    """The subproblem min f~0(x) + c y + d y^2 / 2 s.t. f~1(x) - y <= 0,
    alpha <= x <= beta, y >= 0 is convex, so the KKT conditions, written from
    the primal definitions (not from the dual route's closed form), prove the
    dual route's point optimal: stationarity in each x_j (zero inside the
    limits, the right sign at them), y = max(0, (lambda - c) / d), primal
    feasibility and complementary slackness.  Inactive: lambda = 0; active:
    0 < lambda < c, f~1 = 0; infeasible: lambda > c, y > 0.  A general
    constrained solver (trust-constr) agrees to its own accuracy."""
    c = 1000.0
    x, L, U, alpha, beta, p0, q0, p1, q1, r1 = _subproblem(seed, f1)
    xs, lam, y = mma.solve_subproblem(p0, q0, p1, q1, r1, L, U, alpha, beta, c, d)
    n = x.size
    g1 = mma.approx_value(xs, p1, q1, L, U, r1)
    if regime == "inactive":
        assert lam == 0.0 and y == 0.0 and g1 < 0
    elif regime == "active":
        assert 0.0 < lam < c and y == 0.0 and abs(g1) <= 1e-12 * max(1.0, abs(r1))
    else:
        assert lam > c and y > 0.0 and abs(g1 - y) <= 1e-9 * y
    assert lam >= 0.0 and g1 - y <= 1e-12 * max(1.0, abs(r1))          # dual and primal feasibility
    assert abs(lam * (g1 - y)) <= 1e-9 * max(1.0, lam) * max(1.0, abs(r1))   # complementary slackness
    # stationarity in y: d/dy (c y + d y^2 / 2 - lambda y) = 0 where y > 0, >= 0 at y = 0
    if y > 0.0:
        assert abs(c + d * y - lam) <= 1e-12 * lam
    else:
        assert c - lam >= 0.0
    # stationarity in x: d/dx_j of f~0 + lambda f~1 from the primal terms
    grad = (p0 + lam * p1) / (U - xs) ** 2 - (q0 + lam * q1) / (xs - L) ** 2
    scale = (p0 + lam * p1) / (U - xs) ** 2
    inner = (xs > alpha + 1e-12) & (xs < beta - 1e-12)
    assert np.all(np.abs(grad[inner]) <= 1e-9 * scale[inner])
    assert np.all(grad[xs <= alpha + 1e-12] >= -1e-12 * scale[xs <= alpha + 1e-12])
    assert np.all(grad[xs >= beta - 1e-12] <= 1e-12 * scale[xs >= beta - 1e-12])

    def obj(v):
        return np.sum(p0 / (U - v[:n]) + q0 / (v[:n] - L)) + c * v[n] + 0.5 * d * v[n] ** 2

    def con(v):
        return -(mma.approx_value(v[:n], p1, q1, L, U, r1) - v[n])

    import warnings
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        res = minimize(obj, np.concatenate([0.5 * (alpha + beta), [max(1.0, f1)]]), method="trust-constr",
                       constraints=[{"type": "ineq", "fun": con}], bounds=list(zip(alpha, beta)) + [(0.0, None)],
                       options={"gtol": 1e-12, "xtol": 1e-14, "maxiter": 5000})
    assert np.max(np.abs(xs - res.x[:n])) <= 1e-3


def test_iteration_reaches_the_closed_form_optimum():
    """min sum x s.t. sum c_j / x_j^3 <= 1 on [1, 10] (a cantilever-type
    problem): stationarity 1 = 3 lambda c_j / x_j^4 and the active constraint
    give x*_j = c_j^(1/4) (sum_k c_k^(1/4))^(1/3) and
    lambda* = (sum_k c_k^(1/4))^(4/3) / 3."""
    c = np.array([61.0, 37.0, 7.0, 3.0, 1.0])
    s4 = np.sum(c ** 0.25)
    xstar = c ** 0.25 * s4 ** (1.0 / 3.0)
    x = np.full(c.size, 5.0)
    st = mma.MmaState(x)
    for _ in range(40):
        f1 = float(np.sum(c / x ** 3) - 1.0)
        x, lam = st.step(x, np.ones_like(x), f1, -3.0 * c / x ** 4, xmin=1.0, xmax=10.0)
    assert np.max(np.abs(x - xstar)) <= 1e-12, (x, xstar)
    assert abs(lam - s4 ** (4.0 / 3.0) / 3.0) <= 1e-12 * lam


def test_asymptote_rule_hand_trace():
    """Iteration 2 from hand-chosen iterates: the same-sign variable widens
    (1.2), the opposite-sign one narrows (0.7), the still one keeps its
    distances (1.0), and a too-close lower asymptote is pushed to x - 0.01."""
    x2 = np.array([0.5, 0.5, 0.5, 0.5])
    x1 = np.array([0.6, 0.6, 0.6, 0.5])
    x = np.array([0.7, 0.55, 0.6, 0.5])
    L0 = np.array([0.3, 0.4, 0.2, 0.49999])
    U0 = np.array([0.9, 0.8, 1.0, 0.8])
    L, U = mma.asymptotes(2, x, x1, x2, L0, U0, np.zeros(4), np.ones(4))
    assert np.allclose(L, [0.34, 0.41, 0.2, 0.49], atol=1e-15)
    assert np.allclose(U, [1.06, 0.69, 1.0, 0.8], atol=1e-15)
    L, U = mma.asymptotes(1, x, x1, x2, L0, U0, np.zeros(4), np.ones(4))
    assert np.allclose(L, x - 0.5) and np.allclose(U, x + 0.5)
    # move limits: alpha = max(0, L + 0.1 (x - L), x - 0.5), beta = min(1, U - 0.1 (U - x), x + 0.5)
    al, be = mma.move_limits(np.array([0.7]), np.array([0.34]), np.array([1.06]), np.zeros(1), np.ones(1))
    assert np.allclose(al, [0.376]) and np.allclose(be, [1.0])
    al, be = mma.move_limits(np.array([0.1]), np.array([-0.4]), np.array([0.6]), np.zeros(1), np.ones(1))
    assert np.allclose(al, [0.0]) and np.allclose(be, [0.55])


def test_model2_first_iteration_is_constraint_driven():
    """From a design far from the target (g >> eps) the first MMA step of
    Eq. model2 has an active or violated constraint (lambda > 0), keeps rho in
    [0, 1] and lowers g."""
    from oracle import design
    import workloads as W
    n = 6
    p = design.DesignParams(n=n, kappa_target=W.TARGET_ISOTROPIC, optimizer="mma", cg_tol=1e-12)
    d = design.Design(p, W.initial_density(n, 0.3, 3))
    r0 = d.step()
    assert r0["g"] > p.mma_eps and r0["lam"] > 0.0
    assert np.all(d.rho >= 0.0) and np.all(d.rho <= 1.0)
    r1 = d.step()
    assert r1["g"] < r0["g"]
