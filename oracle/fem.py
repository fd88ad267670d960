"""FP64 finite-element homogenization of an n^3 periodic voxel unit cell.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Mesh convention.  Unit voxels (h = 1, |Omega| = n^3).  Node (x, y, z) and
element (x, y, z) both have index x + n*(y + n*z).  Element (x, y, z) has the
eight corner nodes ((x+a) % n, (y+b) % n, (z+c) % n) with local number
l = a + 2b + 4c; the paper's "K^0_[7-e, .]" indexing (Sec. 2.4) is this
numbering seen from a vertex, which is local corner 7-e of its e-th incident
element.

Parity: pinned (closed-form K^0, solid/uniform/laminate closed forms,
Voigt-Reuss and Hashin-Shtrikman bounds, cube-group equivariance, dense
direct solve, finite differences) -- see tests/test_oracle_fem.py.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# The six independent components in the paper's vector order (Eq. rep):
# [k11, k22, k33, k12, k23, k13] as (i, j) index pairs.
COMPONENTS = ((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2))


def corner_offset(l: int):
    """(a, b, c) offset of local corner l = a + 2b + 4c."""
    return (l & 1, (l >> 1) & 1, (l >> 2) & 1)


def _shape_grads(xi: np.ndarray) -> np.ndarray:
    """Gradients of the 8 trilinear shape functions of the unit cube at xi."""
    g = np.zeros((8, 3))
    for l in range(8):
        a = corner_offset(l)
        val = [xi[d] if a[d] else 1.0 - xi[d] for d in range(3)]
        der = [1.0 if a[d] else -1.0 for d in range(3)]
        g[l, 0] = der[0] * val[1] * val[2]
        g[l, 1] = val[0] * der[1] * val[2]
        g[l, 2] = val[0] * val[1] * der[2]
    return g


def k0_matrix() -> np.ndarray:
    """Element conductivity matrix K^0 (unit conductivity, unit voxel):
    K^0_ab = integral over the cube of grad N_a . grad N_b, evaluated with
    2x2x2 Gauss-Legendre quadrature (exact for these polynomial integrands).
    This is the "element assembly matrix" of Sec. 2.4."""
    pts = (0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0))
    K = np.zeros((8, 8))
    for x in pts:
        for y in pts:
            for z in pts:
                g = _shape_grads(np.array([x, y, z]))
                K += 0.125 * (g @ g.T)
    return K


def test_temperatures() -> np.ndarray:
    """T^0: nodal values on one element of the three unit-gradient test fields
    x_1, x_2, x_3 (Sec. 2.2, T_e^{0(i)}), relative to the element's lower
    corner: t[l, i] = i-th coordinate of corner l.  Shape (8, 3)."""
    t = np.zeros((8, 3))
    for l in range(8):
        t[l, :] = corner_offset(l)
    return t


def element_nodes(n: int) -> np.ndarray:
    """(n^3, 8) global node indices of each element's corners."""
    r = np.arange(n)
    z, y, x = np.meshgrid(r, r, r, indexing="ij")
    x, y, z = x.ravel(), y.ravel(), z.ravel()
    conn = np.empty((n ** 3, 8), dtype=np.int64)
    for l in range(8):
        a, b, c = corner_offset(l)
        conn[:, l] = ((x + a) % n) + n * (((y + b) % n) + n * ((z + c) % n))
    return conn


def assemble(n: int, k: np.ndarray, K0: np.ndarray | None = None) -> sp.csr_matrix:
    """Global matrix K = sum_e k_e K^0 on the periodic mesh (Eq. ktf, with the
    SIMP conductivity k_e of Sec. 2.2 scaling each element)."""
    if K0 is None:
        K0 = k0_matrix()
    conn = element_nodes(n)
    N = n ** 3
    rows = np.repeat(conn, 8, axis=1).astype(np.int64)          # (N, 64): row = conn[:, a]
    cols = np.tile(conn, (1, 8)).astype(np.int64)               # (N, 64): col = conn[:, b]
    vals = k[:, None] * K0.reshape(1, 64)
    A = sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=(N, N))
    return A.tocsr()


def macro_load(n: int, k: np.ndarray, K0: np.ndarray | None = None) -> np.ndarray:
    """enforceMacroLoad (Sec. 2.4): f^(i)_v = sum over the elements e incident
    to v of k_e * f^0[loc(v, e), i], with the 8x3 template f^0 = K^0 T^0.
    Returns shape (3, n^3)."""
    if K0 is None:
        K0 = k0_matrix()
    conn = element_nodes(n)
    f0 = K0 @ test_temperatures()                                # (8, 3)
    N = n ** 3
    f = np.zeros((3, N))
    for i in range(3):
        contrib = k[:, None] * f0[None, :, i]                    # (N, 8)
        f[i] = np.bincount(conn.ravel(), weights=contrib.ravel(), minlength=N)
    return f


def apply_operator(n: int, k: np.ndarray, u: np.ndarray, K0: np.ndarray | None = None) -> np.ndarray:
    """Matrix-free [KT]_v (Sec. 2.4): for each element, K^0 times its nodal
    values, scaled by k_e and scattered back.  u has shape (m, n^3)."""
    if K0 is None:
        K0 = k0_matrix()
    conn = element_nodes(n)
    u = np.atleast_2d(u)
    out = np.zeros_like(u, dtype=np.float64)
    for i in range(u.shape[0]):
        ue = u[i][conn]                                          # (N, 8)
        contrib = k[:, None] * (ue @ K0.T)                       # (N, 8)
        out[i] = np.bincount(conn.ravel(), weights=contrib.ravel(), minlength=n ** 3)
    return out


def apply_operator_at(n: int, k: np.ndarray, u: np.ndarray, nodes, K0: np.ndarray | None = None) -> np.ndarray:
    """[K u]_v (Sec. 2.4) at the listed nodes only: sum over the eight
    incident elements e of k_e (K^0 u_e)_{loc(v, e)}.  u has shape (m, n^3);
    returns (m, len(nodes)).  For sampled checks on grids too large to
    assemble."""
    if K0 is None:
        K0 = k0_matrix()
    u = np.atleast_2d(u)
    out = np.zeros((u.shape[0], len(nodes)))
    for j, v in enumerate(nodes):
        x, y, z = v % n, (v // n) % n, v // (n * n)
        for l in range(8):                      # v is local corner l of element v - offset(l)
            a, b, c = corner_offset(l)
            ex, ey, ez = (x - a) % n, (y - b) % n, (z - c) % n
            e = ex + n * (ey + n * ez)
            corners = []
            for m in range(8):
                am, bm, cm = corner_offset(m)
                corners.append(((ex + am) % n) + n * (((ey + bm) % n) + n * ((ez + cm) % n)))
            out[:, j] += k[e] * (u[:, corners] @ K0[l, :])
    return out


def gauss_seidel_at(n: int, k: np.ndarray, f: np.ndarray, T: np.ndarray, nodes,
                    K0: np.ndarray | None = None) -> np.ndarray:
    """New values at `nodes` of one Gauss-Seidel relaxation of those nodes
    (Sec. 2.4): T_v = (f_v - M_v) / S_v with S_v = sum over incident
    elements of k_e K^0_{ll} and M_v = [K T]_v - S_v T_v.  Exact for a set of
    mutually uncoupled nodes (one colour); f, T of shape (m, n^3)."""
    if K0 is None:
        K0 = k0_matrix()
    KT = apply_operator_at(n, k, T, nodes, K0)
    out = np.zeros((np.atleast_2d(T).shape[0], len(nodes)))
    for j, v in enumerate(nodes):
        x, y, z = v % n, (v // n) % n, v // (n * n)
        S = 0.0
        for l in range(8):
            a, b, c = corner_offset(l)
            e = ((x - a) % n) + n * (((y - b) % n) + n * ((z - c) % n))
            S += k[e] * K0[l, l]
        M = KT[:, j] - S * np.atleast_2d(T)[:, v]
        out[:, j] = (np.atleast_2d(f)[:, v] - M) / S
    return out


def gauss_seidel_pass(K: sp.csr_matrix, f: np.ndarray, T: np.ndarray, nodes) -> np.ndarray:
    """One Gauss-Seidel relaxation over `nodes` in the given order
    (Sec. 2.4): S_v T_v = f_v - M_v with S_v = K_vv and M_v the row of K
    times T without the diagonal term.  Returns the updated copy of T."""
    T = T.astype(np.float64).copy()
    K = K.tocsr()
    for v in nodes:
        lo, hi = K.indptr[v], K.indptr[v + 1]
        cols, vals = K.indices[lo:hi], K.data[lo:hi]
        diag = vals[cols == v].sum()
        m = vals @ T[cols] - diag * T[v]
        T[v] = (f[v] - m) / diag
    return T


def colour_nodes(n: int, colour: int) -> np.ndarray:
    """Nodes of colour (x%2) + 2(y%2) + 4(z%2) (the 8-colour ordering of
    Sec. 2.4)."""
    r = np.arange(n)
    Z, Y, X = np.meshgrid(r, r, r, indexing="ij")
    c = (X % 2) + 2 * (Y % 2) + 4 * (Z % 2)
    return np.flatnonzero(c.ravel() == colour)


def pcg(K: sp.csr_matrix, f: np.ndarray, tol: float = 1e-12, maxit: int | None = None,
        x0: np.ndarray | None = None, observe=None):
    """Jacobi-preconditioned CG for the singular periodic system K x = f.

    The constant vector spans the null space of K, so f and every
    preconditioned residual are projected to zero mean, and the returned x is
    zero-mean.  Stops when ||f - K x|| <= tol * ||f|| (an all-zero f returns
    x = 0).  Returns (x, iterations, true relative residual).  observe, if
    given, is called as observe(iterations, ||r|| / ||f||) with the recurrence
    residual the stopping test just computed (for timing; it changes nothing)."""
    N = f.shape[0]
    if maxit is None:
        maxit = 50 * N + 1000
    f = f - f.mean()
    nf = np.linalg.norm(f)
    if nf == 0.0:
        return np.zeros(N), 0, 0.0
    x = np.zeros(N) if x0 is None else (x0 - x0.mean()).astype(np.float64)
    dinv = 1.0 / K.diagonal()
    r = f - K @ x
    z = dinv * r
    z -= z.mean()
    p = z.copy()
    rz = r @ z
    it = 0
    while it < maxit:
        rn = np.linalg.norm(r)
        if observe is not None:
            observe(it, rn / nf)
        if not rn > tol * nf:
            break
        q = K @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        z = dinv * r
        z -= z.mean()
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    x -= x.mean()
    res = np.linalg.norm(f - K @ x) / nf
    return x, it, res


def element_energies(n: int, chi: np.ndarray, K0: np.ndarray | None = None) -> np.ndarray:
    """E[c, e] = (T^0(i) - T^(i))_e^T K^0 (T^0(j) - T^(j))_e for the six
    components c = (i, j) of Eq. rep (the bracket of the discrete form of
    Eq. homo, without the k_e factor).  chi has shape (3, n^3)."""
    if K0 is None:
        K0 = k0_matrix()
    conn = element_nodes(n)
    t = test_temperatures()
    d = [t[None, :, i] - chi[i][conn] for i in range(3)]        # each (N, 8)
    E = np.empty((6, n ** 3))
    for c, (i, j) in enumerate(COMPONENTS):
        E[c] = np.einsum("el,lm,em->e", d[i], K0, d[j])
    return E


def kappa_from_energies(k: np.ndarray, E: np.ndarray) -> np.ndarray:
    """kappa_c = (1/|Omega|) sum_e k_e E[c, e]  (discrete Eq. homo), with
    |Omega| = n^3 voxels.  Returns the 6-vector of Eq. rep."""
    return (E * k[None, :]).sum(axis=1) / k.shape[0]


def kappa_matrix(kv) -> np.ndarray:
    """3x3 symmetric matrix from the 6-vector [k11,k22,k33,k12,k23,k13]."""
    m = np.zeros((3, 3))
    for c, (i, j) in enumerate(COMPONENTS):
        m[i, j] = m[j, i] = kv[c]
    return m


def kappa_vector(m) -> np.ndarray:
    return np.array([m[i, j] for (i, j) in COMPONENTS])


def homogenize(n: int, k: np.ndarray, tol: float = 1e-12, chi0: np.ndarray | None = None,
               maxit: int | None = None):
    """Homogenized conductivity kappa^H of the cell with element
    conductivities k (Sec. 2.2): assemble K, build the three macro loads,
    solve K T^(i) = f^(i) (Eq. kti) and form the discrete Eq. homo.

    Returns dict(kappa=6-vector, chi=(3, N), iters=[3], resid=[3], f=(3, N))."""
    K0 = k0_matrix()
    K = assemble(n, k, K0)
    f = macro_load(n, k, K0)
    chi = np.zeros((3, n ** 3))
    iters, resid = [], []
    for i in range(3):
        x0 = None if chi0 is None else chi0[i]
        chi[i], it, res = pcg(K, f[i], tol=tol, maxit=maxit, x0=x0)
        iters.append(it)
        resid.append(res)
    E = element_energies(n, chi, K0)
    kappa = kappa_from_energies(k, E)
    return dict(kappa=kappa, chi=chi, iters=iters, resid=resid, f=f, E=E)


# --------------------------------------------------------------------------
# Multigrid hierarchy pieces (Alg. 3): trilinear prolongation on the periodic
# vertex grid, restriction R = P^T, Galerkin coarse operators.
# --------------------------------------------------------------------------

def prolongation(nc: int) -> sp.csr_matrix:
    """Trilinear interpolation from the periodic vertex grid of size nc^3 to
    the grid of size (2 nc)^3: fine node 2I + delta takes weight
    prod_d (1 - |delta_d| / 2) from coarse node I, delta in {-1, 0, 1}^3."""
    nf = 2 * nc
    rows, cols, vals = [], [], []
    r = np.arange(nc)
    Z, Y, X = np.meshgrid(r, r, r, indexing="ij")
    X, Y, Z = X.ravel(), Y.ravel(), Z.ravel()
    I = X + nc * (Y + nc * Z)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                w = (1 - abs(dx) / 2) * (1 - abs(dy) / 2) * (1 - abs(dz) / 2)
                fx = (2 * X + dx) % nf
                fy = (2 * Y + dy) % nf
                fz = (2 * Z + dz) % nf
                rows.append(fx + nf * (fy + nf * fz))
                cols.append(I)
                vals.append(np.full(I.shape, w))
    P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nf ** 3, nc ** 3))
    return P.tocsr()


def galerkin(A: sp.csr_matrix, nc: int) -> sp.csr_matrix:
    """Coarse operator R A P with R = P^T."""
    P = prolongation(nc)
    return (P.T @ A @ P).tocsr()


def level_sizes(n: int):
    """Grid sizes of the hierarchy: halve while the size is even and the half
    is at least 4."""
    sizes = [n]
    while sizes[-1] % 2 == 0 and sizes[-1] // 2 >= 4:
        sizes.append(sizes[-1] // 2)
    return sizes
