"""Pins of the FP64 oracle's finite-element homogenization against what the
mathematics fixes: closed-form K^0, closed-form cells (solid, uniform,
laminates), Voigt/Reuss and Hashin-Shtrikman bounds, cube-group
equivariance, a dense direct solve, and brute force over binary cells."""
import itertools
import os

import numpy as np
import pytest

from oracle import fem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


def test_k0_matches_closed_form():
    K0 = fem.k0_matrix()
    ref = np.array(_golden("k0_times_12.txt")) / 12.0
    assert np.max(np.abs(K0 - ref)) < 1e-15
    # the closed form itself: by popcount of l ^ m
    for l in range(8):
        for m in range(8):
            pc = bin(l ^ m).count("1")
            want = 1 / 3 if pc == 0 else (0.0 if pc == 1 else -1 / 12)
            assert abs(ref[l, m] - want) < 1e-15


def test_k0_properties():
    K0 = fem.k0_matrix()
    assert np.allclose(K0, K0.T, atol=1e-16)
    assert np.max(np.abs(K0.sum(axis=1))) < 1e-15          # constants in the kernel
    ev = np.linalg.eigvalsh(K0)
    assert abs(ev[0]) < 1e-14 and ev[1] > 0.1               # exactly one zero mode
    t = fem.test_temperatures()
    # integral of grad x_i . grad x_j over the unit cube = delta_ij
    assert np.allclose(t.T @ K0 @ t, np.eye(3), atol=1e-15)
    # the macro-load template f^0 = K^0 T^0 is +-1/4 (upper/lower face)
    f0 = K0 @ t
    for l in range(8):
        for i in range(3):
            want = 0.25 if fem.corner_offset(l)[i] else -0.25
            assert abs(f0[l, i] - want) < 1e-15


def test_connectivity_layout():
    n = 5
    conn = fem.element_nodes(n)
    # element (x, y, z) = (4, 2, 3): corner 7 is ((4+1)%5, 3, 4)
    e = 4 + n * (2 + n * 3)
    assert conn[e, 0] == e
    assert conn[e, 7] == 0 + n * (3 + n * 4)
    assert conn[e, 1] == 0 + n * (2 + n * 3)


def test_solid_cell_is_identity():
    n = 4
    h = fem.homogenize(n, np.ones(n ** 3))
    assert np.max(np.abs(h["f"])) < 1e-14
    assert np.allclose(h["kappa"], [1, 1, 1, 0, 0, 0], atol=1e-14)


def test_uniform_cell_scales():
    n = 6
    c = 0.37
    h = fem.homogenize(n, np.full(n ** 3, c))
    assert np.allclose(h["kappa"], [c, c, c, 0, 0, 0], atol=1e-14)


def test_golden_z_laminate():
    rows = _golden("laminate_z4.txt")
    layers, want = np.array(rows[0]), np.array(rows[1])
    n = 4
    k = np.repeat(layers, n * n)             # index x + n(y + n z): z slowest
    h = fem.homogenize(n, k)
    assert np.allclose(h["kappa"], want, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("n", [4, 6])
def test_laminates_arithmetic_and_harmonic(axis, n):
    rng = np.random.default_rng(10 + axis + n)
    layers = 10.0 ** rng.uniform(-3, 0, size=n)
    idx = np.arange(n)
    Z, Y, X = np.meshgrid(idx, idx, idx, indexing="ij")
    coord = (X, Y, Z)[axis].ravel()
    k = layers[coord]
    h = fem.homogenize(n, k)
    M = fem.kappa_matrix(h["kappa"])
    arith, harm = layers.mean(), 1.0 / (1.0 / layers).mean()
    for i in range(3):
        want = harm if i == axis else arith
        assert abs(M[i, i] - want) < 1e-10 * max(1.0, want)
    off = M - np.diag(np.diag(M))
    assert np.max(np.abs(off)) < 1e-12


def _random_k(n, seed, kmin=1e-3):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0, 1, n ** 3)
    return kmin + rho ** 3 * (1 - kmin)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_voigt_reuss_bounds_and_spd(seed):
    n = 6
    k = _random_k(n, seed)
    h = fem.homogenize(n, k)
    M = fem.kappa_matrix(h["kappa"])
    ev = np.linalg.eigvalsh(M)
    voigt, reuss = k.mean(), 1.0 / (1.0 / k).mean()
    assert ev[0] > 0
    assert ev[0] >= reuss * (1 - 1e-10)
    assert ev[-1] <= voigt * (1 + 1e-10)


def _kappa_of_grid(g):
    n = g.shape[0]
    return fem.homogenize(n, g.ravel())["kappa"]


def test_translation_invariance():
    n = 6
    g = _random_k(n, 7).reshape(n, n, n)
    k0 = _kappa_of_grid(g)
    k1 = _kappa_of_grid(np.roll(g, (1, -2, 3), axis=(0, 1, 2)))
    assert np.allclose(k0, k1, rtol=1e-10, atol=1e-13)


def test_axis_permutation_equivariance():
    n = 6
    g = _random_k(n, 8).reshape(n, n, n)        # indexed [z, y, x]
    M = fem.kappa_matrix(_kappa_of_grid(g))
    # swap x and y: new[z, y, x] = old[z, x, y]
    gs = np.transpose(g, (0, 2, 1))
    Ms = fem.kappa_matrix(_kappa_of_grid(gs))
    P = np.array([[0, 1, 0], [1, 0, 0], [0, 0, 1]], dtype=float)
    assert np.allclose(Ms, P @ M @ P.T, rtol=1e-10, atol=1e-13)
    # cyclic x->y->z->x: new(x', y', z') = old(z', x', y')... check via matrix
    gc = np.transpose(g, (1, 2, 0))              # new[z,y,x] = old[y,x,z]
    Mc = fem.kappa_matrix(_kappa_of_grid(gc))
    # new x-axis is old z-axis, new y is old x, new z is old y
    Q = np.zeros((3, 3))
    Q[0, 2] = Q[1, 0] = Q[2, 1] = 1.0
    assert np.allclose(Mc, Q @ M @ Q.T, rtol=1e-10, atol=1e-13)


def test_reflection_flips_cross_terms():
    n = 6
    g = _random_k(n, 9).reshape(n, n, n)
    kv = _kappa_of_grid(g)
    # element x -> n-1-x is the reflection x -> -x of the cell
    kr = _kappa_of_grid(g[:, :, ::-1])
    sign = np.array([1, 1, 1, -1, 1, -1])         # k12 and k13 change sign
    assert np.allclose(kr, sign * kv, rtol=1e-10, atol=1e-13)
    assert abs(kv[3]) > 1e-6 and abs(kv[5]) > 1e-6 and abs(kv[4]) > 1e-6
    kz = _kappa_of_grid(g[::-1, :, :])
    assert np.allclose(kz, np.array([1, 1, 1, 1, -1, -1]) * kv, rtol=1e-10, atol=1e-13)


def test_dense_direct_solve_agrees():
    n = 4
    k = _random_k(n, 11)
    K = fem.assemble(n, k).toarray()
    f = fem.macro_load(n, k)
    h = fem.homogenize(n, k, tol=1e-14)
    for i in range(3):
        x = np.zeros(n ** 3)
        x[1:] = np.linalg.solve(K[1:, 1:], f[i][1:])       # pin node 0
        x -= x.mean()
        assert np.max(np.abs(x - h["chi"][i])) < 1e-9
    # kappa from the dense solution
    chi = np.stack([np.linalg.solve(K[1:, 1:], f[i][1:]) for i in range(3)])
    chi = np.concatenate([np.zeros((3, 1)), chi], axis=1)
    E = fem.element_energies(n, chi)
    assert np.allclose(fem.kappa_from_energies(k, E), h["kappa"], rtol=1e-10, atol=1e-13)


def test_matrix_free_matches_assembled_and_load_sums():
    n = 5
    k = _random_k(n, 12)
    rng = np.random.default_rng(3)
    u = rng.standard_normal((3, n ** 3))
    K = fem.assemble(n, k)
    Ku = fem.apply_operator(n, k, u)
    for i in range(3):
        assert np.allclose(Ku[i], K @ u[i], atol=1e-13)
    f = fem.macro_load(n, k)
    assert np.max(np.abs(f.sum(axis=1))) < 1e-12
    # the assembled operator is the 21-point stencil: face neighbours vanish
    v = 2 + n * (2 + n * 2)
    row = K.getrow(v).toarray().ravel()
    nz = np.flatnonzero(np.abs(row) > 1e-14)
    assert len(nz) == 21


def test_energy_error_is_one_sided():
    """Perturbing the solution only raises the energy: kappa_ii(chi + d)
    - kappa_ii(chi) = d^T K d / N >= 0."""
    n = 4
    k = _random_k(n, 13)
    h = fem.homogenize(n, k, tol=1e-14)
    rng = np.random.default_rng(4)
    d = 1e-3 * rng.standard_normal((3, n ** 3))
    kp = fem.kappa_from_energies(k, fem.element_energies(n, h["chi"] + d))
    K = fem.assemble(n, k)
    for i in range(3):
        want = d[i] @ (K @ d[i]) / n ** 3
        assert kp[i] - h["kappa"][i] > 0
        assert abs((kp[i] - h["kappa"][i]) - want) < 1e-12


def _hs_lower(k1, k2, f2):
    """Hashin-Shtrikman lower bound (k1 < k2, f2 volume fraction of k2)."""
    f1 = 1 - f2
    return k1 + f2 / (1.0 / (k2 - k1) + f1 / (3.0 * k1))


def test_hashin_shtrikman_lower_bound_cubic_inclusion():
    """A centred cubic inclusion of the good conductor is cube-symmetric, so
    kappa is isotropic; the conforming FE value lies above the HS lower bound
    and below the Voigt bound."""
    n = 8
    k1, k2 = 0.05, 1.0
    g = np.full((n, n, n), k1)
    g[2:6, 2:6, 2:6] = k2
    kv = _kappa_of_grid(g)
    M = fem.kappa_matrix(kv)
    assert np.allclose(M, M[0, 0] * np.eye(3), rtol=1e-10, atol=1e-13)
    f2 = (g == k2).mean()
    assert M[0, 0] >= _hs_lower(k1, k2, f2)
    assert M[0, 0] <= k1 * (1 - f2) + k2 * f2


def test_brute_force_binary_2x2x2_cells():
    """All 2^8 binary 2x2x2 motifs tiled to 4^3: SPD, within Voigt/Reuss,
    and the x<->y swapped motif gives P kappa P^T."""
    k1, k2 = 1e-2, 1.0
    P = np.array([[0, 1, 0], [1, 0, 0], [0, 0, 1]], dtype=float)
    for bits in range(256):
        motif = np.array([(bits >> l) & 1 for l in range(8)], dtype=float).reshape(2, 2, 2)
        kk = np.where(motif > 0, k2, k1)
        g = np.tile(kk, (2, 2, 2))
        kv = _kappa_of_grid(g)
        M = fem.kappa_matrix(kv)
        ev = np.linalg.eigvalsh(M)
        k = g.ravel()
        assert ev[0] >= (1.0 / (1.0 / k).mean()) * (1 - 1e-9)
        assert ev[-1] <= k.mean() * (1 + 1e-9)
        if bits % 17 == 0:
            Ms = fem.kappa_matrix(_kappa_of_grid(np.transpose(g, (0, 2, 1))))
            assert np.allclose(Ms, P @ M @ P.T, rtol=1e-9, atol=1e-12)


def test_prolongation_and_galerkin():
    nc = 4
    P = fem.prolongation(nc)
    assert np.allclose(P @ np.ones(nc ** 3), 1.0)
    # column sums of P are 8 (each coarse basis function covers 27 fine nodes
    # with total weight (1/2 + 1 + 1/2)^3 = 8)
    assert np.allclose(np.asarray(P.sum(axis=0)).ravel(), 8.0)
    n = 2 * nc
    k = _random_k(n, 14)
    A = fem.assemble(n, k)
    Ac = fem.galerkin(A, nc)
    assert np.allclose((Ac - Ac.T).toarray(), 0, atol=1e-14)
    assert np.max(np.abs(Ac @ np.ones(nc ** 3))) < 1e-12
    # every row couples to at most 27 nodes
    assert max(np.diff(Ac.indptr)) <= 27


def test_level_sizes():
    assert fem.level_sizes(128) == [128, 64, 32, 16, 8, 4]
    assert fem.level_sizes(16) == [16, 8, 4]
    assert fem.level_sizes(96) == [96, 48, 24, 12, 6]
    assert fem.level_sizes(6) == [6]


def test_apply_operator_at_matches_full():
    n = 5
    k = _random_k(n, 15)
    rng = np.random.default_rng(5)
    u = rng.standard_normal((3, n ** 3))
    full = fem.apply_operator(n, k, u)
    nodes = [0, 7, 63, 124]
    assert np.allclose(fem.apply_operator_at(n, k, u, nodes), full[:, nodes], atol=1e-13)


def test_gauss_seidel_pass_zeroes_residual_on_colour():
    """Nodes of one colour are uncoupled, so after one pass over them their
    residual vanishes exactly (and the order within the colour is
    irrelevant)."""
    n = 6
    k = _random_k(n, 16)
    K = fem.assemble(n, k)
    rng = np.random.default_rng(6)
    f = rng.standard_normal(n ** 3)
    T = rng.standard_normal(n ** 3)
    for colour in range(8):
        nodes = fem.colour_nodes(n, colour)
        T1 = fem.gauss_seidel_pass(K, f, T, nodes)
        T2 = fem.gauss_seidel_pass(K, f, T, nodes[::-1])
        assert np.allclose(T1, T2, atol=1e-13)
        r = f - K @ T1
        assert np.max(np.abs(r[nodes])) < 1e-12
        others = np.setdiff1d(np.arange(n ** 3), nodes)
        assert np.array_equal(T1[others], T[others])


def test_x_parity_pairs_are_uncoupled():
    """Colours differing only in x parity share no matrix entry (face
    neighbours carry 0), so a pass over colour 2c then 2c+1 equals one pass
    over their union."""
    n = 6
    k = _random_k(n, 17)
    K = fem.assemble(n, k).toarray()
    for c in range(0, 8, 2):
        a, b = fem.colour_nodes(n, c), fem.colour_nodes(n, c + 1)
        assert np.max(np.abs(K[np.ix_(a, b)])) < 1e-15


def test_gauss_seidel_at_matches_pass():
    n = 6
    k = _random_k(n, 18)
    K = fem.assemble(n, k)
    rng = np.random.default_rng(7)
    f = rng.standard_normal((1, n ** 3))
    T = rng.standard_normal((1, n ** 3))
    nodes = fem.colour_nodes(n, 5)
    full = fem.gauss_seidel_pass(K, f[0], T[0], nodes)
    assert np.allclose(fem.gauss_seidel_at(n, k, f, T, nodes)[0], full[nodes], atol=1e-12)


def test_pcg_observer_sees_every_iteration_and_changes_nothing():
    """The observer hook the CPU baseline times the solve with: called once
    per stopping test with iterations 0, 1, ..., the recurrence residual
    starting at 1 from a zero start, and the solve bitwise the one without
    it."""
    n = 6
    rng = np.random.default_rng(3)
    k = 1e-3 + rng.random(n ** 3) ** 3
    K = fem.assemble(n, k)
    f = fem.macro_load(n, k)[0]
    seen = []
    x1, it1, r1 = fem.pcg(K, f, tol=1e-10, observe=lambda it, res: seen.append((it, res)))
    x0, it0, r0 = fem.pcg(K, f, tol=1e-10)
    assert it1 == it0 and r1 == r0 and np.array_equal(x1, x0)
    assert [s[0] for s in seen] == list(range(it0 + 1))
    assert abs(seen[0][1] - 1.0) < 1e-12
    assert seen[-1][1] <= 1e-10 < seen[-2][1]
