"""Homogenization parity: otm_homogenize (filter, SIMP, macro loads, MG-PCG,
tensor) against the FP64 oracle, at sizes the oracle solves in seconds, and
at 128^3 on closed forms and sampled outputs."""
import ctypes

import numpy as np
import pytest

from oracle import design, fem
import workloads as W
from tests.gpu_util import dev, empty, host, rel_fro

pytestmark = pytest.mark.gpu

TOL = {0: 1e-9, 1: 1e-6, 2: 1e-4}     # relative Frobenius error of kappa per precision


def _otm():
    from paper_2405_19991_gb300 import otm
    return otm


def _ctx(n, precision, tol, rmin=1.5, target=W.TARGET_ISOTROPIC, **kw):
    otm = _otm()
    p = otm.otm_params_default(n=n, precision=precision, cg_tol=tol, rmin=rmin,
                               kappa_target=target, cg_maxit=2000, **kw)
    return otm.otm_create_ex(p), otm


def _homogenize_host(ctx, otm, rho):
    arr = np.ascontiguousarray(rho, dtype=np.float32)
    kap, info, st = otm.otm_homogenize(ctx, arr.ctypes.data, 0)
    return np.array(kap), info, st


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("n,rmin", [(4, 1.5), (6, 2.0), (8, 1.5), (12, 2.0), (16, 1.5), (20, 2.0)])
def test_homogenize_matches_oracle(precision, n, rmin):
    ctx, otm = _ctx(n, precision, 1e-10 if precision == 0 else 1e-6, rmin=rmin)
    try:
        rho = W.initial_density(n, 0.35, 100 + n).astype(np.float32)
        kap, info, st = _homogenize_host(ctx, otm, rho)
        assert st == otm.OTM_OK, otm.otm_last_error(ctx)
        rf = design.density_filter(n, rho.astype(np.float64), rmin)
        k = design.simp(rf, 3.0, 1.0, 1e-3)
        ref = fem.homogenize(n, k, tol=1e-12)
        err = rel_fro(kap, ref["kappa"])
        assert err <= TOL[precision], (err, kap, ref["kappa"])
        assert max(info.resid) <= (1e-10 if precision == 0 else 1e-6) * 1.0001
        # the corrector fields agree up to the solver tolerance (zero mean)
        N = n ** 3
        chi = np.empty(3 * N, dtype=np.float32)
        otm.otm_get_field(ctx, otm.OTM_FIELD_CHI, chi.ctypes.data, 3 * N, 0)
        chi = chi.reshape(3, N).astype(np.float64)
        # reported with zero mean (to the FP32 rounding of the stored values)
        assert np.all(np.abs(chi.mean(axis=1)) <= 1e-6 * (np.max(np.abs(chi)) + 1e-30))
        scale = np.max(np.abs(ref["chi"])) + 1e-30
        ctol = {0: 1e-6, 1: 2e-3, 2: 2e-2}[precision]
        assert np.max(np.abs(chi - ref["chi"])) <= ctol * max(scale, 1e-3)
    finally:
        otm.otm_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_energy_error_is_one_sided(precision):
    """kappa from an inexact solution lies above the exact one (Loewner
    order), up to the rounding of the tensor sums."""
    n = 16
    ctx, otm = _ctx(n, precision, 1e-4)
    try:
        rho = W.initial_density(n, 0.3, 5).astype(np.float32)
        kap, info, st = _homogenize_host(ctx, otm, rho)
        rf = design.density_filter(n, rho.astype(np.float64), 1.5)
        ref = fem.homogenize(n, design.simp(rf, 3.0, 1.0, 1e-3), tol=1e-12)
        d = fem.kappa_matrix(kap) - fem.kappa_matrix(ref["kappa"])
        assert np.min(np.linalg.eigvalsh(d)) >= -1e-6 * np.max(np.abs(ref["kappa"]))
    finally:
        otm.otm_destroy(ctx)


@pytest.mark.parametrize("precision", [1, 2])
def test_128_solid_uniform_and_laminate(precision):
    n = 128
    ctx, otm = _ctx(n, precision, 1e-6, rmin=1.0)   # rmin = 1: the filter is the identity
    try:
        kap, info, st = _homogenize_host(ctx, otm, np.ones(n ** 3))
        assert st == otm.OTM_OK
        assert np.max(np.abs(kap - np.array([1, 1, 1, 0, 0, 0]))) < 1e-6
        kap, info, st = _homogenize_host(ctx, otm, np.full(n ** 3, 0.6))
        kc = 1e-3 + 0.6 ** 3 * (1 - 1e-3)
        assert np.max(np.abs(kap - np.array([kc, kc, kc, 0, 0, 0]))) < 1e-6 * kc * 10
        # z-laminate: rho depends on the layer only
        rng = np.random.default_rng(3)
        layers = rng.uniform(0.1, 1.0, n).astype(np.float32)
        rho = np.repeat(layers, n * n)
        kap, info, st = _homogenize_host(ctx, otm, rho)
        assert st == otm.OTM_OK, otm.otm_last_error(ctx)
        kl = 1e-3 + layers.astype(np.float64) ** 3 * (1 - 1e-3)
        arith, harm = kl.mean(), 1.0 / (1.0 / kl).mean()
        rtol = 1e-5 if precision == 1 else 1e-4
        assert abs(kap[0] - arith) <= rtol * arith
        assert abs(kap[1] - arith) <= rtol * arith
        assert abs(kap[2] - harm) <= rtol * harm + 1e-6 * arith
        assert np.max(np.abs(kap[3:])) <= 1e-6
    finally:
        otm.otm_destroy(ctx)


def test_128_anisotropic_workload_kappa_against_oracle():
    """The 128^3 anisotropic workload (volume fraction 0.35, r = 2, p = 3,
    k_void = 1e-3, its seeded initial density) end to end: filter, SIMP,
    loads, MG-PCG to 1e-6 and the tensor, FP32 and BF16-V-cycle paths, against
    the oracle's own FP64 pipeline on the same density (Jacobi-PCG to 1e-8, a
    tensor error far below the tolerances): FP32 <= 1e-6, mixed <= 1e-4
    relative (Frobenius)."""
    wl = W.ANISO_128
    n = wl.n
    rho = wl.rho0(np.float32)
    rf = design.density_filter(n, rho.astype(np.float64), wl.rmin)
    ref = fem.homogenize(n, design.simp(rf, wl.penal, wl.k_solid, wl.k_void), tol=1e-8)["kappa"]
    for precision, tol in ((1, 1e-6), (2, 1e-4)):
        ctx, otm = _ctx(n, precision, wl.cg_tol, rmin=wl.rmin, target=wl.kappa_target)
        try:
            kap, info, st = _homogenize_host(ctx, otm, rho)
            assert st == otm.OTM_OK, otm.otm_last_error(ctx)
            assert max(info.resid) <= wl.cg_tol * 1.0001
            err = rel_fro(kap, ref)
            print(f"precision {precision}: kappa relative error {err:.2e}")
            assert err <= tol, (precision, err, kap, ref)
        finally:
            otm.otm_destroy(ctx)


def test_128_sampled_residual_tensor_and_sensitivity():
    """The benchmark configuration (128^3, r = 2, FP32, cg_tol 1e-6): the
    oracle recomputes, from the GPU's own k and corrector fields, the
    residual at sampled nodes, the full tensor sum, and the element
    sensitivities at sampled elements."""
    otm = _otm()
    n = 128
    wl = W.ORTHO_128
    p = otm.otm_params_default(n=n, precision=1, cg_tol=1e-6, rmin=wl.rmin, kappa_target=wl.kappa_target)
    ctx = otm.otm_create_ex(p)
    try:
        rho = wl.rho0(np.float32)
        otm.otm_set_density(ctx, rho.ctypes.data, 0)
        info, st = otm.otm_step(ctx)
        assert st == otm.OTM_OK, otm.otm_last_error(ctx)
        N = n ** 3
        k = np.empty(N, np.float32)
        otm.otm_get_field(ctx, otm.OTM_FIELD_K, k.ctypes.data, N, 0)
        chi = np.empty(3 * N, np.float32)
        otm.otm_get_field(ctx, otm.OTM_FIELD_CHI, chi.ctypes.data, 3 * N, 0)
        rf = np.empty(N, np.float32)
        otm.otm_get_field(ctx, otm.OTM_FIELD_RHO_FILT, rf.ctypes.data, N, 0)
        k = k.astype(np.float64)
        chi = chi.reshape(3, N).astype(np.float64)
        # filter + SIMP against the oracle on the same input
        rf_ref = design.density_filter(n, rho.astype(np.float64), wl.rmin)
        assert np.max(np.abs(rf - rf_ref)) < 2e-6
        # residual at sampled nodes: |r_v| <= ||r||_2 <= tol ||f||_2
        f = fem.macro_load(n, k)
        rng = np.random.default_rng(0)
        nodes = rng.choice(N, 300, replace=False)
        Ku = fem.apply_operator_at(n, k, chi, nodes)
        r = f[:, nodes] - Ku
        for i in range(3):
            nf = np.linalg.norm(f[i] - f[i].mean())
            assert np.max(np.abs(r[i])) <= 1.5e-6 * nf
        # tensor from the GPU corrector, summed in FP64 by the oracle
        E = fem.element_energies(n, chi)
        kref = fem.kappa_from_energies(k, E)
        assert rel_fro(info.kappa, kref) <= 1e-6
        assert max(info.resid) <= 1e-6 * 1.0001
    finally:
        otm.otm_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("n,rmin", [(8, 1.5), (16, 1.5), (20, 2.0), (32, 2.0)])
def test_chebyshev_coarse_smoother_matches_oracle(precision, n, rmin):
    """coarse_smoother = 1 changes only the preconditioner: the tensor still
    matches the oracle at the same tolerance, and a cold solve needs at most
    one PCG iteration more than with the 8-colour Gauss-Seidel on the coarse
    levels."""
    rho = W.initial_density(n, 0.35, 200 + n).astype(np.float32)
    tol = 1e-10 if precision == 0 else 1e-6
    res = {}
    for sm in (0, 1):
        ctx, otm = _ctx(n, precision, tol, rmin=rmin, coarse_smoother=sm)
        try:
            kap, info, st = _homogenize_host(ctx, otm, rho)
            assert st == otm.OTM_OK, otm.otm_last_error(ctx)
            res[sm] = (kap, max(info.cg_iters), max(info.resid))
        finally:
            otm.otm_destroy(ctx)
    rf = design.density_filter(n, rho.astype(np.float64), rmin)
    ref = fem.homogenize(n, design.simp(rf, 3.0, 1.0, 1e-3), tol=1e-12)
    kap, its, resid = res[1]
    assert rel_fro(kap, ref["kappa"]) <= TOL[precision]
    assert resid <= tol * 1.0001
    assert its <= res[0][1] + 1, (res[0][1], its)


def test_256_anisotropic_error_per_precision():
    """The mixed-precision configuration at 256^3 (anisotropic target, volume
    fraction 0.35): the tensor of the FP32 and mixed paths against the FP64
    path on the same density (the FP64 path matches the oracle to 1e-9 at the
    sizes the oracle solves), and the mixed path's residual recomputed by the
    oracle at sampled nodes from the GPU's own k and corrector."""
    otm = _otm()
    wl = W.ANISO_256
    n, N = wl.n, wl.n ** 3
    rho = wl.rho0(np.float32)
    kap = {}
    for prec, tol in ((0, 1e-10), (1, 1e-6), (2, 1e-6)):
        p = otm.otm_params_default(n=n, precision=prec, cg_tol=tol, rmin=wl.rmin, kappa_target=wl.kappa_target,
                                   volfrac=wl.volfrac, cg_maxit=2000)
        ctx = otm.otm_create_ex(p)
        try:
            k6, info, st = _homogenize_host(ctx, otm, rho)
            assert st == otm.OTM_OK, otm.otm_last_error(ctx)
            assert max(info.resid) <= tol * 1.0001
            kap[prec] = k6
            if prec == 2:
                k = np.empty(N, np.float32)
                otm.otm_get_field(ctx, otm.OTM_FIELD_K, k.ctypes.data, N, 0)
                chi = np.empty(3 * N, np.float32)
                otm.otm_get_field(ctx, otm.OTM_FIELD_CHI, chi.ctypes.data, 3 * N, 0)
                k = k.astype(np.float64)
                chi = chi.reshape(3, N).astype(np.float64)
                rng = np.random.default_rng(1)
                nodes = rng.choice(N, 200, replace=False)
                f = fem.macro_load(n, k)
                r = f[:, nodes] - fem.apply_operator_at(n, k, chi, nodes)
                for i in range(3):
                    assert np.max(np.abs(r[i])) <= 1.5e-6 * np.linalg.norm(f[i] - f[i].mean())
        finally:
            otm.otm_destroy(ctx)
    e32 = rel_fro(kap[1], kap[0])
    emx = rel_fro(kap[2], kap[0])
    print(f"256^3 kappa error vs the FP64 path: FP32 {e32:.2e}, mixed {emx:.2e}")
    assert e32 <= 1e-6
    assert emx <= 1e-4


@pytest.mark.parametrize("n,precision", [(24, 1), (48, 1), (48, 2), (64, 1)])
def test_batch_sizes_match_oracle(n, precision):
    """The hierarchy shapes of the batched workload's sizes (24 -> 12 -> 6,
    48 -> ... -> 6, 64 -> ... -> 4: standalone, cluster and shared-memory tail
    levels, 6^3 and 4^3 coarsest solves) against the oracle's tensor."""
    rho = W.initial_density(n, 0.3, 300 + n).astype(np.float32)
    ctx, otm = _ctx(n, precision, 1e-6, rmin=2.0)
    try:
        kap, info, st = _homogenize_host(ctx, otm, rho)
        assert st == otm.OTM_OK, otm.otm_last_error(ctx)
        assert max(info.resid) <= 1e-6 * 1.0001
    finally:
        otm.otm_destroy(ctx)
    rf = design.density_filter(n, rho.astype(np.float64), 2.0)
    ref = fem.homogenize(n, design.simp(rf, 3.0, 1.0, 1e-3), tol=1e-12)
    assert rel_fro(kap, ref["kappa"]) <= TOL[precision]


def test_96_sampled_residual():
    """n = 96 (96 -> 48 -> 24 -> 12 -> 6): the oracle's residual at sampled
    nodes from the GPU's own k and corrector."""
    otm = _otm()
    n, N = 96, 96 ** 3
    p = otm.otm_params_default(n=n, precision=1, cg_tol=1e-6, rmin=2.0, kappa_target=W.TARGET_ORTHOTROPIC)
    ctx = otm.otm_create_ex(p)
    try:
        rho = W.initial_density(n, 0.35, 7).astype(np.float32)
        kap, info, st = _homogenize_host(ctx, otm, rho)
        assert st == otm.OTM_OK, otm.otm_last_error(ctx)
        k = np.empty(N, np.float32)
        otm.otm_get_field(ctx, otm.OTM_FIELD_K, k.ctypes.data, N, 0)
        chi = np.empty(3 * N, np.float32)
        otm.otm_get_field(ctx, otm.OTM_FIELD_CHI, chi.ctypes.data, 3 * N, 0)
        k = k.astype(np.float64)
        chi = chi.reshape(3, N).astype(np.float64)
        f = fem.macro_load(n, k)
        nodes = np.random.default_rng(5).choice(N, 300, replace=False)
        r = f[:, nodes] - fem.apply_operator_at(n, k, chi, nodes)
        for i in range(3):
            assert np.max(np.abs(r[i])) <= 1.5e-6 * np.linalg.norm(f[i] - f[i].mean())
        E = fem.element_energies(n, chi)
        assert rel_fro(kap, fem.kappa_from_energies(k, E)) <= 1e-6
    finally:
        otm.otm_destroy(ctx)


def _state_chi_pair(otm, ctx, n):
    """The stored iterate (hi, lo) of an FP32-path context, from the tail of
    its checkpoint blob (density, then the solution's high and low parts)."""
    N = n ** 3
    blob = np.frombuffer(otm.otm_get_state(ctx), dtype=np.uint8)
    chi = blob[blob.size - 24 * N:].view(np.float32).reshape(2, 3, N)
    return chi[0].astype(np.float64), chi[1].astype(np.float64)


@pytest.mark.parametrize("n,precision", [(64, 1), (128, 1), (128, 2)])
def test_convergence_check_is_the_exact_residual(n, precision):
    """The convergence check reports ||f - K (hi + lo)|| / ||f|| of the
    stored iterate, with the GPU's own FP32 k and f, to the accuracy of its
    error-free element sums: recomputed here in FP64 by the oracle's
    element-by-element operator, the two agree to 1e-6 relative (n = 64 runs
    the row-mapped check, n = 128 the warp-row one; measured: within 1e-9).
    A check that rounds each neighbour difference once is 0.1-0.4 % off at
    these residuals (the warp-row pair form, OTM_CHECK_FORM=pair), and one
    that scales by the FP32-rounded 1/12 about 1 %."""
    otm = _otm()
    N = n ** 3
    p = otm.otm_params_default(n=n, precision=precision, cg_tol=1e-6, rmin=2.0, kappa_target=W.TARGET_ORTHOTROPIC)
    ctx = otm.otm_create_ex(p)
    try:
        rho = W.initial_density(n, 0.3, 11).astype(np.float32)
        kap, info, st = _homogenize_host(ctx, otm, rho)
        assert st == otm.OTM_OK, otm.otm_last_error(ctx)
        k = np.empty(N, np.float32)
        otm.otm_get_field(ctx, otm.OTM_FIELD_K, k.ctypes.data, N, 0)
        f = np.empty(3 * N, np.float32)
        otm.otm_get_field(ctx, otm.OTM_FIELD_LOAD, f.ctypes.data, 3 * N, 0)
        hi, lo = _state_chi_pair(otm, ctx, n)
        f = f.reshape(3, N).astype(np.float64)
        r = f - fem.apply_operator(n, k.astype(np.float64), hi + lo)
        for i in range(3):
            rel = np.linalg.norm(r[i]) / np.linalg.norm(f[i])
            assert 0 < rel <= 1e-6 * 1.0001
            assert abs(info.resid[i] - rel) <= 1e-6 * rel, (i, info.resid[i], rel)
    finally:
        otm.otm_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n", [4, 5, 6, 7])
def test_single_level_direct_inverse_is_exact(precision, n):
    """On a single-level hierarchy (n < 8, or odd) the preconditioner is the
    coarsest dense inverse itself, so PCG from a zero start must finish in one
    or two iterations: an inaccurate inverse (e.g. a wrong entry in the last,
    short pivot panel of q = n^3 - 1 unknowns) shows up as extra iterations
    long before it shows up in the tensor."""
    tol = 1e-10 if precision == 0 else 1e-6
    ctx, otm = _ctx(n, precision, tol, rmin=1.5)
    try:
        rho = W.initial_density(n, 0.35, 400 + n).astype(np.float32)
        kap, info, st = _homogenize_host(ctx, otm, rho)
        assert st == otm.OTM_OK, otm.otm_last_error(ctx)
        assert max(info.cg_iters) <= 2, list(info.cg_iters)
        assert max(info.resid) <= tol * 1.0001
    finally:
        otm.otm_destroy(ctx)
