"""Kernel-level parity: each operator entry point of libotm against the FP64
oracle on the same seeded inputs, in FP64 (to rounding) and FP32 (to a bound
derived from the arithmetic)."""
import numpy as np
import pytest

from oracle import design, fem
import workloads as W
from tests.gpu_util import dev, empty, host

pytestmark = pytest.mark.gpu


def _otm():
    from paper_2405_19991_gb300 import otm
    return otm


def _tdt(dtype):
    import torch
    return torch.float64 if dtype == 0 else torch.float32


def _k(n, seed):
    rho = W.random_density(n, seed)
    return 1e-3 + rho ** 3 * (1 - 1e-3)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n,rmin", [(16, 1.5), (13, 2.0), (10, 2.5), (6, 1.0)])
def test_filter_simp(dtype, n, rmin):
    otm = _otm()
    rho = W.random_density(n, 1)
    t = _tdt(dtype)
    r_d, rf_d, k_d = dev(rho, t), empty(n ** 3, t), empty(n ** 3, t)
    otm.otm_op_filter_simp(dtype, n, rmin, 3.0, 1.0, 1e-3, r_d, rf_d, k_d)
    rho_in = host(r_d)       # the rounded input both sides see
    rf = design.density_filter(n, rho_in, rmin)
    k = design.simp(rf, 3.0, 1.0, 1e-3)
    tol = 1e-13 if dtype == 0 else 2e-6
    assert np.max(np.abs(host(rf_d) - rf)) <= tol
    assert np.max(np.abs(host(k_d) - k)) <= tol


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n,rmin", [(12, 1.5), (9, 2.0), (8, 2.9)])
def test_filter_transpose(dtype, n, rmin):
    otm = _otm()
    rng = np.random.default_rng(2)
    s = rng.standard_normal(n ** 3)
    t = _tdt(dtype)
    s_d, o_d = dev(s, t), empty(n ** 3, t)
    otm.otm_op_filter_transpose(dtype, n, rmin, s_d, o_d)
    ref = design.density_filter_transpose(n, host(s_d), rmin)
    tol = 1e-13 if dtype == 0 else 2e-6 * np.max(np.abs(s))
    assert np.max(np.abs(host(o_d) - ref)) <= tol


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [4, 7, 16])
def test_macro_load(dtype, n):
    otm = _otm()
    k = _k(n, 3)
    t = _tdt(dtype)
    k_d, f_d = dev(k, t), empty(3 * n ** 3, t)
    otm.otm_op_macro_load(dtype, n, k_d, f_d)
    ref = fem.macro_load(n, host(k_d)).ravel()
    tol = 1e-14 if dtype == 0 else 1e-6
    assert np.max(np.abs(host(f_d) - ref)) <= tol


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [4, 5, 8, 13, 16, 32, 64, 96, 128, 256])
def test_apply_K(dtype, n):
    otm = _otm()
    k = _k(n, 4)
    u = W.random_field(n, 5)
    t = _tdt(dtype)
    k_d, u_d, o_d = dev(k, t), dev(u.ravel(), t), empty(3 * n ** 3, t)
    otm.otm_op_apply_K(dtype, n, k_d, u_d, o_d)
    if n <= 128:
        ref = fem.apply_operator(n, host(k_d), host(u_d).reshape(3, -1)).ravel()
        got = host(o_d)
    else:   # sampled nodes, computed one by one
        nodes = np.random.default_rng(n).choice(n ** 3, 400, replace=False)
        ref = fem.apply_operator_at(n, host(k_d), host(u_d).reshape(3, -1), nodes).ravel()
        got = host(o_d).reshape(3, -1)[:, nodes].ravel()
    # FP32: about 40 rounded operations on terms bounded by 16/3 kmax umax
    scale = np.max(k) * np.max(np.abs(u)) * 16.0 / 3.0
    tol = 1e-13 * scale if dtype == 0 else 40 * 6e-8 * scale
    if n <= 128:
        got = host(o_d)
    assert np.max(np.abs(got - ref)) <= tol


def _check_gs_pass(dtype, K, f, before, got, nodes):
    """One relaxation pass against the oracle's, both started from the GPU's
    own field before the pass.  FP64: 1e-11.  FP32: per node, the pass forms
    T_v = (12 f_v + sum of 20 products) / (4 sum k) in about 26 rounded
    operations, so |gpu - ref| <= 32 * 2^-24 * (|f_v| + sum_w |K_vw T_w|) / K_vv
    -- the node's own scale, not the field's maximum.  Nodes outside the pass
    keep their bits."""
    ref = np.empty_like(before)
    for i in range(3):
        ref[i] = fem.gauss_seidel_pass(K, f[i], before[i], nodes)
    if dtype == 0:
        assert np.max(np.abs(got - ref)) <= 1e-11
    else:
        Ka = abs(K).tocsr()
        diag = K.diagonal()
        for i in range(3):
            scale = (np.abs(f[i]) + Ka @ np.abs(before[i]) - np.abs(diag) * np.abs(before[i])) / diag
            tol = 32 * 2.0 ** -24 * scale[nodes] + 1e-30
            err = np.abs(got[i, nodes] - ref[i, nodes])
            assert np.all(err <= tol), float(np.max(err / tol))
    other = np.setdiff1d(np.arange(before.shape[1]), nodes)
    assert np.array_equal(got[:, other], before[:, other])


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [4, 8, 12])
def test_gs_colour_pass(dtype, n):
    otm = _otm()
    k = _k(n, 6)
    rng = np.random.default_rng(7)
    f = rng.standard_normal((3, n ** 3))
    T = rng.standard_normal((3, n ** 3))
    t = _tdt(dtype)
    k_d, f_d, T_d = dev(k, t), dev(f.ravel(), t), dev(T.ravel(), t)
    K = fem.assemble(n, host(k_d))
    fh = host(f_d).reshape(3, -1)
    for colour in (0, 3, 5, 6, 1):
        before = host(T_d).reshape(3, -1)
        otm.otm_op_gs_colour(dtype, n, k_d, f_d, T_d, colour)
        _check_gs_pass(dtype, K, fh, before, host(T_d).reshape(3, -1), fem.colour_nodes(n, colour))


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [6, 16])
def test_kappa_and_sensitivity(dtype, n):
    otm = _otm()
    rho_f = W.random_density(n, 8, 0.05, 0.95)
    k = design.simp(rho_f, 3.0, 1.0, 1e-3)
    chi = 0.3 * W.random_field(n, 9)
    w = np.array([0.2, -0.1, 0.05, 0.3, -0.2, 0.1])
    t = _tdt(dtype)
    k_d, rf_d, chi_d, s_d = dev(k, t), dev(rho_f, t), dev(chi.ravel(), t), empty(n ** 3, t)
    kap = otm.otm_op_kappa_sens(dtype, n, 3.0, 1.0, 1e-3, k_d, rf_d, chi_d, w, s_d)
    kh, rfh, chih = host(k_d), host(rf_d), host(chi_d).reshape(3, -1)
    E = fem.element_energies(n, chih)
    kref = fem.kappa_from_energies(kh, E)
    tol = 1e-12 if dtype == 0 else 1e-6
    assert np.max(np.abs(np.array(kap) - kref)) <= tol * np.max(np.abs(kref))
    s_ref, _ = design.sensitivity(n, rfh, E, w, 3.0, 1.0, 1e-3, 1.5)
    stol = 1e-12 if dtype == 0 else 2e-5
    assert np.max(np.abs(host(s_d) - s_ref)) <= stol * np.max(np.abs(s_ref))


def _oc_case(seed, N, active):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.0, 1.0, N)
    s = rng.standard_normal(N) * 10.0 ** rng.uniform(-3, 0, N)
    if active:
        s = -np.abs(s) * (rng.uniform(size=N) < 0.8) + np.abs(s) * 0.01
    return rho, s


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("case", ["active", "mixed", "inactive", "infeasible"])
@pytest.mark.parametrize("n", [6, 16])
def test_oc_update(dtype, case, n):
    otm = _otm()
    N = n ** 3
    rho, s = _oc_case(11 + n, N, case in ("active", "infeasible"))
    vstar = {"active": rho.mean() - 0.01, "mixed": rho.mean() - 0.004, "inactive": 1.0,
             "infeasible": 0.0}[case]
    t = _tdt(dtype)
    r_d, s_d, o_d = dev(rho, t), dev(s, t), empty(N, t)
    lam = otm.otm_op_oc_update(dtype, n, vstar, 0.05, 0.5, 1e-3, r_d, s_d, o_d)
    ref, lam_ref = design.oc_update(host(r_d), host(s_d), vstar, 0.05, 0.5, 1e-3)
    got = host(o_d)
    tol = 1e-9 if dtype == 0 else 2e-6
    assert np.max(np.abs(got - ref)) <= tol
    if case == "inactive":
        assert lam == 0.0 and lam_ref == 0.0
    elif case == "infeasible":
        assert np.isinf(lam) and np.isinf(lam_ref)
    else:
        assert got.mean() <= vstar + 1e-6
        if np.isfinite(lam_ref) and lam_ref > 0:
            assert abs(lam - lam_ref) <= 1e-4 * lam_ref


@pytest.mark.parametrize("dtype,n", [(0, 8), (1, 8), (0, 16), (1, 16), (0, 32), (1, 32), (1, 64)])
def test_gs_group_pass(dtype, n):
    """Colour 8 + g relaxes colours 2g and 2g+1 together, as the solver does."""
    otm = _otm()
    k = _k(n, 19)
    rng = np.random.default_rng(20)
    f = rng.standard_normal((3, n ** 3))
    T = rng.standard_normal((3, n ** 3))
    t = _tdt(dtype)
    k_d, f_d, T_d = dev(k, t), dev(f.ravel(), t), dev(T.ravel(), t)
    K = fem.assemble(n, host(k_d))
    fh = host(f_d).reshape(3, -1)
    for g in (0, 3, 1, 2):
        before = host(T_d).reshape(3, -1)
        otm.otm_op_gs_colour(dtype, n, k_d, f_d, T_d, 8 + g)
        nodes = np.concatenate([fem.colour_nodes(n, 2 * g), fem.colour_nodes(n, 2 * g + 1)])
        _check_gs_pass(dtype, K, fh, before, host(T_d).reshape(3, -1), nodes)


@pytest.mark.parametrize("n", [128, 256])
def test_gs_group_pass_full_size_sampled(n):
    """The group pass the solver runs, at the benchmark sizes, checked node by node."""
    otm = _otm()
    import torch
    k = _k(n, 21)
    rng = np.random.default_rng(22)
    f = rng.standard_normal((3, n ** 3)).astype(np.float32)
    T = rng.standard_normal((3, n ** 3)).astype(np.float32)
    k_d, f_d, T_d = dev(k, torch.float32), dev(f.ravel(), torch.float32), dev(T.ravel(), torch.float32)
    kh, fh, Th = host(k_d), host(f_d).reshape(3, -1), host(T_d).reshape(3, -1)
    g = 2
    otm.otm_op_gs_colour(1, n, k_d, f_d, T_d, 8 + g)
    got = host(T_d).reshape(3, -1)
    nodes = np.concatenate([fem.colour_nodes(n, 2 * g), fem.colour_nodes(n, 2 * g + 1)])
    sample = rng.choice(nodes, 300, replace=False)
    ref = fem.gauss_seidel_at(n, kh, fh, Th, sample)
    # per node: 32 eps times the node's own scale (|f| + sum |K_vw T_w|) / K_vv, from the oracle's
    # operator on |T| (the 21-point row, all off-diagonal entries <= 0)
    absKT = fem.apply_operator_at(n, kh, np.abs(Th), sample)
    S = np.array([sum(kh[((v % n - a) % n) + n * (((v // n % n - b) % n) + n * ((v // (n * n) - c) % n))]
                      for a in (0, 1) for b in (0, 1) for c in (0, 1)) for v in sample]) / 3.0
    offsum = S * np.abs(Th[:, sample]) - absKT     # sum_w |K_vw| |T_w| = K_vv |T_v| - (K |T|)_v
    scale = (np.abs(fh[:, sample]) + offsum) / S
    assert np.all(np.abs(got[:, sample] - ref) <= 32 * 2.0 ** -24 * scale + 1e-30)
    # nodes of the other groups are untouched
    other = np.setdiff1d(rng.choice(n ** 3, 2000, replace=False), nodes)
    assert np.array_equal(got[:, other], Th[:, other])


@pytest.mark.parametrize("n", [16, 64, 128])
def test_apply_K_async_is_the_same_operator(n):
    otm = _otm()
    import torch
    k = _k(n, 8)
    u = W.random_field(n, 9)
    k_d, u_d = dev(k, torch.float32), dev(u.ravel(), torch.float32)
    a, b = empty(3 * n ** 3, torch.float32), empty(3 * n ** 3, torch.float32)
    otm.otm_op_apply_K(1, n, k_d, u_d, a)
    st = torch.cuda.current_stream()
    otm.otm_op_apply_K_async(1, n, k_d, u_d, b, st.cuda_stream)
    st.synchronize()
    assert torch.equal(a, b)


_FORM_SCRIPT = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2405_19991_gb300 import otm
import workloads as W
n, out = int(sys.argv[2]), sys.argv[3]
rho = W.random_density(n, 21)
k = torch.as_tensor(1e-3 + rho ** 3 * (1 - 1e-3), dtype=torch.float32, device="cuda").contiguous()
u = torch.as_tensor(W.random_field(n, 22).ravel(), dtype=torch.float32, device="cuda").contiguous()
o = torch.empty(3 * n ** 3, dtype=torch.float32, device="cuda")
otm.otm_op_apply_K(1, n, k, u, o)
np.save(out, o.cpu().numpy())
"""


@pytest.mark.parametrize("n", [32, 64, 96, 128, 192, 256])
def test_stencil_forms_are_bitwise_equal(n, tmp_path):
    """The three fine-stencil forms (TMA-staged, tiled, gather) sum the same
    terms per node in the same plane-by-plane order: same bits.  The sizes
    cover 1 to 16 rows per CTA (n = 256 .. 32) and a row of 48 pairs (n = 96,
    where the tiled form also applies)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    got = {}
    for form in ("tma", "tiled", "gather"):
        path = str(tmp_path / f"{form}.npy")
        env = dict(os.environ, OTM_STENCIL=form)
        subprocess.run([sys.executable, "-c", _FORM_SCRIPT, root, str(n), path], env=env, check=True,
                       timeout=300)
        got[form] = np.load(path)
    for form in ("tiled", "gather"):
        assert np.array_equal(got["tma"].view(np.uint32), got[form].view(np.uint32)), form


_GS_FORM_SCRIPT = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2405_19991_gb300 import otm
import workloads as W
n, out = int(sys.argv[2]), sys.argv[3]
rho = W.random_density(n, 31)
k = torch.as_tensor(1e-3 + rho ** 3 * (1 - 1e-3), dtype=torch.float32, device="cuda").contiguous()
f = torch.as_tensor(W.random_field(n, 32).ravel(), dtype=torch.float32, device="cuda").contiguous()
T = torch.as_tensor(W.random_field(n, 33).ravel(), dtype=torch.float32, device="cuda").contiguous()
outs = []
for g in (0, 1, 2, 3, 2, 0):
    otm.otm_op_gs_colour(1, n, k, f, T, 8 + g)
    outs.append(T.cpu().numpy())
np.save(out, np.stack(outs))
"""


def _gs_form_run(n, path, **env_extra):
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **env_extra)
    subprocess.run([sys.executable, "-c", _GS_FORM_SCRIPT, root, str(n), path], env=env, check=True, timeout=300)
    return np.load(path)


@pytest.mark.parametrize("n", [32, 64, 96, 128, 256])
def test_gs_forms_are_bitwise_equal(n, tmp_path):
    """The TMA-staged group pass takes each node's sum in the gather kernel's
    order with the same update expression: after each of six passes over
    all four groups (both y and z parities, so every periodic wrap of the
    staged rows and planes), the same bits.  n = 96 runs the form compiled
    for a run-time n."""
    a = _gs_form_run(n, str(tmp_path / "tma.npy"), OTM_GS="tma")
    b = _gs_form_run(n, str(tmp_path / "gather.npy"), OTM_GS="gather")
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("m,stages", [(1, 4), (3, 6), (7, 8), (64, 5)])
def test_gs_tma_any_runs_and_ring_depth(m, stages, tmp_path):
    """Runs of output planes (one run marching a whole column through the
    ring many times, ragged runs, one plane per run) and ring depths 4..8:
    the same bits as the gather form."""
    a = _gs_form_run(128, str(tmp_path / "a.npy"), OTM_GS="tma", OTM_GS_M=str(m), OTM_GS_STAGES=str(stages))
    b = _gs_form_run(128, str(tmp_path / "b.npy"), OTM_GS="gather")
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("m", [1, 2, 7, 64])
def test_stencil_tma_any_chunking(m, tmp_path):
    """The TMA-staged form's z-chunks (m chunks per column, ragged when m does
    not divide n; one chunk marches the whole column through the ring many
    times): any chunk count gives the same bits."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    paths = []
    for mm in (None, m):
        path = str(tmp_path / f"m{mm}.npy")
        env = dict(os.environ, OTM_STENCIL="tma")
        if mm is not None:
            env["OTM_TMA_M"] = str(mm)
        subprocess.run([sys.executable, "-c", _FORM_SCRIPT, root, "128", path], env=env, check=True, timeout=300)
        paths.append(path)
    a, b = np.load(paths[0]), np.load(paths[1])
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def _mma_case(n, k, regime, seed):
    """Inputs of one MMA iteration of model 2 on n^3 design variables."""
    rng = np.random.default_rng(seed)
    N = n ** 3
    x = rng.uniform(0.05, 0.95, N)
    x1 = np.clip(x + rng.uniform(-0.05, 0.05, N), 0.0, 1.0)
    x2 = np.clip(x1 + rng.uniform(-0.05, 0.05, N), 0.0, 1.0)
    L = x1 - rng.uniform(0.05, 0.5, N)
    U = x1 + rng.uniform(0.05, 0.5, N)
    dg = rng.standard_normal(N) * (1e-2 / N)       # the scale of dg/drho of a tensor objective
    g = {"inactive": 0.0, "active": 3e-3, "infeasible": 10.0}[regime]
    eps = {"inactive": 1.0, "active": 1e-4, "infeasible": 1e-4}[regime]
    return x, x1, x2, L, U, dg, g, eps


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [6, 16])
@pytest.mark.parametrize("k", [0, 1, 3])
@pytest.mark.parametrize("regime", ["inactive", "active", "infeasible"])
def test_mma_update(dtype, n, k, regime):
    """One MMA iteration (otm_op_mma_update) against oracle.mma.mma_update
    on the same (device-rounded) inputs: the new design, the asymptotes, the
    shifted history and the multiplier.  FP64 to 1e-10; FP32 to 2e-5 (the
    per-element arithmetic and the dual sums in FP32 move lambda by about
    1e-6 relative, and x(lambda) carries that)."""
    from oracle import mma
    otm = _otm()
    t = _tdt(dtype)
    x, x1, x2, L, U, dg, g, eps = _mma_case(n, k, regime, 40 + 7 * k + n)
    xd, x1d, x2d, Ld, Ud, dgd = dev(x, t), dev(x1, t), dev(x2, t), dev(L, t), dev(U, t), dev(dg, t)
    xh, x1h, x2h, Lh, Uh, dgh = host(xd), host(x1d), host(x2d), host(Ld), host(Ud), host(dgd)
    N = n ** 3
    lam = otm.otm_op_mma_update(dtype, n, k, g, eps, 0.5, 1000.0, 1.0, xd, dgd, x1d, x2d, Ld, Ud)
    xr, Lr, Ur, lr = mma.mma_update(k, xh, x1h, x2h, Lh, Uh, np.full(N, 1.0 / N), g - eps, dgh)
    tol = 1e-10 if dtype == 0 else 2e-5
    assert np.max(np.abs(host(xd) - xr)) <= tol, np.max(np.abs(host(xd) - xr))
    assert np.max(np.abs(host(Ld) - Lr)) <= (1e-14 if dtype == 0 else 1e-6)
    assert np.max(np.abs(host(Ud) - Ur)) <= (1e-14 if dtype == 0 else 1e-6)
    assert np.array_equal(host(x1d), xh) and np.array_equal(host(x2d), x1h)
    if regime == "inactive":
        assert lam == 0.0 and lr == 0.0
    else:
        assert lr > 0.0 and abs(lam - lr) <= (1e-9 if dtype == 0 else 1e-4) * lr, (lam, lr)
        if regime == "infeasible":
            assert lam > 1000.0
