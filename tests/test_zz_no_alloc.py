"""otm_op_kappa_sens_noalloc: the allocation-free variant of the tensor /
sensitivity entry point, for callers that cannot allocate device memory
(a host framework that owns the device memory through its own pool, or a
loop that cannot afford an allocation's synchronisation).  Its output must
match otm_op_kappa_sens on the same inputs, on two calls in a row (the
second call must not see stale scratch contents from the first).

This file is named to be collected last."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import dev, empty, host

pytestmark = pytest.mark.gpu


def _inputs(n, seed, dtype):
    import torch
    from oracle import design
    t = torch.float64 if dtype == 0 else torch.float32
    rho_f = W.random_density(n, seed, 0.05, 0.95)
    k = design.simp(rho_f, 3.0, 1.0, 1e-3)
    chi = 0.3 * W.random_field(n, seed + 1)
    rng = np.random.default_rng(seed + 2)
    w = rng.uniform(-0.3, 0.3, 6)
    return dev(k, t), dev(rho_f, t), dev(chi.ravel(), t), w, t


def _runtime():
    """The CUDA runtime library this process already loaded (the one
    libotm.so links), to read the stream-ordered allocator's counters."""
    import ctypes
    with open("/proc/self/maps") as fh:
        paths = sorted({ln.split()[-1] for ln in fh if "libcudart.so" in ln})
    assert paths, "no CUDA runtime mapped"
    return ctypes.CDLL(paths[0])


def _pool_high_water(rt, reset=False):
    """High-water mark of the device's current memory pool (the pool the
    allocating entry point's cudaMallocAsync draws from); reset=True first
    lowers it to the pool's current use."""
    import ctypes
    import torch
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    v = ctypes.c_uint64(0)
    if reset:
        assert rt.cudaMemPoolSetAttribute(pool, 8, ctypes.byref(v)) == 0   # cudaMemPoolAttrUsedMemHigh
    assert rt.cudaMemPoolGetAttribute(pool, 8, ctypes.byref(v)) == 0
    return v.value


def test_noalloc_makes_no_device_allocation():
    """The property the entry point exists for.  After its first call on the
    device (which looks up the scratch's address), further calls leave both
    the stream-ordered pool's high-water mark and the device's free memory
    where they were, while the allocating entry point, as a control, does
    raise the pool's mark."""
    import torch
    from paper_2405_19991_gb300 import otm
    n = 64
    k_d, rf_d, chi_d, w, t = _inputs(n, 5, 1)
    s = empty(n ** 3, t)
    otm.otm_op_kappa_sens_noalloc(1, n, 3.0, 1.0, 1e-3, k_d, rf_d, chi_d, w, s)
    torch.cuda.synchronize()
    rt = _runtime()
    base = _pool_high_water(rt, reset=True)
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        otm.otm_op_kappa_sens_noalloc(1, n, 3.0, 1.0, 1e-3, k_d, rf_d, chi_d, w, s)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert _pool_high_water(rt) == base
    assert free1 == free0
    otm.otm_op_kappa_sens(1, n, 3.0, 1.0, 1e-3, k_d, rf_d, chi_d, w, s)
    torch.cuda.synchronize()
    assert _pool_high_water(rt) > base


@pytest.mark.parametrize("dtype", [1, 0])
@pytest.mark.parametrize("n", [16, 128])
def test_noalloc_matches_allocating_entry_point_twice(dtype, n):
    from paper_2405_19991_gb300 import otm
    rtol = 1e-12 if dtype == 0 else 1e-6
    for call, seed in enumerate((31, 47)):
        k_d, rf_d, chi_d, w, t = _inputs(n, seed, dtype)
        s_ref = empty(n ** 3, t)
        s_new = empty(n ** 3, t)
        kap_ref = otm.otm_op_kappa_sens(dtype, n, 3.0, 1.0, 1e-3, k_d, rf_d, chi_d, w, s_ref)
        kap_new = otm.otm_op_kappa_sens_noalloc(dtype, n, 3.0, 1.0, 1e-3, k_d, rf_d, chi_d, w, s_new)
        kr, kn = np.array(kap_ref), np.array(kap_new)
        assert np.max(np.abs(kn - kr)) <= rtol * np.max(np.abs(kr)), (call, kn, kr)
        sr, sn = host(s_ref), host(s_new)
        assert np.max(np.abs(sn - sr)) <= rtol * np.max(np.abs(sr)), call


def test_noalloc_rejects_sizes_beyond_its_limit():
    from paper_2405_19991_gb300 import otm
    import ctypes
    kap = (ctypes.c_double * 6)()
    st = otm.lib.otm_op_kappa_sens_noalloc(1, 600, 3.0, 1.0, 1e-3, 1, None, 1, None, kap, None, None)
    assert st == otm.OTM_EINVAL
    assert "512" in otm.otm_last_error()
