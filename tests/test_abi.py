"""CPU-side checks of the C ABI: the library loads, exports every entry point
declared in include/otm.h, its structs have the header's layout, and the
host-only entry points (target check, Alg. 1 governor, parameter
validation) behave as specified.  No compute call needs a GPU here."""
import ctypes
import itertools
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "otm.h")


def _lib():
    from paper_2405_19991_gb300 import otm
    return otm


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"OTM_API\s+[\w\s\*]+?\b(otm_\w+)\s*\(", src)))


def test_library_exports_every_declared_entry_point():
    otm = _lib()
    names = _declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(otm.lib, name), name
    assert set(names) == set(otm.EXPORTED)
    if shutil.which("nm"):
        out = subprocess.run(["nm", "-D", "--defined-only", otm.LIB_PATH], capture_output=True,
                             text=True).stdout
        exported = set(re.findall(r" T (otm_\w+)", out))
        assert set(names) <= exported
        assert exported <= set(names), exported - set(names)


def test_struct_layout_matches_header(tmp_path):
    otm = _lib()
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    probe = tmp_path / "probe.c"
    probe.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "otm.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(otm_params), sizeof(otm_step_info), sizeof(otm_governor_state));
  printf("%zu %zu %zu %zu %zu\n", offsetof(otm_params, cg_maxit), offsetof(otm_params, fixed_volume),
         offsetof(otm_params, seed), offsetof(otm_params, stream), offsetof(otm_params, device));
  printf("%zu %zu %zu\n", offsetof(otm_step_info, cg_iters), offsetof(otm_step_info, resid),
         offsetof(otm_step_info, stage_ms));
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(otm_config), offsetof(otm_config, tune_us),
         offsetof(otm_config, gs_form), offsetof(otm_config, gs_stages), offsetof(otm_config, head_form),
         offsetof(otm_config, gs_tune_us));
  printf("%zu %zu %zu\n", offsetof(otm_params, optimizer), offsetof(otm_params, mma_eps),
         offsetof(otm_params, mma_d));
  return 0;
}
''')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    s = [int(v) for v in lines[0].split()]
    o1 = [int(v) for v in lines[1].split()]
    o2 = [int(v) for v in lines[2].split()]
    P, I, G = otm.otm_params, otm.otm_step_info, otm.otm_governor_state
    assert s == [ctypes.sizeof(P), ctypes.sizeof(I), ctypes.sizeof(G)]
    assert o1 == [P.cg_maxit.offset, P.fixed_volume.offset, P.seed.offset, P.stream.offset, P.device.offset]
    assert o2 == [I.cg_iters.offset, I.resid.offset, I.stage_ms.offset]
    Cf = otm.otm_config
    o3 = [int(v) for v in lines[3].split()]
    assert o3 == [ctypes.sizeof(Cf), Cf.tune_us.offset, Cf.gs_form.offset, Cf.gs_stages.offset,
                  Cf.head_form.offset, Cf.gs_tune_us.offset]
    o4 = [int(v) for v in lines[4].split()]
    assert o4 == [P.optimizer.offset, P.mma_eps.offset, P.mma_d.offset]


def test_check_target_on_the_papers_traversal_grid():
    """Sec. 4.2 enumerates 6 x 4 x 4 = 96 cross-term combinations around the
    diagonal [0.3, 0.2, 0.1]; the library accepts exactly the positive
    definite ones (checked here by eigenvalues)."""
    otm = _lib()
    acc = 0
    for a, b, c in itertools.product([0, 0.05, 0.1, 0.15, 0.2, 0.24], [0, 0.05, 0.1, 0.15],
                                     [0, 0.05, 0.1, 0.14]):
        t = [0.3, 0.2, 0.1, a, b, c]
        m = np.array([[t[0], t[3], t[5]], [t[3], t[1], t[4]], [t[5], t[4], t[2]]])
        pd = bool(np.all(np.linalg.eigvalsh(m) > 1e-12))
        ok = otm.otm_check_target(t) == otm.OTM_OK
        assert ok == pd, t
        acc += ok
    assert acc == 59
    assert otm.otm_check_target([0.1, 0.1, 0.1, 0, 0, 0]) == otm.OTM_OK
    assert otm.otm_check_target([0.1, -0.1, 0.1, 0, 0, 0]) == otm.OTM_EINVAL
    assert otm.otm_check_target([0.1, 0.1, float("nan"), 0, 0, 0]) == otm.OTM_EINVAL


def test_governor_host_entry_matches_hand_trace():
    otm = _lib()
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", "governor_trace.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    p = otm.otm_params_default()
    s = otm.otm_governor_init()
    assert (s.df, s.vstar, s.g_prev, s.gap, s.count) == (1.0, 1.0, 1.0, 0.0, 0)
    for g, low, vol, vstar, df, count in rows:
        otm.otm_governor_update(s, p, g, low, vol)
        assert abs(s.vstar - vstar) < 1e-14
        assert abs(s.df - df) < 1e-14
        assert s.count == int(count)


@pytest.mark.parametrize("field,value", [
    ("n", 3), ("n", 9), ("n", 600), ("rmin", 3.0), ("rmin", 0.5), ("penal", 0.5),
    ("k_void", 0.0), ("k_void", 2.0), ("move", 0.0), ("cg_tol", 0.0), ("cg_maxit", 0),
    ("precision", 7), ("objective", 5), ("volfrac", 1.5), ("governor", 2),
])
def test_create_rejects_bad_parameters(field, value):
    otm = _lib()
    p = otm.otm_params_default()
    setattr(p, field, value)
    ctx = ctypes.c_void_p()
    st = otm.lib.otm_create_ex(ctypes.byref(p), ctypes.byref(ctx))
    assert st == otm.OTM_EINVAL
    assert ctx.value is None
    assert otm.otm_last_error()


def test_create_rejects_indefinite_target_and_null_arguments():
    otm = _lib()
    p = otm.otm_params_default(kappa_target=[0.3, 0.2, 0.1, 0.24, 0.15, 0.14])
    ctx = ctypes.c_void_p()
    assert otm.lib.otm_create_ex(ctypes.byref(p), ctypes.byref(ctx)) == otm.OTM_EINVAL
    assert "positive definite" in otm.otm_last_error()
    assert otm.lib.otm_create_ex(None, ctypes.byref(ctx)) == otm.OTM_EINVAL
    assert otm.lib.otm_step(None, None) == otm.OTM_EINVAL
    assert otm.lib.otm_destroy(None) == otm.OTM_OK
    # operator entry points validate before touching the device
    assert otm.lib.otm_op_apply_K(9, 8, None, None, None, None) == otm.OTM_EINVAL
    assert otm.lib.otm_op_gs_colour(1, 7, 1, 1, 1, 0, None) == otm.OTM_EINVAL


def test_level_hierarchy_sizes_accepted():
    """Sizes whose halving reaches a coarsest grid of at most 7 pass the
    host-side validation (the create then fails only for lack of a GPU)."""
    otm = _lib()
    for n in (4, 5, 6, 7, 8, 10, 12, 14, 16, 32, 48, 64, 96, 112, 128, 256):
        p = otm.otm_params_default(n=n)
        ctx = ctypes.c_void_p()
        st = otm.lib.otm_create_ex(ctypes.byref(p), ctypes.byref(ctx))
        if st == otm.OTM_OK:
            otm.lib.otm_destroy(ctx)
        else:
            assert st in (otm.OTM_ECUDA, otm.OTM_ENOMEM), (n, otm.otm_last_error())


def test_unet_and_conv_entry_points_validate_sizes_before_touching_the_gpu():
    otm = _lib()
    bad_widths = [(16, 24, 32, 32), (8, 16, 16, 16), (16, 16, 16, 272)]
    for w in bad_widths:
        with pytest.raises(otm.OtmError) as e:
            otm.otm_unet_create(16, w)
        assert e.value.status == otm.OTM_EINVAL
    for n in (4, 12, 520):
        with pytest.raises(otm.OtmError) as e:
            otm.otm_unet_create(n, (16, 16, 16, 16))
        assert e.value.status == otm.OTM_EINVAL
    with pytest.raises(otm.OtmError):
        otm.otm_op_conv3(8, 24, 16, 1, 1, None, 0, 1)
    with pytest.raises(otm.OtmError):
        otm.otm_op_conv3_wgrad(0, 16, 16, 1, 1, 1, None)
    assert otm.lib.otm_set_predictor(None, None, 1.0) == otm.OTM_EINVAL
