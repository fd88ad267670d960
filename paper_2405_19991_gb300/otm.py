"""ctypes binding of libotm.so (include/otm.h).  Argument marshalling only:
every step of the computation runs in the library's CUDA kernels.  Importing
this module raises if the shared library has not been built."""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
# OTM_LIBRARY=check loads the bounds-checking build (libotm_check.so, from
# build.py --check) instead of the normal one.
LIB_PATH = os.path.join(_PKG, "libotm_check.so" if os.environ.get("OTM_LIBRARY") == "check" else "libotm.so")

OTM_OK, OTM_EINVAL, OTM_ENOMEM, OTM_ECUDA, OTM_ENOCONV, OTM_ETIMEOUT, OTM_ESTATE = range(7)
STATUS_NAMES = {0: "OTM_OK", 1: "OTM_EINVAL", 2: "OTM_ENOMEM", 3: "OTM_ECUDA",
                4: "OTM_ENOCONV", 5: "OTM_ETIMEOUT", 6: "OTM_ESTATE"}
OTM_FP64, OTM_FP32, OTM_MIXED = 0, 1, 2
OTM_WS_NONE, OTM_WS_PREV, OTM_WS_LEARNED = 0, 1, 2
OTM_OBJ_MSE, OTM_OBJ_FRACMSE, OTM_OBJ_L1 = 0, 1, 2
OTM_OPT_OC, OTM_OPT_MMA = 0, 1
(OTM_FIELD_RHO, OTM_FIELD_RHO_FILT, OTM_FIELD_K, OTM_FIELD_CHI, OTM_FIELD_LOAD,
 OTM_FIELD_SENS) = range(6)


class otm_params(C.Structure):
    _fields_ = [
        ("n", C.c_int),
        ("kappa_target", C.c_double * 6),
        ("volfrac", C.c_double),
        ("penal", C.c_double),
        ("rmin", C.c_double),
        ("k_solid", C.c_double),
        ("k_void", C.c_double),
        ("move", C.c_double),
        ("damp", C.c_double),
        ("rho_min", C.c_double),
        ("cg_tol", C.c_double),
        ("cg_maxit", C.c_int),
        ("precision", C.c_int),
        ("warm_start", C.c_int),
        ("objective", C.c_int),
        ("governor", C.c_int),
        ("fixed_volume", C.c_double),
        ("gov_bound", C.c_double),
        ("gov_small_rel", C.c_double),
        ("gov_vol_tol", C.c_double),
        ("symmetry", C.c_int),
        ("coarse_smoother", C.c_int),
        ("seed", C.c_uint64),
        ("stream", C.c_void_p),
        ("device", C.c_int),
        ("optimizer", C.c_int),
        ("mma_eps", C.c_double),
        ("mma_move", C.c_double),
        ("mma_c", C.c_double),
        ("mma_d", C.c_double),
    ]


class otm_config(C.Structure):
    _fields_ = [
        ("stencil_form", C.c_int),
        ("stencil_chunks", C.c_int),
        ("levels", C.c_int),
        ("coarsest_n", C.c_int),
        ("cluster_maxn", C.c_int),
        ("cluster_ctas", C.c_int),
        ("tail_maxn", C.c_int),
        ("autotuned", C.c_int),
        ("tune_us", C.c_double * 4),
        ("gs_form", C.c_int),
        ("gs_chunks", C.c_int),
        ("gs_stages", C.c_int),
        ("head_form", C.c_int),
        ("gs_tune_us", C.c_double * 3),
    ]

    def as_dict(self):
        return {f: (list(getattr(self, f)) if f in ("tune_us", "gs_tune_us") else getattr(self, f))
                for f, _ in self._fields_}


class otm_step_info(C.Structure):
    _fields_ = [
        ("g", C.c_double),
        ("kappa", C.c_double * 6),
        ("mean_rho", C.c_double),
        ("mean_rhop", C.c_double),
        ("vstar", C.c_double),
        ("lambda_", C.c_double),
        ("cg_iters", C.c_int * 3),
        ("iteration", C.c_int),
        ("resid", C.c_double * 3),
        ("stage_ms", C.c_float * 8),
        ("kernel_launches", C.c_int),
        ("ws_choice", C.c_int),
        ("ws_resid", (C.c_double * 3) * 4),
    ]

    def as_dict(self):
        return dict(g=self.g, kappa=list(self.kappa), mean_rho=self.mean_rho,
                    mean_rhop=self.mean_rhop, vstar=self.vstar, lam=self.lambda_,
                    cg_iters=list(self.cg_iters), iteration=self.iteration,
                    resid=list(self.resid), stage_ms=list(self.stage_ms),
                    kernel_launches=self.kernel_launches,
                    ws_choice=[(self.ws_choice >> (2 * i)) & 3 for i in range(3)],
                    ws_skipped=bool(self.ws_choice & 64), ws_paid=bool(self.ws_choice & 128),
                    ws_resid=[[self.ws_resid[c][i] for i in range(3)] for c in range(4)])


class otm_governor_state(C.Structure):
    _fields_ = [("df", C.c_double), ("vstar", C.c_double), ("g_prev", C.c_double),
                ("gap", C.c_double), ("count", C.c_int), ("reserved", C.c_int)]


class OtmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libotm.so is not built ({LIB_PATH}); run __graft_entry__.build() or "
            "python paper_2405_19991_gb300/build.py")
    lib = C.CDLL(LIB_PATH)
    vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    P = C.POINTER
    sigs = {
        "otm_params_default": [P(otm_params)],
        "otm_check_target": [P(C.c_double)],
        "otm_create": [i, P(C.c_double), d, d, d, P(vp)],
        "otm_create_ex": [P(otm_params), P(vp)],
        "otm_destroy": [vp],
        "otm_set_density": [vp, vp, i],
        "otm_get_density": [vp, vp, i],
        "otm_get_field": [vp, i, vp, sz, i],
        "otm_get_config": [vp, P(otm_config)],
        "otm_homogenize": [vp, vp, i, P(C.c_double), P(otm_step_info)],
        "otm_step": [vp, P(otm_step_info)],
        "otm_run": [vp, i, P(otm_step_info)],
        "otm_design_batch": [i, P(otm_params), P(vp), i, P(vp), P(C.c_double * 6), P(otm_step_info)],
        "otm_get_state": [vp, vp, P(sz)],
        "otm_set_state": [vp, vp, sz],
        "otm_governor_init": [P(otm_governor_state)],
        "otm_governor_update": [P(otm_governor_state), P(otm_params), d, d, d],
        "otm_op_filter_simp": [i, i, d, d, d, d, vp, vp, vp, vp],
        "otm_op_filter_transpose": [i, i, d, vp, vp, vp],
        "otm_op_macro_load": [i, i, vp, vp, vp],
        "otm_op_apply_K": [i, i, vp, vp, vp, vp],
        "otm_op_apply_K_async": [i, i, vp, vp, vp, vp],
        "otm_op_gs_colour": [i, i, vp, vp, vp, i, vp],
        "otm_op_kappa_sens": [i, i, d, d, d, vp, vp, vp, P(C.c_double), P(C.c_double), vp, vp],
        "otm_op_oc_update": [i, i, d, d, d, d, vp, vp, vp, P(C.c_double), vp],
        "otm_op_mma_update": [i, i, i, d, d, d, d, d, vp, vp, vp, vp, vp, vp, P(C.c_double), vp],
        "otm_check_selftest": [P(C.c_int)],
        "otm_op_kappa_sens_noalloc": [i, i, d, d, d, vp, vp, vp, P(C.c_double), P(C.c_double), vp, vp],
        "otm_unet_create": [i, P(C.c_int), C.c_uint64, vp, P(vp)],
        "otm_unet_destroy": [vp],
        "otm_unet_param_count": [vp, P(sz)],
        "otm_unet_get_params": [vp, vp, i],
        "otm_unet_set_params": [vp, vp, i],
        "otm_unet_forward": [vp, vp, vp, vp],
        "otm_unet_backward": [vp, vp, vp, vp],
        "otm_unet_train_step": [vp, vp, vp, d, d, P(d), vp],
        "otm_unet_eval": [vp, vp, vp, d, P(d), vp],
        "otm_set_predictor": [vp, vp, d],
        "otm_op_conv3": [i, i, i, vp, vp, vp, i, vp, vp],
        "otm_op_conv3_wgrad": [i, i, i, vp, vp, vp, vp, vp],
        "otm_op_conv3_dgrad": [i, i, i, vp, vp, vp, vp],
        "otm_unet_get_activation": [vp, i, i, vp, sz, P(C.c_int), vp],
    }
    for name, args in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.otm_last_error.argtypes = [vp]
    lib.otm_last_error.restype = C.c_char_p
    return lib


lib = _load()

# Entry points whose declarations in include/otm.h the binding mirrors.
EXPORTED = [
    "otm_params_default", "otm_check_target", "otm_create", "otm_create_ex", "otm_destroy",
    "otm_set_density", "otm_get_density", "otm_get_field", "otm_get_config", "otm_homogenize", "otm_step",
    "otm_run", "otm_design_batch", "otm_get_state", "otm_set_state", "otm_last_error",
    "otm_governor_init", "otm_governor_update", "otm_op_filter_simp", "otm_op_filter_transpose",
    "otm_op_macro_load", "otm_op_apply_K", "otm_op_apply_K_async", "otm_op_gs_colour", "otm_op_kappa_sens",
    "otm_op_oc_update", "otm_op_kappa_sens_noalloc", "otm_unet_create", "otm_unet_destroy",
    "otm_unet_param_count", "otm_unet_get_params", "otm_unet_set_params", "otm_unet_forward",
    "otm_unet_backward", "otm_unet_train_step", "otm_unet_eval", "otm_set_predictor", "otm_op_conv3",
    "otm_op_conv3_wgrad", "otm_op_conv3_dgrad", "otm_unet_get_activation", "otm_op_mma_update",
    "otm_check_selftest",
]


def otm_last_error(ctx=None) -> str:
    msg = lib.otm_last_error(ctx)
    return msg.decode() if msg else ""


def check(status, ctx=None, allow=(OTM_OK,)):
    if status not in allow:
        raise OtmError(status, otm_last_error(ctx))
    return status


def otm_params_default(**overrides) -> otm_params:
    p = otm_params()
    check(lib.otm_params_default(C.byref(p)))
    for k, v in overrides.items():
        if k == "kappa_target":
            for c in range(6):
                p.kappa_target[c] = float(v[c])
        elif k == "stream":
            p.stream = C.c_void_p(v)
        else:
            setattr(p, k, v)
    return p


def otm_check_target(kappa_target) -> int:
    arr = (C.c_double * 6)(*[float(v) for v in kappa_target])
    return lib.otm_check_target(arr)


def otm_create(n, kappa_target, volfrac, penal, rmin):
    ctx = C.c_void_p()
    arr = (C.c_double * 6)(*[float(v) for v in kappa_target])
    check(lib.otm_create(n, arr, volfrac, penal, rmin, C.byref(ctx)))
    return ctx


def otm_create_ex(params: otm_params):
    ctx = C.c_void_p()
    check(lib.otm_create_ex(C.byref(params), C.byref(ctx)))
    return ctx


def otm_destroy(ctx):
    return lib.otm_destroy(ctx)


def otm_set_density(ctx, ptr, on_device):
    return check(lib.otm_set_density(ctx, ptr, int(on_device)), ctx)


def otm_get_density(ctx, ptr, on_device):
    return check(lib.otm_get_density(ctx, ptr, int(on_device)), ctx)


def otm_get_config(ctx):
    cfg = otm_config()
    check(lib.otm_get_config(ctx, C.byref(cfg)), ctx)
    return cfg.as_dict()


def otm_get_field(ctx, which, ptr, count, on_device):
    return check(lib.otm_get_field(ctx, which, ptr, count, int(on_device)), ctx)


def otm_homogenize(ctx, ptr, on_device, allow=(OTM_OK, OTM_ENOCONV)):
    kap = (C.c_double * 6)()
    info = otm_step_info()
    st = check(lib.otm_homogenize(ctx, ptr, int(on_device), kap, C.byref(info)), ctx, allow)
    return list(kap), info, st


def otm_step(ctx, allow=(OTM_OK, OTM_ENOCONV)):
    info = otm_step_info()
    st = check(lib.otm_step(ctx, C.byref(info)), ctx, allow)
    return info, st


def otm_run(ctx, iters, allow=(OTM_OK, OTM_ENOCONV)):
    infos = (otm_step_info * max(1, iters))()
    st = check(lib.otm_run(ctx, iters, infos), ctx, allow)
    return [infos[i] for i in range(iters)], st


def otm_design_batch(params_list, rho0_ptrs, iters, rho_out_ptrs, allow=(OTM_OK, OTM_ENOCONV)):
    n = len(params_list)
    parr = (otm_params * n)(*params_list)
    r0 = (C.c_void_p * n)(*rho0_ptrs)
    ro = (C.c_void_p * n)(*rho_out_ptrs)
    kap = ((C.c_double * 6) * n)()
    infos = (otm_step_info * max(1, n * iters))()
    st = check(lib.otm_design_batch(n, parr, r0, iters, ro, kap, infos), None, allow)
    return [list(kap[d]) for d in range(n)], infos, st


def otm_get_state(ctx) -> bytes:
    ln = C.c_size_t(0)
    check(lib.otm_get_state(ctx, None, C.byref(ln)), ctx)
    buf = C.create_string_buffer(ln.value)
    check(lib.otm_get_state(ctx, buf, C.byref(ln)), ctx)
    return buf.raw[:ln.value]


def otm_set_state(ctx, blob: bytes):
    buf = C.create_string_buffer(blob, len(blob))
    return check(lib.otm_set_state(ctx, buf, len(blob)), ctx)


def otm_governor_init() -> otm_governor_state:
    s = otm_governor_state()
    check(lib.otm_governor_init(C.byref(s)))
    return s


def otm_governor_update(state: otm_governor_state, params: otm_params, g, low_bound, vol):
    return check(lib.otm_governor_update(C.byref(state), C.byref(params), g, low_bound, vol))


def _p(x):
    """Device/host pointer of a torch tensor or an integer address."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def otm_op_filter_simp(dtype, n, rmin, penal, k_solid, k_void, rho, rho_f, k, stream=None):
    return check(lib.otm_op_filter_simp(dtype, n, rmin, penal, k_solid, k_void, _p(rho), _p(rho_f),
                                        _p(k), stream))


def otm_op_filter_transpose(dtype, n, rmin, s_f, s, stream=None):
    return check(lib.otm_op_filter_transpose(dtype, n, rmin, _p(s_f), _p(s), stream))


def otm_op_macro_load(dtype, n, k, f, stream=None):
    return check(lib.otm_op_macro_load(dtype, n, _p(k), _p(f), stream))


def otm_op_apply_K(dtype, n, k, u, Ku, stream=None):
    return check(lib.otm_op_apply_K(dtype, n, _p(k), _p(u), _p(Ku), stream))


def otm_op_apply_K_async(dtype, n, k, u, Ku, stream=None):
    return check(lib.otm_op_apply_K_async(dtype, n, _p(k), _p(u), _p(Ku), stream))


def otm_op_gs_colour(dtype, n, k, f, T, colour, stream=None):
    return check(lib.otm_op_gs_colour(dtype, n, _p(k), _p(f), _p(T), colour, stream))


def otm_op_kappa_sens(dtype, n, penal, k_solid, k_void, k, rho_f, chi, w, s_f, stream=None):
    kap = (C.c_double * 6)()
    warr = (C.c_double * 6)(*[float(v) for v in w]) if w is not None else None
    check(lib.otm_op_kappa_sens(dtype, n, penal, k_solid, k_void, _p(k), _p(rho_f), _p(chi), warr, kap,
                                _p(s_f), stream))
    return list(kap)


def otm_op_kappa_sens_noalloc(dtype, n, penal, k_solid, k_void, k, rho_f, chi, w, s_f, stream=None):
    """otm_op_kappa_sens without device allocations (fixed scratch inside the library)."""
    kap = (C.c_double * 6)()
    warr = (C.c_double * 6)(*[float(v) for v in w]) if w is not None else None
    check(lib.otm_op_kappa_sens_noalloc(dtype, n, penal, k_solid, k_void, _p(k), _p(rho_f), _p(chi), warr, kap,
                                        _p(s_f), stream))
    return list(kap)


def otm_op_oc_update(dtype, n, vstar, move, damp, rho_min, rho, s, rho_new, stream=None):
    lam = C.c_double(0.0)
    check(lib.otm_op_oc_update(dtype, n, vstar, move, damp, rho_min, _p(rho), _p(s), _p(rho_new),
                               C.byref(lam), stream))
    return lam.value


def otm_check_selftest():
    """1: the checking build recorded exactly the out-of-range index; raises
    OtmError(OTM_ESTATE) in the normal build."""
    fired = C.c_int(0)
    check(lib.otm_check_selftest(C.byref(fired)))
    return fired.value


def otm_op_mma_update(dtype, n, it, g, eps, move, c, d, x, dg, xold1, xold2, low, upp, stream=None):
    lam = C.c_double(0.0)
    check(lib.otm_op_mma_update(dtype, n, it, g, eps, move, c, d, _p(x), _p(dg), _p(xold1), _p(xold2),
                                _p(low), _p(upp), C.byref(lam), stream))
    return lam.value


# ------------------------------------------------------------ learned warm start

def otm_unet_create(n, widths, seed=0, stream=None):
    u = C.c_void_p()
    w = (C.c_int * 4)(*[int(v) for v in widths])
    check(lib.otm_unet_create(n, w, seed, stream, C.byref(u)))
    return u


def otm_unet_destroy(u):
    return lib.otm_unet_destroy(u)


def otm_unet_param_count(u) -> int:
    c = C.c_size_t(0)
    check(lib.otm_unet_param_count(u, C.byref(c)))
    return c.value


def otm_unet_get_params(u, ptr, on_device):
    return check(lib.otm_unet_get_params(u, _p(ptr), int(on_device)))


def otm_unet_set_params(u, ptr, on_device):
    return check(lib.otm_unet_set_params(u, _p(ptr), int(on_device)))


def otm_unet_forward(u, x, y, stream=None):
    return check(lib.otm_unet_forward(u, _p(x), _p(y), stream))


def otm_unet_backward(u, dy, grads, stream=None):
    return check(lib.otm_unet_backward(u, _p(dy), _p(grads), stream))


def otm_unet_train_step(u, x, target, lr, target_scale=1.0, stream=None) -> float:
    loss = C.c_double(0.0)
    check(lib.otm_unet_train_step(u, _p(x), _p(target), float(target_scale), float(lr), C.byref(loss), stream))
    return loss.value


def otm_unet_eval(u, x, target, target_scale=1.0, stream=None) -> float:
    loss = C.c_double(0.0)
    check(lib.otm_unet_eval(u, _p(x), _p(target), float(target_scale), C.byref(loss), stream))
    return loss.value


def otm_set_predictor(ctx, u, scale):
    return check(lib.otm_set_predictor(ctx, u, float(scale)), ctx)


def otm_op_conv3(n, cin, cout, x, w, bias, relu, out, stream=None):
    return check(lib.otm_op_conv3(n, cin, cout, _p(x), _p(w), _p(bias), int(relu), _p(out), stream))


def otm_op_conv3_wgrad(n, cin, cout, x, g, dw, db, stream=None):
    return check(lib.otm_op_conv3_wgrad(n, cin, cout, _p(x), _p(g), _p(dw), _p(db), stream))


def otm_op_conv3_dgrad(n, cin, cout, g, w, dx, stream=None):
    return check(lib.otm_op_conv3_dgrad(n, cin, cout, _p(g), _p(w), _p(dx), stream))


def otm_unet_get_activation(u, block, which, out, count, stream=None) -> int:
    """Copies one stored activation into `out` (device FP32, [voxel][C]);
    returns C."""
    ch = C.c_int(0)
    check(lib.otm_unet_get_activation(u, int(block), int(which), _p(out), int(count), C.byref(ch), stream))
    return ch.value
