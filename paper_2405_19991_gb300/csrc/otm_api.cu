// C ABI of libotm.so (declared in include/otm.h): argument checking,
// context lifecycle and dispatch to the per-precision solvers.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <thread>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "solver.cuh"

using otm::SolverBase;

struct otm_ctx {
    SolverBase* s = nullptr;
    int device = 0;
};

namespace {

thread_local std::string g_err = "";

otm_status fail(otm_status st, const std::string& msg) {
    g_err = msg;
    return st;
}

otm_status ctx_fail(otm_ctx* ctx, otm_status st, const std::string& msg) {
    if (ctx && ctx->s) ctx->s->err = msg;
    else g_err = msg;
    return st;
}

bool spd6(const double k[6]) {
    const double a = k[0], b = k[1], c = k[2], xy = k[3], yz = k[4], xz = k[5];
    if (!(a > 0)) return false;
    if (!(a * b - xy * xy > 0)) return false;
    const double det = a * (b * c - yz * yz) - xy * (xy * c - yz * xz) + xz * (xy * yz - b * xz);
    return det > 0;
}

std::string check_params(const otm_params* p) {
    if (!p) return "params is NULL";
    if (p->n < 4 || p->n > 512) return "n must be in [4, 512]";
    std::vector<int> sizes;
    otm::level_sizes(p->n, sizes);
    if (sizes.back() > 7)
        return "n must reach a coarsest grid of at most 7^3 nodes by halving (n = c * 2^L, 4 <= c <= 7)";
    for (int c = 0; c < 6; ++c)
        if (!std::isfinite(p->kappa_target[c])) return "kappa_target has a non-finite entry";
    if (!spd6(p->kappa_target)) return "kappa_target is not symmetric positive definite";
    if (!(p->volfrac >= 0.0 && p->volfrac <= 1.0)) return "volfrac must be in [0, 1]";
    if (!(p->penal >= 1.0 && p->penal <= 10.0)) return "penal must be in [1, 10]";
    if (!(p->rmin >= 1.0 && p->rmin < 3.0)) return "rmin must be in [1, 3)";
    if (!(p->k_void > 0.0 && p->k_solid > p->k_void && std::isfinite(p->k_solid)))
        return "need k_solid > k_void > 0";
    if (!(p->move > 0.0 && p->move <= 1.0)) return "move must be in (0, 1]";
    if (!(p->damp > 0.0 && p->damp <= 4.0)) return "damp must be in (0, 4]";
    if (!(p->rho_min >= 0.0 && p->rho_min < 1.0)) return "rho_min must be in [0, 1)";
    if (!(p->cg_tol > 0.0 && p->cg_tol < 1.0)) return "cg_tol must be in (0, 1)";
    if (p->cg_maxit < 1) return "cg_maxit must be >= 1";
    if (p->precision < OTM_FP64 || p->precision > OTM_MIXED) return "unknown precision";
    if (p->warm_start < OTM_WS_NONE || p->warm_start > OTM_WS_LEARNED) return "unknown warm_start";
    if (p->objective < OTM_OBJ_MSE || p->objective > OTM_OBJ_L1) return "unknown objective";
    if (p->governor != 0 && p->governor != 1) return "governor must be 0 or 1";
    if (!p->governor && !(p->fixed_volume > 0.0 && p->fixed_volume <= 1.0))
        return "fixed_volume must be in (0, 1]";
    if (!(p->gov_bound > 0.0 && p->gov_small_rel > 0.0 && p->gov_vol_tol > 0.0))
        return "governor thresholds must be positive";
    if (p->symmetry != 0 && p->symmetry != 1) return "symmetry must be 0 or 1";
    if (p->coarse_smoother != 0 && p->coarse_smoother != 1) return "coarse_smoother must be 0 or 1";
    if (p->optimizer != OTM_OPT_OC && p->optimizer != OTM_OPT_MMA) return "unknown optimizer";
    if (p->optimizer == OTM_OPT_MMA &&
        !(std::isfinite(p->mma_eps) && p->mma_move > 0.0 && p->mma_move <= 1.0 && p->mma_c >= 0.0 &&
          std::isfinite(p->mma_c) && p->mma_d > 0.0 && std::isfinite(p->mma_d)))
        return "MMA parameters: need finite mma_eps, mma_move in (0, 1], mma_c >= 0, mma_d > 0";
    return "";
}

}  // namespace

namespace otm {
void set_thread_error(const std::string& msg) { g_err = msg; }
}  // namespace otm

#define CTX_CHECK(ctx)                                                                  \
    do {                                                                                \
        if (!(ctx) || !(ctx)->s) return fail(OTM_EINVAL, "context is NULL");            \
        cudaSetDevice((ctx)->device);                                                   \
    } while (0)

extern "C" {

otm_status otm_params_default(otm_params* p) {
    if (!p) return fail(OTM_EINVAL, "otm_params_default: NULL");
    memset(p, 0, sizeof(*p));
    p->n = 128;
    const double t[6] = {0.1, 0.1, 0.1, 0.0, 0.0, 0.0};
    for (int c = 0; c < 6; ++c) p->kappa_target[c] = t[c];
    p->volfrac = 0.3;
    p->penal = 3.0;
    p->rmin = 1.5;
    p->k_solid = 1.0;
    p->k_void = 1e-3;
    p->move = 0.05;
    p->damp = 0.5;
    p->rho_min = 1e-3;
    p->cg_tol = 1e-6;
    p->cg_maxit = 500;
    p->precision = OTM_FP32;
    p->warm_start = OTM_WS_PREV;
    p->objective = OTM_OBJ_MSE;
    p->governor = 1;
    p->fixed_volume = 0.3;
    p->gov_bound = 1e-4;
    p->gov_small_rel = 1e-3;
    p->gov_vol_tol = 1e-2;
    p->symmetry = 0;
    p->coarse_smoother = 0;
    p->seed = 0;
    p->stream = nullptr;
    p->device = -1;
    p->optimizer = OTM_OPT_OC;
    p->mma_eps = 1e-4;
    p->mma_move = 0.5;
    p->mma_c = 1000.0;
    p->mma_d = 1.0;
    return OTM_OK;
}

otm_status otm_check_target(const double kappa_target[6]) {
    if (!kappa_target) return fail(OTM_EINVAL, "otm_check_target: NULL");
    for (int c = 0; c < 6; ++c)
        if (!std::isfinite(kappa_target[c])) return fail(OTM_EINVAL, "kappa_target has a non-finite entry");
    if (!spd6(kappa_target)) return fail(OTM_EINVAL, "kappa_target is not symmetric positive definite");
    return OTM_OK;
}

otm_status otm_create_ex(const otm_params* params, otm_ctx** out) {
    if (!out) return fail(OTM_EINVAL, "otm_create_ex: out is NULL");
    *out = nullptr;
    const std::string msg = check_params(params);
    if (!msg.empty()) return fail(OTM_EINVAL, "otm_create_ex: " + msg);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1)
        return fail(OTM_ECUDA, "otm_create_ex: no CUDA device");
    if (params->device >= ndev) return fail(OTM_EINVAL, "otm_create_ex: device ordinal out of range");
    otm_ctx* ctx = new (std::nothrow) otm_ctx();
    if (!ctx) return fail(OTM_ENOMEM, "otm_create_ex: host allocation failed");
    switch (params->precision) {
        case OTM_FP64: ctx->s = otm::make_solver_f64(); break;
        case OTM_FP32: ctx->s = otm::make_solver_f32(); break;
        default: ctx->s = otm::make_solver_mixed(); break;
    }
    otm_status st = ctx->s->init(*params);
    if (st != OTM_OK) {
        const std::string e = "otm_create_ex: " + ctx->s->err;
        delete ctx->s;
        delete ctx;
        return fail(st, e);
    }
    ctx->device = ctx->s->device;
    *out = ctx;
    return OTM_OK;
}

otm_status otm_create(int n, const double kappa_target[6], double volfrac, double penal, double rmin,
                      otm_ctx** out) {
    if (!kappa_target) return fail(OTM_EINVAL, "otm_create: kappa_target is NULL");
    otm_params p;
    otm_params_default(&p);
    p.n = n;
    for (int c = 0; c < 6; ++c) p.kappa_target[c] = kappa_target[c];
    p.volfrac = volfrac;
    p.penal = penal;
    p.rmin = rmin;
    return otm_create_ex(&p, out);
}

otm_status otm_destroy(otm_ctx* ctx) {
    if (!ctx) return OTM_OK;
    if (ctx->s) {
        cudaSetDevice(ctx->device);
        delete ctx->s;
    }
    delete ctx;
    return OTM_OK;
}

otm_status otm_set_density(otm_ctx* ctx, const float* rho, int on_device) {
    CTX_CHECK(ctx);
    if (!rho) return ctx_fail(ctx, OTM_EINVAL, "otm_set_density: rho is NULL");
    return ctx->s->set_density(rho, on_device != 0);
}

otm_status otm_get_density(otm_ctx* ctx, float* rho, int on_device) {
    CTX_CHECK(ctx);
    if (!rho) return ctx_fail(ctx, OTM_EINVAL, "otm_get_density: rho is NULL");
    return ctx->s->get_density(rho, on_device != 0);
}

otm_status otm_get_config(otm_ctx* ctx, otm_config* out) {
    CTX_CHECK(ctx);
    if (!out) return ctx_fail(ctx, OTM_EINVAL, "otm_get_config: out is NULL");
    return ctx->s->get_config(out);
}

otm_status otm_get_field(otm_ctx* ctx, int which, float* out, size_t count, int on_device) {
    CTX_CHECK(ctx);
    if (!out) return ctx_fail(ctx, OTM_EINVAL, "otm_get_field: out is NULL");
    return ctx->s->get_field(which, out, count, on_device != 0);
}

otm_status otm_homogenize(otm_ctx* ctx, const float* rho, int on_device, double kappa_out[6],
                          otm_step_info* info) {
    CTX_CHECK(ctx);
    if (!kappa_out) return ctx_fail(ctx, OTM_EINVAL, "otm_homogenize: kappa_out is NULL");
    if (info) memset(info, 0, sizeof(*info));
    return ctx->s->homogenize(rho, on_device != 0, kappa_out, info);
}

otm_status otm_step(otm_ctx* ctx, otm_step_info* info) {
    CTX_CHECK(ctx);
    return ctx->s->step(info);
}

otm_status otm_run(otm_ctx* ctx, int iters, otm_step_info* infos) {
    CTX_CHECK(ctx);
    if (iters < 0) return ctx_fail(ctx, OTM_EINVAL, "otm_run: iters < 0");
    otm_status worst = OTM_OK;
    for (int i = 0; i < iters; ++i) {
        otm_status st = ctx->s->step(infos ? infos + i : nullptr);
        if (st == OTM_ENOCONV) worst = OTM_ENOCONV;
        else if (st != OTM_OK) return st;
    }
    return worst;
}

otm_status otm_design_batch(int count, const otm_params* params, const float* const* rho0, int iters,
                            float* const* rho_out, double (*kappa_out)[6], otm_step_info* infos) {
    if (count < 0 || iters < 0) return fail(OTM_EINVAL, "otm_design_batch: negative count or iters");
    if (count > 0 && !params) return fail(OTM_EINVAL, "otm_design_batch: params is NULL");
    for (int d = 0; d < count; ++d) {
        const std::string msg = check_params(&params[d]);
        if (!msg.empty()) return fail(OTM_EINVAL, "otm_design_batch: design " + std::to_string(d) + ": " + msg);
    }
    std::vector<otm_ctx*> ctxs(count, nullptr);
    std::vector<otm_status> stat(count, OTM_OK);
    std::vector<std::string> msgs(count);
    // contexts first: their allocations synchronise the device
    for (int d = 0; d < count; ++d) {
        otm_params p = params[d];
        p.stream = nullptr;   // a stream of its own
        stat[d] = otm_create_ex(&p, &ctxs[d]);
        if (stat[d] != OTM_OK) msgs[d] = g_err;
        if (stat[d] == OTM_OK && rho0 && rho0[d]) {
            stat[d] = otm_set_density(ctxs[d], rho0[d], 0);
            if (stat[d] != OTM_OK) msgs[d] = otm_last_error(ctxs[d]);
        }
        // graphs are built here, on the calling thread, before any worker starts
        if (stat[d] == OTM_OK) {
            stat[d] = ctxs[d]->s->prepare();
            if (stat[d] != OTM_OK) msgs[d] = otm_last_error(ctxs[d]);
        }
    }
    int workers = count < 16 ? count : 16;
    if (const char* e = getenv("OTM_BATCH_WORKERS")) {
        const int w = atoi(e);
        if (w >= 1) workers = w < count ? w : count;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    // largest designs first (longest-processing-time order), so the last
    // designs to finish are small ones instead of a large one running alone;
    // each design's result does not depend on when it runs
    std::vector<int> order(count);
    for (int d = 0; d < count; ++d) order[d] = d;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return params[a].n > params[b].n; });
    std::atomic<int> next{0};
    auto work = [&]() {
        cudaSetDevice(dev);
        for (;;) {
            const int j = next.fetch_add(1);
            if (j >= count) break;
            const int d = order[j];
            if (stat[d] != OTM_OK) continue;
            otm_ctx* ctx = ctxs[d];
            otm_status st = OTM_OK;
            bool noconv = false;
            otm_step_info last;
            memset(&last, 0, sizeof(last));
            for (int i = 0; st == OTM_OK && i < iters; ++i) {
                const otm_status s2 = otm_step(ctx, &last);
                if (infos) infos[(size_t)d * iters + i] = last;
                if (s2 == OTM_ENOCONV) noconv = true;
                else if (s2 != OTM_OK) st = s2;
            }
            if (st == OTM_OK && kappa_out)
                for (int c = 0; c < 6; ++c) kappa_out[d][c] = last.kappa[c];
            if (st == OTM_OK && rho_out && rho_out[d]) st = otm_get_density(ctx, rho_out[d], 0);
            if (st != OTM_OK) msgs[d] = otm_last_error(ctx);
            stat[d] = st != OTM_OK ? st : (noconv ? OTM_ENOCONV : OTM_OK);
        }
    };
    std::vector<std::thread> pool;
    for (int w = 1; w < workers; ++w) pool.emplace_back(work);
    work();
    for (auto& t : pool) t.join();
    otm_status first = OTM_OK;
    std::string first_msg;
    for (int d = 0; d < count; ++d) {
        if (stat[d] == OTM_ENOCONV && first == OTM_OK) first = OTM_ENOCONV;
        if (stat[d] != OTM_OK && stat[d] != OTM_ENOCONV && (first == OTM_OK || first == OTM_ENOCONV)) {
            first = stat[d];
            first_msg = "design " + std::to_string(d) + ": " + msgs[d];
        }
        otm_destroy(ctxs[d]);
    }
    if (first != OTM_OK && first != OTM_ENOCONV) g_err = "otm_design_batch: " + first_msg;
    return first;
}

otm_status otm_get_state(otm_ctx* ctx, void* buf, size_t* len) {
    CTX_CHECK(ctx);
    if (!len) return ctx_fail(ctx, OTM_EINVAL, "otm_get_state: len is NULL");
    const size_t need = ctx->s->state_size();
    if (!buf) {
        *len = need;
        return OTM_OK;
    }
    if (*len < need) return ctx_fail(ctx, OTM_EINVAL, "otm_get_state: buffer too small");
    *len = need;
    return ctx->s->get_state(buf);
}

otm_status otm_set_state(otm_ctx* ctx, const void* buf, size_t len) {
    CTX_CHECK(ctx);
    if (!buf) return ctx_fail(ctx, OTM_EINVAL, "otm_set_state: buf is NULL");
    return ctx->s->set_state(buf, len);
}

otm_status otm_set_predictor(otm_ctx* ctx, otm_unet* u, double scale) {
    CTX_CHECK(ctx);
    return ctx->s->set_predictor(u, scale);
}

const char* otm_last_error(const otm_ctx* ctx) {
    if (ctx && ctx->s) return ctx->s->err.c_str();
    return g_err.c_str();
}

otm_status otm_governor_init(otm_governor_state* s) {
    if (!s) return fail(OTM_EINVAL, "otm_governor_init: NULL");
    memset(s, 0, sizeof(*s));
    s->df = 1.0;
    s->vstar = 1.0;
    s->g_prev = 1.0;
    s->gap = 0.0;
    s->count = 0;
    return OTM_OK;
}

otm_status otm_governor_update(otm_governor_state* s, const otm_params* p, double g, double low_bound,
                               double vol) {
    if (!s || !p) return fail(OTM_EINVAL, "otm_governor_update: NULL");
    otm::GovState st;
    st.df = s->df;
    st.vstar = s->vstar;
    st.g_prev = s->g_prev;
    st.gap = s->gap;
    st.count = s->count;
    st.pad = 0;
    otm::GovParams gp{p->gov_bound, p->gov_small_rel, p->gov_vol_tol};
    otm::governor_update(st, gp, g, low_bound, vol);
    s->df = st.df;
    s->vstar = st.vstar;
    s->g_prev = st.g_prev;
    s->gap = st.gap;
    s->count = st.count;
    return OTM_OK;
}

}  // extern "C"
