// Design-loop kernels: density filter and SIMP (Sec. 2.2, 2.3), homogenized
// tensor and element sensitivities (discrete Eq. homo, Eq. sens), the OC
// update (Sec. 3.3) and the adaptive volume bound (Alg. 1).
#pragma once
#include "otm_internal.cuh"

namespace otm {

// Filter weights by squared offset length: d_e(x_i, r) = max(0, r - |o|) for
// |o| < r (Sec. 2.3, unit voxel volumes), offsets |o_d| <= R.
// The parameter blocks carry FP32 copies of their values (filled on the
// host by with_f32, the same roundings a kernel would make), so the FP32
// kernels never convert from FP64 per thread: FP64 conversions and
// arithmetic run at a small fraction of the FP32 rate on this part.
struct FilterW {
    int R;
    int pad;
    double w[13];        // by dx^2 + dy^2 + dz^2 (R <= 2 -> at most 12)
    double inv_wsum;
    float wf[13];
    float inv_wsum_f;
};

struct SimpP {
    double penal, k_solid, k_void;
    int cubic;           // penal == 3
    int pad;
    double sens_scale;   // (k_solid - k_void) / N of the sensitivity kernel
    float k_void_f, dk_f, sens_scale_f;
};

// value of the compute type C: the FP32 copy for float, else the FP64 value
template <class C>
__host__ __device__ __forceinline__ C par(double d, float f) {
    if (sizeof(C) == 4) return (C)f;
    return (C)d;
}
inline FilterW with_f32(FilterW fw) {
    for (int i = 0; i < 13; ++i) fw.wf[i] = (float)fw.w[i];
    fw.inv_wsum_f = (float)fw.inv_wsum;
    return fw;
}
inline SimpP with_f32(SimpP sp, size_t N) {
    sp.sens_scale = (sp.k_solid - sp.k_void) / (double)N;
    sp.k_void_f = (float)sp.k_void;
    sp.dk_f = (float)(sp.k_solid - sp.k_void);
    sp.sens_scale_f = (float)sp.sens_scale;
    return sp;
}

template <class C>
__device__ __forceinline__ C simp_pow(C r, const SimpP& sp) {
    if (sp.cubic) return r * r * r;
    return (C)pow((double)r, sp.penal);
}
template <class C>
__device__ __forceinline__ C simp_dpow(C r, const SimpP& sp) {   // d(r^p)/dr
    if (sp.cubic) return C(3) * r * r;
    return (C)(sp.penal * pow((double)r, sp.penal - 1.0));
}

struct FinFilter {
    DesignScalars* ds;
    __device__ void operator()(const double* s) const {
        ds->sum_rho = s[0];
        ds->sum_rhop = s[1];
    }
};

// out_e = sum_o w(o) in_{e + sgn*o} / sum w.  sgn = -1 is the transpose
// (scatter of each element to the neighbours it gathered from).  RR is the
// offset range (|o_d| <= RR), fixed at compile time so the loops unroll and
// the weights stay in registers.
template <class R, bool SIMP, int RR>
__global__ void __launch_bounds__(256)
k_filter(int n, FilterW fw, int sgn, const R* __restrict__ in, R* __restrict__ out, R* __restrict__ kout,
         SimpP sp, RedBuf rb, FinFilter fin) {
    pdl_enter();
    using C = typename St<R>::C;
    C w[13];
#pragma unroll
    for (int i = 0; i < 13; ++i) w[i] = par<C>(fw.w[i], fw.wf[i]);
    const C inv = par<C>(fw.inv_wsum, fw.inv_wsum_f);
    Acc<C> a_rho, a_rhop;
    OTM_FOR_ROWS(row_, n * n) {
    const int y = row_ % n, z = row_ / n;
    // 32-bit offsets: n^3 < 2^32 for every supported n
    unsigned zo[2 * RR + 1], yo[2 * RR + 1];
#pragma unroll
    for (int d = -RR; d <= RR; ++d) {
        zo[d + RR] = (unsigned)wrapd(z, sgn * d, n) * (unsigned)n * (unsigned)n;
        yo[d + RR] = (unsigned)wrapd(y, sgn * d, n) * (unsigned)n;
    }
    OTM_FOR_X(x, n) {
        const size_t v = (size_t)row_ * n + x;
        int xo[2 * RR + 1];
#pragma unroll
        for (int d = -RR; d <= RR; ++d) xo[d + RR] = wrapd(x, sgn * d, n);
        C acc = 0;
#pragma unroll
        for (int dz = -RR; dz <= RR; ++dz)
#pragma unroll
            for (int dy = -RR; dy <= RR; ++dy)
#pragma unroll
                for (int dx = -RR; dx <= RR; ++dx) {
                    const int d2 = dx * dx + dy * dy + dz * dz;
                    if (d2 > 12) continue;
                    acc += w[d2] * (C)in[(unsigned)xo[dx + RR] + yo[dy + RR] + zo[dz + RR]];
                }
        const C rf = acc * inv;
        out[v] = rf;
        if (SIMP) {
            const C rp = simp_pow(rf, sp);
            kout[v] = par<C>(sp.k_void, sp.k_void_f) + rp * par<C>(sp.k_solid - sp.k_void, sp.dk_f);
            a_rho.add(in[v]);
            a_rhop.add(rp);
        }
    }
    }
    if (SIMP) {
        __shared__ double res[2];
        const Acc<C> sums[2] = {a_rho, a_rhop};
        if (grid_reduce<2>(sums, rb, res)) {
            if (is_thread0()) fin(res);
        }
    }
}

// Dispatch on the filter's offset range.
template <class R, bool SIMP>
inline cudaError_t launch_filter(RowLaunch L, cudaStream_t st, int n, const FilterW& fw, int sgn, const R* in, R* out,
                                 R* kout, const SimpP& sp, RedBuf rb, FinFilter fin) {
    if (fw.R <= 0) return launch_pdl(k_filter<R, SIMP, 0>, L.grid, L.block, st, n, fw, sgn, in, out, kout, sp, rb, fin);
    if (fw.R == 1) return launch_pdl(k_filter<R, SIMP, 1>, L.grid, L.block, st, n, fw, sgn, in, out, kout, sp, rb, fin);
    return launch_pdl(k_filter<R, SIMP, 2>, L.grid, L.block, st, n, fw, sgn, in, out, kout, sp, rb, fin);
}

// Element energies E_c = d^i . K0 d^j, d^i_l = t^i_l - chi^i(corner l) with
// t^i_l the i-th coordinate bit of corner l, (K0 d)_l = (4 d_l - d_{l^3} -
// d_{l^5} - d_{l^6} - d_{l^7}) / 12; components c in the order of Eq. rep.
template <class R, class C>
__device__ __forceinline__ void element_energies(int n, size_t N, int x, int y, int z,
                                                 const R* __restrict__ chi, C (&E)[6]) {
    const int xp = wrapp(x, n), yp = wrapp(y, n), zp = wrapp(z, n);
    size_t idx[8];
#pragma unroll
    for (int l = 0; l < 8; ++l)
        idx[l] = (size_t)((l & 1) ? xp : x) + (size_t)n * (((l >> 1) & 1 ? yp : y) + (size_t)n * ((l >> 2) ? zp : z));
    C d[3][8], kd[3][8];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int l = 0; l < 8; ++l) d[i][l] = (C)((l >> i) & 1) - (C)chi[(size_t)i * N + idx[l]];
#pragma unroll
        for (int l = 0; l < 8; ++l)
            kd[i][l] = (C(4) * d[i][l] - d[i][l ^ 3] - d[i][l ^ 5] - d[i][l ^ 6] - d[i][l ^ 7]) * C(1.0 / 12.0);
    }
    const int ci[6] = {0, 1, 2, 0, 1, 0};
    const int cj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        C s = 0;
#pragma unroll
        for (int l = 0; l < 8; ++l) s += d[ci[c]][l] * kd[cj[c]][l];
        E[c] = s;
    }
}

// Objective value and gradient from kappa (Eq. mse, fracmse, l1).
__device__ inline void objective_eval(DesignScalars* ds) {
    double g = 0.0;
    for (int c = 0; c < 6; ++c) {
        const double kc = ds->kappa[c], tc = ds->target[c];
        double w;
        if (ds->objective == OTM_OBJ_FRACMSE) {
            if (tc != 0.0) {
                const double a = kc / tc - 1.0;
                g += a * a;
                w = 2.0 * a / tc;
            } else {
                g += kc * kc;
                w = 2.0 * kc;
            }
        } else if (ds->objective == OTM_OBJ_L1) {
            const double a = kc - tc;
            g += a < 0 ? -a : a;
            w = a > 0 ? 1.0 : (a < 0 ? -1.0 : 0.0);
        } else {
            const double a = kc - tc;
            g += a * a;
            w = 2.0 * a;
        }
        ds->w[c] = w;
    }
    ds->g = g;
}

struct FinKappa {
    DesignScalars* ds;
    double invN;
    int eval_objective;
    __device__ void operator()(const double* s) const {
        for (int c = 0; c < 6; ++c) ds->kappa[c] = s[c] * invN;
        if (eval_objective) objective_eval(ds);
    }
};

// kappa_c = (1/N) sum_e k_e E_c,e (FP64 sums).
template <class R>
__global__ void __launch_bounds__(256)
k_kappa(int n, const R* __restrict__ k, const R* __restrict__ chi, RedBuf rb, FinKappa fin) {
    pdl_enter();
    using C = typename St<R>::C;
    const size_t N = (size_t)n * n * n;
    Acc<C> acc[6];
    OTM_FOR_ROWS(row_, n * n) {
    const int y = row_ % n, z = row_ / n;
    OTM_FOR_X(x, n) {
        const size_t e = (size_t)row_ * n + x;
        C E[6];
        element_energies<R, C>(n, N, x, y, z, chi, E);
        const C ke = k[e];
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c].add_prod(ke, E[c]);
    }
    }
    __shared__ double res[6];
    if (grid_reduce<6>(acc, rb, res)) {
        if (is_thread0()) fin(res);
    }
}

// s_f,e = (1/N) p rho_f^(p-1) (k_solid - k_void) sum_c w_c E_c,e  (Eq. sens).
template <class R>
__global__ void __launch_bounds__(256)
k_sens(int n, const R* __restrict__ rho_f, const R* __restrict__ chi, const DesignScalars* __restrict__ ds,
       SimpP sp, R* __restrict__ s_f) {
    pdl_enter();
    using C = typename St<R>::C;
    const size_t N = (size_t)n * n * n;
    C w[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) w[c] = (C)ds->w[c];
    const C scale = par<C>(sp.sens_scale, sp.sens_scale_f);
    OTM_FOR_ROWS(row_, n * n) {
    const int y = row_ % n, z = row_ / n;
    OTM_FOR_X(x, n) {
        const size_t e = (size_t)row_ * n + x;
        C E[6];
        element_energies<R, C>(n, N, x, y, z, chi, E);
        C a = 0;
#pragma unroll
        for (int c = 0; c < 6; ++c) a += w[c] * E[c];
        s_f[e] = a * simp_dpow((C)rho_f[e], sp) * scale;
    }
    }
}

// Central symmetry (Sec. 4.1): average element e with N-1-e, the point
// reflection (x, y, z) -> (n-1-x, n-1-y, n-1-z), for rho and s.
template <class R>
__global__ void __launch_bounds__(256)
k_symmetrize(size_t N, R* __restrict__ rho, R* __restrict__ s) {
    pdl_enter();
    using C = typename St<R>::C;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < N / 2;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t f = N - 1 - e;
        const C a = C(0.5) * ((C)rho[e] + (C)rho[f]);
        rho[e] = a;
        rho[f] = a;
        const C b = C(0.5) * ((C)s[e] + (C)s[f]);
        s[e] = b;
        s[f] = b;
    }
}

// ------------------------------------------------------------------------
// OC update.  With mu = lambda^(-eta) and c_e = rho_e max(0, -s_e)^eta the
// new density clamp(rho_e (max(0,-s_e)/lambda)^eta, lo_e, hi_e) is
// clamp(c_e mu, lo_e, hi_e), lo_e = max(rho_min, rho_e - m),
// hi_e = min(1, rho_e + m); the volume is non-decreasing and piecewise linear
// in mu.  The search evaluates kOcCand candidate mu per pass over the field
// (geometric spacing, linear in the last pass), keeps the bracket where the
// volume crosses N V*, and interpolates linearly inside the final bracket.
// ------------------------------------------------------------------------
struct OcP {
    double move, damp, rho_min;
    int half;     // damp == 0.5
    int pad;
    float move_f, rho_min_f;
};
inline OcP with_f32(OcP op) {
    op.move_f = (float)op.move;
    op.rho_min_f = (float)op.rho_min;
    return op;
}

template <class C>
__device__ __forceinline__ void oc_elem(C rho, C s, const OcP& op, C& lo, C& hi, C& c) {
    const C mv = par<C>(op.move, op.move_f), rmin = par<C>(op.rho_min, op.rho_min_f);
    lo = rho - mv;
    if (lo < rmin) lo = rmin;
    hi = rho + mv;
    if (hi > C(1)) hi = C(1);
    const C B = s < C(0) ? -s : C(0);
    C bp;
    if (op.half) bp = sqrt(B);
    else bp = (C)pow((double)B, op.damp);
    c = rho * bp;
}

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

struct FinOcPrep {
    DesignScalars* ds;
    double N;
    __device__ void operator()(const double* s) const {
        ds->oc_vmin = s[0];
        ds->oc_vmax = s[1];
        const double target = ds->vstar * N;
        ds->oc_pass = 0;
        if (s[1] <= target) {
            ds->oc_mode = 1;
            ds->lambda = 0.0;
        } else if (s[0] > target) {
            ds->oc_mode = 2;
            ds->lambda = __longlong_as_double(0x7ff0000000000000LL);
        } else {
            ds->oc_mode = 0;
            const double mmin = __longlong_as_double((long long)__ldcg((const unsigned long long*)&ds->mu_min_seen));
            const double mmax = __longlong_as_double((long long)__ldcg((const unsigned long long*)&ds->mu_max_seen));
            ds->mu_lo = 0.5 * mmin;
            ds->mu_hi = 2.0 * mmax;
            ds->v_lo = s[0];
            ds->v_hi = s[1];
        }
    }
};

template <class R>
__global__ void __launch_bounds__(256)
k_oc_prep(size_t N, const R* __restrict__ rho, const R* __restrict__ s, OcP op, DesignScalars* ds,
          RedBuf rb, FinOcPrep fin) {
    pdl_enter();
    using C = typename St<R>::C;
    Acc<C> vmin, vmax;
    // per-element min / max in the compute type, widened once per warp
    // (exact: the conversion to double is monotone)
    bool seen = false;
    C mumin = 0, mumax = 0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < N;
         e += (size_t)gridDim.x * blockDim.x) {
        C lo, hi, c;
        oc_elem<C>(rho[e], s[e], op, lo, hi, c);
        vmin.add(lo);
        if (c > C(0)) {
            vmax.add(hi);
            const C ic = C(1) / c;
            const C a = lo * ic, b = hi * ic;
            mumin = (!seen || a < mumin) ? a : mumin;
            mumax = (!seen || b > mumax) ? b : mumax;
            seen = true;
        } else {
            vmax.add(lo);
        }
    }
    // warp min / max, then one atomic per warp (order-independent)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const bool s2 = __shfl_xor_sync(0xffffffffu, seen, o);
        const C a = __shfl_xor_sync(0xffffffffu, mumin, o);
        const C b = __shfl_xor_sync(0xffffffffu, mumax, o);
        if (s2) {
            mumin = (!seen || a < mumin) ? a : mumin;
            mumax = (!seen || b > mumax) ? b : mumax;
            seen = true;
        }
    }
    if ((threadIdx.x & 31) == 0 && seen) {
        atomicMin((unsigned long long*)&ds->mu_min_seen, dbits((double)mumin));
        if ((double)mumax > 0.0) atomicMax((unsigned long long*)&ds->mu_max_seen, dbits((double)mumax));
    }
    __shared__ double res[2];
    const Acc<C> sums[2] = {vmin, vmax};
    if (grid_reduce<2>(sums, rb, res)) {
        if (is_thread0()) fin(res);
    }
}

__device__ __forceinline__ double oc_candidate(const DesignScalars* ds, int j, int linear) {
    const double t = (double)(j + 1) / (double)(kOcCand + 1);
    if (linear) return ds->mu_lo + t * (ds->mu_hi - ds->mu_lo);
    return ds->mu_lo * pow(ds->mu_hi / ds->mu_lo, t);
}

struct FinOcSearch {
    DesignScalars* ds;
    double N;
    int linear, last;
    double inv_damp;
    __device__ void operator()(const double* s) const {
        const double target = ds->vstar * N;
        // largest candidate with volume <= target
        double a = ds->mu_lo, va = ds->v_lo, b = ds->mu_hi, vb = ds->v_hi;
        for (int j = 0; j < kOcCand; ++j) {
            const double m = oc_candidate(ds, j, linear);
            if (s[j] <= target) {
                a = m;
                va = s[j];
            } else {
                b = m;
                vb = s[j];
                break;
            }
        }
        ds->mu_lo = a;
        ds->v_lo = va;
        ds->mu_hi = b;
        ds->v_hi = vb;
        ds->oc_pass += 1;
        if (last) {
            double mu = vb > va ? a + (target - va) * (b - a) / (vb - va) : a;
            if (mu < a) mu = a;
            if (mu > b) mu = b;
            ds->mu_star = mu;
            ds->lambda = pow(mu, -inv_damp);
        }
    }
};

template <class R>
__global__ void __launch_bounds__(256)
k_oc_search(size_t N, const R* __restrict__ rho, const R* __restrict__ s, OcP op, DesignScalars* ds,
            int linear, RedBuf rb, FinOcSearch fin) {
    pdl_enter();
    using C = typename St<R>::C;
    if (ds->oc_mode != 0) return;   // uniform across the grid: no reduction needed
    __shared__ C cand[kOcCand];
    for (int j = threadIdx.x; j < kOcCand; j += blockDim.x) cand[j] = (C)oc_candidate(ds, j, linear);
    __syncthreads();
    C sum[kOcCand];
#pragma unroll
    for (int j = 0; j < kOcCand; ++j) sum[j] = 0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < N;
         e += (size_t)gridDim.x * blockDim.x) {
        C lo, hi, c;
        oc_elem<C>(rho[e], s[e], op, lo, hi, c);
#pragma unroll
        for (int j = 0; j < kOcCand; ++j) {
            C v = c * cand[j];
            v = v < lo ? lo : (v > hi ? hi : v);
            sum[j] += v;
        }
    }
    __shared__ double res[kOcCand];
    Acc<C> sums[kOcCand];
#pragma unroll
    for (int j = 0; j < kOcCand; ++j) sums[j].add(sum[j]);
    if (grid_reduce<kOcCand>(sums, rb, res)) {
        if (is_thread0()) fin(res);
    }
}

template <class R>
__global__ void __launch_bounds__(256)
k_oc_apply(size_t N, R* rho, const R* __restrict__ s, OcP op, const DesignScalars* __restrict__ ds) {
    pdl_enter();
    using C = typename St<R>::C;
    const int mode = ds->oc_mode;
    const C mu = (C)ds->mu_star;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < N;
         e += (size_t)gridDim.x * blockDim.x) {
        C lo, hi, c;
        oc_elem<C>(rho[e], s[e], op, lo, hi, c);
        C v;
        if (mode == 1) v = c > C(0) ? hi : lo;
        else if (mode == 2) v = lo;
        else {
            v = c * mu;
            v = v < lo ? lo : (v > hi ? hi : v);
        }
        rho[e] = v;   // in place: element e reads only its own old value
    }
}

// One thread: Alg. 1 (or the fixed bound), then reset the OC min/max slots.
static __global__ void k_governor(DesignScalars* ds, double invN, int use_fixed, double fixed_vstar) {
    pdl_enter();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (use_fixed) {
        ds->vstar = fixed_vstar;
    } else if (ds->governor_on) {
        governor_update(ds->gov, ds->govp, ds->g, ds->sum_rhop * invN, ds->sum_rho * invN);
        ds->vstar = ds->gov.vstar;
    }   // governor off: ds->vstar keeps the fixed bound set by the host
    ds->mu_min_seen = __longlong_as_double(0x7fefffffffffffffLL);
    ds->mu_max_seen = 0.0;
}

}  // namespace otm
