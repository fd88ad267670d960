// Method of Moving Asymptotes for model 2 (Eq. model2: minimise V(rho)
// subject to g(kappa^H, kappa*) <= eps, 0 <= rho <= 1), the optimizer the
// paper runs through MMAOptimizer(nconstraint, nvar, a0, a, c, d) (Sec. 3.3).
//
// The paper gives no formulas; this is Svanberg's method in its standard
// form with one constraint and a = 0 (so the variable z is zero and a0 plays
// no part): per variable, moving asymptotes L < x < U (widened by 1.2 where
// the last two steps agree in sign, narrowed by 0.7 where they disagree),
// move limits alpha <= x <= beta, and the convex separable approximations
// p / (U - x) + q / (x - L) of f0 = V and f1 = g - eps; the subproblem is
// solved through its dual in the one multiplier lambda.  For a fixed lambda
// every x_j has a closed form, so the dual derivative
//   phi(lambda) = r1 + sum_j h_j(x_j(lambda)) - max(0, (lambda - c) / d),
//   h_j(x) = p1_j / (U_j - x) + q1_j / (x - L_j),
// is one reduction over the design, and phi is non-increasing: lambda* = 0
// when phi(0) <= 0, else its root, found like the OC multiplier -- each
// search pass evaluates kMmaCand candidates in one read of the design and
// narrows the bracket (the first pass on a log scale, then linearly), and a
// last linear interpolation of phi gives lambda*.
//
// Device memory per design: the previous two iterates and the asymptotes
// (4 n^3 values); alpha, beta, p and q are recomputed from x, L, U and
// dg/drho in every pass instead of being stored.
#pragma once
#include <type_traits>

#include "otm_internal.cuh"

namespace otm {

constexpr int kMmaCand = 16;

struct MmaP {
    double xmin, xmax;   // box of model 2: 0 <= rho <= 1
    double move;         // move limit as a fraction of xmax - xmin (0.5)
    double c, d;         // penalty of the constraint's slack y: c y + d y^2 / 2
    double df0;          // dV/drho = 1 / n^3
    double eps;          // f1 = g - eps
};

template <class C>
struct MmaElem {
    C L, U, alpha, beta, p0, q0, p1, q1;
};

// alpha, beta, p and q from x and the asymptotes (every pass)
template <class C>
__device__ __forceinline__ void mma_coeffs(C x, C L, C U, C df1, const MmaP& mp, MmaElem<C>& e) {
    const C xmin = (C)mp.xmin, xmax = (C)mp.xmax, span = xmax - xmin;
    e.L = L;
    e.U = U;
    C a = L + C(0.1) * (x - L);
    a = a > xmin ? a : xmin;
    const C am = x - (C)mp.move * span;
    e.alpha = a > am ? a : am;
    C b = U - C(0.1) * (U - x);
    b = b < xmax ? b : xmax;
    const C bm = x + (C)mp.move * span;
    e.beta = b < bm ? b : bm;
    const C reg = C(1e-5) / span;
    const C ux2 = (U - x) * (U - x), xl2 = (x - L) * (x - L);
    const C g0 = (C)mp.df0;
    const C g0p = g0 > C(0) ? g0 : C(0), g0m = g0 < C(0) ? -g0 : C(0);
    const C g1p = df1 > C(0) ? df1 : C(0), g1m = df1 < C(0) ? -df1 : C(0);
    e.p0 = ux2 * (C(1.001) * g0p + C(0.001) * g0m + reg);
    e.q0 = xl2 * (C(0.001) * g0p + C(1.001) * g0m + reg);
    e.p1 = ux2 * (C(1.001) * g1p + C(0.001) * g1m + reg);
    e.q1 = xl2 * (C(0.001) * g1p + C(1.001) * g1m + reg);
}

// the asymptotes of iteration k from the two previous iterates
template <class C>
__device__ __forceinline__ void mma_asymptotes(int k, C x, C x1, C x2, C Lold, C Uold, const MmaP& mp, C& L, C& U) {
    const C span = (C)mp.xmax - (C)mp.xmin;
    if (k < 2) {
        L = x - C(0.5) * span;
        U = x + C(0.5) * span;
        return;
    }
    const C t = (x - x1) * (x1 - x2);
    const C gamma = t > C(0) ? C(1.2) : (t < C(0) ? C(0.7) : C(1));
    L = x - gamma * (x1 - Lold);
    U = x + gamma * (Uold - x1);
    const C lmin = x - C(10) * span, lmax = x - C(0.01) * span;
    const C umin = x + C(0.01) * span, umax = x + C(10) * span;
    L = L > lmin ? L : lmin;
    L = L < lmax ? L : lmax;
    U = U < umax ? U : umax;
    U = U > umin ? U : umin;
}

template <class C>
__device__ __forceinline__ C mma_x(C lam, const MmaElem<C>& e) {
    const C sp = sqrt(e.p0 + lam * e.p1), sq = sqrt(e.q0 + lam * e.q1);
    C x = (sp * e.L + sq * e.U) / (sp + sq);
    x = x > e.alpha ? x : e.alpha;
    return x < e.beta ? x : e.beta;
}
template <class C>
__device__ __forceinline__ C mma_h(C x, const MmaElem<C>& e) {
    return e.p1 / (e.U - x) + e.q1 / (x - e.L);
}

// h_j(x_j(lambda)) without a division per candidate: with r = (U - x) /
// (x - L), the unclamped minimiser has r = sqrt(P / Q), x = L + (U - L) /
// (1 + r) and h = (1 + r) (p1 / r + q1) / (U - L); the box alpha <= x <= beta
// is r_beta <= r <= r_alpha.  r and 1 / r both come from one reciprocal
// square root of P Q.
template <class C>
struct MmaFast {
    C p0, q0, p1, q1, iul;      // coefficients and 1 / (U - L)
    C ra, ira, rb, irb;         // r at alpha (largest) and beta (smallest), and their reciprocals
};
template <class C>
__device__ __forceinline__ void mma_fast(const MmaElem<C>& e, MmaFast<C>& f) {
    f.p0 = e.p0;
    f.q0 = e.q0;
    f.p1 = e.p1;
    f.q1 = e.q1;
    f.iul = C(1) / (e.U - e.L);
    f.ra = (e.U - e.alpha) / (e.alpha - e.L);
    f.ira = (e.alpha - e.L) / (e.U - e.alpha);
    f.rb = (e.U - e.beta) / (e.beta - e.L);
    f.irb = (e.beta - e.L) / (e.U - e.beta);
}
__device__ __forceinline__ float mma_rsqrt(float v) { return rsqrtf(v); }
__device__ __forceinline__ double mma_rsqrt(double v) { return rsqrt(v); }
template <class C>
__device__ __forceinline__ C mma_h_fast(C lam, const MmaFast<C>& f) {
    const C P = f.p0 + lam * f.p1, Q = f.q0 + lam * f.q1;
    const C rs = mma_rsqrt(P * Q);
    C r = P * rs, ir = Q * rs;
    if (r > f.ra) {
        r = f.ra;
        ir = f.ira;
    } else if (r < f.rb) {
        r = f.rb;
        ir = f.irb;
    }
    return (C(1) + r) * (f.p1 * ir + f.q1) * f.iul;
}

__device__ __forceinline__ double mma_phi(const DesignScalars* ds, double lam, double sum, const MmaP& mp) {
    const double y = lam > mp.c ? (lam - mp.c) / mp.d : 0.0;
    return ds->mma_r1 + sum - y;
}

// After the preparation pass: r1 from f1 = g - eps, phi(0), and the upper
// end of the bracket, past which phi < 0 for certain (h on [alpha, beta] is
// at most its larger endpoint value).
struct FinMmaPrep {
    DesignScalars* ds;
    MmaP mp;
    __device__ void operator()(const double* s) const {
        const double r1 = (ds->g - mp.eps) - s[0];
        ds->mma_r1 = r1;
        const double phi0 = r1 + s[1];
        ds->mma_lo = 0.0;
        ds->mma_phi_lo = phi0;
        const double fmax = r1 + s[2];
        ds->mma_hi = mp.c + mp.d * (fmax > 0.0 ? fmax : 0.0) + 1.0;
        ds->mma_phi_hi = -1.0;   // below zero by construction; replaced by the first measured value
        ds->mma_mode = phi0 <= 0.0 ? 1 : 0;
        ds->mma_lam = 0.0;
        ds->mma_pass = 0;
    }
};

// ds->mma_k is the iteration count of the asymptote rule (kept on the
// device, so a captured graph reads the current value).
template <class R>
__global__ void __launch_bounds__(256)
k_mma_prep(size_t N, const R* __restrict__ x, const R* __restrict__ x1, const R* __restrict__ x2, R* L, R* U,
           const R* __restrict__ s, MmaP mp, DesignScalars* ds, RedBuf rb, FinMmaPrep fin) {
    pdl_enter();
    using C = typename St<R>::C;
    const int k = ds->mma_k;
    Acc<C> a_h, a_h0, a_max;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (size_t)gridDim.x * blockDim.x) {
        const C xe = (C)x[e];
        C Le, Ue;
        mma_asymptotes<C>(k, xe, (C)x1[e], (C)x2[e], (C)L[e], (C)U[e], mp, Le, Ue);
        L[e] = (R)Le;   // in place: element e reads only its own old asymptotes
        U[e] = (R)Ue;
        MmaElem<C> m;
        mma_coeffs<C>(xe, Le, Ue, (C)s[e], mp, m);
        a_h.add(mma_h<C>(xe, m));
        a_h0.add(mma_h<C>(mma_x<C>(C(0), m), m));
        const C ha = mma_h<C>(m.alpha, m), hb = mma_h<C>(m.beta, m);
        a_max.add(ha > hb ? ha : hb);
    }
    __shared__ double res[3];
    const Acc<C> sums[3] = {a_h, a_h0, a_max};
    if (grid_reduce<3>(sums, rb, res)) {
        if (is_thread0()) fin(res);
    }
}

// Candidate j of a pass: pass 0 spans [hi 1e-12, hi] on a log scale (the
// multiplier's scale is not known in advance), later passes split the
// bracket (lo, hi) evenly.
__device__ __forceinline__ double mma_candidate(const DesignScalars* ds, int j, int logscale) {
    if (logscale) return ds->mma_hi * pow(10.0, -12.0 * (double)(kMmaCand - 1 - j) / (double)(kMmaCand - 1));
    return ds->mma_lo + (ds->mma_hi - ds->mma_lo) * (double)(j + 1) / (double)(kMmaCand + 1);
}

struct FinMmaSearch {
    DesignScalars* ds;
    MmaP mp;
    int logscale, last;
    __device__ void operator()(const double* s) const {
        double a = ds->mma_lo, pa = ds->mma_phi_lo, b = ds->mma_hi, pb = ds->mma_phi_hi;
        // the first candidate with phi <= 0 closes the bracket from above
        for (int j = 0; j < kMmaCand; ++j) {
            const double lam = mma_candidate(ds, j, logscale);
            const double ph = mma_phi(ds, lam, s[j], mp);
            if (ph > 0.0) {
                a = lam;
                pa = ph;
            } else {
                b = lam;
                pb = ph;
                break;
            }
        }
        ds->mma_lo = a;
        ds->mma_phi_lo = pa;
        ds->mma_hi = b;
        ds->mma_phi_hi = pb;
        ds->mma_pass += 1;
        if (last) {
            double lam = pa > pb ? a + pa * (b - a) / (pa - pb) : 0.5 * (a + b);
            lam = lam < a ? a : (lam > b ? b : lam);
            ds->mma_lam = lam;
        }
    }
};

template <class R>
__global__ void __launch_bounds__(256)
k_mma_search(size_t N, const R* __restrict__ x, const R* __restrict__ L, const R* __restrict__ U,
             const R* __restrict__ s, MmaP mp, DesignScalars* ds, int logscale, RedBuf rb, FinMmaSearch fin) {
    pdl_enter();
    using C = typename St<R>::C;
    if (ds->mma_mode != 0) return;   // uniform across the grid: no reduction needed
    __shared__ C cand[kMmaCand];
    for (int j = threadIdx.x; j < kMmaCand; j += blockDim.x) cand[j] = (C)mma_candidate(ds, j, logscale);
    __syncthreads();
    C sum[kMmaCand];
#pragma unroll
    for (int j = 0; j < kMmaCand; ++j) sum[j] = 0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (size_t)gridDim.x * blockDim.x) {
        MmaElem<C> m;
        const C xe = (C)x[e];
        mma_coeffs<C>(xe, (C)L[e], (C)U[e], (C)s[e], mp, m);
        MmaFast<C> f;
        mma_fast<C>(m, f);
#pragma unroll
        for (int j = 0; j < kMmaCand; ++j) sum[j] += mma_h_fast<C>(cand[j], f);
    }
    __shared__ double res[kMmaCand];
    Acc<C> sums[kMmaCand];
#pragma unroll
    for (int j = 0; j < kMmaCand; ++j) sums[j].add(sum[j]);
    if (grid_reduce<kMmaCand>(sums, rb, res)) {
        if (is_thread0()) fin(res);
    }
}

// x <- x(lambda*), the iterate history shifted (x2 <- x1 <- x), the
// iteration count advanced and lambda* reported.
template <class R>
__global__ void __launch_bounds__(256)
k_mma_apply(size_t N, R* x, R* x1, R* x2, const R* __restrict__ L, const R* __restrict__ U,
            const R* __restrict__ s, MmaP mp, DesignScalars* ds) {
    pdl_enter();
    using C = typename St<R>::C;
    const C lam = ds->mma_mode != 0 ? C(0) : (C)ds->mma_lam;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (size_t)gridDim.x * blockDim.x) {
        MmaElem<C> m;
        const C xe = (C)x[e];
        mma_coeffs<C>(xe, (C)L[e], (C)U[e], (C)s[e], mp, m);
        x2[e] = x1[e];
        x1[e] = (R)xe;
        x[e] = (R)mma_x<C>(lam, m);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {   // one thread of the grid
        ds->mma_k += 1;
        ds->lambda = (double)lam;
    }
}

// Search passes after the log-scale one: each narrows the bracket by
// kMmaCand + 1 = 17, so 12 reach the FP64 spacing of lambda and 6 are past
// FP32's before the final interpolation.
template <class R>
constexpr int mma_linear_passes() {
    return std::is_same<R, double>::value ? 12 : 6;
}

// One MMA iteration on the device: preparation (asymptotes, r1, phi(0) and
// the bracket), the search passes and the update; every kernel on `st`
// with programmatic dependent launch.  Returns the launch count.
template <class R>
inline int mma_enqueue(size_t N, R* x, R* x1, R* x2, R* L, R* U, const R* s, const MmaP& mp, DesignScalars* ds,
                       const RedBuf& rb, int grid, cudaStream_t st) {
    int launches = 0;
    launch_pdl(k_mma_prep<R>, grid, 256, st, N, (const R*)x, (const R*)x1, (const R*)x2, L, U, s, mp, ds, rb,
               FinMmaPrep{ds, mp});
    ++launches;
    const int passes = 1 + mma_linear_passes<R>();
    for (int pidx = 0; pidx < passes; ++pidx) {
        const int logscale = pidx == 0, last = pidx == passes - 1;
        launch_pdl(k_mma_search<R>, grid, 256, st, N, (const R*)x, (const R*)L, (const R*)U, s, mp, ds, logscale, rb,
                   FinMmaSearch{ds, mp, logscale, last});
        ++launches;
    }
    launch_pdl(k_mma_apply<R>, grid, 256, st, N, x, x1, x2, (const R*)L, (const R*)U, s, mp, ds);
    return launches + 1;
}

}  // namespace otm
