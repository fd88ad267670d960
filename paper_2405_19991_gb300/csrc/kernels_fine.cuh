// Finest-grid kernels of the matrix-free periodic conduction operator.
//
// Element matrix.  For the unit trilinear hexahedron with unit conductivity,
// K0 = K1(x)M1(x)M1 + M1(x)K1(x)M1 + M1(x)M1(x)K1 with the 1-D stiffness
// K1 = [[1,-1],[-1,1]] and mass M1 = [[1/3,1/6],[1/6,1/3]], so
// K0[l][m] = 1/3 (l = m), 0 (corners differing in one coordinate),
// -1/12 (differing in two or three).  Hence, for a vertex v at local corner l
// of element e, (K0 u_e)_l = (4 u_l - u_{l^3} - u_{l^5} - u_{l^6} - u_{l^7}) / 12
// and the assembled [K u]_v of Sec. 2.4 is a 21-point stencil: v, its 12
// edge-diagonal and 8 body-diagonal neighbours; face neighbours carry 0.
//
// Let k_abc be the conductivity of the element (x-a, y-b, z-c), a,b,c in
// {0,1}; it lies in the octant s = (1-2a, 1-2b, 1-2c) of v and couples v to
// v+(sx,sy,0), v+(sx,0,sz), v+(0,sy,sz), v+(sx,sy,sz).  Collecting terms:
//   12 [K u]_v = 4 u_v sum_abc k_abc - nb(u),
//   nb(u) = sum_abc k_abc u(v+s) + sum_ab (k_ab0 + k_ab1) u(v+(sx,sy,0))
//         + sum_ac (k_a0c + k_a1c) u(v+(sx,0,sz)) + sum_bc (k_0bc + k_1bc) u(v+(0,sy,sz)).
// The Gauss-Seidel update S_v T_v = f_v - M_v (Sec. 2.4) then has
// S_v = sum k_abc / 3 and M_v = -nb(T) / 12, i.e. T_v = (12 f_v + nb(T)) / (4 sum k).
//
// Nodes whose (y, z) parities agree are never coupled (their x-neighbours are
// face neighbours), so the paper's 8-colour order 0,1,...,7 with colour
// (x%2) + 2(y%2) + 4(z%2) equals four passes over the (y%2, z%2) groups
// {0,1}, {2,3}, {4,5}, {6,7}, bit for bit.
#pragma once
#include "otm_internal.cuh"

namespace otm {

struct Nbr {
    // per-node neighbour geometry
    int X[2], Y[2], Z[2];      // node offsets of x+s (a=0 -> +1, a=1 -> -1), times 1, n, n^2
    int Xe[2], Ye[2], Ze[2];   // element offsets of x-a
    int xc, yc, zc;            // x, y*n, z*n^2
};

__device__ __forceinline__ Nbr make_nbr(int x, int y, int z, int n) {
    Nbr g;
    if (!node_ok(x, y, z, n, kSiteFine)) x = y = z = 0;   // checking build: recorded, then clamped
    const int nn = n * n;
    const int xm = wrapm(x, n), xp = wrapp(x, n);
    const int ym = wrapm(y, n), yp = wrapp(y, n);
    const int zm = wrapm(z, n), zp = wrapp(z, n);
    g.X[0] = xp; g.X[1] = xm;
    g.Y[0] = yp * n; g.Y[1] = ym * n;
    g.Z[0] = zp * nn; g.Z[1] = zm * nn;
    g.Xe[0] = x; g.Xe[1] = xm;
    g.Ye[0] = y * n; g.Ye[1] = ym * n;
    g.Ze[0] = z * nn; g.Ze[1] = zm * nn;
    g.xc = x; g.yc = y * n; g.zc = z * nn;
    return g;
}

template <class KT, class C>
__device__ __forceinline__ void load_k8(const KT* __restrict__ k, const Nbr& g, C (&kk)[2][2][2]) {
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a)
                kk[c][b][a] = St<KT>::ld(k, (size_t)(g.Xe[a] + g.Ye[b] + g.Ze[c]));
}

template <class UT, class C>
__device__ __forceinline__ C nb_sum(const UT* __restrict__ u, const Nbr& g, const C (&kk)[2][2][2]) {
    C acc = 0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a)
                acc += kk[c][b][a] * (C)St<UT>::ld(u, (size_t)(g.X[a] + g.Y[b] + g.Z[c]));
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a)
            acc += (kk[0][b][a] + kk[1][b][a]) * (C)St<UT>::ld(u, (size_t)(g.X[a] + g.Y[b] + g.zc));
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int a = 0; a < 2; ++a)
            acc += (kk[c][0][a] + kk[c][1][a]) * (C)St<UT>::ld(u, (size_t)(g.X[a] + g.yc + g.Z[c]));
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
            acc += (kk[c][b][0] + kk[c][b][1]) * (C)St<UT>::ld(u, (size_t)(g.xc + g.Y[b] + g.Z[c]));
    return acc;
}

// nb_sum split into its loads (in use order) and its arithmetic, so a
// caller can issue the loads of several load cases before any of the sums.
template <class UT, class C>
__device__ __forceinline__ void nb_load(const UT* __restrict__ u, const Nbr& g, C (&w)[20]) {
    int t = 0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) w[t++] = (C)St<UT>::ld(u, (size_t)(g.X[a] + g.Y[b] + g.Z[c]));
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) w[t++] = (C)St<UT>::ld(u, (size_t)(g.X[a] + g.Y[b] + g.zc));
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int a = 0; a < 2; ++a) w[t++] = (C)St<UT>::ld(u, (size_t)(g.X[a] + g.yc + g.Z[c]));
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b) w[t++] = (C)St<UT>::ld(u, (size_t)(g.xc + g.Y[b] + g.Z[c]));
}
template <class C>
__device__ __forceinline__ C nb_from(const C (&w)[20], const C (&kk)[2][2][2]) {
    C acc = 0;
    int t = 0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) acc += kk[c][b][a] * w[t++];
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) acc += (kk[0][b][a] + kk[1][b][a]) * w[t++];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int a = 0; a < 2; ++a) acc += (kk[c][0][a] + kk[c][1][a]) * w[t++];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b) acc += (kk[c][b][0] + kk[c][b][1]) * w[t++];
    return acc;
}

// Difference form of the same sum: nd(u) = sum coef (u_w - u_v) = nb(u) - 4 sum(k) u_v,
// so 12 [K u]_v = -nd(u).  Constant fields cancel exactly, which keeps the
// rounding error of K u proportional to the local differences of u instead
// of to |u|.  The terms are summed plane by plane -- the eight neighbours in
// the plane below (c = 1: body diagonals, x-z, y-z edge diagonals), the four
// in-plane edge diagonals, then the eight in the plane above (c = 0) -- the
// order in which the TMA-staged form (kernels_tma.cuh) meets them while it
// marches in z; every stencil form sums in this order.
template <class UT, class C>
__device__ __forceinline__ C nd_sum(const UT* __restrict__ u, const Nbr& g, const C (&kk)[2][2][2], C uc) {
    C acc = 0;
    auto plane = [&](int c) {
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a)
                acc += kk[c][b][a] * ((C)St<UT>::ld(u, (size_t)(g.X[a] + g.Y[b] + g.Z[c])) - uc);
#pragma unroll
        for (int a = 0; a < 2; ++a)
            acc += (kk[c][0][a] + kk[c][1][a]) * ((C)St<UT>::ld(u, (size_t)(g.X[a] + g.yc + g.Z[c])) - uc);
#pragma unroll
        for (int b = 0; b < 2; ++b)
            acc += (kk[c][b][0] + kk[c][b][1]) * ((C)St<UT>::ld(u, (size_t)(g.xc + g.Y[b] + g.Z[c])) - uc);
    };
    plane(1);
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a)
            acc += (kk[0][b][a] + kk[1][b][a]) * ((C)St<UT>::ld(u, (size_t)(g.X[a] + g.Y[b] + g.zc)) - uc);
    plane(0);
    return acc;
}

// nd of a field held as hi + lo (lo may be null): each difference is formed
// from the pair and rounded once.
template <class C>
__device__ __forceinline__ C nd_sum2(const C* __restrict__ hi, const C* __restrict__ lo, const Nbr& g,
                                     const C (&kk)[2][2][2], size_t v) {
    const C hv = hi[v], lv = lo ? lo[v] : C(0);
    auto D = [&](size_t w) -> C { return df_diff(hi[w], lo ? lo[w] : C(0), hv, lv); };
    C acc = 0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) acc += kk[c][b][a] * D((size_t)(g.X[a] + g.Y[b] + g.Z[c]));
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) acc += (kk[0][b][a] + kk[1][b][a]) * D((size_t)(g.X[a] + g.Y[b] + g.zc));
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int a = 0; a < 2; ++a) acc += (kk[c][0][a] + kk[c][1][a]) * D((size_t)(g.X[a] + g.yc + g.Z[c]));
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b) acc += (kk[c][b][0] + kk[c][b][1]) * D((size_t)(g.xc + g.Y[b] + g.Z[c]));
    return acc;
}

// Convergence check, element form: nd(u) = sum over the node's eight
// elements e of k_e d_e, with d_e = (u_a + u_b + u_c + u_d) - 4 u_v over the
// four corners of e that v couples to (the three face diagonals and the body
// diagonal; the edge neighbours carry K^0 = 0).  Each u = hi + lo.  d_e is
// held unrounded as t + sg: the four high parts are summed with TwoSum and
// 4 hv subtracted with TwoSum (4 hv is exact), the TwoSum errors and the low
// parts going into sg.  k_e d_e = TwoProduct(k_e, t) + k_e sg, summed with
// TwoSum into (s, c).  The result is nd of the stored k and hi + lo with an
// error of order eps^2 of the terms (the pair form below rounds each of the
// 20 differences once: order eps).  The corners of element (a, b, cz) are
// taken in the order (xc, Y[b], Z[cz]), (X[a], Y[b], Z[cz]), (X[a], Y[b],
// zc), (X[a], yc, Z[cz]), the elements with a fastest, then b, then cz.
template <class C>
__device__ __forceinline__ void elem_add(C& t, C& sg, C h, C l) {
    C u, e;
    two_sum(t, h, u, e);
    t = u;
    sg = sg + (e + l);
}
// t - 4 hv with the error and - 4 lv into sg (two_sum(t, -h4), written with
// subtractions as in df_diff)
template <class C>
__device__ __forceinline__ void elem_sub4(C& t, C& sg, C h4, C l4) {
    const C u = t - h4;
    const C bp = u - t;
    const C e = (t - (u - bp)) - (h4 + bp);
    t = u;
    sg = sg + (e - l4);
}
template <class C>
__device__ __forceinline__ void elem_term(C& s, C& c, C kv, C t, C sg) {
    const C p = mul_rn(kv, t);
    const C pe = fma(kv, sg, fma(kv, t, -p));
    C u, e;
    two_sum(s, p, u, e);
    s = u;
    c = c + (e + pe);
}
template <class C>
__device__ __forceinline__ void nd_sum_elem(const C* __restrict__ hi, const C* __restrict__ lo, const Nbr& g,
                                            const C (&kk)[2][2][2], size_t v, C& s_out, C& c_out) {
    const C h4 = C(4) * hi[v], l4 = lo ? C(4) * lo[v] : C(0);
    C s = 0, c = 0;
    auto H = [&](size_t w) -> C { return hi[w]; };
    auto L = [&](size_t w) -> C { return lo ? lo[w] : C(0); };
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const size_t w0 = (size_t)(g.xc + g.Y[b] + g.Z[cz]);
                C t = H(w0), sg = L(w0);
                const size_t w1 = (size_t)(g.X[a] + g.Y[b] + g.Z[cz]);
                elem_add(t, sg, H(w1), L(w1));
                const size_t w2 = (size_t)(g.X[a] + g.Y[b] + g.zc);
                elem_add(t, sg, H(w2), L(w2));
                const size_t w3 = (size_t)(g.X[a] + g.yc + g.Z[cz]);
                elem_add(t, sg, H(w3), L(w3));
                elem_sub4(t, sg, h4, l4);
                elem_term(s, c, kk[cz][b][a], t, sg);
            }
    s_out = s;
    c_out = c;
}

// r = f + (s + c) / 12 for the check: 1/12 as the double-float th + tl (th
// the rounded 1/12, tl its remainder), so the scaling is the exact
// operator's (the rounded 1/12 alone is 3e-8 high in FP32, comparable with
// a converged residual); TwoSum of f and s th, the product's error, s tl and
// c th in the small part, one rounding of the final sum.
template <class C>
__device__ __forceinline__ C resid_exact12(C fv, C s, C c) {
    constexpr C th = C(1.0 / 12.0);
    constexpr C tl = C(1.0 / 12.0 - (double)C(1.0 / 12.0));
    const C s12 = mul_rn(s, th);
    C t, e;
    two_sum(fv, s12, t, e);
    return t + (e + (fma(s, th, -s12) + fma(s, tl, c * th)));
}

// Pair form of the check (the warp-row kernel's OTM_CHECK_FORM=pair, for
// comparisons): every one of the 32 element terms k_e (u_w - u_v) with the
// difference rounded once (df_diff), formed with TwoProduct and summed with
// TwoSum.
template <class C>
__device__ __forceinline__ void nd_sum_exact(const C* __restrict__ hi, const C* __restrict__ lo, const Nbr& g,
                                             const C (&kk)[2][2][2], size_t v, C& s_out, C& c_out) {
    const C hv = hi[v], lv = lo ? lo[v] : C(0);
    C s = 0, c = 0;
    auto term = [&](C kv, C d) {
        const C p = mul_rn(kv, d);
        const C pe = fma(kv, d, -p);
        C t, e;
        two_sum(s, p, t, e);
        s = t;
        c += e + pe;
    };
    auto D = [&](size_t w) -> C { return df_diff(hi[w], lo ? lo[w] : C(0), hv, lv); };
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) term(kk[cz][b][a], D((size_t)(g.X[a] + g.Y[b] + g.Z[cz])));
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const C d = D((size_t)(g.X[a] + g.Y[b] + g.zc));
            term(kk[0][b][a], d);
            term(kk[1][b][a], d);
        }
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const C d = D((size_t)(g.X[a] + g.yc + g.Z[cz]));
            term(kk[cz][0][a], d);
            term(kk[cz][1][a], d);
        }
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const C d = D((size_t)(g.xc + g.Y[b] + g.Z[cz]));
            term(kk[cz][b][0], d);
            term(kk[cz][b][1], d);
        }
    s_out = s;
    c_out = c;
}

template <class C>
__device__ __forceinline__ C ksum8(const C (&kk)[2][2][2]) {
    C s = 0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) s += kk[c][b][a];
    return s;
}

// ----------------------------------------------------------------- finalisers
struct FinNone {
    __device__ void operator()(const double*) const {}
};

// alpha_i = gamma_i / (p_i . K p_i) for active load cases.
struct FinAlpha {
    PcgScalars* ps;
    __device__ void operator()(const double* s) const {
        for (int i = 0; i < 3; ++i) {
            ps->pq[i] = s[i];
            double a = 0.0;
            if (ps->active[i]) {
                if (s[i] > 0.0 && isfinite(s[i]) && isfinite(ps->gamma[i])) {
                    a = ps->gamma[i] / s[i];
                } else {
                    ps->breakdown |= (1 << i);
                    ps->active[i] = 0;
                }
            }
            ps->alpha[i] = a;
        }
    }
};

// Initial residual: record ||f||^2 and ||r||^2, set the active flags (from
// this residual, or with use_true from the last error-free check).
struct FinInit {
    PcgScalars* ps;
    int use_true;
    __device__ void operator()(const double* s) const {
        int na = 0;
        for (int i = 0; i < 3; ++i) {
            ps->rr[i] = s[i];
            ps->ff[i] = s[3 + i];
            ps->iters[i] = 0;
            ps->alpha[i] = ps->beta[i] = 0.0;
            const bool act = use_true ? (ps->true_ff[i] > 0.0 && ps->true_rr[i] > ps->tol2 * ps->true_ff[i])
                                      : (s[3 + i] > 0.0 && s[i] > ps->tol2 * s[3 + i]);
            ps->active[i] = act ? 1 : 0;
            na += act;
        }
        ps->breakdown = 0;
        ps->nactive = na;
        ps->first = 1;
    }
};

// After x += alpha p, r -= alpha q: convergence test on the recurrence residual.
struct FinResid {
    PcgScalars* ps;
    __device__ void operator()(const double* s) const {
        int na = 0;
        for (int i = 0; i < 3; ++i) {
            ps->rz_old[i] = s[3 + i];
            if (ps->active[i]) {
                ps->rr[i] = s[i];
                ps->iters[i] += 1;
                if (!(s[i] > ps->tol2 * ps->ff[i])) ps->active[i] = 0;
                if (!isfinite(s[i])) {
                    ps->active[i] = 0;
                    ps->breakdown |= (1 << i);
                }
            }
            na += ps->active[i];
        }
        ps->nactive = na;
        ps->total += 1;
    }
};

// gamma_new = r . z; beta = (gamma_new - [flexible] r.z_old) / gamma_old.
// The first beta after a pass's residual is 0 (p = z).
struct FinBeta {
    PcgScalars* ps;
    __device__ void operator()(const double* s) const {
        const int first = ps->first;
        ps->pfirst = first;
        ps->first = 0;
        for (int i = 0; i < 3; ++i) {
            double b = 0.0;
            if (!first && ps->active[i] && ps->gamma[i] != 0.0) {
                const double num = ps->flexible ? s[i] - ps->rz_old[i] : s[i];
                b = num / ps->gamma[i];
                if (!isfinite(b)) b = 0.0;
            }
            ps->beta[i] = b;
            if (first || ps->active[i]) ps->gamma[i] = s[i];
        }
    }
};

// ------------------------------------------------------------------ kernels

// out_i = K(k) u_i  (MODE 0) or out_i = f_i - K(k) u_i (MODE 1), i = 0..2,
// evaluated in the difference form.  With DOT, MODE 0 reduces u_i . out_i;
// MODE 1 reduces out_i . out_i and f_i . f_i.  MODE 2 is MODE 1 without the
// store (residual norms only), evaluated in the compute type CT.
template <int MODE, bool DOT, class KT, class UT, class FT, class OT, class Fin,
          class CT = typename St<OT>::C>
__global__ void __launch_bounds__(256)
k_stencil_apply(int n, const KT* __restrict__ k, const UT* __restrict__ u, const FT* __restrict__ f,
                OT* __restrict__ out, RedBuf rb, Fin fin) {
    pdl_enter();
    using C = CT;
    const size_t N = (size_t)n * n * n;
    Acc<C> acc[6];
    OTM_FOR_ROWS(row, n * n) {
    const int y = row % n, z = row / n;
    OTM_FOR_X(x, n) {
        const size_t v = (size_t)row * n + x;
        const Nbr g = make_nbr(x, y, z, n);
        C kk[2][2][2];
        load_k8<KT, C>(k, g, kk);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const UT* ui = u + (size_t)i * N;
            const C uc = (C)St<UT>::ld(ui, v);
            const C Ku = nd_sum<UT, C>(ui, g, kk, uc) * C(-1.0 / 12.0);
            C o;
            if (MODE == 0) {
                o = Ku;
            } else {
                const C fv = (C)St<FT>::ld(f + (size_t)i * N, v);
                o = fv - Ku;
                if (DOT) acc[3 + i].add_prod(fv, fv);
            }
            if (MODE != 2) St<OT>::st(out + (size_t)i * N, v, (typename St<OT>::C)o);
            if (DOT) {
                if (MODE == 0) acc[i].add_prod(uc, o);
                else acc[i].add_prod(o, o);
            }
        }
    }
    }
    if (DOT) {
        __shared__ double res[6];
        if (grid_reduce<6>(acc, rb, res)) {
            if (is_thread0()) fin(res);
        }
    }
}

// r_i = f_i - K x_i with x held as hi + lo (lo may be null); reduces
// ||r_i||^2 and ||f_i||^2 and sets the active flags (FinInit).
template <class R, class Fin>
__global__ void __launch_bounds__(256)
k_residual_x2(int n, const R* __restrict__ k, const R* __restrict__ xh, const R* __restrict__ xl,
              const R* __restrict__ f, R* __restrict__ r, RedBuf rb, Fin fin) {
    pdl_enter();
    using C = typename St<R>::C;
    const size_t N = (size_t)n * n * n;
    Acc<C> acc[6];
    OTM_FOR_ROWS(row, n * n) {
    const int y = row % n, z = row / n;
    OTM_FOR_X(x, n) {
        const size_t v = (size_t)row * n + x;
        const Nbr g = make_nbr(x, y, z, n);
        C kk[2][2][2];
        load_k8<R, C>(k, g, kk);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const size_t o = (size_t)i * N;
            const C fv = f[o + v];
            const C rv = fv + nd_sum2<C>(xh + o, xl ? xl + o : nullptr, g, kk, v) * C(1.0 / 12.0);
            r[o + v] = rv;
            acc[i].add_prod(rv, rv);
            acc[3 + i].add_prod(fv, fv);
        }
    }
    }
    __shared__ double res[6];
    if (grid_reduce<6>(acc, rb, res)) {
        if (is_thread0()) fin(res);
    }
}

// Convergence check (k_true_residual below): ||f_i - K x_i||^2 of the
// stored iterate with error-free element terms (nd_sum_elem; no FP64
// arithmetic on the FP32 paths).

// True residual norms at solver exit.
struct FinTrue {
    PcgScalars* ps;
    __device__ void operator()(const double* s) const {
        for (int i = 0; i < 3; ++i) {
            ps->true_rr[i] = s[i];
            ps->true_ff[i] = s[3 + i];
        }
    }
};

template <class R, class Fin = FinTrue>
__global__ void __launch_bounds__(256)
k_true_residual(int n, const R* __restrict__ k, const R* __restrict__ xh, const R* __restrict__ xl,
                const R* __restrict__ f, RedBuf rb, Fin fin) {
    pdl_enter();
    using C = typename St<R>::C;
    const size_t N = (size_t)n * n * n;
    Acc<C> acc[6];
    OTM_FOR_ROWS(row, n * n) {
    const int y = row % n, z = row / n;
    OTM_FOR_X(x, n) {
        const size_t v = (size_t)row * n + x;
        const Nbr g = make_nbr(x, y, z, n);
        C kk[2][2][2];
        load_k8<R, C>(k, g, kk);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const size_t o = (size_t)i * N;
            C s, c;
            nd_sum_elem<C>(xh + o, xl ? xl + o : nullptr, g, kk, v, s, c);
            // r = f + nd / 12, nd = s + c; one rounding of the final sum
            const C fv = f[o + v];
            const C rv = resid_exact12<C>(fv, s, c);
            acc[i].add_prod(rv, rv);
            acc[3 + i].add_prod(fv, fv);
        }
    }
    }
    __shared__ double res[6];
    if (grid_reduce<6>(acc, rb, res)) {
        if (is_thread0()) fin(res);
    }
}

// Grid of the fine Gauss-Seidel pass: OTM_GS_GRID blocks overrides the
// caller's choice (0 = keep it).
inline int gs_grid_cap() {
    const char* e = getenv("OTM_GS_GRID");
    return e ? std::max(atoi(e), 0) : 0;
}

// One Gauss-Seidel pass over the nodes with y%2 == group&1, z%2 == group>>1
// and, when xpar >= 0, x%2 == xpar.  ZERO: the relaxed field starts at zero;
// the pass also zeroes the other nodes of each 2x2 (y, z) cell, so no
// separate clear is needed (only valid for group 0, xpar < 0).
template <bool ZERO, class KT, class FT, class TT>
__global__ void __launch_bounds__(256)
k_gs_fine(int n, int group, int xpar, const KT* __restrict__ k, const FT* __restrict__ f,
          TT* __restrict__ T) {
    pdl_enter();
    using C = typename St<TT>::C;
    const size_t N = (size_t)n * n * n;
    const int h = n >> 1;
    const int nx = xpar < 0 ? n : h;
    const int yo = group & 1, zo = group >> 1;
    OTM_FOR_ROWS(grow, h * h) {
    const int y = 2 * (grow % h) + yo, z = 2 * (grow / h) + zo;
    OTM_FOR_X(xi, nx) {
        const int x = xpar < 0 ? xi : 2 * xi + xpar;
        const Nbr g = make_nbr(x, y, z, n);
        C kk[2][2][2];
        load_k8<KT, C>(k, g, kk);
        const C inv4k = C(1) / (C(4) * ksum8(kk));
        const size_t v = (size_t)(g.xc + g.yc + g.zc);
        // all three load cases' neighbour values in flight before any sum
        // (the stores below could alias them as far as the compiler knows)
        C w[3][20];
        if (!ZERO) {
#pragma unroll
            for (int i = 0; i < 3; ++i) nb_load<TT, C>(T + (size_t)i * N, g, w[i]);
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            TT* Ti = T + (size_t)i * N;
            const C fv = St<FT>::ld(f + (size_t)i * N, v);
            C nb = 0;
            if (!ZERO) nb = nb_from<C>(w[i], kk);
            St<TT>::st(Ti, v, (C(12) * fv + nb) * inv4k);
            if (ZERO) {
                const size_t y1 = (size_t)(y + 1) * n, z1 = (size_t)(z + 1) * n * n;
                St<TT>::st(Ti, x + y1 + g.zc, C(0));
                St<TT>::st(Ti, x + g.yc + z1, C(0));
                St<TT>::st(Ti, x + y1 + z1, C(0));
            }
        }
    }
    }
}

// enforceMacroLoad (Sec. 2.4).  The template f0 = K0 T0 with T0[l][i] = i-th
// coordinate of corner l is +1/4 on the upper face of axis i and -1/4 on the
// lower face (from the K0 row formula above), so
// f^(i)_v = (sum of k over the four elements below v along axis i
//           - sum over the four above) / 4.
template <class KT, class OT>
__global__ void __launch_bounds__(256)
k_macro_load(int n, const KT* __restrict__ k, OT* __restrict__ f) {
    pdl_enter();
    using C = typename St<OT>::C;
    const size_t N = (size_t)n * n * n;
    OTM_FOR_ROWS(row, n * n) {
    const int y = row % n, z = row / n;
    OTM_FOR_X(x, n) {
        const size_t v = (size_t)row * n + x;
        const Nbr g = make_nbr(x, y, z, n);
        C kk[2][2][2];
        load_k8<KT, C>(k, g, kk);
        C fx = 0, fy = 0, fz = 0;
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const C kv = kk[c][b][a];
                    fx += a ? kv : -kv;
                    fy += b ? kv : -kv;
                    fz += c ? kv : -kv;
                }
        St<OT>::st(f, v, C(0.25) * fx);
        St<OT>::st(f + N, v, C(0.25) * fy);
        St<OT>::st(f + 2 * N, v, C(0.25) * fz);
    }
    }
}

// The periodic operator annihilates constants, so K x = f is solvable only
// for zero-mean f; FP32 rounding of the macro loads leaves a small mean that
// would floor the residual.  Sum, then subtract the mean.
struct FinMean {
    PcgScalars* ps;
    double invN;
    __device__ void operator()(const double* s) const {
        for (int i = 0; i < 3; ++i) ps->fmean[i] = s[i] * invN;
    }
};

template <class R>
__global__ void __launch_bounds__(256)
k_sum3(size_t N, const R* __restrict__ f, RedBuf rb, FinMean fin) {
    pdl_enter();
    using C = typename St<R>::C;
    Acc<C> acc[3];
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
         v += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < 3; ++i) acc[i].add(f[(size_t)i * N + v]);
    }
    __shared__ double res[3];
    if (grid_reduce<3>(acc, rb, res)) {
        if (is_thread0()) fin(res);
    }
}

template <class R>
__global__ void __launch_bounds__(256)
k_sub_mean(size_t N, R* __restrict__ f, const PcgScalars* __restrict__ ps) {
    pdl_enter();
    using C = typename St<R>::C;
    const C m0 = (C)ps->fmean[0], m1 = (C)ps->fmean[1], m2 = (C)ps->fmean[2];
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
         v += (size_t)gridDim.x * blockDim.x) {
        f[v] -= m0;
        f[N + v] -= m1;
        f[2 * N + v] -= m2;
    }
}

// Restriction R = P^T of the trilinear prolongation: coarse node I gathers
// the fine nodes 2I + d, d in {-1,0,1}^3, with weight prod (1 - |d|/2).
// Restriction R = P^T: coarse node I gathers the 27 fine nodes around 2I with
// weights w(dx) w(dy) w(dz), w = (1/2, 1, 1/2).  The fine residual is read
// load-case-major ([3][Nf], the finest level) or node-major ([Nf][4], IN_AOS);
// the coarse right-hand side is written node-major.
template <class IT, class OT, bool IN_AOS>
__device__ __forceinline__ void restrict_node(int nc, int X, int Y, int Z, const IT* __restrict__ rf,
                                              OT* __restrict__ fc) {
    using C = typename St<OT>::C;
    using CI = typename St<IT>::C;
    if (!node_ok(X, Y, Z, nc, kSiteCoarse)) return;
    const int nf = 2 * nc;
    const size_t Nf = (size_t)nf * nf * nf;
    const size_t I = (size_t)X + (size_t)nc * (Y + (size_t)nc * Z);
    int xs[3], ys[3], zs[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        xs[d] = wrapd(2 * X, d - 1, nf);
        ys[d] = wrapd(2 * Y, d - 1, nf) * nf;
        zs[d] = wrapd(2 * Z, d - 1, nf) * nf * nf;
    }
    const C w1[3] = {C(0.5), C(1), C(0.5)};
    C acc[3] = {C(0), C(0), C(0)};
#pragma unroll
    for (int dz = 0; dz < 3; ++dz) {
        C az[3] = {C(0), C(0), C(0)};
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            C ay[3] = {C(0), C(0), C(0)};
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                CI t[3];
                ld_f3_any<IN_AOS, IT>(rf, Nf, (size_t)(xs[dx] + ys[dy] + zs[dz]), t);
#pragma unroll
                for (int i = 0; i < 3; ++i) ay[i] += w1[dx] * (C)t[i];
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) az[i] += w1[dy] * ay[i];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) acc[i] += w1[dz] * az[i];
    }
    st_f3<OT>(fc, I, acc[0], acc[1], acc[2]);
}

template <class IT, class OT, bool IN_AOS>
__global__ void __launch_bounds__(256)
k_restrict(int nc, const IT* __restrict__ rf, OT* __restrict__ fc) {
    pdl_enter();
    OTM_FOR_ROWS(row, nc * nc) {
        const int Y = row % nc, Z = row / nc;
        OTM_FOR_X(X, nc) restrict_node<IT, OT, IN_AOS>(nc, X, Y, Z, rf, fc);
    }
}

// Prolongation and correction: T_v += sum_I P[v, I] Tc_I (trilinear).  The
// coarse field is node-major; the fine one is node-major (OUT_AOS, a coarse
// level) or load-case-major (the finest level).
template <class CT, class TT, bool OUT_AOS>
__device__ __forceinline__ void prolong_node(int nf, int x, int y, int z, const CT* __restrict__ Tc,
                                             TT* __restrict__ T) {
    using C = typename St<TT>::C;
    using CC = typename St<CT>::C;
    if (!node_ok(x, y, z, nf, kSiteCoarse)) return;
    const int nc = nf / 2;
    const size_t Nf = (size_t)nf * nf * nf;
    const size_t v = (size_t)x + (size_t)nf * (y + (size_t)nf * z);
    int xi[2], yi[2], zi[2];
    C wx[2], wy[2], wz[2];
    int cx, cy, cz;
    if (x & 1) { xi[0] = x >> 1; xi[1] = wrapp(x >> 1, nc); wx[0] = wx[1] = C(0.5); cx = 2; }
    else { xi[0] = xi[1] = x >> 1; wx[0] = C(1); wx[1] = 0; cx = 1; }
    if (y & 1) { yi[0] = y >> 1; yi[1] = wrapp(y >> 1, nc); wy[0] = wy[1] = C(0.5); cy = 2; }
    else { yi[0] = yi[1] = y >> 1; wy[0] = C(1); wy[1] = 0; cy = 1; }
    if (z & 1) { zi[0] = z >> 1; zi[1] = wrapp(z >> 1, nc); wz[0] = wz[1] = C(0.5); cz = 2; }
    else { zi[0] = zi[1] = z >> 1; wz[0] = C(1); wz[1] = 0; cz = 1; }
    C acc[3] = {C(0), C(0), C(0)};
    for (int c = 0; c < cz; ++c)
        for (int b = 0; b < cy; ++b)
            for (int a = 0; a < cx; ++a) {
                CC t[3];
                ld_f3<CT>(Tc, (size_t)xi[a] + (size_t)nc * (yi[b] + (size_t)nc * zi[c]), t);
                const C w = wz[c] * wy[b] * wx[a];
#pragma unroll
                for (int i = 0; i < 3; ++i) acc[i] += w * (C)t[i];
            }
    if (OUT_AOS) {
        C t0[3];
        ld_f3<TT>(T, v, t0);
        st_f3<TT>(T, v, t0[0] + acc[0], t0[1] + acc[1], t0[2] + acc[2]);
    } else {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            TT* t = T + (size_t)i * Nf;
            St<TT>::st(t, v, St<TT>::ld(t, v) + acc[i]);
        }
    }
}

template <class CT, class TT, bool OUT_AOS>
__global__ void __launch_bounds__(256)
k_prolong_add(int nf, const CT* __restrict__ Tc, TT* __restrict__ T) {
    pdl_enter();
    OTM_FOR_ROWS(row, nf * nf) {
        const int y = row % nf, z = row / nf;
        OTM_FOR_X(x, nf) prolong_node<CT, TT, OUT_AOS>(nf, x, y, z, Tc, T);
    }
}

// k_prolong_add on a node-major coarse level that loads its first node's own
// field value before waiting on the previous kernel (the level's field was
// last written by its pre-smoothing, two or more kernels back; the coarser
// field it adds comes from the previous kernel and is read after the wait).
// The per-node arithmetic is prolong_node's.
template <class CT, class TT>
__global__ void __launch_bounds__(256)
k_prolong_add_pf(int nf, const CT* __restrict__ Tc, TT* __restrict__ T) {
    using C = typename St<TT>::C;
    const int row0 = blockIdx.x * blockDim.y + threadIdx.y, x = threadIdx.x;
    const bool first = row0 < nf * nf && x < nf;
    const int y = row0 % nf, z = row0 / nf;
    const size_t v = (size_t)x + (size_t)nf * (y + (size_t)nf * z);
    C t0[3];
    if (first) ld_f3<TT>(T, v, t0);
    pdl_enter();
    if (first && node_ok(x, y, z, nf, kSiteCoarse)) {
        const int nc = nf / 2;
        int xi[2], yi[2], zi[2];
        C wx[2], wy[2], wz[2];
        int cx, cy, cz;
        if (x & 1) { xi[0] = x >> 1; xi[1] = wrapp(x >> 1, nc); wx[0] = wx[1] = C(0.5); cx = 2; }
        else { xi[0] = xi[1] = x >> 1; wx[0] = C(1); wx[1] = 0; cx = 1; }
        if (y & 1) { yi[0] = y >> 1; yi[1] = wrapp(y >> 1, nc); wy[0] = wy[1] = C(0.5); cy = 2; }
        else { yi[0] = yi[1] = y >> 1; wy[0] = C(1); wy[1] = 0; cy = 1; }
        if (z & 1) { zi[0] = z >> 1; zi[1] = wrapp(z >> 1, nc); wz[0] = wz[1] = C(0.5); cz = 2; }
        else { zi[0] = zi[1] = z >> 1; wz[0] = C(1); wz[1] = 0; cz = 1; }
        C acc[3] = {C(0), C(0), C(0)};
        for (int c = 0; c < cz; ++c)
            for (int b = 0; b < cy; ++b)
                for (int a = 0; a < cx; ++a) {
                    typename St<CT>::C t[3];
                    ld_f3<CT>(Tc, (size_t)xi[a] + (size_t)nc * (yi[b] + (size_t)nc * zi[c]), t);
                    const C w = wz[c] * wy[b] * wx[a];
#pragma unroll
                    for (int i = 0; i < 3; ++i) acc[i] += w * (C)t[i];
                }
        st_f3<TT>(T, v, t0[0] + acc[0], t0[1] + acc[1], t0[2] + acc[2]);
    }
    OTM_FOR_ROWS(row, nf * nf) {
        const int yy = row % nf, zz = row / nf;
        OTM_FOR_X(xx, nf) {
            if (row == row0 && xx == x) continue;
            prolong_node<CT, TT, true>(nf, xx, yy, zz, Tc, T);
        }
    }
}

// x_i += alpha_i p_i (x held as hi + lo when xl is not null: the update is
// added with TwoSum/TwoProduct and renormalised); r_i -= alpha_i q_i;
// reduce r_i.r_i and (flexible) r_i.z_i.
template <class R, class ZT>
__global__ void __launch_bounds__(256)
k_update_xr(size_t N, R* __restrict__ x, R* __restrict__ xl, R* __restrict__ r, const R* __restrict__ p,
            const R* __restrict__ q, const ZT* __restrict__ z, const PcgScalars* __restrict__ ps,
            RedBuf rb, FinResid fin) {
    pdl_enter();
    using C = typename St<R>::C;
    const C a0 = (C)ps->alpha[0], a1 = (C)ps->alpha[1], a2 = (C)ps->alpha[2];
    const bool flex = ps->flexible != 0;
    Acc<C> acc[6];
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
         v += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const C a = i == 0 ? a0 : (i == 1 ? a1 : a2);
            if (a == C(0)) continue;
            const size_t o = (size_t)i * N + v;
            const C pv = p[o];
            if (xl) {
                const C ap = mul_rn(a, pv);
                const C ep = fma(a, pv, -ap);
                C sh, se;
                two_sum((C)x[o], ap, sh, se);
                const C lo = xl[o] + (se + ep);
                const C hi = sh + lo;
                xl[o] = lo - (hi - sh);
                x[o] = hi;
            } else {
                x[o] = x[o] + a * pv;
            }
            const C rn = r[o] - a * q[o];
            r[o] = rn;
            acc[i].add_prod(rn, rn);
            if (flex) acc[3 + i].add_prod(rn, (C)St<ZT>::ld(z, o));
        }
    }
    __shared__ double res[6];
    if (grid_reduce<6>(acc, rb, res)) {
        if (is_thread0()) fin(res);
    }
}

// Vectorised forms of the three streaming PCG kernels: each thread handles
// four consecutive nodes per load case (N a multiple of 4).  Same arithmetic
// per element as the scalar forms.
template <class R, class ZT>
__global__ void __launch_bounds__(256)
k_update_xr4(size_t N, R* __restrict__ x, R* __restrict__ xl, R* __restrict__ r, const R* __restrict__ p,
             const R* __restrict__ q, const ZT* __restrict__ z, const PcgScalars* __restrict__ ps,
             RedBuf rb, FinResid fin) {
    pdl_enter();
    using C = typename St<R>::C;
    const C al[3] = {(C)ps->alpha[0], (C)ps->alpha[1], (C)ps->alpha[2]};
    const bool flex = ps->flexible != 0;
    Acc<C> acc[6];
    const size_t N4 = N / 4;
    for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < N4; j += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const C a = al[i];
            if (a == C(0)) continue;
            const size_t o = (size_t)i * N + 4 * j;
            const Q4<C> pv = ld4(p, o), qv = ld4(q, o);
            Q4<C> rv = ld4(r, o), xv = ld4(x, o);
            if (xl) {
                Q4<C> lv = ld4(xl, o);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const C ap = mul_rn(a, pv.v[t]);
                    const C ep = fma(a, pv.v[t], -ap);
                    C sh, se;
                    two_sum(xv.v[t], ap, sh, se);
                    const C lo = lv.v[t] + (se + ep);
                    const C hi = sh + lo;
                    lv.v[t] = lo - (hi - sh);
                    xv.v[t] = hi;
                }
                st4(xl, o, lv);
            } else {
#pragma unroll
                for (int t = 0; t < 4; ++t) xv.v[t] = xv.v[t] + a * pv.v[t];
            }
            st4(x, o, xv);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                rv.v[t] = rv.v[t] - a * qv.v[t];
                acc[i].add_prod(rv.v[t], rv.v[t]);
            }
            st4(r, o, rv);
            if (flex) {
                const Q4<C> zv = ld4(z, o);
#pragma unroll
                for (int t = 0; t < 4; ++t) acc[3 + i].add_prod(rv.v[t], zv.v[t]);
            }
        }
    }
    __shared__ double res[6];
    if (grid_reduce<6>(acc, rb, res)) {
        if (is_thread0()) fin(res);
    }
}

template <class R, class ZT>
__global__ void __launch_bounds__(256)
k_dot_rz4(size_t N, const R* __restrict__ r, const ZT* __restrict__ z, RedBuf rb, FinBeta fin) {
    pdl_enter();
    using C = typename St<R>::C;
    Acc<C> acc[3];
    const size_t N4 = N / 4;
    for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < N4; j += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const size_t o = (size_t)i * N + 4 * j;
            const Q4<C> rv = ld4(r, o);
            const Q4<C> zv = ld4(z, o);
#pragma unroll
            for (int t = 0; t < 4; ++t) acc[i].add_prod(rv.v[t], zv.v[t]);
        }
    }
    __shared__ double res[3];
    if (grid_reduce<3>(acc, rb, res)) {
        if (is_thread0()) fin(res);
    }
}

template <class R, class ZT>
__global__ void __launch_bounds__(256)
k_update_p4(size_t N, R* __restrict__ p, const ZT* __restrict__ z, const PcgScalars* __restrict__ ps) {
    pdl_enter();
    using C = typename St<R>::C;
    const int first = ps->pfirst;
    const C be[3] = {(C)ps->beta[0], (C)ps->beta[1], (C)ps->beta[2]};
    const int act[3] = {ps->active[0], ps->active[1], ps->active[2]};
    const size_t N4 = N / 4;
    for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < N4; j += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (!act[i]) continue;
            const size_t o = (size_t)i * N + 4 * j;
            const Q4<C> zv = ld4(z, o);
            Q4<C> pv;
            if (first) {
                pv = zv;
            } else {
                pv = ld4(p, o);
#pragma unroll
                for (int t = 0; t < 4; ++t) pv.v[t] = zv.v[t] + be[i] * pv.v[t];
            }
            st4(p, o, pv);
        }
    }
}

// x = hi + lo rounded to the output type (corrector fields for readers).
template <class R, class Y>
__global__ void __launch_bounds__(256)
k_join(size_t count, const R* __restrict__ hi, const R* __restrict__ lo, Y* __restrict__ out) {
    pdl_enter();
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x)
        St<Y>::st(out, i, (typename St<Y>::C)((double)hi[i] + (lo ? (double)lo[i] : 0.0)));
}

// gamma = r . z (three load cases), then beta via the finaliser.
template <class R, class ZT>
__global__ void __launch_bounds__(256)
k_dot_rz(size_t N, const R* __restrict__ r, const ZT* __restrict__ z, RedBuf rb, FinBeta fin) {
    pdl_enter();
    using C = typename St<R>::C;
    Acc<C> acc[3];
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
         v += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const size_t o = (size_t)i * N + v;
            acc[i].add_prod(r[o], (C)St<ZT>::ld(z, o));
        }
    }
    __shared__ double res[3];
    if (grid_reduce<3>(acc, rb, res)) {
        if (is_thread0()) fin(res);
    }
}

// Device-side loop control of the captured PCG: continue while a load case
// is active and the iteration cap is not reached.
static __global__ void k_set_cond(const PcgScalars* __restrict__ ps, cudaGraphConditionalHandle h, int maxit) {
    pdl_enter();
    if (threadIdx.x == 0 && blockIdx.x == 0)
        cudaGraphSetConditional(h, (ps->nactive > 0 && ps->total < maxit) ? 1u : 0u);
}

static __global__ void k_pcg_reset(PcgScalars* ps) {
    pdl_enter();
    if (threadIdx.x == 0 && blockIdx.x == 0) ps->total = 0;
}

// b = a (type conversion), optionally clamped to [0, 1].
template <class X, class Y>
__global__ void __launch_bounds__(256)
k_convert(size_t count, const X* __restrict__ a, Y* __restrict__ b, int clamp01) {
    pdl_enter();
    using C = typename St<Y>::C;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x) {
        C v = (C)St<X>::ld(a, i);
        if (clamp01) v = v < C(0) ? C(0) : (v > C(1) ? C(1) : v);
        St<Y>::st(b, i, v);
    }
}

// p_i = z_i + beta_i p_i.
template <class R, class ZT>
__global__ void __launch_bounds__(256)
k_update_p(size_t N, R* __restrict__ p, const ZT* __restrict__ z, const PcgScalars* __restrict__ ps) {
    pdl_enter();
    using C = typename St<R>::C;
    const int first = ps->pfirst;
    const C b0 = (C)ps->beta[0], b1 = (C)ps->beta[1], b2 = (C)ps->beta[2];
    const int a0 = ps->active[0], a1 = ps->active[1], a2 = ps->active[2];
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
         v += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int act = i == 0 ? a0 : (i == 1 ? a1 : a2);
            if (!act) continue;
            const C b = i == 0 ? b0 : (i == 1 ? b1 : b2);
            const size_t o = (size_t)i * N + v;
            p[o] = first ? (C)St<ZT>::ld(z, o) : (C)St<ZT>::ld(z, o) + b * p[o];
        }
    }
}

}  // namespace otm
