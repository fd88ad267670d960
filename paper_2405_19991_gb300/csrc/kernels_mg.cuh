// Coarse levels of the V-cycle (Alg. 3).
//
// Coarse operators are Galerkin products A_{l+1} = R A_l P with trilinear P
// and R = P^T.  They are built element by element: a fine element e lies in
// the coarse element E at sub-position s in {0,1}^3, and its eight corners
// are interpolated from E's corners by an 8x8 matrix P_s, so
//   K_E^{l+1} = sum_s P_s^T K_{child(E,s)}^l P_s,   K_e^0 = k_e K0,
// which on the first level is sum_s k_{child(E,s)} B_s with constant
// B_s = P_s^T K0 P_s.  Each level's 27-point node stencil (stored as
// A[o][v], o = (dx+1) + 3(dy+1) + 9(dz+1)) gathers the element matrices of
// the eight elements around v.  P_s[j][m] = prod_d phi(s_d + j_d, m_d) with
// phi(t, 0) = {1, 1/2, 0}[t], phi(t, 1) = {0, 1/2, 1}[t].
#pragma once
#include <type_traits>

#include "otm_internal.cuh"
#include "ptx_async.cuh"

namespace otm {

// Element matrices are stored element-major, Kel[E][64] (entry m * 8 + j),
// so one element is 256 contiguous bytes.

// The eight fine conductivities of first-level element (X, Y, Z) (children
// s = sx + 2 sy + 4 sz of the fine grid of side 2 nc).
template <class KT, class C>
__device__ __forceinline__ void child_k(const KT* __restrict__ k, int nc, int X, int Y, int Z, C (&ks)[8]) {
    const int nf = 2 * nc;
#pragma unroll
    for (int s = 0; s < 8; s += 2) {   // children s, s + 1 are x-neighbours (2X even: one aligned pair)
        const int fy = 2 * Y + ((s >> 1) & 1), fz = 2 * Z + (s >> 2);
        const size_t o = (size_t)(2 * X) + (size_t)nf * (fy + (size_t)nf * fz);
        if (std::is_same<KT, float>::value) {
            const float2 w = *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(k) + o);
            ks[s] = (C)w.x;
            ks[s + 1] = (C)w.y;
        } else {
            ks[s] = (C)St<KT>::ld(k, o);
            ks[s + 1] = (C)St<KT>::ld(k, o + 1);
        }
    }
}

// Eight consecutive values of a shared-memory row (16-byte aligned).
template <class C>
__device__ __forceinline__ void lds8(const C* p, C (&r)[8]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) r[j] = p[j];
}
template <>
__device__ __forceinline__ void lds8<float>(const float* p, float (&r)[8]) {
    const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
    r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
    r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
}

// ---- first coarse level: the node stencil straight from the fine
// conductivities.  Entry (m, j) of the element matrix of E is
// sum_s k_{child(E,s)} B_s[m][j] (s in order); the stencil of node v gathers,
// for its corners m = 0..7 in the eight elements around it, entries j = 0..7
// in order -- the operations of an element-matrix pass followed by a gather,
// without storing the first level's element matrices.
// One thread per node and no loop around it: the 512 weights stay in shared
// memory instead of being hoisted into (spilled) registers.
template <class KT, class C, class AT>
__global__ void __launch_bounds__(128)
k_stencil1_from_k(int nc, const KT* __restrict__ k, const C* __restrict__ Bs, AT* __restrict__ A) {
    pdl_enter();
    __shared__ __align__(16) C bs[8 * 64];
    for (int i = threadIdx.x; i < 8 * 64; i += blockDim.x) bs[i] = Bs[i];
    __syncthreads();
    const size_t Nc = (size_t)nc * nc * nc;
    const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= Nc) return;
    const int x = (int)(v % nc), y = (int)((v / nc) % nc), z = (int)(v / ((size_t)nc * nc));
    C acc[27];
#pragma unroll
    for (int o = 0; o < 27; ++o) acc[o] = 0;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int a = m & 1, b = (m >> 1) & 1, c = m >> 2;
        C ks[8];
        child_k<KT, C>(k, nc, wrapd(x, -a, nc), wrapd(y, -b, nc), wrapd(z, -c, nc), ks);
        C e[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) e[j] = 0;
#pragma unroll
        for (int s = 0; s < 8; ++s) {   // e[j] = sum_s ks[s] B_s[m][j], s in order
            C w[8];
            lds8<C>(bs + s * 64 + m * 8, w);
#pragma unroll
            for (int j = 0; j < 8; ++j) e[j] += ks[s] * w[j];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int dx = (j & 1) - a, dy = ((j >> 1) & 1) - b, dz = (j >> 2) - c;
            acc[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)] += e[j];
        }
    }
    st_arow<AT, C>(A, v, acc);
}

// ---- deeper levels: K_E = sum_s P_s^T K_child P_s, one warp per coarse
// element.  P_s factors into 1-D interpolations along x, y, z (P_s[j][m] =
// prod_d phi(s_d + j_d, m_d)), so both products are three 1-D passes: along
// index bit d with child position s_d, the entry with bit value b becomes
// own + partner / 2 when b == s_d and own / 2 otherwise (partner: the entry
// with bit d flipped).  Lane l holds entries (r, c) = (l / 8, l % 8) and
// (l / 8 + 4, l % 8): column passes exchange with lanes l ^ 1, l ^ 2, l ^ 4,
// row passes with l ^ 8, l ^ 16 and between the lane's two entries.
// FROM_K: the children are first-level elements, their matrices
// sum_s' k B_s' formed on the fly from the fine conductivities k (Kf unused).
template <class C>
__device__ __forceinline__ C interp_pass(C own, C partner, bool up) {
    return up ? own + C(0.5) * partner : C(0.5) * own;
}
template <class C, bool FROM_K, class KT>
__global__ void __launch_bounds__(256)
k_elem_coarsen(int nc, const C* __restrict__ Kf, const KT* __restrict__ k, const C* __restrict__ Bs,
               C* __restrict__ Kc) {
    pdl_enter();
    __shared__ C bs[FROM_K ? 8 * 64 : 1];
    if (FROM_K) {
        for (int i = threadIdx.x; i < 8 * 64; i += blockDim.x) bs[i] = Bs[i];
        __syncthreads();
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int nf = 2 * nc;
    const size_t Nc = (size_t)nc * nc * nc;
    const int cb = lane & 7, rb = lane >> 3;   // column bits; row bits 0, 1 (row bit 2: which entry)
    for (size_t E = (size_t)blockIdx.x * nwarps + warp; E < Nc; E += (size_t)gridDim.x * nwarps) {
        const int X = (int)(E % nc), Y = (int)((E / nc) % nc), Z = (int)(E / ((size_t)nc * nc));
        C out0 = 0, out1 = 0;
#pragma unroll 1
        for (int s = 0; s < 8; ++s) {
            const int fx = 2 * X + (s & 1), fy = 2 * Y + ((s >> 1) & 1), fz = 2 * Z + (s >> 2);
            C v0, v1;   // entries (rb, cb) and (rb + 4, cb) of the child's matrix
            if (FROM_K) {
                C ks[8];
                child_k<KT, C>(k, nf, fx, fy, fz, ks);
                v0 = 0;
                v1 = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    v0 += ks[q] * bs[q * 64 + lane];
                    v1 += ks[q] * bs[q * 64 + 32 + lane];
                }
            } else {
                const size_t e = (size_t)fx + (size_t)nf * (fy + (size_t)nf * fz);
                v0 = Kf[e * 64 + lane];
                v1 = Kf[e * 64 + 32 + lane];
            }
            // K P_s: passes over the column bits
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const bool up = ((cb >> d) & 1) == ((s >> d) & 1);
                const C p0 = __shfl_xor_sync(0xffffffffu, v0, 1 << d);
                const C p1 = __shfl_xor_sync(0xffffffffu, v1, 1 << d);
                v0 = interp_pass(v0, p0, up);
                v1 = interp_pass(v1, p1, up);
            }
            // P_s^T (K P_s): passes over the row bits
#pragma unroll
            for (int d = 0; d < 2; ++d) {
                const bool up = ((rb >> d) & 1) == ((s >> d) & 1);
                const C p0 = __shfl_xor_sync(0xffffffffu, v0, 8 << d);
                const C p1 = __shfl_xor_sync(0xffffffffu, v1, 8 << d);
                v0 = interp_pass(v0, p0, up);
                v1 = interp_pass(v1, p1, up);
            }
            {
                const int sz = (s >> 2) & 1;
                const C a0 = interp_pass(v0, v1, sz == 0), a1 = interp_pass(v1, v0, sz == 1);
                v0 = a0;
                v1 = a1;
            }
            out0 += v0;
            out1 += v1;
        }
        Kc[E * 64 + lane] = out0;
        Kc[E * 64 + 32 + lane] = out1;
    }
}

// ---- node stencils from element matrices ----
template <class C, class AT>
__global__ void __launch_bounds__(128)
k_stencil_from_elem(int n, const C* __restrict__ Kel, AT* __restrict__ A) {
    pdl_enter();
    OTM_FOR_ROWS(row_, n * n) {
    const int y = row_ % n, z = row_ / n;
    OTM_FOR_X(x, n) {
        const size_t v = (size_t)row_ * n + x;
        C acc[27];
#pragma unroll
        for (int o = 0; o < 27; ++o) acc[o] = 0;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int a = m & 1, b = (m >> 1) & 1, c = m >> 2;
            const size_t E = (size_t)wrapd(x, -a, n) + (size_t)n * (wrapd(y, -b, n) + (size_t)n * wrapd(z, -c, n));
            const C* row = Kel + E * 64 + m * 8;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int dx = (j & 1) - a, dy = ((j >> 1) & 1) - b, dz = (j >> 2) - c;
                acc[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)] += row[j];
            }
        }
        st_arow<AT, C>(A, v, acc);
    }
    }
}

// Node stencil of the finest operator itself (used when the hierarchy has a
// single level and the fine grid is solved directly).
template <class KT, class C, class AT>
__global__ void __launch_bounds__(128)
k_stencil_from_k(int n, const KT* __restrict__ k, AT* __restrict__ A) {
    pdl_enter();
    OTM_FOR_ROWS(row_, n * n) {
    const int y = row_ % n, z = row_ / n;
    OTM_FOR_X(x, n) {
        const size_t v = (size_t)row_ * n + x;
        C acc[27];
#pragma unroll
        for (int o = 0; o < 27; ++o) acc[o] = 0;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int a = m & 1, b = (m >> 1) & 1, c = m >> 2;
            const size_t E = (size_t)wrapd(x, -a, n) + (size_t)n * (wrapd(y, -b, n) + (size_t)n * wrapd(z, -c, n));
            const C ke = St<KT>::ld(k, E);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int pc = __popc(j ^ m);
                const C k0 = pc == 0 ? C(1.0 / 3.0) : (pc == 1 ? C(0) : C(-1.0 / 12.0));
                const int dx = (j & 1) - a, dy = ((j >> 1) & 1) - b, dz = (j >> 2) - c;
                acc[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)] += ke * k0;
            }
        }
        st_arow<AT, C>(A, v, acc);
    }
    }
}

// ---- Chebyshev polynomial smoother on a 27-point stencil level ----
// A degree-kChebDeg Chebyshev iteration for D^-1 A on [lmax / kChebRatio,
// lmax], with lmax the level's Gershgorin bound max_v sum_o |A_o(v)| / A_0(v)
// (an upper bound of the spectrum of D^-1 A, so the polynomial never
// amplifies).  Step k: r = f - A T; d = c_d d + c_r D^-1 r; T += d, with
// theta = (lmax + lmin) / 2, delta = (lmax - lmin) / 2, sigma = theta / delta,
// rho_0 = 1 / sigma, rho_k = 1 / (2 sigma - rho_{k-1}); c_d = rho_k rho_{k-1}
// and c_r = 2 rho_k / delta for k > 0, c_d = 0 and c_r = 1 / theta for k = 0.
// The same polynomial before and after the coarse correction keeps the
// V-cycle symmetric, as plain PCG needs.  Each step reads T from one buffer
// and writes the other (Jacobi-type), so a step is one pass over all nodes.
constexpr int kChebDeg = 3;
constexpr float kChebRatio = 30.0f;

__host__ __device__ inline void cheb_coef(float lmax, int k, float& c_d, float& c_r) {
    const float lmin = lmax / kChebRatio;
    const float theta = 0.5f * (lmax + lmin), delta = 0.5f * (lmax - lmin);
    const float sigma = theta / delta;
    if (k == 0) {
        c_d = 0.0f;
        c_r = 1.0f / theta;
        return;
    }
    float rho = 1.0f / sigma, rho_new = rho;
    for (int i = 1; i <= k; ++i) {
        rho_new = 1.0f / (2.0f * sigma - rho);
        if (i < k) rho = rho_new;
    }
    c_d = rho_new * rho;
    c_r = 2.0f * rho_new / delta;
}

// One Chebyshev step at node (x, y, z).  ZERO: T starts at zero (not read).
template <bool ZERO, class AT, class FT, class TT>
__device__ __forceinline__ void cheb_node(int n, size_t N, int x, int y, int z, const AT* __restrict__ A,
                                          const FT* __restrict__ f, const TT* __restrict__ Tin,
                                          TT* __restrict__ Tout, TT* __restrict__ D, float c_d, float c_r) {
    using C = typename St<TT>::C;
    const size_t v = (size_t)x + (size_t)n * (y + (size_t)n * z);
    if (!node_ok(x, y, z, n, kSiteCoarse) || !OTM_BOUND(v, N, kSiteCoarse)) return;
    int xs[3], ys[3], zs[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        xs[d] = wrapd(x, d - 1, n);
        ys[d] = wrapd(y, d - 1, n) * n;
        zs[d] = wrapd(z, d - 1, n) * n * n;
    }
    C a[27];
    ld_arow<AT>(A, v, a);
    const C inv = C(1) / a[13];
    C r[3];
    ld_f3<FT>(f, v, r);
    C t0[3] = {C(0), C(0), C(0)}, dv[3];
    if (!ZERO) {
#pragma unroll
        for (int o = 0; o < 27; ++o) {
            C t[3];
            ld_f3<TT>(Tin, (size_t)(xs[o % 3] + ys[(o / 3) % 3] + zs[o / 9]), t);
#pragma unroll
            for (int i = 0; i < 3; ++i) r[i] -= a[o] * t[i];
        }
        ld_f3<TT>(Tin, v, t0);
        C d0[3];
        ld_f3<TT>(D, v, d0);
#pragma unroll
        for (int i = 0; i < 3; ++i) dv[i] = C(c_d) * d0[i] + C(c_r) * r[i] * inv;
    } else {
#pragma unroll
        for (int i = 0; i < 3; ++i) dv[i] = C(c_r) * r[i] * inv;
    }
    st_f3<TT>(D, v, dv[0], dv[1], dv[2]);
    st_f3<TT>(Tout, v, t0[0] + dv[0], t0[1] + dv[1], t0[2] + dv[2]);
}

template <bool ZERO, class AT, class FT, class TT>
__global__ void __launch_bounds__(256)
k_cheb_stencil(int n, int k, const float* __restrict__ lam, const AT* __restrict__ A, const FT* __restrict__ f,
               const TT* __restrict__ Tin, TT* __restrict__ Tout, TT* __restrict__ D) {
    pdl_enter();
    const size_t N = (size_t)n * n * n;
    float c_d, c_r;
    cheb_coef(*lam, k, c_d, c_r);
    OTM_FOR_ROWS(row_, n * n) {
        const int y = row_ % n, z = row_ / n;
        OTM_FOR_X(x, n) cheb_node<ZERO, AT, FT, TT>(n, N, x, y, z, A, f, Tin, Tout, D, c_d, c_r);
    }
}

// Gershgorin bound of D^-1 A: *lam = max(*lam, max_v sum_o |A_o(v)| / A_0(v))
// (*lam starts at zero; positive floats order like their bit patterns).
template <class AT>
__global__ void __launch_bounds__(256)
k_gershgorin(int n, const AT* __restrict__ A, float* __restrict__ lam) {
    pdl_enter();
    using C = typename St<AT>::C;
    const size_t N = (size_t)n * n * n;
    float g = 0.0f;
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
        C s = 0;
        C a[27];
        ld_arow<AT>(A, v, a);
#pragma unroll
        for (int o = 0; o < 27; ++o) s += a[o] < C(0) ? -a[o] : a[o];
        g = fmaxf(g, (float)(s / a[13]));
    }
    for (int o = 16; o > 0; o >>= 1) g = fmaxf(g, __shfl_xor_sync(0xffffffffu, g, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(lam), __float_as_int(g));
}

// ---- Gauss-Seidel colour pass on a 27-point stencil level ----
// colour = (x%2) + 2(y%2) + 4(z%2); n even.  ZERO (colour 0 only): the field
// starts at zero and the pass zeroes the other seven nodes of each 2x2x2 cell.
// gs_stencil_node relaxes node (x, y, z): T_v = (f_v - sum_{o != 0} A_o T_{v+o}) / A_0.
template <bool ZERO, class AT, class FT, class TT>
__device__ __forceinline__ void gs_stencil_node(int n, size_t N, int x, int y, int z, const AT* __restrict__ A,
                                                const FT* __restrict__ f, TT* __restrict__ T) {
    using C = typename St<TT>::C;
    const size_t v = (size_t)x + (size_t)n * (y + (size_t)n * z);
    if (!node_ok(x, y, z, n, kSiteCoarse) || !OTM_BOUND(v, N, kSiteCoarse)) return;
    int xs[3], ys[3], zs[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        xs[d] = wrapd(x, d - 1, n);
        ys[d] = wrapd(y, d - 1, n) * n;
        zs[d] = wrapd(z, d - 1, n) * n * n;
    }
    C a[27];
    ld_arow<AT>(A, v, a);
    const C inv = C(1) / a[13];
    C s[3];
    ld_f3<FT>(f, v, s);
    if (!ZERO) {
        // per load case the same accumulation order as a scalar sweep over o
#pragma unroll
        for (int o = 0; o < 27; ++o) {
            if (o == 13) continue;
            C t[3];
            ld_f3<TT>(T, (size_t)(xs[o % 3] + ys[(o / 3) % 3] + zs[o / 9]), t);
#pragma unroll
            for (int i = 0; i < 3; ++i) s[i] -= a[o] * t[i];
        }
    }
    st_f3<TT>(T, v, s[0] * inv, s[1] * inv, s[2] * inv);
    if (ZERO) {
#pragma unroll
        for (int q = 1; q < 8; ++q) {
            const size_t w = (size_t)(x + (q & 1)) + (size_t)n * ((y + ((q >> 1) & 1)) + (size_t)n * (z + (q >> 2)));
            st_f3<TT>(T, w, C(0), C(0), C(0));
        }
    }
}

// A colour pass that loads its first node's stencil row -- and, with
// early_f, its right-hand side, and the neighbours that tmask marks (bit o
// for coupling o) -- before waiting on the previous kernel.  The V-cycle
// writes the stencils at setup and f with the restriction before the
// level's first pass (the one launch that passes early_f = 0); a neighbour
// may be read early unless the previous kernel wrote it: the previous colour
// pass writes only its own colour, the zero-start pass and the prolongation
// write every node (tmask = 0).  The L2 round trips of those loads then
// overlap the previous kernel's tail.  The per-node arithmetic is
// gs_stencil_node's (the same bits); nodes past a thread's first, which the
// solver's launch shapes do not produce, take gs_stencil_node itself.
template <bool ZERO, class AT, class FT, class TT>
__global__ void __launch_bounds__(256)
k_gs_stencil_pf(int n, int colour, const AT* __restrict__ A, const FT* __restrict__ f, TT* __restrict__ T, int early_f,
                unsigned tmask) {
    using C = typename St<TT>::C;
    const size_t N = (size_t)n * n * n;
    const int h = n >> 1;
    const int xo = colour & 1, yo = (colour >> 1) & 1, zo = colour >> 2;
    const int row0 = blockIdx.x * blockDim.y + threadIdx.y, xi0 = threadIdx.x;
    const bool first = row0 < h * h && xi0 < h;
    const int x = 2 * xi0 + xo, y = 2 * (row0 % h) + yo, z = 2 * (row0 / h) + zo;
    const size_t v = (size_t)x + (size_t)n * (y + (size_t)n * z);
    int xs[3], ys[3], zs[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        xs[d] = wrapd(x, d - 1, n);
        ys[d] = wrapd(y, d - 1, n) * n;
        zs[d] = wrapd(z, d - 1, n) * n * n;
    }
    C a[27], s[3], t[27][3];
    if (first) {
        ld_arow<AT>(A, v, a);
        if (early_f) ld_f3<FT>(f, v, s);
        if (!ZERO) {
#pragma unroll
            for (int o = 0; o < 27; ++o)
                if (o != 13 && ((tmask >> o) & 1u)) ld_f3<TT>(T, (size_t)(xs[o % 3] + ys[(o / 3) % 3] + zs[o / 9]), t[o]);
        }
    }
    pdl_enter();
    if (first && node_ok(x, y, z, n, kSiteCoarse) && OTM_BOUND(v, N, kSiteCoarse)) {
        if (!early_f) ld_f3<FT>(f, v, s);
        const C inv = C(1) / a[13];
        if (!ZERO) {
#pragma unroll
            for (int o = 0; o < 27; ++o)
                if (o != 13 && !((tmask >> o) & 1u)) ld_f3<TT>(T, (size_t)(xs[o % 3] + ys[(o / 3) % 3] + zs[o / 9]), t[o]);
            // per load case the same accumulation order as a scalar sweep over o
#pragma unroll
            for (int o = 0; o < 27; ++o) {
                if (o == 13) continue;
#pragma unroll
                for (int i = 0; i < 3; ++i) s[i] -= a[o] * t[o][i];
            }
        }
        st_f3<TT>(T, v, s[0] * inv, s[1] * inv, s[2] * inv);
        if (ZERO) {
#pragma unroll
            for (int q = 1; q < 8; ++q) {
                const size_t w = (size_t)(x + (q & 1)) + (size_t)n * ((y + ((q >> 1) & 1)) + (size_t)n * (z + (q >> 2)));
                st_f3<TT>(T, w, C(0), C(0), C(0));
            }
        }
    }
    OTM_FOR_ROWS(row_, h * h) {
        const int yy = 2 * (row_ % h) + yo, zz = 2 * (row_ / h) + zo;
        OTM_FOR_X(xi, h) {
            if (row_ == row0 && xi == xi0) continue;
            gs_stencil_node<ZERO, AT, FT, TT>(n, N, 2 * xi + xo, yy, zz, A, f, T);
        }
    }
}

// Couplings o of a colour-c node whose neighbour the pass of colour prev
// writes (odd offsets flip a coordinate's parity); the complement may be read
// before the wait on that pass.  prev < 0: the previous kernel wrote every
// node.
inline unsigned gs_early_mask(int c, int prev) {
    if (prev < 0) return 0u;
    unsigned m = 0u;
    for (int o = 0; o < 27; ++o) {
        const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
        const int nc = c ^ ((dx & 1) | ((dy & 1) << 1) | ((dz & 1) << 2));
        if (o != 13 && nc != prev) m |= 1u << o;
    }
    return m;
}

template <bool ZERO, class AT, class FT, class TT>
__global__ void __launch_bounds__(256)
k_gs_stencil(int n, int colour, const AT* __restrict__ A, const FT* __restrict__ f, TT* __restrict__ T) {
    pdl_enter();
    const size_t N = (size_t)n * n * n;
    const int h = n >> 1;
    const int xo = colour & 1, yo = (colour >> 1) & 1, zo = colour >> 2;
    OTM_FOR_ROWS(row_, h * h) {
        const int y = 2 * (row_ % h) + yo, z = 2 * (row_ / h) + zo;
        OTM_FOR_X(xi, h) gs_stencil_node<ZERO, AT, FT, TT>(n, N, 2 * xi + xo, y, z, A, f, T);
    }
}

// res = f - A T on a stencil level.
template <class AT, class FT, class TT, class OT>
__device__ __forceinline__ void residual_stencil_node(int n, size_t N, int x, int y, int z, const AT* __restrict__ A,
                                                      const FT* __restrict__ f, const TT* __restrict__ T,
                                                      OT* __restrict__ res) {
    using C = typename St<OT>::C;
    const size_t v = (size_t)x + (size_t)n * (y + (size_t)n * z);
    if (!node_ok(x, y, z, n, kSiteCoarse) || !OTM_BOUND(v, N, kSiteCoarse)) return;
    int xs[3], ys[3], zs[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        xs[d] = wrapd(x, d - 1, n);
        ys[d] = wrapd(y, d - 1, n) * n;
        zs[d] = wrapd(z, d - 1, n) * n * n;
    }
    C a[27];
    ld_arow<AT>(A, v, a);
    C s[3];
    ld_f3<FT>(f, v, s);
#pragma unroll
    for (int o = 0; o < 27; ++o) {
        C t[3];
        ld_f3<TT>(T, (size_t)(xs[o % 3] + ys[(o / 3) % 3] + zs[o / 9]), t);
#pragma unroll
        for (int i = 0; i < 3; ++i) s[i] -= a[o] * t[i];
    }
    st_f3<OT>(res, v, s[0], s[1], s[2]);
}
template <class AT, class FT, class TT, class OT>
__global__ void __launch_bounds__(256)
k_residual_stencil(int n, const AT* __restrict__ A, const FT* __restrict__ f, const TT* __restrict__ T,
                   OT* __restrict__ res) {
    pdl_enter();
    const size_t N = (size_t)n * n * n;
    OTM_FOR_ROWS(row_, n * n) {
        const int y = row_ % n, z = row_ / n;
        OTM_FOR_X(x, n) residual_stencil_node<AT, FT, TT, OT>(n, N, x, y, z, A, f, T, res);
    }
}

// k_residual_stencil that loads its first node's stencil row and right-hand
// side before waiting on the previous kernel (both written two or more
// kernels back in the V-cycle: the stencils at setup, f by the restriction
// before the level's pre-smoothing); the field follows the wait.  The
// per-node arithmetic is residual_stencil_node's.
template <class AT, class FT, class TT, class OT>
__global__ void __launch_bounds__(256)
k_residual_stencil_pf(int n, const AT* __restrict__ A, const FT* __restrict__ f, const TT* __restrict__ T,
                      OT* __restrict__ res) {
    using C = typename St<OT>::C;
    const size_t N = (size_t)n * n * n;
    const int row0 = blockIdx.x * blockDim.y + threadIdx.y, x = threadIdx.x;
    const bool first = row0 < n * n && x < n;
    const int y = row0 % n, z = row0 / n;
    const size_t v = (size_t)x + (size_t)n * (y + (size_t)n * z);
    C a[27], s[3];
    if (first) {
        ld_arow<AT>(A, v, a);
        ld_f3<FT>(f, v, s);
    }
    pdl_enter();
    if (first && node_ok(x, y, z, n, kSiteCoarse) && OTM_BOUND(v, N, kSiteCoarse)) {
        int xs[3], ys[3], zs[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            xs[d] = wrapd(x, d - 1, n);
            ys[d] = wrapd(y, d - 1, n) * n;
            zs[d] = wrapd(z, d - 1, n) * n * n;
        }
#pragma unroll
        for (int o = 0; o < 27; ++o) {
            C t[3];
            ld_f3<TT>(T, (size_t)(xs[o % 3] + ys[(o / 3) % 3] + zs[o / 9]), t);
#pragma unroll
            for (int i = 0; i < 3; ++i) s[i] -= a[o] * t[i];
        }
        st_f3<OT>(res, v, s[0], s[1], s[2]);
    }
    OTM_FOR_ROWS(row_, n * n) {
        const int yy = row_ % n, zz = row_ / n;
        OTM_FOR_X(xx, n) {
            if (row_ == row0 && xx == x) continue;
            residual_stencil_node<AT, FT, TT, OT>(n, N, xx, yy, zz, A, f, T, res);
        }
    }
}

// ---- coarsest level: dense inverse of the node-0-pinned operator ----
// One CTA.  The dense matrix of the stencil without node 0's row and column
// is inverted in place by Gauss-Jordan elimination without pivoting (the
// pinned matrix is SPD, so every pivot -- a Schur-complement diagonal -- is
// positive), in the compute type C, and the result is symmetrised
// ((M + M^T) / 2) so the coarse correction, and with it the V-cycle, stays a
// symmetric operator.  The pivots are taken kInvB at a time: sweeping the
// pivot block K of the current matrix W (D = W[K][K]) is
//   W[K][K] <- D^-1,            W[K][j] <- D^-1 W[K][j],
//   W[i][K] <- -W[i][K] D^-1,   W[i][j] <- W[i][j] - W[i][K] D^-1 W[K][j]
// for i, j outside K -- the same as kInvB single-pivot steps.  D^-1 comes
// from single-pivot steps by one warp; the two panel products run as
// (4 columns or rows) x (4 panel rows or columns) units, one per thread;
// the rank-kInvB update of the rows outside K runs as 4 x 4 register tiles
// (the old panel column and R = D^-1 W[K][j] read as 4-wide vectors).  W has
// a row stride of q rounded up to a multiple of 4 (zero padding), so rows
// are 16-byte aligned and tiles cover it; it lives in shared memory when it
// fits the opt-in limit, else in Wg.  No index needs an integer division
// except the tile number of the update.
constexpr int kInvB = 16;
constexpr int kInvThreads = 512;
// 1 / x correctly rounded (the same value as the division 1 / x)
__device__ __forceinline__ float inv_rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double inv_rcp(double x) { return __drcp_rn(x); }
__host__ __device__ inline int inv_ld(int q) { return (q + 3) & ~3; }
inline size_t invert_smem_bytes(int q, int elem, bool with_w) {
    const size_t ld = (size_t)inv_ld(q);
    return (size_t)elem * ((size_t)kInvB * kInvB + 2 * (size_t)kInvB * ld + (with_w ? ld * ld : 0));
}
template <class AT, class C>
__global__ void __launch_bounds__(kInvThreads)
k_coarse_invert(int n, const AT* __restrict__ A, C* __restrict__ Wg, C* __restrict__ Minv, int use_smem) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char inv_sm[];
    constexpr int B = kInvB;
    const int m = n * n * n;
    const int q = m - 1;
    const int ld = inv_ld(q);
    const int nq = ld >> 2;                    // 4-wide groups of columns (and of rows)
    C* Dp = reinterpret_cast<C*>(inv_sm);      // [B][B]: D, then D^-1 (zero past the panel)
    C* Prow = Dp + B * B;                      // [B][ld]: panel rows W[K][j], then R = D^-1 W[K][j]
    C* PcT = Prow + (size_t)B * ld;            // [B][ld]: panel columns, transposed: PcT[c][i] = W[i][k0 + c]
    C* W = use_smem ? PcT + (size_t)B * ld : Wg;
    const int nthr = blockDim.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
    const Q4<C> zero4 = {{C(0), C(0), C(0), C(0)}};
    for (int i = tid; i < ld * ld; i += nthr) W[i] = C(0);
    __syncthreads();
    for (int v = 1 + tid; v < m; v += nthr) {
        const int x = v % n, y = (v / n) % n, z = v / (n * n);
        for (int o = 0; o < 27; ++o) {
            const int c = wrapd(x, o % 3 - 1, n) + n * (wrapd(y, (o / 3) % 3 - 1, n) + n * wrapd(z, o / 9 - 1, n));
            if (c == 0) continue;
            W[(size_t)(v - 1) * ld + (c - 1)] += (C)St<AT>::ld(A, (size_t)v * cl_aw<AT>() + o);
        }
    }
    __syncthreads();
    const int nu = 4 * nq;   // panel-product units of each kind
    for (int k0 = 0; k0 < q; k0 += B) {
        const int b = min(B, q - k0);
        auto inK = [&](int i) { return (unsigned)(i - k0) < (unsigned)b; };
        // 1. panel rows (zero past b) and panel columns, transposed (zero past b)
        for (int c = warp; c < B; c += nw)
            for (int jq = lane; jq < nq; jq += 32)
                st4(Prow, (size_t)c * ld + 4 * jq, c < b ? ld4(W, (size_t)(k0 + c) * ld + 4 * jq) : zero4);
        for (int t = tid; t < 4 * ld; t += nthr) {
            const int i = t >> 2, cq = t & 3;
            const Q4<C> w = 4 * cq < b ? ld4(W, (size_t)i * ld + k0 + 4 * cq) : zero4;
#pragma unroll
            for (int e = 0; e < 4; ++e) PcT[(size_t)(4 * cq + e) * ld + i] = 4 * cq + e < b ? w.v[e] : C(0);
        }
        __syncthreads();
        // 2. D^-1 by single-pivot steps in one warp's registers: lane l holds
        //    row l / 2, columns 8 (l % 2) .. 8 (l % 2) + 7; the pivot, the
        //    pivot row and the pivot column come by shuffles, read before any
        //    lane updates its entries (the q pivots of the inverse form its
        //    serial chain, so no step goes through shared memory)
        if (warp == 0) {
            const int r = lane >> 1, c0 = 8 * (lane & 1);
            C d[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) d[k] = (r < b && c0 + k < b) ? PcT[(size_t)(c0 + k) * ld + k0 + r] : C(0);
#pragma unroll
            for (int p = 0; p < B; ++p) {
                if (p >= b) break;
                const C ip = inv_rcp(__shfl_sync(0xffffffffu, d[p & 7], 2 * p + (p >> 3)));
                const C colp = __shfl_sync(0xffffffffu, d[p & 7], 2 * r + (p >> 3));
                C rowp[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) rowp[k] = __shfl_sync(0xffffffffu, d[k], 2 * p + (lane & 1));
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int c = c0 + k;
                    if (r < b && c < b) {
                        if (r == p) {
                            d[k] = (c == p ? C(1) : d[k]) * ip;
                        } else {
                            const C wk = (c == p ? C(1) : rowp[k]) * ip;
                            d[k] = (c == p ? C(0) : d[k]) - colp * wk;
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) Dp[r * B + c0 + k] = d[k];
        }
        __syncthreads();
        // 3. R = D^-1 W[K][j] into Prow (zero in the columns of K) and
        //    Cn = -W[i][K] D^-1 into W[i][K] for the rows outside K.  A unit
        //    of R reads all of its four columns of Prow before any unit of
        //    the round writes them; the units of one column group share a
        //    round (nthr is a multiple of 4).
        for (int base = 0; base < 2 * nu; base += nthr) {
            const int u = base + tid;
            const bool isR = u < nu, isC = !isR && u < 2 * nu;
            const int g = isR ? u >> 2 : (u - nu) >> 2, cg = u & 3;
            Q4<C> xs[B];
            if (isR) {
#pragma unroll
                for (int d = 0; d < B; ++d) xs[d] = ld4(Prow, (size_t)d * ld + 4 * g);
            } else if (isC) {
#pragma unroll
                for (int d = 0; d < B; ++d) xs[d] = ld4(PcT, (size_t)d * ld + 4 * g);
            }
            __syncthreads();
            if (isR && 4 * cg < b) {
                // R[c][4g + f] = sum_d D^-1[c][d] Prow[d][4g + f], c = 4cg .. 4cg + 3
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    const int c = 4 * cg + cc;
                    if (c >= b) break;
                    Q4<C> r = zero4;
#pragma unroll
                    for (int d = 0; d < B; ++d) {
                        const C dv = Dp[c * B + d];
#pragma unroll
                        for (int f = 0; f < 4; ++f) r.v[f] += dv * xs[d].v[f];
                    }
#pragma unroll
                    for (int f = 0; f < 4; ++f)
                        if (inK(4 * g + f)) r.v[f] = C(0);
                    st4(Prow, (size_t)c * ld + 4 * g, r);
                }
            } else if (isC && 4 * cg < b && 4 * g < q && !inK(4 * g)) {
                // Cn[4g + e][c] = -sum_d PcT[d][4g + e] D^-1[d][c], c = 4cg .. 4cg + 3
                Q4<C> cn[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) cn[e] = zero4;
#pragma unroll
                for (int d = 0; d < B; ++d) {
                    const Q4<C> dr = ld4(Dp, (size_t)d * B + 4 * cg);
#pragma unroll
                    for (int e = 0; e < 4; ++e)
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) cn[e].v[cc] += xs[d].v[e] * dr.v[cc];
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int i = 4 * g + e;
                    if (i >= q) break;
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc)
                        if (4 * cg + cc < b) W[(size_t)i * ld + k0 + 4 * cg + cc] = -cn[e].v[cc];
                }
            }
        }
        __syncthreads();
        // 4. rank-b update of the rows outside K in 4 x 4 tiles (the columns
        //    of K see R = 0 and keep Cn), and 5. the panel rows: W[K][j] = R
        //    outside K, D^-1 inside (rows disjoint from the tiles')
        for (int t = tid; t < nq * nq; t += nthr) {
            const int iq = t / nq, jq = t - iq * nq;
            if (4 * iq >= q || inK(4 * iq)) continue;
            Q4<C> acc[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[e] = ld4(W, (size_t)(4 * iq + e) * ld + 4 * jq);
            // all B panel columns: those past b are zero in PcT and Prow, so
            // the loop needs no bound and its loads can be issued early
#pragma unroll
            for (int c = 0; c < B; ++c) {
                const Q4<C> a = ld4(PcT, (size_t)c * ld + 4 * iq);
                const Q4<C> r = ld4(Prow, (size_t)c * ld + 4 * jq);
#pragma unroll
                for (int e = 0; e < 4; ++e)
#pragma unroll
                    for (int f = 0; f < 4; ++f) acc[e].v[f] -= a.v[e] * r.v[f];
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) st4(W, (size_t)(4 * iq + e) * ld + 4 * jq, acc[e]);
        }
        for (int c = warp; c < b; c += nw)
            for (int jq = lane; jq < nq; jq += 32) {
                Q4<C> w = ld4(Prow, (size_t)c * ld + 4 * jq);
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    const int j = 4 * jq + f;
                    if (inK(j)) w.v[f] = Dp[c * B + (j - k0)];
                }
                st4(W, (size_t)(k0 + c) * ld + 4 * jq, w);
            }
        __syncthreads();
    }
    for (int i = warp; i < q; i += nw)
        for (int j = lane; j < q; j += 32) Minv[(size_t)i * q + j] = C(0.5) * (W[(size_t)i * ld + j] + W[(size_t)j * ld + i]);
}

// T = Minv f with T_0 = 0, then shifted to zero mean.  Executed by every
// thread of one CTA (block-level synchronisation only).
// AOS: f and T node-major [m][4] (a coarse level); else load-case-major [3][m]
// (the fine grid of a single-level hierarchy).
template <class C, class FT, class TT, bool AOS = true>
__device__ void coarse_solve_block(int n, const C* __restrict__ Minv, const FT* __restrict__ f, TT* __restrict__ T) {
    const int m = n * n * n;
    const int q = m - 1;
    __shared__ C fs[3][343];
    __shared__ C ts[3][343];
    __shared__ Acc<C> red[3][32];
    __shared__ C mean[3];
    for (int i = threadIdx.x; i < 3 * m; i += blockDim.x)
        fs[i / m][i % m] = St<FT>::ld(f, AOS ? (size_t)(i % m) * 4 + i / m : (size_t)i);
    __syncthreads();
    // Minv is symmetric, so row v-1 is read as column v-1: consecutive
    // threads read consecutive words.
    for (int t = threadIdx.x; t < 3 * m; t += blockDim.x) {
        const int r = t / m, v = t % m;
        C a = 0;
        if (v > 0) {
            for (int j = 0; j < q; ++j) a += Minv[(size_t)j * q + (v - 1)] * fs[r][j + 1];
        }
        ts[r][v] = a;
    }
    __syncthreads();
    // load-case means, summed compensated in the compute type
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = 0; r < 3; ++r) {
        Acc<C> a;
        for (int v = threadIdx.x; v < m; v += blockDim.x) a.add(ts[r][v]);
        acc_warp_sum(a);
        if (lane == 0) red[r][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        Acc<C> a = red[threadIdx.x][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) acc_merge(a, red[threadIdx.x][w]);
        mean[threadIdx.x] = (C)(a.value() / m);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * m; t += blockDim.x) {
        const int r = t / m, v = t % m;
        St<TT>::st(T, AOS ? (size_t)v * 4 + r : (size_t)t, ts[r][v] - mean[r]);
    }
}

// Block-wide copy of `bytes` from global to shared memory: every thread
// issues its share of 16-byte asynchronous copies, all in flight at once
// (an element loop would wait one L2 round trip per element: the compiler
// cannot move a global load past a shared store through generic pointers),
// and a ragged tail is copied byte by byte.  Both addresses 16-byte
// aligned.  The caller waits (cp_async_wait_all) and then synchronises the
// block.
__device__ __forceinline__ void block_copy_async(void* dst, const void* src, size_t bytes) {
    unsigned char* d = static_cast<unsigned char*>(dst);
    const unsigned char* s = static_cast<const unsigned char*>(src);
    const size_t n16 = bytes / 16;
    for (size_t i = threadIdx.x; i < n16; i += blockDim.x) cp_async16(d + 16 * i, s + 16 * i);
    for (size_t i = 16 * n16 + threadIdx.x; i < bytes; i += blockDim.x) d[i] = s[i];
}

// Stage Minv in dynamic shared memory when use_smem (blockDim threads copy).
template <class C>
__device__ __forceinline__ const C* stage_minv(const C* __restrict__ Minv_g, int q, int use_smem, unsigned char* sm) {
    if (!use_smem) return Minv_g;
    C* ms = reinterpret_cast<C*>(sm);
    block_copy_async(ms, Minv_g, (size_t)q * q * sizeof(C));
    cp_async_wait_all();
    __syncthreads();
    return ms;
}

template <class C, class FT, class TT, bool AOS = true>
__global__ void __launch_bounds__(1024)
k_coarse_solve(int n, const C* __restrict__ Minv_g, const FT* __restrict__ f, TT* __restrict__ T, int use_smem) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char cs_sm[];
    const C* Minv = stage_minv<C>(Minv_g, n * n * n - 1, use_smem, cs_sm);
    coarse_solve_block<C, FT, TT, AOS>(n, Minv, f, T);
}

}  // namespace otm
