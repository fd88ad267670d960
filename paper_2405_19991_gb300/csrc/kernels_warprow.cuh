// Warp-row forms of finest-grid kernels (n a multiple of 128): the fine
// prolongation, the residual of the FP32-pair iterate and its error-free
// check.
//
// A warp covers 128 consecutive x of one (y, z) row; lane l owns the four
// nodes x = x0 + 4l .. x0 + 4l + 3.  For every neighbouring row the lane
// loads its four values with one vector access, and the values at x - 1 and
// x + 4 come from the neighbouring lanes by shuffle (lane 0 / lane 31 wrap
// periodically when one warp spans the whole row, and load the value
// otherwise).  Rows are folded into the four node sums as they arrive, so
// one row is live at a time.  (Measured at 128^3, this layout is faster than
// the row-mapped kernels for these three, and slower than the tiled stencil
// and the row-mapped Gauss-Seidel pass, which the solver uses instead.)
#pragma once
#include "kernels_fine.cuh"

namespace otm {

inline bool warprow_ok(int n) { return n >= 128 && n % 128 == 0; }

// CTAs per SM the two residual kernels are compiled for (3: 80 registers).
#ifndef OTM_WR_MINB
#define OTM_WR_MINB 3
#endif

// Values of one row at x0+4l-1 .. x0+4l+4 (six floats).
template <class T>
__device__ __forceinline__ void row6(const T* __restrict__ F, size_t ro, int xb, int n, int lane, bool whole,
                                     float (&v)[6]) {
    const Q4<float> q = ld4f(F, ro + (size_t)xb);
    v[1] = q.v[0];
    v[2] = q.v[1];
    v[3] = q.v[2];
    v[4] = q.v[3];
    v[0] = __shfl_sync(0xffffffffu, v[4], (lane + 31) & 31);
    v[5] = __shfl_sync(0xffffffffu, v[1], (lane + 1) & 31);
    if (!whole) {
        if (lane == 0) v[0] = (float)St<T>::ld(F, ro + (size_t)(xb == 0 ? n - 1 : xb - 1));
        if (lane == 31) v[5] = (float)St<T>::ld(F, ro + (size_t)(xb + 4 == n ? 0 : xb + 4));
    }
}

// Row offsets of the 3 x 3 (y, z) neighbourhood: ro[dz+1][dy+1].  32-bit:
// the solver's grids have n <= 512, so an offset within a field is < 2^28.
__device__ __forceinline__ void row_offsets(int n, int y, int z, unsigned (&ro)[3][3]) {
    const unsigned nn = (unsigned)n * n;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
            ro[dz + 1][dy + 1] = (unsigned)wrapd(y, dy, n) * n + (unsigned)wrapd(z, dz, n) * nn;
}

template <class KT>
__device__ __forceinline__ void load_k_rows(const KT* __restrict__ k, int n, int y, int z, int xb, int lane,
                                            bool whole, float (&kr)[2][2][6]) {
    const size_t nn = (size_t)n * n;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
            row6<KT>(k, (size_t)wrapd(y, -b, n) * n + (size_t)wrapd(z, -c, n) * nn, xb, n, lane, whole, kr[c][b]);
}

// Contribution of the neighbouring row (dy, dz) (six values v at x-1..x+4)
// to the neighbour sums of the lane's four nodes.  Coefficients as in
// kernels_fine.cuh: corners carry k_abc, edges the sum of the two elements
// sharing them; face neighbours and the centre carry nothing.  DIFF
// subtracts the centre value uc[j] (difference form).
template <bool DIFF>
__device__ __forceinline__ void add_row(int dy, int dz, const float (&v)[6], const float (&kr)[2][2][6],
                                        const float (&uc)[4], float (&acc)[4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float c0 = DIFF ? uc[j] : 0.f;
        const float vm = v[j] - c0, v0 = v[1 + j] - c0, vp = v[2 + j] - c0;   // x-1, x, x+1
        auto K = [&](int c, int b, int a) -> float { return kr[c][b][1 + j - a]; };
        if (dy != 0 && dz != 0) {
            const int b = (1 - dy) / 2, c = (1 - dz) / 2;
            acc[j] += K(c, b, 0) * vp + K(c, b, 1) * vm + (K(c, b, 0) + K(c, b, 1)) * v0;
        } else if (dy != 0) {
            const int b = (1 - dy) / 2;
            acc[j] += (K(0, b, 0) + K(1, b, 0)) * vp + (K(0, b, 1) + K(1, b, 1)) * vm;
        } else if (dz != 0) {
            const int c = (1 - dz) / 2;
            acc[j] += (K(c, 0, 0) + K(c, 1, 0)) * vp + (K(c, 0, 1) + K(c, 1, 1)) * vm;
        }
    }
}

// Prolongation + correction on the finest grid, T += P Tc (trilinear).  Lane
// l's four fine nodes x = 4l..4l+3 (within the warp's 128) use the coarse
// values at 2l, 2l+1, 2l+2.
template <class CT, class TT>
__global__ void __launch_bounds__(256)
k_prolong_wr(int nf, const CT* __restrict__ Tc, TT* __restrict__ T) {
    pdl_enter();
    const int nc = nf / 2;
    const size_t Nf = (size_t)nf * nf * nf;
    const int lane = threadIdx.x & 31;
    const int wpr = nf / 128;
    const long long nwarps = (long long)nf * nf * wpr;
    for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nwarps;
         w += ((long long)gridDim.x * blockDim.x) >> 5) {
        const int seg = (int)(w % wpr);
        const int row = (int)(w / wpr);
        const int y = row % nf, z = row / nf;
        const int xb = seg * 128 + 4 * lane;
        const int cxb = xb / 2;                      // even
        int yi[2], zi[2];
        float wy[2], wz[2];
        int cy = 1, cz = 1;
        if (y & 1) { yi[0] = y >> 1; yi[1] = wrapp(y >> 1, nc); wy[0] = wy[1] = 0.5f; cy = 2; }
        else { yi[0] = yi[1] = y >> 1; wy[0] = 1.f; wy[1] = 0.f; }
        if (z & 1) { zi[0] = z >> 1; zi[1] = wrapp(z >> 1, nc); wz[0] = wz[1] = 0.5f; cz = 2; }
        else { zi[0] = zi[1] = z >> 1; wz[0] = 1.f; wz[1] = 0.f; }
        const size_t vb = (size_t)row * nf + (size_t)xb;
        // the coarse field is node-major ([Nc][4]): one load brings a node's
        // three load cases; per load case the sums run in the same order
        float s[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        auto tc3 = [&](size_t node, float (&a)[3]) {
            typename St<CT>::C q[3];
            ld_f3<CT>(Tc, node, q);
#pragma unroll
            for (int i = 0; i < 3; ++i) a[i] = (float)q[i];
        };
        for (int c = 0; c < cz; ++c)
            for (int b = 0; b < cy; ++b) {
                const size_t ro = (size_t)yi[b] * nc + (size_t)zi[c] * nc * nc;
                float a0[3], a1[3], a2[3];
                tc3(ro + cxb, a0);
                tc3(ro + cxb + 1, a1);
#pragma unroll
                for (int i = 0; i < 3; ++i) a2[i] = __shfl_sync(0xffffffffu, a0[i], (lane + 1) & 31);
                if (lane == 31 && wpr > 1) tc3(ro + (size_t)(cxb + 2 == nc ? 0 : cxb + 2), a2);
                const float wgt = wz[c] * wy[b];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    s[i][0] += wgt * a0[i];
                    s[i][1] += wgt * a1[i];
                    s[i][2] += wgt * a2[i];
                }
            }
        Q4<float> t[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) t[i] = ld4f(T + (size_t)i * Nf, vb);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            t[i].v[0] += s[i][0];
            t[i].v[1] += 0.5f * (s[i][0] + s[i][1]);
            t[i].v[2] += s[i][1];
            t[i].v[3] += 0.5f * (s[i][1] + s[i][2]);
            st4f(T + (size_t)i * Nf, vb, t[i]);
        }
    }
}

// Values of row (dy, dz) of the pair field hi + lo minus the centre pair, each
// difference rounded once: d[t] for x-1..x+4 relative to node t-1 ... (the
// centre of node j is (hv[j], lv[j])).
__device__ __forceinline__ void pair_row(const float* __restrict__ xh, const float* __restrict__ xl, size_t ro, int xb,
                                         int n, int lane, bool whole, float (&vh)[6], float (&vl)[6]) {
    row6<float>(xh, ro, xb, n, lane, whole, vh);
    if (xl) row6<float>(xl, ro, xb, n, lane, whole, vl);
    else
#pragma unroll
        for (int t = 0; t < 6; ++t) vl[t] = 0.f;
}

// The error-free check processes the lane's four nodes as two pairs, nodes
// (0, 2) and (1, 3), one packed FP32x2 instruction per pair.  Pair jp at
// x-offset dx reads the row values of nodes jp + dx and jp + 2 + dx:
// P[1 + jp + dx] with P[t] = (v[t], v[t + 2]).
__device__ __forceinline__ void pair_cols(const float (&v)[6], float2 (&P)[4]) {
#pragma unroll
    for (int t = 0; t < 4; ++t) P[t] = make_float2(v[t], v[t + 2]);
}

// The pair differences of row (dy, dz) for both node pairs and the three
// x-offsets: D[jp][dx + 1] = (u_w - u_v) of nodes jp and jp + 2, each
// rounded once (df_diff on both lanes).
__device__ __forceinline__ void row_diffs(const float (&vh)[6], const float (&vl)[6], const float2 (&ch)[2],
                                          const float2 (&cl)[2], float2 (&D)[2][3]) {
    float2 PH[4], PL[4];
    pair_cols(vh, PH);
    pair_cols(vl, PL);
#pragma unroll
    for (int jp = 0; jp < 2; ++jp)
#pragma unroll
        for (int t = 0; t < 3; ++t) D[jp][t] = df_diff2(PH[jp + t], PL[jp + t], ch[jp], cl[jp]);
}

// Lane j of the pair layout: node j is lane j >> 1 of pair j & 1.
__device__ __forceinline__ float pair_lane(const float2& p, int j) { return (j >> 1) ? p.y : p.x; }

// r = f - K (hi + lo) (residual of the FP32-pair iterate; lo may be null),
// reducing ||r||^2 and ||f||^2 into FinInit.
template <class Fin>
__global__ void __launch_bounds__(256, OTM_WR_MINB)
k_residual_x2_wr(int n, const float* __restrict__ k, const float* __restrict__ xh, const float* __restrict__ xl,
                 const float* __restrict__ f, float* __restrict__ r, RedBuf rb, Fin fin) {
    pdl_enter();
    const size_t N = (size_t)n * n * n;
    const int lane = threadIdx.x & 31;
    const int wpr = n / 128;
    const bool whole = wpr == 1;
    const long long nwarps = (long long)n * n * wpr;
    Acc<float> acc[6];
    for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nwarps;
         w += ((long long)gridDim.x * blockDim.x) >> 5) {
        const int seg = (int)(w % wpr);
        const int row = (int)(w / wpr);
        const int y = row % n, z = row / n;
        const int xb = seg * 128 + 4 * lane;
        unsigned ro[3][3];
        row_offsets(n, y, z, ro);
        float kr[2][2][6];
        load_k_rows<float>(k, n, y, z, xb, lane, whole, kr);
        const size_t vb = ro[1][1] + (size_t)xb;
#pragma unroll 1
        for (int i = 0; i < 3; ++i) {
            const size_t fo = (size_t)i * N;
            const Q4<float> ch = ld4f(xh + fo, vb);
            Q4<float> cl{{0.f, 0.f, 0.f, 0.f}};
            if (xl) cl = ld4f(xl + fo, vb);
            const float zero4[4] = {0.f, 0.f, 0.f, 0.f};
            float nd[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
                for (int dy = -1; dy <= 1; ++dy) {
                    if (dy == 0 && dz == 0) continue;
                    float vh[6], vl[6];
                    pair_row(xh + fo, xl ? xl + fo : nullptr, ro[dz + 1][dy + 1], xb, n, lane, whole, vh, vl);
                    // the three x-neighbours of node j as pair differences,
                    // placed where add_row reads them for node j (scalar: the
                    // packed form of these differences measured 123 against
                    // 115 us here, its pair moves costing more than it saves)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float d[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                        for (int t = 0; t < 3; ++t) d[j + t] = df_diff(vh[j + t], vl[j + t], ch.v[j], cl.v[j]);
                        float a[4] = {0.f, 0.f, 0.f, 0.f};
                        add_row<false>(dy, dz, d, kr, zero4, a);
                        nd[j] += a[j];
                    }
                }
            const Q4<float> fv = ld4f(f + fo, vb);
            Q4<float> o;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                o.v[j] = fv.v[j] + nd[j] * (1.0f / 12.0f);
                acc[i].add_prod(o.v[j], o.v[j]);
                acc[3 + i].add_prod(fv.v[j], fv.v[j]);
            }
            st4f(r + fo, vb, o);
        }
    }
    __shared__ double res[6];
    if (grid_reduce<6>(acc, rb, res)) {
        if (is_thread0()) fin(res);
    }
}

// Packed forms of elem_add / elem_sub4 (kernels_fine.cuh): each lane runs
// the scalar sequence, so both lanes are bitwise the scalar element form.
__device__ __forceinline__ void elem_add2(float2& t, float2& sg, float2 h, float2 l) {
    float2 u, e;
    two_sum2(t, h, u, e);
    t = u;
    sg = __fadd2_rn(sg, __fadd2_rn(e, l));
}
__device__ __forceinline__ void elem_sub4_2(float2& t, float2& sg, float2 h4, float2 l4) {
    const float2 u = f2_sub(t, h4);
    const float2 bp = f2_sub(u, t);
    const float2 e = f2_sub(f2_sub(t, f2_sub(u, bp)), __fadd2_rn(h4, bp));
    t = u;
    sg = __fadd2_rn(sg, f2_sub(e, l4));
}

// ||f - K (hi + lo)||^2 with error-free element terms (see k_true_residual).
// ELEM (default): the element form of nd_sum_elem -- per node eight element
// sums d_e held unrounded as t + sg and eight TwoProduct terms -- two nodes
// per packed instruction; a quadrant (b, c) of elements reads its three
// neighbour rows (dy, dz), (dy, 0) and (0, dz) in turn.  !ELEM: the pair
// form (OTM_CHECK_FORM=pair): each of the 32 terms k_e (u_w - u_v) with the
// difference rounded once, formed with TwoProduct and summed with TwoSum.
// Measured at 128^3 against the residual of the stored iterate recomputed
// in FP64: the element form within 1e-9 relative, the pair form 0.1-0.4 %
// off; and faster (the design iteration 1974 -> 1951 us at 128^3, 11.47 ->
// 11.16 ms at 256^3), with 44 bytes of spills at 80 registers against the
// pair form's 244.
template <class Fin, bool ELEM = true>
__global__ void __launch_bounds__(256, OTM_WR_MINB)
k_true_residual_wr(int n, const float* __restrict__ k, const float* __restrict__ xh, const float* __restrict__ xl,
                   const float* __restrict__ f, RedBuf rb, Fin fin) {
    pdl_enter();
    const size_t N = (size_t)n * n * n;
    const int lane = threadIdx.x & 31;
    const int wpr = n / 128;
    const bool whole = wpr == 1;
    const long long nwarps = (long long)n * n * wpr;
    Acc<float> acc[6];
    for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nwarps;
         w += ((long long)gridDim.x * blockDim.x) >> 5) {
        const int seg = (int)(w % wpr);
        const int row = (int)(w / wpr);
        const int y = row % n, z = row / n;
        const int xb = seg * 128 + 4 * lane;
        unsigned ro[3][3];
        row_offsets(n, y, z, ro);
        // the pair form holds the four element rows for the whole warp row;
        // the element form loads each quadrant's row where it needs it
        float kr[2][2][6];
        if constexpr (!ELEM) load_k_rows<float>(k, n, y, z, xb, lane, whole, kr);
        const size_t vb = ro[1][1] + (size_t)xb;
#pragma unroll 1
        for (int i = 0; i < 3; ++i) {
            const size_t fo = (size_t)i * N;
            const Q4<float> ch = ld4f(xh + fo, vb);
            Q4<float> cl{{0.f, 0.f, 0.f, 0.f}};
            if (xl) cl = ld4f(xl + fo, vb);
            const float2 ch2[2] = {make_float2(ch.v[0], ch.v[2]), make_float2(ch.v[1], ch.v[3])};
            const float2 cl2[2] = {make_float2(cl.v[0], cl.v[2]), make_float2(cl.v[1], cl.v[3])};
            // running sums s + c of the pair (jp, jp + 2), both lanes at once
            float2 S[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            float2 Cc[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            if constexpr (ELEM) {
                const float2 four = make_float2(4.f, 4.f);
                const float2 H4[2] = {__fmul2_rn(four, ch2[0]), __fmul2_rn(four, ch2[1])};
                const float2 L4[2] = {__fmul2_rn(four, cl2[0]), __fmul2_rn(four, cl2[1])};
                // one quadrant per trip (not unrolled: a quadrant's rows are
                // loaded where it needs them, which bounds the registers and
                // the code size)
#pragma unroll 1
                for (int q = 0; q < 4; ++q) {
                    const int cc = q >> 1, b = q & 1;
                    const int dy = 1 - 2 * b, dz = 1 - 2 * cc;
                    const unsigned nn = (unsigned)n * n;
                    const unsigned oy = (unsigned)wrapd(y, dy, n) * n, oz = (unsigned)wrapd(z, dz, n) * nn;
                    // T[a][jp], G[a][jp]: element (a, b, cc) of the pair jp
                    float2 T[2][2], G[2][2];
                    float kq[6];   // element row (y - b, z - cc)
                    row6<float>(k, (size_t)wrapd(y, -b, n) * n + (size_t)wrapd(z, -cc, n) * nn, xb, n, lane,
                                whole, kq);
                    {
                        float vh[6], vl[6];
                        pair_row(xh + fo, xl ? xl + fo : nullptr, oy + oz, xb, n, lane, whole, vh, vl);
                        float2 PH[4], PL[4];
                        pair_cols(vh, PH);
                        pair_cols(vl, PL);
#pragma unroll
                        for (int a = 0; a < 2; ++a)
#pragma unroll
                            for (int jp = 0; jp < 2; ++jp) {
                                const int dx = 1 - 2 * a;
                                T[a][jp] = PH[1 + jp];   // (x, y + dy, z + dz)
                                G[a][jp] = PL[1 + jp];
                                elem_add2(T[a][jp], G[a][jp], PH[1 + jp + dx], PL[1 + jp + dx]);
                            }
                    }
#pragma unroll
                    for (int r2 = 0; r2 < 2; ++r2) {
                        // rows (dy, 0), then (0, dz)
                        float vh[6], vl[6];
                        pair_row(xh + fo, xl ? xl + fo : nullptr,
                                 r2 == 0 ? oy + (unsigned)z * nn : (unsigned)y * n + oz, xb, n, lane, whole, vh, vl);
                        float2 PH[4], PL[4];
                        pair_cols(vh, PH);
                        pair_cols(vl, PL);
#pragma unroll
                        for (int a = 0; a < 2; ++a)
#pragma unroll
                            for (int jp = 0; jp < 2; ++jp) {
                                const int dx = 1 - 2 * a;
                                elem_add2(T[a][jp], G[a][jp], PH[1 + jp + dx], PL[1 + jp + dx]);
                            }
                    }
#pragma unroll
                    for (int a = 0; a < 2; ++a)
#pragma unroll
                        for (int jp = 0; jp < 2; ++jp) {
                            elem_sub4_2(T[a][jp], G[a][jp], H4[jp], L4[jp]);
                            // conductivity k_{cc,b,a} of nodes jp and jp + 2; TwoProduct per lane
                            const float k0 = kq[1 + jp - a], k1 = kq[3 + jp - a];
                            const float2 t = T[a][jp], sg = G[a][jp];
                            const float2 p = make_float2(__fmul_rn(k0, t.x), __fmul_rn(k1, t.y));
                            const float2 pe = make_float2(fmaf(k0, sg.x, fmaf(k0, t.x, -p.x)),
                                                          fmaf(k1, sg.y, fmaf(k1, t.y, -p.y)));
                            float2 u, e;
                            two_sum2(S[jp], p, u, e);
                            S[jp] = u;
                            Cc[jp] = __fadd2_rn(Cc[jp], __fadd2_rn(e, pe));
                        }
                }
            } else {
#pragma unroll
            for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
                for (int dy = -1; dy <= 1; ++dy) {
                    if (dy == 0 && dz == 0) continue;
                    float vh[6], vl[6];
                    pair_row(xh + fo, xl ? xl + fo : nullptr, ro[dz + 1][dy + 1], xb, n, lane, whole, vh, vl);
                    float2 Dr[2][3];
                    row_diffs(vh, vl, ch2, cl2, Dr);
#pragma unroll
                    for (int jp = 0; jp < 2; ++jp) {
                        // TwoProduct per lane, TwoSum of the pair's running sums
                        auto term = [&](float k0, float k1, float2 d) {
                            const float2 p = make_float2(__fmul_rn(k0, d.x), __fmul_rn(k1, d.y));
                            const float2 pe = make_float2(fmaf(k0, d.x, -p.x), fmaf(k1, d.y, -p.y));
                            float2 t, e;
                            two_sum2(S[jp], p, t, e);
                            S[jp] = t;
                            Cc[jp] = __fadd2_rn(Cc[jp], __fadd2_rn(e, pe));
                        };
                        auto D = [&](int dx) -> float2 { return Dr[jp][dx + 1]; };
                        // conductivity k_{cc,b,a} of nodes jp and jp + 2
                        auto K0 = [&](int cc, int b, int a) -> float { return kr[cc][b][1 + jp - a]; };
                        auto K1 = [&](int cc, int b, int a) -> float { return kr[cc][b][3 + jp - a]; };
                        if (dy != 0 && dz != 0) {
                            const int b = (1 - dy) / 2, cc = (1 - dz) / 2;
                            const float2 d0 = D(0);
                            term(K0(cc, b, 0), K1(cc, b, 0), D(1));
                            term(K0(cc, b, 1), K1(cc, b, 1), D(-1));
                            term(K0(cc, b, 0), K1(cc, b, 0), d0);
                            term(K0(cc, b, 1), K1(cc, b, 1), d0);
                        } else if (dy != 0) {
                            const int b = (1 - dy) / 2;
                            const float2 dp = D(1), dm = D(-1);
                            term(K0(0, b, 0), K1(0, b, 0), dp);
                            term(K0(1, b, 0), K1(1, b, 0), dp);
                            term(K0(0, b, 1), K1(0, b, 1), dm);
                            term(K0(1, b, 1), K1(1, b, 1), dm);
                        } else {
                            const int cc = (1 - dz) / 2;
                            const float2 dp = D(1), dm = D(-1);
                            term(K0(cc, 0, 0), K1(cc, 0, 0), dp);
                            term(K0(cc, 1, 0), K1(cc, 1, 0), dp);
                            term(K0(cc, 0, 1), K1(cc, 0, 1), dm);
                            term(K0(cc, 1, 1), K1(cc, 1, 1), dm);
                        }
                    }
                }
            }
            const Q4<float> fv = ld4f(f + fo, vb);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float fvj = fv.v[j];
                const float sj = pair_lane(S[j & 1], j), cj = pair_lane(Cc[j & 1], j);
                const float rv = resid_exact12<float>(fvj, sj, cj);
                acc[i].add_prod(rv, rv);
                acc[3 + i].add_prod(fvj, fvj);
            }
        }
    }
    __shared__ double res[6];
    if (grid_reduce<6>(acc, rb, res)) {
        if (is_thread0()) fin(res);
    }
}

}  // namespace otm
