// Shared-memory tiled (2.5D) form of the finest-grid 21-point stencil.
//
// A CTA of 32 x 8 threads owns a 32 x 8 tile of nodes in (x, y) and marches
// through TZ consecutive z-planes.  Shared memory holds three planes of the
// three fields (z-1, z, z+1) with a one-node periodic halo in x and y, and two
// planes of element conductivities (z-1, z) with the halo on the low side.
// While plane z is computed, the global loads of the next planes are already
// in flight in registers; they are stored to the free ring slot afterwards.
// Each field value and conductivity is read from global memory once per
// tile (plus the halo), and every neighbour access is a shared-memory load.
// Arithmetic and the difference form are those of kernels_fine.cuh.
#pragma once
#include "kernels_fine.cuh"

namespace otm {

constexpr int kTX = 32, kTY = 8;
constexpr int kPX = kTX + 2, kPY = kTY + 2;   // field plane with halo
constexpr int kKX = kTX + 1, kKY = kTY + 1;   // conductivity plane with low halo
constexpr int kUPlane = 3 * kPY * kPX;         // floats per field plane (3 load cases)
constexpr int kKPlane = kKY * kKX;
constexpr int kUPer = (kUPlane + 255) / 256;   // loads per thread per field plane
constexpr int kKPer = (kKPlane + 255) / 256;

inline bool tiled_ok(int n) { return n >= 8 && n % kTX == 0 && n % kTY == 0; }

// Tiled MODE 0 / 1 (see k_stencil_apply).  Grid: (n/32)(n/8)(n/tz) CTAs.
template <int MODE, bool DOT, class KT, class UT, class FT, class OT, class Fin>
__global__ void __launch_bounds__(256)
k_stencil_tiled(int n, int tz, const KT* __restrict__ k, const UT* __restrict__ u, const FT* __restrict__ f,
                OT* __restrict__ out, RedBuf rb, Fin fin) {
    pdl_enter();
    using C = float;
    __shared__ float us[3][kUPlane];
    __shared__ float ks[2][kKPlane];
    const size_t N = (size_t)n * n * n;
    const int ntx = n / kTX, nty = n / kTY;
    const int b = blockIdx.x;
    const int tix = b % ntx, tiy = (b / ntx) % nty, tiz = b / (ntx * nty);
    const int x0 = tix * kTX, y0 = tiy * kTY, z0 = tiz * tz;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + kTX * ty;
    const size_t nn = (size_t)n * n;

    // geometry of this thread's share of a plane load (fixed for all planes)
    int u_off[kUPer];
    int u_dst[kUPer];
#pragma unroll
    for (int j = 0; j < kUPer; ++j) {
        const int e = tid + 256 * j;
        if (e < kUPlane) {
            const int fi = e / (kPY * kPX), r = e % (kPY * kPX);
            const int yy = r / kPX, xx = r % kPX;
            const int gx = wrapd(x0, xx - 1, n), gy = wrapd(y0, yy - 1, n);
            u_off[j] = fi * 0 + gx + gy * n;   // in-plane offset; the field offset is added below
            u_dst[j] = e;
        } else {
            u_off[j] = -1;
            u_dst[j] = -1;
        }
    }
    int k_off[kKPer];
#pragma unroll
    for (int j = 0; j < kKPer; ++j) {
        const int e = tid + 256 * j;
        if (e < kKPlane) {
            const int yy = e / kKX, xx = e % kKX;
            k_off[j] = wrapd(x0, xx - 1, n) + wrapd(y0, yy - 1, n) * n;
        } else {
            k_off[j] = -1;
        }
    }
    auto field_of = [&](int e) { return e / (kPY * kPX); };

    float ureg[kUPer], kreg[kKPer];
    auto load_u = [&](int zp) {
        const size_t zo = (size_t)wrapd(zp, 0, n) * nn;
#pragma unroll
        for (int j = 0; j < kUPer; ++j)
            if (u_dst[j] >= 0) ureg[j] = (float)St<UT>::ld(u, (size_t)field_of(u_dst[j]) * N + zo + u_off[j]);
    };
    auto store_u = [&](int slot) {
#pragma unroll
        for (int j = 0; j < kUPer; ++j)
            if (u_dst[j] >= 0) us[slot][u_dst[j]] = ureg[j];
    };
    auto load_k = [&](int zp) {
        const size_t zo = (size_t)wrapd(zp, 0, n) * nn;
#pragma unroll
        for (int j = 0; j < kKPer; ++j)
            if (k_off[j] >= 0) kreg[j] = (float)St<KT>::ld(k, zo + k_off[j]);
    };
    auto store_k = [&](int slot) {
#pragma unroll
        for (int j = 0; j < kKPer; ++j)
            if (k_off[j] >= 0) ks[slot][tid + 256 * j] = kreg[j];
    };
    // ring indices: field plane p lives in slot p mod 3, conductivity plane p in slot p mod 2
    auto us3 = [](int p) { return ((p % 3) + 3) % 3; };
    auto ks2 = [](int p) { return p & 1; };

    // prologue: field planes z0-1, z0 and conductivity plane z0-1
    load_u(z0 - 1 + n);
    store_u(us3(z0 - 1));
    load_u(z0);
    store_u(us3(z0));
    load_k(z0 - 1 + n);
    store_k(ks2(z0 - 1 + 2));
    // in flight: field plane z0+1, conductivity plane z0
    load_u(z0 + 1);
    load_k(z0);

    Acc<C> acc[6];
    const int x = x0 + tx, y = y0 + ty;
    for (int z = z0; z < z0 + tz; ++z) {
        __syncthreads();                 // slot of plane z-2 (= z+1) and of k plane z-2 (= z) are free
        store_u(us3(z + 1));
        store_k(ks2(z));
        __syncthreads();
        if (z + 1 < z0 + tz) {           // issue the next planes' loads before computing this one
            load_u(z + 2);
            load_k(z + 1);
        }
        const float* U0 = us[us3(z - 1)];
        const float* U1 = us[us3(z)];
        const float* U2 = us[us3(z + 1)];
        const float* K0p = ks[ks2(z - 1 + 2)];
        const float* K1p = ks[ks2(z)];
        // k_abc: element (x-a, y-b, z-c)
        C kk[2][2][2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float* Kp = c ? K0p : K1p;
#pragma unroll
            for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                for (int a = 0; a < 2; ++a) kk[c][bb][a] = Kp[(ty + 1 - bb) * kKX + (tx + 1 - a)];
        }
        const size_t v = (size_t)x + (size_t)y * n + (size_t)z * nn;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int fo = i * kPY * kPX;
            auto Uat = [&](int dx, int dy, int dz) -> float {
                const float* P = dz < 0 ? U0 : (dz > 0 ? U2 : U1);
                return P[fo + (ty + 1 + dy) * kPX + (tx + 1 + dx)];
            };
            const C uc = Uat(0, 0, 0);
            C acc_nd = 0;
            // plane by plane, as nd_sum (kernels_fine.cuh)
            auto plane = [&](int c) {
#pragma unroll
                for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                    for (int a = 0; a < 2; ++a)
                        acc_nd += kk[c][bb][a] * (Uat(1 - 2 * a, 1 - 2 * bb, 1 - 2 * c) - uc);
#pragma unroll
                for (int a = 0; a < 2; ++a)
                    acc_nd += (kk[c][0][a] + kk[c][1][a]) * (Uat(1 - 2 * a, 0, 1 - 2 * c) - uc);
#pragma unroll
                for (int bb = 0; bb < 2; ++bb)
                    acc_nd += (kk[c][bb][0] + kk[c][bb][1]) * (Uat(0, 1 - 2 * bb, 1 - 2 * c) - uc);
            };
            plane(1);
#pragma unroll
            for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                for (int a = 0; a < 2; ++a)
                    acc_nd += (kk[0][bb][a] + kk[1][bb][a]) * (Uat(1 - 2 * a, 1 - 2 * bb, 0) - uc);
            plane(0);
            const C Ku = acc_nd * C(-1.0 / 12.0);
            C o;
            if (MODE == 0) {
                o = Ku;
            } else {
                const C fv = (C)St<FT>::ld(f + (size_t)i * N, v);
                o = fv - Ku;
                if (DOT) acc[3 + i].add_prod(fv, fv);
            }
            St<OT>::st(out + (size_t)i * N, v, (typename St<OT>::C)o);
            if (DOT) {
                if (MODE == 0) acc[i].add_prod(uc, o);
                else acc[i].add_prod(o, o);
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

// z-planes per CTA: the largest power-of-two divisor of n that still gives
// at least 3 CTAs per SM, and never more CTAs than the reduction partials
// hold.  Returns 0 when no such split exists (the caller then uses the
// gather kernel).
inline int tiled_tz(int n, int sm_count, int max_blocks) {
    if (!tiled_ok(n)) return 0;
    const long long tiles = (long long)(n / kTX) * (n / kTY);
    int tz = n;
    while (tz % 2 == 0 && tz > 4 && tiles * (n / tz) < 3LL * sm_count) tz /= 2;
    if (tiles * (n / tz) > max_blocks) return 0;
    return tz;
}

}  // namespace otm
