// Paired-node form of the finest-grid 21-point stencil (the operator of
// Sec. 2.4 on the three load cases), FP32.
//
// Same 2.5D scheme as kernels_tiled.cuh -- a CTA owns a 64 x 8 tile of nodes
// in (x, y) and marches through tz z-planes with a three-plane ring of the
// fields and a two-plane ring of element conductivities in shared memory,
// the next planes' global loads in flight in registers -- but each thread
// computes two neighbouring nodes (x, x + 1).  Their neighbourhoods overlap,
// so the 21 field values and 8 conductivities a node needs come from 64-bit
// shared loads shared by the pair, and the arithmetic runs on packed FP32
// pairs (__ffma2_rn and friends, one instruction for both nodes).  Each lane
// performs exactly the operations, in the same order, that the tiled and
// gather kernels perform for its node, so all three give bitwise equal
// results.  The stencil is issue-bound in its one-node forms (shared loads
// and FP instructions per node); pairing roughly halves both.
#pragma once
#include <algorithm>
#include <cstdlib>

#include "kernels_fine.cuh"

namespace otm {

constexpr int kX2T = 32, kX2Y = 8;              // threads per CTA: 32 x 8
constexpr int kX2N = 2 * kX2T;                   // nodes per tile in x
constexpr int kX2PX = kX2N + 2, kX2PY = kX2Y + 2;   // field plane with halo (66 x 10)
constexpr int kX2KX = kX2N + 2, kX2KY = kX2Y + 1;   // conductivity plane, low halo (65 used, 66 for alignment)
constexpr int kX2UPlane = 3 * kX2PY * kX2PX;
constexpr int kX2KPlane = kX2KY * kX2KX;
constexpr int kX2UPer = (kX2UPlane + 255) / 256;
constexpr int kX2KPer = (kX2KPlane + 255) / 256;

// Fine-grid stencil form: 0 z-reuse paired (where it applies), 3 paired
// three-plane ring, 1 shared-memory tiled, 2 gather
// (OTM_STENCIL=zr|pair|tiled|gather; default zr), for comparisons.
inline int stencil_choice() {
    static int c = [] {
        const char* e = getenv("OTM_STENCIL");
        if (!e) return 0;
        if (e[0] == 't') return 1;
        if (e[0] == 'g') return 2;
        if (e[0] == 'p') return 3;
        return 0;
    }();
    return c;
}

#ifndef OTM_X2_MINB
#define OTM_X2_MINB 2
#endif
template <bool DOT, class Fin>
__global__ void __launch_bounds__(256, OTM_X2_MINB)
k_stencil_x2(int n, int tz, const float* __restrict__ k, const float* __restrict__ u, float* __restrict__ out,
             RedBuf rb, Fin fin) {
    pdl_enter();
    __shared__ __align__(16) float us[3][kX2UPlane];
    __shared__ __align__(16) float ks[2][kX2KPlane];
    const size_t N = (size_t)n * n * n;
    const int ntx = n / kX2N, nty = n / kX2Y;
    const int b = blockIdx.x;
    const int tix = b % ntx, tiy = (b / ntx) % nty, tiz = b / (ntx * nty);
    const int x0 = tix * kX2N, y0 = tiy * kX2Y, z0 = tiz * tz;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + kX2T * ty;
    const size_t nn = (size_t)n * n;

    // this thread's share of a plane load (fixed for all planes)
    int u_off[kX2UPer];   // in-plane offset; the field is (tid + 256 j) / (kX2PY kX2PX)
#pragma unroll
    for (int j = 0; j < kX2UPer; ++j) {
        const int e = tid + 256 * j;
        if (e < kX2UPlane) {
            const int r = e % (kX2PY * kX2PX);
            const int yy = r / kX2PX, xx = r % kX2PX;
            u_off[j] = wrapd(x0, xx - 1, n) + wrapd(y0, yy - 1, n) * n;
        } else {
            u_off[j] = -1;
        }
    }
    int k_off[kX2KPer];
#pragma unroll
    for (int j = 0; j < kX2KPer; ++j) {
        const int e = tid + 256 * j;
        const int yy = e / kX2KX, xx = e % kX2KX;
        k_off[j] = (e < kX2KPlane && xx <= kX2N) ? wrapd(x0, xx - 1, n) + wrapd(y0, yy - 1, n) * n : -1;
    }

    float ureg[kX2UPer], kreg[kX2KPer];
    auto load_u = [&](int zp) {
        const size_t zo = (size_t)wrapd(zp, 0, n) * nn;
#pragma unroll
        for (int j = 0; j < kX2UPer; ++j)
            if (u_off[j] >= 0) ureg[j] = u[(size_t)((tid + 256 * j) / (kX2PY * kX2PX)) * N + zo + u_off[j]];
    };
    auto store_u = [&](int slot) {
#pragma unroll
        for (int j = 0; j < kX2UPer; ++j)
            if (u_off[j] >= 0) us[slot][tid + 256 * j] = ureg[j];
    };
    auto load_k = [&](int zp) {
        const size_t zo = (size_t)wrapd(zp, 0, n) * nn;
#pragma unroll
        for (int j = 0; j < kX2KPer; ++j)
            if (k_off[j] >= 0) kreg[j] = k[zo + k_off[j]];
    };
    auto store_k = [&](int slot) {
#pragma unroll
        for (int j = 0; j < kX2KPer; ++j)
            if (k_off[j] >= 0) ks[slot][tid + 256 * j] = kreg[j];
    };
    auto us3 = [](int p) { return ((p % 3) + 3) % 3; };
    auto ks2 = [](int p) { return p & 1; };

    load_u(z0 - 1 + n);
    store_u(us3(z0 - 1));
    load_u(z0);
    store_u(us3(z0));
    load_k(z0 - 1 + n);
    store_k(ks2(z0 - 1 + 2));
    load_u(z0 + 1);
    load_k(z0);

    Acc<float> acc[6];
    const int x = x0 + 2 * tx, y = y0 + ty;
    const int c0 = 2 * tx;   // shared column of node x - 1 (fields) / element x - 1 (conductivities)
    const float2 m12 = make_float2(-1.0f / 12.0f, -1.0f / 12.0f);
    for (int z = z0; z < z0 + tz; ++z) {
        __syncthreads();
        store_u(us3(z + 1));
        store_k(ks2(z));
        __syncthreads();
        if (z + 1 < z0 + tz) {
            load_u(z + 2);
            load_k(z + 1);
        }
        const float* U0 = us[us3(z - 1)];
        const float* U1 = us[us3(z)];
        const float* U2 = us[us3(z + 1)];
        const float* K0p = ks[ks2(z - 1 + 2)];
        const float* K1p = ks[ks2(z)];
        // K[c][b][a] = (k of element (x - a, y - b, z - c), same for x + 1)
        float2 K[2][2][2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float* Kp = c ? K0p : K1p;
#pragma unroll
            for (int bb = 0; bb < 2; ++bb) {
                const float* row = Kp + (ty + 1 - bb) * kX2KX;
                const float2 lo = *reinterpret_cast<const float2*>(row + c0);   // elements x - 1, x
                const float hi = row[c0 + 2];                                   // element x + 1
                K[c][bb][1] = lo;
                K[c][bb][0] = make_float2(lo.y, hi);
            }
        }
        const size_t v = (size_t)x + (size_t)y * n + (size_t)z * nn;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            // one load case at a time: the warp barrier keeps the compiler from
            // hoisting the next case's 21 shared loads (register pressure)
            __syncwarp();
            const int fo = i * kX2PY * kX2PX;
            // pair of values at offset (dx, dy, dz) for the nodes (x, x + 1)
            auto Uat = [&](int dx, int dy, int dz) -> float2 {
                const float* P = dz < 0 ? U0 : (dz > 0 ? U2 : U1);
                const float* row = P + fo + (ty + 1 + dy) * kX2PX + c0;
                if (dx < 0) return *reinterpret_cast<const float2*>(row);
                if (dx > 0) return *reinterpret_cast<const float2*>(row + 2);
                return make_float2(row[1], row[2]);
            };
            const float2 uc = Uat(0, 0, 0);
            float2 nd = make_float2(0.f, 0.f);
            // the four groups of neighbours in the order every stencil form
            // sums them; a warp barrier between groups bounds the values the
            // compiler keeps in flight
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                    for (int a = 0; a < 2; ++a)
                        nd = __ffma2_rn(K[c][bb][a], f2_sub(Uat(1 - 2 * a, 1 - 2 * bb, 1 - 2 * c), uc), nd);
            __syncwarp();
#pragma unroll
            for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                for (int a = 0; a < 2; ++a)
                    nd = __ffma2_rn(__fadd2_rn(K[0][bb][a], K[1][bb][a]), f2_sub(Uat(1 - 2 * a, 1 - 2 * bb, 0), uc), nd);
            __syncwarp();
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int a = 0; a < 2; ++a)
                    nd = __ffma2_rn(__fadd2_rn(K[c][0][a], K[c][1][a]), f2_sub(Uat(1 - 2 * a, 0, 1 - 2 * c), uc), nd);
            __syncwarp();
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int bb = 0; bb < 2; ++bb)
                    nd = __ffma2_rn(__fadd2_rn(K[c][bb][0], K[c][bb][1]), f2_sub(Uat(0, 1 - 2 * bb, 1 - 2 * c), uc), nd);
            const float2 o = __fmul2_rn(nd, m12);
            *reinterpret_cast<float2*>(out + (size_t)i * N + v) = o;
            if (DOT) {
                acc[i].add_prod(uc.x, o.x);
                acc[i].add_prod(uc.y, o.y);
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

inline bool x2_ok(int n) { return n >= kX2N && n % kX2N == 0 && n % kX2Y == 0; }

// z-planes per CTA: the largest power-of-two divisor of n that still gives
// at least 3 CTAs per SM and no more CTAs than the reduction partials hold;
// 0 when the paired form does not apply.
inline int x2_tz(int n, int sm_count, int max_blocks) {
    if (!x2_ok(n)) return 0;
    const long long tiles = (long long)(n / kX2N) * (n / kX2Y);
    int tz = n;
    const char* e = getenv("OTM_X2_TZ");
    if (e && atoi(e) >= 1 && n % atoi(e) == 0) {
        tz = atoi(e);
    } else {
        while (tz % 2 == 0 && tz > 2 && tiles * (n / tz) < 3LL * sm_count) tz /= 2;
    }
    if (tiles * (n / tz) > max_blocks) return 0;
    return tz;
}
inline int x2_grid(int n, int tz) { return (n / kX2N) * (n / kX2Y) * (n / tz); }

}  // namespace otm

namespace otm {

// z-reuse form of the paired stencil: a CTA handles one load case of a
// 64 x 8 tile over one of m equal z-chunks (planes c n / m .. (c + 1) n / m;
// 1-D grid, the load case fastest so a tile's three CTAs run together and
// share its conductivities in L2), and keeps, per thread, the node pair's
// neighbour rows (x - 1 .. x + 2 at y - 1 .. y + 1) of planes z - 1, z, z + 1
// and the conductivities of element planes z - 1, z in registers.  Marching
// one plane in z loads only the new plane's rows from shared memory (one
// staged plane, double-buffered; one barrier per plane), about half the
// shared-memory traffic per node of the three-plane ring.  Same arithmetic
// and operation order as every other stencil form (bitwise equal results).
template <bool DOT, class Fin>
__global__ void __launch_bounds__(256, 3)
k_stencil_zr(int n, int m, const float* __restrict__ k, const float* __restrict__ u, float* __restrict__ out,
             RedBuf rb, Fin fin) {
    pdl_enter();
    constexpr int UP = kX2PY * kX2PX;            // one field plane with halo
    constexpr int UPer = (UP + 255) / 256;
    __shared__ __align__(16) float us[2][UP];
    __shared__ __align__(16) float ks[2][kX2KPlane];
    const size_t N = (size_t)n * n * n;
    const int ntx = n / kX2N, nty = n / kX2Y;
    const int fi = blockIdx.x % 3;               // load case
    const int b = blockIdx.x / 3;
    const int tix = b % ntx, tiy = (b / ntx) % nty, tiz = b / (ntx * nty);
    const int x0 = tix * kX2N, y0 = tiy * kX2Y;
    const int z0 = tiz * n / m, z1 = (tiz + 1) * n / m;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + kX2T * ty;
    const size_t nn = (size_t)n * n;
    const float* uf = u + (size_t)fi * N;

    int u_off[UPer];
#pragma unroll
    for (int j = 0; j < UPer; ++j) {
        const int e = tid + 256 * j;
        const int yy = e / kX2PX, xx = e % kX2PX;
        u_off[j] = e < UP ? wrapd(x0, xx - 1, n) + wrapd(y0, yy - 1, n) * n : -1;
    }
    int k_off[kX2KPer];
#pragma unroll
    for (int j = 0; j < kX2KPer; ++j) {
        const int e = tid + 256 * j;
        const int yy = e / kX2KX, xx = e % kX2KX;
        k_off[j] = (e < kX2KPlane && xx <= kX2N) ? wrapd(x0, xx - 1, n) + wrapd(y0, yy - 1, n) * n : -1;
    }
    float ureg[UPer], kreg[kX2KPer];
    auto load_u = [&](int zp) {
        const size_t zo = (size_t)wrapd(zp, 0, n) * nn;
#pragma unroll
        for (int j = 0; j < UPer; ++j)
            if (u_off[j] >= 0) ureg[j] = uf[zo + u_off[j]];
    };
    auto store_u = [&](int slot) {
#pragma unroll
        for (int j = 0; j < UPer; ++j)
            if (u_off[j] >= 0) us[slot][tid + 256 * j] = ureg[j];
    };
    auto load_k = [&](int zp) {
        const size_t zo = (size_t)wrapd(zp, 0, n) * nn;
#pragma unroll
        for (int j = 0; j < kX2KPer; ++j)
            if (k_off[j] >= 0) kreg[j] = k[zo + k_off[j]];
    };
    auto store_k = [&](int slot) {
#pragma unroll
        for (int j = 0; j < kX2KPer; ++j)
            if (k_off[j] >= 0) ks[slot][tid + 256 * j] = kreg[j];
    };
    const int c0 = 2 * tx;
    // rows dy = -1, 0, 1 of a staged field plane: R[dy + 1] = (lo, hi) with
    // lo = (x - 1, x), hi = (x + 1, x + 2)
    auto read_u = [&](int slot, float2 (&R)[3][2]) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float* row = us[slot] + (ty + d) * kX2PX + c0;
            R[d][0] = *reinterpret_cast<const float2*>(row);
            R[d][1] = *reinterpret_cast<const float2*>(row + 2);
        }
    };
    // element conductivities of a staged plane: Kc[b][a] = (k(x - a, y - b), k(x + 1 - a, y - b))
    auto read_k = [&](int slot, float2 (&Kc)[2][2]) {
#pragma unroll
        for (int bb = 0; bb < 2; ++bb) {
            const float* row = ks[slot] + (ty + 1 - bb) * kX2KX;
            const float2 lo = *reinterpret_cast<const float2*>(row + c0);
            const float hi = row[c0 + 2];
            Kc[bb][1] = lo;
            Kc[bb][0] = make_float2(lo.y, hi);
        }
    };

    float2 Um[3][2], U0[3][2], Up[3][2];   // planes z - 1, z, z + 1
    float2 Km[2][2], K0[2][2];             // element planes z - 1, z
    // prologue: planes z0 - 1 and z0 of the field, element plane z0 - 1
    load_u(z0 - 1 + n);
    load_k(z0 - 1 + n);
    store_u(0);
    store_k(0);
    load_u(z0);
    __syncthreads();
    read_u(0, Um);
    read_k(0, Km);
    store_u(1);
    __syncthreads();
    read_u(1, U0);
    // in flight: field plane z0 + 1, element plane z0
    load_u(z0 + 1);
    load_k(z0);
    Acc<float> acc;
    const int x = x0 + 2 * tx, y = y0 + ty;
    const float2 m12 = make_float2(-1.0f / 12.0f, -1.0f / 12.0f);
    int slot = 0;
    for (int z = z0; z < z1; ++z) {
        // slot was last read two planes ago (before the previous barrier)
        store_u(slot);
        store_k(slot);
        __syncthreads();
        if (z + 1 < z1) {
            load_u(z + 2);
            load_k(z + 1);
        }
        read_u(slot, Up);
        read_k(slot, K0);
        slot ^= 1;
        // K[c][b][a]: element (x - a, y - b, z - c)
        auto Kat = [&](int c, int bb, int a) -> float2 { return c ? Km[bb][a] : K0[bb][a]; };
        auto Uat = [&](int dx, int dy, int dz) -> float2 {
            const float2 (&P)[3][2] = dz < 0 ? Um : (dz > 0 ? Up : U0);
            const float2 lo = P[dy + 1][0], hi = P[dy + 1][1];
            if (dx < 0) return lo;
            if (dx > 0) return hi;
            return make_float2(lo.y, hi.x);
        };
        const float2 uc = Uat(0, 0, 0);
        float2 nd = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                for (int a = 0; a < 2; ++a)
                    nd = __ffma2_rn(Kat(c, bb, a), f2_sub(Uat(1 - 2 * a, 1 - 2 * bb, 1 - 2 * c), uc), nd);
#pragma unroll
        for (int bb = 0; bb < 2; ++bb)
#pragma unroll
            for (int a = 0; a < 2; ++a)
                nd = __ffma2_rn(__fadd2_rn(Kat(0, bb, a), Kat(1, bb, a)), f2_sub(Uat(1 - 2 * a, 1 - 2 * bb, 0), uc), nd);
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int a = 0; a < 2; ++a)
                nd = __ffma2_rn(__fadd2_rn(Kat(c, 0, a), Kat(c, 1, a)), f2_sub(Uat(1 - 2 * a, 0, 1 - 2 * c), uc), nd);
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int bb = 0; bb < 2; ++bb)
                nd = __ffma2_rn(__fadd2_rn(Kat(c, bb, 0), Kat(c, bb, 1)), f2_sub(Uat(0, 1 - 2 * bb, 1 - 2 * c), uc), nd);
        const float2 o = __fmul2_rn(nd, m12);
        const size_t v = (size_t)x + (size_t)y * n + (size_t)z * nn;
        *reinterpret_cast<float2*>(out + (size_t)fi * N + v) = o;
        if (DOT) {
            acc.add_prod(uc.x, o.x);
            acc.add_prod(uc.y, o.y);
        }
        // march: z + 1 becomes z, z becomes z - 1
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            Um[d][0] = U0[d][0];
            Um[d][1] = U0[d][1];
            U0[d][0] = Up[d][0];
            U0[d][1] = Up[d][1];
        }
#pragma unroll
        for (int bb = 0; bb < 2; ++bb) {
            Km[bb][0] = K0[bb][0];
            Km[bb][1] = K0[bb][1];
        }
    }
    if (DOT) {
        __shared__ double res[3];
        Acc<float> sums[3];
        if (fi == 0) sums[0] = acc;
        else if (fi == 1) sums[1] = acc;
        else sums[2] = acc;
        if (grid_reduce<3>(sums, rb, res)) {
            if (is_thread0()) fin(res);
        }
    }
}

// Grid of the z-reuse form: 3 load cases x tiles x m z-chunks.
inline int zr_grid(int n, int m) { return 3 * (n / kX2N) * (n / kX2Y) * m; }

// z-chunks per column of the z-reuse form.  Cost model: the launch runs
// ceil(CTAs / resident slots) waves, each as long as one chunk's planes plus
// about 1.5 planes of prologue; m minimises that over chunks of at least 4
// planes and grids the reduction partials hold.  per_sm = resident CTAs per
// SM of the variant launched; 0 when the form does not apply.  OTM_ZR_M
// overrides (for sweeps).
inline int zr_m(int n, int sm_count, int per_sm, int max_blocks) {
    if (!x2_ok(n)) return 0;
    const long long per_m = 3LL * (n / kX2N) * (n / kX2Y);
    const long long slots = (long long)std::max(per_sm, 1) * sm_count;
    const char* e = getenv("OTM_ZR_M");
    if (e && atoi(e) >= 1 && atoi(e) <= n && per_m * atoi(e) <= max_blocks) return atoi(e);
    int best = 0;
    double best_t = 0.0;
    for (int m = 1; m <= n / 4; ++m) {
        if (per_m * m > max_blocks) break;
        const long long waves = (per_m * m + slots - 1) / slots;
        const double t = (double)waves * ((double)n / m + 1.5);
        if (best == 0 || t < best_t - 1e-9) {
            best = m;
            best_t = t;
        }
    }
    return best;
}
template <bool DOT, class Fin>
inline int zr_m_for(int n, int sm_count, int max_blocks) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stencil_zr<DOT, Fin>, kX2T * kX2Y, 0) != cudaSuccess)
        per_sm = 1;
    return zr_m(n, sm_count, per_sm, max_blocks);
}

}  // namespace otm
