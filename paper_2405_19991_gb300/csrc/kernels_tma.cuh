// TMA-staged form of the finest-grid 21-point stencil (the operator [K u]_v
// of Sec. 2.4 on the three load cases).
//
// A CTA owns TY whole x-rows (all n nodes of each, so the periodic x-halo is
// inside the tile) of a z-chunk of planes.  One producer warp issues tensor
// copies (cp.async.bulk.tensor) of each new z-plane -- the three load cases'
// rows y0-1 .. y0+TY and the element conductivities of rows y0-1 .. y0+TY-1
// -- into a ring of S shared-memory stages, each completed through an
// mbarrier transaction count; the y-wrap of the first and last row blocks is
// two copies (the wrapped row on its own), so no copy leaves the tensor and
// no shared byte is written twice.  The consumer warps release a stage
// through a second mbarrier (one arrival per warp) once they are done with
// it, and the producer refills it; no CTA-wide barrier runs inside the march.
// Every consumer thread computes a node pair (x, x + 1) with x odd, so all
// 8-byte shared loads of (x - 1, x) and (x + 1, x + 2) are aligned and the
// pair (n - 1, 0) needs no special case; the arithmetic runs on packed FP32
// pairs held in 64-bit registers.
//
// The march in z splits each node's difference-form sum by plane: when node
// plane z + 1 and element plane z arrive, the nodes of plane z receive their
// in-plane and upper-plane terms (and are finished), and the nodes of plane
// z + 1 receive their lower-plane terms.  Both planes' rows are read from
// the ring (a stage is released one stage after it arrived), so no plane is
// carried in registers.  All three load cases are done by the same thread,
// so the conductivity pair sums of a plane are formed once.  The order of the
// terms is the plane-by-plane order of nd_sum (kernels_fine.cuh), so this
// form, the tiled form and the gather form give the same bits.
//
// Every wait is bounded (about 0.5 s).  A wait that runs out sets *err and a
// shared flag; every warp leaves its march at its next stage, the producer
// stops issuing, the copies still in flight are drained (again bounded)
// before the CTA ends, and the CTA still takes part in the reduction.
#pragma once
#include <cuda.h>   // CUtensorMap and its enums (types only)

#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <type_traits>

#include "kernels_fine.cuh"
#include "ptx_async.cuh"

namespace otm {

// Two FP32 values held as one 64-bit register pair (lane 0 in the low word)
// and operated on with the packed f32x2 instructions.  Keeping the pair in
// one 64-bit value from load to store avoids the register moves that
// splitting and re-forming float2 values around every packed operation
// costs; each lane performs the plain IEEE operation (round to nearest).
typedef unsigned long long f2p;
__device__ __forceinline__ f2p pk(float a, float b) {
    f2p d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float pk_lo(f2p v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return a;
}
__device__ __forceinline__ float pk_hi(f2p v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return b;
}
// (hi word of lo, lo word of hi): the pair (x, x + 1) from (x - 1, x), (x + 1, x + 2)
__device__ __forceinline__ f2p pk_mid(f2p lo, f2p hi) { return pk(pk_hi(lo), pk_lo(hi)); }
__device__ __forceinline__ f2p pk_add(f2p a, f2p b) {
    f2p d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p pk_sub(f2p a, f2p b) {
    f2p d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p pk_mul(f2p a, f2p b) {
    f2p d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p pk_fma(f2p a, f2p b, f2p c) {
    f2p d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// packed-pair loads from a staged row (element index i even)
__device__ __forceinline__ f2p ld_pk(const float* row, int i) { return *reinterpret_cast<const f2p*>(row + i); }
__device__ __forceinline__ f2p ld_pk(const __nv_bfloat16* row, int i) {
    const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(row + i));
    return pk(v.x, v.y);
}
__device__ __forceinline__ float ld_one(const float* row, int i) { return row[i]; }
__device__ __forceinline__ float ld_one(const __nv_bfloat16* row, int i) { return __bfloat162float(row[i]); }

// Compensated dot accumulator on both lanes of a pair (two independent
// Acc<float> sequences, one per lane: TwoProduct and TwoSum, no fusion).
struct Acc2 {
    f2p s = 0ull, c = 0ull;   // +0.0f in both lanes
    __device__ __forceinline__ void add_prod(f2p a, f2p b) {
        const f2p p = pk_mul(a, b);
        const f2p pe = pk_fma(a, b, pk_sub(0ull, p));
        const f2p t = pk_add(s, p);
        const f2p bp = pk_sub(t, s);
        const f2p e = pk_add(pk_sub(s, pk_sub(t, bp)), pk_sub(p, bp));
        c = pk_add(c, pk_add(e, pe));
        s = t;
    }
    __device__ __forceinline__ Acc<float> merged() const {
        Acc<float> a;
        a.s = pk_lo(s);
        a.c = pk_lo(c);
        ff_add(a.s, a.c, pk_hi(s), pk_hi(c));
        return a;
    }
};

// Checking build: a tensor copy of `rows` rows of `row_bytes` starting at row
// `row` of a `total`-row extent, plane z of n, into shared-memory offset
// `off` of a `cap`-byte ring.  A copy that fails is not issued; its stage
// then never completes and the bounded wait ends the launch with its error
// flag set.
__device__ __forceinline__ bool tma_box_ok(long long off, int rows, int row_bytes, long long cap, int row, int total,
                                           int z, int n, int site) {
    return OTM_BOUND(off + (long long)rows * row_bytes - 1, cap, site) && OTM_BOUND(row, total - rows + 1, site) &&
           OTM_BOUND(z, n, site);
}

// ------------------------------------------------------------------ kernel
constexpr int kTmaMaxStages = 8;   // ring depth: 3 .. 8 stages (a launch argument)
constexpr int kTmaThreads = 256;

// Tensor maps of one stencil launch.  u: the three load cases' field,
// [3][n][n][n] (x fastest), boxes of n x rows x 1 x 1 with rows = TY + 2
// (interior row block), TY + 1 (first or last row block) and 1 (the wrapped
// row).  k: the element conductivities [n][n][n], boxes n x (TY + 1), n x TY
// and n x 1.  f (right-hand side of the residual form): [3][n][n][n], boxes
// n x TY.
struct TmaStencilMaps {
    CUtensorMap u_full, u_lo, u_row;
    CUtensorMap k_full, k_lo, k_row;
    CUtensorMap f_rows;
};

// Bytes of one ring stage.
__host__ __device__ inline int tma_stage_bytes(int mode, int n, int ty, int st_size, int ft_size) {
    return 3 * (ty + 2) * n * st_size + (ty + 1) * n * st_size + (mode == 1 ? 3 * ty * n * ft_size : 0);
}

// MODE 0: out_i = K(k) u_i (with DOT: reduces u_i . out_i, i = 0..2).
// MODE 1: out_i = f_i - K(k) u_i (with DOT: reduces out_i . out_i and
// f_i . f_i, i = 0..2, in that order).
// ST: storage of k and u (FP32 or BF16); FT: f; OT: out.  Grid: (n / TY)
// row blocks (fastest) x m z-chunks; block: (n / 2) TY threads.
// Rows per CTA for n known at compile time (the rule of tma_rows below).
__host__ __device__ constexpr int tma_rows_c(int n) {
    int t = n / 2 < 2 * kTmaThreads / n ? n / 2 : 2 * kTmaThreads / n;
    for (; t >= 1; --t)
        if (n % t == 0 && (n / 2) * t <= kTmaThreads && ((n / 2) * t) % 32 == 0 && n / t >= 2) return t;
    return 0;
}

// NC: n at compile time (all shared-memory and plane offsets become
// immediates), or 0 for any n given at run time.
template <int NC, int MODE, bool DOT, class ST, class FT, class OT, class Fin>
__global__ void __maxnreg__(96)
k_stencil_tma(const __grid_constant__ TmaStencilMaps mp, int n_rt, int ty_rt, int m, int S, OT* __restrict__ out, int* err,
              RedBuf rb, Fin fin, int early) {
    extern __shared__ unsigned char tsm_raw[];
    __shared__ __align__(8) uint64_t full[kTmaMaxStages];    // stage landed (transaction count)
    __shared__ __align__(8) uint64_t empty[kTmaMaxStages];   // every consumer warp done with the stage
    __shared__ int bail_s;                                // a bounded wait ran out somewhere
    const int n = NC ? NC : n_rt;
    const int TY = NC ? tma_rows_c(NC) : ty_rt;
    unsigned char* tsm = tsm_raw + ((128u - (smem_u32(tsm_raw) & 127u)) & 127u);
    const int NP = n >> 1;
    const int tid = threadIdx.x;
    const int px = tid % NP, ty = tid / NP;
    const int nyb = n / TY;
    const int yb = blockIdx.x % nyb, zc = blockIdx.x / nyb;
    const int y0 = yb * TY;
    const int z0 = zc * n / m, z1 = (zc + 1) * n / m;
    const int nst = z1 - z0 + 2;
    const int rowU = n * (int)sizeof(ST), rowF = n * (int)sizeof(FT);
    const int uBytes = 3 * (TY + 2) * rowU, kBytes = (TY + 1) * rowU;
    const int stageBytes = tma_stage_bytes(MODE, n, TY, (int)sizeof(ST), (int)sizeof(FT));
    const int N = n * n * n;

    auto wrapz = [n](int z) { return z < 0 ? z + n : (z >= n ? z - n : z); };
    // stage j: node plane z0 - 1 + j, element plane (and f plane) z0 - 2 + j
    // parts & 1: the stage's transaction count and the copies of k (and f);
    // parts & 2: the copies of u
    auto issue = [&](int j, int parts) {
        const int slot = j % S;
        unsigned char* st = tsm + slot * stageBytes;
        uint64_t* bar = &full[slot];
        const int zn = wrapz(z0 - 1 + j), ze = wrapz(z0 - 2 + j);
        const long long cap = (long long)S * stageBytes;
        auto ok = [&](const unsigned char* d, int rows, int rb, int row, int z) {
            return tma_box_ok(d - tsm, rows, rb, cap, row, n, z, n, kSiteTmaStencil);
        };
        if (parts & 1) {
            mbar_expect_tx(bar, (uint32_t)stageBytes);
            unsigned char* dk = st + uBytes;
            if (y0 == 0) {
                if (ok(dk + rowU, TY, rowU, 0, ze)) tma_load_3d(dk + rowU, &mp.k_lo, bar, 0, 0, ze);
                if (ok(dk, 1, rowU, n - 1, ze)) tma_load_3d(dk, &mp.k_row, bar, 0, n - 1, ze);
            } else {
                if (ok(dk, TY + 1, rowU, y0 - 1, ze)) tma_load_3d(dk, &mp.k_full, bar, 0, y0 - 1, ze);
            }
            if (MODE == 1) {
                unsigned char* df = st + uBytes + kBytes;
#pragma unroll 1
                for (int c = 0; c < 3; ++c)
                    if (ok(df + c * TY * rowF, TY, rowF, y0, ze))
                        tma_load_4d(df + c * TY * rowF, &mp.f_rows, bar, 0, y0, ze, c);
            }
        }
        if (!(parts & 2)) return;
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {
            unsigned char* d = st + c * (TY + 2) * rowU;
            if (y0 == 0) {
                if (ok(d + rowU, TY + 1, rowU, 0, zn)) tma_load_4d(d + rowU, &mp.u_lo, bar, 0, 0, zn, c);
                if (ok(d, 1, rowU, n - 1, zn)) tma_load_4d(d, &mp.u_row, bar, 0, n - 1, zn, c);
            } else if (y0 + TY == n) {
                if (ok(d, TY + 1, rowU, y0 - 1, zn)) tma_load_4d(d, &mp.u_lo, bar, 0, y0 - 1, zn, c);
                if (ok(d + (TY + 1) * rowU, 1, rowU, 0, zn))
                    tma_load_4d(d + (TY + 1) * rowU, &mp.u_row, bar, 0, 0, zn, c);
            } else {
                if (ok(d, TY + 2, rowU, y0 - 1, zn)) tma_load_4d(d, &mp.u_full, bar, 0, y0 - 1, zn, c);
            }
        }
    };

    // warps 0 .. C-1 compute (C = (n / 2) TY / 32); warp C only issues copies
    const int ncons = NP * TY;
    if (tid == 0) {
        bail_s = 0;
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], ncons / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    // the consumers' partial sums (zero in the producer warp): MODE 0 p . Kp
    // of the pair's two nodes on the two lanes; MODE 1 r . r on the low lane
    // and f . f on the high lane, the pair's nodes one after the other
    Acc2 acc[3];
    int issued = 0;
    if (tid >= ncons) {
        // Producer: stage i goes into slot i mod S once every consumer warp is
        // done with stage i - S (they release a slot one stage after they
        // first read it, since a stage also reads the slot before it).
        // With `early` (k and f written two or more kernels back) the first
        // stages' k and f copies go out before griddepcontrol.wait; u,
        // which the previous kernel may still be writing, follows it.
        if (tid == ncons) {
            const int pre = early ? (nst < S ? nst : S) : 0;
            for (int i = 0; i < pre; ++i) issue(i, 1);
            pdl_enter();
            bool okp = true;
            for (int i = 0; i < nst && okp; ++i) {
                if (i >= S) {
                    okp = mbar_wait_bounded(&empty[i % S], (uint32_t)(((i - S) / S) & 1)) &&
                          !*(volatile int*)&bail_s;
                    if (!okp) break;
                }
                issue(i, i < pre ? 2 : 3);
                issued = i + 1;
            }
            if (!okp) {
                if (err) *err = 1;
                *(volatile int*)&bail_s = 1;
            }
        } else {
            pdl_enter();
        }
    } else {
    pdl_enter();

    const int xo = 2 * px;                          // index of (x - 1, x), x = 2 px + 1
    const int xh = xo + 2 == n ? 0 : xo + 2;        // index of (x + 1, x + 2)
    const int xa = xo + 1, xb = xh;                 // the pair's own nodes x, x + 1
    const int y = y0 + ty;
    const f2p m12 = pk(-1.0f / 12.0f, -1.0f / 12.0f);
    // per-thread element offsets, fixed for the whole march
    const int su = ty * n;                          // staged u, case 0, row dy = -1
    const int scs = (TY + 2) * n;                   // staged u, case stride
    const int sk1 = ty * n, sk0 = (ty + 1) * n;     // staged k, rows y - 1 (b = 1) and y (b = 0)
    const int sf = ty * n;                          // staged f, case 0
    const int nn = n * n;
    const int oa = y * n + xa, ob = y * n + xb;     // output offsets in a plane
    // checking build: the furthest staged element this thread reads (case 2,
    // row y + 1, x + 2) and the furthest k and f elements; a failure ends
    // the march through the bail flag
    if (!(OTM_BOUND(su + 2 * scs + 2 * n + xh + 1, 3 * (TY + 2) * n, kSiteTmaStencil) &&
          OTM_BOUND(sk0 + xh, (TY + 1) * n, kSiteTmaStencil) &&
          OTM_BOUND(sf + 2 * TY * n + (xa > xb ? xa : xb), MODE == 1 ? 3 * TY * n : 2147483647, kSiteTmaStencil) &&
          OTM_BOUND(oa > ob ? oa : ob, n * n, kSiteTmaStencil)))
        *(volatile int*)&bail_s = 1;

    f2p A[3];               // lower-plane partial sums of node plane zj - 1

    // Stage j: node plane zj and element plane zj - 1 arrive in slot j; node
    // plane zj - 1 is still in slot j - 1 (a slot is refilled only once the
    // stage after it is done), so both planes' rows are read from shared
    // memory and no plane is carried in registers.  Rows are held as
    // R[dy + 1] = {(x - 1, x), (x + 1, x + 2)}.  The terms whose neighbour
    // lies in the node's own x column (y-z edge diagonals) are summed lane
    // by lane in scalar FP32, the others on packed pairs: each lane performs
    // the same operations in the same order either way.  FIN / START select
    // the stage's role at compile time (stage 0 only loads, stage 1 only
    // starts, the last stage only finishes); Kp / Kn (element planes zj - 2,
    // zj - 1) swap roles between calls instead of being copied.
    int j = 0, slot = 0, pslot = S - 1, zf = wrapz(z0 - 2);
    uint32_t phase = 0;
    auto stage = [&](auto fin_c, auto start_c, const f2p (&Kp)[2][2], f2p (&Kn)[2][2]) -> bool {
        constexpr bool FIN = decltype(fin_c)::value, START = decltype(start_c)::value;
        // the decision to leave is taken per warp (every lane agrees), so no
        // lane is left waiting in a later warp-level barrier
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&full[slot], phase) &&
                                                   !*(volatile int*)&bail_s);
        if (!ok) {
            if ((tid & 31) == 0) {
                if (err) *err = 1;
                *(volatile int*)&bail_s = 1;
            }
            return false;
        }
        const unsigned char* st = tsm + slot * stageBytes;
        const ST* U = reinterpret_cast<const ST*>(st) + su;
        const ST* Uo = reinterpret_cast<const ST*>(tsm + pslot * stageBytes) + su;
        const ST* Ks = reinterpret_cast<const ST*>(st + uBytes);
#pragma unroll
        for (int bb = 0; bb < 2; ++bb) {
            const ST* row = Ks + (bb ? sk1 : sk0);
            const f2p lo = ld_pk(row, xo);
            Kn[bb][1] = lo;
            Kn[bb][0] = pk(pk_hi(lo), ld_one(row, xh));
        }
        f2p Pb[2], Pa[2], Pc[2][2];
#pragma unroll
        for (int a = 0; a < 2; ++a) Pb[a] = pk_add(Kn[0][a], Kn[1][a]);
#pragma unroll
        for (int bb = 0; bb < 2; ++bb) Pa[bb] = pk_add(Kn[bb][0], Kn[bb][1]);
        if (FIN) {
#pragma unroll
            for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                for (int a = 0; a < 2; ++a) Pc[bb][a] = pk_add(Kn[bb][a], Kp[bb][a]);
        }
        const int pz = zf * nn;   // the finished node plane
        // y-z edge-diagonal term on both lanes: lane 0 (node x) takes the
        // high word of row lo, lane 1 (node x + 1) the low word of row hi
        auto yz = [](f2p nd, f2p P, f2p lo, f2p hi, f2p uc) -> f2p {
            const float d0 = pk_hi(lo) - pk_lo(uc), d1 = pk_lo(hi) - pk_hi(uc);
            return pk(fmaf(pk_lo(P), d0, pk_lo(nd)), fmaf(pk_hi(P), d1, pk_hi(nd)));
        };
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            __syncwarp();
            f2p Un[3][2], Up[3][2];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int o = c * scs + d * n;
                Un[d][0] = ld_pk(U + o, xo);
                Un[d][1] = ld_pk(U + o, xh);
                if (FIN || START) {
                    Up[d][0] = ld_pk(Uo + o, xo);
                    Up[d][1] = ld_pk(Uo + o, xh);
                }
            }
            if (FIN) {
                const f2p uc = pk_mid(Up[1][0], Up[1][1]);
                f2p nd = A[c];
                // in-plane terms (edge diagonals in x-y, both element planes)
#pragma unroll
                for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                    for (int a = 0; a < 2; ++a)
                        nd = pk_fma(Pc[bb][a], pk_sub(Up[2 - 2 * bb][a ? 0 : 1], uc), nd);
                // upper plane: body diagonals, x-z and y-z edge diagonals
#pragma unroll
                for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                    for (int a = 0; a < 2; ++a)
                        nd = pk_fma(Kn[bb][a], pk_sub(Un[2 - 2 * bb][a ? 0 : 1], uc), nd);
#pragma unroll
                for (int a = 0; a < 2; ++a) nd = pk_fma(Pb[a], pk_sub(Un[1][a ? 0 : 1], uc), nd);
#pragma unroll
                for (int bb = 0; bb < 2; ++bb) nd = yz(nd, Pa[bb], Un[2 - 2 * bb][0], Un[2 - 2 * bb][1], uc);
                OT* o_c = out + (size_t)c * N + pz;
                if (MODE == 0) {
                    const f2p o = pk_mul(nd, m12);
                    St<OT>::st(o_c, oa, pk_lo(o));
                    St<OT>::st(o_c, ob, pk_hi(o));
                    if (DOT) acc[c].add_prod(uc, o);
                } else {
                    const FT* F = reinterpret_cast<const FT*>(st + uBytes + kBytes) + sf + c * TY * n;
                    const float fx = ld_one(F, xa), fy = ld_one(F, xb);
                    const float kx = pk_lo(nd) * (-1.0f / 12.0f), ky = pk_hi(nd) * (-1.0f / 12.0f);
                    const float rx = fx - kx, ry = fy - ky;
                    St<OT>::st(o_c, oa, rx);
                    St<OT>::st(o_c, ob, ry);
                    if constexpr (DOT) {
                        acc[c].add_prod(pk(rx, fx), pk(rx, fx));
                        acc[c].add_prod(pk(ry, fy), pk(ry, fy));
                    }
                }
            }
            if (START) {
                const f2p uc = pk_mid(Un[1][0], Un[1][1]);
                f2p nd = 0ull;
                // lower plane: body diagonals, x-z and y-z edge diagonals
#pragma unroll
                for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                    for (int a = 0; a < 2; ++a)
                        nd = pk_fma(Kn[bb][a], pk_sub(Up[2 - 2 * bb][a ? 0 : 1], uc), nd);
#pragma unroll
                for (int a = 0; a < 2; ++a) nd = pk_fma(Pb[a], pk_sub(Up[1][a ? 0 : 1], uc), nd);
#pragma unroll
                for (int bb = 0; bb < 2; ++bb) nd = yz(nd, Pa[bb], Up[2 - 2 * bb][0], Up[2 - 2 * bb][1], uc);
                A[c] = nd;
            }
        }
        // this warp is done with slot j - 1 (the producer refills it once
        // every consumer warp is)
        if (j >= 1) {
            __syncwarp();
            if ((tid & 31) == 0) mbar_arrive(&empty[pslot]);
        }
        ++j;
        pslot = slot;
        if (++slot == S) {
            slot = 0;
            phase ^= 1u;
        }
        zf = zf + 1 == n ? 0 : zf + 1;
        return true;
    };
    using T_ = std::true_type;
    using F_ = std::false_type;
    f2p KA[2][2], KB[2][2];
    bool bail = !stage(F_{}, F_{}, KB, KA) || !stage(F_{}, T_{}, KA, KB);
    // steady stages 2 .. nst - 2, two per trip (the element planes swap roles)
#pragma unroll 1
    while (!bail && j + 2 <= nst - 1) {
        if (!stage(T_{}, T_{}, KB, KA) || !stage(T_{}, T_{}, KA, KB)) bail = true;
    }
    if (!bail && j < nst - 1 && !stage(T_{}, T_{}, KB, KA)) bail = true;
    // last stage: stage i writes its element plane into KA for even i, KB
    // for odd i, so stage nst - 2 left it in KA when nst is even
    if (!bail) {
        if ((nst & 1) == 0) {
            if (!stage(T_{}, F_{}, KA, KB)) bail = true;
        } else {
            if (!stage(T_{}, F_{}, KB, KA)) bail = true;
        }
    }
    (void)bail;
    }
    // After a wait ran out, the copies still in flight land before the
    // shared memory goes away (on the normal path the consumers have waited
    // for every stage).
    __syncthreads();
    if (tid == ncons && *(volatile int*)&bail_s)
        for (int i = issued > S ? issued - S : 0; i < issued; ++i)
            (void)mbar_wait_bounded(&full[i % S], (uint32_t)((i / S) & 1));
    if constexpr (DOT && MODE == 0) {
        __shared__ double res[3];
        Acc<float> sums[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) sums[c] = acc[c].merged();
        if (grid_reduce<3>(sums, rb, res)) {
            if (is_thread0()) fin(res);
        }
    } else if constexpr (DOT) {
        __shared__ double res[6];
        Acc<float> sums[6];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sums[c].s = pk_lo(acc[c].s);
            sums[c].c = pk_lo(acc[c].c);
            sums[3 + c].s = pk_hi(acc[c].s);
            sums[3 + c].c = pk_hi(acc[c].c);
        }
        if (grid_reduce<6>(sums, rb, res)) {
            if (is_thread0()) fin(res);
        }
    }
}

// ---------------------------------------------------------------- host side
// Fine-grid stencil form: 0 TMA-staged (where it applies), 1 shared-memory
// tiled, 2 gather (OTM_STENCIL=tma|tiled|gather; default tma), for
// comparisons.  All three sum the same terms in the same order.
inline int stencil_choice() {
    static int c = [] {
        const char* e = getenv("OTM_STENCIL");
        if (!e) return 0;
        if (e[0] == 't' && e[1] == 'i') return 1;
        if (e[0] == 'g') return 2;
        return 0;
    }();
    return c;
}

// 1: the solver's TMA kernels issue their k and f copies before waiting on
// the previous kernel (OTM_PDL_EARLY=0 turns it off, for comparisons).
inline int pdl_early() {
    static int v = [] {
        const char* e = getenv("OTM_PDL_EARLY");
        return e && e[0] == '0' ? 0 : 1;
    }();
    return v;
}

typedef CUresult (*TmaEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline TmaEncodeFn tma_encoder() {
    static TmaEncodeFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (TmaEncodeFn) nullptr;
        return (TmaEncodeFn)p;
    }();
    return fn;
}

template <class T> struct TmaType;
template <> struct TmaType<float> {
    static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
};
template <> struct TmaType<__nv_bfloat16> {
    static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
};

// Rows per CTA: the largest divisor TY of n with (n / 2) TY <= 256 threads,
// a whole number of warps and at least two row blocks; 0 when none.
inline int tma_rows(int n) {
    for (int ty = std::min(n / 2, 2 * kTmaThreads / std::max(n, 1)); ty >= 1; --ty)
        if (n % ty == 0 && (n / 2) * ty <= kTmaThreads && ((n / 2) * ty) % 32 == 0 && n / ty >= 2) return ty;
    return 0;
}

// The form applies when every staged row is a multiple of 128 bytes (the
// shared-memory alignment of a tensor copy) and fits one box (<= 256).
inline bool tma_stencil_ok(int n, int st_size, int ft_size) {
    if (n < 32 || n > 256 || n % 2) return false;
    if ((n * st_size) % 128 || (n * ft_size) % 128) return false;
    if ((long long)n * n * n * 3 >= (1LL << 31)) return false;
    return tma_rows(n) > 0 && tma_encoder() != nullptr;
}

// Ring depth (OTM_TMA_STAGES overrides, 3..8): a stage reads its own slot
// and the one before, so depth S keeps S - 2 stages in flight ahead.
inline int tma_stages() {
    static int s = [] {
        const char* e = getenv("OTM_TMA_STAGES");
        const int v = e ? atoi(e) : 0;
        return v >= 3 && v <= kTmaMaxStages ? v : 4;
    }();
    return s;
}
inline size_t tma_smem_bytes(int mode, int n, int st_size, int ft_size) {
    return (size_t)tma_stages() * tma_stage_bytes(mode, n, tma_rows(n), st_size, ft_size) + 128;
}

// z-chunks: minimise (waves) x (stages per chunk) over chunks of at least 2
// planes, within the reduction partials' capacity.  OTM_TMA_M overrides.
inline int tma_m(int n, int sm_count, int per_sm, int max_blocks) {
    const int ty = tma_rows(n);
    if (ty == 0) return 0;
    const long long per_m = n / ty;
    const char* e = getenv("OTM_TMA_M");
    if (e && atoi(e) >= 1 && atoi(e) <= n && per_m * atoi(e) <= max_blocks) return atoi(e);
    const long long slots = (long long)std::max(per_sm, 1) * sm_count;
    int best = 0;
    double best_t = 0.0;
    for (int m = 1; m <= n / 2; ++m) {
        if (per_m * m > max_blocks) break;
        const long long waves = (per_m * m + slots - 1) / slots;
        const double t = (double)waves * ((double)n / m + 2.0);
        if (best == 0 || t < best_t - 1e-9) {
            best = m;
            best_t = t;
        }
    }
    return best;
}

// Encodes the maps of one launch; false when the encoder refuses a map.
template <class ST, class FT>
inline bool tma_make_maps(TmaStencilMaps& mp, int n, const void* k, const void* u, const void* f) {
    TmaEncodeFn enc = tma_encoder();
    if (!enc) return false;
    const int ty = tma_rows(n);
    memset(&mp, 0, sizeof(mp));
    const cuuint32_t es[4] = {1, 1, 1, 1};
    auto map4 = [&](CUtensorMap* m, const void* base, size_t esz, CUtensorMapDataType dt, int rows) {
        const cuuint64_t dims[4] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)n, 3};
        const cuuint64_t str[3] = {(cuuint64_t)n * esz, (cuuint64_t)n * n * esz, (cuuint64_t)n * n * n * esz};
        const cuuint32_t box[4] = {(cuuint32_t)n, (cuuint32_t)rows, 1, 1};
        return enc(m, dt, 4, const_cast<void*>(base), dims, str, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    auto map3 = [&](CUtensorMap* m, const void* base, size_t esz, CUtensorMapDataType dt, int rows) {
        const cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)n};
        const cuuint64_t str[2] = {(cuuint64_t)n * esz, (cuuint64_t)n * n * esz};
        const cuuint32_t box[3] = {(cuuint32_t)n, (cuuint32_t)rows, 1};
        return enc(m, dt, 3, const_cast<void*>(base), dims, str, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    const auto dts = TmaType<ST>::v;
    bool ok = map4(&mp.u_full, u, sizeof(ST), dts, ty + 2) && map4(&mp.u_lo, u, sizeof(ST), dts, ty + 1) &&
              map4(&mp.u_row, u, sizeof(ST), dts, 1) && map3(&mp.k_full, k, sizeof(ST), dts, ty + 1) &&
              map3(&mp.k_lo, k, sizeof(ST), dts, ty) && map3(&mp.k_row, k, sizeof(ST), dts, 1);
    if (ok && f) ok = map4(&mp.f_rows, f, sizeof(FT), TmaType<FT>::v, ty);
    return ok;
}

// Launch shape of the TMA form for one instantiation on this device:
// dynamic shared memory opted in once per device, resident CTAs per SM from
// the occupancy API, z-chunks from the wave model.
struct TmaLaunch {
    int n = 0, ty = 0, m = 0, grid = 0, threads = 0, stages = 0;
    size_t smem = 0;
};
// The instantiation for this n: compile-time n for the common sizes, the
// run-time form otherwise.  This and tma_launch_shape are static: every
// translation unit that launches the kernel registers its own stub of each
// instantiation, and the shared-memory opt-in belongs to the stub, so the
// opt-in and the launch must take the stub of the same unit.
template <int MODE, bool DOT, class ST, class FT, class OT, class Fin>
using TmaKernel = void (*)(TmaStencilMaps, int, int, int, int, OT*, int*, RedBuf, Fin, int);
template <int MODE, bool DOT, class ST, class FT, class OT, class Fin>
static TmaKernel<MODE, DOT, ST, FT, OT, Fin> tma_kernel(int n) {
    if (n == 64) return k_stencil_tma<64, MODE, DOT, ST, FT, OT, Fin>;
    if (n == 128) return k_stencil_tma<128, MODE, DOT, ST, FT, OT, Fin>;
    if (n == 256) return k_stencil_tma<256, MODE, DOT, ST, FT, OT, Fin>;
    return k_stencil_tma<0, MODE, DOT, ST, FT, OT, Fin>;
}

template <int MODE, bool DOT, class ST, class FT, class OT, class Fin>
static bool tma_launch_shape(TmaLaunch& L, int n, int sm_count, int max_blocks) {
    if (!tma_stencil_ok(n, (int)sizeof(ST), (int)sizeof(FT))) return false;
    auto kern = tma_kernel<MODE, DOT, ST, FT, OT, Fin>(n);
    L.n = n;
    L.ty = tma_rows(n);
    L.threads = (n / 2) * L.ty + 32;   // consumer warps + the producer warp
    L.smem = tma_smem_bytes(MODE, n, (int)sizeof(ST), (int)sizeof(FT));
    L.stages = tma_stages();
    {
        // one opt-in per kernel and device, only ever raised
        static std::mutex mu;
        static size_t granted[4][64] = {};
        std::lock_guard<std::mutex> lock(mu);
        int dev = 0;
        cudaGetDevice(&dev);
        const int d = dev >= 0 && dev < 64 ? dev : 0;
        const int ki = n == 64 ? 1 : n == 128 ? 2 : n == 256 ? 3 : 0;
        if (L.smem > granted[ki][d]) {
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem) != cudaSuccess)
                return false;
            // OTM_TMA_CARVEOUT=p: prefer p % of the unified L1 / shared array as
            // shared memory (default: the CUDA runtime's choice)
            if (const char* cv = getenv("OTM_TMA_CARVEOUT"))
                cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, atoi(cv));
            granted[ki][d] = L.smem;
        }
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, L.threads, L.smem) != cudaSuccess || per_sm < 1)
        return false;
    L.m = tma_m(n, sm_count, per_sm, max_blocks);
    if (L.m < 1) return false;
    L.grid = (n / L.ty) * L.m;
    return true;
}

}  // namespace otm
