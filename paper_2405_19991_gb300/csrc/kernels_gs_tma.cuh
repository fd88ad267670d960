// TMA-staged form of the finest-grid Gauss-Seidel group pass (the smoother
// of Sec. 2.4 on the three load cases; a group is the nodes with one
// (y mod 2, z mod 2) parity, which no stencil term joins, so the group's
// nodes are relaxed at once from the values of the other groups).
//
// A CTA owns TY output rows y = y0 + yo + 2t (t < TY) of a run of output
// planes z = zo + 2p, all n nodes of each row.  The march in z visits node
// plane zb - 1 + j and element plane zb - 1 + j in stage j (zb: the first
// output plane), so output plane p reads stages 2p (plane z - 1), 2p + 1
// (plane z, with the right-hand side f) and 2p + 2 (plane z + 1), and stage
// 2p + 2 serves the next output plane too.  A stage holds
//   - the element rows y - 1 and y of every output row (2 TY rows),
//   - for a plane of the other z parity (even j): node rows y0 + yo - 1 ..
//     y0 + yo + 2 TY - 1 of the three load cases (2 TY + 1 rows),
//   - for an own-parity plane (odd j): only the node rows of the other y
//     parity (TY + 1 rows), read through a view of the field that splits y
//     into (y / 2, y mod 2), and the f rows of the output rows (TY rows).
// The group's own nodes in its own planes are never loaded: the pass reads
// exactly the other groups' values, each once.  Copies that would cross
// the periodic y boundary are split in two, as in the TMA stencil.
//
// One producer warp issues the copies into a ring of S stages; the consumer
// warps release the two stages below an output plane (one arrival per warp)
// once they have finished it.  Each consumer thread relaxes the node pair
// (x, x + 1) with x odd, so all 8-byte shared loads are aligned.  Each
// node's sum is taken in the order of nb_from (kernels_fine.cuh) on packed
// FP32 pairs, and the update is the same expression as in k_gs_fine, so the
// two forms give the same bits.  Waits are bounded as in the TMA stencil.
#pragma once
#include "kernels_tma.cuh"

namespace otm {

// Tensor maps of one group-pass launch.  T: [3][n][n][n] rows (x fastest),
// boxes n x (2TY + 1), n x 2TY and n x 1; Tp: the same field as
// (x, y mod 2, y / 2, z, case), boxes n x 1 x (TY + 1), n x 1 x TY and
// n x 1 x 1; k: [n][n][n], boxes n x 2TY, n x (2TY - 1) and n x 1; fp: f as
// (x, y mod 2, y / 2, z, case), box n x 1 x TY.
struct TmaGsMaps {
    CUtensorMap t_full, t_lo, t_row;
    CUtensorMap tp_full, tp_lo, tp_row;
    CUtensorMap k_full, k_lo, k_row;
    CUtensorMap fp_rows;
};

// Byte offsets inside one stage: element rows first, then the node rows
// (case stride (2TY + 1) rows in an even stage, (TY + 1) rows in an odd
// one), then, in an odd stage only, the f rows (case stride TY rows).
__host__ __device__ inline int gs_tma_k_bytes(int n, int ty, int st) { return 2 * ty * n * st; }
__host__ __device__ inline int gs_tma_even_bytes(int n, int ty, int st) {
    return gs_tma_k_bytes(n, ty, st) + 3 * (2 * ty + 1) * n * st;
}
__host__ __device__ inline int gs_tma_odd_bytes(int n, int ty, int st, int ft) {
    return gs_tma_k_bytes(n, ty, st) + 3 * (ty + 1) * n * st + 3 * ty * n * ft;
}
__host__ __device__ inline int gs_tma_stage_bytes(int n, int ty, int st, int ft) {
    const int e = gs_tma_even_bytes(n, ty, st), o = gs_tma_odd_bytes(n, ty, st, ft);
    return e > o ? e : o;
}

// Output rows per CTA: the largest TY with 2 TY | n, (n / 2) TY <= 256
// threads in whole warps, and at least two row blocks; at most 2 from
// n = 128 on (128^3 design iteration: 2.326 ms FP32 with two rows against
// 2.338 with four, 2.294 against 2.299 mixed -- more, smaller CTAs hide the
// ring's fill latency better).
__host__ __device__ constexpr int gs_tma_rows_c(int n) {
    for (int t = n >= 128 ? 2 : n / 4; t >= 1; --t)
        if (n % (2 * t) == 0 && (n / 2) * t <= kTmaThreads && ((n / 2) * t) % 32 == 0 && n / (2 * t) >= 2) return t;
    return 0;
}

// One group pass T <- (12 f + nb(T)) / (4 sum k) on the group (yo, zo) =
// (group & 1, group >> 1).  ST: storage of k and T; FT: f.  Grid: (n / 2TY)
// row blocks (fastest) x m runs of output planes; block: (n / 2) TY
// consumer threads + one producer warp.
template <int NC, class ST, class FT>
__global__ void __maxnreg__(96)
k_gs_tma(const __grid_constant__ TmaGsMaps mp, int n_rt, int ty_rt, int m, int S, int group, ST* __restrict__ T,
         int* err, int early) {
    extern __shared__ unsigned char gsm_raw[];
    __shared__ __align__(8) uint64_t full[kTmaMaxStages];    // stage landed (transaction count)
    __shared__ __align__(8) uint64_t empty[kTmaMaxStages];   // every consumer warp done with the stage
    __shared__ int bail_s;                                // a bounded wait ran out somewhere
    const int n = NC ? NC : n_rt;
    const int TY = NC ? gs_tma_rows_c(NC) : ty_rt;
    unsigned char* tsm = gsm_raw + ((128u - (smem_u32(gsm_raw) & 127u)) & 127u);
    const int NP = n >> 1, P = n >> 1;   // node pairs per row, output planes per group
    const int tid = threadIdx.x;
    const int px = tid % NP, t = tid / NP;
    const int nrb = n / (2 * TY);
    const int yb = blockIdx.x % nrb, zc = blockIdx.x / nrb;
    const int yo = group & 1, zo = group >> 1;
    const int y0 = yb * 2 * TY;
    const int p0 = zc * P / m, p1 = (zc + 1) * P / m;
    const int cnt = p1 - p0;
    const int nst = 2 * cnt + 1;
    const int zb = zo + 2 * p0;                  // first output plane
    const int rowU = n * (int)sizeof(ST), rowF = n * (int)sizeof(FT);
    const int kB = gs_tma_k_bytes(n, TY, (int)sizeof(ST));
    const int stageBytes = gs_tma_stage_bytes(n, TY, (int)sizeof(ST), (int)sizeof(FT));
    const int r0 = y0 + yo - 1;                  // first staged node and element row
    const int h0 = yb * TY - 1 + yo;             // first staged row of the other y parity, as y / 2
    const int q = 1 - yo;                        // that parity
    const int N = n * n * n;

    auto wrapz = [n](int z) { return z < 0 ? z + n : (z >= n ? z - n : z); };
    // parts & 1: the stage's transaction count and the copies of k and f;
    // parts & 2: the copies of T
    auto issue = [&](int j, int parts) {
        const int slot = j % S;
        unsigned char* st = tsm + slot * stageBytes;
        uint64_t* bar = &full[slot];
        const int zp = wrapz(zb - 1 + j);
        const bool odd = (j & 1) != 0, with_k = j < nst - 1;   // the last stage's elements are not used
        unsigned char* d0 = st + kB;
        // checking build: each copy's rows inside its extent (n rows, or P
        // rows of one parity) and its bytes inside the ring
        const long long cap = (long long)S * stageBytes;
        auto ok = [&](const unsigned char* d, int rows, int rb, int row, int total) {
            return tma_box_ok(d - tsm, rows, rb, cap, row, total, zp, n, kSiteTmaGs);
        };
        if (parts & 1) {
            const int bytes =
                (odd ? 3 * (TY + 1) * rowU + 3 * TY * rowF : 3 * (2 * TY + 1) * rowU) + (with_k ? kB : 0);
            mbar_expect_tx(bar, (uint32_t)bytes);
            if (with_k) {
                if (r0 < 0) {
                    if (ok(st, 1, rowU, n - 1, n)) tma_load_3d(st, &mp.k_row, bar, 0, n - 1, zp);
                    if (ok(st + rowU, 2 * TY - 1, rowU, 0, n)) tma_load_3d(st + rowU, &mp.k_lo, bar, 0, 0, zp);
                } else {
                    if (ok(st, 2 * TY, rowU, r0, n)) tma_load_3d(st, &mp.k_full, bar, 0, r0, zp);
                }
            }
            if (odd) {
                unsigned char* df = d0 + 3 * (TY + 1) * rowU;
#pragma unroll 1
                for (int c = 0; c < 3; ++c)
                    if (ok(df + c * TY * rowF, TY, rowF, yb * TY, P))
                        tma_load_5d(df + c * TY * rowF, &mp.fp_rows, bar, 0, yo, yb * TY, zp, c);
            }
        }
        if (!(parts & 2)) return;
        if (!odd) {
#pragma unroll 1
            for (int c = 0; c < 3; ++c) {
                unsigned char* d = d0 + c * (2 * TY + 1) * rowU;
                if (r0 < 0) {
                    if (ok(d, 1, rowU, n - 1, n)) tma_load_4d(d, &mp.t_row, bar, 0, n - 1, zp, c);
                    if (ok(d + rowU, 2 * TY, rowU, 0, n)) tma_load_4d(d + rowU, &mp.t_lo, bar, 0, 0, zp, c);
                } else if (r0 + 2 * TY + 1 > n) {
                    if (ok(d, 2 * TY, rowU, r0, n)) tma_load_4d(d, &mp.t_lo, bar, 0, r0, zp, c);
                    if (ok(d + 2 * TY * rowU, 1, rowU, 0, n))
                        tma_load_4d(d + 2 * TY * rowU, &mp.t_row, bar, 0, 0, zp, c);
                } else {
                    if (ok(d, 2 * TY + 1, rowU, r0, n)) tma_load_4d(d, &mp.t_full, bar, 0, r0, zp, c);
                }
            }
        } else {
#pragma unroll 1
            for (int c = 0; c < 3; ++c) {
                unsigned char* d = d0 + c * (TY + 1) * rowU;
                if (h0 < 0) {
                    if (ok(d, 1, rowU, P - 1, P)) tma_load_5d(d, &mp.tp_row, bar, 0, q, P - 1, zp, c);
                    if (ok(d + rowU, TY, rowU, 0, P)) tma_load_5d(d + rowU, &mp.tp_lo, bar, 0, q, 0, zp, c);
                } else if (h0 + TY + 1 > P) {
                    if (ok(d, TY, rowU, h0, P)) tma_load_5d(d, &mp.tp_lo, bar, 0, q, h0, zp, c);
                    if (ok(d + TY * rowU, 1, rowU, 0, P)) tma_load_5d(d + TY * rowU, &mp.tp_row, bar, 0, q, 0, zp, c);
                } else {
                    if (ok(d, TY + 1, rowU, h0, P)) tma_load_5d(d, &mp.tp_full, bar, 0, q, h0, zp, c);
                }
            }
        }
    };

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

    // Programmatic dependent launch: the previous kernel may still run until
    // griddepcontrol.wait returns.  Every kernel of the solver waits on its
    // own predecessor before it lets its dependent start, so with `early`
    // (set where k and f were written two or more kernels back) the first
    // stages' k and f copies go out before the wait; T, which the previous
    // kernel writes, and every global write follow it.
    int issued = 0;
    if (tid >= ncons) {
        // Producer: stage i goes into slot i mod S once every consumer warp
        // has released stage i - S.
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
    const int y = y0 + yo + 2 * t;
    const int ke1 = 2 * t * n, ke0 = (2 * t + 1) * n;    // element rows y - 1 (b = 1) and y (b = 0)
    const int ne = 2 * t * n;                       // other-parity plane: node row y - 1 (y at +n, y + 1 at +2n)
    const int no = t * n;                           // own plane: node row y - 1 (y + 1 at +n)
    const int csE = (2 * TY + 1) * n, csO = (TY + 1) * n, csF = TY * n;
    const int oa = y * n + xa, ob = y * n + xb;     // output offsets in a plane
    const int fo = 3 * (TY + 1) * n * (int)sizeof(ST);   // f rows, bytes past the node rows
    // checking build: the furthest staged elements this thread reads and the
    // furthest output offset; a failure ends the march through the bail flag
    if (!(OTM_BOUND(ke0 + xh, 2 * TY * n, kSiteTmaGs) && OTM_BOUND(2 * csE + ne + 2 * n + xh + 1, 3 * csE, kSiteTmaGs) &&
          OTM_BOUND(2 * csO + no + n + xh + 1, 3 * csO, kSiteTmaGs) &&
          OTM_BOUND(2 * csF + t * n + (xa > xb ? xa : xb), 3 * csF, kSiteTmaGs) &&
          OTM_BOUND(oa > ob ? oa : ob, n * n, kSiteTmaGs)))
        *(volatile int*)&bail_s = 1;

    // the decision to leave is taken per warp (every lane agrees)
    auto wait = [&](int sl, uint32_t ph) -> bool {
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&full[sl], ph) && !*(volatile int*)&bail_s);
        if (!ok && (tid & 31) == 0) {
            if (err) *err = 1;
            *(volatile int*)&bail_s = 1;
        }
        return ok;
    };
    int sa = 0;          // slot of stage 2i (plane z - 1)
    uint32_t pa = 0;
    bool ok = wait(sa, pa);
#pragma unroll 1
    for (int i = 0; i < cnt && ok; ++i) {
        int sb = sa + 1 == S ? 0 : sa + 1;
        const uint32_t pb = sb == 0 ? pa ^ 1u : pa;
        int sc = sb + 1 == S ? 0 : sb + 1;
        const uint32_t pc = sc == 0 ? pb ^ 1u : pb;
        if (!wait(sb, pb) || !wait(sc, pc)) break;
        const unsigned char* SA = tsm + sa * stageBytes;   // node and element plane z - 1
        const unsigned char* SB = tsm + sb * stageBytes;   // node and element plane z, f
        const unsigned char* SC = tsm + sc * stageBytes;   // node plane z + 1
        // conductivities kk[c][b][a] of element (x - a, y - b, z - c) for node
        // x (lane 0) and x + 1 (lane 1)
        f2p kk[2][2][2];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const ST* row = reinterpret_cast<const ST*>(c ? SA : SB) + (b ? ke1 : ke0);
                const f2p lo = ld_pk(row, xo);
                kk[c][b][1] = lo;
                kk[c][b][0] = pk(pk_hi(lo), ld_one(row, xh));
            }
        // ksum8's order, then 1 / (4 sum) lane by lane
        f2p ks = kk[0][0][0];
#pragma unroll
        for (int e = 1; e < 8; ++e) ks = pk_add(ks, kk[e >> 2][(e >> 1) & 1][e & 1]);
        const float inv0 = 1.0f / (4.0f * pk_lo(ks)), inv1 = 1.0f / (4.0f * pk_hi(ks));
        f2p Pxy[2][2], Pxz[2][2], Pyz[2][2];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                Pxy[u][v] = pk_add(kk[0][u][v], kk[1][u][v]);
                Pxz[u][v] = pk_add(kk[u][0][v], kk[u][1][v]);
                Pyz[u][v] = pk_add(kk[u][v][0], kk[u][v][1]);
            }
        const int zoff = wrapz(zb + 2 * i) * n * n;
#pragma unroll
        for (int cs = 0; cs < 3; ++cs) {
            __syncwarp();
            // W[c][b] = {(x - 1, x), (x + 1, x + 2)} of plane z + 1 (c = 0) or
            // z - 1 (c = 1), row y + 1 (b = 0) or y - 1 (b = 1)
            f2p W[2][2][2], Wy[2][2], Wo[2][2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const ST* U = reinterpret_cast<const ST*>((c ? SA : SC) + kB) + cs * csE + ne;
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    W[c][b][0] = ld_pk(U + (b ? 0 : 2 * n), xo);
                    W[c][b][1] = ld_pk(U + (b ? 0 : 2 * n), xh);
                }
                Wy[c][0] = ld_pk(U + n, xo);
                Wy[c][1] = ld_pk(U + n, xh);
            }
            {
                const ST* U = reinterpret_cast<const ST*>(SB + kB) + cs * csO + no;
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    Wo[b][0] = ld_pk(U + (b ? 0 : n), xo);
                    Wo[b][1] = ld_pk(U + (b ? 0 : n), xh);
                }
            }
            const FT* F = reinterpret_cast<const FT*>(SB + kB + fo) + cs * csF + t * n;
            const float f0 = ld_one(F, xa), f1 = ld_one(F, xb);
            // nb_from's order: body diagonals (c, b, a), x-y edges (b, a),
            // x-z edges (c, a), y-z edges (c, b); neighbour x + 1 (a = 0) is
            // the pair (x + 1, x + 2), x - 1 (a = 1) the pair (x - 1, x)
            f2p acc = 0ull;
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int b = 0; b < 2; ++b)
#pragma unroll
                    for (int a = 0; a < 2; ++a) acc = pk_fma(kk[c][b][a], W[c][b][a ? 0 : 1], acc);
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int a = 0; a < 2; ++a) acc = pk_fma(Pxy[b][a], Wo[b][a ? 0 : 1], acc);
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int a = 0; a < 2; ++a) acc = pk_fma(Pxz[c][a], Wy[c][a ? 0 : 1], acc);
            // y-z edges: the node's own x column, lane 0 from the high word
            // of (x - 1, x), lane 1 from the low word of (x + 1, x + 2)
            float n0 = pk_lo(acc), n1 = pk_hi(acc);
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    n0 = fmaf(pk_lo(Pyz[c][b]), pk_hi(W[c][b][0]), n0);
                    n1 = fmaf(pk_hi(Pyz[c][b]), pk_lo(W[c][b][1]), n1);
                }
            ST* Tc = T + (size_t)cs * N + zoff;
            St<ST>::st(Tc, oa, (12.0f * f0 + n0) * inv0);
            St<ST>::st(Tc, ob, (12.0f * f1 + n1) * inv1);
        }
        // planes z - 1 and z are done with (plane z + 1 serves the next
        // output plane)
        __syncwarp();
        if ((tid & 31) == 0) {
            mbar_arrive(&empty[sa]);
            mbar_arrive(&empty[sb]);
        }
        sa = sc;
        pa = pc;
    }
    }
    // After a wait ran out, the copies still in flight land before the
    // shared memory goes away.
    __syncthreads();
    if (tid == ncons && *(volatile int*)&bail_s)
        for (int i = issued > S ? issued - S : 0; i < issued; ++i)
            (void)mbar_wait_bounded(&full[i % S], (uint32_t)((i / S) & 1));
}

// ---------------------------------------------------------------- host side
// Fine group-pass form: 0 TMA-staged where it applies, 1 the gather kernel
// k_gs_fine (OTM_GS=tma|gather; default tma).  Both give the same bits.
inline int gs_choice() {
    static int c = [] {
        const char* e = getenv("OTM_GS");
        return e && e[0] == 'g' ? 1 : 0;
    }();
    return c;
}

inline int gs_tma_rows(int n) {
    for (int t = n >= 128 ? 2 : n / 4; t >= 1; --t)
        if (n % (2 * t) == 0 && (n / 2) * t <= kTmaThreads && ((n / 2) * t) % 32 == 0 && n / (2 * t) >= 2) return t;
    return 0;
}

// Every staged row a multiple of 128 bytes and one box wide (n <= 256).
inline bool gs_tma_ok(int n, int st_size, int ft_size) {
    if (n < 32 || n > 256 || n % 4) return false;
    if ((n * st_size) % 128 || (n * ft_size) % 128) return false;
    if ((long long)n * n * n * 3 >= (1LL << 31)) return false;
    return gs_tma_rows(n) > 0 && tma_encoder() != nullptr;
}

// Ring depth (OTM_GS_STAGES overrides, 4..8): an output plane holds three
// stages, so depth S keeps S - 3 stages in flight ahead of it.  Five is the
// measured best inside the 128^3 design step on GB300 (FP32: 2.44 ms per
// iteration at 5 stages, 2.45 at 4, 2.59 at 6, 2.55 at 8; six FP32 stages
// fill 215 KB of each SM's shared memory with two CTAs, which costs more
// than the deeper ring gains where the pass overlaps its neighbours).
inline bool gs_tma_stages_fixed() { return getenv("OTM_GS_STAGES") != nullptr; }
inline int gs_tma_stages() {
    static int s = [] {
        const char* e = getenv("OTM_GS_STAGES");
        const int v = e ? atoi(e) : 0;
        return v >= 4 && v <= kTmaMaxStages ? v : 5;
    }();
    return s;
}

// Runs of output planes: minimise (waves) x (stages per run), stages per
// run = 2 (planes) + 1.  OTM_GS_M overrides.
inline int gs_tma_m(int n, int sm_count, int per_sm) {
    const int ty = gs_tma_rows(n);
    if (ty == 0) return 0;
    const int P = n / 2;
    const long long nrb = n / (2 * ty);
    const char* e = getenv("OTM_GS_M");
    if (e && atoi(e) >= 1 && atoi(e) <= P) return atoi(e);
    const long long slots = (long long)std::max(per_sm, 1) * sm_count;
    int best = 0;
    double best_t = 0.0;
    for (int m = 1; m <= P; ++m) {
        const long long waves = (nrb * m + slots - 1) / slots;
        const double t = (double)waves * (2.0 * ((P + m - 1) / m) + 1.0);
        if (best == 0 || t < best_t - 1e-9) {
            best = m;
            best_t = t;
        }
    }
    return best;
}

// Encodes the maps of one launch (T and f of the three load cases, k);
// false when the encoder refuses a map.
template <class ST, class FT>
inline bool gs_tma_make_maps(TmaGsMaps& mp, int n, const void* k, const void* T, const void* f) {
    TmaEncodeFn enc = tma_encoder();
    if (!enc) return false;
    const int ty = gs_tma_rows(n);
    memset(&mp, 0, sizeof(mp));
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    auto go = [&](CUtensorMap* m, int rank, const void* base, CUtensorMapDataType dt, const cuuint64_t* dims,
                  const cuuint64_t* str, const cuuint32_t* box) {
        return enc(m, dt, (cuuint32_t)rank, const_cast<void*>(base), dims, str, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    const cuuint64_t nn = (cuuint64_t)n;
    auto rows4 = [&](CUtensorMap* m, int rows) {   // T as [3][n][n][n]
        const cuuint64_t e = sizeof(ST);
        const cuuint64_t dims[4] = {nn, nn, nn, 3}, str[3] = {nn * e, nn * nn * e, nn * nn * nn * e};
        const cuuint32_t box[4] = {(cuuint32_t)n, (cuuint32_t)rows, 1, 1};
        return go(m, 4, T, TmaType<ST>::v, dims, str, box);
    };
    auto par5 = [&](CUtensorMap* m, const void* base, size_t e, CUtensorMapDataType dt, int rows) {
        // (x, y mod 2, y / 2, z, case)
        const cuuint64_t dims[5] = {nn, 2, nn / 2, nn, 3};
        const cuuint64_t str[4] = {nn * e, 2 * nn * e, nn * nn * e, nn * nn * nn * e};
        const cuuint32_t box[5] = {(cuuint32_t)n, 1, (cuuint32_t)rows, 1, 1};
        return go(m, 5, base, dt, dims, str, box);
    };
    auto rows3 = [&](CUtensorMap* m, int rows) {   // k as [n][n][n]
        const cuuint64_t e = sizeof(ST);
        const cuuint64_t dims[3] = {nn, nn, nn}, str[2] = {nn * e, nn * nn * e};
        const cuuint32_t box[3] = {(cuuint32_t)n, (cuuint32_t)rows, 1};
        return go(m, 3, k, TmaType<ST>::v, dims, str, box);
    };
    const auto dts = TmaType<ST>::v;
    return rows4(&mp.t_full, 2 * ty + 1) && rows4(&mp.t_lo, 2 * ty) && rows4(&mp.t_row, 1) &&
           par5(&mp.tp_full, T, sizeof(ST), dts, ty + 1) && par5(&mp.tp_lo, T, sizeof(ST), dts, ty) &&
           par5(&mp.tp_row, T, sizeof(ST), dts, 1) && rows3(&mp.k_full, 2 * ty) && rows3(&mp.k_lo, 2 * ty - 1) &&
           rows3(&mp.k_row, 1) && par5(&mp.fp_rows, f, sizeof(FT), TmaType<FT>::v, ty);
}

// The instantiation for this n (compile-time n for the common sizes) and
// its launch shape.  Static for the reason given at tma_kernel: the
// shared-memory opt-in belongs to the translation unit's own stub.
template <class ST, class FT>
using GsTmaKernel = void (*)(TmaGsMaps, int, int, int, int, int, ST*, int*, int);
template <class ST, class FT>
static GsTmaKernel<ST, FT> gs_tma_kernel(int n) {
    if (n == 64) return k_gs_tma<64, ST, FT>;
    if (n == 128) return k_gs_tma<128, ST, FT>;
    if (n == 256) return k_gs_tma<256, ST, FT>;
    return k_gs_tma<0, ST, FT>;
}

// stages: ring depth (0: the default, gs_tma_stages)
template <class ST, class FT>
static bool gs_tma_launch_shape(TmaLaunch& L, int n, int sm_count, int stages = 0) {
    if (!gs_tma_ok(n, (int)sizeof(ST), (int)sizeof(FT))) return false;
    auto kern = gs_tma_kernel<ST, FT>(n);
    L.n = n;
    L.ty = gs_tma_rows(n);
    L.threads = (n / 2) * L.ty + 32;   // consumer warps + the producer warp
    L.stages = stages >= 4 && stages <= kTmaMaxStages ? stages : gs_tma_stages();
    L.smem = (size_t)L.stages * gs_tma_stage_bytes(n, L.ty, (int)sizeof(ST), (int)sizeof(FT)) + 128;
    {
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
            granted[ki][d] = L.smem;
        }
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, L.threads, L.smem) != cudaSuccess || per_sm < 1)
        return false;
    L.m = gs_tma_m(n, sm_count, per_sm);
    if (L.m < 1) return false;
    L.grid = (n / (2 * L.ty)) * L.m;
    return true;
}

}  // namespace otm
