// The small levels of the V-cycle (Alg. 3) in one thread-block cluster.
//
// Levels whose grids are at most kClusterMaxN per side hold a few thousand
// nodes, so each of their Gauss-Seidel colour passes, residuals and
// transfers is latency work.  One cluster of kClusterCTAs CTAs runs all of
// them -- the forward sweeps and restrictions down from level lc, the dense
// coarsest solve, the prolongations and reverse sweeps back up to lc -- in a
// single launch, separated by hardware cluster barriers instead of kernel
// boundaries.  A cluster's CTAs are co-scheduled by construction, so the
// barriers cannot wait on a CTA that is not running.  The per-node
// arithmetic is the same device code the standalone kernels use.
#pragma once
#include "kernels_fine.cuh"
#include "kernels_mg.cuh"

namespace otm {

constexpr int kClusterCTAs = 8;        // portable cluster size; 16 (non-portable) where the device allows
constexpr int kClusterThreads = 512;
constexpr int kClusterMaxN = 16;

template <class S, class C>
struct ClusterArgs {
    int lc, L;                 // first level run here, coarsest level
    int minv_smem;             // 1: stage the coarsest inverse in shared memory
    int lb;                    // levels lb..L run in CTA 0 with shared-memory fields (lb > L: none)
    int cheb;                  // 1: Chebyshev smoother on the cluster levels (else 8-colour GS)
    int n[kMaxLevelsDev];
    S* T[kMaxLevelsDev];
    S* F[kMaxLevelsDev];
    S* Rr[kMaxLevelsDev];
    const S* A[kMaxLevelsDev];
    S* T2[kMaxLevelsDev];      // second field buffer and direction of the Chebyshev smoother
    S* D[kMaxLevelsDev];
    const float* lam;          // per-level Gershgorin bounds
    const C* Minv;
    // shared-memory tail layout (byte offsets, from tail_layout on the host)
    unsigned tT[kMaxLevelsDev], tF[kMaxLevelsDev], tA[kMaxLevelsDev], tR, tMinv;
    // dsm = 1: the one cluster-wide level lc (followed by the tail at lb = lc
    // + 1) lives in the CTAs' shared memory; dmg slots per colour and CTA,
    // lg = log2(CTAs); byte offsets of each CTA's stencil rows, right-hand
    // side, field and residual
    int dsm, dmg, dlg;
    unsigned dA, dF, dT, dR;
};

// Cluster-wide barrier.  The arrive has release and the wait acquire
// semantics at cluster scope, which orders every thread's earlier global
// writes before the other CTAs' later reads.
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <bool ZERO, class S>
__device__ __forceinline__ void cl_gs_pass(int n, int colour, const S* A, const S* F, S* T, int t0, int ts) {
    const size_t N = (size_t)n * n * n;
    const int h = n >> 1;
    const int xo = colour & 1, yo = (colour >> 1) & 1, zo = colour >> 2;
    const int M = h * h * h;
    for (int t = t0; t < M; t += ts) {
        const int xi = t % h, yi = (t / h) % h, zi = t / (h * h);
        gs_stencil_node<ZERO, S, S, S>(n, N, 2 * xi + xo, 2 * yi + yo, 2 * zi + zo, A, F, T);
    }
}

// Byte offsets of the shared-memory tail's arrays: per level l in lb..L the
// fields T_l and F_l (3 N_l values each) and the stencil A_l (27 N_l), one
// residual buffer of 3 N_lb values reused by every level, then the staged
// coarsest inverse.  Each array starts on a 16-byte boundary.
struct TailLayout {
    size_t T[kMaxLevelsDev], F[kMaxLevelsDev], A[kMaxLevelsDev], R, minv, total;
};
template <class S, class C>
inline TailLayout tail_layout(int lb, int L, const int* n, int minv_smem) {
    TailLayout t = {};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 15) / 16 * 16;
        return o;
    };
    for (int l = lb; l <= L; ++l) {
        const size_t nodes = (size_t)n[l] * n[l] * n[l];
        t.T[l] = take(4 * nodes * sizeof(S));
        t.F[l] = take(4 * nodes * sizeof(S));
        t.A[l] = take((size_t)cl_aw<S>() * nodes * sizeof(S));
    }
    t.R = take(4 * (size_t)n[lb] * n[lb] * n[lb] * sizeof(S));
    const size_t q = (size_t)n[L] * n[L] * n[L] - 1;
    t.minv = off;
    if (minv_smem) take(q * q * sizeof(C));
    t.total = off;
    return t;
}

// Levels lb..L (including the coarsest solve) in one CTA: the fields and the
// stencils live in shared memory (copied in once per V-cycle), and phases are
// separated by __syncthreads instead of cluster barriers or kernel
// boundaries.  Reads F_lb and A_lb..A_L from, and writes T_lb to, global
// memory.
template <class S, class C>
__device__ void coarse_tail_block(const ClusterArgs<S, C>& a, unsigned char* sm) {
    const int t0 = threadIdx.x, ts = blockDim.x;
    auto Ts = [&](int l) { return reinterpret_cast<S*>(sm + a.tT[l]); };
    auto Fs = [&](int l) { return reinterpret_cast<S*>(sm + a.tF[l]); };
    auto As = [&](int l) { return reinterpret_cast<const S*>(sm + a.tA[l]); };
    S* Rs = reinterpret_cast<S*>(sm + a.tR);
    {
        const int nb = a.n[a.lb];
        // (with the level above in distributed shared memory, its restriction
        // has written F_lb here already)
        if (!a.dsm) block_copy_async(Fs(a.lb), a.F[a.lb], (size_t)4 * nb * nb * nb * sizeof(S));
        // (the stencils were issued at the kernel's start, before its wait on
        // the previous kernel)
        cp_async_wait_all();
    }
    __syncthreads();
    for (int l = a.lb; l < a.L; ++l) {
        const int n = a.n[l];
        const size_t N = (size_t)n * n * n;
        cl_gs_pass<true, S>(n, 0, As(l), Fs(l), Ts(l), t0, ts);
        __syncthreads();
        for (int c = 1; c < 8; ++c) {
            cl_gs_pass<false, S>(n, c, As(l), Fs(l), Ts(l), t0, ts);
            __syncthreads();
        }
        for (int t = t0; t < (int)N; t += ts)
            residual_stencil_node<S, S, S, S>(n, N, t % n, (t / n) % n, t / (n * n), As(l), Fs(l), Ts(l), Rs);
        __syncthreads();
        const int nc = n / 2;
        for (int t = t0; t < nc * nc * nc; t += ts)
            restrict_node<S, S, true>(nc, t % nc, (t / nc) % nc, t / (nc * nc), Rs, Fs(l + 1));
        __syncthreads();
    }
    {
        const int nL = a.n[a.L];
        const C* Minv = stage_minv<C>(a.Minv, nL * nL * nL - 1, a.minv_smem, sm + a.tMinv);
        coarse_solve_block<C, S, S>(nL, Minv, Fs(a.L), Ts(a.L));
    }
    __syncthreads();
    for (int l = a.L - 1; l >= a.lb; --l) {
        const int n = a.n[l];
        for (int t = t0; t < n * n * n; t += ts) prolong_node<S, S, true>(n, t % n, (t / n) % n, t / (n * n), Ts(l + 1), Ts(l));
        __syncthreads();
        for (int c = 7; c >= 0; --c) {
            cl_gs_pass<false, S>(n, c, As(l), Fs(l), Ts(l), t0, ts);
            __syncthreads();
        }
    }
    {
        const int nb = a.n[a.lb];
        const int m = 4 * nb * nb * nb;
        for (int i = t0; i < m; i += ts) a.T[a.lb][i] = Ts(a.lb)[i];
    }
}

// ---- the cluster-wide level in distributed shared memory
//
// Node (x, y, z) of the level (h = n / 2) has colour c = (x & 1) + 2 (y & 1)
// + 4 (z & 1) and index t = (x >> 1) + h ((y >> 1) + h (z >> 1)) among the
// M = h^3 nodes of its colour.  It belongs to CTA t mod G -- the CTA whose
// threads relax it in a colour pass, as in the global-memory form -- at slot
// c MG + t / G of that CTA's arrays (MG = ceil(M / G)).  Each CTA stages its
// nodes' stencil rows and right-hand side once per launch; a colour pass
// reads the neighbours' fields from their owners' shared memory through the
// cluster window, so a phase costs a shared-memory round trip and a cluster
// barrier instead of an L2 round trip.  Every node's arithmetic is the same
// sequence as in the global-memory form (gs_stencil_node, residual_stencil_node,
// restrict_node, prolong_node), so the results are the same bits.
template <class S>
struct DsmLevel {
    int n, h, M, MG, lg;
    S *A, *F, *T, *R;   // this CTA's arrays (generic addresses in its shared memory)
    __device__ __forceinline__ int owner(int x, int y, int z, int& slot) const {
        const int c = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
        const int t = (x >> 1) + h * ((y >> 1) + h * (z >> 1));
        slot = c * MG + (t >> lg);
        return t & ((1 << lg) - 1);
    }
    // node of this CTA's slot (c, j); false past the colour's last node
    __device__ __forceinline__ bool node(int c, int j, int& x, int& y, int& z) const {
        const int t = (int)blockIdx.x + (j << lg);
        if (j >= MG || t >= M) return false;
        x = 2 * (t % h) + (c & 1);
        y = 2 * ((t / h) % h) + ((c >> 1) & 1);
        z = 2 * (t / (h * h)) + (c >> 2);
        return true;
    }
};

template <bool ZERO, class S>
__device__ void dsm_gs_pass(const DsmLevel<S>& L, int c) {
    using C = typename St<S>::C;
    for (int j = threadIdx.x; j < L.MG; j += blockDim.x) {
        int x, y, z;
        if (!L.node(c, j, x, y, z)) break;
        const int slot = c * L.MG + j;
        C a[27];
        ld_arow<S>(L.A, slot, a);
        const C inv = C(1) / a[13];
        C s[3];
        ld_f3<S>(L.F, slot, s);
        if (!ZERO) {
#pragma unroll
            for (int o = 0; o < 27; ++o) {
                if (o == 13) continue;
                int sl;
                const int r = L.owner(wrapd(x, o % 3 - 1, L.n), wrapd(y, (o / 3) % 3 - 1, L.n),
                                      wrapd(z, o / 9 - 1, L.n), sl);
                C t[3];
                ld_f3<S>(dsm_ptr(L.T, (uint32_t)r), sl, t);
#pragma unroll
                for (int i = 0; i < 3; ++i) s[i] -= a[o] * t[i];
            }
        }
        st_f3<S>(L.T, slot, s[0] * inv, s[1] * inv, s[2] * inv);
    }
}

template <class S>
__device__ void dsm_residual(const DsmLevel<S>& L) {
    using C = typename St<S>::C;
    for (int k = threadIdx.x; k < 8 * L.MG; k += blockDim.x) {
        const int c = k / L.MG, j = k - c * L.MG;
        int x, y, z;
        if (!L.node(c, j, x, y, z)) continue;
        C a[27];
        ld_arow<S>(L.A, k, a);
        C s[3];
        ld_f3<S>(L.F, k, s);
#pragma unroll
        for (int o = 0; o < 27; ++o) {
            int sl;
            const int r = L.owner(wrapd(x, o % 3 - 1, L.n), wrapd(y, (o / 3) % 3 - 1, L.n),
                                  wrapd(z, o / 9 - 1, L.n), sl);
            C t[3];
            ld_f3<S>(dsm_ptr(L.T, (uint32_t)r), sl, t);
#pragma unroll
            for (int i = 0; i < 3; ++i) s[i] -= a[o] * t[i];
        }
        st_f3<S>(L.R, k, s[0], s[1], s[2]);
    }
}

// F_c = R r into the tail CTA's right-hand side (CTA 0, node-major)
template <class S>
__device__ void dsm_restrict(const DsmLevel<S>& L, S* Fc0) {
    using C = typename St<S>::C;
    const int nc = L.h, G = 1 << L.lg;
    S* Fc = dsm_ptr(Fc0, 0u);
    for (int I = (int)threadIdx.x * G + (int)blockIdx.x; I < nc * nc * nc; I += G * (int)blockDim.x) {
        const int X = I % nc, Y = (I / nc) % nc, Z = I / (nc * nc);
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
                    int sl;
                    const int r = L.owner(wrapd(2 * X, dx - 1, L.n), wrapd(2 * Y, dy - 1, L.n),
                                          wrapd(2 * Z, dz - 1, L.n), sl);
                    C t[3];
                    ld_f3<S>(dsm_ptr(L.R, (uint32_t)r), sl, t);
#pragma unroll
                    for (int i = 0; i < 3; ++i) ay[i] += w1[dx] * t[i];
                }
#pragma unroll
                for (int i = 0; i < 3; ++i) az[i] += w1[dy] * ay[i];
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) acc[i] += w1[dz] * az[i];
        }
        st_f3<S>(Fc, I, acc[0], acc[1], acc[2]);
    }
}

// T += P T_c with T_c the tail's field, read from global memory where the
// tail stored it (every CTA reading it from CTA 0's shared memory would queue
// all the cluster's loads at that one SM: 20 us against about 2 through L2)
template <class S>
__device__ void dsm_prolong(const DsmLevel<S>& L, const S* __restrict__ Tc) {
    using C = typename St<S>::C;
    const int nc = L.h;
    for (int k = threadIdx.x; k < 8 * L.MG; k += blockDim.x) {
        const int cc = k / L.MG, j = k - cc * L.MG;
        int x, y, z;
        if (!L.node(cc, j, x, y, z)) continue;
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
                    C t[3];
                    ld_f3<S>(Tc, (size_t)xi[a] + (size_t)nc * (yi[b] + (size_t)nc * zi[c]), t);
                    const C w = wz[c] * wy[b] * wx[a];
#pragma unroll
                    for (int i = 0; i < 3; ++i) acc[i] += w * t[i];
                }
        C t0[3];
        ld_f3<S>(L.T, k, t0);
        st_f3<S>(L.T, k, t0[0] + acc[0], t0[1] + acc[1], t0[2] + acc[2]);
    }
}

// Launched as one cluster (the cluster size is the grid size, set at launch).
template <class S, class C>
__global__ void __launch_bounds__(kClusterThreads)
k_coarse_cluster(ClusterArgs<S, C> a) {
    extern __shared__ __align__(16) unsigned char cl_sm[];
    // node index t runs over the CTAs fastest, so a small pass spreads over
    // every SM of the cluster instead of filling CTA 0 first
    const int t0 = threadIdx.x * gridDim.x + blockIdx.x;
    const int ts = gridDim.x * blockDim.x;
    const int lend = a.lb <= a.L ? a.lb : a.L;   // first level not swept by the whole cluster
    // The stencils were written at the hierarchy's setup, so their staging
    // goes out before the wait on the previous kernel (whose output -- the
    // cluster's first right-hand side -- is read only after it): the tail's
    // in CTA 0, and the shared-memory level's rows in every CTA.
    if (blockIdx.x == 0 && a.lb <= a.L)
        for (int l = a.lb; l <= a.L; ++l)
            block_copy_async(cl_sm + a.tA[l], a.A[l], (size_t)cl_aw<S>() * a.n[l] * a.n[l] * a.n[l] * sizeof(S));
    if (a.dsm) {
        const int l = a.lc, n = a.n[l], h = n / 2, M = h * h * h, lg = a.dlg;
        constexpr int kRowBytes = cl_aw<S>() * (int)sizeof(S);   // a multiple of 16
        for (int k = threadIdx.x; k < 8 * a.dmg; k += blockDim.x) {
            const int c = k / a.dmg, j = k - c * a.dmg;
            const int t = (int)blockIdx.x + (j << lg);
            if (t >= M) continue;
            const int x = 2 * (t % h) + (c & 1), y = 2 * ((t / h) % h) + ((c >> 1) & 1), z = 2 * (t / (h * h)) + (c >> 2);
            const size_t v = (size_t)x + (size_t)n * (y + (size_t)n * z);
            const unsigned char* src = reinterpret_cast<const unsigned char*>(a.A[l] + v * cl_aw<S>());
            unsigned char* dst = cl_sm + a.dA + (size_t)k * kRowBytes;
#pragma unroll
            for (int q = 0; q < kRowBytes / 16; ++q) cp_async16(dst + 16 * q, src + 16 * q);
        }
    }
    pdl_enter();
    if (a.dsm) {
        // the one cluster-wide level lc in distributed shared memory, then the tail
        using CS = typename St<S>::C;
        const int l = a.lc;
        DsmLevel<S> Ld;
        Ld.n = a.n[l];
        Ld.h = Ld.n / 2;
        Ld.M = Ld.h * Ld.h * Ld.h;
        Ld.MG = a.dmg;
        Ld.lg = a.dlg;
        Ld.A = reinterpret_cast<S*>(cl_sm + a.dA);
        Ld.F = reinterpret_cast<S*>(cl_sm + a.dF);
        Ld.T = reinterpret_cast<S*>(cl_sm + a.dT);
        Ld.R = reinterpret_cast<S*>(cl_sm + a.dR);
        // this CTA's right-hand side (its stencil rows are in flight since the
        // kernel's start); its field starts at zero
        for (int k = threadIdx.x; k < 8 * Ld.MG; k += blockDim.x) {
            const int c = k / Ld.MG, j = k - c * Ld.MG;
            int x, y, z;
            if (!Ld.node(c, j, x, y, z)) continue;
            const size_t v = (size_t)x + (size_t)Ld.n * (y + (size_t)Ld.n * z);
            CS f3[3];
            ld_f3<S>(a.F[l], v, f3);
            st_f3<S>(Ld.F, k, f3[0], f3[1], f3[2]);
            st_f3<S>(Ld.T, k, CS(0), CS(0), CS(0));
        }
        cp_async_wait_all();
        __syncthreads();
        // forward sweep (colour 0 from zero reads no neighbour), residual,
        // restriction into the tail's right-hand side
        dsm_gs_pass<true, S>(Ld, 0);
        cluster_barrier();
        for (int c = 1; c < 8; ++c) {
            dsm_gs_pass<false, S>(Ld, c);
            cluster_barrier();
        }
        dsm_residual<S>(Ld);
        cluster_barrier();
        dsm_restrict<S>(Ld, reinterpret_cast<S*>(cl_sm + a.tF[a.lb]));
        cluster_barrier();
        if (blockIdx.x == 0) coarse_tail_block<S, C>(a, cl_sm);
        cluster_barrier();
        // correction from the tail's field, reverse sweep
        dsm_prolong<S>(Ld, a.T[a.lb]);
        cluster_barrier();
        for (int c = 7; c >= 0; --c) {
            dsm_gs_pass<false, S>(Ld, c);
            cluster_barrier();   // (also: no CTA leaves while another reads its shared memory)
        }
        // the level's field for the finer level's prolongation
        for (int k = threadIdx.x; k < 8 * Ld.MG; k += blockDim.x) {
            const int c = k / Ld.MG, j = k - c * Ld.MG;
            int x, y, z;
            if (!Ld.node(c, j, x, y, z)) continue;
            CS t3[3];
            ld_f3<S>(Ld.T, k, t3);
            st_f3<S>(a.T[l], (size_t)x + (size_t)Ld.n * (y + (size_t)Ld.n * z), t3[0], t3[1], t3[2]);
        }
        return;
    }
    static_assert(kChebDeg % 2 == 1, "the Chebyshev buffers alternate: an odd degree ends in T2");
    // one Chebyshev smoothing of level l: steps alternate T -> T2 -> T ...;
    // from_zero: the field starts at zero (pre-smoothing, ends in T2), else
    // it starts in T2 (post-smoothing, ends in T)
    auto cheb_smooth = [&](int l, bool from_zero) {
        const int n = a.n[l];
        const size_t N = (size_t)n * n * n;
        for (int k = 0; k < kChebDeg; ++k) {
            float c_d, c_r;
            cheb_coef(a.lam[l], k, c_d, c_r);
            const bool to_t2 = from_zero ? (k % 2 == 0) : (k % 2 == 1);
            const S* Tin = to_t2 ? a.T[l] : a.T2[l];
            S* Tout = to_t2 ? a.T2[l] : a.T[l];
            for (int t = t0; t < (int)N; t += ts) {
                if (from_zero && k == 0)
                    cheb_node<true, S, S, S>(n, N, t % n, (t / n) % n, t / (n * n), a.A[l], a.F[l], Tin, Tout, a.D[l],
                                             c_d, c_r);
                else
                    cheb_node<false, S, S, S>(n, N, t % n, (t / n) % n, t / (n * n), a.A[l], a.F[l], Tin, Tout,
                                              a.D[l], c_d, c_r);
            }
            cluster_barrier();
        }
    };
    // down: forward sweep, residual, restriction
    for (int l = a.lc; l < lend; ++l) {
        const int n = a.n[l];
        const size_t N = (size_t)n * n * n;
        S* Tcur = a.T[l];
        if (a.cheb) {
            cheb_smooth(l, true);
            Tcur = a.T2[l];
        } else {
            cl_gs_pass<true, S>(n, 0, a.A[l], a.F[l], a.T[l], t0, ts);
            cluster_barrier();
            for (int c = 1; c < 8; ++c) {
                cl_gs_pass<false, S>(n, c, a.A[l], a.F[l], a.T[l], t0, ts);
                cluster_barrier();
            }
        }
        for (int t = t0; t < (int)N; t += ts)
            residual_stencil_node<S, S, S, S>(n, N, t % n, (t / n) % n, t / (n * n), a.A[l], a.F[l], Tcur, a.Rr[l]);
        cluster_barrier();
        const int nc = n / 2;
        for (int t = t0; t < nc * nc * nc; t += ts)
            restrict_node<S, S, true>(nc, t % nc, (t / nc) % nc, t / (nc * nc), a.Rr[l], a.F[l + 1]);
        cluster_barrier();
    }
    // coarsest: dense solve in CTA 0, or the shared-memory tail lb..L
    if (blockIdx.x == 0) {
        if (a.lb <= a.L) {
            coarse_tail_block<S, C>(a, cl_sm);
        } else {
            const int nL = a.n[a.L];
            const C* Minv = stage_minv<C>(a.Minv, nL * nL * nL - 1, a.minv_smem, cl_sm);
            coarse_solve_block<C, S, S>(nL, Minv, a.F[a.L], a.T[a.L]);
        }
    }
    cluster_barrier();
    // up: prolongation + correction, reverse sweep
    for (int l = lend - 1; l >= a.lc; --l) {
        const int n = a.n[l];
        S* Tcur = a.cheb ? a.T2[l] : a.T[l];
        for (int t = t0; t < n * n * n; t += ts) prolong_node<S, S, true>(n, t % n, (t / n) % n, t / (n * n), a.T[l + 1], Tcur);
        cluster_barrier();
        if (a.cheb) {
            cheb_smooth(l, false);
        } else {
            for (int c = 7; c >= 0; --c) {
                cl_gs_pass<false, S>(n, c, a.A[l], a.F[l], a.T[l], t0, ts);
                cluster_barrier();
            }
        }
    }
}

}  // namespace otm
