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
        block_copy_async(Fs(a.lb), a.F[a.lb], (size_t)4 * nb * nb * nb * sizeof(S));
        for (int l = a.lb; l <= a.L; ++l)
            block_copy_async(sm + a.tA[l], a.A[l], (size_t)cl_aw<S>() * a.n[l] * a.n[l] * a.n[l] * sizeof(S));
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

// Launched as one cluster (the cluster size is the grid size, set at launch).
template <class S, class C>
__global__ void __launch_bounds__(kClusterThreads)
k_coarse_cluster(ClusterArgs<S, C> a) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char cl_sm[];
    // node index t runs over the CTAs fastest, so a small pass spreads over
    // every SM of the cluster instead of filling CTA 0 first
    const int t0 = threadIdx.x * gridDim.x + blockIdx.x;
    const int ts = gridDim.x * blockDim.x;
    const int lend = a.lb <= a.L ? a.lb : a.L;   // first level not swept by the whole cluster
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
