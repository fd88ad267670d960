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

constexpr int kClusterCTAs = 8;
constexpr int kClusterThreads = 512;
constexpr int kClusterMaxN = 32;

template <class S, class C>
struct ClusterArgs {
    int lc, L;                 // first level run here, coarsest level
    int minv_smem;             // 1: stage the coarsest inverse in shared memory
    int pad;
    int n[kMaxLevelsDev];
    S* T[kMaxLevelsDev];
    S* F[kMaxLevelsDev];
    S* Rr[kMaxLevelsDev];
    const S* A[kMaxLevelsDev];
    const C* Minv;
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

template <class S, class C>
__global__ void __cluster_dims__(kClusterCTAs, 1, 1) __launch_bounds__(kClusterThreads)
k_coarse_cluster(ClusterArgs<S, C> a) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char cl_sm[];
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    const int ts = gridDim.x * blockDim.x;
    // down: forward sweep, residual, restriction
    for (int l = a.lc; l < a.L; ++l) {
        const int n = a.n[l];
        const size_t N = (size_t)n * n * n;
        cl_gs_pass<true, S>(n, 0, a.A[l], a.F[l], a.T[l], t0, ts);
        cluster_barrier();
        for (int c = 1; c < 8; ++c) {
            cl_gs_pass<false, S>(n, c, a.A[l], a.F[l], a.T[l], t0, ts);
            cluster_barrier();
        }
        for (int t = t0; t < (int)N; t += ts)
            residual_stencil_node<S, S, S, S>(n, N, t % n, (t / n) % n, t / (n * n), a.A[l], a.F[l], a.T[l], a.Rr[l]);
        cluster_barrier();
        const int nc = n / 2;
        for (int t = t0; t < nc * nc * nc; t += ts)
            restrict_node<S, S>(nc, t % nc, (t / nc) % nc, t / (nc * nc), a.Rr[l], a.F[l + 1]);
        cluster_barrier();
    }
    // coarsest: dense solve in CTA 0
    if (blockIdx.x == 0) {
        const int nL = a.n[a.L];
        const C* Minv = stage_minv<C>(a.Minv, nL * nL * nL - 1, a.minv_smem, cl_sm);
        coarse_solve_block<C, S, S>(nL, Minv, a.F[a.L], a.T[a.L]);
    }
    cluster_barrier();
    // up: prolongation + correction, reverse sweep
    for (int l = a.L - 1; l >= a.lc; --l) {
        const int n = a.n[l];
        for (int t = t0; t < n * n * n; t += ts) prolong_node<S, S>(n, t % n, (t / n) % n, t / (n * n), a.T[l + 1], a.T[l]);
        cluster_barrier();
        for (int c = 7; c >= 0; --c) {
            cl_gs_pass<false, S>(n, c, a.A[l], a.F[l], a.T[l], t0, ts);
            cluster_barrier();
        }
    }
}

}  // namespace otm
