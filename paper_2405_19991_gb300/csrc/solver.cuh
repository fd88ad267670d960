// Host-side orchestration of one design context on one GPU stream:
// buffers, the multigrid hierarchy, the three-load-case MG-PCG solve and the
// design iteration.  Instantiated per precision in solver_*.cu.
#pragma once
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <type_traits>
#include <vector>

#include "kernels_design.cuh"
#include "kernels_fine.cuh"
#include "kernels_mg.cuh"
#include "kernels_tiled.cuh"
#include "kernels_cluster.cuh"
#include "kernels_warprow.cuh"
#include "kernels_tma.cuh"
#include "kernels_gs_tma.cuh"
#include "kernels_mma.cuh"
#include "kernels_ws.cuh"
#include "otm_internal.cuh"
#include "unet_api.cuh"

namespace otm {

constexpr int kMaxLevels = 12;

// Graph capture and instantiation are done under one process-wide lock:
// contexts stepped from several host threads (otm_design_batch) build their
// graphs one at a time and only launch them concurrently.
inline std::mutex& graph_build_mutex() {
    static std::mutex m;
    return m;
}

// Abstract interface used by the C ABI.
struct SolverBase {
    virtual ~SolverBase() {}
    virtual otm_status init(const otm_params& p) = 0;
    virtual otm_status set_density(const float* rho, bool on_device) = 0;
    virtual otm_status get_density(float* rho, bool on_device) = 0;
    virtual otm_status get_field(int which, float* out, size_t count, bool on_device) = 0;
    virtual otm_status homogenize(const float* rho, bool on_device, double kappa[6], otm_step_info* info) = 0;
    virtual otm_status step(otm_step_info* info) = 0;
    virtual size_t state_size() const = 0;
    virtual otm_status get_state(void* buf) = 0;
    virtual otm_status set_state(const void* buf, size_t len) = 0;
    virtual otm_status set_predictor(otm_unet* u, double scale) = 0;
    // Build the step's CUDA graphs now (they are otherwise built by the first
    // step); graph construction is serialised process-wide.
    virtual otm_status prepare() = 0;
    virtual otm_status get_config(otm_config* out) = 0;
    std::string err;
    otm_params prm;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
};

SolverBase* make_solver_f64();
SolverBase* make_solver_f32();
SolverBase* make_solver_mixed();

// Checks a CUDA call; on failure records the message and returns OTM_ECUDA.
#define OTM_CU(call)                                                                   \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
            return e_ == cudaErrorMemoryAllocation ? OTM_ENOMEM : OTM_ECUDA;           \
        }                                                                              \
    } while (0)
#define OTM_LAUNCH()                                                                   \
    do {                                                                               \
        cudaError_t e_ = cudaGetLastError();                                           \
        if (e_ != cudaSuccess) {                                                       \
            err = std::string("kernel launch: ") + cudaGetErrorString(e_);             \
            return OTM_ECUDA;                                                          \
        }                                                                              \
    } while (0)
#define OTM_TRY(expr)                                                                  \
    do {                                                                               \
        otm_status s_ = (expr);                                                        \
        if (s_ != OTM_OK) return s_;                                                   \
    } while (0)

// Host-side constant tables of the hierarchy (the GPU path's own derivation
// of K0 from the 1-D stiffness and mass matrices, see kernels_fine.cuh).
inline double k0_entry(int l, int m) {
    const int pc = __builtin_popcount(l ^ m);
    return pc == 0 ? 1.0 / 3.0 : (pc == 1 ? 0.0 : -1.0 / 12.0);
}
inline double phi_w(int t, int m) {
    static const double w0[3] = {1.0, 0.5, 0.0};
    static const double w1[3] = {0.0, 0.5, 1.0};
    return m ? w1[t] : w0[t];
}
inline void build_ps(std::vector<double>& Ps, std::vector<double>& Bs) {
    Ps.assign(8 * 64, 0.0);
    Bs.assign(8 * 64, 0.0);
    for (int s = 0; s < 8; ++s) {
        for (int j = 0; j < 8; ++j)
            for (int m = 0; m < 8; ++m) {
                double w = 1.0;
                for (int d = 0; d < 3; ++d) w *= phi_w(((s >> d) & 1) + ((j >> d) & 1), (m >> d) & 1);
                Ps[s * 64 + j * 8 + m] = w;
            }
        for (int m = 0; m < 8; ++m)
            for (int mp = 0; mp < 8; ++mp) {
                double a = 0.0;
                for (int j = 0; j < 8; ++j)
                    for (int jp = 0; jp < 8; ++jp)
                        a += Ps[s * 64 + j * 8 + m] * k0_entry(j, jp) * Ps[s * 64 + jp * 8 + mp];
                Bs[s * 64 + m * 8 + mp] = a;
            }
    }
}

inline FilterW make_filter(double rmin) {
    FilterW fw;
    memset(&fw, 0, sizeof(fw));
    fw.R = (int)std::ceil(rmin) - 1;
    double wsum = 0.0;
    for (int d2 = 0; d2 < 13; ++d2) {
        const double d = std::sqrt((double)d2);
        fw.w[d2] = d < rmin ? rmin - d : 0.0;
    }
    for (int dz = -fw.R; dz <= fw.R; ++dz)
        for (int dy = -fw.R; dy <= fw.R; ++dy)
            for (int dx = -fw.R; dx <= fw.R; ++dx) {
                const int d2 = dx * dx + dy * dy + dz * dz;
                if (d2 <= 12) wsum += fw.w[d2];
            }
    fw.inv_wsum = 1.0 / wsum;
    return fw;
}

inline void level_sizes(int n, std::vector<int>& sizes) {
    sizes.clear();
    sizes.push_back(n);
    while (sizes.back() % 2 == 0 && sizes.back() / 2 >= 4) sizes.push_back(sizes.back() / 2);
}

// R: PCG vectors and design fields.  S: V-cycle storage.
template <class R, class S>
class Solver : public SolverBase {
  public:
    using C = typename St<R>::C;
    int n = 0;
    size_t N = 0;
    int nlev = 0;
    int sz[kMaxLevels];
    size_t Nl[kMaxLevels];
    int sm_count = 0, max_blocks = 0;
    long long nl_ = 0;   // kernel launches issued (for the step report)

    // fine fields
    R *rho = nullptr, *rho_f = nullptr, *kf = nullptr, *s_f = nullptr, *s = nullptr;
    // MMA (optimizer = OTM_OPT_MMA): the two previous iterates and the asymptotes
    R *mx1 = nullptr, *mx2 = nullptr, *mL = nullptr, *mU = nullptr;
    MmaP mp_{};
    bool use_mma() const { return prm.optimizer == OTM_OPT_MMA; }
    R *f = nullptr, *x = nullptr, *xl = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;
    S *z = nullptr, *res0 = nullptr, *k_vc = nullptr;
    // coarse levels 1..nlev-1 (level 0 uses z / r / res0 / k_vc)
    S *Tl[kMaxLevels] = {}, *Fl[kMaxLevels] = {}, *Rl[kMaxLevels] = {}, *Al[kMaxLevels] = {};
    S *T2l[kMaxLevels] = {}, *Dl[kMaxLevels] = {};   // Chebyshev smoother: second field buffer, direction
    float* lam_d = nullptr;                          // per-level Gershgorin bounds of D^-1 A
    bool cheb_ = false;                              // coarse levels smoothed by Chebyshev (coarse_smoother = 1)
    C *Kel[kMaxLevels] = {};
    C *Bs_d = nullptr, *Minv = nullptr;
    double* Wd = nullptr;
    // reductions and scalars
    double* partials = nullptr;
    unsigned int* counter = nullptr;
    double* partials2 = nullptr;       // reductions of the graphs' second branch
    unsigned int* counter2 = nullptr;
    PcgScalars* ps = nullptr;
    DesignScalars* ds = nullptr;
    PcgScalars* ps_h = nullptr;
    DesignScalars* ds_h = nullptr;
    float* stage_f = nullptr;   // float staging for host/device field copies of R != float

    FilterW fw;
    SimpP sp;
    OcP op;
    bool have_prev = false;
    int iteration = 0;
    // learned warm start (OTM_WS_LEARNED with an attached network)
    otm_unet* predictor = nullptr;
    double pred_scale = 1.0;
    float* ynet[2] = {};
    int ycur = 0;
    bool have_y = false;
    R *xc_net = nullptr, *xc_delta = nullptr;
    PcgScalars* ps_c = nullptr;
    WsState* ws = nullptr;
    WsState* ws_h = nullptr;
    // back-off: after a prediction that no load case used, the next
    // ws_period - 1 iterations skip the predictor (ws_period doubles up to
    // kWsMaxPeriod); a prediction that is used resets it to 1
    static constexpr int kWsMaxPeriod = 64;
    int ws_period = 1, ws_wait = 0;
    int y_iter = -2;   // design iteration of the prediction held in ynet[ycur ^ 1]
    bool ws_had_prev = false, ws_had_delta = false;   // candidates scored by the last prediction
    GovState gov_init;
    cudaEvent_t ev[8] = {};

    ~Solver() override { release(); }

    void release() {
        if (gx_first) cudaGraphExecDestroy(gx_first);
        if (gx_pass) cudaGraphExecDestroy(gx_pass);
        if (gx_tail) cudaGraphExecDestroy(gx_tail);
        if (cap2) cudaStreamDestroy(cap2);
        if (side) cudaStreamDestroy(side);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (ev_fork2) cudaEventDestroy(ev_fork2);
        if (ev_join2) cudaEventDestroy(ev_join2);
        if (gx_setup) cudaGraphExecDestroy(gx_setup);
        if (gx_solve0) cudaGraphExecDestroy(gx_solve0);
        void* ptrs[] = {rho, rho_f, kf, s_f, s, rho_save, mx1, mx2, mL, mU, f, x, xl, r, p, q, z, res0, Bs_d, Minv, Wd,
                        partials, counter, partials2, counter2, ps, ds, stage_f, ynet[0], ynet[1], xc_net, xc_delta, ps_c, ws, lam_d};
        for (void* ptr : ptrs)
            if (ptr) cudaFree(ptr);
        if (k_vc && (void*)k_vc != (void*)kf) cudaFree(k_vc);
        for (int l = 0; l < kMaxLevels; ++l) {
            if (Tl[l]) cudaFree(Tl[l]);
            if (Fl[l]) cudaFree(Fl[l]);
            if (Rl[l]) cudaFree(Rl[l]);
            if (T2l[l]) cudaFree(T2l[l]);
            if (Dl[l]) cudaFree(Dl[l]);
            if (Al[l]) cudaFree(Al[l]);
            if (Kel[l]) cudaFree(Kel[l]);
        }
        if (ps_h) cudaFreeHost(ps_h);
        if (ws_h) cudaFreeHost(ws_h);
        if (ds_h) cudaFreeHost(ds_h);
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        if (own_stream && stream) cudaStreamDestroy(stream);
        rho = nullptr;
    }

    RedBuf rbuf() const { return RedBuf{partials, counter, max_blocks}; }
    RedBuf rbuf2() const { return RedBuf{partials2, counter2, max_blocks}; }
    RowLaunch rl(int nx, int nrows, int thr = 256) const { return row_launch(nx, nrows, max_blocks, thr); }
    int tz_ = 0;   // z-planes per CTA of the tiled fine stencil (0: gather kernel)
    // First level of the cluster-run tail of the V-cycle: the first level >= 1
    // with at most kClusterMaxN nodes per side (L + 1 when the hierarchy has
    // a single level).  OTM_NO_CLUSTER=1 disables it.
    bool use_cluster = true;
    int cluster_maxn = kClusterMaxN;   // OTM_CLUSTER_MAXN overrides
    int cl_ctas_ = kClusterCTAs;       // CTAs of the coarse-level cluster
    bool cl16_ok_ = false;             // a 16-CTA cluster is schedulable here
    bool maxn_fixed_ = false, ctas_fixed_ = false;   // set by OTM_CLUSTER_MAXN / OTM_CLUSTER_CTAS
    bool autotune_on_ = true;          // OTM_AUTOTUNE=0 disables the measured choice
    bool tuned_ = false;
    int autotuned_ = 0;
    double tune_us_[4] = {0, 0, 0, 0};
    double gs_tune_us_[3] = {0, 0, 0};   // V-cycle us of the group pass at ring depths 4, 5, 6
    int cluster_lc() const {
        const int L = nlev - 1;
        if (!use_cluster || nlev < 2) return L + 1;
        for (int l = 1; l <= L; ++l)
            if (sz[l] <= cluster_maxn) return l;
        return L;
    }
    // First level of the cluster kernel's shared-memory tail (CTA 0 runs
    // levels lb..L with shared-memory fields): the first cluster level with
    // at most tail_maxn nodes per side whose tail fits the shared-memory
    // budget; L + 1 when none (or no cluster).  OTM_TAIL_MAXN overrides
    // tail_maxn (0 disables the tail).
    int tail_maxn = 8;
    static constexpr size_t kTailSmemBudget = 200 * 1024;
    int tail_lb() const {
        const int L = nlev - 1;
        const int lc = cluster_lc();
        if (lc > L || tail_maxn <= 0) return L + 1;
        int szs[kMaxLevelsDev] = {};
        for (int l = 0; l <= L; ++l) szs[l] = sz[l];
        const int mv = minv_smem_bytes(L) > 0 ? 1 : 0;
        for (int l = lc; l <= L; ++l)
            if (sz[l] <= tail_maxn && tail_layout<S, C>(l, L, szs, mv).total <= kTailSmemBudget) return l;
        return L + 1;
    }
    size_t cluster_smem_base() const {
        const int L = nlev - 1;
        const int lb = tail_lb();
        if (lb > L) return minv_smem_bytes(L);
        int szs[kMaxLevelsDev] = {};
        for (int l = 0; l <= L; ++l) szs[l] = sz[l];
        return tail_layout<S, C>(lb, L, szs, minv_smem_bytes(L) > 0 ? 1 : 0).total;
    }
    // The one cluster-wide level above the tail in the CTAs' shared memory
    // (Gauss-Seidel smoothing only; OTM_CLUSTER_DSM=0 keeps it in global
    // memory): its index, or -1 when that form does not apply.
    bool dsm_on_ = true;
    int dsm_level() const {
        const int L = nlev - 1;
        const int lc = cluster_lc();
        if (!dsm_on_ || cheb_ || lc > L || tail_lb() != lc + 1) return -1;
        return lc;
    }
    static size_t al16(size_t b) { return (b + 15) / 16 * 16; }
    // per-CTA bytes of that level with G CTAs: stencil rows, right-hand side,
    // field and residual of 8 ceil(h^3 / G) slots
    size_t dsm_bytes(int l, int G) const {
        const size_t h = (size_t)sz[l] / 2, slots = 8 * ((h * h * h + G - 1) / G);
        return al16(slots * CL<S>::AW * sizeof(S)) + 3 * al16(slots * 4 * sizeof(S));
    }
    // dynamic shared memory of the cluster kernel: the tail, then (sized for
    // 8 CTAs, the larger share, so either cluster size fits) the level above it
    size_t cluster_smem_bytes() const {
        const size_t base = cluster_smem_base();
        const int dl = dsm_level();
        return dl < 0 ? base : al16(base) + dsm_bytes(dl, 8);
    }
    size_t minv_smem_bytes(int l) const {
        const size_t q = Nl[l] - 1;
        // staged inverse; with the kernel's static arrays this stays within 48 KB
        return q * q * sizeof(C) <= 24 * 1024 ? q * q * sizeof(C) : 0;
    }
    int tiled_grid() const { return (n / kTX) * (n / kTY) * (n / tz_); }
    // TMA-staged fine stencil (FP32 PCG fields, 32 | n or 64 | n for BF16
    // storage): the PCG product q = K p with p . q, and the V-cycle's
    // residual f - K T; grid 0 when the form is not used
    TmaLaunch tma_pcg_, tma_vc_, tma_head_;
    TmaStencilMaps maps_pcg_, maps_vc_, maps_head_;
    void launch_tma_pcg(const RedBuf& rb) {
        if constexpr (std::is_same<R, float>::value)
            launch_pdl_smem(tma_kernel<0, true, float, float, float, FinAlpha>(n), tma_pcg_.grid, tma_pcg_.threads,
                            tma_pcg_.smem, stream, maps_pcg_, n, tma_pcg_.ty, tma_pcg_.m, tma_pcg_.stages, (float*)q, &ps->dev_err, rb,
                            FinAlpha{ps}, pdl_early());
    }
    void launch_tma_vc() {
        if constexpr (std::is_same<R, float>::value && !std::is_same<S, double>::value)
            launch_pdl_smem(tma_kernel<1, false, S, float, S, FinNone>(n), tma_vc_.grid, tma_vc_.threads, tma_vc_.smem,
                            stream, maps_vc_, n, tma_vc_.ty, tma_vc_.m, tma_vc_.stages, res0, &ps->dev_err, rbuf(), FinNone{}, pdl_early());
    }
    // First pass of a solve (FP32 PCG fields): the iterate starts from its
    // high part alone (lo cleared), so the initial residual f - K hi is the
    // stencil's residual form with the ||r||^2 and ||f||^2 reductions; a
    // refinement pass keeps the pair form (lo then carries the solve's
    // accumulated updates).
    bool head_tma(int use_true) const { return !use_true && tma_head_.grid > 0; }
    otm_status clear_lo() {
        if (xl) OTM_CU(cudaMemsetAsync(xl, 0, 3 * N * sizeof(R), stream));
        return OTM_OK;
    }
    void launch_tma_head() {
        if constexpr (std::is_same<R, float>::value)
            launch_pdl_smem(tma_kernel<1, true, float, float, float, FinInit>(n), tma_head_.grid, tma_head_.threads,
                            tma_head_.smem, stream, maps_head_, n, tma_head_.ty, tma_head_.m, tma_head_.stages,
                            (float*)r, &ps->dev_err, rbuf(), FinInit{ps, 0}, pdl_early());
    }
    size_t inv_smem_ = 0;    // dynamic shared memory of the coarsest inverse
    int inv_use_smem_ = 0;   // its working matrix in shared memory
    // warp-row kernels on the finest grid (FP32 / mixed paths, 128 | n)
    bool wr_ = false;
    int wr_grid(long long warps) const {
        long long b = (warps + 7) / 8;
        if (b > max_blocks) b = max_blocks;
        return (int)(b < 1 ? 1 : b);
    }
    int grid(size_t work, int threads = 256) const {
        size_t b = (work + threads - 1) / threads;
        if (b < 1) b = 1;
        if (b > (size_t)max_blocks) b = max_blocks;
        return (int)b;
    }

    // Host-side fault injection for the failure tests: OTM_FAIL_ALLOC_AT=k
    // makes the k-th device allocation of a context (1-based) report an
    // allocation failure without allocating; the context then unwinds as
    // on a real cudaMalloc failure.
    int alloc_seq_ = 0, fail_alloc_at_ = 0;
    template <class T>
    otm_status alloc(T*& ptr, size_t count) {
        if (++alloc_seq_ == fail_alloc_at_) {
            err = "cudaMalloc: injected allocation failure (OTM_FAIL_ALLOC_AT)";
            return OTM_ENOMEM;
        }
        OTM_CU(cudaMalloc((void**)&ptr, count * sizeof(T) + 16));
        OTM_CU(cudaMemsetAsync(ptr, 0, count * sizeof(T) + 16, stream));
        return OTM_OK;
    }

    // The shared-memory opt-in is one attribute of the kernel per device and
    // process, shared by every context of this precision: only ever raise it
    // (a smaller context created later must not lower it under a larger
    // one).  This Solver instantiation lives in one translation unit, so the
    // static below belongs to the kernel stub its launches go through.
    otm_status raise_cluster_smem(size_t bytes) {
        static std::mutex m;
        static size_t granted[64] = {};
        std::lock_guard<std::mutex> lock(m);
        const int d = device >= 0 && device < 64 ? device : 0;
        if (bytes <= granted[d]) return OTM_OK;
        OTM_CU(cudaFuncSetAttribute(k_coarse_cluster<S, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        granted[d] = bytes;
        return OTM_OK;
    }

    otm_status raise_invert_smem(size_t bytes) {
        static std::mutex m;
        static size_t granted[64] = {};
        std::lock_guard<std::mutex> lock(m);
        const int d = device >= 0 && device < 64 ? device : 0;
        if (bytes <= granted[d]) return OTM_OK;
        OTM_CU(cudaFuncSetAttribute(k_coarse_invert<S, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)bytes));
        granted[d] = bytes;
        return OTM_OK;
    }

    otm_status init(const otm_params& pin) override {
        prm = pin;
        if (const char* fa = getenv("OTM_FAIL_ALLOC_AT")) fail_alloc_at_ = atoi(fa);
        n = pin.n;
        N = (size_t)n * n * n;
        std::vector<int> sizes;
        level_sizes(n, sizes);
        nlev = (int)sizes.size();
        for (int l = 0; l < nlev; ++l) {
            sz[l] = sizes[l];
            Nl[l] = (size_t)sizes[l] * sizes[l] * sizes[l];
        }
        if (pin.device >= 0) OTM_CU(cudaSetDevice(pin.device));
        OTM_CU(cudaGetDevice(&device));
        OTM_CU(cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, device));
        max_blocks = sm_count * 8;
        tz_ = stencil_choice() != 2 ? tiled_tz(pin.n, sm_count, max_blocks) : 0;
        wr_ = warprow_ok(pin.n) && std::is_same<R, float>::value;
        // Fine Gauss-Seidel grid: where the fields outgrow L2 (n >= 256) the
        // pass runs best as two full waves of resident blocks (256^3 design
        // iteration: 15.66 ms FP32 and 14.98 ms with the BF16 V-cycle, against
        // 16.06 and 15.39 ms with the 8-per-SM grid's 2.67 waves; one wave
        // 15.67 ms).  At 128^3 it keeps 8 blocks per SM.
        gs_cap_ = gs_grid_cap();
        if (gs_cap_ == 0 && pin.n >= 256) {
            const dim3 blk = rl(pin.n, (pin.n / 2) * (pin.n / 2)).block;
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gs_fine<false, S, R, S>, (int)(blk.x * blk.y),
                                                              0) != cudaSuccess || per_sm < 1)
                per_sm = 1;
            gs_cap_ = 2 * per_sm * sm_count;
        }
        if (pin.stream) {
            stream = (cudaStream_t)pin.stream;
        } else {
            OTM_CU(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
            own_stream = true;
        }
        for (auto& e : ev) OTM_CU(cudaEventCreate(&e));
        OTM_CU(cudaStreamCreateWithFlags(&cap2, cudaStreamNonBlocking));
        OTM_CU(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
        OTM_CU(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
        OTM_CU(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
        OTM_CU(cudaEventCreateWithFlags(&ev_fork2, cudaEventDisableTiming));
        OTM_CU(cudaEventCreateWithFlags(&ev_join2, cudaEventDisableTiming));
        {
            const char* ng = getenv("OTM_NO_GRAPH");
            use_graphs = !(ng && ng[0] == '1');
            const char* nc = getenv("OTM_NO_CLUSTER");
            use_cluster = !(nc && nc[0] == '1');
            const char* cm = getenv("OTM_CLUSTER_MAXN");
            if (cm) {
                cluster_maxn = atoi(cm);
                maxn_fixed_ = true;
            }
            const char* stv = getenv("OTM_SPEC_TENSOR");
            spec_tensor_ = !(stv && stv[0] == '0');
            const char* at = getenv("OTM_AUTOTUNE");
            autotune_on_ = !(at && at[0] == '0');
            const char* tm = getenv("OTM_TAIL_MAXN");
            if (tm) tail_maxn = atoi(tm);
        }

        OTM_TRY(alloc(rho, N));
        OTM_TRY(alloc(rho_f, N));
        OTM_TRY(alloc(kf, N));
        OTM_TRY(alloc(s_f, N));
        OTM_TRY(alloc(s, N));
        OTM_TRY(alloc(rho_save, N));
        if (pin.optimizer == OTM_OPT_MMA) {
            OTM_TRY(alloc(mx1, N));
            OTM_TRY(alloc(mx2, N));
            OTM_TRY(alloc(mL, N));
            OTM_TRY(alloc(mU, N));
            mp_ = MmaP{0.0, 1.0, pin.mma_move, pin.mma_c, pin.mma_d, 1.0 / (double)N, pin.mma_eps};
        }
        OTM_TRY(alloc(f, 3 * N));
        OTM_TRY(alloc(x, 3 * N));
        if (!std::is_same<C, double>::value) OTM_TRY(alloc(xl, 3 * N));
        OTM_TRY(alloc(r, 3 * N));
        OTM_TRY(alloc(p, 3 * N));
        OTM_TRY(alloc(q, 3 * N));
        OTM_TRY(alloc(z, 3 * N));
        OTM_TRY(alloc(res0, 3 * N));
        OTM_TRY(alloc(stage_f, 3 * N));
        if (std::is_same<R, S>::value) k_vc = (S*)kf;
        else OTM_TRY(alloc(k_vc, N));
        if constexpr (std::is_same<R, float>::value && !std::is_same<S, double>::value) {
            if (stencil_choice() == 0) {
                // tensor maps of the fixed fine buffers, encoded once per context
                if (tma_launch_shape<0, true, float, float, float, FinAlpha>(tma_pcg_, n, sm_count, max_blocks) &&
                    !tma_make_maps<float, float>(maps_pcg_, n, kf, p, nullptr))
                    tma_pcg_.grid = 0;
                if (tma_launch_shape<1, false, S, float, S, FinNone>(tma_vc_, n, sm_count, max_blocks) &&
                    !tma_make_maps<S, float>(maps_vc_, n, k_vc, z, r))
                    tma_vc_.grid = 0;
                // OTM_HEAD=pair: the pair form for every pass (for comparisons)
                const char* he = getenv("OTM_HEAD");
                const bool pair_head = he && he[0] == 'p';
                if (xl && !pair_head &&
                    tma_launch_shape<1, true, float, float, float, FinInit>(tma_head_, n, sm_count, max_blocks) &&
                    !tma_make_maps<float, float>(maps_head_, n, kf, x, f))
                    tma_head_.grid = 0;
                cudaGetLastError();   // a refused shape leaves the older forms in place
            }
            if (gs_choice() == 0) {
                if (gs_tma_launch_shape<S, float>(tma_gs_, n, sm_count) &&
                    !gs_tma_make_maps<S, float>(maps_gs_, n, k_vc, z, r))
                    tma_gs_.grid = 0;
                cudaGetLastError();
            }
        }
        for (int l = 1; l < nlev; ++l) {
            // coarse levels are node-major: fields [N][4], stencil [N][CL<S>::AW]
            OTM_TRY(alloc(Tl[l], 4 * Nl[l]));
            OTM_TRY(alloc(Fl[l], 4 * Nl[l]));
            OTM_TRY(alloc(Rl[l], 4 * Nl[l]));
            if (pin.coarse_smoother == 1) {
                OTM_TRY(alloc(T2l[l], 4 * Nl[l]));
                OTM_TRY(alloc(Dl[l], 4 * Nl[l]));
            }
            OTM_TRY(alloc(Al[l], (size_t)CL<S>::AW * Nl[l]));
            if (l >= 2) OTM_TRY(alloc(Kel[l], 64 * Nl[l]));   // element-major [N_l][64]; level 1 is never stored
        }
        if (nlev == 1) OTM_TRY(alloc(Al[0], (size_t)CL<S>::AW * Nl[0]));
        const size_t m = Nl[nlev - 1];
        OTM_TRY(alloc(Wd, (size_t)inv_ld((int)m - 1) * inv_ld((int)m - 1)));   // row stride padded to 4
        OTM_TRY(alloc(Minv, (m - 1) * (m - 1)));
        {
            // the coarsest inverse keeps its working matrix in shared memory
            // when that fits the device's opt-in limit
            const size_t qd = m - 1;
            int optin = 0;
            OTM_CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
            cudaFuncAttributes fa;
            OTM_CU(cudaFuncGetAttributes(&fa, k_coarse_invert<S, C>));
            const size_t full = invert_smem_bytes((int)qd, (int)sizeof(C), true);
            inv_use_smem_ = fa.sharedSizeBytes + full <= (size_t)optin ? 1 : 0;
            inv_smem_ = inv_use_smem_ ? full : invert_smem_bytes((int)qd, (int)sizeof(C), false);
            OTM_TRY(raise_invert_smem(inv_smem_));
        }
        std::vector<double> Ps, Bs;
        build_ps(Ps, Bs);
        std::vector<C> Bsc(Bs.begin(), Bs.end());
        OTM_TRY(alloc(Bs_d, 8 * 64));
        OTM_CU(cudaMemcpyAsync(Bs_d, Bsc.data(), 8 * 64 * sizeof(C), cudaMemcpyHostToDevice, stream));
        {
            // Opt in to exactly the dynamic shared memory the cluster kernel
            // will be launched with (static + dynamic may exceed the default
            // 48 KB); drop the shared-memory tail if the device cannot hold it.
            cudaFuncAttributes fa;
            OTM_CU(cudaFuncGetAttributes(&fa, k_coarse_cluster<S, C>));
            int optin = 0;
            OTM_CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
            if (const char* e = getenv("OTM_CLUSTER_DSM")) dsm_on_ = e[0] != '0';
            if (fa.sharedSizeBytes + cluster_smem_bytes() > (size_t)optin) dsm_on_ = false;
            if (fa.sharedSizeBytes + cluster_smem_bytes() > (size_t)optin) tail_maxn = 0;
            const size_t cs = cluster_smem_bytes();
            if (fa.sharedSizeBytes + cs > (size_t)optin) {
                err = "the coarse-level kernel does not fit the device's shared memory";
                return OTM_ECUDA;
            }
            OTM_TRY(raise_cluster_smem(cs));
            // cluster size: 16 CTAs (non-portable) when the device can co-schedule
            // them with this shared memory, else the portable 8; OTM_CLUSTER_CTAS
            // (8 or 16) overrides
            int want = 16;
            if (const char* e = getenv("OTM_CLUSTER_CTAS")) {
                want = atoi(e) == 8 ? 8 : 16;
                ctas_fixed_ = true;
            }
            cl_ctas_ = kClusterCTAs;
            cl16_ok_ = false;
            if (cudaFuncSetAttribute(k_coarse_cluster<S, C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                cudaSuccess) {
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(16, 1, 1);
                cfg.blockDim = dim3(kClusterThreads, 1, 1);
                cfg.dynamicSmemBytes = cs;
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeClusterDimension;
                at[0].val.clusterDim.x = 16;
                at[0].val.clusterDim.y = 1;
                at[0].val.clusterDim.z = 1;
                cfg.attrs = at;
                cfg.numAttrs = 1;
                int clusters = 0;
                if (cudaOccupancyMaxActiveClusters(&clusters, k_coarse_cluster<S, C>, &cfg) == cudaSuccess &&
                    clusters >= 1)
                    cl16_ok_ = true;
                if (cl16_ok_ && want == 16) cl_ctas_ = 16;
            }
            cudaGetLastError();
        }
        cheb_ = pin.coarse_smoother == 1 && nlev > 1;
        OTM_TRY(alloc(lam_d, kMaxLevels));
        OTM_TRY(alloc(partials, (size_t)max_blocks * kRedMaxVals));
        OTM_TRY(alloc(counter, 4));
        OTM_TRY(alloc(partials2, (size_t)max_blocks * kRedMaxVals));
        OTM_TRY(alloc(counter2, 4));
        OTM_TRY(alloc(ps, 1));
        OTM_TRY(alloc(ps_c, 1));
        OTM_TRY(alloc(ds, 1));
        OTM_CU(cudaMallocHost((void**)&ps_h, sizeof(PcgScalars)));
        OTM_CU(cudaMallocHost((void**)&ds_h, sizeof(DesignScalars)));

        fw = with_f32(make_filter(pin.rmin));
        sp.penal = pin.penal;
        sp.k_solid = pin.k_solid;
        sp.k_void = pin.k_void;
        sp.cubic = pin.penal == 3.0;
        sp = with_f32(sp, N);
        op.move = pin.move;
        op.damp = pin.damp;
        op.rho_min = pin.rho_min;
        op.half = pin.damp == 0.5;
        op = with_f32(op);

        memset(ds_h, 0, sizeof(DesignScalars));
        gov_init.df = 1.0;
        gov_init.vstar = 1.0;
        gov_init.g_prev = 1.0;
        gov_init.gap = 0.0;
        gov_init.count = 0;
        ds_h->gov = gov_init;
        ds_h->govp.bound = pin.gov_bound;
        ds_h->govp.small_rel = pin.gov_small_rel;
        ds_h->govp.vol_tol = pin.gov_vol_tol;
        ds_h->governor_on = pin.governor;
        ds_h->objective = pin.objective;
        for (int c = 0; c < 6; ++c) ds_h->target[c] = pin.kappa_target[c];
        ds_h->vstar = pin.optimizer == OTM_OPT_MMA ? 0.0 : (pin.governor ? 1.0 : pin.fixed_volume);
        OTM_CU(cudaMemcpyAsync(ds, ds_h, sizeof(DesignScalars), cudaMemcpyHostToDevice, stream));
        memset(ps_h, 0, sizeof(PcgScalars));
        ps_h->tol2 = pin.cg_tol * pin.cg_tol;
        ps_h->flexible = std::is_same<R, S>::value ? 0 : 1;
        OTM_CU(cudaMemcpyAsync(ps, ps_h, sizeof(PcgScalars), cudaMemcpyHostToDevice, stream));
        // uniform initial density
        std::vector<float> h(N, (float)pin.volfrac);
        OTM_TRY(set_density(h.data(), false));
        OTM_CU(cudaStreamSynchronize(stream));
        return OTM_OK;
    }

    // ---------------------------------------------------------- conversions
    // float (host or device) -> R field, through the float staging buffer.
    otm_status to_R(const float* src, bool on_device, R* dst, size_t count, bool clamp01) {
        OTM_CU(cudaMemcpyAsync(stage_f, src, count * sizeof(float),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, stream));
        ++nl_;
        launch_pdl(k_convert<float, R>, grid(count), 256, stream, count, stage_f, dst, clamp01 ? 1 : 0);
        OTM_LAUNCH();
        OTM_CU(cudaStreamSynchronize(stream));
        return OTM_OK;
    }
    // R field -> float (host or device).
    otm_status from_R(const R* src, float* dst, size_t count, bool on_device) {
        ++nl_;
        launch_pdl(k_convert<R, float>, grid(count), 256, stream, count, src, stage_f, 0);
        OTM_LAUNCH();
        OTM_CU(cudaMemcpyAsync(dst, stage_f, count * sizeof(float),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream));
        OTM_CU(cudaStreamSynchronize(stream));
        return OTM_OK;
    }

    otm_status set_density(const float* h, bool on_device) override {
        OTM_TRY(to_R(h, on_device, rho, N, true));
        have_prev = false;
        iteration = 0;
        // reset Alg. 1 state
        OTM_CU(cudaMemcpyAsync(&ds->gov, &gov_init, sizeof(GovState), cudaMemcpyHostToDevice, stream));
        const double v0 = use_mma() ? 0.0 : (prm.governor ? 1.0 : prm.fixed_volume);
        OTM_CU(cudaMemcpyAsync(&ds->vstar, &v0, sizeof(double), cudaMemcpyHostToDevice, stream));
        if (use_mma()) {
            // MMA restarts: iteration 0 (the history is read only from iteration 2 on)
            const int k0 = 0;
            OTM_CU(cudaMemcpyAsync(&ds->mma_k, &k0, sizeof(int), cudaMemcpyHostToDevice, stream));
            OTM_CU(cudaMemcpyAsync(mx1, rho, N * sizeof(R), cudaMemcpyDeviceToDevice, stream));
            OTM_CU(cudaMemcpyAsync(mx2, rho, N * sizeof(R), cudaMemcpyDeviceToDevice, stream));
        }
        OTM_CU(cudaStreamSynchronize(stream));
        return OTM_OK;
    }

    otm_status get_density(float* out, bool on_device) override {
        OTM_TRY(from_R(rho, out, N, on_device));
        return OTM_OK;
    }

    otm_status get_field(int which, float* out, size_t count, bool on_device) override {
        const R* src = nullptr;
        size_t len = N;
        switch (which) {
            case OTM_FIELD_RHO: src = rho; break;
            case OTM_FIELD_RHO_FILT: src = rho_f; break;
            case OTM_FIELD_K: src = kf; break;
            case OTM_FIELD_CHI:
                if (count != 3 * N) {
                    err = "otm_get_field: count does not match the field length";
                    return OTM_EINVAL;
                }
                ++nl_;
                launch_pdl(k_join<R, float>, grid(3 * N), 256, stream, 3 * N, x, xl, stage_f);
                // the solutions are defined up to a constant: report the zero-mean one
                nl_ += 2;
                launch_pdl(k_sum3<float>, grid(N), 256, stream, N, (const float*)stage_f, rbuf(),
                           FinMean{ps_c, 1.0 / (double)N});
                launch_pdl(k_sub_mean<float>, grid(N), 256, stream, N, stage_f, (const PcgScalars*)ps_c);
                OTM_LAUNCH();
                OTM_CU(cudaMemcpyAsync(out, stage_f, 3 * N * sizeof(float),
                                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream));
                OTM_CU(cudaStreamSynchronize(stream));
                return OTM_OK;
            case OTM_FIELD_LOAD: src = f; len = 3 * N; break;
            case OTM_FIELD_SENS: src = s; break;
            default: err = "otm_get_field: unknown field"; return OTM_EINVAL;
        }
        if (count != len) {
            err = "otm_get_field: count does not match the field length";
            return OTM_EINVAL;
        }
        return from_R(src, out, len, on_device);
    }

    // --------------------------------------------------------------- stages
    otm_status filter_simp() {
        ++nl_;
        launch_filter<R, true>(rl(n, n * n), stream, n, fw, 1, rho, rho_f, kf, sp, rbuf(), FinFilter{ds});
        OTM_LAUNCH();
        return OTM_OK;
    }

    otm_status build_hierarchy() {
        OTM_TRY(fine_loads());
        return coarse_hierarchy();
    }
    // macro loads (zero-mean) and the V-cycle's copy of k: fine-grid work
    otm_status fine_loads() {
        ++nl_;
        launch_pdl(k_macro_load<R, R>, OTM_ROWS_CFG(rl(n, n * n)), stream, n, kf, f);
        ++nl_;
        launch_pdl(k_sum3<R>, grid(N), 256, stream, N, f, rbuf(), FinMean{ps, 1.0 / (double)N});
        ++nl_;
        launch_pdl(k_sub_mean<R>, grid(N), 256, stream, N, f, ps);
        OTM_LAUNCH();
        if (!std::is_same<R, S>::value) {
            ++nl_;
            launch_pdl(k_convert<R, S>, grid(N), 256, stream, N, kf, k_vc, 0);
            OTM_LAUNCH();
        }
        return OTM_OK;
    }
    // Galerkin stencils of every level and the coarsest inverse (from k only)
    otm_status coarse_hierarchy() {
        if (nlev == 1) {
            ++nl_;
            launch_pdl(k_stencil_from_k<R, C, S>, OTM_ROWS_CFG(rl(n, n * n, 128)), stream, n, kf, Al[0]);
            OTM_LAUNCH();
        } else {
            ++nl_;
            launch_pdl(k_stencil1_from_k<R, C, S>, (int)((Nl[1] + 127) / 128), 128, stream, sz[1], kf, Bs_d, Al[1]);
            OTM_LAUNCH();
            for (int l = 1; l + 1 < nlev; ++l) {
                ++nl_;
                const long long warps = (long long)Nl[l + 1];
                const int cg = (int)std::min<long long>((warps + 7) / 8, (long long)sm_count * 16);
                if (l == 1)
                    launch_pdl(k_elem_coarsen<C, true, R>, cg, 256, stream, sz[l + 1], (const C*)nullptr, kf,
                               Bs_d, Kel[l + 1]);
                else
                    launch_pdl(k_elem_coarsen<C, false, R>, cg, 256, stream, sz[l + 1], (const C*)Kel[l], kf,
                               Bs_d, Kel[l + 1]);
                OTM_LAUNCH();
                ++nl_;
                launch_pdl(k_stencil_from_elem<C, S>, OTM_ROWS_CFG(rl(sz[l + 1], sz[l + 1] * sz[l + 1], 128)), stream, sz[l + 1], Kel[l + 1], Al[l + 1]);
                OTM_LAUNCH();
            }
        }
        const int L = nlev - 1;
        if (cheb_) {
            OTM_CU(cudaMemsetAsync(lam_d, 0, kMaxLevels * sizeof(float), stream));
            for (int l = 1; l < L; ++l) {
                ++nl_;
                launch_pdl(k_gershgorin<S>, grid(Nl[l]), 256, stream, sz[l], (const S*)Al[l], lam_d + l);
            }
            OTM_LAUNCH();
        }
        ++nl_;
        {
            launch_pdl_smem(k_coarse_invert<S, C>, 1, kInvThreads, inv_smem_, stream, sz[L], Al[L], (C*)Wd, Minv,
                            inv_use_smem_);
        }
        OTM_LAUNCH();
        return OTM_OK;
    }

    // z = V(r): one V-cycle of Alg. 3 with a forward 8-colour Gauss-Seidel
    // sweep before and the reverse sweep after the coarse correction.
    // One Chebyshev smoothing of stencil level l (kChebDeg launches): from
    // zero into T2 (pre-smoothing), or from T2 back into T (post-smoothing).
    void cheb_smooth(int l, bool from_zero) {
        for (int k = 0; k < kChebDeg; ++k) {
            const bool to_t2 = from_zero ? (k % 2 == 0) : (k % 2 == 1);
            const S* Tin = to_t2 ? Tl[l] : T2l[l];
            S* Tout = to_t2 ? T2l[l] : Tl[l];
            ++nl_;
            if (from_zero && k == 0)
                launch_pdl(k_cheb_stencil<true, S, S, S>, OTM_ROWS_CFG(rl(sz[l], sz[l] * sz[l])), stream, sz[l], k,
                           (const float*)(lam_d + l), (const S*)Al[l], (const S*)Fl[l], Tin, Tout, Dl[l]);
            else
                launch_pdl(k_cheb_stencil<false, S, S, S>, OTM_ROWS_CFG(rl(sz[l], sz[l] * sz[l])), stream, sz[l], k,
                           (const float*)(lam_d + l), (const S*)Al[l], (const S*)Fl[l], Tin, Tout, Dl[l]);
        }
    }

    // One fine-grid Gauss-Seidel group pass.
    // OTM_COARSE_NBR=0: the coarse colour passes read every neighbour after
    // the wait (for comparisons)
    static bool coarse_nbr_early() {
        static const bool on = [] {
            const char* e = getenv("OTM_COARSE_NBR");
            return !(e && e[0] == '0');
        }();
        return on && !std::is_same<S, __nv_bfloat16>::value;
    }
    // One colour pass of a standalone coarse level l; early_f: f was written
    // two or more kernels back, so it may be loaded before the wait on the
    // previous kernel (the stencil always is); prev: the colour the previous
    // kernel relaxed (-1: it wrote every node), whose neighbours are the only
    // ones read after the wait
    // The prefetching form of a colour pass holds a node's 27 couplings and
    // up to 26 neighbours in registers (about 200 per thread), so it runs
    // where its grid fits in one wave of resident blocks; a larger level
    // (the 128^3 level at n = 256: 1024 blocks of 256 threads, one resident
    // per SM) takes the plain form, whose lower register count keeps more
    // blocks resident.  OTM_CGS_PF=1 takes the prefetching form everywhere
    // (for comparisons).  Decided once per level.
    signed char cgs_pf_[kMaxLevels] = {};   // 0 unknown, 1 prefetching, -1 plain
    bool cgs_prefetch(int l, const RowLaunch& cfg) {
        if (cgs_pf_[l] == 0) {
            const char* e = getenv("OTM_CGS_PF");
            bool pf = e && e[0] == '1';
            if (!pf) {
                int per_sm = 0;
                const int thr = cfg.block.x * cfg.block.y * cfg.block.z;
                pf = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gs_stencil_pf<false, S, S, S>, thr, 0) ==
                         cudaSuccess &&
                     per_sm > 0 && (long long)cfg.grid <= (long long)per_sm * sm_count;
                cudaGetLastError();
            }
            cgs_pf_[l] = pf ? 1 : -1;
        }
        return cgs_pf_[l] > 0;
    }
    template <bool ZERO>
    void coarse_gs_pass(int l, int c, int early_f, int prev) {
        const auto cfg = rl(sz[l] / 2, (sz[l] / 2) * (sz[l] / 2), cgs_thr(sz[l]));
        if (pdl_early() && (ZERO || cgs_prefetch(l, cfg)))
            launch_pdl(k_gs_stencil_pf<ZERO, S, S, S>, OTM_ROWS_CFG(cfg), stream, sz[l], c, Al[l], Fl[l], Tl[l],
                       early_f, coarse_nbr_early() ? gs_early_mask(c, prev) : 0u);
        // (BF16 storage: measured slower with the neighbours read early, 2.160
        // against 2.134 ms per 128^3 design iteration; FP32 2.056 against 2.061)
        else
            launch_pdl(k_gs_stencil<ZERO, S, S, S>, OTM_ROWS_CFG(cfg), stream, sz[l], c, Al[l], Fl[l], Tl[l]);
    }
    // TMA-staged fine group pass (FP32 or BF16 storage, f in FP32); grid 0
    // when the gather form runs
    TmaLaunch tma_gs_;
    TmaGsMaps maps_gs_;
    void fine_gs_pass(int gidx) {
        if constexpr (std::is_same<R, float>::value && !std::is_same<S, double>::value) {
            if (tma_gs_.grid > 0) {
                launch_pdl_smem(gs_tma_kernel<S, float>(n), tma_gs_.grid, tma_gs_.threads, tma_gs_.smem, stream,
                                maps_gs_, n, tma_gs_.ty, tma_gs_.m, tma_gs_.stages, gidx, z, &ps->dev_err, pdl_early());
                return;
            }
        }
        launch_pdl(k_gs_fine<false, S, R, S>, gs_grid(), rl(n, (n / 2) * (n / 2)).block, stream, n, gidx, -1, k_vc, r,
                   z);
    }
    int gs_cap_ = 0;   // grid cap of the fine Gauss-Seidel pass, 0: the row-mapped grid
    // Threads per block of a standalone coarse level's colour passes: 256,
    // or 64 where 256-thread blocks would not cover every SM and a colour's
    // row fills whole warps (the 64^3 level at n = 128 and 256: 512 blocks
    // instead of 128).  OTM_CGS_THREADS overrides.
    int cgs_thr(int m) const {
        const char* e = getenv("OTM_CGS_THREADS");
        if (e) {
            const int t = atoi(e);
            return t >= 32 && t <= 256 && t % 32 == 0 ? t : 256;
        }
        return (m / 2) % 32 == 0 && rl(m / 2, (m / 2) * (m / 2)).grid < sm_count ? 64 : 256;
    }
    int gs_grid() const {
        const RowLaunch c = rl(n, (n / 2) * (n / 2));
        return gs_cap_ > 0 && gs_cap_ < c.grid ? gs_cap_ : c.grid;
    }

    otm_status vcycle() {
        const int L = nlev - 1;
        if (nlev == 1) {
            ++nl_;
            launch_pdl_smem(k_coarse_solve<C, R, S, false>, 1, 1024, minv_smem_bytes(0), stream, sz[0], Minv, r, z, minv_smem_bytes(0) > 0 ? 1 : 0);
            OTM_LAUNCH();
            return OTM_OK;
        }
        // level 0, pre-smooth: groups {0,1}, {2,3}, {4,5}, {6,7}
        ++nl_;
        launch_pdl(k_gs_fine<true, S, R, S>, gs_grid(), rl(n, (n / 2) * (n / 2)).block, stream, n, 0, -1, k_vc, r, z);
        for (int gidx = 1; gidx < 4; ++gidx) {
            ++nl_;
            fine_gs_pass(gidx);
        }
        ++nl_;
        if (tma_vc_.grid > 0)
            launch_tma_vc();
        else if (tz_ > 0 && !std::is_same<S, double>::value)
            launch_pdl(k_stencil_tiled<1, false, S, S, R, S, FinNone>, tiled_grid(), dim3(kTX, kTY), stream, n, tz_,
                       k_vc, z, r, res0, rbuf(), FinNone{});
        else
            launch_pdl(k_stencil_apply<1, false, S, S, R, S, FinNone>, OTM_ROWS_CFG(rl(n, n * n)), stream, n, k_vc, z,
                       r, res0, rbuf(), FinNone{});
        ++nl_;
        launch_pdl(k_restrict<S, S, false>, OTM_ROWS_CFG(rl(sz[1], sz[1] * sz[1])), stream, sz[1], res0, Fl[1]);
        OTM_LAUNCH();
        const int lc = cluster_lc();   // levels lc..L run in one cluster launch (lc > L: none)
        const int Lsep = lc <= L ? lc : L;
        for (int l = 1; l < Lsep; ++l) {
            S* Tcur = Tl[l];
            if (cheb_) {
                cheb_smooth(l, true);
                Tcur = T2l[l];
            } else {
                ++nl_;
                coarse_gs_pass<true>(l, 0, 0, -1);   // f: written by the restriction just before
                for (int c = 1; c < 8; ++c) {
                    ++nl_;
                    coarse_gs_pass<false>(l, c, 1, c == 1 ? -1 : c - 1);   // colour 0 (from zero) wrote every node
                }
            }
            ++nl_;
            if (pdl_early())   // stencil and f loaded before the wait on the last pre-smoothing pass
                launch_pdl(k_residual_stencil_pf<S, S, S, S>, OTM_ROWS_CFG(rl(sz[l], sz[l] * sz[l])), stream, sz[l],
                           Al[l], Fl[l], (const S*)Tcur, Rl[l]);
            else
                launch_pdl(k_residual_stencil<S, S, S, S>, OTM_ROWS_CFG(rl(sz[l], sz[l] * sz[l])), stream, sz[l],
                           Al[l], Fl[l], (const S*)Tcur, Rl[l]);
            ++nl_;
            launch_pdl(k_restrict<S, S, true>, OTM_ROWS_CFG(rl(sz[l + 1], sz[l + 1] * sz[l + 1])), stream, sz[l + 1], Rl[l], Fl[l + 1]);
            OTM_LAUNCH();
        }
        if (lc <= L) {
            ClusterArgs<S, C> ca;
            memset(&ca, 0, sizeof(ca));
            ca.lc = lc;
            ca.L = L;
            ca.minv_smem = minv_smem_bytes(L) > 0 ? 1 : 0;
            ca.lb = tail_lb();
            ca.cheb = cheb_ ? 1 : 0;
            ca.lam = lam_d;
            if (ca.lb <= L) {
                int szs[kMaxLevelsDev] = {};
                for (int l = 0; l <= L; ++l) szs[l] = sz[l];
                const TailLayout tl = tail_layout<S, C>(ca.lb, L, szs, ca.minv_smem);
                for (int l = ca.lb; l <= L; ++l) {
                    ca.tT[l] = (unsigned)tl.T[l];
                    ca.tF[l] = (unsigned)tl.F[l];
                    ca.tA[l] = (unsigned)tl.A[l];
                }
                ca.tR = (unsigned)tl.R;
                ca.tMinv = (unsigned)tl.minv;
            }
            for (int l = 0; l <= L; ++l) {
                ca.n[l] = sz[l];
                ca.T[l] = Tl[l];
                ca.F[l] = Fl[l];
                ca.Rr[l] = Rl[l];
                ca.T2[l] = T2l[l];
                ca.D[l] = Dl[l];
                ca.A[l] = Al[l];
            }
            ca.Minv = Minv;
            const int dl = dsm_level();
            if (dl >= 0) {
                const int G = cl_ctas_;
                const size_t h = (size_t)sz[dl] / 2, mg = (h * h * h + G - 1) / G, slots = 8 * mg;
                size_t off = al16(cluster_smem_base());
                ca.dA = (unsigned)off;
                off += al16(slots * CL<S>::AW * sizeof(S));
                ca.dF = (unsigned)off;
                off += al16(slots * 4 * sizeof(S));
                ca.dT = (unsigned)off;
                off += al16(slots * 4 * sizeof(S));
                ca.dR = (unsigned)off;
                ca.dsm = 1;
                ca.dmg = (int)mg;
                ca.dlg = G == 16 ? 4 : 3;
            }
            OTM_TRY(raise_cluster_smem(cluster_smem_bytes()));
            ++nl_;
            const cudaError_t le = launch_cluster_pdl(k_coarse_cluster<S, C>, cl_ctas_, kClusterThreads,
                                                      cluster_smem_bytes(), stream, ca);
            if (le != cudaSuccess) {
                err = std::string("coarse-level cluster launch: ") + cudaGetErrorString(le);
                return OTM_ECUDA;
            }
        } else {
            ++nl_;
            launch_pdl_smem(k_coarse_solve<C, S, S>, 1, 1024, minv_smem_bytes(L), stream, sz[L], Minv, Fl[L], Tl[L],
                            minv_smem_bytes(L) > 0 ? 1 : 0);
        }
        OTM_LAUNCH();
        for (int l = Lsep - 1; l >= 1; --l) {
            ++nl_;
            if (pdl_early())   // the level's own field loaded before the wait on the coarser level
                launch_pdl(k_prolong_add_pf<S, S>, OTM_ROWS_CFG(rl(sz[l], sz[l] * sz[l])), stream, sz[l], Tl[l + 1],
                           cheb_ ? T2l[l] : Tl[l]);
            else
                launch_pdl(k_prolong_add<S, S, true>, OTM_ROWS_CFG(rl(sz[l], sz[l] * sz[l])), stream, sz[l], Tl[l + 1],
                       cheb_ ? T2l[l] : Tl[l]);
            if (cheb_) {
                cheb_smooth(l, false);
            } else {
                for (int c = 7; c >= 0; --c) {
                    ++nl_;
                    coarse_gs_pass<false>(l, c, 1, c == 7 ? -1 : c + 1);   // the prolongation wrote every node
                }
            }
            OTM_LAUNCH();
        }
        ++nl_;
        if (wr_)
            launch_pdl(k_prolong_wr<S, S>, wr_grid((long long)n * n * (n / 128)), 256, stream, n, (const S*)Tl[1], z);
        else
            launch_pdl(k_prolong_add<S, S, false>, OTM_ROWS_CFG(rl(n, n * n)), stream, n, Tl[1], z);
        for (int gidx = 3; gidx >= 0; --gidx) {
            ++nl_;
            fine_gs_pass(gidx);
        }
        OTM_LAUNCH();
        return OTM_OK;
    }

    // ----------------------------------------------------------------------
    // MG-PCG for the three load cases as iterative refinement.  A pass forms
    // r = f - K x from the stored iterate (x held as an FP32 pair hi + lo in
    // the FP32/mixed paths), runs PCG on the correction until the recurrence
    // residual meets cg_tol (or the iteration cap), and then checks
    // ||f - K x|| / ||f|| with error-free element terms.  Further passes
    // start from the checked residual; a pass that does not halve the worst
    // checked residual ends the solve (OTM_ENOCONV).
    //
    // Graph mode (default): the setup and the first pass are one CUDA graph
    // in which the PCG loop is a device-side conditional while node; later
    // passes and the design tail are graphs too, so a design iteration costs
    // two host synchronisations.  OTM_NO_GRAPH=1 selects the host-driven loop.
    // ----------------------------------------------------------------------
    static constexpr int kMaxRestarts = 6;
    int last_iters[3] = {0, 0, 0};
    bool use_graphs = true;
    cudaStream_t cap2 = nullptr;
    cudaStream_t side = nullptr;              // side branch of the captured setup
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_fork2 = nullptr, ev_join2 = nullptr;
    cudaGraphExec_t gx_first = nullptr, gx_pass = nullptr, gx_tail = nullptr;
    cudaGraphExec_t gx_setup = nullptr, gx_solve0 = nullptr;   // learned warm start: setup, then solve
    long long nlg_first = 0, nlg_pass = 0, nlg_body = 0, nlg_tail = 0, nlg_setup = 0, nlg_solve0 = 0;
    R* rho_save = nullptr;

    // one PCG iteration: z = V(r), beta, p, q = K p, alpha, x and r updates
    otm_status enqueue_body() {
        RedBuf rb = rbuf();
        OTM_TRY(vcycle());
        ++nl_;
        if (N % 4 == 0) launch_pdl(k_dot_rz4<R, S>, grid(N / 4), 256, stream, N, r, z, rb, FinBeta{ps});
        else launch_pdl(k_dot_rz<R, S>, grid(N), 256, stream, N, r, z, rb, FinBeta{ps});
        ++nl_;
        if (N % 4 == 0) launch_pdl(k_update_p4<R, S>, grid(N / 4), 256, stream, N, p, z, ps);
        else launch_pdl(k_update_p<R, S>, grid(N), 256, stream, N, p, z, ps);
        ++nl_;
if (tma_pcg_.grid > 0)
            launch_tma_pcg(rb);
        else if (tz_ > 0 && std::is_same<R, float>::value)
            launch_pdl(k_stencil_tiled<0, true, R, R, R, R, FinAlpha>, tiled_grid(), dim3(kTX, kTY), stream, n, tz_,
                       kf, p, (const R*)nullptr, q, rb, FinAlpha{ps});
        else
            launch_pdl(k_stencil_apply<0, true, R, R, R, R, FinAlpha>, OTM_ROWS_CFG(rl(n, n * n)), stream, n, kf, p,
                       (const R*)nullptr, q, rb, FinAlpha{ps});
        ++nl_;
        if (N % 4 == 0)
            launch_pdl(k_update_xr4<R, S>, grid(N / 4), 256, stream, N, x, xl, r, p, q, z, ps, rb, FinResid{ps});
        else
            launch_pdl(k_update_xr<R, S>, grid(N), 256, stream, N, x, xl, r, p, q, z, ps, rb, FinResid{ps});
        OTM_LAUNCH();
        return OTM_OK;
    }
    otm_status enqueue_pass_head(int use_true, bool lo_cleared = false) {
        ++nl_;
        if (head_tma(use_true)) {
            if (!lo_cleared) OTM_TRY(clear_lo());
            launch_tma_head();
        } else if (wr_)
            launch_pdl(k_residual_x2_wr<FinInit>, wr_grid((long long)n * n * (n / 128)), 256, stream, n,
                       (const float*)kf, (const float*)x, (const float*)xl, (const float*)f, (float*)r, rbuf(),
                       FinInit{ps, use_true});
        else
            launch_pdl(k_residual_x2<R, FinInit>, OTM_ROWS_CFG(rl(n, n * n)), stream, n, kf, x, xl, f, r, rbuf(),
                       FinInit{ps, use_true});
        OTM_LAUNCH();
        return OTM_OK;
    }
    // OTM_CHECK_FORM=pair: the warp-row check in its pair form (each
    // neighbour difference rounded once) instead of the element form, for
    // comparisons
    static bool check_pair_form() {
        static const bool pair = [] {
            const char* e = getenv("OTM_CHECK_FORM");
            return e && e[0] == 'p';
        }();
        return pair;
    }
    otm_status enqueue_check() {
        ++nl_;
        if (wr_ && check_pair_form())
            launch_pdl(k_true_residual_wr<FinTrue, false>, wr_grid((long long)n * n * (n / 128)), 256, stream, n,
                       (const float*)kf, (const float*)x, (const float*)xl, (const float*)f, rbuf(), FinTrue{ps});
        else if (wr_)
            launch_pdl(k_true_residual_wr<FinTrue>, wr_grid((long long)n * n * (n / 128)), 256, stream, n,
                       (const float*)kf, (const float*)x, (const float*)xl, (const float*)f, rbuf(), FinTrue{ps});
        else
            launch_pdl(k_true_residual<R>, OTM_ROWS_CFG(rl(n, n * n)), stream, n, kf, x, xl, f, rbuf(), FinTrue{ps});
        OTM_LAUNCH();
        return OTM_OK;
    }
    otm_status enqueue_setup() {
        OTM_TRY(filter_simp());
        OTM_TRY(build_hierarchy());
        ++nl_;
        launch_pdl(k_pcg_reset, 1, 1, stream, ps);
        OTM_LAUNCH();
        return OTM_OK;
    }
    // design tail: tensor, sensitivity, filter transpose, Alg. 1, OC update
    // (MMA on Eq. model2: no governor; the MMA iteration instead of OC)
    otm_status enqueue_tail(bool with_tensor = true) {
        if (with_tensor) OTM_TRY(tensor_and_sens(true));
        if (!use_mma()) {
            ++nl_;
            launch_pdl(k_governor, 1, 1, stream, ds, 1.0 / (double)N, 0, 0.0);
            OTM_LAUNCH();
        }
        if (prm.symmetry) {
            ++nl_;
            launch_pdl(k_symmetrize<R>, grid(N / 2 + 1), 256, stream, N, rho, s);
            OTM_LAUNCH();
        }
        if (use_mma()) {
            nl_ += mma_enqueue<R>(N, rho, mx1, mx2, mL, mU, s, mp_, ds, rbuf(), grid(N), stream);
            OTM_LAUNCH();
        } else {
            OTM_TRY(oc_update());
        }
        return OTM_OK;
    }

    otm_status read_ps() {
        OTM_CU(cudaMemcpyAsync(ps_h, ps, sizeof(PcgScalars), cudaMemcpyDeviceToHost, stream));
        OTM_CU(cudaStreamSynchronize(stream));
        if (ps_h->dev_err) {
            err = "a bounded device wait ran out (asynchronous copy did not complete)";
            return OTM_ETIMEOUT;
        }
        return OTM_OK;
    }

    // host-driven pass
    otm_status pass_direct(int use_true) {
        OTM_TRY(enqueue_pass_head(use_true));
        OTM_CU(cudaMemcpyAsync(ps_h, ps, sizeof(PcgScalars), cudaMemcpyDeviceToHost, stream));
        OTM_CU(cudaStreamSynchronize(stream));
        while (ps_h->nactive > 0 && ps_h->total < prm.cg_maxit) {
            OTM_TRY(enqueue_body());
            OTM_CU(cudaMemcpyAsync(ps_h, ps, sizeof(PcgScalars), cudaMemcpyDeviceToHost, stream));
            OTM_CU(cudaStreamSynchronize(stream));
        }
        OTM_TRY(enqueue_check());
        return read_ps();
    }

    // Capture [setup] + pass head + while{body} + check into one graph.
    otm_status capture_pass(bool with_setup, int use_true, cudaGraphExec_t* out, long long* fixed) {
        cudaGraph_t g = nullptr;
        OTM_CU(cudaGraphCreate(&g, 0));
        cudaGraphConditionalHandle h;
        cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            err = std::string("cudaGraphConditionalHandleCreate: ") + cudaGetErrorString(e);
            return OTM_ECUDA;
        }
        const long long n0 = nl_;
        cudaStream_t main = stream;
        otm_status st = OTM_OK;
        long long body = 0;
        e = cudaStreamBeginCaptureToGraph(main, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            err = std::string("cudaStreamBeginCaptureToGraph: ") + cudaGetErrorString(e);
            return OTM_ECUDA;
        }
        // With the setup, the coarse hierarchy (which needs only k) runs on a
        // side branch of the graph, beside the macro loads and the pass's
        // initial residual; the branches join before the PCG loop, whose
        // first V-cycle is the first reader of the coarse levels.
        bool forked = false, lo_cleared = false;
        if (with_setup) {
            st = filter_simp();
            if (st == OTM_OK && nlev > 1) {
                e = cudaEventRecord(ev_fork, main);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev_fork, 0);
                if (e == cudaSuccess) {
                    forked = true;
                    stream = side;
                    st = coarse_hierarchy();
                    // the first pass's lo is cleared on this branch too: no
                    // kernel before the PCG loop reads it
                    if (st == OTM_OK && head_tma(use_true)) {
                        st = clear_lo();
                        lo_cleared = true;
                    }
                    stream = main;
                    if (st == OTM_OK) e = cudaEventRecord(ev_join, side);
                }
                if (st == OTM_OK && e == cudaSuccess) st = fine_loads();
            } else if (st == OTM_OK) {
                st = build_hierarchy();
            }
            if (st == OTM_OK && e == cudaSuccess) {
                ++nl_;
                launch_pdl(k_pcg_reset, 1, 1, stream, ps);
                OTM_LAUNCH();
            }
            if (e != cudaSuccess && st == OTM_OK) {
                err = std::string("graph capture of the setup branches: ") + cudaGetErrorString(e);
                st = OTM_ECUDA;
            }
        }
        if (st == OTM_OK) st = enqueue_pass_head(use_true, lo_cleared);
        if (st == OTM_OK && forked) {
            e = cudaStreamWaitEvent(main, ev_join, 0);
            if (e != cudaSuccess) {
                err = std::string("graph capture of the setup join: ") + cudaGetErrorString(e);
                st = OTM_ECUDA;
            }
        }
        if (st == OTM_OK) {
            ++nl_;
            launch_pdl(k_set_cond, 1, 1, stream, ps, h, prm.cg_maxit);
            cudaStreamCaptureStatus cs;
            cudaGraph_t cg = nullptr;
            const cudaGraphNode_t* deps = nullptr;
            size_t nd = 0;
            e = cudaStreamGetCaptureInfo(main, &cs, nullptr, &cg, &deps, nullptr, &nd);
            cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t cn = nullptr;
            if (e == cudaSuccess) e = cudaGraphAddNode(&cn, cg, deps, nullptr, nd, &cp);
            if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(main, &cn, nullptr, 1, cudaStreamSetCaptureDependencies);
            if (e == cudaSuccess) {
                cudaGraph_t bg = cp.conditional.phGraph_out[0];
                e = cudaStreamBeginCaptureToGraph(cap2, bg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
                if (e == cudaSuccess) {
                    stream = cap2;
                    const long long b0 = nl_;
                    st = enqueue_body();
                    ++nl_;
                    launch_pdl(k_set_cond, 1, 1, stream, ps, h, prm.cg_maxit);
                    body = nl_ - b0;
                    stream = main;
                    cudaGraph_t tmp = nullptr;
                    cudaError_t e2 = cudaStreamEndCapture(cap2, &tmp);
                    if (e2 != cudaSuccess) e = e2;
                }
            }
            if (e != cudaSuccess && st == OTM_OK) {
                err = std::string("graph capture of the PCG loop: ") + cudaGetErrorString(e);
                st = OTM_ECUDA;
            }
        }
        // The design tail's tensor, sensitivity and filter transpose read only
        // k, rho_f and this pass's iterate, so they run on a side branch beside
        // the error-free convergence check (with their own reduction buffer).
        // If the check asks for another pass, that pass's graph recomputes
        // them from its own iterate, so the values the tail uses always belong
        // to the last pass.
        bool forked2 = false;
        if (st == OTM_OK && spec_tensor_) {
            e = cudaEventRecord(ev_fork2, main);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev_fork2, 0);
            if (e == cudaSuccess) {
                forked2 = true;
                stream = side;
                st = tensor_and_sens(true, true);
                stream = main;
                if (st == OTM_OK) e = cudaEventRecord(ev_join2, side);
            }
            if (e != cudaSuccess && st == OTM_OK) {
                err = std::string("graph capture of the tensor branch: ") + cudaGetErrorString(e);
                st = OTM_ECUDA;
            }
        }
        if (st == OTM_OK) st = enqueue_check();
        if (st == OTM_OK && forked2) {
            e = cudaStreamWaitEvent(main, ev_join2, 0);
            if (e != cudaSuccess) {
                err = std::string("graph capture of the tensor join: ") + cudaGetErrorString(e);
                st = OTM_ECUDA;
            }
        }
        cudaGraph_t done = nullptr;
        e = cudaStreamEndCapture(main, &done);
        stream = main;
        if (st == OTM_OK && e != cudaSuccess) {
            err = std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e);
            st = OTM_ECUDA;
        }
        const bool captured = st == OTM_OK;
        if (st == OTM_OK) {
            e = cudaGraphInstantiate(out, g, 0);
            if (e != cudaSuccess) {
                err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
                st = OTM_ECUDA;
            }
        }
        // A graph whose capture failed part way (a launch inside the PCG loop's
        // conditional body refused) is left alone: destroying one crashed the
        // driver (in cuGraphDestroy).  The graph leaks only on that error path.
        if (captured) cudaGraphDestroy(g);
        *fixed = (nl_ - n0) - body;
        nlg_body = body;
        nl_ = n0;
        cudaGetLastError();
        return st;
    }

    // The pass graphs compute the tensor, the sensitivity and its filter
    // transpose beside the convergence check (see capture_pass), so the
    // tail graph starts at Alg. 1.
    otm_status capture_tail() { return capture_seq(false, &gx_tail, &nlg_tail, !spec_tensor_); }
    bool spec_tensor_ = true;   // OTM_SPEC_TENSOR=0: tensor and sensitivity in the tail graph instead

    // Capture the design tail (setup = false) or the solve setup (true).
    otm_status capture_seq(bool setup, cudaGraphExec_t* out, long long* count, bool tail_tensor = true) {
        const long long n0 = nl_;
        OTM_CU(cudaStreamBeginCapture(stream, cudaStreamCaptureModeRelaxed));
        otm_status st = setup ? enqueue_setup() : enqueue_tail(tail_tensor);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(stream, &g);
        if (st != OTM_OK) {
            if (g) cudaGraphDestroy(g);
            nl_ = n0;
            return st;
        }
        if (e != cudaSuccess) {
            err = std::string("cudaStreamEndCapture (tail): ") + cudaGetErrorString(e);
            nl_ = n0;
            return OTM_ECUDA;
        }
        e = cudaGraphInstantiate(out, g, 0);
        cudaGraphDestroy(g);
        *count = nl_ - n0;
        nl_ = n0;
        if (e != cudaSuccess) {
            err = std::string("cudaGraphInstantiate (tail): ") + cudaGetErrorString(e);
            return OTM_ECUDA;
        }
        return OTM_OK;
    }

    otm_status prepare() override {
        OTM_TRY(autotune());
        return use_graphs ? ensure_graphs() : OTM_OK;
    }

    // Measured choice of the coarse-level launch configuration: which levels
    // run in the cluster kernel (at most 8 or 16 nodes per side) and its CTA
    // count (8, or 16 where a 16-CTA cluster is schedulable).  Every candidate
    // applies the same per-node operations, so the choice changes no result;
    // it is made once per device, grid size and precision in the process
    // (the first context times V-cycles on its own fields after an eager
    // setup; later ones reuse the choice).
    struct TuneKey {
        int device, n, rbytes, sbytes, cheb;
        bool operator<(const TuneKey& o) const {
            return std::tie(device, n, rbytes, sbytes, cheb) < std::tie(o.device, o.n, o.rbytes, o.sbytes, o.cheb);
        }
    };
    struct TuneVal {
        int maxn, ctas;
        double us[4];
        int gs_stages;      // ring depth of the TMA group pass (0: not tuned)
        double gs_us[3];    // V-cycle us at depths 4, 5, 6 (0: not measured)
    };
    static std::mutex& tune_mutex() {
        static std::mutex m;
        return m;
    }
    static std::map<TuneKey, TuneVal>& tune_cache() {
        static std::map<TuneKey, TuneVal> c;
        return c;
    }
    otm_status autotune() {
        if (tuned_) return OTM_OK;
        tuned_ = true;
        if (!autotune_on_ || !use_cluster || nlev < 3 || (maxn_fixed_ && ctas_fixed_)) return OTM_OK;
        const TuneKey key{device, n, (int)sizeof(R), (int)sizeof(S), cheb_ ? 1 : 0};
        std::lock_guard<std::mutex> lock(tune_mutex());
        auto it = tune_cache().find(key);
        if (it == tune_cache().end()) {
            const int cand[4][2] = {{8, 8}, {8, 16}, {16, 8}, {16, 16}};
            const int keep_maxn = cluster_maxn, keep_ctas = cl_ctas_;
            OTM_TRY(enqueue_setup());
            cudaEvent_t e0, e1;
            OTM_CU(cudaEventCreate(&e0));
            OTM_CU(cudaEventCreate(&e1));
            // microseconds of one V-cycle (two warm-up cycles, four timed)
            auto time_vcycle = [&](otm_status& st) -> double {
                for (int w = 0; w < 2 && st == OTM_OK; ++w) st = vcycle();
                if (st != OTM_OK) return 0.0;
                if (cudaEventRecord(e0, stream) != cudaSuccess) st = OTM_ECUDA;
                for (int r = 0; r < 4 && st == OTM_OK; ++r) st = vcycle();
                if (st == OTM_OK && cudaEventRecord(e1, stream) != cudaSuccess) st = OTM_ECUDA;
                if (st == OTM_OK && cudaEventSynchronize(e1) != cudaSuccess) st = OTM_ECUDA;
                float ms = 0.f;
                if (st == OTM_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = OTM_ECUDA;
                return st == OTM_OK ? 1000.0 * ms / 4.0 : 0.0;
            };
            TuneVal best{keep_maxn, keep_ctas, {0, 0, 0, 0}, 0, {0, 0, 0}};
            double best_us = 0.0;
            otm_status st = OTM_OK;
            for (int c = 0; c < 4 && st == OTM_OK; ++c) {
                if (maxn_fixed_ && cand[c][0] != keep_maxn) continue;
                if (ctas_fixed_ && cand[c][1] != keep_ctas) continue;
                if (cand[c][1] == 16 && !cl16_ok_) continue;
                cluster_maxn = cand[c][0];
                cl_ctas_ = cand[c][1];
                const double us = time_vcycle(st);
                if (st != OTM_OK) break;
                best.us[c] = us;
                if (best_us == 0.0 || us < best_us) {
                    best_us = us;
                    best.maxn = cand[c][0];
                    best.ctas = cand[c][1];
                }
            }
            // then, with that cluster configuration, the TMA group pass's ring
            // depth (a shape change only: every depth gives the same bits)
            if constexpr (std::is_same<R, float>::value && !std::is_same<S, double>::value) {
                if (st == OTM_OK && tma_gs_.grid > 0 && !gs_tma_stages_fixed()) {
                    cluster_maxn = best.maxn;
                    cl_ctas_ = best.ctas;
                    const TmaLaunch keep_gs = tma_gs_;
                    double gbest = 0.0;
                    for (int d = 4; d <= 6 && st == OTM_OK; ++d) {
                        TmaLaunch L;
                        if (!gs_tma_launch_shape<S, float>(L, n, sm_count, d)) {
                            cudaGetLastError();
                            continue;
                        }
                        tma_gs_ = L;
                        const double us = time_vcycle(st);
                        if (st != OTM_OK) break;
                        best.gs_us[d - 4] = us;
                        if (gbest == 0.0 || us < gbest) {
                            gbest = us;
                            best.gs_stages = d;
                        }
                    }
                    tma_gs_ = keep_gs;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            cluster_maxn = keep_maxn;
            cl_ctas_ = keep_ctas;
            if (st != OTM_OK) {
                if (err.empty()) err = "autotune: a timing call failed";
                return st;
            }
            it = tune_cache().emplace(key, best).first;
        }
        cluster_maxn = it->second.maxn;
        cl_ctas_ = it->second.ctas;
        for (int c = 0; c < 4; ++c) tune_us_[c] = it->second.us[c];
        for (int d = 0; d < 3; ++d) gs_tune_us_[d] = it->second.gs_us[d];
        if constexpr (std::is_same<R, float>::value && !std::is_same<S, double>::value) {
            TmaLaunch L;
            if (it->second.gs_stages > 0 && tma_gs_.grid > 0 &&
                gs_tma_launch_shape<S, float>(L, n, sm_count, it->second.gs_stages))
                tma_gs_ = L;
            cudaGetLastError();
        }
        autotuned_ = 1;
        return OTM_OK;
    }

    otm_status get_config(otm_config* out) override {
        OTM_TRY(prepare());
        memset(out, 0, sizeof(*out));
        out->stencil_form = stencil_choice();
        if (out->stencil_form == 0 && tma_pcg_.grid == 0) out->stencil_form = tz_ > 0 ? 1 : 2;
        if (out->stencil_form == 1 && tz_ == 0) out->stencil_form = 2;
        out->stencil_chunks = tma_pcg_.m;
        out->levels = nlev;
        out->coarsest_n = sz[nlev - 1];
        out->cluster_maxn = use_cluster && nlev > 1 ? cluster_maxn : 0;
        out->cluster_ctas = use_cluster && nlev > 1 ? cl_ctas_ : 0;
        out->tail_maxn = tail_maxn;
        out->autotuned = autotuned_;
        for (int c = 0; c < 4; ++c) out->tune_us[c] = tune_us_[c];
        out->gs_form = tma_gs_.grid > 0 ? 0 : 1;
        out->gs_chunks = tma_gs_.grid > 0 ? tma_gs_.m : 0;
        out->gs_stages = tma_gs_.grid > 0 ? tma_gs_.stages : 0;
        for (int d = 0; d < 3; ++d) out->gs_tune_us[d] = gs_tune_us_[d];
        out->head_form = tma_head_.grid > 0 ? 0 : 1;
        return OTM_OK;
    }

    otm_status ensure_graphs() {
        OTM_TRY(autotune());
        if (gx_first) return OTM_OK;
        std::lock_guard<std::mutex> lock(graph_build_mutex());
        OTM_TRY(capture_pass(true, 0, &gx_first, &nlg_first));
        OTM_TRY(capture_pass(false, 1, &gx_pass, &nlg_pass));
        OTM_TRY(capture_tail());
        return OTM_OK;
    }

    otm_status launch_pass(cudaGraphExec_t gx, long long fixed) {
        const int before = ps_h->total;
        OTM_CU(cudaGraphLaunch(gx, stream));
        OTM_TRY(read_ps());
        const int ran = ps_h->total - before;
        nl_ += fixed + nlg_body * (ran > 0 ? ran : 0);
        return OTM_OK;
    }

    // Setup + solve.  Returns OTM_OK / OTM_ENOCONV; fills iterations and the
    // checked residuals.
    otm_status setup_and_solve(bool warm, otm_step_info* info, bool learned = false) {
        OTM_TRY(autotune());
        if (!warm) {
            OTM_CU(cudaMemsetAsync(x, 0, 3 * N * sizeof(R), stream));
            if (xl) OTM_CU(cudaMemsetAsync(xl, 0, 3 * N * sizeof(R), stream));
        }
        int iters[3] = {0, 0, 0};
        ps_h->total = 0;
        if (learned) {
            if (use_graphs) {
                OTM_TRY(ensure_graphs());
                std::unique_lock<std::mutex> lock(graph_build_mutex());
                if (!gx_setup) OTM_TRY(capture_seq(true, &gx_setup, &nlg_setup));
                if (!gx_solve0) {
                    long long fixed = 0;
                    const long long body = nlg_body;
                    OTM_TRY(capture_pass(false, 0, &gx_solve0, &fixed));
                    nlg_solve0 = fixed;
                    nlg_body = body;
                }
                lock.unlock();
                OTM_CU(cudaGraphLaunch(gx_setup, stream));
                nl_ += nlg_setup;
            } else {
                OTM_TRY(enqueue_setup());
            }
            OTM_CU(cudaEventRecord(ev[1], stream));
            OTM_TRY(predict_start(warm));
            OTM_CU(cudaEventRecord(ev[3], stream));
            if (use_graphs) OTM_TRY(launch_pass(gx_solve0, nlg_solve0));
            else OTM_TRY(pass_direct(0));
            if (info) {
                int code = 0;
                for (int i = 0; i < 3; ++i) code |= (ws_h->choice[i] & 3) << (2 * i);
                info->ws_choice = code;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[1], ev[3]);
                info->stage_ms[1] = ms;
            }
        } else if (use_graphs) {
            OTM_TRY(ensure_graphs());
            OTM_TRY(launch_pass(gx_first, nlg_first));
        } else {
            OTM_TRY(enqueue_setup());
            OTM_TRY(pass_direct(0));
        }
        bool converged = false, finite = true;
        double prev_worst = 1e300;
        for (int restart = 0;; ++restart) {
            for (int i = 0; i < 3; ++i) iters[i] += ps_h->iters[i];
            double worst = 0.0;
            bool all_ok = true;
            for (int i = 0; i < 3; ++i) {
                const double ff = ps_h->true_ff[i];
                // a non-finite load or residual (NaN or Inf in rho or in the
                // iterate) never counts as converged
                if (!std::isfinite(ff) || !std::isfinite(ps_h->true_rr[i])) {
                    finite = false;
                    all_ok = false;
                    continue;
                }
                const double rel = ff > 0 ? std::sqrt(ps_h->true_rr[i] / ff) : 0.0;
                worst = rel > worst ? rel : worst;
                if (!(rel <= prm.cg_tol)) all_ok = false;
            }
            if (!finite) break;
            if (all_ok) {
                converged = true;
                break;
            }
            if (restart >= kMaxRestarts || ps_h->total >= prm.cg_maxit || !(worst < 0.5 * prev_worst)) break;
            prev_worst = worst;
            if (use_graphs) OTM_TRY(launch_pass(gx_pass, nlg_pass));
            else OTM_TRY(pass_direct(1));
        }
        for (int i = 0; i < 3; ++i) {
            const double ff = ps_h->true_ff[i];
            const double rel = ff > 0 ? std::sqrt(ps_h->true_rr[i] / ff) : 0.0;
            last_iters[i] = iters[i];
            if (info) {
                info->cg_iters[i] = iters[i];
                info->resid[i] = rel;
            }
        }
        if (!finite) {
            err = "non-finite load or residual (NaN or Inf in the density or the solution)";
            return OTM_ENOCONV;
        }
        if (!converged) {
            err = "PCG did not reach cg_tol (cg_maxit reached or the residual stagnated)";
            return OTM_ENOCONV;
        }
        return OTM_OK;
    }

    // Learned warm start: predict from rho_f, score the candidates by their
    // true residuals and install the best per load case into (x, xl).
    otm_status predict_start(bool have_prev_x) {
        float* y = ynet[ycur];
        const float* yp = ynet[ycur ^ 1];
        const long long u0 = unet_launches();
        OTM_TRY(unet_predict(predictor, rho_f, std::is_same<R, double>::value, y, stream));
        nl_ += unet_launches() - u0;
        // the change of the prediction is only meaningful against the
        // previous iteration's prediction
        const bool delta = have_prev_x && have_y && y_iter == iteration - 1;
        RedBuf rb = rbuf();
        auto score = [&](const R* xh, const R* xlo, int slot) -> otm_status {
            ++nl_;
            if (wr_)
                launch_pdl(k_true_residual_wr<FinStore>, wr_grid((long long)n * n * (n / 128)), 256, stream, n,
                           (const float*)kf, (const float*)xh, (const float*)xlo, (const float*)f, rb,
                           FinStore{&ws->cand[slot][0]});
            else
                launch_pdl(k_true_residual<R, FinStore>, OTM_ROWS_CFG(rl(n, n * n)), stream, n, kf, xh, xlo, f, rb,
                           FinStore{&ws->cand[slot][0]});
            OTM_LAUNCH();
            return OTM_OK;
        };
        auto cand = [&](int mode, R* xc) -> otm_status {
            nl_ += 3;
            k_ws_cand<R><<<grid(3 * N), 256, 0, stream>>>(N, mode, x, xl, y, yp, pred_scale, xc);
            launch_pdl(k_sum3<R>, grid(N), 256, stream, N, (const R*)xc, rb, FinMean{ps_c, 1.0 / (double)N});
            launch_pdl(k_sub_mean<R>, grid(N), 256, stream, N, xc, (const PcgScalars*)ps_c);
            OTM_LAUNCH();
            return score(xc, nullptr, mode);
        };
        ws_had_prev = have_prev_x;
        ws_had_delta = delta;
        OTM_TRY(cand(kWsNet, xc_net));
        if (have_prev_x) OTM_TRY(score(x, xl, kWsPrev));
        if (delta) OTM_TRY(cand(kWsDelta, xc_delta));
        nl_ += 2;
        k_ws_decide<<<1, 32, 0, stream>>>(ws, have_prev_x ? 1 : 0, delta ? 1 : 0);
        k_ws_take<R><<<grid(3 * N), 256, 0, stream>>>(N, ws, xc_net, xc_delta, x, xl);
        OTM_LAUNCH();
        OTM_CU(cudaMemcpyAsync(ws_h, ws, sizeof(WsState), cudaMemcpyDeviceToHost, stream));
        ycur ^= 1;
        have_y = true;
        y_iter = iteration;
        return OTM_OK;
    }

    // after the solve (ws_h is current): update the back-off.  A prediction
    // pays when, for some load case, its residual norm is at most a quarter
    // of the best start without it (about half a PCG iteration saved at the
    // V-cycle's contraction); a smaller gain is still used for the start but
    // does not reset the back-off.
    bool ws_after_prediction() {
        bool used = false;
        for (int i = 0; i < 3; ++i) {
            double best_np = ws_h->cand[kWsNet][3 + i];   // zero start
            if (ws_had_prev) best_np = std::min(best_np, ws_h->cand[kWsPrev][i]);
            double best_p = ws_h->cand[kWsNet][i];
            if (ws_had_delta) best_p = std::min(best_p, ws_h->cand[kWsDelta][i]);
            used |= best_p <= best_np / 16.0;
        }
        if (used) {
            ws_period = 1;
        } else {
            ws_period = ws_period * 2 > kWsMaxPeriod ? kWsMaxPeriod : ws_period * 2;
        }
        ws_wait = ws_period - 1;
        return used;
    }

    otm_status set_predictor(otm_unet* u, double scale) override {
        if (u && unet_grid(u) != n) {
            err = "otm_set_predictor: the network's grid differs from the context's n";
            return OTM_EINVAL;
        }
        if (u && !(std::isfinite(scale) && scale != 0.0)) {
            err = "otm_set_predictor: scale must be finite and nonzero";
            return OTM_EINVAL;
        }
        if (u && !ws) {
            OTM_TRY(alloc(ynet[0], 3 * N));
            OTM_TRY(alloc(ynet[1], 3 * N));
            OTM_TRY(alloc(xc_net, 3 * N));
            OTM_TRY(alloc(xc_delta, 3 * N));
            OTM_TRY(alloc(ws, 1));
            OTM_CU(cudaMallocHost((void**)&ws_h, sizeof(WsState)));
            memset(ws_h, 0, sizeof(WsState));
        }
        OTM_CU(cudaStreamSynchronize(stream));
        predictor = u;
        pred_scale = scale;
        have_y = false;
        ws_period = 1;
        ws_wait = 0;
        return OTM_OK;
    }

    // kappa (and the objective) from x; optionally the sensitivity chain.
    otm_status tensor_and_sens(bool with_sens, bool second_buffer = false) {
        ++nl_;
        launch_pdl(k_kappa<R>, OTM_ROWS_CFG(rl(n, n * n)), stream, n, kf, x, second_buffer ? rbuf2() : rbuf(),
                   FinKappa{ds, 1.0 / (double)N, 1});
        OTM_LAUNCH();
        if (with_sens) {
            ++nl_;
            launch_pdl(k_sens<R>, OTM_ROWS_CFG(rl(n, n * n)), stream, n, rho_f, x, ds, sp, s_f);
            ++nl_;
            launch_filter<R, false>(rl(n, n * n), stream, n, fw, -1, (const R*)s_f, s, (R*)nullptr, sp, rbuf(), FinFilter{ds});
            OTM_LAUNCH();
        }
        return OTM_OK;
    }

    otm_status oc_update() {
        const double dN = (double)N;
        ++nl_;
        launch_pdl(k_oc_prep<R>, grid(N), 256, stream, N, rho, s, op, ds, rbuf(), FinOcPrep{ds, dN});
        OTM_LAUNCH();
        const int passes = std::is_same<C, double>::value ? 7 : 4;
        for (int pidx = 0; pidx < passes; ++pidx) {
            const int linear = pidx == passes - 1;
            ++nl_;
            launch_pdl(k_oc_search<R>, grid(N), 256, stream, N, rho, s, op, ds, linear, rbuf(),
                                                        FinOcSearch{ds, dN, linear, linear, 1.0 / prm.damp});
            OTM_LAUNCH();
        }
        ++nl_;
        launch_pdl(k_oc_apply<R>, grid(N), 256, stream, N, rho, s, op, ds);
        OTM_LAUNCH();
        return OTM_OK;
    }

    void fill_info(otm_step_info& loc) {
        loc.g = ds_h->g;
        for (int c = 0; c < 6; ++c) loc.kappa[c] = ds_h->kappa[c];
        loc.mean_rho = ds_h->sum_rho / (double)N;
        loc.mean_rhop = ds_h->sum_rhop / (double)N;
        loc.vstar = ds_h->vstar;
        loc.iteration = iteration;
    }

    otm_status homogenize(const float* rho_in, bool on_device, double kappa[6], otm_step_info* info) override {
        if (rho_in) {
            OTM_CU(cudaMemcpyAsync(rho_save, rho, N * sizeof(R), cudaMemcpyDeviceToDevice, stream));
            OTM_TRY(to_R(rho_in, on_device, rho, N, true));
        }
        otm_step_info loc;
        memset(&loc, 0, sizeof(loc));
        for (auto& row : loc.ws_resid)
            for (double& v : row) v = -1.0;
        const long long nl0 = nl_;
        otm_status sst = setup_and_solve(false, &loc);
        otm_status st = (sst == OTM_OK || sst == OTM_ENOCONV) ? tensor_and_sens(false) : sst;
        if (rho_in) OTM_CU(cudaMemcpyAsync(rho, rho_save, N * sizeof(R), cudaMemcpyDeviceToDevice, stream));
        if (st != OTM_OK) return st;
        OTM_CU(cudaMemcpyAsync(ds_h, ds, sizeof(DesignScalars), cudaMemcpyDeviceToHost, stream));
        OTM_CU(cudaStreamSynchronize(stream));
        for (int c = 0; c < 6; ++c) kappa[c] = ds_h->kappa[c];
        fill_info(loc);
        loc.lambda = 0.0;
        loc.kernel_launches = (int)(nl_ - nl0);
        if (info) *info = loc;
        have_prev = false;
        OTM_TRY(take_check());
        return sst;
    }

    // relative true residual of each scored candidate start (otm_step_info.ws_resid)
    void fill_ws_resid(otm_step_info& loc) const {
        for (int i = 0; i < 3; ++i) {
            const double ff = ws_h->cand[kWsNet][3 + i];
            auto rel = [&](int c) { return ff > 0 ? std::sqrt(ws_h->cand[c][i] / ff) : 0.0; };
            loc.ws_resid[kWsZero][i] = ff > 0 ? 1.0 : 0.0;
            loc.ws_resid[kWsPrev][i] = ws_had_prev ? rel(kWsPrev) : -1.0;
            loc.ws_resid[kWsNet][i] = rel(kWsNet);
            loc.ws_resid[kWsDelta][i] = ws_had_delta ? rel(kWsDelta) : -1.0;
        }
    }

    otm_status step(otm_step_info* info) override {
        otm_step_info loc;
        memset(&loc, 0, sizeof(loc));
        for (auto& row : loc.ws_resid)
            for (double& v : row) v = -1.0;
        const long long nl0 = nl_;
        OTM_CU(cudaEventRecord(ev[0], stream));
        const bool warm = have_prev && prm.warm_start != OTM_WS_NONE;
        const bool attached = prm.warm_start == OTM_WS_LEARNED && predictor != nullptr;
        const bool learned = attached && (!warm || ws_wait == 0);
        otm_status sst = setup_and_solve(warm, &loc, learned);
        if (learned && (sst == OTM_OK || sst == OTM_ENOCONV)) {
            if (ws_after_prediction()) loc.ws_choice |= 1 << 7;
            fill_ws_resid(loc);
        }
        else if (attached) {
            --ws_wait;
            loc.ws_choice = 1 | (1 << 2) | (1 << 4) | (1 << 6);   // previous start, predictor skipped
        }
        if (sst != OTM_OK && sst != OTM_ENOCONV) return sst;
        have_prev = true;
        OTM_CU(cudaEventRecord(ev[2], stream));
        if (use_graphs) {
            OTM_CU(cudaGraphLaunch(gx_tail, stream));
            nl_ += nlg_tail;
        } else {
            OTM_TRY(enqueue_tail());
        }
        OTM_CU(cudaEventRecord(ev[5], stream));
        OTM_CU(cudaMemcpyAsync(ds_h, ds, sizeof(DesignScalars), cudaMemcpyDeviceToHost, stream));
        OTM_CU(cudaStreamSynchronize(stream));
        fill_info(loc);
        loc.lambda = ds_h->lambda;
        float ms;
        cudaEventElapsedTime(&ms, ev[0], ev[2]); loc.stage_ms[2] = ms;
        cudaEventElapsedTime(&ms, ev[2], ev[5]); loc.stage_ms[4] = ms;
        cudaEventElapsedTime(&ms, ev[0], ev[5]); loc.stage_ms[7] = ms;
        loc.kernel_launches = (int)(nl_ - nl0);
        iteration += 1;
        if (info) *info = loc;
        OTM_TRY(take_check());
        return sst;
    }
    // Checking build: a bounds check that failed in this unit's kernels fails the call.
    otm_status take_check() {
        const std::string c = check_take();
        if (c.empty()) return OTM_OK;
        err = c;
        return OTM_ECUDA;
    }

    // ---------------------------------------------------------- checkpoint
    struct StateHeader {
        uint64_t magic;
        int32_t n, precision, iteration, have_prev;
        GovState gov;
        double vstar;
        uint64_t rho_bytes, chi_bytes;
        int32_t optimizer, mma_k;   // MMA: iteration count, then its four arrays after the solution
        uint64_t mma_bytes;
    };
    size_t chi_bytes() const { return (xl ? 6 : 3) * N * sizeof(R); }
    size_t mma_bytes() const { return use_mma() ? 4 * N * sizeof(R) : 0; }
    size_t state_size() const override { return sizeof(StateHeader) + N * sizeof(R) + chi_bytes() + mma_bytes(); }
    otm_status get_state(void* buf) override {
        StateHeader h;
        memset(&h, 0, sizeof(h));
        h.magic = 0x4f544d5354415445ull;
        h.n = n;
        h.precision = prm.precision;
        h.iteration = iteration;
        h.have_prev = have_prev ? 1 : 0;
        OTM_CU(cudaMemcpyAsync(ds_h, ds, sizeof(DesignScalars), cudaMemcpyDeviceToHost, stream));
        OTM_CU(cudaStreamSynchronize(stream));
        h.gov = ds_h->gov;
        h.vstar = ds_h->vstar;
        h.rho_bytes = N * sizeof(R);
        h.chi_bytes = chi_bytes();
        h.optimizer = prm.optimizer;
        h.mma_k = ds_h->mma_k;
        h.mma_bytes = mma_bytes();
        char* b = (char*)buf;
        memcpy(b, &h, sizeof(h));
        if (use_mma()) {
            char* m = b + sizeof(h) + h.rho_bytes + h.chi_bytes;
            R* arr[4] = {mx1, mx2, mL, mU};
            for (int i = 0; i < 4; ++i)
                OTM_CU(cudaMemcpyAsync(m + i * N * sizeof(R), arr[i], N * sizeof(R), cudaMemcpyDeviceToHost, stream));
        }
        OTM_CU(cudaMemcpyAsync(b + sizeof(h), rho, h.rho_bytes, cudaMemcpyDeviceToHost, stream));
        OTM_CU(cudaMemcpyAsync(b + sizeof(h) + h.rho_bytes, x, 3 * N * sizeof(R), cudaMemcpyDeviceToHost, stream));
        if (xl)
            OTM_CU(cudaMemcpyAsync(b + sizeof(h) + h.rho_bytes + 3 * N * sizeof(R), xl, 3 * N * sizeof(R),
                                   cudaMemcpyDeviceToHost, stream));
        OTM_CU(cudaStreamSynchronize(stream));
        return OTM_OK;
    }
    otm_status set_state(const void* buf, size_t len) override {
        if (len < sizeof(StateHeader)) {
            err = "otm_set_state: blob too short";
            return OTM_ESTATE;
        }
        StateHeader h;
        memcpy(&h, buf, sizeof(h));
        if (h.magic != 0x4f544d5354415445ull || h.n != n || h.precision != prm.precision ||
            h.rho_bytes != N * sizeof(R) || h.chi_bytes != chi_bytes() || h.optimizer != prm.optimizer ||
            h.mma_bytes != mma_bytes() || len < state_size()) {
            err = "otm_set_state: blob does not match this context (n, precision or size)";
            return OTM_ESTATE;
        }
        const char* b = (const char*)buf;
        OTM_CU(cudaMemcpyAsync(rho, b + sizeof(h), h.rho_bytes, cudaMemcpyHostToDevice, stream));
        OTM_CU(cudaMemcpyAsync(x, b + sizeof(h) + h.rho_bytes, 3 * N * sizeof(R), cudaMemcpyHostToDevice, stream));
        if (xl)
            OTM_CU(cudaMemcpyAsync(xl, b + sizeof(h) + h.rho_bytes + 3 * N * sizeof(R), 3 * N * sizeof(R),
                                   cudaMemcpyHostToDevice, stream));
        OTM_CU(cudaMemcpyAsync(&ds->gov, &h.gov, sizeof(GovState), cudaMemcpyHostToDevice, stream));
        OTM_CU(cudaMemcpyAsync(&ds->vstar, &h.vstar, sizeof(double), cudaMemcpyHostToDevice, stream));
        if (use_mma()) {
            const char* m = b + sizeof(h) + h.rho_bytes + h.chi_bytes;
            R* arr[4] = {mx1, mx2, mL, mU};
            for (int i = 0; i < 4; ++i)
                OTM_CU(cudaMemcpyAsync(arr[i], m + i * N * sizeof(R), N * sizeof(R), cudaMemcpyHostToDevice, stream));
            OTM_CU(cudaMemcpyAsync(&ds->mma_k, &h.mma_k, sizeof(int), cudaMemcpyHostToDevice, stream));
        }
        OTM_CU(cudaStreamSynchronize(stream));
        iteration = h.iteration;
        have_prev = h.have_prev != 0;
        have_y = false;
        ws_period = 1;
        ws_wait = 0;
        return OTM_OK;
    }

};

}  // namespace otm
