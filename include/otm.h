/*
 * otm.h -- C ABI of libotm.so: GB300 (sm_103a) periodic thermal-microstructure
 * homogenization and optimality-criteria design, after Quan, Zhai & Fu,
 * "OpenTM: an open-source, single-GPU, large-scale thermal microstructure
 * design framework" (arXiv 2405.19991).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - Grid: an n^3 periodic voxel unit cell, unit voxels, |Omega| = n^3.  A
 *    scalar field is a flat array of n^3 values with x fastest: voxel
 *    (x, y, z) is at x + n*(y + n*z).  Node (x, y, z) is the lower corner of
 *    element (x, y, z); element (x, y, z) has corners ((x+a)%n, (y+b)%n,
 *    (z+c)%n), local number a + 2b + 4c.  A three-load-case field is three
 *    such arrays back to back (load case i at offset i*n^3).
 *  - Tensors: 6-vectors in the order [k11, k22, k33, k12, k23, k13]
 *    (Sec. 2.2, Eq. rep).
 *  - Ownership: pointers passed in are borrowed for the duration of the call
 *    only.  A context owns all device memory it allocates; outputs are
 *    caller-allocated.  `on_device` = 1 means the pointer is device memory on
 *    the context's device, 0 means host memory.
 *  - Streams: work is ordered on the context's stream (params.stream, or a
 *    stream the context creates when that is NULL).  Every call returns after
 *    its work is complete (synchronous on the stream).
 *  - Errors: no exception or abort crosses the ABI.  Every call returns an
 *    otm_status; on failure otm_last_error(ctx) (or otm_last_error(NULL) for
 *    calls without a context, thread-local) describes it.  A call that fails
 *    with OTM_EINVAL has changed nothing.
 *  - Threads: a context must not be used by two threads at once; distinct
 *    contexts are independent.
 */
#ifndef OTM_H
#define OTM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define OTM_API __attribute__((visibility("default")))
#else
#define OTM_API
#endif

typedef enum otm_status {
    OTM_OK = 0,
    OTM_EINVAL = 1,    /* bad argument: size, pointer, parameter range */
    OTM_ENOMEM = 2,    /* device or host allocation failed */
    OTM_ECUDA = 3,     /* a CUDA runtime call or kernel failed */
    OTM_ENOCONV = 4,   /* CG hit cg_maxit or broke down; results hold the best iterate */
    OTM_ETIMEOUT = 5,  /* a bounded device wait ran out */
    OTM_ESTATE = 6     /* call out of order, or a checkpoint blob that does not match */
} otm_status;

/* Arithmetic of the solve (params.precision). */
enum {
    OTM_FP64 = 0,   /* every field and operation in FP64 */
    OTM_FP32 = 1,   /* FP32 fields and arithmetic; inner products, tensor and volume sums accumulated
                       with error-free transformations in FP32 pairs (about 48 significant bits) and
                       handed on as doubles; the iterate kept as an FP32 pair */
    OTM_MIXED = 2   /* FP32 outer CG; V-cycle fields and operators stored in BF16, FP32 arithmetic */
};

/* Initial guess of each homogenization solve (params.warm_start). */
enum {
    OTM_WS_NONE = 0,    /* start from zero */
    OTM_WS_PREV = 1,    /* start from the previous design iteration's solution */
    OTM_WS_LEARNED = 2  /* candidates from the attached U-Net predictor (otm_set_predictor) and the
                           previous solution; per load case the one with the smallest true residual */
};

/* Objective g(kappa^H, kappa*) (params.objective). */
enum {
    OTM_OBJ_MSE = 0,      /* Eq. mse: sum over the 6 components of (kappa - kappa*)^2 */
    OTM_OBJ_FRACMSE = 1,  /* Eq. fracmse: sum of (kappa/kappa* - 1)^2; a zero target component uses kappa^2 */
    OTM_OBJ_L1 = 2        /* Eq. l1: sum of |kappa - kappa*|, d|a|/da = 0 at 0 */
};

/* Design update (params.optimizer). */
enum {
    OTM_OPT_OC = 0,   /* optimality criteria on Eq. model3 (governor on) or Eq. model1 (governor off) */
    OTM_OPT_MMA = 1   /* Method of Moving Asymptotes on Eq. model2: minimise V(rho) subject to
                         g <= mma_eps, 0 <= rho <= 1 (MMAOptimizer, Sec. 3.3) */
};

/* Fields readable with otm_get_field. */
enum {
    OTM_FIELD_RHO = 0,        /* design density rho, n^3 */
    OTM_FIELD_RHO_FILT = 1,   /* filtered density (Sec. 2.3), n^3 */
    OTM_FIELD_K = 2,          /* SIMP element conductivity (Sec. 2.2), n^3 */
    OTM_FIELD_CHI = 3,        /* the three solutions T^(i) of Eq. kti, 3 n^3, zero mean */
    OTM_FIELD_LOAD = 4,       /* the three macro loads f^(i) (Sec. 2.4 enforceMacroLoad), 3 n^3 */
    OTM_FIELD_SENS = 5        /* dg/drho after the filter chain rule (Eq. sens), n^3 */
};

/*
 * Problem and solver parameters.  The problem statement follows the paper's
 * HomoConfig / runInstance inputs (Sec. 3.4, 3.5): resolution, the two
 * conductivities, the target tensor, the initial volume ratio; the OC
 * parameters follow OCOptimizer(min_density, stepLimit, dampExponent)
 * (Sec. 3.3) with the values of Sec. 4 (p = 3, r = 1.5, step 0.05, damping 0.5).
 */
typedef struct otm_params {
    int n;                   /* voxels per side, 4 <= n <= 512; the multigrid
                                hierarchy halves n while it is even and the half
                                is >= 4, and the coarsest size must be <= 7 */
    double kappa_target[6];  /* kappa*, must be symmetric positive definite */
    double volfrac;          /* initial mean density (not a constraint, Sec. 3.4) */
    double penal;            /* SIMP exponent p (Sec. 2.2), >= 1 */
    double rmin;             /* density-filter radius in voxels, 1 <= rmin < 3 */
    double k_solid, k_void;  /* kappa^0 and kappa_min of SIMP, k_solid > k_void > 0 */
    double move;             /* OC step limit (stepLimit) */
    double damp;             /* OC damping exponent eta (dampExponent) */
    double rho_min;          /* OC minimum density (min_density) */
    double cg_tol;           /* relative residual ||f - K x|| / ||f|| per load case */
    int cg_maxit;            /* PCG iteration cap per solve */
    int precision;           /* OTM_FP64 | OTM_FP32 | OTM_MIXED */
    int warm_start;          /* OTM_WS_* */
    int objective;           /* OTM_OBJ_* */
    int governor;            /* 1: adaptive V* of Alg. 1 (model Eq. model3), 0: fixed V* = fixed_volume (Eq. model1) */
    double fixed_volume;     /* V for governor = 0 */
    double gov_bound;        /* Alg. 1 "bound" on g (default 1e-4) */
    double gov_small_rel;    /* Alg. 1 is_small(g^[I-1] - g^[I]): |dg| < gov_small_rel * g (default 1e-3) */
    double gov_vol_tol;      /* Alg. 1 is_small(V - V*): |V - V*| < gov_vol_tol (default 1e-2) */
    int symmetry;            /* 1: central symmetry (Sec. 4.1), average rho and dg/drho over point-symmetric pairs */
    int coarse_smoother;     /* smoother of the coarse V-cycle levels (the finest level always runs the
                                8-colour Gauss-Seidel of Sec. 2.4): 0 = 8-colour symmetric Gauss-Seidel,
                                1 = degree-3 Chebyshev on D^-1 A with a Gershgorin bound (symmetric) */
    uint64_t seed;           /* seed of the learned predictor's initial weights */
    void* stream;            /* cudaStream_t to order work on; NULL = context-owned stream */
    int device;              /* CUDA device ordinal; -1 = current device */
    int optimizer;           /* OTM_OPT_OC | OTM_OPT_MMA; with MMA the governor, vstar and the OC
                                parameters (move, damp, rho_min) are not used */
    double mma_eps;          /* eps of Eq. model2's constraint g <= eps (default 1e-4) */
    double mma_move;         /* MMA move limit, a fraction of the box [0, 1] (default 0.5) */
    double mma_c, mma_d;     /* weights of the constraint's slack y in MMA's standard form,
                                c y + d y^2 / 2 (defaults 1000 and 1) */
} otm_params;

/* Per design-iteration report. */
typedef struct otm_step_info {
    double g;             /* objective at the density the iteration started from */
    double kappa[6];      /* kappa^H at that density */
    double mean_rho;      /* V(rho) = mean rho (Sec. 2.3) */
    double mean_rhop;     /* mean filtered rho^p, Alg. 1 lowBound */
    double vstar;         /* volume bound used by the OC update (0 with OTM_OPT_MMA) */
    double lambda;        /* OC Lagrange multiplier; 0 = constraint inactive, inf = all at lower bound.
                             OTM_OPT_MMA: the multiplier of g <= eps (0 = inactive, above mma_c = the
                             constraint could not be met within the move limits) */
    int cg_iters[3];      /* PCG iterations per load case */
    int iteration;        /* design iteration index (0-based) of this report */
    double resid[3];      /* true relative residual per load case at exit */
    float stage_ms[8];    /* [1] warm-start prediction and choice (OTM_WS_LEARNED), [2] setup and solve,
                             [4] tensor, sensitivity and OC update, [7] total; others 0 */
    int kernel_launches;  /* CUDA kernels this call launched (graph kernel nodes counted per execution) */
    int ws_choice;        /* OTM_WS_LEARNED with a predictor: start chosen per load case i, 2 bits at
                             2i: 0 zero, 1 previous solution, 2 predictor, 3 previous + predictor
                             change; bit 6 set: the predictor was skipped this iteration (back-off);
                             bit 7 set: the prediction paid (see otm_set_predictor) */
    double ws_resid[4][3];  /* when the predictor ran: relative true residual ||f_i - K x0||/||f_i||
                               of each candidate start x0 (index as in ws_choice: zero, previous
                               solution, predictor, previous + predictor change) per load case;
                               -1 for a candidate not scored, and every entry -1 otherwise */
} otm_step_info;

/* State of Alg. 1's adaptive volume bound. */
typedef struct otm_governor_state {
    double df;       /* decrease factor Df */
    double vstar;    /* V* */
    double g_prev;   /* g^[I-1] */
    double gap;      /* last V* - lowBound */
    int count;       /* consecutive stalled iterations */
    int reserved;
} otm_governor_state;

typedef struct otm_ctx otm_ctx;

/* ---------------------------------------------------------------- lifecycle */

/* Fill p with the defaults: n = 128, kappa* = [0.1,0.1,0.1,0,0,0],
 * volfrac 0.3, p = 3, r = 1.5, k = 1 / 1e-3, move 0.05, damp 0.5,
 * rho_min 1e-3, cg_tol 1e-6, cg_maxit 500, OTM_FP32, OTM_WS_PREV, MSE,
 * governor on (bound 1e-4, 1e-3, 1e-2), no symmetry, stream NULL, device -1,
 * OTM_OPT_OC (MMA: eps 1e-4, move 0.5, c 1000, d 1). */
OTM_API otm_status otm_params_default(otm_params* p);

/* OTM_OK if the 6-vector is a symmetric positive definite tensor (every
 * leading principal minor > 0; Sec. 4.2 uses the minors to bound the
 * feasible cross terms), else OTM_EINVAL.  Host only. */
OTM_API otm_status otm_check_target(const double kappa_target[6]);

/* Create a context with the defaults of otm_params_default and the given
 * problem (the call shape of the paper's problem statement: resolution,
 * target tensor, volume fraction, SIMP exponent, filter radius).  The
 * density is initialised to volfrac everywhere. */
OTM_API otm_status otm_create(int n, const double kappa_target[6], double volfrac,
                              double penal, double rmin, otm_ctx** out);

/* Create a context from a full parameter block.  Allocates every device
 * buffer of the solve (about 100 * n^3 bytes in OTM_FP32). */
OTM_API otm_status otm_create_ex(const otm_params* params, otm_ctx** out);

/* Release a context and all its device memory.  NULL is accepted. */
OTM_API otm_status otm_destroy(otm_ctx* ctx);

/* Copy a density field (n^3 floats, values clamped to [0, 1]) into the
 * context and reset the design loop (iteration 0, Alg. 1 initial state,
 * previous solution cleared). */
OTM_API otm_status otm_set_density(otm_ctx* ctx, const float* rho, int on_device);

/* Copy the current density (n^3 floats) out. */
OTM_API otm_status otm_get_density(otm_ctx* ctx, float* rho, int on_device);

/* The launch configuration a context runs with (Alg. 3's V-cycle and the
 * Sec. 2.4 stencil).  Reading it builds the step's CUDA graphs first (as
 * otm_step would), so an automatic choice has been made.
 *   stencil_form    fine stencil: 0 TMA-staged z-march, 1 shared-memory
 *                   tiled, 2 gather (OTM_STENCIL)
 *   stencil_chunks  z-chunks per row block of the TMA-staged form (0: not
 *                   used)
 *   levels, coarsest_n   the hierarchy: level count and the coarsest side
 *   cluster_maxn    levels with at most this many nodes per side run in one
 *                   thread-block cluster launch (0: no cluster)
 *   cluster_ctas    CTAs of that cluster
 *   tail_maxn       levels with at most this many nodes per side run in
 *                   shared memory of the cluster's first CTA
 *   autotuned       1 when cluster_maxn and cluster_ctas were chosen by
 *                   timing V-cycles on this device (OTM_AUTOTUNE, default on;
 *                   the candidates apply the same operations to every node,
 *                   so the choice never changes a result, only its time)
 *   tune_us         measured time of one V-cycle per candidate, in the order
 *                   (maxn 8, 8 CTAs), (8, 16), (16, 8), (16, 16); 0 when not
 *                   measured
 *   gs_form         fine Gauss-Seidel group pass: 0 TMA-staged z-march,
 *                   1 gather (OTM_GS); every form gives the same bits
 *   gs_chunks       runs of output planes per row block of the TMA-staged
 *                   group pass (0: not used)
 *   gs_stages       its ring depth: timed by the tuner after the cluster
 *                   choice, among 4, 5 and 6 (OTM_GS_STAGES fixes it)
 *   gs_tune_us      measured time of one V-cycle at depths 4, 5, 6; 0 when
 *                   not measured
 *   head_form       initial residual of a solve's first pass: 0 the
 *                   TMA-staged stencil's residual form on the iterate's
 *                   high part (its low part cleared first), 1 the pair form
 *                   f - K (hi + lo) (OTM_HEAD=pair; FP64 and sizes the staged
 *                   form does not cover); refinement passes always use the
 *                   pair form
 * Errors: OTM_EINVAL for NULL arguments; CUDA errors as OTM_ECUDA. */
typedef struct {
    int stencil_form;
    int stencil_chunks;
    int levels;
    int coarsest_n;
    int cluster_maxn;
    int cluster_ctas;
    int tail_maxn;
    int autotuned;
    double tune_us[4];
    int gs_form;
    int gs_chunks;
    int gs_stages;
    int head_form;
    double gs_tune_us[3];
} otm_config;
OTM_API otm_status otm_get_config(otm_ctx* ctx, otm_config* out);

/* Copy one of the OTM_FIELD_* arrays (as of the last homogenize or step) out
 * as floats; `count` must equal its length (n^3 or 3 n^3). */
OTM_API otm_status otm_get_field(otm_ctx* ctx, int which, float* out, size_t count, int on_device);

/*
 * Homogenized conductivity of a density field (Sec. 2.2, discrete Eq. homo):
 * filter (Sec. 2.3) -> SIMP -> macro loads (Sec. 2.4) -> MG-preconditioned CG
 * for the three load cases (Sec. 2.4, Alg. 3) -> tensor.  rho = NULL uses the
 * context's current density; otherwise rho (n^3 floats, host or device per
 * on_device) is used for this call only and the current density is left
 * unchanged.  kappa_out is a host array of 6 doubles.  info may be NULL.
 * Returns OTM_ENOCONV if some load case missed cg_tol within cg_maxit
 * (kappa_out still filled).
 */
OTM_API otm_status otm_homogenize(otm_ctx* ctx, const float* rho, int on_device,
                                  double kappa_out[6], otm_step_info* info);

/*
 * One design iteration (Alg. 2 with the loop of Sec. 3.4 and model Eq.
 * model3): homogenize the current density, objective and its gradient
 * (Eq. sens with the filter chain rule), Alg. 1 volume bound, OC update of
 * the density.  info may be NULL.  Returns OTM_ENOCONV when the solve missed
 * cg_tol (the update is still applied).
 */
OTM_API otm_status otm_step(otm_ctx* ctx, otm_step_info* info);

/* `iters` calls of otm_step; infos (may be NULL) receives one report each. */
OTM_API otm_status otm_run(otm_ctx* ctx, int iters, otm_step_info* infos);

/*
 * Run `count` independent designs for `iters` iterations each.  params[d],
 * rho0[d] (host, n_d^3 floats; NULL = uniform volfrac) describe design d;
 * rho_out[d] (host, may be NULL), kappa_out[d] (may be NULL: the tensor of
 * the last iteration) and infos[d*iters + i] (may be NULL) receive results.
 * All contexts are created first (device allocation synchronises the
 * device); then up to `workers` host threads (the environment variable
 * OTM_BATCH_WORKERS, default min(count, 16); 1 = one design after another)
 * each take the next design and step it on that design's own stream, so the
 * designs' kernels run concurrently on the GPU.  Each design's results are
 * bitwise those of running it alone (params[d].stream is ignored: every
 * design gets a stream of its own).
 * Returns the first non-OK status in design order (every design is still
 * attempted).
 */
OTM_API otm_status otm_design_batch(int count, const otm_params* params,
                                    const float* const* rho0, int iters,
                                    float* const* rho_out, double (*kappa_out)[6],
                                    otm_step_info* infos);

/* Checkpoint: serialise density, previous solution, Alg. 1 state and the
 * iteration counter.  With buf == NULL, *len receives the size needed;
 * otherwise *len must be at least that size. */
OTM_API otm_status otm_get_state(otm_ctx* ctx, void* buf, size_t* len);

/* Restore a blob written by otm_get_state for the same n and precision. */
OTM_API otm_status otm_set_state(otm_ctx* ctx, const void* buf, size_t len);

/* Last error message of ctx, or of this thread's context-less calls when
 * ctx is NULL.  Never NULL. */
OTM_API const char* otm_last_error(const otm_ctx* ctx);

/* ------------------------------------------------------- host-side helpers */

/* Initial state of Alg. 1: Df = 1, V* = 1, g^[0] = 1, gap = 0, count = 0. */
OTM_API otm_status otm_governor_init(otm_governor_state* s);

/* One pass of the loop body of Alg. 1 (Sec. 2.3) after the objective g of
 * the current design is known: lowBound = mean filtered rho^p, vol = mean
 * rho.  Uses p->gov_bound, gov_small_rel and gov_vol_tol.  Host only; the
 * same function runs on the device inside otm_step. */
OTM_API otm_status otm_governor_update(otm_governor_state* s, const otm_params* p,
                                       double g, double low_bound, double vol);

/* ------------------------------------------- operator-level entry points
 * For testing and profiling single kernels.  All pointers are device
 * pointers on the current device; `dtype` is OTM_FP32 (float arrays) or
 * OTM_FP64 (double arrays); work is ordered on `stream` (cudaStream_t, NULL
 * = legacy default stream) and completes before return.  Sizes: n as in
 * otm_params, fields n^3, three-load-case fields 3 n^3.                   */

/* Density filter of Sec. 2.3 with weight max(0, r - d) over the periodic
 * neighbourhood d < r, followed by SIMP (Sec. 2.2):
 * rho_f = W rho, k = k_void + rho_f^p (k_solid - k_void). */
OTM_API otm_status otm_op_filter_simp(int dtype, int n, double rmin, double penal,
                                      double k_solid, double k_void,
                                      const void* rho, void* rho_f, void* k, void* stream);

/* Transpose filter s = W^T s_f (the chain rule of Sec. 2.3). */
OTM_API otm_status otm_op_filter_transpose(int dtype, int n, double rmin,
                                           const void* s_f, void* s, void* stream);

/* enforceMacroLoad (Sec. 2.4): f = three load cases from element
 * conductivities k. */
OTM_API otm_status otm_op_macro_load(int dtype, int n, const void* k, void* f, void* stream);

/* Matrix-free [K u]_v of Sec. 2.4 for three fields u (3 n^3) with element
 * conductivities k: Ku = K(k) u. */
OTM_API otm_status otm_op_apply_K(int dtype, int n, const void* k, const void* u,
                                  void* Ku, void* stream);

/* Same as otm_op_apply_K, but only enqueues the work on `stream` and returns
 * without waiting for it (the stream-ordered form, for timing a kernel with
 * events and for use inside a caller's pipeline).  Argument errors and launch
 * errors are reported; errors during execution surface at the caller's next
 * synchronisation of the stream. */
OTM_API otm_status otm_op_apply_K_async(int dtype, int n, const void* k, const void* u,
                                        void* Ku, void* stream);

/* One colour pass of the Gauss-Seidel relaxation of Sec. 2.4,
 * S_v T_v = f_v - M_v, on the finest grid for the nodes of colour
 * c = (x%2) + 2(y%2) + 4(z%2) in [0, 8) (n even); colour 8 + g, g in [0, 4),
 * relaxes the two colours 2g and 2g + 1 together (they share no matrix
 * entry), the pass the solver runs.  Updates T in place. */
OTM_API otm_status otm_op_gs_colour(int dtype, int n, const void* k, const void* f,
                                    void* T, int colour, void* stream);

/* Homogenized tensor and element sensitivities from a solution: for the
 * element conductivities k and filtered density rho_f, the three solutions
 * chi (3 n^3), kappa_out (host, 6 doubles) = discrete Eq. homo, and
 * s_f (device, n^3, may be NULL) = sum_c w_c d kappa_c / d rho_f (Eq. sens)
 * with weights w (host, 6 doubles). */
OTM_API otm_status otm_op_kappa_sens(int dtype, int n, double penal, double k_solid,
                                     double k_void, const void* k, const void* rho_f,
                                     const void* chi, const double w[6],
                                     double kappa_out[6], void* s_f, void* stream);

/* Same computation and arguments as otm_op_kappa_sens, for callers that must
 * not allocate device memory (for instance inside a host framework that has
 * reserved the device through its own memory pool, or in a loop that cannot
 * afford an allocation's possible synchronisation).  The paper has no
 * counterpart: this is a deployment variant.  Its reduction scratch is a
 * fixed device array inside the library (about 50 KB, held on every GPU that
 * loads the library until the process exits); no cudaMalloc, cudaFree or
 * other allocating call is made.  Limit: n <= 512.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  All
 * calls share the scratch and it keeps the last call's contents (the call
 * clears what must start at zero); calls whose GPU work overlaps race on it
 * and must be serialised by the caller.  Like the other operator-level
 * calls it waits for its stream before it returns. */
OTM_API otm_status otm_op_kappa_sens_noalloc(int dtype, int n, double penal, double k_solid,
                                             double k_void, const void* k, const void* rho_f,
                                             const void* chi, const double w[6],
                                             double kappa_out[6], void* s_f, void* stream);

/* OC update (Sec. 3.3) of rho with gradient s under volume bound vstar:
 * writes rho_new (which may be the same array as rho), and *lambda_out
 * (host, may be NULL). */
OTM_API otm_status otm_op_oc_update(int dtype, int n, double vstar, double move,
                                    double damp, double rho_min, const void* rho,
                                    const void* s, void* rho_new, double* lambda_out,
                                    void* stream);


/* One iteration of the Method of Moving Asymptotes for model 2 (Eq. model2:
 * minimise V(rho) = mean(rho) subject to g - eps <= 0, 0 <= rho <= 1; the
 * MMAOptimizer of Sec. 3.3), on device arrays of n^3 values in dtype:
 *   x       in: the design rho^k; out: rho^(k+1)
 *   dg      dg/drho at rho^k (the constraint's gradient); dV/drho = 1/n^3
 *   xold1, xold2   rho^(k-1), rho^(k-2); out: shifted (xold2 <- xold1 <- x)
 *   low, upp       asymptotes of iteration k-1; out: those of iteration k
 * iter = k (0-based; iterations 0 and 1 place the asymptotes at x -/+ 0.5,
 * later ones adapt them), g = g(kappa^H(rho^k)), eps the bound of the
 * constraint, move the move limit (fraction of the box, Svanberg's 0.5),
 * c and d the weights of the constraint's slack (c y + d y^2 / 2; 1000, 1).
 * xold1, xold2, low and upp are only read from iteration 2 on, but must be
 * finite.  *lambda_out (host, may be NULL) receives the multiplier: 0 when
 * the constraint is inactive, above c when it cannot be met within the move
 * limits.  Errors: OTM_EINVAL for NULL arrays, a bad dtype or n, iter < 0,
 * move outside (0, 1], c < 0, d <= 0 or a non-finite g or eps. */
OTM_API otm_status otm_op_mma_update(int dtype, int n, int iter, double g, double eps, double move,
                                     double c, double d, void* x, const void* dg, void* xold1,
                                     void* xold2, void* low, void* upp, double* lambda_out,
                                     void* stream);

/* Bounds-checking build (libotm built with -DOTM_CHECK).  In that build the
 * kernels with index arithmetic that could leave a buffer -- the tensor-copy
 * coordinates and staged reads of the TMA stencil and group pass, the
 * tcgen05 convolution's operand ranges, the node coordinates of the gather
 * and coarse-level kernels -- test each index against its extent; a failing
 * index is recorded in a device flag word and its access skipped or clamped
 * (nothing traps), and the call that launched the kernel returns OTM_ECUDA
 * with the site, index and bound in otm_last_error.  This call checks the
 * mechanism itself: it evaluates one out-of-range and one in-range index
 * (with no memory access behind either) and sets *fired = 1 when exactly the
 * first was recorded, -1 otherwise.  In the normal build it sets *fired = 0
 * and returns OTM_ESTATE.  Errors: OTM_EINVAL for NULL. */
OTM_API otm_status otm_check_selftest(int* fired);

/* ------------------------------------------------- learned warm start (U-Net)
 *
 * A periodic 3-D convolutional U-Net maps the filtered density rho_f (n^3) to
 * three fields y (3 n^3, load case major) that, times a scale, predict the
 * solutions chi of the three load cases (Sec. 2.4).  The paper has no such
 * network; it is the learned initial guess of the homogenization solve.
 *
 * Architecture (widths c0..c3, grid n, n % 8 == 0):
 *   E0 = B(1 -> c0)(x) at n,  E1 = B(c0 -> c1)(pool E0) at n/2,
 *   E2 = B(c1 -> c2)(pool E1) at n/4,  E3 = B(c2 -> c3)(pool E2) at n/8,
 *   D2 = B(c3 + c2 -> c2)(cat(up E3, E2)),  D1 = B(c2 + c1 -> c1)(cat(up D2, E1)),
 *   D0 = B(c1 + c0 -> c0)(cat(up D1, E0)),  y = H D0 + h (1x1 convolution c0 -> 3),
 * B(a -> b) = relu(conv(relu(conv(., a -> b)), b -> b)) with 3x3x3 circular
 * convolutions with bias, pool the 2x2x2 average, up the nearest x2 copy.
 *
 * Parameters are one FP32 vector, per block in the order E0 E1 E2 E3 D2 D1 D0:
 * W1 [27][a][b], b1 [b], W2 [27][b][b], b2 [b]; then H [c0][3], h [3].  A
 * convolution weight W[t][ci][co] multiplies input channel ci at offset
 * (dx, dy, dz) = (t % 3 - 1, (t / 3) % 3 - 1, t / 9 - 1) for output channel co.
 * Computation: BF16 activations and weights, FP32 accumulation (tensor cores),
 * FP32 master parameters, Adam with beta = (0.9, 0.999), eps = 1e-8.
 *
 * Calls taking a stream order their work on it (NULL = the stream given at
 * creation) and return after it completes.  x, y, target and grads are device
 * pointers on the network's device.  One network serves one caller at a time:
 * its activations are held inside it. */
typedef struct otm_unet otm_unet;

/* Create a network for grid n (8 <= n <= 512, n % 8 == 0) with widths
 * c0..c3 (each a multiple of 16 in [16, 256]) and He-normal initial weights
 * drawn from a counter-based generator seeded by `seed`.  Allocates its
 * parameters, Adam moments and activation buffers on the current device.
 * OTM_EINVAL on bad sizes, OTM_ENOMEM when the buffers do not fit. */
OTM_API otm_status otm_unet_create(int n, const int widths[4], uint64_t seed, void* stream,
                                   otm_unet** out);
OTM_API otm_status otm_unet_destroy(otm_unet* u);
/* Number of FP32 parameters. */
OTM_API otm_status otm_unet_param_count(const otm_unet* u, size_t* count);
/* Copy the parameter vector out of / into the network (count = param_count;
 * host or device memory per on_device).  set resets the Adam moments. */
OTM_API otm_status otm_unet_get_params(otm_unet* u, float* p, int on_device);
OTM_API otm_status otm_unet_set_params(otm_unet* u, const float* p, int on_device);
/* y = net(x): x n^3 FP32, y 3 n^3 FP32 (device). */
OTM_API otm_status otm_unet_forward(otm_unet* u, const float* x, float* y, void* stream);
/* Gradient of sum(dy * y) with respect to every parameter, for the x of the
 * last otm_unet_forward: dy 3 n^3 (device), grads param_count FP32 (device,
 * may be NULL: the gradient then stays inside the network). */
OTM_API otm_status otm_unet_backward(otm_unet* u, const float* dy, float* grads, void* stream);
/* Stored activation of the last otm_unet_forward, converted to FP32, for
 * gradient checks that reuse the network's own activations and ReLU masks:
 * block in [0, 7) (E0 E1 E2 E3 D2 D1 D0, the order of the architecture
 * above), which = 0 the block's input (E0: the BF16 density in channel 0 of
 * 16, the others zero; E1..E3: the pooled input; D2..D0: the concatenation
 * (upsampled coarse, skip)), 1 the first convolution's output after ReLU,
 * 2 the block's output.  out (device, FP32) receives [voxel][C] (voxels x
 * fastest at the block's grid n / 2^level), *channels = C; count = the
 * capacity of out.  OTM_ESTATE without a stored forward pass, OTM_EINVAL
 * for bad indices or a too small out. */
OTM_API otm_status otm_unet_get_activation(otm_unet* u, int block, int which, float* out, size_t count,
                                           int* channels, void* stream);
/* One Adam step on L = mean((net(x) - target / target_scale)^2) over the
 * 3 n^3 entries (target_scale > 0; the predictor's scale when the targets are
 * solutions): forward, loss, backward, update.  *loss (host, may be NULL) =
 * L before the update. */
OTM_API otm_status otm_unet_train_step(otm_unet* u, const float* x, const float* target,
                                       double target_scale, double lr, double* loss, void* stream);
/* L = mean((net(x) - target / target_scale)^2) without an update. */
OTM_API otm_status otm_unet_eval(otm_unet* u, const float* x, const float* target,
                                 double target_scale, double* loss, void* stream);
/* Attach a network (grid n equal to the context's) as the predictor used by
 * OTM_WS_LEARNED, with chi_i ~ scale * y_i; NULL detaches.  Each design
 * iteration that runs the predictor scores four starts per load case by
 * their true residual ||f_i - K x_i|| (zero, the previous solution, the
 * zero-mean prediction, the previous solution plus the prediction's change
 * since the previous iteration) and starts PCG from the best.  A prediction
 * that does not pay -- for no load case is its residual norm at most a
 * quarter of the best start without it -- doubles the number of following
 * iterations that skip the predictor and start from the previous solution
 * (up to 63); one that pays resets it.  The context borrows the network: keep it alive
 * while attached, and do not run other calls on it concurrently with the
 * context's steps. */
OTM_API otm_status otm_set_predictor(otm_ctx* ctx, otm_unet* u, double scale);

/* One 3x3x3 circular convolution of the network (operator-level test entry):
 * out[v][co] = act(bias[co] + sum_t sum_ci w[t][ci][co] in[v + d_t][ci]) on an
 * n^3 grid, BF16 in [n^3][cin], w [27][cin][cout], out [n^3][cout] (channels
 * innermost), bias FP32 (may be NULL), act = relu when relu != 0.  cin and
 * cout multiples of 16, <= 512.  Device pointers. */
OTM_API otm_status otm_op_conv3(int n, int cin, int cout, const void* in, const void* w,
                                const float* bias, int relu, void* out, void* stream);
/* Its weight and bias gradients for output gradient g [n^3][cout] (BF16):
 * dw [27][cin][cout] += sum_v in[v + d_t][ci] g[v][co], db[co] += sum_v g[v][co]
 * (FP32, accumulated into; db may be NULL). */
OTM_API otm_status otm_op_conv3_wgrad(int n, int cin, int cout, const void* in, const void* g,
                                      float* dw, float* db, void* stream);
/* Its input gradient, by the network's own backward path: the FP32 weights
 * w [27][cin][cout] are rounded to BF16 and stored tap-flipped and
 * transposed ([26 - t][co][ci]), and the forward convolution runs on that
 * copy: dx[v][ci] = sum_t sum_co w[t][ci][co] g[v - d_t][co], with g
 * [n^3][cout] and dx [n^3][cin] BF16 (device).  Takes its 2 x 27 cin cout
 * BF16 weight scratch from the stream-ordered allocator (OTM_ENOMEM when it
 * cannot). */
OTM_API otm_status otm_op_conv3_dgrad(int n, int cin, int cout, const void* g, const float* w,
                                      void* dx, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* OTM_H */
