// The learned warm start: a periodic 3-D convolutional U-Net on the filtered
// density (include/otm.h, "learned warm start").  Forward, backward, Adam and
// the two operator-level convolution entry points.
#include <atomic>
#include <cmath>
#include <mutex>
#include <cstring>
#include <string>
#include <vector>

#include "conv_tc05.cuh"
#include "otm_internal.cuh"
#include "unet_kernels.cuh"
#include "unet_api.cuh"

namespace otm {
void set_thread_error(const std::string& msg);
}

using otm::nn::bf16;

namespace {

constexpr int kBlocks = 7;                    // E0 E1 E2 E3 D2 D1 D0
constexpr int kLevel[kBlocks] = {0, 1, 2, 3, 2, 1, 0};

otm_status ufail(otm_status st, const std::string& m) {
    otm::set_thread_error(m);
    return st;
}

#define U_CU(call)                                                                                   \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) {                                                                     \
            otm::set_thread_error(std::string(#call) + ": " + cudaGetErrorString(e_));               \
            return e_ == cudaErrorMemoryAllocation ? OTM_ENOMEM : OTM_ECUDA;                         \
        }                                                                                            \
    } while (0)
#define U_LAUNCH() U_CU(cudaGetLastError())
// stream synchronisation of an entry point; in a checking build a failed
// bounds check in this unit's kernels fails the call
#define U_SYNC(st)                                                                                   \
    do {                                                                                             \
        U_CU(cudaStreamSynchronize(st));                                                             \
        const std::string c_ = otm::check_take();                                                    \
        if (!c_.empty()) {                                                                           \
            otm::set_thread_error(c_);                                                               \
            return OTM_ECUDA;                                                                        \
        }                                                                                            \
    } while (0)
#define U_TRY(x)                                                                                     \
    do {                                                                                             \
        otm_status s_ = (x);                                                                         \
        if (s_ != OTM_OK) return s_;                                                                 \
    } while (0)

int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

int elt_grid(size_t work) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    size_t b = (work + 255) / 256;
    if (b < 1) b = 1;
    if (b > (size_t)sms * 16) b = (size_t)sms * 16;
    return (int)b;
}

std::atomic<long long> g_launches{0};

int pick_bn(int cout) { return cout % 64 == 0 ? 64 : (cout % 32 == 0 ? 32 : 16); }

// Opt in to the brick kernel's dynamic shared memory: once per kernel
// instantiation and device (the attribute belongs to each instantiation;
// this translation unit is the only one that launches them).
template <int BN, bool RL>
cudaError_t tile_prepare() {
    static std::mutex m;
    static bool granted[64] = {};
    std::lock_guard<std::mutex> lock(m);
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (granted[dev]) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(otm::nn::k_conv3_tile<BN, RL>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)otm::nn::conv3_tile_smem(BN));
    if (e == cudaSuccess) granted[dev] = true;
    return e;
}

// Convolution form: 0 tcgen05 one-tile (where it applies), 2 the tcgen05
// z-march form where it applies (OTM_CONV=z; bitwise the same, measured
// slower: its MMA issue waits behind each plane's epilogue and loads), 1 the
// mma.sync kernels (OTM_CONV=mma), for comparisons.
int conv_choice() {
    static int c = [] {
        const char* e = getenv("OTM_CONV");
        if (e && e[0] == 'm') return 1;
        if (e && e[0] == 'z') return 2;
        return 0;
    }();
    return c;
}

// Set by a tcgen05 convolution whose bounded wait ran out.
__device__ int g_conv_err;

// After a synchronised operator call: OTM_ETIMEOUT (and the flag cleared)
// when a tcgen05 convolution's bounded wait ran out.
otm_status conv_flag(const char* what) {
    int e = 0;
    U_CU(cudaMemcpyFromSymbol(&e, g_conv_err, sizeof(int)));
    if (!e) return OTM_OK;
    const int zero = 0;
    cudaMemcpyToSymbol(g_conv_err, &zero, sizeof(int));
    return ufail(OTM_ETIMEOUT, std::string(what) + ": a bounded wait for the tensor-core MMAs ran out");
}

// Opt in to a tcgen05 kernel's dynamic shared memory, only ever raising it
// (Z: the pipelined z-march form).
template <bool RL, bool Z>
cudaError_t tc_prepare(size_t bytes) {
    static std::mutex m;
    static size_t granted[64] = {};
    std::lock_guard<std::mutex> lock(m);
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (bytes <= granted[dev]) return cudaSuccess;
    const cudaError_t e =
        Z ? cudaFuncSetAttribute(otm::nn::k_conv3_tcz<RL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)
          : cudaFuncSetAttribute(otm::nn::k_conv3_tc<RL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) granted[dev] = bytes;
    return e;
}

// z-chunks of the pipelined form: one wave of resident CTAs over the tile
// columns (OTM_CONV_M overrides, for sweeps).
template <bool RL>
int tcz_chunks(int n, int cin, int cout) {
    const char* e = getenv("OTM_CONV_M");
    if (e && atoi(e) >= 1 && atoi(e) <= n) return atoi(e);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, otm::nn::k_conv3_tcz<RL>, 128,
                                                      otm::nn::conv3_tcz_smem(cin, cout)) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const long long cols = (long long)(n / otm::nn::kTcX) * (n / otm::nn::kTcY);
    long long mm = ((long long)per_sm * sm_count() + cols - 1) / cols;
    if (mm < 1) mm = 1;
    if (mm > n / 2) mm = n / 2;
    return (int)mm;
}

// out = act(conv3(in) + bias).  wtc: the weights already in the tcgen05
// kernel's packed layout (k_pack_w_tc), or NULL to pack them here into
// stream-ordered scratch.
otm_status conv3(int n, int cin, int cout, const bf16* in, const bf16* w, const float* bias, bool relu, bf16* out,
                 cudaStream_t st, const bf16* wtc = nullptr) {
    const size_t N = (size_t)n * n * n;
    if (conv_choice() != 1 && otm::nn::conv3_tc_ok(n, cin, cout)) {
        const bool zform = conv_choice() == 2 && otm::nn::conv3_tcz_ok(n, cin, cout);
        const size_t smem = zform ? otm::nn::conv3_tcz_smem(cin, cout) : otm::nn::conv3_tc_smem(cout);
        const cudaError_t e = zform ? (relu ? tc_prepare<true, true>(smem) : tc_prepare<false, true>(smem))
                                    : (relu ? tc_prepare<true, false>(smem) : tc_prepare<false, false>(smem));
        if (e != cudaSuccess) return ufail(OTM_ECUDA, std::string("conv3 (tcgen05) shared-memory opt-in: ") + cudaGetErrorString(e));
        bf16* scratch = nullptr;
        if (!wtc) {
            const size_t M = (size_t)27 * cin * cout;
            U_CU(cudaMallocAsync((void**)&scratch, M * sizeof(bf16), st));
            otm::nn::k_pack_w_tc<<<elt_grid(M), 256, 0, st>>>(cin, cout, w, scratch);
            g_launches += 1;
            wtc = scratch;
        }
        int* err = nullptr;
        U_CU(cudaGetSymbolAddress((void**)&err, g_conv_err));
        if (zform) {
            const int m = relu ? tcz_chunks<true>(n, cin, cout) : tcz_chunks<false>(n, cin, cout);
            const unsigned grid = (unsigned)((n / otm::nn::kTcX) * (n / otm::nn::kTcY) * m);
            if (relu)
                otm::nn::k_conv3_tcz<true><<<grid, 128, smem, st>>>(n, cin, cout, m, in, wtc, bias, out, err);
            else
                otm::nn::k_conv3_tcz<false><<<grid, 128, smem, st>>>(n, cin, cout, m, in, wtc, bias, out, err);
        } else {
            const unsigned grid = (unsigned)((n / otm::nn::kTcX) * (n / otm::nn::kTcY) * n);
            if (relu)
                otm::nn::k_conv3_tc<true><<<grid, 128, smem, st>>>(n, cin, cout, in, wtc, bias, out, err);
            else
                otm::nn::k_conv3_tc<false><<<grid, 128, smem, st>>>(n, cin, cout, in, wtc, bias, out, err);
        }
        g_launches += 1;
        if (scratch) cudaFreeAsync(scratch, st);
        U_LAUNCH();
        return OTM_OK;
    }
    if (otm::nn::conv3_tile_ok(n) && cout % 16 == 0 && cin % 16 == 0) {
        // 32 output channels per CTA, unless that leaves a small grid with
        // fewer CTAs than SMs (the 16^3 level): then 16, for twice the CTAs
        const long long bricks = (long long)(n / otm::nn::kBX) * (n / otm::nn::kBY) * (n / otm::nn::kBZ);
        int tb = cout % 32 == 0 ? 32 : 16;
        if (tb == 32 && bricks * (cout / 32) < sm_count()) tb = 16;
        const dim3 grid((unsigned)bricks, (unsigned)(cout / tb));
        const size_t smem = otm::nn::conv3_tile_smem(tb);
        cudaError_t e = cudaSuccess;
#define TILE_CASE(BN, RL)                                                                                  \
    if (tb == BN && relu == RL) {                                                                          \
        e = tile_prepare<BN, RL>();                                                                        \
        if (e == cudaSuccess)                                                                              \
            otm::nn::k_conv3_tile<BN, RL><<<grid, 256, smem, st>>>(n, cin, cout, in, w, bias, out);        \
    }
        TILE_CASE(16, true) TILE_CASE(16, false) TILE_CASE(32, true) TILE_CASE(32, false)
#undef TILE_CASE
        if (e != cudaSuccess) return ufail(OTM_ECUDA, std::string("conv3 shared-memory opt-in: ") + cudaGetErrorString(e));
        g_launches += 1;
        U_LAUNCH();
        return OTM_OK;
    }
    const int bn = pick_bn(cout);
    dim3 grid((unsigned)((N + otm::nn::kCM - 1) / otm::nn::kCM), (unsigned)(cout / bn));
#define CONV_CASE(BN)                                                                                  \
    if (bn == BN) {                                                                                    \
        if (relu) otm::nn::k_conv3<BN, true><<<grid, 128, 0, st>>>(n, cin, cout, in, w, bias, out);   \
        else otm::nn::k_conv3<BN, false><<<grid, 128, 0, st>>>(n, cin, cout, in, w, bias, out);       \
    }
    CONV_CASE(64) else CONV_CASE(32) else CONV_CASE(16)
#undef CONV_CASE
    g_launches += 1;
    U_LAUNCH();
    return OTM_OK;
}

template <int BN>
cudaError_t dw_tile_prepare() {
    static std::mutex m;
    static bool granted[64] = {};
    std::lock_guard<std::mutex> lock(m);
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (granted[dev]) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(otm::nn::k_conv3_dw_tile<BN>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)otm::nn::conv3_dw_tile_smem(BN));
    if (e == cudaSuccess) granted[dev] = true;
    return e;
}

// dW[27][ca][cout] += ..., db += ... (in stored with cin >= ca channels)
otm_status conv3_wgrad(int n, int cin, int ca, int cout, const bf16* in, const bf16* g, float* dw, float* db,
                       cudaStream_t st) {
    const size_t N = (size_t)n * n * n;
    if (otm::nn::conv3_tile_ok(n) && cin % 16 == 0 && cout % 16 == 0) {
        const int tb = cout % 32 == 0 ? 32 : 16;
        int sms = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int nbricks = (n / otm::nn::kBX) * (n / otm::nn::kBY) * (n / otm::nn::kBZ);
        const int per = (cin / 16) * (cout / tb);
        int P = (3 * (sms > 0 ? sms : 1) + per - 1) / per;
        if (P > nbricks) P = nbricks;
        if (P < 1) P = 1;
        const dim3 grid((unsigned)P, (unsigned)(cin / 16), (unsigned)(cout / tb));
        const size_t smem = otm::nn::conv3_dw_tile_smem(tb);
        cudaError_t e;
        if (tb == 32) {
            e = dw_tile_prepare<32>();
            if (e == cudaSuccess) otm::nn::k_conv3_dw_tile<32><<<grid, 256, smem, st>>>(n, cin, ca, cout, in, g, dw, db);
        } else {
            e = dw_tile_prepare<16>();
            if (e == cudaSuccess) otm::nn::k_conv3_dw_tile<16><<<grid, 256, smem, st>>>(n, cin, ca, cout, in, g, dw, db);
        }
        if (e != cudaSuccess) return ufail(OTM_ECUDA, std::string("conv3_wgrad shared-memory opt-in: ") + cudaGetErrorString(e));
        g_launches += 1;
        U_LAUNCH();
        return OTM_OK;
    }
    const int bn = pick_bn(cout);
    const long long per = 27LL * (cin / 16) * (cout / bn);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long want = ((long long)(sms > 0 ? sms : 1) * 16 + per - 1) / per;
    long long chunk = ((long long)N + want - 1) / (want > 0 ? want : 1);
    chunk = (chunk + 63) / 64 * 64;
    if (chunk < 64) chunk = 64;
    const long long chunks = ((long long)N + chunk - 1) / chunk;
    dim3 grid((unsigned)chunks, (unsigned)(cin / 16), (unsigned)(27 * (cout / bn)));
    if (bn == 64) otm::nn::k_conv3_dw<64><<<grid, 128, 0, st>>>(n, cin, ca, cout, (int)chunk, in, g, dw, db);
    else if (bn == 32) otm::nn::k_conv3_dw<32><<<grid, 128, 0, st>>>(n, cin, ca, cout, (int)chunk, in, g, dw, db);
    else otm::nn::k_conv3_dw<16><<<grid, 128, 0, st>>>(n, cin, ca, cout, (int)chunk, in, g, dw, db);
    g_launches += 1;
    U_LAUNCH();
    return OTM_OK;
}

// Counter-based standard normal: SplitMix64 of (seed, index) feeding the
// Box-Muller transform.
uint64_t splitmix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
double normal_at(uint64_t seed, uint64_t i) {
    const double u1 = ((splitmix64(seed * 0x100000001b3ull + 2 * i) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double u2 = ((splitmix64(seed * 0x100000001b3ull + 2 * i + 1) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

}  // namespace

struct otm_unet {
    int n = 0, c[4] = {}, device = 0;
    cudaStream_t stream = nullptr;
    size_t P = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    int adam_t = 0;
    struct Conv {
        int a = 0, ap = 0, b = 0;
        size_t oW = 0, ob = 0;
        bf16 *Wc = nullptr, *Wt = nullptr;
        bf16 *Wc_tc = nullptr, *Wt_tc = nullptr;   // the same in the tcgen05 kernel's packed layout
    };
    Conv cv[2 * kBlocks];
    int blk_a[kBlocks] = {}, blk_b[kBlocks] = {};
    size_t oHW = 0, oHb = 0;
    int side[4] = {};
    size_t Nl[4] = {};
    // activations
    bf16* x0 = nullptr;                                   // [N0][16]
    bf16 *h1[kBlocks] = {}, *h2[kBlocks] = {};
    bf16 *pin[4] = {};                                    // pooled inputs of E1..E3 (index 1..3)
    bf16 *cat[3] = {};                                    // inputs of D2, D1, D0
    float* y = nullptr;                                   // [3][N0]
    float* dy = nullptr;
    // activation gradients
    bf16 *dE[4] = {}, *dD[3] = {}, *dcat[3] = {}, *dP[4] = {};
    bf16* G1 = nullptr;
    double* loss_d = nullptr;
    double* loss_h = nullptr;
    bool have_forward = false;
    std::vector<void*> owned;

    const bf16* block_in(int k) const {
        if (k == 0) return x0;
        if (k <= 3) return pin[k];
        return cat[k - 4];
    }

    template <class T>
    otm_status alloc(T*& ptr, size_t count) {
        void* q = nullptr;
        U_CU(cudaMalloc(&q, count * sizeof(T) + 64));
        owned.push_back(q);
        ptr = (T*)q;
        return OTM_OK;
    }

    ~otm_unet() {
        for (void* q : owned) cudaFree(q);
        if (loss_h) cudaFreeHost(loss_h);
    }

    otm_status init(int n_, const int w[4], uint64_t seed, cudaStream_t st) {
        n = n_;
        stream = st;
        cudaGetDevice(&device);
        for (int i = 0; i < 4; ++i) c[i] = w[i];
        for (int l = 0; l < 4; ++l) {
            side[l] = n >> l;
            Nl[l] = (size_t)side[l] * side[l] * side[l];
        }
        const int A[kBlocks] = {1, c[0], c[1], c[2], c[3] + c[2], c[2] + c[1], c[1] + c[0]};
        const int B[kBlocks] = {c[0], c[1], c[2], c[3], c[2], c[1], c[0]};
        size_t off = 0;
        for (int k = 0; k < kBlocks; ++k) {
            blk_a[k] = A[k];
            blk_b[k] = B[k];
            Conv& c1 = cv[2 * k];
            c1.a = A[k];
            c1.ap = (A[k] + 15) / 16 * 16;
            c1.b = B[k];
            c1.oW = off;
            off += (size_t)27 * A[k] * B[k];
            c1.ob = off;
            off += B[k];
            Conv& c2 = cv[2 * k + 1];
            c2.a = c2.ap = c2.b = B[k];
            c2.oW = off;
            off += (size_t)27 * B[k] * B[k];
            c2.ob = off;
            off += B[k];
        }
        oHW = off;
        off += (size_t)c[0] * 3;
        oHb = off;
        off += 3;
        P = off;
        U_TRY(alloc(p, P));
        U_TRY(alloc(g, P));
        U_TRY(alloc(m, P));
        U_TRY(alloc(v, P));
        for (auto& q : cv) {
            U_TRY(alloc(q.Wc, (size_t)27 * q.ap * q.b));
            U_TRY(alloc(q.Wt, (size_t)27 * q.ap * q.b));
            U_TRY(alloc(q.Wc_tc, (size_t)27 * q.ap * q.b));
            U_TRY(alloc(q.Wt_tc, (size_t)27 * q.ap * q.b));
        }
        U_TRY(alloc(x0, Nl[0] * 16));
        for (int k = 0; k < kBlocks; ++k) {
            U_TRY(alloc(h1[k], Nl[kLevel[k]] * blk_b[k]));
            U_TRY(alloc(h2[k], Nl[kLevel[k]] * blk_b[k]));
        }
        for (int k = 1; k <= 3; ++k) U_TRY(alloc(pin[k], Nl[k] * c[k - 1]));
        for (int j = 0; j < 3; ++j) {   // D2 (level 2), D1 (1), D0 (0)
            const int lev = 2 - j;
            U_TRY(alloc(cat[j], Nl[lev] * (c[lev + 1] + c[lev])));
            U_TRY(alloc(dcat[j], Nl[lev] * (c[lev + 1] + c[lev])));
            U_TRY(alloc(dD[j], Nl[lev] * c[lev]));
        }
        for (int l = 0; l < 4; ++l) U_TRY(alloc(dE[l], Nl[l] * c[l]));
        for (int l = 1; l <= 3; ++l) U_TRY(alloc(dP[l], Nl[l] * c[l - 1]));
        size_t g1 = 0;
        for (int k = 0; k < kBlocks; ++k) g1 = std::max(g1, Nl[kLevel[k]] * (size_t)blk_b[k]);
        U_TRY(alloc(G1, g1));
        U_TRY(alloc(y, 3 * Nl[0]));
        U_TRY(alloc(dy, 3 * Nl[0]));
        U_TRY(alloc(loss_d, 1));
        U_CU(cudaMallocHost((void**)&loss_h, sizeof(double)));
        // He-normal initial parameters (host, counter-based), zero Adam moments
        std::vector<float> h(P, 0.f);
        uint64_t idx = 0;
        for (int k = 0; k < 2 * kBlocks; ++k) {
            const Conv& q = cv[k];
            const double sd = std::sqrt(2.0 / (27.0 * q.a));
            for (size_t i = 0; i < (size_t)27 * q.a * q.b; ++i) h[q.oW + i] = (float)(sd * normal_at(seed, idx++));
            for (int i = 0; i < q.b; ++i) h[q.ob + i] = (float)(0.01 * normal_at(seed, idx++));
        }
        const double sh = std::sqrt(1.0 / c[0]);
        for (int i = 0; i < c[0] * 3; ++i) h[oHW + i] = (float)(sh * normal_at(seed, idx++));
        U_CU(cudaMemcpyAsync(p, h.data(), P * sizeof(float), cudaMemcpyHostToDevice, stream));
        U_TRY(reset_moments(stream));
        U_TRY(pack(stream));
        U_SYNC(stream);
        return OTM_OK;
    }

    otm_status reset_moments(cudaStream_t st) {
        U_CU(cudaMemsetAsync(m, 0, P * sizeof(float), st));
        U_CU(cudaMemsetAsync(v, 0, P * sizeof(float), st));
        adam_t = 0;
        return OTM_OK;
    }

    // BF16 compute copies of the convolution weights (and the flipped,
    // transposed copies used by the input-gradient convolutions)
    otm_status pack(cudaStream_t st) {
        for (auto& q : cv) {
            const size_t M = (size_t)27 * q.ap * q.b;
            otm::nn::k_pack_w<<<elt_grid(M), 256, 0, st>>>(q.a, q.ap, q.b, p + q.oW, q.Wc, q.Wt);
            if (q.ap % 16 == 0 && q.b % 16 == 0) {
                otm::nn::k_pack_w_tc<<<elt_grid(M), 256, 0, st>>>(q.ap, q.b, q.Wc, q.Wc_tc);
                otm::nn::k_pack_w_tc<<<elt_grid(M), 256, 0, st>>>(q.b, q.ap, q.Wt, q.Wt_tc);
            }
        }
        g_launches += 1;
        U_LAUNCH();
        return OTM_OK;
    }

    otm_status block_fwd(int k, cudaStream_t st) {
        const int ns = side[kLevel[k]];
        const Conv &q1 = cv[2 * k], &q2 = cv[2 * k + 1];
        U_TRY(conv3(ns, q1.ap, q1.b, block_in(k), q1.Wc, p + q1.ob, true, h1[k], st, q1.Wc_tc));
        U_TRY(conv3(ns, q2.ap, q2.b, h1[k], q2.Wc, p + q2.ob, true, h2[k], st, q2.Wc_tc));
        return OTM_OK;
    }

    // keep_input: also store the padded input (the first layer's weight
    // gradient needs it); a prediction alone does not.
    template <class T>
    otm_status forward(const T* x, cudaStream_t st, bool keep_input = true) {
        const bool direct = cv[0].b <= 64;   // first convolution on the CUDA cores (k_conv3_in1)
        if (keep_input || !direct) {
            otm::nn::k_input16<T><<<elt_grid(Nl[0]), 256, 0, st>>>(Nl[0], x, x0);
            g_launches += 1;
            U_LAUNCH();
        }
        for (int k = 0; k < 4; ++k) {
            if (k > 0) {
                const size_t M = Nl[k] * c[k - 1];
                otm::nn::k_pool<<<elt_grid(M), 256, 0, st>>>(side[k], c[k - 1], h2[k - 1], pin[k]);
                g_launches += 1;
                U_LAUNCH();
                U_TRY(block_fwd(k, st));
            } else if (!direct) {
                U_TRY(block_fwd(0, st));
            } else {
                // block 0: the first convolution straight from the density
                const Conv &q1 = cv[0], &q2 = cv[1];
                otm::nn::k_conv3_in1<T><<<elt_grid(Nl[0]), 256, 0, st>>>(side[0], x, q1.Wc, q1.ap, q1.b, p + q1.ob,
                                                                          h1[0]);
                g_launches += 1;
                U_LAUNCH();
                U_TRY(conv3(side[0], q2.ap, q2.b, h1[0], q2.Wc, p + q2.ob, true, h2[0], st, q2.Wc_tc));
            }
        }
        // D2 <- (E3, E2), D1 <- (D2, E1), D0 <- (D1, E0)
        const bf16* coarse[3] = {h2[3], h2[4], h2[5]};
        const bf16* skip[3] = {h2[2], h2[1], h2[0]};
        for (int j = 0; j < 3; ++j) {
            const int lev = 2 - j;
            const size_t M = Nl[lev] * (c[lev + 1] + c[lev]);
            otm::nn::k_up_cat<<<elt_grid(M), 256, 0, st>>>(side[lev], c[lev + 1], c[lev], coarse[j], skip[j], cat[j]);
            g_launches += 1;
            U_LAUNCH();
            U_TRY(block_fwd(4 + j, st));
        }
        otm::nn::k_head<<<elt_grid(Nl[0]), 256, 0, st>>>(Nl[0], c[0], h2[6], p + oHW, p + oHb, y);
        g_launches += 1;
        U_LAUNCH();
        have_forward = keep_input;
        return OTM_OK;
    }

    // Backward through block k from the gradient G2 of its output (modified
    // in place); dx (may be null) receives the gradient of its input.
    otm_status block_bwd(int k, bf16* G2, bf16* dx, cudaStream_t st) {
        const int ns = side[kLevel[k]];
        const size_t N = Nl[kLevel[k]];
        const Conv &q1 = cv[2 * k], &q2 = cv[2 * k + 1];
        otm::nn::k_relu_mask<<<elt_grid(N * q2.b), 256, 0, st>>>(N * q2.b, G2, h2[k]);
        g_launches += 1;
        U_LAUNCH();
        U_TRY(conv3_wgrad(ns, q2.ap, q2.a, q2.b, h1[k], G2, g + q2.oW, g + q2.ob, st));
        U_TRY(conv3(ns, q2.b, q2.ap, G2, q2.Wt, nullptr, false, G1, st, q2.Wt_tc));
        otm::nn::k_relu_mask<<<elt_grid(N * q1.b), 256, 0, st>>>(N * q1.b, G1, h1[k]);
        g_launches += 1;
        U_LAUNCH();
        U_TRY(conv3_wgrad(ns, q1.ap, q1.a, q1.b, block_in(k), G1, g + q1.oW, g + q1.ob, st));
        if (dx) U_TRY(conv3(ns, q1.b, q1.ap, G1, q1.Wt, nullptr, false, dx, st, q1.Wt_tc));
        return OTM_OK;
    }

    // parameter gradient of sum(dy * y) into g (y of the last forward)
    otm_status backward(const float* dyp, cudaStream_t st) {
        U_CU(cudaMemsetAsync(g, 0, P * sizeof(float), st));
        otm::nn::k_head_back<<<elt_grid(Nl[0]), 256, 0, st>>>(Nl[0], c[0], h2[6], p + oHW, dyp, dD[2] /*D0 out*/,
                                                              g + oHW, g + oHb);
        g_launches += 1;
        U_LAUNCH();
        // dD[j] is the gradient of block (D2, D1, D0)[j]'s output: D0 is j = 2
        // D0 -> dcat[2] -> (dD[1], dE[0]);  D1 -> dcat[1] -> (dD[0], dE[1]);
        // D2 -> dcat[0] -> (dE[3], dE[2])
        U_TRY(block_bwd(6, dD[2], dcat[2], st));
        otm::nn::k_up_cat_back<<<elt_grid(Nl[0] * c[0]), 256, 0, st>>>(side[0], c[1], c[0], dcat[2], dD[1], dE[0]);
        g_launches += 1;
        U_LAUNCH();
        U_TRY(block_bwd(5, dD[1], dcat[1], st));
        otm::nn::k_up_cat_back<<<elt_grid(Nl[1] * c[1]), 256, 0, st>>>(side[1], c[2], c[1], dcat[1], dD[0], dE[1]);
        g_launches += 1;
        U_LAUNCH();
        U_TRY(block_bwd(4, dD[0], dcat[0], st));
        otm::nn::k_up_cat_back<<<elt_grid(Nl[2] * c[2]), 256, 0, st>>>(side[2], c[3], c[2], dcat[0], dE[3], dE[2]);
        g_launches += 1;
        U_LAUNCH();
        for (int k = 3; k >= 1; --k) {
            U_TRY(block_bwd(k, dE[k], dP[k], st));
            otm::nn::k_pool_back_add<<<elt_grid(Nl[k - 1] * c[k - 1]), 256, 0, st>>>(side[k - 1], c[k - 1], dP[k],
                                                                                       dE[k - 1]);
            g_launches += 1;
            U_LAUNCH();
        }
        U_TRY(block_bwd(0, dE[0], nullptr, st));
        return OTM_OK;
    }

    otm_status loss(const float* target, double tscale, cudaStream_t st) {
        U_CU(cudaMemsetAsync(loss_d, 0, sizeof(double), st));
        otm::nn::k_mse<<<elt_grid(3 * Nl[0]), 256, 0, st>>>(3 * Nl[0], y, target, (float)(1.0 / tscale), dy, loss_d);
        g_launches += 1;
        U_LAUNCH();
        return OTM_OK;
    }

    otm_status adam(double lr, cudaStream_t st) {
        adam_t += 1;
        const double b1 = 0.9, b2 = 0.999;
        const float c1 = (float)(1.0 / (1.0 - std::pow(b1, adam_t)));
        const float c2 = (float)(1.0 / (1.0 - std::pow(b2, adam_t)));
        otm::nn::k_adam<<<elt_grid(P), 256, 0, st>>>(P, p, g, m, v, (float)lr, (float)b1, (float)b2, 1e-8f, c1, c2);
        g_launches += 1;
        U_LAUNCH();
        return pack(st);
    }
};

namespace otm {

otm_status unet_predict(otm_unet* u, const void* x, bool x_double, float* y, cudaStream_t st) {
    if (x_double) U_TRY(u->forward((const double*)x, st, false));
    else U_TRY(u->forward((const float*)x, st, false));
    U_CU(cudaMemcpyAsync(y, u->y, 3 * u->Nl[0] * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return OTM_OK;
}

int unet_grid(const otm_unet* u) { return u ? u->n : 0; }

long long unet_launches() { return g_launches.load(); }

}  // namespace otm

namespace {
cudaStream_t pick(const otm_unet* u, void* s) { return s ? (cudaStream_t)s : u->stream; }
}  // namespace

extern "C" {

OTM_API otm_status otm_unet_create(int n, const int widths[4], uint64_t seed, void* stream, otm_unet** out) {
    if (!out) return ufail(OTM_EINVAL, "otm_unet_create: out is NULL");
    *out = nullptr;
    if (!widths) return ufail(OTM_EINVAL, "otm_unet_create: widths is NULL");
    if (n < 8 || n > 512 || n % 8) return ufail(OTM_EINVAL, "otm_unet_create: n must be a multiple of 8 in [8, 512]");
    for (int i = 0; i < 4; ++i)
        if (widths[i] < 16 || widths[i] > 256 || widths[i] % 16)
            return ufail(OTM_EINVAL, "otm_unet_create: widths must be multiples of 16 in [16, 256]");
    otm_unet* u = new (std::nothrow) otm_unet();
    if (!u) return ufail(OTM_ENOMEM, "otm_unet_create: host allocation failed");
    otm_status st = u->init(n, widths, seed, (cudaStream_t)stream);
    if (st != OTM_OK) {
        delete u;
        return st;
    }
    *out = u;
    return OTM_OK;
}

OTM_API otm_status otm_unet_destroy(otm_unet* u) {
    if (!u) return OTM_OK;
    cudaStreamSynchronize(u->stream);
    delete u;
    return OTM_OK;
}

OTM_API otm_status otm_unet_param_count(const otm_unet* u, size_t* count) {
    if (!u || !count) return ufail(OTM_EINVAL, "otm_unet_param_count: NULL argument");
    *count = u->P;
    return OTM_OK;
}

OTM_API otm_status otm_unet_get_params(otm_unet* u, float* p, int on_device) {
    if (!u || !p) return ufail(OTM_EINVAL, "otm_unet_get_params: NULL argument");
    U_CU(cudaMemcpyAsync(p, u->p, u->P * sizeof(float), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                         u->stream));
    U_SYNC(u->stream);
    return OTM_OK;
}

OTM_API otm_status otm_unet_set_params(otm_unet* u, const float* p, int on_device) {
    if (!u || !p) return ufail(OTM_EINVAL, "otm_unet_set_params: NULL argument");
    U_CU(cudaMemcpyAsync(u->p, p, u->P * sizeof(float), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                         u->stream));
    U_TRY(u->reset_moments(u->stream));
    U_TRY(u->pack(u->stream));
    U_SYNC(u->stream);
    return OTM_OK;
}

OTM_API otm_status otm_unet_forward(otm_unet* u, const float* x, float* y, void* stream) {
    if (!u || !x || !y) return ufail(OTM_EINVAL, "otm_unet_forward: NULL argument");
    cudaStream_t st = pick(u, stream);
    U_TRY(u->forward(x, st));
    U_CU(cudaMemcpyAsync(y, u->y, 3 * u->Nl[0] * sizeof(float), cudaMemcpyDeviceToDevice, st));
    U_SYNC(st);
    return OTM_OK;
}

OTM_API otm_status otm_unet_backward(otm_unet* u, const float* dy, float* grads, void* stream) {
    if (!u || !dy) return ufail(OTM_EINVAL, "otm_unet_backward: NULL argument");
    if (!u->have_forward) return ufail(OTM_ESTATE, "otm_unet_backward: no forward pass to differentiate");
    cudaStream_t st = pick(u, stream);
    U_TRY(u->backward(dy, st));
    if (grads) U_CU(cudaMemcpyAsync(grads, u->g, u->P * sizeof(float), cudaMemcpyDeviceToDevice, st));
    U_SYNC(st);
    return OTM_OK;
}

OTM_API otm_status otm_unet_get_activation(otm_unet* u, int block, int which, float* out, size_t count,
                                           int* channels, void* stream) {
    if (!u || !out || !channels) return ufail(OTM_EINVAL, "otm_unet_get_activation: NULL argument");
    if (block < 0 || block >= kBlocks || which < 0 || which > 2)
        return ufail(OTM_EINVAL, "otm_unet_get_activation: block must be in [0, 7) and which in [0, 2]");
    if (!u->have_forward) return ufail(OTM_ESTATE, "otm_unet_get_activation: no stored forward pass");
    const size_t N = u->Nl[kLevel[block]];
    const int C = which == 0 ? (block == 0 ? 16 : u->cv[2 * block].ap) : u->blk_b[block];
    const bf16* src = which == 0 ? u->block_in(block) : (which == 1 ? u->h1[block] : u->h2[block]);
    if (count < N * C) return ufail(OTM_EINVAL, "otm_unet_get_activation: out holds fewer than N * C values");
    cudaStream_t st = pick(u, stream);
    otm::nn::k_bf16_to_f32<<<elt_grid(N * C), 256, 0, st>>>(N * C, src, out);
    U_LAUNCH();
    U_SYNC(st);
    *channels = C;
    return OTM_OK;
}

OTM_API otm_status otm_unet_train_step(otm_unet* u, const float* x, const float* target, double target_scale,
                                       double lr, double* loss, void* stream) {
    if (!u || !x || !target) return ufail(OTM_EINVAL, "otm_unet_train_step: NULL argument");
    if (!(target_scale > 0.0 && std::isfinite(target_scale)))
        return ufail(OTM_EINVAL, "otm_unet_train_step: target_scale must be finite and > 0");
    if (!(lr >= 0.0 && std::isfinite(lr))) return ufail(OTM_EINVAL, "otm_unet_train_step: lr must be finite, >= 0");
    cudaStream_t st = pick(u, stream);
    U_TRY(u->forward(x, st));
    U_TRY(u->loss(target, target_scale, st));
    U_TRY(u->backward(u->dy, st));
    U_TRY(u->adam(lr, st));
    U_CU(cudaMemcpyAsync(u->loss_h, u->loss_d, sizeof(double), cudaMemcpyDeviceToHost, st));
    U_SYNC(st);
    if (loss) *loss = *u->loss_h;
    return OTM_OK;
}

OTM_API otm_status otm_unet_eval(otm_unet* u, const float* x, const float* target, double target_scale, double* loss,
                                 void* stream) {
    if (!u || !x || !target || !loss) return ufail(OTM_EINVAL, "otm_unet_eval: NULL argument");
    if (!(target_scale > 0.0 && std::isfinite(target_scale)))
        return ufail(OTM_EINVAL, "otm_unet_eval: target_scale must be finite and > 0");
    cudaStream_t st = pick(u, stream);
    U_TRY(u->forward(x, st));
    U_TRY(u->loss(target, target_scale, st));
    U_CU(cudaMemcpyAsync(u->loss_h, u->loss_d, sizeof(double), cudaMemcpyDeviceToHost, st));
    U_SYNC(st);
    *loss = *u->loss_h;
    return OTM_OK;
}

OTM_API otm_status otm_op_conv3(int n, int cin, int cout, const void* in, const void* w, const float* bias, int relu,
                                void* out, void* stream) {
    if (n < 1 || n > 512) return ufail(OTM_EINVAL, "otm_op_conv3: n must be in [1, 512]");
    if (cin < 16 || cin > 512 || cin % 16 || cout < 16 || cout > 512 || cout % 16)
        return ufail(OTM_EINVAL, "otm_op_conv3: cin and cout must be multiples of 16 in [16, 512]");
    if (!in || !w || !out) return ufail(OTM_EINVAL, "otm_op_conv3: NULL pointer");
    cudaStream_t st = (cudaStream_t)stream;
    U_TRY(conv3(n, cin, cout, (const bf16*)in, (const bf16*)w, bias, relu != 0, (bf16*)out, st));
    U_SYNC(st);
    return conv_flag("otm_op_conv3");
}

OTM_API otm_status otm_op_conv3_dgrad(int n, int cin, int cout, const void* g, const float* w, void* dx,
                                      void* stream) {
    if (n < 1 || n > 512) return ufail(OTM_EINVAL, "otm_op_conv3_dgrad: n must be in [1, 512]");
    if (cin < 16 || cin > 512 || cin % 16 || cout < 16 || cout > 512 || cout % 16)
        return ufail(OTM_EINVAL, "otm_op_conv3_dgrad: cin and cout must be multiples of 16 in [16, 512]");
    if (!g || !w || !dx) return ufail(OTM_EINVAL, "otm_op_conv3_dgrad: NULL pointer");
    cudaStream_t st = (cudaStream_t)stream;
    // the network's own input-gradient path: pack the FP32 weights into the
    // BF16 copy and its tap-flipped, transposed copy (k_pack_w), then run the
    // forward convolution on the transposed copy
    const size_t M = (size_t)27 * cin * cout;
    bf16 *wc = nullptr, *wt = nullptr;
    U_CU(cudaMallocAsync((void**)&wc, M * sizeof(bf16), st));
    cudaError_t e = cudaMallocAsync((void**)&wt, M * sizeof(bf16), st);
    if (e != cudaSuccess) {
        cudaFreeAsync(wc, st);
        return ufail(OTM_ENOMEM, "otm_op_conv3_dgrad: scratch");
    }
    otm::nn::k_pack_w<<<elt_grid(M), 256, 0, st>>>(cin, cin, cout, w, wc, wt);
    otm_status s2 = conv3(n, cout, cin, (const bf16*)g, wt, nullptr, false, (bf16*)dx, st);
    cudaFreeAsync(wc, st);
    cudaFreeAsync(wt, st);
    if (s2 != OTM_OK) return s2;
    U_SYNC(st);
    return conv_flag("otm_op_conv3_dgrad");
}

OTM_API otm_status otm_op_conv3_wgrad(int n, int cin, int cout, const void* in, const void* g, float* dw, float* db,
                                      void* stream) {
    if (n < 1 || n > 512) return ufail(OTM_EINVAL, "otm_op_conv3_wgrad: n must be in [1, 512]");
    if (cin < 16 || cin > 512 || cin % 16 || cout < 16 || cout > 512 || cout % 16)
        return ufail(OTM_EINVAL, "otm_op_conv3_wgrad: cin and cout must be multiples of 16 in [16, 512]");
    if (!in || !g || !dw) return ufail(OTM_EINVAL, "otm_op_conv3_wgrad: NULL pointer");
    cudaStream_t st = (cudaStream_t)stream;
    U_TRY(conv3_wgrad(n, cin, cin, cout, (const bf16*)in, (const bf16*)g, dw, db, st));
    U_SYNC(st);
    return OTM_OK;
}

}  // extern "C"
