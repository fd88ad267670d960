// otm_op_kappa_sens_noalloc: the homogenized tensor and element
// sensitivities of otm_op_kappa_sens, for callers that must not allocate
// device memory.
//
// Who needs it: some callers cannot call cudaMalloc/cudaFree (or the
// stream-ordered allocator) at all -- e.g. code embedded in a host framework
// that has reserved the whole device through its own memory pool and forbids
// direct allocations, or a loop with a hard latency budget in which an
// allocation's possible device synchronisation is unacceptable.  The regular
// entry point takes its reduction scratch from the stream-ordered allocator;
// this one uses a fixed scratch area compiled into the library instead.
//
// The scratch is a file-scope device array.  Every GPU that loads the library
// holds it (kScratchBytes) until the process exits.  All calls share it and
// it keeps the last call's contents: the ticket counter the reduction needs
// at zero is cleared at the start of every call, and every other word is
// written before it is read.  Calls whose GPU work overlaps (two streams, or
// two host threads) race on the scratch and must be serialised by the caller.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "kernels_design.cuh"
#include "otm_internal.cuh"

namespace otm {
void set_thread_error(const std::string& msg);
}

namespace {

// Layout: [ticket counter (256 B)] [DesignScalars (rounded up to 256 B)]
//         [partial sums: kMaxBlocks x kVals doubles]
constexpr int kMaxBlocks = 1024;      // grid cap of the kernels launched here
constexpr int kVals = 6;              // values reduced per block by k_kappa
constexpr size_t kCounterBytes = 256;
constexpr size_t kScalarsBytes = (sizeof(otm::DesignScalars) + 255) / 256 * 256;
constexpr size_t kPartialBytes = (size_t)kMaxBlocks * kVals * sizeof(double);
constexpr size_t kScratchBytes = kCounterBytes + kScalarsBytes + kPartialBytes;   // about 50 KB
constexpr int kMaxN = 512;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device ordinal.  In host code the
// array's name is only a host-side stand-in, so the address is looked up
// with cudaGetSymbolAddress once per device, with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

otm_status fail(otm_status st, const std::string& m) {
    otm::set_thread_error(m);
    return st;
}

otm_status scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(OTM_EINVAL, "otm_op_kappa_sens_noalloc: device ordinal too large");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(OTM_ECUDA, std::string("otm_op_kappa_sens_noalloc: cudaGetSymbolAddress failed: ") +
                                       cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    *out = (unsigned char*)g_addr[dev];
    return OTM_OK;
}

otm::SimpP simp_p(double penal, double ks, double kv, size_t N) {
    otm::SimpP sp;
    memset(&sp, 0, sizeof(sp));
    sp.penal = penal;
    sp.k_solid = ks;
    sp.k_void = kv;
    sp.cubic = penal == 3.0;
    return otm::with_f32(sp, N);
}

template <class R>
otm_status run(int n, double penal, double ks, double kv, const void* k, const void* rho_f, const void* chi,
               const double w[6], double kappa_out[6], void* s_f, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(OTM_ECUDA, std::string("otm_op_kappa_sens_noalloc: ") + cudaGetErrorString(e));
    unsigned char* base = nullptr;
    otm_status s = scratch_address(dev, &base);
    if (s != OTM_OK) return s;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t N = (size_t)n * n * n;
    size_t blocks = (N + 255) / 256;
    const size_t cap = (size_t)(sms > 0 ? sms : 1) * 8;
    if (blocks > cap) blocks = cap;
    if (blocks > (size_t)kMaxBlocks) blocks = kMaxBlocks;
    if (blocks * kVals * sizeof(double) > kPartialBytes)
        return fail(OTM_EINVAL, "otm_op_kappa_sens_noalloc: reduction needs more scratch than compiled in");
    unsigned int* counter = (unsigned int*)base;
    otm::DesignScalars* ds = (otm::DesignScalars*)(base + kCounterBytes);
    double* partials = (double*)(base + kCounterBytes + kScalarsBytes);
    otm::RedBuf rb{partials, counter, (int)blocks};
    // the reduction's ticket counter must start at zero
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return fail(OTM_ECUDA, std::string("otm_op_kappa_sens_noalloc: ") + cudaGetErrorString(e));
    const otm::RowLaunch L = otm::row_launch(n, n * n, (int)blocks);
    rb.max_blocks = L.grid;
    otm::k_kappa<R><<<OTM_ROWS_CFG(L), 0, st>>>(n, (const R*)k, (const R*)chi, rb,
                                                 otm::FinKappa{ds, 1.0 / (double)N, 0});
    if (s_f) {
        e = cudaMemcpyAsync(&ds->w[0], w, 6 * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return fail(OTM_ECUDA, std::string("otm_op_kappa_sens_noalloc: ") + cudaGetErrorString(e));
        otm::k_sens<R><<<OTM_ROWS_CFG(L), 0, st>>>(n, (const R*)rho_f, (const R*)chi, ds, simp_p(penal, ks, kv, (size_t)n * n * n),
                                                    (R*)s_f);
    }
    double kap[6];
    e = cudaMemcpyAsync(kap, &ds->kappa[0], 6 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(OTM_ECUDA, std::string("otm_op_kappa_sens_noalloc: ") + cudaGetErrorString(e));
    for (int c = 0; c < 6; ++c) kappa_out[c] = kap[c];
    return OTM_OK;
}

}  // namespace

extern "C" otm_status otm_op_kappa_sens_noalloc(int dtype, int n, double penal, double k_solid, double k_void,
                                                const void* k, const void* rho_f, const void* chi, const double w[6],
                                                double kappa_out[6], void* s_f, void* stream) {
    if (dtype != OTM_FP32 && dtype != OTM_FP64) return fail(OTM_EINVAL, "otm_op_kappa_sens_noalloc: dtype");
    if (n < 4 || n > kMaxN)
        return fail(OTM_EINVAL, "otm_op_kappa_sens_noalloc: n must be in [4, 512] (fixed scratch limit)");
    if (!k || !chi || !kappa_out) return fail(OTM_EINVAL, "otm_op_kappa_sens_noalloc: NULL input or output");
    if (s_f && (!rho_f || !w)) return fail(OTM_EINVAL, "otm_op_kappa_sens_noalloc: s_f needs rho_f and w");
    if (dtype == OTM_FP64)
        return run<double>(n, penal, k_solid, k_void, k, rho_f, chi, w, kappa_out, s_f, (cudaStream_t)stream);
    return run<float>(n, penal, k_solid, k_void, k, rho_f, chi, w, kappa_out, s_f, (cudaStream_t)stream);
}
