// Bounds-checking build (compile with -DOTM_CHECK).
//
// OTM_BOUND(i, n, site) is true when 0 <= i < n.  In a checking build a false
// result also records the first failure of the translation unit -- site,
// index and bound -- in a device flag word; the caller then skips the access
// or clamps the index, so no access leaves its buffer and nothing traps.
// The host side of each unit reads and clears the flag after its calls
// (check_take) and reports a non-empty result as a failed call.  In the
// normal build OTM_BOUND is the constant true and costs nothing.
#pragma once
#include <cuda_runtime.h>

#include <string>

namespace otm {

enum CheckSite {
    kSiteTmaStencil = 1,   // TMA-staged stencil: copy coordinates, stage bytes, staged reads
    kSiteTmaGs = 2,        // TMA-staged group pass
    kSiteFine = 3,         // finest-level gather kernels (node coordinates)
    kSiteCoarse = 4,       // coarse-level stencil kernels, transfers, cluster levels
    kSiteConvTc = 5,       // tcgen05 convolution: tiles, shared-memory operands, TMEM columns
    kSiteSelftest = 99     // otm_check_selftest
};

#ifdef OTM_CHECK
constexpr bool kCheckBuild = true;
// per translation unit: [0] failures seen, [1] first site, [2] its index (low 32 bits), [3] its bound
static __device__ unsigned int g_check[4];
static __device__ __noinline__ bool check_fail(long long i, long long n, int site) {
    if (atomicAdd(&g_check[0], 1u) == 0u) {
        g_check[1] = (unsigned int)site;
        g_check[2] = (unsigned int)(i & 0xffffffffLL);
        g_check[3] = (unsigned int)(n & 0xffffffffLL);
    }
    return false;
}
#define OTM_BOUND(i, n, site)                                                                  \
    (((unsigned long long)(long long)(i) < (unsigned long long)(long long)(n)) ||             \
     ::otm::check_fail((long long)(i), (long long)(n), (site)))
// Reads and clears this unit's flag; empty when no check failed.
static inline std::string check_take() {
    unsigned int h[4] = {0, 0, 0, 0};
    if (cudaMemcpyFromSymbol(h, g_check, sizeof(h)) != cudaSuccess) return "bounds check: flag unreadable";
    if (h[0] == 0) return std::string();
    const unsigned int z[4] = {0, 0, 0, 0};
    cudaMemcpyToSymbol(g_check, z, sizeof(z));
    return "bounds check failed " + std::to_string(h[0]) + " time(s); first at site " + std::to_string(h[1]) +
           ", index " + std::to_string(h[2]) + " of " + std::to_string(h[3]);
}
#else
constexpr bool kCheckBuild = false;
#define OTM_BOUND(i, n, site) true
static inline std::string check_take() { return std::string(); }
#endif

// Node coordinates inside an n^3 grid (every neighbour then follows by the
// periodic wrap).
__device__ __forceinline__ bool node_ok(int x, int y, int z, int n, int site) {
    return OTM_BOUND(x, n, site) && OTM_BOUND(y, n, site) && OTM_BOUND(z, n, site);
}

}  // namespace otm
