// Internal device helpers of libotm: storage/compute types, periodic
// indexing, compensated FP32 accumulation and deterministic grid reductions.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include "otm.h"
#include "check.cuh"

namespace otm {

constexpr int kMaxLevelsDev = 12;   // multigrid levels a context may have

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  Every kernel first waits until the kernel
// it depends on has completed and its writes are visible (griddepcontrol.wait
// returns at once when the launch carried no programmatic dependency), then
// allows its own dependent to be launched, so that launch overlaps this
// kernel's execution instead of following its completion.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// One thread-block cluster of `ctas` CTAs (grid = cluster), with dynamic
// shared memory and programmatic dependent launch.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_cluster_pdl(void (*kern)(KArgs...), int ctas, dim3 block, size_t smem, cudaStream_t st,
                                      Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas, 1, 1);
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = ctas;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kern, ((KArgs)args)...);
}

// Launch with the programmatic-stream-serialisation attribute.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl_smem(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                   Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, ((KArgs)args)...);
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, ((KArgs)args)...);
}

// ---------------------------------------------------------------------------
// Storage type S -> compute type C.  Fields may be stored in FP64, FP32 or
// BF16; BF16 fields are computed on in FP32.
// ---------------------------------------------------------------------------
template <class S> struct St;
template <> struct St<double> {
    using C = double;
    static __device__ __forceinline__ double ld(const double* p, size_t i) { return p[i]; }
    static __device__ __forceinline__ void st(double* p, size_t i, double v) { p[i] = v; }
    static __device__ __forceinline__ double round(double v) { return v; }   // the value st stores
};
template <> struct St<float> {
    using C = float;
    static __device__ __forceinline__ float ld(const float* p, size_t i) { return p[i]; }
    static __device__ __forceinline__ void st(float* p, size_t i, float v) { p[i] = v; }
    static __device__ __forceinline__ float round(float v) { return v; }
};
template <> struct St<__nv_bfloat16> {
    using C = float;
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p, size_t i) {
        return __bfloat162float(p[i]);
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, size_t i, float v) {
        p[i] = __float2bfloat16_rn(v);
    }
    static __device__ __forceinline__ float round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
};

// ---- coarse-level layouts (levels >= 1, and the stencil of a single-level
// hierarchy): node-major, so one node's data is a few 16-byte vector loads.
//   stencil A: [N][kAW<S>] (the 27 couplings o = (dx+1) + 3(dy+1) + 9(dz+1),
//              padded to a 16-byte multiple),
//   fields T, F, residual, and the smoother's buffers: [N][4] (load cases
//              0..2, slot 3 zero).
template <class S>
struct CL {
    static constexpr int AW = sizeof(S) == 2 ? 32 : 28;
};
template <class S>
__host__ __device__ constexpr int cl_aw() { return CL<S>::AW; }

// the 27 couplings of node v
template <class S>
__device__ __forceinline__ void ld_arow(const S* __restrict__ A, size_t v, typename St<S>::C (&a)[27]);
template <>
__device__ __forceinline__ void ld_arow<float>(const float* __restrict__ A, size_t v, float (&a)[27]) {
    const float4* p = reinterpret_cast<const float4*>(A + v * 28);
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        const float4 w = p[q];
        if (4 * q + 0 < 27) a[4 * q + 0] = w.x;
        if (4 * q + 1 < 27) a[4 * q + 1] = w.y;
        if (4 * q + 2 < 27) a[4 * q + 2] = w.z;
        if (4 * q + 3 < 27) a[4 * q + 3] = w.w;
    }
}
template <>
__device__ __forceinline__ void ld_arow<double>(const double* __restrict__ A, size_t v, double (&a)[27]) {
    const double2* p = reinterpret_cast<const double2*>(A + v * 28);
#pragma unroll
    for (int q = 0; q < 14; ++q) {
        const double2 w = p[q];
        if (2 * q + 0 < 27) a[2 * q + 0] = w.x;
        if (2 * q + 1 < 27) a[2 * q + 1] = w.y;
    }
}
template <>
__device__ __forceinline__ void ld_arow<__nv_bfloat16>(const __nv_bfloat16* __restrict__ A, size_t v,
                                                       float (&a)[27]) {
    const uint4* p = reinterpret_cast<const uint4*>(A + v * 32);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint4 w = p[q];
        const unsigned u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const __nv_bfloat162 b2 = *reinterpret_cast<const __nv_bfloat162*>(&u[h]);
            const int e = 8 * q + 2 * h;
            if (e < 27) a[e] = __low2float(b2);
            if (e + 1 < 27) a[e + 1] = __high2float(b2);
        }
    }
}

// store the 27 couplings of node v (padding zeroed) as 16-byte vectors: an
// element-wise store of a row would make every store of a warp touch as many
// sectors as it has lanes; each element is rounded to S exactly as St<S>::st
// rounds it
template <class S, class C>
__device__ __forceinline__ void st_arow(S* __restrict__ A, size_t v, const C (&a)[27]);
template <>
__device__ __forceinline__ void st_arow<float, float>(float* __restrict__ A, size_t v, const float (&a)[27]) {
    float4* p = reinterpret_cast<float4*>(A + v * 28);
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        const int e = 4 * q;
        p[q] = make_float4(a[e], a[e + 1], a[e + 2], e + 3 < 27 ? a[e + 3] : 0.0f);
    }
}
template <>
__device__ __forceinline__ void st_arow<double, double>(double* __restrict__ A, size_t v, const double (&a)[27]) {
    double2* p = reinterpret_cast<double2*>(A + v * 28);
#pragma unroll
    for (int q = 0; q < 14; ++q) {
        const int e = 2 * q;
        p[q] = make_double2(e < 27 ? a[e] : 0.0, e + 1 < 27 ? a[e + 1] : 0.0);
    }
}
template <>
__device__ __forceinline__ void st_arow<__nv_bfloat16, float>(__nv_bfloat16* __restrict__ A, size_t v,
                                                              const float (&a)[27]) {
    uint4* p = reinterpret_cast<uint4*>(A + v * 32);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        unsigned u[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int e = 8 * q + 2 * h;
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(e < 27 ? a[e] : 0.0f, e + 1 < 27 ? a[e + 1] : 0.0f);
            u[h] = *reinterpret_cast<const unsigned*>(&b2);
        }
        p[q] = make_uint4(u[0], u[1], u[2], u[3]);
    }
}

// the three load cases at node v of a [N][4] field
template <class S>
__device__ __forceinline__ void ld_f3(const S* __restrict__ T, size_t v, typename St<S>::C (&t)[3]);
template <>
__device__ __forceinline__ void ld_f3<float>(const float* __restrict__ T, size_t v, float (&t)[3]) {
    const float4 w = *reinterpret_cast<const float4*>(T + 4 * v);
    t[0] = w.x;
    t[1] = w.y;
    t[2] = w.z;
}
template <>
__device__ __forceinline__ void ld_f3<double>(const double* __restrict__ T, size_t v, double (&t)[3]) {
    const double2* p = reinterpret_cast<const double2*>(T + 4 * v);
    const double2 a = p[0], b = p[1];
    t[0] = a.x;
    t[1] = a.y;
    t[2] = b.x;
}
template <>
__device__ __forceinline__ void ld_f3<__nv_bfloat16>(const __nv_bfloat16* __restrict__ T, size_t v, float (&t)[3]) {
    const uint2 w = *reinterpret_cast<const uint2*>(T + 4 * v);
    const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&w.x);
    const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&w.y);
    t[0] = __low2float(lo);
    t[1] = __high2float(lo);
    t[2] = __low2float(hi);
}
template <class S>
__device__ __forceinline__ void st_f3(S* __restrict__ T, size_t v, typename St<S>::C t0, typename St<S>::C t1,
                                      typename St<S>::C t2);
template <>
__device__ __forceinline__ void st_f3<float>(float* __restrict__ T, size_t v, float t0, float t1, float t2) {
    *reinterpret_cast<float4*>(T + 4 * v) = make_float4(t0, t1, t2, 0.0f);
}
template <>
__device__ __forceinline__ void st_f3<double>(double* __restrict__ T, size_t v, double t0, double t1, double t2) {
    double2* p = reinterpret_cast<double2*>(T + 4 * v);
    p[0] = make_double2(t0, t1);
    p[1] = make_double2(t2, 0.0);
}
template <>
__device__ __forceinline__ void st_f3<__nv_bfloat16>(__nv_bfloat16* __restrict__ T, size_t v, float t0, float t1,
                                                     float t2) {
    const __nv_bfloat162 lo = __floats2bfloat162_rn(t0, t1), hi = __floats2bfloat162_rn(t2, 0.0f);
    uint2 w;
    w.x = *reinterpret_cast<const unsigned*>(&lo);
    w.y = *reinterpret_cast<const unsigned*>(&hi);
    *reinterpret_cast<uint2*>(T + 4 * v) = w;
}
// A field read either node-major ([N][4], AOS) or load-case-major ([3][N]).
template <bool AOS, class S>
__device__ __forceinline__ void ld_f3_any(const S* __restrict__ T, size_t N, size_t v, typename St<S>::C (&t)[3]) {
    if (AOS) {
        ld_f3<S>(T, v, t);
    } else {
        t[0] = St<S>::ld(T, v);
        t[1] = St<S>::ld(T, N + v);
        t[2] = St<S>::ld(T, 2 * N + v);
    }
}

// Four consecutive values, loaded and stored with one vector access where
// the storage type allows it (16 B for FP32, 8 B for BF16, two 16 B for FP64).
template <class C>
struct Q4 {
    C v[4];
};
__device__ __forceinline__ Q4<float> ld4(const float* p, size_t i) {
    const float4 a = *reinterpret_cast<const float4*>(p + i);
    return Q4<float>{{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ void st4(float* p, size_t i, const Q4<float>& q) {
    *reinterpret_cast<float4*>(p + i) = make_float4(q.v[0], q.v[1], q.v[2], q.v[3]);
}
__device__ __forceinline__ Q4<double> ld4(const double* p, size_t i) {
    const double2 a = *reinterpret_cast<const double2*>(p + i);
    const double2 b = *reinterpret_cast<const double2*>(p + i + 2);
    return Q4<double>{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(double* p, size_t i, const Q4<double>& q) {
    *reinterpret_cast<double2*>(p + i) = make_double2(q.v[0], q.v[1]);
    *reinterpret_cast<double2*>(p + i + 2) = make_double2(q.v[2], q.v[3]);
}
__device__ __forceinline__ Q4<float> ld4(const __nv_bfloat16* p, size_t i) {
    const uint2 raw = *reinterpret_cast<const uint2*>(p + i);
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&raw.x);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&raw.y);
    return Q4<float>{{__low2float(a), __high2float(a), __low2float(b), __high2float(b)}};
}
__device__ __forceinline__ void st4(__nv_bfloat16* p, size_t i, const Q4<float>& q) {
    __nv_bfloat162 a = __floats2bfloat162_rn(q.v[0], q.v[1]);
    __nv_bfloat162 b = __floats2bfloat162_rn(q.v[2], q.v[3]);
    uint2 raw;
    raw.x = *reinterpret_cast<unsigned int*>(&a);
    raw.y = *reinterpret_cast<unsigned int*>(&b);
    *reinterpret_cast<uint2*>(p + i) = raw;
}

// Four consecutive values as floats, whatever the storage type.
__device__ __forceinline__ Q4<float> ld4f(const float* p, size_t i) { return ld4(p, i); }
__device__ __forceinline__ Q4<float> ld4f(const __nv_bfloat16* p, size_t i) { return ld4(p, i); }
__device__ __forceinline__ Q4<float> ld4f(const double* p, size_t i) {
    const Q4<double> d = ld4(p, i);
    return Q4<float>{{(float)d.v[0], (float)d.v[1], (float)d.v[2], (float)d.v[3]}};
}
__device__ __forceinline__ void st4f(float* p, size_t i, const Q4<float>& q) { st4(p, i, q); }
__device__ __forceinline__ void st4f(__nv_bfloat16* p, size_t i, const Q4<float>& q) { st4(p, i, q); }
__device__ __forceinline__ void st4f(double* p, size_t i, const Q4<float>& q) {
    st4(p, i, Q4<double>{{(double)q.v[0], (double)q.v[1], (double)q.v[2], (double)q.v[3]}});
}

// ---------------------------------------------------------------------------
// Accumulators for inner products and volume/tensor sums.  FP32 products are
// summed with an error-free transformation (TwoSum of the running sum and
// TwoProduct of each product, Ogita-Rump-Oishi "Accurate sum and dot
// product", 2005), so a thread's partial is good to about FP64 before it is
// converted for the FP64 block and grid stages.
// ---------------------------------------------------------------------------
template <class C> struct Acc;
template <> struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        float t = __fadd_rn(s, x);
        float bp = t - s;
        c += (s - (t - bp)) + (x - bp);
        s = t;
    }
    __device__ __forceinline__ void add_prod(float a, float b) {
        float p = __fmul_rn(a, b);
        float pe = fmaf(a, b, -p);
        float t = __fadd_rn(s, p);
        float bp = t - s;
        c += ((s - (t - bp)) + (p - bp)) + pe;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Error-free transformations (Knuth TwoSum, FMA TwoProduct).  The build
// lets the compiler fuse a multiply and a dependent add into one FMA, which
// would silently break both transformations (the rounded product p is then
// not the value the error term assumes).  Products that feed them are formed
// with mul_rn and the leading sum with add_rn, neither of which is fused.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
template <class C>
__device__ __forceinline__ void two_sum(C a, C b, C& s, C& e) {
    s = add_rn(a, b);
    const C bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// a - b on both lanes (one packed FP32 subtract; bitwise a + (-b))
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(d)
        : "l"(*reinterpret_cast<const unsigned long long*>(&a)), "l"(*reinterpret_cast<const unsigned long long*>(&b)));
    return *reinterpret_cast<const float2*>(&d);
}

// TwoSum on both lanes of a pair: each lane runs the scalar sequence, so the
// result is bitwise that of two two_sum calls.
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
    s = __fadd2_rn(a, b);
    const float2 bp = f2_sub(s, a);
    e = __fadd2_rn(f2_sub(a, f2_sub(s, bp)), f2_sub(b, bp));
}

// A value kept as an unevaluated sum hi + lo (double-float when C = float).
template <class C>
__device__ __forceinline__ C df_diff(C hw, C lw, C hv, C lv) {   // (hw + lw) - (hv + lv), rounded once
    C s, e;
    two_sum(hw, -hv, s, e);
    return s + ((lw - lv) + e);
}
// df_diff on both lanes.  two_sum(hw, -hv) is written with subtractions:
// hw + (-hv) = hw - hv and (-hv) - bp = -(hv + bp) exactly, so each lane is
// bitwise the scalar df_diff.
__device__ __forceinline__ float2 df_diff2(float2 hw, float2 lw, float2 hv, float2 lv) {
    const float2 s = f2_sub(hw, hv);
    const float2 bp = f2_sub(s, hw);
    const float2 e = f2_sub(f2_sub(hw, f2_sub(s, bp)), __fadd2_rn(hv, bp));
    return __fadd2_rn(s, __fadd2_rn(f2_sub(lw, lv), e));
}

// ---------------------------------------------------------------------------
// Deterministic grid reduction.  Every block reduces its threads' values in a
// fixed shuffle tree, writes one partial per value, and the last block to
// arrive (counted with an atomic ticket) sums the partials in a fixed order
// and runs the caller's finaliser.  Same grid -> bitwise-identical result.
// ---------------------------------------------------------------------------
struct RedBuf {
    double* partials;        // [max_blocks * kRedMaxVals]
    unsigned int* counter;   // one ticket counter, zero between launches
    int max_blocks;
};
constexpr int kRedMaxVals = 72;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-reduce NV values; thread 0 of the LAST block returns true with the
// grid-wide sums in `out` (shared memory, NV doubles, valid for all threads
// of that block after the call).  All threads of every block must call it.
template <int NV>
__device__ bool grid_reduce(const double (&v)[NV], const RedBuf& rb, double* out) {
    __shared__ double sm[32][NV];
    __shared__ bool is_last;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarp = (nthr + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double w = warp_sum(v[i]);
        if (lane == 0) sm[warp][i] = w;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double w = lane < nwarp ? sm[lane][i] : 0.0;
            w = warp_sum(w);
            if (lane == 0) rb.partials[(size_t)blockIdx.x * NV + i] = w;
        }
    }
    if (tid == 0) {
        __threadfence();
        unsigned int t = atomicAdd(rb.counter, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    // fixed-order sum of the partials: strided per thread, then a fixed tree
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double a = 0.0;
        for (int b = tid; b < (int)gridDim.x; b += nthr)
            a += __ldcg(rb.partials + (size_t)b * NV + i);
        a = warp_sum(a);
        __syncthreads();
        if (lane == 0) sm[warp][i] = a;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < nwarp; ++w) t += sm[w][i];
            out[i] = t;
        }
    }
    if (tid == 0) *rb.counter = 0u;
    __syncthreads();
    return true;
}

// The same reduction for FP32 accumulators, in double-float arithmetic:
// each value travels as its Acc<float> pair (s, c) with value s + c, and
// two pairs combine as TwoSum(s1, s2) = (t, e), c = (c1 + c2) + e, s = t --
// error-free in the leading part, so a sum keeps ~48 significant bits.  No
// FP64 instruction runs except in the last block's thread 0, which forms
// the doubles handed to the finaliser (FP64 units on this part run at a
// small fraction of the FP32 rate, so a per-warp double tree dominated the
// reduction kernels).  The pair combination is symmetric bit for bit (the
// TwoSum error term does not depend on the operand order), so butterfly
// lanes agree and the result is the same for the same grid.
__device__ __forceinline__ void ff_add(float& s, float& c, float s2, float c2) {
    const float t = __fadd_rn(s, s2);
    const float bp = t - s;
    const float e = (s - (t - bp)) + (s2 - bp);
    c = (c + c2) + e;
    s = t;
}
__device__ __forceinline__ void ff_warp_sum(float& s, float& c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
        const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
        ff_add(s, c, s2, c2);
    }
}
// Warp sums and merges of accumulators, in their own precision.
__device__ __forceinline__ void acc_warp_sum(Acc<float>& a) { ff_warp_sum(a.s, a.c); }
__device__ __forceinline__ void acc_warp_sum(Acc<double>& a) { a.s = warp_sum(a.s); }
__device__ __forceinline__ void acc_merge(Acc<float>& a, const Acc<float>& b) { ff_add(a.s, a.c, b.s, b.c); }
__device__ __forceinline__ void acc_merge(Acc<double>& a, const Acc<double>& b) { a.s += b.s; }
template <int NV>
__device__ bool grid_reduce(const Acc<float> (&v)[NV], const RedBuf& rb, double* out) {
    __shared__ float2 sm[32][NV];
    __shared__ bool is_last;
    float2* part = reinterpret_cast<float2*>(rb.partials);   // [blocks][NV] pairs
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarp = (nthr + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        float s = v[i].s, c = v[i].c;
        ff_warp_sum(s, c);
        if (lane == 0) sm[warp][i] = make_float2(s, c);
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            float2 w = lane < nwarp ? sm[lane][i] : make_float2(0.f, 0.f);
            ff_warp_sum(w.x, w.y);
            if (lane == 0) part[(size_t)blockIdx.x * NV + i] = w;
        }
    }
    if (tid == 0) {
        __threadfence();
        unsigned int t = atomicAdd(rb.counter, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    // fixed-order sum of the partials: strided per thread, then a fixed tree
#pragma unroll 1
    for (int i = 0; i < NV; ++i) {
        float s = 0.f, c = 0.f;
        for (int b = tid; b < (int)gridDim.x; b += nthr) {
            const float2 w = __ldcg(part + (size_t)b * NV + i);
            ff_add(s, c, w.x, w.y);
        }
        ff_warp_sum(s, c);
        __syncthreads();
        if (lane == 0) sm[warp][i] = make_float2(s, c);
        __syncthreads();
        if (warp == 0) {
            float2 w = lane < nwarp ? sm[lane][i] : make_float2(0.f, 0.f);
            ff_warp_sum(w.x, w.y);
            if (lane == 0) out[i] = (double)w.x + (double)w.y;
        }
    }
    if (tid == 0) *rb.counter = 0u;
    __syncthreads();
    return true;
}
// FP64 accumulators: the double tree above.
template <int NV>
__device__ bool grid_reduce(const Acc<double> (&v)[NV], const RedBuf& rb, double* out) {
    double vals[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) vals[i] = v[i].value();
    return grid_reduce<NV>(vals, rb, out);
}

// Row mapping of a grid kernel: threadIdx.x runs over x, the (y, z) rows
// (row = y + n z) over blockIdx.x * blockDim.y + threadIdx.y with a grid
// stride.  One 32-bit division per row, none per element.
#define OTM_FOR_ROWS(row, nrows)                                                          \
    for (int row = blockIdx.x * blockDim.y + threadIdx.y; row < (nrows); row += gridDim.x * blockDim.y)
#define OTM_FOR_X(xv, nx) for (int xv = threadIdx.x; xv < (nx); xv += blockDim.x)
// Launch shape for a row-mapped kernel: x threads (a multiple of 32, at most
// `threads`) times rows per block, and a grid over the rows capped at
// max_blocks (the capacity of the reduction partials).
struct RowLaunch {
    int grid;
    dim3 block;
};
inline RowLaunch row_launch(int nx, int nrows, int max_blocks, int threads = 256) {
    int bx = ((nx + 31) / 32) * 32;
    if (bx > threads) bx = threads;
    if (bx < 32) bx = 32;
    int by = threads / bx;
    if (by < 1) by = 1;
    long long g = ((long long)nrows + by - 1) / by;
    if (g > max_blocks) g = max_blocks;
    if (g < 1) g = 1;
    return RowLaunch{(int)g, dim3((unsigned)bx, (unsigned)by, 1)};
}
#define OTM_ROWS_CFG(cfg) (cfg).grid, (cfg).block

__device__ __forceinline__ bool is_thread0() {
    return threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0;
}

// ---------------------------------------------------------------------------
// Periodic grid indexing: node / element (x, y, z) at x + n (y + n z).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrapm(int a, int n) { return a == 0 ? n - 1 : a - 1; }
__device__ __forceinline__ int wrapp(int a, int n) { return a == n - 1 ? 0 : a + 1; }
__device__ __forceinline__ int wrapd(int a, int d, int n) {
    a += d;
    return a < 0 ? a + n : (a >= n ? a - n : a);
}

// ---------------------------------------------------------------------------
// Scalars shared between kernels of a solve (device resident).
// ---------------------------------------------------------------------------
struct PcgScalars {
    double ff[3];        // ||f_i||^2
    double rr[3];        // ||r_i||^2 (recurrence)
    double gamma[3];     // r_i . z_i
    double pq[3];        // p_i . K p_i
    double alpha[3];
    double beta[3];
    double rz_old[3];    // r_{k+1} . z_k (flexible beta)
    double true_rr[3];   // ||f - K x||^2 at the last residual replacement
    double true_ff[3];
    double fmean[3];     // mean of each macro load before projection
    double tol2;         // cg_tol^2
    int active[3];       // 1 while load case i iterates
    int iters[3];
    int nactive;
    int first;           // set by the residual of a pass: the next beta is the first of the pass
    int pfirst;          // the p update after that beta sets p = z
    int total;           // PCG iterations of this solve (all passes)
    int breakdown;       // bit i set: load case i broke down (pq <= 0 or non-finite)
    int flexible;        // 1: Polak-Ribiere beta
    int dev_err;         // set by a kernel whose bounded wait ran out
};

struct GovState {
    double df, vstar, g_prev, gap;
    int count, pad;
};

struct GovParams {
    double bound, small_rel, vol_tol;
};

// Alg. 1, one pass of its loop body, with the thresholds of GovParams.
__host__ __device__ inline void governor_update(GovState& s, const GovParams& p, double g,
                                                double low_bound, double vol) {
    if (g <= p.bound) {
        s.gap = s.vstar - low_bound;
        s.vstar = s.vstar - s.gap * s.df;
        s.df = 0.8 * s.df;
    }
    const double dg = s.g_prev - g;
    const bool cond1 = (dg < 0 ? -dg : dg) < p.small_rel * g;
    const bool cond2 = g > p.bound;
    const double dv = vol - s.vstar;
    const bool cond3 = (dv < 0 ? -dv : dv) < p.vol_tol;
    if (cond1 && cond2 && cond3)
        s.count += 1;
    else
        s.count = 0;
    if (s.count >= 5) {
        s.vstar = s.vstar + 0.3 * s.gap * s.df;
        s.count = 0;
    }
    if (s.vstar > 1.0) s.vstar = 1.0;
    if (s.vstar < 0.0) s.vstar = 0.0;
    s.g_prev = g;
}

constexpr int kOcCand = 64;   // candidates per OC search pass

struct DesignScalars {
    double sum_rho;          // sum of rho
    double sum_rhop;         // sum of rho_f^p
    double kappa[6];
    double g;
    double w[6];             // dg / dkappa_c
    double target[6];
    double vstar;
    GovState gov;
    GovParams govp;
    int governor_on;
    int objective;
    // OC search
    double oc_vmin, oc_vmax;       // sums: all-lower and all-upper (growing) volume
    double mu_lo, mu_hi;           // current bracket of mu = lambda^-eta
    double v_lo, v_hi;             // volume sums at the bracket ends
    double mu_star;
    double lambda;
    int oc_mode;                   // 0 interior, 1 inactive, 2 infeasible
    int oc_pass;
    double mu_min_seen, mu_max_seen;
    // MMA (model 2) dual search
    double mma_r1;                 // r1 of the constraint's approximation
    double mma_lo, mma_hi;         // bracket of lambda
    double mma_phi_lo, mma_phi_hi; // phi at the bracket ends
    double mma_lam;                // lambda*
    int mma_mode;                  // 0 search, 1 constraint inactive (lambda = 0)
    int mma_pass;
    int mma_k;                     // MMA iterations done (asymptote rule)
    int mma_pad;
};

}  // namespace otm
