// 3x3x3 circular convolution of the warm-start network on the fifth-
// generation tensor cores (tcgen05): implicit GEMM with the accumulators in
// tensor memory.
//
//   out[v][co] = act(bias[co] + sum_t sum_ci W[t][ci][co] in[v + d_t][ci])
//
// A CTA of four warps owns one output tile of 8 (x) x 16 (y) voxels in one
// z-plane: M = 128 rows of the MMA, one row per voxel, and all cout output
// channels as N (16..192, a multiple of 16).  For each 16-channel chunk of the input it stages
// in shared memory, with 16-byte asynchronous copies,
//   * the tile's periodic halo, 10 x 18 x 3 voxels, as two planes of
//     [halo voxel][8 channels] (16 bytes per voxel and half-chunk), and
//   * the chunk's weights for the 27 taps, pre-packed as [t][half][co][8],
// both in the no-swizzle K-major canonical layout of 8-row x 16-byte core
// matrices.  The A operand of tap t is then the halo itself at the offset of
// d_t: its 8-row core matrices are 8 consecutive halo voxels in x (128
// contiguous bytes), the next 8 rows are the next y (stride 10 x 16 bytes),
// and the second 8 channels sit one halo plane further (leading offset) --
// so no im2col copy is formed.  One thread issues the chunk's 27 MMAs
// (M = 128, N = cout, K = 16, FP32 accumulation in tensor memory) and
// commits them to an mbarrier; the CTA waits (bounded) before reusing the
// buffers.  The epilogue reads the accumulators with tcgen05.ld (each warp
// its 32 lanes = 32 voxels), adds the bias, applies the ReLU, rounds to BF16
// and stores [voxel][cout].
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "check.cuh"
#include "ptx_async.cuh"

namespace otm {
namespace nn {

constexpr int kTcX = 8, kTcY = 16;                   // output tile in x, y (one z-plane)
constexpr int kTcHX = kTcX + 2, kTcHY = kTcY + 2;    // halo extents
constexpr int kTcHV = kTcHX * kTcHY * 3;             // 540 halo voxels
constexpr int kTcHaloBytes = 2 * kTcHV * 16;         // one 16-channel chunk: 17,280 B

inline bool conv3_tc_ok(int n, int cin, int cout) {
    return n >= 16 && n % kTcY == 0 && cin % 16 == 0 && cout % 16 == 0 && cout >= 16 && cout <= 192 && cin <= 512;
}
// weight bytes of one 16-channel chunk (27 taps, packed)
__host__ __device__ inline int conv3_tc_wbytes(int cout) { return 27 * 2 * cout * 16; }
inline size_t conv3_tc_smem(int cout) { return (size_t)kTcHaloBytes + conv3_tc_wbytes(cout) + 128; }
// tensor-memory columns: a power of two >= 32 holding cout FP32 columns
__host__ __device__ inline uint32_t conv3_tc_cols(int cout) {
    uint32_t c = 32;
    while (c < (uint32_t)cout) c <<= 1;
    return c;
}

// BF16 weights [27][cin][cout] -> the MMA's B layout, chunk-major:
// [cin / 16][t][half][co][8] with element (ci % 8) innermost.
static __global__ void k_pack_w_tc(int cin, int cout, const __nv_bfloat16* __restrict__ w,
                                   __nv_bfloat16* __restrict__ wtc) {
    const unsigned M = 27u * cin * cout;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < M; e += gridDim.x * blockDim.x) {
        const unsigned co = e % cout, r = e / cout;
        const unsigned ci = r % cin, t = r / cin;
        const unsigned chunk = ci >> 4, half = (ci >> 3) & 1, k = ci & 7;
        wtc[((((size_t)chunk * 27 + t) * 2 + half) * cout + co) * 8 + k] = w[e];
    }
}

template <bool RELU>
static __global__ void __launch_bounds__(128)
k_conv3_tc(int n, int cin, int cout, const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ wtc,
           const float* __restrict__ bias, __nv_bfloat16* __restrict__ out, int* err) {
    extern __shared__ unsigned char tc_smem_raw[];
    __shared__ __align__(8) uint64_t mma_done;
    __shared__ uint32_t tmem_slot;
    unsigned char* sm = tc_smem_raw + ((128u - (smem_u32(tc_smem_raw) & 127u)) & 127u);
    unsigned char* halo = sm;                         // [2][540][16 B]
    unsigned char* wts = sm + kTcHaloBytes;           // [27][2][cout][16 B]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntx = n / kTcX, nty = n / kTcY;
    const int b = blockIdx.x;
    const int x0 = (b % ntx) * kTcX, y0 = ((b / ntx) % nty) * kTcY, z = b / (ntx * nty);
    const uint32_t ncols = conv3_tc_cols(cout);

    if (warp == 0) tc_alloc(&tmem_slot, ncols);
    if (tid == 0) {
        mbar_init(&mma_done, 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = tc_idesc_bf16(128, cout);
    const uint32_t halo_s = smem_u32(halo), wts_s = smem_u32(wts);
    const int wbytes = conv3_tc_wbytes(cout);
    const int nchunk = cin / 16;
    bool ok = true;
    int pending = -1;   // chunk whose MMAs were issued but not seen complete

    for (int ck = 0; ck < nchunk; ++ck) {
        // stage the chunk's halo (two 8-channel halves per voxel) and weights
        for (int e = tid; e < 2 * kTcHV; e += 128) {
            const int half = e / kTcHV, h = e - half * kTcHV;
            const int hx = h % kTcHX, hy = (h / kTcHX) % kTcHY, hz = h / (kTcHX * kTcHY);
            int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z + hz - 1;
            gx += gx < 0 ? n : (gx >= n ? -n : 0);
            gy += gy < 0 ? n : (gy >= n ? -n : 0);
            gz += gz < 0 ? n : (gz >= n ? -n : 0);
            const size_t v = (size_t)gx + (size_t)n * ((size_t)gy + (size_t)n * gz);
            if (OTM_BOUND(v * cin + ck * 16 + half * 8 + 7, (long long)n * n * n * cin, kSiteConvTc))
                cp_async16(halo + (size_t)e * 16, in + v * cin + ck * 16 + half * 8);
        }
        const unsigned char* wsrc = reinterpret_cast<const unsigned char*>(wtc) + (size_t)ck * wbytes;
        for (int e = tid; e < wbytes / 16; e += 128) cp_async16(wts + (size_t)e * 16, wsrc + (size_t)e * 16);
        cp_async_wait_all();
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            for (int t = 0; t < 27; ++t) {
                const int dx = t % 3, dy = (t / 3) % 3, dz = t / 9;   // offsets + 1
                const uint32_t a_addr = halo_s + (uint32_t)((dx + kTcHX * (dy + kTcHY * dz)) * 16);
                const uint64_t adesc = tc_smem_desc(a_addr, kTcHV * 16, kTcHX * 16);
                const uint64_t bdesc = tc_smem_desc(wts_s + (uint32_t)(t * 2 * cout * 16), cout * 16, 128);
                // checking build: the last byte each operand reads (the second K half, the last
                // 8-row group, its last row) inside its buffer, and the accumulator's columns
                // inside the allocation
                if (OTM_BOUND((a_addr - halo_s) + kTcHV * 16 + 15 * kTcHX * 16 + 8 * 16 - 1, kTcHaloBytes,
                              kSiteConvTc) &&
                    OTM_BOUND(t * 2 * cout * 16 + cout * 16 + (cout / 8 - 1) * 128 + 127, wbytes, kSiteConvTc) &&
                    OTM_BOUND(cout - 1, (int)ncols, kSiteConvTc))
                    tc_mma_bf16(tmem, adesc, bdesc, idesc, (ck > 0 || t > 0) ? 1u : 0u);
            }
            tc_commit(&mma_done);
        }
        // the MMAs read the buffers: wait for them before the next chunk
        // overwrites them (and before the epilogue reads the accumulators)
        if (!mbar_wait_bounded(&mma_done, (uint32_t)(ck & 1))) ok = false;
        if (__syncthreads_or(!ok)) {
            ok = false;
            pending = ck;
            break;
        }
    }

    if (ok) {
        tc_fence_after();
        // epilogue: warp w holds tensor-memory lanes 32 w .. 32 w + 31, row r
        // = voxel (x0 + r % 8, y0 + r / 8, z)
        const int r = warp * 32 + lane;
        const size_t v = (size_t)(x0 + (r & 7)) + (size_t)n * ((size_t)(y0 + (r >> 3)) + (size_t)n * z);
        __nv_bfloat16* o = out + v * cout;
        for (int c0 = 0; c0 < cout; c0 += 16) {
            float acc[16];
            tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, acc);
            uint32_t pk[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float a0 = acc[2 * i] + (bias ? bias[c0 + 2 * i] : 0.f);
                float a1 = acc[2 * i + 1] + (bias ? bias[c0 + 2 * i + 1] : 0.f);
                if (RELU) {
                    a0 = fmaxf(a0, 0.f);
                    a1 = fmaxf(a1, 0.f);
                }
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(a0, a1);
                pk[i] = *reinterpret_cast<const uint32_t*>(&h2);
            }
            uint4* dst = reinterpret_cast<uint4*>(o + c0);
            dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
    } else {
        if (tid == 0 && err) *err = 1;
        // the MMAs still in flight must finish before their operands and
        // their tensor memory go away (again a bounded wait)
        if (pending >= 0) (void)mbar_wait_bounded(&mma_done, (uint32_t)(pending & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, ncols);
}


// ---------------------------------------------------------------------------
// Pipelined form for layers whose weights fit in shared memory: a CTA owns
// the 8 x 16 tile column at (x0, y0) over a range of z-planes and keeps the
// weights of all input chunks resident.  Halo planes (10 x 18 voxels, all
// channels, layout [chunk][half][180 voxels][16 B]) sit in a ring of five
// slots: output plane z reads halo planes z - 1, z, z + 1, and while its MMAs
// run, plane z + 2 is being copied in (cp.async).  A slot is refilled once
// the MMAs of every output plane that read it have completed (five slots: the
// refill of plane z + 2 replaces plane z - 3, last read by output plane
// z - 2, whose completion the epilogue of plane z - 2 has already waited
// for).  The accumulators are double-buffered in tensor memory, so the
// epilogue of plane z - 1 (tcgen05.ld, bias, ReLU, BF16 store) overlaps the
// MMAs of plane z.
constexpr int kTcRing = 5;
constexpr int kTcPlaneVox = kTcHX * kTcHY;   // 180
__host__ __device__ inline size_t conv3_tcz_smem(int cin, int cout) {
    const int nch = cin / 16;
    return (size_t)nch * conv3_tc_wbytes(cout) + (size_t)kTcRing * nch * 2 * kTcPlaneVox * 16 + 128;
}
inline bool conv3_tcz_ok(int n, int cin, int cout) {
    return conv3_tc_ok(n, cin, cout) && 2 * cout <= 256 && conv3_tcz_smem(cin, cout) <= 200 * 1024;
}

template <bool RELU>
static __global__ void __launch_bounds__(128)
k_conv3_tcz(int n, int cin, int cout, int m, const __nv_bfloat16* __restrict__ in,
            const __nv_bfloat16* __restrict__ wtc, const float* __restrict__ bias, __nv_bfloat16* __restrict__ out,
            int* err) {
    extern __shared__ unsigned char tcz_smem_raw[];
    __shared__ __align__(8) uint64_t mma_done[2];
    __shared__ uint32_t tmem_slot;
    unsigned char* sm = tcz_smem_raw + ((128u - (smem_u32(tcz_smem_raw) & 127u)) & 127u);
    const int nch = cin / 16;
    const int wbytes = conv3_tc_wbytes(cout);
    unsigned char* wts = sm;                                   // [nch][27][2][cout][16 B]
    unsigned char* ring = sm + (size_t)nch * wbytes;           // [R][nch][2][180][16 B]
    const int plane_bytes = nch * 2 * kTcPlaneVox * 16;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntx = n / kTcX, nty = n / kTcY;
    const int col = blockIdx.x % (ntx * nty), zc = blockIdx.x / (ntx * nty);
    const int x0 = (col % ntx) * kTcX, y0 = (col / ntx) * kTcY;
    const int z0 = zc * n / m, z1 = (zc + 1) * n / m, P = z1 - z0;
    const uint32_t ncols = conv3_tc_cols(2 * cout);

    if (warp == 0) tc_alloc(&tmem_slot, ncols);
    if (tid == 0) {
        mbar_init(&mma_done[0], 1);
        mbar_init(&mma_done[1], 1);
        fence_mbar_init();
    }
    // halo plane q (global plane z0 - 1 + q) into its ring slot
    auto load_plane = [&](int q) {
        int gz = z0 - 1 + q;
        gz += gz < 0 ? n : (gz >= n ? -n : 0);
        unsigned char* dst = ring + (size_t)(q % kTcRing) * plane_bytes;
        for (int e = tid; e < nch * 2 * kTcPlaneVox; e += 128) {
            const int ck = e / (2 * kTcPlaneVox), rem = e - ck * 2 * kTcPlaneVox;
            const int half = rem / kTcPlaneVox, h = rem - half * kTcPlaneVox;
            int gx = x0 + h % kTcHX - 1, gy = y0 + h / kTcHX - 1;
            gx += gx < 0 ? n : (gx >= n ? -n : 0);
            gy += gy < 0 ? n : (gy >= n ? -n : 0);
            const size_t v = (size_t)gx + (size_t)n * ((size_t)gy + (size_t)n * gz);
            if (OTM_BOUND(v * cin + ck * 16 + half * 8 + 7, (long long)n * n * n * cin, kSiteConvTc))
                cp_async16(dst + (size_t)e * 16, in + v * cin + ck * 16 + half * 8);
        }
    };
    // prologue: the weights and halo planes q = 0, 1, 2 (output plane 0)
    for (int e = tid; e < nch * wbytes / 16; e += 128)
        cp_async16(wts + (size_t)e * 16, reinterpret_cast<const unsigned char*>(wtc) + (size_t)e * 16);
    load_plane(0);
    load_plane(1);
    load_plane(2);
    asm volatile("cp.async.commit_group;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = tc_idesc_bf16(128, cout);
    const uint32_t ring_s = smem_u32(ring), wts_s = smem_u32(wts);
    const int r = warp * 32 + lane;   // this thread's accumulator row = voxel of the tile
    const size_t vrow = (size_t)(x0 + (r & 7)) + (size_t)n * (size_t)(y0 + (r >> 3));
    bool ok = true;
    int issued = 0;   // planes whose MMAs were issued

    auto epilogue = [&](int i) -> bool {
        // wait for plane i's MMAs (bounded), then read its accumulator buffer
        if (!mbar_wait_bounded(&mma_done[i & 1], (uint32_t)((i >> 1) & 1))) return false;
        tc_fence_after();
        __nv_bfloat16* o = out + (vrow + (size_t)n * n * (size_t)(z0 + i)) * cout;
        for (int c0 = 0; c0 < cout; c0 += 16) {
            float acc[16];
            tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((i & 1) * cout + c0), acc);
            uint32_t pk[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                float a0 = acc[2 * k] + (bias ? bias[c0 + 2 * k] : 0.f);
                float a1 = acc[2 * k + 1] + (bias ? bias[c0 + 2 * k + 1] : 0.f);
                if (RELU) {
                    a0 = fmaxf(a0, 0.f);
                    a1 = fmaxf(a1, 0.f);
                }
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(a0, a1);
                pk[k] = *reinterpret_cast<const uint32_t*>(&h2);
            }
            uint4* dst = reinterpret_cast<uint4*>(o + c0);
            dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
        tc_fence_before();
        return true;
    };

    for (int i = 0; i < P; ++i) {
        // a. prefetch halo plane q = i + 3 (needed by output plane i + 1);
        //    its slot last served output plane i - 2, complete since the
        //    epilogue of plane i - 2 (previous trip)
        if (i + 3 <= P + 1) load_plane(i + 3);
        asm volatile("cp.async.commit_group;" ::: "memory");
        // b. halo planes i .. i + 2 landed (all groups but the newest)
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        fence_proxy_async_smem();
        __syncthreads();
        // c. MMAs of output plane i into accumulator buffer i & 1
        if (tid == 0) {
            tc_fence_after();
            const uint32_t dcol = tmem + (uint32_t)((i & 1) * cout);
            for (int ck = 0; ck < nch; ++ck)
                for (int t = 0; t < 27; ++t) {
                    const int dx = t % 3, dy = (t / 3) % 3, dz = t / 9;   // offsets + 1
                    const uint32_t a_addr = ring_s + (uint32_t)(((i + dz) % kTcRing) * plane_bytes) +
                                            (uint32_t)((ck * 2 * kTcPlaneVox + dx + kTcHX * dy) * 16);
                    const uint64_t adesc = tc_smem_desc(a_addr, kTcPlaneVox * 16, kTcHX * 16);
                    const uint64_t bdesc =
                        tc_smem_desc(wts_s + (uint32_t)((ck * 27 + t) * 2 * cout * 16), cout * 16, 128);
                    tc_mma_bf16(dcol, adesc, bdesc, idesc, (ck > 0 || t > 0) ? 1u : 0u);
                }
            tc_commit(&mma_done[i & 1]);
        }
        issued = i + 1;
        // d. epilogue of plane i - 1 while plane i's MMAs run
        if (i >= 1) ok = epilogue(i - 1);
        if (__syncthreads_or(!ok)) {
            ok = false;
            break;
        }
    }
    if (ok && P >= 1) ok = epilogue(P - 1);
    if (!ok) {
        if (tid == 0 && err) *err = 1;
        // the MMAs still in flight finish before their operands and tensor
        // memory go away (bounded waits on the last two planes issued)
        for (int i = issued - 2 < 0 ? 0 : issued - 2; i < issued; ++i)
            (void)mbar_wait_bounded(&mma_done[i & 1], (uint32_t)((i >> 1) & 1));
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, ncols);
}

}  // namespace nn
}  // namespace otm
