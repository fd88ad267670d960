// Kernels of the periodic 3-D convolutional U-Net used as the learned warm
// start of the homogenization solve (a predictor of the three corrector
// fields from the filtered density).  Activations are BF16, stored voxel-major
// with channels innermost ([voxel][C], C a multiple of 16); weights of a
// 3x3x3 convolution are [27][Cin][Cout] (tap t = (dz+1)*9 + (dy+1)*3 + dx+1,
// Cout innermost); accumulation is FP32.
//
// The 3x3x3 circular convolution is an implicit GEMM (M = voxels,
// N = output channels, K = 27 taps x input channels) on the BF16 tensor
// cores with mma.sync m16n8k16 and ldmatrix fragment loads.  Its gradient
// with respect to the input is the same convolution with flipped taps and
// transposed weights; the weight gradient is a GEMM that reduces over voxels.
#pragma once
#include "otm_internal.cuh"

namespace otm {
namespace nn {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
// c += a (16x16, row) * b (16x8, col), BF16 inputs, FP32 accumulators
__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ int tap_dz(int t) { return t / 9 - 1; }
__device__ __forceinline__ int tap_dy(int t) { return (t / 3) % 3 - 1; }
__device__ __forceinline__ int tap_dx(int t) { return t % 3 - 1; }

constexpr int kCM = 64;   // voxels per CTA of the convolution

// out[v][co] = act(b[co] + sum_t sum_ci W[t][ci][co] in[v + d_t][ci]).
// Grid (N / 64, Cout / BN), 128 threads; warp w computes voxels 16w..16w+15.
// bias may be null; RELU applies max(0, .).  Rows past the last voxel (the
// ragged last tile) load voxel N-1 and are not stored.
template <int BN, bool RELU>
__global__ void __launch_bounds__(128)
k_conv3(int n, int Cin, int Cout, const bf16* __restrict__ in, const bf16* __restrict__ W,
        const float* __restrict__ bias, bf16* __restrict__ out) {
    pdl_enter();
    const size_t N = (size_t)n * n * n;
    __shared__ __align__(16) bf16 As[kCM][24];
    __shared__ __align__(16) bf16 Bs[16][BN + 8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t m0 = (size_t)blockIdx.x * kCM;
    const int n0 = blockIdx.y * BN;
    const int am = tid >> 1, ah = tid & 1;                 // A: voxel am, channels ah*8..ah*8+7
    const size_t v = m0 + am < N ? m0 + am : N - 1;
    const int vx = (int)(v % n), vy = (int)((v / n) % n), vz = (int)(v / ((size_t)n * n));
    constexpr int BCH = BN / 8;                            // 16-byte chunks per B row
    const bool bload = tid < 16 * BCH;
    const int bk = tid / BCH, bc = (tid % BCH) * 8;
    float acc[BN / 8][4];
#pragma unroll
    for (int j = 0; j < BN / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    const int kch = Cin / 16;
    for (int t = 0; t < 27; ++t) {
        const size_t nb = (size_t)wrapd(vx, tap_dx(t), n) +
                          (size_t)n * ((size_t)wrapd(vy, tap_dy(t), n) + (size_t)n * wrapd(vz, tap_dz(t), n));
        for (int c = 0; c < kch; ++c) {
            const uint4 a = *reinterpret_cast<const uint4*>(in + nb * Cin + c * 16 + ah * 8);
            uint4 b = make_uint4(0, 0, 0, 0);
            if (bload) b = *reinterpret_cast<const uint4*>(W + ((size_t)t * Cin + c * 16 + bk) * Cout + n0 + bc);
            __syncthreads();
            *reinterpret_cast<uint4*>(&As[am][ah * 8]) = a;
            if (bload) *reinterpret_cast<uint4*>(&Bs[bk][bc]) = b;
            __syncthreads();
            unsigned af[4];
            ldsm_x4(af, &As[warp * 16 + (lane & 15)][(lane >> 4) * 8]);
#pragma unroll
            for (int j = 0; j < BN / 8; j += 2) {
                unsigned bf[4];
                ldsm_x4_t(bf, &Bs[lane & 15][j * 8 + (lane >> 4) * 8]);
                mma_bf16(acc[j], af, bf[0], bf[1]);
                mma_bf16(acc[j + 1], af, bf[2], bf[3]);
            }
        }
    }
    const int row = warp * 16 + (lane >> 2);
#pragma unroll
    for (int j = 0; j < BN / 8; ++j) {
        const int co = n0 + j * 8 + (lane & 3) * 2;
        const float b0 = bias ? bias[co] : 0.f, b1 = bias ? bias[co + 1] : 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float y0 = acc[j][2 * h] + b0, y1 = acc[j][2 * h + 1] + b1;
            if (RELU) {
                y0 = fmaxf(y0, 0.f);
                y1 = fmaxf(y1, 0.f);
            }
            const size_t m = m0 + row + 8 * h;
            if (m < N) *reinterpret_cast<__nv_bfloat162*>(out + m * Cout + co) = __floats2bfloat162_rn(y0, y1);
        }
    }
}

// dW[t][ci][co] += sum_v in[v + d_t][ci] * g[v][co] over a chunk of voxels
// (input stored with Cin channels, of which the first Ca are real: dW is
// [27][Ca][Cout]),
// and (blockIdx.z == 0 only) db[co] += sum_v g[v][co].  Grid
// (chunks, Cin / 16, 27 * (Cout / BN)), 128 threads; each warp reduces 16
// voxels per step, warps are combined in shared memory, and the CTA adds its
// partial to dW with FP32 atomics.
template <int BN>
__global__ void __launch_bounds__(128)
k_conv3_dw(int n, int Cin, int Ca, int Cout, int chunk, const bf16* __restrict__ in, const bf16* __restrict__ g,
           float* __restrict__ dW, float* __restrict__ db) {
    pdl_enter();
    __shared__ __align__(16) bf16 As[64][24];       // [voxel][ci]
    __shared__ __align__(16) bf16 Bs[64][BN + 8];   // [voxel][co]
    __shared__ float red[4][16][BN];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t N = (size_t)n * n * n;
    const int ci0 = blockIdx.y * 16;
    const int nbt = Cout / BN;
    const int t = blockIdx.z / nbt, n0 = (blockIdx.z % nbt) * BN;
    const size_t v0 = (size_t)blockIdx.x * chunk;
    size_t v1 = v0 + chunk;
    if (v1 > N) v1 = N;
    float acc[BN / 8][4];
#pragma unroll
    for (int j = 0; j < BN / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    float bsum = 0.f;
    constexpr int BCH = BN / 8;
    for (size_t vb = v0; vb < v1; vb += 64) {
        // A: 64 voxels x 16 channels of the shifted input (2 chunks of 8 per voxel)
        {
            const int am = tid >> 1, ah = tid & 1;
            const size_t v = vb + am;
            uint4 a = make_uint4(0, 0, 0, 0);
            if (v < v1) {
                const int vx = (int)(v % n), vy = (int)((v / n) % n), vz = (int)(v / ((size_t)n * n));
                const size_t nb = (size_t)wrapd(vx, tap_dx(t), n) +
                                  (size_t)n * ((size_t)wrapd(vy, tap_dy(t), n) + (size_t)n * wrapd(vz, tap_dz(t), n));
                a = *reinterpret_cast<const uint4*>(in + nb * Cin + ci0 + ah * 8);
            }
            *reinterpret_cast<uint4*>(&As[am][ah * 8]) = a;
        }
        // B: 64 voxels x BN channels of the output gradient
        for (int e = tid; e < 64 * BCH; e += 128) {
            const int bv = e / BCH, bc = (e % BCH) * 8;
            const size_t v = vb + bv;
            uint4 b = make_uint4(0, 0, 0, 0);
            if (v < v1) b = *reinterpret_cast<const uint4*>(g + v * Cout + n0 + bc);
            *reinterpret_cast<uint4*>(&Bs[bv][bc]) = b;
        }
        __syncthreads();
        // warp w reduces voxels 16w..16w+15: A^T fragment via transposed loads
        unsigned af[4];
        ldsm_x4_t(af, &As[warp * 16 + (lane & 7) + ((lane >> 4) << 3)][((lane >> 3) & 1) * 8]);
#pragma unroll
        for (int j = 0; j < BN / 8; j += 2) {
            unsigned bf[4];
            ldsm_x4_t(bf, &Bs[warp * 16 + (lane & 15)][j * 8 + (lane >> 4) * 8]);
            mma_bf16(acc[j], af, bf[0], bf[1]);
            mma_bf16(acc[j + 1], af, bf[2], bf[3]);
        }
        if (db && blockIdx.y == 0 && t == 0 && tid < BN) {
            for (int r = 0; r < 64 && vb + r < v1; ++r) bsum += __bfloat162float(Bs[r][tid]);
        }
        __syncthreads();
    }
    // combine the four warps
#pragma unroll
    for (int j = 0; j < BN / 8; ++j) {
        const int r0 = lane >> 2, c0 = j * 8 + (lane & 3) * 2;
        red[warp][r0][c0] = acc[j][0];
        red[warp][r0][c0 + 1] = acc[j][1];
        red[warp][r0 + 8][c0] = acc[j][2];
        red[warp][r0 + 8][c0 + 1] = acc[j][3];
    }
    __syncthreads();
    for (int e = tid; e < 16 * BN; e += 128) {
        const int r = e / BN, c = e % BN;
        const float s = red[0][r][c] + red[1][r][c] + red[2][r][c] + red[3][r][c];
        if (ci0 + r < Ca) atomicAdd(dW + ((size_t)t * Ca + ci0 + r) * Cout + n0 + c, s);
    }
    if (db && blockIdx.y == 0 && t == 0 && tid < BN) atomicAdd(db + n0 + tid, bsum);
}

// The channel-wise kernels below move 8 channels (16 bytes) per thread and
// step (channel counts are multiples of 16), with 32-bit indices (fewer than
// 2^31 voxel-channels).  Per channel the arithmetic and its order are those
// of a one-element-per-thread loop.
__device__ __forceinline__ void bf8_load(const bf16* p, float (&f)[8]) {
    const uint4 u = *reinterpret_cast<const uint4*>(p);
    const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&w[i]);
        f[2 * i] = __low2float(h);
        f[2 * i + 1] = __high2float(h);
    }
}
__device__ __forceinline__ void bf8_store(bf16* p, const float (&f)[8]) {
    unsigned w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 h = __halves2bfloat162(__float2bfloat16_rn(f[2 * i]), __float2bfloat16_rn(f[2 * i + 1]));
        w[i] = *reinterpret_cast<const unsigned*>(&h);
    }
    *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}
__device__ __forceinline__ void copy8(bf16* d, const bf16* s) {
    *reinterpret_cast<uint4*>(d) = *reinterpret_cast<const uint4*>(s);
}

// g = g * (y > 0): ReLU backward, y the block output (count a multiple of 8).
// BF16 -> FP32 copy (exports of stored activations)
static __global__ void k_bf16_to_f32(size_t count, const bf16* __restrict__ in, float* __restrict__ out) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        out[i] = __bfloat162float(in[i]);
}

static __global__ void k_relu_mask(size_t count, bf16* __restrict__ g, const bf16* __restrict__ y) {
    const unsigned n8 = (unsigned)(count / 8);
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < n8; e += gridDim.x * blockDim.x) {
        float gv[8], yv[8];
        bf8_load(g + 8 * (size_t)e, gv);
        bf8_load(y + 8 * (size_t)e, yv);
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (!(yv[i] > 0.f)) gv[i] = 0.f;
        bf8_store(g + 8 * (size_t)e, gv);
    }
}

// 2x2x2 average pooling, [8 Nc][C] -> [Nc][C] (coarse grid nc per side).
static __global__ void k_pool(int nc, int C, const bf16* __restrict__ in, bf16* __restrict__ out) {
    const unsigned Nc = (unsigned)nc * nc * nc;
    const int nf = 2 * nc, C8 = C / 8;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < Nc * C8; e += gridDim.x * blockDim.x) {
        const unsigned V = e / C8;
        const int c = (int)(e - V * C8) * 8;
        const int X = (int)(V % nc), Y = (int)((V / nc) % nc), Z = (int)(V / ((unsigned)nc * nc));
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int q = 0; q < 8; ++q) {
            const unsigned f = (unsigned)(2 * X + (q & 1)) + (unsigned)nf * ((2 * Y + ((q >> 1) & 1)) + (unsigned)nf * (2 * Z + (q >> 2)));
            float w[8];
            bf8_load(in + (size_t)f * C + c, w);
#pragma unroll
            for (int i = 0; i < 8; ++i) s[i] += w[i];
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) s[i] *= 0.125f;
        bf8_store(out + (size_t)V * C + c, s);
    }
}

// din[v][c] += dout[v / 2][c] / 8 (adjoint of the pooling), fine grid nf.
static __global__ void k_pool_back_add(int nf, int C, const bf16* __restrict__ dout, bf16* __restrict__ din) {
    const unsigned Nf = (unsigned)nf * nf * nf;
    const int nc = nf / 2, C8 = C / 8;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < Nf * C8; e += gridDim.x * blockDim.x) {
        const unsigned v = e / C8;
        const int c = (int)(e - v * C8) * 8;
        const int x = (int)(v % nf), y = (int)((v / nf) % nf), z = (int)(v / ((unsigned)nf * nf));
        const unsigned V = (unsigned)(x >> 1) + (unsigned)nc * ((y >> 1) + (unsigned)nc * (z >> 1));
        float a[8], d[8];
        bf8_load(din + (size_t)v * C + c, a);
        bf8_load(dout + (size_t)V * C + c, d);
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = a[i] + 0.125f * d[i];
        bf8_store(din + (size_t)v * C + c, a);
    }
}

// cat[v][0..Cu) = up(coarse)[v], cat[v][Cu..Cu+Cs) = skip[v]  (fine grid nf)
static __global__ void k_up_cat(int nf, int Cu, int Cs, const bf16* __restrict__ coarse, const bf16* __restrict__ skip,
                                bf16* __restrict__ cat) {
    const unsigned Nf = (unsigned)nf * nf * nf;
    const int nc = nf / 2;
    const int Ct = Cu + Cs, T8 = Ct / 8, U8 = Cu / 8;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < Nf * T8; e += gridDim.x * blockDim.x) {
        const unsigned v = e / T8;
        const int j = (int)(e - v * T8);
        if (j < U8) {
            const int x = (int)(v % nf), y = (int)((v / nf) % nf), z = (int)(v / ((unsigned)nf * nf));
            const unsigned V = (unsigned)(x >> 1) + (unsigned)nc * ((y >> 1) + (unsigned)nc * (z >> 1));
            copy8(cat + (size_t)v * Ct + 8 * j, coarse + (size_t)V * Cu + 8 * j);
        } else {
            copy8(cat + (size_t)v * Ct + 8 * j, skip + (size_t)v * Cs + 8 * (j - U8));
        }
    }
}

// Split the gradient of a concatenation: dcoarse[V][c] = sum over the 8
// children of dcat[v][c] (c < Cu) (the adjoint of the upsampling), and
// dskip[v][c] = dcat[v][Cu + c].
static __global__ void k_up_cat_back(int nf, int Cu, int Cs, const bf16* __restrict__ dcat, bf16* __restrict__ dcoarse,
                                     bf16* __restrict__ dskip) {
    const int nc = nf / 2;
    const unsigned Nc = (unsigned)nc * nc * nc, Nf = (unsigned)nf * nf * nf;
    const int Ct = Cu + Cs, U8 = Cu / 8, S8 = Cs / 8;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < Nc * U8; e += gridDim.x * blockDim.x) {
        const unsigned V = e / U8;
        const int c = (int)(e - V * U8) * 8;
        const int X = (int)(V % nc), Y = (int)((V / nc) % nc), Z = (int)(V / ((unsigned)nc * nc));
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int q = 0; q < 8; ++q) {
            const unsigned f = (unsigned)(2 * X + (q & 1)) + (unsigned)nf * ((2 * Y + ((q >> 1) & 1)) + (unsigned)nf * (2 * Z + (q >> 2)));
            float w[8];
            bf8_load(dcat + (size_t)f * Ct + c, w);
#pragma unroll
            for (int i = 0; i < 8; ++i) s[i] += w[i];
        }
        bf8_store(dcoarse + (size_t)V * Cu + c, s);
    }
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < Nf * S8; e += gridDim.x * blockDim.x) {
        const unsigned v = e / S8;
        const int j = (int)(e - v * S8);
        copy8(dskip + (size_t)v * Cs + 8 * j, dcat + (size_t)v * Ct + Cu + 8 * j);
    }
}

// The network's first convolution, whose input is the single density
// channel: y[v][co] = relu(b[co] + sum_t W[t][0][co] bf16(rho[v + off(t)]))
// with the packed weights [27][16][cout] (only input channel 0 is real), in
// FP32 on the CUDA cores -- the tensor-core path would multiply 15 zero
// channels.  cout <= 64, a multiple of 8.
template <class T>
__global__ void __launch_bounds__(256)
k_conv3_in1(int n, const T* __restrict__ rho, const bf16* __restrict__ W, int ap, int cout,
            const float* __restrict__ bias, bf16* __restrict__ y) {
    __shared__ float w[27][64];
    __shared__ float bs[64];
    for (int i = threadIdx.x; i < 27 * cout; i += blockDim.x) {
        const int t = i / cout, co = i - t * cout;
        w[t][co] = __bfloat162float(W[((size_t)t * ap) * cout + co]);
    }
    for (int i = threadIdx.x; i < cout; i += blockDim.x) bs[i] = bias ? bias[i] : 0.f;
    __syncthreads();
    const unsigned N = (unsigned)n * n * n;
    for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
        const int x = (int)(v % n), yy = (int)((v / n) % n), z = (int)(v / ((unsigned)n * n));
        float r[27];
#pragma unroll
        for (int t = 0; t < 27; ++t) {
            const unsigned o = (unsigned)wrapd(x, tap_dx(t), n) +
                               (unsigned)n * ((unsigned)wrapd(yy, tap_dy(t), n) + (unsigned)n * wrapd(z, tap_dz(t), n));
            r[t] = __bfloat162float(__float2bfloat16_rn((float)rho[o]));
        }
        for (int c0 = 0; c0 < cout; c0 += 8) {
            float a[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = 0.f;
#pragma unroll
            for (int t = 0; t < 27; ++t)
#pragma unroll
                for (int i = 0; i < 8; ++i) a[i] += w[t][c0 + i] * r[t];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = fmaxf(a[i] + bs[c0 + i], 0.f);
            bf8_store(y + (size_t)v * cout + c0, a);
        }
    }
}

// Input layer: x[v][0] = rho[v], channels 1..15 zero (Cin padded to 16).
template <class T>
__global__ void k_input16(size_t N, const T* __restrict__ rho, bf16* __restrict__ x) {
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
        uint4 z = make_uint4(0, 0, 0, 0);
        __nv_bfloat162 a = __floats2bfloat162_rn((float)rho[v], 0.f);
        z.x = *reinterpret_cast<unsigned*>(&a);
        reinterpret_cast<uint4*>(x + v * 16)[0] = z;
        reinterpret_cast<uint4*>(x + v * 16)[1] = make_uint4(0, 0, 0, 0);
    }
}

// Head: y[j][v] = b[j] + sum_c d[v][c] H[c][j], j < 3 (FP32 out, [3][N]).
static __global__ void k_head(size_t N, int C, const bf16* __restrict__ d, const float* __restrict__ H,
                       const float* __restrict__ b, float* __restrict__ y) {
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
        float a0 = b[0], a1 = b[1], a2 = b[2];
        for (int c0 = 0; c0 < C; c0 += 8) {
            float dv[8];
            bf8_load(d + v * C + c0, dv);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int c = c0 + i;
                a0 += dv[i] * H[c * 3 + 0];
                a1 += dv[i] * H[c * 3 + 1];
                a2 += dv[i] * H[c * 3 + 2];
            }
        }
        y[v] = a0;
        y[N + v] = a1;
        y[2 * N + v] = a2;
    }
}

// Head backward: dd[v][c] = sum_j dy[j][v] H[c][j] (written), and the
// sums dH[c][j] += sum_v d[v][c] dy[j][v], db[j] += sum_v dy[j][v]
// (per-thread partials over 16-channel slices, warp and block sums in shared
// memory, then FP32 atomics).  C <= 256, a multiple of 16.
static __global__ void __launch_bounds__(256)
k_head_back(size_t N, int C, const bf16* __restrict__ d, const float* __restrict__ H,
            const float* __restrict__ dy, bf16* __restrict__ dd, float* __restrict__ dH,
            float* __restrict__ db) {
    __shared__ float sH[256 * 3 + 3];
    for (int i = threadIdx.x; i < C * 3 + 3; i += blockDim.x) sH[i] = 0.f;
    __syncthreads();
    for (int cb = 0; cb < C; cb += 16) {
        float lH[48];
        float lb[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 48; ++i) lH[i] = 0.f;
        for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
            const float g0 = dy[v], g1 = dy[N + v], g2 = dy[2 * N + v];
            lb[0] += g0;
            lb[1] += g1;
            lb[2] += g2;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const float dv = __bfloat162float(d[v * C + cb + c]);
                lH[c * 3 + 0] += dv * g0;
                lH[c * 3 + 1] += dv * g1;
                lH[c * 3 + 2] += dv * g2;
                const float* h = H + (cb + c) * 3;
                dd[v * C + cb + c] = __float2bfloat16_rn(g0 * h[0] + g1 * h[1] + g2 * h[2]);
            }
        }
#pragma unroll
        for (int i = 0; i < 48; ++i) {
            float w = lH[i];
            for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
            if ((threadIdx.x & 31) == 0) atomicAdd(&sH[cb * 3 + i], w);
        }
        if (cb == 0) {
            for (int j = 0; j < 3; ++j) {
                float w = lb[j];
                for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
                if ((threadIdx.x & 31) == 0) atomicAdd(&sH[C * 3 + j], w);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < C * 3; i += blockDim.x) atomicAdd(dH + i, sH[i]);
    if (threadIdx.x < 3) atomicAdd(db + threadIdx.x, sH[C * 3 + threadIdx.x]);
}

// MSE loss against the target t * inv_scale (t [3][N]): dy = 2 (y - t') / M;
// loss partials (compensated FP32 per thread and warp) added into *loss
// with one FP64 atomic per warp.
static __global__ void k_mse(size_t M, const float* __restrict__ y, const float* __restrict__ t, float inv_scale,
                             float* __restrict__ dy, double* __restrict__ loss) {
    Acc<float> s;
    const float sc = 2.0f / (float)M;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i] * inv_scale;
        s.add_prod(d, d);
        dy[i] = sc * d;
    }
    acc_warp_sum(s);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, s.value() / (double)M);
}

// Adam update of the FP32 master parameters.
static __global__ void k_adam(size_t P, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

// Copy a [27][a][b] FP32 weight block into the BF16 compute layout
// [27][ap][b] (ap >= a, padded channels zero), optionally also the flipped,
// transposed form [27][b][ap] used by the input-gradient convolution
// (tap t -> 26 - t).
static __global__ void k_pack_w(int a, int ap, int b, const float* __restrict__ w, bf16* __restrict__ wc,
                         bf16* __restrict__ wt) {
    const unsigned M = 27u * ap * b, apb = (unsigned)ap * b;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < M; e += gridDim.x * blockDim.x) {
        const int t = (int)(e / apb);
        const unsigned r = e - t * apb;
        const int ci = (int)(r / b), co = (int)(r - ci * b);
        const float val = ci < a ? w[((unsigned)t * a + ci) * b + co] : 0.f;
        const bf16 bv = __float2bfloat16_rn(val);
        wc[e] = bv;
        if (wt) wt[((unsigned)(26 - t) * b + co) * ap + ci] = bv;
    }
}

}  // namespace nn
}  // namespace otm

namespace otm {
namespace nn {

// Brick-tiled 3x3x3 circular convolution (same contract as k_conv3).  A CTA
// of 8 warps computes an 8 x 8 x 4 brick of output voxels (M = 256) for BN
// output channels.  Per 16-channel input chunk it stages the brick's input
// halo (10 x 10 x 6 voxels, each row padded by 8 BF16 so that ldmatrix rows
// fall on distinct banks) and the chunk's weights for all 27 taps in shared
// memory, then every warp runs the 27 taps -- one ldmatrix of B per tap, one
// ldmatrix of A and BN / 8 MMAs per 16-voxel row block -- without a barrier
// inside the tap loop.  Requires n % 8 == 0 and 4 | n.
constexpr int kBX = 8, kBY = 8, kBZ = 4;
constexpr int kHX = kBX + 2, kHY = kBY + 2, kHZ = kBZ + 2;
constexpr int kHalo = kHX * kHY * kHZ;          // 600 voxels
constexpr int kHRow = 16 + 8;                   // one chunk's channels, padded

inline size_t conv3_tile_smem(int bn) { return (size_t)kHalo * kHRow * 2 + (size_t)27 * 16 * (bn + 8) * 2; }
inline bool conv3_tile_ok(int n) { return n >= kBX && n % kBX == 0 && n % kBZ == 0; }

template <int BN, bool RELU>
__global__ void __launch_bounds__(256)
k_conv3_tile(int n, int Cin, int Cout, const bf16* __restrict__ in, const bf16* __restrict__ W,
             const float* __restrict__ bias, bf16* __restrict__ out) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char conv_sm[];
    bf16* halo = reinterpret_cast<bf16*>(conv_sm);                      // [kHalo][kHRow]
    bf16* ws = halo + kHalo * kHRow;                                      // [27][16][BN + 8]
    constexpr int WROW = BN + 8;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nbx = n / kBX, nby = n / kBY;
    const int bx = blockIdx.x % nbx, by = (blockIdx.x / nbx) % nby, bz = blockIdx.x / (nbx * nby);
    const int x0 = bx * kBX, y0 = by * kBY, z0 = bz * kBZ;
    const int co0 = blockIdx.y * BN;
    // two 16-voxel row blocks per warp: voxel vi = 16 m + r of the brick,
    // (vi % 8, (vi / 8) % 8, vi / 64)
    float acc[2][BN / 8][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int j = 0; j < BN / 8; ++j) acc[m][j][0] = acc[m][j][1] = acc[m][j][2] = acc[m][j][3] = 0.f;
    // this lane's A row (voxel) of each row block, as a halo index at tap (0,0,0)
    int hrow[2];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const int vi = (warp * 2 + m) * 16 + (lane & 15);
        const int vx = vi % kBX, vy = (vi / kBX) % kBY, vz = vi / (kBX * kBY);
        hrow[m] = (vx + 1) + kHX * ((vy + 1) + kHY * (vz + 1));
    }
    const int achunk = (lane >> 4) * 8;   // channel half of the A fragment
    for (int c0 = 0; c0 < Cin; c0 += 16) {
        __syncthreads();   // the previous chunk's tiles are no longer read
        for (int e = tid; e < kHalo * 2; e += 256) {
            const int hv = e >> 1, h = e & 1;
            const int hx = hv % kHX, hy = (hv / kHX) % kHY, hz = hv / (kHX * kHY);
            const size_t g = (size_t)wrapd(x0, hx - 1, n) +
                             (size_t)n * ((size_t)wrapd(y0, hy - 1, n) + (size_t)n * wrapd(z0, hz - 1, n));
            *reinterpret_cast<uint4*>(halo + hv * kHRow + h * 8) =
                *reinterpret_cast<const uint4*>(in + g * Cin + c0 + h * 8);
        }
        constexpr int WCH = BN / 8;
        for (int e = tid; e < 27 * 16 * WCH; e += 256) {
            const int t = e / (16 * WCH), r = (e / WCH) % 16, cc = e % WCH;
            *reinterpret_cast<uint4*>(ws + (t * 16 + r) * WROW + cc * 8) =
                *reinterpret_cast<const uint4*>(W + ((size_t)t * Cin + c0 + r) * Cout + co0 + cc * 8);
        }
        __syncthreads();
#pragma unroll 1
        for (int t = 0; t < 27; ++t) {
            const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
            const int hoff = dx + kHX * (dy + kHY * dz);
            unsigned bfr[BN / 16][4];
#pragma unroll
            for (int j = 0; j < BN / 16; ++j)
                ldsm_x4_t(bfr[j], ws + (t * 16 + (lane & 15)) * WROW + j * 16 + (lane >> 4) * 8);
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                unsigned af[4];
                ldsm_x4(af, halo + (hrow[m] + hoff) * kHRow + achunk);
#pragma unroll
                for (int j = 0; j < BN / 16; ++j) {
                    mma_bf16(acc[m][2 * j], af, bfr[j][0], bfr[j][1]);
                    mma_bf16(acc[m][2 * j + 1], af, bfr[j][2], bfr[j][3]);
                }
            }
        }
    }
    // epilogue: bias, activation, BF16 store
#pragma unroll
    for (int m = 0; m < 2; ++m) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int vi = (warp * 2 + m) * 16 + (lane >> 2) + 8 * h;
            const int vx = vi % kBX, vy = (vi / kBX) % kBY, vz = vi / (kBX * kBY);
            const size_t g = (size_t)(x0 + vx) + (size_t)n * ((size_t)(y0 + vy) + (size_t)n * (z0 + vz));
#pragma unroll
            for (int j = 0; j < BN / 8; ++j) {
                const int co = co0 + j * 8 + (lane & 3) * 2;
                float y0v = acc[m][j][2 * h] + (bias ? bias[co] : 0.f);
                float y1v = acc[m][j][2 * h + 1] + (bias ? bias[co + 1] : 0.f);
                if (RELU) {
                    y0v = fmaxf(y0v, 0.f);
                    y1v = fmaxf(y1v, 0.f);
                }
                *reinterpret_cast<__nv_bfloat162*>(out + g * Cout + co) = __floats2bfloat162_rn(y0v, y1v);
            }
        }
    }
}

}  // namespace nn
}  // namespace otm

namespace otm {
namespace nn {

// Brick-tiled weight gradient (same contract as k_conv3_dw):
//   dW[t][ci][co] += sum_v in[v + d_t][ci] g[v][co],  db[co] += sum_v g[v][co].
// Grid (P, Cin / 16, Cout / BN).  CTA p walks the bricks p, p + P, ... of the
// n^3 grid (8 x 8 x 4 voxels each): it stages the brick's input halo for its
// 16-channel chunk and the brick's output gradient for its BN channels, and
// warp w accumulates the taps w, w + 8, w + 16, w + 24 (< 27) as 16 x BN
// products over the brick's 256 voxels (16 k-steps of 16 voxels; A = the
// shifted input transposed, B = the gradient, both by ldmatrix.trans).  The
// per-tap partials stay in registers across the CTA's bricks and are added
// to dW once, at the end.  Requires n % 8 == 0 and 4 | n.
constexpr int kDwTaps = 4;

inline size_t conv3_dw_tile_smem(int bn) { return (size_t)kHalo * kHRow * 2 + (size_t)kBX * kBY * kBZ * (bn + 8) * 2; }

template <int BN>
__global__ void __launch_bounds__(256)
k_conv3_dw_tile(int n, int Cin, int Ca, int Cout, const bf16* __restrict__ in, const bf16* __restrict__ g,
                float* __restrict__ dW, float* __restrict__ db) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char dw_sm[];
    bf16* halo = reinterpret_cast<bf16*>(dw_sm);        // [kHalo][kHRow]
    bf16* gs = halo + kHalo * kHRow;                      // [256][BN + 8]
    constexpr int GROW = BN + 8;
    constexpr int NV = kBX * kBY * kBZ;                   // 256 voxels per brick
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ci0 = blockIdx.y * 16, co0 = blockIdx.z * BN;
    const int nbx = n / kBX, nby = n / kBY, nbz = n / kBZ;
    const int nbricks = nbx * nby * nbz;
    float acc[kDwTaps][BN / 8][4];
#pragma unroll
    for (int q = 0; q < kDwTaps; ++q)
#pragma unroll
        for (int j = 0; j < BN / 8; ++j) acc[q][j][0] = acc[q][j][1] = acc[q][j][2] = acc[q][j][3] = 0.f;
    float bsum = 0.f;
    const bool do_db = db != nullptr && blockIdx.y == 0 && tid < BN;
    // this lane's voxel (A^T row block: 16 voxels per k-step) and channel half
    const int lr = (lane & 7) + ((lane >> 4) << 3), lc = ((lane >> 3) & 1) * 8;
    for (int b = blockIdx.x; b < nbricks; b += gridDim.x) {
        const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
        const int x0 = bx * kBX, y0 = by * kBY, z0 = bz * kBZ;
        __syncthreads();   // the previous brick's tiles are no longer read
        for (int e = tid; e < kHalo * 2; e += 256) {
            const int hv = e >> 1, h = e & 1;
            const int hx = hv % kHX, hy = (hv / kHX) % kHY, hz = hv / (kHX * kHY);
            const size_t gv = (size_t)wrapd(x0, hx - 1, n) +
                              (size_t)n * ((size_t)wrapd(y0, hy - 1, n) + (size_t)n * wrapd(z0, hz - 1, n));
            *reinterpret_cast<uint4*>(halo + hv * kHRow + h * 8) =
                *reinterpret_cast<const uint4*>(in + gv * Cin + ci0 + h * 8);
        }
        constexpr int GCH = BN / 8;
        for (int e = tid; e < NV * GCH; e += 256) {
            const int vi = e / GCH, cc = e % GCH;
            const int vx = vi % kBX, vy = (vi / kBX) % kBY, vz = vi / (kBX * kBY);
            const size_t gv = (size_t)(x0 + vx) + (size_t)n * ((size_t)(y0 + vy) + (size_t)n * (z0 + vz));
            *reinterpret_cast<uint4*>(gs + vi * GROW + cc * 8) =
                *reinterpret_cast<const uint4*>(g + gv * Cout + co0 + cc * 8);
        }
        __syncthreads();
        if (do_db)
            for (int r = 0; r < NV; ++r) bsum += __bfloat162float(gs[r * GROW + tid]);
#pragma unroll 1
        for (int ks = 0; ks < NV / 16; ++ks) {
            unsigned bfr[BN / 16][4];
#pragma unroll
            for (int j = 0; j < BN / 16; ++j)
                ldsm_x4_t(bfr[j], gs + (ks * 16 + (lane & 15)) * GROW + j * 16 + (lane >> 4) * 8);
            // this lane's voxel of the k-step, as a halo index at tap (0, 0, 0)
            const int vi = ks * 16 + lr;
            const int hv0 = (vi % kBX + 1) + kHX * (((vi / kBX) % kBY + 1) + kHY * (vi / (kBX * kBY) + 1));
#pragma unroll
            for (int q = 0; q < kDwTaps; ++q) {
                const int t = warp + 8 * q;
                if (t < 27) {
                    const int hoff = (t % 3 - 1) + kHX * ((t / 3) % 3 - 1 + kHY * (t / 9 - 1));
                    unsigned af[4];
                    ldsm_x4_t(af, halo + (hv0 + hoff) * kHRow + lc);
#pragma unroll
                    for (int j = 0; j < BN / 16; ++j) {
                        mma_bf16(acc[q][2 * j], af, bfr[j][0], bfr[j][1]);
                        mma_bf16(acc[q][2 * j + 1], af, bfr[j][2], bfr[j][3]);
                    }
                }
            }
        }
    }
    // add the partials: rows ci (lane >> 2, + 8), columns co
#pragma unroll
    for (int q = 0; q < kDwTaps; ++q) {
        const int t = warp + 8 * q;
        if (t >= 27) continue;
#pragma unroll
        for (int j = 0; j < BN / 8; ++j) {
            const int c = co0 + j * 8 + (lane & 3) * 2;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ci = ci0 + (lane >> 2) + 8 * h;
                if (ci < Ca) {
                    atomicAdd(dW + ((size_t)t * Ca + ci) * Cout + c, acc[q][j][2 * h]);
                    atomicAdd(dW + ((size_t)t * Ca + ci) * Cout + c + 1, acc[q][j][2 * h + 1]);
                }
            }
        }
    }
    if (do_db) atomicAdd(db + co0 + tid, bsum);
}

}  // namespace nn
}  // namespace otm
