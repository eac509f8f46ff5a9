// Learned angular reconstruction: the U-Net's layers as BF16 tensor-core
// kernels with FP32 accumulation (activations NHWC bf16, channels padded to
// multiples of 16).
//
//   k_conv3x3     3x3 convolution, stride 1, zero padding 1, + bias, ReLU:
//                 implicit GEMM (pixels x output channels x 9 Cin). A block
//                 takes 8 rows x 32 pixels x 64 (or 32) output channels; per
//                 chunk of 16 input channels it stages (cp.async, two stages,
//                 so copies overlap the MMAs) the 10 x 34 pixel halo tile and
//                 the 64 x 9 x 16 weights in shared memory, and each warp
//                 (one row, two m16 tiles) runs ldmatrix + mma.m16n8k16 over
//                 the 9 taps, reading the tap-shifted pixel rows straight
//                 from the halo tile.
//   k_avgpool2    2x2 average pooling.
//   k_up2_concat  nearest 2x upsampling of one tensor concatenated (along
//                 channels) with another of the upsampled size.
//   k_recon_in    12 rendered views RGBA8 -> the network input (36 channels
//                 of [0, 1] values, zero padded to 48 channels and to a
//                 width divisible by 8).
//   k_recon_out   the 1x1 output layer plus the fixed angular interpolation
//                 of the input views as one tensor-core GEMM per 16 pixels,
//                 clamped and rounded to the 48 output views RGBA8.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "objects.h"

namespace lfdpr {
namespace {

constexpr int kConvTH = 8;           // tile rows (one warp each)
constexpr int kConvTW = 32;          // tile pixels per row (two m16 tiles)
constexpr int kConvCK = 16;          // input channels per chunk
constexpr int kConvRow = kConvCK + 8;  // smem row stride (elements): 48 B, conflict-free ldmatrix rows

__device__ __forceinline__ void ldmatrix_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float* d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// 16-byte global -> shared copy that bypasses L1 (cp.async); src_bytes 0
// fills the 16 bytes with zeros without reading src.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N));
}

// in [H][W][Cin], wgt [Cout][9][Cin] (tap = 3 dy + dx), bias [Cout] f32,
// out [H][W][Cout]; Cin % 16 == 0, Cout % CO == 0 (CO = 32 or 64 output
// channels per block). Grid (ceil(W/32), ceil(H/8), Cout/CO), 256 threads,
// dynamic shared memory conv_smem_bytes(CO): two stages of (halo tile,
// weights) so the next chunk's copies run during this chunk's MMAs.
template <int CO>
__global__ void __launch_bounds__(256) k_conv3x3(const __nv_bfloat16* __restrict__ in, int H, int W, int Cin,
                                                 const __nv_bfloat16* __restrict__ wgt,
                                                 const float* __restrict__ bias, __nv_bfloat16* __restrict__ out,
                                                 int Cout, int relu) {
    constexpr int HP = kConvTH + 2, WP = kConvTW + 2;
    constexpr int NT = CO / 8;                               // n8 tiles per warp
    constexpr int IN_ELEMS = HP * WP * kConvRow, W_ELEMS = CO * 9 * kConvRow;
    constexpr int STAGE = IN_ELEMS + W_ELEMS;                // elements per stage
    extern __shared__ __align__(16) __nv_bfloat16 smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = blockIdx.x * kConvTW, y0 = blockIdx.y * kConvTH, n0 = blockIdx.z * CO;
    float acc[2][NT][4];
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
        for (int t = 0; t < NT; t++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[m][t][q] = 0.0f;

    const uint32_t s_base = uint32_t(__cvta_generic_to_shared(smem));
    // ldmatrix row addresses of this lane: A (pixels) and B (output channels)
    const int a_row = (lane & 7) + 8 * ((lane >> 3) & 1), a_k = 8 * (lane >> 4);
    const int b_row = (lane & 7) + 8 * (lane >> 4), b_k = 8 * ((lane >> 3) & 1);

    // copies of channel chunk c0 into stage st
    auto stage_copy = [&](int c0, int st) {
        const uint32_t s_in = s_base + uint32_t(st * STAGE * 2), s_w = s_in + uint32_t(IN_ELEMS * 2);
        for (int idx = tid; idx < HP * WP * 2; idx += 256) {
            const int p = idx >> 1, part = idx & 1;
            const int gy = y0 + p / WP - 1, gx = x0 + p % WP - 1;
            const bool ok = gy >= 0 && gy < H && gx >= 0 && gx < W;
            const __nv_bfloat16* src = ok ? in + ((size_t)gy * W + gx) * Cin + c0 + 8 * part : in;
            cp_async16(s_in + uint32_t((p * kConvRow + 8 * part) * 2), src, ok ? 16u : 0u);
        }
        for (int idx = tid; idx < CO * 9 * 2; idx += 256) {
            const int row = idx >> 1, part = idx & 1;   // row = co * 9 + tap
            const int co = row / 9, tap = row - 9 * co;
            cp_async16(s_w + uint32_t((row * kConvRow + 8 * part) * 2),
                       wgt + ((size_t)(n0 + co) * 9 + tap) * Cin + c0 + 8 * part, 16u);
        }
        cp_async_commit();
    };

    const int n_chunks = Cin / kConvCK;
    stage_copy(0, 0);
    for (int ch = 0; ch < n_chunks; ch++) {
        if (ch + 1 < n_chunks) {
            stage_copy((ch + 1) * kConvCK, (ch + 1) & 1);
            cp_async_wait<1>();   // this chunk's group has landed
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const uint32_t s_in_a = s_base + uint32_t((ch & 1) * STAGE * 2), s_w_a = s_in_a + uint32_t(IN_ELEMS * 2);
#pragma unroll
        for (int tap = 0; tap < 9; tap++) {
            const int dy = tap / 3, dx = tap - 3 * (tap / 3);
            uint32_t a[2][4];
#pragma unroll
            for (int m = 0; m < 2; m++) {
                const int p = (warp + dy) * WP + 16 * m + a_row + dx;
                ldmatrix_x4(s_in_a + uint32_t((p * kConvRow + a_k) * 2), a[m][0], a[m][1], a[m][2], a[m][3]);
            }
#pragma unroll
            for (int t2 = 0; t2 < NT / 2; t2++) {
                uint32_t b0, b1, b2, b3;
                const int row = (16 * t2 + b_row) * 9 + tap;
                ldmatrix_x4(s_w_a + uint32_t((row * kConvRow + b_k) * 2), b0, b1, b2, b3);
#pragma unroll
                for (int m = 0; m < 2; m++) {
                    mma_bf16(acc[m][2 * t2], a[m][0], a[m][1], a[m][2], a[m][3], b0, b1);
                    mma_bf16(acc[m][2 * t2 + 1], a[m][0], a[m][1], a[m][2], a[m][3], b2, b3);
                }
            }
        }
        __syncthreads();   // the stage is refilled two chunks later
    }
    // epilogue: bias, ReLU, bf16 pairs
    const int y = y0 + warp;
    if (y >= H) return;
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
        for (int t = 0; t < NT; t++) {
            const int co = n0 + 8 * t + 2 * (lane & 3);
            const float b0 = bias[co], b1 = bias[co + 1];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int x = x0 + 16 * m + (lane >> 2) + 8 * h;
                if (x >= W) continue;
                float v0 = acc[m][t][2 * h] + b0, v1 = acc[m][t][2 * h + 1] + b1;
                if (relu) {
                    v0 = fmaxf(v0, 0.0f);
                    v1 = fmaxf(v1, 0.0f);
                }
                *reinterpret_cast<__nv_bfloat162*>(out + ((size_t)y * W + x) * Cout + co) = __floats2bfloat162_rn(v0, v1);
            }
        }
}

constexpr size_t conv_smem_bytes(int co) {
    return size_t(2) * (size_t((kConvTH + 2) * (kConvTW + 2) * kConvRow) + size_t(co * 9 * kConvRow)) * 2;
}

// out [H/2][W/2][C] = mean of 2x2 blocks of in [H][W][C] (H, W even; C % 8 == 0).
__global__ void k_avgpool2(const __nv_bfloat16* __restrict__ in, int H, int W, int C, __nv_bfloat16* __restrict__ out) {
    const int Ho = H / 2, Wo = W / 2, C8 = C / 8;
    const size_t total = (size_t)Ho * Wo * C8;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int c8 = int(i % C8);
        const size_t p = i / C8;
        const int xo = int(p % Wo), yo = int(p / Wo);
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int yy = 2 * yo + (q >> 1), xx = 2 * xo + (q & 1);
            const uint4 v = *reinterpret_cast<const uint4*>(in + ((size_t)yy * W + xx) * C + 8 * c8);
            const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const float2 f = __bfloat1622float2(h[e]);
                s[2 * e] += f.x;
                s[2 * e + 1] += f.y;
            }
        }
        uint4 o;
        __nv_bfloat162* oh = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
        for (int e = 0; e < 4; e++) oh[e] = __floats2bfloat162_rn(0.25f * s[2 * e], 0.25f * s[2 * e + 1]);
        *reinterpret_cast<uint4*>(out + p * C + 8 * c8) = o;
    }
}

// out [H][W][Ca + Cb]: channels [0, Ca) = a [H/2][W/2][Ca] at (y/2, x/2),
// channels [Ca, Ca + Cb) = b [H][W][Cb] (Ca, Cb % 8 == 0).
__global__ void k_up2_concat(const __nv_bfloat16* __restrict__ a, int Ca, const __nv_bfloat16* __restrict__ b, int Cb,
                             int H, int W, __nv_bfloat16* __restrict__ out) {
    const int C = Ca + Cb, C8 = C / 8;
    const size_t total = (size_t)H * W * C8;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int c = 8 * int(i % C8);
        const size_t p = i / C8;
        const int x = int(p % W), y = int(p / W);
        uint4 v;
        if (c < Ca)
            v = *reinterpret_cast<const uint4*>(a + ((size_t)(y / 2) * (W / 2) + x / 2) * Ca + c);
        else
            v = *reinterpret_cast<const uint4*>(b + p * Cb + (c - Ca));
        *reinterpret_cast<uint4*>(out + p * C + c) = v;
    }
}

// x0 [Hp][Wp][48]: channel 3 j + c = channel c of input view j / 255 for
// j < nin (nin <= 16), zero elsewhere and outside the H x W views.
__global__ void k_recon_in(const uint8_t* __restrict__ views, int nin, int H, int W, int Hp, int Wp,
                           __nv_bfloat16* __restrict__ x0) {
    const size_t total = (size_t)Hp * Wp * 6;   // 6 groups of 8 channels
    const size_t npix = (size_t)H * W;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int g = int(i % 6);
        const size_t p = i / 6;
        const int x = int(p % Wp), y = int(p / Wp);
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const int ch = 8 * g + e, j = ch / 3, c = ch - 3 * j;
            v[e] = 0.0f;
            if (j < nin && x < W && y < H)
                v[e] = float(views[((size_t)j * npix + (size_t)y * W + x) * 4 + c]) * (1.0f / 255.0f);
        }
        uint4 o;
        __nv_bfloat162* oh = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
        for (int e = 0; e < 4; e++) oh[e] = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
        *reinterpret_cast<uint4*>(x0 + p * 48 + 8 * g) = o;
    }
}

// The output layer as one tensor-core GEMM per 16 pixels: [d0 (32) | x0 (48)]
// x [w_out ; angular base] (80 x 3 nout, bf16 in shared memory as
// [3 nout][kOutK]) + b_out, clamped to [0, 1], times 255, rounded half to
// even, alpha 255 -> views_out [nout][H][W][4]. The base rows give output
// view k, channel c the linear angular interpolation of the input views
// (input j at output index 4 j + 3/2, clamped at the ends); its weights
// (0, 1/8, 3/8, 5/8, 7/8, 1) are exact in bf16. Each warp stages its 16
// pixels' RGBA8 words in shared memory and writes them view by view.
constexpr int kOutK = 80 + 8;   // smem row stride of the output weights (elements)
__global__ void __launch_bounds__(256) k_recon_out(const __nv_bfloat16* __restrict__ d0,
                                                   const __nv_bfloat16* __restrict__ x0, int nin, int H, int W,
                                                   int Hp, int Wp, const __nv_bfloat16* __restrict__ w_out,
                                                   const float* __restrict__ b_out, uint8_t* __restrict__ views_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nout = 4 * nin, no3 = 3 * nout, nt = no3 / 8;   // n8 tiles (no3 % 8 == 0: nin even)
    __nv_bfloat16* s_w = reinterpret_cast<__nv_bfloat16*>(smem_raw);                        // [no3][kOutK]
    float* s_b = reinterpret_cast<float*>(smem_raw + sizeof(__nv_bfloat16) * no3 * kOutK);  // [no3]
    uint32_t* s_px = reinterpret_cast<uint32_t*>(s_b + no3);                                // [8 warps][16][nout]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < no3 * 80; i += blockDim.x) {
        const int o = i / 80, k = i - 80 * o;
        s_w[o * kOutK + k] = w_out[i];
    }
    for (int i = tid; i < no3; i += blockDim.x) s_b[i] = b_out[i];
    __syncthreads();
    uint32_t* px = s_px + warp * 16 * nout;
    const size_t npix = (size_t)H * W, ptot = (size_t)Hp * Wp;
    const int r0 = lane >> 2, kq = 2 * (lane & 3);
    for (size_t t0 = ((size_t)blockIdx.x * 8 + warp) * 16; t0 < ptot; t0 += (size_t)gridDim.x * 8 * 16) {
        // A fragments: rows t0 + r0 and t0 + r0 + 8 (padded pixels), 5 k16 steps over [d0 | x0]
        uint32_t a[5][4];
#pragma unroll
        for (int ks = 0; ks < 5; ks++)
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const size_t p = t0 + r0 + 8 * (q & 1);
                const int k = 16 * ks + kq + 8 * (q >> 1);
                const __nv_bfloat16* src = k < 32 ? d0 + p * 32 + k : x0 + p * 48 + (k - 32);
                a[ks][q] = p < ptot ? *reinterpret_cast<const uint32_t*>(src) : 0u;
            }
        for (int i = lane; i < 16 * nout; i += 32) px[i] = 0xff000000u;
        __syncwarp();
        for (int t = 0; t < nt; t++) {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            const int n = 8 * t + r0;
#pragma unroll
            for (int ks = 0; ks < 5; ks++) {
                const uint32_t b0 = *reinterpret_cast<const uint32_t*>(s_w + n * kOutK + 16 * ks + kq);
                const uint32_t b1 = *reinterpret_cast<const uint32_t*>(s_w + n * kOutK + 16 * ks + kq + 8);
                mma_bf16(acc, a[ks][0], a[ks][1], a[ks][2], a[ks][3], b0, b1);
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int o = 8 * t + kq + (q & 1), row = r0 + 8 * (q >> 1);
                const float v = fminf(fmaxf(acc[q] + s_b[o], 0.0f), 1.0f) * 255.0f;
                const int kv = o / 3, c = o - 3 * kv;
                reinterpret_cast<uint8_t*>(px + row * nout + kv)[c] = uint8_t(rintf(v));
            }
        }
        __syncwarp();
        // write the 16 pixels' words, view by view
        for (int i = lane; i < 16 * nout; i += 32) {
            const int kv = i >> 4, row = i & 15;
            const size_t p = t0 + row;
            if (p >= ptot) continue;
            const int y = int(p / Wp), x = int(p - (size_t)y * Wp);
            if (y < H && x < W)
                reinterpret_cast<uint32_t*>(views_out)[(size_t)kv * npix + (size_t)y * W + x] = px[row * nout + kv];
        }
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_conv3x3(const __nv_bfloat16* in, int H, int W, int Cin, const __nv_bfloat16* wgt,
                           const float* bias, __nv_bfloat16* out, int Cout, bool relu, cudaStream_t s) {
    if (H < 1 || W < 1 || Cin < kConvCK || Cin % kConvCK || Cout < 32 || Cout % 32) return cudaErrorInvalidValue;
    static bool attrs[64] = {};   // opt in to the two-stage shared memory once per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attrs[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_conv3x3<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(conv_smem_bytes(64)));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_conv3x3<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(conv_smem_bytes(32)));
        if (e != cudaSuccess) return e;
        attrs[dev] = true;
    }
    if (Cout % 64 == 0) {
        const dim3 grid((W + kConvTW - 1) / kConvTW, (H + kConvTH - 1) / kConvTH, Cout / 64);
        k_conv3x3<64><<<grid, 256, conv_smem_bytes(64), s>>>(in, H, W, Cin, wgt, bias, out, Cout, relu ? 1 : 0);
    } else {
        const dim3 grid((W + kConvTW - 1) / kConvTW, (H + kConvTH - 1) / kConvTH, Cout / 32);
        k_conv3x3<32><<<grid, 256, conv_smem_bytes(32), s>>>(in, H, W, Cin, wgt, bias, out, Cout, relu ? 1 : 0);
    }
    return cudaGetLastError();
}

cudaError_t launch_avgpool2(const __nv_bfloat16* in, int H, int W, int C, __nv_bfloat16* out, int sm_count,
                            cudaStream_t s) {
    if (H < 2 || W < 2 || (H & 1) || (W & 1) || C % 8) return cudaErrorInvalidValue;
    k_avgpool2<<<sm_count * 8, 256, 0, s>>>(in, H, W, C, out);
    return cudaGetLastError();
}

cudaError_t launch_up2_concat(const __nv_bfloat16* a, int Ca, const __nv_bfloat16* b, int Cb, int H, int W,
                              __nv_bfloat16* out, int sm_count, cudaStream_t s) {
    if (H < 2 || W < 2 || (H & 1) || (W & 1) || Ca % 8 || Cb % 8) return cudaErrorInvalidValue;
    k_up2_concat<<<sm_count * 8, 256, 0, s>>>(a, Ca, b, Cb, H, W, out);
    return cudaGetLastError();
}

}  // namespace lfdpr

// ---------------------------------------------------------------------------
// The network (host side)
// ---------------------------------------------------------------------------

using namespace lfdpr;

namespace {

struct ConvSpec {
    int cin, cout, level;   // input channels (padded), output channels, resolution level 0..3
};
// The U-Net's 3x3 layers in order (two per level down, a bottleneck pair, two
// per level up; up-path inputs are [upsampled, skip] concatenations).
const ConvSpec kLayers[14] = {{48, 32, 0},  {32, 32, 0},   {32, 64, 1},   {64, 64, 1},   {64, 128, 2},
                              {128, 128, 2}, {128, 256, 3}, {256, 256, 3}, {384, 128, 2}, {128, 128, 2},
                              {192, 64, 1},  {64, 64, 1},   {96, 32, 0},   {32, 32, 0}};

}  // namespace

struct lfdpr_recon {
    int W = 0, H = 0, Wp = 0, Hp = 0, nin = 0, nout = 0, sm_count = 1;
    __nv_bfloat16* w = nullptr;   // all 3x3 weights, layer by layer [cout][9][cin]
    float* b = nullptr;           // all 3x3 biases
    __nv_bfloat16* w_out = nullptr;   // [3 nout][80]: the 1x1 layer (32) then the angular base (48)
    float* b_out = nullptr;           // [3 nout]
    int64_t w_off[14] = {}, b_off[14] = {};
    __nv_bfloat16* act = nullptr;  // activation arena
    __nv_bfloat16 *x0, *e0a, *e0, *p1, *e1a, *e1, *p2, *e2a, *e2, *p3, *ba, *bb, *u2, *d2a, *d2, *u1, *d1a, *d1, *u0,
        *d0a, *d0;
};

namespace {

void free_recon(lfdpr_recon* r) {
    if (!r) return;
    cudaFree(r->w);
    cudaFree(r->b);
    cudaFree(r->w_out);
    cudaFree(r->b_out);
    cudaFree(r->act);
    delete r;
}

}  // namespace

extern "C" {

int64_t lfdpr_recon_weight_count(int32_t in_views) {
    int64_t n = 0;
    for (const auto& L : kLayers) n += int64_t(L.cout) * 9 * L.cin;
    return n + int64_t(3 * 4 * in_views) * 32;
}

int64_t lfdpr_recon_bias_count(int32_t in_views) {
    int64_t n = 0;
    for (const auto& L : kLayers) n += L.cout;
    return n + 3 * 4 * in_views;
}

lfdpr_status lfdpr_create_recon(int32_t view_w, int32_t view_h, int32_t in_views, const uint16_t* weights_bf16,
                                int64_t n_weights, const float* biases, int64_t n_biases, lfdpr_recon** out) {
    lfdpr::g_last_error[0] = 0;
    if (!out || !weights_bf16 || !biases) return fail(LFDPR_EINVAL, "create_recon: null argument");
    *out = nullptr;
    if (in_views < 2 || in_views > 16 || (in_views & 1))
        return fail(LFDPR_EINVAL, "create_recon: in_views must be even, in [2, 16]");
    if (view_w < 8 || view_h < 8 || view_w > 4096 || view_h > 4096)
        return fail(LFDPR_EINVAL, "create_recon: views must be 8..4096 pixels a side");
    if (n_weights != lfdpr_recon_weight_count(in_views) || n_biases != lfdpr_recon_bias_count(in_views))
        return fail(LFDPR_EINVAL, "create_recon: expected %lld weights and %lld biases",
                    (long long)lfdpr_recon_weight_count(in_views), (long long)lfdpr_recon_bias_count(in_views));
    lfdpr_recon* r = new (std::nothrow) lfdpr_recon();
    if (!r) return fail(LFDPR_ENOMEM, "host allocation failed");
    r->W = view_w;
    r->H = view_h;
    r->Wp = (view_w + 7) / 8 * 8;
    r->Hp = (view_h + 7) / 8 * 8;
    r->nin = in_views;
    r->nout = 4 * in_views;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&r->sm_count, cudaDevAttrMultiProcessorCount, dev);
    int64_t wo = 0, bo = 0;
    for (int l = 0; l < 14; l++) {
        r->w_off[l] = wo;
        r->b_off[l] = bo;
        wo += int64_t(kLayers[l].cout) * 9 * kLayers[l].cin;
        bo += kLayers[l].cout;
    }
    // activation arena: every tensor of the forward pass, 256-byte aligned
    const int64_t P0 = int64_t(r->Hp) * r->Wp, P1 = P0 / 4, P2 = P0 / 16, P3 = P0 / 64;
    const int64_t sizes[21] = {P0 * 48, P0 * 32, P0 * 32, P1 * 32, P1 * 64, P1 * 64, P2 * 64,
                               P2 * 128, P2 * 128, P3 * 128, P3 * 256, P3 * 256, P2 * 384, P2 * 128,
                               P2 * 128, P1 * 192, P1 * 64, P1 * 64, P0 * 96, P0 * 32, P0 * 32};
    int64_t offs[21], total = 0;
    for (int k = 0; k < 21; k++) {
        offs[k] = total;
        total += (sizes[k] + 127) / 128 * 128;
    }
    cudaError_t e;
    const int64_t nw3 = wo, nb3 = bo;
    if ((e = cudaMalloc(&r->w, 2 * nw3)) != cudaSuccess || (e = cudaMalloc(&r->b, 4 * nb3)) != cudaSuccess ||
        (e = cudaMalloc(&r->w_out, 2 * int64_t(3 * r->nout) * 80)) != cudaSuccess ||
        (e = cudaMalloc(&r->b_out, 4 * int64_t(3 * r->nout))) != cudaSuccess ||
        (e = cudaMalloc(&r->act, 2 * total)) != cudaSuccess) {
        free_recon(r);
        return cuda_fail(e, "create_recon: cudaMalloc");
    }
    __nv_bfloat16** bufs[21] = {&r->x0, &r->e0a, &r->e0, &r->p1, &r->e1a, &r->e1, &r->p2, &r->e2a, &r->e2, &r->p3,
                                &r->ba, &r->bb,  &r->u2, &r->d2a, &r->d2, &r->u1, &r->d1a, &r->d1, &r->u0, &r->d0a, &r->d0};
    for (int k = 0; k < 21; k++) *bufs[k] = r->act + offs[k];
    // the output layer: its 32 weights, then the angular base over the 48
    // input channels (bf16 bit patterns: 1/8, 3/8, 5/8, 7/8 and 1 are exact)
    const int no3 = 3 * r->nout;
    std::vector<uint16_t> wout(size_t(no3) * 80, 0);
    auto bf16_bits = [](float f) {
        uint32_t u;
        std::memcpy(&u, &f, 4);
        return uint16_t(u >> 16);   // exact for the base weights
    };
    for (int o = 0; o < no3; o++) {
        for (int k = 0; k < 32; k++) wout[size_t(o) * 80 + k] = weights_bf16[nw3 + int64_t(o) * 32 + k];
        const int kv = o / 3, c = o - 3 * kv;
        const float pos = (float(kv) - 1.5f) * 0.25f;
        const int j0 = r->nin > 1 ? std::min(std::max(int(std::floor(pos)), 0), r->nin - 2) : 0;
        const float t = r->nin > 1 ? std::min(std::max(pos - float(j0), 0.0f), 1.0f) : 0.0f;
        const int j1 = r->nin > 1 ? j0 + 1 : j0;
        if (j1 == j0) {
            wout[size_t(o) * 80 + 32 + 3 * j0 + c] = bf16_bits(1.0f);
        } else {
            wout[size_t(o) * 80 + 32 + 3 * j0 + c] = bf16_bits(1.0f - t);
            wout[size_t(o) * 80 + 32 + 3 * j1 + c] = bf16_bits(t);
        }
    }
    if ((e = cudaMemcpy(r->w, weights_bf16, 2 * nw3, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(r->b, biases, 4 * nb3, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(r->w_out, wout.data(), 2 * wout.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(r->b_out, biases + nb3, 4 * int64_t(3 * r->nout), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(r->act, 0, 2 * total)) != cudaSuccess) {
        free_recon(r);
        return cuda_fail(e, "create_recon: upload");
    }
    *out = r;
    return LFDPR_OK;
}

lfdpr_status lfdpr_destroy_recon(lfdpr_recon* r) {
    lfdpr::g_last_error[0] = 0;
    if (!r) return fail(LFDPR_EINVAL, "destroy_recon: null");
    free_recon(r);
    return LFDPR_OK;
}

lfdpr_status lfdpr_recon_forward(lfdpr_recon* r, const uint8_t* in_views, uint8_t* out_views, void* stream) {
    lfdpr::g_last_error[0] = 0;
    if (!r || !in_views || !out_views) return fail(LFDPR_EINVAL, "recon_forward: null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int H0 = r->Hp, W0 = r->Wp, sm = r->sm_count;
    auto conv = [&](int l, const __nv_bfloat16* in, __nv_bfloat16* o, int H, int W) {
        return launch_conv3x3(in, H, W, kLayers[l].cin, r->w + r->w_off[l], r->b + r->b_off[l], o, kLayers[l].cout,
                              true, s);
    };
#define CKR(call, what)                                      \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);   \
    } while (0)
    k_recon_in<<<sm * 8, 256, 0, s>>>(in_views, r->nin, r->H, r->W, H0, W0, r->x0);
    CKR(cudaGetLastError(), "launch k_recon_in");
    CKR(conv(0, r->x0, r->e0a, H0, W0), "conv 0");
    CKR(conv(1, r->e0a, r->e0, H0, W0), "conv 1");
    CKR(launch_avgpool2(r->e0, H0, W0, 32, r->p1, sm, s), "pool 1");
    CKR(conv(2, r->p1, r->e1a, H0 / 2, W0 / 2), "conv 2");
    CKR(conv(3, r->e1a, r->e1, H0 / 2, W0 / 2), "conv 3");
    CKR(launch_avgpool2(r->e1, H0 / 2, W0 / 2, 64, r->p2, sm, s), "pool 2");
    CKR(conv(4, r->p2, r->e2a, H0 / 4, W0 / 4), "conv 4");
    CKR(conv(5, r->e2a, r->e2, H0 / 4, W0 / 4), "conv 5");
    CKR(launch_avgpool2(r->e2, H0 / 4, W0 / 4, 128, r->p3, sm, s), "pool 3");
    CKR(conv(6, r->p3, r->ba, H0 / 8, W0 / 8), "conv 6");
    CKR(conv(7, r->ba, r->bb, H0 / 8, W0 / 8), "conv 7");
    CKR(launch_up2_concat(r->bb, 256, r->e2, 128, H0 / 4, W0 / 4, r->u2, sm, s), "up 2");
    CKR(conv(8, r->u2, r->d2a, H0 / 4, W0 / 4), "conv 8");
    CKR(conv(9, r->d2a, r->d2, H0 / 4, W0 / 4), "conv 9");
    CKR(launch_up2_concat(r->d2, 128, r->e1, 64, H0 / 2, W0 / 2, r->u1, sm, s), "up 1");
    CKR(conv(10, r->u1, r->d1a, H0 / 2, W0 / 2), "conv 10");
    CKR(conv(11, r->d1a, r->d1, H0 / 2, W0 / 2), "conv 11");
    CKR(launch_up2_concat(r->d1, 64, r->e0, 32, H0, W0, r->u0, sm, s), "up 0");
    CKR(conv(12, r->u0, r->d0a, H0, W0), "conv 12");
    CKR(conv(13, r->d0a, r->d0, H0, W0), "conv 13");
    const size_t smem = 2 * size_t(3 * r->nout) * kOutK + 4 * size_t(3 * r->nout) + 4 * size_t(8 * 16 * r->nout);
    CKR(cudaFuncSetAttribute(k_recon_out, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)), "recon_out smem");
    k_recon_out<<<sm * 2, 256, smem, s>>>(r->d0, r->x0, r->nin, r->H, r->W, H0, W0, r->w_out, r->b_out, out_views);
    CKR(cudaGetLastError(), "launch k_recon_out");
#undef CKR
    return LFDPR_OK;
}

lfdpr_status lfdpr_recon_run(lfdpr_recon* r, const lfdpr_display* src, lfdpr_display* dst, void* stream) {
    lfdpr::g_last_error[0] = 0;
    if (!r || !src || !dst) return fail(LFDPR_EINVAL, "recon_run: null argument");
    if (src->dc.nr != r->nin || src->dc.W != r->W || src->dc.H != r->H)
        return fail(LFDPR_EINVAL, "recon_run: source display must render %d views of %dx%d", r->nin, r->W, r->H);
    if (dst->dc.nr != r->nout || dst->dc.W != r->W || dst->dc.H != r->H)
        return fail(LFDPR_EINVAL, "recon_run: target display must hold %d views of %dx%d", r->nout, r->W, r->H);
    return lfdpr_recon_forward(r, src->views, dst->views, stream);
}

lfdpr_status lfdpr_conv3x3_bf16(const void* in, int32_t H, int32_t W, int32_t cin, const void* wgt, const float* bias,
                                void* out, int32_t cout, int32_t relu, void* stream) {
    lfdpr::g_last_error[0] = 0;
    if (!in || !wgt || !bias || !out) return fail(LFDPR_EINVAL, "conv3x3: null argument");
    if (H < 1 || W < 1 || cin < 16 || cin % 16 || cout < 32 || cout % 32)
        return fail(LFDPR_EINVAL, "conv3x3: need cin %% 16 == 0, cout %% 32 == 0");
    const cudaError_t e =
        launch_conv3x3(static_cast<const __nv_bfloat16*>(in), H, W, cin, static_cast<const __nv_bfloat16*>(wgt), bias,
                       static_cast<__nv_bfloat16*>(out), cout, relu != 0, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "conv3x3");
    return LFDPR_OK;
}

}  // extern "C"
