// Mip chain of an RGBA8 texture (Sec. 3.3 relies on mipmapped textures):
// texel (x, y) of level l+1 is the rounded 2x2 box mean (a+b+c+d+2)>>2 of
// level l, indices clamped at the level's edge. One thread per output texel.
#include "lfdpr_internal.cuh"

namespace lfdpr {
namespace {

__global__ void __launch_bounds__(256) k_mip_level(const uint32_t* __restrict__ src, uint32_t sw,
                                                    uint32_t sh, uint32_t* __restrict__ dst, uint32_t dw,
                                                    uint32_t dh) {
    const uint64_t n = (uint64_t)dw * dh;
    for (uint64_t o = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n;
         o += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t y = uint32_t(o / dw), x = uint32_t(o - (uint64_t)y * dw);
        const uint32_t x0 = min(2 * x, sw - 1), x1 = min(2 * x + 1, sw - 1);
        const uint32_t y0 = min(2 * y, sh - 1), y1 = min(2 * y + 1, sh - 1);
        const uint32_t a = src[(uint64_t)y0 * sw + x0], b = src[(uint64_t)y0 * sw + x1];
        const uint32_t c = src[(uint64_t)y1 * sw + x0], d = src[(uint64_t)y1 * sw + x1];
        uint32_t out = 0;
#pragma unroll
        for (int ch = 0; ch < 4; ch++) {
            const uint32_t s = ((a >> (8 * ch)) & 255u) + ((b >> (8 * ch)) & 255u) +
                               ((c >> (8 * ch)) & 255u) + ((d >> (8 * ch)) & 255u);
            out |= ((s + 2u) >> 2) << (8 * ch);
        }
        dst[o] = out;
    }
}

}  // namespace

cudaError_t launch_mip_level(const uint8_t* src, uint32_t sw, uint32_t sh, uint8_t* dst, uint32_t dw,
                             uint32_t dh, cudaStream_t s) {
    const uint64_t n = (uint64_t)dw * dh;
    const uint64_t blocks = (n + 255) / 256;
    const unsigned grid = unsigned(blocks < 4096 ? blocks : 4096);
    k_mip_level<<<grid, 256, 0, s>>>(reinterpret_cast<const uint32_t*>(src), sw, sh,
                                     reinterpret_cast<uint32_t*>(dst), dw, dh);
    return cudaGetLastError();
}

}  // namespace lfdpr
