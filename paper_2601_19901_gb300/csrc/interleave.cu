// Elemental image array construction (Sec. 4): optional angular tent
// reconstruction of the 2N supersampled views, optional +-1 crosstalk mixing,
// then the slanted-lens subpixel interleave. One thread per 4 horizontally
// adjacent panel pixels, one 16-byte store; the view reads are gathers that
// follow the lens phase.
#include "lfdpr_internal.cuh"

namespace lfdpr {
namespace {

__device__ __forceinline__ float texel(const uint8_t* __restrict__ views, uint64_t npix, int view,
                                       uint64_t pix, int ch) {
    return float(__ldg(views + ((uint64_t)view * npix + pix) * 4u + ch));
}

// Display view k, channel ch, at pixel pix, as binary32 before rounding.
__device__ __forceinline__ float display_value(const DispConst& c, const uint8_t* __restrict__ views,
                                               uint64_t npix, int k, uint64_t pix, int ch) {
    if (c.recon != 1) return texel(views, npix, k, pix, ch);
    float acc = 0.0f, ws = 0.0f;
#pragma unroll
    for (int q = 0; q < 3; q++) {
        const int m = 2 * k - 1 + q;
        if (m < 0 || m >= c.nr) continue;
        const float w = q == 1 ? 0.5f : 0.25f;
        acc = fmaf(w, texel(views, npix, m, pix, ch), acc);
        ws += w;
    }
    return __fdiv_rn(acc, ws);
}

__device__ __forceinline__ int view_of_subpixel(const DispConst& c, int x, int y, int ch) {
    const float third = ch == 0 ? (float)(1.0 / 6.0) : (ch == 1 ? 0.5f : (float)(5.0 / 6.0));
    const float cx = float(x) + third;
    const float a = fmaf(c.slant, float(y), cx);
    const float ph = fmaf(a, c.inv_pitch, c.phase_offset);
    const float fr = ph - floorf(ph);
    int k = int(fr * float(c.n_views));
    k = k >= c.n_views ? c.n_views - 1 : (k < 0 ? 0 : k);
    return k;
}

__global__ void __launch_bounds__(256) k_interleave(DispConst c, const uint8_t* __restrict__ views,
                                                     uint8_t* __restrict__ panel) {
    const uint64_t npix = (uint64_t)c.W * c.H;
    const int groups_x = (c.Wp + 3) >> 2;
    const uint64_t total = (uint64_t)groups_x * c.Hp;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const int y = int(g / groups_x);
        const int xg = int(g - (uint64_t)y * groups_x) * 4;
        const int sy = int(((int64_t)(2 * y + 1) * c.H) / (2 * (int64_t)c.Hp));
        uint32_t px[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const int x = xg + e;
            uint32_t o = 0xff000000u;
            if (x < c.Wp) {
                const int sx = int(((int64_t)(2 * x + 1) * c.W) / (2 * (int64_t)c.Wp));
                const uint64_t pix = (uint64_t)sy * c.W + sx;
#pragma unroll
                for (int ch = 0; ch < 3; ch++) {
                    const int k = view_of_subpixel(c, x, y, ch);
                    float val;
                    if (c.xtalk > 0.0f) {
                        const int km = k == 0 ? c.n_views - 1 : k - 1;
                        const int kp = k == c.n_views - 1 ? 0 : k + 1;
                        float acc = display_value(c, views, npix, k, pix, ch) * c.xtalk_c;
                        acc = fmaf(c.xtalk, display_value(c, views, npix, km, pix, ch), acc);
                        acc = fmaf(c.xtalk, display_value(c, views, npix, kp, pix, ch), acc);
                        val = acc;
                    } else {
                        val = display_value(c, views, npix, k, pix, ch);
                    }
                    o |= uint32_t(round_u8(val)) << (8 * ch);
                }
            }
            px[e] = o;
        }
        uint8_t* dst = panel + ((uint64_t)y * c.Wp + xg) * 4u;
        if (xg + 4 <= c.Wp && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0)) {
            *reinterpret_cast<uint4*>(dst) = make_uint4(px[0], px[1], px[2], px[3]);
        } else {
            for (int e = 0; e < 4 && xg + e < c.Wp; e++) reinterpret_cast<uint32_t*>(dst)[e] = px[e];
        }
    }
}

}  // namespace

cudaError_t launch_interleave(const DispConst& dc, const uint8_t* views, uint8_t* panel, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_interleave<<<sms * 8, 256, 0, s>>>(dc, views, panel);
    return cudaGetLastError();
}

}  // namespace lfdpr
