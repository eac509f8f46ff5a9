// Elemental image array construction (Sec. 4): optional angular tent
// reconstruction of the 2N supersampled views, optional +-1 crosstalk mixing,
// then the slanted-lens subpixel interleave.
//
// Every panel pixel samples one view pixel (nearest, pixel centres) of the
// views its three subpixels select, and neighbouring subpixels select
// different views, so reading views straight from global memory is a gather
// touching a new sector per byte. k_interleave_tile instead takes one view
// row and a strip of 1024 panel columns: it stages the strip's source
// segment of that row for every rendered view in shared memory with
// coalesced loads, then forms every panel row that samples that view row,
// one thread per 4 adjacent panel pixels and one 16-byte store per row.
// k_interleave (the direct gather) serves displays whose tile would not fit.
// k_interleave_gauss is the Gaussian reconstruction of Sec. 4 (recon 2, 3):
// per subpixel the mean of the caller's samples, each the nearest rendered
// view to the subpixel's phase plus the sample's angular offset at the view
// pixel holding its spatially offset position. It is bound by its nearest-view
// searches (72 per pixel with crosstalk), not by the gathers (L1 / L2 hits):
// staging bands of views in shared memory measured slower.
#include "lfdpr_internal.cuh"

namespace lfdpr {
namespace {

// View pixel channel as stored: global views [view][H][W][RGBA8].
struct GlobalTexels {
    const uint8_t* __restrict__ views;
    uint64_t npix, pix;
    __device__ __forceinline__ uint32_t byte(int view, int ch) const {
        return __ldg(views + ((uint64_t)view * npix + pix) * 4u + ch);
    }
    __device__ __forceinline__ float operator()(int view, int ch) const { return float(byte(view, ch)); }
};

// The same from a staged row segment: s[view * stride + i], RGBA8 words.
struct SharedTexels {
    const uint32_t* s;
    int stride, i;
    __device__ __forceinline__ uint32_t byte(int view, int ch) const {
        return (s[view * stride + i] >> (8 * ch)) & 255u;
    }
    __device__ __forceinline__ float operator()(int view, int ch) const { return float(byte(view, ch)); }
};

// Display view k, channel ch, as binary32 before rounding.
template <class T>
__device__ __forceinline__ float display_value(const DispConst& c, const T& tex, int k, int ch) {
    if (c.recon != 1) return tex(k, ch);
    float acc = 0.0f, ws = 0.0f;
#pragma unroll
    for (int q = 0; q < 3; q++) {
        const int m = 2 * k - 1 + q;
        if (m < 0 || m >= c.nr) continue;
        const float w = q == 1 ? 0.5f : 0.25f;
        acc = fmaf(w, tex(m, ch), acc);
        ws += w;
    }
    return __fdiv_rn(acc, ws);
}

// Lens phase of subpixel (x, y, ch) on the display-view axis, [0, N).
__device__ __forceinline__ float subpixel_phase(const DispConst& c, int x, int y, int ch) {
    const float third = ch == 0 ? (float)(1.0 / 6.0) : (ch == 1 ? 0.5f : (float)(5.0 / 6.0));
    const float cx = float(x) + third;
    const float a = fmaf(c.slant, float(y), cx);
    const float ph = fmaf(a, c.inv_pitch, c.phase_offset);
    const float fr = ph - floorf(ph);
    return fr * float(c.n_views);
}

__device__ __forceinline__ int view_of_subpixel(const DispConst& c, int x, int y, int ch) {
    int k = int(subpixel_phase(c, x, y, ch));
    k = k >= c.n_views ? c.n_views - 1 : (k < 0 ? 0 : k);
    return k;
}

// Panel pixel (x, y) as RGBA8 (alpha 255) from its view pixel's texels.
template <class T>
__device__ __forceinline__ uint32_t panel_pixel(const DispConst& c, const T& tex, int x, int y) {
    uint32_t o = 0xff000000u;
    if (c.recon != 1 && !(c.xtalk > 0.0f)) {
        // each subpixel shows its view's byte as it is (a byte converted to
        // binary32 and rounded back is the byte)
#pragma unroll
        for (int ch = 0; ch < 3; ch++) o |= tex.byte(view_of_subpixel(c, x, y, ch), ch) << (8 * ch);
        return o;
    }
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        const int k = view_of_subpixel(c, x, y, ch);
        float val;
        if (c.xtalk > 0.0f) {
            const int km = k == 0 ? c.n_views - 1 : k - 1;
            const int kp = k == c.n_views - 1 ? 0 : k + 1;
            float acc = display_value(c, tex, k, ch) * c.xtalk_c;
            acc = fmaf(c.xtalk, display_value(c, tex, km, ch), acc);
            acc = fmaf(c.xtalk, display_value(c, tex, kp, ch), acc);
            val = acc;
        } else {
            val = display_value(c, tex, k, ch);
        }
        o |= uint32_t(round_u8(val)) << (8 * ch);
    }
    return o;
}

// Nearest view pixel of panel column x (row y): pixel centres aligned. In
// 32 bits: (2 x + 1) W < 2^31 for panels up to 32768 and views up to 16384.
__device__ __forceinline__ int source_x(const DispConst& c, int x) {
    return int((2u * uint32_t(x) + 1u) * uint32_t(c.W) / (2u * uint32_t(c.Wp)));
}
__device__ __forceinline__ int source_y(const DispConst& c, int y) {
    return int((2u * uint32_t(y) + 1u) * uint32_t(c.H) / (2u * uint32_t(c.Hp)));
}

__device__ __forceinline__ void store4(const DispConst& c, uint8_t* __restrict__ panel, int xg, int y,
                                       const uint32_t* px) {
    if (!LFDPR_IN_BOUNDS(uint32_t(y), uint32_t(c.Hp), 21) || !LFDPR_IN_BOUNDS(uint32_t(xg), uint32_t(c.Wp), 21)) return;
    uint8_t* dst = panel + ((uint64_t)y * c.Wp + xg) * 4u;
    if (xg + 4 <= c.Wp && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0)) {
        *reinterpret_cast<uint4*>(dst) = make_uint4(px[0], px[1], px[2], px[3]);
    } else {
        for (int e = 0; e < 4 && xg + e < c.Wp; e++) reinterpret_cast<uint32_t*>(dst)[e] = px[e];
    }
}

constexpr int kTileThreads = 256;
constexpr int kTileCols = 4 * kTileThreads;   // panel columns per tile

// Block (strip bx, view row sy): view pixels sx_lo..sx_lo + n - 1 of row sy
// for every rendered view, then the panel rows whose source row is sy.
__global__ void __launch_bounds__(kTileThreads) k_interleave_tile(DispConst c, const uint8_t* __restrict__ views,
                                                                  uint8_t* __restrict__ panel, int stride) {
    wait_previous_kernel();
    allow_next_kernel();
    extern __shared__ uint32_t s_row[];
    const int sy = blockIdx.y;
    const int x0 = blockIdx.x * kTileCols;
    const int x1 = min(x0 + kTileCols, c.Wp);   // exclusive
    // panel rows sampling view row sy: y_first.. while source_y(y) == sy
    int y = max(0, int(uint32_t(sy) * uint32_t(c.Hp) / uint32_t(c.H)) - 1);
    while (y < c.Hp && source_y(c, y) < sy) y++;
    if (y >= c.Hp || source_y(c, y) != sy) return;
    const int sx_lo = source_x(c, x0), n = source_x(c, x1 - 1) - sx_lo + 1;
    const uint64_t npix = (uint64_t)c.W * c.H;
    const uint32_t* v32 = reinterpret_cast<const uint32_t*>(views);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int m = warp; m < c.nr; m += kTileThreads / 32) {
        const uint32_t* src = v32 + (uint64_t)m * npix + (uint64_t)sy * c.W + sx_lo;
        for (int i = lane; i < n; i += 32)
            if (LFDPR_IN_BOUNDS(uint32_t(sx_lo + i), uint32_t(c.W), 20) && LFDPR_IN_BOUNDS(i, stride, 20))
                s_row[m * stride + i] = __ldg(src + i);
    }
    __syncthreads();
    const int xg = x0 + 4 * threadIdx.x;
    if (xg >= x1) return;
    int sxi[4];
#pragma unroll
    for (int e = 0; e < 4; e++) sxi[e] = min(source_x(c, min(xg + e, x1 - 1)) - sx_lo, n - 1);
    for (; y < c.Hp && source_y(c, y) == sy; y++) {
        uint32_t px[4];
#pragma unroll
        for (int e = 0; e < 4; e++) px[e] = panel_pixel(c, SharedTexels{s_row, stride, sxi[e]}, xg + e, y);
        store4(c, panel, xg, y, px);
    }
}

__global__ void __launch_bounds__(256) k_interleave(DispConst c, const uint8_t* __restrict__ views,
                                                     uint8_t* __restrict__ panel) {
    wait_previous_kernel();
    allow_next_kernel();
    const uint64_t npix = (uint64_t)c.W * c.H;
    const int groups_x = (c.Wp + 3) >> 2;
    const uint64_t total = (uint64_t)groups_x * c.Hp;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const int y = int(g / groups_x);
        const int xg = int(g - (uint64_t)y * groups_x) * 4;
        const int sy = source_y(c, y);
        uint32_t px[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const int x = min(xg + e, c.Wp - 1);
            uint64_t pix = (uint64_t)sy * c.W + source_x(c, x);
            if (!LFDPR_IN_BOUNDS(pix, npix, 22)) pix = 0;
            px[e] = panel_pixel(c, GlobalTexels{views, npix, pix}, x, y);
        }
        store4(c, panel, xg, y, px);
    }
}

// Rendered view nearest a on the display-view axis (positions pos[], ties to
// the later view), from the window of four views around it.
__device__ __forceinline__ int nearest_view(const float* pos, int nr, float r, float a) {
    int lo = int(floorf(r * a)) - 2;
    lo = lo > nr - 4 ? nr - 4 : lo;
    lo = lo < 0 ? 0 : lo;
    const int hi = lo + 3 < nr - 1 ? lo + 3 : nr - 1;
    int m = lo;
    float best = fabsf(pos[lo] - a);
#pragma unroll
    for (int q = 1; q < 4; q++) {
        if (lo + q > hi) break;
        const float dq = fabsf(pos[lo + q] - a);
        if (dq <= best) {
            best = dq;
            m = lo + q;
        }
    }
    return m;
}

// Panel pixel (x, y) under Gaussian reconstruction (+ crosstalk): for each
// channel the mean over the samples of the rendered view nearest phi + dphi
// at the view pixel holding (vx + dx, vy + dy), clamped; with crosstalk the
// same at phi - 1 and phi + 1 (wrapping) mixed in. The samples are the outer
// loop (each sample's pixel is found once); each of the nine sums still adds
// its samples in order.
__device__ __forceinline__ uint32_t gauss_pixel(const DispConst& c, const uint32_t* __restrict__ v32, const float* pos,
                                                const float* smp, int ns, int x, int y, float sxw, float syh) {
    const int nr = c.nr, W = c.W, H = c.H;
    const uint64_t npix = (uint64_t)W * H;
    const float r = float(nr / c.n_views), N = float(c.n_views);
    const float vx = (float(x) + 0.5f) * sxw, vy = (float(y) + 0.5f) * syh;
    const bool xt = c.xtalk > 0.0f;
    float phi[3][3];   // [channel][own, -1, +1]
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        const float p0 = subpixel_phase(c, x, y, ch);
        float pm = p0 - 1.0f, pp = p0 + 1.0f;
        if (pm < 0.0f) pm += N;
        if (pp >= N) pp -= N;
        phi[ch][0] = p0;
        phi[ch][1] = pm;
        phi[ch][2] = pp;
    }
    float acc[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    for (int s = 0; s < ns; s++) {
        int px = int(floorf(vx + smp[3 * s])), py = int(floorf(vy + smp[3 * s + 1]));
        px = px < 0 ? 0 : (px >= W ? W - 1 : px);
        py = py < 0 ? 0 : (py >= H ? H - 1 : py);
        const uint32_t* row = v32 + (uint64_t)py * W + px;
        const float dphi = smp[3 * s + 2];
#pragma unroll
        for (int ch = 0; ch < 3; ch++)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (k > 0 && !xt) continue;
                int m = nearest_view(pos, nr, r, phi[ch][k] + dphi);
                if (!LFDPR_IN_BOUNDS(uint32_t(m), uint32_t(nr), 23)) m = 0;
                acc[ch][k] += float((__ldg(row + (uint64_t)m * npix) >> (8 * ch)) & 255u);
            }
    }
    uint32_t o = 0xff000000u;
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        float v = acc[ch][0] / float(ns);
        if (xt) {
            float t = v * c.xtalk_c;
            t = fmaf(c.xtalk, acc[ch][1] / float(ns), t);
            t = fmaf(c.xtalk, acc[ch][2] / float(ns), t);
            v = t;
        }
        o |= uint32_t(round_u8(v)) << (8 * ch);
    }
    return o;
}

__global__ void __launch_bounds__(256) k_interleave_gauss(DispConst c, const uint8_t* __restrict__ views,
                                                          const float* __restrict__ pos,
                                                          const float* __restrict__ samples, int ns,
                                                          uint8_t* __restrict__ panel) {
    wait_previous_kernel();
    allow_next_kernel();
    __shared__ float s_pos[kMaxRenderViews];
    __shared__ float s_smp[3 * 32];
    for (int i = threadIdx.x; i < c.nr; i += blockDim.x) s_pos[i] = pos[i];
    for (int i = threadIdx.x; i < 3 * ns; i += blockDim.x) s_smp[i] = samples[i];
    __syncthreads();
    const uint64_t total = (uint64_t)c.Wp * c.Hp;
    const float sxw = float(c.W) / float(c.Wp), syh = float(c.H) / float(c.Hp);
    const uint32_t* v32 = reinterpret_cast<const uint32_t*>(views);
    for (uint64_t gi = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < total;
         gi += (uint64_t)gridDim.x * blockDim.x) {
        const int y = int(gi / c.Wp), x = int(gi - (uint64_t)y * c.Wp);
        reinterpret_cast<uint32_t*>(panel)[gi] = gauss_pixel(c, v32, s_pos, s_smp, ns, x, y, sxw, syh);
    }
}

}  // namespace

namespace {

// One 2 x 2 box of RGBA8 texels: (a + b + c + d + 2) >> 2 per channel.
__device__ __forceinline__ uint32_t box4(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    uint32_t o = 0u;
#pragma unroll
    for (int ch = 0; ch < 4; ch++) {
        const uint32_t s = ((a >> (8 * ch)) & 255u) + ((b >> (8 * ch)) & 255u) + ((c >> (8 * ch)) & 255u) +
                           ((d >> (8 * ch)) & 255u);
        o |= ((s + 2u) >> 2) << (8 * ch);
    }
    return o;
}

// Mip level L (1 or 2) of every rendered view (Sec. 5.1: with spatial
// supersampling a mipmap of each view is built): L times the 2 x 2 box of the
// level above, with the texture mips' rounding. One thread per level-L texel
// reads its 2^L x 2^L block of level-0 texels with vector loads (W and H are
// multiples of 2^L) and reduces it level by level.
template <int L>
__global__ void __launch_bounds__(256) k_view_mip(const uint8_t* __restrict__ src, uint32_t W, uint32_t H,
                                                  uint32_t nr, uint8_t* __restrict__ dst) {
    wait_previous_kernel();
    allow_next_kernel();
    constexpr int K = 1 << L;
    const uint32_t wl = W >> L, hl = H >> L;
    const uint64_t total = (uint64_t)wl * hl * nr;
    const uint32_t* s32 = reinterpret_cast<const uint32_t*>(src);
    uint32_t* d32 = reinterpret_cast<uint32_t*>(dst);
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x = uint32_t(t % wl);
        const uint64_t r = t / wl;
        const uint32_t y = uint32_t(r % hl), v = uint32_t(r / hl);
        if (!LFDPR_IN_BOUNDS((uint64_t)(y * K + K - 1) * W + x * K + K - 1, (uint64_t)W * H, 24)) continue;
        const uint32_t* base = s32 + (uint64_t)v * W * H + (uint64_t)(y * K) * W + x * K;
        uint32_t px[K][K];
#pragma unroll
        for (int dy = 0; dy < K; dy++) {
            if constexpr (K == 2) {
                const uint2 q = __ldg(reinterpret_cast<const uint2*>(base + (uint64_t)dy * W));
                px[dy][0] = q.x;
                px[dy][1] = q.y;
            } else {
                const uint4 q = __ldg(reinterpret_cast<const uint4*>(base + (uint64_t)dy * W));
                px[dy][0] = q.x;
                px[dy][1] = q.y;
                px[dy][2] = q.z;
                px[dy][3] = q.w;
            }
        }
        uint32_t out;
        if constexpr (K == 2) {
            out = box4(px[0][0], px[0][1], px[1][0], px[1][1]);
        } else {
            const uint32_t a = box4(px[0][0], px[0][1], px[1][0], px[1][1]);
            const uint32_t b = box4(px[0][2], px[0][3], px[1][2], px[1][3]);
            const uint32_t c = box4(px[2][0], px[2][1], px[3][0], px[3][1]);
            const uint32_t e = box4(px[2][2], px[2][3], px[3][2], px[3][3]);
            out = box4(a, b, c, e);
        }
        d32[(uint64_t)v * wl * hl + (uint64_t)y * wl + x] = out;
    }
}

}  // namespace

LFDPR_CHECK_READER(checks_interleave)

cudaError_t launch_view_mip(const uint8_t* views, int W, int H, int nr, int level, uint8_t* out, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (level == 1)
        return launch_after_previous(k_view_mip<1>, dim3(sms * 8), dim3(256), 0, s, views, uint32_t(W), uint32_t(H),
                                     uint32_t(nr), out);
    if (level == 2)
        return launch_after_previous(k_view_mip<2>, dim3(sms * 8), dim3(256), 0, s, views, uint32_t(W), uint32_t(H),
                                     uint32_t(nr), out);
    return cudaErrorInvalidValue;
}

cudaError_t launch_interleave(const DispConst& dc, const uint8_t* views, const float* pos, const float* samples,
                              int n_samples, uint8_t* panel, cudaStream_t s) {
    int dev = 0, sms = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (dc.recon == 2 || dc.recon == 3) {
        if (n_samples < 1 || n_samples > 32) return cudaErrorInvalidValue;
        return launch_after_previous(k_interleave_gauss, dim3(sms * 16), dim3(256), 0, s, dc, views, pos, samples,
                                     n_samples, panel);
    }
    // widest source segment of a tile: (kTileCols - 1) W / Wp + 2 pixels
    const int64_t seg = ((int64_t)(kTileCols - 1) * dc.W) / dc.Wp + 2;
    const int64_t bytes = (int64_t)dc.nr * seg * 4;
    if (bytes <= smem_max / 2) {
        cudaError_t e = cudaFuncSetAttribute(k_interleave_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(bytes));
        if (e != cudaSuccess) return e;
        const dim3 grid((dc.Wp + kTileCols - 1) / kTileCols, dc.H);
        return launch_after_previous(k_interleave_tile, grid, dim3(kTileThreads), size_t(bytes), s, dc, views, panel,
                                     int(seg));
    }
    return launch_after_previous(k_interleave, dim3(sms * 8), dim3(256), 0, s, dc, views, panel);
}

}  // namespace lfdpr
