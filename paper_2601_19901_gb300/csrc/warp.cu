// Depth-guided warp of rendered views to other eyes on the display's eye
// line: the base the learned angular reconstruction refines.
//
// Every eye lies on the line y = 0, z = D, and every view looks through the
// same focal rectangle at z = 0, so a surface point keeps its pixel row in
// every view and only moves along it. A point that view a sees at pixel
// centre x + 1/2 with ray parameter t (the depth key's high word; its depth
// is D (1 - t), the same t from every eye) is seen from eye E at
//     x + 1/2 + (1 - 1/t) (W / fw) (E - E_a)
// (the disparity of project_point: B = (1 - D / (D - z)) W / fw). For an
// output eye E between input eyes E_0 <= E <= E_1 (weight s = (E - E_0) /
// (E_1 - E_0) towards the second):
//  1. Forward: each input pixel of the row holding a depth key moves to E
//     and is kept at pixel floor(x'), the nearest point winning (smallest t,
//     then the first input, then the leftmost source pixel).
//  2. Backward: a pixel with a winner finds the point's position in each of
//     the two inputs and interpolates that input's row linearly there. An
//     input agrees if its own key at the pixel holding that position has a
//     t within 1 % of the winner's. The agreeing inputs are blended with
//     weights (1 - s, s), renormalised (times the reciprocal of their sum);
//     with none agreeing, the winner's own
//     source pixel is taken. A pixel with no winner (disoccluded, or beyond
//     every input's reach) takes the unshifted blend (1 - s) c_0 + s c_1.
// Colours are rounded half to even to 8 bits; alpha is 255. All arithmetic is
// binary32, one rounding per written operation (no contraction), so a plain
// CPU restatement gives the same bytes.
#include <cmath>

#include "lfdpr_recon.h"
#include "objects.h"

namespace lfdpr {
namespace {

constexpr int kWarpThreads = 256;
constexpr uint64_t kNoKey = ~0ull;

struct WarpArgs {
    const uint8_t* views;     // [nin][H][W][4] RGBA8
    const uint64_t* keys;     // [nin][H][W] depth keys (t bits << 32 | point), all ones where empty
    const float* in_eyes;     // [nin] ascending
    const float* out_eyes;    // [nout]
    int nin, nout, W, H;
    float ipw;                // W / fw: view pixels per unit of x on the focal plane
    uint8_t* out;             // [nout][H][W][4] RGBA8
};

__device__ __forceinline__ bool key_depth(uint64_t key, float& t) {
    t = __uint_as_float(uint32_t(key >> 32));
    return key != kNoKey && t > 0.0f && isfinite(t);
}

__device__ __forceinline__ float channel(uint32_t rgba, int c) { return float((rgba >> (8 * c)) & 255u); }

// The input bracket of output eye E: j0 the last input eye at or before E
// (clamped to [0, nin - 2]), s the weight towards input j0 + 1.
__device__ __forceinline__ int bracket(const WarpArgs& a, float E, float& s) {
    int j0 = 0;
    for (int j = 0; j < a.nin; j++)
        if (a.in_eyes[j] <= E) j0 = j;
    j0 = min(j0, a.nin - 2);
    const float e0 = a.in_eyes[j0], e1 = a.in_eyes[j0 + 1];
    s = e1 > e0 ? (E - e0) / (e1 - e0) : 0.0f;
    s = fminf(fmaxf(s, 0.0f), 1.0f);
    return j0;
}

// Views an interval block takes at a time, for view width W.
__host__ __device__ __forceinline__ int views_per_pass(int W) {
    const int v = 32768 / (8 * W);
    return v < 1 ? 1 : (v > 4 ? 4 : v);
}

// (m, r) -> (m, r + step) over rows of length L, for step and r < L.
__device__ __forceinline__ void advance(int& m, int& r, int step, int L) {
    r += step;
    while (r >= L) {
        r -= L;
        m++;
    }
}

// Block (row y, input interval j): every output view whose bracket is
// (j, j + 1), up to views_per_pass(W) of them at a time. The two input rows
// are staged once in shared memory with each pixel's t, disparity factor
// g = (1 - 1/t) W / fw (both NaN where it has no key) and colour as binary32.
// The nearest point per output pixel is the 64-bit minimum of (t bits,
// input, source pixel).
__global__ void __launch_bounds__(kWarpThreads) k_warp_views(WarpArgs a) {
    extern __shared__ __align__(16) uint8_t s_raw[];
    const int y = blockIdx.x, j = blockIdx.y, W = a.W, V = views_per_pass(W);
    if (y >= a.H || j > a.nin - 2) return;
    float4* s_rgb = reinterpret_cast<float4*>(s_raw);                       // [2][W] colour
    float* s_t = reinterpret_cast<float*>(s_rgb + 2 * W);                   // [2][W]
    float* s_g = s_t + 2 * W;                                               // [2][W]
    unsigned long long* s_win = reinterpret_cast<unsigned long long*>(s_g + 2 * W);   // [V][W] nearest point
    __shared__ int s_views[kMaxRenderViews];
    __shared__ float s_w[kMaxRenderViews], s_E[kMaxRenderViews];
    __shared__ int s_n;
    if (threadIdx.x == 0) s_n = 0;
    const size_t npix = size_t(W) * a.H, row = size_t(y) * W;
    for (int q = threadIdx.x; q < 2 * W; q += blockDim.x) {
        const int src = q >= W, i = q - src * W;
        const size_t o = size_t(j + src) * npix + row + i;
        float t;
        const bool ok = key_depth(a.keys[o], t);
        s_t[q] = ok ? t : __int_as_float(0x7fc00000);   // NaN: no key
        s_g[q] = ok ? (1.0f - 1.0f / t) * a.ipw : __int_as_float(0x7fc00000);
        const uint32_t c = reinterpret_cast<const uint32_t*>(a.views)[o];
        s_rgb[q] = make_float4(channel(c, 0), channel(c, 1), channel(c, 2), 0.0f);
    }
    __syncthreads();
    // the output views of this interval with their weights
    for (int k = threadIdx.x; k < a.nout; k += blockDim.x) {
        float s;
        const float E = a.out_eyes[k];
        if (bracket(a, E, s) == j) {
            const int m = atomicAdd(&s_n, 1);
            s_views[m] = k;
            s_w[m] = s;
            s_E[m] = E;
        }
    }
    __syncthreads();
    const int n_views = s_n;
    const float eye[2] = {a.in_eyes[j], a.in_eyes[j + 1]};
    const int step = blockDim.x;
    for (int m0 = 0; m0 < n_views; m0 += V) {
        const int nv = min(V, n_views - m0);
        for (int q = threadIdx.x; q < nv * W; q += step) s_win[q] = kNoKey;
        __syncthreads();
        // 1. forward: the nearest point landing on each pixel (t, then input,
        // then source pixel); candidates (view m, input pixel r) in one sweep
        {
            int m = 0, r = threadIdx.x;
            advance(m, r, 0, 2 * W);
            for (; m < nv; advance(m, r, step, 2 * W)) {
                const float g = s_g[r];
                if (isnan(g)) continue;
                const int src = r >= W, i = r - src * W;
                const float X = (float(i) + 0.5f) + g * (s_E[m0 + m] - eye[src]);
                if (!isfinite(X)) continue;
                const float px = floorf(X);
                if (px < 0.0f || px >= float(W)) continue;
                atomicMin(&s_win[m * W + int(px)],
                          (uint64_t(__float_as_uint(s_t[r])) << 32) | (uint64_t(src) << 16) | uint64_t(i));
            }
        }
        __syncthreads();
        // 2. backward: output pixels (view m, pixel p) in one sweep
        int m = 0, p = threadIdx.x;
        advance(m, p, 0, W);
        for (; m < nv; advance(m, p, step, W)) {
            const int k = s_views[m0 + m];
            const float E = s_E[m0 + m], s = s_w[m0 + m];
            const uint64_t w = s_win[m * W + p];
            float v[3];
            if (w == kNoKey) {
                const float4 c0 = s_rgb[p], c1 = s_rgb[W + p];
                v[0] = (1.0f - s) * c0.x + s * c1.x;
                v[1] = (1.0f - s) * c0.y + s * c1.y;
                v[2] = (1.0f - s) * c0.z + s * c1.z;
            } else {
                const int ws_ = int((w >> 16) & 1u), wi = int(w & 0xffffu);
                const float t = s_t[ws_ * W + wi], g = s_g[ws_ * W + wi];
                float4 vs[2];
                float wt[2];
#pragma unroll
                for (int src = 0; src < 2; src++) {
                    const float X = (float(p) + 0.5f) + g * (eye[src] - E);
                    const float xa = X - 0.5f;
                    const float fl = floorf(xa), fr = xa - fl;
                    const float fn = floorf(X);
                    // indices clamped to the row (X is finite: the winner came from this row)
                    const int i0 = int(fminf(fmaxf(fl, 0.0f), float(W - 1)));
                    const int i1 = int(fminf(fmaxf(fl + 1.0f, 0.0f), float(W - 1)));
                    const int n = int(fminf(fmaxf(fn, 0.0f), float(W - 1)));
                    const float4 ca = s_rgb[src * W + i0], cb = s_rgb[src * W + i1];
                    vs[src] = make_float4(ca.x + fr * (cb.x - ca.x), ca.y + fr * (cb.y - ca.y),
                                          ca.z + fr * (cb.z - ca.z), 0.0f);
                    const float tn = s_t[src * W + n];
                    const bool agree = !isnan(tn) && fabsf(tn - t) <= 0.01f * t;
                    wt[src] = agree ? (src == 0 ? 1.0f - s : s) : 0.0f;
                }
                const float ws = wt[0] + wt[1];
                if (ws > 0.0f) {
                    const float rw = 1.0f / ws;
                    v[0] = (wt[0] * vs[0].x + wt[1] * vs[1].x) * rw;
                    v[1] = (wt[0] * vs[0].y + wt[1] * vs[1].y) * rw;
                    v[2] = (wt[0] * vs[0].z + wt[1] * vs[1].z) * rw;
                } else {
                    const float4 cs = s_rgb[ws_ * W + wi];
                    v[0] = cs.x;
                    v[1] = cs.y;
                    v[2] = cs.z;
                }
            }
            uint32_t o = 0xff000000u;
#pragma unroll
            for (int c = 0; c < 3; c++) o |= uint32_t(rintf(fminf(fmaxf(v[c], 0.0f), 255.0f))) << (8 * c);
            reinterpret_cast<uint32_t*>(a.out)[size_t(k) * npix + row + p] = o;
        }
        __syncthreads();   // this pass's views are done with the minima
    }
}

}  // namespace

cudaError_t launch_warp_views(const uint8_t* views, const uint64_t* keys, const float* in_eyes, int nin,
                              const float* out_eyes, int nout, int W, int H, float ipw, uint8_t* out,
                              cudaStream_t s) {
    if (nin < 2 || nout < 1 || W < 1 || H < 1 || W > kMaxWarpWidth || H > 65535 || nout > kMaxRenderViews || !(ipw > 0.0f))
        return cudaErrorInvalidValue;
    // shared memory: the two input rows (colour, t, g) and the pass's minima:
    // (48 + 8 V) bytes a pixel, at most 224 KB
    const size_t smem = (48u + 8u * size_t(views_per_pass(W))) * size_t(W);
    if (smem > 48u * 1024u) {
        const cudaError_t e = cudaFuncSetAttribute(k_warp_views, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
    }
    WarpArgs a{views, keys, in_eyes, out_eyes, nin, nout, W, H, ipw, out};
    k_warp_views<<<dim3(unsigned(H), unsigned(nin - 1)), kWarpThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lfdpr

extern "C" lfdpr_status lfdpr_warp_views(const uint8_t* in_views, const uint64_t* in_keys, const float* in_eyes,
                                         int32_t in_count, const float* out_eyes, int32_t out_count, int32_t view_w,
                                         int32_t view_h, float pixels_per_unit, uint8_t* out_views, void* stream) {
    lfdpr::g_last_error[0] = 0;
    if (!in_views || !in_keys || !in_eyes || !out_eyes || !out_views)
        return lfdpr::fail(LFDPR_EINVAL, "warp_views: null argument");
    if (in_count < 2 || in_count > lfdpr::kMaxRenderViews || out_count < 1 || out_count > lfdpr::kMaxRenderViews)
        return lfdpr::fail(LFDPR_EINVAL, "warp_views: need 2..%d input and 1..%d output views", lfdpr::kMaxRenderViews,
                           lfdpr::kMaxRenderViews);
    if (view_w < 1 || view_h < 1 || view_w > lfdpr::kMaxWarpWidth || view_h > 16384)
        return lfdpr::fail(LFDPR_EINVAL, "warp_views: views must be 1..%d pixels wide, 1..16384 high",
                           lfdpr::kMaxWarpWidth);
    if (!(pixels_per_unit > 0.0f) || !std::isfinite(pixels_per_unit))
        return lfdpr::fail(LFDPR_EINVAL, "warp_views: pixels_per_unit must be positive and finite");
    if ((reinterpret_cast<uintptr_t>(in_views) & 3u) || (reinterpret_cast<uintptr_t>(out_views) & 3u) ||
        (reinterpret_cast<uintptr_t>(in_keys) & 7u) || (reinterpret_cast<uintptr_t>(in_eyes) & 3u) ||
        (reinterpret_cast<uintptr_t>(out_eyes) & 3u))
        return lfdpr::fail(LFDPR_EINVAL, "warp_views: views and eyes must be 4-byte aligned, keys 8-byte aligned");
    const cudaError_t e = lfdpr::launch_warp_views(in_views, in_keys, in_eyes, in_count, out_eyes, out_count, view_w,
                                                   view_h, pixels_per_unit, out_views, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return lfdpr::cuda_fail(e, "launch k_warp_views");
    return LFDPR_OK;
}
