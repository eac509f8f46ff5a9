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
//     weights (1 - s, s), renormalised; with none agreeing, the winner's own
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

constexpr int kWarpThreads = 128;
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

// Block (row y, output view k).
__global__ void __launch_bounds__(kWarpThreads) k_warp_views(WarpArgs a) {
    extern __shared__ unsigned long long s_win[];   // [W] forward-splat winners
    const int y = blockIdx.x, k = blockIdx.y, W = a.W;
    if (y >= a.H || k >= a.nout) return;
    const float E = a.out_eyes[k];
    int j0 = 0;
    for (int j = 0; j < a.nin; j++)
        if (a.in_eyes[j] <= E) j0 = j;
    j0 = min(j0, a.nin - 2);
    const float e0 = a.in_eyes[j0], e1 = a.in_eyes[j0 + 1];
    float s = e1 > e0 ? (E - e0) / (e1 - e0) : 0.0f;
    s = fminf(fmaxf(s, 0.0f), 1.0f);
    const size_t npix = size_t(W) * a.H, row = size_t(y) * W;
    const uint64_t* key[2] = {a.keys + size_t(j0) * npix + row, a.keys + size_t(j0 + 1) * npix + row};
    const uint32_t* col[2] = {reinterpret_cast<const uint32_t*>(a.views) + size_t(j0) * npix + row,
                              reinterpret_cast<const uint32_t*>(a.views) + size_t(j0 + 1) * npix + row};
    const float eye[2] = {e0, e1};

    for (int i = threadIdx.x; i < W; i += blockDim.x) s_win[i] = kNoKey;
    __syncthreads();
    // 1. forward
#pragma unroll
    for (int src = 0; src < 2; src++) {
        const float dE = E - eye[src];
        for (int i = threadIdx.x; i < W; i += blockDim.x) {
            const uint64_t kk = key[src][i];
            float t;
            if (!key_depth(kk, t)) continue;
            const float f = 1.0f - 1.0f / t;
            const float X = (float(i) + 0.5f) + (f * a.ipw) * dE;
            if (!isfinite(X)) continue;
            const float px = floorf(X);
            if (px < 0.0f || px >= float(W)) continue;
            atomicMin(&s_win[int(px)], (kk & 0xffffffff00000000ull) | (uint64_t(src) << 16) | uint64_t(i));
        }
    }
    __syncthreads();
    // 2. backward
    uint32_t* out = reinterpret_cast<uint32_t*>(a.out) + size_t(k) * npix + row;
    for (int p = threadIdx.x; p < W; p += blockDim.x) {
        const uint64_t w = s_win[p];
        float v[3];
        if (w == kNoKey) {
            const uint32_t c0 = col[0][p], c1 = col[1][p];
#pragma unroll
            for (int c = 0; c < 3; c++) v[c] = (1.0f - s) * channel(c0, c) + s * channel(c1, c);
        } else {
            const float t = __uint_as_float(uint32_t(w >> 32));
            const float f = 1.0f - 1.0f / t;
            float vs[2][3], wt[2];
#pragma unroll
            for (int src = 0; src < 2; src++) {
                const float X = (float(p) + 0.5f) + (f * a.ipw) * (eye[src] - E);
                const float xa = X - 0.5f;
                const float fl = floorf(xa), fr = xa - fl;
                const float fn = floorf(X);
                // indices clamped to the row (X is finite: the winner came from this row)
                const int i0 = int(fminf(fmaxf(fl, 0.0f), float(W - 1)));
                const int i1 = int(fminf(fmaxf(fl + 1.0f, 0.0f), float(W - 1)));
                const int n = int(fminf(fmaxf(fn, 0.0f), float(W - 1)));
                const uint32_t ca = col[src][i0], cb = col[src][i1];
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const float va = channel(ca, c), vb = channel(cb, c);
                    vs[src][c] = va + fr * (vb - va);
                }
                float tn;
                const bool agree = key_depth(key[src][n], tn) && fabsf(tn - t) <= 0.01f * t;
                wt[src] = agree ? (src == 0 ? 1.0f - s : s) : 0.0f;
            }
            const float ws = wt[0] + wt[1];
            if (ws > 0.0f) {
#pragma unroll
                for (int c = 0; c < 3; c++) v[c] = (wt[0] * vs[0][c] + wt[1] * vs[1][c]) / ws;
            } else {
                const int src = int((w >> 16) & 1u), i = int(w & 0xffffu);
                const uint32_t cs = col[src][i];
#pragma unroll
                for (int c = 0; c < 3; c++) v[c] = channel(cs, c);
            }
        }
        uint32_t o = 0xff000000u;
#pragma unroll
        for (int c = 0; c < 3; c++) o |= uint32_t(rintf(fminf(fmaxf(v[c], 0.0f), 255.0f))) << (8 * c);
        out[p] = o;
    }
}

}  // namespace

cudaError_t launch_warp_views(const uint8_t* views, const uint64_t* keys, const float* in_eyes, int nin,
                              const float* out_eyes, int nout, int W, int H, float ipw, uint8_t* out,
                              cudaStream_t s) {
    if (nin < 2 || nout < 1 || W < 1 || H < 1 || W > kMaxWarpWidth || H > 65535 || nout > 65535 || !(ipw > 0.0f))
        return cudaErrorInvalidValue;
    // the winners' row: at most 32 KB of shared memory
    WarpArgs a{views, keys, in_eyes, out_eyes, nin, nout, W, H, ipw, out};
    k_warp_views<<<dim3(unsigned(H), unsigned(nout)), kWarpThreads, sizeof(unsigned long long) * size_t(W), s>>>(a);
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
    const cudaError_t e = lfdpr::launch_warp_views(in_views, in_keys, in_eyes, in_count, out_eyes, out_count, view_w,
                                                   view_h, pixels_per_unit, out_views, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return lfdpr::cuda_fail(e, "launch k_warp_views");
    return LFDPR_OK;
}
