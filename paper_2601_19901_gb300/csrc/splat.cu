// EPR splatting into every view (Sec. 3.2) with the 64-bit depth|id test
// (Sec. 5.1), and the per-view resolve of Eq. 8-9 (Sec. 3.3).
//
//   k_splat    one thread per (point, view) pair, the view index fastest, so a
//              warp holds one point in 32 neighbouring views: the same triangle
//              record, splats of nearly the same size (little divergence), and
//              atomics to 32 different view buffers. The point's cell is
//              projected into the view for a pixel box; every pixel centre in
//              the box whose ray meets the triangle's plane inside the cell and
//              inside the triangle, at a depth in [near, far], does
//              atomicMin(key, float_bits(t) << 32 | point id).
//   k_resolve  one thread per view pixel: the winning point's cell corners are
//              projected for the splat's pixel area (shoelace), Eq. 8 gives the
//              view's texture area, Eq. 9 interpolates tv_min..tv_max.
#include "lfdpr_internal.cuh"

namespace lfdpr {
namespace {

constexpr float kBoxPad = 1.0f / 16.0f;   // pixel-box margin against rounding (pixels)

__device__ __forceinline__ void cell_corner(const float4& q0, const float4& q1, const float4& q2,
                                            const float4& q3, int ia, int jb, float* o) {
    const float cu = float(ia) * q0.w + q2.w;
    const float cv = float(jb) * q1.w + q3.w;
    o[0] = fmaf(cu, q1.x, fmaf(cv, q2.x, q0.x));
    o[1] = fmaf(cu, q1.y, fmaf(cv, q2.y, q0.y));
    o[2] = fmaf(cu, q1.z, fmaf(cv, q2.z, q0.z));
}

__global__ void __launch_bounds__(256) k_splat(FrameArgs a) {
    if (a.ctr->overflow) return;
    const DispConst& c = a.dc;
    const uint64_t n_pairs = (uint64_t)a.ctr->n_points * (uint64_t)c.nr;
    const uint64_t npix = (uint64_t)c.W * c.H;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_pairs;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t p = uint32_t(q / (uint32_t)c.nr);
        const int v = int(q - (uint64_t)p * (uint32_t)c.nr);
        const uint2 pt = *reinterpret_cast<const uint2*>(a.points + p);
        const TriRec* r = a.rec + pt.x;
        const float4 q0 = __ldg(&r->q[0]), q1 = __ldg(&r->q[1]), q2 = __ldg(&r->q[2]);
        const float4 q3 = __ldg(&r->q[3]), q4 = __ldg(&r->q[4]);
        const int i = int(pt.y & 0xffffu), j = int(pt.y >> 16);
        const float Ex = __ldg(a.ex + v);

        // conservative pixel box of the projected cell
        int bx0 = 0, bx1 = c.W - 1, by0 = 0, by1 = c.H - 1;
        {
            float mnx = INFINITY, mxx = -INFINITY, mny = INFINITY, mxy = -INFINITY;
            bool behind = false;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                float C[3];
                cell_corner(q0, q1, q2, q3, i + (k == 1 || k == 2), j + (k >= 2), C);
                const float dep = c.D - C[2];
                if (!(dep > 1e-6f)) { behind = true; break; }
                const float s = __fdiv_rn(c.D, dep);
                const float qx = (fmaf(C[0] - Ex, s, Ex) - c.x0) * c.ipw;
                const float qy = (c.y0 - C[1] * s) * c.iph;
                mnx = fminf(mnx, qx); mxx = fmaxf(mxx, qx);
                mny = fminf(mny, qy); mxy = fmaxf(mxy, qy);
            }
            if (!behind) {
                const float fx0 = ceilf(mnx - 0.5f - kBoxPad), fx1 = floorf(mxx - 0.5f + kBoxPad);
                const float fy0 = ceilf(mny - 0.5f - kBoxPad), fy1 = floorf(mxy - 0.5f + kBoxPad);
                if (fx1 < 0.0f || fy1 < 0.0f || fx0 > float(c.W - 1) || fy0 > float(c.H - 1)) continue;
                bx0 = fx0 < 0.0f ? 0 : int(fx0);
                bx1 = fx1 > float(c.W - 1) ? c.W - 1 : int(fx1);
                by0 = fy0 < 0.0f ? 0 : int(fy0);
                by1 = fy1 > float(c.H - 1) ? c.H - 1 : int(fy1);
            }
        }

        const float qEx = Ex - q0.x, qEy = 0.0f - q0.y, qEz = c.D - q0.z;
        const float num = -dot3(q3.x, q3.y, q3.z, qEx, qEy, qEz);
        const float ulo = float(i) * q0.w, uhi = float(i + 1) * q0.w;
        const float vlo = float(j) * q1.w, vhi = float(j + 1) * q1.w;
        unsigned long long* kv = reinterpret_cast<unsigned long long*>(a.keys) + (uint64_t)v * npix;
        for (int y = by0; y <= by1; y++) {
            const float Fy = fmaf(float(y) + 0.5f, -c.ph, c.y0);
            for (int x = bx0; x <= bx1; x++) {
                const float Fx = fmaf(float(x) + 0.5f, c.pw, c.x0);
                const float dx = Fx - Ex, dy = Fy - 0.0f, dz = -c.D;
                const float den = dot3(q3.x, q3.y, q3.z, dx, dy, dz);
                if (den == 0.0f) continue;
                const float t = __fdiv_rn(num, den);
                const float depth = t * c.D;
                if (!(depth >= c.near_z && depth <= c.far_z)) continue;
                const float hx = fmaf(t, dx, qEx), hy = fmaf(t, dy, qEy), hz = fmaf(t, dz, qEz);
                const float uq = dot3(hx, hy, hz, q1.x, q1.y, q1.z);
                const float vq = dot3(hx, hy, hz, q2.x, q2.y, q2.z);
                const float u = uq - q2.w, vv = vq - q3.w;
                if (!(u >= ulo && u < uhi && vv >= vlo && vv < vhi)) continue;
                const float w0 = edge_fn(q4.x, q4.y, q4.z, q4.w, uq, vq);
                const float w1 = edge_fn(q4.z, q4.w, 0.0f, 0.0f, uq, vq);
                const float w2 = edge_fn(0.0f, 0.0f, q4.x, q4.y, uq, vq);
                if (!inside_either(w0, w1, w2)) continue;
                const unsigned long long key =
                    ((unsigned long long)__float_as_uint(t) << 32) | (unsigned long long)p;
                atomicMin(kv + (uint64_t)y * c.W + x, key);
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_resolve(FrameArgs a) {
    const DispConst& c = a.dc;
    const uint64_t npix = (uint64_t)c.W * c.H;
    const uint64_t total = npix * (uint64_t)c.nr;
    for (uint64_t o = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total;
         o += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = a.keys[o];
        uint32_t out = 0u;
        if (key != ~0ull) {
            const int v = int(o / npix);
            const float Ex = __ldg(a.ex + v);
            const uint4 pt = a.points[uint32_t(key)];
            const TriRec* r = a.rec + pt.x;
            const float4 q0 = __ldg(&r->q[0]), q1 = __ldg(&r->q[1]), q2 = __ldg(&r->q[2]);
            const float4 q3 = __ldg(&r->q[3]), q5 = __ldg(&r->q[5]);
            const int i = int(pt.y & 0xffffu), j = int(pt.y >> 16);
            float X[4], Y[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                float C[3];
                cell_corner(q0, q1, q2, q3, i + (k == 1 || k == 2), j + (k >= 2), C);
                const float s = __fdiv_rn(c.D, c.D - C[2]);
                const float sx = fmaf(C[0] - Ex, s, Ex);
                const float sy = C[1] * s;
                X[k] = (sx - c.x0) * c.ipw;
                Y[k] = (c.y0 - sy) * c.iph;
            }
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int k1 = (k + 1) & 3;
                acc = acc + fmaf(X[k], Y[k1], -(X[k1] * Y[k]));
            }
            const float area_px = 0.5f * fabsf(acc);
            const float vmin = q5.y, vmax = q5.z;
            const float size_vse = __fdiv_rn(q5.x, fminf(1.0f, area_px));
            const float size_vs = fminf(fmaxf(size_vse, vmin), vmax);
            const float w = vmax > vmin ? __fdiv_rn(size_vs - vmin, vmax - vmin) : 0.0f;
#pragma unroll
            for (int ch = 0; ch < 4; ch++) {
                const float lo = float((pt.z >> (8 * ch)) & 255u), hi = float((pt.w >> (8 * ch)) & 255u);
                out |= uint32_t(round_u8(fmaf(w, hi - lo, lo))) << (8 * ch);
            }
        }
        reinterpret_cast<uint32_t*>(a.views)[o] = out;
    }
}

}  // namespace

cudaError_t launch_splat(const FrameArgs& a, cudaStream_t s) {
    k_splat<<<a.sm_count * 8, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_resolve(const FrameArgs& a, cudaStream_t s) {
    k_resolve<<<a.sm_count * 8, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lfdpr
