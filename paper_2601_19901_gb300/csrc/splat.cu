// EPR splatting into every view (Sec. 3.2) with the 64-bit depth|id test
// (Sec. 5.1), and the per-view resolve of Eq. 8-9 (Sec. 3.3).
//
//   k_splat    one warp per point, lanes over the views: every pixel centre
//              inside the point's projected cell and its projected triangle,
//              at a depth in [near, far], does
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

// Plane-space form of the per-pixel test (the oracle's formula): the pixel
// centre's ray meets the triangle's plane at t; accept iff the hit lies in
// the half-open cell and in the closed triangle and t D is in [near, far].
// Used for the rare points whose cell or triangle reaches the eyes' plane,
// where the screen-space form below does not apply; the box is the whole view.
__device__ __noinline__ uint32_t splat_exact(const FrameArgs& a, uint32_t p, int i, int j, int v,
                                             const float4& q0, const float4& q1, const float4& q2,
                                             const float4& q3, const float4& q4) {
    const DispConst& c = a.dc;
    const float Ex = __ldg(a.ex + v);
    const float qEx = Ex - q0.x, qEy = 0.0f - q0.y, qEz = c.D - q0.z;
    const float num = -dot3(q3.x, q3.y, q3.z, qEx, qEy, qEz);
    const float ulo = float(i) * q0.w, uhi = float(i + 1) * q0.w;
    const float vlo = float(j) * q1.w, vhi = float(j + 1) * q1.w;
    unsigned long long* kv = reinterpret_cast<unsigned long long*>(a.keys) + (uint64_t)v * c.W * c.H;
    uint32_t writes = 0;
    for (int y = 0; y < c.H; y++) {
        const float Fy = fmaf(float(y) + 0.5f, -c.ph, c.y0);
        for (int x = 0; x < c.W; x++) {
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
            atomicMin(kv + (uint64_t)y * c.W + x, ((unsigned long long)__float_as_uint(t) << 32) | p);
            writes++;
        }
    }
    return writes;
}

// Screen-space edge function of the directed segment (px, py) -> (qx, qy) at (x, y).
__device__ __forceinline__ float sedge(float px, float py, float qx, float qy, float x, float y) {
    return fmaf(qx - px, y - py, -((qy - py) * (x - px)));
}

// One warp per point, lanes over the rendered views.
//
// Every eye lies on y = 0, z = D, so a world point C projects to pixel
// coordinates qx = A + B Ex, qy, with s = D / (D - C.z), A = (C.x s - x0) W/fw,
// B = (1 - s) W/fw, qy = (y0 - C.y s) H/fh: qy is the same in every view.
// Lanes 0-3 project the cell's corners and lanes 4-6 the triangle's vertices
// (one division each); shuffles give every lane all seven. The candidate rows
// (pixel-centre rows inside both the cell's and the triangle's y-extent) do
// not depend on the view, so a point without any is skipped by the whole warp.
// Per chunk of 32 views each lane forms its view's candidate columns (the
// intersection of the cell's and the triangle's x-extents); a warp scan of
// the candidate counts then gives every lane one candidate pixel per pass, so
// no lane loops over pixels on its own.
//
// The per-pixel test: edge functions of the projected cell (half-open: the
// u = i and v = j sides included, u = i+1 and v = j+1 excluded, so cells,
// which share bit-identical corners, partition their triangle's pixels) and
// of the projected triangle (closed); the orientation sign is the side of the
// triangle's plane the eye is on. A cell inside its triangle skips the
// triangle test; a triangle with a single point lies inside that point's cell
// and skips the cell test. The ray parameter t (the depth key) is divided out
// only for accepted pixels, by the plane-space formula.
constexpr int kSplatWarps = 8;

__global__ void __launch_bounds__(kSplatWarps * 32) k_splat(FrameArgs a) {
    __shared__ float s_ex[kMaxRenderViews];
    const DispConst& c = a.dc;
    for (int v = threadIdx.x; v < c.nr; v += blockDim.x) s_ex[v] = a.ex[v];
    __syncthreads();
    if (a.ctr->overflow) return;
    const uint32_t n = a.ctr->n_points;
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    const float W1 = float(c.W - 1), H1 = float(c.H - 1);
    const uint64_t npix = (uint64_t)c.W * c.H;
    uint32_t writes = 0;

    for (uint32_t p = warp; p < n; p += n_warps) {
        const uint2 pt = *reinterpret_cast<const uint2*>(a.points + p);
        const uint32_t tri = pt.x;
        const TriRec* r = a.rec + tri;
        const float4 q0 = __ldg(&r->q[0]), q1 = __ldg(&r->q[1]), q2 = __ldg(&r->q[2]);
        const float4 q3 = __ldg(&r->q[3]), q4 = __ldg(&r->q[4]);
        const int i = int(pt.y & 0xffffu), j = int(pt.y >> 16);

        // lanes 0-3: cell corners 00, 10, 11, 01; lanes 4-6: triangle vertices
        float pa = 0.0f, pb = 0.0f, py = 0.0f, pz = 0.0f;
        bool beh = false, in_tri = true;
        if (lane < 4) {
            const int ia = i + (lane == 1 || lane == 2), jb = j + (lane >= 2);
            float C[3];
            cell_corner(q0, q1, q2, q3, ia, jb, C);
            const float dep = c.D - C[2];
            beh = !(dep > 1e-4f * c.D);
            const float s = __fdiv_rn(c.D, dep);
            pa = fmaf(C[0], s, -c.x0) * c.ipw;
            pb = (1.0f - s) * c.ipw;
            py = (c.y0 - C[1] * s) * c.iph;
            // is this corner inside the closed 2-D triangle (lattice frame)?
            const float uu = float(ia) * q0.w + q2.w, vv = float(jb) * q1.w + q3.w;
            in_tri = edge_fn(q4.x, q4.y, q4.z, q4.w, uu, vv) >= 0.0f &&
                     edge_fn(q4.z, q4.w, 0.0f, 0.0f, uu, vv) >= 0.0f &&
                     edge_fn(0.0f, 0.0f, q4.x, q4.y, uu, vv) >= 0.0f;
        } else if (lane < 7) {
            const uint32_t vi = __ldg(a.idx + 3 * (size_t)tri + (lane - 4));
            const float x = __ldg(a.xyz + 3 * (size_t)vi), y = __ldg(a.xyz + 3 * (size_t)vi + 1),
                        z = __ldg(a.xyz + 3 * (size_t)vi + 2);
            const float* m = a.model;
            const float X = fmaf(m[0], x, fmaf(m[1], y, fmaf(m[2], z, m[3])));
            const float Y = fmaf(m[4], x, fmaf(m[5], y, fmaf(m[6], z, m[7])));
            const float Z = fmaf(m[8], x, fmaf(m[9], y, fmaf(m[10], z, m[11])));
            const float dep = c.D - Z;
            beh = !(dep > 1e-4f * c.D);
            const float s = __fdiv_rn(c.D, dep);
            pa = fmaf(X, s, -c.x0) * c.ipw;
            pb = (1.0f - s) * c.ipw;
            py = (c.y0 - Y * s) * c.iph;
            pz = Z;
        }
        const bool behind = __any_sync(0xffffffffu, beh);
        const bool interior = __all_sync(0xffffffffu, in_tri);
        const bool single = __ldg(a.counts + tri) == 1u;
        float cA[4], cB[4], cY[4], tA[3], tB[3], tY[3];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            cA[k] = __shfl_sync(0xffffffffu, pa, k);
            cB[k] = __shfl_sync(0xffffffffu, pb, k);
            cY[k] = __shfl_sync(0xffffffffu, py, k);
        }
#pragma unroll
        for (int k = 0; k < 3; k++) {
            tA[k] = __shfl_sync(0xffffffffu, pa, 4 + k);
            tB[k] = __shfl_sync(0xffffffffu, pb, 4 + k);
            tY[k] = __shfl_sync(0xffffffffu, py, 4 + k);
        }
        const float z0 = __shfl_sync(0xffffffffu, pz, 4), z1 = __shfl_sync(0xffffffffu, pz, 5),
                    z2 = __shfl_sync(0xffffffffu, pz, 6);

        if (behind) {   // rare: the cell or triangle reaches the eyes' plane
            for (int v = lane; v < c.nr; v += 32) writes += splat_exact(a, p, i, j, v, q0, q1, q2, q3, q4);
            continue;
        }
        const float zmin = fminf(fminf(z0, z1), z2), zmax = fmaxf(fmaxf(z0, z1), z2);
        const bool depth_ok = (c.D - zmax) >= c.near_z && (c.D - zmin) <= c.far_z;

        // candidate rows: inside both y-extents (view-independent)
        const float cymn = fminf(fminf(cY[0], cY[1]), fminf(cY[2], cY[3]));
        const float cymx = fmaxf(fmaxf(cY[0], cY[1]), fmaxf(cY[2], cY[3]));
        const float tymn = fminf(fminf(tY[0], tY[1]), tY[2]), tymx = fmaxf(fmaxf(tY[0], tY[1]), tY[2]);
        const float fy0 = fmaxf(ceilf(fmaxf(cymn, tymn) - 0.5f - kBoxPad), 0.0f);
        const float fy1 = fminf(floorf(fminf(cymx, tymx) - 0.5f + kBoxPad), H1);
        if (!(fy0 <= fy1)) continue;
        const int y0 = int(fy0);
        const uint32_t ny = uint32_t(int(fy1) - y0 + 1);
        const float kn = fmaf(q3.y, 0.0f - q0.y, q3.z * (c.D - q0.z)) - q3.x * q0.x;

        for (int base = 0; base < c.nr; base += 32) {
            const int v = base + lane;
            float Ex = 0.0f;
            uint32_t nx = 0;
            int x0 = 0;
            if (v < c.nr) {
                Ex = s_ex[v];
                float xmn = INFINITY, xmx = -INFINITY, tmn = INFINITY, tmx = -INFINITY;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const float X = fmaf(cB[k], Ex, cA[k]);
                    xmn = fminf(xmn, X);
                    xmx = fmaxf(xmx, X);
                }
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const float X = fmaf(tB[k], Ex, tA[k]);
                    tmn = fminf(tmn, X);
                    tmx = fmaxf(tmx, X);
                }
                const float fx0 = fmaxf(ceilf(fmaxf(xmn, tmn) - 0.5f - kBoxPad), 0.0f);
                const float fx1 = fminf(floorf(fminf(xmx, tmx) - 0.5f + kBoxPad), W1);
                if (fx0 <= fx1) {
                    x0 = int(fx0);
                    nx = uint32_t(int(fx1) - x0 + 1);
                }
            }
            const uint32_t cnt = nx * ny;
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            const uint32_t excl = incl - cnt;
            for (uint32_t pass = 0; pass < total; pass += 32) {
                const uint32_t q = pass + lane;
                // owner: the first lane whose inclusive count exceeds q
                int own = 0;
#pragma unroll
                for (int st = 16; st >= 1; st >>= 1) {
                    const uint32_t t = __shfl_sync(0xffffffffu, incl, own + st - 1);
                    if (t <= q) own += st;
                }
                own = own > 31 ? 31 : own;
                const uint32_t o_excl = __shfl_sync(0xffffffffu, excl, own);
                const uint32_t o_nx = __shfl_sync(0xffffffffu, nx, own);
                const int o_x0 = __shfl_sync(0xffffffffu, x0, own);
                const float o_Ex = __shfl_sync(0xffffffffu, Ex, own);
                if (q >= total) continue;
                const uint32_t rr = q - o_excl;
                const uint32_t ry = rr / o_nx, rx = rr - ry * o_nx;
                const int x = o_x0 + int(rx), y = y0 + int(ry);
                const float px = float(x) + 0.5f, pyc = float(y) + 0.5f;
                const float nE = fmaf(q3.x, o_Ex, kn);
                if (nE == 0.0f) continue;              // plane seen edge-on
                const float sg = nE > 0.0f ? 1.0f : -1.0f;
                if (!single) {
                    float X[4];
#pragma unroll
                    for (int k = 0; k < 4; k++) X[k] = fmaf(cB[k], o_Ex, cA[k]);
                    const float eL = sg * sedge(X[0], cY[0], X[3], cY[3], px, pyc);
                    const float eR = sg * sedge(X[1], cY[1], X[2], cY[2], px, pyc);
                    const float eB = sg * sedge(X[0], cY[0], X[1], cY[1], px, pyc);
                    const float eT = sg * sedge(X[3], cY[3], X[2], cY[2], px, pyc);
                    if (!(eL >= 0.0f && eR < 0.0f && eB <= 0.0f && eT > 0.0f)) continue;
                }
                if (!interior) {
                    float TX[3];
#pragma unroll
                    for (int k = 0; k < 3; k++) TX[k] = fmaf(tB[k], o_Ex, tA[k]);
                    const float t0 = sg * sedge(TX[0], tY[0], TX[1], tY[1], px, pyc);
                    const float t1 = sg * sedge(TX[1], tY[1], TX[2], tY[2], px, pyc);
                    const float t2 = sg * sedge(TX[2], tY[2], TX[0], tY[0], px, pyc);
                    if (!(t0 <= 0.0f && t1 <= 0.0f && t2 <= 0.0f)) continue;
                }
                const float qEx = o_Ex - q0.x, qEy = 0.0f - q0.y, qEz = c.D - q0.z;
                const float num = -dot3(q3.x, q3.y, q3.z, qEx, qEy, qEz);
                const float Fx = fmaf(px, c.pw, c.x0), Fy = fmaf(pyc, -c.ph, c.y0);
                const float den = dot3(q3.x, q3.y, q3.z, Fx - o_Ex, Fy - 0.0f, -c.D);
                const float t = __fdiv_rn(num, den);
                if (!(t > 0.0f)) continue;
                if (!depth_ok) {
                    const float depth = t * c.D;
                    if (!(depth >= c.near_z && depth <= c.far_z)) continue;
                }
                unsigned long long* kv = reinterpret_cast<unsigned long long*>(a.keys) + (uint64_t)(base + own) * npix;
                atomicMin(kv + (uint64_t)y * c.W + x, ((unsigned long long)__float_as_uint(t) << 32) | p);
                writes++;
            }
        }
    }
    // warp-aggregated count of depth-test writes (the atomics issued)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) writes += __shfl_xor_sync(0xffffffffu, writes, o);
    if (lane == 0 && writes) atomicAdd(&a.ctr->n_writes, writes);
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
    k_splat<<<a.sm_count * 16, kSplatWarps * 32, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_resolve(const FrameArgs& a, cudaStream_t s) {
    k_resolve<<<a.sm_count * 8, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lfdpr
