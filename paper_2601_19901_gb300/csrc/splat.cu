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

__device__ __forceinline__ void cell_corner(const float4& q0, const float4& q1, const float4& q2,
                                            const float4& q3, int ia, int jb, float* o) {
    const float cu = float(ia) * q0.w + q2.w;
    const float cv = float(jb) * q1.w + q3.w;
    o[0] = fmaf(cu, q1.x, fmaf(cv, q2.x, q0.x));
    o[1] = fmaf(cu, q1.y, fmaf(cv, q2.y, q0.y));
    o[2] = fmaf(cu, q1.z, fmaf(cv, q2.z, q0.z));
}

// Screen-space edge function of the directed segment (px, py) -> (qx, qy) at (x, y).
__device__ __forceinline__ float sedge(float px, float py, float qx, float qy, float x, float y) {
    return fmaf(qx - px, y - py, -((qy - py) * (x - px)));
}

// One warp per point of the work list (points with at least one candidate
// pixel row), lanes over the rendered views.
//
// The point's splat record holds its cell corners projected into every view
// (pixel x = A + B Ex, pixel y = Y, the same in all views since every eye
// lies on y = 0, z = D) and its candidate rows: rows inside both the cell's
// and the triangle's y-extent. Per chunk of 32 views each lane forms its
// view's candidate columns (the cell's and the triangle's x-extents
// intersected); a warp scan of the candidate counts then gives every lane one
// candidate pixel per pass, so no lane loops over pixels on its own.
//
// The per-pixel test: edge functions of the projected cell (half-open: the
// u = i and v = j sides included, u = i+1 and v = j+1 excluded, so cells,
// which share bit-identical corners, partition their triangle's pixels) and
// of the projected triangle (closed); the orientation sign is the side of the
// triangle's plane the eye is on. A cell inside its triangle skips the
// triangle test; a triangle with a single point lies inside that point's cell
// and skips the cell test. The ray parameter t (the depth key) is divided out
// only for accepted pixels, by the plane-space formula.
//
// Points whose cell or triangle reaches the eyes' plane (never in front-only
// scenes) take the plane-space form of the test (the oracle's formula) over
// the whole view instead, one view per lane.
constexpr int kSplatWarps = 8;

__global__ void __launch_bounds__(kSplatWarps * 32, 4) k_splat(FrameArgs a) {
    __shared__ float s_ex[kMaxRenderViews];
    const DispConst& c = a.dc;
    for (int v = threadIdx.x; v < c.nr; v += blockDim.x) s_ex[v] = a.ex[v];
    __syncthreads();
    if (a.ctr->overflow) return;
    const uint32_t n = a.ctr->n_work;
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    const float W1 = float(c.W - 1);
    const uint64_t npix = (uint64_t)c.W * c.H;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(a.keys);
    uint32_t writes = 0;

    for (uint32_t k = warp; k < n; k += n_warps) {
        const uint32_t p = __ldg(a.work + k);
        const SplatRec* srp = a.srec + p;
        const float4 cA = __ldg(&srp->A), cB = __ldg(&srp->B), cY = __ldg(&srp->Y);
        const uint4 meta = __ldg(&srp->meta);
        const uint32_t tri = meta.w, flags = meta.z;
        const TriRec* r = a.rec + tri;
        const float4 q0 = __ldg(&r->q[0]), q3 = __ldg(&r->q[3]);

        if (flags & kFlagBehind) {
            const float4 q1 = __ldg(&r->q[1]), q2 = __ldg(&r->q[2]), q4 = __ldg(&r->q[4]);
            const uint2 pt = *reinterpret_cast<const uint2*>(a.points + p);
            const int i = int(pt.y & 0xffffu), j = int(pt.y >> 16);
            const float ulo = float(i) * q0.w, uhi = float(i + 1) * q0.w;
            const float vlo = float(j) * q1.w, vhi = float(j + 1) * q1.w;
            for (int v = lane; v < c.nr; v += 32) {
                const float Ex = s_ex[v];
                const float qEx = Ex - q0.x, qEy = 0.0f - q0.y, qEz = c.D - q0.z;
                const float num = -dot3(q3.x, q3.y, q3.z, qEx, qEy, qEz);
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
                        atomicMin(keys + (uint64_t)v * npix + (uint64_t)y * c.W + x,
                                  ((unsigned long long)__float_as_uint(t) << 32) | p);
                        writes++;
                    }
                }
            }
            continue;
        }

        const TriProj* tpp = a.tproj + tri;
        const float4 tA = __ldg(&tpp->a), tB = __ldg(&tpp->b), tY = __ldg(&tpp->y);
        const int y0 = int(meta.x);
        const uint32_t ny = meta.y;
        const bool single = flags & kFlagSingle, interior = flags & kFlagInterior;
        const bool depth_ok = flags & kFlagDepthOk;
        // n . (E - P0) = n.x Ex + kn
        const float kn = fmaf(q3.y, 0.0f - q0.y, q3.z * (c.D - q0.z)) - q3.x * q0.x;

        for (int base = 0; base < c.nr; base += 32) {
            const int v = base + lane;
            float Ex = 0.0f;
            uint32_t nx = 0;
            int x0 = 0;
            if (v < c.nr) {
                Ex = s_ex[v];
                const float X0 = fmaf(cB.x, Ex, cA.x), X1 = fmaf(cB.y, Ex, cA.y);
                const float X2 = fmaf(cB.z, Ex, cA.z), X3 = fmaf(cB.w, Ex, cA.w);
                const float T0 = fmaf(tB.x, Ex, tA.x), T1 = fmaf(tB.y, Ex, tA.y), T2 = fmaf(tB.z, Ex, tA.z);
                const float xmn = fmaxf(fminf(fminf(X0, X1), fminf(X2, X3)), fminf(fminf(T0, T1), T2));
                const float xmx = fminf(fmaxf(fmaxf(X0, X1), fmaxf(X2, X3)), fmaxf(fmaxf(T0, T1), T2));
                const float fx0 = fmaxf(ceilf(xmn - 0.5f - kBoxPad), 0.0f);
                const float fx1 = fminf(floorf(xmx - 0.5f + kBoxPad), W1);
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
                const uint32_t o_excl = __shfl_sync(0xffffffffu, excl, own);
                const uint32_t o_nx = __shfl_sync(0xffffffffu, nx, own);
                const int o_x0 = __shfl_sync(0xffffffffu, x0, own);
                const float o_Ex = __shfl_sync(0xffffffffu, Ex, own);
                if (q >= total) continue;
                const uint32_t rr = q - o_excl;
                const uint32_t ry = ny == 1 ? 0u : rr / o_nx;
                const uint32_t rx = rr - ry * o_nx;
                const int x = o_x0 + int(rx), y = y0 + int(ry);
                const float px = float(x) + 0.5f, pyc = float(y) + 0.5f;
                const float nE = fmaf(q3.x, o_Ex, kn);
                if (nE == 0.0f) continue;              // plane seen edge-on
                const float sg = nE > 0.0f ? 1.0f : -1.0f;
                if (!single) {
                    const float X0 = fmaf(cB.x, o_Ex, cA.x), X1 = fmaf(cB.y, o_Ex, cA.y);
                    const float X2 = fmaf(cB.z, o_Ex, cA.z), X3 = fmaf(cB.w, o_Ex, cA.w);
                    const float eL = sg * sedge(X0, cY.x, X3, cY.w, px, pyc);
                    const float eR = sg * sedge(X1, cY.y, X2, cY.z, px, pyc);
                    const float eB = sg * sedge(X0, cY.x, X1, cY.y, px, pyc);
                    const float eT = sg * sedge(X3, cY.w, X2, cY.z, px, pyc);
                    if (!(eL >= 0.0f && eR < 0.0f && eB <= 0.0f && eT > 0.0f)) continue;
                }
                if (!interior) {
                    const float T0 = fmaf(tB.x, o_Ex, tA.x), T1 = fmaf(tB.y, o_Ex, tA.y), T2 = fmaf(tB.z, o_Ex, tA.z);
                    const float e0 = sg * sedge(T0, tY.x, T1, tY.y, px, pyc);
                    const float e1 = sg * sedge(T1, tY.y, T2, tY.z, px, pyc);
                    const float e2 = sg * sedge(T2, tY.z, T0, tY.x, px, pyc);
                    if (!(e0 <= 0.0f && e1 <= 0.0f && e2 <= 0.0f)) continue;
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
                atomicMin(keys + (uint64_t)(base + own) * npix + (uint64_t)y * c.W + x,
                          ((unsigned long long)__float_as_uint(t) << 32) | p);
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
