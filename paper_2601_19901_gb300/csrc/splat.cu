// EPR splatting into every view (Sec. 3.2) with the 64-bit depth|id test
// (Sec. 5.1), and the per-view resolve of Eq. 8-9 (Sec. 3.3).
//
//   k_splat    one half-warp per point, lanes over the views: every pixel centre
//              inside the point's projected cell and its projected triangle,
//              at a depth in [near, far], does
//              atomicMin(key, float_bits(t) << 32 | point id).
//   k_resolve  one thread per view pixel: the winning point's cell corners
//              (from its resolve record) are projected for the splat's pixel
//              area (shoelace), Eq. 8 gives the view's texture area, Eq. 9
//              interpolates tv_min..tv_max.
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

// One half-warp (16 lanes) per point of the work list, each lane taking up to
// S views of the point (views g + 16 s + lane of a group g of 16 S views, S
// chosen so that one group holds every rendered view where it can); a warp
// carries two points at a time.
//
// Candidates. Candidate rows are the pixel-centre rows inside both the
// cell's and the triangle's projected y-extent, the same in every view since
// every eye lies on y = 0, z = D. A lane forms each of its views' candidate
// columns between a lower and an upper line x = alpha + beta Ex for the cell
// and for the triangle, which bound each one's projected x-extent within the
// band of candidate rows (the row's exact crossings for most points with one
// row), widened by a small margin. A scan of the lanes' candidate counts over
// the whole group then hands every lane one candidate pixel per pass, so no
// lane loops over pixels on its own and a point with few candidates needs a
// single pass.
//
// Test. Each candidate takes the per-pixel test in the oracle's plane-space
// form: the pixel centre's ray from the eye meets the triangle's plane at t
// (the division also yields the depth key); the hit must lie in the half-open
// cell and in the closed triangle (2-D edge functions of the lattice frame),
// at a depth t D in [near, far]. A cell inside its triangle skips the triangle
// test. The margin of the candidate ranges only admits extra candidates; the
// test alone decides.
//
// Points whose cell or triangle reaches the eyes' plane (none in front-only
// scenes) are listed apart and splatted by k_splat_near.
constexpr int kSplatWarps = 8;
// Ask L2 for the line holding p (no register result).
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// The per-pixel test; every condition is evaluated (no early exits), so the
// two points of a warp and the lanes' different candidates do not diverge.
__device__ __forceinline__ bool pixel_test(const DispConst& c, float Ex, float num, float qEx, float qEy,
                                           float qEz, const float4& q1, const float4& q2, const float4& q3,
                                           const float4& q4, float ulo, float uhi, float vlo, float vhi,
                                           bool interior, bool depth_ok, int x, int y, float& t) {
    const float Fx = fmaf(float(x) + 0.5f, c.pw, c.x0);
    const float Fy = fmaf(float(y) + 0.5f, -c.ph, c.y0);
    const float dx = Fx - Ex, dy = Fy - 0.0f, dz = -c.D;
    const float den = dot3(q3.x, q3.y, q3.z, dx, dy, dz);
    t = __fdiv_rn(num, den);
    const float depth = t * c.D;
    const bool in_depth = depth_ok ? t > 0.0f : (depth >= c.near_z && depth <= c.far_z);
    const float hx = fmaf(t, dx, qEx), hy = fmaf(t, dy, qEy), hz = fmaf(t, dz, qEz);
    const float uq = dot3(hx, hy, hz, q1.x, q1.y, q1.z);
    const float vq = dot3(hx, hy, hz, q2.x, q2.y, q2.z);
    const float u = uq - q2.w, vv = vq - q3.w;
    const bool in_cell = u >= ulo && u < uhi && vv >= vlo && vv < vhi;
    const float w0 = edge_fn(q4.x, q4.y, q4.z, q4.w, uq, vq);
    const float w1 = edge_fn(q4.z, q4.w, 0.0f, 0.0f, uq, vq);
    const float w2 = edge_fn(0.0f, 0.0f, q4.x, q4.y, uq, vq);
    return (den != 0.0f) & in_depth & in_cell & (interior | inside_either(w0, w1, w2));
}

template <int S>
__global__ void __launch_bounds__(kSplatWarps * 32, 4) k_splat(FrameArgs a) {
    __shared__ float s_ex[kMaxRenderViews];
    const DispConst& c = a.dc;
    for (int v = threadIdx.x; v < c.nr; v += blockDim.x) s_ex[v] = a.ex[v];
    __syncthreads();
    if (a.ctr->overflow) return;
    const uint32_t n = a.ctr->n_work;
    const int lane = threadIdx.x & 31, sub = lane & 15, half = lane >> 4;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    const uint64_t npix = (uint64_t)c.W * c.H;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(a.keys);
    uint32_t writes = 0;

    // Every loop below has the same trip count in both halves of the warp
    // (pairs of points; the larger pass count of the two), so each warp
    // instruction serves both points.
    for (uint32_t kk = warp; 2 * kk < n; kk += n_warps) {
        const uint32_t k = 2 * kk + uint32_t(half);
        const bool act = k < n;
        const WorkRec* wr = a.work + (act ? k : 2 * kk);
        if (sub == 0 && k + 2 * n_warps < n) prefetch_l2(a.work + k + 2 * n_warps);   // next pair's record
        const float4 L0 = __ldg(&wr->L0), L1 = __ldg(&wr->L1);
        const uint4 meta = __ldg(&wr->meta);
        const uint32_t tri = meta.z;
        const unsigned long long pid = meta.w;
        const TriRec* r = a.rec + tri;
        const float4 q0 = __ldg(&r->q[0]), q1 = __ldg(&r->q[1]), q2 = __ldg(&r->q[2]);
        const float4 q3 = __ldg(&r->q[3]), q4 = __ldg(&r->q[4]);
        const int y0 = int(meta.x & 0x3fffu);
        const uint32_t ny = act ? (meta.x >> 14) & 0x7fffu : 0u;
        const uint32_t flags = meta.x >> 29;
        const bool interior = flags & kFlagInterior, depth_ok = flags & kFlagDepthOk;
        const int i = int(meta.y & 0xffffu), j = int(meta.y >> 16);
        const float ulo = float(i) * q0.w, uhi = float(i + 1) * q0.w;
        const float vlo = float(j) * q1.w, vhi = float(j + 1) * q1.w;
        const float qEy = 0.0f - q0.y, qEz = c.D - q0.z;

        for (int g = 0; g < c.nr; g += 16 * S) {
            uint32_t pk[S];      // x0 | n_columns << 14 of the lane's views
            uint32_t cnt = 0;
#pragma unroll
            for (int sl = 0; sl < S; sl++) {
                const int v = g + 16 * sl + sub;
                pk[sl] = 0u;
                if (v < c.nr) {
                    const float Ex = s_ex[v];
                    const float lo = fmaxf(fmaf(L0.y, Ex, L0.x), fmaf(L1.y, Ex, L1.x));
                    const float hi = fminf(fmaf(L0.w, Ex, L0.z), fmaf(L1.w, Ex, L1.z));
                    const int ix0 = max(__float2int_ru(lo), 0);
                    const int ix1 = min(__float2int_rd(hi), int(c.W) - 1);
                    if (ix0 <= ix1) {
                        const uint32_t x0 = uint32_t(ix0), nx = uint32_t(ix1 - ix0) + 1u;
                        pk[sl] = x0 | (nx << 14);
                        cnt += nx * ny;
                    }
                }
            }
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 16; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o, 16);
                if (sub >= o) incl += t;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 15, 16);
            const uint32_t both = max(total, __shfl_xor_sync(0xffffffffu, total, 16));
            const uint32_t excl = incl - cnt;
            for (uint32_t pass = 0; pass < both; pass += 16) {
                const uint32_t q = pass + sub;
                // owner: the first lane of this half whose inclusive count exceeds q
                int own = 0;
#pragma unroll
                for (int st = 8; st >= 1; st >>= 1) {
                    const uint32_t t = __shfl_sync(0xffffffffu, incl, own + st - 1, 16);
                    if (t <= q) own += st;
                }
                const uint32_t o_excl = __shfl_sync(0xffffffffu, excl, own, 16);
                uint32_t opk[S];
#pragma unroll
                for (int sl = 0; sl < S; sl++) opk[sl] = __shfl_sync(0xffffffffu, pk[sl], own, 16);
                if (q >= total) continue;
                // the owner's view slot holding candidate q
                uint32_t rr = q - o_excl, sel = opk[0];
                int slot = 0;
#pragma unroll
                for (int sl = 0; sl + 1 < S; sl++) {
                    const uint32_t cs = (opk[sl] >> 14) * ny;
                    if (slot == sl && rr >= cs) {
                        rr -= cs;
                        slot = sl + 1;
                        sel = opk[sl + 1];
                    }
                }
                const uint32_t o_nx = sel >> 14;
                const uint32_t ry = ny == 1 ? 0u : rr / o_nx;
                const int x = int(sel & 0x3fffu) + int(rr - ry * o_nx), y = y0 + int(ry);
                const int vo = g + 16 * slot + own;
                const float Ex_o = s_ex[vo];
                const float qEx = Ex_o - q0.x;
                const float num = -dot3(q3.x, q3.y, q3.z, qEx, qEy, qEz);
                float t;
                if (!pixel_test(c, Ex_o, num, qEx, qEy, qEz, q1, q2, q3, q4, ulo, uhi, vlo, vhi, interior, depth_ok,
                                x, y, t))
                    continue;
                // a view holds at most 2^26 pixels: 32-bit offset within it
                atomicMin(keys + ((uint64_t)uint32_t(vo) * uint32_t(npix) + (uint32_t(y) * uint32_t(c.W) + uint32_t(x))),
                          ((unsigned long long)__float_as_uint(t) << 32) | pid);
                writes++;
            }
        }
    }
    // warp-aggregated count of depth-test writes (the atomics issued)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) writes += __shfl_xor_sync(0xffffffffu, writes, o);
    if (lane == 0 && writes) atomicAdd(&a.ctr->n_writes, writes);
}

// Points whose cell or triangle reaches the eyes' plane: their projections
// are unbounded, so every pixel of every view takes the plane-space test,
// one (point, view) pair per thread. None occur in front-only scenes.
__global__ void __launch_bounds__(256) k_splat_near(FrameArgs a) {
    if (a.ctr->overflow) return;
    const DispConst& c = a.dc;
    const uint32_t n = a.ctr->n_near;
    const uint64_t pairs = (uint64_t)n * c.nr;
    const uint64_t npix = (uint64_t)c.W * c.H;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(a.keys);
    uint32_t writes = 0;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < pairs;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t k = uint32_t(g / c.nr);
        const int v = int(g - (uint64_t)k * c.nr);
        const uint32_t p = a.near[k];
        const uint2 pt = *reinterpret_cast<const uint2*>(a.points + p);
        const TriRec* r = a.rec + pt.x;
        const float4 q0 = __ldg(&r->q[0]), q1 = __ldg(&r->q[1]), q2 = __ldg(&r->q[2]);
        const float4 q3 = __ldg(&r->q[3]), q4 = __ldg(&r->q[4]);
        const int i = int(pt.y & 0xffffu), j = int(pt.y >> 16);
        const float ulo = float(i) * q0.w, uhi = float(i + 1) * q0.w;
        const float vlo = float(j) * q1.w, vhi = float(j + 1) * q1.w;
        const float Ex = __ldg(a.ex + v);
        const float qEx = Ex - q0.x, qEy = 0.0f - q0.y, qEz = c.D - q0.z;
        const float num = -dot3(q3.x, q3.y, q3.z, qEx, qEy, qEz);
        for (int y = 0; y < c.H; y++) {
            for (int x = 0; x < c.W; x++) {
                float t;
                if (!pixel_test(c, Ex, num, qEx, qEy, qEz, q1, q2, q3, q4, ulo, uhi, vlo, vhi, false, false, x, y,
                                t))
                    continue;
                atomicMin(keys + (uint64_t)v * npix + (uint64_t)y * c.W + x,
                          ((unsigned long long)__float_as_uint(t) << 32) | p);
                writes++;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) writes += __shfl_xor_sync(0xffffffffu, writes, o);
    if ((threadIdx.x & 31) == 0 && writes) atomicAdd(&a.ctr->n_writes, writes);
}

// Eq. 8-9 for one view pixel whose depth test kept point record rp (the
// caller has already loaded it): the splat's pixel area in view Ex is the
// shoelace area of its cell corners projected from the eye.
__device__ __forceinline__ uint32_t resolve_pixel(const DispConst& c, float Ex, const float4& c0, const float4& c1,
                                                  const float4& c2, const float4& m, const uint4& tv) {
    const float cx[4] = {c0.x, c0.w, c1.z, c2.y}, cy[4] = {c0.y, c1.x, c1.w, c2.z};
    const float cs[4] = {c0.z, c1.y, c2.x, c2.w};
    float X[4], Y[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const float sx = fmaf(cx[k] - Ex, cs[k], Ex);
        const float sy = cy[k] * cs[k];
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
    const float vmin = m.y, vmax = m.z;
    const float size_vse = __fdiv_rn(m.x, fminf(1.0f, area_px));
    const float size_vs = fminf(fmaxf(size_vse, vmin), vmax);
    const float w = vmax > vmin ? __fdiv_rn(size_vs - vmin, vmax - vmin) : 0.0f;
    uint32_t out = 0u;
#pragma unroll
    for (int ch = 0; ch < 4; ch++) {
        const float lo = float((tv.x >> (8 * ch)) & 255u), hi = float((tv.y >> (8 * ch)) & 255u);
        out |= uint32_t(round_u8(fmaf(w, hi - lo, lo))) << (8 * ch);
    }
    return out;
}

// One view pixel per thread (grid: pixels x views).
__global__ void __launch_bounds__(256) k_resolve(FrameArgs a) {
    const DispConst& c = a.dc;
    const uint32_t npix = uint32_t(c.W) * uint32_t(c.H);
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const int v = blockIdx.y;
    const uint64_t o = (uint64_t)v * npix + p;
    const unsigned long long key = a.keys[o];
    uint32_t out = 0u;
    if (key != ~0ull) {
        const ResolveRec* rp = a.rrec + uint32_t(key);
        out = resolve_pixel(c, __ldg(a.ex + v), __ldg(&rp->c0), __ldg(&rp->c1), __ldg(&rp->c2), __ldg(&rp->m),
                            __ldg(&rp->tv));
    }
    reinterpret_cast<uint32_t*>(a.views)[o] = out;
}

}  // namespace

cudaError_t launch_splat(const FrameArgs& a, cudaStream_t s) {
    // the fewest view slots per lane that hold every rendered view in one
    // group (more than 128 views take several groups of 128)
    const int nr = a.dc.nr, grid = a.sm_count * 16, block = kSplatWarps * 32;
    if (nr <= 16)
        k_splat<1><<<grid, block, 0, s>>>(a);
    else if (nr <= 32)
        k_splat<2><<<grid, block, 0, s>>>(a);
    else if (nr <= 48)
        k_splat<3><<<grid, block, 0, s>>>(a);
    else if (nr <= 64)
        k_splat<4><<<grid, block, 0, s>>>(a);
    else if (nr <= 96)
        k_splat<6><<<grid, block, 0, s>>>(a);
    else
        k_splat<8><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_splat_near(const FrameArgs& a, cudaStream_t s) {
    k_splat_near<<<a.sm_count * 2, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_resolve(const FrameArgs& a, cudaStream_t s) {
    const uint32_t npix = uint32_t(a.dc.W) * uint32_t(a.dc.H);
    const dim3 grid((npix + 255u) / 256u, uint32_t(a.dc.nr));
    k_resolve<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lfdpr
