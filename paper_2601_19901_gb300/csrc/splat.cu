// EPR splatting into every view (Sec. 3.2) with the 64-bit depth|id test
// (Sec. 5.1), and the per-view resolve of Eq. 8-9 (Sec. 3.3).
//
//   k_splat    a half-warp per point forms the candidate pixels of every view,
//              a warp's candidates of several points are pooled into 32-lane
//              passes: every pixel centre inside the point's projected cell
//              and its projected triangle, at a depth in [near, far], does
//              atomicMin(key, float_bits(t) << 32 | point id).
//   k_resolve  one thread per view pixel: the winning point's 32-byte resolve
//              record gives the splat's pixel area in this view
//              (|alpha + beta Ex| / 2), Eq. 8 the view's texture area, Eq. 9
//              interpolates tv_min..tv_max.
#include "lfdpr_internal.cuh"

namespace lfdpr {
namespace {

// A warp takes a unit of 2P consecutive points of the work list: for each of
// its P pairs, one half-warp (16 lanes) per point, each lane taking up to S
// views of the point (views g + 16 s + lane of a group g of 16 S views, S
// chosen so that one group holds every rendered view where it can).
//
// Candidates. Candidate rows are the pixel-centre rows inside both the
// cell's and the triangle's projected y-extent, the same in every view since
// every eye lies on y = 0, z = D. A lane forms each of its views' candidate
// columns between a lower and an upper line x = alpha + beta Ex for the cell
// and for the triangle, which bound each one's projected x-extent within the
// band of candidate rows (the row's exact crossings for most points with one
// row), widened by a small margin.
//
// Pooling. The unit's candidates are numbered in (lane, pair, view slot)
// order; the non-empty (point, view) segments of that numbering go to a
// per-warp list in shared memory with their first number, and the points'
// test constants beside it. Then every pass hands the warp's 32 lanes the
// next 32 candidates of the whole unit: a lane's segment is the last one
// starting at or before its number, found from the OR-reduction of the
// start bits that fall in the pass (segments are numbered in start order).
// Points with few candidates, most of the work list, thus share passes
// instead of each filling a pass on its own.
//
// Test. Each candidate takes the per-pixel test in the oracle's plane-space
// form: the pixel centre's ray from the eye meets the triangle's plane at t
// (the division also yields the depth key); the hit must lie in the half-open
// cell and in the closed triangle (2-D edge functions of the lattice frame),
// at a depth t D in [near, far]. A cell inside its triangle skips the triangle
// test. The margin of the candidate ranges only admits extra candidates; the
// test alone decides.
//
// Points whose cell or triangle reaches within near_z of the eyes' plane come
// with candidate bounds of their cell and triangle clipped to that limit
// (k_fetch) and take the same passes and test.
constexpr int kSplatWarps = 8;

// The per-pixel test; every condition is evaluated (no early exits), so the
// lanes' different candidates do not diverge.
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

// Eye x of view v from the eye array at shared-memory address ex_s.
__device__ __forceinline__ float eye_x(uint32_t ex_s, int v) {
    float e;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(e) : "r"(ex_s + 4u * uint32_t(v)));
    return e;
}

// warp-aggregated count of depth-test writes (the atomics issued)
__device__ __forceinline__ void add_writes(Counters* ctr, uint32_t writes) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) writes += __shfl_xor_sync(0xffffffffu, writes, o);
    if ((threadIdx.x & 31) == 0 && writes) atomicAdd(&ctr->n_writes, writes);
}

// floor(r / n) for n >= 1: below 2^21 one approximate division of r + 1/2
// (its quotient stays at least 1 / (2n) from an integer, more than the 2-ulp
// error of __fdividef), else an integer division.
__device__ __forceinline__ uint32_t div_floor(uint32_t r, uint32_t n) {
    if (r < (1u << 21)) return uint32_t(__fdividef(float(r) + 0.5f, float(n)));
    return r / n;
}

// Units of 2P points per warp: pairs per unit for S view slots per lane.
template <int S>
struct UnitPairs {
    static constexpr int P = S <= 3 ? 2 : 1;
};

// Per-warp shared memory of the pooled splat: the unit's non-empty (point,
// view) segments in candidate order (first candidate number,
// x0 | n_columns << 14, view | point << 16, eye x) and its points' test
// constants: (P0.x, -P0.y, D - P0.z, point id), (u-hat, work meta word),
// (v-hat, u_min), (n-hat, v_min), the 2-D vertices, the cell's u and v bounds.
template <int S>
struct SplatWarpSmem {
    static constexpr int P = UnitPairs<S>::P, kSegs = 32 * S * P;
    uint4 seg[kSegs];
    float4 pt[2 * P][6];
};

// Where the splat's units come from: one scene (its constants in the kernel's
// parameters), or every scene of a batch (constants in shared memory; the
// units of all scenes form one index range, scene by scene).
struct OneScene {
    static constexpr bool kMany = false;
    const FrameArgs& a;
    uint32_t n;       // work points
    uint32_t ex_s;    // shared-memory address of the eye positions
    __device__ __forceinline__ int scene(uint32_t) const { return 0; }
    __device__ __forceinline__ uint32_t first_unit(int) const { return 0u; }
    __device__ __forceinline__ const DispConst& dc(int) const { return a.dc; }
    __device__ __forceinline__ float eye(int, int v) const { return eye_x(ex_s, v); }
    __device__ __forceinline__ uint32_t points(int) const { return n; }
    __device__ __forceinline__ const WorkRec* work(int) const { return a.work; }
    __device__ __forceinline__ const TriRec* rec(int) const { return a.rec; }
    __device__ __forceinline__ unsigned long long* keys(int) const {
        return reinterpret_cast<unsigned long long*>(a.keys);
    }
    __device__ __forceinline__ Counters* ctr(int) const { return a.ctr; }
    __device__ __forceinline__ uint32_t lane_limit() const { return a.splat_lane_limit; }
    __device__ __forceinline__ int view_lo(int) const { return a.view_lo; }
    __device__ __forceinline__ int view_hi(int) const { return a.view_hi; }
};

struct ManyScenes {
    static constexpr bool kMany = true;
    const SplatScene* scenes;
    int n_scenes;
    const DispConst* s_dc;
    const uint32_t* s_unit0;   // first unit of each scene, then the total
    const uint32_t* s_n;       // work points of each scene
    // the scene holding unit g: the last with s_unit0 <= g
    __device__ __forceinline__ int scene(uint32_t g) const {
        int lo = 0, hi = n_scenes - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_unit0[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    }
    __device__ __forceinline__ uint32_t first_unit(int q) const { return s_unit0[q]; }
    __device__ __forceinline__ const DispConst& dc(int q) const { return s_dc[q]; }
    __device__ __forceinline__ float eye(int q, int v) const { return __ldg(scenes[q].ex + v); }
    __device__ __forceinline__ uint32_t points(int q) const { return s_n[q]; }
    __device__ __forceinline__ const WorkRec* work(int q) const { return scenes[q].work; }
    __device__ __forceinline__ const TriRec* rec(int q) const { return scenes[q].rec; }
    __device__ __forceinline__ unsigned long long* keys(int q) const {
        return reinterpret_cast<unsigned long long*>(scenes[q].keys);
    }
    __device__ __forceinline__ Counters* ctr(int q) const { return scenes[q].ctr; }
    __device__ __forceinline__ uint32_t lane_limit() const { return kSplatLaneLimit; }
    __device__ __forceinline__ int view_lo(int) const { return 0; }
    __device__ __forceinline__ int view_hi(int q) const { return s_dc[q].nr; }
};

// Candidate rr of segment e: its pixel, the test, and the depth-test atomic.
template <int S>
__device__ __forceinline__ void test_candidate(const DispConst& c, const SplatWarpSmem<S>& sm, const uint4& e,
                                               uint32_t rr, unsigned long long* keys, uint32_t npix,
                                               uint32_t& writes) {
    const float4* d = sm.pt[e.z >> 16];
    const float4 d0 = d[0], d1 = d[1], q2 = d[2], q3 = d[3], q4 = d[4], b = d[5];
    const uint32_t meta = __float_as_uint(d1.w), flags = meta >> 29;
    const uint32_t nx = e.y >> 14;
    // one row (most segments): no division
    const uint32_t ry = rr < nx ? 0u : div_floor(rr, nx);
    const int x = int(e.y & 0x3fffu) + int(rr - ry * nx), y = int(meta & 0x3fffu) + int(ry);
    const uint32_t vo = e.z & 0xffffu;
    const float Ex = __uint_as_float(e.w);
    const float qEx = Ex - d0.x, qEy = d0.y, qEz = d0.z;
    const float num = -dot3(q3.x, q3.y, q3.z, qEx, qEy, qEz);
    float t;
    if (!pixel_test(c, Ex, num, qEx, qEy, qEz, d1, q2, q3, q4, b.x, b.y, b.z, b.w, flags & kFlagInterior,
                    flags & kFlagDepthOk, x, y, t))
        return;
    if (!LFDPR_IN_BOUNDS(vo, c.nr, 10) || !LFDPR_IN_BOUNDS(uint32_t(x), c.W, 11) ||
        !LFDPR_IN_BOUNDS(uint32_t(y), c.H, 11))
        return;
    // a view holds at most 2^26 pixels: 32-bit offset within it
    atomicMin(keys + ((uint64_t)vo * npix + (uint32_t(y) * uint32_t(c.W) + uint32_t(x))),
              ((unsigned long long)__float_as_uint(t) << 32) | __float_as_uint(d0.w));
    writes++;
}

// The splat proper: warps stride through units 0 .. total-1 of `src` (a
// unit never spans two scenes).
template <int S, class Src>
__device__ __forceinline__ void splat_units(const Src& src, uint32_t total_units, SplatWarpSmem<S>& sm) {
    constexpr int P = UnitPairs<S>::P;
    const int lane = threadIdx.x & 31, sub = lane & 15, half = lane >> 4;
    const uint32_t lanes_below = (1u << lane) - 1u;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    uint32_t writes = 0;
    int cur = 0;

    for (uint32_t g = warp; g < total_units; g += n_warps) {
        const int sc = src.scene(g);
        if constexpr (Src::kMany) {
            if (sc != cur) {
                add_writes(src.ctr(cur), writes);
                writes = 0;
                cur = sc;
            }
        }
        const DispConst& c = src.dc(sc);
        const uint32_t n = src.points(sc);
        const WorkRec* work = src.work(sc);
        unsigned long long* keys = src.keys(sc);
        const uint32_t npix = uint32_t(c.W) * uint32_t(c.H);
        const uint32_t k0 = 2u * P * (g - src.first_unit(sc));   // the unit's first work point
        {
            const uint32_t kn = k0 + 2u * P * n_warps + uint32_t(lane);   // the next unit's records
            if (lane < 2 * P && kn < n) prefetch_l2(work + kn);
        }
        // the next unit's triangles (of one scene): read their ids now (the
        // work records were asked for a unit ago), ask L1 for their records'
        // 128-byte lines once this unit's candidates are formed, so that the
        // next unit's staging finds them there
        uint32_t next_tri = 0xffffffffu;
        if constexpr (!Src::kMany) {
            const uint32_t kn = k0 + 2u * P * n_warps + uint32_t(lane);
            if (lane < 2 * P && kn < n) next_tri = __ldg(&work[kn].meta.z);
        }
        const int vlo = src.view_lo(sc), vhi = src.view_hi(sc);
        for (int g0 = vlo; g0 < vhi; g0 += 16 * S) {
            __syncwarp();   // the previous passes are done with sm
            if (g0 == vlo) {
                // the unit's test constants, one float4 a lane: lane 6 q + f
                // stages float4 f of point k0 + q (a point past the end takes
                // the unit's first record; it has no rows)
                const int q = lane / 6, f = lane - 6 * q;
                if (q < 2 * P) {
                    const uint32_t k = k0 + uint32_t(q);
                    const uint4 meta = __ldg(&work[k < n ? k : k0].meta);
                    const TriRec* r = src.rec(sc) + meta.z;
                    float4 v = __ldg(&r->q[f < 5 ? f : 0]);
                    if (f == 0) {
                        v.y = 0.0f - v.y;
                        v.z = c.D - v.z;
                        v.w = __uint_as_float(meta.w);
                    } else if (f == 1) {
                        v.w = __uint_as_float(meta.x);
                    } else if (f == 5) {
                        const float sv = __ldg(&r->q[1].w);
                        const int i = int(meta.y & 0xffffu), j = int(meta.y >> 16);
                        v = make_float4(float(i) * v.w, float(i + 1) * v.w, float(j) * sv, float(j + 1) * sv);
                    }
                    sm.pt[q][f] = v;
                }
            }
            uint32_t pk[P][S], ny[P];
            float ex[S];   // the lane's views' eyes, the same for every pair
            uint32_t cnt = 0, nz = 0;   // the lane's candidates and non-empty (point, view) segments
#pragma unroll
            for (int p = 0; p < P; p++) {
                // a half past the end takes the unit's first record, with no rows
                const uint32_t k = k0 + 2u * p + uint32_t(half);
                const WorkRec* wr = work + (k < n ? k : k0);
                const float4 l0 = __ldg(&wr->L0), l1 = __ldg(&wr->L1);
                const uint4 meta = __ldg(&wr->meta);
                ny[p] = k < n ? (meta.x >> 14) & 0x7fffu : 0u;
                // branch-free: every slot computes its range, an empty or
                // absent one is masked to zero
#pragma unroll
                for (int sl = 0; sl < S; sl++) {
                    const int v = g0 + 16 * sl + sub;
                    if (p == 0) ex[sl] = src.eye(sc, v < vhi ? v : vlo);
                    const float Ex = ex[sl];
                    const float lo = fmaxf(fmaf(l0.y, Ex, l0.x), fmaf(l1.y, Ex, l1.x));
                    const float hi = fminf(fmaf(l0.w, Ex, l0.z), fmaf(l1.w, Ex, l1.z));
                    const int ix0 = max(__float2int_ru(lo), 0);
                    const int ix1 = min(__float2int_rd(hi), int(c.W) - 1);
                    const bool ok = v < vhi && ix0 <= ix1 && ny[p] > 0u;
                    const uint32_t nx = ok ? uint32_t(ix1 - ix0) + 1u : 0u;
                    pk[p][sl] = ok ? uint32_t(ix0) | (nx << 14) : 0u;
                    cnt += nx * ny[p];
                    nz += ok ? 1u : 0u;
                }
            }
            // a segment holds at most 2^26 candidates (one view), so lanes
            // below the limit (at most 2^24) keep the unit's numbering below 2^32
            const bool big = __any_sync(0xffffffffu, cnt >= src.lane_limit());
            // the unit's candidates and segments numbered in (lane, pair, slot)
            // order: one scan of both counts, the candidates in the high word
            // (wrapping as 32-bit sums would, only when the unit is walked)
            // and the segments (at most 32 S P) in the low one
            unsigned long long incl = ((unsigned long long)cnt << 32) | nz;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const unsigned long long all = __shfl_sync(0xffffffffu, incl, 31);
            const uint32_t total = uint32_t(all >> 32), nseg = uint32_t(all);
            uint32_t first = uint32_t(incl >> 32) - cnt, rank = uint32_t(incl) - nz;
#pragma unroll
            for (int p = 0; p < P; p++)
#pragma unroll
                for (int sl = 0; sl < S; sl++) {
                    const bool ok = pk[p][sl] != 0u;
                    if (ok)
                        sm.seg[rank] = make_uint4(first, pk[p][sl], uint32_t(g0 + 16 * sl + sub) | uint32_t(2 * p + half) << 16,
                                                  __float_as_uint(ex[sl]));
                    rank += ok ? 1u : 0u;
                    first += (pk[p][sl] >> 14) * ny[p];
                }
            if (next_tri != 0xffffffffu && g0 == vlo) prefetch_l1(src.rec(sc) + next_tri);
            __syncwarp();
            if (big) {
                // huge cells: each lane walks whole segments
                for (uint32_t s = uint32_t(lane); s < nseg; s += 32) {
                    const uint4 e = sm.seg[s];
                    const uint32_t ny = (__float_as_uint(sm.pt[e.z >> 16][1].w) >> 14) & 0x7fffu;
                    const uint32_t m = (e.y >> 14) * ny;
                    for (uint32_t rr = 0; rr < m; rr++) test_candidate<S>(c, sm, e, rr, keys, npix, writes);
                }
                continue;
            }
            uint32_t before = 0;   // segments starting before the pass
            for (uint32_t pass = 0; pass < total; pass += 32) {
                const uint32_t kw = before + uint32_t(lane);
                const uint32_t st = kw < nseg ? sm.seg[kw].x : 0xffffffffu;
                const uint32_t off = st - pass;   // starts from `before` on are >= pass
                const uint32_t smask = __reduce_or_sync(0xffffffffu, off < 32u ? 1u << off : 0u);
                const uint32_t own = before + uint32_t(__popc(smask & (lanes_below | (1u << lane)))) - 1u;
                before += uint32_t(__popc(smask));
                const uint32_t q = pass + uint32_t(lane);
                if (q < total) {
                    const uint4 e = sm.seg[own];
                    test_candidate<S>(c, sm, e, q - e.x, keys, npix, writes);
                }
            }
        }
    }
    add_writes(src.ctr(cur), writes);
}

template <int S>
__global__ void __launch_bounds__(kSplatWarps * 32, 4) k_splat(FrameArgs a) {
    wait_previous_kernel();
    allow_next_kernel();
    extern __shared__ __align__(16) uint8_t s_dyn[];
    __shared__ float s_ex[kMaxRenderViews];
    for (int v = threadIdx.x; v < a.dc.nr; v += blockDim.x) s_ex[v] = a.ex[v];
    __syncthreads();
    if (a.ctr->overflow) return;
    const uint32_t n = a.ctr->n_work;
    const OneScene src{a, n, uint32_t(__cvta_generic_to_shared(s_ex))};
    constexpr uint32_t unit = 2u * UnitPairs<S>::P;
    splat_units<S>(src, (n + unit - 1u) / unit, reinterpret_cast<SplatWarpSmem<S>*>(s_dyn)[threadIdx.x >> 5]);
}

// Every scene of a batch in one persistent launch: warps stride through the
// units of all scenes, so scenes of uneven size share the machine. Each block
// keeps every scene's display constants in shared memory.
template <int S>
__global__ void __launch_bounds__(kSplatWarps * 32, 4) k_splat_batch(const SplatScene* __restrict__ scenes,
                                                                     int n_scenes) {
    extern __shared__ __align__(16) uint8_t s_dyn[];
    __shared__ DispConst s_dc[kMaxBatchScenes];
    __shared__ uint32_t s_unit0[kMaxBatchScenes + 1];   // first unit of each scene
    __shared__ uint32_t s_n[kMaxBatchScenes];           // work points (0 after an overflow)
    constexpr uint32_t unit = 2u * UnitPairs<S>::P;
    for (int q = threadIdx.x; q < n_scenes; q += blockDim.x) {
        s_dc[q] = scenes[q].dc;
        const Counters* ct = scenes[q].ctr;
        s_n[q] = ct->overflow ? 0u : ct->n_work;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t u = 0;
        for (int q = 0; q < n_scenes; q++) {
            s_unit0[q] = u;
            u += (s_n[q] + unit - 1u) / unit;
        }
        s_unit0[n_scenes] = u;
    }
    __syncthreads();
    const ManyScenes src{scenes, n_scenes, s_dc, s_unit0, s_n};
    splat_units<S>(src, s_unit0[n_scenes], reinterpret_cast<SplatWarpSmem<S>*>(s_dyn)[threadIdx.x >> 5]);
}

// Eq. 8's interpolation weight for one view pixel whose depth test kept the
// point with resolve record (ra, rb): the splat's pixel area in view Ex is
// the shoelace area of its cell corners projected from the eye,
// |alpha + beta Ex| / 2. The colour it weights is held to the oracle within
// one level of 255, so both quotients take the hardware's approximate
// division (relative error near 1e-7: a colour moves by far less than a
// level, and changes level only where it lies within that of a rounding
// boundary); the divisors are at most 1 and a ratio of texture areas.
__device__ __forceinline__ float eq8_weight(float Ex, const float4& ra, const uint4& rb) {
    const float area_px = 0.5f * fabsf(fmaf(ra.y, Ex, ra.x));
    const float vmin = ra.w, vmax = __uint_as_float(rb.x);
    const float size_vse = __fdividef(ra.z, fminf(1.0f, area_px));
    const float size_vs = fminf(fmaxf(size_vse, vmin), vmax);
    return vmax > vmin ? __fdividef(size_vs - vmin, vmax - vmin) : 0.0f;
}

__device__ __forceinline__ uint32_t resolve_pixel(float Ex, const float4& ra, const uint4& rb) {
    const float w = eq8_weight(Ex, ra, rb);
    uint32_t out = 0u;
#pragma unroll
    for (int ch = 0; ch < 4; ch++) {
        const float lo = float((rb.y >> (8 * ch)) & 255u), hi = float((rb.z >> (8 * ch)) & 255u);
        out |= uint32_t(round_u8(fmaf(w, hi - lo, lo))) << (8 * ch);
    }
    return out;
}

// kResolvePix view pixels per thread, 256 apart (grid: pixel blocks x
// views): every key is loaded, then every winner's record, so each thread
// keeps that many dependent gathers in flight.
constexpr int kResolvePix = 2;
__global__ void __launch_bounds__(256) k_resolve(FrameArgs a) {
    wait_previous_kernel();
    allow_next_kernel();
    const DispConst& c = a.dc;
    const uint32_t npix = uint32_t(c.W) * uint32_t(c.H);
    const uint32_t p0 = blockIdx.x * (256u * kResolvePix) + threadIdx.x;
    const int v = a.view_lo + int(blockIdx.y);
    const uint64_t o0 = (uint64_t)v * npix;
    unsigned long long key[kResolvePix];
#pragma unroll
    for (int k = 0; k < kResolvePix; k++) {
        const uint32_t p = p0 + 256u * k;
        key[k] = p < npix ? a.keys[o0 + p] : ~0ull;
    }
    float4 ra[kResolvePix];
    uint4 rb[kResolvePix];
#pragma unroll
    for (int k = 0; k < kResolvePix; k++) {
        if (key[k] != ~0ull && !LFDPR_IN_BOUNDS(uint32_t(key[k]), a.max_points, 12)) key[k] = ~0ull;
        if (key[k] != ~0ull) {
            const ResolveRec* rp = a.rrec + uint32_t(key[k]);
            ra[k] = __ldg(&rp->a);
            rb[k] = __ldg(&rp->b);
        }
    }
    const float Ex = __ldg(a.ex + v);
#pragma unroll
    for (int k = 0; k < kResolvePix; k++) {
        const uint32_t p = p0 + 256u * k;
        if (p < npix && LFDPR_IN_BOUNDS(uint32_t(v), uint32_t(c.nr), 13))
            reinterpret_cast<uint32_t*>(a.views)[o0 + p] = key[k] != ~0ull ? resolve_pixel(Ex, ra[k], rb[k]) : 0u;
    }
}

// ---------------------------------------------------------------------------
// Physically based resolve of a mesh of materials
// ---------------------------------------------------------------------------

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float dot(const float3& a, const float3& b) {
    return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z));
}
// The shading runs in binary32 against a double-precision oracle with a
// tolerance of one level of 255, so it uses the hardware's approximate
// reciprocal square root and division (relative errors near 1e-7).
__device__ __forceinline__ float3 normalized(const float3& v) {
    const float l2 = dot(v, v);
    const float r = l2 > 0.0f ? rsqrtf(l2) : 0.0f;
    return l2 > 0.0f ? f3(v.x * r, v.y * r, v.z * r) : v;
}

// Outgoing linear RGB of one surface sample (unit n, v, l): metallic-roughness
// microfacet BRDF, GGX distribution D = a^2 / (pi ((n.h)^2 (a^2 - 1) + 1)^2),
// a = r^2 (r >= 0.045), Schlick-GGX visibility G1(x) = x / (x (1 - k) + k),
// k = (r + 1)^2 / 8, Schlick Fresnel F = F0 + (1 - F0)(1 - v.h)^5, F0 = 0.04
// (1 - m) + albedo m, diffuse (1 - F)(1 - m) albedo / pi:
//   rgb = (diffuse + D G F / (4 n.l n.v)) light n.l + ambient albedo.
__device__ __forceinline__ float3 pbr_shade(const float3& albedo, float rough, float metal, const float3& n,
                                            const float3& v, const float3& l, const Shading& sh) {
    const float3 h = normalized(f3(l.x + v.x, l.y + v.y, l.z + v.z));
    const float nl = fmaxf(dot(n, l), 0.0f), nv = fmaxf(dot(n, v), 1e-4f);
    const float nh = fmaxf(dot(n, h), 0.0f), vh = fmaxf(dot(v, h), 0.0f);
    const float r = fmaxf(rough, 0.045f);
    const float a = r * r, a2 = a * a;
    const float dn = fmaf(nh * nh, a2 - 1.0f, 1.0f);
    const float Dg = __fdividef(a2, 3.14159265358979f * dn * dn);
    const float k = (r + 1.0f) * (r + 1.0f) * 0.125f;
    const float G = __fdividef(nl, fmaf(nl, 1.0f - k, k)) * __fdividef(nv, fmaf(nv, 1.0f - k, k));
    const float om = 1.0f - vh;
    const float f5 = (om * om) * (om * om) * om;
    const float den = fmaxf(4.0f * nl * nv, 1e-4f);
    const float spec_dg = __fdividef(Dg * G, den);
    const float alb[3] = {albedo.x, albedo.y, albedo.z};
    float o[3];
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        const float F0 = fmaf(alb[ch], metal, 0.04f * (1.0f - metal));
        const float F = fmaf(1.0f - F0, f5, F0);
        const float diffuse = (1.0f - F) * (1.0f - metal) * alb[ch] * 0.318309886183791f;   // 1 / pi
        o[ch] = fmaf((diffuse + spec_dg * F) * sh.rgb[ch], nl, sh.amb[ch] * alb[ch]);
    }
    return f3(o[0], o[1], o[2]);
}

// One view pixel per thread: Eq. 8's weight as k_resolve; each map's value
// interpolated by Eq. 9 (unrounded); the surface point where the pixel
// centre's ray meets the triangle (the key's t: P = E + t (F - E)); the
// shading normal = the normal map's (2 c / 255 - 1) vector in the triangle's
// frame (tangent and bitangent = world directions of increasing s and t, from
// the inverse of the record's texture map over u-hat, v-hat; tangent made
// orthogonal to N, bitangent = N x T signed by the t direction), flipped when
// the triangle faces away from the eye; RGB = pbr_shade clamped, times 255,
// rounded half to even, alpha 255.
__global__ void __launch_bounds__(256) k_resolve_pbr(FrameArgs a) {
    wait_previous_kernel();
    allow_next_kernel();
    const DispConst& c = a.dc;
    const uint32_t npix = uint32_t(c.W) * uint32_t(c.H);
    const uint32_t px = blockIdx.x * blockDim.x + threadIdx.x;
    if (px >= npix) return;
    const int v = a.view_lo + int(blockIdx.y);
    const uint64_t o = (uint64_t)v * npix + px;
    unsigned long long key = a.keys[o];
    if (key != ~0ull && !LFDPR_IN_BOUNDS(uint32_t(key), a.max_points, 12)) key = ~0ull;
    uint32_t out = 0u;
    if (key != ~0ull) {
        const uint32_t p = uint32_t(key);
        const float t = __uint_as_float(uint32_t(key >> 32));
        const float Ex = __ldg(a.ex + v);
        const ResolveRec* rp = a.rrec + p;
        const float4 ra = __ldg(&rp->a);
        const uint4 rb = __ldg(&rp->b);
        const uint2 nm = __ldg(a.rmat + p);
        const float w = eq8_weight(Ex, ra, rb);
        auto lerp8 = [w](uint32_t lo, uint32_t hi, int ch) {
            const float a0 = float((lo >> (8 * ch)) & 255u), b0 = float((hi >> (8 * ch)) & 255u);
            return fmaf(w, b0 - a0, a0);
        };
        const float3 albedo = f3(lerp8(rb.y, rb.z, 0) * (1.0f / 255.0f), lerp8(rb.y, rb.z, 1) * (1.0f / 255.0f),
                                 lerp8(rb.y, rb.z, 2) * (1.0f / 255.0f));
        const float3 nt = f3(fmaf(lerp8(nm.x, nm.y, 0), 2.0f / 255.0f, -1.0f), fmaf(lerp8(nm.x, nm.y, 1), 2.0f / 255.0f, -1.0f),
                             fmaf(lerp8(nm.x, nm.y, 2), 2.0f / 255.0f, -1.0f));
        const uint32_t rm = rb.w;
        const float rough = fmaf(w, float((rm >> 8) & 255u) - float(rm & 255u), float(rm & 255u)) * (1.0f / 255.0f);
        const float metal =
            fmaf(w, float(rm >> 24) - float((rm >> 16) & 255u), float((rm >> 16) & 255u)) * (1.0f / 255.0f);
        // surface point and view direction
        const int x = int(px % uint32_t(c.W)), y = int(px / uint32_t(c.W));
        const float Fx = fmaf(float(x) + 0.5f, c.pw, c.x0), Fy = fmaf(float(y) + 0.5f, -c.ph, c.y0);
        const float3 P = f3(fmaf(t, Fx - Ex, Ex), t * Fy, fmaf(-t, c.D, c.D));
        const float3 V = normalized(f3(Ex - P.x, -P.y, c.D - P.z));
        // the triangle's shading frame
        const TriRec* r = a.rec + __ldg(&a.points[p].x);
        const float4 q1 = __ldg(&r->q[1]), q2 = __ldg(&r->q[2]), q3 = __ldg(&r->q[3]);
        const float4 q6 = __ldg(&r->q[6]), q7 = __ldg(&r->q[7]);
        const float3 N = f3(q3.x, q3.y, q3.z);
        const float gsu = q6.y, gsv = q6.z, gtu = q7.x, gtv = q7.y;
        const float det = fmaf(gsu, gtv, -(gsv * gtu));
        float dus = 1.0f, dvs = 0.0f, dut = 0.0f, dvt = 1.0f;
        if (det != 0.0f) {
            const float id = 1.0f / det;
            dus = gtv * id;
            dvs = -gtu * id;
            dut = -gsv * id;
            dvt = gsu * id;
        }
        const float3 ts = f3(fmaf(q1.x, dus, q2.x * dvs), fmaf(q1.y, dus, q2.y * dvs), fmaf(q1.z, dus, q2.z * dvs));
        const float3 tt = f3(fmaf(q1.x, dut, q2.x * dvt), fmaf(q1.y, dut, q2.y * dvt), fmaf(q1.z, dut, q2.z * dvt));
        const float dn = dot(ts, N);
        const float3 Tg = normalized(f3(fmaf(-N.x, dn, ts.x), fmaf(-N.y, dn, ts.y), fmaf(-N.z, dn, ts.z)));
        float3 Bt = f3(fmaf(N.y, Tg.z, -(N.z * Tg.y)), fmaf(N.z, Tg.x, -(N.x * Tg.z)), fmaf(N.x, Tg.y, -(N.y * Tg.x)));
        if (dot(Bt, tt) < 0.0f) Bt = f3(-Bt.x, -Bt.y, -Bt.z);
        float3 n = f3(fmaf(nt.x, Tg.x, fmaf(nt.y, Bt.x, nt.z * N.x)), fmaf(nt.x, Tg.y, fmaf(nt.y, Bt.y, nt.z * N.y)),
                      fmaf(nt.x, Tg.z, fmaf(nt.y, Bt.z, nt.z * N.z)));
        if (dot(n, n) == 0.0f) n = N;
        n = normalized(n);
        if (dot(N, V) < 0.0f) n = f3(-n.x, -n.y, -n.z);
        const float3 rgb = pbr_shade(albedo, rough, metal, n, V, f3(a.sh.l[0], a.sh.l[1], a.sh.l[2]), a.sh);
        out = 0xff000000u | (uint32_t(__float2uint_rn(__saturatef(rgb.x) * 255.0f))) |
              (uint32_t(__float2uint_rn(__saturatef(rgb.y) * 255.0f)) << 8) |
              (uint32_t(__float2uint_rn(__saturatef(rgb.z) * 255.0f)) << 16);
    }
    reinterpret_cast<uint32_t*>(a.views)[o] = out;
}

// Launch with the per-warp pooling buffers as dynamic shared memory (above
// 48 KB per block together with the static arrays only for the batched splat
// with 8 view slots, which opts in once).
template <int S>
cudaError_t splat_one(const FrameArgs& a, int grid, cudaStream_t s) {
    const size_t bytes = kSplatWarps * sizeof(SplatWarpSmem<S>);
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_splat<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (attr != cudaSuccess) return attr;
    return launch_after_previous(k_splat<S>, dim3(grid), dim3(kSplatWarps * 32), bytes, s, a);
}

template <int S>
cudaError_t splat_batch(const SplatScene* scenes, int n_scenes, int grid, cudaStream_t s) {
    const size_t bytes = kSplatWarps * sizeof(SplatWarpSmem<S>);
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_splat_batch<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (attr != cudaSuccess) return attr;
    k_splat_batch<S><<<grid, kSplatWarps * 32, bytes, s>>>(scenes, n_scenes);
    return cudaGetLastError();
}

}  // namespace

LFDPR_CHECK_READER(checks_splat)

cudaError_t launch_splat(const FrameArgs& a, cudaStream_t s) {
    // the fewest view slots per lane that hold every view of the range
    // [view_lo, view_hi) in one group (more than 128 views take several
    // groups of 128)
    const int nr = a.view_hi - a.view_lo, grid = a.sm_count * 16;
    if (nr <= 16) return splat_one<1>(a, grid, s);
    if (nr <= 32) return splat_one<2>(a, grid, s);
    if (nr <= 48) return splat_one<3>(a, grid, s);
    if (nr <= 64) return splat_one<4>(a, grid, s);
    if (nr <= 96) return splat_one<6>(a, grid, s);
    return splat_one<8>(a, grid, s);
}

cudaError_t launch_splat_batch(const SplatScene* scenes, int n_scenes, int slots, int grid_per_sm, int sm_count,
                               cudaStream_t s) {
    if (n_scenes < 1 || n_scenes > kMaxBatchScenes || grid_per_sm < 1) return cudaErrorInvalidValue;
    const int grid = sm_count * grid_per_sm;
    switch (slots) {
        case 1: return splat_batch<1>(scenes, n_scenes, grid, s);
        case 2: return splat_batch<2>(scenes, n_scenes, grid, s);
        case 3: return splat_batch<3>(scenes, n_scenes, grid, s);
        case 4: return splat_batch<4>(scenes, n_scenes, grid, s);
        case 6: return splat_batch<6>(scenes, n_scenes, grid, s);
        case 8: return splat_batch<8>(scenes, n_scenes, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_resolve(const FrameArgs& a, cudaStream_t s) {
    const uint32_t npix = uint32_t(a.dc.W) * uint32_t(a.dc.H);
    const uint32_t nv = uint32_t(a.view_hi - a.view_lo);
    const dim3 grid((npix + 255u) / 256u, nv);
    if (a.pbr) return launch_after_previous(k_resolve_pbr, grid, dim3(256), 0, s, a);
    return launch_after_previous(k_resolve, dim3((npix + 256u * kResolvePix - 1u) / (256u * kResolvePix), nv),
                                 dim3(256), 0, s, a);
}

}  // namespace lfdpr
