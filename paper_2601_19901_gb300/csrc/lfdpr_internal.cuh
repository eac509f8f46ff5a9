// Internal declarations of liblfdpr: device data layouts, the display
// constants every kernel reads, and the binary32 helpers of the bit-exact
// steps. Compiled with -fmad=false: the only fused multiply-adds are the
// explicit fmaf() calls, so every rounding below is the one written.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lfdpr.h"

namespace lfdpr {

constexpr int kMaxRenderViews = 512;
constexpr int kMaxCell = 65535;          // lattice indices are stored as u16
constexpr int kMaxLevels = 16;           // mip levels of a texture (16384 = 2^14 texels a side)
constexpr int kSetupThreads = 256;       // triangles per set-up / emit block
constexpr uint32_t kEmitBig = 128;       // points above which a triangle is emitted by a whole warp
constexpr float kBoxPad = 1.0f / 256.0f; // margin (pixels) of candidate pixel ranges against rounding
                                         // (projection error is about 1e-4 pixel)

// Display constants, passed by value to every kernel.
struct DispConst {
    int32_t n_views;      // display views N
    int32_t nr;           // rendered views (2N with angular supersampling)
    int32_t W, H;         // view pixels
    int32_t Wp, Hp;       // panel pixels
    int32_t recon;
    float D;              // eye-line distance
    float fw2, fh2;       // half focal rectangle
    float near_z, far_z;
    float bias_h, bias_v;
    float px, py;         // pixel footprint per unit distance (fw/(D W), fh/(D H))
    float pw, ph;         // pixel size on the focal plane (fw/W, fh/H)
    float ipw, iph;       // W/fw, H/fh
    float x0, y0;         // focal rectangle corner: -fw/2, fh/2
    float ex_max;         // largest |eye x| of the rendered views
    float inv_pitch, slant, phase_offset;
    float xtalk, xtalk_c; // crosstalk weight x and centre weight 1 - 2x
};

// Per-texture descriptor of the mip pool.
struct TexDesc {
    uint64_t offset;      // byte offset of level 0 in the pool
    uint32_t w, h;        // level-0 size (powers of two)
    uint32_t levels;      // number of levels (log2(max(w, h)) + 1)
    uint32_t pad;
};

// Device-side frame counters.
struct Counters {
    uint32_t n_points;
    uint32_t overflow;
    uint32_t cell_overflow;
    uint32_t n_live;
    uint32_t n_writes;    // depth-test atomics the splat issued
    uint32_t n_work;      // points with at least one candidate pixel row
    uint32_t n_near;      // points whose cell or triangle reaches within near_z of the eyes' plane
    uint32_t pad;
};

// One triangle's sampling record: 8 float4 (layout = LFDPR_TRI_* in lfdpr.h).
struct TriRec {
    float4 q[8];
};

// Projection of a world point C into every view (all eyes on y = 0, z = D):
// pixel x = A + B Ex, pixel y = Y, with s = D / (D - C.z), A = (C.x s - x0) W/fw,
// B = (1 - s) W/fw, Y = (y0 - C.y s) H/fh. The same formula for every point,
// so a vertex or cell corner shared by two primitives projects identically.
__device__ __forceinline__ void project_point(float D, float x0, float y0, float ipw, float iph,
                                              float X, float Y, float Z, float& A, float& B, float& Yp) {
    const float s = __fdividef(D, D - Z);
    A = fmaf(X, s, -x0) * ipw;
    B = (1.0f - s) * ipw;
    Yp = (y0 - Y * s) * iph;
}

// Per-triangle projection constants for the splat: the three vertices'
// (A, B, Y), and the triangle's z range.
struct TriProj {
    float4 a;   // A0 A1 A2 zmin
    float4 b;   // B0 B1 B2 zmax
    float4 y;   // Y0 Y1 Y2 (unused)
};

// Splat work record of a point with at least one candidate pixel row.
// Candidate rows are the pixel-centre rows inside both the cell's and the
// triangle's projected y-extent (the same in every view, since every eye lies
// on y = 0, z = D). L0 and L1 bound the x-extent, within that band of rows,
// of the projected cell (L0) and of the projected triangle (L1), each by a
// lower and an upper line x = a + b Ex valid for every eye, so a view's
// candidate columns lie between the larger lower and the smaller upper line
// (k_fetch's band_bounds). Written compacted by the fetch pass, in no
// particular order.
struct WorkRec {
    // lower a, b, upper a, b of the cell's (L0) and triangle's (L1) x-extent,
    // x = a + b Ex, less 1/2 + kBoxPad (lower) and 1/2 - kBoxPad (upper): the
    // candidate pixel columns are ceil(lower) .. floor(upper)
    float4 L0, L1;
    uint4 meta;   // y0 | n_rows << 14 | flags << 29, i | j << 16, triangle, point
};
// Per-point data of the resolve (Eq. 8-9): the splat's pixel area in view
// Ex is |alpha + beta Ex| / 2 (the shoelace sum of its cell's projected
// corners is affine in the eye's x, see k_fetch), the splat's texture area,
// the two Eq. 4-5 bounds and tv_min / tv_max; for a mesh of materials also
// the roughness and metallic tv_min / tv_max (R channels, bytes 0-3 of b.w).
// 32 bytes: one sector per gather.
struct ResolveRec {
    float4 a;     // alpha, beta, splat texture area, vpuv_min
    uint4 b;      // vpuv_max bits, tv_min RGBA8, tv_max RGBA8, roughness/metallic bytes (materials)
};

// Physically based shading of a mesh of materials: one directional light
// (unit direction toward the light, radiance) and an ambient term.
struct Shading {
    float l[3], rgb[3], amb[3];
};

// A live triangle's column summary: for a triangle of at most four lattice
// columns, word i holds column i's first row j0 | its row count << 16 (the
// words past the last column are left unwritten); a wider one holds
// kColSumWalk in word 0 (no column has j0 = rows = 65535, since j0 + rows <=
// kMaxCell + 1), and its points are found by walking the columns again.
constexpr uint32_t kColSumWalk = 0xffffffffu;
constexpr uint32_t kFlagInterior = 1u;  // the cell lies inside its triangle
constexpr uint32_t kFlagDepthOk = 2u;   // every hit on the triangle is within [near, far]

// ---------------------------------------------------------------------------
// binary32 helpers (each rounding explicit)
// ---------------------------------------------------------------------------

__device__ __forceinline__ float dot3(float ax, float ay, float az, float bx, float by, float bz) {
    return fmaf(ax, bx, fmaf(ay, by, az * bz));
}

// Doubled signed area of (p, r, q): edge function of p->r evaluated at q.
__device__ __forceinline__ float edge_fn(float px, float py, float rx, float ry, float qx, float qy) {
    return fmaf(rx - px, qy - py, -((ry - py) * (qx - px)));
}

// Reciprocal squared length of the segment p-r (0 for a zero-length segment).
__device__ __forceinline__ float seg_inv_len2(float px, float py, float rx, float ry) {
    const float ex = rx - px, ey = ry - py;
    const float ee = fmaf(ex, ex, ey * ey);
    return ee > 0.0f ? __fdiv_rn(1.0f, ee) : 0.0f;
}

// Squared distance from q to the segment p-r, inv_ee = seg_inv_len2(p, r):
// the closest point's parameter (q-p).(r-p) / |r-p|^2 clamped to [0, 1].
__device__ __forceinline__ float seg_dist2(float px, float py, float rx, float ry, float inv_ee, float qx,
                                           float qy) {
    const float ex = rx - px, ey = ry - py, wx = qx - px, wy = qy - py;
    float t = fmaf(wx, ex, wy * ey) * inv_ee;
    t = fminf(fmaxf(t, 0.0f), 1.0f);
    const float dx = fmaf(-t, ex, wx), dy = fmaf(-t, ey, wy);
    return fmaf(dx, dx, dy * dy);
}

__device__ __forceinline__ bool inside_either(float w0, float w1, float w2) {
    return (w0 >= 0.0f && w1 >= 0.0f && w2 >= 0.0f) || (w0 <= 0.0f && w1 <= 0.0f && w2 <= 0.0f);
}

// log2 by the atanh series (Eq. 6-7): x = m 2^e from the bits, m folded into
// [sqrt(1/2), sqrt(2)], ln m = 2 atanh(z) with z = (m-1)/(m+1) summed through
// the z^9/9 term, log2 x = e + ln m / ln 2.
__device__ __forceinline__ float log2_series(float x) {
    if (isnan(x)) return x;
    if (x <= 0.0f) return -INFINITY;
    if (isinf(x)) return INFINITY;
    uint32_t b = __float_as_uint(x);
    int e;
    if ((b >> 23) == 0u) {
        b = __float_as_uint(x * 16777216.0f);
        e = int(b >> 23) - 151;
    } else {
        e = int(b >> 23) - 127;
    }
    float m = __uint_as_float((b & 0x007fffffu) | 0x3f800000u);
    if (m > 1.41421356f) { m = m * 0.5f; e += 1; }
    const float z = __fdiv_rn(m - 1.0f, m + 1.0f);
    const float z2 = z * z;
    float s = fmaf(z2, (float)(1.0 / 9.0), (float)(1.0 / 7.0));   // atanh series coefficients
    s = fmaf(z2, s, (float)(1.0 / 5.0));
    s = fmaf(z2, s, (float)(1.0 / 3.0));
    s = fmaf(z2, s, 1.0f);
    const float ln_m = (2.0f * z) * s;
    return fmaf(ln_m, (float)(1.0 / 0.69314718055994530942), float(e));   // / ln 2
}

__device__ __forceinline__ uint8_t round_u8(float v) {
    float r = rintf(v);
    r = fminf(fmaxf(r, 0.0f), 255.0f);   // NaN -> 0 through fmaxf
    return (uint8_t)r;
}

// Angular supersampling renders 2N views (recon 1 and 2).
inline bool supersampled(const lfdpr_display_desc& d) { return d.recon == 1 || d.recon == 2; }

// Eye angle (degrees) of rendered view k at the fraction u of its interval
// (Sec. 3: N equal angular intervals of the cone; Sec. 4: 2N half-intervals
// with angular supersampling, where u = 1/2 puts the even ones on the N view
// centres). Host code; the eye x is D tan(angle), rounded once to binary32.
inline double eye_angle_deg(const lfdpr_display_desc& d, int k, double u) {
    const double cone = d.cone_deg;
    return supersampled(d) ? -cone / 2.0 + cone * (k + 0.5 + u) / (2.0 * d.n_views)
                           : -cone / 2.0 + cone * (k + u) / d.n_views;
}

// Index checks of the checked build (compiled with -DLFDPR_CHECKED=1 into
// liblfdpr_checked.so): LFDPR_IN_BOUNDS(i, n, site) is false when i >= n, and
// then records the first failing site (+1) and counts the failure in this
// translation unit's record, so that the caller skips the access instead of
// faulting. In the regular build it is `true` and costs nothing. Each .cu
// file that uses it defines its reader with LFDPR_CHECK_READER(name).
#ifdef LFDPR_CHECKED
static __device__ unsigned int g_check[2];
__device__ __forceinline__ bool check_index(uint64_t i, uint64_t n, unsigned site) {
    if (i < n) return true;
    atomicCAS(&g_check[0], 0u, site + 1u);
    atomicAdd(&g_check[1], 1u);
    return false;
}
#define LFDPR_IN_BOUNDS(i, n, site) (::lfdpr::check_index(uint64_t(i), uint64_t(n), (site)))
#define LFDPR_CHECK_READER(name)                                                          \
    cudaError_t name(unsigned out[2], bool reset) {                                       \
        cudaError_t e = cudaMemcpyFromSymbol(out, g_check, 2 * sizeof(unsigned));         \
        if (e == cudaSuccess && reset) {                                                   \
            const unsigned zero[2] = {0u, 0u};                                             \
            e = cudaMemcpyToSymbol(g_check, zero, sizeof zero);                            \
        }                                                                                  \
        return e;                                                                          \
    }
#else
#define LFDPR_IN_BOUNDS(i, n, site) true
#define LFDPR_CHECK_READER(name)                                                          \
    cudaError_t name(unsigned out[2], bool) {                                             \
        out[0] = out[1] = 0u;                                                              \
        return cudaSuccess;                                                                \
    }
#endif
// The checked build's records of sample.cu, splat.cu and interleave.cu.
cudaError_t checks_sample(unsigned out[2], bool reset);
cudaError_t checks_splat(unsigned out[2], bool reset);
cudaError_t checks_interleave(unsigned out[2], bool reset);

// Every device and pinned-host allocation of the library goes through these:
// they keep count of what is live (lfdpr_alloc_stats) and can be made to
// fail on purpose (lfdpr_fault_inject_alloc), as if memory had run out.
cudaError_t dev_malloc_raw(void** p, size_t bytes);
cudaError_t dev_malloc_async_raw(void** p, size_t bytes, cudaStream_t s);
cudaError_t host_malloc_raw(void** p, size_t bytes);
void dev_free(void* p);
void dev_free_async(void* p, cudaStream_t s);
void host_free(void* p);
template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
    return dev_malloc_raw(reinterpret_cast<void**>(p), bytes);
}
template <class T>
inline cudaError_t dev_malloc_async(T** p, size_t bytes, cudaStream_t s) {
    return dev_malloc_async_raw(reinterpret_cast<void**>(p), bytes, s);
}
template <class T>
inline cudaError_t host_malloc(T** p, size_t bytes) {
    return host_malloc_raw(reinterpret_cast<void**>(p), bytes);
}

// Per-thread description of the last error, read by lfdpr_last_error().
__attribute__((visibility("hidden"))) extern thread_local char g_last_error[512];

// ---------------------------------------------------------------------------
// Launchers (host side, defined next to their kernels)
// ---------------------------------------------------------------------------

struct FrameArgs {
    DispConst dc;
    const float* ex;                 // eye x per rendered view (device)
    float model[12];                 // affine rows of the model matrix
    const float* model_dev;          // if set, the 12 model values are read from here (device) instead
    const float* xyz;
    const float* uv;
    const uint32_t* idx;
    uint32_t n_verts;
    const uint32_t* tri_tex;         // texture per triangle, or material per triangle when mat_tex is set
    const uint4* mat_tex;            // null, or [materials] texture ids: albedo, normal, roughness, metallic
    int pbr;                         // shade physically (needs mat_tex)
    Shading sh;
    const TexDesc* tex;
    const uint8_t* pool;
    const uint64_t* lvl;             // [n_tex][kMaxLevels] byte offset of each mip level in the pool
    uint32_t n_tris, n_tex;
    uint32_t n_mat;                  // materials of a mesh of materials (0 otherwise)
    TriRec* rec;
    uint32_t* counts;
    uint32_t* offsets;
    uint4* colsum;                   // [n_tris] column summaries (k_setup -> k_emit); null: k_emit walks
    uint32_t* block_sums;            // [n_blocks]
    uint32_t n_blocks;
    uint4* points;
    uint32_t max_points;
    TriProj* tproj;                  // [n_tris] (optional: null skips it)
    WorkRec* work;                   // [max_points] the splat's work list
    uint32_t* near;                  // [max_points] points whose cell or triangle reaches within near_z of the eyes' plane
    ResolveRec* rrec;                // [max_points] per-point resolve data
    uint2* rmat;                     // [max_points] normal-map tv_min, tv_max (meshes of materials)
    uint64_t* keys;
    uint8_t* views;
    Counters* ctr;
    int sm_count;
    uint32_t splat_lane_limit;       // candidates per lane above which a splat unit is walked lane by lane
    int view_lo, view_hi;            // the rendered views [view_lo, view_hi) the splat and resolve cover
    int clear_keys;                  // k_fetch resets every view's keys after its points (else a memset does)
};
// The default splat_lane_limit: with every lane below 2^24 candidates a
// unit's candidate numbers stay below 2^32.
constexpr uint32_t kSplatLaneLimit = 1u << 24;

// Programmatic dependent launch. A kernel launched by launch_after_previous
// may be placed on the SMs while the kernel before it on the stream is still
// running, so its launch overlaps that kernel's last blocks. Each such kernel
// calls wait_previous_kernel() before it reads or writes anything: the wait
// returns once the previous kernel has finished and its writes are visible
// (at once after any other stream operation, or for a plain launch), so the
// stream's order holds as for a plain launch. allow_next_kernel() lets the
// kernel after it be placed early in turn.
__device__ __forceinline__ void wait_previous_kernel() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Ask L2 (L1) for the line holding p (no register result).
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }
__device__ __forceinline__ void allow_next_kernel() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename... P, typename... A>
cudaError_t launch_after_previous(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                  A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...);
}

cudaError_t launch_setup(const FrameArgs& a, cudaStream_t s);
// The depth-guided warp of nin rendered views (RGBA8 and depth keys) to nout
// eyes on the same eye line (warp.cu); views at most kMaxWarpWidth wide.
constexpr int kMaxWarpWidth = 4032;   // the warp block's shared memory: 56 bytes a pixel at the widest
cudaError_t launch_warp_views(const uint8_t* views, const uint64_t* keys, const float* in_eyes, int nin,
                              const float* out_eyes, int nout, int W, int H, float ipw, uint8_t* out,
                              cudaStream_t s);
cudaError_t launch_scan(const FrameArgs& a, cudaStream_t s);
cudaError_t launch_emit(const FrameArgs& a, cudaStream_t s);
cudaError_t launch_fetch(const FrameArgs& a, cudaStream_t s);
cudaError_t launch_fetch_mat(const FrameArgs& a, cudaStream_t s);   // meshes of materials, after launch_fetch
cudaError_t launch_near_work(const FrameArgs& a, cudaStream_t s);   // after launch_fetch
cudaError_t launch_splat(const FrameArgs& a, cudaStream_t s);

// One scene of a batched splat: its display constants and the buffers the
// splat reads and writes.
struct SplatScene {
    DispConst dc;
    const float* ex;
    Counters* ctr;
    const WorkRec* work;
    const TriRec* rec;
    uint64_t* keys;
};
constexpr int kMaxBatchScenes = 64;
constexpr int kMaxBatchViews = 4096;   // rendered views summed over a batch
// Splat every scene of a batch in one persistent launch: grid_per_sm blocks
// per SM, slots view slots per lane (1, 2, 3, 4, 6 or 8).
cudaError_t launch_splat_batch(const SplatScene* scenes, int n_scenes, int slots, int grid_per_sm, int sm_count,
                               cudaStream_t s);
cudaError_t launch_resolve(const FrameArgs& a, cudaStream_t s);
// pos [nr] (views on the display-view axis) and samples [n_samples][3] are
// read only for Gaussian reconstruction (recon 2, 3).
cudaError_t launch_interleave(const DispConst& dc, const uint8_t* views, const float* pos, const float* samples,
                              int n_samples, uint8_t* panel, cudaStream_t s);
// Mip level `level` (1 or 2) of nr views of W x H RGBA8 into out.
cudaError_t launch_view_mip(const uint8_t* views, int W, int H, int nr, int level, uint8_t* out, cudaStream_t s);
cudaError_t launch_mip_level(const uint8_t* src, uint32_t sw, uint32_t sh, uint8_t* dst,
                             uint32_t dw, uint32_t dh, cudaStream_t s);
// mode 0: random global, 1: shared memory, 2: warp-coherent global
cudaError_t launch_probe_atomic(uint64_t* words, uint64_t n_words, const uint32_t* idx,
                                const uint64_t* val, uint64_t n_ops, int mode, int sm_count,
                                cudaStream_t s);

}  // namespace lfdpr
