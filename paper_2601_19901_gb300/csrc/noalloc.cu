// lfdpr_sample_points_noalloc: the point-generation stage (per-triangle set-up
// and count, scan, emission) for callers that may not allocate device memory.
//
// Some callers cannot call cudaMalloc or any allocating routine once they are
// running: a real-time render loop that only allows allocation at start-up, a
// plug-in whose host application owns every device allocation and its memory
// budget, or code that runs while an allocator must not be entered. This
// entry point lets them generate a frame's point set from buffers they already
// own. Its scratch (triangle records, first-point offsets, block sums,
// counters, eye positions and texture sizes) is one file-scope __device__
// array of fixed size, which every GPU that loads the library keeps until the
// process exits. It runs the library's own set-up, scan and emission kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "lfdpr_internal.cuh"

using namespace lfdpr;

namespace {

constexpr uint32_t kNoAllocMaxTris = LFDPR_NOALLOC_MAX_TRIS;
constexpr uint32_t kNoAllocMaxTex = LFDPR_NOALLOC_MAX_TEX;
constexpr uint32_t kNoAllocBlocks = (kNoAllocMaxTris + kSetupThreads - 1) / kSetupThreads;

struct NoAllocScratch {
    TriRec rec[kNoAllocMaxTris];
    uint32_t offsets[kNoAllocMaxTris];
    uint32_t block_sums[kNoAllocBlocks];
    Counters ctr;
    float ex[kMaxRenderViews];
    TexDesc tex[kNoAllocMaxTex];
};

// The scratch. In host code this name is only a stand-in for the symbol, not
// a device address: the address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

// What a call writes into the scratch besides the kernels' own outputs: the
// eye positions and texture sizes, passed by value as one kernel parameter
// (8.2 KB; kernel parameters are copied when the launch is issued, so no host
// buffer has to outlive the call).
struct FillParams {
    float ex[kMaxRenderViews];
    TexDesc tex[kNoAllocMaxTex];
    int nr;
    uint32_t n_tex;
};
static_assert(sizeof(FillParams) < 32000, "kernel parameter limit");

// Clear the counters and store the eyes and texture sizes of one call.
__global__ void k_noalloc_fill(const __grid_constant__ FillParams p, NoAllocScratch* scr) {
    for (int k = threadIdx.x; k < p.nr; k += blockDim.x) scr->ex[k] = p.ex[k];
    for (uint32_t k = threadIdx.x; k < p.n_tex; k += blockDim.x) scr->tex[k] = p.tex[k];
    if (threadIdx.x == 0) scr->ctr = Counters{};
}

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
NoAllocScratch* g_scratch_ptr[kMaxDevices] = {};

lfdpr_status fail(lfdpr_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return s;
}

lfdpr_status cuda_fail(cudaError_t e, const char* what) {
    return fail(LFDPR_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CKN(call, what)                                      \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);   \
    } while (0)

}  // namespace

extern "C" lfdpr_status lfdpr_sample_points_noalloc(
    const lfdpr_display_desc* desc, const float model[16], const float* xyz, const float* uv,
    const uint32_t* idx, const uint32_t* tri_tex, uint32_t n_tris, const uint32_t* tex_wh,
    uint32_t n_tex, uint32_t* points, uint32_t max_points, uint32_t* counts, uint32_t* frame_counters,
    void* stream) {
    g_last_error[0] = 0;
    if (!desc || !model || !points || !counts || !frame_counters || !tex_wh)
        return fail(LFDPR_EINVAL, "sample_points_noalloc: null argument");
    if (n_tris > 0 && (!xyz || !uv || !idx || !tri_tex))
        return fail(LFDPR_EINVAL, "sample_points_noalloc: null mesh array");
    if (n_tris > kNoAllocMaxTris)
        return fail(LFDPR_EINVAL, "sample_points_noalloc: %u triangles exceed the fixed maximum of %u",
                    n_tris, kNoAllocMaxTris);
    if (n_tex == 0 || n_tex > kNoAllocMaxTex)
        return fail(LFDPR_EINVAL, "sample_points_noalloc: %u textures outside [1, %u]", n_tex, kNoAllocMaxTex);
    const lfdpr_display_desc& s = *desc;
    if (s.n_views < 1 || s.n_views > 256 || s.view_w < 1 || s.view_h < 1 || s.view_w > 16384 ||
        s.view_h > 16384 || !(s.view_dist > 0.0f) || !(s.focal_w > 0.0f) || !(s.focal_h > 0.0f) ||
        !(s.near_z > 0.0f) || !(s.far_z > s.near_z) || !std::isfinite(s.far_z) || !(s.cone_deg >= 0.0f) ||
        !(s.cone_deg < 179.0f) || !(s.bias_h > 0.0f) || !(s.bias_v > 0.0f) || !std::isfinite(s.bias_h) ||
        !std::isfinite(s.bias_v) || s.recon < 0 || s.recon > 3)
        return fail(LFDPR_EINVAL, "sample_points_noalloc: invalid display descriptor");
    for (int k = 0; k < 12; k++)
        if (!std::isfinite(model[k])) return fail(LFDPR_EINVAL, "sample_points_noalloc: non-finite model");
    for (uint32_t k = 0; k < n_tex; k++) {
        const uint32_t w = tex_wh[2 * k], h = tex_wh[2 * k + 1];
        if (!w || !h || (w & (w - 1)) || (h & (h - 1)) || w > 16384 || h > 16384)
            return fail(LFDPR_EINVAL, "sample_points_noalloc: texture %u size not a power of two <= 16384", k);
    }

    // one-time set-up per device: the scratch array's device address
    int dev = 0;
    CKN(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(LFDPR_EDEVICE, "sample_points_noalloc: device index too large");
    NoAllocScratch* scr = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
            g_scratch_ptr[dev] = static_cast<NoAllocScratch*>(p);
        }
        scr = g_scratch_ptr[dev];
    }
    int sms = 1;
    CKN(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "sm count");

    const bool ss = s.recon == 1 || s.recon == 2;   // angular supersampling: 2N views
    const int nr = ss ? 2 * s.n_views : s.n_views;
    FrameArgs a{};
    DispConst& c = a.dc;
    c.n_views = s.n_views;
    c.nr = nr;
    c.W = s.view_w;
    c.H = s.view_h;
    c.Wp = s.panel_w;
    c.Hp = s.panel_h;
    c.recon = s.recon;
    c.D = s.view_dist;
    c.fw2 = 0.5f * s.focal_w;
    c.fh2 = 0.5f * s.focal_h;
    c.near_z = s.near_z;
    c.far_z = s.far_z;
    c.bias_h = s.bias_h;
    c.bias_v = s.bias_v;
    c.px = float(double(s.focal_w) / (double(s.view_dist) * s.view_w));
    c.py = float(double(s.focal_h) / (double(s.view_dist) * s.view_h));
    c.pw = float(double(s.focal_w) / s.view_w);
    c.ph = float(double(s.focal_h) / s.view_h);
    c.ipw = float(double(s.view_w) / s.focal_w);
    c.iph = float(double(s.view_h) / s.focal_h);
    c.x0 = -0.5f * s.focal_w;
    c.y0 = 0.5f * s.focal_h;

    FillParams fp{};
    fp.nr = nr;
    fp.n_tex = n_tex;
    for (int k = 0; k < nr; k++)
        fp.ex[k] = float(double(s.view_dist) * std::tan(eye_angle_deg(s, k, 0.5) * M_PI / 180.0));
    for (uint32_t k = 0; k < n_tex; k++) {
        const uint32_t w = tex_wh[2 * k], h = tex_wh[2 * k + 1];
        uint32_t m = w > h ? w : h, l = 0;
        while ((1u << l) < m) l++;
        fp.tex[k].offset = 0;
        fp.tex[k].w = w;
        fp.tex[k].h = h;
        fp.tex[k].levels = l + 1;
        fp.tex[k].pad = 0;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_noalloc_fill<<<1, 256, 0, st>>>(fp, scr);
    CKN(cudaGetLastError(), "launch k_noalloc_fill");

    for (int k = 0; k < 12; k++) a.model[k] = model[k];
    a.ex = scr->ex;
    a.xyz = xyz;
    a.n_verts = 0xffffffffu;   // not known here: vertex indices are the caller's to keep in range
    a.uv = uv;
    a.idx = idx;
    a.tri_tex = tri_tex;
    a.tex = scr->tex;
    a.pool = nullptr;          // the fetch stage is not part of this entry point
    a.n_tris = n_tris;
    a.n_tex = n_tex;
    a.rec = scr->rec;
    a.counts = counts;
    a.offsets = scr->offsets;
    a.block_sums = scr->block_sums;
    a.n_blocks = (n_tris + kSetupThreads - 1) / kSetupThreads;
    a.points = reinterpret_cast<uint4*>(points);
    a.max_points = max_points;
    a.ctr = &scr->ctr;
    a.sm_count = sms;
    if (n_tris) {
        CKN(launch_setup(a, st), "launch k_setup");
        CKN(launch_scan(a, st), "launch k_scan");
        CKN(launch_emit(a, st), "launch k_emit");
    }
    CKN(cudaMemcpyAsync(frame_counters, &scr->ctr, 4 * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st),
        "copy counters");
    return LFDPR_OK;
}
