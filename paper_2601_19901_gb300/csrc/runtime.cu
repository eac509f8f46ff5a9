// C ABI of liblfdpr (declared in include/lfdpr.h): display and mesh objects,
// device allocation, argument validation, and the per-frame launch sequence.
// Host arithmetic that feeds the kernels' bit-exact steps (eye positions,
// pixel footprints) is done in double and rounded once to binary32; this file
// is compiled with -ffp-contract=off so no host multiply-add is fused.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <unordered_map>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "objects.h"

using namespace lfdpr;

namespace lfdpr {
thread_local char g_last_error[512] = "";

namespace {
std::mutex g_alloc_mu;
std::unordered_map<void*, size_t> g_live;     // what the library holds: address -> bytes
int64_t g_live_bytes = 0, g_allocs = 0;
std::atomic<int64_t> g_fail_after{-1};        // the allocation this many from now fails (-1: none)

// Whether this allocation is the one armed to fail (disarms once it fires).
bool fail_now() {
    int64_t v = g_fail_after.load();
    while (v >= 0)
        if (g_fail_after.compare_exchange_weak(v, v - 1)) return v == 0;
    return false;
}

void keep(void* p, size_t bytes) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    g_live[p] = bytes;
    g_live_bytes += int64_t(bytes);
    g_allocs++;
}

bool drop(void* p) {
    if (!p) return false;
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    auto it = g_live.find(p);
    if (it == g_live.end()) return false;
    g_live_bytes -= int64_t(it->second);
    g_live.erase(it);
    return true;
}
}  // namespace

cudaError_t dev_malloc_raw(void** p, size_t bytes) {
    *p = nullptr;
    if (fail_now()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) keep(*p, bytes);
    return e;
}

cudaError_t dev_malloc_async_raw(void** p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (fail_now()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e == cudaSuccess) keep(*p, bytes);
    return e;
}

cudaError_t host_malloc_raw(void** p, size_t bytes) {
    *p = nullptr;
    if (fail_now()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocHost(p, bytes);
    if (e == cudaSuccess) keep(*p, bytes);
    return e;
}

void dev_free(void* p) {
    if (drop(p)) cudaFree(p);
}

void dev_free_async(void* p, cudaStream_t s) {
    if (drop(p)) cudaFreeAsync(p, s);
}

void host_free(void* p) {
    if (drop(p)) cudaFreeHost(p);
}

lfdpr_status fail(lfdpr_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return s;
}

lfdpr_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? LFDPR_ENOMEM : LFDPR_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

FrameArgs frame_args(const lfdpr_display* disp, const lfdpr_mesh* mesh) {
    FrameArgs a{};
    a.dc = disp->dc;
    a.ex = disp->d_ex;
    a.xyz = mesh->xyz;
    a.n_verts = mesh->n_verts;
    a.uv = mesh->uv;
    a.idx = mesh->idx;
    a.tri_tex = mesh->tri_tex;
    a.mat_tex = mesh->mat_tex;
    a.pbr = mesh->mat_tex != nullptr && disp->shading == LFDPR_SHADING_PBR;
    a.sh = disp->sh;
    a.tex = mesh->tex;
    a.pool = mesh->pool;
    a.lvl = mesh->lvl;
    a.n_tris = mesh->n_tris;
    a.n_tex = mesh->n_tex;
    a.n_mat = mesh->n_mat;
    a.rec = mesh->rec;
    a.counts = mesh->counts;
    a.offsets = mesh->offsets;
    a.colsum = mesh->colsum;
    a.block_sums = mesh->block_sums;
    a.n_blocks = mesh->n_blocks;
    a.points = disp->points;
    a.max_points = disp->max_points;
    a.tproj = mesh->tproj;
    a.work = disp->work;
    a.near = disp->near;
    a.rrec = disp->rrec;
    a.rmat = disp->rmat;
    a.keys = disp->keys;
    a.views = disp->views;
    a.ctr = disp->ctr;
    a.sm_count = disp->sm_count;
    a.splat_lane_limit = disp->splat_lane_limit;
    a.view_lo = 0;
    a.view_hi = disp->dc.nr;
    return a;
}

lfdpr_status record_frame_front(lfdpr_display* disp, lfdpr_mesh* mesh, const FrameArgs& a_in, cudaStream_t s,
                                bool marks, bool clear_keys) {
    // with triangles to sample, k_fetch clears the keys after its points;
    // without, a memset does
    FrameArgs a = a_in;
    a.clear_keys = clear_keys && mesh->n_tris ? 1 : 0;
    auto mk = [&](int k) {
        if (marks) cudaEventRecord(disp->ev[k], s);
    };
    const uint64_t npix = uint64_t(disp->dc.W) * disp->dc.H * disp->dc.nr;
#define CKF(call, what)                                      \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);   \
    } while (0)
    CKF(cudaMemsetAsync(disp->ctr, 0, sizeof(Counters), s), "reset counters");
    mk(0);
    if (mesh->n_tris) {
        CKF(launch_setup(a, s), "launch k_setup");
        mk(1);
        CKF(launch_scan(a, s), "launch k_scan");
        mk(2);
        CKF(launch_emit(a, s), "launch k_emit");
        mk(3);
        CKF(launch_fetch(a, s), "launch k_fetch");
        CKF(launch_near_work(a, s), "launch k_near_work");
        disp->launches += 5;
        if (a.mat_tex) {
            CKF(launch_fetch_mat(a, s), "launch k_fetch_mat");
            disp->launches += 1;
        }
    } else {
        for (int k = 1; k <= 3; k++) mk(k);
    }
    mk(4);
    if (clear_keys && !a.clear_keys) CKF(cudaMemsetAsync(disp->keys, 0xff, 8u * npix, s), "clear keys");
    mk(5);
#undef CKF
    return LFDPR_OK;
}

lfdpr_status record_interleave(lfdpr_display* disp, uint8_t* panel, cudaStream_t s) {
    DispConst dc = disp->dc;
    const uint8_t* views = disp->views;
    if (disp->ss_level > 0) {
        const cudaError_t e = launch_view_mip(disp->views, dc.W, dc.H, dc.nr, disp->ss_level, disp->views_mip, s);
        if (e != cudaSuccess) return cuda_fail(e, "launch k_view_mip");
        disp->launches += 1;
        dc.W >>= disp->ss_level;
        dc.H >>= disp->ss_level;
        views = disp->views_mip;
    }
    const cudaError_t e = launch_interleave(dc, views, disp->d_pos, disp->d_samples, disp->n_samples, panel, s);
    if (e != cudaSuccess) return cuda_fail(e, "launch k_interleave");
    disp->launches += 1;
    return LFDPR_OK;
}
}  // namespace lfdpr

namespace {

#define g_err lfdpr::g_last_error

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

bool pow2(uint32_t v) { return v && !(v & (v - 1)); }

uint32_t mip_levels(uint32_t w, uint32_t h) {
    uint32_t m = w > h ? w : h, l = 0;
    while ((1u << l) < m) l++;
    return l + 1;
}

uint64_t mip_bytes(uint32_t w, uint32_t h) {
    uint64_t n = 0;
    const uint32_t L = mip_levels(w, h);
    for (uint32_t l = 0; l < L; l++) {
        const uint64_t lw = (w >> l) ? (w >> l) : 1, lh = (h >> l) ? (h >> l) : 1;
        n += lw * lh * 4u;
    }
    return n;
}

void free_display(lfdpr_display* d) {
    if (!d) return;
    for (auto& e : d->ev)
        if (e) cudaEventDestroy(e);
    for (auto& e : d->band_ev)
        if (e) cudaEventDestroy(e);
    dev_free(d->d_ex);
    dev_free(d->d_pos);
    dev_free(d->d_samples);
    dev_free(d->points);
    dev_free(d->work);
    dev_free(d->near);
    dev_free(d->rrec);
    dev_free(d->rmat);
    dev_free(d->keys);
    dev_free(d->views);
    dev_free(d->panel);
    dev_free(d->views_mip);
    dev_free(d->ctr);
    delete d;
}

void free_mesh(lfdpr_mesh* m) {
    if (!m) return;
    dev_free(m->xyz);
    dev_free(m->uv);
    dev_free(m->idx);
    dev_free(m->tri_tex);
    dev_free(m->mat_tex);
    if (m->owns_textures) {
        dev_free(m->pool);
        dev_free(m->tex);
        dev_free(m->lvl);
    }
    dev_free(m->rec);
    dev_free(m->tproj);
    dev_free(m->counts);
    dev_free(m->offsets);
    dev_free(m->colsum);
    dev_free(m->block_sums);
    delete m;
}

// Eyes, their largest |x| and the views' positions on the display-view axis
// from the display's jitter (host copies; the device copies follow).
void place_eyes(lfdpr_display* d) {
    const int nr = d->dc.nr;
    d->h_ex.resize(nr);
    for (int k = 0; k < nr; k++)
        d->h_ex[k] = float(double(d->desc.view_dist) * std::tan(eye_angle_deg(d->desc, k, d->h_jit[k]) * M_PI / 180.0));
    d->dc.ex_max = 0.0f;
    for (int k = 0; k < nr; k++) d->dc.ex_max = std::fmax(d->dc.ex_max, std::fabs(d->h_ex[k]));
}

std::vector<float> view_positions(const lfdpr_display* d) {
    const int nr = d->dc.nr;
    std::vector<float> pos(nr);
    for (int m = 0; m < nr; m++)
        pos[m] = supersampled(d->desc) ? float((m + 0.5 + double(d->h_jit[m])) / 2.0) : float(m + double(d->h_jit[m]));
    return pos;
}

// Validate and upload n_tex textures with their mip chains into one pool.
// On success the caller owns *pool, *tex, *lvl; on failure nothing is left.
lfdpr_status upload_textures(const uint8_t* const* tex_rgba8, const uint32_t* tex_wh, uint32_t n_tex,
                             cudaStream_t s, uint8_t** pool_out, TexDesc** tex_out, uint64_t** lvl_out) {
    if (n_tex == 0 || !tex_rgba8 || !tex_wh) return fail(LFDPR_EINVAL, "textures: need >= 1 texture");
    std::vector<TexDesc> td(n_tex);
    std::vector<uint64_t> lvl((size_t)n_tex * kMaxLevels, 0);
    uint64_t pool_bytes = 0;
    for (uint32_t k = 0; k < n_tex; k++) {
        const uint32_t w = tex_wh[2 * k], h = tex_wh[2 * k + 1];
        if (!pow2(w) || !pow2(h) || w > 16384 || h > 16384)
            return fail(LFDPR_EINVAL, "textures: texture %u size %ux%u not a power of two <= 16384", k, w, h);
        if (!tex_rgba8[k]) return fail(LFDPR_EINVAL, "textures: null texture %u", k);
        td[k].offset = pool_bytes;
        td[k].w = w;
        td[k].h = h;
        td[k].levels = mip_levels(w, h);
        td[k].pad = 0;
        uint64_t off = pool_bytes;
        for (uint32_t l = 0; l < td[k].levels; l++) {
            lvl[(size_t)k * kMaxLevels + l] = off;
            const uint64_t lw = (w >> l) ? (w >> l) : 1, lh = (h >> l) ? (h >> l) : 1;
            off += lw * lh * 4u;
        }
        pool_bytes += (mip_bytes(w, h) + 255) & ~uint64_t(255);
    }
    uint8_t* pool = nullptr;
    TexDesc* tex = nullptr;
    uint64_t* dl = nullptr;
    auto undo = [&]() {
        dev_free(pool);
        dev_free(tex);
        dev_free(dl);
    };
    cudaError_t e;
    if ((e = dev_malloc(&pool, pool_bytes)) != cudaSuccess ||
        (e = dev_malloc(&tex, sizeof(TexDesc) * n_tex)) != cudaSuccess ||
        (e = dev_malloc(&dl, sizeof(uint64_t) * kMaxLevels * n_tex)) != cudaSuccess) {
        undo();
        return cuda_fail(e, "textures: allocation");
    }
#define CKT(call, what)                 \
    do {                                \
        cudaError_t e_ = (call);        \
        if (e_ != cudaSuccess) {        \
            undo();                     \
            return cuda_fail(e_, what); \
        }                               \
    } while (0)
    CKT(cudaMemcpyAsync(tex, td.data(), sizeof(TexDesc) * n_tex, cudaMemcpyHostToDevice, s), "upload tex table");
    CKT(cudaMemcpyAsync(dl, lvl.data(), sizeof(uint64_t) * kMaxLevels * n_tex, cudaMemcpyHostToDevice, s),
        "upload level offsets");
    for (uint32_t k = 0; k < n_tex; k++) {
        uint32_t w = td[k].w, h = td[k].h;
        uint8_t* cur = pool + td[k].offset;
        CKT(cudaMemcpyAsync(cur, tex_rgba8[k], 4u * (uint64_t)w * h, cudaMemcpyHostToDevice, s), "upload texels");
        for (uint32_t l = 1; l < td[k].levels; l++) {
            const uint32_t nw = w > 1 ? w / 2 : 1, nh = h > 1 ? h / 2 : 1;
            uint8_t* nxt = cur + 4u * (uint64_t)w * h;
            CKT(launch_mip_level(cur, w, h, nxt, nw, nh, s), "mip build");
            cur = nxt;
            w = nw;
            h = nh;
        }
    }
    CKT(cudaStreamSynchronize(s), "textures: synchronize");
#undef CKT
    *pool_out = pool;
    *tex_out = tex;
    *lvl_out = dl;
    return LFDPR_OK;
}

// Validate a mesh's geometry against n_tex textures and upload it into a new
// mesh object whose textures are not yet set. On success *out is the mesh.
lfdpr_status upload_geometry(lfdpr_display* disp, const float* xyz, const float* uv, const uint32_t* idx,
                             const uint32_t* tri_tex, uint32_t n_verts, uint32_t n_tris, uint32_t n_tex,
                             cudaStream_t s, lfdpr_mesh** out) {
    if (n_tris > 0 && (!xyz || !uv || !idx || !tri_tex)) return fail(LFDPR_EINVAL, "upload_mesh: null array");
    if (n_tris > (1u << 30)) return fail(LFDPR_EINVAL, "upload_mesh: too many triangles");
    for (uint64_t k = 0; k < 3ull * n_tris; k++)
        if (idx[k] >= n_verts)
            return fail(LFDPR_EINVAL, "upload_mesh: index %u out of range at %llu", idx[k], (unsigned long long)k);
    for (uint32_t t = 0; t < n_tris; t++)
        if (tri_tex[t] >= n_tex) return fail(LFDPR_EINVAL, "upload_mesh: texture id out of range at triangle %u", t);
    for (uint64_t k = 0; k < 3ull * n_verts; k++)
        if (!std::isfinite(xyz[k])) return fail(LFDPR_EINVAL, "upload_mesh: non-finite vertex coordinate");
    for (uint64_t k = 0; k < 2ull * n_verts; k++)
        if (!std::isfinite(uv[k])) return fail(LFDPR_EINVAL, "upload_mesh: non-finite texture coordinate");
    lfdpr_mesh* m = new (std::nothrow) lfdpr_mesh();
    if (!m) return fail(LFDPR_ENOMEM, "host allocation failed");
    m->disp = disp;
    m->n_verts = n_verts;
    m->n_tris = n_tris;
    m->n_tex = n_tex;
    m->n_blocks = (n_tris + kSetupThreads - 1) / kSetupThreads;
    const uint64_t nt = n_tris ? n_tris : 1, nv = n_verts ? n_verts : 1;
    cudaError_t e;
    if ((e = dev_malloc(&m->xyz, 12u * nv)) != cudaSuccess || (e = dev_malloc(&m->uv, 8u * nv)) != cudaSuccess ||
        (e = dev_malloc(&m->idx, 12u * nt)) != cudaSuccess || (e = dev_malloc(&m->tri_tex, 4u * nt)) != cudaSuccess ||
        (e = dev_malloc(&m->rec, sizeof(TriRec) * nt)) != cudaSuccess ||
        (e = dev_malloc(&m->tproj, sizeof(TriProj) * nt)) != cudaSuccess ||
        (e = dev_malloc(&m->counts, 4u * nt)) != cudaSuccess || (e = dev_malloc(&m->offsets, 4u * nt)) != cudaSuccess ||
        (e = dev_malloc(&m->colsum, sizeof(uint4) * nt)) != cudaSuccess ||
        (e = dev_malloc(&m->block_sums, 4u * (m->n_blocks ? m->n_blocks : 1))) != cudaSuccess) {
        free_mesh(m);
        return cuda_fail(e, "upload_mesh: allocation");
    }
#define CKM(call, what)                 \
    do {                                \
        cudaError_t e_ = (call);        \
        if (e_ != cudaSuccess) {        \
            free_mesh(m);               \
            return cuda_fail(e_, what); \
        }                               \
    } while (0)
    if (n_verts) {
        CKM(cudaMemcpyAsync(m->xyz, xyz, 12u * (uint64_t)n_verts, cudaMemcpyHostToDevice, s), "upload xyz");
        CKM(cudaMemcpyAsync(m->uv, uv, 8u * (uint64_t)n_verts, cudaMemcpyHostToDevice, s), "upload uv");
    }
    if (n_tris) {
        CKM(cudaMemcpyAsync(m->idx, idx, 12u * (uint64_t)n_tris, cudaMemcpyHostToDevice, s), "upload idx");
        CKM(cudaMemcpyAsync(m->tri_tex, tri_tex, 4u * (uint64_t)n_tris, cudaMemcpyHostToDevice, s), "upload tri_tex");
    }
    CKM(cudaStreamSynchronize(s), "upload_mesh: synchronize");
#undef CKM
    *out = m;
    return LFDPR_OK;
}

void mark(lfdpr_display* d, int k, cudaStream_t s) {
    if (d->timing) cudaEventRecord(d->ev[k], s);
}

}  // namespace

extern "C" {

const char* lfdpr_last_error(void) { return g_err; }

lfdpr_status lfdpr_fault_inject_alloc(int64_t after) {
    g_err[0] = 0;
    if (after < -1) return fail(LFDPR_EINVAL, "fault_inject_alloc: %lld < -1", (long long)after);
    lfdpr::g_fail_after.store(after);
    return LFDPR_OK;
}

lfdpr_status lfdpr_checked_status(uint32_t* first_site, uint64_t* failures, int32_t reset) {
    g_err[0] = 0;
#ifndef LFDPR_CHECKED
    (void)first_site;
    (void)failures;
    (void)reset;
    return fail(LFDPR_EINVAL, "checked_status: not the checked build (liblfdpr_checked.so)");
#else
    CK(cudaDeviceSynchronize(), "checked_status: synchronize");
    cudaError_t (*readers[3])(unsigned[2], bool) = {lfdpr::checks_sample, lfdpr::checks_splat,
                                                   lfdpr::checks_interleave};
    uint32_t site = 0;
    uint64_t n = 0;
    for (auto rd : readers) {
        unsigned r[2];
        CK(rd(r, reset != 0), "checked_status: read");
        if (!site && r[0]) site = r[0];
        n += r[1];
    }
    if (first_site) *first_site = site;
    if (failures) *failures = n;
    return LFDPR_OK;
#endif
}

lfdpr_status lfdpr_alloc_stats(int64_t* live_count, int64_t* live_bytes, int64_t* total_count) {
    g_err[0] = 0;
    std::lock_guard<std::mutex> lock(lfdpr::g_alloc_mu);
    if (live_count) *live_count = int64_t(lfdpr::g_live.size());
    if (live_bytes) *live_bytes = lfdpr::g_live_bytes;
    if (total_count) *total_count = lfdpr::g_allocs;
    return LFDPR_OK;
}

int32_t lfdpr_version(void) { return LFDPR_VERSION; }

lfdpr_status lfdpr_create_display(const lfdpr_display_desc* desc, lfdpr_display** out) {
    g_err[0] = 0;
    if (!desc || !out) return fail(LFDPR_EINVAL, "create_display: null argument");
    *out = nullptr;
    const lfdpr_display_desc& s = *desc;
    if (s.n_views < 1 || s.n_views > 256) return fail(LFDPR_EINVAL, "n_views must be in [1, 256]");
    if (s.view_w < 1 || s.view_h < 1 || s.view_w > 16384 || s.view_h > 16384 ||
        (int64_t)s.view_w * s.view_h > (1LL << 26))
        return fail(LFDPR_EINVAL, "view size must be in [1, 16384] with at most 2^26 pixels");
    if (s.panel_w < 1 || s.panel_h < 1 || s.panel_w > 32768 || s.panel_h > 32768)
        return fail(LFDPR_EINVAL, "panel size must be in [1, 32768]");
    if (!(s.view_dist > 0.0f) || !(s.focal_w > 0.0f) || !(s.focal_h > 0.0f))
        return fail(LFDPR_EINVAL, "view_dist, focal_w, focal_h must be positive");
    if (!(s.near_z > 0.0f) || !(s.far_z > s.near_z) || !std::isfinite(s.far_z))
        return fail(LFDPR_EINVAL, "need 0 < near_z < far_z < inf");
    if (!(s.cone_deg >= 0.0f) || !(s.cone_deg < 179.0f)) return fail(LFDPR_EINVAL, "cone_deg must be in [0, 179)");
    if (!(s.bias_h > 0.0f) || !(s.bias_v > 0.0f) || !std::isfinite(s.bias_h) || !std::isfinite(s.bias_v))
        return fail(LFDPR_EINVAL, "bias_h, bias_v must be positive and finite");
    if (!(s.lens_pitch_px > 0.0f) || !std::isfinite(s.slant) || !std::isfinite(s.phase_offset))
        return fail(LFDPR_EINVAL, "lens_pitch_px must be positive; slant, phase_offset finite");
    if (s.recon < 0 || s.recon > 3) return fail(LFDPR_EINVAL, "recon must be 0, 1, 2 or 3");
    if (!(s.crosstalk >= 0.0f) || !(s.crosstalk < 0.5f)) return fail(LFDPR_EINVAL, "crosstalk must be in [0, 0.5)");
    if (s.max_points < 0 || s.max_points > 0x7fffffffLL) return fail(LFDPR_EINVAL, "max_points must be in [0, 2^31)");
    const int nr = supersampled(s) ? 2 * s.n_views : s.n_views;
    if (nr > kMaxRenderViews) return fail(LFDPR_EINVAL, "too many rendered views");

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(LFDPR_EDEVICE, "no CUDA device");
    }
    lfdpr_display* d = new (std::nothrow) lfdpr_display();
    if (!d) return fail(LFDPR_ENOMEM, "host allocation failed");
    d->desc = s;
    if (d->desc.max_points == 0) d->desc.max_points = 1LL << 23;
    d->max_points = uint32_t(d->desc.max_points);
    CK(cudaGetDevice(&d->device), "cudaGetDevice");
    CK(cudaDeviceGetAttribute(&d->sm_count, cudaDevAttrMultiProcessorCount, d->device), "sm count");

    DispConst& c = d->dc;
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
    c.inv_pitch = float(1.0 / double(s.lens_pitch_px));
    c.slant = s.slant;
    c.phase_offset = s.phase_offset;
    c.xtalk = s.crosstalk;
    c.xtalk_c = float(1.0 - 2.0 * double(s.crosstalk));

    d->h_jit.assign(nr, 0.5f);
    place_eyes(d);

    const uint64_t npix = uint64_t(s.view_w) * s.view_h * nr;
    cudaError_t e;
    if ((e = dev_malloc(&d->d_ex, sizeof(float) * nr)) != cudaSuccess ||
        (e = dev_malloc(&d->d_pos, sizeof(float) * nr)) != cudaSuccess ||
        (e = dev_malloc(&d->d_samples, sizeof(float) * 3 * 32)) != cudaSuccess ||
        (e = dev_malloc(&d->points, sizeof(uint4) * (uint64_t)d->max_points)) != cudaSuccess ||
        (e = dev_malloc(&d->work, sizeof(WorkRec) * (uint64_t)d->max_points)) != cudaSuccess ||
        (e = dev_malloc(&d->near, sizeof(uint32_t) * (uint64_t)d->max_points)) != cudaSuccess ||
        (e = dev_malloc(&d->rrec, sizeof(ResolveRec) * (uint64_t)d->max_points)) != cudaSuccess ||
        (e = dev_malloc(&d->keys, 8u * npix)) != cudaSuccess ||
        (e = dev_malloc(&d->views, 4u * npix)) != cudaSuccess ||
        (e = dev_malloc(&d->panel, 4u * uint64_t(s.panel_w) * s.panel_h)) != cudaSuccess ||
        (e = dev_malloc(&d->ctr, sizeof(Counters))) != cudaSuccess) {
        free_display(d);
        return cuda_fail(e, "create_display: allocation");
    }
    const std::vector<float> pos = view_positions(d);
    if ((e = cudaMemcpy(d->d_ex, d->h_ex.data(), sizeof(float) * nr, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(d->d_pos, pos.data(), sizeof(float) * nr, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(d->ctr, 0, sizeof(Counters))) != cudaSuccess ||
        (e = cudaMemset(d->keys, 0xff, 8u * npix)) != cudaSuccess ||
        (e = cudaMemset(d->views, 0, 4u * npix)) != cudaSuccess) {
        free_display(d);
        return cuda_fail(e, "create_display: init");
    }
    *out = d;
    return LFDPR_OK;
}

lfdpr_status lfdpr_destroy_display(lfdpr_display* disp) {
    g_err[0] = 0;
    if (!disp) return fail(LFDPR_EINVAL, "destroy_display: null");
    if (disp->n_meshes != 0) return fail(LFDPR_EINVAL, "destroy_display: meshes still alive");
    free_display(disp);
    return LFDPR_OK;
}

lfdpr_status lfdpr_set_view_jitter(lfdpr_display* disp, const float* u, int32_t n) {
    g_err[0] = 0;
    if (!disp || !u) return fail(LFDPR_EINVAL, "set_view_jitter: null argument");
    if (n != disp->dc.nr) return fail(LFDPR_EINVAL, "set_view_jitter: %d values for %d rendered views", n, disp->dc.nr);
    for (int k = 0; k < n; k++)
        if (!(u[k] >= 0.0f && u[k] <= 1.0f)) return fail(LFDPR_EINVAL, "set_view_jitter: value %d not in [0, 1]", k);
    disp->h_jit.assign(u, u + n);
    place_eyes(disp);
    const std::vector<float> pos = view_positions(disp);
    CK(cudaMemcpy(disp->d_ex, disp->h_ex.data(), sizeof(float) * n, cudaMemcpyHostToDevice), "set_view_jitter: eyes");
    CK(cudaMemcpy(disp->d_pos, pos.data(), sizeof(float) * n, cudaMemcpyHostToDevice), "set_view_jitter: positions");
    return LFDPR_OK;
}

lfdpr_status lfdpr_set_recon_samples(lfdpr_display* disp, const float* samples, int32_t n) {
    g_err[0] = 0;
    if (!disp || !samples) return fail(LFDPR_EINVAL, "set_recon_samples: null argument");
    if (n < 1 || n > 32) return fail(LFDPR_EINVAL, "set_recon_samples: 1..32 samples");
    for (int k = 0; k < 3 * n; k++)
        if (!std::isfinite(samples[k])) return fail(LFDPR_EINVAL, "set_recon_samples: non-finite offset");
    CK(cudaMemcpy(disp->d_samples, samples, sizeof(float) * 3 * n, cudaMemcpyHostToDevice), "set_recon_samples");
    disp->n_samples = n;
    return LFDPR_OK;
}

lfdpr_status lfdpr_view_eyes(const lfdpr_display* disp, float* out, int32_t capacity) {
    if (!disp || !out) return fail(LFDPR_EINVAL, "view_eyes: null");
    if (capacity < disp->dc.nr) return fail(LFDPR_EINVAL, "view_eyes: capacity < rendered views");
    std::memcpy(out, disp->h_ex.data(), sizeof(float) * disp->dc.nr);
    return LFDPR_OK;
}

lfdpr_status lfdpr_upload_mesh(lfdpr_display* disp, const float* xyz, const float* uv, const uint32_t* idx,
                               const uint32_t* tri_tex, uint32_t n_verts, uint32_t n_tris,
                               const uint8_t* const* tex_rgba8, const uint32_t* tex_wh, uint32_t n_tex,
                               void* stream, lfdpr_mesh** out) {
    g_err[0] = 0;
    if (!disp || !out) return fail(LFDPR_EINVAL, "upload_mesh: null display or out");
    *out = nullptr;
    if (n_tex == 0 || !tex_rgba8 || !tex_wh) return fail(LFDPR_EINVAL, "upload_mesh: need >= 1 texture");
    for (uint32_t k = 0; k < n_tex; k++) {
        const uint32_t w = tex_wh[2 * k], h = tex_wh[2 * k + 1];
        if (!pow2(w) || !pow2(h) || w > 16384 || h > 16384)
            return fail(LFDPR_EINVAL, "upload_mesh: texture %u size %ux%u not a power of two <= 16384", k, w, h);
        if (!tex_rgba8[k]) return fail(LFDPR_EINVAL, "upload_mesh: null texture %u", k);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    lfdpr_mesh* m = nullptr;
    lfdpr_status st = upload_geometry(disp, xyz, uv, idx, tri_tex, n_verts, n_tris, n_tex, s, &m);
    if (st != LFDPR_OK) return st;
    st = upload_textures(tex_rgba8, tex_wh, n_tex, s, &m->pool, &m->tex, &m->lvl);
    if (st != LFDPR_OK) {
        free_mesh(m);
        return st;
    }
    m->owns_textures = true;
    disp->n_meshes++;
    *out = m;
    return LFDPR_OK;
}

lfdpr_status lfdpr_create_texture_set(const uint8_t* const* tex_rgba8, const uint32_t* tex_wh, uint32_t n_tex,
                                      void* stream, lfdpr_texture_set** out) {
    g_err[0] = 0;
    if (!out) return fail(LFDPR_EINVAL, "create_texture_set: null out");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(LFDPR_EDEVICE, "no CUDA device");
    }
    lfdpr_texture_set* t = new (std::nothrow) lfdpr_texture_set();
    if (!t) return fail(LFDPR_ENOMEM, "host allocation failed");
    const lfdpr_status st =
        upload_textures(tex_rgba8, tex_wh, n_tex, static_cast<cudaStream_t>(stream), &t->pool, &t->tex, &t->lvl);
    if (st != LFDPR_OK) {
        delete t;
        return st;
    }
    t->n_tex = n_tex;
    *out = t;
    return LFDPR_OK;
}

lfdpr_status lfdpr_destroy_texture_set(lfdpr_texture_set* set) {
    g_err[0] = 0;
    if (!set) return fail(LFDPR_EINVAL, "destroy_texture_set: null");
    if (set->n_meshes != 0) return fail(LFDPR_EINVAL, "destroy_texture_set: meshes still use it");
    dev_free(set->pool);
    dev_free(set->tex);
    dev_free(set->lvl);
    delete set;
    return LFDPR_OK;
}

lfdpr_status lfdpr_upload_mesh_textured(lfdpr_display* disp, const float* xyz, const float* uv, const uint32_t* idx,
                                        const uint32_t* tri_tex, uint32_t n_verts, uint32_t n_tris,
                                        lfdpr_texture_set* set, void* stream, lfdpr_mesh** out) {
    g_err[0] = 0;
    if (!disp || !out || !set) return fail(LFDPR_EINVAL, "upload_mesh_textured: null display, set or out");
    *out = nullptr;
    lfdpr_mesh* m = nullptr;
    const lfdpr_status st = upload_geometry(disp, xyz, uv, idx, tri_tex, n_verts, n_tris, set->n_tex,
                                            static_cast<cudaStream_t>(stream), &m);
    if (st != LFDPR_OK) return st;
    m->shared = set;
    m->pool = set->pool;
    m->tex = set->tex;
    m->lvl = set->lvl;
    set->n_meshes++;
    disp->n_meshes++;
    *out = m;
    return LFDPR_OK;
}

lfdpr_status lfdpr_upload_mesh_materials(lfdpr_display* disp, const float* xyz, const float* uv, const uint32_t* idx,
                                         const uint32_t* tri_mat, uint32_t n_verts, uint32_t n_tris,
                                         const uint32_t* mat_tex, uint32_t n_mat, lfdpr_texture_set* set,
                                         void* stream, lfdpr_mesh** out) {
    g_err[0] = 0;
    if (!disp || !out || !set || !mat_tex) return fail(LFDPR_EINVAL, "upload_mesh_materials: null argument");
    *out = nullptr;
    if (n_mat == 0 || n_mat > (1u << 24)) return fail(LFDPR_EINVAL, "upload_mesh_materials: 1..2^24 materials");
    for (uint64_t k = 0; k < 4ull * n_mat; k++)
        if (mat_tex[k] >= set->n_tex)
            return fail(LFDPR_EINVAL, "upload_mesh_materials: material %llu names texture %u of %u",
                        (unsigned long long)(k / 4), mat_tex[k], set->n_tex);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the display's per-point normal-map values, on its first mesh of materials
    if (!disp->rmat) {
        const cudaError_t e = dev_malloc(&disp->rmat, sizeof(uint2) * (uint64_t)disp->max_points);
        if (e != cudaSuccess) return cuda_fail(e, "upload_mesh_materials: normal-map buffer");
    }
    lfdpr_mesh* m = nullptr;
    // the material ids are checked against n_mat like texture ids
    const lfdpr_status st = upload_geometry(disp, xyz, uv, idx, tri_mat, n_verts, n_tris, n_mat, s, &m);
    if (st != LFDPR_OK) return st;
    cudaError_t e = dev_malloc(&m->mat_tex, 16ull * n_mat);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->mat_tex, mat_tex, 16ull * n_mat, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        free_mesh(m);
        return cuda_fail(e, "upload_mesh_materials: material table");
    }
    m->n_mat = n_mat;
    m->shared = set;
    m->pool = set->pool;
    m->tex = set->tex;
    m->lvl = set->lvl;
    set->n_meshes++;
    disp->n_meshes++;
    *out = m;
    return LFDPR_OK;
}

lfdpr_status lfdpr_set_shading(lfdpr_display* disp, const lfdpr_shading* sh) {
    g_err[0] = 0;
    if (!disp) return fail(LFDPR_EINVAL, "set_shading: null display");
    if (!sh || sh->model == LFDPR_SHADING_UNLIT) {
        disp->shading = LFDPR_SHADING_UNLIT;
        return LFDPR_OK;
    }
    if (sh->model != LFDPR_SHADING_PBR) return fail(LFDPR_EINVAL, "set_shading: unknown model %d", sh->model);
    for (int k = 0; k < 3; k++)
        if (!std::isfinite(sh->light_dir[k]) || !std::isfinite(sh->light_rgb[k]) || !std::isfinite(sh->ambient[k]) ||
            sh->light_rgb[k] < 0.0f || sh->ambient[k] < 0.0f)
            return fail(LFDPR_EINVAL, "set_shading: light values must be finite, radiance and ambient >= 0");
    const double l2 = double(sh->light_dir[0]) * sh->light_dir[0] + double(sh->light_dir[1]) * sh->light_dir[1] +
                      double(sh->light_dir[2]) * sh->light_dir[2];
    if (!(l2 > 0.0)) return fail(LFDPR_EINVAL, "set_shading: zero light direction");
    const double l = std::sqrt(l2);
    for (int k = 0; k < 3; k++) {
        disp->sh.l[k] = float(sh->light_dir[k] / l);
        disp->sh.rgb[k] = sh->light_rgb[k];
        disp->sh.amb[k] = sh->ambient[k];
    }
    disp->shading = LFDPR_SHADING_PBR;
    return LFDPR_OK;
}

lfdpr_status lfdpr_destroy_mesh(lfdpr_mesh* mesh) {
    g_err[0] = 0;
    if (!mesh) return fail(LFDPR_EINVAL, "destroy_mesh: null");
    if (mesh->disp) mesh->disp->n_meshes--;
    if (mesh->shared) mesh->shared->n_meshes--;
    free_mesh(mesh);
    return LFDPR_OK;
}

lfdpr_status lfdpr_render_frame(lfdpr_display* disp, lfdpr_mesh* mesh, const float model[16], void* stream) {
    g_err[0] = 0;
    if (!disp || !mesh || !model) return fail(LFDPR_EINVAL, "render_frame: null argument");
    if (mesh->disp != disp) return fail(LFDPR_EINVAL, "render_frame: mesh uploaded to another display");
    if (disp->shading == LFDPR_SHADING_PBR && !mesh->mat_tex)
        return fail(LFDPR_EINVAL, "render_frame: physically based shading needs a mesh of materials");
    for (int k = 0; k < 12; k++)
        if (!std::isfinite(model[k])) return fail(LFDPR_EINVAL, "render_frame: non-finite model matrix");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FrameArgs a = frame_args(disp, mesh);
    for (int k = 0; k < 12; k++) a.model[k] = model[k];
    const int nr = disp->dc.nr;
    const int band = disp->view_band > 0 && disp->view_band < nr ? disp->view_band : nr;
    const lfdpr_status st = record_frame_front(disp, mesh, a, s, disp->timing, band == nr);
    if (st != LFDPR_OK) return st;
    disp->bands_timed = 0;
    if (band == nr) {
        if (mesh->n_tris) {
            CK(launch_splat(a, s), "launch k_splat");
            disp->launches += 1;
        }
        mark(disp, 6, s);
        CK(launch_resolve(a, s), "launch k_resolve");
        disp->launches += 1;
        mark(disp, 7, s);
    } else {
        // band by band: each band's keys are cleared, hit by the splat and
        // read by the resolve while they can stay in L2
        const int nb = (nr + band - 1) / band;
        if (disp->timing && int(disp->band_ev.size()) < 4 * nb) {
            const size_t have = disp->band_ev.size();
            disp->band_ev.resize(4 * nb, nullptr);
            for (size_t k = have; k < disp->band_ev.size(); k++)
                CK(cudaEventCreate(&disp->band_ev[k]), "cudaEventCreate");
        }
        const uint64_t vpix = uint64_t(disp->dc.W) * disp->dc.H;
        for (int b = 0; b < nb; b++) {
            a.view_lo = b * band;
            a.view_hi = std::min(nr, a.view_lo + band);
            auto bm = [&](int k) {
                if (disp->timing) cudaEventRecord(disp->band_ev[4 * b + k], s);
            };
            bm(0);
            CK(cudaMemsetAsync(disp->keys + vpix * a.view_lo, 0xff, 8u * vpix * (a.view_hi - a.view_lo), s),
               "clear keys");
            bm(1);
            if (mesh->n_tris) {
                CK(launch_splat(a, s), "launch k_splat");
                disp->launches += 1;
            }
            bm(2);
            CK(launch_resolve(a, s), "launch k_resolve");
            disp->launches += 1;
            bm(3);
        }
        mark(disp, 6, s);
        mark(disp, 7, s);
        disp->bands_timed = disp->timing ? nb : 0;
    }
    disp->ev_frame = disp->timing;
    return LFDPR_OK;
}

lfdpr_status lfdpr_interleave(lfdpr_display* disp, uint8_t* panel_rgba8, void* stream) {
    g_err[0] = 0;
    if (!disp || !panel_rgba8) return fail(LFDPR_EINVAL, "interleave: null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // device memory is written in place; pinned host memory through its
    // device mapping (the kernels' stores cross the host link, and no copy
    // follows); pageable memory by a copy of the device scratch panel
    cudaPointerAttributes at;
    bool on_device = false;
    uint8_t* mapped = nullptr;
    if (cudaPointerGetAttributes(&at, panel_rgba8) == cudaSuccess) {
        on_device = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
        if (at.type == cudaMemoryTypeHost && at.devicePointer &&
            (reinterpret_cast<uintptr_t>(at.devicePointer) & 3u) == 0)
            mapped = static_cast<uint8_t*>(at.devicePointer);
    } else {
        cudaGetLastError();
    }
    if (on_device && (reinterpret_cast<uintptr_t>(panel_rgba8) & 3u) != 0)
        return fail(LFDPR_EINVAL, "interleave: a device panel must be 4-byte aligned");
    uint8_t* dst = on_device ? panel_rgba8 : mapped ? mapped : disp->panel;
    mark(disp, LFDPR_N_STAGES, s);
    if ((disp->desc.recon == 2 || disp->desc.recon == 3) && disp->n_samples == 0)
        return fail(LFDPR_EINVAL, "interleave: Gaussian reconstruction needs lfdpr_set_recon_samples");
    const lfdpr_status st = record_interleave(disp, dst, s);
    if (st != LFDPR_OK) return st;
    mark(disp, LFDPR_N_STAGES + 1, s);
    disp->ev_interleave = disp->timing;
    if (mapped) {
        CK(cudaStreamSynchronize(s), "interleave: synchronize");
    } else if (!on_device) {
        const uint64_t bytes = 4u * uint64_t(disp->dc.Wp) * disp->dc.Hp;
        CK(cudaMemcpyAsync(panel_rgba8, disp->panel, bytes, cudaMemcpyDeviceToHost, s), "interleave: copy to host");
        CK(cudaStreamSynchronize(s), "interleave: synchronize");
    }
    return LFDPR_OK;
}

lfdpr_status lfdpr_frame_stats(lfdpr_display* disp, void* stream, lfdpr_stats* out) {
    g_err[0] = 0;
    if (!disp) return fail(LFDPR_EINVAL, "frame_stats: null display");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaStreamSynchronize(s), "frame_stats: synchronize");
    CK(cudaGetLastError(), "frame_stats: pending error");
    Counters c;
    CK(cudaMemcpy(&c, disp->ctr, sizeof c, cudaMemcpyDeviceToHost), "frame_stats: read counters");
    if (out) {
        out->n_points = c.n_points;
        out->n_live_tris = c.n_live;
        out->overflow = int32_t(c.overflow);
        out->cell_overflow = int32_t(c.cell_overflow);
        out->kernel_launches = disp->launches;
        out->n_splat_writes = c.n_writes;
        for (int k = 0; k < LFDPR_N_STAGES; k++) out->stage_ms[k] = 0.0f;
        if (disp->ev_frame)
            for (int k = 0; k < LFDPR_STAGE_INTERLEAVE; k++)
                CK(cudaEventElapsedTime(&out->stage_ms[k], disp->ev[k], disp->ev[k + 1]), "stage time");
        if (disp->ev_frame && disp->bands_timed > 0) {
            // banded frame: clear, splat and resolve summed over the bands
            for (int k = 0; k < 3; k++) out->stage_ms[LFDPR_STAGE_CLEAR + k] = 0.0f;
            for (int b = 0; b < disp->bands_timed; b++)
                for (int k = 0; k < 3; k++) {
                    float ms = 0.0f;
                    CK(cudaEventElapsedTime(&ms, disp->band_ev[4 * b + k], disp->band_ev[4 * b + k + 1]),
                       "band stage time");
                    out->stage_ms[LFDPR_STAGE_CLEAR + k] += ms;
                }
        }
        if (disp->ev_interleave)
            CK(cudaEventElapsedTime(&out->stage_ms[LFDPR_STAGE_INTERLEAVE], disp->ev[LFDPR_N_STAGES],
                                    disp->ev[LFDPR_N_STAGES + 1]),
               "interleave time");
    }
    if (c.overflow)
        return fail(LFDPR_EOVERFLOW, "frame needed %u points, capacity %u", c.n_points, disp->max_points);
    if (c.cell_overflow) return fail(LFDPR_EOVERFLOW, "a triangle needed more than 65535 lattice cells per axis");
    return LFDPR_OK;
}

lfdpr_status lfdpr_set_spatial_supersampling(lfdpr_display* disp, int32_t level) {
    g_err[0] = 0;
    if (!disp) return fail(LFDPR_EINVAL, "set_spatial_supersampling: null display");
    if (level < 0 || level > 2) return fail(LFDPR_EINVAL, "set_spatial_supersampling: level %d outside 0-2", level);
    const int k = 1 << level;
    if (disp->dc.W % k || disp->dc.H % k)
        return fail(LFDPR_EINVAL, "set_spatial_supersampling: views %dx%d not divisible by %d", disp->dc.W, disp->dc.H,
                    k);
    if (level > 0) {
        const uint64_t bytes = 4u * uint64_t(disp->dc.W >> level) * uint64_t(disp->dc.H >> level) * disp->dc.nr;
        uint8_t* p = nullptr;
        CK(dev_malloc(&p, bytes), "set_spatial_supersampling: view mip buffer");
        dev_free(disp->views_mip);
        disp->views_mip = p;
    } else {
        dev_free(disp->views_mip);
        disp->views_mip = nullptr;
    }
    disp->ss_level = level;
    return LFDPR_OK;
}

lfdpr_status lfdpr_set_view_band(lfdpr_display* disp, int32_t band) {
    g_err[0] = 0;
    if (!disp) return fail(LFDPR_EINVAL, "set_view_band: null display");
    if (band < 0) return fail(LFDPR_EINVAL, "set_view_band: band %d < 0", band);
    disp->view_band = band;
    return LFDPR_OK;
}

lfdpr_status lfdpr_set_splat_lane_limit(lfdpr_display* disp, uint32_t limit) {
    g_err[0] = 0;
    if (!disp) return fail(LFDPR_EINVAL, "set_splat_lane_limit: null display");
    if (limit < 1u || limit > lfdpr::kSplatLaneLimit)
        return fail(LFDPR_EINVAL, "set_splat_lane_limit: %u outside [1, 2^24]", limit);
    disp->splat_lane_limit = limit;
    return LFDPR_OK;
}

lfdpr_status lfdpr_set_stage_timing(lfdpr_display* disp, int32_t enable) {
    g_err[0] = 0;
    if (!disp) return fail(LFDPR_EINVAL, "set_stage_timing: null display");
    if (enable && !disp->ev[0]) {
        for (auto& e : disp->ev) CK(cudaEventCreate(&e), "cudaEventCreate");
    }
    disp->timing = enable != 0;
    disp->ev_frame = disp->ev_interleave = false;
    return LFDPR_OK;
}

lfdpr_status lfdpr_get_buffers(lfdpr_display* disp, lfdpr_mesh* mesh, lfdpr_buffers* out) {
    g_err[0] = 0;
    if (!disp || !mesh || !out) return fail(LFDPR_EINVAL, "get_buffers: null argument");
    out->counts = mesh->counts;
    out->offsets = mesh->offsets;
    out->points = reinterpret_cast<const uint32_t*>(disp->points);
    out->tri = reinterpret_cast<const float*>(mesh->rec);
    out->keys = disp->keys;
    out->views = disp->views;
    out->n_tris = mesh->n_tris;
    out->max_points = disp->max_points;
    out->n_render_views = disp->dc.nr;
    out->view_w = disp->dc.W;
    out->view_h = disp->dc.H;
    out->resolve = reinterpret_cast<const uint32_t*>(disp->rrec);
    out->resolve_mat = reinterpret_cast<const uint32_t*>(disp->rmat);
    return LFDPR_OK;
}

lfdpr_status lfdpr_probe_atomic_min(uint64_t* words, uint64_t n_words, const uint32_t* idx, const uint64_t* val,
                                    uint64_t n_ops, int32_t mode, void* stream) {
    g_err[0] = 0;
    if (!words || !idx || !val || n_words == 0) return fail(LFDPR_EINVAL, "probe: null or empty argument");
    if (mode < 0 || mode > 2) return fail(LFDPR_EINVAL, "probe: mode %d outside 0-2", mode);
    if (mode == 1 && n_words > 8192) return fail(LFDPR_EINVAL, "probe: shared variant holds at most 8192 words");
    int dev = 0, sms = 1;
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "sm count");
    CK(launch_probe_atomic(words, n_words, idx, val, n_ops, mode, sms, static_cast<cudaStream_t>(stream)),
       "launch probe");
    return LFDPR_OK;
}

}  // extern "C"
