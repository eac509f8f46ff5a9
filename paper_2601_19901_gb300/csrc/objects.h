// Library objects behind the opaque handles of include/lfdpr.h, shared by
// runtime.cu (displays, meshes, texture sets, single frames) and batch.cu
// (batched frames).
#pragma once
#include <vector>

#include "lfdpr_internal.cuh"

struct lfdpr_texture_set {
    uint32_t n_tex = 0;
    uint8_t* pool = nullptr;
    lfdpr::TexDesc* tex = nullptr;
    uint64_t* lvl = nullptr;
    int n_meshes = 0;
};

struct lfdpr_display {
    lfdpr_display_desc desc;
    lfdpr::DispConst dc;
    int device = 0;
    int sm_count = 1;
    std::vector<float> h_ex;
    std::vector<float> h_jit;     // per rendered view: its place in its interval (1/2: the default eyes)
    float* d_ex = nullptr;
    float* d_pos = nullptr;       // rendered views' positions on the display-view axis
    float* d_samples = nullptr;   // Gaussian reconstruction samples [32][3]
    int n_samples = 0;
    uint4* points = nullptr;
    uint32_t max_points = 0;
    lfdpr::WorkRec* work = nullptr;
    uint32_t* near = nullptr;     // points whose cell or triangle reaches within near_z of the eyes' plane
    lfdpr::ResolveRec* rrec = nullptr;
    uint2* rmat = nullptr;        // normal-map tv_min / tv_max per point (allocated with the first mesh of materials)
    uint64_t* keys = nullptr;
    uint8_t* views = nullptr;
    uint8_t* panel = nullptr;      // device scratch for host-memory panels
    int ss_level = 0;              // spatial supersampling: the interleave reads this mip level of the views
    uint8_t* views_mip = nullptr;  // that level of every rendered view
    lfdpr::Counters* ctr = nullptr;
    int n_meshes = 0;
    int64_t launches = 0;
    bool timing = false;
    cudaEvent_t ev[LFDPR_N_STAGES + 2] = {};
    bool ev_frame = false;        // the frame's stage events were recorded
    bool ev_interleave = false;   // the interleave's events were recorded
    int shading = LFDPR_SHADING_UNLIT;
    uint32_t splat_lane_limit = lfdpr::kSplatLaneLimit;
    int view_band = 0;            // views per band of key clear, splat and resolve (0: all at once)
    std::vector<cudaEvent_t> band_ev;   // per band: before the clear, after it, after the splat, after the resolve
    int bands_timed = 0;          // bands of the last frame whose events were recorded
    lfdpr::Shading sh{};          // light (unit direction), radiance, ambient
};

struct lfdpr_mesh {
    lfdpr_display* disp = nullptr;
    uint32_t n_verts = 0, n_tris = 0, n_tex = 0, n_blocks = 0;
    float* xyz = nullptr;
    float* uv = nullptr;
    uint32_t* idx = nullptr;
    uint32_t* tri_tex = nullptr;              // texture (or, with materials, material) per triangle
    uint4* mat_tex = nullptr;                 // materials: [n_mat] albedo, normal, roughness, metallic texture ids
    uint32_t n_mat = 0;
    lfdpr_texture_set* shared = nullptr;   // the texture set whose pool/tex/lvl the mesh uses
    bool owns_textures = false;            // pool/tex/lvl are the mesh's own (freed with it)
    uint8_t* pool = nullptr;
    lfdpr::TexDesc* tex = nullptr;
    uint64_t* lvl = nullptr;
    lfdpr::TriRec* rec = nullptr;
    lfdpr::TriProj* tproj = nullptr;
    uint32_t* counts = nullptr;
    uint32_t* offsets = nullptr;
    uint4* colsum = nullptr;
    uint32_t* block_sums = nullptr;
};

namespace lfdpr {
// Set the thread's last-error text and return s.
lfdpr_status fail(lfdpr_status s, const char* fmt, ...);
lfdpr_status cuda_fail(cudaError_t e, const char* what);
// The interleave of the display's last views on stream s into `panel`:
// with spatial supersampling, mip level ss_level of every view first.
lfdpr_status record_interleave(lfdpr_display* disp, uint8_t* panel, cudaStream_t s);
// Kernel arguments of one frame of `mesh` on `disp` (model left unset).
FrameArgs frame_args(const lfdpr_display* disp, const lfdpr_mesh* mesh);
// The frame up to the splat on stream s: counters reset, set-up, scan,
// emission, fetch (with the near-limit records), key clear (unless the
// views are cleared band by band); stage events 0-5 recorded if marks.
lfdpr_status record_frame_front(lfdpr_display* disp, lfdpr_mesh* mesh, const FrameArgs& a, cudaStream_t s,
                                bool marks, bool clear_keys = true);
}  // namespace lfdpr
