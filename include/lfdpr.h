/*
 * lfdpr.h — C ABI of liblfdpr.so: light field display point rendering (LFDPR,
 * Gavane & Watson, ACM TOG 2024) on one GB300 GPU (sm_103a).
 *
 * Per frame the library samples a textured triangle mesh into a point cloud
 * fitted to a lenticular display (Sec. 3.1), splats every point into every
 * display view with a 64-bit depth|id test (Sec. 3.2, Sec. 5.1), textures the
 * splats by multiview mipmapping (Sec. 3.3, Eq. 4-9), and interleaves the views
 * into one panel image after optional angular supersampling, reconstruction
 * and crosstalk (Sec. 4).
 *
 * Conventions
 *  - Opaque handles are owned by the library; destroy them with the matching
 *    lfdpr_destroy_*.
 *  - Input arrays passed by pointer are owned by the caller and copied before
 *    the call returns unless stated otherwise.
 *  - Output buffers are owned by the caller.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls that
 *    launch work are asynchronous with respect to the host on that stream.
 *    A frame's kernels after the first are launched as programmatic
 *    dependents of the kernel before them (their launch overlaps its last
 *    blocks) and wait for it before touching memory, so stream order holds
 *    for the caller's own work as for plain launches. Each of them lets the
 *    next kernel start early, so a kernel of the caller's that is itself
 *    launched with programmatic stream serialization right after a call must
 *    wait for its predecessor (griddepcontrol.wait) before reading the
 *    call's results, as programmatic dependent launch requires.
 *  - Every call returns an lfdpr_status and never aborts the process. On error
 *    lfdpr_last_error() (per thread) holds a one-line description. Errors of
 *    asynchronous device work (point-buffer overflow, a launch failure) are
 *    reported by the next lfdpr_frame_stats().
 *  - One display and its meshes must be used from one host thread at a time.
 */
#ifndef LFDPR_H
#define LFDPR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LFDPR_VERSION 1

typedef struct lfdpr_display lfdpr_display;
typedef struct lfdpr_mesh lfdpr_mesh;
typedef struct lfdpr_texture_set lfdpr_texture_set;
typedef struct lfdpr_batch lfdpr_batch;

typedef enum {
    LFDPR_OK = 0,
    LFDPR_EINVAL = 1,     /* invalid argument: null pointer, bad size, bad descriptor */
    LFDPR_ENOMEM = 2,     /* device or host allocation failed */
    LFDPR_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed */
    LFDPR_EOVERFLOW = 4,  /* the frame needed more points than the point buffer holds */
    LFDPR_EDEVICE = 5     /* no usable CUDA device */
} lfdpr_status;

/*
 * Display and view set (Sec. 3: views defined by the LFD; Sec. 5.1: the
 * prototype; Sec. 4: interleave, supersampling, reconstruction).
 * The N views are pinhole eyes on the line y = 0, z = view_dist, at the centres
 * of N equal angular intervals of a cone of cone_deg degrees; all look down -z
 * through one focal rectangle focal_w x focal_h centred on the origin at z = 0.
 * Each view is view_w x view_h pixels. Depths (view_dist - z) outside
 * [near_z, far_z] are not drawn. bias_h, bias_v multiply the horizontal and
 * vertical point spacings (LFD-biased sampling, Sec. 3.1). The panel is
 * panel_w x panel_h RGBA8 under slanted lenses of lens_pitch_px pixels, slant
 * `slant` pixels per row, phase offset phase_offset (in lens periods).
 * recon = 1 renders 2N views at half-interval steps and reconstructs N with a
 * [1/4, 1/2, 1/4] tent; recon = 2 renders 2N views and recon = 3 N views,
 * both reconstructed by the Gaussian filters of Sec. 4 at sample offsets set
 * with lfdpr_set_recon_samples (required before their interleave); crosstalk
 * x > 0 mixes each view with its +-1 neighbours at weight x before
 * interleaving (for recon 2 and 3: the reconstruction one view away). max_points is the point-buffer
 * capacity (0 = 1 << 23); each point of capacity takes 100 B of device
 * memory (the 16-B point record, a 48-B splat work record, a 4-B near-list
 * entry and a 32-B resolve record), and 8 B more once a mesh of materials is
 * uploaded to the display.
 */
typedef struct {
    int32_t n_views, view_w, view_h;
    float cone_deg, view_dist, focal_w, focal_h, near_z, far_z, bias_h, bias_v;
    int32_t panel_w, panel_h;
    float lens_pitch_px, slant, phase_offset;
    int32_t recon;
    float crosstalk;
    int64_t max_points;
} lfdpr_display_desc;

/* Stages of a frame, in launch order (Sec. 5.3 reports point generation,
 * view generation and EIA construction times separately). */
enum {
    LFDPR_STAGE_SETUP = 0,      /* per-triangle set-up and count (Sec. 3.1) */
    LFDPR_STAGE_SCAN = 1,       /* exclusive scan of the counts */
    LFDPR_STAGE_EMIT = 2,       /* point emission */
    LFDPR_STAGE_FETCH = 3,      /* tv_min / tv_max fetch (Sec. 3.3) */
    LFDPR_STAGE_CLEAR = 4,      /* view key buffers reset (done by the fetch pass, and timed
                                   there, when the mesh has triangles) */
    LFDPR_STAGE_SPLAT = 5,      /* splatting with the depth test (Sec. 3.2) */
    LFDPR_STAGE_RESOLVE = 6,    /* Eq. 8-9 per view pixel */
    LFDPR_STAGE_INTERLEAVE = 7, /* reconstruction, crosstalk, interleave (Sec. 4) */
    LFDPR_N_STAGES = 8
};

/* Per-frame counters read back by lfdpr_frame_stats. */
typedef struct {
    int64_t n_points;       /* points the last frame generated */
    int64_t n_live_tris;    /* triangles not culled and of non-zero area */
    int32_t overflow;       /* 1 if n_points exceeded max_points (frame not drawn) */
    int32_t cell_overflow;  /* 1 if a triangle needed more than 65535 lattice columns or rows */
    int64_t kernel_launches;/* kernels this display has launched since its creation */
    int64_t n_splat_writes; /* depth-test atomics (accepted pixel tests) of the last splat */
    float stage_ms[LFDPR_N_STAGES]; /* device time of each stage of the last frame and
                                       interleave, from CUDA events on the caller's
                                       stream; 0 unless lfdpr_set_stage_timing(.., 1) */
} lfdpr_stats;

/* Floats per triangle in the record array exposed by lfdpr_get_buffers. */
#define LFDPR_TRI_FLOATS 32
/* Offsets into one triangle record (float index). */
enum {
    LFDPR_TRI_P0 = 0,        /* 3: transformed first vertex */
    LFDPR_TRI_SU = 3,        /* horizontal point spacing s_u */
    LFDPR_TRI_EU = 4,        /* 3: horizontal sampling axis (T_align) */
    LFDPR_TRI_SV = 7,        /* vertical point spacing s_v */
    LFDPR_TRI_EV = 8,        /* 3: vertical sampling axis */
    LFDPR_TRI_UMIN = 11,     /* lattice origin offset along u */
    LFDPR_TRI_N = 12,        /* 3: unit normal */
    LFDPR_TRI_VMIN = 15,     /* lattice origin offset along v */
    LFDPR_TRI_A1 = 16,       /* 4: 2-D coordinates (a1, b1, a2, b2) of vertices 1, 2 */
    LFDPR_TRI_SPL_UV = 20,   /* splat area in texture space (Eq. 8) */
    LFDPR_TRI_VPUV_MIN = 21, /* Eq. 4 */
    LFDPR_TRI_VPUV_MAX = 22, /* Eq. 5 */
    LFDPR_TRI_UMAX = 23,     /* lattice extent along u */
    LFDPR_TRI_S0 = 24,       /* 3: texture s = s0 + gu u + gv v over the lattice frame */
    LFDPR_TRI_T0 = 27,       /* texture t offset */
    LFDPR_TRI_TGU = 28,      /* 2: texture t gradients */
    LFDPR_TRI_LOD_MIN = 30,  /* Eq. 6 */
    LFDPR_TRI_LOD_MAX = 31   /* Eq. 7 */
};

/*
 * Device buffers of the last frame, borrowed: valid until the next
 * lfdpr_render_frame on the display or its destruction. Read them only after
 * the frame's stream work has finished. Layouts:
 *  counts   u32 [n_tris]                     points per triangle (0 = culled/degenerate)
 *  offsets  u32 [n_tris]                     first point id of each triangle
 *  points   u32 [max_points][4]              triangle id, i | j << 16 (lattice cell),
 *                                            tv_min RGBA8, tv_max RGBA8 (Sec. 3.3)
 *  tri      f32 [n_tris][LFDPR_TRI_FLOATS]   per-triangle sampling record
 *  keys     u64 [n_render_views][view_h][view_w]  float_bits(t) << 32 | point id,
 *                                            all ones where empty (Sec. 3.2)
 *  views    u8  [n_render_views][view_h][view_w][4] resolved RGBA8 views
 *  resolve  u32 [max_points][8]              the resolve's per-point record: alpha, beta (the
 *                                            splat's pixel area in the view of eye x Ex is
 *                                            |alpha + beta Ex| / 2), splat texture area, size_vpuv
 *                                            min, max (f32), tv_min, tv_max (RGBA8), roughness /
 *                                            metallic tv_min, tv_max bytes (R channels; meshes of
 *                                            materials)
 *  resolve_mat u32 [max_points][2]           normal-map tv_min, tv_max RGBA8 (meshes of materials;
 *                                            NULL before the display's first such mesh)
 */
typedef struct {
    const uint32_t *counts, *offsets, *points;
    const float *tri;
    const uint64_t *keys;
    const uint8_t *views;
    int64_t n_tris, max_points;
    int32_t n_render_views, view_w, view_h;
    const uint32_t *resolve, *resolve_mat;
} lfdpr_buffers;

/*
 * lfdpr_create_display: validate `desc` (positive sizes, 1 <= n_views <= 256,
 * views of at most 16384 pixels a side and 2^26 pixels,
 * 0 < near_z < far_z, view_dist > 0, focal sizes > 0, recon in {0, 1, 2, 3},
 * 0 <= crosstalk < 0.5) and allocate the display's device buffers: view key
 * buffers (8 B per rendered-view pixel, Sec. 5.2), RGBA8 views, the point
 * buffers (100 B per point of capacity) and the panel scratch. Uses the current CUDA device.
 * On success *out owns them. Errors: EINVAL, ENOMEM, EDEVICE, ECUDA.
 */
lfdpr_status lfdpr_create_display(const lfdpr_display_desc *desc, lfdpr_display **out);

/* Free a display and every device buffer it owns (meshes must be destroyed first). */
lfdpr_status lfdpr_destroy_display(lfdpr_display *disp);

/*
 * lfdpr_set_view_jitter: place each rendered view at a chosen point of its
 * angular interval (Sec. 4: supersampled views at random angles in the view
 * intervals; the caller draws the numbers). u f32 [n], n = the rendered view
 * count (2N for recon 1 and 2, else N), each in [0, 1] (host, copied). With
 * 2N views, view m's eye is at the angle -cone/2 + cone (m + 1/2 + u_m) / 2N;
 * with N views, -cone/2 + cone (k + u_k) / N; u = 1/2 everywhere gives the
 * default eyes. Applies from the next frame. Errors: EINVAL, ECUDA.
 */
lfdpr_status lfdpr_set_view_jitter(lfdpr_display *disp, const float *u, int32_t n);

/*
 * lfdpr_set_spatial_supersampling: 2x (level 1) or 4x (level 2) spatial
 * supersampling (Sec. 4; Sec. 5.1 builds a mipmap of each light field view
 * for it). The display's views are rendered at view_w x view_h, 2^level times
 * the output resolution per axis; lfdpr_interleave first reduces every
 * rendered view to mip level `level` (level times the 2 x 2 box
 * (a + b + c + d + 2) >> 2 per channel, the textures' mip rounding) and
 * interleaves those output-resolution views (with Gaussian reconstruction the
 * sample offsets are then in output pixels). Level 0 (the default) turns it
 * off. view_w and view_h must be multiples of 2^level; the level's views are
 * allocated here (4 B per output pixel per rendered view). Errors: EINVAL,
 * ENOMEM, ECUDA.
 */
lfdpr_status lfdpr_set_spatial_supersampling(lfdpr_display *disp, int32_t level);

/*
 * lfdpr_set_recon_samples: the sample offsets of the Gaussian
 * reconstruction (recon 2, 3; Sec. 4 integrates its filters with a few
 * random samples; the caller draws them): samples f32 [n][3] (host, copied),
 * 1 <= n <= 32, each (dx, dy) in view pixels and dphi in display views. A
 * panel subpixel at lens phase phi (in display views, [0, N)) shows the mean
 * over the samples of the rendered view nearest (on the display-view axis,
 * where rendered view m sits at (m + 1/2 + u_m) / 2 with 2N views, k + u_k
 * with N; ties to the later view) to phi + dphi, at the view pixel holding
 * ((x + 1/2) W / panel_w + dx, (y + 1/2) H / panel_h + dy), clamped to the
 * view. Errors: EINVAL, ECUDA.
 */
lfdpr_status lfdpr_set_recon_samples(lfdpr_display *disp, const float *samples, int32_t n);

/*
 * lfdpr_upload_mesh: copy a triangle mesh and its textures to the device and
 * build each texture's mip chain there (Sec. 3.3 relies on mipmaps).
 *  xyz      f32 [n_verts][3] object-space positions (host)
 *  uv       f32 [n_verts][2] texture coordinates, wrap addressing (host)
 *  idx      u32 [n_tris][3]  vertex indices < n_verts (host)
 *  tri_tex  u32 [n_tris]     texture id < n_tex per triangle (host)
 *  tex_rgba8[k]  u8 [h][w][4] level-0 texels of texture k (host)
 *  tex_wh   u32 [n_tex][2]   (w, h) of texture k; powers of two, <= 16384
 * All inputs are validated (indices and texture ids in range, sizes) and copied;
 * the call synchronises `stream` before returning. Errors: EINVAL, ENOMEM, ECUDA.
 */
lfdpr_status lfdpr_upload_mesh(lfdpr_display *disp, const float *xyz, const float *uv,
                               const uint32_t *idx, const uint32_t *tri_tex,
                               uint32_t n_verts, uint32_t n_tris,
                               const uint8_t *const *tex_rgba8, const uint32_t *tex_wh,
                               uint32_t n_tex, void *stream, lfdpr_mesh **out);

/* Free a mesh's device buffers. */
lfdpr_status lfdpr_destroy_mesh(lfdpr_mesh *mesh);

/*
 * lfdpr_render_frame: one frame of the hot path (Sec. 3, Fig. 4) on `stream`:
 * transform by `model` (row-major 4x4, host memory, affine rows 0-2 used),
 * cull, per-triangle sampling set-up (Sec. 3.1, Eq. 1-7), scan, point emission,
 * tv_min/tv_max fetch (Sec. 3.3), splatting into every rendered view
 * (Sec. 3.2), and the per-view resolve of Eq. 8-9 into RGBA8 views. No host
 * synchronisation; nothing is allocated. If the frame needs more points than
 * max_points the frame is not drawn and the next lfdpr_frame_stats returns
 * EOVERFLOW. Errors: EINVAL, ECUDA.
 */
lfdpr_status lfdpr_render_frame(lfdpr_display *disp, lfdpr_mesh *mesh, const float model[16],
                                void *stream);

/*
 * lfdpr_interleave: build the elemental image array from the last frame's
 * views (Sec. 4): optional tent reconstruction of 2N supersampled views, then
 * optional crosstalk mixing, then the slanted-lens subpixel interleave.
 * `panel_rgba8` is u8 [panel_h][panel_w][4], caller-owned, in device memory
 * (4-byte aligned) or in host memory (pinned or pageable). Pinned host memory
 * is written by the interleave kernels through its device mapping; pageable
 * memory gets the panel built in device scratch and copied back on `stream`.
 * For host memory the call returns once the panel is complete there.
 * Errors: EINVAL (also a device panel not 4-byte aligned), ECUDA.
 */
lfdpr_status lfdpr_interleave(lfdpr_display *disp, uint8_t *panel_rgba8, void *stream);

/*
 * lfdpr_frame_stats: synchronise `stream`, then report the last frame's
 * counters and any asynchronous error (EOVERFLOW, ECUDA). `out` may be NULL.
 */
lfdpr_status lfdpr_frame_stats(lfdpr_display *disp, void *stream, lfdpr_stats *out);

/*
 * lfdpr_set_stage_timing: enable (1) or disable (0) CUDA events between the
 * stages of lfdpr_render_frame and around lfdpr_interleave, recorded on the
 * caller's stream; lfdpr_frame_stats then reports each stage's device time.
 * The events separate the stages' kernels (no launch overlaps the kernel
 * before it), so a timed frame runs a little longer (about 20 us for the
 * paper-shaped frame). Off by default. Errors: EINVAL.
 */
lfdpr_status lfdpr_set_stage_timing(lfdpr_display *disp, int32_t enable);

/*
 * lfdpr_set_splat_lane_limit: the splat (Sec. 3.2) pools the candidate
 * pixels of four points per warp into 32-lane passes numbered with 32-bit
 * integers; a unit in which some lane's views hold `limit` or more candidates
 * (huge cells) is instead walked segment by segment, one lane per (point,
 * view). The default, and the largest value, 2^24, keeps every number below
 * 2^32; smaller values send more units down the walk, which gives the same
 * keys more slowly. Errors: EINVAL (null display, limit outside [1, 2^24]).
 */
lfdpr_status lfdpr_set_splat_lane_limit(lfdpr_display *disp, uint32_t limit);

/*
 * lfdpr_set_view_band: order the depth test (Sec. 3.2, Sec. 5.1) by view
 * band. With band = b > 0 and fewer than the rendered views, each frame
 * clears, splats and resolves views [0, b), then [b, 2b), ..., so that a
 * band's key buffers (8 B per pixel) can stay resident in L2 while they are
 * hit, when all the views' keys would not fit; results are identical. 0 (the
 * default) treats all views as one band. Errors: EINVAL (null display,
 * band < 0).
 */
lfdpr_status lfdpr_set_view_band(lfdpr_display *disp, int32_t band);

/* lfdpr_get_buffers: borrowed device pointers of the last frame (see lfdpr_buffers). */
lfdpr_status lfdpr_get_buffers(lfdpr_display *disp, lfdpr_mesh *mesh, lfdpr_buffers *out);

/* Eye x positions of the rendered views (host floats, n_render_views of them). */
lfdpr_status lfdpr_view_eyes(const lfdpr_display *disp, float *out, int32_t capacity);

/*
 * lfdpr_probe_atomic_min: roofline probe for the splat's depth test (Sec. 5.1
 * uses 64-bit buffers). Performs n_ops 64-bit atomicMin operations on `words`
 * (u64 [n_words], device) with values val[k] (u64 [n_ops], device), at
 * addresses chosen by `mode` from idx (u32 [n_ops], device):
 *  0  word idx[k] (random indices: every lane of a warp instruction hits its
 *     own line);
 *  1  word idx[k] mod n_words of a per-block copy in shared memory
 *     (n_words <= 8192), merged back with one global atomicMin per word;
 *  2  word (idx[32 q] rounded down to a multiple of 32) + (k mod 32) for
 *     k in the group q of 32 consecutive operations (one warp instruction
 *     hits 32 consecutive words, 256 bytes: the most coherent pattern).
 * Indices at or beyond n_words are skipped. Asynchronous on `stream`.
 * Errors: EINVAL (null or empty buffers, mode outside 0-2), ECUDA.
 */
lfdpr_status lfdpr_probe_atomic_min(uint64_t *words, uint64_t n_words, const uint32_t *idx,
                                    const uint64_t *val, uint64_t n_ops, int32_t mode, void *stream);

/*
 * lfdpr_sample_points_noalloc: the point-generation stage alone (per-triangle
 * set-up and count, scan, emission; the steps of lfdpr_render_frame before the
 * texture fetch) for callers that must not allocate. The paper has no
 * counterpart: it exists because some callers cannot call cudaMalloc, or any
 * routine that allocates, while they run - a real-time render loop that only
 * allocates at start-up, or a plug-in whose host application owns all device
 * memory and its budget. This call allocates nothing: its scratch (triangle
 * records, first-point offsets, block sums, counters, eye positions, texture
 * sizes) is one fixed file-scope device array of about 4.3 MB, held by every
 * GPU that loads the library until the process exits.
 *  desc, model, tex_wh  host: display, row-major 4x4 model matrix, (w, h) of
 *                       each of the n_tex textures (powers of two <= 16384)
 *  xyz, uv, idx, tri_tex  device, caller-owned, layouts as lfdpr_upload_mesh;
 *                       indices and texture ids must be in range (not checked)
 *  points   device u32 [max_points][4]: words 0-1 of each point receive
 *           triangle id and i | j << 16 (words 2-3 are left untouched)
 *  counts   device u32 [n_tris]: points per triangle
 *  frame_counters  device u32 [4]: points needed, overflow flag (points beyond
 *           max_points are not written), lattice-overflow flag, live triangles
 * Limits: n_tris <= LFDPR_NOALLOC_MAX_TRIS, 1 <= n_tex <= LFDPR_NOALLOC_MAX_TEX;
 * larger sizes return EINVAL with a message. The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current and keeps it for the life of the process; make that first call
 * before any stream capture, and make no call after a cudaDeviceReset of that
 * device (the kept address would belong to the destroyed context). The eye
 * positions and texture sizes reach the device as a kernel parameter, so
 * nothing on the host has to outlive the call. Every call shares the one
 * array, which keeps the last call's contents (the counters are cleared by
 * each call): calls that overlap on the GPU, from any stream or thread, race.
 * Asynchronous on `stream`. Errors: EINVAL, EDEVICE, ECUDA.
 */
#define LFDPR_NOALLOC_MAX_TRIS 32768
#define LFDPR_NOALLOC_MAX_TEX 256
lfdpr_status lfdpr_sample_points_noalloc(const lfdpr_display_desc *desc, const float model[16],
                                         const float *xyz, const float *uv, const uint32_t *idx,
                                         const uint32_t *tri_tex, uint32_t n_tris,
                                         const uint32_t *tex_wh, uint32_t n_tex, uint32_t *points,
                                         uint32_t max_points, uint32_t *counts,
                                         uint32_t *frame_counters, void *stream);

/*
 * Texture sets: textures (with their mip chains, Sec. 3.3) uploaded once and
 * shared by any number of meshes, of any display, on the same device.
 *
 * lfdpr_create_texture_set: tex_rgba8[k] u8 [h][w][4] level-0 texels of
 * texture k (host); tex_wh u32 [n_tex][2] their (w, h), powers of two
 * <= 16384. Copied; mip chains built on the device; the call synchronises
 * `stream`. Errors: EINVAL, ENOMEM, ECUDA.
 */
lfdpr_status lfdpr_create_texture_set(const uint8_t *const *tex_rgba8, const uint32_t *tex_wh,
                                      uint32_t n_tex, void *stream, lfdpr_texture_set **out);

/* Free a texture set (EINVAL while meshes still use it). */
lfdpr_status lfdpr_destroy_texture_set(lfdpr_texture_set *set);

/*
 * lfdpr_upload_mesh_textured: lfdpr_upload_mesh with the textures of a
 * texture set (tri_tex ids index it) instead of its own copy. The set must
 * outlive the mesh. Errors as lfdpr_upload_mesh.
 */
lfdpr_status lfdpr_upload_mesh_textured(lfdpr_display *disp, const float *xyz, const float *uv,
                                        const uint32_t *idx, const uint32_t *tri_tex, uint32_t n_verts,
                                        uint32_t n_tris, lfdpr_texture_set *set, void *stream,
                                        lfdpr_mesh **out);

/*
 * Meshes of materials (several textures per triangle, Sec. 3.1 Eq. 1 and
 * Sec. 3.3). A material is four textures of a texture set: albedo (RGB),
 * tangent-space normal map (n = 2 c / 255 - 1 per channel), roughness (R),
 * metallic (R), each with its own resolution. Eq. 1 takes a triangle's
 * texel count as the largest over its material's four textures; each texture
 * is fetched at its own Eq. 6-7 LOD pair (its resolution); the resolve
 * interpolates every texture by Eq. 9 with the same weight.
 *
 * lfdpr_upload_mesh_materials: as lfdpr_upload_mesh_textured with tri_mat u32
 * [n_tris] material per triangle and mat_tex u32 [n_mat][4] the texture ids
 * (albedo, normal, roughness, metallic) of each material. Unlit displays draw
 * the albedo; displays set to LFDPR_SHADING_PBR shade physically.
 * Errors: EINVAL (ids out of range), ENOMEM, ECUDA.
 */
lfdpr_status lfdpr_upload_mesh_materials(lfdpr_display *disp, const float *xyz, const float *uv,
                                         const uint32_t *idx, const uint32_t *tri_mat, uint32_t n_verts,
                                         uint32_t n_tris, const uint32_t *mat_tex, uint32_t n_mat,
                                         lfdpr_texture_set *set, void *stream, lfdpr_mesh **out);

#define LFDPR_SHADING_UNLIT 0
#define LFDPR_SHADING_PBR 1

/*
 * Shading during view generation (Sec. 3.3). LFDPR_SHADING_UNLIT draws the
 * interpolated albedo (the default). LFDPR_SHADING_PBR (meshes of materials
 * only) shades every view pixel where its splat's surface point lies (the
 * pixel centre's ray meets the triangle at the depth-tested t) for that
 * view's own eye, under one directional light:
 *   metallic-roughness microfacet BRDF, GGX distribution with a = r^2
 *   (r >= 0.045), Schlick-GGX visibility with k = (r + 1)^2 / 8, Schlick
 *   Fresnel with F0 = 0.04 (1 - m) + albedo m, diffuse (1 - F)(1 - m)
 *   albedo / pi; rgb = (diffuse + D G F / (4 n.l n.v)) light_rgb n.l
 *   + ambient albedo, clamped to [0, 1], times 255, rounded half to even.
 * The shading normal is the normal map's vector in the triangle's frame
 * (tangent and bitangent along increasing texture s and t), turned toward
 * the eye for triangles seen from behind.
 */
typedef struct {
    int32_t model;        /* LFDPR_SHADING_UNLIT or LFDPR_SHADING_PBR */
    float light_dir[3];   /* direction toward the light (normalised by the library) */
    float light_rgb[3];   /* radiance of the light per channel (>= 0) */
    float ambient[3];     /* ambient term per channel, times albedo (>= 0) */
} lfdpr_shading;

/* lfdpr_set_shading: the display's shading (NULL = unlit). Errors: EINVAL. */
lfdpr_status lfdpr_set_shading(lfdpr_display *disp, const lfdpr_shading *shading);

/*
 * Batched frames: n (display, mesh) scenes, each with its own display (view
 * count, view size, panel), rendered and interleaved together. One call runs
 * every scene's frame, Sec. 3.1-4 as lfdpr_render_frame followed by
 * lfdpr_interleave, as one CUDA graph: per-scene set-up, scan, emission and
 * fetch on `branches` concurrent graph branches, then one persistent splat
 * launch over the point pairs of all scenes, then per-scene resolve and
 * interleave into each display's own panel buffer (lfdpr_batch_panel). The
 * graph is captured on the first lfdpr_render_batch after creation or a
 * configuration change; later calls replay it with new model matrices. Each
 * scene's views, keys and panel are bit-identical to rendering it alone.
 */
typedef struct {
    int32_t branches;             /* concurrent graph branches for the per-scene stages, 1..32 */
    int32_t splat_blocks_per_sm;  /* persistent splat grid: blocks of 256 threads per SM, 1..64 */
    int32_t splat_slots;          /* views per lane in the splat: 1, 2, 3, 4, 6 or 8 */
} lfdpr_batch_config;

/*
 * lfdpr_create_batch: displays[i], meshes[i] for i < n (1 <= n <= 64); each
 * mesh uploaded to its display, each display at most once, rendered views
 * summed over the batch <= 4096. Default configuration: 4 branches, 16
 * blocks per SM, the fewest slots holding the largest view count (up to 8).
 * The batch borrows the displays and meshes: they must outlive it.
 * Errors: EINVAL, ENOMEM, ECUDA.
 */
lfdpr_status lfdpr_create_batch(lfdpr_display *const *displays, lfdpr_mesh *const *meshes, int32_t n,
                                lfdpr_batch **out);
lfdpr_status lfdpr_destroy_batch(lfdpr_batch *batch);
/* Read or replace the configuration (EINVAL outside the ranges above). */
lfdpr_status lfdpr_batch_get_config(const lfdpr_batch *batch, lfdpr_batch_config *out);
lfdpr_status lfdpr_batch_set_config(lfdpr_batch *batch, const lfdpr_batch_config *cfg);

/*
 * lfdpr_render_batch: models f32 [n][16] (host, row-major, as in
 * lfdpr_render_frame) for the scenes in order; asynchronous on `stream`.
 * The graph must be replayed from one host thread at a time. Per-scene
 * overflow is reported by lfdpr_frame_stats on that scene's display.
 * Errors: EINVAL (non-finite model), ECUDA.
 */
lfdpr_status lfdpr_render_batch(lfdpr_batch *batch, const float *models, void *stream);

/*
 * lfdpr_batch_autotune: time every configuration of a fixed candidate set
 * (branches x blocks per SM x slots) over `reps` replays each with the given
 * models, keep the fastest, and return it (and its mean ms per batch) if the
 * pointers are non-NULL. Synchronises `stream`. Errors: EINVAL, ECUDA.
 */
lfdpr_status lfdpr_batch_autotune(lfdpr_batch *batch, const float *models, int32_t reps, void *stream,
                                  lfdpr_batch_config *best, float *best_ms);

/* The last autotune's candidates and their mean ms per batch, in the order
 * tried: the first min(*n, capacity) entries are written (either array may be
 * NULL); *n is the number of candidates (0 before any autotune). */
lfdpr_status lfdpr_batch_autotune_table(const lfdpr_batch *batch, lfdpr_batch_config *cfgs, float *ms,
                                        int32_t capacity, int32_t *n);

/*
 * lfdpr_batch_scene_ms: per-scene frame latency of the last replayed batch:
 * ms[i] = device time from the start of the batch's graph to the end of
 * scene i's interleave (events recorded inside the graph), for i < n
 * (capacity >= n). Waits for the batch to finish. Errors: EINVAL (null, too
 * small, no batch rendered yet), ECUDA.
 */
lfdpr_status lfdpr_batch_scene_ms(const lfdpr_batch *batch, float *ms, int32_t capacity);

/* Device panel u8 [panel_h][panel_w][4] of scene i after lfdpr_render_batch
 * (borrowed; valid until the batch or its display is destroyed). */
lfdpr_status lfdpr_batch_panel(const lfdpr_batch *batch, int32_t i, const uint8_t **panel);

/*
 * Fault injection and allocation accounting (test hooks; the paper has no
 * counterpart). Every device and pinned-host allocation the library makes
 * goes through one layer that counts what is live. lfdpr_fault_inject_alloc
 * arms it: after `after` more successful allocations (0: the next one), one
 * allocation fails as if memory had run out, so the call making it returns
 * LFDPR_ENOMEM having freed what it had allocated; the hook then disarms.
 * -1 disarms it. Process-wide, all threads and devices. Errors: EINVAL
 * (after < -1).
 */
lfdpr_status lfdpr_fault_inject_alloc(int64_t after);

/*
 * lfdpr_checked_status: the checked build (liblfdpr_checked.so, compiled with
 * LFDPR_CHECKED: the frame kernels' global indices are range-checked, and an
 * out-of-range index skips its access and is recorded instead of faulting)
 * reports the first failing check site (0: none; 1-3 set-up vertex, texture
 * and material ids, 4 emitted point, 5 point triangle, 6-9 work and near
 * lists, 10-11 splat key, 12 resolve record, 13 view, 20-23 interleave
 * reads and panel writes, 24 view mip) and the number of failures since the
 * last reset (reset != 0 clears them). Synchronises the device. The regular
 * build returns EINVAL. Errors: EINVAL, ECUDA.
 */
lfdpr_status lfdpr_checked_status(uint32_t *first_site, uint64_t *failures, int32_t reset);

/* Allocations the library holds now (count and bytes) and has made in all
 * since the process started; any pointer may be NULL. */
lfdpr_status lfdpr_alloc_stats(int64_t *live_count, int64_t *live_bytes, int64_t *total_count);

/* Description of the last error on this thread ("" if none). */
const char *lfdpr_last_error(void);

/* LFDPR_VERSION of the library. */
int32_t lfdpr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LFDPR_H */
