"""Python binding of liblfdpr.so: argument marshalling only.

Every function here has the name of the C entry point it calls
(include/lfdpr.h) and converts arguments; all computation happens in the
library's CUDA kernels. Device memory and streams come from PyTorch tensors
(`data_ptr()`) and `torch.cuda.Stream.cuda_stream`. If the library is missing
or no GPU is present, the calls raise: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LFDPR_CHECKED=1 loads the checked build (index checks that record instead of
# faulting; see lfdpr_checked_status) in place of the regular one
CHECKED = os.environ.get("LFDPR_CHECKED", "") == "1"
LIB_PATH = os.path.join(_HERE, "liblfdpr_checked.so" if CHECKED else "liblfdpr.so")

OK, EINVAL, ENOMEM, ECUDA, EOVERFLOW, EDEVICE = range(6)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EOVERFLOW", 5: "EDEVICE"}
TRI_FLOATS = 32
TRI = dict(P0=0, s_u=3, eu=4, s_v=7, ev=8, umin=11, n=12, vmin=15, a1=16, b1=17, a2=18, b2=19,
           spl_uv=20, vpuv_min=21, vpuv_max=22, u_max=23, s0=24, sgu=25, sgv=26, t0=27, tgu=28,
           tgv=29, lod_min=30, lod_max=31)

# Names the C ABI exports (every declaration of include/lfdpr.h).
EXPORTS = ["lfdpr_create_display", "lfdpr_destroy_display", "lfdpr_upload_mesh",
           "lfdpr_destroy_mesh", "lfdpr_render_frame", "lfdpr_interleave", "lfdpr_frame_stats",
           "lfdpr_get_buffers", "lfdpr_view_eyes", "lfdpr_probe_atomic_min", "lfdpr_last_error",
           "lfdpr_version", "lfdpr_set_stage_timing", "lfdpr_set_splat_lane_limit", "lfdpr_sample_points_noalloc",
           "lfdpr_set_view_jitter", "lfdpr_set_recon_samples",
           "lfdpr_create_texture_set", "lfdpr_destroy_texture_set", "lfdpr_upload_mesh_textured",
           "lfdpr_upload_mesh_materials", "lfdpr_set_shading",
           "lfdpr_create_batch", "lfdpr_destroy_batch", "lfdpr_batch_get_config",
           "lfdpr_batch_set_config", "lfdpr_render_batch", "lfdpr_batch_autotune", "lfdpr_batch_panel",
           "lfdpr_batch_autotune_table", "lfdpr_batch_scene_ms", "lfdpr_set_spatial_supersampling",
           "lfdpr_set_view_band", "lfdpr_fault_inject_alloc", "lfdpr_alloc_stats",
           "lfdpr_checked_status",
           "lfdpr_recon_weight_count", "lfdpr_recon_bias_count", "lfdpr_create_recon",
           "lfdpr_destroy_recon", "lfdpr_recon_run", "lfdpr_recon_forward", "lfdpr_recon_status",
           "lfdpr_conv3x3_bf16", "lfdpr_warp_views"]


class LfdprError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class DisplayDesc(C.Structure):
    _fields_ = [("n_views", C.c_int32), ("view_w", C.c_int32), ("view_h", C.c_int32),
                ("cone_deg", C.c_float), ("view_dist", C.c_float), ("focal_w", C.c_float),
                ("focal_h", C.c_float), ("near_z", C.c_float), ("far_z", C.c_float),
                ("bias_h", C.c_float), ("bias_v", C.c_float),
                ("panel_w", C.c_int32), ("panel_h", C.c_int32),
                ("lens_pitch_px", C.c_float), ("slant", C.c_float), ("phase_offset", C.c_float),
                ("recon", C.c_int32), ("crosstalk", C.c_float), ("max_points", C.c_int64)]


N_STAGES = 8
STAGES = ["setup", "scan", "emit", "fetch", "clear", "splat", "resolve", "interleave"]


class Stats(C.Structure):
    _fields_ = [("n_points", C.c_int64), ("n_live_tris", C.c_int64), ("overflow", C.c_int32),
                ("cell_overflow", C.c_int32), ("kernel_launches", C.c_int64),
                ("n_splat_writes", C.c_int64),
                ("stage_ms", C.c_float * N_STAGES)]


class BatchConfig(C.Structure):
    _fields_ = [("branches", C.c_int32), ("splat_blocks_per_sm", C.c_int32), ("splat_slots", C.c_int32)]

    def as_tuple(self):
        return (self.branches, self.splat_blocks_per_sm, self.splat_slots)


class Buffers(C.Structure):
    _fields_ = [("counts", C.c_void_p), ("offsets", C.c_void_p), ("points", C.c_void_p),
                ("tri", C.c_void_p), ("keys", C.c_void_p), ("views", C.c_void_p),
                ("n_tris", C.c_int64), ("max_points", C.c_int64),
                ("n_render_views", C.c_int32), ("view_w", C.c_int32), ("view_h", C.c_int32),
                ("resolve", C.c_void_p), ("resolve_mat", C.c_void_p)]


SHADING_UNLIT, SHADING_PBR = 0, 1


class ShadingDesc(C.Structure):
    _fields_ = [("model", C.c_int32), ("light_dir", C.c_float * 3), ("light_rgb", C.c_float * 3),
                ("ambient", C.c_float * 3)]


_lib = None


def lib() -> C.CDLL:
    """Load liblfdpr.so (built by paper_2601_19901_gb300.build); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("liblfdpr.so is not built (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        P, S = C.c_void_p, C.c_int
        L.lfdpr_create_display.argtypes = [C.POINTER(DisplayDesc), C.POINTER(C.c_void_p)]
        L.lfdpr_destroy_display.argtypes = [P]
        L.lfdpr_upload_mesh.argtypes = [P, P, P, P, P, C.c_uint32, C.c_uint32, P, P, C.c_uint32,
                                        P, C.POINTER(C.c_void_p)]
        L.lfdpr_destroy_mesh.argtypes = [P]
        L.lfdpr_render_frame.argtypes = [P, P, P, P]
        L.lfdpr_interleave.argtypes = [P, P, P]
        L.lfdpr_frame_stats.argtypes = [P, P, C.POINTER(Stats)]
        L.lfdpr_get_buffers.argtypes = [P, P, C.POINTER(Buffers)]
        L.lfdpr_view_eyes.argtypes = [P, P, C.c_int32]
        L.lfdpr_set_stage_timing.argtypes = [P, C.c_int32]
        L.lfdpr_set_splat_lane_limit.argtypes = [P, C.c_uint32]
        L.lfdpr_set_view_jitter.argtypes = [P, P, C.c_int32]
        L.lfdpr_set_recon_samples.argtypes = [P, P, C.c_int32]
        L.lfdpr_set_spatial_supersampling.argtypes = [P, C.c_int32]
        L.lfdpr_set_view_band.argtypes = [P, C.c_int32]
        L.lfdpr_fault_inject_alloc.argtypes = [C.c_int64]
        L.lfdpr_alloc_stats.argtypes = [P, P, P]
        L.lfdpr_checked_status.argtypes = [P, P, C.c_int32]
        L.lfdpr_sample_points_noalloc.argtypes = [C.POINTER(DisplayDesc), P, P, P, P, P, C.c_uint32,
                                                  P, C.c_uint32, P, C.c_uint32, P, P, P]
        L.lfdpr_probe_atomic_min.argtypes = [P, C.c_uint64, P, P, C.c_uint64, C.c_int32, P]
        L.lfdpr_create_texture_set.argtypes = [P, P, C.c_uint32, P, C.POINTER(C.c_void_p)]
        L.lfdpr_destroy_texture_set.argtypes = [P]
        L.lfdpr_upload_mesh_materials.argtypes = [P, P, P, P, P, C.c_uint32, C.c_uint32, P, C.c_uint32, P, P,
                                                  C.POINTER(C.c_void_p)]
        L.lfdpr_set_shading.argtypes = [P, P]
        L.lfdpr_upload_mesh_textured.argtypes = [P, P, P, P, P, C.c_uint32, C.c_uint32, P, P,
                                                 C.POINTER(C.c_void_p)]
        L.lfdpr_create_batch.argtypes = [P, P, C.c_int32, C.POINTER(C.c_void_p)]
        L.lfdpr_destroy_batch.argtypes = [P]
        L.lfdpr_batch_get_config.argtypes = [P, C.POINTER(BatchConfig)]
        L.lfdpr_batch_set_config.argtypes = [P, C.POINTER(BatchConfig)]
        L.lfdpr_render_batch.argtypes = [P, P, P]
        L.lfdpr_batch_autotune.argtypes = [P, P, C.c_int32, P, C.POINTER(BatchConfig),
                                           C.POINTER(C.c_float)]
        L.lfdpr_batch_panel.argtypes = [P, C.c_int32, C.POINTER(C.c_void_p)]
        L.lfdpr_batch_autotune_table.argtypes = [P, P, P, C.c_int32, C.POINTER(C.c_int32)]
        L.lfdpr_batch_scene_ms.argtypes = [P, P, C.c_int32]
        L.lfdpr_recon_weight_count.argtypes = [C.c_int32]
        L.lfdpr_recon_bias_count.argtypes = [C.c_int32]
        L.lfdpr_create_recon.argtypes = [C.c_int32, C.c_int32, C.c_int32, P, C.c_int64, P, C.c_int64,
                                         C.POINTER(C.c_void_p)]
        L.lfdpr_destroy_recon.argtypes = [P]
        L.lfdpr_recon_run.argtypes = [P, P, P, P]
        L.lfdpr_recon_forward.argtypes = [P, P, P, P, P, C.c_float, P, P]
        L.lfdpr_recon_status.argtypes = [P, P]
        L.lfdpr_conv3x3_bf16.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, P, P, P, C.c_int32, P, P]
        L.lfdpr_warp_views.argtypes = [P, P, P, C.c_int32, P, C.c_int32, C.c_int32, C.c_int32, C.c_float, P, P]
        for name in EXPORTS:
            fn = getattr(L, name)
            if name == "lfdpr_last_error":
                fn.restype = C.c_char_p
                fn.argtypes = []
            elif name == "lfdpr_version":
                fn.restype = C.c_int32
                fn.argtypes = []
            elif name in ("lfdpr_recon_weight_count", "lfdpr_recon_bias_count"):
                fn.restype = C.c_int64
            else:
                fn.restype = S
        _lib = L
    return _lib


def _check(status: int):
    if status != OK:
        raise LfdprError(status, lib().lfdpr_last_error().decode())


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


def _stream(stream) -> Optional[int]:
    if stream is None:
        return None
    return int(getattr(stream, "cuda_stream", stream))


def desc_of(display, max_points: int = 0) -> DisplayDesc:
    d = display
    return DisplayDesc(d.n_views, d.view_w, d.view_h, d.cone_deg, d.view_dist, d.focal_w,
                       d.focal_h, d.near_z, d.far_z, d.bias_h, d.bias_v, d.panel_w, d.panel_h,
                       d.lens_pitch_px, d.slant, d.phase_offset, d.recon, d.crosstalk, max_points)


# ---------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def lfdpr_create_display(desc: DisplayDesc) -> int:
    h = C.c_void_p()
    _check(lib().lfdpr_create_display(C.byref(desc), C.byref(h)))
    return h.value


def lfdpr_set_spatial_supersampling(disp: int, level: int):
    _check(lib().lfdpr_set_spatial_supersampling(disp, int(level)))


def lfdpr_set_view_band(disp: int, band: int):
    _check(lib().lfdpr_set_view_band(disp, int(band)))


def lfdpr_fault_inject_alloc(after: int):
    _check(lib().lfdpr_fault_inject_alloc(int(after)))


def lfdpr_checked_status(reset: bool = False):
    """(first failing check site, failures) of the checked build."""
    site, n = C.c_uint32(0), C.c_uint64(0)
    _check(lib().lfdpr_checked_status(C.byref(site), C.byref(n), 1 if reset else 0))
    return site.value, n.value


def lfdpr_alloc_stats():
    """(live allocations, live bytes, allocations made since the process started)."""
    out = [C.c_int64(0) for _ in range(3)]
    _check(lib().lfdpr_alloc_stats(*[C.byref(o) for o in out]))
    return tuple(o.value for o in out)


def create_display(display, max_points: int = 0) -> int:
    """lfdpr_create_display from a scenes.Display, with its spatial
    supersampling level set."""
    h = lfdpr_create_display(desc_of(display, max_points))
    level = getattr(display, "ss_level", 0)
    if level:
        try:
            lfdpr_set_spatial_supersampling(h, level)
        except Exception:
            lfdpr_destroy_display(h)
            raise
    return h


def lfdpr_destroy_display(disp: int):
    _check(lib().lfdpr_destroy_display(disp))


def lfdpr_upload_mesh(disp: int, xyz: np.ndarray, uv: np.ndarray, idx: np.ndarray,
                      tri_tex: np.ndarray, textures: Sequence[np.ndarray], stream=None) -> int:
    xyz = np.ascontiguousarray(xyz, np.float32)
    uv = np.ascontiguousarray(uv, np.float32)
    idx = np.ascontiguousarray(idx, np.uint32)
    tri_tex = np.ascontiguousarray(tri_tex, np.uint32)
    texs = [np.ascontiguousarray(t, np.uint8) for t in textures]
    ptrs = (C.c_void_p * len(texs))(*[t.ctypes.data for t in texs])
    wh = np.array([[t.shape[1], t.shape[0]] for t in texs], np.uint32).ravel()
    h = C.c_void_p()
    _check(lib().lfdpr_upload_mesh(disp, _ptr(xyz), _ptr(uv), _ptr(idx), _ptr(tri_tex),
                                   xyz.shape[0], idx.reshape(-1, 3).shape[0], ptrs, _ptr(wh),
                                   len(texs), _stream(stream), C.byref(h)))
    return h.value


def lfdpr_destroy_mesh(mesh: int):
    _check(lib().lfdpr_destroy_mesh(mesh))


def lfdpr_render_frame(disp: int, mesh: int, model: np.ndarray, stream=None):
    m = np.ascontiguousarray(model, np.float32).ravel()
    _check(lib().lfdpr_render_frame(disp, mesh, _ptr(m), _stream(stream)))


def lfdpr_set_view_jitter(disp: int, u: np.ndarray):
    u = np.ascontiguousarray(u, np.float32).ravel()
    _check(lib().lfdpr_set_view_jitter(disp, _ptr(u), u.size))


def lfdpr_set_recon_samples(disp: int, samples: np.ndarray):
    s = np.ascontiguousarray(samples, np.float32).reshape(-1, 3)
    _check(lib().lfdpr_set_recon_samples(disp, _ptr(s), s.shape[0]))


def lfdpr_interleave(disp: int, panel_ptr: int, stream=None):
    _check(lib().lfdpr_interleave(disp, C.c_void_p(panel_ptr), _stream(stream)))


def lfdpr_frame_stats(disp: int, stream=None) -> Stats:
    st = Stats()
    _check(lib().lfdpr_frame_stats(disp, _stream(stream), C.byref(st)))
    return st


def lfdpr_set_stage_timing(disp: int, enable: bool):
    _check(lib().lfdpr_set_stage_timing(disp, 1 if enable else 0))


def lfdpr_set_splat_lane_limit(disp: int, limit: int):
    _check(lib().lfdpr_set_splat_lane_limit(disp, int(limit)))


def lfdpr_get_buffers(disp: int, mesh: int) -> Buffers:
    b = Buffers()
    _check(lib().lfdpr_get_buffers(disp, mesh, C.byref(b)))
    return b


def lfdpr_view_eyes(disp: int, n: int) -> np.ndarray:
    out = np.zeros(n, np.float32)
    _check(lib().lfdpr_view_eyes(disp, _ptr(out), n))
    return out


PROBE_RANDOM, PROBE_SHARED, PROBE_COHERENT = 0, 1, 2


def lfdpr_probe_atomic_min(words_ptr: int, n_words: int, idx_ptr: int, val_ptr: int, n_ops: int,
                           mode: int, stream=None):
    _check(lib().lfdpr_probe_atomic_min(C.c_void_p(words_ptr), n_words, C.c_void_p(idx_ptr),
                                        C.c_void_p(val_ptr), n_ops, int(mode), _stream(stream)))


NOALLOC_MAX_TRIS = 32768
NOALLOC_MAX_TEX = 256


def lfdpr_sample_points_noalloc(desc: DisplayDesc, model: np.ndarray, xyz_ptr: int, uv_ptr: int,
                                idx_ptr: int, tri_tex_ptr: int, n_tris: int, tex_wh: np.ndarray,
                                points_ptr: int, max_points: int, counts_ptr: int,
                                frame_counters_ptr: int, stream=None):
    """Point generation into caller-owned device buffers, allocating nothing
    (see include/lfdpr.h). Pointers are device addresses (e.g. data_ptr())."""
    m = np.ascontiguousarray(model, np.float32).ravel()
    wh = np.ascontiguousarray(tex_wh, np.uint32).ravel()
    _check(lib().lfdpr_sample_points_noalloc(C.byref(desc), _ptr(m), C.c_void_p(xyz_ptr),
                                             C.c_void_p(uv_ptr), C.c_void_p(idx_ptr),
                                             C.c_void_p(tri_tex_ptr), n_tris, _ptr(wh), len(wh) // 2,
                                             C.c_void_p(points_ptr), max_points,
                                             C.c_void_p(counts_ptr), C.c_void_p(frame_counters_ptr),
                                             _stream(stream)))


def lfdpr_version() -> int:
    return int(lib().lfdpr_version())


def _textures(textures: Sequence[np.ndarray]):
    texs = [np.ascontiguousarray(t, np.uint8) for t in textures]
    ptrs = (C.c_void_p * len(texs))(*[t.ctypes.data for t in texs])
    wh = np.array([[t.shape[1], t.shape[0]] for t in texs], np.uint32).ravel()
    return texs, ptrs, wh


def lfdpr_create_texture_set(textures: Sequence[np.ndarray], stream=None) -> int:
    texs, ptrs, wh = _textures(textures)
    h = C.c_void_p()
    _check(lib().lfdpr_create_texture_set(ptrs, _ptr(wh), len(texs), _stream(stream), C.byref(h)))
    return h.value


def lfdpr_destroy_texture_set(tex_set: int):
    _check(lib().lfdpr_destroy_texture_set(tex_set))


def lfdpr_upload_mesh_textured(disp: int, xyz: np.ndarray, uv: np.ndarray, idx: np.ndarray,
                               tri_tex: np.ndarray, tex_set: int, stream=None) -> int:
    xyz = np.ascontiguousarray(xyz, np.float32)
    uv = np.ascontiguousarray(uv, np.float32)
    idx = np.ascontiguousarray(idx, np.uint32)
    tri_tex = np.ascontiguousarray(tri_tex, np.uint32)
    h = C.c_void_p()
    _check(lib().lfdpr_upload_mesh_textured(disp, _ptr(xyz), _ptr(uv), _ptr(idx), _ptr(tri_tex),
                                            xyz.shape[0], idx.reshape(-1, 3).shape[0], tex_set,
                                            _stream(stream), C.byref(h)))
    return h.value


def lfdpr_upload_mesh_materials(disp: int, xyz: np.ndarray, uv: np.ndarray, idx: np.ndarray,
                                tri_mat: np.ndarray, mat_tex: np.ndarray, tex_set: int, stream=None) -> int:
    xyz = np.ascontiguousarray(xyz, np.float32)
    uv = np.ascontiguousarray(uv, np.float32)
    idx = np.ascontiguousarray(idx, np.uint32)
    tri_mat = np.ascontiguousarray(tri_mat, np.uint32)
    mat_tex = np.ascontiguousarray(mat_tex, np.uint32).reshape(-1, 4)
    h = C.c_void_p()
    _check(lib().lfdpr_upload_mesh_materials(disp, _ptr(xyz), _ptr(uv), _ptr(idx), _ptr(tri_mat), xyz.shape[0],
                                             idx.reshape(-1, 3).shape[0], _ptr(mat_tex), mat_tex.shape[0], tex_set,
                                             _stream(stream), C.byref(h)))
    return h.value


def lfdpr_set_shading(disp: int, shading=None):
    """shading: None (unlit) or an object with light_dir, light_rgb, ambient
    (three floats each; e.g. scenes.Shading) for physically based shading."""
    if shading is None:
        _check(lib().lfdpr_set_shading(disp, None))
        return
    d = ShadingDesc(SHADING_PBR, (C.c_float * 3)(*shading.light_dir), (C.c_float * 3)(*shading.light_rgb),
                    (C.c_float * 3)(*shading.ambient))
    _check(lib().lfdpr_set_shading(disp, C.byref(d)))


def lfdpr_create_batch(displays: Sequence[int], meshes: Sequence[int]) -> int:
    n = len(displays)
    dp = (C.c_void_p * n)(*displays)
    mp = (C.c_void_p * len(meshes))(*meshes)
    h = C.c_void_p()
    _check(lib().lfdpr_create_batch(dp, mp, n, C.byref(h)))
    return h.value


def lfdpr_destroy_batch(batch: int):
    _check(lib().lfdpr_destroy_batch(batch))


def lfdpr_batch_get_config(batch: int) -> BatchConfig:
    c = BatchConfig()
    _check(lib().lfdpr_batch_get_config(batch, C.byref(c)))
    return c


def lfdpr_batch_set_config(batch: int, branches: int, splat_blocks_per_sm: int, splat_slots: int):
    c = BatchConfig(branches, splat_blocks_per_sm, splat_slots)
    _check(lib().lfdpr_batch_set_config(batch, C.byref(c)))


def lfdpr_render_batch(batch: int, models: np.ndarray, stream=None):
    m = np.ascontiguousarray(models, np.float32).reshape(-1, 16)
    _check(lib().lfdpr_render_batch(batch, _ptr(m), _stream(stream)))


def lfdpr_batch_autotune(batch: int, models: np.ndarray, reps: int = 3, stream=None):
    m = np.ascontiguousarray(models, np.float32).reshape(-1, 16)
    c = BatchConfig()
    ms = C.c_float()
    _check(lib().lfdpr_batch_autotune(batch, _ptr(m), reps, _stream(stream), C.byref(c), C.byref(ms)))
    return c, ms.value


def lfdpr_batch_autotune_table(batch: int):
    """[(branches, splat_blocks_per_sm, splat_slots, ms), ...] of the last autotune."""
    n = C.c_int32()
    _check(lib().lfdpr_batch_autotune_table(batch, None, None, 0, C.byref(n)))
    cfgs = (BatchConfig * max(n.value, 1))()
    ms = (C.c_float * max(n.value, 1))()
    _check(lib().lfdpr_batch_autotune_table(batch, cfgs, ms, n.value, C.byref(n)))
    return [cfgs[k].as_tuple() + (ms[k],) for k in range(n.value)]


def lfdpr_batch_scene_ms(batch: int, n: int) -> np.ndarray:
    """Per-scene frame latency (ms) of the last replayed batch."""
    out = np.zeros(n, np.float32)
    _check(lib().lfdpr_batch_scene_ms(batch, _ptr(out), n))
    return out


def lfdpr_batch_panel(batch: int, i: int) -> int:
    h = C.c_void_p()
    _check(lib().lfdpr_batch_panel(batch, i, C.byref(h)))
    return h.value


def lfdpr_recon_weight_count(in_views: int) -> int:
    return int(lib().lfdpr_recon_weight_count(in_views))


def lfdpr_recon_bias_count(in_views: int) -> int:
    return int(lib().lfdpr_recon_bias_count(in_views))


def lfdpr_create_recon(view_w: int, view_h: int, in_views: int, weights_bf16: np.ndarray,
                       biases: np.ndarray) -> int:
    w = np.ascontiguousarray(weights_bf16, np.uint16).ravel()
    b = np.ascontiguousarray(biases, np.float32).ravel()
    h = C.c_void_p()
    _check(lib().lfdpr_create_recon(view_w, view_h, in_views, _ptr(w), w.size, _ptr(b), b.size, C.byref(h)))
    return h.value


def lfdpr_destroy_recon(recon: int):
    _check(lib().lfdpr_destroy_recon(recon))


def lfdpr_recon_run(recon: int, src_disp: int, dst_disp: int, stream=None):
    _check(lib().lfdpr_recon_run(recon, src_disp, dst_disp, _stream(stream)))


def lfdpr_recon_forward(recon: int, in_ptr: int, keys_ptr: int, in_eyes_ptr: int, out_eyes_ptr: int,
                        pixels_per_unit: float, out_ptr: int, stream=None):
    _check(lib().lfdpr_recon_forward(recon, C.c_void_p(in_ptr), C.c_void_p(keys_ptr), C.c_void_p(in_eyes_ptr),
                                     C.c_void_p(out_eyes_ptr), float(pixels_per_unit), C.c_void_p(out_ptr),
                                     _stream(stream)))


def lfdpr_warp_views(in_views_ptr: int, in_keys_ptr: int, in_eyes_ptr: int, in_count: int, out_eyes_ptr: int,
                     out_count: int, view_w: int, view_h: int, pixels_per_unit: float, out_ptr: int, stream=None):
    """Device pointers: RGBA8 views, u64 depth keys, f32 eye x arrays; see lfdpr_recon.h."""
    _check(lib().lfdpr_warp_views(C.c_void_p(in_views_ptr), C.c_void_p(in_keys_ptr), C.c_void_p(in_eyes_ptr),
                                  in_count, C.c_void_p(out_eyes_ptr), out_count, view_w, view_h,
                                  float(pixels_per_unit), C.c_void_p(out_ptr), _stream(stream)))


def lfdpr_recon_status(recon: int) -> int:
    f = C.c_int32(0)
    _check(lib().lfdpr_recon_status(recon, C.byref(f)))
    return int(f.value)


def lfdpr_conv3x3_bf16(in_ptr: int, H: int, W: int, cin: int, w_ptr: int, b_ptr: int, out_ptr: int,
                       cout: int, status_ptr: int, stream=None):
    _check(lib().lfdpr_conv3x3_bf16(C.c_void_p(in_ptr), H, W, cin, C.c_void_p(w_ptr), C.c_void_p(b_ptr),
                                    C.c_void_p(out_ptr), cout, C.c_void_p(status_ptr), _stream(stream)))


# ---------------------------------------------------------------------------
# Owning wrappers (destroy on close)
# ---------------------------------------------------------------------------

class Renderer:
    """One display and one mesh on the current CUDA device."""

    def __init__(self, display, scene, max_points: int = 0, stream=None, shading=None):
        """A scene with materials is uploaded as a mesh of materials (its
        textures as a texture set); `shading` (e.g. scenes.Shading) shades it
        physically."""
        self.display = display
        self.disp = create_display(display, max_points)
        self.mesh = None
        self.texset = None
        try:
            if getattr(scene, "materials", None) is not None:
                self.texset = TextureSet(scene.textures, stream)
                self.mesh = lfdpr_upload_mesh_materials(self.disp, scene.xyz, scene.uv, scene.idx, scene.tri_tex,
                                                        scene.materials, self.texset.handle, stream)
            else:
                self.mesh = lfdpr_upload_mesh(self.disp, scene.xyz, scene.uv, scene.idx,
                                              scene.tri_tex, scene.textures, stream)
            if shading is not None:
                lfdpr_set_shading(self.disp, shading)
        except Exception:
            if self.mesh is not None:
                lfdpr_destroy_mesh(self.mesh)
            if self.texset is not None:
                self.texset.close()
            lfdpr_destroy_display(self.disp)
            raise

    def render(self, model: np.ndarray, stream=None):
        lfdpr_render_frame(self.disp, self.mesh, model, stream)

    def interleave(self, panel_ptr: int, stream=None):
        lfdpr_interleave(self.disp, panel_ptr, stream)

    def set_view_jitter(self, u: np.ndarray):
        lfdpr_set_view_jitter(self.disp, u)

    def set_recon_samples(self, samples: np.ndarray):
        lfdpr_set_recon_samples(self.disp, samples)

    def stats(self, stream=None) -> Stats:
        return lfdpr_frame_stats(self.disp, stream)

    def set_stage_timing(self, enable: bool):
        lfdpr_set_stage_timing(self.disp, enable)

    def buffers(self) -> Buffers:
        return lfdpr_get_buffers(self.disp, self.mesh)

    def eyes(self) -> np.ndarray:
        return lfdpr_view_eyes(self.disp, self.display.n_render_views)

    def close(self):
        if self.mesh is not None:
            lfdpr_destroy_mesh(self.mesh)
            self.mesh = None
        if getattr(self, "texset", None) is not None:
            self.texset.close()
            self.texset = None
        if self.disp is not None:
            lfdpr_destroy_display(self.disp)
            self.disp = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TextureSet:
    """Textures uploaded once and shared by meshes."""

    def __init__(self, textures: Sequence[np.ndarray], stream=None):
        self.n_tex = len(textures)
        self.handle = lfdpr_create_texture_set(textures, stream)

    def close(self):
        if self.handle is not None:
            lfdpr_destroy_texture_set(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Several scenes, each with its own display and a mesh on a shared
    texture set, rendered and interleaved by one replayed CUDA graph."""

    def __init__(self, displays, scenes, tex_set: TextureSet, max_points: Sequence[int] = None,
                 stream=None):
        self.displays = list(displays)
        self.disps, self.meshes = [], []
        self.batch = None
        try:
            for k, (d, sc) in enumerate(zip(displays, scenes)):
                mp = max_points[k] if max_points is not None else 0
                self.disps.append(create_display(d, mp))
                self.meshes.append(lfdpr_upload_mesh_textured(self.disps[-1], sc.xyz, sc.uv, sc.idx,
                                                              sc.tri_tex, tex_set.handle, stream))
            self.batch = lfdpr_create_batch(self.disps, self.meshes)
        except Exception:
            self.close()
            raise

    def render(self, models: np.ndarray, stream=None):
        lfdpr_render_batch(self.batch, models, stream)

    def autotune(self, models: np.ndarray, reps: int = 3, stream=None):
        return lfdpr_batch_autotune(self.batch, models, reps, stream)

    def config(self) -> BatchConfig:
        return lfdpr_batch_get_config(self.batch)

    def set_config(self, branches: int, splat_blocks_per_sm: int, splat_slots: int):
        lfdpr_batch_set_config(self.batch, branches, splat_blocks_per_sm, splat_slots)

    def autotune_table(self):
        return lfdpr_batch_autotune_table(self.batch)

    def panel(self, i: int) -> int:
        return lfdpr_batch_panel(self.batch, i)

    def scene_ms(self) -> np.ndarray:
        return lfdpr_batch_scene_ms(self.batch, len(self.disps))

    def stats(self, i: int, stream=None) -> Stats:
        return lfdpr_frame_stats(self.disps[i], stream)

    def buffers(self, i: int) -> Buffers:
        return lfdpr_get_buffers(self.disps[i], self.meshes[i])

    def close(self):
        if self.batch is not None:
            lfdpr_destroy_batch(self.batch)
            self.batch = None
        for m in self.meshes:
            lfdpr_destroy_mesh(m)
        self.meshes = []
        for d in self.disps:
            lfdpr_destroy_display(d)
        self.disps = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Recon:
    """The learned angular reconstruction network (include/lfdpr_recon.h)."""

    def __init__(self, view_w: int, view_h: int, in_views: int, weights_bf16: np.ndarray, biases: np.ndarray):
        self.in_views = in_views
        self.handle = lfdpr_create_recon(view_w, view_h, in_views, weights_bf16, biases)

    def run(self, src_disp: int, dst_disp: int, stream=None):
        lfdpr_recon_run(self.handle, src_disp, dst_disp, stream)

    def forward(self, in_ptr: int, keys_ptr: int, in_eyes_ptr: int, out_eyes_ptr: int, pixels_per_unit: float,
                out_ptr: int, stream=None):
        lfdpr_recon_forward(self.handle, in_ptr, keys_ptr, in_eyes_ptr, out_eyes_ptr, pixels_per_unit, out_ptr,
                            stream)

    def status(self) -> int:
        return lfdpr_recon_status(self.handle)

    def close(self):
        if self.handle is not None:
            lfdpr_destroy_recon(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class _DeviceArray:
    """Describes library-owned device memory to torch (__cuda_array_interface__)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def device_view(ptr: int, shape, dtype):
    """A torch tensor aliasing device memory at `ptr` (no copy). 64-bit
    unsigned buffers are exposed as int64 (view the numpy copy as uint64)."""
    import torch
    dt = np.dtype(dtype)
    if dt == np.uint64:
        dt = np.dtype(np.int64)
    if dt == np.uint32:
        dt = np.dtype(np.int32)
    return torch.as_tensor(_DeviceArray(ptr, shape, dt.str), device="cuda")


def device_to_numpy(ptr: int, shape, dtype) -> np.ndarray:
    return device_view(ptr, shape, dtype).cpu().numpy().view(dtype).reshape(shape)
