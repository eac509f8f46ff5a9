"""CPU oracle for LFDPR: ctypes wrapper around oracle/lfdpr_oracle.c.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package smoke check and
by the benchmark's CPU-baseline leg. The product path (the CUDA library and its
binding) never imports this package, and this package never imports the
library; they share only the seeded inputs of paper_2601_19901_gb300.scenes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LFDPR_ORACLE_SRC names another copy of the oracle's source (a mutation run
# plants a mistake in such a copy and checks that the pins catch it); it is
# built next to itself.
_SRC = os.environ.get("LFDPR_ORACLE_SRC") or os.path.join(_HERE, "lfdpr_oracle.c")
_LIB = os.path.join(os.path.dirname(os.path.abspath(_SRC)), "liblfdpr_oracle.so") \
    if os.environ.get("LFDPR_ORACLE_SRC") else os.path.join(_HERE, "liblfdpr_oracle.so")
_lock = threading.Lock()
_lib = None

# per-triangle record layout written by orc_setup (indices into 48 floats)
TRI_FLOATS = 48
F = dict(live=0, p0=1, n=4, eu=7, ev=10, umin=13, vmin=14, a1=15, b1=16, a2=17,
         b2=18, U=19, V=22, A_ws=25, A_ts=26, n_tex=27, size_uv=28, d_min=29,
         d_max=30, s_u=31, s_v=32, vpuv_min=33, vpuv_max=34, spl_uv=35,
         lod_min=36, lod_max=37, s0=38, sgu=39, sgv=40, t0=41, tgu=42, tgv=43,
         tex=44, u_max=45, v_max=46)


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler: strict IEEE binary32, no
    contraction of a*b+c into fma other than the explicit fmaf() calls."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off",
           "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class OrcDisplay(C.Structure):
    _fields_ = [("n_views", C.c_int32), ("view_w", C.c_int32), ("view_h", C.c_int32),
                ("cone_deg", C.c_float), ("view_dist", C.c_float), ("focal_w", C.c_float),
                ("focal_h", C.c_float), ("near_z", C.c_float), ("far_z", C.c_float),
                ("bias_h", C.c_float), ("bias_v", C.c_float),
                ("panel_w", C.c_int32), ("panel_h", C.c_int32),
                ("lens_pitch_px", C.c_float), ("slant", C.c_float), ("phase_offset", C.c_float),
                ("recon", C.c_int32), ("crosstalk", C.c_float),
                ("jitter", C.c_void_p), ("samples", C.c_void_p), ("n_samples", C.c_int32),
                ("ss_level", C.c_int32)]


def _disp(d, jitter=None, samples=None) -> OrcDisplay:
    """The C display. jitter (float32 [rendered views], each in [0, 1]) places
    each rendered view in its interval; samples (float32 [n][3]: dx, dy in
    view pixels, dphi in display views) drive Gaussian reconstruction. Both
    arrays are kept alive on the returned structure."""
    o = OrcDisplay(d.n_views, d.view_w, d.view_h, d.cone_deg, d.view_dist,
                   d.focal_w, d.focal_h, d.near_z, d.far_z, d.bias_h, d.bias_v,
                   d.panel_w, d.panel_h, d.lens_pitch_px, d.slant, d.phase_offset,
                   d.recon, d.crosstalk, None, None, 0, getattr(d, "ss_level", 0))
    if jitter is not None:
        o._jitter = np.ascontiguousarray(jitter, np.float32)
        o.jitter = o._jitter.ctypes.data
    if samples is not None:
        o._samples = np.ascontiguousarray(samples, np.float32).reshape(-1, 3)
        o.samples = o._samples.ctypes.data
        o.n_samples = o._samples.shape[0]
    return o


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            L.orc_log2f.restype = C.c_float
            L.orc_log2f.argtypes = [C.c_float]
            L.orc_n_render_views.restype = C.c_int
            L.orc_n_render_views.argtypes = [P]
            L.orc_eyes.argtypes = [P, P]
            L.orc_mip_levels.restype = C.c_int
            L.orc_mip_levels.argtypes = [C.c_uint32, C.c_uint32]
            L.orc_mip_bytes.restype = C.c_size_t
            L.orc_mip_bytes.argtypes = [C.c_uint32, C.c_uint32]
            L.orc_build_mips.argtypes = [P, C.c_uint32, C.c_uint32, P]
            L.orc_trilinear.argtypes = [P, C.c_uint32, C.c_uint32, C.c_float, C.c_float, C.c_float, P]
            L.orc_transform.argtypes = [P, P, P]
            L.orc_setup.restype = C.c_int
            L.orc_setup.argtypes = [P, P, P, P, P, C.c_uint32, P, C.c_uint32, P, P, P]
            L.orc_emit.restype = C.c_int64
            L.orc_emit.argtypes = [P, P, C.c_uint32, P, C.c_int64]
            L.orc_fetch.argtypes = [P, P, C.c_int64, P, P]
            L.orc_splat.argtypes = [P, P, P, C.c_int64, P, C.c_int, P]
            L.orc_resolve.argtypes = [P, P, P, P, P, C.c_int, P]
            L.orc_splat_hits.argtypes = [P, P, P, C.c_int64, P, C.c_int, P]
            L.orc_display_views.argtypes = [P, P, P]
            L.orc_view_of_subpixel.restype = C.c_int
            L.orc_view_of_subpixel.argtypes = [P, C.c_int, C.c_int, C.c_int]
            L.orc_interleave.argtypes = [P, P, P]
            L.orc_view_mip.argtypes = [P, C.c_int, C.c_int, C.c_int, P]
            L.orc_view_pos.restype = C.c_float
            L.orc_view_pos.argtypes = [P, C.c_int]
            L.orc_subpixel_phase.restype = C.c_float
            L.orc_subpixel_phase.argtypes = [P, C.c_int, C.c_int, C.c_int]
            L.orc_setup_mat.restype = C.c_int
            L.orc_setup_mat.argtypes = [P, P, P, P, P, C.c_uint32, P, C.c_uint32, P, C.c_uint32, P, P, P]
            L.orc_fetch_mat.argtypes = [P, P, C.c_int64, P, P, P, P]
            L.orc_resolve_pbr.argtypes = [P, P, P, P, P, P, C.c_int, P, P]
            L.orc_pbr_shade.argtypes = [P, C.c_double, C.c_double, P, P, P, P, P, P]
            L.orc_splat_area_px.restype = C.c_float
            L.orc_splat_area_px.argtypes = [P, P, C.c_int, C.c_int, C.c_float]
            L.orc_raycast.restype = C.c_int32
            L.orc_raycast.argtypes = [P, P, C.c_uint32, C.c_int, C.c_int, C.c_int,
                                      C.POINTER(C.c_double)]
            _lib = L
    return _lib


class OrcShading(C.Structure):
    _fields_ = [("light_dir", C.c_float * 3), ("light_rgb", C.c_float * 3), ("ambient", C.c_float * 3)]


def _shading(sh) -> OrcShading:
    return OrcShading((C.c_float * 3)(*sh.light_dir), (C.c_float * 3)(*sh.light_rgb), (C.c_float * 3)(*sh.ambient))


def pbr_shade(albedo, rough: float, metal: float, n, v, l, light_rgb, ambient) -> np.ndarray:
    """The oracle's BRDF for one sample (unit vectors n, v, l): linear RGB
    before clamping."""
    a = np.ascontiguousarray(albedo, np.float64)
    vecs = [np.ascontiguousarray(x, np.float64) for x in (n, v, l)]
    lr = np.ascontiguousarray(light_rgb, np.float32)
    am = np.ascontiguousarray(ambient, np.float32)
    out = np.zeros(3, np.float64)
    lib().orc_pbr_shade(_p(a), float(rough), float(metal), _p(vecs[0]), _p(vecs[1]), _p(vecs[2]), _p(lr), _p(am),
                        _p(out))
    return out


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------------------
# Unit-level entry points (used by the pins)
# ---------------------------------------------------------------------------

def log2f(x: float) -> float:
    return float(lib().orc_log2f(C.c_float(x)))


def eyes(d, jitter=None) -> np.ndarray:
    dd = _disp(d, jitter)
    out = np.zeros(lib().orc_n_render_views(C.byref(dd)), np.float32)
    lib().orc_eyes(C.byref(dd), _p(out))
    return out


def mip_chain(tex: np.ndarray) -> np.ndarray:
    h, w = tex.shape[:2]
    tex = np.ascontiguousarray(tex, np.uint8)
    out = np.zeros(lib().orc_mip_bytes(w, h), np.uint8)
    lib().orc_build_mips(_p(tex), w, h, _p(out))
    return out


def mip_levels(chain: np.ndarray, w: int, h: int):
    """Split a chain into a list of (h_l, w_l, 4) arrays."""
    out, off, l = [], 0, 0
    while True:
        lw, lh = max(1, w >> l), max(1, h >> l)
        out.append(chain[off:off + lw * lh * 4].reshape(lh, lw, 4))
        off += lw * lh * 4
        if lw == 1 and lh == 1:
            return out
        l += 1


def trilinear(chain: np.ndarray, w: int, h: int, s: float, t: float, lod: float) -> np.ndarray:
    out = np.zeros(4, np.uint8)
    lib().orc_trilinear(_p(chain), w, h, C.c_float(s), C.c_float(t), C.c_float(lod), _p(out))
    return out


def view_of_subpixel(d, x: int, y: int, c: int) -> int:
    dd = _disp(d)
    return int(lib().orc_view_of_subpixel(C.byref(dd), x, y, c))


def subpixel_phase(d, x: int, y: int, c: int) -> float:
    dd = _disp(d)
    return float(lib().orc_subpixel_phase(C.byref(dd), x, y, c))


def view_pos(d, m: int, jitter=None) -> float:
    dd = _disp(d, jitter)
    return float(lib().orc_view_pos(C.byref(dd), m))


def transform(model: np.ndarray, xyz: np.ndarray) -> np.ndarray:
    """(n, 3) float32 points through orc_transform (the per-frame model
    transform, affine rows 0-2 of the row-major 4x4 `model`)."""
    L = lib()
    m = np.ascontiguousarray(model, np.float32).ravel()
    v = np.ascontiguousarray(xyz, np.float32).reshape(-1, 3)
    out = np.zeros_like(v)
    for k in range(len(v)):
        L.orc_transform(_p(m), _p(v[k]), _p(out[k]))
    return out


def transformed_tris(scene, model: np.ndarray) -> np.ndarray:
    """(T, 9) float32 transformed triangle vertices (same fmaf sequence as setup)."""
    L = lib()
    m = np.ascontiguousarray(model, np.float32).ravel()
    v = np.ascontiguousarray(scene.xyz, np.float32)
    tv = np.zeros_like(v)
    o = np.zeros(3, np.float32)
    for k in range(len(v)):
        L.orc_transform(_p(m), _p(v[k]), _p(o))
        tv[k] = o
    return np.ascontiguousarray(tv[scene.idx.astype(np.int64)].reshape(-1, 9))


def splat_area_px(d, rec_row: np.ndarray, i: int, j: int, ex: float) -> float:
    """Eq. 8's projected splat area (view pixels) of lattice cell (i, j) of
    one triangle's record, in the view of eye x `ex`."""
    dd = _disp(d)
    r = np.ascontiguousarray(rec_row, np.float32)
    assert r.shape == (TRI_FLOATS,)
    return float(lib().orc_splat_area_px(C.byref(dd), _p(r), i, j, C.c_float(ex)))


def raycast(d, txyz: np.ndarray, v: int, x: int, y: int):
    dd = _disp(d)
    t = C.c_double(0.0)
    tri = lib().orc_raycast(C.byref(dd), _p(txyz), txyz.shape[0], v, x, y, C.byref(t))
    return int(tri), float(t.value)


# ---------------------------------------------------------------------------
# Whole frame
# ---------------------------------------------------------------------------

@dataclass
class Frame:
    status: int
    tri: np.ndarray          # (T, 48) float32
    counts: np.ndarray       # (T,) uint32
    points: np.ndarray       # (P, 4) uint32: tri, i | j << 16, tv_min, tv_max
    views_list: Optional[np.ndarray] = None
    keys: Optional[np.ndarray] = None    # (n_list, H, W) uint64
    rgba: Optional[np.ndarray] = None    # (n_list, H, W, 4) uint8
    panel: Optional[np.ndarray] = None   # (Hp, Wp, 4) uint8
    tvx: Optional[np.ndarray] = None     # (P, 6) uint32: normal, roughness, metallic tv_min / tv_max (materials)

    @property
    def offsets(self) -> np.ndarray:
        o = np.zeros(len(self.counts) + 1, np.int64)
        np.cumsum(self.counts, out=o[1:])
        return o


class Textures:
    """Mip chains of a scene's textures, built once by the oracle."""

    def __init__(self, textures: Sequence[np.ndarray]):
        self.chains = [mip_chain(t) for t in textures]
        self.wh = np.array([[t.shape[1], t.shape[0]] for t in textures], np.uint32).ravel()
        self.ptrs = (C.c_void_p * len(self.chains))(*[c.ctypes.data for c in self.chains])


def setup(d, scene, model, tex_wh=None, jitter=None):
    """Steps 1-7 only: per-triangle records and point counts. tex_wh overrides
    the texture sizes (setup reads sizes, never texels)."""
    dd = _disp(d, jitter)
    T = scene.n_tris
    tri = np.zeros((T, TRI_FLOATS), np.float32)
    counts = np.zeros(T, np.uint32)
    if tex_wh is None:
        wh = np.array([[t.shape[1], t.shape[0]] for t in scene.textures], np.uint32).ravel()
    else:
        wh = np.ascontiguousarray(tex_wh, np.uint32).ravel()
    args = (C.byref(dd), _p(np.ascontiguousarray(scene.xyz, np.float32)),
            _p(np.ascontiguousarray(scene.uv, np.float32)), _p(np.ascontiguousarray(scene.idx, np.uint32)),
            _p(np.ascontiguousarray(scene.tri_tex, np.uint32)), T, _p(wh), len(wh) // 2)
    mdl = _p(np.ascontiguousarray(model, np.float32).ravel())
    if getattr(scene, "materials", None) is not None:
        mats = np.ascontiguousarray(scene.materials, np.uint32)
        st = lib().orc_setup_mat(*args, _p(mats), mats.shape[0], mdl, _p(tri), _p(counts))
    else:
        st = lib().orc_setup(*args, mdl, _p(tri), _p(counts))
    return st, tri, counts


def emit(tri: np.ndarray, counts: np.ndarray) -> np.ndarray:
    total = int(counts.sum(dtype=np.int64))
    points = np.zeros((max(total, 1), 4), np.uint32)
    n = lib().orc_emit(_p(tri), _p(counts), len(counts), _p(points), total)
    assert n == total
    return points[:total]


def render(d, scene, model, views: Optional[Sequence[int]] = None, panel: bool = True,
           textures: Optional[Textures] = None, splat: bool = True, jitter=None, samples=None,
           shading=None) -> Frame:
    """One frame through every oracle step. `views` lists the rendered views
    to splat and resolve (default all); the panel needs all of them. jitter
    and samples: see _disp. A scene with materials is sampled by Eq. 1 over
    all four of a triangle's textures and fetches all four; `shading` (a
    scenes.Shading) shades it physically (else the albedo is drawn unlit)."""
    L = lib()
    dd = _disp(d, jitter, samples)
    st, tri, counts = setup(d, scene, model, jitter=jitter)
    total = int(counts.sum(dtype=np.int64))
    points = np.zeros((max(total, 1), 4), np.uint32)
    n = L.orc_emit(_p(tri), _p(counts), scene.n_tris, _p(points), total)
    assert n == total
    points = points[:total]
    tx = textures or Textures(scene.textures)
    mats = getattr(scene, "materials", None)
    tvx = None
    if mats is not None:
        mats = np.ascontiguousarray(mats, np.uint32)
        tvx = np.zeros((max(total, 1), 6), np.uint32)
        L.orc_fetch_mat(_p(tri), _p(points), total, tx.ptrs, _p(tx.wh), _p(mats), _p(tvx))
        tvx = tvx[:total]
    else:
        assert shading is None, "physically based shading needs a scene with materials"
        L.orc_fetch(_p(tri), _p(points), total, tx.ptrs, _p(tx.wh))
    fr = Frame(status=st, tri=tri, counts=counts, points=points)
    fr.tvx = tvx
    if not splat:
        return fr
    nr = d.n_render_views
    vl = np.arange(nr, dtype=np.int32) if views is None else np.asarray(views, np.int32)
    keys = np.zeros((len(vl), d.view_h, d.view_w), np.uint64)
    L.orc_splat(C.byref(dd), _p(tri), _p(points), total, _p(vl), len(vl), _p(keys))
    rgba = np.zeros((len(vl), d.view_h, d.view_w, 4), np.uint8)
    if shading is not None:
        sh = _shading(shading)
        tv = np.ascontiguousarray(tvx if total else np.zeros((1, 6), np.uint32))
        L.orc_resolve_pbr(C.byref(dd), _p(tri), _p(points), _p(tv), _p(keys), _p(vl), len(vl), C.byref(sh),
                          _p(rgba))
    else:
        L.orc_resolve(C.byref(dd), _p(tri), _p(points), _p(keys), _p(vl), len(vl), _p(rgba))
    fr.views_list, fr.keys, fr.rgba = vl, keys, rgba
    if panel:
        assert len(vl) == nr and np.all(vl == np.arange(nr)), "the panel needs every view"
        pan = np.zeros((d.panel_h, d.panel_w, 4), np.uint8)
        L.orc_interleave(C.byref(dd), _p(rgba), _p(pan))
        fr.panel = pan
    return fr


def splat_hits(d, tri: np.ndarray, points: np.ndarray, views: Sequence[int]) -> np.ndarray:
    """Per pixel of each listed view: number of splats passing every test."""
    dd = _disp(d)
    vl = np.asarray(views, np.int32)
    hits = np.zeros((len(vl), d.view_h, d.view_w), np.uint32)
    pts = np.ascontiguousarray(points, np.uint32)
    lib().orc_splat_hits(C.byref(dd), _p(tri), _p(pts), len(pts), _p(vl), len(vl), _p(hits))
    return hits


def splat_resolve(d, tri: np.ndarray, points: np.ndarray, views: Sequence[int], jitter=None,
                  tvx: Optional[np.ndarray] = None, shading=None):
    """Steps 9-10 for the listed views, from existing records and points
    (with `shading`, the physically based resolve of a mesh of materials,
    whose other maps' values `tvx` orc_fetch_mat wrote)."""
    dd = _disp(d, jitter)
    vl = np.asarray(views, np.int32)
    pts = np.ascontiguousarray(points, np.uint32)
    keys = np.zeros((len(vl), d.view_h, d.view_w), np.uint64)
    lib().orc_splat(C.byref(dd), _p(tri), _p(pts), len(pts), _p(vl), len(vl), _p(keys))
    rgba = np.zeros((len(vl), d.view_h, d.view_w, 4), np.uint8)
    if shading is not None:
        sh = _shading(shading)
        tv = np.ascontiguousarray(tvx if tvx is not None and len(tvx) else np.zeros((1, 6), np.uint32), np.uint32)
        lib().orc_resolve_pbr(C.byref(dd), _p(tri), _p(pts), _p(tv), _p(keys), _p(vl), len(vl), C.byref(sh),
                              _p(rgba))
    else:
        lib().orc_resolve(C.byref(dd), _p(tri), _p(pts), _p(keys), _p(vl), len(vl), _p(rgba))
    return keys, rgba


def interleave(d, rendered: np.ndarray, jitter=None, samples=None) -> np.ndarray:
    dd = _disp(d, jitter, samples)
    pan = np.zeros((d.panel_h, d.panel_w, 4), np.uint8)
    lib().orc_interleave(C.byref(dd), _p(np.ascontiguousarray(rendered, np.uint8)), _p(pan))
    return pan


def view_mip(view: np.ndarray, level: int) -> np.ndarray:
    """Mip level `level` of one RGBA8 view (h, w, 4)."""
    h, w = view.shape[:2]
    out = np.zeros((h >> level, w >> level, 4), np.uint8)
    lib().orc_view_mip(_p(np.ascontiguousarray(view, np.uint8)), w, h, level, _p(out))
    return out


def display_views(d, rendered: np.ndarray) -> np.ndarray:
    dd = _disp(d)
    out = np.zeros((d.n_views, d.view_h, d.view_w, 4), np.float32)
    lib().orc_display_views(C.byref(dd), _p(np.ascontiguousarray(rendered, np.uint8)), _p(out))
    return out
