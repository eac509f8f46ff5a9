"""Helpers of the GPU parity tests: run one frame through the C ABI, read the
library's buffers back, and compare them with the CPU oracle under the
parity tolerances:
  - per-triangle counts, sampling records and the point set: bit-exact;
  - splat: >= 99.9 % of view pixels carry the same winning point id;
  - colour: max |diff| <= 1 (of 255) on pixels with the same winner, and
    PSNR >= 50 dB over all pixels;
  - interleave: bit-exact given the same views.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional

import numpy as np

import oracle as O
from paper_2601_19901_gb300 import lfdpr

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
ID_AGREEMENT = 0.999
COLOUR_MAX_ABS = 1
PSNR_MIN_DB = 50.0

# Record fields compared bit for bit (oracle field -> library field).
FIELD_PAIRS = [("s_u", "s_u"), ("s_v", "s_v"), ("umin", "umin"), ("vmin", "vmin"),
               ("a1", "a1"), ("b1", "b1"), ("a2", "a2"), ("b2", "b2"),
               ("spl_uv", "spl_uv"), ("vpuv_min", "vpuv_min"), ("vpuv_max", "vpuv_max"),
               ("u_max", "u_max"), ("s0", "s0"), ("sgu", "sgu"), ("sgv", "sgv"), ("t0", "t0"),
               ("tgu", "tgu"), ("tgv", "tgv"), ("lod_min", "lod_min"), ("lod_max", "lod_max")]
VEC_PAIRS = [("p0", "P0"), ("n", "n"), ("eu", "eu"), ("ev", "ev")]


@dataclass
class GpuFrame:
    stats: object
    counts: np.ndarray
    offsets: np.ndarray
    tri: np.ndarray
    points: np.ndarray
    keys: np.ndarray
    views: np.ndarray
    panel: Optional[np.ndarray]
    eyes: np.ndarray


def gpu_frame(display, scene, model, max_points: int = 0, panel: bool = True,
              renderer: Optional[lfdpr.Renderer] = None) -> GpuFrame:
    import torch
    own = renderer is None
    R = renderer or lfdpr.Renderer(display, scene, max_points)
    try:
        s = torch.cuda.current_stream()
        R.render(model, s)
        pan = None
        if panel:
            pt = torch.zeros((display.panel_h, display.panel_w, 4), dtype=torch.uint8, device="cuda")
            R.interleave(pt.data_ptr(), s)
        st = R.stats(s)
        b = R.buffers()
        T = scene.n_tris
        nr = display.n_render_views
        H, W = display.view_h, display.view_w
        rd = lfdpr.device_to_numpy
        counts = rd(b.counts, (T,), np.uint32) if T else np.zeros(0, np.uint32)
        offsets = rd(b.offsets, (T,), np.uint32) if T else np.zeros(0, np.uint32)
        tri = rd(b.tri, (T, lfdpr.TRI_FLOATS), np.float32) if T else np.zeros((0, 32), np.float32)
        n = int(st.n_points) if not st.overflow else 0
        points = rd(b.points, (n, 4), np.uint32) if n else np.zeros((0, 4), np.uint32)
        keys = rd(b.keys, (nr, H, W), np.uint64)
        views = rd(b.views, (nr, H, W, 4), np.uint8)
        if panel:
            pan = pt.cpu().numpy()
        return GpuFrame(st, counts, offsets, tri, points, keys, views, pan, R.eyes())
    finally:
        if own:
            R.close()


def ids_of(keys: np.ndarray) -> np.ndarray:
    ids = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    ids[keys == EMPTY] = -1
    return ids


def psnr(a: np.ndarray, b: np.ndarray) -> float:
    mse = float(np.mean((a.astype(np.float64) - b.astype(np.float64)) ** 2))
    return math.inf if mse == 0 else 10.0 * math.log10(255.0 ** 2 / mse)


def check_sampling(g: GpuFrame, o, msg: str = ""):
    """Counts, records of live triangles and the point set: bit-exact."""
    assert np.array_equal(g.counts, o.counts), msg + " counts differ at %s" % np.nonzero(g.counts != o.counts)[0][:10]
    assert np.array_equal(g.offsets.astype(np.int64), o.offsets[:-1]), msg + " offsets"
    live = o.tri[:, O.F["live"]] == 1
    for fo, fl in FIELD_PAIRS:
        a = o.tri[live, O.F[fo]].view(np.uint32)
        b = g.tri[live, lfdpr.TRI[fl]].view(np.uint32)
        assert np.array_equal(a, b), msg + " field %s differs on %d triangles" % (fo, int((a != b).sum()))
    for fo, fl in VEC_PAIRS:
        a = o.tri[live, O.F[fo]:O.F[fo] + 3].view(np.uint32)
        b = g.tri[live, lfdpr.TRI[fl]:lfdpr.TRI[fl] + 3].view(np.uint32)
        assert np.array_equal(a, b), msg + " vector %s" % fo
    assert g.points.shape == o.points.shape, msg + " point count %s vs %s" % (g.points.shape, o.points.shape)
    assert np.array_equal(g.points[:, :2], o.points[:, :2]), msg + " point set"
    assert np.array_equal(g.points[:, 2:], o.points[:, 2:]), msg + " tv_min / tv_max"


def check_views(g: GpuFrame, o, views=None, msg: str = ""):
    """Winning ids >= 99.9 %; colour <= 1 LSB on same-id pixels; PSNR >= 50 dB."""
    vl = list(range(g.keys.shape[0])) if views is None else list(views)
    gk = g.keys[vl]
    gi, oi = ids_of(gk), ids_of(o.keys)
    agree = float(np.mean(gi == oi))
    assert agree >= ID_AGREEMENT, msg + " id agreement %.6f" % agree
    same = gi == oi
    gv = g.views[vl]
    diff = np.abs(gv.astype(np.int16) - o.rgba.astype(np.int16))
    assert diff[same].max(initial=0) <= COLOUR_MAX_ABS, msg + " colour max abs %d" % diff[same].max()
    p = psnr(gv, o.rgba)
    assert p >= PSNR_MIN_DB, msg + " PSNR %.2f dB" % p
    return agree, p
