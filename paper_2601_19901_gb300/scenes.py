"""Seeded synthetic inputs: display presets, procedural meshes, value-noise textures.

This module holds no step of the rendering method. It only produces the data
that both the CUDA library and the CPU oracle consume, so that the two sides
see identical inputs. Every generator is deterministic given its seed.

The paper measures on four real scenes (sponza, gallery, coconut, car; Sec. 5.1)
that are not available here; the procedural scenes below stand in for them,
shaped like the paper's workloads: about a million triangles tessellated small
(the paper bounds triangles at about a hundred pixels, Sec. 5.1), textures whose
texel density varies by three orders of magnitude, and a scene that rotates
about its centre every frame (Sec. 5.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np


# ----------------------------------------------------------------------------
# Display presets
# ----------------------------------------------------------------------------

@dataclass(frozen=True)
class Display:
    """A horizontal-parallax lenticular display and its rendered views.

    Views are pinhole cameras on the line y = 0, z = view_dist, all looking
    down -z through one shared focal rectangle of focal_w x focal_h at z = 0.
    """
    n_views: int
    view_w: int
    view_h: int
    cone_deg: float
    view_dist: float
    focal_w: float
    focal_h: float
    near_z: float
    far_z: float
    bias_h: float
    bias_v: float
    panel_w: int
    panel_h: int
    lens_pitch_px: float
    slant: float
    phase_offset: float = 0.0
    # 0: render n_views; 1: render 2*n_views, tent down to n_views; 2: render
    # 2*n_views, Gaussian reconstruction; 3: render n_views, Gaussian reconstruction
    recon: int = 0
    crosstalk: float = 0.0  # weight of each +-1 neighbour view before interleave
    # spatial supersampling: the views are rendered at 2^ss_level times the
    # output resolution and the interleave reads mip level ss_level of each
    ss_level: int = 0

    @property
    def n_render_views(self) -> int:
        return self.n_views * (2 if self.recon in (1, 2) else 1)


@dataclass(frozen=True)
class Shading:
    """Physically based shading of scenes with materials: one directional
    light (direction toward the light, radiance per channel) and a constant
    ambient term times albedo."""
    light_dir: tuple = (0.35, 0.8, 0.5)
    light_rgb: tuple = (2.4, 2.3, 2.1)
    ambient: tuple = (0.10, 0.10, 0.12)


def display_tiny() -> Display:
    """8 views over a 30 degree cone, 128x128 each, 512x512 panel, 8 views per
    lenslet with slant 1/6, horizontal:vertical sampling bias 4:1."""
    return Display(n_views=8, view_w=128, view_h=128, cone_deg=30.0,
                   view_dist=4.0, focal_w=2.4, focal_h=2.4,
                   near_z=0.1, far_z=100.0, bias_h=4.0, bias_v=1.0,
                   panel_w=512, panel_h=512, lens_pitch_px=8.0,
                   slant=1.0 / 6.0)


def display_paper() -> Display:
    """48 views over a 40 degree cone, 420 (w) x 560 (h) each, 2560x1600 panel,
    lenslet slant 0.2. The focal rectangle keeps view pixels square."""
    return Display(n_views=48, view_w=420, view_h=560, cone_deg=40.0,
                   view_dist=4.0, focal_w=1.8, focal_h=2.4,
                   near_z=0.1, far_z=100.0, bias_h=1.0, bias_v=1.0,
                   panel_w=2560, panel_h=1600, lens_pitch_px=8.0, slant=0.2)


def display_angular_ss() -> Display:
    """The 48-view display rendered at twice the angular rate (96 views),
    tent-reconstructed to 48, with +-1 neighbour crosstalk of 0.15."""
    return replace(display_paper(), recon=1, crosstalk=0.15)


# ----------------------------------------------------------------------------
# Scenes
# ----------------------------------------------------------------------------

@dataclass
class Scene:
    xyz: np.ndarray        # (V, 3) float32, object space
    uv: np.ndarray         # (V, 2) float32, texture coordinates (wrap addressing)
    idx: np.ndarray        # (T, 3) uint32 vertex indices
    tri_tex: np.ndarray    # (T,) uint32 texture id per triangle (material id when `materials` is set)
    textures: List[np.ndarray] = field(default_factory=list)  # (h, w, 4) uint8
    centre: tuple = (0.0, 0.0, 0.0)
    # (M, 4) uint32 texture ids of each material: albedo, normal, roughness, metallic
    materials: Optional[np.ndarray] = None

    @property
    def n_tris(self) -> int:
        return int(self.idx.shape[0])


def model_matrix(frame: int, deg_per_frame: float = 3.0,
                 centre=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Row-major 4x4 float32: rotation about the vertical axis through
    `centre` by frame * deg_per_frame degrees (the scene turns every frame)."""
    a = math.radians(frame * deg_per_frame)
    c, s = math.cos(a), math.sin(a)
    cx, cy, cz = centre
    m = np.array([[c, 0.0, s, 0.0],
                  [0.0, 1.0, 0.0, 0.0],
                  [-s, 0.0, c, 0.0],
                  [0.0, 0.0, 0.0, 1.0]], dtype=np.float64)
    t0 = np.eye(4)
    t0[:3, 3] = [-cx, -cy, -cz]
    t1 = np.eye(4)
    t1[:3, 3] = [cx, cy, cz]
    return (t1 @ m @ t0).astype(np.float32)


# -- textures -----------------------------------------------------------------

def _periodic_interp(n_out: int, n_lat: int) -> np.ndarray:
    """(n_out, n_lat) matrix: smoothstep interpolation of a periodic lattice."""
    x = (np.arange(n_out) + 0.5) * (n_lat / n_out)
    i0 = np.floor(x).astype(np.int64)
    f = x - i0
    s = f * f * (3.0 - 2.0 * f)
    m = np.zeros((n_out, n_lat), np.float64)
    rows = np.arange(n_out)
    np.add.at(m, (rows, i0 % n_lat), 1.0 - s)
    np.add.at(m, (rows, (i0 + 1) % n_lat), s)
    return m.astype(np.float32)


def value_noise_texture(w: int, h: int, seed: int, base: int = 8,
                        octaves: int = 4) -> np.ndarray:
    """Tileable RGBA8 value noise: per channel, `octaves` octaves of a periodic
    random lattice (base, 2*base, ... cells across) with smoothstep
    interpolation; alpha is 255."""
    rng = np.random.default_rng(seed)
    out = np.empty((h, w, 4), np.uint8)
    for ch in range(3):
        acc = np.zeros((h, w), np.float32)
        amp, tot = 1.0, 0.0
        for k in range(octaves):
            lx = min(base << k, w)
            ly = min(base << k, h)
            g = rng.random((ly, lx), dtype=np.float32)
            my = _periodic_interp(h, ly)
            mx = _periodic_interp(w, lx)
            acc += amp * (my @ g @ mx.T)
            tot += amp
            amp *= 0.5
        acc /= tot
        lo, hi = float(acc.min()), float(acc.max())
        acc = (acc - lo) / max(hi - lo, 1e-6)
        out[:, :, ch] = np.clip(np.rint(acc * 255.0), 0, 255).astype(np.uint8)
    out[:, :, 3] = 255
    return out


def normal_map_texture(w: int, h: int, seed: int, strength: float = 2.0, base: int = 8) -> np.ndarray:
    """Tangent-space normal map (RGBA8, n = 2 c / 255 - 1) of a tileable
    value-noise height field: n = normalize(-s dh/dx, -s dh/dy, 1), with
    periodic central differences in texels scaled to the unit square."""
    hgt = value_noise_texture(w, h, seed, base)[:, :, 0].astype(np.float64) / 255.0
    dx = (np.roll(hgt, -1, 1) - np.roll(hgt, 1, 1)) * (w / 2.0) / w * 8.0
    dy = (np.roll(hgt, -1, 0) - np.roll(hgt, 1, 0)) * (h / 2.0) / h * 8.0
    n = np.stack([-strength * dx, -strength * dy, np.ones_like(hgt)], -1)
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    out = np.empty((h, w, 4), np.uint8)
    out[:, :, :3] = np.clip(np.rint((n * 0.5 + 0.5) * 255.0), 0, 255).astype(np.uint8)
    out[:, :, 3] = 255
    return out


def scalar_texture(w: int, h: int, seed: int, lo: float, hi: float, sharpen: float = 1.0) -> np.ndarray:
    """Tileable scalar map in R (G = B = R, alpha 255): value noise mapped to
    [lo, hi]; sharpen > 1 pushes it towards the ends (a mostly binary mask)."""
    v = value_noise_texture(w, h, seed)[:, :, 0].astype(np.float64) / 255.0
    if sharpen != 1.0:
        v = np.clip((v - 0.5) * sharpen + 0.5, 0.0, 1.0)
    c = np.clip(np.rint((lo + (hi - lo) * v) * 255.0), 0, 255).astype(np.uint8)
    out = np.empty((h, w, 4), np.uint8)
    out[:, :, 0] = out[:, :, 1] = out[:, :, 2] = c
    out[:, :, 3] = 255
    return out


def material_textures(sizes, seed: int) -> List[np.ndarray]:
    """One material's four textures, sizes (albedo, normal, roughness,
    metallic) square powers of two: value-noise albedo, a normal map, roughness
    in [0.15, 0.95], a mostly binary metallic mask."""
    sa, sn, sr, sm = sizes
    return [value_noise_texture(sa, sa, seed), normal_map_texture(sn, sn, seed + 1),
            scalar_texture(sr, sr, seed + 2, 0.15, 0.95), scalar_texture(sm, sm, seed + 3, 0.0, 1.0, sharpen=4.0)]


# -- meshes -------------------------------------------------------------------

def _icosphere(subdiv: int):
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
             (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(v, np.float64) / np.linalg.norm(v) for v in verts]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.array(verts), np.array(faces, np.int64)


def scene_tiny(seed_mesh: int = 1, seed_tex: int = 2, tex_size: int = 256) -> Scene:
    """2,048 triangles: an icosphere of subdivision 3 (1,280 triangles, radius
    0.7, vertices jittered radially) over a ground quad at y = -0.8 tessellated
    into 16 x 24 cells (768 triangles). One value-noise texture with planar x4
    UVs on the ground and spherical UVs on the sphere."""
    rng = np.random.default_rng(seed_mesh)
    v, f = _icosphere(3)
    r = 0.7 * (1.0 + 0.04 * rng.uniform(-1.0, 1.0, size=len(v)))
    pv = v * r[:, None]
    # non-indexed sphere so every triangle can carry a seam-free UV triple
    xyz, uv = [], []
    for a, b, c in f:
        tri = pv[[a, b, c]]
        s = np.arctan2(tri[:, 2], tri[:, 0]) / (2 * math.pi) + 0.5
        tt = np.arccos(np.clip(tri[:, 1] / np.linalg.norm(tri, axis=1), -1, 1)) / math.pi
        if s.max() - s.min() > 0.5:
            s = np.where(s < 0.5, s + 1.0, s)
        xyz.append(tri)
        uv.append(np.stack([s * 2.0, tt], 1))
    xyz = np.concatenate(xyz)
    uv = np.concatenate(uv)
    n_sph = len(f)
    # ground quad, 16 x 24 cells, x in [-1, 1], z in [-1, 1]
    nx, nz = 16, 24
    gx = np.linspace(-1.0, 1.0, nx + 1)
    gz = np.linspace(-1.0, 1.0, nz + 1)
    gxyz, guv = [], []
    for iz in range(nz):
        for ix in range(nx):
            p00 = (gx[ix], -0.8, gz[iz])
            p10 = (gx[ix + 1], -0.8, gz[iz])
            p01 = (gx[ix], -0.8, gz[iz + 1])
            p11 = (gx[ix + 1], -0.8, gz[iz + 1])
            for tri in ((p00, p01, p11), (p00, p11, p10)):
                tri = np.array(tri)
                gxyz.append(tri)
                guv.append(np.stack([(tri[:, 0] + 1) * 2.0, (tri[:, 2] + 1) * 2.0], 1))
    xyz = np.concatenate([xyz, np.concatenate(gxyz)]).astype(np.float32)
    uv = np.concatenate([uv, np.concatenate(guv)]).astype(np.float32)
    n = len(xyz) // 3
    idx = np.arange(3 * n, dtype=np.uint32).reshape(n, 3)
    assert n == n_sph + 2 * nx * nz == 2048
    tex = value_noise_texture(tex_size, tex_size, seed_tex)
    return Scene(xyz=xyz, uv=uv, idx=idx, tri_tex=np.zeros(n, np.uint32),
                 textures=[tex])


def scene_pbr_tiny(seed_mesh: int = 1, seed_tex: int = 5) -> Scene:
    """The tiny scene with two materials (sphere, ground) of four textures
    each (albedo, normal, roughness, metallic), coarse enough that Eq. 1
    lowers the sampling density and with the largest texture not the albedo:
    32/64/16/8 texels a side on the sphere (the normal map largest), 16/32/8/64
    on the ground (the metallic mask largest)."""
    sc = scene_tiny(seed_mesh=seed_mesh)
    n_sph = 1280
    mat = np.zeros(sc.n_tris, np.uint32)
    mat[n_sph:] = 1
    tex = material_textures((32, 64, 16, 8), seed_tex) + material_textures((16, 32, 8, 64), seed_tex + 10)
    return Scene(xyz=sc.xyz, uv=sc.uv, idx=sc.idx, tri_tex=mat, textures=tex,
                 materials=np.arange(8, dtype=np.uint32).reshape(2, 4))


def _param_surface(kind: int, res: int, rng):
    """A res x res quad grid (2*res^2 triangles) over a parametric surface:
    0 displaced sphere, 1 displaced torus, 2 wavy sheet. Returns unit-scale
    vertices ((res+1)^2, 3), grid UVs in [0,1]^2 and indices."""
    u = np.linspace(0.0, 1.0, res + 1)
    uu, vv = np.meshgrid(u, u, indexing="xy")
    ph = rng.uniform(0, 2 * math.pi, size=6)
    fr = rng.integers(2, 6, size=3)
    disp = 0.08 * (np.sin(2 * math.pi * fr[0] * uu + ph[0]) * np.sin(2 * math.pi * fr[1] * vv + ph[1])
                   + 0.5 * np.sin(2 * math.pi * fr[2] * (uu + vv) + ph[2]))
    if kind == 0:
        th = math.pi * vv
        phi = 2 * math.pi * uu
        r = 1.0 + disp
        p = np.stack([r * np.sin(th) * np.cos(phi), r * np.cos(th), r * np.sin(th) * np.sin(phi)], -1)
    elif kind == 1:
        a = 2 * math.pi * uu
        b = 2 * math.pi * vv
        rr = 0.35 * (1.0 + disp)
        p = np.stack([(0.75 + rr * np.cos(b)) * np.cos(a), rr * np.sin(b), (0.75 + rr * np.cos(b)) * np.sin(a)], -1)
    else:
        p = np.stack([2 * uu - 1, 2.0 * disp, 2 * vv - 1], -1)
    p = p.reshape(-1, 3)
    q = np.arange((res + 1) * (res + 1)).reshape(res + 1, res + 1)
    a0 = q[:-1, :-1].ravel()
    a1 = q[:-1, 1:].ravel()
    b0 = q[1:, :-1].ravel()
    b1 = q[1:, 1:].ravel()
    idx = np.concatenate([np.stack([a0, b0, b1], 1), np.stack([a0, b1, a1], 1)])
    return p, np.stack([uu.ravel(), vv.ravel()], 1), idx


def _random_rotation(rng) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def textures_paper(n_textures: int = 64, max_tex: int = 4096, min_tex: int = 64,
                   seed: int = 3) -> List[np.ndarray]:
    """The paper-shaped scene's textures: value noise from min_tex^2 to
    max_tex^2 (powers of two, cycled)."""
    sizes = []
    s = min_tex
    while s <= max_tex:
        sizes.append(s)
        s *= 2
    return [value_noise_texture(sizes[k % len(sizes)], sizes[k % len(sizes)], seed * 1000 + k)
            for k in range(n_textures)]


def geometry_paper(n_instances: int = 200, res: int = 50, n_textures: int = 64, seed: int = 3,
                   r_max: float = 0.2, r_decades: float = 1.5, extent=(0.75, 1.05, 0.9)) -> Scene:
    """The paper-shaped scene's meshes (no textures; texture ids < n_textures):
    n_instances displaced parametric meshes of 2*res^2 triangles each with
    log-uniform radii over r_decades decades, random rotations and positions
    within +-extent, UV repeats of 1, 2 or 4."""
    rng = np.random.default_rng(seed)
    xyz, uv, idx, ttex = [], [], [], []
    base = 0
    for k in range(n_instances):
        kind = int(rng.integers(0, 3))
        p, g, ix = _param_surface(kind, res, rng)
        radius = r_max * 10.0 ** (-r_decades * rng.random())
        rot = _random_rotation(rng)
        pos = rng.uniform(-1.0, 1.0, size=3) * np.array(extent)
        xyz.append((p @ rot.T) * radius + pos)
        rep = float(2 ** int(rng.integers(0, 3)))
        uv.append(g * rep)
        idx.append(ix + base)
        ttex.append(np.full(len(ix), int(rng.integers(0, n_textures)), np.uint32))
        base += len(p)
    return Scene(xyz=np.concatenate(xyz).astype(np.float32),
                 uv=np.concatenate(uv).astype(np.float32),
                 idx=np.concatenate(idx).astype(np.uint32),
                 tri_tex=np.concatenate(ttex), textures=[])


def scene_paper(n_instances: int = 200, res: int = 50, n_textures: int = 64,
                max_tex: int = 4096, min_tex: int = 64, seed: int = 3,
                r_max: float = 0.2, r_decades: float = 1.5,
                extent=(0.75, 1.05, 0.9)) -> Scene:
    """Paper-shaped scene: n_instances displaced parametric meshes of
    2*res^2 triangles each (200 x 5,000 = 10^6 by default). Instance radii are
    log-uniform over r_decades decades, so triangle areas are log-uniform over
    2*r_decades decades. Textures run from min_tex^2 to max_tex^2 (powers of
    two, cycled), assigned per instance, so texel density per triangle varies
    by about three orders of magnitude. With the 48-view display the default
    radius gives about 2.7 million points per frame, the density of the
    paper's sponza and gallery frames (2.29 and 2.60 million points from about
    a million triangles, Table 1)."""
    textures = textures_paper(n_textures, max_tex, min_tex, seed)
    sc = geometry_paper(n_instances, res, n_textures, seed, r_max, r_decades, extent)
    sc.textures = textures
    return sc


def scene_pbr_paper(n_materials: int = 16, seed: int = 3, min_tex: int = 64, max_tex: int = 4096, **geom) -> Scene:
    """The paper-shaped geometry (geometry_paper) with materials instead of
    single textures: n_materials materials of four textures each (64 textures
    for 16 materials, as the plain scene), each texture's size drawn from the
    powers of two min_tex^2 .. max_tex^2, so the four textures of a triangle
    differ in resolution and Eq. 1 takes the largest."""
    rng = np.random.default_rng(seed + 77)
    sizes = []
    s_ = min_tex
    while s_ <= max_tex:
        sizes.append(s_)
        s_ *= 2
    tex = []
    for m in range(n_materials):
        tex += material_textures(tuple(int(sizes[int(rng.integers(0, len(sizes)))]) for _ in range(4)),
                                 seed * 1000 + 17 * m)
    sc = geometry_paper(n_textures=n_materials, seed=seed, **geom)
    sc.textures = tex
    sc.materials = np.arange(4 * n_materials, dtype=np.uint32).reshape(n_materials, 4)
    return sc


def batch_paper(n_scenes: int = 32, seed: int = 11, tris_range=(5.0e4, 2.0e6), res: int = 50,
                n_textures: int = 64):
    """Batched multi-scene workload: n_scenes paper-shaped scenes whose
    triangle counts are log-uniform over tris_range (whole instances of
    2*res^2 triangles), each on its own display: 24, 48 or 96 views over a
    40 degree cone at 420x560 or 640x360 (square pixels), 2560x1600 panel,
    slant 0.2. All scenes index one texture set of n_textures textures
    (textures_paper). Returns (displays, scenes without textures)."""
    rng = np.random.default_rng(seed)
    displays, scenes = [], []
    lo, hi = math.log(tris_range[0]), math.log(tris_range[1])
    per_inst = 2 * res * res
    for k in range(n_scenes):
        tris = math.exp(rng.uniform(lo, hi))
        n_inst = max(1, int(round(tris / per_inst)))
        views = int(rng.choice([24, 48, 96]))
        w, h = [(420, 560), (640, 360)][int(rng.integers(0, 2))]
        displays.append(Display(n_views=views, view_w=w, view_h=h, cone_deg=40.0, view_dist=4.0,
                                focal_w=2.4 * w / h, focal_h=2.4, near_z=0.1, far_z=100.0,
                                bias_h=1.0, bias_v=1.0, panel_w=2560, panel_h=1600,
                                lens_pitch_px=8.0, slant=0.2))
        scenes.append(geometry_paper(n_instances=n_inst, res=res, n_textures=n_textures,
                                     seed=seed * 1000 + k))
    return displays, scenes
