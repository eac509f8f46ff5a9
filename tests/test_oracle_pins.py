"""Pins of the CPU oracle against facts fixed outside it: closed-form point
counts, a double-precision brute-force ray caster, textbook special cases of
the mip/filtering and interleave steps, and the invariants the paper's method
implies. A plausible slip anywhere in the oracle (a dropped term, a wrong sign,
a transposed operand) fails at least one of these."""
import math
import os
from dataclasses import replace

import numpy as np
import pytest

import oracle as O
from paper_2601_19901_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


def unit_display(**kw) -> S.Display:
    """One eye at (0, 0, 4) over a 2 x 2 focal rectangle, 128 x 128 pixels:
    a pixel reverse-projects to exactly 2^-6 at distance 4."""
    base = dict(n_views=1, view_w=128, view_h=128, cone_deg=30.0, view_dist=4.0,
                focal_w=2.0, focal_h=2.0, near_z=0.1, far_z=100.0, bias_h=1.0,
                bias_v=1.0, panel_w=64, panel_h=64, lens_pitch_px=8.0, slant=0.0)
    base.update(kw)
    return S.Display(**base)


def tri_scene(tris, uvs=None, tex=None) -> S.Scene:
    tris = np.asarray(tris, np.float32).reshape(-1, 3, 3)
    n = len(tris)
    uv = np.tile(np.array([[0, 0], [1, 0], [0, 1]], np.float32), (n, 1)) if uvs is None \
        else np.asarray(uvs, np.float32).reshape(-1, 2)
    textures = [tex if tex is not None else np.full((4, 4, 4), 200, np.uint8)]
    return S.Scene(xyz=tris.reshape(-1, 3), uv=uv,
                   idx=np.arange(3 * n, dtype=np.uint32).reshape(n, 3),
                   tri_tex=np.zeros(n, np.uint32), textures=textures)


I4 = np.eye(4, dtype=np.float32)


# ---------------------------------------------------------------------------
# log2 (Eq. 6-7)
# ---------------------------------------------------------------------------

def test_log2_powers_of_two_exact():
    for e in range(-149, 128):
        assert O.log2f(math.ldexp(1.0, e)) == float(e)


def test_log2_error_bound_against_exact():
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.uniform(0.5, 2.0, 4000), 10.0 ** rng.uniform(-44, 38, 4000)]).astype(np.float32)
    worst = 0.0
    for x in xs:
        got = O.log2f(float(x))
        exact = math.log2(float(x))
        ulp = np.spacing(np.float32(abs(exact))) if exact != 0 else np.float32(2 ** -149)
        worst = max(worst, abs(got - exact) / float(ulp))
    assert worst <= 4.0, worst


def test_log2_monotone_on_a_sweep():
    xs = np.float32(1.0) * np.arange(1, 20001, dtype=np.float32) / np.float32(997.0)
    ys = [O.log2f(float(x)) for x in xs]
    assert all(b >= a for a, b in zip(ys, ys[1:]))


def test_log2_special_values():
    assert O.log2f(0.0) == -math.inf
    assert O.log2f(math.inf) == math.inf
    assert math.isnan(O.log2f(math.nan))


# ---------------------------------------------------------------------------
# Views
# ---------------------------------------------------------------------------

def test_single_view_on_axis_and_views_symmetric():
    assert O.eyes(unit_display())[0] == 0.0
    ex = O.eyes(S.display_paper())
    assert np.allclose(ex, -ex[::-1], rtol=0, atol=1e-6)


@pytest.mark.parametrize("d", [S.display_tiny(), S.display_paper(), S.display_angular_ss()])
def test_view_angles_evenly_spaced(d):
    ex = O.eyes(d).astype(np.float64)
    ang = np.degrees(np.arctan(ex / d.view_dist))
    step = d.cone_deg / d.n_render_views
    assert np.allclose(np.diff(ang), step, atol=1e-4)
    if d.recon == 1:   # even supersampled views sit on the display-view centres
        centres = -d.cone_deg / 2 + d.cone_deg * (np.arange(d.n_views) + 0.5) / d.n_views
        assert np.allclose(ang[0::2], centres, atol=1e-4)
    else:
        assert abs(ang[0] + d.cone_deg / 2 - step / 2) < 1e-4


# ---------------------------------------------------------------------------
# Sampling: closed-form point counts (Sec. 3.1, Eq. 1-3)
# ---------------------------------------------------------------------------

def _golden_counts():
    rows = []
    for line in open(os.path.join(GOLDEN, "point_counts.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        f = line.split()
        rows.append(([float(v) for v in f[:6]], float(f[6]), float(f[7]), int(f[8]), int(f[9]), int(f[10])))
    return rows


@pytest.mark.parametrize("row", _golden_counts())
def test_closed_form_point_counts(row):
    verts2, bh, bv, tw, th, expected = row
    s = 2.0 ** -6
    tri = [[verts2[0] * s, verts2[1] * s, 0], [verts2[2] * s, verts2[3] * s, 0],
           [verts2[4] * s, verts2[5] * s, 0]]
    d = unit_display(bias_h=bh, bias_v=bv)
    st, rec, counts = O.setup(d, tri_scene(tri), I4, tex_wh=[tw, th])
    assert st == 0
    assert rec[0, O.F["d_min"]] == 4.0
    assert int(counts[0]) == expected


def test_point_set_of_right_triangle_is_the_staircase():
    s = 2.0 ** -6
    m = 8
    d = unit_display()
    st, rec, counts = O.setup(d, tri_scene([[0, 0, 0], [m * s, 0, 0], [0, m * s, 0]]), I4, tex_wh=[4096, 4096])
    pts = O.emit(rec, counts)
    got = [(int(p[1]) & 0xFFFF, int(p[1]) >> 16) for p in pts]
    want = [(i, j) for i in range(m) for j in range(m - i)]
    assert got == want                           # order: column, then row
    assert rec[0, O.F["s_u"]] == s and rec[0, O.F["s_v"]] == s


def test_square_two_triangles_share_only_the_diagonal():
    s = 2.0 ** -6
    m = 8
    d = unit_display()
    a = [[0, 0, 0], [m * s, 0, 0], [m * s, m * s, 0]]
    b = [[0, 0, 0], [m * s, m * s, 0], [0, m * s, 0]]
    st, rec, counts = O.setup(d, tri_scene(a + b), I4, tex_wh=[4096, 4096])
    pts = O.emit(rec, counts)
    cells = [set(), set()]
    for p in pts:
        cells[int(p[0])].add((int(p[1]) & 0xFFFF, int(p[1]) >> 16))
    assert len(cells[0] | cells[1]) == m * m
    assert cells[0] & cells[1] == {(i, i) for i in range(m)}


def test_texture_limit_never_adds_points_and_matches_texel_area():
    d = S.display_tiny()
    sc = S.scene_tiny()
    m = S.model_matrix(0)
    _, rec_big, c_big = O.setup(d, sc, m, tex_wh=[1 << 14, 1 << 14])
    _, rec_tex, c_tex = O.setup(d, sc, m, tex_wh=[16, 16])
    assert c_tex.sum() < c_big.sum()
    limited = rec_tex[:, O.F["size_uv"]] > rec_tex[:, O.F["s_u"]] * 0 + rec_big[:, O.F["s_u"]] * rec_big[:, O.F["s_v"]]
    assert limited.any()
    # Eq. 3: where the texture limits, the cell area equals the world area per texel
    area = rec_tex[limited, O.F["s_u"]].astype(np.float64) * rec_tex[limited, O.F["s_v"]]
    assert np.allclose(area, rec_tex[limited, O.F["size_uv"]], rtol=1e-5)
    # horizontal:vertical spacing ratio stays the LFD bias
    ratio = rec_tex[:, O.F["s_u"]] / rec_tex[:, O.F["s_v"]]
    live = rec_tex[:, O.F["live"]] == 1
    assert np.allclose(ratio[live], d.bias_h / d.bias_v, rtol=1e-5)


def test_every_live_triangle_emits_and_counts_sum_to_points():
    d = S.display_tiny()
    fr = O.render(d, S.scene_tiny(), S.model_matrix(5), splat=False)
    live = fr.tri[:, O.F["live"]] == 1
    assert np.all(fr.counts[live] >= 1) and np.all(fr.counts[~live] == 0)
    assert len(fr.points) == int(fr.counts.sum())
    # points are grouped by triangle in ascending order
    assert np.all(np.diff(fr.points[:, 0].astype(np.int64)) >= 0)


def test_dmin_is_distance_to_closest_point_double_check():
    """d_min against a dense double-precision sampling of the triangle."""
    d = S.display_tiny()
    sc = S.scene_tiny()
    m = S.model_matrix(2)
    _, rec, _ = O.setup(d, sc, m)
    tx = O.transformed_tris(sc, m).astype(np.float64).reshape(-1, 3, 3)
    ex = O.eyes(d).astype(np.float64)
    E = np.stack([ex, np.zeros_like(ex), np.full_like(ex, d.view_dist)], 1)
    g = np.linspace(0, 1, 61)
    a, b = np.meshgrid(g, g)
    keep = a + b <= 1
    a, b = a[keep], b[keep]
    for t in range(0, sc.n_tris, 97):
        P = tx[t]
        pts = P[0] + a[:, None] * (P[1] - P[0]) + b[:, None] * (P[2] - P[0])
        dist = np.sqrt(((pts[None, :, :] - E[:, None, :]) ** 2).sum(-1)).min()
        got = float(rec[t, O.F["d_min"]])
        edge = max(np.linalg.norm(P[1] - P[0]), np.linalg.norm(P[2] - P[0]))
        assert got <= dist + 1e-5
        assert got >= dist - edge / 60 - 1e-5


# ---------------------------------------------------------------------------
# Visibility (Sec. 3)
# ---------------------------------------------------------------------------

def test_culling_cases():
    d = S.display_tiny()
    left = [[-50, 0, 0], [-49, 0, 0], [-50, 1, 0]]
    behind = [[0, 0, 10], [1, 0, 10], [0, 1, 10]]
    centre = [[0, 0, 0], [0.1, 0, 0], [0, 0.1, 0]]
    # right of every frustum at z = 0 except the rightmost view's
    ex = O.eyes(d)
    fw2 = d.focal_w / 2
    z = -2.0
    x_edge_last = ex[-1] + (fw2 - ex[-1]) * (d.view_dist - z) / d.view_dist
    x_edge_prev = ex[-2] + (fw2 - ex[-2]) * (d.view_dist - z) / d.view_dist
    xm = 0.5 * (x_edge_last + x_edge_prev)
    only_last = [[xm, 0, z], [xm + 0.001, 0, z], [xm, 0.001, z]]
    _, rec, counts = O.setup(d, tri_scene(left + behind + centre + only_last), I4)
    assert list(rec[:, O.F["live"]]) == [0, 0, 1, 1]


# ---------------------------------------------------------------------------
# Per-frame model transform (Sec. 5.1: the scenes move every frame)
# ---------------------------------------------------------------------------

def general_affine() -> np.ndarray:
    """Row-major 4x4: rotations about x (17 deg) and z (-11 deg), a shear of
    x by z, and the translation (0.3, -0.2, 0.5). Not symmetric, so a
    transposed matrix or a translation read from the wrong row or column
    moves points elsewhere."""
    ax, az = math.radians(17.0), math.radians(-11.0)
    rx = np.array([[1, 0, 0], [0, math.cos(ax), -math.sin(ax)], [0, math.sin(ax), math.cos(ax)]])
    rz = np.array([[math.cos(az), -math.sin(az), 0], [math.sin(az), math.cos(az), 0], [0, 0, 1]])
    sh = np.array([[1, 0, 0.15], [0, 1, 0], [0, 0, 1]])
    m = np.eye(4)
    m[:3, :3] = rz @ rx @ sh
    m[:3, 3] = [0.3, -0.2, 0.5]
    return m.astype(np.float32)


def affine_double(m: np.ndarray, xyz: np.ndarray) -> np.ndarray:
    m = m.astype(np.float64)
    return xyz.astype(np.float64) @ m[:3, :3].T + m[:3, 3]


def test_model_transform_is_the_affine_map_in_double():
    m = general_affine()
    rng = np.random.default_rng(17)
    p = rng.uniform(-1.0, 1.0, (500, 3)).astype(np.float32)
    got = O.transform(m, p).astype(np.float64)
    want = affine_double(m, p)
    # three fused multiply-adds per coordinate: within a few ulps of the
    # largest term
    mag = np.abs(p.astype(np.float64)) @ np.abs(m[:3, :3].astype(np.float64)).T + np.abs(m[:3, 3])
    assert np.all(np.abs(got - want) <= 4 * 2.0 ** -24 * mag)
    # and not the transposed map, nor one without the translation column
    mt = m.copy()
    mt[:3, :3] = m[:3, :3].T
    assert np.abs(affine_double(mt, p) - want).max() > 0.1
    assert np.abs(p.astype(np.float64) @ m[:3, :3].astype(np.float64).T - want).max() > 0.1


def test_identity_and_pure_translation_transform_exactly():
    rng = np.random.default_rng(5)
    p = rng.uniform(-2.0, 2.0, (64, 3)).astype(np.float32)
    assert np.array_equal(O.transform(I4, p), p)
    t = np.eye(4, dtype=np.float32)
    t[:3, 3] = [0.25, -0.5, 2.0]
    # dyadic shifts of values in [-2, 2] on a 2^-20 grid: exact in binary32
    q = (np.round(p * 2 ** 20) / 2 ** 20).astype(np.float32)
    assert np.array_equal(O.transform(t, q), q + np.float32([0.25, -0.5, 2.0]))


def test_setup_records_the_transformed_first_vertex():
    d = S.display_tiny()
    sc = S.scene_tiny()
    m = general_affine()
    _, rec, _ = O.setup(d, sc, m)
    v0 = sc.xyz[sc.idx[:, 0].astype(np.int64)]
    want = affine_double(m, v0)
    got = rec[:, O.F["p0"]:O.F["p0"] + 3].astype(np.float64)
    assert np.abs(got - want).max() <= 1e-6


def test_splat_winner_is_raycast_nearest_under_a_general_affine_model():
    """The frame rendered under a rotated, sheared and translated model
    against the ray caster run on vertices transformed here, in double: the
    same triangle wins >= 99.9 % of pixels, every disagreement on a boundary."""
    d = replace(S.display_tiny(), view_w=96, view_h=96)
    sc = S.scene_tiny()
    m = general_affine()
    views = [1, 6]
    fr = O.render(d, sc, m, views=views, panel=False)
    tx = np.ascontiguousarray(affine_double(m, sc.xyz)[sc.idx.astype(np.int64)].reshape(-1, 9).astype(np.float32))
    total = agree = 0
    covered = 0
    for li, v in enumerate(views):
        rc = np.full((d.view_h, d.view_w), -1, np.int64)
        for y in range(d.view_h):
            for x in range(d.view_w):
                rc[y, x] = O.raycast(d, tx, v, x, y)[0]
        k = fr.keys[li]
        win = np.where(k == EMPTY, -1,
                       fr.points[(k & np.uint64(0xFFFFFFFF)).astype(np.int64) % max(len(fr.points), 1), 0].astype(np.int64))
        win[k == EMPTY] = -1
        same = win == rc
        total += same.size
        agree += same.sum()
        covered += int((rc >= 0).sum())
        assert np.all(_boundary(rc)[~same])
    assert covered > 0.2 * total
    assert agree / total >= 0.999


# ---------------------------------------------------------------------------
# Splatting (Sec. 3.2) against brute-force ray casting
# ---------------------------------------------------------------------------

def _boundary(ids):
    b = np.zeros(ids.shape, bool)
    b[1:, :] |= ids[1:, :] != ids[:-1, :]
    b[:-1, :] |= ids[1:, :] != ids[:-1, :]
    b[:, 1:] |= ids[:, 1:] != ids[:, :-1]
    b[:, :-1] |= ids[:, 1:] != ids[:, :-1]
    return b


def test_splat_winner_is_raycast_nearest_triangle():
    d = S.display_tiny()
    sc = S.scene_tiny()
    m = S.model_matrix(7)
    views = [0, 7]
    fr = O.render(d, sc, m, views=views, panel=False)
    tx = O.transformed_tris(sc, m)
    total = agree = 0
    for li, v in enumerate(views):
        rc = np.full((d.view_h, d.view_w), -1, np.int64)
        for y in range(d.view_h):
            for x in range(d.view_w):
                rc[y, x] = O.raycast(d, tx, v, x, y)[0]
        k = fr.keys[li]
        win = np.where(k == EMPTY, -1, fr.points[(k & np.uint64(0xFFFFFFFF)).astype(np.int64) % max(len(fr.points), 1), 0].astype(np.int64))
        win[k == EMPTY] = -1
        same = win == rc
        total += same.size
        agree += same.sum()
        # every disagreement sits on a triangle boundary of the ray-cast image
        assert np.all(_boundary(rc)[~same])
    assert agree / total >= 0.999


def test_single_triangle_each_pixel_filled_exactly_once():
    """Cells are half-open and tile the triangle: on the triangle's pixels
    exactly one of its points passes the tests, elsewhere none (up to pixel
    centres on the triangle's own outline)."""
    d = replace(S.display_tiny(), view_w=64, view_h=64)
    tri = [[-0.6, -0.5, 0.3], [0.7, -0.3, -0.4], [-0.1, 0.6, 0.1]]
    sc = tri_scene(tri, uvs=[[0, 0], [3, 0], [0, 3]], tex=np.full((64, 64, 4), 9, np.uint8))
    m = S.model_matrix(0)
    st, rec, counts = O.setup(d, sc, m)
    pts = O.emit(rec, counts)
    assert len(pts) > 50
    views = [0, 3, 7]
    hits = O.splat_hits(d, rec, pts, views)
    tx = O.transformed_tris(sc, m)
    assert hits.max() == 1
    for li, v in enumerate(views):
        cov = np.array([[O.raycast(d, tx, v, x, y)[0] >= 0 for x in range(d.view_w)] for y in range(d.view_h)])
        diff = (hits[li] == 1) != cov
        assert np.all(_boundary(cov.astype(np.int64))[diff])
        assert diff.sum() <= 2


def test_screen_parallel_square_is_an_exact_raster():
    d = unit_display(view_w=64, view_h=64)
    px = 2.0 / 64
    x0, x1, y0, y1 = -1 + 10 * px, -1 + 30 * px, 1 - 40 * px, 1 - 22 * px
    a = [[x0, y0, 0], [x1, y0, 0], [x1, y1, 0]]
    b = [[x0, y0, 0], [x1, y1, 0], [x0, y1, 0]]
    fr = O.render(d, tri_scene(a + b), I4, panel=False)
    cov = fr.keys[0] != EMPTY
    want = np.zeros_like(cov)
    want[22:40, 10:30] = True            # rows from the top: y in (1 - 40px, 1 - 22px)
    assert np.array_equal(cov, want)
    # the depth is the focal plane: t = 1 exactly
    t = (fr.keys[0][cov] >> np.uint64(32)).astype(np.uint32).view(np.float32)
    assert np.all(t == 1.0)


def test_nearest_surface_invariant_two_layers():
    """Two parallel squares: the nearer one wins every pixel it covers."""
    d = replace(S.display_tiny(), view_w=48, view_h=48)
    far_sq = [[[-0.5, -0.5, -0.5], [0.5, -0.5, -0.5], [0.5, 0.5, -0.5]], [[-0.5, -0.5, -0.5], [0.5, 0.5, -0.5], [-0.5, 0.5, -0.5]]]
    near_sq = [[[-0.2, -0.2, 0.5], [0.2, -0.2, 0.5], [0.2, 0.2, 0.5]], [[-0.2, -0.2, 0.5], [0.2, 0.2, 0.5], [-0.2, 0.2, 0.5]]]
    sc = tri_scene(far_sq + near_sq)
    fr = O.render(d, sc, I4, panel=False)
    tx = O.transformed_tris(sc, I4)
    for li in range(d.n_views):
        k = fr.keys[li]
        win = np.where(k == EMPTY, -1, fr.points[(k & np.uint64(0xFFFFFFFF)).astype(np.int64) % len(fr.points), 0].astype(np.int64))
        for y in range(0, d.view_h, 3):
            for x in range(0, d.view_w, 3):
                tri, t = O.raycast(d, tx, li, x, y)
                if tri >= 2 and not _boundary(win)[y, x]:
                    assert win[y, x] in (2, 3)


# ---------------------------------------------------------------------------
# Mip chain and filtered fetch (Sec. 3.3)
# ---------------------------------------------------------------------------

def test_mip_chain_sizes():
    assert O.lib().orc_mip_bytes(256, 256) == 4 * 87381
    assert O.lib().orc_mip_levels(8, 2) == 4
    assert O.lib().orc_mip_bytes(8, 2) == 4 * (16 + 4 + 2 + 1)


def test_checkerboard_mips_to_exact_mid_grey():
    t = np.zeros((8, 8, 4), np.uint8)
    t[(np.add.outer(np.arange(8), np.arange(8)) % 2) == 1] = 255
    lv = O.mip_levels(O.mip_chain(t), 8, 8)
    for l in lv[1:]:
        assert np.all(l == 128)     # (0 + 255 + 0 + 255 + 2) >> 2


def test_constant_texture_fetches_constant_everywhere():
    t = np.empty((32, 16, 4), np.uint8)
    t[:] = (17, 99, 201, 255)
    ch = O.mip_chain(t)
    rng = np.random.default_rng(1)
    for _ in range(300):
        s, tt = rng.uniform(-5, 5, 2)
        lod = rng.uniform(-2, 9)
        assert list(O.trilinear(ch, 16, 32, s, tt, lod)) == [17, 99, 201, 255]


def test_bilinear_texel_centres_midpoints_and_wrap():
    rng = np.random.default_rng(2)
    t = rng.integers(0, 256, (8, 8, 4), dtype=np.uint8)
    ch = O.mip_chain(t)
    for y in range(8):
        for x in range(8):
            assert np.array_equal(O.trilinear(ch, 8, 8, (x + 0.5) / 8, (y + 0.5) / 8, 0.0), t[y, x])
            assert np.array_equal(O.trilinear(ch, 8, 8, (x + 0.5) / 8 + 3, (y + 0.5) / 8 - 2, 0.0), t[y, x])
    # halfway between texels (x-1, y) and (x, y): mean, rounded half to even
    for y in range(8):
        for x in range(8):
            a = t[y, x - 1].astype(np.float64)
            b = t[y, x].astype(np.float64)
            want = np.round((a + b) / 2)            # numpy rounds half to even
            got = O.trilinear(ch, 8, 8, x / 8, (y + 0.5) / 8, 0.0)
            assert np.array_equal(got, want.astype(np.uint8))


def test_lod_blend_between_levels():
    t = np.zeros((2, 2, 4), np.uint8)
    t[0, 1] = t[1, 0] = 255
    ch = O.mip_chain(t)                 # level 1 = 128
    assert O.trilinear(ch, 2, 2, 0.25, 0.25, 0.5)[0] == 64    # lerp(0, 128, 0.5)
    assert O.trilinear(ch, 2, 2, 0.75, 0.25, 0.5)[0] == 192   # lerp(255, 128, 0.5) = 191.5 -> even
    assert O.trilinear(ch, 2, 2, 0.25, 0.25, 1.0)[0] == 128
    assert O.trilinear(ch, 2, 2, 0.25, 0.25, 7.0)[0] == 128   # clamped to the last level


# ---------------------------------------------------------------------------
# Multiview mipmapping (Eq. 4-9) invariants on a whole frame
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def tiny_frame():
    d = S.display_tiny()
    return d, O.render(d, S.scene_tiny(), S.model_matrix(11))


def test_lod_min_not_above_lod_max(tiny_frame):
    _, fr = tiny_frame
    live = fr.tri[:, O.F["live"]] == 1
    assert np.all(fr.tri[live, O.F["lod_min"]] <= fr.tri[live, O.F["lod_max"]])
    assert np.all(fr.tri[live, O.F["vpuv_min"]] <= fr.tri[live, O.F["vpuv_max"]])


def test_resolved_colour_between_tv_min_and_tv_max(tiny_frame):
    _, fr = tiny_frame
    k = fr.keys
    cov = k != EMPTY
    pid = (k[cov] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    tmin = fr.points[pid, 2:3].copy().view(np.uint8).reshape(-1, 4)
    tmax = fr.points[pid, 3:4].copy().view(np.uint8).reshape(-1, 4)
    col = fr.rgba[cov]
    lo = np.minimum(tmin, tmax)
    hi = np.maximum(tmin, tmax)
    assert np.all(col >= lo) and np.all(col <= hi)
    assert np.all(fr.rgba[~cov] == 0)


def test_one_view_colour_is_tv_min():
    d = replace(S.display_tiny(), n_views=1)
    fr = O.render(d, S.scene_tiny(), S.model_matrix(3))
    live = fr.tri[:, O.F["live"]] == 1
    assert np.array_equal(fr.tri[live, O.F["vpuv_min"]], fr.tri[live, O.F["vpuv_max"]])
    cov = fr.keys[0] != EMPTY
    pid = (fr.keys[0][cov] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    tmin = fr.points[pid, 2:3].copy().view(np.uint8).reshape(-1, 4)
    assert np.array_equal(fr.rgba[0][cov], tmin)


# ---------------------------------------------------------------------------
# Reconstruction, crosstalk, interleave (Sec. 4)
# ---------------------------------------------------------------------------

def test_constant_stack_stays_constant_through_recon_and_crosstalk():
    d = replace(S.display_angular_ss(), view_w=8, view_h=6, panel_w=40, panel_h=24)
    r = np.full((d.n_render_views, 6, 8, 4), 77, np.uint8)
    dv = O.display_views(d, r)
    assert np.all(np.abs(dv - 77) < 1e-4)
    pan = O.interleave(d, r)
    assert np.all(pan[..., :3] == 77) and np.all(pan[..., 3] == 255)


def test_delta_spreads_over_the_tent_then_crosstalk():
    N = 6
    d = replace(S.display_angular_ss(), n_views=N, view_w=1, view_h=1, crosstalk=0.0)
    r = np.zeros((2 * N, 1, 1, 4), np.uint8)
    r[5, 0, 0, 0] = 200                 # odd supersampled view: halfway between views 2 and 3
    dv = O.display_views(d, r)[:, 0, 0, 0]
    assert np.allclose(dv, [0, 0, 50, 50, 0, 0])
    r[:] = 0
    r[4, 0, 0, 0] = 200                 # even: on view 2's centre
    dv = O.display_views(d, r)[:, 0, 0, 0]
    assert np.allclose(dv, [0, 0, 100, 0, 0, 0])
    r[:] = 0
    r[0, 0, 0, 0] = 240                 # left edge: view 0's taps are views 0, 1 only, renormalised by 3/4
    dv = O.display_views(d, r)[:, 0, 0, 0]
    assert np.allclose(dv, [160, 0, 0, 0, 0, 0])
    d2 = replace(d, recon=0, crosstalk=0.15)
    r2 = np.zeros((N, 1, 1, 4), np.uint8)
    r2[0, 0, 0, 0] = 200
    dv = O.display_views(d2, r2)[:, 0, 0, 0]
    assert np.allclose(dv, [140, 30, 0, 0, 0, 30], atol=1e-4)   # wraps to view N-1


@pytest.mark.parametrize("d", [S.display_tiny(), S.display_paper()])
def test_interleave_view_histogram_is_even(d):
    """Over one lens period horizontally and a whole number of slant periods
    vertically, every view is shown equally often, within one subpixel."""
    per_x = int(round(d.lens_pitch_px))
    per_y = int(round(1.0 / d.slant))
    counts = np.zeros(d.n_views, np.int64)
    for y in range(per_y * 2):
        for x in range(per_x):
            for c in range(3):
                counts[O.view_of_subpixel(d, x + 40, y + 7, c)] += 1
    mean = counts.sum() / d.n_views
    assert counts.min() >= math.floor(mean) - 1 and counts.max() <= math.ceil(mean) + 1


def test_interleave_unslanted_is_column_cyclic():
    d = replace(unit_display(), n_views=6, lens_pitch_px=2.0, slant=0.0)
    for y in (0, 5):
        for x in range(64):
            for c in range(3):
                assert O.view_of_subpixel(d, x, y, c) == (3 * x + c) % 6


def test_interleave_nearest_texel_mapping():
    d = replace(unit_display(view_w=4, view_h=2), n_views=1, panel_w=8, panel_h=4)
    r = np.zeros((1, 2, 4, 4), np.uint8)
    r[0, :, :, 0] = np.arange(8).reshape(2, 4) * 10
    pan = O.interleave(d, r)
    assert np.array_equal(pan[..., 0], np.repeat(np.repeat(r[0, :, :, 0], 2, 0), 2, 1))


# ---------------------------------------------------------------------------
# Targeted pins for single steps
# ---------------------------------------------------------------------------

def test_culling_by_near_and_far_alone():
    d = S.display_tiny()
    e4 = float(O.eyes(d)[4])
    too_near = [[e4, 0, 3.95], [e4 + 0.001, 0, 3.95], [e4, 0.001, 3.95]]  # depth 0.05 < near 0.1
    too_far = [[0, 0, -200], [0.5, 0, -200], [0, 0.5, -200]]           # depth 204 > far 100
    just_in = [[e4, 0, 3.8], [e4 + 0.001, 0, 3.8], [e4, 0.001, 3.8]]   # depth 0.2, on view 4's axis
    _, rec, _ = O.setup(d, tri_scene(too_near + too_far + just_in), I4)
    assert list(rec[:, O.F["live"]]) == [0, 0, 1]


def test_cell_centres_fetch_texel_centres():
    """Axis-aligned right triangle at the focal plane whose UVs map one texel
    onto one lattice cell: the cell centre is the texel centre and LOD_min is
    0, so tv_min of point (i, j) is texel (i, j) exactly (a transposed or
    shifted UV map, or a wrong level, picks another texel)."""
    s = 2.0 ** -6
    mu, mv = 8, 4
    rng = np.random.default_rng(5)
    tex = rng.integers(0, 256, (mv, mu, 4), dtype=np.uint8)
    d = unit_display()
    sc = tri_scene([[0, 0, 0], [mu * s, 0, 0], [0, mv * s, 0]], uvs=[[0, 0], [1, 0], [0, 1]], tex=tex)
    fr = O.render(d, sc, I4, splat=False)
    assert fr.tri[0, O.F["lod_min"]] == 0.0
    for p in fr.points:
        i, j = int(p[1]) & 0xFFFF, int(p[1]) >> 16
        assert np.array_equal(np.frombuffer(p[2].tobytes(), np.uint8), tex[j, i]), (i, j)


def test_pixel_centres_on_cell_corners_are_filled_once():
    """The lattice origin sits on a pixel centre and cells are one pixel, so
    every pixel centre is a cell corner: the half-open cells still give each
    pixel exactly one splat, and exactly the pixels of the closed legs and the
    interior are filled (centres on the hypotenuse fall in cells outside the
    triangle)."""
    d = unit_display(view_w=64, view_h=64, focal_w=1.0, focal_h=1.0)   # pixel 2^-6 at z = 0
    px = 2.0 ** -6
    m = 12
    x0, y0 = -0.5 + 28.5 * px, 0.5 - 36.5 * px       # pixel (28, 36) centre; the eye is over the triangle
    tri = [[x0, y0, 0], [x0 + m * px, y0, 0], [x0, y0 + m * px, 0]]
    sc = tri_scene(tri)
    st, rec, counts = O.setup(d, sc, I4, tex_wh=[4096, 4096])
    assert rec[0, O.F["s_u"]] == px and rec[0, O.F["d_min"]] == 4.0
    pts = O.emit(rec, counts)
    hits = O.splat_hits(d, rec, pts, [0])[0]
    assert hits.max() == 1
    want = np.zeros((64, 64), np.int64)
    for a in range(m):              # pixel column 28 + a, rows 36 - b (y grows downwards)
        for b in range(m - a):
            want[36 - b, 28 + a] = 1
    assert np.array_equal(hits.astype(np.int64), want)


def test_eq8_eq9_on_a_screen_parallel_triangle():
    """Closed form of Eq. 8-9: for a triangle parallel to the focal plane the
    splat's pixel area is the cell area scaled by (D/depth)^2 over a pixel's
    area, in every view; the eye distances d_v are the depth and the in-plane
    offset. The expected colour is then tv_min + w (tv_max - tv_min) with
    w = clamp((A_uv / min(1, area_px) - vpuv_min) / (vpuv_max - vpuv_min), 0, 1)."""
    d = replace(unit_display(view_w=128, view_h=128, focal_w=4.0, focal_h=4.0), n_views=2, cone_deg=60.0)
    ex = O.eyes(d).astype(np.float64)
    z0 = 2.0
    dep = d.view_dist - z0
    cx = float(ex[1])
    L = 0.3
    x0 = cx - 0.05
    tri = [[x0, -0.05, z0], [x0 + L, -0.05, z0], [x0, -0.05 + L, z0]]
    tex = np.random.default_rng(9).integers(0, 256, (16, 16, 4), dtype=np.uint8)
    sc = tri_scene(tri, tex=tex)
    fr = O.render(d, sc, I4, panel=False)
    T = fr.tri[0].astype(np.float64)
    # d_v from geometry: eye 1 is over the triangle, eye 0 is off to the left
    d1 = dep
    d0 = math.hypot(dep, x0 - ex[0])
    assert abs(T[O.F["d_min"]] - d1) < 1e-5 and abs(T[O.F["d_max"]] - d0) < 1e-5
    px = d.focal_w / (d.view_dist * d.view_w)
    A_ws, A_ts = L * L / 2, 0.5
    r = A_ts / A_ws
    vmin, vmax = d1 * d1 * px * px * r, d0 * d0 * px * px * r
    su, sv = T[O.F["s_u"]], T[O.F["s_v"]]
    a_uv = su * sv * r
    assert vmin < a_uv < vmax            # texture-limited, so min(1, .) matters
    pix = (d.focal_w / d.view_w) * (d.focal_h / d.view_h)
    area_px = su * sv * (d.view_dist / dep) ** 2 / pix
    assert area_px > 1.0
    w = min(max((a_uv / min(1.0, area_px) - vmin) / (vmax - vmin), 0.0), 1.0)
    assert 0.05 < w < 0.95
    k = fr.keys[1]
    cov = k != EMPTY
    pid = (k[cov] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    tmin = fr.points[pid, 2:3].copy().view(np.uint8).reshape(-1, 4).astype(np.float64)
    tmax = fr.points[pid, 3:4].copy().view(np.uint8).reshape(-1, 4).astype(np.float64)
    want = tmin + w * (tmax - tmin)
    got = fr.rgba[1][cov].astype(np.float64)
    assert np.all(np.abs(got - want) <= 0.5 + 1e-3)
    assert int(cov.sum()) > 100
    assert np.abs(tmax - tmin).max() >= 20     # the two LODs really differ here


def _ndc_quad(d, Ex, corners):
    """NDC corners of a world quad in the view of eye (Ex, 0, D), by the
    textbook route: a look-at of the eye down -z, an off-axis (glFrustum-style)
    projection whose window is the focal rectangle at z = 0, and the
    perspective divide. All double."""
    D = float(d.view_dist)
    n = 0.05
    l, r = (-0.5 * d.focal_w - Ex) * n / D, (0.5 * d.focal_w - Ex) * n / D
    b, t = -0.5 * d.focal_h * n / D, 0.5 * d.focal_h * n / D
    f = 1000.0
    Pm = np.array([[2 * n / (r - l), 0, (r + l) / (r - l), 0],
                   [0, 2 * n / (t - b), (t + b) / (t - b), 0],
                   [0, 0, -(f + n) / (f - n), -2 * f * n / (f - n)],
                   [0, 0, -1, 0]])
    V = np.eye(4)
    V[:3, 3] = [-Ex, 0.0, -D]
    h = np.c_[np.asarray(corners, np.float64), np.ones(len(corners))] @ (Pm @ V).T
    return h[:, 0] / h[:, 3], h[:, 1] / h[:, 3]


def _ndc_quad_area_px(d, Ex, corners):
    """The NDC polygon's area times 0.25 X_v Y_v (Eq. 8): its area in pixels."""
    x, y = _ndc_quad(d, Ex, corners)
    ndc = 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(np.roll(x, -1), y))
    return ndc * 0.25 * d.view_w * d.view_h


def _quad_perimeter_px(d, Ex, corners):
    x, y = _ndc_quad(d, Ex, corners)
    x, y = x * 0.5 * d.view_w, y * 0.5 * d.view_h
    return float(np.hypot(x - np.roll(x, -1), y - np.roll(y, -1)).sum())


def test_eq8_on_tilted_cells_is_the_projected_quad_area():
    """Eq. 8 for cells of a triangle tilted against the focal plane: the
    splat's pixel area in view v is the NDC area of the cell's four corners
    under view v's projection, times 0.25 X_v Y_v (here through a projection
    matrix in double), so the weight, and with it the colour, changes from
    view to view. Expected colour tv_min + w (tv_max - tv_min) with
    w = clamp((A_uv / min(1, area_px) - vpuv_min) / (vpuv_max - vpuv_min), 0, 1)."""
    d = replace(unit_display(view_w=160, view_h=200, focal_w=4.0, focal_h=5.0), n_views=5, cone_deg=70.0)
    ex = O.eyes(d).astype(np.float64)
    tri = [[-0.5, -0.4, 1.2], [0.6, -0.4, 2.4], [-0.5, 0.6, 1.6]]
    tex = np.random.default_rng(21).integers(0, 256, (256, 256, 4), dtype=np.uint8)
    fr = O.render(d, tri_scene(tri, tex=tex), I4, panel=False)
    T = fr.tri[0].astype(np.float64)
    P0, eu, ev = T[O.F["p0"]:O.F["p0"] + 3], T[O.F["eu"]:O.F["eu"] + 3], T[O.F["ev"]:O.F["ev"] + 3]
    su, sv, umin, vmin = T[O.F["s_u"]], T[O.F["s_v"]], T[O.F["umin"]], T[O.F["vmin"]]
    vlo, vhi, a_uv = T[O.F["vpuv_min"]], T[O.F["vpuv_max"]], T[O.F["spl_uv"]]
    assert vhi > vlo

    def area_px(i, j, Ex):
        C = [P0 + (ci * su + umin) * eu + (cj * sv + vmin) * ev
             for ci, cj in ((i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1))]
        return _ndc_quad_area_px(d, Ex, C)

    ws = {}
    devs = []
    n_cov = 0
    for v in range(d.n_render_views):
        k = fr.keys[v]
        cov = k != EMPTY
        pid = (k[cov] & np.uint64(0xFFFFFFFF)).astype(np.int64)
        got = fr.rgba[v][cov].astype(np.float64)
        for p in np.unique(pid):
            i, j = int(fr.points[p, 1] & 0xFFFF), int(fr.points[p, 1] >> 16)
            ar = area_px(i, j, ex[v])
            w = min(max((a_uv / min(1.0, ar) - vlo) / (vhi - vlo), 0.0), 1.0)
            # the oracle's corners are binary32 (errors near 1e-7 of the
            # coordinates), its area and weight rounded once to binary32
            err = 1e-5 * ar
            dw = a_uv * err / (min(1.0, ar - err) ** 2 * (vhi - vlo)) if ar < 1.0 + err else 0.0
            ws.setdefault(int(p), []).append(w)
            tmin = fr.points[p, 2:3].copy().view(np.uint8).astype(np.float64)
            tmax = fr.points[p, 3:4].copy().view(np.uint8).astype(np.float64)
            want = tmin + w * (tmax - tmin)
            tol = 0.5 + 1e-3 + (dw + 1e-6) * np.abs(tmax - tmin)
            dev = np.abs(got[pid == p] - want)
            assert np.all(dev <= tol), (v, p, w, dw)
            devs.append(dev.ravel())
        n_cov += int(cov.sum())
    assert n_cov > 2000
    # beyond the final rounding (at most 1/2, 1/4 on average for the
    # channels that interpolate) the colours do not move
    devs = np.concatenate(devs)
    assert devs.mean() <= 0.26 and np.percentile(devs, 99) <= 0.501
    # the area, and so the weight, really changes with the eye here
    spread = [max(x) - min(x) for x in ws.values() if len(x) >= 3]
    assert len(spread) > 5 and max(spread) > 0.05


def test_eq8_area_of_cells_against_the_projection_matrix():
    """The oracle's Eq. 8 area of lattice cells of the paper-shaped display
    (420 x 560 views, so a swapped width and height shows), in every third
    view, against the NDC area through the projection matrix, within the
    effect of the binary32 rounding of the oracle's corners (the matrix
    route's are double), over
    cells from many times a pixel down to far below one, also far from the
    view centre, where pixel coordinates run into the hundreds."""
    d = S.display_paper()
    sc = S.scene_paper(n_instances=4, res=12, n_textures=4, max_tex=256, min_tex=16, seed=9, r_max=0.6)
    _, rec, counts = O.setup(d, sc, S.model_matrix(1))
    pts = O.emit(rec, counts)
    ex = O.eyes(d).astype(np.float64)
    rng = np.random.default_rng(8)
    areas = []
    for p in rng.choice(len(pts), 300, replace=False):
        t, i, j = int(pts[p, 0]), int(pts[p, 1] & 0xFFFF), int(pts[p, 1] >> 16)
        T = rec[t].astype(np.float64)
        P0, eu, ev = T[O.F["p0"]:O.F["p0"] + 3], T[O.F["eu"]:O.F["eu"] + 3], T[O.F["ev"]:O.F["ev"] + 3]
        su, sv, umin, vmin = T[O.F["s_u"]], T[O.F["s_v"]], T[O.F["umin"]], T[O.F["vmin"]]
        C = [P0 + (ci * su + umin) * eu + (cj * sv + vmin) * ev
             for ci, cj in ((i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1))]
        # the oracle's corners are binary32: each moves by at most a few
        # ulps of the terms that form it; the area by that times the perimeter
        Ca = np.array(C)
        mag = np.abs(P0).max() + abs((i + 1) * su) + abs(umin) + abs((j + 1) * sv) + abs(vmin)
        ppu = max(d.view_w / d.focal_w, d.view_h / d.focal_h) * d.view_dist / (d.view_dist - Ca[:, 2].max())
        for v in range(0, d.n_render_views, 3):
            want = _ndc_quad_area_px(d, ex[v], C)
            perim = _quad_perimeter_px(d, ex[v], C)
            tol = 2 * (2.0 ** -22 * mag * ppu * 2.0) * perim + 1e-6 * want
            got = O.splat_area_px(d, rec[t], i, j, float(ex[v]))
            assert abs(got - want) <= tol, (p, v, got, want, tol)
            areas.append(want)
    areas = np.array(areas)
    assert areas.min() < 0.05 and areas.max() > 4.0


def test_eq8_area_of_a_cell_reaching_the_eyes_plane_is_its_drawable_part():
    """A cell that reaches past the eyes' plane has no bounded projection;
    its Eq. 8 area is that of its part at depth >= near_z. Pinned against
    rays through a dense grid of sub-pixel positions, each hit tested
    against the cell and the near limit, in double."""
    d = replace(unit_display(), n_views=3, cone_deg=30.0)
    D, near = float(d.view_dist), float(d.near_z)
    eu = np.array([1.0, 0.0, 0.0])
    ev = np.array([0.0, 0.6, 0.8])          # tilted toward the eyes: z grows along v
    su, sv = 0.1, 0.5                       # z runs from D - 0.3 to D + 0.1
    nrm = np.cross(eu, ev)
    h = 1.0 / 8.0
    for Ex in O.eyes(d).astype(np.float64):
        # the cell straight in front of this eye
        P0 = np.array([float(np.float32(Ex)) - 0.05, -0.05, D - 0.3])
        T = np.zeros(O.TRI_FLOATS, np.float32)
        T[O.F["p0"]:O.F["p0"] + 3] = P0
        T[O.F["eu"]:O.F["eu"] + 3] = eu
        T[O.F["ev"]:O.F["ev"] + 3] = ev
        T[O.F["s_u"]], T[O.F["s_v"]] = su, sv
        P0 = T[O.F["p0"]:O.F["p0"] + 3].astype(np.float64)
        E = np.array([Ex, 0.0, D])
        xs = np.arange(-300.0, 300.0, h) + h / 2
        X, Y = np.meshgrid(xs, xs)
        F = np.stack([-0.5 * d.focal_w + X * d.focal_w / d.view_w, 0.5 * d.focal_h - Y * d.focal_h / d.view_h,
                      np.zeros_like(X)], -1)
        dirs = F - E
        t = ((P0 - E) @ nrm) / (dirs @ nrm)
        hit = E + t[..., None] * dirs
        q = hit - P0
        u, v = q @ eu, q @ ev
        inside = (u >= 0) & (u < su) & (v >= 0) & (v < sv) & (t * D >= near) & (t > 0)
        assert not inside[0].any() and not inside[-1].any() and not inside[:, 0].any() and not inside[:, -1].any()
        want = inside.sum() * h * h
        ys_, xs_ = np.nonzero(inside)
        perim = 2 * (np.ptp(xs_) + np.ptp(ys_)) * h
        got = O.splat_area_px(d, T, 0, 0, float(Ex))
        assert want > 1000.0
        assert abs(got - want) <= perim * h, (Ex, got, want)


# ---------------------------------------------------------------------------
# Sec. 4's supersampling at random angles and Gaussian reconstruction
# ---------------------------------------------------------------------------

def _gauss_display(recon, n_views=8, crosstalk=0.0):
    # tiny display: 128 x 128 views, 512 x 512 panel (view/panel ratio exact in binary32)
    return replace(S.display_tiny(), n_views=n_views, recon=recon, crosstalk=crosstalk)


def _random_views(d, seed=4):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, (d.n_render_views, d.view_h, d.view_w, 4), dtype=np.uint8)


def test_jitter_of_one_half_gives_the_regular_eyes():
    for recon in (0, 1, 3):
        d = _gauss_display(recon)
        half = np.full(d.n_render_views, 0.5, np.float32)
        assert np.array_equal(O.eyes(d, half), O.eyes(d))


def test_jitter_places_each_eye_inside_its_interval():
    # supersampled: rendered view m covers the half-interval [(m + 1/2), (m + 3/2)] / 2N
    # of the cone; jitter 0 and 1 put the eye at its two ends
    d = _gauss_display(2)
    nr = d.n_render_views
    for u in (0.0, 1.0):
        ex = O.eyes(d, np.full(nr, u, np.float32)).astype(np.float64)
        ang = np.degrees(np.arctan(ex / d.view_dist))
        want = -d.cone_deg / 2 + d.cone_deg * (np.arange(nr) + 0.5 + u) / (2 * d.n_views)
        assert np.allclose(ang, want, atol=1e-4)


def test_gauss_one_centred_sample_is_the_plain_interleave():
    # recon 3 with a single zero offset samples, for each subpixel, the view it
    # falls in at the nearest view pixel: the plain interleave
    d0 = _gauss_display(0)
    d3 = _gauss_display(3)
    v = _random_views(d0)
    assert np.array_equal(O.interleave(d3, v, samples=np.zeros((1, 3), np.float32)), O.interleave(d0, v))


def test_gauss_identical_samples_average_to_one_sample():
    d = _gauss_display(2)
    v = _random_views(d)
    one = np.array([[0.7, -1.3, 0.4]], np.float32)
    assert np.array_equal(O.interleave(d, v, samples=np.repeat(one, 8, 0)), O.interleave(d, v, samples=one))


def test_gauss_constant_views_stay_constant():
    d = _gauss_display(2, crosstalk=0.15)
    v = np.full((d.n_render_views, d.view_h, d.view_w, 4), 77, np.uint8)
    rng = np.random.default_rng(2)
    s = rng.normal(0.0, [0.5625, 0.5625, 0.5], (8, 3)).astype(np.float32)
    jit = rng.random(d.n_render_views).astype(np.float32)
    pan = O.interleave(d, v, jitter=jit, samples=s)
    assert np.all(pan[..., :3] == 77) and np.all(pan[..., 3] == 255)


def test_gauss_spatial_offset_reads_the_next_pixel():
    # a +1 view-pixel offset reads each view one pixel to the right (clamped):
    # the plain interleave of the views shifted left by one pixel
    d0 = _gauss_display(0)
    d3 = _gauss_display(3)
    v = _random_views(d0, 6)
    shifted = np.concatenate([v[:, :, 1:], v[:, :, -1:]], axis=2)
    got = O.interleave(d3, v, samples=np.array([[1.0, 0.0, 0.0]], np.float32))
    assert np.array_equal(got, O.interleave(d0, shifted))


def test_gauss_takes_the_nearest_view_by_brute_force():
    # random eye jitter and one random angular offset: every subpixel shows the
    # rendered view whose position is nearest its phase (ties to the later
    # view), found here by scanning all views
    d = replace(_gauss_display(2), panel_w=96, panel_h=40)
    rng = np.random.default_rng(11)
    jit = rng.random(d.n_render_views).astype(np.float32)
    nr = d.n_render_views
    pos = np.array([O.view_pos(d, m, jit) for m in range(nr)], np.float32)
    v = np.zeros((nr, d.view_h, d.view_w, 4), np.uint8)
    v[..., :3] = (np.arange(nr, dtype=np.uint8) * 11)[:, None, None, None]   # view m carries 11 m
    for dphi in (0.0, 0.37, -1.9, 6.2):
        s = np.array([[0.0, 0.0, dphi]], np.float32)
        pan = O.interleave(d, v, jitter=jit, samples=s)
        for y in range(0, d.panel_h, 7):
            for x in range(0, d.panel_w, 5):
                for c in range(3):
                    a = np.float32(O.subpixel_phase(d, x, y, c)) + np.float32(dphi)
                    dist = np.abs(pos - a)
                    m = int(np.flatnonzero(dist == dist.min())[-1])
                    assert pan[y, x, c] == 11 * m, (dphi, x, y, c)


# ---------------------------------------------------------------------------
# Spatial supersampling (Sec. 4; Sec. 5.1 builds a mipmap of each view)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("recon,level", [(0, 1), (1, 1), (3, 1), (2, 1), (0, 2), (3, 2)])
def test_spatial_ss_of_replicated_views_is_the_plain_interleave(recon, level):
    """Views rendered at 2^L times the output size whose pixels are L-fold
    replicas of an output-size view: their mip level L is that view, so the
    panel equals the plain interleave of it (with the same Gaussian samples,
    in output pixels, and crosstalk)."""
    d0 = replace(_gauss_display(recon, crosstalk=0.15), panel_w=160, panel_h=96)
    k = 1 << level
    d1 = replace(d0, view_w=k * d0.view_w, view_h=k * d0.view_h, ss_level=level)
    v = _random_views(d0, seed=9 + level)
    vk = np.repeat(np.repeat(v, k, axis=1), k, axis=2)
    samples = None
    if recon in (2, 3):
        samples = np.random.default_rng(5).normal(0.0, [0.5625, 0.5625, 0.5], (8, 3)).astype(np.float32)
    assert np.array_equal(O.interleave(d1, vk, samples=samples), O.interleave(d0, v, samples=samples))


def test_spatial_ss_of_checkerboard_views_is_mid_grey():
    d0 = replace(_gauss_display(0), panel_w=128, panel_h=64)
    d1 = replace(d0, view_w=2 * d0.view_w, view_h=2 * d0.view_h, ss_level=1)
    yy, xx = np.mgrid[0:d1.view_h, 0:d1.view_w]
    board = np.where(((xx + yy) & 1)[..., None] == 1, 255, 0).astype(np.uint8)
    v = np.broadcast_to(board, (d1.n_render_views, d1.view_h, d1.view_w, 4)).copy()
    pan = O.interleave(d1, v)
    # (0 + 255 + 0 + 255 + 2) >> 2 = 128 in every channel
    assert np.all(pan[..., :3] == 128) and np.all(pan[..., 3] == 255)
    # level 2 of the same boards: the mid-grey of mid-greys
    assert np.all(O.view_mip(v[0], 2) == 128)


def test_view_mip_of_a_constant_view_is_constant():
    v = np.full((64, 48, 4), 201, np.uint8)
    for level in (1, 2, 3):
        m = O.view_mip(v, level)
        assert m.shape == (64 >> level, 48 >> level, 4) and np.all(m == 201)
