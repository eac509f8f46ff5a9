"""Pins of the oracle's meshes of materials (several textures per triangle,
Sec. 3.1 Eq. 1 and Sec. 3.3) and of its physically based shading, against
facts fixed outside it: closed forms of the microfacet BRDF at normal
incidence, the ambient-only limits, Helmholtz reciprocity, energy
conservation of the directional albedo, and the paper's rule that a
triangle's sampling and each texture's fetch follow from that texture alone
(Eq. 1 takes the largest texel count; Eq. 6-7 use each texture's own
resolution)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2601_19901_gb300 import scenes as S

LIGHT = np.array([1.7, 1.3, 0.9], np.float32)
AMB = np.array([0.11, 0.07, 0.05], np.float32)


def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def test_pbr_without_light_is_ambient_times_albedo():
    alb = np.array([0.2, 0.5, 0.9])
    n = _unit([0.2, 0.3, 1.0])
    for rough, metal in ((0.3, 0.0), (0.9, 1.0), (0.5, 0.4)):
        out = O.pbr_shade(alb, rough, metal, n, _unit([0.1, -0.2, 1.0]), _unit([0.5, 0.5, 0.7]),
                          np.zeros(3, np.float32), AMB)
        assert np.allclose(out, AMB.astype(np.float64) * alb, rtol=0, atol=1e-12)


def test_pbr_light_behind_the_surface_gives_ambient_only():
    alb = np.array([0.6, 0.4, 0.3])
    n = np.array([0.0, 0.0, 1.0])
    out = O.pbr_shade(alb, 0.5, 0.3, n, _unit([0.2, 0.1, 1.0]), _unit([0.3, 0.2, -1.0]), LIGHT, AMB)
    assert np.allclose(out, AMB.astype(np.float64) * alb, rtol=0, atol=1e-12)


def test_pbr_normal_incidence_closed_forms():
    # n = v = l: h = n, so n.h = v.h = 1. With r = 1 (a = 1): D = 1 / pi,
    # k = 1/2, G = 1, F = F0. A dielectric (m = 0): F0 = 0.04, diffuse
    # 0.96 c / pi, specular 0.04 / (4 pi). A metal (m = 1): F0 = c, no diffuse,
    # specular c / (4 pi).
    n = np.array([0.0, 0.0, 1.0])
    c = np.array([0.25, 0.5, 0.75])
    L64, A64 = LIGHT.astype(np.float64), AMB.astype(np.float64)
    out = O.pbr_shade(c, 1.0, 0.0, n, n, n, LIGHT, AMB)
    assert np.allclose(out, (0.96 * c + 0.01) / math.pi * L64 + A64 * c, rtol=1e-12, atol=1e-14)
    out = O.pbr_shade(c, 1.0, 1.0, n, n, n, LIGHT, AMB)
    assert np.allclose(out, c / (4.0 * math.pi) * L64 + A64 * c, rtol=1e-12, atol=1e-14)


def test_pbr_brdf_is_reciprocal():
    # Helmholtz reciprocity: f(l, v) = f(v, l), f = (out - ambient) / (light n.l)
    rng = np.random.default_rng(4)
    n = np.array([0.0, 0.0, 1.0])
    ones = np.ones(3, np.float32)
    for _ in range(200):
        a = _unit(rng.normal(size=3) + [0, 0, 1.5])
        b = _unit(rng.normal(size=3) + [0, 0, 1.5])
        if a[2] < 0.05 or b[2] < 0.05:
            continue
        c = rng.random(3)
        rough, metal = float(rng.uniform(0.05, 1.0)), float(rng.random())
        f_ab = O.pbr_shade(c, rough, metal, n, a, b, ones, np.zeros(3, np.float32)) / b[2]
        f_ba = O.pbr_shade(c, rough, metal, n, b, a, ones, np.zeros(3, np.float32)) / a[2]
        assert np.allclose(f_ab, f_ba, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("rough,metal,bound", [(0.3, 1.0, 1.0), (0.6, 1.0, 1.0), (1.0, 1.0, 1.0),
                                               (0.3, 0.0, 1.05), (1.0, 0.0, 1.05)])
def test_pbr_directional_albedo_conserves_energy(rough, metal, bound):
    # white albedo, unit light: the integral over the hemisphere of f cos(l)
    # (midpoint rule in (cos theta, phi)) for several view angles. A white
    # metal is the microfacet specular lobe alone, whose shadowing-masking can
    # only lose energy: <= 1. A dielectric adds the Lambert term weighted by
    # 1 - F(v.h), which is not an exact complement of the specular albedo:
    # within 5 %.
    n = np.array([0.0, 0.0, 1.0])
    ones = np.ones(3, np.float32)
    nu, nphi = 96, 96
    mus = (np.arange(nu) + 0.5) / nu
    phis = (np.arange(nphi) + 0.5) / nphi * 2 * math.pi
    for mu_v in (0.95, 0.6, 0.25):
        v = np.array([math.sqrt(1 - mu_v * mu_v), 0.0, mu_v])
        tot = 0.0
        for mu in mus:
            st = math.sqrt(1 - mu * mu)
            for ph in phis:
                l = np.array([st * math.cos(ph), st * math.sin(ph), mu])
                out = O.pbr_shade(np.ones(3), rough, metal, n, v, l, ones, np.zeros(3, np.float32))
                tot += out[0]   # = f cos(l) for a unit light
        albedo = tot * (1.0 / nu) * (2 * math.pi / nphi)
        assert 0.0 < albedo <= bound, (mu_v, albedo)


def _plain(scene, tex_of_material):
    """The scene with one texture per triangle: the given texture of its material."""
    tt = np.array([tex_of_material[m] for m in scene.tri_tex], np.uint32)
    return S.Scene(xyz=scene.xyz, uv=scene.uv, idx=scene.idx, tri_tex=tt, textures=scene.textures)


def test_material_sampling_takes_the_largest_texture():
    # Eq. 1: a triangle's texel count is the largest over its material's
    # textures, so its sampling equals that of a mesh textured with the
    # material's largest texture alone
    d = S.display_tiny()
    sc = S.scene_pbr_tiny()
    m = S.model_matrix(2)
    sizes = [t.shape[0] * t.shape[1] for t in sc.textures]
    largest = [int(max(row, key=lambda k: sizes[k])) for row in sc.materials]
    st, tri, counts = O.setup(d, sc, m)
    st2, tri2, counts2 = O.setup(d, _plain(sc, largest), m)
    assert st == st2 == 0
    assert np.array_equal(counts, counts2) and counts.sum() > 1000
    for f in ("s_u", "s_v", "size_uv", "n_tex", "vpuv_min", "vpuv_max"):
        assert np.array_equal(tri[:, O.F[f]].view(np.uint32), tri2[:, O.F[f]].view(np.uint32)), f
    # the albedo is not the largest texture of either material here, so
    # sampling by the albedo alone would differ
    st3, _, counts3 = O.setup(d, _plain(sc, [int(r[0]) for r in sc.materials]), m)
    assert not np.array_equal(counts, counts3)


@pytest.mark.parametrize("slot", [0, 1, 2, 3])
def test_each_texture_is_fetched_as_if_alone(slot):
    # with slot `slot` the largest texture of every material (so the sampling
    # is that texture's), its fetched tv_min / tv_max equal those of the plain
    # fetch of the mesh textured by it alone (Eq. 6-7 at its own resolution)
    d = S.display_tiny()
    base = S.scene_pbr_tiny()
    sz = [64, 32, 32, 32]
    sz[0], sz[slot] = sz[slot], 128
    tex = S.material_textures(tuple(sz), 41) + S.material_textures(tuple(sz), 51)
    sc = S.Scene(xyz=base.xyz, uv=base.uv, idx=base.idx, tri_tex=base.tri_tex, textures=tex,
                 materials=base.materials)
    m = S.model_matrix(5)
    fr = O.render(d, sc, m, splat=False)
    plain = O.render(d, _plain(sc, [int(r[slot]) for r in sc.materials]), m, splat=False)
    assert np.array_equal(fr.counts, plain.counts)
    assert np.array_equal(fr.points[:, :2], plain.points[:, :2])
    got = fr.points[:, 2:] if slot == 0 else fr.tvx[:, 2 * (slot - 1):2 * slot]
    assert np.array_equal(got, plain.points[:, 2:])


def _quad_scene(normal_rgb):
    """A 2 x 2 quad at z = 0 facing the eyes (+z), texture s = (x + 1) / 2 and
    t = (y + 1) / 2, one material: grey albedo, a constant normal map, rough
    dielectric."""
    xyz = np.array([[-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, -1, 0], [1, 1, 0], [-1, 1, 0]], np.float32)
    uv = (xyz[:, :2] + 1.0) / 2.0
    const = lambda rgb: np.concatenate([np.full((4, 4, 3), rgb, np.uint8), np.full((4, 4, 1), 255, np.uint8)], -1)
    tex = [const((128, 128, 128)), const(normal_rgb), const((230, 230, 230)), const((0, 0, 0))]
    return S.Scene(xyz=xyz, uv=uv.astype(np.float32), idx=np.arange(6, dtype=np.uint32).reshape(2, 3),
                   tri_tex=np.zeros(2, np.uint32), textures=tex, materials=np.arange(4, dtype=np.uint32).reshape(1, 4))


@pytest.mark.parametrize("normal_rgb,light,lit", [
    ((128, 128, 255), (1.0, 0.0, 0.02), False),   # geometric normal: grazing light
    ((255, 128, 128), (1.0, 0.0, 0.02), True),    # tilted toward +s = world +x: faces the light
    ((0, 128, 128), (1.0, 0.0, 0.02), False),     # toward -s: faces away
    ((128, 255, 128), (0.0, 1.0, 0.02), True),    # toward +t = world +y
    ((128, 255, 128), (1.0, 0.0, 0.02), False),
])
def test_normal_map_tilts_the_shading_normal_along_the_texture_axes(normal_rgb, light, lit):
    # the shading frame's tangent and bitangent run along increasing texture s
    # and t; a normal map pointing along one of them faces a light from that
    # side (bright), a flat map or the other side leaves ambient only
    d = S.Display(n_views=1, view_w=64, view_h=64, cone_deg=10.0, view_dist=4.0, focal_w=3.0, focal_h=3.0,
                  near_z=0.1, far_z=100.0, bias_h=1.0, bias_v=1.0, panel_w=64, panel_h=64, lens_pitch_px=8.0,
                  slant=0.0)
    sh = S.Shading(light_dir=light, light_rgb=(3.0, 3.0, 3.0), ambient=(0.05, 0.05, 0.05))
    fr = O.render(d, _quad_scene(normal_rgb), np.eye(4, dtype=np.float32), shading=sh, panel=False)
    cov = fr.keys[0] != np.uint64(0xFFFFFFFFFFFFFFFF)
    assert cov.mean() > 0.3
    mean = float(fr.rgba[0][cov][:, :3].mean())
    ambient_only = 0.05 * 128.0   # ambient x albedo (128/255) x 255
    if lit:
        assert mean > 6 * ambient_only, mean
    else:
        assert mean < 2 * ambient_only, mean
