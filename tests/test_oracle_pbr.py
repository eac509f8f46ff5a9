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


def test_pbr_normal_incidence_closed_forms_at_roughness_one_half():
    # n = v = l, r = 1/2: a = r^2 = 1/4, D = 1 / (pi a^2) = 16 / pi, G = 1,
    # F = F0. Dielectric: (0.96 c + 0.04 * 16 / 4) / pi; metal: 4 c / pi.
    n = np.array([0.0, 0.0, 1.0])
    c = np.array([0.25, 0.5, 0.75])
    L64, A64 = LIGHT.astype(np.float64), AMB.astype(np.float64)
    out = O.pbr_shade(c, 0.5, 0.0, n, n, n, LIGHT, AMB)
    assert np.allclose(out, (0.96 * c + 0.16) / math.pi * L64 + A64 * c, rtol=1e-12, atol=1e-14)
    out = O.pbr_shade(c, 0.5, 1.0, n, n, n, LIGHT, AMB)
    assert np.allclose(out, 4.0 * c / math.pi * L64 + A64 * c, rtol=1e-12, atol=1e-14)


def test_pbr_mirror_pair_at_sixty_degrees_closed_forms():
    # n = z, v and l mirrored at 60 degrees: h = n, n.l = n.v = v.h = 1/2.
    # r = 1/2: D = 16 / pi; k = (3/2)^2 / 8 = 9/32, G1(1/2) = (1/2) / (23/64 +
    # 18/64) = 32/41, G = 1024/1681; 4 n.l n.v = 1; Schlick (1 - v.h)^5 = 1/32.
    n = np.array([0.0, 0.0, 1.0])
    s3 = math.sqrt(3.0) / 2.0
    v, l = np.array([s3, 0.0, 0.5]), np.array([-s3, 0.0, 0.5])
    c = np.array([0.2, 0.55, 0.9])
    L64, A64 = LIGHT.astype(np.float64), AMB.astype(np.float64)
    DG = 16.0 / math.pi * 1024.0 / 1681.0
    F = c + (1.0 - c) / 32.0                        # a metal: F0 = albedo
    out = O.pbr_shade(c, 0.5, 1.0, n, v, l, LIGHT, AMB)
    assert np.allclose(out, DG * F * L64 * 0.5 + A64 * c, rtol=1e-12, atol=1e-14)
    F = 0.04 + 0.96 / 32.0                          # a dielectric: F0 = 0.04
    out = O.pbr_shade(c, 0.5, 0.0, n, v, l, LIGHT, AMB)
    assert np.allclose(out, ((1.0 - F) * c / math.pi + DG * F) * L64 * 0.5 + A64 * c, rtol=1e-12, atol=1e-14)


def test_pbr_roughness_below_its_floor_shades_as_the_floor():
    # r is clamped at 0.045 (a = r^2 would make the GGX lobe a delta at 0)
    rng = np.random.default_rng(11)
    n = np.array([0.0, 0.0, 1.0])
    for _ in range(20):
        v = _unit(rng.normal(size=3) + [0, 0, 2.0])
        l = _unit(rng.normal(size=3) + [0, 0, 2.0])
        c, m = rng.random(3), float(rng.random())
        ref = O.pbr_shade(c, 0.045, m, n, v, l, LIGHT, AMB)
        for r in (0.0, 0.01, 0.044):
            out = O.pbr_shade(c, r, m, n, v, l, LIGHT, AMB)
            assert np.all(np.isfinite(out)) and np.array_equal(out, ref)
    assert np.all(np.isfinite(O.pbr_shade(np.ones(3), 0.0, 0.0, n, n, n, LIGHT, AMB)))


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


def _rect_material(slot, seed):
    """One material's four textures, 64 x 64 except slot `slot`: 256 x 32
    (the largest, and not square)."""
    wh = [(64, 64)] * 4
    wh[slot] = (256, 32)
    (wa, ha), (wn, hn), (wr, hr), (wm, hm) = wh
    return [S.value_noise_texture(wa, ha, seed), S.normal_map_texture(wn, hn, seed + 1),
            S.scalar_texture(wr, hr, seed + 2, 0.15, 0.95), S.scalar_texture(wm, hm, seed + 3, 0.0, 1.0)]


@pytest.mark.parametrize("slot", [0, 1, 2, 3])
def test_a_rectangular_texture_is_fetched_at_its_own_size(slot):
    # as above with textures of 256 x 32 texels: Eq. 6-7 take width x height
    d = S.display_tiny()
    base = S.scene_pbr_tiny()
    tex = _rect_material(slot, 61) + _rect_material(slot, 71)
    sc = S.Scene(xyz=base.xyz, uv=base.uv, idx=base.idx, tri_tex=base.tri_tex, textures=tex,
                 materials=base.materials)
    m = S.model_matrix(6)
    fr = O.render(d, sc, m, splat=False)
    plain = O.render(d, _plain(sc, [int(r[slot]) for r in sc.materials]), m, splat=False)
    assert np.array_equal(fr.counts, plain.counts)
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


def test_a_back_facing_quad_is_shaded_two_sided():
    # the quad with its winding reversed (geometric normal -z, away from the
    # eyes), a flat normal map and the light on the eyes' side: the shading
    # frame turns to the viewer, so it is lit as the front face is
    sc = _quad_scene((128, 128, 255))
    back = S.Scene(xyz=sc.xyz, uv=sc.uv, idx=sc.idx[:, ::-1].copy(), tri_tex=sc.tri_tex, textures=sc.textures,
                   materials=sc.materials)
    d = S.Display(n_views=1, view_w=64, view_h=64, cone_deg=10.0, view_dist=4.0, focal_w=3.0, focal_h=3.0,
                  near_z=0.1, far_z=100.0, bias_h=1.0, bias_v=1.0, panel_w=64, panel_h=64, lens_pitch_px=8.0,
                  slant=0.0)
    sh = S.Shading(light_dir=(0.0, 0.0, 1.0), light_rgb=(3.0, 3.0, 3.0), ambient=(0.05, 0.05, 0.05))
    means = []
    for scene in (sc, back):
        fr = O.render(d, scene, np.eye(4, dtype=np.float32), shading=sh, panel=False)
        cov = fr.keys[0] != np.uint64(0xFFFFFFFFFFFFFFFF)
        assert cov.mean() > 0.3
        means.append(float(fr.rgba[0][cov][:, :3].mean()))
    ambient_only = 0.05 * 128.0
    assert means[0] > 6 * ambient_only and means[1] > 6 * ambient_only
    assert abs(means[0] - means[1]) < 0.05 * means[0]


def _maps_scene(rough, metal):
    """The quad of _quad_scene with a flat normal map and constant roughness
    and metallic maps (R channel values)."""
    sc = _quad_scene((128, 128, 255))
    const = lambda v: np.concatenate([np.full((4, 4, 3), v, np.uint8), np.full((4, 4, 1), 255, np.uint8)], -1)
    tex = [sc.textures[0], sc.textures[1], const(rough), const(metal)]
    return S.Scene(xyz=sc.xyz, uv=sc.uv, idx=sc.idx, tri_tex=sc.tri_tex, textures=tex, materials=sc.materials)


def test_roughness_and_metallic_maps_each_drive_their_own_term():
    # grey albedo, light along the view axis: a dielectric is mostly Lambert,
    # a metal of the same roughness has no diffuse term and is much darker;
    # a rough and a smooth dielectric differ through the specular lobe
    d = S.Display(n_views=1, view_w=64, view_h=64, cone_deg=10.0, view_dist=4.0, focal_w=3.0, focal_h=3.0,
                  near_z=0.1, far_z=100.0, bias_h=1.0, bias_v=1.0, panel_w=64, panel_h=64, lens_pitch_px=8.0,
                  slant=0.0)
    sh = S.Shading(light_dir=(0.0, 0.0, 1.0), light_rgb=(3.0, 3.0, 3.0), ambient=(0.0, 0.0, 0.0))

    def mean(rough, metal):
        fr = O.render(d, _maps_scene(rough, metal), np.eye(4, dtype=np.float32), shading=sh, panel=False)
        cov = fr.keys[0] != np.uint64(0xFFFFFFFFFFFFFFFF)
        return float(fr.rgba[0][cov][:, :3].astype(np.float64).mean())

    dielectric, metal = mean(255, 0), mean(255, 255)
    assert dielectric > 2.0 * metal > 0.0
    assert abs(mean(40, 0) - dielectric) > 1.0

