"""Meshes of materials and physically based shading on the GPU against the
oracle (Sec. 3.1 Eq. 1 over several textures, Sec. 3.3 per-texture LOD pairs
and shading during view generation).

Sampling (counts, records, point set, albedo tv) and every texture's fetched
tv_min / tv_max are bit-exact; the shaded views (FP32 on the GPU, double in
the oracle) meet the parity tolerances: >= 99.9 % same winners, colour
within 1 of 255 on same-winner pixels, PSNR >= 50 dB.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle as O
from paper_2601_19901_gb300 import lfdpr, scenes as S
from parity import check_sampling, check_views, gpu_frame, ids_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    from paper_2601_19901_gb300 import build
    build.build()
    O.build()
    return S.scene_pbr_tiny()


def _gpu_tvx(R, n_points: int) -> np.ndarray:
    """The library's per-point normal / roughness / metallic values in the
    oracle's layout: (normal min, normal max, rough min, rough max, metal min,
    metal max), roughness and metallic as R bytes."""
    b = R.buffers()
    rr = lfdpr.device_to_numpy(b.resolve, (n_points, 8), np.uint32)
    nm = lfdpr.device_to_numpy(b.resolve_mat, (n_points, 2), np.uint32)
    rm = rr[:, 7]
    out = np.zeros((n_points, 6), np.uint32)
    out[:, 0] = nm[:, 0]
    out[:, 1] = nm[:, 1]
    for k in range(4):
        out[:, 2 + k] = (rm >> np.uint32(8 * k)) & np.uint32(255)
    return out


def _oracle_tvx_r(tvx: np.ndarray) -> np.ndarray:
    o = tvx.copy()
    o[:, 2:] &= np.uint32(255)
    return o


@pytest.mark.parametrize("frame", [0, 7])
def test_pbr_frame_matches_oracle(env, frame):
    sc = env
    d = S.display_tiny()
    sh = S.Shading()
    m = S.model_matrix(frame)
    with lfdpr.Renderer(d, sc, shading=sh) as R:
        g = gpu_frame(d, sc, m, renderer=R, panel=False)
        tvx = _gpu_tvx(R, g.points.shape[0])
    o = O.render(d, sc, m, shading=sh, panel=False)
    check_sampling(g, o, "pbr frame %d" % frame)
    assert np.array_equal(tvx, _oracle_tvx_r(o.tvx)), "normal / roughness / metallic fetch"
    agree, p = check_views(g, o, msg="pbr frame %d" % frame)
    assert agree > 0.999 and p >= 50.0
    # the views are shaded (not the unlit albedo) and differ between eyes
    assert not np.array_equal(g.views[0], g.views[-1])


def test_unlit_material_frame_matches_oracle(env):
    sc = env
    d = S.display_tiny()
    m = S.model_matrix(3)
    with lfdpr.Renderer(d, sc) as R:
        g = gpu_frame(d, sc, m, renderer=R)
    o = O.render(d, sc, m)
    check_sampling(g, o, "unlit materials")
    check_views(g, o, msg="unlit materials")
    assert np.array_equal(g.panel, O.interleave(d, g.views))


def test_pbr_needs_a_mesh_of_materials(env):
    d = S.display_tiny()
    plain = S.scene_tiny()
    with lfdpr.Renderer(d, plain) as R:
        lfdpr.lfdpr_set_shading(R.disp, S.Shading())
        with pytest.raises(lfdpr.LfdprError) as e:
            R.render(S.model_matrix(0))
        assert e.value.status == lfdpr.EINVAL
        lfdpr.lfdpr_set_shading(R.disp, None)   # back to unlit: renders
        R.render(S.model_matrix(0))


def test_shading_arguments_are_checked(env):
    d = S.display_tiny()
    with lfdpr.Renderer(d, env) as R:
        for bad in (S.Shading(light_dir=(0.0, 0.0, 0.0)), S.Shading(light_rgb=(-1.0, 1.0, 1.0)),
                    S.Shading(ambient=(float("nan"), 0.0, 0.0))):
            with pytest.raises(lfdpr.LfdprError) as e:
                lfdpr.lfdpr_set_shading(R.disp, bad)
            assert e.value.status == lfdpr.EINVAL
    with pytest.raises(lfdpr.LfdprError) as e:
        disp = lfdpr.lfdpr_create_display(lfdpr.desc_of(d))
        try:
            ts = lfdpr.TextureSet(env.textures)
            try:
                bad = np.array(env.materials, np.uint32)
                bad[0, 2] = 99
                lfdpr.lfdpr_upload_mesh_materials(disp, env.xyz, env.uv, env.idx, env.tri_tex, bad, ts.handle)
            finally:
                ts.close()
        finally:
            lfdpr.lfdpr_destroy_display(disp)
    assert e.value.status == lfdpr.EINVAL


def test_pbr_full_size_sampled_views():
    # the paper-shaped scene with materials on the 48-view display, in the
    # configuration the bench times: the whole sampling bit-exact, every
    # texture's fetch bit-exact, and views 0 and 47 against the oracle
    import torch
    from paper_2601_19901_gb300 import build
    build.build()
    O.build()
    sc = S.scene_pbr_paper()
    d = S.display_paper()
    sh = S.Shading()
    m = S.model_matrix(4)
    with lfdpr.Renderer(d, sc, shading=sh) as R:
        g = gpu_frame(d, sc, m, renderer=R, panel=False)
        tvx = _gpu_tvx(R, g.points.shape[0])
    views = [0, 47]
    o = O.render(d, sc, m, views=views, panel=False, shading=sh)
    check_sampling(g, o, "pbr full size")
    assert np.array_equal(tvx, _oracle_tvx_r(o.tvx)), "normal / roughness / metallic fetch"
    check_views(g, o, views=views, msg="pbr full size")
