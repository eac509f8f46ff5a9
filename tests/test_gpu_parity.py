"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs (tolerances in tests/parity.py)."""
from dataclasses import replace

import numpy as np
import pytest

import oracle as O
from paper_2601_19901_gb300 import lfdpr, scenes as S

from parity import check_sampling, check_views, gpu_frame, psnr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2601_19901_gb300 import build
    build.build()
    lfdpr.lib()


def mini_paper_scene(seed=3):
    """Paper-shaped scene at a size the oracle renders in seconds: 6 instances
    of 2 x 20^2 triangles (4,800 triangles: 18 full set-up blocks and a ragged
    tail), textures 16^2 .. 512^2."""
    return S.scene_paper(n_instances=6, res=20, n_textures=6, max_tex=512, min_tex=16, seed=seed,
                         r_max=0.6)


def mini_paper_display(ss=False):
    d = S.display_angular_ss() if ss else S.display_paper()
    return replace(d, view_w=105, view_h=140, panel_w=640, panel_h=400)


def full_check(d, sc, model, views=None):
    o = O.render(d, sc, model)
    g = gpu_frame(d, sc, model)
    assert np.array_equal(g.eyes.view(np.uint32), O.eyes(d).view(np.uint32)), "eye positions"
    assert g.stats.overflow == 0 and g.stats.n_points == len(o.points)
    check_sampling(g, o)
    agree, p = check_views(g, o)
    # interleave: bit-exact on the same views, and close to the oracle's panel
    assert np.array_equal(g.panel, O.interleave(d, g.views))
    assert psnr(g.panel, o.panel) >= 50.0
    return g, o, agree


@pytest.mark.parametrize("frame", [0, 7])
def test_tiny_scene_full_frame(frame):
    d = S.display_tiny()
    sc = S.scene_tiny()
    g, o, agree = full_check(d, sc, S.model_matrix(frame))
    assert g.stats.n_live_tris == int((o.tri[:, O.F["live"]] == 1).sum())


@pytest.mark.parametrize("frame", [0, 3])
def test_paper_shaped_mini_full_frame(frame):
    d = mini_paper_display()
    sc = mini_paper_scene()
    full_check(d, sc, S.model_matrix(frame))


def test_angular_supersampling_mini_full_frame():
    d = mini_paper_display(ss=True)
    assert d.n_render_views == 96 and d.crosstalk == 0.15
    sc = mini_paper_scene(seed=5)
    full_check(d, sc, S.model_matrix(2))


def test_several_frames_on_one_renderer_match_fresh_frames():
    d = S.display_tiny()
    sc = S.scene_tiny()
    with lfdpr.Renderer(d, sc) as R:
        for frame in (1, 40, 2):
            m = S.model_matrix(frame)
            g = gpu_frame(d, sc, m, renderer=R)
            o = O.render(d, sc, m, panel=False)
            check_sampling(g, o)
            check_views(g, o)


@pytest.mark.parametrize("variant", ["tent", "supersampled", "gauss", "view_mips", "odd_width"])
def test_host_panel_equals_device_panel(variant):
    """Device, pinned host (written through its device mapping) and pageable
    host panels (a copy of the device scratch) hold the same bytes, for every
    interleave kernel; pinned memory at a 4-byte offset too."""
    import torch
    base = S.display_tiny()
    d = {"tent": base,
         "supersampled": replace(base, recon=1, crosstalk=0.15),
         "gauss": replace(base, recon=2, crosstalk=0.15),
         "view_mips": replace(base, view_w=256, view_h=256, ss_level=1),
         "odd_width": replace(base, panel_w=509, panel_h=131)}[variant]
    sc = S.scene_tiny()
    with lfdpr.Renderer(d, sc) as R:
        if variant == "gauss":
            R.set_view_jitter(np.random.default_rng(1).random(d.n_render_views).astype(np.float32))
            R.set_recon_samples((np.random.default_rng(2).normal(0.0, 0.3, (8, 3))).astype(np.float32))
        s = torch.cuda.current_stream()
        R.render(S.model_matrix(3), s)
        dev = torch.zeros((d.panel_h, d.panel_w, 4), dtype=torch.uint8, device="cuda")
        R.interleave(dev.data_ptr(), s)
        host = torch.zeros((d.panel_h, d.panel_w, 4), dtype=torch.uint8).pin_memory()
        R.interleave(host.data_ptr(), s)
        pageable = np.zeros((d.panel_h, d.panel_w, 4), np.uint8)
        R.interleave(pageable.ctypes.data, s)
        nb = d.panel_h * d.panel_w * 4
        shifted = torch.zeros(nb + 16, dtype=torch.uint8).pin_memory()
        R.interleave(shifted.data_ptr() + 4, s)
        torch.cuda.synchronize()
        ref = dev.cpu().numpy()
        assert ref.any()
        assert np.array_equal(ref, host.numpy())
        assert np.array_equal(ref, pageable)
        assert np.array_equal(ref.reshape(-1), shifted.numpy()[4:4 + nb])


def test_device_panel_must_be_4_byte_aligned():
    import torch
    d = S.display_tiny()
    with lfdpr.Renderer(d, S.scene_tiny()) as R:
        s = torch.cuda.current_stream()
        R.render(S.model_matrix(3), s)
        buf = torch.zeros(d.panel_h * d.panel_w * 4 + 16, dtype=torch.uint8, device="cuda")
        with pytest.raises(lfdpr.LfdprError, match="4-byte aligned"):
            R.interleave(buf.data_ptr() + 2, s)
        R.interleave(buf.data_ptr() + 4, s)   # 4-byte aligned, not 16: the narrow stores
        torch.cuda.synchronize()


# ---------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------

def tri_scene(tris, uvs=None, tex=None):
    tris = np.asarray(tris, np.float32).reshape(-1, 3, 3)
    n = len(tris)
    uv = np.tile(np.array([[0, 0], [1, 0], [0, 1]], np.float32), (n, 1)) if uvs is None \
        else np.asarray(uvs, np.float32).reshape(-1, 2)
    t = tex if tex is not None else S.value_noise_texture(64, 64, 7)
    return S.Scene(xyz=tris.reshape(-1, 3), uv=uv, idx=np.arange(3 * n, dtype=np.uint32).reshape(n, 3),
                   tri_tex=np.zeros(n, np.uint32), textures=[t])


def test_empty_mesh():
    d = S.display_tiny()
    sc = S.Scene(xyz=np.zeros((0, 3), np.float32), uv=np.zeros((0, 2), np.float32),
                 idx=np.zeros((0, 3), np.uint32), tri_tex=np.zeros(0, np.uint32),
                 textures=[S.value_noise_texture(8, 8, 1)])
    g = gpu_frame(d, sc, S.model_matrix(0))
    assert g.stats.n_points == 0
    assert np.all(g.keys == np.uint64(0xFFFFFFFFFFFFFFFF)) and np.all(g.views == 0)
    assert np.all(g.panel[..., :3] == 0) and np.all(g.panel[..., 3] == 255)


def test_all_culled_and_degenerate_triangles():
    d = S.display_tiny()
    tris = [[[-50, 0, 0], [-49, 0, 0], [-50, 1, 0]],            # outside every view
            [[0, 0, 10], [1, 0, 10], [0, 1, 10]],                # behind the eyes
            [[0, 0, 0], [0.2, 0.2, 0], [0.4, 0.4, 0]],           # zero area
            [[0.1, 0.1, 0], [0.1, 0.1, 0], [0.1, 0.1, 0]],       # a point
            [[-0.3, -0.2, 0.1], [0.3, -0.2, 0.0], [0.0, 0.4, 0.2]]]  # ordinary, degenerate UVs below
    uvs = np.array([[0, 0], [1, 0], [0, 1]] * 4 + [[0.5, 0.5]] * 3, np.float32)
    sc = tri_scene(tris, uvs=uvs)
    m = np.eye(4, dtype=np.float32)
    o = O.render(d, sc, m)
    g = gpu_frame(d, sc, m)
    assert list(g.counts[:4]) == [0, 0, 0, 0] and g.counts[4] > 0
    check_sampling(g, o)
    check_views(g, o)


def test_overflow_reported_then_recovers():
    d = S.display_tiny()
    sc = S.scene_tiny()
    m = S.model_matrix(0)
    need = int(O.setup(d, sc, m)[2].sum())
    with lfdpr.Renderer(d, sc, max_points=need - 1) as R:
        R.render(m)
        with pytest.raises(lfdpr.LfdprError) as e:
            R.stats()
        assert e.value.status == lfdpr.EOVERFLOW
    g = gpu_frame(d, sc, m, max_points=need)
    assert g.stats.n_points == need


@pytest.mark.parametrize("case", ["index", "texture_id", "nan_vertex", "npot_texture", "no_texture"])
def test_invalid_mesh_rejected(case):
    d = S.display_tiny()
    sc = S.scene_tiny()
    xyz, uv, idx, tt, tex = sc.xyz.copy(), sc.uv.copy(), sc.idx.copy(), sc.tri_tex.copy(), list(sc.textures)
    if case == "index":
        idx[5, 1] = len(xyz)
    elif case == "texture_id":
        tt[3] = 1
    elif case == "nan_vertex":
        xyz[2, 0] = np.nan
    elif case == "npot_texture":
        tex = [np.zeros((48, 64, 4), np.uint8)]
    elif case == "no_texture":
        tex = []
    disp = lfdpr.lfdpr_create_display(lfdpr.desc_of(d))
    try:
        with pytest.raises(lfdpr.LfdprError) as e:
            lfdpr.lfdpr_upload_mesh(disp, xyz, uv, idx, tt, tex)
        assert e.value.status == lfdpr.EINVAL
    finally:
        lfdpr.lfdpr_destroy_display(disp)


def test_nonfinite_model_rejected():
    d = S.display_tiny()
    with lfdpr.Renderer(d, S.scene_tiny()) as R:
        m = S.model_matrix(0)
        m[1, 3] = np.inf
        with pytest.raises(lfdpr.LfdprError) as e:
            R.render(m)
        assert e.value.status == lfdpr.EINVAL


@pytest.mark.parametrize("band", [5, 16])
def test_view_bands_give_the_same_frame(band):
    """Clearing, splatting and resolving the views band by band leaves every
    key, view and the panel as rendering all views at once."""
    d = mini_paper_display(ss=True)          # 96 rendered views: 20 bands of 5 (the last of 1), or 6 of 16
    sc = mini_paper_scene(seed=7)
    m = S.model_matrix(4)
    g0 = gpu_frame(d, sc, m)
    with lfdpr.Renderer(d, sc) as R:
        lfdpr.lfdpr_set_view_band(R.disp, band)
        R.set_stage_timing(True)
        g1 = gpu_frame(d, sc, m, renderer=R)
        st = R.stats()
    assert np.array_equal(g0.keys, g1.keys)
    assert np.array_equal(g0.views, g1.views)
    assert np.array_equal(g0.panel, g1.panel)
    assert g1.stats.n_splat_writes == g0.stats.n_splat_writes
    assert st.stage_ms[lfdpr.STAGES.index("splat")] > 0.0 and st.stage_ms[lfdpr.STAGES.index("resolve")] > 0.0


def large_triangles_scene():
    """Triangles of a few hundred to tens of thousands of points each on the
    paper-shaped display (fine textures, so Eq. 3 keeps the cells at pixel
    size), with slanted edges for ragged columns, and some small ones."""
    rng = np.random.default_rng(12)
    tris = [[[-0.9, -0.8, 0.2], [0.7, -0.9, -0.3], [-0.6, 0.9, 0.1]],
            [[0.1, 0.1, 0.5], [0.5, 0.15, 0.4], [0.2, 0.6, 0.45]],
            [[-0.3, -0.2, 0.8], [-0.1, -0.25, 0.7], [-0.2, 0.05, 0.75]],
            [[0.3, -0.7, -0.5], [0.8, -0.2, -0.9], [0.35, -0.1, -0.4]]]
    for _ in range(40):
        c = rng.uniform(-0.8, 0.8, 3)
        tris.append((c + rng.normal(0.0, 0.02, (3, 3))).tolist())
    tris = np.asarray(tris, np.float32)
    n = len(tris)
    uv = rng.uniform(0.0, 4.0, (n * 3, 2)).astype(np.float32)
    tex = rng.integers(0, 256, (1024, 1024, 4), dtype=np.uint8)
    return S.Scene(xyz=tris.reshape(-1, 3), uv=uv, idx=np.arange(3 * n, dtype=np.uint32).reshape(n, 3),
                   tri_tex=np.zeros(n, np.uint32), textures=[tex])


def test_large_triangles_emit_the_oracle_point_set():
    """Triangles of more than 128 points are emitted by a warp each
    (k_emit_big): counts and the whole point set bit-exact, views as usual."""
    d = S.display_paper()
    sc = large_triangles_scene()
    m = S.model_matrix(2)
    o = O.render(d, sc, m, views=[0, 47], panel=False)
    assert o.counts.max() > 10000 and (o.counts > 128).sum() >= 3 and (o.counts[o.counts > 0] <= 128).sum() >= 10
    g = gpu_frame(d, sc, m, panel=False)
    check_sampling(g, o, "large triangles")
    check_views(g, o, views=[0, 47], msg="large triangles")


def test_consecutive_frames_scan_and_emit_like_the_oracle():
    """Set-up, scan and emit over several frames in a row on one renderer,
    each with its own model (one with nothing live): every count,
    first-point offset and point bit-exact."""
    d = S.display_paper()
    sc = S.scene_paper(n_instances=24, res=24, n_textures=4, max_tex=256, min_tex=16, seed=9)
    assert sc.n_tris > 40 * 256
    with lfdpr.Renderer(d, sc) as R:
        for k, f in enumerate((0, 17, 40, 17, 91)):
            m = S.model_matrix(f)
            if k == 3:
                m = m.copy()
                m[0, 3] += 5.0   # the whole mesh out of every view: nothing live
            o = O.render(d, sc, m, splat=False)
            g = gpu_frame(d, sc, m, panel=False, renderer=R)
            assert g.stats.overflow == 0 and g.stats.n_points == len(o.points), (k, g.stats.n_points)
            check_sampling(g, o, "frame %d" % k)
            if k == 3:
                assert g.stats.n_points == 0 and g.stats.n_live_tris == 0


def _column_cases_scene(h: float):
    """A sliver of two lattice columns whose first holds exactly 2^16 rows
    (the most a column may hold), two triangles of many columns, and small
    ones of one to four columns, all facing the eyes at z = 0."""
    rng = np.random.default_rng(21)
    tris = [[[-0.003, -h / 2, 0.0], [0.003, -h / 2, 0.0], [0.0, h / 2, 0.0]],
            [[-0.6, -0.5, 0.0], [-0.45, -0.52, 0.0], [-0.55, -0.47, 0.0]],
            [[0.3, 0.3, 0.0], [0.5, 0.32, 0.0], [0.33, 0.36, 0.0]]]
    for _ in range(60):
        c = np.array([rng.uniform(-0.7, 0.7), rng.uniform(-0.9, 0.9), 0.0])
        tris.append((c + np.concatenate([rng.normal(0.0, 0.006, (3, 2)), np.zeros((3, 1))], 1)).tolist())
    tris = np.asarray(tris, np.float32)
    n = len(tris)
    uv = np.tile(np.asarray([[0.0, 0.0], [1.0, 0.0], [0.5, 1.0]], np.float32), (n, 1))
    tex = np.random.default_rng(22).integers(0, 256, (1024, 1024, 4), dtype=np.uint8)
    return S.Scene(xyz=tris.reshape(-1, 3), uv=uv, idx=np.arange(3 * n, dtype=np.uint32).reshape(n, 3),
                   tri_tex=np.zeros(n, np.uint32), textures=[tex])


def test_column_summaries_and_column_walks_emit_the_oracle_point_set():
    """k_emit writes a triangle of at most four lattice columns from the
    column summary k_setup keeps, and walks the columns again for a wider
    one or for a column of 2^16 rows (which the summary's 16-bit row count
    cannot hold): counts, records and the point set bit-exact either way."""
    d = S.display_paper()
    m = np.eye(4, dtype=np.float32)
    probe = O.render(d, _column_cases_scene(1.0), m, splat=False, panel=False)
    sv = float(probe.tri[0, O.F["s_v"]])
    sc = _column_cases_scene(65535.5 * sv)
    o = O.render(d, sc, m, splat=False, panel=False)
    assert o.status == 0
    tri_of = o.points[:, 0].astype(np.int64)
    col = (o.points[:, 1] & 0xffff).astype(np.int64)
    ncols = np.array([len(np.unique(col[tri_of == t])) for t in range(sc.n_tris)])
    assert ((tri_of == 0) & (col == 0)).sum() == 65536 and ncols[0] == 2
    assert ncols[1] > 4 and ncols[2] > 4
    assert ((ncols >= 1) & (ncols <= 4)).sum() >= 20
    g = gpu_frame(d, sc, m, panel=False)
    assert g.stats.overflow == 0 and g.stats.n_points == len(o.points)
    check_sampling(g, o, "column cases")
