"""The allocation-free point-generation entry point against the regular path.

Callers that cannot allocate device memory while they run - a render loop that
allocates only at start-up, or a plug-in whose host application owns all
device memory - call lfdpr_sample_points_noalloc with buffers they already
own; its scratch is a fixed array inside the library. Its output must equal
the regular path's point generation with the tolerance every sampling test
here uses (bit-exact counts and point set), on two calls in a row: the second
call reuses the scratch the first one left behind. The second call must not
change the device's free memory.
"""
import numpy as np
import pytest

from paper_2601_19901_gb300 import lfdpr, scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    assert torch.cuda.is_available()
    from paper_2601_19901_gb300 import build
    build.build()
    d = S.display_tiny()
    sc = S.scene_tiny()
    dev = torch.device("cuda")
    bufs = dict(xyz=torch.from_numpy(sc.xyz).to(dev), uv=torch.from_numpy(sc.uv).to(dev),
                idx=torch.from_numpy(sc.idx.astype(np.int32)).to(dev),
                tri_tex=torch.from_numpy(sc.tri_tex.astype(np.int32)).to(dev))
    wh = np.array([[t.shape[1], t.shape[0]] for t in sc.textures], np.uint32)
    return d, sc, bufs, wh


def _noalloc(d, sc, bufs, wh, model, cap, stream):
    import torch
    pts = torch.zeros((max(cap, 1), 4), dtype=torch.int32, device="cuda")
    counts = torch.zeros(sc.n_tris, dtype=torch.int32, device="cuda")
    fc = torch.zeros(4, dtype=torch.int32, device="cuda")
    lfdpr.lfdpr_sample_points_noalloc(lfdpr.desc_of(d), model, bufs["xyz"].data_ptr(), bufs["uv"].data_ptr(),
                                      bufs["idx"].data_ptr(), bufs["tri_tex"].data_ptr(), sc.n_tris, wh,
                                      pts.data_ptr(), cap, counts.data_ptr(), fc.data_ptr(), stream)
    torch.cuda.synchronize()
    return (pts.cpu().numpy().view(np.uint32), counts.cpu().numpy().view(np.uint32),
            fc.cpu().numpy().view(np.uint32))


def test_noalloc_matches_the_regular_entry_point_on_two_calls(setup):
    import torch
    d, sc, bufs, wh = setup
    s = torch.cuda.current_stream()
    with lfdpr.Renderer(d, sc) as R:
        for frame in (3, 11):                      # two calls in a row, different frames
            m = S.model_matrix(frame)
            R.render(m, s)
            st = R.stats(s)
            b = R.buffers()
            n = int(st.n_points)
            ref_counts = lfdpr.device_to_numpy(b.counts, (sc.n_tris,), np.uint32)
            ref_pts = lfdpr.device_to_numpy(b.points, (n, 4), np.uint32)[:, :2]
            pts, counts, fc = _noalloc(d, sc, bufs, wh, m, n + 17, s)
            assert fc[0] == n and fc[1] == 0 and fc[2] == 0 and fc[3] == st.n_live_tris
            assert np.array_equal(counts, ref_counts)
            assert np.array_equal(pts[:n, :2], ref_pts)
            assert np.all(pts[n:] == 0)             # nothing written past the point set


def test_noalloc_second_call_leaves_free_device_memory_unchanged(setup):
    import torch
    d, sc, bufs, wh = setup
    s = torch.cuda.current_stream()
    cap = 1 << 16
    pts = torch.zeros((cap, 4), dtype=torch.int32, device="cuda")
    counts = torch.zeros(sc.n_tris, dtype=torch.int32, device="cuda")
    fc = torch.zeros(4, dtype=torch.int32, device="cuda")

    def call(frame):
        lfdpr.lfdpr_sample_points_noalloc(lfdpr.desc_of(d), S.model_matrix(frame), bufs["xyz"].data_ptr(),
                                          bufs["uv"].data_ptr(), bufs["idx"].data_ptr(),
                                          bufs["tri_tex"].data_ptr(), sc.n_tris, wh, pts.data_ptr(), cap,
                                          counts.data_ptr(), fc.data_ptr(), s)
        torch.cuda.synchronize()

    call(1)                                   # loads the kernels and looks up the scratch address
    free0, _ = torch.cuda.mem_get_info()
    call(2)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert fc.cpu()[0] > 0


def test_noalloc_with_angular_supersampling_matches_the_regular_entry_point(setup):
    """2N rendered views (recon 1): the eyes at the half-interval steps."""
    import torch
    from dataclasses import replace
    _, sc, bufs, wh = setup
    d = replace(S.display_tiny(), n_views=5, recon=1)
    s = torch.cuda.current_stream()
    with lfdpr.Renderer(d, sc) as R:
        m = S.model_matrix(6)
        R.render(m, s)
        st = R.stats(s)
        b = R.buffers()
        n = int(st.n_points)
        ref_counts = lfdpr.device_to_numpy(b.counts, (sc.n_tris,), np.uint32)
        ref_pts = lfdpr.device_to_numpy(b.points, (n, 4), np.uint32)[:, :2]
        pts, counts, fc = _noalloc(d, sc, bufs, wh, m, n, s)
        assert fc[0] == n and fc[1] == 0 and fc[3] == st.n_live_tris
        assert np.array_equal(counts, ref_counts)
        assert np.array_equal(pts[:n, :2], ref_pts)


def test_noalloc_with_large_triangles_matches_the_regular_entry_point():
    """Triangles of more than 128 points (a warp writes each one's points,
    its list held in the fixed scratch)."""
    import sys
    import os
    import torch
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from test_gpu_parity import large_triangles_scene
    d = S.display_paper()
    sc = large_triangles_scene()
    dev = torch.device("cuda")
    bufs = dict(xyz=torch.from_numpy(sc.xyz).to(dev), uv=torch.from_numpy(sc.uv).to(dev),
                idx=torch.from_numpy(sc.idx.astype(np.int32)).to(dev),
                tri_tex=torch.from_numpy(sc.tri_tex.astype(np.int32)).to(dev))
    wh = np.array([[t.shape[1], t.shape[0]] for t in sc.textures], np.uint32)
    s = torch.cuda.current_stream()
    with lfdpr.Renderer(d, sc) as R:
        m = S.model_matrix(2)
        R.render(m, s)
        st = R.stats(s)
        b = R.buffers()
        n = int(st.n_points)
        ref_counts = lfdpr.device_to_numpy(b.counts, (sc.n_tris,), np.uint32)
        ref_pts = lfdpr.device_to_numpy(b.points, (n, 4), np.uint32)[:, :2]
        assert ref_counts.max() > 10000
        pts, counts, fc = _noalloc(d, sc, bufs, wh, m, n, s)
        assert fc[0] == n and fc[1] == 0
        assert np.array_equal(counts, ref_counts)
        assert np.array_equal(pts[:n, :2], ref_pts)


def test_noalloc_reports_overflow_without_writing(setup):
    import torch
    d, sc, bufs, wh = setup
    pts, counts, fc = _noalloc(d, sc, bufs, wh, S.model_matrix(0), 100, torch.cuda.current_stream())
    assert fc[0] > 100 and fc[1] == 1
    assert np.all(pts == 0)


def test_noalloc_rejects_sizes_beyond_its_maximum(setup):
    d, sc, bufs, wh = setup
    with pytest.raises(lfdpr.LfdprError) as e:
        lfdpr.lfdpr_sample_points_noalloc(lfdpr.desc_of(d), S.model_matrix(0), 256, 256, 256, 256,
                                          lfdpr.NOALLOC_MAX_TRIS + 1, wh, 256, 10, 256, 256)
    assert e.value.status == lfdpr.EINVAL
    assert "fixed maximum" in lfdpr.lib().lfdpr_last_error().decode()
