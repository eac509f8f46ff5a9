"""GPU parity for geometry near the eyes: triangles whose cells reach within
near_z of the eyes' plane, or past it, are splatted from their cell and
triangle clipped to depth >= near_z (Sec. 3.2's splat of a cell that has no
bounded projection), and Eq. 8 weighs their drawable part. Against the
oracle, which tests every pixel of every view for such points."""
from dataclasses import replace

import numpy as np
import pytest

import oracle as O
from paper_2601_19901_gb300 import lfdpr, scenes as S

from parity import check_sampling, check_views, gpu_frame

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2601_19901_gb300 import build
    build.build()
    lfdpr.lib()


def quad(p0, p1, p2, p3):
    return [[p0, p1, p2], [p0, p2, p3]]


def near_scene(D: float, seed: int = 4) -> S.Scene:
    """A quad crossing the eyes' plane just above the eyes, one that reaches
    from depth 0.5 to 0.04 below them, and a background plane. The two near
    quads carry a 4 x 4 texture, so Eq. 3 gives them cells of several texels
    and the oracle can test every pixel for each of their points."""
    tris = []
    tris += quad([-0.8, -0.3, D - 0.8], [0.8, -0.3, D - 0.8], [0.8, 0.2, D + 0.4], [-0.8, 0.2, D + 0.4])
    tris += quad([-0.3, -0.12, D - 0.5], [0.35, -0.12, D - 0.5], [0.35, -0.004, D - 0.04], [-0.3, -0.004, D - 0.04])
    tris += quad([-1.5, -1.5, -1.0], [1.5, -1.5, -1.0], [1.5, 1.5, -1.0], [-1.5, 1.5, -1.0])
    tris = np.asarray(tris, np.float32)
    n = len(tris)
    uv = np.tile(np.array([[0, 0], [1, 0], [1, 1], [0, 0], [1, 1], [0, 1]], np.float32), (n // 2, 1))
    uv[-6:] *= 8.0                                           # the background: finer texels
    rng = np.random.default_rng(seed)
    coarse = rng.integers(0, 256, (4, 4, 4), dtype=np.uint8)
    fine = rng.integers(0, 256, (64, 64, 4), dtype=np.uint8)
    tri_tex = np.array([0, 0, 0, 0, 1, 1], np.uint32)
    return S.Scene(xyz=tris.reshape(-1, 3), uv=uv, idx=np.arange(3 * n, dtype=np.uint32).reshape(n, 3),
                   tri_tex=tri_tex, textures=[coarse, fine])


@pytest.mark.parametrize("recon", [0, 1])
def test_geometry_reaching_the_eyes_plane_matches_the_oracle(recon):
    d = replace(S.display_tiny(), recon=recon, crosstalk=0.15 if recon else 0.0)
    sc = near_scene(d.view_dist)
    m = np.eye(4, dtype=np.float32)
    o = O.render(d, sc, m)
    g = gpu_frame(d, sc, m)
    assert g.stats.overflow == 0 and g.stats.n_points == len(o.points)
    check_sampling(g, o, "near")
    # the near quads cover much of every view: their splats are drawn
    near_tris = (o.points[:, 0] < 4)
    ids = (g.keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    covered = g.keys != np.uint64(0xFFFFFFFFFFFFFFFF)
    drawn_near = np.isin(ids[covered], np.nonzero(near_tris)[0])
    assert drawn_near.mean() > 0.2
    agree, p = check_views(g, o, msg="near")
    assert agree >= 0.999
    assert np.array_equal(g.panel, O.interleave(d, g.views))
