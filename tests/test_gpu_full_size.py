"""Parity at the full paper-shaped size (10^6 triangles, 48 views of 420x560,
2560x1600 panel) in the launch configuration the benchmark times: the whole
point set and every triangle record bit-exact, and sampled views (the two
outermost and one central) against the oracle's splat and resolve of those
views."""
import numpy as np
import pytest

import oracle as O
from paper_2601_19901_gb300 import lfdpr, scenes as S

from parity import check_sampling, check_views, gpu_frame, psnr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    import torch
    assert torch.cuda.is_available()
    from paper_2601_19901_gb300 import build
    build.build()
    d = S.display_paper()
    sc = S.scene_paper()
    return d, sc


@pytest.mark.parametrize("frame", [0, 17])
def test_full_size_frame(full, frame):
    d, sc = full
    m = S.model_matrix(frame)
    g = gpu_frame(d, sc, m)
    o = O.render(d, sc, m, splat=False)
    assert g.stats.n_points == len(o.points) > 2_000_000
    check_sampling(g, o, "full size")
    views = [0, 23, 47]
    keys, rgba = O.splat_resolve(d, o.tri, o.points, views)

    class Sub:
        pass
    sub = Sub()
    sub.keys, sub.rgba = keys, rgba
    check_views(g, sub, views, "full size")
    # the panel from the GPU's own views is the oracle's interleave of them
    assert np.array_equal(g.panel, O.interleave(d, g.views))
