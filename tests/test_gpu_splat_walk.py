"""The splat's two ways through a unit of four work points (Sec. 3.2): pooled
32-lane passes over the unit's numbered candidates, or, when some lane's
views hold `limit` or more candidates, a walk of the unit's (point, view)
segments one lane each. Both test the same candidates with the same
arithmetic, and atomicMin does not depend on the order, so the view keys
must be bit-identical whatever the limit; the walk is checked against the
oracle as well.
"""
import numpy as np
import pytest

import oracle as O
from paper_2601_19901_gb300 import lfdpr, scenes as S
from parity import check_views, gpu_frame

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    import torch
    assert torch.cuda.is_available()
    from paper_2601_19901_gb300 import build
    build.build()
    O.build()


@pytest.mark.parametrize("limit", [1, 3, 40])
def test_walked_units_give_the_pooled_keys(built, limit):
    d, sc, m = S.display_tiny(), S.scene_tiny(), S.model_matrix(2)
    with lfdpr.Renderer(d, sc) as R:
        pooled = gpu_frame(d, sc, m, renderer=R, panel=False)
        lfdpr.lfdpr_set_splat_lane_limit(R.disp, limit)
        walked = gpu_frame(d, sc, m, renderer=R, panel=False)
    assert pooled.stats.n_splat_writes > 0
    assert walked.stats.n_splat_writes == pooled.stats.n_splat_writes
    assert np.array_equal(walked.keys, pooled.keys)
    assert np.array_equal(walked.views, pooled.views)
    if limit == 1:
        check_views(walked, O.render(d, sc, m, panel=False), msg="lane walk")


def test_walked_units_full_size(built):
    # the paper-shaped frame: every unit walked (limit 1) against the pooled passes
    d, sc, m = S.display_paper(), S.scene_paper(), S.model_matrix(6)
    with lfdpr.Renderer(d, sc) as R:
        pooled = gpu_frame(d, sc, m, renderer=R, panel=False)
        lfdpr.lfdpr_set_splat_lane_limit(R.disp, 1)
        walked = gpu_frame(d, sc, m, renderer=R, panel=False)
    assert walked.stats.n_splat_writes == pooled.stats.n_splat_writes > 10_000_000
    assert np.array_equal(walked.keys, pooled.keys)


def test_lane_limit_is_checked(built):
    d = S.display_tiny()
    with lfdpr.Renderer(d, S.scene_tiny()) as R:
        for bad in (0, (1 << 24) + 1):
            with pytest.raises(lfdpr.LfdprError) as e:
                lfdpr.lfdpr_set_splat_lane_limit(R.disp, bad)
            assert e.value.status == lfdpr.EINVAL
        lfdpr.lfdpr_set_splat_lane_limit(R.disp, 1 << 24)
