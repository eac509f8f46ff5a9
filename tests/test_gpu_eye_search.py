"""GPU parity for the closest and farthest eye (Fig. 5) on geometry chosen to
make the search hard: the set-up kernel evaluates the per-view distance only
for views that convexity along the eye line and a rounding bound cannot rule
out, and its d_min and d_max must still equal the minimum and maximum over
every view (checked through every record field that depends on them, and
the point set, bit for bit against the oracle's loop over all views).

The scene holds:
- quads facing the eyes and a floor under them, where the distance is the
  same for many eyes in exact arithmetic, and quads tilted so slightly that
  the computed distances of neighbouring eyes differ only by rounding;
- triangles with an edge along the eye line (a flat in-plane distance);
- triangles in the plane of the eye line (zero height for every eye);
- far triangles (a large rounding bound against the spacing of the eyes);
- triangles just below the eyes' plane, off to the sides of the eye line and
  point-like ones centred midway between two eyes (ties);
- random triangles of every orientation and size.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle as O
from paper_2601_19901_gb300 import lfdpr, scenes as S

from parity import check_sampling, gpu_frame

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2601_19901_gb300 import build
    build.build()
    lfdpr.lib()
    O.build()


def quad(p0, p1, p2, p3):
    return [[p0, p1, p2], [p0, p2, p3]]


def eye_search_scene(d: S.Display, seed: int = 31) -> S.Scene:
    rng = np.random.default_rng(seed)
    D = d.view_dist
    tris = []
    # facing the eyes, spanning the eye line's x range, and a floor
    tris += quad([-2.0, -0.05, 0.0], [2.0, -0.05, 0.0], [2.0, 0.05, 0.0], [-2.0, 0.05, 0.0])
    tris += quad([-0.5, -0.3, 1.0], [0.5, -0.3, 1.0], [0.5, -0.3, 1.5], [-0.5, -0.3, 1.5])
    # the same, tilted about the vertical by less than the rounding can see,
    # so that the computed distances of neighbouring eyes go up and down
    for k, slope in enumerate((1e-7, 1e-6, -3e-6, 1e-5)):
        y0 = -0.05 if k % 2 == 0 else -0.3
        z0 = 0.0 if k < 2 else -0.5
        tris += quad([-2.0, y0, z0 - 2.0 * slope], [2.0, y0, z0 + 2.0 * slope],
                     [2.0, y0 + 0.1, z0 + 2.0 * slope], [-2.0, y0 + 0.1, z0 - 2.0 * slope])
    # an edge along the eye line's direction: upright and tilted
    tris.append([[-1.5, -0.5, 0.2], [1.5, -0.5, 0.2], [0.0, -1.0, 0.2]])
    tris.append([[-1.2, 0.4, 0.5], [1.2, 0.4, 0.5], [0.1, 0.9, -0.4]])
    # in the plane y = 0, which holds the eye line
    tris.append([[-0.6, 0.0, -0.5], [0.7, 0.0, 0.4], [0.1, 0.0, -1.2]])
    tris.append([[-0.2, 0.0, 1.0], [0.3, 0.0, 1.1], [0.0, 0.0, 0.6]])
    # just below the eyes' plane, and off to the sides
    for x in (-1.3, 0.0, 0.9):
        tris.append([[x, -0.02, D - 0.3], [x + 0.01, -0.02, D - 0.3], [x, 0.0, D - 0.29]])
    for x in (-3.0, 3.0):
        tris.append([[x, -0.2, -4.0], [x + 0.3, -0.2, -4.0], [x, 0.2, -4.1]])
    # point-like triangles centred midway between neighbouring eyes
    ex = O.eyes(d).astype(np.float64)
    for k in range(0, len(ex) - 1, max(1, len(ex) // 6)):
        xm = 0.5 * (ex[k] + ex[k + 1])
        for z in (0.5, -1.0):
            tris.append([[xm - 5e-4, 0.01, z], [xm + 5e-4, 0.01, z], [xm, 0.011, z]])
    # far, then random
    for _ in range(40):
        c = np.array([rng.uniform(-30, 30), rng.uniform(-20, 20), rng.uniform(-90, -60)])
        tris.append((c + rng.normal(0.0, 0.5, (3, 3))).tolist())
    for _ in range(400):
        c = np.array([rng.uniform(-1.5, 1.5), rng.uniform(-1.0, 1.0), rng.uniform(-3.0, 2.0)])
        size = 10.0 ** rng.uniform(-3.5, -0.5)
        tris.append((c + rng.normal(0.0, size, (3, 3))).tolist())
    tris = np.asarray(tris, np.float32)
    n = len(tris)
    uv = rng.uniform(0.0, 1.0, (n * 3, 2)).astype(np.float32)
    tex = rng.integers(0, 256, (4, 4, 4), dtype=np.uint8)
    return S.Scene(xyz=tris.reshape(-1, 3), uv=uv, idx=np.arange(3 * n, dtype=np.uint32).reshape(n, 3),
                   tri_tex=np.zeros(n, np.uint32), textures=[tex])


def _displays():
    tiny = S.display_tiny()
    paper = S.display_paper()
    return {
        "paper": (paper, None),
        "paper_96": (replace(paper, recon=1), None),
        "tiny": (tiny, None),
        "tiny_cone_0": (replace(tiny, cone_deg=0.0), None),
        # jitter 1 then 0 puts two neighbouring eyes at the same x
        "tiny_equal_eyes": (replace(tiny, recon=3),
                            np.array([0.5, 1.0, 0.0, 0.3, 1.0, 0.0, 0.9, 0.1], np.float32)),
    }


@pytest.mark.parametrize("name", list(_displays()))
def test_closest_and_farthest_eye_match_the_loop_over_every_view(name):
    d, jit = _displays()[name]
    sc = eye_search_scene(d)
    for mi, m in enumerate((np.eye(4, dtype=np.float32), S.model_matrix(3))):
        o = O.render(d, sc, m, splat=False, jitter=jit)
        live = o.tri[:, O.F["live"]] == 1
        assert live.sum() >= 100, "%s: %d live triangles" % (name, live.sum())
        if jit is not None:
            with lfdpr.Renderer(d, sc) as R:
                R.set_view_jitter(jit)
                g = gpu_frame(d, sc, m, panel=False, renderer=R)
        else:
            g = gpu_frame(d, sc, m, panel=False)
        assert g.stats.overflow == 0
        check_sampling(g, o, "%s model %d" % (name, mi))
