"""Whole frames on seeded random displays and scenes against the oracle.

Each case draws a display (1 to 13 views, odd view and panel sizes, cones
from 0 to 55 degrees, sampling biases, lens pitch, slant and phase, tent or
Gaussian reconstruction with random eye jitter, crosstalk, spatial
supersampling) and a scene (up to 400 triangles of sizes over two decades,
some degenerate, some reaching the eyes' plane, one to three textures of
power-of-two sizes from 1 to 64 texels a side, wrapped UVs), under a random
rigid model transform. Sampling must be bit-exact, views within the
parity tolerances, and the panel bit-exact against the oracle's
interleave of the GPU's views.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2601_19901_gb300 import lfdpr, scenes as S

from parity import check_sampling, check_views, gpu_frame

pytestmark = pytest.mark.gpu

N_CASES = 64
SIGMA = np.array([2.25 / 4, 2.25 / 4, 2.0 / 4], np.float32)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2601_19901_gb300 import build
    build.build()
    lfdpr.lib()
    O.build()


def _rotation(rng, max_deg):
    axis = rng.normal(0.0, 1.0, 3)
    axis /= np.linalg.norm(axis)
    a = math.radians(rng.uniform(-max_deg, max_deg))
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(a) * K + (1 - math.cos(a)) * K @ K


def random_case(seed: int):
    rng = np.random.default_rng(7000 + seed)
    n_views = int(rng.choice([1, 2, 3, 5, 8, 13]))
    recon = int(rng.choice([0, 0, 1, 2, 3]))
    W, H = int(rng.integers(8, 97)), int(rng.integers(8, 97))
    ss = 0
    if rng.random() < 0.3:
        W, H, ss = 2 * max(W // 2, 8), 2 * max(H // 2, 8), 1
    D = float(rng.choice([2.0, 4.0, 7.5]))
    fh = float(rng.uniform(1.0, 3.0))
    fw = fh * W / H * float(rng.choice([1.0, 1.0, 0.8, 1.25]))
    bh, bv = [(1.0, 1.0), (4.0, 1.0), (1.0, 2.0), (1.5, 1.5)][int(rng.integers(0, 4))]
    d = S.Display(n_views=n_views, view_w=W, view_h=H, cone_deg=float(rng.choice([0.0, 12.0, 30.0, 55.0])),
                  view_dist=D, focal_w=fw, focal_h=fh, near_z=float(rng.choice([0.05, 0.1, 0.3])),
                  far_z=float(rng.choice([20.0, 100.0])), bias_h=bh, bias_v=bv,
                  panel_w=int(rng.integers(16, 300)), panel_h=int(rng.integers(16, 200)),
                  lens_pitch_px=float(rng.uniform(2.5, 9.5)), slant=float(rng.uniform(-0.3, 0.4)),
                  phase_offset=float(rng.uniform(0.0, 1.0)), recon=recon,
                  crosstalk=float(rng.choice([0.0, 0.0, 0.1, 0.2])), ss_level=ss)
    # the scene: triangles in front of the display, a few reaching the eyes' plane
    T = int(rng.integers(1, 401))
    c = rng.uniform(-1.0, 1.0, (T, 3)) * np.array([0.6 * fw, 0.6 * fh, 1.2]) + np.array([0.0, 0.0, -0.2])
    size = 10.0 ** rng.uniform(-2.5, -0.4, T)
    tris = c[:, None, :] + rng.normal(0.0, 1.0, (T, 3, 3)) * size[:, None, None]
    k = T // 16
    tris[:k, 1] = tris[:k, 0]                                   # zero area
    if T > 8:
        tris[-2:, :, 2] = D - rng.uniform(-0.05, 0.4, (2, 3))    # near or past the eyes' plane
        tris[-2:, :, :2] *= 0.2
    tris = tris.astype(np.float32)
    n_tex = int(rng.integers(1, 4))
    textures = [rng.integers(0, 256, (1 << int(rng.integers(0, 7)), 1 << int(rng.integers(0, 7)), 4),
                             dtype=np.uint8) for _ in range(n_tex)]
    sc = S.Scene(xyz=tris.reshape(-1, 3), uv=rng.uniform(-2.0, 3.0, (3 * T, 2)).astype(np.float32),
                 idx=np.arange(3 * T, dtype=np.uint32).reshape(T, 3),
                 tri_tex=rng.integers(0, n_tex, T).astype(np.uint32), textures=textures)
    m = np.eye(4)
    m[:3, :3] = _rotation(rng, 25.0)
    m[:3, 3] = rng.uniform(-0.2, 0.2, 3)
    m = m.astype(np.float32)
    jit = smp = None
    if recon in (2, 3):
        jit = rng.random(d.n_render_views).astype(np.float32)
        smp = (rng.normal(0.0, 1.0, (int(rng.integers(1, 9)), 3)) * SIGMA).astype(np.float32)
    return d, sc, m, jit, smp


@pytest.mark.parametrize("seed", range(N_CASES))
def test_random_frame_matches_the_oracle(seed):
    d, sc, m, jit, smp = random_case(seed)
    o = O.render(d, sc, m, jitter=jit, samples=smp)
    need = len(o.points)
    with lfdpr.Renderer(d, sc, max_points=max(need, 1) + 64) as R:
        if jit is not None:
            R.set_view_jitter(jit)
            R.set_recon_samples(smp)
        g = gpu_frame(d, sc, m, renderer=R)
    assert g.stats.overflow == 0 and g.stats.n_points == need
    msg = "case %d (%d views, %dx%d, recon %d, ss %d)" % (seed, d.n_views, d.view_w, d.view_h, d.recon, d.ss_level)
    check_sampling(g, o, msg)
    check_views(g, o, msg=msg)
    assert np.array_equal(g.panel, O.interleave(d, g.views, jitter=jit, samples=smp)), msg + " panel"
