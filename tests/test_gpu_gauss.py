"""Sec. 4's supersampling at random angles and Gaussian reconstruction on the
GPU against the oracle.

The eyes move with the caller's jitter, so the whole frame (sampling, splat,
resolve) must still match the oracle run with the same jitter under the
parity tolerances; the Gaussian interleave, given the same views, must
match the oracle bit for bit, with and without crosstalk, over 2N and N
views; jitter 1/2 everywhere must give the default frame exactly.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle as O
from paper_2601_19901_gb300 import lfdpr, scenes as S
from parity import check_sampling, check_views, gpu_frame

pytestmark = pytest.mark.gpu

SIGMA = np.array([2.25 / 4, 2.25 / 4, 2.0 / 4], np.float32)   # dx, dy (view pixels), dphi (views)


def _samples(seed, n=8):
    return (np.random.default_rng(seed).normal(0.0, 1.0, (n, 3)) * SIGMA).astype(np.float32)


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    from paper_2601_19901_gb300 import build
    build.build()
    O.build()
    return S.scene_tiny()


@pytest.mark.parametrize("recon,xtalk", [(2, 0.15), (2, 0.0), (3, 0.15)])
def test_gaussian_frame_matches_oracle(env, recon, xtalk):
    sc = env
    d = replace(S.display_tiny(), recon=recon, crosstalk=xtalk)
    rng = np.random.default_rng(recon * 10 + int(xtalk * 100))
    jit = rng.random(d.n_render_views).astype(np.float32)
    smp = _samples(recon + 7)
    m = S.model_matrix(5)
    with lfdpr.Renderer(d, sc) as R:
        R.set_view_jitter(jit)
        R.set_recon_samples(smp)
        g = gpu_frame(d, sc, m, renderer=R)
    assert np.array_equal(g.eyes, O.eyes(d, jit))
    o = O.render(d, sc, m, jitter=jit, samples=smp)
    check_sampling(g, o, "recon %d" % recon)
    check_views(g, o, msg="recon %d" % recon)
    # interleave of the GPU's own views: bit-exact
    assert np.array_equal(g.panel, O.interleave(d, g.views, jitter=jit, samples=smp))


def test_jitter_one_half_is_the_default_frame(env):
    sc = env
    d = replace(S.display_tiny(), recon=1)
    m = S.model_matrix(9)
    g0 = gpu_frame(d, sc, m)
    with lfdpr.Renderer(d, sc) as R:
        R.set_view_jitter(np.full(d.n_render_views, 0.5, np.float32))
        g1 = gpu_frame(d, sc, m, renderer=R)
    assert np.array_equal(g0.keys, g1.keys) and np.array_equal(g0.panel, g1.panel)


def test_gaussian_arguments_are_checked(env):
    import torch
    sc = env
    d = replace(S.display_tiny(), recon=2)
    with lfdpr.Renderer(d, sc) as R:
        R.render(S.model_matrix(0))
        pan = torch.zeros((d.panel_h, d.panel_w, 4), dtype=torch.uint8, device="cuda")
        with pytest.raises(lfdpr.LfdprError) as e:
            R.interleave(pan.data_ptr())          # no samples yet
        assert e.value.status == lfdpr.EINVAL
        for bad in (np.zeros((0, 3), np.float32), np.zeros((33, 3), np.float32),
                    np.full((2, 3), np.nan, np.float32)):
            with pytest.raises(lfdpr.LfdprError) as e:
                R.set_recon_samples(bad)
            assert e.value.status == lfdpr.EINVAL
        for bad in (np.full(d.n_render_views - 1, 0.5, np.float32), np.full(d.n_render_views, 1.5, np.float32)):
            with pytest.raises(lfdpr.LfdprError) as e:
                R.set_view_jitter(bad)
            assert e.value.status == lfdpr.EINVAL
        torch.cuda.synchronize()


# ---------------------------------------------------------------------------
# 2x and 4x spatial supersampling: views at 2^L times the output size, the
# interleave reading mip level L of each (Sec. 5.1 builds a mipmap of each view)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("recon,level,xtalk", [(0, 1, 0.0), (1, 1, 0.15), (2, 1, 0.15), (3, 2, 0.0), (0, 2, 0.15)])
def test_spatial_supersampling_panel_matches_oracle(env, recon, level, xtalk):
    sc = env
    base = S.display_tiny()
    k = 1 << level
    d = replace(base, view_w=k * base.view_w, view_h=k * base.view_h, recon=recon, crosstalk=xtalk,
                ss_level=level)
    m = S.model_matrix(6)
    jit = smp = None
    with lfdpr.Renderer(d, sc) as R:
        if recon in (2, 3):
            jit = np.random.default_rng(level).random(d.n_render_views).astype(np.float32)
            smp = (np.random.default_rng(level + 3).normal(0.0, 1.0, (8, 3)) * SIGMA).astype(np.float32)
            R.set_view_jitter(jit)
            R.set_recon_samples(smp)
        g = gpu_frame(d, sc, m, renderer=R)
    # the render at the supersampled size (two views against the oracle)
    vl = [0, d.n_render_views - 1]
    o = O.render(d, sc, m, views=vl, panel=False, jitter=jit)
    check_sampling(g, o, "ss %d" % level)
    check_views(g, o, views=vl, msg="ss %d" % level)
    # the view mips and the interleave of the GPU's own views: bit-exact
    assert np.array_equal(g.panel, O.interleave(d, g.views, jitter=jit, samples=smp))


def test_spatial_supersampling_arguments_are_checked(env):
    sc = env
    d = replace(S.display_tiny(), view_w=130, view_h=128)
    with lfdpr.Renderer(d, sc) as R:
        for bad in (-1, 3):
            with pytest.raises(lfdpr.LfdprError) as e:
                lfdpr.lfdpr_set_spatial_supersampling(R.disp, bad)
            assert e.value.status == lfdpr.EINVAL
        lfdpr.lfdpr_set_spatial_supersampling(R.disp, 1)      # 130 x 128: divisible by 2
        with pytest.raises(lfdpr.LfdprError) as e:
            lfdpr.lfdpr_set_spatial_supersampling(R.disp, 2)  # 130 is not divisible by 4
        assert e.value.status == lfdpr.EINVAL
        lfdpr.lfdpr_set_spatial_supersampling(R.disp, 0)
