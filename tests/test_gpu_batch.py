"""Batched frames against the oracle and against single frames.

A batch renders several scenes, each on its own display (different view
counts, view sizes, panels, angular supersampling), from one texture set, as
one replayed CUDA graph with a persistent splat over all scenes. Every scene
must match the CPU oracle under the parity tolerances (point sets
bit-exact, >= 99.9 % same winning ids, colour within 1/255, PSNR >= 50 dB,
the interleave bit-exact on the same views); and its keys, views and panel
must be bit-identical to rendering that scene alone with lfdpr_render_frame +
lfdpr_interleave, on consecutive frames (the graph replayed with new model
matrices), under other configurations, and after autotuning.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle as O
from paper_2601_19901_gb300 import lfdpr, scenes as S

from parity import GpuFrame, check_sampling, check_views, psnr

pytestmark = pytest.mark.gpu


def _displays():
    d1 = S.display_tiny()
    d2 = replace(S.display_tiny(), n_views=16, view_w=96, view_h=128, panel_w=384, panel_h=256)
    d3 = replace(S.display_tiny(), n_views=12, recon=1, crosstalk=0.15, panel_w=256, panel_h=320)
    return [d1, d2, d3]


def _scenes():
    # same texture (seed_tex) everywhere, different meshes
    return [S.scene_tiny(seed_mesh=1), S.scene_tiny(seed_mesh=5), S.scene_tiny(seed_mesh=9)]


def _single(display, scene, model):
    import torch
    dev = torch.device("cuda")
    with lfdpr.Renderer(display, scene) as R:
        R.render(model)
        st = R.stats()
        b = R.buffers()
        nr, h, w = b.n_render_views, b.view_h, b.view_w
        keys = lfdpr.device_to_numpy(b.keys, (nr, h, w), np.uint64)
        views = lfdpr.device_to_numpy(b.views, (nr, h, w, 4), np.uint8)
        panel = torch.zeros((display.panel_h, display.panel_w, 4), dtype=torch.uint8, device=dev)
        R.interleave(panel.data_ptr())
        torch.cuda.synchronize()
        return int(st.n_points), keys, views, panel.cpu().numpy()


def _batched(B, i, display):
    import torch
    torch.cuda.synchronize()
    st = B.stats(i)
    b = B.buffers(i)
    nr, h, w = b.n_render_views, b.view_h, b.view_w
    keys = lfdpr.device_to_numpy(b.keys, (nr, h, w), np.uint64)
    views = lfdpr.device_to_numpy(b.views, (nr, h, w, 4), np.uint8)
    panel = lfdpr.device_to_numpy(B.panel(i), (display.panel_h, display.panel_w, 4), np.uint8)
    return int(st.n_points), keys, views, panel


@pytest.fixture(scope="module")
def batch():
    import torch
    assert torch.cuda.is_available()
    from paper_2601_19901_gb300 import build
    build.build()
    ds, scs = _displays(), _scenes()
    ts = lfdpr.TextureSet(scs[0].textures)
    B = lfdpr.Batch(ds, scs, ts)
    yield ds, scs, B
    B.close()
    ts.close()


def _models(frame):
    return np.stack([S.model_matrix(frame + 4 * k) for k in range(3)]).astype(np.float32)


def _check_all(ds, scs, B, frame):
    models = _models(frame)
    B.render(models)
    for i in range(3):
        got = _batched(B, i, ds[i])
        ref = _single(ds[i], scs[i], models[i])
        assert got[0] == ref[0] and got[0] > 0
        assert np.array_equal(got[1], ref[1]), "keys of scene %d" % i
        assert np.array_equal(got[2], ref[2]), "views of scene %d" % i
        assert np.array_equal(got[3], ref[3]), "panel of scene %d" % i


def _batched_frame(B, i, display, scene) -> GpuFrame:
    """Scene i of the last batch as the parity helpers' frame."""
    import torch
    torch.cuda.synchronize()
    st = B.stats(i)
    b = B.buffers(i)
    nr, h, w = b.n_render_views, b.view_h, b.view_w
    T = scene.n_tris
    n = int(st.n_points)
    rd = lfdpr.device_to_numpy
    return GpuFrame(stats=st, counts=rd(b.counts, (T,), np.uint32), offsets=rd(b.offsets, (T,), np.uint32),
                    tri=rd(b.tri, (T, lfdpr.TRI_FLOATS), np.float32), points=rd(b.points, (n, 4), np.uint32),
                    keys=rd(b.keys, (nr, h, w), np.uint64), views=rd(b.views, (nr, h, w, 4), np.uint8),
                    panel=rd(B.panel(i), (display.panel_h, display.panel_w, 4), np.uint8),
                    eyes=lfdpr.lfdpr_view_eyes(B.disps[i], nr))


@pytest.mark.parametrize("frame", [3, 11])
def test_batch_scenes_match_the_oracle(batch, frame):
    ds, scs, B = batch
    models = _models(frame)
    B.render(models)
    for i in range(3):
        g = _batched_frame(B, i, ds[i], scs[i])
        o = O.render(ds[i], scs[i], models[i])
        assert g.stats.overflow == 0 and g.stats.n_points == len(o.points) > 0
        assert np.array_equal(g.eyes.view(np.uint32), O.eyes(ds[i]).view(np.uint32))
        check_sampling(g, o, "batch scene %d" % i)
        check_views(g, o, msg="batch scene %d" % i)
        assert np.array_equal(g.panel, O.interleave(ds[i], g.views)), "panel of scene %d" % i
        assert psnr(g.panel, o.panel) >= 50.0


def test_batch_scene_latencies(batch):
    ds, scs, B = batch
    B.render(_models(4))
    ms = B.scene_ms()
    assert ms.shape == (3,) and np.all(ms > 0.0) and np.all(np.isfinite(ms))
    # scenes on one branch finish in order
    B.set_config(1, 4, 2)
    B.render(_models(4))
    ms = B.scene_ms()
    assert np.all(np.diff(ms) >= 0.0)


def test_batch_matches_single_frames_on_consecutive_frames(batch):
    ds, scs, B = batch
    _check_all(ds, scs, B, 3)
    _check_all(ds, scs, B, 11)   # replay with new model matrices


def test_batch_matches_under_other_configurations(batch):
    ds, scs, B = batch
    for cfg in [(1, 4, 2), (3, 2, 1), (2, 16, 8)]:
        B.set_config(*cfg)
        assert B.config().as_tuple() == cfg
        _check_all(ds, scs, B, 7)


def test_autotune_keeps_a_candidate_and_the_results(batch):
    ds, scs, B = batch
    cfg, ms = B.autotune(_models(2), reps=1)
    assert ms > 0.0 and 1 <= cfg.branches <= 3 and cfg.splat_slots in (1, 2, 3, 4, 6, 8)
    assert B.config().as_tuple() == cfg.as_tuple()
    table = B.autotune_table()
    assert len(table) >= 2 and all(t[3] > 0.0 for t in table)
    assert min(t[3] for t in table) == pytest.approx(ms)
    assert cfg.as_tuple() in [t[:3] for t in table]
    _check_all(ds, scs, B, 5)


def test_batch_rejects_bad_arguments(batch):
    ds, scs, B = batch
    with pytest.raises(lfdpr.LfdprError) as e:
        lfdpr.lfdpr_create_batch([B.disps[0], B.disps[0]], [B.meshes[0], B.meshes[0]])
    assert e.value.status == lfdpr.EINVAL
    with pytest.raises(lfdpr.LfdprError) as e:
        lfdpr.lfdpr_create_batch([B.disps[0]], [B.meshes[1]])
    assert e.value.status == lfdpr.EINVAL
    for bad in [(0, 4, 3), (2, 0, 3), (2, 4, 5)]:
        with pytest.raises(lfdpr.LfdprError) as e:
            B.set_config(*bad)
        assert e.value.status == lfdpr.EINVAL
    bad_models = _models(1)
    bad_models[1, 0, 0] = np.nan
    with pytest.raises(lfdpr.LfdprError) as e:
        B.render(bad_models)
    assert e.value.status == lfdpr.EINVAL
