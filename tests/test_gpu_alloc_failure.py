"""Allocation failure injected through the library's allocation layer.

Every allocating entry point (display, spatial-supersampling views, mesh,
texture set, textured mesh, batch, network) is run with the hook armed to fail
the k-th allocation from now, for k = 0, 1, 2, ... until the whole sequence
succeeds: the failing call must return ENOMEM, the objects made so far must
be destroyable, and afterwards the library must hold exactly what it held
before. A normal frame then still renders and matches the oracle.
"""
import numpy as np
import pytest

import oracle as O
from paper_2601_19901_gb300 import lfdpr, recon_net as RN, scenes as S

from parity import check_sampling, check_views, gpu_frame

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    from paper_2601_19901_gb300 import build
    build.build()
    lfdpr.lib()
    w, b, nin = RN.load_weights()
    return S.scene_tiny(), (w, b, nin)


def _sequence(sc, net, made):
    """The allocating calls, in order; every object made goes to `made`
    (kind, handle) so that it can be destroyed whatever happens."""
    d = S.display_tiny()
    disp = lfdpr.lfdpr_create_display(lfdpr.desc_of(d))
    made.append(("display", disp))
    lfdpr.lfdpr_set_spatial_supersampling(disp, 1)
    mesh = lfdpr.lfdpr_upload_mesh(disp, sc.xyz, sc.uv, sc.idx, sc.tri_tex, sc.textures, None)
    made.append(("mesh", mesh))
    lfdpr.lfdpr_render_frame(disp, mesh, S.model_matrix(1), None)
    assert lfdpr.lfdpr_frame_stats(disp, None).n_points > 0
    ts = lfdpr.TextureSet(sc.textures)
    made.append(("texset", ts))
    disp2 = lfdpr.lfdpr_create_display(lfdpr.desc_of(d))
    made.append(("display", disp2))
    mesh2 = lfdpr.lfdpr_upload_mesh_textured(disp2, sc.xyz, sc.uv, sc.idx, sc.tri_tex, ts.handle, None)
    made.append(("mesh", mesh2))
    batch = lfdpr.lfdpr_create_batch([disp2], [mesh2])
    made.append(("batch", batch))
    w, b, nin = net
    r = lfdpr.Recon(56, 64, nin, w, b)
    made.append(("recon", r))


def _destroy(made):
    for kind, h in reversed(made):
        if kind == "display":
            lfdpr.lfdpr_destroy_display(h)
        elif kind == "mesh":
            lfdpr.lfdpr_destroy_mesh(h)
        elif kind == "texset":
            h.close()
        elif kind == "batch":
            lfdpr.lfdpr_destroy_batch(h)
        elif kind == "recon":
            h.close()
    made.clear()


def test_every_allocation_failure_returns_enomem_and_leaks_nothing(env):
    import torch
    sc, net = env
    torch.cuda.synchronize()
    live0 = lfdpr.lfdpr_alloc_stats()[:2]
    failures = 0
    for k in range(200):
        made = []
        lfdpr.lfdpr_fault_inject_alloc(k)
        try:
            _sequence(sc, net, made)
            done = True
        except lfdpr.LfdprError as e:
            assert e.status == lfdpr.ENOMEM, (k, e)
            failures += 1
            done = False
        finally:
            lfdpr.lfdpr_fault_inject_alloc(-1)
            torch.cuda.synchronize()
            _destroy(made)
        torch.cuda.synchronize()
        assert lfdpr.lfdpr_alloc_stats()[:2] == live0, "allocations leaked after failing allocation %d" % k
        if done:
            break
    assert done, "the sequence never completed"
    assert failures >= 30     # every allocation of the sequence was made to fail once


def test_a_frame_after_the_failures_matches_the_oracle(env):
    sc, _ = env
    d = S.display_tiny()
    m = S.model_matrix(3)
    g = gpu_frame(d, sc, m)
    o = O.render(d, sc, m)
    check_sampling(g, o, "after faults")
    check_views(g, o, msg="after faults")
