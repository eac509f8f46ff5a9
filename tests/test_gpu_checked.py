"""The checked build (liblfdpr_checked.so: every frame kernel's global
indices range-checked; an out-of-range index skips its access and is recorded
instead of faulting) on small cases, in a child process that loads it in place
of the regular library: the frames must match the oracle as the regular build
does and no check may have failed."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + "/tests")
from dataclasses import replace
import numpy as np
import torch
from paper_2601_19901_gb300 import build, lfdpr, scenes as S
build.build(checked=True)
assert lfdpr.CHECKED and lfdpr.LIB_PATH.endswith("liblfdpr_checked.so")
import oracle as O
from parity import check_sampling, check_views, gpu_frame
from test_gpu_near import near_scene

lfdpr.lfdpr_checked_status(reset=True)
sc = S.scene_tiny()
cases = [
    (S.display_tiny(), sc, S.model_matrix(2)),
    (replace(S.display_tiny(), recon=1, crosstalk=0.15), sc, S.model_matrix(5)),
    (replace(S.display_tiny(), view_w=256, view_h=256, ss_level=1), sc, S.model_matrix(1)),
    (S.display_tiny(), near_scene(S.display_tiny().view_dist), np.eye(4, dtype=np.float32)),
]
for d, s, m in cases:
    g = gpu_frame(d, s, m)
    o = O.render(d, s, m)
    check_sampling(g, o, "checked")
    check_views(g, o, msg="checked")
    assert np.array_equal(g.panel, O.interleave(d, g.views))
# a Gaussian reconstruction and a batch of two scenes
d = replace(S.display_tiny(), recon=2)
with lfdpr.Renderer(d, sc) as R:
    R.set_recon_samples(np.array([[0.3, -0.2, 0.1], [-0.5, 0.4, -0.6]], np.float32))
    g = gpu_frame(d, sc, S.model_matrix(3), renderer=R)
    assert np.array_equal(g.panel, O.interleave(d, g.views, samples=np.array([[0.3, -0.2, 0.1], [-0.5, 0.4, -0.6]], np.float32)))
ts = lfdpr.TextureSet(sc.textures)
B = lfdpr.Batch([S.display_tiny(), replace(S.display_tiny(), n_views=12)], [sc, S.scene_tiny(seed_mesh=4)], ts)
B.render(np.stack([S.model_matrix(1), S.model_matrix(9)]).astype(np.float32))
torch.cuda.synchronize()
B.close()
ts.close()
site, n = lfdpr.lfdpr_checked_status()
assert (site, n) == (0, 0), (site, n)
print("checked build ok")
'''


def test_checked_build_frames_match_the_oracle_with_no_failed_checks():
    env = dict(os.environ, LFDPR_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked build ok" in r.stdout

