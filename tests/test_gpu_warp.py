"""The depth-guided warp (lfdpr_warp_views) against a plain numpy restatement
of its definition in include/lfdpr_recon.h, byte for byte: on views and depth
keys LFDPR renders, and on synthetic keys that reach the edge cases (empty
pixels, points that leave the row, coincident input eyes, output eyes
outside the inputs' span, depths far from the focal plane).

The warp's own geometry is pinned too: a fronto-parallel plane at depth z
moves by (1 - D / (D - z)) W / fw pixels per unit of eye motion, so the
warp of renders of it comes much closer to the render from the output eye
than the unshifted blend of the inputs does."""
from dataclasses import replace

import numpy as np
import pytest

from paper_2601_19901_gb300 import lfdpr, scenes as S

pytestmark = pytest.mark.gpu

F32 = np.float32
NO_KEY = np.uint64(0xFFFFFFFFFFFFFFFF)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2601_19901_gb300 import build
    build.build()
    lfdpr.lib()


def _key_t(keys):
    t = (keys >> np.uint64(32)).astype(np.uint32).view(F32)
    with np.errstate(invalid="ignore"):
        ok = (keys != NO_KEY) & (t > 0) & np.isfinite(t)
    return t, ok


def warp_reference(views, keys, in_eyes, out_eyes, ipw):
    """views u8 [nin][H][W][4], keys u64 [nin][H][W], eyes f32 -> u8 [nout][H][W][4]."""
    nin, H, W = keys.shape
    in_eyes = in_eyes.astype(F32)
    ipw = F32(ipw)
    out = np.zeros((len(out_eyes), H, W, 4), np.uint8)
    out[..., 3] = 255
    xs = np.arange(W, dtype=np.int64)
    centre = xs.astype(F32) + F32(0.5)
    rows = np.repeat(np.arange(H), W).reshape(H, W)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        for k, E in enumerate(out_eyes.astype(F32)):
            j0 = 0
            for j in range(nin):
                if in_eyes[j] <= E:
                    j0 = j
            j0 = min(j0, nin - 2)
            e0, e1 = in_eyes[j0], in_eyes[j0 + 1]
            s = (E - e0) / (e1 - e0) if e1 > e0 else F32(0)
            s = F32(min(max(s, F32(0)), F32(1)))
            src_keys = [keys[j0], keys[j0 + 1]]
            src_col = [views[j0, ..., :3].astype(F32), views[j0 + 1, ..., :3].astype(F32)]
            eye = [e0, e1]
            # forward
            win = np.full((H, W), NO_KEY, np.uint64)
            for src in range(2):
                kk = src_keys[src]
                t, ok = _key_t(kk)
                f = F32(1) - F32(1) / t
                X = centre[None, :] + (f * ipw) * (E - eye[src])
                ok &= np.isfinite(X)
                px = np.floor(X)
                ok &= (px >= 0) & (px < W)
                cand = (kk & np.uint64(0xFFFFFFFF00000000)) | np.uint64(src << 16) | xs.astype(np.uint64)[None, :]
                np.minimum.at(win, (rows[ok], px[ok].astype(np.int64)), cand[ok])
            # backward
            has = win != NO_KEY
            t = (win >> np.uint64(32)).astype(np.uint32).view(F32)
            f = F32(1) - F32(1) / t
            vs, wt = [], []
            for src in range(2):
                X = centre[None, :] + (f * ipw) * (eye[src] - E)
                xa = X - F32(0.5)
                fl = np.floor(xa)
                fr = xa - fl
                fn = np.floor(X)
                i0 = np.clip(np.nan_to_num(fl, nan=0.0), 0, W - 1).astype(np.int64)
                i1 = np.clip(np.nan_to_num(fl + F32(1), nan=0.0), 0, W - 1).astype(np.int64)
                n = np.clip(np.nan_to_num(fn, nan=0.0), 0, W - 1).astype(np.int64)
                ca = src_col[src][rows, i0]
                cb = src_col[src][rows, i1]
                vs.append(ca + fr[..., None] * (cb - ca))
                tn, okn = _key_t(src_keys[src][rows, n])
                agree = okn & (np.abs(tn - t) <= F32(0.01) * t)
                wt.append(np.where(agree, (F32(1) - s) if src == 0 else s, F32(0)).astype(F32))
            ws = wt[0] + wt[1]
            blend = (wt[0][..., None] * vs[0] + wt[1][..., None] * vs[1]) * (F32(1) / ws)[..., None]
            ssrc = ((win >> np.uint64(16)) & np.uint64(1)).astype(np.int64)
            sidx = (win & np.uint64(0xFFFF)).astype(np.int64)
            own = np.where((ssrc == 0)[..., None], src_col[0][rows, np.minimum(sidx, W - 1)],
                           src_col[1][rows, np.minimum(sidx, W - 1)])
            hole = (F32(1) - s) * src_col[0] + s * src_col[1]
            v = np.where(has[..., None], np.where((ws > 0)[..., None], blend, own), hole)
            out[k, ..., :3] = np.rint(np.minimum(np.maximum(v, F32(0)), F32(255))).astype(np.uint8)
    return out


def run_gpu(views, keys, in_eyes, out_eyes, ipw):
    import torch
    nin, H, W = keys.shape
    dv = torch.from_numpy(np.ascontiguousarray(views)).cuda()
    dk = torch.from_numpy(np.ascontiguousarray(keys).view(np.int64)).cuda()
    de = torch.from_numpy(in_eyes.astype(F32)).cuda()
    do = torch.from_numpy(out_eyes.astype(F32)).cuda()
    out = torch.zeros((len(out_eyes), H, W, 4), dtype=torch.uint8, device="cuda")
    lfdpr.lfdpr_warp_views(dv.data_ptr(), dk.data_ptr(), de.data_ptr(), nin, do.data_ptr(), len(out_eyes), W, H,
                           ipw, out.data_ptr())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def rendered(d, sc, m):
    from parity import gpu_frame
    g = gpu_frame(d, sc, m, panel=False)
    return g.views, g.keys, g.eyes


def test_warp_of_rendered_views_matches_the_reference():
    d_in = replace(S.display_paper(), n_views=6, view_w=140, view_h=188)
    d_out = replace(d_in, n_views=24)
    sc = S.scene_paper(n_instances=80, res=12, n_textures=4, max_tex=256, min_tex=16, seed=5)
    views, keys, ein = rendered(d_in, sc, S.model_matrix(4))
    eout = np.asarray([F32(v) for v in _eyes(d_out)], F32)
    ipw = F32(d_in.view_w) / F32(d_in.focal_w)
    got = run_gpu(views, keys, ein, eout, ipw)
    ref = warp_reference(views, keys, ein, eout, ipw)
    assert np.array_equal(got, ref), "bytes differ at %d pixels" % int((got != ref).any(-1).sum())
    # enough of every view is covered for the warp to move content
    assert (keys != NO_KEY).mean() > 0.1


def _eyes(d):
    with lfdpr.Renderer(d, S.scene_tiny()) as R:
        return R.eyes()


@pytest.mark.parametrize("case", ["random", "coincident_eyes", "outside_span", "far_and_near", "widest"])
def test_warp_of_synthetic_keys_matches_the_reference(case):
    rng = np.random.default_rng({"random": 1, "coincident_eyes": 2, "outside_span": 3, "far_and_near": 4,
                                 "widest": 5}[case])
    nin, H, W = (5, 7, 173) if case != "widest" else (3, 3, 4032)
    in_eyes = np.sort(rng.uniform(-1.0, 1.0, nin)).astype(F32)
    out_eyes = rng.uniform(-1.0, 1.0, 9).astype(F32)
    if case == "coincident_eyes":
        in_eyes[2] = in_eyes[1]
        out_eyes[:3] = in_eyes[1]
    if case == "outside_span":
        out_eyes[:4] = F32(in_eyes[0] - 0.5), F32(in_eyes[-1] + 0.5), F32(-3.0), F32(3.0)
    lo, hi = (0.05, 3.0) if case != "far_and_near" else (1e-3, 40.0)
    t = rng.uniform(lo, hi, (nin, H, W)).astype(F32)
    if case == "far_and_near":
        t[:, :, ::7] = F32(1.0)      # on the focal plane: no motion
    keys = (t.view(np.uint32).astype(np.uint64) << np.uint64(32)) | rng.integers(0, 1 << 20, (nin, H, W)).astype(np.uint64)
    keys[rng.random((nin, H, W)) < 0.2] = NO_KEY
    views = rng.integers(0, 256, (nin, H, W, 4), dtype=np.uint8)
    ipw = F32(rng.uniform(20.0, 300.0))
    got = run_gpu(views, keys, in_eyes, out_eyes, ipw)
    ref = warp_reference(views, keys, in_eyes, out_eyes, ipw)
    assert np.array_equal(got, ref), "%s: bytes differ at %d pixels" % (case, int((got != ref).any(-1).sum()))


def test_warp_moves_a_plane_by_its_disparity():
    """A textured fronto-parallel plane at depth z: the warp of the input
    renders onto an output eye equals the render from that eye away from the
    plane's edges."""
    d_in = replace(S.display_tiny(), n_views=4, crosstalk=0.0, bias_h=1.0)
    d_out = replace(d_in, n_views=16)
    z = -2.5   # disparity (1 - 4 / 6.5) 128 / 2.4 = 20.5 pixels per unit of eye motion
    tris = np.array([[[-3, -3, z], [3, -3, z], [3, 3, z]], [[-3, -3, z], [3, 3, z], [-3, 3, z]]], np.float32)
    uv = np.array([[0, 0], [1, 0], [1, 1], [0, 0], [1, 1], [0, 1]], np.float32)
    tex = np.repeat(np.repeat(np.random.default_rng(3).integers(0, 256, (16, 16, 4), dtype=np.uint8), 4, 0), 4, 1)
    sc = S.Scene(xyz=tris.reshape(-1, 3), uv=uv, idx=np.arange(6, dtype=np.uint32).reshape(2, 3),
                 tri_tex=np.zeros(2, np.uint32), textures=[tex])
    m = np.eye(4, dtype=np.float32)
    views, keys, ein = rendered(d_in, sc, m)
    vout, _, eout = rendered(d_out, sc, m)
    ipw = F32(d_in.view_w) / F32(d_in.focal_w)
    got = run_gpu(views, keys, ein, eout, ipw)
    # with every key removed the warp is the unshifted blend of the inputs
    naive = run_gpu(views, np.full_like(keys, NO_KEY), ein, eout, ipw)
    # away from the side edges, where the inputs cannot see what an output eye sees
    margin = 12

    def err(a):
        return np.mean(np.abs(a[:, :, margin:-margin, :3].astype(np.int16) -
                              vout[:, :, margin:-margin, :3].astype(np.int16)))
    assert err(got) < 0.3 * err(naive), (err(got), err(naive))


def test_warp_arguments_are_checked():
    import torch
    views = torch.zeros((2, 4, 8, 4), dtype=torch.uint8, device="cuda")
    keys = torch.zeros((2 * 4 * 8 + 1,), dtype=torch.int64, device="cuda")
    eyes = torch.zeros(4, dtype=torch.float32, device="cuda")
    out = torch.zeros((3, 4, 8, 4), dtype=torch.uint8, device="cuda")
    ok = dict(in_views_ptr=views.data_ptr(), in_keys_ptr=keys.data_ptr(), in_eyes_ptr=eyes.data_ptr(), in_count=2,
              out_eyes_ptr=eyes.data_ptr(), out_count=3, view_w=8, view_h=4, pixels_per_unit=50.0,
              out_ptr=out.data_ptr())
    lfdpr.lfdpr_warp_views(**ok)
    torch.cuda.synchronize()
    for bad in (dict(in_count=1), dict(out_count=0), dict(view_w=4033), dict(pixels_per_unit=0.0),
                dict(pixels_per_unit=float("nan")), dict(in_keys_ptr=keys.data_ptr() + 4),
                dict(out_ptr=out.data_ptr() + 2), dict(in_views_ptr=0)):
        with pytest.raises(lfdpr.LfdprError) as e:
            lfdpr.lfdpr_warp_views(**{**ok, **bad})
        assert e.value.status == lfdpr.EINVAL, bad
