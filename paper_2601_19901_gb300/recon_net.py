"""The learned angular reconstruction network in plain PyTorch.

The architecture is the one include/lfdpr_recon.h fixes: n rendered views in,
the 4n views of the full display after angular supersampling and the
[1/4, 1/2, 1/4] tent reconstruction (Sec. 4) out, as a residual over the
input views warped to the output eyes by their depth keys (the library's
lfdpr_warp_views). This module holds

  * the architecture (UNet) and its export to the library's weight layout;
  * reference_forward: the same forward pass in fp32 that rounds to bf16
    wherever the library's kernels store bf16 (the numerics reference the
    tests hold the library's tensor-core kernels to);
  * the ground-truth views (tent_views) and the error measures (psnr, ssim);
  * train: the offline trainer, which learns from view stacks the library
    itself renders (random procedural scenes and poses).

Inference on the product path runs the library's kernels (lfdpr.Recon);
PyTorch here trains the weights and checks the kernels.
"""
from __future__ import annotations

import math
import os
import time
from dataclasses import replace

import numpy as np

# (input channels, output channels, level) of the 3x3 layers, in order
LAYERS = [(48, 32, 0), (32, 32, 0), (32, 64, 1), (64, 64, 1), (64, 128, 2), (128, 128, 2), (128, 256, 3),
          (256, 256, 3), (384, 128, 2), (128, 128, 2), (192, 64, 1), (64, 64, 1), (96, 32, 0), (32, 32, 0)]
IN_CHANNELS = 48


def padded(h: int, w: int):
    return (h + 7) // 8 * 8, (w + 7) // 8 * 8


def pixels_per_unit(d) -> float:
    """view_w / focal_w as the library's display constants hold it."""
    return float(np.float32(float(d.view_w) / float(d.focal_w)))


def warped_base(views_u8, keys, in_eyes, out_eyes, ppu: float):
    """The residual's base: the library's depth-guided warp of the input views
    [nin][H][W][4] (u8 torch, device) with their depth keys (int64 torch,
    device) from input eyes to output eyes (f32 torch, device) -> u8
    [nout][H][W][4] (torch, device)."""
    torch = _torch()
    from . import lfdpr
    nin, h, w, _ = views_u8.shape
    out = torch.empty((len(out_eyes), h, w, 4), dtype=torch.uint8, device=views_u8.device)
    lfdpr.lfdpr_warp_views(views_u8.data_ptr(), keys.data_ptr(), in_eyes.data_ptr(), nin, out_eyes.data_ptr(),
                           len(out_eyes), w, h, ppu, out.data_ptr(), torch.cuda.current_stream())
    return out


def base_input(warp_u8, hp: int, wp: int):
    """[1, 3 nout, hp, wp] float: the warped views' RGB times 1/255 (the
    library's conversion into the base channels), zero outside the views."""
    torch = _torch()
    n, h, w, _ = warp_u8.shape
    x = torch.zeros((1, 3 * n, hp, wp), dtype=torch.float32, device=warp_u8.device)
    x[0, :, :h, :w] = warp_u8[..., :3].permute(0, 3, 1, 2).reshape(3 * n, h, w).float() * np.float32(1.0 / 255.0)
    return x


def _torch():
    import torch
    return torch


def make_unet(nin: int = 12):
    torch = _torch()
    nn, F = torch.nn, torch.nn.functional

    class UNet(nn.Module):
        def __init__(self):
            super().__init__()
            self.nin = nin
            self.convs = nn.ModuleList([nn.Conv2d(ci, co, 3, padding=1) for ci, co, _ in LAYERS])
            self.out = nn.Conv2d(32, 3 * 4 * nin, 1)

        def features(self, x):
            c, r = self.convs, F.relu

            def up(t):
                return F.interpolate(t, scale_factor=2, mode="nearest")

            e0 = r(c[1](r(c[0](x))))
            e1 = r(c[3](r(c[2](F.avg_pool2d(e0, 2)))))
            e2 = r(c[5](r(c[4](F.avg_pool2d(e1, 2)))))
            b = r(c[7](r(c[6](F.avg_pool2d(e2, 2)))))
            d2 = r(c[9](r(c[8](torch.cat([up(b), e2], 1)))))
            d1 = r(c[11](r(c[10](torch.cat([up(d2), e1], 1)))))
            return r(c[13](r(c[12](torch.cat([up(d1), e0], 1)))))

        def forward(self, x, base):
            return self.out(self.features(x)) + base

    return UNet()


def export(model):
    """(weights bf16 as uint16, biases f32) in the library's blob layout."""
    torch = _torch()
    ws, bs = [], []
    for conv in model.convs:
        ws.append(conv.weight.detach().float().permute(0, 2, 3, 1).reshape(-1))
        bs.append(conv.bias.detach().float().reshape(-1))
    ws.append(model.out.weight.detach().float().reshape(-1))
    bs.append(model.out.bias.detach().float().reshape(-1))
    w = torch.cat(ws).to(torch.bfloat16).cpu().view(torch.int16).numpy().view(np.uint16)
    b = torch.cat(bs).cpu().numpy().astype(np.float32)
    return w, b


def network_input(views_u8, nin: int, hp: int, wp: int):
    """[1, 48, hp, wp] float from nin views [nin][H][W][4] (u8 torch tensor)."""
    torch = _torch()
    n, h, w, _ = views_u8.shape
    x = torch.zeros((1, IN_CHANNELS, hp, wp), dtype=torch.float32, device=views_u8.device)
    x[0, :3 * nin, :h, :w] = views_u8[:nin, :, :, :3].permute(0, 3, 1, 2).reshape(3 * nin, h, w).float() / 255.0
    return x


def tent_views(views_u8):
    """The ground-truth views: 2N rendered views [2N][H][W][4] (u8 torch tensor)
    -> the N reconstructed views [N][H][W][3] u8: [1/4, 1/2, 1/4] over the
    rendered views 2k-1, 2k, 2k+1 that exist, divided by the weights used,
    rounded half to even (Sec. 4's tent, as the interleave applies it)."""
    torch = _torch()
    v = views_u8[..., :3].float()
    n2 = v.shape[0]
    n = n2 // 2
    acc = 0.5 * v[0::2]
    ws = torch.full((n, 1, 1, 1), 0.5, device=v.device)
    acc = acc + 0.25 * v[1::2]
    ws = ws + 0.25
    left = torch.zeros_like(acc)
    left[1:] = 0.25 * v[1:n2 - 1:2]
    acc = acc + left
    wl = torch.full((n, 1, 1, 1), 0.25, device=v.device)
    wl[0] = 0.0
    return torch.round((acc / (ws + wl)).clamp(0, 255)).to(torch.uint8)


def psnr(a_u8, b_u8) -> float:
    torch = _torch()
    mse = torch.mean((a_u8.float() - b_u8.float()) ** 2).item()
    return float("inf") if mse == 0 else 10.0 * math.log10(255.0 * 255.0 / mse)


def ssim(a_u8, b_u8) -> float:
    """Mean SSIM over views and RGB channels (11x11 Gaussian window, sigma
    1.5, K1 = 0.01, K2 = 0.03, dynamic range 255): a, b [N][H][W][3] u8."""
    torch = _torch()
    F = torch.nn.functional
    a = a_u8.float().permute(0, 3, 1, 2).reshape(-1, 1, a_u8.shape[1], a_u8.shape[2])
    b = b_u8.float().permute(0, 3, 1, 2).reshape(-1, 1, b_u8.shape[1], b_u8.shape[2])
    g = torch.exp(-((torch.arange(11, device=a.device) - 5.0) ** 2) / (2 * 1.5 ** 2))
    g = g / g.sum()
    win = (g[:, None] * g[None, :])[None, None]

    def f(t):
        return F.conv2d(t, win)

    c1, c2 = (0.01 * 255) ** 2, (0.03 * 255) ** 2
    ma, mb = f(a), f(b)
    va, vb, cab = f(a * a) - ma * ma, f(b * b) - mb * mb, f(a * b) - ma * mb
    s = ((2 * ma * mb + c1) * (2 * cab + c2)) / ((ma * ma + mb * mb + c1) * (va + vb + c2))
    return float(s.mean().item())


def _bf16(t):
    torch = _torch()
    return t.to(torch.bfloat16).float()


def reference_forward(weights_u16: np.ndarray, biases: np.ndarray, views_u8, nin: int, warp_u8):
    """The library's forward pass in fp32, rounding to bf16 where its kernels
    store bf16: views [nin][H][W][4] u8 and their warp to the output eyes
    warp_u8 [4 nin][H][W][4] u8 (torch) -> [4 nin][H][W][4] u8."""
    torch = _torch()
    F = torch.nn.functional
    dev = views_u8.device
    n, h, w, _ = views_u8.shape
    hp, wp = padded(h, w)
    wt = torch.from_numpy(weights_u16.view(np.int16).copy()).view(torch.bfloat16).float().to(dev)
    bt = torch.from_numpy(biases).to(dev)
    x0 = _bf16(network_input(views_u8, nin, hp, wp))
    wo = bo = 0
    convs = []
    for ci, co, _ in LAYERS:
        k = wt[wo:wo + co * 9 * ci].reshape(co, 3, 3, ci).permute(0, 3, 1, 2).contiguous()
        convs.append((k, bt[bo:bo + co]))
        wo += co * 9 * ci
        bo += co
    w_out = wt[wo:].reshape(3 * 4 * nin, 32)
    b_out = bt[bo:]

    def conv(l, t):
        return _bf16(F.relu(F.conv2d(t, convs[l][0], convs[l][1], padding=1)))

    def pool(t):
        return _bf16(F.avg_pool2d(t, 2))

    def up(t):
        return F.interpolate(t, scale_factor=2, mode="nearest")

    e0 = conv(1, conv(0, x0))
    e1 = conv(3, conv(2, pool(e0)))
    e2 = conv(5, conv(4, pool(e1)))
    b = conv(7, conv(6, pool(e2)))
    d2 = conv(9, conv(8, torch.cat([up(b), e2], 1)))
    d1 = conv(11, conv(10, torch.cat([up(d2), e1], 1)))
    d0 = conv(13, conv(12, torch.cat([up(d1), e0], 1)))
    # the library's output layer: the 1x1 product of d0, plus the base (RGB /
    # 255 in binary32), plus the bias
    base = base_input(warp_u8, hp, wp)
    out = (torch.einsum("ok,bkhw->bohw", w_out, d0) + base) + b_out[None, :, None, None]
    v = torch.round(out.clamp(0.0, 1.0) * 255.0)[0, :, :h, :w]
    rgb = v.reshape(4 * nin, 3, h, w).permute(0, 2, 3, 1).to(torch.uint8)
    res = torch.full((4 * nin, h, w, 4), 255, dtype=torch.uint8, device=dev)
    res[..., :3] = rgb
    return res


# ---------------------------------------------------------------------------
# Offline training on view stacks the library renders
# ---------------------------------------------------------------------------

def train(out_path: str, iters: int = 60000, n_scenes: int = 200, seed: int = 0, lr: float = 1e-3,
          log_every: int = 1000, eval_frames: int = 8, pool: int = 16):
    """Train on `iters` stacks: each is a random training scene at a random
    camera pose (a turn about the vertical, a tilt of up to 15 degrees and a
    shift of up to 0.15), rendered by the library as the n-view input and the
    2x-angular full display whose tent reconstruction is the target. The
    scenes are n_scenes procedurally seeded ones (seeds disjoint from the
    evaluation scene's): `pool` of them are uploaded at a time, and one is
    replaced by the next new scene every iters / n_scenes stacks. Writes the
    weights (npz) and returns the timing."""
    torch = _torch()
    from . import build, lfdpr, scenes as S

    build.build()
    dev = torch.device("cuda")
    rng = np.random.default_rng(seed)
    torch.manual_seed(seed)
    nin = 12
    d_in = replace(S.display_paper(), n_views=nin)
    d_full = S.display_angular_ss()
    H, W = d_in.view_h, d_in.view_w
    hp, wp = padded(H, W)
    t0 = time.time()
    ts = lfdpr.TextureSet(S.textures_paper())
    disp_in = lfdpr.lfdpr_create_display(lfdpr.desc_of(d_in, 1 << 23))
    disp_full = lfdpr.lfdpr_create_display(lfdpr.desc_of(d_full, 1 << 23))
    # the base: the input views warped to the 4n output eyes
    d_out = replace(S.display_paper(), n_views=4 * nin)
    disp_out = lfdpr.lfdpr_create_display(lfdpr.desc_of(d_out))
    in_eyes = torch.from_numpy(lfdpr.lfdpr_view_eyes(disp_in, nin)).to(dev)
    out_eyes = torch.from_numpy(lfdpr.lfdpr_view_eyes(disp_out, 4 * nin)).to(dev)
    lfdpr.lfdpr_destroy_display(disp_out)
    ppu = pixels_per_unit(d_in)
    pool = min(pool, n_scenes)
    scene_no = [0]

    def new_scene():
        k = scene_no[0]
        scene_no[0] += 1
        sc = S.geometry_paper(n_instances=int(rng.integers(80, 320)), seed=1000 + 17 * k)
        return (lfdpr.lfdpr_upload_mesh_textured(disp_in, sc.xyz, sc.uv, sc.idx, sc.tri_tex, ts.handle),
                lfdpr.lfdpr_upload_mesh_textured(disp_full, sc.xyz, sc.uv, sc.idx, sc.tri_tex, ts.handle))

    meshes = [new_scene() for _ in range(pool)]
    replace_every = max(1, iters // max(1, n_scenes - pool))

    def pose():
        yaw = math.radians(float(rng.uniform(0.0, 360.0)))
        tilt = math.radians(float(rng.uniform(-15.0, 15.0)))
        cy, sy, ct, st = math.cos(yaw), math.sin(yaw), math.cos(tilt), math.sin(tilt)
        ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
        rx = np.array([[1, 0, 0], [0, ct, -st], [0, st, ct]])
        m = np.eye(4)
        m[:3, :3] = rx @ ry
        m[:3, 3] = rng.uniform(-0.15, 0.15, 3)
        return m.astype(np.float32)

    model = make_unet(nin).to(dev)
    opt = torch.optim.Adam(model.parameters(), lr=lr)
    sched = torch.optim.lr_scheduler.OneCycleLR(opt, max_lr=lr, total_steps=iters, pct_start=0.05)
    stream = torch.cuda.current_stream()
    setup_s = time.time() - t0
    t0 = time.time()
    hist = []

    def stack(m_in, m_full, model_matrix):
        lfdpr.lfdpr_render_frame(disp_in, m_in, model_matrix, stream)
        lfdpr.lfdpr_render_frame(disp_full, m_full, model_matrix, stream)
        bi = lfdpr.lfdpr_get_buffers(disp_in, m_in)
        bf = lfdpr.lfdpr_get_buffers(disp_full, m_full)
        v_in = lfdpr.device_view(bi.views, (nin, H, W, 4), np.uint8)
        k_in = lfdpr.device_view(bi.keys, (nin, H, W), np.uint64)
        v_full = lfdpr.device_view(bf.views, (2 * d_full.n_views, H, W, 4), np.uint8)
        return v_in, k_in, v_full

    for it in range(iters):
        if it > 0 and it % replace_every == 0 and scene_no[0] < n_scenes:
            slot = (scene_no[0] - pool) % pool
            torch.cuda.synchronize()
            lfdpr.lfdpr_destroy_mesh(meshes[slot][0])
            lfdpr.lfdpr_destroy_mesh(meshes[slot][1])
            meshes[slot] = new_scene()
        k = int(rng.integers(pool))
        mm = pose()
        v_in, k_in, v_full = stack(meshes[k][0], meshes[k][1], mm)
        x = network_input(v_in, nin, hp, wp)
        base = base_input(warped_base(v_in, k_in, in_eyes, out_eyes, ppu), hp, wp)
        tgt = tent_views(v_full).permute(0, 3, 1, 2).reshape(1, -1, H, W).float() / 255.0
        with torch.autocast("cuda", dtype=torch.bfloat16):
            pred = model(x, base)
        loss = torch.mean((pred.float()[:, :, :H, :W] - tgt) ** 2)
        opt.zero_grad(set_to_none=True)
        loss.backward()
        opt.step()
        sched.step()
        if (it + 1) % log_every == 0 or it == 0:
            l = loss.item()
            hist.append((it + 1, l))
            print("iter %d loss %.3e (%.1f dB) %.1f s" % (it + 1, l, 10 * math.log10(1.0 / max(l, 1e-12)),
                                                           time.time() - t0), flush=True)
    train_s = time.time() - t0
    w, b = export(model)
    np.savez(out_path, weights=w, biases=b, in_views=np.int32(nin), view_w=np.int32(W), view_h=np.int32(H),
             iters=np.int32(iters), seed=np.int32(seed), scenes=np.int32(scene_no[0]),
             loss_history=np.array(hist, np.float64))
    for m_in, m_full in meshes:
        lfdpr.lfdpr_destroy_mesh(m_in)
        lfdpr.lfdpr_destroy_mesh(m_full)
    lfdpr.lfdpr_destroy_display(disp_in)
    lfdpr.lfdpr_destroy_display(disp_full)
    ts.close()
    return {"setup_s": setup_s, "train_s": train_s, "iters": iters, "scenes": scene_no[0]}


def evaluate(weights: np.ndarray, biases: np.ndarray, nin: int = 12, frames=range(0, 120, 15), stream=None):
    """PSNR and SSIM per frame of the learned path against the plain full
    render on the paper-shaped scene (orbit frames, 3 degrees each): the
    library renders the n-view display and the 2x-angular full display, its
    kernels run the network into the 4n-view display, and the prediction is
    compared with the full render's tent reconstruction; the warped base
    alone is scored too."""
    torch = _torch()
    from . import lfdpr, scenes as S
    sc = S.scene_paper()
    d_in = replace(S.display_paper(), n_views=nin)
    d_full = S.display_angular_ss()
    d_out = replace(S.display_paper(), n_views=4 * nin, crosstalk=d_full.crosstalk)
    H, W = d_in.view_h, d_in.view_w
    ts = lfdpr.TextureSet(sc.textures)
    disps = [lfdpr.lfdpr_create_display(lfdpr.desc_of(d)) for d in (d_in, d_full, d_out)]
    meshes = [lfdpr.lfdpr_upload_mesh_textured(disps[k], sc.xyz, sc.uv, sc.idx, sc.tri_tex, ts.handle)
              for k in range(2)]
    in_eyes = torch.from_numpy(lfdpr.lfdpr_view_eyes(disps[0], nin)).cuda()
    out_eyes = torch.from_numpy(lfdpr.lfdpr_view_eyes(disps[2], 4 * nin)).cuda()
    res = []
    with lfdpr.Recon(W, H, nin, weights, biases) as R:
        for f in frames:
            m = S.model_matrix(f)
            lfdpr.lfdpr_render_frame(disps[0], meshes[0], m, stream)
            lfdpr.lfdpr_render_frame(disps[1], meshes[1], m, stream)
            R.run(disps[0], disps[2], stream)
            bf = lfdpr.lfdpr_get_buffers(disps[1], meshes[1])
            truth = tent_views(lfdpr.device_view(bf.views, (2 * d_full.n_views, H, W, 4), np.uint8))
            bo = lfdpr.lfdpr_get_buffers(disps[2], meshes[0])
            pred = lfdpr.device_view(bo.views, (4 * nin, H, W, 4), np.uint8)[..., :3]
            bi = lfdpr.lfdpr_get_buffers(disps[0], meshes[0])
            inp = lfdpr.device_view(bi.views, (nin, H, W, 4), np.uint8)
            keys = lfdpr.device_view(bi.keys, (nin, H, W), np.uint64)
            base = warped_base(inp, keys, in_eyes, out_eyes, pixels_per_unit(d_in))[..., :3]
            res.append({"frame": int(f), "psnr": psnr(pred, truth), "ssim": ssim(pred, truth),
                        "psnr_warp": psnr(base, truth)})
    for m_ in meshes:
        lfdpr.lfdpr_destroy_mesh(m_)
    for d_ in disps:
        lfdpr.lfdpr_destroy_display(d_)
    ts.close()
    return res


def load_weights(path: str = None):
    """(weights, biases, in_views) of the shipped (or given) weights file."""
    path = path or os.path.join(os.path.dirname(os.path.abspath(__file__)), "recon_weights.npz")
    z = np.load(path)
    return z["weights"], z["biases"], int(z["in_views"])


if __name__ == "__main__":
    import argparse
    p = argparse.ArgumentParser(description="train the angular reconstruction network")
    p.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "recon_weights.npz"))
    p.add_argument("--iters", type=int, default=60000)
    p.add_argument("--scenes", type=int, default=200)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--lr", type=float, default=1e-3)
    p.add_argument("--eval", action="store_true", help="evaluate the written weights on the paper-shaped scene")
    a = p.parse_args()
    import torch
    torch.backends.cudnn.benchmark = True
    print(train(a.out, a.iters, a.scenes, a.seed, a.lr), flush=True)
    if a.eval:
        w, b, nin = load_weights(a.out)
        for r in evaluate(w, b, nin):
            print(r, flush=True)
