"""The learned angular reconstruction's kernels against plain PyTorch fp32.

The library's 3x3 tensor-core convolution (bf16 operands, fp32 accumulation,
bf16 result) must match an fp32 convolution of the same bf16 values to one
bf16 rounding; the whole forward pass (pooling, upsampling, concatenation,
the 1x1 output layer and the angular base) must match the fp32 reference
that rounds where the kernels store bf16, on the u8 output views, apart from
rare one-step roundings that propagate.
"""
from dataclasses import replace

import numpy as np
import pytest

from paper_2601_19901_gb300 import lfdpr, recon_net as RN, scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    torch.backends.cudnn.allow_tf32 = False        # fp32 references stay fp32
    torch.backends.cuda.matmul.allow_tf32 = False
    from paper_2601_19901_gb300 import build
    build.build()
    return torch


@pytest.mark.parametrize("cin,cout,h,w", [(48, 32, 20, 45), (64, 64, 17, 70), (384, 128, 9, 13),
                                          (32, 256, 8, 8), (96, 32, 33, 31), (16, 32, 1, 1),
                                          (32, 32, 70, 300), (256, 256, 12, 20)])
def test_conv3x3_matches_fp32_reference(torch, cin, cout, h, w):
    g = torch.Generator(device="cpu").manual_seed(cin * 1000 + cout + h)
    x = torch.randn((h, w, cin), generator=g).to(torch.bfloat16).cuda()
    wt = (torch.randn((cout, 3, 3, cin), generator=g) * (2.0 / (9 * cin)) ** 0.5).to(torch.bfloat16).cuda()
    b = (torch.randn((cout,), generator=g) * 0.1).float().cuda()
    out = torch.full((h, w, cout), 7.0, dtype=torch.bfloat16, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    lfdpr.lfdpr_conv3x3_bf16(x.data_ptr(), h, w, cin, wt.data_ptr(), b.data_ptr(), out.data_ptr(), cout,
                             status.data_ptr())
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = torch.nn.functional.conv2d(x.float().permute(2, 0, 1)[None], wt.float().permute(0, 3, 1, 2), b,
                                     padding=1)[0].permute(1, 2, 0).relu()
    # one bf16 rounding of the result, plus the fp32 summation-order bound of
    # a dot product of K = 9 cin terms: K 2^-24 sum |x w|
    mag = torch.nn.functional.conv2d(x.float().abs().permute(2, 0, 1)[None], wt.float().abs().permute(0, 3, 1, 2),
                                     b.abs(), padding=1)[0].permute(1, 2, 0)
    got = out.float()
    tol = ref.abs() * 2.0 ** -8 + mag * (9 * cin) * 2.0 ** -24
    err = (got - ref).abs()
    assert torch.all(err <= tol), float((err - tol).max())


def test_conv3x3_rejects_unsupported_channels(torch):
    for cin, cout in ((40, 32), (32, 48), (528, 32), (32, 288)):
        with pytest.raises(lfdpr.LfdprError) as e:
            lfdpr.lfdpr_conv3x3_bf16(256, 8, 8, cin, 256, 256, 256, cout, 256)
        assert e.value.status == lfdpr.EINVAL


def _random_net(torch, seed):
    torch.manual_seed(seed)
    model = RN.make_unet(12)
    return RN.export(model)


@pytest.mark.parametrize("h,w", [(40, 44), (64, 56), (560, 420)])
def test_forward_matches_reference(torch, h, w):
    """The whole forward pass, with its warped base (the warp itself is held
    byte-exact to its own restatement in test_gpu_warp.py), against the fp32
    reference that rounds where the kernels store bf16."""
    wts, bs = _random_net(torch, 7)
    g = torch.Generator(device="cpu").manual_seed(h * w)
    # smooth-ish random views so the network sees image-like inputs
    base = torch.rand((12, h // 4 + 1, w // 4 + 1, 4), generator=g)
    views = torch.nn.functional.interpolate(base.permute(0, 3, 1, 2), size=(h, w), mode="bilinear",
                                            align_corners=False).permute(0, 2, 3, 1)
    views = (views * 255).round().to(torch.uint8).contiguous().cuda()
    # depth keys: ray parameters around the focal plane, a fifth of the pixels empty
    t = (0.6 + 0.8 * torch.rand((12, h, w), generator=g)).numpy().astype(np.float32)
    keys = (t.view(np.uint32).astype(np.uint64) << np.uint64(32))
    keys[np.random.default_rng(h).random((12, h, w)) < 0.2] = np.uint64(0xFFFFFFFFFFFFFFFF)
    keys = torch.from_numpy(keys.view(np.int64)).cuda()
    in_eyes = torch.linspace(-1.4, 1.4, 12, dtype=torch.float32).cuda()
    out_eyes = torch.linspace(-1.45, 1.45, 48, dtype=torch.float32).cuda()
    ppu = 100.0
    out = torch.zeros((48, h, w, 4), dtype=torch.uint8, device="cuda")
    with lfdpr.Recon(w, h, 12, wts, bs) as R:
        R.forward(views.data_ptr(), keys.data_ptr(), in_eyes.data_ptr(), out_eyes.data_ptr(), ppu, out.data_ptr())
        torch.cuda.synchronize()
        assert R.status() == 0
    warp = RN.warped_base(views, keys, in_eyes, out_eyes, ppu)
    ref = RN.reference_forward(wts, bs, views, 12, warp)
    d = (out.int() - ref.int()).abs()
    assert torch.all(out[..., 3] == 255)
    assert int(d.max()) <= 3
    assert float((d > 1).float().mean()) < 1e-3
    assert float(d.float().mean()) < 0.05


def test_counts_and_display_checks(torch):
    assert lfdpr.lfdpr_recon_weight_count(12) == sum(co * 9 * ci for ci, co, _ in RN.LAYERS) + 144 * 32
    assert lfdpr.lfdpr_recon_bias_count(12) == sum(co for _, co, _ in RN.LAYERS) + 144
    wts, bs = _random_net(torch, 3)
    with pytest.raises(lfdpr.LfdprError) as e:
        lfdpr.lfdpr_create_recon(64, 64, 12, wts[:-1], bs)
    assert e.value.status == lfdpr.EINVAL
    d_in = replace(S.display_tiny(), n_views=4)
    d_out = replace(S.display_tiny(), n_views=16)
    with lfdpr.Recon(d_in.view_w, d_in.view_h, 4, *_net4(torch)) as R:
        src = lfdpr.lfdpr_create_display(lfdpr.desc_of(d_in))
        dst = lfdpr.lfdpr_create_display(lfdpr.desc_of(d_out))
        try:
            R.run(src, dst)   # shapes agree
            with pytest.raises(lfdpr.LfdprError) as e:
                R.run(dst, src)
            assert e.value.status == lfdpr.EINVAL
            torch.cuda.synchronize()
        finally:
            lfdpr.lfdpr_destroy_display(src)
            lfdpr.lfdpr_destroy_display(dst)


def _net4(torch):
    torch.manual_seed(5)
    return RN.export(RN.make_unet(4))
