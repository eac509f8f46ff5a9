"""The C ABI without a GPU: the library builds for sm_103a, loads, exports
every entry point include/*.h declares, and rejects invalid descriptors on
the host before touching a device."""
import os
import re
from dataclasses import replace

import pytest

from paper_2601_19901_gb300 import build, lfdpr, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return lfdpr.lib()


def declared_entry_points():
    names = set()
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, h)).read(), flags=re.S)
            names |= set(re.findall(r"\b(lfdpr_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_binding_names():
    assert declared_entry_points() == sorted(lfdpr.EXPORTS)


def test_library_exports_every_declared_symbol(L):
    for name in declared_entry_points():
        assert hasattr(L, name), name


def test_version(L):
    assert lfdpr.lfdpr_version() == 1


def _torch_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.parametrize("field,value", [
    ("n_views", 0), ("n_views", 257), ("view_w", 0), ("near_z", 0.0), ("far_z", 0.05),
    ("view_dist", -1.0), ("recon", 4), ("recon", -1), ("crosstalk", 0.5), ("bias_h", 0.0),
    ("lens_pitch_px", 0.0), ("panel_w", 0), ("cone_deg", 180.0)])
def test_invalid_descriptor_rejected_on_host(L, field, value):
    d = replace(scenes.display_tiny(), **{field: value})
    with pytest.raises(lfdpr.LfdprError) as e:
        lfdpr.lfdpr_create_display(lfdpr.desc_of(d))
    assert e.value.status == lfdpr.EINVAL


def test_negative_capacity_rejected(L):
    with pytest.raises(lfdpr.LfdprError) as e:
        lfdpr.lfdpr_create_display(lfdpr.desc_of(scenes.display_tiny(), max_points=-5))
    assert e.value.status == lfdpr.EINVAL


@pytest.mark.skipif(_torch_gpu(), reason="checks the no-device path")
def test_no_device_reports_edevice(L):
    with pytest.raises(lfdpr.LfdprError) as e:
        lfdpr.lfdpr_create_display(lfdpr.desc_of(scenes.display_tiny()))
    assert e.value.status == lfdpr.EDEVICE


def test_null_arguments_rejected(L):
    assert L.lfdpr_create_display(None, None) == lfdpr.EINVAL
    assert L.lfdpr_destroy_display(None) == lfdpr.EINVAL
    assert L.lfdpr_render_frame(None, None, None, None) == lfdpr.EINVAL
    assert L.lfdpr_interleave(None, None, None) == lfdpr.EINVAL
    assert L.lfdpr_destroy_mesh(None) == lfdpr.EINVAL
    assert L.lfdpr_probe_atomic_min(None, 0, None, None, 0, 0, None) == lfdpr.EINVAL
    assert b"null" in L.lfdpr_last_error()
