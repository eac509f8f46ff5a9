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


def test_fault_injection_hook_on_the_host(L):
    """The allocation-failure hook is armed and disarmed without a device;
    arguments outside its range are rejected; the accounting reads back."""
    live0, bytes0, total0 = lfdpr.lfdpr_alloc_stats()
    assert live0 >= 0 and bytes0 >= 0 and total0 >= live0
    lfdpr.lfdpr_fault_inject_alloc(0)
    lfdpr.lfdpr_fault_inject_alloc(-1)
    with pytest.raises(lfdpr.LfdprError) as e:
        lfdpr.lfdpr_fault_inject_alloc(-2)
    assert e.value.status == lfdpr.EINVAL
    assert L.lfdpr_alloc_stats(None, None, None) == lfdpr.OK


@pytest.mark.skipif(_torch_gpu(), reason="checks the no-device path")
def test_armed_hook_without_a_device_allocates_nothing(L):
    before = lfdpr.lfdpr_alloc_stats()
    lfdpr.lfdpr_fault_inject_alloc(0)
    try:
        with pytest.raises(lfdpr.LfdprError) as e:
            lfdpr.lfdpr_create_display(lfdpr.desc_of(scenes.display_tiny()))
        assert e.value.status == lfdpr.EDEVICE
        assert lfdpr.lfdpr_alloc_stats() == before
    finally:
        lfdpr.lfdpr_fault_inject_alloc(-1)


def test_regular_build_reports_it_is_not_checked(L):
    if lfdpr.CHECKED:
        pytest.skip("this process loaded the checked build")
    with pytest.raises(lfdpr.LfdprError) as e:
        lfdpr.lfdpr_checked_status()
    assert e.value.status == lfdpr.EINVAL
