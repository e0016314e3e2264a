"""C-ABI checks that need no GPU: the library builds and loads, exports every
function `include/gpss.h` declares, and rejects invalid arguments on the host
before any CUDA work is queued."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2603_00280_gb300 import gpss

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gpss.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gpss_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("gpss_scene_create", "gpss_render", "gpss_render_adjoint", "gpss_batch_create",
                 "gpss_eval_sigma_t", "gpss_eval_phase", "gpss_eval_ndf", "gpss_eval_transmittance"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = gpss.load()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert L.gpss_version() >> 16 == 1


def _obj(nx=3, ny=3, nz=3, var=0.01, channels=1, l=0.1, alb=0.5):
    mean = np.zeros((nz, ny, nx), np.float32)
    v = np.full((nz, ny, nx), var, np.float32)
    a = np.full((channels, nz, ny, nx), alb, np.float32)
    return {"mean": mean, "var": v, "albedo": a, "bbox_min": (0, 0, 0), "bbox_max": (1, 1, 1), "length_scale": l}


@pytest.mark.parametrize("bad", [
    dict(nx=1), dict(channels=2), dict(l=0.0), dict(l=-1.0),
])
def test_scene_create_rejects_bad_descriptors(bad):
    kw = dict(bad)
    with pytest.raises(gpss.GpssError) as e:
        gpss.Scene({"objects": [_obj(**kw)], "light": {"type": "sky"}}, stream=0)
    assert e.value.status == 1


@pytest.mark.parametrize("extra", [
    dict(length_scale_b=0.2),                    # l_b != l_t needs a tangent field
    dict(length_scale_n=-0.1),                   # l_n must be 0 or > 0
    dict(length_scale_b=float("nan")),
    dict(ndf="ggx", length_scale_n=0.2),         # height fields take an isotropic kernel
    dict(ndf="beckmann", tangent=np.zeros((3, 3, 3, 3), np.float32)),
])
def test_scene_create_rejects_bad_kernels(extra):
    o = dict(_obj(), **extra)
    with pytest.raises(gpss.GpssError) as e:
        gpss.Scene({"objects": [o], "light": {"type": "sky"}}, stream=0)
    assert e.value.status == 1
    assert b"object 0" in gpss.load().gpss_last_error()


def test_object_descriptor_layout_matches_the_header():
    """The binding's ctypes mirror of gpss_object_desc has the header's fields in order."""
    text = open(HEADER).read()
    body = text[text.index("typedef struct {\n  int nx, ny, nz;"):]
    body = body[:body.index("} gpss_object_desc;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"\b(\w+)(?:\[\d\])?\s*[,;]", body)
    assert [f for f, _ in gpss.ObjectDesc._fields_] == names


def test_scene_create_rejects_bad_counts_and_boxes():
    L = gpss.load()
    h = ctypes.c_void_p()
    descs = (gpss.ObjectDesc * 1)()
    assert L.gpss_scene_create(descs, 0, None, 0, None, ctypes.byref(h)) == 1
    assert L.gpss_scene_create(descs, 5, None, 0, None, ctypes.byref(h)) == 1
    o = _obj()
    o["bbox_max"] = (1, 0, 1)  # empty box
    with pytest.raises(gpss.GpssError):
        gpss.Scene({"objects": [o]}, stream=0)
    assert L.gpss_scene_create(None, 1, None, 0, None, ctypes.byref(h)) == 1


def test_calls_reject_null_and_invalid_arguments():
    L = gpss.load()
    cam = gpss.camera_desc({"type": "perspective", "eye": (0, -2, 0), "look_at": (0, 0, 0), "up": (0, 0, 1),
                            "width": 4, "height": 4})
    opts = gpss.render_opts({"spp": 1, "max_bounces": 1})
    assert L.gpss_render(None, ctypes.byref(cam), ctypes.byref(opts), None, None, None, None) == 1
    assert L.gpss_eval_ndf(-1, None, 1.0, 1.0, 1.0, 1.0, None, None) == 1
    buf = ctypes.c_void_p(1)
    assert L.gpss_eval_ndf(4, buf, 1.0, 0.0, 1.0, 1.0, buf, None) == 1      # zero roughness
    assert L.gpss_eval_ndf(4, buf, -1.0, 1.0, 1.0, 1.0, buf, None) == 1     # negative G
    assert L.gpss_eval_ndf(0, buf, 1.0, 1.0, 1.0, 1.0, buf, None) == 0      # empty input is a no-op
    assert L.gpss_philox4x32_10(1, None, None, None, None) == 1
    assert L.gpss_scene_destroy(None) == 1
    assert L.gpss_scene_set_surface_flight(None, 1) == 1
    assert L.gpss_scene_set_local_majorant(None, 4.0) == 1
    assert L.gpss_scene_set_object_grids(None, 1) == 1
    assert L.gpss_eval_local_piece(None, 1, buf, buf, buf, buf, buf, buf, buf, buf, buf, buf, None) == 1
    assert L.gpss_render_adjoint(None, ctypes.byref(cam), ctypes.byref(opts), buf, None, None, None, None, None,
                                 None, None) == 1
    assert L.gpss_last_error() != b""


def test_option_validation_messages():
    L = gpss.load()
    for opts in ({"spp": 0, "max_bounces": 1}, {"spp": 1, "max_bounces": 0}, {"spp": 1, "max_bounces": 1, "mix_R": 1.0},
                 {"spp": 1, "max_bounces": 70000}):
        o = gpss.render_opts(opts)
        cam = gpss.camera_desc({"type": "perspective", "eye": (0, -2, 0), "look_at": (0, 0, 0), "up": (0, 0, 1),
                                "width": 4, "height": 4})
        assert L.gpss_render(ctypes.c_void_p(8), ctypes.byref(cam), ctypes.byref(o), ctypes.c_void_p(8), None,
                             None, None) == 1


def test_batch_calls_reject_bad_arguments_on_the_host():
    L = gpss.load()
    h = ctypes.c_void_p(7)
    cam = (gpss.Camera * 1)()
    opts = (gpss.RenderOpts * 1)()
    scenes = (ctypes.c_void_p * 1)(None)
    assert L.gpss_batch_create(scenes, cam, opts, 0, 0, None, ctypes.byref(h)) == 1      # empty batch
    assert not h.value
    assert L.gpss_batch_create(scenes, cam, opts, 5000, 0, None, ctypes.byref(h)) == 1   # too many jobs
    assert L.gpss_batch_create(scenes, cam, opts, 1, 96, None, ctypes.byref(h)) == 1     # no such block size
    assert L.gpss_batch_create(None, cam, opts, 1, 0, None, ctypes.byref(h)) == 1
    assert L.gpss_batch_create(scenes, cam, opts, 1, 0, None, None) == 1
    assert L.gpss_batch_render(None, None, None, None, None) == 1
    assert L.gpss_batch_config(None, None, None, None, None) == 1
    assert L.gpss_batch_destroy(None) == 0


def test_object_descriptors_marshal_kernel_fields():
    """gpss._object_descs fills the kernel fields: 0 / NULL by default (the isotropic
    stationary kernel), the given scalars and host pointers otherwise."""
    keep = []
    plain = gpss._object_descs([_obj()], keep)[0]
    assert plain.length_scale_b == 0.0 and plain.length_scale_n == 0.0
    assert not plain.tangent and not plain.correlation_scale
    o = dict(_obj(), length_scale_b=0.2, length_scale_n=0.05, ndf="ggx",
             tangent=np.ones((3, 3, 3, 3), np.float64), correlation_scale=np.full((3, 3, 3), 2.0))
    keep = []
    d = gpss._object_descs([o], keep)[0]
    assert d.length_scale_b == pytest.approx(0.2) and d.length_scale_n == pytest.approx(0.05)
    assert d.ndf == gpss.NDF_KINDS["ggx"]
    arrays = {a.ctypes.data: a for a in keep if isinstance(a, np.ndarray)}
    t, c = arrays[d.tangent], arrays[d.correlation_scale]
    assert t.dtype == np.float32 and t.shape == (3, 3, 3, 3) and t.flags.c_contiguous
    assert c.dtype == np.float32 and np.all(c == 2.0)
