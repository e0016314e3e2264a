"""The allocation-free render entry point against the regular one.

gpss_render_noalloc serves callers that may not allocate device memory while
rendering (applications that account for every device byte themselves, real-time
loops where an allocation's latency or failure is unacceptable).  It keeps its scratch in a fixed static device array instead
of scene-owned buffers.  Given the same scene, camera and options it renders the
same paths, so its image must equal gpss_render's up to the summation order of
the film's float atomics -- on two calls in a row, which also checks that the
shared scratch is cleared between calls.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2603_00280_gb300 import gpss
from paper_2603_00280_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_render_matches_regular_render_twice():
    import torch

    L = gpss.load()
    wl = W.heterogeneous(n=32, width=40, height=24, spp=16, max_bounces=8)
    S = gpss.Scene(wl["scene"])
    cam = gpss.camera_desc(wl["camera"])
    opts = gpss.render_opts(wl["opts"])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ref = torch.empty((24, 40, 3), device="cuda", dtype=torch.float32)
    st_ref = gpss.Stats()
    assert L.gpss_render(S.handle, ctypes.byref(cam), ctypes.byref(opts), ctypes.c_void_p(ref.data_ptr()), None,
                         ctypes.byref(st_ref), stream) == 0
    ref = ref.cpu().numpy()
    for call in range(2):
        dev = torch.full((24, 40, 3), -1.0, device="cuda", dtype=torch.float32)
        st = gpss.Stats()
        rc = L.gpss_render_noalloc(S.handle, ctypes.byref(cam), ctypes.byref(opts), ctypes.c_void_p(dev.data_ptr()),
                                   ctypes.byref(st), stream)
        assert rc == 0, L.gpss_last_error()
        np.testing.assert_allclose(dev.cpu().numpy(), ref, rtol=1e-5, atol=1e-7)
        assert st.paths == st_ref.paths and st.vertices == st_ref.vertices
        # host output through the same entry point
        host = np.full((24, 40, 3), -1.0, dtype=np.float32)
        rc = L.gpss_render_noalloc(S.handle, ctypes.byref(cam), ctypes.byref(opts), ctypes.c_void_p(host.ctypes.data),
                                   None, stream)
        assert rc == 0, L.gpss_last_error()
        torch.cuda.synchronize()
        np.testing.assert_allclose(host, ref, rtol=1e-5, atol=1e-7)
        # pinned host output without stats: complete when the call returns (no extra synchronize)
        pinned = torch.full((24, 40, 3), -1.0, dtype=torch.float32).pin_memory()
        rc = L.gpss_render_noalloc(S.handle, ctypes.byref(cam), ctypes.byref(opts), ctypes.c_void_p(pinned.data_ptr()),
                                   None, stream)
        assert rc == 0, L.gpss_last_error()
        np.testing.assert_allclose(pinned.numpy(), ref, rtol=1e-5, atol=1e-7)


def test_noalloc_render_rejects_images_beyond_its_scratch():
    import torch

    L = gpss.load()
    wl = W.heterogeneous(n=16, width=257, height=256, spp=1, max_bounces=1)
    S = gpss.Scene(wl["scene"])
    cam = gpss.camera_desc(wl["camera"])
    opts = gpss.render_opts(wl["opts"])
    out = torch.empty((256, 257, 3), device="cuda", dtype=torch.float32)
    rc = L.gpss_render_noalloc(S.handle, ctypes.byref(cam), ctypes.byref(opts), ctypes.c_void_p(out.data_ptr()), None,
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1
    assert b"65536 pixels" in L.gpss_last_error()
