"""Python binding of the GPSS C-ABI (``include/gpss.h``).

Argument marshalling only: every step of the renderer runs in the CUDA library
``libgpss.so``.  PyTorch supplies device memory and streams.  There is no CPU
fallback -- if the library cannot be built or loaded, every call raises.

Scene, camera, light and option dictionaries follow ``workloads.py``.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None


class GpssError(RuntimeError):
    def __init__(self, fn: str, status: int, message: str):
        super().__init__("%s failed (status %d): %s" % (fn, status, message))
        self.status = status


STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "TIMEOUT", 5: "UNSUPPORTED"}
FLAG_KEEP_PATH_RADIANCE = 1
FLAG_EXACT_VNDF = 2


class ObjectDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("bbox_min", ctypes.c_float * 3), ("bbox_max", ctypes.c_float * 3),
                ("mean", ctypes.c_void_p), ("variance", ctypes.c_void_p), ("albedo", ctypes.c_void_p),
                ("albedo_channels", ctypes.c_int), ("length_scale", ctypes.c_float), ("ndf", ctypes.c_int),
                ("length_scale_b", ctypes.c_float), ("length_scale_n", ctypes.c_float),
                ("tangent", ctypes.c_void_p), ("correlation_scale", ctypes.c_void_p)]


NDF_KINDS = {"gpss": 0, "beckmann": 1, "ggx": 2}


class LightDesc(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("dir", ctypes.c_float * 3), ("radiance", ctypes.c_float * 3)]


class Camera(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("eye", ctypes.c_float * 3), ("look_at", ctypes.c_float * 3),
                ("up", ctypes.c_float * 3), ("fov_y_deg", ctypes.c_float), ("ortho_w", ctypes.c_float),
                ("ortho_h", ctypes.c_float), ("width", ctypes.c_int), ("height", ctypes.c_int)]


class RenderOpts(ctypes.Structure):
    _fields_ = [("spp", ctypes.c_int), ("max_bounces", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("mix_R", ctypes.c_float), ("flags", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [("paths", ctypes.c_uint64), ("vertices", ctypes.c_uint64), ("null_collisions", ctypes.c_uint64),
                ("shadow_steps", ctypes.c_uint64), ("majorant_cells", ctypes.c_uint64),
                ("truncated", ctypes.c_uint64), ("aborted", ctypes.c_uint64),
                ("max_path_events", ctypes.c_uint64), ("ms", ctypes.c_float), ("nonfinite", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_VP = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float

# name -> argtypes (restype is always int status, except noted)
_SIGS = {
    "gpss_scene_create": [ctypes.POINTER(ObjectDesc), _I, ctypes.POINTER(LightDesc), _I, _VP, ctypes.POINTER(_VP)],
    "gpss_scene_update": [_VP, ctypes.POINTER(ObjectDesc), _I, _VP],
    "gpss_scene_destroy": [_VP],
    "gpss_scene_set_traversal": [_VP, _I, _F, _VP],
    "gpss_scene_set_schedule": [_VP, _I],
    "gpss_scene_set_local_majorant": [_VP, _F],
    "gpss_scene_set_object_grids": [_VP, _I],
    "gpss_scene_set_surface_flight": [_VP, _I],
    "gpss_scene_majorant": [_VP, ctypes.POINTER(_I), _VP, _VP],
    "gpss_render": [_VP, ctypes.POINTER(Camera), ctypes.POINTER(RenderOpts), _VP, _VP, ctypes.POINTER(Stats), _VP],
    "gpss_render_noalloc": [_VP, ctypes.POINTER(Camera), ctypes.POINTER(RenderOpts), _VP, ctypes.POINTER(Stats), _VP],
    "gpss_render_adjoint": [_VP, ctypes.POINTER(Camera), ctypes.POINTER(RenderOpts), _VP, _VP, _VP, _VP, _VP, _VP,
                            ctypes.POINTER(Stats), _VP],
    "gpss_batch_create": [ctypes.POINTER(_VP), ctypes.POINTER(Camera), ctypes.POINTER(RenderOpts), _I, _I, _VP,
                          ctypes.POINTER(_VP)],
    "gpss_batch_render": [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(Stats), _VP],
    "gpss_batch_config": [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "gpss_batch_destroy": [_VP],
    "gpss_eval_sigma_t": [_VP, _I, _VP, _VP, _VP, _VP],
    "gpss_eval_local_majorant": [_VP, _I, _VP, _VP, _VP, _VP, _VP, _VP, _VP],
    "gpss_eval_local_piece": [_VP, _I, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP],
    "gpss_eval_phase": [_VP, _I, _I, _VP, _VP, _VP, _F, _VP, _VP, _VP],
    "gpss_sample_phase": [_VP, _I, _I, _VP, _VP, _VP, _F, _VP, _VP, _VP, _VP],
    "gpss_sample_phase_vndf": [_VP, _I, _I, _VP, _VP, _VP, _VP, _VP, _VP, _VP],
    "gpss_eval_ndf": [_I, _VP, _F, _F, _F, _F, _VP, _VP],
    "gpss_eval_projected_area": [_I, _VP, _F, _F, _F, _F, _VP, _VP],
    "gpss_eval_transmittance": [_VP, _I, _VP, _VP, _VP, _VP, _VP],
    "gpss_estimate_transmittance": [_VP, _I, _VP, _VP, _VP, _I, ctypes.c_uint64, _VP, _VP],
    "gpss_sample_free_flight": [_VP, _I, _VP, _VP, _I, ctypes.c_uint64, _VP, _VP],
    "gpss_philox4x32_10": [_I, _VP, _VP, _VP, _VP],
}


def load():
    """Builds (if stale) and loads libgpss.so; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(_build.build())
            for name, args in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            L.gpss_last_error.restype = ctypes.c_char_p
            L.gpss_last_error.argtypes = []
            L.gpss_version.restype = ctypes.c_int
            L.gpss_version.argtypes = []
            _lib = L
    return _lib


def library_path() -> str:
    return _build.LIB


def _call(name, *args):
    L = load()
    st = getattr(L, name)(*args)
    if st != 0:
        raise GpssError(name, st, L.gpss_last_error().decode())
    return st


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the GPSS library needs a CUDA device")
    return torch


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(x):
    """Device or host pointer of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous
        return ctypes.c_void_p(x.ctypes.data)
    assert x.is_contiguous()
    return ctypes.c_void_p(x.data_ptr())


_LIGHT = {"directional": 0, "sky": 1, "uniform": 2}
_CAM = {"ortho": 0, "perspective": 1}


def light_desc(light: dict) -> LightDesc:
    L = LightDesc()
    L.type = _LIGHT[light["type"]]
    for a in range(3):
        L.dir[a] = float(light.get("dir", (0, 0, 1))[a])
        L.radiance[a] = float(light.get("radiance", (1, 1, 1))[a])
    return L


def camera_desc(cam: dict) -> Camera:
    c = Camera()
    c.type = _CAM[cam["type"]]
    for a in range(3):
        c.eye[a] = float(cam["eye"][a])
        c.look_at[a] = float(cam["look_at"][a])
        c.up[a] = float(cam["up"][a])
    c.fov_y_deg = float(cam.get("fov_y_deg", 40.0))
    c.ortho_w = float(cam.get("ortho_w", 1.0))
    c.ortho_h = float(cam.get("ortho_h", 1.0))
    c.width = int(cam["width"])
    c.height = int(cam["height"])
    return c


def render_opts(opts: dict, flags: int = 0) -> RenderOpts:
    o = RenderOpts()
    o.spp = int(opts["spp"])
    o.max_bounces = int(opts["max_bounces"])
    o.seed = int(opts.get("seed", 0))
    o.mix_R = float(opts.get("mix_R", 0.5))
    o.flags = int(opts.get("flags", 0)) | flags
    sampler = opts.get("sampler", "mixture")
    if sampler == "vndf":
        o.flags |= FLAG_EXACT_VNDF
    elif sampler != "mixture":
        raise ValueError("sampler must be 'mixture' (the paper's) or 'vndf' (exact visible normals)")
    return o


def _f32(a):
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.float32)
    return a.contiguous().float()


def _object_descs(objects, keep):
    """Descriptors of object dicts: mean, var (or variance), albedo ((nz,ny,nx) or
    (channels,nz,ny,nx)), bbox_min, bbox_max, length_scale, optional ndf ("gpss",
    "beckmann", "ggx"), length_scale_b, length_scale_n, tangent (3,nz,ny,nx) and
    correlation_scale (nz,ny,nx); arrays are numpy (host) or CUDA tensors."""
    descs = (ObjectDesc * len(objects))()
    for k, o in enumerate(objects):
        mean, var, alb = o["mean"], o["variance"] if "variance" in o else o["var"], o["albedo"]
        arrs = [_f32(a) for a in (mean, var, alb)]
        keep.extend(arrs)
        mean, var, alb = arrs
        nz, ny, nx = mean.shape
        D = descs[k]
        D.nx, D.ny, D.nz = nx, ny, nz
        for a in range(3):
            D.bbox_min[a] = float(o["bbox_min"][a])
            D.bbox_max[a] = float(o["bbox_max"][a])
        D.mean = _ptr(mean).value
        D.variance = _ptr(var).value
        D.albedo = _ptr(alb).value
        D.albedo_channels = 1 if alb.ndim == 3 else int(alb.shape[0])
        D.length_scale = float(o["length_scale"])
        D.ndf = NDF_KINDS[o.get("ndf", "gpss")]
        D.length_scale_b = float(o.get("length_scale_b", 0.0))
        D.length_scale_n = float(o.get("length_scale_n", 0.0))
        for key in ("tangent", "correlation_scale"):
            if o.get(key) is not None:
                a = _f32(o[key])
                keep.append(a)
                setattr(D, key, _ptr(a).value)
    return descs


class Scene:
    """A scene owned by the library (grids copied into its layout)."""

    def __init__(self, scene: dict, majorant_brick: int = 0, stream=None):
        load()
        self.handle = ctypes.c_void_p()
        keep = []
        descs = _object_descs(scene["objects"], keep)
        self.n_objs = len(scene["objects"])
        self.shapes = [tuple(o["mean"].shape) for o in scene["objects"]]
        self.channels = [1 if o["albedo"].ndim == 3 else int(o["albedo"].shape[0]) for o in scene["objects"]]
        L = light_desc(scene.get("light", {"type": "directional", "dir": (0, 0, 1), "radiance": (1, 1, 1)}))
        _call("gpss_scene_create", descs, self.n_objs, ctypes.byref(L), int(majorant_brick), _stream(stream),
              ctypes.byref(self.handle))

    def update(self, objects, stream=None):
        keep = []
        descs = _object_descs(objects, keep)
        _call("gpss_scene_update", self.handle, descs, len(objects), _stream(stream))
        del keep

    def set_schedule(self, shade_min: int = 24):
        _call("gpss_scene_set_schedule", self.handle, int(shade_min))

    def set_object_grids(self, enable: bool = True):
        _call("gpss_scene_set_object_grids", self.handle, 1 if enable else 0)

    def set_local_majorant(self, hot: float = 4.0):
        _call("gpss_scene_set_local_majorant", self.handle, float(hot))

    def set_surface_flight(self, enable: bool = True):
        _call("gpss_scene_set_surface_flight", self.handle, 1 if enable else 0)

    def set_traversal(self, skip_levels: int = 5, kappa: float = 0.5, stream=None):
        _call("gpss_scene_set_traversal", self.handle, int(skip_levels), float(kappa), _stream(stream))

    def majorant(self, stream=None):
        torch = _torch()
        dims = (ctypes.c_int * 3)()
        _call("gpss_scene_majorant", self.handle, dims, None, _stream(stream))
        out = torch.empty((dims[2], dims[1], dims[0]), device="cuda", dtype=torch.float32)
        _call("gpss_scene_majorant", self.handle, dims, _ptr(out), _stream(stream))
        return out

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load().gpss_scene_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def render(scene: Scene, camera: dict, opts: dict, image=None, sqsum=None, want_sqsum=False, stats=True,
           keep_path_radiance=False, stream=None):
    """Forward render.  Returns (image, sqsum or None, stats dict or None).
    image/sqsum may be preallocated torch CUDA tensors or numpy host arrays (H, W, 3)."""
    torch = _torch()
    H, W = int(camera["height"]), int(camera["width"])
    if image is None:
        image = torch.empty((H, W, 3), device="cuda", dtype=torch.float32)
    if sqsum is None and want_sqsum:
        sqsum = torch.empty((H, W, 3), device="cuda", dtype=torch.float32)
    st = Stats() if stats else None
    c = camera_desc(camera)
    o = render_opts(opts, FLAG_KEEP_PATH_RADIANCE if keep_path_radiance else 0)
    _call("gpss_render", scene.handle, ctypes.byref(c), ctypes.byref(o), _ptr(image), _ptr(sqsum),
          ctypes.byref(st) if st is not None else None, _stream(stream))
    return image, sqsum, (st.as_dict() if st is not None else None)


def render_adjoint(scene: Scene, camera: dict, opts: dict, d_image, d_mean=None, d_variance=None, d_albedo=None,
                   d_length_scale=None, d_correlation_scale=None, stats=True, stream=None):
    st = Stats() if stats else None
    c = camera_desc(camera)
    o = render_opts(opts)
    _call("gpss_render_adjoint", scene.handle, ctypes.byref(c), ctypes.byref(o), _ptr(d_image), _ptr(d_mean),
          _ptr(d_variance), _ptr(d_albedo), _ptr(d_length_scale), _ptr(d_correlation_scale),
          ctypes.byref(st) if st is not None else None, _stream(stream))
    return st.as_dict() if st is not None else None


class Batch:
    """Many (scene, camera, options) jobs rendered by one graph-replayed persistent
    launch (gpss_batch_*).  block_size 0 autotunes the launch shape at creation."""

    def __init__(self, scenes, cameras, opts, block_size: int = 0, stream=None):
        n = len(scenes)
        if not (len(cameras) == n and len(opts) == n):
            raise ValueError("scenes, cameras and opts must have the same length")
        self.scenes = list(scenes)  # keeps the scenes alive as long as the batch
        self.shapes = [(int(c["height"]), int(c["width"]), 3) for c in cameras]
        sh = (_VP * n)(*[sc.handle for sc in self.scenes])
        cams = (Camera * n)(*[camera_desc(c) for c in cameras])
        ops = (RenderOpts * n)(*[render_opts(o) for o in opts])
        h = _VP()
        _call("gpss_batch_create", sh, cams, ops, n, int(block_size), _stream(stream), ctypes.byref(h))
        self.handle = h

    @property
    def config(self):
        b, s, c, g = _I(), _I(), _I(), _I()
        _call("gpss_batch_config", self.handle, ctypes.byref(b), ctypes.byref(s), ctypes.byref(c), ctypes.byref(g))
        return {"block_size": b.value, "shade_min": s.value, "chunk": c.value, "grid": g.value}

    def render(self, images=None, sqsums=None, want_sqsum=False, stats=True, stream=None):
        """Renders every job.  images / sqsums: lists of CUDA tensors (H, W, 3) or None
        (allocated here).  Returns (images, sqsums or None, stats dict or None)."""
        torch = _torch()
        n = len(self.shapes)
        if images is None:
            images = [torch.empty(sh, device="cuda", dtype=torch.float32) for sh in self.shapes]
        if sqsums is None and want_sqsum:
            sqsums = [torch.empty(sh, device="cuda", dtype=torch.float32) for sh in self.shapes]
        for i, im in enumerate(images):
            if tuple(im.shape) != self.shapes[i] or not im.is_cuda or im.dtype != torch.float32:
                raise ValueError("image %d must be a float32 CUDA tensor of shape %s" % (i, self.shapes[i]))
        ip = (_VP * n)(*[im.data_ptr() for im in images])
        sp = (_VP * n)(*[(q.data_ptr() if q is not None else None) for q in sqsums]) if sqsums is not None else None
        st = Stats() if stats else None
        _call("gpss_batch_render", self.handle, ip, sp, ctypes.byref(st) if st is not None else None, _stream(stream))
        return images, sqsums, (st.as_dict() if st is not None else None)

    def close(self):
        if getattr(self, "handle", None):
            _call("gpss_batch_destroy", self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _dev(x):
    torch = _torch()
    return torch.as_tensor(np.asarray(x, dtype=np.float32) if not hasattr(x, "device") else x,
                           dtype=torch.float32).cuda().contiguous()


def eval_sigma_t(scene: Scene, pos, dirs, stream=None):
    torch = _torch()
    pos, dirs = _dev(pos).reshape(-1, 3), _dev(dirs).reshape(-1, 3)
    out = torch.empty(len(pos), device="cuda", dtype=torch.float32)
    _call("gpss_eval_sigma_t", scene.handle, len(pos), _ptr(pos), _ptr(dirs), _ptr(out), _stream(stream))
    return out


def eval_local_majorant(scene: Scene, org, dirs, t0, tmax, stream=None):
    """(t_end, sbar) of the local majorant piece starting at org + t0 dir."""
    torch = _torch()
    org, dirs, t0, tmax = _dev(org), _dev(dirs), _dev(t0), _dev(tmax)
    t_end = torch.empty(len(org), device="cuda")
    sbar = torch.empty(len(org), device="cuda")
    _call("gpss_eval_local_majorant", scene.handle, len(org), _ptr(org), _ptr(dirs), _ptr(t0), _ptr(tmax),
          _ptr(t_end), _ptr(sbar), _stream(stream))
    return t_end, sbar


def eval_local_piece(scene: Scene, org, dirs, t0, tmax, tau, stream=None):
    """Returns (t_end, lin, depth, t_hit, sbar_hit) of the traversal's local pieces."""
    torch = _torch()
    org, dirs, t0, tmax, tau = _dev(org), _dev(dirs), _dev(t0), _dev(tmax), _dev(tau)
    n = len(org)
    outs = [torch.empty(n, device="cuda") for _ in range(5)]
    outs[1] = torch.empty(n, device="cuda", dtype=torch.int32)
    t_end, lin, depth, t_hit, sbar_hit = outs
    _call("gpss_eval_local_piece", scene.handle, n, _ptr(org), _ptr(dirs), _ptr(t0), _ptr(tmax), _ptr(tau),
          _ptr(t_end), _ptr(lin), _ptr(depth), _ptr(t_hit), _ptr(sbar_hit), _stream(stream))
    return t_end, lin, depth, t_hit, sbar_hit


def eval_phase(scene: Scene, k: int, pos, d_in, d_out, mix_R=0.5, stream=None):
    torch = _torch()
    pos, d_in, d_out = (_dev(a).reshape(-1, 3) for a in (pos, d_in, d_out))
    p = torch.empty((len(pos), 3), device="cuda", dtype=torch.float32)
    pdf = torch.empty(len(pos), device="cuda", dtype=torch.float32)
    _call("gpss_eval_phase", scene.handle, int(k), len(pos), _ptr(pos), _ptr(d_in), _ptr(d_out), float(mix_R),
          _ptr(p), _ptr(pdf), _stream(stream))
    return p, pdf


def sample_phase(scene: Scene, k: int, pos, d_in, u, mix_R=0.5, stream=None):
    torch = _torch()
    pos, d_in, u = (_dev(a).reshape(-1, 3) for a in (pos, d_in, u))
    d_out = torch.empty((len(pos), 3), device="cuda", dtype=torch.float32)
    w = torch.empty((len(pos), 3), device="cuda", dtype=torch.float32)
    pdf = torch.empty(len(pos), device="cuda", dtype=torch.float32)
    _call("gpss_sample_phase", scene.handle, int(k), len(pos), _ptr(pos), _ptr(d_in), _ptr(u), float(mix_R),
          _ptr(d_out), _ptr(w), _ptr(pdf), _stream(stream))
    return d_out, w, pdf


def sample_phase_vndf(scene: Scene, k: int, pos, d_in, u, stream=None):
    """Exact visible-normal samples: (d_out, weight = F, pdf = p/F)."""
    torch = _torch()
    pos, d_in, u = _dev(pos), _dev(d_in), _dev(u)
    n = len(pos)
    d_out = torch.empty((n, 3), device="cuda")
    w = torch.empty((n, 3), device="cuda")
    pdf = torch.empty(n, device="cuda")
    _call("gpss_sample_phase_vndf", scene.handle, int(k), n, _ptr(pos), _ptr(d_in), _ptr(u), _ptr(d_out), _ptr(w),
          _ptr(pdf), _stream(stream))
    return d_out, w, pdf


def eval_ndf(m, G, ax, ay, az, stream=None):
    torch = _torch()
    m = _dev(m).reshape(-1, 3)
    out = torch.empty(len(m), device="cuda", dtype=torch.float32)
    _call("gpss_eval_ndf", len(m), _ptr(m), float(G), float(ax), float(ay), float(az), _ptr(out), _stream(stream))
    return out


def eval_projected_area(w, G, ax, ay, az, stream=None):
    torch = _torch()
    w = _dev(w).reshape(-1, 3)
    out = torch.empty(len(w), device="cuda", dtype=torch.float32)
    _call("gpss_eval_projected_area", len(w), _ptr(w), float(G), float(ax), float(ay), float(az), _ptr(out),
          _stream(stream))
    return out


def eval_transmittance(scene: Scene, org, dirs, tmax, stream=None):
    torch = _torch()
    org, dirs = _dev(org).reshape(-1, 3), _dev(dirs).reshape(-1, 3)
    tmax = _dev(tmax).reshape(-1)
    out = torch.empty(len(org), device="cuda", dtype=torch.float32)
    _call("gpss_eval_transmittance", scene.handle, len(org), _ptr(org), _ptr(dirs), _ptr(tmax), _ptr(out),
          _stream(stream))
    return out


def estimate_transmittance(scene: Scene, org, dirs, tmax, samples, seed=0, stream=None):
    torch = _torch()
    org, dirs = _dev(org).reshape(-1, 3), _dev(dirs).reshape(-1, 3)
    tmax = _dev(tmax).reshape(-1)
    out = torch.empty(len(org), device="cuda", dtype=torch.float32)
    _call("gpss_estimate_transmittance", scene.handle, len(org), _ptr(org), _ptr(dirs), _ptr(tmax), int(samples),
          int(seed), _ptr(out), _stream(stream))
    return out


def sample_free_flight(scene: Scene, org, dirs, samples, seed=0, stream=None):
    torch = _torch()
    org, dirs = _dev(org).reshape(-1, 3), _dev(dirs).reshape(-1, 3)
    out = torch.empty((len(org), int(samples)), device="cuda", dtype=torch.float32)
    _call("gpss_sample_free_flight", scene.handle, len(org), _ptr(org), _ptr(dirs), int(samples), int(seed),
          _ptr(out), _stream(stream))
    return out


def philox4x32_10(ctr, key, stream=None):
    torch = _torch()
    c = torch.as_tensor(np.asarray(ctr, dtype=np.uint32).view(np.int32)).cuda().contiguous()
    k = torch.as_tensor(np.asarray(key, dtype=np.uint32).view(np.int32)).cuda().contiguous()
    n = c.numel() // 4
    out = torch.empty(4 * n, device="cuda", dtype=torch.int32)
    _call("gpss_philox4x32_10", n, _ptr(c), _ptr(k), _ptr(out), _stream(stream))
    return out.cpu().numpy().view(np.uint32).reshape(n, 4)


# ----------------------------------------------------------------- differentiable rendering
class _RenderFn:
    """torch.autograd.Function wrapper (defined lazily so that importing this
    module needs no CUDA).  Forward: upload the parameter tensors into the scene
    (single object) and render.  Backward: gpss_render_adjoint with the incoming
    image gradient; returns gradients for mean, variance, albedo, length scale
    and (when given) the correlation-scale grid."""
    fn = None

    @classmethod
    def get(cls):
        if cls.fn is None:
            import torch

            class RenderFunction(torch.autograd.Function):
                @staticmethod
                def forward(ctx, mean, var, albedo, length_scale, cscale, scene, obj, camera, opts):
                    o = dict(obj)
                    o["mean"], o["var"], o["albedo"] = mean.detach(), var.detach(), albedo.detach()
                    o["length_scale"] = float(length_scale)
                    if cscale is not None:
                        o["correlation_scale"] = cscale.detach()
                    ctx.has_cs = cscale is not None
                    scene.update([o])
                    image, _, _ = render(scene, camera, opts, stats=False, keep_path_radiance=True)
                    ctx.scene, ctx.camera, ctx.opts = scene, camera, opts
                    ctx.shapes = (mean.shape, var.shape, albedo.shape)
                    return image

                @staticmethod
                def backward(ctx, grad_image):
                    g = grad_image.contiguous().float()
                    dm = torch.zeros(ctx.shapes[0], device="cuda", dtype=torch.float32)
                    dv = torch.zeros(ctx.shapes[1], device="cuda", dtype=torch.float32)
                    da = torch.zeros(ctx.shapes[2], device="cuda", dtype=torch.float32)
                    dl = torch.zeros(1, device="cuda", dtype=torch.float32)
                    dc = torch.zeros(ctx.shapes[0], device="cuda", dtype=torch.float32) if ctx.has_cs else None
                    render_adjoint(ctx.scene, ctx.camera, ctx.opts, g, dm, dv, da, dl, dc, stats=False)
                    return dm, dv, da, dl[0], dc, None, None, None, None

            cls.fn = RenderFunction
        return cls.fn


def render_differentiable(scene: Scene, obj: dict, mean, var, albedo, length_scale, camera: dict, opts: dict,
                          correlation_scale=None):
    """Differentiable render of a single-object scene.  mean/var/albedo are CUDA
    tensors shaped like the scene's grids; length_scale a 0-d CUDA tensor;
    correlation_scale (optional) a CUDA tensor shaped like mean.  obj supplies the
    box (bbox_min, bbox_max).  Returns the (H, W, 3) image."""
    return _RenderFn.get().apply(mean, var, albedo, length_scale, correlation_scale, scene, obj, camera, opts)
