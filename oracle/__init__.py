"""FP64 CPU oracle for the GPSS macrofacet medium -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library (the CUDA path in
``paper_2603_00280_gb300``) never imports, links or calls it, and the two share
no source.  The arithmetic lives in the C files next to this module
(``gpss_oracle_medium.c``, ``gpss_oracle_transport.c``, and the dual numbers of the
adjoint in ``gpss_oracle_dual.c``); this module only
compiles them with gcc and marshals arguments through ctypes.

Scenes, cameras, lights and options are the plain dictionaries produced by
``paper_2603_00280_gb300.workloads`` (seeded synthetic inputs, no method
arithmetic).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["gpss_oracle_medium.c", "gpss_oracle_transport.c", "gpss_oracle_dual.c"]
_HEADERS = ["gpss_oracle.h", "gpss_oracle_internal.h"]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, no fast-math)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    deps = srcs + [os.path.join(_HERE, h) for h in _HEADERS]
    if not force and os.path.exists(_LIB):
        if os.path.getmtime(_LIB) >= max(os.path.getmtime(p) for p in deps):
            return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm", "-lpthread"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class _Object(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("bmin", ctypes.c_double * 3), ("bmax", ctypes.c_double * 3),
        ("mean", ctypes.POINTER(ctypes.c_float)), ("var", ctypes.POINTER(ctypes.c_float)),
        ("albedo", ctypes.POINTER(ctypes.c_float)), ("channels", ctypes.c_int),
        ("length_scale", ctypes.c_double), ("ndf", ctypes.c_int),
        ("length_scale_b", ctypes.c_double), ("length_scale_n", ctypes.c_double),
        ("tangent", ctypes.POINTER(ctypes.c_float)), ("cscale", ctypes.POINTER(ctypes.c_float)),
    ]


class _Light(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("dir", ctypes.c_double * 3), ("radiance", ctypes.c_double * 3)]


class _Camera(ctypes.Structure):
    _fields_ = [
        ("type", ctypes.c_int), ("eye", ctypes.c_double * 3), ("look_at", ctypes.c_double * 3),
        ("up", ctypes.c_double * 3), ("fov_y_deg", ctypes.c_double), ("ortho_w", ctypes.c_double),
        ("ortho_h", ctypes.c_double), ("width", ctypes.c_int), ("height", ctypes.c_int),
    ]


class _Scene(ctypes.Structure):
    _fields_ = [("objs", ctypes.POINTER(_Object)), ("n_objs", ctypes.c_int), ("light", _Light)]


class _Opts(ctypes.Structure):
    _fields_ = [
        ("spp", ctypes.c_int), ("max_bounces", ctypes.c_int), ("seed", ctypes.c_uint64),
        ("mix_R", ctypes.c_double), ("row_begin", ctypes.c_int), ("row_end", ctypes.c_int),
        ("row_step", ctypes.c_int), ("col_begin", ctypes.c_int), ("col_end", ctypes.c_int),
        ("threads", ctypes.c_int), ("sampler", ctypes.c_int),
    ]


class _Stats(ctypes.Structure):
    _fields_ = [("paths", ctypes.c_uint64), ("vertices", ctypes.c_uint64), ("truncated", ctypes.c_uint64)]


_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)


class _GradOut(ctypes.Structure):
    _fields_ = [
        ("nodes", ctypes.POINTER(ctypes.c_int64)), ("n_nodes", ctypes.c_int64),
        ("d_mean", _PD), ("d_var", _PD), ("d_albedo", _PD), ("d_cscale", _PD), ("d_l", _PD),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_erfcx.restype = _D
            L.orc_erfcx.argtypes = [_D]
            L.orc_log_ndtr.restype = _D
            L.orc_log_ndtr.argtypes = [_D]
            L.orc_inv_mills.restype = _D
            L.orc_inv_mills.argtypes = [_D]
            L.orc_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
            L.orc_field.restype = ctypes.c_int
            L.orc_field.argtypes = [ctypes.POINTER(_Object), _PD, _PD, _PD, _PD, _PD]
            L.orc_projected_area_local.restype = _D
            L.orc_projected_area_local.argtypes = [_PD, _D, _D, _D, _D]
            L.orc_ndf_local.restype = _D
            L.orc_ndf_local.argtypes = [_PD, _D, _D, _D, _D]
            L.orc_ndf_hf.restype = _D
            L.orc_ndf_hf.argtypes = [_PD, ctypes.c_int, _D]
            L.orc_projected_area_hf.restype = _D
            L.orc_projected_area_hf.argtypes = [_PD, ctypes.c_int, _D]
            L.orc_sigma_t.restype = _D
            L.orc_sigma_t.argtypes = [ctypes.POINTER(_Scene), _PD, _PD]
            L.orc_sigma_t_object.restype = _D
            L.orc_sigma_t_object.argtypes = [ctypes.POINTER(_Object), _PD, _PD]
            L.orc_phase_eval.restype = ctypes.c_int
            L.orc_phase_eval.argtypes = [ctypes.POINTER(_Scene), ctypes.c_int, _PD, _PD, _PD, _D, _PD, _PD]
            L.orc_phase_sample.restype = ctypes.c_int
            L.orc_phase_sample.argtypes = [ctypes.POINTER(_Scene), ctypes.c_int, _PD, _PD, _D, _PD, _PD, _PD, _PD]
            L.orc_phase_sample_exact.restype = ctypes.c_int
            L.orc_phase_sample_exact.argtypes = [ctypes.POINTER(_Scene), ctypes.c_int, _PD, _PD, _PD, _PD, _PD, _PD]
            L.orc_optical_depth.restype = _D
            L.orc_optical_depth.argtypes = [ctypes.POINTER(_Scene), _PD, _PD, _D]
            L.orc_transmittance.restype = _D
            L.orc_transmittance.argtypes = [ctypes.POINTER(_Scene), _PD, _PD, _D]
            L.orc_render.restype = ctypes.c_int
            L.orc_render.argtypes = [ctypes.POINTER(_Scene), ctypes.POINTER(_Camera), ctypes.POINTER(_Opts),
                                     _PD, _PD, ctypes.POINTER(_Stats)]
            L.orc_render_diff.restype = ctypes.c_int
            L.orc_render_diff.argtypes = [ctypes.POINTER(_Scene), ctypes.POINTER(_Scene), ctypes.POINTER(_Camera),
                                          ctypes.POINTER(_Opts), _PD, _PD, ctypes.POINTER(_Stats)]
            L.orc_camera_ray.argtypes = [ctypes.POINTER(_Camera), ctypes.c_int, ctypes.c_int, _D, _D, _PD, _PD]
            L.orc_render_grad.restype = ctypes.c_int
            L.orc_render_grad.argtypes = [ctypes.POINTER(_Scene), ctypes.POINTER(_Camera), ctypes.POINTER(_Opts), _PD,
                                          ctypes.POINTER(_GradOut), ctypes.POINTER(_Stats),
                                          ctypes.POINTER(ctypes.c_uint64)]
            L.orc_dual_eval.restype = ctypes.c_int
            L.orc_dual_eval.argtypes = [ctypes.POINTER(_Object), ctypes.c_int, _PD, _PD, _PD, _PD, _PD,
                                        ctypes.POINTER(ctypes.c_int64)]
            _lib = L
    return _lib


def _vec(v, n=3):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(n))
    return a, a.ctypes.data_as(_PD)


_LIGHT_TYPES = {"directional": 0, "sky": 1, "uniform": 2}
_CAMERA_TYPES = {"ortho": 0, "perspective": 1}


NDF_KINDS = {"gpss": 0, "beckmann": 1, "ggx": 2}


class Scene:
    """ctypes view of a scene dictionary; keeps the float32 grids alive."""

    def __init__(self, scene: dict):
        objs = scene["objects"]
        self._keep = []
        self._objs = (_Object * len(objs))()
        for k, o in enumerate(objs):
            mean = np.ascontiguousarray(o["mean"], dtype=np.float32)
            var = np.ascontiguousarray(o["var"], dtype=np.float32)
            alb = np.ascontiguousarray(o["albedo"], dtype=np.float32)
            if alb.ndim == 3:
                alb = alb[None]
            nz, ny, nx = mean.shape
            assert var.shape == mean.shape and alb.shape[1:] == mean.shape and alb.shape[0] in (1, 3)
            self._keep += [mean, var, alb]
            ob = self._objs[k]
            ob.nx, ob.ny, ob.nz = nx, ny, nz
            for a in range(3):
                ob.bmin[a] = float(o["bbox_min"][a])
                ob.bmax[a] = float(o["bbox_max"][a])
            fp = ctypes.POINTER(ctypes.c_float)
            ob.mean = mean.ctypes.data_as(fp)
            ob.var = var.ctypes.data_as(fp)
            ob.albedo = alb.ctypes.data_as(fp)
            ob.channels = alb.shape[0]
            ob.length_scale = float(o["length_scale"])
            ob.ndf = NDF_KINDS[o.get("ndf", "gpss")]
            ob.length_scale_b = float(o.get("length_scale_b", 0.0))
            ob.length_scale_n = float(o.get("length_scale_n", 0.0))
            if o.get("tangent") is not None:
                t = np.ascontiguousarray(o["tangent"], dtype=np.float32)
                assert t.shape == (3,) + mean.shape
                self._keep.append(t)
                ob.tangent = t.ctypes.data_as(fp)
            if o.get("correlation_scale") is not None:
                c = np.ascontiguousarray(o["correlation_scale"], dtype=np.float32)
                assert c.shape == mean.shape and np.all(c > 0)
                self._keep.append(c)
                ob.cscale = c.ctypes.data_as(fp)
        self.s = _Scene()
        self.s.objs = ctypes.cast(self._objs, ctypes.POINTER(_Object))
        self.s.n_objs = len(objs)
        light = scene.get("light", {"type": "directional", "dir": (0, 0, 1), "radiance": (1, 1, 1)})
        self.s.light.type = _LIGHT_TYPES[light["type"]]
        for a in range(3):
            self.s.light.dir[a] = float(light.get("dir", (0, 0, 1))[a])
            self.s.light.radiance[a] = float(light.get("radiance", (1, 1, 1))[a])

    @property
    def ptr(self):
        return ctypes.byref(self.s)


def _camera(cam: dict) -> _Camera:
    c = _Camera()
    c.type = _CAMERA_TYPES[cam["type"]]
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


# ---------------------------------------------------------------- scalars
def erfcx(x: float) -> float:
    return lib().orc_erfcx(float(x))


def log_ndtr(u: float) -> float:
    return lib().orc_log_ndtr(float(u))


def inv_mills(u: float) -> float:
    return lib().orc_inv_mills(float(u))


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    out = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, out)
    return [int(v) for v in out]


def projected_area_local(w, G, ax, ay, az) -> float:
    wa, wp = _vec(w)
    return lib().orc_projected_area_local(wp, float(G), float(ax), float(ay), float(az))


def ndf_local(m, G, ax, ay, az) -> float:
    ma, mp = _vec(m)
    return lib().orc_ndf_local(mp, float(G), float(ax), float(ay), float(az))


def ndf_hf(m, kind: str, alpha) -> float:
    """Height-field macrofacet NDF (Sec. 4.1) in the frame n = z."""
    ma, mp = _vec(m)
    return lib().orc_ndf_hf(mp, NDF_KINDS[kind], float(alpha))


def projected_area_hf(w, kind: str, alpha) -> float:
    """Lambda(w) cos(theta) of a height-field macrofacet for the marching direction w."""
    wa, wp = _vec(w)
    return lib().orc_projected_area_hf(wp, NDF_KINDS[kind], float(alpha))


# ---------------------------------------------------------------- scene queries
def field(scene: Scene, k: int, x):
    xa, xp = _vec(x)
    mu, var = ctypes.c_double(), ctypes.c_double()
    g = np.zeros(3)
    al = np.zeros(3)
    ok = lib().orc_field(ctypes.byref(scene._objs[k]), xp, ctypes.byref(mu), g.ctypes.data_as(_PD),
                         ctypes.byref(var), al.ctypes.data_as(_PD))
    if not ok:
        return None
    return {"mean": mu.value, "grad": g, "var": var.value, "albedo": al}


def sigma_t(scene: Scene, pos, dirs) -> np.ndarray:
    pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
    dirs = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 3))
    out = np.empty(len(pos))
    L = lib()
    for i in range(len(pos)):
        out[i] = L.orc_sigma_t(scene.ptr, pos[i].ctypes.data_as(_PD), dirs[i].ctypes.data_as(_PD))
    return out


def phase_eval(scene: Scene, k: int, pos, d_in, d_out, R: float = 0.5):
    pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
    d_in = np.ascontiguousarray(np.asarray(d_in, dtype=np.float64).reshape(-1, 3))
    d_out = np.ascontiguousarray(np.asarray(d_out, dtype=np.float64).reshape(-1, 3))
    p = np.zeros((len(pos), 3))
    pdf = np.zeros(len(pos))
    L = lib()
    tmp = np.zeros(3)
    for i in range(len(pos)):
        v = ctypes.c_double()
        L.orc_phase_eval(scene.ptr, int(k), pos[i].ctypes.data_as(_PD), d_in[i].ctypes.data_as(_PD),
                         d_out[i].ctypes.data_as(_PD), float(R), tmp.ctypes.data_as(_PD), ctypes.byref(v))
        p[i] = tmp
        pdf[i] = v.value
    return p, pdf


def phase_sample(scene: Scene, k: int, pos, d_in, u, R: float = 0.5):
    """u: (n,3) uniforms.  Returns (d_out, weight rgb, pdf, ok)."""
    pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
    d_in = np.ascontiguousarray(np.asarray(d_in, dtype=np.float64).reshape(-1, 3))
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1, 3))
    n = len(pos)
    d2, w, pdf, ok = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n), np.zeros(n, bool)
    L = lib()
    a, b = np.zeros(3), np.zeros(3)
    for i in range(n):
        v = ctypes.c_double()
        ok[i] = bool(L.orc_phase_sample(scene.ptr, int(k), pos[i].ctypes.data_as(_PD), d_in[i].ctypes.data_as(_PD),
                                        float(R), u[i].ctypes.data_as(_PD), a.ctypes.data_as(_PD),
                                        b.ctypes.data_as(_PD), ctypes.byref(v)))
        d2[i], w[i], pdf[i] = a, b, v.value
    return d2, w, pdf, ok


def phase_sample_exact(scene: Scene, k: int, pos, d_in, u):
    """Exact visible-normal samples (GPSS objects, Beckmann height fields): returns
    (d_out, weight rgb (= F), pdf (= p/F), ok)."""
    pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
    d_in = np.ascontiguousarray(np.asarray(d_in, dtype=np.float64).reshape(-1, 3))
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1, 3))
    n = len(pos)
    d2, w, pdf, ok = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n), np.zeros(n, bool)
    L = lib()
    a, b = np.zeros(3), np.zeros(3)
    for i in range(n):
        v = ctypes.c_double()
        ok[i] = bool(L.orc_phase_sample_exact(scene.ptr, int(k), pos[i].ctypes.data_as(_PD),
                                              d_in[i].ctypes.data_as(_PD), u[i].ctypes.data_as(_PD),
                                              a.ctypes.data_as(_PD), b.ctypes.data_as(_PD), ctypes.byref(v)))
        d2[i], w[i], pdf[i] = a, b, v.value
    return d2, w, pdf, ok


def optical_depth(scene: Scene, org, d, tmax=np.inf) -> float:
    oa, op = _vec(org)
    da, dp = _vec(d)
    return lib().orc_optical_depth(scene.ptr, op, dp, float(tmax))


def transmittance(scene: Scene, org, d, tmax=np.inf) -> float:
    oa, op = _vec(org)
    da, dp = _vec(d)
    return lib().orc_transmittance(scene.ptr, op, dp, float(tmax))


def camera_ray(cam: dict, px: int, py: int, jx: float, jy: float):
    c = _camera(cam)
    o, d = np.zeros(3), np.zeros(3)
    lib().orc_camera_ray(ctypes.byref(c), int(px), int(py), float(jx), float(jy), o.ctypes.data_as(_PD),
                         d.ctypes.data_as(_PD))
    return o, d


def _opts(cam, opts, rows, cols, threads):
    o = _Opts()
    o.spp = int(opts["spp"])
    o.max_bounces = int(opts["max_bounces"])
    o.seed = int(opts.get("seed", 0))
    o.mix_R = float(opts.get("mix_R", 0.5))
    r = rows if rows is not None else (0, cam["height"], 1)
    c = cols if cols is not None else (0, cam["width"])
    o.row_begin, o.row_end, o.row_step = int(r[0]), int(r[1]), int(r[2]) if len(r) > 2 else 1
    o.col_begin, o.col_end = int(c[0]), int(c[1])
    o.threads = int(threads)
    o.sampler = {"mixture": 0, "vndf": 1}[opts.get("sampler", "mixture")]
    return o


def render(scene: Scene, cam: dict, opts: dict, rows=None, cols=None, threads: int = 0):
    """Returns (sum, sumsq, stats): per-pixel sums over samples of the path
    radiance, shape (H, W, 3), and a dict of counts."""
    H, W = int(cam["height"]), int(cam["width"])
    s = np.zeros((H, W, 3))
    s2 = np.zeros((H, W, 3))
    st = _Stats()
    c = _camera(cam)
    o = _opts(cam, opts, rows, cols, threads)
    rc = lib().orc_render(scene.ptr, ctypes.byref(c), ctypes.byref(o), s.ctypes.data_as(_PD),
                          s2.ctypes.data_as(_PD), ctypes.byref(st))
    if rc != 0:
        raise ValueError("oracle render rejected its arguments")
    return s, s2, {"paths": st.paths, "vertices": st.vertices, "truncated": st.truncated}


def render_diff(scene_a: Scene, scene_b: Scene, cam: dict, opts: dict, rows=None, cols=None, threads: int = 0):
    """Per-pixel sum and sum of squares of L_a - L_b over paths rendered with
    identical random numbers (common random numbers)."""
    H, W = int(cam["height"]), int(cam["width"])
    s = np.zeros((H, W, 3))
    s2 = np.zeros((H, W, 3))
    st = _Stats()
    c = _camera(cam)
    o = _opts(cam, opts, rows, cols, threads)
    rc = lib().orc_render_diff(scene_a.ptr, scene_b.ptr, ctypes.byref(c), ctypes.byref(o),
                               s.ctypes.data_as(_PD), s2.ctypes.data_as(_PD), ctypes.byref(st))
    if rc != 0:
        raise ValueError("oracle render rejected its arguments")
    return s, s2, {"paths": st.paths, "vertices": st.vertices, "truncated": st.truncated}


# number of derivative slots of the oracle's dual numbers and their layout
DUAL_SLOTS = 33
SLOT_MEAN, SLOT_VAR, SLOT_CS, SLOT_L, SLOT_ALB = 0, 8, 16, 24, 25
_DUAL_WHAT = {"sigma_t": 0, "projected_area": 1, "ndf": 2, "log_phase": 3}


def dual_eval(scene: Scene, k: int, what: str, x, d, d2=None):
    """The oracle's dual-number evaluation of one quantity at x in object k: returns
    (value, derivative slots (33,), corner node indices (8,)) or None where it is
    undefined (see gpss_oracle.h, orc_dual_eval)."""
    xa, xp = _vec(x)
    da, dp = _vec(d)
    d2a, d2p = _vec(d2 if d2 is not None else d)
    v = ctypes.c_double()
    der = np.zeros(DUAL_SLOTS)
    node = np.zeros(8, dtype=np.int64)
    ok = lib().orc_dual_eval(ctypes.byref(scene._objs[k]), _DUAL_WHAT[what], xp, dp, d2p, ctypes.byref(v),
                             der.ctypes.data_as(_PD), node.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if not ok:
        return None
    return v.value, der, node


def render_grad(scene: Scene, cam: dict, opts: dict, d_image, rows=None, cols=None, threads: int = 0,
                nodes=None, want=("mean", "var", "albedo", "l")):
    """The oracle's adjoint: gradient of sum(d_image * image) over the selected pixels
    with respect to each object's grids and length scale (path replay of the
    regular-tracking estimator, partials from dual numbers).  nodes: None (every
    node) or one array of node indices per object (x fastest); the outputs then
    follow that order.  Returns (list of dicts per object with the wanted keys of
    'mean', 'var', 'albedo' (channels, n), 'cscale', 'l'), stats)."""
    H, Wd = int(cam["height"]), int(cam["width"])
    g = np.ascontiguousarray(np.asarray(d_image, dtype=np.float64).reshape(H, Wd, 3))
    n_objs = scene.s.n_objs
    outs = (_GradOut * n_objs)()
    res, keep = [], []
    for k in range(n_objs):
        ob = scene._objs[k]
        N = ob.nx * ob.ny * ob.nz
        o = outs[k]
        if nodes is not None and nodes[k] is not None:
            nd = np.ascontiguousarray(np.asarray(nodes[k], dtype=np.int64))
            keep.append(nd)
            o.nodes = nd.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
            o.n_nodes = len(nd)
            n = len(nd)
        else:
            n = N
        r = {}
        for key, field, size in (("mean", "d_mean", n), ("var", "d_var", n), ("albedo", "d_albedo", n * ob.channels),
                                 ("cscale", "d_cscale", n), ("l", "d_l", 1)):
            if key in want and (key != "cscale" or bool(ob.cscale)):
                a = np.zeros(size)
                r[key] = a
                setattr(o, field, a.ctypes.data_as(_PD))
        if "albedo" in r:
            r["albedo"] = r["albedo"].reshape(ob.channels, n)
        res.append(r)
    st = _Stats()
    mism = ctypes.c_uint64()
    c = _camera(cam)
    op = _opts(cam, opts, rows, cols, threads)
    rc = lib().orc_render_grad(scene.ptr, ctypes.byref(c), ctypes.byref(op), g.ctypes.data_as(_PD), outs,
                               ctypes.byref(st), ctypes.byref(mism))
    if rc == 2:
        raise NotImplementedError("oracle adjoint: isotropic GPSS objects only")
    if rc != 0:
        raise ValueError("oracle adjoint rejected its arguments")
    for r in res:
        if "l" in r:
            r["l"] = float(r["l"][0])
    return res, {"paths": st.paths, "vertices": st.vertices, "truncated": st.truncated, "mismatch": mism.value}
