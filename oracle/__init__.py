"""The oracle: TEST INFRASTRUCTURE, not part of the product path.

A plain, slow, sequential CPU implementation of SLIM-VDB scan integration
(arXiv 2512.12945; Sec. III-A, Theorem 1 / Eq. alpha_update, Eq. dir_to_cat,
Theorem 2 / Eqs. norm_update_1-4 with the Sec. III-D simplification
lambda = 2 nu = W, and the open-set cosine / softmax / T_p read-out). The
arithmetic lives in ``slim_oracle.cpp``; this module only builds it and
marshals numpy arrays. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it. It shares no code with the
CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "slim_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CLOSED_ONEHOT, CLOSED_SOFT, OPEN, CLOSED_LATEST = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with strict IEEE float semantics (no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("voxel_size", ctypes.c_float), ("trunc", ctypes.c_float),
                ("min_range", ctypes.c_float), ("max_range", ctypes.c_float),
                ("mode", ctypes.c_int32), ("num_classes", ctypes.c_int32),
                ("embed_dim", ctypes.c_int32), ("fp64_geometry", ctypes.c_int32),
                ("alpha0", ctypes.c_double),
                ("body_from_sensor", ctypes.c_double * 16),
                ("weighting", ctypes.c_int32), ("weight_eps", ctypes.c_float)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.ora_create.restype = P
            lib.ora_create.argtypes = [ctypes.POINTER(_Params)]
            lib.ora_destroy.argtypes = [P]
            lib.ora_integrate.restype = ctypes.c_int64
            lib.ora_integrate.argtypes = [P, P, ctypes.c_int64, P, P]
            lib.ora_scan_pairs.restype = ctypes.c_int64
            lib.ora_scan_pairs.argtypes = [ctypes.POINTER(_Params), P, ctypes.c_int64, P,
                                           P, P, P, ctypes.c_int64]
            lib.ora_point_visits.restype = ctypes.c_int64
            lib.ora_point_visits.argtypes = [ctypes.POINTER(_Params), P, P, P, ctypes.c_int64]
            lib.ora_count.restype = ctypes.c_int64
            lib.ora_count.argtypes = [P]
            lib.ora_extract.restype = ctypes.c_int64
            lib.ora_extract.argtypes = [P, P, P, P, P, P, ctypes.c_int32]
            lib.ora_uncertainty.restype = ctypes.c_int64
            lib.ora_uncertainty.argtypes = [P, P]
            F = ctypes.c_float
            lib.ora_integrate_depth.restype = ctypes.c_int64
            lib.ora_integrate_depth.argtypes = [P, P, ctypes.c_int32, ctypes.c_int32, F, F, F, F,
                                                P, P]
            lib.ora_render.restype = ctypes.c_int64
            lib.ora_render.argtypes = [P, P, F, F, F, F, ctypes.c_int32, ctypes.c_int32, F, F,
                                       P, P, P, P, P]
            lib.ora_pixel_visits.restype = ctypes.c_int64
            lib.ora_pixel_visits.argtypes = [F, P, F, F, F, F, ctypes.c_int32, ctypes.c_int32,
                                             F, F, P, ctypes.c_int64]
            lib.ora_query.restype = None
            lib.ora_query.argtypes = [P, ctypes.c_int64, ctypes.c_int32, P, ctypes.c_int32,
                                      ctypes.c_double, ctypes.c_double, P, P, P]
            lib.ora_backward_scan.restype = ctypes.c_int64
            lib.ora_backward_scan.argtypes = [P, P, ctypes.c_int64, P, P, P, P, P, P, P]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a, cols=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if cols is not None:
        a = a.reshape(-1, cols)
    return a


def _pose(pose):
    return np.ascontiguousarray(np.asarray(pose, dtype=np.float64).reshape(16))


def make_params(voxel_size, trunc, mode=CLOSED_ONEHOT, num_classes=0, embed_dim=0,
                min_range=0.0, max_range=1e30, alpha0=1.0, fp64_geometry=False,
                body_from_sensor=None, weighting=0, weight_eps=0.0):
    """weighting 0: w~ = 1 (Sec. III-A); 1: linear decay behind the surface
    (w~ = 1 for d >= -weight_eps, (tau + d) / (tau - weight_eps) below),
    closed-set modes only."""
    p = _Params()
    p.voxel_size = voxel_size
    p.trunc = trunc
    p.min_range = min_range
    p.max_range = max_range
    p.mode = mode
    p.num_classes = num_classes
    p.embed_dim = embed_dim
    p.fp64_geometry = int(bool(fp64_geometry))
    p.alpha0 = alpha0
    p.weighting = int(weighting)
    p.weight_eps = float(weight_eps)
    ext = np.eye(4) if body_from_sensor is None else np.asarray(body_from_sensor, np.float64)
    for k, val in enumerate(ext.reshape(16)):
        p.body_from_sensor[k] = float(val)
    return p


def sem_width(p):
    return p.embed_dim if p.mode == OPEN else p.num_classes


class OracleMap:
    """One map held by the oracle: integrate scans, then extract or query."""

    def __init__(self, **kw):
        self.lib = _load()
        self.params = make_params(**kw)
        self.h = self.lib.ora_create(ctypes.byref(self.params))
        if not self.h:
            raise ValueError("unsupported oracle parameters (weighting applies to the closed "
                             "set, with 0 <= weight_eps < trunc)")
        self.w = sem_width(self.params)

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.ora_destroy(self.h)
            self.h = None

    def integrate(self, pts, pose, sem):
        pts = _f32(pts, 3)
        sem = _f32(sem, self.w)
        assert sem.shape[0] == pts.shape[0]
        pose = _pose(pose)
        return self.lib.ora_integrate(self.h, _ptr(pts), pts.shape[0], _ptr(pose), _ptr(sem))

    def integrate_depth(self, depth, fx, fy, cx, cy, pose, sem):
        """One row-major z-depth image (H, W) float32 with per-pixel semantics
        (H*W, w); returns the number of valid points."""
        depth = np.ascontiguousarray(depth, np.float32)
        h, w = depth.shape
        sem = _f32(sem, self.w)
        assert sem.shape[0] == h * w
        return self.lib.ora_integrate_depth(self.h, _ptr(depth), w, h, fx, fy, cx, cy,
                                            _ptr(_pose(pose)), _ptr(sem))

    def count(self):
        return self.lib.ora_count(self.h)

    def extract(self, posterior=False):
        """Dict of ijk (n,3) int32, D, W (n,) f64, sem (n,w) f64 [, beta (n,w)]."""
        n = self.count()
        ijk = np.zeros((n, 3), np.int32)
        D = np.zeros(n)
        W = np.zeros(n)
        sem = np.zeros((n, self.w))
        beta = np.zeros((n, self.w)) if self.params.mode == OPEN else None
        self.lib.ora_extract(self.h, _ptr(ijk), _ptr(D), _ptr(W), _ptr(sem), _ptr(beta),
                             int(bool(posterior)))
        out = dict(ijk=ijk, D=D, W=W, sem=sem)
        if beta is not None:
            out["beta"] = beta
        return out

    def uncertainty(self):
        """Closed set: (n, K+1) Dirichlet class-probability variances and the
        posterior-predictive entropy; open set: (n, l) Student-t predictive
        variances (+inf where W <= 2). Same voxel order as extract()."""
        n = self.count()
        w = self.w + 1 if self.params.mode != OPEN else self.w
        unc = np.zeros((n, w))
        self.lib.ora_uncertainty(self.h, _ptr(unc))
        return unc

    def render(self, world_from_camera, fx, fy, cx, cy, width, height, near, far, q=None):
        """Ray-cast render from a pinhole camera: dict of depth (H, W) f64
        (+inf on a miss), ijk (H, W, 3) int32 of the voxel after the zero
        crossing (INT32_MIN on a miss), label (H, W) int32 (closed set), and
        sim (H, W) f64 (open set with a query q)."""
        depth = np.zeros((height, width))
        ijk = np.zeros((height, width, 3), np.int32)
        label = np.zeros((height, width), np.int32)
        sim = np.zeros((height, width))
        qq = None if q is None else _f32(q).reshape(-1)
        self.lib.ora_render(self.h, _ptr(_pose(world_from_camera)), fx, fy, cx, cy, width,
                            height, near, far, None if qq is None else _ptr(qq), _ptr(depth),
                            _ptr(ijk), _ptr(label), _ptr(sim))
        return dict(depth=depth, ijk=ijk, label=label, sim=sim)

    def backward_scan(self, pts, pose, sem, gD, gS, gB=None):
        """Per-point dL/dsem (n,w) and dL/dxyz (n,3); call extract() first."""
        pts = _f32(pts, 3)
        sem = _f32(sem, self.w)
        pose = _pose(pose)
        gD = np.ascontiguousarray(gD, np.float64)
        gS = np.ascontiguousarray(gS, np.float64)
        gB = None if gB is None else np.ascontiguousarray(gB, np.float64)
        n = pts.shape[0]
        gsem = np.zeros((n, self.w))
        gxyz = np.zeros((n, 3))
        rc = self.lib.ora_backward_scan(self.h, _ptr(pts), n, _ptr(pose), _ptr(sem), _ptr(gD),
                                        _ptr(gS), _ptr(gB), _ptr(gsem), _ptr(gxyz))
        if rc == -2:
            raise RuntimeError("ora_backward_scan: the adjoint is for w~ = 1 maps")
        if rc != 0:
            raise RuntimeError("ora_backward_scan: extract() must be called first")
        return gsem, gxyz


def scan_pairs(params, pts, pose):
    """All (voxel ijk, point index, d) observations of one scan."""
    lib = _load()
    pts = _f32(pts, 3)
    pose = _pose(pose)
    n = lib.ora_scan_pairs(ctypes.byref(params), _ptr(pts), pts.shape[0], _ptr(pose),
                           None, None, None, 0)
    ijk = np.zeros((n, 3), np.int32)
    pt = np.zeros(n, np.int64)
    d = np.zeros(n)
    lib.ora_scan_pairs(ctypes.byref(params), _ptr(pts), pts.shape[0], _ptr(pose),
                       _ptr(ijk), _ptr(pt), _ptr(d), n)
    return ijk, pt, d


def point_visits(params, pt, pose):
    """Voxels the band DDA of one point enters, or None for an invalid point."""
    lib = _load()
    pt = _f32(pt).reshape(3)
    pose = _pose(pose)
    cap = 256
    ijk = np.zeros((cap, 3), np.int32)
    n = lib.ora_point_visits(ctypes.byref(params), _ptr(pt), _ptr(pose), _ptr(ijk), cap)
    if n < 0:
        return None
    assert n <= cap
    return ijk[:n].copy()


def pixel_visits(voxel_size, world_from_camera, fx, fy, cx, cy, px, py, near, far):
    """Voxels the render ray of pixel (px, py) enters, in order."""
    lib = _load()
    cap = 1 << 16
    ijk = np.zeros((cap, 3), np.int32)
    n = lib.ora_pixel_visits(voxel_size, _ptr(_pose(world_from_camera)), fx, fy, cx, cy, px, py,
                             near, far, _ptr(ijk), cap)
    assert n <= cap
    return ijk[:n].copy()


def query(rows, q, temperature, tp):
    """Open-set read-out: (label int32, prob f64, cosine f64 (n,Q))."""
    lib = _load()
    rows = np.ascontiguousarray(rows, np.float64)
    q = _f32(q)
    n, l = rows.shape
    Q = q.shape[0]
    assert q.shape[1] == l
    label = np.zeros(n, np.int32)
    prob = np.zeros(n)
    cos = np.zeros((n, Q))
    lib.ora_query(_ptr(rows), n, l, _ptr(q), Q, float(temperature), float(tp),
                  _ptr(label), _ptr(prob), _ptr(cos))
    return label, prob, cos
