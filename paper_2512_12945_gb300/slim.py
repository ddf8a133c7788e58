"""Thin Python binding of the C ABI in include/slim_gb300.h.

Argument marshalling only: tensors are checked and passed to the library as
raw device pointers on the current torch CUDA stream; every step of the
scan-integration path runs in the CUDA library. The functions keep the C
names (slim_map_create, slim_integrate, ...); `Map` is a small owner of a
handle on top of them. Importing this module does not load the library; the
first call does, and fails loudly when it has not been built.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import build as _build

SLIM_CLOSED_ONEHOT, SLIM_CLOSED_SOFT, SLIM_OPEN, SLIM_CLOSED_LATEST = 0, 1, 2, 3
SLIM_STORE_F32, SLIM_STORE_BF16 = 0, 1
SLIM_EXTRACT_POSTERIOR = 1
AGGREGATION = {"auto": 0, "sort": 1, "hash": 2, "direct": 3}
WEIGHTING = {"constant": 0, "linear": 1}  # slim_weighting
MODES = {"onehot": SLIM_CLOSED_ONEHOT, "soft": SLIM_CLOSED_SOFT, "open": SLIM_OPEN,
         "latest": SLIM_CLOSED_LATEST}
STATUS = {0: "SLIM_OK", 1: "SLIM_ERR_ARG", 2: "SLIM_ERR_CUDA", 3: "SLIM_ERR_CAPACITY",
          4: "SLIM_ERR_TIMEOUT", 5: "SLIM_ERR_NOMEM", 6: "SLIM_ERR_UNSUPPORTED",
          7: "SLIM_ERR_INTERNAL"}


class SlimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class slim_map_params(ctypes.Structure):
    _fields_ = [("voxel_size", ctypes.c_float), ("trunc", ctypes.c_float),
                ("min_range", ctypes.c_float), ("max_range", ctypes.c_float),
                ("mode", ctypes.c_int32), ("num_classes", ctypes.c_int32),
                ("embed_dim", ctypes.c_int32), ("embed_storage", ctypes.c_int32),
                ("alpha0", ctypes.c_double), ("body_from_sensor", ctypes.c_double * 16),
                ("block_capacity", ctypes.c_int64), ("hash_capacity", ctypes.c_int64),
                ("voxel_capacity", ctypes.c_int64), ("max_points", ctypes.c_int64),
                ("aggregation", ctypes.c_int32), ("tile_points", ctypes.c_int32),
                ("weighting", ctypes.c_int32), ("weight_eps", ctypes.c_float),
                ("image_width", ctypes.c_int32), ("embed_bound", ctypes.c_float)]


class slim_stats(ctypes.Structure):
    _fields_ = [("blocks", ctypes.c_int64), ("voxels", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("scans", ctypes.c_int64),
                ("status", ctypes.c_uint32)]


class slim_batch_item(ctypes.Structure):
    _fields_ = [("map", ctypes.c_void_p), ("pts_dev", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("pose", ctypes.c_double * 16), ("sem_dev", ctypes.c_void_p)]


EXPORTS = ["slim_map_params_default", "slim_map_create", "slim_map_destroy", "slim_map_reset",
           "slim_integrate", "slim_integrate_host", "slim_map_sync", "slim_map_stats",
           "slim_extract_tsdf", "slim_query", "slim_backward", "slim_integrate_batch",
           "slim_profile_enable", "slim_profile_read", "slim_autotune", "slim_query_rows_static",
           "slim_extract_uncertainty", "slim_render", "slim_integrate_depth", "slim_record_pairs",
           "slim_backward_pairs", "slim_last_error"]
KERNELS = ["traverse", "fuse_closed", "open_tile", "open_apply", "query", "backward", "batch",
           "reset", "render"]
N_KINDS = 16

_lock = threading.Lock()
_lib = None


def library_path():
    return _build.LIB


def lib():
    """The loaded C library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with "
                              "`python -m paper_2512_12945_gb300.build` (nvcc, sm_103a)")
        L = ctypes.CDLL(path)
        P, I64, I32, F = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float
        sig = {
            "slim_map_params_default": [ctypes.POINTER(slim_map_params)],
            "slim_map_create": [ctypes.POINTER(slim_map_params), ctypes.POINTER(P)],
            "slim_map_destroy": [P],
            "slim_map_reset": [P, P],
            "slim_integrate": [P, P, I64, P, P, P],
            "slim_integrate_host": [P, P, I64, P, P, P],
            "slim_map_sync": [P, P],
            "slim_map_stats": [P, ctypes.POINTER(slim_stats), P],
            "slim_extract_tsdf": [P, P, P, P, P, P, P, I64, ctypes.POINTER(I64), I32, P],
            "slim_query": [P, P, I32, F, F, P, P, P, P],
            "slim_backward": [P, P, I64, P, P, P, P, P, P, P, P],
            "slim_integrate_batch": [ctypes.POINTER(slim_batch_item), I32, P],
            "slim_profile_enable": [P, I32],
            "slim_profile_read": [P, P, P],
            "slim_autotune": [P, P, I64, P, P, P, ctypes.POINTER(I32)],
            "slim_query_rows_static": [P, I64, I32, P, I32, F, F, P, P, P],
            "slim_extract_uncertainty": [P, P, I64, ctypes.POINTER(I64), P],
            "slim_render": [P, P, F, F, F, F, I32, I32, F, F, P, P, P, P, P, P],
            "slim_integrate_depth": [P, P, I32, I32, F, F, F, F, P, P, P],
            "slim_record_pairs": [P, P, I64, P, P, P, I64, ctypes.POINTER(I64), P],
            "slim_backward_pairs": [P, P, I64, P, P, P, P, P, P, P, P],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.slim_last_error.argtypes = []
        L.slim_last_error.restype = ctypes.c_char_p
        _lib = L
        return L


def _check(status, what):
    if status != 0:
        raise SlimError(status, f"{what}: {lib().slim_last_error().decode()}")


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, dtype, name, shape=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _pose_arr(pose):
    a = np.ascontiguousarray(np.asarray(pose, np.float64).reshape(16))
    return a, a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------- C names
def slim_map_params_default():
    p = slim_map_params()
    _check(lib().slim_map_params_default(ctypes.byref(p)), "slim_map_params_default")
    return p


def slim_map_create(params):
    h = ctypes.c_void_p()
    _check(lib().slim_map_create(ctypes.byref(params), ctypes.byref(h)), "slim_map_create")
    return h


def slim_map_destroy(h):
    _check(lib().slim_map_destroy(h), "slim_map_destroy")


def slim_map_reset(h, stream=None):
    _check(lib().slim_map_reset(h, _stream(stream)), "slim_map_reset")


def slim_integrate(h, pts, pose, sem, width, stream=None):
    n = pts.shape[0]
    p_pts = _dev_ptr(pts, torch.float32, "pts", (n, 3))
    p_sem = _dev_ptr(sem, torch.float32, "sem", (n, width))
    keep, p_pose = _pose_arr(pose)
    _check(lib().slim_integrate(h, p_pts, n, p_pose, p_sem, _stream(stream)), "slim_integrate")


def slim_integrate_depth(h, depth, fx, fy, cx, cy, pose, sem, width, stream=None):
    """depth: (H, W) float32 z-depth on the device; sem: (H*W, width)."""
    H, W = depth.shape
    keep, p_pose = _pose_arr(pose)
    _check(lib().slim_integrate_depth(h, _dev_ptr(depth, torch.float32, "depth", (H, W)), W, H,
                                      float(fx), float(fy), float(cx), float(cy), p_pose,
                                      _dev_ptr(sem, torch.float32, "sem", (H * W, width)),
                                      _stream(stream)), "slim_integrate_depth")


def slim_integrate_host(h, pts, pose, sem, width, stream=None):
    pts = pts if isinstance(pts, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(pts))
    sem = sem if isinstance(sem, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(sem))
    n = pts.shape[0]
    for t, nm, w in ((pts, "pts", 3), (sem, "sem", width)):
        if t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or \
                tuple(t.shape) != (n, w):
            raise ValueError(f"{nm} must be a contiguous host float32 tensor of shape ({n}, {w})")
    keep, p_pose = _pose_arr(pose)
    _check(lib().slim_integrate_host(h, ctypes.c_void_p(pts.data_ptr()), n, p_pose,
                                     ctypes.c_void_p(sem.data_ptr()), _stream(stream)),
           "slim_integrate_host")


def slim_map_sync(h, stream=None):
    _check(lib().slim_map_sync(h, _stream(stream)), "slim_map_sync")


def slim_map_stats(h, stream=None):
    s = slim_stats()
    _check(lib().slim_map_stats(h, ctypes.byref(s), _stream(stream)), "slim_map_stats")
    return dict(blocks=s.blocks, voxels=s.voxels, device_bytes=s.device_bytes, scans=s.scans,
                status=s.status)


def slim_extract_tsdf(h, mode, width, posterior=False, index=False, stream=None, device=None):
    n = ctypes.c_int64(0)
    st = _stream(stream)
    flags = SLIM_EXTRACT_POSTERIOR if posterior else 0
    _check(lib().slim_extract_tsdf(h, None, None, None, None, None, None, 0, ctypes.byref(n),
                                   flags, st), "slim_extract_tsdf(size)")
    cnt = n.value
    dev = device or torch.device("cuda", torch.cuda.current_device())
    out = dict(ijk=torch.empty((cnt, 3), dtype=torch.int32, device=dev),
               D=torch.empty(cnt, dtype=torch.float32, device=dev),
               W=torch.empty(cnt, dtype=torch.float32, device=dev),
               sem=torch.empty((cnt, width), dtype=torch.float32, device=dev))
    if mode == SLIM_OPEN:
        out["beta"] = torch.empty((cnt, width), dtype=torch.float32, device=dev)
    if index:
        out["index"] = torch.empty(cnt, dtype=torch.int32, device=dev)
    ptr = lambda k: ctypes.c_void_p(out[k].data_ptr()) if k in out else None  # noqa: E731
    _check(lib().slim_extract_tsdf(h, ptr("ijk"), ptr("D"), ptr("W"), ptr("sem"), ptr("beta"),
                                   ptr("index"), max(cnt, 1), ctypes.byref(n), flags, st),
           "slim_extract_tsdf")
    return out


def slim_extract_uncertainty(h, mode, width, stream=None, device=None):
    """Closed set: (n, K+1) class-probability variances + predictive entropy;
    open set: (n, l) Student-t predictive variances (inf where W <= 2)."""
    n = ctypes.c_int64(0)
    st = _stream(stream)
    _check(lib().slim_extract_uncertainty(h, None, 0, ctypes.byref(n), st),
           "slim_extract_uncertainty(size)")
    cnt = n.value
    dev = device or torch.device("cuda", torch.cuda.current_device())
    w = width if mode == SLIM_OPEN else width + 1
    unc = torch.empty((cnt, w), dtype=torch.float32, device=dev)
    _check(lib().slim_extract_uncertainty(h, ctypes.c_void_p(unc.data_ptr()), max(cnt, 1),
                                          ctypes.byref(n), st), "slim_extract_uncertainty")
    return unc


def slim_render(h, world_from_camera, fx, fy, cx, cy, width, height, near, far, q=None,
                stream=None, device=None):
    """Ray-cast render: dict of depth (H, W) float32 (+inf on a miss), ijk
    (H, W, 3) int32, label (H, W) int32 and, with a query q (open set,
    float32 l-vector on the device), sim (H, W) float32."""
    dev = device or torch.device("cuda", torch.cuda.current_device())
    depth = torch.empty((height, width), dtype=torch.float32, device=dev)
    ijk = torch.empty((height, width, 3), dtype=torch.int32, device=dev)
    label = torch.empty((height, width), dtype=torch.int32, device=dev)
    sim = torch.empty((height, width), dtype=torch.float32, device=dev) if q is not None else None
    keep, p_pose = _pose_arr(world_from_camera)
    qp = None if q is None else _dev_ptr(q, torch.float32, "q")
    _check(lib().slim_render(h, p_pose, float(fx), float(fy), float(cx), float(cy), int(width),
                             int(height), float(near), float(far), qp,
                             ctypes.c_void_p(depth.data_ptr()), ctypes.c_void_p(ijk.data_ptr()),
                             ctypes.c_void_p(label.data_ptr()),
                             None if sim is None else ctypes.c_void_p(sim.data_ptr()),
                             _stream(stream)), "slim_render")
    out = dict(depth=depth, ijk=ijk, label=label)
    if sim is not None:
        out["sim"] = sim
    return out


def slim_query(h, q_bf16, temperature, tp, n_rows, scores=False, stream=None):
    q = q_bf16
    if q.dtype != torch.bfloat16:
        raise TypeError("queries must be bfloat16")
    Q = q.shape[0]
    p_q = _dev_ptr(q.view(torch.int16), torch.int16, "q")
    dev = q.device
    label = torch.empty(n_rows, dtype=torch.int32, device=dev)
    prob = torch.empty(n_rows, dtype=torch.float32, device=dev)
    sc = torch.empty((n_rows, Q), dtype=torch.float32, device=dev) if scores else None
    _check(lib().slim_query(h, p_q, Q, float(temperature), float(tp),
                            ctypes.c_void_p(label.data_ptr()), ctypes.c_void_p(prob.data_ptr()),
                            None if sc is None else ctypes.c_void_p(sc.data_ptr()),
                            _stream(stream)), "slim_query")
    return label, prob, sc


def slim_query_rows_static(rows_bf16, q_bf16, temperature=0.01, tp=0.1, label=None, prob=None,
                           stream=None):
    """Read-out over caller-held BF16 rows with no device allocation inside
    the library (outputs may be passed in, preallocated)."""
    if rows_bf16.dtype != torch.bfloat16 or q_bf16.dtype != torch.bfloat16:
        raise TypeError("rows and queries must be bfloat16")
    n, l = rows_bf16.shape
    Q = q_bf16.shape[0]
    dev = rows_bf16.device
    if label is None:
        label = torch.empty(n, dtype=torch.int32, device=dev)
    if prob is None:
        prob = torch.empty(n, dtype=torch.float32, device=dev)
    _check(lib().slim_query_rows_static(
        _dev_ptr(rows_bf16.view(torch.int16), torch.int16, "rows"), n, l,
        _dev_ptr(q_bf16.view(torch.int16), torch.int16, "q"), Q, float(temperature), float(tp),
        _dev_ptr(label, torch.int32, "label", (n,)), _dev_ptr(prob, torch.float32, "prob", (n,)),
        _stream(stream)), "slim_query_rows_static")
    return label, prob


def slim_backward(h, pts, pose, sem, gD, gS, gB, width, stream=None):
    n = pts.shape[0]
    dev = pts.device
    gsem = torch.empty((n, width), dtype=torch.float32, device=dev)
    gxyz = torch.empty((n, 3), dtype=torch.float32, device=dev)
    keep, p_pose = _pose_arr(pose)
    _check(lib().slim_backward(h, _dev_ptr(pts, torch.float32, "pts", (n, 3)), n, p_pose,
                               _dev_ptr(sem, torch.float32, "sem", (n, width)),
                               _dev_ptr(gD, torch.float32, "gD"),
                               _dev_ptr(gS, torch.float32, "gS"),
                               _dev_ptr(gB, torch.float32, "gB"),
                               ctypes.c_void_p(gsem.data_ptr()), ctypes.c_void_p(gxyz.data_ptr()),
                               _stream(stream)), "slim_backward")
    return gsem, gxyz


def slim_record_pairs(h, pts, pose, stream=None):
    """The stored pair list of one scan of the map: (offsets int32 [n + 1],
    voxel indices int32 [pairs]), CSR by point (size query, then the list)."""
    n = pts.shape[0]
    dev = pts.device
    offsets = torch.empty(n + 1, dtype=torch.int32, device=dev)
    keep, p_pose = _pose_arr(pose)
    pp = _dev_ptr(pts, torch.float32, "pts", (n, 3))
    total = ctypes.c_int64(0)
    _check(lib().slim_record_pairs(h, pp, n, p_pose, ctypes.c_void_p(offsets.data_ptr()), None, 0,
                                   ctypes.byref(total), _stream(stream)), "slim_record_pairs")
    vox = torch.empty(max(total.value, 1), dtype=torch.int32, device=dev)
    _check(lib().slim_record_pairs(h, pp, n, p_pose, ctypes.c_void_p(offsets.data_ptr()),
                                   ctypes.c_void_p(vox.data_ptr()), vox.numel(),
                                   ctypes.byref(total), _stream(stream)), "slim_record_pairs")
    return offsets, vox[:total.value]


def slim_backward_pairs(h, pts, pose, offsets, vox, gD, gS, width, stream=None):
    n = pts.shape[0]
    dev = pts.device
    gsem = torch.empty((n, width), dtype=torch.float32, device=dev)
    gxyz = torch.empty((n, 3), dtype=torch.float32, device=dev)
    keep, p_pose = _pose_arr(pose)
    _check(lib().slim_backward_pairs(h, _dev_ptr(pts, torch.float32, "pts", (n, 3)), n, p_pose,
                                     _dev_ptr(offsets, torch.int32, "offsets", (n + 1,)),
                                     ctypes.c_void_p(vox.data_ptr()),
                                     _dev_ptr(gD, torch.float32, "gD"),
                                     _dev_ptr(gS, torch.float32, "gS"),
                                     ctypes.c_void_p(gsem.data_ptr()),
                                     ctypes.c_void_p(gxyz.data_ptr()), _stream(stream)),
           "slim_backward_pairs")
    return gsem, gxyz


def slim_profile_enable(h, on):
    _check(lib().slim_profile_enable(h, int(bool(on))), "slim_profile_enable")


def slim_profile_read(h):
    """{kernel name: (launches, total ms)} since the last read."""
    n = (ctypes.c_int64 * N_KINDS)()
    ms = (ctypes.c_double * N_KINDS)()
    _check(lib().slim_profile_read(h, n, ms), "slim_profile_read")
    return {KERNELS[k]: (int(n[k]), float(ms[k])) for k in range(len(KERNELS)) if n[k]}


def slim_autotune(h, pts, pose, sem, width, stream=None):
    n = pts.shape[0]
    keep, p_pose = _pose_arr(pose)
    best = ctypes.c_int32(0)
    _check(lib().slim_autotune(h, _dev_ptr(pts, torch.float32, "pts", (n, 3)), n, p_pose,
                               _dev_ptr(sem, torch.float32, "sem", (n, width)), _stream(stream),
                               ctypes.byref(best)), "slim_autotune")
    return best.value


def slim_integrate_batch(items, stream=None):
    """items: list of (Map, pts, pose, sem)."""
    arr = (slim_batch_item * max(len(items), 1))()
    for k, (m, pts, pose, sem) in enumerate(items):
        n = pts.shape[0]
        arr[k].map = m.handle
        arr[k].pts_dev = _dev_ptr(pts, torch.float32, "pts", (n, 3))
        arr[k].n = n
        for j, v in enumerate(np.asarray(pose, np.float64).reshape(16)):
            arr[k].pose[j] = float(v)
        arr[k].sem_dev = _dev_ptr(sem, torch.float32, "sem", (n, m.width))
    _check(lib().slim_integrate_batch(arr, len(items), _stream(stream)), "slim_integrate_batch")


# ------------------------------------------------------------------ owner
class Map:
    """One map on the current CUDA device."""

    def __init__(self, voxel_size=0.1, trunc=0.3, mode="onehot", num_classes=20, embed_dim=512,
                 embed_storage="f32", min_range=0.0, max_range=1e30, alpha0=1.0,
                 body_from_sensor=None, block_capacity=100000, hash_capacity=262144,
                 voxel_capacity=1000000, max_points=1 << 18, aggregation="auto",
                 tile_points=0, weighting="constant", weight_eps=0.0, image_width=0,
                 embed_bound=1.0):
        p = slim_map_params_default()
        p.voxel_size = voxel_size
        p.trunc = trunc
        p.min_range = min_range
        p.max_range = max_range
        p.mode = MODES[mode] if isinstance(mode, str) else int(mode)
        p.num_classes = num_classes
        p.embed_dim = embed_dim
        p.embed_storage = SLIM_STORE_BF16 if embed_storage in ("bf16", SLIM_STORE_BF16) else \
            SLIM_STORE_F32
        p.alpha0 = alpha0
        ext = np.eye(4) if body_from_sensor is None else np.asarray(body_from_sensor, np.float64)
        for k, v in enumerate(ext.reshape(16)):
            p.body_from_sensor[k] = float(v)
        p.block_capacity = block_capacity
        p.hash_capacity = hash_capacity
        p.voxel_capacity = voxel_capacity
        p.max_points = max_points
        p.aggregation = AGGREGATION[aggregation] if isinstance(aggregation, str) else aggregation
        p.tile_points = tile_points
        p.weighting = WEIGHTING[weighting] if isinstance(weighting, str) else int(weighting)
        p.weight_eps = weight_eps
        p.image_width = image_width
        p.embed_bound = embed_bound
        self.params = p
        self.mode = p.mode
        self.width = embed_dim if p.mode == SLIM_OPEN else num_classes
        self.handle = slim_map_create(p)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            slim_map_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, stream=None):
        slim_map_reset(self.handle, stream)

    def integrate(self, pts, pose, sem, stream=None):
        slim_integrate(self.handle, pts, pose, sem, self.width, stream)

    def integrate_depth(self, depth, fx, fy, cx, cy, pose, sem, stream=None):
        slim_integrate_depth(self.handle, depth, fx, fy, cx, cy, pose, sem, self.width, stream)

    def integrate_host(self, pts, pose, sem, stream=None):
        slim_integrate_host(self.handle, pts, pose, sem, self.width, stream)

    def sync(self, stream=None):
        slim_map_sync(self.handle, stream)

    def stats(self, stream=None):
        return slim_map_stats(self.handle, stream)

    def extract(self, posterior=False, index=False, stream=None):
        return slim_extract_tsdf(self.handle, self.mode, self.width, posterior, index, stream)

    def render(self, world_from_camera, fx, fy, cx, cy, width, height, near, far, q=None,
               stream=None):
        return slim_render(self.handle, world_from_camera, fx, fy, cx, cy, width, height, near,
                           far, q, stream)

    def uncertainty(self, stream=None):
        return slim_extract_uncertainty(self.handle, self.mode, self.width, stream)

    def query(self, q_bf16, temperature=0.01, tp=0.1, scores=False, stream=None):
        rows = self.stats(stream)["voxels"]
        return slim_query(self.handle, q_bf16, temperature, tp, rows, scores, stream)

    def autotune(self, pts, pose, sem, stream=None):
        return slim_autotune(self.handle, pts, pose, sem, self.width, stream)

    def backward(self, pts, pose, sem, gD, gS, gB=None, stream=None):
        return slim_backward(self.handle, pts, pose, sem, gD, gS, gB, self.width, stream)

    def record_pairs(self, pts, pose, stream=None):
        return slim_record_pairs(self.handle, pts, pose, stream)

    def backward_pairs(self, pts, pose, offsets, vox, gD, gS, stream=None):
        return slim_backward_pairs(self.handle, pts, pose, offsets, vox, gD, gS, self.width,
                                   stream)
