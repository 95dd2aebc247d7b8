"""Python front end of the multi-volume TSDF library: torch tensors in, C ABI calls out.

``Mapper`` owns one ``mv_ctx``.  It only marshals arguments (device pointers
of torch tensors, the current CUDA stream, poses as float64) to the functions
of ``include/mvtsdf.h``; every step of integration and raycasting runs in
``libmvtsdf.so``.  Paper: Salvato, Finman, Leonard, arXiv 1511.07106.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import _abi
from ._abi import MVError


@dataclass
class Config:
    """Method parameters; see mv_config in include/mvtsdf.h."""
    trunc_voxels: float = 4.0
    w_max: float = 128.0
    color_w_max: int = 255
    z_min: float = 0.0
    z_max: float = float("inf")
    ray_step: float = 1.0
    n_bisect: int = 8

    def _c(self):
        return _abi.mv_config(self.trunc_voxels, self.w_max, int(self.color_w_max), self.z_min,
                              self.z_max, self.ray_step, int(self.n_bisect))


def intrinsics(cam) -> "_abi.mv_intrinsics":
    return _abi.mv_intrinsics(float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy),
                              int(cam.width), int(cam.height))


def _pose(T):
    a = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(16))
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def _dptr(t, dtype=None, numel=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


def decode(raw: np.ndarray, fmt: int):
    """Raw per-voxel storage (as returned by read_volume) -> (F, W) float64."""
    if fmt == _abi.MV_TSDF_F32:
        return raw[..., 0].astype(np.float64), raw[..., 1].astype(np.float64)
    lo = (raw & 0xFFFF).astype(np.uint16)
    W = (raw >> 16).astype(np.float64)
    if fmt == _abi.MV_TSDF_F16:
        F = lo.view(np.float16).astype(np.float64)
    else:
        F = lo.view(np.int16).astype(np.float64) / 32767.0
    return F, W


def encode(F: np.ndarray, W: np.ndarray, fmt: int) -> np.ndarray:
    """(F, W) -> raw per-voxel storage (inverse of decode up to the format's rounding)."""
    if fmt == _abi.MV_TSDF_F32:
        return np.stack([F, W], -1).astype(np.float32)
    Wq = np.clip(np.rint(W), 0, 65535).astype(np.uint32)
    if fmt == _abi.MV_TSDF_F16:
        lo = np.asarray(F, np.float16).view(np.uint16).astype(np.uint32)
    else:
        lo = np.clip(np.rint(np.asarray(F, np.float64) * 32767.0), -32767, 32767).astype(np.int16)
        lo = lo.view(np.uint16).astype(np.uint32)
    return (lo | (Wq << 16)).astype(np.uint32)


class Mapper:
    """A set of TSDF subvolumes on one GPU (the paper's set H)."""

    def __init__(self, config: Optional[Config] = None, device: int = 0):
        self._lib = _abi.lib()
        self.config = config or Config()
        cfg = self.config._c()
        h = C.c_void_p()
        st = self._lib.mv_create(C.byref(cfg), int(device), C.byref(h))
        if st != _abi.MV_OK:
            raise MVError(st, "mv_create failed")
        self._h = h
        self.device = device
        self._fmt = {}

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.mv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st):
        if st != _abi.MV_OK:
            msg = self._lib.mv_last_error(self._h)
            raise MVError(st, msg.decode() if msg else "")

    # -- volumes ----------------------------------------------------------
    def add_volume(self, h_t, h_r, voxel_size: float, fmt="f32") -> int:
        f = _abi.FORMATS[fmt] if isinstance(fmt, str) else int(fmt)
        d = _abi.mv_volume_desc((C.c_int32 * 3)(*[int(a) for a in h_t]),
                                (C.c_int32 * 3)(*[int(a) for a in h_r]), float(voxel_size), f)
        out = C.c_int32()
        self._check(self._lib.mv_add_volume(self._h, C.byref(d), C.byref(out)))
        self._fmt[out.value] = f
        return out.value

    def reserve_host(self, h_r, fmt="f32", count=2):
        """Pin `count` spare host buffer sets now for volumes of h_r voxels (see
        mv_reserve_host)."""
        f = _abi.FORMATS[fmt] if isinstance(fmt, str) else int(fmt)
        d = _abi.mv_volume_desc((C.c_int32 * 3)(0, 0, 0), (C.c_int32 * 3)(*[int(a) for a in h_r]), 1.0, f)
        self._check(self._lib.mv_reserve_host(self._h, C.byref(d), int(count)))

    def remove_volume(self, vid: int):
        self._check(self._lib.mv_remove_volume(self._h, int(vid)))
        self._fmt.pop(vid, None)

    def query(self, vid: int) -> dict:
        info = _abi.mv_volume_info()
        self._check(self._lib.mv_query(self._h, int(vid), C.byref(info)))
        d = info.desc
        return dict(h_t=tuple(d.h_t), h_r=tuple(d.h_r), voxel_size=d.voxel_size, fmt=d.fmt,
                    resident=bool(info.resident), device_bytes=info.device_bytes,
                    host_bytes=info.host_bytes)

    def volumes(self) -> list:
        n = C.c_int32()
        self._check(self._lib.mv_list_volumes(self._h, None, 0, C.byref(n)))
        ids = (C.c_int32 * max(n.value, 1))()
        self._check(self._lib.mv_list_volumes(self._h, ids, n.value, C.byref(n)))
        return list(ids[: n.value])

    # -- per frame --------------------------------------------------------
    def integrate(self, depth, rgb, cam, T, stream=None):
        """Integrate one frame into every resident volume (one batched pass)."""
        import torch
        K = intrinsics(cam)
        n = cam.width * cam.height
        _, Tp = keep = _pose(T)
        self._check(self._lib.mv_integrate(
            self._h, _dptr(depth, torch.float32, n, "depth"), _dptr(rgb, torch.uint8, 3 * n, "rgb"),
            C.byref(K), Tp, _stream(stream)))
        del keep

    def integrate_volume(self, vid, depth, rgb, cam, T, stream=None):
        import torch
        K = intrinsics(cam)
        n = cam.width * cam.height
        _, Tp = keep = _pose(T)
        self._check(self._lib.mv_integrate_volume(
            self._h, int(vid), _dptr(depth, torch.float32, n, "depth"),
            _dptr(rgb, torch.uint8, 3 * n, "rgb"), C.byref(K), Tp, _stream(stream)))
        del keep

    def alloc_maps(self, cam, vertex=True):
        import torch
        dev = torch.device("cuda", self.device)
        H, W = cam.height, cam.width
        out = dict(depth=torch.empty((H, W), dtype=torch.float32, device=dev),
                   normal=torch.empty((H, W, 3), dtype=torch.float32, device=dev),
                   rgba=torch.empty((H, W, 4), dtype=torch.uint8, device=dev),
                   vol_id=torch.empty((H, W), dtype=torch.int32, device=dev))
        if vertex:
            out["vertex"] = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
        return out

    def _map_ptrs(self, out, cam):
        import torch
        n = cam.width * cam.height
        return (_dptr(out.get("depth"), torch.float32, n, "depth"),
                _dptr(out.get("normal"), torch.float32, 3 * n, "normal"),
                _dptr(out.get("rgba"), torch.uint8, 4 * n, "rgba"),
                _dptr(out.get("vertex"), torch.float32, 3 * n, "vertex"),
                _dptr(out.get("vol_id"), torch.int32, n, "vol_id"))

    def raycast(self, cam, T, out=None, stream=None) -> dict:
        """Raycast all resident volumes into depth/normal/rgba/vertex/vol_id maps."""
        out = out if out is not None else self.alloc_maps(cam)
        K = intrinsics(cam)
        _, Tp = keep = _pose(T)
        self._check(self._lib.mv_raycast(self._h, C.byref(K), Tp, *self._map_ptrs(out, cam),
                                         _stream(stream)))
        del keep
        return out

    def raycast_batch(self, cam, poses, out=None, stream=None) -> dict:
        """Raycast n views (poses: (n, 4, 4) host) in one launch
        (mv_raycast_batch); out: maps with a leading view axis, e.g. depth
        (n, H, W) -- each may be missing; default depth, rgba and vol_id."""
        import torch
        P = np.ascontiguousarray(np.asarray(poses, np.float64).reshape(-1, 16))
        n = P.shape[0]
        if out is None:
            dev = torch.device("cuda", self.device)
            H, W = cam.height, cam.width
            out = dict(depth=torch.empty((n, H, W), dtype=torch.float32, device=dev),
                       rgba=torch.empty((n, H, W, 4), dtype=torch.uint8, device=dev),
                       vol_id=torch.empty((n, H, W), dtype=torch.int32, device=dev))
        K = intrinsics(cam)
        px = n * cam.width * cam.height
        self._check(self._lib.mv_raycast_batch(
            self._h, C.byref(K), P.ctypes.data_as(C.POINTER(C.c_double)), n,
            _dptr(out.get("depth"), torch.float32, px, "depth"), _dptr(out.get("normal"), torch.float32, 3 * px, "normal"),
            _dptr(out.get("rgba"), torch.uint8, 4 * px, "rgba"), _dptr(out.get("vertex"), torch.float32, 3 * px, "vertex"),
            _dptr(out.get("vol_id"), torch.int32, px, "vol_id"), _stream(stream)))
        return out

    def frame(self, depth, rgb, cam, T, out=None, stream=None) -> dict:
        """Integrate the frame and raycast the same view, as one CUDA graph."""
        import torch
        out = out if out is not None else self.alloc_maps(cam)
        K = intrinsics(cam)
        n = cam.width * cam.height
        _, Tp = keep = _pose(T)
        self._check(self._lib.mv_frame(self._h, _dptr(depth, torch.float32, n, "depth"),
                                       _dptr(rgb, torch.uint8, 3 * n, "rgb"), C.byref(K), Tp,
                                       *self._map_ptrs(out, cam), _stream(stream)))
        del keep
        return out

    def alloc_host_maps(self, cam, vertex=False, vol_id=False):
        """Page-locked host maps for frame_host: depth, normal, rgba (and
        optionally vertex, vol_id)."""
        import torch
        H, W = cam.height, cam.width
        out = {"depth": torch.empty((H, W), dtype=torch.float32).pin_memory(),
               "normal": torch.empty((H, W, 3), dtype=torch.float32).pin_memory(),
               "rgba": torch.empty((H, W, 4), dtype=torch.uint8).pin_memory()}
        if vertex:
            out["vertex"] = torch.empty((H, W, 3), dtype=torch.float32).pin_memory()
        if vol_id:
            out["vol_id"] = torch.empty((H, W), dtype=torch.int32).pin_memory()
        return out

    def frame_host(self, depth, rgb, cam, T, out) -> int:
        """mv_frame_host: host depth (H, W) float32 and rgb (H, W, 3) uint8 (or
        None) in, host maps (dict of CPU tensors or numpy arrays, from
        alloc_host_maps) out.  Asynchronous; returns the ticket for
        frame_host_wait.  Every buffer must stay alive until that wait."""
        K = intrinsics(cam)
        _, Tp = keep = _pose(T)
        n = cam.width * cam.height

        def hp(a, numel, name, dtype):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                if a.is_cuda or not a.is_contiguous() or a.numel() != numel or str(a.dtype) != dtype:
                    raise ValueError(f"{name} must be a contiguous CPU {dtype} tensor of {numel} elements")
                return C.c_void_p(a.data_ptr())
            if not a.flags["C_CONTIGUOUS"] or a.size != numel or str(a.dtype) != dtype.split(".")[-1]:
                raise ValueError(f"{name} must be a contiguous {dtype} array of {numel} elements")
            return C.c_void_p(a.ctypes.data)

        ticket = C.c_uint64()
        self._check(self._lib.mv_frame_host(
            self._h, hp(depth, n, "depth", "torch.float32"), hp(rgb, 3 * n, "rgb", "torch.uint8"), C.byref(K), Tp,
            hp(out.get("depth"), n, "depth_out", "torch.float32"),
            hp(out.get("normal"), 3 * n, "normal", "torch.float32"),
            hp(out.get("rgba"), 4 * n, "rgba", "torch.uint8"),
            hp(out.get("vertex"), 3 * n, "vertex", "torch.float32"),
            hp(out.get("vol_id"), n, "vol_id", "torch.int32"), C.byref(ticket)))
        del keep
        return int(ticket.value)

    def frame_host_wait(self, ticket: int):
        self._check(self._lib.mv_frame_host_wait(self._h, C.c_uint64(int(ticket))))

    def frame_streamed(self, depth, rgb, cam, T, out=None, n_slots=2, stream=None) -> dict:
        """Integrate the frame into every volume and raycast the same view,
        streaming the swapped-out volumes through n_slots device slots."""
        import torch
        out = out if out is not None else self.alloc_maps(cam)
        K = intrinsics(cam)
        n = cam.width * cam.height
        _, Tp = keep = _pose(T)
        self._check(self._lib.mv_frame_streamed(self._h, _dptr(depth, torch.float32, n, "depth"),
                                                _dptr(rgb, torch.uint8, 3 * n, "rgb"), C.byref(K), Tp,
                                                *self._map_ptrs(out, cam), int(n_slots), _stream(stream)))
        del keep
        return out

    def extract_points(self, vid, cap=None, rgb=True, edges=True, stream=None) -> dict:
        """Surface points of a resident volume: {"xyz": (n, 3) float32,
        "rgb": (n, 3) uint8, "edge": (n,) int64} as CUDA tensors (unordered)."""
        import torch
        dev = torch.device("cuda", self.device)
        if cap is None:  # a first guess; grown to the exact count if too small
            cap = int(np.prod(self.query(vid)["h_r"])) // 16 + 4096
        while True:
            xyz = torch.empty((max(cap, 1), 3), dtype=torch.float32, device=dev)
            col = torch.empty((max(cap, 1), 3), dtype=torch.uint8, device=dev) if rgb else None
            edge = torch.empty(max(cap, 1), dtype=torch.int64, device=dev) if edges else None
            n = C.c_uint64(0)
            st = self._lib.mv_extract_points(self._h, int(vid), C.c_void_p(xyz.data_ptr()),
                                             C.c_void_p(col.data_ptr()) if rgb else None,
                                             C.c_void_p(edge.data_ptr()) if edges else None, int(cap),
                                             C.byref(n), _stream(stream))
            if st == _abi.MV_ERR_CAPACITY:
                cap = int(n.value)
                continue
            self._check(st)
            k = int(n.value)
            out = {"xyz": xyz[:k]}
            if rgb:
                out["rgb"] = col[:k]
            if edges:
                out["edge"] = edge[:k]
            return out

    # -- tracking -------------------------------------------------------------
    def depth_to_maps(self, depth, cam, T=None, stream=None):
        """(vertex, normal) float32 CUDA tensors (H, W, 3) of a depth frame;
        world frame with T, camera frame without."""
        import torch
        dev = torch.device("cuda", self.device)
        n = cam.width * cam.height
        v = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device=dev)
        nn = torch.empty_like(v)
        K = intrinsics(cam)
        if T is None:
            Tp, keep = None, None
        else:
            keep = _pose(T)
            Tp = keep[1]
        self._check(self._lib.mv_depth_to_maps(self._h, _dptr(depth, torch.float32, n, "depth"), C.byref(K), Tp,
                                               C.c_void_p(v.data_ptr()), C.c_void_p(nn.data_ptr()),
                                               _stream(stream)))
        del keep
        return v, nn

    @staticmethod
    def _icp_cfg(iterations, dist, cos_min):
        return _abi.mv_icp_config(int(iterations), float(dist), float(cos_min))

    @staticmethod
    def _icp_out(r):
        return {"A": np.array(r.A[:]).reshape(6, 6), "b": np.array(r.b[:]), "error": r.error, "count": r.inliers}

    def icp_linearize(self, vertex, normal, cam, T_est, model_vertex, model_normal, T_model, dist=0.1,
                      cos_min=0.8, stream=None) -> dict:
        """One point-to-plane linearisation (see mv_icp_linearize)."""
        import torch
        n = 3 * cam.width * cam.height
        r = _abi.mv_icp_system()
        cfg = self._icp_cfg(1, dist, cos_min)
        ke, Te = _pose(T_est)
        km, Tm = _pose(T_model)
        self._check(self._lib.mv_icp_linearize(
            self._h, _dptr(vertex, torch.float32, n, "vertex"), _dptr(normal, torch.float32, n, "normal"),
            C.byref(intrinsics(cam)), Te, _dptr(model_vertex, torch.float32, n, "model_vertex"),
            _dptr(model_normal, torch.float32, n, "model_normal"), Tm, C.byref(cfg), C.byref(r), _stream(stream)))
        del ke, km
        return self._icp_out(r)

    def track(self, depth, cam, model_vertex, model_normal, T_model, T_init, iterations=10, dist=0.1,
              cos_min=0.8, stream=None):
        """Track a depth frame against model maps: (T (4, 4) float64, last system)."""
        import torch
        n = cam.width * cam.height
        r = _abi.mv_icp_system()
        cfg = self._icp_cfg(iterations, dist, cos_min)
        km, Tm = _pose(T_model)
        ki, Ti = _pose(T_init)
        out = np.zeros(16)
        self._check(self._lib.mv_track(
            self._h, _dptr(depth, torch.float32, n, "depth"), C.byref(intrinsics(cam)),
            _dptr(model_vertex, torch.float32, 3 * n, "model_vertex"),
            _dptr(model_normal, torch.float32, 3 * n, "model_normal"), Tm, Ti, C.byref(cfg),
            out.ctypes.data_as(C.POINTER(C.c_double)), C.byref(r), _stream(stream)))
        del km, ki
        return out.reshape(4, 4), self._icp_out(r)

    def raycast_volume(self, vid, first, cam, T, out, stream=None) -> dict:
        K = intrinsics(cam)
        _, Tp = keep = _pose(T)
        self._check(self._lib.mv_raycast_volume(self._h, int(vid), int(bool(first)), C.byref(K), Tp,
                                                *self._map_ptrs(out, cam), _stream(stream)))
        del keep
        return out

    def raycast_backward(self, cam, poses, depth, vol_id, grad_depth, grad_rgb, grad_pose,
                         targets=None, stream=None):
        """Raycast gradients (see mv_raycast_backward).  poses: (n, 4, 4) host
        float64; depth/vol_id: (n, H, W) device maps of the forward; grad_pose
        (n, 6) float32 device output; targets: {volume id: float32 device
        tensor shaped like the volume} receiving += dL/dF."""
        import torch
        P = np.ascontiguousarray(np.asarray(poses, np.float64).reshape(-1, 16))
        n = P.shape[0]
        npx = n * cam.width * cam.height
        K = intrinsics(cam)
        targets = targets or {}
        arr = (_abi.mv_grad_target * max(len(targets), 1))()
        for i, (vid, t) in enumerate(targets.items()):
            arr[i] = _abi.mv_grad_target(int(vid), _dptr(t, torch.float32, None, "grad_tsdf").value)
        self._check(self._lib.mv_raycast_backward(
            self._h, C.byref(K), P.ctypes.data_as(C.POINTER(C.c_double)), n,
            _dptr(depth, torch.float32, npx, "depth"), _dptr(vol_id, torch.int32, npx, "vol_id"),
            _dptr(grad_depth, torch.float32, npx, "grad_depth"),
            _dptr(grad_rgb, torch.float32, 3 * npx, "grad_rgb"),
            _dptr(grad_pose, torch.float32, 6 * n, "grad_pose"), arr, len(targets), _stream(stream)))

    def raycast_backward_l1(self, cam, poses, depth, rgba, vol_id, ref_depth, ref_rgba, colour_weight,
                            grad_pose, loss, stream=None):
        """The L1 loss of pose refinement and its pose gradient in one call
        (mv_raycast_backward_l1).  poses: (n, 4, 4) host float64; depth (n, H,
        W) float32, rgba (n, H, W, 4) uint8 and vol_id (n, H, W) int32: the
        forward's maps; ref_depth / ref_rgba: the reference renders, same
        shapes; grad_pose (n, 6) float32 and loss (1,) float32: device
        outputs."""
        import torch
        P = np.ascontiguousarray(np.asarray(poses, np.float64).reshape(-1, 16))
        n = P.shape[0]
        npx = n * cam.width * cam.height
        K = intrinsics(cam)
        self._check(self._lib.mv_raycast_backward_l1(
            self._h, C.byref(K), P.ctypes.data_as(C.POINTER(C.c_double)), n,
            _dptr(depth, torch.float32, npx, "depth"), _dptr(rgba, torch.uint8, 4 * npx, "rgba"),
            _dptr(vol_id, torch.int32, npx, "vol_id"), _dptr(ref_depth, torch.float32, npx, "ref_depth"),
            _dptr(ref_rgba, torch.uint8, 4 * npx, "ref_rgba"), float(colour_weight),
            _dptr(grad_pose, torch.float32, 6 * n, "grad_pose"), _dptr(loss, torch.float32, 1, "loss"),
            _stream(stream)))

    # -- memory passing ---------------------------------------------------
    def swap_out(self, vid, stream=None):
        self._check(self._lib.mv_swap_out(self._h, int(vid), _stream(stream)))

    def swap_in(self, vid, stream=None):
        self._check(self._lib.mv_swap_in(self._h, int(vid), _stream(stream)))

    def read_volume(self, vid, rgba=True):
        """Synchronous read -> (raw storage [z,y,x,...], rgba [z,y,x,4] or None)."""
        q = self.query(vid)
        rx, ry, rz = q["h_r"]
        if q["fmt"] == _abi.MV_TSDF_F32:
            raw = np.empty((rz, ry, rx, 2), np.float32)
        else:
            raw = np.empty((rz, ry, rx), np.uint32)
        col = np.empty((rz, ry, rx, 4), np.uint8) if rgba else None
        self._check(self._lib.mv_read_volume(self._h, int(vid), raw.ctypes.data_as(C.c_void_p),
                                             None if col is None else col.ctypes.data_as(C.c_void_p)))
        return raw, col

    def read_box(self, vid, lo, n, rgba=True):
        """Synchronous read of the voxel box lo .. lo + n - 1 (x, y, z) ->
        (raw storage [z, y, x, ...], rgba [z, y, x, 4] or None)."""
        q = self.query(vid)
        nx, ny, nz = (int(a) for a in n)
        if q["fmt"] == _abi.MV_TSDF_F32:
            raw = np.empty((nz, ny, nx, 2), np.float32)
        else:
            raw = np.empty((nz, ny, nx), np.uint32)
        col = np.empty((nz, ny, nx, 4), np.uint8) if rgba else None
        lo3 = (C.c_int32 * 3)(*(int(a) for a in lo))
        n3 = (C.c_int32 * 3)(nx, ny, nz)
        self._check(self._lib.mv_read_box(self._h, int(vid), lo3, n3, raw.ctypes.data_as(C.c_void_p),
                                          None if col is None else col.ctypes.data_as(C.c_void_p)))
        return raw, col

    def read_box_decoded(self, vid, lo, n):
        """read_box -> (F, W, rgba) with F, W as float64 [z, y, x]."""
        raw, col = self.read_box(vid, lo, n)
        F, W = decode(raw, self.query(vid)["fmt"])
        return F, W, col

    def read_decoded(self, vid):
        """Synchronous read -> (F, W, rgba) with F, W as float64 [z, y, x]."""
        raw, col = self.read_volume(vid)
        F, W = decode(raw, self.query(vid)["fmt"])
        return F, W, col

    def read_brick_flags(self, vid):
        """Per-brick summary flags [nbz, nby, nbx] (bit 0 observed-positive, bit 1 unobserved)."""
        q = self.query(vid)
        nb = [(r + 7) // 8 for r in q["h_r"]]
        out = np.empty((nb[2], nb[1], nb[0]), np.uint8)
        self._check(self._lib.mv_read_brick_flags(self._h, int(vid), out.ctypes.data_as(C.c_void_p),
                                                  C.c_uint64(out.size)))
        return out

    def write_volume(self, vid, raw, rgba=None):
        raw = np.ascontiguousarray(raw)
        col = None if rgba is None else np.ascontiguousarray(rgba, np.uint8)
        self._check(self._lib.mv_write_volume(self._h, int(vid), raw.ctypes.data_as(C.c_void_p),
                                              None if col is None else col.ctypes.data_as(C.c_void_p)))

    def write_decoded(self, vid, F, W, rgba=None):
        self.write_volume(vid, encode(np.asarray(F), np.asarray(W), self.query(vid)["fmt"]), rgba)

    # -- misc ---------------------------------------------------------------
    def stats(self, reset=False) -> dict:
        s = _abi.mv_stats()
        self._check(self._lib.mv_get_stats(self._h, C.byref(s), int(bool(reset))))
        return {k: getattr(s, k) for k, _ in _abi.mv_stats._fields_}

    def autotune(self, depth, rgb, cam, T, stream=None) -> dict:
        """Time the raycast tile shapes and integration grid sizes on this
        frame (the map is not modified) and keep the fastest."""
        import torch
        K = intrinsics(cam)
        n = cam.width * cam.height
        t = _abi.mv_tuning()
        _, Tp = keep = _pose(T)
        self._check(self._lib.mv_autotune(self._h, _dptr(depth, torch.float32, n, "depth"),
                                          _dptr(rgb, torch.uint8, 3 * n, "rgb"), C.byref(K), Tp,
                                          C.byref(t), _stream(stream)))
        del keep
        return dict(raycast_tile=t.raycast_tile, integrate_ctas_per_sm=t.integrate_ctas_per_sm,
                    raycast_ms=list(t.raycast_ms), integrate_ms=list(t.integrate_ms))

    def set_tuning(self, raycast_tile: int, integrate_ctas_per_sm: int, work_list_levels: int = None):
        """Launch shapes; work_list_levels (0 automatic, 1, 2) is kept when None."""
        t = _abi.mv_tuning()
        self._check(self._lib.mv_get_tuning(self._h, C.byref(t)))
        t.raycast_tile, t.integrate_ctas_per_sm = int(raycast_tile), int(integrate_ctas_per_sm)
        if work_list_levels is not None:
            t.work_list_levels = int(work_list_levels)
        self._check(self._lib.mv_set_tuning(self._h, C.byref(t)))

    def tuning(self) -> dict:
        t = _abi.mv_tuning()
        self._check(self._lib.mv_get_tuning(self._h, C.byref(t)))
        return dict(raycast_tile=t.raycast_tile, integrate_ctas_per_sm=t.integrate_ctas_per_sm,
                    work_list_levels=t.work_list_levels)

    def set_timing(self, enable: bool):
        self._check(self._lib.mv_set_timing(self._h, int(bool(enable))))

    def timings(self, reset=False) -> dict:
        """{kernel: (launches, summed ms, timed launches)} since the last reset."""
        t = _abi.mv_timings()
        self._check(self._lib.mv_get_timings(self._h, C.byref(t), int(bool(reset))))
        return {name: (t.launches[k], t.ms[k], t.timed[k]) for k, name in _abi.KERNEL_NAMES.items()}

    def synchronize(self):
        self._check(self._lib.mv_synchronize(self._h))


class Placer:
    """Dynamic volume placement on a Mapper (the paper's top-n cells of ray
    endpoints, with hysteresis): see mv_placer_* in include/mvtsdf.h."""

    def __init__(self, mapper: Mapper, cell_voxels: int, volume_voxels: int, voxel_size: float,
                 max_volumes: int, hysteresis: float = 1.5, min_count: int = 1, fmt="f32"):
        self._lib = mapper._lib
        self.mapper = mapper
        f = _abi.FORMATS[fmt] if isinstance(fmt, str) else int(fmt)
        cfg = _abi.mv_placement_config(int(cell_voxels), int(volume_voxels), float(voxel_size), f,
                                       int(max_volumes), float(hysteresis), int(min_count))
        h = C.c_void_p()
        st = self._lib.mv_placer_create(mapper._h, C.byref(cfg), C.byref(h))
        if st != _abi.MV_OK:
            raise MVError(st, "mv_placer_create failed")
        self._h = h
        self.cell_voxels = int(cell_voxels)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mv_placer_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != _abi.MV_OK:
            msg = self._lib.mv_placer_last_error(self._h)
            raise MVError(st, msg.decode() if msg else "")

    def histogram(self, depth, cam, T, cap=None, stream=None) -> dict:
        """c(l) of one frame as {(x, y, z): count}."""
        import torch
        n = cam.width * cam.height
        cap = n if cap is None else int(cap)
        cells = np.zeros((max(cap, 1), 3), np.int32)
        counts = np.zeros(max(cap, 1), np.uint32)
        m = C.c_int32(0)
        K = intrinsics(cam)
        _, Tp = keep = _pose(T)
        self._check(self._lib.mv_placer_histogram(
            self._h, _dptr(depth, torch.float32, n, "depth"), C.byref(K), Tp,
            cells.ctypes.data_as(C.POINTER(C.c_int32)), counts.ctypes.data_as(C.POINTER(C.c_uint32)),
            cap, C.byref(m), _stream(stream)))
        del keep
        return {tuple(int(v) for v in cells[i]): int(counts[i]) for i in range(m.value)}

    def update(self, depth, cam, T, stream=None) -> dict:
        """One insertion / removal step on this frame's depth."""
        import torch
        n = cam.width * cam.height
        r = _abi.mv_placement_result()
        K = intrinsics(cam)
        _, Tp = keep = _pose(T)
        self._check(self._lib.mv_placer_update(self._h, _dptr(depth, torch.float32, n, "depth"), C.byref(K),
                                               Tp, C.byref(r), _stream(stream)))
        del keep
        return {k: getattr(r, k) for k, _ in _abi.mv_placement_result._fields_}

    def volumes(self) -> list:
        """[(id, (x, y, z) cell, resident)] by increasing id."""
        m = C.c_int32(0)
        self._check(self._lib.mv_placer_list(self._h, None, None, None, 0, C.byref(m)))
        n = max(m.value, 1)
        ids = np.zeros(n, np.int32)
        cells = np.zeros((n, 3), np.int32)
        res = np.zeros(n, np.int32)
        self._check(self._lib.mv_placer_list(self._h, ids.ctypes.data_as(C.POINTER(C.c_int32)),
                                             cells.ctypes.data_as(C.POINTER(C.c_int32)),
                                             res.ctypes.data_as(C.POINTER(C.c_int32)), n, C.byref(m)))
        return [(int(ids[i]), tuple(int(v) for v in cells[i]), bool(res[i])) for i in range(m.value)]
