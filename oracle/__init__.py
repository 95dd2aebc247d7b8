"""FP64 CPU oracle for multi-volume TSDF integration and raycasting.

TEST INFRASTRUCTURE ONLY: the parity reference the CUDA library is checked
against.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` import this package; the library never does, and this package
imports nothing from the library.  The arithmetic lives in
``mvtsdf_oracle.c`` (plain C, double precision, one voxel / one ray at a time,
following the paper's steps); this module only marshals numpy arrays.

Paper: Salvato, Finman, Leonard, "Multi-Volume High Resolution RGB-D Mapping
with Dynamic Volume Placement", arXiv 1511.07106 -- Sec. Volumetric
Integration, Sec. Raycasting, Algorithm 1, Sec. Comparison to KinectFusion.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "mvtsdf_oracle.c")]
_LIB = os.path.join(_HERE, "liboracle_mvtsdf.so")

# per-voxel integration flags (decision within a margin of its threshold)
IF_Z, IF_PIX, IF_GATE, IF_BAND = 1, 2, 4, 8
# per-pixel raycast flags
RF_SIGN, RF_CELL, RF_RANGE, RF_FACE, RF_TIE, RF_GRAD = 1, 2, 4, 8, 16, 32
# pixels excluded from raycast gradients
GX_NOHIT, GX_CELL, GX_FACE, GX_GRAZE = 1, 2, 4, 8


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) into an in-tree shared object."""
    srcs = [s for s in _SRC if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-fopenmp",
                               "-o", tmp, *srcs, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Volume(C.Structure):
    _fields_ = [("h", C.c_int32 * 3), ("r", C.c_int32 * 3), ("s", C.c_double),
                ("F", C.POINTER(C.c_double)), ("W", C.POINTER(C.c_double)),
                ("rgba", C.POINTER(C.c_uint8))]


class _Intr(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("width", C.c_int32), ("height", C.c_int32)]


class _Cfg(C.Structure):
    _fields_ = [("trunc_vox", C.c_double), ("w_max", C.c_double), ("color_w_max", C.c_int32),
                ("z_min", C.c_double), ("z_max", C.c_double), ("step_vox", C.c_double),
                ("eps_px", C.c_double), ("eps_sdf", C.c_double), ("eps_z", C.c_double),
                ("eps_f", C.c_double), ("eps_q", C.c_double), ("eps_tau", C.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        dp, u8p, i64p, i32p = (C.POINTER(C.c_double), C.POINTER(C.c_uint8),
                               C.POINTER(C.c_int64), C.POINTER(C.c_int32))
        fp = C.POINTER(C.c_float)
        _lib.orc_integrate.argtypes = [C.POINTER(_Volume), fp, u8p, C.POINTER(_Intr), dp,
                                       C.POINTER(_Cfg), u8p, i64p]
        _lib.orc_integrate_voxels.argtypes = [C.POINTER(_Volume), i64p, C.c_int64, fp, u8p,
                                              C.POINTER(_Intr), dp, C.POINTER(_Cfg), u8p, i64p]
        _lib.orc_raycast.argtypes = [C.POINTER(_Volume), i32p, C.c_int32, C.POINTER(_Intr), dp,
                                     C.POINTER(_Cfg), dp, dp, u8p, dp, i32p, u8p]
        _lib.orc_raycast_pixels.argtypes = [C.POINTER(_Volume), i32p, C.c_int32, C.POINTER(_Intr),
                                            dp, C.POINTER(_Cfg), i64p, C.c_int64, dp, dp, u8p, dp,
                                            i32p, u8p]
        _lib.orc_raycast_footprint.argtypes = [C.POINTER(_Volume), C.c_int32, C.POINTER(_Intr), dp,
                                               C.POINTER(_Cfg), i64p, C.c_int64, i64p]
        _lib.orc_raycast_footprint.restype = C.c_int
        _lib.orc_sample.argtypes = [C.POINTER(_Volume), dp, i32p]
        _lib.orc_sample.restype = C.c_double
        _lib.orc_raycast_grad.argtypes = [C.POINTER(_Volume), i32p, C.c_int32, C.POINTER(_Intr),
                                          dp, C.POINTER(_Cfg), dp, dp, dp, dp, dp, dp,
                                          C.POINTER(C.POINTER(C.c_double)), u8p]
        _lib.orc_raycast_grad_pixels.argtypes = (_lib.orc_raycast_grad.argtypes[:6] + [i64p, C.c_int64] +
                                                 _lib.orc_raycast_grad.argtypes[6:])
        _lib.orc_endpoint_cells.argtypes = [fp, C.POINTER(_Intr), dp, C.c_double, C.c_double, C.c_double,
                                            i64p, u8p]
        _lib.orc_extract_points.argtypes = [C.POINTER(_Volume), dp, u8p, i64p, C.c_int64]
        _lib.orc_extract_points.restype = C.c_int64
        _lib.orc_threads.restype = C.c_int
        _lib.orc_set_threads.argtypes = [C.c_int]
        _lib.orc_depth_maps.argtypes = [fp, C.POINTER(_Intr), dp, C.c_double, C.c_double, dp, dp]
        _lib.orc_icp_system.argtypes = [dp, dp, C.POINTER(_Intr), dp, fp, fp, dp, C.c_double, C.c_double,
                                        dp, dp, dp, i64p, u8p, dp, dp, dp]
    return _lib


@dataclass
class Config:
    """Method parameters (the paper leaves all of them unstated)."""
    trunc_vox: float = 4.0
    w_max: float = 128.0
    color_w_max: int = 255
    z_min: float = 0.0
    z_max: float = float("inf")
    step_vox: float = 1.0
    eps_px: float = 1e-3
    eps_sdf: float = 1e-3
    eps_z: float = 1e-5
    eps_f: float = 1e-4
    eps_q: float = 1e-3
    eps_tau: float = 1e-3

    def _c(self) -> _Cfg:
        return _Cfg(self.trunc_vox, self.w_max, int(self.color_w_max), self.z_min, self.z_max,
                    self.step_vox, self.eps_px, self.eps_sdf, self.eps_z, self.eps_f, self.eps_q,
                    self.eps_tau)


@dataclass
class Volume:
    """One TSDF (sub)volume: lattice offset h (voxels), dims r, pitch s.

    Arrays are indexed [z, y, x].  F is the TSDF in units of the truncation
    distance, W the weight, rgba the colour with the colour weight in A."""
    h: tuple
    r: tuple
    s: float
    F: np.ndarray = field(default=None)
    W: np.ndarray = field(default=None)
    rgba: np.ndarray = field(default=None)

    def __post_init__(self):
        rx, ry, rz = (int(v) for v in self.r)
        if self.F is None:
            self.F = np.zeros((rz, ry, rx), np.float64)
        if self.W is None:
            self.W = np.zeros((rz, ry, rx), np.float64)
        if self.rgba is None:
            self.rgba = np.zeros((rz, ry, rx, 4), np.uint8)
        self.F = np.ascontiguousarray(self.F, np.float64)
        self.W = np.ascontiguousarray(self.W, np.float64)
        self.rgba = np.ascontiguousarray(self.rgba, np.uint8)
        assert self.F.shape == (rz, ry, rx) and self.W.shape == (rz, ry, rx)
        assert self.rgba.shape == (rz, ry, rx, 4)

    def _c(self) -> _Volume:
        v = _Volume()
        v.h[:] = [int(a) for a in self.h]
        v.r[:] = [int(a) for a in self.r]
        v.s = float(self.s)
        v.F = self.F.ctypes.data_as(C.POINTER(C.c_double))
        v.W = self.W.ctypes.data_as(C.POINTER(C.c_double))
        v.rgba = self.rgba.ctypes.data_as(C.POINTER(C.c_uint8))
        return v

    def copy(self) -> "Volume":
        return Volume(tuple(self.h), tuple(self.r), self.s, self.F.copy(), self.W.copy(),
                      self.rgba.copy())


def _intr(cam) -> _Intr:
    return _Intr(float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy), int(cam.width),
                 int(cam.height))


def _pose(T) -> np.ndarray:
    T = np.ascontiguousarray(np.asarray(T, np.float64).reshape(4, 4))
    return T


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def integrate(vol: Volume, depth, rgb, cam, T, cfg: Config = Config(), want_flags: bool = False):
    """Integrate one frame into ``vol`` in place.  Returns (counts, flags):
    counts = [updated voxels, colour-band voxels]; flags = per-voxel IF_* bits
    (or None)."""
    lib = _load()
    depth = np.ascontiguousarray(depth, np.float32)
    assert depth.shape == (cam.height, cam.width)
    rgb = None if rgb is None else np.ascontiguousarray(rgb, np.uint8)
    T = _pose(T)
    flags = np.zeros(vol.F.shape, np.uint8) if want_flags else None
    counts = np.zeros(2, np.int64)
    cv, ci, cc = vol._c(), _intr(cam), cfg._c()
    lib.orc_integrate(C.byref(cv), _ptr(depth, C.c_float), _ptr(rgb, C.c_uint8), C.byref(ci),
                      _ptr(T, C.c_double), C.byref(cc), _ptr(flags, C.c_uint8),
                      _ptr(counts, C.c_int64))
    return counts, flags


def integrate_voxels(vol: Volume, idx, depth, rgb, cam, T, cfg: Config = Config()):
    """Integrate one frame into the listed voxels only (linear x-fastest
    indices).  Returns (counts, flags over the whole volume; only the listed
    voxels are written)."""
    lib = _load()
    idx = np.ascontiguousarray(idx, np.int64)
    depth = np.ascontiguousarray(depth, np.float32)
    rgb = None if rgb is None else np.ascontiguousarray(rgb, np.uint8)
    T = _pose(T)
    flags = np.zeros(vol.F.shape, np.uint8)
    counts = np.zeros(2, np.int64)
    cv, ci, cc = vol._c(), _intr(cam), cfg._c()
    lib.orc_integrate_voxels(C.byref(cv), _ptr(idx, C.c_int64), C.c_int64(idx.size),
                             _ptr(depth, C.c_float), _ptr(rgb, C.c_uint8), C.byref(ci),
                             _ptr(T, C.c_double), C.byref(cc), _ptr(flags, C.c_uint8),
                             _ptr(counts, C.c_int64))
    return counts, flags


def raycast(vols, cam, T, cfg: Config = Config(), ids=None, pixels=None):
    """Raycast all volumes into one map.  Returns a dict of numpy arrays:
    depth (H,W) [0 = no hit], normal (H,W,3), rgba (H,W,4), vertex (H,W,3),
    vol (H,W) [-1 = no hit], flags (H,W) RF_* bits.  With ``pixels`` (linear
    indices y*W + x) only those pixels are computed; the rest stay 0."""
    lib = _load()
    vols = list(vols)
    n = len(vols)
    ids = np.arange(n, dtype=np.int32) if ids is None else np.ascontiguousarray(ids, np.int32)
    arr = (_Volume * max(n, 1))()
    for i, v in enumerate(vols):
        arr[i] = v._c()
    H, W = int(cam.height), int(cam.width)
    out = dict(depth=np.zeros((H, W)), normal=np.zeros((H, W, 3)), rgba=np.zeros((H, W, 4), np.uint8),
               vertex=np.zeros((H, W, 3)), vol=np.zeros((H, W), np.int32),
               flags=np.zeros((H, W), np.uint8))
    T = _pose(T)
    ci, cc = _intr(cam), cfg._c()
    outs = (_ptr(out["depth"], C.c_double), _ptr(out["normal"], C.c_double),
            _ptr(out["rgba"], C.c_uint8), _ptr(out["vertex"], C.c_double),
            _ptr(out["vol"], C.c_int32), _ptr(out["flags"], C.c_uint8))
    if pixels is None:
        lib.orc_raycast(arr, _ptr(ids, C.c_int32), C.c_int32(n), C.byref(ci), _ptr(T, C.c_double),
                        C.byref(cc), *outs)
    else:
        pix = np.ascontiguousarray(pixels, np.int64)
        lib.orc_raycast_pixels(arr, _ptr(ids, C.c_int32), C.c_int32(n), C.byref(ci),
                               _ptr(T, C.c_double), C.byref(cc), _ptr(pix, C.c_int64),
                               C.c_int64(pix.size), *outs)
    return out


def raycast_footprint(vols, cam, T, cfg: Config = Config(), pixels=None):
    """The voxels a dense march of this view must read (Sec. Raycasting: every
    sample of every ray until its zero crossing, in every volume): per volume
    (distinct voxels whose TSDF and weight are read -- the 2x2x2 neighbourhoods
    of the samples and bisection midpoints --, distinct voxels whose colour the
    hits read).  With ``pixels`` (linear indices) only those rays count."""
    lib = _load()
    vols = list(vols)
    n = len(vols)
    arr = (_Volume * max(n, 1))()
    for i, v in enumerate(vols):
        arr[i] = v._c()
    counts = np.zeros(2 * max(n, 1), np.int64)
    T = _pose(T)
    ci, cc = _intr(cam), cfg._c()
    pix = None if pixels is None else np.ascontiguousarray(pixels, np.int64)
    rc = lib.orc_raycast_footprint(arr, C.c_int32(n), C.byref(ci), _ptr(T, C.c_double), C.byref(cc),
                                   None if pix is None else _ptr(pix, C.c_int64),
                                   C.c_int64(0 if pix is None else pix.size), _ptr(counts, C.c_int64))
    if rc != 0:
        raise MemoryError("raycast_footprint: bitmap allocation failed")
    return [(int(counts[2 * i]), int(counts[2 * i + 1])) for i in range(n)]


def sample(vol: Volume, q):
    """Trilinear TSDF value and validity at voxel coordinates q (x, y, z)."""
    lib = _load()
    qa = np.ascontiguousarray(q, np.float64)
    valid = C.c_int32(0)
    cv = vol._c()
    val = lib.orc_sample(C.byref(cv), _ptr(qa, C.c_double), C.byref(valid))
    return float(val), bool(valid.value)


def raycast_grad(vols, cam, T, grad_depth=None, grad_rgb=None, cfg: Config = Config(), ids=None,
                 want_tsdf=True, pixels=None):
    """Gradients of the raycast (left se(3) pose perturbation xi = (rho, phi)
    in the world frame, and the TSDF voxel values).  grad_depth (H, W) and
    grad_rgb (H, W, 3; colour in [0, 1]) are the upstream gradients (None =
    0).  Returns dict: depth, grad_pose (6,), jac_tau (H, W, 6), jac_rgb
    (H, W, 3, 6), grad_F (list of arrays like each volume's F, or None),
    excluded (H, W) GX_* bits.  With ``pixels`` (linear indices y*W + x,
    ascending) only those pixels are computed and summed; the rest stay 0."""
    lib = _load()
    vols = list(vols)
    n = len(vols)
    ids = np.arange(n, dtype=np.int32) if ids is None else np.ascontiguousarray(ids, np.int32)
    arr = (_Volume * max(n, 1))()
    for i, v in enumerate(vols):
        arr[i] = v._c()
    H, W = int(cam.height), int(cam.width)
    gd = None if grad_depth is None else np.ascontiguousarray(grad_depth, np.float64)
    gc = None if grad_rgb is None else np.ascontiguousarray(grad_rgb, np.float64)
    out = dict(depth=np.zeros((H, W)), grad_pose=np.zeros(6), jac_tau=np.zeros((H, W, 6)),
               jac_rgb=np.zeros((H, W, 3, 6)), excluded=np.zeros((H, W), np.uint8))
    gF = [np.zeros_like(v.F) for v in vols] if want_tsdf else None
    ptrs = (C.POINTER(C.c_double) * max(n, 1))()
    if gF is not None:
        for i, g in enumerate(gF):
            ptrs[i] = g.ctypes.data_as(C.POINTER(C.c_double))
    T = _pose(T)
    ci, cc = _intr(cam), cfg._c()
    outs = (_ptr(out["depth"], C.c_double), _ptr(gd, C.c_double), _ptr(gc, C.c_double),
            _ptr(out["grad_pose"], C.c_double), _ptr(out["jac_tau"], C.c_double),
            _ptr(out["jac_rgb"], C.c_double), ptrs if gF is not None else None,
            _ptr(out["excluded"], C.c_uint8))
    if pixels is None:
        lib.orc_raycast_grad(arr, _ptr(ids, C.c_int32), C.c_int32(n), C.byref(ci), _ptr(T, C.c_double),
                             C.byref(cc), *outs)
    else:
        pix = np.ascontiguousarray(pixels, np.int64)
        lib.orc_raycast_grad_pixels(arr, _ptr(ids, C.c_int32), C.c_int32(n), C.byref(ci), _ptr(T, C.c_double),
                                    C.byref(cc), _ptr(pix, C.c_int64), C.c_int64(pix.size), *outs)
    out["grad_F"] = gF
    return out


def se3_exp(xi):
    """exp of a twist xi = (rho, phi) as a 4x4 matrix (Rodrigues + V rho)."""
    rho, phi = np.asarray(xi[:3], np.float64), np.asarray(xi[3:], np.float64)
    th = np.linalg.norm(phi)
    Px = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    if th < 1e-12:
        Rm = np.eye(3) + Px
        V = np.eye(3) + 0.5 * Px
    else:
        a, b = np.sin(th) / th, (1 - np.cos(th)) / th ** 2
        cc = (th - np.sin(th)) / th ** 3
        Rm = np.eye(3) + a * Px + b * Px @ Px
        V = np.eye(3) + b * Px + cc * Px @ Px
    E = np.eye(4)
    E[:3, :3], E[:3, 3] = Rm, V @ rho
    return E


# ---------------------------------------------------------------------------
# Dynamic placement (Sec. Dynamic Mapping for SLAM)
# ---------------------------------------------------------------------------
def endpoint_cells(depth, cam, T, cell_m, z_min=0.0, z_max=np.inf, f32_intrinsics=True):
    """Per pixel: the lattice cell (int64 x, y, z) of the ray endpoint
    e = T (D K^-1 [x, y, 1]^T), and whether the depth is valid.  With
    f32_intrinsics the intrinsics are first rounded to float32, the precision
    in which the library receives them."""
    lib = _load()
    depth = np.ascontiguousarray(depth, np.float32)
    H, W = depth.shape
    k = [float(np.float32(v)) if f32_intrinsics else float(v) for v in (cam.fx, cam.fy, cam.cx, cam.cy)]
    K = _Intr(k[0], k[1], k[2], k[3], int(cam.width), int(cam.height))
    Tm = _pose(T)
    cells = np.zeros((H, W, 3), np.int64)
    valid = np.zeros((H, W), np.uint8)
    lib.orc_endpoint_cells(_ptr(depth, C.c_float), C.byref(K), _ptr(Tm, C.c_double), float(z_min),
                           float(z_max), float(cell_m), _ptr(cells, C.c_int64), _ptr(valid, C.c_uint8))
    return cells, valid.astype(bool)


def endpoint_histogram(depth, cam, T, cell_m, z_min=0.0, z_max=np.inf):
    """c(l): the number of valid pixels whose endpoint falls in cell l, as a
    dict {(x, y, z): count}."""
    cells, valid = endpoint_cells(depth, cam, T, cell_m, z_min, z_max)
    keys, counts = np.unique(cells[valid], axis=0, return_counts=True)
    return {tuple(int(v) for v in k): int(c) for k, c in zip(keys, counts)}


@dataclass
class PlacementState:
    """Placed volumes by lattice cell: resident ones, and those moved out."""
    resident: set = field(default_factory=set)
    evicted: set = field(default_factory=set)


def place(state: PlacementState, hist: dict, max_volumes: int, hysteresis: float, min_count: int = 1):
    """One insertion/removal step (Sec. Insertion and Removal, Sec. Dynamic
    Mapping for SLAM): keep the cells with the largest counts c(l), at most
    max_volumes resident; a cell that is not resident enters while a slot is
    free, otherwise only by displacing the resident cell with the lowest count
    when its own count exceeds that count times `hysteresis`.  Candidates are
    taken by decreasing count, ties by increasing (z, y, x); the displaced cell
    is the resident one with the lowest count, ties by increasing (z, y, x).
    Returns (added, restored, evicted) lists of cells and updates `state`."""
    def order(cell):
        return (cell[2], cell[1], cell[0])

    count = lambda cell: hist.get(cell, 0)
    cands = [c for c in hist if hist[c] >= min_count and c not in state.resident]
    cands.sort(key=lambda c: (-hist[c],) + order(c))
    added, restored, evicted = [], [], []

    def enter(cell):
        if cell in state.evicted:
            state.evicted.discard(cell)
            restored.append(cell)
        else:
            added.append(cell)
        state.resident.add(cell)

    i = 0
    while i < len(cands) and len(state.resident) < max_volumes:
        enter(cands[i])
        i += 1
    for cell in cands[i:]:
        if not state.resident:
            break
        low = min(state.resident, key=lambda c: (count(c),) + order(c))
        if not count(cell) > hysteresis * count(low):
            break
        state.resident.discard(low)
        state.evicted.add(low)
        evicted.append(low)
        enter(cell)
    return added, restored, evicted


# ---------------------------------------------------------------------------
# Surface points (Sec. Insertion and Removal; Table 1 vertex counts)
# ---------------------------------------------------------------------------
def extract_points(vol: "Volume") -> dict:
    """Zero crossings of the TSDF along voxel edges: {"xyz" (n, 3) float64,
    "rgb" (n, 3) uint8, "edge" (n,) int64}, by increasing edge id."""
    lib = _load()
    cv = vol._c()
    n = lib.orc_extract_points(C.byref(cv), None, None, None, 0)
    xyz = np.zeros((max(n, 1), 3), np.float64)
    rgb = np.zeros((max(n, 1), 3), np.uint8)
    edge = np.zeros(max(n, 1), np.int64)
    lib.orc_extract_points(C.byref(cv), _ptr(xyz, C.c_double), _ptr(rgb, C.c_uint8), _ptr(edge, C.c_int64), n)
    return {"xyz": xyz[:n], "rgb": rgb[:n], "edge": edge[:n]}


# ---------------------------------------------------------------------------
# Depth-map conversion and tracking (Sec. Depth Map Conversion, Sec. Camera
# Tracking)
# ---------------------------------------------------------------------------
def _intr32(cam) -> _Intr:
    k = [float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy)]
    return _Intr(k[0], k[1], k[2], k[3], int(cam.width), int(cam.height))


def depth_maps(depth, cam, T=None, z_min=0.0, z_max=np.inf):
    """Vertex and normal maps (H, W, 3) float64 of a depth frame; world frame
    with T, camera frame without."""
    lib = _load()
    depth = np.ascontiguousarray(depth, np.float32)
    H, W = depth.shape
    v = np.zeros((H, W, 3), np.float64)
    n = np.zeros((H, W, 3), np.float64)
    Tm = None if T is None else _pose(T)
    lib.orc_depth_maps(_ptr(depth, C.c_float), C.byref(_intr32(cam)), _ptr(Tm, C.c_double), float(z_min),
                       float(z_max), _ptr(v, C.c_double), _ptr(n, C.c_double))
    return v, n


def icp_system(vertex, normal, cam, T_est, model_vertex, model_normal, T_model, dist, cos_min):
    """One point-to-plane linearisation: dict A (6, 6), b (6,), error, count,
    flags (H, W) of marginal association decisions and the sums of |term| over
    them (absA, absb, abse = (sum r^2, count))."""
    lib = _load()
    vertex = np.ascontiguousarray(vertex, np.float64)
    normal = np.ascontiguousarray(normal, np.float64)
    mv = np.ascontiguousarray(model_vertex, np.float32)
    mn = np.ascontiguousarray(model_normal, np.float32)
    H, W = vertex.shape[:2]
    A = np.zeros(36)
    b = np.zeros(6)
    err = C.c_double(0.0)
    cnt = C.c_int64(0)
    flags = np.zeros((H, W), np.uint8)
    absA, absb, abse = np.zeros(36), np.zeros(6), np.zeros(2)
    Te, Tm = _pose(T_est), _pose(T_model)
    lib.orc_icp_system(_ptr(vertex, C.c_double), _ptr(normal, C.c_double), C.byref(_intr32(cam)),
                       _ptr(Te, C.c_double), _ptr(mv, C.c_float), _ptr(mn, C.c_float), _ptr(Tm, C.c_double),
                       float(dist), float(cos_min), _ptr(A, C.c_double), _ptr(b, C.c_double), C.byref(err),
                       C.byref(cnt), _ptr(flags, C.c_uint8), _ptr(absA, C.c_double), _ptr(absb, C.c_double),
                       _ptr(abse, C.c_double))
    return {"A": A.reshape(6, 6), "b": b, "error": err.value, "count": cnt.value, "flags": flags.astype(bool),
            "absA": absA.reshape(6, 6), "absb": absb, "abse": abse}


def track(depth, cam, model_vertex, model_normal, T_model, T_init, iterations, dist, cos_min,
          z_min=0.0, z_max=np.inf):
    """Gauss-Newton point-to-plane ICP: maps of the frame (camera frame), then
    `iterations` times solve A x = b and set T <- exp(x^) T; stops early below
    6 associations or when A is not positive definite.  Returns (T, last)."""
    v, n = depth_maps(depth, cam, None, z_min, z_max)
    T = np.array(T_init, np.float64).reshape(4, 4).copy()
    last = None
    for _ in range(iterations):
        last = icp_system(v, n, cam, T, model_vertex, model_normal, T_model, dist, cos_min)
        if last["count"] < 6:
            break
        try:
            L = np.linalg.cholesky(last["A"])
        except np.linalg.LinAlgError:
            break
        x = np.linalg.solve(L.T, np.linalg.solve(L, last["b"]))
        T = se3_exp(x) @ T
    return T, last


def threads() -> int:
    """Threads the oracle's OpenMP loops use."""
    return int(_load().orc_threads())


def set_threads(n: int) -> None:
    """Threads for the oracle's OpenMP loops."""
    _load().orc_set_threads(int(n))
