"""Seeded synthetic RGB-D inputs shaped like the paper's workloads.

This module is the one input source shared by the CUDA path's tests, the
benchmark and the FP64 oracle's tests.  It contains no TSDF arithmetic: it
renders analytic scenes (planes, spheres, axis-aligned boxes and hollow rooms)
by exact ray--primitive intersection at pixel centres, adds the axial depth
noise of a structured-light sensor, and generates camera trajectories.

Conventions (shared with the library):
  * camera frame: x right, y down, z forward; world frame: z up;
  * poses are 4x4 row-major camera-to-world matrices T = [R | t];
  * depth is float32 z-depth in metres, 0 where there is no valid return;
  * RGB is uint8 (H, W, 3), registered to depth with the same intrinsics;
  * a volume is (h, r, s): integer lattice offset h (voxels), dims r, pitch s
    (metres); voxel i sits at world position (h + i) * s.

Random numbers: a counter-based Philox stream keyed by (seed, frame), so any
frame can be regenerated alone.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass(frozen=True)
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int


@dataclass
class Scene:
    planes: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))   # n (unit), d: n.p = d
    spheres: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))  # centre, radius
    boxes: np.ndarray = field(default_factory=lambda: np.zeros((0, 6)))    # min xyz, max xyz (solid)
    rooms: np.ndarray = field(default_factory=lambda: np.zeros((0, 6)))    # min xyz, max xyz (seen from inside)
    colors: dict = field(default_factory=dict)  # (kind, index) -> (r, g, b)

    def color(self, kind: str, i: int):
        key = {"room": 0, "plane": 1, "sphere": 2, "box": 3}[kind] * 1000 + i
        return self.colors.get((kind, i), _palette(key))


def _palette(k: int):
    rs = np.random.Generator(np.random.Philox(key=0x5EED0000 + k))
    return tuple(int(v) for v in rs.integers(40, 250, size=3))


# --------------------------------------------------------------------------
# geometry helpers
# --------------------------------------------------------------------------

def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Camera-to-world pose at ``eye`` looking at ``target`` (x right, y down)."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    if np.linalg.norm(r) < 1e-9:
        r = np.cross(f, np.array([0.0, 1.0, 0.0]))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    T = np.eye(4)
    T[:3, 0], T[:3, 1], T[:3, 2], T[:3, 3] = r, d, f, eye
    return T


def rotation(axis, angle_rad) -> np.ndarray:
    axis = np.asarray(axis, np.float64)
    axis = axis / np.linalg.norm(axis)
    x, y, z = axis
    c, s = math.cos(angle_rad), math.sin(angle_rad)
    C = 1 - c
    return np.array([[c + x * x * C, x * y * C - z * s, x * z * C + y * s],
                     [y * x * C + z * s, c + y * y * C, y * z * C - x * s],
                     [z * x * C - y * s, z * y * C + x * s, c + z * z * C]])


def pixel_rays(cam: Camera, T) -> tuple:
    """World-frame ray origin and directions d = R [ (x-cx)/fx, (y-cy)/fy, 1 ]
    for every pixel centre (H, W, 3); the ray parameter is z-depth."""
    T = np.asarray(T, np.float64)
    xs = (np.arange(cam.width) - cam.cx) / cam.fx
    ys = (np.arange(cam.height) - cam.cy) / cam.fy
    dc = np.stack(np.broadcast_arrays(xs[None, :], ys[:, None], np.ones((1, 1))), axis=-1)
    d = dc @ T[:3, :3].T
    return T[:3, 3].copy(), d


def _hit_planes(o, d, planes, best, bid, base):
    for i, (nx, ny, nz, dd) in enumerate(planes):
        n = np.array([nx, ny, nz])
        den = d @ n
        with np.errstate(divide="ignore", invalid="ignore"):
            t = (dd - o @ n) / den
        ok = (t > 1e-9) & (t < best)
        best[ok], bid[ok] = t[ok], base + i


def _hit_spheres(o, d, spheres, best, bid, base):
    for i, (cx, cy, cz, rad) in enumerate(spheres):
        oc = o - np.array([cx, cy, cz])
        a = np.einsum("...k,...k->...", d, d)
        b = 2.0 * (d @ oc)
        c = oc @ oc - rad * rad
        disc = b * b - 4 * a * c
        sq = np.sqrt(np.maximum(disc, 0.0))
        t = (-b - sq) / (2 * a)
        ok = (disc >= 0) & (t > 1e-9) & (t < best)
        best[ok], bid[ok] = t[ok], base + i


def _slab(o, d, lo, hi):
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        t0 = (np.asarray(lo) - o) * inv
        t1 = (np.asarray(hi) - o) * inv
    tmin = np.nanmax(np.minimum(t0, t1), axis=-1)
    tmax = np.nanmin(np.maximum(t0, t1), axis=-1)
    return tmin, tmax


def _hit_boxes(o, d, boxes, best, bid, base):
    for i, bx in enumerate(boxes):
        tmin, tmax = _slab(o, d, bx[:3], bx[3:])
        ok = (tmin <= tmax) & (tmin > 1e-9) & (tmin < best)
        best[ok], bid[ok] = tmin[ok], base + i


def _hit_rooms(o, d, rooms, best, bid, base):
    for i, bx in enumerate(rooms):
        tmin, tmax = _slab(o, d, bx[:3], bx[3:])
        ok = (tmin <= tmax) & (tmax > 1e-9) & (tmax < best)
        best[ok], bid[ok] = tmax[ok], base + i


def render(scene: Scene, cam: Camera, T, *, seed: Optional[int] = None, frame: int = 0,
           noise: bool = True, z_range=(0.3, 5.0)):
    """Render depth (H, W) float32 z-depth and rgb (H, W, 3) uint8.

    Noise: z + N(0, (0.0012 z^2)^2), drawn from Philox keyed by (seed, frame).
    Pixels with no return, or outside ``z_range`` after noise, get depth 0
    (their RGB keeps the surface colour)."""
    o, d = pixel_rays(cam, T)
    H, W = cam.height, cam.width
    best = np.full((H, W), np.inf)
    bid = np.full((H, W), -1, np.int64)
    kinds = []
    for kind, arr, fn, width in (("room", scene.rooms, _hit_rooms, 6),
                                 ("plane", scene.planes, _hit_planes, 4),
                                 ("sphere", scene.spheres, _hit_spheres, 4),
                                 ("box", scene.boxes, _hit_boxes, 6)):
        arr = np.asarray(arr, np.float64).reshape(-1, width)
        fn(o, d, arr, best, bid, len(kinds))
        kinds += [(kind, i) for i in range(len(arr))]
    depth = np.where(np.isfinite(best), best, 0.0)
    rgb = np.zeros((H, W, 3), np.uint8)
    for k, (kind, i) in enumerate(kinds):
        m = bid == k
        if m.any():
            rgb[m] = scene.color(kind, i)
    if noise:
        if seed is None:
            raise ValueError("noise needs a seed")
        rng = np.random.Generator(np.random.Philox(key=(int(seed) << 32) | int(frame)))
        sigma = 0.0012 * depth * depth
        depth = depth + rng.standard_normal((H, W)) * sigma
    depth = np.where((depth >= z_range[0]) & (depth <= z_range[1]), depth, 0.0)
    return depth.astype(np.float32), rgb


# --------------------------------------------------------------------------
# trajectories
# --------------------------------------------------------------------------

def circle_trajectory(n: int, radius: float, height: float, target) -> List[np.ndarray]:
    """n poses on a circle around the z axis, all looking at ``target``."""
    out = []
    for i in range(n):
        th = 2 * math.pi * i / n
        eye = (radius * math.cos(th), radius * math.sin(th), height)
        out.append(look_at(eye, target))
    return out


def _rot_angle(Ra, Rb) -> float:
    c = (np.trace(Ra.T @ Rb) - 1.0) / 2.0
    return math.acos(max(-1.0, min(1.0, c)))


def handheld_trajectory(n: int, seed: int, centre, extent, look_radius: float,
                        look_height: float, v_max: float = 0.5, w_max_deg: float = 30.0,
                        fps: float = 30.0) -> List[np.ndarray]:
    """A smooth handheld-like path: the eye wanders on low-frequency sinusoids
    inside ``centre +- extent`` while the camera looks at a point sweeping
    around it at ``look_radius``.  Speeds are scaled so that every
    frame-to-frame step moves at most v_max/fps metres and turns at most
    w_max/fps degrees."""
    rng = np.random.Generator(np.random.Philox(key=(int(seed) << 32) | 0xC0FFEE))
    centre = np.asarray(centre, np.float64)
    extent = np.asarray(extent, np.float64)
    freqs = rng.uniform(0.5, 1.5, size=(3,))
    phases = rng.uniform(0, 2 * math.pi, size=(5,))
    sweep = rng.uniform(0.5, 0.7) * math.radians(w_max_deg) / fps  # radians per frame of yaw
    yaw0 = rng.uniform(0, 2 * math.pi)

    def pose(u, scale):
        eye = centre + scale * extent * np.sin(2 * math.pi * freqs * u * n / 300.0 + phases[:3])
        yaw = yaw0 + sweep * u * n
        pitch_h = look_height + 0.3 * math.sin(2 * math.pi * u * n / 150.0 + phases[3])
        tgt = centre + np.array([look_radius * math.cos(yaw), look_radius * math.sin(yaw), 0.0])
        tgt[2] = pitch_h
        return look_at(eye, tgt)

    scale = 1.0
    for _ in range(40):
        poses = [pose(i / max(n - 1, 1), scale) for i in range(n)]
        vmax = max((np.linalg.norm(poses[i + 1][:3, 3] - poses[i][:3, 3]) for i in range(n - 1)), default=0)
        wmax = max((_rot_angle(poses[i][:3, :3], poses[i + 1][:3, :3]) for i in range(n - 1)), default=0)
        if vmax <= v_max / fps and wmax <= math.radians(w_max_deg) / fps:
            return poses
        if vmax > v_max / fps:
            scale *= 0.9
        if wmax > math.radians(w_max_deg) / fps:
            sweep *= 0.9
    return poses


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

@dataclass
class VolumeSpec:
    h: tuple      # lattice offset, voxels
    r: tuple      # voxels per axis
    s: float      # pitch, metres


@dataclass
class Workload:
    name: str
    cam: Camera
    scene: Scene
    poses: list
    volumes: List[VolumeSpec]
    seed: int
    trunc_vox: float = 4.0
    w_max: float = 128.0
    z_range: tuple = (0.3, 5.0)

    def frame(self, i: int, noise: bool = True):
        return render(self.scene, self.cam, self.poses[i], seed=self.seed, frame=i, noise=noise,
                      z_range=self.z_range)

    @property
    def n_frames(self) -> int:
        return len(self.poses)


def _f32(x: float) -> float:
    return float(np.float32(x))


def single_volume_128(frames: int = 30, seed: int = 1, res: int = 128) -> Workload:
    """Plain single volume: res^3 voxels over a 3 m cube, 320x240 frames on a
    circle of radius 1.2 m at 1.0 m height looking at (0, 0, 0.3); a floor,
    three spheres (r 0.2-0.5 m) and one 0.4 x 0.3 x 0.5 m box."""
    rng = np.random.Generator(np.random.Philox(key=(seed << 32) | 0xABC))
    s = _f32(3.0 / res)
    h = (-res // 2, -res // 2, -int(round(0.25 / s)))
    scene = Scene()
    scene.planes = np.array([[0.0, 0.0, 1.0, 0.0]])
    sph = []
    for _ in range(3):
        r = rng.uniform(0.2, 0.5)
        sph.append([rng.uniform(-0.8, 0.8), rng.uniform(-0.8, 0.8), r, r])
    scene.spheres = np.array(sph)
    bx, by = rng.uniform(-0.6, 0.6, size=2)
    scene.boxes = np.array([[bx - 0.2, by - 0.15, 0.0, bx + 0.2, by + 0.15, 0.5]])
    cam = Camera(262.5, 262.5, 160.0, 120.0, 320, 240)
    poses = circle_trajectory(frames, 1.2, 1.0, (0.0, 0.0, 0.3))
    return Workload("single-volume 128^3, 3 m cube, 320x240", cam, scene, poses,
                    [VolumeSpec(h, (res, res, res), s)], seed)


def _room_scene(rng, lo, hi, n_boxes, n_spheres, keep_out_centre, keep_out_radius):
    scene = Scene()
    scene.rooms = np.array([list(lo) + list(hi)], np.float64)
    boxes, sph = [], []
    kc = np.asarray(keep_out_centre, np.float64)
    while len(boxes) < n_boxes:
        sx, sy, sz = rng.uniform(0.15, 0.6, size=3)
        x = rng.uniform(lo[0] + sx / 2, hi[0] - sx / 2)
        y = rng.uniform(lo[1] + sy / 2, hi[1] - sy / 2)
        if math.hypot(x - kc[0], y - kc[1]) < keep_out_radius + max(sx, sy):
            continue
        z0 = lo[2] if rng.uniform() < 0.7 else rng.uniform(lo[2], lo[2] + 1.0)
        boxes.append([x - sx / 2, y - sy / 2, z0, x + sx / 2, y + sy / 2, z0 + sz])
    while len(sph) < n_spheres:
        r = rng.uniform(0.1, 0.3)
        x = rng.uniform(lo[0] + r, hi[0] - r)
        y = rng.uniform(lo[1] + r, hi[1] - r)
        if math.hypot(x - kc[0], y - kc[1]) < keep_out_radius + r:
            continue
        z = rng.uniform(lo[2] + r, lo[2] + 1.6)
        sph.append([x, y, z, r])
    scene.boxes = np.array(boxes).reshape(-1, 6)
    scene.spheres = np.array(sph).reshape(-1, 4)
    return scene


def room_512(frames: int = 300, seed: int = 2, res: int = 512, width: int = 640,
             height: int = 480) -> Workload:
    """KinectFusion-scale: one res^3 volume over a 3 m cube (5.86 mm voxels
    at 512) holding a 2.9 x 2.9 x 2.7 m room with 10 boxes and 6 spheres,
    640x480 frames (fx = fy = 525) along a smooth handheld path (<= 0.5 m/s,
    <= 30 deg/s at 30 fps)."""
    rng = np.random.Generator(np.random.Philox(key=(seed << 32) | 0xABC))
    s = _f32(3.0 / res)
    h = (-res // 2, -res // 2, -int(round(0.15 / s)))
    lo, hi = (-1.45, -1.45, 0.0), (1.45, 1.45, 2.7)
    scene = _room_scene(rng, lo, hi, 10, 6, (0.0, 0.0), 0.75)
    f = 525.0 * width / 640.0
    cam = Camera(f, f, (width - 1) / 2.0, (height - 1) / 2.0, width, height)
    poses = handheld_trajectory(frames, seed, (0.0, 0.0, 1.4), (0.35, 0.35, 0.2), 1.5, 0.9)
    return Workload(f"single-volume {res}^3, 3 m room, {width}x{height}", cam, scene, poses,
                    [VolumeSpec(h, (res, res, res), s)], seed)


def tiled(wl: Workload, split: int = 2) -> Workload:
    """The same scene and frames mapped by split^3 subvolumes that tile the
    single volume of ``wl`` on the lattice h_t = k (r - 2) (two-voxel
    overlap, Sec. Initialization): requires r_single = split (r - 2) + 2."""
    (v,) = wl.volumes
    R = v.r[0]
    if (R - 2) % split:
        raise ValueError("single-volume size must be split*(r-2)+2")
    r = (R - 2) // split + 2
    vols = []
    for kz in range(split):
        for ky in range(split):
            for kx in range(split):
                hh = (v.h[0] + kx * (r - 2), v.h[1] + ky * (r - 2), v.h[2] + kz * (r - 2))
                vols.append(VolumeSpec(hh, (r, r, r), v.s))
    return Workload(wl.name + f" as {split}^3 tiles of {r}^3", wl.cam, wl.scene, wl.poses, vols,
                    wl.seed, wl.trunc_vox, wl.w_max, wl.z_range)


def room_tiles(res: int = 256, pitch: float = 0.002, split: int = 2, frames: int = 300, seed: int = 5,
               width: int = 640, height: int = 480) -> Workload:
    """Differentiable-raycast workload: split^3 subvolumes of res^3 voxels at
    `pitch` on the lattice h_t = k (res - 2) (two-voxel overlap) covering a
    cube of side (split (res - 2) + 2) pitch, holding a scaled room with 6
    boxes and 4 spheres; a handheld path scaled to the room (frames at
    640x480, fx = fy = 525)."""
    rng = np.random.Generator(np.random.Philox(key=(seed << 32) | 0xABC))
    side = (split * (res - 2) + 2) * pitch
    half = side / 2.0
    s = _f32(pitch)
    h0 = -int(round(half / s))
    margin = 0.04 * side
    lo = (-half + margin, -half + margin, margin)
    hi = (half - margin, half - margin, side - margin)
    scene = Scene()
    scene.rooms = np.array([list(lo) + list(hi)])
    boxes, sph = [], []
    L = side / 3.0
    while len(boxes) < 6:
        sx, sy, sz = rng.uniform(0.05, 0.2, size=3) * L
        x = rng.uniform(lo[0] + sx, hi[0] - sx)
        y = rng.uniform(lo[1] + sy, hi[1] - sy)
        if math.hypot(x, y) < 0.25 * side:
            continue
        boxes.append([x - sx / 2, y - sy / 2, lo[2], x + sx / 2, y + sy / 2, lo[2] + sz])
    while len(sph) < 4:
        r = rng.uniform(0.04, 0.1) * L
        x = rng.uniform(lo[0] + r, hi[0] - r)
        y = rng.uniform(lo[1] + r, hi[1] - r)
        if math.hypot(x, y) < 0.25 * side + r:
            continue
        sph.append([x, y, rng.uniform(lo[2] + r, lo[2] + 0.5 * side), r])
    scene.boxes = np.array(boxes)
    scene.spheres = np.array(sph)
    f = 525.0 * width / 640.0
    cam = Camera(f, f, (width - 1) / 2.0, (height - 1) / 2.0, width, height)
    poses = handheld_trajectory(frames, seed, (0.0, 0.0, 0.45 * side), (0.08 * side, 0.08 * side, 0.05 * side),
                                0.4 * side, 0.35 * side, v_max=0.5 * side / 3.0)
    vols = []
    for kz in range(split):
        for ky in range(split):
            for kx in range(split):
                vols.append(VolumeSpec((h0 + kx * (res - 2), h0 + ky * (res - 2), kz * (res - 2) - 2),
                                       (res, res, res), s))
    return Workload(f"{split ** 3} x {res}^3 tiles at {pitch * 1e3:g} mm, {width}x{height}", cam, scene,
                    poses, vols, seed, z_range=(0.1, 5.0))


def perturb_poses(poses, seed: int = 6, sigma_t: float = 0.02, sigma_r_deg: float = 1.0):
    """Each pose moved on the left by a random twist: translation N(0, sigma_t)
    per axis, rotation by N(0, sigma_r) degrees about a random axis."""
    rng = np.random.Generator(np.random.Philox(key=(int(seed) << 32) | 0x5E3))
    out = []
    for T in poses:
        axis = rng.normal(size=3)
        ang = math.radians(rng.normal() * sigma_r_deg)
        D = np.eye(4)
        D[:3, :3] = rotation(axis, ang)
        D[:3, 3] = rng.normal(size=3) * sigma_t
        # rotate about the camera centre, then translate
        c = np.asarray(T)[:3, 3]
        P = np.eye(4)
        P[:3, :3] = D[:3, :3]
        P[:3, 3] = c - D[:3, :3] @ c + D[:3, 3]
        out.append(P @ np.asarray(T))
    return out


def uneven_volumes(n_volumes: int = 64, frames: int = 300, seed: int = 4, width: int = 640,
                   height: int = 480, edges=(128, 192, 256, 384, 512, 768), pitch_mm=(1.0, 8.0),
                   half_extent: float = 9.0, height_m: float = 8.0) -> Workload:
    """Batched uneven volumes: n volumes with edge lengths drawn uniformly from
    `edges` and voxel pitch uniform in `pitch_mm`, placed without overlap
    (largest first, each on its own pitch lattice) in a hall of
    2 half_extent x 2 half_extent x height_m metres holding 40 boxes and
    spheres; 640x480 frames along a handheld path at the hall's centre.  With
    the defaults the 64 volumes hold about 7 G voxels."""
    rng = np.random.Generator(np.random.Philox(key=(seed << 32) | 0xABC))
    specs = []
    for _ in range(n_volumes):
        e = int(rng.choice(edges))
        s = _f32(rng.uniform(*pitch_mm) * 1e-3)
        specs.append((e, s))
    specs.sort(key=lambda es: -es[0] * es[1])
    lo_b = np.array([-half_extent, -half_extent, 0.0])
    hi_b = np.array([half_extent, half_extent, height_m])
    boxes_placed = []
    vols = []
    for e, s in specs:
        side = e * s
        for attempt in range(5000):
            p = rng.uniform(lo_b, np.maximum(lo_b, hi_b - side))
            h = np.round(p / s).astype(int)
            a = h * s
            b = a + (e - 1) * s
            if any(np.all(a < bb) and np.all(aa < b) for aa, bb in boxes_placed):
                continue
            boxes_placed.append((a, b))
            vols.append(VolumeSpec(tuple(int(x) for x in h), (e, e, e), s))
            break
        else:
            raise RuntimeError("could not place all volumes; enlarge the hall")
    scene = _room_scene(rng, tuple(lo_b + 0.05), tuple(hi_b - 0.05), 24, 16, (0.0, 0.0), 1.0)
    f = 525.0 * width / 640.0
    cam = Camera(f, f, (width - 1) / 2.0, (height - 1) / 2.0, width, height)
    poses = handheld_trajectory(frames, seed, (0.0, 0.0, 1.5), (0.6, 0.6, 0.2), 3.0, 1.2)
    return Workload(f"{n_volumes} uneven volumes (edges {edges[0]}-{edges[-1]}, {pitch_mm[0]:g}-"
                    f"{pitch_mm[1]:g} mm), {width}x{height}", cam, scene, poses, vols, seed)


@dataclass
class PlacementWorkload:
    """Frames of a scene to be mapped by dynamically placed volumes: volumes
    of volume_voxels^3 at voxel_size on the lattice h_t = k cell_voxels
    (cell_voxels = volume_voxels - 2)."""
    wl: Workload
    volume_voxels: int
    voxel_size: float
    max_volumes: int

    @property
    def cell_voxels(self) -> int:
        return self.volume_voxels - 2


def placement_room(frames: int = 1000, seed: int = 3, width: int = 640, height: int = 480,
                   volume_voxels: int = 512, side_m: float = 0.75, max_volumes: int = 16) -> PlacementWorkload:
    """Multi-volume dynamic placement: a 6 x 5 x 3 m room with 40 random boxes
    and spheres, a handheld path through it (640x480), volumes of
    volume_voxels^3 over side_m metres (1.46 mm voxels at 512 over 0.75 m),
    at most max_volumes resident."""
    rng = np.random.Generator(np.random.Philox(key=(seed << 32) | 0xABC))
    lo, hi = (-3.0, -2.5, 0.0), (3.0, 2.5, 3.0)
    scene = _room_scene(rng, lo, hi, 24, 16, (0.0, 0.0), 0.8)
    f = 525.0 * width / 640.0
    cam = Camera(f, f, (width - 1) / 2.0, (height - 1) / 2.0, width, height)
    poses = handheld_trajectory(frames, seed, (0.0, 0.0, 1.4), (1.2, 1.0, 0.2), 2.0, 1.0)
    wl = Workload(f"6x5x3 m room, 40 objects, {width}x{height}", cam, scene, poses, [], seed)
    return PlacementWorkload(wl, volume_voxels, _f32(side_m / volume_voxels), max_volumes)
