"""Shared helpers of the GPU parity tests: move inputs to the device, rebuild
oracle volumes from the CUDA path's state, and compare raycast maps under the
tolerances stated below.

Tolerances (derived from the arithmetic of the FP32 path against the FP64 oracle):
  * TSDF, float32 storage: |dF| <= 1e-4 (units of mu) per lockstep frame on
    voxels whose FP64 decisions are not within the oracle's margins;
  * TSDF, half / int16 storage: 1e-4 + half a storage quantum at the value;
  * weights: exact; colour: exact (integer arithmetic), off-band only;
  * raycast: hit/miss identical on unflagged pixels (<= 0.1 % allowed),
    depth within 0.1 voxel along the ray, normals within 1 degree, colour
    within 1 LSB.
"""
import numpy as np

import oracle

F32_TOL = 1e-4
DEPTH_TOL_VOX = 0.1
NORMAL_TOL_DEG = 1.0


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def oracle_volume_from_gpu(m, vid, spec):
    F, W, rgba = m.read_decoded(vid)
    return oracle.Volume(tuple(spec.h), tuple(spec.r), float(spec.s), F, W, rgba)


def storage_quantum(F, fmt):
    """Half a quantum of the storage format at value F (0 for float32)."""
    if fmt == "f16":
        return np.spacing(np.abs(F).astype(np.float16)).astype(np.float64) / 2
    if fmt == "i16":
        return np.full(np.shape(F), 0.5 / 32767.0)
    return np.zeros(np.shape(F))


def check_lockstep(before, F, W, rgba, flags, fmt="f32", tol=F32_TOL, with_colour=True):
    """Compare the GPU state after one frame with the oracle's update of the
    same prior state; returns (max |dF| on checked voxels, flagged fraction)."""
    dec = (flags & (oracle.IF_Z | oracle.IF_PIX | oracle.IF_GATE)) != 0
    ok = ~dec
    dF = np.abs(F - before.F)
    lim = tol + storage_quantum(before.F, fmt)
    bad = ok & (dF > lim)
    assert not bad.any(), (f"{bad.sum()} voxels exceed the TSDF tolerance; worst "
                           f"{dF[bad].max():.3g} at {np.argwhere(bad)[:5].tolist()}")
    badw = ok & (W != before.W)
    assert not badw.any(), f"{badw.sum()} weights differ, e.g. {np.argwhere(badw)[:5].tolist()}"
    if with_colour:
        okc = ok & ((flags & oracle.IF_BAND) == 0)
        badc = okc[..., None] & (rgba != before.rgba)
        assert not badc.any(), f"{badc.any(-1).sum()} colours differ"
    return float(dF[ok].max()) if ok.any() else 0.0, float(dec.mean())


def compare_raycast(g, o, cam, T, pitch, mask=None, require_hits=0.05):
    """g: GPU maps (numpy), o: oracle maps.  mask: pixels to compare (the
    oracle's sampled pixels), default all.  Returns a summary dict."""
    H, W = cam.height, cam.width
    if mask is None:
        mask = np.ones((H, W), bool)
    hard = (o["flags"] & (oracle.RF_SIGN | oracle.RF_CELL | oracle.RF_RANGE | oracle.RF_TIE)) != 0
    ok = mask & ~hard
    gh, oh = g["depth"] > 0, o["depth"] > 0
    mism = ok & (gh != oh)
    assert mism.sum() <= max(1, 1e-3 * ok.sum()), f"hit/miss differs on {mism.sum()} of {ok.sum()} pixels"
    both = ok & gh & oh
    assert both.sum() >= require_hits * mask.sum(), f"too few hits to compare ({both.sum()})"
    # metric length of the ray direction per unit tau
    xs = (np.arange(W) - cam.cx) / cam.fx
    ys = (np.arange(H) - cam.cy) / cam.fy
    dn = np.sqrt(xs[None, :] ** 2 + ys[:, None] ** 2 + 1.0)
    derr = np.abs(g["depth"].astype(np.float64) - o["depth"]) * dn / pitch
    assert derr[both].max() <= DEPTH_TOL_VOX, f"depth error {derr[both].max():.3g} voxel"
    assert np.all(g["vol_id"][both] == o["vol"][both])
    shade_ok = both & ((o["flags"] & (oracle.RF_FACE | oracle.RF_GRAD)) == 0)
    on = np.linalg.norm(o["normal"], axis=-1) > 0.5
    cmp_n = shade_ok & on
    cosang = np.sum(g["normal"].astype(np.float64) * o["normal"], -1)
    assert cosang[cmp_n].min() >= np.cos(np.radians(NORMAL_TOL_DEG)), \
        f"normal error {np.degrees(np.arccos(np.clip(cosang[cmp_n].min(), -1, 1))):.3g} deg"
    assert np.all(np.linalg.norm(g["normal"][shade_ok & ~on], axis=-1) == 0)
    dc = np.abs(g["rgba"].astype(np.int32) - o["rgba"].astype(np.int32))
    assert dc[shade_ok].max(initial=0) <= 1, "colour differs by more than 1 LSB"
    verr = np.linalg.norm(g["vertex"].astype(np.float64) - o["vertex"], axis=-1) / pitch
    assert verr[both].max() <= DEPTH_TOL_VOX + 1e-3 * np.abs(o["vertex"][both]).max() / pitch
    return dict(compared=int(ok.sum()), flagged=int((mask & hard).sum()), hits=int(both.sum()),
                max_depth_err_vox=float(derr[both].max()), mismatches=int(mism.sum()))


def gpu_maps(out):
    return {k: host(v) for k, v in out.items()}


def check_brick_flags(m, vid, spec, min_free_recall=0.0):
    """Soundness of the per-brick summaries the raycast skips over: FREE implies
    every voxel of the brick (padding included) observed with F > 0, EMPTY
    implies none observed.  Returns the fraction of all-observed-positive
    bricks that carry the FREE flag."""
    flags = m.read_brick_flags(vid)
    F, W, _ = m.read_decoded(vid)
    nbz, nby, nbx = flags.shape
    pad = np.zeros((nbz * 8, nby * 8, nbx * 8), bool)
    pos = np.zeros_like(pad)
    rz, ry, rx = F.shape
    pad[:rz, :ry, :rx] = W > 0
    pos[:rz, :ry, :rx] = (W > 0) & (F > 0)
    b_all_pos = pos.reshape(nbz, 8, nby, 8, nbx, 8).all(axis=(1, 3, 5))
    b_none = ~pad.reshape(nbz, 8, nby, 8, nbx, 8).any(axis=(1, 3, 5))
    free = (flags & 1) != 0
    empty = (flags & 2) != 0
    noneg = (flags & 4) != 0
    neg = np.zeros_like(pad)
    neg[:rz, :ry, :rx] = (W > 0) & ~(F > 0)
    b_no_neg = ~neg.reshape(nbz, 8, nby, 8, nbx, 8).any(axis=(1, 3, 5))
    assert not np.any(free & ~b_all_pos), "FREE flag on a brick with an unobserved or non-positive voxel"
    assert not np.any(empty & ~b_none), "EMPTY flag on a brick with an observed voxel"
    assert not np.any(noneg & ~b_no_neg), "NONEG flag on a brick with an observed voxel F <= 0"
    recall = free[b_all_pos].mean() if b_all_pos.any() else 1.0
    assert recall >= min_free_recall, f"only {recall:.2%} of free bricks flagged"
    return float(recall)


def observed_box(m, vid, spec, margin=2):
    """Voxel box (lo, n) per axis x, y, z covering the volume's observed bricks
    (brick flags without the EMPTY bit) widened by `margin` voxels and clipped
    to the volume, or None when nothing is observed."""
    fl = m.read_brick_flags(vid)  # [nbz, nby, nbx]
    obs = (fl & 2) == 0
    if not obs.any():
        return None
    lo, n = [], []
    for a, ax in enumerate((2, 1, 0)):  # x, y, z = array axes 2, 1, 0
        other = tuple(b for b in range(3) if b != ax)
        idx = np.flatnonzero(obs.any(axis=other))
        l = max(0, int(idx[0]) * 8 - margin)
        h = min(int(spec.r[a]), (int(idx[-1]) + 1) * 8 + margin)
        lo.append(l)
        n.append(h - l)
    return lo, n


def frustum_box(spec, cam, T, z_far, margin=2):
    """Voxel box (lo, n) of the volume covering the part of the camera's
    viewing pyramid up to depth z_far (metres), widened by `margin` voxels and
    clipped to the volume, or None when they do not meet."""
    T = np.asarray(T, np.float64)
    corners = [T[:3, 3]]
    for x in (-0.5, cam.width - 0.5):
        for y in (-0.5, cam.height - 0.5):
            dc = np.array([(x - cam.cx) / cam.fx, (y - cam.cy) / cam.fy, 1.0])
            corners.append(T[:3, 3] + z_far * (T[:3, :3] @ dc))
    q = np.array(corners) / spec.s - np.array(spec.h)
    lo = np.maximum(np.floor(q.min(0)) - margin, 0).astype(int)
    hi = np.minimum(np.ceil(q.max(0)) + margin + 1, np.array(spec.r)).astype(int)
    if np.any(hi <= lo):
        return None
    return list(lo), list(hi - lo)


def union_box(a, b):
    if a is None:
        return b
    if b is None:
        return a
    lo = [min(x, y) for x, y in zip(a[0], b[0])]
    hi = [max(x + u, y + w) for x, u, y, w in zip(a[0], a[1], b[0], b[1])]
    return lo, [h - l for l, h in zip(lo, hi)]
