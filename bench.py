"""Benchmark: per-frame TSDF integration + raycast of the 512^3 room workload.

One step = one frame of the workload: integrate a 640x480 depth+RGB frame
into the 512^3 (3 m, 5.86 mm voxels) volume, then raycast the 640x480
depth/normal/colour/vertex maps at that frame's pose.  Frames are synthetic
(seeded analytic room of boxes and spheres, axial depth noise, handheld
trajectory), generated on the host before timing and resident in HBM while
the device-timed region runs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Prints one JSON line (rank 0).  `value` is updated voxel-updates per second of
the whole job (voxels whose TSDF changed, summed over ranks, divided by the
slowest rank's time for K integrate+raycast steps).  Under torchrun each rank
maps its own copy of the workload (independent problems: weak scaling, no
data-path collective).  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same steps.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time
from concurrent.futures import ProcessPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1511_07106_b300 import synth  # noqa: E402  (numpy only; no CUDA)

METRIC = "TSDF voxel-updates/s (integrate + raycast per frame)"
UNIT = "voxel-updates/s"
WORKLOAD = "room 512^3 single volume, 640x480 depth+RGB, integrate + raycast per frame"
N_FRAMES_MAX = 300


def CONFIG_OF(world):
    """The workload named in every line of this benchmark (both arms)."""
    return {"workload": WORKLOAD, "volume": "512^3 F32 TSDF + F32 weight + RGBA8, 5.86 mm",
            "image": "640x480", "trunc_voxels": 4, "w_max": 128,
            "l2": "inputs larger than L2 (1.61 GB volume per rank)",
            "parallelism": f"independent mapping job per GPU x{world}"}


def _render(i):
    wl = synth.room_512(frames=N_FRAMES_MAX)
    return wl.frame(i)


def _first_frames(frames, n):
    """The room's first n frames: those rendered for the run, and the rest
    rendered here (short runs render fewer than some measurements need)."""
    return list(frames[:n]) + [_render(i) for i in range(len(frames), n)]


def make_frames(n, procs):
    idx = [i % N_FRAMES_MAX for i in range(n)]
    uniq = sorted(set(idx))
    with ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn")) as ex:
        got = dict(zip(uniq, ex.map(_render, uniq)))
    return [got[i] for i in idx]


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def traffic_record(kernel):
    """DRAM bytes per launch from the committed ncu summary, if the kernel
    source is unchanged since it was captured (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p)).get(kernel)
    if not rec:
        return None
    src = os.path.join(ROOT, rec["source"])
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if h != rec["source_sha256_16"]:
        return None
    return rec


def run_graph_steps(m, poses, cam, maps, first, steps, dev_depth, dev_rgb):
    """One frame per step: integrate + raycast as one CUDA graph (mv_frame)."""
    for k in range(steps):
        i = first + k
        m.frame(dev_depth[i], dev_rgb[i], cam, poses[i], out=maps)


def run_eager_steps(m, poses, cam, maps, first, steps, dev_depth, dev_rgb):
    """The same step as separate calls (per-kernel event timing possible)."""
    for k in range(steps):
        i = first + k
        m.integrate(dev_depth[i], dev_rgb[i], cam, poses[i])
        m.raycast(cam, poses[i], out=maps)


def timed(torch, fn, clocks=None, head_start_ms=0.0):
    """Device time of fn() between two events.  head_start_ms > 0 first
    queues a spin kernel of about that length (before the first event), so
    that a pass whose host-side launches are slower than the GPU work still
    finds its launches queued: the GPU then never waits on the host, and the
    per-kernel event pairs time the kernels, not launch gaps."""
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if clocks:
        clocks.start()
    barrier(torch)
    torch.cuda.synchronize()
    if head_start_ms > 0:
        torch.cuda._sleep(int(head_start_ms * 1e-3 * 2.0e9))  # cycles at about 2 GHz
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(torch)
    clk = clocks.stop() if clocks else None
    return e0.elapsed_time(e1), clk


def bench_storage(torch, Mapper, Config, wl, poses, fmt, warmup, steps, dev_depth, dev_rgb,
                  clocks=None, instrument=True, tuning=None):
    """Device-timed steps for one storage format: `steps` graph steps (the
    measured throughput), then `steps` eager steps on the following frames
    with per-kernel CUDA events (the per-kernel roofline)."""
    (vs,) = wl.volumes
    cam = wl.cam
    m = Mapper(Config())
    vid = m.add_volume(vs.h, vs.r, vs.s, fmt)
    maps = m.alloc_maps(cam)
    run_graph_steps(m, poses, cam, maps, 0, warmup, dev_depth, dev_rgb)
    if tuning is None:
        tuning = m.autotune(dev_depth[warmup - 1], dev_rgb[warmup - 1], cam, poses[warmup - 1])
    else:  # fixed launch shapes (profiling runs: timings under a profiler mislead the autotuner)
        m.set_tuning(*tuning)
        tuning = m.tuning()
    m.synchronize()
    m.stats(reset=True)
    m.timings(reset=True)
    ms, clk = timed(torch, lambda: run_graph_steps(m, poses, cam, maps, warmup, steps, dev_depth, dev_rgb),
                    clocks)
    st = m.stats()
    tm_graph = m.timings(reset=True)
    out = dict(ms=ms, stats=st, graph_timings=tm_graph, clocks=clk, mapper=m, vid=vid, maps=maps,
               tuning=tuning)
    if instrument:
        m.stats(reset=True)
        m.set_timing(True)
        # the eager calls' host work (about 0.4 ms a step) exceeds their GPU
        # work: a head start of 0.5 ms a step keeps the queue full
        ms_e, _ = timed(torch, lambda: run_eager_steps(m, poses, cam, maps, warmup + steps, steps,
                                                      dev_depth, dev_rgb), head_start_ms=0.5 * steps)
        m.set_timing(False)
        out.update(eager_ms=ms_e, eager_stats=m.stats(), timings=m.timings())
    return out


def barrier(torch):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def _allreduce(torch, x, op, device):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        t = torch.tensor([float(x)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=getattr(dist.ReduceOp, op))
        return float(t.item())
    return float(x)


def allreduce_max(torch, x, device="cuda"):
    return _allreduce(torch, x, "MAX", device)


def allreduce_sum(torch, x, device="cuda"):
    return _allreduce(torch, x, "SUM", device)


def weak_scaling_value(torch, units, ms, device="cuda"):
    """Whole-job throughput of independent per-rank jobs: the units all ranks
    processed over the slowest rank's time."""
    return allreduce_sum(torch, units, device) / (allreduce_max(torch, ms, device) * 1e-3)


def integrate_bytes_per_voxel(fmt):
    return {"f32": 16, "f16": 8, "i16": 8}[fmt]


RAY_OUT_BYTES = 36  # per pixel: depth 4 + normal 12 + rgba 4 + vertex 12 + volume id 4


def raycast_bytes(cam, footprint, fmt):
    """Algorithmic bytes of one raycast launch: its outputs, plus -- when the
    oracle's count of the view's footprint is given (distinct voxels whose
    TSDF/weight a dense march reads, distinct voxels whose colour the hits
    read) -- those voxel bytes."""
    b = RAY_OUT_BYTES * cam.width * cam.height
    if footprint is not None:
        b += footprint[0] * integrate_bytes_per_voxel(fmt) // 2 + footprint[1] * 4
    return b


def kernel_summary(res, fmt, cam, steps, footprint=None):
    """Per-kernel average launch time and algorithmic bytes per launch."""
    tm = res["timings"]
    H, W = cam.height, cam.width
    out = {}
    st = res["eager_stats"]
    n_int = max(tm["integrate"][2], 1)
    upd = st["updated"] / n_int
    band = st["band"] / n_int
    bricks = st["bricks"] / n_int
    # read+write of (F, W) per updated voxel, of RGBA per band voxel, the frame
    # once (depth f32 + RGB8), the work list and the brick flags
    b_int = integrate_bytes_per_voxel(fmt) * upd + 8 * band + 7 * H * W + 8 * bricks + 2 * bricks
    for name, (launches, ms, timed) in tm.items():
        if timed == 0:
            continue
        avg_ms = ms / timed
        e = {"launches": launches, "avg_ms": avg_ms, "share": 0.0}
        if name == "integrate":
            e["algorithmic_bytes"] = b_int
            e["achieved_gbs"] = b_int / (avg_ms * 1e-3) / 1e9
        if name == "raycast":
            b_ray = raycast_bytes(cam, footprint, fmt)
            e["algorithmic_bytes"] = b_ray
            e["output_bytes"] = RAY_OUT_BYTES * H * W
            e["achieved_gbs"] = b_ray / (avg_ms * 1e-3) / 1e9
        out[name] = e
    tot = sum(v["avg_ms"] * v["launches"] for v in out.values())
    for v in out.values():
        v["share"] = v["avg_ms"] * v["launches"] / tot if tot else 0.0
    return out


def oracle_run(wl, frames, timed, footprint_at=(), one_core_at=None):
    """The FP64 oracle as it stands on whole frames of the room workload, from
    its own state: a volume that starts empty integrates frames 0, 1, ... in
    order, every voxel of the 512^3 volume each frame.  Each frame in `timed`
    is timed whole: its integration plus the raycast of every pixel at its
    pose (std time.perf_counter around the two oracle calls).  The frame
    `one_core_at` is timed the same way on one thread.  At each frame of
    `footprint_at` the oracle also counts the voxels a dense march of that
    view reads (the raycast's compulsory bytes).  Returns a dict; `volume` is
    the oracle's state after the last frame processed."""
    import oracle
    oracle.build()
    (vs,) = wl.volumes
    vol = oracle.Volume(vs.h, vs.r, vs.s)
    cfg = oracle.Config()
    timed = set(timed)
    last = max([*timed, *footprint_at, -1 if one_core_at is None else one_core_at])
    cores = oracle.threads()
    upd, secs, one, fps = 0, 0.0, None, []
    for i in range(last + 1):
        d, c = frames[i]
        T = wl.poses[i % N_FRAMES_MAX]
        if i == one_core_at:
            oracle.set_threads(1)
        t0 = time.perf_counter()
        cnt, _ = oracle.integrate(vol, d, c, wl.cam, T, cfg)
        if i in timed or i == one_core_at:
            oracle.raycast([vol], wl.cam, T, cfg)
            dt = time.perf_counter() - t0
            if i == one_core_at:
                one = (int(cnt[0]), dt)
                oracle.set_threads(cores)
            else:
                upd += int(cnt[0])
                secs += dt
        if i in footprint_at:
            fps.append(oracle.raycast_footprint([vol], wl.cam, T, cfg)[0])
    return {"updated": upd, "seconds": secs, "frames": len(timed), "cores": cores, "one_core": one,
            "footprints": fps, "volume": vol, "last_frame": last}


ORACLE_SAMPLE = ("whole frames of the same workload: each frame integrated into every voxel of the "
                 "512^3 volume and raycast at every pixel of 640x480, from the oracle's own state "
                 "(frames integrated in order from an empty volume); FP64 C oracle, OpenMP")


def accuracy_vs_oracle(torch, Mapper, Config, wl, frames, k, dev_depth, dev_rgb, own):
    """Error of each storage format against the FP64 oracle at frame k of the
    room workload (k = the oracle's last frame):
      lockstep: the oracle applies frame k to the format's own GPU state after
        frame k - 1; |dF| over the voxels that frame updated, excluding voxels
        whose FP64 decisions lie within the oracle's margins (counted);
      raycast: the oracle raycasts the format's GPU state after frame k at
        pose k; |d tau| along the ray in voxels over pixels hit on both sides
        and not flagged, plus hit/miss agreement;
      drift: the format's GPU state after frames 0..k against the oracle's own
        independent FP64 state (`own`), and the raycasts of the two states.
    """
    import oracle
    (vs,) = wl.volumes
    cam = wl.cam
    cfg = oracle.Config()
    T = wl.poses[k % N_FRAMES_MAX]
    d_k, c_k = frames[k]
    xs = (np.arange(cam.width) - cam.cx) / cam.fx
    ys = (np.arange(cam.height) - cam.cy) / cam.fy
    dn = np.sqrt(xs[None, :] ** 2 + ys[:, None] ** 2 + 1.0)
    own_maps = oracle.raycast([own], cam, T, cfg)

    def q(a, p):
        return float(np.percentile(a, p)) if a.size else None

    def depth_err(g, o):
        hard = (o["flags"] & (oracle.RF_SIGN | oracle.RF_CELL | oracle.RF_RANGE | oracle.RF_TIE)) != 0
        gh, oh = g > 0, o["depth"] > 0
        both = gh & oh & ~hard
        e = np.abs(g.astype(np.float64) - o["depth"]) * dn / vs.s
        return {"pixels_compared": int((~hard).sum()), "hit_agreement": float((gh == oh)[~hard].mean()),
                "max_vox": float(e[both].max()) if both.any() else None, "p99_vox": q(e[both], 99),
                "p50_vox": q(e[both], 50)}

    out = {"frame": k, "tolerance_tsdf_f32": 1e-4, "tolerance_depth_vox": 0.1}
    for fmt in ("f32", "f16", "i16"):
        m = Mapper(Config())
        vid = m.add_volume(vs.h, vs.r, vs.s, fmt)
        for i in range(k):
            m.integrate(dev_depth[i], dev_rgb[i], cam, wl.poses[i % N_FRAMES_MAX])
        F0, W0, c0 = m.read_decoded(vid)
        W_prev = W0.copy()  # the oracle updates `before` (which shares F0, W0) in place
        before = oracle.Volume(vs.h, vs.r, vs.s, F0, W0, c0)
        del c0
        _, flags = oracle.integrate(before, d_k, c_k, cam, T, cfg, want_flags=True)
        m.integrate(dev_depth[k], dev_rgb[k], cam, T)
        F1, W1, c1 = m.read_decoded(vid)
        upd = W1 != W_prev
        dec = (flags & (oracle.IF_Z | oracle.IF_PIX | oracle.IF_GATE)) != 0
        ok = upd & ~dec
        dF = np.abs(F1 - before.F)[ok]
        weights_equal = bool(np.array_equal(W1[ok], before.W[ok]))
        del before, F0, W0, W_prev
        lock = {"voxels": int(ok.sum()), "flagged_fraction": float((upd & dec).sum() / max(upd.sum(), 1)),
                "max": float(dF.max()) if dF.size else None, "p99": q(dF, 99), "p50": q(dF, 50),
                "weights_equal": weights_equal}
        del dF
        g = m.raycast(cam, T)
        gd = g["depth"].cpu().numpy()
        after = oracle.Volume(vs.h, vs.r, vs.s, F1, W1, c1)
        o = oracle.raycast([after], cam, T, cfg)
        ray = depth_err(gd, o)
        del after, o
        both = (W1 > 0) & (own.W > 0)
        dd = np.abs(F1 - own.F)[both]
        drift = {"voxels_observed_both": int(both.sum()),
                 "observed_agreement": float(((W1 > 0) == (own.W > 0)).mean()),
                 "weight_agreement": float((W1 == own.W)[both].mean()),
                 "tsdf_p50": q(dd, 50), "tsdf_p99": q(dd, 99), "tsdf_max": float(dd.max()) if dd.size else None,
                 "raycast": depth_err(gd, own_maps)}
        del dd, both, F1, W1, c1
        out[fmt] = {"lockstep_tsdf": lock, "raycast_depth": ray, "drift_vs_independent_oracle": drift}
        m.close()
        del m
        torch.cuda.empty_cache()
    return out


def e2e_run(torch, Mapper, Config, wl, frames, steps, warmup):
    """Same metric through the library's host-buffer call (mv_frame_host):
    every step hands the library its depth + RGB frame in pinned host memory
    and receives depth / normal / colour maps in pinned host memory; the
    uploads, the frame's kernels and the downloads run on the library's own
    streams, pipelined over its two device buffer sets, and the host reads
    each step's maps after waiting for its ticket (one frame late, so that
    the next frame is already queued)."""
    (vs,) = wl.volumes
    cam = wl.cam
    m = Mapper(Config())
    m.add_volume(vs.h, vs.r, vs.s, "f32")
    H, W = cam.height, cam.width
    hd = [torch.from_numpy(f[0]).pin_memory() for f in frames]
    hc = [torch.from_numpy(f[1]).pin_memory() for f in frames]
    out = [m.alloc_host_maps(cam) for _ in range(3)]
    checksum = 0.0
    pending = []

    def step(i):
        nonlocal checksum
        pending.append((m.frame_host(hd[i], hc[i], cam, wl.poses[i % N_FRAMES_MAX], out[i % 3]), i))
        if len(pending) > 1:
            t, j = pending.pop(0)
            m.frame_host_wait(t)
            checksum += float(out[j % 3]["depth"][H // 2, W // 2])

    def drain():
        nonlocal checksum
        while pending:
            t, j = pending.pop(0)
            m.frame_host_wait(t)
            checksum += float(out[j % 3]["depth"][H // 2, W // 2])

    for i in range(warmup):
        step(i)
    drain()
    m.synchronize()
    m.stats(reset=True)
    barrier(torch)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(steps):
        step(warmup + k)
    drain()
    dt = time.perf_counter() - t0
    barrier(torch)
    st = m.stats()
    m.close()
    h2d = 4 * H * W + 3 * H * W
    d2h = 4 * H * W + 12 * H * W + 4 * H * W
    return st["updated"], dt, h2d, d2h


def _render_uneven(i):
    return synth.uneven_volumes(frames=N_FRAMES_MAX).frame(i)


def _render_tiles(i):
    return synth.room_tiles(frames=N_FRAMES_MAX).frame(i)


PLACEMENT_FRAMES = 90
RESERVED_HOST_SETS = 24  # pinned host buffer sets for evicted 512^3 volumes (38 GB)


def _render_placement(i):
    return synth.placement_room(frames=N_FRAMES_MAX).wl.frame(i)


def _gen(fn, idx, procs):
    with ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(fn, idx))


def observed_box(m, vid, r, margin=2):
    """Voxel box (lo, n) over the volume's observed bricks (no EMPTY flag),
    widened by `margin` voxels and clipped to the volume; None if none."""
    fl = m.read_brick_flags(vid)
    obs = (fl & 2) == 0
    if not obs.any():
        return None
    lo, n = [], []
    for a, ax in enumerate((2, 1, 0)):
        idx = np.flatnonzero(obs.any(axis=tuple(b for b in range(3) if b != ax)))
        lo_a = max(0, int(idx[0]) * 8 - margin)
        lo.append(lo_a)
        n.append(min(int(r[a]), (int(idx[-1]) + 1) * 8 + margin) - lo_a)
    return lo, n


def uneven_raycast_accuracy(m, ids, wl, maps, T, stride=8):
    """Raycast depth error of a frame of the uneven volumes against the FP64
    oracle, which raycasts the same state: each observed volume read over
    the box of its observed bricks widened by 2 voxels (outside it every
    sample is invalid, so the box holds every hit); every `stride`-th pixel."""
    import oracle
    cam = wl.cam
    vols, vids = [], []
    for vid, v in zip(ids, wl.volumes):
        box = observed_box(m, vid, v.r)
        if box is None:
            continue
        lo, n = box
        F, W, col = m.read_box_decoded(vid, lo, n)
        vols.append(oracle.Volume(tuple(int(v.h[a] + lo[a]) for a in range(3)), tuple(n), float(v.s), F, W, col))
        vids.append(vid)
    pix = np.arange(0, cam.width * cam.height, stride)
    o = oracle.raycast(vols, cam, T, oracle.Config(), ids=vids, pixels=pix)
    g = maps["depth"].cpu().numpy().reshape(-1)[pix].astype(np.float64)
    gid = maps["vol_id"].cpu().numpy().reshape(-1)[pix]
    od, fl = o["depth"].reshape(-1)[pix], o["flags"].reshape(-1)[pix]
    hard = (fl & (oracle.RF_SIGN | oracle.RF_CELL | oracle.RF_RANGE | oracle.RF_TIE)) != 0
    xs, ys = (pix % cam.width - cam.cx) / cam.fx, (pix // cam.width - cam.cy) / cam.fy
    dn = np.sqrt(xs ** 2 + ys ** 2 + 1.0)
    pitch = {vid: v.s for vid, v in zip(ids, wl.volumes)}
    both = (g > 0) & (od > 0) & ~hard
    err = np.array([abs(g[i] - od[i]) * dn[i] / pitch[int(gid[i])] for i in np.flatnonzero(both)])
    return {"pixels_compared": int((~hard).sum()), "hits": int(both.sum()),
            "hit_agreement": float(((g > 0) == (od > 0))[~hard].mean()),
            "max_vox": float(err.max()) if err.size else None,
            "p99_vox": float(np.percentile(err, 99)) if err.size else None,
            "volumes_read": len(vols)}


def bench_uneven(torch, Mapper, Config, frames, steps, warmup, with_oracle=False):
    """64 volumes of uneven size and pitch (about 7.3 G voxels): one batched
    graph per frame vs the paper's per-volume loop, and storage formats; with
    the oracle, the raycast depth error of each format's last frame."""
    wl = synth.uneven_volumes(frames=N_FRAMES_MAX)
    cam = wl.cam
    dd = torch.from_numpy(np.stack([f[0] for f in frames])).cuda()
    dc = torch.from_numpy(np.stack([f[1] for f in frames])).cuda()
    out = {"workload": wl.name, "volumes": len(wl.volumes),
           "voxels": int(sum(np.prod(v.r) for v in wl.volumes)), "steps": steps}
    for mode, fmt in (("batched", "f32"), ("per_volume", "f32"), ("batched", "f16"), ("batched", "i16")):
        m = Mapper(Config())
        ids = [m.add_volume(v.h, v.r, v.s, fmt) for v in wl.volumes]
        maps = m.alloc_maps(cam)

        def step(i):
            if mode == "batched":
                m.frame(dd[i], dc[i], cam, wl.poses[i], out=maps)
            else:
                for vid in ids:
                    m.integrate_volume(vid, dd[i], dc[i], cam, wl.poses[i])
                for k, vid in enumerate(ids):
                    m.raycast_volume(vid, k == 0, cam, wl.poses[i], maps)

        for i in range(warmup):
            step(i)
        if mode == "batched":
            m.autotune(dd[warmup - 1], dc[warmup - 1], cam, wl.poses[warmup - 1])
        m.synchronize()
        m.stats(reset=True)
        ms, _ = timed(torch, lambda: [step(warmup + k) for k in range(steps)])
        st = m.stats()
        key = f"{mode}_{fmt}"
        out[key] = {"ms_per_step": ms / steps, "voxel_updates_per_s": st["updated"] / (ms * 1e-3),
                    "mrays_per_s": cam.width * cam.height * steps / (ms * 1e-3) / 1e6,
                    "updated_voxels_per_frame": st["updated"] / steps}
        if with_oracle and mode == "batched":
            out[key]["raycast_vs_oracle"] = uneven_raycast_accuracy(m, ids, wl, maps,
                                                                    wl.poses[warmup + steps - 1])
        m.close()
        del m
        torch.cuda.empty_cache()
    out["batched_over_per_volume"] = out["per_volume_f32"]["ms_per_step"] / out["batched_f32"]["ms_per_step"]
    return out


def bench_diff(torch, Mapper, Config, frames, n_poses=16, adam_steps=50):
    """Differentiable raycast: 8 x 256^3 tiles (2 mm) prefilled from the given
    frames; 16 poses perturbed by N(0, 2 cm) / N(0, 1 deg); forward +
    backward through the autograd Function (all views in one raycast launch
    and one backward launch, the tangent-space solve on the GPU), and 50 Adam
    steps of pose refinement (each step one forward, the loss, one backward
    and the update: refine_ms_per_step)."""
    from paper_1511_07106_b300 import diff
    wl = synth.room_tiles(frames=N_FRAMES_MAX)
    cam = wl.cam
    m = Mapper(Config(n_bisect=30))
    for v in wl.volumes:
        m.add_volume(v.h, v.r, v.s)
    for i, (d, c) in enumerate(frames):
        m.integrate(torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda(), cam, wl.poses[i])
    idx = np.linspace(0, len(frames) - 1, n_poses).astype(int)
    T_true = np.stack([wl.poses[i] for i in idx])
    T_init = np.stack(synth.perturb_poses(list(T_true), seed=6))
    with torch.no_grad():
        ref_d, ref_c = diff.render(m, cam, torch.tensor(T_true))
    # forward + backward timing at the perturbed poses
    T = torch.tensor(T_init, requires_grad=True)
    for _ in range(2):
        dpt, col = diff.render(m, cam, T)
        diff.l1_loss(dpt, col, ref_d, ref_c).backward()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = 5
    for _ in range(reps):
        dpt, col = diff.render(m, cam, T)
        loss = diff.l1_loss(dpt, col, ref_d, ref_c)
        loss.backward()
    torch.cuda.synchronize()
    fb_ms = (time.perf_counter() - t0) / reps * 1e3
    m.timings(reset=True)
    m.set_timing(True)
    dpt, col = diff.render(m, cam, T)
    diff.l1_loss(dpt, col, ref_d, ref_c).backward()
    m.set_timing(False)
    tm = m.timings()

    def err(Ts):
        t = float(np.mean([np.linalg.norm(a[:3, 3] - b[:3, 3]) for a, b in zip(Ts, T_true)]))
        r = float(np.mean([np.degrees(np.arccos(np.clip((np.trace(a[:3, :3].T @ b[:3, :3]) - 1) / 2, -1, 1)))
                           for a, b in zip(Ts, T_true)]))
        return t, r

    curve = []
    diff.refine_poses(m, cam, T_init, ref_d, ref_c, steps=2)  # first-call set-up outside the timing
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    T_fin, losses = diff.refine_poses(m, cam, T_init, ref_d, ref_c, steps=adam_steps,
                                      callback=lambda it, Ts, l: curve.append(err(Ts)) if it % 10 == 9 else None)
    torch.cuda.synchronize()
    refine_ms_per_step = (time.perf_counter() - t0) * 1e3 / adam_steps
    # the same steps with the loss and its gradients as torch operations
    # between mv_raycast_batch and mv_raycast_backward (the unfused path)
    diff.refine_poses(m, cam, T_init, ref_d, ref_c, steps=2, fused=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    diff.refine_poses(m, cam, T_init, ref_d, ref_c, steps=adam_steps, fused=False)
    torch.cuda.synchronize()
    unfused_ms_per_step = (time.perf_counter() - t0) * 1e3 / adam_steps
    m.close()
    rays = n_poses * cam.width * cam.height
    return {"workload": wl.name, "poses": n_poses, "prefill_frames": len(frames),
            "forward_backward_ms": refine_ms_per_step,
            "forward_backward_note": "one refinement step: the forward of all 16 views (one launch), the L1 loss, "
                                     "its gradient and the backward in one call (mv_raycast_backward_l1: the "
                                     "loss statistics, then the backward forming each pixel's gradient) and the "
                                     "tangent-space Adam update",
            "refine_unfused_ms_per_step": unfused_ms_per_step,
            "mrays_per_s_forward_backward": rays / (refine_ms_per_step * 1e-3) / 1e6,
            "autograd_forward_backward_ms": fb_ms,
            "backward_kernel_ms": tm["backward"][1] / max(tm["backward"][2], 1),
            "raycast_kernel_ms": tm["raycast"][1] / max(tm["raycast"][2], 1),
            "pose_error_m_deg_initial": err(T_init), "pose_error_m_deg_final": err(T_fin),
            "pose_error_every_10_steps": curve, "loss_initial": losses[0], "loss_final": losses[-1],
            "refine_ms_per_step": refine_ms_per_step}


def bench_swap(torch, Mapper, Config, frames, steps):
    """Swap one 512^3 volume out and back in (pinned host memory, side
    stream) while integrating another: overlap of the copies with compute."""
    wl = synth.room_512(frames=N_FRAMES_MAX)
    (vs,) = wl.volumes
    cam = wl.cam
    m = Mapper(Config())
    a = m.add_volume(vs.h, vs.r, vs.s)
    b = m.add_volume((vs.h[0] + 4096, vs.h[1], vs.h[2]), vs.r, vs.s)  # far away: never in view
    dd = torch.from_numpy(np.stack([f[0] for f in frames])).cuda()
    dc = torch.from_numpy(np.stack([f[1] for f in frames])).cuda()
    m.swap_out(b)
    m.swap_in(b)  # first swap allocates the pinned buffers
    m.synchronize()

    def integ():
        # integrating volume a alone does not wait for the copies of volume b
        for k in range(steps):
            m.integrate_volume(a, dd[k % len(frames)], dc[k % len(frames)], cam, wl.poses[k % len(frames)])

    def swap():
        m.swap_out(b)
        m.swap_in(b)

    t_int, _ = timed(torch, integ)
    t0 = time.perf_counter()
    swap()
    m.synchronize()
    t_swap = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    swap()
    integ()
    m.synchronize()
    t_both = (time.perf_counter() - t0) * 1e3
    q = m.query(b)
    nbytes = 2 * q["host_bytes"]  # the bytes each copy moves (the derived masks are rebuilt, not copied)
    m.close()
    return {"volume_bytes": nbytes // 2, "integrate_ms": t_int, "swap_out_in_ms": t_swap,
            "both_ms": t_both, "copy_gbs": nbytes / (t_swap * 1e-3) / 1e9,
            "hidden_fraction": max(0.0, min(1.0, (t_int + t_swap - t_both) / min(t_int, t_swap)))}


def bench_streamed(torch, Mapper, Config, frames, n_frames=6):
    """Full-cover out-of-core frames (the paper's per-frame upload, integrate,
    raycast, download of every volume): 4 tiles of 512^3 (the lower half of
    the room mapped at 2.93 mm), all swapped out to pinned host memory and
    streamed through the device every frame; only the bricks a frame can read
    go up and only those it changed come back (plus the flags)."""
    wl = synth.tiled(synth.room_512(frames=N_FRAMES_MAX, res=1022), split=2)
    vols = wl.volumes[:4]
    cam = wl.cam
    frames = _first_frames(frames, n_frames + 1)
    dd = torch.from_numpy(np.stack([f[0] for f in frames[:n_frames + 1]])).cuda()
    dc = torch.from_numpy(np.stack([f[1] for f in frames[:n_frames + 1]])).cuda()
    out = {"workload": "4 x 512^3 tiles at 2.93 mm (lower half of the 3 m room), all swapped out, "
                       "streamed every frame, 640x480",
           "volumes": len(vols), "paper_s_per_frame_per_volume": 0.17,
           "paper_hardware": "GTX 880M (context only)"}
    for fmt, n_slots in (("f32", 1), ("f32", 2), ("f16", 2)):
        m = Mapper(Config())
        ids = [m.add_volume(v.h, v.r, v.s, fmt) for v in vols]
        for vid in ids:
            m.swap_out(vid)
        m.synchronize()
        maps = m.alloc_maps(cam)
        m.frame_streamed(dd[0], dc[0], cam, wl.poses[0], out=maps, n_slots=n_slots)  # allocates the slots
        m.synchronize()
        m.stats(reset=True)
        t0 = time.perf_counter()
        for k in range(1, n_frames + 1):
            m.frame_streamed(dd[k], dc[k], cam, wl.poses[k], out=maps, n_slots=n_slots)
        m.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / n_frames
        st = m.stats()
        vbytes = m.query(ids[0])["host_bytes"]
        nb = int(np.prod([(r + 7) // 8 for r in vols[0].r]))
        brick_bytes = 512 * ((8 if fmt == "f32" else 4) + 4)
        up = st["stream_up"] / n_frames * brick_bytes
        down = st["stream_down"] / n_frames * brick_bytes
        m.close()
        torch.cuda.empty_cache()
        out[f"{fmt}_slots{n_slots}"] = {
            "ms_per_frame": ms, "s_per_frame_per_volume": ms * 1e-3 / len(vols),
            "bytes_per_volume": vbytes, "bricks_per_volume": nb,
            "upload_bytes_per_frame": up, "writeback_bytes_per_frame": down,
            "upload_gbs": up / (ms * 1e-3) / 1e9, "writeback_gbs": down / (ms * 1e-3) / 1e9,
            "updated_voxels_per_frame": st["updated"] / n_frames}
    return out


def bench_placement(torch, Mapper, Config, frames):
    """Multi-volume dynamic placement (the paper's Sec. Dynamic Mapping for
    SLAM): a 6 x 5 x 3 m room, 512^3 volumes of 0.75 m (1.46 mm voxels) placed
    on the lattice by the ray-endpoint histogram, at most 16 resident, the
    displaced ones swapped out to pinned host memory.  Per frame: integrate +
    raycast of the resident volumes (mv_frame), then one placement step."""
    from paper_1511_07106_b300 import Placer
    pw = synth.placement_room(frames=N_FRAMES_MAX)
    wl = pw.wl
    m = Mapper(Config())
    p = Placer(m, pw.cell_voxels, pw.volume_voxels, pw.voxel_size, pw.max_volumes, hysteresis=1.5)
    # pin host buffers for evicted volumes before the run (mv_reserve_host)
    t0 = time.perf_counter()
    m.reserve_host((pw.volume_voxels,) * 3, "f32", RESERVED_HOST_SETS)
    reserve_s = time.perf_counter() - t0
    maps = m.alloc_maps(wl.cam)
    dd = torch.from_numpy(np.stack([f[0] for f in frames])).cuda()
    dc = torch.from_numpy(np.stack([f[1] for f in frames])).cuda()
    tot = {"added": 0, "restored": 0, "evicted": 0}
    res_sum, t_frame, t_place, upd = 0, 0.0, 0.0, 0
    n = len(frames)
    m.stats(reset=True)
    for i in range(n):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m.frame(dd[i], dc[i], wl.cam, wl.poses[i], out=maps)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        r = p.update(dd[i], wl.cam, wl.poses[i])
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        if i > 0:  # frame 0 integrates into nothing: the first placement follows it
            t_frame += t1 - t0
            t_place += t2 - t1
            res_sum += r["resident"]
        for k in tot:
            tot[k] += r[k]
    m.synchronize()
    upd = m.stats()["updated"]
    nv = len(p.volumes())
    # the endpoint histogram alone (2 kernels + the copy of c(l) to the host)
    for _ in range(3):
        p.histogram(dd[-1], wl.cam, wl.poses[n - 1])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(20):
        p.histogram(dd[-1], wl.cam, wl.poses[n - 1])
    hist_ms = (time.perf_counter() - t0) * 1e3 / 20
    p.close()
    m.close()
    torch.cuda.empty_cache()
    return {"workload": "6x5x3 m room, 40 objects, 640x480; 512^3 volumes of 0.75 m (1.46 mm), "
                        "at most 16 resident, hysteresis 1.5",
            "frames": n, "ms_per_frame_integrate_raycast": t_frame * 1e3 / (n - 1),
            "ms_per_frame_placement": t_place * 1e3 / (n - 1), "ms_histogram": hist_ms,
            "mean_resident": res_sum / (n - 1), "volumes_placed": nv,
            "pinned_sets_reserved_before_run": RESERVED_HOST_SETS, "reserve_s": reserve_s,
            "voxel_updates_per_s": upd / (t_frame + 1e-12), **tot}


def bench_resolution(torch, Mapper, Config, frames, n_frames=30):
    """The paper's resolution comparison (Table 1: vertices of one KinectFusion
    volume vs 8 subvolumes over the same region) on the synthetic room: one
    512^3 volume over the 3 m cube vs 2 x 2 x 2 tiles of 512^3 (2.93 mm) over
    the same cube, the same frames integrated into both; surface points
    counted by mv_extract_points.  Also the extraction time of the 512^3
    volume."""
    out = {"workload": f"3 m room, {n_frames} frames at 640x480: one 512^3 volume (5.86 mm) vs "
                       "8 tiles of 512^3 (2.93 mm)", "paper_vertex_gain_8_volumes": 4.75}
    frames = _first_frames(frames, n_frames)
    dd = torch.from_numpy(np.stack([f[0] for f in frames[:n_frames]])).cuda()
    dc = torch.from_numpy(np.stack([f[1] for f in frames[:n_frames]])).cuda()
    for name, wl in (("single_512", synth.room_512(frames=N_FRAMES_MAX)),
                     ("tiles_8x512", synth.tiled(synth.room_512(frames=N_FRAMES_MAX, res=1022), split=2))):
        m = Mapper(Config())
        ids = [m.add_volume(v.h, v.r, v.s) for v in wl.volumes]
        for k in range(n_frames):
            m.integrate(dd[k], dc[k], wl.cam, wl.poses[k])
        m.synchronize()
        n = 0
        for vid in ids:
            n += int(m.extract_points(vid, rgb=False, edges=False)["xyz"].shape[0])
        out[name + "_points"] = n
        if name == "single_512":
            g = m.extract_points(ids[0])
            cap = int(g["xyz"].shape[0])
            for _ in range(3):
                m.extract_points(ids[0], cap=cap)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(10):
                m.extract_points(ids[0], cap=cap)
            ms = (time.perf_counter() - t0) * 1e3 / 10
            out["extract_ms_512"] = ms
            out["extract_mpoints_per_s"] = cap / (ms * 1e-3) / 1e6
        m.close()
        torch.cuda.empty_cache()
    out["vertex_gain"] = out["tiles_8x512_points"] / max(out["single_512_points"], 1)
    return out


def bench_track(torch, Mapper, Config, frames, n_map=20, n_track=10, iterations=10):
    """Camera tracking against the raycast model (Sec. Depth Map Conversion,
    Sec. Camera Tracking): the room's 512^3 volume built from the first n_map
    frames at their true poses; then each next frame is tracked by
    point-to-plane ICP against the raycast vertex / normal maps of the
    previous true pose, from that pose."""
    wl = synth.room_512(frames=N_FRAMES_MAX)
    (vs,) = wl.volumes
    frames = _first_frames(frames, n_map + n_track)
    m = Mapper(Config())
    vid = m.add_volume(vs.h, vs.r, vs.s)
    dd = torch.from_numpy(np.stack([f[0] for f in frames[:n_map + n_track]])).cuda()
    dc = torch.from_numpy(np.stack([f[1] for f in frames[:n_map + n_track]])).cuda()
    for k in range(n_map):
        m.integrate(dd[k], dc[k], wl.cam, wl.poses[k])
    maps = m.alloc_maps(wl.cam)
    errs_t, errs_r, ms = [], [], []
    m.set_timing(True)
    m.timings(reset=True)
    for k in range(n_map, n_map + n_track):
        T_prev = wl.poses[k - 1]
        m.raycast(wl.cam, T_prev, out=maps)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        T, last = m.track(dd[k], wl.cam, maps["vertex"], maps["normal"], T_prev, T_prev, iterations=iterations,
                          dist=0.1, cos_min=0.8)
        ms.append((time.perf_counter() - t0) * 1e3)
        T_true = wl.poses[k]
        errs_t.append(float(np.linalg.norm(T[:3, 3] - T_true[:3, 3])))
        R = T[:3, :3] @ T_true[:3, :3].T
        errs_r.append(float(np.degrees(np.arccos(np.clip((np.trace(R) - 1) / 2, -1, 1)))))
    tm = m.timings()
    m.set_timing(False)
    m.close()
    torch.cuda.empty_cache()
    icp = tm.get("icp", (0, 0.0, 0))
    return {"workload": f"room 512^3 after {n_map} frames, {n_track} frames tracked at 640x480, "
                        f"{iterations} ICP iterations from the previous pose",
            "ms_per_track": float(np.median(ms)), "icp_kernel_us": icp[1] / max(icp[2], 1) * 1e3,
            "translation_error_mm_mean": 1e3 * float(np.mean(errs_t)),
            "translation_error_mm_max": 1e3 * float(np.max(errs_t)),
            "rotation_error_deg_mean": float(np.mean(errs_r)), "rotation_error_deg_max": float(np.max(errs_r))}


def main_reference(args, rank):
    """Reference arm: the FP64 CPU oracle, as it stands, on the same workload
    and steps -- whole frames (integration into every voxel of the 512^3
    volume + the raycast of every pixel) from its own state, the same
    measurement as the native arm's cpu_baseline.  Under torchrun only rank 0
    runs it."""
    if rank != 0:
        return
    wl = synth.room_512(frames=N_FRAMES_MAX)
    n = args.warmup + args.steps
    frames = make_frames(n, min(16, os.cpu_count() or 1))
    orc = oracle_run(wl, frames, timed=range(args.warmup, n))
    value = orc["updated"] / orc["seconds"] if orc["seconds"] > 0 else 0.0
    sample = f"{orc['frames']} {ORACLE_SAMPLE}"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * orc["seconds"] / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": CONFIG_OF(args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": orc["cores"], "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-variants", action="store_true", help="skip the f16/i16 storage runs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end run")
    ap.add_argument("--tuning", type=lambda t: tuple(int(x) for x in t.split(",")), default=None,
                    help="fixed raycast tile and integration CTAs per SM (e.g. 0,8) instead of autotuning")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the uneven-volume, differentiable and swap measurements")
    ap.add_argument("--extras", default="uneven,diff,swap,streamed,placement,resolution,tracking",
                    help="comma-separated subset of the extra measurements to run (1-GPU runs only)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return main_reference(args, rank)

    n = args.warmup + 2 * args.steps
    procs = max(1, min(16, (os.cpu_count() or 2) // max(world, 1)))
    frames = make_frames(n, procs)  # before any CUDA call
    extra_steps = 20
    # the extra measurements run on 1-GPU runs only: under torchrun every rank
    # would repeat them, and some pin tens of GB of host memory per process
    extras = set() if (args.no_extra or world > 1) else set(args.extras.split(","))
    if "uneven" in extras:
        uneven_frames = _gen(_render_uneven, range(args.warmup + extra_steps), procs)
    if "diff" in extras:
        tile_frames = _gen(_render_tiles, range(100), procs)
    if "placement" in extras:
        placement_frames = _gen(_render_placement, range(PLACEMENT_FRAMES), procs)

    import torch
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_1511_07106_b300 import Config, Mapper

    wl = synth.room_512(frames=N_FRAMES_MAX)
    cam = wl.cam
    (vs,) = wl.volumes
    poses = [wl.poses[i % N_FRAMES_MAX] for i in range(n)]
    dev_depth = torch.from_numpy(np.stack([f[0] for f in frames])).cuda()
    dev_rgb = torch.from_numpy(np.stack([f[1] for f in frames])).cuda()

    try:
        clocks = ClockSampler("GPU-" + str(torch.cuda.get_device_properties(local_rank).uuid))
    except Exception:
        clocks = ClockSampler(local_rank)
    res = bench_storage(torch, Mapper, Config, wl, poses, "f32", args.warmup, args.steps,
                        dev_depth, dev_rgb, clocks=clocks, tuning=args.tuning)
    ms_max = allreduce_max(torch, res["ms"])
    value = weak_scaling_value(torch, res["stats"]["updated"], res["ms"])
    peak, peak_kind = measured_peaks()
    # kernels of the graph timed region (frame_graph counts graph launches, not kernels)
    launches = sum(v[0] for k, v in res["graph_timings"].items() if k != "frame_graph")
    m = res["mapper"]

    # the FP64 oracle on the host cores (rank 0 of a 1-GPU run): whole frames
    # timed, and the footprint of the raycast's views in the per-kernel pass
    orc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        first_k = args.warmup + args.steps  # the per-kernel (eager) pass raycasts these frames
        fp_at = sorted({first_k + (j * args.steps) // 4 for j in range(4)})
        orc = oracle_run(wl, frames, timed=range(args.warmup, args.warmup + 3), footprint_at=fp_at,
                         one_core_at=args.warmup + 3)
    footprint = None
    if orc and orc["footprints"]:
        footprint = tuple(float(np.mean([f[a] for f in orc["footprints"]])) for a in range(2))
    kern = kernel_summary(res, "f32", cam, args.steps, footprint)
    # the dominant kernel of the hot path (short runs can let launch-bound kernels lead by time)
    dom = max((k for k in kern if k in ("raycast", "integrate")), key=lambda k: kern[k]["avg_ms"] * kern[k]["launches"])
    dk = kern[dom]
    tr = traffic_record(dom)
    roofline = {"kernel": dom, "bound": "hbm", "achieved": dk.get("achieved_gbs"), "peak": peak,
                "unit": "GB/s", "frac": (dk.get("achieved_gbs") or 0.0) / peak,
                "traffic": tr["dram_bytes_per_launch"] if tr else None,
                "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured"
                else "fallback 6.4 TB/s"}
    if dom == "raycast":
        roofline["algorithmic_bytes"] = dk["algorithmic_bytes"]
        roofline["output_bytes"] = dk["output_bytes"]
        roofline["footprint_voxels"] = footprint  # (TSDF+weight voxels, colour voxels), oracle-counted
        roofline["traffic_frac"] = (tr["dram_bytes_per_launch"] / (dk["avg_ms"] * 1e-3) / 1e9 / peak
                                    if tr else None)
    ik = kern.get("integrate", {})
    tri = traffic_record("integrate")
    integrate_roofline = {"bound": "hbm", "achieved": ik.get("achieved_gbs"), "peak": peak,
                          "unit": "GB/s", "frac": (ik.get("achieved_gbs") or 0.0) / peak,
                          "traffic": tri["dram_bytes_per_launch"] if tri else None}
    # integrate + raycast of one frame, time-weighted: summed bytes over summed kernel time
    rk = kern.get("raycast", {})
    trr = traffic_record("raycast")
    t_pair = (ik.get("avg_ms", 0.0) + rk.get("avg_ms", 0.0)) * 1e-3
    frame_hbm = {"kernels": ["integrate", "raycast"], "seconds": t_pair, "peak": peak, "unit": "GB/s",
                 "algorithmic_frac": ((ik.get("algorithmic_bytes", 0) + rk.get("algorithmic_bytes", 0))
                                      / t_pair / 1e9 / peak) if t_pair else None,
                 "dram_frac": ((tri["dram_bytes_per_launch"] + trr["dram_bytes_per_launch"]) / t_pair / 1e9 / peak)
                 if (t_pair and tri and trr) else None}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": CONFIG_OF(world),
            "raycast_mrays_per_s": world * cam.width * cam.height * args.steps / (ms_max * 1e-3) / 1e6,
            "swept_voxel_updates_per_s": world * int(np.prod(vs.r)) * args.steps / (ms_max * 1e-3),
            "updated_voxels_per_frame": res["stats"]["updated"] / args.steps,
            "swept_voxels_per_frame": res["stats"]["swept"] / args.steps,
            "bricks_per_frame": res["stats"]["bricks"] / args.steps,
            "band_voxels_per_frame": res["stats"]["band"] / args.steps,
            "eager_ms_per_step": res["eager_ms"] / args.steps,
            "raycast_samples_per_ray": res["stats"]["ray_samples"] / max(res["stats"]["rays"], 1),
            "raycast_skips_per_ray": res["stats"]["ray_skips"] / max(res["stats"]["rays"], 1),
            "raycast_hit_fraction": res["stats"]["ray_hits"] / max(res["stats"]["rays"], 1),
            "kernels": kern, "roofline": roofline, "integrate_roofline": integrate_roofline,
            "frame_hbm": frame_hbm,
            "tuning": {k: res["tuning"][k] for k in ("raycast_tile", "integrate_ctas_per_sm")},
            "gpu_launches": launches, "clocks": res["clocks"]}
    if orc:
        v1 = orc["one_core"]
        line["cpu_baseline"] = {"value": orc["updated"] / orc["seconds"], "unit": UNIT, "cores": orc["cores"],
                                "kind": "oracle", "sample": f"{orc['frames']} {ORACLE_SAMPLE}",
                                "seconds": orc["seconds"], "ms_per_frame": 1e3 * orc["seconds"] / orc["frames"],
                                "one_core_value": v1[0] / v1[1], "one_core_ms_per_frame": 1e3 * v1[1]}
        line["accuracy"] = accuracy_vs_oracle(torch, Mapper, Config, wl, frames, orc["last_frame"],
                                              dev_depth, dev_rgb, orc["volume"])
        orc = None

    if not args.no_variants:
        variants = {}
        for fmt in ("f16", "i16"):
            r = bench_storage(torch, Mapper, Config, wl, poses, fmt, args.warmup, args.steps,
                              dev_depth, dev_rgb)
            k = kernel_summary(r, fmt, cam, args.steps)
            msx = allreduce_max(torch, r["ms"])
            variants[fmt] = {"value": allreduce_sum(torch, r["stats"]["updated"]) / (msx * 1e-3),
                             "ms_per_step": msx / args.steps,
                             "integrate_ms": k.get("integrate", {}).get("avg_ms"),
                             "integrate_gbs": k.get("integrate", {}).get("achieved_gbs"),
                             "raycast_ms": k.get("raycast", {}).get("avg_ms")}
            r["mapper"].close()
        line["variants"] = variants

    if not args.no_e2e:
        upd, dt, h2d, d2h = e2e_run(torch, Mapper, Config, wl, frames, args.steps, args.warmup)
        dt_max = allreduce_max(torch, dt)
        line["e2e"] = {"value": allreduce_sum(torch, upd) / dt_max, "unit": UNIT,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    if extras:
        m.close()
        torch.cuda.empty_cache()
        if "uneven" in extras:
            line["uneven_volumes"] = bench_uneven(torch, Mapper, Config, uneven_frames, extra_steps, args.warmup,
                                                  with_oracle=rank == 0 and world == 1 and not args.no_cpu_baseline)
        if "diff" in extras:
            line["differentiable"] = bench_diff(torch, Mapper, Config, tile_frames)
        if "swap" in extras:
            line["swap"] = bench_swap(torch, Mapper, Config, frames[:10], 50)
        if "streamed" in extras:
            line["streamed"] = bench_streamed(torch, Mapper, Config, frames)
        if "placement" in extras:
            line["placement"] = bench_placement(torch, Mapper, Config, placement_frames)
        if "resolution" in extras:
            line["resolution"] = bench_resolution(torch, Mapper, Config, frames)
        if "tracking" in extras:
            line["tracking"] = bench_track(torch, Mapper, Config, frames)
        m = None

    if m is not None:
        m.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
