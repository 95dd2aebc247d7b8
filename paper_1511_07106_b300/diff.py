"""Differentiable raycast: torch.autograd.Function over the library's raycast.

Not in the paper: rendered depth/colour of the TSDF volumes as a function of
the camera poses (and of the TSDF values), for gradient-based pose refinement.
The forward pass is ``mv_raycast_batch`` (one CUDA launch for all views);
the backward pass is ``mv_raycast_backward`` (one launch for all views), which
re-derives each hit from the saved depth and volume id.  Colour is differentiated as the
unrounded trilinear colour (the 8-bit rounding of the forward is passed
straight through).

The library returns dL/dxi for the left perturbation T(xi) = exp(xi^) T.  The
Function's input is the 4x4 pose itself; it returns dL/dT as the tangent-space
vector field with exactly those directional derivatives, so any smooth
parametrisation of T built in torch (e.g. ``pose_from_twist``) gets the exact
gradient by autograd.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi
from .mapper import Mapper, intrinsics


def _generators(dtype=torch.float64, device="cpu"):
    """se(3) generators G_k with xi^ = sum_k xi_k G_k, xi = (rho, phi)."""
    G = torch.zeros(6, 4, 4, dtype=dtype, device=device)
    for k in range(3):
        G[k, k, 3] = 1.0
    # [e_x]_x, [e_y]_x, [e_z]_x
    G[3, 1, 2], G[3, 2, 1] = -1.0, 1.0
    G[4, 0, 2], G[4, 2, 0] = 1.0, -1.0
    G[5, 0, 1], G[5, 1, 0] = -1.0, 1.0
    return G


def hat(xi: torch.Tensor) -> torch.Tensor:
    """(..., 6) twists -> (..., 4, 4) matrices xi^."""
    G = _generators(xi.dtype, xi.device)
    return torch.einsum("...k,kij->...ij", xi, G)


def pose_from_twist(xi: torch.Tensor, T0: torch.Tensor) -> torch.Tensor:
    """T = exp(xi^) T0 (differentiable in xi)."""
    return torch.matrix_exp(hat(xi)) @ T0


def tangent_cotangent(T: torch.Tensor, g_xi: torch.Tensor) -> torch.Tensor:
    """dL/dT whose Frobenius pairing with the tangent directions G_k T gives
    g_xi[k] exactly, taken in their span: sum_k c_k G_k T with the Gram
    system of the directions solved in closed form.  For T = [R | t] with R
    orthonormal the Gram matrix is [[I, C], [C^T, (2 + |t|^2) I - t t^T]]
    with C e_j = e_j x t, whose Schur complement is 2 I; so c_phi =
    (g_phi - t x g_rho) / 2, c_rho = g_rho - c_phi x t, and
    dL/dT = [[c_phi]_x R, g_rho; 0, 0]."""
    R, t = T[:, :3, :3], T[:, :3, 3]
    g_rho, g_phi = g_xi[:, :3], g_xi[:, 3:]
    c = 0.5 * (g_phi - torch.cross(t, g_rho, dim=1))
    out = torch.zeros_like(T)
    out[:, :3, :3] = hat_so3(c) @ R
    out[:, :3, 3] = g_rho
    return out


def hat_so3(w: torch.Tensor) -> torch.Tensor:
    """(n, 3) -> (n, 3, 3) cross-product matrices [w]_x."""
    z = torch.zeros_like(w[:, 0])
    return torch.stack([torch.stack([z, -w[:, 2], w[:, 1]], -1),
                        torch.stack([w[:, 2], z, -w[:, 0]], -1),
                        torch.stack([-w[:, 1], w[:, 0], z], -1)], -2)


class RaycastFn(torch.autograd.Function):
    """depth (n, H, W), colour (n, H, W, 3) in [0, 1] = f(T (n, 4, 4), *tsdf).

    ``tsdf`` are placeholder leaves, one per entry of ``tsdf_ids``, shaped like
    each volume (h_r[2], h_r[1], h_r[0]); their .grad receives dL/dF."""

    @staticmethod
    def forward(ctx, T, mapper: Mapper, cam, tsdf_ids, *tsdf):
        n = T.shape[0]
        H, W = cam.height, cam.width
        dev = torch.device("cuda", mapper.device)
        depth = torch.empty((n, H, W), dtype=torch.float32, device=dev)
        vid = torch.empty((n, H, W), dtype=torch.int32, device=dev)
        rgba = torch.empty((n, H, W, 4), dtype=torch.uint8, device=dev)
        Tn = T.detach().to("cpu", torch.float64).contiguous().numpy()
        mapper.raycast_batch(cam, Tn, out={"depth": depth, "vol_id": vid, "rgba": rgba})
        colour = rgba[..., :3].float() / 255.0
        ctx.mapper, ctx.cam, ctx.tsdf_ids = mapper, cam, list(tsdf_ids)
        ctx.poses = Tn
        ctx.tsdf_shapes = [t.shape for t in tsdf]
        ctx.save_for_backward(T, depth, vid)
        ctx.mark_non_differentiable(vid)
        return depth, colour

    @staticmethod
    def backward(ctx, g_depth, g_colour):
        T, depth, vid = ctx.saved_tensors
        mapper, cam = ctx.mapper, ctx.cam
        n = T.shape[0]
        dev = depth.device
        gd = None if g_depth is None else g_depth.contiguous().float()
        gc = None if g_colour is None else g_colour.contiguous().float()
        grad_xi = torch.zeros((n, 6), dtype=torch.float32, device=dev)
        gts = [torch.zeros(s, dtype=torch.float32, device=dev) for s in ctx.tsdf_shapes]
        mapper.raycast_backward(cam, ctx.poses, depth, vid, gd, gc, grad_xi,
                                dict(zip(ctx.tsdf_ids, gts)))
        # dL/dT on the pose's own device (a closed form: no linear solve)
        gT = tangent_cotangent(T.detach().to(torch.float64), grad_xi.to(T.device, torch.float64))
        return (gT.to(T.dtype), None, None, None, *gts)


def render(mapper: Mapper, cam, T: torch.Tensor, tsdf=None):
    """Differentiable render of the mapper's volumes at poses T (n, 4, 4).
    tsdf: optional {volume id: placeholder leaf} for TSDF gradients."""
    tsdf = tsdf or {}
    return RaycastFn.apply(T, mapper, cam, list(tsdf.keys()), *tsdf.values())


def tsdf_leaf(mapper: Mapper, vid: int) -> torch.Tensor:
    """A zero tensor shaped like volume vid whose .grad receives dL/dF."""
    rx, ry, rz = mapper.query(vid)["h_r"]
    return torch.zeros((rz, ry, rx), dtype=torch.float32, device=torch.device("cuda", mapper.device),
                       requires_grad=True)


def l1_loss(depth, colour, ref_depth, ref_colour, colour_weight=0.1):
    """Mean L1 over pixels valid in both renders: depth + colour_weight * colour."""
    valid = (depth > 0) & (ref_depth > 0)
    nv = valid.sum().clamp(min=1)
    ld = (torch.abs(depth - ref_depth) * valid).sum() / nv
    lc = (torch.abs(colour - ref_colour).sum(-1) * valid).sum() / nv
    return ld + colour_weight * lc


def l1_loss_grad(depth, colour, ref_depth, ref_colour, colour_weight=0.1):
    """l1_loss and its gradients with respect to depth and colour in closed
    form (what autograd returns: the derivative of |x| is sign(x), 0 at 0):
    (loss as a 0-d tensor, dL/ddepth, dL/dcolour)."""
    valid = (depth > 0) & (ref_depth > 0)
    w = valid / valid.sum().clamp(min=1)
    dd = depth - ref_depth
    dc = colour - ref_colour
    loss = (torch.abs(dd) * w).sum() + colour_weight * (torch.abs(dc).sum(-1) * w).sum()
    return loss, torch.sign(dd) * w, (colour_weight * torch.sign(dc)) * w[..., None]


def so3_exp(phi: np.ndarray) -> np.ndarray:
    """(n, 3) rotation vectors -> (n, 3, 3) rotations (Rodrigues; below 1e-4
    rad the coefficients from their Maclaurin series)."""
    th2 = np.sum(phi * phi, axis=1)[:, None, None]
    small = th2 < 1e-8
    th = np.sqrt(np.where(small, 1.0, th2))
    a = np.where(small, 1.0 - th2 / 6.0, np.sin(th) / th)
    b = np.where(small, 0.5 - th2 / 24.0, (1.0 - np.cos(th)) / np.where(small, 1.0, th2))
    K = np.zeros((phi.shape[0], 3, 3))
    K[:, 0, 1], K[:, 0, 2], K[:, 1, 2] = -phi[:, 2], phi[:, 1], -phi[:, 0]
    K[:, 1, 0], K[:, 2, 0], K[:, 2, 1] = phi[:, 2], -phi[:, 1], phi[:, 0]
    return np.eye(3)[None] + a * K + b * (K @ K)


def centred_gradient(t: torch.Tensor, g_xi: torch.Tensor) -> torch.Tensor:
    """Gradient in camera-centred coordinates (translation rho_c of the camera
    centre, rotation phi_c about it: R' = exp(phi_c) R, t' = t + rho_c) from
    the gradient g_xi = (g_rho, g_phi) of the left perturbation exp(xi^) T,
    whose rotation turns about the world origin: to first order rho = rho_c -
    phi_c x t, so the centred gradient is (g_rho, g_phi - t x g_rho).  t, g_xi:
    (n, 3), (n, 6)."""
    return torch.cat([g_xi[:, :3], g_xi[:, 3:] - torch.cross(t, g_xi[:, :3], dim=1)], dim=1)


def refine_poses(mapper: Mapper, cam, T_init, ref_depth, ref_colour, steps=50, lr=(3e-3, 1.5e-3),
                 colour_weight=0.1, callback=None, lr_final=1.0, centred=True, fused=True):
    """Pose refinement by Adam in the tangent space of each pose.  Every step
    renders the n views at the current poses (mv_raycast_batch), takes the
    loss l1_loss against the reference renders and, from the loss's gradients
    with respect to the rendered depth and colour, its gradient with respect
    to the left perturbation xi = (rho, phi) of every pose at xi = 0
    (mv_raycast_backward returns exactly that, so no tangent-space solve is
    needed).  With `centred` the step is taken in coordinates centred on the
    camera -- a rotation phi_c about the camera centre and a translation rho_c
    of it, R <- exp(phi_c) R, t <- t + rho_c -- whose gradient is
    (g_rho, g_phi - t x g_rho): a rotation step then no longer moves the camera
    centre, which the left perturbation's rotation about the world origin does
    (by phi x t), coupling the two blocks for cameras far from the origin.
    The loss's gradients come in closed form (l1_loss_grad); each step reads
    the n x 6 pose gradient back once, and Adam and the pose update run on
    the host (the poses are host data of mv_raycast_batch anyway).  lr:
    (metres, radians) per step for translation and rotation, or one number
    for both, decayed by a cosine from lr to lr * lr_final over the steps
    (lr_final = 1: constant, which did best on the 8 x 256^3 workload, as did
    centred steps).  With `fused` the loss, its gradients and the backward
    are one library call (mv_raycast_backward_l1: the same gradient bits,
    without the per-pixel gradient tensors); otherwise l1_loss_grad and
    mv_raycast_backward.  Returns (T_final (n, 4, 4) float64 numpy, losses)."""
    import math
    dev = torch.device("cuda", mapper.device)
    T = np.array(T_init, dtype=np.float64)
    n = T.shape[0]
    lr_t, lr_r = (lr, lr) if np.isscalar(lr) else lr
    rate = np.array([lr_t] * 3 + [lr_r] * 3, dtype=np.float64)
    m1 = np.zeros((n, 6))
    m2 = np.zeros((n, 6))
    b1, b2, eps = 0.9, 0.999, 1e-12
    H, W = cam.height, cam.width
    out = dict(depth=torch.empty((n, H, W), dtype=torch.float32, device=dev),
               rgba=torch.empty((n, H, W, 4), dtype=torch.uint8, device=dev),
               vol_id=torch.empty((n, H, W), dtype=torch.int32, device=dev))
    grad_xi = torch.empty((n, 6), dtype=torch.float32, device=dev)
    if fused:
        # the reference colour back to its bytes (c = byte / 255 exactly
        # recovers them), so that equal colours compare equal on the device
        ref_rgba = torch.zeros((n, H, W, 4), dtype=torch.uint8, device=dev)
        ref_rgba[..., :3] = torch.round(ref_colour * 255.0).clamp(0, 255).to(torch.uint8)
        ref_d = ref_depth.contiguous()
        loss_t = torch.empty(1, dtype=torch.float32, device=dev)
    losses = []
    for it in range(steps):
        mapper.raycast_batch(cam, T, out=out)
        if fused:
            mapper.raycast_backward_l1(cam, T, out["depth"], out["rgba"], out["vol_id"], ref_d, ref_rgba,
                                       colour_weight, grad_xi, loss_t)
            loss = loss_t
        else:
            colour = out["rgba"][..., :3].float() / 255.0
            loss, gd, gc = l1_loss_grad(out["depth"], colour, ref_depth, ref_colour, colour_weight)
            mapper.raycast_backward(cam, T, out["depth"], out["vol_id"], gd, gc, grad_xi, {})
        # the step's one read-back: the pose gradient, for Adam on the host
        g = grad_xi.cpu().numpy().astype(np.float64)
        if centred:
            g = np.concatenate([g[:, :3], g[:, 3:] - np.cross(T[:, :3, 3], g[:, :3])], axis=1)
        m1 = b1 * m1 + (1 - b1) * g
        m2 = b2 * m2 + (1 - b2) * g * g
        scale = lr_final + (1 - lr_final) * 0.5 * (1 + math.cos(math.pi * it / max(steps - 1, 1)))
        delta = -(rate * scale) * (m1 / (1 - b1 ** (it + 1))) / (np.sqrt(m2 / (1 - b2 ** (it + 1))) + eps)
        T = T.copy()
        if centred:
            T[:, :3, :3] = so3_exp(delta[:, 3:]) @ T[:, :3, :3]
            T[:, :3, 3] = T[:, :3, 3] + delta[:, :3]
        else:
            T = torch.matrix_exp(hat(torch.from_numpy(delta))).numpy() @ T
        losses.append(float(loss))
        if callback:
            callback(it, T.copy(), losses[-1])
    return T, losses
