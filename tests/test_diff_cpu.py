"""Host-side pieces of the differentiable raycast (CPU): the se(3) helpers
and the change of tangent coordinates used by the pose refinement, checked
against torch autograd on a smooth function of the pose."""
import numpy as np
import torch

from paper_1511_07106_b300 import diff


def smooth_loss(T):
    p = torch.tensor([0.3, -0.2, 1.1], dtype=torch.float64)
    x = T[:3, :3] @ p + T[:3, 3]
    w = torch.arange(9, dtype=torch.float64).reshape(3, 3)
    return (x ** 3).sum() + 0.1 * (T[:3, :3] ** 2 * w).sum()


def test_centred_gradient_matches_autograd():
    """d/d(rho_c, phi_c) of L(R' = exp(phi_c) R, t' = t + rho_c) at 0 equals
    centred_gradient(t, dL/dxi) of the left perturbation exp(xi^) T."""
    torch.manual_seed(0)
    G = diff._generators(torch.float64)
    for _ in range(5):
        T0 = diff.pose_from_twist(torch.randn(6, dtype=torch.float64) * 0.7, torch.eye(4, dtype=torch.float64))
        T0[:3, 3] += torch.randn(3, dtype=torch.float64) * 2.0  # a camera far from the origin
        xi = torch.zeros(6, dtype=torch.float64, requires_grad=True)
        smooth_loss(diff.pose_from_twist(xi, T0)).backward()
        d = torch.zeros(6, dtype=torch.float64, requires_grad=True)
        R = torch.matrix_exp(torch.einsum("k,kij->ij", d[3:], G[3:, :3, :3])) @ T0[:3, :3]
        T = torch.cat([torch.cat([R, (T0[:3, 3] + d[:3])[:, None]], 1), T0[3:]], 0)
        smooth_loss(T).backward()
        got = diff.centred_gradient(T0[None, :3, 3], xi.grad[None])[0]
        np.testing.assert_allclose(got.numpy(), d.grad.numpy(), rtol=1e-12, atol=1e-12)


def test_tangent_cotangent_pairs_with_generators():
    """dL/dT from tangent_cotangent pairs with each tangent direction G_k T to
    give back the k-th component of the twist gradient."""
    torch.manual_seed(1)
    T = diff.pose_from_twist(torch.randn(2, 6, dtype=torch.float64) * 0.5, torch.eye(4, dtype=torch.float64))
    g = torch.randn(2, 6, dtype=torch.float64)
    gT = diff.tangent_cotangent(T, g)
    G = diff._generators(torch.float64)
    for n in range(2):
        for k in range(6):
            assert abs(float((gT[n] * (G[k] @ T[n])).sum()) - float(g[n, k])) < 1e-12


def test_tangent_cotangent_closed_form_equals_the_gram_solve():
    """The closed form (Schur complement 2 I) equals solving the 6 x 6 Gram
    system of the tangent directions G_k T, for poses far from the origin."""
    torch.manual_seed(2)
    n = 6
    T = diff.pose_from_twist(torch.randn(n, 6, dtype=torch.float64) * 0.8, torch.eye(4, dtype=torch.float64))
    T[:, :3, 3] += torch.randn(n, 3, dtype=torch.float64) * 3.0
    g = torch.randn(n, 6, dtype=torch.float64)
    G = diff._generators(torch.float64)
    B = torch.einsum("kij,njl->nkil", G, T).reshape(n, 6, 16)
    coeff = torch.linalg.solve(B @ B.transpose(1, 2), g.unsqueeze(-1)).squeeze(-1)
    ref = (coeff.unsqueeze(-1) * B).sum(1).reshape(-1, 4, 4)
    np.testing.assert_allclose(diff.tangent_cotangent(T, g).numpy(), ref.numpy(), rtol=0, atol=1e-12)


def test_l1_loss_grad_equals_autograd():
    """The closed-form gradient of the refinement loss equals autograd's,
    including pixels invalid in either render and exact zeros of the
    differences (where the derivative of |x| is taken as 0)."""
    g = torch.Generator().manual_seed(3)
    n, H, W = 2, 7, 9
    depth = torch.rand((n, H, W), generator=g, dtype=torch.float32) + 0.5
    ref = depth + 0.05 * torch.randn((n, H, W), generator=g)
    depth[0, :2] = 0.0
    ref[1, :, :3] = 0.0
    ref[0, 5, 5] = depth[0, 5, 5]  # an exact zero of the difference
    col = torch.rand((n, H, W, 3), generator=g)
    rcol = torch.rand((n, H, W, 3), generator=g)
    rcol[1, 2, 2] = col[1, 2, 2]
    d = depth.clone().requires_grad_(True)
    c = col.clone().requires_grad_(True)
    loss = diff.l1_loss(d, c, ref, rcol, 0.1)
    gd, gc = torch.autograd.grad(loss, (d, c))
    loss2, gd2, gc2 = diff.l1_loss_grad(depth, col, ref, rcol, 0.1)
    torch.testing.assert_close(loss2, loss.detach(), rtol=1e-6, atol=0)
    torch.testing.assert_close(gd2, gd, rtol=0, atol=0)
    torch.testing.assert_close(gc2, gc, rtol=0, atol=0)


def test_so3_exp_equals_matrix_exponential():
    rng = np.random.default_rng(4)
    phi = np.concatenate([rng.normal(size=(5, 3)) * s for s in (1.0, 1e-3, 1e-5)] + [np.zeros((1, 3))])
    got = diff.so3_exp(phi)
    want = torch.matrix_exp(diff.hat_so3(torch.from_numpy(phi))).numpy()
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)


def test_float_colours_give_back_their_bytes_and_byte_order():
    """The fused L1 path (mv_raycast_backward_l1) takes colours as the forward's
    bytes while the closed form (l1_loss_grad) takes them as byte / 255 in
    float32: every byte comes back from its float by round(c * 255), and the
    sign of a float difference is the sign of the byte difference for all
    65536 pairs, so both give each pixel the same colour gradient."""
    import torch
    b = torch.arange(256, dtype=torch.uint8)
    c = b.float() / 255.0
    assert torch.equal(torch.round(c * 255.0).to(torch.uint8), b)
    a_f, b_f = c[:, None], c[None, :]
    a_i, b_i = b.to(torch.int32)[:, None], b.to(torch.int32)[None, :]
    assert torch.equal(torch.sign(a_f - b_f), torch.sign(a_i - b_i).float())
