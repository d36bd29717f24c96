"""torch.autograd.Function around the internal force and its hand-written
adjoint: f = f_int(u, udot; mu_e, lambda_e) (Sec. 4.3) forward through
tlfe_internal_force, and the vector-Jacobian products
(K_t^T r, C^T r, r . df/d(mu_e, lambda_e)) backward through tlfe_vjp."""

from __future__ import annotations

import torch

from .tlfe import Mesh


class InternalForce(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mesh: Mesh, u, udot, theta):
        if theta is not None:
            mesh.set_elem_mu_lambda(theta.detach().contiguous())
        f = mesh.internal_force(u.detach().double().contiguous(),
                                None if udot is None else udot.detach().to(mesh.torch_dtype).contiguous())
        ctx.mesh = mesh
        ctx.has_udot = udot is not None
        ctx.has_theta = theta is not None
        ctx.save_for_backward(u, udot if udot is not None else u, theta if theta is not None else u)
        return f

    @staticmethod
    def backward(ctx, gf):
        u, udot, theta = ctx.saved_tensors
        mesh = ctx.mesh
        if ctx.has_theta:
            mesh.set_elem_mu_lambda(theta.detach().contiguous())
        need_u, need_ud, need_th = ctx.needs_input_grad[1], ctx.needs_input_grad[2], ctx.needs_input_grad[3]
        gu, gud, gth = mesh.vjp(u.detach().double().contiguous(),
                                udot.detach().to(mesh.torch_dtype).contiguous() if ctx.has_udot else None,
                                gf.detach().to(mesh.torch_dtype).contiguous(), want_u=True,
                                want_udot=need_ud, want_theta=need_th)
        if gu is not None:
            gu = gu.to(u.dtype)
        if gud is not None:
            gud = gud.to(udot.dtype)
        return (None, gu if need_u else None, gud if (need_ud and ctx.has_udot) else None,
                gth if (need_th and ctx.has_theta) else None)


def internal_force(mesh: Mesh, u, udot=None, theta=None):
    """Differentiable f_int(u, udot, theta): u (n_nodes, 3) displacement (used in
    FP64), udot in the mesh dtype, theta (n_elem, 2) float64 (mu_e, lambda_e)."""
    return InternalForce.apply(mesh, u, udot, theta)


class InterfaceSumFn(torch.autograd.Function):
    """y = x with the rows of the interface nodes summed over the GPUs sharing
    them (shard.InterfaceSum). The sum is linear and symmetric in the ranks,
    so its adjoint is the same sum applied to the cotangent: every rank
    holding an interface node gets the full cotangent there."""

    @staticmethod
    def forward(ctx, x, xs):
        ctx.xs = xs
        y = x.detach().clone().contiguous()
        xs(y)
        return y

    @staticmethod
    def backward(ctx, g):
        g2 = g.detach().clone().contiguous()
        ctx.xs(g2)
        return g2, None


def interface_sum(x, xs):
    """Differentiable interface sum of a split body (see InterfaceSumFn)."""
    return InterfaceSumFn.apply(x, xs)
