"""Differentiable Wilson operator, normal-equation solve and pseudofermion action.

Forward and backward passes call libcola's kernels: D and D^dag through the
packed hopping kernel, the link gradient through the spin-traced outer-product
kernel, solves through the CG.  Complex gradients follow torch's convention
(grad = 2 dL/d conj(z)).  The backward of a solve runs a second (adjoint)
solve instead of storing anything per CG iteration.

For X = A^-1 phi with A = D^dag D, a real loss L with upstream gX gives
  Z = A^-1 gX,  grad_phi = Z,
  grad_U = -(G(Z, D X) + G(X, D Z)),
where G(psi, g) is the link gradient of Re<g, D psi> (dirac_link_grad), from
dA = dD^dag D + D^dag dD.
"""
from __future__ import annotations

import torch

from .api import Gauge, apply_dirac, cg_solve, dirac_link_grad


def _gauge(links, dims, kappa, bc, precisions=("f64",)):
    return Gauge(links.detach().contiguous(), dims, kappa, bc, precisions=precisions, recon={"f64": 18, "f32": 12})


class DiracOp(torch.autograd.Function):
    """y = D[U] psi on canonical complex128 fields (csw != 0: D = A - kappa H).

    Gradients with respect to psi (D^dag gy) and to the links (the raw complex
    gradient, hopping and clover parts) in PyTorch's convention.
    """

    @staticmethod
    def forward(ctx, links, psi, dims, kappa, bc, csw=0.0):
        g = _gauge(links, dims, kappa, bc)
        if csw:
            g.attach_clover(csw)
        psi_c = psi.detach().contiguous()
        y = apply_dirac(g, psi_c)
        ctx.save_for_backward(psi_c)
        ctx.g = g
        return y

    @staticmethod
    def backward(ctx, gy):
        (psi,) = ctx.saved_tensors
        g = ctx.g
        gy = gy.contiguous()
        grad_links = dirac_link_grad(g, psi, gy) if ctx.needs_input_grad[0] else None
        grad_psi = apply_dirac(g, gy, dagger=True) if ctx.needs_input_grad[1] else None
        return grad_links, grad_psi, None, None, None, None


def _solve(g, rhs, tol, inner):
    x, info = cg_solve(g, rhs, tol=tol, op="full", system="normal", inner=inner, delta=0.1)
    return x, info


class SolveNormal(torch.autograd.Function):
    """X = (D^dag D)^-1 phi on the whole lattice (csw != 0: D = A - kappa H)."""

    @staticmethod
    def forward(ctx, links, phi, dims, kappa, bc, tol=1e-12, inner="f32", csw=0.0):
        g = _gauge(links, dims, kappa, bc, precisions=("f64", "f32") if inner != "f64" else ("f64",))
        if csw:
            g.attach_clover(csw)
        x, _ = _solve(g, phi.detach().contiguous(), tol, inner)
        ctx.save_for_backward(x)
        ctx.g, ctx.tol, ctx.inner = g, tol, inner
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        g = ctx.g
        z, _ = _solve(g, gx.contiguous(), ctx.tol, ctx.inner)
        grad_links = None
        if ctx.needs_input_grad[0]:
            y = apply_dirac(g, x)
            w = apply_dirac(g, z)
            grad_links = -(dirac_link_grad(g, z, y) + dirac_link_grad(g, x, w))
        return grad_links, z, None, None, None, None, None, None


class PseudofermionAction(torch.autograd.Function):
    """S = phi^dag (D^dag D)^-1 phi (real; csw != 0: D = A - kappa H); dS/dU is the fermion force."""

    @staticmethod
    def forward(ctx, links, phi, dims, kappa, bc, tol=1e-12, inner="f32", csw=0.0):
        g = _gauge(links, dims, kappa, bc, precisions=("f64", "f32") if inner != "f64" else ("f64",))
        if csw:
            g.attach_clover(csw)
        x, _ = _solve(g, phi.detach().contiguous(), tol, inner)
        ctx.save_for_backward(x)
        ctx.g = g
        return torch.vdot(phi.detach().reshape(-1), x.reshape(-1)).real

    @staticmethod
    def backward(ctx, gs):
        (x,) = ctx.saved_tensors
        g = ctx.g
        grad_links = grad_phi = None
        if ctx.needs_input_grad[0]:
            y = apply_dirac(g, x)
            grad_links = -2.0 * gs * dirac_link_grad(g, x, y)
        if ctx.needs_input_grad[1]:
            grad_phi = 2.0 * gs * x
        return grad_links, grad_phi, None, None, None, None, None, None
