"""torch.autograd wrappers for DSC and the dictionary, with hand-written backward
passes that run in the CUDA library.

DSC computes y = M(D) w (Eq. 1 with Eq. 3-4).  For a loss L(y) with upstream
gradient gy = dL/dy, the chain rule through y[θ,v] = Σ_{(a,v,f)} D[θ,a]·val·w[f]
gives

    dL/dw[f]   = Σ_{(a,v,f)} val · Σ_θ D[θ,a] gy[θ,v]   = (M^T gy)[f]   (the WC kernel)
    dL/dD[θ,a] = Σ_{(a,v,f)} val · w[f] · gy[θ,v]                      (life_dsc_grad_D)

and, through the dictionary of canonical diffusion atoms built from the axial
diffusivity λ (D = column-demeaned exp(-b λ (g_θ·u_a)^2)),

    dL/dλ = Σ_{θ,a} dL/dD[θ,a] · dD[θ,a]/dλ                           (life_dot_f32)

where dD/dλ is itself demeaned, which carries the demeaning's Jacobian (a
symmetric projection) into the sum.
"""
from __future__ import annotations

import torch

from ._native import LifeIndex, life_dictionary, life_dot_f32, life_dsc, life_dsc_grad_D, life_wc


class LifeDSC(torch.autograd.Function):
    """y = M(D) w as a differentiable op: ``LifeDSC.apply(index, D, w)``.

    D is float32 [Nθ·Na] column-major, w float32 [Nf]; y is float32 [Nθ·Nv].
    The index (Phi) is a constant of the op.
    """

    @staticmethod
    def forward(ctx, index: LifeIndex, D: torch.Tensor, w: torch.Tensor):
        D = D.contiguous()
        w = w.contiguous()
        y, _ = life_dsc(index, D, w)
        ctx.index = index
        ctx.save_for_backward(D, w)
        return y

    @staticmethod
    def backward(ctx, gy: torch.Tensor):
        D, w = ctx.saved_tensors
        gy = gy.contiguous()
        gD = gw = None
        if ctx.needs_input_grad[2]:
            gw, _ = life_wc(ctx.index, D, gy)
        if ctx.needs_input_grad[1]:
            gD = life_dsc_grad_D(ctx.index, gy, w)
        return None, gD, gw


class LifeDictionary(torch.autograd.Function):
    """D(λ) as a differentiable op: ``LifeDictionary.apply(lam, grad_dirs, atom_dirs, bval)``.

    ``lam`` is a one-element tensor (its value is read on the host to build D);
    grad_dirs [Nθ,3] and atom_dirs [Na,3] are unit vectors; bval is a float.
    Returns D float32 [Nθ·Na] column-major.
    """

    @staticmethod
    def forward(ctx, lam: torch.Tensor, grad_dirs, atom_dirs, bval: float):
        need = ctx.needs_input_grad[0]
        D, dD = life_dictionary(grad_dirs, atom_dirs, bval, float(lam.detach().reshape(-1)[0].item()),
                                with_derivative=need)
        ctx.lam_meta = (lam.shape, lam.dtype, lam.device)
        if need:
            ctx.save_for_backward(dD)
        return D

    @staticmethod
    def backward(ctx, gD: torch.Tensor):
        (dD,) = ctx.saved_tensors
        shape, dtype, device = ctx.lam_meta
        glam = life_dot_f32(gD.contiguous(), dD)
        return glam.reshape(shape).to(device=device, dtype=dtype), None, None, None


def dsc(index: LifeIndex, D: torch.Tensor, w: torch.Tensor) -> torch.Tensor:
    """Differentiable y = M(D) w."""
    return LifeDSC.apply(index, D, w)


def dictionary(lam: torch.Tensor, grad_dirs, atom_dirs, bval: float) -> torch.Tensor:
    """Differentiable dictionary D(λ)."""
    return LifeDictionary.apply(lam, grad_dirs, atom_dirs, bval)
