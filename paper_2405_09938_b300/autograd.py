"""torch.autograd wrapper of the echo accumulator and its hand-written adjoint.

``HarmEcho.apply(sigma0_cells, uv_cells, scene, n0, np, cell_m, iq_dtype)`` returns
the IQ of pulses [n0, n0 + np) ([n_channels, np, n_range], complex64 or, with
iq_dtype = torch.complex128, complex128) for the per-cell NRCS base
``sigma0_cells`` [ncy, ncx] and current ``uv_cells`` [ncy, ncx, 2] (float64 CUDA
tensors). Its backward runs ``harm_echo_adjoint`` (the transposed scatter as a
gather over range bins, facet states recomputed) and returns the gradients with
respect to both cell fields. The incoming gradient keeps its precision: a
complex128 gradient is passed to the adjoint as a complex128 residual.

With PyTorch's convention for a real loss L of a complex output z, the incoming
gradient is G = dL/dz* (for L = sum |z - t|^2, G = 2 (z - t)), and for a real
parameter theta dL/dtheta = Re sum conj(G) dz/dtheta. The library computes
2 Re sum conj(r) dz/dtheta for a residual r, so it is called with r = G / 2.
"""
from __future__ import annotations

import torch

from . import harm


class HarmEcho(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma0_cells, uv_cells, scene, n0, np_, cell_m, iq_dtype=torch.complex64):
        if sigma0_cells.dtype != torch.float64 or uv_cells.dtype != torch.float64:
            raise harm.HarmError(harm.HARM_E_INVALID, "cell fields must be float64")
        if iq_dtype not in (torch.complex64, torch.complex128):
            raise harm.HarmError(harm.HARM_E_INVALID, "iq_dtype must be complex64 or complex128")
        s0 = sigma0_cells.detach().contiguous()
        uv = uv_cells.detach().contiguous()
        ncy, ncx = s0.shape
        harm.harm_scene_set_cells(scene, ncx, ncy, cell_m, s0, uv)
        d = scene.desc
        iq = torch.empty((len(d["rx"]), np_, d["n_range"]), dtype=iq_dtype, device=s0.device)
        harm.harm_echo_accumulate(scene, n0, np_, iq, zero_first=True)
        ctx.scene, ctx.n0, ctx.np_, ctx.cell_m = scene, n0, np_, cell_m
        ctx.save_for_backward(s0, uv)
        return iq

    @staticmethod
    def backward(ctx, grad_iq):
        s0, uv = ctx.saved_tensors
        ncy, ncx = s0.shape
        harm.harm_scene_set_cells(ctx.scene, ncx, ncy, ctx.cell_m, s0, uv)
        rdt = torch.complex128 if grad_iq.dtype == torch.complex128 else torch.complex64
        resid = (0.5 * grad_iq).to(rdt).contiguous()
        gs = torch.zeros_like(s0)
        guv = torch.zeros_like(uv)
        harm.harm_echo_adjoint(ctx.scene, ctx.n0, ctx.np_, resid, gs, guv)
        return gs, guv, None, None, None, None, None


def echo(sigma0_cells, uv_cells, scene, n0, np_, cell_m, iq_dtype=torch.complex64):
    """Differentiable IQ of pulses [n0, n0 + np) for per-cell NRCS and current
    (complex64, or complex128 with iq_dtype = torch.complex128)."""
    return HarmEcho.apply(sigma0_cells, uv_cells, scene, n0, np_, cell_m, iq_dtype)
