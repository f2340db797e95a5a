"""``torch.autograd.Function`` around ``dp_compute_device``.

The forward pass runs the whole DPA-1 path on the GPU, including the
hand-written adjoint kernels, and keeps the forces and the virial; the
backward pass returns -dL/dE * F for the coordinates (F = -dE/dx,
Eq. eq_forceGradE).  PyTorch only provides device memory and the stream.
"""

from __future__ import annotations

import torch

from .binding import DPA1


class DPA1Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coord: torch.Tensor, model: DPA1, box: torch.Tensor, atype: torch.Tensor):
        n = coord.shape[0]
        c = coord.detach().to(torch.float64).contiguous()
        energy = torch.zeros(1, dtype=torch.float64, device=coord.device)
        force = torch.empty((n, 3), dtype=torch.float64, device=coord.device)
        virial = torch.empty(9, dtype=torch.float64, device=coord.device)
        model.compute_device(c, box, atype, energy, force, virial)
        ctx.save_for_backward(force)
        ctx.virial = virial
        return energy[0].to(coord.dtype)

    @staticmethod
    def backward(ctx, grad_e):
        (force,) = ctx.saved_tensors
        return (-grad_e * force).to(grad_e.dtype), None, None, None


def energy(coord: torch.Tensor, model: DPA1, box: torch.Tensor, atype: torch.Tensor) -> torch.Tensor:
    return DPA1Energy.apply(coord, model, box, atype)
