"""``torch.autograd.Function`` around ``dp_compute_device``.

The forward pass runs the whole DPA-1 path on the GPU, including the
hand-written adjoint kernels, and keeps the forces and the virial.  The
backward pass returns, for the coordinates, -dL/dE * F (F = -dE/dx,
Eq. eq_forceGradE) and, for the box, dL/dE * dE/dh at fixed Cartesian
coordinates.  PyTorch only provides device memory and the stream.

Box gradient.  With h the cell (rows = cell vectors) every pair displacement
is r_ij = x_j - x_i + n_ij h for an integer image vector n_ij, so
dE/dh = sum_ij n_ij^T (dE/dr_ij).  The virial W = -sum_ij r_ij (x) dE/dr_ij
splits into the coordinate part, -sum_k x_k (x) dE/dx_k = sum_k x_k (x) F_k,
and h^T dE/dh, hence dE/dh = h^{-T} (sum_k x_k (x) F_k - W).  Without
periodic images this is zero, which is the identity W = sum_k x_k (x) F_k
of an isolated system.
"""

from __future__ import annotations

import torch

from .binding import DPA1


def box_gradient(coord: torch.Tensor, box: torch.Tensor, force: torch.Tensor, virial: torch.Tensor) -> torch.Tensor:
    """dE/dh [9] (row-major, h = box.view(3, 3)) from the coordinates the
    call was given, its forces and its virial (all float64)."""
    h = box.reshape(3, 3).to(torch.float64)
    xf = coord.to(torch.float64).transpose(0, 1) @ force.to(torch.float64)
    return torch.linalg.solve(h.transpose(0, 1), xf - virial.reshape(3, 3).to(torch.float64)).reshape(9)


class DPA1Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coord: torch.Tensor, model: DPA1, box: torch.Tensor, atype: torch.Tensor):
        n = coord.shape[0]
        c = coord.detach().to(torch.float64).contiguous()
        b = box.detach().to(torch.float64).contiguous()
        energy = torch.zeros(1, dtype=torch.float64, device=coord.device)
        force = torch.empty((n, 3), dtype=torch.float64, device=coord.device)
        virial = torch.empty(9, dtype=torch.float64, device=coord.device)
        model.compute_device(c, b, atype, energy, force, virial)
        ctx.save_for_backward(c, b, force, virial)
        ctx.box_dtype = box.dtype
        return energy[0].to(coord.dtype)

    @staticmethod
    def backward(ctx, grad_e):
        c, b, force, virial = ctx.saved_tensors
        g_coord = (-grad_e * force).to(grad_e.dtype)
        g_box = None
        if ctx.needs_input_grad[2]:
            g_box = (grad_e * box_gradient(c, b, force, virial)).to(ctx.box_dtype)
        return g_coord, None, g_box, None


def energy(coord: torch.Tensor, model: DPA1, box: torch.Tensor, atype: torch.Tensor) -> torch.Tensor:
    return DPA1Energy.apply(coord, model, box, atype)
