"""torch.autograd.Function for the MBD energy: forward runs mbd_energy_forces,
backward returns the gradient dE/dR = -F that the force kernels computed."""
from __future__ import annotations

import torch

from .system import MBDSystem


class MBDEnergy(torch.autograd.Function):
    """E_MBD(R) for positions R [N, 3] (float64); the system's geometry is set to R."""

    @staticmethod
    def forward(ctx, positions: torch.Tensor, system: MBDSystem, n_probes: int, n_steps: int, seed: int):
        system.update_positions(positions.detach().cpu().numpy())
        energy, forces = system.energy_forces(n_probes, n_steps, seed)
        ctx.save_for_backward(forces)
        ctx.out_device = positions.device
        return torch.tensor(energy, dtype=torch.float64, device=positions.device)

    @staticmethod
    def backward(ctx, grad_out):
        (forces,) = ctx.saved_tensors
        grad = (-forces).to(ctx.out_device) * grad_out
        return grad, None, None, None, None


def mbd_energy(positions: torch.Tensor, system: MBDSystem, n_probes: int, n_steps: int, seed: int) -> torch.Tensor:
    return MBDEnergy.apply(positions, system, n_probes, n_steps, seed)
