"""torch.autograd wrapper of the SOFT-STE rollout (vcs_soft_rollout /
vcs_backward through the C ABI).

Inputs: the ROM as a weight tensor [n_carts][batch.rom_stride], the RAM at the start of
the rollout [n_envs][128] and the joystick inputs [n_steps][n_envs][5]
(right, left, down, up, fire).  Outputs: RAM [n_steps][n_envs][128] and
screens [n_steps][n_envs][210][160], equal to the hard machine's (Theorem 1).
The backward returns the surrogate gradients (Corollary 1); the ROM gradient
is summed over the envs of each cart.
"""
from __future__ import annotations

import torch

from . import Batch


class SoftRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rom, ram0, u, batch: Batch, tau: float, frame_skip: int):
        n_steps, n_envs = int(u.shape[0]), int(u.shape[1])
        dev = u.device
        ram_out = torch.empty((n_steps, n_envs, 128), dtype=torch.float32, device=dev)
        scr_out = torch.empty((n_steps, n_envs, 210, 160), dtype=torch.float32, device=dev)
        tape = batch.soft_rollout(tau, u.contiguous(), frame_skip, rom_f32=rom.contiguous(),
                                  ram0=ram0.contiguous(), ram_out=ram_out, screen_out=scr_out)
        ctx.tape = tape
        ctx.shapes = (rom.shape, ram0.shape, u.shape)
        return ram_out, scr_out

    @staticmethod
    def backward(ctx, g_ram, g_scr):
        rs, r0s, us = ctx.shapes
        dev = g_ram.device if g_ram is not None else g_scr.device
        g_rom = torch.empty(rs, dtype=torch.float32, device=dev)
        g_ram0 = torch.empty(r0s, dtype=torch.float32, device=dev)
        g_u = torch.empty(us, dtype=torch.float32, device=dev)
        ctx.tape.backward(grad_ram=None if g_ram is None else g_ram.contiguous(),
                          grad_screen=None if g_scr is None else g_scr.contiguous(),
                          grad_ram0=g_ram0, grad_u=g_u, grad_rom_per_cart=g_rom)
        return g_rom, g_ram0, g_u, None, None, None


def soft_rollout(batch: Batch, rom, ram0, u, tau: float, frame_skip: int = 1):
    """Differentiable rollout: returns (ram, screens) as float tensors."""
    return SoftRollout.apply(rom, ram0, u, batch, tau, frame_skip)
