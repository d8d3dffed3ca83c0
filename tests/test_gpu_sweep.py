"""The soft backward's two reverse sweeps (vcs_config.sweep_mode): one env
per warp (k_soft_sweep) and one env per lane (k_soft_sweep_lanes) apply the
same per-record arithmetic to each env's tape in the same order, so every
gradient output must be the same bits.  Covered: several checkpoint
segments (the carry between sweeps), Superchip and E0 carts (the Superchip's
RAM adjoints), the whole TIA with the graphics-bit surrogate, the position
sampler, instruction-granular steps with loss weights, and env counts that
leave a block partly filled.  The sweeps' gradients themselves are checked
against the FP64 oracle in the soft-mode tests.
"""
import numpy as np
import pytest

from paper_2606_22447_b300 import synth
from tests.gpu_util import gpu_rollout, make_batch, torch_cuda

pytestmark = pytest.mark.gpu


def _run(roms, mappers, env_cart, sweep_mode, n_steps, frame_skip, tau, warm, per_step, cfg):
    torch = torch_cuda()
    n_envs = len(env_cart)
    b = make_batch(roms, mappers, env_cart, sweep_mode=sweep_mode, **cfg)
    if warm:
        gpu_rollout(b, synth.actions(warm, n_envs, 2), 1, screens=False)
    u = torch.from_numpy(synth.action_inputs(synth.actions(91, n_envs, n_steps))).cuda()
    tape = b.soft_rollout(tau, u, frame_skip)
    out = {"grad_rom": torch.full((n_envs, 32768), 7.0, device="cuda"),
           "grad_ram0": torch.full((n_envs, 128), 7.0, device="cuda"),
           "grad_cart_ram0": torch.full((n_envs, 128), 7.0, device="cuda"),
           "grad_u": torch.full((n_steps, n_envs, 5), 7.0, device="cuda"),
           "grad_rom_per_cart": torch.full((len(roms), 32768), 7.0, device="cuda")}
    if per_step:
        gr = torch.from_numpy(synth.normal_f32(92, (n_steps, n_envs, 128), 1)).cuda()
        gs = None
        if cfg.get("step_instructions", 0) == 0:
            gs = torch.from_numpy(synth.normal_f32(92, (n_steps, n_envs, 210, 160), 2)).cuda()
        tape.backward(grad_ram=gr, grad_screen=gs, **out)
    else:
        w = torch.zeros(128, device="cuda")
        w[torch.arange(0, 128, 9, device="cuda")] = 1.0
        tape.backward(w_ram=w, **out)
    b.sync()
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    tape.free()
    b.close()
    return res


CASES = {
    # name: (mappers, n_envs, n_steps, frame_skip, tau, per-step gradients, config)
    "segments_superchip_e0": ([synth.MAPPER_2K, synth.MAPPER_E0, synth.MAPPER_F8SC], 45, 5, 1, 0.3, True,
                              {"segment_frames": 2}),
    "whole_tia_graphics_bits": ([synth.MAPPER_4K, synth.MAPPER_F6SC], 37, 3, 2, 0.1, True,
                                {"segment_frames": 2, "full_tia": 1, "graphics_bits": 1}),
    "position_sampler": ([synth.MAPPER_4K], 33, 3, 1, 0.5, True, {"position_sampler": 1}),
    "instruction_steps": ([synth.MAPPER_4K, synth.MAPPER_F8], 70, 3, 1, 0.1, False,
                          {"step_instructions": 700, "segment_frames": 2}),
}


@pytest.mark.parametrize("case", list(CASES))
def test_lane_sweep_equals_warp_sweep(case):
    mappers, n_envs, n_steps, frame_skip, tau, per_step, cfg = CASES[case]
    roms = synth.config_carts(93, mappers, full_tia=bool(cfg.get("full_tia", 0)))
    env_cart = (np.arange(n_envs) % len(mappers)).astype(np.int32)
    warm = 94 if cfg.get("step_instructions", 0) == 0 else 0
    want = _run(roms, mappers, env_cart, 1, n_steps, frame_skip, tau, warm, per_step, cfg)
    got = _run(roms, mappers, env_cart, 2, n_steps, frame_skip, tau, warm, per_step, cfg)
    assert np.abs(want["grad_rom"][:, :4096]).max() > 0
    if warm:   # from power-on the reset code clears the RAM, so its start carries no gradient
        assert np.abs(want["grad_ram0"]).max() > 0
    for k in want:
        assert np.array_equal(got[k], want[k]), f"{case}: {k} differs between the two sweeps"


def test_automatic_sweep_choice_at_large_batches():
    """From 16,384 envs the default (sweep_mode 0) walks one env per lane; the
    gradients are the one-env-per-warp sweep's bits."""
    mappers = [synth.MAPPER_4K]
    roms = synth.config_carts(95, mappers)
    env_cart = np.zeros(16384, np.int32)
    cfg = {"step_instructions": 300}
    want = _run(roms, mappers, env_cart, 1, 2, 1, 0.1, 0, False, cfg)
    got = _run(roms, mappers, env_cart, 0, 2, 1, 0.1, 0, False, cfg)
    for k in want:
        assert np.array_equal(got[k], want[k]), f"{k} differs between the automatic and the warp sweep"
