"""Shared helpers for the GPU parity tests: run the same seeded inputs through
the CUDA path (through the C ABI) and through the oracle, env by env."""
import numpy as np

import oracle
from paper_2606_22447_b300 import synth


def torch_cuda():
    import torch
    return torch


def gpu_rollout(batch, actions, frame_skip, screens=True):
    """actions uint8 [n_steps][n_envs] -> (ram, screen, status) numpy arrays."""
    torch = torch_cuda()
    n_steps, n_envs = actions.shape
    a = torch.from_numpy(np.ascontiguousarray(actions)).cuda()
    ram = torch.empty((n_steps, n_envs, 128), dtype=torch.uint8, device="cuda")
    scr = torch.empty((n_steps, n_envs, 210, 160), dtype=torch.uint8, device="cuda") if screens else None
    st = torch.empty((n_steps, n_envs), dtype=torch.uint8, device="cuda")
    batch.rollout(a, frame_skip, ram, scr, st)
    batch.sync()
    return ram.cpu().numpy(), (scr.cpu().numpy() if screens else None), st.cpu().numpy()


def oracle_rollout(rom, mapper, actions, frame_skip, ystart=34, ep_len=None, screens=True, boot=None,
                   start=None, full_tia=False):
    """One env through the oracle; ep_len (frames per episode, cyclic)
    reproduces the library's auto-reset at step ends; boot = (noop frames,
    reset frames) and start (this env's start-NOOP counts, cyclic) reproduce
    the boot sequence after every power-on."""
    o = oracle.Oracle(rom, mapper, ystart, full_tia=full_tia)

    def do_boot(episode):
        if boot is not None or start is not None:
            nb, rb = boot if boot is not None else (0, 0)
            o.boot(nb, rb, 0 if start is None else int(start[episode % len(start)]))
    do_boot(0)
    n = len(actions)
    rams = np.zeros((n, 128), np.uint8)
    scrs = np.zeros((n, 210, 160), np.uint8) if screens else None
    status = np.zeros(n, np.uint8)
    epf, epi = 0, 0
    for t, a in enumerate(actions):
        r, s, st = o.step(int(a), frame_skip)
        rams[t] = r
        if screens:
            scrs[t] = s
        if ep_len is not None:
            epf += frame_skip
            if epf >= ep_len[epi % len(ep_len)]:
                st |= 4
                o.reset()
                epf, epi = 0, epi + 1
                do_boot(epi)
        status[t] = st
    return rams, scrs, status


def make_batch(roms, mappers, env_cart, **cfg):
    from paper_2606_22447_b300 import Batch, default_config
    return Batch(roms, mappers, env_cart, default_config(**cfg))


def assert_env_equal(env, got, want, what):
    if not np.array_equal(got, want):
        diff = np.argwhere(got != want)
        raise AssertionError(f"{what} mismatch for env {env}: {len(diff)} elements differ, first at {diff[0].tolist()}")
