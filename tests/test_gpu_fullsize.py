"""Parity at the workloads' full sizes, in the launch configuration the
benchmark uses, on sampled envs the oracle recomputes one by one:

* 4096 envs of one 4 KB cart, frame-skip 4 (the benchmark's workload);
* 65,536 envs over 16 carts (6 x 2K, 6 x 4K, 4 x F8) with geometric episode
  lengths (mean 2,000 frames) and auto-reset;
* 1024 envs of one 4 KB cart, 64-frame SOFT-STE rollouts at tau in
  {1, 0.1, 0.01}: forward equal to hard for every env, gradients (dense
  seeded gradients on RAM for every env and on every pixel for 16 sampled
  envs) against the FP64 oracle on those 16 envs;
* 4096 envs of 4 x 4K + 4 x F8 carts, a 128-frame SOFT-STE prefix of the
  long-horizon rollout (tau = 0.1, 64-frame checkpoint segments, broadcast
  loss weights on 8 RAM bytes and 256 pixels).
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2606_22447_b300 import synth
from tests.gpu_util import assert_env_equal, gpu_rollout, make_batch, oracle_rollout, torch_cuda
from tests.test_gpu_soft import assert_grad_close

pytestmark = pytest.mark.gpu


def test_bench_workload_4096_envs_sampled():
    rom = synth.generate_cart(2, 0, synth.MAPPER_4K)
    n = 4096
    b = make_batch([rom], [synth.MAPPER_4K], np.zeros(n, np.int32))
    acts = synth.actions(2, n, 6)
    ram, scr, st = gpu_rollout(b, acts, 4)
    for e in np.random.default_rng(0).choice(n, 12, replace=False):
        r2, s2, st2 = oracle_rollout(rom, synth.MAPPER_4K, acts[:, e], 4)
        assert_env_equal(e, ram[:, e], r2, "RAM")
        assert_env_equal(e, scr[:, e], s2, "screen")
        assert_env_equal(e, st[:, e], st2, "status")


def test_mixed_65536_envs_auto_reset_sampled():
    torch = torch_cuda()
    roms = synth.config_carts(3, synth.MIX16)
    n = 65536
    env_cart = synth.env_cart_round_robin(n, 16, sort=False)
    ep = synth.episode_lengths(3, n, 8)
    ep[:64] = np.array([1, 2, 3, 4, 5, 6, 7, 8], np.uint32)   # some envs reset inside the test window
    b = make_batch(roms, synth.MIX16, env_cart)
    b.set_episodes(ep)
    n_steps = 4
    acts = torch.from_numpy(synth.actions(3, n, n_steps)).cuda()
    ram = torch.empty((n_steps, n, 128), dtype=torch.uint8, device="cuda")
    st = torch.empty((n_steps, n), dtype=torch.uint8, device="cuda")
    scr = torch.empty((n, 210, 160), dtype=torch.uint8, device="cuda")
    for t in range(n_steps - 1):
        b.step(acts[t], 4, ram[t], None, st[t])
    b.step(acts[n_steps - 1], 4, ram[n_steps - 1], scr, st[n_steps - 1])
    b.sync()
    ram, st, scr = ram.cpu().numpy(), st.cpu().numpy(), scr.cpu().numpy()
    acts = acts.cpu().numpy()
    sample = list(range(0, 64, 7)) + list(np.random.default_rng(1).choice(n, 8, replace=False))
    for e in sample:
        c = int(env_cart[e])
        r2, s2, st2 = oracle_rollout(roms[c], synth.MIX16[c], acts[:, e], 4, ep_len=list(ep[e]))
        assert_env_equal(e, ram[:, e], r2, "RAM")
        assert_env_equal(e, st[:, e], st2, "status")
        assert_env_equal(e, scr[e], s2[-1], "screen")
    assert (st & 4).any()


def test_soft_1024_envs_64_frames():
    torch = torch_cuda()
    rom = synth.generate_cart(4, 0, synth.MAPPER_4K)
    n, n_steps = 1024, 64
    acts = synth.actions(4, n, n_steps)
    u = torch.from_numpy(synth.action_inputs(acts)).cuda()
    b_h = make_batch([rom], [synth.MAPPER_4K], np.zeros(n, np.int32))
    ram_h = torch.empty((n_steps, n, 128), dtype=torch.uint8, device="cuda")
    b_h.rollout(torch.from_numpy(acts).cuda(), 1, ram_h)
    b_h.sync()
    ram_h = ram_h.cpu().numpy().astype(np.float32)
    # 16 seeded envs (the first and last among them) get dense gradients on
    # RAM and on every pixel; the others dense RAM gradients only
    sample = sorted(set(np.random.default_rng(1024).choice(n, 14, replace=False).tolist()) | {0, n - 1})
    gr = synth.normal_f32(4, (n_steps, n, 128), 1)
    gs = torch.zeros((n_steps, n, 210, 160), device="cuda")
    gs_e = {e: synth.normal_f32(4, (n_steps, 210, 160), 100 + e) for e in sample}
    for e in sample:
        gs[:, e] = torch.from_numpy(gs_e[e]).cuda()
    for tau in (1.0, 0.1, 0.01):
        b = make_batch([rom], [synth.MAPPER_4K], np.zeros(n, np.int32))
        ram_s = torch.empty((n_steps, n, 128), device="cuda")
        tape = b.soft_rollout(tau, u, 1, ram_out=ram_s)
        g_rom = torch.empty((n, 8192), device="cuda")
        g_ram0 = torch.empty((n, 128), device="cuda")
        g_u = torch.empty((n_steps, n, 5), device="cuda")
        tape.backward(torch.from_numpy(gr).cuda(), gs, grad_rom=g_rom, grad_ram0=g_ram0, grad_u=g_u)
        b.sync()
        assert np.array_equal(ram_s.cpu().numpy(), ram_h)        # Theorem 1, every env
        g_rom, g_ram0, g_u = g_rom.cpu().numpy(), g_ram0.cpu().numpy(), g_u.cpu().numpy()

        def oracle_grads(e):
            o = oracle.Oracle(rom, synth.MAPPER_4K)
            g, _, _ = o.soft_rollout(synth.action_inputs(acts[:, e]).astype(np.float64), 1, tau, 6.0,
                                     gr[:, e].astype(np.float64), gs_e[e].astype(np.float64), outputs=False)
            return g.reverse()

        with ThreadPoolExecutor(4) as ex:
            wants = list(ex.map(oracle_grads, sample))
        for e, (o_rom, o_ram0, o_u) in zip(sample, wants):
            assert_grad_close(g_rom[e, :4096], o_rom, f"tau {tau} env {e} grad_rom")
            assert_grad_close(g_ram0[e], o_ram0, f"tau {tau} env {e} grad_ram0")
            assert_grad_close(g_u[:, e], o_u, f"tau {tau} env {e} grad_u")
        tape.free()


def test_long_horizon_prefix_4096_envs_loss_weights():
    torch = torch_cuda()
    mappers = synth.MIX8
    roms = synth.config_carts(5, mappers)
    n, n_steps = 4096, 128
    env_cart = synth.env_cart_round_robin(n, 8)
    b = make_batch(roms, mappers, env_cart, segment_frames=64)
    acts = synth.actions(5, n, n_steps)
    u = torch.from_numpy(synth.action_inputs(acts)).cuda()
    rng = np.random.default_rng(5)
    w_ram = np.zeros(128, np.float32)
    w_ram[rng.choice(128, 8, replace=False)] = rng.standard_normal(8)
    w_scr = np.zeros(210 * 160, np.float32)
    w_scr[rng.choice(210 * 160, 256, replace=False)] = rng.standard_normal(256)
    tape = b.soft_rollout(0.1, u, 1)
    g_pc = torch.empty((8, 8192), device="cuda")
    g_rom = torch.empty((n, 8192), device="cuda")
    g_u = torch.empty((n_steps, n, 5), device="cuda")
    tape.backward(w_ram=torch.from_numpy(w_ram).cuda(), w_screen=torch.from_numpy(w_scr).cuda(), grad_rom=g_rom,
                  grad_u=g_u, grad_rom_per_cart=g_pc)
    b.sync()
    g_rom, g_u, g_pc = g_rom.cpu().numpy(), g_u.cpu().numpy(), g_pc.cpu().numpy()
    for e in (0, 4095, 2222):
        c = int(env_cart[e])
        o = oracle.Oracle(roms[c], mappers[c])
        g, _, _ = o.soft_rollout(synth.action_inputs(acts[:, e]).astype(np.float64), 1, 0.1, 6.0,
                                 np.broadcast_to(w_ram, (n_steps, 128)).astype(np.float64),
                                 np.broadcast_to(w_scr.reshape(210, 160), (n_steps, 210, 160)).astype(np.float64),
                                 outputs=False)
        o_rom, _, o_u = g.reverse()
        assert_grad_close(g_rom[e, :len(roms[c])], o_rom, f"env {e} grad_rom")
        assert_grad_close(g_u[:, e], o_u, f"env {e} grad_u")
    for c in range(8):
        assert_grad_close(g_pc[c], g_rom[env_cart == c].sum(0), f"cart {c} per-cart sum")
