"""The whole TIA on the GPU (batches with full_tia = 1) against the oracle in
the same mode: player 1, the missiles and the ball with NUSIZ copies and
sizes, REFP, vertical delay, RESMP and HMOVE of every object, score mode and
the collision latches, bit for bit on RAM, screens and status (the carts
read the latches into RAM); the subset machine on the same carts; COLUP1 as
a differentiable colour (gradients against the FP64 oracle); and the fully
relaxed forward in the same mode."""
import numpy as np
import pytest

import oracle
from paper_2606_22447_b300 import synth
from tests.gpu_util import assert_env_equal, gpu_rollout, make_batch, oracle_rollout, torch_cuda
from tests.test_gpu_soft import assert_grad_close

pytestmark = pytest.mark.gpu

ALL10 = [synth.MAPPER_2K, synth.MAPPER_4K, synth.MAPPER_F8, synth.MAPPER_F6, synth.MAPPER_F4,
         synth.MAPPER_F8SC, synth.MAPPER_F6SC, synth.MAPPER_F4SC, synth.MAPPER_E0, synth.MAPPER_FE]


def _check(roms, mappers, env_cart, acts, frame_skip, full, **cfg):
    b = make_batch(roms, mappers, env_cart, full_tia=1 if full else 0, **cfg)
    ram, scr, st = gpu_rollout(b, acts, frame_skip)
    for e in range(len(env_cart)):
        c = int(env_cart[e])
        r2, s2, st2 = oracle_rollout(roms[c], mappers[c], acts[:, e], frame_skip, full_tia=full)
        assert_env_equal(e, ram[:, e], r2, "RAM")
        assert_env_equal(e, scr[:, e], s2, "screen")
        assert_env_equal(e, st[:, e], st2, "status")
    return b


@pytest.mark.parametrize("epb,tpe", [(16, 1), (32, 4), (64, 2)])
def test_full_tia_carts_match_oracle(epb, tpe):
    """Full-TIA carts of all ten formats, envs unsorted over several blocks
    and a ragged tail, in both machine modes."""
    roms = synth.config_carts(311, ALL10, full_tia=True)
    env_cart = np.random.default_rng(11).permutation(np.arange(45) % len(ALL10)).astype(np.int32)
    acts = synth.actions(311, 45, 6)
    _check(roms, ALL10, env_cart, acts, 2, True, envs_per_block=epb, threads_per_env=tpe)
    if tpe == 1:
        _check(roms, ALL10, env_cart, acts, 2, False, envs_per_block=epb)


def test_plain_carts_in_full_tia_mode():
    """The default synthetic carts (whose random stack writes and reads reach
    some of the other object and collision registers) with the whole TIA."""
    mappers = synth.MIX8
    roms = synth.config_carts(312, mappers)
    env_cart = (np.arange(24) % len(mappers)).astype(np.int32)
    _check(roms, mappers, env_cart, synth.actions(312, 24, 5), 4, True)


def test_tia_pin_programs_on_the_gpu():
    """The oracle's hand-derived TIA pins (copies, sizes, widths, priority,
    score mode, vertical delay, HMOVE of every object, RESMP, collisions)
    run on the GPU equal the oracle."""
    from tests.microrom import rom4k
    from tests import test_oracle_machine as m
    programs = []
    for writes in ([("COLUBK", 0x12), ("GRP1", 0xC1), ("NUSIZ1", 3), ("COLUP1", 0x44), ("REFP1", 8), ("RESP1", None)],
                   [("GRP0", 0xC1), ("NUSIZ0", 7), ("COLUP0", 0x44), ("RESP0", None)],
                   [("COLUBK", 0x12), ("COLUP0", 0x44), ("COLUP1", 0x66), ("COLUPF", 0x88), ("ENAM0", 2),
                    ("NUSIZ0", 0x20), ("ENAM1", 2), ("NUSIZ1", 0x12), ("ENABL", 2), ("CTRLPF", 0x30),
                    ("RESM0", None), ("RESM1", None), ("RESBL", None)],
                   [("COLUP0", 0x44), ("COLUP1", 0x66), ("PF1", 0xFF), ("CTRLPF", 2)],
                   [("COLUP0", 0x44), ("VDELP0", 1), ("GRP0", 0xFF), ("GRP1", 0), ("RESP0", None)],
                   [("COLUP1", 0x66), ("COLUPF", 0x88), ("GRP1", 0x80), ("ENAM0", 2), ("ENABL", 2), ("HMP1", 0xF0),
                    ("HMM0", 0x10), ("HMBL", 0x20), ("RESP1", None), ("RESM0", None), ("RESBL", None),
                    ("HMOVE", None), ("HMCLR", None), ("HMOVE", None), ("RESMP0", 2), ("RESMP0", 0)]):
        def build(a, writes=writes):
            a.op("LDA", "imm", 0)
            a.op("STA", "zp", m.VBLANK)
            a.label("FRAME")
            a.op("LDA", "imm", 2)
            a.op("STA", "zp", m.WSYNC)
            a.op("STA", "zp", m.VSYNC)
            a.op("LDA", "imm", 0)
            a.op("STA", "zp", m.VSYNC)
            for reg in (0x02, 0x07, 0x00, 0x03, 0x06):      # collision latches into RAM, then CXCLR
                a.op("LDA", "zp", reg)
                a.op("STA", "zp", 0x80 + reg)
            a.op("STA", "zp", m.T["CXCLR"])
            m._frame_setup(a, writes)
            a.op("LDX", "imm", 200)
            a.label("LINE")
            a.op("STA", "zp", m.WSYNC)
            a.op("DEX")
            a.op("BNE", "rel", "LINE")
            a.op("JMP", "abs", "FRAME")
        programs.append(rom4k(build))
    mappers = [synth.MAPPER_4K] * len(programs)
    _check(programs, mappers, np.arange(len(programs), dtype=np.int32), synth.actions(313, len(programs), 4), 1, True)


@pytest.mark.parametrize("tpe,seg,sampler", [(1, 64, 0), (4, 2, 0), (2, 2, 1)])
def test_full_tia_gradients_match_fp64_oracle(tpe, seg, sampler):
    """Soft mode with the whole TIA: pixels owned by COLUP1 (player 1,
    missile 1, the right half of a score-mode playfield) and the general
    drawing path's per-owner sums, with and without the position sampler
    (whose colour difference then comes from the priority logic over every
    object); ROM, initial RAM and input gradients within 1e-5 of the FP64
    oracle over one and several segments, on plain, Superchip and E0 carts.
    The tolerance of every gradient test (normwise 1e-5, elementwise 1e-5
    for entries within 20x of the largest)."""
    torch = torch_cuda()
    mappers = [synth.MAPPER_4K, synth.MAPPER_F8, synth.MAPPER_2K, synth.MAPPER_E0, synth.MAPPER_F6SC]
    n_envs, n_steps, tau = 10, 3, 0.1
    roms = synth.config_carts(314, mappers, full_tia=True)
    env_cart = (np.arange(n_envs) % len(mappers)).astype(np.int32)
    b = make_batch(roms, mappers, env_cart, full_tia=1, envs_per_block=8, threads_per_env=tpe, segment_frames=seg,
                   position_sampler=sampler)
    wa = synth.actions(315, n_envs, 2)
    gpu_rollout(b, wa, 1, screens=False)
    acts = synth.actions(314, n_envs, n_steps)
    u = synth.action_inputs(acts)
    gr = synth.normal_f32(314, (n_steps, n_envs, 128), 1)
    gs = synth.normal_f32(314, (n_steps, n_envs, 210, 160), 2)
    ram_s = torch.empty((n_steps, n_envs, 128), device="cuda")
    scr_s = torch.empty((n_steps, n_envs, 210, 160), device="cuda")
    tape = b.soft_rollout(tau, torch.from_numpy(u).cuda(), 1, ram_out=ram_s, screen_out=scr_s)
    g_rom = torch.empty((n_envs, b.rom_stride), device="cuda")
    g_ram0 = torch.empty((n_envs, 128), device="cuda")
    g_u = torch.empty((n_steps, n_envs, 5), device="cuda")
    tape.backward(torch.from_numpy(gr).cuda(), torch.from_numpy(gs).cuda(), grad_rom=g_rom, grad_ram0=g_ram0,
                  grad_u=g_u)
    b.sync()
    g_rom, g_ram0, g_u = g_rom.cpu().numpy(), g_ram0.cpu().numpy(), g_u.cpu().numpy()
    scr_s = scr_s.cpu().numpy()
    for e in range(n_envs):
        c = env_cart[e]
        o = oracle.Oracle(roms[c], mappers[c], full_tia=True)
        o.rollout(wa[:, e], 1, screens=False)
        o.set_sampler(bool(sampler))
        g, _, scr_o = o.soft_rollout(u[:, e].astype(np.float64), 1, tau, 6.0, gr[:, e].astype(np.float64),
                                     gs[:, e].astype(np.float64))
        assert np.array_equal(scr_s[:, e], scr_o), f"env {e}: soft screens"
        o_rom, o_ram0, o_u = g.reverse()
        assert_grad_close(g_rom[e, :len(roms[c])], o_rom, f"grad_rom env {e}")
        assert_grad_close(g_ram0[e], o_ram0, f"grad_ram0 env {e}")
        assert_grad_close(g_u[:, e], o_u, f"grad_u env {e}")


def test_full_tia_first_divergence():
    """The fully relaxed forward study in full-TIA mode equals the oracle's
    (collision latches and the cold registers are part of the compared
    state)."""
    torch = torch_cuda()
    from tests.test_gpu_full import _oracle_study  # noqa: F401  (the same study, full TIA below)
    mappers = [synth.MAPPER_4K, synth.MAPPER_F8, synth.MAPPER_2K]
    roms = synth.config_carts(316, mappers, full_tia=True)
    ec = (np.arange(6) % 3).astype(np.int32)
    b = make_batch(roms, mappers, ec, full_tia=1, envs_per_block=8)
    acts = synth.actions(317, 6, 1)[0]
    T, alpha, n = 0.15, 6.0, 2000
    n_div, _, ram = b.full_divergence(T, alpha, n, actions=torch.from_numpy(acts).cuda())
    b.sync()
    n_div, ram = n_div.cpu().numpy(), ram.cpu().numpy()
    for e in range(6):
        c = ec[e]
        def start(mode):
            o = oracle.Oracle(roms[c], mappers[c], full_tia=True)
            o.set_full(mode, T, alpha)
            return o
        h, f = start(0), start(2)
        want = 0
        for k in range(1, n + 1):
            h.trace(int(acts[e]), 1)
            f.trace(int(acts[e]), 1)
            if not want and not (np.array_equal(h.state(), f.state()) and np.array_equal(h.ram(), f.ram())):
                want = k
        assert n_div[e] == want, (e, n_div[e], want)
        assert np.array_equal(ram[e], f.ram())
