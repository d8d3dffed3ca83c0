"""Instruction-granular steps (the paper's throughput unit, Section 6: one
step = one emulated instruction) on the GPU against the oracle: RAM and
status after every step of n instruction slots bit-exact (step ends inside
frames and inside timer poll loops, a jammed CPU's idle slots), soft forward
equal to hard, gradients within 1e-5 of the FP64 oracle across checkpoint
segments, and the refusals of frame-only features."""
import numpy as np
import pytest

import oracle
from paper_2606_22447_b300 import VcsError, synth
from paper_2606_22447_b300._lib import VCS_ERR_ARG
from tests.gpu_util import assert_env_equal, gpu_rollout, make_batch, torch_cuda
from tests.test_gpu_soft import assert_grad_close

pytestmark = pytest.mark.gpu

MAPPERS = [synth.MAPPER_2K, synth.MAPPER_4K, synth.MAPPER_F8]


def _oracle_steps(rom, mapper, actions, n_instr):
    o = oracle.Oracle(rom, mapper)
    o.set_step_instructions(n_instr)
    rams = np.zeros((len(actions), 128), np.uint8)
    status = np.zeros(len(actions), np.uint8)
    for t, a in enumerate(actions):
        r, _, st = o.step(int(a), 1)
        rams[t], status[t] = r, st
    return rams, status


@pytest.mark.parametrize("n_instr,spl,epb,banked", [(1000, 0, 0, False), (997, 2, 8, False), (3001, 0, 32, False),
                                                    (1, 0, 0, False), (1999, 0, 0, True), (1501, 0, 0, "ext"),
                                                    (777, 0, 0, "fe")])
def test_hard_instruction_steps_match_oracle(n_instr, spl, epb, banked):
    n_envs = 33
    steps = 6 if n_instr > 1 else 40
    mappers = ([synth.MAPPER_F8SC, synth.MAPPER_E0, synth.MAPPER_F4SC] if banked == "ext" else
               [synth.MAPPER_FE, synth.MAPPER_4K, synth.MAPPER_FE] if banked == "fe" else
               [synth.MAPPER_F6, synth.MAPPER_F4, synth.MAPPER_F8] if banked else MAPPERS)
    roms = synth.config_carts(81, mappers)
    ec = (np.arange(n_envs) % 3).astype(np.int32)
    b = make_batch(roms, mappers, ec, step_instructions=n_instr, steps_per_launch=spl, envs_per_block=epb)
    acts = synth.actions(82, n_envs, steps)
    ram, _, st = gpu_rollout(b, acts, 1, screens=False)
    for e in range(n_envs):
        r, s = _oracle_steps(roms[ec[e]], mappers[ec[e]], acts[:, e], n_instr)
        assert_env_equal(e, ram[:, e], r, "RAM")
        assert_env_equal(e, st[:, e], s, "status")


def test_instruction_steps_inside_poll_loops_and_jams():
    """Budgets that end inside timer poll loops (many step sizes over a cart
    whose frames wait on INTIM) and a jammed CPU's idle slots."""
    from tests.microrom import rom4k
    def jam(asm):
        asm.op("LDA", "imm", 1)
        asm.op("STA", "zp", 0x80)
        asm.byte(0x02)
    roms = [synth.config_carts(83, [synth.MAPPER_4K])[0], rom4k(jam)]
    mappers = [synth.MAPPER_4K, synth.MAPPER_4K]
    for n_instr in (5, 7, 13, 101):
        ec = np.array([0] * 8 + [1] * 2, np.int32)
        b = make_batch(roms, mappers, ec, step_instructions=n_instr)
        acts = synth.actions(84 + n_instr, len(ec), 300)
        ram, _, st = gpu_rollout(b, acts, 1, screens=False)
        for e in range(len(ec)):
            r, s = _oracle_steps(roms[ec[e]], mappers[ec[e]], acts[:, e], n_instr)
            assert_env_equal(e, ram[:, e], r, f"RAM (n = {n_instr})")
            assert_env_equal(e, st[:, e], s, f"status (n = {n_instr})")
        assert np.all(st[-1, 8:] & 2), "the jam cart must end jammed"


def test_instruction_steps_refuse_frame_only_features():
    torch = torch_cuda()
    roms = synth.config_carts(85, [synth.MAPPER_4K])
    b = make_batch(roms, [synth.MAPPER_4K], [0] * 4, step_instructions=100)
    acts = torch.zeros((1, 4), dtype=torch.uint8, device="cuda")
    scr = torch.empty((1, 4, 210, 160), dtype=torch.uint8, device="cuda")
    with pytest.raises(VcsError) as ei:
        b.rollout(acts, 1, None, scr)
    assert ei.value.status == VCS_ERR_ARG
    with pytest.raises(VcsError):
        b.set_episodes(np.full((4, 2), 100, np.uint32))
    with pytest.raises(VcsError):
        make_batch(roms, [synth.MAPPER_4K], [0] * 4, step_instructions=100, boot_noop_frames=2)
    u = torch.zeros((1, 4, 5), device="cuda")
    with pytest.raises(VcsError):
        b.soft_rollout(0.1, u, 1, screen_out=torch.empty((1, 4, 210, 160), device="cuda"))
    tape = b.soft_rollout(0.1, u, 1)
    with pytest.raises(VcsError):
        tape.backward(w_screen=torch.ones(210 * 160, device="cuda"))
    tape.free()


@pytest.mark.parametrize("tau,seg", [(0.1, 64), (1.0, 2), (0.01, 1)])
def test_soft_instruction_steps_gradients_match_fp64_oracle(tau, seg):
    torch = torch_cuda()
    n_envs, n_steps, n_instr = 6, 4, 1500
    roms = synth.config_carts(86, MAPPERS)
    ec = (np.arange(n_envs) % 3).astype(np.int32)
    b = make_batch(roms, MAPPERS, ec, step_instructions=n_instr, segment_frames=seg, envs_per_block=8,
                   threads_per_env=4)
    wa = synth.actions(87, n_envs, 2)
    gpu_rollout(b, wa, 1, screens=False)
    acts = synth.actions(88, n_envs, n_steps)
    u = synth.action_inputs(acts)
    gr = synth.normal_f32(88, (n_steps, n_envs, 128), 1)
    blob = b.save_state()
    ram_h, _, _ = gpu_rollout(b, acts, 1, screens=False)
    b.load_state(blob)
    ram_s = torch.empty((n_steps, n_envs, 128), device="cuda")
    tape = b.soft_rollout(tau, torch.from_numpy(u).cuda(), 1, ram_out=ram_s)
    g_rom = torch.empty((n_envs, 8192), device="cuda")
    g_ram0 = torch.empty((n_envs, 128), device="cuda")
    g_u = torch.empty((n_steps, n_envs, 5), device="cuda")
    tape.backward(torch.from_numpy(gr).cuda(), None, grad_rom=g_rom, grad_ram0=g_ram0, grad_u=g_u)
    b.sync()
    assert np.array_equal(ram_s.cpu().numpy(), ram_h.astype(np.float32)), "soft forward == hard"
    g_rom, g_ram0, g_u = g_rom.cpu().numpy(), g_ram0.cpu().numpy(), g_u.cpu().numpy()
    for e in range(n_envs):
        c = ec[e]
        o = oracle.Oracle(roms[c], MAPPERS[c])
        o.set_step_instructions(n_instr)
        o.rollout(wa[:, e], 1, screens=False)
        g, _, _ = o.soft_rollout(u[:, e].astype(np.float64), 1, tau, 6.0, gr[:, e].astype(np.float64), None)
        o_rom, o_ram0, o_u = g.reverse()
        assert_grad_close(g_rom[e, :len(roms[c])], o_rom, f"grad_rom env {e}")
        assert_grad_close(g_ram0[e], o_ram0, f"grad_ram0 env {e}")
        assert_grad_close(g_u[:, e], o_u, f"grad_u env {e}")
        assert np.abs(o_rom).max() > 0
