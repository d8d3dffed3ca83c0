"""Parity over the workloads' full lengths, against the oracle on sampled
envs (digests of RAM and screen per env-step where the outputs are too
large to keep), and the ALU exhaustively on the GPU:

* 4096 envs of one 4 KB cart, frame-skip 4, 10,000 steps (the bench
  workload's full length): every env's digests for the first 16 steps and a
  seeded 32-env sample for all 10,000;
* 65,536 envs over 16 carts (6 x 2K, 6 x 4K, 4 x F8) with the seeded
  geometric episode table (mean 2,000 frames, no lengths forced short),
  5,000 steps of frame-skip 4 (20,000 frames): a 32-env sample whose envs
  pass through natural auto-resets (timer renormalisation and long drift
  included);
* the long-horizon soft rollout (4096 envs of 4 x 4K + 4 x F8 carts, 2,048
  frames at tau = 0.1, 64-frame checkpoint segments, broadcast loss weights
  on 8 RAM bytes and 256 pixels): gradients of an env of every cart and of
  the first, middle and last env against the FP64 oracle over the whole
  horizon;
* ADC and SBC over every A x operand x carry x decimal-flag combination
  (262,144 envs, one combination each, set through the soft rollout's
  initial RAM), bit-exact against the oracle's interpreter.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2606_22447_b300 import synth
from tests.gpu_util import make_batch, oracle_rollout, torch_cuda
from tests.microrom import rom4k
from tests.test_gpu_soft import assert_grad_close

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 8


def _oracle_digests(rom, mapper, acts, frame_skip, ep_len=None):
    r, s, st = oracle_rollout(rom, mapper, acts, frame_skip, ep_len=ep_len)
    return np.array([oracle.digest(r[t], s[t]) for t in range(len(acts))], dtype=np.uint64), st


def _gpu_digests(b, acts, frame_skip, chunk, keep=None):
    """Per-step digests [n_steps][len(keep)] (RAM and screen) and status of
    a rollout of acts [n_steps][n_envs], run `chunk` steps per call."""
    torch = torch_cuda()
    n_steps, n = acts.shape
    ram = torch.empty((chunk, n, 128), dtype=torch.uint8, device="cuda")
    scr = torch.empty((chunk, n, 210, 160), dtype=torch.uint8, device="cuda")
    st = torch.empty((chunk, n), dtype=torch.uint8, device="cuda")
    keep_t = None if keep is None else torch.from_numpy(np.asarray(keep, np.int64)).cuda()
    digs, stats = [], []
    for t0 in range(0, n_steps, chunk):
        k = min(chunk, n_steps - t0)
        b.rollout(torch.from_numpy(np.ascontiguousarray(acts[t0:t0 + k])).cuda(), frame_skip, ram[:k], scr[:k],
                  st[:k])
        d = b.digest(ram[:k], scr[:k])
        s = st[:k]
        if keep_t is not None:
            d, s = d[:, keep_t], s[:, keep_t]
        digs.append(d.cpu().numpy().view(np.uint64).copy())
        stats.append(s.cpu().numpy().copy())
    b.sync()
    return np.concatenate(digs), np.concatenate(stats)


def test_bench_workload_10000_steps():
    n, steps, first = 4096, 10000, 16
    rom = synth.generate_cart(2, 0, synth.MAPPER_4K)
    acts = synth.actions(2, n, steps)
    b = make_batch([rom], [synth.MAPPER_4K], np.zeros(n, np.int32))
    dig, _ = _gpu_digests(b, acts, 4, 50)
    sample = np.random.default_rng(10000).choice(n, 32, replace=False)
    with ThreadPoolExecutor(THREADS) as ex:
        long = list(ex.map(lambda e: _oracle_digests(rom, synth.MAPPER_4K, acts[:, e], 4)[0], sample))
        short = list(ex.map(lambda e: _oracle_digests(rom, synth.MAPPER_4K, acts[:first, e], 4)[0], range(n)))
    for e, want in zip(sample, long):
        bad = np.flatnonzero(dig[:, e] != want)
        assert bad.size == 0, f"env {e}: {bad.size} of {steps} steps differ, first at step {bad[0]}"
    for e, want in enumerate(short):
        bad = np.flatnonzero(dig[:first, e] != want)
        assert bad.size == 0, f"env {e}: step {bad[0]} differs"


def test_mixed_65536_envs_natural_episodes_20000_frames():
    n, steps = 65536, 5000
    roms = synth.config_carts(3, synth.MIX16)
    env_cart = synth.env_cart_round_robin(n, 16, sort=False)
    ep = synth.episode_lengths(3, n, 8)   # geometric, mean 2,000 frames, as drawn
    b = make_batch(roms, synth.MIX16, env_cart)
    b.set_episodes(ep)
    acts = synth.actions(3, n, steps)
    sample = np.random.default_rng(65536).choice(n, 32, replace=False)
    dig, st = _gpu_digests(b, acts, 4, 8, keep=sample)
    with ThreadPoolExecutor(THREADS) as ex:
        wants = list(ex.map(lambda e: _oracle_digests(roms[env_cart[e]], synth.MIX16[env_cart[e]], acts[:, e], 4,
                                                      ep_len=list(ep[e])), sample))
    resets = 0
    for j, (e, (want, want_st)) in enumerate(zip(sample, wants)):
        bad = np.flatnonzero(dig[:, j] != want)
        assert bad.size == 0, f"env {e}: {bad.size} of {steps} steps differ, first at step {bad[0]}"
        assert np.array_equal(st[:, j], want_st), f"env {e}: status differs"
        resets += int((want_st & 4).astype(bool).sum())
    assert resets >= 160, f"only {resets} natural auto-resets in the sample"


def test_long_horizon_2048_frames_gradients():
    torch = torch_cuda()
    mappers = synth.MIX8
    roms = synth.config_carts(5, mappers)
    n, n_steps = 4096, 2048
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
    g_rom = torch.empty((n, 8192), device="cuda")
    g_u = torch.empty((n_steps, n, 5), device="cuda")
    g_ram0 = torch.empty((n, 128), device="cuda")
    tape.backward(w_ram=torch.from_numpy(w_ram).cuda(), w_screen=torch.from_numpy(w_scr).cuda(), grad_rom=g_rom,
                  grad_u=g_u, grad_ram0=g_ram0)
    b.sync()
    tape.free()
    g_rom, g_u, g_ram0 = g_rom.cpu().numpy(), g_u.cpu().numpy(), g_ram0.cpu().numpy()
    # one env of every cart (the first, a middle and the last env among them)
    envs = [int(np.flatnonzero(env_cart == c)[(c * 229) % int((env_cart == c).sum())]) for c in range(len(mappers))]
    envs = sorted(set(envs) | {0, 2047, 4095})

    def oracle_grads(e):
        c = int(env_cart[e])
        o = oracle.Oracle(roms[c], mappers[c])
        g, _, _ = o.soft_rollout(synth.action_inputs(acts[:, e]).astype(np.float64), 1, 0.1, 6.0,
                                 np.broadcast_to(w_ram, (n_steps, 128)).astype(np.float64),
                                 np.broadcast_to(w_scr.reshape(210, 160), (n_steps, 210, 160)).astype(np.float64),
                                 outputs=False)
        return g.reverse()

    with ThreadPoolExecutor(4) as ex:   # about 1.1 GB of host memory per oracle rollout
        wants = list(ex.map(oracle_grads, envs))
    for e, (o_rom, o_ram0, o_u) in zip(envs, wants):
        c = int(env_cart[e])
        assert np.abs(o_rom).max() < 1e30, "overflow-class gradient"
        assert_grad_close(g_rom[e, :len(roms[c])], o_rom, f"env {e} grad_rom")
        assert_grad_close(g_ram0[e], o_ram0, f"env {e} grad_ram0")
        assert_grad_close(g_u[:, e], o_u, f"env {e} grad_u")


def _alu_sweep_rom():
    """A = $80, operand = $81, carry = bit 0 of $82, decimal flag = $83 != 0:
    ADC $81 into $84 with the flags (PHP) in $85, then SBC $81 into $86 with
    the flags in $87, then CLD and a loop on itself."""
    def build(a):
        a.op("LDA", "zp", 0x83)
        a.op("BEQ", "rel", "BIN")
        a.op("SED")
        a.label("BIN")
        for op, res, flags in (("ADC", 0x84, 0x85), ("SBC", 0x86, 0x87)):
            a.op("LDA", "zp", 0x82)
            a.op("LSR", "acc")
            a.op("LDA", "zp", 0x80)
            a.op(op, "zp", 0x81)
            a.op("STA", "zp", res)
            a.op("PHP")
            a.op("PLA")
            a.op("STA", "zp", flags)
        a.op("CLD")
        a.label("HALT")
        a.op("JMP", "abs", "HALT")
    return rom4k(build)


def test_adc_sbc_exhaustive_on_the_gpu():
    """Every (A, M, C, D): result and N V Z C flags of ADC and SBC, bit-exact
    against the oracle's interpreter (itself pinned exhaustively against
    integer and decimal arithmetic and the NMOS decimal-mode note)."""
    torch = torch_cuda()
    rom = _alu_sweep_rom()
    n = 2 * 2 * 256 * 256
    d, c, a, m = np.meshgrid(np.arange(2), np.arange(2), np.arange(256), np.arange(256), indexing="ij")
    ram0 = np.zeros((n, 128), np.float32)
    ram0[:, 0], ram0[:, 1], ram0[:, 2], ram0[:, 3] = a.ravel(), m.ravel(), c.ravel(), d.ravel()
    b = make_batch([rom], [synth.MAPPER_4K], np.zeros(n, np.int32), step_instructions=24)
    u = torch.zeros((1, n, 5), device="cuda")
    ram = torch.empty((1, n, 128), device="cuda")
    tape = b.soft_rollout(0.1, u, 1, ram0=torch.from_numpy(ram0).cuda(), ram_out=ram)
    b.sync()
    tape.free()
    got = ram.cpu().numpy()[0, :, 4:8].astype(np.int64)
    # the oracle's interpreter, one instruction at a time from set registers
    o = oracle.Oracle(rom4k(lambda asm: (asm.op("ADC", "absy", 0xFE00), asm.at(0x10),
                                         asm.op("SBC", "absy", 0xFE00))), synth.MAPPER_4K)
    want = np.zeros((n, 4), np.int64)
    for i, (dd, cc, aa, mm) in enumerate(zip(d.ravel(), c.ravel(), a.ravel(), m.ravel())):
        for k, pc in enumerate((0xF000, 0xF010)):
            o.set_regs(A=int(aa), Y=int(mm), P=(0x08 if dd else 0) | (0x01 if cc else 0), PC=pc)
            o.exec_one()
            s = o.state()
            want[i, 2 * k], want[i, 2 * k + 1] = s[0], s[4]
    nvzc = 0xC3
    for col, what in ((0, "ADC result"), (2, "SBC result")):
        bad = np.flatnonzero(got[:, col] != want[:, col])
        assert bad.size == 0, f"{what}: {bad.size} combinations differ, first (D, C, A, M) index {bad[0]}"
    for col, what in ((1, "ADC flags"), (3, "SBC flags")):
        bad = np.flatnonzero((got[:, col] & nvzc) != (want[:, col] & nvzc))
        assert bad.size == 0, f"{what}: {bad.size} combinations differ, first (D, C, A, M) index {bad[0]}"
