"""SOFT-STE on the GPU against the oracle (FP64).

* Theorem 1: the soft forward's RAM and screens equal the hard path's bit
  for bit at tau in {1, 0.1, 0.01};
* Corollary 1 / the surrogate rulebook: the CUDA backward (FP32) equals the
  oracle's FP64 reverse sweep to 1e-5 relative, per output tensor and env:
  max |g - g64| <= 1e-5 max(|g64|_inf, 1e-30) (normwise), and
  |g - g64| <= 1e-5 |g64| wherever |g64| >= 5e-2 |g64|_inf (elementwise,
  for entries within 20x of the largest).  The floor is one number for
  every gradient test, set from a measurement over all of them (645
  comparisons): the largest floor any comparison needed was 3.0e-2 and the
  largest normwise error 6.0e-6; an entry that is the difference of large
  contributions of both signs (pixel sums of random upstream gradients,
  ADC's (1, 1) against SBC's (1, -1)) keeps a float32 error of a few units
  in the last place of those contributions, so its relative error grows as
  it goes to zero (ROM bytes per env, initial RAM, joystick inputs);
* checkpoint/recompute over several segments gives the same gradient as one
  segment; broadcast loss weights equal the dense gradients they expand to;
  the autograd Function returns the C ABI's gradients.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2606_22447_b300 import synth
from tests.gpu_util import gpu_rollout, make_batch, torch_cuda

pytestmark = pytest.mark.gpu
REL = 1e-5


def _report(what, got, want, err, scale):
    """With VCS_GRAD_REPORT set to a file path, append one JSON line per
    comparison: the normwise error and the smallest elementwise floor that
    this comparison would pass (a measurement aid; no effect on the test)."""
    path = os.environ.get("VCS_GRAD_REPORT")
    if not path:
        return
    rel = err / np.maximum(np.abs(want), 1e-300)
    bad = rel > REL
    need = float((np.abs(want[bad]) / scale).max()) if bad.any() else 0.0
    test = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]
    with open(path, "a") as f:
        f.write(json.dumps({"test": test, "what": what, "normwise": float(err.max() / scale), "floor_needed": need,
                            "n": int(want.size)}) + "\n")
    if need > 1e-2:   # keep the arrays of the worst comparisons for a closer look
        np.savez(f"{path}.{abs(hash((test, what))) % 10**8}.npz", got=got, want=want)


# the elementwise floor of every gradient comparison (see the module docstring)
FLOOR = 5e-2


def assert_grad_close(got, want, what, floor=FLOOR):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    scale = max(np.abs(want).max(), 1e-30)
    err = np.abs(got - want)
    _report(what, got, want, err, scale)
    assert err.max() <= REL * scale, f"{what}: max abs err {err.max():.3e} vs scale {scale:.3e}"
    big = np.abs(want) >= floor * scale
    if big.any():
        r = np.where(big, err / np.where(big, np.abs(want), 1.0), 0.0)
        k = np.unravel_index(np.argmax(r), r.shape)
        assert r[k] <= REL, (f"{what}: elementwise rel err {r[k]:.3e} at {k}: got {got[k]:.9e} "
                             f"want {want[k]:.9e} (scale {scale:.3e})")


def _setup(mappers, n_envs, n_steps, seed, warm=2, frame_skip=1, **cfg):
    torch = torch_cuda()
    roms = synth.config_carts(seed, mappers)
    env_cart = (np.arange(n_envs) % len(mappers)).astype(np.int32)
    b = make_batch(roms, mappers, env_cart, **cfg)
    wa = synth.actions(seed + 1, n_envs, warm)
    gpu_rollout(b, wa, 1, screens=False)          # start from a state a few frames in
    acts = synth.actions(seed, n_envs, n_steps)
    u = synth.action_inputs(acts)                  # [n_steps][n_envs][5]
    return torch, roms, env_cart, b, wa, acts, u


def _oracle_grads(rom, mapper, warm_acts, u, frame_skip, tau, gr, gs, sampler=False):
    o = oracle.Oracle(rom, mapper)
    o.rollout(warm_acts, 1, screens=False)
    o.set_sampler(sampler)
    g, ram_out, scr_out = o.soft_rollout(u.astype(np.float64), frame_skip, tau, 6.0,
                                         None if gr is None else gr.astype(np.float64),
                                         None if gs is None else gs.astype(np.float64))
    return g.reverse(), ram_out, scr_out


@pytest.mark.parametrize("tau", [1.0, 0.1, 0.01])
def test_theorem1_soft_forward_equals_hard(tau):
    torch, roms, env_cart, b, wa, acts, u = _setup(synth.MIX16[::3], 24, 6, 31)
    blob = b.save_state()
    ram_h, scr_h, _ = gpu_rollout(b, acts, 2)
    b.load_state(blob)
    ram_s = torch.empty((6, 24, 128), device="cuda")
    scr_s = torch.empty((6, 24, 210, 160), device="cuda")
    tape = b.soft_rollout(tau, torch.from_numpy(u).cuda(), 2, ram_out=ram_s, screen_out=scr_s)
    b.sync()
    assert np.array_equal(ram_s.cpu().numpy(), ram_h.astype(np.float32))
    assert np.array_equal(scr_s.cpu().numpy(), scr_h.astype(np.float32))
    # and the batch state advanced exactly as the hard path's
    blob_soft = b.save_state()
    b.load_state(blob)
    gpu_rollout(b, acts, 2, screens=False)
    assert np.array_equal(b.save_state(), blob_soft)
    tape.free()


@pytest.mark.parametrize("tau,frame_skip,tpe", [(1.0, 1, 4), (0.1, 1, 4), (0.01, 1, 4), (0.1, 2, 4), (0.1, 1, 1),
                                                 (1.0, 1, 2)])
def test_gradients_match_fp64_oracle(tau, frame_skip, tpe):
    mappers = [synth.MAPPER_2K, synth.MAPPER_4K, synth.MAPPER_F8]
    n_envs, n_steps = 6, 4
    torch, roms, env_cart, b, wa, acts, u = _setup(mappers, n_envs, n_steps, 41, frame_skip=frame_skip,
                                                   envs_per_block=8, threads_per_env=tpe)
    gr = synth.normal_f32(41, (n_steps, n_envs, 128), 1)
    gs = synth.normal_f32(41, (n_steps, n_envs, 210, 160), 2)
    tape = b.soft_rollout(tau, torch.from_numpy(u).cuda(), frame_skip)
    g_rom = torch.empty((n_envs, 8192), device="cuda")
    g_ram0 = torch.empty((n_envs, 128), device="cuda")
    g_u = torch.empty((n_steps, n_envs, 5), device="cuda")
    tape.backward(torch.from_numpy(gr).cuda(), torch.from_numpy(gs).cuda(), grad_rom=g_rom, grad_ram0=g_ram0,
                  grad_u=g_u)
    b.sync()
    g_rom, g_ram0, g_u = g_rom.cpu().numpy(), g_ram0.cpu().numpy(), g_u.cpu().numpy()
    for e in range(n_envs):
        c = env_cart[e]
        (o_rom, o_ram0, o_u), _, _ = _oracle_grads(roms[c], mappers[c], wa[:, e], u[:, e], frame_skip, tau,
                                                   gr[:, e], gs[:, e])
        size = len(roms[c])
        assert_grad_close(g_rom[e, :size], o_rom, f"grad_rom env {e}")
        assert np.all(g_rom[e, size:] == 0)
        assert_grad_close(g_ram0[e], o_ram0, f"grad_ram0 env {e}")
        assert_grad_close(g_u[:, e], o_u, f"grad_u env {e}")
        assert np.abs(o_rom).max() > 0


def test_segments_and_loss_weights_and_per_cart_sum():
    torch = torch_cuda()
    mappers = [synth.MAPPER_4K, synth.MAPPER_F8]
    n_envs, n_steps = 8, 9
    seed = 51
    res = {}
    for seg in (64, 3):
        _, roms, env_cart, b, wa, acts, u = _setup(mappers, n_envs, n_steps, seed, segment_frames=seg)
        wr = synth.normal_f32(seed, (128,), 3)
        ws = synth.normal_f32(seed, (210, 160), 4)
        tape = b.soft_rollout(0.1, torch.from_numpy(u).cuda(), 1)
        out = {}
        for mode in ("weights", "dense"):
            g_rom = torch.empty((n_envs, 8192), device="cuda")
            g_pc = torch.empty((2, 8192), device="cuda")
            g_ram0 = torch.empty((n_envs, 128), device="cuda")
            g_u = torch.empty((n_steps, n_envs, 5), device="cuda")
            if mode == "weights":
                tape.backward(w_ram=torch.from_numpy(wr).cuda(), w_screen=torch.from_numpy(ws).cuda(),
                              grad_rom=g_rom, grad_ram0=g_ram0, grad_u=g_u, grad_rom_per_cart=g_pc)
            else:
                gr = np.broadcast_to(wr, (n_steps, n_envs, 128)).copy()
                gs = np.broadcast_to(ws, (n_steps, n_envs, 210, 160)).copy()
                tape.backward(torch.from_numpy(gr).cuda(), torch.from_numpy(gs).cuda(), grad_rom=g_rom,
                              grad_ram0=g_ram0, grad_u=g_u, grad_rom_per_cart=g_pc)
            b.sync()
            out[mode] = [x.cpu().numpy() for x in (g_rom, g_ram0, g_u, g_pc)]
        for x, y in zip(out["weights"], out["dense"]):
            assert_grad_close(x, y, "weights vs dense")
        # per-cart sum = sum of the per-env rows of that cart
        g_rom, _, _, g_pc = out["dense"]
        for c in range(2):
            assert_grad_close(g_pc[c], g_rom[env_cart == c].sum(0), "per-cart sum")
        res[seg] = out["dense"]
        # oracle on two envs
        for e in (0, 5):
            c = env_cart[e]
            (o_rom, o_ram0, o_u), _, _ = _oracle_grads(roms[c], mappers[c], wa[:, e], u[:, e], 1, 0.1,
                                                       np.broadcast_to(wr, (n_steps, 128)),
                                                       np.broadcast_to(ws, (n_steps, 210, 160)))
            assert_grad_close(g_rom[e, :len(roms[c])], o_rom, "grad_rom")
            assert_grad_close(res[seg][1][e], o_ram0, "grad_ram0")
            assert_grad_close(res[seg][2][:, e], o_u, "grad_u")
    for x, y in zip(res[64], res[3]):
        assert_grad_close(x, y, "3-frame segments vs one segment")


def test_autograd_function_and_float_inputs():
    torch = torch_cuda()
    from paper_2606_22447_b300.autograd import soft_rollout
    mappers = [synth.MAPPER_2K, synth.MAPPER_4K]
    n_envs, n_steps = 4, 3
    _, roms, env_cart, b, wa, acts, u = _setup(mappers, n_envs, n_steps, 61)
    rom_f = np.zeros((2, 8192), np.float32)
    for c, r in enumerate(roms):
        rom_f[c, :len(r)] = np.frombuffer(r, np.uint8)
    ram0 = synth.normal_f32(61, (n_envs, 128), 5) * 0 + np.arange(128, dtype=np.float32)[None] % 256
    rom_t = torch.from_numpy(rom_f).cuda().requires_grad_()
    ram0_t = torch.from_numpy(ram0.astype(np.float32)).cuda().requires_grad_()
    u_t = torch.from_numpy(u).cuda().requires_grad_()
    ram, scr = soft_rollout(b, rom_t, ram0_t, u_t, tau=0.1, frame_skip=1)
    gr = synth.normal_f32(61, (n_steps, n_envs, 128), 1)
    gs = synth.normal_f32(61, (n_steps, n_envs, 210, 160), 2)
    loss = (ram * torch.from_numpy(gr).cuda()).sum() + (scr * torch.from_numpy(gs).cuda()).sum()
    g_rom, g_ram0, g_u = torch.autograd.grad(loss, [rom_t, ram0_t, u_t])
    g_rom, g_ram0, g_u = g_rom.cpu().numpy(), g_ram0.cpu().numpy(), g_u.cpu().numpy()
    want_pc = np.zeros((2, 8192))
    for e in range(n_envs):
        c = env_cart[e]
        o = oracle.Oracle(roms[c], mappers[c])
        o.rollout(wa[:, e], 1, screens=False)
        o.set_ram(ram0[e].astype(np.uint8))
        g, ram_o, _ = o.soft_rollout(u[:, e].astype(np.float64), 1, 0.1, 6.0, gr[:, e].astype(np.float64),
                                     gs[:, e].astype(np.float64))
        assert np.array_equal(ram.detach().cpu().numpy()[:, e], ram_o.astype(np.float32))
        o_rom, o_ram0, o_u = g.reverse()
        want_pc[c, :len(roms[c])] += o_rom
        assert_grad_close(g_ram0[e], o_ram0, "grad_ram0 through autograd")
        assert_grad_close(g_u[:, e], o_u, "grad_u through autograd")
    assert_grad_close(g_rom, want_pc, "per-cart ROM gradient through autograd")


def test_gradients_through_the_extra_opcode_bytes():
    """LAX, SAX and USBC carry adjoints by their rules (LAX: both registers to
    the operand; SAX: the cell to A and X; USBC: as SBC); the unofficial NOPs
    carry none.  GPU gradients against the FP64 oracle on the extra-opcode
    cart."""
    from tests.microrom import extra_ops_rom
    torch = torch_cuda()
    rom = extra_ops_rom()
    n_envs, n_steps, tau = 4, 3, 0.1
    b = make_batch([rom], [synth.MAPPER_4K], [0] * n_envs)
    wa = synth.actions(39, n_envs, 2)
    gpu_rollout(b, wa, 1, screens=False)
    acts = synth.actions(38, n_envs, n_steps)
    u = synth.action_inputs(acts)
    gr = synth.normal_f32(38, (n_steps, n_envs, 128), 1)
    gs = synth.normal_f32(38, (n_steps, n_envs, 210, 160), 2)
    tape = b.soft_rollout(tau, torch.from_numpy(u).cuda(), 1)
    g_rom = torch.empty((n_envs, 8192), device="cuda")
    g_ram0 = torch.empty((n_envs, 128), device="cuda")
    g_u = torch.empty((n_steps, n_envs, 5), device="cuda")
    tape.backward(torch.from_numpy(gr).cuda(), torch.from_numpy(gs).cuda(), grad_rom=g_rom, grad_ram0=g_ram0,
                  grad_u=g_u)
    b.sync()
    g_rom, g_ram0, g_u = g_rom.cpu().numpy(), g_ram0.cpu().numpy(), g_u.cpu().numpy()
    for e in range(n_envs):
        (o_rom, o_ram0, o_u), _, _ = _oracle_grads(rom, synth.MAPPER_4K, wa[:, e], u[:, e], 1, tau,
                                                   gr[:, e], gs[:, e])
        assert np.abs(o_ram0).max() > 0 and np.abs(o_rom).max() > 0
        assert_grad_close(g_rom[e, :4096], o_rom, f"grad_rom env {e}")
        assert_grad_close(g_ram0[e], o_ram0, f"grad_ram0 env {e}")
        assert_grad_close(g_u[:, e], o_u, f"grad_u env {e}")


@pytest.mark.parametrize("cart,tpe,seg", [("synthetic", 4, 64), ("synthetic", 1, 2), ("resp_each_frame", 4, 64),
                                          ("resp_each_frame_pf_first", 2, 64), ("resp_once", 4, 2),
                                          ("resp_once", 1, 64)])
def test_position_sampler_gradients_match_oracle(cart, tpe, seg):
    """The position sampler (Section 3) on the GPU against the FP64 oracle:
    synthetic carts (RESP0, HMP0 and HMOVE among their writes, three
    mappers) and the sampler carts, whose joystick moves player 0 through
    HMP0 each frame; with two-frame segments the position and HMP0 adjoints
    cross segment boundaries."""
    from tests.microrom import sampler_rom
    torch = torch_cuda()
    if cart == "synthetic":
        mappers = [synth.MAPPER_2K, synth.MAPPER_4K, synth.MAPPER_F8]
        roms = synth.config_carts(61, mappers)
    else:
        mappers = [synth.MAPPER_4K]
        roms = [sampler_rom(cart != "resp_once", 4 if cart.endswith("pf_first") else 0)]
    n_envs, n_steps, tau = 6, 5, 0.1
    env_cart = (np.arange(n_envs) % len(mappers)).astype(np.int32)
    b = make_batch(roms, mappers, env_cart, envs_per_block=8, threads_per_env=tpe, segment_frames=seg,
                   position_sampler=1)
    wa = synth.actions(62, n_envs, 2)
    gpu_rollout(b, wa, 1, screens=False)
    u = synth.action_inputs(synth.actions(63, n_envs, n_steps))
    gr = synth.normal_f32(63, (n_steps, n_envs, 128), 1)
    gs = synth.normal_f32(63, (n_steps, n_envs, 210, 160), 2)
    tape = b.soft_rollout(tau, torch.from_numpy(u).cuda(), 1)
    g_rom = torch.empty((n_envs, 8192), device="cuda")
    g_ram0 = torch.empty((n_envs, 128), device="cuda")
    g_u = torch.empty((n_steps, n_envs, 5), device="cuda")
    tape.backward(torch.from_numpy(gr).cuda(), torch.from_numpy(gs).cuda(), grad_rom=g_rom, grad_ram0=g_ram0,
                  grad_u=g_u)
    b.sync()
    g_rom, g_ram0, g_u = g_rom.cpu().numpy(), g_ram0.cpu().numpy(), g_u.cpu().numpy()
    for e in range(n_envs):
        c = env_cart[e]
        (o_rom, o_ram0, o_u), _, _ = _oracle_grads(roms[c], mappers[c], wa[:, e], u[:, e], 1, tau,
                                                   gr[:, e], gs[:, e], sampler=True)
        size = len(roms[c])
        assert_grad_close(g_rom[e, :size], o_rom, f"grad_rom env {e}")
        assert_grad_close(g_ram0[e], o_ram0, f"grad_ram0 env {e}")
        assert_grad_close(g_u[:, e], o_u, f"grad_u env {e}")
        if cart != "synthetic":
            assert np.abs(o_u).max() > 100, "the joystick must move the sprite"


def test_backward_geometry_past_its_shared_memory():
    """128 envs per block: the backward runs on its own 64-env block table
    (same permutation) and gives the gradients of an 8-env geometry, bit for
    bit (each env's arithmetic does not depend on the blocking)."""
    torch = torch_cuda()
    mappers = [synth.MAPPER_4K, synth.MAPPER_F8]
    n_envs, n_steps = 150, 3
    res = []
    for epb in (8, 128):
        _, roms, env_cart, b, wa, acts, u = _setup(mappers, n_envs, n_steps, 91, envs_per_block=epb)
        gr = synth.normal_f32(91, (n_steps, n_envs, 128), 1)
        tape = b.soft_rollout(0.1, torch.from_numpy(u).cuda(), 1)
        g_rom = torch.empty((n_envs, 8192), device="cuda")
        g_u = torch.empty((n_steps, n_envs, 5), device="cuda")
        tape.backward(torch.from_numpy(gr).cuda(), None, grad_rom=g_rom, grad_u=g_u)
        b.sync()
        res.append((g_rom.cpu().numpy(), g_u.cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert np.abs(res[1][0]).max() > 0


@pytest.mark.parametrize("tpe", [1, 4])
def test_gradients_on_f6_f4_carts(tpe):
    """Bank-switched 16 and 32 KB carts: ROM gradients over the whole image
    (rows of the batch's 32 KB ROM stride; reads relaxed within their 4 KB
    bank), initial RAM and inputs against the FP64 oracle."""
    mappers = [synth.MAPPER_F6, synth.MAPPER_F4, synth.MAPPER_4K]
    n_envs, n_steps, tau = 6, 4, 0.1
    torch, roms, env_cart, b, wa, acts, u = _setup(mappers, n_envs, n_steps, 71, envs_per_block=8,
                                                   threads_per_env=tpe)
    assert b.rom_stride == 32768
    gr = synth.normal_f32(71, (n_steps, n_envs, 128), 1)
    gs = synth.normal_f32(71, (n_steps, n_envs, 210, 160), 2)
    tape = b.soft_rollout(tau, torch.from_numpy(u).cuda(), 1)
    g_rom = torch.empty((n_envs, b.rom_stride), device="cuda")
    g_ram0 = torch.empty((n_envs, 128), device="cuda")
    g_u = torch.empty((n_steps, n_envs, 5), device="cuda")
    g_pc = torch.empty((len(mappers), b.rom_stride), device="cuda")
    tape.backward(torch.from_numpy(gr).cuda(), torch.from_numpy(gs).cuda(), grad_rom=g_rom, grad_ram0=g_ram0,
                  grad_u=g_u, grad_rom_per_cart=g_pc)
    b.sync()
    g_rom, g_ram0, g_u, g_pc = g_rom.cpu().numpy(), g_ram0.cpu().numpy(), g_u.cpu().numpy(), g_pc.cpu().numpy()
    want_pc = np.zeros_like(g_pc)
    for e in range(n_envs):
        c = env_cart[e]
        (o_rom, o_ram0, o_u), _, _ = _oracle_grads(roms[c], mappers[c], wa[:, e], u[:, e], 1, tau, gr[:, e],
                                                   gs[:, e])
        size = len(roms[c])
        assert_grad_close(g_rom[e, :size], o_rom, f"grad_rom env {e}")
        assert np.all(g_rom[e, size:] == 0)
        assert_grad_close(g_ram0[e], o_ram0, f"grad_ram0 env {e}")
        assert_grad_close(g_u[:, e], o_u, f"grad_u env {e}")
        want_pc[c, :size] += o_rom
    assert_grad_close(g_pc, want_pc, "per-cart ROM gradient")


def test_wide_recompute_of_a_large_segment_group():
    """32 one-frame segments x 512 envs = 16,384 machines: the group's
    recompute runs one lane per env (blocks of 32) instead of the batch's 4
    replicas; the gradients match the FP64 oracle and a one-segment-at-a-time
    backward (tape budget of 1 MB)."""
    torch = torch_cuda()
    mappers = [synth.MAPPER_4K, synth.MAPPER_F8]
    n_envs, n_steps, tau = 512, 32, 0.1
    res = []
    for budget in (0, 1):
        _, roms, env_cart, b, wa, acts, u = _setup(mappers, n_envs, n_steps, 93, segment_frames=1,
                                                   threads_per_env=4, tape_budget_mb=budget)
        gr = synth.normal_f32(93, (n_steps, n_envs, 128), 1)
        wscr = synth.normal_f32(94, (210 * 160,), 1)
        tape = b.soft_rollout(tau, torch.from_numpy(u).cuda(), 1)
        g_rom = torch.empty((n_envs, 8192), device="cuda")
        g_u = torch.empty((n_steps, n_envs, 5), device="cuda")
        tape.backward(torch.from_numpy(gr).cuda(), None, grad_rom=g_rom, grad_u=g_u)
        b.sync()
        res.append((g_rom.cpu().numpy(), g_u.cpu().numpy()))
    for e in (0, 1, 257, 511):
        c = env_cart[e]
        (o_rom, _, o_u), _, _ = _oracle_grads(roms[c], mappers[c], wa[:, e], u[:, e], 1, tau, gr[:, e], None)
        for g_rom, g_u in res:
            assert_grad_close(g_rom[e, :len(roms[c])], o_rom, f"grad_rom env {e}")
            assert_grad_close(g_u[:, e], o_u, f"grad_u env {e}")


@pytest.mark.parametrize("tpe,seg", [(1, 64), (4, 2)])
def test_gradients_on_superchip_carts(tpe, seg):
    """F8SC / F6SC / F4SC carts: the cartridge RAM is a second RAM tensor
    (relaxed reads within it, one-hot writes), so its adjoints ride the
    sweep and the checkpoint carry; grad_cart_ram0, ROM, initial RAM and
    input gradients against the FP64 oracle, over one and several segments."""
    mappers = [synth.MAPPER_F8SC, synth.MAPPER_F6SC, synth.MAPPER_F4SC, synth.MAPPER_4K]
    n_envs, n_steps, tau = 8, 4, 0.3
    torch, roms, env_cart, b, wa, acts, u = _setup(mappers, n_envs, n_steps, 75, envs_per_block=8,
                                                   threads_per_env=tpe, segment_frames=seg)
    gr = synth.normal_f32(75, (n_steps, n_envs, 128), 1)
    gs = synth.normal_f32(75, (n_steps, n_envs, 210, 160), 2)
    tape = b.soft_rollout(tau, torch.from_numpy(u).cuda(), 1)
    g_rom = torch.empty((n_envs, b.rom_stride), device="cuda")
    g_ram0 = torch.empty((n_envs, 128), device="cuda")
    g_cram0 = torch.full((n_envs, 128), 7.0, device="cuda")
    g_u = torch.empty((n_steps, n_envs, 5), device="cuda")
    tape.backward(torch.from_numpy(gr).cuda(), torch.from_numpy(gs).cuda(), grad_rom=g_rom, grad_ram0=g_ram0,
                  grad_u=g_u, grad_cart_ram0=g_cram0)
    b.sync()
    g_rom, g_ram0, g_cram0, g_u = (x.cpu().numpy() for x in (g_rom, g_ram0, g_cram0, g_u))
    for e in range(n_envs):
        c = env_cart[e]
        o = oracle.Oracle(roms[c], mappers[c])
        o.rollout(wa[:, e], 1, screens=False)
        g, _, _ = o.soft_rollout(u[:, e].astype(np.float64), 1, tau, 6.0, gr[:, e].astype(np.float64),
                                 gs[:, e].astype(np.float64))
        o_rom, o_ram0, o_u, o_cram0 = g.reverse(cart_ram=True)
        size = len(roms[c])
        assert_grad_close(g_rom[e, :size], o_rom, f"grad_rom env {e}")
        assert_grad_close(g_ram0[e], o_ram0, f"grad_ram0 env {e}")
        assert_grad_close(g_cram0[e], o_cram0, f"grad_cart_ram0 env {e}")
        assert_grad_close(g_u[:, e], o_u, f"grad_u env {e}")
        if mappers[c] == synth.MAPPER_4K:
            assert not g_cram0[e].any()
        else:
            assert np.abs(o_cram0).max() > 0


@pytest.mark.parametrize("tpe", [1, 4])
def test_gradients_on_e0_carts(tpe):
    """E0 carts: ROM reads are relaxed within the 1 KB slice their segment
    shows (the tape keeps the slice per record); ROM, initial RAM and input
    gradients against the FP64 oracle, with Superchip and FE carts (reads
    relaxed within the 4 KB bank JSR and RTS selected) in the same batch and
    several checkpoint segments."""
    mappers = [synth.MAPPER_E0, synth.MAPPER_F6SC, synth.MAPPER_E0, synth.MAPPER_FE]
    n_envs, n_steps, tau = 8, 4, 0.1
    torch, roms, env_cart, b, wa, acts, u = _setup(mappers, n_envs, n_steps, 77, envs_per_block=8,
                                                   threads_per_env=tpe, segment_frames=2)
    gr = synth.normal_f32(77, (n_steps, n_envs, 128), 1)
    gs = synth.normal_f32(77, (n_steps, n_envs, 210, 160), 2)
    tape = b.soft_rollout(tau, torch.from_numpy(u).cuda(), 1)
    g_rom = torch.empty((n_envs, b.rom_stride), device="cuda")
    g_ram0 = torch.empty((n_envs, 128), device="cuda")
    g_u = torch.empty((n_steps, n_envs, 5), device="cuda")
    g_pc = torch.empty((len(mappers), b.rom_stride), device="cuda")
    tape.backward(torch.from_numpy(gr).cuda(), torch.from_numpy(gs).cuda(), grad_rom=g_rom, grad_ram0=g_ram0,
                  grad_u=g_u, grad_rom_per_cart=g_pc)
    b.sync()
    g_rom, g_ram0, g_u, g_pc = (x.cpu().numpy() for x in (g_rom, g_ram0, g_u, g_pc))
    want_pc = np.zeros_like(g_pc)
    for e in range(n_envs):
        c = env_cart[e]
        (o_rom, o_ram0, o_u), _, _ = _oracle_grads(roms[c], mappers[c], wa[:, e], u[:, e], 1, tau, gr[:, e],
                                                   gs[:, e])
        size = len(roms[c])
        assert_grad_close(g_rom[e, :size], o_rom, f"grad_rom env {e}")
        assert np.all(g_rom[e, size:] == 0)
        assert_grad_close(g_ram0[e], o_ram0, f"grad_ram0 env {e}")
        assert_grad_close(g_u[:, e], o_u, f"grad_u env {e}")
        want_pc[c, :size] += o_rom
        if mappers[c] == synth.MAPPER_E0:
            assert np.count_nonzero(np.abs(o_rom.reshape(8, 1024)).sum(1)) >= 3   # several slices read
    assert_grad_close(g_pc, want_pc, "per-cart ROM gradient")


def test_soft_step_entry_point():
    """vcs_soft_step (the problem statement's soft step) through the C ABI:
    its forward equals vcs_soft_rollout's from the batch's own ROMs and RAM
    bit for bit (and so the hard path's, Theorem 1); the backward of its
    tape equals that of vcs_soft_rollout's bit for bit and the FP64
    oracle's within the gradient tolerance; tau <= 0 is refused."""
    import ctypes as C

    from paper_2606_22447_b300 import _lib
    torch = torch_cuda()
    mappers = [synth.MAPPER_4K, synth.MAPPER_F8]
    n_envs, n_steps = 6, 3
    _, roms, env_cart, b, wa, acts, u = _setup(mappers, n_envs, n_steps, 67)
    L = _lib.load()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda t: C.c_void_p(t.data_ptr())
    u_t = torch.from_numpy(u).cuda()
    blob = b.save_state()
    outs = []
    for entry in ("vcs_soft_step", "vcs_soft_rollout"):
        b.load_state(blob)
        ram = torch.empty((n_steps, n_envs, 128), device="cuda")
        scr = torch.empty((n_steps, n_envs, 210, 160), device="cuda")
        h = C.c_void_p()
        if entry == "vcs_soft_step":
            st = L.vcs_soft_step(b.h, 0.1, p(u_t), n_steps, 1, p(ram), p(scr), C.byref(h), s)
        else:
            st = L.vcs_soft_rollout(b.h, 0.1, None, None, p(u_t), n_steps, 1, p(ram), p(scr), C.byref(h), s)
        _lib.check(st, b.h)
        g_ram0 = torch.zeros((n_envs, 128), device="cuda")
        g_u = torch.zeros((n_steps, n_envs, 5), device="cuda")
        g_rom = torch.zeros((n_envs, b.rom_stride), device="cuda")
        gr = torch.from_numpy(synth.normal_f32(67, (n_steps, n_envs, 128), 1)).cuda()
        _lib.check(L.vcs_backward(h, p(gr), None, None, p(g_rom), p(g_ram0), None, p(g_u), None, s), b.h)
        b.sync()
        outs.append([x.cpu().numpy() for x in (ram, scr, g_rom, g_ram0, g_u)])
        L.vcs_tape_free(h)
    for x, y in zip(*outs):
        assert np.array_equal(x, y)
    ram, scr, g_rom, g_ram0, g_u = outs[0]
    gr = synth.normal_f32(67, (n_steps, n_envs, 128), 1)
    for e in range(n_envs):
        c = env_cart[e]
        (o_rom, o_ram0, o_u), ram_o, scr_o = _oracle_grads(roms[c], mappers[c], wa[:, e], u[:, e], 1, 0.1,
                                                           gr[:, e], None)
        assert np.array_equal(ram[:, e], ram_o.astype(np.float32))
        assert np.array_equal(scr[:, e], scr_o.astype(np.float32))
        assert_grad_close(g_ram0[e], o_ram0, f"env {e}: grad_ram0")
        assert_grad_close(g_u[:, e], o_u, f"env {e}: grad_u")
        assert_grad_close(g_rom[e, :len(o_rom)], o_rom, f"env {e}: grad_rom")
    h = C.c_void_p()
    assert L.vcs_soft_step(b.h, 0.0, p(u_t), n_steps, 1, None, None, C.byref(h), s) == _lib.VCS_ERR_ARG
    assert not h.value


@pytest.mark.parametrize("ctrlpf,tpe", [(0, 1), (1, 4), (4, 4), (4, 1)])
def test_graphics_bit_gradients_on_the_graphics_cart(ctrlpf, tpe):
    """The graphics-bit surrogate on the GPU (vcs_config.graphics_bits): the
    oracle's pin cart (GRP0 from the joystick, PF0-2 from immediates, plain,
    reflected and playfield-first priority), joystick and ROM gradients
    against the FP64 oracle."""
    from tests.microrom import graphics_rom
    torch = torch_cuda()
    rom, _ = graphics_rom(ctrlpf)
    n_envs, n_steps, tau = 6, 4, 0.01
    b = make_batch([rom], [synth.MAPPER_4K], np.zeros(n_envs, np.int32), graphics_bits=1, threads_per_env=tpe,
                   envs_per_block=8, segment_frames=2)
    acts = synth.actions(91 + ctrlpf, n_envs, n_steps)
    u = synth.action_inputs(acts)
    gs = synth.normal_f32(91, (n_steps, n_envs, 210, 160), 2)
    tape = b.soft_rollout(tau, torch.from_numpy(u).cuda(), 1)
    g_rom = torch.empty((n_envs, b.rom_stride), device="cuda")
    g_u = torch.empty((n_steps, n_envs, 5), device="cuda")
    tape.backward(None, torch.from_numpy(gs).cuda(), grad_rom=g_rom, grad_u=g_u)
    b.sync()
    g_rom, g_u = g_rom.cpu().numpy(), g_u.cpu().numpy()
    for e in range(n_envs):
        o = oracle.Oracle(rom, synth.MAPPER_4K)
        o.set_graphics(True)
        g, _, _ = o.soft_rollout(u[:, e].astype(np.float64), 1, tau, 6.0, None, gs[:, e].astype(np.float64),
                                 outputs=False)
        o_rom, _, o_u = g.reverse()
        assert np.abs(o_u).max() > 1.0
        assert_grad_close(g_u[:, e], o_u, f"env {e} grad_u")
        assert_grad_close(g_rom[e, :4096], o_rom, f"env {e} grad_rom")


@pytest.mark.parametrize("tpe,seg", [(1, 64), (4, 2)])
def test_graphics_bit_gradients_on_synthetic_carts(tpe, seg):
    """Generated carts of several formats (their kernels store GRP0 and the
    playfield on every line) with the graphics-bit surrogate on and the
    position sampler on in one case: ROM, initial RAM and input gradients
    against the FP64 oracle over one and several checkpoint segments."""
    mappers = [synth.MAPPER_4K, synth.MAPPER_F8, synth.MAPPER_2K, synth.MAPPER_FE]
    n_envs, n_steps, tau = 8, 4, 0.1
    sampler = seg == 2
    torch, roms, env_cart, b, wa, acts, u = _setup(mappers, n_envs, n_steps, 93, envs_per_block=8,
                                                   threads_per_env=tpe, segment_frames=seg, graphics_bits=1,
                                                   position_sampler=1 if sampler else 0)
    gr = synth.normal_f32(93, (n_steps, n_envs, 128), 1)
    gs = synth.normal_f32(93, (n_steps, n_envs, 210, 160), 2)
    tape = b.soft_rollout(tau, torch.from_numpy(u).cuda(), 1)
    g_rom = torch.empty((n_envs, b.rom_stride), device="cuda")
    g_ram0 = torch.empty((n_envs, 128), device="cuda")
    g_u = torch.empty((n_steps, n_envs, 5), device="cuda")
    tape.backward(torch.from_numpy(gr).cuda(), torch.from_numpy(gs).cuda(), grad_rom=g_rom, grad_ram0=g_ram0,
                  grad_u=g_u)
    b.sync()
    g_rom, g_ram0, g_u = g_rom.cpu().numpy(), g_ram0.cpu().numpy(), g_u.cpu().numpy()
    for e in range(n_envs):
        c = env_cart[e]
        o = oracle.Oracle(roms[c], mappers[c])
        o.rollout(wa[:, e], 1, screens=False)
        o.set_graphics(True)
        o.set_sampler(sampler)
        g, _, _ = o.soft_rollout(u[:, e].astype(np.float64), 1, tau, 6.0, gr[:, e].astype(np.float64),
                                 gs[:, e].astype(np.float64), outputs=False)
        o_rom, o_ram0, o_u = g.reverse()
        assert_grad_close(g_rom[e, :len(roms[c])], o_rom, f"env {e} grad_rom")
        assert_grad_close(g_ram0[e], o_ram0, f"env {e} grad_ram0")
        assert_grad_close(g_u[:, e], o_u, f"env {e} grad_u")


@pytest.mark.parametrize("ctrlpf,vdel,tpe", [(0, False, 1), (4, False, 4), (0, True, 4)])
def test_whole_tia_graphics_bits_on_the_pin_cart(ctrlpf, vdel, tpe):
    """The graphics-bit surrogate with the whole TIA: the oracle's pin cart
    (player 1 from the joystick, GRP0, ENAM0, ENABL and PF0-2 from
    immediates; playfield-first priority; player 1 through its delayed
    copy), joystick and ROM gradients against the FP64 oracle."""
    from tests.microrom import graphics_full_tia_rom
    torch = torch_cuda()
    rom, _ = graphics_full_tia_rom(ctrlpf, vdel)
    n_envs, n_steps, tau = 8, 4, 0.01
    b = make_batch([rom], [synth.MAPPER_4K], np.zeros(n_envs, np.int32), graphics_bits=1, full_tia=1,
                   threads_per_env=tpe, envs_per_block=8, segment_frames=2)
    acts = synth.actions(97 + ctrlpf + vdel, n_envs, n_steps)
    u = synth.action_inputs(acts)
    gs = synth.normal_f32(97, (n_steps, n_envs, 210, 160), 2)
    tape = b.soft_rollout(tau, torch.from_numpy(u).cuda(), 1)
    g_rom = torch.empty((n_envs, b.rom_stride), device="cuda")
    g_u = torch.empty((n_steps, n_envs, 5), device="cuda")
    tape.backward(None, torch.from_numpy(gs).cuda(), grad_rom=g_rom, grad_u=g_u)
    b.sync()
    g_rom, g_u = g_rom.cpu().numpy(), g_u.cpu().numpy()
    for e in range(n_envs):
        o = oracle.Oracle(rom, synth.MAPPER_4K, full_tia=True)
        o.set_graphics(True)
        g, _, _ = o.soft_rollout(u[:, e].astype(np.float64), 1, tau, 6.0, None, gs[:, e].astype(np.float64),
                                 outputs=False)
        o_rom, _, o_u = g.reverse()
        assert np.abs(o_u).max() > 1.0
        assert_grad_close(g_u[:, e], o_u, f"env {e} grad_u")
        assert_grad_close(g_rom[e, :4096], o_rom, f"env {e} grad_rom")


@pytest.mark.parametrize("tpe,seg", [(1, 64), (4, 2)])
def test_whole_tia_graphics_bits_on_synthetic_carts(tpe, seg):
    """Full-TIA carts (players, missiles, ball, sizes, delays, collisions)
    with the graphics-bit surrogate: ROM, initial RAM and input gradients
    against the FP64 oracle over one and several segments."""
    torch = torch_cuda()
    mappers = [synth.MAPPER_4K, synth.MAPPER_F8, synth.MAPPER_E0, synth.MAPPER_F6SC]
    n_envs, n_steps, tau = 8, 3, 0.1
    roms = synth.config_carts(99, mappers, full_tia=True)
    env_cart = (np.arange(n_envs) % len(mappers)).astype(np.int32)
    b = make_batch(roms, mappers, env_cart, full_tia=1, graphics_bits=1, envs_per_block=8, threads_per_env=tpe,
                   segment_frames=seg)
    wa = synth.actions(100, n_envs, 2)
    gpu_rollout(b, wa, 1, screens=False)
    u = synth.action_inputs(synth.actions(99, n_envs, n_steps))
    gr = synth.normal_f32(99, (n_steps, n_envs, 128), 1)
    gs = synth.normal_f32(99, (n_steps, n_envs, 210, 160), 2)
    tape = b.soft_rollout(tau, torch.from_numpy(u).cuda(), 1)
    g_rom = torch.empty((n_envs, b.rom_stride), device="cuda")
    g_ram0 = torch.empty((n_envs, 128), device="cuda")
    g_u = torch.empty((n_steps, n_envs, 5), device="cuda")
    tape.backward(torch.from_numpy(gr).cuda(), torch.from_numpy(gs).cuda(), grad_rom=g_rom, grad_ram0=g_ram0,
                  grad_u=g_u)
    b.sync()
    g_rom, g_ram0, g_u = g_rom.cpu().numpy(), g_ram0.cpu().numpy(), g_u.cpu().numpy()
    for e in range(n_envs):
        c = env_cart[e]
        o = oracle.Oracle(roms[c], mappers[c], full_tia=True)
        o.rollout(wa[:, e], 1, screens=False)
        o.set_graphics(True)
        g, _, _ = o.soft_rollout(u[:, e].astype(np.float64), 1, tau, 6.0, gr[:, e].astype(np.float64),
                                 gs[:, e].astype(np.float64), outputs=False)
        o_rom, o_ram0, o_u = g.reverse()
        assert_grad_close(g_rom[e, :len(roms[c])], o_rom, f"env {e} grad_rom")
        assert_grad_close(g_ram0[e], o_ram0, f"env {e} grad_ram0")
        assert_grad_close(g_u[:, e], o_u, f"env {e} grad_u")
