"""Deferred rasterisation: the step kernel logs the returned frame's
picture-register writes and the raster kernel draws the screens from the
logs.  Its screens must equal, bit for bit, both the step kernel's own
drawing (inline_render = 1) and the oracle's, including frames that write
a picture register every few cycles for 512 lines, boot frames, auto-resets
and CUDA-graph replays."""
import numpy as np
import pytest

import oracle
from paper_2606_22447_b300 import synth
from tests.gpu_util import assert_env_equal, gpu_rollout, make_batch, oracle_rollout, torch_cuda
from tests.microrom import brk_pushes_rom, dense_writes_rom, graphics_full_tia_rom

pytestmark = pytest.mark.gpu

# every cartridge format of the subset machine's kernels, two carts each
MAPPERS = [synth.MAPPER_2K, synth.MAPPER_4K, synth.MAPPER_F8, synth.MAPPER_F6, synth.MAPPER_F4,
           synth.MAPPER_F8SC, synth.MAPPER_E0, synth.MAPPER_FE] * 2


def _pair(roms, mappers, env_cart, acts, frame_skip, setup=None, **cfg):
    """The same rollout with deferred and with inline drawing."""
    out = []
    for inline in (0, 1):
        b = make_batch(roms, mappers, env_cart, inline_render=inline, **cfg)
        if setup:
            setup(b)
        out.append(gpu_rollout(b, acts, frame_skip))
        b.close()
    return out


@pytest.mark.parametrize("frame_skip", [1, 4])
@pytest.mark.parametrize("epb", [16, 128])
def test_deferred_equals_inline_every_format(frame_skip, epb):
    roms = synth.config_carts(707, MAPPERS)
    n = 150   # ragged blocks
    env_cart = np.random.default_rng(7).permutation(np.arange(n) % len(MAPPERS)).astype(np.int32)
    acts = synth.actions(707, n, 6)
    (r0, s0, t0), (r1, s1, t1) = _pair(roms, MAPPERS, env_cart, acts, frame_skip, envs_per_block=epb)
    assert np.array_equal(r0, r1) and np.array_equal(t0, t1)
    bad = np.argwhere(s0 != s1)
    assert bad.size == 0, f"{len(bad)} pixels differ, first at {bad[0].tolist()}"


@pytest.mark.parametrize("which", ["dense", "brk"])
@pytest.mark.parametrize("frame_skip", [1, 2])
def test_frames_with_ten_thousand_writes(which, frame_skip):
    """Frames that write a picture register every three cycles (or three
    in seven, BRK pushing onto the TIA) for 512 lines: logs of over ten
    thousand entries, drawn bit-exact with the oracle."""
    rom = dense_writes_rom() if which == "dense" else brk_pushes_rom()
    o = oracle.Oracle(rom, synth.MAPPER_4K)
    o.step(0, 1)
    assert o.counters()["tia_writes"] > 10000
    n = 8
    acts = synth.actions(808, n, 3)
    b = make_batch([rom], [synth.MAPPER_4K], np.zeros(n, np.int32))
    ram, scr, st = gpu_rollout(b, acts, frame_skip)
    for e in range(n):
        r2, s2, st2 = oracle_rollout(rom, synth.MAPPER_4K, acts[:, e], frame_skip)
        assert_env_equal(e, ram[:, e], r2, "RAM")
        assert_env_equal(e, scr[:, e], s2, "screen")
        assert_env_equal(e, st[:, e], st2, "status")


def test_boot_frames_and_auto_reset():
    """Episodes end inside the rollout and power on again with a boot
    sequence (frames without screens) before the next step."""
    mappers = [synth.MAPPER_4K, synth.MAPPER_F8]
    roms = synth.config_carts(909, mappers)
    n = 24
    env_cart = (np.arange(n) % 2).astype(np.int32)
    acts = synth.actions(909, n, 10)
    ep = np.random.default_rng(9).integers(2, 9, size=(n, 3)).astype(np.uint32)
    b = make_batch(roms, mappers, env_cart, boot_noop_frames=3, boot_reset_frames=2)
    b.set_episodes(ep)
    ram, scr, st = gpu_rollout(b, acts, 2)
    assert (st & 4).any()
    for e in range(n):
        c = int(env_cart[e])
        r2, s2, st2 = oracle_rollout(roms[c], mappers[c], acts[:, e], 2, ep_len=ep[e], boot=(3, 2))
        assert_env_equal(e, ram[:, e], r2, "RAM")
        assert_env_equal(e, scr[:, e], s2, "screen")
        assert_env_equal(e, st[:, e], st2, "status")


def test_graph_replay_with_deferred_raster():
    torch = torch_cuda()
    roms = synth.config_carts(1010, synth.MIX16)
    n = 256
    env_cart = synth.env_cart_round_robin(n, 16)
    acts = torch.from_numpy(synth.actions(1010, n, 3)).cuda()
    outs = []
    for use_graph in (False, True):
        b = make_batch(roms, synth.MIX16, env_cart)
        ram = torch.empty((3, n, 128), dtype=torch.uint8, device="cuda")
        scr = torch.empty((3, n, 210, 160), dtype=torch.uint8, device="cuda")
        if use_graph:
            g = b.graph(acts, 4, ram, scr)
            g.launch()
            torch.cuda.synchronize()
            g.destroy()
        else:
            b.rollout(acts, 4, ram, scr)
        b.sync()
        outs.append((ram.cpu().numpy(), scr.cpu().numpy()))
        b.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


FT_MAPPERS = [synth.MAPPER_2K, synth.MAPPER_4K, synth.MAPPER_F8, synth.MAPPER_F6, synth.MAPPER_F4,
              synth.MAPPER_F8SC, synth.MAPPER_F6SC, synth.MAPPER_F4SC, synth.MAPPER_E0, synth.MAPPER_FE]


@pytest.mark.parametrize("frame_skip", [1, 4])
@pytest.mark.parametrize("epb", [16, 64])
def test_whole_tia_deferred_equals_inline(frame_skip, epb):
    """The whole TIA: carts of all ten formats that draw with every object
    and read the collision latches; the raster kernel replays the logged
    writes (delayed graphics, missile locks, HMOVE of every object) and
    draws with the general renderer, bit for bit as the step kernel does."""
    roms = synth.config_carts(1111, FT_MAPPERS, full_tia=True)
    n = 90
    env_cart = np.random.default_rng(11).permutation(np.arange(n) % len(FT_MAPPERS)).astype(np.int32)
    acts = synth.actions(1111, n, 5)
    (r0, s0, t0), (r1, s1, t1) = _pair(roms, FT_MAPPERS, env_cart, acts, frame_skip, envs_per_block=epb,
                                       full_tia=1)
    assert np.array_equal(r0, r1) and np.array_equal(t0, t1)
    bad = np.argwhere(s0 != s1)
    assert bad.size == 0, f"{len(bad)} pixels differ, first at {bad[0].tolist()}"


@pytest.mark.parametrize("ctrlpf,vdel", [(0, False), (4, True), (2, True)])
def test_whole_tia_deferred_matches_oracle(ctrlpf, vdel):
    """Every object, vertical delay, playfield priority and score mode,
    deferred, against the oracle's colour-clock renderer."""
    rom, _ = graphics_full_tia_rom(ctrlpf=ctrlpf, vdel=vdel)
    n = 6
    acts = synth.actions(1212, n, 4)
    b = make_batch([rom], [synth.MAPPER_4K], np.zeros(n, np.int32), full_tia=1)
    ram, scr, st = gpu_rollout(b, acts, 2)
    for e in range(n):
        r2, s2, st2 = oracle_rollout(rom, synth.MAPPER_4K, acts[:, e], 2, full_tia=True)
        assert_env_equal(e, ram[:, e], r2, "RAM")
        assert_env_equal(e, scr[:, e], s2, "screen")
        assert_env_equal(e, st[:, e], st2, "status")


@pytest.mark.parametrize("full_tia", [0, 1])
def test_steps_without_screens_equal_inline(full_tia):
    """Without screens the step kernel built without drawing runs the whole
    rollout in one launch; RAM and status equal the drawing kernel's."""
    mappers = FT_MAPPERS if full_tia else MAPPERS
    roms = synth.config_carts(1313, mappers, full_tia=bool(full_tia))
    n = 70
    env_cart = (np.arange(n) % len(mappers)).astype(np.int32)
    acts = synth.actions(1313, n, 6)
    out = []
    for inline in (0, 1):
        b = make_batch(roms, mappers, env_cart, inline_render=inline, full_tia=full_tia)
        b.set_episodes(np.full((n, 2), 9, np.uint32))
        out.append(gpu_rollout(b, acts, 3, screens=False))
        b.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][2], out[1][2])



def test_kernel_timing_counts_the_two_kernels():
    """vcs_time_kernels / vcs_kernel_times: every timed step records the step
    kernel and the raster kernel, and the raster kernel counts the log
    entries it drew (one per picture-register write of the returned frame)."""
    torch = torch_cuda()
    rom = synth.generate_cart(2, 0, synth.MAPPER_4K)
    n = 64
    b = make_batch([rom], [synth.MAPPER_4K], np.zeros(n, np.int32))
    acts = torch.from_numpy(synth.actions(2, n, 3)).cuda()
    ram = torch.empty((n, 128), dtype=torch.uint8, device="cuda")
    scr = torch.empty((n, 210, 160), dtype=torch.uint8, device="cuda")
    b.step(acts[0], 4, ram, scr)
    b.time_kernels(True)
    for t in (1, 2):
        b.step(acts[t], 4, ram, scr)
    kt = b.kernel_times()
    b.time_kernels(False)
    assert kt["launches"] == 2 and kt["step_ms"] > 0 and kt["raster_ms"] > 0
    assert kt["log_entries"] > 100 * 2 * n   # a few hundred picture writes per env and frame
    assert b.kernel_times()["launches"] == 0   # reading clears the sums
    b.sync()
    b.close()
