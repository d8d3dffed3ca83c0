"""Pins of the oracle's instruction-granular steps (the paper's throughput
unit, Section 6: one step = one emulated instruction).

A frame step ends right after the instruction whose VSYNC write ends the
frame, so a frame step that executed D instructions (the oracle's counter)
and an instruction step of D slots from the same state must leave the same
machine; soft rollouts of the two must give the same gradients for a RAM
loss.  The counter itself is pinned to the per-instruction trace.
"""
import numpy as np
import pytest

from paper_2606_22447_b300 import synth

oracle = pytest.importorskip("oracle")

MAPPERS = [synth.MAPPER_2K, synth.MAPPER_4K, synth.MAPPER_F8]


def _cart(i, seed=71):
    return synth.config_carts(seed, MAPPERS)[i], MAPPERS[i]


@pytest.mark.parametrize("cart", [0, 1, 2])
def test_instruction_steps_equal_frame_steps(cart):
    rom, mapper = _cart(cart)
    acts = synth.actions(72, 1, 6)[:, 0]
    a = oracle.Oracle(rom, mapper)
    b = oracle.Oracle(rom, mapper)
    for t in range(6):
        n0 = a.counters()["instructions"]
        ram_a, _, st_a = a.step(int(acts[t]), 1)
        d = a.counters()["instructions"] - n0
        assert st_a == 0 and d > 100
        b.set_step_instructions(d)
        ram_b, _, st_b = b.step(int(acts[t]), 1)
        assert st_b == 0
        assert np.array_equal(ram_a, ram_b)
        assert np.array_equal(a.state(), b.state()), f"step {t}"
        assert b.counters()["instructions"] == a.counters()["instructions"]
        assert b.counters()["frames"] == a.counters()["frames"]


def test_instruction_step_counts_slots_and_crosses_frames():
    """A step of n slots executes exactly n instructions (no jam), whatever
    frames end inside it; the state matches the per-instruction trace."""
    rom, mapper = _cart(1)
    a = oracle.Oracle(rom, mapper)
    b = oracle.Oracle(rom, mapper)
    a.set_step_instructions(7919)
    for t in range(4):
        n0, f0 = a.counters()["instructions"], a.counters()["frames"]
        a.step(3, 1)
        assert a.counters()["instructions"] - n0 == 7919
        assert a.counters()["frames"] - f0 in (2, 3, 4)   # a few thousand instructions per frame
        b.trace(3, 7919)
        assert np.array_equal(a.state(), b.state())
        assert np.array_equal(a.ram(), b.ram())


def test_jammed_cpu_slots_count():
    """A jammed CPU idles one line per slot: n slots advance n lines."""
    def build(asm):
        asm.op("LDA", "imm", 1)
        asm.byte(0x02)              # an undocumented byte outside the paper's 38: jams
    from tests.microrom import rom4k
    o = oracle.Oracle(rom4k(build), synth.MAPPER_4K)
    o.set_step_instructions(10)
    o.step(0, 1)                    # LDA, the jam, then 8 idle slots
    s = o.state()
    assert s[28] == 1               # jammed
    assert int(s[6]) % 76 == 0 and int(s[6]) // 76 == 8


@pytest.mark.parametrize("tau", [0.1, 1.0])
def test_soft_instruction_step_equals_frame_step_gradients(tau):
    rom, mapper = _cart(2)
    acts = synth.actions(73, 1, 3)[:, 0]
    r = np.random.default_rng(74)
    u = (r.random((1, 5)) < 0.5).astype(float)
    gr = r.standard_normal((1, 128))
    outs = []
    for mode in ("frames", "instructions"):
        o = oracle.Oracle(rom, mapper)
        o.rollout(acts, 1, screens=False)
        if mode == "frames":
            n0 = o.counters()["instructions"]
        else:
            o.set_step_instructions(d)
        g, ram, _ = o.soft_rollout(u, 1, tau, 6.0, gr, None)
        if mode == "frames":
            d = o.counters()["instructions"] - n0
        outs.append((g.reverse(), ram))
    (g1, ram1), (g2, ram2) = outs
    assert np.array_equal(ram1, ram2)
    for x, y in zip(g1, g2):
        assert np.array_equal(x, y)
    assert np.abs(g1[0]).max() > 0


def test_soft_instruction_steps_reverse_equals_tangent_and_differences():
    rom, mapper = _cart(1)
    o = oracle.Oracle(rom, mapper)
    o.rollout(synth.actions(76, 1, 2)[:, 0], 1, screens=False)   # past the RAM-clearing init
    o.set_step_instructions(1500)
    r = np.random.default_rng(75)
    n = 4
    u = (r.random((n, 5)) < 0.5).astype(float)
    gr = r.standard_normal((n, 128))
    g, _, _ = o.soft_rollout(u, 1, 0.1, 6.0, gr, None)
    g_rom, g_ram0, g_u = g.reverse()
    d_rom, d_ram, d_u = r.standard_normal(len(rom)), r.standard_normal(128), r.standard_normal((n, 5))
    lin = (g_rom * d_rom).sum() + (g_ram0 * d_ram).sum() + (g_u * d_u).sum()
    assert g.tangent(d_rom, d_ram, d_u) == pytest.approx(lin, rel=1e-10, abs=1e-8)
    h = 1e-3
    fd = (g.eval(d_rom * h, d_ram * h, d_u * h) - g.eval(-d_rom * h, -d_ram * h, -d_u * h)) / (2 * h)
    assert fd == pytest.approx(lin, rel=1e-8, abs=1e-6)
    assert np.abs(g_ram0).max() > 0 and np.abs(g_rom).max() > 0
