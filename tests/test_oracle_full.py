"""Pins of the oracle's fully relaxed forward (FULL mode: the soft branch
without the straight-through correction and temperature-T reads, cast back
to integers; Section 4 and the supplement's temperature-limit study).

The boundaries come from the cast conditions in closed form, derived here
from the definitions rather than from the oracle's code:
* a read of a 0 byte whose neighbours in the window are all 255 returns
  255 S / (1 + S), S = sum_{k=1..W} 2 e^{-k/T}, and stays exact while that
  is below 1/2 (the paper's T <= 0.14 boundary, near 1/ln 1018);
* a branch of offset delta with a crisp flag lands on the hard counter
  while |delta| < tau_b(alpha) = (1 + e^alpha) / 2.
"""
import math

import numpy as np
import pytest

from paper_2606_22447_b300 import synth
from tests.microrom import FULL_T_LOOP, full_branch_rom, full_temperature_rom

oracle = pytest.importorskip("oracle")


def first_divergence(rom, mapper, T, alpha, n, action=0):
    """First instruction (1-based) after which the FULL machine's state
    differs from the hard machine's (registers, timer, TIA, RAM, clocks), or
    0 when the two agree for all n instructions."""
    h = oracle.Oracle(rom, mapper)
    f = oracle.Oracle(rom, mapper)
    f.set_full(2, T, alpha)
    for k in range(1, n + 1):
        h.trace(action, 1)
        f.trace(action, 1)
        if not (np.array_equal(h.state(), f.state()) and np.array_equal(h.ram(), f.ram())):
            return k
    return 0


def _window(T):
    return max(1, math.ceil(12 * T))


def _max_contrast_value(T):
    s = sum(2 * math.exp(-k / T) for k in range(1, _window(T) + 1))
    return 255 * s / (1 + s)


def _t_star():
    lo, hi = 0.10, 0.17
    for _ in range(100):
        mid = (lo + hi) / 2
        lo, hi = (mid, hi) if _max_contrast_value(mid) < 0.5 else (lo, mid)
    return lo


N_NOPS = FULL_T_LOOP - 0xF000


def test_temperature_boundary():
    t_star = _t_star()
    assert 0.144 < t_star < 0.1445          # the paper's exact side T <= 0.14, 1/ln(1018) = 0.1444
    rom = full_temperature_rom()
    for T in (0.08, 0.10, 0.12, 0.14, t_star - 1e-3):
        assert first_divergence(rom, 1, T, 6.0, N_NOPS + 30) == 0, T
    for T in (t_star + 1e-3, 0.15, 0.16, 0.17):
        assert first_divergence(rom, 1, T, 6.0, N_NOPS + 30) == N_NOPS + 1, T   # the first LDA


@pytest.mark.parametrize("T", [0.15, 0.16, 0.17])
def test_temperature_read_value(T):
    rom = full_temperature_rom()
    o = oracle.Oracle(rom, 1)
    o.set_full(2, T, 6.0)
    o.trace(0, N_NOPS + 2)                  # the NOPs, LDA, STA $80
    assert o.ram()[0] == round(_max_contrast_value(T)) == 1


@pytest.mark.parametrize("offset,taken", [(-3, True), (40, True), (40, False), (100, True), (-100, False)])
def test_branch_boundary(offset, taken):
    a_star = math.log(2 * abs(offset) - 1)  # |delta| = tau_b(alpha*)
    rom = full_branch_rom(offset, taken)
    at = 0x100 + 2                           # NOPs, LDX, the branch
    T = 0.05                                 # operand reads exact
    assert first_divergence(rom, 1, T, a_star - 0.05, at + 5) == at
    assert first_divergence(rom, 1, T, a_star + 0.05, at + 5) == 0


@pytest.mark.parametrize("mapper", [synth.MAPPER_2K, synth.MAPPER_4K, synth.MAPPER_F8])
def test_full_equals_hard_in_the_limit(mapper):
    """T -> 0 and alpha -> infinity: the FULL trajectory is the hard one."""
    rom = synth.config_carts(11, [mapper])[0]
    assert first_divergence(rom, mapper, 0.01, 20.0, 3000, action=3) == 0
    o = oracle.Oracle(rom, mapper)
    o.set_full(1, 0.01, 20.0)
    o.trace(3, 3000)
    c = o.counters()
    assert c["relaxed_reads"] > 1000 and c["relaxed_reads_exact"] == c["relaxed_reads"]
    assert c["branches"] > 100 and c["branches_exact"] == c["branches"]


def test_probe_mode_stays_hard_and_counts_cast_misses():
    """Probe mode executes the hard machine and counts the casts that would
    round off; the first count of a miss comes no later than the FULL
    machine's divergence."""
    rom = synth.config_carts(12, [synth.MAPPER_4K])[0]
    h = oracle.Oracle(rom, 1)
    p = oracle.Oracle(rom, 1)
    p.set_full(1, 0.2, 2.0)
    first_miss = 0
    for k in range(1, 801):
        h.trace(0, 1)
        p.trace(0, 1)
        assert np.array_equal(h.state(), p.state()) and np.array_equal(h.ram(), p.ram())
        c = p.counters()
        if not first_miss and (c["relaxed_reads_exact"] < c["relaxed_reads"] or
                               c["branches_exact"] < c["branches"]):
            first_miss = k
    assert first_miss > 0
    assert first_divergence(rom, 1, 0.2, 2.0, 800) >= first_miss
