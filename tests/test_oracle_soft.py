"""Pins of the oracle's soft (SOFT-STE) mode.

* the gate-gradient values and read/branch bounds the paper prints
  (tests/golden/relaxation_constants.txt);
* the relaxed read collapses to the one-hot read at small temperature and
  its address derivative matches finite differences;
* Theorem 1: the soft rollout's forward outputs equal the hard rollout's
  bit for bit at tau in {1, 0.1, 0.01};
* the reverse sweep equals the tangent sweep (transpose identity) and
  central finite differences of the frozen-switch relaxation;
* an analytic micro-program: d(sum of pixels)/d(ROM byte of LDA #k before
  STA COLUP0) equals the number of P0-owned pixels.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2606_22447_b300 import synth
from tests.microrom import rom4k

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "relaxation_constants.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("--")[0].strip()
        if line and not line.startswith("#"):
            name, v, tol = line.split()
            out[name] = (float(v), float(tol))
    return out


def test_gate_gradient_study_values():
    g = _golden()
    s = {a: oracle.gate_slope(a, 0.25) for a in (2.0, 6.0, 20.0)}
    peak = max(s.values())
    for a, key in ((2.0, "gate_rel_peak_alpha2"), (6.0, "gate_rel_peak_alpha6"), (20.0, "gate_rel_peak_alpha20")):
        v, tol = g[key]
        assert abs(s[a] / peak - v) <= tol, (a, s[a] / peak)
    v, tol = g["gate_abs_peak_alpha6"]
    assert abs(s[6.0] - v) <= tol


def _pull(T):
    r = np.array([255.0, 255.0, 0.0, 255.0, 255.0])
    v, _ = oracle.relaxed_read(r, 2, 2.0, T)
    return v


def test_read_pull_and_bounds():
    g = _golden()
    v, tol = g["read_pull_T014"]
    assert abs(_pull(0.14) - v) <= tol
    # the pull crosses 1/2 at the printed temperature bound
    lo, hi = 0.12, 0.17
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if _pull(mid) < 0.5 else (lo, mid)
    v, tol = g["read_bound_T"]
    assert abs(lo - v) <= tol, lo
    # branch: a taken gate with offset d rounds correctly iff d < (1 + e^a)/2
    v, tol = g["branch_bound_alpha"]
    alpha_min = math.log(2 * 127 - 1)
    assert abs(alpha_min - v) <= tol
    for a in (5.0, 6.0):
        gate = 1.0 / (1.0 + math.exp(-a))
        ok = all(abs((1 - gate) * d) < 0.5 for d in range(1, 128))
        assert ok == (a >= alpha_min)


def test_relaxed_read_limits_and_derivative():
    rng = np.random.default_rng(1)
    r = rng.integers(0, 256, 64).astype(np.float64)
    for a0 in (0, 1, 30, 63):
        v, d = oracle.relaxed_read(r, a0, float(a0), 0.01)
        assert abs(v - r[a0]) < 1e-30 and abs(d) < 1e-30
    for tau in (1.0, 0.3):
        for a in (10.3, 20.6):
            a0 = int(round(a))
            h = 1e-5
            vp, _ = oracle.relaxed_read(r, a0, a + h, tau)
            vm, _ = oracle.relaxed_read(r, a0, a - h, tau)
            _, d = oracle.relaxed_read(r, a0, a, tau)
            assert abs((vp - vm) / (2 * h) - d) < 1e-6 * max(1.0, abs(d))
    # weights are a normalised distance-softmax: a constant tensor reads back
    c = np.full(16, 7.0)
    v, d = oracle.relaxed_read(c, 5, 5.0, 1.0)
    assert abs(v - 7.0) < 1e-12 and abs(d) < 1e-12


def _cart(seed=3, mapper=synth.MAPPER_4K):
    return synth.generate_cart(seed, 0, mapper)


@pytest.mark.parametrize("tau", [1.0, 0.1, 0.01])
def test_theorem1_soft_forward_equals_hard(tau):
    rom = _cart()
    acts = synth.actions(5, 1, 6)[:, 0]
    hard = oracle.Oracle(rom, synth.MAPPER_4K)
    rams, scrs, _ = hard.rollout(acts, 1)
    soft = oracle.Oracle(rom, synth.MAPPER_4K)
    u = synth.action_inputs(acts).astype(np.float64)
    g, ram_out, scr_out = soft.soft_rollout(u, 1, tau)
    assert np.array_equal(ram_out, rams.astype(np.float64))
    assert np.array_equal(scr_out, scrs.astype(np.float64))


def _soft_case(tau, n_steps=3, frame_skip=1, mapper=synth.MAPPER_4K, seed=3):
    rom = _cart(seed, mapper)
    acts = synth.actions(seed, 1, n_steps)[:, 0]
    o = oracle.Oracle(rom, mapper)
    # start from a state a few frames in
    o.rollout(synth.actions(seed + 1, 1, 2)[:, 0], 1, screens=False)
    u = synth.action_inputs(acts).astype(np.float64)
    gr = synth.normal_f32(seed, (n_steps, 128), 1).astype(np.float64)
    gs = synth.normal_f32(seed, (n_steps, 210, 160), 2).astype(np.float64)
    g, _, _ = o.soft_rollout(u, frame_skip, tau, 6.0, gr, gs, outputs=False)
    return g


@pytest.mark.parametrize("tau", [1.0, 0.1])
def test_reverse_equals_tangent(tau):
    g = _soft_case(tau)
    g_rom, g_ram0, g_u = g.reverse()
    rng = np.random.default_rng(7)
    for _ in range(3):
        d_rom = rng.standard_normal(g.rom_size)
        d_ram0 = rng.standard_normal(128)
        d_u = rng.standard_normal((g.n_steps, 5))
        lhs = float(g_rom @ d_rom + g_ram0 @ d_ram0 + (g_u * d_u).sum())
        rhs = g.tangent(d_rom, d_ram0, d_u)
        assert abs(lhs - rhs) <= 1e-9 * max(1.0, abs(lhs)), (lhs, rhs)


@pytest.mark.parametrize("tau,mapper", [(1.0, synth.MAPPER_4K), (0.1, synth.MAPPER_4K),
                                        (0.1, synth.MAPPER_F8), (0.3, synth.MAPPER_2K)])
def test_reverse_equals_finite_differences(tau, mapper):
    g = _soft_case(tau, mapper=mapper)
    g_rom, g_ram0, g_u = g.reverse()
    h = 1e-4
    rng = np.random.default_rng(11)
    idx = np.argsort(-np.abs(g_rom))[:12].tolist() + rng.integers(0, g.rom_size, 4).tolist()
    for i in idx:
        d = np.zeros(g.rom_size)
        d[i] = h
        fd = (g.eval(d_rom=d) - g.eval(d_rom=-d)) / (2 * h)
        assert abs(fd - g_rom[i]) <= 1e-6 * max(1.0, abs(g_rom).max()), (i, fd, g_rom[i])
    for i in np.argsort(-np.abs(g_ram0))[:6]:
        d = np.zeros(128)
        d[i] = h
        fd = (g.eval(d_ram0=d) - g.eval(d_ram0=-d)) / (2 * h)
        assert abs(fd - g_ram0[i]) <= 1e-6 * max(1.0, abs(g_ram0).max())
    for t in range(g.n_steps):
        for k in range(5):
            d = np.zeros((g.n_steps, 5))
            d[t, k] = h
            fd = (g.eval(d_u=d) - g.eval(d_u=-d)) / (2 * h)
            assert abs(fd - g_u[t, k]) <= 1e-6 * max(1.0, abs(g_u).max())
    assert np.abs(g_rom).max() > 0 and np.abs(g_u).max() > 0


def test_colour_gradient_counts_owned_pixels():
    """LDA #k; STA COLUP0 with GRP0 = $FF at position 0 and no playfield:
    each frame has 8 x 210 P0-owned pixels, so d(sum pixels)/d(ROM[imm])
    is 1680 per frame whose COLUP0 came from that byte."""
    def build(a):
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", 0x01)
        a.op("LDA", "imm", 0xFF)
        a.op("STA", "zp", 0x1B)
        a.label("FRAME")
        a.op("LDA", "imm", 2)
        a.op("STA", "zp", 0x02)
        a.op("STA", "zp", 0x00)
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", 0x00)
        a.label("IMM")
        a.op("LDA", "imm", 0x57)
        a.op("STA", "zp", 0x06)
        a.op("LDX", "imm", 0)
        a.label("L")
        a.op("STA", "zp", 0x02)
        a.op("DEX")
        a.op("BNE", "rel", "L")
        a.op("JMP", "abs", "FRAME")
        imm_addr.append(a.labels["IMM"] + 1)
    imm_addr = []
    rom = rom4k(build)
    o = oracle.Oracle(rom, synth.MAPPER_4K)
    n = 4
    u = np.zeros((n, 5))
    gs = np.ones((n, 210, 160))
    for tau in (0.01, 1.0):
        o.reset()
        g, _, scr = o.soft_rollout(u, 1, tau, 6.0, None, gs)
        assert (scr[1:] == 0x56).sum() == 3 * 1680
        g_rom, _, _ = g.reverse()
        i = imm_addr[0] - 0xF000
        if tau == 0.01:
            assert g_rom[i] == pytest.approx(3 * 1680, rel=1e-12)
            g_rom[i] = 0
            assert np.abs(g_rom).max() < 1e-20
        else:
            # the relaxed read spreads the same total over its window (W = 12)
            lo, hi = i - 12, i + 12
            assert g_rom[lo:hi + 1].sum() == pytest.approx(3 * 1680, rel=1e-12)
            assert g_rom[i] > g_rom[i - 1] > g_rom[i - 2] > 0
            assert g_rom[i - 1] == pytest.approx(g_rom[i + 1], rel=1e-12)
            g_rom[lo:hi + 1] = 0
            assert np.abs(g_rom).max() < 1e-12


def test_superchip_ram_is_a_second_read_tensor():
    """LDA #k; STA $1005; LDA $1085; STA $80; LDA $1086; STA $81 on an F8SC
    cart, L = RAM[$80] + 2 RAM[$81]: the cartridge RAM is a 128-cell tensor
    of its own, so the reads of cells 5 and 6 are relaxed within it
    (weights e^{-|i - a| / tau} over |i - a| <= W, renormalised), the write
    of cell 5 is one-hot (the imm byte's read takes cell 5's weight) and the
    initial cartridge RAM takes the other cells' weights."""
    tau = 0.5
    W = max(1, math.ceil(12 * tau))
    def weights(a):
        w = np.array([math.exp(-abs(i - a) / tau) if abs(i - a) <= W else 0.0 for i in range(128)])
        return w / w.sum()
    b1 = synth.Asm(0xF000, 4096)
    b1.at(0x100)
    b1.op("LDA", "imm", 0x3C)
    b1.op("STA", "abs", 0x1005)
    b1.op("LDA", "abs", 0x1085)
    b1.op("STA", "zp", 0x80)
    b1.op("LDA", "abs", 0x1086)
    b1.op("STA", "zp", 0x81)
    b1.label("HALT")
    b1.op("JMP", "abs", "HALT")
    b1.at(4096 - 6)
    b1.word(0xF100), b1.word(0xF100), b1.word(0xF100)
    b0 = synth.Asm(0xF000, 4096)
    b0.at(4096 - 6)
    b0.word(0xF100), b0.word(0xF100), b0.word(0xF100)
    rom = bytes(b0.resolve()) + bytes(b1.resolve())
    o = oracle.Oracle(rom, synth.MAPPER_F8SC)
    gr = np.zeros((1, 128))
    gr[0, 0], gr[0, 1] = 1.0, 2.0
    g, ram_out, _ = o.soft_rollout(np.zeros((1, 5)), 1, tau, 6.0, gr, None)
    assert ram_out[0, 0] == 0x3C and ram_out[0, 1] == 0
    g_rom, g_ram0, g_u, g_cram0 = g.reverse(cart_ram=True)
    w = weights(5) + 2 * weights(6)
    # the imm byte's own read is relaxed over its 4 KB bank (an interior
    # index: the same window shape, centred on offset $101)
    imm = 4096 + 0x101
    w_rom = np.zeros(g.rom_size)
    w_rom[imm - W:imm + W + 1] = [math.exp(-abs(d) / tau) for d in range(-W, W + 1)]
    w_rom /= w_rom.sum()
    assert np.allclose(g_rom, w[5] * w_rom, rtol=0, atol=1e-12)
    want = w.copy()
    want[5] = 0.0
    assert np.allclose(g_cram0, want, rtol=0, atol=1e-12)
    assert not g_ram0.any() and not g_u.any()


def test_superchip_reverse_equals_tangent_and_finite_differences():
    """The transpose identity and central differences on a generated F6SC
    cart, including the initial cartridge RAM's leaves."""
    g = _soft_case(0.3, mapper=synth.MAPPER_F6SC)
    g_rom, g_ram0, g_u, g_cram0 = g.reverse(cart_ram=True)
    assert np.abs(g_cram0).max() > 0
    rng = np.random.default_rng(9)
    d_rom = rng.standard_normal(g.rom_size)
    d_ram0 = rng.standard_normal(256)
    d_u = rng.standard_normal((g.n_steps, 5))
    lhs = float(g_rom @ d_rom + np.concatenate([g_ram0, g_cram0]) @ d_ram0 + (g_u * d_u).sum())
    rhs = g.tangent(d_rom, d_ram0, d_u)
    assert abs(lhs - rhs) <= 1e-9 * max(1.0, abs(lhs)), (lhs, rhs)
    h = 1e-4
    for i in np.argsort(-np.abs(g_cram0))[:6]:
        d = np.zeros(256)
        d[128 + i] = h
        fd = (g.eval(d_ram0=d) - g.eval(d_ram0=-d)) / (2 * h)
        assert abs(fd - g_cram0[i]) <= 1e-6 * max(1.0, abs(g_cram0).max())


def test_e0_read_is_relaxed_within_its_slice():
    """LDA $1002 with slice 3 in segment 0, L = RAM[$80]: the read's tensor
    is the 1 KB slice (the window is clipped at the slice's first byte and
    renormalised there; nothing reaches slice 2's last bytes, which precede
    it in the image)."""
    tau = 0.5
    W = max(1, math.ceil(12 * tau))
    def program(a):
        a.at(0x100)
        a.op("LDA", "abs", 0x1FE3)
        a.op("LDA", "abs", 0x1002)
        a.op("STA", "zp", 0x80)
        a.label("HALT")
        a.op("JMP", "abs", "HALT")
    from tests.test_oracle_machine import _e0_image
    rom = _e0_image(program)
    o = oracle.Oracle(rom, synth.MAPPER_E0)
    gr = np.zeros((1, 128))
    gr[0, 0] = 1.0
    g, ram_out, _ = o.soft_rollout(np.zeros((1, 5)), 1, tau, 6.0, gr, None)
    assert ram_out[0, 0] == 0xA3
    g_rom, _, _ = g.reverse()
    w = np.array([math.exp(-abs(i - 2) / tau) for i in range(0, 2 + W + 1)])
    want = np.zeros(8192)
    want[3 * 1024:3 * 1024 + len(w)] = w / w.sum()
    assert np.allclose(g_rom, want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("score", [False, True])
def test_colup1_owns_player1_and_score_pixels(score):
    """LDA #k; STA COLUP1 with GRP1 = $FF, NUSIZ1 = 7 (quad width: 32
    columns) and no playfield: 32 x 210 COLUP1-owned pixels per frame; in
    score mode with PF2 = $FF (columns 48..79, repeated at 128..159) the
    right half's 32 columns are COLUP1's too, and the left half's COLUP0's."""
    def build(a):
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", 0x01)
        a.op("LDA", "imm", 0xFF)
        a.op("STA", "zp", 0x1C)                 # GRP1
        a.op("LDA", "imm", 7)
        a.op("STA", "zp", 0x05)                 # NUSIZ1: quad width
        if score:
            a.op("LDA", "imm", 0xFF)
            a.op("STA", "zp", 0x0F)             # PF2
            a.op("LDA", "imm", 2)
            a.op("STA", "zp", 0x0A)             # CTRLPF: score mode
        a.label("FRAME")
        a.op("LDA", "imm", 2)
        a.op("STA", "zp", 0x02)
        a.op("STA", "zp", 0x00)
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", 0x00)
        a.op("STA", "zp", 0x02)
        a.op("STA", "zp", 0x11)                 # RESP1 in HBLANK: position 3
        a.label("IMM")
        a.op("LDA", "imm", 0x57)
        a.op("STA", "zp", 0x07)                 # COLUP1
        a.op("LDX", "imm", 0)
        a.label("L")
        a.op("STA", "zp", 0x02)
        a.op("DEX")
        a.op("BNE", "rel", "L")
        a.op("JMP", "abs", "FRAME")
        imm.append(a.labels["IMM"] + 1 - 0xF000)
    imm = []
    rom = rom4k(build)
    o = oracle.Oracle(rom, synth.MAPPER_4K, full_tia=True)
    n = 4
    g, _, scr = o.soft_rollout(np.zeros((n, 5)), 1, 0.01, 6.0, None, np.ones((n, 210, 160)))
    per_frame = 210 * (32 + (32 if score else 0))
    assert (scr[1:] == 0x56).sum() == 3 * per_frame
    g_rom, _, _ = g.reverse()
    assert g_rom[imm[0]] == pytest.approx(3 * per_frame, rel=1e-12)
