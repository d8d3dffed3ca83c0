"""Pins of the oracle's graphics-bit surrogate (Section 3.1: with the
stored switch, sprite colours and graphics bits are differentiable).

The expected gradients are computed here from the definition of the
relaxation, independently of the oracle: each object's coverage of a pixel
is its graphics bit b, relaxed to a real number, and the colours blend in
priority order (the top object's colour times its coverage plus the rest
times one minus it), which equals the hard priority logic at binary bits;
every bit's derivative with respect to its register byte is 1 (the
straight-through rule for the shift and mask that extract it).  Central
finite differences of that blend in a register's bits (all of them moved
together) give d pixel / d byte; the oracle gets the same numbers from its
deviation graph and a with-minus-without colour rule.
"""
import numpy as np
import pytest

from paper_2606_22447_b300 import synth
from tests.microrom import GRAPHICS_COLOURS, GRAPHICS_PF, graphics_rom

oracle = pytest.importorskip("oracle")

# d SWCHA / d u for (R, L, D, U, FIRE): the joystick bits are active low
D_SWCHA = np.array([-128.0, -64.0, -32.0, -16.0, 0.0])


def _pf_index(x, ctrlpf):
    i = x // 4 if x < 80 else (x - 80) // 4
    return 19 - i if (x >= 80 and ctrlpf & 1) else i


def _pf_bits(pf):
    """The 20 playfield bits (PF0 bits 4-7, PF1 bits 7..0, PF2 bits 0..7)
    with the register each comes from."""
    bits, reg = [], []
    for k in range(4):
        bits.append((pf[0] >> (4 + k)) & 1), reg.append(0)
    for k in range(8):
        bits.append((pf[1] >> (7 - k)) & 1), reg.append(1)
    for k in range(8):
        bits.append((pf[2] >> k) & 1), reg.append(2)
    return np.array(bits, float), np.array(reg)


def _relaxed_row(pos, grp0, d_grp0, d_pf, ctrlpf):
    """Colours of one line with every GRP0 bit moved by d_grp0 and every bit
    of playfield register k by d_pf[k] (relaxed coverages, priority blend)."""
    c = {k: float(v & 0xFE) for k, v in GRAPHICS_COLOURS.items()}
    pfb, pfreg = _pf_bits(GRAPHICS_PF)
    row = np.zeros(160)
    for x in range(160):
        i = _pf_index(x, ctrlpf)
        b_pf = pfb[i] + d_pf[pfreg[i]]
        d = (x - pos) % 160
        b_p0 = (((grp0 >> (7 - d)) & 1) + d_grp0) if d < 8 else 0.0
        if ctrlpf & 4:   # the playfield above the player
            row[x] = b_pf * c["pf"] + (1 - b_pf) * (b_p0 * c["p0"] + (1 - b_p0) * c["bk"])
        else:
            row[x] = b_p0 * c["p0"] + (1 - b_p0) * (b_pf * c["pf"] + (1 - b_pf) * c["bk"])
    return row


def _hard_pos(row, grp0, ctrlpf):
    hits = [p for p in range(160) if np.array_equal(_relaxed_row(p, grp0, 0, (0, 0, 0), ctrlpf), row)]
    assert len(hits) == 1, hits
    return hits[0]


def _swcha(u):
    return int(0xFF - (u[:4] * np.array([128, 64, 32, 16])).sum())


@pytest.mark.parametrize("ctrlpf", [0, 1, 4])
def test_graphics_bit_gradients_follow_the_relaxed_blend(ctrlpf):
    rom, pf_offs = graphics_rom(ctrlpf)
    n = 4
    r = np.random.default_rng(40 + ctrlpf)
    u = (r.random((n, 5)) < 0.5).astype(float)
    gs = r.standard_normal((n, 210, 160))
    o = oracle.Oracle(rom, synth.MAPPER_4K)
    o.set_graphics(True)
    g, _, scr = o.soft_rollout(u, 1, 0.01, 6.0, None, gs)
    g_rom, _, g_u = g.reverse()
    h = 0.25
    want_u = np.zeros((n, 5))
    want_pf = np.zeros(3)
    for t in range(1, n):   # step 0 runs from power-on: its frame has no GRP0 yet
        grp0 = _swcha(u[t])
        rows = scr[t]
        assert np.all(rows == rows[100][None, :]), "every visible line is the same"
        pos = _hard_pos(rows[100], grp0, ctrlpf)
        wsum = gs[t].sum(0)   # every row is the same line
        d = (_relaxed_row(pos, grp0, h, (0, 0, 0), ctrlpf) - _relaxed_row(pos, grp0, -h, (0, 0, 0), ctrlpf)) / (2 * h)
        want_u[t] = (wsum * d).sum() * D_SWCHA
        for k in range(3):
            dp = [0, 0, 0]
            dp[k] = h
            dm = [0, 0, 0]
            dm[k] = -h
            dk = (_relaxed_row(pos, grp0, 0, dp, ctrlpf) - _relaxed_row(pos, grp0, 0, dm, ctrlpf)) / (2 * h)
            want_pf[k] += (wsum * dk).sum()
    assert np.abs(want_u[1:, :4]).min() > 1.0 and np.abs(want_pf).min() > 1.0
    np.testing.assert_allclose(g_u[1:], want_u[1:], rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(g_rom[pf_offs], want_pf, rtol=1e-12, atol=1e-9)


def test_graphics_off_leaves_the_other_gradients_alone():
    """With the surrogate off the joystick reaches nothing here (SWCHA only
    feeds GRP0) and the PF immediates get nothing; the colour registers'
    gradients are the same either way."""
    rom, pf_offs = graphics_rom(0)
    n = 3
    r = np.random.default_rng(47)
    u = (r.random((n, 5)) < 0.5).astype(float)
    gs = r.standard_normal((n, 210, 160))
    out = []
    for on in (False, True):
        o = oracle.Oracle(rom, synth.MAPPER_4K)
        o.set_graphics(on)
        g, _, _ = o.soft_rollout(u, 1, 0.01, 6.0, None, gs)
        out.append(g.reverse())
    (rom0, _, u0), (rom1, _, u1) = out
    assert np.abs(u0).max() == 0 and np.abs(rom0[pf_offs]).max() == 0
    assert np.abs(u1).max() > 0
    others = np.ones(len(rom0), bool)
    others[pf_offs] = False
    np.testing.assert_allclose(rom1[others], rom0[others], rtol=1e-12, atol=1e-9)


def _ft_row(st, grp0, grp1_shown, ctrlpf, d):
    """One line of the whole-TIA graphics cart with the relaxed coverages of
    each object moved by d[name] (all bits of a register together): colours
    blend in priority order, objects of one colour group combining as
    1 - (1 - b)(1 - b')."""
    from tests.microrom import GRAPHICS_FT_COLOURS as COL, GRAPHICS_FT_PF as PF
    c = {k: float(v & 0xFE) for k, v in COL.items()}
    p0pos, p1pos, m0pos, blpos = int(st[24]), int(st[50]), int(st[51]), int(st[53])
    pfb, pfreg = _pf_bits(PF)
    row = np.zeros(160)
    for x in range(160):
        i = _pf_index(x, ctrlpf)
        b_pf = pfb[i] + d["pf%d" % pfreg[i]]
        k0, k1 = (x - p0pos) % 160, (x - p1pos) % 160
        b_p0 = (((grp0 >> (7 - k0)) & 1) + d["grp0"]) if k0 < 8 else 0.0
        b_p1 = (((grp1_shown >> (7 - k1)) & 1) + d["grp1"]) if k1 < 8 else 0.0
        b_m0 = (1.0 + d["enam0"]) if (x - m0pos) % 160 < 2 else 0.0
        b_bl = (1.0 + d["enabl"]) if (x - blpos) % 160 < 4 else 0.0
        g_c0 = 1 - (1 - b_p0) * (1 - b_m0)
        g_c1 = b_p1
        g_pf = 1 - (1 - b_pf) * (1 - b_bl)
        if ctrlpf & 4:
            row[x] = g_pf * c["pf"] + (1 - g_pf) * (g_c0 * c["p0"] + (1 - g_c0) * (g_c1 * c["p1"] + (1 - g_c1) * c["bk"]))
        else:
            row[x] = g_c0 * c["p0"] + (1 - g_c0) * (g_c1 * c["p1"] + (1 - g_c1) * (g_pf * c["pf"] + (1 - g_pf) * c["bk"]))
    return row


@pytest.mark.parametrize("ctrlpf,vdel", [(0, False), (4, False), (0, True)])
def test_whole_tia_graphics_bits_follow_the_relaxed_blend(ctrlpf, vdel):
    """The whole TIA: player 1's GRP1 (from the joystick, or its delayed copy
    with VDELP1), GRP0, ENAM0, ENABL and PF0-2, central differences of the
    priority blend against the oracle's input and ROM gradients; with VDELP1
    the GRP1 byte stored after the copy is not shown and gets nothing."""
    from tests.microrom import graphics_full_tia_rom
    rom, offs = graphics_full_tia_rom(ctrlpf, vdel)
    n = 4
    r = np.random.default_rng(60 + ctrlpf + vdel)
    u = (r.random((n, 5)) < 0.5).astype(float)
    gs = r.standard_normal((n, 210, 160))
    o = oracle.Oracle(rom, synth.MAPPER_4K, full_tia=True)
    o.set_graphics(True)
    g, _, scr = o.soft_rollout(u, 1, 0.01, 6.0, None, gs)
    g_rom, _, g_u = g.reverse()
    h = 0.25
    names = ["grp0", "grp1", "enam0", "enabl", "pf0", "pf1", "pf2"]
    want = {k: 0.0 for k in names}
    want_u = np.zeros((n, 5))
    # positions and screens come from a plain run of the same inputs
    ref = oracle.Oracle(rom, synth.MAPPER_4K, full_tia=True)
    for t in range(n):
        ref.set_graphics(False)
        _, _, s_ref = ref.soft_rollout(u[t:t + 1], 1, 0.01, 6.0, None, None)
        st = ref.state()
        if t == 0:
            continue   # step 0 runs from power-on: its frame has no graphics stores yet
        grp1_shown = _swcha(u[t])
        assert np.array_equal(s_ref[0], scr[t])
        zero = {k: 0.0 for k in names}
        assert np.array_equal(_ft_row(st, 0xA5, grp1_shown, ctrlpf, zero), scr[t][100].astype(float))
        wsum = gs[t].sum(0)
        for k in names:
            dp, dm = dict(zero), dict(zero)
            dp[k], dm[k] = h, -h
            dk = (_ft_row(st, 0xA5, grp1_shown, ctrlpf, dp) - _ft_row(st, 0xA5, grp1_shown, ctrlpf, dm)) / (2 * h)
            v = float((wsum * dk).sum())
            if k == "grp1":
                want_u[t] = v * D_SWCHA
            else:
                want[k] += v
    assert min(abs(want[k]) for k in ("grp0", "enam0", "enabl")) > 1.0 and np.abs(want_u[1:, :4]).min() > 1.0, (want, want_u)
    np.testing.assert_allclose(g_u[1:], want_u[1:], rtol=1e-12, atol=1e-9)
    for k in ("grp0", "enam0", "enabl", "pf0", "pf1", "pf2"):
        np.testing.assert_allclose(g_rom[offs[k]], want[k], rtol=1e-12, atol=1e-9, err_msg=k)
    if vdel:
        assert abs(g_rom[offs["grp1"]]) < 1e-12   # stored after the copy: not shown
