"""Pins of the oracle's differentiable position sampler (Section 3, the
sub-pixel kernel over sprite position).

The expected gradients here are computed from the definition of the relaxed
sprite coverage, cov(x) = sum_k b_k tri(x - pos - k) with tri(u) = max(0,
1 - |u|) over the 160 columns of a line, by finite differences of the
rendered colours in pos, and from the chain HMP0 -> HMOVE -> pos: a player
moved by minus the high nibble of HMP0 moves by minus a sixteenth of a
deviation of HMP0.  The oracle computes the same gradient through its
deviation graph and a closed-form slope; the two share nothing but the cart.
"""
import numpy as np
import pytest

from paper_2606_22447_b300 import synth
from tests.microrom import SAMPLER_COLOURS, SAMPLER_GRP0, SAMPLER_PF2, sampler_rom

oracle = pytest.importorskip("oracle")

# d SWCHA / d u for (R, L, D, U, FIRE): the joystick bits are active low
D_SWCHA = np.array([-128.0, -64.0, -32.0, -16.0, 0.0])
# d pos / d u: HMOVE moves the player by minus HMP0's high nibble
D_POS = -D_SWCHA / 16.0


def _pf_cols():
    """Columns covered by the playfield of the sampler cart (PF2 only, the
    right half repeated)."""
    pf = np.zeros(160, bool)
    for x in range(160):
        i = (x if x < 80 else x - 80) // 4
        if 12 <= i < 20:
            pf[x] = (SAMPLER_PF2 >> (i - 12)) & 1
    return pf


def _relaxed_row(pos, ctrlpf):
    """Colours of one line with the player at real position pos, from the
    relaxed coverage (pixel = under + (C_P0 - under) cov, or the playfield
    colour where the playfield has priority and covers the pixel)."""
    pf = _pf_cols()
    c = {k: v & 0xFE for k, v in SAMPLER_COLOURS.items()}
    under = np.where(pf, c["pf"], c["bk"]).astype(float)
    x = np.arange(160, dtype=float)
    cov = np.zeros(160)
    for k in range(8):
        if (SAMPLER_GRP0 >> (7 - k)) & 1:
            u = (x - pos - k + 80.0) % 160.0 - 80.0     # wrapped to [-80, 80)
            cov += np.maximum(0.0, 1.0 - np.abs(u))
    row = under + (c["p0"] - under) * cov
    if ctrlpf & 4:
        row = np.where(pf, c["pf"], row)
    return row


def _hard_pos(screen_row, ctrlpf):
    """The integer position whose hard rendering is this screen row (unique)."""
    hits = [p for p in range(160) if np.array_equal(_relaxed_row(float(p), ctrlpf), screen_row)]
    assert len(hits) == 1, hits
    return hits[0]


def _dL_dpos(screen, w, ctrlpf, h=0.25):
    """d (sum w * pixels) / d pos of one frame, by central differences of the
    relaxed rendering (exact for the piecewise-linear kernel and h < 1)."""
    rows = screen.shape[0]
    if not np.any(screen == (SAMPLER_COLOURS["p0"] & 0xFE)):
        return 0.0
    p = _hard_pos(screen[rows // 2], ctrlpf)
    for r in (0, rows - 1):
        assert np.array_equal(screen[r], screen[rows // 2])
    d = (_relaxed_row(p + h, ctrlpf) - _relaxed_row(p - h, ctrlpf)) / (2 * h)
    return float((w * d[None, :]).sum())


def _run(rom, u, gs, sampler, tau=0.1):
    o = oracle.Oracle(rom, synth.MAPPER_4K)
    o.set_sampler(sampler)
    g, ram, scr = o.soft_rollout(u, 1, tau, 6.0, None, gs)
    g_rom, g_ram0, g_u = g.reverse()
    return g, g_rom, g_u, ram, scr


def _inputs(seed, n):
    r = np.random.default_rng(seed)
    u = (r.random((n, 5)) < 0.5).astype(float)
    gs = r.standard_normal((n, 210, 160))
    return u, gs


@pytest.mark.parametrize("ctrlpf", [0, 4])
def test_sampler_gradient_per_frame_position(ctrlpf):
    """RESP0 every frame: step t's input moves only step t's sprite, so
    d L / d u_t = (d L_t / d pos) (d pos / d u)."""
    n = 4
    u, gs = _inputs(31 + ctrlpf, n)
    _, g_rom, g_u, _, scr = _run(sampler_rom(True, ctrlpf), u, gs, True)
    want = np.array([_dL_dpos(scr[t], gs[t], ctrlpf) * D_POS for t in range(n)])
    assert np.abs(want[1:]).max() > 100, "the sprite edges must carry gradient"
    np.testing.assert_allclose(g_u, want, rtol=1e-12, atol=1e-9)


def test_sampler_gradient_accumulates_motions():
    """RESP0 once: every HMOVE adds its frame's motion, so the input of step
    s moves the sprite of every later frame: d L / d u_s =
    sum_{t >= s} (d L_t / d pos) (d pos / d u).  Step 0 runs from power-on to
    the first VSYNC and strobes no HMOVE: its input moves nothing."""
    n = 4
    u, gs = _inputs(37, n)
    _, _, g_u, _, scr = _run(sampler_rom(False, 0), u, gs, True)
    per_frame = np.array([_dL_dpos(scr[t], gs[t], 0) for t in range(n)])
    want = np.array([per_frame[s:].sum() * D_POS if s > 0 else 0 * D_POS for s in range(n)])
    assert np.abs(want).max() > 100
    np.testing.assert_allclose(g_u, want, rtol=1e-12, atol=1e-9)


def test_sampler_positions_follow_hmove():
    """The hard rendering the pins rely on: the sprite moves by minus the
    signed high nibble of SWCHA each frame (and only through HMOVE)."""
    n = 5
    u, gs = _inputs(41, n)
    _, _, _, _, scr = _run(sampler_rom(False, 0), u, gs, True)
    pos = [_hard_pos(scr[t][100], 0) for t in range(1, n)]
    for t in range(2, n):
        swcha = 0xFF - int(u[t] @ -D_SWCHA)
        m = (swcha - 256 if swcha >= 128 else swcha) >> 4
        assert pos[t - 1] == (pos[t - 2] - m) % 160


@pytest.mark.parametrize("resp", [True, False])
def test_sampler_off_leaves_inputs_without_gradient(resp):
    """Without the sampler the joystick reaches only HMP0, whose hard effect
    (an integer move) has no deviation: the inputs get zero gradient, and the
    forward outputs do not depend on the switch."""
    u, gs = _inputs(43, 3)
    _, g_rom0, g_u0, ram0, scr0 = _run(sampler_rom(resp, 0), u, gs, False)
    _, g_rom1, g_u1, ram1, scr1 = _run(sampler_rom(resp, 0), u, gs, True)
    assert np.all(g_u0 == 0)
    assert np.abs(g_u1).max() > 0
    assert np.array_equal(ram0, ram1) and np.array_equal(scr0, scr1)
    np.testing.assert_array_equal(g_rom0, g_rom1)   # ROM bytes do not reach the position


@pytest.mark.parametrize("tau", [0.1, 1.0])
def test_sampler_reverse_equals_tangent_and_differences(tau):
    """On synthetic carts (RESP0, HMP0 and HMOVE among their writes) the
    graph with the sampler keeps reverse == tangent == finite differences."""
    rom = synth.config_carts(5, [synth.MAPPER_4K])[0]
    n = 3
    r = np.random.default_rng(47)
    u = (r.random((n, 5)) < 0.5).astype(float)
    gs = r.standard_normal((n, 210, 160))
    grm = r.standard_normal((n, 128))
    o = oracle.Oracle(rom, synth.MAPPER_4K)
    o.set_sampler(True)
    g, _, _ = o.soft_rollout(u, 1, tau, 6.0, grm, gs)
    g_rom, g_ram0, g_u = g.reverse()
    d_rom = r.standard_normal(len(rom))
    d_ram = r.standard_normal(128)
    d_u = r.standard_normal((n, 5))
    t = g.tangent(d_rom, d_ram, d_u)
    lin = (g_rom * d_rom).sum() + (g_ram0 * d_ram).sum() + (g_u * d_u).sum()
    assert t == pytest.approx(lin, rel=1e-10, abs=1e-8)
    h = 1e-3
    fd = (g.eval(d_rom * h, d_ram * h, d_u * h) - g.eval(-d_rom * h, -d_ram * h, -d_u * h)) / (2 * h)
    assert fd == pytest.approx(lin, rel=1e-8, abs=1e-6)
    o.reset()
    o.set_sampler(False)
    g_off, _, _ = o.soft_rollout(u, 1, tau, 6.0, grm, gs)
    assert np.abs(g_off.reverse()[0] - g_rom).max() > 1.0, "the sampler must reach this cart's ROM"
