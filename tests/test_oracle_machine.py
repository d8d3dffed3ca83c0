"""Pins of the oracle's bus, RIOT and TIA against fixed facts:

* colour-clock invariants: 3 colour clocks per CPU cycle, 228 per scanline,
  WSYNC resumes at line clock 0, a 262-WSYNC frame is 262 lines and 19,912
  cycles (NTSC);
* the RIOT timer against its closed form (reading A8);
* F8 bank switching happens only on the two hotspot addresses;
* hand-derived pixels for playfield, player and priority cases (A3-A6).
"""
import numpy as np
import pytest

import oracle
from paper_2606_22447_b300 import synth
from tests.microrom import rom4k

WSYNC, VSYNC, VBLANK = 0x02, 0x00, 0x01


def _frame_rom():
    def build(a):
        a.op("LDA", "imm", 2)
        a.op("LDY", "imm", 0)
        a.op("STA", "zp", WSYNC)
        a.label("FRAME")
        a.op("STA", "zp", VSYNC)
        a.op("STY", "zp", VSYNC)
        a.op("LDX", "imm", 5)
        a.label("L1")
        a.op("STA", "zp", WSYNC)
        a.op("DEX")
        a.op("BNE", "rel", "L1")
        a.label("L2")
        a.op("STA", "zp", WSYNC)
        a.op("DEX")
        a.op("BNE", "rel", "L2")
        a.op("STA", "zp", WSYNC)
        a.op("JMP", "abs", "FRAME")
    return rom4k(build)


def test_ntsc_frame_262_lines_19912_cycles():
    o = oracle.Oracle(_frame_rom(), synth.MAPPER_4K)
    o.step(0, 1)
    cyc = []
    for _ in range(4):
        o.step(0, 1)
        s = o.state()
        cyc.append(int(s[6]) | (int(s[7]) << 32))
    assert np.all(np.diff(cyc) == 19912)
    # at each frame end (just after the VSYNC write) the beam is at line 0
    assert o.state()[26] == 0


def test_colour_clocks_per_cycle_and_wsync():
    o = oracle.Oracle(_frame_rom(), synth.MAPPER_4K)
    tr = o.trace(0, 3000).astype(np.int64)
    pc, op, cyc, line, hclk = tr[:, 0], tr[:, 1], tr[:, 7], tr[:, 8], tr[:, 9]
    for i in range(1, len(tr)):
        if line[i] >= line[i - 1]:          # same frame
            assert (line[i] * 228 + hclk[i]) - (line[i - 1] * 228 + hclk[i - 1]) == 3 * (cyc[i] - cyc[i - 1])
        assert 0 <= hclk[i] < 228 and hclk[i] % 3 == 0
    # every instruction after STA WSYNC starts at line clock 0, and the
    # absolute beam position is 3 x cycles modulo 228
    after = np.where((op[:-1] == 0x85) & (np.arange(len(tr) - 1) >= 0))[0]
    wsync_next = [i + 1 for i in after if o.rom[(pc[i] - 0xF000) + 1] == WSYNC]
    assert len(wsync_next) > 100
    assert np.all(hclk[wsync_next] == 0)
    assert np.all((3 * cyc) % 228 == hclk)


# ---------------------------------------------------------------------------
# RIOT timer
# ---------------------------------------------------------------------------

def _timer_closed_form(V, I, k):
    """INTIM and TIMINT bit 7 at k >= 1 cycles after writing V to an
    interval-I register."""
    if k <= V * I:
        return V - (-(-k // I)), 0
    ku = V * I + 1
    return (0xFF - (k - ku)) & 0xFF, 0x80


@pytest.mark.parametrize("V,reg,I", [(0, 0x294, 1), (1, 0x294, 1), (5, 0x295, 8), (43, 0x296, 64),
                                     (2, 0x297, 1024), (255, 0x294, 1), (7, 0x296, 64), (1, 0x297, 1024)])
def test_timer_closed_form(V, reg, I):
    def build(a):
        a.op("LDA", "imm", V)
        a.op("STA", "abs", reg)       # write at cycle 4 of this instruction
        a.label("LOOP")
        a.op("LDA", "abs", 0x284)     # INTIM read at cycle 4
        a.op("LDX", "abs", 0x285)     # TIMINT read at cycle 4
        a.op("NOP")
        a.op("JMP", "abs", "LOOP")
    o = oracle.Oracle(rom4k(build), synth.MAPPER_4K)
    n = min(3 * (V * I + 2000) // 13 + 50, 60000)
    tr = o.trace(0, n).astype(np.int64)
    pc, A, X, cyc = tr[:, 0], tr[:, 2], tr[:, 3], tr[:, 7]
    tw = cyc[1] + 4
    checked = 0
    for i in range(2, len(tr) - 1):
        if pc[i] == 0xF005:                    # LDA INTIM
            k = cyc[i] + 4 - tw
            assert A[i + 1] == _timer_closed_form(V, I, k)[0], (k, A[i + 1])
            checked += 1
        elif pc[i] == 0xF008:                  # LDX TIMINT
            k = cyc[i] + 4 - tw
            assert X[i + 1] == _timer_closed_form(V, I, k)[1], k
    assert checked > 100


def test_timer_power_on_state():
    """Power-on behaves as a write of 0 to T1024T at cycle 0."""
    def build(a):
        a.label("LOOP")
        a.op("LDA", "abs", 0x284)
        a.op("JMP", "abs", "LOOP")
    o = oracle.Oracle(rom4k(build), synth.MAPPER_4K)
    tr = o.trace(0, 200).astype(np.int64)
    for i in range(0, len(tr) - 1, 2):
        k = tr[i, 7] + 4
        assert tr[i + 1, 2] == _timer_closed_form(0, 1024, k)[0]


# ---------------------------------------------------------------------------
# F8 bank switching
# ---------------------------------------------------------------------------

def test_f8_switches_only_on_hotspots():
    """Bank 1 runs reads of addresses next to the hotspots, then LDA $1FF8
    (-> bank 0); bank 0 continues at the same offset and writes $1FF9."""
    b1 = synth.Asm(0xF000, 4096)
    b1.op("LDA", "abs", 0x1FF7)
    b1.op("LDA", "abs", 0x1FFA)
    b1.op("STA", "abs", 0x1FFB)
    b1.op("LDA", "abs", 0x0FF8)      # not a cartridge address (A12 = 0)
    b1.op("LDA", "abs", 0x1FF8)      # -> bank 0
    b1.at(4096 - 6)
    b1.word(0xF000), b1.word(0xF000), b1.word(0xF000)
    b0 = synth.Asm(0xF000, 4096)
    b0.at(15)
    b0.op("STA", "abs", 0xFFF9)      # mirror of $1FF9 -> bank 1
    b0.at(4096 - 6)
    b0.word(0xF000), b0.word(0xF000), b0.word(0xF000)
    rom = bytes(b0.resolve()) + bytes(b1.resolve())
    o = oracle.Oracle(rom, synth.MAPPER_F8)
    assert o.bank() == 1
    for _ in range(4):
        o.exec_one()
        assert o.bank() == 1
    o.exec_one()
    assert o.bank() == 0
    assert o.state()[5] == 0xF00F and o.peek(0xF00F) == 0x8D
    o.exec_one()
    assert o.bank() == 1


@pytest.mark.parametrize("mapper", [synth.MAPPER_F6, synth.MAPPER_F4])
def test_f6_f4_hotspots_select_each_bank(mapper):
    """Power-on in the last bank; a read or write of hotspot j selects bank
    j (reads in even banks, writes in odd ones), the neighbours of the
    hotspot range and the range's image below A12 select nothing.  Bank j
    holds at offset 3 j the access to hotspot j + 1, so the chain visits
    every bank in order and wraps back to the last."""
    nb, hot = synth.MAPPER_BANKS[mapper], synth.MAPPER_HOTSPOT[mapper]
    banks = []
    for j in range(nb):
        a = synth.Asm(0xF000, 4096)
        if j == nb - 1:
            a.op("LDA", "abs", hot - 1)            # below the range
            a.op("LDA", "abs", hot + nb)           # above it
            a.op("LDA", "abs", hot - 0x1000)       # A12 = 0: not the cartridge
            a.op("LDA", "abs", hot)                # -> bank 0 at offset 12
        else:
            a.at(12 + 3 * j)
            target = hot + j + 1
            if j % 2:
                a.op("STA", "abs", target)
            else:
                a.op("LDA", "abs", target)
        a.at(4096 - 6)
        a.word(0xF000), a.word(0xF000), a.word(0xF000)
        banks.append(bytes(a.resolve()))
    o = oracle.Oracle(b"".join(banks), mapper)
    assert o.bank() == nb - 1
    for _ in range(3):
        o.exec_one()
        assert o.bank() == nb - 1
    for j in range(nb):
        o.exec_one()
        assert o.bank() == j, j
        assert o.state()[5] == 0xF000 + 12 + 3 * j


def test_f6_f4_carts_visit_their_banks():
    """The generated F6 / F4 carts run frames of a few thousand instructions
    (no jam, no watchdog) and enter several kernel banks under random
    joystick input."""
    for mapper in (synth.MAPPER_F6, synth.MAPPER_F4):
        rom = synth.config_carts(17, [mapper])[0]
        assert len(rom) == synth.MAPPER_SIZE[mapper]
        o = oracle.Oracle(rom, mapper)
        seen = set()
        for a in synth.actions(18, 1, 40)[:, 0]:
            for _ in range(600):
                o.trace(int(a), 1)
                seen.add(int(o.state()[8]))
        c = o.counters()
        assert c["watchdog"] == 0 and o.state()[28] == 0
        assert 1500 < c["instructions"] / c["frames"] < 4000
        assert len(seen) >= 3 and synth.MAPPER_BANKS[mapper] - 1 in seen


# ---------------------------------------------------------------------------
# pixels
# ---------------------------------------------------------------------------

def _screen_of(build_line, ystart=0, frames=2):
    """Run a kernel where every scanline executes `build_line` after WSYNC;
    return the last frame."""
    def build(a):
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", VBLANK)
        a.label("FRAME")
        a.op("LDA", "imm", 2)
        a.op("STA", "zp", WSYNC)
        a.op("STA", "zp", VSYNC)
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", VSYNC)
        a.op("LDX", "imm", 230)
        a.label("LINE")
        a.op("STA", "zp", WSYNC)
        build_line(a)
        a.op("DEX")
        a.op("BNE", "rel", "LINE")
        a.op("JMP", "abs", "FRAME")
    o = oracle.Oracle(rom4k(build), synth.MAPPER_4K, ystart=ystart)
    for _ in range(frames):
        _, scr, st = o.step(0, 1)
    assert st == 0
    return scr


def test_playfield_bits_and_reflection():
    def line(a):
        a.op("LDA", "imm", 0x44)
        a.op("STA", "zp", 0x08)       # COLUPF
        a.op("LDA", "imm", 0x12)
        a.op("STA", "zp", 0x09)       # COLUBK
        a.op("LDA", "imm", 0x10)
        a.op("STA", "zp", 0x0D)       # PF0 bit 4 -> playfield bit 0
        a.op("LDA", "imm", 0x40)
        a.op("STA", "zp", 0x0E)       # PF1 bit 6 -> playfield bit 5
        a.op("LDA", "imm", 0x80)
        a.op("STA", "zp", 0x0F)       # PF2 bit 7 -> playfield bit 19
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", 0x0A)       # no reflection
    row = _screen_of(line)[20]
    lit = set(np.where(row == 0x44)[0])
    exp = set(range(0, 4)) | set(range(20, 24)) | set(range(76, 80))
    exp |= {x + 80 for x in exp}
    assert lit == exp
    assert np.all(row[[x for x in range(160) if x not in exp]] == 0x12)

    def line_r(a):
        line(a)
        a.op("LDA", "imm", 1)
        a.op("STA", "zp", 0x0A)       # reflect right half
    row = _screen_of(line_r)[20]
    lit = set(np.where(row == 0x44)[0])
    left = set(range(0, 4)) | set(range(20, 24)) | set(range(76, 80))
    assert lit == left | {159 - x for x in left}


def test_colour_write_mid_line_and_lsb_masked():
    """STA COLUBK at line cycle c changes pixels from colour clock 3c on."""
    def line(a):
        a.op("LDA", "imm", 0x21)       # odd: the pixel keeps only bits 7..1
        a.op("STA", "zp", 0x09)        # write at cycle 5 -> clock 15 (HBLANK)
        a.op("LDA", "imm", 0x60)
        for _ in range(12):
            a.op("NOP")                # cycles 6..29
        a.op("STA", "zp", 0x09)        # cycles 32..34 -> write at cycle 34 = clock 102
    row = _screen_of(line)[30]
    x0 = 3 * 34 - 68
    assert np.all(row[:x0] == 0x20) and np.all(row[x0:] == 0x60)


def _player_line(ctrlpf, nops):
    def line(a):
        a.op("LDA", "imm", 0x80)
        a.op("STA", "zp", 0x06)    # COLUP0 = $80
        a.op("LDA", "imm", 0xF0)
        a.op("STA", "zp", 0x0D)    # PF0 = $F0: pixels 0..15 and 80..95
        a.op("LDA", "imm", 0x40)
        a.op("STA", "zp", 0x08)    # COLUPF
        a.op("LDA", "imm", 0xA5)
        a.op("STA", "zp", 0x1B)    # GRP0 = 10100101
        a.op("LDA", "imm", ctrlpf)
        a.op("STA", "zp", 0x0A)
        for _ in range(nops):
            a.op("NOP")
        a.op("STA", "zp", 0x10)    # RESP0
    return line


def test_player_position_and_priority():
    """RESP0 written at line cycle c puts P0 at (3c - 68 + 5) mod 160; GRP0
    is drawn MSB first; P0 beats PF unless CTRLPF bit 2."""
    bits = [1, 0, 1, 0, 0, 1, 0, 1]
    # 5 x (LDA # + STA zp) = 25 cycles, NOPs, then STA RESP0 writes at +3
    c = 25 + 2 * 5 + 3
    pos = 3 * c - 68 + 5
    assert pos == 51
    row = _screen_of(_player_line(0, 5))[40]
    for i, b in enumerate(bits):
        assert row[pos + i] == (0x80 if b else 0x00), (i, row[pos + i])
    assert row[pos - 1] == 0 and row[pos + 8] == 0
    # 6 more NOPs: c = 50 -> position 87, inside the PF0 block 80..95
    pos = 3 * (c + 12) - 68 + 5
    assert pos == 87
    r0 = _screen_of(_player_line(0, 11))[40]
    r4 = _screen_of(_player_line(4, 11))[40]
    for i, b in enumerate(bits):
        assert r0[pos + i] == (0x80 if b else 0x40)
        assert r4[pos + i] == 0x40


def test_resp0_in_hblank_gives_position_3():
    def line(a):
        a.op("LDA", "imm", 0x80)
        a.op("STA", "zp", 0x06)
        a.op("LDA", "imm", 0xFF)
        a.op("STA", "zp", 0x1B)
        a.op("STA", "zp", 0x10)        # cycle 13 -> clock 39 < 68
    row = _screen_of(line)[40]
    assert set(np.where(row == 0x80)[0]) == set(range(3, 11))


def test_hmove_blank_and_motion():
    """HMOVE right after WSYNC blanks pixels 0..7 of that line and moves P0
    left by the signed HMP0 nibble."""
    def line(a):
        a.op("STA", "zp", 0x2A)        # HMOVE at cycle 3 -> clock 9
        a.op("LDA", "imm", 0x0E)
        a.op("STA", "zp", 0x09)        # COLUBK = $0E
    row = _screen_of(line)[10]
    assert np.all(row[:8] == 0) and np.all(row[8:] == 0x0E)


def test_vblank_blacks_out():
    def line(a):
        a.op("LDA", "imm", 0x3C)
        a.op("STA", "zp", 0x09)
        a.op("LDA", "imm", 2)
        a.op("STA", "zp", 0x01)        # VBLANK on from cycle 10 -> clock 30
    row = _screen_of(line)[10]
    assert np.all(row == 0)


def test_stored_bench_counts_are_current():
    """bench.py reads its instruction counts from tests/golden/bench_counts.json
    (the roofline's work and the paper's unit); they must be what the
    committed script computes from the oracle today."""
    import json
    import os
    import sys
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    sys.path.insert(0, here)
    import make_bench_counts
    stored = json.load(open(os.path.join(here, "bench_counts.json")))
    assert stored == make_bench_counts.counts()


def test_boot_protocol_frames_and_reset_switch():
    """The boot protocol (60 NOOP + 4 RESET frames, then the episode's extra
    NOOPs) as the cart sees it: the frame counter advances by the number of
    boot frames, SWCHB reads $0A exactly during the RESET frames and $0B
    otherwise."""
    from paper_2606_22447_b300 import synth
    from tests.microrom import switches_rom
    o = oracle.Oracle(switches_rom(), synth.MAPPER_4K)
    o.boot(60, 4, 7)
    ram = o.ram()
    # the power-on frame ends at the cart's first VSYNC, before its first
    # increment; every later boot frame adds one
    assert ram[0x00] == 60 + 4 + 7 - 1
    assert ram[0x01] == 0x0A and ram[0x02] == 0x0B      # RESET was seen, and released again
    o2 = oracle.Oracle(switches_rom(), synth.MAPPER_4K)
    o2.boot(60, 0, 0)
    assert o2.ram()[0x00] == 60 - 1 and o2.ram()[0x01] == 0x0B   # no RESET frames: never pressed


# ---------------------------------------------------------------------------
# Superchip cartridge RAM
# ---------------------------------------------------------------------------

def _superchip_image(mapper):
    """Banked image whose last bank writes the cartridge RAM through the
    write port, reads it back through the read port (plain and indexed),
    reads the write port (ROM), writes the read port (nothing), copies a
    three-byte routine into the RAM and calls it there, then switches to
    bank 0, which reads the RAM again.  Each bank's byte at offset $005 is
    $77 + bank and its bytes at $080-$0FF are $E0 + bank, so a read that
    reaches the ROM instead of the RAM is recognisable."""
    nb, hot = synth.MAPPER_BANKS[mapper], synth.MAPPER_HOTSPOT[mapper]

    def header(a, j):
        a.at(0x005)
        a.byte(0x77 + j)
        a.at(0x080)
        for _ in range(0x80):
            a.byte(0xE0 + j)
        a.at(0x100)

    def vectors(a):
        a.at(4096 - 6)
        a.word(0xF100), a.word(0xF100), a.word(0xF100)
        return bytes(a.resolve())

    a = synth.Asm(0xF000, 4096)
    header(a, nb - 1)
    a.op("LDA", "imm", 0x5A)
    a.op("STA", "abs", 0x1005)        # cart RAM[5] = $5A
    a.op("LDA", "imm", 0xC3)
    a.op("LDX", "imm", 2)
    a.op("STA", "absx", 0x1010)       # cart RAM[$12] = $C3
    a.op("LDA", "abs", 0x1085)
    a.op("STA", "zp", 0x80)           # RAM[0] = cart RAM[5]
    a.op("LDY", "imm", 0x0D)
    a.op("LDA", "absy", 0x1085)
    a.op("STA", "zp", 0x81)           # RAM[1] = cart RAM[$12]
    a.op("LDA", "abs", 0x1005)
    a.op("STA", "zp", 0x82)           # RAM[2] = the ROM under the write port
    a.op("LDA", "imm", 0x99)
    a.op("STA", "abs", 0x1080)        # a write to the read port: nothing
    a.op("LDA", "abs", 0x1080)
    a.op("STA", "zp", 0x83)           # RAM[3] = cart RAM[0]
    for k, v in enumerate((0xA9, 0x42, 0x60)):   # LDA #$42; RTS
        a.op("LDA", "imm", v)
        a.op("STA", "abs", 0x1020 + k)
    a.op("JSR", "abs", 0x10A0)        # run it from the cartridge RAM
    a.op("STA", "zp", 0x84)
    a.op("LDA", "abs", hot)           # -> bank 0, which resumes at the next offset
    resume = a.pc - 0xF000
    last = vectors(a)
    banks = []
    for j in range(nb - 1):
        b = synth.Asm(0xF000, 4096)
        header(b, j)
        b.at(resume)
        b.op("LDA", "abs", 0x1085)
        b.op("STA", "zp", 0x85)
        b.label("HALT")
        b.op("JMP", "abs", "HALT")
        banks.append(vectors(b))
    return b"".join(banks) + last


@pytest.mark.parametrize("mapper", [synth.MAPPER_F8SC, synth.MAPPER_F6SC, synth.MAPPER_F4SC])
def test_superchip_ram_ports(mapper):
    """Writes at $1000-$107F store into the cartridge RAM, reads at
    $1080-$10FF return it (in every bank, and as code), a read of the write
    port returns the ROM byte there and a write to the read port changes
    nothing.  The same image as a plain banked cart reads ROM throughout."""
    nb = synth.MAPPER_BANKS[mapper]
    rom = _superchip_image(mapper)
    o = oracle.Oracle(rom, mapper)
    for _ in range(200):
        o.exec_one()
    ram, cram = o.ram(), o.cart_ram()
    assert o.bank() == 0
    assert list(ram[:6]) == [0x5A, 0xC3, 0x77 + nb - 1, 0x00, 0x42, 0x5A]
    want = np.zeros(128, np.uint8)
    want[0x05], want[0x12], want[0x20:0x23] = 0x5A, 0xC3, (0xA9, 0x42, 0x60)
    assert np.array_equal(cram, want)
    base = synth.MAPPER_SC_BASE[mapper]
    p = oracle.Oracle(rom, base)
    for _ in range(200):
        p.exec_one()
    top = 0xE0 + nb - 1
    # the plain cart: reads of $1085, $1092 and $1080 return ROM; its JSR
    # then runs ROM bytes, so only the first four cells are pinned
    assert list(p.ram()[:4]) == [top, top, 0x77 + nb - 1, top]
    assert not p.cart_ram().any()


def test_superchip_carts_use_their_ram():
    """The generated Superchip carts run well-formed frames, keep code out of
    the RAM ports' 256 bytes and leave values in the cartridge RAM."""
    for mapper in (synth.MAPPER_F8SC, synth.MAPPER_F6SC, synth.MAPPER_F4SC):
        rom = synth.config_carts(19, [mapper])[0]
        assert len(rom) == synth.MAPPER_SIZE[mapper]
        o = oracle.Oracle(rom, mapper)
        for a in synth.actions(20, 1, 12)[:, 0]:
            assert o.step(int(a), 2)[2] == 0
        c = o.counters()
        assert c["watchdog"] == 0 and c["frames"] == 24
        assert np.count_nonzero(o.cart_ram()) >= 4


# ---------------------------------------------------------------------------
# E0 slices
# ---------------------------------------------------------------------------

def _e0_image(program):
    """8 KB E0 image: byte i of slice k is $A0 + k at offsets 0..3 and
    $10 * k + (i & 15) elsewhere; slice 7 (segment 3, $FC00) holds the
    program at $FD00 and the vectors."""
    slices = []
    for k in range(8):
        a = synth.Asm(0xFC00 if k == 7 else 0xF000, 1024)
        for i in range(4):
            a.byte(0xA0 + k)
        while len(a.buf) < 0x100:
            a.byte((0x10 * k + (len(a.buf) & 15)) & 0xFF)
        if k == 7:
            program(a)
            a.at(1024 - 6)
            a.word(0xFD00), a.word(0xFD00), a.word(0xFD00)
        slices.append(bytes(a.resolve()))
    return b"".join(slices)


def test_e0_hotspots_map_slices():
    """Power-on shows slices 4, 5, 6 in segments 0..2 and slice 7 in segment
    3; an access (read or write) to $1FE0+j, $1FE8+j, $1FF0+j maps slice j
    into segment 0, 1, 2; $1FDF, $1FF8 and the hotspots' image below A12
    change nothing."""
    def program(a):
        a.at(0x100)
        for seg, dst in ((0, 0x80), (1, 0x81), (2, 0x82), (3, 0x83)):
            a.op("LDA", "abs", 0x1000 + 0x400 * seg)
            a.op("STA", "zp", dst)
        a.op("LDA", "abs", 0x1FE2)             # segment 0 <- slice 2
        a.op("STA", "abs", 0x1FEF)             # segment 1 <- slice 7 (a write)
        a.op("LDA", "abs", 0xFFF1)             # segment 2 <- slice 1 (A13-A15 ignored)
        a.op("LDA", "abs", 0x1FDF)             # not a hotspot
        a.op("LDA", "abs", 0x1FF8)             # not a hotspot
        a.op("LDA", "abs", 0x0FE3)             # A12 = 0: not the cartridge
        for seg, dst in ((0, 0x84), (1, 0x85), (2, 0x86), (3, 0x87)):
            a.op("LDA", "abs", 0x1000 + 0x400 * seg)
            a.op("STA", "zp", dst)
        a.op("LDA", "abs", 0x1004)              # segment 0 (slice 2), offset 4: $10 * 2 + 4
        a.op("STA", "zp", 0x88)
        a.label("HALT")
        a.op("JMP", "abs", "HALT")
    o = oracle.Oracle(_e0_image(program), synth.MAPPER_E0)
    assert o.bank() == 4 | 5 << 3 | 6 << 6
    for _ in range(40):
        o.exec_one()
    ram = o.ram()
    assert list(ram[:9]) == [0xA4, 0xA5, 0xA6, 0xA7, 0xA2, 0xA7, 0xA1, 0xA7, 0x24]
    assert o.bank() == 2 | 7 << 3 | 1 << 6


def test_e0_carts_map_several_slices():
    """The generated E0 carts run well-formed frames (no jam, no watchdog)
    and map every slice of each segment's set over a few frames of random
    input."""
    rom = synth.config_carts(21, [synth.MAPPER_E0])[0]
    assert len(rom) == 8192
    o = oracle.Oracle(rom, synth.MAPPER_E0)
    seen = [set(), set(), set()]
    for a in synth.actions(22, 1, 60)[:, 0]:
        for _ in range(400):
            o.trace(int(a), 1)
            b = int(o.state()[8])
            for k in range(3):
                seen[k].add((b >> (3 * k)) & 7)
    c = o.counters()
    assert c["watchdog"] == 0 and o.state()[28] == 0
    assert 1500 < c["instructions"] / c["frames"] < 4000
    assert {0, 1} <= seen[0] and {2, 3, 4} <= seen[1] and {5, 6} <= seen[2]


def _fe_image():
    """Bank 0 ($F000, the image's first 4 KB) and bank 1 ($D000): each has
    the marker A0 / B1 at offset $800, read as LDA $F800 (the address's top
    bits do not reach the cartridge)."""
    b0 = synth.Asm(0xF000, 4096)
    b0.op("JMP", "abs", 0xF100)
    b0.at(0x010)                       # $D010 seen through bank 0
    b0.op("LDA", "abs", 0xF800)
    b0.op("STA", "zp", 0x84)
    b0.op("RTS")
    b0.at(0x100)
    b0.op("LDX", "imm", 0xFF)
    b0.op("TXS")
    b0.op("LDA", "abs", 0xF800)        # power-on: bank 0
    b0.op("STA", "zp", 0x80)
    b0.op("JSR", "abs", 0xD000)        # S = $FF, target high byte $D0: bank 1
    b0.op("LDA", "abs", 0xF800)        # its RTS (S = $FD, return high byte $F1): bank 0
    b0.op("STA", "zp", 0x83)
    b0.op("LDA", "imm", 0)
    b0.op("PHA")
    b0.op("PHA")                       # S = $FD
    b0.op("JSR", "abs", 0xD010)        # not from the top of the stack: no switch
    b0.op("PLA")
    b0.op("PLA")
    b0.op("LDX", "imm", 0xFE)
    b0.op("TXS")
    b0.op("PHA")                       # a push to $01FE (then STA's opcode $8D, bit 5 clear)
    b0.op("STA", "zp", 0x87)
    b0.op("LDA", "abs", 0xF800)        # not a JSR or RTS: no switch
    b0.op("STA", "zp", 0x88)
    b0.op("LDX", "imm", 0xFF)
    b0.op("TXS")
    b0.op("LDA", "imm", 0xD0)
    b0.op("PHA")
    b0.op("LDA", "imm", 0x1F)
    b0.op("PHA")                       # S = $FD; $01FE holds $1F, $01FF $D0
    b0.op("RTS")                       # pulls $D01F: bank 1, continues at $D020
    b0.at(0x200)
    b0.op("LDA", "abs", 0xF800)        # reached from bank 1 by JSR $F200 (high byte $F2)
    b0.op("STA", "zp", 0x86)
    b0.label("HALT")
    b0.op("JMP", "abs", "HALT")
    b0.at(0x800)
    b0.byte(0xA0)
    b0.at(4096 - 6)
    b0.word(0xF100), b0.word(0xF100), b0.word(0xF100)
    b1 = synth.Asm(0xD000, 4096)
    b1.op("LDA", "abs", 0xF800)
    b1.op("STA", "zp", 0x81)
    b1.op("RTS")
    b1.at(0x020)
    b1.op("LDA", "abs", 0xF800)
    b1.op("STA", "zp", 0x85)
    b1.op("JSR", "abs", 0xF200)        # S = $FF again, high byte $F2: bank 0
    b1.at(0x800)
    b1.byte(0xB1)
    b1.at(4096 - 6)
    b1.word(0xD000), b1.word(0xD000), b1.word(0xD000)
    return bytes(b0.resolve()) + bytes(b1.resolve())


def test_fe_switches_through_jsr_and_rts_at_the_top_of_the_stack():
    """FE (two 4 KB banks, the image's first shown at power-on): a JSR with
    the stack pointer at $FF and an RTS with it at $FD select the bank from
    bit 5 of the next bus byte (the target's, or the return address's, high
    byte: set -> the first 4 KB, clear -> the second); a JSR deeper in the
    stack and a plain push to $01FE switch nothing."""
    o = oracle.Oracle(_fe_image(), synth.MAPPER_FE)
    assert o.bank() == 0
    for _ in range(60):
        o.exec_one()
    ram = o.ram()
    assert list(ram[0:2]) == [0xA0, 0xB1]
    assert list(ram[3:7]) == [0xA0, 0xA0, 0xB1, 0xA0]
    assert ram[8] == 0xA0
    assert o.bank() == 0


def test_fe_carts_use_both_banks():
    """The generated FE carts run well-formed frames and spend frames in
    both banks' kernels."""
    rom = synth.config_carts(23, [synth.MAPPER_FE])[0]
    assert len(rom) == 8192
    o = oracle.Oracle(rom, synth.MAPPER_FE)
    seen = set()
    for a in synth.actions(24, 1, 40)[:, 0]:
        for _ in range(400):
            o.trace(int(a), 1)
            seen.add(int(o.state()[8]))
    c = o.counters()
    assert c["watchdog"] == 0 and o.state()[28] == 0
    assert 1500 < c["instructions"] / c["frames"] < 4000
    assert seen == {0, 1}


# ---------------------------------------------------------------------------
# the rest of the TIA: player 1, missiles, ball, sizes, delays, collisions
# (expected pixels worked out by hand from the register definitions)
# ---------------------------------------------------------------------------

T = dict(NUSIZ0=0x04, NUSIZ1=0x05, COLUP0=0x06, COLUP1=0x07, COLUPF=0x08, COLUBK=0x09, CTRLPF=0x0A,
         REFP0=0x0B, REFP1=0x0C, PF0=0x0D, PF1=0x0E, PF2=0x0F, RESP0=0x10, RESP1=0x11, RESM0=0x12,
         RESM1=0x13, RESBL=0x14, GRP0=0x1B, GRP1=0x1C, ENAM0=0x1D, ENAM1=0x1E, ENABL=0x1F, HMP0=0x20,
         HMP1=0x21, HMM0=0x22, HMM1=0x23, HMBL=0x24, VDELP0=0x25, VDELP1=0x26, VDELBL=0x27, RESMP0=0x28,
         RESMP1=0x29, HMOVE=0x2A, HMCLR=0x2B, CXCLR=0x2C)


def _frame_setup(a, writes):
    """One scanline per register write, each stored right after WSYNC (line
    clock 15, inside HBLANK: RESPx -> 3, RESMx / RESBL -> 2); value None is
    a strobe."""
    for reg, v in writes:
        a.op("STA", "zp", WSYNC)
        if v is not None:
            a.op("LDA", "imm", v)
        a.op("STA", "zp", T[reg])


def _screen_after(writes):
    """Row 100 of a frame whose first lines make `writes` (then plain
    lines)."""
    def build(a):
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", VBLANK)
        a.label("FRAME")
        a.op("LDA", "imm", 2)
        a.op("STA", "zp", WSYNC)
        a.op("STA", "zp", VSYNC)
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", VSYNC)
        _frame_setup(a, writes)
        a.op("LDX", "imm", 200)
        a.label("LINE")
        a.op("STA", "zp", WSYNC)
        a.op("DEX")
        a.op("BNE", "rel", "LINE")
        a.op("JMP", "abs", "FRAME")
    o = oracle.Oracle(rom4k(build), synth.MAPPER_4K, ystart=0, full_tia=True)
    for _ in range(2):
        _, scr, st = o.step(0, 1)
    assert st == 0
    return scr[100]


def _lit(row, colour):
    return sorted(np.where(row == colour)[0].tolist())


@pytest.mark.parametrize("refl", [0, 8])
def test_player1_copies_and_reflection(refl):
    """GRP1 = %11000001, NUSIZ1 = 3 (three copies 16 apart), RESP1 in HBLANK
    (position 3): bits 7, 6, 0 at +0, +1, +7 of each copy, or with REFP1 bit 3
    set (bit k at +k) at +7, +6, +0."""
    row = _screen_after([("COLUBK", 0x12), ("GRP1", 0xC1), ("NUSIZ1", 3), ("COLUP1", 0x44),
                         ("REFP1", refl), ("RESP1", None)])
    rel = (0, 1, 7) if not refl else (7, 6, 0)
    assert _lit(row, 0x44) == sorted(3 + c + r for c in (0, 16, 32) for r in rel)
    assert set(row.tolist()) == {0x12, 0x44}


@pytest.mark.parametrize("mode,scale", [(5, 2), (7, 4)])
def test_player_double_and_quad_width(mode, scale):
    row = _screen_after([("GRP0", 0xC1), ("NUSIZ0", mode), ("COLUP0", 0x44), ("RESP0", None)])
    assert _lit(row, 0x44) == sorted(3 + b * scale + j for b in (0, 1, 7) for j in range(scale))


def test_missiles_ball_widths_copies_and_priority():
    """M0 4 wide at 2; M1 2 wide, two copies 32 apart (NUSIZ1 mode 2) at 2 and
    34; the ball 8 wide at 2: M0 > M1 > BL where they overlap."""
    row = _screen_after([("COLUBK", 0x12), ("COLUP0", 0x44), ("COLUP1", 0x66), ("COLUPF", 0x88),
                         ("ENAM0", 2), ("NUSIZ0", 0x20), ("ENAM1", 2), ("NUSIZ1", 0x12),
                         ("ENABL", 2), ("CTRLPF", 0x30), ("RESM0", None), ("RESM1", None), ("RESBL", None)])
    assert _lit(row, 0x44) == [2, 3, 4, 5]
    assert _lit(row, 0x66) == [34, 35]
    assert _lit(row, 0x88) == [6, 7, 8, 9]


@pytest.mark.parametrize("ctrl,left,right", [(2, 0x44, 0x66), (6, 0x88, 0x88), (0, 0x88, 0x88)])
def test_score_mode(ctrl, left, right):
    """PF1 = $FF covers columns 16..47 and (repeated) 96..127; score mode
    (CTRLPF bit 1) colours them COLUP0 / COLUP1 by half, unless the
    playfield has priority (bit 2)."""
    row = _screen_after([("COLUBK", 0x12), ("COLUP0", 0x44), ("COLUP1", 0x66), ("COLUPF", 0x88),
                         ("PF1", 0xFF), ("CTRLPF", ctrl)])
    if left != right:
        assert _lit(row, left) == list(range(16, 48)) and _lit(row, right) == list(range(96, 128))
    else:
        assert _lit(row, left) == list(range(16, 48)) + list(range(96, 128))


@pytest.mark.parametrize("copy", [False, True])
def test_vertical_delay(copy):
    """VDELP0 set: player 0 shows the delayed GRP0, which only a GRP1 write
    updates (from GRP0)."""
    writes = [("COLUP0", 0x44), ("VDELP0", 1), ("GRP0", 0xFF)] + ([("GRP1", 0)] if copy else [])
    row = _screen_after(writes + [("RESP0", None)])
    assert _lit(row, 0x44) == (list(range(3, 11)) if copy else [])


def test_hmove_moves_every_object_and_resmp_locks():
    """HMOVE moves P1 by -(-1), M0 by -1 and the ball by -2 from their strobe
    positions 3, 2, 2 (then HMCLR: a second HMOVE moves nothing); a missile
    locked with RESMP0 is hidden and, once released, sits at its player's
    position + 3."""
    row = _screen_after([("COLUBK", 0x12), ("COLUP0", 0x44), ("COLUP1", 0x66), ("COLUPF", 0x88),
                         ("GRP1", 0x80), ("ENAM0", 2), ("ENABL", 2), ("HMP1", 0xF0), ("HMM0", 0x10),
                         ("HMBL", 0x20), ("RESP1", None), ("RESM0", None), ("RESBL", None),
                         ("HMOVE", None), ("HMCLR", None), ("HMOVE", None)])
    assert _lit(row, 0x66) == [4] and _lit(row, 0x44) == [1] and _lit(row, 0x88) == [0]
    row = _screen_after([("COLUP0", 0x44), ("ENAM0", 2), ("RESP0", None), ("RESMP0", 2)])
    assert _lit(row, 0x44) == []
    row = _screen_after([("COLUP0", 0x44), ("ENAM0", 2), ("RESP0", None), ("RESMP0", 2), ("RESMP0", 0)])
    assert _lit(row, 0x44) == [6]


def test_collision_latches():
    """Each frame reads CXP0FB, CXPPMM, CXM0P into RAM, then CXCLR; every
    line P0 (columns 3..10) overlaps PF0 (0..15) and M0 overlaps M1 (both 1
    wide at 2, off the player): D7 of CXP0FB, D6 of CXPPMM, nothing in
    CXM0P.  Without the playfield, CXP0FB stays clear."""
    def run(pf0):
        def build(a):
            a.label("FRAME")
            a.op("LDA", "imm", 2)
            a.op("STA", "zp", WSYNC)
            a.op("STA", "zp", VSYNC)
            a.op("LDA", "imm", 0)
            a.op("STA", "zp", VSYNC)
            for reg, dst in ((0x02, 0x80), (0x07, 0x81), (0x00, 0x82)):
                a.op("LDA", "zp", reg)
                a.op("STA", "zp", dst)
            a.op("STA", "zp", T["CXCLR"])
            a.op("LDX", "imm", 230)
            a.label("LINE")
            a.op("STA", "zp", WSYNC)
            for reg in ("RESP0", "RESM0", "RESM1"):   # strobes first, inside HBLANK: 3, 2, 2
                a.op("STA", "zp", T[reg])
            for reg, v in (("GRP0", 0xFF), ("PF0", pf0), ("ENAM0", 2), ("ENAM1", 2)):
                a.op("LDA", "imm", v)
                a.op("STA", "zp", T[reg])
            a.op("DEX")
            a.op("BNE", "rel", "LINE")
            a.op("JMP", "abs", "FRAME")
        o = oracle.Oracle(rom4k(build), synth.MAPPER_4K, full_tia=full)
        for _ in range(3):
            o.step(0, 1)
        return list(o.ram()[:3])
    full = True
    assert run(0xF0) == [0x80, 0x40, 0x00]
    assert run(0x00) == [0x00, 0x40, 0x00]
    full = False   # the subset machine: collision registers read 0
    assert run(0xF0) == [0x00, 0x00, 0x00]
