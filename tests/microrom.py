"""Tiny hand-assembled test cartridges built with the input module's assembler."""
from paper_2606_22447_b300 import synth


def rom4k(build, origin=0xF000, table=True):
    """4K image: `build(asm)` emits code at $F000; an identity table sits at
    $FE00 (value i at $FE00+i) and the reset vector points at $F000."""
    a = synth.Asm(origin, 4096)
    build(a)
    if table:
        a.at(0xE00)
        for i in range(256):
            a.byte(i)
    a.at(4096 - 6)
    a.word(0xF000)
    a.word(0xF000)
    a.word(0xF000)
    return bytes(a.resolve())


# The paper's 38 extra opcode bytes, by addressing mode (raw bytes: the
# assembler knows the documented opcodes only).
EXTRA_IMP = (0x1A, 0x3A, 0x5A, 0x7A, 0xDA, 0xFA)
EXTRA_IMM = (0x80, 0x82, 0x89, 0xC2, 0xE2, 0xEB)          # NOPs #imm and USBC #imm
EXTRA_ZP = (0x04, 0x44, 0x64, 0xA7, 0x87)                 # NOP zp, LAX zp, SAX zp
EXTRA_ZPXY = (0x14, 0x34, 0x54, 0x74, 0xD4, 0xF4, 0xB7, 0x97)   # NOP zp,X; LAX zp,Y; SAX zp,Y
EXTRA_ABS = (0x0C, 0xAF, 0x8F)                            # NOP abs, LAX abs, SAX abs
EXTRA_ABSXY = (0x1C, 0x3C, 0x5C, 0x7C, 0xDC, 0xFC, 0xBF)  # NOP abs,X; LAX abs,Y
EXTRA_IND = (0xA3, 0xB3, 0x83)                            # LAX (zp,X), LAX (zp),Y, SAX (zp,X)


def extra_ops_rom():
    """A frame loop that runs all 38 extra opcode bytes on joystick-dependent
    data each line and shows the results in the colour registers: LAX / SAX
    on RAM and TIA addresses, USBC in binary and decimal mode, NOPs reading
    RAM, INTIM and SWCHA (page-crossing abs,X included).  Index registers are
    masked before indexed and indirect accesses so that every store lands in
    RAM or a colour register."""
    def build(a):
        a.op("LDX", "imm", 0xFF)
        a.op("TXS")
        for k, target in enumerate((0x90, 0x94, 0x98, 0x9C, 0x90)):   # pointers $80.. and $88
            a.op("LDA", "imm", target)
            a.op("STA", "zp", 0x80 + 2 * k)
            a.op("LDA", "imm", 0x00)
            a.op("STA", "zp", 0x81 + 2 * k)
        a.label("F")
        a.op("LDA", "imm", 2)
        a.op("STA", "zp", 0x02)
        a.op("STA", "zp", 0x00)
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", 0x00)
        a.op("LDA", "abs", 0x0280)     # joystick into $90
        a.op("STA", "zp", 0x90)
        a.op("LDA", "imm", 80)
        a.op("STA", "zp", 0x8A)        # loop turns (about 2.5 lines each)
        a.label("L")
        a.op("STA", "zp", 0x02)
        a.byte(0xA7, 0x90)             # LAX $90
        a.op("INX")
        a.byte(0x87, 0x91)             # SAX $91
        a.byte(0x87, 0x09)             # SAX COLUBK (a TIA write)
        a.op("SEC")
        a.byte(0xEB, 0x07)             # USBC #7 (binary)
        a.op("STA", "zp", 0x90)
        a.op("SED")
        a.byte(0xEB, 0x15)             # USBC #$15 (decimal)
        a.op("CLD")
        a.op("STA", "zp", 0x08)
        for op in EXTRA_IMP:
            a.byte(op)
        for op in EXTRA_IMM[:-1]:
            a.byte(op, 0x5A)
        a.byte(0x04, 0x90)
        a.byte(0x44, 0x91)
        a.byte(0x64, 0x92)
        a.op("TXA")                    # X in {0, 2, 4, 6}
        a.op("AND", "imm", 0x06)
        a.op("TAX")
        for op in EXTRA_ZPXY[:6]:
            a.byte(op, 0x90)           # NOP $90,X
        a.op("LDA", "zp", 0x91)        # Y in 0..31
        a.op("AND", "imm", 0x1F)
        a.op("TAY")
        a.byte(0xB7, 0x8E)             # LAX $8E,Y
        a.op("TXA")
        a.op("AND", "imm", 0x06)
        a.op("TAX")
        a.byte(0x97, 0xC0)             # SAX $C0,Y
        a.byte(0x0C, 0x84, 0x02)       # NOP INTIM
        a.byte(0xAF, 0x80, 0x02)       # LAX SWCHA
        a.op("TXA")
        a.op("AND", "imm", 0x06)
        a.op("TAX")
        a.byte(0x8F, 0x94, 0x00)       # SAX $0094
        a.op("LDX", "zp", 0x91)
        for op in EXTRA_ABSXY[:6]:
            a.byte(op, 0xF8, 0xFE)     # NOP $FEF8,X (crosses a page for X >= 8)
        a.byte(0xBF, 0x10, 0xFE)       # LAX $FE10,Y
        a.op("TXA")
        a.op("AND", "imm", 0x06)
        a.op("TAX")
        a.byte(0xA3, 0x80)             # LAX ($80,X)
        a.op("TXA")
        a.op("AND", "imm", 0x06)
        a.op("TAX")
        a.byte(0xB3, 0x88)             # LAX ($88),Y
        a.byte(0x83, 0x80)             # SAX ($80,X)
        a.op("STA", "zp", 0x06)
        a.op("STY", "zp", 0x1B)
        a.op("DEC", "zp", 0x8A)
        a.op("BEQ", "rel", "D")
        a.op("JMP", "abs", "L")
        a.label("D")
        a.op("JMP", "abs", "F")
    return rom4k(build)


def switches_rom():
    """Counts frames in $80, keeps the AND of every SWCHB read in $81 (bit 0
    clears once RESET has been seen) and the last SWCHB in $82, and draws
    the frame count in the background colour."""
    def build(a):
        a.op("SEI")
        a.op("CLD")
        a.op("LDX", "imm", 0xFF)
        a.op("TXS")
        a.op("LDA", "imm", 0xFF)
        a.op("STA", "zp", 0x81)
        a.label("F")
        a.op("LDA", "imm", 2)
        a.op("STA", "zp", 0x02)
        a.op("STA", "zp", 0x00)
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", 0x00)
        a.op("INC", "zp", 0x80)
        a.op("LDA", "abs", 0x0282)
        a.op("AND", "zp", 0x81)
        a.op("STA", "zp", 0x81)
        a.op("LDA", "abs", 0x0282)
        a.op("STA", "zp", 0x82)
        a.op("LDA", "abs", 0x0280)
        a.op("EOR", "zp", 0x80)
        a.op("STA", "zp", 0x83)
        a.op("LDY", "imm", 100)
        a.label("L")
        a.op("STA", "zp", 0x02)
        a.op("LDA", "zp", 0x80)
        a.op("STA", "zp", 0x09)
        a.op("LDA", "zp", 0x83)
        a.op("STA", "zp", 0x08)
        a.op("DEY")
        a.op("BNE", "rel", "L")
        a.op("JMP", "abs", "F")
    return rom4k(build)


SAMPLER_COLOURS = {"bk": 0x20, "pf": 0x44, "p0": 0x86}
SAMPLER_GRP0 = 0xB7
SAMPLER_PF2 = 0x30


def sampler_rom(resp_each_frame=True, ctrlpf=0):
    """Player 0 (GRP0 = $B7) over a background with a two-block playfield
    (PF2 = $30, columns 64..71 and 144..151); every frame copies SWCHA into
    HMP0 and strobes HMOVE at the start of scanline 2, above the visible
    rows.  With `resp_each_frame` RESP0 is strobed mid-way through scanline 1
    of every frame (so each frame's position depends on that frame's input
    only), otherwise once before the first frame (positions accumulate the
    motions of every frame)."""
    def resp0(a):
        a.op("STA", "zp", 0x02)            # WSYNC
        for _ in range(20):
            a.op("NOP")
        a.op("STA", "zp", 0x10)            # RESP0

    def build(a):
        a.op("LDA", "imm", SAMPLER_COLOURS["bk"])
        a.op("STA", "zp", 0x09)
        a.op("LDA", "imm", SAMPLER_COLOURS["pf"])
        a.op("STA", "zp", 0x08)
        a.op("LDA", "imm", SAMPLER_COLOURS["p0"])
        a.op("STA", "zp", 0x06)
        a.op("LDA", "imm", SAMPLER_GRP0)
        a.op("STA", "zp", 0x1B)
        a.op("LDA", "imm", SAMPLER_PF2)
        a.op("STA", "zp", 0x0F)
        a.op("LDA", "imm", ctrlpf)
        a.op("STA", "zp", 0x0A)
        if not resp_each_frame:
            resp0(a)
        a.label("FRAME")
        a.op("LDA", "imm", 2)
        a.op("STA", "zp", 0x02)
        a.op("STA", "zp", 0x00)            # VSYNC on: the frame boundary
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", 0x00)
        if resp_each_frame:
            resp0(a)
        else:
            a.op("STA", "zp", 0x02)
        a.op("LDA", "abs", 0x0280)         # SWCHA
        a.op("STA", "zp", 0x20)            # HMP0
        a.op("STA", "zp", 0x02)
        a.op("STA", "zp", 0x2A)            # HMOVE at the start of scanline 2
        a.op("LDX", "imm", 0)
        a.label("L")
        a.op("STA", "zp", 0x02)
        a.op("DEX")
        a.op("BNE", "rel", "L")
        a.op("JMP", "abs", "FRAME")
    return rom4k(build, table=False)


FULL_T_LOOP = 0xF09E     # the loop of the temperature cart
FULL_T_DATA = 0xF8D2     # its max-contrast byte


def full_temperature_rom():
    """NOPs from $F000 to the loop at $F09E, then `LDA $F8D2; STA $80;
    JMP $F09E`: the byte at $F8D2 is 0 with $FF on every side (the largest
    pull a temperature read can see), while every operand byte of the loop
    sits between neighbours that nearly balance (low byte $D2 between $AD
    and $F8, $9E between $4C and $F0, ...), so that the loop's own reads
    stay exact up to T = 0.17."""
    a = synth.Asm(0xF000, 4096)
    for _ in range(FULL_T_LOOP - 0xF000):
        a.op("NOP")
    a.op("LDA", "abs", FULL_T_DATA)
    a.op("STA", "zp", 0x80)
    a.op("JMP", "abs", FULL_T_LOOP)
    a.at(0xF8C0 - 0xF000)
    for i in range(0x40):
        a.byte(0x00 if 0xF8C0 + i == FULL_T_DATA else 0xFF)
    a.at(4096 - 6)
    a.word(0xF000)
    a.word(0xF000)
    a.word(0xF000)
    return bytes(a.resolve())


def full_branch_rom(offset, taken):
    """`LDX #1` (Z clear), then a branch of signed offset `offset` that is
    taken (BNE) or not (BEQ), landing on NOPs; NOPs all around."""
    a = synth.Asm(0xF000, 4096)
    for _ in range(0x100):
        a.op("NOP")
    a.op("LDX", "imm", 1)
    a.byte(0xD0 if taken else 0xF0, offset & 0xFF)
    for _ in range(0x300):
        a.op("NOP")
    a.at(4096 - 6)
    a.word(0xF000)
    a.word(0xF000)
    a.word(0xF000)
    return bytes(a.resolve())


GRAPHICS_COLOURS = {"bk": 0x20, "pf": 0x44, "p0": 0x86}
GRAPHICS_PF = (0xA0, 0x5C, 0x93)   # PF0, PF1, PF2


def graphics_rom(ctrlpf=0):
    """Player 0 over a playfield, both drawn on every visible line: each
    frame strobes RESP0 mid-way through scanline 1 (a fixed position),
    copies SWCHA into GRP0 (the joystick drives the sprite's bits) and
    stores PF0, PF1 and PF2 from immediates.  Returns (image, the ROM
    offsets of the PF0, PF1 and PF2 immediates)."""
    offs = []

    def build(a):
        a.op("LDA", "imm", GRAPHICS_COLOURS["bk"])
        a.op("STA", "zp", 0x09)
        a.op("LDA", "imm", GRAPHICS_COLOURS["pf"])
        a.op("STA", "zp", 0x08)
        a.op("LDA", "imm", GRAPHICS_COLOURS["p0"])
        a.op("STA", "zp", 0x06)
        a.op("LDA", "imm", ctrlpf)
        a.op("STA", "zp", 0x0A)
        a.label("FRAME")
        a.op("LDA", "imm", 2)
        a.op("STA", "zp", 0x02)
        a.op("STA", "zp", 0x00)            # VSYNC on: the frame boundary
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", 0x00)
        a.op("STA", "zp", 0x02)            # WSYNC
        for _ in range(20):
            a.op("NOP")
        a.op("STA", "zp", 0x10)            # RESP0
        a.op("LDA", "abs", 0x0280)         # SWCHA
        a.op("STA", "zp", 0x1B)            # GRP0
        for reg, v in zip((0x0D, 0x0E, 0x0F), GRAPHICS_PF):
            offs.append(a.pc + 1 - 0xF000)
            a.op("LDA", "imm", v)
            a.op("STA", "zp", reg)
        a.op("LDX", "imm", 0)
        a.label("L")
        a.op("STA", "zp", 0x02)
        a.op("DEX")
        a.op("BNE", "rel", "L")
        a.op("JMP", "abs", "FRAME")
    return rom4k(build, table=False), offs


GRAPHICS_FT_COLOURS = {"bk": 0x20, "pf": 0x44, "p0": 0x86, "p1": 0xC8}
GRAPHICS_FT_PF = (0x30, 0x81, 0x0C)


def graphics_full_tia_rom(ctrlpf=0, vdel=False):
    """Every object of the whole TIA on every visible line: player 0, player
    1, missile 0 (2 wide), the ball (4 wide) and a playfield, each strobed to
    its own position on the scanlines above the visible rows.  Each frame
    copies SWCHA into GRP1 (the joystick drives player 1's bits) and stores
    GRP0, ENAM0, ENABL and PF0-2 from immediates.  With `vdel` player 1 shows
    its delayed graphic (VDELP1): SWCHA is stored to GRP1, then GRP0's store
    copies it to the delayed register, then an immediate is stored to GRP1
    (which the screen then does not show).  Returns (image, ROM offsets of
    the immediates by name)."""
    offs = {}

    def imm(a, name, v, reg):
        offs[name] = a.pc + 1 - 0xF000
        a.op("LDA", "imm", v)
        a.op("STA", "zp", reg)

    def build(a):
        for reg, v in ((0x09, GRAPHICS_FT_COLOURS["bk"]), (0x08, GRAPHICS_FT_COLOURS["pf"]),
                       (0x06, GRAPHICS_FT_COLOURS["p0"]), (0x07, GRAPHICS_FT_COLOURS["p1"]),
                       (0x0A, ctrlpf | 0x20), (0x04, 0x10), (0x26, 1 if vdel else 0)):
            a.op("LDA", "imm", v)
            a.op("STA", "zp", reg)
        a.label("FRAME")
        a.op("LDA", "imm", 2)
        a.op("STA", "zp", 0x02)
        a.op("STA", "zp", 0x00)            # VSYNC on: the frame boundary
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", 0x00)
        for reg, nops in ((0x10, 12), (0x11, 22), (0x12, 26), (0x14, 17)):   # RESP0 RESP1 RESM0 RESBL
            a.op("STA", "zp", 0x02)        # WSYNC
            for _ in range(nops):
                a.op("NOP")
            a.op("STA", "zp", reg)
        a.op("LDA", "abs", 0x0280)         # SWCHA
        a.op("STA", "zp", 0x1C)            # GRP1
        imm(a, "grp0", 0xA5, 0x1B)
        if vdel:
            imm(a, "grp1", 0x3C, 0x1C)
        imm(a, "enam0", 0x02, 0x1D)
        imm(a, "enabl", 0x02, 0x1F)
        for name, reg, v in zip(("pf0", "pf1", "pf2"), (0x0D, 0x0E, 0x0F), GRAPHICS_FT_PF):
            imm(a, name, v, reg)
        a.op("LDX", "imm", 0)
        a.label("L")
        a.op("STA", "zp", 0x02)
        a.op("DEX")
        a.op("BNE", "rel", "L")
        a.op("JMP", "abs", "FRAME")
    return rom4k(build, table=False), offs


def dense_writes_rom():
    """Writes a picture register every three cycles, never ending a frame by
    VSYNC (the 512-line watchdog ends each one): every register the raster
    log records (VBLANK, colours, CTRLPF, playfield, GRP0, RESP0, HMOVE) with
    a value that changes each turn, over ten thousand writes per frame."""
    def build(a):
        a.op("SEI")
        a.op("CLD")
        a.op("LDA", "imm", 0x11)
        a.label("L")
        for reg in (0x09, 0x06, 0x08, 0x0D, 0x0E, 0x0F, 0x1B, 0x0A, 0x10, 0x20, 0x2A, 0x01):
            a.op("STA", "zp", reg)
        a.op("ADC", "imm", 0x07)
        a.op("JMP", "abs", "L")
    return rom4k(build)


def brk_pushes_rom():
    """BRK with the stack pointer at $0F: each BRK pushes its three bytes to
    $010F, $010E and $010D, the TIA's PF2, PF1 and PF0 (the densest writer: 3
    writes in 7 cycles), and its vector (the reset address) runs LDX #$0F;
    TXS; BRK again: 3 writes every 11 cycles."""
    def build(a):
        a.op("LDX", "imm", 0x0F)
        a.op("TXS")
        a.op("BRK")
    return rom4k(build)
