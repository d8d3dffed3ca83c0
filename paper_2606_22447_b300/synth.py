"""Seeded synthetic inputs for the VCS emulator: cartridges, action streams,
episode lengths and gradient seeds.

This module is an input producer only.  It assembles 6507 programs from
random templates and draws random numbers; it never executes a program and
holds none of the emulator's arithmetic.  Its only machine knowledge is an
assembler encoding table and a conservative per-instruction cycle budget,
used to keep each generated scanline block below 76 CPU cycles so that the
programs are well-formed NTSC-style frames.  Both the CPU oracle and the CUDA
path consume the bytes produced here.

Randomness comes from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): a 64-bit Weyl sequence with
increment 0x9E3779B97F4A7C15 passed through the variant-13 finaliser.

Cartridge shapes follow the paper's workloads: the 2K, 4K and F8 mappers of
the conformance set (per-game table, supplement; F6, F4, the Superchip
variants and E0 widen it to the nine mappers of Section 3, and FE to the
ten formats the conformance table's caption counts), 128 B of RIOT
RAM, a 160x210 screen window and NTSC frames of about 262 scanlines (Section 2.2).
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15

MAPPER_2K, MAPPER_4K, MAPPER_F8, MAPPER_F6, MAPPER_F4 = 0, 1, 2, 3, 4
# Superchip variants: the banked format plus 128 bytes of cartridge RAM,
# written at $1000-$107F and read at $1080-$10FF
MAPPER_F8SC, MAPPER_F6SC, MAPPER_F4SC = 5, 6, 7
MAPPER_SC_BASE = {MAPPER_F8SC: MAPPER_F8, MAPPER_F6SC: MAPPER_F6, MAPPER_F4SC: MAPPER_F4}
# E0: 8 KB in eight 1 KB slices; an access to $1FE0+j / $1FE8+j / $1FF0+j
# maps slice j into segment 0 / 1 / 2 of the cartridge window, segment 3
# always shows slice 7
MAPPER_E0 = 8
E0_HOTSPOT = (0x1FE0, 0x1FE8, 0x1FF0)
# FE: 8 KB in two 4 KB banks; a JSR made with the stack pointer at $FF (its
# return address's low byte pushed to $01FE) or an RTS made with it at $FD
# (the low byte pulled from $01FE) selects the bank from bit 5 of the next
# byte on the bus (the target's or the return address's high byte): set
# ($Fx) the image's first 4 KB, clear ($Dx) the second
MAPPER_FE = 9
MAPPER_SIZE = {MAPPER_2K: 2048, MAPPER_4K: 4096, MAPPER_F8: 8192, MAPPER_F6: 16384, MAPPER_F4: 32768,
               MAPPER_F8SC: 8192, MAPPER_F6SC: 16384, MAPPER_F4SC: 32768, MAPPER_E0: 8192, MAPPER_FE: 8192}
# banked mappers: number of 4 KB banks and the first hotspot (bank j at hot + j)
MAPPER_BANKS = {MAPPER_F8: 2, MAPPER_F6: 4, MAPPER_F4: 8, MAPPER_F8SC: 2, MAPPER_F6SC: 4, MAPPER_F4SC: 8}
MAPPER_HOTSPOT = {MAPPER_F8: 0x1FF8, MAPPER_F6: 0x1FF6, MAPPER_F4: 0x1FF4,
                  MAPPER_F8SC: 0x1FF8, MAPPER_F6SC: 0x1FF6, MAPPER_F4SC: 0x1FF4}
SC_WRITE, SC_READ = 0x1000, 0x1080

# ALE action order (18 actions) and their joystick components
# (right, left, down, up, fire).
ACTION_NAMES = (
    "NOOP", "FIRE", "UP", "RIGHT", "LEFT", "DOWN", "UPRIGHT", "UPLEFT",
    "DOWNRIGHT", "DOWNLEFT", "UPFIRE", "RIGHTFIRE", "LEFTFIRE", "DOWNFIRE",
    "UPRIGHTFIRE", "UPLEFTFIRE", "DOWNRIGHTFIRE", "DOWNLEFTFIRE",
)


def action_components(action: int) -> tuple:
    """(right, left, down, up, fire) in {0,1} for an ALE action index."""
    name = ACTION_NAMES[action]
    return (int("RIGHT" in name), int("LEFT" in name), int("DOWN" in name),
            int("UP" in name), int("FIRE" in name))


ACTION_TABLE = np.array([action_components(a) for a in range(18)], dtype=np.float32)


# --------------------------------------------------------------------------
# splitmix64
# --------------------------------------------------------------------------

def mix64(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def key3(seed: int, a: int, b: int) -> int:
    """Fold three integers into one 64-bit stream key."""
    h = mix64(seed + GAMMA)
    h = mix64(h ^ ((a + 1) * GAMMA))
    return mix64(h ^ ((b + 1) * 0xD1B54A32D192ED03))


class SplitMix64:
    def __init__(self, seed: int, a: int = 0, b: int = 0):
        self.state = key3(seed, a, b)

    def next(self) -> int:
        self.state = (self.state + GAMMA) & MASK64
        return mix64(self.state)

    def below(self, n: int) -> int:
        return self.next() % n

    def range(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi]."""
        return lo + self.below(hi - lo + 1)

    def chance(self, p: float) -> bool:
        return self.next() < int(p * (1 << 64))

    def pick(self, seq):
        return seq[self.below(len(seq))]

    def unit(self) -> float:
        return (self.next() >> 11) * (1.0 / (1 << 53))


def _np_mix64(z):
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def np_key3(seed: int, a, b):
    """Vectorised key3 over numpy arrays a, b (broadcast)."""
    with np.errstate(over="ignore"):
        a = np.asarray(a, dtype=np.uint64)
        b = np.asarray(b, dtype=np.uint64)
        h = np.uint64(mix64(seed + GAMMA))
        h = _np_mix64(h ^ ((a + np.uint64(1)) * np.uint64(GAMMA)))
        return _np_mix64(h ^ ((b + np.uint64(1)) * np.uint64(0xD1B54A32D192ED03)))


# --------------------------------------------------------------------------
# Actions, episode lengths, gradient seeds
# --------------------------------------------------------------------------

ACTION_STREAM = 0x41C7


def actions(seed: int, n_envs: int, n_steps: int, first_step: int = 0) -> np.ndarray:
    """uint8 [n_steps][n_envs], uniform over the 18 ALE actions."""
    env = np.arange(n_envs, dtype=np.uint64)[None, :]
    step = np.arange(first_step, first_step + n_steps, dtype=np.uint64)[:, None]
    with np.errstate(over="ignore"):
        k = np_key3(seed ^ ACTION_STREAM, env, step)
        k = _np_mix64(k + np.uint64(GAMMA))
    return (k % np.uint64(18)).astype(np.uint8)


def action_inputs(acts: np.ndarray) -> np.ndarray:
    """float32 [..., 5] joystick components (R, L, D, U, FIRE) of actions."""
    return ACTION_TABLE[np.asarray(acts, dtype=np.int64)]


def episode_lengths(seed: int, n_envs: int, n_episodes: int, mean_frames: float = 2000.0) -> np.ndarray:
    """uint32 [n_envs][n_episodes] geometric episode lengths (frames, >= 1)."""
    p = 1.0 / mean_frames
    env = np.arange(n_envs, dtype=np.uint64)[:, None]
    ep = np.arange(n_episodes, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        k = _np_mix64(np_key3(seed ^ 0xE915, env, ep) + np.uint64(GAMMA))
    u = ((k >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / (1 << 53))
    length = 1 + np.floor(np.log(u) / math.log1p(-p))
    return np.clip(length, 1, 2 ** 31).astype(np.uint32)


def start_noops(seed: int, n_envs: int, n_episodes: int, most: int = 30) -> np.ndarray:
    """uint8 [n_envs][n_episodes] NOOP frames starting each episode, uniform in
    0..most (the paper's episode-start randomisation)."""
    env = np.arange(n_envs, dtype=np.uint64)[:, None]
    ep = np.arange(n_episodes, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        k = _np_mix64(np_key3(seed ^ 0x5707, env, ep) + np.uint64(GAMMA))
    return (k % np.uint64(most + 1)).astype(np.uint8)


def normal_f32(seed: int, shape, stream: int = 0) -> np.ndarray:
    """Seeded standard normal float32 array (Box-Muller over splitmix64)."""
    n = int(np.prod(shape))
    idx = np.arange((n + 1) // 2, dtype=np.uint64)
    with np.errstate(over="ignore"):
        k1 = _np_mix64(np_key3(seed ^ 0x6A09, stream, idx) + np.uint64(GAMMA))
        k2 = _np_mix64(k1 + np.uint64(GAMMA))
    u1 = ((k1 >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / (1 << 53))
    u2 = (k2 >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])[:n]
    return z.reshape(shape).astype(np.float32)


# --------------------------------------------------------------------------
# A small 6502 assembler
# --------------------------------------------------------------------------

# (mnemonic, mode) -> opcode.  Modes: imp acc imm zp zpx zpy abs absx absy
# indx indy ind rel.
_OPS = {}


def _fill(mnem, pairs):
    for mode, code in pairs:
        _OPS[(mnem, mode)] = code


_ALU_MODES = ("imm", "zp", "zpx", "abs", "absx", "absy", "indx", "indy")
for _m, _base in (("ORA", 0x00), ("AND", 0x20), ("EOR", 0x40), ("ADC", 0x60),
                  ("LDA", 0xA0), ("CMP", 0xC0), ("SBC", 0xE0)):
    _fill(_m, zip(_ALU_MODES, (_base + 0x09, _base + 0x05, _base + 0x15, _base + 0x0D,
                               _base + 0x1D, _base + 0x19, _base + 0x01, _base + 0x11)))
_fill("STA", (("zp", 0x85), ("zpx", 0x95), ("abs", 0x8D), ("absx", 0x9D),
              ("absy", 0x99), ("indx", 0x81), ("indy", 0x91)))
for _m, _base in (("ASL", 0x00), ("ROL", 0x20), ("LSR", 0x40), ("ROR", 0x60)):
    _fill(_m, (("acc", _base + 0x0A), ("zp", _base + 0x06), ("zpx", _base + 0x16),
               ("abs", _base + 0x0E), ("absx", _base + 0x1E)))
_fill("INC", (("zp", 0xE6), ("zpx", 0xF6), ("abs", 0xEE), ("absx", 0xFE)))
_fill("DEC", (("zp", 0xC6), ("zpx", 0xD6), ("abs", 0xCE), ("absx", 0xDE)))
_fill("LDX", (("imm", 0xA2), ("zp", 0xA6), ("zpy", 0xB6), ("abs", 0xAE), ("absy", 0xBE)))
_fill("LDY", (("imm", 0xA0), ("zp", 0xA4), ("zpx", 0xB4), ("abs", 0xAC), ("absx", 0xBC)))
_fill("STX", (("zp", 0x86), ("zpy", 0x96), ("abs", 0x8E)))
_fill("STY", (("zp", 0x84), ("zpx", 0x94), ("abs", 0x8C)))
_fill("CPX", (("imm", 0xE0), ("zp", 0xE4), ("abs", 0xEC)))
_fill("CPY", (("imm", 0xC0), ("zp", 0xC4), ("abs", 0xCC)))
_fill("BIT", (("zp", 0x24), ("abs", 0x2C)))
_fill("JMP", (("abs", 0x4C), ("ind", 0x6C)))
_fill("JSR", (("abs", 0x20),))
for _m, _c in (("BPL", 0x10), ("BMI", 0x30), ("BVC", 0x50), ("BVS", 0x70),
               ("BCC", 0x90), ("BCS", 0xB0), ("BNE", 0xD0), ("BEQ", 0xF0)):
    _OPS[(_m, "rel")] = _c
for _m, _c in (("BRK", 0x00), ("PHP", 0x08), ("CLC", 0x18), ("PLP", 0x28), ("SEC", 0x38),
               ("RTI", 0x40), ("PHA", 0x48), ("CLI", 0x58), ("RTS", 0x60), ("PLA", 0x68),
               ("SEI", 0x78), ("DEY", 0x88), ("TXA", 0x8A), ("TYA", 0x98), ("TXS", 0x9A),
               ("TAY", 0xA8), ("TAX", 0xAA), ("CLV", 0xB8), ("TSX", 0xBA), ("INY", 0xC8),
               ("DEX", 0xCA), ("CLD", 0xD8), ("INX", 0xE8), ("NOP", 0xEA), ("SED", 0xF8)):
    _OPS[(_m, "imp")] = _c

_LEN = {"imp": 1, "acc": 1, "imm": 2, "zp": 2, "zpx": 2, "zpy": 2, "rel": 2,
        "abs": 3, "absx": 3, "absy": 3, "indx": 2, "indy": 2, "ind": 3}

_RMW = {"ASL", "ROL", "LSR", "ROR", "INC", "DEC"}
_STORE = {"STA", "STX", "STY"}


def budget_cycles(mnem: str, mode: str) -> int:
    """Conservative upper bound on the cycles of one instruction, for
    scheduling only (page-cross and taken-branch penalties included)."""
    if mode == "rel":
        return 4
    if mnem in ("BRK",):
        return 7
    if mnem in ("JSR", "RTS", "RTI"):
        return 6
    if mnem in ("PHA", "PHP"):
        return 3
    if mnem in ("PLA", "PLP"):
        return 4
    if mnem == "JMP":
        return 3 if mode == "abs" else 5
    if mnem in _RMW and mode != "acc":
        return {"zp": 5, "zpx": 6, "abs": 6, "absx": 7}[mode]
    return {"imp": 2, "acc": 2, "imm": 2, "zp": 3, "zpx": 4, "zpy": 4, "abs": 4,
            "absx": 5, "absy": 5, "indx": 6, "indy": 6}[mode]




class Asm:
    """Byte emitter with labels and label fixups.

    An operand may be an int or a label reference: "NAME", ("NAME", offset),
    ("<", "NAME") for the low byte or (">", "NAME") for the high byte of a
    label's address.  `cycles` accumulates the scheduling budget of the
    instructions emitted since it was last reset.
    """

    def __init__(self, origin: int, size: int):
        self.origin = origin
        self.size = size
        self.buf = bytearray()
        self.labels = {}
        self.fix_word = []
        self.fix_byte = []
        self.fix_rel = []
        self.cycles = 0

    @property
    def pc(self) -> int:
        return self.origin + len(self.buf)

    def label(self, name: str):
        assert name not in self.labels, name
        self.labels[name] = self.pc

    def byte(self, *vals):
        for v in vals:
            if isinstance(v, tuple) and v[0] in ("<", ">"):
                self.fix_byte.append((len(self.buf), v))
                self.buf.append(0)
            else:
                self.buf.append(v & 0xFF)

    def word(self, v):
        if isinstance(v, (str, tuple)):
            self.fix_word.append((len(self.buf), v))
            self.buf += b"\0\0"
        else:
            self.byte(v & 0xFF, v >> 8)

    def op(self, mnem: str, mode: str = "imp", arg=None):
        self.byte(_OPS[(mnem, mode)])
        n = _LEN[mode]
        if n == 2:
            if mode == "rel":
                self.fix_rel.append((len(self.buf), arg))
                self.buf.append(0)
            else:
                self.byte(arg)
        elif n == 3:
            self.word(arg)
        self.cycles += budget_cycles(mnem, mode)

    def at(self, offset: int):
        """Pad with NOP bytes up to a fixed offset within the image."""
        if len(self.buf) > offset:
            raise OverflowError(f"code reaches offset {len(self.buf):#x} > {offset:#x}")
        while len(self.buf) < offset:
            self.buf.append(0xEA)

    def _addr(self, ref) -> int:
        if isinstance(ref, str):
            return self.labels[ref]
        if ref[0] in ("<", ">"):
            v = self._addr(ref[1])
            return v & 0xFF if ref[0] == "<" else v >> 8
        return self.labels[ref[0]] + ref[1]

    def resolve(self) -> bytearray:
        for pos, ref in self.fix_word:
            v = self._addr(ref)
            self.buf[pos] = v & 0xFF
            self.buf[pos + 1] = (v >> 8) & 0xFF
        for pos, ref in self.fix_byte:
            self.buf[pos] = self._addr(ref)
        for pos, name in self.fix_rel:
            d = self.labels[name] - (self.origin + pos + 1)
            assert -128 <= d <= 127, (name, d)
            self.buf[pos] = d & 0xFF
        if len(self.buf) > self.size:
            raise OverflowError(f"image overflow: {len(self.buf)} > {self.size}")
        out = bytearray(self.buf)
        out += b"\xea" * (self.size - len(out))
        return out


# --------------------------------------------------------------------------
# Cartridge program generator
# --------------------------------------------------------------------------

# Hardware register addresses used by the generated programs.
VSYNC, VBLANK, WSYNC = 0x00, 0x01, 0x02
COLUP0, COLUPF, COLUBK, CTRLPF = 0x06, 0x08, 0x09, 0x0A
PF0, PF1, PF2, RESP0, GRP0, HMP0, HMOVE = 0x0D, 0x0E, 0x0F, 0x10, 0x1B, 0x20, 0x2A
INPT4, INPT5 = 0x0C, 0x0D
SWCHA, SWCHB, INTIM, TIMINT, TIM64T = 0x0280, 0x0282, 0x0284, 0x0285, 0x0296

# Zero-page plan: $80 line loop counter, $81 work loop counter, $82/$83
# pointer into RAM, $84/$85 pointer into a ROM table, $86..$EF work cells,
# $F0..$FF stack.
LINE_CTR, WORK_CTR, RAM_PTR, ROM_PTR = 0x80, 0x81, 0x82, 0x84
WORK_LO, WORK_HI = 0x86, 0xEF
RAM_PTR_TARGET = 0x0088
TABLE_LEN = 64 + 256

VISUAL_REGS = (COLUP0, COLUP0, COLUPF, COLUPF, COLUBK, PF0, PF1, PF2, PF1, GRP0,
               GRP0, GRP0, RESP0, RESP0, HMP0, CTRLPF)
# the rest of the TIA (full-TIA carts): player 1, missiles, ball, sizes,
# reflection, motion, vertical delay, missile locks, collision clear
NUSIZ0, NUSIZ1, COLUP1, REFP0, REFP1 = 0x04, 0x05, 0x07, 0x0B, 0x0C
RESP1, RESM0, RESM1, RESBL, GRP1, ENAM0, ENAM1, ENABL = 0x11, 0x12, 0x13, 0x14, 0x1C, 0x1D, 0x1E, 0x1F
HMP1, HMM0, HMM1, HMBL, VDELP0, VDELP1, VDELBL, RESMP0, RESMP1, HMCLR, CXCLR = (
    0x21, 0x22, 0x23, 0x24, 0x25, 0x26, 0x27, 0x28, 0x29, 0x2B, 0x2C)
FULL_TIA_REGS = VISUAL_REGS + (COLUP1, COLUP1, GRP1, GRP1, NUSIZ0, NUSIZ1, REFP0, REFP1, RESP1, RESM0,
                               RESM1, RESBL, ENAM0, ENAM1, ENABL, ENABL, HMP1, HMM0, HMM1, HMBL, VDELP0,
                               VDELP1, VDELBL, RESMP0, RESMP1, HMCLR, CXCLR)
VBLANK_TIMER = 43    # x64 cycles
OVERSCAN_TIMER = 35


class _Gen:
    """Random instruction templates over an assembler."""

    def __init__(self, rng: SplitMix64, asm: Asm):
        self.r = rng
        self.a = asm
        self.full_tia = _FULL_TIA[0]   # store to every TIA object register, read the collision latches
        self.subs = []          # (label, budget cycles of body + RTS)
        self.ptrs = []          # (pointer label, target label) for JMP (ind)
        self.n_lbl = 0
        self.allow_brk = True
        self.cram = False       # Superchip cart: also read and write its RAM

    def lbl(self, prefix="L"):
        self.n_lbl += 1
        return f"_{prefix}{self.n_lbl}"

    def work_cell(self):
        return self.r.range(WORK_LO, WORK_HI)

    def read_src(self, mnem: str, allow_io=True):
        """Emit a read-class instruction `mnem` from a random source."""
        r, a = self.r, self.a
        mode = r.pick([m for m in _ALU_MODES if (mnem, m) in _OPS])
        if mode == "imm":
            a.op(mnem, "imm", r.below(256))
        elif mode == "zp":
            if allow_io and self.full_tia and r.chance(0.15):
                a.op(mnem, "zp", r.below(8))        # a collision latch register
            elif allow_io and r.chance(0.1):
                a.op(mnem, "zp", r.pick((INPT4, INPT5, 0x00, 0x03)))
            else:
                a.op(mnem, "zp", r.range(0x80, 0xFF))
        elif mode in ("zpx", "zpy"):
            a.op(mnem, mode, r.range(0x80, 0xFF))
        elif mode == "abs":
            c = r.below(10)
            if self.cram and r.chance(0.3):
                a.op(mnem, "abs", SC_READ + r.below(128))
            elif c < 4:
                a.op(mnem, "abs", r.range(0x0080, 0x00FF))
            elif c < 7 or not allow_io:
                a.op(mnem, "abs", ("TABLE", r.below(TABLE_LEN)))
            else:
                a.op(mnem, "abs", r.pick((SWCHA, SWCHB, INTIM, TIMINT, INPT4)))
        elif mode in ("absx", "absy"):
            if self.cram and r.chance(0.3):
                a.op(mnem, mode, SC_READ + r.below(128))
            elif r.chance(0.5):
                a.op(mnem, mode, ("TABLE", r.below(64)))
            else:
                a.op(mnem, mode, r.range(0x0080, 0x00FF))
        elif mode == "indx":
            z = r.below(256)
            a.op("LDX", "imm", (r.pick((RAM_PTR, ROM_PTR)) - z) & 0xFF)
            a.op(mnem, "indx", z)
        else:
            a.op(mnem, "indy", r.pick((RAM_PTR, ROM_PTR)))

    def store(self, mnem: str):
        """Emit a store of the register named by `mnem` into the work area."""
        r, a = self.r, self.a
        reg = mnem[2]
        if self.cram and r.chance(0.3):   # into the Superchip's RAM (write port)
            j = r.below(128)
            if reg == "A" and r.chance(0.5):
                k = r.below(j + 1)
                ix = r.pick(("X", "Y"))
                a.op("LD" + ix, "imm", k)
                a.op(mnem, "abs" + ix.lower(), SC_WRITE + j - k)
            else:
                a.op(mnem, "abs", SC_WRITE + j)
            return
        choices = ["zp", "abs"] + {"A": ["zpx", "absx", "absy", "indx", "indy"],
                                   "X": ["zpy"], "Y": ["zpx"]}[reg]
        mode = r.pick(choices)
        t = self.work_cell()
        if mode in ("zp", "abs"):
            a.op(mnem, mode, t)
        elif mode in ("zpx", "absx"):
            k = r.below(t - WORK_LO + 1)
            a.op("LDX", "imm", k)
            a.op(mnem, mode, t - k)
        elif mode in ("zpy", "absy"):
            k = r.below(t - WORK_LO + 1)
            a.op("LDY", "imm", k)
            a.op(mnem, mode, t - k)
        elif mode == "indx":
            z = r.below(256)
            a.op("LDX", "imm", (RAM_PTR - z) & 0xFF)
            a.op(mnem, "indx", z)
        else:
            a.op("LDY", "imm", r.below(WORK_HI - RAM_PTR_TARGET + 1))
            a.op(mnem, "indy", RAM_PTR)

    def rmw(self):
        r, a = self.r, self.a
        m = r.pick(("ASL", "ROL", "LSR", "ROR", "INC", "DEC"))
        mode = r.pick(("zp", "zpx", "abs", "absx"))
        t = self.work_cell()
        if mode in ("zpx", "absx"):
            k = r.below(t - WORK_LO + 1)
            a.op("LDX", "imm", k)
            a.op(m, mode, t - k)
        else:
            a.op(m, mode, t)

    def simple(self):
        """One instruction (or a short fixed group) with no control flow."""
        r, a = self.r, self.a
        c = r.below(100)
        if c < 22:
            self.read_src(r.pick(("LDA", "LDA", "LDX", "LDY")))
        elif c < 44:
            self.read_src(r.pick(("ADC", "SBC", "AND", "ORA", "EOR", "CMP")))
        elif c < 58:
            self.store(r.pick(("STA", "STA", "STX", "STY")))
        elif c < 66:
            self.rmw()
        elif c < 72:
            a.op(r.pick(("ASL", "ROL", "LSR", "ROR")), "acc")
        elif c < 84:
            a.op(r.pick(("INX", "INY", "DEX", "DEY", "TAX", "TAY", "TXA", "TYA", "TSX",
                         "NOP", "CLC", "SEC", "CLV", "CLI", "SEI")))
        elif c < 88:
            m = r.pick(("CPX", "CPY"))
            mode = r.pick(("imm", "zp", "abs"))
            a.op(m, mode, r.below(256) if mode == "imm" else r.range(0x80, 0xFF))
        elif c < 91:
            a.op("BIT", r.pick(("zp", "abs")), r.range(0x80, 0xFF))
        elif c < 95:
            reg = r.pick("AXY")
            a.op("LD" + reg, "abs", r.pick((SWCHA, INTIM, INPT4, SWCHA, SWCHB)))
            self.store("ST" + reg)
        else:
            a.op(r.pick(("STA", "STX", "STY")), "zp",
                 r.pick((COLUBK, COLUP0, COLUPF, PF1, GRP0, HMP0)))

    def decimal_block(self):
        r, a = self.r, self.a
        a.op("SED")
        for _ in range(r.range(1, 2)):
            a.op(r.pick(("CLC", "SEC")))
            self.read_src("LDA", allow_io=False)
            self.read_src(r.pick(("ADC", "SBC")), allow_io=False)
            self.store("STA")
        a.op("CLD")

    def branch_block(self):
        r, a = self.r, self.a
        skip = self.lbl("B")
        if r.chance(0.3):
            if r.chance(0.5):        # branch on a joystick direction
                a.op("LDA", "abs", SWCHA)
                a.op("AND", "imm", 0x10 << r.below(4))
                a.op(r.pick(("BEQ", "BNE")), "rel", skip)
            else:                    # branch on the fire button
                a.op("BIT", "zp", INPT4)
                a.op(r.pick(("BMI", "BPL")), "rel", skip)
        else:
            a.op(r.pick(("BPL", "BMI", "BVC", "BVS", "BCC", "BCS", "BNE", "BEQ")), "rel", skip)
        for _ in range(r.range(1, 3)):
            self.simple()
        a.label(skip)

    def stack_block(self):
        r, a = self.r, self.a
        push, pull = ("PHA", "PLA") if r.chance(0.5) else ("PHP", "PLP")
        a.op(push)
        for _ in range(r.range(1, 2)):
            self.simple()
        a.op(pull)

    def jump_block(self):
        r, a = self.r, self.a
        over = self.lbl("J")
        c = r.below(3)
        if c == 0:
            a.op("JMP", "abs", over)
            for _ in range(r.range(0, 3)):
                a.byte(r.below(256))
        elif c == 1:
            ptr = self.lbl("P")
            a.op("JMP", "ind", ptr)
            self.ptrs.append((ptr, over))
            for _ in range(r.range(0, 2)):
                a.byte(r.below(256))
        elif self.allow_brk:
            a.op("BRK")
            a.byte(r.below(256))
            a.cycles += 6      # the handler's RTI
        a.label(over)

    def call_block(self):
        if not self.subs:
            self.simple()
            return
        name, cyc = self.r.pick(self.subs)
        self.a.op("JSR", "abs", name)
        self.a.cycles += cyc

    def random_work(self, max_cycles: int):
        """Random straight-line work whose budget stays within max_cycles."""
        a, r = self.a, self.r
        start = a.cycles
        while a.cycles - start < max_cycles - 100:
            c = r.below(100)
            if c < 62:
                self.simple()
            elif c < 70:
                self.decimal_block()
            elif c < 80:
                self.branch_block()
            elif c < 86:
                self.stack_block()
            elif c < 92:
                self.call_block()
            else:
                self.jump_block()

    def emit_subs(self, n: int):
        a = self.a
        for i in range(n):
            name = f"_SUB{i}"
            a.label(name)
            c0 = a.cycles
            for _ in range(self.r.range(2, 5)):
                self.simple()
            a.op("RTS")
            self.subs.append((name, a.cycles - c0))
            a.cycles = c0

    def emit_ptrs(self):
        for ptr, target in self.ptrs:
            if (self.a.pc & 0xFF) == 0xFF:     # keep pointers off a page end
                self.a.byte(0xEA)
            self.a.label(ptr)
            self.a.word(target)
        self.ptrs = []

    def line_block(self, budget: int):
        """One visible scanline: STA WSYNC, then a prep block and 1-4 stores
        to colour / playfield / player registers, within `budget` cycles."""
        r, a = self.r, self.a
        a.op("STA", "zp", WSYNC)
        a.cycles = 0
        if r.chance(0.15):
            a.op("STA", "zp", HMOVE)
        n_store = r.range(1, 4)
        reserve = 4 * n_store
        while a.cycles + reserve + 8 <= budget and not r.chance(0.3):
            c = r.below(10)
            if c < 5:
                m = r.pick(("LDA", "LDX", "LDY"))
                if m == "LDA":
                    self.read_src("LDA", allow_io=False)
                elif r.chance(0.5):
                    a.op(m, "imm", r.below(256))
                else:
                    a.op(m, "zp", r.range(0x80, 0xFF))
            elif c < 8:
                m = r.pick(("ADC", "EOR", "AND", "ORA"))
                if r.chance(0.5):
                    a.op(m, "imm", r.below(256))
                else:
                    a.op(m, "zp", r.range(0x80, 0xFF))
            else:
                a.op(r.pick(("INX", "DEX", "INY", "DEY", "NOP", "TXA", "TAY")))
        for _ in range(n_store):
            if r.chance(0.2) and a.cycles + 6 <= budget:
                a.op("NOP")
            if a.cycles + 3 > budget:
                break
            a.op(r.pick(("STA", "STA", "STX", "STY")), "zp", r.pick(FULL_TIA_REGS if self.full_tia else VISUAL_REGS))
        assert a.cycles <= budget


def _emit_kernel(a: Asm, g: _Gen, n_lines: int, exit_label: str):
    a.op("LDA", "imm", 192 // n_lines)
    a.op("STA", "zp", LINE_CTR)
    a.label("KTOP")
    for i in range(n_lines):
        # next STA WSYNC writes 3 cycles in; the last block also pays
        # DEC zp (5) + BEQ (<= 4) + JMP (3)
        g.line_block(73 - (12 if i == n_lines - 1 else 0))
    a.op("DEC", "zp", LINE_CTR)
    a.op("BEQ", "rel", "KDONE")
    a.op("JMP", "abs", "KTOP")
    a.label("KDONE")
    a.op("JMP", "abs", exit_label)


def _emit_table(a: Asm, r: SplitMix64):
    a.label("TABLE")
    for _ in range(TABLE_LEN):
        a.byte(r.below(256))


def generate_cart(seed: int, cart: int, mapper: int, full_tia: bool = False) -> bytes:
    """Seed -> ROM image (2048, 4096, 8192, 16384 or 32768 bytes) of a well-formed frame loop.

    Layout: reset vector -> init (SEI, CLD, stack, RAM clear, pointers) ->
    frame loop: VSYNC for 3 lines; TIM64T=43 and random work over RAM,
    inputs and the timer during VBLANK, ending on an INTIM poll; 192 visible
    lines of WSYNC + random block + stores to colour / playfield / player
    registers; overscan with TIM64T=35 and more work; JMP back.  F8 images
    place the visible kernel in bank 0 and switch banks through trampolines
    at the same offsets in both banks.  Superchip variants (F8SC, F6SC,
    F4SC) are the banked images with their code moved past the cartridge
    RAM ports ($1000-$10FF) and random reads and stores of that RAM.
    full_tia: the scanline stores also reach player 1, the missiles, the
    ball and their size / motion / delay / lock registers and CXCLR, and
    the random work also reads the collision latches (into RAM).
    """
    _FULL_TIA[0] = full_tia
    try:
        return _generate_cart(seed, cart, mapper)
    finally:
        _FULL_TIA[0] = False


_FULL_TIA = [False]


def _generate_cart(seed: int, cart: int, mapper: int) -> bytes:
    if mapper == MAPPER_E0:
        return _generate_e0(seed, cart)
    if mapper == MAPPER_FE:
        return _generate_fe(seed, cart)
    sc = mapper in MAPPER_SC_BASE
    mapper = MAPPER_SC_BASE.get(mapper, mapper)
    if mapper in (MAPPER_F6, MAPPER_F4):
        return _generate_multibank(seed, cart, mapper, sc)
    r = SplitMix64(seed, cart, 0x0CA7)
    origin = 0xF800 if mapper == MAPPER_2K else 0xF000
    bank_size = 2048 if mapper == MAPPER_2K else 4096
    n_lines = 8 if mapper == MAPPER_2K else 16
    vb_budget, vb_loops = (650, 3) if mapper == MAPPER_2K else (1000, 2)
    os_budget = 350 if mapper == MAPPER_2K else 900
    tramp = bank_size - 0x40          # F8 trampolines (both banks)
    stub = bank_size - 0x30           # F8 bank-0 reset stub
    irq = bank_size - 0x20            # BRK handler (both banks)

    a = Asm(origin, bank_size)
    g = _Gen(r, a)
    if sc:   # the Superchip's RAM ports hide the first 256 bytes of each bank
        a.at(0x100)
        g.cram = True
    # leaf subroutines first: only reachable through JSR
    g.emit_subs(4)
    a.label("RESET")
    a.op("SEI")
    a.op("CLD")
    a.op("LDX", "imm", 0xFF)
    a.op("TXS")
    a.op("LDA", "imm", 0)
    a.op("LDX", "imm", 0x7F)
    a.label("CLR")
    a.op("STA", "zpx", 0x80)
    a.op("DEX")
    a.op("BPL", "rel", "CLR")
    a.op("LDA", "imm", RAM_PTR_TARGET & 0xFF)
    a.op("STA", "zp", RAM_PTR)
    a.op("LDA", "imm", RAM_PTR_TARGET >> 8)
    a.op("STA", "zp", RAM_PTR + 1)
    a.op("LDA", "imm", ("<", "TABLE"))
    a.op("STA", "zp", ROM_PTR)
    a.op("LDA", "imm", (">", "TABLE"))
    a.op("STA", "zp", ROM_PTR + 1)
    for _ in range(r.range(4, 10)):
        a.op("LDA", "imm", r.below(256))
        a.op("STA", "zp", g.work_cell())
    for reg in (COLUP0, COLUPF, COLUBK):
        a.op("LDA", "imm", r.below(256))
        a.op("STA", "zp", reg)
    a.op("LDA", "imm", r.pick((0, 1, 4, 5)))
    a.op("STA", "zp", CTRLPF)
    # frame loop
    a.label("FRAME")
    a.op("LDA", "imm", 2)
    a.op("STA", "zp", VBLANK)
    a.op("STA", "zp", WSYNC)
    a.op("STA", "zp", VSYNC)
    for _ in range(3):
        a.op("STA", "zp", WSYNC)
    a.op("LDA", "imm", 0)
    a.op("STA", "zp", VSYNC)
    a.op("LDA", "imm", VBLANK_TIMER)
    a.op("STA", "abs", TIM64T)
    a.op("LDA", "imm", vb_loops)
    a.op("STA", "zp", WORK_CTR)
    a.label("VBL")
    a.op("JSR", "abs", "VBWORK")
    a.op("DEC", "zp", WORK_CTR)
    a.op("BNE", "rel", "VBL")
    a.label("VBWAIT")
    a.op("LDA", "abs", INTIM)
    a.op("BNE", "rel", "VBWAIT")
    a.op("STA", "zp", WSYNC)
    a.op("LDA", "imm", 0)
    a.op("STA", "zp", VBLANK)
    a.op("JMP", "abs", "TRAMP" if mapper == MAPPER_F8 else "KERNEL")
    a.label("OVERSCAN")
    a.op("STA", "zp", WSYNC)
    a.op("LDA", "imm", 2)
    a.op("STA", "zp", VBLANK)
    a.op("LDA", "imm", OVERSCAN_TIMER)
    a.op("STA", "abs", TIM64T)
    a.cycles = 0
    g.random_work(os_budget)
    a.label("OSWAIT")
    a.op("LDA", "abs", INTIM)
    a.op("BNE", "rel", "OSWAIT")
    a.op("JMP", "abs", "FRAME")
    a.label("VBWORK")
    a.cycles = 0
    g.random_work(vb_budget)
    a.op("RTS")
    g.emit_ptrs()
    if mapper != MAPPER_F8:
        a.label("KERNEL")
        _emit_kernel(a, g, n_lines, "OVERSCAN")
    _emit_table(a, r)
    if mapper == MAPPER_F8:
        # bank 1: [tramp] BIT $1FF8 -> bank 0 continues at tramp+3;
        # bank 0 returns through BIT $1FF9 at tramp+6 -> bank 1 resumes at tramp+9.
        a.at(tramp)
        a.label("TRAMP")
        a.op("BIT", "abs", 0x1FF8)
        a.at(tramp + 9)
        a.op("JMP", "abs", "OVERSCAN")
        # bank 0's reset stub at `stub` switches to bank 1, which resumes at stub+3.
        a.at(stub + 3)
        a.op("JMP", "abs", "RESET")
    a.at(irq)
    a.label("IRQ")
    a.op("RTI")
    a.at(bank_size - 6)
    a.word("IRQ")        # NMI
    a.word("RESET")
    a.word("IRQ")        # IRQ / BRK
    bank1 = a.resolve()
    if mapper != MAPPER_F8:
        return bytes(bank1)

    b = Asm(origin, bank_size)
    g0 = _Gen(SplitMix64(seed, cart, 0x0CA8), b)
    if sc:
        b.at(0x100)
        g0.cram = True
    b.label("KERNEL0")
    _emit_kernel(b, g0, n_lines, "TRAMP0")
    _emit_table(b, g0.r)
    b.at(tramp + 3)
    b.op("JMP", "abs", "KERNEL0")
    b.label("TRAMP0")
    b.op("BIT", "abs", 0x1FF9)
    b.at(stub)
    b.label("STUB")
    b.op("BIT", "abs", 0x1FF9)
    b.at(irq)
    b.label("IRQ")
    b.op("RTI")
    b.at(bank_size - 6)
    b.word("IRQ")
    b.word("STUB")
    b.word("IRQ")
    bank0 = b.resolve()
    return bytes(bank0) + bytes(bank1)


def _generate_multibank(seed: int, cart: int, mapper: int, sc: bool = False) -> bytes:
    """F6 / F4 images: the last bank (where the machine powers on) holds the
    init, VBLANK and overscan code; each other bank k holds its own visible
    kernel.  Every frame the main bank picks a kernel bank from the
    joystick's high nibble and a work cell (low bits; the values past the
    last kernel bank pick bank 0) and enters it through a
    trampoline: BIT of hotspot k at offset tramp + 3k, bank k continuing at
    tramp + 3k + 3 with a JMP to its kernel; bank k returns with BIT of the
    main bank's hotspot at ret + 3k, the main bank continuing at ret + 3k + 3
    with a JMP to the overscan.  Superchip images (sc) start their code past
    the RAM ports' 256 bytes and use the cartridge RAM."""
    nb, hot = MAPPER_BANKS[mapper], MAPPER_HOTSPOT[mapper]
    main = nb - 1
    bank_size, origin = 4096, 0xF000
    tramp, ret, stub, irq = bank_size - 0x80, bank_size - 0x60, bank_size - 0x30, bank_size - 0x20
    r = SplitMix64(seed, cart, 0x0CA7)
    n_lines, vb_budget, vb_loops, os_budget = 16, 1000, 2, 900
    a = Asm(origin, bank_size)
    g = _Gen(r, a)
    if sc:
        a.at(0x100)
        g.cram = True
    g.emit_subs(4)
    a.label("RESET")
    a.op("SEI")
    a.op("CLD")
    a.op("LDX", "imm", 0xFF)
    a.op("TXS")
    a.op("LDA", "imm", 0)
    a.op("LDX", "imm", 0x7F)
    a.label("CLR")
    a.op("STA", "zpx", 0x80)
    a.op("DEX")
    a.op("BPL", "rel", "CLR")
    a.op("LDA", "imm", RAM_PTR_TARGET & 0xFF)
    a.op("STA", "zp", RAM_PTR)
    a.op("LDA", "imm", RAM_PTR_TARGET >> 8)
    a.op("STA", "zp", RAM_PTR + 1)
    a.op("LDA", "imm", ("<", "TABLE"))
    a.op("STA", "zp", ROM_PTR)
    a.op("LDA", "imm", (">", "TABLE"))
    a.op("STA", "zp", ROM_PTR + 1)
    for _ in range(r.range(4, 10)):
        a.op("LDA", "imm", r.below(256))
        a.op("STA", "zp", g.work_cell())
    for reg in (COLUP0, COLUPF, COLUBK):
        a.op("LDA", "imm", r.below(256))
        a.op("STA", "zp", reg)
    a.op("LDA", "imm", r.pick((0, 1, 4, 5)))
    a.op("STA", "zp", CTRLPF)
    a.label("FRAME")
    a.op("LDA", "imm", 2)
    a.op("STA", "zp", VBLANK)
    a.op("STA", "zp", WSYNC)
    a.op("STA", "zp", VSYNC)
    for _ in range(3):
        a.op("STA", "zp", WSYNC)
    a.op("LDA", "imm", 0)
    a.op("STA", "zp", VSYNC)
    a.op("LDA", "imm", VBLANK_TIMER)
    a.op("STA", "abs", TIM64T)
    a.op("LDA", "imm", vb_loops)
    a.op("STA", "zp", WORK_CTR)
    a.label("VBL")
    a.op("JSR", "abs", "VBWORK")
    a.op("DEC", "zp", WORK_CTR)
    a.op("BNE", "rel", "VBL")
    a.label("VBWAIT")
    a.op("LDA", "abs", INTIM)
    a.op("BNE", "rel", "VBWAIT")
    a.op("STA", "zp", WSYNC)
    a.op("LDA", "imm", 0)
    a.op("STA", "zp", VBLANK)
    # pick this frame's kernel bank from the joystick and a work cell
    a.op("LDA", "abs", SWCHA)
    for _ in range(4):
        a.op("LSR", "acc")
    a.op("EOR", "zp", WORK_LO)
    a.op("AND", "imm", 7 if nb == 8 else 3)
    for k in range(1, nb - 1):
        a.op("CMP", "imm", k)
        a.op("BNE", "rel", f"SEL{k}")
        a.op("JMP", "abs", origin + tramp + 3 * k)
        a.label(f"SEL{k}")
    a.op("JMP", "abs", origin + tramp)
    a.label("OVERSCAN")
    a.op("STA", "zp", WSYNC)
    a.op("LDA", "imm", 2)
    a.op("STA", "zp", VBLANK)
    a.op("LDA", "imm", OVERSCAN_TIMER)
    a.op("STA", "abs", TIM64T)
    a.cycles = 0
    g.random_work(os_budget)
    a.label("OSWAIT")
    a.op("LDA", "abs", INTIM)
    a.op("BNE", "rel", "OSWAIT")
    a.op("JMP", "abs", "FRAME")
    a.label("VBWORK")
    a.cycles = 0
    g.random_work(vb_budget)
    a.op("RTS")
    g.emit_ptrs()
    _emit_table(a, r)
    for k in range(nb - 1):
        a.at(tramp + 3 * k)
        a.op("BIT", "abs", hot + k)
    for k in range(nb - 1):
        a.at(ret + 3 * k + 3)
        a.op("JMP", "abs", "OVERSCAN")
    a.at(stub + 3)
    a.op("JMP", "abs", "RESET")
    a.at(irq)
    a.label("IRQ")
    a.op("RTI")
    a.at(bank_size - 6)
    a.word("IRQ")
    a.word("RESET")
    a.word("IRQ")
    banks = {main: bytes(a.resolve())}
    for k in range(nb - 1):
        b = Asm(origin, bank_size)
        gk = _Gen(SplitMix64(seed, cart, 0x0CA8 + k), b)
        if sc:
            b.at(0x100)
            gk.cram = True
        b.label("KERNEL")
        _emit_kernel(b, gk, n_lines, "RET")
        _emit_table(b, gk.r)
        b.at(tramp + 3 * k + 3)
        b.op("JMP", "abs", "KERNEL")
        b.at(ret + 3 * k)
        b.label("RET")
        b.op("BIT", "abs", hot + main)
        b.at(stub)
        b.label("STUB")
        b.op("BIT", "abs", hot + main)
        b.at(irq)
        b.label("IRQ")
        b.op("RTI")
        b.at(bank_size - 6)
        b.word("IRQ")
        b.word("STUB")
        b.word("IRQ")
        banks[k] = bytes(b.resolve())
    return b"".join(banks[k] for k in range(nb))


def _generate_fe(seed: int, cart: int) -> bytes:
    """FE image: bank 0 (the image's first 4 KB, addressed $F000-$FFFF,
    shown at power-on) holds the init, the frame loop, the VBLANK and
    overscan work and one visible kernel; bank 1 (addressed $D000-$DFFF)
    holds another visible kernel.  Each frame the loop, at the top of the
    stack, calls one of the two kernels as a subroutine, picked from the
    joystick and a work cell: JSR $D000 switches to bank 1 (the target's
    high byte has bit 5 clear), and the kernel's RTS switches back (the
    return address's high byte, $Fx, has it set); JSR to the bank-0 kernel
    keeps bank 0.  The random work's own subroutine calls run deeper in the
    stack and switch nothing."""
    r = SplitMix64(seed, cart, 0x0CA7)
    n_lines, vb_budget, vb_loops, os_budget = 16, 1000, 2, 900
    bank_size, irq = 4096, 4096 - 0x20
    a = Asm(0xF000, bank_size)
    g = _Gen(r, a)
    g.emit_subs(4)
    a.label("RESET")
    a.op("SEI")
    a.op("CLD")
    a.op("LDX", "imm", 0xFF)
    a.op("TXS")
    a.op("LDA", "imm", 0)
    a.op("LDX", "imm", 0x7F)
    a.label("CLR")
    a.op("STA", "zpx", 0x80)
    a.op("DEX")
    a.op("BPL", "rel", "CLR")
    a.op("LDA", "imm", RAM_PTR_TARGET & 0xFF)
    a.op("STA", "zp", RAM_PTR)
    a.op("LDA", "imm", RAM_PTR_TARGET >> 8)
    a.op("STA", "zp", RAM_PTR + 1)
    a.op("LDA", "imm", ("<", "TABLE"))
    a.op("STA", "zp", ROM_PTR)
    a.op("LDA", "imm", (">", "TABLE"))
    a.op("STA", "zp", ROM_PTR + 1)
    for _ in range(r.range(4, 10)):
        a.op("LDA", "imm", r.below(256))
        a.op("STA", "zp", g.work_cell())
    for reg in (COLUP0, COLUPF, COLUBK):
        a.op("LDA", "imm", r.below(256))
        a.op("STA", "zp", reg)
    a.op("LDA", "imm", r.pick((0, 1, 4, 5)))
    a.op("STA", "zp", CTRLPF)
    a.label("FRAME")
    a.op("LDA", "imm", 2)
    a.op("STA", "zp", VBLANK)
    a.op("STA", "zp", WSYNC)
    a.op("STA", "zp", VSYNC)
    for _ in range(3):
        a.op("STA", "zp", WSYNC)
    a.op("LDA", "imm", 0)
    a.op("STA", "zp", VSYNC)
    a.op("LDA", "imm", VBLANK_TIMER)
    a.op("STA", "abs", TIM64T)
    a.op("LDA", "imm", vb_loops)
    a.op("STA", "zp", WORK_CTR)
    a.label("VBL")
    a.op("JSR", "abs", "VBWORK")
    a.op("DEC", "zp", WORK_CTR)
    a.op("BNE", "rel", "VBL")
    a.label("VBWAIT")
    a.op("LDA", "abs", INTIM)
    a.op("BNE", "rel", "VBWAIT")
    a.op("STA", "zp", WSYNC)
    a.op("LDA", "imm", 0)
    a.op("STA", "zp", VBLANK)
    # this frame's kernel: bank 1's (through the FE switch) or bank 0's
    a.op("LDA", "abs", SWCHA)
    a.op("EOR", "zp", WORK_LO)
    a.op("AND", "imm", 0x30)
    a.op("BEQ", "rel", "KF")
    a.op("JSR", "abs", 0xD000)
    a.op("JMP", "abs", "OVERSCAN")
    a.label("KF")
    a.op("JSR", "abs", "KERNEL")
    a.label("OVERSCAN")
    a.op("STA", "zp", WSYNC)
    a.op("LDA", "imm", 2)
    a.op("STA", "zp", VBLANK)
    a.op("LDA", "imm", OVERSCAN_TIMER)
    a.op("STA", "abs", TIM64T)
    a.cycles = 0
    g.random_work(os_budget)
    a.label("OSWAIT")
    a.op("LDA", "abs", INTIM)
    a.op("BNE", "rel", "OSWAIT")
    a.op("JMP", "abs", "FRAME")
    a.label("VBWORK")
    a.cycles = 0
    g.random_work(vb_budget)
    a.op("RTS")
    g.emit_ptrs()
    a.label("KERNEL")
    _emit_kernel(a, g, n_lines, "KRET")
    a.label("KRET")
    a.op("RTS")
    _emit_table(a, r)
    a.at(irq)
    a.label("IRQ")
    a.op("RTI")
    a.at(bank_size - 6)
    a.word("IRQ")
    a.word("RESET")
    a.word("IRQ")
    bank0 = bytes(a.resolve())

    b = Asm(0xD000, bank_size)
    g1 = _Gen(SplitMix64(seed, cart, 0x0CA8), b)
    b.label("KERNEL1")
    _emit_kernel(b, g1, n_lines, "KRET1")
    b.label("KRET1")
    b.op("RTS")
    _emit_table(b, g1.r)
    b.at(irq)
    b.label("IRQ")
    b.op("RTI")
    b.at(bank_size - 6)
    b.word("IRQ")
    b.word("IRQ")
    b.word("IRQ")
    return bank0 + bytes(b.resolve())


def _generate_e0(seed: int, cart: int) -> bytes:
    """E0 image: slice 7 (segment 3, $FC00, always mapped) holds a table,
    the init, the frame loop and the leaf subroutines; each frame the loop
    maps a VBLANK-work slice (0 or 1) into segment 0, a visible-kernel slice
    (2, 3 or 4) into segment 1 and an overscan-work slice (5 or 6) into
    segment 2, picked from the joystick and a work cell, and calls or jumps
    there.  Every slice is assembled for the segment it is mapped into; the
    shared table, subroutines and BRK handler are addressed in slice 7."""
    r = SplitMix64(seed, cart, 0x0CE0)
    n_lines, vb_budget, vb_loops, os_budget = 12, 1000, 2, 900
    seg_base = (0xF000, 0xF400, 0xF800, 0xFC00)
    a = Asm(seg_base[3], 1024)
    g = _Gen(r, a)
    _emit_table(a, r)                       # $FC00..: reads of TABLE + 319 stay below the hotspots
    g.emit_subs(3)
    a.label("RESET")
    a.op("SEI")
    a.op("CLD")
    a.op("LDX", "imm", 0xFF)
    a.op("TXS")
    a.op("LDA", "imm", 0)
    a.op("LDX", "imm", 0x7F)
    a.label("CLR")
    a.op("STA", "zpx", 0x80)
    a.op("DEX")
    a.op("BPL", "rel", "CLR")
    a.op("LDA", "imm", RAM_PTR_TARGET & 0xFF)
    a.op("STA", "zp", RAM_PTR)
    a.op("LDA", "imm", RAM_PTR_TARGET >> 8)
    a.op("STA", "zp", RAM_PTR + 1)
    a.op("LDA", "imm", ("<", "TABLE"))
    a.op("STA", "zp", ROM_PTR)
    a.op("LDA", "imm", (">", "TABLE"))
    a.op("STA", "zp", ROM_PTR + 1)
    for _ in range(r.range(4, 10)):
        a.op("LDA", "imm", r.below(256))
        a.op("STA", "zp", g.work_cell())
    for reg in (COLUP0, COLUPF, COLUBK):
        a.op("LDA", "imm", r.below(256))
        a.op("STA", "zp", reg)
    a.op("LDA", "imm", r.pick((0, 1, 4, 5)))
    a.op("STA", "zp", CTRLPF)
    a.label("FRAME")
    a.op("LDA", "imm", 2)
    a.op("STA", "zp", VBLANK)
    a.op("STA", "zp", WSYNC)
    a.op("STA", "zp", VSYNC)
    for _ in range(3):
        a.op("STA", "zp", WSYNC)
    a.op("LDA", "imm", 0)
    a.op("STA", "zp", VSYNC)
    a.op("LDA", "imm", VBLANK_TIMER)
    a.op("STA", "abs", TIM64T)
    # segment 0 <- slice 0 or 1 (joystick up)
    a.op("LDA", "abs", SWCHA)
    a.op("AND", "imm", 0x10)
    a.op("BEQ", "rel", "V1")
    a.op("LDA", "abs", E0_HOTSPOT[0] + 0)
    a.op("JMP", "abs", "VGO")
    a.label("V1")
    a.op("LDA", "abs", E0_HOTSPOT[0] + 1)
    a.label("VGO")
    a.op("LDA", "imm", vb_loops)
    a.op("STA", "zp", WORK_CTR)
    a.label("VBL")
    a.op("JSR", "abs", seg_base[0])
    a.op("DEC", "zp", WORK_CTR)
    a.op("BNE", "rel", "VBL")
    a.label("VBWAIT")
    a.op("LDA", "abs", INTIM)
    a.op("BNE", "rel", "VBWAIT")
    a.op("STA", "zp", WSYNC)
    a.op("LDA", "imm", 0)
    a.op("STA", "zp", VBLANK)
    # segment 1 <- slice 2, 3 or 4 (joystick high nibble ^ a work cell, mod 4; 0 and 3 pick slice 2)
    a.op("LDA", "abs", SWCHA)
    for _ in range(4):
        a.op("LSR", "acc")
    a.op("EOR", "zp", WORK_LO)
    a.op("AND", "imm", 3)
    a.op("CMP", "imm", 1)
    a.op("BNE", "rel", "K2")
    a.op("LDA", "abs", E0_HOTSPOT[1] + 3)
    a.op("JMP", "abs", seg_base[1])
    a.label("K2")
    a.op("CMP", "imm", 2)
    a.op("BNE", "rel", "K0")
    a.op("LDA", "abs", E0_HOTSPOT[1] + 4)
    a.op("JMP", "abs", seg_base[1])
    a.label("K0")
    a.op("LDA", "abs", E0_HOTSPOT[1] + 2)
    a.op("JMP", "abs", seg_base[1])
    a.label("KEXIT")                        # the kernels end here
    a.op("STA", "zp", WSYNC)
    a.op("LDA", "imm", 2)
    a.op("STA", "zp", VBLANK)
    a.op("LDA", "imm", OVERSCAN_TIMER)
    a.op("STA", "abs", TIM64T)
    # segment 2 <- slice 5 or 6 (a work cell's low bit)
    a.op("LDA", "zp", WORK_LO)
    a.op("LSR", "acc")
    a.op("BCC", "rel", "O5")
    a.op("LDA", "abs", E0_HOTSPOT[2] + 6)
    a.op("JMP", "abs", "OGO")
    a.label("O5")
    a.op("LDA", "abs", E0_HOTSPOT[2] + 5)
    a.label("OGO")
    a.op("JSR", "abs", seg_base[2])
    a.label("OSWAIT")
    a.op("LDA", "abs", INTIM)
    a.op("BNE", "rel", "OSWAIT")
    a.op("JMP", "abs", "FRAME")
    a.label("IRQ")
    a.op("RTI")
    a.at(0x3E0)                             # the hotspots $1FE0-$1FF7 hold no code
    a.at(1024 - 6)
    a.word("IRQ")
    a.word("RESET")
    a.word("IRQ")
    slices = {7: bytes(a.resolve())}
    shared = {name: a.labels[name] for name in ("TABLE", "IRQ", "KEXIT")}
    shared.update({name: a.labels[name] for name, _ in g.subs})
    for k in range(7):
        seg = 0 if k < 2 else (1 if k < 5 else 2)
        b = Asm(seg_base[seg], 1024)
        gk = _Gen(SplitMix64(seed, cart, 0x0CE8 + k), b)
        b.labels.update(shared)
        gk.subs = list(g.subs)
        if seg == 1:
            _emit_kernel(b, gk, n_lines, "KEXIT")
        else:
            b.cycles = 0
            gk.random_work(vb_budget if seg == 0 else os_budget)
            b.op("RTS")
        gk.emit_ptrs()
        slices[k] = bytes(b.resolve())
    return b"".join(slices[k] for k in range(8))


def config_carts(seed: int, mappers, full_tia: bool = False) -> list:
    """ROM images for a list of mappers, cart index = position."""
    return [generate_cart(seed, i, m, full_tia) for i, m in enumerate(mappers)]


MIX16 = [MAPPER_2K] * 6 + [MAPPER_4K] * 6 + [MAPPER_F8] * 4
MIX8 = [MAPPER_4K] * 4 + [MAPPER_F8] * 4


def env_cart_round_robin(n_envs: int, n_carts: int, sort: bool = True) -> np.ndarray:
    """Envs assigned to carts round-robin; sorted by cart when `sort`."""
    ec = np.arange(n_envs, dtype=np.int32) % n_carts
    return np.sort(ec) if sort else ec
