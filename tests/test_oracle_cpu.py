"""Pins of the oracle's 6507 core against what the chip documentation and
arithmetic fix, independently of the oracle's own code:

* exhaustive ADC/SBC over A x operand x carry x decimal, binary results
  against integer arithmetic and the signed-overflow definition, decimal
  results against decimal arithmetic for valid BCD operands and against a
  second, table-driven derivation of the NMOS decimal adjust for all others
  (the published decimal-mode note);
* the MOS 6500 instruction table: length, base cycles and the page-cross
  penalty of every documented opcode, and which status flags each changes.
"""
import numpy as np
import pytest

import oracle
from paper_2606_22447_b300 import synth
from tests.microrom import rom4k

FC, FZ, FI, FD, FB, F5, FV, FN = 1, 2, 4, 8, 16, 32, 64, 128


def _alu_rom():
    def build(a):
        a.op("ADC", "absy", 0xFE00)     # $F000
        a.at(0x10)
        a.op("SBC", "absy", 0xFE00)     # $F010
    return rom4k(build)


@pytest.fixture(scope="module")
def alu_results():
    """Run every (op, A, M, C, D) through the oracle's interpreter."""
    o = oracle.Oracle(_alu_rom(), synth.MAPPER_4K)
    out = {}
    for op, pc in (("ADC", 0xF000), ("SBC", 0xF010)):
        res = np.zeros((2, 2, 256, 256, 2), np.int32)   # d, c, a, m -> (A', P')
        for d in (0, 1):
            for c in (0, 1):
                p0 = (FD if d else 0) | (FC if c else 0)
                for a in range(256):
                    for m in range(256):
                        o.set_regs(A=a, Y=m, P=p0, PC=pc)
                        cyc = o.exec_one()
                        st = o.state()
                        res[d, c, a, m] = (st[0], st[4])
                assert cyc == 4
        out[op] = res
    return out


def _signed(x):
    return x - 256 if x >= 128 else x


def test_binary_adc_exhaustive(alu_results):
    r = alu_results["ADC"][0]
    for c in (0, 1):
        for a in range(0, 256):
            m = np.arange(256)
            t = a + m + c
            assert np.array_equal(r[c, a, :, 0], t % 256)
            p = r[c, a, :, 1]
            assert np.array_equal((p & FC) != 0, t > 255)
            sv = np.array([_signed(a) + _signed(int(x)) + c for x in m])
            assert np.array_equal((p & FV) != 0, (sv < -128) | (sv > 127))
            assert np.array_equal((p & FZ) != 0, t % 256 == 0)
            assert np.array_equal((p & FN) != 0, (t % 256) >= 128)


def test_binary_sbc_exhaustive(alu_results):
    r = alu_results["SBC"][0]
    for c in (0, 1):
        for a in range(256):
            m = np.arange(256)
            t = a - m - (1 - c)
            assert np.array_equal(r[c, a, :, 0], t % 256)
            p = r[c, a, :, 1]
            assert np.array_equal((p & FC) != 0, t >= 0)          # carry = no borrow
            sv = np.array([_signed(a) - _signed(int(x)) - (1 - c) for x in m])
            assert np.array_equal((p & FV) != 0, (sv < -128) | (sv > 127))
            assert np.array_equal((p & FZ) != 0, t % 256 == 0)


def _bcd(x):
    return (x >> 4) * 10 + (x & 15)


def _to_bcd(n):
    return ((n // 10) << 4) | (n % 10)


def test_decimal_valid_bcd_against_decimal_arithmetic(alu_results):
    valid = [v for v in range(256) if (v >> 4) < 10 and (v & 15) < 10]
    ra, rs = alu_results["ADC"][1], alu_results["SBC"][1]
    for c in (0, 1):
        for a in valid:
            for m in valid:
                s = _bcd(a) + _bcd(m) + c
                assert ra[c, a, m, 0] == _to_bcd(s % 100), (a, m, c)
                assert bool(ra[c, a, m, 1] & FC) == (s >= 100)
                d = _bcd(a) - _bcd(m) - (1 - c)
                assert rs[c, a, m, 0] == _to_bcd(d % 100), (a, m, c)
                assert bool(rs[c, a, m, 1] & FC) == (d >= 0)
                # Z follows the binary sum, N/V and SBC's flags the binary rules
                assert bool(ra[c, a, m, 1] & FZ) == ((a + m + c) % 256 == 0)
                assert bool(rs[c, a, m, 1] & FZ) == ((a - m - (1 - c)) % 256 == 0)


def _nmos_adc_table(a, m, c):
    """NMOS decimal ADC as a digit table: each nibble is corrected with a
    lookup of (digit sum -> (digit, carry)) built from the note's rule
    'a nibble result of 10 or more is adjusted by 6 and carries'; the high
    nibble is adjusted by comparing the unadjusted high sum with $A0."""
    lo_tab = {}
    for s in range(0, 32):
        lo_tab[s] = ((s + 6) & 15, 1) if s >= 10 else (s, 0)
    ld, lc = lo_tab[(a & 15) + (m & 15) + c]
    hi = (a >> 4) + (m >> 4) + lc                 # may exceed 15
    raw = (hi << 4) | ld
    n = (raw >> 7) & 1
    sh = _signed(a & 0xF0) + _signed(m & 0xF0) + (lc << 4) + ld
    v = int(sh < -128 or sh > 127)
    if raw >= 0xA0:
        raw += 0x60
    return raw & 0xFF, int(raw >= 0x100), n, v


def _nmos_sbc_table(a, m, c):
    lo = (a & 15) - (m & 15) - (1 - c)
    borrow = 0
    if lo < 0:
        lo = (lo - 6) & 15
        borrow = 1
    hi = (a >> 4) - (m >> 4) - borrow
    res = ((hi << 4) | lo)
    if hi < 0:
        res -= 0x60
    return res & 0xFF


def test_decimal_all_operands_against_table_derivation(alu_results):
    ra, rs = alu_results["ADC"][1], alu_results["SBC"][1]
    for c in (0, 1):
        for a in range(256):
            for m in range(256):
                r, cy, n, v = _nmos_adc_table(a, m, c)
                p = ra[c, a, m, 1]
                assert ra[c, a, m, 0] == r, ("ADC", a, m, c)
                assert bool(p & FC) == bool(cy)
                assert bool(p & FN) == bool(n)
                assert bool(p & FV) == bool(v)
                assert rs[c, a, m, 0] == _nmos_sbc_table(a, m, c), ("SBC", a, m, c)


# ---------------------------------------------------------------------------
# MOS instruction table: (mnemonic, mode, bytes, cycles, +1 on page cross)
# ---------------------------------------------------------------------------

def _group(m, codes, modes=("imm", "zp", "zpx", "abs", "absx", "absy", "indx", "indy")):
    timing = {"imm": (2, 2, 0), "zp": (2, 3, 0), "zpx": (2, 4, 0), "abs": (3, 4, 0),
              "absx": (3, 4, 1), "absy": (3, 4, 1), "indx": (2, 6, 0), "indy": (2, 5, 1)}
    return {c: (m, mo) + timing[mo] for c, mo in zip(codes, modes)}


MOS = {}
for _m, _codes in (("ADC", (0x69, 0x65, 0x75, 0x6D, 0x7D, 0x79, 0x61, 0x71)),
                   ("AND", (0x29, 0x25, 0x35, 0x2D, 0x3D, 0x39, 0x21, 0x31)),
                   ("CMP", (0xC9, 0xC5, 0xD5, 0xCD, 0xDD, 0xD9, 0xC1, 0xD1)),
                   ("EOR", (0x49, 0x45, 0x55, 0x4D, 0x5D, 0x59, 0x41, 0x51)),
                   ("LDA", (0xA9, 0xA5, 0xB5, 0xAD, 0xBD, 0xB9, 0xA1, 0xB1)),
                   ("ORA", (0x09, 0x05, 0x15, 0x0D, 0x1D, 0x19, 0x01, 0x11)),
                   ("SBC", (0xE9, 0xE5, 0xF5, 0xED, 0xFD, 0xF9, 0xE1, 0xF1))):
    MOS.update(_group(_m, _codes))
for _m, _b in (("ASL", 0x00), ("ROL", 0x20), ("LSR", 0x40), ("ROR", 0x60)):
    MOS.update({_b + 0x0A: (_m, "acc", 1, 2, 0), _b + 0x06: (_m, "zp", 2, 5, 0),
                _b + 0x16: (_m, "zpx", 2, 6, 0), _b + 0x0E: (_m, "abs", 3, 6, 0),
                _b + 0x1E: (_m, "absx", 3, 7, 0)})
for _m, _c in (("INC", (0xE6, 0xF6, 0xEE, 0xFE)), ("DEC", (0xC6, 0xD6, 0xCE, 0xDE))):
    MOS.update({_c[0]: (_m, "zp", 2, 5, 0), _c[1]: (_m, "zpx", 2, 6, 0),
                _c[2]: (_m, "abs", 3, 6, 0), _c[3]: (_m, "absx", 3, 7, 0)})
MOS.update({0x85: ("STA", "zp", 2, 3, 0), 0x95: ("STA", "zpx", 2, 4, 0), 0x8D: ("STA", "abs", 3, 4, 0),
            0x9D: ("STA", "absx", 3, 5, 0), 0x99: ("STA", "absy", 3, 5, 0),
            0x81: ("STA", "indx", 2, 6, 0), 0x91: ("STA", "indy", 2, 6, 0),
            0x86: ("STX", "zp", 2, 3, 0), 0x96: ("STX", "zpy", 2, 4, 0), 0x8E: ("STX", "abs", 3, 4, 0),
            0x84: ("STY", "zp", 2, 3, 0), 0x94: ("STY", "zpx", 2, 4, 0), 0x8C: ("STY", "abs", 3, 4, 0),
            0xA2: ("LDX", "imm", 2, 2, 0), 0xA6: ("LDX", "zp", 2, 3, 0), 0xB6: ("LDX", "zpy", 2, 4, 0),
            0xAE: ("LDX", "abs", 3, 4, 0), 0xBE: ("LDX", "absy", 3, 4, 1),
            0xA0: ("LDY", "imm", 2, 2, 0), 0xA4: ("LDY", "zp", 2, 3, 0), 0xB4: ("LDY", "zpx", 2, 4, 0),
            0xAC: ("LDY", "abs", 3, 4, 0), 0xBC: ("LDY", "absx", 3, 4, 1),
            0xE0: ("CPX", "imm", 2, 2, 0), 0xE4: ("CPX", "zp", 2, 3, 0), 0xEC: ("CPX", "abs", 3, 4, 0),
            0xC0: ("CPY", "imm", 2, 2, 0), 0xC4: ("CPY", "zp", 2, 3, 0), 0xCC: ("CPY", "abs", 3, 4, 0),
            0x24: ("BIT", "zp", 2, 3, 0), 0x2C: ("BIT", "abs", 3, 4, 0),
            0x4C: ("JMP", "abs", 3, 3, 0), 0x6C: ("JMP", "ind", 3, 5, 0), 0x20: ("JSR", "abs", 3, 6, 0),
            0x60: ("RTS", "imp", 1, 6, 0), 0x40: ("RTI", "imp", 1, 6, 0), 0x00: ("BRK", "imp", 1, 7, 0),
            0x48: ("PHA", "imp", 1, 3, 0), 0x08: ("PHP", "imp", 1, 3, 0),
            0x68: ("PLA", "imp", 1, 4, 0), 0x28: ("PLP", "imp", 1, 4, 0)})
for _m, _c in (("CLC", 0x18), ("CLD", 0xD8), ("CLI", 0x58), ("CLV", 0xB8), ("SEC", 0x38),
               ("SED", 0xF8), ("SEI", 0x78), ("NOP", 0xEA), ("TAX", 0xAA), ("TAY", 0xA8),
               ("TSX", 0xBA), ("TXA", 0x8A), ("TXS", 0x9A), ("TYA", 0x98), ("INX", 0xE8),
               ("INY", 0xC8), ("DEX", 0xCA), ("DEY", 0x88)):
    MOS[_c] = (_m, "imp", 1, 2, 0)
for _m, _c in (("BPL", 0x10), ("BMI", 0x30), ("BVC", 0x50), ("BVS", 0x70),
               ("BCC", 0x90), ("BCS", 0xB0), ("BNE", 0xD0), ("BEQ", 0xF0)):
    MOS[_c] = (_m, "rel", 2, 2, 0)

# status flags each instruction may change (MOS programming manual)
FLAGS = {"ADC": FN | FV | FZ | FC, "SBC": FN | FV | FZ | FC, "AND": FN | FZ, "ORA": FN | FZ,
         "EOR": FN | FZ, "ASL": FN | FZ | FC, "LSR": FN | FZ | FC, "ROL": FN | FZ | FC,
         "ROR": FN | FZ | FC, "BIT": FN | FV | FZ, "CMP": FN | FZ | FC, "CPX": FN | FZ | FC,
         "CPY": FN | FZ | FC, "INC": FN | FZ, "DEC": FN | FZ, "INX": FN | FZ, "INY": FN | FZ,
         "DEX": FN | FZ, "DEY": FN | FZ, "LDA": FN | FZ, "LDX": FN | FZ, "LDY": FN | FZ,
         "TAX": FN | FZ, "TAY": FN | FZ, "TSX": FN | FZ, "TXA": FN | FZ, "TYA": FN | FZ,
         "PLA": FN | FZ, "CLC": FC, "SEC": FC, "CLD": FD, "SED": FD, "CLI": FI, "SEI": FI,
         "CLV": FV, "BRK": FI}


# The paper's 38 extra opcode bytes (unofficial NMOS opcodes; lengths and
# cycle counts from the public unofficial-opcode documentation): USBC, the
# NOPs with and without operands, LAX and SAX.
EXTRA = {0xEB: ("USBC", "imm", 2, 2, 0)}
EXTRA.update({c: ("NOP", "imp", 1, 2, 0) for c in (0x1A, 0x3A, 0x5A, 0x7A, 0xDA, 0xFA)})
EXTRA.update({c: ("NOPR", "imm", 2, 2, 0) for c in (0x80, 0x82, 0x89, 0xC2, 0xE2)})
EXTRA.update({c: ("NOPR", "zp", 2, 3, 0) for c in (0x04, 0x44, 0x64)})
EXTRA.update({c: ("NOPR", "zpx", 2, 4, 0) for c in (0x14, 0x34, 0x54, 0x74, 0xD4, 0xF4)})
EXTRA.update({0x0C: ("NOPR", "abs", 3, 4, 0)})
EXTRA.update({c: ("NOPR", "absx", 3, 4, 1) for c in (0x1C, 0x3C, 0x5C, 0x7C, 0xDC, 0xFC)})
EXTRA.update({0xA7: ("LAX", "zp", 2, 3, 0), 0xB7: ("LAX", "zpy", 2, 4, 0), 0xAF: ("LAX", "abs", 3, 4, 0),
              0xBF: ("LAX", "absy", 3, 4, 1), 0xA3: ("LAX", "indx", 2, 6, 0), 0xB3: ("LAX", "indy", 2, 5, 1),
              0x87: ("SAX", "zp", 2, 3, 0), 0x97: ("SAX", "zpy", 2, 4, 0), 0x8F: ("SAX", "abs", 3, 4, 0),
              0x83: ("SAX", "indx", 2, 6, 0)})
FLAGS.update({"USBC": FN | FV | FZ | FC, "LAX": FN | FZ})


def test_table_has_151_documented_opcodes():
    assert len(MOS) == 151


def test_extra_table_has_the_papers_38_bytes():
    assert len(EXTRA) == 38 and not set(EXTRA) & set(MOS)


def _operand_bytes(mode, cross):
    """Operand bytes placing the access (or crossing) as requested."""
    if mode in ("zp", "zpx", "zpy"):
        return [0x90]
    if mode in ("abs",):
        return [0x90, 0x00]
    if mode in ("absx", "absy"):
        return [0x01, 0xFE] if cross else [0x00, 0xFE]
    if mode in ("indx",):
        return [0x90]
    if mode in ("indy",):
        return [0xA0]
    if mode == "imm":
        return [0x5A]
    if mode == "ind":
        return [0x00, 0xFD]
    return []


def _exec_opcode(op, cross=False, regs=None, ram=None):
    m, mode, n, _, _ = MOS.get(op) or EXTRA[op]
    body = [op] + _operand_bytes(mode, cross) if mode != "rel" else [op, 0x10]
    if m == "JSR" or (m == "JMP" and mode == "abs"):
        body = [op, 0x00, 0xF8]

    def build(a):
        a.byte(*body)
        a.at(0xD00)
        a.byte(0x34, 0x12)          # JMP ($FD00) target
    rom = rom4k(build)
    o = oracle.Oracle(rom, synth.MAPPER_4K)
    r = np.zeros(128, np.uint8) if ram is None else ram.copy()
    # pointers: $90/$91 -> $0098 (indx with X=0), $A0/$A1 -> $FE00 or $FE01
    r[0x10], r[0x11] = 0x98, 0x00
    r[0x20], r[0x21] = (0x01 if cross else 0x00), 0xFE
    o.set_ram(r)
    regs = dict(A=0x33, X=0, Y=0, SP=0xFF, P=0x30, PC=0xF000) if regs is None else regs
    if cross and mode in ("absx", "absy", "indy"):
        regs = dict(regs, X=0xFF, Y=0xFF)
    o.set_regs(**regs)
    s0 = o.state()
    cyc = o.exec_one()
    return o, s0, o.state(), cyc


ALL = {**MOS, **EXTRA}


@pytest.mark.parametrize("op", sorted(k for k, v in ALL.items() if v[1] != "rel"))
def test_opcode_cycles_and_length(op):
    m, mode, n, cyc, pen = ALL[op]
    o, s0, s1, c = _exec_opcode(op)
    assert c == cyc, (hex(op), m, mode, c, cyc)
    if m not in ("JMP", "JSR", "RTS", "RTI", "BRK"):
        assert s1[5] - s0[5] == n
    if mode in ("absx", "absy", "indy"):
        o, s0, s1, c2 = _exec_opcode(op, cross=True)
        assert c2 == cyc + pen, (hex(op), m, mode, c2)


@pytest.mark.parametrize("op", sorted(k for k, v in MOS.items() if v[1] == "rel"))
def test_branch_cycles(op):
    m = MOS[op][0]
    flag = {"BPL": FN, "BMI": FN, "BVC": FV, "BVS": FV, "BCC": FC, "BCS": FC, "BNE": FZ, "BEQ": FZ}[m]
    when_set = m in ("BMI", "BVS", "BCS", "BEQ")
    for taken in (False, True):
        p = flag if (taken == when_set) else 0
        for pc, off, cross in ((0xF000, 0x10, False), (0xF0F0, 0x20, True), (0xF010, 0xE0, True)):
            def build(a, pc=pc, off=off):
                a.at(pc - 0xF000)
                a.byte(op, off)
            o = oracle.Oracle(rom4k(build), synth.MAPPER_4K)
            o.set_regs(P=p, PC=pc)
            c = o.exec_one()
            target = (pc + 2 + (off - 256 if off >= 128 else off)) & 0xFFFF
            pc1 = o.state()[5]
            if taken:
                assert pc1 == target
                assert c == 3 + (1 if ((target ^ (pc + 2)) & 0xFF00) else 0), (m, hex(pc), off)
                assert bool((target ^ (pc + 2)) & 0xFF00) == cross
            else:
                assert pc1 == pc + 2 and c == 2


@pytest.mark.parametrize("op", sorted(k for k, v in ALL.items() if v[0] not in ("PLP", "RTI")))
def test_opcode_flag_effects(op):
    m, mode = ALL[op][:2]
    allowed = FLAGS.get(m, 0)
    rng = np.random.default_rng(op)
    changed = 0
    for trial in range(48):
        ram = rng.integers(0, 256, 128).astype(np.uint8)
        regs = dict(A=int(rng.integers(256)), X=0, Y=0, SP=0xFF,
                    P=int(rng.integers(256)) | 0x30, PC=0xF000)
        o, s0, s1, _ = _exec_opcode(op, regs=regs, ram=ram)
        diff = (int(s0[4]) ^ int(s1[4])) & 0xFF
        assert diff & ~allowed == 0, (hex(op), m, hex(diff))
        assert s1[4] & 0x30 == 0x30
        changed |= diff
    if m not in ("BRK",):
        assert changed == allowed, (hex(op), m, hex(changed), hex(allowed))


def test_jmp_indirect_page_wrap():
    """JMP ($xxFF) takes the high byte from $xx00 (documented NMOS behaviour)."""
    def build(a):
        a.byte(0x6C, 0xFF, 0xF1)
        a.at(0x100)
        a.byte(0x56)          # $F100: high byte used by the wrap
        a.at(0x1FF)
        a.byte(0x34)          # $F1FF: low byte
        a.byte(0x99)          # $F200: not used
    o = oracle.Oracle(rom4k(build), synth.MAPPER_4K)
    o.set_regs(PC=0xF000)
    assert o.exec_one() == 5
    assert o.state()[5] == 0x5634


def test_stack_and_subroutines():
    """JSR pushes the address of its last byte; RTS returns past it; PHP
    pushes bits 4 and 5 set; BRK pushes PC+2 and vectors through $FFFE."""
    def build(a):
        a.op("JSR", "abs", 0xF100)    # F000
        a.op("PHP")                   # F003
        a.op("BRK")                   # F004
        a.byte(0xEE)
        a.op("NOP")                   # F006
        a.at(0x100)
        a.op("RTS")                   # F100
        a.at(0x200)
        a.op("RTI")                   # F200
    rom = bytearray(rom4k(build))
    rom[0xFFE], rom[0xFFF] = 0x00, 0xF2
    o = oracle.Oracle(bytes(rom), synth.MAPPER_4K)
    o.set_regs(SP=0xFF, P=0x00, PC=0xF000)
    assert o.exec_one() == 6
    ram = o.ram()
    assert (ram[0x7F], ram[0x7E]) == (0xF0, 0x02)
    assert o.state()[3] == 0xFD
    assert o.exec_one() == 6 and o.state()[5] == 0xF003
    assert o.exec_one() == 3 and o.ram()[0x7F] & 0x30 == 0x30
    assert o.exec_one() == 7
    s = o.state()
    assert s[5] == 0xF200 and s[4] & FI
    ram = o.ram()
    assert (ram[0x7E], ram[0x7D]) == (0xF0, 0x06)
    assert o.exec_one() == 6 and o.state()[5] == 0xF006


def test_extra_opcode_behaviour():
    """LAX loads A and X with the operand; SAX stores A & X and leaves the
    flags; USBC is SBC immediate for every A, operand, carry and decimal
    flag; the NOPs change no register or RAM."""
    rng = np.random.default_rng(38)
    for _ in range(64):
        ram = rng.integers(0, 256, 128).astype(np.uint8)
        a, x = int(rng.integers(256)), int(rng.integers(256))
        p = int(rng.integers(256)) | 0x30
        o, s0, s1, _ = _exec_opcode(0xA7, regs=dict(A=a, X=x, Y=0, SP=0xFF, P=p, PC=0xF000), ram=ram)
        assert s1[0] == s1[1] == 0x98               # LAX $90: cell $10, which the set-up points at $0098
        o, s0, s1, _ = _exec_opcode(0x87, regs=dict(A=a, X=x, Y=0, SP=0xFF, P=p, PC=0xF000), ram=ram)
        assert o.ram()[0x10] == a & x and s1[4] == s0[4] and s1[0] == a and s1[1] == x
        set_up = ram.copy()
        set_up[0x10], set_up[0x11], set_up[0x20], set_up[0x21] = 0x98, 0x00, 0x00, 0xFE   # _exec_opcode's pointers
        for op in (0x1A, 0x80, 0x04, 0x14, 0x0C, 0x1C):
            o, s0, s1, _ = _exec_opcode(op, regs=dict(A=a, X=x, Y=0, SP=0xFF, P=p, PC=0xF000), ram=ram)
            assert list(s1[:5]) == list(s0[:5]) and np.array_equal(o.ram(), set_up)

    def build(a):
        a.byte(0xEB, 0x00)       # $F000: USBC #$00 (operand patched per case below)
        a.at(0x10)
        a.byte(0xE9, 0x00)       # $F010: SBC #$00
    for m in (0x00, 0x01, 0x09, 0x10, 0x7F, 0x80, 0x99, 0xFF):
        img = bytearray(rom4k(build))
        img[1] = img[0x11] = m
        o = oracle.Oracle(bytes(img), synth.MAPPER_4K)
        for a in range(0, 256, 7):
            for p in (0x30, 0x31, 0x38, 0x39):
                o.set_regs(A=a, P=p, PC=0xF000)
                o.exec_one()
                r1 = o.state()[[0, 4]]
                o.set_regs(A=a, P=p, PC=0xF010)
                o.exec_one()
                assert np.array_equal(r1, o.state()[[0, 4]])


def test_extra_nop_reads_have_side_effects():
    """An unofficial NOP with an absolute operand reads it like a load: a
    read of $1FF8 selects F8 bank 0."""
    def bank(b):
        a = synth.Asm(0xF000, 4096)
        a.byte(0x0C, 0xF8, 0xFF)   # NOP $FFF8
        a.at(0xFFA)
        a.word(0xF000)
        a.word(0xF000)
        a.word(0xF000)
        return bytes(a.resolve())
    o = oracle.Oracle(bank(0) + bank(1), synth.MAPPER_F8)
    assert o.bank() == 1
    o.exec_one()
    assert o.bank() == 0
