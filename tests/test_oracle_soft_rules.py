"""The oracle's surrogate rulebook, coefficient by coefficient, pinned by
micro-programs whose gradients are derived by hand from the rules (Section
3.1: Eq. peek's one-hot read, Eq. ste's straight-through rule for casts and
the stored-switch rule; Corollary 1), not from the oracle's deviation graph.

Every program runs one frame at tau = 0.01, where a read's window weights
beyond the read cell are e^-100 (the one-hot read of Eq. peek), then loops
on itself until the 512-line cap ends the frame.  The loss is a weighted sum
of RAM bytes at the end of the step; the expected gradient with respect to
each ROM byte, initial RAM cell and joystick input follows from the rules:

  ADC (1, +1), SBC and USBC (1, -1), in binary and decimal mode;
  AND / ORA / EOR (1, 1); shifts, rotates, INC / DEC / INX ... 1 (the
  straight-through rule); loads, stores, transfers, PHA / PLA 1; LAX sends
  both A's and X's adjoints to the operand; SAX's cell takes A and X with
  (1, 1); CMP / BIT / flags / the carry-in no content gradient; TSX, PHP and
  the return address pushed by JSR 0 (SP, P and PC are indices or bits);
  pointers 0 (an address is a stored switch); writes one-hot;
  SWCHA = 255 - 128 u_R - 64 u_L - 32 u_D - 16 u_U, INPT4 = 128 (1 - u_F);
  INTIM: 1 with respect to the value written to the timer before the
  underflow, 0 after it.

A plausible mistake in any of these sites of the oracle (a flipped sign, a
rule of one opcode applied to another, a dropped adjoint) changes one of the
expected values below.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_22447_b300 import synth
from tests.microrom import rom4k

TAU = 0.01
U_RIGHT, U_LEFT, U_DOWN, U_UP, U_FIRE = range(5)


class Prog:
    """A micro-program: `emit(a, m)` writes code through the assembler `a`;
    m.imm(name, mnem, value) emits `mnem #value` and remembers the ROM offset
    of its operand byte under `name`."""

    def __init__(self, a):
        self.a = a
        self.off = {}

    def imm(self, name, mnem, value):
        self.off[name] = self.a.pc + 1 - 0xF000
        self.a.op(mnem, "imm", value)

    def raw_imm(self, name, opcode, value):
        self.off[name] = self.a.pc + 1 - 0xF000
        self.a.byte(opcode, value)


def run(emit, loss, ram0=None, u=None, tau=TAU):
    """Assemble, run one soft frame and return (g_rom, g_ram0, g_u, ram, offsets)."""
    holder = {}

    def build(a):
        m = Prog(a)
        emit(a, m)
        a.label("HALT")
        a.op("JMP", "abs", "HALT")
        holder["m"] = m
    rom = rom4k(build)
    o = oracle.Oracle(rom, synth.MAPPER_4K)
    if ram0 is not None:
        o.set_ram(np.asarray(ram0, np.uint8))
    u = np.zeros((1, 5)) if u is None else np.asarray(u, np.float64).reshape(1, 5)
    gr = np.zeros((1, 128))
    for cell, w in loss.items():
        gr[0, cell - 0x80] = w
    g, ram, _ = o.soft_rollout(u, 1, tau, 6.0, gr, None)
    g_rom, g_ram0, g_u = g.reverse()
    return g_rom, g_ram0, g_u[0], ram[0], holder["m"].off


def expect(g, want, what, tol=1e-12):
    """g equals the sparse expectation `want` ({index: value}) everywhere."""
    full = np.zeros_like(g)
    for i, v in want.items():
        full[i] = v
    bad = np.flatnonzero(np.abs(g - full) > tol)
    assert bad.size == 0, (f"{what}: at {bad[:6].tolist()} got {g[bad[:6]].tolist()} "
                           f"want {full[bad[:6]].tolist()}")


def rom_grad(emit, loss, want, **kw):
    g_rom, g_ram0, g_u, ram, off = run(emit, loss, **kw)
    expect(g_rom, {off[k]: v for k, v in want.items()}, "grad_rom")
    return g_ram0, g_u, ram


# ---------------------------------------------------------------- ALU rules

@pytest.mark.parametrize("decimal", [False, True])
def test_adc_is_one_and_plus_one(decimal):
    def emit(a, m):
        a.op("SED" if decimal else "CLD")
        m.imm("a", "LDA", 0x25)
        a.op("CLC")
        m.imm("b", "ADC", 0x19)
        a.op("STA", "zp", 0x80)
        a.op("CLD")
    g_ram0, g_u, ram = rom_grad(emit, {0x80: 1.0}, {"a": 1.0, "b": 1.0})
    assert ram[0] == (0x44 if decimal else 0x3E)
    expect(g_ram0, {}, "grad_ram0")
    expect(g_u, {}, "grad_u")


@pytest.mark.parametrize("decimal", [False, True])
@pytest.mark.parametrize("opcode", [0xE9, 0xEB])   # SBC #imm and its alias USBC
def test_sbc_and_usbc_are_one_and_minus_one(decimal, opcode):
    def emit(a, m):
        a.op("SED" if decimal else "CLD")
        m.imm("a", "LDA", 0x42)
        a.op("SEC")
        m.raw_imm("b", opcode, 0x17)
        a.op("STA", "zp", 0x80)
        a.op("CLD")
    _, _, ram = rom_grad(emit, {0x80: 1.0}, {"a": 1.0, "b": -1.0})
    assert ram[0] == (0x25 if decimal else 0x2B)


@pytest.mark.parametrize("mnem", ["ADC", "SBC"])
def test_adc_sbc_with_memory_operands_reach_initial_ram(mnem):
    """LDA $90; (CLC | SEC); ADC / SBC $91; STA $80, weight 2 on $80:
    d/d ram0[$10] = 2, d/d ram0[$11] = +-2; the carry flag gives nothing."""
    def emit(a, m):
        a.op("LDA", "zp", 0x90)
        a.op("CLC" if mnem == "ADC" else "SEC")
        a.op(mnem, "zp", 0x91)
        a.op("STA", "zp", 0x80)
    ram0 = np.zeros(128, np.uint8)
    ram0[0x10], ram0[0x11] = 0x60, 0x21
    g_rom, g_ram0, _, _, _ = run(emit, {0x80: 2.0}, ram0=ram0)
    expect(g_ram0, {0x10: 2.0, 0x11: 2.0 if mnem == "ADC" else -2.0}, "grad_ram0")
    expect(g_rom, {}, "grad_rom")


@pytest.mark.parametrize("mnem", ["AND", "ORA", "EOR"])
def test_logic_operations_are_one_and_one(mnem):
    def emit(a, m):
        m.imm("a", "LDA", 0x5C)
        m.imm("b", mnem, 0x3A)
        a.op("STA", "zp", 0x80)
    rom_grad(emit, {0x80: 1.0}, {"a": 1.0, "b": 1.0})


@pytest.mark.parametrize("mnem", ["ASL", "ROL", "LSR", "ROR"])
@pytest.mark.parametrize("where", ["acc", "zp", "abs"])
@pytest.mark.parametrize("carry", ["SEC", "CLC"])
def test_shifts_and_rotates_are_straight_through(mnem, where, carry):
    """The shifted value's derivative is 1 (Eq. ste's straight-through rule
    for the cast); the rotated-in carry is a flag and gives nothing."""
    def emit(a, m):
        m.imm("a", "LDA", 0x96)
        if where == "acc":
            a.op(carry)
            a.op(mnem, "acc")
        else:
            addr = 0x90 if where == "zp" else 0x0091
            a.op("STA", where, addr)
            a.op(carry)
            a.op(mnem, where, addr)
            a.op("LDA", where, addr)
        a.op("STA", "zp", 0x80)
    rom_grad(emit, {0x80: 3.0}, {"a": 3.0})


@pytest.mark.parametrize("code", ["INC", "DEC", "INX", "DEX", "INY", "DEY"])
def test_increments_and_decrements_are_one(code):
    def emit(a, m):
        if code in ("INC", "DEC"):
            m.imm("a", "LDA", 0x7F)
            a.op("STA", "zp", 0x90)
            a.op(code, "zp", 0x90)
            a.op("LDA", "zp", 0x90)
            a.op("STA", "zp", 0x80)
        elif code.endswith("X"):
            m.imm("a", "LDX", 0x7F)
            a.op(code)
            a.op("STX", "zp", 0x80)
        else:
            m.imm("a", "LDY", 0x7F)
            a.op(code)
            a.op("STY", "zp", 0x80)
    rom_grad(emit, {0x80: 1.0}, {"a": 1.0})


@pytest.mark.parametrize("mnem", ["CMP", "BIT"])
def test_compare_and_bit_give_no_content_gradient(mnem):
    def emit(a, m):
        m.imm("a", "LDA", 0x40)
        if mnem == "CMP":
            m.imm("b", "CMP", 0x33)
        else:
            a.op("BIT", "zp", 0x90)
        a.op("STA", "zp", 0x80)
    ram0 = np.full(128, 0xC3, np.uint8)
    g_ram0, _, _ = rom_grad(emit, {0x80: 1.0}, {"a": 1.0}, ram0=ram0)
    expect(g_ram0, {}, "grad_ram0")


def test_branch_flags_give_no_gradient():
    """LDA $90; BEQ skip; LDA #k; skip: STA $80 with ram0[$10] != 0: A comes
    from the immediate, and the branch's flag (from the RAM cell) passes
    nothing back."""
    def emit(a, m):
        a.op("LDA", "zp", 0x90)
        a.op("BEQ", "rel", "SKIP")
        m.imm("k", "LDA", 0x11)
        a.label("SKIP")
        a.op("STA", "zp", 0x80)
    ram0 = np.zeros(128, np.uint8)
    ram0[0x10] = 9
    g_ram0, _, _ = rom_grad(emit, {0x80: 1.0}, {"k": 1.0}, ram0=ram0)
    expect(g_ram0, {}, "grad_ram0")


# ------------------------------------------------------ transfers and stack

@pytest.mark.parametrize("path", ["TAX", "TXA", "TAY", "TYA"])
def test_register_transfers_are_one(path):
    def emit(a, m):
        src = path[1]
        m.imm("a", "LD" + src, 0x66)
        a.op("LDA" if src != "A" else "LDX", "imm", 0)   # clobber another register
        if src != "A":
            a.op("LDA", "imm", 0)
        a.op(path)
        dst = path[2]
        a.op("ST" + dst, "zp", 0x80)
    rom_grad(emit, {0x80: 1.0}, {"a": 1.0})


def test_tsx_reads_the_stack_pointer_which_carries_nothing():
    def emit(a, m):
        m.imm("a", "LDX", 0xF0)
        a.op("TXS")
        a.op("LDX", "imm", 0)
        a.op("TSX")
        a.op("STX", "zp", 0x80)
    _, _, ram = rom_grad(emit, {0x80: 1.0}, {})
    assert ram[0] == 0xF0


def test_pha_pla_carry_the_value_through_the_stack_cell():
    def emit(a, m):
        a.op("LDX", "imm", 0xFF)
        a.op("TXS")
        m.imm("a", "LDA", 0x3D)
        a.op("PHA")
        a.op("LDA", "imm", 0)
        a.op("PLA")
        a.op("STA", "zp", 0x80)
    g_ram0, _, _ = rom_grad(emit, {0x80: 1.0}, {"a": 1.0})
    expect(g_ram0, {}, "grad_ram0")


def test_data_around_jsr_and_rts():
    """LDA #a; PHA; LDA #b; JSR SUB; STA $81; PLA; STA $80 with SUB: RTS:
    JSR and RTS move the stack pointer around the pushed value, and A
    passes through the call."""
    def emit(a, m):
        a.op("LDX", "imm", 0xFF)
        a.op("TXS")
        m.imm("a", "LDA", 0x12)
        a.op("PHA")
        m.imm("b", "LDA", 0x34)
        a.op("JSR", "abs", "SUB")
        a.op("STA", "zp", 0x81)
        a.op("PLA")
        a.op("STA", "zp", 0x80)
        a.op("JMP", "abs", "END")
        a.label("SUB")
        a.op("RTS")
        a.label("END")
    _, _, ram = rom_grad(emit, {0x80: 1.0, 0x81: 5.0}, {"a": 1.0, "b": 5.0})
    assert (ram[0], ram[1]) == (0x12, 0x34)


def test_return_address_and_pushed_status_carry_nothing():
    """LDA #a; JSR SUB; SUB: PLA; STA $80; PLA; STA $81; LDA #b; PHP; PLA;
    STA $82: the pulled bytes are the program counter and P, indices and
    bits, whatever A held when they were pushed; the stack cells' initial
    values are overwritten by the pushes."""
    def emit(a, m):
        a.op("LDX", "imm", 0xFF)
        a.op("TXS")
        m.imm("a", "LDA", 0x21)
        a.op("JSR", "abs", "SUB")
        a.label("SUB")
        a.op("PLA")
        a.op("STA", "zp", 0x80)
        a.op("PLA")
        a.op("STA", "zp", 0x81)
        m.imm("b", "LDA", 0x43)
        a.op("PHP")
        a.op("PLA")
        a.op("STA", "zp", 0x82)
    ram0 = np.full(128, 0x55, np.uint8)
    g_ram0, _, ram = rom_grad(emit, {0x80: 1.0, 0x81: 1.0, 0x82: 1.0}, {}, ram0=ram0)
    expect(g_ram0, {}, "grad_ram0")
    assert ram[1] == 0xF0   # high byte of the return address


# -------------------------------------------------------- the extra opcodes

def test_lax_sends_both_adjoints_to_the_operand():
    """LAX $90; STX $80; STA $81 with weights 1 and 2: d/d ram0[$10] = 3;
    LAX $FE37 (the ROM's identity table) likewise for the ROM byte."""
    def emit(a, m):
        a.byte(0xA7, 0x90)        # LAX $90
        a.op("STX", "zp", 0x80)
        a.op("STA", "zp", 0x81)
    ram0 = np.zeros(128, np.uint8)
    ram0[0x10] = 0x77
    g_rom, g_ram0, _, ram, _ = run(emit, {0x80: 1.0, 0x81: 2.0}, ram0=ram0)
    expect(g_ram0, {0x10: 3.0}, "grad_ram0")
    expect(g_rom, {}, "grad_rom")
    assert (ram[0], ram[1]) == (0x77, 0x77)

    def emit2(a, m):
        a.byte(0xAF, 0x37, 0xFE)  # LAX $FE37
        a.op("STX", "zp", 0x80)
        a.op("STA", "zp", 0x81)
    g_rom, _, _, ram, _ = run(emit2, {0x80: 1.0, 0x81: 2.0})
    expect(g_rom, {0xE37: 3.0}, "grad_rom")
    assert (ram[0], ram[1]) == (0x37, 0x37)


def test_sax_stores_a_and_x_with_one_and_one():
    def emit(a, m):
        m.imm("a", "LDA", 0xF3)
        m.imm("x", "LDX", 0x3C)
        a.byte(0x87, 0x80)        # SAX $80
    _, _, ram = rom_grad(emit, {0x80: 1.0}, {"a": 1.0, "x": 1.0})
    assert ram[0] == 0x30


# ------------------------------------------------------ writes and pointers

def test_writes_are_one_hot():
    def emit(a, m):
        m.imm("a", "LDA", 0x01)
        a.op("STA", "zp", 0x90)
        m.imm("b", "LDA", 0x02)
        a.op("STA", "zp", 0x90)
        a.op("LDA", "zp", 0x90)
        a.op("STA", "zp", 0x80)
    g_ram0, _, _ = rom_grad(emit, {0x80: 1.0}, {"b": 1.0})
    expect(g_ram0, {}, "grad_ram0")


@pytest.mark.parametrize("mode", ["indy", "indx"])
def test_pointers_are_stored_switches(mode):
    """LDA ($90),Y / LDA ($90,X) through a pointer in RAM to $A0: the data
    cell's initial value gets the gradient, the pointer bytes none."""
    def emit(a, m):
        a.op("LDY", "imm", 0)
        a.op("LDX", "imm", 0)
        a.op("LDA", mode, 0x90)
        a.op("STA", "zp", 0x80)
    ram0 = np.zeros(128, np.uint8)
    ram0[0x10], ram0[0x11], ram0[0x20] = 0xA0, 0x00, 0x5B
    g_rom, g_ram0, _, ram, _ = run(emit, {0x80: 1.0}, ram0=ram0)
    assert ram[0] == 0x5B
    expect(g_ram0, {0x20: 1.0}, "grad_ram0")
    expect(g_rom, {}, "grad_rom")


# ------------------------------------------------------------------ I/O rules

def test_swcha_coefficients():
    """LDA SWCHA; STA $80: SWCHA = 255 - 128 u_R - 64 u_L - 32 u_D - 16 u_U."""
    def emit(a, m):
        a.op("LDA", "abs", 0x0280)
        a.op("STA", "zp", 0x80)
    g_rom, g_ram0, g_u, ram, _ = run(emit, {0x80: 1.0}, u=[0, 1, 0, 1, 0])
    assert ram[0] == 0xFF - 64 - 16
    expect(g_u, {U_RIGHT: -128.0, U_LEFT: -64.0, U_DOWN: -32.0, U_UP: -16.0}, "grad_u")
    expect(g_rom, {}, "grad_rom")


@pytest.mark.parametrize("fire", [0, 1])
def test_inpt4_coefficient(fire):
    """LDA INPT4; STA $80: INPT4 = 128 (1 - u_F), bit 7 clear while fire is
    pressed."""
    def emit(a, m):
        a.op("LDA", "zp", 0x0C)
        a.op("STA", "zp", 0x80)
    g_rom, _, g_u, ram, _ = run(emit, {0x80: 2.0}, u=[0, 0, 0, 0, fire])
    assert ram[0] == (0x00 if fire else 0x80)
    expect(g_u, {U_FIRE: -256.0}, "grad_u")
    expect(g_rom, {}, "grad_rom")


@pytest.mark.parametrize("live", [True, False])
def test_intim_is_one_before_the_underflow_and_zero_after(live):
    """LDA #v; STA TIM64T (or TIM1T); NOP x 3; LDA INTIM; STA $80.  At 64
    cycles per count the read comes about 10 cycles after the write, so
    INTIM = v - 1 with derivative 1 in v; at one cycle per count and v = 2
    the timer has underflowed by then, and the read carries nothing."""
    def emit(a, m):
        m.imm("v", "LDA", 0x21 if live else 0x02)
        a.op("STA", "abs", 0x0296 if live else 0x0294)
        for _ in range(3):
            a.op("NOP")
        a.op("LDA", "abs", 0x0284)
        a.op("STA", "zp", 0x80)
    _, _, ram = rom_grad(emit, {0x80: 1.0}, {"v": 1.0} if live else {})
    if live:
        assert ram[0] == 0x20
    else:
        assert ram[0] > 0xF0   # counting down from $FF after the underflow


# ----------------------------------------------------- the relaxed read window

def _weights(a, M, tau):
    W = max(1, math.ceil(12 * tau))
    w = np.array([math.exp(-abs(i - a) / tau) if abs(i - a) <= W else 0.0 for i in range(M)])
    return w / w.sum()


@pytest.mark.parametrize("tau", [0.5, 1.0])
@pytest.mark.parametrize("cell", [0x90, 0x81])
def test_ram_read_window(tau, cell):
    """LDA cell; STA $F0 at tau > 0.01: d/d ram0[i] is the read's window
    weight e^{-|i - a| / tau}, |i - a| <= max(1, ceil(12 tau)), clipped to
    the 128 cells and renormalised (Eq. s-read); $81 sits next to the
    tensor's start, so its window is clipped."""
    def emit(a, m):
        a.op("LDA", "zp", cell)
        a.op("STA", "zp", 0xF0)
    ram0 = np.arange(128, dtype=np.uint8)
    g_rom, g_ram0, _, _, _ = run(emit, {0xF0: 1.0}, ram0=ram0, tau=tau)
    w = _weights(cell - 0x80, 128, tau)
    assert np.allclose(g_ram0, w, rtol=1e-12, atol=1e-15)
    expect(g_rom, {}, "grad_rom")


@pytest.mark.parametrize("tau", [0.5, 1.0])
def test_rom_read_window(tau):
    """LDA $FE37; STA $80: the 4K image is the read's tensor, so ROM bytes
    around offset $E37 take the window's weights."""
    def emit(a, m):
        a.op("LDA", "abs", 0xFE37)
        a.op("STA", "zp", 0x80)
    g_rom, _, _, _, _ = run(emit, {0x80: 1.0}, tau=tau)
    w = _weights(0xE37, 4096, tau)
    assert np.allclose(g_rom, w, rtol=1e-12, atol=1e-15)
