"""Parity of the CUDA hard path with the oracle, bit for bit, on RAM,
screens and status, through the C ABI (HARD mode of the supplement's
execution-mode table; the paper's RAM-exact / pixel-exact metrics of
Section 5, with the oracle standing in for the reference emulator)."""
import numpy as np
import pytest

import oracle
from paper_2606_22447_b300 import synth
from tests.gpu_util import assert_env_equal, gpu_rollout, make_batch, oracle_rollout, torch_cuda
from tests.microrom import extra_ops_rom, rom4k, switches_rom

pytestmark = pytest.mark.gpu


def _check_all(roms, mappers, env_cart, actions, frame_skip, screens=True, envs=None, **cfg):
    b = make_batch(roms, mappers, env_cart, **cfg)
    ram, scr, st = gpu_rollout(b, actions, frame_skip, screens)
    envs = range(len(env_cart)) if envs is None else envs
    for e in envs:
        c = int(env_cart[e])
        r2, s2, st2 = oracle_rollout(roms[c], mappers[c], actions[:, e], frame_skip, screens=screens)
        assert_env_equal(e, ram[:, e], r2, "RAM")
        if screens:
            assert_env_equal(e, scr[:, e], s2, "screen")
        assert_env_equal(e, st[:, e], st2, "status")
    return b


def test_single_env_2k_60_frames():
    rom = synth.generate_cart(101, 0, synth.MAPPER_2K)
    acts = synth.actions(101, 1, 60)
    _check_all([rom], [synth.MAPPER_2K], [0], acts, 1)


@pytest.mark.parametrize("mapper", [synth.MAPPER_2K, synth.MAPPER_4K, synth.MAPPER_F8, synth.MAPPER_F6,
                                    synth.MAPPER_F4])
def test_many_envs_one_cart_ragged(mapper):
    rom = synth.generate_cart(202, 1, mapper)
    n_envs = 75      # several blocks and a ragged tail
    acts = synth.actions(202, n_envs, 8)
    _check_all([rom], [mapper], [0] * n_envs, acts, 4)


def test_mixed_carts_unsorted_envs():
    roms = synth.config_carts(303, synth.MIX16)
    env_cart = np.random.default_rng(3).permutation(np.arange(96) % 16).astype(np.int32)
    acts = synth.actions(303, 96, 5)
    _check_all(roms, synth.MIX16, env_cart, acts, 2)


@pytest.mark.parametrize("epb,tpe", [(16, 1), (128, 1), (32, 4)])
def test_all_five_mappers_in_one_batch(epb, tpe):
    """2K, 4K, F8, F6 and F4 carts in one batch (32 KB ROM stride, the blocks
    of the F6 and F4 carts switching among 4 and 8 banks), envs unsorted."""
    mappers = [synth.MAPPER_2K, synth.MAPPER_4K, synth.MAPPER_F8, synth.MAPPER_F6, synth.MAPPER_F4] * 2
    roms = synth.config_carts(305, mappers)
    env_cart = np.random.default_rng(5).permutation(np.arange(60) % 10).astype(np.int32)
    acts = synth.actions(305, 60, 8)
    b = _check_all(roms, mappers, env_cart, acts, 2, envs_per_block=epb, threads_per_env=tpe)
    assert b.rom_stride == 32768


def test_f6_f4_hotspot_chains():
    """Every hotspot of F6 and F4 selects its bank on the GPU as in the
    oracle: the chain of the oracle's hotspot pin, then a frame loop."""
    for mapper in (synth.MAPPER_F6, synth.MAPPER_F4):
        nb, hot = synth.MAPPER_BANKS[mapper], synth.MAPPER_HOTSPOT[mapper]
        banks = []
        for j in range(nb):
            a = synth.Asm(0xF000, 4096)
            if j == nb - 1:
                a.op("LDA", "abs", hot - 1)
                a.op("LDA", "abs", hot + nb)
                a.op("LDA", "abs", hot - 0x1000)
                a.op("LDA", "abs", hot)
            else:
                a.at(12 + 3 * j)
                a.op("STA" if j % 2 else "LDA", "abs", hot + j + 1)
            a.at(0x100)
            a.label("LOOP")             # every bank: a frame loop that shows its bank number
            a.op("LDA", "imm", 2)
            a.op("STA", "zp", 0x02)
            a.op("STA", "zp", 0x00)
            a.op("LDA", "imm", 0)
            a.op("STA", "zp", 0x00)
            a.op("LDA", "imm", 0x10 * (j + 1))
            a.op("STA", "zp", 0x09)
            a.op("STA", "zp", 0x80 + j)
            a.op("LDX", "imm", 0)
            a.label("L")
            a.op("STA", "zp", 0x02)
            a.op("DEX")
            a.op("BNE", "rel", "L")
            a.op("JMP", "abs", "LOOP")
            a.at(4096 - 6)
            a.word(0xF000), a.word(0xF000), a.word(0xF000)
            banks.append(bytes(a.resolve()))
        rom = b"".join(banks)
        acts = synth.actions(306, 3, 4)
        _check_all([rom], [mapper], [0, 0, 0], acts, 1)


@pytest.mark.parametrize("epb,tpe", [(8, 1), (16, 1), (32, 1), (64, 1), (128, 1), (8, 2), (8, 4), (8, 8),
                                     (16, 8), (32, 4), (64, 2)])
def test_block_sizes_agree(epb, tpe):
    """Every launch geometry (envs per block x threads per env) computes the
    same bits; replicas split the drawing and the row writes."""
    rom = synth.generate_cart(404, 2, synth.MAPPER_4K)
    acts = synth.actions(404, 40, 4)
    b = make_batch([rom], [synth.MAPPER_4K], [0] * 40, envs_per_block=epb, threads_per_env=tpe)
    ram, scr, st = gpu_rollout(b, acts, 3)
    for e in (0, 17, 39):
        r2, s2, _ = oracle_rollout(rom, synth.MAPPER_4K, acts[:, e], 3)
        assert_env_equal(e, ram[:, e], r2, "RAM")
        assert_env_equal(e, scr[:, e], s2, "screen")


def test_ystart_and_frame_skip_variants():
    rom = synth.generate_cart(505, 0, synth.MAPPER_4K)
    acts = synth.actions(505, 3, 6)
    for fs in (1, 3):
        b = make_batch([rom], [synth.MAPPER_4K], [0, 0, 0], ystart=0)
        ram, scr, _ = gpu_rollout(b, acts, fs)
        for e in range(3):
            o = oracle.Oracle(rom, synth.MAPPER_4K, ystart=0)
            r2, s2, _ = o.rollout(acts[:, e], fs)
            assert_env_equal(e, ram[:, e], r2, "RAM")
            assert_env_equal(e, scr[:, e], s2, "screen")


# ---------------------------------------------------------------------------
# edge cases on hand-made cartridges
# ---------------------------------------------------------------------------

def _jam_rom():
    def build(a):
        a.op("LDA", "imm", 0x42)
        a.op("STA", "zp", 0x09)
        a.byte(0x02)                  # undocumented opcode: the CPU halts
    return rom4k(build)


def _runaway_rom():
    """Never writes VSYNC: every frame ends at the 512-line cap."""
    def build(a):
        a.label("L")
        a.op("INC", "zp", 0x80)
        a.op("LDA", "zp", 0x80)
        a.op("STA", "zp", 0x09)
        a.op("STA", "zp", 0x02)
        a.op("JMP", "abs", "L")
    return rom4k(build)


def _timer_rom():
    """Timer reads at every interval and odd cycle offsets stored to RAM and
    the screen, plus mid-line RESP0/HMOVE/playfield writes."""
    def build(a):
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", 0x01)
        a.label("F")
        a.op("LDA", "imm", 2)
        a.op("STA", "zp", 0x02)
        a.op("STA", "zp", 0x00)
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", 0x00)
        a.op("LDA", "imm", 0x70)
        a.op("STA", "zp", 0x20)       # HMP0: move by 7
        a.op("LDY", "imm", 0)
        a.label("L")
        a.op("STA", "zp", 0x02)
        a.op("STA", "zp", 0x2A)       # early HMOVE
        a.op("TYA")
        a.op("STA", "abs", 0x0294 + (0 if True else 0))
        a.op("LDA", "abs", 0x0284)
        a.op("STA", "zp", 0x06)
        a.op("STA", "zp", 0x1B)
        a.op("LDX", "abs", 0x0285)
        a.op("STX", "zp", 0x0E)
        a.op("STA", "zp", 0x10)
        a.op("TYA")
        a.op("STA", "abs", 0x0296)
        a.op("LDA", "abs", 0x0284)
        a.op("STA", "zp", 0x08)
        a.op("STA", "zp", 0x80)
        a.op("INY")
        a.op("CPY", "imm", 240)
        a.op("BNE", "rel", "L")
        a.op("JMP", "abs", "F")
    return rom4k(build)


def _decimal_stack_rom():
    """Decimal ADC/SBC, BRK/RTI, JSR/RTS, PHP/PLP, JMP (ind) in a frame loop."""
    def build(a):
        a.op("LDX", "imm", 0xFF)
        a.op("TXS")
        a.label("F")
        a.op("LDA", "imm", 2)
        a.op("STA", "zp", 0x02)
        a.op("STA", "zp", 0x00)
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", 0x00)
        a.op("LDX", "imm", 200)
        a.label("L")
        a.op("STA", "zp", 0x02)
        a.op("SED")
        a.op("TXA")
        a.op("ADC", "zp", 0x81)
        a.op("STA", "zp", 0x81)
        a.op("SBC", "imm", 0x19)
        a.op("STA", "zp", 0x09)
        a.op("CLD")
        a.op("PHP")
        a.op("JSR", "abs", "S")
        a.op("PLP")
        a.op("BRK")
        a.byte(0xEA)
        a.op("JMP", "ind", "P")
        a.label("BACK")
        a.op("DEX")
        a.op("BNE", "rel", "L")
        a.op("JMP", "abs", "F")
        a.label("S")
        a.op("LDA", "abs", 0x0280)
        a.op("EOR", "zp", 0x82)
        a.op("STA", "zp", 0x82)
        a.op("STA", "zp", 0x0F)
        a.op("RTS")
        a.label("P")
        a.word("BACK")
        a.label("IRQ")
        a.op("INC", "zp", 0x83)
        a.op("RTI")
    a_img = bytearray(rom4k(build))
    return bytes(a_img)


def _with_irq(rom, target):
    img = bytearray(rom)
    img[0xFFE], img[0xFFF] = target & 0xFF, target >> 8
    return bytes(img)


def test_edge_case_carts():
    rom_d = _decimal_stack_rom()
    # BRK vector -> the IRQ label: find "INC $83" (E6 83) followed by RTI
    irq = 0xF000 + bytes(rom_d).find(bytes([0xE6, 0x83, 0x40]))
    rom_d = _with_irq(rom_d, irq)
    roms = [_jam_rom(), _runaway_rom(), _timer_rom(), rom_d]
    maps = [synth.MAPPER_4K] * 4
    env_cart = np.arange(8) % 4
    acts = synth.actions(606, 8, 5)
    _check_all(roms, maps, env_cart, acts, 2)
    b = make_batch(roms, maps, env_cart)
    _, _, st = gpu_rollout(b, acts, 2, screens=False)
    assert np.all(st[:, 0] & 2) and np.all(st[:, 1] & 1) and not np.any(st[:, 2:4])


def _poll_rom(timer_reg, value, page_cross=False):
    """Frame loop around a timer poll "L: LDA INTIM; BNE L", entered after a
    joystick-dependent delay, so envs and steps poll from different timer
    phases.  timer_reg $94/$95/$96/$97 = TIM1T/TIM8T/TIM64T/T1024T."""
    def build(a):
        a.label("F")
        a.op("LDA", "imm", 2)
        a.op("STA", "zp", 0x02)
        a.op("STA", "zp", 0x00)
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", 0x00)
        a.op("LDA", "abs", 0x0280)       # SWCHA: delay of 0..15 loop turns
        a.op("LSR", "acc"); a.op("LSR", "acc"); a.op("LSR", "acc"); a.op("LSR", "acc")
        a.op("TAX")
        a.label("D")
        a.op("DEX")
        a.op("BPL", "rel", "D")
        a.op("LDA", "imm", value)
        a.op("STA", "abs", 0x0200 | timer_reg)
        a.op("JMP", "abs", "P")
        if page_cross:
            a.at(0x0FD)                   # LDA at $F0FD, BNE at $F100: the taken branch crosses a page
        a.label("P")
        a.op("LDA", "abs", 0x0284)
        a.op("BNE", "rel", "P")
        a.op("LDA", "abs", 0x0284)
        a.op("STA", "zp", 0x80)
        a.op("LDA", "abs", 0x0285)
        a.op("STA", "zp", 0x81)
        a.op("INC", "zp", 0x82)
        a.op("LDA", "zp", 0x82)
        a.op("STA", "zp", 0x09)
        a.op("STA", "zp", 0x02)
        a.op("STA", "zp", 0x08)
        a.op("JMP", "abs", "F")
    return rom4k(build)


def test_timer_poll_loops():
    """Poll loops at every timer interval: TIM64T and TIM8T (the loop lands in
    the zero window), TIM1T (a 7-cycle loop can step over the 1-cycle zero
    window and keeps polling after the underflow), T1024T with a wait longer
    than the 512-line watchdog (frames end inside the loop), and a loop
    whose taken branch crosses a page (8-cycle turns)."""
    roms = [_poll_rom(0x96, 43), _poll_rom(0x95, 200), _poll_rom(0x94, 101), _poll_rom(0x94, 250),
            _poll_rom(0x97, 100), _poll_rom(0x96, 37, page_cross=True), _poll_rom(0x97, 0)]
    maps = [synth.MAPPER_4K] * len(roms)
    env_cart = np.arange(3 * len(roms)) % len(roms)
    acts = synth.actions(707, len(env_cart), 8)
    _check_all(roms, maps, env_cart, acts, 2)


def _ram_code_rom():
    """Copies a routine into RAM and calls it every line (code executing from
    $0080 takes the bus-fetch path), and runs code in the last bytes of the
    cartridge window ($FFF0-$FFF9, also fetched through the bus)."""
    routine = [0xA9, 0x2A, 0x65, 0x91, 0x85, 0x09, 0xE6, 0x90, 0xA5, 0x90, 0x85, 0x08, 0x60]  # LDA #; ADC; STA; INC; LDA; STA; RTS

    def build(a):
        a.op("LDX", "imm", 0xFF)
        a.op("TXS")
        a.op("LDX", "imm", 0)
        a.label("C")
        a.op("LDA", "absx", "TAB")
        a.op("STA", "zpx", 0x80)
        a.op("INX")
        a.op("CPX", "imm", len(routine))
        a.op("BNE", "rel", "C")
        a.label("F")
        a.op("LDA", "imm", 2)
        a.op("STA", "zp", 0x02)
        a.op("STA", "zp", 0x00)
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", 0x00)
        a.op("LDA", "abs", 0x0280)
        a.op("STA", "zp", 0x91)
        a.op("LDY", "imm", 100)
        a.label("L")
        a.op("STA", "zp", 0x02)
        a.op("JSR", "abs", 0x0080)
        a.op("JMP", "abs", 0xFFF0)
        a.label("BACK")
        a.op("DEY")
        a.op("BNE", "rel", "L")
        a.op("JMP", "abs", "F")
        a.label("TAB")
        for b in routine:
            a.byte(b)
        a.at(0xFF0)                       # $FFF0: INC $92; LDA $92; STA $0E; JMP BACK (ends at $FFF8)
        a.op("INC", "zp", 0x92)
        a.op("LDA", "zp", 0x92)
        a.op("STA", "zp", 0x0E)
        a.byte(0x4C)
        a.word("BACK")
    return rom4k(build, table=False)


def _f8_window_end_rom():
    """F8 image whose bank-1 code falls through $FFF4..$FFF7: the opcode
    fetch at $FFF8 selects bank 0 (where it reads BNE), the operand fetch at
    $FFF9 selects bank 1 again (the offset comes from there), and the branch
    lands on a JMP back to the frame loop in bank 1."""
    def bank(b):
        a = synth.Asm(0xF000, 4096)
        if b == 1:
            a.label("F")
            a.op("LDA", "imm", 2)
            a.op("STA", "zp", 0x02)
            a.op("STA", "zp", 0x00)
            a.op("LDA", "imm", 0)
            a.op("STA", "zp", 0x00)
            a.op("LDX", "imm", 150)
            a.label("L")
            a.op("STA", "zp", 0x02)
            a.op("INC", "zp", 0x80)
            a.op("LDA", "zp", 0x80)
            a.op("STA", "zp", 0x09)
            a.op("DEX")
            a.op("BNE", "rel", "L")
            a.op("LDA", "imm", 1)              # Z clear: the BNE below is taken
            a.op("JMP", "abs", 0xFFF4)
            a.at(0xFE6)
            a.op("JMP", "abs", "F")            # $FFE6, the branch target
            a.at(0xFF4)
            for _ in range(4):
                a.op("NOP")                    # $FFF4-$FFF7
            a.byte(0xEA)                       # $FFF8 (not reached in this bank)
            a.byte(0xEC)                       # $FFF9: the branch offset, -20 -> $FFE6
        else:
            a.at(0xFF8)
            a.byte(0xD0)                       # $FFF8 in bank 0: BNE
            a.byte(0xEA)
        a.at(0xFFA)
        a.word(0xF000)
        a.word(0xF000)
        a.word(0xF000)
        return bytes(a.resolve())
    return bank(0) + bank(1)


def test_code_fetched_through_the_bus():
    """Code in RAM, in the last bytes of the 4 KB window and across the F8
    hotspots runs through the bus-fetch path; it must match the oracle."""
    roms = [_ram_code_rom(), _f8_window_end_rom()]
    maps = [synth.MAPPER_4K, synth.MAPPER_F8]
    env_cart = np.arange(8) % 2
    acts = synth.actions(717, 8, 6)
    _check_all(roms, maps, env_cart, acts, 2)


def _f8_nop_hotspot_rom():
    """An unofficial NOP absolute read of $1FF8 / $1FF9 switches F8 banks."""
    def bank(b):
        a = synth.Asm(0xF000, 4096)
        a.label("F")
        a.op("LDA", "imm", 2)
        a.op("STA", "zp", 0x02)
        a.op("STA", "zp", 0x00)
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", 0x00)
        a.op("LDX", "imm", 100)
        a.label("L")
        a.op("STA", "zp", 0x02)
        a.op("INC", "zp", 0x80 + b)
        a.op("LDA", "zp", 0x80 + b)
        a.op("STA", "zp", 0x09 if b else 0x08)
        a.op("DEX")
        a.op("BNE", "rel", "L")
        a.byte(0x0C, 0xF8 + (1 - b), 0xFF)   # NOP $FFF8 / $FFF9: switch to the other bank
        a.op("JMP", "abs", "F")
        a.at(0xFFA)
        a.word(0xF000)
        a.word(0xF000)
        a.word(0xF000)
        return bytes(a.resolve())
    return bank(0) + bank(1)


def test_extra_opcode_bytes():
    """The paper's 38 extra opcode bytes (USBC, unofficial NOPs, LAX, SAX)
    against the oracle, bit for bit, including an F8 bank switch by a NOP
    read."""
    roms = [extra_ops_rom(), _f8_nop_hotspot_rom()]
    maps = [synth.MAPPER_4K, synth.MAPPER_F8]
    env_cart = np.arange(10) % 2
    acts = synth.actions(738, 10, 6)
    _check_all(roms, maps, env_cart, acts, 2)
    b = make_batch(roms, maps, env_cart)
    _, _, st = gpu_rollout(b, acts, 2, screens=False)
    assert not np.any(st & 2), "no slot may jam"


def test_boot_protocol_and_episode_starts():
    """The paper's protocol on the GPU: 60 NOOP + 4 RESET boot frames after
    every power-on (creation, auto-reset, a masked reset), then each
    episode's own number of random start NOOPs; bit for bit against the
    oracle running the same sequence."""
    torch = torch_cuda()
    roms = [switches_rom(), synth.generate_cart(818, 1, synth.MAPPER_F8)]
    maps = [synth.MAPPER_4K, synth.MAPPER_F8]
    n = 12
    env_cart = np.arange(n) % 2
    acts = synth.actions(818, n, 12)
    ep = synth.episode_lengths(818, n, 4, mean_frames=10.0)
    starts = synth.start_noops(818, n, 4)
    b = make_batch(roms, maps, env_cart, boot_noop_frames=60, boot_reset_frames=4)
    b.set_start_noops(starts)
    b.reset()            # boot again, now with the start-noop table
    b.set_episodes(ep)
    ram, scr, st = gpu_rollout(b, acts, 2)
    assert np.any(st & 4), "some episodes must end inside the rollout"
    for e in range(n):
        c = int(env_cart[e])
        r2, s2, st2 = oracle_rollout(roms[c], maps[c], acts[:, e], 2, ep_len=ep[e], boot=(60, 4), start=starts[e])
        assert_env_equal(e, ram[:, e], r2, "RAM")
        assert_env_equal(e, scr[:, e], s2, "screen")
        assert_env_equal(e, st[:, e], st2, "status")
    # a masked reset powers on and boots env 0 alone, with the start count of
    # its current episode (a masked reset keeps the episode count)
    epi0 = int(np.count_nonzero(st[:, 0] & 4))
    mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
    mask[0] = 1
    b.reset(mask)
    ram2, _, _ = gpu_rollout(b, acts[:1], 2, screens=False)
    o = oracle.Oracle(roms[0], maps[0])
    o.boot(60, 4, int(starts[0][epi0 % 4]))
    r3, _, _ = o.step(int(acts[0, 0]), 2)
    assert np.array_equal(ram2[0, 0], r3)


def test_generated_carts_cover_the_instruction_set():
    """The seeded carts execute (nearly) every documented opcode."""
    seen = set()
    for mapper in (synth.MAPPER_2K, synth.MAPPER_4K, synth.MAPPER_F8):
        for c in range(3):
            o = oracle.Oracle(synth.generate_cart(707, c, mapper), mapper)
            tr = o.trace(3, 30000)
            seen |= set(int(x) for x in tr[:, 1])
    assert len(seen) >= 140, len(seen)


# ---------------------------------------------------------------------------
# batching features
# ---------------------------------------------------------------------------

def test_auto_reset_episodes():
    roms = synth.config_carts(808, [synth.MAPPER_2K, synth.MAPPER_4K, synth.MAPPER_F8])
    env_cart = np.array([0, 1, 2, 0, 1, 2], np.int32)
    ep = np.array([[3, 9, 5], [4, 4, 4], [10, 2, 7], [1, 1, 20], [6, 30, 2], [2, 5, 3]], np.uint32)
    b = make_batch(roms, [synth.MAPPER_2K, synth.MAPPER_4K, synth.MAPPER_F8], env_cart)
    b.set_episodes(ep)
    acts = synth.actions(808, 6, 12)
    ram, scr, st = gpu_rollout(b, acts, 2)
    for e in range(6):
        c = env_cart[e]
        r2, s2, st2 = oracle_rollout(roms[c], [0, 1, 2][c], acts[:, e], 2, ep_len=list(ep[e]))
        assert_env_equal(e, ram[:, e], r2, "RAM")
        assert_env_equal(e, scr[:, e], s2, "screen")
        assert_env_equal(e, st[:, e], st2, "status")


def test_step_host_and_state_roundtrip():
    torch = torch_cuda()
    rom = synth.generate_cart(909, 0, synth.MAPPER_F8)
    b = make_batch([rom], [synth.MAPPER_F8], [0] * 10)
    acts = synth.actions(909, 10, 4)
    blob = b.save_state()
    ram, scr, _ = gpu_rollout(b, acts, 2)
    b.load_state(blob)
    for t in range(4):
        rh = np.zeros((10, 128), np.uint8)
        sh = np.zeros((10, 210, 160), np.uint8)
        b.step_host(acts[t], 2, rh, sh)
        assert np.array_equal(rh, ram[t]) and np.array_equal(sh, scr[t])
    # the pipelined host rollout (two device buffer sets, copies overlapping
    # the next step) gives the same outputs, on pinned and pageable buffers
    for pinned in (True, False):
        b.load_state(blob)
        if pinned:
            rh = torch.zeros((4, 10, 128), dtype=torch.uint8).pin_memory().numpy()
            sh = torch.zeros((4, 10, 210, 160), dtype=torch.uint8).pin_memory().numpy()
        else:
            rh, sh = np.zeros((4, 10, 128), np.uint8), np.zeros((4, 10, 210, 160), np.uint8)
        th = np.zeros((4, 10), np.uint8)
        b.rollout_host(acts, 2, rh, sh, th)
        assert np.array_equal(rh, ram) and np.array_equal(sh, scr) and not th.any()
    # reset of a subset
    mask = torch.zeros(10, dtype=torch.uint8, device="cuda")
    mask[3] = 1
    b.reset(mask)
    ram2, _, _ = gpu_rollout(b, acts[:1], 2, screens=False)
    r3, _, _ = oracle_rollout(rom, synth.MAPPER_F8, acts[:1, 3], 2, screens=False)
    assert np.array_equal(ram2[0, 3], r3[0])


SC_MAPPERS = [synth.MAPPER_F8SC, synth.MAPPER_F6SC, synth.MAPPER_F4SC]


@pytest.mark.parametrize("epb,tpe", [(16, 1), (128, 1), (32, 4)])
def test_superchip_carts_match_oracle(epb, tpe):
    """F8SC, F6SC and F4SC carts next to plain ones in one batch: RAM,
    screens, status and the cartridge RAM (vcs_cart_ram) bit-exact, envs
    unsorted over several blocks and a ragged tail; a state blob round trip
    carries the cartridge RAM."""
    torch = torch_cuda()
    mappers = SC_MAPPERS + [synth.MAPPER_4K, synth.MAPPER_F8]
    roms = synth.config_carts(307, mappers)
    n_envs = 45
    env_cart = np.random.default_rng(7).permutation(np.arange(n_envs) % len(mappers)).astype(np.int32)
    acts = synth.actions(307, n_envs, 6)
    b = make_batch(roms, mappers, env_cart, envs_per_block=epb, threads_per_env=tpe)
    blob = b.save_state()
    ram, scr, st = gpu_rollout(b, acts, 2)
    cram = b.cart_ram().cpu().numpy()
    for e in range(n_envs):
        c = int(env_cart[e])
        o = oracle.Oracle(roms[c], mappers[c])
        for t in range(acts.shape[0]):
            r, s, stt = o.step(int(acts[t, e]), 2)
            assert_env_equal(e, ram[t, e], r, f"RAM step {t}")
            assert_env_equal(e, scr[t, e], s, f"screen step {t}")
            assert st[t, e] == stt
        assert_env_equal(e, cram[e], o.cart_ram(), "cartridge RAM")
        if mappers[c] in SC_MAPPERS:
            assert cram[e].any()
    b.load_state(blob)
    assert not b.cart_ram().cpu().numpy().any()
    ram2, _, _ = gpu_rollout(b, acts, 2, screens=False)
    assert np.array_equal(ram2, ram) and np.array_equal(b.cart_ram().cpu().numpy(), cram)


def test_superchip_ports_on_the_gpu():
    """The oracle's port pin on the GPU: writes through $1000-$107F, reads
    through $1080-$10FF plain and indexed, the write port reading ROM, the
    read port ignoring writes, a routine run from the cartridge RAM (fetched
    through the bus), in every Superchip format and as plain banked carts."""
    from tests.test_oracle_machine import _superchip_image
    for mapper in SC_MAPPERS:
        rom = _superchip_image(mapper)
        base = synth.MAPPER_SC_BASE[mapper]
        b = make_batch([rom, rom], [mapper, base], [0, 1, 0, 1])
        acts = synth.actions(308, 4, 2)
        ram, _, st = gpu_rollout(b, acts, 1, screens=False)
        cram = b.cart_ram().cpu().numpy()
        for e, m in enumerate((mapper, base, mapper, base)):
            r, _, s = oracle_rollout(rom, m, acts[:, e], 1, screens=False)
            assert_env_equal(e, ram[:, e], r, "RAM")
            assert_env_equal(e, st[:, e], s, "status")
        o = oracle.Oracle(rom, mapper)
        o.rollout(acts[:, 0], 1, screens=False)
        assert np.array_equal(cram[0], o.cart_ram()) and cram[0, 0x20] == 0xA9
        assert not cram[1].any()


@pytest.mark.parametrize("epb,tpe", [(16, 1), (64, 2)])
def test_e0_carts_match_oracle(epb, tpe):
    """E0 carts (slices mapped per frame from the joystick) next to
    Superchip and plain carts in one batch: RAM, screens and status
    bit-exact against the oracle, envs unsorted, several blocks."""
    mappers = [synth.MAPPER_E0, synth.MAPPER_E0, synth.MAPPER_F8SC, synth.MAPPER_2K]
    roms = synth.config_carts(309, mappers)
    env_cart = np.random.default_rng(9).permutation(np.arange(40) % len(mappers)).astype(np.int32)
    acts = synth.actions(309, 40, 8)
    _check_all(roms, mappers, env_cart, acts, 2, envs_per_block=epb, threads_per_env=tpe)


@pytest.mark.parametrize("epb,tpe", [(16, 1), (32, 4)])
def test_fe_carts_match_oracle(epb, tpe):
    """FE carts (a bank-1 or bank-0 kernel called each frame from the top
    of the stack, picked by the joystick) next to E0 and plain carts in one
    batch: RAM, screens and status bit-exact against the oracle."""
    mappers = [synth.MAPPER_FE, synth.MAPPER_FE, synth.MAPPER_E0, synth.MAPPER_4K]
    roms = synth.config_carts(311, mappers)
    env_cart = np.random.default_rng(11).permutation(np.arange(40) % len(mappers)).astype(np.int32)
    acts = synth.actions(311, 40, 8)
    _check_all(roms, mappers, env_cart, acts, 2, envs_per_block=epb, threads_per_env=tpe)


def test_fe_switching_on_the_gpu():
    """The oracle's FE pin on the GPU: JSR at the top of the stack, RTS,
    a deeper JSR and a plain push to $01FE, checked through the RAM each
    step leaves."""
    from tests.test_oracle_machine import _fe_image
    rom = _fe_image()
    acts = synth.actions(312, 2, 2)
    _check_all([rom], [synth.MAPPER_FE], [0, 0], acts, 1)


def test_e0_hotspots_on_the_gpu():
    """The oracle's E0 hotspot pin on the GPU (reads and writes of each
    segment's hotspots, neighbours and the image below A12 ignored), then
    a frame loop that remaps segments 0..2 through indexed hotspot reads
    and reads the mapped slices."""
    from tests.test_oracle_machine import _e0_image

    def program(a):
        a.at(0x100)
        a.op("LDA", "abs", 0x1FE2)
        a.op("STA", "abs", 0x1FEF)
        a.op("LDA", "abs", 0xFFF1)
        a.op("LDA", "abs", 0x1FDF)
        a.op("LDA", "abs", 0x1FF8)
        a.op("LDA", "abs", 0x0FE3)
        for seg, dst in ((0, 0x84), (1, 0x85), (2, 0x86), (3, 0x87)):
            a.op("LDA", "abs", 0x1000 + 0x400 * seg)
            a.op("STA", "zp", dst)
        a.label("FRAME")
        a.op("LDA", "imm", 2)
        a.op("STA", "zp", 0x02)
        a.op("STA", "zp", 0x00)
        a.op("LDA", "imm", 0)
        a.op("STA", "zp", 0x00)
        a.op("LDX", "imm", 0)
        a.label("L")
        a.op("STA", "zp", 0x02)
        a.op("LDA", "absx", 0x1FE0)             # X < 24: segment X / 8 <- slice X % 8
        a.op("LDA", "absx", 0x1000)             # byte X of segment 0
        a.op("STA", "zp", 0x09)
        a.op("INX")
        a.op("BNE", "rel", "L")
        a.op("JMP", "abs", "FRAME")
    rom = _e0_image(program)
    acts = synth.actions(310, 3, 3)
    _check_all([rom], [synth.MAPPER_E0], [0, 0, 0], acts, 1)
