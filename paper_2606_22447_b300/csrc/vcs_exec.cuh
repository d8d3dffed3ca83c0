// Instruction execution for the per-thread VCS machine (see vcs_machine.cuh).
//
// Bus timing: an instruction starting at cycle t makes its k-th bus access
// at cycle t + k (the cycle is charged before the access).  Only accesses
// whose effect depends on time carry k: TIA and timer writes and INTIM /
// TIMINT reads.  Data reads happen on the instruction's last cycle (after
// any page-cross penalty), stores on the last cycle, read-modify-write
// instructions read two cycles before their final write, and pushes / pulls
// sit on the cycles of the MOS cycle-by-cycle sequences.  Dummy reads and
// the RMW dummy write have no side effect.
//
// All writes of an instruction go through one call site at its end, in bus
// order.  This is exact: the only reads that follow a write inside one
// instruction are JSR's high-byte fetch and BRK's vector fetch, both from
// the cartridge, which no stack write can reach.  A frame that a VSYNC write
// ends is closed after the instruction, which is also exact: the stack
// writes that can follow a VSYNC write in one instruction land on TIA
// register $3F or in RAM, neither of which is drawn.
#pragma once
#include "vcs_machine.cuh"

namespace vcs {

struct Step {
  int32_t frames_done;
  int32_t frame_skip;
  int32_t stall;       // WSYNC cycles added inside the current instruction
  int32_t fe_at;       // frame cycle of a VSYNC frame end in this instruction, or -1
  uint32_t status;     // kSt* bits of this step
  bool want_screen;
};

// TIA write registers whose value changes the picture.
constexpr uint64_t kVisualRegs = (1ull << 0x01) | (1ull << 0x06) | (1ull << 0x08) | (1ull << 0x09) |
                                 (1ull << 0x0A) | (1ull << 0x0D) | (1ull << 0x0E) | (1ull << 0x0F) |
                                 (1ull << 0x10) | (1ull << 0x1B) | (1ull << 0x2A);

template <class Tape>
__device__ __forceinline__ void tia_write(const Ctx& c, Regs& r, Render& rd, Step& st, Tape& tape, uint32_t reg,
                                          uint32_t v, int32_t fcw) {
  if (((kVisualRegs >> reg) & 1) && rd.on) render_to(c, r, rd, tape, 3 * fcw);
  switch (reg) {
    case 0x00:
      if (!(r.vsync & 2) && (v & 2)) st.fe_at = fcw;
      r.vsync = v;
      break;
    case 0x01: r.vblank = v; break;
    case 0x02: {
      uint32_t m = (uint32_t)fcw % 76u;
      if (m) st.stall += 76 - (int32_t)m;
      break;
    }
    case 0x06: tape.colour_write(0); r.col0 = v; break;
    case 0x08: tape.colour_write(1); r.colpf = v; break;
    case 0x09: tape.colour_write(2); r.colbk = v; break;
    case 0x0A: r.ctrl = v; break;
    case 0x0D: r.pf0 = v; break;
    case 0x0E: r.pf1 = v; break;
    case 0x0F: r.pf2 = v; break;
    case 0x10: {
      uint32_t h = 3u * ((uint32_t)fcw % 76u);
      r.pos = h < 68 ? 3u : (h - 68u + 5u) % 160u;
      break;
    }
    case 0x1B: r.grp0 = v; break;
    case 0x20: r.hmp0 = v; break;
    case 0x2A: {
      int32_t m = ((int32_t)(int8_t)(uint8_t)r.hmp0) >> 4;
      r.pos = (uint32_t)(((int32_t)r.pos - m + 160) % 160);
      uint32_t h = 3u * ((uint32_t)fcw % 76u);
      if (h <= 9) r.hml = (int32_t)div76((uint32_t)fcw);
      break;
    }
    case 0x2B: r.hmp0 = 0; break;
    default: break;
  }
}

// One bus read at cycle index idx of the current instruction.  A read of
// INTIM also records whether the timer had underflowed (r.intim_live), which
// the soft path's tape keeps for the backward sweep.
__device__ __forceinline__ uint32_t bus_read(const Ctx& c, Regs& r, const Step& st, uint32_t addr, int idx) {
  uint32_t a = addr & 0x1FFF;
  if (a & 0x1000) {
    if (c.f8 && (a & 0x1FFE) == 0x1FF8) r.bank = a & 1;
    return c.rom[(r.bank << 12) | (a & 0xFFF)];
  }
  if (!(a & 0x80)) {
    uint32_t q = a & 0xF;
    return q == 0xC ? r.inpt4 : (q == 0xD ? 0x80u : 0u);
  }
  if (!(a & 0x200)) return ram_rd(c, a);
  if (!(a & 4)) {
    uint32_t q = a & 3;
    return q == 0 ? r.swcha : (q == 2 ? 0x0Bu : 0u);
  }
  uint32_t t = r.cyc + (uint32_t)(idx + st.stall);
  if (a & 1) return timint_at(r, t);
  r.intim_live = (t - r.tw) <= (r.tv << r.tsh) ? 1u : 0u;
  return intim_at(r, t);
}

template <class Tape>
__device__ __forceinline__ void bus_write(const Ctx& c, Regs& r, Render& rd, Step& st, Tape& tape, uint32_t addr,
                                          uint32_t v, int idx) {
  uint32_t a = addr & 0x1FFF;
  if (a & 0x1000) {
    if (c.f8 && (a & 0x1FFE) == 0x1FF8) r.bank = a & 1;
    return;
  }
  if (!(a & 0x80)) {
    tia_write(c, r, rd, st, tape, a & 0x3F, v & 0xFF, r.fc + idx + st.stall);
    return;
  }
  if (!(a & 0x200)) {
    ram_wr(c, a, v);
    return;
  }
  if ((a & 0x14) == 0x14) {
    r.tw = r.cyc + (uint32_t)(idx + st.stall);
    r.tv = v & 0xFF;
    r.tsh = (0x0A060300u >> (8 * (a & 3))) & 0xFF;
  }
}

__device__ __forceinline__ void set_nz(Regs& r, uint32_t v) {
  r.zsrc = v & 0xFF;
  r.nsrc = v & 0xFF;
}

__device__ __forceinline__ void do_adc(Regs& r, uint32_t m) {
  uint32_t a = r.A, cin = r.fC;
  if (r.fD) {
    // NMOS decimal mode (published decimal-mode note): nibble-wise adjust,
    // N and V from the signed intermediate, Z from the binary sum.
    int32_t al = (int32_t)(a & 0xF) + (int32_t)(m & 0xF) + (int32_t)cin;
    if (al >= 0xA) al = ((al + 6) & 0xF) + 0x10;
    int32_t s = (int32_t)(a & 0xF0) + (int32_t)(m & 0xF0) + al;
    int32_t ss = (int32_t)(int8_t)(uint8_t)(a & 0xF0) + (int32_t)(int8_t)(uint8_t)(m & 0xF0) + al;
    r.nsrc = (uint32_t)ss & 0x80;
    r.fV = (ss < -128 || ss > 127) ? 1u : 0u;
    r.zsrc = (a + m + cin) & 0xFF;
    if (s >= 0xA0) s += 0x60;
    r.fC = s >= 0x100 ? 1u : 0u;
    r.A = (uint32_t)s & 0xFF;
  } else {
    uint32_t t = a + m + cin;
    uint32_t res = t & 0xFF;
    r.fC = t >> 8;
    r.fV = ((~(a ^ m) & (a ^ res)) >> 7) & 1;
    r.A = res;
    set_nz(r, res);
  }
}

__device__ __forceinline__ void do_sbc(Regs& r, uint32_t m) {
  uint32_t a = r.A, cin = r.fC;
  uint32_t t = a + (m ^ 0xFF) + cin;
  uint32_t res = t & 0xFF;
  r.fC = t >> 8;
  r.fV = ((~(a ^ (m ^ 0xFF)) & (a ^ res)) >> 7) & 1;
  set_nz(r, res);
  if (r.fD) {
    int32_t al = (int32_t)(a & 0xF) - (int32_t)(m & 0xF) + (int32_t)cin - 1;
    if (al < 0) al = ((al - 6) & 0xF) - 0x10;
    int32_t s = (int32_t)(a & 0xF0) - (int32_t)(m & 0xF0) + al;
    if (s < 0) s -= 0x60;
    res = (uint32_t)s & 0xFF;
  }
  r.A = res;
}

__device__ __forceinline__ void do_cmp(Regs& r, uint32_t reg, uint32_t m) {
  r.fC = reg >= m ? 1u : 0u;
  set_nz(r, (reg - m) & 0xFF);
}

// Shift/rotate: k = 0 ASL, 1 ROL, 2 LSR, 3 ROR.
__device__ __forceinline__ uint32_t do_shift(Regs& r, uint32_t k, uint32_t v) {
  uint32_t cin = r.fC, res;
  if (k < 2) {
    r.fC = (v >> 7) & 1;
    res = ((v << 1) | (k == 1 ? cin : 0u)) & 0xFF;
  } else {
    r.fC = v & 1;
    res = (v >> 1) | (k == 3 ? (cin << 7) : 0u);
  }
  set_nz(r, res);
  return res;
}

__device__ __forceinline__ uint32_t pull(const Ctx& c, Regs& r, Step& st, int idx) {
  r.SP = (r.SP + 1) & 0xFF;
  return bus_read(c, r, st, 0x100u | r.SP, idx);
}

// Tape hook: called once per executed instruction with its opcode, a
// reference address and flag bits (the soft path records these; the hard
// path compiles the hook away).
struct NoTape {
  static constexpr bool kAcc = false;
  __device__ __forceinline__ void rec(uint32_t, uint32_t, uint32_t) {}
  __device__ __forceinline__ void colour_write(int) {}
  __device__ __forceinline__ void pixels(float, float, float) {}
};

// Instruction length of each addressing mode, two bits per mode.
constexpr uint32_t kModeLen = 1u | (1u << 2) | (2u << 4) | (2u << 6) | (2u << 8) | (2u << 10) | (3u << 12) |
                              (3u << 14) | (3u << 16) | (2u << 18) | (2u << 20) | (2u << 22) | (3u << 24) |
                              (1u << 26);

// Execute one instruction slot (an instruction, or for a jammed CPU an idle
// to the next line start) and advance the clocks.
//
// Fetch: inside the cartridge and away from the F8 hotspots and the end of
// the 4 KB window the opcode and both operand bytes are read at once (three
// independent shared-memory loads; such reads have no side effect and do not
// depend on time).  Elsewhere the operand bytes are real bus accesses and are
// read one by one, only as many as the instruction has.  Each instruction
// then makes at most one data read (read and read-modify-write classes) and
// its writes, through single call sites.
template <class Tape>
__device__ __forceinline__ void exec_one(const Ctx& c, Regs& r, Render& rd, Step& st, Tape& tape) {
  if (r.jam) {
    uint32_t d = 76u - (uint32_t)r.fc % 76u;
    r.cyc += d;
    r.fc += (int32_t)d;
    return;
  }
  const uint32_t opaddr = r.PC;
  r.intim_live = 0;
  const uint32_t off = opaddr & 0xFFF;
  const bool fast = (opaddr & 0x1000) != 0 && off <= 0xFF5;
  uint32_t op, b1 = 0, b2 = 0;
  if (fast) {
    const uint8_t* q = c.rom + ((r.bank << 12) | off);
    op = q[0];
    b1 = q[1];
    b2 = q[2];
  } else {
    op = bus_read(c, r, st, opaddr, 1);
  }
  const uint32_t mc = c.dt->mode_cyc[op], co = c.dt->cls_op[op];
  const uint32_t mode = mc & 15, cls = co & 3, id = co >> 2;
  uint32_t n = mc >> 4;
  const uint32_t len = (kModeLen >> (2 * mode)) & 3;
  const uint32_t pc1 = (opaddr + 1) & 0xFFFF;
  if (!fast) {
    if (len >= 2) b1 = bus_read(c, r, st, pc1, 2);
    if (len >= 3) b2 = bus_read(c, r, st, (opaddr + 2) & 0xFFFF, id == OP_JSR ? 6 : 3);
  }
  if (mode == AM_JAM) {   // undocumented opcode: the CPU jams after the fetch
    r.PC = pc1;
    r.jam = 1;
    r.cyc += 1;
    r.fc += 1;
    return;
  }
  r.PC = (opaddr + len) & 0xFFFF;
  uint32_t ea = 0;
  bool cross = false;
  switch (mode) {
    case AM_IMM: ea = pc1; break;
    case AM_ZP: ea = b1; break;
    case AM_ZPX: ea = (b1 + r.X) & 0xFF; break;
    case AM_ZPY: ea = (b1 + r.Y) & 0xFF; break;
    case AM_ABS: ea = b1 | (b2 << 8); break;
    case AM_ABX:
    case AM_ABY: {
      const uint32_t base = b1 | (b2 << 8);
      ea = (base + (mode == AM_ABX ? r.X : r.Y)) & 0xFFFF;
      cross = ((base ^ ea) & 0xFF00) != 0;
      break;
    }
    case AM_INX: {
      const uint32_t p = (b1 + r.X) & 0xFF;
      const uint32_t lo = bus_read(c, r, st, p, 4);
      const uint32_t hi = bus_read(c, r, st, (p + 1) & 0xFF, 5);
      ea = lo | (hi << 8);
      break;
    }
    case AM_INY: {
      const uint32_t lo = bus_read(c, r, st, b1, 3);
      const uint32_t hi = bus_read(c, r, st, (b1 + 1) & 0xFF, 4);
      const uint32_t base = lo | (hi << 8);
      ea = (base + r.Y) & 0xFFFF;
      cross = ((base ^ ea) & 0xFF00) != 0;
      break;
    }
    default: break;
  }

  // the one data read: read-class instructions read on their last cycle
  // (after any page-cross cycle), read-modify-write two cycles before the end
  uint32_t m = 0;
  if (cls == CL_READ) {
    n += cross ? 1u : 0u;
    m = mode == AM_IMM ? b1 : bus_read(c, r, st, ea, (int)n);
  } else if (cls == CL_RMW) {
    m = bus_read(c, r, st, ea, (int)n - 2);
  }
  uint32_t tref = ea, tfl = 0;
  // pending writes: nw bytes of wv (low byte first) at cycles widx, widx+1,
  // ... to ea, or to the stack (0x100 | SP, descending) when wstack
  uint32_t nw = 0, wv = 0, widx = n;
  bool wstack = false;
  switch (id) {
    case OP_LDA: r.A = m; set_nz(r, m); break;
    case OP_LDX: r.X = m; set_nz(r, m); break;
    case OP_LDY: r.Y = m; set_nz(r, m); break;
    case OP_ORA: r.A |= m; set_nz(r, r.A); break;
    case OP_AND: r.A &= m; set_nz(r, r.A); break;
    case OP_EOR: r.A ^= m; set_nz(r, r.A); break;
    case OP_ADC: do_adc(r, m); break;
    case OP_SBC: do_sbc(r, m); break;
    case OP_CMP: do_cmp(r, r.A, m); break;
    case OP_CPX: do_cmp(r, r.X, m); break;
    case OP_CPY: do_cmp(r, r.Y, m); break;
    case OP_BIT:
      r.nsrc = m & 0x80;
      r.fV = (m >> 6) & 1;
      r.zsrc = r.A & m;
      break;
    case OP_STA: nw = 1; wv = r.A; break;
    case OP_STX: nw = 1; wv = r.X; break;
    case OP_STY: nw = 1; wv = r.Y; break;
    case OP_ASL: case OP_ROL: case OP_LSR: case OP_ROR:
      wv = do_shift(r, id - OP_ASL, m);
      nw = 1;
      break;
    case OP_DEC: case OP_INC:
      wv = (id == OP_DEC ? m - 1 : m + 1) & 0xFF;
      set_nz(r, wv);
      nw = 1;
      break;
    case OP_ASLA: case OP_ROLA: case OP_LSRA: case OP_RORA:
      r.A = do_shift(r, id - OP_ASLA, r.A);
      break;
    case OP_BRANCH: {
      uint32_t flag;
      switch (op >> 6) {
        case 0: flag = (r.nsrc >> 7) & 1; break;
        case 1: flag = r.fV; break;
        case 2: flag = r.fC; break;
        default: flag = (r.zsrc & 0xFF) == 0 ? 1u : 0u; break;
      }
      const uint32_t taken = ((op >> 5) & 1) == flag ? 1u : 0u;
      if (taken) {
        const uint32_t next = r.PC;
        const uint32_t t = (next + (uint32_t)(int32_t)(int8_t)(uint8_t)b1) & 0xFFFF;
        n += 1 + (((t ^ next) & 0xFF00) ? 1u : 0u);
        r.PC = t;
      }
      tref = pc1;
      tfl = taken;
      break;
    }
    case OP_JMP: r.PC = ea; break;
    case OP_JMPI: {
      const uint32_t p = b1 | (b2 << 8);
      const uint32_t l2 = bus_read(c, r, st, p, 4);
      const uint32_t h2 = bus_read(c, r, st, (p & 0xFF00) | ((p + 1) & 0xFF), 5);
      r.PC = l2 | (h2 << 8);
      break;
    }
    case OP_JSR: {
      const uint32_t ret = (opaddr + 2) & 0xFFFF;
      r.PC = b1 | (b2 << 8);
      nw = 2; wstack = true; wv = (ret >> 8) | ((ret & 0xFF) << 8); widx = 4;
      break;
    }
    case OP_RTS: {
      const uint32_t lo = pull(c, r, st, 4);
      const uint32_t hi = pull(c, r, st, 5);
      r.PC = ((lo | (hi << 8)) + 1) & 0xFFFF;
      break;
    }
    case OP_RTI: {
      const uint32_t p = pull(c, r, st, 4);
      const uint32_t lo = pull(c, r, st, 5);
      const uint32_t hi = pull(c, r, st, 6);
      unpack_p(r, p | 0x30);
      r.PC = lo | (hi << 8);
      break;
    }
    case OP_BRK: {
      const uint32_t ret = (opaddr + 2) & 0xFFFF;
      nw = 3; wstack = true; wv = (ret >> 8) | ((ret & 0xFF) << 8) | (pack_p(r) << 16); widx = 3;
      r.fI = 1;
      const uint32_t lo = bus_read(c, r, st, 0xFFFE, 6);
      const uint32_t hi = bus_read(c, r, st, 0xFFFF, 7);
      r.PC = lo | (hi << 8);
      break;
    }
    case OP_PHA: nw = 1; wstack = true; wv = r.A; widx = 3; break;
    case OP_PHP: nw = 1; wstack = true; wv = pack_p(r); widx = 3; break;
    case OP_PLA:
      r.A = pull(c, r, st, 4);
      set_nz(r, r.A);
      tref = 0x100u | r.SP;
      break;
    case OP_PLP: unpack_p(r, pull(c, r, st, 4) | 0x30); break;
    case OP_CLC: r.fC = 0; break;
    case OP_SEC: r.fC = 1; break;
    case OP_CLI: r.fI = 0; break;
    case OP_SEI: r.fI = 1; break;
    case OP_CLV: r.fV = 0; break;
    case OP_CLD: r.fD = 0; break;
    case OP_SED: r.fD = 1; break;
    case OP_TAX: r.X = r.A; set_nz(r, r.X); break;
    case OP_TXA: r.A = r.X; set_nz(r, r.A); break;
    case OP_TAY: r.Y = r.A; set_nz(r, r.Y); break;
    case OP_TYA: r.A = r.Y; set_nz(r, r.A); break;
    case OP_TSX: r.X = r.SP; set_nz(r, r.X); break;
    case OP_TXS: r.SP = r.X; break;
    case OP_INX: r.X = (r.X + 1) & 0xFF; set_nz(r, r.X); break;
    case OP_DEX: r.X = (r.X - 1) & 0xFF; set_nz(r, r.X); break;
    case OP_INY: r.Y = (r.Y + 1) & 0xFF; set_nz(r, r.Y); break;
    case OP_DEY: r.Y = (r.Y - 1) & 0xFF; set_nz(r, r.Y); break;
    default: break;   // NOP
  }
  if (wstack) tref = 0x100u | r.SP;
  for (uint32_t i = 0; i < nw; i++) {
    uint32_t addr = ea;
    if (wstack) {
      addr = 0x100u | r.SP;
      r.SP = (r.SP - 1) & 0xFF;
    }
    bus_write(c, r, rd, st, tape, addr, (wv >> (8 * i)) & 0xFF, (int)(widx + i));
  }
  tape.rec(op, tref, tfl | (r.bank << 1) | (r.intim_live << 2));
  r.cyc += n + (uint32_t)st.stall;
  r.fc += (int32_t)n + st.stall;
  st.stall = 0;
}

}  // namespace vcs
