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

// Execute one instruction slot (an instruction, or for a jammed CPU an idle
// to the next line start) and advance the clocks.
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
  const uint32_t op = bus_read(c, r, st, opaddr, 1);
  const uint32_t mc = c.dt->mode_cyc[op];
  const uint32_t mode = mc & 15;
  uint32_t n = mc >> 4;
  const uint32_t pc1 = (opaddr + 1) & 0xFFFF;
  uint32_t ea = 0;
  bool cross = false;
  switch (mode) {
    case AM_IMP:
    case AM_ACC:
      r.PC = pc1;
      break;
    case AM_IMM:
      ea = pc1;
      r.PC = (opaddr + 2) & 0xFFFF;
      break;
    case AM_ZP:
      ea = bus_read(c, r, st, pc1, 2);
      r.PC = (opaddr + 2) & 0xFFFF;
      break;
    case AM_ZPX:
      ea = (bus_read(c, r, st, pc1, 2) + r.X) & 0xFF;
      r.PC = (opaddr + 2) & 0xFFFF;
      break;
    case AM_ZPY:
      ea = (bus_read(c, r, st, pc1, 2) + r.Y) & 0xFF;
      r.PC = (opaddr + 2) & 0xFFFF;
      break;
    case AM_ABS:
    case AM_ABX:
    case AM_ABY: {
      uint32_t lo = bus_read(c, r, st, pc1, 2);
      uint32_t hi = bus_read(c, r, st, (opaddr + 2) & 0xFFFF, 3);
      uint32_t base = lo | (hi << 8);
      ea = (base + (mode == AM_ABX ? r.X : (mode == AM_ABY ? r.Y : 0u))) & 0xFFFF;
      cross = ((base ^ ea) & 0xFF00) != 0;
      r.PC = (opaddr + 3) & 0xFFFF;
      break;
    }
    case AM_INX: {
      uint32_t p = (bus_read(c, r, st, pc1, 2) + r.X) & 0xFF;
      uint32_t lo = bus_read(c, r, st, p, 4);
      uint32_t hi = bus_read(c, r, st, (p + 1) & 0xFF, 5);
      ea = lo | (hi << 8);
      r.PC = (opaddr + 2) & 0xFFFF;
      break;
    }
    case AM_INY: {
      uint32_t z = bus_read(c, r, st, pc1, 2);
      uint32_t lo = bus_read(c, r, st, z, 3);
      uint32_t hi = bus_read(c, r, st, (z + 1) & 0xFF, 4);
      uint32_t base = lo | (hi << 8);
      ea = (base + r.Y) & 0xFFFF;
      cross = ((base ^ ea) & 0xFF00) != 0;
      r.PC = (opaddr + 2) & 0xFFFF;
      break;
    }
    case AM_REL:
    case AM_IND:
      break;
    default:  // undocumented opcode: the CPU jams after the fetch
      r.PC = pc1;
      r.jam = 1;
      r.cyc += 1;
      r.fc += 1;
      return;
  }

  // read-class instructions pay the page-cross cycle and read last
  const uint32_t rcyc = n + (cross ? 1u : 0u);
  uint32_t tref = ea, tfl = 0;
  // pending writes: nw bytes of wv (low byte first) at cycles widx, widx+1,
  // ... to wea, or to the stack (0x100 | SP, descending) when wstack
  uint32_t nw = 0, wea = ea, wv = 0, widx = n;
  bool wstack = false;
  switch (op) {
    // ---- loads ----
    case 0xA9: case 0xA5: case 0xB5: case 0xAD: case 0xBD: case 0xB9: case 0xA1: case 0xB1:
      n = rcyc;
      r.A = bus_read(c, r, st, ea, (int)n);
      set_nz(r, r.A);
      break;
    case 0xA2: case 0xA6: case 0xB6: case 0xAE: case 0xBE:
      n = rcyc;
      r.X = bus_read(c, r, st, ea, (int)n);
      set_nz(r, r.X);
      break;
    case 0xA0: case 0xA4: case 0xB4: case 0xAC: case 0xBC:
      n = rcyc;
      r.Y = bus_read(c, r, st, ea, (int)n);
      set_nz(r, r.Y);
      break;
    // ---- ALU ----
    case 0x09: case 0x05: case 0x15: case 0x0D: case 0x1D: case 0x19: case 0x01: case 0x11:
      n = rcyc;
      r.A |= bus_read(c, r, st, ea, (int)n);
      set_nz(r, r.A);
      break;
    case 0x29: case 0x25: case 0x35: case 0x2D: case 0x3D: case 0x39: case 0x21: case 0x31:
      n = rcyc;
      r.A &= bus_read(c, r, st, ea, (int)n);
      set_nz(r, r.A);
      break;
    case 0x49: case 0x45: case 0x55: case 0x4D: case 0x5D: case 0x59: case 0x41: case 0x51:
      n = rcyc;
      r.A ^= bus_read(c, r, st, ea, (int)n);
      set_nz(r, r.A);
      break;
    case 0x69: case 0x65: case 0x75: case 0x6D: case 0x7D: case 0x79: case 0x61: case 0x71:
      n = rcyc;
      do_adc(r, bus_read(c, r, st, ea, (int)n));
      break;
    case 0xE9: case 0xE5: case 0xF5: case 0xED: case 0xFD: case 0xF9: case 0xE1: case 0xF1:
      n = rcyc;
      do_sbc(r, bus_read(c, r, st, ea, (int)n));
      break;
    case 0xC9: case 0xC5: case 0xD5: case 0xCD: case 0xDD: case 0xD9: case 0xC1: case 0xD1:
      n = rcyc;
      do_cmp(r, r.A, bus_read(c, r, st, ea, (int)n));
      break;
    case 0xE0: case 0xE4: case 0xEC:
      do_cmp(r, r.X, bus_read(c, r, st, ea, (int)n));
      break;
    case 0xC0: case 0xC4: case 0xCC:
      do_cmp(r, r.Y, bus_read(c, r, st, ea, (int)n));
      break;
    case 0x24: case 0x2C: {
      uint32_t m = bus_read(c, r, st, ea, (int)n);
      r.nsrc = m & 0x80;
      r.fV = (m >> 6) & 1;
      r.zsrc = r.A & m;
      break;
    }
    // ---- stores ----
    case 0x85: case 0x95: case 0x8D: case 0x9D: case 0x99: case 0x81: case 0x91:
      nw = 1; wv = r.A;
      break;
    case 0x86: case 0x96: case 0x8E:
      nw = 1; wv = r.X;
      break;
    case 0x84: case 0x94: case 0x8C:
      nw = 1; wv = r.Y;
      break;
    // ---- read-modify-write ----
    case 0x0A: r.A = do_shift(r, 0, r.A); break;
    case 0x2A: r.A = do_shift(r, 1, r.A); break;
    case 0x4A: r.A = do_shift(r, 2, r.A); break;
    case 0x6A: r.A = do_shift(r, 3, r.A); break;
    case 0x06: case 0x16: case 0x0E: case 0x1E:
    case 0x26: case 0x36: case 0x2E: case 0x3E:
    case 0x46: case 0x56: case 0x4E: case 0x5E:
    case 0x66: case 0x76: case 0x6E: case 0x7E:
    case 0xC6: case 0xD6: case 0xCE: case 0xDE:
    case 0xE6: case 0xF6: case 0xEE: case 0xFE: {
      uint32_t m = bus_read(c, r, st, ea, (int)n - 2);
      uint32_t k = op >> 5;
      if (k < 4) {
        wv = do_shift(r, k, m);
      } else {
        wv = (k == 6 ? m - 1 : m + 1) & 0xFF;
        set_nz(r, wv);
      }
      nw = 1;
      break;
    }
    // ---- branches ----
    case 0x10: case 0x30: case 0x50: case 0x70: case 0x90: case 0xB0: case 0xD0: case 0xF0: {
      uint32_t off = bus_read(c, r, st, pc1, 2);
      uint32_t next = (opaddr + 2) & 0xFFFF;
      uint32_t flag;
      switch (op >> 6) {
        case 0: flag = (r.nsrc >> 7) & 1; break;
        case 1: flag = r.fV; break;
        case 2: flag = r.fC; break;
        default: flag = (r.zsrc & 0xFF) == 0 ? 1u : 0u; break;
      }
      uint32_t taken = ((op >> 5) & 1) == flag ? 1u : 0u;
      r.PC = next;
      if (taken) {
        uint32_t t = (next + (uint32_t)(int32_t)(int8_t)(uint8_t)off) & 0xFFFF;
        n += 1 + (((t ^ next) & 0xFF00) ? 1u : 0u);
        r.PC = t;
      }
      tref = pc1;
      tfl = taken;
      break;
    }
    // ---- jumps / subroutines ----
    case 0x4C:
      r.PC = ea;
      break;
    case 0x6C: {
      uint32_t lo = bus_read(c, r, st, pc1, 2);
      uint32_t hi = bus_read(c, r, st, (opaddr + 2) & 0xFFFF, 3);
      uint32_t p = lo | (hi << 8);
      uint32_t l2 = bus_read(c, r, st, p, 4);
      uint32_t h2 = bus_read(c, r, st, (p & 0xFF00) | ((p + 1) & 0xFF), 5);
      r.PC = l2 | (h2 << 8);
      break;
    }
    case 0x20: {
      uint32_t lo = bus_read(c, r, st, pc1, 2);
      uint32_t ret = (opaddr + 2) & 0xFFFF;
      uint32_t hi = bus_read(c, r, st, ret, 6);
      r.PC = lo | (hi << 8);
      nw = 2; wstack = true; wv = (ret >> 8) | ((ret & 0xFF) << 8); widx = 4;
      break;
    }
    case 0x60: {
      uint32_t lo = pull(c, r, st, 4);
      uint32_t hi = pull(c, r, st, 5);
      r.PC = ((lo | (hi << 8)) + 1) & 0xFFFF;
      break;
    }
    case 0x40: {
      uint32_t p = pull(c, r, st, 4);
      uint32_t lo = pull(c, r, st, 5);
      uint32_t hi = pull(c, r, st, 6);
      unpack_p(r, p | 0x30);
      r.PC = lo | (hi << 8);
      break;
    }
    case 0x00: {
      uint32_t ret = (opaddr + 2) & 0xFFFF;
      nw = 3; wstack = true; wv = (ret >> 8) | ((ret & 0xFF) << 8) | (pack_p(r) << 16); widx = 3;
      r.fI = 1;
      uint32_t lo = bus_read(c, r, st, 0xFFFE, 6);
      uint32_t hi = bus_read(c, r, st, 0xFFFF, 7);
      r.PC = lo | (hi << 8);
      break;
    }
    // ---- stack ----
    case 0x48: nw = 1; wstack = true; wv = r.A; widx = 3; break;
    case 0x08: nw = 1; wstack = true; wv = pack_p(r); widx = 3; break;
    case 0x68:
      r.A = pull(c, r, st, 4);
      set_nz(r, r.A);
      tref = 0x100u | r.SP;
      break;
    case 0x28:
      unpack_p(r, pull(c, r, st, 4) | 0x30);
      break;
    // ---- flags and register transfers ----
    case 0x18: r.fC = 0; break;
    case 0x38: r.fC = 1; break;
    case 0x58: r.fI = 0; break;
    case 0x78: r.fI = 1; break;
    case 0xB8: r.fV = 0; break;
    case 0xD8: r.fD = 0; break;
    case 0xF8: r.fD = 1; break;
    case 0xEA: break;
    case 0xAA: r.X = r.A; set_nz(r, r.X); break;
    case 0x8A: r.A = r.X; set_nz(r, r.A); break;
    case 0xA8: r.Y = r.A; set_nz(r, r.Y); break;
    case 0x98: r.A = r.Y; set_nz(r, r.A); break;
    case 0xBA: r.X = r.SP; set_nz(r, r.X); break;
    case 0x9A: r.SP = r.X; break;
    case 0xE8: r.X = (r.X + 1) & 0xFF; set_nz(r, r.X); break;
    case 0xCA: r.X = (r.X - 1) & 0xFF; set_nz(r, r.X); break;
    case 0xC8: r.Y = (r.Y + 1) & 0xFF; set_nz(r, r.Y); break;
    case 0x88: r.Y = (r.Y - 1) & 0xFF; set_nz(r, r.Y); break;
    default: break;
  }
  if (wstack) tref = 0x100u | r.SP;
  for (uint32_t i = 0; i < nw; i++) {
    uint32_t addr = wea;
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
