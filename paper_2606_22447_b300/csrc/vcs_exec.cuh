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
#include <initializer_list>
#include <type_traits>

#include "vcs_machine.cuh"
#include "vcs_tia.cuh"

namespace vcs {

struct Step {
  int32_t frames_done;
  int32_t frame_skip;
  int32_t stall;       // WSYNC cycles added inside the current instruction
  int32_t fe_at;       // frame cycle of a VSYNC frame end in this instruction, or -1
  uint32_t status;     // kSt* bits of this step
  bool want_screen;
  int32_t instr_left;  // instruction-granular steps: slots left in the step
};

constexpr uint64_t reg_bits(std::initializer_list<int> regs) {
  uint64_t m = 0;
  for (int r : regs) m |= 1ull << r;
  return m;
}

// TIA write registers whose value changes the picture: of the subset
// machine, and of the whole TIA.
constexpr uint64_t kVisualSubset = reg_bits({0x01, 0x06, 0x08, 0x09, 0x0A, 0x0D, 0x0E, 0x0F, 0x10, 0x1B, 0x2A});
constexpr uint64_t kVisualRegs = reg_bits({0x01, 0x04, 0x05, 0x06, 0x07, 0x08, 0x09, 0x0A, 0x0B, 0x0C, 0x0D, 0x0E,
                                           0x0F, 0x10, 0x11, 0x12, 0x13, 0x14, 0x1B, 0x1C, 0x1D, 0x1E, 0x1F, 0x25,
                                           0x26, 0x27, 0x28, 0x29, 0x2A});

// TIA write registers that can change which objects overlap (collisions
// are evaluated up to such a write first).
constexpr uint64_t kObjRegs = reg_bits({0x04, 0x05, 0x0A, 0x0B, 0x0C, 0x0D, 0x0E, 0x0F, 0x10, 0x11, 0x12, 0x13,
                                        0x14, 0x1B, 0x1C, 0x1D, 0x1E, 0x1F, 0x25, 0x26, 0x27, 0x28, 0x29, 0x2A});

// Registers kept only in the cold words (vcs_tia.cuh), and the hot ones
// whose write may also touch them (GRP0's vertical-delay copy, HMOVE and
// RESP0 for moved or locked cold objects, HMCLR).
constexpr uint64_t kColdRegs = reg_bits({0x04, 0x05, 0x07, 0x0B, 0x0C, 0x11, 0x12, 0x13, 0x14, 0x1C, 0x1D, 0x1E,
                                         0x1F, 0x21, 0x22, 0x23, 0x24, 0x25, 0x26, 0x27, 0x28, 0x29, 0x2C});
constexpr uint64_t kColdMaybe = reg_bits({0x10, 0x1B, 0x2A, 0x2B});

// TIA write registers whose write opens a new version of a differentiable
// quantity (the soft path's tapes): the four colour registers, and player
// 0's position (RESP0, HMOVE) for the position sampler.
constexpr uint64_t kVersionRegs = reg_bits({0x06, 0x07, 0x08, 0x09, 0x10, 0x2A});
// With the graphics-bit surrogate, GRP0 and the playfield registers open
// versions too.
constexpr uint64_t kGraphicsRegs = reg_bits({0x0D, 0x0E, 0x0F, 0x1B});
// With the whole TIA also GRP1, ENAM0, ENAM1 and ENABL; a GRP0 write opens
// one more version (GRP1's delayed copy) and a GRP1 write two more (GRP0's
// and ENABL's).
constexpr uint64_t kGraphicsRegsFT = reg_bits({0x1C, 0x1D, 0x1E, 0x1F});

// With the whole TIA and deferred rasterisation, the writes the raster
// replays: every register drawing depends on, the motion registers included
// (HMOVE reads them), not the collision clear.
constexpr uint64_t kRasterRegsFT = (kVisualRegs | kColdRegs | kColdMaybe | reg_bits({0x20})) & ~reg_bits({0x2C});

// Tape hook: called for each executed instruction the backward sweep acts on
// (reverse_needed) with its opcode, a reference address and flag bits (the
// soft path records these; the hard path compiles the hook away).
struct NoTape {
  static constexpr bool kAcc = false;
  static constexpr bool sampler = false;
  __device__ __forceinline__ void rec(uint32_t, uint32_t, uint32_t) {}
  __device__ __forceinline__ void version_write(uint32_t) {}
  __device__ __forceinline__ void pixels(float, float, float, float, float) {}
};

// The hard machine with deferred rasterisation (vcs_machine.cuh): the
// returned frame's picture-register writes go to the env's log instead of
// being drawn.
struct DeferTape : NoTape {
  uint32_t* log;   // this env's log entries (kRasterLogCap of them)
  uint32_t* hdr;   // this env's header (kRasterHdr words)
  int32_t* err;    // the batch's device error word
  uint32_t n;
};
template <class Tape>
constexpr bool kDefers = std::is_same<Tape, DeferTape>::value;

// The returned frame starts: its drawing registers (with the whole TIA also
// HMP0 and the cold words) and first colour clock go to the header, and the
// log starts empty.
__device__ __forceinline__ void raster_begin(const Ctx& c, const Regs& r, const Render& rd, DeferTape& tape) {
  tape.n = 0;
  tape.hdr[1] = (uint32_t)rd.cur;
  raster_snapshot(r, tape.hdr);
  if (c.ft) {
    tape.hdr[5] |= (r.hmp0 & 0xFF) << 16;
    for (uint32_t k = 0; k < 4; k++) tape.hdr[7 + k] = c.tx[k * c.E];
  }
}

// The returned frame ends at colour clock `end`.  kRasterLogCap bounds the
// picture-register writes of any frame; a log past it would mean a broken
// bound, so the entries past it are dropped and the batch's error word set.
__device__ __forceinline__ void raster_end(DeferTape& tape, int32_t end) {
  tape.hdr[0] = tape.n < (uint32_t)kRasterLogCap ? tape.n : (uint32_t)kRasterLogCap;
  tape.hdr[2] = (uint32_t)end;
  if (tape.n > (uint32_t)kRasterLogCap) atomicExch(tape.err, kErrRasterLog);
}

// A write to a cold register (or a hot one with cold effects) at line clock
// h: updates the cold words at tx (stride E) and returns the new summary
// bits and collision word (x: Regs::xo, y: Regs::cx).  Out of line and
// called with plain values, so the interpreter's registers stay registers.
static __device__ __noinline__ uint2 tia_write_cold(uint32_t* tx, uint32_t E, uint32_t reg, uint32_t v, uint32_t h,
                                             uint32_t grp0, uint32_t pos0, uint32_t cx);

// The hot registers' part of a write of v to TIA register reg at scanline
// `line`, colour clock h within it (the interpreter's registers; the raster
// kernels replay writes with it too).
__device__ __forceinline__ void tia_hot(Regs& r, uint32_t reg, uint32_t v, uint32_t line, uint32_t h) {
  r.vsync = reg == 0x00 ? v : r.vsync;
  r.vblank = reg == 0x01 ? v : r.vblank;
  r.col0 = reg == 0x06 ? v : r.col0;
  r.colpf = reg == 0x08 ? v : r.colpf;
  r.colbk = reg == 0x09 ? v : r.colbk;
  r.ctrl = reg == 0x0A ? v : r.ctrl;
  r.pf0 = reg == 0x0D ? v : r.pf0;
  r.pf1 = reg == 0x0E ? v : r.pf1;
  r.pf2 = reg == 0x0F ? v : r.pf2;
  r.grp0 = reg == 0x1B ? v : r.grp0;
  // RESP0: colour clock 3 in HBLANK, else the beam position plus 5, mod 160
  const uint32_t resp = h < 68 ? 3u : (h - 68u + 5u) % 160u;
  // HMOVE: move by the signed high nibble of HMP0 (positive = left)
  const int32_t mv = ((int32_t)(int8_t)(uint8_t)r.hmp0) >> 4;
  const uint32_t hmov = (uint32_t)(((int32_t)r.pos - mv + 160) % 160);
  r.pos = reg == 0x10 ? resp : (reg == 0x2A ? hmov : r.pos);
  r.hml = (reg == 0x2A && h <= 9) ? (int32_t)line : r.hml;
  r.hmp0 = reg == 0x20 ? v : (reg == 0x2B ? 0u : r.hmp0);
}

// Whether a write to reg touches the cold words (vcs_tia.cuh) given the
// summary bits xo.
__device__ __forceinline__ bool cold_write(uint32_t reg, uint32_t xo) {
  return ((kColdRegs >> reg) & 1) || (((kColdMaybe >> reg) & 1) && (xo & (kXoG1 | kXoMove | kXoLock)));
}

// A TIA register write at frame cycle fcw.  A write that changes the picture
// first draws the pending span with the old registers (with deferred
// rasterisation it goes to the log instead).  The register update itself is
// a set of selects rather than a switch: one indirect branch per write costs
// more than the few dozen independent integer operations.
template <class Tape>
__device__ __forceinline__ void tia_write(const Ctx& c, Regs& r, Render& rd, Step& st, Tape& tape, uint32_t reg,
                                          uint32_t v, int32_t fcw) {
  if constexpr (!kDefers<Tape>) {
    if ((((c.ft ? kVisualRegs : kVisualSubset) >> reg) & 1) && rd.on) render_to(c, r, rd, tape, 3 * fcw);
  }
  if (c.ft && ((kObjRegs >> reg) & 1)) cx_catchup(c, r, 3 * fcw);
  tape.version_write(reg);
  const uint32_t line = div76((uint32_t)fcw);
  const uint32_t m = (uint32_t)fcw - 76u * line;   // CPU cycle within the line
  const uint32_t h = 3u * m;                       // colour clock within the line
  st.fe_at = (reg == 0x00 && !(r.vsync & 2) && (v & 2)) ? fcw : st.fe_at;
  st.stall += (reg == 0x02 && m != 0) ? (int32_t)(76u - m) : 0;
  tia_hot(r, reg, v, line, h);
  if constexpr (kDefers<Tape>) {
    // the subset machine's entries carry player 0's new position for RESP0
    // and HMOVE; the whole TIA's are the raw writes its raster replays
    if ((((c.ft ? kRasterRegsFT : kVisualSubset) >> reg) & 1) && rd.on) {
      if (tape.n < (uint32_t)kRasterLogCap)
        tape.log[tape.n] = c.ft ? ((uint32_t)fcw << 16) | (reg << 8) | v
                                : ((uint32_t)fcw << 16) | ((reg == 0x2A && h <= 9) ? kRasterEarly : 0u) |
                                      (reg << 8) | ((reg == 0x10 || reg == 0x2A) ? r.pos : v);
      tape.n++;
    }
  }
  if (!c.ft) return;   // the subset machine ignores the rest of the TIA
  if ((kObjRegs >> reg) & 1) mirror_hot(c, r);
  if (cold_write(reg, r.xo)) {
    const uint2 o = tia_write_cold(c.tx, c.E, reg, v, h, r.grp0, r.pos, r.cx);
    r.xo = o.x;
    r.cx = o.y;
    if (reg == 0x2C) r.cxc = 3 * fcw;   // CXCLR: nothing before the clear counts
  }
}

// Missiles locked to their players (RESMP bit 1): at the player's position
// + 4 x its width - 1.
__device__ __forceinline__ void relock(uint32_t pos0, uint32_t& w3, uint32_t w0) {
  if (w0 & kW0Resmp0) {
    const uint32_t p = (pos0 + 4u * player_scale((w0 >> 8) & 7) - 1u) % 160u;
    w3 = (w3 & ~0xFF00u) | (p << 8);
  }
  if (w0 & kW0Resmp1) {
    const uint32_t p = ((w3 & 0xFF) + 4u * player_scale((w0 >> 16) & 7) - 1u) % 160u;
    w3 = (w3 & ~0xFF0000u) | (p << 16);
  }
}

static __device__ __noinline__ uint2 tia_write_cold(uint32_t* tx, uint32_t E, uint32_t reg, uint32_t v, uint32_t h,
                                             uint32_t grp0, uint32_t pos0, uint32_t cx) {
  uint32_t w0 = tx[0], w1 = tx[E], w2 = tx[2 * E], w3 = tx[3 * E];
  auto set = [](uint32_t& w, uint32_t shift, uint32_t mask, uint32_t x) { w = (w & ~(mask << shift)) | ((x & mask) << shift); };
  auto flag = [](uint32_t& w, uint32_t bit, bool on) { w = on ? (w | bit) : (w & ~bit); };
  const uint32_t resp = h < 68 ? 3u : (h - 68u + 5u) % 160u, resm = h < 68 ? 2u : (h - 68u + 4u) % 160u;
  auto moved = [](uint32_t p, uint32_t hm) { return (uint32_t)(((int32_t)p - (((int32_t)(int8_t)(uint8_t)hm) >> 4) + 160) % 160); };
  switch (reg) {
    case 0x04: set(w0, 8, 0xFF, v); break;                           // NUSIZ0
    case 0x05: set(w0, 16, 0xFF, v); break;                          // NUSIZ1
    case 0x07: set(w0, 0, 0xFF, v); break;                           // COLUP1
    case 0x0B: flag(w0, kW0Refp0, v & 8); break;                     // REFP0
    case 0x0C: flag(w0, kW0Refp1, v & 8); break;                     // REFP1
    case 0x11: set(w3, 0, 0xFF, resp); break;                        // RESP1
    case 0x12: set(w3, 8, 0xFF, resm); break;                        // RESM0
    case 0x13: set(w3, 16, 0xFF, resm); break;                       // RESM1
    case 0x14: set(w3, 24, 0xFF, resm); break;                       // RESBL
    case 0x1B: set(w1, 16, 0xFF, w1 & 0xFF); break;                  // GRP0: delayed GRP1 <- GRP1
    case 0x1C:                                                       // GRP1: delayed GRP0 <- GRP0, delayed ENABL <- ENABL
      set(w1, 0, 0xFF, v);
      set(w1, 8, 0xFF, grp0);
      flag(w1, kW1EnablOld, (w1 & kW1Enabl) != 0);
      break;
    case 0x1D: flag(w1, kW1Enam0, v & 2); break;                     // ENAM0
    case 0x1E: flag(w1, kW1Enam1, v & 2); break;                     // ENAM1
    case 0x1F: flag(w1, kW1Enabl, v & 2); break;                     // ENABL
    case 0x21: set(w2, 0, 0xFF, v); break;                           // HMP1
    case 0x22: set(w2, 8, 0xFF, v); break;                           // HMM0
    case 0x23: set(w2, 16, 0xFF, v); break;                          // HMM1
    case 0x24: set(w2, 24, 0xFF, v); break;                          // HMBL
    case 0x25: flag(w0, kW0Vdelp0, v & 1); break;                    // VDELP0
    case 0x26: flag(w0, kW0Vdelp1, v & 1); break;                    // VDELP1
    case 0x27: flag(w0, kW0Vdelbl, v & 1); break;                    // VDELBL
    case 0x28: flag(w0, kW0Resmp0, v & 2); break;                    // RESMP0
    case 0x29: flag(w0, kW0Resmp1, v & 2); break;                    // RESMP1
    case 0x2A:                                                       // HMOVE: the cold objects move too
      w3 = moved(w3 & 0xFF, w2) | (moved((w3 >> 8) & 0xFF, w2 >> 8) << 8) |
           (moved((w3 >> 16) & 0xFF, w2 >> 16) << 16) | (moved(w3 >> 24, w2 >> 24) << 24);
      break;
    case 0x2B: w2 = 0; break;                                        // HMCLR
    case 0x2C: cx &= 0xFFFF0000u; break;                            // CXCLR
    default: break;
  }
  relock(pos0, w3, w0);
  tx[0] = w0;
  tx[E] = w1;
  tx[2 * E] = w2;
  tx[3 * E] = w3;
  return cold_summary_of(w0, w1, w2, cx);
}

// Fully relaxed casts (FM template argument of the interpreter): 0 = the
// hard machine; 1 = probe: the hard machine that also counts which casts
// would round off the hard value; 2 = FULL: the fully relaxed forward of
// Section 4, whose ROM and RAM reads by instructions (operand bytes, data,
// pointers, stack; not the opcode fetch) are temperature reads cast back to
// bytes and whose conditional branches take the rounded blend of Eq. branch.
//
// Temperature read of index a of a tensor of M bytes (get(k) = byte k):
// round(sum_k w_k t_k / sum_k w_k), w_k = ek[|k - a|], over |k - a| <= W
// clipped to the tensor, in float32 with the terms added in index order and
// no fused multiply-add, rounded half to even, clamped to 0..255.
template <class Get>
__device__ __forceinline__ uint32_t relaxed_byte(const FullParams& fp, int32_t M, int32_t a, Get get) {
  const int32_t lo = a - fp.W < 0 ? 0 : a - fp.W, hi = a + fp.W > M - 1 ? M - 1 : a + fp.W;
  float num = 0.f, den = 0.f;
  for (int32_t k = lo; k <= hi; k++) {
    const float w = fp.ek[k > a ? k - a : a - k];
    num = __fadd_rn(num, __fmul_rn(w, (float)get(k)));
    den = __fadd_rn(den, w);
  }
  const float v = rintf(__fdiv_rn(num, den));
  return (uint32_t)fminf(fmaxf(v, 0.f), 255.f);
}
// The ROM tensor is the cart image (2K), the current 4K bank, or the E0
// slice the address's segment shows.
__device__ __forceinline__ uint32_t rom_relaxed(const Ctx& c, const Regs& r, uint32_t addr) {
  const int32_t M = c.fp->rom_m;
  const uint32_t base = rom_off(c, r, addr & 0x1FFF) & ~(uint32_t)(M - 1);
  return relaxed_byte(*c.fp, M, (int32_t)(addr & (uint32_t)(M - 1)), [&](int32_t k) { return (uint32_t)c.rom[base | (uint32_t)k]; });
}
__device__ __forceinline__ uint32_t ram_relaxed(const Ctx& c, uint32_t addr) {
  return relaxed_byte(*c.fp, 128, (int32_t)(addr & 0x7F), [&](int32_t k) { return ram_rd(c, (uint32_t)k); });
}
// The Superchip's RAM is a 128-byte tensor of its own.
__device__ __forceinline__ uint32_t cram_relaxed(const Ctx& c, uint32_t addr) {
  return relaxed_byte(*c.fp, 128, (int32_t)(addr & 0x7F), [&](int32_t k) { return cram_rd(c, (uint32_t)k); });
}
// A cast of a read whose hard value is `exact`: counted in probe and FULL
// machines, applied in FULL.
template <int FM>
__device__ __forceinline__ uint32_t cast_read(Regs& r, uint32_t exact, uint32_t relaxed) {
  r.fr_reads++;
  r.fr_exact += relaxed == exact ? 1u : 0u;
  return FM == 2 ? relaxed : exact;
}

// One bus read at cycle index idx of the current instruction, for any
// address.  Every source is read and the result selected, which costs fewer
// cycles than branching on the address region (the Superchip's read port,
// a block-uniform case, is the exception).  Side effects: a read of a
// bank-switch hotspot switches the bank, and a read of INTIM records whether
// the timer had underflowed (r.intim_live, kept by the soft path's tape).
template <int FM = 0>
__device__ __forceinline__ uint32_t bus_read(const Ctx& c, Regs& r, const Step& st, uint32_t addr, int idx) {
  const uint32_t a = addr & 0x1FFF;
  hotspot(c, r, a);
  const uint32_t vrom = c.rom[rom_off(c, r, a)];
  const uint32_t vram = ram_rd(c, a);
  const uint32_t q = a & 0xF;
  uint32_t vtia = q == 0xC ? (r.inpt4 & 0xFF) : (q == 0xD ? 0x80u : 0u);
  if (c.ft && !(a & 0x1080) && q < 8) vtia = cx_read(c, r, q, 3 * (r.fc + idx + st.stall));   // a collision latch
  const uint32_t q3 = a & 3;
  const uint32_t vio = q3 == 0 ? r.swcha : (q3 == 2 ? 0x0Bu ^ (r.inpt4 >> 8) : 0u);
  const uint32_t k = r.cyc + (uint32_t)(idx + st.stall) - r.tw;
  const uint32_t vi = r.tv << r.tsh;
  const bool live = k <= vi;
  const uint32_t vint = live ? r.tv - ((k + (1u << r.tsh) - 1) >> r.tsh) : ((vi - k) & 0xFF);
  const uint32_t vtim = (a & 1) ? (live ? 0u : 0x80u) : vint;
  const bool timer = (a & 0x1284) == 0x0284;
  r.intim_live = (timer && !(a & 1)) ? (live ? 1u : 0u) : r.intim_live;
  const bool cport = sc_read_port(c, a);
  const uint32_t vcart = cport ? cram_rd(c, a) : vrom;
  if constexpr (FM >= 1) {
    if (cport) return cast_read<FM>(r, vcart, cram_relaxed(c, a));
    if (a & 0x1000) return cast_read<FM>(r, vrom, rom_relaxed(c, r, a));
    if ((a & 0x280) == 0x080) return cast_read<FM>(r, vram, ram_relaxed(c, a));
  }
  return (a & 0x1000) ? vcart : !(a & 0x80) ? vtia : !(a & 0x200) ? vram : !(a & 4) ? vio : vtim;
}

// A read inside page zero or one (zero-page modes, the stack) at cycle idx
// of the instruction: RAM or the TIA read registers (a collision latch is
// brought up to that cycle first), no other side effects.
template <int FM = 0>
__device__ __forceinline__ uint32_t zp_read(const Ctx& c, Regs& r, const Step& st, uint32_t a, int idx) {
  const uint32_t vram = ram_rd(c, a);
  const uint32_t q = a & 0xF;
  uint32_t vtia = q == 0xC ? (r.inpt4 & 0xFF) : (q == 0xD ? 0x80u : 0u);
  if (c.ft && !(a & 0x80) && q < 8) vtia = cx_read(c, r, q, 3 * (r.fc + idx + st.stall));
  if constexpr (FM >= 1) {
    if (a & 0x80) return cast_read<FM>(r, vram, ram_relaxed(c, a));
  }
  return (a & 0x80) ? vram : vtia;
}

template <class Tape>
__device__ __forceinline__ void bus_write(const Ctx& c, Regs& r, Render& rd, Step& st, Tape& tape, uint32_t addr,
                                          uint32_t v, int idx) {
  const uint32_t a = addr & 0x1FFF;
  hotspot(c, r, a);
  if (sc_write_port(c, a)) cram_wr(c, a, v);
  if ((a & 0x1080) == 0) {   // TIA
    tia_write(c, r, rd, st, tape, a & 0x3F, v & 0xFF, r.fc + idx + st.stall);
    return;
  }
  if ((a & 0x1280) == 0x0080) ram_wr(c, a, v);
  const bool timer = (a & 0x1294) == 0x0294;   // TIM1T, TIM8T, TIM64T, T1024T
  r.tw = timer ? r.cyc + (uint32_t)(idx + st.stall) : r.tw;
  r.tv = timer ? (v & 0xFF) : r.tv;
  r.tsh = timer ? (0x0A060300u >> (8 * (a & 3))) & 0xFF : r.tsh;
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

template <int FM = 0>
__device__ __forceinline__ uint32_t pull(const Ctx& c, Regs& r, const Step& st, int idx) {
  r.SP = (r.SP + 1) & 0xFF;
  return zp_read<FM>(c, r, st, 0x100u | r.SP, idx);
}

// Instruction length of each addressing mode, two bits per mode.
constexpr uint32_t kModeLen = 1u | (1u << 2) | (2u << 4) | (2u << 6) | (2u << 8) | (2u << 10) | (3u << 12) |
                              (3u << 14) | (3u << 16) | (2u << 18) | (2u << 20) | (2u << 22) | (3u << 24) |
                              (1u << 26);

// The implemented opcodes (op_info gives each one's mode, cycles and
// operation): the 151 documented ones, dispatched by the main switch (the
// list below, then SBC #imm and NOP, whose handlers also serve USBC and the
// implied extra NOPs), and the rest of the paper's 38 extra bytes, run by
// exec_extra from the switch's default (real programs seldom use them, and
// one compact run-time-decoded handler keeps the switch's code as compact as
// without them).  Every other byte jams the CPU.

#define VCS_DOCUMENTED_OPS(X) \
  X(0x00) X(0x01) X(0x05) X(0x06) X(0x08) X(0x09) X(0x0A) X(0x0D) X(0x0E) X(0x10) X(0x11) X(0x15) \
  X(0x16) X(0x18) X(0x19) X(0x1D) X(0x1E) X(0x20) X(0x21) X(0x24) X(0x25) X(0x26) X(0x28) X(0x29) \
  X(0x2A) X(0x2C) X(0x2D) X(0x2E) X(0x30) X(0x31) X(0x35) X(0x36) X(0x38) X(0x39) X(0x3D) X(0x3E) \
  X(0x40) X(0x41) X(0x45) X(0x46) X(0x48) X(0x49) X(0x4A) X(0x4C) X(0x4D) X(0x4E) X(0x50) X(0x51) \
  X(0x55) X(0x56) X(0x58) X(0x59) X(0x5D) X(0x5E) X(0x60) X(0x61) X(0x65) X(0x66) X(0x68) X(0x69) \
  X(0x6A) X(0x6C) X(0x6D) X(0x6E) X(0x70) X(0x71) X(0x75) X(0x76) X(0x78) X(0x79) X(0x7D) X(0x7E) \
  X(0x81) X(0x84) X(0x85) X(0x86) X(0x88) X(0x8A) X(0x8C) X(0x8D) X(0x8E) X(0x90) X(0x91) X(0x94) \
  X(0x95) X(0x96) X(0x98) X(0x99) X(0x9A) X(0x9D) X(0xA0) X(0xA1) X(0xA2) X(0xA4) X(0xA5) X(0xA6) \
  X(0xA8) X(0xA9) X(0xAA) X(0xAC) X(0xAD) X(0xAE) X(0xB0) X(0xB1) X(0xB4) X(0xB5) X(0xB6) X(0xB8) \
  X(0xB9) X(0xBA) X(0xBC) X(0xBD) X(0xBE) X(0xC0) X(0xC1) X(0xC4) X(0xC5) X(0xC6) X(0xC8) X(0xC9) \
  X(0xCA) X(0xCC) X(0xCD) X(0xCE) X(0xD0) X(0xD1) X(0xD5) X(0xD6) X(0xD8) X(0xD9) X(0xDD) X(0xDE) \
  X(0xE0) X(0xE1) X(0xE4) X(0xE5) X(0xE6) X(0xE8) X(0xEC) X(0xED) X(0xEE) X(0xF0) \
  X(0xF1) X(0xF5) X(0xF6) X(0xF8) X(0xF9) X(0xFD) X(0xFE)

// What an instruction leaves for the common tail of exec_one: its cycle
// count, its writes (nw bytes of wv, low byte first, at cycle indices widx,
// widx + 1, ... to ea, or pushed on the stack when wstack) and its tape
// record (reference address and flag bits).
struct Pend {
  uint32_t n, ea, nw, wv, widx, tref, tfl;
  bool wstack, rec;
  bool seq;   // the next instruction follows at a PC that every lane executing this one shares
};

template <uint32_t MODE>
__host__ __device__ constexpr bool page_zero_mode() {
  return MODE == AM_ZP || MODE == AM_ZPX || MODE == AM_ZPY;
}

// Timer poll loop "L: LDA INTIM; BNE L" (AD 84 02 D0 FB) entered at its LDA,
// before the timer's underflow: advance the clocks over the iterations that
// read a nonzero value, so that the LDA about to execute is the first one
// that reads zero (or the last one before the scanline watchdog).  Exact:
// the skipped iterations write nothing and every register they set is set
// again by that LDA; the timer value read k cycles after the write of V with
// interval I is V - ceil(k / I), zero for (V - 1) I < k <= V I.  A loop that
// would step over that window (only possible for I = 1) or that starts after
// the underflow is left to the interpreter.  An instruction-granular step
// skips at most the whole iterations its remaining slots hold (two each, the
// LDA about to execute counted in the step), and `budget` loses them.
__device__ __forceinline__ void skip_timer_poll(Regs& r, uint32_t opaddr, int32_t& budget) {
  const uint32_t period = 7u + ((((opaddr + 5u) ^ opaddr) & 0xFF00) ? 1u : 0u);   // LDA 4 + BNE taken 3 (+1 page cross)
  const uint32_t vi = r.tv << r.tsh;
  const uint32_t k0 = r.cyc + 4u - r.tw;   // the LDA reads on its fourth cycle
  if (r.tv == 0 || k0 > vi) return;
  const uint32_t lo = (r.tv - 1u) << r.tsh;
  uint32_t j = k0 > lo ? 0u : (period == 7u ? (lo - k0) / 7u : (lo - k0) >> 3) + 1u;
  if (k0 + j * period > vi) return;
  const int32_t room = kLineCap * kLineCycles - 1 - r.fc;   // stay below the watchdog
  const uint32_t jw = room > 0 ? (period == 7u ? (uint32_t)room / 7u : (uint32_t)room >> 3) : 0u;
  j = j < jw ? j : jw;
  const uint32_t jb = budget > 0 ? (uint32_t)(budget - 1) >> 1 : 0u;
  j = j < jb ? j : jb;
  budget -= (int32_t)(2 * j);
  r.cyc += j * period;
  r.fc += (int32_t)(j * period);
}

// One documented instruction, specialised on its opcode: mode, class and
// operation are compile-time constants, so the only run-time dispatch of an
// instruction is the opcode switch in exec_one.  LDA absolute first checks
// for the head of a timer poll loop.  The skip is exact in soft mode too:
// every skipped LDA overwrites A before anything reads it, so in the
// backward sweep each meets a zero adjoint of A and its tape record would do
// nothing; the LDA that exits the loop is executed and recorded.
template <uint32_t OP, int FM = 0>
__device__ __forceinline__ void exec_op(const Ctx& c, Regs& r, Step& st, uint32_t opaddr, uint32_t b1, uint32_t b2,
                                        Pend& p) {
  if constexpr (OP == 0xAD && FM == 0) {   // the skip assumes exact operand bytes
    const uint32_t off = opaddr & 0xFFF;
    if (b1 == 0x84 && b2 == 0x02 && (opaddr & 0x1000) && plain_rom(c, off, 5)) {
      const uint8_t* q = c.rom + rom_off(c, r, opaddr & 0x1FFF);
      if (q[3] == 0xD0 && q[4] == 0xFB) skip_timer_poll(r, opaddr, st.instr_left);
    }
  }
  constexpr OpInfo I = op_info(OP);
  constexpr uint32_t mode = I.mode, cls = I.cls, id = I.id;
  constexpr uint32_t len = (kModeLen >> (2 * mode)) & 3;
  uint32_t n = I.cyc;
  const uint32_t pc1 = (opaddr + 1) & 0xFFFF;
  r.PC = (opaddr + len) & 0xFFFF;
  uint32_t ea = 0;
  bool cross = false;
  if constexpr (mode == AM_IMM) {
    ea = pc1;
  } else if constexpr (mode == AM_ZP) {
    ea = b1;
  } else if constexpr (mode == AM_ZPX) {
    ea = (b1 + r.X) & 0xFF;
  } else if constexpr (mode == AM_ZPY) {
    ea = (b1 + r.Y) & 0xFF;
  } else if constexpr (mode == AM_ABS) {
    ea = b1 | (b2 << 8);
  } else if constexpr (mode == AM_ABX || mode == AM_ABY) {
    const uint32_t base = b1 | (b2 << 8);
    ea = (base + (mode == AM_ABX ? r.X : r.Y)) & 0xFFFF;
    cross = ((base ^ ea) & 0xFF00) != 0;
  } else if constexpr (mode == AM_INX) {
    const uint32_t q = (b1 + r.X) & 0xFF;
    ea = zp_read<FM>(c, r, st, q, 4) | (zp_read<FM>(c, r, st, (q + 1) & 0xFF, 5) << 8);
  } else if constexpr (mode == AM_INY) {
    const uint32_t base = zp_read<FM>(c, r, st, b1, 3) | (zp_read<FM>(c, r, st, (b1 + 1) & 0xFF, 4) << 8);
    ea = (base + r.Y) & 0xFFFF;
    cross = ((base ^ ea) & 0xFF00) != 0;
  }

  // the one data read: read-class instructions read on their last cycle
  // (after any page-cross cycle), read-modify-write two cycles before the end
  uint32_t m = 0;
  if constexpr (cls == CL_READ) {
    if constexpr (mode == AM_IMM) {
      m = b1;
    } else {
      n += cross ? 1u : 0u;
      if constexpr (page_zero_mode<mode>()) m = zp_read<FM>(c, r, st, ea, (int)n);
      else m = bus_read<FM>(c, r, st, ea, (int)n);
    }
  } else if constexpr (cls == CL_RMW) {
    if constexpr (page_zero_mode<mode>()) m = zp_read<FM>(c, r, st, ea, (int)n - 2);
    else m = bus_read<FM>(c, r, st, ea, (int)n - 2);
  }
  p.tref = ea;
  p.tfl = 0;
  p.nw = 0;
  p.wv = 0;
  p.widx = n;
  p.wstack = false;
  p.rec = reverse_needed(OP);   // a tape record only where the backward sweep acts
  // JMP and JSR go to the same place for every lane; branches, RTS, RTI,
  // JMP (ind) and BRK end a run of lockstep instructions
  p.seq = !(id == OP_BRANCH || id == OP_JMPI || id == OP_RTS || id == OP_RTI || id == OP_BRK);
  if constexpr (id == OP_LDA) { r.A = m; set_nz(r, m); }
  else if constexpr (id == OP_LDX) { r.X = m; set_nz(r, m); }
  else if constexpr (id == OP_LDY) { r.Y = m; set_nz(r, m); }
  else if constexpr (id == OP_ORA) { r.A |= m; set_nz(r, r.A); }
  else if constexpr (id == OP_AND) { r.A &= m; set_nz(r, r.A); }
  else if constexpr (id == OP_EOR) { r.A ^= m; set_nz(r, r.A); }
  else if constexpr (id == OP_ADC) { do_adc(r, m); }
  else if constexpr (id == OP_SBC) { do_sbc(r, m); }
  else if constexpr (id == OP_CMP) { do_cmp(r, r.A, m); }
  else if constexpr (id == OP_CPX) { do_cmp(r, r.X, m); }
  else if constexpr (id == OP_CPY) { do_cmp(r, r.Y, m); }
  else if constexpr (id == OP_BIT) {
    r.nsrc = m & 0x80;
    r.fV = (m >> 6) & 1;
    r.zsrc = r.A & m;
  }
  else if constexpr (id == OP_LAX) { r.A = m; r.X = m; set_nz(r, m); }
  else if constexpr (id == OP_SAX) { p.nw = 1; p.wv = r.A & r.X; }
  else if constexpr (id == OP_STA) { p.nw = 1; p.wv = r.A; }
  else if constexpr (id == OP_STX) { p.nw = 1; p.wv = r.X; }
  else if constexpr (id == OP_STY) { p.nw = 1; p.wv = r.Y; }
  else if constexpr (id == OP_ASL || id == OP_ROL || id == OP_LSR || id == OP_ROR) {
    p.wv = do_shift(r, id - OP_ASL, m);
    p.nw = 1;
  }
  else if constexpr (id == OP_DEC || id == OP_INC) {
    p.wv = (id == OP_DEC ? m - 1 : m + 1) & 0xFF;
    set_nz(r, p.wv);
    p.nw = 1;
  }
  else if constexpr (id == OP_ASLA || id == OP_ROLA || id == OP_LSRA || id == OP_RORA) {
    r.A = do_shift(r, id - OP_ASLA, r.A);
  }
  else if constexpr (id == OP_BRANCH) {
    uint32_t flag;
    if constexpr ((OP >> 6) == 0) flag = (r.nsrc >> 7) & 1;
    else if constexpr ((OP >> 6) == 1) flag = r.fV;
    else if constexpr ((OP >> 6) == 2) flag = r.fC;
    else flag = (r.zsrc & 0xFF) == 0 ? 1u : 0u;
    const bool taken = ((OP >> 5) & 1) == flag;
    const uint32_t next = r.PC;
    const uint32_t t = (next + (uint32_t)(int32_t)(int8_t)(uint8_t)b1) & 0xFFFF;
    uint32_t to = taken ? t : next;
    if constexpr (FM >= 1) {
      // Eq. branch without the straight-through correction: z = +1 when the
      // condition holds, else -1; pc = round(pc_fall + sigma(alpha z) delta)
      const float g = taken ? c.fp->g1 : c.fp->g0;
      const float pcf = __fadd_rn((float)next, __fmul_rn(g, (float)(int32_t)(int8_t)(uint8_t)b1));
      const uint32_t rel = (uint32_t)(int32_t)rintf(pcf) & 0xFFFF;
      r.fr_br++;
      r.fr_br_exact += rel == to ? 1u : 0u;
      if constexpr (FM == 2) to = rel;
    }
    n += taken ? 1u + (((to ^ next) & 0xFF00) ? 1u : 0u) : 0u;
    r.PC = to;
    p.tref = pc1;
    p.tfl = taken ? 1u : 0u;
  }
  else if constexpr (id == OP_JMP) { r.PC = ea; }
  else if constexpr (id == OP_JMPI) {
    const uint32_t q = b1 | (b2 << 8);
    const uint32_t l2 = bus_read<FM>(c, r, st, q, 4);
    const uint32_t h2 = bus_read<FM>(c, r, st, (q & 0xFF00) | ((q + 1) & 0xFF), 5);
    r.PC = l2 | (h2 << 8);
  }
  else if constexpr (id == OP_JSR) {
    const uint32_t ret = (opaddr + 2) & 0xFFFF;
    r.PC = b1 | (b2 << 8);
    p.nw = 2; p.wstack = true; p.wv = (ret >> 8) | ((ret & 0xFF) << 8); p.widx = 4;
    // FE: the return address's low byte goes to $01FE and the next cycle
    // fetches the target's high byte, whose bit 5 picks the bank
    if (c.fe && r.SP == 0xFFu) r.bank = (b2 & 0x20u) ? 0u : 1u;
  }
  else if constexpr (id == OP_RTS) {
    const bool fe = c.fe && r.SP == 0xFDu;   // FE: the low byte comes from $01FE
    const uint32_t lo = pull<FM>(c, r, st, 4);
    const uint32_t hi = pull<FM>(c, r, st, 5);
    r.PC = ((lo | (hi << 8)) + 1) & 0xFFFF;
    if (fe) r.bank = (hi & 0x20u) ? 0u : 1u;
  }
  else if constexpr (id == OP_RTI) {
    const uint32_t pp = pull<FM>(c, r, st, 4);
    const uint32_t lo = pull<FM>(c, r, st, 5);
    const uint32_t hi = pull<FM>(c, r, st, 6);
    unpack_p(r, pp | 0x30);
    r.PC = lo | (hi << 8);
  }
  else if constexpr (id == OP_BRK) {
    const uint32_t ret = (opaddr + 2) & 0xFFFF;
    p.nw = 3; p.wstack = true; p.wv = (ret >> 8) | ((ret & 0xFF) << 8) | (pack_p(r) << 16); p.widx = 3;
    r.fI = 1;
    const uint32_t lo = bus_read<FM>(c, r, st, 0xFFFE, 6);
    const uint32_t hi = bus_read<FM>(c, r, st, 0xFFFF, 7);
    r.PC = lo | (hi << 8);
  }
  else if constexpr (id == OP_PHA) { p.nw = 1; p.wstack = true; p.wv = r.A; p.widx = 3; }
  else if constexpr (id == OP_PHP) { p.nw = 1; p.wstack = true; p.wv = pack_p(r); p.widx = 3; }
  else if constexpr (id == OP_PLA) {
    r.A = pull<FM>(c, r, st, 4);
    set_nz(r, r.A);
    p.tref = 0x100u | r.SP;
  }
  else if constexpr (id == OP_PLP) { unpack_p(r, pull<FM>(c, r, st, 4) | 0x30); }
  else if constexpr (id == OP_CLC) { r.fC = 0; }
  else if constexpr (id == OP_SEC) { r.fC = 1; }
  else if constexpr (id == OP_CLI) { r.fI = 0; }
  else if constexpr (id == OP_SEI) { r.fI = 1; }
  else if constexpr (id == OP_CLV) { r.fV = 0; }
  else if constexpr (id == OP_CLD) { r.fD = 0; }
  else if constexpr (id == OP_SED) { r.fD = 1; }
  else if constexpr (id == OP_TAX) { r.X = r.A; set_nz(r, r.X); }
  else if constexpr (id == OP_TXA) { r.A = r.X; set_nz(r, r.A); }
  else if constexpr (id == OP_TAY) { r.Y = r.A; set_nz(r, r.Y); }
  else if constexpr (id == OP_TYA) { r.A = r.Y; set_nz(r, r.A); }
  else if constexpr (id == OP_TSX) { r.X = r.SP; set_nz(r, r.X); }
  else if constexpr (id == OP_TXS) { r.SP = r.X; }
  else if constexpr (id == OP_INX) { r.X = (r.X + 1) & 0xFF; set_nz(r, r.X); }
  else if constexpr (id == OP_DEX) { r.X = (r.X - 1) & 0xFF; set_nz(r, r.X); }
  else if constexpr (id == OP_INY) { r.Y = (r.Y + 1) & 0xFF; set_nz(r, r.Y); }
  else if constexpr (id == OP_DEY) { r.Y = (r.Y - 1) & 0xFF; set_nz(r, r.Y); }
  // OP_NOP and OP_NOPR (its operand read above): nothing
  p.n = n;
  p.ea = ea;
}

// The rest of the paper's 38 extra opcode bytes (the unofficial NOPs with an
// operand, LAX, SAX) and the jam of every other undocumented byte, decoded
// at run time from the decode tables.  Real programs seldom execute them,
// so one compact handler serves all of them: specialised handlers for each
// would add instruction-cache pressure to every other instruction.  A NOP's
// operand read has no effect but a hotspot's bank switch (page-zero
// reads and INTIM reads change nothing), so NOPs read nothing.
template <int FM = 0>
__device__ __forceinline__ void exec_extra(const Ctx& c, Regs& r, Step& st, uint32_t op, uint32_t opaddr,
                                           uint32_t b1, uint32_t b2, Pend& p) {
  const uint32_t mc = c.dt->mode_cyc[op & 0xFF], co = c.dt->cls_op[op & 0xFF];   // op = 0x100: jammed
  const uint32_t mode = mc & 15, id = co >> 2;
  p.nw = 0;
  p.wv = 0;
  p.wstack = false;
  p.tfl = 0;
  p.seq = true;
  if (r.jam || mode == AM_JAM) {   // the CPU jams after the fetch; a jammed CPU idles to the next line
    p.n = r.jam ? 76u - (uint32_t)r.fc % 76u : 1u;
    r.PC = r.jam ? r.PC : (opaddr + 1) & 0xFFFF;
    r.jam = 1;
    p.rec = false;
    p.seq = false;
    p.ea = 0;
    p.tref = 0;
    return;
  }
  uint32_t n = mc >> 4;
  r.PC = (opaddr + ((kModeLen >> (2 * mode)) & 3)) & 0xFFFF;
  // effective address: zero-page modes wrap in page zero; (zp,X) and (zp),Y
  // read their pointer from page zero
  const uint32_t idx = mode == AM_ZPX || mode == AM_ABX ? r.X : (mode == AM_ZPY || mode == AM_ABY ? r.Y : 0u);
  uint32_t ea;
  bool cross = false;
  if (mode == AM_ZP || mode == AM_ZPX || mode == AM_ZPY) {
    ea = (b1 + idx) & 0xFF;
  } else if (mode == AM_INX || mode == AM_INY) {
    const uint32_t q = mode == AM_INX ? (b1 + r.X) & 0xFF : b1;
    const int i0 = mode == AM_INX ? 4 : 3;   // the pointer's cycles
    const uint32_t base = zp_read<FM>(c, r, st, q, i0) | (zp_read<FM>(c, r, st, (q + 1) & 0xFF, i0 + 1) << 8);
    ea = (base + (mode == AM_INY ? r.Y : 0u)) & 0xFFFF;
    cross = mode == AM_INY && ((base ^ ea) & 0xFF00) != 0;
  } else {
    const uint32_t base = b1 | (b2 << 8);
    ea = (base + idx) & 0xFFFF;
    cross = (mode == AM_ABX || mode == AM_ABY) && ((base ^ ea) & 0xFF00) != 0;
  }
  if (mode != AM_IMM && mode != AM_IMP && id != OP_SAX) n += cross ? 1u : 0u;   // reads pay the page cross
  if (id == OP_LAX) {   // the data read on the last cycle
    const uint32_t m = (mode == AM_ZP || mode == AM_ZPY) ? zp_read<FM>(c, r, st, ea, (int)n) : bus_read<FM>(c, r, st, ea, (int)n);
    r.A = m;
    r.X = m;
    set_nz(r, m);
  } else if (id == OP_SAX) {
    p.nw = 1;
    p.wv = r.A & r.X;
  } else if (mode == AM_ABS || mode == AM_ABX) {   // NOP abs / abs,X: only a hotspot read matters
    if constexpr (FM >= 1) (void)bus_read<FM>(c, r, st, ea, (int)n);   // the read is a cast to count
    else hotspot(c, r, ea & 0x1FFF);
  } else if (FM >= 1 && (mode == AM_ZP || mode == AM_ZPX)) {
    (void)zp_read<FM>(c, r, st, ea, (int)n);
  }
  p.widx = n;
  p.rec = id == OP_LAX || id == OP_SAX;   // reverse_needed of these bytes
  p.tref = ea;
  p.n = n;
  p.ea = ea;
}

// Instruction bytes at the program counter, fetched ahead: opcode | first
// operand << 8 | second operand << 16, or kSlowFetch when the bytes must be
// read through the bus at execution time (outside the cartridge window, near
// its end or the bank-switch hotspots, in a Superchip's RAM ports at its
// start, across an E0 segment boundary).  Fetching from the cartridge ROM
// has no side
// effect and does not depend on time, so it may happen as soon as the
// program counter and bank are known.
constexpr uint32_t kSlowFetch = 1u << 24;

__device__ __forceinline__ uint32_t prefetch(const Ctx& c, const Regs& r) {
  const uint32_t off = r.PC & 0xFFF;
  const bool fast = (r.PC & 0x1000) != 0 && plain_rom(c, off, 3);
  const uint8_t* q = c.rom + (fast ? rom_off(c, r, r.PC & 0x1FFF) : 0u);
  return (uint32_t)q[0] | ((uint32_t)q[1] << 8) | ((uint32_t)q[2] << 16) | (fast ? 0u : kSlowFetch);
}

// Probe and FULL machines: the temperature reads of the two operand bytes
// after the opcode (fetched ahead with it; counted only for the bytes the
// instruction takes).
__device__ __forceinline__ uint32_t prefetch_relaxed(const Ctx& c, const Regs& r, uint32_t pf) {
  if (pf & kSlowFetch) return 0u;
  return rom_relaxed(c, r, (r.PC + 1) & 0xFFFF) | (rom_relaxed(c, r, (r.PC + 2) & 0xFFFF) << 8);
}

// Execute one instruction slot (an instruction, or for a jammed CPU an idle
// to the next line start), advance the clocks and prefetch the next
// instruction's bytes into pf.  Returns true when the next instruction is at
// a program counter that every lane executing this one shares (no branch or
// data-dependent jump), so the warp may go on without re-scheduling.
//
// One switch runs the instruction's specialised handler; the two rare slots
// (a fetch through the bus, a jammed CPU) are cases of the same switch, so
// the common path has a single dispatch.  A bus fetch reads the operand
// bytes one by one, only as many as the instruction has, and dispatches
// again.  Writes go through the single write site below.
template <class Tape, int FM = 0>
__device__ __forceinline__ bool exec_one(const Ctx& c, Regs& r, Render& rd, Step& st, Tape& tape, uint32_t& pf) {
  const uint32_t opaddr = r.PC;
  r.intim_live = 0;
  uint32_t op = pf & 0xFF, b1 = (pf >> 8) & 0xFF, b2 = (pf >> 16) & 0xFF;
  if constexpr (FM >= 1) {   // the operand bytes fetched ahead are casts
    if (!(pf & kSlowFetch) && !r.jam) {
      const uint32_t len = (kModeLen >> (2 * (c.dt->mode_cyc[op] & 15))) & 3;
      if (len >= 2) b1 = cast_read<FM>(r, b1, r.pfr & 0xFF);
      if (len >= 3) b2 = cast_read<FM>(r, b2, (r.pfr >> 8) & 0xFF);
    }
  }
  uint32_t sel = r.jam ? 0x100u : ((pf & kSlowFetch) ? 0x101u : op);
  Pend p;
  for (;;) {
    switch (sel) {
#define VCS_CASE(x) \
  case x: exec_op<x, FM>(c, r, st, opaddr, b1, b2, p); break;
      VCS_DOCUMENTED_OPS(VCS_CASE)
      // SBC #imm and NOP share their handlers with the extra bytes of the
      // same semantics (USBC; the implied NOPs): one inlined body each
      case 0xE9: case 0xEB: exec_op<0xE9, FM>(c, r, st, opaddr, b1, b2, p); break;
      case 0xEA: case 0x1A: case 0x3A: case 0x5A: case 0x7A: case 0xDA: case 0xFA:
        exec_op<0xEA, FM>(c, r, st, opaddr, b1, b2, p); break;
      case 0x101: {   // fetch through the bus, then dispatch on what was read
        op = bus_read(c, r, st, opaddr, 1);   // the opcode fetch is never a cast
        const uint32_t len = (kModeLen >> (2 * (c.dt->mode_cyc[op] & 15))) & 3;
        if (len >= 2) b1 = bus_read<FM>(c, r, st, (opaddr + 1) & 0xFFFF, 2);
        if (len >= 3) b2 = bus_read<FM>(c, r, st, (opaddr + 2) & 0xFFFF, op == 0x20 ? 6 : 3);
        sel = op;
        continue;
      }
      default:
        exec_extra<FM>(c, r, st, sel, opaddr, b1, b2, p);
        break;
#undef VCS_CASE
    }
    break;
  }
  if (p.nw) {
    if (p.wstack) p.tref = 0x100u | r.SP;
    uint32_t i = 0;
    do {
      uint32_t addr = p.ea;
      if (p.wstack) {
        addr = 0x100u | r.SP;
        r.SP = (r.SP - 1) & 0xFF;
      }
      bus_write(c, r, rd, st, tape, addr, (p.wv >> (8 * i)) & 0xFF, (int)(p.widx + i));
    } while (++i < p.nw);
  }
  if (p.rec) tape.rec(op, p.tref, p.tfl | (r.intim_live << 1) | (rec_unit(c, r, p.tref & 0x1FFF) << 2));
  r.cyc += p.n + (uint32_t)st.stall;
  r.fc += (int32_t)p.n + st.stall;
  st.stall = 0;
  pf = prefetch(c, r);
  if constexpr (FM >= 1) r.pfr = prefetch_relaxed(c, r, pf);
  return p.seq && !(pf & kSlowFetch);
}

}  // namespace vcs
