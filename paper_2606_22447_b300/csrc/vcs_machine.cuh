// Per-thread VCS machine for sm_103a: one thread emulates one env.
//
// The machine follows the paper's VCS (Section 2.2): 6507 CPU, RIOT (RAM,
// timer, ports), TIA video, 2K/4K/F8/F6/F4, Superchip and E0 cartridges.
// Where the paper is silent the readings are: frames end at a VSYNC write
// that sets D1 or after 512 scanlines; screen row r is scanline ystart + r
// over line clocks 68..227; pixel = colour & 0xFE, black under VBLANK D1 and
// for 8 pixels after an HMOVE at line clock <= 9; a write at the k-th cycle
// of an instruction starting at cycle t takes effect at colour clock 3 (t +
// k); RESP0 puts P0 at 3 in HBLANK else (clock - 68 + 5) mod 160; WSYNC
// halts to the next multiple of 76 cycles; the RIOT timer reads V - ceil(k /
// I) k cycles after a write of V, then (0xFF - (k - V I - 1)) & 0xFF with
// TIMINT bit 7 set; power-on A=X=Y=0, SP=$FD, P=$34; NMOS decimal mode.
//
// Time is kept per thread as two counters: `cyc`, the CPU cycle count
// modulo 2^32 (only differences are used, for the timer), and `fc`, the
// cycle index within the current frame (76 * scanline + cycle in line).
// The TIA is rendered lazily: on each write that changes what is drawn,
// pixels from the render cursor up to the write's colour clock are drawn
// with the old registers (span catch-up), and only on the frame a step
// returns.  Memory lives in shared memory: the cart ROM image (4 to 32 KB,
// 2K carts mirrored), RAM as 32 words per env (64 when the batch holds a
// Superchip cart: its cartridge RAM follows) interleaved across the block
// (word w of env j at word w * E + j, so a warp touching the same address
// hits 32 different banks), and a 160-byte line buffer per env laid out
// the same way.
#pragma once
#include <cstdint>

namespace vcs {

constexpr int kLineCycles = 76;
constexpr int kLineCap = 512;
constexpr int kScreenH = 210;
constexpr int kScreenW = 160;

enum : uint32_t { kStWatchdog = 1, kStJammed = 2, kStDone = 4 };

// Addressing modes of the documented opcodes.
enum : uint8_t { AM_IMP, AM_ACC, AM_IMM, AM_ZP, AM_ZPX, AM_ZPY, AM_ABS, AM_ABX, AM_ABY,
                 AM_INX, AM_INY, AM_REL, AM_IND, AM_JAM };

// Instruction classes and compact operation ids of the decode table.
enum : uint8_t { CL_OTHER = 0, CL_READ = 1, CL_STORE = 2, CL_RMW = 3 };
enum : uint8_t {
  OP_LDA, OP_LDX, OP_LDY, OP_ORA, OP_AND, OP_EOR, OP_ADC, OP_SBC, OP_CMP, OP_CPX, OP_CPY, OP_BIT,
  OP_STA, OP_STX, OP_STY,
  OP_ASL, OP_ROL, OP_LSR, OP_ROR, OP_DEC, OP_INC,
  OP_ASLA, OP_ROLA, OP_LSRA, OP_RORA,
  OP_BRANCH, OP_JMP, OP_JMPI, OP_JSR, OP_RTS, OP_RTI, OP_BRK,
  OP_PHA, OP_PHP, OP_PLA, OP_PLP,
  OP_CLC, OP_SEC, OP_CLI, OP_SEI, OP_CLV, OP_CLD, OP_SED, OP_NOP,
  OP_TAX, OP_TXA, OP_TAY, OP_TYA, OP_TSX, OP_TXS, OP_INX, OP_DEX, OP_INY, OP_DEY,
  OP_LAX, OP_SAX, OP_NOPR,   // of the paper's extra opcode bytes (NOPR: a NOP that reads its operand)
  OP_JAM = 63
};

// Per-opcode decode: mode (low 4 bits) | base cycles << 4, and
// class (low 2 bits) | operation id << 2.
struct DecodeTables {
  uint8_t mode_cyc[256];
  uint8_t cls_op[256];
};

// Addressing mode, base cycle count (MOS 6500 data sheet; the unofficial-
// opcode tables for the extra bytes), class and operation of one opcode.
// Implemented: the 151 documented opcodes and the paper's 38 extra bytes
// (USBC = SBC #imm, the unofficial NOPs, LAX, SAX); every other byte decodes
// as AM_JAM.  This is the one definition of the instruction set: the step
// kernel specialises its handlers on it at compile time and the host builds
// DecodeTables from it.
struct OpInfo {
  uint8_t mode, cyc, cls, id;
};

__host__ __device__ constexpr OpInfo op_info(uint32_t op) {
  if ((op & 3) == 1) {   // the regular column: ORA AND EOR ADC STA LDA CMP SBC over eight modes
    const uint32_t aaa = op >> 5, bbb = (op >> 2) & 7;
    const uint8_t modes[8] = {AM_INX, AM_ZP, AM_IMM, AM_ABS, AM_INY, AM_ZPX, AM_ABY, AM_ABX};
    const uint8_t cyc[8] = {6, 3, 2, 4, 5, 4, 4, 4};
    const uint8_t ids[8] = {OP_ORA, OP_AND, OP_EOR, OP_ADC, OP_STA, OP_LDA, OP_CMP, OP_SBC};
    if (aaa == 4) {   // STA: no immediate form ($89 is an extra NOP #imm); indexed stores pay the fix-up cycle
      if (modes[bbb] == AM_IMM) return OpInfo{AM_IMM, 2, CL_READ, OP_NOPR};
      const uint8_t c = modes[bbb] == AM_INY ? 6 : (modes[bbb] == AM_ABX || modes[bbb] == AM_ABY) ? 5 : cyc[bbb];
      return OpInfo{modes[bbb], c, CL_STORE, OP_STA};
    }
    return OpInfo{modes[bbb], cyc[bbb], CL_READ, ids[aaa]};
  }
  const uint32_t hi = op & 0xE0, lo = op & 0x1F;
  if (hi <= 0x60 || hi == 0xC0 || hi == 0xE0) {   // shifts, rotates, DEC, INC
    const uint8_t id = hi == 0x00 ? OP_ASL : hi == 0x20 ? OP_ROL : hi == 0x40 ? OP_LSR
                     : hi == 0x60 ? OP_ROR : hi == 0xC0 ? OP_DEC : OP_INC;
    if (lo == 0x0A && hi <= 0x60) return OpInfo{AM_ACC, 2, CL_OTHER, (uint8_t)(OP_ASLA + (id - OP_ASL))};
    if (lo == 0x06) return OpInfo{AM_ZP, 5, CL_RMW, id};
    if (lo == 0x16) return OpInfo{AM_ZPX, 6, CL_RMW, id};
    if (lo == 0x0E) return OpInfo{AM_ABS, 6, CL_RMW, id};
    if (lo == 0x1E) return OpInfo{AM_ABX, 7, CL_RMW, id};
  }
  switch (op) {
    case 0xA2: return OpInfo{AM_IMM, 2, CL_READ, OP_LDX};
    case 0xA6: return OpInfo{AM_ZP, 3, CL_READ, OP_LDX};
    case 0xB6: return OpInfo{AM_ZPY, 4, CL_READ, OP_LDX};
    case 0xAE: return OpInfo{AM_ABS, 4, CL_READ, OP_LDX};
    case 0xBE: return OpInfo{AM_ABY, 4, CL_READ, OP_LDX};
    case 0xA0: return OpInfo{AM_IMM, 2, CL_READ, OP_LDY};
    case 0xA4: return OpInfo{AM_ZP, 3, CL_READ, OP_LDY};
    case 0xB4: return OpInfo{AM_ZPX, 4, CL_READ, OP_LDY};
    case 0xAC: return OpInfo{AM_ABS, 4, CL_READ, OP_LDY};
    case 0xBC: return OpInfo{AM_ABX, 4, CL_READ, OP_LDY};
    case 0x86: return OpInfo{AM_ZP, 3, CL_STORE, OP_STX};
    case 0x96: return OpInfo{AM_ZPY, 4, CL_STORE, OP_STX};
    case 0x8E: return OpInfo{AM_ABS, 4, CL_STORE, OP_STX};
    case 0x84: return OpInfo{AM_ZP, 3, CL_STORE, OP_STY};
    case 0x94: return OpInfo{AM_ZPX, 4, CL_STORE, OP_STY};
    case 0x8C: return OpInfo{AM_ABS, 4, CL_STORE, OP_STY};
    case 0xE0: return OpInfo{AM_IMM, 2, CL_READ, OP_CPX};
    case 0xE4: return OpInfo{AM_ZP, 3, CL_READ, OP_CPX};
    case 0xEC: return OpInfo{AM_ABS, 4, CL_READ, OP_CPX};
    case 0xC0: return OpInfo{AM_IMM, 2, CL_READ, OP_CPY};
    case 0xC4: return OpInfo{AM_ZP, 3, CL_READ, OP_CPY};
    case 0xCC: return OpInfo{AM_ABS, 4, CL_READ, OP_CPY};
    case 0x24: return OpInfo{AM_ZP, 3, CL_READ, OP_BIT};
    case 0x2C: return OpInfo{AM_ABS, 4, CL_READ, OP_BIT};
    case 0x10: case 0x30: case 0x50: case 0x70: case 0x90: case 0xB0: case 0xD0: case 0xF0:
      return OpInfo{AM_REL, 2, CL_OTHER, OP_BRANCH};
    case 0x4C: return OpInfo{AM_ABS, 3, CL_OTHER, OP_JMP};
    case 0x6C: return OpInfo{AM_IND, 5, CL_OTHER, OP_JMPI};
    case 0x20: return OpInfo{AM_IND, 6, CL_OTHER, OP_JSR};
    case 0x60: return OpInfo{AM_IMP, 6, CL_OTHER, OP_RTS};
    case 0x40: return OpInfo{AM_IMP, 6, CL_OTHER, OP_RTI};
    case 0x00: return OpInfo{AM_IMP, 7, CL_OTHER, OP_BRK};
    case 0x48: return OpInfo{AM_IMP, 3, CL_OTHER, OP_PHA};
    case 0x08: return OpInfo{AM_IMP, 3, CL_OTHER, OP_PHP};
    case 0x68: return OpInfo{AM_IMP, 4, CL_OTHER, OP_PLA};
    case 0x28: return OpInfo{AM_IMP, 4, CL_OTHER, OP_PLP};
    case 0x18: return OpInfo{AM_IMP, 2, CL_OTHER, OP_CLC};
    case 0x38: return OpInfo{AM_IMP, 2, CL_OTHER, OP_SEC};
    case 0x58: return OpInfo{AM_IMP, 2, CL_OTHER, OP_CLI};
    case 0x78: return OpInfo{AM_IMP, 2, CL_OTHER, OP_SEI};
    case 0xB8: return OpInfo{AM_IMP, 2, CL_OTHER, OP_CLV};
    case 0xD8: return OpInfo{AM_IMP, 2, CL_OTHER, OP_CLD};
    case 0xF8: return OpInfo{AM_IMP, 2, CL_OTHER, OP_SED};
    case 0xEA: return OpInfo{AM_IMP, 2, CL_OTHER, OP_NOP};
    case 0xAA: return OpInfo{AM_IMP, 2, CL_OTHER, OP_TAX};
    case 0x8A: return OpInfo{AM_IMP, 2, CL_OTHER, OP_TXA};
    case 0xA8: return OpInfo{AM_IMP, 2, CL_OTHER, OP_TAY};
    case 0x98: return OpInfo{AM_IMP, 2, CL_OTHER, OP_TYA};
    case 0xBA: return OpInfo{AM_IMP, 2, CL_OTHER, OP_TSX};
    case 0x9A: return OpInfo{AM_IMP, 2, CL_OTHER, OP_TXS};
    case 0xE8: return OpInfo{AM_IMP, 2, CL_OTHER, OP_INX};
    case 0xCA: return OpInfo{AM_IMP, 2, CL_OTHER, OP_DEX};
    case 0xC8: return OpInfo{AM_IMP, 2, CL_OTHER, OP_INY};
    case 0x88: return OpInfo{AM_IMP, 2, CL_OTHER, OP_DEY};
    // the paper's extra opcode bytes
    case 0xEB: return OpInfo{AM_IMM, 2, CL_READ, OP_SBC};   // USBC
    case 0x1A: case 0x3A: case 0x5A: case 0x7A: case 0xDA: case 0xFA:
      return OpInfo{AM_IMP, 2, CL_OTHER, OP_NOP};
    case 0x80: case 0x82: case 0xC2: case 0xE2: return OpInfo{AM_IMM, 2, CL_READ, OP_NOPR};
    case 0x04: case 0x44: case 0x64: return OpInfo{AM_ZP, 3, CL_READ, OP_NOPR};
    case 0x14: case 0x34: case 0x54: case 0x74: case 0xD4: case 0xF4: return OpInfo{AM_ZPX, 4, CL_READ, OP_NOPR};
    case 0x0C: return OpInfo{AM_ABS, 4, CL_READ, OP_NOPR};
    case 0x1C: case 0x3C: case 0x5C: case 0x7C: case 0xDC: case 0xFC: return OpInfo{AM_ABX, 4, CL_READ, OP_NOPR};
    case 0xA7: return OpInfo{AM_ZP, 3, CL_READ, OP_LAX};
    case 0xB7: return OpInfo{AM_ZPY, 4, CL_READ, OP_LAX};
    case 0xAF: return OpInfo{AM_ABS, 4, CL_READ, OP_LAX};
    case 0xBF: return OpInfo{AM_ABY, 4, CL_READ, OP_LAX};
    case 0xA3: return OpInfo{AM_INX, 6, CL_READ, OP_LAX};
    case 0xB3: return OpInfo{AM_INY, 5, CL_READ, OP_LAX};
    case 0x87: return OpInfo{AM_ZP, 3, CL_STORE, OP_SAX};
    case 0x97: return OpInfo{AM_ZPY, 4, CL_STORE, OP_SAX};
    case 0x8F: return OpInfo{AM_ABS, 4, CL_STORE, OP_SAX};
    case 0x83: return OpInfo{AM_INX, 6, CL_STORE, OP_SAX};
    default: return OpInfo{AM_JAM, 1, CL_OTHER, OP_JAM};
  }
}


// Whether the backward sweep does anything for an instruction: moves an
// adjoint between a register and memory (loads, stores, logic and
// arithmetic reads, read-modify-writes, transfers) or clears a cell or
// register it overwrites with a value that carries no gradient (pushes, TSX).
// Branches, compares, BIT, flag operations, register increments, jumps,
// returns, PLP, TXS and NOP leave every adjoint as it is, so the tape does
// not record them.
__host__ __device__ constexpr bool reverse_needed(uint32_t op) {
  const uint32_t id = op_info(op).id;
  return id == OP_LDA || id == OP_LDX || id == OP_LDY || id == OP_ORA || id == OP_AND || id == OP_EOR ||
         id == OP_ADC || id == OP_SBC || id == OP_STA || id == OP_STX || id == OP_STY || id == OP_ASL ||
         id == OP_ROL || id == OP_LSR || id == OP_ROR || id == OP_DEC || id == OP_INC || id == OP_TAX ||
         id == OP_TXA || id == OP_TAY || id == OP_TYA || id == OP_TSX || id == OP_PHA || id == OP_PHP ||
         id == OP_PLA || id == OP_JSR || id == OP_BRK || id == OP_LAX || id == OP_SAX;
}

// Machine registers of one env (kept in registers inside a launch).
struct Regs {
  uint32_t A, X, Y, SP, PC;
  uint32_t fC, fV, fD, fI;   // flags as 0/1
  uint32_t zsrc, nsrc;       // Z = (zsrc == 0), N = nsrc bit 7
  uint32_t bank, jam;
  uint32_t cyc;              // CPU cycles mod 2^32
  int32_t fc;                // 76 * scanline + line cycle, frame relative
  uint32_t fs;               // line cycle at which the current frame began
  uint32_t tw, tv, tsh;      // timer: write cycle, value, log2 interval
  uint32_t col0, colpf, colbk, ctrl, pf0, pf1, pf2, grp0, hmp0, pos, vblank, vsync;
  int32_t hml;               // scanline of the last early HMOVE (-1 none)
  // the rest of the TIA lives in shared memory (vcs_tia.cuh); here only its
  // summary bits, the collision latches and possible pairs, and the colour
  // clock up to which collisions have been evaluated
  uint32_t xo, cx;
  int32_t cxc;
  uint32_t swcha;
  uint32_t inpt4;            // INPT4 in bits 0-7; bit 8 holds the console RESET switch down
                             // (SWCHB then reads $0A instead of $0B)
  uint32_t intim_live;       // the last INTIM read came before underflow
  // fully relaxed casts only (probe and FULL machines): the relaxed operand
  // bytes fetched ahead, and the cast counts (ROM/RAM reads by instructions
  // and the exact ones, conditional branches and the exact ones)
  uint32_t pfr;
  uint32_t fr_reads, fr_exact, fr_br, fr_br_exact;
};

__device__ __forceinline__ uint32_t pack_p(const Regs& r) {
  return (r.nsrc & 0x80) | (r.fV << 6) | 0x30 | (r.fD << 3) | (r.fI << 2) |
         ((r.zsrc & 0xFF) == 0 ? 2u : 0u) | r.fC;
}
__device__ __forceinline__ void unpack_p(Regs& r, uint32_t p) {
  r.nsrc = p & 0x80;
  r.zsrc = (p & 2) ? 0u : 1u;
  r.fV = (p >> 6) & 1;
  r.fD = (p >> 3) & 1;
  r.fI = (p >> 2) & 1;
  r.fC = p & 1;
}

// The fully relaxed forward's constants (Section 4's temperature-limit
// study): float32 weights e^{-k/T} of the temperature read for k <= W, the
// float32 gate values sigma(alpha) and sigma(-alpha) of a crisp-flag branch,
// and the size of the block's ROM tensor (2048 for 2K carts, 1024 for E0
// carts, whose reads are relaxed within their slice, else 4096: a banked
// read is relaxed within its bank).
constexpr int kMaxFullW = 120;
struct FullParams {
  float ek[kMaxFullW + 1];
  int32_t W;
  float g1, g0;
  int32_t rom_m;
};

// First hotspot of a bank-switched cart of nb banks: F8 $1FF8-9, F6
// $1FF6-9, F4 $1FF4-B; no hotspot for the others.
__host__ __device__ constexpr uint32_t first_hotspot(uint32_t nb) {
  return nb == 2 ? 0x1FF8u : nb == 4 ? 0x1FF6u : nb == 8 ? 0x1FF4u : 0xFFFFu;
}

// Everything a thread needs besides its registers.
struct Ctx {
  const uint8_t* rom;        // shared: cart image (4 KB, or 8 KB for F8)
  uint8_t* ram;              // shared: this env's RAM byte 0 (stride e4 per word)
  uint32_t* line;            // shared: this env's line-buffer word 0 (stride E)
  uint32_t* tx;              // shared: this env's cold TIA words (6, stride E; vcs_tia.cuh)
  uint32_t ft;               // 1: the whole TIA; 0: the subset machine (player 0, playfield,
                             // background; the other object registers ignored, collisions read 0)
  const DecodeTables* dt;    // shared
  uint32_t e4;               // 4 * envs per block
  uint32_t E;                // envs per block
  uint32_t nb;               // 4 KB banks of a bank-switched cart (F8 2, F6 4, F4 8), else 0
  uint32_t hot;              // its first hotspot: an access to hot + j selects bank j
  uint32_t sc;               // 1: Superchip cart, whose 128 bytes of cartridge RAM are RAM
                             // words 32..63 (written at $1000-$107F, read at $1080-$10FF)
  uint32_t e0;               // 1: E0 cart: Regs::bank holds the slices of segments 0..2
                             // (3 bits each); segment 3 shows slice 7
  uint32_t fe;               // 1: FE cart: two 4 KB banks chosen by JSR and RTS made at the
                             // top of the stack (exec_op), no hotspot
  uint32_t rw;               // RAM words of this env: 32, or 64 with the Superchip's RAM
  int32_t ystart;
  // Threads per env: T lanes run one env's machine in lockstep (identical
  // registers; their identical shared-memory writes coincide) and split the
  // data-parallel work by chunks of four 4-pixel groups (16 pixels): chunk q
  // of a scanline belongs to replica q mod T, which alone draws, flushes,
  // zeroes and sums it, so no replica reads what another wrote.
  uint32_t rank, T;
  uint32_t gmask;            // warp lanes of this env's replicas
  const FullParams* fp;      // shared: the relaxed casts' constants (FULL study kernel only)
};

__device__ __forceinline__ bool owns_chunk(const Ctx& c, uint32_t q) { return (q & (c.T - 1)) == c.rank; }

// First chunk at or after q0 that this replica owns (T is a power of two).
__device__ __forceinline__ uint32_t first_owned_chunk(const Ctx& c, uint32_t q0) {
  return q0 + ((c.rank - q0) & (c.T - 1));
}

__device__ __forceinline__ uint32_t ram_rd(const Ctx& c, uint32_t a) {
  a &= 0x7F;
  return c.ram[(a >> 2) * c.e4 + (a & 3)];
}
__device__ __forceinline__ void ram_wr(const Ctx& c, uint32_t a, uint32_t v) {
  a &= 0x7F;
  c.ram[(a >> 2) * c.e4 + (a & 3)] = (uint8_t)v;
}
// The Superchip's RAM byte a & 0x7F (RAM words 32..63).
__device__ __forceinline__ uint32_t cram_rd(const Ctx& c, uint32_t a) {
  a &= 0x7F;
  return c.ram[(32 + (a >> 2)) * c.e4 + (a & 3)];
}
__device__ __forceinline__ void cram_wr(const Ctx& c, uint32_t a, uint32_t v) {
  a &= 0x7F;
  c.ram[(32 + (a >> 2)) * c.e4 + (a & 3)] = (uint8_t)v;
}
// Offset in the block's cart image of cartridge address a (13-bit): the
// bank's 4 KB (2K images are mirrored, 4K images have bank 0), or for E0 the
// 1 KB slice its segment shows.
__device__ __forceinline__ uint32_t rom_off(const Ctx& c, const Regs& r, uint32_t a) {
  if (c.e0) {
    const uint32_t seg = (a >> 10) & 3u;
    const uint32_t slice = seg == 3u ? 7u : (r.bank >> (3u * seg)) & 7u;
    return (slice << 10) | (a & 0x3FFu);
  }
  return (r.bank << 12) | (a & 0xFFFu);
}
// The bank (E0: slice) a tape record keeps for a cartridge reference: the
// backward maps a ROM read at `a` back to its image byte with it.
__device__ __forceinline__ uint32_t rec_unit(const Ctx& c, const Regs& r, uint32_t a) {
  return c.e0 ? (rom_off(c, r, a) >> 10) & 7u : r.bank;
}
// Bank switching on an access (read or write) to 13-bit address a: F8 / F6
// / F4 hotspot j selects bank j; E0's $1FE0+j / $1FE8+j / $1FF0+j map slice
// j into segment 0 / 1 / 2.
__device__ __forceinline__ void hotspot(const Ctx& c, Regs& r, uint32_t a) {
  r.bank = a - c.hot < c.nb ? a - c.hot : r.bank;
  if (c.e0) {
    const uint32_t j = a - 0x1FE0u;
    if (j < 24u) {
      const uint32_t sh = 3u * (j >> 3);
      r.bank = (r.bank & ~(7u << sh)) | ((j & 7u) << sh);
    }
  }
}
// The n (<= 5) cartridge bytes from window offset `off` are plain ROM under
// one mapping: no bank-switch hotspot ($1FF4 on; E0 $1FE0 on) and no
// Superchip port among them, and for E0 all in one segment.  Fetch-ahead
// and the timer-poll check read only such bytes.
__device__ __forceinline__ bool plain_rom(const Ctx& c, uint32_t off, uint32_t n) {
  if (c.e0) return (off & 0x3FFu) + n <= 0x400u && off + n <= 0xFE0u;
  return off + n <= 0xFF4u && off >= (c.sc << 8);
}

// Superchip ports of a 13-bit address: the read port $1080-$10FF and the
// write port $1000-$107F (a read there returns the ROM byte, a write to the
// read port does nothing).
__device__ __forceinline__ bool sc_read_port(const Ctx& c, uint32_t a) { return c.sc && (a & 0x1F80) == 0x1080; }
__device__ __forceinline__ bool sc_write_port(const Ctx& c, uint32_t a) { return c.sc && (a & 0x1F80) == 0x1000; }

__device__ __forceinline__ uint32_t div76(uint32_t x) { return x / 76u; }
__device__ __forceinline__ uint32_t div228(uint32_t x) { return x / 228u; }

// Timer value read k = t - tw cycles after the last write.
__device__ __forceinline__ uint32_t intim_at(const Regs& r, uint32_t t) {
  uint32_t k = t - r.tw;
  uint32_t vi = r.tv << r.tsh;
  if (k <= vi) return r.tv - ((k + (1u << r.tsh) - 1) >> r.tsh);
  return (vi - k) & 0xFF;
}
__device__ __forceinline__ uint32_t timint_at(const Regs& r, uint32_t t) {
  uint32_t k = t - r.tw;
  return k > (r.tv << r.tsh) ? 0x80u : 0u;
}

// Shared-memory index of the staged gradients of 4-pixel group g (0..39) of
// env slot `slot` in a block of E envs (a power of two): row g, the slot
// rotated by g's chunk (g / 4).  The T replicas of an env read different
// chunks at once; without the rotation they all hit the same four banks.
__device__ __forceinline__ uint32_t grow_at(uint32_t g, uint32_t E, uint32_t slot) {
  return g * E + (slot ^ ((g >> 2) & (E - 1)));
}

}  // namespace vcs

// The rest of the TIA (player 1, missiles, ball, collisions) needs Ctx and
// Regs above; the span renderer below needs its general path.
#include "vcs_tia.cuh"

namespace vcs {

// ----------------------------------------------------------------------------
// TIA rendering (span catch-up)
// ----------------------------------------------------------------------------

struct Render {
  bool on;                   // drawing the frame this step returns
  int32_t cur;               // render cursor, colour clock in frame coordinates
  uint8_t* out_u8;           // screen of this env (uint8 [210][160]) or null
  float* out_f32;            // screen of this env (f32) or null
  const float* gs;           // pixel gradients of the returned frame [210][160]
                             // (backward recompute only) or null
  float4* grow;              // shared: the block's staged gradient rows (grow_at)
  uint32_t gslot;            // this env's slot in the block
  int32_t gline;             // frame line held in grow, or -1
};


// Stage the gradient row of frame line `line` into shared memory: the 40
// loads go out in four batches of ten, so a row costs a few memory latencies
// instead of one per 4-pixel group.
__device__ __forceinline__ void stage_grad_row(const Ctx& c, Render& rd, int32_t line) {
  const float4* src = reinterpret_cast<const float4*>(rd.gs + (line - c.ystart) * kScreenW);
  // this replica's chunks, two at a time (eight loads in flight)
  for (uint32_t q = c.rank; q < 10; q += 2 * c.T) {
    const uint32_t q2 = q + c.T;
    float4 t[8];
#pragma unroll
    for (int k = 0; k < 4; k++) t[k] = __ldg(src + 4 * q + k);
#pragma unroll
    for (int k = 0; k < 4; k++) t[4 + k] = q2 < 10 ? __ldg(src + 4 * q2 + k) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 4; k++) rd.grow[grow_at(4 * q + k, c.E, rd.gslot)] = t[k];
    if (q2 < 10) {
#pragma unroll
      for (int k = 0; k < 4; k++) rd.grow[grow_at(4 * q2 + k, c.E, rd.gslot)] = t[4 + k];
    }
  }
  rd.gline = line;
}

// 40-bit playfield mask, one bit per 4-pixel block (left half then right).
__device__ __forceinline__ uint64_t pf_mask(const Regs& r) {
  uint32_t p20 = ((r.pf0 >> 4) & 0xF) | ((__brev(r.pf1) >> 24) << 4) | ((r.pf2 & 0xFF) << 12);
  uint32_t right = (r.ctrl & 1) ? (__brev(p20) >> 12) : p20;
  return (uint64_t)p20 | ((uint64_t)right << 20);
}

// Four pixels of group g (pixels 4g..4g+3) as one word, pixel 4g in the low
// byte.  Playfield bits cover whole groups; the player's eight pixels start
// at `pos` and may wrap past column 159.
__device__ __forceinline__ uint32_t group_pixels(uint32_t g, uint64_t pfm, uint32_t grev, uint32_t pos,
                                                 uint32_t on_pf, uint32_t off_pf, uint32_t on_bk,
                                                 uint32_t off_bk) {
  int32_t d0 = (int32_t)(4 * g) - (int32_t)pos;
  d0 += d0 < 0 ? 160 : 0;
  uint32_t nib = d0 < 8 ? (grev >> d0) & 0xF : (d0 > 156 ? (grev << (160 - d0)) & 0xF : 0u);
  bool pf = (pfm >> g) & 1;
  uint32_t on = pf ? on_pf : on_bk, off = pf ? off_pf : off_bk;
  uint32_t m = ((nib & 1) | ((nib & 2) << 7) | ((nib & 4) << 14) | ((nib & 8) << 21)) * 0xFFu;
  return (on & m) | (off & ~m);
}

// Draw pixels [x0, x1) of one scanline into this env's line buffer, or, when
// the tape accumulates pixel gradients (backward recompute), add each pixel's
// gradient to the colour register that owns it.
template <class Tape>
__device__ __forceinline__ void render_span(const Ctx& c, const Regs& r, const Render& rd, Tape& tape, uint32_t x0,
                                            uint32_t x1, int32_t line) {
  const uint32_t g0 = x0 >> 2, g1 = (x1 + 3) >> 2;
  const bool blank_all = (r.vblank & 2) != 0;
  const uint64_t pfm = pf_mask(r);
  const uint32_t grev = __brev(r.grp0 & 0xFF) >> 24;   // bit k = player pixel k
  const uint32_t cp0 = (r.col0 & 0xFE) * 0x01010101u, cpf = (r.colpf & 0xFE) * 0x01010101u,
                 cbk = (r.colbk & 0xFE) * 0x01010101u;
  // colour where the player bit is set / clear, over playfield / background
  const bool pf_first = (r.ctrl & 4) != 0;
  // score mode (CTRLPF bit 1 without bit 2): the playfield takes COLUP0 in
  // the left half (groups 0..19) and COLUP1 in the right one
  const bool score = c.ft && (r.ctrl & 6) == 2;
  const uint32_t col1 = score ? tx_rd(c, 0) & 0xFF : 0u;
  const uint32_t cpfL = score ? cp0 : cpf, cpfR = score ? (col1 & 0xFE) * 0x01010101u : cpf;
  const uint32_t on_pf = pf_first ? cpf : cp0, on_bk = cp0, off_bk = cbk;
  const uint32_t blank_g = (line == r.hml) ? 2u : 0u;
  // objects beyond player 0 and the playfield (or a copied, sized, reflected
  // or delayed player 0) take the general path, out of line
  const bool general = c.ft && (r.xo & kXoGen) != 0;
  if constexpr (Tape::kAcc) {
    // Sum the span's pixel gradients per owning colour register: plain FP32
    // within the span (at most 160 terms), one compensated add per owner per
    // span into the version sums.  A group without player pixels belongs
    // wholly to the playfield or the background colour.
    if (blank_all || !rd.gs) return;
    // with the graphics-bit surrogate every object of the whole TIA has bits
    // in play somewhere, drawn or not: the general path sums them
    if (general || (c.ft && Tape::graphics)) {
      const OwnerSums s = sums_general(make_view(c, r), rd.grow, c.E, rd.gslot, c.rank, c.T, x0, x1, blank_g,
                                       tape.sampler);
      tape.pixels(s.s0, s.s1, s.s2, s.pos, s.s3);
      if constexpr (Tape::graphics) {
        const GbSums gb = gbits_general(make_view(c, r), rd.grow, c.E, rd.gslot, c.rank, c.T, x0, x1, blank_g);
        tape.gbits_all(gb.v);
      }
      return;
    }
    const float4* gl = rd.grow;   // this line's gradients, staged by render_to
    const uint32_t gs0 = g0 < blank_g ? blank_g : g0;
    // graphics-bit surrogate: the player's groups are summed pixel by pixel
    // even when GRP0 is zero (its bits' with-minus-without colours still
    // count there), and each playfield register gets the sum of its
    // columns' gradients times (C_with - C_without)
    constexpr bool kGB = Tape::graphics;
    // Bulk pass: whole groups inside the span that hold no player pixel
    // belong wholly to COLUPF (playfield bit set) or COLUBK; four groups per
    // turn (g1 <= 40 keeps every guarded load inside the row).  The at most five other groups (the span's two
    // edge groups, the player's three) are summed pixel by pixel below.
    const uint32_t gp = r.pos >> 2;
    auto special = [&](uint32_t g) {
      uint32_t dp = g + 40u - gp;
      dp -= dp >= 40u ? 40u : 0u;
      const bool player = (kGB || grev != 0) && dp < 3u;
      return player || 4 * g < x0 || 4 * g + 4 > x1;
    };
    // the playfield register of group g: PF0 bits cover groups 0-3 of a
    // half, PF1 4-11, PF2 12-19; the right half mirrors with CTRLPF bit 0
    auto pf_reg = [&](uint32_t g) -> uint32_t {
      uint32_t i = g < 20u ? g : ((r.ctrl & 1) ? 39u - g : g - 20u);
      return i < 4u ? 0u : (i < 12u ? 1u : 2u);
    };
    float gb_pf[3] = {0.f, 0.f, 0.f};   // plain groups' gradient sums per playfield register
    float gb_g = 0.f, gb_f[3] = {0.f, 0.f, 0.f};   // pixel-by-pixel graphics-bit sums
    // s_pf: the playfield (its left half in score mode), s_pfR: the right
    // half in score mode
    float s_p0 = 0.f, s_pf = 0.f, s_bk = 0.f, s_pf2 = 0.f, s_bk2 = 0.f, s_pfR = 0.f;
    for (uint32_t ch = first_owned_chunk(c, gs0 >> 2); 4 * ch < g1; ch += c.T) {
      const uint32_t g = 4 * ch;
      const bool right = score && g >= 20;   // a chunk lies wholly in one half
      float4 q[4];
#pragma unroll
      for (uint32_t k = 0; k < 4; k++)
        q[k] = (g + k >= gs0 && g + k < g1) ? gl[grow_at(g + k, c.E, rd.gslot)] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (uint32_t k = 0; k < 4; k++) {
        const uint32_t gg = g + k;
        const float t = (gg < gs0 || gg >= g1 || special(gg)) ? 0.f : (q[k].x + q[k].y) + (q[k].z + q[k].w);
        const bool pf = (pfm >> gg) & 1;
        if constexpr (kGB) {
          const uint32_t rg = pf_reg(gg);
          gb_pf[0] += rg == 0u ? t : 0.f;
          gb_pf[1] += rg == 1u ? t : 0.f;
          gb_pf[2] += rg == 2u ? t : 0.f;
        }
        if (right) {
          s_pfR += pf ? t : 0.f;
          (k & 1 ? s_bk2 : s_bk) += pf ? 0.f : t;
        } else if (k & 1) {
          s_pf2 += pf ? t : 0.f;
          s_bk2 += pf ? 0.f : t;
        } else {
          s_pf += pf ? t : 0.f;
          s_bk += pf ? 0.f : t;
        }
      }
    }
    s_pf += s_pf2;
    s_bk += s_bk2;
    // special groups, each once: pixel ownership with the edge masks
    uint32_t cand[5] = {g0, g1 - 1, gp, gp + 1 >= 40u ? gp + 1 - 40u : gp + 1, gp + 2 >= 40u ? gp + 2 - 40u : gp + 2};
#pragma unroll
    for (int ci = 0; ci < 5; ci++) {
      const uint32_t g = cand[ci];
      bool dup = false;
#pragma unroll
      for (int cj = 0; cj < ci; cj++) dup |= cand[cj] == g;
      if (dup || g < gs0 || g >= g1 || !special(g) || !owns_chunk(c, g >> 2)) continue;
      const float4 q = gl[grow_at(g, c.E, rd.gslot)];
      const uint32_t xb = 4 * g;
      const float v[4] = {(xb + 0 >= x0 && xb + 0 < x1) ? q.x : 0.f, (xb + 1 >= x0 && xb + 1 < x1) ? q.y : 0.f,
                          (xb + 2 >= x0 && xb + 2 < x1) ? q.z : 0.f, (xb + 3 >= x0 && xb + 3 < x1) ? q.w : 0.f};
      int32_t d0 = (int32_t)xb - (int32_t)r.pos;
      d0 += d0 < 0 ? 160 : 0;
      const uint32_t nib = d0 < 8 ? (grev >> d0) & 0xF : (d0 > 156 ? (grev << (160 - d0)) & 0xF : 0u);
      const bool pf = (pfm >> g) & 1;
      // player pixels belong to COLUP0 unless the playfield has priority
      // here; the others to COLUPF over the playfield, else to COLUBK
      float tp = 0.f, tn = 0.f;
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const bool p0 = (nib >> j) & 1;
        tp += p0 ? v[j] : 0.f;
        tn += p0 ? 0.f : v[j];
      }
      const bool pf_wins = pf_first && pf;
      s_p0 += pf_wins ? 0.f : tp;
      (score && g >= 20 ? s_pfR : s_pf) += (pf ? tn : 0.f) + (pf_wins ? tp : 0.f);
      s_bk += pf ? 0.f : tn;
      if constexpr (kGB) {
        // C_with - C_without of the pixel's GRP0 bit (inside the player's
        // 8-pixel span) and of its playfield bit, from the priority logic
        const uint32_t span = d0 < 8 ? (0xFFu >> d0) & 0xF : (d0 > 156 ? (0xFFu << (160 - d0)) & 0xF : 0u);
        const float c0 = (float)(r.col0 & 0xFE), cf = (float)(r.colpf & 0xFE), cb = (float)(r.colbk & 0xFE);
        const float dgrp = pf_wins ? 0.f : (pf ? c0 - cf : c0 - cb);
        float tg = 0.f, tf = 0.f;
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const bool p0 = (nib >> j) & 1;
          tg += ((span >> j) & 1) ? v[j] * dgrp : 0.f;
          tf += v[j] * (p0 ? (pf_first ? cf - c0 : 0.f) : cf - cb);
        }
        gb_g += tg;
        const uint32_t rg = pf_reg(g);
        gb_f[0] += rg == 0u ? tf : 0.f;
        gb_f[1] += rg == 1u ? tf : 0.f;
        gb_f[2] += rg == 2u ? tf : 0.f;
      }
    }
    // Position sampler (Section 3): the player's coverage relaxed with a
    // triangular kernel has, at the integer position, the symmetric slope
    // (b(d - 1) - b(d + 1)) / 2 in pos at column x = pos + d, nonzero only
    // for d in -1..8.  Each such drawn, unblanked column where the player is
    // not behind a playfield pixel adds (C_P0 - C_under) x slope x gradient.
    float s_pos = 0.f;
    if (tape.sampler && grev) {
      const uint32_t xb = 4 * blank_g > x0 ? 4 * blank_g : x0;
      const int32_t cp = (int32_t)(r.col0 & 0xFE);
#pragma unroll 1
      for (int32_t i = 0; i < 10; i++) {
        int32_t x = (int32_t)r.pos - 1 + i;
        x += x < 0 ? 160 : 0;
        x -= x >= 160 ? 160 : 0;
        const uint32_t ux = (uint32_t)x;
        const int32_t d = i - 1;
        const int32_t bl = d >= 1 ? (int32_t)((grev >> (d - 1)) & 1) : 0;
        const int32_t br = d + 1 < 8 ? (int32_t)((grev >> (d + 1)) & 1) : 0;
        if (bl == br || ux < xb || ux >= x1 || !owns_chunk(c, ux >> 4)) continue;
        const uint32_t g = ux >> 2;
        const bool pf = (pfm >> g) & 1;
        if (pf_first && pf) continue;
        const float4 q = gl[grow_at(g, c.E, rd.gslot)];
        const uint32_t k = ux & 3;
        const float w = k == 0 ? q.x : (k == 1 ? q.y : (k == 2 ? q.z : q.w));
        const uint32_t cpfx = score ? (ux < 80 ? r.col0 : col1) : r.colpf;   // the playfield's colour here
        const int32_t under = (int32_t)((pf ? cpfx : r.colbk) & 0xFE);
        s_pos += (0.5f * (float)((bl - br) * (cp - under))) * w;
      }
    }
    // score mode: the playfield sums belong to COLUP0 (left) and COLUP1 (right)
    if (score) tape.pixels(s_p0 + s_pf, 0.f, s_bk, s_pos, s_pfR);
    else tape.pixels(s_p0, s_pf, s_bk, s_pos, 0.f);
    if constexpr (kGB) {
      // a plain group holds no player column: its playfield bit's colours
      // are COLUPF with the bit and COLUBK without
      const float dpf = (float)(r.colpf & 0xFE) - (float)(r.colbk & 0xFE);
      tape.gbits(gb_g, gb_f[0] + dpf * gb_pf[0], gb_f[1] + dpf * gb_pf[1], gb_f[2] + dpf * gb_pf[2]);
    }
  } else {
    // Groups g0 and gl may be partly inside [x0, x1); the ones between are
    // whole words.  Background and playfield first (one select per group,
    // the interior unrolled so independent stores overlap), then the
    // player's two or three groups and the HMOVE blank redrawn on top.
    uint32_t* const line = c.line;
    const uint32_t E = c.E, gl = g1 - 1;
    const uint32_t m0 = 0xFFFFFFFFu << (8 * (x0 & 3));
    const uint32_t m1 = (x1 & 3) ? 0xFFFFFFFFu >> (8 * (4 - (x1 & 3))) : 0xFFFFFFFFu;
    auto put = [&](uint32_t g, uint32_t w) {
      const uint32_t mask = (g == g0 ? m0 : 0xFFFFFFFFu) & (g == gl ? m1 : 0xFFFFFFFFu);
      uint32_t* dst = line + g * E;
      *dst = mask == 0xFFFFFFFFu ? w : ((*dst & ~mask) | (w & mask));
    };
    // The two edge groups (partly inside the span) are masked; the interior
    // ones are plain stores, this replica's chunks of four groups only.
    if (blank_all) {
      if (owns_chunk(c, g0 >> 2)) put(g0, 0u);
      if (gl > g0 && owns_chunk(c, gl >> 2)) put(gl, 0u);
      for (uint32_t ch = first_owned_chunk(c, (g0 + 1) >> 2); 4 * ch < gl; ch += c.T)
#pragma unroll
        for (uint32_t k = 0; k < 4; k++)
          if (4 * ch + k > g0 && 4 * ch + k < gl) line[(4 * ch + k) * E] = 0u;
      return;
    }
    if (general) {
      draw_general(make_view(c, r), c.line, c.E, c.rank, c.T, x0, x1, blank_g);
      return;
    }
    if (owns_chunk(c, g0 >> 2)) put(g0, ((pfm >> g0) & 1) ? (g0 < 20 ? cpfL : cpfR) : cbk);
    if (gl > g0 && owns_chunk(c, gl >> 2)) put(gl, ((pfm >> gl) & 1) ? (gl < 20 ? cpfL : cpfR) : cbk);
    for (uint32_t ch = first_owned_chunk(c, (g0 + 1) >> 2); 4 * ch < gl; ch += c.T) {
      const uint32_t g = 4 * ch;
      const uint32_t pfs = (uint32_t)(pfm >> g) & 0xF;
      const uint32_t cpf = g < 20 ? cpfL : cpfR;   // a chunk lies wholly in one half
      if (g > g0 && g + 4 <= gl) {   // the whole chunk is interior
#pragma unroll
        for (uint32_t k = 0; k < 4; k++) line[(g + k) * E] = ((pfs >> k) & 1) ? cpf : cbk;
      } else {
#pragma unroll
        for (uint32_t k = 0; k < 4; k++)
          if (g + k > g0 && g + k < gl) line[(g + k) * E] = ((pfs >> k) & 1) ? cpf : cbk;
      }
    }
    if (grev) {
      const uint32_t gp = r.pos >> 2;
#pragma unroll
      for (uint32_t k = 0; k < 3; k++) {
        uint32_t g = gp + k;
        g -= g >= 40 ? 40u : 0u;
        if (g >= g0 && g < g1 && owns_chunk(c, g >> 2))
          put(g, group_pixels(g, pfm, grev, r.pos, on_pf, g < 20 ? cpfL : cpfR, on_bk, off_bk));
      }
    }
    for (uint32_t g = g0; g < blank_g && g < g1; g++)
      if (owns_chunk(c, g >> 2)) put(g, 0u);
  }
}

__device__ __forceinline__ void flush_row(const Ctx& c, Render& rd, int32_t row) {
  if (rd.out_u8) {
    uint4* dst = reinterpret_cast<uint4*>(rd.out_u8 + row * kScreenW);
#pragma unroll
    for (uint32_t q = 0; q < 10; q++) {
      if (!owns_chunk(c, q)) continue;
      uint4 v;
      v.x = c.line[(4 * q + 0) * c.E];
      v.y = c.line[(4 * q + 1) * c.E];
      v.z = c.line[(4 * q + 2) * c.E];
      v.w = c.line[(4 * q + 3) * c.E];
      dst[q] = v;
    }
  } else if (rd.out_f32) {
    float4* dst = reinterpret_cast<float4*>(rd.out_f32 + row * kScreenW);
#pragma unroll 2
    for (uint32_t q = 0; q < 10; q++)
#pragma unroll
      for (uint32_t k = 0; k < 4; k++) {
        if (!owns_chunk(c, q)) continue;
        const uint32_t v = c.line[(4 * q + k) * c.E];
        dst[4 * q + k] = make_float4((float)(v & 0xFF), (float)((v >> 8) & 0xFF), (float)((v >> 16) & 0xFF),
                                     (float)(v >> 24));
      }
  }
#pragma unroll
  for (uint32_t q = 0; q < 10; q++)
#pragma unroll
    for (uint32_t k = 0; k < 4; k++)
      if (owns_chunk(c, q)) c.line[(4 * q + k) * c.E] = 0u;
}

__device__ __forceinline__ void zero_rows(const Ctx& c, Render& rd, int32_t row0) {
  if (row0 < 0) row0 = 0;
  for (int32_t row = row0; row < kScreenH; row++) {
    if (rd.out_u8) {
      uint4* dst = reinterpret_cast<uint4*>(rd.out_u8 + row * kScreenW);
#pragma unroll
      for (uint32_t q = 0; q < 10; q++)
        if (owns_chunk(c, q)) dst[q] = make_uint4(0, 0, 0, 0);
    } else if (rd.out_f32) {
      float4* dst = reinterpret_cast<float4*>(rd.out_f32 + row * kScreenW);
      for (uint32_t q = c.rank; q < 10; q += c.T)
#pragma unroll
        for (uint32_t k = 0; k < 4; k++) dst[4 * q + k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

// Draw colour clocks [rd.cur, target) of the current frame.
template <class Tape>
__device__ __forceinline__ void render_to(const Ctx& c, const Regs& r, Render& rd, Tape& tape, int32_t target) {
  const int32_t top = 228 * c.ystart, bottom = 228 * (c.ystart + kScreenH);
  if (rd.cur < top) rd.cur = target < top ? target : top;
  if (target > bottom) target = bottom;
  while (rd.cur < target) {
    int32_t line = (int32_t)div228((uint32_t)rd.cur);
    int32_t lbeg = 228 * line, lend = lbeg + 228;
    int32_t seg = target < lend ? target : lend;
    int32_t h0 = rd.cur - lbeg, h1 = seg - lbeg;
    uint32_t x0 = (uint32_t)(h0 > 68 ? h0 : 68) - 68u;
    uint32_t x1 = (uint32_t)(h1 > 68 ? h1 : 68) - 68u;
    if constexpr (Tape::kAcc) {
      if (x1 > x0 && rd.gs && line != rd.gline) stage_grad_row(c, rd, line);
    }
    if (x1 > x0) render_span(c, r, rd, tape, x0, x1, line);
    if (!Tape::kAcc && seg == lend) flush_row(c, rd, line - c.ystart);
    rd.cur = seg;
  }
  __syncwarp(c.gmask);   // replicas leave the split work together
}

// Close the returned frame at colour clock `end`: draw up to it, flush the
// partly drawn row and zero the rows the frame never reached.
template <class Tape>
__device__ __forceinline__ void finish_frame(const Ctx& c, const Regs& r, Render& rd, Tape& tape, int32_t end) {
  render_to(c, r, rd, tape, end);
  if (Tape::kAcc || rd.cur >= 228 * (c.ystart + kScreenH)) return;
  int32_t row = (int32_t)div228((uint32_t)rd.cur) - c.ystart;
  if (row >= 0) {
    flush_row(c, rd, row);
    zero_rows(c, rd, row + 1);
  } else {
    zero_rows(c, rd, 0);
  }
  __syncwarp(c.gmask);
}

// ----------------------------------------------------------------------------
// Deferred rasterisation (hard mode, subset machine, steps that return screens)
// ----------------------------------------------------------------------------
// The interpreter does not draw the frame a step returns.  It appends each
// write to a register that changes the picture (VBLANK, COLUP0, COLUPF,
// COLUBK, CTRLPF, PF0-2, GRP0, RESP0, HMOVE) to a log of its env in global
// memory, after the state of those registers when the frame began, and the
// raster kernel (vcs_raster.cu) then draws every scanline of every env in
// parallel.  The interpreter's dependent chain loses the drawing work.
//
// A log entry: frame cycle of the write << 16 | early-HMOVE flag (bit 14) |
// register << 8 | value; for RESP0 and HMOVE the value is player 0's new
// position, which the interpreter has computed, so the raster only assigns.
// The header of an env (kRasterHdr words): [0] entries logged; [1] the
// colour clock at which the frame began; [2] the one at which it ended; [3]
// COLUP0 | COLUPF << 8 | COLUBK << 16 | CTRLPF << 24, [4] PF0 | PF1 << 8 |
// PF2 << 16 | GRP0 << 24, [5] player 0's position | VBLANK << 8 (| HMP0 <<
// 16 with the whole TIA) and [6] the early-HMOVE line (int32, -1 none), all
// when the frame began; with the whole TIA [7..10] the cold words w0..w3.
// The whole TIA's entries are raw writes (frame cycle << 16 | register << 8
// | value) that its raster replays with the interpreter's own functions.
//
// The log never fills: a frame's instructions start before cycle kLineCap x
// kLineCycles (the watchdog ends it after the first that reaches it), the
// last one writes within 7 cycles plus a WSYNC halt of at most 75, and no
// instruction writes more than 3 times in 7 cycles (BRK pushes 3 bytes in 7,
// which land on TIA registers when the stack pointer is below $80; JSR 2 in
// 6; stores and pushes 1 in 3 or more).
constexpr int kRasterHdr = 12;
constexpr int kRasterLogCap = ((kLineCap * kLineCycles + 7 + 75) * 3 + 6) / 7;
constexpr uint32_t kRasterEarly = 1u << 14;
constexpr int32_t kErrRasterLog = 3;   // device error word: a log passed kRasterLogCap

__device__ __forceinline__ void raster_snapshot(const Regs& r, uint32_t* h) {
  h[3] = (r.col0 & 0xFF) | ((r.colpf & 0xFF) << 8) | ((r.colbk & 0xFF) << 16) | ((r.ctrl & 0xFF) << 24);
  h[4] = (r.pf0 & 0xFF) | ((r.pf1 & 0xFF) << 8) | ((r.pf2 & 0xFF) << 16) | ((r.grp0 & 0xFF) << 24);
  h[5] = (r.pos & 0xFF) | ((r.vblank & 0xFF) << 8);
  h[6] = (uint32_t)r.hml;
}

// The drawing registers from header words 3..6.
__device__ __forceinline__ void raster_restore(Regs& r, uint32_t w3, uint32_t w4, uint32_t w5, uint32_t w6) {
  r.col0 = w3 & 0xFF; r.colpf = (w3 >> 8) & 0xFF; r.colbk = (w3 >> 16) & 0xFF; r.ctrl = w3 >> 24;
  r.pf0 = w4 & 0xFF; r.pf1 = (w4 >> 8) & 0xFF; r.pf2 = (w4 >> 16) & 0xFF; r.grp0 = w4 >> 24;
  r.pos = w5 & 0xFF; r.vblank = (w5 >> 8) & 0xFF;
  r.hml = (int32_t)w6;
}

// Apply one log entry to the drawing registers.
__device__ __forceinline__ void raster_apply(Regs& r, uint32_t e) {
  const uint32_t reg = (e >> 8) & 0x3F, v = e & 0xFF;
  r.vblank = reg == 0x01 ? v : r.vblank;
  r.col0 = reg == 0x06 ? v : r.col0;
  r.colpf = reg == 0x08 ? v : r.colpf;
  r.colbk = reg == 0x09 ? v : r.colbk;
  r.ctrl = reg == 0x0A ? v : r.ctrl;
  r.pf0 = reg == 0x0D ? v : r.pf0;
  r.pf1 = reg == 0x0E ? v : r.pf1;
  r.pf2 = reg == 0x0F ? v : r.pf2;
  r.grp0 = reg == 0x1B ? v : r.grp0;
  r.pos = (reg == 0x10 || reg == 0x2A) ? v : r.pos;
  r.hml = (e & kRasterEarly) ? (int32_t)div76(e >> 16) : r.hml;
}

}  // namespace vcs
