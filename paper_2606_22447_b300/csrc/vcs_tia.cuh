// The rest of the TIA for the per-thread machine: player 1, the two
// missiles, the ball, NUSIZ copies and sizes, REFP reflection, vertical
// delay, missile locks, score mode and the collision latches.
//
// Readings (the same constants as the oracle's): players are 8-bit graphics,
// bit 7 leftmost unless REFP bit 3 reflects them, scaled x1 / x2 / x4 and
// copied at +16 / +32 / +64 by NUSIZ; missiles 1 / 2 / 4 / 8 wide (NUSIZ
// bits 4-5) in the player's copies, the ball 1 / 2 / 4 / 8 wide (CTRLPF
// bits 4-5); RESP1 puts player 1 at 3 in HBLANK else at the beam plus 5,
// RESM0 / RESM1 / RESBL at 2, else the beam plus 4; HMOVE moves every object
// by minus its signed motion nibble; RESMP hides a missile at its player's
// position + 4 x width - 1; a GRP0 write copies GRP1 to its delayed
// register and a GRP1 write copies GRP0 and ENABL, shown when VDEL is set.
// Priority P0/M0 > P1/M1 > PF/BL > BK (score mode: the playfield in COLUP0 /
// COLUP1 by half), or PF/BL first with CTRLPF bit 2.  Collisions latch on
// every visible column of every line until CXCLR.
//
// Layout.  Player 0 and the playfield stay in the interpreter's registers
// (the common carts draw nothing else); the other objects' registers are
// four words per env in shared memory ("cold" words, stride E):
//   w0  COLUP1 | NUSIZ0 << 8 | NUSIZ1 << 16 | flags << 24: REFP0, REFP1,
//       VDELP0, VDELP1, VDELBL, RESMP0, RESMP1 (bits 24..30)
//   w1  GRP1 | delayed GRP0 << 8 | delayed GRP1 << 16 | ENAM0, ENAM1,
//       ENABL, delayed ENABL (bits 24..27)
//   w2  HMP1 | HMM0 << 8 | HMM1 << 16 | HMBL << 24
//   w3  positions of P1 | M0 << 8 | M1 << 16 | BL << 24
//   w4  a copy of PF0 | PF1 << 8 | PF2 << 16 | CTRLPF << 24 and
//   w5  of GRP0 | player 0's position << 8, refreshed at every object
//       write, so the out-of-line collision routine needs no arguments
//       from the interpreter's registers
// and Regs::xo summarises them for the hot path (which cases need the cold
// words at all), Regs::cx holds the collision latches (bits 0..15: bit 2r+1
// = D7 and bit 2r = D6 of read register r) and the pairs that can still
// collide (bits 16..31), Regs::cxc the colour clock up to which collisions
// have been evaluated.  Collisions are evaluated lazily, span by span, only
// while some possible pair has not latched yet, so carts whose collisions
// have all happened pay one compare per object write.
#pragma once
#include <cstdint>

#include "vcs_machine.cuh"

namespace vcs {

enum : uint32_t {
  kW0Refp0 = 1u << 24, kW0Refp1 = 1u << 25, kW0Vdelp0 = 1u << 26, kW0Vdelp1 = 1u << 27, kW0Vdelbl = 1u << 28,
  kW0Resmp0 = 1u << 29, kW0Resmp1 = 1u << 30,
  kW1Enam0 = 1u << 24, kW1Enam1 = 1u << 25, kW1Enabl = 1u << 26, kW1EnablOld = 1u << 27,
};

// Regs::xo bits: kXoGen - drawing needs the general path (player 1, a
// missile or the ball may show, or player 0 is copied, scaled, reflected
// or delayed); kXoG1 - a GRP0 write must copy GRP1 to its delayed register
// (they differ); kXoMove - a cold object's motion register is nonzero;
// kXoLock - a missile is locked to its player.
enum : uint32_t { kXoGen = 1, kXoG1 = 2, kXoMove = 4, kXoLock = 8 };

// Object bits of the collision pairs: P0, P1, M0, M1, BL, PF.
enum : uint32_t { kObP0 = 1, kObP1 = 2, kObM0 = 4, kObM1 = 8, kObBL = 16, kObPF = 32 };

// Latch bits of the pairs among the objects in `act` (read register r's D7
// at bit 2r + 1, D6 at bit 2r): CXM0P (M0P1, M0P0), CXM1P (M1P0, M1P1),
// CXP0FB (P0PF, P0BL), CXP1FB (P1PF, P1BL), CXM0FB (M0PF, M0BL), CXM1FB
// (M1PF, M1BL), CXBLPF (BLPF), CXPPMM (P0P1, M0M1).
__host__ __device__ constexpr uint32_t cx_pairs(uint32_t act) {
  auto both = [act](uint32_t a, uint32_t b) { return (act & a) && (act & b); };
  return (both(kObM0, kObP0) ? 1u << 0 : 0u) | (both(kObM0, kObP1) ? 1u << 1 : 0u) |
         (both(kObM1, kObP1) ? 1u << 2 : 0u) | (both(kObM1, kObP0) ? 1u << 3 : 0u) |
         (both(kObP0, kObBL) ? 1u << 4 : 0u) | (both(kObP0, kObPF) ? 1u << 5 : 0u) |
         (both(kObP1, kObBL) ? 1u << 6 : 0u) | (both(kObP1, kObPF) ? 1u << 7 : 0u) |
         (both(kObM0, kObBL) ? 1u << 8 : 0u) | (both(kObM0, kObPF) ? 1u << 9 : 0u) |
         (both(kObM1, kObBL) ? 1u << 10 : 0u) | (both(kObM1, kObPF) ? 1u << 11 : 0u) |
         (both(kObBL, kObPF) ? 1u << 13 : 0u) | (both(kObM0, kObM1) ? 1u << 14 : 0u) |
         (both(kObP0, kObP1) ? 1u << 15 : 0u);
}

__device__ __forceinline__ uint32_t tx_rd(const Ctx& c, uint32_t w) { return c.tx[w * c.E]; }
__device__ __forceinline__ void tx_wr(const Ctx& c, uint32_t w, uint32_t v) { c.tx[w * c.E] = v; }

// Summary bits (x) and the collision word with its possible pairs (y) from
// the cold words (player 0 and the playfield always count as possible).
__device__ __forceinline__ uint2 cold_summary_of(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t cx) {
  const uint32_t g1 = (w0 & kW0Vdelp1) ? (w1 >> 16) & 0xFF : w1 & 0xFF;
  const bool m0 = (w1 & kW1Enam0) && !(w0 & kW0Resmp0), m1 = (w1 & kW1Enam1) && !(w0 & kW0Resmp1);
  const bool bl = (w0 & kW0Vdelbl) ? (w1 & kW1EnablOld) != 0 : (w1 & kW1Enabl) != 0;
  const bool gen = g1 != 0 || m0 || m1 || bl || ((w0 >> 8) & 7) != 0 || (w0 & (kW0Refp0 | kW0Vdelp0));
  const uint32_t xo = (gen ? kXoGen : 0u) | (((w1 & 0xFF) != ((w1 >> 16) & 0xFF)) ? kXoG1 : 0u) |
                      ((w2 & 0xF0F0F0F0u) ? kXoMove : 0u) | ((w0 & (kW0Resmp0 | kW0Resmp1)) ? kXoLock : 0u);
  const uint32_t act = kObP0 | kObPF | (g1 ? kObP1 : 0u) | (m0 ? kObM0 : 0u) | (m1 ? kObM1 : 0u) | (bl ? kObBL : 0u);
  return make_uint2(xo, (cx & 0xFFFFu) | (cx_pairs(act) << 16));
}
__device__ __forceinline__ void cold_summary(const Ctx& c, Regs& r) {
  const uint2 o = cold_summary_of(tx_rd(c, 0), tx_rd(c, 1), tx_rd(c, 2), r.cx);
  r.xo = o.x;
  r.cx = o.y;
}

// NUSIZ number-and-size field: copy offsets (bits of a mask over 0 / 16 /
// 32 / 64: bit k = copy at 16 k) and the player's scale.
__device__ __forceinline__ uint32_t nusiz_copies(uint32_t mode) {
  // modes 0..7: {0}, {0,16}, {0,32}, {0,16,32}, {0,64}, {0}, {0,32,64}, {0}
  return (0x1D19'7531u >> (4 * (mode & 7))) & 0xF;   // nibble per mode: bit0 +0, bit1 +16, bit2 +32, bit3 +64
}
__device__ __forceinline__ uint32_t player_scale(uint32_t mode) { return mode == 5 ? 2u : (mode == 7 ? 4u : 1u); }

// A snapshot of everything drawing and collisions read, passed by value to
// the out-of-line routines.
struct TiaView {
  uint32_t col;    // COLUP0 | COLUPF << 8 | COLUBK << 16 | COLUP1 << 24
  uint32_t pf;     // PF0 | PF1 << 8 | PF2 << 16 | CTRLPF << 24
  uint32_t p0;     // GRP0 | player 0's position << 8
  uint32_t w0, w1, w3;   // the cold words (w2, the motion registers, plays no part)
};

__device__ __forceinline__ TiaView make_view(const Ctx& c, const Regs& r) {
  TiaView v;
  v.w0 = tx_rd(c, 0);
  v.w1 = tx_rd(c, 1);
  v.w3 = tx_rd(c, 3);
  v.col = (r.col0 & 0xFF) | ((r.colpf & 0xFF) << 8) | ((r.colbk & 0xFF) << 16) | ((v.w0 & 0xFF) << 24);
  v.pf = (r.pf0 & 0xFF) | ((r.pf1 & 0xFF) << 8) | ((r.pf2 & 0xFF) << 16) | ((r.ctrl & 0xFF) << 24);
  v.p0 = (r.grp0 & 0xFF) | ((r.pos & 0xFF) << 8);
  return v;
}

// OR a pattern of `width` (<= 32) columns (bit j = column pos + j, wrapping
// at 160) into a 160-bit mask of five words.
__device__ __forceinline__ void place(uint32_t* m, uint32_t pat, uint32_t width, uint32_t pos) {
  if (!pat) return;
  // split at the wrap: columns pos .. 159 then 0 ..
  const uint32_t first = width < 160u - pos ? width : 160u - pos;
  const uint32_t lo = first >= 32 ? pat : pat & ((1u << first) - 1u), hi = first >= 32 ? 0u : pat >> first;
  const uint32_t w = pos >> 5, s = pos & 31;
  m[w] |= lo << s;
  if (s && w + 1 < 5) m[w + 1] |= (uint32_t)((uint64_t)lo >> (32 - s));
  m[0] |= hi;
}

// Spread the 8 graphic bits (column order: bit j = column j) by scale 1, 2
// or 4 into up to 32 columns.
__device__ __forceinline__ uint32_t scale_bits(uint32_t g, uint32_t sc) {
  if (sc == 1) return g;
  uint32_t out = 0;
  for (uint32_t j = 0; j < 8; j++)
    if ((g >> j) & 1) out |= ((1u << sc) - 1u) << (j * sc);
  return out;
}

// Column masks of the six objects over one scanline (five words each,
// bit x & 31 of word x >> 5 = column x).
struct LineMasks {
  uint32_t p0[5], p1[5], m0[5], m1[5], bl[5], pf[5];
};

// objs: the kOb* objects whose masks are wanted (the others stay empty).
static __device__ __noinline__ void line_masks(const TiaView v, LineMasks& L, uint32_t objs = 0x3F) {
  for (int k = 0; k < 5; k++) L.p0[k] = L.p1[k] = L.m0[k] = L.m1[k] = L.bl[k] = L.pf[k] = 0;
  const uint32_t ctrl = v.pf >> 24, w0 = v.w0, w1 = v.w1, w3 = v.w3;
  // playfield: 20 bits x 4 columns, right half repeated or reflected
  const uint32_t pf0 = v.pf & 0xFF, pf1 = (v.pf >> 8) & 0xFF, pf2 = (v.pf >> 16) & 0xFF;
  const uint32_t p20 = ((pf0 >> 4) & 0xF) | ((__brev(pf1) >> 24) << 4) | (pf2 << 12);
  const uint32_t right = (ctrl & 1) ? (__brev(p20) >> 12) : p20;
  const uint64_t g40 = (uint64_t)p20 | ((uint64_t)right << 20);
  for (uint32_t k = 0; k < 5 && (objs & kObPF); k++) {   // 8 playfield groups -> 32 columns: each bit to a nibble
    uint32_t x = (uint32_t)(g40 >> (8 * k)) & 0xFF;
    x = (x | (x << 12)) & 0x000F000Fu;
    x = (x | (x << 6)) & 0x03030303u;
    x = (x | (x << 3)) & 0x11111111u;
    L.pf[k] = x * 0xFu;
  }
  // players
  for (uint32_t i = 0; i < 2; i++) {
    const uint32_t mode = i ? (w0 >> 16) & 7 : (w0 >> 8) & 7;
    const bool vdel = (w0 & (i ? kW0Vdelp1 : kW0Vdelp0)) != 0, refl = (w0 & (i ? kW0Refp1 : kW0Refp0)) != 0;
    const uint32_t g = vdel ? (w1 >> (i ? 16 : 8)) & 0xFF : (i ? w1 & 0xFF : v.p0 & 0xFF);
    const uint32_t pos = i ? w3 & 0xFF : (v.p0 >> 8) & 0xFF;
    if (!g || !(objs & (i ? kObP1 : kObP0))) continue;
    const uint32_t cols = refl ? g : (__brev(g) >> 24);   // bit j = column j of the copy
    const uint32_t sc = player_scale(mode), pat = scale_bits(cols, sc), cp = nusiz_copies(mode);
    uint32_t* m = i ? L.p1 : L.p0;
    for (uint32_t k = 0; k < 4; k++)
      if ((cp >> k) & 1) {
        const uint32_t p = pos + (k == 3 ? 64u : 16u * k);
        place(m, pat, 8 * sc, p >= 160 ? p - 160 : p);
      }
  }
  // missiles: in the player's copies (one for the double and quad sizes)
  for (uint32_t i = 0; i < 2; i++) {
    const bool on = (w1 & (i ? kW1Enam1 : kW1Enam0)) && !(w0 & (i ? kW0Resmp1 : kW0Resmp0));
    if (!on || !(objs & (i ? kObM1 : kObM0))) continue;
    const uint32_t nus = i ? (w0 >> 16) & 0xFF : (w0 >> 8) & 0xFF;
    const uint32_t wid = 1u << ((nus >> 4) & 3), cp = nusiz_copies(nus & 7);
    const uint32_t pos = (w3 >> (i ? 16 : 8)) & 0xFF;
    uint32_t* m = i ? L.m1 : L.m0;
    for (uint32_t k = 0; k < 4; k++)
      if ((cp >> k) & 1) {
        const uint32_t p = pos + (k == 3 ? 64u : 16u * k);
        place(m, (1u << wid) - 1u, wid, p >= 160 ? p - 160 : p);
      }
  }
  // ball
  const bool bl = (w0 & kW0Vdelbl) ? (w1 & kW1EnablOld) != 0 : (w1 & kW1Enabl) != 0;
  if (bl && (objs & kObBL)) {
    const uint32_t wid = 1u << ((ctrl >> 4) & 3);
    place(L.bl, (1u << wid) - 1u, wid, (w3 >> 24) & 0xFF);
  }
}

// Colour owner of column x from the objects there (0 COLUP0, 1 COLUPF,
// 2 COLUBK, 3 COLUP1).
__device__ __forceinline__ uint32_t owner_of(uint32_t ctrl, uint32_t x, bool p0, bool m0, bool p1, bool m1, bool pf,
                                             bool bl) {
  if (ctrl & 4) {
    if (pf || bl) return 1u;
    if (p0 || m0) return 0u;
    if (p1 || m1) return 3u;
    return 2u;
  }
  if (p0 || m0) return 0u;
  if (p1 || m1) return 3u;
  if (pf) return (ctrl & 2) ? (x < 80 ? 0u : 3u) : 1u;
  if (bl) return 1u;
  return 2u;
}
__device__ __forceinline__ uint32_t bit_at(const uint32_t* m, uint32_t x) { return (m[x >> 5] >> (x & 31)) & 1u; }
// The four columns of group g (4g .. 4g+3) of a mask, and a nibble spread to
// one byte of ones per set bit.
__device__ __forceinline__ uint32_t nib_at(const uint32_t* m, uint32_t g) { return (m[g >> 3] >> (4 * (g & 7))) & 0xFu; }
__device__ __forceinline__ uint32_t bytes_of(uint32_t n) {
  return ((n & 1) | ((n & 2) << 7) | ((n & 4) << 14) | ((n & 8) << 21)) * 0xFFu;
}

// Owner nibbles of group g (bit j = column 4g + j) from the object masks:
// COLUP0, COLUP1, the playfield colour (COLUPF, or COLUP0 / COLUP1 by half
// in score mode), the ball's COLUPF, COLUBK (see owner_of).
struct GroupOwners {
  uint32_t o0, o3, opf, obl, obk;
};
__device__ __forceinline__ GroupOwners group_owners(const LineMasks& L, uint32_t ctrl, uint32_t g) {
  const uint32_t P = nib_at(L.p0, g) | nib_at(L.m0, g), Q = nib_at(L.p1, g) | nib_at(L.m1, g);
  const uint32_t F = nib_at(L.pf, g), B = nib_at(L.bl, g);
  GroupOwners o;
  if (ctrl & 4) {
    o.opf = F;
    o.obl = B & ~F;
    o.o0 = P & ~(F | B);
    o.o3 = Q & ~(F | B | P);
  } else {
    o.o0 = P;
    o.o3 = Q & ~P;
    o.opf = F & ~(P | Q);
    o.obl = B & ~(P | Q | F);
  }
  o.obk = 0xFu & ~(o.o0 | o.o3 | o.opf | o.obl);
  return o;
}

// The objects in the pairs of a set of latch bits.
__host__ __device__ constexpr uint32_t pair_objects(uint32_t pairs) {
  return ((pairs & 0x8039u) ? kObP0 : 0u) | ((pairs & 0x80C6u) ? kObP1 : 0u) | ((pairs & 0x4303u) ? kObM0 : 0u) |
         ((pairs & 0x4C0Cu) ? kObM1 : 0u) | ((pairs & 0x2550u) ? kObBL : 0u) | ((pairs & 0x2AA0u) ? kObPF : 0u);
}

// Collision latch bits of the pairs in `want` that overlap on columns
// [x0, x1) of one scanline, from its column masks.
__device__ __forceinline__ uint32_t collide_span(const LineMasks& L, uint32_t want, uint32_t x0, uint32_t x1) {
  uint32_t got = 0;
  for (uint32_t k = 0; k < 5; k++) {
    const uint32_t c0 = 32 * k;
    if (c0 >= x1 || c0 + 32 <= x0) continue;
    uint32_t span = 0xFFFFFFFFu;
    if (x0 > c0) span &= 0xFFFFFFFFu << (x0 - c0);
    if (x1 < c0 + 32) span &= 0xFFFFFFFFu >> (c0 + 32 - x1);
    const uint32_t p0 = L.p0[k] & span, p1 = L.p1[k] & span, m0 = L.m0[k] & span, m1 = L.m1[k] & span;
    const uint32_t bl = L.bl[k] & span, pf = L.pf[k] & span;
    got |= ((m0 & p0) ? 1u << 0 : 0u) | ((m0 & p1) ? 1u << 1 : 0u) | ((m1 & p1) ? 1u << 2 : 0u) |
           ((m1 & p0) ? 1u << 3 : 0u) | ((p0 & bl) ? 1u << 4 : 0u) | ((p0 & pf) ? 1u << 5 : 0u) |
           ((p1 & bl) ? 1u << 6 : 0u) | ((p1 & pf) ? 1u << 7 : 0u) | ((m0 & bl) ? 1u << 8 : 0u) |
           ((m0 & pf) ? 1u << 9 : 0u) | ((m1 & bl) ? 1u << 10 : 0u) | ((m1 & pf) ? 1u << 11 : 0u) |
           ((bl & pf) ? 1u << 13 : 0u) | ((m0 & m1) ? 1u << 14 : 0u) | ((p0 & p1) ? 1u << 15 : 0u);
  }
  return got & want;
}

// Player 0 against the playfield alone (no other object can draw, player
// 0 plain: one copy, no scale, reflection or delay) on columns [x0, x1).
__device__ __forceinline__ bool p0_pf_overlap(const TiaView& v, uint32_t x0, uint32_t x1) {
  const uint32_t g = v.p0 & 0xFF, pos = (v.p0 >> 8) & 0xFF;
  if (!g) return false;
  const uint32_t ctrl = v.pf >> 24, pf0 = v.pf & 0xFF, pf1 = (v.pf >> 8) & 0xFF, pf2 = (v.pf >> 16) & 0xFF;
  const uint32_t p20 = ((pf0 >> 4) & 0xF) | ((__brev(pf1) >> 24) << 4) | (pf2 << 12);
  const uint32_t right = (ctrl & 1) ? (__brev(p20) >> 12) : p20;
  const uint64_t g40 = (uint64_t)p20 | ((uint64_t)right << 20);
  const uint32_t cols = __brev(g) >> 24;   // bit j = column pos + j
  for (uint32_t j = 0; j < 8; j++) {
    uint32_t x = pos + j;
    x -= x >= 160 ? 160u : 0u;
    if (((cols >> j) & 1) && x >= x0 && x < x1 && ((g40 >> (x >> 2)) & 1)) return true;
  }
  return false;
}

// Collision latches gained from the cursor cxc up to colour clock `target`
// (frame coordinates) by the pairs in `want`: line segment by line segment
// with the current registers (cold words at tx, stride E), stopping once
// every wanted pair has latched.  Out of line: it runs only while some
// possible pair has not latched yet.
static __device__ __noinline__ uint32_t cx_advance(const uint32_t* tx, uint32_t E, uint32_t xo, uint32_t want,
                                                   int32_t cxc, int32_t target) {
  TiaView v;
  v.col = 0;   // colours play no part in collisions
  v.pf = tx[4 * E];
  v.p0 = tx[5 * E];
  v.w0 = tx[0];
  v.w1 = tx[E];
  v.w3 = tx[3 * E];
  const bool simple = !(xo & kXoGen) && want == (1u << 5);   // player 0 against the playfield only
  // The registers are constant over the catch-up: one set of masks, of the
  // objects in the wanted pairs only, built at the first visible column (a
  // catch-up inside the horizontal blank, as between the writes that follow
  // a WSYNC, builds none); once a whole line has been seen the lines after
  // it, being the same, latch nothing new.
  LineMasks L;
  bool built = false;
  uint32_t got = 0;
  int32_t cur = cxc;
  while (cur < target && (want & ~got)) {
    const int32_t line = (int32_t)div228((uint32_t)cur), lbeg = 228 * line;
    const int32_t seg = target < lbeg + 228 ? target : lbeg + 228;
    const int32_t h0 = cur - lbeg, h1 = seg - lbeg;
    const uint32_t x0 = (uint32_t)(h0 > 68 ? h0 : 68) - 68u, x1 = (uint32_t)(h1 > 68 ? h1 : 68) - 68u;
    if (x1 > x0) {
      if (simple) {
        got |= p0_pf_overlap(v, x0, x1) ? want : 0u;
      } else {
        if (!built) {
          line_masks(v, L, pair_objects(want));
          built = true;
        }
        got |= collide_span(L, want & ~got, x0, x1);
      }
      if (x0 == 0 && x1 == 160) break;
    }
    cur = seg;
  }
  return got;
}

// Evaluate collisions up to colour clock `target`, if any possible pair has
// not latched; the cursor moves to `target` either way.
__device__ __forceinline__ void cx_catchup(const Ctx& c, Regs& r, int32_t target) {
  const uint32_t want = (r.cx >> 16) & ~r.cx & 0xFFFFu;
  if (want && target > r.cxc) r.cx |= cx_advance(c.tx, c.E, r.xo, want, r.cxc, target);
  r.cxc = target;
}

// Refresh the copy of the hot object registers in the cold words (w4, w5).
__device__ __forceinline__ void mirror_hot(const Ctx& c, const Regs& r) {
  tx_wr(c, 4, (r.pf0 & 0xFF) | ((r.pf1 & 0xFF) << 8) | ((r.pf2 & 0xFF) << 16) | ((r.ctrl & 0xFF) << 24));
  tx_wr(c, 5, (r.grp0 & 0xFF) | ((r.pos & 0xFF) << 8));
}

// A collision read register r (0..7) at colour clock t: D7 and D6.
__device__ __forceinline__ uint32_t cx_read(const Ctx& c, Regs& r, uint32_t reg, int32_t t) {
  cx_catchup(c, r, t);
  return ((r.cx >> (2 * (reg & 7))) & 3u) << 6;
}

// Out-of-line general drawing of pixels [x0, x1) of one scanline into this
// replica's chunks of the line buffer (blank_g leading groups blacked by an
// early HMOVE).
static __device__ __noinline__ void draw_general(const TiaView v, uint32_t* line, uint32_t E, uint32_t rank, uint32_t T,
                                                 uint32_t x0, uint32_t x1, uint32_t blank_g) {
  LineMasks L;
  line_masks(v, L);
  const uint32_t ctrl = v.pf >> 24;
  const bool score = (ctrl & 6) == 2;
  auto rep4 = [](uint32_t c) { return (c & 0xFE) * 0x01010101u; };
  const uint32_t c0 = rep4(v.col), cpf = rep4(v.col >> 8), cbk = rep4(v.col >> 16), c3 = rep4(v.col >> 24);
  for (uint32_t g = x0 >> 2; 4 * g < x1; g++) {
    if (((g >> 2) & (T - 1)) != rank) continue;
    uint32_t word = 0;
    if (g >= blank_g) {
      const GroupOwners o = group_owners(L, ctrl, g);
      const uint32_t cpfg = score ? (g < 20 ? c0 : c3) : cpf;
      word = (bytes_of(o.o0) & c0) | (bytes_of(o.o3) & c3) | (bytes_of(o.opf) & cpfg) | (bytes_of(o.obl) & cpf) |
             (bytes_of(o.obk) & cbk);
    }
    // the span's edge groups keep their bytes outside [x0, x1)
    uint32_t mask = 0xFFFFFFFFu;
    if (4 * g < x0) mask &= 0xFFFFFFFFu << (8 * (x0 - 4 * g));
    if (4 * g + 4 > x1) mask &= 0xFFFFFFFFu >> (8 * (4 * g + 4 - x1));
    line[g * E] = mask == 0xFFFFFFFFu ? word : ((line[g * E] & ~mask) | (word & mask));
  }
}

// Graphics-bit quantities (graphics-bit surrogate): GRP0, PF0, PF1, PF2,
// and with the whole TIA GRP1, ENAM0, ENAM1, ENABL and the delayed copies
// of GRP0, GRP1 and ENABL (a GRP1 write copies GRP0 and ENABL into theirs,
// a GRP0 write copies GRP1).
enum : int { kGbGrp0 = 0, kGbPf0 = 1, kGbGrp1 = 4, kGbEnam0 = 5, kGbEnam1 = 6, kGbEnabl = 7, kGbGrp0Old = 8,
             kGbGrp1Old = 9, kGbEnablOld = 10, kGbN = 11 };

// Pixel-gradient sums of pixels [x0, x1) by owning colour register (COLUP0,
// COLUPF, COLUBK, COLUP1) and, with the position sampler, player 0's
// position sum: (C_with - C_without) (b(x - 1) - b(x + 1)) / 2 per pixel.
struct OwnerSums {
  float s0, s1, s2, s3, pos;
};
static __device__ __noinline__ OwnerSums sums_general(const TiaView v, const float4* grow, uint32_t E, uint32_t slot,
                                                      uint32_t rank,
                                                      uint32_t T, uint32_t x0, uint32_t x1, uint32_t blank_g,
                                                      bool sampler) {
  LineMasks L;
  line_masks(v, L);
  const uint32_t ctrl = v.pf >> 24;
  const bool score = (ctrl & 6) == 2;
  OwnerSums s{0.f, 0.f, 0.f, 0.f, 0.f};
  for (uint32_t g = x0 >> 2; 4 * g < x1; g++) {
    if (((g >> 2) & (T - 1)) != rank || g < blank_g) continue;
    const float4 q = grow[grow_at(g, E, slot)];
    uint32_t in = 0xF;   // the group's columns inside [x0, x1)
    if (4 * g < x0) in &= 0xFu << (x0 - 4 * g);
    if (4 * g + 4 > x1) in &= 0xFu >> (4 * g + 4 - x1);
    const float gv[4] = {q.x, q.y, q.z, q.w};
    auto sum = [&](uint32_t n) {
      n &= in;
      return ((n & 1) ? gv[0] : 0.f) + ((n & 2) ? gv[1] : 0.f) + ((n & 4) ? gv[2] : 0.f) + ((n & 8) ? gv[3] : 0.f);
    };
    const GroupOwners o = group_owners(L, ctrl, g);
    const float tpf = sum(o.opf);
    s.s0 += sum(o.o0) + (score && g < 20 ? tpf : 0.f);
    s.s3 += sum(o.o3) + (score && g >= 20 ? tpf : 0.f);
    s.s1 += (score ? 0.f : tpf) + sum(o.obl);
    s.s2 += sum(o.obk);
    if (sampler && (nib_at(L.p0, g) | nib_at(L.p0, g == 0 ? 39u : g - 1) | nib_at(L.p0, g == 39 ? 0u : g + 1))) {
      for (uint32_t j = 0; j < 4; j++) {
        const uint32_t x = 4 * g + j;
        if (!((in >> j) & 1)) continue;
        const int32_t db = (int32_t)bit_at(L.p0, x == 0 ? 159u : x - 1) - (int32_t)bit_at(L.p0, x == 159 ? 0u : x + 1);
        if (!db) continue;
        const bool m0 = bit_at(L.m0, x), p1 = bit_at(L.p1, x), m1 = bit_at(L.m1, x), pf = bit_at(L.pf, x);
        const bool bl = bit_at(L.bl, x);
        const uint32_t ow = owner_of(ctrl, x, true, m0, p1, m1, pf, bl), on = owner_of(ctrl, x, false, m0, p1, m1, pf, bl);
        const int32_t cw = (int32_t)((v.col >> (8 * ow)) & 0xFE), cn = (int32_t)((v.col >> (8 * on)) & 0xFE);
        s.pos += (0.5f * (float)(db * (cw - cn))) * gv[j];
      }
    }
  }
  return s;
}

// Graphics-bit surrogate over pixels [x0, x1) of the whole TIA: for each
// drawn pixel and each object whose graphics bit decides its coverage there
// (a player's GRP bit over its copies' spans, a missile's ENAM byte over
// its span unless it is locked to its player, the ball's ENABL byte over
// its span, the playfield register of the column), the pixel's gradient
// times the colour with that bit set minus the colour with it clear (the
// priority logic decides both, the other objects as drawn), summed per
// quantity (kGb*; a delayed graphic's sum goes to its delayed copy).
struct GbSums {
  float v[kGbN];
};
static __device__ __noinline__ GbSums gbits_general(const TiaView v, const float4* grow, uint32_t E, uint32_t slot,
                                                    uint32_t rank, uint32_t T, uint32_t x0, uint32_t x1,
                                                    uint32_t blank_g) {
  LineMasks L;
  line_masks(v, L);
  const uint32_t ctrl = v.pf >> 24, w0 = v.w0, w3 = v.w3;
  // the objects' spans: where their graphics bits are in play
  uint32_t S[5][5];   // P0, M0, P1, M1, BL
  for (int k = 0; k < 5; k++)
    for (int q = 0; q < 5; q++) S[k][q] = 0;
  for (uint32_t i = 0; i < 2; i++) {
    const uint32_t mode = i ? (w0 >> 16) & 7 : (w0 >> 8) & 7;
    const uint32_t sc = player_scale(mode), cp = nusiz_copies(mode);
    const uint32_t pos = i ? w3 & 0xFF : (v.p0 >> 8) & 0xFF;
    const uint32_t pat = sc == 4 ? 0xFFFFFFFFu : (1u << (8 * sc)) - 1u;
    for (uint32_t k = 0; k < 4; k++)
      if ((cp >> k) & 1) {
        const uint32_t p = pos + (k == 3 ? 64u : 16u * k);
        place(S[i ? 2 : 0], pat, 8 * sc, p >= 160 ? p - 160 : p);
      }
    if (!(w0 & (i ? kW0Resmp1 : kW0Resmp0))) {
      const uint32_t nus = i ? (w0 >> 16) & 0xFF : (w0 >> 8) & 0xFF;
      const uint32_t wid = 1u << ((nus >> 4) & 3), mcp = nusiz_copies(nus & 7);
      const uint32_t mpos = (w3 >> (i ? 16 : 8)) & 0xFF;
      for (uint32_t k = 0; k < 4; k++)
        if ((mcp >> k) & 1) {
          const uint32_t p = mpos + (k == 3 ? 64u : 16u * k);
          place(S[i ? 3 : 1], (1u << wid) - 1u, wid, p >= 160 ? p - 160 : p);
        }
    }
  }
  {
    const uint32_t wid = 1u << ((ctrl >> 4) & 3);
    place(S[4], (1u << wid) - 1u, wid, (w3 >> 24) & 0xFF);
  }
  const int dst[6] = {(w0 & kW0Vdelp0) ? kGbGrp0Old : kGbGrp0, kGbEnam0, (w0 & kW0Vdelp1) ? kGbGrp1Old : kGbGrp1,
                      kGbEnam1, kGbPf0, (w0 & kW0Vdelbl) ? kGbEnablOld : kGbEnabl};
  GbSums out;
  for (int k = 0; k < kGbN; k++) out.v[k] = 0.f;
  for (uint32_t g = x0 >> 2; 4 * g < x1; g++) {
    if (((g >> 2) & (T - 1)) != rank || g < blank_g) continue;
    const float4 q = grow[grow_at(g, E, slot)];
    const float gv[4] = {q.x, q.y, q.z, q.w};
    for (uint32_t j = 0; j < 4; j++) {
      const uint32_t x = 4 * g + j;
      if (x < x0 || x >= x1 || gv[j] == 0.f) continue;
      bool b[6] = {bit_at(L.p0, x) != 0, bit_at(L.m0, x) != 0, bit_at(L.p1, x) != 0, bit_at(L.m1, x) != 0,
                   bit_at(L.pf, x) != 0, bit_at(L.bl, x) != 0};
      const bool in[6] = {bit_at(S[0], x) != 0, bit_at(S[1], x) != 0, bit_at(S[2], x) != 0, bit_at(S[3], x) != 0,
                          true, bit_at(S[4], x) != 0};
      // the playfield register of the column (right half mirrored with CTRLPF bit 0)
      uint32_t i = x < 80 ? x >> 2 : (x - 80) >> 2;
      if (x >= 80 && (ctrl & 1)) i = 19 - i;
      const int pfk = kGbPf0 + (i < 4 ? 0 : (i < 12 ? 1 : 2));
      for (int k = 0; k < 6; k++) {
        if (!in[k]) continue;
        const bool keep = b[k];
        b[k] = true;
        const uint32_t ow = owner_of(ctrl, x, b[0], b[1], b[2], b[3], b[4], b[5]);
        b[k] = false;
        const uint32_t on = owner_of(ctrl, x, b[0], b[1], b[2], b[3], b[4], b[5]);
        b[k] = keep;
        const int32_t d = (int32_t)((v.col >> (8 * ow)) & 0xFE) - (int32_t)((v.col >> (8 * on)) & 0xFE);
        if (d) out.v[k == 4 ? pfk : dst[k]] += (float)d * gv[j];
      }
    }
  }
  return out;
}

}  // namespace vcs
