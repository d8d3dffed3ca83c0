// SOFT-STE backward pass (Corollary 1) and the soft entry points of the C ABI.
//
// The forward pass of soft mode is the step kernel on rounded inputs (it
// equals the hard machine, Theorem 1) plus a state checkpoint at the start of
// every segment.  The backward pass runs in two kernels:
//   1. k_soft_recompute recomputes a group of segments at once, each from its
//      checkpoint, recording one 4-byte tape entry per instruction the sweep
//      acts on (opcode, reference address, flags; reverse_needed) and, on the
//      frames a step returns, the sum of the pixel gradients owned by each
//      colour-register version (the stored priority switch);
//   2. k_soft_sweep, segment by segment from the last, sweeps the tape
//      backwards (one env per warp), carrying adjoints of A, X, Y, the timer
//      value, the four colour registers and the 128 RAM cells (256 with a
//      Superchip's cartridge RAM; in shared memory), with the surrogate rules:
//        reads   relaxed read of Eq. s-read w.r.t. memory contents: RAM reads
//                spread the adjoint over |i - a| <= W with weights
//                exp(-|i - a| / tau) normalised in the clipped window; ROM
//                reads add an impulse at a, spread by the same weights later;
//                SWCHA / INPT4 reads give the joystick inputs -128, -64, -32,
//                -16 / -128; INTIM before underflow gives the timer value 1;
//        writes  the cell's adjoint moves to the written register;
//        ALU     ADC (1, 1), SBC (1, -1), AND/ORA/EOR (1, 1), shifts,
//                rotates, increments and transfers 1, compares nothing;
//        indices addresses, PC, SP and flags carry nothing;
//      and hands the adjoints at the segment start to the previous segment.
// A final pass spreads the ROM impulses with the read window and optionally
// sums the per-env ROM gradients per cartridge (a segmented reduction over
// the envs of each cart, no atomics).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <new>
#include <vector>

#include "vcs_api_internal.h"
#include "vcs_exec.cuh"
#include "vcs_kernels.cuh"
#include "vcs_run.cuh"

namespace vcs {

// carried adjoints: aA aX aY aV aC0 aC1 aC2, aRAM[128] and its compensation,
// those of player 0's position and of HMP0 (position sampler), the Superchip
// RAM's adjoints [128] and their compensation, COLUP1's, then those of
// the graphics-bit surrogate's quantities (GRP0, PF0-2, GRP1, ENAM0,
// ENAM1, ENABL and the three delayed copies)
constexpr int kCarryPos = 7 + 256;
constexpr int kCarryCram = kCarryPos + 2;
constexpr int kCarryC3 = kCarryCram + 256;
constexpr int kCarryGB = kCarryC3 + 1;   // the graphics-bit surrogate's eleven quantities
constexpr int kCarry = kCarryGB + 11;
constexpr int kMaxW = 120;        // window half-width limit (tau <= 10)

// Compensated (Neumaier) sum: s + c carries the running total.
__device__ __forceinline__ void comp_add(float& s, float& c, float x) {
  const float t = s + x;
  c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
  s = t;
}


// SAMPLER: the position sampler is on (its pixel sums are compiled out of
// the other instantiation, which then carries zero position adjoints).
// GB: the graphics-bit surrogate is on: its quantities are versioned too,
// their pixel sums the renderer's with-minus-without colours; FT: the whole
// TIA (the surrogate's eleven quantities, else its first four).
template <bool SAMPLER, bool GB, bool FT = false>
struct RecTape {
  static constexpr bool kAcc = true;
  static constexpr bool sampler = SAMPLER;
  static constexpr bool graphics = GB;
  static constexpr int kNG = GB ? (FT ? kGbN : 4) : 0;   // graphics-bit quantities
  uint32_t* buf;
  float* cw;
  uint32_t n, cap, ncw, capcw;
  // versions 0..2: the colour registers COLUP0, COLUPF, COLUBK; version 3:
  // player 0's position (its pixel sums are the sampler's, zero when off);
  // version 4: COLUP1
  int32_t slot0, slot1, slot2, slot3, slot4;  // float slot of each live version
  float s0, s1, s2, s3, s4, c0, c1, c2, c3, c4;  // compensated pixel-gradient sums of the live versions
  float p0, p1, p2, p3, p4;        // sums of the versions alive at the segment start
  // the graphics-bit quantities' live versions (slot, compensated sum, sum of
  // the version alive at the segment start); indices are compile-time
  int32_t gsl[kGbN];
  float gs[kGbN], gc[kGbN], gp[kGbN];
  bool overflow;
  uint32_t T, gmask;               // replicas of this env and their warp lanes
  // The replicas of an env each sum the pixel chunks they own; a version's
  // total is their sum (a butterfly over the replicas' lanes, so every
  // replica holds the same total).
  __device__ __forceinline__ float replica_sum(float v) const {
    for (uint32_t o = 1; o < T; o <<= 1) v += __shfl_xor_sync(gmask, v, o);
    return v;
  }
  __device__ __forceinline__ void rec(uint32_t op, uint32_t ref, uint32_t fl) {
    if (n < cap) __stcs(buf + n, op | ((ref & 0xFFFF) << 8) | (fl << 24));   // written once, read once: evict first
    else overflow = true;
    n++;
  }
  __device__ __forceinline__ void close_version(int32_t slot, float s, float& pinit) {
    const float tot = replica_sum(s);
    if (slot >= 0) cw[slot] = tot;
    else if (slot == -1) pinit += tot;
  }
  __device__ __forceinline__ int32_t fresh_slot() {
    int32_t fresh = ncw < capcw ? (int32_t)ncw : -2;
    if (fresh == -2) overflow = true;
    ncw++;
    return fresh;
  }
  __device__ __forceinline__ void colour_write(int r) {
    const int32_t fresh = fresh_slot();
    if (r == 0) { close_version(slot0, s0 + c0, p0); s0 = c0 = 0.f; slot0 = fresh; }
    else if (r == 1) { close_version(slot1, s1 + c1, p1); s1 = c1 = 0.f; slot1 = fresh; }
    else if (r == 2) { close_version(slot2, s2 + c2, p2); s2 = c2 = 0.f; slot2 = fresh; }
    else if (r == 3) { close_version(slot3, s3 + c3, p3); s3 = c3 = 0.f; slot3 = fresh; }
    else { close_version(slot4, s4 + c4, p4); s4 = c4 = 0.f; slot4 = fresh; }
  }
  template <int K>
  __device__ __forceinline__ void graphics_write() {
    const int32_t fresh = fresh_slot();
    close_version(gsl[K], gs[K] + gc[K], gp[K]);
    gs[K] = gc[K] = 0.f;
    gsl[K] = fresh;
  }
  __device__ __forceinline__ void version_write(uint32_t reg) {
    if (reg == 0x06) colour_write(0);
    else if (reg == 0x08) colour_write(1);
    else if (reg == 0x09) colour_write(2);
    else if (reg == 0x10 || reg == 0x2A) colour_write(3);
    else if (reg == 0x07) colour_write(4);
    if constexpr (GB) {
      if (reg == 0x1B) {                      // GRP0 (with the whole TIA: GRP1's delayed copy too)
        graphics_write<kGbGrp0>();
        if constexpr (FT) graphics_write<kGbGrp1Old>();
      } else if (reg == 0x0D) graphics_write<kGbPf0>();
      else if (reg == 0x0E) graphics_write<kGbPf0 + 1>();
      else if (reg == 0x0F) graphics_write<kGbPf0 + 2>();
      if constexpr (FT) {
        if (reg == 0x1C) {                    // GRP1, GRP0's and ENABL's delayed copies
          graphics_write<kGbGrp1>();
          graphics_write<kGbGrp0Old>();
          graphics_write<kGbEnablOld>();
        } else if (reg == 0x1D) graphics_write<kGbEnam0>();
        else if (reg == 0x1E) graphics_write<kGbEnam1>();
        else if (reg == 0x1F) graphics_write<kGbEnabl>();
      }
    }
  }
  // pixel-gradient sums of one drawn span, per owner (COLUP0, COLUPF,
  // COLUBK, COLUP1), and the sampler's sum
  __device__ __forceinline__ void pixels(float v0, float v1, float v2, float v3, float v4) {
    comp_add(s0, c0, v0);
    comp_add(s1, c1, v1);
    comp_add(s2, c2, v2);
    if constexpr (SAMPLER) comp_add(s3, c3, v3);
    if (v4 != 0.f) comp_add(s4, c4, v4);
  }
  // graphics-bit sums of one drawn span: GRP0, PF0, PF1, PF2
  __device__ __forceinline__ void gbits(float g, float f0, float f1, float f2) {
    comp_add(gs[kGbGrp0], gc[kGbGrp0], g);
    comp_add(gs[kGbPf0], gc[kGbPf0], f0);
    comp_add(gs[kGbPf0 + 1], gc[kGbPf0 + 1], f1);
    comp_add(gs[kGbPf0 + 2], gc[kGbPf0 + 2], f2);
  }
  // the whole TIA's graphics-bit sums of one drawn span, all eleven
  __device__ __forceinline__ void gbits_all(const float (&v)[kGbN]) {
#pragma unroll
    for (int k = 0; k < kNG; k++) comp_add(gs[k], gc[k], v[k]);
  }
  __device__ __forceinline__ void finish() {
    close_version(slot0, s0 + c0, p0);
    close_version(slot1, s1 + c1, p1);
    close_version(slot2, s2 + c2, p2);
    close_version(slot3, s3 + c3, p3);
    close_version(slot4, s4 + c4, p4);
    s0 = s1 = s2 = s3 = s4 = c0 = c1 = c2 = c3 = c4 = 0.f;
#pragma unroll
    for (int k = 0; k < kNG; k++) {
      close_version(gsl[k], gs[k] + gc[k], gp[k]);
      gs[k] = gc[k] = 0.f;
    }
  }
};

struct BwdParams {
  int32_t n_envs, n_steps, frame_skip, seg, seg_steps, ystart, first;
  int32_t seg0;               // first segment of the group whose tapes are held (slot = seg - seg0)
  int32_t tpe;                // threads per env
  const int4* blocks;
  const int32_t* perm;
  const uint8_t* roms;        // rounded ROM images of the rollout [n_carts][rom_stride]
  const uint8_t* cart_banks;  // bank byte per cart (banks | kCartSC | kCartE0)
  int32_t ram_words;          // RAM words per env in the recompute's shared memory (32 or 64)
  int32_t xmap;               // the batch holds Superchip or E0 carts (their kernels' instantiation)
  int32_t full_tia;           // the whole TIA (its kernels' instantiation)
  uint32_t rom_stride;
  const uint8_t* cart_2k;
  const int32_t* env_cart;    // [n_envs]
  const DecodeTables* dt;
  const uint32_t* ckpt;       // every segment's checkpoint [n_seg][kStateWords][n_envs]
  const uint8_t* act_bits;    // [n_steps][n_envs]
  const float* grad_ram;      // [n_steps][n_envs][128] or null
  const float* grad_screen;   // [n_steps][n_envs][210][160] or null
  const float* w_ram;         // [128] weights on every step, or null
  const float* w_screen;      // [210][160] weights on every step, or null
  uint32_t* rec;              // [G][n_envs][cap_rec]
  uint32_t cap_rec;
  float* cw;                  // [G][n_envs][cap_cw]
  uint32_t cap_cw;
  uint32_t* step_end;         // [G][seg_steps][n_envs]
  float* meta;                // [G][n_envs][kMeta]
  float* carry;               // [kCarry][n_envs]
  float* imp;                 // ROM impulses [n_envs][rom_stride] x (value, compensation) pairs
  float* grad_u;              // [n_steps][n_envs][5] or null
  float* grad_ram0;           // [n_envs][128] or null (segment 0)
  float* grad_cart_ram0;      // [n_envs][128] or null (segment 0): the Superchip's RAM
  float tau;
  int32_t W;
  uint32_t sched_policy, sched_window;
  int32_t sampler;            // the position sampler is on
  int32_t graphics;           // the graphics-bit surrogate is on
  int32_t step_instr;         // > 0: instruction-granular steps of this many slots
  int32_t sweep_lanes;        // the reverse sweep walks one env per lane (k_soft_sweep_lanes)
  int32_t* err;
};

// A compensated adjoint (Neumaier): s + c is its value.  Over a long
// rollout an adjoint can pass thousands of times between a RAM cell and a
// register (a byte loaded, updated and stored back every frame); one
// float32 rounding per hop would then add up to more than the gradient
// tolerance, so the registers hold such pairs and a write hands its cell's
// pair to the register whole.
struct Acc {
  float s, c;
  __device__ __forceinline__ float v() const { return s + c; }
  __device__ __forceinline__ void operator+=(float x) { comp_add(s, c, x); }
  __device__ __forceinline__ void operator+=(const Acc& o) {
    s += o.s;
    c += o.c;
  }
  __device__ __forceinline__ Acc take() {
    const Acc r = *this;
    s = c = 0.f;
    return r;
  }
  __device__ __forceinline__ void clear() { s = c = 0.f; }
  __device__ __forceinline__ bool zero() const { return s == 0.f && c == 0.f; }
};
__device__ __forceinline__ Acc acc(float x) { return Acc{x, 0.f}; }
__device__ __forceinline__ Acc operator-(const Acc& x) { return Acc{-x.s, -x.c}; }

struct Adj {
  Acc A, X, Y, V, C0, C1, C2, C3;   // C3: COLUP1
  Acc G[kGbN];         // the graphics-bit surrogate's quantities (kGb*)
  bool ft;             // the whole TIA (its graphics-bit quantities are versioned)
  float P, H;          // player 0's position and HMP0 (position sampler)
  float u[5], uc[5];   // joystick-input adjoints of the current step (compensated)
};

// ROM impulses waiting to be added to the env's impulse row: the sweep's
// lane queues (index, adjoint) pairs and the warp adds them in order after
// each block of records (shared memory, one queue per env).
struct RomQueue {
  uint32_t* idx;
  float* g;
  uint32_t n;
  __device__ __forceinline__ void push(uint32_t i, float v) {
    idx[n] = i;
    g[n] = v;
    n++;
  }
};
// The same queue for a sweep that walks one env per lane (kLaneEnvs envs a
// block): lane l's entry e sits at e * kLaneEnvs + l (consecutive lanes in
// consecutive banks), and the lane adds its own impulses.
constexpr int kLaneEnvs = 8;
struct LaneQueue {
  uint32_t* idx;
  float* g;
  uint32_t n;
  __device__ __forceinline__ void push(uint32_t i, float v) {
    idx[n * kLaneEnvs] = i;
    g[n * kLaneEnvs] = v;
    n++;
  }
};

// Cart kind bits of the sweep: the 2K image (ROM index within 2 KB), the
// Superchip's RAM ports and E0's 1 KB slices (a record's bank field is then
// the slice its reference's segment showed).
enum : uint32_t { kKind2K = 1, kKindSC = 2, kKindE0 = 4 };

// Relaxed read of cell i of a 128-cell RAM tensor whose adjoints start at
// cell `base` (0: RIOT RAM, 128: the Superchip's RAM).  The read cell's own
// weight, 1 / z_i, is close to 1 at small temperatures, and an adjoint that
// passes through the same read every frame is multiplied by it thousands of
// times: a float32 rounding of the weight would then compound into a bias
// (2,048 frames x up to 3e-8 per factor).  So the read cell takes
// g - g (z_i - 1) / z_i, the small complement being accurate to float32's
// relative precision (izr[128 + i]); its neighbours take
// g e^{-|j - i| / tau} / z_i.
__device__ __forceinline__ void spread_ram(float* aram, float* aramc, uint32_t E, const float* ek, const float* izr,
                                           int W, int base, int i, const Acc& g) {
  const int lo = i - W < 0 ? 0 : i - W, hi = i + W > 127 ? 127 : i + W;
  const float gv = g.v(), gz = gv * izr[i];
  for (int j = lo; j <= hi; j++) {
    float* cs = aram + (base + j) * E;
    float* cc = aramc + (base + j) * E;
    float s = *cs, c = *cc;
    if (j == i) {   // the read cell: the pair whole, less its neighbours' share
      comp_add(s, c, g.s);
      c += g.c;
      comp_add(s, c, -__fmul_rn(gv, izr[128 + i]));
    } else {
      comp_add(s, c, __fmul_rn(gz, ek[j > i ? j - i : i - j]));
    }
    *cs = s;
    *cc = c;
  }
}

// Adjoint of a value read from `ref` (13-bit bus address) flows back to the
// memory it came from.  RAM cells, ROM impulses and joystick adjoints are
// compensated sums (value + compensation), since long rollouts add many
// terms of both signs into them.
// XM: the sweep's batch may hold Superchip or E0 carts (their ports and
// slices are compiled out otherwise).
template <bool XM, class Q>
__device__ __forceinline__ void scatter_read(Adj& a, float* aram, float* aramc, uint32_t E, const float* ek,
                                             const float* izr, int W, Q& rq,
                                             uint32_t kind, uint32_t ref, uint32_t fl, const Acc& ga) {
  const uint32_t ad = ref & 0x1FFF;
  if (ga.zero()) return;
  const float g = ga.v();   // ROM impulses and joystick sums are compensated where they accumulate
  if (XM && (kind & kKindSC) && (ad & 0x1F80) == 0x1080) {   // the Superchip's read port
    spread_ram(aram, aramc, E, ek, izr, W, 128, (int)(ad & 0x7F), ga);
  } else if (ad & 0x1000) {
    const uint32_t unit = (fl >> 2) & 7u;   // the read's bank (E0: slice)
    rq.push((kind & kKind2K) ? (ad & 0x7FF)
            : (XM && (kind & kKindE0)) ? ((unit << 10) | (ad & 0x3FF)) : ((unit << 12) | (ad & 0xFFF)), g);
  } else if (!(ad & 0x80)) {
    if ((ad & 0xF) == 0xC) comp_add(a.u[4], a.uc[4], -128.f * g);
  } else if (!(ad & 0x200)) {
    spread_ram(aram, aramc, E, ek, izr, W, 0, (int)(ad & 0x7F), ga);
  } else if (!(ad & 4)) {
    if ((ad & 3) == 0) {
      comp_add(a.u[0], a.uc[0], -128.f * g);
      comp_add(a.u[1], a.uc[1], -64.f * g);
      comp_add(a.u[2], a.uc[2], -32.f * g);
      comp_add(a.u[3], a.uc[3], -16.f * g);
    }
  } else if (!(ad & 1) && (fl & 2)) {
    a.V += ga;
  }
}

// The colour / position version sums of an env's tape, popped last to
// first (j counts the sums not yet popped): straight from the tape, or
// (CwAhead, the lane sweep) with the next sum loaded ahead, so that a pop
// waits for no load.
__device__ __forceinline__ float cw_pop(const float* cw, uint32_t& j) { return cw[--j]; }
struct CwAhead {
  const float* p;
  float next;   // p[j - 1] (0 once j is 0)
};
__device__ __forceinline__ float cw_pop(CwAhead& cw, uint32_t& j) {
  const float v = cw.next;
  --j;
  cw.next = j ? cw.p[j - 1] : 0.f;
  return v;
}

// Adjoint of the value written to `ref`: taken from the cell (which is then
// cleared, the write being one-hot).
template <bool SAMPLER, bool GB, bool XM, class CW>
__device__ __forceinline__ Acc take_write(Adj& a, float* aram, float* aramc, uint32_t E, CW& cw,
                                          uint32_t& j, uint32_t kind, uint32_t ref) {
  const uint32_t ad = ref & 0x1FFF;
  if (ad & 0x1000) {
    if (!XM || !(kind & kKindSC) || (ad & 0x1F80) != 0x1000) return acc(0.f);
    const uint32_t o = (128 + (ad & 0x7F)) * E;   // the Superchip's write port
    const Acc g{aram[o], aramc[o]};
    aram[o] = 0.f;
    aramc[o] = 0.f;
    return g;
  }
  if (!(ad & 0x80)) {
    const uint32_t reg = ad & 0x3F;
    if (reg == 0x06) { if (j) a.C0 += cw_pop(cw, j); return a.C0.take(); }
    if (reg == 0x08) { if (j) a.C1 += cw_pop(cw, j); return a.C1.take(); }
    if (reg == 0x09) { if (j) a.C2 += cw_pop(cw, j); return a.C2.take(); }
    if (reg == 0x07) { if (j) a.C3 += cw_pop(cw, j); return a.C3.take(); }
    if constexpr (GB) {
      // graphics-bit surrogate: a version's sum goes to the written value.
      // A delayed copy's versions open at the other player's GRP write (the
      // later slots of its record, popped first) and belong to the value
      // the copy took: the source register's live version.
      auto pop = [&](int k) { if (j) a.G[k] += cw_pop(cw, j); };
      if (reg == 0x1B) {
        if (a.ft) {
          pop(kGbGrp1Old);
          a.G[kGbGrp1] += a.G[kGbGrp1Old].take();
        }
        pop(kGbGrp0);
        return a.G[kGbGrp0].take();
      }
      if (reg >= 0x0D && reg <= 0x0F) {
        const int k = kGbPf0 + (int)(reg - 0x0D);
        pop(k);
        return a.G[k].take();
      }
      if (a.ft) {
        if (reg == 0x1C) {
          pop(kGbEnablOld);
          a.G[kGbEnabl] += a.G[kGbEnablOld].take();
          pop(kGbGrp0Old);
          a.G[kGbGrp0] += a.G[kGbGrp0Old].take();
          pop(kGbGrp1);
          return a.G[kGbGrp1].take();
        }
        if (reg >= 0x1D && reg <= 0x1F) {
          const int k = kGbEnam0 + (int)(reg - 0x1D);
          pop(k);
          return a.G[k].take();
        }
      }
    }
    // RESP0 and HMOVE open a position version (its slot pops either way)
    if (reg == 0x2A || reg == 0x10) {
      const float sv = j ? cw_pop(cw, j) : 0.f;
      if constexpr (SAMPLER) {
        if (reg == 0x2A) {   // HMOVE: pos' = pos - HMP0 / 16 (the written value is ignored)
          a.P += sv;
          a.H -= 0.0625f * a.P;
        } else {             // RESP0: the new position is a constant
          a.P = 0.f;
        }
      }
      return acc(0.f);
    }
    if constexpr (SAMPLER) {
      if (reg == 0x20) {   // HMP0
        const float g = a.H;
        a.H = 0.f;
        return acc(g);
      }
      if (reg == 0x2B) { a.H = 0.f; return acc(0.f); }   // HMCLR
    }
    return acc(0.f);
  }
  if (!(ad & 0x200)) {
    const uint32_t o = (ad & 0x7F) * E;
    const Acc g{aram[o], aramc[o]};
    aram[o] = 0.f;
    aramc[o] = 0.f;
    return g;
  }
  if ((ad & 0x14) == 0x14) return a.V.take();
  return acc(0.f);
}

__device__ __forceinline__ uint32_t stack_addr(uint32_t ref, uint32_t k) { return 0x100u | ((ref - k) & 0xFF); }

template <bool SAMPLER, bool GB, bool XM, class Q, class CW>
__device__ __forceinline__ void reverse_one(Adj& a, float* aram, float* aramc, uint32_t E, const float* ek,
                                            const float* izr, int W, Q& rq,
                                            uint32_t kind, CW& cw, uint32_t& j, uint32_t rec) {
  const uint32_t op = rec & 0xFF, ref = (rec >> 8) & 0xFFFF, fl = rec >> 24;
  switch (op) {
    case 0xA9: case 0xA5: case 0xB5: case 0xAD: case 0xBD: case 0xB9: case 0xA1: case 0xB1: {
      const Acc g = a.A.take();
      scatter_read<XM>(a, aram, aramc, E, ek, izr, W, rq, kind, ref, fl, g);
      break;
    }
    case 0xA2: case 0xA6: case 0xB6: case 0xAE: case 0xBE: {
      const Acc g = a.X.take();
      scatter_read<XM>(a, aram, aramc, E, ek, izr, W, rq, kind, ref, fl, g);
      break;
    }
    case 0xA0: case 0xA4: case 0xB4: case 0xAC: case 0xBC: {
      const Acc g = a.Y.take();
      scatter_read<XM>(a, aram, aramc, E, ek, izr, W, rq, kind, ref, fl, g);
      break;
    }
    case 0x09: case 0x05: case 0x15: case 0x0D: case 0x1D: case 0x19: case 0x01: case 0x11:
    case 0x29: case 0x25: case 0x35: case 0x2D: case 0x3D: case 0x39: case 0x21: case 0x31:
    case 0x49: case 0x45: case 0x55: case 0x4D: case 0x5D: case 0x59: case 0x41: case 0x51:
    case 0x69: case 0x65: case 0x75: case 0x6D: case 0x7D: case 0x79: case 0x61: case 0x71:
      scatter_read<XM>(a, aram, aramc, E, ek, izr, W, rq, kind, ref, fl, a.A);
      break;
    case 0xE9: case 0xE5: case 0xF5: case 0xED: case 0xFD: case 0xF9: case 0xE1: case 0xF1:
    case 0xEB:                                                      // USBC: SBC's alias
      scatter_read<XM>(a, aram, aramc, E, ek, izr, W, rq, kind, ref, fl, -a.A);
      break;
    case 0xA7: case 0xB7: case 0xAF: case 0xBF: case 0xA3: case 0xB3: {   // LAX: A = X = M
      Acc g = a.A.take();
      g += a.X.take();
      scatter_read<XM>(a, aram, aramc, E, ek, izr, W, rq, kind, ref, fl, g);
      break;
    }
    case 0x87: case 0x97: case 0x8F: case 0x83: {                   // SAX: M = A & X, the (1, 1) rule
      const Acc g = take_write<SAMPLER, GB, XM>(a, aram, aramc, E, cw, j, kind, ref);
      a.A += g;
      a.X += g;
      break;
    }
    case 0x85: case 0x95: case 0x8D: case 0x9D: case 0x99: case 0x81: case 0x91:
      a.A += take_write<SAMPLER, GB, XM>(a, aram, aramc, E, cw, j, kind, ref);
      break;
    case 0x86: case 0x96: case 0x8E:
      a.X += take_write<SAMPLER, GB, XM>(a, aram, aramc, E, cw, j, kind, ref);
      break;
    case 0x84: case 0x94: case 0x8C:
      a.Y += take_write<SAMPLER, GB, XM>(a, aram, aramc, E, cw, j, kind, ref);
      break;
    case 0x06: case 0x16: case 0x0E: case 0x1E:
    case 0x26: case 0x36: case 0x2E: case 0x3E:
    case 0x46: case 0x56: case 0x4E: case 0x5E:
    case 0x66: case 0x76: case 0x6E: case 0x7E:
    case 0xC6: case 0xD6: case 0xCE: case 0xDE:
    case 0xE6: case 0xF6: case 0xEE: case 0xFE: {
      const Acc g = take_write<SAMPLER, GB, XM>(a, aram, aramc, E, cw, j, kind, ref);
      scatter_read<XM>(a, aram, aramc, E, ek, izr, W, rq, kind, ref, fl, g);
      break;
    }
    case 0xAA: a.A += a.X.take(); break;   // TAX
    case 0x8A: a.X += a.A.take(); break;   // TXA
    case 0xA8: a.A += a.Y.take(); break;   // TAY
    case 0x98: a.Y += a.A.take(); break;   // TYA
    case 0xBA: a.X.clear(); break;         // TSX: SP carries nothing
    case 0x48: a.A += take_write<SAMPLER, GB, XM>(a, aram, aramc, E, cw, j, kind, ref); break;   // PHA
    case 0x08: take_write<SAMPLER, GB, XM>(a, aram, aramc, E, cw, j, kind, ref); break;           // PHP
    case 0x68: {                                                    // PLA
      const Acc g = a.A.take();
      scatter_read<XM>(a, aram, aramc, E, ek, izr, W, rq, kind, ref, fl, g);
      break;
    }
    case 0x20:                                                      // JSR: two pushes
      take_write<SAMPLER, GB, XM>(a, aram, aramc, E, cw, j, kind, stack_addr(ref, 1));
      take_write<SAMPLER, GB, XM>(a, aram, aramc, E, cw, j, kind, stack_addr(ref, 0));
      break;
    case 0x00:                                                      // BRK: three pushes
      take_write<SAMPLER, GB, XM>(a, aram, aramc, E, cw, j, kind, stack_addr(ref, 2));
      take_write<SAMPLER, GB, XM>(a, aram, aramc, E, cw, j, kind, stack_addr(ref, 1));
      take_write<SAMPLER, GB, XM>(a, aram, aramc, E, cw, j, kind, stack_addr(ref, 0));
      break;
    default:
      break;
  }
}

// Shared tables of the relaxed read: ek[k] = exp(-k / tau) for k <= W; for
// every RAM cell i the inverse window normaliser 1 / z_i (izr[i]) and the
// complement of the cell's own weight, (z_i - 1) / z_i (izr[128 + i]),
// computed from the off-centre terms so that it keeps float32's relative
// precision however small it is.
__device__ __forceinline__ void read_tables(float* ek, float* izr, float tau, int W) {
  for (int k = threadIdx.x; k <= W; k += blockDim.x) ek[k] = expf(-(float)k / tau);
  __syncthreads();
  for (int i = threadIdx.x; i < 128; i += blockDim.x) {
    const int lo = i - W < 0 ? 0 : i - W, hi = i + W > 127 ? 127 : i + W;
    float off = 0.f;
    for (int q = lo; q <= hi; q++) off += q == i ? 0.f : ek[q > i ? q - i : i - q];
    const float z = 1.f + off;
    izr[i] = 1.f / z;
    izr[128 + i] = off / z;
  }
  __syncthreads();
}

// The backward runs in two kernels.  The recompute of a segment needs only
// its checkpoint, so a group of segments is recomputed at once (one grid
// row per segment: many more independent machines than envs, which the
// latency-bound interpreter turns into throughput); the reverse sweeps then
// run one segment at a time, last to first, each handing its adjoints to
// the next.  Per (segment slot g, env) the recompute leaves the tape rows,
// the colour / position version sums, the step ends and a small record
// (kMeta words: version count, overflow flag, the sums of the sixteen
// versions alive at the segment start).
constexpr int kMeta = 18;

// Recompute shared memory: the step kernel's layout, then the staged
// gradient rows (16-byte aligned).
__host__ __device__ constexpr size_t rc_row_offset(int E, uint32_t rom_stride, int ram_words) {
  return (smem_bytes(E, rom_stride, ram_words) + 15) & ~(size_t)15;
}
size_t rc_smem_bytes(int E, uint32_t rom_stride, int ram_words) {
  return rc_row_offset(E, rom_stride, ram_words) + (size_t)40 * 16 * E;
}
// The sweep runs one env per warp: envs' tapes differ, so lanes of one warp
// walking different tapes would serialise over their different records,
// while one env per warp lets each SM sub-partition interleave several envs
// (hiding the latency of the global ROM-impulse updates).
constexpr int kSweepEnvs = 4;   // envs (warps) per block
constexpr int kSweepBlock = 128;   // records a warp stages at a time (32 lanes x 4)
constexpr int kSweepWarpWords = 3 * kSweepBlock;   // staged records, then the ROM queue's indices and adjoints
// Sweep shared memory: the RAM adjoints and their compensation
// [2][256][kSweepEnvs] (RIOT RAM, then the Superchip's RAM), the read
// tables, then each warp's staging words.
constexpr int kSweepCells = 256;
__host__ __device__ constexpr size_t sw_tables_end() {
  return ((size_t)2 * kSweepCells * 4 * kSweepEnvs + (kMaxW + 1 + 256) * 4 + 15) & ~(size_t)15;
}
__host__ __device__ constexpr size_t sw_smem_bytes() { return sw_tables_end() + (size_t)kSweepEnvs * kSweepWarpWords * 4; }

template <int T, bool SAMPLER, bool GB, bool INSTR, bool XM, bool FT>
__global__ void __launch_bounds__(128) k_soft_recompute(BwdParams p) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int E = blockDim.x / T, tid = threadIdx.x, slot = tid / T, rank = tid % T;
  BlockSmem bs = carve_smem(smem, E, p.rom_stride, p.ram_words);
  float4* grow = reinterpret_cast<float4*>(smem + rc_row_offset(E, p.rom_stride, p.ram_words));  // [40][E] staged gradient rows
  const int4 bi = p.blocks[blockIdx.x];
  const int cart = bi.x;
  const uint32_t cb = p.cart_banks[cart];
  const int g = blockIdx.y, seg = p.seg0 + g;
  if (!stage_block(bs, p.dt, p.roms + (size_t)cart * p.rom_stride, cart_image_bytes(cb), p.err)) return;
  const bool active = slot < bi.z;
  const int env = active ? p.perm[bi.y + slot] : 0;
  const int n = p.n_envs;
  const uint32_t lanes = warp_lanes(E * T);
  Ctx c = make_ctx<XM, FT>(bs, E, slot, rank, T, cb, p.ystart);
  Regs r;
  if (active) {
    load_env(soa_at(const_cast<uint32_t*>(p.ckpt + (size_t)seg * kStateWords * n), n), n, env, c, r);
  } else {
    power_on(c, r);
  }
  RecTape<SAMPLER, GB, FT> tape;
  tape.buf = p.rec + ((size_t)g * n + env) * p.cap_rec;
  tape.cw = p.cw + ((size_t)g * n + env) * p.cap_cw;
  tape.n = 0; tape.cap = p.cap_rec;
  tape.ncw = 0; tape.capcw = p.cap_cw;
  tape.slot0 = tape.slot1 = tape.slot2 = tape.slot3 = tape.slot4 = -1;
  tape.s0 = tape.s1 = tape.s2 = tape.s3 = tape.s4 = 0.f;
  tape.c0 = tape.c1 = tape.c2 = tape.c3 = tape.c4 = 0.f;
  tape.p0 = tape.p1 = tape.p2 = tape.p3 = tape.p4 = 0.f;
#pragma unroll
  for (int k = 0; k < kGbN; k++) {
    tape.gsl[k] = -1;
    tape.gs[k] = tape.gc[k] = tape.gp[k] = 0.f;
  }
  tape.overflow = false;
  tape.T = (uint32_t)T;
  tape.gmask = c.gmask;
  const int t0 = seg * p.seg_steps;
  const int t1 = min(t0 + p.seg_steps, p.n_steps);
  uint32_t* step_end = p.step_end + (size_t)g * p.seg_steps * n;
  Render rd;
  rd.on = false;
  rd.cur = 0;
  rd.out_u8 = nullptr;
  rd.out_f32 = nullptr;
  rd.grow = grow;
  rd.gslot = (uint32_t)slot;
  for (int t = t0; t < t1; t++) {
    set_input_bits(r, active ? p.act_bits[(size_t)t * n + env] : 0u);
    Step st;
    st.frame_skip = p.frame_skip;
    st.status = 0;
    rd.gs = p.grad_screen ? p.grad_screen + ((size_t)t * n + env) * (kScreenH * kScreenW) : p.w_screen;
    rd.gline = -1;
    st.want_screen = rd.gs != nullptr;
    st.instr_left = p.step_instr;
    run_frames<INSTR>(c, r, rd, st, tape, active, lanes, p.sched_policy, p.sched_window);
    if (active) {
      normalise_timer(r);
      step_end[(size_t)(t - t0) * n + env] = tape.n;
    }
  }
  if (!active) return;
  tape.finish();
  if (rank != 0) return;
  float* m = p.meta + ((size_t)g * n + env) * kMeta;
  m[0] = __uint_as_float(tape.ncw);
  m[1] = tape.overflow ? 1.f : 0.f;
  m[2] = tape.p0;
  m[3] = tape.p1;
  m[4] = tape.p2;
  m[5] = tape.p3;
  m[6] = tape.p4;
#pragma unroll
  for (int k = 0; k < kGbN; k++) m[7 + k] = tape.gp[k];
  if (tape.overflow) atomicExch(p.err, 2);
}

// The reverse sweep of segment p.seg (slot p.seg - p.seg0 of the group), one
// env per warp (lane 0): adjoints of A, X, Y, the timer value, the colour
// registers, player 0's position and HMP0 in registers, the 128 RAM cells and
// the Superchip's 128 (compensated) in shared memory.
template <bool SAMPLER, bool GB, bool XM>
__global__ void __launch_bounds__(32 * kSweepEnvs) k_soft_sweep(BwdParams p) {
  extern __shared__ __align__(128) uint8_t smem[];
  constexpr int E = kSweepEnvs;
  const int slot = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* aram_s = reinterpret_cast<float*>(smem);   // [256][E]
  float* aramc_s = aram_s + kSweepCells * E;         // [256][E] compensation
  float* ek = aramc_s + kSweepCells * E;             // [kMaxW + 1]
  float* izr = ek + (kMaxW + 1);                     // [256]: 1 / z_i, then (z_i - 1) / z_i
  uint32_t* wbuf = reinterpret_cast<uint32_t*>(smem + sw_tables_end()) + slot * kSweepWarpWords;
  uint32_t* recs = wbuf;                             // [kSweepBlock] records of the current block
  RomQueue rq;
  rq.idx = wbuf + kSweepBlock;                       // [kSweepBlock]
  rq.g = reinterpret_cast<float*>(wbuf + 2 * kSweepBlock);   // [kSweepBlock]
  rq.n = 0;
  read_tables(ek, izr, p.tau, p.W);
  const int env = blockIdx.x * E + slot;
  if (env >= p.n_envs) return;   // whole warps leave together
  const uint32_t cart = (uint32_t)p.env_cart[env];
  const uint32_t kind = (p.cart_2k[cart] ? kKind2K : 0u) | (XM && cart_is_sc(p.cart_banks[cart]) ? kKindSC : 0u) |
                        (XM && cart_is_e0(p.cart_banks[cart]) ? kKindE0 : 0u);
  constexpr int cells = XM ? kSweepCells : 128;   // adjoint cells the sweep keeps
  const int n = p.n_envs, g = p.seg - p.seg0;
  const float* m = p.meta + ((size_t)g * n + env) * kMeta;
  if (m[1] != 0.f) return;   // overflow: the error word is set
  const bool lead = lane == 0;   // lane 0 runs the sweep; the warp loads records and adds ROM impulses
  float* aram = aram_s + slot;
  float* aramc = aramc_s + slot;
  Adj a;
  a.ft = p.full_tia != 0;
  if (lead) {
    if (p.first) {
      a.A = a.X = a.Y = a.V = a.C0 = a.C1 = a.C2 = a.C3 = acc(0.f);
#pragma unroll
      for (int k = 0; k < kGbN; k++) a.G[k] = acc(0.f);
      a.P = a.H = 0.f;
      for (int i = 0; i < cells; i++) aram[i * E] = 0.f;
      for (int i = 0; i < cells; i++) aramc[i * E] = 0.f;
    } else {
      const float* cr = p.carry;
      a.A = acc(cr[0 * n + env]); a.X = acc(cr[1 * n + env]); a.Y = acc(cr[2 * n + env]);
      a.V = acc(cr[3 * n + env]);
      a.C0 = acc(cr[4 * n + env]); a.C1 = acc(cr[5 * n + env]); a.C2 = acc(cr[6 * n + env]);
      a.C3 = acc(cr[(size_t)kCarryC3 * n + env]);
#pragma unroll
      for (int k = 0; k < kGbN; k++) a.G[k] = acc(GB ? cr[(size_t)(kCarryGB + k) * n + env] : 0.f);
      a.P = SAMPLER ? cr[(size_t)kCarryPos * n + env] : 0.f;
      a.H = SAMPLER ? cr[(size_t)(kCarryPos + 1) * n + env] : 0.f;
      for (int i = 0; i < 128; i++) aram[i * E] = cr[(size_t)(7 + i) * n + env];
      for (int i = 0; i < 128; i++) aramc[i * E] = cr[(size_t)(7 + 128 + i) * n + env];
      if constexpr (XM) {
        for (int i = 0; i < 128; i++) {
          aram[(128 + i) * E] = (kind & kKindSC) ? cr[(size_t)(kCarryCram + i) * n + env] : 0.f;
          aramc[(128 + i) * E] = (kind & kKindSC) ? cr[(size_t)(kCarryCram + 128 + i) * n + env] : 0.f;
        }
      }
    }
  }
  float2* imp = reinterpret_cast<float2*>(p.imp) + (size_t)env * p.rom_stride;
  const uint4* rec4 = reinterpret_cast<const uint4*>(p.rec + ((size_t)g * n + env) * p.cap_rec);
  const float* cw = p.cw + ((size_t)g * n + env) * p.cap_cw;
  const uint32_t* step_end = p.step_end + (size_t)g * p.seg_steps * n;
  uint32_t j = __float_as_uint(m[0]);
  const int t0 = p.seg * p.seg_steps;
  const int t1 = min(t0 + p.seg_steps, p.n_steps);
  constexpr uint32_t kChunks = kSweepBlock / 4;   // 4-record chunks per block (one per lane)
  for (int t = t1 - 1; t >= t0; t--) {
    if (lead) {
      const float* gr = p.grad_ram ? p.grad_ram + ((size_t)t * n + env) * 128 : p.w_ram;
      if (gr)
        for (int i = 0; i < 128; i++) comp_add(aram[i * E], aramc[i * E], gr[i]);
      for (int q = 0; q < 5; q++) a.u[q] = a.uc[q] = 0.f;
    }
    const uint32_t k_end = step_end[(size_t)(t - t0) * n + env];
    const uint32_t k_beg = t > t0 ? step_end[(size_t)(t - 1 - t0) * n + env] : 0u;
    // records are read backwards a block of 32 aligned 4-record chunks at a
    // time (tape rows are 16-byte aligned), each lane loading one chunk, the
    // next block in flight while lane 0 sweeps the current one
    const uint32_t cb = k_beg >> 2;
    auto block_base = [&](uint32_t k) {   // first chunk of the block that ends at record k
      const uint32_t ct = (k - 1) >> 2;
      return ct >= cb + (kChunks - 1) ? ct - (kChunks - 1) : cb;
    };
    auto load = [&](uint32_t k, uint32_t c0) {
      return c0 + lane <= ((k - 1) >> 2) ? __ldcs(rec4 + c0 + lane) : make_uint4(0u, 0u, 0u, 0u);
    };
    uint32_t k = k_end;
    uint32_t c0 = k > k_beg ? block_base(k) : 0u;
    uint4 v = k > k_beg ? load(k, c0) : make_uint4(0u, 0u, 0u, 0u);
    while (k > k_beg) {
      reinterpret_cast<uint4*>(recs)[lane] = v;
      __syncwarp();
      const uint32_t lo = 4 * c0 > k_beg ? 4 * c0 : k_beg;
      uint32_t c1 = 0;
      if (lo > k_beg) {
        c1 = block_base(lo);
        v = load(lo, c1);
      }
      if (lead)
        for (uint32_t q = k; q > lo; q--)
          reverse_one<SAMPLER, GB, XM>(a, aram, aramc, E, ek, izr, p.W, rq, kind, cw, j, recs[q - 1 - 4 * c0]);
      // the warp adds the block's ROM impulses: lane l takes the indices
      // congruent to l mod 32, each in queue order
      const uint32_t qn = __shfl_sync(0xFFFFFFFFu, rq.n, 0);
      __syncwarp();
      for (uint32_t e = 0; e < qn; e++) {
        const uint32_t ix = rq.idx[e];
        if ((ix & 31) == (uint32_t)lane) {
          float2 w = imp[ix];   // value and compensation in one 8-byte access
          comp_add(w.x, w.y, rq.g[e]);
          imp[ix] = w;
        }
      }
      __syncwarp();
      rq.n = 0;
      k = lo;
      c0 = c1;
    }
    if (lead && p.grad_u) {
      float* gu = p.grad_u + ((size_t)t * n + env) * 5;
      for (int q = 0; q < 5; q++) gu[q] = a.u[q] + a.uc[q];
    }
  }
  if (!lead) return;
  // versions alive at the segment start continue into the previous segment
  a.C0 += m[2];
  a.C1 += m[3];
  a.C2 += m[4];
  a.C3 += m[6];
  if constexpr (SAMPLER) a.P += m[5];
  if constexpr (GB) {
#pragma unroll
    for (int k = 0; k < kGbN; k++) a.G[k] += m[7 + k];
  }
  if (p.seg == 0) {
    if (p.grad_ram0)
      for (int i = 0; i < 128; i++) p.grad_ram0[(size_t)env * 128 + i] = aram[i * E] + aramc[i * E];
    if (p.grad_cart_ram0)
      for (int i = 0; i < 128; i++)
        p.grad_cart_ram0[(size_t)env * 128 + i] = XM ? aram[(128 + i) * E] + aramc[(128 + i) * E] : 0.f;
  } else {
    float* cr = p.carry;
    cr[0 * n + env] = a.A.v(); cr[1 * n + env] = a.X.v(); cr[2 * n + env] = a.Y.v(); cr[3 * n + env] = a.V.v();
    cr[4 * n + env] = a.C0.v(); cr[5 * n + env] = a.C1.v(); cr[6 * n + env] = a.C2.v();
    cr[(size_t)kCarryC3 * n + env] = a.C3.v();
    if constexpr (GB) {
#pragma unroll
      for (int k = 0; k < kGbN; k++) cr[(size_t)(kCarryGB + k) * n + env] = a.G[k].v();
    }
    cr[(size_t)kCarryPos * n + env] = a.P; cr[(size_t)(kCarryPos + 1) * n + env] = a.H;
    for (int i = 0; i < 128; i++) cr[(size_t)(7 + i) * n + env] = aram[i * E];
    for (int i = 0; i < 128; i++) cr[(size_t)(7 + 128 + i) * n + env] = aramc[i * E];
    if (XM && (kind & kKindSC)) {
      for (int i = 0; i < 128; i++) cr[(size_t)(kCarryCram + i) * n + env] = aram[(128 + i) * E];
      for (int i = 0; i < 128; i++) cr[(size_t)(kCarryCram + 128 + i) * n + env] = aramc[(128 + i) * E];
    }
  }
}

// The reverse sweep with one env per lane (kLaneEnvs envs a block, a
// quarter of a warp: several small warps an SMSP hide more of the walkers'
// latency than one full one; measured backward at 16,384 / 65,536 envs and
// 3,000-instruction steps: 32 a block 3.23 / 9.61 ms, 16 3.06 / 9.13, 8
// 2.98 / 9.10):
// each lane walks its own env's tape with the same per-record arithmetic as
// k_soft_sweep and adds its own ROM impulses, so every env's sums take the
// same terms in the same order and the gradients are the same bits.  Lanes
// of a warp whose next records are of one kind share the instructions; for
// batches of more envs than one wave of k_soft_sweep's warps, where that
// kernel's issue slots go to its single walking lane, this is the faster.
constexpr int kLaneQ = 8;   // ROM impulses a lane queues before adding them
__host__ __device__ constexpr size_t swl_smem_bytes(int cells) {
  return ((size_t)2 * cells * kLaneEnvs + (kMaxW + 1 + 256) + (size_t)2 * kLaneQ * kLaneEnvs) * 4;
}

template <bool SAMPLER, bool GB, bool XM>
__global__ void __launch_bounds__(kLaneEnvs) k_soft_sweep_lanes(BwdParams p) {
  extern __shared__ __align__(128) uint8_t smem[];
  constexpr int E = kLaneEnvs;
  constexpr int cells = XM ? kSweepCells : 128;   // adjoint cells the sweep keeps
  const int lane = threadIdx.x;
  float* aram_s = reinterpret_cast<float*>(smem);   // [cells][E]
  float* aramc_s = aram_s + cells * E;              // [cells][E] compensation
  float* ek = aramc_s + cells * E;                  // [kMaxW + 1]
  float* izr = ek + (kMaxW + 1);                    // [256]
  uint32_t* q_idx = reinterpret_cast<uint32_t*>(izr + 256);   // [kLaneQ][E]
  float* q_g = reinterpret_cast<float*>(q_idx + kLaneQ * E);   // [kLaneQ][E]
  read_tables(ek, izr, p.tau, p.W);
  const int env = blockIdx.x * E + lane;
  if (env >= p.n_envs) return;
  const uint32_t cart = (uint32_t)p.env_cart[env];
  const uint32_t kind = (p.cart_2k[cart] ? kKind2K : 0u) | (XM && cart_is_sc(p.cart_banks[cart]) ? kKindSC : 0u) |
                        (XM && cart_is_e0(p.cart_banks[cart]) ? kKindE0 : 0u);
  const int n = p.n_envs, g = p.seg - p.seg0;
  const float* m = p.meta + ((size_t)g * n + env) * kMeta;
  if (m[1] != 0.f) return;   // overflow: the error word is set
  float* aram = aram_s + lane;
  float* aramc = aramc_s + lane;
  LaneQueue rq{q_idx + lane, q_g + lane, 0u};
  Adj a;
  a.ft = p.full_tia != 0;
  if (p.first) {
    a.A = a.X = a.Y = a.V = a.C0 = a.C1 = a.C2 = a.C3 = acc(0.f);
#pragma unroll
    for (int k = 0; k < kGbN; k++) a.G[k] = acc(0.f);
    a.P = a.H = 0.f;
    for (int i = 0; i < cells; i++) aram[i * E] = 0.f;
    for (int i = 0; i < cells; i++) aramc[i * E] = 0.f;
  } else {
    const float* cr = p.carry;
    a.A = acc(cr[0 * n + env]); a.X = acc(cr[1 * n + env]); a.Y = acc(cr[2 * n + env]);
    a.V = acc(cr[3 * n + env]);
    a.C0 = acc(cr[4 * n + env]); a.C1 = acc(cr[5 * n + env]); a.C2 = acc(cr[6 * n + env]);
    a.C3 = acc(cr[(size_t)kCarryC3 * n + env]);
#pragma unroll
    for (int k = 0; k < kGbN; k++) a.G[k] = acc(GB ? cr[(size_t)(kCarryGB + k) * n + env] : 0.f);
    a.P = SAMPLER ? cr[(size_t)kCarryPos * n + env] : 0.f;
    a.H = SAMPLER ? cr[(size_t)(kCarryPos + 1) * n + env] : 0.f;
    for (int i = 0; i < 128; i++) aram[i * E] = cr[(size_t)(7 + i) * n + env];
    for (int i = 0; i < 128; i++) aramc[i * E] = cr[(size_t)(7 + 128 + i) * n + env];
    if constexpr (XM) {
      for (int i = 0; i < 128; i++) {
        aram[(128 + i) * E] = (kind & kKindSC) ? cr[(size_t)(kCarryCram + i) * n + env] : 0.f;
        aramc[(128 + i) * E] = (kind & kKindSC) ? cr[(size_t)(kCarryCram + 128 + i) * n + env] : 0.f;
      }
    }
  }
  float2* imp = reinterpret_cast<float2*>(p.imp) + (size_t)env * p.rom_stride;
  // the queued impulses, in queue order: all loads first (in flight
  // together), an index that repeats in the queue taking its earlier
  // entry's updated pair, then the stores in order (a repeated index ends
  // with its last, fully updated pair)
  auto flush = [&]() {
    uint32_t ix[kLaneQ];
    float2 w[kLaneQ];
#pragma unroll
    for (int e = 0; e < kLaneQ; e++)
      if (e < (int)rq.n) {
        ix[e] = rq.idx[e * E];
        w[e] = imp[ix[e]];
      }
#pragma unroll
    for (int e = 0; e < kLaneQ; e++)
      if (e < (int)rq.n) {
#pragma unroll
        for (int f = 0; f < e; f++)
          if (ix[f] == ix[e]) w[e] = w[f];
        comp_add(w[e].x, w[e].y, rq.g[e * E]);
      }
#pragma unroll
    for (int e = 0; e < kLaneQ; e++)
      if (e < (int)rq.n) imp[ix[e]] = w[e];
    rq.n = 0;
  };
  const uint4* rec4 = reinterpret_cast<const uint4*>(p.rec + ((size_t)g * n + env) * p.cap_rec);
  uint32_t j = __float_as_uint(m[0]);
  CwAhead cw{p.cw + ((size_t)g * n + env) * p.cap_cw, 0.f};
  if (j) cw.next = cw.p[j - 1];
  const uint32_t* step_end = p.step_end + (size_t)g * p.seg_steps * n;
  const int t0 = p.seg * p.seg_steps;
  const int t1 = min(t0 + p.seg_steps, p.n_steps);
  // records are read backwards four at a time (16-byte tape rows; a
  // segment's records are contiguous, step after step), the chunk below the
  // current one in flight.  The loads are unconditional (chunk 0 stands in
  // below chunk 0; the tape holds at least one chunk), so no value waits on
  // a load that a select might discard.
  const uint32_t k_last = step_end[(size_t)(t1 - 1 - t0) * n + env];
  uint32_t cc = k_last ? (k_last - 1) >> 2 : 0u;   // chunk held in cur
  uint4 cur = __ldcs(rec4 + cc);
  uint4 nxt = __ldcs(rec4 + (cc ? cc - 1 : 0u));
  for (int t = t1 - 1; t >= t0; t--) {
    const float* gr = p.grad_ram ? p.grad_ram + ((size_t)t * n + env) * 128 : p.w_ram;
    if (gr)
      for (int i = 0; i < 128; i++) comp_add(aram[i * E], aramc[i * E], gr[i]);
    for (int q = 0; q < 5; q++) a.u[q] = a.uc[q] = 0.f;
    const uint32_t k_end = step_end[(size_t)(t - t0) * n + env];
    const uint32_t k_beg = t > t0 ? step_end[(size_t)(t - 1 - t0) * n + env] : 0u;
    for (uint32_t k = k_end; k > k_beg; k--) {
      const uint32_t c = (k - 1) >> 2;
      if (c != cc) {   // c == cc - 1
        cur = nxt;
        nxt = __ldcs(rec4 + (c ? c - 1 : 0u));
        cc = c;
      }
      const uint32_t w = (k - 1) & 3;
      const uint32_t r = w == 0 ? cur.x : w == 1 ? cur.y : w == 2 ? cur.z : cur.w;
      reverse_one<SAMPLER, GB, XM>(a, aram, aramc, E, ek, izr, p.W, rq, kind, cw, j, r);
      // the lanes flush together when one queue is full: one wait for the
      // impulse rows' loads instead of one for every lane at another record
      if (__any_sync(__activemask(), rq.n == kLaneQ)) flush();
    }
    if (p.grad_u) {
      float* gu = p.grad_u + ((size_t)t * n + env) * 5;
      for (int q = 0; q < 5; q++) gu[q] = a.u[q] + a.uc[q];
    }
  }
  flush();
  // versions alive at the segment start continue into the previous segment
  a.C0 += m[2];
  a.C1 += m[3];
  a.C2 += m[4];
  a.C3 += m[6];
  if constexpr (SAMPLER) a.P += m[5];
  if constexpr (GB) {
#pragma unroll
    for (int k = 0; k < kGbN; k++) a.G[k] += m[7 + k];
  }
  if (p.seg == 0) {
    if (p.grad_ram0)
      for (int i = 0; i < 128; i++) p.grad_ram0[(size_t)env * 128 + i] = aram[i * E] + aramc[i * E];
    if (p.grad_cart_ram0)
      for (int i = 0; i < 128; i++)
        p.grad_cart_ram0[(size_t)env * 128 + i] = XM ? aram[(128 + i) * E] + aramc[(128 + i) * E] : 0.f;
  } else {
    float* cr = p.carry;
    cr[0 * n + env] = a.A.v(); cr[1 * n + env] = a.X.v(); cr[2 * n + env] = a.Y.v(); cr[3 * n + env] = a.V.v();
    cr[4 * n + env] = a.C0.v(); cr[5 * n + env] = a.C1.v(); cr[6 * n + env] = a.C2.v();
    cr[(size_t)kCarryC3 * n + env] = a.C3.v();
    if constexpr (GB) {
#pragma unroll
      for (int k = 0; k < kGbN; k++) cr[(size_t)(kCarryGB + k) * n + env] = a.G[k].v();
    }
    cr[(size_t)kCarryPos * n + env] = a.P; cr[(size_t)(kCarryPos + 1) * n + env] = a.H;
    for (int i = 0; i < 128; i++) cr[(size_t)(7 + i) * n + env] = aram[i * E];
    for (int i = 0; i < 128; i++) cr[(size_t)(7 + 128 + i) * n + env] = aramc[i * E];
    if (XM && (kind & kKindSC)) {
      for (int i = 0; i < 128; i++) cr[(size_t)(kCarryCram + i) * n + env] = aram[(128 + i) * E];
      for (int i = 0; i < 128; i++) cr[(size_t)(kCarryCram + 128 + i) * n + env] = aramc[(128 + i) * E];
    }
  }
}

// Which sweep a batch runs (vcs_config.sweep_mode): 1 = k_soft_sweep (one
// env per warp), 2 = k_soft_sweep_lanes (one env per lane), 0 = the lanes
// from kSweepLanesFrom envs, about four waves of k_soft_sweep's warps (28
// an SM at its 72 registers).  Measured backward times (ms, same box, one
// 4 KB cart; 3,000-instruction steps / 64 frames): 8192 envs 2.31 / 130
// with the warps against 2.74 / 142 with the lanes; 16,384 envs 3.47 / 199
// against 2.98 / 154; 65,536 envs 12.4 / 730 against 9.1 / 523.
constexpr int kSweepLanesFrom = 16384;
static int sweep_lanes(const vcs_batch* b) {
  return b->cfg.sweep_mode == 2 || (b->cfg.sweep_mode == 0 && b->n_envs >= kSweepLanesFrom);
}

template <class Kern>
static cudaError_t allow_smem(Kern kern, size_t smem) {
  return smem > 48u * 1024u ? cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                            : cudaSuccess;
}

// Recompute segments seg0 .. seg0 + G - 1 (grid rows), envs in blocks of E
// with T lanes each.
static cudaError_t launch_recompute(const BwdParams& p, int G, int n_blocks, int E, int T, size_t smem,
                                    cudaStream_t s) {
  const dim3 grid(n_blocks, G);
  cudaError_t e = cudaSuccess;
  auto go = [&](auto kern, int threads) {
    if ((e = allow_smem(kern, smem)) == cudaSuccess) kern<<<grid, threads, smem, s>>>(p);
  };
  auto pick = [&](auto xm, auto ft) {
    constexpr bool XM = decltype(xm)::value, FT = decltype(ft)::value;
    // instruction-granular steps draw nothing (no pixel sums, no position
    // sampler), so one lane per env serves them
    if (p.step_instr > 0) {
      go(k_soft_recompute<1, false, false, true, XM, FT>, E);
    } else if (p.graphics) {
      // the graphics-bit surrogate is built for one lane per env and for
      // four replicas: 2 runs as 1 and 8 as 4
      if (p.sampler) {
        if (T >= 4) go(k_soft_recompute<4, true, true, false, XM, FT>, 4 * E);
        else go(k_soft_recompute<1, true, true, false, XM, FT>, E);
      } else {
        if (T >= 4) go(k_soft_recompute<4, false, true, false, XM, FT>, 4 * E);
        else go(k_soft_recompute<1, false, true, false, XM, FT>, E);
      }
    } else if (p.sampler) {
      switch (T) {
        case 1: go(k_soft_recompute<1, true, false, false, XM, FT>, E); break;
        case 2: go(k_soft_recompute<2, true, false, false, XM, FT>, 2 * E); break;
        case 4: go(k_soft_recompute<4, true, false, false, XM, FT>, 4 * E); break;
        default: go(k_soft_recompute<8, true, false, false, XM, FT>, 8 * E); break;
      }
    } else {
      switch (T) {
        case 1: go(k_soft_recompute<1, false, false, false, XM, FT>, E); break;
        case 2: go(k_soft_recompute<2, false, false, false, XM, FT>, 2 * E); break;
        case 4: go(k_soft_recompute<4, false, false, false, XM, FT>, 4 * E); break;
        default: go(k_soft_recompute<8, false, false, false, XM, FT>, 8 * E); break;
      }
    }
  };
  if (p.full_tia) pick(std::true_type{}, std::true_type{});
  else if (p.xmap) pick(std::true_type{}, std::false_type{});
  else pick(std::false_type{}, std::false_type{});
  return e != cudaSuccess ? e : cudaGetLastError();
}

static cudaError_t launch_sweep(const BwdParams& p, cudaStream_t s) {
  const bool sampler = p.sampler && p.step_instr <= 0, gb = p.graphics != 0, xm = p.xmap != 0;
  if (p.sweep_lanes) {
    const dim3 grid((p.n_envs + kLaneEnvs - 1) / kLaneEnvs), block(kLaneEnvs);
    const size_t sm = swl_smem_bytes(xm ? kSweepCells : 128);
    cudaError_t e = cudaSuccess;
    auto go = [&](auto kern) {
      if ((e = allow_smem(kern, sm)) == cudaSuccess) kern<<<grid, block, sm, s>>>(p);
    };
    if (gb) {
      if (sampler && xm) go(k_soft_sweep_lanes<true, true, true>);
      else if (sampler) go(k_soft_sweep_lanes<true, true, false>);
      else if (xm) go(k_soft_sweep_lanes<false, true, true>);
      else go(k_soft_sweep_lanes<false, true, false>);
    } else {
      if (sampler && xm) go(k_soft_sweep_lanes<true, false, true>);
      else if (sampler) go(k_soft_sweep_lanes<true, false, false>);
      else if (xm) go(k_soft_sweep_lanes<false, false, true>);
      else go(k_soft_sweep_lanes<false, false, false>);
    }
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  const int n_blocks = (p.n_envs + kSweepEnvs - 1) / kSweepEnvs;
  const dim3 grid(n_blocks), block(32 * kSweepEnvs);
  const size_t sm = sw_smem_bytes();
  if (gb) {
    if (sampler && xm) k_soft_sweep<true, true, true><<<grid, block, sm, s>>>(p);
    else if (sampler) k_soft_sweep<true, true, false><<<grid, block, sm, s>>>(p);
    else if (xm) k_soft_sweep<false, true, true><<<grid, block, sm, s>>>(p);
    else k_soft_sweep<false, true, false><<<grid, block, sm, s>>>(p);
  } else {
    if (sampler && xm) k_soft_sweep<true, false, true><<<grid, block, sm, s>>>(p);
    else if (sampler) k_soft_sweep<true, false, false><<<grid, block, sm, s>>>(p);
    else if (xm) k_soft_sweep<false, false, true><<<grid, block, sm, s>>>(p);
    else k_soft_sweep<false, false, false><<<grid, block, sm, s>>>(p);
  }
  return cudaGetLastError();
}

// ROM impulses -> ROM gradient: spread each impulse at a over the read
// window of its tensor (the 2K image, the 4K image, one 4 KB bank of a
// bank-switched cart or one 1 KB slice of an E0 cart) with the relaxed
// read's weights.  One thread per (env,
// ROM byte); rows are rom_stride floats.
__global__ void k_rom_spread(const float* imp, float* out, const int32_t* env_cart, const uint8_t* cart_banks,
                             const uint8_t* cart_2k, int32_t n_envs, uint32_t rom_stride, float tau, int32_t W) {
  // FP64 here: the impulses are compensated float pairs whose sum the spread
  // must not round before the weights cancel neighbouring terms (a tiny
  // kernel next to the backward)
  __shared__ double ek[kMaxW + 2];
  __shared__ double suf[kMaxW + 2];   // suf[k] = sum_{q = k..W} ek[q]
  for (int k = threadIdx.x; k <= W; k += blockDim.x) ek[k] = exp(-(double)k / (double)tau);
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0;
    suf[W + 1] = 0.0;
    for (int k = W; k >= 0; k--) {
      acc += ek[k];
      suf[k] = acc;
    }
  }
  __syncthreads();
  const int env = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (env >= n_envs || i >= (int)rom_stride) return;
  const int cart = env_cart[env];
  const uint32_t cb = cart_banks[cart];
  const int M = cart_2k[cart] ? 2048 : (cart_is_e0(cb) ? 1024 : 4096);   // the read tensor
  float* o = out + (size_t)env * rom_stride;
  if (i >= (cart_2k[cart] ? 2048 : (int)cart_image_bytes(cb))) {
    o[i] = 0.f;
    return;
  }
  const int base = i & ~(M - 1);
  const int ii = i - base;
  const float2* im = reinterpret_cast<const float2*>(imp) + (size_t)env * rom_stride + base;
  const int lo = ii - W < 0 ? 0 : ii - W, hi = ii + W > M - 1 ? M - 1 : ii + W;
  const double zint = ek[0] + 2.0 * suf[1];
  double acc = 0.0;
  for (int q = lo; q <= hi; q++) {
    const double v = (double)im[q].x + (double)im[q].y;
    if (v == 0.0) continue;
    double z = zint;
    if (q < W) z -= suf[q + 1];
    if (M - 1 - q < W) z -= suf[M - q];
    acc += v * ek[q > ii ? q - ii : ii - q] / z;
  }
  o[i] = (float)acc;
}

// Per-cart sum of the per-env ROM gradients: envs of cart c are slots
// cart_begin[c] .. cart_begin[c+1]-1 of perm; a fixed order, no atomics.
__global__ void k_cart_reduce(const float* grad_rom, float* out, const int32_t* perm, const int32_t* cart_begin,
                              int32_t n_carts, uint32_t rom_stride) {
  const int c = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_carts || i >= (int)rom_stride) return;
  double acc = 0.0;   // thousands of envs per cart: FP64 keeps the sum to its last float bit
  for (int s = cart_begin[c]; s < cart_begin[c + 1]; s++) acc += grad_rom[(size_t)perm[s] * rom_stride + i];
  out[(size_t)c * rom_stride + i] = (float)acc;
}

// Rounded ROM bytes from the float ROM tensor (forward value of the STE
// round), 2K images mirrored into 4 KB like the hard path's copy.
__global__ void k_rom_round(const float* rom_f32, uint8_t* out, const uint8_t* cart_2k, int32_t n_carts,
                            uint32_t rom_stride) {
  const int c = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_carts || i >= (int)rom_stride) return;
  const int src = cart_2k[c] ? (i & 2047) : i;
  float v = rintf(rom_f32[(size_t)c * rom_stride + src]);
  out[(size_t)c * rom_stride + i] = (uint8_t)(v <= 0.f ? 0.f : (v >= 255.f ? 255.f : v));
}

}  // namespace vcs

using namespace vcs;

struct vcs_tape {
  vcs_batch* b = nullptr;
  int32_t n_steps = 0, frame_skip = 1, seg_steps = 1, n_seg = 0, W = 1;
  float tau = 1.f;
  uint8_t* rom_bytes = nullptr;
  uint32_t* ckpt = nullptr;
  uint8_t* act_bits = nullptr;
  uint32_t* seg_counts = nullptr;
  // backward scratch (allocated by the first vcs_backward): the tapes of a
  // group of G segments
  int32_t G = 0;
  uint32_t* rec = nullptr;
  size_t cap_rec = 0;
  float* cw = nullptr;
  size_t cap_cw = 0;
  uint32_t* step_end = nullptr;
  float* meta = nullptr;
  float* carry = nullptr;
  float* imp = nullptr;
  float* grad_rom_tmp = nullptr;
};

static void free_tape(vcs_tape* t) {
  if (!t) return;
  cudaFree(t->rom_bytes);
  cudaFree(t->ckpt);
  cudaFree(t->act_bits);
  cudaFree(t->seg_counts);
  cudaFree(t->rec);
  cudaFree(t->cw);
  cudaFree(t->step_end);
  cudaFree(t->meta);
  cudaFree(t->carry);
  cudaFree(t->imp);
  cudaFree(t->grad_rom_tmp);
  delete t;
}

static int half_width(float tau) {
  int w = (int)std::ceil(12.0 * (double)tau);
  return w < 1 ? 1 : w;
}

// Machines (segments x envs) from which a recompute group runs one lane per
// env rather than the batch's replicas.
constexpr size_t kWideRecomputeMachines = 16384;

// Segments last to first in groups of G: recompute the group's segments at
// once, then sweep them one by one (p's tape pointers hold G slots).
static vcs_status run_backward_groups(vcs_batch* b, const vcs_tape* t, BwdParams& p, int G, cudaStream_t s) {
  const int4* blocks;
  int nbl, E, T = b->tpe;
  vcs_bwd_geometry(b, &blocks, &nbl, &E);
  // A group of many machines (segments x envs) keeps every SM sub-partition
  // busy: issue slots, not one lane's latency, then bound the recompute, and
  // one lane per env in blocks of kWideEnvsPerBlock spends a quarter of the
  // slots that replicated lanes would on the interpreter.
  if ((size_t)G * (size_t)b->n_envs >= kWideRecomputeMachines) {
    blocks = b->wide_blocks;
    nbl = b->wide_n_blocks;
    E = kWideEnvsPerBlock;
    T = 1;
  }
  p.blocks = blocks;
  p.ckpt = t->ckpt;
  const size_t smem = rc_smem_bytes(E, b->rom_stride, b->ram_words);
  cudaError_t e;
  for (int hi = t->n_seg - 1; hi >= 0; hi -= G) {
    const int lo = hi - G + 1 > 0 ? hi - G + 1 : 0;
    p.seg0 = lo;
    if ((e = launch_recompute(p, hi - lo + 1, nbl, E, T, smem, s))) return vcs_cuda_fail(b, e, "recompute launch");
    for (int q = hi; q >= lo; q--) {
      p.seg = q;
      p.first = q == t->n_seg - 1;
      if ((e = launch_sweep(p, s))) return vcs_cuda_fail(b, e, "reverse sweep launch");
    }
  }
  return VCS_OK;
}

// Tape bytes of one segment (records, version sums, step ends, meta).
static size_t segment_tape_bytes(size_t n, size_t cap_rec, size_t cap_cw, int seg_steps) {
  return n * (cap_rec + cap_cw + (size_t)seg_steps + kMeta) * 4;
}

extern "C" {

vcs_status vcs_soft_rollout(vcs_batch* b, float tau, const float* rom_f32, const float* ram0, const float* u,
                            int32_t n_steps, int32_t frame_skip, float* ram_out, float* screen_out,
                            vcs_tape** tape_out, void* stream) {
  if (!b) return VCS_ERR_ARG;
  if (!tape_out) return vcs_fail(b, VCS_ERR_ARG, "tape_out is NULL");
  *tape_out = nullptr;
  if (!u) return vcs_fail(b, VCS_ERR_ARG, "u (joystick inputs) is NULL");
  if (!(tau > 0.f) || !(tau <= 10.f)) return vcs_fail(b, VCS_ERR_ARG, "tau must be in (0, 10]");
  if (n_steps < 1 || frame_skip < 1) return vcs_fail(b, VCS_ERR_ARG, "n_steps >= 1 and frame_skip >= 1 required");
  if (screen_out && b->cfg.step_instructions > 0)
    return vcs_fail(b, VCS_ERR_ARG, "instruction steps return no screens");
  vcs_tape* t = new (std::nothrow) vcs_tape;
  if (!t) return vcs_fail(b, VCS_ERR_OOM, "host allocation failed");
  t->b = b;
  t->n_steps = n_steps;
  t->frame_skip = frame_skip;
  t->tau = tau;
  t->W = half_width(tau);
  // a checkpoint segment is segment_frames frames, or segment_frames
  // instruction-granular steps
  const int32_t seg_div = b->cfg.step_instructions > 0 ? 1 : frame_skip;
  t->seg_steps = b->cfg.segment_frames / seg_div > 0 ? b->cfg.segment_frames / seg_div : 1;
  t->n_seg = (n_steps + t->seg_steps - 1) / t->seg_steps;
  const size_t n = (size_t)b->n_envs;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  const size_t rs = b->rom_stride;
  if ((e = cudaMalloc(&t->rom_bytes, (size_t)b->n_carts * rs)) ||
      (e = cudaMalloc(&t->ckpt, (size_t)t->n_seg * kStateWords * n * 4)) ||
      (e = cudaMalloc(&t->act_bits, (size_t)n_steps * n)) ||
      (e = cudaMalloc(&t->seg_counts, (size_t)t->n_seg * 2 * 4))) {
    vcs_status st = vcs_cuda_fail(b, e, "tape allocation");
    free_tape(t);
    return st;
  }
  cudaMemsetAsync(t->seg_counts, 0, (size_t)t->n_seg * 2 * 4, s);
  if (rom_f32) {
    dim3 grid((unsigned)(rs / 256), b->n_carts);
    k_rom_round<<<grid, 256, 0, s>>>(rom_f32, t->rom_bytes, b->cart_2k, b->n_carts, b->rom_stride);
  } else {
    cudaMemcpyAsync(t->rom_bytes, b->roms, (size_t)b->n_carts * rs, cudaMemcpyDeviceToDevice, s);
  }
  StepParams p = vcs_base_params(b);
  p.roms = t->rom_bytes;
  p.n_steps = n_steps;
  p.frame_skip = frame_skip;
  p.u = u;
  p.ram0 = ram0;
  p.act_bits = t->act_bits;
  p.ram_out_f = ram_out;
  p.screen_out_f = screen_out;
  p.ckpt = t->ckpt;
  p.seg_steps = t->seg_steps;
  p.seg_counts = t->seg_counts;
  // Without screen outputs the forward draws nothing, so replicas have no
  // work to share: one lane per env in blocks of kWideFwdEnvsPerBlock
  // (measured 31 % faster than four replicas on 4096 envs of the 4K / F8 mix)
  int le;
  if (!screen_out) {
    p.blocks = b->wide_fwd_blocks;
    p.tpe = 1;
    le = launch_soft_forward(p, b->wide_fwd_n_blocks, kWideFwdEnvsPerBlock, stream);
  } else {
    le = launch_soft_forward(p, b->n_blocks, b->E, stream);
  }
  if (le) {
    vcs_status st = vcs_cuda_fail(b, (cudaError_t)le, "soft forward launch");
    free_tape(t);
    return st;
  }
  *tape_out = t;
  return VCS_OK;
}

vcs_status vcs_soft_step(vcs_batch* b, float tau, const float* action_inputs, int32_t n_steps, int32_t frame_skip,
                         float* ram_out, float* screen_out, vcs_tape** tape_out, void* stream) {
  return vcs_soft_rollout(b, tau, nullptr, nullptr, action_inputs, n_steps, frame_skip, ram_out, screen_out,
                          tape_out, stream);
}

vcs_status vcs_tape_free(vcs_tape* t) {
  if (!t) return VCS_ERR_ARG;
  free_tape(t);
  return VCS_OK;
}

vcs_status vcs_backward(vcs_tape* t, const float* grad_ram, const float* grad_screen, const vcs_loss_weights* w,
                        float* grad_rom, float* grad_ram0, float* grad_cart_ram0, float* grad_u,
                        float* grad_rom_per_cart, void* stream) {
  if (!t || !t->b) return VCS_ERR_ARG;
  vcs_batch* b = t->b;
  if ((grad_ram || grad_screen) && w && (w->ram || w->screen))
    return vcs_fail(b, VCS_ERR_ARG, "give either per-step gradients or loss weights, not both");
  if (b->cfg.step_instructions > 0 && (grad_screen || (w && w->screen)))
    return vcs_fail(b, VCS_ERR_ARG, "instruction steps return no screens: no screen gradients");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  const size_t n = (size_t)b->n_envs;
  // size the tape from the forward's per-segment counts
  std::vector<uint32_t> counts((size_t)t->n_seg * 2);
  if ((e = cudaMemcpyAsync(counts.data(), t->seg_counts, counts.size() * 4, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaStreamSynchronize(s)))
    return vcs_cuda_fail(b, e, "tape sizes");
  size_t need_rec = 1, need_cw = 1;
  for (int q = 0; q < t->n_seg; q++) {
    need_rec = std::max<size_t>(need_rec, counts[2 * q]);
    need_cw = std::max<size_t>(need_cw, counts[2 * q + 1]);
  }
  need_rec = (need_rec + 3) & ~(size_t)3;   // 16-byte rows: the reverse sweep reads 4 records at once
  // as many segments per group as the tape budget holds
  size_t budget = (size_t)b->cfg.tape_budget_mb << 20;
  if (budget == 0) {   // default: a quarter of the free device memory
    size_t free_b = 0, total_b = 0;
    if ((e = cudaMemGetInfo(&free_b, &total_b))) return vcs_cuda_fail(b, e, "device memory query");
    budget = free_b / 4;
  }
  const size_t per_seg = segment_tape_bytes(n, need_rec, need_cw, t->seg_steps);
  int G = (int)std::min<size_t>((size_t)t->n_seg, std::max<size_t>(1, budget / per_seg));
  if (need_rec > t->cap_rec || need_cw > t->cap_cw || G > t->G) {
    cudaFree(t->rec);
    cudaFree(t->cw);
    cudaFree(t->step_end);
    cudaFree(t->meta);
    t->rec = nullptr;
    t->cw = nullptr;
    t->step_end = nullptr;
    t->meta = nullptr;
    t->G = 0;
    if ((e = cudaMalloc(&t->rec, (size_t)G * need_rec * n * 4)) || (e = cudaMalloc(&t->cw, (size_t)G * need_cw * n * 4)) ||
        (e = cudaMalloc(&t->step_end, (size_t)G * t->seg_steps * n * 4)) ||
        (e = cudaMalloc(&t->meta, (size_t)G * n * kMeta * 4)))
      return vcs_cuda_fail(b, e, "tape allocation");
    t->cap_rec = need_rec;
    t->cap_cw = need_cw;
    t->G = G;
  }
  G = t->G;
  if (!t->carry) {
    if ((e = cudaMalloc(&t->carry, (size_t)kCarry * n * 4)) || (e = cudaMalloc(&t->imp, 2 * n * b->rom_stride * 4)))
      return vcs_cuda_fail(b, e, "backward scratch");
  }
  float* grom = grad_rom;
  if (!grom && grad_rom_per_cart) {
    if (!t->grad_rom_tmp && (e = cudaMalloc(&t->grad_rom_tmp, n * b->rom_stride * 4)))
      return vcs_cuda_fail(b, e, "backward scratch");
    grom = t->grad_rom_tmp;
  }
  cudaMemsetAsync(t->imp, 0, 2 * n * b->rom_stride * 4, s);

  BwdParams p{};
  p.n_envs = b->n_envs;
  p.n_steps = t->n_steps;
  p.frame_skip = t->frame_skip;
  p.seg_steps = t->seg_steps;
  p.ystart = b->cfg.ystart;
  p.perm = b->perm;
  p.roms = t->rom_bytes;
  p.cart_banks = b->cart_banks;
  p.ram_words = b->ram_words;
  p.xmap = b->xmap;
  p.full_tia = b->cfg.full_tia;
  p.rom_stride = b->rom_stride;
  p.cart_2k = b->cart_2k;
  p.env_cart = b->env_cart_dev;
  p.dt = b->dt;
  p.act_bits = t->act_bits;
  p.grad_ram = grad_ram;
  p.grad_screen = grad_screen;
  p.w_ram = w ? w->ram : nullptr;
  p.w_screen = w ? w->screen : nullptr;
  p.rec = t->rec;
  p.cap_rec = (uint32_t)t->cap_rec;
  p.cw = t->cw;
  p.cap_cw = (uint32_t)t->cap_cw;
  p.step_end = t->step_end;
  p.meta = t->meta;
  p.carry = t->carry;
  p.imp = t->imp;
  p.grad_u = grad_u;
  p.grad_ram0 = grad_ram0;
  p.grad_cart_ram0 = grad_cart_ram0;
  p.tau = t->tau;
  p.W = t->W;
  p.tpe = b->tpe;
  p.sampler = b->cfg.position_sampler;
  p.graphics = b->cfg.graphics_bits && b->cfg.step_instructions <= 0;
  p.step_instr = b->cfg.step_instructions;
  p.sweep_lanes = sweep_lanes(b);
  p.sched_policy = b->sched_policy;
  p.sched_window = b->sched_window;
  p.err = b->err;
  vcs_status st = run_backward_groups(b, t, p, G, s);
  if (st != VCS_OK) return st;
  if (grom) {
    dim3 grid(b->rom_stride / 256, b->n_envs);
    k_rom_spread<<<grid, 256, 0, s>>>(t->imp, grom, b->env_cart_dev, b->cart_banks, b->cart_2k, b->n_envs,
                                      b->rom_stride, t->tau, t->W);
    if ((e = cudaGetLastError())) return vcs_cuda_fail(b, e, "ROM spread launch");
  }
  if (grad_rom_per_cart) {
    dim3 grid(b->rom_stride / 256, b->n_carts);
    k_cart_reduce<<<grid, 256, 0, s>>>(grom, grad_rom_per_cart, b->perm, b->cart_begin, b->n_carts, b->rom_stride);
    if ((e = cudaGetLastError())) return vcs_cuda_fail(b, e, "per-cart reduction launch");
  }
  return VCS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Backward pass that allocates nothing (vcs_backward_static).
//
// Some callers cannot let a library allocate device memory: an application
// whose GPU memory is owned by an allocator it does not control (a
// framework's caching pool that has reserved the device, say), or one held
// to a fixed device-memory budget, where a cudaMalloc behind its back can
// fail or fragment the pool.  This variant of the backward pass takes all of
// its scratch (tape, adjoint carries, ROM impulses) from one fixed array
// compiled into the library.  Every GPU that loads the library keeps this
// array until the process exits.  All calls share it and it keeps the last
// call's contents, so calls whose work overlaps on the GPU race with each
// other.
// ---------------------------------------------------------------------------

static constexpr size_t kStaticScratchBytes = 64ull << 20;   // 64 MiB
static __device__ __align__(256) unsigned char g_backward_scratch[kStaticScratchBytes];

static std::mutex g_scratch_mutex;
struct ScratchSlot {
  unsigned long long ctx_id;   // the context the address belongs to (0 = none looked up yet)
  void* ptr;
};
static ScratchSlot g_scratch_slot[64] = {};

// Unique id of the calling thread's current context (0 if none is current
// or the driver cannot say).  A context that is destroyed and made again
// (cudaDeviceReset, or another library resetting the primary context) gets
// a new id, and its module, with the array, is loaded again at a new
// address; the ids keep a stale address from being used.
static unsigned long long current_context_id() {
  typedef CUresult (*GetCurrent)(CUcontext*);
  typedef CUresult (*GetId)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the static scratch on the current device.  The array's
// host-side name is not a device address: the address is looked up with
// cudaGetSymbolAddress, with the device current, once per device and
// context (the first call on a device, and the first after its context was
// made again), and kept for later calls.
static cudaError_t static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  ScratchSlot& slot = g_scratch_slot[dev];
  unsigned long long id = current_context_id();
  if (!slot.ptr || id == 0 || slot.ctx_id != id) {
    void* p = nullptr;
    // binds the device's context to this thread if no runtime call has yet
    e = cudaGetSymbolAddress(&p, g_backward_scratch);
    if (e) return e;
    if (id == 0) id = current_context_id();
    slot.ptr = p;
    slot.ctx_id = id;
  }
  *out = slot.ptr;
  return cudaSuccess;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" vcs_status vcs_backward_static(vcs_tape* t, const float* grad_ram, const float* grad_screen,
                                          const vcs_loss_weights* w, float* grad_rom, float* grad_ram0,
                                          float* grad_cart_ram0, float* grad_u, float* grad_rom_per_cart,
                                          void* stream) {
  if (!t || !t->b) return VCS_ERR_ARG;
  vcs_batch* b = t->b;
  if ((grad_ram || grad_screen) && w && (w->ram || w->screen))
    return vcs_fail(b, VCS_ERR_ARG, "give either per-step gradients or loss weights, not both");
  if (b->cfg.step_instructions > 0 && (grad_screen || (w && w->screen)))
    return vcs_fail(b, VCS_ERR_ARG, "instruction steps return no screens: no screen gradients");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  void* base = nullptr;
  if ((e = static_scratch(&base))) return vcs_cuda_fail(b, e, "static scratch address");
  const size_t n = (size_t)b->n_envs;
  // tape sizes from the forward's per-segment counts (a copy, no allocation)
  uint32_t counts[2 * 64];
  std::vector<uint32_t> counts_big;
  uint32_t* cnt = counts;
  if (t->n_seg > 64) {
    counts_big.assign((size_t)t->n_seg * 2, 0);
    cnt = counts_big.data();
  }
  if ((e = cudaMemcpyAsync(cnt, t->seg_counts, (size_t)t->n_seg * 2 * 4, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaStreamSynchronize(s)))
    return vcs_cuda_fail(b, e, "tape sizes");
  size_t cap_rec = 1, cap_cw = 1;
  for (int q = 0; q < t->n_seg; q++) {
    cap_rec = std::max<size_t>(cap_rec, cnt[2 * q]);
    cap_cw = std::max<size_t>(cap_cw, cnt[2 * q + 1]);
  }
  cap_rec = (cap_rec + 3) & ~(size_t)3;   // 16-byte rows, as in vcs_backward
  const bool need_tmp = !grad_rom && grad_rom_per_cart;
  const size_t o_carry = 0;
  const size_t o_imp = align256(o_carry + (size_t)kCarry * n * 4);
  const size_t o_tmp = align256(o_imp + 2 * n * b->rom_stride * 4);
  const size_t o_tapes = align256(o_tmp + (need_tmp ? n * b->rom_stride * 4 : 0));
  // as many segments per group as the rest of the array holds (at least one)
  const size_t per_seg = segment_tape_bytes(n, cap_rec, cap_cw, t->seg_steps) + 4 * 256;
  const size_t room = kStaticScratchBytes > o_tapes ? kStaticScratchBytes - o_tapes : 0;
  const int G = (int)std::max<size_t>(1, std::min<size_t>((size_t)t->n_seg, room / per_seg));
  const size_t o_step = o_tapes;
  const size_t o_meta = align256(o_step + (size_t)G * t->seg_steps * n * 4);
  const size_t o_rec = align256(o_meta + (size_t)G * n * kMeta * 4);
  const size_t o_cw = align256(o_rec + (size_t)G * cap_rec * n * 4);
  const size_t total = align256(o_cw + (size_t)G * cap_cw * n * 4);
  if (total > kStaticScratchBytes)
    return vcs_fail(b, VCS_ERR_ARG,
                    "vcs_backward_static needs %zu bytes of scratch for %zu envs (%zu instructions per segment), "
                    "above its fixed %zu-byte array; use vcs_backward or fewer envs / shorter segments",
                    total, n, cap_rec, kStaticScratchBytes);
  unsigned char* sc = static_cast<unsigned char*>(base);
  float* imp = reinterpret_cast<float*>(sc + o_imp);
  float* grom = grad_rom ? grad_rom : (need_tmp ? reinterpret_cast<float*>(sc + o_tmp) : nullptr);
  // the impulses are sums and must start at zero; everything else is
  // written before it is read
  if ((e = cudaMemsetAsync(imp, 0, 2 * n * b->rom_stride * 4, s))) return vcs_cuda_fail(b, e, "scratch clear");

  BwdParams p{};
  p.n_envs = b->n_envs;
  p.n_steps = t->n_steps;
  p.frame_skip = t->frame_skip;
  p.seg_steps = t->seg_steps;
  p.ystart = b->cfg.ystart;
  p.perm = b->perm;
  p.roms = t->rom_bytes;
  p.cart_banks = b->cart_banks;
  p.ram_words = b->ram_words;
  p.xmap = b->xmap;
  p.full_tia = b->cfg.full_tia;
  p.rom_stride = b->rom_stride;
  p.cart_2k = b->cart_2k;
  p.env_cart = b->env_cart_dev;
  p.dt = b->dt;
  p.act_bits = t->act_bits;
  p.grad_ram = grad_ram;
  p.grad_screen = grad_screen;
  p.w_ram = w ? w->ram : nullptr;
  p.w_screen = w ? w->screen : nullptr;
  p.rec = reinterpret_cast<uint32_t*>(sc + o_rec);
  p.cap_rec = (uint32_t)cap_rec;
  p.cw = reinterpret_cast<float*>(sc + o_cw);
  p.cap_cw = (uint32_t)cap_cw;
  p.step_end = reinterpret_cast<uint32_t*>(sc + o_step);
  p.meta = reinterpret_cast<float*>(sc + o_meta);
  p.carry = reinterpret_cast<float*>(sc + o_carry);
  p.imp = imp;
  p.grad_u = grad_u;
  p.grad_ram0 = grad_ram0;
  p.grad_cart_ram0 = grad_cart_ram0;
  p.tau = t->tau;
  p.W = t->W;
  p.tpe = b->tpe;
  p.sampler = b->cfg.position_sampler;
  p.graphics = b->cfg.graphics_bits && b->cfg.step_instructions <= 0;
  p.step_instr = b->cfg.step_instructions;
  p.sweep_lanes = sweep_lanes(b);
  p.sched_policy = b->sched_policy;
  p.sched_window = b->sched_window;
  p.err = b->err;
  vcs_status st = run_backward_groups(b, t, p, G, s);
  if (st != VCS_OK) return st;
  if (grom) {
    dim3 grid(b->rom_stride / 256, b->n_envs);
    k_rom_spread<<<grid, 256, 0, s>>>(imp, grom, b->env_cart_dev, b->cart_banks, b->cart_2k, b->n_envs, b->rom_stride,
                                      t->tau, t->W);
    if ((e = cudaGetLastError())) return vcs_cuda_fail(b, e, "ROM spread launch");
  }
  if (grad_rom_per_cart) {
    dim3 grid(b->rom_stride / 256, b->n_carts);
    k_cart_reduce<<<grid, 256, 0, s>>>(grom, grad_rom_per_cart, b->perm, b->cart_begin, b->n_carts, b->rom_stride);
    if ((e = cudaGetLastError())) return vcs_cuda_fail(b, e, "per-cart reduction launch");
  }
  return VCS_OK;
}
