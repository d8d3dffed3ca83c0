// Block set-up, state load/store and the frame loop shared by the kernels.
#pragma once
#include <cuda_runtime.h>

#include "vcs_exec.cuh"
#include "vcs_kernels.cuh"
#include "vcs_tia.cuh"

namespace vcs {

// Shared-memory layout of one block of E envs; the cartridge image region
// is the batch's ROM stride (8, 16 or 32 KB: the largest image it holds).
struct BlockSmem {
  uint8_t* rom;         // cartridge image (rom_bytes)
  DecodeTables* dt;     // 512 B
  uint64_t* mbar;       // TMA completion barrier
  uint32_t* ram;        // [ram_words][E] words: RIOT RAM, then the Superchip's RAM
  uint32_t* line;       // [40][E] words
  uint32_t* tx;         // [6][E] words: the cold TIA registers and the hot copy (vcs_tia.cuh)
};

// ram_words: 32, or 64 in a batch that holds a Superchip cart.
__host__ __device__ constexpr size_t smem_bytes(int E, uint32_t rom_bytes, int ram_words) {
  return rom_bytes + 512 + 16 + (size_t)(ram_words + 40 + 6) * 4 * E;
}

__device__ __forceinline__ BlockSmem carve_smem(uint8_t* smem, int E, uint32_t rom_bytes, int ram_words) {
  BlockSmem b;
  b.rom = smem;
  b.dt = reinterpret_cast<DecodeTables*>(smem + rom_bytes);
  b.mbar = reinterpret_cast<uint64_t*>(smem + rom_bytes + 512);
  b.ram = reinterpret_cast<uint32_t*>(smem + rom_bytes + 512 + 16);
  b.line = b.ram + ram_words * E;
  b.tx = b.line + 40 * E;
  return b;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Stage the decode table (plain loads) and the cartridge image (one TMA bulk
// copy completing on an mbarrier).  Returns false if the copy did not land
// within the wait budget: the block then raises the device error word
// (*err = 1, which the host reports as VCS_ERR_WATCHDOG; the batch is then
// unusable), waits once more, again bounded, for the copy still in flight
// to this block's shared memory, and every thread leaves the kernel.
__device__ __forceinline__ bool stage_block(const BlockSmem& b, const DecodeTables* dt, const uint8_t* src,
                                            uint32_t bytes, int32_t* err) {
  const uint32_t bar = smem_addr(b.mbar);
  for (int i = threadIdx.x; i < (int)(sizeof(DecodeTables) / 4); i += blockDim.x)
    reinterpret_cast<uint32_t*>(b.dt)[i] = reinterpret_cast<const uint32_t*>(dt)[i];
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(b.rom)),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
  }
  auto wait = [&](uint32_t polls) {
    uint32_t done = 0;
    for (uint32_t spin = 0; spin < polls && !done; spin++) {
      asm volatile(
          "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
          : "=r"(done)
          : "r"(bar)
          : "memory");
    }
    return done != 0;
  };
  const bool done = wait(1u << 24);
  if (!done) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    (void)wait(1u << 24);   // let the copy in flight land before the block's shared memory is released
  }
  __syncthreads();
  return done;
}

// Context of one replica: env slot `slot` of the block (E envs), replica
// `rank` of T, of a cart whose bank byte is cb (banks | kCartSC | kCartE0).
// XM: the batch may hold Superchip or E0 carts; without it their ports and
// slices are compiled out.  FT: the whole TIA (compiled out without it).
template <bool XM, bool FT>
__device__ __forceinline__ Ctx make_ctx(const BlockSmem& b, int E, int slot, int rank, int T, uint32_t cb,
                                        int32_t ystart) {
  const uint32_t nb = cart_banks_of(cb);
  Ctx c;
  c.rom = b.rom;
  c.ram = reinterpret_cast<uint8_t*>(b.ram + slot);
  c.line = b.line + slot;
  c.tx = b.tx + slot;
  c.dt = b.dt;
  c.e4 = 4u * (uint32_t)E;
  c.E = (uint32_t)E;
  c.nb = nb;
  c.fe = XM ? cart_is_fe(cb) : 0u;
  c.hot = c.fe ? 0xFFFFu : first_hotspot(nb);
  c.sc = XM ? cart_is_sc(cb) : 0u;
  c.e0 = XM ? cart_is_e0(cb) : 0u;
  c.rw = c.sc ? 64u : 32u;
  c.ft = FT ? 1u : 0u;
  c.ystart = ystart;
  c.rank = (uint32_t)rank;
  c.T = (uint32_t)T;
  const uint32_t lane = threadIdx.x & 31;
  c.gmask = ((1u << T) - 1u) << (lane & ~(uint32_t)(T - 1));
  c.fp = nullptr;
  return c;
}

__device__ __forceinline__ void load_env(const SoA& s, int n, int e, const Ctx& c, Regs& r) {
  uint32_t v = s.reg[e];
  r.A = v & 0xFF; r.X = (v >> 8) & 0xFF; r.Y = (v >> 16) & 0xFF; r.SP = v >> 24;
  v = s.pcp[e];
  r.PC = v & 0xFFFF;
  unpack_p(r, (v >> 16) & 0xFF);
  r.jam = (v >> 24) & 1;
  r.cyc = s.cyc[e];
  v = s.fcs[e];
  r.fc = (int32_t)(v & 0xFFFF);
  r.fs = v >> 16;
  r.tw = s.tw[e];
  v = s.tv[e];
  r.tv = v & 0xFF; r.tsh = (v >> 8) & 0xFF; r.bank = v >> 16;
  v = s.t0[e];
  r.col0 = v & 0xFF; r.colpf = (v >> 8) & 0xFF; r.colbk = (v >> 16) & 0xFF; r.ctrl = v >> 24;
  v = s.t1[e];
  r.pf0 = v & 0xFF; r.pf1 = (v >> 8) & 0xFF; r.pf2 = (v >> 16) & 0xFF; r.grp0 = v >> 24;
  v = s.t2[e];
  r.hmp0 = v & 0xFF; r.pos = (v >> 8) & 0xFF; r.vblank = (v >> 16) & 0xFF; r.vsync = v >> 24;
  r.hml = (int32_t)s.t3[e];
  r.xo = r.cx = 0;
  r.cxc = 0;
  if (c.ft) {
    for (uint32_t k = 0; k < 4; k++) tx_wr(c, k, s.tx[(size_t)k * n + e]);
    r.cx = s.cx[e];
    r.cxc = (int32_t)s.cxc[e];
    cold_summary(c, r);
    mirror_hot(c, r);
  }
  uint32_t* w = reinterpret_cast<uint32_t*>(c.ram);
  for (uint32_t i = 0; i < c.rw; i++) w[i * c.E] = s.ram[(size_t)i * n + e];
  for (uint32_t q = c.rank; q < 10; q += c.T)
    for (uint32_t k = 0; k < 4; k++) c.line[(4 * q + k) * c.E] = 0;
  __syncwarp(c.gmask);
}

__device__ __forceinline__ void store_env(const SoA& s, int n, int e, const Ctx& c, const Regs& r) {
  s.reg[e] = r.A | (r.X << 8) | (r.Y << 16) | (r.SP << 24);
  s.pcp[e] = r.PC | (pack_p(r) << 16) | (r.jam << 24);
  s.cyc[e] = r.cyc;
  s.fcs[e] = ((uint32_t)r.fc & 0xFFFF) | (r.fs << 16);
  s.tw[e] = r.tw;
  s.tv[e] = r.tv | (r.tsh << 8) | (r.bank << 16);
  s.t0[e] = r.col0 | (r.colpf << 8) | (r.colbk << 16) | (r.ctrl << 24);
  s.t1[e] = r.pf0 | (r.pf1 << 8) | (r.pf2 << 16) | (r.grp0 << 24);
  s.t2[e] = r.hmp0 | (r.pos << 8) | (r.vblank << 16) | (r.vsync << 24);
  s.t3[e] = (uint32_t)r.hml;
  if (c.ft) {
    for (uint32_t k = 0; k < 4; k++) s.tx[(size_t)k * n + e] = tx_rd(c, k);
    s.cx[e] = r.cx & 0xFFFFu;
    s.cxc[e] = (uint32_t)r.cxc;
  }
  const uint32_t* w = reinterpret_cast<const uint32_t*>(c.ram);
  for (uint32_t i = 0; i < c.rw; i++) s.ram[(size_t)i * n + e] = w[i * c.E];
}

// Power-on state: A = X = Y = 0, SP = $FD, P = $34, RAM (and the
// Superchip's RAM) and TIA zero, timer as if 0 had been written to T1024T at
// cycle 0, banked carts in their last bank (FE in its first), E0 segments
// 0..2 showing slices 4, 5, 6, PC from the reset vector.
__device__ __forceinline__ void power_on(const Ctx& c, Regs& r) {
  r.A = r.X = r.Y = 0;
  r.SP = 0xFD;
  unpack_p(r, 0x34);
  r.bank = c.e0 ? (4u | 5u << 3 | 6u << 6) : (c.nb && !c.fe ? c.nb - 1u : 0u);
  r.jam = 0;
  r.cyc = 0;
  r.fc = 0;
  r.fs = 0;
  r.tw = 0; r.tv = 0; r.tsh = 10;
  r.col0 = r.colpf = r.colbk = r.ctrl = r.pf0 = r.pf1 = r.pf2 = r.grp0 = r.hmp0 = 0;
  r.pos = 0; r.vblank = 0; r.vsync = 0;
  r.hml = -1;
  r.xo = r.cx = 0;
  r.cxc = 0;
  if (c.ft) {
    for (uint32_t k = 0; k < 4; k++) tx_wr(c, k, 0u);
    cold_summary(c, r);
    mirror_hot(c, r);
  }
  uint32_t* w = reinterpret_cast<uint32_t*>(c.ram);
  for (uint32_t i = 0; i < c.rw; i++) w[i * c.E] = 0;
  r.PC = c.rom[rom_off(c, r, 0x1FFC)] | ((uint32_t)c.rom[rom_off(c, r, 0x1FFD)] << 8);
}

// ALE action -> joystick bits: bit0 right, bit1 left, bit2 down, bit3 up,
// bit4 fire (ALE action order NOOP, FIRE, UP, RIGHT, LEFT, DOWN, UPRIGHT,
// UPLEFT, DOWNRIGHT, DOWNLEFT, then the same eight with FIRE).
__device__ __forceinline__ uint32_t action_bits(uint32_t action) {
  // direction bits of actions 2..9 (and 10..17), one byte each
  const uint64_t t0 = 0x06050A0904020108ull;    // actions 2..9 (R,L,D,U bits), low byte = action 2
  uint32_t dir = 0, fire = 0;
  if (action == 1) fire = 1;
  else if (action >= 2 && action <= 9) dir = (uint32_t)(t0 >> (8 * (action - 2))) & 0xF;
  else if (action >= 10 && action <= 17) {
    fire = 1;
    dir = (uint32_t)(t0 >> (8 * (action - 10))) & 0xF;
  }
  return dir | (fire << 4);
}

// Joystick bits (bit0 right, bit1 left, bit2 down, bit3 up, bit4 fire) ->
// SWCHA and INPT4.
__device__ __forceinline__ void set_input_bits(Regs& r, uint32_t b) {
  // SWCHA player-0 nibble, active low: bit7 right, bit6 left, bit5 down, bit4 up
  r.swcha = 0xFFu - (((b & 1) << 7) | (((b >> 1) & 1) << 6) | (((b >> 2) & 1) << 5) | (((b >> 3) & 1) << 4));
  r.inpt4 = (b & 0x10) ? 0x00u : 0x80u;   // and the RESET switch released
}

__device__ __forceinline__ void set_inputs(Regs& r, uint32_t action) { set_input_bits(r, action_bits(action)); }

template <class Tape>
__device__ __forceinline__ void frame_end(const Ctx& c, Regs& r, Render& rd, Step& st, Tape& tape, int32_t fcw) {
  if (rd.on) {
    if constexpr (kDefers<Tape>) {   // the raster kernel draws it
      raster_end(tape, 3 * fcw);
    } else {
      finish_frame(c, r, rd, tape, 3 * fcw);
    }
    rd.on = false;
  }
  if (c.ft) cx_catchup(c, r, 3 * fcw);   // collisions up to the frame end, then in the new frame's clocks
  st.frames_done++;
  int32_t l = (int32_t)div76((uint32_t)fcw);
  r.fc -= 76 * l;
  r.fs = (uint32_t)(fcw - 76 * l);
  if (c.ft) r.cxc = 3 * (int32_t)r.fs;
  r.hml = -1;
  if (st.want_screen && st.frames_done == st.frame_skip - 1) {
    rd.on = true;
    rd.cur = 3 * (int32_t)r.fs;
    if constexpr (kDefers<Tape>) raster_begin(c, r, rd, tape);
  }
}

// Run instruction slots until `frame_skip` frames have ended, or, for
// instruction-granular steps (INSTR), until the step's slots have run.
//
// Warp scheduling.  Envs of one cart run the same program, but after a
// data-dependent branch or a timer poll loop they sit at different points of
// it, and plain SIMT execution never brings them back together: every
// iteration would then serialise over the lanes' different opcodes.  Each
// iteration the warp therefore picks which lanes execute:
//  - policy 0 (program order): the lanes in the earliest frame at the lowest
//    program counter.  Lanes that skipped code wait at the join point while
//    the others catch up, so they meet at the same instruction again.
//  - policy 1 (emulated time): the lanes whose step-relative time is within
//    `window` cycles of the earliest lane's.
// The chosen lanes then run to the end of their basic block (exec_one says
// when an instruction can change control flow).  Each lane's emulation is
// independent, so the order changes no result.
// `lanes` is the mask of the warp's launched lanes; inactive lanes only take
// part in the reduction.
template <bool INSTR = false, class Tape>
__device__ __forceinline__ void run_frames(const Ctx& c, Regs& r, Render& rd, Step& st, Tape& tape, bool active,
                                           uint32_t lanes, uint32_t policy, uint32_t window) {
  // INSTR: the step is st.instr_left instruction slots (frames end inside it
  // as they come); otherwise st.frame_skip frames, and the slot budget that
  // caps the timer-poll skip is unbounded
  st.frames_done = 0;
  st.stall = 0;
  st.fe_at = -1;
  if constexpr (!INSTR) st.instr_left = 0x7FFFFFFF;
  rd.on = active && st.want_screen && st.frame_skip == 1;
  rd.cur = 3 * (int32_t)r.fs;
  if constexpr (kDefers<Tape>) {
    if (rd.on) raster_begin(c, r, rd, tape);
  }
  uint32_t pf = prefetch(c, r);
  while (true) {
    const bool live = active && (INSTR ? st.instr_left > 0 : st.frames_done < st.frame_skip);
    const uint32_t pos = policy == 0 ? (r.jam ? 0xFFFFu : r.PC) : (uint32_t)r.fc;
    const uint32_t key = live ? (((uint32_t)st.frames_done << 16) | pos) : 0xFFFFFFFFu;
    const uint32_t kmin = __reduce_min_sync(lanes, key);
    if (kmin == 0xFFFFFFFFu) break;
    if (key - kmin > (policy == 0 ? 0u : window)) continue;
    // run the chosen lanes up to the end of their basic block: instructions
    // that cannot change control flow leave lanes that were together at the
    // same next instruction, so they need no new choice
    bool more;
    do {
      more = exec_one(c, r, rd, st, tape, pf);
      if constexpr (INSTR) more = (--st.instr_left > 0) && more;
      if ((st.fe_at >= 0) | (r.fc >= kLineCap * kLineCycles)) {   // VSYNC frame end, else the watchdog
        const bool dog = st.fe_at < 0;
        frame_end(c, r, rd, st, tape, dog ? r.fc : st.fe_at);
        st.fe_at = -1;
        if (dog) st.status |= kStWatchdog;
        more = false;
      }
    } while (more);
  }
  if (active && r.jam) st.status |= kStJammed;
}

__device__ __forceinline__ uint32_t warp_lanes(int E) {
  return E >= 32 ? 0xFFFFFFFFu : ((1u << E) - 1u);
}

// Keep the timer's elapsed count small once it has long underflowed, without
// changing any value it can read (past underflow only k mod 256 matters).
__device__ __forceinline__ void normalise_timer(Regs& r) {
  uint32_t k = r.cyc - r.tw, vi = r.tv << r.tsh;
  if (k > vi + 512u) r.tw += ((k - vi - 256u) & ~255u);
}

__device__ __forceinline__ void write_ram_f32(const Ctx& c, float* dst) {
  const uint32_t* w = reinterpret_cast<const uint32_t*>(c.ram);
  float4* d4 = reinterpret_cast<float4*>(dst);
  for (uint32_t q = c.rank; q < 32; q += c.T) {
    uint32_t v = w[q * c.E];
    d4[q] = make_float4((float)(v & 0xFF), (float)((v >> 8) & 0xFF), (float)((v >> 16) & 0xFF), (float)(v >> 24));
  }
}

__device__ __forceinline__ void write_ram(const Ctx& c, uint8_t* dst8) {
  uint4* dst = reinterpret_cast<uint4*>(dst8);
  const uint32_t* w = reinterpret_cast<const uint32_t*>(c.ram);
#pragma unroll
  for (uint32_t q = 0; q < 8; q++)
    if (owns_chunk(c, q))
      dst[q] = make_uint4(w[(4 * q) * c.E], w[(4 * q + 1) * c.E], w[(4 * q + 2) * c.E], w[(4 * q + 3) * c.E]);
}

}  // namespace vcs
