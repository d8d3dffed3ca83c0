// Kernel-side declarations shared by the launchers and the C ABI.
#pragma once
#include <cstdint>

#include "vcs_machine.cuh"

namespace vcs {

// Struct-of-arrays machine state: each pointer is one field for all envs
// (u32 [n_envs]), so a warp's loads and stores of a field are coalesced.
struct SoA {
  uint32_t* reg;   // A | X << 8 | Y << 16 | SP << 24
  uint32_t* pcp;   // PC | P << 16 | jam << 24
  uint32_t* cyc;   // CPU cycles mod 2^32
  uint32_t* fcs;   // fc | fs << 16
  uint32_t* tw;    // timer write cycle
  uint32_t* tv;    // timer value | log2 interval << 8 | bank << 16 (E0: three 3-bit slices)
  uint32_t* t0;    // COLUP0 | COLUPF << 8 | COLUBK << 16 | CTRLPF << 24
  uint32_t* t1;    // PF0 | PF1 << 8 | PF2 << 16 | GRP0 << 24
  uint32_t* t2;    // HMP0 | P0 position << 8 | VBLANK << 16 | VSYNC << 24
  uint32_t* t3;    // scanline of the last early HMOVE (int32, -1 = none)
  uint32_t* epf;   // frames elapsed in the current episode
  uint32_t* epi;   // episode index
  uint32_t* tx;    // the cold TIA words [4][n_envs] (player 1, missiles, ball; vcs_tia.cuh)
  uint32_t* cx;    // collision latches (16 bits)
  uint32_t* cxc;   // colour clock (frame coordinates) up to which collisions are evaluated
  uint32_t* ram;   // RAM words [64][n_envs]: RIOT RAM, then the Superchip's RAM (zero for other carts)
};
constexpr int kSoAFields = 18;
constexpr int kStateWords = kSoAFields + 64;   // per env

// Per-cart bank byte: the 4 KB banks of a bank-switched cart (2, 4, 8; 0 for
// 2K, 4K and E0 images) | kCartSC for the Superchip variants | kCartE0 for
// E0 (eight 1 KB slices) | kCartFE for FE (2 banks chosen through JSR and
// RTS, no hotspot).
constexpr uint32_t kCartSC = 0x80, kCartE0 = 0x40, kCartFE = 0x20;
__host__ __device__ constexpr uint32_t cart_banks_of(uint32_t cb) { return cb & 0x0F; }
__host__ __device__ constexpr uint32_t cart_is_sc(uint32_t cb) { return cb >> 7; }
__host__ __device__ constexpr uint32_t cart_is_e0(uint32_t cb) { return (cb >> 6) & 1u; }
__host__ __device__ constexpr uint32_t cart_is_fe(uint32_t cb) { return (cb >> 5) & 1u; }
// Bytes of the device image a block stages (2K images are mirrored to 4 KB).
__host__ __device__ constexpr uint32_t cart_image_bytes(uint32_t cb) {
  return cart_is_e0(cb) ? 8192u : (cart_banks_of(cb) ? cart_banks_of(cb) * 4096u : 4096u);
}

struct StepParams {
  SoA s;
  int32_t n_envs;
  const int4* blocks;       // per block: {cart, first slot, env count, 0}
  const int32_t* perm;      // slot -> env (envs grouped by cart)
  const uint8_t* roms;      // [n_carts][rom_stride]; 2K images mirrored to 4 KB
  const uint8_t* cart_banks;  // [n_carts] bank byte: 4 KB banks of bank-switched carts (2, 4, 8), else 0,
                              // | kCartSC for a Superchip cart | kCartE0 for an E0 cart
  int32_t ram_words;        // RAM words per env in shared memory: 32, or 64 when a cart is Superchip
  int32_t xmap;             // the batch holds Superchip or E0 carts: launch the kernels built for them
  int32_t full_tia;         // the whole TIA (player 1, missiles, ball, collisions): its own kernels
  int32_t graphics;         // soft forward: count GRP0 / PF0-2 writes as versions (graphics-bit surrogate)
  uint32_t rom_stride;      // bytes per cart image (8, 16 or 32 KB): also the shared-memory ROM region
  const DecodeTables* dt;
  const uint8_t* actions;   // [n_steps][n_envs] or null (NOOP)
  int32_t n_steps;
  int32_t frame_skip;
  uint8_t* ram_out;         // [n_steps][n_envs][128] or null
  uint8_t* screen_out;      // [n_steps][n_envs][210][160] or null
  uint8_t* status_out;      // [n_steps][n_envs] or null
  const uint32_t* ep_len;   // [n_envs][n_episodes] or null
  int32_t n_episodes;
  int32_t ystart;
  const uint8_t* reset_mask;  // per env, or null
  int32_t reset_all;        // power on every env before stepping
  int32_t* err;             // device error word (nonzero after a failure)
  int32_t tpe;              // threads per env (1, 2, 4 or 8)
  int32_t boot_frames;      // nonzero if powered-on envs run a boot sequence
  int32_t boot_noop, boot_reset;   // boot: NOOP frames, then frames with RESET pressed
  const uint8_t* start_noops;      // [n_envs][n_start] NOOP frames starting each episode, or null
  int32_t n_start;
  int32_t step_instr;       // > 0: a step is this many instruction slots (not frames)
  uint32_t sched_policy;    // warp scheduling: 0 program order, 1 emulated time (run_frames)
  uint32_t sched_window;    // time window in cycles for policy 1
  // soft forward only
  const float* u;           // joystick inputs [n_steps][n_envs][5] (R, L, D, U, FIRE)
  const float* ram0;        // RAM at the start of the rollout [n_envs][128] or null
  uint8_t* act_bits;        // rounded joystick bits per step [n_steps][n_envs]
  float* ram_out_f;         // [n_steps][n_envs][128] or null
  float* screen_out_f;      // [n_steps][n_envs][210][160] or null
  uint32_t* ckpt;           // [n_segments][kStateWords][n_envs]
  int32_t seg_steps;        // steps per checkpoint segment
  uint32_t* seg_counts;     // [n_segments][2]: max instructions, max colour writes
  // deferred rasterisation (hard frame steps; vcs_machine.cuh): dr selects
  // the step kernel that draws nothing; with screens it logs the returned
  // frame (one step per launch) to dr_log / dr_hdr
  int32_t dr;
  uint32_t* dr_log;         // [n_envs][kRasterLogCap] log entries, or null without screens
  uint32_t* dr_hdr;         // [n_envs][kRasterHdr] headers
};

__host__ __device__ inline SoA soa_at(uint32_t* base, int32_t n_envs) {
  SoA s;
  const size_t n = (size_t)n_envs;
  s.reg = base; s.pcp = base + n; s.cyc = base + 2 * n; s.fcs = base + 3 * n; s.tw = base + 4 * n;
  s.tv = base + 5 * n; s.t0 = base + 6 * n; s.t1 = base + 7 * n; s.t2 = base + 8 * n; s.t3 = base + 9 * n;
  s.epf = base + 10 * n; s.epi = base + 11 * n; s.tx = base + 12 * n; s.cx = base + 16 * n;
  s.cxc = base + 17 * n; s.ram = base + kSoAFields * n;
  return s;
}

void build_decode_tables(DecodeTables* t);
size_t step_smem_bytes(int envs_per_block, uint32_t rom_stride, int ram_words);
int launch_cart_ram(const SoA& s, int32_t n_envs, uint8_t* out, void* stream);
int launch_int_peak(int sms, int32_t iters, uint32_t* sink, void* stream);
int launch_digest(const uint8_t* ram, const uint8_t* screen, uint64_t n_digests, uint64_t* out, void* stream);
// Launch the step kernel over `n_blocks` blocks of `envs_per_block`
// (soft = the SOFT-STE forward: float inputs / outputs and checkpoints).
int launch_step(const StepParams& p, int n_blocks, int envs_per_block, void* stream);
int launch_soft_forward(const StepParams& p, int n_blocks, int envs_per_block, void* stream);
// The same for batches with Superchip or E0 carts (p.xmap), and for
// batches with the whole TIA (p.full_tia; those kernels also take every
// cartridge format).
int launch_step_xm(const StepParams& p, int n_blocks, int envs_per_block, void* stream);
int launch_soft_forward_xm(const StepParams& p, int n_blocks, int envs_per_block, void* stream);
int launch_step_ft(const StepParams& p, int n_blocks, int envs_per_block, void* stream);
// The hard step kernel with deferred rasterisation (p.dr set; with screens one step),
// and the raster kernel that then draws the step's screens [n_envs][210][160]
// from the logs (vcs_raster.cu), adding the entries it draws to *entries
// when that is non-null.
int launch_step_dr(const StepParams& p, int n_blocks, int envs_per_block, void* stream);
int launch_raster(const uint32_t* hdr, const uint32_t* log, int32_t n_envs, int32_t ystart, uint8_t* screen,
                  unsigned long long* entries, void* stream);
int launch_raster_ft(const uint32_t* hdr, const uint32_t* log, int32_t n_envs, int32_t ystart, uint8_t* screen,
                     unsigned long long* entries, void* stream);
int launch_soft_forward_ft(const StepParams& p, int n_blocks, int envs_per_block, void* stream);

}  // namespace vcs
