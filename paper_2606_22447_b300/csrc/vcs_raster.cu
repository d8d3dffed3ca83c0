// Deferred rasterisation: the hard step kernel's instantiations that log the
// returned frame instead of drawing it, and the raster kernel that draws
// every scanline of every env from the logs in parallel (the log and header
// formats are in vcs_machine.cuh).
//
// Why: one lane interprets one env, and the step time is that lane's chain
// of dependent instructions; drawing the returned frame inside that chain
// cost about an eighth of it.  Scanlines are independent once the register
// state at each line start is known, so they are drawn here with a warp per
// env: the warp first walks the env's log 32 entries at a time (warp ballots
// find each register's last writer) to record each screen row's starting
// registers and first entry in shared memory, then
// each lane draws whole rows with the interpreter's own span renderer and
// stores them as ten 16-byte words.
#include <cuda_runtime.h>

#include "vcs_step.cuh"

namespace vcs {

int launch_step_dr(const StepParams& p, int n_blocks, int E, void* stream) {
  // the whole TIA's kernels take every cartridge format
  if (p.full_tia) return launch_run_dr<true, true>(p, n_blocks, E, stream);
  return p.xmap ? launch_run_dr<true, false>(p, n_blocks, E, stream) : launch_run_dr<false, false>(p, n_blocks, E, stream);
}

constexpr int kRasterWarps = 4;   // envs per block

// Per screen row: the ten drawing registers when the row starts (bytes 0..9
// in the order of header words 3..5: COLUP0, COLUPF, COLUBK, CTRLPF, PF0, PF1,
// PF2, GRP0, player 0's position, VBLANK) and the row's first log entry
// (bytes 10..11; a log holds at most kRasterLogCap < 2^16 entries).  12 bytes
// a row and 160 bytes of line buffer a lane keep a warp under 7.7 KB, so 28
// warps fit an SM and 4096 envs run in one wave.
struct RasterSmem {
  uint32_t line[kRasterWarps][40][32];           // line buffers: word g of lane l at [g][l]
  uint32_t row[kRasterWarps][kScreenH][3];
};
static_assert(kRasterLogCap < 65536, "row starts are 16-bit");

// Log register of each walked register (HMOVE also moves player 0).
__device__ __forceinline__ bool walk_match(uint32_t reg, int k) {
  constexpr uint8_t regs[10] = {0x06, 0x08, 0x09, 0x0A, 0x0D, 0x0E, 0x0F, 0x1B, 0x10, 0x01};
  return reg == regs[k] || (k == 8 && reg == 0x2A);
}

// entries: when non-null, the log entries drawn are added to it (kernel
// timing's count of the bytes read).
__global__ void __launch_bounds__(32 * kRasterWarps) k_raster(const uint32_t* hdr, const uint32_t* log,
                                                               int32_t n_envs, int32_t ystart, uint8_t* screen,
                                                               unsigned long long* entries) {
  __shared__ RasterSmem sm;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int env = blockIdx.x * kRasterWarps + w;
  if (env >= n_envs) return;   // whole warps leave together
  const uint32_t* h = hdr + (size_t)env * kRasterHdr;
  const uint32_t n = h[0];
  if (entries && lane == 0) atomicAdd(entries, (unsigned long long)n);
  const int32_t start = (int32_t)h[1], end = (int32_t)h[2];
  const uint32_t* lg = log + (size_t)env * kRasterLogCap;
  const uint32_t below = (1u << lane) - 1u;

  // Walk the log 32 entries at a time.  Row r starts with the registers left
  // by every entry before its first colour clock 228 (ystart + r); an entry
  // at exactly that clock belongs to the row (it takes effect before the
  // row's first pixel).  Lane j holds entry j of the chunk; for each register
  // a ballot finds the last lane below j that writes it, so each lane knows
  // the registers just before its entry, and records the rows its entry
  // opens (the rows after the previous entry's row, up to its own).  The
  // early-HMOVE line needs no snapshot: at a row's start it names an earlier
  // line, which does not blank this one.
  uint32_t carry[10];
#pragma unroll
  for (int k = 0; k < 10; k++) carry[k] = (h[3 + k / 4] >> (8 * (k & 3))) & 0xFF;
  int32_t next = 0;   // first row not yet recorded
  auto put_row = [&](int32_t r, const uint32_t* v, uint32_t first) {
    uint32_t* d = sm.row[w][r];
    d[0] = v[0] | (v[1] << 8) | (v[2] << 16) | (v[3] << 24);
    d[1] = v[4] | (v[5] << 8) | (v[6] << 16) | (v[7] << 24);
    d[2] = v[8] | (v[9] << 8) | (first << 16);
  };
  for (uint32_t j0 = 0; j0 < n && next < kScreenH; j0 += 32) {
    const bool valid = j0 + lane < n;
    const uint32_t e = valid ? lg[j0 + lane] : 0xFFFFFFFFu;
    const uint32_t reg = (e >> 8) & 0x3F;
    const int32_t line = valid ? (int32_t)div228(3 * (e >> 16)) : 0x7FFFFFF;
    int32_t mine = line - ystart;                 // the row this entry falls in
    mine = mine < -1 ? -1 : (mine > kScreenH ? kScreenH : mine);
    int32_t prev = __shfl_up_sync(0xFFFFFFFFu, mine, 1);
    if (lane == 0) prev = next - 1;
    uint32_t v[10];
#pragma unroll
    for (int k = 0; k < 10; k++) {
      const uint32_t writers = __ballot_sync(0xFFFFFFFFu, valid && walk_match(reg, k));
      const uint32_t before = writers & below;
      const uint32_t src = before ? 31u - __clz(before) : 0u;
      const uint32_t got = __shfl_sync(0xFFFFFFFFu, e & 0xFF, (int)src);
      v[k] = before ? got : carry[k];
      carry[k] = writers ? __shfl_sync(0xFFFFFFFFu, e & 0xFF, 31 - __clz(writers)) : carry[k];
    }
    // rows (prev, mine] inside the screen open at this entry
    const int32_t r0 = prev + 1 > next ? prev + 1 : next;
    for (int32_t r = r0; valid && r <= mine && r < kScreenH; r++) put_row(r, v, j0 + lane);
    const int32_t hi = __reduce_max_sync(0xFFFFFFFFu, valid ? mine : -1);
    next = hi + 1 > next ? hi + 1 : next;
  }
  // rows after the last entry keep the final registers
  for (int32_t r = next + lane; r < kScreenH; r += 32) put_row(r, carry, n);
  __syncwarp();

  // Draw rows lane, lane + 32, ...: the colour clocks of the row inside the
  // frame, the row's entries applied at their clocks, into the lane's line
  // buffer, then one 160-byte store.  A row the frame covers from before its
  // first visible column to its end is written whole by the spans; the
  // others are zeroed first (where the frame drew nothing).
  Ctx c{};
  c.line = &sm.line[w][0][lane];
  c.E = 32;
  c.ft = 0;
  c.rank = 0;
  c.T = 1;
  c.gmask = 1u << lane;
  c.ystart = ystart;
  Render rd{};
  NoTape nt;
  Regs r{};
  uint8_t* out = screen + (size_t)env * (kScreenH * kScreenW);
  for (uint32_t rr = (uint32_t)lane; rr < (uint32_t)kScreenH; rr += 32) {
    const uint32_t* sn = sm.row[w][rr];
    raster_restore(r, sn[0], sn[1], sn[2] & 0xFFFF, 0xFFFFFFFFu);
    const uint32_t j0 = sn[2] >> 16, j1 = rr + 1 < (uint32_t)kScreenH ? sm.row[w][rr + 1][2] >> 16 : n;
    const int32_t line = ystart + (int32_t)rr, lbeg = 228 * line, lend = lbeg + 228;
    int32_t cur = start > lbeg ? start : lbeg;
    const int32_t stop = end < lend ? end : lend;
    if (cur > lbeg + 68 || stop < lend) {
#pragma unroll
      for (uint32_t g = 0; g < 40; g++) c.line[g * 32] = 0u;
    }
    auto draw = [&](int32_t to) {
      if (to > stop) to = stop;
      if (to <= cur) return;
      const int32_t h0 = cur - lbeg, h1 = to - lbeg;
      const uint32_t x0 = (uint32_t)(h0 > 68 ? h0 : 68) - 68u, x1 = (uint32_t)(h1 > 68 ? h1 : 68) - 68u;
      if (x1 > x0) render_span(c, r, rd, nt, x0, x1, line);
      cur = to;
    };
    // the row's entries, four loads in flight at a time
    for (uint32_t j = j0; j < j1; j += 4) {
      uint32_t q[4];
#pragma unroll
      for (uint32_t k = 0; k < 4; k++) q[k] = j + k < j1 ? lg[j + k] : 0u;
#pragma unroll
      for (uint32_t k = 0; k < 4; k++) {
        if (j + k >= j1) break;
        draw(3 * (int32_t)(q[k] >> 16));
        raster_apply(r, q[k]);
      }
    }
    draw(stop);
    uint4* dst = reinterpret_cast<uint4*>(out + rr * kScreenW);
#pragma unroll
    for (uint32_t q = 0; q < 10; q++)
      dst[q] = make_uint4(c.line[(4 * q) * 32], c.line[(4 * q + 1) * 32], c.line[(4 * q + 2) * 32],
                          c.line[(4 * q + 3) * 32]);
  }
}

// ---------------------------------------------------------------------------
// The whole TIA.  Its logs hold the raw writes; a write's effect depends on
// other registers (HMOVE on every motion register, GRP0 and GRP1 on each
// other's delayed copies, missile locks on the players' positions), so the
// walk replays them in order with the interpreter's own functions (tia_hot,
// tia_write_cold) rather than by ballots: every lane of the warp replays the
// same writes on the same registers (the entries fetched 32 at a time and
// broadcast).  Rows go in groups of 32: the walk runs to the start of the
// group's last row, lane l keeping row 32 g + l's starting state (the
// drawing registers, HMP0, the four cold words, its first entry) in its own
// registers as the walk passes it, and then every lane draws its row,
// replaying the row's writes on its own copy of the cold words, before the
// walk goes on.  Keeping the rows' states in registers leaves 5.8 KB of
// shared memory per warp (36 warps an SM).
// ---------------------------------------------------------------------------
constexpr int kRasterFtWarps = 4;   // envs per block

struct RasterFtSmem {
  uint32_t line[kRasterFtWarps][40][32];      // line buffers: word g of lane l at [g][l]
  uint32_t tx[kRasterFtWarps][6][32];         // each lane's cold words (stride 32)
  uint32_t walk[kRasterFtWarps][6];           // the walk's cold words (stride 1)
};

// Replay one logged write of the whole TIA on r and the cold words at tx
// (stride E).
__device__ __forceinline__ void raster_replay(Regs& r, uint32_t* tx, uint32_t E, uint32_t e) {
  const uint32_t fcw = e >> 16, reg = (e >> 8) & 0x3F, v = e & 0xFF;
  const uint32_t line = div76(fcw), h = 3u * (fcw - 76u * line);
  tia_hot(r, reg, v, line, h);
  if (cold_write(reg, r.xo)) {
    const uint2 o = tia_write_cold(tx, E, reg, v, h, r.grp0, r.pos, r.cx);
    r.xo = o.x;
    r.cx = o.y;
  }
}

__global__ void __launch_bounds__(32 * kRasterFtWarps, 8) k_raster_ft(const uint32_t* hdr, const uint32_t* log,
                                                                     int32_t n_envs, int32_t ystart, uint8_t* screen,
                                                                     unsigned long long* entries) {
  __shared__ RasterFtSmem sm;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int env = blockIdx.x * kRasterFtWarps + w;
  if (env >= n_envs) return;   // whole warps leave together
  const uint32_t* h = hdr + (size_t)env * kRasterHdr;
  const uint32_t n = h[0];
  if (entries && lane == 0) atomicAdd(entries, (unsigned long long)n);
  const int32_t start = (int32_t)h[1], end = (int32_t)h[2];
  const uint32_t* lg = log + (size_t)env * kRasterLogCap;

  // the walk's state: rows start with the state left by every write before
  // their first colour clock (a write at exactly that clock belongs to the row)
  Regs r{};
  raster_restore(r, h[3], h[4], h[5] & 0xFFFF, 0xFFFFFFFFu);
  r.hmp0 = (h[5] >> 16) & 0xFF;
  uint32_t* tw = sm.walk[w];
  if (lane == 0)
    for (int k = 0; k < 4; k++) tw[k] = h[7 + k];
  __syncwarp();
  r.cx = 0;
  r.xo = cold_summary_of(tw[0], tw[1], tw[2], 0).x;

  Ctx c{};
  c.line = &sm.line[w][0][lane];
  c.tx = &sm.tx[w][0][lane];
  c.E = 32;
  c.ft = 1;
  c.rank = 0;
  c.T = 1;
  c.gmask = 1u << lane;
  c.ystart = ystart;
  Render rd{};
  NoTape nt;
  uint8_t* out = screen + (size_t)env * (kScreenH * kScreenW);

  uint32_t row = 0, j = 0, j0 = 0xFFFFFFFFu, mine = 0;
  uint32_t s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0, s6 = 0, sfirst = 0;   // this lane's row's start
  auto record = [&]() {   // the walk's state opens row `row`
    if ((uint32_t)lane == (row & 31u)) {
      s0 = (r.col0 & 0xFF) | ((r.colpf & 0xFF) << 8) | ((r.colbk & 0xFF) << 16) | ((r.ctrl & 0xFF) << 24);
      s1 = (r.pf0 & 0xFF) | ((r.pf1 & 0xFF) << 8) | ((r.pf2 & 0xFF) << 16) | ((r.grp0 & 0xFF) << 24);
      s2 = (r.pos & 0xFF) | ((r.vblank & 0xFF) << 8) | ((r.hmp0 & 0xFF) << 16);
      s3 = tw[0];
      s4 = tw[1];
      s5 = tw[2];
      s6 = tw[3];
      sfirst = j;
    }
    row++;
  };
  for (uint32_t g0 = 0; g0 < (uint32_t)kScreenH; g0 += 32) {
    const uint32_t gend = g0 + 32 < (uint32_t)kScreenH ? g0 + 32 : (uint32_t)kScreenH;
    // walk to the start of the group's last row
    while (row < gend) {
      if (j >= n) {
        record();
        continue;
      }
      if ((j & ~31u) != j0) {   // the next 32 entries, one a lane
        j0 = j & ~31u;
        mine = j0 + lane < n ? lg[j0 + lane] : 0u;
      }
      const uint32_t e = __shfl_sync(0xFFFFFFFFu, mine, (int)(j & 31u));
      const int32_t cc = 3 * (int32_t)(e >> 16);
      while (row < gend && cc >= 228 * (ystart + (int32_t)row)) record();
      if (row >= gend) break;   // entry j belongs to a later row: the walk resumes there
      __syncwarp();
      raster_replay(r, tw, 1, e);   // every lane writes the same words
      __syncwarp();
      j++;
    }
    // draw row g0 + lane from its start, through its entries
    const uint32_t rr = g0 + (uint32_t)lane;
    if (rr < gend) {
      Regs q{};
      raster_restore(q, s0, s1, s2 & 0xFFFF, 0xFFFFFFFFu);
      q.hmp0 = (s2 >> 16) & 0xFF;
      c.tx[0] = s3;
      c.tx[32] = s4;
      c.tx[64] = s5;
      c.tx[96] = s6;
      q.cx = 0;
      q.xo = cold_summary_of(s3, s4, s5, 0).x;
      const int32_t line = ystart + (int32_t)rr, lbeg = 228 * line, lend = lbeg + 228;
      int32_t cur = start > lbeg ? start : lbeg;
      const int32_t stop = end < lend ? end : lend;
      if (cur > lbeg + 68 || stop < lend) {
#pragma unroll
        for (uint32_t g = 0; g < 40; g++) c.line[g * 32] = 0u;
      }
      auto draw = [&](int32_t to) {
        if (to > stop) to = stop;
        if (to <= cur) return;
        const int32_t h0 = cur - lbeg, h1 = to - lbeg;
        const uint32_t x0 = (uint32_t)(h0 > 68 ? h0 : 68) - 68u, x1 = (uint32_t)(h1 > 68 ? h1 : 68) - 68u;
        if (x1 > x0) render_span(c, q, rd, nt, x0, x1, line);
        cur = to;
      };
      for (uint32_t k = sfirst; k < n; k++) {   // the row's entries: up to the next row's first clock
        const uint32_t e = lg[k];
        const int32_t cc = 3 * (int32_t)(e >> 16);
        if (cc >= lend) break;
        draw(cc);
        raster_replay(q, c.tx, 32, e);
      }
      draw(stop);
      uint4* dst = reinterpret_cast<uint4*>(out + rr * kScreenW);
#pragma unroll
      for (uint32_t qq = 0; qq < 10; qq++)
        dst[qq] = make_uint4(c.line[(4 * qq) * 32], c.line[(4 * qq + 1) * 32], c.line[(4 * qq + 2) * 32],
                             c.line[(4 * qq + 3) * 32]);
    }
    __syncwarp();
  }
}

int launch_raster_ft(const uint32_t* hdr, const uint32_t* log, int32_t n_envs, int32_t ystart, uint8_t* screen,
                     unsigned long long* entries, void* stream) {
  if (n_envs <= 0) return 0;
  const int blocks = (n_envs + kRasterFtWarps - 1) / kRasterFtWarps;
  k_raster_ft<<<blocks, 32 * kRasterFtWarps, 0, (cudaStream_t)stream>>>(hdr, log, n_envs, ystart, screen, entries);
  return (int)cudaGetLastError();
}

int launch_raster(const uint32_t* hdr, const uint32_t* log, int32_t n_envs, int32_t ystart, uint8_t* screen,
                  unsigned long long* entries, void* stream) {
  if (n_envs <= 0) return 0;
  const int blocks = (n_envs + kRasterWarps - 1) / kRasterWarps;
  k_raster<<<blocks, 32 * kRasterWarps, 0, (cudaStream_t)stream>>>(hdr, log, n_envs, ystart, screen, entries);
  return (int)cudaGetLastError();
}

}  // namespace vcs
