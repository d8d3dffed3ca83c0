// Deferred rasterisation: the hard step kernel's instantiations that log the
// returned frame instead of drawing it, and the raster kernel that draws
// every scanline of every env from the logs in parallel (the log and header
// formats are in vcs_machine.cuh).
//
// Why: one lane interprets one env, and the step time is that lane's chain
// of dependent instructions; drawing the returned frame inside that chain
// cost about an eighth of it.  Scanlines are independent once the register
// state at each line start is known, so they are drawn here with a warp per
// env: the warp first walks the env's log once (every lane the same walk,
// the entries fetched 32 at a time and broadcast by shuffles) to record each
// screen row's starting registers and first entry in shared memory, then
// each lane draws whole rows with the interpreter's own span renderer and
// stores them as ten 16-byte words.
#include <cuda_runtime.h>

#include "vcs_step.cuh"

namespace vcs {

int launch_step_dr(const StepParams& p, int n_blocks, int E, void* stream) {
  return p.xmap ? launch_run_dr<true>(p, n_blocks, E, stream) : launch_run_dr<false>(p, n_blocks, E, stream);
}

constexpr int kRasterWarps = 4;   // envs per block

struct RasterSmem {
  uint32_t line[kRasterWarps][40][32];           // line buffers: word g of lane l at [g][l]
  uint8_t snap[kRasterWarps][kScreenH][12];      // registers at each screen row's start (header words 3..5)
  uint32_t first[kRasterWarps][kScreenH + 1];    // each row's first log entry
};

// The register lane k of the log walk follows, and its byte in a row's
// snapshot (header words 3..5): COLUP0, COLUPF, COLUBK, CTRLPF, PF0, PF1,
// PF2, GRP0, player 0's position (RESP0 and HMOVE), VBLANK.
__constant__ uint8_t kWalkReg[10] = {0x06, 0x08, 0x09, 0x0A, 0x0D, 0x0E, 0x0F, 0x1B, 0x10, 0x01};

__global__ void __launch_bounds__(32 * kRasterWarps) k_raster(const uint32_t* hdr, const uint32_t* log,
                                                               int32_t n_envs, int32_t ystart, uint8_t* screen) {
  __shared__ RasterSmem sm;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int env = blockIdx.x * kRasterWarps + w;
  if (env >= n_envs) return;   // whole warps leave together
  const uint32_t* h = hdr + (size_t)env * kRasterHdr;
  const uint32_t n = h[0];
  const int32_t start = (int32_t)h[1], end = (int32_t)h[2];
  const uint32_t* lg = log + (size_t)env * kRasterLogCap;

  // Walk the log once: row r starts with the registers left by every entry
  // before its first colour clock 228 (ystart + r); an entry at exactly that
  // clock belongs to the row (it takes effect before the row's first pixel).
  // Lane k < 10 follows register k alone, so an entry costs each lane one
  // compare and select; the entries are fetched 32 at a time and broadcast.
  // The early-HMOVE line needs no snapshot: at a row's start it names an
  // earlier line, which does not blank this one.
  const uint32_t myreg = lane < 10 ? kWalkReg[lane] : 0xFFu;
  const uint32_t alt = lane == 8 ? 0x2Au : 0xFFu;   // HMOVE moves player 0 too
  uint32_t val = lane < 10 ? (h[3 + lane / 4] >> (8 * (lane & 3))) & 0xFF : 0u;
  uint32_t row = 0;
  auto record = [&](uint32_t j) {
    if (lane < 10) sm.snap[w][row][lane] = (uint8_t)val;
    if (lane == 0) sm.first[w][row] = j;
    row++;
  };
  for (uint32_t j0 = 0; j0 < n && row < (uint32_t)kScreenH; j0 += 32) {
    const uint32_t mine = j0 + lane < n ? lg[j0 + lane] : 0u;
    const uint32_t m = n - j0 < 32u ? n - j0 : 32u;
    for (uint32_t k = 0; k < m; k++) {
      const uint32_t e = __shfl_sync(0xFFFFFFFFu, mine, (int)k);
      const int32_t cc = 3 * (int32_t)(e >> 16);
      while (row < (uint32_t)kScreenH && cc >= 228 * (ystart + (int32_t)row)) record(j0 + k);
      const uint32_t reg = (e >> 8) & 0x3F;
      val = (reg == myreg || reg == alt) ? e & 0xFF : val;
    }
  }
  while (row < (uint32_t)kScreenH) record(n);
  if (lane == 0) sm.first[w][kScreenH] = n;
  __syncwarp();

  // Draw rows lane, lane + 32, ...: the colour clocks of the row inside the
  // frame, the row's entries applied at their clocks, into the lane's line
  // buffer (zero where the frame drew nothing), then one 160-byte store.
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
    const uint32_t* sn = reinterpret_cast<const uint32_t*>(sm.snap[w][rr]);
    raster_restore(r, sn[0], sn[1], sn[2], 0xFFFFFFFFu);
    const int32_t line = ystart + (int32_t)rr, lbeg = 228 * line, lend = lbeg + 228;
    int32_t cur = start > lbeg ? start : lbeg;
    const int32_t stop = end < lend ? end : lend;
#pragma unroll
    for (uint32_t g = 0; g < 40; g++) c.line[g * 32] = 0u;
    auto draw = [&](int32_t to) {
      if (to > stop) to = stop;
      if (to <= cur) return;
      const int32_t h0 = cur - lbeg, h1 = to - lbeg;
      const uint32_t x0 = (uint32_t)(h0 > 68 ? h0 : 68) - 68u, x1 = (uint32_t)(h1 > 68 ? h1 : 68) - 68u;
      if (x1 > x0) render_span(c, r, rd, nt, x0, x1, line);
      cur = to;
    };
    const uint32_t j1 = sm.first[w][rr + 1];
    for (uint32_t j = sm.first[w][rr]; j < j1; j++) {
      const uint32_t e = lg[j];
      draw(3 * (int32_t)(e >> 16));
      raster_apply(r, e);
    }
    draw(stop);
    uint4* dst = reinterpret_cast<uint4*>(out + rr * kScreenW);
#pragma unroll
    for (uint32_t q = 0; q < 10; q++)
      dst[q] = make_uint4(c.line[(4 * q) * 32], c.line[(4 * q + 1) * 32], c.line[(4 * q + 2) * 32],
                          c.line[(4 * q + 3) * 32]);
  }
}

int launch_raster(const uint32_t* hdr, const uint32_t* log, int32_t n_envs, int32_t ystart, uint8_t* screen,
                  void* stream) {
  if (n_envs <= 0) return 0;
  const int blocks = (n_envs + kRasterWarps - 1) / kRasterWarps;
  k_raster<<<blocks, 32 * kRasterWarps, 0, (cudaStream_t)stream>>>(hdr, log, n_envs, ystart, screen);
  return (int)cudaGetLastError();
}

}  // namespace vcs
