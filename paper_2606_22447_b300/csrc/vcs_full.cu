// The fully relaxed forward (Section 4's temperature-limit bound, Theorem 2,
// and the supplement's forward bit-exactness study) and its C-ABI entry
// point vcs_full_divergence.
//
// The study runs two machines per env side by side, one instruction slot at
// a time, from the env's current state: the hard machine, which also counts
// the casts that would round off its values (probe), and the FULL machine,
// whose ROM and RAM reads by instructions are temperature-T reads cast back
// to bytes and whose conditional branches take the rounded blend of
// Eq. branch (the interpreter's FM template argument).  The first slot after
// which the two states differ (registers and flags, clocks, timer, TIA
// registers, bank, jam flag, RAM and a Superchip's RAM) is the env's first
// divergence.  One thread
// per env; the batch state is read, never written.
#include <cuda_runtime.h>

#include <cmath>

#include "vcs_api_internal.h"
#include "vcs_exec.cuh"
#include "vcs_kernels.cuh"
#include "vcs_run.cuh"

namespace vcs {

struct FullDivParams {
  SoA s;
  int32_t n_envs;
  const int4* blocks;
  const int32_t* perm;
  const uint8_t* roms;
  const uint8_t* cart_banks;  // bank byte per cart (banks | kCartSC | kCartE0)
  int32_t ram_words;          // RAM words per env in shared memory (32 or 64)
  int32_t full_tia;           // the whole TIA, or the subset machine
  const uint8_t* cart_2k;
  uint32_t rom_stride;
  const DecodeTables* dt;
  const uint8_t* actions;   // [n_envs] ALE actions held for the whole run, or null (NOOP)
  int32_t n_instr;
  int32_t ystart;
  int32_t* n_div;           // [n_envs]
  uint32_t* counts;         // [n_envs][4] or null
  uint8_t* ram_full;        // [n_envs][128] or null (the RIOT RAM)
  int32_t* err;
};

__host__ __device__ constexpr size_t full_smem_bytes(int E, uint32_t rom_stride, int ram_words) {
  return smem_bytes(E, rom_stride, ram_words) + (size_t)(ram_words + 6) * 4 * E + sizeof(FullParams);
}

__device__ __forceinline__ bool machines_differ(const Ctx& ch, const Regs& a, const Ctx& cf, const Regs& b) {
  bool d = a.A != b.A || a.X != b.X || a.Y != b.Y || a.SP != b.SP || a.PC != b.PC || pack_p(a) != pack_p(b) ||
           a.bank != b.bank || a.jam != b.jam || a.cyc != b.cyc || a.fc != b.fc || a.fs != b.fs ||
           a.tw != b.tw || a.tv != b.tv || a.tsh != b.tsh || a.col0 != b.col0 || a.colpf != b.colpf ||
           a.colbk != b.colbk || a.ctrl != b.ctrl || a.pf0 != b.pf0 || a.pf1 != b.pf1 || a.pf2 != b.pf2 ||
           a.grp0 != b.grp0 || a.hmp0 != b.hmp0 || a.pos != b.pos || a.vblank != b.vblank ||
           a.vsync != b.vsync || a.hml != b.hml;
  d = d || a.cx != b.cx || a.cxc != b.cxc;
  for (uint32_t w = 0; w < 4 && !d; w++) d = tx_rd(ch, w) != tx_rd(cf, w);
  const uint32_t* wa = reinterpret_cast<const uint32_t*>(ch.ram);
  const uint32_t* wb = reinterpret_cast<const uint32_t*>(cf.ram);
  for (uint32_t w = 0; w < ch.rw && !d; w++) d = wa[w * ch.E] != wb[w * cf.E];
  return d;
}

// One instruction slot of one machine, then the frame end it caused (a
// VSYNC write, else the scanline watchdog).
template <int FM>
__device__ __forceinline__ void full_slot(const Ctx& c, Regs& r, Render& rd, Step& st, NoTape& tape, uint32_t& pf) {
  exec_one<NoTape, FM>(c, r, rd, st, tape, pf);
  if ((st.fe_at >= 0) | (r.fc >= kLineCap * kLineCycles)) {
    frame_end(c, r, rd, st, tape, st.fe_at >= 0 ? st.fe_at : r.fc);
    st.fe_at = -1;
  }
}

__global__ void __launch_bounds__(128) k_full(FullDivParams p, FullParams fp0) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int E = blockDim.x, slot = threadIdx.x;
  BlockSmem bs = carve_smem(smem, E, p.rom_stride, p.ram_words);
  // the FULL machine's RAM [ram_words][E]
  uint32_t* ram_f = reinterpret_cast<uint32_t*>(smem + smem_bytes(E, p.rom_stride, p.ram_words));
  uint32_t* tx_f = ram_f + p.ram_words * E;   // and its cold TIA words [6][E]
  FullParams* fp = reinterpret_cast<FullParams*>(tx_f + 6 * E);
  const int4 bi = p.blocks[blockIdx.x];
  const int cart = bi.x;
  const uint32_t cb = p.cart_banks[cart];
  if (slot == 0) {
    *fp = fp0;
    fp->rom_m = p.cart_2k[cart] ? 2048 : (cart_is_e0(cb) ? 1024 : 4096);
  }
  if (!stage_block(bs, p.dt, p.roms + (size_t)cart * p.rom_stride, cart_image_bytes(cb), p.err)) return;   // synchronises the block
  if (slot >= bi.z) return;
  const int env = p.perm[bi.y + slot];
  const int n = p.n_envs;
  // the study is not a hot path: one instantiation serves every batch, the
  // Superchip ports and E0 slices decoded at run time (off for other carts)
  Ctx ch = make_ctx<true, true>(bs, E, slot, 0, 1, cb, p.ystart);
  ch.ft = (uint32_t)p.full_tia;   // decided at run time here
  ch.fp = fp;
  Ctx cf = ch;
  cf.ram = reinterpret_cast<uint8_t*>(ram_f + slot);
  cf.tx = tx_f + slot;
  Regs rh;
  load_env(p.s, n, env, ch, rh);
  for (uint32_t w = 0; w < ch.rw; w++) ram_f[w * E + slot] = reinterpret_cast<const uint32_t*>(ch.ram)[w * E];
  for (uint32_t w = 0; w < 6; w++) tx_f[w * E + slot] = tx_rd(ch, w);
  set_inputs(rh, p.actions ? p.actions[env] : 0u);
  rh.fr_reads = rh.fr_exact = rh.fr_br = rh.fr_br_exact = 0;
  Regs rf = rh;
  Render rdh, rdf;
  rdh.on = rdf.on = false;
  rdh.cur = rdf.cur = 0;
  rdh.out_u8 = rdf.out_u8 = nullptr;
  rdh.out_f32 = rdf.out_f32 = nullptr;
  rdh.gs = rdf.gs = nullptr;
  rdh.grow = rdf.grow = nullptr;
  rdh.gline = rdf.gline = -1;
  Step sh;
  sh.frames_done = 0;
  sh.frame_skip = 1;
  sh.stall = 0;
  sh.fe_at = -1;
  sh.status = 0;
  sh.want_screen = false;
  sh.instr_left = 0x7FFFFFFF;
  Step sf = sh;
  NoTape tape;
  uint32_t pfh = prefetch(ch, rh), pff = prefetch(cf, rf);
  rh.pfr = prefetch_relaxed(ch, rh, pfh);
  rf.pfr = prefetch_relaxed(cf, rf, pff);
  int32_t ndiv = 0;
  for (int32_t k = 1; k <= p.n_instr; k++) {
    full_slot<1>(ch, rh, rdh, sh, tape, pfh);
    full_slot<2>(cf, rf, rdf, sf, tape, pff);
    if (ndiv == 0 && machines_differ(ch, rh, cf, rf)) ndiv = k;
  }
  p.n_div[env] = ndiv;
  if (p.counts) {
    uint32_t* o = p.counts + (size_t)env * 4;
    o[0] = rh.fr_reads;
    o[1] = rh.fr_exact;
    o[2] = rh.fr_br;
    o[3] = rh.fr_br_exact;
  }
  if (p.ram_full) write_ram(cf, p.ram_full + (size_t)env * 128);
}

}  // namespace vcs

using namespace vcs;

extern "C" vcs_status vcs_full_divergence(vcs_batch* b, float T, float alpha, const uint8_t* actions,
                                          int32_t n_instr, int32_t* n_div, uint32_t* counts, uint8_t* ram_full,
                                          void* stream) {
  if (!b) return VCS_ERR_ARG;
  if (!n_div) return vcs_fail(b, VCS_ERR_ARG, "n_div is NULL");
  if (!(T > 0.f) || !(T <= 10.f)) return vcs_fail(b, VCS_ERR_ARG, "T must be in (0, 10]");
  if (!std::isfinite(alpha) || n_instr < 0) return vcs_fail(b, VCS_ERR_ARG, "alpha finite and n_instr >= 0 required");
  FullParams fp{};
  const int W = (int)std::ceil(12.0 * (double)T);
  fp.W = W < 1 ? 1 : W;
  for (int k = 0; k <= fp.W; k++) fp.ek[k] = (float)std::exp(-(double)k / (double)T);
  fp.g1 = (float)(1.0 / (1.0 + std::exp(-(double)alpha)));
  fp.g0 = (float)(1.0 / (1.0 + std::exp((double)alpha)));
  fp.rom_m = 4096;
  FullDivParams p{};
  p.s = b->soa();
  p.n_envs = b->n_envs;
  p.blocks = b->blocks;
  p.perm = b->perm;
  p.roms = b->roms;
  p.cart_banks = b->cart_banks;
  p.ram_words = b->ram_words;
  p.full_tia = b->cfg.full_tia;
  p.rom_stride = b->rom_stride;
  p.cart_2k = b->cart_2k;
  p.dt = b->dt;
  p.actions = actions;
  p.n_instr = n_instr;
  p.ystart = b->cfg.ystart;
  p.n_div = n_div;
  p.counts = counts;
  p.ram_full = ram_full;
  p.err = b->err;
  const size_t smem = full_smem_bytes(b->E, b->rom_stride, b->ram_words);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_full, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
    return vcs_cuda_fail(b, e, "FULL kernel shared memory");
  k_full<<<b->n_blocks, b->E, smem, (cudaStream_t)stream>>>(p, fp);
  if ((e = cudaGetLastError())) return vcs_cuda_fail(b, e, "FULL kernel launch");
  return VCS_OK;
}
