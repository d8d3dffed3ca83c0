// C ABI of libvcs (include/vcs.h): batch set-up, memory ownership and launch
// of the hard-mode kernels.  No exception crosses the interface; every entry
// point returns a vcs_status and records a message for vcs_last_error.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdint>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/vcs.h"
#include "vcs_api_internal.h"

using namespace vcs;

static thread_local std::string g_create_error;

vcs_status vcs_fail(vcs_batch* b, vcs_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (b)
    b->last_error = buf;
  else
    g_create_error = buf;
  return st;
}

vcs_status vcs_cuda_fail(vcs_batch* b, cudaError_t e, const char* what) {
  return vcs_fail(b, e == cudaErrorMemoryAllocation ? VCS_ERR_OOM : VCS_ERR_CUDA, "%s: %s", what,
                  cudaGetErrorString(e));
}

SoA vcs_batch::soa() const { return soa_of(state, n_envs); }

SoA vcs::soa_of(uint32_t* state, int32_t n_envs) { return soa_at(state, n_envs); }

static int pick_envs_per_block(int n_envs, int sms) {
  // enough blocks to cover every SM twice, blocks of 8..128 envs
  int e = 128;
  while (e > 8 && (n_envs + e - 1) / e < 2 * sms) e /= 2;
  return e;
}

StepParams vcs_base_params(vcs_batch* b) {
  StepParams p{};
  p.s = b->soa();
  p.n_envs = b->n_envs;
  p.blocks = b->blocks;
  p.perm = b->perm;
  p.roms = b->roms;
  p.cart_banks = b->cart_banks;
  p.ram_words = b->ram_words;
  p.xmap = b->xmap;
  p.full_tia = b->cfg.full_tia;
  p.graphics = b->cfg.graphics_bits && b->cfg.step_instructions <= 0;   // instruction steps draw nothing
  p.rom_stride = b->rom_stride;
  p.dt = b->dt;
  p.ystart = b->cfg.ystart;
  p.err = b->err;
  p.sched_policy = b->sched_policy;
  p.sched_window = b->sched_window;
  p.tpe = b->tpe;
  p.boot_noop = b->cfg.boot_noop_frames;
  p.boot_reset = b->cfg.boot_reset_frames;
  p.start_noops = b->start_noops;
  p.n_start = b->n_start;
  p.boot_frames = (p.boot_noop + p.boot_reset > 0 || b->start_noops) ? 1 : 0;
  p.step_instr = b->cfg.step_instructions;
  return p;
}

// Group envs by cart (stable) and cut each cart's run into blocks of E, so
// that a block stages one ROM image; upload the block table and the
// permutation.  Replaces any previous geometry.
static vcs_status set_geometry(vcs_batch* b, int E) {
  const int n_envs = b->n_envs;
  const std::vector<int32_t>& env_cart = b->env_cart;
  std::vector<int32_t> perm(n_envs);
  for (int e = 0; e < n_envs; e++) perm[e] = e;
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int c) { return env_cart[a] < env_cart[c]; });
  auto cut = [&](int per_block) {
    std::vector<int4> blocks;
    for (int i = 0; i < n_envs;) {
      const int c = env_cart[perm[i]];
      int j = i;
      while (j < n_envs && env_cart[perm[j]] == c && j - i < per_block) j++;
      blocks.push_back(make_int4(c, i, j - i, 0));
      i = j;
    }
    return blocks;
  };
  const std::vector<int4> blocks = cut(E);
  const std::vector<int4> bwd = E > kBwdMaxEnvsPerBlock ? cut(kBwdMaxEnvsPerBlock) : std::vector<int4>();
  const std::vector<int4> wide = cut(kWideEnvsPerBlock);
  const std::vector<int4> widef = cut(kWideFwdEnvsPerBlock);
  int4* dblocks = nullptr;
  int4* dbwd = nullptr;
  int4* dwide = nullptr;
  int4* dwidef = nullptr;
  int32_t* dperm = nullptr;
  cudaError_t e;
  if ((e = cudaMalloc(&dblocks, blocks.size() * sizeof(int4))) || (e = cudaMalloc(&dperm, n_envs * sizeof(int32_t))) ||
      (!bwd.empty() && (e = cudaMalloc(&dbwd, bwd.size() * sizeof(int4)))) ||
      (e = cudaMalloc(&dwide, wide.size() * sizeof(int4))) ||
      (e = cudaMemcpy(dwide, wide.data(), wide.size() * sizeof(int4), cudaMemcpyHostToDevice)) ||
      (e = cudaMalloc(&dwidef, widef.size() * sizeof(int4))) ||
      (e = cudaMemcpy(dwidef, widef.data(), widef.size() * sizeof(int4), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(dblocks, blocks.data(), blocks.size() * sizeof(int4), cudaMemcpyHostToDevice)) ||
      (!bwd.empty() && (e = cudaMemcpy(dbwd, bwd.data(), bwd.size() * sizeof(int4), cudaMemcpyHostToDevice))) ||
      (e = cudaMemcpy(dperm, perm.data(), n_envs * sizeof(int32_t), cudaMemcpyHostToDevice))) {
    cudaFree(dblocks);
    cudaFree(dbwd);
    cudaFree(dwide);
    cudaFree(dwidef);
    cudaFree(dperm);
    return vcs_cuda_fail(b, e, "launch geometry");
  }
  cudaFree(b->blocks);
  cudaFree(b->bwd_blocks);
  cudaFree(b->wide_blocks);
  b->wide_blocks = dwide;
  b->wide_n_blocks = (int)wide.size();
  cudaFree(b->wide_fwd_blocks);
  b->wide_fwd_blocks = dwidef;
  b->wide_fwd_n_blocks = (int)widef.size();
  cudaFree(b->perm);
  b->blocks = dblocks;
  b->bwd_blocks = dbwd;
  b->bwd_n_blocks = (int)bwd.size();
  b->bwd_E = bwd.empty() ? 0 : kBwdMaxEnvsPerBlock;
  b->perm = dperm;
  b->n_blocks = (int)blocks.size();
  b->perm_host = perm;
  b->E = E;
  b->geometry_gen++;
  return VCS_OK;
}

static bool valid_epb(int E) { return E == 8 || E == 16 || E == 32 || E == 64 || E == 128; }
static bool valid_tpe(int E, int T) { return (T == 1 || T == 2 || T == 4 || T == 8) && E * T <= 128; }



// Hard frame steps that return screens run the step kernel built without
// drawing (deferred rasterisation; its logs go to the raster kernel, one step
// per launch), unless the batch asks for drawing in the step kernel.
// Without screens the whole TIA runs that build too (its interpreter is the
// faster one there), the subset machine its regular kernel (the faster one
// there: 2.79 against 2.91 ms per bench step on one box).
static bool raster_applies(const vcs_batch* b, const StepParams& p) {
  return p.n_steps > 0 && p.step_instr <= 0 && b->cfg.inline_render == 0;
}

// The logs take kRasterLogCap entries per env (67 KB, the most picture-
// register writes a frame can make: the log never fills).  If the device
// cannot hold them the batch draws in the step kernel from then on
// (inline_render = 1), which needs no logs: screens are the same.
static vcs_status ensure_raster(vcs_batch* b) {
  if (b->dr_log) return VCS_OK;
  const size_t n = (size_t)b->n_envs;
  cudaError_t e;
  if ((e = cudaMalloc(&b->dr_log, n * (size_t)kRasterLogCap * sizeof(uint32_t))) ||
      (e = cudaMalloc(&b->dr_hdr, n * kRasterHdr * sizeof(uint32_t)))) {
    cudaFree(b->dr_log);
    b->dr_log = nullptr;
    b->dr_hdr = nullptr;
    if (e == cudaErrorMemoryAllocation) {
      (void)cudaGetLastError();   // the failed allocation leaves no sticky error
      b->cfg.inline_render = 1;
      return VCS_OK;
    }
    return vcs_cuda_fail(b, e, "raster logs");
  }
  return VCS_OK;
}

// The next three timing events of a timed launch (null when not timing or
// the stream is being captured).
static cudaEvent_t* timing_events(vcs_batch* b, void* stream) {
  if (!b->timing) return nullptr;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
    return nullptr;
  while (b->tk_events.size() < b->tk_used + 3) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    b->tk_events.push_back(e);
  }
  cudaEvent_t* ev = &b->tk_events[b->tk_used];
  b->tk_used += 3;
  return ev;
}

// One launch of the step kernel over p.n_steps steps; with deferred
// rasterisation one step per launch, each followed by the raster kernel
// that draws its screens from the logs.
static vcs_status launch(vcs_batch* b, StepParams& p, void* stream) {
  if (raster_applies(b, p) && !p.screen_out && p.full_tia) {   // nothing to draw: the lean kernel, as many steps as asked
    StepParams q = p;
    q.dr = 1;
    cudaEvent_t* ev = timing_events(b, stream);
    if (ev) cudaEventRecord(ev[0], (cudaStream_t)stream);
    int e = launch_step(q, b->n_blocks, b->E, stream);
    if (e) return vcs_cuda_fail(b, (cudaError_t)e, "step kernel launch");
    if (ev) {
      cudaEventRecord(ev[1], (cudaStream_t)stream);
      cudaEventRecord(ev[2], (cudaStream_t)stream);
    }
    return VCS_OK;
  }
  if (raster_applies(b, p) && p.screen_out) {
    vcs_status st = ensure_raster(b);
    if (st != VCS_OK) return st;
  }
  if (raster_applies(b, p) && p.screen_out) {   // still deferring: the logs are there
    const size_t n = (size_t)b->n_envs;
    for (int32_t t = 0; t < p.n_steps; t++) {
      StepParams q = p;
      q.n_steps = 1;
      if (t > 0) {   // power-on requests belong to the first launch
        q.reset_all = 0;
        q.reset_mask = nullptr;
      }
      q.actions = p.actions ? p.actions + (size_t)t * n : nullptr;
      q.ram_out = p.ram_out ? p.ram_out + (size_t)t * n * 128 : nullptr;
      q.screen_out = p.screen_out + (size_t)t * n * kScreenH * kScreenW;
      q.status_out = p.status_out ? p.status_out + (size_t)t * n : nullptr;
      q.dr = 1;
      q.dr_log = b->dr_log;
      q.dr_hdr = b->dr_hdr;
      cudaEvent_t* ev = timing_events(b, stream);
      if (ev) cudaEventRecord(ev[0], (cudaStream_t)stream);
      int e = launch_step(q, b->n_blocks, b->E, stream);
      if (e) return vcs_cuda_fail(b, (cudaError_t)e, "step kernel launch");
      if (ev) cudaEventRecord(ev[1], (cudaStream_t)stream);
      e = (p.full_tia ? launch_raster_ft : launch_raster)(b->dr_hdr, b->dr_log, b->n_envs, b->cfg.ystart,
                                                         q.screen_out, ev ? b->tk_entries : nullptr, stream);
      if (e) return vcs_cuda_fail(b, (cudaError_t)e, "raster kernel launch");
      if (ev) cudaEventRecord(ev[2], (cudaStream_t)stream);
    }
    return VCS_OK;
  }
  cudaEvent_t* ev = p.n_steps > 0 ? timing_events(b, stream) : nullptr;
  if (ev) cudaEventRecord(ev[0], (cudaStream_t)stream);
  int e = launch_step(p, b->n_blocks, b->E, stream);
  if (e) return vcs_cuda_fail(b, (cudaError_t)e, "step kernel launch");
  if (ev) {
    cudaEventRecord(ev[1], (cudaStream_t)stream);
    cudaEventRecord(ev[2], (cudaStream_t)stream);
  }
  return VCS_OK;
}

static void free_batch(vcs_batch* b) {
  if (!b) return;
  cudaFree(b->state);
  cudaFree(b->roms);
  cudaFree(b->cart_banks);
  cudaFree(b->cart_2k);
  cudaFree(b->env_cart_dev);
  cudaFree(b->cart_begin);
  cudaFree(b->dt);
  cudaFree(b->blocks);
  cudaFree(b->bwd_blocks);
  cudaFree(b->wide_blocks);
  cudaFree(b->wide_fwd_blocks);
  cudaFree(b->perm);
  cudaFree(b->ep_len);
  cudaFree(b->dr_log);
  cudaFree(b->dr_hdr);
  cudaFree(b->start_noops);
  cudaFree(b->err);
  cudaFree(b->h_actions);
  cudaFree(b->h_ram);
  cudaFree(b->h_screen);
  cudaFree(b->h2_actions);
  cudaFree(b->h2_ram);
  cudaFree(b->h2_screen);
  cudaFree(b->h_status[0]);
  cudaFree(b->h_status[1]);
  for (int k = 0; k < 2; k++) {
    if (b->ev_kernel[k]) cudaEventDestroy(b->ev_kernel[k]);
    if (b->ev_copy[k]) cudaEventDestroy(b->ev_copy[k]);
  }
  if (b->copy_stream) cudaStreamDestroy(b->copy_stream);
  for (cudaEvent_t e : b->tk_events) cudaEventDestroy(e);
  cudaFree(b->tk_entries);
  delete b;
}

extern "C" {

vcs_status vcs_config_default(vcs_config* cfg) {
  if (!cfg) return VCS_ERR_ARG;
  cfg->alpha = 6.0f;
  cfg->ystart = 34;
  cfg->boot_noop_frames = 0;
  cfg->boot_reset_frames = 0;
  cfg->envs_per_block = 0;
  cfg->segment_frames = 64;
  cfg->sched_policy = 0;
  cfg->sched_window = 4;
  cfg->steps_per_launch = 0;
  cfg->threads_per_env = 0;
  cfg->position_sampler = 0;
  cfg->step_instructions = 0;
  cfg->tape_budget_mb = 0;
  cfg->full_tia = 0;
  cfg->graphics_bits = 0;
  cfg->inline_render = 0;
  cfg->sweep_mode = 0;
  return VCS_OK;
}

const char* vcs_last_error(const vcs_batch* b) { return b ? b->last_error.c_str() : g_create_error.c_str(); }

vcs_status vcs_rom_stride(const vcs_batch* b, int32_t* rom_stride) {
  if (!b || !rom_stride) return VCS_ERR_ARG;
  *rom_stride = (int32_t)b->rom_stride;
  return VCS_OK;
}

// Whether every 4 KB bank repeats its first 128 bytes in the next 128.
static bool superchip_filler(const uint8_t* rom, uint32_t size) {
  for (uint32_t b = 0; b < size; b += 4096)
    if (memcmp(rom + b, rom + b + 128, 128) != 0) return false;
  return true;
}

// Absolute-mode accesses (LDA, STA, BIT, NOP abs) whose address is a
// cartridge mirror of [lo, hi].
static int abs_accesses(const uint8_t* rom, uint32_t size, uint32_t lo, uint32_t hi) {
  int n = 0;
  for (uint32_t i = 0; i + 2 < size; i++) {
    const uint8_t op = rom[i];
    if (op != 0xAD && op != 0x8D && op != 0x2C && op != 0x0C) continue;
    const uint32_t a = ((uint32_t)rom[i + 1] | ((uint32_t)rom[i + 2] << 8)) & 0x1FFF;
    n += a >= lo && a <= hi;
  }
  return n;
}

// JSR instructions whose target's high byte is $D0-$DF: a call into the
// second bank of an FE image (its first bank is addressed at $F000, its
// second at $D000; bit 5 of the high byte selects the bank).
static int fe_calls(const uint8_t* rom, uint32_t size) {
  int n = 0;
  for (uint32_t i = 0; i + 2 < size; i++) n += rom[i] == 0x20 && (rom[i + 2] & 0xF0) == 0xD0;
  return n;
}

vcs_status vcs_detect_mapper(const uint8_t* rom, uint32_t size, uint8_t* mapper) {
  if (!rom || !mapper) return vcs_fail(nullptr, VCS_ERR_ARG, "rom and mapper must not be NULL");
  switch (size) {
    case 2048: *mapper = VCS_MAPPER_2K; return VCS_OK;
    case 4096: *mapper = VCS_MAPPER_4K; return VCS_OK;
    case 8192:
      if (abs_accesses(rom, size, 0x1FE0, 0x1FF7) > 0 && abs_accesses(rom, size, 0x1FF8, 0x1FF9) == 0) {
        *mapper = VCS_MAPPER_E0;
        return VCS_OK;
      }
      if (abs_accesses(rom, size, 0x1FF8, 0x1FF9) == 0 && fe_calls(rom, size) > 0) {
        *mapper = VCS_MAPPER_FE;
        return VCS_OK;
      }
      *mapper = superchip_filler(rom, size) ? VCS_MAPPER_F8SC : VCS_MAPPER_F8;
      return VCS_OK;
    case 16384: *mapper = superchip_filler(rom, size) ? VCS_MAPPER_F6SC : VCS_MAPPER_F6; return VCS_OK;
    case 32768: *mapper = superchip_filler(rom, size) ? VCS_MAPPER_F4SC : VCS_MAPPER_F4; return VCS_OK;
    default: return vcs_fail(nullptr, VCS_ERR_ROM_SIZE, "no cartridge format of %u bytes", size);
  }
}

vcs_status vcs_batch_info(const vcs_batch* b, int32_t* n_envs, int32_t* n_carts, int32_t* epb) {
  if (!b) return VCS_ERR_ARG;
  if (n_envs) *n_envs = b->n_envs;
  if (n_carts) *n_carts = b->n_carts;
  if (epb) *epb = b->E;
  return VCS_OK;
}

vcs_status vcs_destroy(vcs_batch* b) {
  if (!b) return VCS_ERR_ARG;
  free_batch(b);
  return VCS_OK;
}

vcs_status vcs_create_batch(const uint8_t* const* roms, const uint32_t* rom_sizes, const uint8_t* mappers,
                            int32_t n_carts, const int32_t* env_cart, int32_t n_envs, const vcs_config* cfg,
                            vcs_batch** out) {
  if (!out) return vcs_fail(nullptr, VCS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!roms || !rom_sizes || !mappers || !env_cart)
    return vcs_fail(nullptr, VCS_ERR_ARG, "null roms / rom_sizes / mappers / env_cart");
  if (n_carts <= 0 || n_envs <= 0) return vcs_fail(nullptr, VCS_ERR_ARG, "n_carts and n_envs must be positive");
  static const uint32_t want[10] = {2048, 4096, 8192, 16384, 32768, 8192, 16384, 32768, 8192, 8192};
  uint32_t rom_stride = 8192;   // the largest image, at least 8 KB
  for (int c = 0; c < n_carts; c++) {
    if (mappers[c] > VCS_MAPPER_FE)
      return vcs_fail(nullptr, VCS_ERR_MAPPER, "cart %d: unknown mapper %d", c, mappers[c]);
    if (rom_sizes[c] != want[mappers[c]])
      return vcs_fail(nullptr, VCS_ERR_ROM_SIZE, "cart %d: %u bytes for mapper %d (want %u)", c, rom_sizes[c],
                      mappers[c], want[mappers[c]]);
    if (!roms[c]) return vcs_fail(nullptr, VCS_ERR_ARG, "cart %d: null ROM", c);
    rom_stride = std::max(rom_stride, rom_sizes[c]);
  }
  for (int e = 0; e < n_envs; e++)
    if (env_cart[e] < 0 || env_cart[e] >= n_carts)
      return vcs_fail(nullptr, VCS_ERR_ARG, "env %d: cart %d out of range", e, env_cart[e]);

  vcs_batch* b = new (std::nothrow) vcs_batch;
  if (!b) return vcs_fail(nullptr, VCS_ERR_OOM, "host allocation failed");
  if (cfg)
    b->cfg = *cfg;
  else
    vcs_config_default(&b->cfg);
  if (b->cfg.ystart < 0 || b->cfg.ystart > 400 || b->cfg.boot_noop_frames < 0 || b->cfg.boot_reset_frames < 0 ||
      b->cfg.segment_frames < 1) {
    free_batch(b);
    return vcs_fail(nullptr, VCS_ERR_ARG, "config out of range (ystart 0..400, boot frames >= 0, segment >= 1)");
  }
  if (b->cfg.inline_render < 0 || b->cfg.inline_render > 1) {
    free_batch(b);
    return vcs_fail(nullptr, VCS_ERR_ARG, "inline_render must be 0 or 1");
  }
  if (b->cfg.sweep_mode < 0 || b->cfg.sweep_mode > 2) {
    free_batch(b);
    return vcs_fail(nullptr, VCS_ERR_ARG, "sweep_mode must be 0, 1 or 2");
  }
  b->n_envs = n_envs;
  b->n_carts = n_carts;
  b->env_cart.assign(env_cart, env_cart + n_envs);
  b->mapper.assign(mappers, mappers + n_carts);
  b->rom_size.assign(rom_sizes, rom_sizes + n_carts);

  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->sms = sms;
  int E = b->cfg.envs_per_block;
  if (E == 0) E = pick_envs_per_block(n_envs, sms);
  if (!valid_epb(E)) {
    free_batch(b);
    return vcs_fail(nullptr, VCS_ERR_ARG, "envs_per_block must be 0, 8, 16, 32, 64 or 128");
  }
  if (b->cfg.steps_per_launch < 0) {
    free_batch(b);
    return vcs_fail(nullptr, VCS_ERR_ARG, "steps_per_launch must be >= 0");
  }
  b->steps_per_launch = b->cfg.steps_per_launch;
  // replicas only pay where rendering is a large share of the work, so the
  // default is one thread per env; vcs_autotune measures the others
  int T = b->cfg.threads_per_env;
  if (T == 0) T = 1;
  if (!valid_tpe(E, T)) {
    free_batch(b);
    return vcs_fail(nullptr, VCS_ERR_ARG, "threads_per_env must be 0, 1, 2, 4 or 8 with envs_per_block x it <= 128");
  }
  b->tpe = T;
  if (b->cfg.step_instructions < 0 ||
      (b->cfg.step_instructions > 0 && b->cfg.boot_noop_frames + b->cfg.boot_reset_frames > 0)) {
    free_batch(b);
    return vcs_fail(nullptr, VCS_ERR_ARG, "step_instructions must be >= 0, and 0 with boot frames");
  }
  if (b->cfg.full_tia < 0 || b->cfg.full_tia > 1) {
    free_batch(b);
    return vcs_fail(nullptr, VCS_ERR_ARG, "full_tia must be 0 or 1");
  }
  if (b->cfg.position_sampler < 0 || b->cfg.position_sampler > 1) {
    free_batch(b);
    return vcs_fail(nullptr, VCS_ERR_ARG, "position_sampler must be 0 or 1");
  }
  if (b->cfg.graphics_bits < 0 || b->cfg.graphics_bits > 1) {
    free_batch(b);
    return vcs_fail(nullptr, VCS_ERR_ARG, "graphics_bits must be 0 or 1");
  }
  if (b->cfg.sched_policy < 0 || b->cfg.sched_policy > 1) {
    free_batch(b);
    return vcs_fail(nullptr, VCS_ERR_ARG, "sched_policy must be 0 or 1");
  }
  b->sched_policy = (uint32_t)b->cfg.sched_policy;
  b->sched_window = b->cfg.sched_window < 0 ? 0xFFFFFFFFu : (uint32_t)b->cfg.sched_window;

  // device images: 2K mirrored into 4 KB, bank-switched carts as their banks
  b->rom_stride = rom_stride;
  std::vector<uint8_t> img((size_t)n_carts * rom_stride, 0);
  std::vector<uint8_t> banks(n_carts), is2k(n_carts);
  for (int c = 0; c < n_carts; c++) {
    uint8_t* d = img.data() + (size_t)c * rom_stride;
    if (mappers[c] == VCS_MAPPER_2K) {
      memcpy(d, roms[c], 2048);
      memcpy(d + 2048, roms[c], 2048);
    } else {
      memcpy(d, roms[c], rom_sizes[c]);
    }
    banks[c] = mappers[c] >= VCS_MAPPER_F8 && mappers[c] != VCS_MAPPER_E0 ? (uint8_t)(rom_sizes[c] / 4096) : 0;
    if (mappers[c] >= VCS_MAPPER_F8SC && mappers[c] <= VCS_MAPPER_F4SC) {
      banks[c] |= (uint8_t)kCartSC;
      b->ram_words = 64;   // every block reserves room for the Superchip's RAM
      b->xmap = 1;
    }
    if (mappers[c] == VCS_MAPPER_E0) {
      banks[c] = (uint8_t)kCartE0;
      b->xmap = 1;
    }
    if (mappers[c] == VCS_MAPPER_FE) {   // two banks, switched by JSR / RTS: the extended kernels
      banks[c] = (uint8_t)(2u | kCartFE);
      b->xmap = 1;
    }
    is2k[c] = mappers[c] == VCS_MAPPER_2K;
  }
  std::vector<int32_t> cart_begin(n_carts + 1, 0);
  for (int e = 0; e < n_envs; e++) cart_begin[env_cart[e] + 1]++;
  for (int c = 0; c < n_carts; c++) cart_begin[c + 1] += cart_begin[c];
  DecodeTables dt;
  build_decode_tables(&dt);

  cudaError_t e;
  const size_t nst = (size_t)kStateWords * n_envs * sizeof(uint32_t);
  if ((e = cudaMalloc(&b->state, nst)) || (e = cudaMalloc(&b->roms, img.size())) ||
      (e = cudaMalloc(&b->cart_banks, n_carts)) || (e = cudaMalloc(&b->dt, sizeof(DecodeTables))) ||
      (e = cudaMalloc(&b->err, sizeof(int32_t))) ||
      (e = cudaMalloc(&b->cart_2k, n_carts)) || (e = cudaMalloc(&b->env_cart_dev, n_envs * sizeof(int32_t))) ||
      (e = cudaMalloc(&b->cart_begin, (n_carts + 1) * sizeof(int32_t)))) {
    vcs_status st = vcs_cuda_fail(nullptr, e, "device allocation");
    free_batch(b);
    return st;
  }
  if ((e = cudaMemcpy(b->roms, img.data(), img.size(), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->cart_banks, banks.data(), n_carts, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->dt, &dt, sizeof dt, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->cart_2k, is2k.data(), n_carts, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->env_cart_dev, env_cart, n_envs * sizeof(int32_t), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->cart_begin, cart_begin.data(), (n_carts + 1) * sizeof(int32_t), cudaMemcpyHostToDevice)) ||
      (e = cudaMemset(b->err, 0, sizeof(int32_t))) || (e = cudaMemset(b->state, 0, nst))) {
    vcs_status st = vcs_cuda_fail(nullptr, e, "device upload");
    free_batch(b);
    return st;
  }
  if (set_geometry(b, E) != VCS_OK) {
    g_create_error = b->last_error;
    free_batch(b);
    return VCS_ERR_CUDA;
  }
  // power on every env (plus the configured boot frames)
  StepParams p = vcs_base_params(b);
  p.reset_all = 1;
  p.n_steps = 0;        // the launch powers on and boots; no env-step
  p.frame_skip = 1;
  vcs_status st = launch(b, p, nullptr);
  if (st == VCS_OK && (e = cudaDeviceSynchronize())) st = vcs_cuda_fail(b, e, "power-on");
  if (st != VCS_OK) {
    g_create_error = b->last_error;
    free_batch(b);
    return st;
  }
  *out = b;
  return VCS_OK;
}

vcs_status vcs_set_episodes(vcs_batch* b, const uint32_t* ep_len, int32_t n_episodes) {
  if (!b) return VCS_ERR_ARG;
  if (n_episodes < 0 || (n_episodes > 0 && !ep_len)) return vcs_fail(b, VCS_ERR_ARG, "bad episode table");
  if (n_episodes > 0 && b->cfg.step_instructions > 0)
    return vcs_fail(b, VCS_ERR_ARG, "episode tables need frame steps (step_instructions = 0)");
  cudaFree(b->ep_len);
  b->ep_len = nullptr;
  b->n_episodes = 0;
  if (n_episodes == 0) return VCS_OK;
  size_t bytes = (size_t)b->n_envs * n_episodes * sizeof(uint32_t);
  cudaError_t e;
  if ((e = cudaMalloc(&b->ep_len, bytes))) return vcs_cuda_fail(b, e, "episode table");
  if ((e = cudaMemcpy(b->ep_len, ep_len, bytes, cudaMemcpyHostToDevice))) return vcs_cuda_fail(b, e, "episode table");
  b->n_episodes = n_episodes;
  return VCS_OK;
}

vcs_status vcs_set_start_noops(vcs_batch* b, const uint8_t* counts, int32_t n_per_env) {
  if (!b) return VCS_ERR_ARG;
  if (n_per_env < 0 || (n_per_env > 0 && !counts)) return vcs_fail(b, VCS_ERR_ARG, "bad start-noop table");
  if (n_per_env > 0 && b->cfg.step_instructions > 0)
    return vcs_fail(b, VCS_ERR_ARG, "start NOOPs need frame steps (step_instructions = 0)");
  cudaFree(b->start_noops);
  b->start_noops = nullptr;
  b->n_start = 0;
  if (n_per_env == 0) return VCS_OK;
  const size_t bytes = (size_t)b->n_envs * n_per_env;
  cudaError_t e;
  if ((e = cudaMalloc(&b->start_noops, bytes))) return vcs_cuda_fail(b, e, "start-noop table");
  if ((e = cudaMemcpy(b->start_noops, counts, bytes, cudaMemcpyHostToDevice))) return vcs_cuda_fail(b, e, "start-noop table");
  b->n_start = n_per_env;
  return VCS_OK;
}

vcs_status vcs_reset(vcs_batch* b, const uint8_t* env_mask, void* stream) {
  if (!b) return VCS_ERR_ARG;
  StepParams p = vcs_base_params(b);
  p.reset_all = env_mask ? 0 : 1;
  p.reset_mask = env_mask;
  p.n_steps = 0;        // the launch powers on and boots; no env-step
  p.frame_skip = 1;
  vcs_status st = launch(b, p, stream);
  if (st != VCS_OK) return st;
  if (!env_mask) {   // fresh episodes
    SoA s = b->soa();
    cudaMemsetAsync(s.epf, 0, b->n_envs * sizeof(uint32_t), (cudaStream_t)stream);
    cudaMemsetAsync(s.epi, 0, b->n_envs * sizeof(uint32_t), (cudaStream_t)stream);
  }
  return VCS_OK;
}

vcs_status vcs_rollout(vcs_batch* b, const uint8_t* actions, int32_t n_steps, int32_t frame_skip,
                       uint8_t* ram_out, uint8_t* screen_out, uint8_t* status_out, void* stream) {
  if (!b) return VCS_ERR_ARG;
  if (!actions) return vcs_fail(b, VCS_ERR_ARG, "actions is NULL");
  if (n_steps < 0 || frame_skip < 1) return vcs_fail(b, VCS_ERR_ARG, "n_steps >= 0 and frame_skip >= 1 required");
  if (screen_out && b->cfg.step_instructions > 0)
    return vcs_fail(b, VCS_ERR_ARG, "instruction steps return no screens");
  const int32_t k = b->steps_per_launch > 0 ? b->steps_per_launch : (n_steps > 0 ? n_steps : 1);
  const size_t n = (size_t)b->n_envs;
  for (int32_t t0 = 0; t0 < n_steps; t0 += k) {
    StepParams p = vcs_base_params(b);
    p.actions = actions + (size_t)t0 * n;
    p.n_steps = std::min(k, n_steps - t0);
    p.frame_skip = frame_skip;
    p.ram_out = ram_out ? ram_out + (size_t)t0 * n * 128 : nullptr;
    p.screen_out = screen_out ? screen_out + (size_t)t0 * n * kScreenH * kScreenW : nullptr;
    p.status_out = status_out ? status_out + (size_t)t0 * n : nullptr;
    p.ep_len = b->ep_len;
    p.n_episodes = b->n_episodes;
    vcs_status st = launch(b, p, stream);
    if (st != VCS_OK) return st;
  }
  return VCS_OK;
}

vcs_status vcs_step(vcs_batch* b, const uint8_t* actions, int32_t frame_skip, uint8_t* ram_out,
                    uint8_t* screen_out, uint8_t* status_out, void* stream) {
  return vcs_rollout(b, actions, 1, frame_skip, ram_out, screen_out, status_out, stream);
}

vcs_status vcs_step_host(vcs_batch* b, const uint8_t* actions_host, int32_t frame_skip, uint8_t* ram_out_host,
                         uint8_t* screen_out_host, void* stream) {
  if (!b) return VCS_ERR_ARG;
  if (!actions_host) return vcs_fail(b, VCS_ERR_ARG, "actions_host is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  const size_t n = (size_t)b->n_envs;
  if (!b->h_actions) {
    if ((e = cudaMalloc(&b->h_actions, n)) || (e = cudaMalloc(&b->h_ram, n * 128)) ||
        (e = cudaMalloc(&b->h_screen, n * kScreenH * kScreenW)))
      return vcs_cuda_fail(b, e, "staging buffers");
  }
  if ((e = cudaMemcpyAsync(b->h_actions, actions_host, n, cudaMemcpyHostToDevice, s)))
    return vcs_cuda_fail(b, e, "actions upload");
  vcs_status st = vcs_step(b, b->h_actions, frame_skip, ram_out_host ? b->h_ram : nullptr,
                           screen_out_host ? b->h_screen : nullptr, nullptr, stream);
  if (st != VCS_OK) return st;
  if (ram_out_host && (e = cudaMemcpyAsync(ram_out_host, b->h_ram, n * 128, cudaMemcpyDeviceToHost, s)))
    return vcs_cuda_fail(b, e, "RAM download");
  if (screen_out_host &&
      (e = cudaMemcpyAsync(screen_out_host, b->h_screen, n * kScreenH * kScreenW, cudaMemcpyDeviceToHost, s)))
    return vcs_cuda_fail(b, e, "screen download");
  if ((e = cudaStreamSynchronize(s))) return vcs_cuda_fail(b, e, "step");
  return VCS_OK;
}

vcs_status vcs_rollout_host(vcs_batch* b, const uint8_t* actions_host, int32_t n_steps, int32_t frame_skip,
                            uint8_t* ram_host, uint8_t* screen_host, uint8_t* status_host, void* stream) {
  if (!b) return VCS_ERR_ARG;
  if (!actions_host || n_steps < 0 || frame_skip < 1)
    return vcs_fail(b, VCS_ERR_ARG, "actions_host, n_steps >= 0 and frame_skip >= 1 required");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  const size_t n = (size_t)b->n_envs, scr = n * kScreenH * kScreenW;
  if (!b->h_actions && ((e = cudaMalloc(&b->h_actions, n)) || (e = cudaMalloc(&b->h_ram, n * 128)) ||
                        (e = cudaMalloc(&b->h_screen, scr))))
    return vcs_cuda_fail(b, e, "staging buffers");
  if (!b->h2_actions) {
    if ((e = cudaMalloc(&b->h2_actions, n)) || (e = cudaMalloc(&b->h2_ram, n * 128)) ||
        (e = cudaMalloc(&b->h2_screen, scr)) || (e = cudaMalloc(&b->h_status[0], n)) ||
        (e = cudaMalloc(&b->h_status[1], n)) ||
        (e = cudaStreamCreateWithFlags(&b->copy_stream, cudaStreamNonBlocking)))
      return vcs_cuda_fail(b, e, "staging buffers");
    for (int k = 0; k < 2; k++)
      if ((e = cudaEventCreateWithFlags(&b->ev_kernel[k], cudaEventDisableTiming)) ||
          (e = cudaEventCreateWithFlags(&b->ev_copy[k], cudaEventDisableTiming)))
        return vcs_cuda_fail(b, e, "staging events");
  }
  uint8_t* act[2] = {b->h_actions, b->h2_actions};
  uint8_t* ram[2] = {b->h_ram, b->h2_ram};
  uint8_t* sc[2] = {b->h_screen, b->h2_screen};
  const cudaStream_t c = b->copy_stream;
  for (int32_t t = 0; t < n_steps; t++) {
    const int k = t & 1;
    // buffer set k is free once the download of step t - 2 has finished
    if (t >= 2 && (e = cudaStreamWaitEvent(s, b->ev_copy[k], 0))) return vcs_cuda_fail(b, e, "rollout_host");
    if ((e = cudaMemcpyAsync(act[k], actions_host + (size_t)t * n, n, cudaMemcpyHostToDevice, s)))
      return vcs_cuda_fail(b, e, "actions upload");
    vcs_status st = vcs_step(b, act[k], frame_skip, ram_host ? ram[k] : nullptr, screen_host ? sc[k] : nullptr,
                             status_host ? b->h_status[k] : nullptr, stream);
    if (st != VCS_OK) return st;
    if ((e = cudaEventRecord(b->ev_kernel[k], s)) || (e = cudaStreamWaitEvent(c, b->ev_kernel[k], 0)))
      return vcs_cuda_fail(b, e, "rollout_host");
    if (ram_host && (e = cudaMemcpyAsync(ram_host + (size_t)t * n * 128, ram[k], n * 128, cudaMemcpyDeviceToHost, c)))
      return vcs_cuda_fail(b, e, "RAM download");
    if (screen_host && (e = cudaMemcpyAsync(screen_host + (size_t)t * scr, sc[k], scr, cudaMemcpyDeviceToHost, c)))
      return vcs_cuda_fail(b, e, "screen download");
    if (status_host && (e = cudaMemcpyAsync(status_host + (size_t)t * n, b->h_status[k], n, cudaMemcpyDeviceToHost, c)))
      return vcs_cuda_fail(b, e, "status download");
    if ((e = cudaEventRecord(b->ev_copy[k], c))) return vcs_cuda_fail(b, e, "rollout_host");
  }
  if ((e = cudaStreamSynchronize(c)) || (e = cudaStreamSynchronize(s))) return vcs_cuda_fail(b, e, "rollout_host");
  return VCS_OK;
}

vcs_status vcs_cart_ram(vcs_batch* b, uint8_t* out, void* stream) {
  if (!b || !out) return VCS_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(out) & 3) return vcs_fail(b, VCS_ERR_ARG, "out must be 4-byte aligned");
  const int e = launch_cart_ram(b->soa(), b->n_envs, out, stream);
  if (e) return vcs_cuda_fail(b, (cudaError_t)e, "cart RAM kernel launch");
  return VCS_OK;
}

vcs_status vcs_state_bytes(const vcs_batch* b, size_t* bytes) {
  if (!b || !bytes) return VCS_ERR_ARG;
  *bytes = (size_t)kStateWords * b->n_envs * sizeof(uint32_t);
  return VCS_OK;
}

vcs_status vcs_save_state(vcs_batch* b, void* blob_host, void* stream) {
  if (!b || !blob_host) return VCS_ERR_ARG;
  size_t bytes = (size_t)kStateWords * b->n_envs * sizeof(uint32_t);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(blob_host, b->state, bytes, cudaMemcpyDeviceToHost, (cudaStream_t)stream)) ||
      (e = cudaStreamSynchronize((cudaStream_t)stream)))
    return vcs_cuda_fail(b, e, "save state");
  return VCS_OK;
}

vcs_status vcs_load_state(vcs_batch* b, const void* blob_host, void* stream) {
  if (!b || !blob_host) return VCS_ERR_ARG;
  size_t bytes = (size_t)kStateWords * b->n_envs * sizeof(uint32_t);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(b->state, blob_host, bytes, cudaMemcpyHostToDevice, (cudaStream_t)stream)) ||
      (e = cudaStreamSynchronize((cudaStream_t)stream)))
    return vcs_cuda_fail(b, e, "load state");
  return VCS_OK;
}

}  // extern "C"

// Tuning results of this process, keyed by GPU, batch shape, cartridge mix
// (envs per format), frame-skip, which outputs the rollouts write,
// instruction-granular steps and the TIA mode.
static std::mutex g_tune_mu;
static std::map<std::string, vcs_tune> g_tune_cache;

static std::string tune_key(const vcs_batch* b, int32_t frame_skip, bool ram, bool screen) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  std::string name = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? prop.name : "?";
  int per_mapper[VCS_MAPPER_FE + 1] = {};
  for (int e = 0; e < b->n_envs; e++) per_mapper[b->mapper[b->env_cart[e]]]++;
  std::string mix;
  for (int m = 0; m <= VCS_MAPPER_FE; m++) mix += "|" + std::to_string(per_mapper[m]);
  char buf[256];
  snprintf(buf, sizeof buf, "|%d|%d|%d|%d|%d|%d|%d", b->sms, b->n_envs, b->n_carts, frame_skip,
           (ram ? 1 : 0) | (screen ? 2 : 0), b->cfg.step_instructions, b->cfg.full_tia);
  return name + buf + mix;
}

static vcs_status apply_tune(vcs_batch* b, const vcs_tune& t) {
  if (b->E != t.envs_per_block) {
    vcs_status st = set_geometry(b, t.envs_per_block);
    if (st != VCS_OK) return st;
  }
  if (b->tpe != t.threads_per_env || b->steps_per_launch != t.steps_per_launch) b->geometry_gen++;   // graphs hold both
  b->tpe = t.threads_per_env;
  b->sched_policy = (uint32_t)t.sched_policy;
  b->sched_window = (uint32_t)t.sched_window;
  b->steps_per_launch = t.steps_per_launch;
  b->cfg.envs_per_block = b->E;
  b->cfg.threads_per_env = b->tpe;
  b->cfg.sched_policy = t.sched_policy;
  b->cfg.sched_window = t.sched_window;
  b->cfg.steps_per_launch = t.steps_per_launch;
  return VCS_OK;
}

extern "C" {

vcs_status vcs_autotune_cache_clear(void) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune_cache.clear();
  return VCS_OK;
}

vcs_status vcs_autotune(vcs_batch* b, int32_t frame_skip, int32_t n_steps, const uint8_t* actions,
                        uint8_t* ram_out, uint8_t* screen_out, vcs_tune* out, void* stream) {
  if (!b) return VCS_ERR_ARG;
  if (frame_skip < 1 || n_steps < 1) return vcs_fail(b, VCS_ERR_ARG, "frame_skip >= 1 and n_steps >= 1 required");
  const std::string key = tune_key(b, frame_skip, ram_out != nullptr, screen_out != nullptr);
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      vcs_tune t = it->second;
      vcs_status st = apply_tune(b, t);
      if (st != VCS_OK) return st;
      t.n_trials = 0;
      if (out) *out = t;
      return VCS_OK;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)b->n_envs;
  const size_t nst = (size_t)kStateWords * n * sizeof(uint32_t);
  uint32_t* saved = nullptr;
  uint8_t* noop = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e;
  auto cleanup = [&]() {
    cudaFree(saved);
    cudaFree(noop);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if ((e = cudaMalloc(&saved, nst)) || (e = cudaEventCreate(&e0)) || (e = cudaEventCreate(&e1)) ||
      (e = cudaMemcpyAsync(saved, b->state, nst, cudaMemcpyDeviceToDevice, s))) {
    cleanup();
    return vcs_cuda_fail(b, e, "autotune set-up");
  }
  if (!actions) {
    if ((e = cudaMalloc(&noop, (size_t)n_steps * n)) || (e = cudaMemsetAsync(noop, 0, (size_t)n_steps * n, s))) {
      cleanup();
      return vcs_cuda_fail(b, e, "autotune set-up");
    }
    actions = noop;
  }
  int32_t trials = 0;
  // one trial of the batch's current geometry: a warm-up rollout, then the
  // faster of two timed ones, the state restored before each and after
  auto trial = [&](float* ms) -> vcs_status {
    vcs_status st;
    if ((st = vcs_rollout(b, actions, n_steps, frame_skip, ram_out, screen_out, nullptr, stream)) != VCS_OK) return st;
    *ms = 1e30f;
    for (int rep = 0; rep < 2; rep++) {
      float t = 0.f;
      if ((e = cudaMemcpyAsync(b->state, saved, nst, cudaMemcpyDeviceToDevice, s))) return vcs_cuda_fail(b, e, "autotune");
      if ((e = cudaEventRecord(e0, s))) return vcs_cuda_fail(b, e, "autotune");
      if ((st = vcs_rollout(b, actions, n_steps, frame_skip, ram_out, screen_out, nullptr, stream)) != VCS_OK) return st;
      if ((e = cudaEventRecord(e1, s)) || (e = cudaEventSynchronize(e1)) || (e = cudaEventElapsedTime(&t, e0, e1)))
        return vcs_cuda_fail(b, e, "autotune");
      *ms = t < *ms ? t : *ms;
    }
    if ((e = cudaMemcpyAsync(b->state, saved, nst, cudaMemcpyDeviceToDevice, s))) return vcs_cuda_fail(b, e, "autotune");
    trials++;
    return VCS_OK;
  };
  vcs_status st = VCS_OK;
  float best = 1e30f, ms = 0.f;
  // 1. envs per block and threads per env, under program-order scheduling and one launch
  b->sched_policy = 0;
  b->steps_per_launch = 0;
  int bestE = b->E, bestT = b->tpe;
  const int cand_e[5] = {8, 16, 32, 64, 128};
  // hard frame steps run the step kernel without drawing, one lane per env
  // (deferred rasterisation), so replicas are not tried for them
  const int maxT = (b->cfg.inline_render == 0 && b->cfg.step_instructions <= 0) ? 1 : 4;
  for (int E : cand_e) {
    if (E > 8 && (int)((n + E / 2 - 1) / (E / 2)) <= 1) break;   // no larger block helps a tiny batch
    if ((st = set_geometry(b, E)) != VCS_OK) break;
    for (int T = 1; st == VCS_OK && valid_tpe(E, T) && T <= maxT; T *= 2) {
      b->tpe = T;
      if ((st = trial(&ms)) != VCS_OK) break;
      if (ms < best) { best = ms; bestE = E; bestT = T; }
    }
    if (st != VCS_OK) break;
  }
  b->tpe = bestT;
  if (st == VCS_OK && b->E != bestE) st = set_geometry(b, bestE);
  // 2. scheduling policy
  uint32_t bestP = 0, bestW = b->sched_window;
  const uint32_t cand_w[2] = {4, 32};
  for (int i = 0; st == VCS_OK && i < 2; i++) {
    b->sched_policy = 1;
    b->sched_window = cand_w[i];
    if ((st = trial(&ms)) != VCS_OK) break;
    if (ms < best) { best = ms; bestP = 1; bestW = cand_w[i]; }
  }
  b->sched_policy = bestP;
  b->sched_window = bestW;
  // 3. env-steps per launch
  int32_t bestK = 0;
  const int32_t cand_k[2] = {1, 4};
  for (int i = 0; st == VCS_OK && i < 2; i++) {
    if (cand_k[i] >= n_steps) continue;
    b->steps_per_launch = cand_k[i];
    if ((st = trial(&ms)) != VCS_OK) break;
    if (ms < best) { best = ms; bestK = cand_k[i]; }
  }
  b->steps_per_launch = bestK;
  cleanup();
  if (st != VCS_OK) return st;
  vcs_tune t;
  t.envs_per_block = b->E;
  t.threads_per_env = b->tpe;
  t.sched_policy = (int32_t)b->sched_policy;
  t.sched_window = (int32_t)b->sched_window;
  t.steps_per_launch = b->steps_per_launch;
  t.ms_per_step = best / (float)n_steps;
  t.n_trials = trials;
  if ((st = apply_tune(b, t)) != VCS_OK) return st;
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache[key] = t;
  }
  if (out) *out = t;
  return VCS_OK;
}

}  // extern "C"

struct vcs_graph {
  vcs_batch* b = nullptr;
  uint32_t gen = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" {

vcs_status vcs_graph_create(vcs_batch* b, const uint8_t* actions, int32_t n_steps, int32_t frame_skip,
                            uint8_t* ram_out, uint8_t* screen_out, uint8_t* status_out, vcs_graph** out) {
  if (!b || !out) return VCS_ERR_ARG;
  *out = nullptr;
  if (!actions || n_steps < 1 || frame_skip < 1)
    return vcs_fail(b, VCS_ERR_ARG, "actions, n_steps >= 1 and frame_skip >= 1 required");
  if (screen_out && b->cfg.step_instructions <= 0 && b->cfg.inline_render == 0) {
    vcs_status st = ensure_raster(b);   // allocated before the capture, not inside it
    if (st != VCS_OK) return st;
  }
  vcs_graph* g = new (std::nothrow) vcs_graph;
  if (!g) return vcs_fail(b, VCS_ERR_OOM, "host allocation failed");
  cudaStream_t s = nullptr;
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) ||
      (e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal))) {
    if (s) cudaStreamDestroy(s);
    delete g;
    return vcs_cuda_fail(b, e, "graph capture");
  }
  vcs_status st = vcs_rollout(b, actions, n_steps, frame_skip, ram_out, screen_out, status_out, s);
  e = cudaStreamEndCapture(s, &g->graph);
  if (st == VCS_OK && e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  cudaStreamDestroy(s);
  if (st != VCS_OK || e != cudaSuccess) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return st != VCS_OK ? st : vcs_cuda_fail(b, e, "graph capture");
  }
  g->b = b;
  g->gen = b->geometry_gen;
  *out = g;
  return VCS_OK;
}

vcs_status vcs_graph_launch(vcs_graph* g, void* stream) {
  if (!g || !g->b) return VCS_ERR_ARG;
  if (g->gen != g->b->geometry_gen)
    return vcs_fail(g->b, VCS_ERR_STATE, "graph made under an older launch geometry; create it again");
  cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
  if (e) return vcs_cuda_fail(g->b, e, "graph launch");
  return VCS_OK;
}

vcs_status vcs_graph_destroy(vcs_graph* g) {
  if (!g) return VCS_ERR_ARG;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return VCS_OK;
}

vcs_status vcs_int_peak(double* ops_per_s, void* stream) {
  if (!ops_per_s) return VCS_ERR_ARG;
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
    return vcs_cuda_fail(nullptr, e, "device query");
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const int32_t iters = 4096;
  float ms = 0.f;
  if (!(e = cudaMalloc(&sink, (size_t)sms * 2 * sizeof(uint32_t))) && !(e = cudaEventCreate(&e0)) &&
      !(e = cudaEventCreate(&e1))) {
    launch_int_peak(sms, iters, sink, stream);   // warm-up
    if (!(e = cudaEventRecord(e0, s))) {
      int le = launch_int_peak(sms, iters, sink, stream);
      if (le) e = (cudaError_t)le;
      else if (!(e = cudaEventRecord(e1, s)) && !(e = cudaEventSynchronize(e1))) e = cudaEventElapsedTime(&ms, e0, e1);
    }
  }
  cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e) return vcs_cuda_fail(nullptr, e, "integer peak");
  // 72 operations per thread per loop turn (k_int_peak)
  *ops_per_s = (double)sms * 2 * 1024 * (double)iters * 72.0 / (ms * 1e-3);
  return VCS_OK;
}

vcs_status vcs_digest(vcs_batch* b, const uint8_t* ram, const uint8_t* screen, int32_t n_steps, uint64_t* out,
                      void* stream) {
  if (!b) return VCS_ERR_ARG;
  if (!ram || !out || n_steps < 0) return vcs_fail(b, VCS_ERR_ARG, "ram and out are required, n_steps >= 0");
  if (((uintptr_t)ram & 15) || ((uintptr_t)screen & 15) || ((uintptr_t)out & 7))
    return vcs_fail(b, VCS_ERR_ARG, "ram and screen must be 16-byte aligned, out 8-byte aligned");
  int e = launch_digest(ram, screen, (uint64_t)n_steps * (uint64_t)b->n_envs, out, stream);
  if (e) return vcs_cuda_fail(b, (cudaError_t)e, "digest kernel launch");
  return VCS_OK;
}

vcs_status vcs_time_kernels(vcs_batch* b, int32_t on) {
  if (!b || (on != 0 && on != 1)) return VCS_ERR_ARG;
  b->timing = on != 0;
  if (on) {
    b->tk_used = 0;
    cudaError_t e;
    if (!b->tk_entries && (e = cudaMalloc(&b->tk_entries, sizeof(unsigned long long))))
      return vcs_cuda_fail(b, e, "timing counter");
    if ((e = cudaMemset(b->tk_entries, 0, sizeof(unsigned long long)))) return vcs_cuda_fail(b, e, "timing counter");
  }
  return VCS_OK;
}

vcs_status vcs_kernel_times(vcs_batch* b, float* step_ms, float* raster_ms, int32_t* n_launches,
                            double* log_entries) {
  if (!b || !step_ms || !raster_ms || !n_launches) return VCS_ERR_ARG;
  double s = 0.0, r = 0.0;
  for (size_t i = 0; i + 3 <= b->tk_used; i += 3) {
    float a = 0.f, c = 0.f;
    cudaError_t e;
    if ((e = cudaEventSynchronize(b->tk_events[i + 2])) ||
        (e = cudaEventElapsedTime(&a, b->tk_events[i], b->tk_events[i + 1])) ||
        (e = cudaEventElapsedTime(&c, b->tk_events[i + 1], b->tk_events[i + 2])))
      return vcs_cuda_fail(b, e, "kernel timing events");
    s += a;
    r += c;
  }
  *step_ms = (float)s;
  *raster_ms = (float)r;
  *n_launches = (int32_t)(b->tk_used / 3);
  b->tk_used = 0;
  if (log_entries) {
    unsigned long long c = 0;
    cudaError_t e;
    if (b->tk_entries && (e = cudaMemcpy(&c, b->tk_entries, sizeof c, cudaMemcpyDeviceToHost)))
      return vcs_cuda_fail(b, e, "timing counter");
    *log_entries = (double)c;
    if (b->tk_entries) cudaMemset(b->tk_entries, 0, sizeof c);
  }
  return VCS_OK;
}

vcs_status vcs_sync(vcs_batch* b, void* stream) {
  if (!b) return VCS_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e) return vcs_cuda_fail(b, e, "synchronize");
  int32_t err = 0;
  if ((e = cudaMemcpy(&err, b->err, sizeof err, cudaMemcpyDeviceToHost))) return vcs_cuda_fail(b, e, "error word");
  if (err == 2) return vcs_fail(b, VCS_ERR_STATE, "backward tape overflow (recompute diverged from the forward)");
  if (err == kErrRasterLog) return vcs_fail(b, VCS_ERR_STATE, "a raster log passed its bound");
  if (err) return vcs_fail(b, VCS_ERR_WATCHDOG, "a device wait gave up (code %d); batch unusable", err);
  return VCS_OK;
}

}  // extern "C"
