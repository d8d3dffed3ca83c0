// The step kernel (hard mode and the SOFT-STE forward) as a template, shared
// by the translation units that instantiate it: vcs_kernels.cu for batches
// without Superchip or E0 carts, vcs_kernels_xm.cu for batches with them
// (XM), so that the cartridge-RAM ports and the slice mapping cost the other
// batches nothing.
//
// One thread per env, one block per run of envs of the same cartridge (the
// host groups envs by cart), so the block stages exactly one ROM image into
// shared memory.  The image is brought in by one TMA bulk copy
// (cp.async.bulk, completion tracked by an mbarrier with a bounded wait).
// Each thread keeps its machine in registers for the whole launch, its RAM
// and scanline buffer in shared memory, and writes RAM and finished
// scanlines (16-byte stores) straight to the caller's buffers.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "vcs_exec.cuh"
#include "vcs_kernels.cuh"
#include "vcs_run.cuh"

namespace vcs {

// Counts instructions and colour-register writes per checkpoint segment (the
// soft forward sizes the backward's tape with these).
struct CountTape {
  static constexpr bool kAcc = false;
  uint32_t n = 0, ncw = 0;
  uint64_t vregs = kVersionRegs;   // | kGraphicsRegs (| kGraphicsRegsFT) with the graphics-bit surrogate
  bool ftgb = false;               // the surrogate with the whole TIA: the delayed copies' versions
  __device__ __forceinline__ void rec(uint32_t, uint32_t, uint32_t) { n++; }
  static constexpr bool sampler = false;
  __device__ __forceinline__ void version_write(uint32_t reg) {
    ncw += (uint32_t)(vregs >> reg) & 1u;
    if (ftgb) ncw += reg == 0x1B ? 1u : (reg == 0x1C ? 2u : 0u);
  }
  __device__ __forceinline__ void pixels(float, float, float, float, float) {}
};

__device__ __forceinline__ uint32_t round_byte(float v) {
  float x = rintf(v);
  return x <= 0.f ? 0u : (x >= 255.f ? 255u : (uint32_t)x);
}

// One launch = n_steps env-steps for every env.  SOFT selects the SOFT-STE
// forward: joystick bits come from rounded float inputs, outputs are float,
// the RAM may be overridden from float values first, and the full state is
// checkpointed at the start of every segment of seg_steps steps.
// XM: the batch holds Superchip or E0 carts (blocks of other carts run with
// those features off all the same); FT: the whole TIA.  DR: deferred
// rasterisation (hard mode, one lane per env, no drawing code): the returned
// frames go to the raster logs p.dr_log / p.dr_hdr, drawn by the raster
// kernels; without screens nothing is logged.
template <bool SOFT, int T, bool BOOT, bool INSTR, bool XM, bool FT, bool DR = false>
__global__ void __launch_bounds__(128, 1) k_run(StepParams p) {
  extern __shared__ __align__(128) uint8_t smem[];
  // T threads per env (a compile-time constant, so T = 1 carries no replica
  // logic): thread tid is replica tid % T of env slot tid / T
  const int E = blockDim.x / T, tid = threadIdx.x, slot = tid / T, rank = tid % T;
  BlockSmem bs = carve_smem(smem, E, p.rom_stride, p.ram_words);
  const int4 bi = p.blocks[blockIdx.x];
  const int cart = bi.x;
  const uint32_t cb = p.cart_banks[cart];
  if (!stage_block(bs, p.dt, p.roms + (size_t)cart * p.rom_stride, cart_image_bytes(cb), p.err)) return;
  // lanes past the block's env count idle but stay for the warp reductions
  const bool active = slot < bi.z;
  const int env = active ? p.perm[bi.y + slot] : 0;
  const int n = p.n_envs;
  const uint32_t lanes = warp_lanes(E * T);
  Ctx c = make_ctx<XM, FT>(bs, E, slot, rank, T, cb, p.ystart);
  const bool lead = rank == 0;   // the replica that writes per-env results

  Regs r;
  uint32_t epf = 0, epi = 0;
  bool booting = false;
  if (active) {
    load_env(p.s, n, env, c, r);
    epf = p.s.epf[env];
    epi = p.s.epi[env];
    if (p.reset_all || (p.reset_mask && p.reset_mask[env])) {
      power_on(c, r);
      epf = 0;
      if (p.reset_all) epi = 0;
      booting = true;
    }
    if (SOFT && p.ram0) {
      uint32_t* w = reinterpret_cast<uint32_t*>(c.ram);
      const float* src = p.ram0 + (size_t)env * 128;
      for (int i = 0; i < 32; i++)
        w[i * c.E] = round_byte(src[4 * i]) | (round_byte(src[4 * i + 1]) << 8) |
                     (round_byte(src[4 * i + 2]) << 16) | (round_byte(src[4 * i + 3]) << 24);
    }
  } else {
    power_on(c, r);
  }

  typename std::conditional<SOFT, CountTape, typename std::conditional<DR, DeferTape, NoTape>::type>::type tape;
  if constexpr (DR) {
    tape.log = p.dr_log ? p.dr_log + (size_t)env * kRasterLogCap : nullptr;   // null: no screens, nothing logged
    tape.hdr = p.dr_hdr ? p.dr_hdr + (size_t)env * kRasterHdr : nullptr;
    tape.err = p.err;
    tape.n = 0;
  }
  if constexpr (SOFT) {
    tape.vregs = kVersionRegs | (p.graphics ? kGraphicsRegs | (FT ? kGraphicsRegsFT : 0ull) : 0ull);
    tape.ftgb = FT && p.graphics;
  }
  Render rd;
  rd.on = false;
  rd.cur = 0;
  rd.out_u8 = nullptr;
  rd.out_f32 = nullptr;
  rd.gs = nullptr;
  rd.grow = nullptr;
  rd.gline = -1;
  // One loop, one frame-loop call site (the interpreter is inlined once):
  // each turn is either a boot frame for the lanes that just powered on
  // (hard mode: n_noop NOOP frames, n_reset frames with RESET pressed, then
  // the episode's start NOOPs), with the other lanes idle, or an env-step.
  const uint32_t n_noop = (uint32_t)p.boot_noop, n_reset = (uint32_t)p.boot_reset;
  auto boot_len = [&](bool b) -> uint32_t {
    if (!BOOT || !b) return 0u;
    const uint32_t extra = p.start_noops ? p.start_noops[(size_t)env * p.n_start + epi % (uint32_t)p.n_start] : 0u;
    return n_noop + n_reset + extra;
  };
  uint32_t boot_left = boot_len(booting), boot_f = 0;
  int t = 0;
  while (true) {
    const bool boot_turn = BOOT && __any_sync(lanes, boot_left > 0);
    if (!boot_turn && t >= p.n_steps) break;
    Step st;
    st.status = 0;
    bool run_active;
    if (boot_turn) {
      run_active = boot_left > 0;
      if (run_active) {
        set_input_bits(r, 0);
        r.inpt4 |= (boot_f >= n_noop && boot_f < n_noop + n_reset) ? 0x100u : 0u;   // RESET held
      }
      st.frame_skip = 1;
      st.want_screen = false;
      rd.out_u8 = nullptr;
      rd.out_f32 = nullptr;
    } else {
      if constexpr (SOFT) {
        if (t % p.seg_steps == 0) {
          const int seg = t / p.seg_steps;
          if (seg > 0 && active && lead) {
            atomicMax(p.seg_counts + 2 * (seg - 1), tape.n);
            atomicMax(p.seg_counts + 2 * (seg - 1) + 1, tape.ncw);
          }
          tape.n = tape.ncw = 0;
          if (active && lead) store_env(soa_at(p.ckpt + (size_t)seg * kStateWords * n, n), n, env, c, r);
        }
      }
      uint32_t bits = 0;
      if (SOFT) {
        if (active) {
          const float* u = p.u + ((size_t)t * n + env) * 5;
          bits = (u[0] >= 0.5f ? 1u : 0u) | (u[1] >= 0.5f ? 2u : 0u) | (u[2] >= 0.5f ? 4u : 0u) |
                 (u[3] >= 0.5f ? 8u : 0u) | (u[4] >= 0.5f ? 16u : 0u);
          if (lead) p.act_bits[(size_t)t * n + env] = (uint8_t)bits;
        }
        set_input_bits(r, bits);
      } else {
        set_inputs(r, (p.actions && active) ? p.actions[(size_t)t * n + env] : 0u);
      }
      st.frame_skip = p.frame_skip;
      if (SOFT) {
        st.want_screen = p.screen_out_f != nullptr;
        rd.out_f32 = (p.screen_out_f && active)
                         ? p.screen_out_f + ((size_t)t * n + env) * (kScreenH * kScreenW) : nullptr;
      } else {
        st.want_screen = p.screen_out != nullptr;
        rd.out_u8 = (p.screen_out && active) ? p.screen_out + ((size_t)t * n + env) * (kScreenH * kScreenW) : nullptr;
      }
      run_active = active;
    }
    st.instr_left = p.step_instr;
    run_frames<INSTR>(c, r, rd, st, tape, run_active, lanes, p.sched_policy, p.sched_window);
    if (boot_turn) {
      if (boot_left > 0) {
        boot_left--;
        boot_f++;
        if (boot_left == 0) {
          r.inpt4 &= 0xFF;
          normalise_timer(r);
        }
      }
      continue;
    }
    if (active) {
      normalise_timer(r);
      if (SOFT) {
        if (p.ram_out_f) write_ram_f32(c, p.ram_out_f + ((size_t)t * n + env) * 128);
      } else {
        if (p.ram_out) write_ram(c, p.ram_out + ((size_t)t * n + env) * 128);
      }
      if (!SOFT && !INSTR && p.n_episodes > 0) {
        epf += (uint32_t)p.frame_skip;
        uint32_t len = p.ep_len[(size_t)env * p.n_episodes + (epi % (uint32_t)p.n_episodes)];
        if (epf >= len) {   // auto-reset: power on, boot before the next step
          st.status |= kStDone;
          power_on(c, r);
          epf = 0;
          epi++;
          boot_left = boot_len(true);
          boot_f = 0;
        }
      }
      if (p.status_out && lead) p.status_out[(size_t)t * n + env] = (uint8_t)st.status;
    }
    t++;
  }
  if (!active) return;
  if (!lead) return;
  if constexpr (SOFT) {
    if (p.n_steps > 0) {
      const int seg = (p.n_steps - 1) / p.seg_steps;
      atomicMax(p.seg_counts + 2 * seg, tape.n);
      atomicMax(p.seg_counts + 2 * seg + 1, tape.ncw);
    }
  }
  store_env(p.s, n, env, c, r);
  p.s.epf[env] = epf;
  p.s.epi[env] = epi;
}

// Launch one specialisation of the step kernel, with the shared memory the
// batch's ROM stride needs (above the default 48 KB for 16 and 32 KB carts).
template <class Kern>
static void launch_kernel(Kern kern, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const StepParams& p) {
  if (smem > 48u * 1024u) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kern<<<grid, block, smem, s>>>(p);
}

// The hard step kernel with deferred rasterisation: one lane per env,
// whatever the batch's threads per env (the drawing they would share is the
// raster kernel's).
template <bool XM, bool FT>
static int launch_run_dr(const StepParams& p, int n_blocks, int E, void* stream) {
  if (n_blocks <= 0) return 0;
  const size_t smem = step_smem_bytes(E, p.rom_stride, p.ram_words);
  cudaStream_t s = (cudaStream_t)stream;
  if (p.boot_frames) launch_kernel(k_run<false, 1, true, false, XM, FT, true>, dim3(n_blocks), dim3(E), smem, s, p);
  else launch_kernel(k_run<false, 1, false, false, XM, FT, true>, dim3(n_blocks), dim3(E), smem, s, p);
  return (int)cudaGetLastError();
}

template <bool SOFT, bool XM, bool FT>
static int launch_run(const StepParams& p, int n_blocks, int E, void* stream) {
  if (n_blocks <= 0) return 0;
  const dim3 grid(n_blocks), block(E * p.tpe);
  const size_t smem = step_smem_bytes(E, p.rom_stride, p.ram_words);
  cudaStream_t s = (cudaStream_t)stream;
  // instruction-granular steps draw nothing, so one lane per env serves them
  if (p.step_instr > 0) {
    launch_kernel(k_run<SOFT, 1, false, true, XM, FT>, grid, dim3(E), smem, s, p);
    return (int)cudaGetLastError();
  }
  // the boot sequence exists in the hard step kernel only when a batch asks
  // for it, so that default launches carry none of its code
  const bool boot = !SOFT && p.boot_frames;
  switch (p.tpe * 2 + (boot ? 1 : 0)) {
    case 2: launch_kernel(k_run<SOFT, 1, false, false, XM, FT>, grid, block, smem, s, p); break;
    case 4: launch_kernel(k_run<SOFT, 2, false, false, XM, FT>, grid, block, smem, s, p); break;
    case 8: launch_kernel(k_run<SOFT, 4, false, false, XM, FT>, grid, block, smem, s, p); break;
    case 16: launch_kernel(k_run<SOFT, 8, false, false, XM, FT>, grid, block, smem, s, p); break;
    case 3: launch_kernel(k_run<false, 1, true, false, XM, FT>, grid, block, smem, s, p); break;
    case 5: launch_kernel(k_run<false, 2, true, false, XM, FT>, grid, block, smem, s, p); break;
    case 9: launch_kernel(k_run<false, 4, true, false, XM, FT>, grid, block, smem, s, p); break;
    case 17: launch_kernel(k_run<false, 8, true, false, XM, FT>, grid, block, smem, s, p); break;
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

}  // namespace vcs
