// Step kernel: lockstep emulation of many independent VCS envs (hard mode,
// and the SOFT-STE forward, which is the same machine on rounded inputs).
//
// One thread per env, one block per run of envs of the same cartridge (the
// host groups envs by cart), so the block stages exactly one ROM image into
// shared memory.  The image is brought in by one TMA bulk copy
// (cp.async.bulk, completion tracked by an mbarrier with a bounded wait).
// Each thread keeps its machine in registers for the whole launch, its RAM
// and scanline buffer in shared memory, and writes RAM and finished
// scanlines (16-byte stores) straight to the caller's buffers.
#include <cuda_runtime.h>

#include <type_traits>

#include "vcs_exec.cuh"
#include "vcs_kernels.cuh"
#include "vcs_run.cuh"

namespace vcs {

// Decode table for the paths that decode at run time (the operand fetch
// outside the cartridge window), built from op_info.

void build_decode_tables(DecodeTables* t) {
  for (uint32_t op = 0; op < 256; op++) {
    const OpInfo i = op_info(op);
    t->mode_cyc[op] = (uint8_t)(i.mode | (i.cyc << 4));
    t->cls_op[op] = (uint8_t)(i.cls | (i.id << 2));
  }
}

// Counts instructions and colour-register writes per checkpoint segment (the
// soft forward sizes the backward's tape with these).
struct CountTape {
  static constexpr bool kAcc = false;
  uint32_t n = 0, ncw = 0;
  __device__ __forceinline__ void rec(uint32_t, uint32_t, uint32_t) { n++; }
  static constexpr bool sampler = false;
  __device__ __forceinline__ void version_write(uint32_t reg) { ncw += (uint32_t)(kVersionRegs >> reg) & 1u; }
  __device__ __forceinline__ void pixels(float, float, float, float) {}
};

__device__ __forceinline__ uint32_t round_byte(float v) {
  float x = rintf(v);
  return x <= 0.f ? 0u : (x >= 255.f ? 255u : (uint32_t)x);
}

// One launch = n_steps env-steps for every env.  SOFT selects the SOFT-STE
// forward: joystick bits come from rounded float inputs, outputs are float,
// the RAM may be overridden from float values first, and the full state is
// checkpointed at the start of every segment of seg_steps steps.
template <bool SOFT, int T, bool BOOT, bool INSTR = false>
__global__ void __launch_bounds__(128, 1) k_run(StepParams p) {
  extern __shared__ __align__(128) uint8_t smem[];
  // T threads per env (a compile-time constant, so T = 1 carries no replica
  // logic): thread tid is replica tid % T of env slot tid / T
  const int E = blockDim.x / T, tid = threadIdx.x, slot = tid / T, rank = tid % T;
  BlockSmem bs = carve_smem(smem, E, p.rom_stride);
  const int4 bi = p.blocks[blockIdx.x];
  const int cart = bi.x;
  const uint32_t nb = p.cart_banks[cart];
  if (!stage_block(bs, p.dt, p.roms + (size_t)cart * p.rom_stride, nb ? nb * 4096u : 4096u)) {
    if (tid == 0) atomicExch(p.err, 1);
    return;
  }
  // lanes past the block's env count idle but stay for the warp reductions
  const bool active = slot < bi.z;
  const int env = active ? p.perm[bi.y + slot] : 0;
  const int n = p.n_envs;
  const uint32_t lanes = warp_lanes(E * T);
  Ctx c = make_ctx(bs, E, slot, rank, T, nb, p.ystart);
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

  typename std::conditional<SOFT, CountTape, NoTape>::type tape;
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

// ---------------------------------------------------------------------------
// Output digests for parity at scale: for each (step, env) the sum mod 2^64
// of F((i << 32) | w_i) over the 32-bit little-endian words w_i of the RAM
// row followed by the screen (F the splitmix64 finaliser).  One warp per
// digest; the sum is order-free, so lanes take strided words and reduce.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t digest_fin(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_digest(const uint8_t* ram, const uint8_t* screen, uint64_t n_digests, uint64_t* out) {
  const uint64_t d = (uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const uint32_t lane = threadIdx.x & 31;
  if (d >= n_digests) return;   // whole warps leave together
  uint64_t acc = 0;
  const uint32_t rw = reinterpret_cast<const uint32_t*>(ram + d * 128)[lane];   // 32 RAM words
  acc += digest_fin(((uint64_t)lane << 32) | rw);
  if (screen) {
    const uint4* sp = reinterpret_cast<const uint4*>(screen + d * (kScreenH * kScreenW));
    for (uint32_t j = lane; j < kScreenH * kScreenW / 16; j += 32) {
      const uint4 v = sp[j];
      const uint64_t i0 = 32 + 4 * (uint64_t)j;
      acc += digest_fin(((i0 + 0) << 32) | v.x) + digest_fin(((i0 + 1) << 32) | v.y) +
             digest_fin(((i0 + 2) << 32) | v.z) + digest_fin(((i0 + 3) << 32) | v.w);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
  if (lane == 0) out[d] = acc;
}

int launch_digest(const uint8_t* ram, const uint8_t* screen, uint64_t n_digests, uint64_t* out, void* stream) {
  if (n_digests == 0) return 0;
  const uint64_t blocks = (n_digests + 7) / 8;
  k_digest<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(ram, screen, n_digests, out);
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Integer issue peak: every thread runs eight independent chains of 32-bit
// add, shift and logic operations (the instruction kinds the emulator issues
// most), at full occupancy, so the measured rate is the SMs' integer
// throughput.  Each chain does nine operations per loop turn as written (72
// per thread); the compiler fuses some of them (three-input adds and logic),
// as it does in the emulator.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_int_peak(uint32_t seed, int32_t iters, uint32_t* sink) {
  uint32_t a[8];
#pragma unroll
  for (int k = 0; k < 8; k++) a[k] = seed + 0x9E3779B9u * (threadIdx.x * 8 + k + 1);
  const uint32_t m = seed | 1u;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < 8; k++) {
      a[k] = a[k] + (a[k] >> 3) + m;     // add of three operands
      a[k] = (a[k] ^ m) & (a[k] | 0x5A5A5A5Au);   // a three-input logic operation
      a[k] = a[k] + 0x3C6EF372u;
      a[k] = a[k] ^ (a[k] << 5);
    }
  }
  uint32_t x = 0;
#pragma unroll
  for (int k = 0; k < 8; k++) x ^= a[k];
  if (x == seed) sink[blockIdx.x] = x;   // keeps the work alive; practically never taken
}

int launch_int_peak(int sms, int32_t iters, uint32_t* sink, void* stream) {
  k_int_peak<<<sms * 2, 1024, 0, (cudaStream_t)stream>>>(0x1234567u, iters, sink);
  return (int)cudaGetLastError();
}

size_t step_smem_bytes(int E, uint32_t rom_stride) { return smem_bytes(E, rom_stride); }

// Launch one specialisation of the step kernel, with the shared memory the
// batch's ROM stride needs (above the default 48 KB for 16 and 32 KB carts).
template <class Kern>
static void launch_kernel(Kern kern, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const StepParams& p) {
  if (smem > 48u * 1024u) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kern<<<grid, block, smem, s>>>(p);
}

template <bool SOFT>
static int launch_run(const StepParams& p, int n_blocks, int E, void* stream) {
  if (n_blocks <= 0) return 0;
  const dim3 grid(n_blocks), block(E * p.tpe);
  const size_t smem = step_smem_bytes(E, p.rom_stride);
  cudaStream_t s = (cudaStream_t)stream;
  // instruction-granular steps draw nothing, so one lane per env serves them
  if (p.step_instr > 0) {
    launch_kernel(k_run<SOFT, 1, false, true>, grid, dim3(E), smem, s, p);
    return (int)cudaGetLastError();
  }
  // the boot sequence exists in the hard step kernel only when a batch asks
  // for it, so that default launches carry none of its code
  const bool boot = !SOFT && p.boot_frames;
  switch (p.tpe * 2 + (boot ? 1 : 0)) {
    case 2: launch_kernel(k_run<SOFT, 1, false>, grid, block, smem, s, p); break;
    case 4: launch_kernel(k_run<SOFT, 2, false>, grid, block, smem, s, p); break;
    case 8: launch_kernel(k_run<SOFT, 4, false>, grid, block, smem, s, p); break;
    case 16: launch_kernel(k_run<SOFT, 8, false>, grid, block, smem, s, p); break;
    case 3: launch_kernel(k_run<false, 1, true>, grid, block, smem, s, p); break;
    case 5: launch_kernel(k_run<false, 2, true>, grid, block, smem, s, p); break;
    case 9: launch_kernel(k_run<false, 4, true>, grid, block, smem, s, p); break;
    case 17: launch_kernel(k_run<false, 8, true>, grid, block, smem, s, p); break;
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

int launch_step(const StepParams& p, int n_blocks, int E, void* stream) {
  return launch_run<false>(p, n_blocks, E, stream);
}

int launch_soft_forward(const StepParams& p, int n_blocks, int E, void* stream) {
  return launch_run<true>(p, n_blocks, E, stream);
}

}  // namespace vcs
