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

// ---------------------------------------------------------------------------
// decode table (MOS 6500 instruction set: addressing mode, base cycles)
// ---------------------------------------------------------------------------

void build_decode_tables(DecodeTables* t) {
  for (int i = 0; i < 256; i++) {
    t->mode_cyc[i] = AM_JAM | (1 << 4);
    t->cls_op[i] = CL_OTHER | (OP_JAM << 2);
  }
  auto set = [&](int op, int mode, int cyc, int cls, int id) {
    t->mode_cyc[op] = (uint8_t)(mode | (cyc << 4));
    t->cls_op[op] = (uint8_t)(cls | (id << 2));
  };
  // the regular "cc = 01" column: ORA AND EOR ADC STA LDA CMP SBC
  const int m01[8] = {AM_INX, AM_ZP, AM_IMM, AM_ABS, AM_INY, AM_ZPX, AM_ABY, AM_ABX};
  const int c01[8] = {6, 3, 2, 4, 5, 4, 4, 4};
  const int id01[8] = {OP_ORA, OP_AND, OP_EOR, OP_ADC, OP_STA, OP_LDA, OP_CMP, OP_SBC};
  for (int aaa = 0; aaa < 8; aaa++)
    for (int bbb = 0; bbb < 8; bbb++) {
      int op = (aaa << 5) | (bbb << 2) | 1;
      int cyc = c01[bbb];
      if (aaa == 4) {            // STA: no immediate; indexed stores pay the fix-up cycle
        if (m01[bbb] == AM_IMM) continue;
        if (m01[bbb] == AM_INY) cyc = 6;
        if (m01[bbb] == AM_ABX || m01[bbb] == AM_ABY) cyc = 5;
        set(op, m01[bbb], cyc, CL_STORE, OP_STA);
      } else {
        set(op, m01[bbb], cyc, CL_READ, id01[aaa]);
      }
    }
  // shifts, rotates, DEC, INC
  const int rmw[6] = {0x00, 0x20, 0x40, 0x60, 0xC0, 0xE0};
  const int idm[6] = {OP_ASL, OP_ROL, OP_LSR, OP_ROR, OP_DEC, OP_INC};
  const int ida[4] = {OP_ASLA, OP_ROLA, OP_LSRA, OP_RORA};
  for (int k = 0; k < 6; k++) {
    int b = rmw[k];
    if (k < 4) set(b + 0x0A, AM_ACC, 2, CL_OTHER, ida[k]);
    set(b + 0x06, AM_ZP, 5, CL_RMW, idm[k]);
    set(b + 0x16, AM_ZPX, 6, CL_RMW, idm[k]);
    set(b + 0x0E, AM_ABS, 6, CL_RMW, idm[k]);
    set(b + 0x1E, AM_ABX, 7, CL_RMW, idm[k]);
  }
  set(0xA2, AM_IMM, 2, CL_READ, OP_LDX); set(0xA6, AM_ZP, 3, CL_READ, OP_LDX);
  set(0xB6, AM_ZPY, 4, CL_READ, OP_LDX); set(0xAE, AM_ABS, 4, CL_READ, OP_LDX);
  set(0xBE, AM_ABY, 4, CL_READ, OP_LDX);
  set(0xA0, AM_IMM, 2, CL_READ, OP_LDY); set(0xA4, AM_ZP, 3, CL_READ, OP_LDY);
  set(0xB4, AM_ZPX, 4, CL_READ, OP_LDY); set(0xAC, AM_ABS, 4, CL_READ, OP_LDY);
  set(0xBC, AM_ABX, 4, CL_READ, OP_LDY);
  set(0x86, AM_ZP, 3, CL_STORE, OP_STX); set(0x96, AM_ZPY, 4, CL_STORE, OP_STX); set(0x8E, AM_ABS, 4, CL_STORE, OP_STX);
  set(0x84, AM_ZP, 3, CL_STORE, OP_STY); set(0x94, AM_ZPX, 4, CL_STORE, OP_STY); set(0x8C, AM_ABS, 4, CL_STORE, OP_STY);
  set(0xE0, AM_IMM, 2, CL_READ, OP_CPX); set(0xE4, AM_ZP, 3, CL_READ, OP_CPX); set(0xEC, AM_ABS, 4, CL_READ, OP_CPX);
  set(0xC0, AM_IMM, 2, CL_READ, OP_CPY); set(0xC4, AM_ZP, 3, CL_READ, OP_CPY); set(0xCC, AM_ABS, 4, CL_READ, OP_CPY);
  set(0x24, AM_ZP, 3, CL_READ, OP_BIT); set(0x2C, AM_ABS, 4, CL_READ, OP_BIT);
  for (int op : {0x10, 0x30, 0x50, 0x70, 0x90, 0xB0, 0xD0, 0xF0}) set(op, AM_REL, 2, CL_OTHER, OP_BRANCH);
  set(0x4C, AM_ABS, 3, CL_OTHER, OP_JMP); set(0x6C, AM_IND, 5, CL_OTHER, OP_JMPI); set(0x20, AM_IND, 6, CL_OTHER, OP_JSR);
  set(0x60, AM_IMP, 6, CL_OTHER, OP_RTS); set(0x40, AM_IMP, 6, CL_OTHER, OP_RTI); set(0x00, AM_IMP, 7, CL_OTHER, OP_BRK);
  set(0x48, AM_IMP, 3, CL_OTHER, OP_PHA); set(0x08, AM_IMP, 3, CL_OTHER, OP_PHP);
  set(0x68, AM_IMP, 4, CL_OTHER, OP_PLA); set(0x28, AM_IMP, 4, CL_OTHER, OP_PLP);
  const int imp_ops[18][2] = {{0x18, OP_CLC}, {0x38, OP_SEC}, {0x58, OP_CLI}, {0x78, OP_SEI}, {0xB8, OP_CLV},
                              {0xD8, OP_CLD}, {0xF8, OP_SED}, {0xEA, OP_NOP}, {0xAA, OP_TAX}, {0x8A, OP_TXA},
                              {0xA8, OP_TAY}, {0x98, OP_TYA}, {0xBA, OP_TSX}, {0x9A, OP_TXS}, {0xE8, OP_INX},
                              {0xCA, OP_DEX}, {0xC8, OP_INY}, {0x88, OP_DEY}};
  for (auto& q : imp_ops) set(q[0], AM_IMP, 2, CL_OTHER, q[1]);
}

// Counts instructions and colour-register writes per checkpoint segment (the
// soft forward sizes the backward's tape with these).
struct CountTape {
  static constexpr bool kAcc = false;
  uint32_t n = 0, ncw = 0;
  __device__ __forceinline__ void rec(uint32_t, uint32_t, uint32_t) { n++; }
  __device__ __forceinline__ void colour_write(int) { ncw++; }
  __device__ __forceinline__ void pixels(float, float, float) {}
};

__device__ __forceinline__ uint32_t round_byte(float v) {
  float x = rintf(v);
  return x <= 0.f ? 0u : (x >= 255.f ? 255u : (uint32_t)x);
}

// One launch = n_steps env-steps for every env.  SOFT selects the SOFT-STE
// forward: joystick bits come from rounded float inputs, outputs are float,
// the RAM may be overridden from float values first, and the full state is
// checkpointed at the start of every segment of seg_steps steps.
template <bool SOFT>
__global__ void __launch_bounds__(128) k_run(StepParams p) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int E = blockDim.x, tid = threadIdx.x;
  BlockSmem bs = carve_smem(smem, E);
  const int4 bi = p.blocks[blockIdx.x];
  const int cart = bi.x;
  const uint32_t f8 = p.cart_f8[cart];
  if (!stage_block(bs, p.dt, p.roms + (size_t)cart * 8192, f8 ? 8192u : 4096u)) {
    if (tid == 0) atomicExch(p.err, 1);
    return;
  }
  // lanes past the block's env count idle but stay for the warp reductions
  const bool active = tid < bi.z;
  const int env = active ? p.perm[bi.y + tid] : 0;
  const int n = p.n_envs;
  const uint32_t lanes = warp_lanes(E);
  Ctx c = make_ctx(bs, E, tid, f8, p.ystart);

  Regs r;
  uint32_t epf = 0, epi = 0;
  if (active) {
    load_env(p.s, n, env, c, r);
    epf = p.s.epf[env];
    epi = p.s.epi[env];
    if (p.reset_all || (p.reset_mask && p.reset_mask[env])) {
      power_on(c, r);
      epf = 0;
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
  for (int t = 0; t < p.n_steps; t++) {
    if constexpr (SOFT) {
      if (t % p.seg_steps == 0) {
        const int seg = t / p.seg_steps;
        if (seg > 0 && active) {
          atomicMax(p.seg_counts + 2 * (seg - 1), tape.n);
          atomicMax(p.seg_counts + 2 * (seg - 1) + 1, tape.ncw);
        }
        tape.n = tape.ncw = 0;
        if (active) store_env(soa_at(p.ckpt + (size_t)seg * kStateWords * n, n), n, env, c, r);
      }
    }
    uint32_t bits = 0;
    if (SOFT) {
      if (active) {
        const float* u = p.u + ((size_t)t * n + env) * 5;
        bits = (u[0] >= 0.5f ? 1u : 0u) | (u[1] >= 0.5f ? 2u : 0u) | (u[2] >= 0.5f ? 4u : 0u) |
               (u[3] >= 0.5f ? 8u : 0u) | (u[4] >= 0.5f ? 16u : 0u);
        p.act_bits[(size_t)t * n + env] = (uint8_t)bits;
      }
      set_input_bits(r, bits);
    } else {
      set_inputs(r, (p.actions && active) ? p.actions[(size_t)t * n + env] : 0u);
    }
    Step st;
    st.frame_skip = p.frame_skip;
    st.status = 0;
    if (SOFT) {
      st.want_screen = p.screen_out_f != nullptr;
      rd.out_f32 = (p.screen_out_f && active)
                       ? p.screen_out_f + ((size_t)t * n + env) * (kScreenH * kScreenW) : nullptr;
    } else {
      st.want_screen = p.screen_out != nullptr;
      rd.out_u8 = (p.screen_out && active) ? p.screen_out + ((size_t)t * n + env) * (kScreenH * kScreenW) : nullptr;
    }
    run_frames(c, r, rd, st, tape, active, lanes, p.sched_policy, p.sched_window);
    if (!active) continue;
    normalise_timer(r);
    if (SOFT) {
      if (p.ram_out_f) write_ram_f32(c, p.ram_out_f + ((size_t)t * n + env) * 128);
    } else {
      if (p.ram_out) write_ram(c, p.ram_out + ((size_t)t * n + env) * 128);
    }
    if (!SOFT && p.n_episodes > 0) {
      epf += (uint32_t)p.frame_skip;
      uint32_t len = p.ep_len[(size_t)env * p.n_episodes + (epi % (uint32_t)p.n_episodes)];
      if (epf >= len) {
        st.status |= kStDone;
        power_on(c, r);
        epf = 0;
        epi++;
      }
    }
    if (p.status_out) p.status_out[(size_t)t * n + env] = (uint8_t)st.status;
  }
  if (!active) return;
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

size_t step_smem_bytes(int E) { return smem_bytes(E); }

int launch_step(const StepParams& p, int n_blocks, int E, void* stream) {
  if (n_blocks <= 0) return 0;
  k_run<false><<<n_blocks, E, step_smem_bytes(E), (cudaStream_t)stream>>>(p);
  return (int)cudaGetLastError();
}

int launch_soft_forward(const StepParams& p, int n_blocks, int E, void* stream) {
  if (n_blocks <= 0) return 0;
  k_run<true><<<n_blocks, E, step_smem_bytes(E), (cudaStream_t)stream>>>(p);
  return (int)cudaGetLastError();
}

}  // namespace vcs
