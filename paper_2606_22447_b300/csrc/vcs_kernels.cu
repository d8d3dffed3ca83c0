// Step kernel launchers: lockstep emulation of many independent VCS envs
// (hard mode, and the SOFT-STE forward, which is the same machine on rounded
// inputs; the kernel template is in vcs_step.cuh), and the small kernels
// beside it (output digests, the integer-issue peak, the cartridge-RAM
// readout).  Batches with Superchip or E0 carts launch the instantiations of
// vcs_kernels_xm.cu.
#include <cuda_runtime.h>

#include "vcs_step.cuh"

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

// The Superchip's RAM of every env (state RAM words 32..63) as bytes
// [n_envs][128]: one thread per (env, word).
__global__ void k_cart_ram(const uint32_t* ram_words, int32_t n_envs, uint8_t* out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)n_envs * 32) return;
  const uint32_t e = (uint32_t)(i >> 5), w = (uint32_t)(i & 31);
  reinterpret_cast<uint32_t*>(out)[(size_t)e * 32 + w] = ram_words[(size_t)(32 + w) * n_envs + e];
}

int launch_cart_ram(const SoA& s, int32_t n_envs, uint8_t* out, void* stream) {
  const size_t n = (size_t)n_envs * 32;
  k_cart_ram<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(s.ram, n_envs, out);
  return (int)cudaGetLastError();
}

size_t step_smem_bytes(int E, uint32_t rom_stride, int ram_words) { return smem_bytes(E, rom_stride, ram_words); }

int launch_step(const StepParams& p, int n_blocks, int E, void* stream) {
  if (p.dr) return launch_step_dr(p, n_blocks, E, stream);
  if (p.full_tia) return launch_step_ft(p, n_blocks, E, stream);
  if (p.xmap) return launch_step_xm(p, n_blocks, E, stream);
  return launch_run<false, false, false>(p, n_blocks, E, stream);
}

int launch_soft_forward(const StepParams& p, int n_blocks, int E, void* stream) {
  if (p.full_tia) return launch_soft_forward_ft(p, n_blocks, E, stream);
  if (p.xmap) return launch_soft_forward_xm(p, n_blocks, E, stream);
  return launch_run<true, false, false>(p, n_blocks, E, stream);
}

}  // namespace vcs
