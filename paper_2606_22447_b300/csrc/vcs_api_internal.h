// Host-side batch object shared by the C-ABI translation units.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/vcs.h"
#include "vcs_kernels.cuh"

struct vcs_batch {
  int32_t n_envs = 0, n_carts = 0, E = 32, n_blocks = 0, sms = 148;
  vcs_config cfg{};
  std::vector<int32_t> env_cart, perm_host;
  std::vector<uint8_t> mapper;
  std::vector<uint32_t> rom_size;
  // device memory owned by the batch
  uint32_t* state = nullptr;      // kStateWords x n_envs
  uint8_t* roms = nullptr;        // n_carts x rom_stride
  uint32_t rom_stride = 8192;     // bytes per cart image: the largest image, at least 8 KB
  uint8_t* cart_banks = nullptr;  // bank byte of each cart: 4 KB banks of a bank-switched cart, else 0,
                                  // | kCartSC for a Superchip cart | kCartE0 for an E0 cart
  int32_t ram_words = 32;         // RAM words per env in shared memory: 64 when a cart is Superchip
  int32_t xmap = 0;               // a cart is Superchip or E0: launch the kernels built for them
  uint8_t* cart_2k = nullptr;
  int32_t* env_cart_dev = nullptr;
  int32_t* cart_begin = nullptr;  // [n_carts + 1] first perm slot of each cart
  vcs::DecodeTables* dt = nullptr;
  int4* blocks = nullptr;
  int32_t* perm = nullptr;
  // the backward's blocks when envs_per_block is above what its shared
  // memory holds (kBwdMaxEnvsPerBlock envs; same permutation), else null
  int4* bwd_blocks = nullptr;
  int32_t bwd_n_blocks = 0, bwd_E = 0;
  // blocks of kWideEnvsPerBlock envs (same permutation): the backward's
  // recompute of a large group of segments, one lane per env
  int4* wide_blocks = nullptr;
  int32_t wide_n_blocks = 0;
  // blocks of kWideFwdEnvsPerBlock envs (same permutation): the soft
  // forward without screens, one lane per env
  int4* wide_fwd_blocks = nullptr;
  int32_t wide_fwd_n_blocks = 0;
  // deferred rasterisation (vcs_raster.cu): per env a log of the returned
  // frame's picture-register writes and a header, made at the first step
  // that returns screens
  uint32_t* dr_log = nullptr;      // [n_envs][kRasterLogCap]
  uint32_t* dr_hdr = nullptr;      // [n_envs][kRasterHdr]
  // kernel timing (vcs_time_kernels): three events per timed launch (before
  // the step kernel, after it, after the raster kernel), reused
  bool timing = false;
  std::vector<cudaEvent_t> tk_events;
  size_t tk_used = 0;
  unsigned long long* tk_entries = nullptr;   // device: log entries the timed raster launches drew
  uint32_t* ep_len = nullptr;
  int32_t n_episodes = 0;
  uint8_t* start_noops = nullptr;  // [n_envs][n_start] NOOP frames starting each episode
  int32_t n_start = 0;
  uint32_t sched_policy = 0;       // warp scheduling policy (see vcs_config)
  uint32_t sched_window = 4;       // time window for policy 1 (cycles)
  int32_t steps_per_launch = 0;    // vcs_rollout launch split (0 = one launch)
  int32_t tpe = 1;                 // threads per env
  uint32_t geometry_gen = 0;       // bumped whenever blocks / perm are rebuilt
  int32_t* err = nullptr;
  // staging for the host-pointer entry points: vcs_step_host uses set 0,
  // vcs_rollout_host alternates sets 0 and 1
  uint8_t* h_actions = nullptr;
  uint8_t* h_ram = nullptr;
  uint8_t* h_screen = nullptr;
  uint8_t* h2_actions = nullptr;
  uint8_t* h2_ram = nullptr;
  uint8_t* h2_screen = nullptr;
  uint8_t* h_status[2] = {nullptr, nullptr};
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_kernel[2] = {nullptr, nullptr}, ev_copy[2] = {nullptr, nullptr};
  std::string last_error;
  vcs::SoA soa() const;
};

namespace vcs {
SoA soa_of(uint32_t* state, int32_t n_envs);
}

vcs_status vcs_fail(vcs_batch* b, vcs_status st, const char* fmt, ...);
vcs_status vcs_cuda_fail(vcs_batch* b, cudaError_t e, const char* what);
vcs::StepParams vcs_base_params(vcs_batch* b);

// Largest envs per block whose backward shared memory (about 9.7 KB +
// 1.9 KB per env) fits in a block.
constexpr int kBwdMaxEnvsPerBlock = 64;
// One lane per env: the recompute of large segment groups runs in blocks of
// kWideEnvsPerBlock envs, the soft forward without screens in blocks of
// kWideFwdEnvsPerBlock (each the fastest of 8 / 16 / 32 / 64 / 128 on 4096
// envs of the 4K / F8 mix over 2,048 frames).
constexpr int kWideEnvsPerBlock = 64;
constexpr int kWideFwdEnvsPerBlock = 128;

// The backward's launch geometry (its own block table past
// kBwdMaxEnvsPerBlock envs per block).
inline void vcs_bwd_geometry(const vcs_batch* b, const int4** blocks, int* n_blocks, int* E) {
  *blocks = b->bwd_blocks ? b->bwd_blocks : b->blocks;
  *n_blocks = b->bwd_blocks ? b->bwd_n_blocks : b->n_blocks;
  *E = b->bwd_blocks ? b->bwd_E : b->E;
}
