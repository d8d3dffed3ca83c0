/*
 * libvcs: batched Atari VCS emulation on one GPU (sm_103a), hard and soft.
 *
 * The machine is the paper's VCS (Section 2.2, the architecture figure): a
 * 6507 CPU executing a cartridge ROM (2K, 4K, the F8 / F6 / F4 bank-switched
 * formats, their Superchip variants with 128 B of cartridge RAM, E0 or FE), the
 * RIOT (128 B of RAM, interval timer, joystick and console-switch ports) and
 * the TIA, which turns register writes into 160x210 palette-index frames one
 * colour clock at a time (player 0, playfield and background by default;
 * the whole TIA with vcs_config.full_tia).  Many independent machines run in lockstep, one
 * per CUDA thread.
 *
 * Modes (supplement, table of execution modes):
 *  - HARD: bit-exact integer emulation (vcs_step, vcs_rollout);
 *  - SOFT-STE: the same forward pass, bit-exact with HARD at every finite
 *    temperature (Theorem 1), plus a hand-written backward pass giving
 *    surrogate gradients (Corollary 1) with respect to ROM bytes, the RAM
 *    at the start of the rollout and the per-step joystick inputs.
 *
 * Conventions
 *  - Every call returns a vcs_status; 0 is success.  No C++ exception
 *    crosses this interface.  vcs_last_error() describes the last failure
 *    of a batch in words.
 *  - "device pointer" arguments are CUDA device addresses owned by the
 *    caller (for instance PyTorch tensors) and must stay valid until the
 *    work queued on `stream` has finished.  "host pointer" arguments are
 *    read or written before the call returns.
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy stream.
 *  - The library owns the machine state, its ROM copies, checkpoints and
 *    tapes.  ROMs are copied at creation, so the caller may free them.
 *  - One batch must not be used from two host threads or streams at once.
 *  - Env order is the caller's: output row e always belongs to env e.
 */
#ifndef VCS_H
#define VCS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VCS_OK = 0,
  VCS_ERR_ARG = 1,       /* bad argument (null pointer, size, range) */
  VCS_ERR_ROM_SIZE = 2,  /* ROM size does not match its mapper */
  VCS_ERR_MAPPER = 3,    /* unknown mapper code */
  VCS_ERR_CUDA = 4,      /* a CUDA call failed; see vcs_last_error */
  VCS_ERR_OOM = 5,       /* device allocation failed */
  VCS_ERR_WATCHDOG = 6,  /* a device wait gave up (the batch is unusable) */
  VCS_ERR_STATE = 7      /* call out of order (e.g. backward of a freed tape) */
} vcs_status;

/* Cartridge formats: 2K and 4K images; F8 (8 KB), F6 (16 KB) and F4 (32 KB)
 * bank-switched in 4 KB banks, an access (read or write) to hotspot j
 * ($1FF8 + j for F8, $1FF6 + j for F6, $1FF4 + j for F4) selecting bank j,
 * power-on in the last bank; and their Superchip variants F8SC, F6SC, F4SC
 * (the paper's mapper list, Section 4): the same banking plus 128 bytes of
 * cartridge RAM, written at $1000-$107F and read at $1080-$10FF of the
 * cartridge window in every bank (a read of the write port returns the ROM
 * byte there; a write to the read port does nothing), zero at power-on. */
/* E0 (8 KB, eight 1 KB slices): the cartridge window is four 1 KB segments;
 * an access to $1FE0+j, $1FE8+j or $1FF0+j maps slice j into segment 0, 1
 * or 2, segment 3 always shows slice 7, and power-on shows slices 4, 5, 6.
 * A relaxed ROM read's tensor is the slice its segment shows. */
/* FE (8 KB, two 4 KB banks; the conformance table of Section 5 counts it
 * among the implemented formats): the cartridge takes the bank from bit 5
 * of the bus byte that follows an access to $01FE.  Reading: the accesses
 * modelled are a JSR made with the stack pointer at $FF (it pushes the
 * return address's low byte to $01FE, then fetches the target's high byte)
 * and an RTS made with it at $FD (it pulls the low byte from $01FE, then
 * the high byte); bit 5 set ($Fx) shows the image's first 4 KB, clear ($Dx)
 * the second; power-on shows the first.  A relaxed ROM read's tensor is
 * the current 4 KB bank. */
enum { VCS_MAPPER_2K = 0, VCS_MAPPER_4K = 1, VCS_MAPPER_F8 = 2, VCS_MAPPER_F6 = 3, VCS_MAPPER_F4 = 4,
       VCS_MAPPER_F8SC = 5, VCS_MAPPER_F6SC = 6, VCS_MAPPER_F4SC = 7, VCS_MAPPER_E0 = 8,
       VCS_MAPPER_FE = 9 };

/* Per-env status bits reported by vcs_step / vcs_rollout. */
enum {
  VCS_ENV_WATCHDOG = 1,  /* a frame was ended by the 512-scanline cap */
  VCS_ENV_JAMMED = 2,    /* the CPU met an opcode outside the documented set and the
                            paper's 38 extra bytes, and halted */
  VCS_ENV_DONE = 4       /* the episode ended at this step (auto-reset) */
};

#define VCS_SCREEN_H 210
#define VCS_SCREEN_W 160
#define VCS_RAM 128
#define VCS_ROM_MAX 32768

typedef struct vcs_config {
  float alpha;              /* branch-gate sharpness (Eq. branch), default 6 */
  int32_t ystart;           /* first scanline of screen row 0, default 34 */
  int32_t boot_noop_frames; /* boot: NOOP frames after each power-on, default 0
                               (the paper's protocol: 60) */
  int32_t boot_reset_frames;/* boot: then frames with the console RESET switch
                               pressed (SWCHB bit 0 low), default 0 (the
                               paper: 4) */
  int32_t envs_per_block;   /* 0 = automatic; else 8, 16, 32, 64 or 128 */
  int32_t segment_frames;   /* soft checkpoint interval in frames, default 64 */
  int32_t sched_policy;     /* which lanes of a warp execute each iteration:
                               0 = the earliest frame's lowest program counter
                               (default), 1 = emulated time within
                               sched_window cycles of the earliest lane */
  int32_t sched_window;     /* window of policy 1 in CPU cycles, -1 = any;
                               default 4 */
  int32_t steps_per_launch; /* vcs_rollout: env-steps per kernel launch, 0 =
                               the whole rollout in one launch (default) */
  int32_t threads_per_env;  /* 0 = automatic (1); else 1, 2, 4 or 8 with
                               envs_per_block x threads_per_env <= 128: that
                               many lanes run each env in lockstep and share
                               its rendering, output and pixel-gradient work
                               (4 suits soft rollouts with screen losses,
                               whose backward sums every frame's pixels) */
  int32_t position_sampler; /* 1 = the differentiable position sampler of
                               Section 3 in soft backward passes: player 0's
                               position carries a deviation (zero at each
                               RESP0; an HMOVE adds minus a sixteenth of
                               HMP0's deviation) and each drawn pixel within
                               one column of a sprite edge adds
                               (C_P0 - C_under)(b(d-1) - b(d+1))/2 times its
                               gradient to it, d = x - pos and b the player's
                               pixel bits (the symmetric derivative of the
                               triangular-kernel coverage).  0 = off
                               (default).  Forward outputs do not depend on it. */
  int32_t step_instructions;/* 0 = frame steps (default): a step runs
                               frame_skip frames.  n > 0 = instruction-
                               granular steps, the paper's throughput unit
                               (Section 6, one step = one emulated
                               instruction): every step of vcs_step,
                               vcs_rollout and vcs_soft_rollout runs n
                               instruction slots (an executed instruction, or
                               a jammed CPU's idle to the next line), frames
                               ending inside a step as they come, and
                               frame_skip is ignored.  Such steps return RAM
                               only: screen outputs, screen gradients and
                               screen loss weights, boot frames, start NOOPs
                               and episode tables are refused
                               (VCS_ERR_ARG), and soft checkpoints are taken
                               every segment_frames steps. */
  int32_t tape_budget_mb;   /* device memory in MB for the backward's tapes,
                               0 = a quarter of the free device memory at the
                               first vcs_backward (default).  The backward recomputes as
                               many checkpoint segments at once as fit (at
                               least one), then sweeps them last to first:
                               more segments per group, more parallel
                               recompute.  vcs_backward_static uses its fixed
                               array instead. */
  int32_t full_tia;         /* 1 = the whole TIA (Section 2.2): player 1, the
                               missiles and the ball (NUSIZ copies and sizes,
                               REFP, VDEL, RESMP, HMOVE of every object),
                               score mode and collision latches (CXCLR; read
                               in D7 / D6 of CXM0P .. CXPPMM), COLUP1 as a
                               fourth differentiable colour; 0 (default) = the
                               subset machine: player 0, playfield and
                               background, the other object registers
                               ignored and the collision registers read 0.
                               The subset runs in kernels without the rest
                               (about a quarter faster on the synthetic
                               carts). */
  int32_t graphics_bits;    /* 1 = the graphics-bit surrogate of Section 3.1
                               (with the switch stored, graphics bits are
                               differentiable) in soft backward passes: each
                               drawn pixel adds (C_with - C_without) times
                               its gradient to the byte of each graphics bit
                               deciding an object's coverage there, C_with
                               and C_without being the pixel's colours with
                               that bit forced to 1 and to 0 (the bit's
                               derivative with respect to its byte is 1):
                               GRP0 over player 0's span and the playfield
                               register (PF0, PF1 or PF2) of the column; with
                               full_tia also GRP1 over player 1's copies,
                               ENAM0 / ENAM1 and ENABL over the missiles' and
                               the ball's spans, a delayed graphic's sum going
                               to the value its copy took.  The written values
                               of these registers then receive the sums.
                               0 = off (default).  Forward outputs do not
                               depend on it. */
  int32_t inline_render;    /* 0 (default) = deferred rasterisation for hard
                               frame steps that return screens: the step
                               kernel logs the returned frame's TIA writes
                               that drawing depends on (after the registers'
                               state when the frame began) and a raster
                               kernel draws all scanlines of all envs in
                               parallel from the logs, one step per launch;
                               the logs hold 67 KB per env, made at the first
                               such step (if the device cannot hold them the
                               batch switches to 1).  1 = the step kernel
                               draws the frame itself as it runs.  Screens
                               are the same either way. */
  int32_t sweep_mode;       /* the soft backward's reverse sweep: 1 = one
                               env per warp (its lane 0 walks the tape, the
                               warp stages records and adds ROM impulses),
                               2 = one env per lane (8 envs a block, each
                               lane walking its own tape), 0 (default) =
                               2 from 16,384 envs, else 1.  Gradients are the
                               same bits either way. */
} vcs_config;

typedef struct vcs_batch vcs_batch;
typedef struct vcs_tape vcs_tape;

/* Loss weights applied at every step of a rollout (device pointers, each
 * nullable): L = sum over steps and envs of ram . ram_t + screen . screen_t. */
typedef struct vcs_loss_weights {
  const float* ram;      /* [128] */
  const float* screen;   /* [210 * 160] */
} vcs_loss_weights;

/* Content-based mapper detection (the paper's ports detect the format from
 * the image, Section 4).  Rules, from the formats' definitions:
 *   2048 -> 2K; 4096 -> 4K;
 *   8192 -> E0 when the image holds an absolute load, store, BIT or NOP
 *           (opcodes $AD $8D $2C $0C) of a cartridge mirror of an E0
 *           hotspot ($1FE0-$1FF7 after masking to 13 bits) and no such
 *           access to the F8 hotspots $1FF8-$1FF9; else FE when it holds
 *           no such access to the F8 hotspots and a JSR ($20) to
 *           $D000-$DFFF (a call into an FE image's second bank); else F8SC
 *           or F8;
 *   16384 -> F6SC or F6; 32768 -> F4SC or F4;
 * where the Superchip variant is chosen when every 4 KB bank repeats its
 * first 128 bytes in the next 128 (the RAM ports hide those 256 bytes, so
 * images fill them with one pattern).  Any other size: VCS_ERR_ROM_SIZE.
 * A host-only call (no device work); rom is a host pointer. */
vcs_status vcs_detect_mapper(const uint8_t* rom, uint32_t size, uint8_t* mapper);

/* Fill *cfg with the defaults listed above. */
vcs_status vcs_config_default(vcs_config* cfg);

/* Create a batch of n_envs machines over n_carts cartridges (Section 2.2;
 * "ROM as a weight tensor", Section 3.1).
 *  roms[c]      host pointer to cart c's image (rom_sizes[c] bytes: 2048,
 *               4096, 8192, 16384 or 32768 for mapper 2K, 4K, F8, F6, F4;
 *               8192, 16384, 32768 for F8SC, F6SC, F4SC; 8192 for E0 and
 *               FE);
 *               copied.
 *  mappers[c]   VCS_MAPPER_* of cart c.
 *  env_cart     host int32[n_envs]: the cart of each env (0..n_carts-1).
 *  cfg          nullable (defaults).
 * The machines start in the power-on state (vcs_reset semantics).
 * Errors: VCS_ERR_ARG, _ROM_SIZE, _MAPPER, _OOM, _CUDA.  On error *out is
 * NULL and nothing is leaked. */
vcs_status vcs_create_batch(const uint8_t* const* roms, const uint32_t* rom_sizes,
                            const uint8_t* mappers, int32_t n_carts,
                            const int32_t* env_cart, int32_t n_envs,
                            const vcs_config* cfg, vcs_batch** out);
vcs_status vcs_destroy(vcs_batch* b);
/* Human-readable description of the last error of `b` (or of the last
 * failed vcs_create_batch when b is NULL).  Valid until the next call. */
const char* vcs_last_error(const vcs_batch* b);
vcs_status vcs_batch_info(const vcs_batch* b, int32_t* n_envs, int32_t* n_carts,
                          int32_t* envs_per_block);
/* *rom_stride = the floats (bytes) per cart of the ROM tensors of the soft
 * API (rom_f32, grad_rom, grad_rom_per_cart): the batch's largest image,
 * at least 8192 (so 8192 unless it holds an F6 or F4 cart).  Byte i of
 * cart c's tensor row is image byte i (2K images: bytes 0..2047); the rest
 * of the row is padding (zero gradient). */
vcs_status vcs_rom_stride(const vcs_batch* b, int32_t* rom_stride);

/* Per-env episode lengths in frames for auto-reset: ep_len is a host
 * uint32[n_envs][n_episodes]; env e's k-th episode ends at the end of the
 * step in which its frame count reaches ep_len[e][k mod n_episodes]; the env
 * then returns to the power-on state and reports VCS_ENV_DONE for that step.
 * n_episodes = 0 disables auto-reset (the default).  The paper's protocol
 * restarts games between episodes (Section 5); lengths are the caller's. */
vcs_status vcs_set_episodes(vcs_batch* b, const uint32_t* ep_len, int32_t n_episodes);

/* Power-on state (A=X=Y=0, SP=$FD, P=$34, PC from the reset vector, RAM
 * and TIA registers zero, timer as written with 0 at T1024T, F8 bank 1),
 * then the boot sequence of the paper's protocol (supplement, settings
 * table): cfg.boot_noop_frames NOOP frames, cfg.boot_reset_frames frames with
 * RESET pressed, then the env's start-NOOP count for its episode (below).
 * Every power-on runs it: at creation, here, and at each episode auto-reset.
 * env_mask: device uint8[n_envs] (nonzero = reset) or NULL for all (which
 * also starts every env's episode count again). */
vcs_status vcs_reset(vcs_batch* b, const uint8_t* env_mask, void* stream);

/* Episode-start randomisation (the paper: 0-30 random NOOPs): counts is a
 * host uint8[n_envs][n_per_env]; env e's k-th episode starts with
 * counts[e][k mod n_per_env] NOOP frames after the boot frames.  The random
 * draw is the caller's (the library draws nothing).  n_per_env = 0 removes
 * the table (the default: no extra frames). */
vcs_status vcs_set_start_noops(vcs_batch* b, const uint8_t* counts, int32_t n_per_env);

/* One env-step for every env (the paper's conformance protocol, Section 5):
 * set each joystick from actions[e] (device uint8[n_envs], ALE action index
 * 0..17), run frame_skip >= 1 frames (a frame ends at the VSYNC write that
 * sets D1, or after 512 scanlines), then write
 *   ram_out     device uint8[n_envs][128]       (nullable)
 *   screen_out  device uint8[n_envs][210][160]  (nullable) the last frame
 *   status_out  device uint8[n_envs]            (nullable) VCS_ENV_* bits
 * Pixel = colour register & 0xFE; row r is scanline ystart + r. */
vcs_status vcs_step(vcs_batch* b, const uint8_t* actions, int32_t frame_skip,
                    uint8_t* ram_out, uint8_t* screen_out, uint8_t* status_out,
                    void* stream);

/* n_steps env-steps: actions device uint8[n_steps][n_envs]; ram_out
 * [n_steps][n_envs][128], screen_out [n_steps][n_envs][210][160],
 * status_out [n_steps][n_envs] (all nullable).  Equivalent to n_steps calls
 * of vcs_step.  The machine stays in registers for all the steps of one
 * launch (a persistent kernel over steps, episodes auto-resetting inside
 * it); cfg.steps_per_launch > 0 splits the rollout into launches of that
 * many steps. */
vcs_status vcs_rollout(vcs_batch* b, const uint8_t* actions, int32_t n_steps,
                       int32_t frame_skip, uint8_t* ram_out, uint8_t* screen_out,
                       uint8_t* status_out, void* stream);

/* vcs_step through host memory: actions_host uint8[n_envs] is copied to
 * the device, the step runs, and ram_out_host / screen_out_host (nullable,
 * host) are filled before the call returns (the stream is synchronised).
 * The library allocates its device staging buffers on the first call. */
vcs_status vcs_step_host(vcs_batch* b, const uint8_t* actions_host, int32_t frame_skip,
                         uint8_t* ram_out_host, uint8_t* screen_out_host, void* stream);

/* ---------------------------------------------------------------------------
 * Launch geometry, autotuning and CUDA graphs (deployment features; the
 * paper's batched rollouts have no counterpart: its GPU path is a traced
 * program).  None of them changes a result: every geometry computes the
 * same bits.
 *
 * vcs_autotune picks the batch's launch geometry by timing it: envs per
 * block (8..128) jointly with threads per env (1, 2, 4), then the warp
 * scheduling policy (program order, or emulated time with windows 4 and 32
 * cycles), then env-steps per launch (1, 4, or the whole rollout).  Each trial runs
 * n_steps env-steps of frame_skip frames from the batch's current state
 * with actions (device uint8[n_steps][n_envs], nullable = NOOP) and writes
 * ram_out / screen_out (device, nullable, sized as for vcs_rollout); the
 * state is restored after every trial, so the batch ends where it began.
 * The winner is applied to the batch and described in *out (nullable).
 * Allocates a state-sized scratch buffer for the call; synchronises
 * `stream`.  Graphs made before the call must be made again (their launch
 * then fails with VCS_ERR_STATE).  Results are cached for the process per
 * (GPU, SM count, n_envs, n_carts, envs per mapper, frame_skip, which
 * outputs are written): a later call with the same key applies the cached
 * choice without trials (n_trials = 0); vcs_autotune_cache_clear forgets
 * them. */
typedef struct vcs_tune {
  int32_t envs_per_block;
  int32_t threads_per_env;
  int32_t sched_policy;
  int32_t sched_window;
  int32_t steps_per_launch;
  float ms_per_step;        /* the winner's measured time per env-step */
  int32_t n_trials;
} vcs_tune;
vcs_status vcs_autotune(vcs_batch* b, int32_t frame_skip, int32_t n_steps, const uint8_t* actions,
                        uint8_t* ram_out, uint8_t* screen_out, vcs_tune* out, void* stream);
vcs_status vcs_autotune_cache_clear(void);

/* A CUDA graph of one vcs_rollout call (its launch sequence under the
 * batch's current geometry), for loops that replay the same rollout shape
 * on fixed buffers: refill `actions` in place, then vcs_graph_launch.  The
 * buffers are the vcs_rollout arguments and must outlive the graph.  The
 * graph is tied to the batch's geometry: after vcs_autotune its launch
 * returns VCS_ERR_STATE.  Capture happens on a private stream. */
typedef struct vcs_graph vcs_graph;
vcs_status vcs_graph_create(vcs_batch* b, const uint8_t* actions, int32_t n_steps, int32_t frame_skip,
                            uint8_t* ram_out, uint8_t* screen_out, uint8_t* status_out,
                            vcs_graph** out);
vcs_status vcs_graph_launch(vcs_graph* g, void* stream);
vcs_status vcs_graph_destroy(vcs_graph* g);

/* Digests of rollout outputs, for parity checks at scale (test
 * infrastructure; the paper has none): out[t][e] (device uint64[n_steps]
 * [n_envs]) = sum mod 2^64 over i of F((i << 32) | w_i), where w_i are the
 * little-endian 32-bit words of ram[t][e] (128 bytes) followed by
 * screen[t][e] (33,600 bytes; screen nullable = RAM only) and F is the
 * splitmix64 finaliser (variant 13).  ram and screen are device buffers laid
 * out as vcs_rollout writes them, 16-byte aligned. */
vcs_status vcs_digest(vcs_batch* b, const uint8_t* ram, const uint8_t* screen, int32_t n_steps,
                      uint64_t* out, void* stream);

/* vcs_rollout through host memory, pipelined: actions_host uint8[n_steps]
 * [n_envs]; ram_host [n_steps][n_envs][128], screen_host [n_steps][n_envs]
 * [210][160], status_host [n_steps][n_envs] (host, nullable).  Step t's
 * outputs are copied to the host on a second stream while step t + 1 runs
 * (two device buffer sets, allocated by the library on the first call); the
 * call returns when every output is on the host.  Host buffers should be
 * pinned (page-locked) for the copies to overlap. */
vcs_status vcs_rollout_host(vcs_batch* b, const uint8_t* actions_host, int32_t n_steps, int32_t frame_skip,
                            uint8_t* ram_host, uint8_t* screen_host, uint8_t* status_host, void* stream);

/* Measured integer issue rate of the current device (the roofline
 * denominator of the integer-bound emulator; a measurement utility with no
 * counterpart in the paper): a kernel at full occupancy running independent
 * chains of 32-bit add, shift and logic operations, timed with CUDA events;
 * *ops_per_s receives operations per second.  Synchronises `stream`. */
vcs_status vcs_int_peak(double* ops_per_s, void* stream);

/* Kernel timing (a measurement aid with no counterpart in the paper): while
 * on, every frame-step launch of the batch records CUDA events on its
 * stream around the step kernel and, with deferred rasterisation, the raster
 * kernel; launches inside a stream capture are not timed.  `on` = 1 starts
 * (clearing the sums; allocates an 8-byte counter the first time), 0 stops.
 * vcs_kernel_times waits for the recorded events and returns the summed
 * milliseconds of each kernel, the number of launches timed and (when
 * log_entries is non-null) the raster log entries those launches drew,
 * then clears the sums. */
vcs_status vcs_time_kernels(vcs_batch* b, int32_t on);
vcs_status vcs_kernel_times(vcs_batch* b, float* step_ms, float* raster_ms, int32_t* n_launches,
                            double* log_entries);

/* Fully relaxed forward, the temperature-limit study of Section 4 (Theorem 2
 * and the supplement's forward bit-exactness table).  From each env's
 * current state (read, not modified) two machines run n_instr instruction
 * slots side by side with the joystick held at actions[env] (device uint8
 * [n_envs], ALE actions; nullable = NOOP):
 *   - the hard machine, which also counts the casts that would round off:
 *     counts[env] (device uint32[n_envs][4], nullable) = {ROM and RAM reads
 *     by instructions (operand bytes, data, pointers, stack; not opcode
 *     fetches), those whose temperature read equals the byte, conditional
 *     branches, those whose relaxed counter equals the hard one}: the
 *     quantities of the paper's cast-margin model (rho, p_read, f_b,
 *     p_branch);
 *   - the FULL machine, without the straight-through correction: each such
 *     read returns round(sum_k w_k t_k / sum_k w_k), w_k = e^{-|k - a| / T}
 *     over |k - a| <= max(1, ceil(12 T)) clipped to the tensor (the 2K
 *     image, the 4K image, or the current F8 bank; RAM 128 bytes), and a
 *     conditional branch sets pc = round(pc_fall + sigma(alpha z) delta),
 *     z = +1 when its condition holds else -1; float32 throughout, weights
 *     and gate values the float32 roundings of e^{-k/T} and
 *     sigma(+-alpha), terms summed in index order, no fused multiply-add,
 *     rounding half to even.  A taken branch pays its cycle and a page
 *     cross between the fall-through and the new counter.
 * n_div[env] (device int32[n_envs]) receives the first slot (1-based) after
 * which the two machines' states differ (registers, flags, clocks, timer,
 * TIA registers, bank, jam flag, RAM), 0 if they agree throughout;
 * ram_full[env] (device uint8[n_envs][128], nullable) the FULL machine's
 * RAM after the last slot.  The relaxed path is forward only (no tape).
 * Errors: VCS_ERR_ARG (T outside (0, 10], n_instr < 0, alpha not finite,
 * n_div NULL), VCS_ERR_CUDA. */
vcs_status vcs_full_divergence(vcs_batch* b, float T, float alpha, const uint8_t* actions, int32_t n_instr,
                               int32_t* n_div, uint32_t* counts, uint8_t* ram_full, void* stream);

/* Wait for `stream` and report device-side failures: VCS_ERR_WATCHDOG if a
 * kernel's bounded wait gave up (the batch is then unusable: destroy it;
 * a block whose ROM staging timed out waited once more, also bounded, for
 * its copy before leaving), VCS_ERR_CUDA for an asynchronous CUDA error. */
vcs_status vcs_sync(vcs_batch* b, void* stream);

/* ---------------------------------------------------------------------------
 * SOFT-STE mode (Section 3.1, Eq. peek / Eq. branch / Eq. ste / Eq. s-read;
 * Theorem 1; Corollary 1).
 *
 * vcs_soft_rollout: n_steps env-steps from the batch's current state, like
 * vcs_rollout, with the inputs of the relaxation as floats:
 *   rom_f32  device float[n_carts][rom_stride] (nullable: the batch's ROMs) - the
 *            ROM as a weight tensor; the forward uses round(value) clamped
 *            to 0..255 (2K images use bytes 0..2047);
 *   ram0     device float[n_envs][128] (nullable: the current RAM) - the RAM
 *            at the start of the rollout, rounded likewise;
 *   u        device float[n_steps][n_envs][5] - joystick inputs (right,
 *            left, down, up, fire), a button counts as pressed when >= 0.5;
 *   tau      read temperature in (0, 10]: only the backward pass uses it.
 * Outputs (device, nullable): ram_out float[n_steps][n_envs][128] and
 * screen_out float[n_steps][n_envs][210][160]; they hold the hard values
 * exactly (Theorem 1).  The batch state advances as in vcs_rollout (no
 * episode auto-reset in soft mode).  The library checkpoints the state every
 * cfg.segment_frames frames into *tape (owned by the caller until
 * vcs_tape_free; it refers to the batch, which must outlive it). */
vcs_status vcs_soft_rollout(vcs_batch* b, float tau, const float* rom_f32, const float* ram0,
                            const float* u, int32_t n_steps, int32_t frame_skip,
                            float* ram_out, float* screen_out, vcs_tape** tape, void* stream);

/* vcs_soft_step: the soft step of the problem statement, n_steps SOFT-STE
 * env-steps of frame_skip frames from the batch's current state with the
 * batch's own ROM images and RAM (Section 3.1; Theorem 1: the forward is
 * bit-exact with vcs_rollout at every temperature; Corollary 1: tau only
 * sets the relaxation that vcs_backward differentiates).  It is
 * vcs_soft_rollout with rom_f32 = NULL and ram0 = NULL:
 *   action_inputs  device float[n_steps][n_envs][5] (right, left, down, up,
 *                  fire; a button counts as pressed when >= 0.5);
 *   tau            in (0, 10], else VCS_ERR_ARG;
 *   ram_out        device float[n_steps][n_envs][128] (nullable);
 *   screen_out     device float[n_steps][n_envs][210][160] (nullable);
 *   *tape          receives the tape (caller-owned until vcs_tape_free).
 * vcs_backward on the tape gives the surrogate gradients with respect to
 * the ROM bytes (at the batch's images), the RAM at the start and the
 * action inputs.  Errors as vcs_soft_rollout. */
vcs_status vcs_soft_step(vcs_batch* b, float tau, const float* action_inputs, int32_t n_steps,
                         int32_t frame_skip, float* ram_out, float* screen_out, vcs_tape** tape,
                         void* stream);

/* Surrogate gradients of L = sum grad_ram . ram_out + sum grad_screen .
 * screen_out (or of the broadcast loss weights `w`) with respect to
 *   grad_rom           device float[n_envs][rom_stride] per env (nullable)
 *   grad_ram0          device float[n_envs][128] (nullable)
 *   grad_cart_ram0     device float[n_envs][128] (nullable): the Superchip
 *                      RAM at the start of the rollout (a second RAM tensor:
 *                      relaxed reads within it, one-hot writes); zero for
 *                      envs of other carts
 *   grad_u             device float[n_steps][n_envs][5] (nullable)
 *   grad_rom_per_cart  device float[n_carts][rom_stride] summed over each cart's
 *                      envs (nullable)
 * grad_ram [n_steps][n_envs][128] and grad_screen [n_steps][n_envs][210][160]
 * are device pointers (each nullable); give either those or `w`.  The pass
 * recomputes each checkpoint segment, so the forward's outputs need not be
 * kept.  It may be called several times on one tape; the first call sizes
 * and allocates the tape's scratch (after one stream synchronisation). */
vcs_status vcs_backward(vcs_tape* tape, const float* grad_ram, const float* grad_screen,
                        const vcs_loss_weights* w, float* grad_rom, float* grad_ram0,
                        float* grad_cart_ram0, float* grad_u, float* grad_rom_per_cart, void* stream);
vcs_status vcs_tape_free(vcs_tape* tape);

/* vcs_backward without any device allocation (the paper has no counterpart:
 * this is a deployment variant).  For callers that cannot let a library
 * allocate device memory: an application whose GPU memory is owned by an
 * allocator it does not control (for instance a framework's caching pool
 * that has reserved the device) or that runs under a fixed device-memory
 * budget, where a cudaMalloc behind its back can fail or fragment the pool.
 * Same arguments and results as vcs_backward; the caller passes the tape,
 * inputs and outputs, and all scratch (tape entries, adjoint carries, ROM
 * impulses) comes from one fixed 64 MiB array compiled into the library,
 * which every GPU that loads the library keeps until the process exits.
 *  - The scratch a call needs, per env: 2,104 bytes of adjoint carries
 *    plus 8 x rom_stride bytes of ROM impulses (64 KB for 8 KB images),
 *    plus 4 x rom_stride more (32 KB) when grad_rom_per_cart is asked for
 *    without grad_rom; and per env and checkpoint segment held at once
 *    (at least one): 4 x (tape records + colour versions + steps per
 *    segment + 8) bytes, the records being about one per instruction of
 *    the segment.  Problems that do not fit are rejected with
 *    VCS_ERR_ARG and a message giving the size needed.
 *  - The first call on a device (and the first after that device's
 *    context was destroyed and made again) looks up the array's device
 *    address, with that device current, and keeps it; make that first call
 *    before any stream capture.
 *  - All calls share the array and it keeps the last call's contents (the
 *    call clears what must start at zero); calls whose GPU work overlaps,
 *    on two streams or two host threads, race with each other.
 *  - It synchronises `stream` on every call, to read the tape's sizes.
 *  - Its gradients equal vcs_backward's bit for bit when both recompute
 *    the same number of segments at once, or both fewer or both more than
 *    16,384 machines (segments x envs) per group; across that line the
 *    recompute sums pixel gradients in another order (last-bit changes). */
vcs_status vcs_backward_static(vcs_tape* tape, const float* grad_ram, const float* grad_screen,
                               const vcs_loss_weights* w, float* grad_rom, float* grad_ram0,
                               float* grad_cart_ram0, float* grad_u, float* grad_rom_per_cart,
                               void* stream);

/* Copy the machine state out / in as an opaque blob (checkpoint/resume).
 * vcs_state_bytes gives the size; blob is a host pointer; both calls
 * synchronise `stream`. */
vcs_status vcs_state_bytes(const vcs_batch* b, size_t* bytes);
/* The Superchip RAM of every env: out is device uint8[n_envs][128] (4-byte
 * aligned), zero for envs of other carts.  Asynchronous on `stream`. */
vcs_status vcs_cart_ram(vcs_batch* b, uint8_t* out, void* stream);
vcs_status vcs_save_state(vcs_batch* b, void* blob_host, void* stream);
vcs_status vcs_load_state(vcs_batch* b, const void* blob_host, void* stream);

#ifdef __cplusplus
}
#endif
#endif
