/*
 * CPU oracle for the VCS hot path: TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, cycle-by-cycle emulator of the Atari VCS (6507 CPU, RIOT,
 * TIA video: by default the subset of player 0, playfield and background,
 * or with ovcs_set_full_tia the whole TIA with player 1, missiles, ball and
 * collisions; 2K, 4K, F8, F6, F4, the Superchip variants of the last three,
 * E0 and FE cartridges) written from the paper's machine description (Section
 * 2.2 and the architecture figure) and the public chip documentation (MOS
 * 6500 manuals, 6532 datasheet, TIA programmer's guide, the published note
 * on NMOS decimal mode).  Every CPU cycle is charged before its bus access;
 * the RIOT timer ticks once per cycle and the TIA is advanced one colour
 * clock at a time, three per cycle.
 *
 * Parity unpinned against real hardware and the paper's reference emulator
 * (neither is available): the timing constants and the TIA's object rules
 * are this oracle's readings of the documentation, pinned by the test
 * suite's hand-derived values, closed forms and exhaustive tables.
 *
 * Soft mode (SOFT-STE, Section 3.1; Theorem 1; Corollary 1): the same
 * interpreter optionally records a deviation graph.  Every value carries a
 * node whose value under perturbation is hard + (soft(x) - soft(x_hard)),
 * with every discrete choice frozen (the stored-switch rule of Section 3.1).
 * Surrogate rulebook: a ROM or RAM read takes the Jacobian of the relaxed
 * read (Eq. s-read) with respect to the memory contents, i.e. weights
 * w_i ~ exp(-|i - a| / tau) over the window |i - a| <= W = max(1,
 * ceil(12 tau)) clipped to the tensor; addresses, the program counter and
 * flags are indices or bits and so carry no gradient; writes move the
 * cell's adjoint to the written value; ADC/SBC have derivatives (1, +-1),
 * AND/ORA/EOR (1, 1), increments, transfers, shifts and rotates 1 (the
 * straight-through rule for integer casts); SWCHA/INPT4 are linear in the
 * joystick inputs and INTIM in the last timer value before underflow;
 * pixels take the derivative 1 of the owning colour register.  Reverse
 * mode, tangent mode and a direct re-evaluation (for finite differences)
 * run over the graph in double precision.
 *
 * Only the test suite, the package's smoke check and the benchmark's CPU
 * baseline call this library; the product path never does.
 */
#ifndef VCS_ORACLE_H
#define VCS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ovcs ovcs;

/* Counters accumulated over the emulator's lifetime (reset by ovcs_reset). */
typedef struct {
  uint64_t instructions;   /* executed instructions (jam steps excluded) */
  uint64_t cycles;         /* CPU cycles */
  uint64_t frames;         /* completed frames */
  uint64_t tia_writes;     /* writes to TIA registers */
  uint64_t ram_reads, ram_writes, rom_reads;
  uint64_t pixels;         /* pixels composited into an output frame */
  uint64_t watchdog;       /* frames ended by the line cap */
  /* casts of the fully relaxed forward (ovcs_set_full modes 1 and 2): ROM
   * and RAM reads by instructions (opcode fetches excluded) and the ones
   * whose temperature read rounds to the stored byte; executed conditional
   * branches and the ones whose relaxed counter rounds to the hard one */
  uint64_t relaxed_reads, relaxed_reads_exact, branches, branches_exact;
} ovcs_counters;

/* mapper: 0 = 2K, 1 = 4K, 2 = F8 (8 KB, hotspots $1FF8-9), 3 = F6 (16 KB,
 * $1FF6-9), 4 = F4 (32 KB, $1FF4-B): any access to hotspot j selects 4 KB
 * bank j; 5, 6, 7 = F8SC, F6SC, F4SC: the same with 128 bytes of cartridge
 * RAM written at $1000-$107F and read at $1080-$10FF; 8 = E0 (8 KB in eight
 * 1 KB slices; an access to $1FE0+j / $1FE8+j / $1FF0+j maps slice j into
 * segment 0 / 1 / 2 of the window, segment 3 shows slice 7); 9 = FE (8 KB
 * in two 4 KB banks, the first shown at power-on: a JSR made with the stack
 * pointer at $FF or an RTS made with it at $FD selects the bank from bit 5
 * of the high address byte it moves next: set -> the first 4 KB, clear ->
 * the second).  rom is copied.  NULL on a bad size. */
ovcs* ovcs_new(const uint8_t* rom, uint32_t rom_size, int mapper, int ystart);
void ovcs_free(ovcs* s);
/* Power-on state (A7 of the design notes). */
void ovcs_reset(ovcs* s);
/* Console switches as SWCHB reads them (power-on: $0B = colour, difficulty
 * B, RESET and SELECT released; $0A holds RESET down). */
void ovcs_set_switches(ovcs* s, uint8_t swchb);
/* Differentiable position sampler (Section 3) in soft rollouts: 1 = on.
 * Off by default; the hard outputs do not depend on it. */
void ovcs_set_sampler(ovcs* s, int on);
/* Graphics-bit surrogate (Section 3.1's stored-switch paragraph) in soft
 * rollouts: 1 = on.  Every drawn pixel adds (C_with - C_without) x its
 * gradient to the register byte of each graphics bit deciding an object's
 * coverage there (GRP0 / GRP1 or their delayed copies, ENAM0 / ENAM1,
 * ENABL or its delayed copy, PF0 / PF1 / PF2), C_with and C_without being
 * the pixel's colours with that bit forced to 1 and to 0.  Off by default;
 * the hard outputs do not depend on it. */
void ovcs_set_graphics(ovcs* s, int on);
/* Instruction-granular steps (the paper's throughput unit: one step = one
 * emulated instruction): n > 0 makes every following step (ovcs_step, soft
 * rollouts) run n instruction slots (an executed instruction, or a jammed
 * CPU's idle to the next line) instead of frame_skip frames; 0 restores
 * frame steps.  The screen of such a step is the last frame completed. */
void ovcs_set_step_instructions(ovcs* s, int n);
/* Fully relaxed casts (Section 4's temperature-limit study, Theorem 2):
 * mode 2 = FULL: every ROM and RAM read by an instruction (operand bytes,
 * data, pointers, stack; not the opcode fetch) returns the temperature-T
 * read round(sum w_k t[k] / sum w_k), w_k = e^{-|k-a|/T} in the window
 * |k - a| <= max(1, ceil(12 T)) clipped to the tensor, and a conditional
 * branch sets pc = round(pc_fall + sigma(alpha z) delta) with z = +1 when
 * its condition holds, else -1; all in float32 (weights and gate values the
 * float32 roundings of e^{-k/T} and sigma(+-alpha)).  Mode 1 = probe: the
 * machine stays hard and only counts which casts would round off the hard
 * value (the counters' relaxed_* and branches* fields).  Mode 0 = off. */
void ovcs_set_full(ovcs* s, int mode, double T, double alpha);
/* One env-step: set the joystick from `action` (ALE index 0..17), run
 * `frame_skip` frames, copy RAM (128 B) and the last frame (210x160) out.
 * Returns a status bit set: 1 = a frame ended by the line cap, 2 = jammed. */
int ovcs_step(ovcs* s, int action, int frame_skip, uint8_t* ram_out, uint8_t* screen_out);
void ovcs_get_counters(const ovcs* s, ovcs_counters* out);
/* Machine state as 32 words (layout in the .c file). */
void ovcs_get_state(const ovcs* s, uint32_t* out64);   /* registers, clocks, TIA (64 words) */
void ovcs_get_ram(const ovcs* s, uint8_t* out128);
/* on = 1: the whole TIA (player 1, missiles, ball, NUSIZ, REFP, VDEL,
 * RESMP, score mode, collisions); 0 (default): the subset machine (player
 * 0, playfield, background; the other object registers ignored, the
 * collision registers read 0). */
void ovcs_set_full_tia(ovcs* s, int on);
void ovcs_get_cart_ram(const ovcs* s, uint8_t* out128);   /* Superchip RAM (zero otherwise) */
/* Run n instructions, recording per instruction: pc, opcode, A, X, Y, SP,
 * P, cycle (low 32 bits), scanline, line clock.  Returns instructions run. */
int ovcs_trace(ovcs* s, int action, int n, uint32_t* out10);

/* Test hooks: set registers / RAM / memory state directly. */
void ovcs_set_regs(ovcs* s, int A, int X, int Y, int SP, int P, int PC);
void ovcs_set_ram(ovcs* s, const uint8_t* ram128);
/* Execute exactly one instruction; returns its cycle count. */
int ovcs_exec_one(ovcs* s);
uint8_t ovcs_peek(ovcs* s, uint16_t addr);   /* side-effect-free debug read */
int ovcs_bank(const ovcs* s);

/* ---------------- soft mode (FP64 deviation graph) ---------------- */

typedef struct ogrf ogrf;

/* Run a soft rollout from the current state for n_steps env-steps.
 * u[n_steps][5] are the joystick inputs (R, L, D, U, FIRE) in {0,1};
 * tau > 0 is the read temperature and alpha the gate sharpness.
 * grad_ram [n_steps][128] and grad_screen [n_steps][210*160] (either may be
 * NULL) are the loss weights L = sum grad * output.  ram_out/screen_out
 * (nullable) receive the forward outputs as doubles.  Returns the graph. */
ogrf* ovcs_soft_rollout(ovcs* s, const double* u, int n_steps, int frame_skip,
                        double tau, double alpha,
                        const double* grad_ram, const double* grad_screen,
                        double* ram_out, double* screen_out);
void ogrf_free(ogrf* g);
/* Reverse sweep: d L / d (ROM bytes [rom_size], initial RAM [256]: the
 * RIOT RAM then the Superchip's cartridge RAM, inputs [n_steps][5]).  The
 * tangent and evaluation sweeps take d_ram0 in the same 256-cell layout. */
void ogrf_reverse(ogrf* g, double* grad_rom, double* grad_ram0, double* grad_u);
/* Tangent sweep: directional derivative of L along (d_rom, d_ram0, d_u). */
double ogrf_tangent(ogrf* g, const double* d_rom, const double* d_ram0, const double* d_u);
/* Exact re-evaluation of L - L_hard of the frozen-switch relaxation at the
 * hard inputs plus the given perturbation (finite differences). */
double ogrf_eval(ogrf* g, const double* d_rom, const double* d_ram0, const double* d_u);
int64_t ogrf_nodes(const ogrf* g);
/* The relaxed read primitive on its own (Eq. s-read with the frozen window
 * of half-width W = max(1, ceil(12 tau)) clipped to [0, M)): value and
 * derivative with respect to the (real) address a around integer a0. */
/* Digest of one env-step's outputs, for parity checks at scale (test
 * infrastructure, no counterpart in the paper): the 128 RAM bytes followed by
 * the 33,600 screen bytes (screen may be NULL: RAM only) read as
 * little-endian 32-bit words w_i, i = 0, 1, ...; the digest is the sum mod
 * 2^64 over i of F((i << 32) | w_i), F the splitmix64 finaliser (Steele, Lea
 * and Flood 2014, variant 13). */
uint64_t ovcs_digest(const uint8_t* ram128, const uint8_t* screen);

double ovcs_relaxed_read(const double* r, int M, int a0, double a, double tau, double* d_da);
/* Gate derivative alpha * s(alpha z) (1 - s(alpha z)) of Eq. s-branch. */
double ovcs_gate_slope(double alpha, double z);

#ifdef __cplusplus
}
#endif
#endif
