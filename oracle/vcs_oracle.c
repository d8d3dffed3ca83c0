/*
 * CPU oracle for the VCS hot path: TEST INFRASTRUCTURE ONLY (see the header).
 *
 * Machine readings where the paper is silent (each one is a constant of this
 * oracle; the names A1..A12 are the design notes' labels):
 *  A1 a frame ends (and the next begins, scanline 0) at a VSYNC write that
 *     sets D1 while D1 was clear;
 *  A2 a frame is also ended at an instruction boundary once 512 scanlines
 *     have elapsed without VSYNC (the env's watchdog flag is raised);
 *  A3 screen row r is scanline ystart + r; columns are line clocks 68..227;
 *  A4 pixel = colour register & 0xFE; 0 while VBLANK D1 is set and for the
 *     first 8 pixels of a line whose HMOVE strobe hit line clock <= 9;
 *  A5 a write takes effect at colour clock 3 x (cycle count after the cycle
 *     of the write is charged): clocks rendered before it see the old value;
 *  A6 RESP0 / RESP1 -> position 3 during HBLANK, else (clock - 68 + 5) mod
 *     160; RESM0 / RESM1 / RESBL -> 2, else (clock - 68 + 4) mod 160; HMOVE
 *     subtracts each object's signed motion nibble; WSYNC halts the CPU
 *     until the cycle count is a multiple of 76; playfield 20 bits x 4
 *     clocks with the right half repeated or reflected (CTRLPF bit 0);
 *     players of 8 bits (REFP bit 3 reflects; GRP delayed by VDELP), sized
 *     and copied by NUSIZ (copies at +16 / +32 / +64, double and quad
 *     width), missiles and ball 1 / 2 / 4 / 8 wide (NUSIZ bits 4-5, CTRLPF
 *     bits 4-5), RESMP hides a missile at its player's position + 4 x width
 *     - 1; priority P0/M0 > P1/M1 > PF/BL > BK (score mode: the playfield in
 *     COLUP0 / COLUP1 by half) unless CTRLPF bit 2 (PF/BL first);
 *  A7 power-on: A=X=Y=0, SP=$FD, P=$34, PC from $1FFC/D, RAM and TIA zero,
 *     the timer as if 0 had been written to T1024T at cycle 0, banked carts
 *     (F8, F6, F4 and their Superchip variants) in their last bank, the
 *     Superchip's RAM zero;
 *  A8 timer: a write of V at cycle t_w makes INTIM = V - ceil(k / I) at
 *     t_w + k until that would go negative; from k_u = V*I + 1 on it reads
 *     (0xFF - (k - k_u)) & 0xFF and TIMINT bit 7 is set;
 *  A9 only architectural accesses have side effects (dummy reads and the
 *     RMW dummy write are idle cycles);
 *  A10 undriven TIA read bits are 0; collisions latch on every visible
 *     column of every line (blanked or not) until CXCLR and read in D7 / D6
 *     of CXM0P .. CXPPMM;
 *  A11 NMOS decimal mode per the published note on decimal mode;
 *  A12 pushed P always has bits 4 and 5 set (PHP and BRK are the only
 *     pushes of P on a 6507); BRK vectors through $1FFE.
 *  E0 carts (8 KB in eight 1 KB slices): the cartridge window is four 1 KB
 *  segments; an access (read or write) to $1FE0+j, $1FE8+j or $1FF0+j maps
 *  slice j into segment 0, 1 or 2, and segment 3 always shows slice 7; at
 *  power-on segments 0..2 show slices 4, 5, 6.  A relaxed ROM read's tensor
 *  is the 1 KB slice the read's segment shows.
 *  FE carts (8 KB in two 4 KB banks, the first at power-on): a JSR made
 *  with the stack pointer at $FF (the return address's low byte pushed to
 *  $01FE) or an RTS made with it at $FD (the low byte pulled from $01FE)
 *  selects the bank from bit 5 of the bus byte of the next cycle (the
 *  target's or the return address's high byte): set -> the first 4 KB,
 *  clear -> the second.  Other accesses to $01FE switch nothing.
 *  Superchip carts (F8SC, F6SC, F4SC: the banked formats plus 128 bytes of
 *  cartridge RAM) write that RAM at $1000-$107F and read it at $1080-$10FF
 *  of the cartridge window, in every bank; a read of the write port returns
 *  the ROM byte under it and writes nothing (no bus-contention model).  In
 *  soft mode the cartridge RAM is a second 128-cell memory tensor: its
 *  reads are relaxed within it and its writes are one-hot, like RIOT RAM.
 *  The paper's 38 extra opcode bytes (USBC, the unofficial NOPs, LAX, SAX)
 *  are executed; every other undocumented opcode jams the CPU: from then on
 *  each instruction slot
 *  idles to the next line start, so the frame ends by the 512-line cap.
 *  With the position sampler on (ovcs_set_sampler), soft rollouts also carry
 *  the deviation of player 0's position: zero at each RESP0, minus a
 *  sixteenth of HMP0's deviation added at each HMOVE, and its pixels take the
 *  slope of the triangular coverage kernel (sampler_slope).
 */
#include "vcs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define LINE_CAP 512
#define SCR_W 160
#define SCR_H 210

/* ------------------------------------------------------------------ */
/* deviation graph                                                     */
/* ------------------------------------------------------------------ */

enum { NK_ZERO = 0, NK_LEAF, NK_LIN, NK_RROM, NK_RRAM };

typedef struct {
  uint8_t kind, n;
  int16_t lo, a0;      /* read: first window cell, hard address (tensor index) */
  int32_t base;        /* read_rom: ROM offset of the tensor */
  int32_t in[4];
  double c[4];
  int64_t pool;        /* read_ram: offset of the window's cells in the pool */
} onode;

struct ogrf {
  onode* nd;
  double* seed;
  int64_t n, cap;
  int32_t* pnode;      /* read_ram window: node of each cell */
  int64_t pn, pcap;
  const uint8_t* rom;  /* the emulator's ROM copy (owned by ovcs) */
  uint8_t* rom_copy;
  int rom_size;
  int32_t rom0, ram0, u0;
  double ram0_val[256];   /* RIOT RAM, then cartridge RAM */
  double* u_val;
  int n_steps;
  double tau, alpha;
  int W;
};

/* ------------------------------------------------------------------ */
/* machine                                                             */
/* ------------------------------------------------------------------ */

typedef struct { uint8_t v; int32_t n; } val;

struct ovcs {
  /* CPU */
  uint8_t A, X, Y, SP, P;
  uint16_t pc;
  uint64_t cyc;
  int jammed;
  /* memory */
  uint8_t ram[256];        /* RIOT RAM, then the Superchip's cartridge RAM */
  uint8_t* rom;
  uint32_t rom_size;
  int mapper, bank;
  int sc;                  /* Superchip variant (cartridge RAM at $1000-$10FF) */
  int e0;                  /* E0 cart: e0seg[k] = the slice segment k (0..2) shows */
  int fe;                  /* FE cart: two 4 KB banks chosen through JSR and RTS */
  int e0seg[3];
  /* RIOT */
  uint8_t intim;
  uint32_t interval, phase;
  int underflow;
  uint8_t swcha, swchb, inpt4;
  /* TIA */
  uint8_t vsync, vblank, colup0, colupf, colubk, ctrlpf, pf0, pf1, pf2, grp0, hmp0;
  int p0pos;
  /* the rest of the TIA: player 1, the missiles and the ball */
  uint8_t colup1, nusiz[2], refp[2], grp1, grpo[2], enam[2], enabl, enablo;
  uint8_t hmp1, hmm[2], hmbl, vdelp[2], vdelbl, resmp[2];
  int p1pos, mpos[2], blpos;
  uint16_t cx;             /* collision latches: bit 2 r + 1 = D7 and bit 2 r = D6 of read register r */
  int full_tia;            /* 1: the whole TIA; 0: the subset machine (player 0, playfield,
                            * background; other object registers ignored, collisions read 0) */
  int hclk, line;
  int hmove_line;
  int wsync;
  int ystart;
  uint8_t fb[SCR_H * SCR_W];
  uint8_t last_fb[SCR_H * SCR_W];
  int frames_in_step;
  ovcs_counters cnt;
  /* soft mode */
  ogrf* g;
  int32_t nA, nX, nY, nV, nC[4], nRAM[256];   /* nC: COLUP0, COLUPF, COLUBK, COLUP1 */
  int32_t nPos, nHM;       /* deviations of the P0 position and of HMP0 (sampler) */
  int sampler;             /* 1: the differentiable position sampler is on */
  /* graphics-bit surrogate: the written values of GRP0, GRP1, ENAM0, ENAM1,
   * ENABL, PF0, PF1, PF2 (nG) and of the delayed GRP0, GRP1, ENABL (nGo) */
  int32_t nG[8], nGo[3];
  int graphics;            /* 1: graphics bits carry gradient */
  int step_instr;          /* > 0: a step is this many instruction slots, not frames */
  /* fully relaxed casts (Section 4's temperature-limit study): 0 = off,
   * 1 = probe (count the casts that would round off the hard value), 2 =
   * FULL (execute the relaxed casts) */
  int full;
  int full_W;
  float full_ek[256];      /* float32 weights e^{-k/T} of the relaxed read */
  float full_g1, full_g0;  /* float32 gate values sigma(alpha), sigma(-alpha) */
  int32_t u_leaf;
  const double* gs_all;   /* grad_screen for all steps (or NULL) */
  const double* gs;       /* grad_screen of the frame being rendered */
  int soft_step, frame_skip;
};

/* ---------------- graph helpers ---------------- */

static int32_t g_new(ovcs* s, int kind) {
  ogrf* g = s->g;
  if (g->n == g->cap) {
    g->cap = g->cap ? g->cap * 2 : 4096;
    g->nd = (onode*)realloc(g->nd, (size_t)g->cap * sizeof(onode));
    g->seed = (double*)realloc(g->seed, (size_t)g->cap * sizeof(double));
  }
  int32_t id = (int32_t)g->n++;
  memset(&g->nd[id], 0, sizeof(onode));
  g->nd[id].kind = (uint8_t)kind;
  g->seed[id] = 0.0;
  return id;
}

/* Linear combination of up to four deviations; zero terms are dropped and a
 * single unit-coefficient term returns its input node unchanged. */
static int32_t g_lin(ovcs* s, int k, const int32_t* in, const double* c) {
  if (!s->g) return 0;
  int32_t ii[4];
  double cc[4];
  int m = 0;
  for (int j = 0; j < k; j++)
    if (in[j] != 0 && c[j] != 0.0) { ii[m] = in[j]; cc[m] = c[j]; m++; }
  if (m == 0) return 0;
  if (m == 1 && cc[0] == 1.0) return ii[0];
  int32_t id = g_new(s, NK_LIN);
  onode* nd = &s->g->nd[id];
  nd->n = (uint8_t)m;
  for (int j = 0; j < m; j++) { nd->in[j] = ii[j]; nd->c[j] = cc[j]; }
  return id;
}
static int32_t lin1(ovcs* s, int32_t a, double ca) {
  int32_t in[1] = {a}; double c[1] = {ca}; return g_lin(s, 1, in, c);
}
static int32_t lin2(ovcs* s, int32_t a, double ca, int32_t b, double cb) {
  int32_t in[2] = {a, b}; double c[2] = {ca, cb}; return g_lin(s, 2, in, c);
}
static void window(int W, int M, int a0, int* lo, int* hi) {
  *lo = a0 - W < 0 ? 0 : a0 - W;
  *hi = a0 + W > M - 1 ? M - 1 : a0 + W;
}

static int32_t g_read_rom(ovcs* s, int base, int M, int a0) {
  if (!s->g) return 0;
  int lo, hi;
  window(s->g->W, M, a0, &lo, &hi);
  int32_t id = g_new(s, NK_RROM);
  onode* nd = &s->g->nd[id];
  nd->lo = (int16_t)lo; nd->n = (uint8_t)(hi - lo + 1); nd->a0 = (int16_t)a0;
  nd->base = base;
  return id;
}

/* Relaxed read of cell a0 of the 128-cell RAM tensor whose cells start at
 * index tb of the RAM nodes (0: RIOT RAM, 128: the Superchip's RAM). */
static int32_t g_read_ram(ovcs* s, int tb, int a0) {
  if (!s->g) return 0;
  ogrf* g = s->g;
  int lo, hi;
  window(g->W, 128, a0, &lo, &hi);
  int n = hi - lo + 1;
  if (g->pn + n > g->pcap) {
    g->pcap = g->pcap ? g->pcap * 2 : 65536;
    g->pnode = (int32_t*)realloc(g->pnode, (size_t)g->pcap * sizeof(int32_t));
  }
  int32_t id = g_new(s, NK_RRAM);
  onode* nd = &g->nd[id];
  nd->lo = (int16_t)lo; nd->n = (uint8_t)n; nd->a0 = (int16_t)a0;
  nd->pool = g->pn;
  for (int i = 0; i < n; i++) g->pnode[g->pn + i] = s->nRAM[tb + lo + i];
  g->pn += n;
  return id;
}

/* ---------------- TIA ---------------- */

static void frame_end(ovcs* s);

static int pf_bit(const ovcs* s, int x) {
  int i = x < 80 ? x / 4 : (x - 80) / 4;
  if (x >= 80 && (s->ctrlpf & 1)) i = 19 - i;
  if (i < 4) return (s->pf0 >> (4 + i)) & 1;
  if (i < 12) return (s->pf1 >> (7 - (i - 4))) & 1;
  return (s->pf2 >> (i - 12)) & 1;
}

/* NUSIZ number-and-size field (bits 0-2): the copies' offsets in columns
 * and the player's pixel width. */
static int nusiz_copies(int mode, int off[3]) {
  static const int n[8] = {1, 2, 2, 3, 2, 1, 3, 1};
  static const int o[8][3] = {{0, 0, 0}, {0, 16, 0}, {0, 32, 0}, {0, 16, 32},
                              {0, 64, 0}, {0, 0, 0}, {0, 32, 64}, {0, 0, 0}};
  for (int k = 0; k < 3; k++) off[k] = o[mode][k];
  return n[mode];
}
static int player_scale(int mode) { return mode == 5 ? 2 : (mode == 7 ? 4 : 1); }

/* Player i at visible column x: graphic GRPi (the delayed copy when VDELPi
 * is set), bit 7 leftmost unless REFPi bit 3 reflects it, each bit
 * `scale` columns wide, in every copy NUSIZi asks for, wrapping at 160. */
static int player_bit(const ovcs* s, int i, int x) {
  const int mode = s->nusiz[i] & 7, sc = player_scale(mode);
  const int g = (s->vdelp[i] & 1) ? s->grpo[i] : (i ? s->grp1 : s->grp0);
  const int pos = i ? s->p1pos : s->p0pos;
  int off[3];
  const int n = nusiz_copies(mode, off);
  for (int k = 0; k < n; k++) {
    const int d = ((x - pos - off[k]) % 160 + 160) % 160;
    if (d < 8 * sc) {
      const int b = d / sc;
      if ((s->refp[i] & 8) ? (g >> b) & 1 : (g >> (7 - b)) & 1) return 1;
    }
  }
  return 0;
}
static int p0_bit(const ovcs* s, int x) { return player_bit(s, 0, x); }

/* Missile i: ENAMi bit 1 and not locked to its player (RESMPi bit 1),
 * 1 << NUSIZi bits 4-5 columns wide, in the player's copies (one copy for
 * the double and quad sizes). */
static int missile_bit(const ovcs* s, int i, int x) {
  if (!(s->enam[i] & 2) || (s->resmp[i] & 2)) return 0;
  const int mode = s->nusiz[i] & 7, w = 1 << ((s->nusiz[i] >> 4) & 3);
  int off[3];
  const int n = nusiz_copies(mode, off);
  for (int k = 0; k < n; k++)
    if (((x - s->mpos[i] - off[k]) % 160 + 160) % 160 < w) return 1;
  return 0;
}

/* The ball: ENABL bit 1 (the delayed copy when VDELBL is set), 1 << CTRLPF
 * bits 4-5 columns wide. */
static int ball_bit(const ovcs* s, int x) {
  const int en = (s->vdelbl & 1) ? s->enablo : s->enabl;
  if (!(en & 2)) return 0;
  return ((x - s->blpos) % 160 + 160) % 160 < (1 << ((s->ctrlpf >> 4) & 3));
}

/* Colour owner of a column from the objects present there: 0 = COLUP0
 * (P0, M0), 3 = COLUP1 (P1, M1), 1 = COLUPF (PF, BL), 2 = COLUBK.  CTRLPF
 * bit 2 clear: P0/M0 > P1/M1 > PF/BL > BK, the playfield taking COLUP0 in
 * the left half and COLUP1 in the right one in score mode (bit 1); bit 2
 * set: PF/BL > P0/M0 > P1/M1 > BK. */
static int owner_of(const ovcs* s, int x, int p0, int m0, int p1, int m1, int pf, int bl) {
  if (!s->full_tia && !(s->ctrlpf & 4)) return p0 ? 0 : (pf ? 1 : 2);   /* no score mode in the subset */
  if (s->ctrlpf & 4) {
    if (pf || bl) return 1;
    if (p0 || m0) return 0;
    if (p1 || m1) return 3;
    return 2;
  }
  if (p0 || m0) return 0;
  if (p1 || m1) return 3;
  if (pf) return (s->ctrlpf & 2) ? (x < 80 ? 0 : 3) : 1;
  if (bl) return 1;
  return 2;
}
static uint8_t owner_colour(const ovcs* s, int o) {
  return o == 0 ? s->colup0 : (o == 1 ? s->colupf : (o == 2 ? s->colubk : s->colup1));
}

/* Collisions at column x (every visible column of every line, whether or
 * not VBLANK or the HMOVE blank hides it): latch each overlapping pair. */
static void collide(ovcs* s, int x) {
  const int p0 = player_bit(s, 0, x), p1 = player_bit(s, 1, x), m0 = missile_bit(s, 0, x);
  const int m1 = missile_bit(s, 1, x), bl = ball_bit(s, x), pf = pf_bit(s, x);
  const int pair[16] = {m0 && p0, m0 && p1, m1 && p1, m1 && p0, p0 && bl, p0 && pf, p1 && bl, p1 && pf,
                        m0 && bl, m0 && pf, m1 && bl, m1 && pf, 0, bl && pf, m0 && m1, p0 && p1};
  for (int k = 0; k < 16; k++)
    if (pair[k]) s->cx |= (uint16_t)(1u << k);
}

/* Registers only the whole TIA has (the subset machine ignores writes to
 * them): NUSIZ0/1, COLUP1, REFP0/1, RESP1, RESM0/1, RESBL, GRP1, ENAM0/1,
 * ENABL, HMP1, HMM0/1, HMBL, VDELP0/1, VDELBL, RESMP0/1, CXCLR. */
static int full_tia_reg(int reg) {
  return reg == 0x04 || reg == 0x05 || reg == 0x07 || reg == 0x0B || reg == 0x0C || (reg >= 0x11 && reg <= 0x14) ||
         (reg >= 0x1C && reg <= 0x1F) || (reg >= 0x21 && reg <= 0x29) || reg == 0x2C;
}

/* Differentiable position sampler (Section 3, the sub-pixel bilinear kernel
 * over sprite position): player 0's coverage of column x relaxed with a
 * triangular kernel, cov(x) = sum_k b_k tri(x - pos - k) over its drawn
 * columns (copies, size and reflection included).  Its derivative with
 * respect to pos at the integer hard point, taken symmetrically, is
 * (b(x - 1) - b(x + 1)) / 2 with b the hard coverage, so d pixel / d pos =
 * (C_with - C_without) (b(x - 1) - b(x + 1)) / 2, where C_with and
 * C_without are the colours the pixel has with and without a player-0
 * pixel there (the priority logic decides both; zero where the player is
 * hidden).  Blanked pixels carry nothing (the caller skips them). */
static double sampler_slope(const ovcs* s, int x) {
  /* the player's relaxed coverage slope at x, times the colour the pixel
   * has with a player pixel there minus the colour without one */
  const int db = p0_bit(s, ((x - 1) % 160 + 160) % 160) - p0_bit(s, (x + 1) % 160);
  if (!db) return 0.0;
  const int p1 = player_bit(s, 1, x), m0 = missile_bit(s, 0, x), m1 = missile_bit(s, 1, x);
  const int bl = ball_bit(s, x), pf = pf_bit(s, x);
  const int with = owner_colour(s, owner_of(s, x, 1, m0, p1, m1, pf, bl)) & 0xFE;
  const int without = owner_colour(s, owner_of(s, x, 0, m0, p1, m1, pf, bl)) & 0xFE;
  return 0.5 * (double)db * (double)(with - without);
}

/* Graphics-bit surrogate (Section 3.1, the stored-switch paragraph: sprite
 * colours and graphics bits are differentiable with the switch stored).
 * Reading: the pixel's colour is relaxed in the graphics bit that decides
 * whether object k covers column x, as C_without + (C_with - C_without) b,
 * where C_with and C_without are the colours the priority logic gives
 * with that bit forced to 1 and to 0 (the other objects as drawn, colours
 * & 0xFE); the bit's derivative with respect to its register byte is 1
 * (the straight-through rule for the shift and mask that extract it, as
 * for LSR and AND).  So every drawn pixel adds (C_with - C_without) x its
 * gradient to the byte of each bit in play there: the player's GRP bit at
 * that column (the delayed copy when VDELP is set), the missile's ENAM and
 * the ball's ENABL byte where the object's span covers x (the delayed
 * ENABL with VDELBL; a missile locked to its player is not in play), and
 * the playfield byte (PF0, PF1 or PF2) of x.  The subset machine has only
 * player 0 and the playfield. */
static int player_span(const ovcs* s, int i, int x) {
  const int mode = s->nusiz[i] & 7, w = 8 * player_scale(mode);
  const int pos = i ? s->p1pos : s->p0pos;
  int off[3];
  const int n = nusiz_copies(mode, off);
  for (int k = 0; k < n; k++)
    if (((x - pos - off[k]) % 160 + 160) % 160 < w) return 1;
  return 0;
}
static int missile_span(const ovcs* s, int i, int x) {
  if (s->resmp[i] & 2) return 0;
  const int mode = s->nusiz[i] & 7, w = 1 << ((s->nusiz[i] >> 4) & 3);
  int off[3];
  const int n = nusiz_copies(mode, off);
  for (int k = 0; k < n; k++)
    if (((x - s->mpos[i] - off[k]) % 160 + 160) % 160 < w) return 1;
  return 0;
}
static int ball_span(const ovcs* s, int x) {
  return ((x - s->blpos) % 160 + 160) % 160 < (1 << ((s->ctrlpf >> 4) & 3));
}
/* The playfield register (0 PF0, 1 PF1, 2 PF2) of column x. */
static int pf_reg(const ovcs* s, int x) {
  int i = x < 80 ? x / 4 : (x - 80) / 4;
  if (x >= 80 && (s->ctrlpf & 1)) i = 19 - i;
  return i < 4 ? 0 : (i < 12 ? 1 : 2);
}
static void graphics_seed(ovcs* s, int x, double w) {
  int b[6] = {player_bit(s, 0, x), missile_bit(s, 0, x), player_bit(s, 1, x), missile_bit(s, 1, x),
              pf_bit(s, x), ball_bit(s, x)};   /* P0, M0, P1, M1, PF, BL */
  int32_t node[6] = {0, 0, 0, 0, 0, 0};
  if (player_span(s, 0, x)) node[0] = (s->vdelp[0] & 1) ? s->nGo[0] : s->nG[0];
  node[4] = s->nG[5 + pf_reg(s, x)];
  if (s->full_tia) {
    if (missile_span(s, 0, x)) node[1] = s->nG[2];
    if (player_span(s, 1, x)) node[2] = (s->vdelp[1] & 1) ? s->nGo[1] : s->nG[1];
    if (missile_span(s, 1, x)) node[3] = s->nG[3];
    if (ball_span(s, x)) node[5] = (s->vdelbl & 1) ? s->nGo[2] : s->nG[4];
  }
  for (int k = 0; k < 6; k++) {
    if (!node[k]) continue;
    const int keep = b[k];
    b[k] = 1;
    const int with = owner_colour(s, owner_of(s, x, b[0], b[1], b[2], b[3], b[4], b[5])) & 0xFE;
    b[k] = 0;
    const int without = owner_colour(s, owner_of(s, x, b[0], b[1], b[2], b[3], b[4], b[5])) & 0xFE;
    b[k] = keep;
    if (with != without) s->g->seed[node[k]] += w * (double)(with - without);
  }
}

/* Pixel at visible column x of the current scanline; *owner = the colour
 * register that owns it (owner_of) or -1 (blanked). */
static uint8_t pixel(const ovcs* s, int x, int* owner) {
  if (s->vblank & 2) { *owner = -1; return 0; }
  if (s->hmove_line == s->line && x < 8) { *owner = -1; return 0; }
  const int o = owner_of(s, x, player_bit(s, 0, x), missile_bit(s, 0, x), player_bit(s, 1, x),
                         missile_bit(s, 1, x), pf_bit(s, x), ball_bit(s, x));
  *owner = o;
  return owner_colour(s, o) & 0xFE;
}

static void tia_clock(ovcs* s) {
  if (s->hclk >= 68) {
    int x = s->hclk - 68, row = s->line - s->ystart;
    if (s->full_tia) collide(s, x);
    if (row >= 0 && row < SCR_H) {
      int owner;
      s->fb[row * SCR_W + x] = pixel(s, x, &owner);
      s->cnt.pixels++;
      if (s->g && s->gs && owner >= 0) {
        double w = s->gs[row * SCR_W + x];
        if (s->nC[owner]) s->g->seed[s->nC[owner]] += w;
        if (s->sampler && s->nPos) s->g->seed[s->nPos] += w * sampler_slope(s, x);
        if (s->graphics) graphics_seed(s, x, w);
      }
    }
  }
  if (++s->hclk == 228) { s->hclk = 0; s->line++; }
}

/* RESMPi bit 1 set: missile i is hidden and sits at its player's position
 * plus 4 x the player's pixel width minus 1 (near the player's centre). */
static void lock_missiles(ovcs* s) {
  for (int i = 0; i < 2; i++)
    if (s->resmp[i] & 2)
      s->mpos[i] = ((i ? s->p1pos : s->p0pos) + 4 * player_scale(s->nusiz[i] & 7) - 1) % 160;
}

static void tia_write(ovcs* s, int reg, val x) {
  uint8_t v = x.v;
  s->cnt.tia_writes++;
  if (!s->full_tia && full_tia_reg(reg)) return;
  switch (reg) {
    case 0x00:
      if (!(s->vsync & 2) && (v & 2)) frame_end(s);
      s->vsync = v;
      break;
    case 0x01: s->vblank = v; break;
    case 0x02: s->wsync = 1; break;
    case 0x04: s->nusiz[0] = v; lock_missiles(s); break;
    case 0x05: s->nusiz[1] = v; lock_missiles(s); break;
    case 0x06: s->colup0 = v; s->nC[0] = x.n; break;
    case 0x07: s->colup1 = v; s->nC[3] = x.n; break;
    case 0x08: s->colupf = v; s->nC[1] = x.n; break;
    case 0x09: s->colubk = v; s->nC[2] = x.n; break;
    case 0x0A: s->ctrlpf = v; break;
    case 0x0B: s->refp[0] = v; break;
    case 0x0C: s->refp[1] = v; break;
    case 0x0D: s->pf0 = v; s->nG[5] = x.n; break;
    case 0x0E: s->pf1 = v; s->nG[6] = x.n; break;
    case 0x0F: s->pf2 = v; s->nG[7] = x.n; break;
    case 0x10:   /* RESP0: a position from strobe timing carries no deviation */
      s->p0pos = s->hclk < 68 ? 3 : (s->hclk - 68 + 5) % 160;
      s->nPos = 0;
      lock_missiles(s);
      break;
    case 0x11: s->p1pos = s->hclk < 68 ? 3 : (s->hclk - 68 + 5) % 160; lock_missiles(s); break;
    /* RESM0, RESM1, RESBL: 2 in HBLANK, else the beam position plus 4 */
    case 0x12: s->mpos[0] = s->hclk < 68 ? 2 : (s->hclk - 68 + 4) % 160; lock_missiles(s); break;
    case 0x13: s->mpos[1] = s->hclk < 68 ? 2 : (s->hclk - 68 + 4) % 160; lock_missiles(s); break;
    case 0x14: s->blpos = s->hclk < 68 ? 2 : (s->hclk - 68 + 4) % 160; break;
    /* vertical delay: a GRP0 write copies GRP1 to its delayed register, a
     * GRP1 write copies GRP0 and ENABL to theirs */
    case 0x1B: s->grp0 = v; s->grpo[1] = s->grp1; s->nG[0] = x.n; s->nGo[1] = s->nG[1]; break;
    case 0x1C:
      s->grp1 = v; s->grpo[0] = s->grp0; s->enablo = s->enabl;
      s->nG[1] = x.n; s->nGo[0] = s->nG[0]; s->nGo[2] = s->nG[4];
      break;
    case 0x1D: s->enam[0] = v; s->nG[2] = x.n; break;
    case 0x1E: s->enam[1] = v; s->nG[3] = x.n; break;
    case 0x1F: s->enabl = v; s->nG[4] = x.n; break;
    case 0x20: s->hmp0 = v; s->nHM = x.n; break;
    case 0x21: s->hmp1 = v; break;
    case 0x22: s->hmm[0] = v; break;
    case 0x23: s->hmm[1] = v; break;
    case 0x24: s->hmbl = v; break;
    case 0x25: s->vdelp[0] = v; break;
    case 0x26: s->vdelp[1] = v; break;
    case 0x27: s->vdelbl = v; break;
    case 0x28: s->resmp[0] = v; lock_missiles(s); break;
    case 0x29: s->resmp[1] = v; lock_missiles(s); break;
    case 0x2A: {   /* HMOVE: every object moves by minus its signed motion nibble (the subset: player 0) */
      int m = ((int8_t)s->hmp0) >> 4;
      s->p0pos = ((s->p0pos - m) % 160 + 160) % 160;
      /* the motion is minus the high nibble of HMP0: a deviation of HMP0
       * moves the player by minus a sixteenth of it (straight-through) */
      if (s->sampler) s->nPos = lin2(s, s->nPos, 1.0, s->nHM, -1.0 / 16.0);
      s->p1pos = ((s->p1pos - (((int8_t)s->hmp1) >> 4)) % 160 + 160) % 160;
      for (int i = 0; i < 2; i++) s->mpos[i] = ((s->mpos[i] - (((int8_t)s->hmm[i]) >> 4)) % 160 + 160) % 160;
      s->blpos = ((s->blpos - (((int8_t)s->hmbl) >> 4)) % 160 + 160) % 160;
      lock_missiles(s);
      if (s->hclk <= 9) s->hmove_line = s->line;
      break;
    }
    case 0x2B:   /* HMCLR */
      s->hmp0 = 0; s->nHM = 0;
      s->hmp1 = s->hmm[0] = s->hmm[1] = s->hmbl = 0;
      break;
    case 0x2C: s->cx = 0; break;   /* CXCLR */
    default: break;
  }
}

/* ---------------- RIOT ---------------- */

static void riot_tick(ovcs* s) {
  if (s->underflow) {
    s->intim--;
  } else {
    if (s->phase == 0) {
      if (s->intim == 0) { s->intim = 0xFF; s->underflow = 1; }
      else s->intim--;
    }
    s->phase = (s->phase + 1) % s->interval;
  }
}

static void timer_write(ovcs* s, int sel, val x) {
  static const uint32_t iv[4] = {1, 8, 64, 1024};
  s->intim = x.v;
  s->interval = iv[sel];
  s->phase = 0;
  s->underflow = 0;
  s->nV = x.n;
}

/* ---------------- bus ---------------- */

static void tick(ovcs* s) {
  s->cyc++;
  s->cnt.cycles++;
  riot_tick(s);
  tia_clock(s);
  tia_clock(s);
  tia_clock(s);
}

static void idle(ovcs* s) { tick(s); }

/* The banked format under a Superchip variant (F8SC -> F8, ...). */
static int base_mapper(const ovcs* s) { return s->fe ? 2 : s->sc ? s->mapper - 3 : s->mapper; }

static void hotspot(ovcs* s, uint16_t a) {
  if (s->fe) return;   /* FE has no hotspot: see fe_switch */
  if (s->e0) {   /* $1FE0-$1FE7, $1FE8-$1FEF, $1FF0-$1FF7: segment 0, 1, 2 */
    if (a >= 0x1FE0 && a <= 0x1FF7) s->e0seg[(a - 0x1FE0) / 8] = (a - 0x1FE0) % 8;
    return;
  }
  /* F8: $1FF8-$1FF9, F6: $1FF6-$1FF9, F4: $1FF4-$1FFB select banks 0.. */
  static const int first[5] = {0, 0, 0x1FF8, 0x1FF6, 0x1FF4}, count[5] = {0, 0, 2, 4, 8};
  const int m = base_mapper(s);
  if (a >= first[m] && a < first[m] + count[m]) {
    s->bank = a - first[m];
  }
}

/* FE (8 KB, two 4 KB banks): the cartridge watches the bus for an access
 * to $01FE and takes the bank from bit 5 of the byte on the data bus in the
 * next cycle: set (a high address byte $Fx) shows the image's first 4 KB,
 * clear ($Dx) the second.  Reading: the accesses modelled are the two that
 * the format's carts switch with, made at the top of the stack: a JSR
 * whose push of the return address's low byte lands on $01FE (the stack
 * pointer was $FF; the next cycle fetches the target's high byte) and an
 * RTS whose pull of the low byte reads $01FE (the stack pointer was $FD;
 * the next cycle pulls the high byte).  The byte decides the bank from the
 * cycle after it on; power-on shows the first 4 KB. */
static void fe_switch(ovcs* s, uint8_t next_byte) { s->bank = (next_byte & 0x20) ? 0 : 1; }

/* Superchip ports: cell of the cartridge RAM read (write) at cartridge
 * address a, or -1. */
static int sc_read_cell(const ovcs* s, uint16_t a) {
  return s->sc && (a & 0x1F80) == 0x1080 ? 128 + (a & 0x7F) : -1;
}
static int sc_write_cell(const ovcs* s, uint16_t a) {
  return s->sc && (a & 0x1F80) == 0x1000 ? 128 + (a & 0x7F) : -1;
}

static void rom_map(const ovcs* s, uint16_t a, int* base, int* M, int* idx) {
  if (s->e0) {
    const int seg = (a >> 10) & 3;
    *base = 1024 * (seg == 3 ? 7 : s->e0seg[seg]);
    *M = 1024;
    *idx = a & 0x3FF;
    return;
  }
  if (base_mapper(s) == 0) { *base = 0; *M = 2048; *idx = a & 0x7FF; }
  else if (base_mapper(s) == 1) { *base = 0; *M = 4096; *idx = a & 0xFFF; }
  else { *base = s->bank * 4096; *M = 4096; *idx = a & 0xFFF; }
}

/* FULL mode's temperature read (Section 4, the fully relaxed forward): the
 * byte at index a of a memory tensor t[0..M) read as
 * round(sum_k w_k t[k] / sum_k w_k) with w_k = e^{-|k - a| / T} over the
 * frozen window |k - a| <= W clipped to the tensor, in float32 (the soft
 * state's precision), terms added in index order, rounded half to even. */
static uint8_t full_read(const ovcs* s, const uint8_t* t, int M, int a) {
  const int lo = a - s->full_W < 0 ? 0 : a - s->full_W;
  const int hi = a + s->full_W > M - 1 ? M - 1 : a + s->full_W;
  float num = 0.0f, den = 0.0f;
  for (int k = lo; k <= hi; k++) {
    const float w = s->full_ek[k > a ? k - a : a - k];
    num += w * (float)t[k];
    den += w;
  }
  float v = rintf(num / den);
  if (v < 0.0f) v = 0.0f;
  if (v > 255.0f) v = 255.0f;
  return (uint8_t)v;
}

/* A read of a memory tensor through the relaxed cast: counted in probe and
 * FULL modes, applied in FULL mode. */
static uint8_t full_cast(ovcs* s, const uint8_t* t, int M, int a) {
  const uint8_t v = full_read(s, t, M, a);
  s->cnt.relaxed_reads++;
  if (v == t[a]) s->cnt.relaxed_reads_exact++;
  return s->full == 2 ? v : t[a];
}

/* Collision read register r (CXM0P .. CXPPMM): its two latches in D7, D6. */
static uint8_t collision_reg(const ovcs* s, int r) { return (uint8_t)(((s->cx >> (2 * r)) & 3) << 6); }

/* One bus read cycle. */
static val rd(ovcs* s, uint16_t addr) {
  tick(s);
  uint16_t a = addr & 0x1FFF;
  val r = {0, 0};
  if (sc_read_cell(s, a) >= 0) {   /* the Superchip's read port */
    const int i = a & 0x7F;
    r.v = s->full ? full_cast(s, s->ram + 128, 128, i) : s->ram[128 + i];
    r.n = g_read_ram(s, 128, i);
    s->cnt.ram_reads++;
  } else if (a & 0x1000) {
    hotspot(s, a);
    int base, M, idx;
    rom_map(s, a, &base, &M, &idx);
    r.v = s->full ? full_cast(s, s->rom + base, M, idx) : s->rom[base + idx];
    r.n = g_read_rom(s, base, M, idx);
    s->cnt.rom_reads++;
  } else if (!(a & 0x80)) {
    switch (a & 0x0F) {
      case 0x0C: r.v = s->inpt4; r.n = s->g ? lin1(s, s->u_leaf + 4, -128.0) : 0; break;
      case 0x0D: r.v = 0x80; break;
      default: r.v = (a & 0x0F) < 8 ? collision_reg(s, a & 7) : 0; break;   /* no gradient: latched switches */
    }
  } else if (!(a & 0x200)) {
    r.v = s->full ? full_cast(s, s->ram, 128, a & 0x7F) : s->ram[a & 0x7F];
    r.n = g_read_ram(s, 0, a & 0x7F);
    s->cnt.ram_reads++;
  } else if (!(a & 0x04)) {
    switch (a & 3) {
      case 0:
        r.v = s->swcha;
        if (s->g) {
          int32_t in[4] = {s->u_leaf + 0, s->u_leaf + 1, s->u_leaf + 2, s->u_leaf + 3};
          double c[4] = {-128.0, -64.0, -32.0, -16.0};
          r.n = g_lin(s, 4, in, c);
        }
        break;
      case 2: r.v = s->swchb; break;
      default: r.v = 0; break;
    }
  } else if (a & 1) {
    r.v = s->underflow ? 0x80 : 0x00;
  } else {
    r.v = s->intim;
    r.n = s->underflow ? 0 : s->nV;
  }
  return r;
}

/* Side-effect-free read (opcode and debug); still a bus cycle when `cycle`. */
static uint8_t peek_raw(ovcs* s, uint16_t addr) {
  uint16_t a = addr & 0x1FFF;
  if (sc_read_cell(s, a) >= 0) return s->ram[sc_read_cell(s, a)];
  if (a & 0x1000) {
    int base, M, idx;
    rom_map(s, a, &base, &M, &idx);
    return s->rom[base + idx];
  }
  if (!(a & 0x80))
    return (a & 0x0F) == 0x0C ? s->inpt4 : ((a & 0x0F) == 0x0D ? 0x80 : ((a & 0x0F) < 8 ? collision_reg(s, a & 7) : 0));
  if (!(a & 0x200)) return s->ram[a & 0x7F];
  if (!(a & 0x04)) return (a & 3) == 0 ? s->swcha : ((a & 3) == 2 ? s->swchb : 0);
  return (a & 1) ? (s->underflow ? 0x80 : 0) : s->intim;
}

/* Opcode fetch: a full read cycle whose value is a switch (no deviation). */
static uint8_t fetch_opcode(ovcs* s) {
  tick(s);
  uint16_t a = s->pc & 0x1FFF;
  if (a & 0x1000) { hotspot(s, a); s->cnt.rom_reads++; }
  uint8_t v = peek_raw(s, s->pc);
  s->pc++;
  return v;
}

static void wr(ovcs* s, uint16_t addr, val x) {
  tick(s);
  uint16_t a = addr & 0x1FFF;
  if (a & 0x1000) {
    hotspot(s, a);
    const int cell = sc_write_cell(s, a);
    if (cell >= 0) {   /* the Superchip's write port */
      s->ram[cell] = x.v;
      s->nRAM[cell] = x.n;
      s->cnt.ram_writes++;
    }
    return;
  }
  if (!(a & 0x80)) {
    tia_write(s, a & 0x3F, x);
    if (s->wsync) {
      s->wsync = 0;
      while (s->cyc % 76 != 0) tick(s);
    }
    return;
  }
  if (!(a & 0x200)) {
    s->ram[a & 0x7F] = x.v;
    s->nRAM[a & 0x7F] = x.n;
    s->cnt.ram_writes++;
    return;
  }
  if ((a & 0x04) && (a & 0x10)) timer_write(s, a & 3, x);
}

/* ---------------- frames ---------------- */

static void set_gs(ovcs* s) {
  /* pixel gradients weigh the frame a frame step returns (none in
   * instruction-granular steps) */
  if (s->g && s->gs_all && s->step_instr == 0 && s->frames_in_step == s->frame_skip - 1)
    s->gs = s->gs_all + (size_t)s->soft_step * SCR_H * SCR_W;
  else
    s->gs = NULL;
}

static void frame_end(ovcs* s) {
  memcpy(s->last_fb, s->fb, sizeof s->fb);
  memset(s->fb, 0, sizeof s->fb);
  s->line = 0;
  s->hmove_line = -1;
  s->frames_in_step++;
  s->cnt.frames++;
  set_gs(s);
}

/* ---------------- CPU ---------------- */

#define FC 0x01
#define FZ 0x02
#define FI 0x04
#define FD 0x08
#define FV 0x40
#define FN 0x80

static void set_nz(ovcs* s, uint8_t v) {
  s->P = (uint8_t)((s->P & ~(FN | FZ)) | (v & 0x80) | (v ? 0 : FZ));
}

static val fetch_operand(ovcs* s) {
  val r = rd(s, s->pc);
  s->pc++;
  return r;
}

/* Effective address of the memory operand.  Addresses are indices and so
 * stored switches in soft mode: they carry no deviation. */
enum { M_IMP, M_ACC, M_IMM, M_ZP, M_ZPX, M_ZPY, M_ABS, M_ABX, M_ABY, M_INX, M_INY };
enum { K_READ, K_WRITE, K_RMW };

static uint16_t address(ovcs* s, int mode, int kind) {
  uint16_t ea = 0;
  switch (mode) {
    case M_ZP:
      ea = fetch_operand(s).v;
      break;
    case M_ZPX:
    case M_ZPY: {
      uint8_t o = fetch_operand(s).v;
      idle(s);
      ea = (uint8_t)(o + (mode == M_ZPX ? s->X : s->Y));
      break;
    }
    case M_ABS: {
      uint8_t lo = fetch_operand(s).v;
      uint8_t hi = fetch_operand(s).v;
      ea = (uint16_t)(lo | (hi << 8));
      break;
    }
    case M_ABX:
    case M_ABY: {
      uint8_t lo = fetch_operand(s).v;
      uint8_t hi = fetch_operand(s).v;
      uint16_t base = (uint16_t)(lo | (hi << 8));
      ea = (uint16_t)(base + (mode == M_ABX ? s->X : s->Y));
      if (kind != K_READ || ((base & 0xFF00) != (ea & 0xFF00))) idle(s);
      break;
    }
    case M_INX: {
      uint8_t o = fetch_operand(s).v;
      idle(s);
      uint8_t p = (uint8_t)(o + s->X);
      uint8_t lo = rd(s, p).v;
      uint8_t hi = rd(s, (uint8_t)(p + 1)).v;
      ea = (uint16_t)(lo | (hi << 8));
      break;
    }
    case M_INY: {
      uint8_t o = fetch_operand(s).v;
      uint8_t lo = rd(s, o).v;
      uint8_t hi = rd(s, (uint8_t)(o + 1)).v;
      uint16_t base = (uint16_t)(lo | (hi << 8));
      ea = (uint16_t)(base + s->Y);
      if (kind != K_READ || ((base & 0xFF00) != (ea & 0xFF00))) idle(s);
      break;
    }
    default: break;
  }
  return ea;
}

/* Operand value for read instructions (immediate or memory). */
static val operand(ovcs* s, int mode) {
  if (mode == M_IMM) return fetch_operand(s);
  return rd(s, address(s, mode, K_READ));
}

static void push(ovcs* s, val x) {
  wr(s, (uint16_t)(0x100 | s->SP), x);
  s->SP--;
}
static val pull(ovcs* s) {
  s->SP++;
  return rd(s, (uint16_t)(0x100 | s->SP));
}

static void op_adc(ovcs* s, uint8_t m) {
  int c = s->P & FC;
  if (s->P & FD) {
    uint8_t bin = (uint8_t)(s->A + m + c);
    int al = (s->A & 0x0F) + (m & 0x0F) + c;
    if (al >= 0x0A) al = ((al + 0x06) & 0x0F) + 0x10;
    int sum = (s->A & 0xF0) + (m & 0xF0) + al;
    int ssum = (int)(int8_t)(s->A & 0xF0) + (int)(int8_t)(m & 0xF0) + al;
    uint8_t p = (uint8_t)(s->P & ~(FN | FV | FZ | FC));
    if (ssum & 0x80) p |= FN;
    if (ssum < -128 || ssum > 127) p |= FV;
    if (bin == 0) p |= FZ;
    if (sum >= 0xA0) sum += 0x60;
    if (sum >= 0x100) p |= FC;
    s->A = (uint8_t)sum;
    s->P = p;
  } else {
    int t = s->A + m + c;
    uint8_t r = (uint8_t)t;
    uint8_t p = (uint8_t)(s->P & ~(FN | FV | FZ | FC));
    if (t > 0xFF) p |= FC;
    if (~(s->A ^ m) & (s->A ^ r) & 0x80) p |= FV;
    s->A = r;
    s->P = p;
    set_nz(s, r);
  }
}

static void op_sbc(ovcs* s, uint8_t m) {
  int c = s->P & FC;
  /* flags are those of the binary subtraction in both modes */
  int t = s->A + (m ^ 0xFF) + c;
  uint8_t r = (uint8_t)t;
  uint8_t p = (uint8_t)(s->P & ~(FN | FV | FZ | FC));
  if (t > 0xFF) p |= FC;
  if (~(s->A ^ (m ^ 0xFF)) & (s->A ^ r) & 0x80) p |= FV;
  if (r & 0x80) p |= FN;
  if (r == 0) p |= FZ;
  if (s->P & FD) {
    int al = (s->A & 0x0F) - (m & 0x0F) + c - 1;
    if (al < 0) al = ((al - 0x06) & 0x0F) - 0x10;
    int sum = (s->A & 0xF0) - (m & 0xF0) + al;
    if (sum < 0) sum -= 0x60;
    r = (uint8_t)sum;
  }
  s->A = r;
  s->P = p;
}

static void op_cmp(ovcs* s, uint8_t reg, uint8_t m) {
  uint8_t t = (uint8_t)(reg - m);
  s->P = (uint8_t)((s->P & ~FC) | (reg >= m ? FC : 0));
  set_nz(s, t);
}

/* shift/rotate: kind 0 ASL, 1 ROL, 2 LSR, 3 ROR */
static uint8_t op_shift(ovcs* s, int kind, uint8_t v) {
  int cin = s->P & FC;
  int cout;
  uint8_t r;
  switch (kind) {
    case 0: cout = v >> 7; r = (uint8_t)(v << 1); break;
    case 1: cout = v >> 7; r = (uint8_t)((v << 1) | cin); break;
    case 2: cout = v & 1; r = (uint8_t)(v >> 1); break;
    default: cout = v & 1; r = (uint8_t)((v >> 1) | (cin << 7)); break;
  }
  s->P = (uint8_t)((s->P & ~FC) | (cout ? FC : 0));
  set_nz(s, r);
  return r;
}

/* Conditional branch.  In soft mode the STE gate of Eq. s-branch returns the
 * hard counter; the counter is an index (a stored switch), so the gate's
 * derivative has no consumer among the gradient outputs. */
static void branch(ovcs* s, int cond) {
  uint8_t off = fetch_operand(s).v;
  if (s->full) {
    /* Eq. branch without the straight-through correction: the crisp flag
     * gives z = +1 (condition holds) or -1, gate g = sigma(alpha z), and the
     * counter is the blend rounded back to an integer, in float32:
     * round(pc_fall + g delta).  A taken branch pays its cycle, and the page
     * cross is between the fall-through and the new counter. */
    const uint16_t fall = s->pc;
    const float g = cond ? s->full_g1 : s->full_g0;
    const float pcf = (float)fall + g * (float)(int8_t)off;
    const uint16_t rel = (uint16_t)(long)rintf(pcf);
    const uint16_t hard = cond ? (uint16_t)(fall + (int8_t)off) : fall;
    s->cnt.branches++;
    if (rel == hard) s->cnt.branches_exact++;
    if (s->full == 2) {
      if (cond) {
        idle(s);
        if ((rel & 0xFF00) != (fall & 0xFF00)) idle(s);
      }
      s->pc = rel;
      return;
    }
  }
  if (cond) {
    uint16_t t = (uint16_t)(s->pc + (int8_t)off);
    idle(s);
    if ((t & 0xFF00) != (s->pc & 0xFF00)) idle(s);
    s->pc = t;
  }
}

/* group tables for the regular ALU column (cc = 01) */
static const int mode01[8] = {M_INX, M_ZP, M_IMM, M_ABS, M_INY, M_ZPX, M_ABY, M_ABX};

static void exec(ovcs* s) {
  uint8_t op = fetch_opcode(s);
  s->cnt.instructions++;
  int aaa = op >> 5, bbb = (op >> 2) & 7, cc = op & 3;

  if (cc == 1) {                       /* ORA AND EOR ADC STA LDA CMP SBC */
    int mode = mode01[bbb];
    if (aaa == 4) {                    /* STA */
      if (mode == M_IMM) {             /* $89: no STA #imm; one of the extra NOP #imm bytes */
        (void)operand(s, M_IMM);
        return;
      }
      val x = {s->A, s->nA};
      wr(s, address(s, mode, K_WRITE), x);
      return;
    }
    val m = operand(s, mode);
    switch (aaa) {
      case 0: s->A |= m.v; s->nA = lin2(s, s->nA, 1.0, m.n, 1.0); set_nz(s, s->A); break;
      case 1: s->A &= m.v; s->nA = lin2(s, s->nA, 1.0, m.n, 1.0); set_nz(s, s->A); break;
      case 2: s->A ^= m.v; s->nA = lin2(s, s->nA, 1.0, m.n, 1.0); set_nz(s, s->A); break;
      case 3: op_adc(s, m.v); s->nA = lin2(s, s->nA, 1.0, m.n, 1.0); break;
      case 5: s->A = m.v; s->nA = m.n; set_nz(s, s->A); break;
      case 6: op_cmp(s, s->A, m.v); break;
      case 7: op_sbc(s, m.v); s->nA = lin2(s, s->nA, 1.0, m.n, -1.0); break;
    }
    return;
  }

  switch (op) {
    /* ---- shifts / rotates / inc / dec on memory and A ---- */
    case 0x0A: case 0x2A: case 0x4A: case 0x6A: {
      idle(s);
      s->A = op_shift(s, aaa, s->A);   /* straight-through: unit derivative */
      return;
    }
    case 0x06: case 0x16: case 0x0E: case 0x1E:
    case 0x26: case 0x36: case 0x2E: case 0x3E:
    case 0x46: case 0x56: case 0x4E: case 0x5E:
    case 0x66: case 0x76: case 0x6E: case 0x7E:
    case 0xC6: case 0xD6: case 0xCE: case 0xDE:
    case 0xE6: case 0xF6: case 0xEE: case 0xFE: {
      int mode = bbb == 1 ? M_ZP : bbb == 3 ? M_ABS : bbb == 5 ? M_ZPX : M_ABX;
      uint16_t ea = address(s, mode, K_RMW);
      val m = rd(s, ea);
      idle(s);                         /* RMW dummy write (not modelled) */
      val r;
      if (aaa <= 3) {
        r.v = op_shift(s, aaa, m.v);   /* straight-through: unit derivative */
        r.n = m.n;
      } else {
        r.v = (uint8_t)(aaa == 6 ? m.v - 1 : m.v + 1);
        r.n = m.n;
        set_nz(s, r.v);
      }
      wr(s, ea, r);
      return;
    }
    /* ---- loads / stores of X and Y ---- */
    case 0xA2: case 0xA6: case 0xB6: case 0xAE: case 0xBE: {
      int mode = op == 0xA2 ? M_IMM : op == 0xA6 ? M_ZP : op == 0xB6 ? M_ZPY : op == 0xAE ? M_ABS : M_ABY;
      val m = operand(s, mode);
      s->X = m.v; s->nX = m.n; set_nz(s, s->X);
      return;
    }
    case 0xA0: case 0xA4: case 0xB4: case 0xAC: case 0xBC: {
      int mode = op == 0xA0 ? M_IMM : op == 0xA4 ? M_ZP : op == 0xB4 ? M_ZPX : op == 0xAC ? M_ABS : M_ABX;
      val m = operand(s, mode);
      s->Y = m.v; s->nY = m.n; set_nz(s, s->Y);
      return;
    }
    case 0x86: case 0x96: case 0x8E: {
      val x = {s->X, s->nX};
      wr(s, address(s, op == 0x86 ? M_ZP : op == 0x96 ? M_ZPY : M_ABS, K_WRITE), x);
      return;
    }
    case 0x84: case 0x94: case 0x8C: {
      val x = {s->Y, s->nY};
      wr(s, address(s, op == 0x84 ? M_ZP : op == 0x94 ? M_ZPX : M_ABS, K_WRITE), x);
      return;
    }
    /* ---- compares and BIT ---- */
    case 0xE0: case 0xE4: case 0xEC: {
      val m = operand(s, op == 0xE0 ? M_IMM : op == 0xE4 ? M_ZP : M_ABS);
      op_cmp(s, s->X, m.v);
      return;
    }
    case 0xC0: case 0xC4: case 0xCC: {
      val m = operand(s, op == 0xC0 ? M_IMM : op == 0xC4 ? M_ZP : M_ABS);
      op_cmp(s, s->Y, m.v);
      return;
    }
    case 0x24: case 0x2C: {
      val m = operand(s, op == 0x24 ? M_ZP : M_ABS);
      s->P = (uint8_t)((s->P & ~(FN | FV | FZ)) | (m.v & (FN | FV)) | ((s->A & m.v) ? 0 : FZ));
      return;
    }
    /* ---- branches ---- */
    case 0x10: branch(s, !(s->P & FN)); return;
    case 0x30: branch(s, (s->P & FN) != 0); return;
    case 0x50: branch(s, !(s->P & FV)); return;
    case 0x70: branch(s, (s->P & FV) != 0); return;
    case 0x90: branch(s, !(s->P & FC)); return;
    case 0xB0: branch(s, (s->P & FC) != 0); return;
    case 0xD0: branch(s, !(s->P & FZ)); return;
    case 0xF0: branch(s, (s->P & FZ) != 0); return;
    /* ---- jumps and subroutines ---- */
    case 0x4C: {
      uint8_t lo = fetch_operand(s).v;
      uint8_t hi = fetch_operand(s).v;
      s->pc = (uint16_t)(lo | (hi << 8));
      return;
    }
    case 0x6C: {
      uint8_t lo = fetch_operand(s).v;
      uint8_t hi = fetch_operand(s).v;
      uint16_t p = (uint16_t)(lo | (hi << 8));
      uint8_t l2 = rd(s, p).v;
      uint8_t h2 = rd(s, (uint16_t)((p & 0xFF00) | ((p + 1) & 0xFF))).v;
      s->pc = (uint16_t)(l2 | (h2 << 8));
      return;
    }
    case 0x20: {
      uint8_t lo = fetch_operand(s).v;
      idle(s);
      val ph = {(uint8_t)(s->pc >> 8), 0};
      val pl = {(uint8_t)(s->pc & 0xFF), 0};
      const int fe = s->fe && s->SP == 0xFF;   /* the low byte goes to $01FE */
      push(s, ph);
      push(s, pl);
      uint8_t hi = rd(s, s->pc).v;
      if (fe) fe_switch(s, hi);
      s->pc = (uint16_t)(lo | (hi << 8));
      return;
    }
    case 0x60: {
      idle(s);
      idle(s);
      const int fe = s->fe && s->SP == 0xFD;   /* the low byte comes from $01FE */
      uint8_t lo = pull(s).v;
      uint8_t hi = pull(s).v;
      if (fe) fe_switch(s, hi);
      idle(s);
      s->pc = (uint16_t)((lo | (hi << 8)) + 1);
      return;
    }
    case 0x40: {
      idle(s);
      idle(s);
      uint8_t p = pull(s).v;
      uint8_t lo = pull(s).v;
      uint8_t hi = pull(s).v;
      s->P = (uint8_t)(p | 0x30);
      s->pc = (uint16_t)(lo | (hi << 8));
      return;
    }
    case 0x00: {
      idle(s);                         /* padding byte */
      s->pc++;
      val ph = {(uint8_t)(s->pc >> 8), 0};
      val pl = {(uint8_t)(s->pc & 0xFF), 0};
      val pp = {(uint8_t)(s->P | 0x30), 0};
      push(s, ph);
      push(s, pl);
      push(s, pp);
      s->P |= FI;
      uint8_t lo = rd(s, 0xFFFE).v;
      uint8_t hi = rd(s, 0xFFFF).v;
      s->pc = (uint16_t)(lo | (hi << 8));
      return;
    }
    /* ---- stack ---- */
    case 0x48: { idle(s); val x = {s->A, s->nA}; push(s, x); return; }
    case 0x08: { idle(s); val x = {(uint8_t)(s->P | 0x30), 0}; push(s, x); return; }
    case 0x68: { idle(s); idle(s); val m = pull(s); s->A = m.v; s->nA = m.n; set_nz(s, s->A); return; }
    case 0x28: { idle(s); idle(s); val m = pull(s); s->P = (uint8_t)(m.v | 0x30); return; }
    /* ---- implied ---- */
    case 0x18: idle(s); s->P &= (uint8_t)~FC; return;
    case 0x38: idle(s); s->P |= FC; return;
    case 0x58: idle(s); s->P &= (uint8_t)~FI; return;
    case 0x78: idle(s); s->P |= FI; return;
    case 0xB8: idle(s); s->P &= (uint8_t)~FV; return;
    case 0xD8: idle(s); s->P &= (uint8_t)~FD; return;
    case 0xF8: idle(s); s->P |= FD; return;
    case 0xEA: idle(s); return;
    case 0xAA: idle(s); s->X = s->A; s->nX = s->nA; set_nz(s, s->X); return;
    case 0x8A: idle(s); s->A = s->X; s->nA = s->nX; set_nz(s, s->A); return;
    case 0xA8: idle(s); s->Y = s->A; s->nY = s->nA; set_nz(s, s->Y); return;
    case 0x98: idle(s); s->A = s->Y; s->nA = s->nY; set_nz(s, s->A); return;
    case 0xBA: idle(s); s->X = s->SP; s->nX = 0; set_nz(s, s->X); return;
    case 0x9A: idle(s); s->SP = s->X; return;
    case 0xE8: idle(s); s->X++; set_nz(s, s->X); return;
    case 0xCA: idle(s); s->X--; set_nz(s, s->X); return;
    case 0xC8: idle(s); s->Y++; set_nz(s, s->Y); return;
    case 0x88: idle(s); s->Y--; set_nz(s, s->Y); return;
    /* ---- the paper's 38 extra opcode bytes (unofficial NMOS opcodes) ---- */
    case 0xEB: {                       /* USBC #imm: SBC's alias */
      val m = operand(s, M_IMM);
      op_sbc(s, m.v);
      s->nA = lin2(s, s->nA, 1.0, m.n, -1.0);
      return;
    }
    case 0x1A: case 0x3A: case 0x5A: case 0x7A: case 0xDA: case 0xFA:
      idle(s);                         /* NOP */
      return;
    case 0x80: case 0x82: case 0x89: case 0xC2: case 0xE2:
      (void)operand(s, M_IMM);         /* NOP #imm */
      return;
    case 0x04: case 0x44: case 0x64:   /* NOP zp: the operand is read and dropped */
      (void)operand(s, M_ZP);
      return;
    case 0x14: case 0x34: case 0x54: case 0x74: case 0xD4: case 0xF4:
      (void)operand(s, M_ZPX);
      return;
    case 0x0C:
      (void)operand(s, M_ABS);
      return;
    case 0x1C: case 0x3C: case 0x5C: case 0x7C: case 0xDC: case 0xFC:
      (void)operand(s, M_ABX);
      return;
    case 0xA7: case 0xB7: case 0xAF: case 0xBF: case 0xA3: case 0xB3: {   /* LAX: A = X = M */
      int mode = op == 0xA7 ? M_ZP : op == 0xB7 ? M_ZPY : op == 0xAF ? M_ABS : op == 0xBF ? M_ABY
               : op == 0xA3 ? M_INX : M_INY;
      val m = operand(s, mode);
      s->A = s->X = m.v;
      s->nA = s->nX = m.n;
      set_nz(s, m.v);
      return;
    }
    case 0x87: case 0x97: case 0x8F: case 0x83: {                         /* SAX: M = A & X */
      int mode = op == 0x87 ? M_ZP : op == 0x97 ? M_ZPY : op == 0x8F ? M_ABS : M_INX;
      val x = {(uint8_t)(s->A & s->X), lin2(s, s->nA, 1.0, s->nX, 1.0)};
      wr(s, address(s, mode, K_WRITE), x);
      return;
    }
    default: break;
  }
jam:
  s->jammed = 1;
  s->cnt.instructions--;
}

/* One instruction slot: an instruction, or a jammed idle to the next line. */
static int step_instruction(ovcs* s) {
  uint64_t c0 = s->cyc;
  if (s->jammed) {
    do tick(s); while (s->cyc % 76 != 0);
  } else {
    exec(s);
  }
  return (int)(s->cyc - c0);
}

/* ------------------------------------------------------------------ */
/* public API                                                          */
/* ------------------------------------------------------------------ */

ovcs* ovcs_new(const uint8_t* rom, uint32_t rom_size, int mapper, int ystart) {
  static const uint32_t sz[10] = {2048, 4096, 8192, 16384, 32768, 8192, 16384, 32768, 8192, 8192};
  if (mapper < 0 || mapper > 9 || rom_size != sz[mapper]) return NULL;
  ovcs* s = (ovcs*)calloc(1, sizeof(ovcs));
  s->rom = (uint8_t*)malloc(rom_size);
  memcpy(s->rom, rom, rom_size);
  s->rom_size = rom_size;
  s->mapper = mapper;
  s->sc = mapper >= 5 && mapper <= 7;
  s->e0 = mapper == 8;
  s->fe = mapper == 9;
  s->ystart = ystart;
  ovcs_reset(s);
  return s;
}

void ovcs_set_switches(ovcs* s, uint8_t swchb) { s->swchb = swchb; }
void ovcs_set_sampler(ovcs* s, int on) { s->sampler = on != 0; }
void ovcs_set_graphics(ovcs* s, int on) { s->graphics = on != 0; }
void ovcs_set_full_tia(ovcs* s, int on) { s->full_tia = on != 0; }
void ovcs_set_step_instructions(ovcs* s, int n) { s->step_instr = n > 0 ? n : 0; }

static int half_width(double tau);
void ovcs_set_full(ovcs* s, int mode, double T, double alpha) {
  s->full = mode >= 0 && mode <= 2 && T > 0.0 ? mode : 0;
  if (!s->full) return;
  s->full_W = half_width(T);
  for (int k = 0; k <= s->full_W && k < 256; k++) s->full_ek[k] = (float)exp(-(double)k / T);
  s->full_g1 = (float)(1.0 / (1.0 + exp(-alpha)));
  s->full_g0 = (float)(1.0 / (1.0 + exp(alpha)));
}

void ovcs_free(ovcs* s) {
  if (!s) return;
  free(s->rom);
  free(s);
}

void ovcs_reset(ovcs* s) {
  s->A = s->X = s->Y = 0;
  s->SP = 0xFD;
  s->P = 0x34;
  s->cyc = 0;
  s->jammed = 0;
  memset(s->ram, 0, sizeof s->ram);
  /* F8 / F6 / F4 and their Superchip variants: the last bank; FE: the first */
  s->bank = s->mapper >= 2 && !s->e0 && !s->fe ? (int)(s->rom_size / 4096) - 1 : 0;
  s->e0seg[0] = 4;
  s->e0seg[1] = 5;
  s->e0seg[2] = 6;
  s->intim = 0;
  s->interval = 1024;
  s->phase = 0;
  s->underflow = 0;
  s->swcha = 0xFF;
  s->swchb = 0x0B;
  s->inpt4 = 0x80;
  s->vsync = s->vblank = s->colup0 = s->colupf = s->colubk = 0;
  s->ctrlpf = s->pf0 = s->pf1 = s->pf2 = s->grp0 = s->hmp0 = 0;
  s->p0pos = 0;
  s->colup1 = s->grp1 = s->enabl = s->enablo = s->hmp1 = s->hmbl = s->vdelbl = 0;
  for (int i = 0; i < 2; i++) {
    s->nusiz[i] = s->refp[i] = s->grpo[i] = s->enam[i] = s->hmm[i] = s->vdelp[i] = s->resmp[i] = 0;
    s->mpos[i] = 0;
  }
  s->p1pos = s->blpos = 0;
  s->cx = 0;
  s->hclk = 0;
  s->line = 0;
  s->hmove_line = -1;
  s->wsync = 0;
  memset(s->fb, 0, sizeof s->fb);
  memset(s->last_fb, 0, sizeof s->last_fb);
  memset(&s->cnt, 0, sizeof s->cnt);
  s->pc = (uint16_t)(peek_raw(s, 0x1FFC) | (peek_raw(s, 0x1FFD) << 8));
  s->frames_in_step = 0;
}

static void set_inputs(ovcs* s, const int u[5]) {
  s->swcha = (uint8_t)(0xFF - 128 * u[0] - 64 * u[1] - 32 * u[2] - 16 * u[3]);
  s->inpt4 = (uint8_t)(u[4] ? 0x00 : 0x80);
}

static const char* const kActionNames[18] = {
  "NOOP", "FIRE", "UP", "RIGHT", "LEFT", "DOWN", "UPRIGHT", "UPLEFT",
  "DOWNRIGHT", "DOWNLEFT", "UPFIRE", "RIGHTFIRE", "LEFTFIRE", "DOWNFIRE",
  "UPRIGHTFIRE", "UPLEFTFIRE", "DOWNRIGHTFIRE", "DOWNLEFTFIRE"};

static void action_bits(int action, int u[5]) {
  const char* n = kActionNames[action % 18];
  u[0] = strstr(n, "RIGHT") != NULL;
  u[1] = strstr(n, "LEFT") != NULL;
  u[2] = strstr(n, "DOWN") != NULL;
  u[3] = strstr(n, "UP") != NULL;
  u[4] = strstr(n, "FIRE") != NULL;
}

/* One env-step: frame_skip frames, or, in instruction-granular mode (the
 * paper's throughput unit, Section 6: one step = one emulated instruction),
 * step_instr instruction slots (an instruction, or a jammed CPU's idle to the
 * next line), frames ending inside the step as they come. */
static int run_frames(ovcs* s, int frame_skip) {
  int status = 0;
  s->frames_in_step = 0;
  s->frame_skip = frame_skip;
  set_gs(s);
  for (long k = 0; s->step_instr > 0 ? k < s->step_instr : s->frames_in_step < frame_skip; k++) {
    step_instruction(s);
    if (s->line >= LINE_CAP) {
      frame_end(s);
      s->cnt.watchdog++;
      status |= 1;
    }
  }
  if (s->jammed) status |= 2;
  return status;
}

int ovcs_step(ovcs* s, int action, int frame_skip, uint8_t* ram_out, uint8_t* screen_out) {
  int u[5];
  action_bits(action, u);
  set_inputs(s, u);
  int st = run_frames(s, frame_skip);
  if (ram_out) memcpy(ram_out, s->ram, 128);
  if (screen_out) memcpy(screen_out, s->last_fb, sizeof s->last_fb);
  return st;
}

void ovcs_get_counters(const ovcs* s, ovcs_counters* out) { *out = s->cnt; }

void ovcs_get_state(const ovcs* s, uint32_t* o) {
  memset(o, 0, 64 * sizeof(uint32_t));
  o[0] = s->A; o[1] = s->X; o[2] = s->Y; o[3] = s->SP; o[4] = s->P; o[5] = s->pc;
  o[6] = (uint32_t)s->cyc; o[7] = (uint32_t)(s->cyc >> 32);
  o[8] = (uint32_t)ovcs_bank(s); o[9] = s->intim; o[10] = s->interval; o[11] = s->phase; o[12] = s->underflow;
  o[13] = s->vsync; o[14] = s->vblank; o[15] = s->colup0; o[16] = s->colupf; o[17] = s->colubk;
  o[18] = s->ctrlpf; o[19] = s->pf0; o[20] = s->pf1; o[21] = s->pf2; o[22] = s->grp0;
  o[23] = s->hmp0; o[24] = (uint32_t)s->p0pos; o[25] = (uint32_t)s->hclk; o[26] = (uint32_t)s->line;
  o[27] = (uint32_t)s->hmove_line; o[28] = (uint32_t)s->jammed;
  o[29] = s->colup1; o[30] = s->nusiz[0]; o[31] = s->nusiz[1]; o[32] = s->refp[0]; o[33] = s->refp[1];
  o[34] = s->grp1; o[35] = s->grpo[0]; o[36] = s->grpo[1]; o[37] = s->enam[0]; o[38] = s->enam[1];
  o[39] = s->enabl; o[40] = s->enablo; o[41] = s->hmp1; o[42] = s->hmm[0]; o[43] = s->hmm[1];
  o[44] = s->hmbl; o[45] = s->vdelp[0]; o[46] = s->vdelp[1]; o[47] = s->vdelbl; o[48] = s->resmp[0];
  o[49] = s->resmp[1]; o[50] = (uint32_t)s->p1pos; o[51] = (uint32_t)s->mpos[0]; o[52] = (uint32_t)s->mpos[1];
  o[53] = (uint32_t)s->blpos; o[54] = s->cx;
}

void ovcs_get_ram(const ovcs* s, uint8_t* out128) { memcpy(out128, s->ram, 128); }
void ovcs_get_cart_ram(const ovcs* s, uint8_t* out128) { memcpy(out128, s->ram + 128, 128); }

int ovcs_trace(ovcs* s, int action, int n, uint32_t* out) {
  int u[5];
  action_bits(action, u);
  set_inputs(s, u);
  int i;
  for (i = 0; i < n; i++) {
    uint32_t* o = out + 10 * i;
    o[0] = s->pc; o[1] = peek_raw(s, s->pc); o[2] = s->A; o[3] = s->X; o[4] = s->Y;
    o[5] = s->SP; o[6] = s->P; o[7] = (uint32_t)s->cyc; o[8] = (uint32_t)s->line; o[9] = (uint32_t)s->hclk;
    step_instruction(s);
    if (s->line >= LINE_CAP) frame_end(s);
  }
  return i;
}

void ovcs_set_regs(ovcs* s, int A, int X, int Y, int SP, int P, int PC) {
  s->A = (uint8_t)A; s->X = (uint8_t)X; s->Y = (uint8_t)Y; s->SP = (uint8_t)SP;
  s->P = (uint8_t)(P | 0x30); s->pc = (uint16_t)PC;
}
void ovcs_set_ram(ovcs* s, const uint8_t* ram128) { memcpy(s->ram, ram128, 128); }
int ovcs_exec_one(ovcs* s) { return step_instruction(s); }
uint8_t ovcs_peek(ovcs* s, uint16_t addr) { return peek_raw(s, addr); }
int ovcs_bank(const ovcs* s) {
  /* E0: the three switchable segments' slices, 3 bits each */
  return s->e0 ? s->e0seg[0] | (s->e0seg[1] << 3) | (s->e0seg[2] << 6) : s->bank;
}

/* ------------------------------------------------------------------ */
/* soft mode                                                           */
/* ------------------------------------------------------------------ */

static int half_width(double tau) {
  int w = (int)ceil(12.0 * tau);
  return w < 1 ? 1 : w;
}

/* Weights of the relaxed read over cells lo..lo+n-1 at real address a;
 * returns the normaliser-free quantities via out arrays. */
static void read_weights(int lo, int n, double a, double tau, double* w) {
  double z = 0.0;
  for (int i = 0; i < n; i++) {
    w[i] = exp(-fabs((double)(lo + i) - a) / tau);
    z += w[i];
  }
  for (int i = 0; i < n; i++) w[i] /= z;
}

static double sgn(double x) { return x > 0 ? 1.0 : (x < 0 ? -1.0 : 0.0); }

double ovcs_relaxed_read(const double* r, int M, int a0, double a, double tau, double* d_da) {
  int lo, hi;
  window(half_width(tau), M, a0, &lo, &hi);
  int n = hi - lo + 1;
  double w[256];
  read_weights(lo, n, a, tau, w);
  double v = 0, sw = 0, swr = 0;
  for (int i = 0; i < n; i++) {
    double si = sgn((double)(lo + i) - a);
    v += w[i] * r[lo + i];
    sw += w[i] * si;
    swr += w[i] * si * r[lo + i];
  }
  if (d_da) *d_da = (swr - v * sw) / tau;
  return v;
}

double ovcs_gate_slope(double alpha, double z) {
  double g = 1.0 / (1.0 + exp(-alpha * z));
  return alpha * g * (1.0 - g);
}

ogrf* ovcs_soft_rollout(ovcs* s, const double* u, int n_steps, int frame_skip,
                        double tau, double alpha,
                        const double* grad_ram, const double* grad_screen,
                        double* ram_out, double* screen_out) {
  ogrf* g = (ogrf*)calloc(1, sizeof(ogrf));
  g->tau = tau;
  g->alpha = alpha;
  g->W = half_width(tau);
  g->n_steps = n_steps;
  g->rom_size = (int)s->rom_size;
  g->rom_copy = (uint8_t*)malloc(s->rom_size);
  memcpy(g->rom_copy, s->rom, s->rom_size);
  g->rom = g->rom_copy;
  s->g = g;
  g_new(s, NK_ZERO);
  g->rom0 = (int32_t)g->n;
  for (uint32_t i = 0; i < s->rom_size; i++) g_new(s, NK_LEAF);
  g->ram0 = (int32_t)g->n;
  for (int i = 0; i < 256; i++) g_new(s, NK_LEAF);   /* RIOT RAM, then cartridge RAM */
  g->u0 = (int32_t)g->n;
  for (int i = 0; i < 5 * n_steps; i++) g_new(s, NK_LEAF);
  for (int i = 0; i < 256; i++) g->ram0_val[i] = s->ram[i];
  g->u_val = (double*)malloc(sizeof(double) * (size_t)(5 * n_steps > 0 ? 5 * n_steps : 1));
  for (int i = 0; i < 5 * n_steps; i++) g->u_val[i] = u[i];
  /* ROM-read nodes address ROM leaves at rom0 + base + index */
  for (int i = 0; i < 256; i++) s->nRAM[i] = g->ram0 + i;
  s->nA = s->nX = s->nY = s->nV = 0;
  s->nC[0] = s->nC[1] = s->nC[2] = s->nC[3] = 0;
  s->nPos = s->nHM = 0;
  memset(s->nG, 0, sizeof s->nG);
  memset(s->nGo, 0, sizeof s->nGo);
  s->gs_all = grad_screen;
  for (int t = 0; t < n_steps; t++) {
    int bits[5];
    for (int k = 0; k < 5; k++) bits[k] = u[5 * t + k] >= 0.5;
    set_inputs(s, bits);
    s->u_leaf = g->u0 + 5 * t;
    s->soft_step = t;
    run_frames(s, frame_skip);
    for (int i = 0; i < 128; i++) {
      if (grad_ram && s->nRAM[i]) g->seed[s->nRAM[i]] += grad_ram[128 * t + i];
      if (ram_out) ram_out[128 * t + i] = s->ram[i];
    }
    if (screen_out)
      for (int i = 0; i < SCR_H * SCR_W; i++) screen_out[(size_t)SCR_H * SCR_W * t + i] = s->last_fb[i];
  }
  s->g = NULL;
  s->gs = s->gs_all = NULL;
  for (int i = 0; i < 256; i++) s->nRAM[i] = 0;
  s->nA = s->nX = s->nY = s->nV = 0;
  s->nC[0] = s->nC[1] = s->nC[2] = s->nC[3] = 0;
  s->nPos = s->nHM = 0;
  memset(s->nG, 0, sizeof s->nG);
  memset(s->nGo, 0, sizeof s->nGo);
  return g;
}

void ogrf_free(ogrf* g) {
  if (!g) return;
  free(g->nd); free(g->seed); free(g->pnode); free(g->u_val); free(g->rom_copy);
  free(g);
}

int64_t ogrf_nodes(const ogrf* g) { return g->n; }

/* node id of a read node's cell i */
static int32_t cell_node(const ogrf* g, const onode* nd, int i) {
  if (nd->kind == NK_RROM) return g->rom0 + nd->base + nd->lo + i;
  return g->pnode[nd->pool + i];
}

void ogrf_reverse(ogrf* g, double* grad_rom, double* grad_ram0, double* grad_u) {
  double* adj = (double*)malloc((size_t)g->n * sizeof(double));
  memcpy(adj, g->seed, (size_t)g->n * sizeof(double));
  double w[256];
  for (int64_t k = g->n - 1; k > 0; k--) {
    const onode* nd = &g->nd[k];
    double a = adj[k];
    if (a == 0.0) continue;
    if (nd->kind == NK_LIN) {
      for (int j = 0; j < nd->n; j++) adj[nd->in[j]] += nd->c[j] * a;
    } else if (nd->kind == NK_RROM || nd->kind == NK_RRAM) {
      read_weights(nd->lo, nd->n, (double)nd->a0, g->tau, w);
      for (int i = 0; i < nd->n; i++) {
        int32_t c = cell_node(g, nd, i);
        if (c) adj[c] += w[i] * a;
      }
    }
  }
  for (int i = 0; i < g->rom_size; i++) grad_rom[i] = adj[g->rom0 + i];
  for (int i = 0; i < 256; i++) grad_ram0[i] = adj[g->ram0 + i];
  for (int i = 0; i < 5 * g->n_steps; i++) grad_u[i] = adj[g->u0 + i];
  free(adj);
}

static void set_leaves(const ogrf* g, double* d, const double* d_rom, const double* d_ram0, const double* d_u) {
  for (int i = 0; i < g->rom_size; i++) d[g->rom0 + i] = d_rom ? d_rom[i] : 0.0;
  for (int i = 0; i < 256; i++) d[g->ram0 + i] = d_ram0 ? d_ram0[i] : 0.0;
  for (int i = 0; i < 5 * g->n_steps; i++) d[g->u0 + i] = d_u ? d_u[i] : 0.0;
}

double ogrf_tangent(ogrf* g, const double* d_rom, const double* d_ram0, const double* d_u) {
  double* d = (double*)calloc((size_t)g->n, sizeof(double));
  set_leaves(g, d, d_rom, d_ram0, d_u);
  double w[256];
  double out = 0.0;
  for (int64_t k = 1; k < g->n; k++) {
    const onode* nd = &g->nd[k];
    if (nd->kind == NK_LIN) {
      double v = 0;
      for (int j = 0; j < nd->n; j++) v += nd->c[j] * d[nd->in[j]];
      d[k] = v;
    } else if (nd->kind == NK_RROM || nd->kind == NK_RRAM) {
      read_weights(nd->lo, nd->n, (double)nd->a0, g->tau, w);
      double v = 0;
      for (int i = 0; i < nd->n; i++) {
        int32_t c = cell_node(g, nd, i);
        if (c) v += w[i] * d[c];
      }
      d[k] = v;
    }
    out += g->seed[k] * d[k];
  }
  free(d);
  return out;
}

/* Exact evaluation of L(x) - L(x_hard) of the frozen-switch relaxation.
 * With addresses frozen every node is affine in its inputs, so this equals
 * the tangent sweep up to rounding; it is kept as a separate, direct
 * evaluation (hard + soft(x) - soft(x_hard) per node) for finite differences. */
double ogrf_eval(ogrf* g, const double* d_rom, const double* d_ram0, const double* d_u) {
  double* x = (double*)calloc((size_t)g->n, sizeof(double));   /* soft value of each node */
  double* h = (double*)calloc((size_t)g->n, sizeof(double));   /* its value at the hard point */
  for (int i = 0; i < g->rom_size; i++) {
    h[g->rom0 + i] = g->rom[i];
    x[g->rom0 + i] = g->rom[i] + (d_rom ? d_rom[i] : 0.0);
  }
  for (int i = 0; i < 256; i++) {
    h[g->ram0 + i] = g->ram0_val[i];
    x[g->ram0 + i] = g->ram0_val[i] + (d_ram0 ? d_ram0[i] : 0.0);
  }
  for (int i = 0; i < 5 * g->n_steps; i++) {
    h[g->u0 + i] = g->u_val[i];
    x[g->u0 + i] = g->u_val[i] + (d_u ? d_u[i] : 0.0);
  }
  double w[256];
  double out = 0.0;
  for (int64_t k = 1; k < g->n; k++) {
    const onode* nd = &g->nd[k];
    double sx = 0.0, sh = 0.0;
    if (nd->kind == NK_LIN) {
      for (int j = 0; j < nd->n; j++) {
        sx += nd->c[j] * x[nd->in[j]];
        sh += nd->c[j] * h[nd->in[j]];
      }
    } else if (nd->kind == NK_RROM || nd->kind == NK_RRAM) {
      read_weights(nd->lo, nd->n, (double)nd->a0, g->tau, w);
      for (int i = 0; i < nd->n; i++) {
        int32_t c = cell_node(g, nd, i);
        sx += w[i] * x[c];
        sh += w[i] * h[c];
      }
    } else {
      out += g->seed[k] * (x[k] - h[k]);    /* leaf seeded directly */
      continue;
    }
    /* node value = hard + soft(x) - soft(x_hard); its hard value is
     * represented by sh (the soft value at the hard point) */
    x[k] = sx;
    h[k] = sh;
    out += g->seed[k] * (sx - sh);
  }
  free(x);
  free(h);
  return out;
}

/* ------------------------------------------------------------------------
 * Output digest (declared in vcs_oracle.h): a plain loop over the words.
 * ---------------------------------------------------------------------- */
static uint64_t digest_fin(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static uint32_t le_word(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

uint64_t ovcs_digest(const uint8_t* ram128, const uint8_t* screen) {
  uint64_t d = 0;
  uint64_t i = 0;
  for (int k = 0; k < 128; k += 4, i++) d += digest_fin((i << 32) | le_word(ram128 + k));
  if (screen)
    for (int k = 0; k < 210 * 160; k += 4, i++) d += digest_fin((i << 32) | le_word(screen + k));
  return d;
}
