/*
 * kpz_oracle.c -- CPU oracle for the 2+1-dimensional octahedron (KPZ) lattice model.
 *
 * TEST INFRASTRUCTURE ONLY. This file is a plain, slow, single-threaded
 * restatement of the method, used by the tests, by the smoke check and by the
 * CPU-baseline leg of the benchmark. The product path (the CUDA library) never
 * links, loads or calls it, and it shares no code with that path.
 *
 * What it follows (Kelling, Odor, Nagy, Schulz, Heinig, arXiv:1204.5072):
 *   - Sec. 2.1, eq. (rule): octahedron slopes sigma_x, sigma_y = +-1 per site;
 *     a local minimum is raised by 2 with probability p, a local maximum is
 *     lowered by 2 with probability q.
 *   - Sec. 2.1: flat start, periodic boundaries, height reconstruction from the
 *     slopes, squared interface width W^2 (eq. Wdef).
 *   - Sec. 3: dead-border decomposition at the device layer with a randomly moved
 *     origin; Sec. 3.1: single-hit double tiling at the work-group layer (four
 *     sets of cells, one random set per round, one attempt per active cell,
 *     repeated until each site had one chance on average).
 *   - Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 *     numbers: as easy as 1, 2, 3", SC'11), written from that paper's definition.
 *
 * Encoding (all arrays row-major, index j*L + i, i = x column, j = y row):
 *   sx[j*L+i] = 1 if sigma_x(i,j) = h(i+1,j) - h(i,j) = +1, else 0
 *   sy[j*L+i] = 1 if sigma_y(i,j) = h(i,j+1) - h(i,j) = +1, else 0
 *
 * Schedule of one sweep s (one Monte Carlo step, L*L attempts), parameters
 * (L, Bx, By, seed, sample, Tp, Tq); cells are 4x4 sites, bisected into four
 * 2x2 quadrant sets; 16 single-hit rounds per sweep:
 *   key  = (seed & 0xffffffff, seed >> 32)
 *   ctr  = (tag << 28 | index, c1, s, sample)
 *   origin:   w = philox(0<<28, 0, s, sample); ox = w0 & (L-1); oy = w1 & (L-1)
 *   tile (tx,ty), id T = ty*(L/Bx) + tx, anchored at (ox + tx*Bx, oy + ty*By) mod L
 *   set of round r: k = (philox(1<<28, T, s, sample).w0 >> 2r) & 3, qx = k&1, qy = k>>1
 *   cell (cx,cy) of the tile, word wx = cx>>5, bit b = cx&31, nwx = ceil(Bx/128):
 *     P = philox(2<<28 | ((cy*nwx+wx)<<3) | (r>>1), T, s, sample)
 *     xi = bit b of P[2*(r&1)], yi = bit b of P[2*(r&1)+1]
 *     u = 4cx + 2qx + xi, v = 4cy + 2qy + yi  (tile-local); dead if u==0 or v==0
 *     site (i,j) = ((ox + tx*Bx + u) mod L, (oy + ty*By + v) mod L)
 *   acceptance (16-bit number U, a minimum flips iff U < Tp, a maximum iff
 *   U < Tq, Tp = min(65536, floor(p*65536 + 0.5)), likewise Tq). The attempts
 *   of one round are decided together per row word rw = cy*nwx + wx (the 32
 *   cells cx = 32 wx + b, b = 0..31, of cell row cy), on the surface before
 *   the round (attempts of a round never touch each other's sites):
 *     candidates: cells whose attempted site is live and a local minimum with
 *       0 < Tp < 65536 or a local maximum with 0 < Tq < 65536 (Tp = 65536
 *       accepts and Tp = 0 rejects every minimum without a draw; same for q);
 *     top four bits of U of cell b: bit b of A[0], A[1], A[2], A[3] (most
 *       significant first), A = philox(3<<28 | rw<<4 | r, T, s, sample);
 *     a candidate is tied when its top four bits equal those of its threshold
 *       (bits 15..12); only a tied candidate draws the low twelve bits: the
 *       k-th tied candidate of the row word (k = 0, 1, ... in increasing b)
 *       takes the 16-bit half H of a deep block D, low 12 bits of H,
 *         k < 4:  D = philox(8<<28 | rw<<8 | (r & 14)<<3, T, s, sample),
 *                 half 4 (r & 1) + k,
 *         k >= 4: D = philox(8<<28 | rw<<8 | r<<3 | (1 + (k-4)/8), T, s, sample),
 *                 half (k-4) mod 8,
 *       half 2i of a block is the low and half 2i+1 the high 16 bits of word i;
 *     U = top << 12 | low (low = 0 when not tied: U < T is then decided by
 *       the top bits alone).
 * C = 2 variant (orc_sweep_c2): 2 x 2 cells, 4 rounds, no position draw.
 * Dead border at both layers (orc_sweep_db2): tags 9, 10, 11.
 * Colour-class random-sequential reference (orc_sweep_colour): tags 6 and 7.
 * Tile-set variant (orc_sweep_tilesets): same origin and tiles, no dead border,
 * the four sets (tx & 1) + 2 (ty & 1) swept in an order drawn from
 * philox(5<<28, 0, s, sample) (orc_tileset_order).
 * Random-sequential reference (no decomposition), attempt a of sweep s:
 *   w = philox(4<<28 | (a>>32), a & 0xffffffff, s, sample)
 *   site (w0 & (L-1), w1 & (L-1)), U = w2 >> 16.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 3 and Table 2).                  */
/* ------------------------------------------------------------------------- */
static const uint32_t PHILOX_M0 = 0xD2511F53u; /* round multipliers */
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u; /* Weyl key increments */
static const uint32_t PHILOX_W1 = 0xBB67AE85u;

/* One Philox S-box round on 4 words: two 32x32->64 multiplications, their
 * high halves XORed with the other two words and the round key. */
static void philox_round(uint32_t x[4], const uint32_t k[2]) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * x[0];
    uint64_t p1 = (uint64_t)PHILOX_M1 * x[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x[1] ^ k[0];
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x[3] ^ k[1];
    uint32_t y3 = lo0;
    x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3;
}

void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k[0] += PHILOX_W0; k[1] += PHILOX_W1; }
        philox_round(x, k);
    }
    out[0] = x[0]; out[1] = x[1]; out[2] = x[2]; out[3] = x[3];
}

static void philox_at(uint32_t tag_index, uint32_t c1, uint32_t s, uint32_t sample,
                      uint64_t seed, uint32_t out[4]) {
    uint32_t ctr[4] = {tag_index, c1, s, sample};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    orc_philox(ctr, key, out);
}

enum { TAG_ORIGIN = 0, TAG_SET = 1, TAG_POS = 2, TAG_ACC = 3, TAG_RSU = 4, TAG_PHASE = 5,
       TAG_CLASS = 6, TAG_CACC = 7, TAG_DEEP = 8, TAG_DBOFF = 9, TAG_DBSITE = 10, TAG_DBACC = 11 };

/* ------------------------------------------------------------------------- */
/* Model (Sec. 2.1).                                                          */
/* ------------------------------------------------------------------------- */

/* Acceptance threshold out of 2^16 for a per-attempt probability (eq. rule). */
uint32_t orc_threshold(double p) {
    if (!(p > 0.0)) return 0;           /* also maps NaN to 0 */
    if (p >= 1.0) return 65536u;
    double t = p * 65536.0 + 0.5;
    uint32_t T = (uint32_t)t;           /* floor for t >= 0 */
    return T > 65536u ? 65536u : T;
}

/* Flat start: heights h(i,j) = (i+j) & 1, so every slope is +1 where i+j is
 * even and -1 where it is odd (Sec. 2.1, "flat initial configuration"). */
void orc_init_flat(uint32_t L, uint8_t* sx, uint8_t* sy) {
    for (uint32_t j = 0; j < L; ++j)
        for (uint32_t i = 0; i < L; ++i) {
            uint8_t up = ((i + j) & 1u) == 0u;
            sx[(size_t)j * L + i] = up;
            sy[(size_t)j * L + i] = up;
        }
}

/* Eq. (rule) at site (i,j) of the periodic lattice. Reads the two x-slopes
 * entering and leaving the site and the two y-slopes; the pattern
 * (-1,+1 ; -1,+1) is a local minimum (all four neighbours are higher), the
 * pattern (+1,-1 ; +1,-1) a local maximum. A flip negates all four slopes,
 * which moves h(i,j) by +2 (minimum, if acc_min) or -2 (maximum, if acc_max).
 * Returns the height change of the site. */
static int attempt_at(uint8_t* sx, uint8_t* sy, size_t here, size_t left, size_t below,
                      int acc_min, int acc_max) {
    int a = sx[left], b = sx[here], c = sy[below], d = sy[here];
    int is_min = (a == 0 && b == 1 && c == 0 && d == 1);
    int is_max = (a == 1 && b == 0 && c == 1 && d == 0);
    if ((is_min && acc_min) || (is_max && acc_max)) {
        sx[left] ^= 1; sx[here] ^= 1; sy[below] ^= 1; sy[here] ^= 1;
        return is_min ? 2 : -2;
    }
    return 0;
}

int orc_attempt(uint32_t L, uint8_t* sx, uint8_t* sy, uint32_t i, uint32_t j,
                int acc_min, int acc_max) {
    uint32_t im = (i + L - 1) & (L - 1), jm = (j + L - 1) & (L - 1);
    size_t here = (size_t)j * L + i, left = (size_t)j * L + im, below = (size_t)jm * L + i;
    return attempt_at(sx, sy, here, left, below, acc_min, acc_max);
}

/* ------------------------------------------------------------------------- */
/* Random numbers of the decomposed schedule (header comment).                */
/* ------------------------------------------------------------------------- */

typedef struct {
    uint32_t L, Bx, By, Tp, Tq, sample;
    uint64_t seed;
    int live_border;   /* 1: no dead border (tile-set variant); 0: the paper's dead border */
} orc_params;

/* One-entry memo of the last Philox block, so that the 32 cells that share a
 * block do not recompute it; the values are exactly philox_at(...). */
typedef struct { int valid; uint32_t tag_index, c1, s, sample; uint64_t seed; uint32_t w[4]; } memo;

static const uint32_t* memo_philox(memo* m, uint32_t tag_index, uint32_t c1, uint32_t s,
                                   uint32_t sample, uint64_t seed) {
    if (!(m->valid && m->tag_index == tag_index && m->c1 == c1 && m->s == s &&
          m->sample == sample && m->seed == seed)) {
        philox_at(tag_index, c1, s, sample, seed, m->w);
        m->valid = 1; m->tag_index = tag_index; m->c1 = c1; m->s = s;
        m->sample = sample; m->seed = seed;
    }
    return m->w;
}

static uint32_t words_per_cell_row(uint32_t Bx) { return (Bx / 4 + 31) / 32; }

/* Position bits (xi, yi) of cell (cx,cy) in round r of tile T, sweep s. */
static void position_bits(const orc_params* P, memo* m, uint32_t T, uint32_t s,
                          uint32_t cx, uint32_t cy, uint32_t r, uint32_t* xi, uint32_t* yi) {
    uint32_t nwx = words_per_cell_row(P->Bx);
    uint32_t row_word = cy * nwx + (cx >> 5);
    uint32_t idx = ((uint32_t)TAG_POS << 28) | (row_word << 3) | (r >> 1);
    const uint32_t* w = memo_philox(m, idx, T, s, P->sample, P->seed);
    uint32_t b = cx & 31u;
    *xi = (w[2 * (r & 1u)] >> b) & 1u;
    *yi = (w[2 * (r & 1u) + 1] >> b) & 1u;
}

/* 16-bit half h (0..7) of a Philox block: half 2i = low, 2i+1 = high 16 bits of word i. */
static uint32_t half16(const uint32_t w[4], uint32_t h) { return (w[h >> 1] >> (16u * (h & 1u))) & 0xffffu; }

/* Acceptance decisions of one round for the 32 cells of row word rw of tile
 * T, sweep s (header comment): cand_min / cand_max mark the cells whose
 * attempted site is a live local minimum / maximum. Returns the mask of
 * accepted attempts; U (32 entries, may be NULL) receives each drawn
 * candidate's number (top << 12 | low), 0xffffffff for cells without a draw;
 * *tied (may be NULL) the mask of tied candidates. */
static uint32_t row_acceptance(const orc_params* P, uint32_t T, uint32_t s, uint32_t r, uint32_t rw,
                               uint32_t cand_min, uint32_t cand_max, uint32_t* U, uint32_t* tied) {
    uint32_t draw_min = (P->Tp > 0u && P->Tp < 65536u) ? cand_min : 0u;
    uint32_t draw_max = (P->Tq > 0u && P->Tq < 65536u) ? cand_max : 0u;
    uint32_t acc = (P->Tp == 65536u ? cand_min : 0u) | (P->Tq == 65536u ? cand_max : 0u);
    uint32_t tmask = 0;
    if (U)
        for (uint32_t b = 0; b < 32; ++b) U[b] = 0xffffffffu;
    if (draw_min | draw_max) {
        uint32_t A[4], D[4], Dx[4];
        uint32_t k = 0, have_main = 0, ext = 0xffffffffu;
        philox_at(((uint32_t)TAG_ACC << 28) | (rw << 4) | r, T, s, P->sample, P->seed, A);
        for (uint32_t b = 0; b < 32; ++b) {
            if (!(((draw_min | draw_max) >> b) & 1u)) continue;
            uint32_t thr = ((draw_min >> b) & 1u) ? P->Tp : P->Tq;
            uint32_t top = 0;
            for (uint32_t n = 0; n < 4; ++n) top |= ((A[n] >> b) & 1u) << (3 - n);
            uint32_t u = top << 12;
            if (top == (thr >> 12)) {        /* tied: draw the low twelve bits */
                uint32_t H;
                if (k < 4) {
                    if (!have_main) {
                        philox_at(((uint32_t)TAG_DEEP << 28) | (rw << 8) | ((r & 14u) << 3), T, s,
                                  P->sample, P->seed, D);
                        have_main = 1;
                    }
                    H = half16(D, 4u * (r & 1u) + k);
                } else {
                    uint32_t e = (k - 4) / 8;
                    if (e != ext) {
                        philox_at(((uint32_t)TAG_DEEP << 28) | (rw << 8) | (r << 3) | (1u + e), T, s,
                                  P->sample, P->seed, Dx);
                        ext = e;
                    }
                    H = half16(Dx, (k - 4) % 8);
                }
                u |= H & 0xfffu;
                tmask |= 1u << b;
                ++k;
            }
            if (U) U[b] = u;
            if (u < thr) acc |= 1u << b;
        }
    }
    if (tied) *tied = tmask;
    return acc;
}

/* Exported for the tests: row_acceptance with the rates given as thresholds. */
int orc_row_acceptance(uint64_t seed, uint32_t sample, uint32_t Tp, uint32_t Tq, uint32_t T, uint32_t s,
                       uint32_t r, uint32_t rw, uint32_t cand_min, uint32_t cand_max,
                       uint32_t* accept, uint32_t* tied, uint32_t* U) {
    if (Tp > 65536u || Tq > 65536u || r >= 16u || (cand_min & cand_max) || rw >= (1u << 20)) return -1;
    orc_params P = {0, 0, 0, Tp, Tq, sample, seed, 0};
    *accept = row_acceptance(&P, T, s, r, rw, cand_min, cand_max, U, tied);
    return 0;
}

/* Quadrant set (0..3) active in round r of a tile whose set word is setw0 =
 * word 0 of philox(1<<28, T, s, sample): two bits per round (Sec. 3.1: one
 * of the four sets at random each round, with replacement). */
static uint32_t set_of_round(uint32_t setw0, uint32_t r) { return (setw0 >> (2 * r)) & 3u; }

/* Device layer (Sec. 3): the origin (ox, oy) of sweep s's tile grid, a
 * uniformly random site: the low bits of words 0 and 1 of
 * philox(0<<28, 0, s, sample). */
void orc_origin(uint32_t L, uint64_t seed, uint32_t sample, uint32_t s, uint32_t* ox, uint32_t* oy) {
    uint32_t w[4];
    philox_at((uint32_t)TAG_ORIGIN << 28, 0, s, sample, seed, w);
    *ox = w[0] & (L - 1);
    *oy = w[1] & (L - 1);
}

/* Attempted site of cell (cx, cy) of tile T in round r of sweep s (Sec. 3.1):
 * the round's quadrant set k (0..3), then the tile-local site
 * (u, v) = (4 cx + 2 (k & 1) + xi, 4 cy + 2 (k >> 1) + yi). For the tests. */
int orc_attempt_site(uint32_t L, uint32_t Bx, uint32_t By, uint64_t seed, uint32_t sample, uint32_t s,
                     uint32_t T, uint32_t r, uint32_t cx, uint32_t cy, uint32_t* u, uint32_t* v, uint32_t* k) {
    if (L < 4 || Bx < 4 || By < 4 || Bx > L || By > L || r >= 16u || cx >= Bx / 4 || cy >= By / 4 ||
        T >= (L / Bx) * (L / By))
        return -1;
    orc_params P = {L, Bx, By, 0, 0, sample, seed, 0};
    memo m = {0};
    uint32_t setw[4], xi, yi;
    philox_at((uint32_t)TAG_SET << 28, T, s, sample, seed, setw);
    *k = set_of_round(setw[0], r);
    position_bits(&P, &m, T, s, cx, cy, r, &xi, &yi);
    *u = 4 * cx + 2 * (*k & 1u) + xi;
    *v = 4 * cy + 2 * (*k >> 1) + yi;
    return 0;
}

/* A fixed pseudo-random permutation used only to reorder independent work
 * (tiles, cells) in the order-independence tests; it is not part of the
 * schedule's randomness. */
static void shuffle(uint32_t* a, uint32_t n, uint64_t state) {
    for (uint32_t i = 0; i < n; ++i) a[i] = i;
    if (state == 0) return;
    for (uint32_t i = n; i > 1; --i) {
        state ^= state << 13; state ^= state >> 7; state ^= state << 17;
        uint32_t jdx = (uint32_t)(state % i);
        uint32_t t = a[i - 1]; a[i - 1] = a[jdx]; a[jdx] = t;
    }
}

/* Per-cell working storage of one tile's round (ncells = Bx*By/16 entries). */
typedef struct {
    uint32_t n;
    uint32_t* order;   /* order in which the moves of a round are made */
    uint32_t* u;       /* attempted site (tile-local), u = DEAD on the dead border */
    uint32_t* v;
    uint8_t* kind;     /* on the surface before the round: 1 minimum, 2 maximum, 0 neither */
    uint8_t* acc;      /* 1: the attempt is accepted */
} cell_work;

enum { DEAD = 0xffffffffu };

static void cell_work_free(cell_work* w) {
    free(w->order); free(w->u); free(w->v); free(w->kind); free(w->acc);
    memset(w, 0, sizeof *w);
}

static int cell_work_alloc(cell_work* w, uint32_t ncells) {
    w->n = ncells;
    w->order = (uint32_t*)malloc(sizeof(uint32_t) * ncells);
    w->u = (uint32_t*)malloc(sizeof(uint32_t) * ncells);
    w->v = (uint32_t*)malloc(sizeof(uint32_t) * ncells);
    w->kind = (uint8_t*)malloc(ncells);
    w->acc = (uint8_t*)malloc(ncells);
    if (!w->order || !w->u || !w->v || !w->kind || !w->acc) { cell_work_free(w); return -1; }
    return 0;
}

/* Slope indices of an attempt at tile-local (u, v), u, v >= 1 when windowed:
 * win: the tile's Bx x By window (stride Bx); else the periodic L x L lattice. */
static void site_index(const orc_params* P, int win, uint32_t x0, uint32_t y0, uint32_t u, uint32_t v,
                       size_t* here, size_t* left, size_t* below) {
    if (win) {
        *here = (size_t)v * P->Bx + u; *left = *here - 1; *below = *here - P->Bx;
    } else {
        uint32_t L = P->L, i = (x0 + u) & (L - 1), j = (y0 + v) & (L - 1);
        uint32_t im = (i + L - 1) & (L - 1), jm = (j + L - 1) & (L - 1);
        *here = (size_t)j * L + i; *left = (size_t)j * L + im; *below = (size_t)jm * L + i;
    }
}

/* Eq. (rule) pattern of a site: 1 local minimum, 2 local maximum, 0 neither. */
static int site_kind(const uint8_t* sx, const uint8_t* sy, size_t here, size_t left, size_t below) {
    int a = sx[left], b = sx[here], c = sy[below], d = sy[here];
    if (a == 0 && b == 1 && c == 0 && d == 1) return 1;
    if (a == 1 && b == 0 && c == 1 && d == 0) return 2;
    return 0;
}

/* The 16 single-hit rounds of tile T of sweep s (work-group layer, Sec. 3.1).
 * win == NULL: (sx, sy) is the L x L lattice. win != NULL: (sx, sy) hold only
 * this tile's Bx x By window (row-major, stride Bx, local (u, v) = global
 * ((x0 + u) mod L, (y0 + v) mod L)); an attempt at live (u, v), u, v >= 1,
 * reads and writes sigma_x(u-1, v), sigma_x(u, v), sigma_y(u, v-1),
 * sigma_y(u, v), all inside the window, so a tile evolves from its window
 * alone; *win receives the height change of global site (0, 0) if the tile
 * holds it. cw is scratch for Bx*By/16 cells. */
static void tile_rounds(const orc_params* P, uint32_t s, uint32_t T, uint32_t ox, uint32_t oy,
                        uint32_t rounds, uint64_t order, cell_work* cw, memo* mpos,
                        uint8_t* sx, uint8_t* sy, int64_t* win, int64_t* h00) {
    uint32_t L = P->L, Bx = P->Bx, By = P->By;
    uint32_t ntx = L / Bx;
    uint32_t ncx = Bx / 4, ncy = By / 4, ncells = ncx * ncy, nwx = words_per_cell_row(Bx);
    uint32_t tx = T % ntx, ty = T / ntx;
    uint32_t x0 = ox + tx * Bx, y0 = oy + ty * By;
    uint32_t setw[4];
    philox_at((uint32_t)TAG_SET << 28, T, s, P->sample, P->seed, setw);

    /* Work-group layer: 16 single-hit rounds; each picks one of the four
     * quadrant sets at random (possibly the same as before) and gives every
     * cell one attempt inside its active quadrant. */
    for (uint32_t r = 0; r < rounds; ++r) {
        uint32_t k = set_of_round(setw[0], r);
        uint32_t qx = k & 1u, qy = k >> 1;

        /* 1. Each cell's attempted site and its pattern before the round. */
        for (uint32_t cell = 0; cell < ncells; ++cell) {
            uint32_t cx = cell % ncx, cy = cell / ncx, xi, yi;
            position_bits(P, mpos, T, s, cx, cy, r, &xi, &yi);
            uint32_t u = 4 * cx + 2 * qx + xi;
            uint32_t v = 4 * cy + 2 * qy + yi;
            cw->acc[cell] = 0;
            if (!P->live_border && (u == 0 || v == 0)) {   /* dead border of the tile */
                cw->u[cell] = DEAD; cw->v[cell] = DEAD; cw->kind[cell] = 0;
                continue;
            }
            size_t here, left, below;
            site_index(P, win != NULL, x0, y0, u, v, &here, &left, &below);
            cw->u[cell] = u; cw->v[cell] = v;
            cw->kind[cell] = (uint8_t)site_kind(sx, sy, here, left, below);
        }

        /* 2. Acceptance, one row word of 32 cells at a time. */
        for (uint32_t cy = 0; cy < ncy; ++cy)
            for (uint32_t wx = 0; wx < nwx; ++wx) {
                uint32_t cmin = 0, cmax = 0;
                for (uint32_t b = 0; b < 32 && 32 * wx + b < ncx; ++b) {
                    uint32_t kd = cw->kind[cy * ncx + 32 * wx + b];
                    if (kd == 1) cmin |= 1u << b;
                    if (kd == 2) cmax |= 1u << b;
                }
                uint32_t acc = row_acceptance(P, T, s, r, cy * nwx + wx, cmin, cmax, NULL, NULL);
                for (uint32_t b = 0; b < 32 && 32 * wx + b < ncx; ++b)
                    cw->acc[cy * ncx + 32 * wx + b] = (uint8_t)((acc >> b) & 1u);
            }

        /* 3. The accepted moves (their sites are never neighbours, so any order). */
        shuffle(cw->order, ncells, order >= 2 ? order * 0x9E3779B97F4A7C15ull + T + 1 : 0);
        if (order == 1)
            for (uint32_t c = 0; c < ncells; ++c) cw->order[c] = ncells - 1 - c;
        for (uint32_t c = 0; c < ncells; ++c) {
            uint32_t cell = cw->order[c];
            if (cw->u[cell] == DEAD || !cw->acc[cell]) continue;
            size_t here, left, below;
            site_index(P, win != NULL, x0, y0, cw->u[cell], cw->v[cell], &here, &left, &below);
            int dh = attempt_at(sx, sy, here, left, below, 1, 1);
            uint32_t i = (x0 + cw->u[cell]) & (L - 1), j = (y0 + cw->v[cell]) & (L - 1);
            if (dh != 0 && i == 0 && j == 0) {
                if (h00) *h00 += dh;
                if (win) *win += dh;
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* One sweep of the decomposed dynamics (Sec. 3 and 3.1).                      */
/* order: 0 = tiles and cells in natural order, 1 = both reversed, >= 2 = both */
/* shuffled with a permutation seeded by `order` (result must not change).    */
/* rounds: number of single-hit rounds to perform (16 = the full sweep; fewer */
/* only for tests that look inside a sweep). Returns 0, or -1 on bad input.   */
/* ------------------------------------------------------------------------- */
int orc_sweep(uint32_t L, uint32_t Bx, uint32_t By, uint32_t Tp, uint32_t Tq,
              uint64_t seed, uint32_t sample, uint32_t s,
              uint8_t* sx, uint8_t* sy, int64_t* h00, uint64_t order, uint32_t rounds) {
    if (rounds > 16) return -1;
    if (L < 4 || (L & (L - 1)) || Bx < 4 || By < 4 || (Bx & (Bx - 1)) || (By & (By - 1)) ||
        Bx > L || By > L || Tp > 65536u || Tq > 65536u)
        return -1;
    orc_params P = {L, Bx, By, Tp, Tq, sample, seed, 0};

    /* Device layer: the origin of the tile grid moves to a random site each sweep. */
    uint32_t ox, oy;
    orc_origin(L, seed, sample, s, &ox, &oy);

    uint32_t ntx = L / Bx, nty = L / By, ntiles = ntx * nty;
    uint32_t* tile_order = (uint32_t*)malloc(sizeof(uint32_t) * ntiles);
    cell_work cw;
    if (!tile_order || cell_work_alloc(&cw, (Bx / 4) * (By / 4))) { free(tile_order); return -1; }
    shuffle(tile_order, ntiles, order >= 2 ? order : 0);
    if (order == 1)
        for (uint32_t n = 0; n < ntiles; ++n) tile_order[n] = ntiles - 1 - n;

    memo mpos = {0};
    for (uint32_t n = 0; n < ntiles; ++n) {
        uint32_t T = tile_order[n];
        tile_rounds(&P, s, T, ox, oy, rounds, order, &cw, &mpos, sx, sy, NULL, h00);
    }
    free(tile_order);
    cell_work_free(&cw);
    return 0;
}

/* The C = 2 limit of the work-group layer (cells of 2 x 2 sites, their four
 * 1 x 1 quadrants as the sets, 4 single-hit rounds per sweep): in round r of
 * tile T the set k = (philox(1<<28, T, s, sample).w0 >> 2r) & 3 is active, and
 * every 2 x 2 cell (cx, cy) attempts its site u = 2cx + (k & 1),
 * v = 2cy + (k >> 1) (no position draw; dead if u == 0 or v == 0). The
 * acceptance number of that attempt (16 bits, level 0 most significant):
 *   with 4 x 4 storage cell (c4x, c4y) = (u >> 2, v >> 2), site index inside
 *   it a = 2 ((v >> 1) & 1) + ((u >> 1) & 1), word wx = c4x >> 5,
 *   nwx = ceil(Bx/128): A_m = philox(3<<28 | ((c4y*nwx+wx) << 6) | (r << 4)
 *   | (a << 2) | m, T, s, sample), level n from bit (c4x & 31) of
 *   A_{n>>2}[n&3]. Returns 0, or -1 on bad input. */
/* The first `rounds` (<= 4) rounds of that sweep; orc_sweep_c2 runs all four. */
int orc_sweep_c2_rounds(uint32_t L, uint32_t Bx, uint32_t By, uint32_t Tp, uint32_t Tq,
                        uint64_t seed, uint32_t sample, uint32_t s,
                        uint8_t* sx, uint8_t* sy, int64_t* h00, uint64_t order, uint32_t rounds) {
    if (L < 4 || (L & (L - 1)) || Bx < 4 || By < 4 || (Bx & (Bx - 1)) || (By & (By - 1)) ||
        Bx > L || By > L || Tp > 65536u || Tq > 65536u || rounds > 4)
        return -1;
    uint32_t ox, oy;
    orc_origin(L, seed, sample, s, &ox, &oy);
    uint32_t ntx = L / Bx, nty = L / By, ntiles = ntx * nty;
    uint32_t ncx = Bx / 2, ncy = By / 2, ncells = ncx * ncy, nwx = words_per_cell_row(Bx);
    uint32_t* tile_order = (uint32_t*)malloc(sizeof(uint32_t) * ntiles);
    uint32_t* cell_order = (uint32_t*)malloc(sizeof(uint32_t) * ncells);
    if (!tile_order || !cell_order) { free(tile_order); free(cell_order); return -1; }
    shuffle(tile_order, ntiles, order >= 2 ? order : 0);
    if (order == 1)
        for (uint32_t n = 0; n < ntiles; ++n) tile_order[n] = ntiles - 1 - n;
    memo macc[4] = {{0}};
    for (uint32_t n = 0; n < ntiles; ++n) {
        uint32_t T = tile_order[n], tx = T % ntx, ty = T / ntx;
        uint32_t x0 = ox + tx * Bx, y0 = oy + ty * By;
        uint32_t setw[4];
        philox_at((uint32_t)TAG_SET << 28, T, s, sample, seed, setw);
        for (uint32_t r = 0; r < rounds; ++r) {
            uint32_t k = (setw[0] >> (2 * r)) & 3u;
            shuffle(cell_order, ncells, order >= 2 ? order * 0x9E3779B97F4A7C15ull + T + 1 : 0);
            if (order == 1)
                for (uint32_t c = 0; c < ncells; ++c) cell_order[c] = ncells - 1 - c;
            for (uint32_t c = 0; c < ncells; ++c) {
                uint32_t cell = cell_order[c];
                uint32_t u = 2 * (cell % ncx) + (k & 1u), v = 2 * (cell / ncx) + (k >> 1);
                if (u == 0 || v == 0) continue;          /* dead border of the tile */
                uint32_t c4x = u >> 2, c4y = v >> 2, a = 2 * ((v >> 1) & 1u) + ((u >> 1) & 1u);
                uint32_t row_word = c4y * nwx + (c4x >> 5), b = c4x & 31u, U = 0;
                for (uint32_t lev = 0; lev < 16; ++lev) {
                    uint32_t mi = lev >> 2;
                    uint32_t idx = ((uint32_t)TAG_ACC << 28) | (row_word << 6) | (r << 4) | (a << 2) | mi;
                    const uint32_t* aw = memo_philox(&macc[mi], idx, T, s, sample, seed);
                    U |= ((aw[lev & 3u] >> b) & 1u) << (15 - lev);
                }
                uint32_t i = (x0 + u) & (L - 1), j = (y0 + v) & (L - 1);
                int dh = orc_attempt(L, sx, sy, i, j, U < Tp, U < Tq);
                if (dh != 0 && i == 0 && j == 0 && h00) *h00 += dh;
            }
        }
    }
    free(tile_order);
    free(cell_order);
    return 0;
}

int orc_sweep_c2(uint32_t L, uint32_t Bx, uint32_t By, uint32_t Tp, uint32_t Tq,
                 uint64_t seed, uint32_t sample, uint32_t s,
                 uint8_t* sx, uint8_t* sy, int64_t* h00, uint64_t order) {
    return orc_sweep_c2_rounds(L, Bx, By, Tp, Tq, seed, sample, s, sx, sy, h00, order, 4);
}

/* Tile T of sweep s computed on its own Bx x By window (tiles of one sweep do
 * not interact, Sec. 3): on entry (sx_win, sy_win) hold the window's slopes
 * when sweep s starts (row-major, stride Bx, local (u, v) = global
 * ((x0+u) mod L, (y0+v) mod L) with (x0, y0) the tile's anchor, which
 * *anchor_x / *anchor_y receive); on return the slopes after the sweep;
 * *dh00 the height change of site (0, 0) (0 unless the tile holds it).
 * With window == 0 the anchor is returned and nothing else is touched.
 * Returns 0, or -1 on bad input. */
int orc_window_tile_sweep(uint32_t L, uint32_t Bx, uint32_t By, uint32_t Tp, uint32_t Tq,
                          uint64_t seed, uint32_t sample, uint32_t s, uint32_t T, int window,
                          uint8_t* sx_win, uint8_t* sy_win, uint32_t* anchor_x, uint32_t* anchor_y,
                          int64_t* dh00) {
    if (L < 4 || (L & (L - 1)) || Bx < 4 || By < 4 || (Bx & (Bx - 1)) || (By & (By - 1)) ||
        Bx > L || By > L || Tp > 65536u || Tq > 65536u || T >= (L / Bx) * (L / By))
        return -1;
    orc_params P = {L, Bx, By, Tp, Tq, sample, seed, 0};
    uint32_t ox, oy;
    orc_origin(L, seed, sample, s, &ox, &oy);
    uint32_t ntx = L / Bx, tx = T % ntx, ty = T / ntx;
    *anchor_x = (ox + tx * Bx) & (L - 1);
    *anchor_y = (oy + ty * By) & (L - 1);
    if (!window) return 0;
    cell_work cw;
    if (cell_work_alloc(&cw, (Bx / 4) * (By / 4))) return -1;
    memo mpos = {0};
    int64_t d = 0;
    tile_rounds(&P, s, T, ox, oy, 16, 0, &cw, &mpos, sx_win, sy_win, &d, NULL);
    cell_work_free(&cw);
    *dh00 = d;
    return 0;
}

/* Tile T of sweep s started from the flat configuration (Sec. 2.1): the
 * window of orc_window_tile_sweep filled with the flat start h = (i+j) & 1
 * (exact for a lattice that is flat when sweep s starts). */
int orc_flat_tile_sweep(uint32_t L, uint32_t Bx, uint32_t By, uint32_t Tp, uint32_t Tq,
                        uint64_t seed, uint32_t sample, uint32_t s, uint32_t T,
                        uint8_t* sx_win, uint8_t* sy_win, uint32_t* anchor_x, uint32_t* anchor_y,
                        int64_t* dh00) {
    uint32_t x0, y0;
    if (orc_window_tile_sweep(L, Bx, By, Tp, Tq, seed, sample, s, T, 0, sx_win, sy_win, &x0, &y0, dh00))
        return -1;
    for (uint32_t v = 0; v < By; ++v)
        for (uint32_t u = 0; u < Bx; ++u) {
            uint8_t up = (((x0 + u) + (y0 + v)) & 1u) == 0u;   /* flat start */
            sx_win[(size_t)v * Bx + u] = up;
            sy_win[(size_t)v * Bx + u] = up;
        }
    return orc_window_tile_sweep(L, Bx, By, Tp, Tq, seed, sample, s, T, 1, sx_win, sy_win,
                                 anchor_x, anchor_y, dh00);
}

/* Dead border at both layers (the paper's earlier KPZ scheme, Sec. 3.1: the
 * dead-border rule of Sec. 3 applied at the work-group layer as well as at
 * the device layer). Device layer as in orc_sweep: random origin, Bx x By
 * tiles, each with a dead low row and column. Work-group layer: 16 rounds per
 * sweep; in round r the tile is cut into 4 x 4 blocks anchored at the
 * tile-local offset (dx, dy), wrapping inside the tile; a block's low row and
 * column are its dead border, and each block makes one attempt at a
 * uniformly random site of its 3 x 3 live interior. A site is in a block's
 * interior with probability 9/16 over the offset and then chosen with
 * probability 1/9, so it has on average one attempt per sweep; attempts of
 * one round never touch each other's slopes (blocks are separated by their
 * dead borders, tiles by theirs). Random numbers of tile T, sweep s:
 *   offsets: S = philox(9<<28, T, s, sample), round r:
 *            dx = (S[r>>3] >> 4(r&7)) & 3, dy = (S[r>>3] >> (4(r&7) + 2)) & 3;
 *   block k = ky (Bx/4) + kx in round r:
 *            w = philox(10<<28 | r<<20 | k>>2, T, s, sample)[k&3],
 *            n = floor(9 w / 2^32), (i, j) = (1 + n mod 3, 1 + n div 3),
 *            site u = (dx + 4 kx + i) mod Bx, v = (dy + 4 ky + j) mod By,
 *            no attempt if u = 0 or v = 0 (the tile's dead border);
 *   acceptance: U = philox(11<<28 | r<<20 | k>>2, T, s, sample)[k&3] >> 16,
 *            a minimum flips iff U < Tp, a maximum iff U < Tq.
 * (n is uniform over 0..8 up to 9 / 2^32.) */
static void db2_site(uint32_t Bx, uint32_t By, uint64_t seed, uint32_t sample, uint32_t s, uint32_t T,
                     uint32_t r, uint32_t kx, uint32_t ky, uint32_t* u, uint32_t* v, uint32_t* U) {
    uint32_t S[4], w[4], a[4];
    philox_at((uint32_t)TAG_DBOFF << 28, T, s, sample, seed, S);
    uint32_t dx = (S[r >> 3] >> (4 * (r & 7))) & 3u, dy = (S[r >> 3] >> (4 * (r & 7) + 2)) & 3u;
    uint32_t k = ky * (Bx / 4) + kx;
    philox_at(((uint32_t)TAG_DBSITE << 28) | (r << 20) | (k >> 2), T, s, sample, seed, w);
    philox_at(((uint32_t)TAG_DBACC << 28) | (r << 20) | (k >> 2), T, s, sample, seed, a);
    uint32_t n = (uint32_t)(((uint64_t)w[k & 3] * 9u) >> 32);
    *u = (dx + 4 * kx + 1 + n % 3) & (Bx - 1);
    *v = (dy + 4 * ky + 1 + n / 3) & (By - 1);
    *U = a[k & 3] >> 16;
}

/* For the tests: the tile-local site (u, v) block (kx, ky) of tile T attempts
 * in round r of sweep s, and its acceptance number. Returns 0, or -1. */
int orc_db2_site(uint32_t L, uint32_t Bx, uint32_t By, uint64_t seed, uint32_t sample, uint32_t s,
                 uint32_t T, uint32_t r, uint32_t kx, uint32_t ky, uint32_t* u, uint32_t* v, uint32_t* U) {
    if (L < 4 || Bx < 4 || By < 4 || Bx > L || By > L || (Bx & (Bx - 1)) || (By & (By - 1)) || r >= 16u ||
        kx >= Bx / 4 || ky >= By / 4 || T >= (L / Bx) * (L / By) || (Bx / 4) * (By / 4) > (1u << 22))
        return -1;
    db2_site(Bx, By, seed, sample, s, T, r, kx, ky, u, v, U);
    return 0;
}

int orc_sweep_db2(uint32_t L, uint32_t Bx, uint32_t By, uint32_t Tp, uint32_t Tq,
                  uint64_t seed, uint32_t sample, uint32_t s,
                  uint8_t* sx, uint8_t* sy, int64_t* h00, uint64_t order) {
    if (L < 4 || (L & (L - 1)) || Bx < 4 || By < 4 || (Bx & (Bx - 1)) || (By & (By - 1)) ||
        Bx > L || By > L || Tp > 65536u || Tq > 65536u || (Bx / 4) * (By / 4) > (1u << 22))
        return -1;
    uint32_t ox, oy;
    orc_origin(L, seed, sample, s, &ox, &oy);
    uint32_t ntx = L / Bx, nty = L / By, ntiles = ntx * nty, nbx = Bx / 4, nblk = nbx * (By / 4);
    uint32_t* tile_order = (uint32_t*)malloc(sizeof(uint32_t) * ntiles);
    uint32_t* blk_order = (uint32_t*)malloc(sizeof(uint32_t) * nblk);
    if (!tile_order || !blk_order) { free(tile_order); free(blk_order); return -1; }
    shuffle(tile_order, ntiles, order >= 2 ? order : 0);
    if (order == 1)
        for (uint32_t n = 0; n < ntiles; ++n) tile_order[n] = ntiles - 1 - n;
    for (uint32_t n = 0; n < ntiles; ++n) {
        uint32_t T = tile_order[n], tx = T % ntx, ty = T / ntx;
        uint32_t x0 = ox + tx * Bx, y0 = oy + ty * By;
        for (uint32_t r = 0; r < 16; ++r) {
            shuffle(blk_order, nblk, order >= 2 ? order * 0x9E3779B97F4A7C15ull + T + 1 : 0);
            if (order == 1)
                for (uint32_t c = 0; c < nblk; ++c) blk_order[c] = nblk - 1 - c;
            for (uint32_t c = 0; c < nblk; ++c) {
                uint32_t k = blk_order[c], u, v, U;
                db2_site(Bx, By, seed, sample, s, T, r, k % nbx, k / nbx, &u, &v, &U);
                if (u == 0 || v == 0) continue;   /* the tile's dead border */
                uint32_t i = (x0 + u) & (L - 1), j = (y0 + v) & (L - 1);
                int dh = orc_attempt(L, sx, sy, i, j, U < Tp, U < Tq);
                if (dh != 0 && i == 0 && j == 0 && h00) *h00 += dh;
            }
        }
    }
    free(tile_order);
    free(blk_order);
    return 0;
}

/* The same sweep with the tiles spread over nthreads OpenMP threads (natural
 * order inside each tile). Tiles of one sweep read and write disjoint slopes
 * (dead border, Sec. 3), so the result equals orc_sweep's bit for bit; used
 * to time the oracle on all host cores. Returns 0, or -1 on bad input. */
int orc_sweep_threads(uint32_t L, uint32_t Bx, uint32_t By, uint32_t Tp, uint32_t Tq,
                      uint64_t seed, uint32_t sample, uint32_t s,
                      uint8_t* sx, uint8_t* sy, int64_t* h00, int nthreads) {
    if (L < 4 || (L & (L - 1)) || Bx < 4 || By < 4 || (Bx & (Bx - 1)) || (By & (By - 1)) ||
        Bx > L || By > L || Tp > 65536u || Tq > 65536u || nthreads < 1)
        return -1;
    orc_params P = {L, Bx, By, Tp, Tq, sample, seed, 0};
    uint32_t ox, oy;
    orc_origin(L, seed, sample, s, &ox, &oy);
    int64_t ntiles = (int64_t)(L / Bx) * (L / By);
    uint32_t ncells = (Bx / 4) * (By / 4);
    int64_t dh = 0;
    int bad = 0;
#pragma omp parallel num_threads(nthreads) reduction(+ : dh) reduction(| : bad)
    {
        cell_work cw;
        memo mpos = {0};
        int ok = cell_work_alloc(&cw, ncells) == 0;
        if (!ok) bad = 1;
#pragma omp for schedule(dynamic, 16)
        for (int64_t T = 0; T < ntiles; ++T)
            if (ok)
                tile_rounds(&P, s, (uint32_t)T, ox, oy, 16, 0, &cw, &mpos, sx, sy, NULL, &dh);
        if (ok) cell_work_free(&cw);
    }
    if (bad) return -1;
    if (h00) *h00 += dh;
    return 0;
}

/* Variant of the device layer (KMC-style double tiling, Sec. 3.2 describes it
 * for the KMC model): the same random origin and Bx x By tiles, grouped into
 * four sets by (tx mod 2, ty mod 2); the sets are swept one after the other in
 * an order drawn per sweep, and there is no dead border: every site of a tile
 * is live, and the neighbours it reads across the tile edge belong to tiles of
 * other sets, which are idle meanwhile. Set order of sweep s:
 *   w = philox(5<<28, 0, s, sample); perm = (0, 1, 2, 3);
 *   for i = 3, 2, 1: swap perm[i] and perm[w[3-i] mod (i+1)]  (Fisher-Yates)
 * and phase i sweeps set perm[i] = (tx & 1) + 2 (ty & 1). The work-group layer
 * (16 single-hit rounds per tile) and its random streams are unchanged.
 * order as in orc_sweep (tile and cell order inside a phase; no effect).
 * Needs an even number of tiles per row and column. Returns 0, or -1. */
int orc_tileset_order(uint32_t s, uint32_t sample, uint64_t seed, uint32_t perm[4]) {
    uint32_t w[4];
    philox_at((uint32_t)TAG_PHASE << 28, 0, s, sample, seed, w);
    for (uint32_t i = 0; i < 4; ++i) perm[i] = i;
    for (uint32_t i = 3; i >= 1; --i) {
        uint32_t j = w[3 - i] % (i + 1), t = perm[i];
        perm[i] = perm[j]; perm[j] = t;
    }
    return 0;
}

int orc_sweep_tilesets(uint32_t L, uint32_t Bx, uint32_t By, uint32_t Tp, uint32_t Tq,
                       uint64_t seed, uint32_t sample, uint32_t s,
                       uint8_t* sx, uint8_t* sy, int64_t* h00, uint64_t order) {
    if (L < 4 || (L & (L - 1)) || Bx < 4 || By < 4 || (Bx & (Bx - 1)) || (By & (By - 1)) ||
        2 * Bx > L || 2 * By > L || Tp > 65536u || Tq > 65536u)
        return -1;
    orc_params P = {L, Bx, By, Tp, Tq, sample, seed, 1};
    uint32_t ox, oy;
    orc_origin(L, seed, sample, s, &ox, &oy);
    uint32_t perm[4];
    orc_tileset_order(s, sample, seed, perm);
    uint32_t ntx = L / Bx, nty = L / By, ntiles = ntx * nty;
    uint32_t* tile_order = (uint32_t*)malloc(sizeof(uint32_t) * ntiles);
    cell_work cw;
    if (!tile_order || cell_work_alloc(&cw, (Bx / 4) * (By / 4))) { free(tile_order); return -1; }
    shuffle(tile_order, ntiles, order >= 2 ? order : 0);
    if (order == 1)
        for (uint32_t n = 0; n < ntiles; ++n) tile_order[n] = ntiles - 1 - n;
    memo mpos = {0};
    for (uint32_t phase = 0; phase < 4; ++phase)
        for (uint32_t n = 0; n < ntiles; ++n) {
            uint32_t T = tile_order[n], tx = T % ntx, ty = T / ntx;
            if ((tx & 1u) + 2u * (ty & 1u) != perm[phase]) continue;
            tile_rounds(&P, s, T, ox, oy, 16, order, &cw, &mpos, sx, sy, NULL, h00);
        }
    free(tile_order);
    cell_work_free(&cw);
    return 0;
}

/* Random-sequential updates by colour classes (a parallel reference for the
 * random-sequential dynamics, no decomposition): sweep s is K = 4 * 2^m
 * sub-steps i; sub-step i draws one of the four period-2 sublattices,
 *   c = philox(6<<28 | i, 0xffffffff, s, sample).w0 & 3, sites x = c & 1,
 *   y = c >> 1 (mod 2),
 * and attempts each of its sites with probability 2^-m. Sites of one class
 * are never neighbours, so the attempts of a sub-step commute, and as m grows
 * the dynamics approaches random-sequential updates (each site one attempt
 * per sweep on average). Bit layout of the draws: 128 x 128 tiles anchored at
 * (0, 0), tile T = ty * (L/128) + tx; cell row cy = v >> 2, storage cell
 * c4 = u >> 2 (u, v tile-local), class site a = 2 ((v >> 1) & 1) + ((u >> 1) & 1):
 *   selected iff bit c4 of S[0] & ... & S[m-1], S = philox(6<<28 | i << 9 |
 *   cy << 2 | a, T, s, sample) (m <= 4);
 *   acceptance U (16 bits, level 0 most significant), level n from bit c4 of
 *   A_{n>>2}[n&3], A_k = philox(7<<28 | i << 9 | cy << 4 | a << 2 | k, T, s, sample).
 * Needs L >= 128. Returns 0, or -1 on bad input. */
/* The first `nsub` sub-steps of that sweep (nsub >= 4 * 2^m: all of them). */
int orc_sweep_colour_steps(uint32_t L, uint32_t Tp, uint32_t Tq, uint32_t m, uint64_t seed, uint32_t sample,
                           uint32_t s, uint8_t* sx, uint8_t* sy, int64_t* h00, uint32_t nsub) {
    if (L < 128 || (L & (L - 1)) || m > 4 || Tp > 65536u || Tq > 65536u) return -1;
    const uint32_t B = 128, ntx = L / B, K = nsub < (4u << m) ? nsub : (4u << m);
    memo msel = {0}, macc[4] = {{0}};
    for (uint32_t i = 0; i < K; ++i) {
        uint32_t w[4];
        philox_at(((uint32_t)TAG_CLASS << 28) | i, 0xffffffffu, s, sample, seed, w);
        uint32_t c = w[0] & 3u, cx = c & 1u, cyc = c >> 1;
        for (uint32_t j = cyc; j < L; j += 2)
            for (uint32_t x = cx; x < L; x += 2) {
                uint32_t T = (j / B) * ntx + x / B, u = x % B, v = j % B;
                uint32_t c4 = u >> 2, cy = v >> 2, a = 2 * ((v >> 1) & 1u) + ((u >> 1) & 1u);
                uint32_t sel = 1;
                if (m) {
                    const uint32_t* S = memo_philox(&msel, ((uint32_t)TAG_CLASS << 28) | (i << 9) | (cy << 2) | a,
                                                    T, s, sample, seed);
                    uint32_t word = ~0u;
                    for (uint32_t k = 0; k < m; ++k) word &= S[k];
                    sel = (word >> c4) & 1u;
                }
                if (!sel) continue;
                uint32_t U = 0;
                for (uint32_t lev = 0; lev < 16; ++lev) {
                    uint32_t mi = lev >> 2;
                    const uint32_t* A = memo_philox(&macc[mi], ((uint32_t)TAG_CACC << 28) | (i << 9) | (cy << 4) |
                                                    (a << 2) | mi, T, s, sample, seed);
                    U |= ((A[lev & 3u] >> c4) & 1u) << (15 - lev);
                }
                int dh = orc_attempt(L, sx, sy, x, j, U < Tp, U < Tq);
                if (dh != 0 && x == 0 && j == 0 && h00) *h00 += dh;
            }
    }
    return 0;
}

int orc_sweep_colour(uint32_t L, uint32_t Tp, uint32_t Tq, uint32_t m, uint64_t seed, uint32_t sample,
                     uint32_t s, uint8_t* sx, uint8_t* sy, int64_t* h00) {
    return orc_sweep_colour_steps(L, Tp, Tq, m, seed, sample, s, sx, sy, h00, 4u << m);
}

/* n sweeps s = t0 .. t0+n-1 in natural order. */
int orc_run(uint32_t L, uint32_t Bx, uint32_t By, uint32_t Tp, uint32_t Tq,
            uint64_t seed, uint32_t sample, uint32_t t0, uint32_t n,
            uint8_t* sx, uint8_t* sy, int64_t* h00) {
    for (uint32_t k = 0; k < n; ++k) {
        int rc = orc_sweep(L, Bx, By, Tp, Tq, seed, sample, t0 + k, sx, sy, h00, 0, 16);
        if (rc) return rc;
    }
    return 0;
}

/* Random-sequential update: L*L attempts at uniformly random sites per sweep,
 * no decomposition (the dynamics the decomposition approximates). */
int orc_rsu_run(uint32_t L, uint32_t Tp, uint32_t Tq, uint64_t seed, uint32_t sample,
                uint32_t t0, uint32_t n, uint8_t* sx, uint8_t* sy, int64_t* h00) {
    if (L < 4 || (L & (L - 1)) || Tp > 65536u || Tq > 65536u) return -1;
    uint64_t N = (uint64_t)L * L;
    for (uint32_t k = 0; k < n; ++k) {
        uint32_t s = t0 + k;
        for (uint64_t a = 0; a < N; ++a) {
            uint32_t w[4];
            philox_at(((uint32_t)TAG_RSU << 28) | (uint32_t)(a >> 32), (uint32_t)a, s, sample, seed, w);
            uint32_t i = w[0] & (L - 1), j = w[1] & (L - 1), U = w[2] >> 16;
            int dh = orc_attempt(L, sx, sy, i, j, U < Tp, U < Tq);
            if (dh != 0 && i == 0 && j == 0 && h00) *h00 += dh;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Heights and width (Sec. 2.1).                                               */
/* ------------------------------------------------------------------------- */

/* Height reconstruction in the gauge h(0,0) = 0: walk along row 0 to column i,
 * then up column i to row j:  h(i,j) = sum_{l<i} sigma_x(l,0) + sum_{k<j} sigma_y(i,k). */
void orc_heights(uint32_t L, const uint8_t* sx, const uint8_t* sy, int64_t* h) {
    int64_t base = 0;
    for (uint32_t i = 0; i < L; ++i) {
        int64_t hh = base;
        for (uint32_t j = 0; j < L; ++j) {
            h[(size_t)j * L + i] = hh;
            hh += sy[(size_t)j * L + i] ? 1 : -1;
        }
        base += sx[i] ? 1 : -1;   /* sigma_x(i, 0) */
    }
}

/* Exact sums S1 = sum h, S2 = sum h^2 (S2 as two 64-bit halves). */
void orc_sums(uint32_t L, const int64_t* h, int64_t* S1, uint64_t* S2_lo, uint64_t* S2_hi) {
    int64_t s1 = 0;
    unsigned __int128 s2 = 0;
    uint64_t N = (uint64_t)L * L;
    for (uint64_t n = 0; n < N; ++n) {
        s1 += h[n];
        s2 += (unsigned __int128)((__int128)h[n] * h[n]);
    }
    *S1 = s1;
    *S2_lo = (uint64_t)s2;
    *S2_hi = (uint64_t)(s2 >> 64);
}

/* Eq. (Wdef): W^2 = (1/N) sum h^2 - ((1/N) sum h)^2 with N = L^2 sites,
 * evaluated as (N*S2 - S1^2) / N^2 with the numerator exact in 128 bits. */
double orc_w2(uint64_t N, int64_t S1, uint64_t S2_lo, uint64_t S2_hi) {
    unsigned __int128 S2 = ((unsigned __int128)S2_hi << 64) | S2_lo;
    unsigned __int128 num = (unsigned __int128)N * S2 - (unsigned __int128)((__int128)S1 * S1);
    return (double)num / ((double)N * (double)N);
}

/* Canonical packed exchange format: row j occupies L/16 words; site i sits in
 * word j*(L/16) + i/16 at bits 2(i%16) (sigma_x) and 2(i%16)+1 (sigma_y). */
void orc_pack(uint32_t L, const uint8_t* sx, const uint8_t* sy, uint32_t* words) {
    size_t W = (size_t)L * L / 16;
    memset(words, 0, W * sizeof(uint32_t));
    for (uint32_t j = 0; j < L; ++j)
        for (uint32_t i = 0; i < L; ++i) {
            size_t n = (size_t)j * L + i, wi = (size_t)j * (L / 16) + i / 16;
            words[wi] |= ((uint32_t)sx[n] << (2 * (i % 16))) | ((uint32_t)sy[n] << (2 * (i % 16) + 1));
        }
}

void orc_unpack(uint32_t L, const uint32_t* words, uint8_t* sx, uint8_t* sy) {
    for (uint32_t j = 0; j < L; ++j)
        for (uint32_t i = 0; i < L; ++i) {
            size_t n = (size_t)j * L + i, wi = (size_t)j * (L / 16) + i / 16;
            sx[n] = (words[wi] >> (2 * (i % 16))) & 1u;
            sy[n] = (words[wi] >> (2 * (i % 16) + 1)) & 1u;
        }
}
