/*
 * Oracle for the synchronous Nagel-Schreckenberg (NaSch) step on a ring road.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * CPU statement of what the GPU library computes.  It is built and called by
 * the test-suite, by the package's smoke check and by the benchmark's CPU
 * baseline leg; the library itself never links, loads or calls it, and it
 * shares no source, header or table with the library.
 *
 * What it follows (van Zon & Ponce, "Parallelizing a 1-Dim
 * Nagel-Schreckenberg Traffic Model", EduHPC-23):
 *   - Handout, "The Nagel-Schreckenberg traffic model": the four rules
 *     (accelerate, brake to d-1, random slowdown with probability p, move)
 *     and their summary equation; the rule-3 formula is garbled there as
 *     "(0, v-1)" and is read as max(0, v-1), as the rule-3 sentence says.
 *   - Same section, the Bernoulli draw: r uniform on [0,1), slow down iff
 *     r < p.  With r = u * 2^-32 for a 32-bit integer u this is exactly
 *     u < ceil(p * 2^32)  (see oracle_slow_threshold).
 *   - Handout, "Starter Code": cars start from random positions on a road
 *     with periodic boundary conditions (a ring, no inflow or outflow).
 *   - "Concepts Covered": the two representations, grid (one value per road
 *     cell) and agent-based (two length-N vectors of positions and
 *     velocities).
 *   - "Concepts Covered" and the assignment's item 1: results must not
 *     depend on how the work is split.  Randomness therefore comes from a
 *     counter-based generator, Philox4x32-10 (Salmon, Moraes, Dror & Shaw,
 *     SC'11, "Parallel Random Numbers: As Easy as 1, 2, 3"), keyed by the
 *     seed and countered by (cell at the start of the step, step, road, tag).
 *
 * Readings where the paper is silent (every one is listed in the design
 * notes of the repository):
 *   - the update is synchronous: every gap is taken from the positions at
 *     the start of the step (double buffering);
 *   - the headway d to the car ahead is (x_lead - x) mod L, with d = L when
 *     a car is alone on the ring (it is its own leader);
 *   - initial velocities are 0; initial positions are N distinct cells drawn
 *     by Floyd's sampling algorithm (Bentley & Floyd, CACM 1987, "A sample of
 *     brilliance") from Philox draws with tag 1, then sorted;
 *   - per step the oracle reports sum_v = sum of velocities used for the
 *     move and crossings = number of cars whose move passes cell L-1 -> 0.
 *
 * Built twice: serially, and with -fopenmp for the CPU baseline.  The
 * OpenMP loops are race-free because every step reads one buffer and writes
 * another, and the sums are integers, so both builds agree bit for bit.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)
#define ORACLE_ECOLLIDE (-3)

#define ORACLE_TAG_SLOWDOWN 0u
#define ORACLE_TAG_INIT 1u
#define ORACLE_TAG_EXIT 2u
#define ORACLE_TAG_ENTRY 3u

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, section on the Philox family).       */
/* One round: two 32x32->64 products of counter words 0 and 2 by the round  */
/* multipliers; the high halves are xored with the other two counter words  */
/* and the key, and the words are permuted.  The key is bumped by the Weyl  */
/* constants (golden ratio, sqrt(3)-1) between rounds.                       */
/* ------------------------------------------------------------------------ */
static const uint32_t PHILOX_MUL_A = 0xD2511F53u;
static const uint32_t PHILOX_MUL_B = 0xCD9E8D57u;
static const uint32_t PHILOX_WEYL_A = 0x9E3779B9u;
static const uint32_t PHILOX_WEYL_B = 0xBB67AE85u;

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_WEYL_A;
            k1 += PHILOX_WEYL_B;
        }
        uint64_t prod_a = (uint64_t)PHILOX_MUL_A * (uint64_t)c0;
        uint64_t prod_b = (uint64_t)PHILOX_MUL_B * (uint64_t)c2;
        uint32_t hi_a = (uint32_t)(prod_a >> 32), lo_a = (uint32_t)prod_a;
        uint32_t hi_b = (uint32_t)(prod_b >> 32), lo_b = (uint32_t)prod_b;
        uint32_t n0 = hi_b ^ c1 ^ k0;
        uint32_t n1 = lo_b;
        uint32_t n2 = hi_a ^ c3 ^ k1;
        uint32_t n3 = lo_a;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Bulk form for tests: out[4*i + w] = Philox(ctr[4*i .. 4*i+3], key)[w]. */
void oracle_philox_many(int64_t n, const uint32_t *ctr, const uint32_t key[2], uint32_t *out)
{
    for (int64_t i = 0; i < n; ++i)
        oracle_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* Slowdown threshold: the paper draws r uniform on [0,1) and slows down iff
 * r < p.  With r = u * 2^-32, u a 32-bit word, r < p  <=>  u < p*2^32  <=>
 * u < ceil(p*2^32) since u is an integer.  p*2^32 is exact in double (a
 * power-of-two scaling), so the ceiling is exact.  p = 1 gives 2^32, which
 * every 32-bit u is below (always slow down); p = 0 gives 0 (never). */
uint64_t oracle_slow_threshold(double p)
{
    if (!(p > 0.0)) return 0;          /* also maps NaN to "never" */
    if (p >= 1.0) return (uint64_t)1 << 32;
    double scaled = p * 4294967296.0;
    uint64_t t = (uint64_t)scaled;     /* floor for positive values */
    if ((double)t < scaled) t += 1;    /* ceiling */
    return t;
}

/* The draw of rule 3 for the car that sits on `cell` at the start of `step`:
 * word 0 of Philox(ctr = (cell, step, road, 0), key = (seed lo, seed hi)). */
static uint32_t slowdown_word(uint64_t seed, uint32_t road, int64_t cell, uint64_t step)
{
    uint32_t ctr[4] = {(uint32_t)cell, (uint32_t)step, road, ORACLE_TAG_SLOWDOWN};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[0];
}

/* ------------------------------------------------------------------------ */
/* Initial positions: Floyd's algorithm.  For m = 0..N-1 let j = L-N+m, draw */
/* t uniformly from {0..j}; insert t unless it is already in the set, in     */
/* which case insert j.  The result is a uniformly random N-subset of        */
/* {0..L-1}.  The uniform draw on {0..j} is Lemire's multiply-shift of a     */
/* 64-bit word r = (w1 << 32) | w0 from Philox(ctr = (m, 0, road, 1)):       */
/* t = floor(r * (j+1) / 2^64).  The set is a bitmap over the L cells, so    */
/* reading it in cell order gives the sorted positions.                      */
/* ------------------------------------------------------------------------ */
int oracle_floyd_init(int64_t L, int64_t N, uint64_t seed, uint32_t road, int32_t *x_out)
{
    if (L < 1 || L > ((int64_t)1 << 31) || N < 0 || N > L) return ORACLE_EINVAL;
    if (N == 0) return ORACLE_OK;
    int64_t words = (L + 63) / 64;
    uint64_t *chosen = (uint64_t *)calloc((size_t)words, sizeof(uint64_t));
    if (!chosen) return ORACLE_ENOMEM;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t m = 0; m < N; ++m) {
        int64_t j = L - N + m;
        uint32_t ctr[4] = {(uint32_t)m, 0u, road, ORACLE_TAG_INIT};
        uint32_t w[4];
        oracle_philox4x32_10(ctr, key, w);
        uint64_t r = ((uint64_t)w[1] << 32) | (uint64_t)w[0];
        uint64_t t = (uint64_t)(((unsigned __int128)r * (unsigned __int128)(uint64_t)(j + 1)) >> 64);
        int64_t pick = (chosen[t / 64] >> (t % 64)) & 1u ? j : (int64_t)t;
        chosen[pick / 64] |= (uint64_t)1 << (pick % 64);
    }
    int64_t n = 0;
    for (int64_t c = 0; c < L; ++c)
        if ((chosen[c / 64] >> (c % 64)) & 1u) x_out[n++] = (int32_t)c;
    free(chosen);
    return n == N ? ORACLE_OK : ORACLE_EINVAL;
}

/* ------------------------------------------------------------------------ */
/* Agent-based representation: car i has position x[i] and velocity v[i];   */
/* cars are stored in cyclic order, so the car ahead of i is (i+1) mod N.    */
/* ------------------------------------------------------------------------ */
int oracle_agent_run(int64_t L, int64_t N, int32_t vmax, uint64_t thr, uint64_t seed,
                     uint32_t road, uint64_t step0, int64_t T, int32_t *x, uint8_t *v,
                     uint64_t *sum_v, uint64_t *crossings)
{
    if (L < 1 || L > ((int64_t)1 << 31) || N < 0 || N > L || vmax < 0 || vmax > 127 || T < 0)
        return ORACLE_EINVAL;
    if (N == 0) {
        for (int64_t t = 0; t < T; ++t) {
            if (sum_v) sum_v[t] = 0;
            if (crossings) crossings[t] = 0;
        }
        return ORACLE_OK;
    }
    int32_t *x_next = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    uint8_t *v_next = (uint8_t *)malloc((size_t)N);
    if (!x_next || !v_next) {
        free(x_next);
        free(v_next);
        return ORACLE_ENOMEM;
    }
    for (int64_t t = 0; t < T; ++t) {
        uint64_t step = step0 + (uint64_t)t;
        uint64_t moved = 0, wrapped = 0;
#pragma omp parallel for schedule(static) reduction(+ : moved, wrapped)
        for (int64_t i = 0; i < N; ++i) {
            int64_t xi = x[i];
            int64_t lead = x[(i + 1) % N];
            int64_t d = lead - xi;               /* headway, cells */
            if (d <= 0) d += L;                  /* ring; alone: d = L */
            int64_t vel = (int64_t)v[i] + 1;     /* rule 1 */
            if (vel > vmax) vel = vmax;
            if (vel > d - 1) vel = d - 1;        /* rule 2 */
            if (vel > 0) {                       /* rule 3 */
                if ((uint64_t)slowdown_word(seed, road, xi, step) < thr) vel -= 1;
            }
            int64_t nx = xi + vel;               /* rule 4 */
            if (nx >= L) {
                nx -= L;
                wrapped += 1;
            }
            x_next[i] = (int32_t)nx;
            v_next[i] = (uint8_t)vel;
            moved += (uint64_t)vel;
        }
        memcpy(x, x_next, (size_t)N * sizeof(int32_t));
        memcpy(v, v_next, (size_t)N);
        if (sum_v) sum_v[t] = moved;
        if (crossings) crossings[t] = wrapped;
    }
    free(x_next);
    free(v_next);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* One synchronous step of the agent form with the rule-3 outcome given      */
/* instead of drawn: slow[i] != 0 means car i's Bernoulli trial succeeded    */
/* (r < p).  Rules 1-4 as in oracle_agent_run (Handout, "The                 */
/* Nagel-Schreckenberg traffic model"); a car that is stopped after rule 2   */
/* stays stopped whatever its trial.  This is the model's one-step           */
/* transition for one outcome of the N independent trials, so enumerating    */
/* all 2^N outcomes (each with probability p^k (1-p)^(N-k)) gives the whole  */
/* one-step distribution.  `count` independent states of N cars each are     */
/* stepped: state s is x[s*N .. s*N+N-1], v[...], slow[...] (cars in cyclic  */
/* order, distinct cells in [0, L)); results go to x_out and v_out.          */
/* ------------------------------------------------------------------------ */
int oracle_agent_step_masked(int64_t L, int64_t N, int32_t vmax, int64_t count, const int32_t *x,
                             const uint8_t *v, const uint8_t *slow, int32_t *x_out, uint8_t *v_out)
{
    if (L < 1 || L > ((int64_t)1 << 31) || N < 1 || N > L || vmax < 0 || vmax > 127 || count < 0)
        return ORACLE_EINVAL;
    for (int64_t s = 0; s < count; ++s) {
        const int32_t *xs = x + s * N;
        const uint8_t *vs = v + s * N;
        const uint8_t *ms = slow + s * N;
        for (int64_t i = 0; i < N; ++i) {
            int64_t xi = xs[i];
            int64_t d = (int64_t)xs[(i + 1) % N] - xi;   /* headway */
            if (d <= 0) d += L;                          /* ring; alone: d = L */
            int64_t vel = (int64_t)vs[i] + 1;            /* rule 1 */
            if (vel > vmax) vel = vmax;
            if (vel > d - 1) vel = d - 1;                /* rule 2 */
            if (vel > 0 && ms[i]) vel -= 1;              /* rule 3 */
            int64_t nx = xi + vel;                       /* rule 4 */
            if (nx >= L) nx -= L;
            x_out[s * N + i] = (int32_t)nx;
            v_out[s * N + i] = (uint8_t)vel;
        }
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Grid representation: one int8 per cell, -1 empty, otherwise the velocity  */
/* of the car on it.  The gap is found by scanning forward over empty cells  */
/* (at most the accelerated velocity); the successor grid starts all empty   */
/* and every car writes its new cell.  Two cars never land on one cell;      */
/* if they did, the rules would be broken and the oracle reports it.         */
/* ------------------------------------------------------------------------ */
int oracle_grid_run(int64_t L, int32_t vmax, uint64_t thr, uint64_t seed, uint32_t road,
                    uint64_t step0, int64_t T, int8_t *cells, uint64_t *sum_v,
                    uint64_t *crossings)
{
    if (L < 1 || L > ((int64_t)1 << 31) || vmax < 0 || vmax > 127 || T < 0) return ORACLE_EINVAL;
    int8_t *next = (int8_t *)malloc((size_t)L);
    if (!next) return ORACLE_ENOMEM;
    int status = ORACLE_OK;
    for (int64_t t = 0; t < T && status == ORACLE_OK; ++t) {
        uint64_t step = step0 + (uint64_t)t;
        uint64_t moved = 0, wrapped = 0;
        int collided = 0;
        memset(next, -1, (size_t)L);
#pragma omp parallel for schedule(static) reduction(+ : moved, wrapped, collided)
        for (int64_t j = 0; j < L; ++j) {
            if (cells[j] < 0) continue;
            int64_t vel = (int64_t)cells[j] + 1;              /* rule 1 */
            if (vel > vmax) vel = vmax;
            int64_t gap = 0;                                  /* rule 2 */
            while (gap < vel) {
                int64_t ahead = (j + gap + 1) % L;            /* ring */
                if (cells[ahead] >= 0) break;                 /* includes itself */
                gap += 1;
            }
            if (vel > gap) vel = gap;
            if (vel > 0) {                                    /* rule 3 */
                if ((uint64_t)slowdown_word(seed, road, j, step) < thr) vel -= 1;
            }
            int64_t dest = j + vel;                           /* rule 4 */
            if (dest >= L) {
                dest -= L;
                wrapped += 1;
            }
            if (next[dest] != -1) collided += 1;
            next[dest] = (int8_t)vel;
            moved += (uint64_t)vel;
        }
        if (collided) status = ORACLE_ECOLLIDE;
        memcpy(cells, next, (size_t)L);
        if (sum_v) sum_v[t] = moved;
        if (crossings) crossings[t] = wrapped;
    }
    free(next);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Open road (the handout's "Variations": other boundary conditions).  The   */
/* road is cells 0..L-1 with an entry before cell 0 and an exit after cell    */
/* L-1, no ring.  The paper gives no rules for them; the reading:             */
/*   - the exit is open at step t with probability beta: word 0 of            */
/*     Philox(ctr = (0, t, road, 2)) < ceil(beta * 2^32).  The leading car    */
/*     (no car ahead of it on the road) sees an unbounded road when the exit  */
/*     is open, and the end of the road (L-1-x empty cells) when it is        */
/*     closed; a car whose move passes cell L-1 leaves the road;              */
/*   - rules 1-4 otherwise as on the ring, from start-of-step positions;      */
/*   - after the moves, if cell 0 is empty, a car enters there with velocity  */
/*     0 with probability alpha: word 0 of Philox(ctr = (0, t, road, 3)) <    */
/*     ceil(alpha * 2^32).                                                    */
/* Per step: sum_v = velocities of the moves (the leaving cars included),     */
/* crossings = cars that left.                                               */
/* ------------------------------------------------------------------------ */
static uint32_t boundary_word(uint64_t seed, uint32_t road, uint64_t step, uint32_t tag)
{
    uint32_t ctr[4] = {0u, (uint32_t)step, road, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[0];
}

int oracle_open_run(int64_t L, int32_t vmax, uint64_t thr, uint64_t thr_entry, uint64_t thr_exit, uint64_t seed,
                    uint32_t road, uint64_t step0, int64_t T, int8_t *cells, uint64_t *sum_v, uint64_t *crossings)
{
    if (L < 1 || L > ((int64_t)1 << 31) || vmax < 0 || vmax > 127 || T < 0) return ORACLE_EINVAL;
    int8_t *next = (int8_t *)malloc((size_t)L);
    if (!next) return ORACLE_ENOMEM;
    int status = ORACLE_OK;
    for (int64_t t = 0; t < T && status == ORACLE_OK; ++t) {
        uint64_t step = step0 + (uint64_t)t;
        const int exit_open = (uint64_t)boundary_word(seed, road, step, ORACLE_TAG_EXIT) < thr_exit;
        uint64_t moved = 0, left = 0;
        int collided = 0;
        memset(next, -1, (size_t)L);
        for (int64_t j = 0; j < L; ++j) {
            if (cells[j] < 0) continue;
            int64_t vel = (int64_t)cells[j] + 1;              /* rule 1 */
            if (vel > vmax) vel = vmax;
            int64_t gap = 0;                                  /* rule 2 */
            while (gap < vel) {
                int64_t ahead = j + gap + 1;
                if (ahead >= L) {                             /* past the end of the road */
                    if (!exit_open) break;                    /* closed: the road ends at L-1 */
                    gap = vel;                                /* open: nothing ahead */
                    break;
                }
                if (cells[ahead] >= 0) break;
                gap += 1;
            }
            if (vel > gap) vel = gap;
            if (vel > 0) {                                    /* rule 3 */
                if ((uint64_t)slowdown_word(seed, road, j, step) < thr) vel -= 1;
            }
            int64_t dest = j + vel;                           /* rule 4 */
            moved += (uint64_t)vel;
            if (dest >= L) {                                  /* leaves the road */
                left += 1;
                continue;
            }
            if (next[dest] != -1) collided += 1;
            next[dest] = (int8_t)vel;
        }
        if (collided) status = ORACLE_ECOLLIDE;
        if (next[0] < 0 && (uint64_t)boundary_word(seed, road, step, ORACLE_TAG_ENTRY) < thr_entry)
            next[0] = 0;                                      /* a car enters at rest */
        memcpy(cells, next, (size_t)L);
        if (sum_v) sum_v[t] = moved;
        if (crossings) crossings[t] = left;
    }
    free(next);
    return status;
}

/* Agent -> grid: cell x[i] holds v[i]; every other cell is -1. */
int oracle_agent_to_grid(int64_t L, int64_t N, const int32_t *x, const uint8_t *v, int8_t *cells)
{
    if (L < 1 || N < 0 || N > L) return ORACLE_EINVAL;
    memset(cells, -1, (size_t)L);
    for (int64_t i = 0; i < N; ++i) {
        if (x[i] < 0 || x[i] >= L || cells[x[i]] != -1) return ORACLE_EINVAL;
        cells[x[i]] = (int8_t)v[i];
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Light-cone forms for sampled checks on roads too long to run whole.       */
/* The rules are local: a car's next state depends on itself and the car     */
/* ahead (agent), a cell's next value on the cells within vmax of it (grid). */
/* So M consecutive cars determine the first M-T of them T steps later, and  */
/* W consecutive cells determine the middle W - 2*T*vmax cells.              */
/* ------------------------------------------------------------------------ */

/* x[0..M-1], v[0..M-1]: consecutive cars in cyclic order (car m+1 is ahead of
 * car m).  On return the first M-T entries hold their state T steps later. */
int oracle_agent_segment(int64_t L, int64_t M, int32_t vmax, uint64_t thr, uint64_t seed,
                         uint32_t road, uint64_t step0, int64_t T, int32_t *x, uint8_t *v)
{
    if (L < 1 || L > ((int64_t)1 << 31) || M < 1 || T < 0 || T >= M || vmax < 0 || vmax > 127)
        return ORACLE_EINVAL;
    int32_t *x_next = (int32_t *)malloc((size_t)M * sizeof(int32_t));
    uint8_t *v_next = (uint8_t *)malloc((size_t)M);
    if (!x_next || !v_next) {
        free(x_next);
        free(v_next);
        return ORACLE_ENOMEM;
    }
    int64_t live = M;                    /* cars whose state is still exact */
    for (int64_t t = 0; t < T; ++t) {
        uint64_t step = step0 + (uint64_t)t;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < live - 1; ++i) {
            int64_t xi = x[i];
            int64_t d = (int64_t)x[i + 1] - xi;
            if (d <= 0) d += L;
            int64_t vel = (int64_t)v[i] + 1;
            if (vel > vmax) vel = vmax;
            if (vel > d - 1) vel = d - 1;
            if (vel > 0 && (uint64_t)slowdown_word(seed, road, xi, step) < thr) vel -= 1;
            int64_t nx = xi + vel;
            if (nx >= L) nx -= L;
            x_next[i] = (int32_t)nx;
            v_next[i] = (uint8_t)vel;
        }
        live -= 1;
        memcpy(x, x_next, (size_t)live * sizeof(int32_t));
        memcpy(v, v_next, (size_t)live);
    }
    free(x_next);
    free(v_next);
    return ORACLE_OK;
}

/* cells[0..W-1] hold road cells first, first+1, ... (mod L).  On return
 * cells[T*vmax .. W-T*vmax-1] hold those cells T steps later; the margins are
 * left as computed from an unknown outside and must not be used. */
int oracle_grid_segment(int64_t L, int64_t W, int64_t first, int32_t vmax, uint64_t thr,
                        uint64_t seed, uint32_t road, uint64_t step0, int64_t T, int8_t *cells)
{
    if (L < 1 || L > ((int64_t)1 << 31) || W < 1 || T < 0 || vmax < 0 || vmax > 127 ||
        2 * T * (int64_t)vmax >= W || first < 0 || first >= L)
        return ORACLE_EINVAL;
    int8_t *next = (int8_t *)malloc((size_t)W);
    if (!next) return ORACLE_ENOMEM;
    for (int64_t t = 0; t < T; ++t) {
        uint64_t step = step0 + (uint64_t)t;
        memset(next, -1, (size_t)W);
        for (int64_t j = 0; j < W; ++j) {
            if (cells[j] < 0) continue;
            int64_t vel = (int64_t)cells[j] + 1;
            if (vel > vmax) vel = vmax;
            int64_t gap = 0;
            while (gap < vel && j + gap + 1 < W && cells[j + gap + 1] < 0) gap += 1;
            if (vel > gap) vel = gap;
            int64_t cell = (first + j) % L;
            if (vel > 0 && (uint64_t)slowdown_word(seed, road, cell, step) < thr) vel -= 1;
            if (j + vel < W) next[j + vel] = (int8_t)vel;
        }
        memcpy(cells, next, (size_t)W);
    }
    free(next);
    return ORACLE_OK;
}

/* Thread control for the OpenMP build (the serial build reports 1). */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
