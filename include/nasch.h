/*
 * nasch.h: C ABI of the GB300 (sm_103a) Nagel-Schreckenberg library.
 *
 * The operation is the synchronous time step of the 1-D Nagel-Schreckenberg
 * model on a ring road of L cells (van Zon & Ponce, "Parallelizing a 1-Dim
 * Nagel-Schreckenberg Traffic Model", EduHPC-23; Handout, "The
 * Nagel-Schreckenberg traffic model", rules 1-4), applied to every car at
 * once:
 *     v <- min(v + 1, vmax)                      rule 1, accelerate
 *     v <- min(v, d - 1), d = headway ahead      rule 2, brake
 *     v <- max(v - 1, 0) with probability p      rule 3, random slowdown
 *     x <- (x + v) mod L                         rule 4, move on the ring
 * The model's parameters are those of the handout's parameter file
 * (Handout, "Starter Code": L, T, N, p, vmax, seed).
 *
 * Randomness.  The rule-3 draw of the car that sits on cell c at the start
 * of step t is word 0 of Philox4x32-10 (Salmon et al., SC'11) of counter
 * (c, t mod 2^32, road_id, 0) under key (seed mod 2^32, seed >> 32); the car
 * slows down iff that word is below ceil(p * 2^32).  That is the handout's
 * "draw r uniform on [0,1), slow down iff r < p" with r = word * 2^-32, and
 * it makes every result independent of how the work is split over threads,
 * tiles, launches or batches (the assignment's reproducibility requirement,
 * item 1).  Initial positions are N distinct cells chosen by Floyd's
 * algorithm from Philox counters (m, 0, road_id, 1), sorted; all v = 0.
 *
 * Representations ("Concepts Covered"): agent-based (int32 positions x[N],
 * uint8 velocities v[N], cars in cyclic order, the car ahead of car i is car
 * (i+1) mod N) and grid (int8 cells[L], -1 empty, else the velocity of the
 * car on that cell).  Both give identical results.
 *
 * Statistics.  Every step records two exact integers: sum_v, the sum of the
 * velocities used for the move (flux J = sum_v / L, mean velocity
 * sum_v / N), and crossings, the number of cars whose move passes from cell
 * L-1 to cell 0.
 *
 * Conventions.
 *   - Every function returns NASCH_OK (0) or a negative status; on error,
 *     nasch_last_error() returns a message for the calling thread.  No C++
 *     exception crosses this interface.
 *   - Pointers named *_host are caller-owned host memory; the library copies
 *     from or into them and keeps no reference.  Device state is owned by
 *     the library and freed by nasch_destroy / nasch_batch_destroy.
 *   - Work is enqueued on the handle's CUDA stream and runs asynchronously;
 *     functions that return results to the host synchronise that stream.
 *   - Limits: 1 <= L <= 2^31, 0 <= N <= L, 0 <= vmax <= 127, 0 <= p <= 1
 *     (p = 1 always slows a moving car down).  Anything else is
 *     NASCH_EINVAL.
 *   - A handle is not thread-safe; distinct handles may be used from
 *     distinct threads.
 */
#ifndef NASCH_H
#define NASCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define NASCH_OK 0
#define NASCH_EINVAL (-1)    /* invalid argument or state */
#define NASCH_ENOMEM (-2)    /* device or host allocation failed, or budget exceeded */
#define NASCH_ECUDA (-3)     /* a CUDA runtime call failed (message has the CUDA error) */
#define NASCH_ETIMEOUT (-4)  /* a bounded wait ran out; the work is still in flight */
#define NASCH_EBUSY (-5)     /* the object is in use by enqueued work */
#define NASCH_ECANCELED (-6) /* the batch or request was cancelled */

/* State layouts. */
#define NASCH_LAYOUT_AUTO 0  /* agent below the crossover density, grid above */
#define NASCH_LAYOUT_AGENT 1
#define NASCH_LAYOUT_GRID 2

typedef struct nasch_road *nasch_handle;
typedef struct nasch_batch_s *nasch_batch;

/* Parameters of one road.  Fill with nasch_params_init, then set fields. */
typedef struct nasch_params {
    int64_t L;        /* ring length in cells, 1..2^31 */
    int64_t N;        /* number of cars, 0..L */
    int32_t vmax;     /* maximum velocity, 0..127 */
    double p;         /* slowdown probability, 0..1 */
    uint64_t seed;    /* Philox key */
    uint32_t road_id; /* Philox counter word 2: distinguishes roads sharing a seed */
    int32_t layout;   /* NASCH_LAYOUT_* */
    int32_t k;        /* steps fused per launch (temporal blocking); 0 = library choice */
    int32_t tile;     /* cars (agent) or cells (grid) per tile; 0 = library choice */
    void *stream;     /* cudaStream_t to enqueue on; NULL = a stream owned by the handle */
} nasch_params;

/* Read-only description of a handle. */
typedef struct nasch_info {
    int64_t L, N;
    int32_t vmax;
    int32_t layout;       /* NASCH_LAYOUT_AGENT or NASCH_LAYOUT_GRID, as resolved */
    int32_t k;            /* fusion depth in use */
    int32_t tile;         /* tile in use (cars or cells) */
    uint64_t step;        /* global index of the next step to run */
    uint64_t stats_first; /* first step whose statistics are kept */
    uint64_t threshold;   /* ceil(p * 2^32) */
    int32_t ring_kernel;  /* 1 if the whole ring runs in one thread block */
    int32_t blocks;       /* thread blocks of the tiled kernel (persistent grid) */
} nasch_info;

/* Defaults: L = N = 0, vmax = 5, p = 0, seed = 0, road 0, AUTO, k = tile = 0, stream NULL. */
void nasch_params_init(nasch_params *prm);

/* Create one road with Floyd-sampled start positions and v = 0 at step 0
 * (Handout, "Starter Code": cars start from random positions on a ring).
 * Allocates the device state on the current CUDA device. */
int nasch_create(int64_t L, int64_t N, int vmax, double p, uint64_t seed, nasch_handle *out);

/* As nasch_create with every parameter of nasch_params. */
int nasch_create_ex(const nasch_params *prm, nasch_handle *out);

/* An open road (Handout, "Variations": other boundary conditions): cells
 * 0..L-1 with an entry before cell 0 and an exit after cell L-1 instead of
 * the ring.  Each step: the exit is open with probability beta (word 0 of
 * Philox with counter (0, step, road, 2) below ceil(beta * 2^32)); the
 * leading car then sees an unbounded road, else the road's end; the four
 * rules move every car as on the ring, and a car whose move passes cell L-1
 * leaves (counted in the step's crossings); then, if cell 0 is empty, a car
 * enters it at rest with probability alpha (counter (0, step, road, 3)).
 * The road starts with N cars placed as by nasch_create.  Grid layout only
 * (layout AUTO or GRID; AGENT is NASCH_EINVAL), one step per launch (k and
 * tile are ignored), any L >= 1.  The car count changes: read the state
 * with nasch_read_grid (nasch_read_state is NASCH_EINVAL);
 * nasch_set_state takes any N in 0..L.  NASCH_EINVAL also for alpha or beta
 * outside [0, 1]. */
int nasch_create_open(const nasch_params *prm, double alpha, double beta, nasch_handle *out);

/* Replace the state: N cars (N must equal the handle's N) at positions
 * x_host[0..N-1] (distinct, in [0, L), in cyclic order: a rotation of an
 * increasing sequence; a grid road takes any order) with velocities
 * v_host[0..N-1] <= vmax; the next step run is `step`.  Statistics kept so
 * far are dropped.  Copies the host arrays to the device on the handle's
 * stream, checks them there and returns once the check is complete.  A
 * state that breaks a rule is NASCH_EINVAL (the message names the first bad
 * car, or the shared cell) and leaves the road's state as it was. */
int nasch_set_state(nasch_handle h, const int32_t *x_host, const uint8_t *v_host, int64_t N,
                    uint64_t step);

/* Enqueue `steps` synchronous time steps (each: rules 1-4 for every car,
 * then the per-step sum_v and crossings).  Asynchronous. */
int nasch_run(nasch_handle h, int64_t steps);

/* Run with output: the handout's `per` parameter (Handout, parameter file
 * and output: a density and velocity picture of the road every `per`
 * steps, none when per = 0) and its space-time diagram (Fig. 1).  Enqueues
 * `steps` steps; after each full chunk of `per` steps (counted from this
 * call) takes snapshot j = 0, 1, ...:
 *   snap_host (may be NULL): the road's L cells (-1 empty, else the velocity;
 *     an agent road is scattered into cells) go to snap_host + (j mod
 *     snap_cap) * L, so snap_cap >= steps / per keeps them all; caller-owned,
 *     pinned host memory lets the copy overlap the following steps;
 *   raster_host (may be NULL): one row of raster_width pixels (1 <=
 *     raster_width <= L) goes to raster_host + (j mod raster_cap) *
 *     raster_width; pixel i covers the cells c with floor(c * raster_width /
 *     L) = i and holds floor(255 * cars / cells) of them.
 * A partial last chunk (steps not a multiple of per) runs without a
 * snapshot.  per = 0, or both outputs NULL, runs the steps with no output.
 * Returns once every copy is in host memory (synchronises the stream).
 * NASCH_EINVAL for negative steps or per, or a capacity or width out of
 * range; NASCH_ECUDA if staging memory cannot be allocated. */
int nasch_run_output(nasch_handle h, int64_t steps, int64_t per, int8_t *snap_host, int64_t snap_cap,
                     uint8_t *raster_host, int32_t raster_width, int64_t raster_cap);

/* Copy the current state to the host.  Agent layout: cars in their cyclic
 * order.  Grid layout: cars in increasing cell order.  cap is the capacity
 * of both arrays in elements and must be >= N.  Synchronises the stream. */
int nasch_read_state(nasch_handle h, int32_t *x_host, uint8_t *v_host, int64_t cap);

/* Copy the current state as a grid (cells_host[0..L-1], -1 empty, else the
 * velocity).  cap must be >= L.  Synchronises the stream. */
int nasch_read_grid(nasch_handle h, int8_t *cells_host, int64_t cap);

/* Copy the statistics of steps first_step .. first_step+count-1 (global
 * step indices; they must lie between nasch_info.stats_first and the
 * current step).  Either output may be NULL.  Synchronises the stream. */
int nasch_stats(nasch_handle h, uint64_t first_step, int64_t count, uint64_t *sum_v_host,
                uint64_t *crossings_host);

int nasch_get_info(nasch_handle h, nasch_info *info);

/* Block until all work enqueued on the handle has finished. */
int nasch_synchronize(nasch_handle h);

/* Free the handle and its device memory (synchronises first).  NULL is a no-op. */
void nasch_destroy(nasch_handle h);

/* Message of the last failing call on this thread ("" if none). */
const char *nasch_last_error(void);

/* The library's slowdown threshold ceil(p * 2^32) (2^32 for p = 1). */
uint64_t nasch_slow_threshold(double p);

/* The library's Floyd initialisation on the host: N sorted distinct cells of
 * the ring for (seed, road_id), written to x_host[0..N-1]. */
int nasch_floyd_init(int64_t L, int64_t N, uint64_t seed, uint32_t road_id, int32_t *x_host);

/* Philox4x32-10 evaluated by the library's device code, for testing: for
 * i < n, out_host[4i..4i+3] = Philox(ctr_host[4i..4i+3], key (seed lo, seed
 * hi)).  Runs one kernel and synchronises. */
int nasch_philox_device(int64_t n, const uint32_t *ctr_host, uint64_t seed, uint32_t *out_host);

/* ------------------------------------------------------------------------
 * Batches: many independent roads (a parameter study run as one job - the
 * paper's "Variations": a series of parameter cases as embarrassingly
 * parallel work).  Road i has parameters roads[i] (layout AUTO picks agent or
 * grid by density; k and tile may be left 0) and runs steps[i] steps from a
 * Floyd start keyed by (roads[i].seed, roads[i].road_id).  All roads advance
 * together in super-steps: one persistent launch per super-step pulls
 * (road, tile) items from a work-list, each item running that road's k fused
 * steps; the launch sequence is captured in CUDA graphs.  Every road's result
 * equals the same road run alone with nasch_create_ex/nasch_run.
 * The stream of roads[0] is used (NULL: the batch owns one).  The call
 * returns once the work is enqueued.
 * ------------------------------------------------------------------------ */
typedef struct nasch_batch_info {
    int64_t n_roads;
    int64_t super_steps;    /* launches in the job */
    int64_t items;          /* (road, tile) items of the first super-step */
    int64_t device_bytes;   /* device memory held by the batch */
    int64_t vehicle_steps;  /* sum over roads of N * steps */
    int64_t cell_steps;     /* sum over roads of L * steps */
    int32_t blocks;         /* persistent thread blocks per launch */
    int32_t graphs;         /* CUDA graphs the launches were captured in */
    double run_seconds;     /* GPU time from the first launch to the last (after the start state is
                               built); 0 until the batch has finished */
} nasch_batch_info;

int nasch_submit(const nasch_params *roads, int64_t n_roads, const int64_t *steps, nasch_batch *out);

/* Wait up to timeout_ms (< 0: no limit) for the batch to finish.  Returns
 * NASCH_OK, NASCH_ETIMEOUT if it is still running (nothing is lost; wait
 * again), or NASCH_ECANCELED if it was cancelled. */
int nasch_batch_wait(nasch_batch b, int64_t timeout_ms);

/* Ask the batch to stop: launches still to run skip their work.  The batch
 * must still be waited for before its results (then undefined) or memory
 * are released. */
int nasch_batch_cancel(nasch_batch b);

/* Final state and statistics of road i (after nasch_batch_wait returned OK).
 * Statistics are indexed by the road's global step (0 .. steps[i]-1). */
int nasch_batch_read_state(nasch_batch b, int64_t i, int32_t *x_host, uint8_t *v_host, int64_t cap);
int nasch_batch_read_grid(nasch_batch b, int64_t i, int8_t *cells_host, int64_t cap);
int nasch_batch_stats(nasch_batch b, int64_t i, uint64_t first_step, int64_t count, uint64_t *sum_v_host,
                      uint64_t *crossings_host);
/* Sums of the per-step statistics of road i over steps [first, first + count). */
int nasch_batch_stats_sum(nasch_batch b, int64_t i, uint64_t first_step, int64_t count, uint64_t *sum_v_total,
                          uint64_t *crossings_total);
int nasch_batch_get_info(nasch_batch b, nasch_batch_info *info);
/* Layout chosen for road i (NASCH_LAYOUT_AGENT or NASCH_LAYOUT_GRID). */
int nasch_batch_road_layout(nasch_batch b, int64_t i, int32_t *layout);

/* Wait for the batch (no limit) and free it.  NULL is a no-op. */
void nasch_batch_destroy(nasch_batch b);

/* Tuning of the automatic choices (process-wide; the autotuner sets these):
 * rho_star - density below which AUTO picks the agent layout (default 1:
 * with fused steps the agent step is the faster one at every density; a
 * single AUTO road whose state would need more than half of the free device
 * memory at rho_star, or a batch that would need more than 85 % of it
 * (states, statistics and start-state bit maps), uses 0.2 instead, the
 * density where the agent state (10 bytes per car) and the grid state (2
 * per cell) are equal);
 * k_agent, k_grid - fused steps per launch of tiled roads (0 leaves a value
 * unchanged). */
int nasch_set_tuning(double rho_star, int32_t k_agent, int32_t k_grid);
int nasch_get_tuning(double *rho_star, int32_t *k_agent, int32_t *k_grid);

/* Per-road tuning of batched and served roads (process-wide; the
 * autotuner fills it from timings of each bucket of roads).  An entry
 * matches a road with L_min <= L < L_max, rho_min <= N / L < rho_max,
 * vmax_min <= vmax <= vmax_max and the draw mode `draw` (-1 any p; 0: p = 0;
 * 1: 0 < p < 1; 2: p = 1); the first matching entry decides, for the
 * choices the road leaves to the library: the layout of an AUTO road
 * (NASCH_LAYOUT_AGENT or _GRID; AUTO keeps the density rule), the fusion
 * depth of a road with k = 0 (0 keeps the default), and the tile of a grid
 * road with tile = 0 (2048: warp-tiles of the list method; 8192: block-wide
 * spans; 0 keeps the default).  A road no entry matches uses the global
 * tuning above.  A batch that would need more than 85 % of the free device
 * memory ignores the table's layouts and uses the state-byte crossover.  The
 * choice never changes a road's result, only its speed. */
typedef struct nasch_tuning_entry {
    int64_t L_min, L_max;
    double rho_min, rho_max;
    int32_t vmax_min, vmax_max;
    int32_t draw;
    int32_t layout;
    int32_t k;
    int32_t tile;
} nasch_tuning_entry;

/* Replace the table by entries[0..n-1] (n = 0 clears it); NASCH_EINVAL for
 * an entry out of range (empty ranges, k outside 0..64, an unknown layout
 * or tile), leaving the table as it was. */
int nasch_set_tuning_table(const nasch_tuning_entry *entries, int64_t n);
/* Copy up to cap entries to out; *n receives the table's length. */
int nasch_get_tuning_table(nasch_tuning_entry *out, int64_t cap, int64_t *n);
/* The layout (NASCH_LAYOUT_AGENT or _GRID), fusion depth and tile a batch
 * would give `road` from the tuning above and the table, memory permitting
 * (host arithmetic only; needs no GPU).  tile: 2048 or 8192 for grid roads
 * on tiles, 256 for agent roads on warp-tiles, 0 for roads stepped as a
 * whole ring in one item. */
int nasch_tuned_choice(const nasch_params *road, int32_t *layout, int32_t *k, int32_t *tile);

/* ------------------------------------------------------------------------
 * Serving: a request loop with continuous batching.  Requests (one road
 * each, the paper's parameter set plus a step count) queue in arrival order;
 * each scheduling round admits queued requests, oldest first, while their
 * state and statistics fit the device-memory budget, and enqueues one tick
 * of launches over every resident road, each continuing from its own step -
 * requests admitted later run in the same launches as earlier ones.  A tick
 * is at least steps_per_tick super-step launches, and more (up to
 * max_steps_per_tick) while the resident roads are too few to keep the GPU
 * busy for target_tick_ms per tick; up to ticks_in_flight ticks are queued
 * on the GPU at once, so the host plans the next while the GPU runs.  The
 * per-step statistics of a running request can be streamed back as its
 * steps finish (nasch_server_poll_series).  Finished requests return their
 * per-step statistics (and, with keep_state, their final state) to the host
 * and their memory to the budget.  A request's result equals the same road
 * run alone.
 * ------------------------------------------------------------------------ */
typedef struct nasch_server_s *nasch_server;

typedef struct nasch_server_config {
    int64_t memory_budget;   /* device bytes for resident roads (one slab, allocated at create) */
    int32_t steps_per_tick;  /* fewest super-step launches per scheduling round (default 8) */
    int32_t max_resident;    /* most roads resident at once (default 4096) */
    int32_t keep_state;      /* nonzero: also copy each request's final state back */
    void *stream;            /* cudaStream_t; NULL = one owned by the server */
    int32_t max_steps_per_tick; /* most super-step launches per round (default 256; >= steps_per_tick) */
    int32_t ticks_in_flight;    /* ticks queued on the GPU at once, 1..4 (default 3) */
    double target_tick_ms;      /* GPU time a tick aims at (default 4; 0: always steps_per_tick) */
} nasch_server_config;

typedef struct nasch_request_result {
    uint64_t request_id;
    int32_t status;          /* NASCH_OK or NASCH_ECANCELED */
    int32_t layout;
    int64_t steps;
    int64_t vehicles;
    double submit_time;      /* seconds since the server was created (host clock) */
    double admit_time;
    double done_time;        /* when the host saw the last launch finish */
} nasch_request_result;

typedef struct nasch_server_info {
    int64_t queued, resident, completed;
    int64_t bytes_in_use;
    int64_t ticks;
    int64_t vehicle_steps_done;
    int32_t blocks;
    double now;              /* seconds since the server was created (host clock) */
    double gpu_busy_seconds; /* GPU time of the finished ticks (first launch to last, per tick) */
    int32_t last_tick_super_steps;  /* launches in the latest tick */
    int32_t pad;
} nasch_server_info;

/* One piece of a request's per-step series (nasch_server_poll_series):
 * steps first_step .. first_step+count-1 of request request_id, stored at
 * sum_v_host[offset ..] and crossings_host[offset ..]. */
typedef struct nasch_series_chunk {
    uint64_t request_id;
    int64_t first_step;
    int64_t count;
    int64_t offset;
} nasch_series_chunk;

/* Defaults: 40 GiB budget, 8 to 256 launches per tick aiming at 4 ms of GPU
 * time, 3 ticks in flight, 4096 resident roads. */
void nasch_server_config_init(nasch_server_config *cfg);
int nasch_server_create(const nasch_server_config *cfg, nasch_server *out);
/* Queue one request (thread-safe).  NASCH_ENOMEM if it could never fit the budget. */
int nasch_server_submit(nasch_server s, const nasch_params *road, int64_t steps, uint64_t request_id);
/* One scheduling round: retire finished requests, admit queued ones, enqueue
 * a tick (blocks only while two ticks are already in flight).  *pending
 * (may be NULL) receives the queued plus resident requests. */
int nasch_server_step(nasch_server s, int64_t *pending);
/* Rounds until every submitted request has finished (timeout_ms < 0: no limit). */
int nasch_server_drain(nasch_server s, int64_t timeout_ms);
/* Take up to cap finished requests' results (each is returned once). */
int nasch_server_poll(nasch_server s, nasch_request_result *out, int64_t cap, int64_t *n_out);
/* Copy a finished request's per-step statistics (cap_steps >= its steps) and,
 * with keep_state, its final state (cap_cars >= N): an agent road's cars in
 * their cyclic order, as nasch_read_state gives them; a grid road's cars in
 * increasing cell order.  Any output may be NULL. */
int nasch_server_result(nasch_server s, uint64_t request_id, uint64_t *sum_v_host, uint64_t *crossings_host,
                        int64_t cap_steps, int32_t *x_host, uint8_t *v_host, int64_t cap_cars);
/* Stream the per-step statistics of admitted requests as their steps finish:
 * copies, for each request with steps that the GPU has finished and that
 * were not returned before, those steps' sum_v and crossings into
 * sum_v_host / crossings_host (one chunk per request, in order, at most
 * cap_steps steps in all) and describes each chunk in chunks[0..*n_chunks).
 * A request's chunks come in step order and, put together, are its whole
 * series; the last one may come after the request has finished (poll it
 * with nasch_server_poll as usual, and call this before releasing it).
 * Either output array may be NULL; cap_chunks or cap_steps 0 returns
 * nothing.  Reads what finished ticks wrote, on a stream of its own, and
 * does not wait for running ticks. */
int nasch_server_poll_series(nasch_server s, nasch_series_chunk *chunks, int64_t cap_chunks, uint64_t *sum_v_host,
                             uint64_t *crossings_host, int64_t cap_steps, int64_t *n_chunks);
/* Forget a finished, polled request (frees its host copies). */
int nasch_server_release(nasch_server s, uint64_t request_id);
/* Cancel a queued or running request; it finishes with NASCH_ECANCELED. */
int nasch_server_cancel(nasch_server s, uint64_t request_id);
int nasch_server_get_info(nasch_server s, nasch_server_info *info);
/* Wait for all work, then free the server.  NULL is a no-op. */
void nasch_server_destroy(nasch_server s);

/* One rank's share of a ring road split into contiguous cell ranges (the
 * grid layout's 1-D domain decomposition; the paper's "Variations":
 * distributed memory).  The rank owns the `owned` cells first_cell ..
 * first_cell + owned - 1 (mod L) and holds them with `halo` cells on each
 * side: seg_in_dev[i] (caller-owned device memory, int8 cells, -1 empty) is
 * ring cell first_cell - halo + i (mod L) at global step step0, for i <
 * owned + 2 * halo.  Enqueues k steps (rules 1-4, the rule-3 draw keyed by
 * the ring cell as for the whole road) on `stream` (a cudaStream_t, NULL
 * for the default stream) and writes the owned cells at step step0 + k to
 * seg_out_dev[halo .. halo + owned - 1]; the halo parts of seg_out_dev are
 * not written (refresh both halos from the ring neighbours before the next
 * call).  Per step s < k, adds to sum_v_dev[s] and crossings_dev[s]
 * (caller-owned device uint64 arrays, zeroed by the caller) the velocities
 * and the crossings of the cars whose cell at the start of the step is
 * owned, so the ranks' series add up to the whole road's.  Cell j at step
 * t+1 depends only on cells j - vmax .. j + vmax at step t, so the result
 * is exact when k * vmax <= halo.  Requires: halo a multiple of 16 with
 * k * vmax <= halo <= 512; 1 <= k <= 64; 1 <= owned <= L; both buffers
 * 16-byte aligned and not overlapping; anything else is NASCH_EINVAL. */
int nasch_segment_run(const int8_t *seg_in_dev, int8_t *seg_out_dev, int64_t owned, int32_t halo,
                      int64_t first_cell, int64_t L, int32_t vmax, double p, uint64_t seed, uint32_t road_id,
                      uint64_t step0, int32_t k, uint64_t *sum_v_dev, uint64_t *crossings_dev, void *stream);

/* Start positions of one road, computed on the GPU without allocating any
 * device memory.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory - a process whose device memory
 * is all owned by another allocator (a framework's caching pool, an arena set
 * up at start), or one that forbids allocation after start-up.
 * Writes the N sorted Floyd positions of (seed, road_id), the same as
 * nasch_floyd_init, into the caller's device buffer x_dev[0..N-1],
 * asynchronously on `stream` (a cudaStream_t, NULL for the default stream);
 * the caller synchronises before reading x_dev.  It calls no allocating
 * routine: its scratch bit map is a fixed 2 MiB array in the library's device
 * memory, held by every GPU that loads the library until the process exits,
 * so L is limited to 2^24 cells (a longer road is NASCH_EINVAL).  Every
 * call looks up that array's device address with the calling thread's
 * device current (the first call on a device also loads the library's
 * device code there); make that first call before any stream capture.  All calls share
 * the array and the bits of the previous call stay in it (each call clears
 * the part it uses first), so calls whose work overlaps on the GPU race and
 * give wrong positions: issue them on one stream, or synchronise between
 * them. */
int nasch_floyd_init_device_noalloc(int64_t L, int64_t N, uint64_t seed, uint32_t road_id, int32_t *x_dev,
                                    void *stream);

/* Calibration: the rate (draws per second) at which the GPU evaluates the
 * rule-3 draw, word 0 of Philox4x32-10, with nothing else to do - the
 * integer-pipe ceiling of the step, one draw per car-step.  Runs one
 * kernel of draws_per_thread draws per thread on a full grid and
 * synchronises; seconds (may be NULL) receives the kernel's duration. */
int nasch_calibrate_philox(int64_t draws_per_thread, double *draws_per_second, double *seconds);

/* Self-test of failure detection without a GPU fault: runs a kernel whose
 * bounded wait (on an mbarrier that nothing completes) gives up after
 * limit_ms (1..5000).  The kernel records the timeout in a status word and
 * returns, leaving the context usable; the call returns NASCH_ETIMEOUT with
 * that word in *status_out (may be NULL).  The same bounded waits guard the
 * asynchronous copies of the tiled grid kernel, whose timeouts surface as
 * NASCH_ETIMEOUT from the next call that synchronises the road. */
int nasch_selftest_bounded_wait(int64_t limit_ms, uint32_t *status_out);

#ifdef __cplusplus
}
#endif

#endif /* NASCH_H */
