// Grid NaSch step kernels: one int8 per cell, -1 empty, else the velocity of
// the car on it ("Concepts Covered": the grid representation; Handout,
// model section rules 1-4).
//
// Tiled kernels.  After one step a cell depends on the cells within vmax of
// it (a car arriving from behind, the gap of that car ahead), so a tile
// staged with a halo of H >= k * vmax cells on each side is exact in its
// middle after k fused steps.  Staging is by 1-D bulk (TMA) copies into
// shared memory, completion counted on mbarriers whose waits are bounded
// (status word), and results leave by bulk stores.  Rule 2 makes every
// scatter collision-free.  The first and last tiles take their halo across
// the ring boundary (modular cell index, plain loads).
//  - grid_k1_kernel (k = 1, vmax <= 16): independent warps on 3040-cell
//    tiles stepped in place; a warp car list sorted by cell, padded to whole
//    groups of 32, gaps from the next entry.
//  - grid_warp_kernel (the rest with H = round_up(k vmax, 16) <= 512):
//    independent warps on 2048-cell spans; the span's cars become a sorted
//    list, the k steps run on the list (grid_warp_steps) and the cars of the
//    tile's own cells are scattered back.
//  - grid_tiled_kernel (H > 512): the same on 8192-cell spans by a whole
//    block.
// Statistics of the cars that start a step in a tile's own cells are
// reduced per warp (and block) and added to the per-step series.
//
// Ring kernel.  For L <= kGridRingMaxCells one block holds the whole ring
// in shared memory and runs any number of steps in one launch.
#include <atomic>

#include "road_output.h"
#include "tile_device.cuh"

namespace nasch {
namespace {

constexpr uint32_t kGridWarps = (uint32_t)kGridThreads / 32u;
constexpr int kMaxDevices = 64;
constexpr uint32_t kGridStages = 2;   // spans in flight per block: the current one and one prefetched
constexpr uint32_t kGridListCap = (uint32_t)kGridSpan;   // every span's cars fit the list

template <Draw D>
__global__ void __launch_bounds__(kGridThreads) grid_tiled_kernel(const GridStep g, const GridTileGeom geo)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t s_full[kGridStages];
    __shared__ unsigned long long s_sum[kMaxFusedSteps];
    __shared__ unsigned long long s_cross[kMaxFusedSteps];
    __shared__ uint32_t s_first[2 * kGridThreads];
    __shared__ uint32_t s_count[kGridWarps + 1];

    const RoadConst rc = g.rc;
    const uint32_t L = rc.L;
    const uint32_t H = geo.halo;
    const uint32_t C = geo.tile;
    const uint32_t W = (uint32_t)kGridSpan;
    const uint32_t WP = geo.padded;
    const uint32_t tid = threadIdx.x;
    int8_t *const pool = reinterpret_cast<int8_t *>(smem);
    // stages 0, 1 (bulk-load targets), outputs 2, 3 (alternating by tile),
    // then the car list: positions (uint16) and velocities
    auto buf = [&](uint32_t b) { return pool + b * WP; };
    uint16_t *const s_pos = reinterpret_cast<uint16_t *>(pool + 4u * WP);
    uint8_t *const s_vel = reinterpret_cast<uint8_t *>(s_pos + kGridListCap);

    for (int i = tid; i < g.ksteps; i += kGridThreads) {
        s_sum[i] = 0ull;
        s_cross[i] = 0ull;
    }
    if (tid == 0) {
        for (uint32_t b = 0; b < kGridStages; ++b) mbar_init(&s_full[b], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto bulk_ok = [&](uint32_t tile) {
        const uint32_t t0 = tile * C;
        return t0 >= H && t0 + C + H <= L;
    };
    uint32_t parity = 0;   // bit b: phase parity of s_full[b]
    uint32_t tile = blockIdx.x;
    if (tid == 0 && tile < geo.n_tiles && bulk_ok(tile)) {
        fence_proxy_async();
        mbar_expect_tx(&s_full[0], W);
        bulk_load(buf(0), g.c_in + (tile * C - H), W, &s_full[0]);
    }
    for (uint32_t it = 0; tile < geo.n_tiles; tile += gridDim.x, ++it) {
        const uint32_t sb = it & 1u;
        const uint32_t t0 = tile * C;
        const uint32_t own_cells = min(C, L - t0);
        const uint32_t base = t0 >= H ? t0 - H : t0 + L - H;   // road cell of buffer index 0
        const uint32_t next = tile + gridDim.x;
        if (tid == 0) {
            // earlier bulk stores must have read their source before buffers are reused
            bulk_wait_read_all();
            if (next < geo.n_tiles && bulk_ok(next)) {
                fence_proxy_async();
                mbar_expect_tx(&s_full[sb ^ 1u], W);
                bulk_load(buf(sb ^ 1u), g.c_in + (next * C - H), W, &s_full[sb ^ 1u]);
            }
        }
        int8_t *in = buf(sb);
        bool ok = true;
        if (bulk_ok(tile)) {
            // one thread waits for the span; the barrier below releases the
            // others (waiting warps would otherwise take issue slots)
            if (tid == 0) ok = mbar_wait_bounded(&s_full[sb], (parity >> sb) & 1u);
            parity ^= 1u << sb;
        } else {
            for (uint32_t i = tid; i < W; i += kGridThreads) {
                uint32_t cell = base + i;
                if (cell >= L) cell -= L;
                in[i] = g.c_in[cell];
            }
        }
        if (!__syncthreads_and(ok)) {
            if (tid == 0) {
                atomicOr(g.status, kStatusTimeout);
                if (next < geo.n_tiles && bulk_ok(next)) mbar_wait_bounded(&s_full[sb ^ 1u], (parity >> (sb ^ 1u)) & 1u);
                bulk_wait_all();
            }
            return;
        }
        int8_t *out = buf(2u + sb);
        grid_span_steps<D>(rc, in, out, H, own_cells, base, g.step0, g.ksteps, s_pos, s_vel, kGridListCap, s_first,
                           s_count, s_sum, s_cross);
        fence_proxy_async();   // the result leaves by bulk store
        __syncthreads();
        if (own_cells == C) {
            if (tid == 0) {
                bulk_store(g.c_out + t0, out + H, C);
                bulk_commit();
            }
        } else {
            for (uint32_t i = tid; i < own_cells; i += kGridThreads) g.c_out[t0 + i] = out[H + i];
        }
    }
    if (tid == 0) bulk_wait_all();
    __syncthreads();
    for (int i = tid; i < g.ksteps; i += kGridThreads) {
        if (s_sum[i]) atomicAdd(&g.sum_v[i], s_sum[i]);
        if (s_cross[i]) atomicAdd(&g.crossings[i], s_cross[i]);
    }
}

// k = 1 and vmax <= 16: the one-step kernel.  Every warp works alone (no
// block barrier after set-up) on tiles of kK1Cells cells: it stages the tile
// with 16 halo cells on each side (kK1Span cells, one bulk copy on the
// warp's own mbarrier), steps it in place, and writes the tile back by one
// bulk store.  Per tile:
//   1. each lane turns its 32 * kK1Words cells into occupancy bits and counts
//      its cars;
//   2. a warp prefix sum gives each lane its slots in the car list: the
//      span index of every car of the span in ascending order, followed by
//      dummy cars in the padding after the span, up to a multiple of 32
//      entries and one more;
//   3. the lanes take the list 32 cars at a time, three groups interleaved,
//      so every lane draws for the same number of cars; a car's leader is
//      the next list entry, so its gap is the difference of the two indices
//      less one.  Each car reads its velocity from its cell, empties the
//      cell and writes its new velocity at its new cell (in place): no other
//      car writes a car's cell in the same step, since the car behind stops
//      before it and every destination is an empty cell or the car's own.
// Only the cars the tile owns are counted in the statistics; the others
// (halo cars, the dummy) are stepped with the rest and their results fall
// outside the cells written back: a car in the left halo may move into the
// tile and is stepped exactly, a car in the right halo may lack its leader
// (beyond the span) but moves only further right.  The last owned car sees
// its leader, or the dummy at least vmax cells ahead.
// A tile with more cars than the list holds is listed and stepped in passes,
// in cell order and in place like the groups of one pass.  The warp's
// buffers form a ring (kK1Bufs = 2: the tile being stepped and the next
// tile), and a tile's copy is issued once the tile that last used its buffer
// has been read by its store.  The rule-3 draw uses the counter-independent
// parts of Philox computed on the host (SlowdownKey).
// Open (an open road, cells 0..L-1): cells off the road read as empty, a
// closed exit is a car standing on cell L (seen by the car behind it, never
// written back), cars that pass cell L - 1 leave and are counted as
// crossings, and after the step a car enters cell 0 at rest if `entry` and
// the cell is empty.  The host decides the exit and the entry of the step.
constexpr uint32_t kK1Words = 3;                         // occupancy words (32 cells each) per lane
constexpr uint32_t kK1Halo = 16;                         // cells staged on each side: vmax <= 16
constexpr uint32_t kK1Span = 1024u * kK1Words;           // staged cells
constexpr uint32_t kK1Cells = kK1Span - 2u * kK1Halo;    // cells written per warp-tile
constexpr uint32_t kK1Buf = kK1Span + 32u;               // + padding: the dummy car's and halo cars' moves
constexpr uint32_t kK1ListCap = 112u * kK1Words / 32u * 32u;   // cars per pass; a denser tile is done in passes
constexpr uint32_t kK1ListLen = kK1ListCap + 32u;        // + padding to whole groups and one leader
constexpr uint32_t kK1Dummy = kK1Span;                   // span index of the dummy cars (padding)
constexpr uint32_t kK1Bufs = 2;                          // buffers per warp: the tile stepped and the copy ahead (a third buffer costs more in resident warps than it gains)
constexpr int8_t kEmptyCell = -1;
constexpr int kK1Warps = 4;                              // warps per block
static_assert(kK1ListCap % 32u == 0u, "whole groups");

struct __align__(16) K1WarpSmem {
    int8_t buf[kK1Bufs][kK1Buf];
    uint16_t list[kK1ListLen];    // span index of each listed car
    uint64_t full[kK1Bufs];       // bulk-copy completion, one per buffer
};

// G groups of 32 listed cars (list: the first group's entries), rules 1-4,
// with the draws of the G groups interleaved.  A car's entry is its span
// index and its leader is the next entry; its velocity is read from `span`
// and its result written to `out` (the same buffer when stepping in place).
// W: the span holds cell L - 1, so cells wrap and crossings are possible
// (warp-uniform; on a ring false on every tile but the first and the last).
// The statistics take the cars on the tile's own cells.
template <int G, Draw D, bool W>
__device__ __forceinline__ void k1_groups(const uint16_t *list, uint32_t lane, const int8_t *span, int8_t *out,
                                          uint32_t base, uint32_t L, uint32_t vmax, uint32_t thr,
                                          const SlowdownKey &sk, uint32_t own, uint32_t &tsum, uint32_t &tcross)
{
    uint32_t rr[G], lead[G], v0[G];
#pragma unroll
    for (int q = 0; q < G; ++q) {
        rr[q] = list[32 * q + lane];
        lead[q] = list[32 * q + lane + 1];
    }
#pragma unroll
    for (int q = 0; q < G; ++q) v0[q] = (uint8_t)span[rr[q]];   // every read before any write of the groups
#pragma unroll
    for (int q = 0; q < G; ++q) {
        const uint32_t r = rr[q];
        const uint32_t gap = lead[q] - r - 1u;                                            // empty cells ahead
        uint32_t vel = min(min(v0[q] + 1u, vmax), gap);                                   // rules 1, 2
        uint32_t cell = base + r;
        if (W && cell >= L) cell -= L;
        if (D == Draw::kAlways) {
            vel -= vel != 0u ? 1u : 0u;                                                    // rule 3, p = 1
        } else if (D == Draw::kPhilox) {
            const uint32_t u = slowdown_word0(cell, sk);
            vel -= (vel != 0u && u < thr) ? 1u : 0u;                                       // rule 3
        }
        out[r] = kEmptyCell;                                                              // rule 4
        if (NASCH_DCHECK(r + vel < kK1Buf, kDbgGridWrite)) out[r + vel] = (int8_t)vel;
        const bool mine = r - kK1Halo < own;
        tsum += mine ? vel : 0u;
        if (W) tcross += (mine && cell + vel >= L) ? 1u : 0u;
    }
}

// All `padded` listed cars (a multiple of 32), three groups at a time.
template <Draw D, bool W>
__device__ __forceinline__ void k1_cars(const uint16_t *list, uint32_t padded, uint32_t lane, const int8_t *span,
                                        int8_t *out, uint32_t base, uint32_t L, uint32_t vmax, uint32_t thr,
                                        const SlowdownKey &sk, uint32_t own, uint32_t &tsum, uint32_t &tcross)
{
    uint32_t gi = 0;
    for (; gi + 96u <= padded; gi += 96u)
        k1_groups<3, D, W>(list + gi, lane, span, out, base, L, vmax, thr, sk, own, tsum, tcross);
    if (padded - gi == 64u)
        k1_groups<2, D, W>(list + gi, lane, span, out, base, L, vmax, thr, sk, own, tsum, tcross);
    else if (padded - gi == 32u)
        k1_groups<1, D, W>(list + gi, lane, span, out, base, L, vmax, thr, sk, own, tsum, tcross);
}

template <Draw D, bool Open>
__global__ void __launch_bounds__(32 * kK1Warps) grid_k1_kernel(const GridStep g, const uint32_t n_tiles,
                                                                const SlowdownKey sk, const int exit_open,
                                                                const int entry)
{
    __shared__ K1WarpSmem s_w[kK1Warps];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    K1WarpSmem &w = s_w[warp];
    const uint32_t L = g.rc.L, vmax = g.rc.vmax, thr = (uint32_t)g.rc.thr;
    const uint32_t nw = gridDim.x * (uint32_t)kK1Warps;

    if (lane == 0) {
        for (uint32_t b = 0; b < kK1Bufs; ++b) mbar_init(&w.full[b], 1);
        fence_mbar_init();
    }
    for (uint32_t b = 0; b < kK1Bufs; ++b) w.buf[b][kK1Span + lane] = kEmptyCell;   // the dummies' cells
    __syncthreads();

    auto bulk_ok = [&](uint32_t t) {
        const uint32_t t0 = t * kK1Cells;
        return t0 >= kK1Halo && t0 + kK1Cells + kK1Halo <= L;
    };
    auto issue_load = [&](uint32_t t, uint32_t b) {   // lane 0
        fence_proxy_async();
        mbar_expect_tx(&w.full[b], kK1Span);
        bulk_load(w.buf[b], g.c_in + (t * kK1Cells - kK1Halo), kK1Span, &w.full[b]);
    };
    uint32_t tile = blockIdx.x * (uint32_t)kK1Warps + warp;
    // the ring of buffers: this warp's n-th tile goes to buffer n mod kK1Bufs,
    // and the copies of the next kK1Bufs - 1 tiles are in flight while a tile
    // is stepped
    uint32_t pending = 0;                // lane 0: bit b, a copy into buffer b not yet waited for
    if (lane == 0)
        for (uint32_t b = 0; b + 1u < kK1Bufs; ++b) {
            const uint32_t t = tile + b * nw;
            if (t < n_tiles && bulk_ok(t)) {
                issue_load(t, b);
                pending |= 1u << b;
            }
        }
    uint32_t parity = 0;                 // bit b: phase parity of full[b]
    uint32_t bi = 0;                     // buffer of the tile being stepped
    uint32_t tsum = 0, tcross = 0;       // statistics of this lane's cars
    for (; tile < n_tiles; tile += nw) {
        const uint32_t bp = bi == 0u ? kK1Bufs - 1u : bi - 1u;   // the tile before's buffer: the copy ahead goes there
        int8_t *span = w.buf[bi];
        const uint32_t t0 = tile * kK1Cells;
        const uint32_t own = min(kK1Cells, L - t0);
        // road cell of span index 0 (an open road: modulo 2^32, before the road on tile 0)
        const uint32_t base = Open ? t0 - kK1Halo : (t0 >= kK1Halo ? t0 - kK1Halo : t0 + L - kK1Halo);
        bool ok = true;
        if (bulk_ok(tile)) {
            if (lane == 0) {
                ok = mbar_wait_bounded(&w.full[bi], (parity >> bi) & 1u);
                if (ok) pending &= ~(1u << bi);
            }
            parity ^= 1u << bi;
        } else {
            for (uint32_t i = lane; i < kK1Span; i += 32u) {
                uint32_t c = base + i;
                if (Open) {
                    span[i] = c < L ? g.c_in[c] : kEmptyCell;
                } else {
                    if (c >= L) c -= L;
                    span[i] = g.c_in[c];
                }
            }
            if (Open && !exit_open) {   // a closed exit: a car on cell L, if the span holds it
                __syncwarp();
                const uint32_t e = L - base;
                if (lane == 0 && e < kK1Span) span[e] = 0;
            }
        }
        if (!__all_sync(0xFFFFFFFFu, ok)) {
            if (lane == 0) {
                atomicOr(g.status, kStatusTimeout);
                // let the other copies in flight land (bounded) before the block's memory is released
                for (uint32_t b = 0; b < kK1Bufs; ++b)
                    if (b != bi && (pending >> b & 1u)) mbar_wait_bounded(&w.full[b], (parity >> b) & 1u);
                bulk_wait_all();
            }
            break;
        }
        __syncwarp();   // lane 0's completed wait (or the lanes' plain loads) before any lane reads the span
        // 1. this lane's cars: occupancy of its 32 * kK1Words cells
        const uint32_t c0 = 32u * kK1Words * lane;
        const uint4 *q = reinterpret_cast<const uint4 *>(span + c0);
        uint32_t m[kK1Words];
        uint32_t n = 0;
#pragma unroll
        for (uint32_t j = 0; j < kK1Words; ++j) {
            m[j] = occupancy16(q[2u * j]) | (occupancy16(q[2u * j + 1u]) << 16);
            n += __popc(m[j]);
        }
        // 2. list slots
        uint32_t incl = n;
#pragma unroll
        for (uint32_t d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
            if (lane >= d) incl += t;
        }
        const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        const bool wraps = base + kK1Buf > L;   // the span holds cell L - 1: crossings possible
        // a tile with more cars than the list holds is listed and stepped in
        // passes (in cell order, in place: a pass's cars read only their own
        // cells, which no car of an earlier pass writes)
        const bool dense = total > kK1ListCap;   // warp-uniform
        for (uint32_t chunk = 0; chunk == 0u || chunk < total; chunk += kK1ListCap) {
            const uint32_t count = total > chunk ? min(kK1ListCap, total - chunk) : 0u;
            const uint32_t padded = (count + 31u) & ~31u;
            uint32_t pos = incl - n;
            if (!dense) {
#pragma unroll
                for (uint32_t j = 0; j < kK1Words; ++j)
                    for (uint32_t mm = m[j]; mm; mm &= mm - 1u)
                        w.list[pos++] = (uint16_t)(c0 + 32u * j + __clz(__brev(mm)));
            } else {   // ranks chunk .. chunk + count (the last one: the pass's leader entry)
#pragma unroll
                for (uint32_t j = 0; j < kK1Words; ++j)
                    for (uint32_t mm = m[j]; mm; mm &= mm - 1u, ++pos)
                        if (pos - chunk <= count) w.list[pos - chunk] = (uint16_t)(c0 + 32u * j + __clz(__brev(mm)));
            }
            // dummies after the last car, and the leader of the last group
            // (a pass before the last is a whole number of groups, its leader entry a car)
            if (chunk + count == total && lane <= padded - count) w.list[count + lane] = (uint16_t)kK1Dummy;
            __syncwarp();
            if (chunk == 0u && lane == 0) {
                // the copy kK1Bufs - 1 tiles ahead, into the tile before's
                // buffer once its store has read it
                bulk_wait_read_all();
                const uint32_t nx = tile + (kK1Bufs - 1u) * nw;
                if (nx < n_tiles && bulk_ok(nx)) {
                    issue_load(nx, bp);
                    pending |= 1u << bp;
                }
            }
            // 3. the cars, 32 at a time, three groups interleaved
            if (wraps)
                k1_cars<D, true>(w.list, padded, lane, span, span, base, L, vmax, thr, sk, own, tsum, tcross);
            else
                k1_cars<D, false>(w.list, padded, lane, span, span, base, L, vmax, thr, sk, own, tsum, tcross);
            __syncwarp();   // the list is rewritten by the next pass
        }
        if (Open && entry && tile == 0) {   // a car enters cell 0 at rest
            __syncwarp();
            if (lane == 0 && span[kK1Halo] < 0) span[kK1Halo] = 0;
        }
        // 4. the result leaves by bulk store (or plain stores for a short last tile)
        fence_proxy_async();
        __syncwarp();
        if (own == kK1Cells) {
            if (lane == 0) {
                bulk_store(g.c_out + t0, span + kK1Halo, kK1Cells);
                bulk_commit();
            }
        } else {
            for (uint32_t i = lane; i < own; i += 32u) g.c_out[t0 + i] = span[kK1Halo + i];
        }
        bi = bi + 1u == kK1Bufs ? 0u : bi + 1u;
    }
    if (lane == 0) bulk_wait_all();
    unsigned long long acc_sum = tsum, acc_cross = tcross;
    for (uint32_t d = 16; d >= 1; d >>= 1) {
        acc_sum += __shfl_xor_sync(0xFFFFFFFFu, acc_sum, d);
        acc_cross += __shfl_xor_sync(0xFFFFFFFFu, acc_cross, d);
    }
    if (lane == 0) {
        if (acc_sum) atomicAdd(&g.sum_v[0], acc_sum);
        if (acc_cross) atomicAdd(&g.crossings[0], acc_cross);
    }
}

// k >= 2 with k * vmax <= 512: the fused warp kernel.  Every warp works alone
// (no block barrier after set-up) on tiles of kKwSpan - 2H cells, H =
// round_up(k * vmax, 16): it stages the tile with its halos by one bulk copy
// on its own mbarrier, runs the k steps by the list method
// (grid_warp_steps), and writes the tile back by one bulk store.  Two
// buffers per warp alternate: the next tile's copy is issued as soon as the
// list is built, once the store of the tile before has read its buffer.
constexpr int kKwWarps = 4;                             // warps per block

struct __align__(16) KwWarpSmem {
    int8_t buf[2][kKwBuf];
    uint16_t pos[kKwListSmem];    // the list of a span whose cars fit; denser spans use global scratch
    uint8_t vel[kKwListSmem];
    uint32_t sum[kMaxFusedSteps];     // statistics of the warp's tiles, by step
    uint32_t cross[kMaxFusedSteps];
    uint64_t full[2];
};

template <Draw D>
__global__ void __launch_bounds__(32 * kKwWarps) grid_warp_kernel(const GridStep g, const uint32_t H,
                                                                  const uint32_t n_tiles, const SlowdownKey sk)
{
    __shared__ KwWarpSmem s_w[kKwWarps];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    KwWarpSmem &w = s_w[warp];
    const uint32_t L = g.rc.L;
    const uint32_t C = kKwSpan - 2u * H;                  // cells written per tile
    const uint32_t nw = gridDim.x * (uint32_t)kKwWarps;
    const int ksteps = g.ksteps;

    if (lane == 0) {
        for (uint32_t b = 0; b < 2u; ++b) mbar_init(&w.full[b], 1);
        fence_mbar_init();
    }
    for (uint32_t s = lane; s < (uint32_t)kMaxFusedSteps; s += 32u) w.sum[s] = w.cross[s] = 0u;
    __syncthreads();

    auto bulk_ok = [&](uint32_t t) {
        const uint32_t t0 = t * C;
        return t0 >= H && t0 + C + H <= L;
    };
    auto issue_load = [&](uint32_t t, uint32_t b) {   // lane 0
        fence_proxy_async();
        mbar_expect_tx(&w.full[b], kKwSpan);
        bulk_load(w.buf[b], g.c_in + (t * C - H), kKwSpan, &w.full[b]);
    };
    uint32_t tile = blockIdx.x * (uint32_t)kKwWarps + warp;
    if (lane == 0 && tile < n_tiles && bulk_ok(tile)) issue_load(tile, 0);
    uint32_t parity = 0, bi = 0;
    for (; tile < n_tiles; tile += nw) {
        const uint32_t bn = bi ^ 1u;
        int8_t *span = w.buf[bi];
        const uint32_t t0 = tile * C;
        const uint32_t own = min(C, L - t0);
        const uint32_t base = t0 >= H ? t0 - H : t0 + L - H;   // road cell of span index 0
        bool ok = true;
        if (bulk_ok(tile)) {
            if (lane == 0) ok = mbar_wait_bounded(&w.full[bi], (parity >> bi) & 1u);
            parity ^= 1u << bi;
        } else {
            for (uint32_t i = lane; i < kKwSpan; i += 32u) {
                uint32_t c = base + i;
                if (c >= L) c -= L;
                span[i] = g.c_in[c];
            }
        }
        if (!__all_sync(0xFFFFFFFFu, ok)) {
            if (lane == 0) {
                atomicOr(g.status, kStatusTimeout);
                bulk_wait_all();
            }
            break;
        }
        __syncwarp();
        uint8_t *big = g.list_scratch + (size_t)(blockIdx.x * (uint32_t)kKwWarps + warp) * (3u * kKwList);
        grid_warp_steps<D>(
            g.rc, FoldedDraws{sk, {}}, span,
            WarpList{w.pos, w.vel, kKwListSmem, reinterpret_cast<uint16_t *>(big), big + 2u * kKwList}, H, own,
            base, g.step0, ksteps,
            [&]() {   // the next tile goes into the other buffer once the store of the tile before has read it
                if (lane == 0) {
                    bulk_wait_read_all();
                    const uint32_t nx = tile + nw;
                    if (nx < n_tiles && bulk_ok(nx)) issue_load(nx, bn);
                }
            },
            [&](int s, uint32_t sum, uint32_t cross) {
                w.sum[s] += sum;
                w.cross[s] += cross;
            });
        fence_proxy_async();
        __syncwarp();
        if (own == C) {
            if (lane == 0) {
                bulk_store(g.c_out + t0, span + H, C);
                bulk_commit();
            }
        } else {
            for (uint32_t i = lane; i < own; i += 32u) g.c_out[t0 + i] = span[H + i];
        }
        bi = bn;
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
    for (uint32_t s = lane; s < (uint32_t)ksteps; s += 32u) {
        if (w.sum[s]) atomicAdd(&g.sum_v[s], (unsigned long long)w.sum[s]);
        if (w.cross[s]) atomicAdd(&g.crossings[s], (unsigned long long)w.cross[s]);
    }
}

// Whole ring in one block (L <= kGridRingMaxCells).
__global__ void __launch_bounds__(1024) grid_ring_kernel(const GridStep g)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t s_psum[32];
    __shared__ uint32_t s_pcross[32];
    int8_t *cur = reinterpret_cast<int8_t *>(smem);
    int8_t *nxt = cur + ((g.rc.L + 15u) / 16u) * 16u;
    grid_ring_steps(g.c_in, g.c_out, g.rc, g.step0, g.ksteps, cur, nxt, g.sum_v, g.crossings, s_psum, s_pcross);
}

GridTileGeom make_geom(int ksteps, uint32_t vmax, uint32_t L)
{
    GridTileGeom geo;
    geo.halo = grid_halo(ksteps, vmax);
    geo.tile = (uint32_t)kGridSpan - 2u * geo.halo;
    geo.padded = (uint32_t)kGridSpan;   // the span method never reads or writes past the span
    geo.n_tiles = (L + geo.tile - 1u) / geo.tile;
    geo.nwork = 2;
    return geo;
}

// two stages, two outputs, and the car list (uint16 position + uint8 velocity)
size_t grid_tiled_smem(const GridTileGeom &geo) { return 4u * (size_t)geo.padded + 3u * (size_t)kGridListCap; }

template <Draw D, bool Open>
cudaError_t launch_k1_variant(const GridStep &g, uint32_t n_tiles, cudaStream_t s, bool exit_open = false,
                              bool entry = false)
{
    // blocks per SM from the occupancy calculator, once per device
    static std::atomic<int> per_sm[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    int n = per_sm[dev].load();
    if (n == 0) {
        int sms = 0, b = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, grid_k1_kernel<D, Open>, 32 * kK1Warps, 0);
        if (e != cudaSuccess) return e;
        n = sms * (b > 0 ? b : 1);
        per_sm[dev].store(n);
    }
    const uint32_t need = (n_tiles + (uint32_t)kK1Warps - 1u) / (uint32_t)kK1Warps;
    const int grid = (int)((uint32_t)n < need ? (uint32_t)n : need);
    const SlowdownKey sk = make_slowdown_key(g.step0, g.rc.road, g.rc.key0, g.rc.key1);
    grid_k1_kernel<D, Open><<<grid, 32 * kK1Warps, 0, s>>>(g, n_tiles, sk, exit_open ? 1 : 0, entry ? 1 : 0);
    return cudaGetLastError();
}

template <Draw D>
cudaError_t launch_kw_variant(const GridStep &g, uint32_t H, uint32_t n_tiles, cudaStream_t s)
{
    static std::atomic<int> per_sm[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    int n = per_sm[dev].load();
    if (n == 0) {
        int sms = 0, b = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, grid_warp_kernel<D>, 32 * kKwWarps, 0);
        if (e != cudaSuccess) return e;
        n = sms * (b > 0 ? b : 1);
        per_sm[dev].store(n);
    }
    const uint32_t need = (n_tiles + (uint32_t)kKwWarps - 1u) / (uint32_t)kKwWarps;
    const int grid = (int)((uint32_t)n < need ? (uint32_t)n : need);
    const SlowdownKey sk = make_slowdown_key(g.step0, g.rc.road, g.rc.key0, g.rc.key1);
    grid_warp_kernel<D><<<grid, 32 * kKwWarps, 0, s>>>(g, H, n_tiles, sk);
    return cudaGetLastError();
}

// Static plus dynamic shared memory exceeds the default 48 KB, so the
// dynamic size is allowed explicitly (a per-device function attribute).
template <Draw D>
cudaError_t launch_grid_variant(const GridStep &g, const GridTileGeom &geo, int grid, size_t smem, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(grid_tiled_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    grid_tiled_kernel<D><<<grid, kGridThreads, smem, s>>>(g, geo);
    return cudaGetLastError();
}

}  // namespace

size_t grid_list_scratch_bytes()
{
    int dev = 0, sms = 0, most = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, grid_warp_kernel<Draw::kNever>, 32 * kKwWarps, 0) != cudaSuccess)
        return 0;
    most = b;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, grid_warp_kernel<Draw::kAlways>, 32 * kKwWarps, 0) != cudaSuccess)
        return 0;
    most = b > most ? b : most;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, grid_warp_kernel<Draw::kPhilox>, 32 * kKwWarps, 0) != cudaSuccess)
        return 0;
    most = b > most ? b : most;
    return (size_t)sms * (size_t)(most > 0 ? most : 1) * (size_t)kKwWarps * 3u * (size_t)kKwList;
}

int grid_tiled_blocks_per_sm()
{
    const GridTileGeom geo = make_geom(1, 5, 1u << 20);
    const size_t smem = grid_tiled_smem(geo);
    if (cudaFuncSetAttribute(grid_tiled_kernel<Draw::kPhilox>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, grid_tiled_kernel<Draw::kPhilox>, kGridThreads, smem) !=
        cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_grid_tiled(const GridStep &g, int blocks, cudaStream_t s)
{
    if (g.ksteps <= 0) return cudaSuccess;
    if (g.ksteps > kMaxFusedSteps || g.rc.vmax > 127u) return cudaErrorInvalidValue;
    const GridTileGeom geo = make_geom(g.ksteps, g.rc.vmax, g.rc.L);
    // the tile must own cells, and the staged span must not wrap the ring twice
    if (2u * geo.halo >= (uint32_t)kGridSpan || g.rc.L < (uint32_t)kGridSpan) return cudaErrorInvalidValue;
    if (g.ksteps == 1 && g.rc.vmax <= 16u) {
        const uint32_t n_tiles = (g.rc.L + kK1Cells - 1u) / kK1Cells;
        if (g.rc.thr == 0) return launch_k1_variant<Draw::kNever, false>(g, n_tiles, s);
        if (g.rc.thr > 0xFFFFFFFFull) return launch_k1_variant<Draw::kAlways, false>(g, n_tiles, s);
        return launch_k1_variant<Draw::kPhilox, false>(g, n_tiles, s);
    }
    if (geo.halo <= kKwMaxHalo) {
        if (!g.list_scratch) return cudaErrorInvalidValue;   // dense spans need it
        const uint32_t n_tiles = (g.rc.L + (kKwSpan - 2u * geo.halo) - 1u) / (kKwSpan - 2u * geo.halo);
        if (g.rc.thr == 0) return launch_kw_variant<Draw::kNever>(g, geo.halo, n_tiles, s);
        if (g.rc.thr > 0xFFFFFFFFull) return launch_kw_variant<Draw::kAlways>(g, geo.halo, n_tiles, s);
        return launch_kw_variant<Draw::kPhilox>(g, geo.halo, n_tiles, s);
    }
    const size_t smem = grid_tiled_smem(geo);
    const int grid = (int)((uint32_t)blocks < geo.n_tiles ? (uint32_t)blocks : geo.n_tiles);
    if (g.rc.thr == 0) return launch_grid_variant<Draw::kNever>(g, geo, grid, smem, s);
    if (g.rc.thr > 0xFFFFFFFFull) return launch_grid_variant<Draw::kAlways>(g, geo, grid, smem, s);
    return launch_grid_variant<Draw::kPhilox>(g, geo, grid, smem, s);
}

cudaError_t launch_grid_k1_open(const GridStep &g, bool exit_open, bool entry, cudaStream_t s)
{
    if (g.ksteps != 1 || g.rc.vmax > kK1Halo || g.rc.L == 0) return cudaErrorInvalidValue;
    const uint32_t n_tiles = (g.rc.L + kK1Cells - 1u) / kK1Cells;
    if (g.rc.thr == 0) return launch_k1_variant<Draw::kNever, true>(g, n_tiles, s, exit_open, entry);
    if (g.rc.thr > 0xFFFFFFFFull) return launch_k1_variant<Draw::kAlways, true>(g, n_tiles, s, exit_open, entry);
    return launch_k1_variant<Draw::kPhilox, true>(g, n_tiles, s, exit_open, entry);
}

cudaError_t launch_grid_ring(const GridStep &g, cudaStream_t s)
{
    if (g.ksteps <= 0) return cudaSuccess;
    if (g.rc.L == 0 || g.rc.L > (uint32_t)kGridRingMaxCells) return cudaErrorInvalidValue;
    const size_t smem = 2u * (((size_t)g.rc.L + 15u) / 16u * 16u);
    if (smem > 48u * 1024u) {
        cudaError_t e = cudaFuncSetAttribute(grid_ring_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    uint32_t threads = (g.rc.L + 31u) / 32u * 32u;
    if (threads > 1024u) threads = 1024u;
    grid_ring_kernel<<<1, threads, smem, s>>>(g);
    return cudaGetLastError();
}

// This unit's debug word (zero in release builds).
NASCH_DEBUG_READER(debug_word_grid)

}  // namespace nasch
