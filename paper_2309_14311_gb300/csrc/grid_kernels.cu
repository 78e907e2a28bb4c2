// Grid NaSch step kernels: one int8 per cell, -1 empty, else the velocity of
// the car on it ("Concepts Covered": the grid representation; Handout,
// model section rules 1-4).
//
// Tiled kernel.  A span of kGridSpan = 8192 cells is staged in shared
// memory: the tile's own C = 8192 - 2H cells and a halo of H =
// round_up(k * vmax, 16) cells on each side.  After one step a cell depends
// on the cells within vmax of it (a car arriving from behind, the gap of
// that car ahead), so after k fused steps the middle C cells are exact.
// Persistent blocks walk the tiles; each span arrives by one bulk (TMA)
// copy issued while the previous tile computes, completion counted on an
// mbarrier, and the tile leaves by one bulk store.  Per step each of the 8
// warps takes one 1024-cell row: lanes turn their 32 cells into an
// occupancy bit mask, the warp compacts the row's cars into a list so the
// draws are spread evenly over the lanes, each car's gap comes from
// find-first-set on the masks of the cells ahead, and the car is scattered
// into the next buffer, which was cleared to -1 one step earlier (rotating
// buffers, one barrier per step).  Rule 2 makes the scatter collision-free.
// Statistics of the cars that start the step in the tile's own cells are
// reduced per warp, per block, and added to the per-step series once per
// block.  The first and last tiles take their halo across the ring boundary
// (modular cell index, plain loads).
//
// Ring kernel.  For L <= kGridRingMaxCells one block holds the whole ring
// in shared memory and runs any number of steps in one launch.
#include "tile_device.cuh"

namespace nasch {
namespace {

constexpr uint32_t kGridWarps = (uint32_t)kGridThreads / 32u;
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

// k = 1: the mask-step kernel.  One step per tile does not repay turning the
// span into a list, so each warp steps its 1024-cell row directly from the
// occupancy masks (grid_step): two staged spans, two work buffers rotating
// with the stage, car lists of up to 512 entries per warp.
constexpr uint32_t kMaskStages = 2;
constexpr uint32_t kMaskListCap = 512;

template <Draw D, bool kWide>
__global__ void __launch_bounds__(kGridThreads) grid_mask_kernel(const GridStep g, const GridTileGeom geo)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t s_full[kMaskStages];
    __shared__ unsigned long long s_sum[kMaxFusedSteps];
    __shared__ unsigned long long s_cross[kMaxFusedSteps];
    __shared__ uint16_t s_list[kGridWarps][kMaskListCap];

    const RoadConst rc = g.rc;
    const uint32_t L = rc.L;
    const uint32_t H = geo.halo;
    const uint32_t C = geo.tile;
    const uint32_t W = (uint32_t)kGridSpan;
    const uint32_t WP = geo.padded;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    int8_t *const pool = reinterpret_cast<int8_t *>(smem);
    // five buffers: stages 0..2 (bulk-load targets), work 3, work 4.  A tile's
    // steps rotate over (its stage, work a, work b): the stage is free once
    // step 0 has read it, until it is refilled for the tile three ahead.
    auto buf = [&](uint32_t b) { return pool + b * WP; };

    for (int i = tid; i < g.ksteps; i += kGridThreads) {
        s_sum[i] = 0ull;
        s_cross[i] = 0ull;
    }
    if (tid == 0) {
        for (uint32_t b = 0; b < kMaskStages; ++b) mbar_init(&s_full[b], 1);
        fence_mbar_init();
    }
    // stage padding (never written by the loads) and both work buffers start empty
    for (uint32_t b = 0; b < kMaskStages; ++b)
        for (uint32_t c = W / 16u + tid; c < WP / 16u; c += kGridThreads) reinterpret_cast<uint4 *>(buf(b))[c] = kEmpty4;
    for (uint32_t c = tid; c < 2u * WP / 16u; c += kGridThreads)
        reinterpret_cast<uint4 *>(buf(kMaskStages))[c] = kEmpty4;
    __syncthreads();

    auto bulk_ok = [&](uint32_t tile) {
        const uint32_t t0 = tile * C;
        return t0 >= H && t0 + C + H <= L;
    };
    uint32_t parity = 0;                  // bit b: phase parity of s_full[b]
    int clean = (int)kMaskStages;         // a work buffer known to be all -1, or -1 if none
    uint32_t tile = blockIdx.x;
    if (tid == 0) {
        // the first two spans of this block
        for (uint32_t b = 0; b + 1 < kMaskStages; ++b) {
            const uint32_t t = tile + b * gridDim.x;
            if (t < geo.n_tiles && bulk_ok(t)) {
                fence_proxy_async();
                mbar_expect_tx(&s_full[b], W);
                bulk_load(buf(b), g.c_in + (t * C - H), W, &s_full[b]);
            }
        }
    }
    for (uint32_t it = 0; tile < geo.n_tiles; tile += gridDim.x, ++it) {
        const uint32_t sb = it % kMaskStages;
        const uint32_t t0 = tile * C;
        const uint32_t own_cells = min(C, L - t0);
        const uint32_t base = t0 >= H ? t0 - H : t0 + L - H;   // road cell of buffer index 0
        const uint32_t ahead = tile + (kMaskStages - 1u) * gridDim.x;
        const uint32_t ab = (it + kMaskStages - 1u) % kMaskStages;   // its stage: the one tile it-1 used
        if (tid == 0) {
            // earlier bulk stores must have read their source before buffers are reused
            bulk_wait_read_all();
            if (ahead < geo.n_tiles && bulk_ok(ahead)) {
                fence_proxy_async();
                mbar_expect_tx(&s_full[ab], W);
                bulk_load(buf(ab), g.c_in + (ahead * C - H), W, &s_full[ab]);
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
                // let the loads still in flight land before the block's memory goes
                for (uint32_t d = 1; d < kMaskStages; ++d) {
                    const uint32_t t = tile + d * gridDim.x, b = (it + d) % kMaskStages;
                    if (t < geo.n_tiles && bulk_ok(t)) mbar_wait_bounded(&s_full[b], (parity >> b) & 1u);
                }
                bulk_wait_all();
            }
            return;
        }
        // rotation (stage, wa, wb); step 0 writes wa, which must be empty
        const uint32_t wa = clean >= 0 ? (uint32_t)clean : kMaskStages;
        const uint32_t wb = wa == kMaskStages ? kMaskStages + 1u : kMaskStages;
        if (clean < 0) {
            for (uint32_t c = tid; c < WP / 16u; c += kGridThreads) reinterpret_cast<uint4 *>(buf(wa))[c] = kEmpty4;
            __syncthreads();
        }
        // buffer at rotation position i (selected arithmetically: no local array)
        auto rot = [&](uint32_t i) { return i == 0u ? sb : (i == 1u ? wa : wb); };
        for (int s = 0; s < g.ksteps; ++s) {
            const uint32_t i0 = (uint32_t)s % 3u;
            const uint32_t i1 = i0 == 2u ? 0u : i0 + 1u;
            const uint32_t i2 = i1 == 2u ? 0u : i1 + 1u;
            uint32_t tsum = 0, tcross = 0;
            grid_step<D, kWide, kGridCellsPerLane, kMaskListCap>(rc, buf(rot(i0)), buf(rot(i1)), buf(rot(i2)), geo,
                                                                 own_cells, base, g.step0 + (uint32_t)s, s_list[warp],
                                                                 tsum, tcross);
            tsum = __reduce_add_sync(0xFFFFFFFFu, tsum);
            tcross = __reduce_add_sync(0xFFFFFFFFu, tcross);
            if (lane == 0 && (tsum | tcross)) {
                atomicAdd(&s_sum[s], (unsigned long long)tsum);
                atomicAdd(&s_cross[s], (unsigned long long)tcross);
            }
            // the result may leave by bulk store, and a cleared stage may be
            // refilled by a bulk load
            if (s + 1 == g.ksteps) fence_proxy_async();
            __syncthreads();
        }
        const uint32_t k3 = (uint32_t)g.ksteps % 3u;
        const int8_t *fin = buf(rot(k3));
        const uint32_t cleared = rot(k3 == 2u ? 0u : k3 + 1u);   // cleared during the last step
        clean = cleared >= kMaskStages ? (int)cleared : -1;

        if (own_cells == C) {
            if (tid == 0) {
                bulk_store(g.c_out + t0, fin + H, C);
                bulk_commit();
            }
        } else {
            for (uint32_t i = tid; i < own_cells; i += kGridThreads) g.c_out[t0 + i] = fin[H + i];
            // the next tile may clear or scatter into this buffer
            __syncthreads();
        }
    }
    if (tid == 0) bulk_wait_all();
    __syncthreads();
    for (int i = tid; i < g.ksteps; i += kGridThreads) {
        if (s_sum[i]) atomicAdd(&g.sum_v[i], s_sum[i]);
        if (s_cross[i]) atomicAdd(&g.crossings[i], s_cross[i]);
    }
}

// k = 1 and vmax <= 16: the one-step kernel.  A span is the tile's C =
// 8192 - 2H owned cells with H = 16 halo cells on each side (H = 0 when
// vmax = 0).  Per tile:
//   1. each thread turns its 32 cells into an occupancy word (kept in shared
//      memory for the gaps) and counts the cars it must step: those left of
//      the right halo (a car in the right halo can only move out of the
//      tile; one in the left halo may move in, and is stepped but not
//      counted in the statistics);
//   2. a block-wide prefix sum of the counts gives each thread its slots in
//      one car list, which is padded to a multiple of 32 with a dummy car
//      that reads and writes only padding;
//   3. the warps take the list 32 cars at a time (two groups per warp
//      interleaved), so every lane draws for the same number of cars and no
//      lane is idle; a car's gap is the count of trailing zeros of the
//      occupancy words after its cell (vmax <= 16 < 32 cells in view);
//   4. cars are scattered into an all -1 buffer, which leaves by one bulk
//      store; three result buffers rotate, so the one cleared during a tile
//      was stored two tiles earlier.
// The rule-3 draw uses the counter-independent parts of Philox computed on
// the host (SlowdownKey).
constexpr uint32_t kK1Stages = 2;       // staged spans: the tile being stepped and the next one loading
constexpr uint32_t kK1Outs = 3;         // result buffers: scattered into, being stored, being cleared
constexpr uint32_t kK1Pad = 32;         // padding after each span buffer: the dummy car's cell and moves
constexpr uint32_t kK1Buf = (uint32_t)kGridSpan + kK1Pad;
constexpr uint32_t kK1ListCap = 1024;   // car-list entries; a denser tile is listed and stepped in passes
constexpr uint32_t kK1Dummy = (uint32_t)kGridSpan;   // span index of the dummy car (empty padding)
static_assert(kGridSpan == 32 * kGridThreads, "32 cells per thread");

// One car: rules 1-4.  r: span index of its cell (kK1Dummy for padding);
// returns the velocity used by the move.
template <Draw D>
__device__ __forceinline__ uint32_t k1_car(uint32_t r, const int8_t *__restrict__ in, int8_t *__restrict__ out,
                                           const uint32_t *__restrict__ occ, uint32_t base, uint32_t L,
                                           uint32_t vmax, uint32_t thr, const SlowdownKey &sk, uint32_t &cell)
{
    const uint32_t w = r >> 5;
    const uint32_t gap = __clz(__brev(__funnelshift_rc(occ[w], occ[w + 1u], (r & 31u) + 1u)));   // empty cells ahead
    uint32_t vel = min(min((uint32_t)(uint8_t)in[r] + 1u, vmax), gap);                             // rules 1, 2
    cell = base + r;
    if (cell >= L) cell -= L;
    if (D == Draw::kAlways) {
        vel -= vel != 0u ? 1u : 0u;                                                                  // rule 3, p = 1
    } else if (D == Draw::kPhilox) {
        const uint32_t u = slowdown_word0(cell, sk);
        vel -= (vel != 0u && u < thr) ? 1u : 0u;                                                     // rule 3
    }
    out[r + vel] = (int8_t)vel;                                                                      // rule 4
    return vel;
}

template <Draw D>
__global__ void __launch_bounds__(kGridThreads) grid_k1_kernel(const GridStep g, const GridTileGeom geo,
                                                               const SlowdownKey sk)
{
    __shared__ __align__(128) int8_t s_in[kK1Stages][kK1Buf];
    __shared__ __align__(128) int8_t s_out[kK1Outs][kK1Buf];
    __shared__ uint32_t s_occ[kGridThreads + 2];   // occupancy of each thread's cells; two empty words after
    __shared__ uint16_t s_list[kK1ListCap];
    __shared__ __align__(16) uint32_t s_warp[kGridWarps];
    __shared__ __align__(8) uint64_t s_full[kK1Stages];

    const uint32_t L = g.rc.L, vmax = g.rc.vmax, thr = (uint32_t)g.rc.thr;
    const uint32_t H = geo.halo, C = geo.tile, W = (uint32_t)kGridSpan;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t c0 = 32u * tid;                 // first span index of this thread's cells
    // the thread that issues the copies and waits for them; its warp varies
    // with the block, so the waits of the blocks on one SM spread over its
    // schedulers
    const uint32_t leader = (blockIdx.x % kGridWarps) * 32u;

    if (tid == leader) {
        for (uint32_t b = 0; b < kK1Stages; ++b) mbar_init(&s_full[b], 1);
        fence_mbar_init();
    }
    for (uint32_t c = tid; c < W / 16u; c += kGridThreads) reinterpret_cast<uint4 *>(s_out[0])[c] = kEmpty4;
    if (tid < kK1Stages * (kK1Pad / 16u)) {   // the padding the loads never write: empty cells
        const uint32_t b = tid / (kK1Pad / 16u), q = tid % (kK1Pad / 16u);
        reinterpret_cast<uint4 *>(s_in[b] + W)[q] = kEmpty4;
    }
    if (tid < 2u) s_occ[kGridThreads + tid] = 0u;
    __syncthreads();

    auto bulk_ok = [&](uint32_t tile) {
        const uint32_t t0 = tile * C;
        return t0 >= H && t0 + C + H <= L;
    };
    uint32_t tile = blockIdx.x;
    if (tid == leader && tile < geo.n_tiles && bulk_ok(tile)) {
        mbar_expect_tx(&s_full[0], W);
        bulk_load(s_in[0], g.c_in + (tile * C - H), W, &s_full[0]);
    }
    uint32_t parity = 0;
    bool prev_stored = false;             // the previous tile left by a bulk store (leader only)
    uint32_t tsum = 0, tcross = 0;        // statistics of this thread's cars, reduced at the end
    for (uint32_t it = 0; tile < geo.n_tiles; tile += gridDim.x, ++it) {
        const uint32_t sb = it & 1u;
        const uint32_t ob = it % kK1Outs;
        const uint32_t cb = ob + 1u == kK1Outs ? 0u : ob + 1u;   // cleared now, scattered into by the next tile
        const uint32_t t0 = tile * C;
        const uint32_t own_cells = min(C, L - t0);
        const uint32_t base = t0 >= H ? t0 - H : t0 + L - H;     // road cell of span index 0
        int8_t *in = s_in[sb];
        int8_t *out = s_out[ob];
        if (tid == leader) {
            // the other stage was read by the previous tile, which every thread has finished
            const uint32_t ahead = tile + gridDim.x;
            if (ahead < geo.n_tiles && bulk_ok(ahead)) {
                fence_proxy_async();
                mbar_expect_tx(&s_full[sb ^ 1u], W);
                bulk_load(s_in[sb ^ 1u], g.c_in + (ahead * C - H), W, &s_full[sb ^ 1u]);
            }
            // buffer cb was last stored two tiles ago: that store must have read it
            if (prev_stored) bulk_wait_read_1();
            else bulk_wait_read_all();
        }
        bool ok = true;
        if (bulk_ok(tile)) {
            if (tid == leader) ok = mbar_wait_bounded(&s_full[sb], (parity >> sb) & 1u);
            parity ^= 1u << sb;
        } else {
            for (uint32_t i = tid; i < W; i += kGridThreads) {
                uint32_t cell = base + i;
                if (cell >= L) cell -= L;
                in[i] = g.c_in[cell];
            }
        }
        if (!__syncthreads_and(ok)) {
            if (tid == leader) {
                atomicOr(g.status, kStatusTimeout);
                const uint32_t ahead = tile + gridDim.x;   // its load may still be in flight
                if (ahead < geo.n_tiles && bulk_ok(ahead))
                    mbar_wait_bounded(&s_full[sb ^ 1u], (parity >> (sb ^ 1u)) & 1u);
                bulk_wait_all();
            }
            return;
        }
        // 1. occupancy; clear this thread's cells of the buffer for the next tile
        reinterpret_cast<uint4 *>(s_out[cb] + c0)[0] = kEmpty4;
        reinterpret_cast<uint4 *>(s_out[cb] + c0)[1] = kEmpty4;
        const uint4 *q = reinterpret_cast<const uint4 *>(in + c0);
        const uint32_t occ = occupancy16(q[0]) | (occupancy16(q[1]) << 16);
        s_occ[tid] = occ;
        const uint32_t own_end = H + own_cells;   // cars from here on are not stepped
        uint32_t mine = occ;
        if (c0 + 32u > own_end) mine = c0 >= own_end ? 0u : mine & ((1u << (own_end - c0)) - 1u);
        // 2. block-wide prefix sum of the car counts
        const uint32_t n = __popc(mine);
        uint32_t incl = n;
#pragma unroll
        for (uint32_t d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
            if (lane >= d) incl += t;
        }
        if (lane == 31u) s_warp[warp] = incl;
        __syncthreads();
        uint32_t before = 0, total = 0;
#pragma unroll
        for (uint32_t j = 0; j < kGridWarps; ++j) {
            const uint32_t t = s_warp[j];
            before += j < warp ? t : 0u;
            total += t;
        }
        const uint32_t first_slot = before + incl - n;
        const bool wraps = base + W + kK1Pad > L;   // the span holds cell L - 1: crossings possible
        for (uint32_t chunk = 0; chunk < total; chunk += kK1ListCap) {
            const uint32_t count = min(kK1ListCap, total - chunk);
            const uint32_t padded = (count + 31u) & ~31u;
            uint32_t pos = first_slot;
            if (total <= kK1ListCap) {   // block-uniform: the whole tile at once
                for (uint32_t mm = mine; mm; mm &= mm - 1u) s_list[pos++] = (uint16_t)(c0 + __clz(__brev(mm)));
            } else {
                for (uint32_t mm = mine; mm; mm &= mm - 1u, ++pos)
                    if (pos - chunk < kK1ListCap) s_list[pos - chunk] = (uint16_t)(c0 + __clz(__brev(mm)));
            }
            if (tid < padded - count) s_list[count + tid] = (uint16_t)kK1Dummy;
            __syncthreads();
            // 3. groups of 32 cars: warp w takes groups w, w + 8, ...; two at a time
            const uint32_t groups = padded >> 5;
            for (uint32_t gi = warp; gi < groups; gi += 2u * kGridWarps) {
                uint32_t cell0, cell1;
                const uint32_t r0 = s_list[32u * gi + lane];
                if (gi + kGridWarps < groups) {   // warp-uniform
                    const uint32_t r1 = s_list[32u * (gi + kGridWarps) + lane];
                    const uint32_t v0 = k1_car<D>(r0, in, out, s_occ, base, L, vmax, thr, sk, cell0);
                    const uint32_t v1 = k1_car<D>(r1, in, out, s_occ, base, L, vmax, thr, sk, cell1);
                    const bool own0 = r0 - H < own_cells, own1 = r1 - H < own_cells;
                    tsum += (own0 ? v0 : 0u) + (own1 ? v1 : 0u);
                    if (wraps) tcross += (own0 && cell0 + v0 >= L ? 1u : 0u) + (own1 && cell1 + v1 >= L ? 1u : 0u);
                } else {
                    const uint32_t v0 = k1_car<D>(r0, in, out, s_occ, base, L, vmax, thr, sk, cell0);
                    const bool own0 = r0 - H < own_cells;
                    tsum += own0 ? v0 : 0u;
                    if (wraps) tcross += own0 && cell0 + v0 >= L ? 1u : 0u;
                }
            }
            // 4. the scattered result leaves by bulk store; the list and the
            // occupancy words are rewritten by the next pass or tile; the
            // stage is refilled by a bulk load
            fence_proxy_async();
            __syncthreads();
        }
        if (total == 0u) {
            fence_proxy_async();
            __syncthreads();
        }
        if (own_cells == C) {
            if (tid == leader) {
                bulk_store(g.c_out + t0, out + H, C);
                bulk_commit();
                prev_stored = true;
            }
        } else {
            for (uint32_t i = tid; i < own_cells; i += kGridThreads) g.c_out[t0 + i] = out[H + i];
            prev_stored = false;
        }
    }
    if (tid == leader) bulk_wait_all();
    // a thread's sums stay far below 2^32 (at most 32 cars x vmax per tile);
    // the warp's total may not
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

// the mask-step kernel reads past the span (look-ahead) and scatters up to
// vmax cells past it: padded buffers, two stages and two work buffers
GridTileGeom make_mask_geom(uint32_t vmax, uint32_t L)
{
    GridTileGeom geo = make_geom(1, vmax, L);
    geo.padded = (uint32_t)kGridSpan + 16u * ((vmax + 15u) / 16u + 2u);
    return geo;
}
size_t grid_mask_smem(const GridTileGeom &geo) { return 4u * (size_t)geo.padded; }

template <Draw D, bool kWide>
cudaError_t launch_mask_variant(const GridStep &g, const GridTileGeom &geo, int grid, size_t smem, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(grid_mask_kernel<D, kWide>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    grid_mask_kernel<D, kWide><<<grid, kGridThreads, smem, s>>>(g, geo);
    return cudaGetLastError();
}

template <bool kWide>
cudaError_t launch_mask_draw(const GridStep &g, const GridTileGeom &geo, int grid, size_t smem, cudaStream_t s)
{
    if (g.rc.thr == 0) return launch_mask_variant<Draw::kNever, kWide>(g, geo, grid, smem, s);
    if (g.rc.thr > 0xFFFFFFFFull) return launch_mask_variant<Draw::kAlways, kWide>(g, geo, grid, smem, s);
    return launch_mask_variant<Draw::kPhilox, kWide>(g, geo, grid, smem, s);
}

template <Draw D>
cudaError_t launch_k1_variant(const GridStep &g, const GridTileGeom &geo, int grid, cudaStream_t s)
{
    const SlowdownKey sk = make_slowdown_key(g.step0, g.rc.road, g.rc.key0, g.rc.key1);
    grid_k1_kernel<D><<<grid, kGridThreads, 0, s>>>(g, geo, sk);
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
        // 5 blocks per SM (42 KB of shared memory each) where the list kernel fits 3
        const int kblocks = blocks * 5 / 3;
        const int grid = (int)((uint32_t)kblocks < geo.n_tiles ? (uint32_t)kblocks : geo.n_tiles);
        if (g.rc.thr == 0) return launch_k1_variant<Draw::kNever>(g, geo, grid, s);
        if (g.rc.thr > 0xFFFFFFFFull) return launch_k1_variant<Draw::kAlways>(g, geo, grid, s);
        return launch_k1_variant<Draw::kPhilox>(g, geo, grid, s);
    }
    if (g.ksteps == 1) {
        const GridTileGeom mg = make_mask_geom(g.rc.vmax, g.rc.L);
        const size_t msmem = grid_mask_smem(mg);
        const int mblocks = blocks * 5 / 3;   // the mask kernel fits 5 blocks per SM where the list kernel fits 3
        const int grid = (int)((uint32_t)mblocks < mg.n_tiles ? (uint32_t)mblocks : mg.n_tiles);
        return g.rc.vmax > 16u ? launch_mask_draw<true>(g, mg, grid, msmem, s)
                               : launch_mask_draw<false>(g, mg, grid, msmem, s);
    }
    const size_t smem = grid_tiled_smem(geo);
    const int grid = (int)((uint32_t)blocks < geo.n_tiles ? (uint32_t)blocks : geo.n_tiles);
    if (g.rc.thr == 0) return launch_grid_variant<Draw::kNever>(g, geo, grid, smem, s);
    if (g.rc.thr > 0xFFFFFFFFull) return launch_grid_variant<Draw::kAlways>(g, geo, grid, smem, s);
    return launch_grid_variant<Draw::kPhilox>(g, geo, grid, smem, s);
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

}  // namespace nasch
