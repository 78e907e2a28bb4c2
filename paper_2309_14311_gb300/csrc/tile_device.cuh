// Device building blocks shared by the single-road and batched kernels:
// the agent warp-tile step, the agent whole-ring step loop, the grid
// span step, the grid whole-ring step loop, and the PTX wrappers for
// mbarriers and 1-D bulk (TMA) copies.  Every routine applies the four rules
// of the handout's model section ("The Nagel-Schreckenberg traffic model",
// rules 1-4) with the rule-3 draw keyed by (cell, step, road).
#pragma once

#include "kernels.h"

namespace nasch {
namespace {

// R consecutive cars starting at car g (g a multiple of 8): x by 16-byte
// loads, v by 8-byte loads.
template <int R>
__device__ __forceinline__ void load_cars_vec(const int32_t *__restrict__ x_in,
                                              const uint8_t *__restrict__ v_in, uint32_t g,
                                              uint32_t (&x)[R], uint32_t (&v)[R])
{
    static_assert(R % 8 == 0, "vector path loads 8 cars at a time");
#pragma unroll
    for (int q = 0; q < R / 4; ++q) {
        const int4 xq = __ldg(reinterpret_cast<const int4 *>(x_in + g) + q);
        x[4 * q] = (uint32_t)xq.x;
        x[4 * q + 1] = (uint32_t)xq.y;
        x[4 * q + 2] = (uint32_t)xq.z;
        x[4 * q + 3] = (uint32_t)xq.w;
    }
#pragma unroll
    for (int q = 0; q < R / 8; ++q) {
        const uint2 vv = __ldg(reinterpret_cast<const uint2 *>(v_in + g) + q);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            v[8 * q + r] = (vv.x >> (8 * r)) & 0xFFu;
            v[8 * q + r + 4] = (vv.y >> (8 * r)) & 0xFFu;
        }
    }
}

template <int R>
__device__ __forceinline__ void store_cars_vec(int32_t *__restrict__ x_out,
                                               uint8_t *__restrict__ v_out, uint32_t g,
                                               const uint32_t (&x)[R], const uint32_t (&v)[R])
{
    static_assert(R % 8 == 0, "vector path stores 8 cars at a time");
#pragma unroll
    for (int q = 0; q < R / 4; ++q)
        reinterpret_cast<int4 *>(x_out + g)[q] =
            make_int4((int)x[4 * q], (int)x[4 * q + 1], (int)x[4 * q + 2], (int)x[4 * q + 3]);
#pragma unroll
    for (int q = 0; q < R / 8; ++q) {
        uint2 vv;
        vv.x = v[8 * q] | (v[8 * q + 1] << 8) | (v[8 * q + 2] << 16) | (v[8 * q + 3] << 24);
        vv.y = v[8 * q + 4] | (v[8 * q + 5] << 8) | (v[8 * q + 6] << 16) | (v[8 * q + 7] << 24);
        reinterpret_cast<uint2 *>(v_out + g)[q] = vv;
    }
}

// How rule 3 is decided for a whole launch: p = 0 never slows down, p = 1
// always does (no draw needed), anything else draws.
enum class Draw { kNever, kAlways, kPhilox };

__host__ __device__ __forceinline__ Draw draw_mode(uint64_t thr) { return thr == 0 ? Draw::kNever : (thr > 0xFFFFFFFFull ? Draw::kAlways : Draw::kPhilox); }

// The k fused steps of one warp-tile held in registers (32 lanes x R cars).
// On the ring (kInterior false) the gap is taken modulo L and cars crossing
// L-1 -> 0 wrap.  kInterior: the tile is interior (agent_interior_steps
// states the condition) and steps in plain cell order, with no crossings.
template <int R, Draw D, bool kFull, bool kInterior>
__device__ __forceinline__ void agent_tile_steps(const AgentStep &a, uint32_t (&x)[R], uint32_t (&v)[R],
                                                 uint32_t n_own, unsigned long long *s_sum,
                                                 unsigned long long *s_cross)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t L = a.rc.L;
    const uint32_t Lm1 = L - 1u;
    const uint32_t vmax = a.rc.vmax;
    const uint32_t thr = (uint32_t)a.rc.thr;
    for (int s = 0; s < a.ksteps; ++s) {
        const uint32_t step = a.step0 + (uint32_t)s;
        // leader of the lane's last car: the next lane's first car (start-of-step)
        const uint32_t lead_last = __shfl_down_sync(0xFFFFFFFFu, x[0], 1);
        uint32_t tsum = 0, tcross = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t xi = x[r];
            const uint32_t lead = (r + 1 < R) ? x[r + 1] : lead_last;
            // empty cells ahead: (lead - x - 1) mod L, or L - 1 if the car is
            // its own leader; on the ring as the smaller of two unsigned values
            const uint32_t d = lead - xi;
            const uint32_t gap = kInterior ? d - 1u : min(d - 1u, d + Lm1);
            uint32_t vel = min(min(v[r] + 1u, vmax), gap);            // rules 1, 2
            if (D == Draw::kAlways) {
                vel -= vel > 0u ? 1u : 0u;                              // rule 3, p = 1
            } else if (D == Draw::kPhilox) {
                const uint32_t u = philox_word0(xi, step, a.rc.road, kTagSlowdown, a.rc.key0, a.rc.key1);
                vel -= (vel > 0u && u < thr) ? 1u : 0u;                 // rule 3
            }
            uint32_t nx = xi + vel;                                     // rule 4
            bool wrap = false;
            if (!kInterior) {
                wrap = nx >= L;
                nx = wrap ? nx - L : nx;
            }
            (void)NASCH_DCHECK(nx < L, kDbgAgentPosition);
            (void)NASCH_DCHECK(vel <= vmax, kDbgAgentVelocity);
            x[r] = nx;
            v[r] = vel;
            if (kFull || (uint32_t)r < n_own) {
                tsum += vel;
                if (!kInterior) tcross += wrap ? 1u : 0u;
            }
        }
        if (kFull && n_own == 0u) tsum = tcross = 0u;   // halo lanes
        tsum = __reduce_add_sync(0xFFFFFFFFu, tsum);
        if (!kInterior) tcross = __reduce_add_sync(0xFFFFFFFFu, tcross);
        if (lane == 0 && (tsum | tcross)) {
            atomicAdd(&s_sum[s], (unsigned long long)tsum);
            if (!kInterior) atomicAdd(&s_cross[s], (unsigned long long)tcross);
        }
    }
}

// The k fused steps of an interior warp-tile: no car of the tile can reach
// cell L-1 within the launch (the tile does not wrap round the ring and its
// last car, moving at most vmax a step, stays below L), so every leader lies
// ahead of its car in plain cell order, no car crosses L-1 -> 0 and the step
// needs no modular arithmetic and no crossing count.  The tile is full:
// every lane is all-owned or all-halo.  Lane 31's last car is halo whose
// result is discarded (its leader is its own lane's first car); its
// velocity stays <= vmax, which keeps its moves inside the bound the
// interior test assumes.
//
// Two rewrites of the same step keep the per-car work small: during the
// loop the velocity registers hold w = v + 1, so rule 1's increment is
// carried from the previous step (the move adds w' - 1 = v'); and a lane's
// velocity sum at a step is the growth of the sum of its cars' positions,
// taken mod 2^32 (the true value, at most R x 127, is far below 2^32).
// They cost a few operations per car at the launch's start and end, which
// launches of few steps do not win back (agent_tile_steps with kInterior
// serves those).
template <int R, Draw D>
__device__ __forceinline__ void agent_interior_steps(const AgentStep &a, uint32_t (&x)[R], uint32_t (&v)[R],
                                                     uint32_t n_own, unsigned long long *s_sum)
{
    static_assert(R % 2 == 0, "positions are summed in pairs");
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t vmax = a.rc.vmax;
    const uint32_t thr = (uint32_t)a.rc.thr;
    uint32_t X = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) X += x[r];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] += 1u;
    for (int s = 0; s < a.ksteps; ++s) {
        const uint32_t step = a.step0 + (uint32_t)s;
        const uint32_t lead_last = __shfl_down_sync(0xFFFFFFFFu, x[0], 1);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t xi = x[r];
            const uint32_t lead = (r + 1 < R) ? x[r + 1] : lead_last;
            const uint32_t gap = lead - xi - 1u;
            const uint32_t vel = min(min(v[r], vmax), gap);                         // rules 1, 2
            bool slow = false;                                                        // rule 3
            if (D == Draw::kAlways) {
                slow = vel > 0u;
            } else if (D == Draw::kPhilox) {
                const uint32_t u = philox_word0(xi, step, a.rc.road, kTagSlowdown, a.rc.key0, a.rc.key1);
                slow = vel > 0u && u < thr;
            }
            const uint32_t w = vel + (slow ? 0u : 1u);                                // v' + 1
            x[r] = xi + w - 1u;                                                       // rule 4
            v[r] = w;
            (void)NASCH_DCHECK(xi + w - 1u < a.rc.L, kDbgAgentPosition);
            (void)NASCH_DCHECK(w <= vmax + 1u, kDbgAgentVelocity);
        }
        uint32_t Xn = 0;
#pragma unroll
        for (int r = 0; r < R; r += 2) Xn = Xn + x[r] + x[r + 1];
        uint32_t tsum = Xn - X;
        X = Xn;
        if (n_own == 0u) tsum = 0u;   // halo lanes
        tsum = __reduce_add_sync(0xFFFFFFFFu, tsum);
        if (lane == 0 && tsum) atomicAdd(&s_sum[s], (unsigned long long)tsum);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] -= 1u;
}

// One warp-tile: 32 lanes x R consecutive cars in registers.  kFull: the
// tile lies inside [0, N) and every owned car of a lane is owned (lanes are
// either all-owned or all-halo), so no per-car ownership test is needed.
// kCarry: an interior tile steps by agent_interior_steps (for launches of
// many steps), else by agent_tile_steps in plain cell order.
template <int R, Draw D, bool kFull, bool kCarry>
__device__ __forceinline__ void agent_warp_tile(const AgentStep &a, uint32_t t0, uint32_t owned,
                                                unsigned long long *s_sum, unsigned long long *s_cross)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t e0 = lane * R;
    const uint32_t N = a.N;
    uint32_t x[R], v[R];
    if (kFull) {
        load_cars_vec<R>(a.x_in, a.v_in, t0 + e0, x, v);
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t g = (t0 + e0 + (uint32_t)r) % N;   // halo wraps round the ring
            x[r] = (uint32_t)a.x_in[g];
            v[r] = a.v_in[g];
        }
    }
    // cars of this lane that the tile owns (statistics and write-back)
    const uint32_t own_end = min(owned, N - t0);
    const uint32_t n_own = e0 >= own_end ? 0u : min((uint32_t)R, own_end - e0);
    bool interior = false;
    if (kFull) {
        // cars in cyclic order: a tile that does not wrap round the ring has
        // its first car at or below its last; its last car (halo) moves at
        // most k * vmax cells in the launch (L + k * vmax < 2^32)
        const uint32_t first = __shfl_sync(0xFFFFFFFFu, x[0], 0);
        const uint32_t last = __shfl_sync(0xFFFFFFFFu, x[R - 1], 31);
        interior = first <= last && last + (uint32_t)a.ksteps * a.rc.vmax < a.rc.L;
    }
    if (kFull && interior) {
        if (kCarry)
            agent_interior_steps<R, D>(a, x, v, n_own, s_sum);
        else
            agent_tile_steps<R, D, true, true>(a, x, v, n_own, s_sum, s_cross);
    } else {
        agent_tile_steps<R, D, kFull, false>(a, x, v, n_own, s_sum, s_cross);
    }

    if (n_own == (uint32_t)R) {
        store_cars_vec<R>(a.x_out, a.v_out, t0 + e0, x, v);
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if ((uint32_t)r < n_own) {
                a.x_out[t0 + e0 + r] = (int32_t)x[r];
                a.v_out[t0 + e0 + r] = (uint8_t)v[r];
            }
        }
    }
}

// Occupancy bits of four cells packed in a 32-bit word (bit b = byte b has
// its sign bit clear, i.e. holds a car).
__device__ __forceinline__ uint32_t occupancy4(uint32_t w)
{
    // sign bits of the bytes, inverted, at bits 7, 15, 23, 31; the multiply
    // gathers them into bits 28..31 (the partial products below bit 28 add
    // up to less than 2^24, so nothing carries into them)
    return ((~w & 0x80808080u) * 0x00204081u) >> 28;
}

__device__ __forceinline__ uint32_t occupancy16(const uint4 q)
{
    return occupancy4(q.x) | (occupancy4(q.y) << 4) | (occupancy4(q.z) << 8) | (occupancy4(q.w) << 12);
}

constexpr uint4 kEmpty4 = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
constexpr uint64_t kWaitLimitNs = 1000000000ull;    // bounded wait on an async copy: 1 s

// ---- PTX wrappers: shared-memory mbarriers and 1-D bulk (TMA) copies ----
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Orders this thread's generic-proxy shared-memory accesses before later
// async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the phase of `bar` with the given parity, for at most limit_ns
// (1 s by default); false if the wait ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns = kWaitLimitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

// global -> shared, completion counted in bytes on `bar`
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// shared -> global, tracked by bulk groups
__device__ __forceinline__ void bulk_store(void *dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// at most the most recent bulk group may still be reading its source
__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

struct GridTileGeom {
    uint32_t halo;      // H, multiple of 16
    uint32_t tile;      // C = kGridSpan - 2H cells owned per tile
    uint32_t padded;    // kGridSpan + pad: buffer length (multiple of 16)
    uint32_t n_tiles;
    uint32_t nwork;     // rotating output buffers: 2 for k = 1, else 3
};

// ---- the list method for one warp (fused grid steps) ----
//
// A warp-tile is a staged span of kKwSpan cells: the tile's own cells with a
// halo of H >= k * vmax cells on each side.  The warp lists the span's cars
// in cell order (position, velocity) and clears the span, runs the k steps
// on the list, and scatters the cars that end in the tile's own cells back
// into the span.  A car's leader is the next list entry; the lanes take the
// list 32 cars at a time in ascending order, three groups at once, and every
// lane reads (its car and the leader) before any lane writes, so each car
// sees its leader's start-of-step position (the later groups have not moved
// yet).  After the last car come dummy cars far beyond the span, so the last
// car's gap is at least the distance to the span's end; that is wrong only
// for cars within vmax of the end, and the error moves back at most vmax
// cells a step, which keeps it in the right halo.  Statistics count the cars
// whose cell at the start of a step is one of the tile's own.

// Rule-3 draws for grid_warp_steps.  FoldedDraws: the key of the road
// computed on the host (a kernel parameter), with the two step words
// recomputed per step.  PlainDraws: Philox from the road's constants, for
// code that has no folded key at hand.
struct FoldedDraws {
    const SlowdownKey &sk;
    StepWords sw;
    __device__ __forceinline__ void at_step(uint32_t step) { sw = slowdown_step_words(sk, step); }
    __device__ __forceinline__ uint32_t operator()(uint32_t cell) const { return slowdown_word0_at(cell, sk, sw); }
};
struct PlainDraws {
    const RoadConst &rc;
    uint32_t step;
    __device__ __forceinline__ void at_step(uint32_t s) { step = s; }
    __device__ __forceinline__ uint32_t operator()(uint32_t cell) const
    {
        return philox_word0(cell, step, rc.road, kTagSlowdown, rc.key0, rc.key1);
    }
};

// One step of G groups of 32 list entries from i0 (= first group + lane),
// their draws interleaved.  Every lane reads its cars and their leaders
// before any lane writes.  W: cells may wrap past L - 1 (warp-uniform).
template <int G, Draw D, bool W, class Draws>
__device__ __forceinline__ void warp_list_groups(uint16_t *pos, uint8_t *vel, uint32_t i0, const Draws &draws,
                                                 uint32_t L, uint32_t vmax, uint32_t thr, uint32_t base, uint32_t H,
                                                 uint32_t own, uint32_t &tsum, uint32_t &tcross)
{
    uint32_t x[G], lead[G], v[G];
#pragma unroll
    for (int q = 0; q < G; ++q) {
        const uint32_t i = i0 + 32u * (uint32_t)q;
        x[q] = pos[i];
        lead[q] = pos[i + 1u];
        v[q] = vel[i];
    }
    __syncwarp();   // every lane has read before any lane writes
#pragma unroll
    for (int q = 0; q < G; ++q) {
        uint32_t vq = min(min(v[q] + 1u, vmax), lead[q] - x[q] - 1u);              // rules 1, 2
        uint32_t cell = base + x[q];
        if (W && cell >= L) cell -= L;
        if (D == Draw::kAlways) {
            vq -= vq != 0u ? 1u : 0u;                                              // rule 3, p = 1
        } else if (D == Draw::kPhilox) {
            const uint32_t u = draws(cell);
            vq -= (vq != 0u && u < thr) ? 1u : 0u;                                 // rule 3
        }
        const uint32_t i = i0 + 32u * (uint32_t)q;
        (void)NASCH_DCHECK(vq <= vmax, kDbgListVelocity);
        pos[i] = (uint16_t)(x[q] + vq);                                            // rule 4
        vel[i] = (uint8_t)vq;
        const bool mine = x[q] - H < own;
        tsum += mine ? vq : 0u;
        if (W) tcross += (mine && cell + vq >= L) ? 1u : 0u;
    }
}

// One step of the whole list (`padded` entries, whole groups) in ascending
// order, three groups at a time: a group's leaders belong to later groups,
// which have not moved yet.
template <Draw D, bool W, class Draws>
__device__ __forceinline__ void warp_list_step(uint16_t *pos, uint8_t *vel, uint32_t padded, uint32_t lane,
                                               const Draws &draws, uint32_t L, uint32_t vmax, uint32_t thr,
                                               uint32_t base, uint32_t H, uint32_t own, uint32_t &tsum,
                                               uint32_t &tcross)
{
    uint32_t gi = 0;
    for (; gi + 96u <= padded; gi += 96u)
        warp_list_groups<3, D, W>(pos, vel, gi + lane, draws, L, vmax, thr, base, H, own, tsum, tcross);
    if (padded - gi == 64u)
        warp_list_groups<2, D, W>(pos, vel, gi + lane, draws, L, vmax, thr, base, H, own, tsum, tcross);
    else if (padded - gi == 32u)
        warp_list_groups<1, D, W>(pos, vel, gi + lane, draws, L, vmax, thr, base, H, own, tsum, tcross);
}

// Where grid_warp_steps keeps a warp-tile's car list: `cap` entries at pos /
// vel (shared memory), and, for a span with more cars, kKwList entries at
// pos_big / vel_big (this warp's part of a global scratch; null when cap is
// kKwList, which every span fits).
struct WarpList {
    uint16_t *pos;
    uint8_t *vel;
    uint32_t cap;
    uint16_t *pos_big;
    uint8_t *vel_big;
};

// Steps 1 (second half) to 3 of grid_warp_steps with the list at pos / vel.
template <Draw D, class Draws, class AfterList, class Add>
__device__ __forceinline__ void grid_warp_list_run(const RoadConst &rc, Draws &draws, int8_t *span, uint16_t *pos,
                                                   uint8_t *vel, const uint32_t (&m)[kKwSpan / 1024u], uint32_t p,
                                                   uint32_t total, uint32_t padded, uint32_t H, uint32_t own,
                                                   uint32_t base, uint32_t step0, int ksteps, AfterList &after_list,
                                                   Add &add)
{
    constexpr uint32_t kWords = kKwSpan / 1024u;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t L = rc.L, vmax = rc.vmax, thr = (uint32_t)rc.thr;
    const uint32_t c0 = 32u * kWords * lane;
#pragma unroll
    for (uint32_t j = 0; j < kWords; ++j)
        for (uint32_t mm = m[j]; mm; mm &= mm - 1u, ++p) {
            const uint32_t c = c0 + 32u * j + __clz(__brev(mm));
            pos[p] = (uint16_t)c;
            vel[p] = (uint8_t)span[c];
        }
    for (uint32_t i = total + lane; i <= padded; i += 32u) {
        pos[i] = (uint16_t)kKwDummy;
        vel[i] = 0;
    }
    __syncwarp();
    // the span is free until the scatter
#pragma unroll
    for (uint32_t k = 0; k < kKwSpan / 512u; ++k) reinterpret_cast<uint4 *>(span)[lane + 32u * k] = kEmpty4;
    after_list();
    const bool wraps = base + kKwSpan + (uint32_t)ksteps * vmax > L;   // crossings possible
    // 2. k steps on the list
    for (int s = 0; s < ksteps; ++s) {
        draws.at_step(step0 + (uint32_t)s);
        uint32_t tsum = 0, tcross = 0;
        if (wraps)
            warp_list_step<D, true>(pos, vel, padded, lane, draws, L, vmax, thr, base, H, own, tsum, tcross);
        else
            warp_list_step<D, false>(pos, vel, padded, lane, draws, L, vmax, thr, base, H, own, tsum, tcross);
        tsum = __reduce_add_sync(0xFFFFFFFFu, tsum);
        tcross = __reduce_add_sync(0xFFFFFFFFu, tcross);
        if (lane == 0) add(s, tsum, tcross);
        __syncwarp();
    }
    // 3. the cars that end in the tile's own cells go back into the span
    for (uint32_t i = lane; i < total; i += 32u) {
        const uint32_t x = pos[i];
        if (x - H < own) span[x] = (int8_t)vel[i];
    }
    __syncwarp();
}

// Fused steps of one warp-tile.  span: kKwBuf bytes of shared memory holding
// the staged cells (span index 0 = road cell `base`); on return its cells
// [H, H + own) hold the result.  wl: where the car list goes (a span whose
// cars, padded to whole groups and one leader, exceed wl.cap takes the big
// list).  draws: FoldedDraws or PlainDraws of the road.  after_list() is
// called by every lane once the span has been read (it may be reused from
// then on); add(s, sum, cross) by lane 0 with step s's statistics of this
// warp-tile.
template <Draw D, class Draws, class AfterList, class Add>
__device__ __forceinline__ void grid_warp_steps(const RoadConst &rc, Draws draws, int8_t *span, const WarpList wl,
                                                uint32_t H, uint32_t own, uint32_t base, uint32_t step0, int ksteps,
                                                AfterList after_list, Add add)
{
    constexpr uint32_t kWords = kKwSpan / 1024u;          // occupancy words per lane
    const uint32_t lane = threadIdx.x & 31u;
    // 1. the list: cars in cell order
    const uint32_t c0 = 32u * kWords * lane;
    const uint4 *q = reinterpret_cast<const uint4 *>(span + c0);
    uint32_t m[kWords];
    uint32_t n = 0;
#pragma unroll
    for (uint32_t j = 0; j < kWords; ++j) {
        m[j] = occupancy16(q[2u * j]) | (occupancy16(q[2u * j + 1u]) << 16);
        n += __popc(m[j]);
    }
    uint32_t incl = n;
#pragma unroll
    for (uint32_t d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += t;
    }
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    const uint32_t padded = (total + 31u) & ~31u;   // whole groups
    if (wl.pos_big == nullptr || padded + 1u <= wl.cap)   // warp-uniform
        grid_warp_list_run<D>(rc, draws, span, wl.pos, wl.vel, m, incl - n, total, padded, H, own, base, step0,
                              ksteps, after_list, add);
    else
        grid_warp_list_run<D>(rc, draws, span, wl.pos_big, wl.vel_big, m, incl - n, total, padded, H, own, base,
                              step0, ksteps, after_list, add);
}

// The span-list method of a grid tile (used when the staged span's cars fit
// the list): the cars of the staged span `in` become a list sorted by
// position (cell index within the span, velocity); k synchronous steps are
// applied to the list as in the agent form - a car's leader is the next
// entry, and the last car, whose leader is beyond the span, sees at least
// vmax empty cells; then the list is scattered into `out`, which must be all
// -1.  Only cars within k*vmax cells of the span's ends can be wrong (the
// same light cone as the cell-by-cell step), so the middle C cells are
// exact.  Threads own consecutive runs of the list; each step a thread
// publishes its first car's position, and after one barrier updates its cars
// in ascending order in place (car j reads car j+1 before car j+1 moves).
// Shared scratch: s_pos[cap], s_vel[cap], s_first[2 * blockDim.x],
// s_count[warps + 1].  Returns false (doing nothing) if the cars exceed cap.
template <Draw D>
__device__ __forceinline__ bool grid_span_steps(const RoadConst &rc, const int8_t *__restrict__ in, int8_t *out,
                                                uint32_t H, uint32_t own_cells, uint32_t base, uint32_t step0,
                                                int ksteps, uint16_t *s_pos, uint8_t *s_vel, uint32_t cap,
                                                uint32_t *s_first, uint32_t *s_count, unsigned long long *s_sum,
                                                unsigned long long *s_cross)
{
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t nthreads = blockDim.x, nwarps = nthreads >> 5;
    const uint32_t L = rc.L;
    const uint32_t W = (uint32_t)kGridSpan;
    const uint32_t cells_per_thread = W / nthreads;   // 32 (256 threads)
    // 1. cars of this thread's cells -> list ranks
    const uint32_t c0 = tid * cells_per_thread;
    uint32_t m = 0;
    for (uint32_t q = 0; q < cells_per_thread / 16u; ++q)
        m |= occupancy16(reinterpret_cast<const uint4 *>(in + c0)[q]) << (16u * q);
    const uint32_t n = __popc(m);
    uint32_t incl = n;
#pragma unroll
    for (uint32_t d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += t;
    }
    if (lane == 31) s_count[warp] = incl;
    __syncthreads();
    if (tid == 0) {
        uint32_t acc = 0;
        for (uint32_t w = 0; w < nwarps; ++w) {
            const uint32_t t = s_count[w];
            s_count[w] = acc;
            acc += t;
        }
        s_count[nwarps] = acc;
    }
    __syncthreads();
    const uint32_t count = s_count[nwarps];
    if (count > cap) return false;   // uniform: every thread reads the same total
    uint32_t pos = s_count[warp] + incl - n;
    for (uint32_t mm = m; mm; mm &= mm - 1u, ++pos) {
        const uint32_t cell = c0 + (uint32_t)(__ffs(mm) - 1);
        s_pos[pos] = (uint16_t)cell;
        s_vel[pos] = (uint8_t)in[cell];
    }
    // the output starts empty (its previous contents were stored before this
    // tile's first barrier)
    for (uint32_t c = tid; c < W / 16u; c += nthreads) reinterpret_cast<uint4 *>(out)[c] = kEmpty4;
    // 2. k steps on the list; thread t owns list entries [t*per, (t+1)*per)
    const uint32_t per = (count + nthreads - 1u) / nthreads;
    const uint32_t j0 = min(tid * per, count), j1 = min(j0 + per, count);
    const uint32_t far = 0xFFFFu + 1u + rc.vmax;   // no leader within reach
    __syncthreads();   // the list is complete
    for (int s = 0; s < ksteps; ++s) {
        const uint32_t ph = (uint32_t)s & 1u;
        // publish this thread's first car (start of step); two slots by step
        // parity, so a fast thread cannot overwrite one still being read
        s_first[ph * nthreads + tid] = j0 < j1 ? (uint32_t)s_pos[j0] : far;
        __syncthreads();
        // leader of this thread's last car: the next thread's first car
        const uint32_t lead_last = j1 < count ? s_first[ph * nthreads + tid + 1u] : far;
        const uint32_t step = step0 + (uint32_t)s;
        uint32_t tsum = 0, tcross = 0;
        for (uint32_t j = j0; j < j1; ++j) {
            const uint32_t x = s_pos[j];
            const uint32_t lead = j + 1u < j1 ? (uint32_t)s_pos[j + 1u] : lead_last;
            const uint32_t gap = lead - x - 1u;                           // >= vmax when far
            uint32_t vel = min(min((uint32_t)s_vel[j] + 1u, rc.vmax), gap);   // rules 1, 2
            const uint32_t c = base + x;
            uint32_t cell = c >= L ? c - L : c;
            cell = cell >= L ? cell - L : cell;
            if (D == Draw::kAlways) {
                vel -= vel > 0u ? 1u : 0u;                                   // rule 3, p = 1
            } else if (D == Draw::kPhilox) {
                const uint32_t u = philox_word0(cell, step, rc.road, kTagSlowdown, rc.key0, rc.key1);
                vel -= (vel > 0u && u < (uint32_t)rc.thr) ? 1u : 0u;         // rule 3
            }
            s_pos[j] = (uint16_t)(x + vel);                                  // rule 4
            s_vel[j] = (uint8_t)vel;
            const bool own = x - H < own_cells;
            tsum += own ? vel : 0u;
            tcross += (own && cell + vel >= L) ? 1u : 0u;
        }
        tsum = __reduce_add_sync(0xFFFFFFFFu, tsum);
        tcross = __reduce_add_sync(0xFFFFFFFFu, tcross);
        if (lane == 0 && (tsum | tcross)) {
            atomicAdd(&s_sum[s], (unsigned long long)tsum);
            atomicAdd(&s_cross[s], (unsigned long long)tcross);
        }
    }
    // 3. scatter into the empty output (cars that left the span are dropped);
    // a thread's own entries need no barrier, the output's clear had one
    for (uint32_t j = j0; j < j1; ++j) {
        const uint32_t x = s_pos[j];
        if (x < W) out[x] = (int8_t)s_vel[j];
    }
    return true;
}

// Whole ring in one block, agent form: thread t holds cars [t*R, t*R + R)
// of the N <= blockDim.x * R cars; the car after thread t's last car is
// thread t+1's first, or car 0.  Runs ksteps steps; step s's totals go to
// out_sum[s], out_cross[s] (written by thread 0).  Shared scratch:
// s_first[2 * blockDim.x], s_psum[2 * 32], s_pcross[2 * 32].
template <int R>
__device__ __forceinline__ void agent_ring_steps(const int32_t *__restrict__ x_in, const uint8_t *__restrict__ v_in,
                                                 int32_t *x_out, uint8_t *v_out, uint32_t N, const RoadConst &rc,
                                                 uint32_t step0, int ksteps, unsigned long long *out_sum,
                                                 unsigned long long *out_cross, uint32_t *s_first, uint32_t *s_psum,
                                                 uint32_t *s_pcross)
{
    const uint32_t tid = threadIdx.x;
    const uint32_t lane = tid & 31u, warp = tid >> 5;
    const uint32_t nthreads = blockDim.x, nwarps = nthreads >> 5;
    const uint32_t e0 = tid * R;
    const int cnt = e0 < N ? (int)min((uint32_t)R, N - e0) : 0;
    const uint32_t next_owner = (e0 + R < N) ? tid + 1 : 0u;

    uint32_t x[R], v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        x[r] = r < cnt ? (uint32_t)x_in[e0 + r] : 0u;
        v[r] = r < cnt ? (uint32_t)v_in[e0 + r] : 0u;
    }
    for (int s = 0; s < ksteps; ++s) {
        const uint32_t ph = (uint32_t)s & 1u;
        const uint32_t step = step0 + (uint32_t)s;
        if (cnt > 0) s_first[ph * nthreads + tid] = x[0];
        __syncthreads();
        if (tid == 0 && s > 0) {
            unsigned long long sv = 0, cr = 0;
            for (uint32_t w = 0; w < nwarps; ++w) {
                sv += s_psum[(ph ^ 1u) * 32u + w];
                cr += s_pcross[(ph ^ 1u) * 32u + w];
            }
            out_sum[s - 1] = sv;
            out_cross[s - 1] = cr;
        }
        const uint32_t lead_last = s_first[ph * nthreads + next_owner];
        uint32_t tsum = 0, tcross = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (r < cnt) {
                const uint32_t xi = x[r];
                const uint32_t lead = (r + 1 < cnt) ? x[r + 1] : lead_last;
                const uint32_t vel = new_velocity(rc, v[r], agent_gap(xi, lead, rc.L), xi, step);
                uint32_t nx = xi + vel;
                const bool wrap = nx >= rc.L;
                if (wrap) nx -= rc.L;
                x[r] = nx;
                v[r] = vel;
                tsum += vel;
                tcross += wrap ? 1u : 0u;
            }
        }
        tsum = __reduce_add_sync(0xFFFFFFFFu, tsum);
        tcross = __reduce_add_sync(0xFFFFFFFFu, tcross);
        if (lane == 0) {
            s_psum[ph * 32u + warp] = tsum;
            s_pcross[ph * 32u + warp] = tcross;
        }
    }
    __syncthreads();
    if (tid == 0 && ksteps > 0) {
        const uint32_t ph = (uint32_t)(ksteps - 1) & 1u;
        unsigned long long sv = 0, cr = 0;
        for (uint32_t w = 0; w < nwarps; ++w) {
            sv += s_psum[ph * 32u + w];
            cr += s_pcross[ph * 32u + w];
        }
        out_sum[ksteps - 1] = sv;
        out_cross[ksteps - 1] = cr;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (r < cnt) {
            x_out[e0 + r] = (int32_t)x[r];
            v_out[e0 + r] = (uint8_t)v[r];
        }
    }
}

// Whole ring in one block, grid form: the L cells and their successor in
// shared memory (cur, nxt, each >= L bytes); gaps and moves wrap modulo L.
// Step s's totals go to out_sum[s], out_cross[s] (thread 0).  Shared
// scratch: s_psum[32], s_pcross[32].
__device__ __forceinline__ void grid_ring_steps(const int8_t *__restrict__ c_in, int8_t *c_out, const RoadConst &rc,
                                                uint32_t step0, int ksteps, int8_t *cur, int8_t *nxt,
                                                unsigned long long *out_sum, unsigned long long *out_cross,
                                                uint32_t *s_psum, uint32_t *s_pcross)
{
    const uint32_t L = rc.L;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t nwarps = blockDim.x >> 5;
    for (uint32_t i = tid; i < L; i += blockDim.x) cur[i] = c_in[i];
    for (int s = 0; s < ksteps; ++s) {
        const uint32_t step = step0 + (uint32_t)s;
        for (uint32_t i = tid; i < L; i += blockDim.x) nxt[i] = -1;
        __syncthreads();
        uint32_t tsum = 0, tcross = 0;
        for (uint32_t i = tid; i < L; i += blockDim.x) {
            const int8_t here = cur[i];
            if (here < 0) continue;
            const uint32_t limit = min((uint32_t)here + 1u, rc.vmax);
            uint32_t gap = 0;
            uint32_t ahead = i + 1u == L ? 0u : i + 1u;
            while (gap < limit && cur[ahead] < 0) {   // reaches the car itself after L-1 cells
                ++gap;
                ahead = ahead + 1u == L ? 0u : ahead + 1u;
            }
            const uint32_t vel = new_velocity(rc, (uint32_t)here, gap, i, step);
            uint32_t dest = i + vel;
            const bool wrap = dest >= L;
            if (wrap) dest -= L;
            nxt[dest] = (int8_t)vel;
            tsum += vel;
            tcross += wrap ? 1u : 0u;
        }
        tsum = __reduce_add_sync(0xFFFFFFFFu, tsum);
        tcross = __reduce_add_sync(0xFFFFFFFFu, tcross);
        if (lane == 0) {
            s_psum[warp] = tsum;
            s_pcross[warp] = tcross;
        }
        __syncthreads();
        if (tid == 0) {
            unsigned long long sv = 0, cr = 0;
            for (uint32_t w = 0; w < nwarps; ++w) {
                sv += s_psum[w];
                cr += s_pcross[w];
            }
            out_sum[s] = sv;
            out_cross[s] = cr;
        }
        int8_t *t = cur;
        cur = nxt;
        nxt = t;
        // the next step's clear of nxt (the old cur) must wait for this step's
        // reads, and thread 0's reads of s_psum for the next step's writes
        __syncthreads();
    }
    for (uint32_t i = tid; i < L; i += blockDim.x) c_out[i] = cur[i];
}

}  // namespace
}  // namespace nasch
