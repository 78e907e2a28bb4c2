// Device primitives of the NaSch step: Philox4x32-10 in registers and the
// per-car application of the four rules (Handout, "The Nagel-Schreckenberg
// traffic model", rules 1-4).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nasch {

// Debug builds (compiled with -DNASCH_DEBUG) check device-side values and
// indices at the points where a wrong one would corrupt the state or memory;
// a failing check sets the bit of its site in a device word of its
// translation unit and the access it guards is skipped: nothing traps.  The
// host reads and clears the words after every launch (debug_words()).
// Release builds compile the checks to `true`.
enum DebugSite : unsigned int {
    kDbgAgentPosition = 0,   // a moved car outside [0, L)
    kDbgAgentVelocity = 1,   // a velocity above vmax
    kDbgGridWrite = 2,       // a grid kernel's write outside its staged span
    kDbgSegmentWrite = 3,    // the segment kernel's write outside the owned cells
    kDbgListVelocity = 4,    // a listed car's velocity above vmax
};
#ifdef NASCH_DEBUG
static __device__ unsigned int g_debug_word;   // one per translation unit
#define NASCH_DCHECK(cond, site) ((cond) ? true : (atomicOr(&::nasch::g_debug_word, 1u << (site)), false))
// Defines `unsigned int name()`: this unit's debug word, then cleared.
#define NASCH_DEBUG_READER(name)                                                        \
    unsigned int name()                                                                 \
    {                                                                                   \
        unsigned int w = 0, z = 0;                                                      \
        if (cudaMemcpyFromSymbol(&w, ::nasch::g_debug_word, sizeof(w)) != cudaSuccess) \
            return 0x80000000u;                                                         \
        cudaMemcpyToSymbol(::nasch::g_debug_word, &z, sizeof(z));                       \
        return w;                                                                       \
    }
#else
#define NASCH_DCHECK(cond, site) true
#define NASCH_DEBUG_READER(name) \
    unsigned int name() { return 0u; }
#endif

// Philox4x32-10 constants (Salmon, Moraes, Dror & Shaw, SC'11): the two round
// multipliers and the two Weyl increments of the key schedule.
constexpr uint32_t kMulA = 0xD2511F53u;
constexpr uint32_t kMulB = 0xCD9E8D57u;
constexpr uint32_t kWeylA = 0x9E3779B9u;
constexpr uint32_t kWeylB = 0xBB67AE85u;

// Counter word 3 separates the library's two uses of the stream.
constexpr uint32_t kTagSlowdown = 0u;
constexpr uint32_t kTagInit = 1u;

struct Words4 {
    uint32_t w0, w1, w2, w3;
};

// Full Philox4x32-10; usable on host (Floyd initialisation) and device.
__host__ __device__ __forceinline__ Words4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                         uint32_t c3, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t pa = (uint64_t)kMulA * c0;
        const uint64_t pb = (uint64_t)kMulB * c2;
        const uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)pb;
        c3 = (uint32_t)pa;
        c0 = n0;
        c2 = n2;
        k0 += kWeylA;
        k1 += kWeylB;
    }
    return Words4{c0, c1, c2, c3};
}

// Word 0 only, as the rule-3 draw needs.  The last round needs just the high
// half of one product; the compiler drops the rest.
__device__ __forceinline__ uint32_t philox_word0(uint32_t c0, uint32_t c1, uint32_t c2,
                                                 uint32_t c3, uint32_t k0, uint32_t k1)
{
    return philox4x32_10(c0, c1, c2, c3, k0, k1).w0;
}

// The rule-3 draw of one step with the parts that do not depend on the
// cell computed once.  The counter is (cell, step, road, 0): in round 1 the
// product of word 2 (road) is the same for every car, so words 0 and 1 of
// round 1's output are constants; in round 2 so is the product of word 0,
// and round 3 xors a constant into word 2.  The key schedule is folded in
// as well.  slowdown_word0(cell, make_slowdown_key(...)) equals
// philox_word0(cell, step, road, kTagSlowdown, k0, k1) for every cell.
// Only x2b and x3 depend on the step (slowdown_step_words).
struct SlowdownKey {
    uint32_t k1_0;     // round 1: word 2 = hi(A * cell) ^ k1_0
    uint32_t x2a;      // round 2: word 0 = hi(B * word 2) ^ x2a
    uint32_t x2b;      // round 2: word 2 = round-1 word 3 ^ x2b
    uint32_t x3;       // round 3: word 2 = hi(A * word 0) ^ x3
    uint32_t h0;       // round-1 output word 0 = h0 ^ step
    uint32_t k0[10];   // key word 0 of each round
    uint32_t k1[10];   // key word 1 of each round
};

__host__ __device__ inline SlowdownKey make_slowdown_key(uint32_t step, uint32_t road, uint32_t k0, uint32_t k1)
{
    SlowdownKey s;
    for (int r = 0; r < 10; ++r) {
        s.k0[r] = k0 + (uint32_t)r * kWeylA;
        s.k1[r] = k1 + (uint32_t)r * kWeylB;
    }
    const uint64_t pb1 = (uint64_t)kMulB * road;                       // round 1, word 2's product
    s.h0 = (uint32_t)(pb1 >> 32) ^ s.k0[0];
    const uint32_t u0 = s.h0 ^ step;                                   // round-1 output word 0
    const uint32_t u1 = (uint32_t)pb1;                                 // round-1 output word 1
    const uint64_t pa2 = (uint64_t)kMulA * u0;                         // round 2, word 0's product
    s.k1_0 = s.k1[0];
    s.x2a = u1 ^ s.k0[1];
    s.x2b = (uint32_t)(pa2 >> 32) ^ s.k1[1];
    s.x3 = (uint32_t)pa2 ^ s.k1[2];                                    // round-2 output word 3, then round 3's key
    return s;
}

// x2b and x3 of `s` for another step (the rest of the key is the same).
struct StepWords {
    uint32_t x2b, x3;
};
__host__ __device__ __forceinline__ StepWords slowdown_step_words(const SlowdownKey &s, uint32_t step)
{
    const uint64_t pa2 = (uint64_t)kMulA * (s.h0 ^ step);
    return StepWords{(uint32_t)(pa2 >> 32) ^ s.k1[1], (uint32_t)pa2 ^ s.k1[2]};
}

// The draw with the step words given apart from the key.
__host__ __device__ __forceinline__ uint32_t slowdown_word0_at(uint32_t cell, const SlowdownKey &s, StepWords sw)
{
    uint64_t pa = (uint64_t)kMulA * cell;                              // round 1
    uint32_t c2 = (uint32_t)(pa >> 32) ^ s.k1_0;
    uint32_t c3 = (uint32_t)pa;
    uint64_t pb = (uint64_t)kMulB * c2;                                // round 2
    uint32_t c0 = (uint32_t)(pb >> 32) ^ s.x2a;
    uint32_t c1 = (uint32_t)pb;
    c2 = c3 ^ sw.x2b;
    pa = (uint64_t)kMulA * c0;                                         // round 3
    pb = (uint64_t)kMulB * c2;
    c0 = (uint32_t)(pb >> 32) ^ c1 ^ s.k0[2];
    c2 = (uint32_t)(pa >> 32) ^ sw.x3;
    c1 = (uint32_t)pb;
    c3 = (uint32_t)pa;
#pragma unroll
    for (int r = 3; r < 9; ++r) {                                      // rounds 4-9
        pa = (uint64_t)kMulA * c0;
        pb = (uint64_t)kMulB * c2;
        const uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ s.k0[r];
        const uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ s.k1[r];
        c1 = (uint32_t)pb;
        c3 = (uint32_t)pa;
        c0 = n0;
        c2 = n2;
    }
    return (uint32_t)(((uint64_t)kMulB * c2) >> 32) ^ c1 ^ s.k0[9];   // round 10, word 0
}

__host__ __device__ __forceinline__ uint32_t slowdown_word0(uint32_t cell, const SlowdownKey &s)
{
    return slowdown_word0_at(cell, s, StepWords{s.x2b, s.x3});
}

// Parameters every step kernel shares.
struct RoadConst {
    uint32_t L;        // ring length, 1..2^31
    uint32_t vmax;     // 0..127
    uint64_t thr;      // ceil(p * 2^32): 0 never slows, 2^32 always slows
    uint32_t key0;     // seed low word
    uint32_t key1;     // seed high word
    uint32_t road;     // Philox counter word 2
};

// Rule 3 for the car on `cell` at the start of `step`.
__device__ __forceinline__ bool slows_down(const RoadConst &rc, uint32_t cell, uint32_t step)
{
    if (rc.thr == 0) return false;
    if (rc.thr > 0xFFFFFFFFull) return true;
    return philox_word0(cell, step, rc.road, kTagSlowdown, rc.key0, rc.key1) < (uint32_t)rc.thr;
}

// Rules 1-3 for one car with velocity v and `gap` empty cells ahead (gap =
// headway - 1); returns the velocity used by rule 4.
__device__ __forceinline__ uint32_t new_velocity(const RoadConst &rc, uint32_t v, uint32_t gap,
                                                 uint32_t cell, uint32_t step)
{
    uint32_t vel = min(v + 1u, rc.vmax);   // rule 1
    vel = min(vel, gap);                    // rule 2
    if (vel > 0u && slows_down(rc, cell, step)) vel -= 1u;   // rule 3
    return vel;
}

// Empty cells between a car at x and the car ahead at `lead` on the ring
// (positions in [0, L)); a car that is its own leader sees L - 1.
__device__ __forceinline__ uint32_t agent_gap(uint32_t x, uint32_t lead, uint32_t L)
{
    const uint32_t headway = lead > x ? lead - x : lead + L - x;   // in [1, L]
    return headway - 1u;
}

}  // namespace nasch
