// Floyd's sampling algorithm (Bentley & Floyd, CACM 1987) for one road, by a
// whole thread block, 1024 draws at a time, with exactly the sequential
// algorithm's result.
//
// The sequential algorithm: for m = 0..N-1 with j_m = L-N+m, draw t_m uniform
// on 0..j_m (Lemire's multiply-shift of the Philox word pair of counter
// (m, 0, road, 1)); insert t_m into the set S, or j_m if t_m is already in S.
// The draws do not depend on S, and its membership test has a closed form:
// every value enters S at the first step that draws it (j_m is new at step m,
// since every earlier draw is at most j_{m-1} < j_m), so t_m is in S_{m-1}
// iff (a) some earlier draw had the same value, or (b) t_m = j_i for an
// earlier i whose own draw t_i was rejected (then j_i was inserted).  A group
// of draws [m0, m0 + B) is therefore decided from
//   - the bit map of S before the group (both (a) and (b) for i < m0);
//   - duplicates inside the group (the smallest index per value, by a
//     shared-memory hash table);
//   - chains inside the group: t_m = j_i with m0 <= i < m makes t_m's
//     rejection equal t_i's; pointer jumping resolves every chain in
//     log2(B) rounds (a rejection is the OR of the chain's own reasons);
// and then every thread sets its pick (j_m if rejected, else t_m) in the bit
// map.  The set, and so the sorted positions, equal the sequential
// algorithm's.
#pragma once

#include "nasch_device.cuh"

namespace nasch {

constexpr int kFloydBlock = 1024;            // draws per group = threads per block
constexpr uint32_t kFloydSlots = 2048;       // shared hash table of a group's draws
constexpr uint32_t kFloydSlotBits = 11;
constexpr uint32_t kFloydEmpty = 0xFFFFFFFFu;
constexpr uint16_t kFloydNoParent = 0xFFFFu;
constexpr int kFloydRounds = 10;             // pointer jumping: chains of up to 1024 draws

struct FloydSmem {
    uint32_t key[kFloydSlots];               // draw value of the slot
    uint32_t first[kFloydSlots];             // smallest group index that drew it
    uint16_t parent[2][kFloydBlock];         // group index whose rejection this one's follows
    uint8_t why[2][kFloydBlock];             // 1: rejected for a reason of its own (or found on its chain)
};

// Sets the N chosen cells of a road in bm (bit c of word c / 64; the bit map
// must start cleared).  Called by all kFloydBlock threads of a block.
__device__ __forceinline__ void floyd_road_bits(uint64_t L, uint64_t N, uint32_t road, uint32_t k0, uint32_t k1,
                                                unsigned long long *bm, FloydSmem &sm)
{
    const uint32_t tid = threadIdx.x;
    const uint64_t jbase = L - N;            // j_m = jbase + m
    for (uint64_t m0 = 0; m0 < N; m0 += (uint64_t)kFloydBlock) {
        for (uint32_t s = tid; s < kFloydSlots; s += (uint32_t)kFloydBlock) {
            sm.key[s] = kFloydEmpty;
            sm.first[s] = kFloydEmpty;
        }
        __syncthreads();
        const uint64_t m = m0 + tid;
        const bool live = m < N;
        uint32_t t = 0, slot = 0;
        bool in_set = false;
        if (live) {
            const uint64_t j = jbase + m;
            const Words4 w = philox4x32_10((uint32_t)m, 0u, road, kTagInit, k0, k1);
            const uint64_t r = ((uint64_t)w.w1 << 32) | w.w0;
            t = (uint32_t)__umul64hi(r, j + 1);              // uniform on 0..j
            in_set = (__ldcg(bm + (t >> 6)) >> (t & 63)) & 1ull;
            slot = (t * 2654435761u) >> (32u - kFloydSlotBits);
            for (;;) {                                        // linear probing; never full
                const uint32_t prev = atomicCAS(&sm.key[slot], kFloydEmpty, t);
                if (prev == kFloydEmpty || prev == t) break;
                slot = (slot + 1u) & (kFloydSlots - 1u);
            }
            atomicMin(&sm.first[slot], tid);
        }
        __syncthreads();
        uint8_t why = 0;
        uint16_t parent = kFloydNoParent;
        if (live) {
            why = (in_set || sm.first[slot] < tid) ? 1 : 0;
            // t = j_i for a draw i of this group before m: rejected iff t_i was
            if (!why && (uint64_t)t >= jbase + m0) {
                const uint64_t i = (uint64_t)t - jbase;
                if (i < m) parent = (uint16_t)(i - m0);
            }
        }
        sm.why[0][tid] = why;
        sm.parent[0][tid] = parent;
        int cur = 0;
        if (__syncthreads_or(parent != kFloydNoParent)) {
            for (int round = 0; round < kFloydRounds; ++round) {
                const uint16_t p = sm.parent[cur][tid];
                uint8_t w2 = sm.why[cur][tid];
                uint16_t p2 = kFloydNoParent;
                if (p != kFloydNoParent) {
                    w2 |= sm.why[cur][p];
                    p2 = sm.parent[cur][p];
                }
                sm.why[cur ^ 1][tid] = w2;
                sm.parent[cur ^ 1][tid] = p2;
                cur ^= 1;
                __syncthreads();
            }
        }
        if (live) {
            const uint64_t pick = sm.why[cur][tid] ? jbase + m : (uint64_t)t;
            atomicOr(bm + (pick >> 6), 1ull << (pick & 63));
        }
        __syncthreads();   // the group's picks are in the bit map before the next group reads it
    }
}

}  // namespace nasch
