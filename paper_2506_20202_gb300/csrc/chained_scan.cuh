// Decoupled look-back ("chained scan") across thread blocks, with bounded waits.
//
// A block takes a partition ticket from a global counter when it starts, so every
// partition it waits on belongs to a block that is already running or finished; the wait
// therefore always ends. It is still bounded: after kSpinLimit polls the block records
// kStatusLookbackTimeout in the status word and continues with what it has (the host
// reports RARA_ERR_TIMEOUT and the frame is invalid).
#pragma once

#include "rara_internal.cuh"

namespace rara {

constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagIncl = 2ull << 62;
constexpr unsigned long long kValueMask = (1ull << 62) - 1;

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Exclusive prefix of `total` over partitions 0..part-1. Must be called by all 32 lanes
// of ONE warp of the block; returns the prefix in every lane. spin_limit bounds the polls
// of one wait (kSpinLimit unless a test lowers it).
__device__ __forceinline__ unsigned long long warp_chained_prefix(unsigned long long *lookback, int part,
                                                                  unsigned long long total,
                                                                  unsigned int *status,
                                                                  int spin_limit = kSpinLimit)
{
    const int lane = threadIdx.x & 31;
    if (part == 0) {
        if (lane == 0) st_relaxed_u64(&lookback[0], kFlagIncl | total);
        return 0ull;
    }
    if (lane == 0) st_relaxed_u64(&lookback[part], kFlagAgg | total);
    unsigned long long excl = 0;
    int end = part - 1;  // newest predecessor still to read
    int spins = 0;
    while (end >= 0) {
        const int idx = end - lane;
        unsigned long long v = idx >= 0 ? ld_relaxed_u64(&lookback[idx]) : kFlagIncl;
        const unsigned long long flag = v & ~kValueMask;
        const unsigned waiting = __ballot_sync(0xffffffffu, flag == 0);
        const unsigned incl = __ballot_sync(0xffffffffu, flag == kFlagIncl);
        // Only the predecessors up to the nearest inclusive prefix matter.
        if (waiting && (!incl || __ffs(waiting) < __ffs(incl))) {
            if (++spins > spin_limit) {
                if (lane == 0) atomicOr(status, kStatusLookbackTimeout);
                break;
            }
            __nanosleep(32);
            continue;
        }
        unsigned long long val = v & kValueMask;
        if (incl) {
            const int first = __ffs(incl) - 1;  // nearest predecessor with an inclusive prefix
            if (lane > first) val = 0;
        }
        for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
        excl += val;
        if (incl) break;
        end -= 32;
    }
    if (lane == 0) st_relaxed_u64(&lookback[part], kFlagIncl | (excl + total));
    return excl;
}

}  // namespace rara
