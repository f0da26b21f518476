// Stable LSD radix sort of (uint32 key, uint32 value) pairs, one-sweep style.
//
// 1. The producer of the keys counts every 8-bit digit of every key for all digit passes
//    (the compaction and emission kernels do it on the fly).
// 2. Each digit pass is one persistent kernel. A block takes partition tickets, ranks keys
//    with warp-level __match_any_sync (peers with the same digit) and per-warp counters,
//    publishes its digit counts, finds its global offsets with a per-digit decoupled
//    look-back over earlier partitions (bounded wait), reorders the keys by digit in
//    shared memory and writes each digit run out contiguously.
// Keys are ranked in input order (warp-striped: warp w owns a contiguous slice of the
// partition, processed 32 keys at a time in lane order), so each pass is stable.
#include "chained_scan.cuh"
#include "rara_internal.cuh"

namespace rara {

namespace {

constexpr int kRadix = 256;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kItems = 16;                       // keys per thread per partition
constexpr int kPart = kSortThreads * kItems;     // keys per partition (4096)
constexpr uint32_t kLbAgg = 1u << 30, kLbIncl = 2u << 30, kLbMask = (1u << 30) - 1u;
constexpr int kLbWidth = 8;                      // predecessors read per look-back step

// Exclusive scan of 256 values held one per thread, result per thread (block of 256).
__device__ __forceinline__ uint32_t block_excl_scan_256(uint32_t v, uint32_t *s_tmp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s_tmp[warp] = incl;
    __syncthreads();
    uint32_t wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += s_tmp[w];
    __syncthreads();
    return wbase + incl - v;
}

__global__ void __launch_bounds__(kSortThreads, 3) k_onesweep(uint32_t *keys_a, uint32_t *vals_a, uint32_t *keys_b,
                                                           uint32_t *vals_b, const unsigned long long *n_ptr,
                                                           uint32_t cap, int pass, int passes,
                                                           const uint32_t *__restrict__ hist, uint32_t *lookback,
                                                           unsigned int *ticket, unsigned int *status,
                                                           unsigned int *result_in_b,
                                                           const uint32_t *__restrict__ seg_base, int num_segs,
                                                           int first_seg_pass, int digit_bits)
{
    __shared__ uint32_t s_warp_hist[kSortWarps][kRadix];
    __shared__ uint32_t s_keys[kPart];
    __shared__ uint32_t s_vals[kPart];
    __shared__ uint32_t s_local_excl[kRadix];   // start of each digit run inside the block
    __shared__ uint32_t s_out_base[kRadix];     // global position of the run start, minus its local start
    __shared__ uint32_t s_gstart[kRadix];       // global start of each digit
    __shared__ uint32_t s_tmp[kSortWarps];
    __shared__ uint32_t s_part;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned long long nn = *n_ptr;
    const int n = (int)(nn < cap ? nn : cap);
    // A pass is skipped when one digit value holds every key; the passes that run alternate
    // between the A and B buffers.
    int flips_before = 0, flips_total = 0;
    bool trivial_here = false;
    for (int q = 0; q < passes; ++q) {
        const bool triv = __syncthreads_or(hist[q * kRadix + tid] == (uint32_t)n) != 0;
        if (q == pass) trivial_here = triv;
        if (!triv) {
            ++flips_total;
            if (q < pass) ++flips_before;
        }
    }
    if (blockIdx.x == 0 && tid == 0) *result_in_b = (unsigned)(flips_total & 1);
    if (trivial_here || n <= 0) return;
    const uint32_t *keys_in = (flips_before & 1) ? keys_b : keys_a;
    const uint32_t *vals_in = (flips_before & 1) ? vals_b : vals_a;
    uint32_t *keys_out = (flips_before & 1) ? keys_a : keys_b;
    uint32_t *vals_out = (flips_before & 1) ? vals_a : vals_b;
    const bool seg_pass = num_segs > 0 && pass >= first_seg_pass;
    const int shift = seg_pass ? 8 * (pass - first_seg_pass) : digit_bits * pass;
    const uint32_t dmask = seg_pass ? 0xffu : (1u << digit_bits) - 1u;
    const int parts = (n + kPart - 1) / kPart;
    s_gstart[tid] = block_excl_scan_256(hist[pass * kRadix + tid], s_tmp);

    for (;;) {
        if (tid == 0) s_part = atomicAdd(ticket, 1u);
        for (int t = tid; t < kSortWarps * kRadix; t += kSortThreads) (&s_warp_hist[0][0])[t] = 0;
        __syncthreads();
        const int part = (int)s_part;
        if (part >= parts) break;
        const int base = part * kPart + warp * (32 * kItems);

        uint32_t key[kItems], val[kItems], rank[kItems];
        const unsigned lt = (1u << lane) - 1u;
        // Issue every load of the partition before ranking, so they are in flight together.
#pragma unroll
        for (int r = 0; r < kItems; ++r) {
            const int idx = base + r * 32 + lane;
            key[r] = idx < n ? __ldg(&keys_in[idx]) : 0u;
        }
#pragma unroll
        for (int r = 0; r < kItems; ++r) {
            const int idx = base + r * 32 + lane;
            val[r] = idx < n ? __ldg(&vals_in[idx]) : 0u;
        }
        if (seg_pass) {  // key = segment of the value (binary search over the segment starts)
#pragma unroll
            for (int r = 0; r < kItems; ++r) {
                int lo = 0, hi = num_segs - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (__ldg(&seg_base[mid]) <= val[r]) lo = mid;
                    else hi = mid - 1;
                }
                key[r] = (uint32_t)lo;
            }
        }
#pragma unroll
        for (int r = 0; r < kItems; ++r) {
            const int idx = base + r * 32 + lane;
            const bool ok = idx < n;
            const uint32_t digit = ok ? ((key[r] >> shift) & dmask) : 0x100u;
            const unsigned peers = __match_any_sync(0xffffffffu, digit);
            const int leader = 31 - __clz(peers);
            uint32_t prev = 0;
            if (ok) prev = s_warp_hist[warp][digit];
            __syncwarp();
            if (ok && lane == leader) s_warp_hist[warp][digit] = prev + __popc(peers);
            __syncwarp();
            rank[r] = prev + __popc(peers & lt);
        }
        __syncthreads();

        // Per digit (one thread each): total over warps, exclusive prefix over warps.
        uint32_t total = 0;
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = s_warp_hist[w][tid];
            s_warp_hist[w][tid] = total;
            total += c;
        }
        // Publish this partition's count for digit `tid`, then look back for the prefix.
        uint32_t *lb = lookback + (size_t)part * kRadix + tid;
        if (part == 0) st_relaxed_u32(lb, kLbIncl | total);
        else st_relaxed_u32(lb, kLbAgg | total);
        uint32_t excl = 0;
        if (part > 0) {
            // Walk back over the predecessors' words for this digit, kLbWidth at a time (the
            // loads of one step are in flight together), summing aggregates up to the
            // nearest inclusive prefix.
            int p = part - 1;
            int spins = 0;
            while (p >= 0) {
                uint32_t v[kLbWidth];
#pragma unroll
                for (int k = 0; k < kLbWidth; ++k)
                    v[k] = p - k >= 0 ? ld_relaxed_u32(lookback + (size_t)(p - k) * kRadix + tid) : kLbIncl;
                int k = 0;
                bool found = false;
#pragma unroll
                for (int u = 0; u < kLbWidth; ++u) {
                    if (found || k < u) continue;        // stopped earlier in this step
                    const uint32_t flag = v[u] & ~kLbMask;
                    if (flag == 0u) continue;            // not published yet: retry from here
                    excl += v[u] & kLbMask;
                    k = u + 1;
                    if (flag == kLbIncl) found = true;
                }
                if (found) break;
                p -= k;
                if (k < kLbWidth) {
                    if (++spins > kSpinLimit) { atomicOr(status, kStatusLookbackTimeout); break; }
                    __nanosleep(32);
                }
            }
            st_relaxed_u32(lb, kLbIncl | (excl + total));
        }
        const uint32_t lstart = block_excl_scan_256(total, s_tmp);
        s_local_excl[tid] = lstart;
        s_out_base[tid] = s_gstart[tid] + excl - lstart;
        __syncthreads();

        // Reorder in shared memory by digit (stable), then write runs out contiguously.
#pragma unroll
        for (int r = 0; r < kItems; ++r) {
            const int idx = base + r * 32 + lane;
            if (idx < n) {
                const uint32_t digit = (key[r] >> shift) & dmask;
                const uint32_t pos = s_local_excl[digit] + s_warp_hist[warp][digit] + rank[r];
                s_keys[pos] = key[r];
                s_vals[pos] = val[r];
            }
        }
        __syncthreads();
        const int count = min(kPart, n - part * kPart);
        for (int j = tid; j < count; j += kSortThreads) {
            const uint32_t k = s_keys[j];
            const uint32_t dst = s_out_base[(k >> shift) & dmask] + j;
            if (dst < (uint32_t)n) {  // always true unless a bounded wait gave up
                keys_out[dst] = k;
                vals_out[dst] = s_vals[j];
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t sort_scratch_bytes(int64_t cap, int passes)
{
    const int64_t parts = (cap + kPart - 1) / kPart;
    return sizeof(uint32_t) * ((size_t)passes * (size_t)(parts > 0 ? parts : 1) * kRadix);
}

int sort_blocks_per_sm()
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_onesweep, kSortThreads, 0) != cudaSuccess || b < 1) {
        cudaGetLastError();
        b = 1;
    }
    return b;
}

int sort_launch(uint32_t *keys_a, uint32_t *vals_a, uint32_t *keys_b, uint32_t *vals_b, const unsigned long long *n,
                uint32_t cap, int passes, const uint32_t *hist, void *scratch, unsigned int *tickets,
                unsigned int *status, unsigned int *result_in_b, int grid, cudaStream_t s,
                const uint32_t *seg_base, int num_segs, int first_seg_pass, int digit_bits)
{
    if (passes <= 0 || grid <= 0) return 0;
    const int64_t parts = ((int64_t)cap + kPart - 1) / kPart;
    cudaMemsetAsync(scratch, 0, sort_scratch_bytes(cap, passes), s);
    for (int p = 0; p < passes; ++p) {
        uint32_t *lb = (uint32_t *)scratch + (size_t)p * (size_t)(parts > 0 ? parts : 1) * kRadix;
        k_onesweep<<<grid, kSortThreads, 0, s>>>(keys_a, vals_a, keys_b, vals_b, n, cap, p, passes, hist, lb,
                                                 tickets + p, status, result_in_b, seg_base, num_segs,
                                                 first_seg_pass, digit_bits);
    }
    return passes;
}

}  // namespace rara
