// Stable LSD radix sort of (uint32 key, uint32 value) pairs, one-sweep style.
//
// 1. One histogram pass counts every 8-bit digit of every key for all digit passes.
// 2. Each digit pass is one kernel. A block takes a partition ticket, ranks its keys
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
constexpr int kItems = 12;                       // keys per thread per partition
constexpr int kPart = kSortThreads * kItems;     // keys per partition (3072)
constexpr int kMaxPasses = 4;
constexpr uint32_t kLbAgg = 1u << 30, kLbIncl = 2u << 30, kLbMask = (1u << 30) - 1u;

__global__ void __launch_bounds__(kSortThreads) k_histogram(const uint32_t *__restrict__ keys, int n,
                                                            int passes, uint32_t *__restrict__ hist)
{
    __shared__ uint32_t s_hist[kMaxPasses][kRadix];
    for (int t = threadIdx.x; t < kMaxPasses * kRadix; t += blockDim.x) (&s_hist[0][0])[t] = 0;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&s_hist[p][(k >> (8 * p)) & 0xffu], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < passes * kRadix; t += blockDim.x) {
        const uint32_t v = (&s_hist[0][0])[t];
        if (v) atomicAdd(&hist[t], v);
    }
}

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

__global__ void __launch_bounds__(kSortThreads) k_onesweep(const uint32_t *__restrict__ keys_in,
                                                           const uint32_t *__restrict__ vals_in,
                                                           uint32_t *__restrict__ keys_out,
                                                           uint32_t *__restrict__ vals_out, int n, int shift,
                                                           const uint32_t *__restrict__ hist,
                                                           uint32_t *lookback, uint32_t *ticket,
                                                           uint32_t *status)
{
    __shared__ uint32_t s_warp_hist[kSortWarps][kRadix];
    __shared__ uint32_t s_keys[kPart];
    __shared__ uint32_t s_vals[kPart];
    __shared__ uint32_t s_local_excl[kRadix];   // start of each digit run inside the block
    __shared__ uint32_t s_out_base[kRadix];     // global position of the run start, minus its local start
    __shared__ uint32_t s_tmp[kSortWarps];
    __shared__ uint32_t s_part;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_part = atomicAdd(ticket, 1u);
    for (int t = tid; t < kSortWarps * kRadix; t += kSortThreads) (&s_warp_hist[0][0])[t] = 0;
    __syncthreads();
    const int part = (int)s_part;
    const int base = part * kPart + warp * (32 * kItems);

    uint32_t key[kItems], val[kItems], rank[kItems];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int idx = base + r * 32 + lane;
        const bool ok = idx < n;
        key[r] = ok ? keys_in[idx] : 0u;
        val[r] = ok ? vals_in[idx] : 0u;
        const uint32_t digit = ok ? ((key[r] >> shift) & 0xffu) : 0x100u;
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
        int p = part - 1;
        int spins = 0;
        while (p >= 0) {
            const uint32_t v = ld_relaxed_u32(lookback + (size_t)p * kRadix + tid);
            const uint32_t flag = v & ~kLbMask;
            if (flag == 0u) {
                if (++spins > kSpinLimit) { atomicOr(status, kStatusLookbackTimeout); break; }
                __nanosleep(32);
                continue;
            }
            excl += v & kLbMask;
            if (flag == kLbIncl) break;
            --p;
        }
        st_relaxed_u32(lb, kLbIncl | (excl + total));
    }
    // Global start of digit tid = exclusive scan of the histogram; local start = exclusive
    // scan of this block's totals.
    const uint32_t gstart = block_excl_scan_256(hist[tid], s_tmp);
    const uint32_t lstart = block_excl_scan_256(total, s_tmp);
    s_local_excl[tid] = lstart;
    s_out_base[tid] = gstart + excl - lstart;
    __syncthreads();

    // Reorder in shared memory by digit (stable), then write runs out contiguously.
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int idx = base + r * 32 + lane;
        if (idx < n) {
            const uint32_t digit = (key[r] >> shift) & 0xffu;
            const uint32_t pos = s_local_excl[digit] + s_warp_hist[warp][digit] + rank[r];
            s_keys[pos] = key[r];
            s_vals[pos] = val[r];
        }
    }
    __syncthreads();
    const int count = min(kPart, n - part * kPart);
    for (int j = tid; j < count; j += kSortThreads) {
        const uint32_t k = s_keys[j];
        const uint32_t dst = s_out_base[(k >> shift) & 0xffu] + j;
        if (dst < (uint32_t)n) {  // always true unless a bounded wait gave up
            keys_out[dst] = k;
            vals_out[dst] = s_vals[j];
        }
    }
}

struct SortScratch {
    uint32_t *hist;      // [kMaxPasses][256]
    uint32_t *tickets;   // [kMaxPasses]
    uint32_t *lookback;  // [kMaxPasses][parts][256]
};

SortScratch carve(void *scratch, int parts)
{
    SortScratch s;
    uint32_t *p = (uint32_t *)scratch;
    s.hist = p;
    s.tickets = p + kMaxPasses * kRadix;
    s.lookback = s.tickets + 64;  // keep 256-byte alignment
    (void)parts;
    return s;
}

}  // namespace

size_t sort_scratch_bytes(int64_t n, int key_bits)
{
    const int64_t parts = (n + kPart - 1) / kPart;
    const int passes = (key_bits + 7) / 8;
    return sizeof(uint32_t) * ((size_t)kMaxPasses * kRadix + 64 + (size_t)passes * (size_t)parts * kRadix);
}

int sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *alt_keys, uint32_t *alt_vals, int n, int key_bits,
               void *scratch, uint32_t *status, cudaStream_t s, bool *result_in_alt)
{
    *result_in_alt = false;
    if (n <= 1 || key_bits <= 0) return 0;
    const int passes = (key_bits + 7) / 8;
    const int parts = (n + kPart - 1) / kPart;
    SortScratch sc = carve(scratch, parts);
    cudaMemsetAsync(scratch, 0, sort_scratch_bytes(n, key_bits), s);
    int launches = 0;
    const int hist_blocks = min(1024, (n + 4095) / 4096);
    k_histogram<<<hist_blocks, kSortThreads, 0, s>>>(keys, n, passes, sc.hist);
    ++launches;
    uint32_t *ki = keys, *vi = vals, *ko = alt_keys, *vo = alt_vals;
    for (int p = 0; p < passes; ++p) {
        k_onesweep<<<parts, kSortThreads, 0, s>>>(ki, vi, ko, vo, n, 8 * p, sc.hist + p * kRadix,
                                                  sc.lookback + (size_t)p * parts * kRadix, sc.tickets + p,
                                                  status);
        ++launches;
        uint32_t *t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
    }
    *result_in_alt = (passes & 1) != 0;
    return launches;
}

}  // namespace rara
