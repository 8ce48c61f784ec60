// k_sort.cu -- stable LSD radix sort of (uint32 key, uint32 value) pairs.
//
// Digit passes of up to 9 bits (512 buckets). Every pass ranks 4096-key tiles
// the same way: the lanes of a warp that share a digit are found with one
// warp ballot per digit bit (measured faster than match.any), warps in order;
// the tile is staged in shared memory in digit order and written out, so
// global writes are contiguous within each digit run. Keys and ranks are the
// only per-item registers; the values are loaded after the keys are placed.
//
// Inputs below 2^30 keys take the single-pass form of each digit pass
// (Onesweep, Adinets & Merrill 2022): one histogram kernel counts the digits
// of every pass up front; each pass is then one kernel whose blocks claim
// tiles in launch order, rank their tile, publish its per-digit counts, and
// find the counts of all earlier tiles by decoupled look-back over the
// published words, four tiles at a time. A block only waits on tiles claimed
// before its own, whose blocks are already running, so the waits end; every
// wait is still bounded, and one that runs out sets the caller's error word
// (or a spare word of the temp buffer) and the pass goes on, its output wrong
// but never hung.
//
// Larger inputs take three kernels per pass: an upsweep histogram per block
// over a contiguous share of tiles, an exclusive scan of the (digit, block)
// counts in digit-major order, and a downsweep over the same tiles; no block
// waits for another.
//
// Used twice per render: the per-record depth sort (32 bits, 4 passes) and the
// per-key tile sort (ceil(log2(tiles)) bits, 2 passes up to 18 bits). Sorting
// records by depth and then keys stably by tile gives the order of a stable
// sort on (tile << 32 | depth), the per-tile depth ordering of Eq. 3.
#include <atomic>

#include "swgs_internal.cuh"

namespace swgs {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096
constexpr int kWarpSpan = 32 * kSortItems;             // 512 keys per warp
constexpr int kMaxDigitBits = 9;
constexpr int kMaxBins = 1 << kMaxDigitBits;           // 512
constexpr int kBinsPerThread = kMaxBins / kSortThreads;  // 2

SortPlan make_sort_plan(int begin_bit, int end_bit) {
    SortPlan p{};
    int total = end_bit - begin_bit;
    if (total <= 0) { p.passes = 0; p.begin_bit = begin_bit; return p; }
    p.passes = (total + kMaxDigitBits - 1) / kMaxDigitBits;
    int base = total / p.passes, extra = total % p.passes;
    for (int i = 0; i < p.passes; ++i) p.bits_per_pass[i] = base + (i < extra ? 1 : 0);
    p.begin_bit = begin_bit;
    return p;
}

static int sort_grid(long long n, int num_sms) {
    long long tiles = (n + kSortTile - 1) / kSortTile;
    long long g = (long long)num_sms * 4;
    if (tiles < g) g = tiles;
    return (int)(g < 1 ? 1 : g);
}

// single-pass layout: the histograms of every pass, the tile counters, then
// the status words of each pass (tiles x bins)
constexpr size_t kOneHistBytes = 4 * 4 * 512;   // kMaxOnePasses x kMaxBins words
constexpr size_t kOneCounterBytes = 256;
static size_t one_status_words(long long n) { return (size_t)((n + kSortTile - 1) / kSortTile) * 512; }

size_t radix_temp_bytes(long long n, int num_sms) {
    int G = sort_grid(n, num_sms);
    long long hist = (long long)kMaxBins * G + 1;
    size_t b = (size_t)hist * sizeof(uint32_t);
    b = (b + 255) & ~(size_t)255;
    b += scan_u32_temp_bytes(hist);
    b = (b + 255) & ~(size_t)255;
    b += 256;  // total
    const size_t one = kOneHistBytes + kOneCounterBytes + 4 * 4 * one_status_words(n);
    return b > one ? b : one;
}

__global__ void __launch_bounds__(kSortThreads)
radix_upsweep(const uint32_t* __restrict__ keys, long long n, int shift, int bins,
              int tiles_per_block, long long n_tiles, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[kSortWarps][kMaxBins];
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * kMaxBins; i += kSortThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    const uint32_t mask = (uint32_t)bins - 1u;
    const long long t0 = (long long)blockIdx.x * tiles_per_block;
    long long t1 = t0 + tiles_per_block;
    if (t1 > n_tiles) t1 = n_tiles;
    for (long long t = t0; t < t1; ++t) {
        const long long base = t * kSortTile;
        if (base + kSortTile <= n) {
            const uint4* k4 = reinterpret_cast<const uint4*>(keys + base);
#pragma unroll
            for (int it = 0; it < kSortItems / 4; ++it) {
                const uint4 q = k4[it * kSortThreads + threadIdx.x];
                atomicAdd(&h[warp][(q.x >> shift) & mask], 1u);
                atomicAdd(&h[warp][(q.y >> shift) & mask], 1u);
                atomicAdd(&h[warp][(q.z >> shift) & mask], 1u);
                atomicAdd(&h[warp][(q.w >> shift) & mask], 1u);
            }
        } else {
            for (int it = 0; it < kSortItems; ++it) {
                long long i = base + (long long)it * kSortThreads + threadIdx.x;
                if (i < n) atomicAdd(&h[warp][(keys[i] >> shift) & mask], 1u);
            }
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < bins; d += kSortThreads) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) s += h[w][d];
        hist[(long long)d * gridDim.x + blockIdx.x] = s;
    }
}

struct DownSmem {
    uint32_t keys[kSortTile];
    uint32_t vals[kSortTile];
    uint32_t whist[kSortWarps][kMaxBins + 1];
    uint32_t digoff[kMaxBins + 1];
    uint32_t run[kMaxBins];
    uint32_t cnt[kMaxBins + 1];
    uint32_t warp_tot[kSortWarps];
};

__global__ void __launch_bounds__(kSortThreads, 4)
radix_downsweep(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, long long n,
                int shift, int bins, int tiles_per_block, long long n_tiles,
                const uint32_t* __restrict__ offsets) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DownSmem& S = *reinterpret_cast<DownSmem*>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t mask = (uint32_t)bins - 1u;
    const int bits_here = __ffs(bins) - 1;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int d = threadIdx.x; d < bins; d += kSortThreads)
        S.run[d] = offsets[(long long)d * gridDim.x + blockIdx.x];
    const long long t0 = (long long)blockIdx.x * tiles_per_block;
    long long t1 = t0 + tiles_per_block;
    if (t1 > n_tiles) t1 = n_tiles;
    for (long long t = t0; t < t1; ++t) {
        const long long base = t * kSortTile;
        const int valid = (int)((n - base) < kSortTile ? (n - base) : kSortTile);
        for (int i = threadIdx.x; i < kSortWarps * (kMaxBins + 1); i += kSortThreads)
            (&S.whist[0][0])[i] = 0;
        __syncthreads();
        uint32_t k[kSortItems], rk[kSortItems];
#pragma unroll
        for (int it = 0; it < kSortItems; ++it) {
            const int local = warp * kWarpSpan + it * 32 + lane;
            k[it] = local < valid ? keys_in[base + local] : 0xffffffffu;
        }
        // rank each item among equal digits of its warp, in (item, lane) order
#pragma unroll
        for (int it = 0; it < kSortItems; ++it) {
            const int local = warp * kWarpSpan + it * 32 + lane;
            const bool ok = local < valid;
            const uint32_t d = ok ? (k[it] >> shift) & mask : (uint32_t)bins;
            // lanes with the same digit (and the same validity): one ballot per digit bit
            const unsigned vm = __ballot_sync(0xffffffffu, ok);
            unsigned peers = ok ? vm : ~vm;
            for (int b = 0; b < bits_here; ++b) {
                const bool bit = (d >> b) & 1u;
                const unsigned bb = __ballot_sync(0xffffffffu, bit);
                peers &= bit ? bb : ~bb;
            }
            const int leader = __ffs(peers) - 1;
            uint32_t b = 0;
            if (lane == leader) {
                b = S.whist[warp][d];
                S.whist[warp][d] = b + (uint32_t)__popc(peers);
            }
            b = __shfl_sync(0xffffffffu, b, leader);
            rk[it] = b + (uint32_t)__popc(peers & lt_mask);
        }
        __syncthreads();
        // per digit: exclusive prefix over warps, and the tile's digit count
        for (int d = threadIdx.x; d <= bins; d += kSortThreads) {
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) {
                const uint32_t c = S.whist[w][d];
                S.whist[w][d] = run;
                run += c;
            }
            S.cnt[d] = run;
        }
        __syncthreads();
        // exclusive scan of the digit counts: two consecutive digits per thread
        {
            const int d0 = threadIdx.x * kBinsPerThread;
            uint32_t c[kBinsPerThread], sum = 0;
#pragma unroll
            for (int e = 0; e < kBinsPerThread; ++e) {
                c[e] = d0 + e < bins ? S.cnt[d0 + e] : 0u;
                sum += c[e];
            }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) S.warp_tot[warp] = incl;
            __syncthreads();
            uint32_t run = incl - sum;
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) run += (w < warp) ? S.warp_tot[w] : 0u;
#pragma unroll
            for (int e = 0; e < kBinsPerThread; ++e) {
                if (d0 + e < bins) S.digoff[d0 + e] = run;
                run += c[e];
            }
            if (threadIdx.x == 0) S.digoff[bins] = (uint32_t)valid;
        }
        __syncthreads();
        // place the keys; rk becomes the tile-local position
#pragma unroll
        for (int it = 0; it < kSortItems; ++it) {
            const int local = warp * kWarpSpan + it * 32 + lane;
            if (local < valid) {
                const uint32_t d = (k[it] >> shift) & mask;
                rk[it] += S.digoff[d] + S.whist[warp][d];
                S.keys[rk[it]] = k[it];
            }
        }
        // then the values, read with the same coalesced pattern
#pragma unroll
        for (int it = 0; it < kSortItems; ++it) {
            const int local = warp * kWarpSpan + it * 32 + lane;
            if (local < valid)
                S.vals[rk[it]] = vals_in ? vals_in[base + local] : (uint32_t)(base + local);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < valid; i += kSortThreads) {
            const uint32_t key = S.keys[i];
            const uint32_t d = (key >> shift) & mask;
            const uint32_t g = S.run[d] + ((uint32_t)i - S.digoff[d]);
            keys_out[g] = key;
            vals_out[g] = S.vals[i];
        }
        __syncthreads();
        for (int d = threadIdx.x; d < bins; d += kSortThreads) S.run[d] += S.cnt[d];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Single-pass digit passes (decoupled look-back)
// ---------------------------------------------------------------------------
constexpr int kMaxOnePasses = 4;
constexpr int kHistCopies = 4;                 // warp-pair private histograms
constexpr uint32_t kStatAgg = 1u << 30;        // the tile's own digit count
constexpr uint32_t kStatInc = 2u << 30;        // count of the tile and every tile before it
constexpr uint32_t kStatVal = (1u << 30) - 1u;
constexpr long long kOneMaxKeys = 1LL << 30;   // counts must fit the 30-bit field
constexpr int kLookbackSpins = 1 << 20;        // per wait (~1 us each: about a second)

struct OnePlan {
    int passes;
    int shift[kMaxOnePasses];
    int bins[kMaxOnePasses];
};
static_assert(kOneHistBytes == (size_t)kMaxOnePasses * kMaxBins * 4, "histogram layout");
static_assert(kOneCounterBytes >= (2 * kMaxOnePasses + 2) * 4,
              "tile counters, the spare error word, the finished-block count, the trivial flags");

// Digit counts of every pass in one read of the keys. The block that finishes
// last also marks each pass whose keys all share one digit (trivial[p] = 1):
// that pass leaves the order as it is.
__global__ void __launch_bounds__(kSortThreads)
radix_hist_kernel(const uint32_t* __restrict__ keys, long long cap, OnePlan pl,
                  uint32_t* __restrict__ hist, uint32_t* __restrict__ done,
                  uint32_t* __restrict__ trivial, const unsigned long long* __restrict__ n_dev) {
    const long long n = dev_count(cap, n_dev);
    __shared__ uint32_t h[kHistCopies][kMaxOnePasses][kMaxBins];
    for (int i = threadIdx.x; i < kHistCopies * kMaxOnePasses * kMaxBins; i += kSortThreads)
        (&h[0][0][0])[i] = 0;
    __syncthreads();
    const int copy = (threadIdx.x >> 5) & (kHistCopies - 1);
    for (long long i = (long long)blockIdx.x * kSortThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kSortThreads) {
        const uint32_t k = keys[i];
#pragma unroll
        for (int p = 0; p < kMaxOnePasses; ++p)
            if (p < pl.passes)
                atomicAdd(&h[copy][p][(k >> pl.shift[p]) & (uint32_t)(pl.bins[p] - 1)], 1u);
    }
    __syncthreads();
    for (int p = 0; p < pl.passes; ++p)
        for (int d = threadIdx.x; d < pl.bins[p]; d += kSortThreads) {
            uint32_t c = 0;
#pragma unroll
            for (int q = 0; q < kHistCopies; ++q) c += h[q][p][d];
            if (c) atomicAdd(&hist[p * kMaxBins + d], c);
        }
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int p = 0; p < pl.passes; ++p)
        for (int d = threadIdx.x; d < pl.bins[p]; d += kSortThreads)
            if (*(volatile const uint32_t*)&hist[p * kMaxBins + d] == (uint32_t)n) trivial[p] = 1u;
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct OneSmem {
    uint32_t keys[kSortTile];
    uint32_t vals[kSortTile];
    uint32_t whist[kSortWarps][kMaxBins + 1];
    uint32_t digoff[kMaxBins + 1];  // tile-local exclusive digit offsets
    uint32_t gbase[kMaxBins];       // output position of the tile's first key of each digit
    uint32_t cnt[kMaxBins + 1];
    uint32_t warp_tot[kSortWarps];
    int tile;
    int trivial;
};

// Exclusive scan of c[0..bins) (two digits per thread) into out; every thread
// of the block calls it.
__device__ __forceinline__ void block_digit_scan(const uint32_t* c_in, uint32_t* out, int bins,
                                                 uint32_t* warp_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d0 = threadIdx.x * kBinsPerThread;
    uint32_t c[kBinsPerThread], sum = 0;
#pragma unroll
    for (int e = 0; e < kBinsPerThread; ++e) {
        c[e] = d0 + e < bins ? c_in[d0 + e] : 0u;
        sum += c[e];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    uint32_t run = incl - sum;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) run += (w < warp) ? warp_tot[w] : 0u;
#pragma unroll
    for (int e = 0; e < kBinsPerThread; ++e) {
        if (d0 + e < bins) out[d0 + e] = run;
        run += c[e];
    }
    __syncthreads();
}

// One digit pass: grid = one block per tile.
__global__ void __launch_bounds__(kSortThreads, 4)
radix_onesweep(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
               uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, long long n,
               int shift, int bins, const uint32_t* __restrict__ hist,
               const uint32_t* __restrict__ trivial, uint32_t* status,
               uint32_t* tile_counter, uint32_t* err,
               const unsigned long long* __restrict__ n_dev) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    OneSmem& S = *reinterpret_cast<OneSmem*>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t mask = (uint32_t)bins - 1u;
    const int bits_here = __ffs(bins) - 1;
    const unsigned lt_mask = (1u << lane) - 1u;
    if (threadIdx.x == 0) {
        S.tile = (int)atomicAdd(tile_counter, 1u);
        S.trivial = *trivial;
    }
    for (int i = threadIdx.x; i < kSortWarps * (kMaxBins + 1); i += kSortThreads)
        (&S.whist[0][0])[i] = 0;
    __syncthreads();
    const int tile = S.tile;
    const long long base = (long long)tile * kSortTile;
    // deferred sizing: the grid covers the capacity; tiles past the true count
    // hold no key (tiles are claimed in order, so no real tile waits on them)
    if (n_dev) {
        const long long nn = dev_count(n, n_dev);
        if (base >= nn && tile > 0) return;
        n = nn;
    }
    const int valid = (int)((n - base) < kSortTile ? (n - base) : kSortTile);
    // a pass whose digit is the same for every key keeps their order: each tile
    // is copied through (the flag comes from the digit-count kernel, so every
    // tile decides alike and none waits on another)
    if (S.trivial) {
        for (int i = threadIdx.x; i < valid; i += kSortThreads) {
            keys_out[base + i] = keys_in[base + i];
            vals_out[base + i] = vals_in ? vals_in[base + i] : (uint32_t)(base + i);
        }
        return;
    }
    uint32_t k[kSortItems], rk[kSortItems];
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const int local = warp * kWarpSpan + it * 32 + lane;
        k[it] = local < valid ? keys_in[base + local] : 0xffffffffu;
    }
    // rank each item among equal digits of its warp, in (item, lane) order
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const int local = warp * kWarpSpan + it * 32 + lane;
        const bool ok = local < valid;
        const uint32_t d = ok ? (k[it] >> shift) & mask : (uint32_t)bins;
        const unsigned vm = __ballot_sync(0xffffffffu, ok);
        unsigned peers = ok ? vm : ~vm;
        for (int b = 0; b < bits_here; ++b) {
            const bool bit = (d >> b) & 1u;
            const unsigned bb = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? bb : ~bb;
        }
        const int leader = __ffs(peers) - 1;
        uint32_t b = 0;
        if (lane == leader) {
            b = S.whist[warp][d];
            S.whist[warp][d] = b + (uint32_t)__popc(peers);
        }
        b = __shfl_sync(0xffffffffu, b, leader);
        rk[it] = b + (uint32_t)__popc(peers & lt_mask);
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, and the tile's digit count
    for (int d = threadIdx.x; d < bins; d += kSortThreads) {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = S.whist[w][d];
            S.whist[w][d] = run;
            run += c;
        }
        S.cnt[d] = run;
        // publish the tile's count at once, so that later tiles can look past it
        st_relaxed(&status[(long long)tile * bins + d], (tile == 0 ? kStatInc : kStatAgg) | run);
    }
    __syncthreads();
    // this pass's global digit offsets (exclusive scan of the histogram) into gbase
    block_digit_scan(hist, S.gbase, bins, S.warp_tot);
    // decoupled look-back: the count of every earlier tile, digit by digit
    for (int d = threadIdx.x; d < bins; d += kSortThreads) {
        uint32_t prefix = 0;
        bool done = false;
        for (int t0 = tile - 1; t0 >= 0 && !done; t0 -= 4) {
            // the next four predecessors' words in flight together
            uint32_t v4[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                v4[q] = t0 - q >= 0 ? ld_relaxed(&status[(long long)(t0 - q) * bins + d]) : kStatInc;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (done || t0 - q < 0) continue;
                const uint32_t* w = &status[(long long)(t0 - q) * bins + d];
                uint32_t v = v4[q];
                int spins = 0;
                while ((v & ~kStatVal) == 0u) {
                    if (++spins > kLookbackSpins) {
                        atomicExch(err, 1u);
                        break;
                    }
                    __nanosleep(32);
                    v = ld_relaxed(w);
                }
                prefix += v & kStatVal;
                if ((v & kStatInc) || spins > kLookbackSpins) done = true;
            }
        }
        if (tile > 0)
            st_relaxed(&status[(long long)tile * bins + d], kStatInc | ((prefix + S.cnt[d]) & kStatVal));
        S.gbase[d] += prefix;
    }
    // tile-local digit offsets
    block_digit_scan(S.cnt, S.digoff, bins, S.warp_tot);
    if (threadIdx.x == 0) S.digoff[bins] = (uint32_t)valid;
    __syncthreads();
    // place the keys; rk becomes the tile-local position
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const int local = warp * kWarpSpan + it * 32 + lane;
        if (local < valid) {
            const uint32_t d = (k[it] >> shift) & mask;
            rk[it] += S.digoff[d] + S.whist[warp][d];
            S.keys[rk[it]] = k[it];
        }
    }
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const int local = warp * kWarpSpan + it * 32 + lane;
        if (local < valid)
            S.vals[rk[it]] = vals_in ? vals_in[base + local] : (uint32_t)(base + local);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < valid; i += kSortThreads) {
        const uint32_t key = S.keys[i];
        const uint32_t d = (key >> shift) & mask;
        const uint32_t g = S.gbase[d] + ((uint32_t)i - S.digoff[d]);
        keys_out[g] = key;
        vals_out[g] = S.vals[i];
    }
}

static cudaError_t radix_sort_one(uint32_t* keys_a, uint32_t* vals_a, uint32_t* keys_b,
                                  uint32_t* vals_b, long long n, const SortPlan& plan, void* temp,
                                  int num_sms, bool vals_iota, bool* in_b, uint32_t* err,
                                  const unsigned long long* n_dev, cudaStream_t s) {
    uint32_t* hist = (uint32_t*)temp;
    uint32_t* counters = (uint32_t*)((char*)temp + kOneHistBytes);
    uint32_t* status = (uint32_t*)((char*)temp + kOneHistBytes + kOneCounterBytes);
    if (!err) err = counters + kMaxOnePasses;  // a scratch word when the caller keeps none
    uint32_t* done = counters + kMaxOnePasses + 1;     // digit-count blocks finished
    uint32_t* trivial = counters + kMaxOnePasses + 2;  // per pass: one digit for every key
    const long long tiles = (n + kSortTile - 1) / kSortTile;
    OnePlan pl{};
    pl.passes = plan.passes;
    size_t status_words = 0;
    int shift = plan.begin_bit;
    for (int p = 0; p < plan.passes; ++p) {
        pl.shift[p] = shift;
        pl.bins[p] = 1 << plan.bits_per_pass[p];
        shift += plan.bits_per_pass[p];
        status_words += (size_t)tiles * pl.bins[p];
    }
    // histograms, counters and status words start at zero
    cudaError_t e = cudaMemsetAsync(temp, 0, kOneHistBytes + kOneCounterBytes + 4 * status_words, s);
    if (e != cudaSuccess) return e;
    // the shared-memory opt-in is a per-device function attribute
    constexpr int kMaxDevices = 64;
    static std::atomic<bool> attr_set[kMaxDevices];
    const size_t smem = sizeof(OneSmem);
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices || !attr_set[dev].load()) {
        e = cudaFuncSetAttribute(radix_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < kMaxDevices) attr_set[dev].store(true);
    }
    long long hg = div_up(n, (long long)kSortThreads * 8);
    if (hg > 4LL * num_sms) hg = 4LL * num_sms;
    note_launch();
    radix_hist_kernel<<<(unsigned)hg, kSortThreads, 0, s>>>(keys_a, n, pl, hist, done, trivial,
                                                              n_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    uint32_t *ki = keys_a, *vi = vals_a, *ko = keys_b, *vo = vals_b;
    uint32_t* st = status;
    for (int p = 0; p < plan.passes; ++p) {
        const uint32_t* vread = (p == 0 && vals_iota) ? nullptr : vi;
        note_launch();
        radix_onesweep<<<(unsigned)tiles, kSortThreads, smem, s>>>(
            ki, vread, ko, vo, n, pl.shift[p], pl.bins[p], hist + p * kMaxBins, trivial + p, st,
            counters + p, err, n_dev);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        st += (size_t)tiles * pl.bins[p];
        uint32_t* tk = ki; ki = ko; ko = tk;
        uint32_t* tv = vi; vi = vo; vo = tv;
        *in_b = !*in_b;
    }
    return cudaSuccess;
}

// The look-back timeout check: scratch = 2 x kSortTile keys, 2 x kSortTile out
// keys and values, the status words of two 128-bin tiles, a counter and the
// error word (sort_timeout_scratch_bytes). The counter starts at 1, so the one
// block takes tile 1 and waits on tile 0, which nobody publishes.
size_t sort_timeout_scratch_bytes() {
    return (size_t)(3 * 2 * kSortTile + 2 * 128 + kMaxBins + 64) * sizeof(uint32_t);
}

cudaError_t launch_sort_timeout_check(void* scratch, uint32_t* err, cudaStream_t s) {
    uint32_t* keys = (uint32_t*)scratch;
    uint32_t* keys_out = keys + 2 * kSortTile;
    uint32_t* vals_out = keys_out + 2 * kSortTile;
    uint32_t* status = vals_out + 2 * kSortTile;
    uint32_t* hist = status + 2 * 128;
    uint32_t* counter = hist + kMaxBins;
    cudaError_t e = cudaMemsetAsync(scratch, 0, sort_timeout_scratch_bytes(), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(counter, 1, 1, s);  // counter = 1
    if (e != cudaSuccess) return e;
    constexpr int kMaxDevices = 64;
    static std::atomic<bool> attr_set[kMaxDevices];
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices || !attr_set[dev].load()) {
        e = cudaFuncSetAttribute(radix_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(OneSmem));
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < kMaxDevices) attr_set[dev].store(true);
    }
    note_launch();
    radix_onesweep<<<1, kSortThreads, sizeof(OneSmem), s>>>(
        keys, nullptr, keys_out, vals_out, 2LL * kSortTile, 0, 128, hist, hist, status, counter,
        err, nullptr);
    return cudaGetLastError();
}

cudaError_t radix_sort_pairs(uint32_t* keys_a, uint32_t* vals_a, uint32_t* keys_b,
                             uint32_t* vals_b, long long n, const SortPlan& plan, void* temp,
                             int num_sms, bool vals_iota, bool* in_b, bool single_pass,
                             uint32_t* err, cudaStream_t s, const unsigned long long* n_dev) {
    *in_b = false;
    if (n <= 0 || plan.passes == 0) return cudaSuccess;
    if (n_dev && !(single_pass && n < kOneMaxKeys && plan.passes <= kMaxOnePasses))
        return cudaErrorInvalidValue;  // a device count needs the single-pass form
    if (single_pass && n < kOneMaxKeys && plan.passes <= kMaxOnePasses)
        return radix_sort_one(keys_a, vals_a, keys_b, vals_b, n, plan, temp, num_sms, vals_iota,
                              in_b, err, n_dev, s);
    const int G = sort_grid(n, num_sms);
    const long long n_tiles = (n + kSortTile - 1) / kSortTile;
    const int tpb = (int)((n_tiles + G - 1) / G);
    uint32_t* hist = (uint32_t*)temp;
    size_t off = ((size_t)(kMaxBins * (long long)G + 1) * sizeof(uint32_t) + 255) & ~(size_t)255;
    void* scan_tmp = (char*)temp + off;
    off += scan_u32_temp_bytes((long long)kMaxBins * G + 1);
    off = (off + 255) & ~(size_t)255;
    unsigned long long* total = (unsigned long long*)((char*)temp + off);
    // the shared-memory opt-in is a per-device function attribute
    constexpr int kMaxDevices = 64;
    static std::atomic<bool> attr_set[kMaxDevices];
    const size_t smem = sizeof(DownSmem);
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) return e0;
    if (dev < 0 || dev >= kMaxDevices || !attr_set[dev].load()) {
        cudaError_t e = cudaFuncSetAttribute(radix_downsweep,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < kMaxDevices) attr_set[dev].store(true);
    }
    uint32_t *ki = keys_a, *vi = vals_a, *ko = keys_b, *vo = vals_b;
    int shift = plan.begin_bit;
    for (int p = 0; p < plan.passes; ++p) {
        const int bits = plan.bits_per_pass[p];
        const int bins = 1 << bits;
        note_launch();
        radix_upsweep<<<G, kSortThreads, 0, s>>>(ki, n, shift, bins, tpb, n_tiles, hist);
        cudaError_t e = exclusive_scan_u32(hist, hist, (long long)bins * G, scan_tmp, total, s);
        if (e != cudaSuccess) return e;
        const uint32_t* vread = (p == 0 && vals_iota) ? nullptr : vi;
        note_launch();
        radix_downsweep<<<G, kSortThreads, smem, s>>>(ki, vread, ko, vo, n, shift, bins, tpb,
                                                      n_tiles, hist);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        shift += bits;
        uint32_t* tk = ki; ki = ko; ko = tk;
        uint32_t* tv = vi; vi = vo; vo = tv;
        *in_b = !*in_b;
    }
    return cudaSuccess;
}

}  // namespace swgs
