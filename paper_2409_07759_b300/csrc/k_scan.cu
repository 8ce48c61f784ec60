// k_scan.cu -- device prefix sums in two launches: the block totals, then the
// scan of each block's elements from the sum of the earlier blocks' totals
// (each block adds those up itself). Used for the compaction block counts, the
// key offsets of the tiles touched in depth order, the radix histograms and the
// integer CDF of the relocation weights.
#include "swgs_internal.cuh"

namespace swgs {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Exclusive block scan of one value per thread; returns the block total in *total.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* total) {
    __shared__ T warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = warp_incl_scan(v);
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = warp_tot[lane];
        T wi = warp_incl_scan(w);
        warp_tot[lane] = wi - w;
        if (lane == 31) *total = wi;
    }
    __syncthreads();
    T r = incl - v + warp_tot[warp];
    __syncthreads();
    return r;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads)
scan_reduce_kernel(const T* __restrict__ in, long long cap, unsigned long long* __restrict__ part,
                   const unsigned long long* __restrict__ n_dev) {
    const long long n = dev_count(cap, n_dev);
    const long long base = (long long)blockIdx.x * kScanTile;
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        long long i = base + (long long)k * kScanThreads + threadIdx.x;
        if (i < n) s += (unsigned long long)in[i];
    }
    __shared__ unsigned long long tot;
    block_excl_scan<unsigned long long>(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// INCL = false: exclusive, out[n] = total. INCL = true: inclusive. The last
// block writes the grand total to *total (if given).
template <typename T, bool INCL>
__global__ void __launch_bounds__(kScanThreads)
scan_final_kernel(const T* __restrict__ in, T* __restrict__ out, long long cap,
                  const unsigned long long* __restrict__ part,
                  const unsigned long long* __restrict__ n_dev,
                  unsigned long long* __restrict__ total) {
    const long long n = dev_count(cap, n_dev);
    // this block's offset: the earlier blocks' totals
    unsigned long long p = 0;
    for (long long b = threadIdx.x; b < (long long)blockIdx.x; b += kScanThreads) p += part[b];
    __shared__ unsigned long long off;
    block_excl_scan<unsigned long long>(p, &off);
    const long long base = (long long)blockIdx.x * kScanTile;
    const long long first = base + (long long)threadIdx.x * kScanItems;
    T v[kScanItems];
    T s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        long long i = first + k;
        v[k] = i < n ? in[i] : (T)0;
        s += v[k];
    }
    __shared__ T tot;
    T e = block_excl_scan<T>(s, &tot);
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
        *total = off + (unsigned long long)tot;
    T run = (T)off + e;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        long long i = first + k;
        if (INCL) run += v[k];
        if (i < n) out[i] = run;
        if (!INCL) run += v[k];
        if (!INCL && i == n - 1) out[n] = run;
    }
    if (!INCL && n == 0 && blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
}

size_t scan_u32_temp_bytes(long long n) {
    long long nb = (n + kScanTile - 1) / kScanTile;
    return (size_t)(nb + 1) * sizeof(unsigned long long);
}

cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, long long n, void* temp,
                               unsigned long long* total, cudaStream_t s,
                               const unsigned long long* n_dev) {
    if (n <= 0) {
        cudaError_t e = cudaMemsetAsync(out, 0, sizeof(uint32_t), s);
        if (e != cudaSuccess) return e;
        if (total) return cudaMemsetAsync(total, 0, sizeof(unsigned long long), s);
        return cudaSuccess;
    }
    long long nb = (n + kScanTile - 1) / kScanTile;
    unsigned long long* part = (unsigned long long*)temp;
    note_launch();
    scan_reduce_kernel<uint32_t><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, part, n_dev);
    note_launch();
    scan_final_kernel<uint32_t, false><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, part,
                                                                             n_dev, total);
    return cudaGetLastError();
}

size_t scan_u64_temp_bytes(long long n) { return scan_u32_temp_bytes(n); }

cudaError_t inclusive_scan_u64(const unsigned long long* in, unsigned long long* out, long long n,
                               void* temp, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    long long nb = (n + kScanTile - 1) / kScanTile;
    unsigned long long* part = (unsigned long long*)temp;
    note_launch();
    scan_reduce_kernel<unsigned long long><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, part,
                                                                                 nullptr);
    note_launch();
    scan_final_kernel<unsigned long long, true><<<(unsigned)nb, kScanThreads, 0, s>>>(
        in, out, n, part, nullptr, nullptr);
    return cudaGetLastError();
}

}  // namespace swgs
