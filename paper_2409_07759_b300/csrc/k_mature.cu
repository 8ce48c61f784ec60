// k_mature.cu -- maturation of Alg. 1 (procedure mature) and the expiry
// staggering that follows the first window (schedule_expire), on a buffer
// whose slots [0, num_gs) hold the optimisable Gaussians (gs) and whose slots
// [num_gs, 2 num_gs) hold the ring of the last num_gs matured rows.
#include "swgs_internal.cuh"

namespace swgs {

constexpr int kMatureBlock = 256;

// Per block: how many gs slots have start < st.
__global__ void __launch_bounds__(kMatureBlock)
mature_count_kernel(const int32_t* __restrict__ start, long long n, int st,
                    uint32_t* __restrict__ block_counts) {
    const long long i = (long long)blockIdx.x * kMatureBlock + threadIdx.x;
    const bool m = i < n && start[i] < st;
    const int c = __syncthreads_count(m);
    if (threadIdx.x == 0) block_counts[blockIdx.x] = (uint32_t)c;
}

// The slots with start < st, ascending, at the scanned block offsets (warp
// ballots rank them inside the block).
__global__ void __launch_bounds__(kMatureBlock)
mature_ids_kernel(const int32_t* __restrict__ start, long long n, int st,
                  const uint32_t* __restrict__ block_offsets, int32_t* __restrict__ ids) {
    __shared__ int warp_off[kMatureBlock / 32];
    const long long i = (long long)blockIdx.x * kMatureBlock + threadIdx.x;
    const bool m = i < n && start[i] < st;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, m);
    if (lane == 0) warp_off[warp] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < kMatureBlock / 32; ++w) {
            const int c = warp_off[w];
            warp_off[w] = run;
            run += c;
        }
    }
    __syncthreads();
    if (m) ids[block_offsets[blockIdx.x] + warp_off[warp] + __popc(bal & ((1u << lane) - 1u))] =
        (int32_t)i;
}

struct MatureArrays {
    const void* src[9];   // buf arrays
    void* ring[9];        // buf arrays (rows num_gs + ...)
    void* snap[9];        // snapshot rows 0..n-1 (device)
    long long words[9];   // 4-byte words per row (frozen: bytes)
};

// Row j = gs slot ids[j], every array (blockIdx.y): copied as it is to the
// snapshot row j and to ring slot num_gs + (head + j) mod num_gs; the ring
// copy's frozen flag is 1.
__global__ void __launch_bounds__(256)
mature_copy_kernel(MatureArrays a, const int32_t* __restrict__ ids, long long n, long long num_gs,
                   long long head) {
    const int arr = blockIdx.y;
    if (a.src[arr] == nullptr) return;
    const long long w = a.words[arr];
    const long long total = n * w;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long j = e / w, k = e - j * w;
        const long long slot = ids[j];
        const long long rs = num_gs + (head + j) % num_gs;
        if (arr == 8) {  // uint8 frozen flags
            const uint8_t v = ((const uint8_t*)a.src[arr])[slot];
            ((uint8_t*)a.ring[arr])[rs] = 1;
            if (a.snap[arr]) ((uint8_t*)a.snap[arr])[j] = v;
        } else {
            const uint32_t v = ((const uint32_t*)a.src[arr])[slot * w + k];
            ((uint32_t*)a.ring[arr])[rs * w + k] = v;
            if (a.snap[arr]) ((uint32_t*)a.snap[arr])[j * w + k] = v;
        }
    }
}

// The matured gs slots start their next lifespan: birth = expire, start =
// expire, expire = start + swin_size (after the copies above have read them).
__global__ void mature_rebirth_kernel(const int32_t* __restrict__ ids, long long n,
                                      int32_t* __restrict__ start, int32_t* __restrict__ expire,
                                      int32_t* __restrict__ birth, int swin_size) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int32_t slot = ids[j];
    const int32_t e = expire[slot];
    if (birth) birth[slot] = e;
    start[slot] = e;
    expire[slot] = e + swin_size;
}

// Slice k of the gs slots (slice_size = num_gs / swin_size) gets expire = k,
// slice 0 expire = swin_size: expiries on distinct frames modulo swin_size.
__global__ void schedule_expire_kernel(int32_t* __restrict__ expire, long long num_gs,
                                       int swin_size) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= num_gs) return;
    const long long slice_size = num_gs / swin_size;
    const long long k = i / slice_size;
    if (k < swin_size) expire[i] = k >= 1 ? (int32_t)k : swin_size;
}

cudaError_t launch_mature_ids(const int32_t* start, long long n, int st, uint32_t* block_counts,
                              void* scan_tmp, unsigned long long* total, int32_t* ids,
                              cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const long long nb = div_up(n, kMatureBlock);
    note_launch();
    mature_count_kernel<<<(unsigned)nb, kMatureBlock, 0, s>>>(start, n, st, block_counts);
    cudaError_t e = exclusive_scan_u32(block_counts, block_counts, nb, scan_tmp, total, s);
    if (e != cudaSuccess) return e;
    note_launch();
    mature_ids_kernel<<<(unsigned)nb, kMatureBlock, 0, s>>>(start, n, st, block_counts, ids);
    return cudaGetLastError();
}

cudaError_t launch_mature_move(const swgs_gaussians& buf, const int32_t* ids, long long n,
                               long long num_gs, long long head, int swin_size,
                               void* const snap[9], cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int K = (buf.sh_degree + 1) * (buf.sh_degree + 1);
    MatureArrays a{};
    const void* src[9] = {buf.means, buf.log_scales, buf.quats, buf.opacity_logits, buf.sh,
                          buf.start, buf.expire, buf.birth, buf.frozen};
    const long long w[9] = {3, 3, 4, 1, 3LL * K, 1, 1, 1, 1};
    for (int i = 0; i < 9; ++i) {
        a.src[i] = src[i];
        a.ring[i] = const_cast<void*>(src[i]);
        a.snap[i] = snap[i];
        a.words[i] = w[i];
    }
    int gx = div_up(n * 3LL * K, 256);
    if (gx > 1184) gx = 1184;
    note_launch();
    mature_copy_kernel<<<dim3(gx, 9), 256, 0, s>>>(a, ids, n, num_gs, head);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    note_launch();
    mature_rebirth_kernel<<<div_up(n, 256), 256, 0, s>>>(ids, n, buf.start, buf.expire, buf.birth,
                                                         swin_size);
    return cudaGetLastError();
}

cudaError_t launch_schedule_expire(int32_t* expire, long long num_gs, int swin_size,
                                   cudaStream_t s) {
    if (num_gs <= 0) return cudaSuccess;
    note_launch();
    schedule_expire_kernel<<<div_up(num_gs, 256), 256, 0, s>>>(expire, num_gs, swin_size);
    return cudaGetLastError();
}

}  // namespace swgs
