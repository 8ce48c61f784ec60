// k_compact.cu -- per-frame lifespan compaction (Sec. 4.2; Alg. 1 gs.filter,
// Alg. 2 buffer.filter): the slots i with start[i] <= frame < expire[i], in
// ascending order, for several frames at once.
//
// Two passes over the 8 B/slot of lifespans, each thread reading its slot's
// lifespan once and testing it against every frame: a per-block count per
// frame, an exclusive scan of the counts (flattened over frames, so each
// frame's ids come out contiguous and frames follow one another), then a
// stable write that ranks every active slot inside its block with warp
// ballots.
#include "swgs_internal.cuh"

namespace swgs {

__global__ void __launch_bounds__(kCompactBlock)
active_count_kernel(const int32_t* __restrict__ start, const int32_t* __restrict__ expire,
                    long long n, const int32_t* __restrict__ frames, int n_frames,
                    uint32_t* __restrict__ block_counts, int n_blocks) {
    const long long i = (long long)blockIdx.x * kCompactBlock + threadIdx.x;
    int st = 0, ex = 0;  // empty lifespan past the end
    if (i < n) {
        st = start[i];
        ex = expire[i];
    }
    for (int g = 0; g < n_frames; ++g) {
        const int frame = frames[g];
        const int c = __syncthreads_count(st <= frame && frame < ex);
        if (threadIdx.x == 0) block_counts[(long long)g * n_blocks + blockIdx.x] = (uint32_t)c;
    }
}

__global__ void __launch_bounds__(kCompactBlock)
active_write_kernel(const int32_t* __restrict__ start, const int32_t* __restrict__ expire,
                    long long n, const int32_t* __restrict__ frames, int n_frames,
                    const uint32_t* __restrict__ block_offsets, int n_blocks,
                    int32_t* __restrict__ out_ids, int32_t* __restrict__ out_counts) {
    __shared__ int warp_off[kCompactBlock / 32];
    const long long i = (long long)blockIdx.x * kCompactBlock + threadIdx.x;
    int st = 0, ex = 0;  // empty lifespan past the end
    if (i < n) {
        st = start[i];
        ex = expire[i];
    }
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int g = 0; g < n_frames; ++g) {
        const int frame = frames[g];
        const bool act = st <= frame && frame < ex;
        const unsigned ballot = __ballot_sync(0xffffffffu, act);
        if (lane == 0) warp_off[warp] = __popc(ballot);
        __syncthreads();
        if (warp == 0) {
            int v = warp_off[lane];
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, incl, o);
                if ((int)lane >= o) incl += y;
            }
            warp_off[lane] = incl - v;
        }
        __syncthreads();
        const long long gbase = (long long)g * n_blocks;
        if (act) {
            const unsigned rank = __popc(ballot & ((1u << lane) - 1u));
            out_ids[block_offsets[gbase + blockIdx.x] + warp_off[warp] + rank] = (int32_t)i;
        }
        if (out_counts && blockIdx.x == 0 && threadIdx.x == 0) {
            const uint32_t first = block_offsets[gbase];
            // the entry after this frame's last block is the next frame's first
            // (or the grand total, stored right after the offsets)
            const uint32_t next = block_offsets[gbase + n_blocks];
            out_counts[g] = (int32_t)(next - first);
        }
        __syncthreads();  // warp_off is rewritten for the next frame
    }
}

cudaError_t launch_active_flags_count(const int32_t* start, const int32_t* expire, long long n,
                                      const int32_t* frames, int n_frames, uint32_t* block_counts,
                                      int n_blocks, cudaStream_t s) {
    note_launch();
    active_count_kernel<<<n_blocks, kCompactBlock, 0, s>>>(start, expire, n, frames, n_frames,
                                                           block_counts, n_blocks);
    return cudaGetLastError();
}

cudaError_t launch_active_write(const int32_t* start, const int32_t* expire, long long n,
                                const int32_t* frames, int n_frames, const uint32_t* block_offsets,
                                int n_blocks, int32_t* out_ids, long long /*ids_stride*/,
                                int32_t* out_counts, cudaStream_t s) {
    note_launch();
    active_write_kernel<<<n_blocks, kCompactBlock, 0, s>>>(start, expire, n, frames, n_frames,
                                                           block_offsets, n_blocks, out_ids,
                                                           out_counts);
    return cudaGetLastError();
}

}  // namespace swgs
