// k_keys.cu -- tile keys of the depth-ordered records and the per-tile ranges
// of the sorted key list (the per-tile depth order that Eq. 3 composites in).
#include "swgs_internal.cuh"

namespace swgs {

// out[k] = tiles touched by the k-th record in depth order.
__global__ void gather_tiles_kernel(const uint32_t* __restrict__ order,
                                    const int32_t* __restrict__ tiles, uint32_t* __restrict__ out,
                                    long long n) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = (uint32_t)tiles[order[k]];
}

cudaError_t launch_gather_tiles(const uint32_t* order, const int32_t* tiles, uint32_t* out,
                                long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    gather_tiles_kernel<<<div_up(n, 256), 256, 0, s>>>(order, tiles, out, n);
    return cudaGetLastError();
}

// The k-th record in depth order writes one (global tile id, record) pair per
// tile of its rectangle at offsets[k]. Records with the same depth keep their
// (slot-ascending) record order, so a stable sort by tile gives each tile's
// list in (depth, slot) order.
__global__ void __launch_bounds__(256)
emit_keys_kernel(const uint32_t* __restrict__ order, const uint32_t* __restrict__ offsets,
                 long long n_rec, const int32_t* __restrict__ tiles,
                 const short4* __restrict__ rects, const ViewDev* __restrict__ views, int n_views,
                 uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_rec) return;
    const uint32_t r = order[k];
    const int n = tiles[r];
    if (n == 0) return;
    const int vi = find_view_by_record(views, n_views, (int)r);
    const int base_tile = views[vi].tile_base, ntx = views[vi].ntx;
    const short4 rc = rects[r];
    uint32_t o = offsets[k];
    for (int ty = rc.z; ty <= rc.w; ++ty) {
        const uint32_t row = (uint32_t)(base_tile + ty * ntx);
        for (int tx = rc.x; tx <= rc.y; ++tx) {
            keys[o] = row + (uint32_t)tx;
            vals[o] = r;
            ++o;
        }
    }
}

cudaError_t launch_emit_keys(const uint32_t* order, const uint32_t* offsets, long long n_rec,
                             const Records rec, const ViewDev* views, int n_views,
                             uint32_t* keys, uint32_t* vals, cudaStream_t s) {
    if (n_rec <= 0) return cudaSuccess;
    emit_keys_kernel<<<div_up(n_rec, 256), 256, 0, s>>>(order, offsets, n_rec, rec.tiles,
                                                        rec.rect, views, n_views, keys, vals);
    return cudaGetLastError();
}

// ranges[t] = [first, last+1) of tile t in the sorted keys (ranges zeroed before).
__global__ void tile_ranges_kernel(const uint32_t* __restrict__ keys, long long n,
                                   int2* __restrict__ ranges) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t t = keys[i];
    if (i == 0 || keys[i - 1] != t) ranges[t].x = (int)i;
    if (i == n - 1 || keys[i + 1] != t) ranges[t].y = (int)(i + 1);
}

cudaError_t launch_tile_ranges(const uint32_t* keys, long long n_keys, int2* ranges,
                               cudaStream_t s) {
    if (n_keys <= 0) return cudaSuccess;
    tile_ranges_kernel<<<div_up(n_keys, 256), 256, 0, s>>>(keys, n_keys, ranges);
    return cudaGetLastError();
}

}  // namespace swgs
