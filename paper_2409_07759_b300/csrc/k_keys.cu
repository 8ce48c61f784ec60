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
    note_launch();
    gather_tiles_kernel<<<div_up(n, 256), 256, 0, s>>>(order, tiles, out, n);
    return cudaGetLastError();
}

// The k-th record in depth order writes one (global tile id, record) pair per
// tile its 3-sigma ellipse covers, at offsets[k]. One warp per record: lane i
// computes the kept run of tile row i (row rule) and a warp scan places the
// runs; then every lane writes consecutive outputs, finding its row by a
// shuffle binary search over the run offsets (fully coalesced stores).
// Records with the same depth keep their (slot-ascending) record order, so a
// stable sort by tile gives each tile's list in (depth, slot) order.
__global__ void __launch_bounds__(256)
emit_keys_kernel(const uint32_t* __restrict__ order, const uint32_t* __restrict__ offsets,
                 long long n_rec, Records rec, const ViewDev* __restrict__ views, int n_views,
                 int tile_w, int tile_h, uint32_t* __restrict__ keys,
                 uint32_t* __restrict__ vals) {
    const unsigned F = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long k = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n_rec;
         k += nw) {
        const uint32_t r = order[k];
        const int n = rec.tiles[r];
        if (n == 0) continue;
        const int vi = find_view_by_record(views, n_views, (int)r);
        const int base_tile = views[vi].tile_base, ntx = views[vi].ntx;
        const short4 rc = rec.rect[r];
        const int h = rc.w - rc.z + 1;
        uint32_t o = offsets[k];
        const uint32_t o_end = o + (uint32_t)n;  // never past this record's range
        for (int r0 = 0; r0 < h; r0 += 32) {
            int f = 0, l = 0, cnt = 0;
            const int row = r0 + lane;
            const bool wide = rc.y - rc.x >= 255;  // runs do not fit one byte: recompute
            if (row < h) {
                if (row < kRunRows && !wide) {
                    const uint16_t run = rec.runs[(long long)r * kRunRows + row];
                    cnt = run >> 8;
                    f = rc.x + (run & 0xff);
                } else {  // taller than the stored rows: recompute
                    const float4 ga = rec.a[r];
                    const float4 gb = rec.b[r];
                    const KmEllipse el = km_ellipse(gb.x, gb.y, gb.z);
                    cnt = km_row_run_fast(el, ga.x, ga.y, rc.x, rc.y, rc.z + row, tile_w,
                                          tile_h, &f, &l);
                }
            }
            int incl = cnt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(F, incl, d);
                if (lane >= d) incl += y;
            }
            const int tot = __shfl_sync(F, incl, 31);
            for (int t0 = 0; t0 < tot; t0 += 32) {
                const int t = t0 + lane;
                // first row j whose inclusive count exceeds t
                int j = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int cand = j + step - 1;
                    const int v = __shfl_sync(F, incl, cand);
                    if (v <= t) j += step;
                }
                const int fj = __shfl_sync(F, f, j);
                const int ej = __shfl_sync(F, incl - cnt, j);
                const uint32_t pos = o + (uint32_t)t;
                if (t < tot && pos < o_end) {
                    keys[pos] = (uint32_t)(base_tile + (rc.z + r0 + j) * ntx + fj + (t - ej));
                    vals[pos] = r;
                }
            }
            o += (uint32_t)tot;
        }
    }
}

cudaError_t launch_emit_keys(const uint32_t* order, const uint32_t* offsets, long long n_rec,
                             const Records rec, const ViewDev* views, int n_views, int tile_w,
                             int tile_h, int num_sms, uint32_t* keys, uint32_t* vals,
                             cudaStream_t s) {
    if (n_rec <= 0) return cudaSuccess;
    long long blocks = (n_rec + 7) / 8;
    if (blocks > (long long)num_sms * 8) blocks = (long long)num_sms * 8;
    note_launch();
    emit_keys_kernel<<<(int)blocks, 256, 0, s>>>(order, offsets, n_rec, rec, views, n_views,
                                                 tile_w, tile_h, keys, vals);
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
    note_launch();
    tile_ranges_kernel<<<div_up(n_keys, 256), 256, 0, s>>>(keys, n_keys, ranges);
    return cudaGetLastError();
}

}  // namespace swgs
