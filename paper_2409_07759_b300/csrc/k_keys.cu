// k_keys.cu -- keys of the depth-ordered records, the ranges of a sorted key
// list, and the per-tile depth-ordered lists that Eq. 3 composites in.
#include "swgs_internal.cuh"

namespace swgs {

// Tile keys are emitted per super tile (a block of SX x SY tiles) rather than
// per tile: a record keys each super tile its tile rectangle overlaps, the
// (super tile, record) keys are sorted stably by super tile, and each super
// tile's depth-ordered candidate list is then expanded into the exact per-tile
// lists by the coverage rule (the row runs). Filtering preserves order, so each
// tile's list is the same depth-ordered list a per-tile key sort gives, from a
// sort over about a fifth as many keys (4x4 super tiles of 16x16-pixel tiles).

// out[k] = super tiles keyed by the k-th record in depth order; *exact += the
// records' exact tile counts (the number of per-tile list entries).
// A bounded grid strides over the records and sums the tile counts per block,
// so the single total word takes one atomic per block (same-address atomics
// serialise in L2).
__global__ void __launch_bounds__(256)
gather_supers_kernel(const uint32_t* __restrict__ order, Records rec, int sx, int sy,
                     uint32_t* __restrict__ out, unsigned long long* __restrict__ exact,
                     long long cap, const unsigned long long* __restrict__ n_dev) {
    __shared__ unsigned long long part[8];
    const long long n = dev_count(cap, n_dev);
    unsigned long long t = 0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const uint32_t r = order[k];
        // a depth sort whose look-back wait ran out may leave stale words in
        // order: never index past the records with one (the call then fails)
        if (r >= (uint32_t)n) { out[k] = 0; continue; }
        out[k] = (uint32_t)rec.supers[r];
        t += (unsigned long long)rec.tiles[r];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int w = 0; w < 8; ++w) s += part[w];
        if (s) atomicAdd(exact, s);
    }
}

cudaError_t launch_gather_supers(const uint32_t* order, const Records rec, int sx, int sy,
                                 uint32_t* out, unsigned long long* exact, long long n,
                                 int num_sms, cudaStream_t s, const unsigned long long* n_dev) {
    if (n <= 0) return cudaSuccess;
    long long grid = div_up(n, 256);
    if (grid > 8LL * num_sms) grid = 8LL * num_sms;
    note_launch();
    gather_supers_kernel<<<(unsigned)grid, 256, 0, s>>>(order, rec, sx, sy, out, exact, n, n_dev);
    return cudaGetLastError();
}

// Kept tile run [first, first + count) of record r in absolute tile row ty
// (the row rule: stored for the first kRunRows rows of narrow records,
// recomputed otherwise).
__device__ __forceinline__ int record_row_run(const Records& rec, uint32_t r, short4 rc, int ty,
                                              int tile_w, int tile_h, int* first) {
    const int row = ty - rc.z;
    const bool wide = rc.y - rc.x >= 255;
    if (row < kRunRows && !wide) {
        const uint16_t run = rec.runs[(long long)r * kRunRows + row];
        *first = rc.x + (run & 0xff);
        return run >> 8;
    }
    const float4 ga = rec.a[r];
    const float4 gb = rec.b[r];
    const KmEllipse el = km_ellipse(gb.x, gb.y, gb.z);
    int l = 0;
    return km_row_run_fast(el, ga.x, ga.y, rc.x, rc.y, ty, tile_w, tile_h, first, &l);
}

// The k-th record in depth order writes, for every super tile of its super
// rectangle that holds one of its tiles (row-major, at offsets[k]), the key
// (global super tile id) | (coverage mask << 16) and the value r. Bit
// ly*SX + lx of the mask is set when the record covers tile (lx, ly) of the
// super tile by the row rule. The sort reads only the low 16 bits (the super
// tile id), so the mask rides along. Per super row only the super columns its
// tile rows' runs reach are visited. Positions of the record's range left over
// (the projection's count is an upper bound) get the key of its first super
// tile with an empty mask, which the expansion passes over. The super tile's
// shape (SX x SY tiles) is a template parameter, so the mask loops run over
// its SY rows only.
template <int SX, int SY>
__global__ void __launch_bounds__(256)
emit_supers_kernel(const uint32_t* __restrict__ order, const uint32_t* __restrict__ offsets,
                   long long n_rec, Records rec, const ViewDev* __restrict__ views, int n_views,
                   int tile_w, int tile_h, uint32_t* __restrict__ keys,
                   uint32_t* __restrict__ vals, const unsigned long long* __restrict__ n_dev) {
    static_assert(SX * SY == 16, "16 tiles per super tile");
    constexpr int sx = SX, sy = SY;
    n_rec = dev_count(n_rec, n_dev);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n_rec;
         k += (long long)gridDim.x * blockDim.x) {
        const uint32_t r = order[k];
        const int tiles = rec.tiles[r];
        if (tiles == 0) continue;
        const short4 rc = rec.rect[r];
        const ViewDev& V = views[find_view_by_record(views, n_views, (int)r)];
        const int x0 = rc.x / sx, y0 = rc.z / sy, y1 = rc.w / sy;
        uint32_t o = offsets[k];
        const uint32_t o_end = o + (uint32_t)rec.supers[r];
        for (int y = y0; y <= y1; ++y) {
            int f[SY], n[SY];
#pragma unroll
            for (int ly = 0; ly < SY; ++ly) {
                f[ly] = 0;
                n[ly] = 0;
                const int ty = y * sy + ly;
                if (ty >= rc.z && ty <= rc.w)
                    n[ly] = record_row_run(rec, r, rc, ty, tile_w, tile_h, &f[ly]);
            }
            // only the super columns the rows' runs reach (the rest have empty masks)
            int cmin = 0x7fffffff, cmax = -1;
#pragma unroll
            for (int ly = 0; ly < SY; ++ly) {
                if (n[ly] > 0) {
                    cmin = min(cmin, f[ly]);
                    cmax = max(cmax, f[ly] + n[ly] - 1);
                }
            }
            if (cmax < 0) continue;
            for (int x = cmin / sx; x <= cmax / sx; ++x) {
                const int tx0 = x * sx;
                unsigned m = 0;
#pragma unroll
                for (int ly = 0; ly < SY; ++ly) {
                    const int lo = max(f[ly], tx0), hi = min(f[ly] + n[ly], tx0 + sx);
                    if (lo < hi) m |= ((1u << (hi - lo)) - 1u) << (lo - tx0 + ly * sx);
                }
                if (m != 0 && o < o_end) {
                    keys[o] = (uint32_t)(V.super_base + y * V.nsx + x) | (m << 16);
                    vals[o] = r;
                    ++o;
                }
            }
        }
        for (; o < o_end; ++o) {
            keys[o] = (uint32_t)(V.super_base + y0 * V.nsx + x0);
            vals[o] = r;
        }
    }
}

cudaError_t launch_emit_supers(const uint32_t* order, const uint32_t* offsets, long long n_rec,
                               const Records rec, const ViewDev* views, int n_views, int sx,
                               int sy, int tile_w, int tile_h, int num_sms, uint32_t* keys,
                               uint32_t* vals, cudaStream_t s, const unsigned long long* n_dev) {
    if (n_rec <= 0) return cudaSuccess;
    long long blocks = div_up(n_rec, 256);
    if (blocks > (long long)num_sms * 16) blocks = (long long)num_sms * 16;
    note_launch();
    if (sx == 4 && sy == 4)
        emit_supers_kernel<4, 4><<<(int)blocks, 256, 0, s>>>(order, offsets, n_rec, rec, views,
                                                             n_views, tile_w, tile_h, keys, vals,
                                                             n_dev);
    else if (sx == 2 && sy == 8)
        emit_supers_kernel<2, 8><<<(int)blocks, 256, 0, s>>>(order, offsets, n_rec, rec, views,
                                                             n_views, tile_w, tile_h, keys, vals,
                                                             n_dev);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

__device__ __forceinline__ int find_view_by_super(const ViewDev* views, int n_views, int sup) {
    int lo = 0, hi = n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (views[mid].super_base <= sup) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Spread the 16 mask bits of m over the 16 bytes of out[0..3] (bit 4k+e of m
// becomes byte e of out[k]), so that a warp sum of out counts, per bit, the
// lanes that have it set (at most 32 per byte).
__device__ __forceinline__ void spread_mask(unsigned m, unsigned out[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned v = (m >> (4 * k)) & 0xfu;
        out[k] = (v & 1u) | ((v & 2u) << 7) | ((v & 4u) << 14) | ((v & 8u) << 21);
    }
}

// Per-tile lists of one part of one super tile (NW warps a block). Without
// SPLIT every super tile is one block (block = super tile). With SPLIT the
// super tiles of view v are cut into expand_view_parts(its super
// tiles) parts each: the view's blocks follow those of the views before it,
// its super tiles in order and each one's parts in order, and its slots of
// the per-(tile, part) counts follow theirs likewise (tile by tile, parts
// inner). A part is a consecutive run of the super tile's depth-ordered keys,
// which the block takes in chunks of one key per thread, warp w holding keys
// [32w, 32w + 32) of a chunk. For each chunk:
//  - every warp counts, per tile bit, its keys with the bit set (the spread
//    mask summed over the warp: four warp reductions for 16 tiles);
//  - the counting pass adds the counts up per tile and writes the part's
//    count of each tile to its slot of tcount;
//  - the writing pass takes, per tile, the count of earlier warps of the chunk
//    plus the part's running total as the warp's offset and appends its keys
//    with the bit set at offset + (rank among the warp's set lanes). The
//    offsets come from the exclusive scan of tcount, whose slots run view by
//    view, tile by tile and part by part in key order, so every tile's list is
//    contiguous, in tile order, and keeps the depth order whatever the number
//    of parts. The last part writes the tiles' ranges (never past cap).
template <int SX, int SY, int NW, bool WRITE, bool SPLIT>
__global__ void __launch_bounds__(NW * 32)
expand_tiles_kernel(const int2* __restrict__ sranges, const uint32_t* __restrict__ skeys,
                    const uint32_t* __restrict__ svals, const ViewDev* __restrict__ views,
                    int n_views, int num_sms, uint32_t* __restrict__ tcount,
                    const uint32_t* __restrict__ toff, uint32_t* __restrict__ vals, long long cap,
                    int2* __restrict__ ranges, const uint32_t* __restrict__ sort_err) {
    static_assert(SX * SY == 16, "16 tiles per super tile");
    constexpr int NT = NW * 32;
    __shared__ __align__(16) uint32_t s_cnt[NW][4];
    int vi, sup, part = 0, parts = 1;
    long long slot_base;  // the view's first slot of tcount / toff
    if (SPLIT) {
        // the view holding this block, from the views' block counts
        int bb = 0;
        slot_base = 0;
        for (vi = 0;; ++vi) {
            const ViewDev& U = views[vi];
            parts = expand_view_parts(U.nsx * U.nsy, num_sms);
            const int nb = U.nsx * U.nsy * parts;
            if ((int)blockIdx.x < bb + nb || vi == n_views - 1) break;
            bb += nb;
            slot_base += (long long)U.ntx * U.nty * parts;
        }
        const int local = (int)blockIdx.x - bb;
        const int sl = local / parts;
        part = local - sl * parts;
        sup = views[vi].super_base + sl;
    } else {
        sup = blockIdx.x;
        vi = find_view_by_super(views, n_views, sup);
        slot_base = views[vi].tile_base;
    }
    const ViewDev& V = views[vi];
    const int ls = sup - V.super_base;
    const int tx0 = (ls % V.nsx) * SX, ty0 = (ls / V.nsx) * SY;
    const int2 sr = sranges[sup];
    // a super-key sort whose look-back wait ran out leaves stale keys and
    // values: every tile then gets an empty list (the call reports the failure)
    const bool sort_failed = sort_err && *sort_err != 0u;
    const int Ls = sort_failed ? 0 : sr.y - sr.x;
    // this part's run of the super tile's keys: [p seg, (p + 1) seg) within Ls
    const int seg = (Ls + parts - 1) / parts;
    const int p0 = min(part * seg, Ls), p1 = min(p0 + seg, Ls);
    const int b = sr.x + p0, L = p1 - p0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    // lane t < 16 of every warp tracks tile t of the super tile
    const int ltx = tx0 + (lane & 15) % SX, lty = ty0 + (lane & 15) / SX;
    const bool lvalid = lane < 16 && ltx < V.ntx && lty < V.nty;
    const int ltile = V.tile_base + lty * V.ntx + ltx;
    // offsets in 32 bits: a batch holds fewer than 2^31 tile keys (checked when
    // it is sized), so cap and every offset below fit
    const uint32_t cap32 = (uint32_t)(cap < 0x7fffffffLL ? cap : 0x7fffffffLL);
    // this tile's first slot of tcount / toff, and this part's
    const long long tslot0 = slot_base + (long long)(ltile - V.tile_base) * parts;
    const long long lslot = tslot0 + part;
    uint32_t run = (WRITE && lvalid) ? toff[lslot] : 0u;  // tile's next offset
    uint32_t total = 0;                                  // counting pass
    for (int c0 = 0; c0 < L; c0 += NT) {
        const int i = c0 + threadIdx.x;
        unsigned m = 0;
        uint32_t r = 0;
        if (i < L) {
            m = skeys[b + i] >> 16;
            if (WRITE) r = svals[b + i];
        }
        unsigned sp[4];
        spread_mask(m, sp);
#pragma unroll
        for (int k = 0; k < 4; ++k) sp[k] = __reduce_add_sync(0xffffffffu, sp[k]);
        if (lane == 0)
            *reinterpret_cast<uint4*>(s_cnt[warp]) = make_uint4(sp[0], sp[1], sp[2], sp[3]);
        __syncthreads();
        // lane t < 16: tile t's count in the warps before this one, and in the chunk
        uint32_t before = 0, chunk = 0;
        if (lane < 16) {
            const int k = lane >> 2, sh = 8 * (lane & 3);
            for (int w = 0; w < NW; ++w) {
                const uint32_t c = (s_cnt[w][k] >> sh) & 0xffu;
                before += w < warp ? c : 0;
                chunk += c;
            }
        }
        if (WRITE) {
            const uint32_t base = run + before;
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const bool hit = (m >> t) & 1u;
                const unsigned bal = __ballot_sync(0xffffffffu, hit);
                const uint32_t o = __shfl_sync(0xffffffffu, base, t) + (uint32_t)__popc(bal & lt);
                if (hit && o < cap32) vals[o] = r;
            }
            run += chunk;
        } else {
            total += chunk;
        }
        __syncthreads();
    }
    if (warp == 0 && lvalid) {
        if (WRITE) {
            if (part == parts - 1) {
                const uint32_t s0 = toff[tslot0];
                ranges[ltile] = make_int2((int)(s0 < cap32 ? s0 : cap32),
                                          (int)(run < cap32 ? run : cap32));
            }
        } else {
            tcount[lslot] = (uint32_t)total;
        }
    }
}

template <int NW, bool WRITE>
static void expand_shape(const int2* sranges, const uint32_t* skeys, const uint32_t* svals,
                         const ViewDev* views, int n_views, const ExpandPlan& xp, int tile_w,
                         int num_sms, uint32_t* tcount, const uint32_t* toff, uint32_t* vals,
                         long long cap, int2* ranges, const uint32_t* sort_err, cudaStream_t s) {
    if (tile_w == 32 && xp.split)
        expand_tiles_kernel<2, 8, NW, WRITE, true><<<xp.blocks, NW * 32, 0, s>>>(
            sranges, skeys, svals, views, n_views, num_sms, tcount, toff, vals, cap, ranges,
            sort_err);
    else if (tile_w == 32)
        expand_tiles_kernel<2, 8, NW, WRITE, false><<<xp.blocks, NW * 32, 0, s>>>(
            sranges, skeys, svals, views, n_views, num_sms, tcount, toff, vals, cap, ranges,
            sort_err);
    else if (xp.split)
        expand_tiles_kernel<4, 4, NW, WRITE, true><<<xp.blocks, NW * 32, 0, s>>>(
            sranges, skeys, svals, views, n_views, num_sms, tcount, toff, vals, cap, ranges,
            sort_err);
    else
        expand_tiles_kernel<4, 4, NW, WRITE, false><<<xp.blocks, NW * 32, 0, s>>>(
            sranges, skeys, svals, views, n_views, num_sms, tcount, toff, vals, cap, ranges,
            sort_err);
}

// A block's time is its run of keys. One block per super tile suits a grid of
// many super tiles with short lists (a training window: 40 views, 95 super
// tiles per SM, about 570 super keys per super tile); a grid of few super
// tiles, or a serving batch of up to 16 views whose super tiles hold thousands
// of keys, leaves SMs waiting on its longest lists -- longest in its smallest
// views -- so each view's super tiles are cut into expand_view_parts parts:
// always below 16 super tiles per SM, and below 48 when the lists average at
// least 2048 keys. (Each split block walks the views' part counts to find its
// own, and the per-block fixed work grows with the parts; on the training
// window that costs more than the shorter lists save.)
ExpandPlan expand_plan(const ViewDev* views, int n_views, long long total_supers,
                       long long total_tiles, long long super_keys, int num_sms) {
    ExpandPlan xp{};
    xp.split = n_views <= 64 &&
               (total_supers < 16LL * num_sms ||
                (total_supers < 48LL * num_sms && super_keys >= 2048LL * total_supers));
    if (!xp.split) {
        xp.blocks = total_supers;
        xp.slots = total_tiles;
        return xp;
    }
    for (int v = 0; v < n_views; ++v) {
        const int p = expand_view_parts(views[v].nsx * views[v].nsy, num_sms);
        xp.blocks += (long long)views[v].nsx * views[v].nsy * p;
        xp.slots += (long long)views[v].ntx * views[v].nty * p;
    }
    return xp;
}

// Warps per super tile: a block's time is its super tile's list, so a grid of
// few super tiles (a batch of one or a few views) takes more warps per list,
// and a grid of many (a training window) fewer, leaving no warp idle on the
// short lists. Measured (ranges stage, ms): one 1280x720 view (240 super
// tiles) 0.282 / 0.180 / 0.155 at 4 / 8 / 16 warps; three (720) 0.365 / 0.237
// / 0.311; eight (1,920) 0.480 / 0.460 / 0.454; 40 views of 1352x1014
// (14,080) 0.191 / 0.226 / 0.323.
int expand_warps(int total_supers, int num_sms) {
    if (total_supers < 2 * num_sms) return 16;
    if (total_supers < 16 * num_sms) return 8;
    return 4;
}

template <bool WRITE>
static cudaError_t run_expand(const int2* sranges, const uint32_t* skeys, const uint32_t* svals,
                              const ViewDev* views, int n_views, const ExpandPlan& xp,
                              int tile_w, int num_sms, uint32_t* tcount, const uint32_t* toff,
                              uint32_t* vals, long long cap, int2* ranges,
                              const uint32_t* sort_err, cudaStream_t s) {
    if (xp.blocks <= 0) return cudaSuccess;
    if (xp.blocks > 0x7fffffffLL || n_views <= 0) return cudaErrorInvalidValue;
    note_launch();
    const int nw = expand_warps((int)xp.blocks, num_sms);
    if (nw == 16)
        expand_shape<16, WRITE>(sranges, skeys, svals, views, n_views, xp, tile_w, num_sms,
                                tcount, toff, vals, cap, ranges, sort_err, s);
    else if (nw == 8)
        expand_shape<8, WRITE>(sranges, skeys, svals, views, n_views, xp, tile_w, num_sms,
                               tcount, toff, vals, cap, ranges, sort_err, s);
    else
        expand_shape<4, WRITE>(sranges, skeys, svals, views, n_views, xp, tile_w, num_sms,
                               tcount, toff, vals, cap, ranges, sort_err, s);
    return cudaGetLastError();
}

// CUDA loads a kernel's module at its first launch unless told otherwise.
// The expansion picks one of 24 instantiations by batch shape, so a serving
// loop would meet some of them for the first time mid-run and stall on the
// load; querying each one's attributes loads them all up front.
template <int SX, int SY, int NW>
static cudaError_t load_expand_shape() {
    cudaFuncAttributes fa;
    cudaError_t e;
    if ((e = cudaFuncGetAttributes(&fa, expand_tiles_kernel<SX, SY, NW, false, false>)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncGetAttributes(&fa, expand_tiles_kernel<SX, SY, NW, false, true>)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncGetAttributes(&fa, expand_tiles_kernel<SX, SY, NW, true, false>)) !=
        cudaSuccess)
        return e;
    return cudaFuncGetAttributes(&fa, expand_tiles_kernel<SX, SY, NW, true, true>);
}

cudaError_t load_expand_kernels() {
    cudaError_t e;
    if ((e = load_expand_shape<4, 4, 4>()) != cudaSuccess) return e;
    if ((e = load_expand_shape<4, 4, 8>()) != cudaSuccess) return e;
    if ((e = load_expand_shape<4, 4, 16>()) != cudaSuccess) return e;
    if ((e = load_expand_shape<2, 8, 4>()) != cudaSuccess) return e;
    if ((e = load_expand_shape<2, 8, 8>()) != cudaSuccess) return e;
    return load_expand_shape<2, 8, 16>();
}

cudaError_t launch_expand_count(const int2* sranges, const uint32_t* skeys, const ViewDev* views,
                                int n_views, const ExpandPlan& xp, int tile_w, int num_sms,
                                uint32_t* tcount, const uint32_t* sort_err, cudaStream_t s) {
    return run_expand<false>(sranges, skeys, nullptr, views, n_views, xp, tile_w, num_sms,
                             tcount, nullptr, nullptr, 0, nullptr, sort_err, s);
}

cudaError_t launch_expand_write(const int2* sranges, const uint32_t* skeys, const uint32_t* svals,
                                const ViewDev* views, int n_views, const ExpandPlan& xp,
                                int tile_w, int num_sms, const uint32_t* toff, uint32_t* vals,
                                long long cap, int2* ranges, const uint32_t* sort_err,
                                cudaStream_t s) {
    return run_expand<true>(sranges, skeys, svals, views, n_views, xp, tile_w, num_sms, nullptr,
                            toff, vals, cap, ranges, sort_err, s);
}

// sranges[t] = [first, last+1) of super tile t (the low 16 key bits) in the
// sorted super keys (sranges zeroed before). Four consecutive keys a thread
// (one 16-byte load; the key buffers are 16-byte aligned) and the keys on
// either side.
__global__ void super_ranges_kernel(const uint32_t* __restrict__ keys, long long cap,
                                    long long n_supers, int2* __restrict__ ranges,
                                    const unsigned long long* __restrict__ n_dev) {
    const long long n = dev_count(cap, n_dev);
    const long long i0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (i0 >= n) return;
    constexpr uint32_t kNone = 0xffffffffu;  // no key: differs from every 16-bit id
    uint32_t t[6];
    t[0] = i0 > 0 ? (keys[i0 - 1] & 0xffffu) : kNone;
    if (i0 + 4 <= n) {
        const uint4 v = *reinterpret_cast<const uint4*>(keys + i0);
        t[1] = v.x & 0xffffu;
        t[2] = v.y & 0xffffu;
        t[3] = v.z & 0xffffu;
        t[4] = v.w & 0xffffu;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) t[j + 1] = i0 + j < n ? (keys[i0 + j] & 0xffffu) : kNone;
    }
    t[5] = i0 + 4 < n ? (keys[i0 + 4] & 0xffffu) : kNone;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t c = t[j + 1];
        if (c >= (uint32_t)n_supers) continue;  // also past n (kNone)
        if (t[j] != c) ranges[c].x = (int)(i0 + j);
        if (t[j + 2] != c) ranges[c].y = (int)(i0 + j + 1);
    }
}

cudaError_t launch_super_ranges(const uint32_t* keys, long long n, long long n_supers,
                                int2* ranges, cudaStream_t s, const unsigned long long* n_dev) {
    if (n <= 0) return cudaSuccess;
    note_launch();
    super_ranges_kernel<<<div_up(div_up(n, 4), 256), 256, 0, s>>>(keys, n, n_supers, ranges,
                                                                   n_dev);
    return cudaGetLastError();
}

}  // namespace swgs
