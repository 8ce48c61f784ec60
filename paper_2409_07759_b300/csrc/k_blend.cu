// k_blend.cu -- per-tile front-to-back alpha compositing (Sec. 2.1 Eq. 3) and
// its reverse-order backward (Alg. 1 loss.backward).
//
// Persistent launch: a grid of (SMs x resident blocks) pulls (view, tile) work
// items from one atomic counter, over every view of the batch at once. One
// thread per pixel; Gaussians of the tile's depth-sorted list are staged in
// shared memory BATCH at a time (converted once per block to the log2-domain
// form the inner loop needs). A thread leaves the inner loop as soon as its
// pixel saturates, so a warp stops when all 32 of its pixels are done and the
// block stops staging when all its pixels are.
//
// The backward walks the list from the block's largest last-contributor index
// down to the front, recovering each T from the saved final transmittance by
// division, and reduces the nine 2D gradients of each Gaussian across the warp
// (a transposing butterfly, 14 shuffles for 9 values), then across the block
// in shared memory, before one vector atomic per Gaussian per tile.
#include "swgs_internal.cuh"

namespace swgs {

__device__ __forceinline__ void stage_gaussian(const Records& rec, uint32_t r, float4* s0,
                                               float4* s1, float4* s2) {
    const float4 A = rec.a[r];
    const float4 B = rec.b[r];
    const float4 Cc = rec.c[r];
    *s0 = make_float4(A.x, A.y, __fmul_rn(B.x, -0.5f * kLog2e), __fmul_rn(B.y, -kLog2e));
    *s1 = make_float4(__fmul_rn(B.z, -0.5f * kLog2e), __log2f(A.z), A.z, 0.f);
    *s2 = Cc;
}

template <int TW, int TH, int BATCH>
__global__ void __launch_bounds__(TW * TH) blend_fwd_kernel(BlendArgs a) {
    constexpr int NT = TW * TH;
    __shared__ float4 s0[BATCH], s1[BATCH], s2[BATCH];
    __shared__ int s_item;
    const int tid = threadIdx.x;
    const int lx = tid % TW, ly = tid / TW;
    unsigned long long pairs = 0;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(a.work_counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= a.total_tiles) break;
        const int vi = find_view_by_tile(a.views, a.n_views, item);
        const ViewDev& V = a.views[vi];
        const int W = V.W, H = V.H;
        const int lt = item - V.tile_base;
        const int x = (lt % V.ntx) * TW + lx, y = (lt / V.ntx) * TH + ly;
        const bool inside = x < W && y < H;
        const float px = (float)x + 0.5f, py = (float)y + 0.5f;
        const int2 rg = a.ranges[item];
        float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
        int last = 0;
        bool done = !inside;
        int stop = rg.y;
        for (int b0 = rg.x; b0 < rg.y; b0 += BATCH) {
            if (__syncthreads_count(done) == NT) break;
            for (int k = tid; k < BATCH; k += NT) {
                const int idx = b0 + k;
                if (idx < rg.y) stage_gaussian(a.rec, a.vals[idx], &s0[k], &s1[k], &s2[k]);
            }
            __syncthreads();
            const int cnt = min(BATCH, rg.y - b0);
            if (!done) {
                for (int j = 0; j < cnt; ++j) {
                    const float4 g0 = s0[j];
                    const float2 g1 = make_float2(s1[j].x, s1[j].y);
                    float dx, dy, au;
                    const float q = pair_q(px, py, g0, g1.x, &dx, &dy);
                    if (q < kQMin) continue;
                    const float al = pair_alpha(q, g1.y, &au);
                    if (al < kAlphaMin) continue;
                    const float tT = __fmul_rn(T, __fsub_rn(1.f, al));
                    if (tT < kTStop) {
                        done = true;
                        stop = b0 + j;
                        break;
                    }
                    const float w = __fmul_rn(al, T);
                    const float4 c = s2[j];
                    C0 = __fmaf_rn(c.x, w, C0);
                    C1 = __fmaf_rn(c.y, w, C1);
                    C2 = __fmaf_rn(c.z, w, C2);
                    T = tT;
                    last = b0 + j - rg.x + 1;
                }
            }
        }
        if (inside) {
            const long long hw = (long long)W * H, p = (long long)y * W + x;
            V.out_rgb[p] = C0 + T * V.bg[0];
            V.out_rgb[hw + p] = C1 + T * V.bg[1];
            V.out_rgb[2 * hw + p] = C2 + T * V.bg[2];
            if (V.out_T) V.out_T[p] = T;
            if (a.T) a.T[V.pix_base + p] = T;
            if (a.last) a.last[V.pix_base + p] = last;
            pairs += (unsigned long long)((stop < rg.y ? stop + 1 : rg.y) - rg.x);
        }
        __syncthreads();
    }
    if (a.pairs) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
        if ((tid & 31) == 0 && pairs) atomicAdd(a.pairs, pairs);
    }
}

// Sum 9 per-lane values over the warp and add the sums to acc[0..9) in
// shared memory. Steps 1-3 halve the values each lane holds while doubling
// the lanes summed, so lane 4m ends with value m (m < 8); value 8 takes a
// plain butterfly.
__device__ __forceinline__ void warp_sum9_to_smem(const float* v, float* acc) {
    const unsigned F = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool bA = lane & 16, bB = lane & 8, bC = lane & 4;
    float w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float send = bA ? v[k] : v[k + 4];
        const float keep = bA ? v[k + 4] : v[k];
        w[k] = keep + __shfl_xor_sync(F, send, 16);
    }
    float x[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float send = bB ? w[k] : w[k + 2];
        const float keep = bB ? w[k + 2] : w[k];
        x[k] = keep + __shfl_xor_sync(F, send, 8);
    }
    float y = (bC ? x[1] : x[0]) + __shfl_xor_sync(F, bC ? x[0] : x[1], 4);
    y += __shfl_xor_sync(F, y, 2);
    y += __shfl_xor_sync(F, y, 1);
    float v8 = v[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v8 += __shfl_xor_sync(F, v8, o);
    if ((lane & 3) == 0 && y != 0.f) atomicAdd(&acc[lane >> 2], y);
    if (lane == 0 && v8 != 0.f) atomicAdd(&acc[8], v8);
}

template <int TW, int TH, int BATCH>
__global__ void __launch_bounds__(TW * TH) blend_bwd_kernel(BlendArgs a) {
    constexpr int NT = TW * TH;
    __shared__ float4 s0[BATCH], s1[BATCH], s2[BATCH], s3[BATCH];
    __shared__ uint32_t s_rec[BATCH];
    __shared__ float s_acc[BATCH * 9];
    __shared__ int s_item, s_maxlast;
    const int tid = threadIdx.x;
    const int lx = tid % TW, ly = tid / TW;
    for (int k = tid; k < BATCH * 9; k += NT) s_acc[k] = 0.f;
    for (;;) {
        if (tid == 0) { s_item = atomicAdd(a.work_counter, 1); s_maxlast = 0; }
        __syncthreads();
        const int item = s_item;
        if (item >= a.total_tiles) break;
        const int vi = find_view_by_tile(a.views, a.n_views, item);
        const ViewDev& V = a.views[vi];
        const int W = V.W, H = V.H;
        const int lt = item - V.tile_base;
        const int x = (lt % V.ntx) * TW + lx, y = (lt / V.ntx) * TH + ly;
        const bool inside = x < W && y < H;
        const float px = (float)x + 0.5f, py = (float)y + 0.5f;
        const int2 rg = a.ranges[item];
        float T = 1.f, dL0 = 0.f, dL1 = 0.f, dL2 = 0.f;
        int last = 0;
        if (inside) {
            const long long hw = (long long)W * H, p = (long long)y * W + x;
            T = a.T[V.pix_base + p];
            last = a.last[V.pix_base + p];
            dL0 = V.dL[p];
            dL1 = V.dL[hw + p];
            dL2 = V.dL[2 * hw + p];
        }
        float B0 = V.bg[0], B1 = V.bg[1], B2 = V.bg[2];
        if (last > 0) atomicMax(&s_maxlast, last);
        __syncthreads();
        const int end = rg.x + s_maxlast;
        for (int b1 = end; b1 > rg.x; b1 -= BATCH) {
            const int b0 = max(rg.x, b1 - BATCH);
            const int cnt = b1 - b0;
            __syncthreads();
            for (int k = tid; k < cnt; k += NT) {
                const uint32_t r = a.vals[b0 + k];
                s_rec[k] = r;
                stage_gaussian(a.rec, r, &s0[k], &s1[k], &s2[k]);
                s3[k] = a.rec.b[r];
            }
            __syncthreads();
            for (int j = cnt - 1; j >= 0; --j) {
                const int pos = b0 + j - rg.x;
                float g[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) g[k] = 0.f;
                bool contrib = false;
                if (pos < last) {
                    const float4 g0 = s0[j];
                    const float4 g1 = s1[j];
                    float dx, dy, au;
                    const float q = pair_q(px, py, g0, g1.x, &dx, &dy);
                    if (q >= kQMin) {
                        const float al = pair_alpha(q, g1.y, &au);
                        if (al >= kAlphaMin) {
                            contrib = true;
                            const float om = __fsub_rn(1.f, al);
                            T = __fdividef(T, om);
                            const float w = al * T;
                            const float4 c = s2[j];
                            g[6] = w * dL0;
                            g[7] = w * dL1;
                            g[8] = w * dL2;
                            const float ga = T * (dL0 * (c.x - B0) + dL1 * (c.y - B1) + dL2 * (c.z - B2));
                            B0 = al * c.x + om * B0;
                            B1 = al * c.y + om * B1;
                            B2 = al * c.z + om * B2;
                            if (au <= kAlphaMax) {
                                const float4 cn = s3[j];
                                g[5] = ga * au / g1.z;
                                const float gm = -0.5f * au * ga;
                                g[2] = gm * dx * dx;
                                g[3] = 2.f * gm * dx * dy;
                                g[4] = gm * dy * dy;
                                g[0] = -2.f * gm * (cn.x * dx + cn.y * dy);
                                g[1] = -2.f * gm * (cn.y * dx + cn.z * dy);
                            }
                        }
                    }
                }
                if (__any_sync(0xffffffffu, contrib)) warp_sum9_to_smem(g, &s_acc[j * 9]);
            }
            __syncthreads();
            for (int k = tid; k < cnt; k += NT) {
                float* acc = &s_acc[k * 9];
                float* dst = a.grad2d + 12ll * s_rec[k];
                bool nz = false;
#pragma unroll
                for (int e = 0; e < 9; ++e) nz |= acc[e] != 0.f;
                if (nz) {
                    red_add_v4(dst, acc[0], acc[1], acc[2], acc[3]);
                    red_add_v4(dst + 4, acc[4], acc[5], acc[6], acc[7]);
                    red_add(dst + 8, acc[8]);
#pragma unroll
                    for (int e = 0; e < 9; ++e) acc[e] = 0.f;
                }
            }
        }
        __syncthreads();
    }
}

template <int TW, int TH, int BATCH>
static cudaError_t run_fwd(const BlendArgs& a, int grid, cudaStream_t s) {
    blend_fwd_kernel<TW, TH, BATCH><<<grid, TW * TH, 0, s>>>(a);
    return cudaGetLastError();
}

template <int TW, int TH, int BATCH>
static cudaError_t run_bwd(const BlendArgs& a, int grid, cudaStream_t s) {
    blend_bwd_kernel<TW, TH, BATCH><<<grid, TW * TH, 0, s>>>(a);
    return cudaGetLastError();
}

template <int TW, int TH, int BATCH>
static int occ(bool bwd) {
    int n = 0;
    if (bwd)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, blend_bwd_kernel<TW, TH, BATCH>, TW * TH, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, blend_fwd_kernel<TW, TH, BATCH>, TW * TH, 0);
    return n < 1 ? 1 : n;
}

#define SWGS_TILE_DISPATCH(FN, ...)                                                  \
    do {                                                                             \
        if (tile_w == 16 && tile_h == 16) {                                          \
            if (batch == 32) return FN<16, 16, 32>(__VA_ARGS__);                     \
            if (batch == 64) return FN<16, 16, 64>(__VA_ARGS__);                     \
            if (batch == 128) return FN<16, 16, 128>(__VA_ARGS__);                   \
            if (batch == 256) return FN<16, 16, 256>(__VA_ARGS__);                   \
        } else if (tile_w == 8 && tile_h == 8) {                                     \
            if (batch == 32) return FN<8, 8, 32>(__VA_ARGS__);                       \
            if (batch == 64) return FN<8, 8, 64>(__VA_ARGS__);                       \
            if (batch == 128) return FN<8, 8, 128>(__VA_ARGS__);                     \
            if (batch == 256) return FN<8, 8, 256>(__VA_ARGS__);                     \
        } else if (tile_w == 32 && tile_h == 8) {                                    \
            if (batch == 32) return FN<32, 8, 32>(__VA_ARGS__);                      \
            if (batch == 64) return FN<32, 8, 64>(__VA_ARGS__);                      \
            if (batch == 128) return FN<32, 8, 128>(__VA_ARGS__);                    \
            if (batch == 256) return FN<32, 8, 256>(__VA_ARGS__);                    \
        }                                                                            \
    } while (0)

cudaError_t launch_blend_fwd(const BlendArgs& a, int tile_w, int tile_h, int batch, int grid,
                             cudaStream_t s) {
    if (a.total_tiles <= 0) return cudaSuccess;
    SWGS_TILE_DISPATCH(run_fwd, a, grid, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_blend_bwd(const BlendArgs& a, int tile_w, int tile_h, int batch, int grid,
                             cudaStream_t s) {
    if (a.total_tiles <= 0) return cudaSuccess;
    SWGS_TILE_DISPATCH(run_bwd, a, grid, s);
    return cudaErrorInvalidValue;
}

int blend_blocks_per_sm(int tile_w, int tile_h, int batch, bool backward) {
    SWGS_TILE_DISPATCH(occ, backward);
    return 1;
}

}  // namespace swgs
