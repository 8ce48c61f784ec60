// k_blend.cu -- per-tile front-to-back alpha compositing (Sec. 2.1 Eq. 3) and
// its reverse-order backward (Alg. 1 loss.backward).
//
// Persistent launch: a grid of (SMs x resident blocks) pulls (view, tile) work
// items from one atomic counter, over every view of the batch at once. Each
// thread owns PPT vertically adjacent pixels of the tile; the Gaussians of the
// tile's depth-sorted list are staged in shared memory BATCH at a time
// (converted once per block to the log2-domain form the inner loop needs).
// The inner loops are branch-free: every lane of a warp walks the list in
// lockstep with predicated updates, so no lane diverges at the per-pair
// tests, and the warp leaves as soon as a vote says all its pixels saturated;
// the block stops staging when all its pixels have.
//
// The backward walks the list from the block's largest last-contributor index
// down to the front, recovering each T from the saved final transmittance by
// division. Per Gaussian it accumulates nine moments -- sum of gm, gm dx,
// gm dy, gm dx^2, gm dx dy, gm dy^2 (gm = dL/dm) and of the colour weights --
// over the thread's pixels, sums them across the warp (a transposing butterfly,
// 14 shuffles for 9 values) and across the block in shared memory, and turns
// them into the nine 2D gradients (centre, conic, opacity, colour) once per
// Gaussian per tile before one vector atomic.
#include "swgs_internal.cuh"

namespace swgs {

__device__ __forceinline__ void stage_gaussian(const Records& rec, uint32_t r, float4* s0,
                                               float4* s1, float4* s2) {
    const float4 A = rec.a[r];
    const float4 B = rec.b[r];
    const float4 Cc = rec.c[r];
    *s0 = make_float4(A.x, A.y, __fmul_rn(B.x, -0.5f * kLog2e), __fmul_rn(B.y, -kLog2e));
    const float lo = __log2f(A.z);
    *s1 = make_float4(__fmul_rn(B.z, -0.5f * kLog2e), lo, pair_qmin(lo), 0.f);
    *s2 = Cc;
}

template <int TW, int TH, int PPT>
struct TileGeom {
    static constexpr int NT = TW * TH / PPT;
    static_assert(NT % 32 == 0, "a tile block must be whole warps");
    static_assert(TH % PPT == 0, "pixels per thread must divide the tile height");
};

constexpr int kFwdUnroll = 8;
constexpr int kBwdUnroll = 2;

template <int TW, int TH, int BATCH, int PPT, bool COUNT>
__global__ void __launch_bounds__(TW * TH / PPT) blend_fwd_kernel(BlendArgs a) {
    constexpr int NT = TileGeom<TW, TH, PPT>::NT;
    __shared__ float4 s0[BATCH], s1[BATCH], s2[BATCH];
    __shared__ int s_item;
    const unsigned F = 0xffffffffu;
    const int tid = threadIdx.x;
    const int lx = tid % TW, ly = (tid / TW) * PPT;
    unsigned long long pairs = 0;
    float l1 = 0.f;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(a.work_counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= a.total_tiles) break;
        const int vi = find_view_by_tile(a.views, a.n_views, item);
        const ViewDev& V = a.views[vi];
        const int W = V.W, H = V.H;
        const int lt = item - V.tile_base;
        const int x = (lt % V.ntx) * TW + lx, y0 = (lt / V.ntx) * TH + ly;
        const float px = (float)x + 0.5f;
        const int2 rg = a.ranges[item];
        float T[PPT], C0[PPT], C1[PPT], C2[PPT], py[PPT];
        int last[PPT], stop[PPT];
        bool done[PPT];
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            T[p] = 1.f; C0[p] = C1[p] = C2[p] = 0.f; last[p] = 0; stop[p] = rg.y;
            py[p] = (float)(y0 + p) + 0.5f;
            done[p] = !(x < W && y0 + p < H);
        }
        for (int b0 = rg.x; b0 < rg.y; b0 += BATCH) {
            bool tdone = true;
#pragma unroll
            for (int p = 0; p < PPT; ++p) tdone &= done[p];
            if (__syncthreads_count(tdone) == NT) break;
            for (int k = tid; k < BATCH; k += NT) {
                const int idx = b0 + k;
                if (idx < rg.y) stage_gaussian(a.rec, a.vals[idx], &s0[k], &s1[k], &s2[k]);
            }
            __syncthreads();
            const int cnt = min(BATCH, rg.y - b0);
            // kFwdUnroll staged Gaussians per iteration, in list order (one warp
            // vote and one loop test for all); a pixel done after one of them
            // ignores the rest
            for (int j2 = 0; j2 < cnt; j2 += kFwdUnroll) {
                if (__all_sync(F, tdone)) break;
#pragma unroll
                for (int jj = 0; jj < kFwdUnroll; ++jj) {
                const int j = j2 + jj;
                if (j >= cnt) break;
                const float4 g0 = s0[j];
                const float4 g1 = s1[j];
                const float4 c = s2[j];
                const int pos = b0 + j, pos1 = pos - rg.x + 1;
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    float dx, dy, au;
                    const float q = pair_q(px, py[p], g0, g1.x, &dx, &dy);
                    const float al = pair_alpha(q, g1.y, &au);
                    const bool ok = !done[p] && q >= g1.z;
                    // T (1 - alpha), rounded once: the stopping test
                    const float tT = __fmaf_rn(-al, T[p], T[p]);
                    const bool inc = ok && tT >= kTStop;
                    if (COUNT) stop[p] = (ok && !inc) ? pos : stop[p];
                    done[p] = done[p] || (ok && !inc);
                    const float w = __fmul_rn(inc ? al : 0.f, T[p]);
                    C0[p] = __fmaf_rn(c.x, w, C0[p]);
                    C1[p] = __fmaf_rn(c.y, w, C1[p]);
                    C2[p] = __fmaf_rn(c.z, w, C2[p]);
                    T[p] = __fsub_rn(T[p], w);
                    last[p] = inc ? pos1 : last[p];
                }
                }
                tdone = true;
#pragma unroll
                for (int p = 0; p < PPT; ++p) tdone &= done[p];
            }
        }
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int y = y0 + p;
            if (x < W && y < H) {
                const long long hw = (long long)W * H, q = (long long)y * W + x;
                const float r0 = C0[p] + T[p] * V.bg[0];
                const float r1 = C1[p] + T[p] * V.bg[1];
                const float r2 = C2[p] + T[p] * V.bg[2];
                V.out_rgb[q] = r0;
                V.out_rgb[hw + q] = r1;
                V.out_rgb[2 * hw + q] = r2;
                if (V.out_T) V.out_T[q] = T[p];
                if (a.T) a.T[V.pix_base + q] = T[p];
                if (a.last) a.last[V.pix_base + q] = last[p];
                if (COUNT)
                    pairs += (unsigned long long)((stop[p] < rg.y ? stop[p] + 1 : rg.y) - rg.x);
                if (V.target || V.target_u8) {
                    // L1 term of the loss and its gradient, sign(0) = 0
                    float t0, t1, t2;
                    if (V.target_u8) {  // k x (1/255) in FP32
                        constexpr float kInv255 = 1.0f / 255.0f;
                        t0 = __fmul_rn((float)V.target_u8[q], kInv255);
                        t1 = __fmul_rn((float)V.target_u8[hw + q], kInv255);
                        t2 = __fmul_rn((float)V.target_u8[2 * hw + q], kInv255);
                    } else {
                        t0 = V.target[q];
                        t1 = V.target[hw + q];
                        t2 = V.target[2 * hw + q];
                    }
                    const float e0 = r0 - t0, e1 = r1 - t1, e2 = r2 - t2;
                    const float s = V.l1_scale;
                    V.dL_out[q] = e0 > 0.f ? s : (e0 < 0.f ? -s : 0.f);
                    V.dL_out[hw + q] = e1 > 0.f ? s : (e1 < 0.f ? -s : 0.f);
                    V.dL_out[2 * hw + q] = e2 > 0.f ? s : (e2 < 0.f ? -s : 0.f);
                    l1 += (fabsf(e0) + fabsf(e1) + fabsf(e2)) * s;
                }
            }
        }
        __syncthreads();
    }
    if (a.loss) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l1 += __shfl_xor_sync(F, l1, o);
        if ((tid & 31) == 0 && l1 != 0.f) atomicAdd(a.loss, l1);
    }
    if (COUNT) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(F, pairs, o);
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

template <int TW, int TH, int BATCH, int PPT>
__global__ void __launch_bounds__(TW * TH / PPT) blend_bwd_kernel(BlendArgs a) {
    constexpr int NT = TileGeom<TW, TH, PPT>::NT;
    __shared__ float4 s0[BATCH], s1[BATCH], s2[BATCH];
    __shared__ uint32_t s_rec[BATCH];
    __shared__ float s_acc[BATCH * 9];
    __shared__ int s_item, s_maxlast;
    const unsigned F = 0xffffffffu;
    const int tid = threadIdx.x;
    const int lx = tid % TW, ly = (tid / TW) * PPT;
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
        const int x = (lt % V.ntx) * TW + lx, y0 = (lt / V.ntx) * TH + ly;
        const float px = (float)x + 0.5f;
        const int2 rg = a.ranges[item];
        // Per pixel: T (recovered back to front), dL/dC, and D = sum_ch dL_ch B_ch with
        // B the colour composited behind the current Gaussian (starts at the
        // background). With E = sum_ch dL_ch c_ch: dL/dalpha = T (E - D) and the
        // step to the next Gaussian in front is D' = D + alpha (E - D).
        float T[PPT], dL0[PPT], dL1[PPT], dL2[PPT], D[PPT], py[PPT];
        int last[PPT];
        int mylast = 0;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int y = y0 + p;
            py[p] = (float)y + 0.5f;
            T[p] = 1.f; dL0[p] = dL1[p] = dL2[p] = 0.f; last[p] = 0;
            if (x < W && y < H) {
                const long long hw = (long long)W * H, q = (long long)y * W + x;
                T[p] = a.T[V.pix_base + q];
                last[p] = a.last[V.pix_base + q];
                dL0[p] = V.dL[q];
                dL1[p] = V.dL[hw + q];
                dL2[p] = V.dL[2 * hw + q];
            }
            D[p] = fmaf(dL0[p], V.bg[0], fmaf(dL1[p], V.bg[1], dL2[p] * V.bg[2]));
            mylast = max(mylast, last[p]);
        }
        if (mylast > 0) atomicMax(&s_maxlast, mylast);
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
            }
            __syncthreads();
            // kBwdUnroll staged Gaussians per iteration, back to front; the
            // group is skipped when it lies beyond every pixel's last
            for (int j2 = cnt - 1; j2 >= 0; j2 -= kBwdUnroll) {
                if (__all_sync(F, b0 + max(j2 - kBwdUnroll + 1, 0) - rg.x >= mylast)) continue;
#pragma unroll
                for (int jj = 0; jj < kBwdUnroll; ++jj) {
                const int j = j2 - jj;
                if (j < 0) break;
                const int pos = b0 + j - rg.x;
                const float4 g0 = s0[j];
                const float4 g1 = s1[j];
                const float4 c = s2[j];
                // The thread's pixels share x, so dx is common to them: only
                // sum gm, sum gm dy and sum gm dy^2 run per pixel; the dx terms
                // are applied once below. gm here is alpha dL/dalpha (the
                // factor -1/2 of dalpha/dm is applied at the flush).
                float s0m = 0.f, sy = 0.f, syy = 0.f, m6 = 0.f, m7 = 0.f, m8 = 0.f, dx = 0.f;
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    float dy, au;
                    const float q = pair_q(px, py[p], g0, g1.x, &dx, &dy);
                    const float al = pair_alpha(q, g1.y, &au);
                    const bool ok = pos < last[p] && q >= g1.z;
                    const float a1 = ok ? al : 0.f;
                    // T before this Gaussian, recovered from the T after it (a
                    // pair that does not count has a1 = 0 and leaves T as is)
                    T[p] = __fdividef(T[p], __fsub_rn(1.f, a1));
                    const float w = a1 * T[p];
                    m6 = fmaf(w, dL0[p], m6);
                    m7 = fmaf(w, dL1[p], m7);
                    m8 = fmaf(w, dL2[p], m8);
                    const float e = fmaf(dL0[p], c.x, fmaf(dL1[p], c.y, dL2[p] * c.z));
                    const float diff = e - D[p];
                    const float ga = T[p] * diff;
                    D[p] = fmaf(a1, diff, D[p]);
                    // dalpha/dm needs the unclamped alpha: a1 = au when it counts
                    const float gm = au <= kAlphaMax ? a1 * ga : 0.f;
                    const float gy = gm * dy;
                    s0m += gm;
                    sy += gy;
                    syy = fmaf(gy, dy, syy);
                }
                // a Gaussian no pixel of the warp counted leaves every sum at zero
                const bool any = s0m != 0.f || m6 != 0.f || m7 != 0.f || m8 != 0.f;
                if (__any_sync(F, any)) {
                    float m[9];
                    m[0] = s0m;
                    m[1] = s0m * dx;
                    m[2] = sy;
                    m[3] = m[1] * dx;
                    m[4] = sy * dx;
                    m[5] = syy;
                    m[6] = m6;
                    m[7] = m7;
                    m[8] = m8;
                    warp_sum9_to_smem(m, &s_acc[j * 9]);
                }
                }
            }
            __syncthreads();
            for (int k = tid; k < cnt; k += NT) {
                float* acc = &s_acc[k * 9];
                bool nz = false;
#pragma unroll
                for (int e = 0; e < 9; ++e) nz |= acc[e] != 0.f;
                if (!nz) continue;
                const uint32_t r = s_rec[k];
                const float4 ra = a.rec.a[r];   // u, v, opacity, depth
                const float4 rb = a.rec.b[r];   // A, B, C
                // acc[0..5] hold sums of alpha dL/dalpha times (1, dx, dy, dx^2,
                // dx dy, dy^2); dL/dm = -1/2 of them (G = exp(-m/2)).
                // m = A dx^2 + 2B dx dy + C dy^2, dx = px - u: dm/du = -2(A dx + B dy)
                const float m1 = -0.5f * acc[1], m2 = -0.5f * acc[2];
                const float du = -2.f * (rb.x * m1 + rb.y * m2);
                const float dv = -2.f * (rb.y * m1 + rb.z * m2);
                // alpha = o G, dalpha/do = G = alpha/o
                const float dop = acc[0] / ra.z;
                float* dst = a.grad2d + 12ll * r;
                red_add_v4(dst, du, dv, -0.5f * acc[3], -acc[4]);
                red_add_v4(dst + 4, -0.5f * acc[5], dop, acc[6], acc[7]);
                red_add(dst + 8, acc[8]);
#pragma unroll
                for (int e = 0; e < 9; ++e) acc[e] = 0.f;
            }
        }
        __syncthreads();
    }
}

template <int TW, int TH, int BATCH, int PPT>
static cudaError_t run_fwd(const BlendArgs& a, int grid, cudaStream_t s) {
    note_launch();
    if (a.pairs)
        blend_fwd_kernel<TW, TH, BATCH, PPT, true><<<grid, TW * TH / PPT, 0, s>>>(a);
    else
        blend_fwd_kernel<TW, TH, BATCH, PPT, false><<<grid, TW * TH / PPT, 0, s>>>(a);
    return cudaGetLastError();
}

template <int TW, int TH, int BATCH, int PPT>
static cudaError_t run_bwd(const BlendArgs& a, int grid, cudaStream_t s) {
    note_launch();
    blend_bwd_kernel<TW, TH, BATCH, PPT><<<grid, TW * TH / PPT, 0, s>>>(a);
    return cudaGetLastError();
}

template <int TW, int TH, int BATCH, int PPT>
static int occ_fwd() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, blend_fwd_kernel<TW, TH, BATCH, PPT, false>,
                                                  TW * TH / PPT, 0);
    return n < 1 ? 1 : n;
}

template <int TW, int TH, int BATCH, int PPT>
static int occ_bwd() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, blend_bwd_kernel<TW, TH, BATCH, PPT>,
                                                  TW * TH / PPT, 0);
    return n < 1 ? 1 : n;
}

#define SWGS_BATCH_DISPATCH(FN, TW, TH, PPT, ...)                  \
    do {                                                           \
        if (batch == 32) return FN<TW, TH, 32, PPT>(__VA_ARGS__);  \
        if (batch == 64) return FN<TW, TH, 64, PPT>(__VA_ARGS__);  \
        if (batch == 128) return FN<TW, TH, 128, PPT>(__VA_ARGS__); \
        if (batch == 256) return FN<TW, TH, 256, PPT>(__VA_ARGS__); \
    } while (0)

#define SWGS_TILE_DISPATCH(FN, ...)                                              \
    do {                                                                         \
        if (tile_w == 16 && tile_h == 16) {                                      \
            if (ppt == 1) SWGS_BATCH_DISPATCH(FN, 16, 16, 1, __VA_ARGS__);       \
            if (ppt == 2) SWGS_BATCH_DISPATCH(FN, 16, 16, 2, __VA_ARGS__);       \
            if (ppt == 4) SWGS_BATCH_DISPATCH(FN, 16, 16, 4, __VA_ARGS__);       \
        } else if (tile_w == 8 && tile_h == 8) {                                 \
            if (ppt == 1) SWGS_BATCH_DISPATCH(FN, 8, 8, 1, __VA_ARGS__);         \
            if (ppt == 2) SWGS_BATCH_DISPATCH(FN, 8, 8, 2, __VA_ARGS__);         \
        } else if (tile_w == 32 && tile_h == 8) {                                \
            if (ppt == 1) SWGS_BATCH_DISPATCH(FN, 32, 8, 1, __VA_ARGS__);        \
            if (ppt == 2) SWGS_BATCH_DISPATCH(FN, 32, 8, 2, __VA_ARGS__);        \
            if (ppt == 4) SWGS_BATCH_DISPATCH(FN, 32, 8, 4, __VA_ARGS__);        \
        }                                                                        \
    } while (0)

// the reverse blend also has 8 pixels per thread (one warp per 16x16 or 32x8 tile)
#define SWGS_TILE_DISPATCH_BWD(FN, ...)                                          \
    do {                                                                         \
        if (ppt == 8 && tile_w == 16 && tile_h == 16)                            \
            SWGS_BATCH_DISPATCH(FN, 16, 16, 8, __VA_ARGS__);                     \
        if (ppt == 8 && tile_w == 32 && tile_h == 8)                             \
            SWGS_BATCH_DISPATCH(FN, 32, 8, 8, __VA_ARGS__);                      \
        SWGS_TILE_DISPATCH(FN, __VA_ARGS__);                                     \
    } while (0)

cudaError_t launch_blend_fwd(const BlendArgs& a, int tile_w, int tile_h, int batch, int ppt,
                             int grid, cudaStream_t s) {
    if (a.total_tiles <= 0) return cudaSuccess;
    SWGS_TILE_DISPATCH(run_fwd, a, grid, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_blend_bwd(const BlendArgs& a, int tile_w, int tile_h, int batch, int ppt,
                             int grid, cudaStream_t s) {
    if (a.total_tiles <= 0) return cudaSuccess;
    SWGS_TILE_DISPATCH_BWD(run_bwd, a, grid, s);
    return cudaErrorInvalidValue;
}

int blend_blocks_per_sm(int tile_w, int tile_h, int batch, int ppt, bool backward) {
    if (backward) SWGS_TILE_DISPATCH_BWD(occ_bwd);
    else SWGS_TILE_DISPATCH(occ_fwd);
    return 1;
}

bool blend_config_valid(int tile_w, int tile_h, int batch, int ppt, bool backward) {
    if (!(batch == 32 || batch == 64 || batch == 128 || batch == 256)) return false;
    if (tile_w == 16 && tile_h == 16)
        return ppt == 1 || ppt == 2 || ppt == 4 || (backward && ppt == 8);
    if (tile_w == 8 && tile_h == 8) return ppt == 1 || ppt == 2;
    if (tile_w == 32 && tile_h == 8)
        return ppt == 1 || ppt == 2 || ppt == 4 || (backward && ppt == 8);
    return false;
}

}  // namespace swgs
