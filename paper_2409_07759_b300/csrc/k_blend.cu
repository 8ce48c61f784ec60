// k_blend.cu -- per-tile front-to-back alpha compositing (Sec. 2.1 Eq. 3) and
// its reverse-order backward (Alg. 1 loss.backward).
//
// Persistent launch: a grid of (SMs x resident blocks) pulls (view, tile) work
// items from one atomic counter, over every view of the batch at once. Each
// thread owns PPT vertically adjacent pixels of the tile; the Gaussians of the
// tile's depth-sorted list are staged in shared memory BATCH at a time
// (converted once per block to the log2-domain form the inner loop needs).
// The inner loops are branch-free per pair: every lane of a warp walks the
// list in lockstep with predicated updates, so no lane diverges at the
// per-pair tests, and the warp leaves as soon as a vote says all its pixels
// saturated; the block stops staging when all its pixels have. The only
// branch inside is warp-uniform: it skips the 0.99 alpha clamp's work for
// Gaussians whose opacity cannot reach it.
//
// With an even number of pixels per thread (the defaults: 4 forward, 8
// reverse) the pixels are taken two at a time as float2 and every per-pixel
// step is one packed FP32x2 instruction; one pixel per thread keeps the scalar
// kernels (blend_fwd_kernel, blend_bwd_kernel).
//
// The backward walks the list from the block's largest last-contributor index
// down to the front, recovering each T from the saved final transmittance by
// division. Per Gaussian it accumulates nine moments -- sum of gm, gm dx,
// gm dy, gm dx^2, gm dx dy, gm dy^2 (gm = dL/dm) and of the colour weights --
// over the thread's pixels, sums them across the warp (a transposing butterfly,
// 14 shuffles for 9 values) and across the block in shared memory, and turns
// them into the nine 2D gradients (centre, conic, opacity, colour) once per
// Gaussian per tile before one vector atomic. At 8 pixels per thread a block
// is one warp: each lane leaves six column sums per Gaussian in shared memory
// and the warp reduces four Gaussians at a time, 8 lanes per Gaussian, with
// the x moments taken about the tile's centre column (round_reduce). Besides
// the clamp split, Gaussians in front of every pixel's last contributor (below
// the warp's smallest last) take a body without the per-pixel last test; in a
// one-warp block both choices are made once per round of four.
#include "swgs_internal.cuh"
#include <type_traits>

namespace swgs {

__device__ __forceinline__ void stage_gaussian(const Records& rec, uint32_t r, float4* s0,
                                               float4* s1, float4* s2) {
    const float4 A = rec.a[r];
    const float4 B = rec.b[r];
    const float4 Cc = rec.c[r];
    *s0 = make_float4(A.x, A.y, __fmul_rn(B.x, -0.5f * kLog2e), __fmul_rn(B.y, -kLog2e));
    const float lo = __log2f(A.z);
    *s1 = make_float4(__fmul_rn(B.z, -0.5f * kLog2e), lo, pair_vmin(lo), 0.f);
    *s2 = Cc;
}

template <int TW, int TH, int PPT>
struct TileGeom {
    static constexpr int NT = TW * TH / PPT;
    static_assert(NT % 32 == 0, "a tile block must be whole warps");
    static_assert(TH % PPT == 0, "pixels per thread must divide the tile height");
};

constexpr int kFwdUnroll = 8;
// row coordinate of a finished pixel in the packed forward: (kGone - y)^2
// overflows, so v = -inf for every Gaussian (no NaN: |t1 dx| stays finite)
constexpr float kGone = 3.0e30f;
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
                    const float v = pair_v(px, py[p], g0, g1.x, g1.y, &dx, &dy);
                    const float al = pair_alpha(v, &au);
                    const bool ok = !done[p] && v >= g1.z;
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
                if (V.out_rgb) {
                    V.out_rgb[q] = r0;
                    V.out_rgb[hw + q] = r1;
                    V.out_rgb[2 * hw + q] = r2;
                }
                if (V.out_rgb8) {
                    uint8_t* o8 = V.out_rgb8 + 3 * q;
                    o8[0] = rgb8_of(r0);
                    o8[1] = rgb8_of(r1);
                    o8[2] = rgb8_of(r2);
                }
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

// Forward with the pixels of a thread taken two at a time as float2: every
// per-pixel step is one packed FP32x2 instruction (__fadd2_rn, __fmul2_rn,
// __ffma2_rn round each half exactly like the scalar _rn forms), so the
// result is bit-identical to blend_fwd_kernel with half the issue slots on
// the FMA pipe. The staged terms are duplicated into pairs; the centre and the
// colour are staged negated so that w is carried as -w:
// -w = (-alpha) T, C + c w = C + (-c)(-w) and T - w = T + (-w), all exact
// rewrites of the same roundings.
// INT_FLAG: the clamp flag in the last word is the integer 1 (tested as a
// bit; the reverse blend runs faster so) rather than the float 1 (tested by
// a float compare; the forward runs faster so).
template <bool INT_FLAG>
__device__ __forceinline__ bool stage_gaussian_x2(const Records& rec, uint32_t r, float4* sa,
                                                  float4* sb, float4* sc, float4* sd,
                                                  float4* se) {
    const float4 A = rec.a[r];
    const float4 B = rec.b[r];
    const float4 Cc = rec.c[r];
    const float qa = __fmul_rn(B.x, -0.5f * kLog2e), qb = __fmul_rn(B.y, -kLog2e);
    const float qc = __fmul_rn(B.z, -0.5f * kLog2e);
    const float lo = __log2f(A.z);
    *sa = make_float4(-A.x, -A.x, -A.y, -A.y);
    *sb = make_float4(qa, qa, qb, qb);
    *sc = make_float4(qc, qc, lo, lo);
    *sd = make_float4(-Cc.x, -Cc.x, -Cc.y, -Cc.y);
    // alpha = min(0.99, o G) with G <= 1 reaches the clamp only when o > 0.99:
    // the blends skip the clamp's work for the others (a warp-uniform branch)
    const bool clamp = A.z > kAlphaMax;
    *se = make_float4(-Cc.z, -Cc.z, pair_vmin(lo),
                      INT_FLAG ? __uint_as_float(clamp ? 1u : 0u) : (clamp ? 1.f : 0.f));
    return clamp;
}

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// Forward staging: the terms of stage_gaussian_x2, with the Gaussian's 1-based
// position in its tile's list in the last word (the value `last` takes when
// the Gaussian is included). Returns whether its opacity exceeds 0.99, the
// only case in which alpha can take the 0.99 clamp.
__device__ __forceinline__ bool stage_gaussian_fwd(const Records& rec, uint32_t r, int pos1,
                                                   float4* sa, float4* sb, float4* sc, float4* sd,
                                                   float4* se, float* opacity) {
    const float4 A = rec.a[r];
    const float4 B = rec.b[r];
    const float4 Cc = rec.c[r];
    const float qa = __fmul_rn(B.x, -0.5f * kLog2e), qb = __fmul_rn(B.y, -kLog2e);
    const float qc = __fmul_rn(B.z, -0.5f * kLog2e);
    const float lo = __log2f(A.z);
    *sa = make_float4(-A.x, -A.x, -A.y, -A.y);
    *sb = make_float4(qa, qa, qb, qb);
    *sc = make_float4(qc, qc, lo, lo);
    *sd = make_float4(-Cc.x, -Cc.x, -Cc.y, -Cc.y);
    *se = make_float4(-Cc.z, -Cc.z, pair_vmin(lo), __int_as_float(pos1));
    *opacity = A.z;
    return A.z > kAlphaMax;
}

// One staged Gaussian against the thread's pixel pairs (the forward's inner
// step). CLAMP: alpha takes min(0.99, .) -- exact for every Gaussian, needed
// only for those whose opacity exceeds 0.99, so chunks without one skip it;
// the reverse blend splits on the same per-Gaussian flag, and both passes take
// the same alpha. COUNT: also records each pixel's stopping position (the
// pair-counting form, not timed).
template <bool CLAMP, int NP, bool COUNT, bool NOSTOP = false>
__device__ __forceinline__ void fwd_pairs(float4 ga, float4 gb, float4 gc, float4 gd, float4 ge,
                                          float2 bdx, float2 k, int pos,
                                          float2 (&T)[NP], float2 (&C0)[NP], float2 (&C1)[NP],
                                          float2 (&C2)[NP], float2 (&py)[NP], int (&last)[2 * NP],
                                          int (&stop)[2 * NP]) {
    const int pos1 = __float_as_int(ge.w);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const float2 dy = __fadd2_rn(py[i], hi2(ga));
        const float2 v = __ffma2_rn(__ffma2_rn(lo2(gc), dy, bdx), dy, k);
        // -alpha = -min(0.99, 2^v)
        float2 nal = make_float2(-ex2_approx(v.x), -ex2_approx(v.y));
        if (CLAMP) {
            nal.x = fmaxf(-kAlphaMax, nal.x);
            nal.y = fmaxf(-kAlphaMax, nal.y);
        }
        if (NOSTOP) {
            // no pixel can stop in this chunk (the caller's bound): every
            // pair that passes the threshold is included
            const bool ok0 = v.x >= ge.z, ok1 = v.y >= ge.z;
            nal.x = ok0 ? nal.x : 0.f;
            nal.y = ok1 ? nal.y : 0.f;
            last[2 * i] = ok0 ? pos1 : last[2 * i];
            last[2 * i + 1] = ok1 ? pos1 : last[2 * i + 1];
            const float2 nw = __fmul2_rn(nal, T[i]);      // -w
            C0[i] = __ffma2_rn(lo2(gd), nw, C0[i]);
            C1[i] = __ffma2_rn(hi2(gd), nw, C1[i]);
            C2[i] = __ffma2_rn(lo2(ge), nw, C2[i]);
            T[i] = __fadd2_rn(T[i], nw);
            continue;
        }
        // T (1 - alpha), rounded once: the stopping test
        const float2 tT = __ffma2_rn(nal, T[i], T[i]);
        const bool ok0 = v.x >= ge.z, ok1 = v.y >= ge.z;
        const bool inc0 = ok0 && tT.x >= kTStop, inc1 = ok1 && tT.y >= kTStop;
        if (COUNT) {
            stop[2 * i] = (ok0 && !inc0) ? pos : stop[2 * i];
            stop[2 * i + 1] = (ok1 && !inc1) ? pos : stop[2 * i + 1];
        }
        py[i].x = (ok0 && !inc0) ? kGone : py[i].x;
        py[i].y = (ok1 && !inc1) ? kGone : py[i].y;
        nal.x = inc0 ? nal.x : 0.f;
        nal.y = inc1 ? nal.y : 0.f;
        last[2 * i] = inc0 ? pos1 : last[2 * i];
        last[2 * i + 1] = inc1 ? pos1 : last[2 * i + 1];
        const float2 nw = __fmul2_rn(nal, T[i]);      // -w
        C0[i] = __ffma2_rn(lo2(gd), nw, C0[i]);
        C1[i] = __ffma2_rn(hi2(gd), nw, C1[i]);
        C2[i] = __ffma2_rn(lo2(ge), nw, C2[i]);
        T[i] = __fadd2_rn(T[i], nw);
    }
}

// One staged Gaussian j: its terms from shared memory, then fwd_pairs.
template <bool CLAMP, int NP, bool COUNT, bool NOSTOP = false>
__device__ __forceinline__ void fwd_step(const float4* sa, const float4* sb, const float4* sc,
                                         const float4* sd, const float4* se, int j, int pos,
                                         float2 px2, float2 (&T)[NP], float2 (&C0)[NP],
                                         float2 (&C1)[NP], float2 (&C2)[NP], float2 (&py)[NP],
                                         int (&last)[2 * NP], int (&stop)[2 * NP]) {
    const float4 ga = sa[j], gb = sb[j], gc = sc[j], gd = sd[j], ge = se[j];
    const float2 dx = __fadd2_rn(px2, lo2(ga));
    const float2 bdx = __fmul2_rn(hi2(gb), dx);
    const float2 k = __ffma2_rn(__fmul2_rn(lo2(gb), dx), dx, hi2(gc));
    fwd_pairs<CLAMP, NP, COUNT, NOSTOP>(ga, gb, gc, gd, ge, bdx, k, pos, T, C0, C1, C2, py, last,
                                        stop);
}

// Whether every pixel of the thread has stopped (or lies outside the image).
template <int NP>
__device__ __forceinline__ bool all_gone(const float2 (&py)[NP]) {
    bool d = true;
#pragma unroll
    for (int i = 0; i < NP; ++i) d &= (py[i].x == kGone) & (py[i].y == kGone);
    return d;
}

// 4 pixels a thread: at least 16 blocks of 64 threads per SM (64 registers;
// 14 blocks at 72 registers and 12 at 80 measured slower).
// The staged Gaussians are taken kFwdUnroll at a time (one warp vote for
// all). A full chunk holding no Gaussian of opacity > 0.99 (one bit per staged
// Gaussian, set at staging) runs the body without the clamp, unrolled with no
// per-Gaussian test; any other chunk -- one with such a Gaussian, or the
// batch's partial last chunk -- runs the clamp body, exact for every
// Gaussian, with a bound test per Gaussian.
template <int TW, int TH, int BATCH, int PPT, bool COUNT>
__global__ void __launch_bounds__(TW * TH / PPT, (PPT == 4 ? 16 : 1)) blend_fwd_x2_kernel(BlendArgs a) {
    static_assert(PPT % 2 == 0, "pixels are taken in pairs");
    static_assert(BATCH % kFwdUnroll == 0 && 32 % kFwdUnroll == 0, "chunks within a mask word");
    constexpr int NT = TileGeom<TW, TH, PPT>::NT;
    constexpr int NP = PPT / 2;
    __shared__ float4 sa[BATCH], sb[BATCH], sc[BATCH], sd[BATCH], se[BATCH];
    __shared__ unsigned s_cm[BATCH / 32];  // clamp bits of the staged Gaussians
    // per chunk of kFwdUnroll staged Gaussians: a lower bound on the product
    // of their (1 - alpha) (each alpha is at most the Gaussian's opacity)
    __shared__ float s_cp[BATCH / kFwdUnroll];
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
        const float2 px2 = make_float2(px, px);
        const int2 rg = a.ranges[item];
        float2 T[NP], C0[NP], C1[NP], C2[NP], py[NP];
        int last[PPT], stop[PPT];
        // a pixel that has stopped (or lies outside the image) moves its row
        // coordinate to kGone: v is then -inf, so no later pair passes the
        // v >= vmin test and no per-pixel flag is carried through the loop
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            T[i] = make_float2(1.f, 1.f);
            C0[i] = C1[i] = C2[i] = make_float2(0.f, 0.f);
            const int ya = y0 + 2 * i, yb = ya + 1;
            py[i] = make_float2(x < W && ya < H ? (float)ya + 0.5f : kGone,
                                x < W && yb < H ? (float)yb + 0.5f : kGone);
        }
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            last[p] = 0;
            stop[p] = rg.y;
        }
        for (int b0 = rg.x; b0 < rg.y; b0 += BATCH) {
            bool tdone = all_gone<NP>(py);
            if (__syncthreads_count(tdone) == NT) break;
            for (int k = tid; k < BATCH; k += NT) {
                const int idx = b0 + k;
                bool cl = false;
                float op = 0.f;
                if (idx < rg.y)
                    cl = stage_gaussian_fwd(a.rec, a.vals[idx], idx - rg.x + 1, &sa[k], &sb[k],
                                            &sc[k], &sd[k], &se[k], &op);
                const unsigned m = __ballot_sync(F, cl);
                if ((tid & 31) == 0) s_cm[k >> 5] = m;
                // 1% below (1 - opacity) a Gaussian: covers the FP32 rounding
                // of alpha and of T over a chunk
                float f = (1.f - fminf(op, kAlphaMax)) * 0.99f;
#pragma unroll
                for (int o = 1; o < kFwdUnroll; o <<= 1) f *= __shfl_xor_sync(F, f, o);
                if ((k & (kFwdUnroll - 1)) == 0) s_cp[k / kFwdUnroll] = f;
            }
            __syncthreads();
            const int cnt = min(BATCH, rg.y - b0);
            int j2 = 0;
            for (; j2 < cnt; j2 += kFwdUnroll) {
                if (__all_sync(F, tdone)) break;
                const unsigned cm = (s_cm[j2 >> 5] >> (j2 & 31)) & ((1u << kFwdUnroll) - 1u);
                // the warp's smallest transmittance over its pixels still going
                float tmin = INFINITY;
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    tmin = fminf(tmin, py[i].x == kGone ? INFINITY : T[i].x);
                    tmin = fminf(tmin, py[i].y == kGone ? INFINITY : T[i].y);
                }
                tmin = __uint_as_float(__reduce_min_sync(F, __float_as_uint(tmin)));
                if (cm == 0u && j2 + kFwdUnroll <= cnt && tmin * s_cp[j2 / kFwdUnroll] >= kTStop) {
                    // T (1 - alpha) stays at or above the stop threshold for every
                    // pixel and Gaussian of the chunk: no stop test is needed
#pragma unroll
                    for (int jj = 0; jj < kFwdUnroll; ++jj)
                        fwd_step<false, NP, COUNT, true>(sa, sb, sc, sd, se, j2 + jj,
                                                         b0 + j2 + jj, px2, T, C0, C1, C2, py,
                                                         last, stop);
                } else if (cm == 0u && j2 + kFwdUnroll <= cnt) {
#pragma unroll
                    for (int jj = 0; jj < kFwdUnroll; ++jj)
                        fwd_step<false, NP, COUNT>(sa, sb, sc, sd, se, j2 + jj, b0 + j2 + jj,
                                                   px2, T, C0, C1, C2, py, last, stop);
                } else {
#pragma unroll
                    for (int jj = 0; jj < kFwdUnroll; ++jj) {
                        if (j2 + jj >= cnt) break;
                        fwd_step<true, NP, COUNT>(sa, sb, sc, sd, se, j2 + jj, b0 + j2 + jj,
                                                  px2, T, C0, C1, C2, py, last, stop);
                    }
                }
                tdone = all_gone<NP>(py);
            }
        }
        // the view's fields, read before the stores below (which may alias them)
        const float bg0 = V.bg[0], bg1 = V.bg[1], bg2 = V.bg[2];
        float* const out_rgb = V.out_rgb;
        uint8_t* const out_rgb8 = V.out_rgb8;
        float* const out_T = V.out_T;
        const long long pix_base = V.pix_base;
        const float* const tgt = V.target;
        const uint8_t* const tgt8 = V.target_u8;
        float* const dL_out = V.dL_out;
        const float l1s = V.l1_scale;
        const long long hw = (long long)W * H;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int y = y0 + p;
            const float Tp = (p & 1) ? T[p / 2].y : T[p / 2].x;
            const float c0 = (p & 1) ? C0[p / 2].y : C0[p / 2].x;
            const float c1 = (p & 1) ? C1[p / 2].y : C1[p / 2].x;
            const float c2 = (p & 1) ? C2[p / 2].y : C2[p / 2].x;
            if (x < W && y < H) {
                const long long q = (long long)y * W + x;
                const float r0 = c0 + Tp * bg0;
                const float r1 = c1 + Tp * bg1;
                const float r2 = c2 + Tp * bg2;
                if (out_rgb) {
                    out_rgb[q] = r0;
                    out_rgb[hw + q] = r1;
                    out_rgb[2 * hw + q] = r2;
                }
                if (out_rgb8) {
                    uint8_t* o8 = out_rgb8 + 3 * q;
                    o8[0] = rgb8_of(r0);
                    o8[1] = rgb8_of(r1);
                    o8[2] = rgb8_of(r2);
                }
                if (out_T) out_T[q] = Tp;
                if (a.T) a.T[pix_base + q] = Tp;
                if (a.last) a.last[pix_base + q] = last[p];
                if (COUNT)
                    pairs += (unsigned long long)((stop[p] < rg.y ? stop[p] + 1 : rg.y) - rg.x);
                if (tgt || tgt8) {
                    // L1 term of the loss and its gradient, sign(0) = 0
                    float t0, t1, t2;
                    if (tgt8) {  // k x (1/255) in FP32
                        constexpr float kInv255 = 1.0f / 255.0f;
                        t0 = __fmul_rn((float)tgt8[q], kInv255);
                        t1 = __fmul_rn((float)tgt8[hw + q], kInv255);
                        t2 = __fmul_rn((float)tgt8[2 * hw + q], kInv255);
                    } else {
                        t0 = tgt[q];
                        t1 = tgt[hw + q];
                        t2 = tgt[2 * hw + q];
                    }
                    const float e0 = r0 - t0, e1 = r1 - t1, e2 = r2 - t2;
                    dL_out[q] = e0 > 0.f ? l1s : (e0 < 0.f ? -l1s : 0.f);
                    dL_out[hw + q] = e1 > 0.f ? l1s : (e1 < 0.f ? -l1s : 0.f);
                    dL_out[2 * hw + q] = e2 > 0.f ? l1s : (e2 < 0.f ? -l1s : 0.f);
                    l1 += (fabsf(e0) + fabsf(e1) + fabsf(e2)) * l1s;
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

// Steps 1-3 of a transposing butterfly on v[0..8): each step halves the
// values a lane holds while doubling the lanes summed, so lane l ends with
// value l >> 2 summed over the 8 lanes that differ from it in bits 2-4.
__device__ __forceinline__ float warp_sum8_part(const float* v) {
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
    return (bC ? x[1] : x[0]) + __shfl_xor_sync(F, bC ? x[0] : x[1], 4);
}

// Sum 9 per-lane values over the warp (value 8 by a plain butterfly) and add
// the sums to acc[0..9) in shared memory, which the block's other warps also
// add to.
__device__ __forceinline__ void warp_sum9_to_smem(const float* v, float* acc) {
    const unsigned F = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float y = warp_sum8_part(v);
    y += __shfl_xor_sync(F, y, 2);
    y += __shfl_xor_sync(F, y, 1);
    float v8 = v[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v8 += __shfl_xor_sync(F, v8, o);
    if ((lane & 3) == 0 && y != 0.f) atomicAdd(&acc[lane >> 2], y);
    if (lane == 0 && v8 != 0.f) atomicAdd(&acc[8], v8);
}

// Staged Gaussians whose per-lane sums one shared-memory round reduces in a
// block of one warp.
constexpr int kRoundG = 4;

// The reduction of kRoundG staged Gaussians in a block of one warp. Lane l
// has written, for slot g, its column sums ma[g][l] = (S0, SY, SYY, M6) and
// mb[g][l] = (M7, M8): S0 = sum gm, SY = sum gm dy, SYY = sum gm dy^2 over its
// pixels and M_c = sum (-w) dL_c. The slot's LPG = 32 / kRoundG lanes sum it:
// lane L takes slot L / LPG over source lanes L % LPG + LPG i (i < kRoundG).
// A source's column in the tile is its lane mod TW, so a lane's sources fall
// in min(kRoundG, TW / LPG) columns. Against the tile's centre column (x
// offset xl = column + 1/2 - TW/2) it forms
//   P0 = sum S0, P1 = sum S0 xl, P2 = sum S0 xl^2, Q0 = sum SY,
//   Q1 = sum SY xl, R = sum SYY and the three colour sums,
// then sums them over the slot's lanes (a transposing butterfly on the first
// eight: lane L ends with values n (L % LPG) + k, k < n = 8 / LPG; every lane
// with the ninth) and stores them to acc[9 j ..] for the slot's Gaussian
// j = j_top - g (slots with j < 0 were not staged and are dropped). With
// dx = xl + c, c = tile centre - u, the x moments follow at the flush:
// sum gm dx = P1 + c P0, sum gm dx^2 = P2 + 2c P1 + c^2 P0,
// sum gm dx dy = Q1 + c Q0.
template <int TW>
__device__ __forceinline__ void round_reduce(const float4 (*ma)[32], const float2 (*mb)[32],
                                             float* acc, int j_top) {
    constexpr int LPG = 32 / kRoundG;
    constexpr int NCOL = kRoundG < TW / LPG ? kRoundG : TW / LPG;
    static_assert(LPG >= 2 && LPG <= 8 && NCOL >= 1 && kRoundG % NCOL == 0,
                  "2 to 16 Gaussians a round, whole columns");
    const unsigned F = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int g = lane / LPG, part = lane % LPG;
    float4 ca[NCOL];
    float2 cb[NCOL];
#pragma unroll
    for (int i = 0; i < kRoundG; ++i) {
        const float4 sa = ma[g][part + LPG * i];
        const float2 sb = mb[g][part + LPG * i];
        const int c = i % NCOL;
        if (i < NCOL) {
            ca[c] = sa;
            cb[c] = sb;
        } else {
            const float2 lo = __fadd2_rn(lo2(ca[c]), lo2(sa));
            const float2 hi = __fadd2_rn(hi2(ca[c]), hi2(sa));
            ca[c] = make_float4(lo.x, lo.y, hi.x, hi.y);
            cb[c] = __fadd2_rn(cb[c], sb);
        }
    }
    float2 p0q0 = make_float2(0.f, 0.f), p1q1 = p0q0, rm6 = p0q0, m78 = p0q0;
    float p2 = 0.f;
#pragma unroll
    for (int c = 0; c < NCOL; ++c) {
        const float xl = (float)(part + LPG * c) + (0.5f - 0.5f * TW);
        const float2 sq = lo2(ca[c]);                       // (S0, SY)
        const float2 t = __fmul2_rn(sq, make_float2(xl, xl));
        p0q0 = __fadd2_rn(p0q0, sq);
        p1q1 = __fadd2_rn(p1q1, t);
        p2 = fmaf(t.x, xl, p2);
        rm6 = __fadd2_rn(rm6, hi2(ca[c]));                  // (SYY, M6)
        m78 = __fadd2_rn(m78, cb[c]);
    }
    float v[8] = {p0q0.x, p1q1.x, p2, p0q0.y, p1q1.y, rm6.x, rm6.y, m78.x};
    float v8 = m78.y;
    int n = 8;
#pragma unroll
    for (int o = LPG / 2; o >= 1; o >>= 1) {
        const bool b = lane & o;
        n >>= 1;
#pragma unroll
        for (int k = 0; k < n; ++k) {
            const float send = b ? v[k] : v[k + n];
            const float keep = b ? v[k + n] : v[k];
            v[k] = keep + __shfl_xor_sync(F, send, o);
        }
        v8 += __shfl_xor_sync(F, v8, o);
    }
    const int j = j_top - g;
    if (j >= 0) {
#pragma unroll
        for (int k = 0; k < 8 / LPG; ++k) acc[9 * j + (8 / LPG) * part + k] = v[k];
        if (part == 0) acc[9 * j + 8] = v8;
    }
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// A block of one warp synchronises its lanes alone (shared-memory ordering
// included); larger blocks take the block barrier.
template <int NT>
__device__ __forceinline__ void block_sync() {
    if constexpr (NT == 32) __syncwarp(); else __syncthreads();
}

// Reverse blend with the pixels of a thread taken two at a time as float2 (the
// packed FP32x2 instructions of the forward). It uses the forward's packed
// staging (centre and colour negated) and carries -alpha, so every sign
// folds into an exact rewrite: 1 - a = 1 + (-a), w = -((-a) T),
// D + a (E - D) = D + (-a)(D + (-E)), and dL/dm's factor a (T (E - D)) =
// (-a)(T (D + (-E))). Each thread's per-pixel sums are kept as two partial
// sums (the halves) and added before the warp reduction.
// One staged Gaussian against the thread's pixel pairs (the reverse blend's
// inner step): T recovery, the colour-behind update and the per-pixel sums.
// CLAMP: alpha takes min(0.99, .) (where dalpha/dm is then zero) -- needed
// only when the Gaussian's opacity exceeds 0.99, and bit-identical to the
// body without it for every other Gaussian. ALL: the Gaussian lies in front of
// every pixel's last contributor (pos below the warp's smallest last), so no
// pixel needs the pos < last test.
template <bool CLAMP, bool ALL, int NP>
__device__ __forceinline__ void bwd_pairs(float4 ga, float4 gb, float4 gc, float4 gd, float4 ge,
                                          float2 bdx, float2 k, int pos, const float2 (&py)[NP],
                                          const int (&last)[2 * NP], float2 (&T)[NP],
                                          float2 (&D)[NP], const float2 (&dL0)[NP],
                                          const float2 (&dL1)[NP], const float2 (&dL2)[NP],
                                          float2& S0, float2& SY, float2& SYY, float2& M6,
                                          float2& M7, float2& M8) {
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const float2 dy = __fadd2_rn(py[i], hi2(ga));
        const float2 v = __ffma2_rn(__ffma2_rn(lo2(gc), dy, bdx), dy, k);
        const float u0 = ex2_approx(v.x), u1 = ex2_approx(v.y);
        const bool ok0 = (ALL || pos < last[2 * i]) && v.x >= ge.z;
        const bool ok1 = (ALL || pos < last[2 * i + 1]) && v.y >= ge.z;
        // -alpha of a counted pair, 0 otherwise; -alpha where dalpha/dm is
        // nonzero (the unclamped alpha), 0 otherwise
        float2 na;
        if (CLAMP) {
            na.x = ok0 ? fmaxf(-kAlphaMax, -u0) : 0.f;
            na.y = ok1 ? fmaxf(-kAlphaMax, -u1) : 0.f;
        } else {
            na.x = ok0 ? -u0 : 0.f;
            na.y = ok1 ? -u1 : 0.f;
        }
        // T before this Gaussian, recovered from the T after it (a pair that
        // does not count has alpha = 0 and leaves T as is)
        // (scalar: the reciprocals need not be made a register pair)
        T[i].x = __fmul_rn(T[i].x, rcp_approx(__fadd_rn(1.f, na.x)));
        T[i].y = __fmul_rn(T[i].y, rcp_approx(__fadd_rn(1.f, na.y)));
        const float2 nw = __fmul2_rn(na, T[i]);            // -w
        M6 = __ffma2_rn(nw, dL0[i], M6);
        M7 = __ffma2_rn(nw, dL1[i], M7);
        M8 = __ffma2_rn(nw, dL2[i], M8);
        // -E = sum_ch dL_ch (-c_ch); nd = D - E
        const float2 ne = __ffma2_rn(dL0[i], lo2(gd),
                                     __ffma2_rn(dL1[i], hi2(gd), __fmul2_rn(dL2[i], lo2(ge))));
        const float2 nd = __fadd2_rn(D[i], ne);
        D[i] = __ffma2_rn(na, nd, D[i]);
        // gm = alpha T (E - D) = (-w)(D - E); zero where alpha takes the clamp
        // (dalpha/dm = 0 there). Unclamped, both bodies round it alike.
        float2 gm = __fmul2_rn(nw, nd);
        if (CLAMP) {
            gm.x = u0 <= kAlphaMax ? gm.x : 0.f;
            gm.y = u1 <= kAlphaMax ? gm.y : 0.f;
        }
        const float2 gy = __fmul2_rn(gm, dy);
        S0 = __fadd2_rn(S0, gm);
        SY = __fadd2_rn(SY, gy);
        SYY = __ffma2_rn(gy, dy, SYY);
    }
}

// 8 pixels a thread (one warp a tile): at least 16 warps per SM (128
// registers) hide the ex2 -> rcp latency better than 15 at the unbounded 136,
// and better than 18-20 with their spills
template <int TW, int TH, int BATCH, int PPT>
__global__ void __launch_bounds__(TW * TH / PPT, (PPT == 8 ? 16 : 1)) blend_bwd_x2_kernel(BlendArgs a) {
    static_assert(PPT % 2 == 0, "pixels are taken in pairs");
    constexpr int NT = TileGeom<TW, TH, PPT>::NT;
    constexpr int NP = PPT / 2;
    __shared__ float4 sa[BATCH], sb[BATCH], sc[BATCH], sd[BATCH], se[BATCH];
    __shared__ uint32_t s_rec[BATCH];
    __shared__ float s_acc[BATCH * 9];
    __shared__ int s_item, s_maxlast;
    // a block of one warp reduces its per-lane sums through shared memory,
    // kRoundG Gaussians a round (round_reduce); larger blocks by shuffles
    constexpr bool kRound = NT == 32;
    static_assert(BATCH % kRoundG == 0, "rounds within a batch");
    __shared__ float4 s_ma[kRound ? kRoundG : 1][32];
    __shared__ float2 s_mb[kRound ? kRoundG : 1][32];
    // clamp bits of the staged Gaussians, read 64 at a time
    __shared__ __align__(8) unsigned s_bcm[kRound ? (BATCH + 63) / 64 * 2 : 1];
    const unsigned F = 0xffffffffu;
    const int tid = threadIdx.x;
    const int lx = tid % TW, ly = (tid / TW) * PPT;
    for (int k = tid; k < BATCH * 9; k += NT) s_acc[k] = 0.f;
    for (;;) {
        if (tid == 0) { s_item = atomicAdd(a.work_counter, 1); s_maxlast = 0; }
        block_sync<NT>();
        const int item = s_item;
        if (item >= a.total_tiles) break;
        const int vi = find_view_by_tile(a.views, a.n_views, item);
        const ViewDev& V = a.views[vi];
        const int W = V.W, H = V.H;
        const int lt = item - V.tile_base;
        const int x = (lt % V.ntx) * TW + lx, y0 = (lt / V.ntx) * TH + ly;
        const float px = (float)x + 0.5f;
        const float2 px2 = make_float2(px, px);
        const int2 rg = a.ranges[item];
        // Per pixel: T (recovered back to front), dL/dC, and D = sum_ch dL_ch B_ch with
        // B the colour composited behind the current Gaussian (starts at the
        // background). With E = sum_ch dL_ch c_ch: dL/dalpha = T (E - D) and the
        // step to the next Gaussian in front is D' = D + alpha (E - D).
        float Tv[PPT], dLa[PPT], dLb[PPT], dLc[PPT], Dv[PPT];
        int last[PPT];
        int mylast = 0;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int y = y0 + p;
            Tv[p] = 1.f; dLa[p] = dLb[p] = dLc[p] = 0.f; last[p] = 0;
            if (x < W && y < H) {
                const long long hw = (long long)W * H, q = (long long)y * W + x;
                Tv[p] = a.T[V.pix_base + q];
                last[p] = a.last[V.pix_base + q];
                dLa[p] = V.dL[q];
                dLb[p] = V.dL[hw + q];
                dLc[p] = V.dL[2 * hw + q];
            }
            Dv[p] = fmaf(dLa[p], V.bg[0], fmaf(dLb[p], V.bg[1], dLc[p] * V.bg[2]));
            mylast = max(mylast, last[p]);
        }
        float2 T[NP], dL0[NP], dL1[NP], dL2[NP], D[NP], py[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            T[i] = make_float2(Tv[2 * i], Tv[2 * i + 1]);
            dL0[i] = make_float2(dLa[2 * i], dLa[2 * i + 1]);
            dL1[i] = make_float2(dLb[2 * i], dLb[2 * i + 1]);
            dL2[i] = make_float2(dLc[2 * i], dLc[2 * i + 1]);
            D[i] = make_float2(Dv[2 * i], Dv[2 * i + 1]);
            py[i] = make_float2((float)(y0 + 2 * i) + 0.5f, (float)(y0 + 2 * i + 1) + 0.5f);
        }
        if (NT > 32 && mylast > 0) atomicMax(&s_maxlast, mylast);
        // below the warp's smallest last every pixel of the warp takes part
        int myfirst = last[0];
#pragma unroll
        for (int p = 1; p < PPT; ++p) myfirst = min(myfirst, last[p]);
        const int wfirst = __reduce_min_sync(F, myfirst);
        block_sync<NT>();
        const int end = rg.x + (NT == 32 ? __reduce_max_sync(F, mylast) : s_maxlast);
        for (int b1 = end; b1 > rg.x; b1 -= BATCH) {
            const int b0 = max(rg.x, b1 - BATCH);
            const int cnt = b1 - b0;
            block_sync<NT>();
            if constexpr (kRound) {
                for (int k0 = 0; k0 < cnt; k0 += 32) {
                    const int k = k0 + tid;
                    bool cl = false;
                    if (k < cnt) {
                        const uint32_t r = a.vals[b0 + k];
                        s_rec[k] = r;
                        cl = stage_gaussian_x2<true>(a.rec, r, &sa[k], &sb[k], &sc[k], &sd[k],
                                                     &se[k]);
                    }
                    const unsigned m = __ballot_sync(F, cl);
                    if (tid == 0) s_bcm[k0 >> 5] = m;
                }
            } else {
                for (int k = tid; k < cnt; k += NT) {
                    const uint32_t r = a.vals[b0 + k];
                    s_rec[k] = r;
                    stage_gaussian_x2<true>(a.rec, r, &sa[k], &sb[k], &sc[k], &sd[k], &se[k]);
                }
            }
            block_sync<NT>();
            if constexpr (kRound) {
            // kRoundG staged Gaussians per round, back to front: each lane
            // leaves its column sums in s_ma/s_mb (the thread's pixels share
            // x, so only sum gm, sum gm dy and sum gm dy^2 run per pixel; gm
            // is alpha dL/dalpha, its factor -1/2 applied at the flush), then
            // the warp reduces the round. The body is chosen once a round: the
            // clamp body if a Gaussian of the round has opacity > 0.99 (exact,
            // and bit-identical for the others), else the one without the
            // pos < last test if the round lies below the warp's smallest last.
            const unsigned long long* cm64 = reinterpret_cast<const unsigned long long*>(s_bcm);
            auto round = [&](int j4, auto clamp_tag, auto all_tag) {
                constexpr bool kClamp = decltype(clamp_tag)::value;
                constexpr bool kAll = decltype(all_tag)::value;
#pragma unroll
                for (int jj = 0; jj < kRoundG; ++jj) {
                    const int j = j4 - jj;
                    if (j < 0) break;
                    const int pos = b0 + j - rg.x;
                    const float4 ga = sa[j], gb = sb[j], gc = sc[j], gd = sd[j], ge = se[j];
                    const float2 dx = __fadd2_rn(px2, lo2(ga));
                    const float2 bdx = __fmul2_rn(hi2(gb), dx);
                    const float2 k = __ffma2_rn(__fmul2_rn(lo2(gb), dx), dx, hi2(gc));
                    float2 S0 = make_float2(0.f, 0.f), SY = S0, SYY = S0, M6 = S0, M7 = S0,
                           M8 = S0;
                    bwd_pairs<kClamp, kAll, NP>(ga, gb, gc, gd, ge, bdx, k, pos, py, last, T, D,
                                                dL0, dL1, dL2, S0, SY, SYY, M6, M7, M8);
                    s_ma[jj][tid] =
                        make_float4(S0.x + S0.y, SY.x + SY.y, SYY.x + SYY.y, M6.x + M6.y);
                    s_mb[jj][tid] = make_float2(M7.x + M7.y, M8.x + M8.y);
                }
            };
            for (int j4 = cnt - 1; j4 >= 0; j4 -= kRoundG) {
                const int jlo = max(j4 - (kRoundG - 1), 0);
                unsigned long long cm = cm64[jlo >> 6] >> (jlo & 63);
                if ((j4 >> 6) != (jlo >> 6)) cm |= cm64[j4 >> 6] << (64 - (jlo & 63));
                using T1 = std::integral_constant<bool, true>;
                using T0 = std::integral_constant<bool, false>;
                if (cm & ((2ull << (j4 - jlo)) - 1ull))
                    round(j4, T1{}, T0{});
                else if (b0 + j4 - rg.x < wfirst)
                    round(j4, T0{}, T1{});
                else
                    round(j4, T0{}, T0{});
                __syncwarp();
                round_reduce<TW>(s_ma, s_mb, s_acc, j4);
                __syncwarp();
            }
            } else {
            // kBwdUnroll staged Gaussians per iteration, back to front; the
            // group is skipped when it lies beyond every pixel of the warp's last
            for (int j2 = cnt - 1; j2 >= 0; j2 -= kBwdUnroll) {
                if (__all_sync(F, b0 + max(j2 - kBwdUnroll + 1, 0) - rg.x >= mylast)) continue;
#pragma unroll
                for (int jj = 0; jj < kBwdUnroll; ++jj) {
                const int j = j2 - jj;
                if (j < 0) break;
                const int pos = b0 + j - rg.x;
                const float4 ga = sa[j], gb = sb[j], gc = sc[j], gd = sd[j], ge = se[j];
                const float2 dx = __fadd2_rn(px2, lo2(ga));
                const float2 bdx = __fmul2_rn(hi2(gb), dx);
                const float2 k = __ffma2_rn(__fmul2_rn(lo2(gb), dx), dx, hi2(gc));
                // The thread's pixels share x, so dx is common to them: only
                // sum gm, sum gm dy and sum gm dy^2 run per pixel; the dx terms
                // are applied once below. gm here is alpha dL/dalpha (the
                // factor -1/2 of dalpha/dm is applied at the flush).
                float2 S0 = make_float2(0.f, 0.f), SY = S0, SYY = S0, M6 = S0, M7 = S0, M8 = S0;
                if (__float_as_uint(ge.w) & 1u)
                    bwd_pairs<true, false, NP>(ga, gb, gc, gd, ge, bdx, k, pos, py, last, T, D,
                                               dL0, dL1, dL2, S0, SY, SYY, M6, M7, M8);
                else if (pos < wfirst)
                    bwd_pairs<false, true, NP>(ga, gb, gc, gd, ge, bdx, k, pos, py, last, T, D,
                                               dL0, dL1, dL2, S0, SY, SYY, M6, M7, M8);
                else
                    bwd_pairs<false, false, NP>(ga, gb, gc, gd, ge, bdx, k, pos, py, last, T, D,
                                                dL0, dL1, dL2, S0, SY, SYY, M6, M7, M8);
                float m[9];
                m[0] = S0.x + S0.y;
                m[2] = SY.x + SY.y;
                m[5] = SYY.x + SYY.y;
                m[6] = -(M6.x + M6.y);
                m[7] = -(M7.x + M7.y);
                m[8] = -(M8.x + M8.y);
                // every staged Gaussian is reduced: nearly all in a tile's list
                // reach some pixel, so a vote to skip the rest costs more than it
                // saves (the flush skips the all-zero sums)
                m[1] = m[0] * dx.x;
                m[3] = m[1] * dx.x;
                m[4] = m[2] * dx.x;
                warp_sum9_to_smem(m, &s_acc[j * 9]);
                }
            }
            }
            block_sync<NT>();
            for (int k = tid; k < cnt; k += NT) {
                float* acc = &s_acc[k * 9];
                bool nz = false;
#pragma unroll
                for (int e = 0; e < 9; ++e) nz |= acc[e] != 0.f;
                if (!nz) continue;
                const uint32_t r = s_rec[k];
                const float4 ra = a.rec.a[r];   // u, v, opacity, depth
                const float4 rb = a.rec.b[r];   // A, B, C
                float* dst = a.grad2d + 12ll * r;
                if constexpr (kRound) {
                    // round_reduce's sums about the tile's centre column:
                    // (P0, P1, P2, Q0, Q1, R, M6, M7, M8), dx = xl + c
                    const float c = (float)(x - lx + TW / 2) - ra.x;
                    const float sx = fmaf(c, acc[0], acc[1]);
                    const float sxx = fmaf(c, fmaf(c, acc[0], 2.f * acc[1]), acc[2]);
                    const float sxy = fmaf(c, acc[3], acc[4]);
                    const float m1 = -0.5f * sx, m2 = -0.5f * acc[3];
                    const float du = -2.f * (rb.x * m1 + rb.y * m2);
                    const float dv = -2.f * (rb.y * m1 + rb.z * m2);
                    const float dop = acc[0] / ra.z;
                    red_add_v4(dst, du, dv, -0.5f * sxx, -sxy);
                    red_add_v4(dst + 4, -0.5f * acc[5], dop, -acc[6], -acc[7]);
                    red_add(dst + 8, -acc[8]);
                    continue;
                }
                // acc[0..5] hold sums of alpha dL/dalpha times (1, dx, dy, dx^2,
                // dx dy, dy^2); dL/dm = -1/2 of them (G = exp(-m/2)).
                // m = A dx^2 + 2B dx dy + C dy^2, dx = px - u: dm/du = -2(A dx + B dy)
                const float m1 = -0.5f * acc[1], m2 = -0.5f * acc[2];
                const float du = -2.f * (rb.x * m1 + rb.y * m2);
                const float dv = -2.f * (rb.y * m1 + rb.z * m2);
                // alpha = o G, dalpha/do = G = alpha/o
                const float dop = acc[0] / ra.z;
                red_add_v4(dst, du, dv, -0.5f * acc[3], -acc[4]);
                red_add_v4(dst + 4, -0.5f * acc[5], dop, acc[6], acc[7]);
                red_add(dst + 8, acc[8]);
#pragma unroll
                for (int e = 0; e < 9; ++e) acc[e] = 0.f;
            }
        }
        block_sync<NT>();
    }
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
                    const float v = pair_v(px, py[p], g0, g1.x, g1.y, &dx, &dy);
                    const float al = pair_alpha(v, &au);
                    const bool ok = pos < last[p] && v >= g1.z;
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
                    D[p] = fmaf(a1, diff, D[p]);
                    // dalpha/dm needs the unclamped alpha: a1 = au when it counts
                    const float gm = au <= kAlphaMax ? w * diff : 0.f;
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

// even pixel counts per thread take the packed kernel
template <int TW, int TH, int BATCH, int PPT, bool COUNT>
static void* fwd_kernel_ptr() {
    if constexpr (PPT % 2 == 0)
        return (void*)blend_fwd_x2_kernel<TW, TH, BATCH, PPT, COUNT>;
    else
        return (void*)blend_fwd_kernel<TW, TH, BATCH, PPT, COUNT>;
}

template <int TW, int TH, int BATCH, int PPT>
static cudaError_t run_fwd(const BlendArgs& a, int grid, cudaStream_t s) {
    note_launch();
    if constexpr (PPT % 2 == 0) {
        if (a.pairs)
            blend_fwd_x2_kernel<TW, TH, BATCH, PPT, true><<<grid, TW * TH / PPT, 0, s>>>(a);
        else
            blend_fwd_x2_kernel<TW, TH, BATCH, PPT, false><<<grid, TW * TH / PPT, 0, s>>>(a);
    } else {
        if (a.pairs)
            blend_fwd_kernel<TW, TH, BATCH, PPT, true><<<grid, TW * TH / PPT, 0, s>>>(a);
        else
            blend_fwd_kernel<TW, TH, BATCH, PPT, false><<<grid, TW * TH / PPT, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template <int TW, int TH, int BATCH, int PPT>
static void* bwd_kernel_ptr() {
    if constexpr (PPT % 2 == 0)
        return (void*)blend_bwd_x2_kernel<TW, TH, BATCH, PPT>;
    else
        return (void*)blend_bwd_kernel<TW, TH, BATCH, PPT>;
}

template <int TW, int TH, int BATCH, int PPT>
static cudaError_t run_bwd(const BlendArgs& a, int grid, cudaStream_t s) {
    note_launch();
    if constexpr (PPT % 2 == 0)
        blend_bwd_x2_kernel<TW, TH, BATCH, PPT><<<grid, TW * TH / PPT, 0, s>>>(a);
    else
        blend_bwd_kernel<TW, TH, BATCH, PPT><<<grid, TW * TH / PPT, 0, s>>>(a);
    return cudaGetLastError();
}

template <int TW, int TH, int BATCH, int PPT>
static int occ_fwd() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fwd_kernel_ptr<TW, TH, BATCH, PPT, false>(),
                                                  TW * TH / PPT, 0);
    return n < 1 ? 1 : n;
}

template <int TW, int TH, int BATCH, int PPT>
static int occ_bwd() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bwd_kernel_ptr<TW, TH, BATCH, PPT>(),
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
