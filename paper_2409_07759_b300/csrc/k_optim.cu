// k_optim.cu -- the steps of Alg. 1 after the backward pass, on the Gaussians
// eligible at this step (active at one of the step's frames, not frozen):
//   - an optional bias-corrected Adam step (the optimiser of [14]);
//   - the SGLD noise mu += lr * noise_lr * sigmoid(-k (o - t)) * Sigma eta
//     (Alg. 1 noise step, Sec. 4.4; the noise form of [14]);
//   - relocation of dead Gaussians onto alive ones sampled in proportion to
//     opacity, with the opacity and scale adjustment of [14] (Sec. 3.2,
//     Alg. 1 relocate).
// Random numbers come from Philox4x64-10 keyed by (seed, purpose) with counter
// (slot, step), so every draw is independent of launch shape and order.
#include "swgs_internal.cuh"

namespace swgs {

constexpr int kMaxStepFrames = 64;

struct SgldArgs {
    swgs_gaussians g;
    swgs_gaussians grads;
    swgs_adam_state adam;
    int has_grads, has_adam;
    const uint8_t* elig;  // eligible slots (launch_eligible)
    const uint32_t* gate;  // nonzero: the forward before this step failed, do nothing
    swgs_sgld_params p;
    float bc1, bc2;  // Adam bias corrections 1 - beta^(step+1)
    unsigned long long seed, step;
};

struct StepFrames {
    int frames[kMaxStepFrames];
    int n;
};

__device__ __forceinline__ bool is_eligible(const swgs_gaussians& g, long long i,
                                            const int* frames, int nf) {
    if (g.frozen && g.frozen[i]) return false;
    const int s = g.start[i], e = g.expire[i];
    for (int f = 0; f < nf; ++f)
        if (s <= frames[f] && frames[f] < e) return true;
    return false;
}

// One byte per slot, computed once per step and read by the Adam, noise and
// relocation-weight kernels (instead of each re-testing every frame).
__global__ void __launch_bounds__(256) eligible_kernel(swgs_gaussians g, StepFrames f,
                                                       uint8_t* __restrict__ elig) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.capacity) return;
    elig[i] = is_eligible(g, i, f.frames, f.n) ? 1 : 0;
}

cudaError_t launch_eligible(const swgs_gaussians& g, const int32_t* frames, int n_frames,
                            uint8_t* elig, cudaStream_t s) {
    if (n_frames > kMaxStepFrames) return cudaErrorInvalidValue;
    if (g.capacity <= 0) return cudaSuccess;
    StepFrames f{};
    for (int k = 0; k < n_frames; ++k) f.frames[k] = frames[k];
    f.n = n_frames;
    note_launch();
    eligible_kernel<<<div_up(g.capacity, 256), 256, 0, s>>>(g, f, elig);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gradient rows of the eligible slots, packed for a data-parallel sum: only
// those rows can hold a nonzero gradient, and every replica finds the same
// set (same state, same frames), so the ranks exchange count x R floats
// instead of the whole buffer. Row layout: means 3, log_scales 3, quats 4,
// opacity logit 1, sh 3K (R = 11 + 3K); rows in ascending slot order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int grad_row_floats(int K) { return 11 + 3 * K; }

__global__ void __launch_bounds__(256)
elig_count_kernel(const uint8_t* __restrict__ elig, long long n, uint32_t* __restrict__ counts) {
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    const int c = __syncthreads_count(i < n && elig[i]);
    if (threadIdx.x == 0) counts[blockIdx.x] = (uint32_t)c;
}

template <bool PACK>
__device__ __forceinline__ void grad_row_copy(const swgs_gaussians& gr, long long slot, int K,
                                              float* row, float scale) {
    const int nsh = 3 * K;
    float* dst[5] = {gr.means + 3 * slot, gr.log_scales + 3 * slot, gr.quats + 4 * slot,
                     gr.opacity_logits + slot, gr.sh + (long long)nsh * slot};
    const int len[5] = {3, 3, 4, 1, nsh};
    int o = 0;
#pragma unroll
    for (int a = 0; a < 5; ++a) {
        for (int e = 0; e < len[a]; ++e) {
            if (PACK) row[o + e] = dst[a][e] * scale;
            else dst[a][e] = row[o + e];
        }
        o += len[a];
    }
}

__global__ void __launch_bounds__(256)
grad_pack_kernel(swgs_gaussians gr, const uint8_t* __restrict__ elig, long long n,
                 const uint32_t* __restrict__ block_off, int K, float scale,
                 int32_t* __restrict__ ids, float* __restrict__ packed) {
    __shared__ uint32_t warp_off[8];
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    const bool m = i < n && elig[i];
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, m);
    if (lane == 0) warp_off[warp] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int w = 0; w < 8; ++w) {
            const uint32_t c = warp_off[w];
            warp_off[w] = run;
            run += c;
        }
    }
    __syncthreads();
    if (!m) return;
    const long long pos = (long long)block_off[blockIdx.x] + warp_off[warp] +
                          __popc(bal & ((1u << lane) - 1u));
    ids[pos] = (int32_t)i;
    grad_row_copy<true>(gr, i, K, packed + pos * grad_row_floats(K), scale);
}

__global__ void __launch_bounds__(256)
grad_unpack_kernel(swgs_gaussians gr, const int32_t* __restrict__ ids,
                   const long long* __restrict__ count, int K, const float* __restrict__ packed) {
    const long long k = (long long)blockIdx.x * 256 + threadIdx.x;
    if (k >= *count) return;
    grad_row_copy<false>(gr, ids[k], K, const_cast<float*>(packed) + k * grad_row_floats(K), 1.f);
}

cudaError_t launch_grad_pack(const swgs_gaussians& g, const swgs_gaussians& grads,
                             const int32_t* frames, int n_frames, float scale, uint8_t* elig,
                             uint32_t* block_cnt, void* scan_tmp, int32_t* ids, long long* count,
                             float* packed, cudaStream_t s) {
    const long long n = g.capacity;
    cudaError_t e = launch_eligible(g, frames, n_frames, elig, s);
    if (e != cudaSuccess) return e;
    const long long nb = div_up(n, 256);
    note_launch();
    elig_count_kernel<<<(unsigned)nb, 256, 0, s>>>(elig, n, block_cnt);
    e = exclusive_scan_u32(block_cnt, block_cnt, nb, scan_tmp, (unsigned long long*)count, s);
    if (e != cudaSuccess) return e;
    const int K = (g.sh_degree + 1) * (g.sh_degree + 1);
    note_launch();
    grad_pack_kernel<<<(unsigned)nb, 256, 0, s>>>(grads, elig, n, block_cnt, K, scale, ids,
                                                  packed);
    return cudaGetLastError();
}

cudaError_t launch_grad_unpack(const swgs_gaussians& grads, const int32_t* ids,
                               const long long* count, long long capacity, const float* packed,
                               cudaStream_t s) {
    if (capacity <= 0) return cudaSuccess;
    const int K = (grads.sh_degree + 1) * (grads.sh_degree + 1);
    note_launch();
    grad_unpack_kernel<<<(unsigned)div_up(capacity, 256), 256, 0, s>>>(grads, ids, count, K,
                                                                       packed);
    return cudaGetLastError();
}

__device__ __forceinline__ void adam1(float* p, float* m, float* v, float g, float lr,
                                      const SgldArgs& a) {
    const float mm = a.p.beta1 * *m + (1.f - a.p.beta1) * g;
    const float vv = a.p.beta2 * *v + (1.f - a.p.beta2) * g * g;
    const float mh = mm / a.bc1, vh = vv / a.bc2;
    *p = *p - lr * mh / (sqrtf(vh) + a.p.eps);
    *m = mm;
    *v = vv;
}

// The eligible slots among a block's 256 consecutive slots, gathered into
// s_ids (ascending) by one ballot a warp; returns their count. Eligible slots
// are a small, scattered fraction of the buffer, so the per-slot work below
// runs on packed lanes instead of leaving most lanes of most warps idle. Every
// thread of the block must call it.
__device__ __forceinline__ int gather_block_slots(bool take, long long i, int32_t* s_ids) {
    __shared__ int s_wcnt[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, take);
    if (lane == 0) s_wcnt[warp] = __popc(bal);
    __syncthreads();
    int off = 0, c = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const int n = s_wcnt[w];
        off += w < warp ? n : 0;
        c += n;
    }
    if (take) s_ids[off + __popc(bal & ((1u << lane) - 1u))] = (int32_t)i;
    __syncthreads();
    return c;
}

// Adam over one parameter array of W floats per slot for the c gathered
// slots, element-wise (a slot's W floats are contiguous); W is a compile-time
// width so the slot index is a multiply. With clear_grads each gradient
// element is zeroed once read.
template <int W, int ARR>
__device__ __forceinline__ void adam_slots(const SgldArgs& a, const int32_t* ids, int c,
                                           float* P, float* M, float* V, float* G, float lr) {
    for (int f = threadIdx.x; f < c * W; f += blockDim.x) {
        const int cs = f / W;
        const long long i = ids[cs];
        const long long e = i * W + (f - cs * W);
        float g = G[e];
        float l = lr;
        if (ARR == 0 && a.p.mean_grad_decay != 1.f && a.p.swin_size > 0) {
            // Sec. 4.5.1: the means gradient shrinks with the windows that have
            // trained the slot's current lifespan
            const int k = max(1, a.p.window_start - a.g.start[i] + a.p.swin_size);
            g *= exp2f((float)(k - 1) * log2f(a.p.mean_grad_decay));
        }
        if (ARR == 4 && (f - cs * W) < 3) l = a.p.lr_sh_dc;  // the DC band
        adam1(&P[e], &M[e], &V[e], g, l, a);
        if (a.p.clear_grads) G[e] = 0.f;
    }
}

template <int W>
__device__ __forceinline__ void clear_slots(const int32_t* ids, int c, float* G) {
    for (int f = threadIdx.x; f < c * W; f += blockDim.x) {
        const int cs = f / W;
        G[(long long)ids[cs] * W + (f - cs * W)] = 0.f;
    }
}

// SGLD noise of one eligible slot, from its (possibly updated) opacity and
// covariance: mu += lr_means noise_lr sigmoid(-k (o - t)) Sigma eta.
__device__ __forceinline__ void noise_slot(const SgldArgs& a, long long i) {
    const float o = 1.f / (1.f + expf(-a.g.opacity_logits[i]));
    const float gate = 1.f / (1.f + expf(a.p.noise_k * (o - a.p.noise_t)));
    const float scale = a.p.lr_means * a.p.noise_lr * gate;
    if (scale == 0.f) return;
    float s[3];
    for (int k = 0; k < 3; ++k) s[k] = expf(a.g.log_scales[3 * i + k]);
    const float4 q4 = reinterpret_cast<const float4*>(a.g.quats)[i];
    const float qi = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float w = q4.x * qi, x = q4.y * qi, y = q4.z * qi, z = q4.w * qi;
    const float R[3][3] = {
        {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
        {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
        {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
    const U64x4 rnd = philox4x64_10((unsigned long long)i, a.step, 0ULL, 0ULL, a.seed, kTagNoise);
    float u[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) u[k] = ((float)(rnd.v[k] >> 40) + 1.0f) * 0x1p-24f;
    const float r0 = sqrtf(-2.f * logf(u[0])), r1 = sqrtf(-2.f * logf(u[2]));
    float sn0, cs0, sn1, cs1;
    sincospif(2.f * u[1], &sn0, &cs0);
    sincospif(2.f * u[3], &sn1, &cs1);
    const float eta[3] = {r0 * cs0, r0 * sn0, r1 * cs1};
    // Sigma eta = R S^2 R^T eta
    float tq[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) tq[k] = (R[0][k] * eta[0] + R[1][k] * eta[1] + R[2][k] * eta[2]) * s[k] * s[k];
#pragma unroll
    for (int k = 0; k < 3; ++k)
        a.g.means[3 * i + k] += scale * (R[k][0] * tq[0] + R[k][1] * tq[1] + R[k][2] * tq[2]);
}

// One block per 256 slots: the eligible ones are gathered, take the Adam step
// (if on) array by array, then, once the block's updates are done, the noise.
template <int WSH>
__device__ __forceinline__ void adam_sgld_block(const SgldArgs& a) {
    __shared__ int32_t s_ids[256];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = gather_block_slots(i < a.g.capacity && a.elig[i], i, s_ids);
    if (c == 0) return;
    const swgs_gaussians& g = a.g;
    const swgs_gaussians& d = a.grads;
    const swgs_adam_state& m = a.adam;
    if (a.p.adam && a.has_grads && a.has_adam) {
        adam_slots<3, 0>(a, s_ids, c, g.means, m.m_means, m.v_means, d.means, a.p.lr_means);
        adam_slots<3, 1>(a, s_ids, c, g.log_scales, m.m_log_scales, m.v_log_scales,
                         d.log_scales, a.p.lr_log_scales);
        adam_slots<4, 2>(a, s_ids, c, g.quats, m.m_quats, m.v_quats, d.quats, a.p.lr_quats);
        adam_slots<1, 3>(a, s_ids, c, g.opacity_logits, m.m_logits, m.v_logits,
                         d.opacity_logits, a.p.lr_logits);
        adam_slots<WSH, 4>(a, s_ids, c, g.sh, m.m_sh, m.v_sh, d.sh, a.p.lr_sh_rest);
        __syncthreads();  // the noise reads the updated opacity and covariance
    } else if (a.p.clear_grads && a.has_grads) {
        // no Adam: the gradients are still left zero for the next backward
        clear_slots<3>(s_ids, c, d.means);
        clear_slots<3>(s_ids, c, d.log_scales);
        clear_slots<4>(s_ids, c, d.quats);
        clear_slots<1>(s_ids, c, d.opacity_logits);
        clear_slots<WSH>(s_ids, c, d.sh);
    }
    for (int t = threadIdx.x; t < c; t += blockDim.x) noise_slot(a, s_ids[t]);
}

__global__ void __launch_bounds__(256) adam_sgld_kernel(SgldArgs a) {
    if (a.gate && *a.gate) return;
    switch (a.g.sh_degree) {
        case 0: adam_sgld_block<3>(a); break;
        case 1: adam_sgld_block<12>(a); break;
        case 2: adam_sgld_block<27>(a); break;
        default: adam_sgld_block<48>(a); break;
    }
}

cudaError_t launch_sgld(const swgs_gaussians& g, const swgs_gaussians* grads,
                        const swgs_adam_state* adam, const uint8_t* elig,
                        const swgs_sgld_params& p, unsigned long long seed,
                        unsigned long long step, cudaStream_t s, const uint32_t* gate) {
    if (g.capacity <= 0) return cudaSuccess;
    SgldArgs a{};
    a.g = g;
    a.gate = gate;
    if (grads) a.grads = *grads;
    if (adam) a.adam = *adam;
    a.has_grads = grads != nullptr;
    a.has_adam = adam != nullptr;
    a.elig = elig;
    a.p = p;
    a.bc1 = (float)(1.0 - pow((double)p.beta1, (double)(step + 1)));
    a.bc2 = (float)(1.0 - pow((double)p.beta2, (double)(step + 1)));
    a.seed = seed;
    a.step = step;
    note_launch();
    adam_sgld_kernel<<<div_up(g.capacity, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Relocation
// ---------------------------------------------------------------------------
struct RelocArgs {
    swgs_gaussians g;
    const uint8_t* elig;
    const uint32_t* gate;  // nonzero: no slot is dead (nothing is relocated)
};

// weight = floor(sigmoid(logit) 2^32) for alive eligible slots, 0 otherwise;
// the sigmoid uses the polynomial exp so the integer matches any IEEE-754
// implementation of the same operation sequence.
// The FP64 arithmetic runs on the block's alive eligible slots gathered onto
// packed lanes (FP64 issue is the cost; those slots are a small fraction).
__global__ void __launch_bounds__(256)
reloc_weights_kernel(RelocArgs a, unsigned long long* __restrict__ weights,
                     uint8_t* __restrict__ dead) {
    __shared__ int32_t s_ids[256];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < a.g.capacity;
    const bool el = live && a.elig[i] && !(a.gate && *a.gate);
    const float lg = el ? a.g.opacity_logits[i] : 0.f;
    const bool d = el && lg <= kLogitDead;
    const bool need = el && !d;
    if (live) {
        dead[i] = d ? 1 : 0;
        if (!need) weights[i] = 0;
    }
    const int c = gather_block_slots(need, i, s_ids);
    for (int t = threadIdx.x; t < c; t += blockDim.x) {
        const long long j = s_ids[t];
        const double e = kd_exp(-(double)a.g.opacity_logits[j]);
        const double o = __ddiv_rn(1.0, __dadd_rn(1.0, e));
        double f = floor(__dmul_rn(o, 4294967296.0));
        if (f > 4294967295.0) f = 4294967295.0;
        weights[j] = (unsigned long long)f;
    }
}

cudaError_t launch_reloc_weights(const swgs_gaussians& g, const uint8_t* elig,
                                 unsigned long long* weights, uint8_t* dead, cudaStream_t s,
                                 const uint32_t* gate) {
    RelocArgs a{};
    a.g = g;
    a.elig = elig;
    a.gate = gate;
    note_launch();
    reloc_weights_kernel<<<div_up(g.capacity, 256), 256, 0, s>>>(a, weights, dead);
    return cudaGetLastError();
}

// target = first j with cdf[j] > floor(r * total / 2^64), r the slot's draw.
__global__ void __launch_bounds__(256)
reloc_sample_kernel(long long n, const uint8_t* __restrict__ dead,
                    const unsigned long long* __restrict__ cdf, unsigned long long seed,
                    unsigned long long step, int32_t* __restrict__ targets,
                    int32_t* __restrict__ counts, unsigned long long* __restrict__ n_dead) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long total = cdf[n - 1];
    int32_t tg = -1;
    if (dead[i] && total > 0) {
        const U64x4 r = philox4x64_10((unsigned long long)i, step, 0ULL, 0ULL, seed, kTagReloc);
        const unsigned long long x = __umul64hi(r.v[0], total);
        long long lo = 0, hi = n - 1;
        while (lo < hi) {
            const long long mid = lo + ((hi - lo) >> 1);
            if (cdf[mid] > x) hi = mid; else lo = mid + 1;
        }
        tg = (int32_t)lo;
        atomicAdd(&counts[lo], 1);
        atomicAdd(n_dead, 1ULL);
    }
    targets[i] = tg;
}

cudaError_t launch_reloc_sample(const swgs_gaussians& g, const uint8_t* dead,
                                const unsigned long long* cdf, unsigned long long seed,
                                unsigned long long step, int32_t* targets, int32_t* counts,
                                unsigned long long* n_dead, cudaStream_t s) {
    note_launch();
    reloc_sample_kernel<<<div_up(g.capacity, 256), 256, 0, s>>>(g.capacity, dead, cdf, seed,
                                                                 step, targets, counts, n_dead);
    return cudaGetLastError();
}

// 1 - (1-o)^(1/N) and the scale ratio o / sum_{k=1..N} C(N,k) (-1)^(k-1) o'^k / sqrt(k),
// which equals [14]'s double sum over i <= N, k < i (hockey-stick identity).
__device__ __forceinline__ void reloc_values(double o, int n, double* on, double* ratio) {
    const double onew = 1.0 - pow(1.0 - o, 1.0 / (double)n);
    double den = 0.0, c = 1.0, pw = 1.0;
    for (int k = 1; k <= n; ++k) {
        c = c * (double)(n - k + 1) / (double)k;
        pw *= onew;
        den += ((k & 1) ? 1.0 : -1.0) * c * pw / sqrt((double)k);
    }
    *on = onew;
    *ratio = o / den;
}

__device__ __forceinline__ void zero_moments(const swgs_adam_state& m, long long i, int K) {
    if (!m.m_means) return;
    for (int k = 0; k < 3; ++k) {
        m.m_means[3 * i + k] = 0.f; m.v_means[3 * i + k] = 0.f;
        m.m_log_scales[3 * i + k] = 0.f; m.v_log_scales[3 * i + k] = 0.f;
    }
    for (int k = 0; k < 4; ++k) { m.m_quats[4 * i + k] = 0.f; m.v_quats[4 * i + k] = 0.f; }
    m.m_logits[i] = 0.f; m.v_logits[i] = 0.f;
    for (int k = 0; k < 3 * K; ++k) { m.m_sh[i * 3 * K + k] = 0.f; m.v_sh[i * 3 * K + k] = 0.f; }
}

// Phase 0: each target's relocated values, once (FP64, on the block's target
// slots gathered onto packed lanes): log(ratio), the log-scale shift, and the
// new opacity logit log(o') - log(1 - o').
__global__ void __launch_bounds__(256)
reloc_values_kernel(swgs_gaussians g, const int32_t* __restrict__ counts, int max_n,
                    double* __restrict__ lr, float* __restrict__ nl) {
    __shared__ int32_t s_ids[256];
    const long long j0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = gather_block_slots(j0 < g.capacity && counts[j0] != 0, j0, s_ids);
    if ((int)threadIdx.x >= c) return;
    const long long j = s_ids[threadIdx.x];
    int nn = counts[j] + 1;
    if (nn > max_n) nn = max_n;
    const double o = 1.0 / (1.0 + exp(-(double)g.opacity_logits[j]));
    double on, ratio;
    reloc_values(o, nn, &on, &ratio);
    lr[j] = log(ratio);
    nl[j] = (float)(log(on) - log1p(-on));
}

// Phase 1 (before the targets change): each dead slot copies its target with
// the target's relocated opacity and scale. Both phases gather the block's
// slots that have work onto packed lanes.
__global__ void __launch_bounds__(256)
reloc_copy_kernel(swgs_gaussians g, swgs_adam_state m, const int32_t* __restrict__ targets,
                  const double* __restrict__ lr, const float* __restrict__ nl) {
    __shared__ int32_t s_ids[256];
    const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = gather_block_slots(i0 < g.capacity && targets[i0] >= 0, i0, s_ids);
    if ((int)threadIdx.x >= c) return;
    const long long i = s_ids[threadIdx.x];
    const long long j = targets[i];
    const int K = (g.sh_degree + 1) * (g.sh_degree + 1);
    const double l = lr[j];
    for (int k = 0; k < 3; ++k) {
        g.means[3 * i + k] = g.means[3 * j + k];
        g.log_scales[3 * i + k] = (float)((double)g.log_scales[3 * j + k] + l);
    }
    for (int k = 0; k < 4; ++k) g.quats[4 * i + k] = g.quats[4 * j + k];
    g.opacity_logits[i] = nl[j];
    for (int k = 0; k < 3 * K; ++k) g.sh[i * 3 * K + k] = g.sh[j * 3 * K + k];
    zero_moments(m, i, K);
}

// Phase 2: every target takes its own relocated opacity and scale.
__global__ void __launch_bounds__(256)
reloc_target_kernel(swgs_gaussians g, swgs_adam_state m, const int32_t* __restrict__ counts,
                    const double* __restrict__ lr, const float* __restrict__ nl) {
    __shared__ int32_t s_ids[256];
    const long long j0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = gather_block_slots(j0 < g.capacity && counts[j0] != 0, j0, s_ids);
    if ((int)threadIdx.x >= c) return;
    const long long j = s_ids[threadIdx.x];
    const int K = (g.sh_degree + 1) * (g.sh_degree + 1);
    const double l = lr[j];
    for (int k = 0; k < 3; ++k)
        g.log_scales[3 * j + k] = (float)((double)g.log_scales[3 * j + k] + l);
    g.opacity_logits[j] = nl[j];
    zero_moments(m, j, K);
}

cudaError_t launch_reloc_apply(const swgs_gaussians& g, const swgs_adam_state* adam,
                               const int32_t* targets, const int32_t* counts, int max_n,
                               double* lr, float* nl, cudaStream_t s) {
    swgs_adam_state m{};
    if (adam) m = *adam;
    const int grid = div_up(g.capacity, 256);
    note_launch();
    reloc_values_kernel<<<grid, 256, 0, s>>>(g, counts, max_n, lr, nl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    note_launch();
    reloc_copy_kernel<<<grid, 256, 0, s>>>(g, m, targets, lr, nl);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    note_launch();
    reloc_target_kernel<<<grid, 256, 0, s>>>(g, m, counts, lr, nl);
    return cudaGetLastError();
}

}  // namespace swgs
