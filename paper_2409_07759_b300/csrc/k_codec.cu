// k_codec.cu -- the streamed-slice codec: Table 6 attribute quantisation
// (Sec. 5.6.2: means and log-scales fp16, rotation uint8, opacity uint8, only
// the DC of the SH kept at full precision) and the Sec. 5.5 tail drop of a
// slice's lowest-opacity Gaussians, on the device.
//
// Packet: a 32-byte header (magic, version, count, keep, sh_degree, birth,
// start, expire) and 16-byte-aligned sections: slot index u32[keep] (only when
// keep < count), means f16[keep][3], log_scales f16[keep][3], quaternion
// codes u8[keep][4], opacity codes u8[keep], DC f32[keep][3].
#include <cuda_fp16.h>

#include "swgs_internal.cuh"

namespace swgs {

__host__ __device__ inline size_t codec_align(size_t x) { return (x + 15) & ~(size_t)15; }

void codec_layout(long long count, long long keep, CodecLayout* L) {
    size_t o = kCodecHeaderBytes;
    L->index = 0;
    if (keep < count) {
        L->index = o;
        o += codec_align(4 * (size_t)keep);
    }
    L->means = o;
    o += codec_align(6 * (size_t)keep);
    L->log_scales = o;
    o += codec_align(6 * (size_t)keep);
    L->quats = o;
    o += codec_align(4 * (size_t)keep);
    L->opacity = o;
    o += codec_align((size_t)keep);
    L->dc = o;
    o += codec_align(12 * (size_t)keep);
    L->total = o;
}

// Descending-logit sort key (stable ascending sort => highest opacity first,
// equal logits in slot order).
__global__ void codec_keys_kernel(const float* __restrict__ logits, long long n,
                                  uint32_t* __restrict__ keys) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t u = __float_as_uint(logits[i]);
    const uint32_t asc = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    keys[i] = ~asc;
}

// flags[sorted_slot[j]] = 1 for the first `keep` entries of the ranking. A
// sort whose look-back wait ran out may leave stale words in the ranking:
// those past the slice are dropped (the error word reports the failure).
__global__ void codec_flag_kernel(const uint32_t* __restrict__ ranked, long long keep,
                                  long long count, uint8_t* __restrict__ flags) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < keep) {
        const uint32_t r = ranked[j];
        if ((long long)r < count) flags[r] = 1;
    }
}

__global__ void __launch_bounds__(256)
codec_flag_count_kernel(const uint8_t* __restrict__ flags, long long n,
                        uint32_t* __restrict__ block_counts) {
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    const int c = __syncthreads_count(i < n && flags[i]);
    if (threadIdx.x == 0) block_counts[blockIdx.x] = (uint32_t)c;
}

__global__ void __launch_bounds__(256)
codec_flag_write_kernel(const uint8_t* __restrict__ flags, long long n,
                        const uint32_t* __restrict__ block_offsets, uint32_t* __restrict__ idx) {
    __shared__ int warp_off[8];
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    const bool m = i < n && flags[i];
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, m);
    if (lane == 0) warp_off[warp] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < 8; ++w) {
            const int c = warp_off[w];
            warp_off[w] = run;
            run += c;
        }
    }
    __syncthreads();
    if (m) idx[block_offsets[blockIdx.x] + warp_off[warp] + __popc(bal & ((1u << lane) - 1u))] =
        (uint32_t)i;
}

// Row j of the packet = slot idx[j] of src (or slot j when idx is null).
__global__ void codec_encode_kernel(swgs_gaussians src, const uint32_t* __restrict__ idx,
                                    long long count, long long keep, CodecLayout L,
                                    unsigned char* __restrict__ out) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int K = (src.sh_degree + 1) * (src.sh_degree + 1);
    if (j == 0) {
        int32_t* h = (int32_t*)out;
        h[0] = (int32_t)kCodecMagic;
        h[1] = kCodecVersion;
        h[2] = (int32_t)count;
        h[3] = (int32_t)keep;
        h[4] = src.sh_degree;
        h[5] = count > 0 ? src.birth[0] : 0;
        h[6] = count > 0 ? src.start[0] : 0;
        h[7] = count > 0 ? src.expire[0] : 0;
    }
    if (j >= keep) return;
    const long long i = idx ? (long long)idx[j] : j;
    if (idx) ((uint32_t*)(out + L.index))[j] = (uint32_t)i;
    __half* m = (__half*)(out + L.means) + 3 * j;
    __half* s = (__half*)(out + L.log_scales) + 3 * j;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        m[c] = __float2half_rn(src.means[3 * i + c]);
        s[c] = __float2half_rn(src.log_scales[3 * i + c]);
    }
    // unit quaternion, component c -> rint((q_c + 1) * 127.5)
    const float q0 = src.quats[4 * i], q1 = src.quats[4 * i + 1], q2 = src.quats[4 * i + 2],
                q3 = src.quats[4 * i + 3];
    float nn = kmul(q0, q0);
    nn = kadd(nn, kmul(q1, q1));
    nn = kadd(nn, kmul(q2, q2));
    nn = kadd(nn, kmul(q3, q3));
    const float n = __fsqrt_rn(nn);
    const float qs[4] = {q0, q1, q2, q3};
    unsigned char* qc = out + L.quats + 4 * j;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float t = rintf(kmul(kadd(__fdiv_rn(qs[c], n), 1.0f), 127.5f));
        t = fminf(fmaxf(t, 0.0f), 255.0f);
        qc[c] = (unsigned char)t;
    }
    // opacity -> rint(255 sigmoid(logit)), the sigmoid through the key-mode exp
    const float o = __fdiv_rn(1.0f, kadd(1.0f, km_exp(-src.opacity_logits[i])));
    float t = rintf(kmul(o, 255.0f));
    t = fminf(fmaxf(t, 0.0f), 255.0f);
    out[L.opacity + j] = (unsigned char)t;
    float* dc = (float*)(out + L.dc) + 3 * j;
    const float* sh = src.sh + (long long)i * K * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) dc[c] = sh[c];
}

// Every slot of the slice emptied: zero attributes, start = expire = the
// slice's start (never active), birth, frozen = 1.
__global__ void codec_clear_kernel(swgs_gaussians dst, long long first, long long count,
                                   int32_t birth, int32_t start) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= count) return;
    const long long i = first + r;
    const int K = (dst.sh_degree + 1) * (dst.sh_degree + 1);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        dst.means[3 * i + c] = 0.f;
        dst.log_scales[3 * i + c] = 0.f;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) dst.quats[4 * i + c] = 0.f;
    dst.opacity_logits[i] = 0.f;
    for (int c = 0; c < 3 * K; ++c) dst.sh[i * 3 * K + c] = 0.f;
    dst.start[i] = start;
    dst.expire[i] = start;
    if (dst.birth) dst.birth[i] = birth;
    if (dst.frozen) dst.frozen[i] = 1;
}

__global__ void codec_decode_kernel(swgs_gaussians dst, long long first, long long keep,
                                    CodecLayout L, const unsigned char* __restrict__ in,
                                    int32_t birth, int32_t start, int32_t expire,
                                    bool has_index) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= keep) return;
    const long long i = first + (has_index ? (long long)((const uint32_t*)(in + L.index))[j] : j);
    const int K = (dst.sh_degree + 1) * (dst.sh_degree + 1);
    const __half* m = (const __half*)(in + L.means) + 3 * j;
    const __half* s = (const __half*)(in + L.log_scales) + 3 * j;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        dst.means[3 * i + c] = __half2float(m[c]);
        dst.log_scales[3 * i + c] = __half2float(s[c]);
    }
    const unsigned char* qc = in + L.quats + 4 * j;
#pragma unroll
    for (int c = 0; c < 4; ++c) dst.quats[4 * i + c] = ksub(kmul((float)qc[c], 2.0f / 255.0f), 1.0f);
    const float o = __fdiv_rn(fminf(fmaxf((float)in[L.opacity + j], 0.5f), 254.5f), 255.0f);
    dst.opacity_logits[i] = logf(__fdiv_rn(o, ksub(1.0f, o)));
    const float* dc = (const float*)(in + L.dc) + 3 * j;
    float* sh = dst.sh + i * 3 * K;
#pragma unroll
    for (int c = 0; c < 3; ++c) sh[c] = dc[c];
    for (int c = 3; c < 3 * K; ++c) sh[c] = 0.f;
    dst.start[i] = start;
    dst.expire[i] = expire;
    if (dst.birth) dst.birth[i] = birth;
    if (dst.frozen) dst.frozen[i] = 1;
}

cudaError_t launch_codec_select(const float* logits, long long count, long long keep,
                                CodecScratch& w, int num_sms, uint32_t** out_idx, cudaStream_t s) {
    // ranking by descending logit (stable: ties in slot order)
    note_launch();
    codec_keys_kernel<<<div_up(count, 256), 256, 0, s>>>(logits, count, w.keys_a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const SortPlan plan = make_sort_plan(0, 32);
    bool in_b = false;
    e = radix_sort_pairs(w.keys_a, w.vals_a, w.keys_b, w.vals_b, count, plan, w.sort_tmp, num_sms,
                         true, &in_b, w.sort_single_pass, w.sort_err, s);
    if (e != cudaSuccess) return e;
    const uint32_t* ranked = in_b ? w.vals_b : w.vals_a;
    e = cudaMemsetAsync(w.flags, 0, (size_t)count, s);
    if (e != cudaSuccess) return e;
    note_launch();
    codec_flag_kernel<<<div_up(keep, 256), 256, 0, s>>>(ranked, keep, count, w.flags);
    const long long nb = div_up(count, 256);
    note_launch();
    codec_flag_count_kernel<<<(unsigned)nb, 256, 0, s>>>(w.flags, count, w.block_cnt);
    e = exclusive_scan_u32(w.block_cnt, w.block_cnt, nb, w.scan_tmp, w.total, s);
    if (e != cudaSuccess) return e;
    note_launch();
    codec_flag_write_kernel<<<(unsigned)nb, 256, 0, s>>>(w.flags, count, w.block_cnt, w.idx);
    *out_idx = w.idx;
    return cudaGetLastError();
}

cudaError_t launch_codec_encode(const swgs_gaussians& src, const uint32_t* idx, long long count,
                                long long keep, const CodecLayout& L, unsigned char* out,
                                cudaStream_t s) {
    note_launch();
    codec_encode_kernel<<<div_up(keep > 0 ? keep : 1, 256), 256, 0, s>>>(src, idx, count, keep, L,
                                                                         out);
    return cudaGetLastError();
}

cudaError_t launch_codec_decode(const swgs_gaussians& dst, long long first, long long count,
                                long long keep, const CodecLayout& L, const unsigned char* in,
                                int32_t birth, int32_t start, int32_t expire, cudaStream_t s) {
    if (keep < count && count > 0) {
        note_launch();
        codec_clear_kernel<<<div_up(count, 256), 256, 0, s>>>(dst, first, count, birth, start);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (keep <= 0) return cudaSuccess;
    note_launch();
    codec_decode_kernel<<<div_up(keep, 256), 256, 0, s>>>(dst, first, keep, L, in, birth, start,
                                                          expire, keep < count);
    return cudaGetLastError();
}

}  // namespace swgs
