// k_misc.cu -- the L1 photometric term (Alg. 1 loss_func) and the
// device-to-device slice copy of the per-frame update (Alg. 2 update_thread).
#include "swgs_internal.cuh"

namespace swgs {

struct L1Args {
    const long long* pix_off;   // [V+1] pixel offsets of the views
    const float* const* rgb;    // [V] device pointers
    const float* const* target;
    float* const* dl;
    int n_views;
    long long total_pix;
    float* loss;
};

__global__ void __launch_bounds__(256) loss_l1_kernel(L1Args a) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float part = 0.f;
    if (p < a.total_pix) {
        int lo = 0, hi = a.n_views - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (a.pix_off[mid] <= p) lo = mid; else hi = mid - 1;
        }
        const long long hw = a.pix_off[lo + 1] - a.pix_off[lo], q = p - a.pix_off[lo];
        const float inv = 1.0f / (3.0f * (float)hw * (float)a.n_views);
        const float* c = a.rgb[lo];
        const float* t = a.target[lo];
        float* d = a.dl[lo];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float diff = c[ch * hw + q] - t[ch * hw + q];
            part += fabsf(diff);
            d[ch * hw + q] = diff > 0.f ? inv : (diff < 0.f ? -inv : 0.f);
        }
        part *= inv;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    __shared__ float ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < 8; ++w) s += ws[w];
        if (s != 0.f) atomicAdd(a.loss, s);
    }
}

cudaError_t launch_loss_l1(const ViewDev*, int n_views, long long total_pix,
                           const long long* pix_offsets, const float* const* rgb,
                           const float* const* target, float* const* dl, float* loss,
                           cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), s);
    if (e != cudaSuccess || total_pix <= 0) return e;
    L1Args a{pix_offsets, rgb, target, dl, n_views, total_pix, loss};
    note_launch();
    loss_l1_kernel<<<div_up(total_pix, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

// Copy `count` slots of every attribute array: blockIdx.y picks the array.
struct SliceArgs {
    void* dst[9];
    const void* src[9];
    long long words[9];    // 32-bit words per slot (frozen: counted in bytes)
    long long count;
    long long first;
};

__global__ void __launch_bounds__(256) copy_slice_kernel(SliceArgs a) {
    const int arr = blockIdx.y;
    if (a.dst[arr] == nullptr) return;
    const long long n = a.count * a.words[arr];
    if (arr == 8) {  // uint8 frozen flags
        uint8_t* d = (uint8_t*)a.dst[arr] + a.first;
        const uint8_t* s = (const uint8_t*)a.src[arr];
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x)
            d[i] = s[i];
        return;
    }
    uint32_t* d = (uint32_t*)a.dst[arr] + a.first * a.words[arr];
    const uint32_t* s = (const uint32_t*)a.src[arr];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        d[i] = s[i];
}

cudaError_t launch_copy_slice(const swgs_gaussians& dst, long long first, long long count,
                              const swgs_gaussians& src, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int K = (dst.sh_degree + 1) * (dst.sh_degree + 1);
    SliceArgs a{};
    void* d[9] = {dst.means, dst.log_scales, dst.quats, dst.opacity_logits, dst.sh,
                  dst.start, dst.expire, dst.birth, dst.frozen};
    const void* sp[9] = {src.means, src.log_scales, src.quats, src.opacity_logits, src.sh,
                         src.start, src.expire, src.birth, src.frozen};
    const long long w[9] = {3, 3, 4, 1, 3LL * K, 1, 1, 1, 1};
    for (int i = 0; i < 9; ++i) {
        a.dst[i] = sp[i] ? d[i] : nullptr;
        a.src[i] = sp[i];
        a.words[i] = w[i];
    }
    a.count = count;
    a.first = first;
    long long mx = count * 3LL * K;
    int gx = div_up(mx, 256);
    if (gx > 1184) gx = 1184;
    note_launch();
    copy_slice_kernel<<<dim3(gx, 9), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace swgs
