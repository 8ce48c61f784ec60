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

// ---------------------------------------------------------------------------
// Deferred sizing: the tables and totals of a batch from device counts.
// ---------------------------------------------------------------------------
__global__ void plan_kernel(GroupDev* groups, int n_groups, ViewDev* views,
                            const int32_t* __restrict__ counts, unsigned long long* totals,
                            long long rec_cap, long long act_cap) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    long long act = 0, rec = 0;
    for (int k = 0; k < n_groups; ++k) {
        GroupDev& G = groups[k];
        const int n = counts[k];
        G.n_active = n;
        G.act_base = (int)act;
        G.rec_base = (int)rec;
        G.reg_o = n > 0 ? (float)(G.reg_o_num / (double)n) : 0.f;
        G.reg_s = n > 0 ? (float)(G.reg_s_num / (double)n) : 0.f;
        for (int j = 0; j < G.view_count; ++j) {
            ViewDev& V = views[G.view_begin + j];
            V.rec_base = (int)(rec + (long long)j * n);
            V.n_rec = n;
        }
        act += n;
        rec += (long long)n * G.view_count;
    }
    if (totals) {
        totals[kTotNeedRecords] = (unsigned long long)rec;
        totals[kTotNeedActive] = (unsigned long long)act;
        if (rec > rec_cap || act > act_cap) {
            totals[kTotStatus] |= 1ull;
            rec = 0;
            act = 0;
        }
        totals[kTotRecords] = (unsigned long long)rec;
        totals[kTotActive] = (unsigned long long)act;
    }
}

cudaError_t launch_plan(GroupDev* groups, int n_groups, ViewDev* views, const int32_t* counts,
                        unsigned long long* totals, long long rec_cap, long long act_cap,
                        cudaStream_t s) {
    note_launch();
    plan_kernel<<<1, 32, 0, s>>>(groups, n_groups, views, counts, totals, rec_cap, act_cap);
    return cudaGetLastError();
}

__global__ void check_keys_kernel(const unsigned long long* __restrict__ key_totals,
                                  unsigned long long* totals, long long super_cap,
                                  long long key_cap, uint32_t* sort_err, uint32_t* gate) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long st = totals[kTotStatus];
    if (sort_err && *sort_err) {
        st |= 4ull;
        *sort_err = 0u;
    }
    if (key_totals) {
        // before the key emission: a wait that ran out left the depth order
        // unusable, so it stops the batch like an overflow does
        const unsigned long long sk = key_totals[0], tk = key_totals[1];
        totals[kTotNeedSuperKeys] = sk;
        totals[kTotNeedTileKeys] = tk;
        if ((long long)sk > super_cap || (long long)tk > key_cap) st |= 2ull;
        const bool stop = (st & 7ull) != 0ull;
        totals[kTotSuperKeys] = stop ? 0ull : sk;
        totals[kTotTileKeys] = stop ? 0ull : tk;
        if (stop) {
            totals[kTotRecords] = 0ull;
            totals[kTotActive] = 0ull;
        }
    }
    totals[kTotStatus] = st;
    if (gate && st) atomicOr(gate, (uint32_t)st);
}

cudaError_t launch_check_keys(const unsigned long long* key_totals, unsigned long long* totals,
                              long long super_cap, long long key_cap, uint32_t* sort_err,
                              uint32_t* gate, cudaStream_t s) {
    note_launch();
    check_keys_kernel<<<1, 32, 0, s>>>(key_totals, totals, super_cap, key_cap, sort_err, gate);
    return cudaGetLastError();
}

}  // namespace swgs
