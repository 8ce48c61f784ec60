// noalloc.cu -- the active-set compaction without any allocation.
//
// Some callers cannot let a library allocate device memory: their device
// memory is owned by one allocator or budget (a host engine's pool, a
// memory-capped serving process), so an extra cudaMalloc breaks their
// accounting, or they run on latency-critical threads where cudaMalloc's
// device-wide synchronisation is not acceptable. swgs_active_ids_noalloc
// serves them: it runs the same count / scan / write kernels as
// swgs_active_ids, but its scratch (per-block counts, scan partials, the frame
// word) lives in one fixed array compiled into the library, so it needs no
// context and allocates nothing.
#include "swgs_internal.cuh"

namespace swgs {

namespace {

constexpr long long kNoAllocMaxBlocks =
    (SWGS_NOALLOC_MAX_SLOTS + kCompactBlock - 1) / kCompactBlock;
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }
// layout: [frame int32 | scan total u64] [block counts u32 x (blocks+1)] [scan partials]
constexpr size_t kOffTotal = 64;
constexpr size_t kOffCounts = kAlign;
constexpr size_t kOffParts =
    kOffCounts + align_up(sizeof(uint32_t) * (size_t)(kNoAllocMaxBlocks + 1));
constexpr size_t kPartsBytes = sizeof(unsigned long long) * ((kNoAllocMaxBlocks + 1 + 4095) / 4096 + 1);
constexpr size_t kScratchBytes = kOffParts + align_up(kPartsBytes);

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the array in the current context, looked up on every
// call: cudaGetSymbolAddress allocates nothing and costs little, and an
// address cached across calls would go stale after cudaDeviceReset or under
// another context on the same device. (Host code must not pass the array's
// own name to a kernel: in host code that name is only a stand-in.)
cudaError_t scratch_address(void** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

__global__ void set_frame_kernel(int32_t* dst, int32_t frame) { *dst = frame; }

}  // namespace

}  // namespace swgs

using namespace swgs;

extern "C" swgs_status swgs_active_ids_noalloc(const int32_t* start, const int32_t* expire,
                                               int64_t n, int32_t frame, int32_t* out_ids,
                                               int32_t* out_count, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (n < 0 || n > (int64_t)SWGS_NOALLOC_MAX_SLOTS || !out_count ||
        (n > 0 && (!start || !expire || !out_ids)))
        return SWGS_EINVAL;
    if (n == 0) return cudaMemsetAsync(out_count, 0, sizeof(int32_t), s) == cudaSuccess
                           ? SWGS_OK : SWGS_ECUDA;
    void* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return SWGS_ECUDA;
    char* b = (char*)base;
    int32_t* frame_dev = (int32_t*)b;
    unsigned long long* total = (unsigned long long*)(b + kOffTotal);
    uint32_t* counts = (uint32_t*)(b + kOffCounts);
    void* parts = b + kOffParts;
    const int nb = (int)((n + kCompactBlock - 1) / kCompactBlock);
    // every word the kernels read is written earlier in this call, so nothing
    // from the previous call needs clearing
    note_launch();
    set_frame_kernel<<<1, 1, 0, s>>>(frame_dev, frame);
    if (cudaGetLastError() != cudaSuccess) return SWGS_ECUDA;
    if (launch_active_flags_count(start, expire, n, frame_dev, 1, counts, nb, s) != cudaSuccess ||
        exclusive_scan_u32(counts, counts, nb, parts, total, s) != cudaSuccess ||
        launch_active_write(start, expire, n, frame_dev, 1, counts, nb, out_ids, 0, out_count, s) !=
            cudaSuccess)
        return SWGS_ECUDA;
    return SWGS_OK;
}
