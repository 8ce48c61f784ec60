// swgs_internal.cuh -- device-side building blocks shared by the kernels of
// libswgs (SwinGS frame-t splatting, arXiv 2409.07759).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/swgs.h"

namespace swgs {

constexpr int kMaxViewsPerBatch = 512;
constexpr int kMaxShCoeffs = 16;  // degree 3

// ---------------------------------------------------------------------------
// Per-view and per-frame-group descriptors (device copies live in the saved
// state of a forward call).
// ---------------------------------------------------------------------------
struct ViewDev {
    int W, H, ntx, nty;
    int tile_base;     // first global tile id of this view inside its batch
    int super_base;    // first global super-tile id of this view inside its batch
    int nsx, nsy;      // super tiles across and down
    int rec_base;      // first record of this view
    int n_rec;         // records of this view (= active Gaussians of its frame)
    int group;         // frame group index
    long long pix_base;  // first pixel of this view in the batch's pixel arrays
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    float campos[3];
    float bg[3];
    float* out_rgb;    // [3,H,W] or null
    uint8_t* out_rgb8; // [H,W,3] 8-bit RGB (round(255 clamp(c, 0, 1))) or null
    float* out_T;      // [H,W] or null
    const float* dL;   // [3,H,W] (backward only)
    const float* target;  // [3,H,W] (forward fused with the L1 term) or null
    const uint8_t* target_u8;  // or [3,H,W] 8-bit, value k / 255
    float* dL_out;        // [3,H,W] written with the L1 gradient (fused forward)
    float l1_scale;       // 1 / (3 H W V)
};

struct GroupDev {
    int frame;
    int n_active;      // active Gaussians of this frame
    int act_base;      // offset of this group's ids in the ids array
    int rec_base;      // first record of this group
    int view_begin;    // first view of this group (views of a group are contiguous)
    int view_count;
    float reg_o, reg_s;  // regulariser weights of one active Gaussian (backward)
    // the weights before the division by n_active (set by the host; the plan
    // kernel divides once the count is known on the device)
    double reg_o_num, reg_s_num;
};

// Device totals of one batch (deferred sizing keeps them on the device; the
// plan and check kernels write them, later launches read their counts).
enum BatchTotal {
    kTotRecords = 0,    // records (view, active Gaussian)
    kTotActive = 1,     // active ids over the frame groups
    kTotSuperKeys = 2,  // (super tile, record) keys
    kTotTileKeys = 3,   // per-tile list entries
    kTotStatus = 4,     // bit 0: records over capacity, bit 1: keys over capacity,
                        // bit 2: a sort's look-back wait ran out
    kTotNeedRecords = 5, kTotNeedSuperKeys = 6, kTotNeedTileKeys = 7, kTotNeedActive = 8,
    kTotWords = 9
};

// Records of one (view, Gaussian) pair, structure of float4 arrays.
struct Records {
    float4* a;         // u, v, opacity, depth
    float4* b;         // conic A, B, C (m = A dx^2 + 2B dx dy + C dy^2), 0
    float4* c;         // r, g, b, 0
    int32_t* tiles;    // tiles touched (0 if culled)
    short4* rect;      // tx0, tx1, ty0, ty1
    uint32_t* depth_key;  // FP32 depth bits, 0xffffffff if no tiles
    uint16_t* runs;    // kRunRows per record: first - tx0 (low byte), length (high byte)
    int32_t* supers;   // super tiles holding at least one of the record's tiles
};

// Rows of a record whose tile runs are stored; taller rectangles recompute the rest.
constexpr int kRunRows = 32;

// ---------------------------------------------------------------------------
// Thresholds of the per-pixel compositing rule (Eq. 3 plus the readings of
// the renderer details the paper leaves to 3DGS).
// ---------------------------------------------------------------------------
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTStop = 1e-4f;
constexpr float kDilation = 0.3f;
constexpr float kGuard = 1.3f;
// m <= 9 written in the log2 domain q = -m/2 * log2(e)
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kQMin = -4.5f * 1.4426950408889634f;
// alpha >= 1/255 written in the log2 domain: q + log2(o) >= log2(1/255)
constexpr float kLog2AlphaMin = -7.99435343685885793f;
constexpr float kLn2 = 0.6931471805599453f;

// ---------------------------------------------------------------------------
// Key mode: one correctly rounded FP32 operation per step, never contracted
// into FMA, so that the discrete quantities (culling, tile rectangle, tile
// count, depth key) are reproducible bit for bit by an independent CPU
// implementation of the same operation sequence.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float kadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float ksub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float kmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float kdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float ksqrt(float a) { return __fsqrt_rn(a); }

// exp(x) for the discrete path: Cody-Waite reduction x = k ln2 + r (ln2 split
// into a 16-bit head and a tail), the degree-7 Taylor polynomial of exp(r) by
// Horner's rule, and an exact scaling by 2^k.
__device__ __forceinline__ float km_exp(float x) {
    x = x < -80.0f ? -80.0f : (x > 80.0f ? 80.0f : x);
    float t = kmul(x, 0x1.715476p+0f);
    t = kadd(t, 0.5f);
    float k = floorf(t);
    float r = ksub(x, kmul(k, 0x1.62e4p-1f));
    r = ksub(r, kmul(k, 0x1.7f7d1cp-20f));
    float p = 0x1.a01a02p-13f;
    p = kadd(kmul(p, r), 0x1.6c16c2p-10f);
    p = kadd(kmul(p, r), 0x1.111112p-7f);
    p = kadd(kmul(p, r), 0x1.555556p-5f);
    p = kadd(kmul(p, r), 0x1.555556p-3f);
    p = kadd(kmul(p, r), 0.5f);
    p = kadd(kmul(p, r), 1.0f);
    p = kadd(kmul(p, r), 1.0f);
    int e = (int)k;
    return kmul(p, __int_as_float((e + 127) << 23));
}

// Same construction in FP64 (degree 13); used where an integer is derived
// from a float (the relocation weights).
__device__ __forceinline__ double kd_exp(double x) {
    x = x < -700.0 ? -700.0 : (x > 700.0 ? 700.0 : x);
    double t = __dmul_rn(x, 0x1.71547652b82fep+0);
    t = __dadd_rn(t, 0.5);
    double k = floor(t);
    double r = __dsub_rn(x, __dmul_rn(k, 0x1.62e42feep-1));
    r = __dsub_rn(r, __dmul_rn(k, 0x1.a39ef35793c76p-33));
    const double P[14] = {
        0x1p+0, 0x1p+0, 0x1p-1, 0x1.5555555555555p-3, 0x1.5555555555555p-5,
        0x1.1111111111111p-7, 0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13,
        0x1.a01a01a01a01ap-16, 0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22,
        0x1.ae64567f544e4p-26, 0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33};
    double p = P[13];
#pragma unroll
    for (int i = 12; i >= 0; --i) p = __dadd_rn(__dmul_rn(p, r), P[i]);
    long long e = (long long)k;
    return __dmul_rn(p, __longlong_as_double((e + 1023) << 52));
}

// A tile is kept when the ellipse {m <= 9.009} reaches the rectangle spanned
// by its pixel centres: the 3-sigma support plus 0.1%, so FP32 rounding never
// drops a tile holding a pixel with m <= 9.
constexpr float kTileMahal = 9.009f;

// Row rule (key mode): the ellipse meets a band of pixel-centre rows in a
// convex set, so the kept tiles of a tile row form one run; its x-extent
// [left, right] over the band comes from the chord ends c(y) -+ w(y) at the
// band ends (c = -(B/A) y, w = sqrt(A T - det_c y^2) / A) and from the
// ellipse's extreme points (+-xm, -+(B/C) xm), xm = sqrt(C T / det_c).
struct KmEllipse {
    float AT, detc, rBA, iA, rBC, xm, ym;
};

__device__ __forceinline__ KmEllipse km_ellipse(float A, float B, float C) {
    KmEllipse e;
    e.AT = kmul(A, kTileMahal);
    e.detc = ksub(kmul(A, C), kmul(B, B));
    e.rBA = kdiv(B, A);
    e.iA = kdiv(1.0f, A);
    e.rBC = kdiv(B, C);
    e.xm = ksqrt(kdiv(kmul(C, kTileMahal), e.detc));
    e.ym = ksqrt(kdiv(e.AT, e.detc));
    return e;
}

// The two ends c(y) -+ w(y) of the ellipse's chord at row offset y.
__device__ __forceinline__ void km_chord(const KmEllipse& e, float y, float* l, float* r) {
    const float c = -kmul(e.rBA, y);
    float q = ksub(e.AT, kmul(kmul(e.detc, y), y));
    q = q < 0.0f ? 0.0f : q;
    const float w = kmul(ksqrt(q), e.iA);
    *l = ksub(c, w);
    *r = kadd(c, w);
}

__device__ __forceinline__ bool km_row_extent(const KmEllipse& e, float ya, float yb,
                                              float* left, float* right) {
    const float lo = ya > -e.ym ? ya : -e.ym;
    const float hi = yb < e.ym ? yb : e.ym;
    if (!(lo <= hi)) return false;
    const float t = kmul(e.rBC, e.xm);
    const float dyr = -t, dyl = t;
    float l0, r0, l1, r1;
    km_chord(e, lo, &l0, &r0);
    km_chord(e, hi, &l1, &r1);
    *right = (lo <= dyr && dyr <= hi) ? e.xm : (r0 > r1 ? r0 : r1);
    *left = (lo <= dyl && dyl <= hi) ? -e.xm : (l0 < l1 ? l0 : l1);
    return true;
}

// Same result as km_row_run, with the two end searches started from a guess
// and adjusted: both predicates (pixel-centre span end >= left, start <=
// right) are monotone in the tile index, so the smallest / largest index
// satisfying them is unique whatever the starting point.
__device__ __forceinline__ int km_row_run_fast(const KmEllipse& e, float u, float v, int tx0,
                                               int tx1, int ty, int tile_w, int tile_h,
                                               int* first, int* last) {
    if (!(e.detc > 0.0f)) { *first = tx0; *last = tx1; return tx1 - tx0 + 1; }
    const float by = (float)(ty * tile_h);
    const float ya = ksub(kadd(by, 0.5f), v);
    const float yb = ksub(kadd(by, (float)tile_h - 0.5f), v);
    float left, right;
    if (!km_row_extent(e, ya, yb, &left, &right)) return 0;
    const float itw = 1.0f / (float)tile_w;
    const float hi_off = (float)tile_w - 0.5f;
    auto xb_of = [&](int t) { return ksub(kadd((float)(t * tile_w), hi_off), u); };
    auto xa_of = [&](int t) { return ksub(kadd((float)(t * tile_w), 0.5f), u); };
    float ga = floorf((left + u) * itw);
    ga = fminf(fmaxf(ga, (float)tx0), (float)(tx1 + 1));
    int a = (int)ga;
    while (a > tx0 && xb_of(a - 1) >= left) --a;
    while (a <= tx1 && !(xb_of(a) >= left)) ++a;
    if (a > tx1) return 0;
    float gb = floorf((right + u) * itw);
    gb = fminf(fmaxf(gb, (float)a), (float)tx1);
    int b = (int)gb;
    while (b < tx1 && xa_of(b + 1) <= right) ++b;
    while (b > a && !(xa_of(b) <= right)) --b;
    // [left, right] may fall short of tile a's span (left of its first pixel
    // centre, or in the gap between two tiles' pixel centres): no tile then
    if (!(xa_of(b) <= right)) return 0;
    *first = a;
    *last = b;
    return b - a + 1;
}

// Kept run [first, last] of tile row ty within [tx0, tx1]; returns its length.
__device__ __forceinline__ int km_row_run(const KmEllipse& e, float u, float v, int tx0, int tx1,
                                          int ty, int tile_w, int tile_h, int* first, int* last) {
    if (!(e.detc > 0.0f)) { *first = tx0; *last = tx1; return tx1 - tx0 + 1; }
    const float by = (float)(ty * tile_h);
    const float ya = ksub(kadd(by, 0.5f), v);
    const float yb = ksub(kadd(by, (float)tile_h - 0.5f), v);
    float left, right;
    if (!km_row_extent(e, ya, yb, &left, &right)) return 0;
    int a = tx0;
    while (a <= tx1) {
        const float xb = ksub(kadd((float)(a * tile_w), (float)tile_w - 0.5f), u);
        if (xb >= left) break;
        ++a;
    }
    if (a > tx1) return 0;
    int b = tx1;
    while (b > a) {
        const float xa = ksub(kadd((float)(b * tile_w), 0.5f), u);
        if (xa <= right) break;
        --b;
    }
    if (!(ksub(kadd((float)(a * tile_w), 0.5f), u) <= right)) return 0;
    *first = a;
    *last = b;
    return b - a + 1;
}

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter-based, so any
// (seed, step, slot) draw is reproducible without state.
// ---------------------------------------------------------------------------
struct U64x4 { unsigned long long v[4]; };

__device__ __forceinline__ U64x4 philox4x64_10(unsigned long long c0, unsigned long long c1,
                                               unsigned long long c2, unsigned long long c3,
                                               unsigned long long k0, unsigned long long k1) {
    const unsigned long long M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        unsigned long long hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        unsigned long long hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        unsigned long long n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    U64x4 r;
    r.v[0] = c0; r.v[1] = c1; r.v[2] = c2; r.v[3] = c3;
    return r;
}

constexpr unsigned long long kTagNoise = 0x53474c44ULL;  // "SGLD"
constexpr unsigned long long kTagReloc = 0x52454c4fULL;  // "RELO"

// Dead: sigmoid(logit) <= 0.005, decided on the FP32 logit against the largest
// float not above ln(0.005 / 0.995).
constexpr float kLogitDead = -0x1.52c582p+2f;

// Element count of a launch sized by a host capacity `cap`: with deferred
// sizing the true count lives on the device (n, written by an earlier launch)
// and is capped by the capacity; without it (n null) the capacity is exact.
__device__ __forceinline__ long long dev_count(long long cap, const unsigned long long* n) {
    if (!n) return cap;
    const long long v = (long long)*n;
    return v < cap ? v : cap;
}

// 8-bit display value of a colour channel: round(255 clamp(c, 0, 1)), ties to even.
__device__ __forceinline__ uint8_t rgb8_of(float c) {
    return (uint8_t)__float2int_rn(__fmul_rn(fminf(fmaxf(c, 0.f), 1.f), 255.f));
}

// ---------------------------------------------------------------------------
// Compositing of one (pixel, Gaussian) pair. The forward and the backward
// blend call this same function; every operation is an explicit intrinsic so
// both recompute identical alphas (the backward relies on it to retrace the
// forward's decisions).
//   staged: (u, v, qa, qb) and (qc, lo): qa = -A/2 log2e, qb = -B log2e,
//   qc = -C/2 log2e, lo = log2(opacity).
// pair_v returns v = q + lo, q = -m/2 log2e, as (qc dy + qb dx) dy + k with
// k = qa dx dx + lo (lo added inside the FMA of the dx term); pair_alpha
// gives min(0.99, 2^v) and the unclamped *au = o G = 2^v.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float pair_v(float px, float py, float4 g0, float qc, float lo,
                                        float* dx, float* dy) {
    float ddx = __fsub_rn(px, g0.x);
    float ddy = __fsub_rn(py, g0.y);
    // q + lo = (qc dy + qb dx) dy + (qa dx dx + lo): the dx terms are common
    // to every pixel of a column
    const float k = __fmaf_rn(__fmul_rn(g0.z, ddx), ddx, lo);
    const float bdx = __fmul_rn(g0.w, ddx);
    *dx = ddx;
    *dy = ddy;
    return __fmaf_rn(__fmaf_rn(qc, ddy, bdx), ddy, k);
}

// Per-Gaussian lower bound on v = q + lo for a pair to count: m <= 9 and
// alpha >= 1/255 (alpha = min(0.99, 2^v) with lo = log2(o)). Both blends test
// v against it, so their decisions agree exactly.
__device__ __forceinline__ float pair_vmin(float lo) {
    return fmaxf(__fadd_rn(kQMin, lo), kLog2AlphaMin);
}

__device__ __forceinline__ float pair_alpha(float v, float* au) {
    float u = ex2_approx(v);
    *au = u;
    return fminf(kAlphaMax, u);
}

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_view_by_tile(const ViewDev* views, int n_views, int tile) {
    int lo = 0, hi = n_views - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (views[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_view_by_record(const ViewDev* views, int n_views, int rec) {
    int lo = 0, hi = n_views - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (views[mid].rec_base <= rec) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b),
                 "f"(c), "f"(d)
                 : "memory");
}

__device__ __forceinline__ void red_add(float* addr, float a) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(addr), "f"(a) : "memory");
}

inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

// Kernel launches issued by the library (reported by the benchmark).
extern std::atomic<long long> g_kernel_launches;
inline void note_launch(int n = 1) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// Host-side launchers (one translation unit each).
// ---------------------------------------------------------------------------
struct DeviceLimits {
    int num_sms;
};

// k_compact.cu
cudaError_t launch_active_flags_count(const int32_t* start, const int32_t* expire, long long n,
                                      const int32_t* frames, int n_frames, uint32_t* block_counts,
                                      int n_blocks, cudaStream_t s);
cudaError_t launch_active_write(const int32_t* start, const int32_t* expire, long long n,
                                const int32_t* frames, int n_frames, const uint32_t* block_offsets,
                                int n_blocks, int32_t* out_ids, long long ids_stride,
                                int32_t* out_counts, cudaStream_t s);
constexpr int kCompactBlock = 1024;

// k_scan.cu
size_t scan_u32_temp_bytes(long long n);
// n_dev (optional): the true count on the device, at most n (deferred sizing)
cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, long long n, void* temp,
                               unsigned long long* total, cudaStream_t s,
                               const unsigned long long* n_dev = nullptr);
size_t scan_u64_temp_bytes(long long n);
cudaError_t inclusive_scan_u64(const unsigned long long* in, unsigned long long* out, long long n,
                               void* temp, cudaStream_t s);

// k_preprocess.cu
cudaError_t launch_preprocess(const swgs_gaussians& g, const ViewDev* views, const GroupDev* groups,
                              int n_groups, const int32_t* ids, long long total_active,
                              long long n_rec, int tile_w, int tile_h, float near_plane,
                              Records rec, cudaStream_t s,
                              const unsigned long long* n_dev = nullptr);
cudaError_t launch_preprocess_bwd(const swgs_gaussians& g, const swgs_gaussians& grads,
                                  const ViewDev* views, const GroupDev* groups, int n_groups,
                                  const int32_t* ids, long long total_active,
                                  const float* grad2d, bool reg, float* loss, cudaStream_t s,
                                  const unsigned long long* n_dev = nullptr);

// k_sort.cu
struct SortPlan {
    int passes;
    int bits_per_pass[8];
    int begin_bit;
};
SortPlan make_sort_plan(int begin_bit, int end_bit);
size_t radix_temp_bytes(long long n, int num_sms);
// Stable LSD sort of (key, value) pairs. Results end in keys_b/vals_b after an
// odd number of passes, else in keys_a/vals_a; *in_b receives which.
// vals_iota: the values start as 0..n-1 (vals_a is not read).
// One digit pass whose look-back wait runs out by construction (the failure
// path check); scratch of sort_timeout_scratch_bytes().
size_t sort_timeout_scratch_bytes();
cudaError_t launch_sort_timeout_check(void* scratch, uint32_t* err, cudaStream_t s);
// err: a device word set to 1 if a look-back wait of the single-pass form ran
// out (the output is then wrong); null keeps no record.
// single_pass: one kernel per digit pass (inputs below 2^30 keys); false, or
// larger inputs: three kernels per pass. The sorted order is the same.
cudaError_t radix_sort_pairs(uint32_t* keys_a, uint32_t* vals_a, uint32_t* keys_b,
                             uint32_t* vals_b, long long n, const SortPlan& plan, void* temp,
                             int num_sms, bool vals_iota, bool* in_b, bool single_pass,
                             uint32_t* err, cudaStream_t s,
                             const unsigned long long* n_dev = nullptr);

// k_keys.cu
// Super tiles: SX x SY tiles (4 x 4, or 2 x 8 for 32x8 tiles); at most 2^16 per
// batch (their ids share a 32-bit key with a 16-bit tile coverage mask).
constexpr long long kMaxSupersPerBatch = 1 << 16;
inline int super_w(int tile_w) { return tile_w == 32 ? 2 : 4; }
inline int super_h(int tile_w) { return tile_w == 32 ? 8 : 4; }
cudaError_t launch_gather_supers(const uint32_t* order, const Records rec, int sx, int sy,
                                 uint32_t* out, unsigned long long* exact, long long n,
                                 int num_sms, cudaStream_t s,
                                 const unsigned long long* n_dev = nullptr);
cudaError_t launch_emit_supers(const uint32_t* order, const uint32_t* offsets, long long n_rec,
                               const Records rec, const ViewDev* views, int n_views, int sx,
                               int sy, int tile_w, int tile_h, int num_sms, uint32_t* keys,
                               uint32_t* vals, cudaStream_t s,
                               const unsigned long long* n_dev = nullptr);
cudaError_t launch_super_ranges(const uint32_t* keys, long long n, long long n_supers,
                                int2* ranges, cudaStream_t s,
                                const unsigned long long* n_dev = nullptr);
// warps per block of the expansion for a grid of `blocks` blocks
int expand_warps(int blocks, int num_sms);
// Blocks per super tile of a view with view_supers super tiles when the
// expansion splits (see expand_plan): about four blocks per SM for that view
// alone, at most 16.
__host__ __device__ __forceinline__ int expand_view_parts(int view_supers, int num_sms) {
    const int target = 4 * num_sms;
    if (view_supers <= 0 || view_supers >= target) return 1;
    const int p = (target + view_supers - 1) / view_supers;
    return p < 16 ? p : 16;
}
// The expansion's launch: split (a batch of fewer than 16 super tiles per SM,
// or of fewer than 48 whose super tiles average at least 2048 keys, cuts each
// view's super tiles into expand_view_parts parts), its blocks, and
// the entries of its per-(tile, part) counts and offsets (the tiles when not
// split), over which the exclusive scan runs.
struct ExpandPlan {
    bool split;
    long long blocks, slots;
};
// A split view with S super tiles has at most S x 16 tiles in at most
// ceil(4 SMs / S) <= 4 SMs / S + 1 parts: at most 64 SMs + 16 S slots, and a
// split batch (fewer than 48 x SMs super tiles over at most 64 views) fewer
// than 64 x 64 SMs + 16 x 48 SMs. The counts and offsets are always sized to
// this bound, so that no split batch grows them (a serving loop sized by its
// largest batch then allocates nothing more).
inline long long expand_slots_bound(int num_sms) { return (64LL * 64 + 16 * 48) * num_sms; }
ExpandPlan expand_plan(const ViewDev* views, int n_views, long long total_supers,
                       long long total_tiles, long long super_keys, int num_sms);
// loads every instantiation of the expansion on the current device
cudaError_t load_expand_kernels();
cudaError_t launch_expand_count(const int2* sranges, const uint32_t* skeys, const ViewDev* views,
                                int n_views, const ExpandPlan& xp, int tile_w, int num_sms,
                                uint32_t* tcount, const uint32_t* sort_err, cudaStream_t s);
cudaError_t launch_expand_write(const int2* sranges, const uint32_t* skeys, const uint32_t* svals,
                                const ViewDev* views, int n_views, const ExpandPlan& xp,
                                int tile_w, int num_sms, const uint32_t* toff, uint32_t* vals,
                                long long cap, int2* ranges, const uint32_t* sort_err,
                                cudaStream_t s);

// k_mature.cu (Alg. 1 mature, schedule_expire)
cudaError_t launch_mature_ids(const int32_t* start, long long n, int st, uint32_t* block_counts,
                              void* scan_tmp, unsigned long long* total, int32_t* ids,
                              cudaStream_t s);
cudaError_t launch_mature_move(const swgs_gaussians& buf, const int32_t* ids, long long n,
                               long long num_gs, long long head, int swin_size,
                               void* const snap[9], cudaStream_t s);
cudaError_t launch_schedule_expire(int32_t* expire, long long num_gs, int swin_size,
                                   cudaStream_t s);

// k_codec.cu (Table 6 codec, Sec. 5.5 tail drop)
constexpr size_t kCodecHeaderBytes = 32;
constexpr uint32_t kCodecMagic = 0x43574753u;  // "SGWC" little-endian
constexpr int32_t kCodecVersion = 1;
struct CodecLayout {
    size_t index, means, log_scales, quats, opacity, dc, total;  // byte offsets
};
void codec_layout(long long count, long long keep, CodecLayout* L);
struct CodecScratch {
    uint32_t *keys_a, *keys_b, *vals_a, *vals_b, *block_cnt, *idx;
    uint8_t* flags;
    void *sort_tmp, *scan_tmp;
    unsigned long long* total;
    uint32_t* sort_err;  // the sort's look-back error word (may be null)
    bool sort_single_pass;
};
cudaError_t launch_codec_select(const float* logits, long long count, long long keep,
                                CodecScratch& w, int num_sms, uint32_t** out_idx, cudaStream_t s);
cudaError_t launch_codec_encode(const swgs_gaussians& src, const uint32_t* idx, long long count,
                                long long keep, const CodecLayout& L, unsigned char* out,
                                cudaStream_t s);
cudaError_t launch_codec_decode(const swgs_gaussians& dst, long long first, long long count,
                                long long keep, const CodecLayout& L, const unsigned char* in,
                                int32_t birth, int32_t start, int32_t expire, cudaStream_t s);

// k_blend.cu
struct BlendArgs {
    const ViewDev* views;
    int n_views;
    int total_tiles;
    const int2* ranges;
    const uint32_t* vals;
    Records rec;
    float* T;          // per pixel (batch-local)
    int32_t* last;     // per pixel
    int* work_counter;
    unsigned long long* pairs;  // optional
    float* grad2d;     // backward: 12 floats per record
    float* loss;       // fused L1 forward: accumulated loss (device float)
};
cudaError_t launch_blend_fwd(const BlendArgs& a, int tile_w, int tile_h, int batch, int ppt,
                             int grid, cudaStream_t s);
cudaError_t launch_blend_bwd(const BlendArgs& a, int tile_w, int tile_h, int batch, int ppt,
                             int grid, cudaStream_t s);
int blend_blocks_per_sm(int tile_w, int tile_h, int batch, int ppt, bool backward);
bool blend_config_valid(int tile_w, int tile_h, int batch, int ppt, bool backward);

// k_misc.cu
cudaError_t launch_loss_l1(const ViewDev* views, int n_views, long long total_pix,
                           const long long* pix_offsets, const float* const* rgb,
                           const float* const* target, float* const* dl, float* loss,
                           cudaStream_t s);
cudaError_t launch_copy_slice(const swgs_gaussians& dst, long long first, long long count,
                              const swgs_gaussians& src, cudaStream_t s);
// The count-dependent fields of a batch's tables from the active counts on the
// device (n_active, act_base, rec_base per frame group, rec_base / n_rec per
// view, the regulariser weights); with `totals`, also the record and active
// totals, checked against rec_cap and act_cap (over: status bit 0 and the
// counts zeroed, so every later launch of the batch does nothing).
cudaError_t launch_plan(GroupDev* groups, int n_groups, ViewDev* views, const int32_t* counts,
                        unsigned long long* totals, long long rec_cap, long long act_cap,
                        cudaStream_t s);
// Copies the key totals (super keys, tile-list entries; none when key_totals
// is null) into the batch totals and checks them against the capacities (over:
// status bit 1, counts zeroed); takes the sort's look-back error word into
// status bit 2 and clears it; ORs the status into *gate (the context's word
// that its later optimiser steps test).
cudaError_t launch_check_keys(const unsigned long long* key_totals, unsigned long long* totals,
                              long long super_cap, long long key_cap, uint32_t* sort_err,
                              uint32_t* gate, cudaStream_t s);

// k_optim.cu
// elig: one byte per slot, 1 = active at a frame of the step and not frozen
cudaError_t launch_eligible(const swgs_gaussians& g, const int32_t* frames, int n_frames,
                            uint8_t* elig, cudaStream_t s);
// data-parallel exchange: eligible slots' gradient rows packed [count, 11 + 3K]
cudaError_t launch_grad_pack(const swgs_gaussians& g, const swgs_gaussians& grads,
                             const int32_t* frames, int n_frames, float scale, uint8_t* elig,
                             uint32_t* block_cnt, void* scan_tmp, int32_t* ids, long long* count,
                             float* packed, cudaStream_t s);
cudaError_t launch_grad_unpack(const swgs_gaussians& grads, const int32_t* ids,
                               const long long* count, long long capacity, const float* packed,
                               cudaStream_t s);
cudaError_t launch_sgld(const swgs_gaussians& g, const swgs_gaussians* grads,
                        const swgs_adam_state* adam, const uint8_t* elig,
                        const swgs_sgld_params& p, unsigned long long seed,
                        unsigned long long step, cudaStream_t s,
                        const uint32_t* gate = nullptr);
cudaError_t launch_reloc_weights(const swgs_gaussians& g, const uint8_t* elig,
                                 unsigned long long* weights, uint8_t* dead, cudaStream_t s,
                                 const uint32_t* gate = nullptr);
cudaError_t launch_reloc_sample(const swgs_gaussians& g, const uint8_t* dead,
                                const unsigned long long* cdf, unsigned long long seed,
                                unsigned long long step, int32_t* targets, int32_t* counts,
                                unsigned long long* n_dead, cudaStream_t s);
// lr, nl: capacity-sized scratch (per target: log of the scale ratio, new logit)
cudaError_t launch_reloc_apply(const swgs_gaussians& g, const swgs_adam_state* adam,
                               const int32_t* targets, const int32_t* counts, int max_n,
                               double* lr, float* nl, cudaStream_t s);

}  // namespace swgs
