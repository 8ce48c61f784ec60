// swgs_api.cu -- the C ABI of libswgs: context and memory management, and
// the orchestration of each call on the caller's stream.
//
// Render pipeline of one batch of views (every stage one launch over all the
// batch's views):
//   1. compaction of the active set of each distinct frame (Sec. 4.2)
//   2. [sync: active counts]  projection + SH into one record per
//      (view, active Gaussian)
//   3. depth sort of the records, scan of their tile counts in depth order
//   4. [sync: key count]  emission of (tile, record) keys, stable sort by tile,
//      per-tile ranges
//   5. persistent blend over all (view, tile) work items (Eq. 3)
// The backward reuses the saved records, sorted lists, final T and last
// contributor: reverse blend, then projection backward into the caller's
// gradient buffers.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "swgs_internal.cuh"

using namespace swgs;

namespace swgs {
std::atomic<long long> g_kernel_launches{0};
}

namespace {

struct ProfEvent {
    int stage;
    cudaEvent_t a, b;
};

struct Buf {
    void* p = nullptr;
    size_t cap = 0;
};

struct BatchState {
    int n_views = 0, n_groups = 0;
    long long total_active = 0, n_rec = 0, n_keys = 0, n_tiles = 0, n_pix = 0;
    long long n_sort_keys = 0, n_supers = 0;
    std::vector<ViewDev> h_views;   // table order (grouped by frame)
    std::vector<GroupDev> h_groups;
    std::vector<int> call_index;    // table entry -> index in the call's view list
    Buf views, groups, ids, rec_a, rec_b, rec_c, rec_tiles, rec_rect, rec_depth, rec_runs, vals,
        ranges, T, last, grad2d, rec_supers;
    bool has_grad2d = false;
    // deferred sizing: the counts live on the device (counts_b: active per
    // frame group; dtot: BatchTotal words); a pinned slot receives them with
    // the batch, and `ev` marks its arrival
    Buf counts_b, dtot;
    void* h_slot = nullptr;       // pinned: kTotWords u64, then the group counts
    cudaEvent_t ev = nullptr;
    bool deferred = false, resolved = true;
    long long rec_cap = 0, act_cap = 0;
    swgs_status status = SWGS_OK;
};

constexpr size_t kSlotBytes = sizeof(unsigned long long) * kTotWords + 4 * kMaxViewsPerBatch;

}  // namespace

struct swgs_saved {
    swgs_ctx* ctx = nullptr;
    std::vector<BatchState> batches;
    int n_batches = 0;
    int n_views = 0;
    Buf pairs;  // unsigned long long
    bool count_pairs = false;
};

struct swgs_ctx {
    swgs_config cfg{};
    swgs_alloc_fn alloc = nullptr;
    swgs_free_fn free_fn = nullptr;
    void* user = nullptr;
    int device = 0;
    int num_sms = 148;
    std::string err;
    cudaStream_t last_stream = nullptr;
    // transient scratch
    Buf frames, block_cnt, scan_tmp, counts, order_a, order_b, tcount, koff, keys_a, keys_b,
        vals_tmp, vals_b, sranges, tile_cnt, tile_off, mature_ids, mature_stage, codec_keys_a,
        codec_keys_b, codec_vals_a, codec_vals_b, codec_flags, codec_idx, codec_stage, sort_tmp,
        counter, totals, l1_tab, elig, reloc_w, reloc_cdf, reloc_dead, reloc_tg, reloc_cnt,
        reloc_nd, reloc_lr, reloc_nl, sort_err;
    void* pinned = nullptr;
    size_t pinned_cap = 0;
    // deferred sizing: capacities learned from earlier calls, and the word the
    // forward raises when a batch outgrew them (the optimiser step tests it)
    long long cap_rec = 0, cap_sk = 0, cap_keys = 0, cap_act = 0;
    Buf gate;
    std::vector<swgs_saved*> pool;
    std::vector<swgs_saved*> all_saved;
    // stage profiling
    bool prof = false;
    std::vector<ProfEvent> prof_pending;
    std::vector<cudaEvent_t> prof_free;
    double prof_ms[SWGS_NUM_STAGES] = {};
    long long prof_calls[SWGS_NUM_STAGES] = {};
};

namespace {

swgs_status fail(swgs_ctx* c, swgs_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return st;
}

#define CK(expr)                                                                      \
    do {                                                                              \
        cudaError_t _e = (expr);                                                      \
        if (_e != cudaSuccess)                                                        \
            return fail(ctx, SWGS_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(_e)); \
    } while (0)

cudaEvent_t prof_event(swgs_ctx* c) {
    if (!c->prof_free.empty()) {
        cudaEvent_t e = c->prof_free.back();
        c->prof_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Records a pair of events around one stage on the caller's stream.
struct StageScope {
    swgs_ctx* c;
    int stage;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    StageScope(swgs_ctx* c_, int st, cudaStream_t s_) : c(c_), stage(st), s(s_) {
        if (c->prof) {
            a = prof_event(c);
            cudaEventRecord(a, s);
        }
    }
    ~StageScope() {
        if (c->prof && a) {
            cudaEvent_t b = prof_event(c);
            cudaEventRecord(b, s);
            c->prof_pending.push_back({stage, a, b});
        }
    }
};

void* ctx_alloc(swgs_ctx* c, size_t bytes, cudaStream_t s) {
    if (c->alloc) {
        void* p = c->alloc(c->user, bytes, (void*)s);
        // the kernels read scratch with 16-byte vector loads
        if (p && (reinterpret_cast<uintptr_t>(p) & 255u) != 0) {
            if (c->free_fn) c->free_fn(c->user, p, bytes, (void*)s);
            return nullptr;
        }
        return p;
    }
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) return nullptr;
    return p;
}

void ctx_free(swgs_ctx* c, Buf& b, cudaStream_t s) {
    if (b.p) {
        if (c->free_fn) c->free_fn(c->user, b.p, b.cap, (void*)s);
        else cudaFreeAsync(b.p, s);
    }
    b.p = nullptr;
    b.cap = 0;
}

bool ensure(swgs_ctx* c, Buf& b, size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) return true;
    ctx_free(c, b, s);
    size_t nb = bytes + bytes / 4 + 256;
    b.p = ctx_alloc(c, nb, s);
    if (!b.p) return false;
    b.cap = nb;
    return true;
}

template <typename T>
T* P(Buf& b) { return reinterpret_cast<T*>(b.p); }

// The sorts' look-back error word, zeroed when first allocated; read back with
// the key totals (null if it cannot be allocated: the sort then keeps none).
uint32_t* sort_err_word(swgs_ctx* c, cudaStream_t s) {
    if (!c->sort_err.p) {
        if (!ensure(c, c->sort_err, 16, s)) return nullptr;
        if (cudaMemsetAsync(c->sort_err.p, 0, 16, s) != cudaSuccess) return nullptr;
    }
    return P<uint32_t>(c->sort_err);
}

// The context's gate word: raised by a forward whose batch outgrew the deferred
// capacities, so that the optimiser steps after it do nothing (zeroed at the
// start of each deferred forward call).
uint32_t* gate_word(swgs_ctx* c, cudaStream_t s) {
    if (!c->gate.p) {
        if (!ensure(c, c->gate, 16, s)) return nullptr;
        if (cudaMemsetAsync(c->gate.p, 0, 16, s) != cudaSuccess) return nullptr;
    }
    return P<uint32_t>(c->gate);
}

bool valid_tile(int w, int h) { return (w == 16 && h == 16) || (w == 8 && h == 8) || (w == 32 && h == 8); }
bool valid_batch(int b) { return b == 32 || b == 64 || b == 128 || b == 256; }

swgs_status check_gaussians(swgs_ctx* ctx, const swgs_gaussians* g, bool need_life) {
    if (!g) return fail(ctx, SWGS_EINVAL, "null Gaussian state");
    if (g->capacity < 0 || g->capacity > 0x7fffffffLL)
        return fail(ctx, SWGS_EINVAL, "capacity %lld out of range", (long long)g->capacity);
    if (g->sh_degree < 0 || g->sh_degree > 3)
        return fail(ctx, SWGS_EINVAL, "sh_degree %d not in 0..3", g->sh_degree);
    if (g->capacity > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh))
        return fail(ctx, SWGS_EINVAL, "null attribute array");
    if (g->capacity > 0 && ((uintptr_t)g->quats & 15))
        return fail(ctx, SWGS_EINVAL, "quats must be 16-byte aligned");
    if (need_life && g->capacity > 0 && (!g->start || !g->expire))
        return fail(ctx, SWGS_EINVAL, "null lifespan array");
    return SWGS_OK;
}

swgs_status resolve_batch(swgs_ctx* c, BatchState& B, bool wait);

swgs_saved* acquire_saved(swgs_ctx* c) {
    swgs_saved* s;
    if (!c->pool.empty()) {
        s = c->pool.back();
        c->pool.pop_back();
    } else {
        s = new swgs_saved();
        s->ctx = c;
        c->all_saved.push_back(s);
    }
    for (auto& b : s->batches) resolve_batch(c, b, true);  // long finished by now
    s->n_batches = 0;
    s->n_views = 0;
    return s;
}

void free_saved_buffers(swgs_ctx* c, swgs_saved* s, cudaStream_t st) {
    for (auto& b : s->batches) {
        Buf* bs[] = {&b.views, &b.groups, &b.ids, &b.rec_a, &b.rec_b, &b.rec_c, &b.rec_tiles,
                     &b.rec_rect, &b.rec_depth, &b.rec_runs, &b.vals, &b.ranges, &b.T, &b.last,
                     &b.grad2d, &b.rec_supers, &b.counts_b, &b.dtot};
        for (Buf* x : bs) ctx_free(c, *x, st);
        if (b.h_slot) cudaFreeHost(b.h_slot);
        if (b.ev) cudaEventDestroy(b.ev);
        b.h_slot = nullptr;
        b.ev = nullptr;
    }
    ctx_free(c, s->pairs, st);
}

long long grow_cap(long long x) { return x + x / 8 + 4096; }

// The host tables' count-dependent fields from the active counts, as the
// plan kernel computes them on the device.
void tables_from_counts(BatchState& B, const int32_t* counts) {
    long long act = 0, rec = 0;
    for (size_t k = 0; k < B.h_groups.size(); ++k) {
        GroupDev& G = B.h_groups[k];
        const int n = counts[k];
        G.n_active = n;
        G.act_base = (int)act;
        G.rec_base = (int)rec;
        for (int j = 0; j < G.view_count; ++j) {
            ViewDev& V = B.h_views[(size_t)G.view_begin + j];
            V.rec_base = (int)(rec + (long long)j * n);
            V.n_rec = n;
        }
        act += n;
        rec += (long long)n * G.view_count;
    }
}

// Deferred sizing: take a finished batch's totals from its pinned slot (wait:
// block until they have arrived; else SWGS_EPENDING if they have not), fill
// its host counts and tables, grow the context's capacities to what it needed,
// and return its status: SWGS_EDEVICE when it outgrew the capacities (its
// outputs are background and every later launch of it did nothing: render it
// again), SWGS_ETIMEOUT when a sort's look-back wait ran out.
swgs_status resolve_batch(swgs_ctx* c, BatchState& B, bool wait) {
    if (!B.deferred || B.resolved) return B.status;
    const cudaError_t e = wait ? cudaEventSynchronize(B.ev) : cudaEventQuery(B.ev);
    if (e == cudaErrorNotReady) return SWGS_EPENDING;
    if (e != cudaSuccess) return fail(c, SWGS_ECUDA, "deferred totals: %s", cudaGetErrorString(e));
    unsigned long long tot[kTotWords];
    memcpy(tot, B.h_slot, sizeof(tot));
    tables_from_counts(B, (const int32_t*)((const char*)B.h_slot + sizeof(tot)));
    B.n_rec = (long long)tot[kTotRecords];
    B.total_active = (long long)tot[kTotActive];
    B.n_sort_keys = (long long)tot[kTotSuperKeys];
    B.n_keys = (long long)tot[kTotTileKeys];
    const unsigned long long st = tot[kTotStatus];
    c->cap_rec = std::max(c->cap_rec, grow_cap((long long)tot[kTotNeedRecords]));
    c->cap_act = std::max(c->cap_act, grow_cap((long long)tot[kTotNeedActive]));
    c->cap_sk = std::max(c->cap_sk, grow_cap((long long)tot[kTotNeedSuperKeys]));
    c->cap_keys = std::max(c->cap_keys, grow_cap((long long)tot[kTotNeedTileKeys]));
    if ((st & 1ull) && B.rec_cap > 0) {
        // the records did not fit, so the keys were never counted: grow their
        // capacities in proportion, so that the call issued again likely fits
        const double f = (double)tot[kTotNeedRecords] / (double)B.rec_cap;
        c->cap_sk = std::max(c->cap_sk, grow_cap((long long)(f * (double)c->cap_sk)));
        c->cap_keys = std::max(c->cap_keys, grow_cap((long long)(f * (double)c->cap_keys)));
    }
    B.status = (st & 3ull) ? SWGS_EDEVICE : ((st & 4ull) ? SWGS_ETIMEOUT : SWGS_OK);
    B.resolved = true;
    return B.status;
}

Records records_of(BatchState& b) {
    Records r;
    r.a = P<float4>(b.rec_a);
    r.b = P<float4>(b.rec_b);
    r.c = P<float4>(b.rec_c);
    r.tiles = P<int32_t>(b.rec_tiles);
    r.rect = P<short4>(b.rec_rect);
    r.depth_key = P<uint32_t>(b.rec_depth);
    r.runs = P<uint16_t>(b.rec_runs);
    r.supers = P<int32_t>(b.rec_supers);
    return r;
}

int ceil_log2(long long x) {
    int b = 0;
    while ((1LL << b) < x) ++b;
    return b;
}

// Render one batch of views (indices idx[] into the call's view list).
swgs_status render_batch(swgs_ctx* ctx, const swgs_gaussians* g, const swgs_view* views,
                         const std::vector<int>& idx, const float* bg, float* const* out_rgb,
                         uint8_t* const* out_rgb8,
                         float* const* out_T, const void* const* targets, int target_u8,
                         float* const* dls,
                         float* loss, int n_views_total, BatchState& B,
                         unsigned long long* pairs, cudaStream_t s) {
    const int tw = ctx->cfg.tile_w, th = ctx->cfg.tile_h;
    const long long N = g->capacity;
    // group the views by frame, in order of first appearance
    std::vector<int> frames;
    std::vector<std::vector<int>> members;
    for (int v : idx) {
        int f = views[v].frame;
        size_t k = 0;
        while (k < frames.size() && frames[k] != f) ++k;
        if (k == frames.size()) { frames.push_back(f); members.emplace_back(); }
        members[k].push_back(v);
    }
    const int F = (int)frames.size();
    B.n_views = (int)idx.size();
    B.n_groups = F;
    B.has_grad2d = false;
    // deferred sizing: once capacities are known, nothing is read back here;
    // the counts stay on the device and size every launch from there
    const bool deferred = ctx->cfg.deferred_sizing != 0 && ctx->cap_rec > 0 &&
                          ctx->cfg.sort_single_pass != 0 && ctx->cap_rec < (1LL << 30) &&
                          ctx->cap_sk < (1LL << 30);
    B.deferred = deferred;
    B.resolved = !deferred;
    B.status = SWGS_OK;
    // 1. compaction
    const int nb = N > 0 ? (int)((N + kCompactBlock - 1) / kCompactBlock) : 0;
    if (!ensure(ctx, ctx->frames, sizeof(int32_t) * F, s) ||
        !ensure(ctx, ctx->block_cnt, sizeof(uint32_t) * ((size_t)F * nb + 1), s) ||
        !ensure(ctx, ctx->scan_tmp, scan_u32_temp_bytes((long long)F * nb + 1) + 64, s) ||
        !ensure(ctx, B.counts_b, sizeof(int32_t) * F, s) || !ensure(ctx, ctx->totals, 64, s) ||
        !ensure(ctx, B.dtot, sizeof(unsigned long long) * kTotWords, s) ||
        !ensure(ctx, B.ids, sizeof(int32_t) * ((size_t)F * (N > 0 ? N : 1)), s))
        return fail(ctx, SWGS_ENOMEM, "allocation failed (compaction)");
    if (deferred && !B.h_slot) {
        if (cudaMallocHost(&B.h_slot, kSlotBytes) != cudaSuccess ||
            cudaEventCreateWithFlags(&B.ev, cudaEventDisableTiming) != cudaSuccess)
            return fail(ctx, SWGS_ENOMEM, "allocation failed (deferred totals)");
    }
    CK(cudaMemsetAsync(B.dtot.p, 0, sizeof(unsigned long long) * kTotWords, s));
    // the active ids over the groups: at most F N (their buffer's size); the
    // launches over them are sized by the learned capacity when deferred
    B.act_cap = (long long)F * (N > 0 ? N : 1);
    if (deferred) B.act_cap = std::min(B.act_cap, ctx->cap_act);
    CK(cudaMemcpyAsync(ctx->frames.p, frames.data(), sizeof(int32_t) * F, cudaMemcpyHostToDevice, s));
    std::vector<int> n_act(F, 0);
    if (N > 0) {
        StageScope sc_(ctx, SWGS_STAGE_COMPACT, s);
        CK(launch_active_flags_count(g->start, g->expire, N, P<int32_t>(ctx->frames), F,
                                     P<uint32_t>(ctx->block_cnt), nb, s));
        CK(exclusive_scan_u32(P<uint32_t>(ctx->block_cnt), P<uint32_t>(ctx->block_cnt),
                              (long long)F * nb, ctx->scan_tmp.p, P<unsigned long long>(ctx->totals), s));
        CK(launch_active_write(g->start, g->expire, N, P<int32_t>(ctx->frames), F,
                               P<uint32_t>(ctx->block_cnt), nb, P<int32_t>(B.ids), 0,
                               P<int32_t>(B.counts_b), s));
    } else {
        CK(cudaMemsetAsync(B.counts_b.p, 0, sizeof(int32_t) * F, s));
    }
    if (N > 0 && !deferred) {
        CK(cudaMemcpyAsync(ctx->pinned, B.counts_b.p, sizeof(int32_t) * F, cudaMemcpyDeviceToHost,
                           s));
        CK(cudaStreamSynchronize(s));
        memcpy(n_act.data(), ctx->pinned, sizeof(int32_t) * F);
    }
    // 2. tables
    B.h_groups.assign(F, GroupDev{});
    B.h_views.clear();
    B.call_index.clear();
    const int SX = super_w(tw), SY = super_h(tw);
    long long act = 0, rec = 0, tiles = 0, supers = 0, pix = 0;
    for (int k = 0; k < F; ++k) {
        GroupDev& G = B.h_groups[k];
        G.frame = frames[k];
        G.n_active = n_act[k];
        G.act_base = (int)act;
        G.rec_base = (int)rec;
        G.view_begin = (int)B.h_views.size();
        G.view_count = (int)members[k].size();
        for (size_t j = 0; j < members[k].size(); ++j) {
            const int v = members[k][j];
            const swgs_view& sv = views[v];
            ViewDev V{};
            V.W = sv.width;
            V.H = sv.height;
            V.ntx = (sv.width + tw - 1) / tw;
            V.nty = (sv.height + th - 1) / th;
            V.tile_base = (int)tiles;
            V.nsx = (V.ntx + SX - 1) / SX;
            V.nsy = (V.nty + SY - 1) / SY;
            V.super_base = (int)supers;
            V.rec_base = (int)(rec + (long long)j * n_act[k]);
            V.n_rec = n_act[k];
            V.group = k;
            V.pix_base = pix;
            V.fx = sv.fx; V.fy = sv.fy; V.cx = sv.cx; V.cy = sv.cy;
            for (int e = 0; e < 9; ++e) V.R[e] = sv.R[e];
            for (int e = 0; e < 3; ++e) V.t[e] = sv.t[e];
            for (int e = 0; e < 3; ++e) {
                double c = 0.0;
                for (int r = 0; r < 3; ++r) c -= (double)sv.R[3 * r + e] * (double)sv.t[r];
                V.campos[e] = (float)c;
            }
            for (int e = 0; e < 3; ++e) V.bg[e] = bg ? bg[e] : 0.f;
            V.out_rgb = out_rgb ? out_rgb[v] : nullptr;
            V.out_rgb8 = out_rgb8 ? out_rgb8[v] : nullptr;
            V.out_T = out_T ? out_T[v] : nullptr;
            V.dL = nullptr;
            V.target = (targets && !target_u8) ? (const float*)targets[v] : nullptr;
            V.target_u8 = (targets && target_u8) ? (const uint8_t*)targets[v] : nullptr;
            V.dL_out = dls ? dls[v] : nullptr;
            V.l1_scale = 1.0f / (3.0f * (float)sv.width * (float)sv.height * (float)n_views_total);
            tiles += (long long)V.ntx * V.nty;
            supers += (long long)V.nsx * V.nsy;
            pix += (long long)sv.width * sv.height;
            B.h_views.push_back(V);
            B.call_index.push_back(v);
        }
        act += n_act[k];
        rec += (long long)n_act[k] * members[k].size();
    }
    if (rec > 0x7fffffffLL || tiles > 0x7fffffffLL)
        return fail(ctx, SWGS_EINVAL, "too many records (%lld) or tiles (%lld) in one batch", rec, tiles);
    if (supers > kMaxSupersPerBatch)
        return fail(ctx, SWGS_EINVAL, "%lld super tiles in one batch (at most %lld)", supers,
                    kMaxSupersPerBatch);
    B.total_active = act;
    B.n_rec = rec;
    B.n_tiles = tiles;
    B.n_supers = supers;
    B.n_sort_keys = 0;
    B.n_pix = pix;
    if (deferred) rec = ctx->cap_rec;  // every record launch is sized by it
    B.rec_cap = rec;
    const size_t R = (size_t)rec;
    unsigned long long* dtot = P<unsigned long long>(B.dtot);
    const unsigned long long* n_rec_dev = deferred ? dtot + kTotRecords : nullptr;
    if (!ensure(ctx, B.views, sizeof(ViewDev) * B.h_views.size(), s) ||
        !ensure(ctx, B.groups, sizeof(GroupDev) * F, s) ||
        !ensure(ctx, B.rec_a, sizeof(float4) * R, s) || !ensure(ctx, B.rec_b, sizeof(float4) * R, s) ||
        !ensure(ctx, B.rec_c, sizeof(float4) * R, s) ||
        !ensure(ctx, B.rec_tiles, sizeof(int32_t) * R, s) ||
        !ensure(ctx, B.rec_supers, sizeof(int32_t) * R, s) ||
        !ensure(ctx, B.rec_rect, sizeof(short4) * R, s) ||
        !ensure(ctx, B.rec_depth, sizeof(uint32_t) * R, s) ||
        !ensure(ctx, B.rec_runs, sizeof(uint16_t) * kRunRows * R, s) ||
        !ensure(ctx, B.ranges, sizeof(int2) * (size_t)tiles, s) ||
        !ensure(ctx, B.T, sizeof(float) * (size_t)pix, s) ||
        !ensure(ctx, B.last, sizeof(int32_t) * (size_t)pix, s) ||
        !ensure(ctx, ctx->order_a, sizeof(uint32_t) * R, s) ||
        !ensure(ctx, ctx->order_b, sizeof(uint32_t) * R, s) ||
        !ensure(ctx, ctx->tcount, sizeof(uint32_t) * R, s) ||
        !ensure(ctx, ctx->koff, sizeof(uint32_t) * (R + 1), s) ||
        !ensure(ctx, ctx->totals, 64, s) || !ensure(ctx, ctx->counter, 64, s))
        return fail(ctx, SWGS_ENOMEM, "allocation failed (records)");
    CK(cudaMemcpyAsync(B.views.p, B.h_views.data(), sizeof(ViewDev) * B.h_views.size(),
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.groups.p, B.h_groups.data(), sizeof(GroupDev) * F, cudaMemcpyHostToDevice, s));
    if (deferred)
        CK(launch_plan(P<GroupDev>(B.groups), F, P<ViewDev>(B.views), P<int32_t>(B.counts_b), dtot,
                       ctx->cap_rec, B.act_cap, s));
    Records rc = records_of(B);
    {
        StageScope sc_(ctx, SWGS_STAGE_PREPROCESS, s);
        CK(launch_preprocess(*g, P<ViewDev>(B.views), P<GroupDev>(B.groups), F, P<int32_t>(B.ids),
                             act, rec, tw, th, ctx->cfg.near_plane, rc, s, n_rec_dev));
    }
    // 3. depth order of the records and their key offsets
    long long n_keys = 0;
    if (rec > 0) {
        const SortPlan dp = make_sort_plan(0, 32);
        if (!ensure(ctx, ctx->sort_tmp, radix_temp_bytes((long long)R, ctx->num_sms), s))
            return fail(ctx, SWGS_ENOMEM, "allocation failed (sort)");
        bool in_b = false;
        {
            StageScope sc_(ctx, SWGS_STAGE_DEPTH_SORT, s);
            CK(radix_sort_pairs(P<uint32_t>(B.rec_depth), P<uint32_t>(ctx->order_a),
                                P<uint32_t>(ctx->order_b), P<uint32_t>(ctx->tcount), (long long)R,
                                dp, ctx->sort_tmp.p, ctx->num_sms, true, &in_b,
                                ctx->cfg.sort_single_pass != 0, sort_err_word(ctx, s), s,
                                n_rec_dev));
        }
        // 4 passes: results back in (rec_depth, order_a)
        const uint32_t* order = in_b ? P<uint32_t>(ctx->tcount) : P<uint32_t>(ctx->order_a);
        uint32_t* cnt = in_b ? P<uint32_t>(ctx->order_a) : P<uint32_t>(ctx->tcount);
        if (!ensure(ctx, ctx->scan_tmp, scan_u32_temp_bytes((long long)R) + 64, s))
            return fail(ctx, SWGS_ENOMEM, "allocation failed (scan)");
        {
            StageScope sc_(ctx, SWGS_STAGE_KEY_SCAN, s);
            CK(cudaMemsetAsync(ctx->totals.p, 0, 16, s));
            CK(launch_gather_supers(order, rc, SX, SY, cnt,
                                    P<unsigned long long>(ctx->totals) + 1, (long long)R,
                                    ctx->num_sms, s, n_rec_dev));
            CK(exclusive_scan_u32(cnt, P<uint32_t>(ctx->koff), (long long)R, ctx->scan_tmp.p,
                                  P<unsigned long long>(ctx->totals), s, n_rec_dev));
        }
        long long n_sk = 0;
        if (deferred) {
            // sized by the capacities; a batch over them stops here on the device
            n_sk = ctx->cap_sk;
            n_keys = ctx->cap_keys;
            CK(launch_check_keys(P<unsigned long long>(ctx->totals), dtot, n_sk, n_keys,
                                 sort_err_word(ctx, s), gate_word(ctx, s), s));
        } else {
            CK(cudaMemcpyAsync(ctx->pinned, ctx->totals.p, 2 * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, s));
            uint32_t* serr = sort_err_word(ctx, s);
            if (serr)
                CK(cudaMemcpyAsync((char*)ctx->pinned + 16, serr, 4, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            unsigned long long tot[2] = {0, 0};
            memcpy(tot, ctx->pinned, sizeof(tot));
            uint32_t sort_failed = 0;
            if (serr) memcpy(&sort_failed, (char*)ctx->pinned + 16, 4);
            if (sort_failed) {
                CK(cudaMemsetAsync(serr, 0, 4, s));
                return fail(ctx, SWGS_ETIMEOUT,
                            "a radix-sort look-back wait ran out (this call's depth order, or "
                            "the previous call's sorted keys, are wrong)");
            }
            if (tot[1] > 0x7fffffffULL || tot[0] > 0x7fffffffULL)
                return fail(ctx, SWGS_EINVAL,
                            "%llu tile keys (%llu super-tile keys) exceed the 2^31 limit of one "
                            "batch; render fewer views per call", tot[1], tot[0]);
            n_keys = (long long)tot[1];
            n_sk = (long long)tot[0];
            // the capacities a later deferred call starts from
            ctx->cap_rec = std::max(ctx->cap_rec, grow_cap(rec));
            ctx->cap_act = std::max(ctx->cap_act, grow_cap(act));
            ctx->cap_sk = std::max(ctx->cap_sk, grow_cap(n_sk));
            ctx->cap_keys = std::max(ctx->cap_keys, grow_cap(n_keys));
        }
        B.n_keys = n_keys;
        B.n_sort_keys = n_sk;
        const unsigned long long* n_sk_dev = deferred ? dtot + kTotSuperKeys : nullptr;
        // 4. super-tile keys, their stable sort by super tile, per-tile lists
        const SortPlan sp = make_sort_plan(0, ceil_log2(supers));
        const size_t K = (size_t)n_sk;
        // the expansion's launch; its counts and offsets hold one entry per
        // tile and part
        const ExpandPlan xp = expand_plan(B.h_views.data(), (int)B.h_views.size(), supers,
                                          tiles, (long long)K, ctx->num_sms);
        const long long tslots = xp.slots;
        const long long tslots_cap =
            tslots > expand_slots_bound(ctx->num_sms) ? tslots : expand_slots_bound(ctx->num_sms);
        if (!ensure(ctx, ctx->keys_a, sizeof(uint32_t) * K, s) ||
            !ensure(ctx, ctx->keys_b, sizeof(uint32_t) * K, s) ||
            !ensure(ctx, ctx->vals_tmp, sizeof(uint32_t) * K, s) ||
            !ensure(ctx, ctx->vals_b, sizeof(uint32_t) * K, s) ||
            !ensure(ctx, ctx->sranges, sizeof(int2) * (size_t)supers, s) ||
            !ensure(ctx, B.vals, sizeof(uint32_t) * (size_t)n_keys, s) ||
            !ensure(ctx, ctx->tile_cnt, sizeof(uint32_t) * (size_t)tslots_cap, s) ||
            !ensure(ctx, ctx->tile_off, sizeof(uint32_t) * (size_t)tslots_cap, s) ||
            !ensure(ctx, ctx->scan_tmp, scan_u32_temp_bytes(tslots_cap) + 64, s) ||
            !ensure(ctx, ctx->sort_tmp, radix_temp_bytes((long long)K, ctx->num_sms), s))
            return fail(ctx, SWGS_ENOMEM, "allocation failed (keys)");
        {
            StageScope sc_(ctx, SWGS_STAGE_EMIT, s);
            CK(launch_emit_supers(order, P<uint32_t>(ctx->koff), (long long)R, rc,
                                  P<ViewDev>(B.views), (int)B.h_views.size(), SX, SY, tw, th,
                                  ctx->num_sms, P<uint32_t>(ctx->keys_a),
                                  P<uint32_t>(ctx->vals_tmp), s, n_rec_dev));
        }
        bool kb = false;
        {
            StageScope sc_(ctx, SWGS_STAGE_TILE_SORT, s);
            CK(radix_sort_pairs(P<uint32_t>(ctx->keys_a), P<uint32_t>(ctx->vals_tmp),
                                P<uint32_t>(ctx->keys_b), P<uint32_t>(ctx->vals_b), (long long)K,
                                sp, ctx->sort_tmp.p, ctx->num_sms, false, &kb,
                                ctx->cfg.sort_single_pass != 0, sort_err_word(ctx, s), s,
                                n_sk_dev));
        }
        const uint32_t* skeys = kb ? P<uint32_t>(ctx->keys_b) : P<uint32_t>(ctx->keys_a);
        const uint32_t* svals = kb ? P<uint32_t>(ctx->vals_b) : P<uint32_t>(ctx->vals_tmp);
        {
            StageScope sc_(ctx, SWGS_STAGE_RANGES, s);
            CK(cudaMemsetAsync(ctx->sranges.p, 0, sizeof(int2) * (size_t)supers, s));
            CK(launch_super_ranges(skeys, (long long)K, supers, P<int2>(ctx->sranges), s,
                                   n_sk_dev));
            CK(launch_expand_count(P<int2>(ctx->sranges), skeys, P<ViewDev>(B.views),
                                   (int)B.h_views.size(), xp, tw, ctx->num_sms,
                                   P<uint32_t>(ctx->tile_cnt), sort_err_word(ctx, s), s));
            CK(exclusive_scan_u32(P<uint32_t>(ctx->tile_cnt), P<uint32_t>(ctx->tile_off),
                                  tslots, ctx->scan_tmp.p,
                                  P<unsigned long long>(ctx->totals) + 2, s));
            CK(launch_expand_write(P<int2>(ctx->sranges), skeys, svals, P<ViewDev>(B.views),
                                   (int)B.h_views.size(), xp, tw, ctx->num_sms,
                                   P<uint32_t>(ctx->tile_off), P<uint32_t>(B.vals), n_keys,
                                   P<int2>(B.ranges), sort_err_word(ctx, s), s));
        }
    } else {
        B.n_keys = 0;
        CK(cudaMemsetAsync(B.ranges.p, 0, sizeof(int2) * (size_t)tiles, s));
        if (!ensure(ctx, B.vals, 16, s)) return fail(ctx, SWGS_ENOMEM, "allocation failed");
    }
    // 5. blend
    BlendArgs ba{};
    ba.views = P<ViewDev>(B.views);
    ba.n_views = (int)B.h_views.size();
    ba.total_tiles = (int)tiles;
    ba.ranges = P<int2>(B.ranges);
    ba.vals = P<uint32_t>(B.vals);
    ba.rec = rc;
    ba.T = P<float>(B.T);
    ba.last = P<int32_t>(B.last);
    ba.work_counter = P<int>(ctx->counter);
    ba.pairs = pairs;
    ba.grad2d = nullptr;
    ba.loss = targets ? loss : nullptr;
    const int ppt = ctx->cfg.pixels_per_thread;
    int bps = ctx->cfg.blocks_per_sm > 0
                  ? ctx->cfg.blocks_per_sm
                  : blend_blocks_per_sm(tw, th, ctx->cfg.batch, ppt, false);
    long long grid = (long long)ctx->num_sms * bps;
    if (grid > tiles) grid = tiles;
    if (grid < 1) grid = 1;
    CK(cudaMemsetAsync(ctx->counter.p, 0, sizeof(int), s));
    {
        StageScope sc_(ctx, SWGS_STAGE_BLEND_FWD, s);
        CK(launch_blend_fwd(ba, tw, th, ctx->cfg.batch, ppt, (int)grid, s));
    }
    if (deferred) {
        // the tile sort's wait into the status, then the totals and the group
        // counts to this batch's pinned slot
        CK(launch_check_keys(nullptr, dtot, 0, 0, sort_err_word(ctx, s), gate_word(ctx, s), s));
        CK(cudaMemcpyAsync(B.h_slot, dtot, sizeof(unsigned long long) * kTotWords,
                           cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync((char*)B.h_slot + sizeof(unsigned long long) * kTotWords, B.counts_b.p,
                           sizeof(int32_t) * F, cudaMemcpyDeviceToHost, s));
        CK(cudaEventRecord(B.ev, s));
    }
    return SWGS_OK;
}

swgs_status backward_batch(swgs_ctx* ctx, const swgs_gaussians* g, BatchState& B,
                           const float* const* dL, const swgs_gaussians* grads,
                           const swgs_reg_params* reg, int n_views_total, float* loss,
                           cudaStream_t s) {
    const int tw = ctx->cfg.tile_w, th = ctx->cfg.tile_h;
    for (size_t i = 0; i < B.h_views.size(); ++i) {
        B.h_views[i].dL = dL[B.call_index[i]];
        if (!B.h_views[i].dL) return fail(ctx, SWGS_EINVAL, "null dL_drgb for view %d", B.call_index[i]);
    }
    // deferred sizing, forward not yet resolved: the counts are on the device
    // only, so sizes come from the batch's capacities and launches read the
    // device totals (a batch that outgrew them has zero counts there)
    const bool dev = B.deferred && !B.resolved;
    unsigned long long* dtot = P<unsigned long long>(B.dtot);
    const bool use_reg = reg && (reg->opacity_reg != 0.f || reg->scale_reg != 0.f);
    if (use_reg) {
        // per-frame weights of one active Gaussian in the view-mean of reg():
        // view_count / (V n_active) times each weight (the division by n_active
        // on the device when the count is only there)
        const int V = reg->n_views_total > 0 ? reg->n_views_total : n_views_total;
        for (GroupDev& G : B.h_groups) {
            G.reg_o_num = (double)reg->opacity_reg * G.view_count / (double)V;
            G.reg_s_num = (double)reg->scale_reg * G.view_count / (3.0 * V);
            G.reg_o = G.n_active > 0 ? (float)(G.reg_o_num / (double)G.n_active) : 0.f;
            G.reg_s = G.n_active > 0 ? (float)(G.reg_s_num / (double)G.n_active) : 0.f;
        }
        CK(cudaMemcpyAsync(B.groups.p, B.h_groups.data(), sizeof(GroupDev) * B.h_groups.size(),
                           cudaMemcpyHostToDevice, s));
    }
    CK(cudaMemcpyAsync(B.views.p, B.h_views.data(), sizeof(ViewDev) * B.h_views.size(),
                       cudaMemcpyHostToDevice, s));
    if (dev)  // the uploads carried no counts: restore them (and the weights) on the device
        CK(launch_plan(P<GroupDev>(B.groups), B.n_groups, P<ViewDev>(B.views),
                       P<int32_t>(B.counts_b), nullptr, 0, 0, s));
    const long long n_rec = dev ? B.rec_cap : B.n_rec;
    if (!ensure(ctx, B.grad2d, sizeof(float) * 12 * (size_t)(n_rec > 0 ? n_rec : 1), s) ||
        !ensure(ctx, ctx->counter, 64, s))
        return fail(ctx, SWGS_ENOMEM, "allocation failed (grad2d)");
    CK(cudaMemsetAsync(B.grad2d.p, 0, sizeof(float) * 12 * (size_t)(n_rec > 0 ? n_rec : 1), s));
    B.has_grad2d = true;
    if (n_rec == 0) return SWGS_OK;
    BlendArgs ba{};
    ba.views = P<ViewDev>(B.views);
    ba.n_views = (int)B.h_views.size();
    ba.total_tiles = (int)B.n_tiles;
    ba.ranges = P<int2>(B.ranges);
    ba.vals = P<uint32_t>(B.vals);
    ba.rec = records_of(B);
    ba.T = P<float>(B.T);
    ba.last = P<int32_t>(B.last);
    ba.work_counter = P<int>(ctx->counter);
    ba.pairs = nullptr;
    ba.grad2d = P<float>(B.grad2d);
    ba.loss = nullptr;
    const int ppt = ctx->cfg.bwd_pixels_per_thread;
    const int bbatch = ctx->cfg.bwd_batch;
    int bps = ctx->cfg.blocks_per_sm > 0
                  ? ctx->cfg.blocks_per_sm
                  : blend_blocks_per_sm(tw, th, bbatch, ppt, true);
    long long grid = (long long)ctx->num_sms * bps;
    if (grid > B.n_tiles) grid = B.n_tiles;
    if (grid < 1) grid = 1;
    CK(cudaMemsetAsync(ctx->counter.p, 0, sizeof(int), s));
    {
        StageScope sc_(ctx, SWGS_STAGE_BLEND_BWD, s);
        CK(launch_blend_bwd(ba, tw, th, bbatch, ppt, (int)grid, s));
    }
    {
        StageScope sc_(ctx, SWGS_STAGE_PREPROCESS_BWD, s);
        CK(launch_preprocess_bwd(*g, *grads, P<ViewDev>(B.views), P<GroupDev>(B.groups),
                                 B.n_groups, P<int32_t>(B.ids),
                                 dev ? B.act_cap : B.total_active, P<float>(B.grad2d), use_reg,
                                 use_reg ? loss : nullptr, s, dev ? dtot + kTotActive : nullptr));
    }
    return SWGS_OK;
}

// Device bytes of one batch's data at the sizes it needed, with the element
// sizes render_batch allocates: *rec = the record-proportional part (active
// ids of each frame group's slots, the per-record arrays of the saved state
// and the record-order scratch), *all = that plus the keys, tile lists, tile
// ranges and per-pixel arrays.
void batch_device_bytes(const BatchState& B, long long* rec, long long* all) {
    const long long per_record = 3 * 16 + 4 + 4 + 8 + 4 + 2 * kRunRows  // saved records
                                 + 4 * 4;                               // order, counts, offsets
    const long long ids = 4LL * B.total_active;
    *rec = ids + per_record * B.n_rec;
    *all = *rec + 16LL * B.n_sort_keys     // super keys and values, ping-pong
           + 4LL * B.n_keys                // per-tile lists
           + 16LL * B.n_tiles              // tile ranges, counts, offsets
           + 8LL * B.n_supers              // super-tile ranges
           + 8LL * B.n_pix;                // final T and last
}

// ---- export helpers -------------------------------------------------------
__global__ void export_record_kernel(int what, const ViewDev* views, int n_views,
                                     const GroupDev* groups, const int32_t* ids, Records rec,
                                     const int* call_index_dev, long long n, void* out) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int vi = find_view_by_record(views, n_views, (int)r);
    const ViewDev& V = views[vi];
    const GroupDev& G = groups[V.group];
    const int i = (int)(r - V.rec_base);
    switch (what) {
        case SWGS_EXPORT_RECORD_SLOT: ((int32_t*)out)[r] = ids[G.act_base + i]; break;
        case SWGS_EXPORT_RECORD_VIEW: ((int32_t*)out)[r] = call_index_dev[vi]; break;
        case SWGS_EXPORT_RECORD_TILES: ((int32_t*)out)[r] = rec.tiles[r]; break;
        case SWGS_EXPORT_RECORD_DEPTH: ((float*)out)[r] = rec.a[r].w; break;
        case SWGS_EXPORT_RECORD_RECT: {
            const short4 q = rec.rect[r];
            int32_t* o = (int32_t*)out + 4 * r;
            o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
            break;
        }
        case SWGS_EXPORT_RECORD_2D: {
            float4* o = (float4*)out + 3 * r;
            o[0] = rec.a[r]; o[1] = rec.b[r]; o[2] = rec.c[r];
            break;
        }
    }
}

// The per-tile lists, compacted in tile order (CSR at coff), as slots: one
// warp per tile.
__global__ void export_lists_kernel(const int2* ranges, const int32_t* coff, long long n_tiles,
                                    const uint32_t* vals, const ViewDev* views, int n_views,
                                    const GroupDev* groups, const int32_t* ids, int32_t* out) {
    const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= n_tiles) return;
    const int2 rg = ranges[t];
    const int o = coff[t];
    for (int i = rg.x + lane; i < rg.y; i += 32) {
        const int r = (int)vals[i];
        const ViewDev& V = views[find_view_by_record(views, n_views, r)];
        out[o + (i - rg.x)] = ids[groups[V.group].act_base + (r - V.rec_base)];
    }
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int32_t swgs_abi_version(void) { return SWGS_ABI_VERSION; }

swgs_status swgs_default_config(swgs_config* cfg) {
    if (!cfg) return SWGS_EINVAL;
    cfg->tile_w = 16;
    cfg->tile_h = 16;
    cfg->batch = 64;
    cfg->near_plane = 0.2f;
    cfg->blocks_per_sm = 0;
    cfg->count_pairs = 0;
    cfg->pixels_per_thread = 4;
    cfg->bwd_pixels_per_thread = 8;
    cfg->bwd_batch = 32;
    cfg->sort_single_pass = 1;
    cfg->deferred_sizing = 0;
    return SWGS_OK;
}

swgs_status swgs_create(const swgs_config* cfg, swgs_alloc_fn alloc, swgs_free_fn free_fn,
                        void* user, swgs_ctx** out) {
    if (!out) return SWGS_EINVAL;
    *out = nullptr;
    swgs_config c{};
    if (cfg) c = *cfg; else swgs_default_config(&c);
    if (c.bwd_pixels_per_thread == 0) c.bwd_pixels_per_thread = c.pixels_per_thread;
    if (c.bwd_batch == 0) c.bwd_batch = c.batch;
    if (!valid_tile(c.tile_w, c.tile_h) || !valid_batch(c.batch) || !(c.near_plane > 0.f) ||
        c.blocks_per_sm < 0 || (c.sort_single_pass != 0 && c.sort_single_pass != 1) ||
        (c.deferred_sizing != 0 && c.deferred_sizing != 1) ||
        !blend_config_valid(c.tile_w, c.tile_h, c.batch, c.pixels_per_thread, false) ||
        !blend_config_valid(c.tile_w, c.tile_h, c.bwd_batch, c.bwd_pixels_per_thread, true))
        return SWGS_EINVAL;
    if ((alloc == nullptr) != (free_fn == nullptr)) return SWGS_EINVAL;
    swgs_ctx* ctx = new swgs_ctx();
    ctx->cfg = c;
    ctx->alloc = alloc;
    ctx->free_fn = free_fn;
    ctx->user = user;
    if (cudaGetDevice(&ctx->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) !=
            cudaSuccess ||
        cudaMallocHost(&ctx->pinned, 4096) != cudaSuccess) {
        delete ctx;
        return SWGS_ECUDA;
    }
    ctx->pinned_cap = 4096;
    // every expansion instantiation loaded now, not at its first launch
    if (load_expand_kernels() != cudaSuccess) {
        cudaFreeHost(ctx->pinned);
        delete ctx;
        return SWGS_ECUDA;
    }
    *out = ctx;
    return SWGS_OK;
}

void swgs_destroy(swgs_ctx* ctx) {
    if (!ctx) return;
    cudaStream_t s = ctx->last_stream;
    cudaStreamSynchronize(s);
    Buf* bs[] = {&ctx->frames, &ctx->block_cnt, &ctx->scan_tmp, &ctx->counts, &ctx->order_a,
                 &ctx->order_b, &ctx->tcount, &ctx->koff, &ctx->keys_a, &ctx->keys_b,
                 &ctx->vals_tmp, &ctx->vals_b, &ctx->sranges, &ctx->tile_cnt, &ctx->tile_off,
                 &ctx->mature_ids, &ctx->mature_stage, &ctx->codec_keys_a, &ctx->codec_keys_b,
                 &ctx->codec_vals_a, &ctx->codec_vals_b, &ctx->codec_flags, &ctx->codec_idx,
                 &ctx->codec_stage, &ctx->sort_tmp, &ctx->counter, &ctx->totals, &ctx->l1_tab,
                 &ctx->elig, &ctx->reloc_w, &ctx->reloc_cdf, &ctx->reloc_dead, &ctx->reloc_tg,
                 &ctx->reloc_cnt, &ctx->reloc_nd, &ctx->reloc_lr, &ctx->reloc_nl, &ctx->sort_err,
                 &ctx->gate};
    for (Buf* b : bs) ctx_free(ctx, *b, s);
    for (swgs_saved* sv : ctx->all_saved) {
        free_saved_buffers(ctx, sv, s);
        delete sv;
    }
    cudaStreamSynchronize(s);
    for (const ProfEvent& e : ctx->prof_pending) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    for (cudaEvent_t e : ctx->prof_free) cudaEventDestroy(e);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    delete ctx;
}

const char* swgs_last_error(const swgs_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

swgs_status swgs_slice_range(int64_t target_frame, int64_t swin_size, int64_t num_gs,
                             int64_t* first, int64_t* count) {
    if (swin_size <= 0 || num_gs < 0 || !first || !count || num_gs % swin_size != 0)
        return SWGS_EINVAL;
    int64_t slice = target_frame % swin_size;
    if (slice < 0) slice += swin_size;
    *count = num_gs / swin_size;
    *first = slice * (*count);
    return SWGS_OK;
}

swgs_status swgs_active_ids(swgs_ctx* ctx, const int32_t* start, const int32_t* expire, int64_t n,
                            int32_t frame, int32_t* out_ids, int32_t* out_count, void* stream) {
    if (!ctx) return SWGS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    if (n < 0 || n > 0x7fffffffLL || !out_count || (n > 0 && (!start || !expire || !out_ids)))
        return fail(ctx, SWGS_EINVAL, "bad arguments to swgs_active_ids");
    if (n == 0) {
        CK(cudaMemsetAsync(out_count, 0, sizeof(int32_t), s));
        return SWGS_OK;
    }
    const int nb = (int)((n + kCompactBlock - 1) / kCompactBlock);
    if (!ensure(ctx, ctx->frames, sizeof(int32_t), s) ||
        !ensure(ctx, ctx->block_cnt, sizeof(uint32_t) * ((size_t)nb + 1), s) ||
        !ensure(ctx, ctx->scan_tmp, scan_u32_temp_bytes(nb + 1) + 64, s) ||
        !ensure(ctx, ctx->totals, 64, s))
        return fail(ctx, SWGS_ENOMEM, "allocation failed");
    CK(cudaMemcpyAsync(ctx->frames.p, &frame, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CK(launch_active_flags_count(start, expire, n, P<int32_t>(ctx->frames), 1,
                                 P<uint32_t>(ctx->block_cnt), nb, s));
    CK(exclusive_scan_u32(P<uint32_t>(ctx->block_cnt), P<uint32_t>(ctx->block_cnt), nb,
                          ctx->scan_tmp.p, P<unsigned long long>(ctx->totals), s));
    CK(launch_active_write(start, expire, n, P<int32_t>(ctx->frames), 1, P<uint32_t>(ctx->block_cnt),
                           nb, out_ids, 0, out_count, s));
    return SWGS_OK;
}

swgs_status swgs_frame_update(swgs_ctx* ctx, const swgs_gaussians* dst, int64_t first,
                              int64_t count, const swgs_gaussians* src, int32_t src_on_host,
                              void* stream) {
    if (!ctx) return SWGS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    swgs_status st = check_gaussians(ctx, dst, true);
    if (st != SWGS_OK) return st;
    if (!src || first < 0 || count < 0 || first + count > dst->capacity || src->capacity < count ||
        src->sh_degree != dst->sh_degree)
        return fail(ctx, SWGS_EINVAL, "bad slice [%lld, %lld) for capacity %lld",
                    (long long)first, (long long)(first + count), (long long)dst->capacity);
    if (count == 0) return SWGS_OK;
    const int K = (dst->sh_degree + 1) * (dst->sh_degree + 1);
    StageScope sc_(ctx, SWGS_STAGE_UPDATE, s);
    if (src_on_host) {
        struct { void* d; const void* s; size_t w; } arr[9] = {
            {dst->means, src->means, 12}, {dst->log_scales, src->log_scales, 12},
            {dst->quats, src->quats, 16}, {dst->opacity_logits, src->opacity_logits, 4},
            {dst->sh, src->sh, (size_t)12 * K}, {dst->start, src->start, 4},
            {dst->expire, src->expire, 4}, {dst->birth, src->birth, 4},
            {dst->frozen, src->frozen, 1}};
        for (auto& a : arr) {
            if (!a.s || !a.d) continue;
            CK(cudaMemcpyAsync((char*)a.d + a.w * (size_t)first, a.s, a.w * (size_t)count,
                               cudaMemcpyHostToDevice, s));
        }
        return SWGS_OK;
    }
    CK(launch_copy_slice(*dst, first, count, *src, s));
    return SWGS_OK;
}

static swgs_status check_mature_buffer(swgs_ctx* ctx, const swgs_gaussians* buf, int64_t num_gs,
                                       int32_t swin_size) {
    swgs_status st = check_gaussians(ctx, buf, true);
    if (st != SWGS_OK) return st;
    if (!buf->birth || !buf->frozen)
        return fail(ctx, SWGS_EINVAL, "maturation needs the birth and frozen arrays");
    if (num_gs <= 0 || buf->capacity < 2 * num_gs)
        return fail(ctx, SWGS_EINVAL, "capacity %lld cannot hold gs and the matured ring of %lld",
                    (long long)buf->capacity, (long long)num_gs);
    if (swin_size <= 0 || num_gs % swin_size != 0)
        return fail(ctx, SWGS_EINVAL, "num_gs %lld is not a multiple of swin_size %d",
                    (long long)num_gs, swin_size);
    return SWGS_OK;
}

size_t swgs_slice_packet_bytes(int64_t count, int64_t keep) {
    if (count < 0 || keep < 0 || keep > count) return 0;
    CodecLayout L;
    codec_layout(count, keep, &L);
    return L.total;
}

swgs_status swgs_slice_encode(swgs_ctx* ctx, const swgs_gaussians* src, int64_t count,
                              int64_t keep, void* out, size_t out_capacity, int32_t out_on_host,
                              size_t* out_bytes, void* stream) {
    if (!ctx) return SWGS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    swgs_status st = check_gaussians(ctx, src, true);
    if (st != SWGS_OK) return st;
    if (!src->birth || count < 0 || count > src->capacity || keep < 0 || keep > count ||
        count > 0x7fffffffLL || !out || !out_bytes)
        return fail(ctx, SWGS_EINVAL, "bad slice encode arguments (count %lld, keep %lld)",
                    (long long)count, (long long)keep);
    CodecLayout L;
    codec_layout(count, keep, &L);
    if (out_capacity < L.total)
        return fail(ctx, SWGS_EINVAL, "packet needs %zu bytes, buffer has %zu", L.total,
                    out_capacity);
    *out_bytes = L.total;
    const uint32_t* idx = nullptr;
    if (keep > 0 && keep < count) {
        const long long nb = (count + 255) / 256;
        const size_t n = (size_t)count;
        if (!ensure(ctx, ctx->codec_keys_a, 4 * n, s) || !ensure(ctx, ctx->codec_keys_b, 4 * n, s) ||
            !ensure(ctx, ctx->codec_vals_a, 4 * n, s) || !ensure(ctx, ctx->codec_vals_b, 4 * n, s) ||
            !ensure(ctx, ctx->codec_flags, n, s) || !ensure(ctx, ctx->codec_idx, 4 * n, s) ||
            !ensure(ctx, ctx->block_cnt, 4 * (size_t)(nb + 1), s) ||
            !ensure(ctx, ctx->scan_tmp, scan_u32_temp_bytes(nb + 1) + 64, s) ||
            !ensure(ctx, ctx->totals, 64, s) ||
            !ensure(ctx, ctx->sort_tmp, radix_temp_bytes(count, ctx->num_sms), s))
            return fail(ctx, SWGS_ENOMEM, "allocation failed (slice encode)");
        CodecScratch w{P<uint32_t>(ctx->codec_keys_a), P<uint32_t>(ctx->codec_keys_b),
                       P<uint32_t>(ctx->codec_vals_a), P<uint32_t>(ctx->codec_vals_b),
                       P<uint32_t>(ctx->block_cnt), P<uint32_t>(ctx->codec_idx),
                       P<uint8_t>(ctx->codec_flags), ctx->sort_tmp.p, ctx->scan_tmp.p,
                       P<unsigned long long>(ctx->totals), sort_err_word(ctx, s),
                       ctx->cfg.sort_single_pass != 0};
        uint32_t* sel = nullptr;
        CK(launch_codec_select(src->opacity_logits, count, keep, w, ctx->num_sms, &sel, s));
        idx = sel;
    }
    unsigned char* dst = (unsigned char*)out;
    if (out_on_host) {
        if (!ensure(ctx, ctx->codec_stage, L.total, s))
            return fail(ctx, SWGS_ENOMEM, "allocation failed (slice encode)");
        dst = P<unsigned char>(ctx->codec_stage);
    }
    CK(launch_codec_encode(*src, idx, count, keep, L, dst, s));
    if (out_on_host) CK(cudaMemcpyAsync(out, dst, L.total, cudaMemcpyDeviceToHost, s));
    return SWGS_OK;
}

swgs_status swgs_slice_decode(swgs_ctx* ctx, const void* packet, size_t bytes,
                              int32_t packet_on_host, const swgs_gaussians* dst, int64_t first,
                              void* stream) {
    if (!ctx) return SWGS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    swgs_status st = check_gaussians(ctx, dst, true);
    if (st != SWGS_OK) return st;
    if (!packet || bytes < kCodecHeaderBytes)
        return fail(ctx, SWGS_EINVAL, "packet shorter than its header");
    int32_t h[8];
    if (packet_on_host) {
        memcpy(h, packet, sizeof(h));
    } else {
        CK(cudaMemcpyAsync(ctx->pinned, packet, sizeof(h), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        memcpy(h, ctx->pinned, sizeof(h));
    }
    const long long count = h[2], keep = h[3];
    if ((uint32_t)h[0] != kCodecMagic || h[1] != kCodecVersion || count < 0 || keep < 0 ||
        keep > count || h[4] != dst->sh_degree)
        return fail(ctx, SWGS_EINVAL, "not a slice packet of this version and SH degree");
    CodecLayout L;
    codec_layout(count, keep, &L);
    if (bytes < L.total) return fail(ctx, SWGS_EINVAL, "packet truncated (%zu < %zu)", bytes, L.total);
    if (first < 0 || first + count > dst->capacity)
        return fail(ctx, SWGS_EINVAL, "slice [%lld, %lld) outside capacity %lld", (long long)first,
                    (long long)(first + count), (long long)dst->capacity);
    const unsigned char* in = (const unsigned char*)packet;
    if (packet_on_host) {
        if (!ensure(ctx, ctx->codec_stage, L.total, s))
            return fail(ctx, SWGS_ENOMEM, "allocation failed (slice decode)");
        CK(cudaMemcpyAsync(ctx->codec_stage.p, packet, L.total, cudaMemcpyHostToDevice, s));
        in = P<unsigned char>(ctx->codec_stage);
    }
    StageScope sc_(ctx, SWGS_STAGE_UPDATE, s);
    CK(launch_codec_decode(*dst, first, count, keep, L, in, h[5], h[6], h[7], s));
    return SWGS_OK;
}

swgs_status swgs_schedule_expire(swgs_ctx* ctx, const swgs_gaussians* buf, int64_t num_gs,
                                 int32_t swin_size, void* stream) {
    if (!ctx) return SWGS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    swgs_status st = check_mature_buffer(ctx, buf, num_gs, swin_size);
    if (st != SWGS_OK) return st;
    CK(launch_schedule_expire(buf->expire, num_gs, swin_size, s));
    return SWGS_OK;
}

swgs_status swgs_mature(swgs_ctx* ctx, const swgs_gaussians* buf, int64_t num_gs, int32_t st_frame,
                        int32_t swin_size, int64_t* head, const swgs_gaussians* snapshot,
                        int32_t snapshot_on_host, int64_t* n_out, void* stream) {
    if (!ctx) return SWGS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    swgs_status st = check_mature_buffer(ctx, buf, num_gs, swin_size);
    if (st != SWGS_OK) return st;
    if (!head || *head < 0 || *head >= num_gs || !n_out)
        return fail(ctx, SWGS_EINVAL, "bad ring head or null count");
    if (snapshot && (snapshot->capacity < num_gs || snapshot->sh_degree != buf->sh_degree))
        return fail(ctx, SWGS_EINVAL, "snapshot must hold num_gs rows of the same SH degree");
    const long long n_blocks = (num_gs + 255) / 256;
    if (!ensure(ctx, ctx->block_cnt, sizeof(uint32_t) * (size_t)(n_blocks + 1), s) ||
        !ensure(ctx, ctx->scan_tmp, scan_u32_temp_bytes(n_blocks + 1) + 64, s) ||
        !ensure(ctx, ctx->totals, 64, s) ||
        !ensure(ctx, ctx->mature_ids, sizeof(int32_t) * (size_t)num_gs, s))
        return fail(ctx, SWGS_ENOMEM, "allocation failed (maturation)");
    // 1. mature_idx: the gs slots with start < st, ascending
    CK(launch_mature_ids(buf->start, num_gs, st_frame, P<uint32_t>(ctx->block_cnt),
                         ctx->scan_tmp.p, P<unsigned long long>(ctx->totals),
                         P<int32_t>(ctx->mature_ids), s));
    CK(cudaMemcpyAsync(ctx->pinned, ctx->totals.p, sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    unsigned long long n = 0;
    memcpy(&n, ctx->pinned, sizeof(n));
    *n_out = (int64_t)n;
    if (n == 0) return SWGS_OK;
    // 2-4. snapshot and ring copies of the rows as they are, then their rebirth
    const int K = (buf->sh_degree + 1) * (buf->sh_degree + 1);
    const size_t row_b[9] = {12, 12, 16, 4, (size_t)12 * K, 4, 4, 4, 1};
    void* snap[9] = {nullptr, nullptr, nullptr, nullptr, nullptr,
                     nullptr, nullptr, nullptr, nullptr};
    void* const hs[9] = {snapshot ? snapshot->means : nullptr,
                         snapshot ? snapshot->log_scales : nullptr,
                         snapshot ? snapshot->quats : nullptr,
                         snapshot ? snapshot->opacity_logits : nullptr,
                         snapshot ? snapshot->sh : nullptr,
                         snapshot ? snapshot->start : nullptr,
                         snapshot ? snapshot->expire : nullptr,
                         snapshot ? snapshot->birth : nullptr,
                         snapshot ? (void*)snapshot->frozen : nullptr};
    if (snapshot && snapshot_on_host) {
        // staged on the device, then one copy per array to the pinned rows
        size_t off[9], tot = 0;
        for (int i = 0; i < 9; ++i) {
            off[i] = tot;
            tot += (row_b[i] * (size_t)n + 255) & ~(size_t)255;
        }
        if (!ensure(ctx, ctx->mature_stage, tot, s))
            return fail(ctx, SWGS_ENOMEM, "allocation failed (maturation snapshot)");
        for (int i = 0; i < 9; ++i) snap[i] = hs[i] ? (char*)ctx->mature_stage.p + off[i] : nullptr;
    } else if (snapshot) {
        for (int i = 0; i < 9; ++i) snap[i] = hs[i];
    }
    CK(launch_mature_move(*buf, P<int32_t>(ctx->mature_ids), (long long)n, num_gs, *head,
                          swin_size, snap, s));
    if (snapshot && snapshot_on_host)
        for (int i = 0; i < 9; ++i)
            if (hs[i])
                CK(cudaMemcpyAsync(hs[i], snap[i], row_b[i] * (size_t)n, cudaMemcpyDeviceToHost, s));
    *head = (int64_t)((*head + (long long)n) % num_gs);
    return SWGS_OK;
}

static swgs_status render_fwd_impl(swgs_ctx* ctx, const swgs_gaussians* g, int32_t n_views,
                                   const swgs_view* views, const float* bg,
                                   float* const* out_rgb, uint8_t* const* out_rgb8,
                                   float* const* out_T,
                                   const void* const* targets, int target_u8,
                                   float* const* dls, float* loss,
                                   int32_t batched, swgs_saved** saved, void* stream);

swgs_status swgs_render_fwd(swgs_ctx* ctx, const swgs_gaussians* g, int32_t n_views,
                            const swgs_view* views, const float* bg, float* const* out_rgb,
                            float* const* out_T, int32_t batched, swgs_saved** saved,
                            void* stream) {
    return render_fwd_impl(ctx, g, n_views, views, bg, out_rgb, nullptr, out_T, nullptr, 0,
                           nullptr, nullptr, batched, saved, stream);
}

swgs_status swgs_render_fwd_rgb8(swgs_ctx* ctx, const swgs_gaussians* g, int32_t n_views,
                                 const swgs_view* views, const float* bg,
                                 uint8_t* const* out_rgb8, float* const* out_T, int32_t batched,
                                 swgs_saved** saved, void* stream) {
    return render_fwd_impl(ctx, g, n_views, views, bg, nullptr, out_rgb8, out_T, nullptr, 0,
                           nullptr, nullptr, batched, saved, stream);
}

static swgs_status render_fwd_l1_impl(swgs_ctx* ctx, const swgs_gaussians* g, int32_t n_views,
                                      const swgs_view* views, const float* bg,
                                      float* const* out_rgb, float* const* out_T,
                                      const void* const* target, int target_u8,
                                      float* const* dL_drgb, float* loss, int32_t batched,
                                      swgs_saved** saved, void* stream) {
    if (!ctx) return SWGS_EINVAL;
    if (!target || !dL_drgb || !loss) return fail(ctx, SWGS_EINVAL, "null target, dL or loss");
    if (n_views > 0 && !views) return fail(ctx, SWGS_EINVAL, "null view list");
    for (int v = 0; v < n_views; ++v)
        if (!target[v] || !dL_drgb[v]) return fail(ctx, SWGS_EINVAL, "view %d: null target or dL", v);
    if (cudaMemsetAsync(loss, 0, sizeof(float), (cudaStream_t)stream) != cudaSuccess)
        return fail(ctx, SWGS_ECUDA, "clearing the loss failed");
    return render_fwd_impl(ctx, g, n_views, views, bg, out_rgb, nullptr, out_T, target, target_u8,
                           dL_drgb, loss, batched, saved, stream);
}

swgs_status swgs_render_fwd_l1(swgs_ctx* ctx, const swgs_gaussians* g, int32_t n_views,
                               const swgs_view* views, const float* bg, float* const* out_rgb,
                               float* const* out_T, const float* const* target,
                               float* const* dL_drgb, float* loss, int32_t batched,
                               swgs_saved** saved, void* stream) {
    return render_fwd_l1_impl(ctx, g, n_views, views, bg, out_rgb, out_T,
                              (const void* const*)target, 0, dL_drgb, loss, batched, saved,
                              stream);
}

swgs_status swgs_render_fwd_l1_u8(swgs_ctx* ctx, const swgs_gaussians* g, int32_t n_views,
                                  const swgs_view* views, const float* bg, float* const* out_rgb,
                                  float* const* out_T, const uint8_t* const* target,
                                  float* const* dL_drgb, float* loss, int32_t batched,
                                  swgs_saved** saved, void* stream) {
    return render_fwd_l1_impl(ctx, g, n_views, views, bg, out_rgb, out_T,
                              (const void* const*)target, 1, dL_drgb, loss, batched, saved,
                              stream);
}

static swgs_status render_fwd_impl(swgs_ctx* ctx, const swgs_gaussians* g, int32_t n_views,
                                   const swgs_view* views, const float* bg,
                                   float* const* out_rgb, uint8_t* const* out_rgb8,
                                   float* const* out_T,
                                   const void* const* targets, int target_u8,
                                   float* const* dls, float* loss,
                                   int32_t batched, swgs_saved** saved, void* stream) {
    if (!ctx) return SWGS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    ctx->err.clear();
    swgs_status st = check_gaussians(ctx, g, true);
    if (st != SWGS_OK) return st;
    // the L1 forms need no image: their outputs are the loss and its gradient
    if (n_views <= 0 || !views || (!out_rgb && !out_rgb8 && !targets))
        return fail(ctx, SWGS_EINVAL, "need at least one view and its output buffer");
    if (n_views > kMaxViewsPerBatch)
        return fail(ctx, SWGS_EINVAL, "at most %d views per call", kMaxViewsPerBatch);
    for (int v = 0; v < n_views; ++v) {
        const swgs_view& w = views[v];
        if (w.width <= 0 || w.height <= 0 || w.width > 16384 || w.height > 16384 ||
            !(w.fx > 0.f) || !(w.fy > 0.f) ||
            (out_rgb ? !out_rgb[v] : (out_rgb8 && !out_rgb8[v])))
            return fail(ctx, SWGS_EINVAL, "view %d: bad size, focal length or output", v);
    }
    if (saved) *saved = nullptr;
    if (ctx->cfg.deferred_sizing) {
        // learn the capacities from every earlier call that has finished, and
        // lower the gate for this call's optimiser steps
        for (swgs_saved* o : ctx->all_saved)
            for (auto& b : o->batches) resolve_batch(ctx, b, false);
        uint32_t* gw = gate_word(ctx, s);
        if (!gw) return fail(ctx, SWGS_ENOMEM, "allocation failed (gate word)");
        CK(cudaMemsetAsync(gw, 0, 4, s));
    }
    swgs_saved* sv = acquire_saved(ctx);
    sv->n_views = n_views;
    sv->count_pairs = ctx->cfg.count_pairs != 0;
    // batches: one per view (plain), or consecutive runs of views holding at
    // most kMaxSupersPerBatch super tiles each (batched)
    std::vector<std::vector<int>> parts;
    {
        const int tw = ctx->cfg.tile_w, th = ctx->cfg.tile_h;
        const int SX = super_w(tw), SY = super_h(tw);
        long long acc = 0;
        for (int v = 0; v < n_views; ++v) {
            const long long ntx = (views[v].width + tw - 1) / tw, nty = (views[v].height + th - 1) / th;
            const long long sup = ((ntx + SX - 1) / SX) * ((nty + SY - 1) / SY);
            if (sup > kMaxSupersPerBatch) {
                ctx->pool.push_back(sv);
                return fail(ctx, SWGS_EINVAL,
                            "view %d has %lld super tiles of %dx%d tiles (at most %lld): "
                            "use larger tiles", v, sup, SX, SY, kMaxSupersPerBatch);
            }
            if (parts.empty() || !batched || acc + sup > kMaxSupersPerBatch) {
                parts.emplace_back();
                acc = 0;
            }
            parts.back().push_back(v);
            acc += sup;
        }
    }
    const int nb = (int)parts.size();
    if ((int)sv->batches.size() < nb) sv->batches.resize(nb);
    sv->n_batches = nb;
    unsigned long long* pairs = nullptr;
    if (sv->count_pairs) {
        if (!ensure(ctx, sv->pairs, sizeof(unsigned long long), s)) {
            ctx->pool.push_back(sv);
            return fail(ctx, SWGS_ENOMEM, "allocation failed");
        }
        pairs = P<unsigned long long>(sv->pairs);
        cudaError_t e = cudaMemsetAsync(pairs, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) {
            ctx->pool.push_back(sv);
            return fail(ctx, SWGS_ECUDA, "memset: %s", cudaGetErrorString(e));
        }
    }
    for (int b = 0; b < nb; ++b) {
        st = render_batch(ctx, g, views, parts[b], bg, out_rgb, out_rgb8, out_T, targets,
                          target_u8, dls,
                          loss, n_views,
                          sv->batches[b], pairs, s);
        if (st != SWGS_OK) {
            // a failed call leaves no deferred totals to wait for
            for (int k = 0; k <= b; ++k) {
                sv->batches[k].resolved = true;
                sv->batches[k].status = st;
            }
            ctx->pool.push_back(sv);
            return st;
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        ctx->pool.push_back(sv);
        return fail(ctx, SWGS_ECUDA, "render: %s", cudaGetErrorString(e));
    }
    if (saved) *saved = sv;
    else ctx->pool.push_back(sv);
    return SWGS_OK;
}

swgs_status swgs_render_bwd(swgs_ctx* ctx, const swgs_gaussians* g, const swgs_saved* saved,
                            const float* const* dL_drgb, const swgs_gaussians* grads,
                            void* stream) {
    return swgs_render_bwd_reg(ctx, g, saved, dL_drgb, grads, nullptr, nullptr, stream);
}

swgs_status swgs_render_bwd_reg(swgs_ctx* ctx, const swgs_gaussians* g, const swgs_saved* saved,
                                const float* const* dL_drgb, const swgs_gaussians* grads,
                                const swgs_reg_params* reg, float* loss, void* stream) {
    if (!ctx) return SWGS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    ctx->err.clear();
    swgs_status st = check_gaussians(ctx, g, true);
    if (st != SWGS_OK) return st;
    if (!saved || saved->ctx != ctx) return fail(ctx, SWGS_ESTATE, "saved state from another context");
    if (!dL_drgb || !grads || grads->capacity != g->capacity || grads->sh_degree != g->sh_degree ||
        !grads->means || !grads->log_scales || !grads->quats || !grads->opacity_logits || !grads->sh)
        return fail(ctx, SWGS_EINVAL, "gradient buffers do not match the Gaussian state");
    swgs_saved* sv = const_cast<swgs_saved*>(saved);
    if (reg && (!(reg->opacity_reg >= 0.f) || !(reg->scale_reg >= 0.f) || reg->n_views_total < 0))
        return fail(ctx, SWGS_EINVAL, "regulariser weights must be >= 0");
    for (int b = 0; b < sv->n_batches; ++b) {
        st = backward_batch(ctx, g, sv->batches[b], dL_drgb, grads, reg, sv->n_views, loss, s);
        if (st != SWGS_OK) return st;
    }
    return SWGS_OK;
}

swgs_status swgs_saved_release(swgs_ctx* ctx, swgs_saved* saved) {
    if (!ctx || !saved || saved->ctx != ctx) return SWGS_EINVAL;
    ctx->pool.push_back(saved);
    return SWGS_OK;
}

swgs_status swgs_saved_status(swgs_ctx* ctx, const swgs_saved* saved, int32_t wait) {
    if (!ctx || !saved || saved->ctx != ctx) return SWGS_EINVAL;
    swgs_status out = SWGS_OK;
    for (int b = 0; b < saved->n_batches; ++b) {
        BatchState& B = const_cast<swgs_saved*>(saved)->batches[b];
        const swgs_status st = resolve_batch(ctx, B, wait != 0);
        if (st == SWGS_EPENDING) return SWGS_EPENDING;
        if (st != SWGS_OK && out == SWGS_OK) out = st;
    }
    if (out == SWGS_EDEVICE)
        return fail(ctx, SWGS_EDEVICE,
                    "a batch outgrew the deferred capacities (its outputs are background); the "
                    "context has grown them to %lld records, %lld super keys, %lld tile keys: "
                    "render it again", ctx->cap_rec, ctx->cap_sk, ctx->cap_keys);
    if (out == SWGS_ETIMEOUT)
        return fail(ctx, SWGS_ETIMEOUT, "a radix-sort look-back wait ran out in this call");
    return out;
}

// Every batch's host counts, waiting for deferred ones.
static swgs_status resolve_all(swgs_ctx* ctx, const swgs_saved* saved) {
    for (int b = 0; b < saved->n_batches; ++b) {
        const swgs_status st =
            resolve_batch(ctx, const_cast<swgs_saved*>(saved)->batches[b], true);
        if (st == SWGS_ECUDA) return st;
    }
    return SWGS_OK;
}

swgs_status swgs_saved_query(swgs_ctx* ctx, const swgs_saved* saved, swgs_saved_info* info) {
    if (!ctx || !saved || !info) return SWGS_EINVAL;
    if (resolve_all(ctx, saved) != SWGS_OK) return SWGS_ECUDA;
    swgs_saved_info o{};
    o.n_views = saved->n_views;
    o.n_batches = saved->n_batches;
    for (int b = 0; b < saved->n_batches; ++b) {
        const BatchState& B = saved->batches[b];
        o.n_records += B.n_rec;
        o.n_keys += B.n_keys;
        o.n_tiles += B.n_tiles;
        o.n_pixels += B.n_pix;
        o.n_sort_keys += B.n_sort_keys;
        o.n_supers += B.n_supers;
        long long rb = 0, db = 0;
        batch_device_bytes(B, &rb, &db);
        o.record_bytes += rb;
        o.device_bytes += db;
    }
    if (saved->count_pairs && saved->pairs.p) {
        cudaStream_t s = ctx->last_stream;
        if (cudaMemcpyAsync(ctx->pinned, saved->pairs.p, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(ctx, SWGS_ECUDA, "reading the pair counter failed");
        unsigned long long p;
        memcpy(&p, ctx->pinned, 8);
        o.pairs = (int64_t)p;
    } else {
        o.pairs = -1;
    }
    *info = o;
    return SWGS_OK;
}

swgs_status swgs_saved_count(swgs_ctx* ctx, const swgs_saved* saved, int32_t what, int64_t* count) {
    if (!ctx || !saved || !count) return SWGS_EINVAL;
    if (resolve_all(ctx, saved) != SWGS_OK) return SWGS_ECUDA;
    long long n = 0;
    for (int b = 0; b < saved->n_batches; ++b) {
        const BatchState& B = saved->batches[b];
        switch (what) {
            case SWGS_EXPORT_RECORD_SLOT: case SWGS_EXPORT_RECORD_VIEW: case SWGS_EXPORT_RECORD_TILES:
            case SWGS_EXPORT_RECORD_DEPTH: case SWGS_EXPORT_RECORD_RECT: case SWGS_EXPORT_GRAD2D:
            case SWGS_EXPORT_RECORD_2D:
                n += B.n_rec; break;
            case SWGS_EXPORT_SORTED_SLOT: n += B.n_keys; break;
            case SWGS_EXPORT_TILE_RANGES: n += B.n_tiles; break;
            case SWGS_EXPORT_LAST: case SWGS_EXPORT_FINAL_T: n += B.n_pix; break;
            case 11: n += (long long)B.h_views.size(); break;
            default: return fail(ctx, SWGS_EINVAL, "unknown export %d", what);
        }
    }
    *count = n;
    return SWGS_OK;
}

// what == 11: the view table, int32 x 6 per view in batch order: call index,
// tile_base, pix_base, rec_base, ntx, nty (bases global over the batches).
swgs_status swgs_saved_export(swgs_ctx* ctx, const swgs_saved* saved, int32_t what, void* dst,
                              size_t bytes, void* stream) {
    if (!ctx || !saved || !dst) return SWGS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    int64_t n = 0;
    swgs_status st = swgs_saved_count(ctx, saved, what, &n);
    if (st != SWGS_OK) return st;
    size_t el = 4;
    if (what == SWGS_EXPORT_RECORD_RECT) el = 16;
    if (what == SWGS_EXPORT_TILE_RANGES) el = 8;
    if (what == SWGS_EXPORT_GRAD2D || what == SWGS_EXPORT_RECORD_2D) el = 48;
    if (what == 11) el = 24;
    if (bytes != el * (size_t)n)
        return fail(ctx, SWGS_EINVAL, "export %d needs %zu bytes, got %zu", what, el * (size_t)n, bytes);
    // device staging for kernels that write host memory indirectly
    cudaPointerAttributes pa{};
    bool dst_dev = cudaPointerGetAttributes(&pa, dst) == cudaSuccess &&
                   (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    Buf stage;
    char* out = (char*)dst;
    if (!dst_dev) {
        if (!ensure(ctx, stage, bytes, s)) return fail(ctx, SWGS_ENOMEM, "allocation failed");
        out = (char*)stage.p;
    }
    long long rec_off = 0, key_off = 0, tile_off = 0, pix_off = 0;
    char* cur = out;
    std::vector<int32_t> table;
    for (int b = 0; b < saved->n_batches; ++b) {
        BatchState& B = const_cast<swgs_saved*>(saved)->batches[b];
        long long m = 0;
        switch (what) {
            case SWGS_EXPORT_RECORD_SLOT: case SWGS_EXPORT_RECORD_VIEW: case SWGS_EXPORT_RECORD_TILES:
            case SWGS_EXPORT_RECORD_DEPTH: case SWGS_EXPORT_RECORD_RECT: case SWGS_EXPORT_RECORD_2D: {
                m = B.n_rec;
                if (m == 0) break;
                Buf ci;
                if (!ensure(ctx, ci, sizeof(int) * B.call_index.size(), s))
                    return fail(ctx, SWGS_ENOMEM, "allocation failed");
                CK(cudaMemcpyAsync(ci.p, B.call_index.data(), sizeof(int) * B.call_index.size(),
                                   cudaMemcpyHostToDevice, s));
                note_launch();
                export_record_kernel<<<div_up(m, 256), 256, 0, s>>>(
                    what, P<ViewDev>(B.views), (int)B.h_views.size(), P<GroupDev>(B.groups),
                    P<int32_t>(B.ids), records_of(B), P<int>(ci), m, cur);
                CK(cudaGetLastError());
                ctx_free(ctx, ci, s);
                break;
            }
            case SWGS_EXPORT_GRAD2D:
                m = B.n_rec;
                if (m == 0) break;
                if (!B.has_grad2d) return fail(ctx, SWGS_ESTATE, "no backward has run on this state");
                CK(cudaMemcpyAsync(cur, B.grad2d.p, 48 * (size_t)m, cudaMemcpyDeviceToDevice, s));
                break;
            case SWGS_EXPORT_SORTED_SLOT:
            case SWGS_EXPORT_TILE_RANGES: {
                // the lists live in per-tile regions of a capacity buffer;
                // both exports give them compacted in tile order
                m = what == SWGS_EXPORT_SORTED_SLOT ? B.n_keys : B.n_tiles;
                if (m == 0 || B.n_tiles == 0) break;
                std::vector<int2> hr((size_t)B.n_tiles);
                CK(cudaMemcpyAsync(hr.data(), B.ranges.p, sizeof(int2) * hr.size(),
                                   cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                std::vector<int32_t> coff(hr.size() + 1, 0);
                for (size_t t = 0; t < hr.size(); ++t) coff[t + 1] = coff[t] + (hr[t].y - hr[t].x);
                if (what == SWGS_EXPORT_TILE_RANGES) {
                    std::vector<int2> cr(hr.size());
                    for (size_t t = 0; t < hr.size(); ++t)
                        cr[t] = make_int2((int)(coff[t] + key_off), (int)(coff[t + 1] + key_off));
                    CK(cudaMemcpyAsync(cur, cr.data(), sizeof(int2) * cr.size(),
                                       cudaMemcpyHostToDevice, s));
                    CK(cudaStreamSynchronize(s));
                    break;
                }
                Buf dco;
                if (!ensure(ctx, dco, sizeof(int32_t) * coff.size(), s))
                    return fail(ctx, SWGS_ENOMEM, "allocation failed");
                CK(cudaMemcpyAsync(dco.p, coff.data(), sizeof(int32_t) * coff.size(),
                                   cudaMemcpyHostToDevice, s));
                note_launch();
                export_lists_kernel<<<div_up(B.n_tiles * 32, 256), 256, 0, s>>>(
                    P<int2>(B.ranges), P<int32_t>(dco), B.n_tiles, P<uint32_t>(B.vals),
                    P<ViewDev>(B.views), (int)B.h_views.size(), P<GroupDev>(B.groups),
                    P<int32_t>(B.ids), (int32_t*)cur);
                CK(cudaGetLastError());
                CK(cudaStreamSynchronize(s));
                ctx_free(ctx, dco, s);
                break;
            }
            case SWGS_EXPORT_LAST:
                m = B.n_pix;
                CK(cudaMemcpyAsync(cur, B.last.p, 4 * (size_t)m, cudaMemcpyDeviceToDevice, s));
                break;
            case SWGS_EXPORT_FINAL_T:
                m = B.n_pix;
                CK(cudaMemcpyAsync(cur, B.T.p, 4 * (size_t)m, cudaMemcpyDeviceToDevice, s));
                break;
            case 11:
                m = (long long)B.h_views.size();
                for (const ViewDev& V : B.h_views) {
                    table.push_back(B.call_index[&V - B.h_views.data()]);
                    table.push_back((int32_t)(V.tile_base + tile_off));
                    table.push_back((int32_t)(V.pix_base + pix_off));
                    table.push_back((int32_t)(V.rec_base + rec_off));
                    table.push_back(V.ntx);
                    table.push_back(V.nty);
                }
                break;
        }
        cur += el * (size_t)m;
        rec_off += B.n_rec;
        key_off += B.n_keys;
        tile_off += B.n_tiles;
        pix_off += B.n_pix;
    }
    if (what == 11) {
        CK(cudaMemcpyAsync(out, table.data(), bytes, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    }
    if (!dst_dev) {
        CK(cudaMemcpyAsync(dst, out, bytes, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        ctx_free(ctx, stage, s);
    }
    return SWGS_OK;
}

swgs_status swgs_loss_l1(swgs_ctx* ctx, int32_t n_views, const swgs_view* views,
                         const float* const* rgb, const float* const* target,
                         float* const* dL_drgb, float* loss, void* stream) {
    if (!ctx) return SWGS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    if (n_views <= 0 || !views || !rgb || !target || !dL_drgb || !loss)
        return fail(ctx, SWGS_EINVAL, "bad arguments to swgs_loss_l1");
    // table: pix offsets [V+1] (int64) then 3 pointer arrays [V]
    std::vector<long long> off(n_views + 1, 0);
    for (int v = 0; v < n_views; ++v) {
        if (views[v].width <= 0 || views[v].height <= 0 || !rgb[v] || !target[v] || !dL_drgb[v])
            return fail(ctx, SWGS_EINVAL, "view %d: bad size or buffer", v);
        off[v + 1] = off[v] + (long long)views[v].width * views[v].height;
    }
    std::vector<unsigned char> tab(8 * (n_views + 1) + 3 * 8 * n_views);
    memcpy(tab.data(), off.data(), 8 * (n_views + 1));
    memcpy(tab.data() + 8 * (n_views + 1), rgb, 8 * n_views);
    memcpy(tab.data() + 8 * (n_views + 1) + 8 * n_views, target, 8 * n_views);
    memcpy(tab.data() + 8 * (n_views + 1) + 16 * n_views, dL_drgb, 8 * n_views);
    if (!ensure(ctx, ctx->l1_tab, tab.size(), s)) return fail(ctx, SWGS_ENOMEM, "allocation failed");
    CK(cudaMemcpyAsync(ctx->l1_tab.p, tab.data(), tab.size(), cudaMemcpyHostToDevice, s));
    char* base = (char*)ctx->l1_tab.p;
    StageScope sc_(ctx, SWGS_STAGE_LOSS, s);
    CK(launch_loss_l1(nullptr, n_views, off[n_views], (const long long*)base,
                      (const float* const*)(base + 8 * (n_views + 1)),
                      (const float* const*)(base + 8 * (n_views + 1) + 8 * n_views),
                      (float* const*)(base + 8 * (n_views + 1) + 16 * n_views), loss, s));
    return SWGS_OK;
}

swgs_status swgs_grad_pack(swgs_ctx* ctx, const swgs_gaussians* g, const swgs_gaussians* grads,
                           const int32_t* frames, int32_t n_frames, float scale, int32_t* ids,
                           int64_t* count, float* packed, void* stream) {
    if (!ctx) return SWGS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    ctx->err.clear();
    swgs_status st = check_gaussians(ctx, g, true);
    if (st != SWGS_OK) return st;
    st = check_gaussians(ctx, grads, false);
    if (st != SWGS_OK) return st;
    if (grads->capacity != g->capacity || grads->sh_degree != g->sh_degree)
        return fail(ctx, SWGS_EINVAL, "gradients must match the state's capacity and SH degree");
    if (n_frames < 0 || n_frames > 64 || (n_frames > 0 && !frames) || !count ||
        (g->capacity > 0 && (!ids || !packed)))
        return fail(ctx, SWGS_EINVAL, "bad frames or output buffers (at most 64 frames)");
    const long long N = g->capacity;
    if (N == 0) {
        CK(cudaMemsetAsync(count, 0, sizeof(int64_t), s));
        return SWGS_OK;
    }
    const long long nb = (N + 255) / 256;
    if (!ensure(ctx, ctx->elig, (size_t)N, s) ||
        !ensure(ctx, ctx->block_cnt, sizeof(uint32_t) * (size_t)(nb + 1), s) ||
        !ensure(ctx, ctx->scan_tmp, scan_u32_temp_bytes(nb + 1) + 64, s))
        return fail(ctx, SWGS_ENOMEM, "allocation failed (gradient packing)");
    CK(launch_grad_pack(*g, *grads, frames, n_frames, scale, P<uint8_t>(ctx->elig),
                        P<uint32_t>(ctx->block_cnt), ctx->scan_tmp.p, ids, (long long*)count,
                        packed, s));
    return SWGS_OK;
}

swgs_status swgs_grad_unpack(swgs_ctx* ctx, const swgs_gaussians* grads, const int32_t* ids,
                             const int64_t* count, const float* packed, void* stream) {
    if (!ctx) return SWGS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    ctx->err.clear();
    swgs_status st = check_gaussians(ctx, grads, false);
    if (st != SWGS_OK) return st;
    if (!count || (grads->capacity > 0 && (!ids || !packed)))
        return fail(ctx, SWGS_EINVAL, "null ids, count or packed rows");
    CK(launch_grad_unpack(*grads, ids, (const long long*)count, grads->capacity, packed, s));
    return SWGS_OK;
}

swgs_status swgs_sgld_step(swgs_ctx* ctx, const swgs_gaussians* g, const swgs_gaussians* grads,
                           const swgs_adam_state* adam, const int32_t* frames, int32_t n_frames,
                           const swgs_sgld_params* params, uint64_t seed, uint64_t step,
                           int32_t* targets, int64_t* n_relocated, void* stream) {
    if (!ctx) return SWGS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    ctx->err.clear();
    swgs_status st = check_gaussians(ctx, g, true);
    if (st != SWGS_OK) return st;
    if (!params || n_frames < 0 || n_frames > 64 || (n_frames > 0 && !frames))
        return fail(ctx, SWGS_EINVAL, "bad frames or parameters (at most 64 frames)");
    if (params->adam && (!grads || !adam))
        return fail(ctx, SWGS_EINVAL, "an Adam step needs gradients and moments");
    if (params->max_n < 1) return fail(ctx, SWGS_EINVAL, "max_n must be >= 1");
    const long long N = g->capacity;
    if (N == 0) {
        if (n_relocated) *n_relocated = 0;
        return SWGS_OK;
    }
    {
        StageScope sc_(ctx, SWGS_STAGE_SGLD, s);
        if (!ensure(ctx, ctx->elig, (size_t)N, s))
            return fail(ctx, SWGS_ENOMEM, "allocation failed (eligible slots)");
        CK(launch_eligible(*g, frames, n_frames, P<uint8_t>(ctx->elig), s));
        CK(launch_sgld(*g, grads, adam, P<uint8_t>(ctx->elig), *params, seed, step, s,
                       ctx->cfg.deferred_sizing ? gate_word(ctx, s) : nullptr));
    }
    long long nd = 0;
    if (params->relocate) {
        StageScope sc_(ctx, SWGS_STAGE_RELOCATE, s);
        if (!ensure(ctx, ctx->reloc_w, 8 * (size_t)N, s) ||
            !ensure(ctx, ctx->reloc_cdf, 8 * (size_t)N, s) ||
            !ensure(ctx, ctx->reloc_dead, (size_t)N, s) ||
            !ensure(ctx, ctx->reloc_cnt, 4 * (size_t)N, s) ||
            !ensure(ctx, ctx->reloc_nd, 64, s) ||
            !ensure(ctx, ctx->reloc_lr, 8 * (size_t)N, s) ||
            !ensure(ctx, ctx->reloc_nl, 4 * (size_t)N, s) ||
            !ensure(ctx, ctx->scan_tmp, scan_u64_temp_bytes(N) + 64, s) ||
            (!targets && !ensure(ctx, ctx->reloc_tg, 4 * (size_t)N, s)))
            return fail(ctx, SWGS_ENOMEM, "allocation failed (relocation)");
        int32_t* tg = targets ? targets : P<int32_t>(ctx->reloc_tg);
        CK(launch_reloc_weights(*g, P<uint8_t>(ctx->elig), P<unsigned long long>(ctx->reloc_w),
                                P<uint8_t>(ctx->reloc_dead), s,
                                ctx->cfg.deferred_sizing ? gate_word(ctx, s) : nullptr));
        CK(inclusive_scan_u64(P<unsigned long long>(ctx->reloc_w), P<unsigned long long>(ctx->reloc_cdf),
                              N, ctx->scan_tmp.p, s));
        CK(cudaMemsetAsync(ctx->reloc_cnt.p, 0, 4 * (size_t)N, s));
        CK(cudaMemsetAsync(ctx->reloc_nd.p, 0, 8, s));
        CK(launch_reloc_sample(*g, P<uint8_t>(ctx->reloc_dead), P<unsigned long long>(ctx->reloc_cdf),
                               seed, step, tg, P<int32_t>(ctx->reloc_cnt),
                               P<unsigned long long>(ctx->reloc_nd), s));
        CK(launch_reloc_apply(*g, adam, tg, P<int32_t>(ctx->reloc_cnt), params->max_n,
                              P<double>(ctx->reloc_lr), P<float>(ctx->reloc_nl), s));
        if (n_relocated) {
            CK(cudaMemcpyAsync(ctx->pinned, ctx->reloc_nd.p, 8, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            unsigned long long v;
            memcpy(&v, ctx->pinned, 8);
            nd = (long long)v;
        }
    } else if (targets) {
        CK(cudaMemsetAsync(targets, 0xff, 4 * (size_t)N, s));
    }
    if (n_relocated) *n_relocated = nd;
    return SWGS_OK;
}

swgs_status swgs_selftest_sort_timeout(swgs_ctx* ctx, void* stream) {
    if (!ctx) return SWGS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    ctx->err.clear();
    if (!ensure(ctx, ctx->sort_tmp, sort_timeout_scratch_bytes(), s))
        return fail(ctx, SWGS_ENOMEM, "allocation failed (sort check)");
    uint32_t* serr = sort_err_word(ctx, s);
    if (!serr) return fail(ctx, SWGS_ENOMEM, "allocation failed (sort error word)");
    CK(launch_sort_timeout_check(ctx->sort_tmp.p, serr, s));
    CK(cudaMemcpyAsync(ctx->pinned, serr, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    uint32_t raised = 0;
    memcpy(&raised, ctx->pinned, 4);
    CK(cudaMemsetAsync(serr, 0, 4, s));
    if (raised) return fail(ctx, SWGS_ETIMEOUT, "the sort's look-back wait ran out (expected)");
    return SWGS_OK;
}

swgs_status swgs_profile_enable(swgs_ctx* ctx, int32_t on) {
    if (!ctx) return SWGS_EINVAL;
    ctx->prof = on != 0;
    return SWGS_OK;
}

swgs_status swgs_profile_read(swgs_ctx* ctx, swgs_profile* out, int32_t reset) {
    if (!ctx || !out) return SWGS_EINVAL;
    for (const ProfEvent& e : ctx->prof_pending) {
        CK(cudaEventSynchronize(e.b));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e.a, e.b));
        ctx->prof_ms[e.stage] += ms;
        ctx->prof_calls[e.stage] += 1;
        ctx->prof_free.push_back(e.a);
        ctx->prof_free.push_back(e.b);
    }
    ctx->prof_pending.clear();
    for (int i = 0; i < SWGS_NUM_STAGES; ++i) {
        out->ms[i] = ctx->prof_ms[i];
        out->calls[i] = ctx->prof_calls[i];
    }
    if (reset) {
        for (int i = 0; i < SWGS_NUM_STAGES; ++i) { ctx->prof_ms[i] = 0.0; ctx->prof_calls[i] = 0; }
    }
    return SWGS_OK;
}

int64_t swgs_kernel_launches(void) { return (int64_t)g_kernel_launches.load(); }

}  // extern "C"
