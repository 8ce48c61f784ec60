/*
 * swgs.h -- C ABI of libswgs, a B300 (sm_103a) implementation of the hot path
 * of SwinGS (arXiv 2409.07759): differentiable tile-based splatting of the
 * frame-t active set, the SGLD noise / relocation step, and per-frame slice
 * replacement.
 *
 * Conventions shared by every entry point:
 *  - All Gaussian, image and gradient buffers are caller-owned DEVICE memory
 *    unless an argument says "host". The library never frees them.
 *  - Scratch memory is obtained only through the alloc/free callbacks given to
 *    swgs_create (or cudaMallocAsync/cudaFreeAsync when they are NULL) and is
 *    cached inside the context between calls.
 *  - Work is enqueued on the CUDA stream passed as `stream` (a cudaStream_t,
 *    NULL = legacy default stream). A context must be used from one stream at a
 *    time; use one context per stream for concurrent work.
 *  - Every call returns a swgs_status. On failure swgs_last_error(ctx) gives a
 *    description. No entry point aborts, asserts or traps on the device.
 *  - Inputs must be finite; quaternions need not be normalised.
 */
#ifndef SWGS_H
#define SWGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SWGS_ABI_VERSION 5

typedef enum swgs_status {
    SWGS_OK = 0,
    SWGS_EINVAL = 1,   /* bad shape, pointer or argument */
    SWGS_ENOMEM = 2,   /* the allocator failed */
    SWGS_ECUDA = 3,    /* a CUDA runtime call failed */
    SWGS_ETIMEOUT = 4, /* a bounded device wait expired */
    SWGS_EDEVICE = 5,  /* a kernel raised the device error word, or a batch
                          outgrew the capacities of deferred sizing */
    SWGS_ESTATE = 6,   /* stale or mismatched saved state / slice */
    SWGS_EPENDING = 7  /* deferred sizing: the call's result has not arrived yet */
} swgs_status;

/* Scratch allocator: returns device memory usable on `stream` (NULL on
 * failure), aligned to 256 bytes as cudaMalloc's is (the kernels read their
 * scratch with 16-byte vector loads; a pointer aligned less is freed and the
 * call fails with SWGS_ENOMEM). free receives the same pointer and size. */
typedef void *(*swgs_alloc_fn)(void *user, size_t bytes, void *stream);
typedef void (*swgs_free_fn)(void *user, void *ptr, size_t bytes, void *stream);

/* Renderer configuration (the paper leaves the renderer to 3DGS [13]; these
 * are the launch shapes the autotuner chooses among). */
typedef struct swgs_config {
    int32_t tile_w, tile_h;  /* 8x8, 16x16 or 32x8 pixels per tile */
    int32_t batch;           /* Gaussians staged in shared memory per block step:
                                32, 64, 128 or 256 */
    float near_plane;        /* camera-space z below which Gaussians are culled */
    int32_t blocks_per_sm;   /* persistent blend grid = SMs x this; 0 = auto */
    int32_t count_pairs;     /* 1: count evaluated (pixel, Gaussian) pairs */
    int32_t pixels_per_thread; /* forward blend pixels per thread: 1, 2 or 4 (not 4 with 8x8) */
    int32_t bwd_pixels_per_thread; /* reverse blend: 1, 2, 4 or 8 (16x16, 32x8: up to 8;
                                      8x8: up to 2); 0 = pixels_per_thread */
    int32_t bwd_batch;       /* reverse blend staging batch; 0 = batch */
    int32_t sort_single_pass; /* 1: each radix digit pass is one kernel (decoupled
                                 look-back; inputs below 2^30 keys); 0: three
                                 kernels per pass (histogram, scan, scatter).
                                 Same sorted order either way. */
    int32_t deferred_sizing;  /* 0: a forward reads its active and key counts back
                                 (two stream synchronisations per batch) and sizes
                                 its buffers exactly. 1: after a context's first
                                 forward, buffers are sized from capacities learned
                                 on earlier calls (1/8 headroom) and the counts
                                 stay on the device: no synchronisation. A batch
                                 that outgrows them renders background, makes this
                                 context's next swgs_sgld_step do nothing, and is
                                 reported by swgs_saved_status (SWGS_EDEVICE: render
                                 again; the capacities have grown). Needs
                                 sort_single_pass = 1. */
} swgs_config;

/*
 * Gaussian state, slot-major structure of arrays, all device pointers
 * (Sec. 2.1 Eq. 1-2 attributes; Sec. 4.2 lifespans):
 *   means[N*3], log_scales[N*3] (scale = exp), quats[N*4] (w,x,y,z,
 *   unnormalised), opacity_logits[N] (opacity = sigmoid), sh[N*K*3]
 *   (K = (sh_degree+1)^2 coefficients, each an rgb triple),
 *   start[N], expire[N], birth[N] (int32 frames; a slot renders at frame t iff
 *   start <= t < expire -- Alg. 1 and Alg. 2 filters),
 *   frozen[N] (uint8, 1 = matured: rendered, never receives a gradient, noise
 *   or relocation -- Alg. 1 'matured').
 * For gradient buffers only the five float arrays are used.
 */
typedef struct swgs_gaussians {
    float *means;
    float *log_scales;
    float *quats;
    float *opacity_logits;
    float *sh;
    int32_t *start;
    int32_t *expire;
    int32_t *birth;
    uint8_t *frozen;
    int64_t capacity;
    int32_t sh_degree; /* 0..3 (the paper trains with 1, Sec. 8.1) */
} swgs_gaussians;

/* Pinhole view, OpenCV axes (x right, y down, z forward): p_cam = R p + t
 * with R row-major; pixel (i, j) is sampled at (i + 0.5, j + 0.5) where the
 * projection is u = fx x/z + cx, v = fy y/z + cy. `frame` selects the active
 * set this view renders (Alg. 1 sample_frame_between / Alg. 2 frame). */
typedef struct swgs_view {
    int32_t width, height;
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    int32_t frame;
} swgs_view;

typedef struct swgs_ctx swgs_ctx;
typedef struct swgs_saved swgs_saved;

/* Fills cfg with 16x16 tiles; forward batch 64 with 4 pixels per thread;
 * reverse blend batch 64 with 8 pixels per thread; near plane 0.2; auto grid;
 * single-pass sort. */
swgs_status swgs_default_config(swgs_config *cfg);

/* Creates a context on the current CUDA device. alloc/free may be NULL. */
swgs_status swgs_create(const swgs_config *cfg, swgs_alloc_fn alloc, swgs_free_fn free_fn,
                        void *user, swgs_ctx **out);

/* Releases every scratch buffer and saved state of the context. */
void swgs_destroy(swgs_ctx *ctx);

/* Text of the last error of this context ("" if none). Valid until the next call. */
const char *swgs_last_error(const swgs_ctx *ctx);

/* Library ABI version (SWGS_ABI_VERSION). */
int32_t swgs_abi_version(void);

/*
 * Active-set compaction (Sec. 4.2; Alg. 1 gs.filter / Alg. 2 buffer.filter):
 * writes the slots i with start[i] <= frame < expire[i], ascending, to
 * out_ids[0..count) (device, capacity n) and count to *out_count (device
 * int32). start/expire: device int32[n].
 */
swgs_status swgs_active_ids(swgs_ctx *ctx, const int32_t *start, const int32_t *expire, int64_t n,
                            int32_t frame, int32_t *out_ids, int32_t *out_count, void *stream);

/*
 * Allocation-free variant of swgs_active_ids, for callers that cannot let a
 * library allocate device memory: processes whose device memory belongs to one
 * allocator or budget (an engine's pool, a memory-capped server), where an
 * extra cudaMalloc would break the accounting, and latency-critical threads
 * that cannot afford cudaMalloc's device-wide synchronisation. The paper has no
 * counterpart; this is a deployment convenience.
 *
 * Same arguments and result as swgs_active_ids, but no context: its scratch
 * (about 66 KB) is a fixed array compiled into the library, which every GPU
 * that loads the library holds until the process exits. Every call looks up
 * that array's device address in the current context (cudaGetSymbolAddress,
 * which allocates nothing), so the first call on a device may load the
 * library's module there: make a first call before any stream capture. It
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *   - n must be at most SWGS_NOALLOC_MAX_SLOTS; larger n returns SWGS_EINVAL
 *     and enqueues nothing.
 *   - All calls on a device share the one array: calls whose work overlaps on
 *     the GPU (different streams, not ordered by events) race and give wrong
 *     results. Calls ordered on one stream are safe; nothing left in the
 *     array by a previous call is read.
 */
#define SWGS_NOALLOC_MAX_SLOTS (1 << 24)
swgs_status swgs_active_ids_noalloc(const int32_t *start, const int32_t *expire, int64_t n,
                                    int32_t frame, int32_t *out_ids, int32_t *out_count,
                                    void *stream);

/*
 * Per-frame slice replacement (Alg. 2 update_thread, Alg. 1 mature rewrite):
 * overwrites slots [first, first+count) of dst with src's slots [0, count):
 * every attribute, the three lifespan arrays and frozen. src lives in pinned
 * host memory when src_on_host = 1 (copied by DMA), else on the device
 * (copied by a kernel). Both must have the same sh_degree; dst must hold
 * first+count slots. Renders enqueued earlier on the same stream see the old
 * slice; later ones the new.
 */
swgs_status swgs_frame_update(swgs_ctx *ctx, const swgs_gaussians *dst, int64_t first,
                              int64_t count, const swgs_gaussians *src, int32_t src_on_host,
                              void *stream);

/*
 * Maturation of Alg. 1 (procedure mature, Sec. 4.2) on the device. buf holds
 * the optimisable Gaussians (gs) in slots [0, num_gs) and the ring of the last
 * num_gs matured rows in slots [num_gs, 2 num_gs) (frozen = 1; ring slots never
 * written yet keep an empty lifespan, start = expire). Requires
 * buf->capacity >= 2 num_gs, num_gs a multiple of swin_size, and the birth and
 * frozen arrays. In the algorithm's order:
 *  1. mature_idx = the gs slots with start < st, ascending;
 *  2. stream.write: those rows as they are (every array, lifespans included)
 *     go to rows 0..n-1 of `snapshot` (optional, same layout, capacity >=
 *     num_gs; pinned host memory when snapshot_on_host = 1, else device; host
 *     rows are complete when the stream reaches this point);
 *  3. matured += the rows, keeping the last num_gs: row j goes to ring slot
 *     num_gs + (*head + j) mod num_gs with frozen = 1, and *head advances by n
 *     (mod num_gs; the ring read from *head is the matured list oldest first);
 *  4. the gs rows start their next lifespan: birth = expire, start = expire,
 *     expire = start + swin_size.
 * *n_out receives n = |mature_idx|. The call synchronises the stream once (to
 * read n). SWGS_EINVAL: bad buffer, head, sizes or snapshot.
 */
swgs_status swgs_mature(swgs_ctx *ctx, const swgs_gaussians *buf, int64_t num_gs, int32_t st,
                        int32_t swin_size, int64_t *head, const swgs_gaussians *snapshot,
                        int32_t snapshot_on_host, int64_t *n_out, void *stream);

/*
 * Streamed-slice codec: the attribute quantisation of Table 6 as the paper
 * practises it (Sec. 5.6.2: means and log-scales fp16, rotation uint8,
 * opacity uint8, only the DC of the SH kept, at full precision) and the ABR
 * tail drop of Sec. 5.5 (keep the `keep` highest-opacity Gaussians of the
 * slice, ties by slot; the others travel as nothing and decode as empty).
 *
 * Packet layout (all little-endian): int32 header[8] = {magic 0x43574753,
 * version 1, count, keep, sh_degree, birth, start, expire}, then sections each
 * starting on a 16-byte boundary: slot index uint32[keep] (only when keep <
 * count), means fp16[keep][3], log_scales fp16[keep][3], rotation
 * uint8[keep][4] = rint((q_c / |q| + 1) * 127.5), opacity uint8[keep] =
 * rint(255 sigmoid(logit)) (FP32, the key-mode exp), DC float[keep][3]. Rows
 * are in slot order; the slice's lifespan (shared by its rows, Sec. 4.2.1)
 * is taken from its row 0. 29 bytes per kept Gaussian (+4 with the index).
 */
size_t swgs_slice_packet_bytes(int64_t count, int64_t keep); /* 0 if keep > count */

/* Encode rows [0, count) of src (device) into `out` (device, or pinned host
 * when out_on_host = 1; complete when the stream reaches this point). */
swgs_status swgs_slice_encode(swgs_ctx *ctx, const swgs_gaussians *src, int64_t count,
                              int64_t keep, void *out, size_t out_capacity, int32_t out_on_host,
                              size_t *out_bytes, void *stream);

/* Decode a packet into slots [first, first + count) of dst (Alg. 2's slice
 * replacement): kept rows get their attributes (q_c = k * 2/255 - 1, logit =
 * ln(o / (1 - o)) with o = clamp(k, 0.5, 254.5) / 255, DC and zero higher SH
 * bands), the slice's lifespan and frozen = 1; dropped rows are emptied (zero
 * attributes, start = expire: never active). A device packet costs one stream
 * synchronisation (to read its header). SWGS_EINVAL: bad or truncated packet,
 * SH degree mismatch, slots outside dst. */
swgs_status swgs_slice_decode(swgs_ctx *ctx, const void *packet, size_t bytes,
                              int32_t packet_on_host, const swgs_gaussians *dst, int64_t first,
                              void *stream);

/*
 * Alg. 1 schedule_expire, which the paper leaves undefined (reading): after the
 * first window, slice k of the gs slots (slice_size = num_gs / swin_size)
 * gets expire = k for k >= 1 and slice 0 expire = swin_size, so that exactly
 * one slice matures per frame and each streamed slice lands, by Alg. 2's
 * birth mod swin_size rule, on the slice whose data just expired. Same buffer
 * requirements as swgs_mature.
 */
swgs_status swgs_schedule_expire(swgs_ctx *ctx, const swgs_gaussians *buf, int64_t num_gs,
                                 int32_t swin_size, void *stream);

/*
 * Forward render (Sec. 2.1 Eq. 3 over the frame-t active set) of n_views views,
 * each at its own frame.
 *   bg: host float[3] background; out_rgb[v]: device float[3*H*W] planar;
 *   out_T[v] (optional, may be NULL or hold NULLs): device float[H*W] final
 *   transmittance.
 *   batched = 1: every stage runs once over all views; the blend is one
 *   persistent launch over all (view, tile) work items. Views are taken in
 *   consecutive batches of at most 2^16 super tiles (a super tile is 4x4 tiles,
 *   2x8 for 32x8 tiles); one batch holds every view of typical calls.
 *   batched = 0: the plain method, each view through its own launches.
 *   saved: if non-NULL, receives the state the backward pass needs (final T,
 *   last-contributor index, sorted lists, 2D records); release it with
 *   swgs_saved_release. If NULL the call only renders.
 * The call synchronises the stream twice per batch (to size the record and key
 * buffers). SWGS_EINVAL: bad sizes or pointers, more than the view limit, or a
 * single view with more than 2^16 super tiles (with 8x8 tiles, views beyond
 * about 8192 x 8192 pixels).
 */
swgs_status swgs_render_fwd(swgs_ctx *ctx, const swgs_gaussians *g, int32_t n_views,
                            const swgs_view *views, const float *bg, float *const *out_rgb,
                            float *const *out_T, int32_t batched, swgs_saved **saved,
                            void *stream);

/*
 * swgs_render_fwd writing 8-bit images instead of float ones, for delivery to
 * a viewer: out_rgb8[v] is device uint8 [H,W,3] (interleaved RGB), each value
 * round(255 clamp(c, 0, 1)) of the channel c that swgs_render_fwd writes (ties
 * to even). out_T, saved, batched and errors as in swgs_render_fwd; a saved
 * state serves swgs_render_bwd as well.
 */
swgs_status swgs_render_fwd_rgb8(swgs_ctx *ctx, const swgs_gaussians *g, int32_t n_views,
                                 const swgs_view *views, const float *bg,
                                 uint8_t *const *out_rgb8, float *const *out_T, int32_t batched,
                                 swgs_saved **saved, void *stream);

/*
 * swgs_render_fwd fused with the L1 term of Alg. 1 loss_func (same as
 * swgs_loss_l1 on the rendered images, without a separate pass over them):
 * besides out_rgb it reads target[v] (device float[3*H*W]), writes
 * dL_drgb[v] = sign(rgb - target)/(3*H*W*V) and overwrites *loss (device
 * float) with the mean over views of mean |rgb - target|. out_rgb may be NULL:
 * no image is written (a training step needs only the loss and dL_drgb).
 */
swgs_status swgs_render_fwd_l1(swgs_ctx *ctx, const swgs_gaussians *g, int32_t n_views,
                               const swgs_view *views, const float *bg, float *const *out_rgb,
                               float *const *out_T, const float *const *target,
                               float *const *dL_drgb, float *loss, int32_t batched,
                               swgs_saved **saved, void *stream);

/*
 * swgs_render_fwd_l1 with 8-bit targets (the form video frames arrive in):
 * target[v] is device uint8_t[3*H*W] planar, read as k * (1/255) in FP32
 * (within one ulp of k / 255). Same outputs, errors and ownership otherwise.
 */
swgs_status swgs_render_fwd_l1_u8(swgs_ctx *ctx, const swgs_gaussians *g, int32_t n_views,
                                  const swgs_view *views, const float *bg,
                                  float *const *out_rgb, float *const *out_T,
                                  const uint8_t *const *target, float *const *dL_drgb,
                                  float *loss, int32_t batched, swgs_saved **saved,
                                  void *stream);

/*
 * Backward of swgs_render_fwd (Alg. 1 loss.backward): given dL/drgb[v]
 * (device float[3*H*W] planar, same views as the saved forward), ACCUMULATES
 * into grads (device arrays with g's layout: means, log_scales, quats,
 * opacity_logits, sh) the gradient with respect to the raw parameters. Frozen
 * slots receive nothing. The blend is recomputed back to front from the saved
 * final transmittance and last-contributor index. g must be unchanged since
 * the forward.
 */
swgs_status swgs_render_bwd(swgs_ctx *ctx, const swgs_gaussians *g, const swgs_saved *saved,
                            const float *const *dL_drgb, const swgs_gaussians *grads,
                            void *stream);

/*
 * Regularisers of Alg. 1 reg(active_gs) (Sec. 4.4, weights in Sec. 8.1; the
 * terms of [14]): for a loss that is the mean over the forward's views, view
 * v (frame f_v) adds
 *   opacity_reg * mean_{i active at f_v} sigmoid(logit_i)
 *   + scale_reg * mean_{i active at f_v, c} exp(log_scale_ic) / V.
 * Matured (frozen) Gaussians count in the means but get no gradient.
 * n_views_total: V (0 = the forward's number of views).
 */
typedef struct swgs_reg_params {
    float opacity_reg, scale_reg;
    int32_t n_views_total;
} swgs_reg_params;

/*
 * swgs_render_bwd plus the gradient of the regularisers (reg may be NULL: no
 * regulariser). If loss (device float) is non-NULL the regulariser value is
 * ADDED to it.
 */
swgs_status swgs_render_bwd_reg(swgs_ctx *ctx, const swgs_gaussians *g, const swgs_saved *saved,
                                const float *const *dL_drgb, const swgs_gaussians *grads,
                                const swgs_reg_params *reg, float *loss, void *stream);

/* Returns a saved state to the context's pool (stream-ordered reuse). */
swgs_status swgs_saved_release(swgs_ctx *ctx, swgs_saved *saved);

typedef struct swgs_saved_info {
    int32_t n_views;
    int32_t n_batches;     /* 1 when batched, n_views for the plain path */
    int64_t n_records;     /* (view, active Gaussian) pairs */
    int64_t n_keys;        /* (Gaussian, tile) instances */
    int64_t n_tiles;       /* tiles over all views */
    int64_t n_pixels;      /* pixels over all views */
    int64_t pairs;         /* evaluated (pixel, Gaussian) pairs (count_pairs = 1) */
    int64_t n_sort_keys;   /* (super tile, Gaussian) keys sorted to build the tile lists */
    int64_t n_supers;      /* super tiles over all views */
    /* Device bytes the forward's data takes at the sizes it needed (the saved
     * state and the context scratch it used; the caller's images excluded), and
     * the part of it that grows with the records (the active-set ids and the
     * per-record arrays). A server can size its admission from these. */
    int64_t device_bytes;
    int64_t record_bytes;
} swgs_saved_info;

swgs_status swgs_saved_query(swgs_ctx *ctx, const swgs_saved *saved, swgs_saved_info *info);

/* Outcome of the forward that made `saved`. With deferred sizing the forward
 * returned before its counts were known: wait = 1 blocks until its batches'
 * totals have arrived, wait = 0 returns SWGS_EPENDING if they have not.
 * SWGS_OK; SWGS_EDEVICE: a batch outgrew the capacities (its images are
 * background, its backward does nothing): render the views again -- the
 * context's capacities have grown to what it needed; SWGS_ETIMEOUT: a sort's
 * look-back wait ran out. Without deferred sizing the forward already
 * returned its status and this returns SWGS_OK. swgs_saved_query,
 * swgs_saved_count and swgs_saved_export wait the same way. */
swgs_status swgs_saved_status(swgs_ctx *ctx, const swgs_saved *saved, int32_t wait);

/* Intermediate arrays of a saved forward, copied to `dst` (device or host,
 * `bytes` must match). Records, keys and tiles are concatenated over batches
 * in view order; see the constants for element types. */
enum {
    SWGS_EXPORT_RECORD_SLOT = 0,  /* int32 per record: Gaussian slot */
    SWGS_EXPORT_RECORD_VIEW = 1,  /* int32 per record: view index */
    SWGS_EXPORT_RECORD_TILES = 2, /* int32 per record: tiles touched */
    SWGS_EXPORT_RECORD_DEPTH = 3, /* float per record: camera depth (key) */
    SWGS_EXPORT_RECORD_RECT = 4,  /* int32 x4 per record: tx0, tx1, ty0, ty1 */
    SWGS_EXPORT_SORTED_SLOT = 5,  /* int32 per key: slot, per-tile depth order */
    SWGS_EXPORT_TILE_RANGES = 6,  /* int32 x2 per tile: [begin, end) into keys */
    SWGS_EXPORT_LAST = 7,         /* int32 per pixel: 1 + tile-list position */
    SWGS_EXPORT_FINAL_T = 8,      /* float per pixel */
    SWGS_EXPORT_GRAD2D = 9,       /* float x12 per record after a backward:
                                     du, dv, dA, dB, dC, dopacity, dr, dg, db */
    SWGS_EXPORT_RECORD_2D = 10    /* float x12 per record: u, v, opacity, depth,
                                     A, B, C, -, r, g, b, - */
};
swgs_status swgs_saved_export(swgs_ctx *ctx, const swgs_saved *saved, int32_t what, void *dst,
                              size_t bytes, void *stream);
/* Element count of an export (records, keys, tiles or pixels). */
swgs_status swgs_saved_count(swgs_ctx *ctx, const swgs_saved *saved, int32_t what,
                             int64_t *count);

/*
 * L1 photometric term of Alg. 1 loss_func: loss = mean over views of
 * mean |rgb - target| over 3*H*W; dL_drgb[v] = sign(rgb - target)/(3*H*W*V)
 * (sign(0) = 0). rgb, target, dL_drgb: device float[3*H*W] per view; loss:
 * device float[1], overwritten.
 */
swgs_status swgs_loss_l1(swgs_ctx *ctx, int32_t n_views, const swgs_view *views,
                         const float *const *rgb, const float *const *target,
                         float *const *dL_drgb, float *loss, void *stream);

/* Optimiser / SGLD / relocation hyper-parameters (Sec. 4.4, 8.1; [14]). */
typedef struct swgs_sgld_params {
    float lr_means, lr_log_scales, lr_quats, lr_logits, lr_sh_dc, lr_sh_rest;
    float beta1, beta2, eps;   /* Adam */
    float noise_lr;            /* 5e4 in Sec. 8.1 */
    float noise_k, noise_t;    /* noise gate sigmoid(-k (opacity - t)) */
    int32_t adam;              /* 1: Adam step from grads before the noise */
    int32_t relocate;          /* 1: relocate dead Gaussians after the noise */
    int32_t max_n;             /* cap on copies per target in the formulas */
    /* Sec. 4.5.1 (formula not given; reading): the means gradient of slot i is
     * scaled by mean_grad_decay^(k-1) before the Adam step, k = max(1,
     * window_start - start_i + swin_size) the windows that have trained the
     * slot's current lifespan. Off when mean_grad_decay == 1 or swin_size <= 0. */
    float mean_grad_decay;
    int32_t window_start;
    int32_t swin_size;
    /* 1 (grads given): after the Adam step has read them, the gradients of the
     * eligible slots are set to zero, so the next backward starts its sums from
     * zero without a clearing pass. Gradients of other slots are left as they
     * are (a backward over frames outside `frames` writes some there).
     * 0: grads is only read. */
    int32_t clear_grads;
} swgs_sgld_params;

/* Adam moments, device arrays shaped like the five float parameter arrays. */
typedef struct swgs_adam_state {
    float *m_means, *v_means, *m_log_scales, *v_log_scales, *m_quats, *v_quats,
          *m_logits, *v_logits, *m_sh, *v_sh;
} swgs_adam_state;

/*
 * Alg. 1 steps after the backward, on the Gaussians eligible at this step
 * (active at any of frames[0..n_frames) -- host int32 -- and not frozen):
 *   1. if params->adam: one bias-corrected Adam step (step count step+1) from
 *      grads (may be NULL otherwise);
 *   2. SGLD noise mu += lr_means * noise_lr * sigmoid(-k (o - t)) Sigma eta,
 *      eta ~ N(0, I) drawn from Philox4x64-10 keyed by (seed, step, slot);
 *   3. if params->relocate: every dead (opacity <= 0.005) Gaussian copies an
 *      alive one sampled in proportion to opacity, and both take the opacity
 *      1 - (1 - o)^(1/N) and the rescaled scale of [14]; Adam moments of every
 *      touched slot are zeroed (adam may be NULL when no Adam is used).
 * targets: optional device int32[capacity]; receives for every slot the slot
 * it copied in step 3, or -1.
 * n_relocated: optional host pointer; if non-NULL the call synchronises and
 * stores the number of relocated slots.
 */
swgs_status swgs_sgld_step(swgs_ctx *ctx, const swgs_gaussians *g, const swgs_gaussians *grads,
                           const swgs_adam_state *adam, const int32_t *frames, int32_t n_frames,
                           const swgs_sgld_params *params, uint64_t seed, uint64_t step,
                           int32_t *targets, int64_t *n_relocated, void *stream);

/* Alg. 2: slot range [first, first+count) that the update for target_frame
 * overwrites: slice = target_frame mod swin_size, count = num_gs / swin_size. */
swgs_status swgs_slice_range(int64_t target_frame, int64_t swin_size, int64_t num_gs,
                             int64_t *first, int64_t *count);

/* ---- measurement (not part of the method) -------------------------------
 * With profiling on, every stage of every call records a pair of CUDA events
 * on the caller's stream; swgs_profile_read synchronises those events and
 * returns the summed device time per stage. */
enum {
    SWGS_STAGE_COMPACT = 0,      /* active-set compaction */
    SWGS_STAGE_PREPROCESS = 1,   /* projection + SH */
    SWGS_STAGE_DEPTH_SORT = 2,   /* record depth sort */
    SWGS_STAGE_KEY_SCAN = 3,     /* super tiles keyed per record, in depth order + scan */
    SWGS_STAGE_EMIT = 4,         /* (super tile, record) key emission */
    SWGS_STAGE_TILE_SORT = 5,    /* stable sort of the keys by super tile */
    SWGS_STAGE_RANGES = 6,       /* super-tile ranges + expansion into per-tile lists */
    SWGS_STAGE_BLEND_FWD = 7,    /* forward blend (one kernel) */
    SWGS_STAGE_BLEND_BWD = 8,    /* reverse blend (one kernel) */
    SWGS_STAGE_PREPROCESS_BWD = 9,
    SWGS_STAGE_LOSS = 10,
    SWGS_STAGE_SGLD = 11,        /* Adam + noise (one kernel) */
    SWGS_STAGE_RELOCATE = 12,
    SWGS_STAGE_UPDATE = 13,      /* slice replacement */
    SWGS_NUM_STAGES = 14
};
typedef struct swgs_profile {
    double ms[SWGS_NUM_STAGES];      /* summed device milliseconds */
    int64_t calls[SWGS_NUM_STAGES];  /* stage executions */
} swgs_profile;
swgs_status swgs_profile_enable(swgs_ctx *ctx, int32_t on);
/* Synchronises the recorded events; reset = 1 clears the sums afterwards. */
swgs_status swgs_profile_read(swgs_ctx *ctx, swgs_profile *out, int32_t reset);
/* Kernels launched by this library in this process so far (all contexts). */
int64_t swgs_kernel_launches(void);

/* Failure-path check of the radix sort's bounded look-back wait (no paper
 * counterpart). Runs one digit pass over two 4096-key tiles of scratch data
 * with the tile counter started at 1: the one block takes tile 1, and tile 0,
 * which no block takes, never publishes its counts, so the block's look-back
 * wait runs out after its iteration limit (about a second) and
 * the pass finishes with its output wrong. Every access stays inside the
 * scratch buffers. Synchronises `stream`; returns SWGS_ETIMEOUT when the
 * sort's error word was raised (the expected result), SWGS_OK if it was not.
 * The context stays usable. */
swgs_status swgs_selftest_sort_timeout(swgs_ctx *ctx, void *stream);

/*
 * Data-parallel gradient exchange (no paper counterpart: the paper trains on
 * one GPU; this serves a window step sharded by views over several GPUs, each
 * holding a replica of the state). Only the eligible slots -- active at one of
 * `frames` (host int32[n_frames], at most 64) and not frozen, the slots the
 * Adam/noise step of swgs_sgld_step reads gradients of -- can carry a nonzero
 * gradient, and every replica finds the same ones, so the ranks sum those rows
 * only.
 *
 * swgs_grad_pack writes the eligible slots, ascending, to ids (device int32,
 * capacity g->capacity), their number to *count (device int64) and their
 * gradient rows to packed (device float, capacity g->capacity x R), row k =
 * the gradients of slot ids[k]: means 3, log_scales 3, quats 4, opacity logit
 * 1, sh 3K, so R = 11 + 3K with K = (sh_degree + 1)^2, each value multiplied
 * by `scale` (a rank's share of the window's views). grads has the state's
 * capacity and SH degree. The caller reads the count, sums packed[0, count x R)
 * over the ranks, and calls
 * swgs_grad_unpack, which writes row k back to slot ids[k] of grads for
 * k < *count (other slots are left as they are). Both are asynchronous on
 * `stream`; buffers are caller-owned. SWGS_EINVAL for bad arguments.
 */
swgs_status swgs_grad_pack(swgs_ctx *ctx, const swgs_gaussians *g, const swgs_gaussians *grads,
                           const int32_t *frames, int32_t n_frames, float scale, int32_t *ids,
                           int64_t *count, float *packed, void *stream);
swgs_status swgs_grad_unpack(swgs_ctx *ctx, const swgs_gaussians *grads, const int32_t *ids,
                             const int64_t *count, const float *packed, void *stream);

/* FP32-pipe throughput probe (no paper counterpart): the measured peak that
 * the blends' roofline is taken against. Launches `blocks` blocks of 256
 * threads on `stream`; every thread runs 8 independent multiply-add chains
 * for `iters` iterations, as scalar FP32 FMAs (packed = 0) or packed FP32x2
 * FMAs (packed = 1, two FMAs per instruction), and writes its chains' sum to
 * sink[thread] (device float[blocks * 256], caller-owned). *flops receives the
 * launch's floating-point operations (an FMA counts 2). The caller times the
 * launch with events on `stream`. SWGS_EINVAL for bad arguments. */
swgs_status swgs_fp32_peak_launch(int32_t packed, int32_t blocks, int32_t iters, float *sink,
                                  double *flops, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SWGS_H */
