/*
 * gs.h -- C ABI of libgs, a GB300 (sm_103a) differentiable tile-based
 * Gaussian-splat rasterizer for isosurface 3D Gaussian Splatting.
 *
 * The paper (Sec. II) trains 3D Gaussian Splatting per spatial partition
 * ("Data Partitioning", "Parallel Training") and merges the splats of all
 * partitions for the final render ("Global Reconstruction"); the masks of
 * "Image Rendering and Masking" restrict the loss to a partition's pixels.
 * It does not restate the rasterizer itself, which is the standard 3D-GS
 * one; the steps below follow that definition with the constants fixed here.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every pointer argument is a DEVICE pointer owned by the caller unless
 *    its comment says "host".  The library never allocates or frees memory;
 *    calls that need scratch take a caller-provided workspace whose size is
 *    given by the matching *_workspace_size() query.
 *  - Every call enqueues work on `stream` and returns without synchronising.
 *    Host-side argument checks happen before anything is enqueued: on a bad
 *    argument the call returns GS_ERR_INVALID and enqueues nothing.
 *  - Errors found on the device (instance capacity overflow, non-finite
 *    values) are OR-ed into the caller's device word `d_status` (bits of
 *    gs_status).  gs_status_read() synchronises the stream and returns it.
 *  - A launch failure reported by the CUDA runtime returns GS_ERR_CUDA.
 *  - All floating point is IEEE fp32 except the MLP GEMM operands (bf16).
 *
 * Data layout
 * -----------
 *  Gaussian parameters: `params` is n_planes x N float4 ("planes"), plane p
 *  of Gaussian i at params + 4 * (p * N + i):
 *     plane 0  mean        (x, y, z, unused)
 *     plane 1  scale/op    (log sx, log sy, log sz, logit opacity)
 *     plane 2  rotation    (w, x, y, z), any non-zero norm
 *     plane 3+ SH          the 3 (d+1)^2 colour coefficients, coefficient-major
 *                          (k0.r k0.g k0.b k1.r ...), packed 4 per plane
 *  n_planes = gs_param_planes(sh_degree) = 3 + ceil(3 (d+1)^2 / 4).
 *  Gradients, Adam moments use the same layout.
 *
 *  Units: one "unit" is one (partition, view) pair.  Unit u renders the
 *  Gaussians [gauss_begin[u], gauss_begin[u] + gauss_count[u]) with camera
 *  cams[u]; its projected records occupy the contiguous range
 *  [proj_base[u], proj_base[u] + gauss_count[u]) with proj_base the exclusive
 *  prefix sum of gauss_count.  A single view of one scene is one unit
 *  covering all N Gaussians.  All units share one image size.
 *
 *  Images: img [U][3][H][W] fp32, final_T and n_contrib [U][H][W].
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* gs_stream_t; /* a cudaStream_t */

enum gs_status {
  GS_OK = 0,
  GS_ERR_INVALID = 1,   /* bad argument (host check; nothing enqueued) */
  GS_ERR_CAPACITY = 2,  /* more tile instances than the buffers hold; lists truncated */
  GS_ERR_TIMEOUT = 4,   /* a bounded wait expired */
  GS_ERR_NONFINITE = 8, /* a non-finite value was produced */
  GS_ERR_CUDA = 16      /* CUDA runtime error at launch */
};

/* Rasterizer constants (the 3D-GS definition; none is stated in the paper). */
#define GS_TILE 16             /* tile edge in pixels */
#define GS_MAX_UNITS 256       /* units per call */
#define GS_MAX_PARTS 64        /* partitions for the ghost filter */

/* Pinhole camera, world -> camera: X_cam = R X + t with viewmat = [R | t]
 * row-major 3x4.  Camera space: +x right, +y down, +z forward.  Pixel of a
 * camera-space point: (fx x/z + cx, fy y/z + cy); pixel (px, py) is centred at
 * integer coordinates.  tan_fov* = tan(fov/2); Gaussians with z <= znear are
 * culled.  96 bytes. */
typedef struct gs_camera {
  float viewmat[12];
  float fx, fy, cx, cy;
  float tan_fovx, tan_fovy;
  float campos[3];
  float znear;
  int32_t width, height;
} gs_camera;

/* Per (unit, Gaussian) projected records, indexed by projected index. */
typedef struct gs_proj {
  float* xy;        /* [P][4]  pixel-space mean as float pairs (x, y, x_lo,
                     y_lo): u = x + x_lo, v = y + y_lo with |lo| at most half
                     an ulp of the high part; both parts together carry the
                     position to ~2^-44 relative (float32 alone would carry
                     ~6e-5 px at u ~ 10^3, which moves alpha near the 1/255
                     edge of sub-pixel splats)                             */
  float* conic_op;  /* [P][4]  (A, B, C, opacity), conic = inverse 2D cov  */
  float* rgb;       /* [P][4]  (r, g, b, f) after SH, +0.5 and clamp at 0;
                     f: power below which alpha < 1/255 for certain      */
  float* depth;     /* [P]     camera-space z                              */
  int32_t* radius;  /* [P]     3-sigma radius in pixels, 0 = culled        */
  uint32_t* tiles;  /* [P]     number of 16x16 tiles the splat touches     */
} gs_proj;

/* Screen-space gradients (accumulated by gs_render_bwd / gs_blend_bwd).
 * fixed: NULL (float atomics: sums depend on the order in which warps add,
 * within float rounding), or [P][9] int64 scratch (deterministic mode): the
 * nine values per record (dx, dy, dA, dB, dC, d opacity, dr, dg, db)
 * accumulate as fixed point value x 2^40 (|value| clamped to 2^22, NaN adds
 * 0), whose integer sums do not depend on order, and are converted into
 * dxy / dconic_op / drgb at the end of the call: gradients are bitwise
 * reproducible. */
typedef struct gs_grad2d {
  float* dxy;       /* [P][2] */
  float* dconic_op; /* [P][4] (dA, dB, dC, d opacity) */
  float* drgb;      /* [P][4] */
  unsigned long long* fixed; /* [P][9] or NULL */
} gs_grad2d;

/* Blend schedule (all device buffers; see gs_bin_sort and the blend calls):
 * tile_order   [U * n_tiles]      blocks ordered by decreasing list length class
 * block_masks  [max_instances]    per sorted instance: bit 4 by + bx set iff the
 *                                 record's alpha >= 1/255 ellipse (a conservative
 *                                 box of it) reaches 4x4 pixel block (bx, by)
 * job_base     [U * n_tiles + 1]  exclusive prefix (in tile_order) of the number
 *                                 of chunks of each list; job_base[U n_tiles] = jobs
 * jobs         [2 * max_jobs]     (order position, chunk) of every chunk job; the
 *                                 last entry, which no job reaches, is the blend
 *                                 kernels' work counter (reset by each call)
 * checkpoints  [max_checkpoints][256][4]  per pixel, at every interior chunk
 *                                 boundary: T there and the colour composited
 *                                 behind it per unit T (r, g, b), written by
 *                                 the forward for the chunked backward
 * chunk_last   [max_checkpoints][256]     forward scratch (per pixel and
 *                                 chunk: last blended entry and stop flag, then
 *                                 the T in front of the chunk)
 * stop_queue   [8 * max_jobs + 1] forward scratch: the (chunk job, pixel block)
 *                                 units in which some pixel stops, for the
 *                                 forward's re-walk pass; the last entry counts
 *                                 them
 * chunk        entries per chunk (a multiple of 32); max_jobs >= U n_tiles +
 *              max_instances / chunk + 1, max_checkpoints >= max_instances /
 *              chunk + 1 (gs_schedule_sizes).
 * walk_whole_lists  0: the forward composites the chunks of a list in
 *              parallel and combines them (training views, whose pixels rarely
 *              stop early); 1: one warp per (list, pixel block) walks the whole
 *              list and stops at its last pixel's stop (opaque renders). */
typedef struct gs_schedule {
  uint32_t* tile_order;
  uint16_t* block_masks;
  uint32_t* job_base;
  uint32_t* jobs;
  float* checkpoints;
  uint32_t* chunk_last;
  uint32_t* stop_queue;
  int64_t max_jobs;
  int64_t max_checkpoints;
  int32_t chunk;
  int32_t walk_whole_lists;
} gs_schedule;

/* Unit table (host arrays, copied by value into the launch). */
typedef struct gs_units {
  int32_t n_units;               /* 1 .. GS_MAX_UNITS */
  const int64_t* gauss_begin;    /* host [n_units] */
  const int64_t* gauss_count;    /* host [n_units] */
} gs_units;

/* Optional ghost-cell filter of the merge (Sec. II, "Global Reconstruction"):
 * Gaussian i of partition k (part_offsets[k] <= i < part_offsets[k+1]) is
 * kept iff its mean lies in box k = (xmin, ymin, zmin, xmax, ymax, zmax),
 * lower bounds closed, upper bounds half-open unless closed_hi has bit a set
 * for axis a.  All host arrays. */
typedef struct gs_owned {
  int32_t n_parts;               /* 0 disables the filter, else 1 .. GS_MAX_PARTS */
  const int64_t* part_offsets;   /* host [n_parts + 1] */
  const float* boxes;            /* host [n_parts][6] */
  const int32_t* closed_hi;      /* host [n_parts], bits 0..2 */
} gs_owned;

/* Number of float4 planes per Gaussian for SH degree 0..3; -1 if invalid. */
int gs_param_planes(int sh_degree);

/* Synchronise `stream`, read the device status word, return it (and clear it
 * when `clear` is non-zero). */
int gs_status_read(int* d_status, int clear, gs_stream_t stream);

/* ---- a1: projection (EWA splatting; 3D-GS preprocess) --------------------
 * For every unit u and Gaussian i of that unit: camera-space mean t = R mu + t,
 * cull if t.z <= znear; Sigma3D = R(q) diag(e^{2 ls}) R(q)^T;
 * Sigma2D = J W Sigma3D W^T J^T + 0.3 I with J the perspective Jacobian at t
 * (x/z and y/z clamped to +-1.3 tan(fov/2) inside J); conic = Sigma2D^-1
 * (culled if det <= 0); radius = ceil(3 sqrt(lambda_max)) with
 * lambda_max = mid + sqrt(max(0.1, mid^2 - det)); tile rectangle
 * [floor((u - r)/16), floor((u + r + 15)/16)) clamped to the grid (likewise
 * y), culled if empty; rgb = sum_k Y_k(dir) c_k + 0.5 clamped at 0 with
 * dir = normalise(mu - campos) and real SH Y_k of degree <= 3 (Condon-Shortley
 * phase, m = -l..l); opacity = sigmoid(logit).
 * params: planes layout above (N Gaussians).  cams: device [n_units].
 * owned: may be NULL (no filter).  Writes every field of `proj` for visible
 * records and radius = tiles = 0 for culled ones. */
int gs_preprocess(const float* params, int64_t n_gauss, int sh_degree, const gs_units* units,
                  const gs_camera* cams, int width, int height, const gs_owned* owned,
                  const gs_proj* proj, int* d_status, gs_stream_t stream);

/* ---- a2: duplication + radix sort + tile ranges ---------------------------
 * Each visible record p of unit u has one instance per covered tile; each
 * (unit, tile) list holds the instances of its records ordered by
 * (float32 depth, record index p), i.e. the order of a stable sort by depth of
 * the records in index order.
 * ranges[u * n_tiles + tile] = [start, end) into sorted_vals.
 * sched (may be NULL): also fills the blend schedule: tile order (heaviest
 * lists first), per-instance block masks and the chunk jobs of every list
 * (see gs_schedule); the blend calls use it to skip records that cannot touch
 * a warp's pixels and to replay long lists in parallel chunks.
 * max_instances: capacity of the instance buffers; on overflow GS_ERR_CAPACITY
 * is set in d_status and the lists are truncated.  d_num_instances: device
 * uint32 receiving the instance count.  Workspace: gs_bin_sort_workspace_size. */
size_t gs_bin_sort_workspace_size(int64_t n_proj, int64_t max_instances);
int gs_bin_sort(const gs_proj* proj, const gs_units* units, int width, int height,
                int64_t max_instances, void* workspace, size_t workspace_bytes,
                uint32_t* sorted_vals, uint32_t* ranges, uint32_t* d_num_instances,
                const gs_schedule* sched, int* d_status, gs_stream_t stream);

/* How gs_bin_sort orders the lists: it compacts the visible records (tiles >
 * 0) in index order, sorts them by their float32 depth bits taken relative to
 * the nearest visible depth with stable LSD radix passes (four 8-bit digits;
 * a digit that every key shares is skipped on the device, so the top pass runs
 * only when the view's depths span more than a factor of ~4), emits each record's instances in that order as 32-bit keys
 * (block mask << 16 | unit << tile_bits | tile) and sorts those stably on the
 * unit | tile bits (one or two 8-bit passes): stability leaves every list in
 * (depth, record index) order.  It needs unit | tile ids of at most 16 bits
 * (one 4K unit: 15 bits; eight 1080p units: 16); for more it runs
 * gs_bin_sort_global.  On capacity overflow the nearest instances are kept.
 *
 * gs_bin_sort_global and gs_bin_sort_bucketed: the same lists, ranges,
 * instance count and schedule as gs_bin_sort (same arguments and workspace)
 * by the other two sort designs.  gs_bin_sort_global sorts the
 * (unit | tile | depth) keys of all instances with one global stable LSD radix
 * sort (5 passes of 9-bit digits over the 45 key bits of one 1080p unit); on
 * capacity overflow it keeps the first instances in record order.
 * gs_bin_sort_bucketed gathers the instances per (unit, tile) list with
 * atomics (arbitrary order inside a list), then sorts every list over its own
 * depth range: lists of up to 4096 instances in one CTA's shared memory, longer
 * ones cut into 4096-key jobs that run stable 9-bit passes together (as many
 * passes as the list's depth offsets have 9-bit digits); equal depths are then
 * ordered by record index.  Requires n_units * n_tiles <= 256 * 240 * 135
 * (else GS_ERR_INVALID).  In a list longer than 4096 instances, a run of
 * equal depths is put in record-index order by one thread (heapsort): fast for
 * the short runs of real scenes, slow (seconds) for runs of ~10^6 instances at
 * one depth in one tile. */
int gs_bin_sort_global(const gs_proj* proj, const gs_units* units, int width, int height,
                       int64_t max_instances, void* workspace, size_t workspace_bytes,
                       uint32_t* sorted_vals, uint32_t* ranges, uint32_t* d_num_instances,
                       const gs_schedule* sched, int* d_status, gs_stream_t stream);
int gs_bin_sort_bucketed(const gs_proj* proj, const gs_units* units, int width, int height,
                         int64_t max_instances, void* workspace, size_t workspace_bytes,
                         uint32_t* sorted_vals, uint32_t* ranges, uint32_t* d_num_instances,
                         const gs_schedule* sched, int* d_status, gs_stream_t stream);

/* Buffer sizes of a gs_schedule for n_units units of width x height and the
 * given instance capacity and chunk length: *max_jobs, *max_checkpoints. */
int gs_schedule_sizes(int n_units, int width, int height, int64_t max_instances, int chunk,
                      int64_t* max_jobs, int64_t* max_checkpoints);

/* ---- gs_bin_sort without a caller workspace ----------------------------
 * The paper has no counterpart: this is a deployment variant of gs_bin_sort
 * for callers that cannot allocate device memory (a host framework or plugin
 * that owns every allocation, or a program that must not allocate after
 * start-up).  It takes only the inputs and outputs of gs_bin_sort; its
 * scratch is a fixed array of GS_STATIC_SORT_SCRATCH_BYTES in the library's
 * own device memory, held on every GPU that loads the library until exit.
 * Limits: at most GS_STATIC_SORT_MAX_RECORDS records (sum of gauss_count)
 * and GS_STATIC_SORT_MAX_INSTANCES instances (the capacity: more set
 * GS_ERR_CAPACITY in d_status and truncate, as in gs_bin_sort); more records
 * return GS_ERR_INVALID with a message on stderr and enqueue nothing.
 * sorted_vals must hold GS_STATIC_SORT_MAX_INSTANCES entries.  All calls share
 * the array and it keeps the last call's contents (each call clears what must
 * start at zero): calls whose work overlaps on the GPU race.  The first call
 * on a device looks up the array's address with that device current, and a
 * call from a new context of the device (after cudaDeviceReset) looks it up
 * again; make those calls before any stream capture.  It builds no blend
 * schedule: the blend calls that read its lists take sched = NULL. */
#define GS_STATIC_SORT_MAX_RECORDS 131072
#define GS_STATIC_SORT_MAX_INSTANCES 524288
#define GS_STATIC_SORT_SCRATCH_BYTES 13631488
int gs_bin_sort_static(const gs_proj* proj, const gs_units* units, int width, int height,
                       uint32_t* sorted_vals, uint32_t* ranges, uint32_t* d_num_instances,
                       int* d_status, gs_stream_t stream);

/* ---- a3: front-to-back blend per 16x16 tile -------------------------------
 * For pixel (px, py) over its tile's list in order: d = xy - (px, py)
 * (evaluated as ((x - o) + x_lo) - (px - o) with o the tile's corner),
 * power = -(A dx^2 + C dy^2)/2 - B dx dy, skipped if > 0;
 * alpha = min(0.99, opacity e^power), skipped if < 1/255; if T (1 - alpha) <
 * 1e-4 the entry is not blended and the pixel stops; else C += alpha T rgb,
 * T *= 1 - alpha.  Finally C += T bg.  n_contrib = 1-based list position of
 * the last blended entry, final_T = T.  bg: host float[3].
 * variant: execution shape only (results are identical): each warp owns a
 * BW x 32/BW pixel block of the tile, BW = 8 (0), 16 (1) or 4 (2).
 * sched: NULL (one CTA per tile, natural order) or gs_bin_sort's schedule:
 * one-warp jobs per (tile, 8x4 block) in heaviest-first order that skip
 * records whose block mask misses their pixels, and write the per-pixel
 * checkpoints the chunked backward starts from; lists are composited in
 * parallel chunks of sched->chunk entries and combined in order.  Blended
 * entries, n_contrib and the stop decisions are those of the sequential walk;
 * image and final_T agree with it to float rounding. */
int gs_render_fwd(const gs_proj* proj, const uint32_t* sorted_vals, const uint32_t* ranges,
                  int n_units, int width, int height, const float* bg, float* img,
                  float* final_T, uint32_t* n_contrib, int variant, const gs_schedule* sched,
                  gs_stream_t stream);

/* Diagnostic work counters of the last gs_render_fwd (device uint64 [5]):
 * d_count[0] = blended (pixel, record) pairs (records before n_contrib whose
 * alpha reaches 1/255); d_count[1] = (pixel, list entry) pairs a sequential
 * front-to-back walk evaluates up to and including the entry that stops the
 * pixel; d_count[2] = sum of n_contrib over pixels (the entries the reverse
 * replay walks); d_count[3], d_count[4] = the pairs of d_count[1] and
 * d_count[2] whose block mask (block_masks of gs_bin_sort's schedule, in
 * sorted order; NULL gives 0) reaches the pixel's 4x4 block: the work of a
 * walk that skips records whose alpha box misses the pixel's block. */
int gs_blend_pairs(const gs_proj* proj, const uint32_t* sorted_vals, const uint32_t* ranges,
                   int n_units, int width, int height, const uint32_t* n_contrib,
                   const uint16_t* block_masks, unsigned long long* d_count, gs_stream_t stream);

/* ---- a4: masked photometric loss (mask: Sec. II, "Image Rendering and
 * Masking") ---------------------------------------------------------------
 * Per unit: L = (1 - lambda) L1 + lambda (1 - SSIM), with
 * L1 = sum_{p in M} sum_c |img - gt| / (3 |M|) and SSIM the mean over mask
 * pixels and channels of the SSIM map (11x11 Gaussian window, sigma 1.5,
 * zero-padded same convolution, C1 = 0.01^2, C2 = 0.03^2).  A unit with an
 * empty mask contributes 0.  The reported loss and its gradient are the mean
 * over units.  mask: uint8 [U][H][W] (non-zero = in).  d_loss: device float[1].
 * dL_dimg: [U][3][H][W], overwritten.  Workspace: gs_loss_workspace_size. */
size_t gs_loss_workspace_size(int n_units, int width, int height);
int gs_loss(const float* img, const float* gt, const uint8_t* mask, int n_units, int width,
            int height, float lambda_ssim, void* workspace, size_t workspace_bytes, float* d_loss,
            float* dL_dimg, gs_stream_t stream);

/* Background-opacity penalty, a variant of the masked loss (the paper's mask
 * removes the pixels a partition does not own, Sec. II "Image Rendering and
 * Masking"; this term also asks those pixels to stay transparent).  Per unit
 * with n_bg > 0 pixels outside the mask: P = lambda_bg sum_{p not in M}
 * (1 - final_T[p]) / n_bg (0 when n_bg = 0); the mean over units is ADDED to
 * *d_loss (call it after gs_loss).  dL_dT: [U][H][W] float, overwritten with
 * dP/dT_final (-lambda_bg / (U n_bg) outside the mask, 0 inside), the input of
 * the same name of gs_render_bwd / gs_blend_bwd.  lambda_bg >= 0, finite.
 * Workspace: gs_bg_penalty_workspace_size(n_units) bytes, 256-byte aligned. */
size_t gs_bg_penalty_workspace_size(int n_units);
int gs_bg_penalty(const float* final_T, const uint8_t* mask, int n_units, int width, int height,
                  float lambda_bg, void* workspace, size_t workspace_bytes, float* d_loss, float* dL_dT,
                  gs_stream_t stream);

/* ---- a5: backward ---------------------------------------------------------
 * Blend backward: per pixel, the tile list is replayed back to front from
 * n_contrib, recovering T_i = T_{i+1} / (1 - alpha_i) from final_T (no
 * per-pixel lists are stored); with S the colour behind entry i,
 * dL/drgb_i = alpha_i T_i g, dL/dalpha_i = T_i (rgb_i - S) . g, and, when
 * alpha was not clamped, dL/dopacity = e^power dL/dalpha, and dL/dpower =
 * alpha dL/dalpha onto the conic and the mean.  Per-Gaussian values are
 * reduced across each warp with shuffles, then across the tile in shared
 * memory, then added to `g2d` with one set of global atomics per (tile,
 * Gaussian).  g2d is zeroed by this call.
 * dL_dT: NULL, or dL/dT_final [U][H][W] of a loss term on the final
 * transmittance (gs_bg_penalty): since T_final = prod_k (1 - alpha_k) over
 * the blended entries, every blended entry i of the pixel adds
 * -dL_dT T_final / (1 - alpha_i) to dL/dalpha_i.
 * Projection backward: chain rule of a1 onto all parameters, summed over the
 * units containing each Gaussian; grads (planes layout) are overwritten.
 * variant, sched: as for gs_render_fwd.  With a schedule, each list is
 * replayed in chunks of sched->chunk entries by independent warps: a chunk
 * starts from the forward's checkpoint at its end (the transmittance there
 * and the colour composited behind it per unit transmittance).
 * img: the forward's image (required with a schedule). */
int gs_render_bwd(const float* params, int64_t n_gauss, int sh_degree, const gs_units* units,
                  const gs_camera* cams, const gs_proj* proj, const uint32_t* sorted_vals,
                  const uint32_t* ranges, int width, int height, const float* bg, const float* img,
                  const float* final_T, const uint32_t* n_contrib, const float* dL_dimg,
                  const float* dL_dT, const gs_grad2d* g2d, float* grads, int variant,
                  const gs_schedule* sched, gs_stream_t stream);

/* Blend backward only: g2d ([n_proj] records) is zeroed, then accumulated. */
int gs_blend_bwd(const gs_proj* proj, const uint32_t* sorted_vals, const uint32_t* ranges,
                 int n_units, int width, int height, const float* bg, const float* img,
                 const float* final_T, const uint32_t* n_contrib, const float* dL_dimg,
                 const float* dL_dT, const gs_grad2d* g2d,
                 int64_t n_proj, int variant, const gs_schedule* sched, gs_stream_t stream);

/* Projection backward only (grads overwritten). */
int gs_project_bwd(const float* params, int64_t n_gauss, int sh_degree, const gs_units* units,
                   const gs_camera* cams, const gs_proj* proj, const gs_grad2d* g2d,
                   float* grads, gs_stream_t stream);

/* ---- a6: Adam --------------------------------------------------------------
 * Textbook Adam with bias correction on the planes layout: t = *d_step + 1,
 * m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 * Learning rates per plane component: lr = lr_init * (lr_final / lr_init)^
 * (min(t, lr_steps) / lr_steps) (log-linear; constant when init == final);
 * lr_init, lr_final: host float[n_planes][4].  If zero_grad, g is set to 0.
 * d_step: device int32, read only (advance it with gs_step_advance).
 * A float4 of gradients holding a non-finite value sets GS_ERR_NONFINITE in
 * d_status (may be NULL) and its four parameters and moments keep their
 * values. */
int gs_adam_step(float* params, float* grads, float* m, float* v, int64_t n_gauss, int n_planes,
                 const float* lr_init, const float* lr_final, int32_t lr_steps, float beta1,
                 float beta2, float eps, const int32_t* d_step, int zero_grad, int* d_status,
                 gs_stream_t stream);

/* Projection backward fused with the Adam step (same arithmetic as
 * gs_project_bwd followed by gs_adam_step with zero_grad = 0): each
 * Gaussian's parameter gradient is formed in registers and applied at once.
 * grads may be NULL; otherwise it also receives the gradient.  A Gaussian
 * whose screen-space or parameter gradient holds a non-finite value sets
 * GS_ERR_NONFINITE in d_status (may be NULL) and keeps its parameters and
 * moments.  sparse != 0: a Gaussian whose gradient is zero in this step (no
 * view of the call reaches it with a non-zero screen-space gradient) keeps its
 * parameters and moments too, and costs no parameter or moment traffic (the
 * sparse Adam of 3D-GS updates only the Gaussians a view touches). */
int gs_project_bwd_adam(float* params, int64_t n_gauss, int sh_degree, const gs_units* units,
                        const gs_camera* cams, const gs_proj* proj, const gs_grad2d* g2d, float* m,
                        float* v, const float* lr_init, const float* lr_final, int32_t lr_steps,
                        float beta1, float beta2, float eps, const int32_t* d_step, float* grads,
                        int sparse, int* d_status, gs_stream_t stream);

/* gs_project_bwd_adam followed, in the same kernel, by a1 of the next step:
 * every Gaussian of a unit, as stored after its update (its old values where
 * it kept them), is projected for next_cams[unit] (device [n_units]; width x
 * height) and its record written over `proj` (position, conic and opacity,
 * colour, depth, radius, tiles: exactly what gs_preprocess with no owned
 * filter writes for those parameters and cameras).  The parameters are not
 * read again from memory.  Requires every Gaussian in at most one unit (else
 * GS_ERR_INVALID) and proj's record arrays.  A non-finite projection sets
 * GS_ERR_NONFINITE and culls the record, as gs_preprocess does. */
int gs_project_bwd_adam_next(float* params, int64_t n_gauss, int sh_degree, const gs_units* units,
                             const gs_camera* cams, const gs_proj* proj, const gs_grad2d* g2d, float* m,
                             float* v, const float* lr_init, const float* lr_final, int32_t lr_steps,
                             float beta1, float beta2, float eps, const int32_t* d_step, float* grads,
                             int sparse, const gs_camera* next_cams, int width, int height, int* d_status,
                             gs_stream_t stream);

/* *d_step += 1 on the device (keeps CUDA-graph replays advancing). */
int gs_step_advance(int32_t* d_step, gs_stream_t stream);

/* ---- a7: one batched training step of all (partition, view) units -------
 * The paper trains every data partition independently on its own views
 * (Sec. II, "Data Partitioning", "Parallel Training"); here the partitions
 * and views_per_step views of each are the units of one call.  Unit
 * u = (partition k = u / views_per_step, slot j = u % views_per_step) trains
 * partition k's Gaussians (units->gauss_begin / gauss_count) on view
 *     v = train_views[(t * views_per_step + j + k) mod n_train],  t = *d_step,
 * i.e. consecutive steps walk the training views and partitions are
 * staggered by one view.  The call enqueues, on `stream` and without any host
 * work that depends on t: gs_gather_views (camera, ground truth and mask of
 * each unit into the step buffers), gs_preprocess, gs_bin_sort,
 * gs_render_fwd, gs_loss, gs_blend_bwd, gs_project_bwd_adam (Adam step t + 1)
 * and gs_step_advance.  A CUDA graph that captures one call therefore
 * replays every later step.  All pointers are caller-owned; "host" marks host
 * arrays, every other pointer is device memory.  Device errors (capacity,
 * non-finite values) go to d_status as in the individual calls. */
typedef struct gs_train_batch_desc {
  float* params;                 /* [n_planes][n_gauss][4], updated in place */
  float* adam_m;                 /* Adam moments, same layout */
  float* adam_v;
  int64_t n_gauss;
  int32_t sh_degree;
  int32_t views_per_step;
  const gs_units* units;         /* host unit table, n_parts * views_per_step units */
  const gs_camera* cam_pool;     /* [n_views] cameras of the training set */
  const float* gt_pool;          /* [n_parts][n_views][3][H][W] each partition's ground truth */
  const uint8_t* mask_pool;      /* [n_parts][n_views][H][W] its background masks */
  const int32_t* train_views;    /* [n_train] view ids used for training */
  int32_t n_views;
  int32_t n_train;
  int32_t width;
  int32_t height;
  float lambda_ssim;             /* loss weight of 1 - SSIM (gs_loss) */
  float bg[3];                   /* background colour */
  const float* lr_init;          /* host [n_planes][4] (gs_adam_step) */
  const float* lr_final;         /* host [n_planes][4] or NULL */
  int32_t lr_steps;
  float beta1;
  float beta2;
  float eps;
  int32_t* d_step;               /* [1] step counter t, advanced by one per call */
  gs_camera* cams_step;          /* [U] step buffers written by the gather */
  float* gt_step;                /* [U][3][H][W] */
  uint8_t* mask_step;            /* [U][H][W] */
  const gs_proj* proj;           /* host struct of [P] record buffers, P = sum of gauss_count */
  int64_t max_instances;         /* capacity of sorted_vals and of the sort workspace */
  void* sort_ws;                 /* gs_bin_sort_workspace_size(P, max_instances) bytes */
  size_t sort_ws_bytes;
  uint32_t* sorted_vals;         /* [max_instances] */
  uint32_t* ranges;              /* [U * n_tiles][2] */
  uint32_t* d_num_instances;     /* [1] */
  const gs_schedule* sched;      /* host struct of the blend schedule buffers, or NULL */
  float* img;                    /* [U][3][H][W] */
  float* final_T;                /* [U][H][W] */
  uint32_t* n_contrib;           /* [U][H][W] */
  void* loss_ws;                 /* gs_loss_workspace_size(U, W, H) bytes */
  size_t loss_ws_bytes;
  float* d_loss;                 /* [1] mean loss over the units */
  float* dL_dimg;                /* [U][3][H][W] */
  const gs_grad2d* g2d;          /* host struct of [P] screen-space gradient buffers */
  float* grads;                  /* parameter gradient (planes layout) or NULL */
  int32_t variant;               /* blend execution shape (gs_render_fwd) */
  int32_t sparse_adam;           /* gs_project_bwd_adam's sparse flag */
  float lambda_bg;               /* > 0: add gs_bg_penalty with this weight (then the next three are needed) */
  void* bg_ws;                   /* gs_bg_penalty_workspace_size(U) bytes */
  size_t bg_ws_bytes;
  float* dL_dT;                  /* [U][H][W] */
} gs_train_batch_desc;

int gs_train_batch(const gs_train_batch_desc* desc, int* d_status, gs_stream_t stream);

/* The gather step alone: the views of step *d_step (same rule) into
 * cams_step, gt_step and mask_step (16-byte copies when pointers and sizes
 * allow).  Lets a caller inspect or size a step without training it. */
int gs_gather_views(const gs_train_batch_desc* desc, const int32_t* d_step, gs_stream_t stream);

/* ---- a8: merged render of all partitions (Sec. II, "Global Reconstruction")
 * The splats of all partitions, concatenated in partition order, are rendered
 * as one scene after the ghost filter: a Gaussian of partition k is kept iff
 * its (trained) mean lies in partition k's owned box (see gs_owned).  One
 * camera (device, 1 entry), one image [3][H][W].  Equivalent to
 * gs_preprocess (one unit over all N, with `owned`) + gs_bin_sort +
 * gs_render_fwd; proj must hold N records and the workspace
 * gs_bin_sort_workspace_size(N, max_instances) bytes.  sched: NULL, or a
 * schedule sized for one unit of width x height and max_instances (see
 * gs_schedule), which the sort fills and the forward uses (block masks,
 * heaviest-first order). */
int gs_merge_render(const float* params, int64_t n_gauss, int sh_degree, const gs_owned* owned,
                    const gs_camera* cam, int width, int height, const float* bg,
                    const gs_proj* proj, int64_t max_instances, void* workspace,
                    size_t workspace_bytes, uint32_t* sorted_vals, uint32_t* ranges,
                    uint32_t* d_num_instances, float* img, float* final_T, uint32_t* n_contrib,
                    const gs_schedule* sched, int* d_status, gs_stream_t stream);

/* ---- adaptive density control (3D-GS densification) ----------------------
 * The optimisation each partition is trained with (Sec. II, "Parallel
 * Training") is standard 3D Gaussian Splatting, which clones, splits and
 * prunes Gaussians as it trains.  Reading of its rules:
 *   statistics per training view, for every record with radius > 0 of
 *   Gaussian i: grad_accum[i] += |(dL/du W/2, dL/dv H/2)| (u, v: its pixel
 *   position; dxy of gs_grad2d), denom[i] += 1, max_radius[i] = max(., radius);
 *   plan at step t: g = grad_accum / denom (0 if denom = 0), smax = largest
 *   scale, o = opacity; prune if o < min_opacity or (t > reset_interval and
 *   (max_radius > max_screen or smax > 0.1 extent)); otherwise, if
 *   g >= grad_threshold: split if smax > percent_dense extent, else clone;
 *   apply: kept sources (not pruned, not split) in index order, then copies of
 *   the cloned sources, then two children per split source (mean + R(q)(s * z),
 *   log scales - log 1.6, all else copied); Adam moments copied for kept
 *   sources, zero for new Gaussians;
 *   opacity reset: logit opacity = min(logit opacity, logit(max_opacity)) and
 *   the opacity's Adam moments = 0.
 * grad_accum, denom, max_radius: device float [n_gauss] (caller zeroes them
 * after each plan). */
typedef struct gs_densify_cfg {
  float grad_threshold;  /* 2e-4 in 3D-GS */
  float percent_dense;   /* 0.01 */
  float min_opacity;     /* 0.005 */
  float max_screen;      /* 20 px */
  float extent;          /* scene extent (> 0) */
  int32_t step;          /* current optimisation step */
  int32_t reset_interval;/* opacity reset period (3000); screen / world size pruning only after it */
} gs_densify_cfg;

/* Accumulates one step's statistics (proj and g2d of that step's units). */
int gs_densify_stats(const gs_proj* proj, const gs_grad2d* g2d, const gs_units* units, int width,
                     int height, float* grad_accum, float* denom, float* max_radius,
                     gs_stream_t stream);

/* Plan: each Gaussian's action and the exclusive prefixes of the kept /
 * cloned / split counts (in the workspace, gs_densify_workspace_size(n));
 * d_counts (device uint32[3]) receives (kept, cloned, split).  The output of
 * gs_densify_apply holds kept + cloned + 2 split Gaussians. */
size_t gs_densify_workspace_size(int64_t n_gauss);
int gs_densify_plan(const float* params, int64_t n_gauss, const float* grad_accum,
                    const float* denom, const float* max_radius, const gs_densify_cfg* cfg,
                    void* workspace, size_t workspace_bytes, uint32_t* d_counts,
                    gs_stream_t stream);

/* Apply the plan in `workspace` (same n_gauss): params / m / v planes
 * [planes][n_gauss][4] in, out_* planes [planes][n_out][4] out; z: device
 * float [n_gauss][2][3] standard normal draws (used for split sources).
 * Positions at or past n_out are not written and set GS_ERR_CAPACITY. */
int gs_densify_apply(const float* params, const float* m, const float* v, int64_t n_gauss,
                     int sh_degree, const float* z, const void* workspace, size_t workspace_bytes,
                     float* out_params, float* out_m, float* out_v, int64_t n_out, int* d_status,
                     gs_stream_t stream);

/* Opacity reset of 3D-GS (see above); max_opacity in (0, 1), 0.01 in 3D-GS. */
int gs_opacity_reset(float* params, float* m, float* v, int64_t n_gauss, float max_opacity,
                     gs_stream_t stream);

/* ---- a9: learned initialiser --------------------------------------------
 * Not in the paper: its Sec. II initialises the Gaussians from the extracted
 * isosurface points.  The plain form used there sets each Gaussian's scale
 * from its neighbours' distances; the learned form predicts scale, rotation
 * and opacity from the kNN geometry with a small MLP trained on converged
 * splats, and keeps the plain form as fallback.
 *
 * gs_knn: exact k nearest neighbours (self excluded) of n points [n][3] on a
 * uniform grid of grid_dims[0..2] cells of edge cell_size starting at
 * grid_lo (host float[3]; the grid must cover the points' bounding box),
 * k in {3, 8, 16}.  idx [n][k] int32, dist [n][k] fp32 (Euclidean),
 * ordered by (distance, index); -1 / inf when fewer than k other points
 * exist.  Workspace: gs_knn_workspace_size(n, grid_dims (host int32[3])). */
size_t gs_knn_workspace_size(int64_t n, const int32_t* grid_dims);
int gs_knn(const float* points, int64_t n, int k, const float* grid_lo, float cell_size,
           const int32_t* grid_dims, void* workspace, size_t workspace_bytes, int32_t* idx,
           float* dist, gs_stream_t stream);

/* MLP 112 -> 64 -> 64 -> 8 with ReLU.  Parameters: one fp32 buffer of
 * gs_mlp_param_count() = 11912 values: W1 [112][64] (input-major), b1[64],
 * W2 [64][64], b2[64], W3 [64][8], b3[8].  Features of point i from its 16
 * nearest neighbours (idx/dist from gs_knn with k = 16): offsets / mean
 * neighbour distance [0,48), neighbour normals [48,96), own normal [96,99),
 * zeros [99,112).  GEMM operands bf16 (round to nearest even), fp32
 * accumulation; activations and back-propagated signals rounded to bf16
 * where they become GEMM operands.  Outputs [n][8]:
 * (log-scale offsets (3), rotation (w, x, y, z), logit opacity). */
int gs_mlp_param_count(void);
/* features [n][112] as bf16 bit patterns (for inspection and tests) */
int gs_mlp_features(const float* points, const float* normals, const int32_t* knn_idx,
                    const float* knn_dist, int64_t n, uint16_t* features, gs_stream_t stream);
int gs_mlp_forward(const float* points, const float* normals, const int32_t* knn_idx,
                   const float* knn_dist, int64_t n, const float* weights, float* out,
                   gs_stream_t stream);
/* One Adam step (lr, betas 0.9 / 0.999, eps 1e-8, t = *d_step + 1) on the
 * loss sum (out - targets)^2 / (8 n) over all n points.  grad: fp32 scratch
 * [11912] (overwritten); m, v: Adam moments [11912]; d_loss: device float. */
int gs_mlp_train_step(const float* points, const float* normals, const int32_t* knn_idx,
                      const float* knn_dist, const float* targets, int64_t n, float* weights,
                      float* grad, float* m, float* v, float lr, const int32_t* d_step,
                      float* d_loss, gs_stream_t stream);
/* Initial Gaussians 0..n-1 of a planes buffer of n_gauss Gaussians: mean =
 * point; plain form (weights NULL): isotropic log-scale log(d3), d3 the mean
 * of the 3 nearest distances (floored at 1e-7), identity rotation, logit
 * opacity logit_default; learned form: log-scale log(d3) + out[0:3],
 * rotation out[3:7], logit out[7], falling back to the plain values for a
 * Gaussian whose outputs are non-finite or whose rotation has norm < 1e-6.
 * SH planes are not touched.  knn_k >= 3 (16 with weights). */
int gs_init_gaussians(const float* points, const float* normals, const int32_t* knn_idx,
                      const float* knn_dist, int knn_k, int64_t n, const float* weights,
                      float logit_default, float* params, int64_t n_gauss, gs_stream_t stream);

/* ---- issue-rate microbenchmark (the blend kernels' roofline denominator) -
 * The blend stages are bound by instruction issue, not by HBM or the tensor
 * cores, so their peak is the rate at which the SMs retire FP32 and MUFU
 * lane-operations, measured by this kernel on the device it runs on.
 * Every thread runs GS_PEAK_CHAINS independent chains of `iters` steps:
 * mode 0: x = fma(x, a, b) (one FP32 lane-operation per step); mode 1:
 * x = ex2.approx(x) - b (one MUFU ex2 and one FP32 add per step).  Chain j
 * starts at x = -j/8; out[t] = the sum of thread t's chains (device float
 * [gs_peak_threads(n_sms)], caller-owned).  Lane-operations per launch =
 * gs_peak_threads(n_sms) x GS_PEAK_CHAINS x iters; the caller times the
 * launch with events on `stream`.  Bad mode, sizes or a NULL out return
 * GS_ERR_INVALID. */
#define GS_PEAK_CHAINS 8
int gs_peak_threads(int n_sms);
int gs_peak_issue(int mode, int n_sms, int iters, float a, float b, float* out,
                  gs_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* GS_H */
