/*
 * ofv.h -- C ABI of the GB300 (sm_103a) dense optical-flow velocimetry
 * estimator of Pimienta & Aider, "High Resolution and High-Speed Live Optical
 * Flow Velocimetry" (arXiv 2509.25924).
 *
 * The estimator turns two frames I^t, I^t' into one displacement vector
 * V = (u, v) per pixel, in px/frame (the velocity is V / dt; Eq. 1).  It
 * follows the six-step pipeline of Sec. 2: local intensity normalization,
 * Burt-Adelson Gaussian pyramid with PSL sub-levels, per-pixel Lucas-Kanade
 * estimate minimising the symmetric SSD of Eq. 2 by IT Gauss-Newton
 * iterations over a (2KR+1)^2 window, and x2 up-sampling of the field from
 * each level to the next finer one.
 *
 * Conventions shared by every entry point
 *   - Images and fields are dense row-major H x W arrays (no row padding):
 *     element (i, j) is row i, column j, at offset i*W + j.  u is the
 *     displacement along +x (columns), v along +y (rows), attributed to the
 *     pixel centre taken as the midpoint between the two exposures.
 *   - Unless an entry point says "host", every data pointer is a device
 *     pointer of the device that was current when the handle was created.
 *     The caller owns all image, field and weight buffers; the handle owns
 *     its workspace (pyramids, ping-pong fields, staging).
 *   - Work is enqueued on the given stream (NULL = the legacy default stream)
 *     and the call returns without synchronising; results are valid once the
 *     stream has reached them.  Buffers passed to a call must stay valid until
 *     then.
 *   - No exception crosses the ABI.  Every call returns an ofv_status.
 *     Argument and shape errors are detected on the host before any work is
 *     enqueued.  An asynchronous device error is reported as OFV_ERR_CUDA by
 *     the call that observes it.  ofv_last_error() describes the most recent
 *     failure in the calling thread.
 *   - A handle is not thread-safe, and work of one handle on different
 *     streams must not overlap (the workspace is shared): order it, or use
 *     one stream.  Distinct handles on distinct streams are independent.
 *   - The fused kernels stage image tiles with TMA copies and wait for them
 *     with a bound (2 s).  If a wait ever expires the kernel records it in a
 *     handle-owned word of page-locked host memory, and every later compute,
 *     graph-launch and backward call on that handle returns OFV_ERR_TIMEOUT
 *     without enqueuing work.
 */
#ifndef OFV_H
#define OFV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t / CUstream. */
typedef struct CUstream_st *ofv_stream_t;

typedef enum {
    OFV_OK = 0,
    OFV_ERR_INVALID_ARG = 1, /* null pointer, out-of-range parameter */
    OFV_ERR_SHAPE = 2,       /* image too small for PSL and KR, or too large */
    OFV_ERR_ALLOC = 3,       /* device or pinned-host allocation failed */
    OFV_ERR_CUDA = 4,        /* a CUDA call failed (message in ofv_last_error) */
    OFV_ERR_TIMEOUT = 5,     /* a bounded device-side wait expired */
    OFV_ERR_UNSUPPORTED = 6  /* valid request this build does not implement */
} ofv_status;

typedef enum { OFV_IN_U8 = 0, OFV_IN_U16 = 1, OFV_IN_F32 = 2 } ofv_input_t;

/* Storage of the level images (normalized input and pyramid).  Sums, solve
   and fields are always FP32. */
typedef enum { OFV_STORE_F32 = 0, OFV_STORE_F16 = 1, OFV_STORE_BF16 = 2 } ofv_storage_t;

/* OFV_PATH_FUSED: one kernel per (level, iteration) doing warp, gradients,
   products, window sums and the solve on chip: for KR <= 10 the block kernel
   (both images staged in shared memory over a 48x48 or 32x32 output tile,
   window sums by additions only), for larger KR the tile kernel.
   OFV_PATH_TILE: always the tile kernel (one CTA per 32x32 output tile with
   the products of tile and halo in shared memory); kept for comparison.
   OFV_PATH_PLAIN: the same arithmetic split into separate kernels that pass
   five product planes through device memory (kept for comparison). */
typedef enum { OFV_PATH_FUSED = 0, OFV_PATH_PLAIN = 1, OFV_PATH_TILE = 2 } ofv_path_t;

/* Weights of the window N(m) of Eq. 2.  The paper names only its radius KR
   (Sec. 2); the default is the uniform (2KR+1)^2 box.  OFV_WINDOW_GAUSS
   weights tap (a, b) of the box by exp(-(a^2 + b^2) / (2 sigma^2)), sigma =
   window_sigma (a variant; the box is still truncated at the image border). */
typedef enum { OFV_WINDOW_BOX = 0, OFV_WINDOW_GAUSS = 1 } ofv_window_t;

typedef struct {
    int levels_psl;     /* PSL >= 0 pyramid sub-levels; levels = PSL + 1 (Sec. 2; Table 2 uses 2..4) */
    int kernel_radius;  /* KR, 1..16: window (2KR+1)^2, uniform weights (Sec. 2; Table 2 uses 2..7) */
    int iterations;     /* IT, 1..64 Gauss-Newton iterations per level (Sec. 2; Table 2 uses 1..4) */
    int norm_radius;    /* NR, 0..16 local normalization radius; 0 = off (Sec. 2; Table 2 uses 1..4) */
    int input;          /* ofv_input_t of the frames passed to compute calls */
    int bit_depth;      /* integer inputs: significant bits, 1..16 (u8: <= 8); I = raw / (2^bits - 1) */
    int storage;        /* ofv_storage_t */
    int path;           /* ofv_path_t */
    int prefilter;      /* 1: 5x5 correlation (weights set by ofv_set_prefilter) after normalization */
    float det_rel_eps;  /* guard: keep V0 where det <= eps * (Sxx + Syy)^2 (default 1e-6) */
    float det_abs_eps;  /* guard: keep V0 where Sxx + Syy <= eps (default 1e-20) */
    float norm_eps;     /* normalization floor: (I - mu) / sqrt(var + eps^2) (default 1e-2) */
    int max_batch;      /* pairs of a sequence per iteration launch, 0..8; 0 = auto (as many as keep
                           about 16 Mp per launch).  Each costs three more pyramids and six fields
                           of workspace (three groups of a sequence are in flight). */
    /* Estimator variants (defaults: 0, i.e. the estimator as read from Sec. 2). */
    int window;         /* ofv_window_t (every forward path; ofv_backward covers the box only) */
    float window_sigma; /* OFV_WINDOW_GAUSS: sigma in px, finite and > 0 */
    int increment_form; /* 1: each Gauss-Newton step solves for the increment,
                           V(m) = V0(m) + H^-1 sum G (-It), instead of H V = sum G (G.V0 - It) */
    int warm_start;     /* sequences only, 0..56: 0 = every pair starts from V = 0; d > 0 = pair k >= d
                           starts its coarsest level from pair k-d's field sampled at that level's pixels,
                           V_L(i, j) = V(2^L i, 2^L j) / 2^L (pairs k < d start from 0).  d <= B (the
                           pairs-per-launch): groups of d pairs, each waiting for the previous one.  A
                           multiple d = m B (m <= 7, device sequences only): groups of B pairs, each
                           waiting for the group m back, so the m - 1 groups between still overlap. */
    int tile_edge;      /* fused block kernel (KR 1..10) output tile edge in px: 0 = the radius's default
                           (48 for KR <= 5, 64 for KR 6..10); or the alternative, 32.  With 0,
                           ofv_compute_batched's autotuner picks one of
                           the two per batch signature (ofv_batch_tuning reports it); nonzero fixes it.
                           The window sums' rounding follows the tile grid, so fields of different tile
                           edges agree to FP32 rounding, not bitwise.  The estimator variants (Gaussian
                           window, increment form, region mask) and the reverse mode run the default. */
} ofv_params;

typedef struct ofv_handle ofv_handle;

/* Fill *p with the defaults: PSL 2, KR 4, IT 3, NR 0, 12-bit uint16 input,
   FP32 storage, fused path, no pre-filter, guards 1e-6 / 1e-20, floor 1e-2,
   box window, direct form, no warm start. */
void ofv_default_params(ofv_params *p);

/* Create a handle for H x W frames with parameters *p (copied): the
   parameters of Sec. 2 and Sec. 6 (pyramid levels PSL, window radius KR,
   iterations IT, normalization radius NR).  Allocates the whole workspace
   on the current device: the level images of the pyramid (Sec. 2, step 2)
   and the displacement fields of the iterations (Eq. 2).  Every level must be at least
   max(8, 2KR+1) pixels in both dimensions (else OFV_ERR_SHAPE); H * W must
   not exceed 2^31 - 1.  On failure *out is set to NULL and nothing leaks. */
ofv_status ofv_create(int H, int W, const ofv_params *p, ofv_handle **out);

/* Free the handle and its workspace (synchronises the device work it owns).
   NULL is accepted. */
ofv_status ofv_destroy(ofv_handle *h);

/* Copy the 25 pre-filter weights (row-major 5x5, device pointer) into the
   handle, on stream s.  out(i,j) = sum_{a,b=-2..2} w[(a+2)*5+(b+2)] * I(i+a, j+b),
   clamp-to-edge.  Only meaningful when params.prefilter = 1; the weights
   start as the identity (1 at the centre). */
ofv_status ofv_set_prefilter(ofv_handle *h, const float *w25, ofv_stream_t s);

/* Region mask (a variant; the masked regions of Sec. 7, such as a model and
   its shadow): mask is H x W bytes (device), nonzero = valid.  Level l uses
   the mask at (2^l i, 2^l j).  A masked pixel's products are left out of
   every window sum at every level, and its output is NaN (no vector).  The
   mask is copied into handle-owned level masks on stream s and applies to
   every later compute, sequence and graph-creation call of the handle; NULL
   clears it.  While a mask is set, ofv_compute_batched and ofv_backward
   return OFV_ERR_UNSUPPORTED. */
ofv_status ofv_set_mask(ofv_handle *h, const uint8_t *mask, ofv_stream_t s);

/* Estimate the displacement field between frames I1 (time t) and I2 (time
   t + dt), both H x W of the handle's input type: Sec. 2 steps 1-6 (local
   normalization, the pyramid, and per level IT Gauss-Newton iterations of
   the symmetric SSD of Eq. 2 with the window sums of its normal equations),
   giving V = (u, v) in px per frame, the velocity of Eq. 1 times dt.
   Writes u and v (H x W float each).  I1, I2, u and v are device pointers; u and v must not alias
   the inputs. */
ofv_status ofv_compute(ofv_handle *h, const void *I1, const void *I2, float *u, float *v,
                       ofv_stream_t s);

/* As ofv_compute, but I1, I2, u and v are HOST pointers.  The frames are
   copied to handle-owned device staging, the field is copied back, all on
   stream s; the host outputs are valid once s has been synchronised.  Use
   page-locked host memory for asynchronous copies. */
ofv_status ofv_compute_host(ofv_handle *h, const void *I1, const void *I2, float *u, float *v,
                            ofv_stream_t s);

/* Time-resolved sequence: n_frames >= 2 frames F_0..F_{n-1}, frame k at
   frames + k * frame_stride_bytes (device), give n_frames - 1 fields, pair
   k = (F_k, F_{k+1}), written to u + k * field_stride and v + k * field_stride
   (elements).  Each frame is normalized and reduced once and its pyramid is
   reused by the two pairs it belongs to.  Pairs run in groups of the
   handle's pairs-per-launch; with the fused path consecutive groups run on
   library-owned streams so that one group's coarse levels overlap another's
   fine levels.  Work queued on s before the call runs first, and s reaches
   the end of the call only when every field is written.  With
   params.warm_start = d, pair k >= d starts from pair k-d's field
   (OFV_ERR_INVALID_ARG unless d <= B or d = m B with m <= 7; B = the
   pairs-per-launch; the host-memory form below accepts d <= B only). */
ofv_status ofv_compute_sequence(ofv_handle *h, int n_frames, const void *frames,
                                size_t frame_stride_bytes, float *u, float *v, size_t field_stride,
                                ofv_stream_t s);

/* As ofv_compute_sequence, but frames, u and v are HOST pointers (use
   page-locked memory for the copies to overlap).  The sequence runs in
   groups of the handle's pairs-per-launch; each frame is uploaded once, and
   the upload of the next group and the download of the previous group's
   fields run on two library-owned copy streams while the groups compute
   (as in ofv_compute_sequence).  A device ring of groups (frames and
   fields) is allocated on first use and kept.  Work queued on s before the call runs
   first; the host outputs are valid once s has been synchronised. */
ofv_status ofv_compute_sequence_host(ofv_handle *h, int n_frames, const void *frames,
                                     size_t frame_stride_bytes, float *u, float *v,
                                     size_t field_stride, ofv_stream_t s);

/* ---- derived quantities (Sec. 7) ------------------------------------------
 * Computed from the fields in real time, like the vorticity maps and the
 * recirculation-area time series of the paper's cylinder-wake experiment.
 * Both take n fields of a sequence at u + k * field_stride (and v + k *
 * field_stride), H x W dense each, device pointers, 1 <= n <= 65535.
 *
 * ofv_vorticity writes omega = dv/dx - du/dy per field (u along columns x,
 * v along rows y; omega + k * field_stride), with second-order central
 * differences inside and first-order one-sided differences on the first and
 * last column / row; for px/frame fields the unit is 1/frame (divide by the
 * frame interval for 1/s).
 *
 * ofv_recirculation_area writes counts[k] (device, unsigned 64-bit) = the
 * number of pixels of field k where u < 0 (H(-u) = 1 in Eq. 6), inside the
 * region mask (H x W bytes, nonzero = inside; NULL = every pixel).  RA(t) is
 * counts[k] times the pixel area dx dz.  counts is cleared on stream s
 * first. */
ofv_status ofv_vorticity(int H, int W, int n, const float *u, const float *v, size_t field_stride,
                         float *omega, ofv_stream_t s);
ofv_status ofv_recirculation_area(int H, int W, int n, const float *u, size_t field_stride,
                                  const uint8_t *mask, unsigned long long *counts, ofv_stream_t s);

/* Point probes: the time series of the field at npts points, as a probe
 * of the live measurement would record it.  xy (device, npts x 2 floats,
 * 8-byte aligned) holds the points (x along columns, y along rows) in pixel
 * coordinates; out (device, n x npts x 2 floats, 8-byte aligned) receives
 * (u, v) of field k at point p at out[2 (k npts + p)].  The field is sampled
 * bilinearly with clamp-to-edge taps, the interpolation of the estimator; a
 * tap on a pixel without a vector (region mask) gives NaN.  1 <= n <= 65535. */
ofv_status ofv_probe(int H, int W, int n, const float *u, const float *v, size_t field_stride, int npts,
                     const float *xy, float *out, ofv_stream_t s);

/* ---- reverse mode -------------------------------------------------------
 * The paper defines no derivative; this is the chain rule through the steps
 * of Sec. 2 (Eq. 2 and its Gauss-Newton linearisation, the pyramid, the
 * up-sampling) in reverse order, for training a pre-filter or chaining the
 * estimator inside a differentiable model.
 *
 * Given a loss L(u, v) and its gradients gu = dL/du, gv = dL/dv (H x W
 * float, device), writes gI1 = dL/dI1 and gI2 = dL/dI2 (H x W float, device,
 * gradients with respect to the raw input values) and, when gw25 is not
 * NULL, gw25 = dL/dw (25 floats, device, row-major 5x5 pre-filter weights;
 * zeros when params.prefilter = 0).  The forward pass is recomputed from I1
 * and I2 with the fused kernels and each stage's fields and window sums are
 * kept in a handle-owned workspace (grown on demand: one float2 field and
 * five float planes per stage at its level's size plus about 17 float planes
 * of the level-0 size).  A pixel whose 2x2
 * system was guarded keeps V0, so its gradient passes to V0 unchanged; at a
 * bilinear cell boundary the derivative is that of the cell floor() picks.
 * Float atomics scatter the gradients, so the last bits vary between runs.
 * The handle's pyramid slots are overwritten (as by ofv_compute).
 * Local normalization (NR > 0) is differentiated: its statistics are
 * recomputed per frame and the adjoint of (I - mu) / s over the in-image box
 * takes three more box sums.  OFV_ERR_UNSUPPORTED with the Gaussian window,
 * the increment form or a region mask (the reverse mode covers the direct
 * form with the uniform box). */
ofv_status ofv_backward(ofv_handle *h, const void *I1, const void *I2, const float *gu,
                        const float *gv, float *gI1, float *gI2, float *gw25, ofv_stream_t s);

/* ---- one field as horizontal strips (multi-GPU decomposition) -----------
 * The paper names spreading the computation over 2 or 3 GPUs as the way to
 * raise the rate further (Conclusions).  ofv_compute_strips computes one
 * field as nstrips horizontal strips, each with a workspace of its own (here
 * all on the handle's device, one strip after another on stream s): at
 * every level a strip owns whole tile rows of the block kernel's tile grid
 * and computes the rows of its pyramids it reads (own rows plus a redundant
 * halo, from the input rows around them), so images need no exchange; after
 * every Gauss-Newton iteration it copies from their owners the rows of the
 * new field its next iteration reads (the window halo, or the coarse rows
 * the next level's up-sampling reads).  The field equals ofv_compute's
 * bitwise while no warp reaches farther than max_disp px (level-0 units);
 * max_disp only sizes the image halo.  Fused path with KR 1..10, no region
 * mask (else OFV_ERR_UNSUPPORTED); nstrips 1..64.  Workspace: nstrips full
 * pyramids and two fields, grown on demand and owned by the handle; I1, I2,
 * u, v as for ofv_compute. */
typedef struct {
    int own_row0, own_row1;       /* rows of the level the strip outputs (whole tile rows) */
    int img_row0, img_row1;       /* rows of the level's images it computes (own rows and the halo) */
    int fld_row0, fld_row1;       /* rows of the level's field its iterations read */
    int up_row0, up_row1;         /* rows of the next coarser level's field read when up-sampling to this level */
    int ingest_row0, ingest_row1; /* level 0: input rows it ingests (0, 0 at other levels) */
} ofv_strip_rows;
/* The rows strip `strip` of `nstrips` works on at `level` (host only, no
   device work): for checking the decomposition. */
ofv_status ofv_strip_plan(int H, int W, const ofv_params *params, int nstrips, int max_disp, int level, int strip,
                          ofv_strip_rows *out);
ofv_status ofv_compute_strips(ofv_handle *h, int nstrips, int max_disp, const void *I1, const void *I2, float *u,
                              float *v, ofv_stream_t s);

/* ---- allocation-free variant -------------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot call cudaMalloc: host applications whose device memory belongs to
 * another allocator (a framework's caching allocator, or a pool sized at
 * start-up that a cudaMalloc behind its back would starve), and real-time
 * acquisition loops that forbid allocation once running (cudaMalloc may
 * block the host thread and synchronise the device).
 *
 * ofv_compute_noalloc computes the same field as ofv_create + ofv_compute,
 * bitwise, with the same iteration kernels (fused path only; params->path
 * must be OFV_PATH_FUSED, else OFV_ERR_UNSUPPORTED), but allocates nothing:
 * its workspace is a fixed device array of OFV_NOALLOC_SCRATCH_BYTES inside
 * the library, which every GPU that loads the library holds until the
 * process exits.  It keeps no TMA tensor maps, so the iteration kernel
 * stages its image tiles by cp.async (same arithmetic, so the same field).
 * params->max_batch and params->warm_start are range-checked as ofv_create
 * checks them and otherwise ignored; params->tile_edge is checked and used
 * as by ofv_create.  The caller passes the frames I1, I2 (H x W, params->input type),
 * the outputs u, v (H x W float) and, when params->prefilter = 1, the 25
 * pre-filter weights w25 (device, row-major 5x5; may be NULL otherwise).
 * A request whose workspace would exceed the array (about 27 bytes per pixel
 * at FP32 storage: 1024 x 1024 fits, 2048 x 2048 does not) is rejected with
 * OFV_ERR_SHAPE and a message giving the bytes needed.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture begins.  All calls share the one array and
 * leave their intermediates in it; every intermediate is written before it
 * is read, so no call depends on what an earlier one left.  Calls whose GPU
 * work overlaps (different streams, or different host threads, without
 * ordering between them) race on the array and corrupt each other's
 * results: order them on one stream. */
#define OFV_NOALLOC_SCRATCH_BYTES (64u << 20)
ofv_status ofv_compute_noalloc(int H, int W, const ofv_params *params, const float *w25, const void *I1,
                               const void *I2, float *u, float *v, ofv_stream_t s);

/* ---- many pairs of unequal size -----------------------------------------
 * One pair of a batch: frames I1, I2 (H x W, the handle's input type) and
 * outputs u, v (H x W float), all device pointers. */
typedef struct {
    int H, W;
    const void *I1, *I2;
    float *u, *v;
} ofv_pair;

/* Estimate n pairs of any sizes (each within the shape limits of
 * ofv_create for the handle's parameters; the handle's own H, W do not
 * matter) with the handle's parameters, 1 <= n <= 32767: the estimator of
 * Sec. 2 (steps 1-6, Eq. 2) for every pair, as ofv_compute computes it.
 * pairs is a HOST array.  All 2n frames are ingested by one launch and each
 * pyramid level of all of them is reduced by one launch; then every (level,
 * iteration, tile) of every pair runs in ONE persistent launch of the fused
 * kernel: CTAs take work units from a queue in the order of a schedule, and
 * a unit of one Gauss-Newton iteration waits (bounded) until the previous
 * iteration of its pair is complete.  The first batch of a given signature
 * (sorted sizes and parameters) runs the autotuner: each candidate -- tile
 * shape (see ofv_params.tile_edge), schedule (all pairs stage by stage, or
 * groups of 8 pairs) and persistent grid (the resident CTAs per SM, or one
 * fewer) -- is timed on the batch itself and the fastest is kept
 * for later batches of that signature (that first call waits for its
 * timings).  Otherwise the call enqueues the batch on s and returns; the
 * fields are valid once s reaches them, and the next call's host work
 * overlaps this batch.  The schedule and the tensor maps of a layout are
 * uploaded once and reused.  A workspace for the batch is allocated on first
 * use and grown when a larger batch arrives (growing waits for s).  Needs the
 * fused path with KR <= 10 (else OFV_ERR_UNSUPPORTED).  A dependency wait
 * that expires (5 s) is recorded in a handle-owned word of page-locked host
 * memory: the first batched call that observes it, and every later one,
 * returns OFV_ERR_TIMEOUT without enqueuing work (the tuning call observes
 * its own). */
ofv_status ofv_compute_batched(ofv_handle *h, int n, const ofv_pair *pairs, ofv_stream_t s);

/* Configuration used by the last ofv_compute_batched call: schedule (0 =
 * stage-major over all pairs, else group size), persistent CTAs per SM, the
 * output tile edge of the block kernel in px (with ofv_params.tile_edge = 0
 * the autotuner tries the radius's default and alternative edges, except
 * with the Gaussian window or the increment form, which have the default
 * only; a nonzero tile_edge fixes the edge),
 * duration of its persistent launch in ms, and whether that call tuned.  A
 * handle created with tile_edge set to the reported edge computes, through
 * ofv_compute, bitwise the fields the batch computed. */
ofv_status ofv_batch_tuning(const ofv_handle *h, int *schedule, int *ctas_per_sm, int *tile_edge, double *ms,
                            int *tuned);

/* Test hook for the bounded waits of the persistent launch: runs one CTA
 * whose work unit depends on a counter nothing increments.  Expected result:
 * OFV_ERR_TIMEOUT after about timeout_us, *error_word = 1 (the device word),
 * the same value in the mapped host word that asynchronous batches report
 * through (OFV_ERR_CUDA if it differs), the device still usable. */
ofv_status ofv_queue_selftest(int timeout_us, int *error_word);

/* ---- debugging hooks -----------------------------------------------------
 * For tests of the error paths and of workspace hygiene; no effect on the
 * estimator otherwise.
 *
 * ofv_debug_fail_alloc(n): the n-th device allocation of the library from
 * now on (workspaces of ofv_create, of the host-pointer, host-sequence,
 * batched and reverse-mode entry points, the mask levels) fails as if the
 * device were out of memory; n <= 0 cancels.  The entry point then returns
 * OFV_ERR_ALLOC and leaves nothing allocated.
 *
 * ofv_debug_poison(h, s): fills the handle's scratch (pyramids, fields,
 * staging, reverse-mode and batch workspaces) with all-ones bytes (NaN in
 * every float) on stream s.  A compute call must then give bitwise the same
 * result as before: no output depends on scratch it did not write first.
 * The pre-filter weights and the region mask are state, not scratch, and
 * are kept.
 *
 * ofv_debug_reciprocal(x, y, n, s): y[i] = 1 / x[i] as the fused path's
 * 2x2 solve forms it (Eq. 2's normal equations are solved by Cramer's rule
 * with one reciprocal of the determinant): the hardware approximation
 * refined by one Newton-Raphson step.  x and y are device arrays of n
 * floats; for testing its error against 1/x. */
void ofv_debug_fail_alloc(int n);
ofv_status ofv_debug_poison(ofv_handle *h, ofv_stream_t s);
ofv_status ofv_debug_reciprocal(const float *x, float *y, int n, ofv_stream_t s);

/* ---- CUDA-graph replay (live loop) -------------------------------------
 * A live acquisition hands the estimator a new pair into the same device
 * buffers at a fixed rate (Sec. 6, live mode).  ofv_graph_create records the
 * whole launch sequence of ofv_compute(h, I1, I2, u, v) for those fixed
 * buffers into a CUDA graph (after one eager run that prepares the kernels),
 * so each new pair costs one ofv_graph_launch instead of ~PSL + L*IT + 1
 * launches.  ofv_graph_create synchronises the device first (the eager run
 * uses the handle's workspace on a stream of its own).  The graph uses the
 * handle's workspace: the handle must outlive it, and launches of graphs and
 * compute calls of one handle must be ordered (one stream).  Kernel timing
 * is not recorded inside graphs. */
typedef struct ofv_graph ofv_graph;
ofv_status ofv_graph_create(ofv_handle *h, const void *I1, const void *I2, float *u, float *v, ofv_graph **out);
ofv_status ofv_graph_launch(ofv_graph *g, ofv_stream_t s);
ofv_status ofv_graph_destroy(ofv_graph *g);

/* The batched form for camera streams of uneven size (Sec. 6: several
 * cameras or streams at fixed rates): records ofv_compute_batched(h, n,
 * pairs) -- the ingest and reduce launches of every frame and the one
 * persistent launch of all (level, iteration, tile) units -- into a CUDA
 * graph, so a new set of pairs written into the same buffers costs one
 * ofv_graph_launch and no host work.  pairs is a HOST array as for
 * ofv_compute_batched; its buffers are the ones every launch reads and
 * writes.  Synchronises the device, then runs the batch eagerly (tuning a new
 * signature, as ofv_compute_batched does) before recording it.  The graph
 * takes the handle's batch workspace and frees it in ofv_graph_destroy;
 * later batched calls of the handle allocate a new one, so they and the
 * graph do not overwrite each other's data.  The handle (its parameters,
 * pre-filter weights and error words) must outlive the graph, and launches
 * of graphs and compute calls of one handle must be ordered (one stream).
 * Errors as ofv_compute_batched; nothing is recorded on failure and *out is
 * NULL.  A dependency wait that expires in a replayed launch sets the
 * handle's error word: the handle's next batched call returns
 * OFV_ERR_TIMEOUT. */
ofv_status ofv_graph_create_batched(ofv_handle *h, int n, const ofv_pair *pairs, ofv_graph **out);

/* Dimensions of pyramid level l (0 = full resolution). */
ofv_status ofv_level_shape(const ofv_handle *h, int level, int *H, int *W);

/* Copy level l of frame f (0 = I1, 1 = I2) of the last computed pair, as
   dense FP32, into dst (device, level H x W floats). */
ofv_status ofv_read_level(ofv_handle *h, int frame, int level, float *dst, ofv_stream_t s);

/* ---- kernel timing --------------------------------------------------- */
/* Kernel classes reported by ofv_profile_read. */
typedef enum {
    OFV_K_INGEST = 0,   /* scale (+ normalize, + pre-filter) into level 0 */
    OFV_K_REDUCE = 1,   /* one pyramid reduction, both frames */
    OFV_K_ITERATE = 2,  /* one Gauss-Newton iteration of one level (the fused kernel,
                           or the group of kernels of the plain path) */
    OFV_K_COUNT = 3
} ofv_kernel_class;

/* enable != 0: from now on every launch of this handle is bracketed by CUDA
   events on its stream; disable to stop.  Enabling clears earlier records. */
ofv_status ofv_profile_enable(ofv_handle *h, int enable);

/* Synchronise the recorded events and report, for kernel class k, the total
   device time (ms), the number of launches and the algorithmic bytes those
   launches must move (inputs read once, outputs written once). */
ofv_status ofv_profile_read(ofv_handle *h, int k, double *total_ms, int64_t *launches,
                            double *alg_bytes);

/* Message describing the most recent failure in the calling thread.  It
   takes no handle: errors are recorded per thread, so a failed ofv_create
   (which has no handle to return) reports through the same call. */
const char *ofv_last_error(void);

/* Name of a status code. */
const char *ofv_status_string(ofv_status s);

/* Library version, major * 10000 + minor * 100 + patch. */
int ofv_version(void);

#ifdef __cplusplus
}
#endif
#endif /* OFV_H */
