/*
 * screen.h -- C ABI of the GPU screening library (libscreen.so).
 *
 * The library implements the data-parallel hot path of the rotation- and
 * scale-invariant template-matching pre-screener of Liu, Shu and Wu,
 * "Fast Screening Algorithm for Rotation and Scale Invariant Template
 * Matching" (arXiv 1707.05647):
 *
 *   a1  upright summed-area tables of I and I^2        (Sec. 3, Eq. T_1, S_sigma)
 *   a2  45-degree ("cone") summed-area tables of I, I^2 (Sec. 4, triangular map)
 *   a3  octagonal-star features at every position and scale by table-corner
 *       lookups: mean, variance, inner-star-vs-ring contrast
 *                                         (Sec. 3 Eq. S_1; Sec. 4 Eq. S_os; Sec. 5)
 *   a4  threshold against the template's feature bounds -> candidate bitmask
 *                                         (Sec. 5, Algorithm 1)
 *   a5  compaction of the bitmask -> ascending list of surviving candidates
 *                                         (Sec. 5, Algorithm 1, R <- R u {P})
 *
 * Every result is an exact integer: the tables are exact modulo 2^w, window sums
 * are exact whenever they are below 2^32 (checked per scale), and the threshold
 * tests compare integers against bounds computed from exact rationals, so the
 * mask and the list are bit-exact against any correct implementation.
 *
 * Geometry (definitions used throughout):
 *   Image I: H x W uint8, row y (slow index), column x.
 *   Star radius R >= 1: diamond half-diagonal h = R, square half-side n = the
 *   unique integer with (2n-1)^2 < 2R^2 < (2n+1)^2; star = square (rows
 *   y-n+1..y+n, columns x-n+1..x+n) superposed on the diamond (pixels with
 *   |x'-x| < h and y-h+|x'-x| < y' <= y+h-|x'-x|); sums pooled over area
 *   A = 4n^2 + 2h^2.  Inner star: radius floor(R/2).  A candidate (y, x) is
 *   valid when its whole star lies inside the image.
 *
 * Conventions:
 *   - Every entry point returns SCR_OK (0) or a negative SCR_E* code; the
 *     message of the last failure on the calling thread is screen_last_error().
 *     No C++ exception crosses the ABI.  On failure, outputs are unspecified.
 *   - "_dev" pointers are CUDA device pointers on the context's device; they are
 *     owned by the caller unless stated otherwise.  "_host" pointers are host
 *     memory.  Handles (scr_tables, scr_tmpl) are owned by the library and freed
 *     by their *_release call; their device memory counts against the context's
 *     HBM budget.
 *   - A stream argument is a cudaStream_t (NULL = the legacy default stream).
 *     Calls are stream-ordered and return without waiting unless documented.
 *   - A context may be used from several host threads; calls are serialised
 *     on the context's host-side state.
 *   - There is no CPU fallback: if the device is missing or the kernels cannot
 *     run, calls fail with SCR_ECUDA.
 */
#ifndef SCREEN_H
#define SCREEN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct scr_ctx scr_ctx;
typedef struct scr_tables scr_tables;
typedef struct scr_tmpl scr_tmpl;
typedef void *scr_stream; /* cudaStream_t */

enum {
    SCR_OK = 0,
    SCR_EINVAL = -1,      /* bad argument (sizes, null pointers, radii, tolerances) */
    SCR_ENOMEM = -2,      /* device or host allocation failed */
    SCR_EBUDGET = -3,     /* the allocation would exceed the context's HBM budget */
    SCR_ECUDA = -4,       /* a CUDA runtime call or kernel launch failed */
    SCR_ETIMEOUT = -5,    /* reserved: a bounded device-side wait gave up */
    SCR_EOVERFLOW = -6,   /* more survivors than list capacity (mask still complete) */
    SCR_EEVICTED = -7,    /* the image's tables and host copy were dropped (server_forget) */
    SCR_EUNSUPPORTED = -8 /* valid request outside what the library implements */
};

enum { SCR_F_MEAN = 1, SCR_F_VAR = 2, SCR_F_GRAD = 4, SCR_F_PREWITT = 8 };

/* Exact rational num/den, den > 0, |num| and den <= 2^20. */
typedef struct {
    int64_t num, den;
} scr_rat;

/* Screening parameters.
 *   radii[n_scales]: star radius R_s per scale (host array, 1 <= n_scales <= 32,
 *                    2 <= R_s <= 181 so that every window sum of I^2 is below 2^32).
 *   features:        OR of SCR_F_*; a candidate must pass every enabled test.
 *   mean_rel tm, std_rel ts, grad_rel tg (each in [0, 1)), grad_abs dg (>= 0):
 *     mean     S/A in [(1-tm) mu_lo, (1+tm) mu_hi]
 *     std      sqrt(V)/A in [(1-ts) sd_lo, (1+ts) sd_hi]         (compared squared)
 *     contrast N/(A_in A_ring) in [g_lo - tg|g_lo| - dg, g_hi + tg|g_hi| + dg]
 *   where [mu_lo, mu_hi], ... are the template's feature hulls over its central
 *   radii t in [t_min, r] (Sec. 5, Eq. F_n; see template_features).
 *   prewitt_rel tp (in [0, 1)), prewitt_abs dp (>= 0), used with SCR_F_PREWITT:
 *     the Prewitt gradient of the star's 2n x 2n square (Sec. 3, Eq. S_y and
 *     Eq. T_x; magnitude of Sec. 4) about the square's centre (y + 1/2, x + 1/2),
 *     Gx2 = sum (2x' - 2x - 1) I, Gy2 = sum (2y' - 2y - 1) I, J2 = (2n)^2 (4n^2 - 1)/3,
 *     phi^2 = 4 n^2 (Gx2^2 + Gy2^2) / J2^2 (slope times half-side, squared), and
 *     phi^2 in [max(0, (1-tp)^2 p_lo - dp^2), (1+tp)^2 p_hi + dp^2] with [p_lo, p_hi]
 *     the hull of the template's central squares' phi^2.  Needs moment tables
 *     (build_moment_tables) and a template computed with SCR_F_PREWITT. */
typedef struct {
    int32_t n_scales;
    const int32_t *radii;
    uint32_t features;
    scr_rat mean_rel, std_rel, grad_rel, grad_abs;
    scr_rat prewitt_rel, prewitt_abs;
} scr_params;

/* Inclusive integer bounds of one scale (INT64_MIN / INT64_MAX when the
 * feature is disabled).  S = pooled star sum, V = A*Q - S^2, N = S_in*A_ring -
 * S_ring*A_in. */
typedef struct {
    int64_t S_lo, S_hi, V_lo, V_hi, N_lo, N_hi;
} scr_bounds;

typedef struct {
    uint64_t kernel_launches; /* kernels launched by this context so far */
    uint64_t bytes_in_use;    /* live device bytes charged to the budget */
    uint64_t bytes_peak;      /* high-water mark of bytes_in_use */
    uint64_t budget;          /* the HBM budget given to screen_init */
} scr_stats;

/* ---- context ---------------------------------------------------------- */

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the device
 * memory the context may hold at once (0 = no cap).  Fails with SCR_ECUDA if
 * the device is absent or not an sm_103 part the kernels were built for. */
int screen_init(scr_ctx **ctx, int device, uint64_t hbm_budget_bytes);

/* Wait for the context's work, free every handle it still owns, destroy it. */
void screen_shutdown(scr_ctx *ctx);

/* Message of the last failed call on this host thread ("" if none).  The
 * pointer stays valid until the thread's next failing call. */
const char *screen_last_error(void);

int screen_stats(const scr_ctx *ctx, scr_stats *out);

/* ---- a1, a2: tables --------------------------------------------------- */

/* Build the four tables of the H x W image at img_dev (row pitch `pitch` bytes,
 * pitch >= W), 1 <= H, W <= 65535.
 *   which 0: L1, upright table of I,   (H+1) x (W+1), L[a][b] = sum_{y<a,x<b} I(y,x)
 *   which 1: L2, upright table of I^2, (H+1) x (W+1)
 *   which 2: T1, cone table of I,      (H+1) x (W+2), T[a][b] = cone(a-1, b-1),
 *            cone(r,c) = sum of I(y,x) over y <= r, |x-c| <= r-y (inside the image)
 *   which 3: T2, cone table of I^2
 * L1 and T1 are stored with sum_bits, L2 and T2 with sq_bits (32 or 64); values
 * are exact modulo 2^bits.  (Sec. 3, Eq. T_1: built in linear time by row and
 * column passes; Sec. 4: the rotated table by two diagonal passes.)
 * Stream-ordered on `stream`; the image must stay valid until the work ends. */
int build_tables(scr_ctx *ctx, const uint8_t *img_dev, int32_t H, int32_t W, int64_t pitch,
                 int32_t sum_bits, int32_t sq_bits, scr_stream stream, scr_tables **out);

/* Packed filter planes for later single-image table builds (an implementation
 * device of this library; the paper has no counterpart).  windows holds
 * n_windows (0..2) pairs (kS, kQ), 0 <= kS <= 14, 0 <= kQ <= 16.  Tables built
 * afterwards by build_tables, screen_host and frames_create on this context
 * carry, per window, one extra 32-bit upright plane and one cone plane:
 * element (a, b) holds bits kS..kS+15 of L1 (T1) in its low half and bits
 * kQ..kQ+15 of L2 (T2) in its high half.  screen_positions / screen_features
 * on such tables first bound each candidate's pooled sums S and Q from its
 * star's eight packed corners (8 reads instead of the 16 exact ones), reject
 * the candidates whose variance is certainly below the variance interval,
 * and read the exact corners only where a candidate is left.  Each scale uses
 * the narrowest window whose range holds every candidate that can pass its
 * mean and variance intervals and that is at most 3 bits coarser than the
 * scale's smallest such shifts (coarser ones reject little); scales with no
 * such window, screens without the variance test and the Prewitt variant
 * read exact corners only.  Masks
 * and lists are unchanged (bit-exact).  The planes cost 8 bytes per pixel per
 * window in the build; they pay when most candidates pass the mean test and
 * fail the variance test on a background flatter than the template (measured
 * on the 8192 x 8192, 16-scale workload: screen 2.6 -> 1.6 ms, build
 * 0.55 -> 0.79 ms); where the mean test already rejects most candidates they
 * only cost.  n_windows = 0 turns the planes off.  The batched and serving
 * paths ignore the setting; tables already built keep what they have.
 * SCR_EINVAL for bad counts or shifts. */
int screen_set_filter(scr_ctx *ctx, int32_t n_windows, const int32_t *windows);

/* Suggested windows for screening with template tm and parameters p (host
 * computation).  For every scale, the smallest shifts whose range holds the
 * candidates that can pass.  The widest window fits every scale; when
 * max_windows >= 2 and it is more than 3 bits coarser than some scale's
 * smallest shifts, a second window, the smallest that fits all those scales,
 * is returned first.  windows (host) must hold 2 * min(max_windows, 2)
 * int32 values; *n_windows (kS, kQ) pairs are written, 0 when the variance
 * test is off or max_windows is 0.  SCR_EINVAL for a null argument, a negative
 * max_windows or invalid parameters. */
int screen_filter_windows(const scr_tmpl *tm, const scr_params *p, int32_t max_windows, int32_t *windows,
                          int32_t *n_windows);

/* The packed window each scale of a screen with (t, tm, p) would use: writes
 * p->n_scales entries to window_per_scale (host), the window index or -1 when
 * the scale reads exact corners only (no planes, no window whose range holds
 * the candidates that can pass, an empty scale, no variance test, or the
 * Prewitt variant).
 * Host computation. */
int screen_filter_plan(const scr_tables *t, const scr_tmpl *tm, const scr_params *p, int32_t *window_per_scale);

/* Borrowed device view of table `which` (0..3; 6 + 2w and 7 + 2w: the upright
 * and the cone packed plane of filter window w, 32-bit).  Layout: 32-bit words;
 * element (a, b) of a 32-bit table is word a*pitch + b + offset of *dev_ptr,
 * where *dev_ptr points at word 0; a 64-bit table is two such planes, the low
 * 32 bits at *dev_ptr and the high 32 bits plane_stride words further.
 * rows x cols is the logical size; pitch and plane_stride are in 32-bit words. */
int tables_view(const scr_tables *t, int which, const void **dev_ptr, int64_t *rows,
                int64_t *cols, int64_t *pitch, int64_t *offset, int64_t *plane_stride,
                int32_t *bits);

/* Copy table `which` into a dense rows x cols uint64 host array (values zero-
 * extended from 32-bit tables); which 4 and 5 are the moment tables Mx and My
 * ((H + 1) x (W + 1), after build_moment_tables); 6 + 2w and 7 + 2w the packed
 * filter planes of window w.  Synchronous. */
int tables_copy_to_host(scr_ctx *ctx, const scr_tables *t, int which, uint64_t *dst_host);

void tables_release(scr_ctx *ctx, scr_tables *t);

/* ---- template side (Sec. 5, Eq. F_n) ----------------------------------- */

/* Features of a (2r+1) x (2r+1) template (host array, row-major, side = 2r+1,
 * 2 <= r <= 181): star sums S_t, Q_t, S_in,t of the central star of radius t at
 * the template centre (r, r) for every t in [t_min, r] (t_min >= 2 when
 * SCR_F_GRAD is used), and the hulls of mean, variance and contrast over t.
 * Computed on the device with the same table kernels; synchronous.  With
 * SCR_F_PREWITT also the doubled Prewitt moments of each central square and the
 * hull of their phi^2 (see scr_params), summed on the host from the pixels. */
int template_features(scr_ctx *ctx, const uint8_t *tmpl_host, int32_t side, int32_t r,
                      int32_t t_min, uint32_t features, scr_tmpl **out);

/* out[0..2] = S_t, Q_t, S_in,t of central radius t in [t_min, r]. */
int template_sums(const scr_tmpl *tm, int32_t t, int64_t out[3]);

void template_release(scr_ctx *ctx, scr_tmpl *tm);

/* Per-scale inclusive integer bounds (host computation, exact 128-bit
 * rationals).  out has p->n_scales entries. */
int screen_bounds(const scr_tmpl *tm, const scr_params *p, scr_bounds *out);

/* Add the moment tables of the Prewitt gradient to t: Mx(a, b) = sum_{y<a, x<b}
 * x I and My(a, b) = sum_{y<a, x<b} y I (Sec. 3, Eq. T_x), 64-bit, same rows,
 * pitch and column offset as the upright tables; img_dev is the image the
 * tables were built from.  Charged to the HBM budget; freed with the tables.
 * Stream-ordered. */
int build_moment_tables(scr_ctx *ctx, const uint8_t *img_dev, int32_t H, int32_t W, int64_t pitch,
                        scr_tables *t, scr_stream stream);

/* ---- a3, a4: features and threshold ------------------------------------ */

/* Evaluate every candidate (s, y, x) and write the bitmask
 *   mask_dev[(s*H + y)*ceil(W/32) + x/32] bit (x % 32) = candidate survives,
 * zero for invalid positions.  mask_words must be >= n_scales*H*ceil(W/32).
 * Stream-ordered. */
int screen_features(scr_ctx *ctx, const scr_tables *t, const scr_tmpl *tm, const scr_params *p,
                    uint32_t *mask_dev, uint64_t mask_words, scr_stream stream);

/* ---- joint-vector membership over nested central areas ------------------ */

/* The exact test of Sec. 5 (Algorithm 1 with the feature set F_n of Eq. F_n)
 * in place of per-feature intervals, for up to three central areas of every
 * candidate (the closing paragraphs of Sec. 5).  Each enabled feature of a star
 * (mean S/A, standard deviation sqrt(V)/A with V = A*Q - S^2, contrast
 * N/(A_in*A_ring)) is quantised with Q(f) = floor(f/q + 1/2) (q per feature,
 * in grey levels); area j's set F_j marks, for every template central radius t
 * in band[j], the cell vectors whose every component is Q(f_t - q/2) or
 * Q(f_t + q/2) (= floor(f_t/q) or floor(f_t/q) + 1); a candidate survives iff
 * the quantised vector of each of its areas is in that area's set. */
typedef struct {
    int32_t n_areas;            /* 1..3 */
    const int32_t *area_radii;  /* host [n_scales][n_areas]: star radius of area j at scale s,
                                   2 <= area_radii[s][j] <= radii[s] (area 0 is normally radii[s]) */
    int32_t band[3][2];         /* inclusive template central-radius band of each area, inside the
                                   template's [t_min, r] */
    scr_rat q[3];               /* quantisation factors (mean, std, contrast): 1 <= num <= 65536,
                                   1 <= den <= 16 */
} scr_joint;

/* Write the candidate mask (layout as screen_features) of the joint membership
 * screen.  p supplies radii and features (its tolerances are not used); the
 * template must cover every band and carry SCR_F_GRAD when contrast is on.
 * The sets are bit arrays over the cell ranges they span; SCR_EINVAL if they
 * would exceed 2^26 bits (quantisation too fine for the spread of the band).
 * Device memory for the sets comes from the context's pool.  Returns when the
 * mask is written (it synchronises the stream: the host copy of the sets is
 * released on return). */
int screen_joint(scr_ctx *ctx, const scr_tables *t, const scr_tmpl *tm, const scr_params *p,
                 const scr_joint *j, uint32_t *mask_dev, uint64_t mask_words, scr_stream stream);

/* ---- a5: compaction ----------------------------------------------------- */

/* Ascending keys (s << 48) | (y << 24) | x of the set bits of a mask laid out
 * as above, written to list_dev[0 .. min(count, list_cap)); the exact count is
 * written to *count_dev (device).  list_dev may be NULL when list_cap == 0.
 * Stream-ordered. */
int compact_mask(scr_ctx *ctx, const uint32_t *mask_dev, int32_t n_scales, int32_t H, int32_t W,
                 uint64_t *list_dev, uint64_t list_cap, uint64_t *count_dev, scr_stream stream);

/* Allocation-free variant of compact_mask, for callers that cannot allocate
 * device memory where they compact: real-time loops that must never enter an
 * allocator (an allocation can stall on the driver for an unbounded time),
 * processes whose device memory all belongs to another framework's allocator,
 * and embedded runtimes that fix every buffer when they start.  The paper has
 * no counterpart; this is a deployment convenience.
 *   Inputs, outputs and results are exactly those of compact_mask, on the
 *   CUDA device that is current for the calling thread; no context is used.
 *   Scratch: a fixed array of about 0.75 MiB inside the library, held by every
 *   GPU that loads the library until the process exits.  Masks of more than
 *   268435456 words (65536 chunks of 4096 words) are rejected with SCR_EINVAL.
 *   The call allocates nothing: no cudaMalloc, cudaFree or allocating library
 *   routine.  The first call on each device does a one-time set-up (it looks
 *   up the array's device address, which also creates the device's context if
 *   there is none yet); make that first call before any stream capture.  The
 *   set-up runs again on the first call after the device's context has been
 *   re-created (cudaDeviceReset), since the array may then have moved.
 *   All calls share the one array and it keeps the last call's contents (each
 *   call rewrites what it reads): calls whose work overlaps on the GPU (for
 *   example on two streams, or on one stream from two threads without
 *   ordering) race and must be ordered by the caller.
 *   Errors return SCR_E* codes; their message is compact_mask_noalloc_error(). */
int compact_mask_noalloc(const uint32_t *mask_dev, int32_t n_scales, int32_t H, int32_t W,
                         uint64_t *list_dev, uint64_t list_cap, uint64_t *count_dev, scr_stream stream);
const char *compact_mask_noalloc_error(void);

/* ---- a3..a5 together ----------------------------------------------------- */

/* The whole screen of Sec. 5, Algorithm 1 on resident tables: every candidate
 * (scale, position) whose features pass the template's bounds goes into the
 * result set R.  screen_features + compact_mask, then wait for the stream and
 * return the survivor count in *n_survivors (host).  Returns SCR_EOVERFLOW when the count
 * exceeds list_cap (the mask is complete and the list holds the first list_cap
 * keys). */
int screen_positions(scr_ctx *ctx, const scr_tables *t, const scr_tmpl *tm, const scr_params *p,
                     uint32_t *mask_dev, uint64_t mask_words, uint64_t *list_dev,
                     uint64_t list_cap, uint64_t *n_survivors, scr_stream stream);

/* As screen_positions, but the count goes to *count_dev and nothing waits. */
int screen_positions_async(scr_ctx *ctx, const scr_tables *t, const scr_tmpl *tm,
                           const scr_params *p, uint32_t *mask_dev, uint64_t mask_words,
                           uint64_t *list_dev, uint64_t list_cap, uint64_t *count_dev,
                           scr_stream stream);

/* ---- batched screening (many images x many templates) -------------------- */

/* One unit of batched work: screen image `image` with template `tmpl`. */
typedef struct {
    int32_t image, tmpl;
} scr_pair;

/* Launch shape of the batched kernel; words_per_warp 0 = autotune. */
typedef struct {
    int32_t words_per_warp; /* 2, 4 or 8 mask words (x 32 positions) per warp */
    int32_t blocks_per_sm;  /* persistent blocks per SM */
} scr_batch_tuning;

typedef struct {
    int64_t n_groups;       /* (image, star radius) groups */
    int64_t n_records;      /* (pair, scale) tests */
    int64_t n_units;        /* units of work (one row of one image x one star radius) */
    uint64_t candidates;    /* (pair, scale, valid position) candidates per run */
    int32_t words_per_warp, blocks_per_sm;
    uint64_t union_words;   /* words of the union mask */
    int32_t sort_passes;    /* 8-bit radix passes over the keys packed to their used widths */
    int32_t reserved;
} scr_batch_info;

typedef struct scr_batch scr_batch;

/* Plan a batched screen of n_pairs (image, template) pairs over n_images
 * tables handles and n_tmpls templates (params[t] gives template t's radii,
 * features and tolerances).  Every (pair, scale) becomes one test; tests are
 * grouped per image by star radius so each (position, radius) feature vector
 * is computed once and compared with every test of that radius (Sec. 5,
 * Algorithm 1, applied to many templates at once).  One run screens every
 * candidate (pair, scale, valid position) and writes, all caller-owned:
 *   counts_dev[n_pairs]   survivors per pair (exact);
 *   offsets_dev[n_pairs]  exclusive prefix of counts_dev (may be NULL);
 *   union_mask_dev        per image, in image order, H x ceil(W/32) words:
 *                         bit set when some template survives there at some
 *                         scale (may be NULL);
 *   keys_dev[keys_cap]    survivor keys (pair << 37) | (scale << 32) | (y << 16) | x
 *                         in ascending order, i.e. per pair in the (scale, row,
 *                         column) order of compact_mask;
 *   n_keys_dev[2]         [0] = the exact number of survivors (keys_dev[0 ..
 *                         n_keys_dev[0]) are the keys), [1] = key slots used.
 *                         Slots are handed out to warps 256 at a time, so [1]
 *                         can exceed [0] by at most about 290 per resident warp
 *                         (< 3 M); the list is complete iff [1] <= keys_cap,
 *                         otherwise the keys are unspecified (counts, offsets
 *                         and the union mask stay exact).
 * Images up to 65535 x 65535, n_pairs < 2^26.  tuning NULL (or words_per_warp
 * 0) autotunes the launch shape on this batch and caches the choice in the
 * context.  The run (zeroing, screening kernel, radix sort, offsets) is
 * captured once into a CUDA graph; the tables, templates and output buffers
 * must stay valid while the plan exists.  Synchronous. */
int screen_batch_create(scr_ctx *ctx, const scr_tables *const *tables, int32_t n_images,
                        const scr_tmpl *const *tmpls, const scr_params *params, int32_t n_tmpls,
                        const scr_pair *pairs, int32_t n_pairs, uint64_t *counts_dev,
                        uint64_t *offsets_dev, uint32_t *union_mask_dev, uint64_t *keys_dev,
                        uint64_t keys_cap, uint64_t *n_keys_dev, const scr_batch_tuning *tuning,
                        scr_stream stream, scr_batch **out);

/* Replay the plan's graph on `stream` (stream-ordered, no host sync). */
int screen_batch_run(scr_batch *b, scr_stream stream);

int screen_batch_info(const scr_batch *b, scr_batch_info *out);

void screen_batch_release(scr_ctx *ctx, scr_batch *b);

/* ---- serving loop ---------------------------------------------------------
 *
 * A server owns three threads, each with its own stream on the context's
 * device.  Clients upload images (the server keeps a host copy, or borrows the
 * caller's) and submit screen requests from any thread; both return at once
 * with a request id.  Two builder threads build the tables of uploaded images,
 * and rebuild from the host copy the tables of images evicted earlier: they admit
 * new tables by the table budget, evicting least recently used tables that no
 * queued or running screen holds, and waits for running screens to release
 * tables when the rest does not make room.  The screener thread serves the
 * screens whose tables are resident, in one of two modes:
 *   SCR_SERVE_BATCHED (continuous batching): whenever screens are ready and
 *   there is room in flight, it takes them all (at most max_batch) as one batch,
 *   orders the batch shortest first and enqueues every screen without waiting
 *   (the screening kernel into a stream-ordered mask, the compaction straight
 *   into mapped host memory); screens of at most 2^small_log2 candidate slots
 *   (scales x pixels) run on a higher-priority stream, so they overtake large
 *   screens already on the device; each screen completes as soon as its own
 *   work is done, while later batches are admitted.  In flight at most
 *   max_inflight screens and 4 GiB of their masks.
 *   SCR_SERVE_PLAIN: one screen_features + compact_mask per screen, each
 *   waited for before the next.
 * The builders' copies and table builds overlap on the device with both;
 * screens whose tables are being built join a later batch.  Each request's survivor list, in
 * compact_mask's key format and order, goes to the caller's host buffer.  A
 * request's result does not depend on which other requests share its batch, nor
 * on the mode.  This is the paper's screen (Sec. 5, Algorithm 1) served to many
 * clients; the paper has no serving loop. */
typedef struct scr_server scr_server;

enum { SCR_SERVE_BATCHED = 0, SCR_SERVE_PLAIN = 1 };

typedef struct {
    uint64_t table_budget_bytes; /* resident tables above this are evicted, LRU first; 0 = no limit */
    int32_t sum_bits, sq_bits;   /* table widths for every image (32 or 64) */
    int32_t mode;                /* SCR_SERVE_BATCHED or SCR_SERVE_PLAIN */
    int32_t max_batch;           /* most requests per batch; 0 = every queued request */
    int32_t start_held;          /* 1: queue requests without serving them until server_hold(s, 0) */
    int32_t small_log2;          /* batched: priority lane for screens of <= 2^small_log2 candidate slots (0 = 24) */
    int32_t max_inflight;        /* batched: screens enqueued and not yet complete, at most (0 = 64) */
    int32_t reserved;
} scr_server_config;

typedef struct {
    int32_t status;     /* SCR_OK; SCR_EOVERFLOW (list truncated to list_cap, count exact); or an error */
    int32_t kind;       /* 0 upload (tables built), 1 screen, 2 evict */
    uint64_t count;     /* survivors of a screen */
    int64_t arrival_ns; /* the arrival stamp given at submission (server_clock_ns clock) */
    int64_t start_ns;   /* when the worker took the request's batch */
    int64_t done_ns;    /* when the result was written */
    uint64_t batch;     /* sequence number of the batch that served it */
    int32_t batch_size; /* requests in that batch */
    int32_t built;      /* 1 when this request built or rebuilt tables */
} scr_request_result;

typedef struct {
    uint64_t requests, batches, uploads, screens;
    uint64_t builds, rebuilds, evictions;
    uint64_t resident_images, resident_bytes, peak_resident_bytes;
    uint64_t mask_bytes;         /* device bytes of the plain path's mask buffer */
    uint64_t launches;           /* kernels the server launched */
    uint64_t build_ns;           /* time the builders spent on uploads, rebuilds and evictions (summed), of which: */
    uint64_t build_copy_ns;      /*   copying images to the device */
    uint64_t build_alloc_ns;     /*   allocating tables */
    uint64_t build_run_ns;       /*   building tables (launch to completion) */
    uint64_t build_gpu_ns;       /*   of which the device ran the builds (events) */
    uint64_t screen_ns;          /* time the screener spent running batches, of which: */
    uint64_t plan_ns;            /*   planning and launching (host) */
    uint64_t wait_ns;            /*   waiting for the device */
    uint64_t copy_ns;            /*   copying results to the callers' buffers */
} scr_server_stats;

/* CLOCK_MONOTONIC in nanoseconds: the clock of arrival, start and done stamps. */
int64_t server_clock_ns(void);

/* Create a server on ctx (screen_shutdown destroys servers still open).  An
 * image whose tables alone exceed table_budget_bytes fails with SCR_EBUDGET. */
int server_create(scr_ctx *ctx, const scr_server_config *cfg, scr_server **out);

/* Queue an upload: H x W uint8 at img_host (pitch bytes per row).  borrow = 0
 * copies the pixels now (the caller may reuse its buffer at once); borrow = 1
 * keeps the pointer, which must stay valid until server_forget or destroy.
 * *image_id names the image from now on; the request completes when its tables
 * are built.  arrival_ns = 0 stamps the call time. */
int server_upload(scr_server *s, const uint8_t *img_host, int32_t H, int32_t W, int64_t pitch, int32_t borrow,
                  int64_t arrival_ns, int64_t *image_id, uint64_t *request_id);

/* Queue a screen of image image_id against tm with params p (copied, radii
 * included; tm must stay valid until the request completes).  list_host
 * (caller-owned host memory, list_cap keys, may be NULL with list_cap 0) gets
 * the first list_cap survivor keys (s << 48) | (y << 24) | x in ascending order. */
int server_screen(scr_server *s, int64_t image_id, const scr_tmpl *tm, const scr_params *p, uint64_t *list_host,
                  uint64_t list_cap, int64_t arrival_ns, uint64_t *request_id);

/* Queue an eviction of the image's tables (the host copy stays; a later
 * screen rebuilds them). */
int server_evict(scr_server *s, int64_t image_id, uint64_t *request_id);

/* Drop the image: its tables when the worker next runs, and the host copy.
 * Screens queued or submitted later on it complete with SCR_EEVICTED. */
int server_forget(scr_server *s, int64_t image_id);

/* Wait up to timeout_us (< 0: forever) for the request; on completion write its
 * result and forget the id.  SCR_ETIMEOUT if still pending, SCR_EINVAL for an
 * unknown or already collected id. */
int server_wait(scr_server *s, uint64_t request_id, int64_t timeout_us, scr_request_result *out);

/* Wait up to timeout_us (< 0: forever) for any completed request not yet
 * collected, in completion order; write its id and result and forget it.
 * SCR_ETIMEOUT if none completes in time. */
int server_next(scr_server *s, int64_t timeout_us, uint64_t *request_id, scr_request_result *out);

/* hold = 1: the screener takes no new batch (the one running completes; the
 * builders keep building); hold = 0: screening resumes. */
int server_hold(scr_server *s, int32_t hold);

/* *resident = 1 when the image's tables are on the device now. */
int server_resident(scr_server *s, int64_t image_id, int32_t *resident);

int server_stats(scr_server *s, scr_server_stats *out);

/* Finish every queued request, stop the worker and free the server. */
void server_destroy(scr_server *s);

/* Eviction policy of the serving loop, pure host code: among n resident tables
 * with sizes bytes[i], last-use stamps last_use[i] (larger = more recent) and
 * pinned[i] != 0 for tables the current batch uses, pick victims least
 * recently used first (ties: lower index first), skipping pinned ones, until
 * resident - freed + need <= budget.  Writes their indices in eviction order
 * to victims (room for n) and their number to *n_victims.  Returns SCR_EBUDGET
 * when evicting every unpinned table is not enough (then *n_victims = 0). */
int server_lru_victims(const uint64_t *bytes, const uint64_t *last_use, const int32_t *pinned, int32_t n,
                       uint64_t resident, uint64_t budget, uint64_t need, int32_t *victims, int32_t *n_victims);

/* ---- whole path from host memory ----------------------------------------- */

/* End-to-end call for host-resident data: copy the image (host, pitch bytes per
 * row) to the device, build its tables, screen it against the template, and
 * return the count and the first list_cap keys in list_host.  When list_host
 * is pinned, mapped host memory (cudaHostAlloc / cudaMallocHost), the device
 * writes the keys into it directly and the call synchronises once; otherwise
 * the count and the keys are copied back.  Device buffers come from the
 * context's pool and are returned before the call ends.  Synchronous; returns
 * SCR_EOVERFLOW like screen_positions. */
int screen_host(scr_ctx *ctx, const uint8_t *img_host, int32_t H, int32_t W, int64_t pitch,
                int32_t sum_bits, int32_t sq_bits, const scr_tmpl *tm, const scr_params *p,
                uint64_t *list_host, uint64_t list_cap, uint64_t *n_survivors,
                scr_stream stream);

/* ---- a stream of same-sized host images (video frames) -------------------- */

/* The whole path of screen_host for a sequence of H x W host images screened
 * against one template with one parameter set, as in the paper's tracking use
 * (Sec. 6: every frame of a video screened for the target): Algorithm 1 on each
 * frame, with the copy of frame k+1 to the device overlapping the tables,
 * screen and compaction of frame k.
 *
 * frames_create reserves, once, every device buffer the path needs (depth image
 * slots of H x W bytes, one set of four tables, the table-build and compaction
 * scratch, one S x H x ceil(W/32) mask, a list of list_cap keys), charged to
 * the context's budget, and two streams of its own (copies; compute).  depth
 * (1..4) is the number of frames that may be in flight: 2 overlaps one copy
 * with one computation.  The template and the parameters are copied; the
 * template handle must outlive the pipeline.  SCR_EINVAL for bad geometry,
 * widths or parameters, SCR_EBUDGET / SCR_ENOMEM when the buffers do not fit.
 *
 * frames_submit queues one frame: img_host (H rows of W bytes, pitch bytes
 * apart; pinned memory makes the copy asynchronous) and list_host, room for
 * list_cap keys (s << 48) | (y << 24) | x in pinned host memory the device can
 * address (cudaHostAlloc / cudaMallocHost), into which the device writes the
 * frame's ascending survivor keys.  Both buffers belong to the pipeline until
 * frames_wait returns for that frame: the caller must neither change img_host
 * nor read list_host before then.  Returns the frame's ticket (0, 1, 2, ... in
 * submission order).  SCR_EINVAL when depth frames are already in flight (wait
 * for the oldest first) or list_host is not device-addressable pinned memory
 * (list_cap > 0); list_host may be NULL when list_cap is 0 (count only).
 *
 * frames_wait blocks until the frame with the given ticket is done and returns
 * its survivor count; tickets are waited for in submission order (SCR_EINVAL
 * otherwise).  SCR_EOVERFLOW when the count exceeds list_cap (the first
 * list_cap keys are in list_host, *n_survivors is the true count).
 *
 * frames_destroy waits for every frame in flight and frees the pipeline; so
 * does screen_shutdown for pipelines still alive.  One pipeline may be used
 * from several host threads (calls are serialised on it). */
typedef struct scr_frames scr_frames;
int frames_create(scr_ctx *ctx, int32_t H, int32_t W, int32_t sum_bits, int32_t sq_bits, const scr_tmpl *tm,
                  const scr_params *p, uint64_t list_cap, int32_t depth, scr_frames **out);
int frames_submit(scr_frames *f, const uint8_t *img_host, int64_t pitch, uint64_t *list_host, int64_t *ticket);
int frames_wait(scr_frames *f, int64_t ticket, uint64_t *n_survivors);
void frames_destroy(scr_frames *f);

#ifdef __cplusplus
}
#endif

#endif /* SCREEN_H */
