// Internal host runtime shared by the C ABI (api.cu) and the serving loop
// (serve.cu): the opaque handle types, the context's budgeted device pool,
// the exact per-scale bounds, table builds and the batched plan.
#pragma once

#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <vector>

#include "batch.h"
#include "internal.h"
#include "screen.h"

typedef __int128 i128;

namespace scr_rt {
// records the message returned by screen_last_error (thread-local) and returns code
int fail(int code, const char *fmt, ...);
const std::string &last_error();
}  // namespace scr_rt

#define CUDA_TRY(expr)                                                                     \
    do {                                                                                   \
        cudaError_t e__ = (expr);                                                          \
        if (e__ != cudaSuccess)                                                            \
            return scr_rt::fail(SCR_ECUDA, "%s: %s (%s)", #expr, cudaGetErrorName(e__),    \
                                cudaGetErrorString(e__));                                  \
    } while (0)

struct scr_tables {
    scr::TableDesc t[4];
    scr::FilterPlanes F;             // packed filter planes (screen_set_filter), inside [base, base + bytes)
    void *base = nullptr;
    size_t bytes = 0;
    int H = 0, W = 0;
    // Prewitt moment tables (build_moment_tables): 64-bit, same rows, pitch and
    // column offset as the upright tables (pitch in 64-bit words)
    void *mom = nullptr;
    size_t mom_bytes = 0;
    uint64_t *Mx = nullptr, *My = nullptr;
    cudaStream_t stream = nullptr;   // stream of the last use (frees are ordered on it)
};

struct scr_tmpl {
    int r = 0, t_min = 0;
    uint32_t features = 0;
    std::vector<int64_t> S, Q, Si;   // index t - t_min
    // hulls as exact rationals num/den (den > 0)
    int64_t mu_lo_n = 0, mu_lo_d = 1, mu_hi_n = 0, mu_hi_d = 1;
    int64_t v_lo_n = 0, v_lo_d = 1, v_hi_n = 0, v_hi_d = 1;
    int64_t g_lo_n = 0, g_lo_d = 1, g_hi_n = 0, g_hi_d = 1;
    // Prewitt (SCR_F_PREWITT): doubled moments of each central square, and the
    // hull of phi^2 = 4 n^2 (Gx2^2 + Gy2^2) / J2^2 as num/den
    std::vector<int64_t> Gx2, Gy2;
    unsigned __int128 p_lo_n = 0, p_lo_d = 1, p_hi_n = 0, p_hi_d = 1;
};

struct scr_batch;
struct scr_server;
struct scr_frames;

struct scr_ctx {
    int device = 0;
    uint64_t budget = 0;
    std::atomic<uint64_t> in_use{0}, peak{0}, launches{0};
    cudaMemPool_t pool = nullptr;
    std::mutex mu;
    std::set<scr_tables *> tables;
    std::set<scr_tmpl *> tmpls;
    std::set<scr_batch *> batches;
    std::set<scr_server *> servers;
    std::set<scr_frames *> frames;   // frame pipelines (frames_create)
    std::map<std::string, std::pair<int, int>> tuned;   // batch shape -> (words per warp, blocks per SM)
    uint64_t *pinned = nullptr;      // 8-byte pinned slot for counts
    uint64_t *pinned_dev = nullptr;  // the same slot as the device sees it (null if not mapped)
    // packed filter windows (kS, kQ) for the single-image builds (screen_set_filter)
    int n_filter = 0;
    int filter_k[scr::kMaxFilterWindows][2] = {{0, 0}, {0, 0}};
};

struct scr_batch {
    scr_ctx *ctx = nullptr;
    int n_images = 0, n_pairs = 0;
    std::vector<scr::BImage> images;
    std::vector<scr::BGroup> groups;
    std::vector<scr::BRecord> records;
    void *desc = nullptr;            // device copy of images, groups, records
    size_t desc_bytes = 0;
    void *sort_buf = nullptr;        // radix-sort histogram + ping-pong keys
    size_t sort_bytes = 0;
    scr::BatchArgs args = {};
    scr::SortArgs sargs = {};
    int sort_passes = 0;             // 8-bit radix passes over the packed keys
    int wpw = 8, blocks_per_sm = 4, grid = 0;
    int64_t n_units = 0;
    uint64_t candidates = 0;         // (record, valid position) pairs screened per run
    uint64_t *offsets = nullptr;
    uint64_t *n_keys = nullptr;      // caller's total-survivor count
    uint64_t *n_reserved = nullptr;  // device counters of reserved key slots and handed-out units (in sort_buf)
    uint64_t union_words = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace scr_rt {

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess)
            prev = -1;
        if (prev != dev)
            ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev)
            cudaSetDevice(prev);
    }
};

struct Geo {
    int n, h, ni, hi;
    int64_t A, Ain, Aring;
};

Geo geometry(int R);
int dev_alloc(scr_ctx *c, size_t bytes, cudaStream_t st, void **p);
void dev_free(scr_ctx *c, void *p, size_t bytes, cudaStream_t st);
int check_ctx(const scr_ctx *c);
int validate_params(const scr_params *p);
void bounds_for(const scr_tmpl *tm, const scr_params *p, int R, scr_bounds *b);
int64_t table_plane_words(int H, int W);
// device bytes of one image's four tables and n_filter pairs of packed filter planes
size_t tables_bytes(int H, int W, int sum_bits, int sq_bits, int n_filter = 0);
// the four tables (and the filter planes of the windows fk[0 .. n_filter)) of an
// H x W image laid out in the device block [base, base + bytes)
void layout_tables(scr_tables *t, void *base, size_t bytes, int H, int W, int sum_bits, int sq_bits,
                   cudaStream_t st, int n_filter = 0, const int (*fk)[2] = nullptr);
int alloc_tables(scr_ctx *c, int H, int W, int sum_bits, int sq_bits, cudaStream_t st, scr_tables **out,
                 int n_filter = 0, const int (*fk)[2] = nullptr);
int run_build(scr_ctx *c, const uint8_t *img, int H, int W, int64_t pitch, scr_tables *t, cudaStream_t st);
// as run_build with caller-provided scratch of TableScratch::bytes
int run_build_in(scr_ctx *c, const uint8_t *img, int H, int W, int64_t pitch, scr_tables *t, void *scratch,
                 cudaStream_t st);
void free_tables(scr_ctx *c, scr_tables *t);

// A device buffer charged to the context and returned on scope exit
// (stream-ordered on the stream it was taken on).
struct Scoped {
    scr_ctx *c;
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t st;
    Scoped(scr_ctx *c_, cudaStream_t st_) : c(c_), st(st_) {}
    int take(size_t b) {
        bytes = b;
        return dev_alloc(c, b, st, &p);
    }
    ~Scoped() { dev_free(c, p, bytes, st); }
};

int fill_screen_args(const scr_tables *t, const scr_tmpl *tm, const scr_params *p, scr::ScreenArgs *a);
int check_screen_inputs(const scr_tables *t, const scr_tmpl *tm, const scr_params *p);

// batched plan (see screen_batch_create)
void plan_layout(scr_batch *b);
int build_plan(scr_ctx *c, scr_batch *b, const scr_tables *const *tables, int n_images, const scr_tmpl *const *tmpls,
               const scr_params *params, int n_tmpls, const scr_pair *pairs, int n_pairs);
void pack_plan(const scr_batch *b, void *dst);   // the device descriptor image (desc_bytes) into dst
int upload_plan(scr_batch *b, cudaStream_t st);
size_t desc_size(const scr_batch *b);
void set_args(scr_batch *b);
int sm_count(int device);
int enqueue_run(scr_batch *b, cudaStream_t st, uint64_t *launches);
void free_batch(scr_ctx *c, scr_batch *b);
// frees a batch without graph whose buffers are stream-ordered on st (runs may be in flight there)
void free_batch_on(scr_ctx *c, scr_batch *b, cudaStream_t st);
// plan, device buffers and launch arguments of a batch (inputs already
// validated, context lock held); no tuning and no graph
int batch_prepare(scr_ctx *c, const scr_tables *const *tables, int n_images, const scr_tmpl *const *tmpls,
                  const scr_params *params, int n_tmpls, const scr_pair *pairs, int n_pairs, uint64_t *counts_dev,
                  uint64_t *offsets_dev, uint32_t *union_mask_dev, uint64_t *keys_dev, uint64_t keys_cap,
                  uint64_t *n_keys_dev, cudaStream_t st, scr_batch **out);
// launch shape and unit layout (host side; upload_plan copies it to the device)
void batch_set_shape(scr_batch *b, int wpw, int blocks_per_sm);
// serving loop (serve.cu)
void destroy_servers(scr_ctx *c);
// frame pipelines still alive at shutdown (api.cu)
void destroy_frames(scr_ctx *c);

}  // namespace scr_rt

namespace scr {
// Copy min(*count, cap) keys of a device list to dst and *count to count_out,
// both host memory the device can address (one kernel of `blocks` blocks;
// compact.cu).  A copy on the critical path uses kCopyBlocksSync; one that
// overlaps other work (the frame pipeline's, during the next frame) uses
// kCopyBlocksOverlapped, so that it holds few SM slots while the host link,
// not the SMs, sets its pace.  Measured on the 8192 x 8192 pipeline (2.2 M
// keys per frame): 2.51 ms per frame with 608 blocks, 2.48 with 152, 2.43
// with 38; one synchronous call took 2.875 ms with 608 and 2.883 with 38.
constexpr int kCopyBlocksSync = 608;
constexpr int kCopyBlocksOverlapped = 38;
cudaError_t launch_copy_keys(const uint64_t *src, const uint64_t *count, uint64_t cap, uint64_t *dst,
                             uint64_t *count_out, cudaStream_t st, uint64_t *launches, int blocks);
}  // namespace scr
