// Internal structures of the batched screening path (see batch.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace scr {

struct BImage {                        // one image's tables (low planes) and mask layout
    const uint32_t *L1, *L2, *T1, *T2;
    int64_t pitch;                     // words per table row
    int32_t H, W, Wwords, pad;
    int64_t mask_offset;               // first word of this image in the union mask
    // units of this image: one per (row, group), row-major, so the blocks that
    // run together read the same table rows for every radius and the tables
    // stream from DRAM about once
    int64_t unit0;                     // first unit of the image
    int32_t y_first, rows;             // rows y_first .. y_first + rows - 1
    int32_t g0, n_grp;                 // groups g0 .. g0 + n_grp - 1 belong to this image
};

struct BGroup {                        // one (image, star radius R) and the records testing it
    int32_t image, R;
    int32_t y_lo, y_hi, x_lo, x_hi;    // valid candidates (inclusive)
    int32_t w_lo, w_hi;                // mask words covering [x_lo, x_hi]
    int32_t oL[4], oT[4], oLi[4], oTi[4];   // corner offsets for this image's pitch
    uint32_t A, Ain, Aring;
    uint32_t S_lo_hull, S_rng_hull;    // union of the records' mean intervals
    uint32_t need;                     // features any record of the group tests
    int32_t rec0, rec1;                // records [rec0, rec1)
    uint32_t all_var;                  // 1: every record tests the variance
    int64_t V_lo_hull;                 // with all_var: union of the records' variance
    uint64_t V_rng_hull;               //   intervals, (V - V_lo_hull) <= V_rng_hull
};

struct BRecord {                       // one (pair, scale) test
    uint32_t pair, s, features;
    uint32_t S_lo, S_rng;
    int64_t V_lo;
    uint64_t V_rng;
    int64_t N_lo;
    uint64_t N_rng;
};

struct BatchArgs {
    const BImage *images;
    const BGroup *groups;
    const BRecord *records;
    int32_t n_images;
    int32_t n_groups;
    int64_t n_units;                   // units this launch processes
    int64_t unit_stride;               // unit u of the launch is unit u * unit_stride of the plan
    uint64_t *counts;                  // per pair
    uint32_t *union_mask;              // per image [H][Wwords], may be null
    uint64_t *keys;
    uint64_t keys_cap;
    uint64_t *n_reserved;              // key slots handed out (chunks of kKeyChunk)
    uint64_t *next_unit;               // next unit to hand out (zero before the launch)
};

constexpr int kBatchWarpsPerBlock = 8;     // warps of a k_batch block
constexpr uint64_t kKeySentinel = ~0ull;   // fills unused reserved slots; sorts last
constexpr int kKeyChunk = 256;             // key slots a warp reserves at a time

struct SortArgs {
    uint64_t *src, *dst;               // ping-pong key buffers (src holds the unsorted keys)
    uint32_t *hist;                    // [256][tiles] digit counts, then chunk-local offsets
    uint64_t *csum;                    // per scan chunk: sum, then exclusive offset
    const uint64_t *n_keys;            // slots to sort (clamped to cap)
    uint64_t cap;
    uint64_t max_tiles;
    // sort on the key's fields packed to their used widths (column, row, scale,
    // pair), so fewer 8-bit passes are needed; each field keeps its rank
    uint32_t xb, yb, sb, pb;
};

cudaError_t launch_batch(const BatchArgs &a, int words_per_warp, int grid, cudaStream_t st, uint64_t *launches);
size_t sort_hist_bytes(uint64_t cap);
size_t sort_csum_bytes(uint64_t cap);
uint64_t sort_max_tiles(uint64_t cap);
constexpr int kSortLaunchesPerPass = 5;
// passes 8-bit passes; the result is in a.src after an even number, a.dst after an odd one
cudaError_t launch_sort(const SortArgs &a, int passes, int grid, cudaStream_t st, uint64_t *launches);
// For each pair k < n: out[stage[2k + 1] + i] = the single-image key (s << 48) | (y << 24) | x of
// sorted batched key offsets[k] + i, for i < min(counts[k], stage[2k]); then out_counts[k] =
// counts[k] and out_counts[n + 0..1] = total[0..1].  stage, out and out_counts may be host-mapped.
cudaError_t launch_gather_lists(const uint64_t *keys, const uint64_t *counts, const uint64_t *offsets,
                                const uint64_t *total, const uint64_t *stage, uint64_t *out, uint64_t *out_counts,
                                int n, int grid, cudaStream_t st, uint64_t *launches);
// keys[i] = the single-image key (s << 48) | (y << 24) | x of batched key i, for i < min(*n, cap)
cudaError_t launch_keys_to_lists(uint64_t *keys, const uint64_t *n, uint64_t cap, int grid, cudaStream_t st,
                                 uint64_t *launches);
cudaError_t launch_pair_offsets(const uint64_t *counts, uint64_t *offsets, uint64_t *total, const uint64_t *reserved,
                                int n, cudaStream_t st, uint64_t *launches);

}  // namespace scr
