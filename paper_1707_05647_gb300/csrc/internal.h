// Internal declarations shared by the library's translation units.
// Nothing here is part of the C ABI (include/screen.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "screen.h"

namespace scr {

// ---------------------------------------------------------------------------
// Table storage.
//
// A table of R rows x C columns is stored as 32-bit words: element (a, b)
// lives at word a*pitch + b + kColOffset of the low plane; a 64-bit table
// has a second (high) plane plane_stride words after the low one.  The column
// offset of 3 puts column b = 1 on a 16-byte boundary, so the kernels store
// eight consecutive columns b = 8k+1 .. 8k+8 with two aligned 16-byte stores
// per plane.  pitch is a multiple of 32 words (128 bytes).
// ---------------------------------------------------------------------------
constexpr int kColOffset = 3;

struct TableDesc {
    uint32_t *lo = nullptr;   // low 32 bits (the whole value for 32-bit tables)
    uint32_t *hi = nullptr;   // high 32 bits, nullptr for 32-bit tables
    int64_t pitch = 0;        // words per row
    int64_t rows = 0, cols = 0;
    int bits = 32;
};

// Build geometry of the table kernels (see tables.cu).
constexpr int kBand = 32;                  // rows per band
constexpr int kTileSlots = 1024;           // accumulator columns per tile
constexpr int kHalo = kBand;               // halo columns on each side of a tile
constexpr int kTileCols = kTileSlots - 2 * kHalo;   // 960 core columns
constexpr int kWinLo = -34;                // first carry column kept per band

inline int64_t table_pitch_words(int64_t W) { return ((W + 16 + 31) / 32) * 32; }

// ---------------------------------------------------------------------------
// Packed filter planes (optional, screen_set_filter).  For a window (kS, kQ)
// element (a, b) of the upright plane holds bits kS .. kS+15 of L1(a, b) in its
// low half and bits kQ .. kQ+15 of L2(a, b) in its high half; the cone plane
// holds the same bits of T1 and T2.  Same rows, pitch and column offset as the
// tables.  A star's eight signed corners of one packed plane give its pooled
// sums of I and I^2 to within a few units of 2^kS and 2^kQ, which is enough
// to reject most candidates before any exact corner is read (features.cu).
// ---------------------------------------------------------------------------
constexpr int kMaxFilterWindows = 2;
constexpr int kMaxFilterShiftS = 14;   // kS in 0 .. 14: the filter's sum bounds stay inside 32-bit integers
constexpr int kMaxFilterShiftQ = 16;   // kQ in 0 .. 16: the window's bits stay inside the low 32-bit plane
struct FilterPlanes {
    int n = 0;                                       // windows written (0 .. kMaxFilterWindows)
    uint32_t *up[kMaxFilterWindows] = {nullptr, nullptr};
    uint32_t *cone[kMaxFilterWindows] = {nullptr, nullptr};
    int kS[kMaxFilterWindows] = {0, 0}, kQ[kMaxFilterWindows] = {0, 0};
};

// ---------------------------------------------------------------------------
// Screening parameters handed to the feature kernel (one record per scale).
// ---------------------------------------------------------------------------
constexpr int kMaxScales = 32;

// Per-scale record, precomputed on the host.  Corner offsets are element
// offsets relative to the candidate's own element (y, x) of the table (both
// table kinds share one pitch), so the kernel forms each corner address with
// one multiply-add from a per-thread base pointer.  Interval tests use the
// unsigned-range form (v - lo) <= (hi - lo).
struct ScaleParam {
    int32_t y_lo, y_hi, x_lo, x_hi;   // valid candidate rectangle (inclusive)
    int32_t oL[4];                    // square corners: (+n+1,+n+1) (-n+1,+n+1) (+n+1,-n+1) (-n+1,-n+1)
    int32_t oT[4];                    // diamond corners: (h+1, 1) (1, 1-h) (1, h+1) (1-h, 1)
    int32_t oLi[4], oTi[4];           // the same for the inner star (radius floor(R/2))
    uint32_t S_lo, S_rng;             // mean:     (S - S_lo) <= S_rng        (32-bit)
    uint32_t A, Ain, Aring;           // pooled areas
    uint32_t empty;                   // 1: an interval is empty, nothing survives
    int64_t V_lo;
    uint64_t V_rng;                   // variance: (V - V_lo) <= V_rng       (64-bit)
    int64_t N_lo;
    uint64_t N_rng;                   // contrast: (N - N_lo) <= N_rng       (64-bit)
    unsigned __int128 P_lo, P_rng;    // Prewitt:  (Gx2^2 + Gy2^2 - P_lo) <= P_rng (128-bit)
    // packed-plane pre-filter (FilterPlanes): window index, -1 for none, and
    // its single-precision constants (see filter_pass in features.cu)
    int32_t fw;
    float f2S, fS0;                   // 2^kS, -2^kS (2^23 + 8)
    float fSlo;                       // mean lower bound, at least 0, rounded down
    float fc, fQ0;                    // A 2^kQ, -A 2^kQ 2^23
    float fVlo;                       // variance lower bound lowered by the rounding margin
};

struct ScreenArgs {
    const uint32_t *L1, *L2, *T1, *T2;   // low planes (window sums read mod 2^32)
    const uint32_t *FU[kMaxFilterWindows], *FC[kMaxFilterWindows];   // packed planes (upright, cone)
    const uint64_t *Mx, *My;             // Prewitt moment tables (with SCR_F_PREWITT)
    int64_t pitch;                       // words per row (all four tables)
    int32_t H, W, Wwords, n_scales;
    uint32_t features;
    uint32_t *mask;
    ScaleParam sp[kMaxScales];
};

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  Every kernel of the library begins with
// pdl_begin(): it waits until the grids it depends on have completed and their
// memory is visible (no memory operation of the kernel precedes the wait), then
// lets the next kernel in the stream be scheduled.  Kernels are launched with
// launch_pdl(), so a kernel's CTAs are placed on the GPU while its predecessor
// drains instead of after it has fully retired.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st,
                              Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------------------
// Launchers (return cudaError_t of the launch).  `launches` is incremented by
// the number of kernels enqueued.
// ---------------------------------------------------------------------------
struct TableScratch {
    // sizes in bytes of the scratch regions the table build needs
    static size_t bytes(int H, int W, int sum_bits, int sq_bits);
};

cudaError_t launch_build_tables(const uint8_t *img, int H, int W, int64_t pitch,
                                const TableDesc &L1, const TableDesc &L2, const TableDesc &T1,
                                const TableDesc &T2, const FilterPlanes &F, void *scratch, cudaStream_t st,
                                uint64_t *launches);

cudaError_t launch_template_sums(const TableDesc &L1, const TableDesc &L2, const TableDesc &T1,
                                 const TableDesc &T2, int r, int t_min, int64_t *out_dev,
                                 cudaStream_t st, uint64_t *launches);

cudaError_t launch_screen(const ScreenArgs &args, cudaStream_t st, uint64_t *launches);

// Joint-vector membership screen (joint.cu).
struct JointScale {                   // per scale: valid rectangle of the outermost area
    int32_t y_lo, y_hi, x_lo, x_hi;
    uint32_t empty, pad[3];
};
struct JointArea {                    // per (scale, area): corner offsets and areas of its star
    int32_t oL[4], oT[4], oLi[4], oTi[4];
    uint32_t A, Ain, Aring, pad;
    uint32_t S_lo, S_rng;             // star sums whose mean cell lies in the set's range
};
struct JointSet {                     // per area: the membership bit array over cell vectors
    uint64_t bit0;                    // first bit in the shared bit array
    int32_t cmin[3];                  // lowest cell of each enabled feature (in mean, std, contrast order)
    uint32_t dim[3];                  // cells per enabled feature (index = sum (c - cmin) * stride)
};
struct JointArgs {
    const uint32_t *L1, *L2, *T1, *T2;   // low planes
    int64_t pitch;
    int32_t H, W, Wwords, n_scales, n_areas;
    uint32_t features;
    uint64_t qn[3], qd[3];                // quantisation factors q = qn / qd: mean, std, contrast
    const JointScale *scales;             // [n_scales]
    const JointArea *areas;               // [n_scales][n_areas]
    const JointSet *sets;                 // [n_areas]
    const uint32_t *bits;
    uint32_t *mask;
};
cudaError_t launch_screen_joint(const JointArgs &a, cudaStream_t st, uint64_t *launches);

// Prewitt moment tables (moments.cu)
size_t moment_scratch_bytes(int H, int W);
cudaError_t launch_moment_tables(const uint8_t *img, int64_t ipitch, int H, int W, int64_t pitch, uint64_t *Mx,
                                 uint64_t *My, void *scratch, cudaStream_t st, uint64_t *launches);

size_t compact_scratch_bytes(uint64_t total_words);
cudaError_t launch_compact(const uint32_t *mask, uint64_t total_words, int H, int Wwords,
                           uint64_t *list, uint64_t cap, uint64_t *count, void *scratch,
                           cudaStream_t st, uint64_t *launches);

// Square half-side n of star radius R: (2n-1)^2 < 2R^2 < (2n+1)^2.
int square_half(int R);

}  // namespace scr
