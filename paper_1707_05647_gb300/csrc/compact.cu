// Compaction of the candidate bitmask into the ascending list of surviving
// candidates (Sec. 5, Algorithm 1: R <- R u {P} for every patch that passes).
//
// The list order is the mask order (scale, row, column), so an exclusive scan
// of per-word popcounts gives every set bit its final slot; ties cannot occur
// and the list is identical to any correct compaction.  Three launches, no
// inter-CTA waiting: per-chunk counts, one scan of the chunk counts, and a
// per-chunk scan + scatter.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>

#include "internal.h"

namespace scr {
namespace {

constexpr int kThreads = 256;
constexpr int kWordsPerThread = 16;
constexpr int kChunk = kThreads * kWordsPerThread;   // 4096 words per block

__device__ __forceinline__ void load_words(const uint32_t *mask, uint64_t total, uint64_t first,
                                           uint32_t (&w)[kWordsPerThread]) {
    if (first + kWordsPerThread <= total) {
        const uint4 *p = reinterpret_cast<const uint4 *>(mask + first);
#pragma unroll
        for (int q = 0; q < kWordsPerThread / 4; ++q) {
            const uint4 v = __ldg(p + q);
            w[4 * q] = v.x;
            w[4 * q + 1] = v.y;
            w[4 * q + 2] = v.z;
            w[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kWordsPerThread; ++k)
            w[k] = (first + k < total) ? mask[first + k] : 0u;
    }
}

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *sh, uint32_t &total) {
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o)
            inc += u;
    }
    if (lane == 31)
        sh[wp] = inc;
    __syncthreads();
    if (wp == 0) {
        const uint32_t s = lane < kThreads / 32 ? sh[lane] : 0u;
        uint32_t si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o)
                si += u;
        }
        if (lane < kThreads / 32)
            sh[32 + lane] = si - s;
        if (lane == 31)
            sh[64] = si;
    }
    __syncthreads();
    total = sh[64];
    return sh[32 + wp] + inc - v;
}

__global__ void __launch_bounds__(kThreads) k_count(const uint32_t *mask, uint64_t total, uint32_t *counts,
                                                    uint32_t nchunks) {
    pdl_begin();
    __shared__ uint32_t sh[72];
    for (uint32_t b = blockIdx.x; b < nchunks; b += gridDim.x) {   // grid-stride over chunks
        const uint64_t first = (uint64_t)b * kChunk + (uint64_t)threadIdx.x * kWordsPerThread;
        uint32_t w[kWordsPerThread];
        load_words(mask, total, first, w);
        uint32_t c = 0;
#pragma unroll
        for (int k = 0; k < kWordsPerThread; ++k)
            c += __popc(w[k]);
        uint32_t tot;
        block_excl_scan(c, sh, tot);
        if (threadIdx.x == 0)
            counts[b] = tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_scan_counts(const uint32_t *counts, uint64_t *offsets, int nchunks,
                                                      uint64_t *count_out) {
    pdl_begin();
    __shared__ uint64_t sh[72];
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    uint64_t carry = 0;
    for (int base = 0; base < nchunks; base += 1024) {
        const int k = base + t;
        const uint64_t v = k < nchunks ? counts[k] : 0;
        uint64_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o)
                inc += u;
        }
        if (lane == 31)
            sh[wp] = inc;
        __syncthreads();
        if (wp == 0) {
            const uint64_t s = sh[lane];
            uint64_t si = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t u = __shfl_up_sync(0xffffffffu, si, o);
                if (lane >= o)
                    si += u;
            }
            sh[32 + lane] = si - s;
            if (lane == 31)
                sh[64] = si;
        }
        __syncthreads();
        if (k < nchunks)
            offsets[k] = carry + sh[32 + wp] + inc - v;
        carry += sh[64];
        __syncthreads();
    }
    if (t == 0)
        *count_out = carry;
}

__global__ void __launch_bounds__(kThreads) k_scatter(const uint32_t *mask, uint64_t total, int H, int Wwords,
                                                      const uint32_t *counts, const uint64_t *offsets,
                                                      uint64_t *list, uint64_t cap, uint32_t nchunks) {
    pdl_begin();
    __shared__ uint32_t sh[72];
    const uint64_t rowWords = (uint64_t)Wwords;
    const uint64_t planeWords = (uint64_t)H * rowWords;
    for (uint32_t b = blockIdx.x; b < nchunks; b += gridDim.x) {   // grid-stride over chunks
        if (counts[b] == 0 || offsets[b] >= cap)   // block-uniform: nothing to write here
            continue;
        const uint64_t first = (uint64_t)b * kChunk + (uint64_t)threadIdx.x * kWordsPerThread;
        uint32_t w[kWordsPerThread];
        load_words(mask, total, first, w);
        uint32_t c = 0;
#pragma unroll
        for (int k = 0; k < kWordsPerThread; ++k)
            c += __popc(w[k]);
        uint32_t tot;
        uint64_t pos = offsets[b] + block_excl_scan(c, sh, tot);
        __syncthreads();
        if (__all_sync(0xffffffffu, c == 0 || pos >= cap))   // warp-uniform: nothing to write
            continue;
        // (scale, row, word) of the thread's first word by division, then by
        // stepping through its consecutive words
        uint64_t sc = 0;
        uint32_t y = 0, xw = 0;
        if (c != 0) {
            sc = first / planeWords;
            const uint32_t rem = (uint32_t)(first - sc * planeWords);
            y = rem / (uint32_t)rowWords;
            xw = rem - y * (uint32_t)rowWords;
        }
        // Word slot k of every lane in turn.  Survivors cluster, so a slot often
        // holds one or a few dense words: then the warp writes each such word's
        // bits together, one bit per lane (the key's slot from a popcount of the
        // lower bits), instead of waiting on the lane that walks the most bits.
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int k = 0; k < kWordsPerThread; ++k) {
            const uint32_t wk = w[k];
            const uint32_t nz = __ballot_sync(0xffffffffu, wk != 0);
            const uint64_t keyb = (sc << 48) | ((uint64_t)y << 24) | ((uint64_t)xw * 32);
            if (nz) {   // warp-uniform
                const uint32_t mx = __reduce_max_sync(0xffffffffu, (uint32_t)__popc(wk));
                if (2 * mx > 3 * (uint32_t)__popc(nz)) {   // warp-uniform
                    for (uint32_t m = nz; m; m &= m - 1) {
                        const int src = __ffs(m) - 1;
                        const uint32_t word = __shfl_sync(0xffffffffu, wk, src);
                        const uint64_t kb = __shfl_sync(0xffffffffu, keyb, src);
                        const uint64_t base = __shfl_sync(0xffffffffu, pos, src);
                        if ((word >> lane) & 1u) {
                            const uint64_t at = base + __popc(word & ((1u << lane) - 1u));
                            if (at < cap)
                                list[at] = kb + lane;
                        }
                    }
                } else {
                    uint32_t bits = wk;
                    uint64_t at = pos;
                    while (bits) {
                        const int bit = __ffs(bits) - 1;
                        bits &= bits - 1;
                        if (at < cap)
                            list[at] = keyb + bit;
                        ++at;
                    }
                }
            }
            pos += __popc(wk);
            if (++xw == (uint32_t)rowWords) {
                xw = 0;
                if (++y == (uint32_t)H) {
                    y = 0;
                    ++sc;
                }
            }
        }
    }
}

// Copy a compacted list (device) and its count to host memory the device can
// address (pinned, mapped): min(count, cap) keys with coalesced stores, and the
// count.  The host then needs one synchronisation and no copy of its own.
__global__ void __launch_bounds__(kThreads) k_copy_keys(const uint64_t *src, const uint64_t *count, uint64_t cap,
                                                          uint64_t *dst, uint64_t *count_out) {
    pdl_begin();
    const uint64_t c = *count, n = c < cap ? c : cap;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        *count_out = c;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

}  // namespace

cudaError_t launch_copy_keys(const uint64_t *src, const uint64_t *count, uint64_t cap, uint64_t *dst,
                             uint64_t *count_out, cudaStream_t st, uint64_t *launches, int blocks) {
    if (launches)
        *launches += 1;
    return launch_pdl(k_copy_keys, dim3(blocks > 0 ? blocks : 1), dim3(kThreads), st, src, count, cap, dst,
                      count_out);
}

size_t compact_scratch_bytes(uint64_t total_words) {
    const uint64_t nchunks = (total_words + kChunk - 1) / kChunk;
    return ((nchunks * 4 + 255) & ~uint64_t(255)) + nchunks * 8 + 256;
}

cudaError_t launch_compact(const uint32_t *mask, uint64_t total_words, int H, int Wwords,
                           uint64_t *list, uint64_t cap, uint64_t *count, void *scratch,
                           cudaStream_t st, uint64_t *launches) {
    const uint64_t nchunks = (total_words + kChunk - 1) / kChunk;
    uint32_t *counts = (uint32_t *)scratch;
    uint64_t *offsets = (uint64_t *)((char *)scratch + ((nchunks * 4 + 255) & ~uint64_t(255)));
    cudaError_t e;
    if (launches)
        *launches += 3;
    // grid-stride kernels: a few blocks per SM, each walking many chunks
    const unsigned grid = (unsigned)std::min<uint64_t>(nchunks, 152 * 4);
    if ((e = launch_pdl(k_count, dim3(grid), dim3(kThreads), st, mask, total_words, counts, (uint32_t)nchunks)) !=
        cudaSuccess)
        return e;
    if ((e = launch_pdl(k_scan_counts, dim3(1), dim3(1024), st, (const uint32_t *)counts, offsets, (int)nchunks,
                        count)) != cudaSuccess)
        return e;
    return launch_pdl(k_scatter, dim3(grid), dim3(kThreads), st, mask, total_words, H, Wwords,
                      (const uint32_t *)counts, (const uint64_t *)offsets, list, cap, (uint32_t)nchunks);
}

}  // namespace scr

// ---------------------------------------------------------------------------
// Allocation-free compaction.
//
// Some callers cannot allocate device memory at the point where they compact
// a mask: real-time loops that must never enter an allocator (an allocation
// can block on the driver for an unbounded time), hosts whose device memory is
// all owned by another framework's allocator with no hook for a foreign
// library, and embedded runtimes that fix every buffer when they start.
// compact_mask_noalloc serves them: its scratch (per-chunk bit counts and
// their prefix offsets) lives in the fixed device array below instead of
// coming from an allocation.
//
// The array is a file-scope __device__ variable, so every GPU that loads this
// library holds it (kStaticCompactBytes) until the process exits.  In host
// code its name is only a host-side stand-in; the device address is looked up
// with cudaGetSymbolAddress, with the device current, once per device -- and
// once more if that device's context has been re-created since (after
// cudaDeviceReset the module is loaded again and the array may move), which
// the entry point notices by the context's unique id.
// ---------------------------------------------------------------------------
namespace scr {
namespace {

constexpr uint64_t kStaticChunks = 65536;   // chunks of 4096 mask words
constexpr size_t kStaticCompactBytes = 256 * 3 + kStaticChunks * 4 + kStaticChunks * 8;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_compact_scratch[kStaticCompactBytes];

std::mutex g_static_mu;
void *g_static_ptr[kMaxDevices] = {nullptr};
unsigned long long g_static_ctx[kMaxDevices] = {0};   // unique id of the context the address belongs to
thread_local char g_noalloc_err[256];

// Unique id of the calling thread's current context (cuCtxGetCurrent +
// cuCtxGetId, reached through the runtime so the library needs no link to the
// driver library).  0 when it cannot be read.
unsigned long long current_context_id() {
    using GetCurrent = int (*)(void **);
    using GetId = int (*)(void *, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {   // called with g_static_mu held
        looked_up = true;
        void *f = nullptr, *g = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<GetCurrent>(f);
            get_id = reinterpret_cast<GetId>(g);
        }
        cudaGetLastError();
    }
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0)
        return 0;
    return id;
}

int noalloc_fail(int code, const char *msg) {
    snprintf(g_noalloc_err, sizeof g_noalloc_err, "%s", msg);
    return code;
}

}  // namespace
}  // namespace scr

extern "C" const char *compact_mask_noalloc_error(void) { return scr::g_noalloc_err; }

extern "C" int compact_mask_noalloc(const uint32_t *mask_dev, int32_t n_scales, int32_t H, int32_t W,
                                    uint64_t *list_dev, uint64_t list_cap, uint64_t *count_dev,
                                    scr_stream stream) {
    using namespace scr;
    if (!mask_dev || !count_dev || (list_cap && !list_dev))
        return noalloc_fail(SCR_EINVAL, "null mask, count or list");
    if (((uintptr_t)mask_dev & 15) || ((uintptr_t)count_dev & 7) || ((uintptr_t)list_dev & 7))
        return noalloc_fail(SCR_EINVAL, "mask must be 16-byte aligned, list and count 8-byte aligned");
    if (n_scales < 1 || n_scales > 65535 || H < 1 || W < 1 || H > 65535 || W > 65535)
        return noalloc_fail(SCR_EINVAL, "bad mask geometry");
    const int Ww = (W + 31) / 32;
    const uint64_t total = (uint64_t)n_scales * H * Ww;
    const uint64_t nchunks = (total + 4095) / 4096;
    if (nchunks > kStaticChunks)
        return noalloc_fail(SCR_EINVAL, "mask larger than the fixed scratch allows "
                                        "(at most 65536 * 4096 = 268435456 words)");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(SCR_ECUDA, "no usable current CUDA device");
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        const unsigned long long ctx = current_context_id();   // 0: no context yet, or unreadable
        if (!g_static_ptr[dev] || ctx == 0 || ctx != g_static_ctx[dev]) {
            // set-up for this device (the current device), once per context;
            // cudaGetSymbolAddress also creates the context if there is none yet
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_compact_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return noalloc_fail(SCR_ECUDA, "cudaGetSymbolAddress of the fixed compaction scratch failed");
            }
            g_static_ptr[dev] = p;
            g_static_ctx[dev] = current_context_id();
        }
        scratch = g_static_ptr[dev];
    }
    // counts and offsets are fully rewritten by every call: nothing to clear
    const cudaError_t e = launch_compact(mask_dev, total, H, Ww, list_dev, list_cap, count_dev, scratch,
                                         (cudaStream_t)stream, nullptr);
    if (e != cudaSuccess)
        return noalloc_fail(SCR_ECUDA, cudaGetErrorString(e));
    return SCR_OK;
}
