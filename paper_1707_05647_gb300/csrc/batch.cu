// Batched screening: many images of uneven size against many templates and
// scales in one persistent launch.
//
// Every (template, scale) that a pair (image, template) asks for becomes a
// "record" (its pair, its scale index and its integer bounds).  Records are
// grouped per image by star radius R: the features at each (position, R) --
// star sum S, variance numerator V, contrast numerator N (Sec. 3, 4, 5) -- are
// computed once and tested against every record of the group.  A group is cut
// into units of one row x 64 mask words; a persistent grid walks the units.
//
// Survivors are written as keys (pair << 37 | s << 32 | y << 16 | x) into
// slots each warp reserves 256 at a time (one global atomic per chunk; unused
// slots of a chunk get a sentinel that sorts last), counted per pair, and
// OR-ed into a per-image union mask; a stable LSD radix sort then puts the
// keys in ascending order, so the per-pair lists come out in the canonical
// (scale, row, column) order of the single-image path.  No kernel waits on
// another CTA.
#include <cuda_runtime.h>
#include <stdint.h>

#include "batch.h"
#include "internal.h"

namespace scr {
namespace {

__device__ __forceinline__ uint32_t ldb(const uint32_t *p) { return __ldg(p); }

template <int WPW>
__device__ __forceinline__ void corner_sums(const uint32_t *L, const uint32_t *T, const int32_t (&oL)[4],
                                            const int32_t (&oT)[4], uint32_t live, uint32_t (&out)[WPW]) {
    const uint32_t *p0 = L + oL[0], *p1 = L + oL[1], *p2 = L + oL[2], *p3 = L + oL[3];
    const uint32_t *q0 = T + oT[0], *q1 = T + oT[1], *q2 = T + oT[2], *q3 = T + oT[3];
#pragma unroll
    for (int j = 0; j < WPW; ++j) {
        out[j] = 0;
        if ((live >> j) & 1u) {
            const int d = 32 * j;
            out[j] = ldb(p0 + d) - ldb(p1 + d) - ldb(p2 + d) + ldb(p3 + d) + ldb(q0 + d) - ldb(q1 + d) -
                     ldb(q2 + d) + ldb(q3 + d);
        }
    }
}

// Two window sums (square, diamond) of one table pair, each exact mod 2^32,
// added in 64 bits (for the sums of squares).
template <int WPW>
__device__ __forceinline__ void corner_sums64(const uint32_t *L, const uint32_t *T, const int32_t (&oL)[4],
                                              const int32_t (&oT)[4], uint32_t live, uint64_t (&out)[WPW]) {
#pragma unroll
    for (int j = 0; j < WPW; ++j) {
        out[j] = 0;
        if ((live >> j) & 1u) {
            const int d = 32 * j;
            const uint32_t a = ldb(L + oL[0] + d) - ldb(L + oL[1] + d) - ldb(L + oL[2] + d) + ldb(L + oL[3] + d);
            const uint32_t b = ldb(T + oT[0] + d) - ldb(T + oT[1] + d) - ldb(T + oT[2] + d) + ldb(T + oT[3] + d);
            out[j] = (uint64_t)a + b;
        }
    }
}

// The eight corner pointers of the star sum (square on L, diamond on T) of one
// warp-chunk; word j reads at the immediate offset 32 * j.
struct StarCorners {
    const uint32_t *p[8];
    __device__ __forceinline__ StarCorners(const uint32_t *L, const uint32_t *T, const int32_t (&oL)[4],
                                           const int32_t (&oT)[4]) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            p[k] = L + oL[k];
            p[4 + k] = T + oT[k];
        }
    }
    __device__ __forceinline__ uint32_t sum(int j) const {
        const int d = 32 * j;
        return ldb(p[0] + d) - ldb(p[1] + d) - ldb(p[2] + d) + ldb(p[3] + d) + ldb(p[4] + d) - ldb(p[5] + d) -
               ldb(p[6] + d) + ldb(p[7] + d);
    }
};

constexpr int kBatchWarps = kBatchWarpsPerBlock;

// Register budget per variant: 3 resident blocks (80 registers) with 8 words
// per warp, 4 (64 registers) with fewer, neither spilling; more warps per SM
// hide the L2 latency of the corner loads.
template <int WPW>
__global__ void __launch_bounds__(32 * kBatchWarps, (WPW >= 8 ? 3 : 4)) k_batch(const BatchArgs a) {
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint64_t cpos = 0, cend = 0;   // this warp's reserved key slots [cpos, cend) (warp-uniform)
    auto fill_rest = [&]() {       // sentinel into the unused slots of the current chunk
        for (uint64_t k = cpos + lane; k < cend; k += 32)
            if (k < a.keys_cap)
                a.keys[k] = kKeySentinel;
    };
    // Each warp takes whole units from a global counter, in increasing order,
    // so the units in flight stay within a few rows of each other and the
    // table rows they read are still in L2 when the next radius needs them.
    // The next index is fetched one unit ahead to hide the atomic's latency.
    int img = -1;   // image of the current unit (warp-uniform)
    uint64_t next = 0;
    if (lane == 0)
        next = atomicAdd((unsigned long long *)a.next_unit, 1ull);
    next = __shfl_sync(0xffffffffu, next, 0);
    while (next < (uint64_t)a.n_units) {
        const int64_t u = (int64_t)next * a.unit_stride;
        if (lane == 0)
            next = atomicAdd((unsigned long long *)a.next_unit, 1ull);
        next = __shfl_sync(0xffffffffu, next, 0);
        if (img < 0) {
            // first unit of this warp: last image with unit0 <= u (binary search)
            int l = 0, h = a.n_images - 1;
            while (l < h) {
                const int mid = (l + h + 1) >> 1;
                if (__ldg(&a.images[mid].unit0) <= u)
                    l = mid;
                else
                    h = mid - 1;
            }
            img = l;
        } else {
            while (img + 1 < a.n_images && __ldg(&a.images[img + 1].unit0) <= u)
                ++img;
        }
        const BImage *ip = a.images + img;
        const int n_grp = __ldg(&ip->n_grp);
        const uint32_t local = (uint32_t)(u - __ldg(&ip->unit0));   // < rows * n_grp
        const int y = __ldg(&ip->y_first) + (int)(local / (uint32_t)n_grp);
        const BGroup *gp = a.groups + __ldg(&ip->g0) + (int)(local % (uint32_t)n_grp);
        if (y < __ldg(&gp->y_lo) || y > __ldg(&gp->y_hi))
            continue;
        // the unit's constants, in registers for the walk along the row
        const int x_lo = __ldg(&gp->x_lo), x_hi = __ldg(&gp->x_hi);
        const int w_lo = __ldg(&gp->w_lo), w_hi = __ldg(&gp->w_hi);
        const uint32_t h_lo = __ldg(&gp->S_lo_hull), h_rng = __ldg(&gp->S_rng_hull);
        const int rec0 = __ldg(&gp->rec0), rec1 = __ldg(&gp->rec1);
        const int64_t pitch = __ldg(&ip->pitch);
        const uint32_t *L1 = (const uint32_t *)__ldg((const unsigned long long *)&ip->L1);
        const uint32_t *T1 = (const uint32_t *)__ldg((const unsigned long long *)&ip->T1);
        const int64_t row = (int64_t)y * pitch + kColOffset + lane;   // this lane's element at x = lane
        int32_t oL[4], oT[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            oL[k] = __ldg(&gp->oL[k]);
            oT[k] = __ldg(&gp->oT[k]);
        }
        // the warp walks the row's mask words WPW at a time
        for (int w0 = w_lo; w0 <= w_hi; w0 += WPW) {
            const int xs = w0 * 32;   // the warp covers x in [xs, xs + 32 * WPW)
            const int x0 = xs + lane;
            const int64_t e = row + xs;
            const StarCorners c(L1 + e, T1 + e, oL, oT);
            uint32_t S[WPW], live = 0;
            if (xs >= x_lo && xs + 32 * WPW - 1 <= x_hi) {   // warp-uniform: every position valid
                // all corner reads written before any sum: issued back to back
                uint32_t v[WPW][8];
#pragma unroll
                for (int j = 0; j < WPW; ++j)
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        v[j][k] = ldb(c.p[k] + 32 * j);
#pragma unroll
                for (int j = 0; j < WPW; ++j)
                    S[j] = v[j][0] - v[j][1] - v[j][2] + v[j][3] + v[j][4] - v[j][5] - v[j][6] + v[j][7];
                live = (1u << WPW) - 1;
            } else {
                const uint32_t span = (uint32_t)(x_hi - x_lo);
#pragma unroll
                for (int j = 0; j < WPW; ++j) {
                    S[j] = 0;
                    if ((uint32_t)(x0 + 32 * j - x_lo) <= span) {
                        S[j] = c.sum(j);
                        live |= 1u << j;
                    }
                }
            }
            // fast reject against the hull of every record's mean interval
            uint32_t alive = 0;
#pragma unroll
            for (int j = 0; j < WPW; ++j)
                alive |= ((S[j] - h_lo) <= h_rng ? 1u : 0u) << j;
            alive &= live;
            if (!__any_sync(0xffffffffu, alive))
                continue;
            // V and N are shared by every record of the group and computed on first
            // use (warp-uniform), only if some lane still needs them
            uint64_t V[WPW], N[WPW];
            bool haveV = false, haveN = false;
            uint32_t ubits[WPW];
#pragma unroll
            for (int j = 0; j < WPW; ++j)
                V[j] = N[j] = 0, ubits[j] = 0;
            // when every record tests the variance, a position whose V lies outside
            // the union of their variance intervals fails them all: reject it
            // before the walk over the records (on a background flatter than the
            // templates this ends most positions here)
            if (__ldg(&gp->all_var)) {
                const uint32_t *L2 = (const uint32_t *)__ldg((const unsigned long long *)&ip->L2);
                const uint32_t *T2 = (const uint32_t *)__ldg((const unsigned long long *)&ip->T2);
                uint64_t Q[WPW];
                corner_sums64<WPW>(L2 + e, T2 + e, oL, oT, alive, Q);
                const uint64_t A = __ldg(&gp->A);
                const uint64_t vlo = (uint64_t)__ldg((const long long *)&gp->V_lo_hull);
                const uint64_t vrng = __ldg((const unsigned long long *)&gp->V_rng_hull);
#pragma unroll
                for (int j = 0; j < WPW; ++j) {
                    V[j] = A * Q[j] - (uint64_t)S[j] * S[j];
                    if ((V[j] - vlo) > vrng)
                        alive &= ~(1u << j);
                }
                haveV = true;
                if (!__any_sync(0xffffffffu, alive))
                    continue;
            }
            // the warp's range of means among alive positions: records are sorted
            // by interval start (records without a mean test start at 0 and span
            // everything), so the walk skips disjoint intervals and stops early
            uint32_t smin = 0, smax = UINT32_MAX;
            if (rec1 - rec0 > 1) {
                smin = UINT32_MAX;
                smax = 0;
#pragma unroll
                for (int j = 0; j < WPW; ++j)
                    if ((alive >> j) & 1u) {
                        smin = min(smin, S[j]);
                        smax = max(smax, S[j]);
                    }
                smin = __reduce_min_sync(0xffffffffu, smin);
                smax = __reduce_max_sync(0xffffffffu, smax);
            }
            for (int r = rec0; r < rec1; ++r) {
                const BRecord *rc = a.records + r;
                const uint32_t slo = __ldg(&rc->S_lo), srng = __ldg(&rc->S_rng);
                if (slo > smax)
                    break;
                if (slo + srng < smin)
                    continue;
                const uint32_t feats = __ldg(&rc->features);
                uint32_t keep = alive;
                if (feats & SCR_F_MEAN) {
#pragma unroll
                    for (int j = 0; j < WPW; ++j)
                        if ((S[j] - slo) > srng)
                            keep &= ~(1u << j);
                }
                if (feats & SCR_F_VAR) {
                    if (!haveV && __any_sync(0xffffffffu, keep)) {
                        const uint32_t *L2 = (const uint32_t *)__ldg((const unsigned long long *)&ip->L2);
                        const uint32_t *T2 = (const uint32_t *)__ldg((const unsigned long long *)&ip->T2);
                        uint64_t Q[WPW];
                        corner_sums64<WPW>(L2 + e, T2 + e, oL, oT, alive, Q);
                        const uint64_t A = __ldg(&gp->A);
#pragma unroll
                        for (int j = 0; j < WPW; ++j)
                            V[j] = A * Q[j] - (uint64_t)S[j] * S[j];
                        haveV = true;
                    }
                    const uint64_t vlo = (uint64_t)__ldg(&rc->V_lo), vrng = __ldg(&rc->V_rng);
#pragma unroll
                    for (int j = 0; j < WPW; ++j)
                        if ((V[j] - vlo) > vrng)
                            keep &= ~(1u << j);
                }
                if (feats & SCR_F_GRAD) {
                    if (!haveN && __any_sync(0xffffffffu, keep)) {
                        int32_t oLi[4], oTi[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            oLi[k] = __ldg(&gp->oLi[k]);
                            oTi[k] = __ldg(&gp->oTi[k]);
                        }
                        uint32_t Si[WPW];
                        corner_sums<WPW>(L1 + e, T1 + e, oLi, oTi, alive, Si);
                        const uint64_t Ain = __ldg(&gp->Ain), Aring = __ldg(&gp->Aring);
#pragma unroll
                        for (int j = 0; j < WPW; ++j)
                            N[j] = (uint64_t)((int64_t)((uint64_t)Si[j] * Aring) -
                                              (int64_t)((uint64_t)(S[j] - Si[j]) * Ain));
                        haveN = true;
                    }
                    const uint64_t nlo = (uint64_t)__ldg(&rc->N_lo), nrng = __ldg(&rc->N_rng);
#pragma unroll
                    for (int j = 0; j < WPW; ++j)
                        if ((N[j] - nlo) > nrng)
                            keep &= ~(1u << j);
                }
                if (!__any_sync(0xffffffffu, keep))
                    continue;
                const uint64_t key_hi = ((uint64_t)__ldg(&rc->pair) << 37) | ((uint64_t)__ldg(&rc->s) << 32) |
                                        ((uint64_t)y << 16);
                uint32_t nrec = 0;   // survivors of this record in the warp's words
#pragma unroll
                for (int j = 0; j < WPW; ++j) {
                    const bool kj = (keep >> j) & 1u;
                    const uint32_t bits = __ballot_sync(0xffffffffu, kj);
                    if (!bits)
                        continue;
                    ubits[j] |= bits;
                    const uint32_t cnt = __popc(bits);
                    nrec += cnt;
                    if (cpos + cnt > cend) {   // new chunk of key slots
                        fill_rest();
                        uint64_t base = 0;
                        if (lane == 0)
                            base = atomicAdd((unsigned long long *)a.n_reserved, (unsigned long long)kKeyChunk);
                        cpos = __shfl_sync(0xffffffffu, base, 0);
                        cend = cpos + kKeyChunk;
                    }
                    if (kj) {
                        const uint64_t pos = cpos + __popc(bits & lt_mask);
                        if (pos < a.keys_cap)
                            a.keys[pos] = key_hi | (uint64_t)(x0 + 32 * j);
                    }
                    cpos += cnt;
                }
                if (lane == 0 && nrec)
                    atomicAdd((unsigned long long *)&a.counts[__ldg(&rc->pair)], (unsigned long long)nrec);
            }
            if (a.union_mask && lane < WPW) {   // one OR per word of the unit: lane j writes word j
                uint32_t mine = 0;
#pragma unroll
                for (int j = 0; j < WPW; ++j)
                    mine = lane == j ? ubits[j] : mine;
                if (mine)
                    atomicOr(a.union_mask + __ldg(&ip->mask_offset) + (int64_t)y * __ldg(&ip->Wwords) + w0 + lane,
                             mine);
            }
        }
    }
    fill_rest();
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of the keys, 8 bits per pass.  The key count lives in
// device memory, so every kernel walks tiles with a grid stride and the grid
// size is fixed (the sequence can be captured in a CUDA graph).
// ---------------------------------------------------------------------------
constexpr int RS_T = 256;                   // threads
constexpr int RS_R = 8;                     // rounds (keys per thread) per tile
constexpr int RS_TILE = RS_T * RS_R;        // 2048 keys per tile
constexpr int RS_E = 32;                    // scan entries per thread
constexpr int RS_CH = RS_T * RS_E;          // 8192 histogram entries per scan chunk

__device__ __forceinline__ uint64_t sort_count(const SortArgs &a) {
    const uint64_t n = *a.n_keys;
    return n < a.cap ? n : a.cap;
}

// The key (pair << 37 | s << 32 | y << 16 | x) with each field cut to its used
// width; the sentinel ~0 becomes all ones and stays last because every real
// pair index is below 2^pb - 1.
__device__ __forceinline__ uint32_t sort_digit(uint64_t k, const SortArgs &a, int shift) {
    const uint64_t x = k & 0xFFFFu, y = (k >> 16) & 0xFFFFu, s = (k >> 32) & 31u, p = k >> 37;
    const uint64_t c = (x & ((1ull << a.xb) - 1)) | ((y & ((1ull << a.yb) - 1)) << a.xb) |
                       ((s & ((1ull << a.sb) - 1)) << (a.xb + a.yb)) |
                       ((p & ((1ull << a.pb) - 1)) << (a.xb + a.yb + a.sb));
    return (uint32_t)(c >> shift) & 255u;
}

// hist[d * ntiles + t] = keys of tile t with digit d (one shared-memory atomic
// per key).  Measured per pass over 1.27e9 keys: 3.3 ms; aggregating equal
// digits of a warp with __match_any_sync first, 4.8 ms; one atomic of 32 when
// __match_all_sync finds the warp's digits equal, 3.6 ms.
__global__ void __launch_bounds__(RS_T) k_rs_hist(const SortArgs a, int shift) {
    pdl_begin();
    __shared__ uint32_t h[256];
    const uint64_t n = sort_count(a);
    const uint64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        h[threadIdx.x] = 0;
        __syncthreads();
        for (int k = 0; k < RS_R; ++k) {
            const uint64_t i = t * RS_TILE + (uint64_t)k * RS_T + threadIdx.x;
            if (i < n)
                atomicAdd(&h[sort_digit(a.src[i], a, shift)], 1u);
        }
        __syncthreads();
        a.hist[(uint64_t)threadIdx.x * ntiles + t] = h[threadIdx.x];
        __syncthreads();
    }
}

// Exclusive scan of 256 values of one block (one per thread); returns the total.
__device__ __forceinline__ uint32_t block_exscan256(uint32_t v, uint32_t *sh, uint32_t &total) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o)
            inc += x;
    }
    if (lane == 31)
        sh[w] = inc;
    __syncthreads();
    uint32_t before = 0;
    total = 0;
#pragma unroll
    for (int q = 0; q < RS_T / 32; ++q) {
        const uint32_t c = sh[q];
        before += q < w ? c : 0u;
        total += c;
    }
    __syncthreads();
    return before + inc - v;
}

// csum[c] = sum of histogram chunk c (RS_CH entries in digit-major order)
__global__ void __launch_bounds__(RS_T) k_rs_reduce(const SortArgs a) {
    pdl_begin();
    __shared__ uint32_t sh[RS_T / 32];
    const uint64_t n = sort_count(a);
    const uint64_t m = 256 * ((n + RS_TILE - 1) / RS_TILE);
    const uint64_t nc = (m + RS_CH - 1) / RS_CH;
    for (uint64_t c = blockIdx.x; c < nc; c += gridDim.x) {
        const uint64_t i0 = c * RS_CH + (uint64_t)threadIdx.x * RS_E;   // m is a multiple of RS_E
        uint32_t v = 0;
        if (i0 < m) {
            const uint4 *p = reinterpret_cast<const uint4 *>(a.hist + i0);
#pragma unroll
            for (int q = 0; q < RS_E / 4; ++q) {
                const uint4 x = p[q];
                v += x.x + x.y + x.z + x.w;
            }
        }
        uint32_t total;
        block_exscan256(v, sh, total);
        if (threadIdx.x == 0)
            a.csum[c] = total;
    }
}

// Exclusive scan of the chunk sums, in place (one block).
__global__ void __launch_bounds__(1024) k_rs_scan(const SortArgs a) {
    pdl_begin();
    __shared__ uint64_t sh[72];
    const uint64_t n = sort_count(a);
    const uint64_t m = 256 * ((n + RS_TILE - 1) / RS_TILE);
    const uint64_t nc = (m + RS_CH - 1) / RS_CH;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint64_t carry = 0;
    for (uint64_t b0 = 0; b0 < nc; b0 += 1024) {
        const uint64_t i = b0 + t;
        const uint64_t v = i < nc ? a.csum[i] : 0;
        uint64_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t x = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o)
                inc += x;
        }
        if (lane == 31)
            sh[w] = inc;
        __syncthreads();
        if (w == 0) {
            const uint64_t s = sh[lane];
            uint64_t si = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t x = __shfl_up_sync(0xffffffffu, si, o);
                if (lane >= o)
                    si += x;
            }
            sh[32 + lane] = si - s;
            if (lane == 31)
                sh[64] = si;
        }
        __syncthreads();
        if (i < nc)
            a.csum[i] = carry + sh[32 + w] + inc - v;
        carry += sh[64];
        __syncthreads();
    }
}

// hist entries become offsets within their chunk (below RS_CH * RS_TILE)
__global__ void __launch_bounds__(RS_T) k_rs_down(const SortArgs a) {
    pdl_begin();
    __shared__ uint32_t sh[RS_T / 32];
    const uint64_t n = sort_count(a);
    const uint64_t m = 256 * ((n + RS_TILE - 1) / RS_TILE);
    const uint64_t nc = (m + RS_CH - 1) / RS_CH;
    for (uint64_t c = blockIdx.x; c < nc; c += gridDim.x) {
        const uint64_t i0 = c * RS_CH + (uint64_t)threadIdx.x * RS_E;
        uint4 *p = reinterpret_cast<uint4 *>(a.hist + i0);
        uint4 x[RS_E / 4];
        uint32_t v = 0;
        if (i0 < m) {
#pragma unroll
            for (int q = 0; q < RS_E / 4; ++q) {
                x[q] = p[q];
                v += x[q].x + x[q].y + x[q].z + x[q].w;
            }
        }
        uint32_t total;
        uint32_t run = block_exscan256(v, sh, total);
        if (i0 < m) {
#pragma unroll
            for (int q = 0; q < RS_E / 4; ++q) {
                uint4 o;
                o.x = run; run += x[q].x;
                o.y = run; run += x[q].y;
                o.z = run; run += x[q].z;
                o.w = run; run += x[q].w;
                p[q] = o;
            }
        }
    }
}

// Stable scatter of one tile: warp w owns keys [w * 256, w * 256 + 256) of the
// tile (in order), counts them per digit, the warps' counts are scanned per
// digit, and each warp puts its keys at the digit's running position in a copy
// of the tile sorted by digit in shared memory.  The block then writes that
// copy out, consecutive threads to consecutive addresses within each digit's
// run, instead of one scattered 8-byte store per key (measured on the
// 64-image x 256-template batch: 5.7 ms per pass over 1.27e9 keys against
// 12.4 ms).
__global__ void __launch_bounds__(RS_T) k_rs_scatter(const SortArgs a, int shift) {
    pdl_begin();
    constexpr int NW = RS_T / 32;
    __shared__ uint32_t wofs[NW][256];
    __shared__ uint64_t start[256];
    __shared__ uint32_t lofs[256];          // first slot of each digit in the sorted tile
    __shared__ uint32_t ssh[RS_T / 32];
    __shared__ uint64_t skey[RS_TILE];      // the tile, sorted by digit (stable)
    __shared__ uint8_t sdig[RS_TILE];
    const uint64_t n = sort_count(a);
    const uint64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t h = (uint64_t)t * ntiles + tile;
        start[t] = a.csum[h / RS_CH] + a.hist[h];   // where digit t of this tile starts
#pragma unroll
        for (int q = 0; q < NW; ++q)
            wofs[q][t] = 0;
        __syncthreads();
        uint64_t key[RS_R];
        uint32_t dg[RS_R], peers[RS_R];
        const uint64_t base = tile * RS_TILE + (uint64_t)w * (RS_R * 32) + lane;
#pragma unroll
        for (int r = 0; r < RS_R; ++r) {
            const uint64_t i = base + 32 * r;
            const bool has = i < n;
            key[r] = has ? a.src[i] : 0;
            dg[r] = has ? sort_digit(key[r], a, shift) : 256u + lane;   // distinct dummy digits
        }
#pragma unroll
        for (int r = 0; r < RS_R; ++r) {
            peers[r] = __match_any_sync(0xffffffffu, dg[r]);
            if (dg[r] < 256u && (peers[r] & lt_mask) == 0)   // lowest lane of its digit group
                wofs[w][dg[r]] += __popc(peers[r]);
            __syncwarp();
        }
        __syncthreads();
        uint32_t acc = 0;   // digit t: warps before each warp
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            const uint32_t c = wofs[q][t];
            wofs[q][t] = acc;
            acc += c;
        }
        uint32_t ntile;
        lofs[t] = block_exscan256(acc, ssh, ntile);   // acc: the tile's keys with digit t
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RS_R; ++r) {
            const uint32_t d = dg[r];
            uint32_t before = 0;
            if (d < 256u) {
                before = wofs[w][d];
                const uint32_t at = lofs[d] + before + __popc(peers[r] & lt_mask);
                skey[at] = key[r];
                sdig[at] = (uint8_t)d;
            }
            __syncwarp();
            if (d < 256u && (peers[r] & lt_mask) == 0)
                wofs[w][d] = before + __popc(peers[r]);
            __syncwarp();
        }
        __syncthreads();
        for (uint32_t i = t; i < ntile; i += RS_T) {
            const uint32_t d = sdig[i];
            a.dst[start[d] + (i - lofs[d])] = skey[i];
        }
        __syncthreads();
    }
}

// offsets[p] = sum of counts[q] for q < p (one block, grid-independent).
__global__ void __launch_bounds__(1024) k_pair_offsets(const uint64_t *counts, uint64_t *offsets, uint64_t *total,
                                                       const uint64_t *reserved, int n) {
    pdl_begin();
    __shared__ uint64_t sh[72];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint64_t carry = 0;
    for (int b0 = 0; b0 < n; b0 += 1024) {
        const int i = b0 + t;
        const uint64_t v = i < n ? counts[i] : 0;
        uint64_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t x = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o)
                inc += x;
        }
        if (lane == 31)
            sh[w] = inc;
        __syncthreads();
        if (w == 0) {
            const uint64_t s = sh[lane];
            uint64_t si = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t x = __shfl_up_sync(0xffffffffu, si, o);
                if (lane >= o)
                    si += x;
            }
            sh[32 + lane] = si - s;
            if (lane == 31)
                sh[64] = si;
        }
        __syncthreads();
        if (i < n && offsets)
            offsets[i] = carry + sh[32 + w] + inc - v;
        carry += sh[64];
        __syncthreads();
    }
    if (t == 0) {
        total[0] = carry;                     // survivors
        total[1] = reserved ? *reserved : 0;  // key slots used (>= survivors)
    }
}

// Batched keys (pair << 37 | s << 32 | y << 16 | x) to the single-image key
// format of compact_mask, in place; the pair's keys are contiguous after the sort.
__global__ void __launch_bounds__(256) k_keys_to_lists(uint64_t *keys, const uint64_t *n, uint64_t cap) {
    pdl_begin();
    const uint64_t m = *n < cap ? *n : cap;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        keys[i] = (((k >> 32) & 31u) << 48) | (((k >> 16) & 0xFFFFu) << 24) | (k & 0xFFFFu);
    }
}

// One block per pair (grid-stride): the pair's first keys, converted, into its
// staging slot.
__global__ void __launch_bounds__(256) k_gather_lists(const uint64_t *keys, const uint64_t *counts,
                                                      const uint64_t *offsets, const uint64_t *total,
                                                      const uint64_t *stage, uint64_t *out, uint64_t *out_counts,
                                                      int n) {
    pdl_begin();
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const uint64_t c = counts[k], cap = stage[2 * k], dst = stage[2 * k + 1], src = offsets[k];
        const uint64_t m = c < cap ? c : cap;
        for (uint64_t i = threadIdx.x; i < m; i += blockDim.x) {
            const uint64_t key = keys[src + i];
            out[dst + i] = (((key >> 32) & 31u) << 48) | (((key >> 16) & 0xFFFFu) << 24) | (key & 0xFFFFu);
        }
        if (threadIdx.x == 0)
            out_counts[k] = c;
    }
    if (blockIdx.x == 0 && threadIdx.x < 2)
        out_counts[n + threadIdx.x] = total[threadIdx.x];
}

}  // namespace

cudaError_t launch_gather_lists(const uint64_t *keys, const uint64_t *counts, const uint64_t *offsets,
                                const uint64_t *total, const uint64_t *stage, uint64_t *out, uint64_t *out_counts,
                                int n, int grid, cudaStream_t st, uint64_t *launches) {
    if (launches)
        *launches += 1;
    return launch_pdl(k_gather_lists, dim3(grid), dim3(256), st, keys, counts, offsets, total, stage, out, out_counts,
                      n);
}

cudaError_t launch_keys_to_lists(uint64_t *keys, const uint64_t *n, uint64_t cap, int grid, cudaStream_t st,
                                 uint64_t *launches) {
    if (launches)
        *launches += 1;
    return launch_pdl(k_keys_to_lists, dim3(grid), dim3(256), st, keys, n, cap);
}

cudaError_t launch_batch(const BatchArgs &a, int words_per_warp, int grid, cudaStream_t st, uint64_t *launches) {
    const dim3 block(32 * kBatchWarps);
    cudaError_t e;
    switch (words_per_warp) {
        case 2: e = launch_pdl(k_batch<2>, dim3(grid), block, st, a); break;
        case 4: e = launch_pdl(k_batch<4>, dim3(grid), block, st, a); break;
        default: e = launch_pdl(k_batch<8>, dim3(grid), block, st, a); break;
    }
    if (launches)
        *launches += 1;
    return e;
}

size_t sort_hist_bytes(uint64_t cap) {
    const uint64_t tiles = (cap + RS_TILE - 1) / RS_TILE;
    return (size_t)tiles * 256 * 4;
}

size_t sort_csum_bytes(uint64_t cap) {
    const uint64_t m = 256 * ((cap + RS_TILE - 1) / RS_TILE);
    return (size_t)((m + RS_CH - 1) / RS_CH + 1) * 8;
}

uint64_t sort_max_tiles(uint64_t cap) { return (cap + RS_TILE - 1) / RS_TILE; }

cudaError_t launch_sort(const SortArgs &base, int passes, int grid, cudaStream_t st, uint64_t *launches) {
    SortArgs a = base;
    uint64_t *bufs[2] = {base.src, base.dst};
    cudaError_t e = cudaSuccess;
    for (int p = 0; p < passes; ++p) {
        a.src = bufs[p & 1];
        a.dst = bufs[(p + 1) & 1];
        if ((e = launch_pdl(k_rs_hist, dim3(grid), dim3(RS_T), st, a, 8 * p)) != cudaSuccess ||
            (e = launch_pdl(k_rs_reduce, dim3(grid), dim3(RS_T), st, a)) != cudaSuccess ||
            (e = launch_pdl(k_rs_scan, dim3(1), dim3(1024), st, a)) != cudaSuccess ||
            (e = launch_pdl(k_rs_down, dim3(grid), dim3(RS_T), st, a)) != cudaSuccess ||
            (e = launch_pdl(k_rs_scatter, dim3(grid), dim3(RS_T), st, a, 8 * p)) != cudaSuccess)
            return e;
        if (launches)
            *launches += kSortLaunchesPerPass;
    }
    return e;
}

cudaError_t launch_pair_offsets(const uint64_t *counts, uint64_t *offsets, uint64_t *total, const uint64_t *reserved,
                                int n, cudaStream_t st, uint64_t *launches) {
    if (launches)
        *launches += 1;
    return launch_pdl(k_pair_offsets, dim3(1), dim3(1024), st, counts, offsets, total, reserved, n);
}

}  // namespace scr
