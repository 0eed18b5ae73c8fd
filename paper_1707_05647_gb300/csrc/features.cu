// Octagonal-star features at every candidate position and scale, and the
// threshold test that turns them into the candidate bitmask.
//
//   square sum   (Sec. 3, Eq. S_1): L(y+n+1, x+n+1) - L(y-n+1, x+n+1)
//                                   - L(y+n+1, x-n+1) + L(y-n+1, x-n+1)
//   diamond sum  (Sec. 4, four cone corners, half-diagonal h):
//                T(y+h+1, x+1) - T(y+1, x-h+1) - T(y+1, x+h+1) + T(y-h+1, x+1)
//   star         (Sec. 4, Eq. S_os): square and diamond pooled, A = 4n^2 + 2h^2
//   variance     (Sec. 3, Eq. S_sigma) scaled by A^2: V = A*Q - S^2
//   contrast     (Sec. 5, central areas): inner star of radius floor(R/2)
//                against the ring, N = S_in*A_ring - (S - S_in)*A_in
//   test         (Sec. 5, Algorithm 1): every enabled feature inside its
//                inclusive integer bounds.
//
// Each window sum is below 2^32 (the host checks this per scale), so the
// kernel reads only the low 32-bit plane of every table and subtracts modulo
// 2^32: the result is the exact sum.  Products are formed in 64 bits.
//
// Packed-plane pre-filter (optional, on tables built with filter windows): a
// scale that has a window first sums its star's eight corners of one packed
// plane, which carries 16 bits of the sum table and 16 bits of the squares'
// table per element, so one 32-bit read per corner yields both the pooled sum
// S and the pooled square sum Q to within a few units of 2^kS and 2^kQ.
// From those bounds the kernel rejects every candidate whose variance is
// certainly below the variance interval, and reads the exact corners only for
// the words where some candidate is left; the exact tests then decide as
// without the filter, so the mask is the same bit for bit.
//
// Mapping: one warp evaluates WPW consecutive mask words (32 x each) of one
// row for every scale, so each corner read is a coalesced 128-byte row segment
// and each word is formed with one warp ballot.  The tests run in order mean,
// variance, contrast and each later test's corner reads are issued only for
// lanes still alive, so a warp whose candidates all fail the mean test reads
// 8 of the 24 corners.  Corner offsets are precomputed per scale, so a read is
// one load at an immediate offset.  The tables are served from L2 across
// scales; the kernel is bound by the L1 data pipe and by the latency of those
// L2-served reads, which is why a scale's reads are issued together.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "screen.h"

namespace scr {
namespace {

// Warps per block: 16 (4096 x of one row) for the exact reads, whose left and
// right corner segments then meet in one SM's L1; 1 when a scale pre-filters
// on packed planes, where a warp's work varies with how many of its words
// need exact reads and a block slot should free as soon as its warp is done.
// Measured on the 8192^2, 16-scale workload: exact reads 2.61 ms with 16-warp
// blocks against 2.67 / 2.71 / 2.79 / 2.95 ms with 8 / 4 / 2 / 1; pre-filter
// 1.68 ms with 1-warp blocks against 1.75 / 1.76 / 1.87 / 2.26 ms with
// 2 / 4 / 8 / 16 (4 words per warp: 2.11 ms with 4-warp blocks), before the
// bias folding and vote guards below took the 1-warp form to 1.59-1.61 ms.
constexpr int kExactWarpsPerBlock = 16;
constexpr int kFilterWarpsPerBlock = 1;

__device__ __forceinline__ uint32_t ld(const uint32_t *p) { return __ldg(p); }

// Eight corner pointers of one star shape pair (square + diamond) for the
// first word of a warp; word j reads 32*j elements further (immediate offset).
struct Corners {
    const uint32_t *p[8];
    __device__ __forceinline__ Corners(const uint32_t *L, const uint32_t *T, const int32_t (&oL)[4],
                                       const int32_t (&oT)[4]) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            p[k] = L + oL[k];
            p[4 + k] = T + oT[k];
        }
    }
    // square + diamond sum of word j (mod 2^32; exact since the sum is < 2^32)
    __device__ __forceinline__ uint32_t sum(int j) const {
        const int d = 32 * j;
        return ld(p[0] + d) - ld(p[1] + d) - ld(p[2] + d) + ld(p[3] + d) + ld(p[4] + d) - ld(p[5] + d) -
               ld(p[6] + d) + ld(p[7] + d);
    }
};

// Pre-filter of one candidate from tot, the signed sum of its star's eight
// packed corners (mod 2^32).  Its low half, plus 4, is s + 4 where
// s = sum of floor(corner / 2^kS) (mod 2^16) lies strictly within 4 of
// S / 2^kS; its high half, plus 8, is q + 8 where q is the same for Q and 2^kQ
// with the low half's carry (-4 .. 3), strictly within 8 below and 7 above.
// The host picked the window so that neither wraps for a candidate that can
// pass.  So S >= 2^kS (s - 4) and Q <= 2^kQ (q + 8), and the variance
// numerator V = A Q - S^2 of a candidate whose S passes the mean test is at
// most A 2^kQ (q + 8) - max(2^kS (s - 4), S_lo)^2.  The filter rejects the
// candidate when that bound is below V_lo, the variance test's usual failure
// on a background flatter than the template; every other failure is left to
// the exact tests.  It runs in single precision: both halves become floats
// exactly (a byte permute puts them under the exponent of 2^23), the two box
// corners come from one fused multiply-add each (exact products, one
// rounding), and the host lowered V_lo by 4 u (A 2^kQ 65535 + |V_lo|) + 1,
// u = 2^-24, which covers every rounding here.  Candidates the window's range
// does not cover fail the exact tests anyway, so the mask is exact.
// The caller passes tot + kFilterBias: 4 in the low half and 8 in the high
// half, added inside the corner sum.  Adding 4 to the low half carries into
// the high half only for s in -3..-1, which raises q + 8 by one: a larger
// upper bound on Q, still below 2^16 (q + 8 <= 2^16 - 2 in the window's range).
constexpr uint32_t kFilterBias = (8u << 16) + 4u;

__device__ __forceinline__ bool filter_pass(uint32_t biased, const ScaleParam &p) {
    const float ms = __int_as_float(__byte_perm(biased, 0x4B000000u, 0x7610));   // 2^23 + s + 4
    const float mq = __int_as_float(__byte_perm(biased, 0x4B000000u, 0x7632));  // 2^23 + q + 8 (+ 1)
    const float slo = fmaxf(fmaf(p.f2S, ms, p.fS0), p.fSlo);   // max(2^kS (s - 4), S_lo)
    const float x = fmaf(p.fc, mq, p.fQ0);                     // A 2^kQ (q + 8)
    return fmaf(-slo, slo, x) >= p.fVlo;
}

// WPW: mask words per warp.  The warp covers 32*WPW consecutive x; corner
// pointers are formed once per scale and every word reads at an immediate
// offset from them, and the per-scale bookkeeping is shared by all words.
// Warps whose whole span lies inside the valid range take a branch-free path.
// The star-sum reads of all words of a scale are issued back to back; the
// survivors of each test are kept as a per-lane bitmask (bit j = word j); the
// variance and contrast reads are issued only when some lane of the warp is
// still alive (a warp-uniform vote), and only for the live words.
constexpr int WPW = 8;

// PW: the Prewitt gradient test of the star's square (Sec. 3, Eq. S_y with
// the moment tables of Eq. T_x; magnitude of Sec. 4) runs after the others,
// compared squared in 128 bits.  The default kernel has no Prewitt code.
// 64 registers (WB warps per block, 32 / WB blocks per SM) let the batched
// star-sum reads stay in flight together: measured 182 us against 189 us at
// 48 registers and 192 us at 80 on the 4096^2 workload.
template <bool PW, int WB>
__global__ void __launch_bounds__(32 * WB, 32 / WB)
k_screen(const __grid_constant__ ScreenArgs a) {
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * WB + (threadIdx.x >> 5)) * WPW;   // first word
    const int y = blockIdx.y;
    if (w0 >= a.Wwords)
        return;
    const int x0 = w0 * 32 + lane;
    // this candidate's element in every table; corners are fixed offsets from it
    const int64_t e = (int64_t)y * a.pitch + x0 + kColOffset;
    const uint32_t *L1 = a.L1 + e, *L2 = a.L2 + e, *T1 = a.T1 + e, *T2 = a.T2 + e;
    uint32_t *out = a.mask + (int64_t)y * a.Wwords + w0;
    const int64_t plane = (int64_t)a.H * a.Wwords;
    const bool fm = a.features & SCR_F_MEAN, fv = a.features & SCR_F_VAR, fg = a.features & SCR_F_GRAD;
    const bool store_word = lane < WPW && w0 + lane < a.Wwords;
    const int xw_lo = w0 * 32, xw_hi = (w0 + WPW) * 32 - 1;   // span of this warp
#pragma unroll 1
    for (int s = 0; s < a.n_scales; ++s) {
        const ScaleParam &p = a.sp[s];
        uint32_t keep = 0;   // bit j: the candidate of word j is still alive
        if (!p.empty && y >= p.y_lo && y <= p.y_hi) {   // block-uniform
            uint32_t S[WPW];
            if (!PW && p.fw >= 0) {   // block-uniform: pre-filter on a packed plane
                const Corners cf(a.FU[p.fw] + e, a.FC[p.fw] + e, p.oL, p.oT);
                if (xw_lo >= p.x_lo && xw_hi <= p.x_hi) {
                    uint32_t v[WPW][8];
#pragma unroll
                    for (int j = 0; j < WPW; ++j)
#pragma unroll
                        for (int k = 0; k < 8; ++k)
                            v[j][k] = ld(cf.p[k] + 32 * j);
#pragma unroll
                    for (int j = 0; j < WPW; ++j) {
                        const uint32_t tot = v[j][0] - v[j][1] - v[j][2] + v[j][3] + v[j][4] - v[j][5] - v[j][6] +
                                             v[j][7] + kFilterBias;
                        keep |= (filter_pass(tot, p) ? 1u : 0u) << j;
                    }
                } else {
                    const uint32_t span = (uint32_t)(p.x_hi - p.x_lo);
#pragma unroll
                    for (int j = 0; j < WPW; ++j)
                        if ((uint32_t)(x0 + 32 * j - p.x_lo) <= span && filter_pass(cf.sum(j) + kFilterBias, p))
                            keep |= 1u << j;
                }
                // exact star sums of the candidates the filter kept
#pragma unroll
                for (int j = 0; j < WPW; ++j)
                    S[j] = 0;
                if (__any_sync(0xffffffffu, keep != 0)) {
                    const Corners c(L1, T1, p.oL, p.oT);
#pragma unroll
                    for (int j = 0; j < WPW; ++j)
                        if ((keep >> j) & 1u)
                            S[j] = c.sum(j);
                }
            } else if (xw_lo >= p.x_lo && xw_hi <= p.x_hi) {   // warp-uniform: every word valid
                // star sum: square (upright table) + diamond (cone table), Sec. 4
                const Corners c(L1, T1, p.oL, p.oT);
                // all 8 x WPW corner reads are written before any sum, which lets
                // the scheduler issue them back to back (measured ~4% faster than
                // summing word by word)
                uint32_t v[WPW][8];
#pragma unroll
                for (int j = 0; j < WPW; ++j)
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        v[j][k] = ld(c.p[k] + 32 * j);
#pragma unroll
                for (int j = 0; j < WPW; ++j)
                    S[j] = v[j][0] - v[j][1] - v[j][2] + v[j][3] + v[j][4] - v[j][5] - v[j][6] + v[j][7];
                keep = (1u << WPW) - 1;
            } else {
                const Corners c(L1, T1, p.oL, p.oT);
                const uint32_t span = (uint32_t)(p.x_hi - p.x_lo);
#pragma unroll
                for (int j = 0; j < WPW; ++j) {
                    S[j] = 0;
                    if ((uint32_t)(x0 + 32 * j - p.x_lo) <= span) {
                        S[j] = c.sum(j);
                        keep |= 1u << j;
                    }
                }
            }
            if (fm && __any_sync(0xffffffffu, keep != 0)) {
                uint32_t k2 = 0;
#pragma unroll
                for (int j = 0; j < WPW; ++j)
                    k2 |= ((S[j] - p.S_lo) <= p.S_rng ? 1u : 0u) << j;
                keep &= k2;
            }
            if (fv && __any_sync(0xffffffffu, keep != 0)) {
                // the square and diamond sums of I^2 are each below 2^32 but
                // their sum may not be: add them in 64 bits.  The reads of
                // half the words (those still alive) are issued together
                // before any of them is used, so a warp waits for the L2 twice
                // per scale, not once per word: on workloads whose mean test
                // passes most candidates this path runs for nearly every word.
                const Corners cq(L2, T2, p.oL, p.oT);
#pragma unroll
                for (int h = 0; h < WPW; h += WPW / 2) {
                    // a lane with a live word in this half reads all of the
                    // half's corners (one condition, not one per read); the
                    // test of a word that was already dead changes nothing
                    if (!((keep >> h) & ((1u << (WPW / 2)) - 1)))
                        continue;
                    uint32_t q[WPW / 2][8];
#pragma unroll
                    for (int j = 0; j < WPW / 2; ++j)
#pragma unroll
                        for (int k = 0; k < 8; ++k)
                            q[j][k] = ld(cq.p[k] + 32 * (h + j));
#pragma unroll
                    for (int j = 0; j < WPW / 2; ++j) {
                        const uint32_t qs = q[j][0] - q[j][1] - q[j][2] + q[j][3];
                        const uint32_t qd = q[j][4] - q[j][5] - q[j][6] + q[j][7];
                        const uint64_t Q = (uint64_t)qs + qd;
                        const uint64_t V = (uint64_t)p.A * Q - (uint64_t)S[h + j] * S[h + j];   // A^2 * variance
                        if ((V - (uint64_t)p.V_lo) > p.V_rng)
                            keep &= ~(1u << (h + j));
                    }
                }
            }
            if (fg && __any_sync(0xffffffffu, keep != 0)) {
                const Corners ci(L1, T1, p.oLi, p.oTi);   // inner star
#pragma unroll
                for (int j = 0; j < WPW; ++j) {
                    if (!((keep >> j) & 1u))
                        continue;
                    const uint32_t Si = ci.sum(j);
                    const int64_t N = (int64_t)((uint64_t)Si * p.Aring) -
                                      (int64_t)((uint64_t)(S[j] - Si) * p.Ain);
                    if (((uint64_t)N - (uint64_t)p.N_lo) > p.N_rng)
                        keep &= ~(1u << j);
                }
            }
            if (PW && __any_sync(0xffffffffu, keep != 0)) {
                // moments about the square's centre (y + 1/2, x + 1/2), doubled:
                // Gx2 = 2 [Mx window] - (2x + 1) S_sq, Gy2 = 2 [My window] - (2y + 1) S_sq
                const uint64_t *MX = a.Mx + e, *MY = a.My + e;
#pragma unroll
                for (int j = 0; j < WPW; ++j) {
                    if (!((keep >> j) & 1u))
                        continue;
                    const int d = 32 * j;
                    const uint32_t Ssq = ld(L1 + p.oL[0] + d) - ld(L1 + p.oL[1] + d) - ld(L1 + p.oL[2] + d) +
                                         ld(L1 + p.oL[3] + d);
                    const uint64_t mx = __ldg(MX + p.oL[0] + d) - __ldg(MX + p.oL[1] + d) -
                                        __ldg(MX + p.oL[2] + d) + __ldg(MX + p.oL[3] + d);
                    const uint64_t my = __ldg(MY + p.oL[0] + d) - __ldg(MY + p.oL[1] + d) -
                                        __ldg(MY + p.oL[2] + d) + __ldg(MY + p.oL[3] + d);
                    const int64_t gx = (int64_t)(2 * mx - (uint64_t)(2 * (x0 + d) + 1) * Ssq);
                    const int64_t gy = (int64_t)(2 * my - (uint64_t)(2 * y + 1) * Ssq);
                    const uint64_t ax = (uint64_t)(gx < 0 ? -gx : gx), ay = (uint64_t)(gy < 0 ? -gy : gy);
                    const unsigned __int128 g2 = (unsigned __int128)ax * ax + (unsigned __int128)ay * ay;
                    if (g2 - p.P_lo > p.P_rng)
                        keep &= ~(1u << j);
                }
            }
        }
        uint32_t mine = 0;
        if (__any_sync(0xffffffffu, keep != 0)) {
#pragma unroll
            for (int j = 0; j < WPW; ++j) {
                const uint32_t bits = __ballot_sync(0xffffffffu, (keep >> j) & 1u);
                mine = lane == j ? bits : mine;
            }
        }
        if (store_word)
            out[s * plane + lane] = mine;
    }
}

// Star sums of the template's central stars (Sec. 5: features of the central
// areas of the scaled template).  One thread per central radius t; 64-bit
// values assembled from both planes.
struct TmplArgs {
    const uint32_t *L1lo, *L1hi, *L2lo, *L2hi, *T1lo, *T1hi, *T2lo, *T2hi;
    int64_t pL, pT;
    int r, t_min;
    int64_t *out;
};

__device__ __forceinline__ uint64_t v64(const uint32_t *lo, const uint32_t *hi, int64_t pitch, int a, int b) {
    const int64_t o = (int64_t)a * pitch + b + kColOffset;
    return (uint64_t)lo[o] | ((uint64_t)hi[o] << 32);
}

__device__ __forceinline__ uint64_t sq64(const uint32_t *lo, const uint32_t *hi, int64_t p, int y, int x, int n) {
    return v64(lo, hi, p, y + n + 1, x + n + 1) - v64(lo, hi, p, y - n + 1, x + n + 1) -
           v64(lo, hi, p, y + n + 1, x - n + 1) + v64(lo, hi, p, y - n + 1, x - n + 1);
}

__device__ __forceinline__ uint64_t dm64(const uint32_t *lo, const uint32_t *hi, int64_t p, int y, int x, int h) {
    return v64(lo, hi, p, y + h + 1, x + 1) - v64(lo, hi, p, y + 1, x - h + 1) -
           v64(lo, hi, p, y + 1, x + h + 1) + v64(lo, hi, p, y - h + 1, x + 1);
}

__device__ __forceinline__ int square_half_dev(int R) {
    // n with (2n-1)^2 < 2R^2 < (2n+1)^2, from the integer square root of 2R^2
    const int64_t v = 2 * (int64_t)R * R;
    int64_t m = (int64_t)sqrt((double)v);
    while (m * m > v) --m;
    while ((m + 1) * (m + 1) <= v) ++m;
    return (int)((m + 1) / 2);
}

__global__ void k_template_sums(const TmplArgs a) {
    pdl_begin();
    const int t = a.t_min + blockIdx.x * blockDim.x + threadIdx.x;
    if (t > a.r)
        return;
    const int n = square_half_dev(t), ri = t / 2, ni = square_half_dev(ri);
    const int y = a.r, x = a.r;
    const uint64_t S = sq64(a.L1lo, a.L1hi, a.pL, y, x, n) + dm64(a.T1lo, a.T1hi, a.pT, y, x, t);
    const uint64_t Q = sq64(a.L2lo, a.L2hi, a.pL, y, x, n) + dm64(a.T2lo, a.T2hi, a.pT, y, x, t);
    uint64_t Si = 0;
    if (ri >= 1)
        Si = sq64(a.L1lo, a.L1hi, a.pL, y, x, ni) + dm64(a.T1lo, a.T1hi, a.pT, y, x, ri);
    int64_t *o = a.out + 3 * (int64_t)(t - a.t_min);
    o[0] = (int64_t)S;
    o[1] = (int64_t)Q;
    o[2] = (int64_t)Si;
}

}  // namespace

cudaError_t launch_screen(const ScreenArgs &args, cudaStream_t st, uint64_t *launches) {
    const int warps = (args.Wwords + WPW - 1) / WPW;
    bool filtered = false;   // some scale pre-filters on packed planes
    for (int s = 0; s < args.n_scales; ++s)
        filtered |= args.sp[s].fw >= 0;
    cudaError_t e;
    if (args.features & SCR_F_PREWITT) {
        constexpr int WB = kExactWarpsPerBlock;
        e = launch_pdl(k_screen<true, WB>, dim3((warps + WB - 1) / WB, args.H), dim3(32 * WB), st, args);
    } else if (filtered) {
        constexpr int WB = kFilterWarpsPerBlock;
        e = launch_pdl(k_screen<false, WB>, dim3((warps + WB - 1) / WB, args.H), dim3(32 * WB), st, args);
    } else {
        constexpr int WB = kExactWarpsPerBlock;
        e = launch_pdl(k_screen<false, WB>, dim3((warps + WB - 1) / WB, args.H), dim3(32 * WB), st, args);
    }
    if (launches)
        *launches += 1;
    return e;
}

cudaError_t launch_template_sums(const TableDesc &L1, const TableDesc &L2, const TableDesc &T1,
                                 const TableDesc &T2, int r, int t_min, int64_t *out_dev,
                                 cudaStream_t st, uint64_t *launches) {
    TmplArgs a{L1.lo, L1.hi, L2.lo, L2.hi, T1.lo, T1.hi, T2.lo, T2.hi, L1.pitch, T1.pitch, r, t_min, out_dev};
    const int cnt = r - t_min + 1;
    const cudaError_t e = launch_pdl(k_template_sums, dim3((cnt + 127) / 128), dim3(128), st, a);
    if (launches)
        *launches += 1;
    return e;
}

}  // namespace scr
