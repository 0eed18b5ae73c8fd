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
// Mapping: one warp evaluates one mask word -- 32 consecutive x of one row --
// for every scale, so each corner read is a coalesced 128-byte row segment and
// the word is formed with one warp ballot.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace scr {
namespace {

constexpr int kWarpsPerBlock = 8;

__device__ __forceinline__ uint32_t ld(const uint32_t *p) { return __ldg(p); }

__device__ __forceinline__ uint32_t square_sum(const uint32_t *L, int64_t pitch, int y, int x, int n) {
    const uint32_t *r1 = L + (int64_t)(y + n + 1) * pitch + kColOffset;
    const uint32_t *r0 = L + (int64_t)(y - n + 1) * pitch + kColOffset;
    return ld(r1 + x + n + 1) - ld(r0 + x + n + 1) - ld(r1 + x - n + 1) + ld(r0 + x - n + 1);
}

__device__ __forceinline__ uint32_t diamond_sum(const uint32_t *T, int64_t pitch, int y, int x, int h) {
    const uint32_t *rc = T + (int64_t)(y + 1) * pitch + kColOffset;
    return ld(T + (int64_t)(y + h + 1) * pitch + kColOffset + x + 1) - ld(rc + x - h + 1) -
           ld(rc + x + h + 1) + ld(T + (int64_t)(y - h + 1) * pitch + kColOffset + x + 1);
}

__global__ void __launch_bounds__(32 * kWarpsPerBlock)
k_screen(const __grid_constant__ ScreenArgs a) {
    const int lane = threadIdx.x & 31;
    const int word = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int y = blockIdx.y;
    if (word >= a.Wwords)
        return;
    const int x = word * 32 + lane;
    for (int s = 0; s < a.n_scales; ++s) {
        const ScaleParam &p = a.sp[s];
        bool keep = false;
        if (y >= p.y_lo && y <= p.y_hi && x >= p.x_lo && x <= p.x_hi) {
            const uint32_t S = square_sum(a.L1, a.pitchL, y, x, p.n) + diamond_sum(a.T1, a.pitchT, y, x, p.h);
            keep = true;
            if (a.features & SCR_F_MEAN)
                keep = (int64_t)S >= p.S_lo && (int64_t)S <= p.S_hi;
            if (keep && (a.features & SCR_F_VAR)) {
                const uint64_t Q = (uint64_t)square_sum(a.L2, a.pitchL, y, x, p.n) +
                                   (uint64_t)diamond_sum(a.T2, a.pitchT, y, x, p.h);
                const int64_t V = (int64_t)((uint64_t)p.A * Q - (uint64_t)S * S);
                keep = V >= p.V_lo && V <= p.V_hi;
            }
            if (keep && (a.features & SCR_F_GRAD)) {
                const uint32_t Si = square_sum(a.L1, a.pitchL, y, x, p.ni) + diamond_sum(a.T1, a.pitchT, y, x, p.hi);
                const int64_t N = (int64_t)Si * p.Aring - ((int64_t)S - (int64_t)Si) * p.Ain;
                keep = N >= p.N_lo && N <= p.N_hi;
            }
        }
        const uint32_t bits = __ballot_sync(0xffffffffu, keep);
        if (lane == 0)
            a.mask[((int64_t)s * a.H + y) * a.Wwords + word] = bits;
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
    dim3 grid((args.Wwords + kWarpsPerBlock - 1) / kWarpsPerBlock, args.H);
    k_screen<<<grid, 32 * kWarpsPerBlock, 0, st>>>(args);
    if (launches)
        *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_template_sums(const TableDesc &L1, const TableDesc &L2, const TableDesc &T1,
                                 const TableDesc &T2, int r, int t_min, int64_t *out_dev,
                                 cudaStream_t st, uint64_t *launches) {
    TmplArgs a{L1.lo, L1.hi, L2.lo, L2.hi, T1.lo, T1.hi, T2.lo, T2.hi, L1.pitch, T1.pitch, r, t_min, out_dev};
    const int cnt = r - t_min + 1;
    k_template_sums<<<(cnt + 127) / 128, 128, 0, st>>>(a);
    if (launches)
        *launches += 1;
    return cudaGetLastError();
}

}  // namespace scr
