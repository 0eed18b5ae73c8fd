// Moment tables for the Prewitt gradient (Sec. 3, Eq. T_x and its vertical
// counterpart): Mx(a, b) = sum_{y<a, x<b} x I(y, x) and My(a, b) =
// sum_{y<a, x<b} y I(y, x), 64-bit (exact modulo 2^64), laid out like the
// upright tables (element (a, b) at a * pitch + b + kColOffset).
//
// Three kernels: row prefixes of x I and y I (one block per row, a block scan
// per 1024-pixel chunk with a carry); band sums of each column (64-row bands);
// then per (band, column) a walk down the band adding the exclusive prefix of
// the band sums above it, in place.  No kernel waits on another CTA.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace scr {
namespace {

constexpr int MT = 256;          // threads
constexpr int MBAND = 64;        // rows per band of the column pass

struct MomArgs {
    const uint8_t *img;
    int64_t ipitch;
    int H, W;
    int64_t pitch;               // words (u64) per table row
    uint64_t *Mx, *My;
    uint64_t *bandx, *bandy;     // [nbands][W + 1] band sums
    int nbands;
};

// Row y: Mx[y+1][b] = sum_{x<b} x I(y, x), My[y+1][b] = y * sum_{x<b} I(y, x), b = 0..W;
// block 0 also zeroes row 0.
__global__ void __launch_bounds__(MT) k_mom_rows(const MomArgs a) {
    pdl_begin();
    __shared__ uint64_t shx[MT / 32], shi[MT / 32];
    const int y = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint8_t *row = a.img + (int64_t)y * a.ipitch;
    uint64_t *ox = a.Mx + (int64_t)(y + 1) * a.pitch + kColOffset;
    uint64_t *oy = a.My + (int64_t)(y + 1) * a.pitch + kColOffset;
    if (blockIdx.x == 0)
        for (int b = t; b <= a.W; b += MT) {
            a.Mx[b + kColOffset] = 0;
            a.My[b + kColOffset] = 0;
        }
    if (t == 0) {
        ox[0] = 0;
        oy[0] = 0;
    }
    uint64_t carry_x = 0, carry_i = 0;
    for (int c0 = 0; c0 < a.W; c0 += 4 * MT) {
        uint64_t px[4], pi[4];
        uint64_t sx = 0, si = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int x = c0 + 4 * t + k;
            const uint64_t v = x < a.W ? row[x] : 0u;
            sx += (uint64_t)x * v;
            si += v;
            px[k] = sx;
            pi[k] = si;
        }
        // block-wide inclusive scan of the thread totals
        uint64_t ix = sx, ii = si;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t ux = __shfl_up_sync(0xffffffffu, ix, o), ui = __shfl_up_sync(0xffffffffu, ii, o);
            if (lane >= o) {
                ix += ux;
                ii += ui;
            }
        }
        if (lane == 31) {
            shx[w] = ix;
            shi[w] = ii;
        }
        __syncthreads();
        uint64_t bx = 0, bi = 0, tx = 0, ti = 0;
#pragma unroll
        for (int q = 0; q < MT / 32; ++q) {
            bx += q < w ? shx[q] : 0;
            bi += q < w ? shi[q] : 0;
            tx += shx[q];
            ti += shi[q];
        }
        __syncthreads();
        const uint64_t ex = carry_x + bx + ix - sx, ei = carry_i + bi + ii - si;   // before this thread
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int x = c0 + 4 * t + k;
            if (x < a.W) {
                ox[x + 1] = ex + px[k];
                oy[x + 1] = (uint64_t)y * (ei + pi[k]);
            }
        }
        carry_x += tx;
        carry_i += ti;
    }
}

// band sums: thread per (band, column b)
__global__ void __launch_bounds__(MT) k_mom_bands(const MomArgs a) {
    pdl_begin();
    const int b = blockIdx.x * MT + threadIdx.x, band = blockIdx.y;
    if (b > a.W)
        return;
    const int r0 = 1 + band * MBAND, r1 = min(r0 + MBAND, a.H + 1);
    uint64_t sx = 0, sy = 0;
    for (int r = r0; r < r1; ++r) {
        sx += a.Mx[(int64_t)r * a.pitch + b + kColOffset];
        sy += a.My[(int64_t)r * a.pitch + b + kColOffset];
    }
    a.bandx[(int64_t)band * (a.W + 1) + b] = sx;
    a.bandy[(int64_t)band * (a.W + 1) + b] = sy;
}

// per (band, column): the sum of the bands above, then a walk down the band
__global__ void __launch_bounds__(MT) k_mom_apply(const MomArgs a) {
    pdl_begin();
    const int b = blockIdx.x * MT + threadIdx.x, band = blockIdx.y;
    if (b > a.W)
        return;
    uint64_t cx = 0, cy = 0;
    for (int q = 0; q < band; ++q) {
        cx += a.bandx[(int64_t)q * (a.W + 1) + b];
        cy += a.bandy[(int64_t)q * (a.W + 1) + b];
    }
    const int r0 = 1 + band * MBAND, r1 = min(r0 + MBAND, a.H + 1);
    for (int r = r0; r < r1; ++r) {
        uint64_t *px = a.Mx + (int64_t)r * a.pitch + b + kColOffset;
        uint64_t *py = a.My + (int64_t)r * a.pitch + b + kColOffset;
        cx += *px;
        cy += *py;
        *px = cx;
        *py = cy;
    }
}

}  // namespace

size_t moment_scratch_bytes(int H, int W) {
    const int nb = (H + MBAND - 1) / MBAND;
    return (size_t)2 * nb * (W + 1) * 8 + 256;
}

cudaError_t launch_moment_tables(const uint8_t *img, int64_t ipitch, int H, int W, int64_t pitch, uint64_t *Mx,
                                 uint64_t *My, void *scratch, cudaStream_t st, uint64_t *launches) {
    MomArgs a;
    a.img = img;
    a.ipitch = ipitch;
    a.H = H;
    a.W = W;
    a.pitch = pitch;
    a.Mx = Mx;
    a.My = My;
    a.nbands = (H + MBAND - 1) / MBAND;
    a.bandx = (uint64_t *)scratch;
    a.bandy = a.bandx + (size_t)a.nbands * (W + 1);
    cudaError_t e;
    if (launches)
        *launches += 3;
    if ((e = launch_pdl(k_mom_rows, dim3(H), dim3(MT), st, a)) != cudaSuccess)
        return e;
    const dim3 grid((W + 1 + MT - 1) / MT, a.nbands);
    if ((e = launch_pdl(k_mom_bands, grid, dim3(MT), st, a)) != cudaSuccess)
        return e;
    return launch_pdl(k_mom_apply, grid, dim3(MT), st, a);
}

}  // namespace scr
