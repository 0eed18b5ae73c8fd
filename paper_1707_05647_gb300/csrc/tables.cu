// Summed-area tables of I and I^2: upright (Sec. 3, Eq. T_1) and 45-degree
// "cone" tables (Sec. 4, triangular summed-area map), built together.
//
// Definitions (row y, column x; P(y, x) = sum_{x' <= x} I(y, x') is the row
// prefix, zero for x < 0 and the row total for x >= W):
//   L(a, b)   = sum_{y < a, x < b} I(y, x)          = sum_{y < a} P(y, b-1)
//   cone(r,c) = sum of I over y <= r, |x - c| <= r - y
//             = D1(r, c) - D2(r, c), with
//   D1(r, c)  = sum_{y <= r} P(y, c + (r - y))      (anti-diagonal prefix)
//   D2(r, c)  = sum_{y <= r} P(y, c - 1 - (r - y))  (diagonal prefix)
// because row y's part of the cone is P(y, c + r - y) - P(y, c - r + y - 1).
// The paper builds its rotated table with "two diagonal passes of cumulative
// sum" (Sec. 4); D1 and D2 are those two passes.
//
// Work decomposition.  The image is cut into bands of kBand rows and each band
// into tiles of kTileCols columns.  A tile needs, for its first row, the values
// of L, D1 and D2 on the row just above its band -- "carries" that depend on
// every pixel above.  They are linear in the pixels, so they are assembled from
// per-band partial sums in three stages, with no inter-CTA waiting:
//   k_tab_reduce  per tile: column sums, anti-diagonal and diagonal sums of the
//                 band (each restricted to the band), row sums.
//   k_tab_carry   per column / diagonal index: exclusive prefix over bands.
//   k_tab_prefix  per band: prefix along the row of those sums -> the carry
//                 rows L(r0, .), D1(r0-1, .), D2(r0-1, .) and per-tile row carries.
//   k_tab_write   one warp per (band, 192-column warp tile): lane l owns 8
//                 adjacent columns of the tile's 256 slots (32 halo slots on
//                 each side) and keeps L, D1, D2 for them in registers.  Per row
//                 it forms P with one warp scan of the lanes' pixel sums plus
//                 the tile's row carry, adds P to L, moves D1 one column left
//                 and D2 one column right (register moves plus one neighbour
//                 shuffle), puts the core columns' L and T = D1 - D2 into a
//                 double-buffered shared-memory row, and one lane writes each
//                 plane's 768-byte row segment with a bulk copy (cp.async.bulk).
//                 No block barrier and no inter-warp exchange.
// A warp tile carries kHalo extra columns on each side so its D1 (which flows
// in from the right) and D2 (from the left) stay exact over its core columns
// for the kBand rows of a band.  When packed filter planes are requested
// (FilterPlanes, up to two bit windows), the writer packs the same registers'
// L1/L2 and T1/T2 bits into them and copies their rows out with the others.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace scr {
namespace {

// Programmatic dependent launch for the table kernels: each waits for its
// predecessor at its start but does not release its successor early, so the
// successor's blocks launch when this grid has finished instead of waiting in
// the SM slots its last wave frees.  Measured: build 0.552 -> 0.548 ms on
// 8192x8192 (u64 tables) and 0.151 -> 0.142 ms on 4096x4096; releasing the
// screening kernel at the writer's start (see k_tab_write) cost 0.5 ms.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

constexpr int B = kBand;
constexpr int CW = kTileCols;
constexpr int HALO = kHalo;
constexpr int SLOTS = kTileSlots;            // 1024 accumulator columns per tile
constexpr int NT = 256;                      // threads of k_tab_reduce
constexpr int WK = 8;                        // columns per k_tab_write lane
constexpr int WS = 32 * WK;                  // 256 slots per warp tile
constexpr int WCW = WS - 2 * HALO;           // 192 core columns per warp tile
constexpr int WPR = CW / WCW;                // warp tiles per reduce tile (5)
constexpr int CL = kWinLo;                   // first carry column
static_assert(CW % WCW == 0, "a reduce tile holds whole warp-tile chunks");
static_assert(B == 32, "row carries are held one per lane");

struct Geometry {
    int H, W, n, m;          // bands, reduce tiles (CW core columns each)
    int mw;                  // warp tiles per band (WCW core columns each)
    int XW;                  // carry columns c in [CL, W+1]
    int XWp;                 // row pitch of the carry arrays (XW rounded up to 4)
    int DMIN, DN;            // anti-diagonal lanes d in [DMIN, DMIN+DN)
    int FMIN, FN;            // diagonal lanes f in [FMIN, FMIN+FN)
    Geometry(int H_, int W_) : H(H_), W(W_) {
        n = (H + B - 1) / B;
        m = W / CW + 1;      // the core columns of the tiles reach past column W
        mw = W / WCW + 1;
        XW = W + 1 - CL + 1;
        XWp = (XW + 3) & ~3;
        DMIN = CL - 1;
        DN = (n - 1) * B + W + 2 - DMIN;
        FMIN = CL - (n - 1) * B;
        FN = (W + 1) - FMIN + 1;
    }
};

// Scratch layout (32-bit words unless noted), carved from one buffer.
struct Scratch {
    uint32_t *cs1, *cs2;     // [n][W]        column sums of the band
    uint32_t *ad1, *ad2;     // [n][W+B-1]    anti-diagonal sums, x' + B-1
    uint32_t *md1, *md2;     // [n][W+B-1]    diagonal sums, x''
    uint32_t *rs1, *rs2;     // [n][mw][B]    row sums over each warp tile's shifted chunk
    uint32_t *csx1, *csx2;   // [n][XWp]      exclusive band prefix of cs at x = c (0 outside the image)
    uint32_t *adx1, *adx2;   // [n][XWp]      AD_i(r0-1+c)
    uint32_t *mdx1, *mdx2;   // [n][XWp]      MD_i(c-r0)
    uint32_t *adf1, *adf2;   // [DN]          full anti-diagonal sums, index d - DMIN
    uint32_t *rc1, *rc2;     // [n][mw][B]    row carries P(r, c0-HALO-1) of each warp tile
    void *xl1, *xl2, *x11, *x12, *x21, *x22;   // [n][XWp] carry rows, table width
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

size_t carve(const Geometry &g, int sb, int qb, Scratch *s, char *base) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    const size_t n = g.n, W = g.W, m = g.mw, XW = g.XWp;
    s->cs1 = (uint32_t *)take(n * W * 4);
    s->cs2 = (uint32_t *)take(n * W * 4);
    s->ad1 = (uint32_t *)take(n * (W + B - 1) * 4);
    s->ad2 = (uint32_t *)take(n * (W + B - 1) * 4);
    s->md1 = (uint32_t *)take(n * (W + B - 1) * 4);
    s->md2 = (uint32_t *)take(n * (W + B - 1) * 4);
    s->rs1 = (uint32_t *)take(n * m * B * 4);
    s->rs2 = (uint32_t *)take(n * m * B * 4);
    s->csx1 = (uint32_t *)take(n * XW * 4);
    s->csx2 = (uint32_t *)take(n * XW * 4);
    s->adx1 = (uint32_t *)take(n * XW * 4);
    s->adx2 = (uint32_t *)take(n * XW * 4);
    s->mdx1 = (uint32_t *)take(n * XW * 4);
    s->mdx2 = (uint32_t *)take(n * XW * 4);
    s->adf1 = (uint32_t *)take((size_t)g.DN * 4);
    s->adf2 = (uint32_t *)take((size_t)g.DN * 4);
    s->rc1 = (uint32_t *)take(n * m * B * 4);
    s->rc2 = (uint32_t *)take(n * m * B * 4);
    const size_t es = sb / 8, eq = qb / 8;
    s->xl1 = take(n * XW * es);
    s->xl2 = take(n * XW * eq);
    s->x11 = take(n * XW * es);
    s->x12 = take(n * XW * eq);
    s->x21 = take(n * XW * es);
    s->x22 = take(n * XW * eq);
    return off;
}

// ----------------------------------------------------------------------------
// Stage 1: per-tile band sums.
// ----------------------------------------------------------------------------
struct ReduceArgs {
    const uint8_t *img;
    int64_t pitch;
    Geometry g;
    Scratch s;
    int aligned8;
};

__device__ __forceinline__ uint2 load8(const uint8_t *img, int64_t pitch, int H, int W, int aligned8, int y,
                                       int cs) {
    if (y < H && aligned8 && cs >= 0 && cs + 8 <= W)
        return __ldg(reinterpret_cast<const uint2 *>(img + (int64_t)y * pitch + cs));
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int x = cs + k;
        const uint32_t b = (y < H && x >= 0 && x < W) ? (uint32_t)__ldg(img + (int64_t)y * pitch + x) : 0u;
        if (k < 4)
            lo |= b << (8 * k);
        else
            hi |= b << (8 * (k - 4));
    }
    return make_uint2(lo, hi);
}

constexpr int TROW = SLOTS + 32;   // smem bytes per tile row: word reads past the last slot stay inside

// Rows r..r+3 (one 32-bit word each, byte k = column k) -> c[k] = column k's four rows.
__device__ __forceinline__ void transpose4(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3, uint32_t (&c)[4]) {
    const uint32_t t0 = __byte_perm(r0, r1, 0x5140), t1 = __byte_perm(r0, r1, 0x7362);
    const uint32_t t2 = __byte_perm(r2, r3, 0x5140), t3 = __byte_perm(r2, r3, 0x7362);
    c[0] = __byte_perm(t0, t2, 0x5410);
    c[1] = __byte_perm(t0, t2, 0x7632);
    c[2] = __byte_perm(t1, t3, 0x5410);
    c[3] = __byte_perm(t1, t3, 0x7632);
}

// Sums of I and I^2 over the band's B rows along four adjacent lines whose
// pixels in row rr start at smem byte O + off(rr), O a multiple of 4:
// MODE 0 columns (off = 0), MODE 1 anti-diagonals (off = B-1-rr: the line
// through (r_end - k, x' + k)), MODE 2 diagonals (off = rr-(B-1): through
// (r_end - k, x'' - k)).  One 32-bit window per row (a funnel shift of two
// aligned words), 4x4 byte transposes, dp4a for both sums.
template <int MODE>
__device__ __forceinline__ void line_sums(const uint32_t *t32, int O, uint32_t (&s1)[4], uint32_t (&s2)[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
        s1[k] = s2[k] = 0;
    const int Ow = O >> 2;
#pragma unroll
    for (int r = 0; r < B; r += 4) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int rr = r + q;
            const int off = MODE == 0 ? 0 : (MODE == 1 ? B - 1 - rr : rr - (B - 1));
            const int sh = off & 3;                       // O is a multiple of 4
            const uint32_t *row = t32 + rr * (TROW / 4) + Ow + (off - sh) / 4;
            w[q] = sh ? __funnelshift_r(row[0], row[1], 8 * sh) : row[0];
        }
        uint32_t c[4];
        transpose4(w[0], w[1], w[2], w[3], c);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            s1[k] = __dp4a(c[k], 0x01010101u, s1[k]);
            s2[k] = __dp4a(c[k], c[k], s2[k]);
        }
    }
}

__global__ void __launch_bounds__(NT) k_tab_reduce(const ReduceArgs a) {
    pdl_wait();
    __shared__ __align__(16) uint8_t tile[B][TROW];
    const Geometry &g = a.g;
    const int j = blockIdx.x, i = blockIdx.y, t = threadIdx.x;
    const int r0 = i * B;
    const int c0 = j * CW;
    const int c1 = min(c0 + CW, g.W);
    const int base = c0 - HALO;                  // smem column 0 (a multiple of 4)
    // load the band (zero outside the image): thread t covers 8 columns of
    // B / (NT / 128) rows, all loads in flight
    {
        constexpr int RPT = B / (NT / 128);      // rows per thread
        const int cs = base + 8 * (t & 127);
        const int rb = (t >> 7) * RPT;
        uint2 w[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k)
            w[k] = load8(a.img, a.pitch, g.H, g.W, a.aligned8, r0 + rb + k, cs);
#pragma unroll
        for (int k = 0; k < RPT; ++k)
            *reinterpret_cast<uint2 *>(&tile[rb + k][8 * (t & 127)]) = w[k];
        if (t < B)   // the row pads are read only for lines past the tile, whose sums are dropped
            *reinterpret_cast<uint4 *>(&tile[t][SLOTS]) = make_uint4(0, 0, 0, 0);
    }
    __syncthreads();
    const uint32_t *t32 = reinterpret_cast<const uint32_t *>(&tile[0][0]);
    // row sums over the warp tiles' shifted chunks [c0w-HALO, c0w-HALO+WCW),
    // c0w = (j*WPR + q)*WCW: 8 threads per (row, chunk), 6 words each
    {
        constexpr int TPI = 8;
        constexpr int WPI = WCW / 4 / TPI;
        const int sub = t % TPI;
#pragma unroll 1
        for (int u = t / TPI; u < B * WPR; u += NT / TPI) {
            const int rr = u / WPR, q = u % WPR;
            const uint32_t *row = t32 + rr * (TROW / 4) + q * (WCW / 4) + sub * WPI;
            uint32_t s1 = 0, s2 = 0;
#pragma unroll
            for (int w4i = 0; w4i < WPI; ++w4i) {
                const uint32_t w4 = row[w4i];
                s1 = __dp4a(w4, 0x01010101u, s1);
                s2 = __dp4a(w4, w4, s2);
            }
#pragma unroll
            for (int o = 1; o < TPI; o <<= 1) {
                s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            }
            const int jw = j * WPR + q;
            if (sub == 0 && jw < g.mw) {
                const size_t o = ((size_t)i * g.mw + jw) * B + rr;
                a.s.rs1[o] = s1;
                a.s.rs2[o] = s2;
            }
        }
    }
    const size_t W = g.W, WD = g.W + B - 1;
    uint32_t s1[4], s2[4];
    // column sums, four columns per step
    for (int x0 = c0 + 4 * t; x0 < c1; x0 += 4 * NT) {
        line_sums<0>(t32, x0 - base, s1, s2);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (x0 + k < c1) {
                a.s.cs1[(size_t)i * W + x0 + k] = s1[k];
                a.s.cs2[(size_t)i * W + x0 + k] = s2[k];
            }
    }
    // anti-diagonal sums through (r_end, x'): sum_k I(r_end-k, x'+k), x' in [xa0, c1)
    const int xa0 = (j == 0) ? -(B - 1) : c0;
    for (int xp0 = (j == 0 ? -B : c0) + 4 * t; xp0 < c1; xp0 += 4 * NT) {
        line_sums<1>(t32, xp0 - base, s1, s2);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int xp = xp0 + k;
            if (xp >= xa0 && xp < c1) {
                a.s.ad1[(size_t)i * WD + xp + B - 1] = s1[k];
                a.s.ad2[(size_t)i * WD + xp + B - 1] = s2[k];
            }
        }
    }
    // diagonal sums through (r_end, x''): sum_k I(r_end-k, x''-k), x'' in [c0, xm1)
    const int xm1 = (j == g.m - 1) ? g.W + B - 1 : c1;
    for (int xpp0 = c0 + 4 * t; xpp0 < xm1; xpp0 += 4 * NT) {
        line_sums<2>(t32, xpp0 - base, s1, s2);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int xpp = xpp0 + k;
            if (xpp < xm1) {
                a.s.md1[(size_t)i * WD + xpp] = s1[k];
                a.s.md2[(size_t)i * WD + xpp] = s2[k];
            }
        }
    }
}

// ----------------------------------------------------------------------------
// Stage 2: exclusive prefix over bands, per column (cs), anti-diagonal (ad)
// and diagonal (md) index.  Block = 32 lanes x 32 band groups.
// ----------------------------------------------------------------------------
struct CarryArgs {
    Geometry g;
    Scratch s;
    int chunksCS, chunksAD;   // 32-lane chunks of the first two parts
};

__device__ __forceinline__ void carry_contrib(const CarryArgs &a, int part, int lane_idx, int band,
                                              uint32_t &v1, uint32_t &v2) {
    const Geometry &g = a.g;
    const size_t WD = g.W + B - 1;
    v1 = v2 = 0;
    if (part == 0) {
        const int x = lane_idx + CL;                        // column c of the carry window
        if (x >= 0 && x < g.W) {
            const size_t o = (size_t)band * g.W + x;
            v1 = a.s.cs1[o];
            v2 = a.s.cs2[o];
        }
    } else if (part == 1) {
        const int xp = g.DMIN + lane_idx - (band * B + B - 1);     // d - r_end
        if (xp >= -(B - 1) && xp <= g.W - 1) {
            const size_t o = (size_t)band * WD + xp + B - 1;
            v1 = a.s.ad1[o];
            v2 = a.s.ad2[o];
        }
    } else {
        const int f = g.FMIN + lane_idx;
        const int xpp = f + band * B + B - 1;             // f + r_end
        if (xpp >= 0 && xpp <= g.W + B - 2) {
            const size_t o = (size_t)band * WD + xpp;
            v1 = a.s.md1[o];
            v2 = a.s.md2[o];
        }
    }
}

constexpr int CG = 8;   // band groups per carry block
constexpr int CQ = 16;  // bands per group kept in registers (more bands: reloaded)

__global__ void __launch_bounds__(32 * CG, 5) k_tab_carry(const CarryArgs a) {
    pdl_wait();
    __shared__ uint32_t sum1[CG][33], sum2[CG][33];
    const Geometry &g = a.g;
    const int lane = threadIdx.x, grp = threadIdx.y;
    int chunk = blockIdx.x, part, nlanes;
    if (chunk < a.chunksCS) {
        part = 0;
        nlanes = g.XW;
    } else if (chunk < a.chunksCS + a.chunksAD) {
        part = 1;
        chunk -= a.chunksCS;
        nlanes = g.DN;
    } else {
        part = 2;
        chunk -= a.chunksCS + a.chunksAD;
        nlanes = g.FN;
    }
    const int idx = chunk * 32 + lane;
    const bool live = idx < nlanes;
    const int q = (g.n + CG - 1) / CG;
    const int b0 = grp * q, b1 = min(g.n, b0 + q);
    uint32_t c1[CQ], c2[CQ];
    uint32_t t1 = 0, t2 = 0;
#pragma unroll
    for (int k = 0; k < CQ; ++k) {
        c1[k] = c2[k] = 0;
        if (live && b0 + k < b1)
            carry_contrib(a, part, idx, b0 + k, c1[k], c2[k]);
        t1 += c1[k];
        t2 += c2[k];
    }
    if (live)
        for (int b = b0 + CQ; b < b1; ++b) {
            uint32_t v1, v2;
            carry_contrib(a, part, idx, b, v1, v2);
            t1 += v1;
            t2 += v2;
        }
    sum1[grp][lane] = t1;
    sum2[grp][lane] = t2;
    __syncthreads();
    if (grp == 0) {
        uint32_t r1 = 0, r2 = 0;
        for (int k = 0; k < CG; ++k) {
            const uint32_t u1 = sum1[k][lane], u2 = sum2[k][lane];
            sum1[k][lane] = r1;
            sum2[k][lane] = r2;
            r1 += u1;
            r2 += u2;
        }
        if (part == 1 && live) {
            a.s.adf1[idx] = r1;
            a.s.adf2[idx] = r2;
        }
    }
    __syncthreads();
    if (!live)
        return;
    uint32_t run1 = sum1[grp][lane], run2 = sum2[grp][lane];
    const size_t XW = g.XWp;
    auto put = [&](int b) {
        if (part == 0) {
            const size_t o = (size_t)b * XW + idx;
            a.s.csx1[o] = run1;
            a.s.csx2[o] = run2;
        } else if (part == 1) {
            const int c = g.DMIN + idx - (b * B - 1);     // d = r0 - 1 + c
            if (c >= CL && c <= g.W + 1) {
                a.s.adx1[(size_t)b * XW + (size_t)(c - CL)] = run1;
                a.s.adx2[(size_t)b * XW + (size_t)(c - CL)] = run2;
            }
        } else {
            const int c = g.FMIN + idx + b * B;           // f = c - r0
            if (c >= CL && c <= g.W + 1) {
                a.s.mdx1[(size_t)b * XW + (size_t)(c - CL)] = run1;
                a.s.mdx2[(size_t)b * XW + (size_t)(c - CL)] = run2;
            }
        }
    };
#pragma unroll
    for (int k = 0; k < CQ; ++k) {
        if (b0 + k >= b1)
            break;
        put(b0 + k);
        run1 += c1[k];
        run2 += c2[k];
    }
    for (int b = b0 + CQ; b < b1; ++b) {
        put(b);
        uint32_t v1, v2;
        carry_contrib(a, part, idx, b, v1, v2);
        run1 += v1;
        run2 += v2;
    }
}

// ----------------------------------------------------------------------------
// Stage 3: per band, prefix along the row -> carry rows in table width.
// ----------------------------------------------------------------------------
struct PrefixArgs {
    Geometry g;
    Scratch s;
};

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v += u;
    }
    return v;
}

// One CTA per (band, sequence).  Each warp scans a contiguous segment of the
// row 32 entries at a time (coalesced), after one pass that sums the segment.
constexpr int PT = 256;

template <typename TS, typename TQ>
__global__ void __launch_bounds__(PT, 4) k_tab_prefix(const PrefixArgs a) {
    pdl_wait();
    __shared__ uint64_t wsum[PT / 32], red[PT / 32];
    const Geometry &g = a.g;
    const int i = blockIdx.x, q = blockIdx.y, t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int r0 = i * B;
    const int XW = g.XW;
    if (q == 6) {   // row carries per warp tile: sum of the row sums of the chunks to the left
        // lane = row of the band; warp w takes a contiguous run of chunks
        __shared__ uint32_t tot1[PT / 32][B], tot2[PT / 32][B];
        const int seg = (g.mw + PT / 32 - 1) / (PT / 32);
        const int j0 = w * seg, j1 = min(g.mw, j0 + seg);
        uint32_t s1 = 0, s2 = 0;
        for (int j = j0; j < j1; ++j) {
            const size_t o = ((size_t)i * g.mw + j) * B + lane;
            s1 += a.s.rs1[o];
            s2 += a.s.rs2[o];
        }
        tot1[w][lane] = s1;
        tot2[w][lane] = s2;
        __syncthreads();
        uint32_t c1 = 0, c2 = 0;
        for (int u = 0; u < w; ++u) {
            c1 += tot1[u][lane];
            c2 += tot2[u][lane];
        }
        for (int j = j0; j < j1; ++j) {
            const size_t o = ((size_t)i * g.mw + j) * B + lane;
            const uint32_t v1 = a.s.rs1[o], v2 = a.s.rs2[o];
            a.s.rc1[o] = c1;
            a.s.rc2[o] = c2;
            c1 += v1;
            c2 += v2;
        }
        return;
    }
    // q: 0,1 = L (column prefix), 2,3 = D1 (anti-diagonal), 4,5 = D2 (diagonal);
    // even = sum table, odd = sum-of-squares table
    const uint32_t *src;
    void *dst;
    switch (q) {
        case 0: src = a.s.csx1; dst = a.s.xl1; break;
        case 1: src = a.s.csx2; dst = a.s.xl2; break;
        case 2: src = a.s.adx1; dst = a.s.x11; break;
        case 3: src = a.s.adx2; dst = a.s.x12; break;
        case 4: src = a.s.mdx1; dst = a.s.x21; break;
        default: src = a.s.mdx2; dst = a.s.x22; break;
    }
    // every sequence is a row of XWp words (16-byte aligned); each lane takes 4
    // consecutive entries per step, each warp a contiguous segment
    const uint32_t *row = src + (size_t)i * g.XWp;
    constexpr int MAXIT = 5;                                   // 128-entry steps kept in registers
    const int seg = ((XW + PT / 32 - 1) / (PT / 32) + 127) / 128 * 128;   // entries per warp
    const int k0 = w * seg, k1 = min(XW, k0 + seg);
    auto load4 = [&](int k) -> uint4 {                         // k multiple of 4
        if (k + 4 <= k1)
            return *reinterpret_cast<const uint4 *>(row + k);
        uint32_t v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            v[u] = (k + u < k1) ? row[k + u] : 0u;
        return make_uint4(v[0], v[1], v[2], v[3]);
    };
    uint64_t tri = 0;
    if (q == 2 || q == 3) {
        // anti-diagonals d < r0 - 1 + CL lie entirely above the band
        const uint32_t *adf = q == 2 ? a.s.adf1 : a.s.adf2;
        const int dend = r0 - 1 + CL;
        for (int d = t; d < dend; d += PT)
            tri += adf[d - g.DMIN];
    }
    uint4 v[MAXIT];
    uint64_t part = 0;
#pragma unroll
    for (int it = 0; it < MAXIT; ++it) {
        const int k = k0 + 128 * it + 4 * lane;
        v[it] = (k < k1) ? load4(k) : make_uint4(0, 0, 0, 0);
        part += (uint64_t)v[it].x + v[it].y + v[it].z + v[it].w;
    }
    for (int k = k0 + 128 * MAXIT + 4 * lane; k < k1; k += 128) {   // very wide images only
        const uint4 u = load4(k);
        part += (uint64_t)u.x + u.y + u.z + u.w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        part += __shfl_xor_sync(0xffffffffu, part, o);
        tri += __shfl_xor_sync(0xffffffffu, tri, o);
    }
    if (lane == 0) {
        wsum[w] = part;
        red[w] = tri;
    }
    __syncthreads();
    uint64_t carry = 0;
    for (int u = 0; u < PT / 32; ++u) {
        carry += red[u];
        if (u < w)
            carry += wsum[u];
    }
    auto step = [&](int k, uint4 u) {
        const uint64_t p0 = u.x, p1 = p0 + u.y, p2 = p1 + u.z, p3 = p2 + u.w;
        const uint64_t incl = warp_incl_scan(p3, lane);
        const uint64_t base = carry + incl - p3;
        if (k < k1) {
            const uint64_t o[4] = {base + p0, base + p1, base + p2, base + p3};
            if (q & 1) {
                TQ *d = (TQ *)dst + (size_t)i * g.XWp + k;
                if (k + 4 <= k1 && sizeof(TQ) == 4)
                    *reinterpret_cast<uint4 *>(d) = make_uint4((uint32_t)o[0], (uint32_t)o[1], (uint32_t)o[2], (uint32_t)o[3]);
                else
                    for (int e = 0; e < 4; ++e)
                        if (k + e < k1) d[e] = (TQ)o[e];
            } else {
                TS *d = (TS *)dst + (size_t)i * g.XWp + k;
                if (k + 4 <= k1 && sizeof(TS) == 4)
                    *reinterpret_cast<uint4 *>(d) = make_uint4((uint32_t)o[0], (uint32_t)o[1], (uint32_t)o[2], (uint32_t)o[3]);
                else
                    for (int e = 0; e < 4; ++e)
                        if (k + e < k1) d[e] = (TS)o[e];
            }
        }
        carry += __shfl_sync(0xffffffffu, incl, 31);
    };
#pragma unroll
    for (int it = 0; it < MAXIT; ++it) {
        const int kb = k0 + 128 * it;
        if (kb >= k1)
            break;
        step(kb + 4 * lane, v[it]);
    }
    for (int kb = k0 + 128 * MAXIT; kb < k1; kb += 128) {
        const int k = kb + 4 * lane;
        step(k, k < k1 ? load4(k) : make_uint4(0, 0, 0, 0));
    }
}

// ----------------------------------------------------------------------------
// Stage 4: per warp tile, walk the band's rows and write L1, L2, T1, T2.
// ----------------------------------------------------------------------------
struct WriteArgs {
    const uint8_t *img;
    int64_t pitch;
    Geometry g;
    Scratch s;
    uint32_t *L1lo, *L1hi, *L2lo, *L2hi, *T1lo, *T1hi, *T2lo, *T2hi;
    int64_t pL, pT;
    int aligned8;
    FilterPlanes F;   // packed planes (pitch pL for the upright, pT for the cone planes)
};

// bits kS .. kS+15 of a and kQ .. kQ+15 of b in one word (low, high half)
__device__ __forceinline__ uint32_t pack_window(uint32_t a, uint32_t b, int kS, int kQ) {
    return ((a >> kS) & 0xffffu) | ((b >> kQ) << 16);
}

template <typename TS, typename TQ>
__device__ __forceinline__ void pack8(const TS (&a)[WK], const TQ (&b)[WK], int kS, int kQ, uint32_t (&o)[WK]) {
#pragma unroll
    for (int k = 0; k < WK; ++k)
        o[k] = pack_window((uint32_t)a[k], (uint32_t)b[k], kS, kQ);
}

// WK consecutive values at a 16-byte aligned word: two 16-byte stores per plane
template <typename T>
__device__ __forceinline__ void store8(uint32_t *lo, uint32_t *hi, int64_t word, const T (&v)[WK]) {
    uint4 *pl = reinterpret_cast<uint4 *>(lo + word);
    pl[0] = make_uint4((uint32_t)v[0], (uint32_t)v[1], (uint32_t)v[2], (uint32_t)v[3]);
    pl[1] = make_uint4((uint32_t)v[4], (uint32_t)v[5], (uint32_t)v[6], (uint32_t)v[7]);
    if (sizeof(T) == 8) {
        uint4 *ph = reinterpret_cast<uint4 *>(hi + word);
        ph[0] = make_uint4((uint32_t)((uint64_t)v[0] >> 32), (uint32_t)((uint64_t)v[1] >> 32),
                           (uint32_t)((uint64_t)v[2] >> 32), (uint32_t)((uint64_t)v[3] >> 32));
        ph[1] = make_uint4((uint32_t)((uint64_t)v[4] >> 32), (uint32_t)((uint64_t)v[5] >> 32),
                           (uint32_t)((uint64_t)v[6] >> 32), (uint32_t)((uint64_t)v[7] >> 32));
    }
}

// WK consecutive values into a shared-memory row (low words; high words into hi
// when the table is 64-bit; hi aliases lo otherwise and is not written)
template <typename T>
__device__ __forceinline__ void put8(uint32_t *lo, uint32_t *hi, int at, const T (&v)[WK]) {
    uint4 *pl = reinterpret_cast<uint4 *>(lo + at);
    pl[0] = make_uint4((uint32_t)v[0], (uint32_t)v[1], (uint32_t)v[2], (uint32_t)v[3]);
    pl[1] = make_uint4((uint32_t)v[4], (uint32_t)v[5], (uint32_t)v[6], (uint32_t)v[7]);
    if (sizeof(T) == 8) {
        uint4 *ph = reinterpret_cast<uint4 *>(hi + at);
        ph[0] = make_uint4((uint32_t)((uint64_t)v[0] >> 32), (uint32_t)((uint64_t)v[1] >> 32),
                           (uint32_t)((uint64_t)v[2] >> 32), (uint32_t)((uint64_t)v[3] >> 32));
        ph[1] = make_uint4((uint32_t)((uint64_t)v[4] >> 32), (uint32_t)((uint64_t)v[5] >> 32),
                           (uint32_t)((uint64_t)v[6] >> 32), (uint32_t)((uint64_t)v[7] >> 32));
    }
}

template <typename T>
__device__ __forceinline__ void store1(uint32_t *lo, uint32_t *hi, int64_t word, T v) {
    lo[word] = (uint32_t)v;
    if (sizeof(T) == 8)
        hi[word] = (uint32_t)((uint64_t)v >> 32);
}

// One warp per (band, warp tile); lane l owns the WK adjacent columns
// cs = c0 - HALO + WK*l .. cs + WK - 1 of the tile's WS slots.  Per row the
// lane scans its pixels, a warp scan plus the tile's row carry gives P, D1
// moves one column left and D2 one column right (register moves plus one
// neighbour shuffle), and the core lanes store L and T = D1 - D2.  The warp
// needs no other warp: D1 and D2 values that flow in from outside the tile are
// taken as the tile's own edge value (right) or 0 (left); an error entering at
// an edge moves one column per row, so after the band's B rows it has crossed
// at most B = HALO columns and never reaches the core.  At the right end of the
// image D1 is constant in the column, so there the edge value is exact.
//
// Programmatic dependent launch: the writer waits for the prefix kernel at its
// start, and lets the next kernel (the screening kernel) launch only when its
// own rows are written.  Released at the start, the screening kernel's blocks
// took the SM slots freed during the writer's last wave and waited there, and
// the build-then-screen sequence took 3.87 ms instead of 3.35 on the
// 8192x8192 workload (measured).
template <typename TS, typename TQ, int NF>
__global__ void __launch_bounds__(32) k_tab_write(const WriteArgs a) {
    // planes of a row in obuf: L1 (lo[, hi]), L2 (lo[, hi]), NF packed upright
    // planes, T1 (lo[, hi]), T2 (lo[, hi]), NF packed cone planes
    constexpr int HS = sizeof(TS) == 8 ? 1 : 0, HQ = sizeof(TQ) == 8 ? 1 : 0;
    constexpr int PL1 = 0, PL2 = PL1 + 1 + HS, PFU = PL2 + 1 + HQ, PT1 = PFU + NF, PT2 = PT1 + 1 + HS;
    constexpr int PFC = PT2 + 1 + HQ, NPL = PFC + NF;
    pdl_wait();
    const Geometry &g = a.g;
    const int j = blockIdx.x, i = blockIdx.y, lane = threadIdx.x;
    const int r0 = i * B;
    const int rows = min(B, g.H - r0);
    const int c0 = j * WCW;
    const bool last = (j == g.mw - 1);
    const int cs = c0 - HALO + WK * lane;
    const int cTmax = last ? g.W : c0 + WCW - 1;     // last T column this tile writes
    const int cLmax = last ? g.W - 1 : c0 + WCW - 1; // last L column (b = c+1 <= W)
    const bool wT = cs >= c0 && cs <= cTmax;
    const bool wL = cs >= c0 && cs <= cLmax;
    const bool wEdge = (j == 0) && (cs == -WK);     // holds column c = -1 (b = 0)

    // carries from the row above the band
    TS L1a[WK], D1a[WK], D2a[WK];
    TQ L2a[WK], D1b[WK], D2b[WK];
    {
        const size_t XW = g.XWp;
        const TS *xl1 = (const TS *)a.s.xl1, *x11 = (const TS *)a.s.x11, *x21 = (const TS *)a.s.x21;
        const TQ *xl2 = (const TQ *)a.s.xl2, *x12 = (const TQ *)a.s.x12, *x22 = (const TQ *)a.s.x22;
#pragma unroll
        for (int k = 0; k < WK; ++k) {
            int c = cs + k;
            c = c < CL ? CL : (c > g.W + 1 ? g.W + 1 : c);
            const size_t o = (size_t)i * XW + (size_t)(c - CL);
            L1a[k] = xl1[o];
            L2a[k] = xl2[o];
            D1a[k] = x11[o];
            D1b[k] = x12[o];
            D2a[k] = x21[o];
            D2b[k] = x22[o];
        }
    }
    // row carries P(r0 + lane, c0 - HALO - 1), one row per lane
    uint32_t rcv1 = 0, rcv2 = 0;
    if (lane < rows) {
        const size_t o = ((size_t)i * g.mw + j) * B + lane;
        rcv1 = a.s.rc1[o];
        rcv2 = a.s.rc2[o];
    }
    // row 0 of every table is zero
    if (i == 0) {
        TS z1[WK];
        TQ z2[WK];
#pragma unroll
        for (int k = 0; k < WK; ++k) {
            z1[k] = 0;
            z2[k] = 0;
        }
        uint32_t z0[WK];
#pragma unroll
        for (int k = 0; k < WK; ++k)
            z0[k] = 0;
        if (wL) {
            store8(a.L1lo, a.L1hi, cs + 1 + kColOffset, z1);
            store8(a.L2lo, a.L2hi, cs + 1 + kColOffset, z2);
#pragma unroll
            for (int f = 0; f < NF; ++f)
                store8(a.F.up[f], a.F.up[f], cs + 1 + kColOffset, z0);
        }
        if (wT) {
            store8(a.T1lo, a.T1hi, cs + 1 + kColOffset, z1);
            store8(a.T2lo, a.T2hi, cs + 1 + kColOffset, z2);
#pragma unroll
            for (int f = 0; f < NF; ++f)
                store8(a.F.cone[f], a.F.cone[f], cs + 1 + kColOffset, z0);
        }
        if (wEdge) {
            store1(a.L1lo, a.L1hi, kColOffset, (TS)0);
            store1(a.L2lo, a.L2hi, kColOffset, (TQ)0);
            store1(a.T1lo, a.T1hi, kColOffset, (TS)0);
            store1(a.T2lo, a.T2hi, kColOffset, (TQ)0);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                a.F.up[f][kColOffset] = 0;
                a.F.cone[f][kColOffset] = 0;
            }
        }
    }
    // pixel rows are prefetched two rows ahead
    uint2 nxt0 = load8(a.img, a.pitch, g.H, g.W, a.aligned8, r0, cs);
    uint2 nxt1 = load8(a.img, a.pitch, g.H, g.W, a.aligned8, r0 + 1, cs);
    // core columns of the current row, one 192-word row per plane, two rows in flight
    __shared__ __align__(128) uint32_t obuf[2][NPL][WCW];
    const int ob = cs - c0;                              // this lane's first word in an obuf row
    // columns of the L and T rows this tile stores, rounded up to 16-byte multiples
    const uint32_t bytesL = (uint32_t)((max(0, min(WCW, cLmax - c0 + 1)) + 3) / 4 * 16);
    const uint32_t bytesT = (uint32_t)((min(WCW, cTmax - c0 + 1) + 3) / 4 * 16);

#pragma unroll 1
    for (int rr = 0; rr < rows; ++rr) {
        const int y = r0 + rr;
        const int par = rr & 1;
        const uint2 q = nxt0;
        nxt0 = nxt1;
        if (rr + 2 < rows)
            nxt1 = load8(a.img, a.pitch, g.H, g.W, a.aligned8, y + 2, cs);
        uint32_t p1[WK], p2[WK];
#pragma unroll
        for (int k = 0; k < WK; ++k) {
            const uint32_t v = ((k < 4 ? q.x : q.y) >> (8 * (k & 3))) & 0xffu;
            p1[k] = (k ? p1[k - 1] : 0u) + v;
            p2[k] = (k ? p2[k - 1] : 0u) + v * v;
        }
        // warp inclusive scan of the lane totals
        uint32_t s1 = p1[WK - 1], s2 = p2[WK - 1];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u1 = __shfl_up_sync(0xffffffffu, s1, o);
            const uint32_t u2 = __shfl_up_sync(0xffffffffu, s2, o);
            if (lane >= o) {
                s1 += u1;
                s2 += u2;
            }
        }
        // e = P(y, cs - 1)
        const uint32_t e1 = __shfl_sync(0xffffffffu, rcv1, rr) + s1 - p1[WK - 1];
        const uint32_t e2 = __shfl_sync(0xffffffffu, rcv2, rr) + s2 - p2[WK - 1];
        // neighbours before the update
        TS n1a = __shfl_down_sync(0xffffffffu, D1a[0], 1);
        TQ n1b = __shfl_down_sync(0xffffffffu, D1b[0], 1);
        TS n2a = __shfl_up_sync(0xffffffffu, D2a[WK - 1], 1);
        TQ n2b = __shfl_up_sync(0xffffffffu, D2b[WK - 1], 1);
        if (lane == 31) {
            n1a = D1a[WK - 1];
            n1b = D1b[WK - 1];
        }
        if (lane == 0) {
            n2a = 0;
            n2b = 0;
        }
        uint32_t P1[WK], P2[WK];
#pragma unroll
        for (int k = 0; k < WK; ++k) {
            P1[k] = e1 + p1[k];
            P2[k] = e2 + p2[k];
        }
        // D2 moves one column right: D2(y, c) = P(y, c-1) + D2(y-1, c-1)
#pragma unroll
        for (int k = WK - 1; k >= 1; --k) {
            D2a[k] = (TS)P1[k - 1] + D2a[k - 1];
            D2b[k] = (TQ)P2[k - 1] + D2b[k - 1];
        }
        D2a[0] = (TS)e1 + n2a;
        D2b[0] = (TQ)e2 + n2b;
        // D1 moves one column left: D1(y, c) = P(y, c) + D1(y-1, c+1)
#pragma unroll
        for (int k = 0; k < WK - 1; ++k) {
            D1a[k] = (TS)P1[k] + D1a[k + 1];
            D1b[k] = (TQ)P2[k] + D1b[k + 1];
        }
        D1a[WK - 1] = (TS)P1[WK - 1] + n1a;
        D1b[WK - 1] = (TQ)P2[WK - 1] + n1b;
        TS T1v[WK];
        TQ T2v[WK];
#pragma unroll
        for (int k = 0; k < WK; ++k) {
            L1a[k] += (TS)P1[k];
            L2a[k] += (TQ)P2[k];
            T1v[k] = D1a[k] - D2a[k];
            T2v[k] = D1b[k] - D2b[k];
        }
        const int64_t rowL = (int64_t)(y + 1) * a.pL + kColOffset;
        const int64_t rowT = (int64_t)(y + 1) * a.pT + kColOffset;
        // the buffer of row rr - 2 is free once its copies have read it
        if (rr >= 2 && lane == 0)
            asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        __syncwarp();
        if (wL) {
            put8(obuf[par][PL1], obuf[par][PL1 + HS], ob, L1a);
            put8(obuf[par][PL2], obuf[par][PL2 + HQ], ob, L2a);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                uint32_t pk[WK];
                pack8(L1a, L2a, a.F.kS[f], a.F.kQ[f], pk);
                put8(obuf[par][PFU + f], obuf[par][PFU + f], ob, pk);
            }
        }
        if (wT) {
            put8(obuf[par][PT1], obuf[par][PT1 + HS], ob, T1v);
            put8(obuf[par][PT2], obuf[par][PT2 + HQ], ob, T2v);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                uint32_t pk[WK];
                pack8(T1v, T2v, a.F.kS[f], a.F.kQ[f], pk);
                put8(obuf[par][PFC + f], obuf[par][PFC + f], ob, pk);
            }
        }
        if (wEdge) {   // b = 0: L is zero, T is cone(y, -1) = D1(y, -1)
            store1(a.L1lo, a.L1hi, rowL, (TS)0);
            store1(a.L2lo, a.L2hi, rowL, (TQ)0);
            store1(a.T1lo, a.T1hi, rowT, T1v[WK - 1]);
            store1(a.T2lo, a.T2hi, rowT, T2v[WK - 1]);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                a.F.up[f][rowL] = 0;
                a.F.cone[f][rowT] = pack_window((uint32_t)T1v[WK - 1], (uint32_t)T2v[WK - 1], a.F.kS[f], a.F.kQ[f]);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {   // row (y + 1), columns b = c0 + 1 .. : 16-byte aligned in every plane
            uint32_t *dst[NPL];
            int k = 0;
            dst[k++] = a.L1lo + rowL + c0 + 1;
            if (HS) dst[k++] = a.L1hi + rowL + c0 + 1;
            dst[k++] = a.L2lo + rowL + c0 + 1;
            if (HQ) dst[k++] = a.L2hi + rowL + c0 + 1;
#pragma unroll
            for (int f = 0; f < NF; ++f)
                dst[k++] = a.F.up[f] + rowL + c0 + 1;
            dst[k++] = a.T1lo + rowT + c0 + 1;
            if (HS) dst[k++] = a.T1hi + rowT + c0 + 1;
            dst[k++] = a.T2lo + rowT + c0 + 1;
            if (HQ) dst[k++] = a.T2hi + rowT + c0 + 1;
#pragma unroll
            for (int f = 0; f < NF; ++f)
                dst[k++] = a.F.cone[f] + rowT + c0 + 1;
#pragma unroll
            for (int pl = 0; pl < NPL; ++pl) {
                const uint32_t nb = pl < PT1 ? bytesL : bytesT;
                if (nb)
                    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst[pl]),
                                 "r"((uint32_t)__cvta_generic_to_shared(&obuf[par][pl][0])), "r"(nb)
                                 : "memory");
            }
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
    }
    // the copies read shared memory until they complete
    if (lane == 0)
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    __syncwarp();
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename TS, typename TQ>
cudaError_t launch_all(const Geometry &g, const Scratch &s, const uint8_t *img, int64_t pitch,
                       int aligned8, const TableDesc &L1, const TableDesc &L2,
                       const TableDesc &T1, const TableDesc &T2, const FilterPlanes &F, cudaStream_t st) {
    cudaError_t e;
    ReduceArgs ra{img, pitch, g, s, aligned8};
    if ((e = launch_pdl(k_tab_reduce, dim3(g.m, g.n), dim3(NT), st, ra)) != cudaSuccess)
        return e;
    CarryArgs ca{g, s, (g.XW + 31) / 32, (g.DN + 31) / 32};
    const int chunks = ca.chunksCS + ca.chunksAD + (g.FN + 31) / 32;
    if ((e = launch_pdl(k_tab_carry, dim3(chunks), dim3(32, CG), st, ca)) != cudaSuccess)
        return e;
    PrefixArgs pa{g, s};
    if ((e = launch_pdl(k_tab_prefix<TS, TQ>, dim3(g.n, 7), dim3(PT), st, pa)) != cudaSuccess)
        return e;
    WriteArgs wa{img, pitch, g, s, L1.lo, L1.hi, L2.lo, L2.hi, T1.lo, T1.hi, T2.lo, T2.hi,
                 L1.pitch, T1.pitch, aligned8, F};
    if (F.n == 1)
        return launch_pdl(k_tab_write<TS, TQ, 1>, dim3(g.mw, g.n), dim3(32), st, wa);
    if (F.n == 2)
        return launch_pdl(k_tab_write<TS, TQ, 2>, dim3(g.mw, g.n), dim3(32), st, wa);
    return launch_pdl(k_tab_write<TS, TQ, 0>, dim3(g.mw, g.n), dim3(32), st, wa);
}

}  // namespace

size_t TableScratch::bytes(int H, int W, int sum_bits, int sq_bits) {
    Geometry g(H, W);
    Scratch s;
    return carve(g, sum_bits, sq_bits, &s, nullptr);
}

cudaError_t launch_build_tables(const uint8_t *img, int H, int W, int64_t pitch,
                                const TableDesc &L1, const TableDesc &L2, const TableDesc &T1,
                                const TableDesc &T2, const FilterPlanes &F, void *scratch, cudaStream_t st,
                                uint64_t *launches) {
    if (F.n < 0 || F.n > kMaxFilterWindows)
        return cudaErrorInvalidValue;
    Geometry g(H, W);
    Scratch s;
    carve(g, L1.bits, L2.bits, &s, (char *)scratch);
    const int aligned8 = ((uintptr_t)img % 8 == 0) && (pitch % 8 == 0);   // also 4-byte aligned
    cudaError_t e;
    const bool s64 = L1.bits == 64, q64 = L2.bits == 64;
    if (!s64 && !q64)
        e = launch_all<uint32_t, uint32_t>(g, s, img, pitch, aligned8, L1, L2, T1, T2, F, st);
    else if (!s64 && q64)
        e = launch_all<uint32_t, uint64_t>(g, s, img, pitch, aligned8, L1, L2, T1, T2, F, st);
    else if (s64 && !q64)
        e = launch_all<uint64_t, uint32_t>(g, s, img, pitch, aligned8, L1, L2, T1, T2, F, st);
    else
        e = launch_all<uint64_t, uint64_t>(g, s, img, pitch, aligned8, L1, L2, T1, T2, F, st);
    if (launches)
        *launches += 4;
    return e;
}

}  // namespace scr
