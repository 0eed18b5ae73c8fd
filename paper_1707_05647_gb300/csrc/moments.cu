// Moment tables for the Prewitt gradient (Sec. 3, Eq. T_x and its vertical
// counterpart): Mx(a, b) = sum_{y<a, x<b} x I(y, x) and My(a, b) =
// sum_{y<a, x<b} y I(y, x), 64-bit (exact modulo 2^64), laid out like the
// upright tables (element (a, b) at a * pitch + b + kColOffset).
//
// The decomposition of the summed-area tables without their diagonals (so
// without halos).  The image is cut into 32-row bands; a band needs Mx and My
// on the row above it, and each 256-column writer tile the prefix of x I and
// of I left of it on every row.  Those carries are linear in the pixels and are
// assembled from band sums with no inter-CTA waiting:
//   k_mom_reduce  per (band, 1024-column tile): the column sums of I and of
//                 (y - r0) I over the band, and per (row, 256-column chunk) the
//                 sums of I and of (x - x0) I (x0 the chunk's first column).
//   k_mom_carry   per column: the exclusive prefix over bands of the column
//                 sums of I and of y I (the sums above each band).
//   k_mom_prefix  per band: the prefix along the row of x * (sum of I above)
//                 and of (sum of y I above) -> Mx(r0, .), My(r0, .); per band
//                 and row, the chunk prefixes -> the writer tiles' row carries.
//   k_mom_write   one warp per (band, tile): each lane owns 8 adjacent
//                 columns, keeps Mx and My for them in registers and walks the
//                 band's rows (warp scans of I and (x - x0) I plus the row
//                 carries give the row prefixes), writing each row of both
//                 tables through shared memory with bulk copies.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace scr {
namespace {

constexpr int MB = 32;           // rows per band
constexpr int MRT = 1024;        // columns per reduce tile
constexpr int MWT = 256;         // columns per writer tile (8 per lane)
constexpr int MWK = MWT / 32;
constexpr int MCH = MRT / MWT;   // writer chunks per reduce tile
constexpr int MNT = 256;         // threads of k_mom_reduce / k_mom_prefix
constexpr int MCG = 8;           // band groups per k_mom_carry block
constexpr int MCQ = 16;          // bands per group kept in registers
static_assert(MB == 32, "row carries are held one per lane");

struct MomGeom {
    int H = 0, W = 0, n = 0, mr = 0, mw = 0;   // bands, reduce tiles, writer tiles
    MomGeom() = default;
    MomGeom(int H_, int W_) : H(H_), W(W_) {
        n = (H + MB - 1) / MB;
        mr = (W + MRT - 1) / MRT;
        mw = (W + MWT - 1) / MWT;
    }
};

struct MomScratch {
    uint32_t *cs, *cy;           // [n][W]      band column sums of I and of (y - r0) I
    uint32_t *rs, *rk;           // [n][mw][B]  row chunk sums of I and of (x - x0) I
    uint32_t *csa;               // [n][W]      sum of I above the band, per column
    uint64_t *ysa;               // [n][W]      sum of y I above the band, per column
    uint64_t *mxc, *myc;         // [n][W]      Mx(r0, c+1), My(r0, c+1)
    uint64_t *rcx;               // [n][mw][B]  sum of x I left of the tile on the row
    uint32_t *rci;               // [n][mw][B]  sum of I left of the tile on the row
};

size_t mom_align(size_t v) { return (v + 255) & ~size_t(255); }

size_t mom_carve(const MomGeom &g, MomScratch *s, char *base) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += mom_align(bytes);
        return p;
    };
    const size_t n = g.n, W = g.W, R = (size_t)g.n * g.mw * MB;
    s->cs = (uint32_t *)take(n * W * 4);
    s->cy = (uint32_t *)take(n * W * 4);
    s->rs = (uint32_t *)take(R * 4);
    s->rk = (uint32_t *)take(R * 4);
    s->csa = (uint32_t *)take(n * W * 4);
    s->ysa = (uint64_t *)take(n * W * 8);
    s->mxc = (uint64_t *)take(n * W * 8);
    s->myc = (uint64_t *)take(n * W * 8);
    s->rcx = (uint64_t *)take(R * 8);
    s->rci = (uint32_t *)take(R * 4);
    return off;
}

struct MomArgs {
    const uint8_t *img;
    int64_t ipitch;
    int aligned8;
    MomGeom g;
    MomScratch s;
    int64_t pitch;               // elements (u64) per table row
    uint64_t *Mx, *My;
};

__device__ __forceinline__ uint2 mload8(const MomArgs &a, int y, int x) {
    const MomGeom &g = a.g;
    if (y < g.H && a.aligned8 && x >= 0 && x + 8 <= g.W)
        return __ldg(reinterpret_cast<const uint2 *>(a.img + (int64_t)y * a.ipitch + x));
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int xx = x + k;
        const uint32_t b = (y < g.H && xx >= 0 && xx < g.W) ? (uint32_t)__ldg(a.img + (int64_t)y * a.ipitch + xx) : 0u;
        if (k < 4)
            lo |= b << (8 * k);
        else
            hi |= b << (8 * (k - 4));
    }
    return make_uint2(lo, hi);
}

// rows r..r+3 (one word each, byte k = column k) -> c[k] = column k's four rows
__device__ __forceinline__ void mtranspose4(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3, uint32_t (&c)[4]) {
    const uint32_t t0 = __byte_perm(r0, r1, 0x5140), t1 = __byte_perm(r0, r1, 0x7362);
    const uint32_t t2 = __byte_perm(r2, r3, 0x5140), t3 = __byte_perm(r2, r3, 0x7362);
    c[0] = __byte_perm(t0, t2, 0x5410);
    c[1] = __byte_perm(t0, t2, 0x7632);
    c[2] = __byte_perm(t1, t3, 0x5410);
    c[3] = __byte_perm(t1, t3, 0x7632);
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(MNT) k_mom_reduce(const MomArgs a) {
    pdl_begin();
    __shared__ __align__(16) uint8_t tile[MB][MRT];
    const MomGeom &g = a.g;
    const int j = blockIdx.x, i = blockIdx.y, t = threadIdx.x;
    const int r0 = i * MB, c0 = j * MRT, c1 = min(c0 + MRT, g.W);
    {
        constexpr int RPT = MB / (MNT / 128);   // rows per thread
        const int x = c0 + 8 * (t & 127), rb = (t >> 7) * RPT;
        uint2 w[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k)
            w[k] = mload8(a, r0 + rb + k, x);
#pragma unroll
        for (int k = 0; k < RPT; ++k)
            *reinterpret_cast<uint2 *>(&tile[rb + k][8 * (t & 127)]) = w[k];
    }
    __syncthreads();
    const uint32_t *t32 = reinterpret_cast<const uint32_t *>(&tile[0][0]);
    // column sums of I and of (y - r0) I, four columns per step
    for (int x0 = c0 + 4 * t; x0 < c1; x0 += 4 * MNT) {
        uint32_t s1[4] = {0, 0, 0, 0}, sy[4] = {0, 0, 0, 0};
#pragma unroll
        for (int r = 0; r < MB; r += 4) {
            const uint32_t *row = t32 + (x0 - c0) / 4;
            uint32_t c[4];
            mtranspose4(row[r * (MRT / 4)], row[(r + 1) * (MRT / 4)], row[(r + 2) * (MRT / 4)],
                        row[(r + 3) * (MRT / 4)], c);
            const uint32_t wy = (uint32_t)r | (uint32_t)(r + 1) << 8 | (uint32_t)(r + 2) << 16 | (uint32_t)(r + 3) << 24;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                s1[k] = __dp4a(c[k], 0x01010101u, s1[k]);
                sy[k] = __dp4a(c[k], wy, sy[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (x0 + k < c1) {
                a.s.cs[(size_t)i * g.W + x0 + k] = s1[k];
                a.s.cy[(size_t)i * g.W + x0 + k] = sy[k];
            }
    }
    // per (row, 256-column chunk): sums of I and of (x - x0) I; 8 threads per item
    {
        constexpr int TPI = 8, WPI = MWT / 4 / TPI;    // 8 words per thread
        const int sub = t % TPI;
#pragma unroll 1
        for (int u = t / TPI; u < MB * MCH; u += MNT / TPI) {
            const int rr = u / MCH, q = u % MCH;
            const uint32_t *row = t32 + rr * (MRT / 4) + q * (MWT / 4) + sub * WPI;
            uint32_t s1 = 0, sk = 0;
#pragma unroll
            for (int w = 0; w < WPI; ++w) {
                const uint32_t k0 = 4 * (sub * WPI + w);    // column of byte 0 within the chunk (< 256)
                const uint32_t wk = k0 | (k0 + 1) << 8 | (k0 + 2) << 16 | (k0 + 3) << 24;
                s1 = __dp4a(row[w], 0x01010101u, s1);
                sk = __dp4a(row[w], wk, sk);
            }
#pragma unroll
            for (int o = 1; o < TPI; o <<= 1) {
                s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                sk += __shfl_xor_sync(0xffffffffu, sk, o);
            }
            const int jw = j * MCH + q;
            if (sub == 0 && jw < g.mw) {
                const size_t o = ((size_t)i * g.mw + jw) * MB + rr;
                a.s.rs[o] = s1;
                a.s.rk[o] = sk;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// per column x (a lane): exclusive prefix over bands; block = 32 columns x
// MCG band groups
__global__ void __launch_bounds__(32 * MCG) k_mom_carry(const MomArgs a) {
    pdl_begin();
    __shared__ uint32_t sum1[MCG][33];
    __shared__ uint64_t sumy[MCG][33];
    const MomGeom &g = a.g;
    const int lane = threadIdx.x, grp = threadIdx.y;
    const int x = blockIdx.x * 32 + lane;
    const bool live = x < g.W;
    const int q = (g.n + MCG - 1) / MCG;
    const int b0 = grp * q, b1 = min(g.n, b0 + q);
    uint32_t c1[MCQ], cyv[MCQ];
    uint32_t t1 = 0;
    uint64_t ty = 0;
#pragma unroll
    for (int k = 0; k < MCQ; ++k) {
        c1[k] = cyv[k] = 0;
        if (live && b0 + k < b1) {
            c1[k] = a.s.cs[(size_t)(b0 + k) * g.W + x];
            cyv[k] = a.s.cy[(size_t)(b0 + k) * g.W + x];
        }
        t1 += c1[k];
        ty += (uint64_t)(b0 + k) * MB * c1[k] + cyv[k];
    }
    if (live)
        for (int b = b0 + MCQ; b < b1; ++b) {
            const uint32_t v = a.s.cs[(size_t)b * g.W + x];
            t1 += v;
            ty += (uint64_t)b * MB * v + a.s.cy[(size_t)b * g.W + x];
        }
    sum1[grp][lane] = t1;
    sumy[grp][lane] = ty;
    __syncthreads();
    if (grp == 0) {
        uint32_t r1 = 0;
        uint64_t ry = 0;
        for (int k = 0; k < MCG; ++k) {
            const uint32_t u1 = sum1[k][lane];
            const uint64_t uy = sumy[k][lane];
            sum1[k][lane] = r1;
            sumy[k][lane] = ry;
            r1 += u1;
            ry += uy;
        }
    }
    __syncthreads();
    if (!live)
        return;
    uint32_t run1 = sum1[grp][lane];
    uint64_t runy = sumy[grp][lane];
#pragma unroll
    for (int k = 0; k < MCQ; ++k) {
        if (b0 + k >= b1)
            break;
        a.s.csa[(size_t)(b0 + k) * g.W + x] = run1;
        a.s.ysa[(size_t)(b0 + k) * g.W + x] = runy;
        run1 += c1[k];
        runy += (uint64_t)(b0 + k) * MB * c1[k] + cyv[k];
    }
    for (int b = b0 + MCQ; b < b1; ++b) {
        a.s.csa[(size_t)b * g.W + x] = run1;
        a.s.ysa[(size_t)b * g.W + x] = runy;
        const uint32_t v = a.s.cs[(size_t)b * g.W + x];
        run1 += v;
        runy += (uint64_t)b * MB * v + a.s.cy[(size_t)b * g.W + x];
    }
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t mwarp_incl_scan(uint64_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v += u;
    }
    return v;
}

// blockIdx.y: 0 = Mx carries (prefix of x * csa), 1 = My carries (prefix of
// ysa), 2 = the writer tiles' row carries; blockIdx.x = band
__global__ void __launch_bounds__(MNT, 4) k_mom_prefix(const MomArgs a) {
    pdl_begin();
    __shared__ uint64_t wsum[MNT / 32];
    __shared__ uint64_t totx[MNT / 32][MB];
    __shared__ uint32_t toti[MNT / 32][MB];
    const MomGeom &g = a.g;
    const int i = blockIdx.x, q = blockIdx.y, t = threadIdx.x, lane = t & 31, w = t >> 5;
    constexpr int NW = MNT / 32;
    if (q == 2) {   // lane = row of the band; warp w takes a contiguous run of chunks
        const int seg = (g.mw + NW - 1) / NW;
        const int j0 = w * seg, j1 = min(g.mw, j0 + seg);
        uint64_t sx = 0;
        uint32_t si = 0;
        for (int j = j0; j < j1; ++j) {
            const size_t o = ((size_t)i * g.mw + j) * MB + lane;
            const uint32_t v = a.s.rs[o];
            si += v;
            sx += (uint64_t)j * MWT * v + a.s.rk[o];
        }
        totx[w][lane] = sx;
        toti[w][lane] = si;
        __syncthreads();
        uint64_t cx = 0;
        uint32_t ci = 0;
        for (int u = 0; u < w; ++u) {
            cx += totx[u][lane];
            ci += toti[u][lane];
        }
        for (int j = j0; j < j1; ++j) {
            const size_t o = ((size_t)i * g.mw + j) * MB + lane;
            const uint32_t v = a.s.rs[o];
            a.s.rcx[o] = cx;
            a.s.rci[o] = ci;
            ci += v;
            cx += (uint64_t)j * MWT * v + a.s.rk[o];
        }
        return;
    }
    // inclusive prefix along the row of f(x) = x * csa[x] (q = 0) or ysa[x] (q = 1);
    // each warp a contiguous segment, 32 entries per step
    const size_t rb = (size_t)i * g.W;
    const int seg = ((g.W + NW - 1) / NW + 31) / 32 * 32;
    const int k0 = w * seg, k1 = min(g.W, k0 + seg);
    auto f = [&](int x) -> uint64_t {
        return q == 0 ? (uint64_t)x * a.s.csa[rb + x] : a.s.ysa[rb + x];
    };
    uint64_t part = 0;
    for (int x = k0 + lane; x < k1; x += 32)
        part += f(x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0)
        wsum[w] = part;
    __syncthreads();
    uint64_t carry = 0;
    for (int u = 0; u < w; ++u)
        carry += wsum[u];
    uint64_t *out = (q == 0 ? a.s.mxc : a.s.myc) + rb;
    for (int xb = k0; xb < k1; xb += 32) {
        const int x = xb + lane;
        const uint64_t v = x < k1 ? f(x) : 0;
        const uint64_t incl = mwarp_incl_scan(v, lane);
        if (x < k1)
            out[x] = carry + incl;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32) k_mom_write(const MomArgs a) {
    pdl_begin();
    __shared__ __align__(128) uint64_t obuf[2][2][MWT];   // [row parity][Mx, My][column]
    const MomGeom &g = a.g;
    const int j = blockIdx.x, i = blockIdx.y, lane = threadIdx.x;
    const int r0 = i * MB, rows = min(MB, g.H - r0);
    const int c0 = j * MWT;
    const int cs = c0 + MWK * lane;                 // this lane's first column c (table column c + 1)
    const int ncol = min(MWT, g.W - c0);            // columns of this tile inside the image
    const uint32_t nbytes = (uint32_t)((ncol + 1) / 2 * 16);   // 16-byte multiple
    const bool wcol = cs < g.W;
    // carries from the row above the band
    uint64_t Mx[MWK], My[MWK];
#pragma unroll
    for (int k = 0; k < MWK; ++k) {
        const int c = min(cs + k, g.W - 1);
        Mx[k] = a.s.mxc[(size_t)i * g.W + c];
        My[k] = a.s.myc[(size_t)i * g.W + c];
    }
    // row carries of this tile: row r0 + lane
    uint64_t rcx = 0;
    uint32_t rci = 0;
    if (lane < rows) {
        const size_t o = ((size_t)i * g.mw + j) * MB + lane;
        rcx = a.s.rcx[o];
        rci = a.s.rci[o];
    }
    // row 0 and column 0 of both tables are zero: band 0 writes row 0 (its tile 0
    // also the corner), tile 0 of every band column 0 of the band's rows
    if (i == 0 && wcol)
#pragma unroll
        for (int k = 0; k < MWK; ++k)
            if (cs + k < g.W) {
                a.Mx[cs + k + 1 + kColOffset] = 0;
                a.My[cs + k + 1 + kColOffset] = 0;
            }
    if (j == 0) {
        if (lane < rows) {
            const int64_t e = (int64_t)(r0 + 1 + lane) * a.pitch + kColOffset;
            a.Mx[e] = 0;
            a.My[e] = 0;
        }
        if (i == 0 && lane == 0) {
            a.Mx[kColOffset] = 0;
            a.My[kColOffset] = 0;
        }
    }
    uint2 nxt0 = mload8(a, r0, cs), nxt1 = mload8(a, r0 + 1, cs);
#pragma unroll 1
    for (int rr = 0; rr < rows; ++rr) {
        const int y = r0 + rr, par = rr & 1;
        const uint2 px = nxt0;
        nxt0 = nxt1;
        if (rr + 2 < rows)
            nxt1 = mload8(a, y + 2, cs);
        uint32_t pi[MWK], pk[MWK];
#pragma unroll
        for (int k = 0; k < MWK; ++k) {
            const uint32_t v = ((k < 4 ? px.x : px.y) >> (8 * (k & 3))) & 0xffu;
            pi[k] = (k ? pi[k - 1] : 0u) + v;
            pk[k] = (k ? pk[k - 1] : 0u) + (uint32_t)(MWK * lane + k) * v;
        }
        uint32_t si = pi[MWK - 1], sk = pk[MWK - 1];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t ui = __shfl_up_sync(0xffffffffu, si, o);
            const uint32_t uk = __shfl_up_sync(0xffffffffu, sk, o);
            if (lane >= o) {
                si += ui;
                sk += uk;
            }
        }
        // prefixes before this lane's first column, within the tile and the row
        const uint32_t ei = si - pi[MWK - 1], ek = sk - pk[MWK - 1];
        const uint64_t rowx = __shfl_sync(0xffffffffu, rcx, rr);
        const uint32_t rowi = __shfl_sync(0xffffffffu, rci, rr);
#pragma unroll
        for (int k = 0; k < MWK; ++k) {
            const uint32_t ti = ei + pi[k];                    // sum of I over [c0, c]
            const uint64_t Px = rowx + (uint64_t)c0 * ti + (ek + pk[k]);   // sum_{x <= c} x I
            const uint64_t Pi = (uint64_t)rowi + ti;                        // sum_{x <= c} I
            Mx[k] += Px;
            My[k] += (uint64_t)y * Pi;
        }
        // the buffer of row rr - 2 is free once its copies have read it
        if (rr >= 2 && lane == 0)
            asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        __syncwarp();
        {
            uint4 *bx = reinterpret_cast<uint4 *>(&obuf[par][0][MWK * lane]);
            uint4 *by = reinterpret_cast<uint4 *>(&obuf[par][1][MWK * lane]);
#pragma unroll
            for (int k = 0; k < MWK / 2; ++k) {
                bx[k] = make_uint4((uint32_t)Mx[2 * k], (uint32_t)(Mx[2 * k] >> 32), (uint32_t)Mx[2 * k + 1],
                                   (uint32_t)(Mx[2 * k + 1] >> 32));
                by[k] = make_uint4((uint32_t)My[2 * k], (uint32_t)(My[2 * k] >> 32), (uint32_t)My[2 * k + 1],
                                   (uint32_t)(My[2 * k + 1] >> 32));
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {   // row y + 1, columns b = c0 + 1 ..: a 16-byte aligned run in both tables
            const int64_t e = (int64_t)(y + 1) * a.pitch + kColOffset + c0 + 1;
            asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(a.Mx + e),
                         "r"((uint32_t)__cvta_generic_to_shared(&obuf[par][0][0])), "r"(nbytes)
                         : "memory");
            asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(a.My + e),
                         "r"((uint32_t)__cvta_generic_to_shared(&obuf[par][1][0])), "r"(nbytes)
                         : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
    }
    // the copies read shared memory until they complete
    if (lane == 0)
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    __syncwarp();
}

}  // namespace

size_t moment_scratch_bytes(int H, int W) {
    MomGeom g(H, W);
    MomScratch s;
    return mom_carve(g, &s, nullptr) + 256;
}

cudaError_t launch_moment_tables(const uint8_t *img, int64_t ipitch, int H, int W, int64_t pitch, uint64_t *Mx,
                                 uint64_t *My, void *scratch, cudaStream_t st, uint64_t *launches) {
    MomArgs a;
    a.img = img;
    a.ipitch = ipitch;
    a.aligned8 = ((uintptr_t)img % 8 == 0) && (ipitch % 8 == 0);
    a.g = MomGeom(H, W);
    mom_carve(a.g, &a.s, (char *)scratch);
    a.pitch = pitch;
    a.Mx = Mx;
    a.My = My;
    cudaError_t e;
    if (launches)
        *launches += 4;
    if ((e = launch_pdl(k_mom_reduce, dim3(a.g.mr, a.g.n), dim3(MNT), st, a)) != cudaSuccess)
        return e;
    if ((e = launch_pdl(k_mom_carry, dim3((W + 31) / 32), dim3(32, MCG), st, a)) != cudaSuccess)
        return e;
    if ((e = launch_pdl(k_mom_prefix, dim3(a.g.n, 3), dim3(MNT), st, a)) != cudaSuccess)
        return e;
    return launch_pdl(k_mom_write, dim3(a.g.mw, a.g.n), dim3(32), st, a);
}

}  // namespace scr
