/*
 * CPU oracle for the screening path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * arm may load this library.  The CUDA library never links or calls it, and it
 * shares no code, header or table with the CUDA sources.
 *
 * Plain, slow, obviously-correct restatement of the paper's screening steps,
 * in exact unsigned 64-bit arithmetic (no wrap-around: every value stays far
 * below 2^64 for images up to 65535 x 65535):
 *
 *   upright summed-area table   Sec. 3, Eq. (T_1): L(a,b) = sum_{y<a, x<b} I(y,x)
 *   table of squares            Sec. 3, second-moment table of I^2
 *   rotated ("cone") table      Sec. 4, the triangular summed-area map L_dmd,
 *                               read with the inner condition j <= y-|x-i| as its
 *                               definition (the printed outer limits are garbled);
 *                               built here by the Lienhart-Kuranov recurrence the
 *                               paper cites for the 45-degree table
 *   square / diamond sums       Sec. 3, Eq. (S_1); Sec. 4, diamond 4-corner form
 *   octagonal star              Sec. 4, star = square superposed on a diamond of
 *                               the same size (sums pooled, areas added)
 *   variance                    Sec. 3, Eq. (S_sigma), as A*Q - S^2
 *   central-area contrast       Sec. 5, central areas of a patch: inner star of
 *                               radius floor(R/2) against the remaining ring
 *   screening loop              Sec. 5, Algorithm 1: a candidate survives when
 *                               its features lie inside the template's bounds
 *
 * Table layouts (dense, row-major):
 *   L1, L2 : (H+1) x (W+1),  L[a][b] = sum over y < a, x < b
 *   T1, T2 : (H+1) x (W+2),  T[a][b] = cone(a-1, b-1),
 *            cone(r,c) = sum of I(y,x) over y <= r, |x-c| <= r-y, inside the image
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PX(img, pitch, y, x) ((uint64_t)(img)[(int64_t)(y) * (pitch) + (x)])

/* Square half-side n for star radius R: the unique integer with
 * (2n-1)^2 < 2R^2 < (2n+1)^2 (the square and the diamond of half-diagonal R
 * have the "same size", Sec. 4).  Found by plain counting. */
int orc_square_half(int R)
{
    int64_t two_r2 = 2 * (int64_t)R * R;
    int n = 0;
    while ((int64_t)(2 * n + 1) * (2 * n + 1) < two_r2)
        n++;
    return n;
}

/* Upright tables by the textbook recurrence
 * L(a,b) = I(a-1,b-1) + L(a-1,b) + L(a,b-1) - L(a-1,b-1). */
void orc_upright(const uint8_t *img, int H, int W, int64_t pitch,
                 uint64_t *L1, uint64_t *L2)
{
    const int64_t P = (int64_t)W + 1;
    for (int64_t b = 0; b <= W; b++) {
        L1[b] = 0;
        L2[b] = 0;
    }
    for (int64_t a = 1; a <= H; a++) {
        L1[a * P] = 0;
        L2[a * P] = 0;
        for (int64_t b = 1; b <= W; b++) {
            uint64_t v = PX(img, pitch, a - 1, b - 1);
            L1[a * P + b] = v + L1[(a - 1) * P + b] + L1[a * P + b - 1] - L1[(a - 1) * P + b - 1];
            L2[a * P + b] = v * v + L2[(a - 1) * P + b] + L2[a * P + b - 1] - L2[(a - 1) * P + b - 1];
        }
    }
}

/* Cone tables by the recurrence
 *   cone(r,c) = cone(r-1,c-1) + cone(r-1,c+1) - cone(r-2,c) + I(r,c) + I(r-1,c)
 * (the two upper cones overlap in the cone two rows up; the apex pixel and the
 * pixel just above it are the only ones neither upper cone holds).
 * The recurrence reaches one column further out on each row, so it runs on a
 * working row that extends E = H + 2 columns past both image edges; the
 * truncation error at the ends of that row moves inward one column per row
 * and never reaches the stored columns -1..W. */
void orc_cone(const uint8_t *img, int H, int W, int64_t pitch,
              uint64_t *T1, uint64_t *T2)
{
    const int64_t E = (int64_t)H + 2;
    const int64_t WX = (int64_t)W + 2 * E;       /* working columns c in [-E, W-1+E] */
    const int64_t P = (int64_t)W + 2;
    uint64_t *rows = (uint64_t *)calloc((size_t)(6 * WX), sizeof(uint64_t));
    uint64_t *a1 = rows, *b1 = rows + WX, *c1 = rows + 2 * WX;   /* r-2, r-1, r  (sum) */
    uint64_t *a2 = rows + 3 * WX, *b2 = rows + 4 * WX, *c2 = rows + 5 * WX;   /* (sum of squares) */
    for (int64_t b = 0; b < P; b++) {
        T1[b] = 0;
        T2[b] = 0;
    }
    for (int64_t r = 0; r < H; r++) {
        for (int64_t k = 0; k < WX; k++) {
            int64_t c = k - E;
            uint64_t left1 = k > 0 ? b1[k - 1] : 0, right1 = k + 1 < WX ? b1[k + 1] : 0;
            uint64_t left2 = k > 0 ? b2[k - 1] : 0, right2 = k + 1 < WX ? b2[k + 1] : 0;
            uint64_t p0 = 0, p1 = 0;
            if (c >= 0 && c < W) {
                p0 = PX(img, pitch, r, c);
                if (r >= 1)
                    p1 = PX(img, pitch, r - 1, c);
            }
            c1[k] = left1 + right1 - a1[k] + p0 + p1;
            c2[k] = left2 + right2 - a2[k] + p0 * p0 + p1 * p1;
        }
        for (int64_t b = 0; b < P; b++) {      /* stored columns c = b-1 in [-1, W] */
            T1[(r + 1) * P + b] = c1[b - 1 + E];
            T2[(r + 1) * P + b] = c2[b - 1 + E];
        }
        uint64_t *t;
        t = a1; a1 = b1; b1 = c1; c1 = t;
        t = a2; a2 = b2; b2 = c2; c2 = t;
    }
    free(rows);
}

/* Window sums of one star (radius R) at candidate (y, x) from the oracle's
 * own tables.  Square: rows y-n+1..y+n, columns x-n+1..x+n (Eq. S_1).
 * Diamond: pixels |x'-x| < h, y-h+|x'-x| < y' <= y+h-|x'-x|, from four cone
 * corners (Sec. 4).  Caller guarantees the star lies inside the image. */
static void star_sums(const uint64_t *L1, const uint64_t *L2, const uint64_t *T1,
                      const uint64_t *T2, int W, int y, int x, int n, int h, int want_sq,
                      uint64_t *S, uint64_t *Q)
{
    const int64_t PL = (int64_t)W + 1, PT = (int64_t)W + 2;
#define LA(t, a, b) (t)[(int64_t)(a) * PL + (b)]
#define TA(t, a, b) (t)[(int64_t)(a) * PT + (b)]
    uint64_t s_sq = LA(L1, y + n + 1, x + n + 1) - LA(L1, y - n + 1, x + n + 1)
                  - LA(L1, y + n + 1, x - n + 1) + LA(L1, y - n + 1, x - n + 1);
    uint64_t s_dm = TA(T1, y + h + 1, x + 1) - TA(T1, y + 1, x - h + 1)
                  - TA(T1, y + 1, x + h + 1) + TA(T1, y - h + 1, x + 1);
    *S = s_sq + s_dm;
    if (want_sq) {
        uint64_t q_sq = LA(L2, y + n + 1, x + n + 1) - LA(L2, y - n + 1, x + n + 1)
                      - LA(L2, y + n + 1, x - n + 1) + LA(L2, y - n + 1, x - n + 1);
        uint64_t q_dm = TA(T2, y + h + 1, x + 1) - TA(T2, y + 1, x - h + 1)
                      - TA(T2, y + 1, x + h + 1) + TA(T2, y - h + 1, x + 1);
        *Q = q_sq + q_dm;
    }
#undef LA
#undef TA
}

/* Every pixel of the star of radius R (square half-side n, diamond
 * half-diagonal h = R) at (y, x) lies inside the H x W image. */
static int star_inside(int H, int W, int y, int x, int n, int h)
{
    if (y - n + 1 < 0 || y + n > H - 1 || x - n + 1 < 0 || x + n > W - 1)
        return 0;
    if (y - h + 1 < 0 || y + h > H - 1 || x - h + 1 < 0 || x + h - 1 > W - 1)
        return 0;
    return 1;
}

/* Features of the candidates (ys[i], xs[i]) at star radius R >= 2.
 * out[i*6 + 0..5] = S, Q, S_in, V = A*Q - S^2, N = S_in*A_ring - S_ring*A_in,
 * valid (1/0).  Invalid positions get zeros. */
void orc_features_at(const uint64_t *L1, const uint64_t *L2, const uint64_t *T1,
                     const uint64_t *T2, int H, int W, int R, int64_t count,
                     const int32_t *ys, const int32_t *xs, int64_t *out)
{
    int n = orc_square_half(R), h = R;
    int ri = R / 2;
    int ni = orc_square_half(ri), hi = ri;
    int64_t A = 4 * (int64_t)n * n + 2 * (int64_t)h * h;
    int64_t Ain = 4 * (int64_t)ni * ni + 2 * (int64_t)hi * hi;
    int64_t Aring = A - Ain;
    for (int64_t i = 0; i < count; i++) {
        int64_t *o = out + 6 * i;
        memset(o, 0, 6 * sizeof(int64_t));
        if (!star_inside(H, W, ys[i], xs[i], n, h))
            continue;
        uint64_t S, Q, Si, dummy;
        star_sums(L1, L2, T1, T2, W, ys[i], xs[i], n, h, 1, &S, &Q);
        if (ri >= 1)
            star_sums(L1, L2, T1, T2, W, ys[i], xs[i], ni, hi, 0, &Si, &dummy);
        else
            Si = 0;
        o[0] = (int64_t)S;
        o[1] = (int64_t)Q;
        o[2] = (int64_t)Si;
        o[3] = (int64_t)((uint64_t)A * Q - S * S);
        o[4] = (int64_t)Si * Aring - ((int64_t)S - (int64_t)Si) * Ain;
        o[5] = 1;
    }
}

/* Screening (Algorithm 1's hot loop over every patch of every scale).
 * radii[s]: star radius of scale s.  bounds[s*6 + 0..5]: inclusive integer
 * bounds S_lo, S_hi, V_lo, V_hi, N_lo, N_hi.  features: 1 mean, 2 variance,
 * 4 contrast.  mask: S x H x ceil(W/32) words, bit b of word w of row y is
 * x = 32w + b.  list: ascending keys (s<<48)|(y<<24)|x, at most cap of them.
 * Returns the number of surviving candidates. */
int64_t orc_screen(const uint64_t *L1, const uint64_t *L2, const uint64_t *T1,
                   const uint64_t *T2, int H, int W, int nscales, const int32_t *radii,
                   const int64_t *bounds, unsigned features, uint32_t *mask,
                   uint64_t *list, int64_t cap)
{
    const int64_t Wwords = ((int64_t)W + 31) / 32;
    memset(mask, 0, (size_t)(nscales * (int64_t)H * Wwords) * sizeof(uint32_t));
    for (int s = 0; s < nscales; s++) {
        const int R = radii[s];
        const int n = orc_square_half(R), h = R;
        const int ri = R / 2;
        const int ni = orc_square_half(ri), hi = ri;
        const int64_t A = 4 * (int64_t)n * n + 2 * (int64_t)h * h;
        const int64_t Ain = 4 * (int64_t)ni * ni + 2 * (int64_t)hi * hi;
        const int64_t Aring = A - Ain;
        const int64_t *bd = bounds + 6 * s;
        #pragma omp parallel for schedule(dynamic, 4)
        for (int y = 0; y < H; y++) {
            uint32_t *row = mask + ((int64_t)s * H + y) * Wwords;
            for (int x = 0; x < W; x++) {
                if (!star_inside(H, W, y, x, n, h))
                    continue;
                uint64_t S, Q = 0, Si = 0, dummy;
                star_sums(L1, L2, T1, T2, W, y, x, n, h, (features & 2) != 0, &S, &Q);
                int ok = 1;
                if (features & 1)
                    ok = ok && (int64_t)S >= bd[0] && (int64_t)S <= bd[1];
                if (ok && (features & 2)) {
                    int64_t V = (int64_t)((uint64_t)A * Q - S * S);
                    ok = V >= bd[2] && V <= bd[3];
                }
                if (ok && (features & 4)) {
                    star_sums(L1, L2, T1, T2, W, y, x, ni, hi, 0, &Si, &dummy);
                    int64_t N = (int64_t)Si * Aring - ((int64_t)S - (int64_t)Si) * Ain;
                    ok = N >= bd[4] && N <= bd[5];
                }
                if (ok)
                    row[x >> 5] |= 1u << (x & 31);
            }
        }
    }
    int64_t count = 0;
    for (int s = 0; s < nscales; s++)
        for (int64_t y = 0; y < H; y++)
            for (int64_t x = 0; x < W; x++) {
                uint32_t wd = mask[((int64_t)s * H + y) * Wwords + (x >> 5)];
                if ((wd >> (x & 31)) & 1u) {
                    if (count < cap)
                        list[count] = ((uint64_t)s << 48) | ((uint64_t)y << 24) | (uint64_t)x;
                    count++;
                }
            }
    return count;
}


/* Threads the screening loop uses (OpenMP over rows); n <= 0 leaves it as is.
 * Returns the count in effect. */
int orc_threads(int n) {
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
