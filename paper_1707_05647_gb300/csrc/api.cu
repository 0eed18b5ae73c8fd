// Host side of the C ABI declared in include/screen.h: contexts, the device
// memory pool with its HBM budget, table and template handles, the exact
// bound computation, and the entry points that enqueue the kernels.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <vector>

#include <array>
#include <cmath>

#include "runtime.h"

using namespace scr;
using namespace scr_rt;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

int scr_rt::fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

const std::string &scr_rt::last_error() { return g_last_error; }

namespace scr_rt {

int dev_alloc(scr_ctx *c, size_t bytes, cudaStream_t st, void **p) {
    bytes = std::max<size_t>(bytes, 256);
    const uint64_t now = c->in_use.fetch_add(bytes) + bytes;
    if (c->budget && now > c->budget) {
        c->in_use.fetch_sub(bytes);
        return fail(SCR_EBUDGET, "allocation of %zu bytes exceeds the HBM budget (%llu in use, budget %llu)",
                    bytes, (unsigned long long)(now - bytes), (unsigned long long)c->budget);
    }
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, c->pool, st);
    if (e != cudaSuccess) {
        c->in_use.fetch_sub(bytes);
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? SCR_ENOMEM : SCR_ECUDA,
                    "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    uint64_t pk = c->peak.load();
    while (now > pk && !c->peak.compare_exchange_weak(pk, now)) {
    }
    return SCR_OK;
}

void dev_free(scr_ctx *c, void *p, size_t bytes, cudaStream_t st) {
    if (!p)
        return;
    bytes = std::max<size_t>(bytes, 256);
    cudaFreeAsync(p, st);
    c->in_use.fetch_sub(bytes);
}

int check_ctx(const scr_ctx *c) {
    if (!c)
        return fail(SCR_EINVAL, "null context");
    return SCR_OK;
}

// (2n-1)^2 < 2R^2 < (2n+1)^2 via the integer square root of 2R^2.
int64_t isqrt64(int64_t v) {
    int64_t m = (int64_t)__builtin_sqrt((double)v);
    while (m * m > v) --m;
    while ((m + 1) * (m + 1) <= v) ++m;
    return m;
}

Geo geometry(int R) {
    Geo g;
    g.n = square_half(R);
    g.h = R;
    g.hi = R / 2;
    g.ni = square_half(g.hi);
    g.A = 4 * (int64_t)g.n * g.n + 2 * (int64_t)g.h * g.h;
    g.Ain = 4 * (int64_t)g.ni * g.ni + 2 * (int64_t)g.hi * g.hi;
    g.Aring = g.A - g.Ain;
    return g;
}

i128 floor_div(i128 a, i128 b) {   // b > 0
    i128 q = a / b;
    if ((a % b != 0) && (a < 0))
        --q;
    return q;
}

i128 ceil_div(i128 a, i128 b) {    // b > 0
    i128 q = a / b;
    if ((a % b != 0) && (a > 0))
        ++q;
    return q;
}

int64_t clamp64(i128 v) {
    const i128 lo = (i128)INT64_MIN, hi = (i128)INT64_MAX;
    return (int64_t)(v < lo ? lo : (v > hi ? hi : v));
}

int check_rat(const scr_rat &r, bool below_one, const char *name) {
    const int64_t lim = (int64_t)1 << 20;
    if (r.den <= 0 || r.den > lim || r.num < 0 || r.num > lim)
        return fail(SCR_EINVAL, "%s = %lld/%lld: need 0 <= num <= 2^20, 0 < den <= 2^20", name,
                    (long long)r.num, (long long)r.den);
    if (below_one && r.num >= r.den)
        return fail(SCR_EINVAL, "%s must be below 1", name);
    return SCR_OK;
}

int validate_params(const scr_params *p) {
    if (!p)
        return fail(SCR_EINVAL, "null params");
    if (p->n_scales < 1 || p->n_scales > kMaxScales || !p->radii)
        return fail(SCR_EINVAL, "n_scales must be in [1, %d] with a radii array", kMaxScales);
    if (p->features & ~15u)
        return fail(SCR_EINVAL, "unknown feature bits 0x%x", p->features);
    for (int s = 0; s < p->n_scales; ++s) {
        const int R = p->radii[s];
        if (R < 2 || R > 181)
            return fail(SCR_EINVAL, "radius %d at scale %d outside [2, 181] (window sums of I^2 must stay below 2^32)", R, s);
    }
    int rc;
    if ((rc = check_rat(p->mean_rel, true, "mean_rel")) || (rc = check_rat(p->std_rel, true, "std_rel")) ||
        (rc = check_rat(p->grad_rel, true, "grad_rel")) || (rc = check_rat(p->grad_abs, false, "grad_abs")))
        return rc;
    if ((p->features & SCR_F_PREWITT) &&
        ((rc = check_rat(p->prewitt_rel, true, "prewitt_rel")) || (rc = check_rat(p->prewitt_abs, false, "prewitt_abs"))))
        return rc;
    return SCR_OK;
}

// Per-scale bounds from the template hulls (exact; see include/screen.h).
void bounds_for(const scr_tmpl *tm, const scr_params *p, int R, scr_bounds *b) {
    const Geo g = geometry(R);
    b->S_lo = INT64_MIN;
    b->S_hi = INT64_MAX;
    b->V_lo = INT64_MIN;
    b->V_hi = INT64_MAX;
    b->N_lo = INT64_MIN;
    b->N_hi = INT64_MAX;
    if (p->features & SCR_F_MEAN) {
        const i128 a = p->mean_rel.num, d = p->mean_rel.den;
        b->S_lo = clamp64(ceil_div((d - a) * tm->mu_lo_n * g.A, d * tm->mu_lo_d));
        b->S_hi = clamp64(floor_div((d + a) * tm->mu_hi_n * g.A, d * tm->mu_hi_d));
    }
    if (p->features & SCR_F_VAR) {
        const i128 a = p->std_rel.num, d = p->std_rel.den;
        const i128 A2 = (i128)g.A * g.A;
        b->V_lo = clamp64(ceil_div((d - a) * (d - a) * tm->v_lo_n * A2, d * d * tm->v_lo_d));
        b->V_hi = clamp64(floor_div((d + a) * (d + a) * tm->v_hi_n * A2, d * d * tm->v_hi_d));
    }
    if (p->features & SCR_F_GRAD) {
        const i128 a = p->grad_rel.num, bb = p->grad_rel.den;
        const i128 e = p->grad_abs.num, f = p->grad_abs.den;
        const i128 D = (i128)g.Ain * g.Aring;
        {
            const i128 Nn = tm->g_lo_n, Nd = tm->g_lo_d;
            const i128 absN = Nn < 0 ? -Nn : Nn;
            const i128 num = Nn * bb * f - a * absN * f - e * bb * Nd;
            b->N_lo = clamp64(ceil_div(num * D, bb * f * Nd));
        }
        {
            const i128 Nn = tm->g_hi_n, Nd = tm->g_hi_d;
            const i128 absN = Nn < 0 ? -Nn : Nn;
            const i128 num = Nn * bb * f + a * absN * f + e * bb * Nd;
            b->N_hi = clamp64(floor_div(num * D, bb * f * Nd));
        }
    }
}

// words of one u32 plane of a table: (H + 1) rows at the padded pitch, 256-byte multiple
int64_t table_plane_words(int H, int W) {
    const int64_t rows = (int64_t)H + 1;
    return ((rows * table_pitch_words(W) + 63) / 64) * 64;
}

size_t tables_bytes(int H, int W, int sum_bits, int sq_bits, int n_filter) {
    return (size_t)table_plane_words(H, W) * 4 *
           (size_t)(2 * (sum_bits / 32) + 2 * (sq_bits / 32) + 2 * n_filter);
}

void layout_tables(scr_tables *t, void *base, size_t bytes, int H, int W, int sum_bits, int sq_bits,
                   cudaStream_t st, int n_filter, const int (*fk)[2]) {
    const int64_t pitch = table_pitch_words(W);
    const int64_t rows = (int64_t)H + 1;
    const int64_t plane = table_plane_words(H, W);
    const int bits[4] = {sum_bits, sq_bits, sum_bits, sq_bits};
    const int64_t cols[4] = {(int64_t)W + 1, (int64_t)W + 1, (int64_t)W + 2, (int64_t)W + 2};
    t->base = base;
    t->bytes = bytes;
    uint32_t *p = (uint32_t *)base;
    for (int k = 0; k < 4; ++k) {
        TableDesc &d = t->t[k];
        d.lo = p;
        p += plane;
        d.hi = nullptr;
        if (bits[k] == 64) {
            d.hi = p;
            p += plane;
        }
        d.pitch = pitch;
        d.rows = rows;
        d.cols = cols[k];
        d.bits = bits[k];
    }
    t->F = FilterPlanes();
    t->F.n = n_filter;
    for (int f = 0; f < n_filter; ++f) {
        t->F.up[f] = p;
        p += plane;
        t->F.cone[f] = p;
        p += plane;
        t->F.kS[f] = fk[f][0];
        t->F.kQ[f] = fk[f][1];
    }
    t->H = H;
    t->W = W;
    t->stream = st;
}

int alloc_tables(scr_ctx *c, int H, int W, int sum_bits, int sq_bits, cudaStream_t st, scr_tables **out,
                 int n_filter, const int (*fk)[2]) {
    auto *t = new (std::nothrow) scr_tables();
    if (!t)
        return fail(SCR_ENOMEM, "host allocation failed");
    const size_t bytes = tables_bytes(H, W, sum_bits, sq_bits, n_filter);
    void *base = nullptr;
    int rc = dev_alloc(c, bytes, st, &base);
    if (rc) {
        delete t;
        return rc;
    }
    layout_tables(t, base, bytes, H, W, sum_bits, sq_bits, st, n_filter, fk);
    *out = t;
    return SCR_OK;
}

int run_build_in(scr_ctx *c, const uint8_t *img, int H, int W, int64_t pitch, scr_tables *t, void *scratch,
                 cudaStream_t st) {
    uint64_t n = 0;
    cudaError_t e = launch_build_tables(img, H, W, pitch, t->t[0], t->t[1], t->t[2], t->t[3], t->F, scratch, st, &n);
    c->launches += n;
    CUDA_TRY(e);
    return SCR_OK;
}

int run_build(scr_ctx *c, const uint8_t *img, int H, int W, int64_t pitch, scr_tables *t, cudaStream_t st) {
    Scoped scratch(c, st);
    int rc = scratch.take(TableScratch::bytes(H, W, t->t[0].bits, t->t[1].bits));
    if (rc)
        return rc;
    return run_build_in(c, img, H, W, pitch, t, scratch.p, st);
}

void free_tables(scr_ctx *c, scr_tables *t) {
    dev_free(c, t->base, t->bytes, t->stream);
    if (t->mom)
        dev_free(c, t->mom, t->mom_bytes, t->stream);
    delete t;
}

// ---- exact wide integers for the Prewitt bounds ----------------------------
// Non-negative integers as base-2^32 limbs (little end first): enough for the
// products of the Prewitt bound rationals, which outgrow 128 bits.
struct Big {
    std::vector<uint32_t> d;
    Big() {}
    explicit Big(unsigned __int128 v) {
        while (v) {
            d.push_back((uint32_t)v);
            v >>= 32;
        }
    }
};

int big_cmp(const Big &a, const Big &b) {
    if (a.d.size() != b.d.size())
        return a.d.size() < b.d.size() ? -1 : 1;
    for (size_t i = a.d.size(); i-- > 0;)
        if (a.d[i] != b.d[i])
            return a.d[i] < b.d[i] ? -1 : 1;
    return 0;
}

void big_trim(Big &a) {
    while (!a.d.empty() && a.d.back() == 0)
        a.d.pop_back();
}

Big big_mul(const Big &a, const Big &b) {
    Big r;
    if (a.d.empty() || b.d.empty())
        return r;
    r.d.assign(a.d.size() + b.d.size(), 0);
    for (size_t i = 0; i < a.d.size(); ++i) {
        uint64_t carry = 0;
        for (size_t j = 0; j < b.d.size(); ++j) {
            const uint64_t cur = (uint64_t)a.d[i] * b.d[j] + r.d[i + j] + carry;
            r.d[i + j] = (uint32_t)cur;
            carry = cur >> 32;
        }
        size_t k = i + b.d.size();
        while (carry) {
            const uint64_t cur = (uint64_t)r.d[k] + carry;
            r.d[k++] = (uint32_t)cur;
            carry = cur >> 32;
        }
    }
    big_trim(r);
    return r;
}

Big big_add(const Big &a, const Big &b) {
    Big r;
    uint64_t carry = 0;
    for (size_t i = 0; i < std::max(a.d.size(), b.d.size()) || carry; ++i) {
        const uint64_t cur = carry + (i < a.d.size() ? a.d[i] : 0) + (i < b.d.size() ? b.d[i] : 0);
        r.d.push_back((uint32_t)cur);
        carry = cur >> 32;
    }
    big_trim(r);
    return r;
}

Big big_sub(const Big &a, const Big &b) {   // a >= b
    Big r = a;
    int64_t borrow = 0;
    for (size_t i = 0; i < r.d.size(); ++i) {
        int64_t cur = (int64_t)r.d[i] - borrow - (i < b.d.size() ? (int64_t)b.d[i] : 0);
        borrow = cur < 0;
        if (cur < 0)
            cur += (int64_t)1 << 32;
        r.d[i] = (uint32_t)cur;
    }
    big_trim(r);
    return r;
}

size_t big_bits(const Big &a) {
    if (a.d.empty())
        return 0;
    return 32 * (a.d.size() - 1) + (32 - __builtin_clz(a.d.back()));
}

bool big_bit(const Big &a, size_t i) { return (a.d[i / 32] >> (i % 32)) & 1u; }

// floor(a / b) (b > 0) by shift and subtract; also whether the division was exact
Big big_div(const Big &a, const Big &b, bool *exact) {
    Big q, r;
    const size_t n = big_bits(a);
    q.d.assign((n + 31) / 32 + 1, 0);
    for (size_t i = n; i-- > 0;) {
        r = big_add(r, r);
        if (big_bit(a, i))
            r = big_add(r, Big(1));
        if (big_cmp(r, b) >= 0) {
            r = big_sub(r, b);
            q.d[i / 32] |= 1u << (i % 32);
        }
    }
    big_trim(q);
    if (exact)
        *exact = r.d.empty();
    return q;
}

unsigned __int128 big_u128_sat(const Big &a) {
    if (a.d.size() > 4)
        return ~(unsigned __int128)0;
    unsigned __int128 v = 0;
    for (size_t i = a.d.size(); i-- > 0;)
        v = (v << 32) | a.d[i];
    return v;
}

// doubled Prewitt normaliser of a 2n x 2n square: sum (2x' - 2x - 1)^2 = (2n)^2 (4n^2 - 1) / 3
uint64_t prewitt_j2(int64_t n) { return (uint64_t)((2 * n) * (2 * n) * (4 * n * n - 1) / 3); }

// Inclusive bounds on Gx2^2 + Gy2^2 at star radius R (scr_params: phi^2 in
// [max(0, (1-tp)^2 p_lo - dp^2), (1+tp)^2 p_hi + dp^2], phi^2 = 4 n^2 G2 / J2^2),
// exact: L = ceil(lo J2^2 / (4 n^2)), U = floor(hi J2^2 / (4 n^2)), U saturated.
void prewitt_bounds(const scr_tmpl *tm, const scr_params *p, int R, unsigned __int128 *L, unsigned __int128 *U) {
    const int64_t n = geometry(R).n;
    const Big J2(prewitt_j2(n)), J2sq = big_mul(J2, J2);
    const uint64_t tn = (uint64_t)p->prewitt_rel.num, td = (uint64_t)p->prewitt_rel.den;
    const uint64_t dn = (uint64_t)p->prewitt_abs.num, dd = (uint64_t)p->prewitt_abs.den;
    // lo = ((td - tn)^2 A_lo dd^2 - dn^2 td^2 B_lo) / (td^2 B_lo dd^2); hi likewise with +
    auto part = [&](unsigned __int128 A, unsigned __int128 B, uint64_t tf, bool minus, Big *num, Big *den, bool *neg) {
        const Big a = big_mul(big_mul(Big(A), Big((unsigned __int128)tf * tf)), Big((unsigned __int128)dd * dd));
        const Big b = big_mul(Big((unsigned __int128)dn * dn * td * td), Big(B));
        *neg = false;
        if (minus) {
            if (big_cmp(a, b) <= 0) {
                *neg = true;
                *num = Big();
            } else {
                *num = big_sub(a, b);
            }
        } else {
            *num = big_add(a, b);
        }
        *den = big_mul(big_mul(Big((unsigned __int128)td * td), Big(B)), Big((unsigned __int128)dd * dd));
    };
    Big num, den;
    bool neg;
    part(tm->p_lo_n, tm->p_lo_d, td - tn, true, &num, &den, &neg);
    const Big fden = big_mul(den, Big((unsigned __int128)(4 * n * n)));
    if (neg) {
        *L = 0;
    } else {
        bool exact = false;
        Big q = big_div(big_mul(num, J2sq), fden, &exact);
        if (!exact)
            q = big_add(q, Big(1));
        *L = big_u128_sat(q);
    }
    part(tm->p_hi_n, tm->p_hi_d, td + tn, false, &num, &den, &neg);
    *U = big_u128_sat(big_div(big_mul(num, J2sq), big_mul(den, Big((unsigned __int128)(4 * n * n))), nullptr));
}

// ---- packed-plane pre-filter: which window a scale may use -------------------
//
// A packed plane holds, per table element, bits kS .. kS+15 of the sum table
// and bits kQ .. kQ+15 of the sum-of-squares table.  The signed sum of a
// star's eight packed corners gives u = sum of floor(corner / 2^kS) modulo 2^16,
// which lies strictly within 4 of S / 2^kS (four corners add and four
// subtract, each dropping less than one unit), and likewise for Q with a
// further carry of -4 .. 3 from the low half.  The window is usable at a
// scale when every candidate that can pass the exact tests has S and Q small
// enough that u does not wrap: S <= S_hi' <= 2^kS (2^16 - 8) and
// Q <= Q_hi' <= 2^kQ (2^16 - 16), where S_hi' is the mean test's upper bound
// (at most 255 A) and Q_hi' = floor((V_hi + S_hi'^2) / A) (at most 65025 A),
// since V = A Q - S^2 <= V_hi.  Candidates with larger S or Q fail the exact
// tests whatever the filter decides.
struct FilterRange {
    bool usable;              // the variance test is on (the pre-filter tests its lower bound)
    int64_t S_lo, S_hi;       // mean interval clipped to [0, 255 A]
    i128 Q_hi;                // largest Q of a candidate that can pass
    int64_t V_lo, V_hi;       // variance interval (full range when off)
};

static FilterRange filter_range(const scr_params *p, const scr_bounds &b, int64_t A) {
    FilterRange r;
    const bool fm = p->features & SCR_F_MEAN, fv = p->features & SCR_F_VAR;
    r.usable = fv;
    r.S_lo = fm ? std::max<int64_t>(b.S_lo, 0) : 0;
    r.S_hi = fm ? std::min<int64_t>(b.S_hi, 255 * A) : 255 * A;
    r.Q_hi = (i128)65025 * A;
    if (fv) {
        const i128 v = (i128)b.V_hi + (i128)r.S_hi * r.S_hi;
        r.Q_hi = std::min<i128>(r.Q_hi, v < 0 ? 0 : v / A);
    }
    r.V_lo = fv ? b.V_lo : INT64_MIN;
    r.V_hi = fv ? b.V_hi : INT64_MAX;
    return r;
}

static bool window_fits(const FilterRange &r, int kS, int kQ) {
    return r.usable && (i128)r.S_hi <= ((i128)1 << kS) * (65536 - 8) && r.Q_hi <= ((i128)1 << kQ) * (65536 - 16);
}

// A window more than this many bits coarser than the narrowest usable shifts
// rejects little (measured on the 8192 x 8192, 16-scale workload: 99% of
// candidates at up to 3 bits, 3-78% at 4), so such a scale reads exact corners.
constexpr int kFilterSlackBits = 3;

// smallest shifts (kS, kQ) at which a window is usable for this range; false if none
static bool min_window(const FilterRange &r, int *kS, int *kQ);

// window f of F usable for range r and at most kFilterSlackBits coarser than its narrowest shifts
static bool window_suits(const FilterRange &r, const FilterPlanes &F, int f) {
    int ks = 0, kq = 0;
    return window_fits(r, F.kS[f], F.kQ[f]) && min_window(r, &ks, &kq) && F.kS[f] <= ks + kFilterSlackBits &&
           F.kQ[f] <= kq + kFilterSlackBits;
}

static bool min_window(const FilterRange &r, int *kS, int *kQ) {
    if (!r.usable)
        return false;
    int a = 0, q = 0;
    while (a <= kMaxFilterShiftS && (i128)r.S_hi > ((i128)1 << a) * (65536 - 8))
        ++a;
    while (q <= kMaxFilterShiftQ && r.Q_hi > ((i128)1 << q) * (65536 - 16))
        ++q;
    if (a > kMaxFilterShiftS || q > kMaxFilterShiftQ)
        return false;
    *kS = a;
    *kQ = q;
    return true;
}

// float nearest to v on the side that widens an interval: down (dir < 0) or up
static float float_toward(double v, int dir) {
    float f = (float)v;
    if (dir < 0 && (double)f > v)
        f = nextafterf(f, -INFINITY);
    if (dir > 0 && (double)f < v)
        f = nextafterf(f, INFINITY);
    return f;
}

// Single-precision constants of the kernel's pre-filter (filter_pass in
// features.cu) for window (kS, kQ).  2^kS, A 2^kQ and their products with 2^23
// and 2^23 + 8 are exact floats (A < 2^17, kS <= 14, kQ <= 16).  The mean lower
// bound is rounded down; the variance lower bound moves down by
// M = 4 u (X + |V_lo|) + 1 with X = A 2^kQ 65535 the largest corner product and
// u = 2^-24, more than the kernel's roundings can move a computed A Q - S^2.
static void filter_constants(const FilterRange &r, uint32_t A, int kS, int kQ, ScaleParam *sp) {
    const double two23 = 8388608.0, u = 1.0 / 16777216.0;
    const double s2 = ldexp(1.0, kS), c = (double)A * ldexp(1.0, kQ);
    sp->f2S = (float)s2;
    sp->fS0 = (float)(-s2 * (two23 + 8));
    sp->fSlo = float_toward((double)r.S_lo, -1);
    sp->fc = (float)c;
    sp->fQ0 = (float)(-c * two23);
    if (r.V_lo == INT64_MIN) {
        sp->fVlo = -INFINITY;
    } else {
        const double v = (double)r.V_lo, X = c * 65535.0;
        sp->fVlo = float_toward(v - (4 * u * (X + fabs(v)) + 1), -1);
    }
}

int fill_screen_args(const scr_tables *t, const scr_tmpl *tm, const scr_params *p, ScreenArgs *a) {
    memset(a, 0, sizeof *a);
    a->L1 = t->t[0].lo;
    a->L2 = t->t[1].lo;
    a->T1 = t->t[2].lo;
    a->T2 = t->t[3].lo;
    const int64_t P = t->t[0].pitch;   // all four tables share the pitch
    a->pitch = P;
    a->H = t->H;
    a->W = t->W;
    a->Wwords = (t->W + 31) / 32;
    a->n_scales = p->n_scales;
    a->features = p->features;
    for (int s = 0; s < p->n_scales; ++s) {
        const int R = p->radii[s];
        const Geo g = geometry(R);
        ScaleParam &sp = a->sp[s];
        const int64_t n = g.n, h = g.h, ni = g.ni, hi = g.hi;
        const int64_t oL[4] = {(n + 1) * P + (n + 1), (1 - n) * P + (n + 1), (n + 1) * P + (1 - n), (1 - n) * P + (1 - n)};
        const int64_t oT[4] = {(h + 1) * P + 1, P + (1 - h), P + (h + 1), (1 - h) * P + 1};
        const int64_t oLi[4] = {(ni + 1) * P + (ni + 1), (1 - ni) * P + (ni + 1), (ni + 1) * P + (1 - ni),
                                (1 - ni) * P + (1 - ni)};
        const int64_t oTi[4] = {(hi + 1) * P + 1, P + (1 - hi), P + (hi + 1), (1 - hi) * P + 1};
        for (int k = 0; k < 4; ++k) {
            sp.oL[k] = (int32_t)oL[k];
            sp.oT[k] = (int32_t)oT[k];
            sp.oLi[k] = (int32_t)oLi[k];
            sp.oTi[k] = (int32_t)oTi[k];
        }
        sp.y_lo = std::max(g.n, g.h) - 1;
        sp.y_hi = t->H - 1 - std::max(g.n, g.h);
        sp.x_lo = std::max(g.n, g.h) - 1;
        sp.x_hi = std::min(t->W - 1 - g.n, t->W - g.h);
        sp.A = (uint32_t)g.A;
        sp.Ain = (uint32_t)g.Ain;
        sp.Aring = (uint32_t)g.Aring;
        scr_bounds b;
        bounds_for(tm, p, R, &b);
        // no valid position at this scale (the star does not fit in the image)
        sp.empty = (sp.x_hi < sp.x_lo || sp.y_hi < sp.y_lo) ? 1u : 0u;
        sp.S_lo = 0;
        sp.S_rng = UINT32_MAX;
        if (p->features & SCR_F_MEAN) {
            const int64_t lo = std::max<int64_t>(b.S_lo, 0), hi2 = std::min<int64_t>(b.S_hi, UINT32_MAX);
            if (lo > hi2)
                sp.empty = 1;
            else {
                sp.S_lo = (uint32_t)lo;
                sp.S_rng = (uint32_t)(hi2 - lo);
            }
        }
        if (p->features & SCR_F_VAR) {
            if (b.V_lo > b.V_hi)
                sp.empty = 1;
            sp.V_lo = b.V_lo;
            sp.V_rng = (uint64_t)((i128)b.V_hi - (i128)b.V_lo);
        }
        if (p->features & SCR_F_GRAD) {
            if (b.N_lo > b.N_hi)
                sp.empty = 1;
            sp.N_lo = b.N_lo;
            sp.N_rng = (uint64_t)((i128)b.N_hi - (i128)b.N_lo);
        }
        sp.P_lo = 0;
        sp.P_rng = ~(unsigned __int128)0;
        if (p->features & SCR_F_PREWITT) {
            unsigned __int128 L, U;
            prewitt_bounds(tm, p, R, &L, &U);
            if (L > U)
                sp.empty = 1;
            else {
                sp.P_lo = L;
                sp.P_rng = U - L;
            }
        }
    }
    a->Mx = t->Mx;
    a->My = t->My;
    for (int f = 0; f < t->F.n; ++f) {
        a->FU[f] = t->F.up[f];
        a->FC[f] = t->F.cone[f];
    }
    // each scale takes the narrowest packed window whose range holds every
    // candidate that can pass (no window: the scale reads the exact corners only)
    for (int s = 0; s < p->n_scales; ++s) {
        ScaleParam &sp = a->sp[s];
        sp.fw = -1;
        if (!t->F.n || sp.empty || (p->features & SCR_F_PREWITT))   // the Prewitt variant reads exact corners only
            continue;
        scr_bounds b;
        bounds_for(tm, p, p->radii[s], &b);
        const FilterRange r = filter_range(p, b, sp.A);
        int best = -1;
        for (int f = 0; f < t->F.n; ++f)
            if (window_suits(r, t->F, f) &&
                (best < 0 || t->F.kS[f] < t->F.kS[best] ||
                 (t->F.kS[f] == t->F.kS[best] && t->F.kQ[f] < t->F.kQ[best])))
                best = f;
        if (best < 0)
            continue;
        sp.fw = best;
        filter_constants(r, sp.A, t->F.kS[best], t->F.kQ[best], &sp);
    }
    return SCR_OK;
}

int check_screen_inputs(const scr_tables *t, const scr_tmpl *tm, const scr_params *p) {
    if (!t || !tm)
        return fail(SCR_EINVAL, "null tables or template");
    int rc = validate_params(p);
    if (rc)
        return rc;
    if ((p->features & SCR_F_GRAD) && !(tm->features & SCR_F_GRAD))
        return fail(SCR_EINVAL, "template features were computed without SCR_F_GRAD");
    if ((p->features & SCR_F_PREWITT) && !(tm->features & SCR_F_PREWITT))
        return fail(SCR_EINVAL, "template features were computed without SCR_F_PREWITT");
    if ((p->features & SCR_F_PREWITT) && !t->Mx)
        return fail(SCR_EINVAL, "SCR_F_PREWITT needs the moment tables (build_moment_tables)");
    return SCR_OK;
}

}  // namespace scr_rt

int scr::square_half(int R) {
    const int64_t m = isqrt64(2 * (int64_t)R * R);
    return (int)((m + 1) / 2);
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *screen_last_error(void) { return g_last_error.c_str(); }

int screen_init(scr_ctx **ctx, int device, uint64_t hbm_budget_bytes) {
    if (!ctx)
        return fail(SCR_EINVAL, "null ctx out-pointer");
    *ctx = nullptr;
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev)
        return fail(SCR_EINVAL, "device %d out of range (%d devices)", device, ndev);
    cudaDeviceProp prop;
    CUDA_TRY(cudaGetDeviceProperties(&prop, device));
    if (prop.major * 10 + prop.minor != 103)
        return fail(SCR_ECUDA, "device %d is sm_%d%d; this library is built for sm_103a only", device,
                    prop.major, prop.minor);
    DeviceGuard dg(device);
    if (!dg.ok)
        return fail(SCR_ECUDA, "cudaSetDevice(%d) failed", device);
    auto *c = new (std::nothrow) scr_ctx();
    if (!c)
        return fail(SCR_ENOMEM, "host allocation failed");
    c->device = device;
    c->budget = hbm_budget_bytes;
    cudaMemPoolProps pp;
    memset(&pp, 0, sizeof pp);
    pp.allocType = cudaMemAllocationTypePinned;
    pp.handleTypes = cudaMemHandleTypeNone;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = device;
    cudaError_t e = cudaMemPoolCreate(&c->pool, &pp);
    if (e == cudaSuccess) {
        uint64_t thr = hbm_budget_bytes ? hbm_budget_bytes : UINT64_MAX;
        e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&c->pinned, 64);
    if (e == cudaSuccess && cudaHostGetDevicePointer((void **)&c->pinned_dev, c->pinned, 0) != cudaSuccess) {
        c->pinned_dev = nullptr;   // screen_host then reads the count back with a copy
        cudaGetLastError();
    }
    if (e != cudaSuccess) {
        if (c->pool)
            cudaMemPoolDestroy(c->pool);
        delete c;
        return fail(SCR_ECUDA, "context setup failed: %s", cudaGetErrorString(e));
    }
    *ctx = c;
    return SCR_OK;
}

void screen_shutdown(scr_ctx *c) {
    if (!c)
        return;
    DeviceGuard dg(c->device);
    destroy_servers(c);
    destroy_frames(c);
    cudaDeviceSynchronize();
    {
        std::lock_guard<std::mutex> lk(c->mu);
        for (auto *t : c->tables) {
            cudaFreeAsync(t->base, nullptr);
            if (t->mom)
                cudaFreeAsync(t->mom, nullptr);
            delete t;
        }
        c->tables.clear();
        for (auto *tm : c->tmpls)
            delete tm;
        c->tmpls.clear();
        for (auto *b : c->batches)
            free_batch(c, b);
        c->batches.clear();
    }
    cudaDeviceSynchronize();
    if (c->pinned)
        cudaFreeHost(c->pinned);
    cudaMemPoolDestroy(c->pool);
    delete c;
}

int screen_stats(const scr_ctx *c, scr_stats *out) {
    if (check_ctx(c) || !out)
        return fail(SCR_EINVAL, "null argument");
    out->kernel_launches = c->launches.load();
    out->bytes_in_use = c->in_use.load();
    out->bytes_peak = c->peak.load();
    out->budget = c->budget;
    return SCR_OK;
}

int build_tables(scr_ctx *c, const uint8_t *img_dev, int32_t H, int32_t W, int64_t pitch, int32_t sum_bits,
                 int32_t sq_bits, scr_stream stream, scr_tables **out) {
    int rc;
    if ((rc = check_ctx(c)))
        return rc;
    if (!img_dev || !out)
        return fail(SCR_EINVAL, "null image or out-pointer");
    if (H < 1 || W < 1 || H > 65535 || W > 65535)
        return fail(SCR_EINVAL, "image %d x %d outside 1..65535", H, W);
    if (pitch < W)
        return fail(SCR_EINVAL, "pitch %lld < width %d", (long long)pitch, W);
    if ((sum_bits != 32 && sum_bits != 64) || (sq_bits != 32 && sq_bits != 64))
        return fail(SCR_EINVAL, "table widths must be 32 or 64 bits");
    *out = nullptr;
    DeviceGuard dg(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(c->mu);
    scr_tables *t = nullptr;
    if ((rc = alloc_tables(c, H, W, sum_bits, sq_bits, st, &t, c->n_filter, c->filter_k)))
        return rc;
    if ((rc = run_build(c, img_dev, H, W, pitch, t, st))) {
        free_tables(c, t);
        return rc;
    }
    c->tables.insert(t);
    *out = t;
    return SCR_OK;
}

int screen_set_filter(scr_ctx *c, int32_t n_windows, const int32_t *windows) {
    int rc;
    if ((rc = check_ctx(c)))
        return rc;
    if (n_windows < 0 || n_windows > kMaxFilterWindows || (n_windows && !windows))
        return fail(SCR_EINVAL, "n_windows %d outside 0..%d (or null windows)", n_windows, kMaxFilterWindows);
    for (int f = 0; f < n_windows; ++f)
        if (windows[2 * f] < 0 || windows[2 * f] > kMaxFilterShiftS || windows[2 * f + 1] < 0 ||
            windows[2 * f + 1] > kMaxFilterShiftQ)
            return fail(SCR_EINVAL, "window %d: shifts (%d, %d) outside 0..%d, 0..%d", f, windows[2 * f],
                        windows[2 * f + 1], kMaxFilterShiftS, kMaxFilterShiftQ);
    std::lock_guard<std::mutex> lk(c->mu);
    c->n_filter = n_windows;
    for (int f = 0; f < n_windows; ++f) {
        c->filter_k[f][0] = windows[2 * f];
        c->filter_k[f][1] = windows[2 * f + 1];
    }
    return SCR_OK;
}

int screen_filter_windows(const scr_tmpl *tm, const scr_params *p, int32_t max_windows, int32_t *windows,
                          int32_t *n_windows) {
    if (!tm || !windows || !n_windows || max_windows < 0)
        return fail(SCR_EINVAL, "null argument or negative max_windows");
    int rc;
    if ((rc = validate_params(p)))
        return rc;
    *n_windows = 0;
    // the narrowest usable shifts of every scale, and their largest values
    std::vector<std::pair<int, int>> need;
    int hs = -1, hq = -1;
    for (int s = 0; s < p->n_scales; ++s) {
        scr_bounds b;
        bounds_for(tm, p, p->radii[s], &b);
        const FilterRange r = filter_range(p, b, geometry(p->radii[s]).A);
        int kS, kQ;
        if (!min_window(r, &kS, &kQ))
            continue;
        need.push_back({kS, kQ});
        hs = std::max(hs, kS);
        hq = std::max(hq, kQ);
    }
    if (need.empty() || max_windows == 0)
        return SCR_OK;
    // the widest window fits every scale; a second one, the smallest that fits
    // every scale the first would serve more than kFilterSlackBits too coarse
    windows[0] = hs;
    windows[1] = hq;
    *n_windows = 1;
    if (max_windows >= 2) {
        int ns = -1, nq = -1;
        for (const auto &k : need)
            if (hs > k.first + kFilterSlackBits || hq > k.second + kFilterSlackBits) {
                ns = std::max(ns, k.first);
                nq = std::max(nq, k.second);
            }
        if (ns >= 0 && (ns < hs || nq < hq)) {
            windows[2] = windows[0];
            windows[3] = windows[1];
            windows[0] = ns;
            windows[1] = nq;
            *n_windows = 2;
        }
    }
    return SCR_OK;
}

int screen_filter_plan(const scr_tables *t, const scr_tmpl *tm, const scr_params *p, int32_t *window_per_scale) {
    if (!window_per_scale)
        return fail(SCR_EINVAL, "null output");
    int rc;
    if ((rc = check_screen_inputs(t, tm, p)))
        return rc;
    ScreenArgs a;
    if ((rc = fill_screen_args(t, tm, p, &a)))
        return rc;
    for (int s = 0; s < p->n_scales; ++s)
        window_per_scale[s] = a.sp[s].fw;
    return SCR_OK;
}

int tables_view(const scr_tables *t, int which, const void **dev_ptr, int64_t *rows, int64_t *cols, int64_t *pitch,
                int64_t *offset, int64_t *plane_stride, int32_t *bits) {
    if (t && which >= 6 && which < 6 + 2 * t->F.n) {   // packed filter planes
        const int f = (which - 6) / 2, cone = (which - 6) % 2;
        if (dev_ptr) *dev_ptr = cone ? t->F.cone[f] : t->F.up[f];
        if (rows) *rows = t->t[0].rows;
        if (cols) *cols = cone ? t->t[2].cols : t->t[0].cols;
        if (pitch) *pitch = t->t[0].pitch;
        if (offset) *offset = kColOffset;
        if (plane_stride) *plane_stride = 0;
        if (bits) *bits = 32;
        return SCR_OK;
    }
    if (!t || which < 0 || which > 3)
        return fail(SCR_EINVAL, "bad tables handle or index %d", which);
    const TableDesc &d = t->t[which];
    if (dev_ptr) *dev_ptr = d.lo;
    if (rows) *rows = d.rows;
    if (cols) *cols = d.cols;
    if (pitch) *pitch = d.pitch;
    if (offset) *offset = kColOffset;
    if (plane_stride) *plane_stride = d.hi ? (int64_t)(d.hi - d.lo) : 0;
    if (bits) *bits = d.bits;
    return SCR_OK;
}

int tables_copy_to_host(scr_ctx *c, const scr_tables *t, int which, uint64_t *dst) {
    int rc;
    if ((rc = check_ctx(c)))
        return rc;
    if (t && dst && which >= 6 && which < 6 + 2 * t->F.n) {   // packed filter planes, 32-bit values
        DeviceGuard dg(c->device);
        const int f = (which - 6) / 2, cone = (which - 6) % 2;
        const uint32_t *src = cone ? t->F.cone[f] : t->F.up[f];
        const int64_t rows = t->t[0].rows, cols = cone ? t->t[2].cols : t->t[0].cols, P = t->t[0].pitch;
        std::vector<uint32_t> v((size_t)rows * cols);
        CUDA_TRY(cudaStreamSynchronize(t->stream));
        CUDA_TRY(cudaMemcpy2D(v.data(), cols * 4, src + kColOffset, P * 4, cols * 4, rows, cudaMemcpyDeviceToHost));
        for (size_t k = 0; k < v.size(); ++k)
            dst[k] = v[k];
        return SCR_OK;
    }
    if (!t || which < 0 || which > 5 || !dst || (which >= 4 && !t->Mx))
        return fail(SCR_EINVAL, "bad arguments");
    DeviceGuard dg(c->device);
    if (which >= 4) {   // moment tables: (H + 1) x (W + 1) 64-bit values
        const uint64_t *src = which == 4 ? t->Mx : t->My;
        const int64_t P = t->t[0].pitch;
        CUDA_TRY(cudaStreamSynchronize(t->stream));
        CUDA_TRY(cudaMemcpy2D(dst, (size_t)(t->W + 1) * 8, src + kColOffset, (size_t)P * 8, (size_t)(t->W + 1) * 8,
                              t->H + 1, cudaMemcpyDeviceToHost));
        return SCR_OK;
    }
    const TableDesc &d = t->t[which];
    std::vector<uint32_t> lo((size_t)d.rows * d.cols), hi;
    CUDA_TRY(cudaStreamSynchronize(t->stream));
    CUDA_TRY(cudaMemcpy2D(lo.data(), d.cols * 4, d.lo + kColOffset, d.pitch * 4, d.cols * 4, d.rows,
                          cudaMemcpyDeviceToHost));
    if (d.hi) {
        hi.resize(lo.size());
        CUDA_TRY(cudaMemcpy2D(hi.data(), d.cols * 4, d.hi + kColOffset, d.pitch * 4, d.cols * 4, d.rows,
                              cudaMemcpyDeviceToHost));
    }
    for (size_t k = 0; k < lo.size(); ++k)
        dst[k] = (uint64_t)lo[k] | (d.hi ? ((uint64_t)hi[k] << 32) : 0);
    return SCR_OK;
}

void tables_release(scr_ctx *c, scr_tables *t) {
    if (!c || !t)
        return;
    DeviceGuard dg(c->device);
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->tables.erase(t))
        free_tables(c, t);
}

int template_features(scr_ctx *c, const uint8_t *tmpl_host, int32_t side, int32_t r, int32_t t_min,
                      uint32_t features, scr_tmpl **out) {
    int rc;
    if ((rc = check_ctx(c)))
        return rc;
    if (!tmpl_host || !out)
        return fail(SCR_EINVAL, "null template or out-pointer");
    if (r < 2 || r > 181 || side != 2 * r + 1)
        return fail(SCR_EINVAL, "template side %d must be 2r+1 with 2 <= r <= 181 (r = %d)", side, r);
    if (t_min < 1 || t_min > r || ((features & SCR_F_GRAD) && t_min < 2))
        return fail(SCR_EINVAL, "t_min %d outside [%d, r]", t_min, (features & SCR_F_GRAD) ? 2 : 1);
    if (features & ~15u)
        return fail(SCR_EINVAL, "unknown feature bits");
    *out = nullptr;
    DeviceGuard dg(c->device);
    std::lock_guard<std::mutex> lk(c->mu);
    cudaStream_t st = nullptr;
    const int cnt = r - t_min + 1;
    Scoped img(c, st), sums(c, st);
    if ((rc = img.take((size_t)side * side)) || (rc = sums.take((size_t)cnt * 3 * 8)))
        return rc;
    CUDA_TRY(cudaMemcpyAsync(img.p, tmpl_host, (size_t)side * side, cudaMemcpyHostToDevice, st));
    scr_tables *t = nullptr;
    if ((rc = alloc_tables(c, side, side, 64, 64, st, &t)))
        return rc;
    rc = run_build(c, (const uint8_t *)img.p, side, side, side, t, st);
    if (!rc) {
        uint64_t n = 0;
        cudaError_t e = launch_template_sums(t->t[0], t->t[1], t->t[2], t->t[3], r, t_min, (int64_t *)sums.p, st, &n);
        c->launches += n;
        if (e != cudaSuccess)
            rc = fail(SCR_ECUDA, "template kernel: %s", cudaGetErrorString(e));
    }
    std::vector<int64_t> host((size_t)cnt * 3);
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(host.data(), sums.p, host.size() * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(st);
        if (e != cudaSuccess)
            rc = fail(SCR_ECUDA, "template sums: %s", cudaGetErrorString(e));
    }
    free_tables(c, t);
    if (rc)
        return rc;
    auto *tm = new (std::nothrow) scr_tmpl();
    if (!tm)
        return fail(SCR_ENOMEM, "host allocation failed");
    tm->r = r;
    tm->t_min = t_min;
    tm->features = features;
    bool first = true;
    for (int k = 0; k < cnt; ++k) {
        const int tt = t_min + k;
        const int64_t S = host[3 * k], Q = host[3 * k + 1], Si = host[3 * k + 2];
        tm->S.push_back(S);
        tm->Q.push_back(Q);
        tm->Si.push_back(Si);
        const Geo g = geometry(tt);
        // mean S/A, variance V/A^2, contrast N/(Ain*Aring)
        const int64_t mu_n = S, mu_d = g.A;
        const int64_t v_n = g.A * Q - S * S, v_d = g.A * g.A;
        const int64_t g_n = Si * g.Aring - (S - Si) * g.Ain, g_d = g.Ain * g.Aring;
        if (first) {
            tm->mu_lo_n = tm->mu_hi_n = mu_n;
            tm->mu_lo_d = tm->mu_hi_d = mu_d;
            tm->v_lo_n = tm->v_hi_n = v_n;
            tm->v_lo_d = tm->v_hi_d = v_d;
            tm->g_lo_n = tm->g_hi_n = g_n;
            tm->g_lo_d = tm->g_hi_d = g_d > 0 ? g_d : 1;
            first = false;
            continue;
        }
        if ((i128)mu_n * tm->mu_lo_d < (i128)tm->mu_lo_n * mu_d) { tm->mu_lo_n = mu_n; tm->mu_lo_d = mu_d; }
        if ((i128)mu_n * tm->mu_hi_d > (i128)tm->mu_hi_n * mu_d) { tm->mu_hi_n = mu_n; tm->mu_hi_d = mu_d; }
        if ((i128)v_n * tm->v_lo_d < (i128)tm->v_lo_n * v_d) { tm->v_lo_n = v_n; tm->v_lo_d = v_d; }
        if ((i128)v_n * tm->v_hi_d > (i128)tm->v_hi_n * v_d) { tm->v_hi_n = v_n; tm->v_hi_d = v_d; }
        if (g_d > 0) {
            if ((i128)g_n * tm->g_lo_d < (i128)tm->g_lo_n * g_d) { tm->g_lo_n = g_n; tm->g_lo_d = g_d; }
            if ((i128)g_n * tm->g_hi_d > (i128)tm->g_hi_n * g_d) { tm->g_hi_n = g_n; tm->g_hi_d = g_d; }
        }
    }
    if (features & SCR_F_PREWITT) {
        // doubled moments of each central square about the template centre
        // (r + 1/2, r + 1/2): Gx2 = sum (2x - 2r - 1) I, Gy2 = sum (2y - 2r - 1) I;
        // and the hull of phi^2 = 4 n^2 (Gx2^2 + Gy2^2) / J2^2 (Sec. 3-4)
        bool firstp = true;
        for (int tt = t_min; tt <= r; ++tt) {
            const int64_t n = geometry(tt).n;
            int64_t gx = 0, gy = 0;
            for (int64_t y = r - n + 1; y <= r + n; ++y)
                for (int64_t x = r - n + 1; x <= r + n; ++x) {
                    const int64_t v = tmpl_host[y * side + x];
                    gx += (2 * x - 2 * r - 1) * v;
                    gy += (2 * y - 2 * r - 1) * v;
                }
            tm->Gx2.push_back(gx);
            tm->Gy2.push_back(gy);
            const unsigned __int128 num = (unsigned __int128)(4 * n * n) *
                                          ((unsigned __int128)((i128)gx * gx) + (unsigned __int128)((i128)gy * gy));
            const unsigned __int128 j = prewitt_j2(n), den = j * j;
            if (firstp) {
                tm->p_lo_n = tm->p_hi_n = num;
                tm->p_lo_d = tm->p_hi_d = den;
                firstp = false;
                continue;
            }
            if (big_cmp(big_mul(Big(num), Big(tm->p_lo_d)), big_mul(Big(tm->p_lo_n), Big(den))) < 0) {
                tm->p_lo_n = num;
                tm->p_lo_d = den;
            }
            if (big_cmp(big_mul(Big(num), Big(tm->p_hi_d)), big_mul(Big(tm->p_hi_n), Big(den))) > 0) {
                tm->p_hi_n = num;
                tm->p_hi_d = den;
            }
        }
    }
    c->tmpls.insert(tm);
    *out = tm;
    return SCR_OK;
}

int build_moment_tables(scr_ctx *c, const uint8_t *img_dev, int32_t H, int32_t W, int64_t pitch, scr_tables *t,
                        scr_stream stream) {
    int rc;
    if ((rc = check_ctx(c)))
        return rc;
    if (!img_dev || !t)
        return fail(SCR_EINVAL, "null image or tables");
    if (H != t->H || W != t->W || pitch < W)
        return fail(SCR_EINVAL, "image %d x %d (pitch %lld) does not match the tables (%d x %d)", H, W,
                    (long long)pitch, t->H, t->W);
    DeviceGuard dg(c->device);
    std::lock_guard<std::mutex> lk(c->mu);
    cudaStream_t st = (cudaStream_t)stream;
    if (!t->mom) {
        const int64_t P = t->t[0].pitch;
        const size_t one = (size_t)(H + 1) * P * 8;
        const size_t bytes = 2 * ((one + 255) & ~size_t(255));
        if ((rc = dev_alloc(c, bytes, st, &t->mom)))
            return rc;
        t->mom_bytes = bytes;
        t->Mx = (uint64_t *)t->mom;
        t->My = (uint64_t *)((char *)t->mom + ((one + 255) & ~size_t(255)));
    }
    Scoped scratch(c, st);
    if ((rc = scratch.take(moment_scratch_bytes(H, W))))
        return rc;
    uint64_t n = 0;
    cudaError_t e = launch_moment_tables(img_dev, pitch, H, W, t->t[0].pitch, t->Mx, t->My, scratch.p, st, &n);
    c->launches += n;
    CUDA_TRY(e);
    t->stream = st;
    return SCR_OK;
}

int template_sums(const scr_tmpl *tm, int32_t t, int64_t out[3]) {
    if (!tm || !out || t < tm->t_min || t > tm->r)
        return fail(SCR_EINVAL, "bad template handle or radius %d", t);
    const int k = t - tm->t_min;
    out[0] = tm->S[k];
    out[1] = tm->Q[k];
    out[2] = tm->Si[k];
    return SCR_OK;
}

void template_release(scr_ctx *c, scr_tmpl *tm) {
    if (!c || !tm)
        return;
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->tmpls.erase(tm))
        delete tm;
}

int screen_bounds(const scr_tmpl *tm, const scr_params *p, scr_bounds *out) {
    if (!tm || !out)
        return fail(SCR_EINVAL, "null argument");
    int rc = validate_params(p);
    if (rc)
        return rc;
    for (int s = 0; s < p->n_scales; ++s)
        bounds_for(tm, p, p->radii[s], &out[s]);
    return SCR_OK;
}

int screen_features(scr_ctx *c, const scr_tables *t, const scr_tmpl *tm, const scr_params *p, uint32_t *mask_dev,
                    uint64_t mask_words, scr_stream stream) {
    int rc;
    if ((rc = check_ctx(c)) || (rc = check_screen_inputs(t, tm, p)))
        return rc;
    const uint64_t need = (uint64_t)p->n_scales * t->H * ((t->W + 31) / 32);
    if (!mask_dev || mask_words < need)
        return fail(SCR_EINVAL, "mask needs %llu words, got %llu", (unsigned long long)need,
                    (unsigned long long)mask_words);
    DeviceGuard dg(c->device);
    ScreenArgs a;
    fill_screen_args(t, tm, p, &a);
    a.mask = mask_dev;
    uint64_t n = 0;
    cudaError_t e = launch_screen(a, (cudaStream_t)stream, &n);
    c->launches += n;
    CUDA_TRY(e);
    const_cast<scr_tables *>(t)->stream = (cudaStream_t)stream;
    return SCR_OK;
}

}  // extern "C"

namespace {

uint64_t isqrt_u64(uint64_t z) {   // floor(sqrt(z)), exact
    uint64_t w = (uint64_t)std::sqrt((long double)z);
    while (w > 0 && w * w > z)
        --w;
    while ((w + 1) * (w + 1) <= z)
        ++w;
    return w;
}

// floor(f/q) of the template's central star of radius t for the enabled
// features (mean, std, contrast order); exact (128-bit where needed)
void template_cells(const scr_tmpl *tm, int t, uint32_t features, const scr_rat q[3], int64_t out[3]) {
    const Geo g = geometry(t);
    const i128 S = tm->S[t - tm->t_min], Q = tm->Q[t - tm->t_min], Si = tm->Si[t - tm->t_min];
    int k = 0;
    if (features & SCR_F_MEAN)
        out[k++] = (int64_t)floor_div(S * q[0].den, (i128)g.A * q[0].num);
    if (features & SCR_F_VAR) {
        const i128 V = (i128)g.A * Q - S * S;
        const uint64_t w = isqrt_u64((uint64_t)(V * q[1].den * q[1].den));
        out[k++] = (int64_t)floor_div((i128)w, (i128)g.A * q[1].num);
    }
    if (features & SCR_F_GRAD) {
        const i128 N = Si * g.Aring - (S - Si) * g.Ain;
        out[k++] = (int64_t)floor_div(N * q[2].den, (i128)g.Ain * g.Aring * q[2].num);
    }
}

}  // namespace

extern "C" {

int screen_joint(scr_ctx *c, const scr_tables *t, const scr_tmpl *tm, const scr_params *p, const scr_joint *jt,
                 uint32_t *mask_dev, uint64_t mask_words, scr_stream stream) {
    int rc;
    if ((rc = check_ctx(c)) || (rc = check_screen_inputs(t, tm, p)))
        return rc;
    if (!jt || !mask_dev || jt->n_areas < 1 || jt->n_areas > 3 || !jt->area_radii)
        return fail(SCR_EINVAL, "joint screen needs 1..3 areas, their radii and a mask");
    if (p->features & SCR_F_PREWITT)
        return fail(SCR_EUNSUPPORTED, "the joint membership screen has no Prewitt feature");
    const uint32_t feats = p->features & 7u;
    if (!feats)
        return fail(SCR_EINVAL, "no feature enabled");
    const int S = p->n_scales, NA = jt->n_areas;
    const uint64_t need = (uint64_t)S * t->H * ((t->W + 31) / 32);
    if (mask_words < need)
        return fail(SCR_EINVAL, "mask has %llu words, needs %llu", (unsigned long long)mask_words,
                    (unsigned long long)need);
    for (int k = 0; k < 3; ++k)
        if (jt->q[k].num < 1 || jt->q[k].num > 65536 || jt->q[k].den < 1 || jt->q[k].den > 16)
            return fail(SCR_EINVAL, "q[%d] = %lld/%lld: need 1 <= num <= 65536, 1 <= den <= 16", k,
                        (long long)jt->q[k].num, (long long)jt->q[k].den);
    for (int j = 0; j < NA; ++j)
        if (jt->band[j][0] > jt->band[j][1] || jt->band[j][0] < tm->t_min || jt->band[j][1] > tm->r ||
            jt->band[j][0] < 2)
            return fail(SCR_EINVAL, "band %d [%d, %d] outside the template's central radii [%d, %d]", j,
                        jt->band[j][0], jt->band[j][1], std::max(tm->t_min, 2), tm->r);
    for (int s = 0; s < S; ++s)
        for (int j = 0; j < NA; ++j) {
            const int rho = jt->area_radii[s * NA + j];
            if (rho < 2 || rho > p->radii[s])
                return fail(SCR_EINVAL, "area radius %d at scale %d, area %d: need 2 <= radius <= %d", rho, s, j,
                            p->radii[s]);
        }
    // membership sets: bit arrays over the cell ranges each area's band spans
    const int nf = __builtin_popcount(feats);
    std::vector<JointSet> sets(NA);
    std::vector<uint32_t> bits;
    uint64_t nbits = 0;
    for (int j = 0; j < NA; ++j) {
        std::vector<std::array<int64_t, 3>> base;
        int64_t lo[3] = {INT64_MAX, INT64_MAX, INT64_MAX}, hi[3] = {INT64_MIN, INT64_MIN, INT64_MIN};
        for (int tt = jt->band[j][0]; tt <= jt->band[j][1]; ++tt) {
            std::array<int64_t, 3> cb = {0, 0, 0};
            template_cells(tm, tt, feats, jt->q, cb.data());
            for (int k = 0; k < nf; ++k) {
                lo[k] = std::min(lo[k], cb[k]);
                hi[k] = std::max(hi[k], cb[k] + 1);
            }
            base.push_back(cb);
        }
        JointSet &st = sets[j];
        uint64_t total = 1;
        for (int k = 0; k < 3; ++k) {
            st.cmin[k] = 0;
            st.dim[k] = 1;
            if (k < nf) {
                if (hi[k] - lo[k] + 1 > (1 << 26) || lo[k] < INT32_MIN || lo[k] > INT32_MAX)
                    return fail(SCR_EINVAL, "area %d: quantisation too fine for the spread of its band", j);
                st.cmin[k] = (int32_t)lo[k];
                st.dim[k] = (uint32_t)(hi[k] - lo[k] + 1);
                total *= st.dim[k];
            }
        }
        if (total > (1ull << 26) || nbits + total > (1ull << 28))
            return fail(SCR_EINVAL, "area %d: its membership array would hold %llu bits (at most 2^26)", j,
                        (unsigned long long)total);
        st.bit0 = nbits;
        nbits += (total + 31) & ~uint64_t(31);
        bits.resize((size_t)(nbits / 32), 0u);
        for (const auto &cb : base)
            for (int m = 0; m < (1 << nf); ++m) {
                uint64_t idx = 0, stride = 1;
                for (int k = 0; k < nf; ++k) {
                    idx += (uint64_t)(cb[k] + ((m >> k) & 1) - st.cmin[k]) * stride;
                    stride *= st.dim[k];
                }
                const uint64_t b = st.bit0 + idx;
                bits[b >> 5] |= 1u << (b & 31);
            }
    }
    // per scale and area: star corner offsets for this pitch
    const int64_t P = t->t[0].pitch;
    std::vector<JointScale> scales(S);
    std::vector<JointArea> areas((size_t)S * NA);
    for (int s = 0; s < S; ++s) {
        const Geo g = geometry(p->radii[s]);
        JointScale &sc = scales[s];
        memset(&sc, 0, sizeof sc);
        sc.y_lo = std::max(g.n, g.h) - 1;
        sc.y_hi = t->H - 1 - std::max(g.n, g.h);
        sc.x_lo = std::max(g.n, g.h) - 1;
        sc.x_hi = std::min(t->W - 1 - g.n, t->W - g.h);
        sc.empty = (sc.x_hi < sc.x_lo || sc.y_hi < sc.y_lo) ? 1u : 0u;
        for (int j = 0; j < NA; ++j) {
            const Geo ga = geometry(jt->area_radii[s * NA + j]);
            JointArea &ar = areas[(size_t)s * NA + j];
            memset(&ar, 0, sizeof ar);
            const int64_t n = ga.n, h = ga.h, ni = ga.ni, hi = ga.hi;
            const int64_t oL[4] = {(n + 1) * P + (n + 1), (1 - n) * P + (n + 1), (n + 1) * P + (1 - n),
                                   (1 - n) * P + (1 - n)};
            const int64_t oT[4] = {(h + 1) * P + 1, P + (1 - h), P + (h + 1), (1 - h) * P + 1};
            const int64_t oLi[4] = {(ni + 1) * P + (ni + 1), (1 - ni) * P + (ni + 1), (ni + 1) * P + (1 - ni),
                                    (1 - ni) * P + (1 - ni)};
            const int64_t oTi[4] = {(hi + 1) * P + 1, P + (1 - hi), P + (hi + 1), (1 - hi) * P + 1};
            for (int k = 0; k < 4; ++k) {
                ar.oL[k] = (int32_t)oL[k];
                ar.oT[k] = (int32_t)oT[k];
                ar.oLi[k] = (int32_t)oLi[k];
                ar.oTi[k] = (int32_t)oTi[k];
            }
            ar.A = (uint32_t)ga.A;
            ar.Ain = (uint32_t)ga.Ain;
            ar.Aring = (uint32_t)ga.Aring;
            // the sums S whose mean cell floor((2 S qd + A qn) / (2 A qn)) lies in
            // [cmin, cmin + dim - 1]: S >= ceil(A qn (2 cmin - 1) / (2 qd)) and
            // S <= ceil(A qn (2 cmax + 1) / (2 qd)) - 1 (the cell grows with S)
            ar.S_lo = 0;
            ar.S_rng = UINT32_MAX;
            if (feats & SCR_F_MEAN) {
                const i128 Aq = (i128)ga.A * jt->q[0].num, d2 = 2 * (i128)jt->q[0].den;
                const i128 cmin = sets[j].cmin[0], cmax = cmin + sets[j].dim[0] - 1;
                const i128 lo = std::max<i128>(ceil_div(Aq * (2 * cmin - 1), d2), 0);
                const i128 hi = std::min<i128>(ceil_div(Aq * (2 * cmax + 1), d2) - 1, (i128)UINT32_MAX);
                if (lo > hi) {
                    ar.S_lo = 1;   // no sum qualifies
                    ar.S_rng = 0;
                } else {
                    ar.S_lo = (uint32_t)lo;
                    ar.S_rng = (uint32_t)(hi - lo);
                }
                if (lo > hi)
                    sc.empty = 1u;   // this area rejects every candidate of the scale
            }
        }
    }
    // one device buffer: scales | areas | sets | bits
    const size_t o_areas = (S * sizeof(JointScale) + 255) & ~size_t(255);
    const size_t o_sets = o_areas + ((areas.size() * sizeof(JointArea) + 255) & ~size_t(255));
    const size_t o_bits = o_sets + ((sets.size() * sizeof(JointSet) + 255) & ~size_t(255));
    const size_t total = o_bits + bits.size() * 4 + 4;
    std::vector<char> host(total, 0);
    memcpy(host.data(), scales.data(), S * sizeof(JointScale));
    memcpy(host.data() + o_areas, areas.data(), areas.size() * sizeof(JointArea));
    memcpy(host.data() + o_sets, sets.data(), sets.size() * sizeof(JointSet));
    memcpy(host.data() + o_bits, bits.data(), bits.size() * 4);
    DeviceGuard dg(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    Scoped buf(c, st);
    if ((rc = buf.take(total)))
        return rc;
    CUDA_TRY(cudaMemcpyAsync(buf.p, host.data(), total, cudaMemcpyHostToDevice, st));
    JointArgs a;
    memset(&a, 0, sizeof a);
    a.L1 = t->t[0].lo;
    a.L2 = t->t[1].lo;
    a.T1 = t->t[2].lo;
    a.T2 = t->t[3].lo;
    a.pitch = P;
    a.H = t->H;
    a.W = t->W;
    a.Wwords = (t->W + 31) / 32;
    a.n_scales = S;
    a.n_areas = NA;
    a.features = feats;
    for (int k = 0; k < 3; ++k) {
        a.qn[k] = (uint64_t)jt->q[k].num;
        a.qd[k] = (uint64_t)jt->q[k].den;
    }
    a.scales = (const JointScale *)buf.p;
    a.areas = (const JointArea *)((char *)buf.p + o_areas);
    a.sets = (const JointSet *)((char *)buf.p + o_sets);
    a.bits = (const uint32_t *)((char *)buf.p + o_bits);
    a.mask = mask_dev;
    uint64_t n = 0;
    cudaError_t e = launch_screen_joint(a, st, &n);
    c->launches += n;
    CUDA_TRY(e);
    CUDA_TRY(cudaStreamSynchronize(st));   // the host copy of the sets must outlive the upload
    return SCR_OK;
}

int compact_mask(scr_ctx *c, const uint32_t *mask_dev, int32_t n_scales, int32_t H, int32_t W, uint64_t *list_dev,
                 uint64_t list_cap, uint64_t *count_dev, scr_stream stream) {
    int rc;
    if ((rc = check_ctx(c)))
        return rc;
    if (!mask_dev || !count_dev || (list_cap && !list_dev))
        return fail(SCR_EINVAL, "null mask, count or list");
    if (((uintptr_t)mask_dev & 15) || ((uintptr_t)count_dev & 7) || ((uintptr_t)list_dev & 7))
        return fail(SCR_EINVAL, "mask must be 16-byte aligned, list and count 8-byte aligned");
    if (n_scales < 1 || n_scales > 65535 || H < 1 || W < 1 || H > 65535 || W > 65535)
        return fail(SCR_EINVAL, "bad mask geometry");
    DeviceGuard dg(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int Ww = (W + 31) / 32;
    const uint64_t total = (uint64_t)n_scales * H * Ww;
    Scoped scratch(c, st);
    if ((rc = scratch.take(compact_scratch_bytes(total))))
        return rc;
    uint64_t n = 0;
    cudaError_t e = launch_compact(mask_dev, total, H, Ww, list_dev, list_cap, count_dev, scratch.p, st, &n);
    c->launches += n;
    CUDA_TRY(e);
    return SCR_OK;
}

int screen_positions_async(scr_ctx *c, const scr_tables *t, const scr_tmpl *tm, const scr_params *p,
                           uint32_t *mask_dev, uint64_t mask_words, uint64_t *list_dev, uint64_t list_cap,
                           uint64_t *count_dev, scr_stream stream) {
    int rc = screen_features(c, t, tm, p, mask_dev, mask_words, stream);
    if (rc)
        return rc;
    return compact_mask(c, mask_dev, p->n_scales, t->H, t->W, list_dev, list_cap, count_dev, stream);
}

int screen_positions(scr_ctx *c, const scr_tables *t, const scr_tmpl *tm, const scr_params *p, uint32_t *mask_dev,
                     uint64_t mask_words, uint64_t *list_dev, uint64_t list_cap, uint64_t *n_survivors,
                     scr_stream stream) {
    int rc;
    if ((rc = check_ctx(c)))
        return rc;
    if (!n_survivors)
        return fail(SCR_EINVAL, "null n_survivors");
    DeviceGuard dg(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    Scoped cnt(c, st);
    if ((rc = cnt.take(8)))
        return rc;
    if ((rc = screen_positions_async(c, t, tm, p, mask_dev, mask_words, list_dev, list_cap, (uint64_t *)cnt.p, stream)))
        return rc;
    std::lock_guard<std::mutex> lk(c->mu);
    CUDA_TRY(cudaMemcpyAsync(c->pinned, cnt.p, 8, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    *n_survivors = c->pinned[0];
    if (*n_survivors > list_cap)
        return fail(SCR_EOVERFLOW, "%llu survivors exceed list capacity %llu", (unsigned long long)*n_survivors,
                    (unsigned long long)list_cap);
    return SCR_OK;
}

int screen_host(scr_ctx *c, const uint8_t *img_host, int32_t H, int32_t W, int64_t pitch, int32_t sum_bits,
                int32_t sq_bits, const scr_tmpl *tm, const scr_params *p, uint64_t *list_host, uint64_t list_cap,
                uint64_t *n_survivors, scr_stream stream) {
    int rc;
    if ((rc = check_ctx(c)))
        return rc;
    if (!img_host || !n_survivors || (list_cap && !list_host))
        return fail(SCR_EINVAL, "null argument");
    if (H < 1 || W < 1 || H > 65535 || W > 65535 || pitch < W)
        return fail(SCR_EINVAL, "bad image geometry");
    if ((rc = validate_params(p)))
        return rc;
    DeviceGuard dg(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t dpitch = (W + 15) / 16 * 16;
    // the image copy goes first, so the host work below overlaps it
    Scoped img(c, st), mask(c, st), list(c, st);
    if ((rc = img.take((size_t)dpitch * H)))
        return rc;
    CUDA_TRY(cudaMemcpy2DAsync(img.p, dpitch, img_host, pitch, W, H, cudaMemcpyHostToDevice, st));
    // A pinned, mapped list buffer (cudaHostAlloc / cudaMallocHost memory)
    // gets the keys and the count (to the context's pinned slot) from one
    // copy kernel after the compaction into device memory: one synchronisation
    // instead of a count read, a list copy and two.  (The compaction writing
    // the keys into host memory itself is slower for long lists: 0.45 ms more
    // for 2.2 M keys, measured.)
    uint64_t *list_map = nullptr;
    if (list_cap && c->pinned_dev) {
        cudaPointerAttributes pa;
        void *d = nullptr;
        // pinned host memory that this device can address (asked with the
        // context's device current); anything else takes the copy-back path
        if (cudaPointerGetAttributes(&pa, list_host) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            cudaHostGetDevicePointer(&d, list_host, 0) == cudaSuccess && d)
            list_map = (uint64_t *)d;
        cudaGetLastError();
    }
    const uint64_t words = (uint64_t)p->n_scales * H * ((W + 31) / 32);
    // an error from here on returns only after the copy has stopped reading img_host
    if ((rc = mask.take(words * 4)) || (rc = list.take(std::max<uint64_t>(list_cap, 1) * 8 + 64))) {
        cudaStreamSynchronize(st);
        return rc;
    }
    scr_tables *t = nullptr;
    if ((rc = build_tables(c, (const uint8_t *)img.p, H, W, dpitch, sum_bits, sq_bits, stream, &t))) {
        cudaStreamSynchronize(st);
        return rc;
    }
    uint64_t *cnt_dev = (uint64_t *)((char *)list.p + std::max<uint64_t>(list_cap, 1) * 8);
    if (list_map) {
        std::lock_guard<std::mutex> lk(c->mu);   // the pinned count slot
        rc = screen_positions_async(c, t, tm, p, (uint32_t *)mask.p, words, (uint64_t *)list.p, list_cap, cnt_dev,
                                    stream);
        if (!rc) {
            uint64_t n = 0;
            cudaError_t e = launch_copy_keys((const uint64_t *)list.p, cnt_dev, list_cap, list_map, c->pinned_dev,
                                             st, &n, kCopyBlocksSync);
            c->launches += n;
            if (e == cudaSuccess)
                e = cudaStreamSynchronize(st);
            if (e == cudaSuccess)
                *n_survivors = c->pinned[0];
            else
                rc = fail(SCR_ECUDA, "screen_host: %s", cudaGetErrorString(e));
        }
    } else {
        rc = screen_positions_async(c, t, tm, p, (uint32_t *)mask.p, words, list_cap ? (uint64_t *)list.p : nullptr,
                                    list_cap, cnt_dev, stream);
        if (!rc) {
            std::lock_guard<std::mutex> lk(c->mu);
            cudaError_t e = cudaMemcpyAsync(c->pinned, cnt_dev, 8, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess)
                e = cudaStreamSynchronize(st);
            if (e == cudaSuccess) {
                *n_survivors = c->pinned[0];
                const uint64_t k = std::min<uint64_t>(*n_survivors, list_cap);
                if (k)
                    e = cudaMemcpyAsync(list_host, list.p, k * 8, cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess)
                    e = cudaStreamSynchronize(st);
            }
            if (e != cudaSuccess)
                rc = fail(SCR_ECUDA, "screen_host: %s", cudaGetErrorString(e));
        }
    }
    if (rc)   // nothing queued may still read img_host or write list_host
        cudaStreamSynchronize(st);
    tables_release(c, t);
    if (!rc && *n_survivors > list_cap)
        return fail(SCR_EOVERFLOW, "%llu survivors exceed list capacity %llu", (unsigned long long)*n_survivors,
                    (unsigned long long)list_cap);
    return rc;
}

// ---------------------------------------------------------------------------
// A stream of same-sized host images (frames_*)
// ---------------------------------------------------------------------------
}  // extern "C"

static constexpr int kMaxFrameDepth = 4;

// Every buffer is reserved once at creation; per frame, the copy stream moves
// the image into its slot while the compute stream builds the tables, screens
// and compacts the previous frame, and the output stream moves the frame
// before that one's keys to the host.  Events order them: the compute of a
// frame waits for its image; the copy into a slot waits until the table build
// of the frame that used the slot before has read it; the key copy of a frame
// waits for its compaction, and the next compaction into the same slot's list
// waits for that key copy.
struct scr_frames {
    scr_ctx *c = nullptr;
    int H = 0, W = 0, depth = 0;
    int64_t dpitch = 0;
    uint64_t list_cap = 0, mask_words = 0;
    ScreenArgs args;                       // fixed: same tables, template and bounds every frame
    scr_tables tabs;                       // laid out in tab_base (not a context-owned handle)
    cudaStream_t st_copy = nullptr, st_comp = nullptr, st_out = nullptr;
    void *img[kMaxFrameDepth] = {};
    void *list_dev[kMaxFrameDepth] = {};   // per slot: keys, then the count
    void *tab_base = nullptr, *build_scratch = nullptr, *compact_scratch = nullptr;
    size_t img_bytes = 0, tab_bytes = 0, build_bytes = 0, compact_bytes = 0, list_bytes = 0, mask_bytes = 0;
    uint32_t *mask = nullptr;
    uint64_t *cnt_host = nullptr;          // pinned, mapped: one count per slot
    uint64_t *cnt_host_dev = nullptr;
    cudaEvent_t ev_img[kMaxFrameDepth] = {}, ev_free[kMaxFrameDepth] = {}, ev_cmp[kMaxFrameDepth] = {},
                ev_done[kMaxFrameDepth] = {};
    int64_t next = 0, oldest = 0;          // frames in flight: tickets [oldest, next)
    std::mutex mu;
};

namespace {

void frames_free(scr_frames *f) {
    scr_ctx *c = f->c;
    if (f->st_copy)
        cudaStreamSynchronize(f->st_copy);
    if (f->st_comp)
        cudaStreamSynchronize(f->st_comp);
    if (f->st_out)
        cudaStreamSynchronize(f->st_out);
    cudaStream_t st = f->st_comp;
    for (int k = 0; k < kMaxFrameDepth; ++k) {
        dev_free(c, f->img[k], f->img_bytes, st);
        dev_free(c, f->list_dev[k], f->list_bytes, st);
    }
    dev_free(c, f->tab_base, f->tab_bytes, st);
    dev_free(c, f->build_scratch, f->build_bytes, st);
    dev_free(c, f->compact_scratch, f->compact_bytes, st);
    dev_free(c, f->mask, f->mask_bytes, st);
    if (st)
        cudaStreamSynchronize(st);
    for (int k = 0; k < kMaxFrameDepth; ++k) {
        if (f->ev_img[k]) cudaEventDestroy(f->ev_img[k]);
        if (f->ev_free[k]) cudaEventDestroy(f->ev_free[k]);
        if (f->ev_cmp[k]) cudaEventDestroy(f->ev_cmp[k]);
        if (f->ev_done[k]) cudaEventDestroy(f->ev_done[k]);
    }
    if (f->cnt_host)
        cudaFreeHost(f->cnt_host);
    if (f->st_copy)
        cudaStreamDestroy(f->st_copy);
    if (f->st_comp)
        cudaStreamDestroy(f->st_comp);
    if (f->st_out)
        cudaStreamDestroy(f->st_out);
    delete f;
}

}  // namespace

void scr_rt::destroy_frames(scr_ctx *c) {
    std::set<scr_frames *> all;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        all.swap(c->frames);
    }
    for (auto *f : all)
        frames_free(f);
}

extern "C" {

int frames_create(scr_ctx *c, int32_t H, int32_t W, int32_t sum_bits, int32_t sq_bits, const scr_tmpl *tm,
                  const scr_params *p, uint64_t list_cap, int32_t depth, scr_frames **out) {
    int rc;
    if ((rc = check_ctx(c)))
        return rc;
    if (!out || !tm)
        return fail(SCR_EINVAL, "null template or out-pointer");
    *out = nullptr;
    if (H < 1 || W < 1 || H > 65535 || W > 65535)
        return fail(SCR_EINVAL, "image %d x %d outside 1..65535", H, W);
    if ((sum_bits != 32 && sum_bits != 64) || (sq_bits != 32 && sq_bits != 64))
        return fail(SCR_EINVAL, "table widths must be 32 or 64 bits");
    if (depth < 1 || depth > kMaxFrameDepth)
        return fail(SCR_EINVAL, "depth %d outside 1..%d", depth, kMaxFrameDepth);
    if ((rc = validate_params(p)))
        return rc;
    if (p->features & SCR_F_PREWITT)
        return fail(SCR_EUNSUPPORTED, "frame pipelines do not build moment tables (SCR_F_PREWITT)");
    if ((p->features & SCR_F_GRAD) && !(tm->features & SCR_F_GRAD))
        return fail(SCR_EINVAL, "template features were computed without SCR_F_GRAD");
    if (list_cap > ((uint64_t)1 << 40))
        return fail(SCR_EINVAL, "list capacity %llu too large", (unsigned long long)list_cap);
    DeviceGuard dg(c->device);
    auto *f = new (std::nothrow) scr_frames();
    if (!f)
        return fail(SCR_ENOMEM, "host allocation failed");
    f->c = c;
    f->H = H;
    f->W = W;
    f->depth = depth;
    f->dpitch = (W + 15) / 16 * 16;
    f->list_cap = list_cap;
    f->mask_words = (uint64_t)p->n_scales * H * ((W + 31) / 32);
    cudaError_t e = cudaStreamCreateWithFlags(&f->st_copy, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&f->st_comp, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&f->st_out, cudaStreamNonBlocking);
    for (int k = 0; k < depth && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&f->ev_img[k], cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&f->ev_free[k], cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&f->ev_cmp[k], cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&f->ev_done[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess)
        e = cudaHostAlloc((void **)&f->cnt_host, kMaxFrameDepth * 8, cudaHostAllocMapped);
    if (e == cudaSuccess)
        e = cudaHostGetDevicePointer((void **)&f->cnt_host_dev, f->cnt_host, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        frames_free(f);
        return fail(SCR_ECUDA, "frame pipeline setup failed: %s", cudaGetErrorString(e));
    }
    cudaStream_t st = f->st_comp;
    f->img_bytes = (size_t)f->dpitch * H;
    int nfil = 0, fk[kMaxFilterWindows][2];
    {
        std::lock_guard<std::mutex> lk(c->mu);
        nfil = c->n_filter;
        memcpy(fk, c->filter_k, sizeof fk);
    }
    f->tab_bytes = tables_bytes(H, W, sum_bits, sq_bits, nfil);
    f->build_bytes = TableScratch::bytes(H, W, sum_bits, sq_bits);
    f->compact_bytes = compact_scratch_bytes(f->mask_words);
    f->mask_bytes = f->mask_words * 4;
    f->list_bytes = std::max<uint64_t>(list_cap, 1) * 8 + 64;
    rc = SCR_OK;
    for (int k = 0; k < depth && !rc; ++k)
        if (!(rc = dev_alloc(c, f->img_bytes, st, &f->img[k])))
            rc = dev_alloc(c, f->list_bytes, st, &f->list_dev[k]);
    if (!rc) rc = dev_alloc(c, f->tab_bytes, st, &f->tab_base);
    if (!rc) rc = dev_alloc(c, f->build_bytes, st, &f->build_scratch);
    if (!rc) rc = dev_alloc(c, f->compact_bytes, st, &f->compact_scratch);
    if (!rc) rc = dev_alloc(c, f->mask_bytes, st, (void **)&f->mask);
    if (!rc && (e = cudaStreamSynchronize(st)) != cudaSuccess)   // the other streams use the slots too
        rc = fail(SCR_ECUDA, "frame pipeline allocation: %s", cudaGetErrorString(e));
    if (rc) {
        frames_free(f);
        return rc;
    }
    layout_tables(&f->tabs, f->tab_base, f->tab_bytes, H, W, sum_bits, sq_bits, st, nfil, fk);
    fill_screen_args(&f->tabs, tm, p, &f->args);
    f->args.mask = f->mask;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->frames.insert(f);
    }
    *out = f;
    return SCR_OK;
}

int frames_submit(scr_frames *f, const uint8_t *img_host, int64_t pitch, uint64_t *list_host, int64_t *ticket) {
    if (!f || !img_host || !ticket)
        return fail(SCR_EINVAL, "null pipeline, image or ticket");
    if (pitch < f->W)
        return fail(SCR_EINVAL, "pitch %lld < width %d", (long long)pitch, f->W);
    scr_ctx *c = f->c;
    DeviceGuard dg(c->device);
    uint64_t *list_map = nullptr;
    if (f->list_cap) {
        cudaPointerAttributes pa;
        void *d = nullptr;
        if (!list_host || cudaPointerGetAttributes(&pa, list_host) != cudaSuccess || pa.type != cudaMemoryTypeHost ||
            cudaHostGetDevicePointer(&d, list_host, 0) != cudaSuccess || !d) {
            cudaGetLastError();
            return fail(SCR_EINVAL, "list_host must be pinned host memory the device can address");
        }
        list_map = (uint64_t *)d;
    }
    std::lock_guard<std::mutex> lk(f->mu);
    if (f->next - f->oldest >= f->depth)
        return fail(SCR_EINVAL, "%d frames in flight: wait for ticket %lld first", f->depth, (long long)f->oldest);
    const int k = (int)(f->next % f->depth);
    uint64_t n = 0;
    cudaError_t e = cudaStreamWaitEvent(f->st_copy, f->ev_free[k], 0);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(f->img[k], f->dpitch, img_host, pitch, f->W, f->H, cudaMemcpyHostToDevice, f->st_copy);
    if (e == cudaSuccess)
        e = cudaEventRecord(f->ev_img[k], f->st_copy);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(f->st_comp, f->ev_img[k], 0);
    const TableDesc *t = f->tabs.t;
    if (e == cudaSuccess)
        e = launch_build_tables((const uint8_t *)f->img[k], f->H, f->W, f->dpitch, t[0], t[1], t[2], t[3],
                                f->tabs.F, f->build_scratch, f->st_comp, &n);
    if (e == cudaSuccess)
        e = cudaEventRecord(f->ev_free[k], f->st_comp);
    if (e == cudaSuccess)
        e = launch_screen(f->args, f->st_comp, &n);
    uint64_t *keys = (uint64_t *)f->list_dev[k];
    uint64_t *cnt = (uint64_t *)((char *)keys + std::max<uint64_t>(f->list_cap, 1) * 8);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(f->st_comp, f->ev_done[k], 0);
    if (e == cudaSuccess)
        e = launch_compact(f->mask, f->mask_words, f->H, (f->W + 31) / 32, f->list_cap ? keys : nullptr, f->list_cap,
                           cnt, f->compact_scratch, f->st_comp, &n);
    if (e == cudaSuccess)
        e = cudaEventRecord(f->ev_cmp[k], f->st_comp);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(f->st_out, f->ev_cmp[k], 0);
    if (e == cudaSuccess)
        e = launch_copy_keys(keys, cnt, f->list_cap, list_map, f->cnt_host_dev + k, f->st_out, &n,
                             kCopyBlocksOverlapped);
    if (e == cudaSuccess)
        e = cudaEventRecord(f->ev_done[k], f->st_out);
    c->launches += n;
    if (e != cudaSuccess) {
        // nothing queued may still read img_host or write list_host
        cudaStreamSynchronize(f->st_copy);
        cudaStreamSynchronize(f->st_comp);
        cudaStreamSynchronize(f->st_out);
        return fail(SCR_ECUDA, "frames_submit: %s", cudaGetErrorString(e));
    }
    *ticket = f->next++;
    return SCR_OK;
}

int frames_wait(scr_frames *f, int64_t ticket, uint64_t *n_survivors) {
    if (!f || !n_survivors)
        return fail(SCR_EINVAL, "null pipeline or count");
    DeviceGuard dg(f->c->device);
    std::lock_guard<std::mutex> lk(f->mu);
    if (f->oldest == f->next || ticket != f->oldest)
        return fail(SCR_EINVAL, "ticket %lld is not the oldest frame in flight", (long long)ticket);
    const int k = (int)(ticket % f->depth);
    cudaError_t e = cudaEventSynchronize(f->ev_done[k]);
    if (e != cudaSuccess)
        return fail(SCR_ECUDA, "frames_wait: %s", cudaGetErrorString(e));
    ++f->oldest;
    *n_survivors = ((volatile uint64_t *)f->cnt_host)[k];
    if (*n_survivors > f->list_cap)
        return fail(SCR_EOVERFLOW, "%llu survivors exceed list capacity %llu", (unsigned long long)*n_survivors,
                    (unsigned long long)f->list_cap);
    return SCR_OK;
}

void frames_destroy(scr_frames *f) {
    if (!f)
        return;
    scr_ctx *c = f->c;
    DeviceGuard dg(c->device);
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->frames.erase(f);
    }
    frames_free(f);
}


// ---------------------------------------------------------------------------
// Batched screening (many images x many templates, one persistent launch)
// ---------------------------------------------------------------------------
}  // extern "C"

namespace scr_rt {

// Lay the units out row by row: for each image and row, one unit per group of
// the image (groups whose valid rows exclude the row leave that unit empty).
// The groups of an image are contiguous in b->groups.
void plan_layout(scr_batch *b) {
    std::vector<int> first(b->images.size(), -1), count(b->images.size(), 0);
    for (size_t g = 0; g < b->groups.size(); ++g) {
        const int i = b->groups[g].image;
        if (first[i] < 0)
            first[i] = (int)g;
        ++count[i];
    }
    int64_t u = 0;
    for (size_t i = 0; i < b->images.size(); ++i) {
        BImage &im = b->images[i];
        im.unit0 = u;
        im.g0 = std::max(first[i], 0);
        im.n_grp = count[i];
        im.y_first = 0;
        im.rows = 0;
        if (!count[i])
            continue;
        int ylo = INT32_MAX, yhi = -1;
        for (int g = first[i]; g < first[i] + count[i]; ++g) {
            ylo = std::min(ylo, b->groups[g].y_lo);
            yhi = std::max(yhi, b->groups[g].y_hi);
        }
        im.y_first = ylo;
        im.rows = yhi - ylo + 1;
        u += (int64_t)im.rows * im.n_grp;
    }
    b->n_units = u;
}

int build_plan(scr_ctx *c, scr_batch *b, const scr_tables *const *tables, int n_images, const scr_tmpl *const *tmpls,
               const scr_params *params, int n_tmpls, const scr_pair *pairs, int n_pairs) {
    b->images.resize(n_images);
    uint64_t moff = 0;
    for (int i = 0; i < n_images; ++i) {
        const scr_tables *t = tables[i];
        BImage &im = b->images[i];
        im.L1 = t->t[0].lo;
        im.L2 = t->t[1].lo;
        im.T1 = t->t[2].lo;
        im.T2 = t->t[3].lo;
        im.pitch = t->t[0].pitch;
        im.H = t->H;
        im.W = t->W;
        im.Wwords = (t->W + 31) / 32;
        im.mask_offset = (int64_t)moff;
        moff += (uint64_t)t->H * im.Wwords;
    }
    b->union_words = moff;
    // records per (image, R), in (pair, scale) order
    std::vector<std::map<int, std::vector<BRecord>>> byR(n_images);
    b->candidates = 0;
    for (int p = 0; p < n_pairs; ++p) {
        const int i = pairs[p].image, t = pairs[p].tmpl;
        const scr_params *pp = &params[t];
        for (int s = 0; s < pp->n_scales; ++s) {
            const int R = pp->radii[s];
            scr_bounds bd;
            bounds_for(tmpls[t], pp, R, &bd);
            BRecord rc = {};
            rc.pair = (uint32_t)p;
            rc.s = (uint32_t)s;
            rc.features = pp->features;
            rc.S_lo = 0;
            rc.S_rng = UINT32_MAX;
            bool empty = false;
            if (pp->features & SCR_F_MEAN) {
                const int64_t lo = std::max<int64_t>(bd.S_lo, 0), hi = std::min<int64_t>(bd.S_hi, UINT32_MAX);
                if (lo > hi)
                    empty = true;
                else {
                    rc.S_lo = (uint32_t)lo;
                    rc.S_rng = (uint32_t)(hi - lo);
                }
            }
            if (pp->features & SCR_F_VAR) {
                empty = empty || bd.V_lo > bd.V_hi;
                rc.V_lo = bd.V_lo;
                rc.V_rng = (uint64_t)((i128)bd.V_hi - (i128)bd.V_lo);
            }
            if (pp->features & SCR_F_GRAD) {
                empty = empty || bd.N_lo > bd.N_hi;
                rc.N_lo = bd.N_lo;
                rc.N_rng = (uint64_t)((i128)bd.N_hi - (i128)bd.N_lo);
            }
            const Geo g = geometry(R);
            const int H = b->images[i].H, W = b->images[i].W;
            const int ylo = std::max(g.n, g.h) - 1, yhi = H - 1 - std::max(g.n, g.h);
            const int xlo = std::max(g.n, g.h) - 1, xhi = std::min(W - 1 - g.n, W - g.h);
            if (yhi < ylo || xhi < xlo)
                continue;   // no valid position at this scale
            b->candidates += (uint64_t)(yhi - ylo + 1) * (uint64_t)(xhi - xlo + 1);
            if (!empty)
                byR[i][R].push_back(rc);
        }
    }
    b->groups.clear();
    b->records.clear();
    for (int i = 0; i < n_images; ++i) {
        const BImage &im = b->images[i];
        const int64_t P = im.pitch;
        for (auto &kv : byR[i]) {
            const int R = kv.first;
            const Geo g = geometry(R);
            BGroup gr = {};
            gr.image = i;
            gr.R = R;
            gr.y_lo = std::max(g.n, g.h) - 1;
            gr.y_hi = im.H - 1 - std::max(g.n, g.h);
            gr.x_lo = std::max(g.n, g.h) - 1;
            gr.x_hi = std::min(im.W - 1 - g.n, im.W - g.h);
            gr.w_lo = gr.x_lo / 32;
            gr.w_hi = gr.x_hi / 32;
            const int64_t n = g.n, h = g.h, ni = g.ni, hi = g.hi;
            const int64_t oL[4] = {(n + 1) * P + (n + 1), (1 - n) * P + (n + 1), (n + 1) * P + (1 - n), (1 - n) * P + (1 - n)};
            const int64_t oT[4] = {(h + 1) * P + 1, P + (1 - h), P + (h + 1), (1 - h) * P + 1};
            const int64_t oLi[4] = {(ni + 1) * P + (ni + 1), (1 - ni) * P + (ni + 1), (ni + 1) * P + (1 - ni),
                                    (1 - ni) * P + (1 - ni)};
            const int64_t oTi[4] = {(hi + 1) * P + 1, P + (1 - hi), P + (hi + 1), (1 - hi) * P + 1};
            for (int k = 0; k < 4; ++k) {
                gr.oL[k] = (int32_t)oL[k];
                gr.oT[k] = (int32_t)oT[k];
                gr.oLi[k] = (int32_t)oLi[k];
                gr.oTi[k] = (int32_t)oTi[k];
            }
            gr.A = (uint32_t)g.A;
            gr.Ain = (uint32_t)g.Ain;
            gr.Aring = (uint32_t)g.Aring;
            uint64_t hlo = UINT32_MAX, hhi = 0;
            i128 vlo = (i128)INT64_MAX, vhi = (i128)INT64_MIN;
            gr.need = 0;
            gr.all_var = 1;
            for (const BRecord &rc : kv.second) {
                gr.need |= rc.features;
                if (rc.features & SCR_F_VAR) {
                    vlo = std::min<i128>(vlo, (i128)rc.V_lo);
                    vhi = std::max<i128>(vhi, (i128)rc.V_lo + (i128)rc.V_rng);
                } else {
                    gr.all_var = 0;
                }
                if (rc.features & SCR_F_MEAN) {
                    hlo = std::min<uint64_t>(hlo, rc.S_lo);
                    hhi = std::max<uint64_t>(hhi, (uint64_t)rc.S_lo + rc.S_rng);
                } else {
                    hlo = 0;
                    hhi = UINT32_MAX;
                }
            }
            gr.S_lo_hull = (uint32_t)hlo;
            gr.S_rng_hull = (uint32_t)(hhi - hlo);
            if (kv.second.empty() || vlo > vhi)
                gr.all_var = 0;
            if (gr.all_var) {
                gr.V_lo_hull = (int64_t)vlo;
                gr.V_rng_hull = (uint64_t)(vhi - vlo);
            }
            gr.rec0 = (int32_t)b->records.size();
            // ascending mean-interval start, so a warp stops at the first record
            // whose interval starts above every mean it holds
            std::stable_sort(kv.second.begin(), kv.second.end(),
                             [](const BRecord &x, const BRecord &y) { return x.S_lo < y.S_lo; });
            b->records.insert(b->records.end(), kv.second.begin(), kv.second.end());
            gr.rec1 = (int32_t)b->records.size();
            b->groups.push_back(gr);
        }
    }
    (void)c;
    return SCR_OK;
}

void pack_plan(const scr_batch *b, void *dst) {
    char *host = (char *)dst;
    size_t off = 0;
    memcpy(host + off, b->images.data(), b->images.size() * sizeof(BImage));
    off += (b->images.size() * sizeof(BImage) + 255) & ~size_t(255);
    memcpy(host + off, b->groups.data(), b->groups.size() * sizeof(BGroup));
    off += (b->groups.size() * sizeof(BGroup) + 255) & ~size_t(255);
    memcpy(host + off, b->records.data(), b->records.size() * sizeof(BRecord));
}

int upload_plan(scr_batch *b, cudaStream_t st) {
    std::vector<char> host(b->desc_bytes);
    pack_plan(b, host.data());
    CUDA_TRY(cudaMemcpyAsync(b->desc, host.data(), b->desc_bytes, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return SCR_OK;
}

size_t desc_size(const scr_batch *b) {
    return ((b->images.size() * sizeof(BImage) + 255) & ~size_t(255)) +
           ((b->groups.size() * sizeof(BGroup) + 255) & ~size_t(255)) +
           ((b->records.size() * sizeof(BRecord) + 255) & ~size_t(255)) + 256;
}

void set_args(scr_batch *b) {
    char *base = (char *)b->desc;
    b->args.images = (const BImage *)base;
    base += (b->images.size() * sizeof(BImage) + 255) & ~size_t(255);
    b->args.groups = (const BGroup *)base;
    base += (b->groups.size() * sizeof(BGroup) + 255) & ~size_t(255);
    b->args.records = (const BRecord *)base;
    b->args.n_images = (int32_t)b->images.size();
    b->args.n_groups = (int32_t)b->groups.size();
    b->args.n_units = b->n_units;
    b->args.unit_stride = 1;
}

int sm_count(int device) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device);
    return n > 0 ? n : 1;
}

// One run: zero the outputs, screen, sort, offsets.
int enqueue_run(scr_batch *b, cudaStream_t st, uint64_t *launches) {
    if (b->union_words && b->args.union_mask)
        CUDA_TRY(cudaMemsetAsync(b->args.union_mask, 0, b->union_words * 4, st));
    CUDA_TRY(cudaMemsetAsync(b->args.counts, 0, (size_t)b->n_pairs * 8, st));
    CUDA_TRY(cudaMemsetAsync(b->n_reserved, 0, 16, st));   // slot counter, unit counter
    if (b->n_units > 0 && !b->groups.empty())
        CUDA_TRY(launch_batch(b->args, b->wpw, b->grid, st, launches));
    if (b->args.keys_cap > 0) {
        CUDA_TRY(launch_sort(b->sargs, b->sort_passes, sm_count(b->ctx->device) * 4, st, launches));
    }
    CUDA_TRY(launch_pair_offsets(b->args.counts, b->offsets, b->n_keys, b->n_reserved, b->n_pairs, st, launches));
    return SCR_OK;
}

void free_batch_on(scr_ctx *c, scr_batch *b, cudaStream_t st) {
    dev_free(c, b->desc, b->desc_bytes, st);
    dev_free(c, b->sort_buf, b->sort_bytes, st);
    delete b;
}

void free_batch(scr_ctx *c, scr_batch *b) {
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    if (b->graph)
        cudaGraphDestroy(b->graph);
    if (b->cap_stream) {
        cudaStreamSynchronize(b->cap_stream);
        cudaStreamDestroy(b->cap_stream);
    }
    dev_free(c, b->desc, b->desc_bytes, nullptr);
    dev_free(c, b->sort_buf, b->sort_bytes, nullptr);
    delete b;
}

int batch_prepare(scr_ctx *c, const scr_tables *const *tables, int n_images, const scr_tmpl *const *tmpls,
                  const scr_params *params, int n_tmpls, const scr_pair *pairs, int n_pairs, uint64_t *counts_dev,
                  uint64_t *offsets_dev, uint32_t *union_mask_dev, uint64_t *keys_dev, uint64_t keys_cap,
                  uint64_t *n_keys_dev, cudaStream_t st, scr_batch **out) {
    int rc;
    auto *b = new (std::nothrow) scr_batch();
    if (!b)
        return fail(SCR_ENOMEM, "host allocation failed");
    b->ctx = c;
    b->n_images = n_images;
    b->n_pairs = n_pairs;
    build_plan(c, b, tables, n_images, tmpls, params, n_tmpls, pairs, n_pairs);
    b->desc_bytes = desc_size(b);
    // sort on the key fields cut to their used widths: column, row, scale, and
    // pair with one value to spare so that the all-ones sentinel sorts last
    auto bits_for = [](uint64_t v) {   // bits to hold 0 .. v
        uint32_t k = 1;
        while (k < 64 && (v >> k))
            ++k;
        return k;
    };
    int maxH = 1, maxW = 1, maxS = 1;
    for (int i = 0; i < n_images; ++i) {
        maxH = std::max(maxH, tables[i]->H);
        maxW = std::max(maxW, tables[i]->W);
    }
    for (int t = 0; t < n_tmpls; ++t)
        maxS = std::max(maxS, params[t].n_scales);
    b->sargs.xb = bits_for((uint64_t)maxW - 1);
    b->sargs.yb = bits_for((uint64_t)maxH - 1);
    b->sargs.sb = bits_for((uint64_t)maxS - 1);
    b->sargs.pb = bits_for((uint64_t)n_pairs);
    b->sort_passes = (int)((b->sargs.xb + b->sargs.yb + b->sargs.sb + b->sargs.pb + 7) / 8);
    const uint64_t cap1 = keys_cap ? keys_cap : 1;
    const uint64_t tiles = sort_max_tiles(cap1);
    const size_t hist_bytes = (sort_hist_bytes(cap1) + 255) & ~size_t(255);
    const size_t csum_bytes = (sort_csum_bytes(cap1) + 255) & ~size_t(255);
    b->sort_bytes = hist_bytes + csum_bytes + (size_t)cap1 * 8 + 256;
    if ((rc = dev_alloc(c, b->desc_bytes, st, &b->desc)) || (rc = dev_alloc(c, b->sort_bytes, st, &b->sort_buf))) {
        free_batch(c, b);
        return rc;
    }
    b->n_reserved = (uint64_t *)((char *)b->sort_buf + b->sort_bytes - 256);
    b->n_keys = n_keys_dev;
    uint64_t *scratch = (uint64_t *)((char *)b->sort_buf + hist_bytes + csum_bytes);
    // the screening kernel writes the unsorted keys where an odd or even number
    // of sort passes ends in the caller's buffer
    uint64_t *first = (b->sort_passes & 1) ? scratch : keys_dev;
    b->args.counts = counts_dev;
    b->args.union_mask = union_mask_dev;
    b->args.keys = first;
    b->args.keys_cap = keys_cap;
    b->args.n_reserved = b->n_reserved;
    b->args.next_unit = b->n_reserved + 1;
    b->offsets = offsets_dev;
    b->sargs.src = first;
    b->sargs.dst = (b->sort_passes & 1) ? keys_dev : scratch;
    b->sargs.hist = (uint32_t *)b->sort_buf;
    b->sargs.csum = (uint64_t *)((char *)b->sort_buf + hist_bytes);
    b->sargs.n_keys = b->n_reserved;
    b->sargs.cap = keys_cap;
    b->sargs.max_tiles = tiles;
    *out = b;
    return SCR_OK;
}

void batch_set_shape(scr_batch *b, int wpw, int blocks_per_sm) {
    b->wpw = wpw;
    b->blocks_per_sm = blocks_per_sm;
    b->grid = sm_count(b->ctx->device) * blocks_per_sm;
    plan_layout(b);
    set_args(b);
}

}  // namespace scr_rt

extern "C" {

int screen_batch_create(scr_ctx *c, const scr_tables *const *tables, int32_t n_images, const scr_tmpl *const *tmpls,
                        const scr_params *params, int32_t n_tmpls, const scr_pair *pairs, int32_t n_pairs,
                        uint64_t *counts_dev, uint64_t *offsets_dev, uint32_t *union_mask_dev, uint64_t *keys_dev,
                        uint64_t keys_cap, uint64_t *n_keys_dev, const scr_batch_tuning *tuning, scr_stream stream,
                        scr_batch **out) {
    int rc;
    if ((rc = check_ctx(c)))
        return rc;
    if (!out || !tables || !tmpls || !params || !pairs || n_images < 1 || n_tmpls < 1 || n_pairs < 1)
        return fail(SCR_EINVAL, "null or empty batch description");
    if (n_pairs >= (1 << 26))
        return fail(SCR_EINVAL, "at most 2^26 pairs");
    if (!counts_dev || !n_keys_dev || (keys_cap && !keys_dev))
        return fail(SCR_EINVAL, "null counts, key count or keys");
    for (int i = 0; i < n_images; ++i) {
        if (!tables[i])
            return fail(SCR_EINVAL, "null tables for image %d", i);
        if (tables[i]->H > 65535 || tables[i]->W > 65535)
            return fail(SCR_EINVAL, "image %d too large for 16-bit key fields", i);
    }
    for (int t = 0; t < n_tmpls; ++t) {
        if ((rc = check_screen_inputs(tables[0], tmpls[t], &params[t])))
            return fail(rc, "template %d: %s", t, g_last_error.c_str());
        if (params[t].n_scales > 32)
            return fail(SCR_EINVAL, "template %d: more than 32 scales", t);
        if (params[t].features & SCR_F_PREWITT)
            return fail(SCR_EUNSUPPORTED, "template %d: the batched screen has no Prewitt test", t);
    }
    for (int p = 0; p < n_pairs; ++p)
        if (pairs[p].image < 0 || pairs[p].image >= n_images || pairs[p].tmpl < 0 || pairs[p].tmpl >= n_tmpls)
            return fail(SCR_EINVAL, "pair %d out of range", p);
    *out = nullptr;
    DeviceGuard dg(c->device);
    std::lock_guard<std::mutex> lk(c->mu);
    cudaStream_t st = (cudaStream_t)stream;
    scr_batch *b = nullptr;
    if ((rc = batch_prepare(c, tables, n_images, tmpls, params, n_tmpls, pairs, n_pairs, counts_dev, offsets_dev,
                            union_mask_dev, keys_dev, keys_cap, n_keys_dev, st, &b)))
        return rc;
    const int sms = sm_count(c->device);
    // tuning: given, cached for this batch shape, or measured now
    char key[160];
    snprintf(key, sizeof key, "dev%d/img%d/pairs%d/groups%zu/records%zu/cand%llu", c->device, n_images, n_pairs,
             b->groups.size(), b->records.size(), (unsigned long long)b->candidates);
    std::vector<std::pair<int, int>> cand;
    if (tuning && tuning->words_per_warp > 0) {
        cand.push_back({tuning->words_per_warp, tuning->blocks_per_sm > 0 ? tuning->blocks_per_sm : 4});
    } else if (c->tuned.count(key)) {
        cand.push_back(c->tuned[key]);
    } else {
        for (int w : {2, 4, 8})
            for (int bps : {2, 4, 8})
                cand.push_back({w, bps});
    }
    for (auto &cf : cand)
        if (cf.first != 2 && cf.first != 4 && cf.first != 8)
            cf.first = 8;
    float best = 1e30f;
    std::pair<int, int> chosen = cand[0];
    if (cand.size() > 1) {
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (auto cf : cand) {
            b->wpw = cf.first;
            b->blocks_per_sm = cf.second;
            b->grid = sms * cf.second;
            plan_layout(b);
            if ((rc = upload_plan(b, st))) {
                free_batch(c, b);
                return rc;
            }
            set_args(b);
            // time an evenly strided sample of about 2^17 units of this layout
            BatchArgs sample = b->args;
            sample.unit_stride = std::max<int64_t>(1, b->n_units >> 17);
            sample.n_units = b->n_units / sample.unit_stride;
            float ms = 0;
            for (int rep = 0; rep < 2; ++rep) {   // first run warms up, second is timed
                cudaMemsetAsync(b->args.counts, 0, (size_t)n_pairs * 8, st);
                cudaMemsetAsync(b->n_reserved, 0, 16, st);
                cudaEventRecord(e0, st);
                if (b->n_units > 0 && !b->groups.empty())
                    launch_batch(sample, b->wpw, b->grid, st, nullptr);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ms, e0, e1);
            }
            if (cudaGetLastError() != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                free_batch(c, b);
                return fail(SCR_ECUDA, "batch kernel failed during tuning");
            }
            if (ms < best) {
                best = ms;
                chosen = cf;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c->tuned[key] = chosen;
    }
    b->wpw = chosen.first;
    b->blocks_per_sm = chosen.second;
    b->grid = sms * chosen.second;
    plan_layout(b);
    if ((rc = upload_plan(b, st))) {
        free_batch(c, b);
        return rc;
    }
    set_args(b);
    // capture one run into a CUDA graph on a private stream
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        free_batch(c, b);
        return fail(SCR_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    }
    uint64_t n_launch = 0;
    rc = enqueue_run(b, b->cap_stream, &n_launch);
    e = cudaStreamEndCapture(b->cap_stream, &b->graph);
    if (rc || e != cudaSuccess) {
        free_batch(c, b);
        return rc ? rc : fail(SCR_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
        free_batch(c, b);
        return fail(SCR_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    c->batches.insert(b);
    *out = b;
    return SCR_OK;
}

int screen_batch_run(scr_batch *b, scr_stream stream) {
    if (!b)
        return fail(SCR_EINVAL, "null batch");
    DeviceGuard dg(b->ctx->device);
    CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    // the graph holds the screening kernel, the sort passes and the offsets
    b->ctx->launches += 2 + (uint64_t)(b->args.keys_cap ? b->sort_passes * kSortLaunchesPerPass : 0);
    return SCR_OK;
}

int screen_batch_info(const scr_batch *b, scr_batch_info *out) {
    if (!b || !out)
        return fail(SCR_EINVAL, "null argument");
    out->n_groups = (int64_t)b->groups.size();
    out->n_records = (int64_t)b->records.size();
    out->n_units = b->n_units;
    out->candidates = b->candidates;
    out->words_per_warp = b->wpw;
    out->blocks_per_sm = b->blocks_per_sm;
    out->union_words = b->union_words;
    out->sort_passes = b->args.keys_cap ? b->sort_passes : 0;
    out->reserved = 0;
    return SCR_OK;
}

void screen_batch_release(scr_ctx *c, scr_batch *b) {
    if (!c || !b)
        return;
    DeviceGuard dg(c->device);
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->batches.erase(b))
        free_batch(c, b);
}

}  // extern "C"
