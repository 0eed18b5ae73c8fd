// Joint-vector membership screen (Sec. 5): the paper's uniform quantiser
// Q(f) = floor(f/q + 1/2) applied to the star's mean, standard deviation and
// inner-star contrast, the quantised vector tested for membership in the
// template's feature set F (a bit array over cell vectors, built on the host
// from the template's central stars of each area's band), for up to three
// nested central areas of the candidate (Sec. 5, features of several central
// areas): a candidate survives only if every area is a member.  Exact integer
// arithmetic throughout; the quantiser is evaluated by integer division and,
// for the standard deviation, an exact integer square root.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "screen.h"

namespace scr {
namespace {

__device__ __forceinline__ uint32_t ldj(const uint32_t *p) { return __ldg(p); }

__device__ __forceinline__ uint32_t sum8(const uint32_t *L, const uint32_t *T, const int32_t (&oL)[4],
                                         const int32_t (&oT)[4]) {
    return ldj(L + oL[0]) - ldj(L + oL[1]) - ldj(L + oL[2]) + ldj(L + oL[3]) + ldj(T + oT[0]) - ldj(T + oT[1]) -
           ldj(T + oT[2]) + ldj(T + oT[3]);
}

// floor(sqrt(z)) for z < 2^62: the double square root, then made exact by
// integer comparison (a double is within one of the true root at this size)
__device__ __forceinline__ uint64_t isqrt_exact(uint64_t z) {
    uint64_t w = (uint64_t)sqrt((double)z);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (w * w > z)
            --w;
        if ((w + 1) * (w + 1) <= z)
            ++w;
    }
    return w;
}

__device__ __forceinline__ int64_t floor_div(int64_t a, int64_t b) {   // b > 0
    int64_t q = a / b;
    if ((a % b != 0) && (a < 0))
        --q;
    return q;
}

// Is the candidate at element e of the tables, whose area `ar` has star sum S,
// in set `st`?  (S has passed the set's exact range test on the mean cell.)
__device__ __noinline__ bool member_cells(const JointArgs &a, const JointArea &ar, const JointSet &st, int64_t e,
                                           uint32_t S) {
    const uint64_t A = ar.A;
    uint64_t idx = 0, stride = 1;
    int k = 0;
    if (a.features & SCR_F_MEAN) {
        const uint64_t qn = a.qn[0], qd = a.qd[0];
        const int64_t c = (int64_t)((2 * (uint64_t)S * qd + A * qn) / (2 * A * qn));
        const int64_t d = c - st.cmin[k];
        if (d < 0 || d >= (int64_t)st.dim[k])
            return false;
        idx += (uint64_t)d * stride;
        stride *= st.dim[k];
        ++k;
    }
    if (a.features & SCR_F_VAR) {
        const uint32_t *L2 = a.L2 + e, *T2 = a.T2 + e;
        const uint32_t qs = ldj(L2 + ar.oL[0]) - ldj(L2 + ar.oL[1]) - ldj(L2 + ar.oL[2]) + ldj(L2 + ar.oL[3]);
        const uint32_t qdm = ldj(T2 + ar.oT[0]) - ldj(T2 + ar.oT[1]) - ldj(T2 + ar.oT[2]) + ldj(T2 + ar.oT[3]);
        const uint64_t Q = (uint64_t)qs + qdm;
        const uint64_t V = A * Q - (uint64_t)S * S;
        const uint64_t qn = a.qn[1], qd = a.qd[1];
        const uint64_t w = isqrt_exact(4 * qd * qd * V);
        const int64_t c = (int64_t)((w + A * qn) / (2 * A * qn));
        const int64_t d = c - st.cmin[k];
        if (d < 0 || d >= (int64_t)st.dim[k])
            return false;
        idx += (uint64_t)d * stride;
        stride *= st.dim[k];
        ++k;
    }
    if (a.features & SCR_F_GRAD) {
        const uint32_t Si = sum8(a.L1 + e, a.T1 + e, ar.oLi, ar.oTi);
        const int64_t N = (int64_t)((uint64_t)Si * ar.Aring) - (int64_t)((uint64_t)(S - Si) * ar.Ain);
        const int64_t D = (int64_t)ar.Ain * ar.Aring;
        const int64_t qn = (int64_t)a.qn[2], qd = (int64_t)a.qd[2];
        const int64_t c = floor_div(2 * N * qd + D * qn, 2 * D * qn);
        const int64_t d = c - st.cmin[k];
        if (d < 0 || d >= (int64_t)st.dim[k])
            return false;
        idx += (uint64_t)d * stride;
    }
    const uint64_t bit = st.bit0 + idx;
    return (__ldg(a.bits + (bit >> 5)) >> (bit & 31)) & 1u;
}

__device__ __forceinline__ bool member(const JointArgs &a, const JointArea &ar, const JointSet &st, int64_t e) {
    const uint32_t S = sum8(a.L1 + e, a.T1 + e, ar.oL, ar.oT);
    if (S - ar.S_lo > ar.S_rng)   // its mean cell is outside the set's range (exact)
        return false;
    return member_cells(a, ar, st, e, S);
}

constexpr int kJointWarps = 8;
constexpr int kJointWPW = 8;   // mask words per warp
constexpr int kMaxAreas = 3;

// One warp covers kJointWPW consecutive mask words of a row for every scale.
// The per-scale records are staged in shared memory once per block.  Per
// scale, the outermost area's star sums of all words are read back to back
// (8 corners at immediate offsets from pointers formed once) and tested
// against the set's exact range on the mean cell, which rejects nearly every
// candidate; the quantised cells, the membership bit and the inner areas are
// evaluated only for the words where some lane survives.
__global__ void __launch_bounds__(32 * kJointWarps) k_screen_joint(const JointArgs a) {
    pdl_begin();
    __shared__ JointScale s_sc[kMaxScales];
    __shared__ JointArea s_ar[kMaxScales * kMaxAreas];
    __shared__ JointSet s_st[kMaxAreas];
    {
        const int t = threadIdx.x;
        const int nsc = a.n_scales * (int)(sizeof(JointScale) / 4);
        const int nar = a.n_scales * a.n_areas * (int)(sizeof(JointArea) / 4);
        const int nst = a.n_areas * (int)(sizeof(JointSet) / 4);
        for (int k = t; k < nsc; k += blockDim.x)
            reinterpret_cast<uint32_t *>(s_sc)[k] = __ldg(reinterpret_cast<const uint32_t *>(a.scales) + k);
        for (int k = t; k < nar; k += blockDim.x)
            reinterpret_cast<uint32_t *>(s_ar)[k] = __ldg(reinterpret_cast<const uint32_t *>(a.areas) + k);
        for (int k = t; k < nst; k += blockDim.x)
            reinterpret_cast<uint32_t *>(s_st)[k] = __ldg(reinterpret_cast<const uint32_t *>(a.sets) + k);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * kJointWarps + (threadIdx.x >> 5)) * kJointWPW;
    const int y = blockIdx.y;
    if (w0 >= a.Wwords)
        return;
    const int64_t plane = (int64_t)a.H * a.Wwords;
    const int x0 = w0 * 32 + lane;
    const int64_t e0 = (int64_t)y * a.pitch + x0 + kColOffset;   // word 0's candidate
    const bool store_word = lane < kJointWPW && w0 + lane < a.Wwords;
#pragma unroll 1
    for (int s = 0; s < a.n_scales; ++s) {
        const JointScale &sc = s_sc[s];
        uint32_t keep = 0;   // bit j: word j's candidate is still alive
        if (!sc.empty && y >= sc.y_lo && y <= sc.y_hi) {   // block-uniform
            const JointArea &ar0 = s_ar[s * a.n_areas];
            const uint32_t *L = a.L1 + e0, *T = a.T1 + e0;
            const uint32_t *p0 = L + ar0.oL[0], *p1 = L + ar0.oL[1], *p2 = L + ar0.oL[2], *p3 = L + ar0.oL[3];
            const uint32_t *q0 = T + ar0.oT[0], *q1 = T + ar0.oT[1], *q2 = T + ar0.oT[2], *q3 = T + ar0.oT[3];
            const uint32_t span = (uint32_t)(sc.x_hi - sc.x_lo);
            uint32_t S[kJointWPW];
            const int xw_lo = w0 * 32, xw_hi = xw_lo + 32 * kJointWPW - 1;
            if (xw_lo >= sc.x_lo && xw_hi <= sc.x_hi) {   // warp-uniform: every word valid
                // all corner reads written before any sum: issued back to back
                uint32_t v[kJointWPW][8];
#pragma unroll
                for (int j = 0; j < kJointWPW; ++j) {
                    const int d = 32 * j;
                    v[j][0] = ldj(p0 + d), v[j][1] = ldj(p1 + d), v[j][2] = ldj(p2 + d), v[j][3] = ldj(p3 + d);
                    v[j][4] = ldj(q0 + d), v[j][5] = ldj(q1 + d), v[j][6] = ldj(q2 + d), v[j][7] = ldj(q3 + d);
                }
#pragma unroll
                for (int j = 0; j < kJointWPW; ++j) {
                    S[j] = v[j][0] - v[j][1] - v[j][2] + v[j][3] + v[j][4] - v[j][5] - v[j][6] + v[j][7];
                    keep |= (S[j] - ar0.S_lo <= ar0.S_rng ? 1u : 0u) << j;
                }
            } else {
#pragma unroll
                for (int j = 0; j < kJointWPW; ++j) {
                    const int d = 32 * j;
                    S[j] = 0;
                    if ((uint32_t)(x0 + d - sc.x_lo) <= span) {
                        S[j] = ldj(p0 + d) - ldj(p1 + d) - ldj(p2 + d) + ldj(p3 + d) + ldj(q0 + d) - ldj(q1 + d) -
                               ldj(q2 + d) + ldj(q3 + d);
                        keep |= (S[j] - ar0.S_lo <= ar0.S_rng ? 1u : 0u) << j;
                    }
                }
            }
            if (__any_sync(0xffffffffu, keep != 0)) {
                // rare: the quantised cells of the survivors of the range test
#pragma unroll 1
                for (int j = 0; j < kJointWPW; ++j) {
                    if (!((keep >> j) & 1u))
                        continue;
                    uint32_t Sj = 0;
#pragma unroll
                    for (int q = 0; q < kJointWPW; ++q)
                        Sj = q == j ? S[q] : Sj;
                    const int64_t e = e0 + 32 * j;
                    bool pass = member_cells(a, ar0, s_st[0], e, Sj);
                    for (int k = 1; k < a.n_areas && pass; ++k)
                        pass = member(a, s_ar[s * a.n_areas + k], s_st[k], e);
                    if (!pass)
                        keep &= ~(1u << j);
                }
            }
        }
        uint32_t mine = 0;
#pragma unroll
        for (int j = 0; j < kJointWPW; ++j) {
            const uint32_t bits = __ballot_sync(0xffffffffu, (keep >> j) & 1u);
            mine = lane == j ? bits : mine;
        }
        if (store_word)
            a.mask[s * plane + (int64_t)y * a.Wwords + w0 + lane] = mine;
    }
}

}  // namespace

cudaError_t launch_screen_joint(const JointArgs &a, cudaStream_t st, uint64_t *launches) {
    const int words_per_block = kJointWarps * kJointWPW;
    const dim3 grid((a.Wwords + words_per_block - 1) / words_per_block, a.H);
    if (launches)
        *launches += 1;
    return launch_pdl(k_screen_joint, grid, dim3(32 * kJointWarps), st, a);
}

}  // namespace scr
