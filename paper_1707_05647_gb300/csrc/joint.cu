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

// Is the candidate at element e of the tables (area `ar`) in set `st`?
__device__ __forceinline__ bool member(const JointArgs &a, const JointArea &ar, const JointSet &st, int64_t e) {
    const uint32_t *L1 = a.L1 + e, *T1 = a.T1 + e;
    const uint32_t S = sum8(L1, T1, ar.oL, ar.oT);
    if (S - ar.S_lo > ar.S_rng)   // its mean cell is outside the set's range (exact)
        return false;
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
        const uint32_t Si = sum8(L1, T1, ar.oLi, ar.oTi);
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

constexpr int kJointWarps = 8;
constexpr int kJointWPW = 2;   // mask words per warp

__global__ void __launch_bounds__(32 * kJointWarps) k_screen_joint(const JointArgs a) {
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * kJointWarps + (threadIdx.x >> 5)) * kJointWPW;
    const int y = blockIdx.y;
    if (w0 >= a.Wwords)
        return;
    const int64_t plane = (int64_t)a.H * a.Wwords;
    const int64_t row = (int64_t)y * a.pitch + kColOffset;
#pragma unroll 1
    for (int s = 0; s < a.n_scales; ++s) {
        const JointScale sc = a.scales[s];
        const bool row_ok = !sc.empty && y >= sc.y_lo && y <= sc.y_hi;
        uint32_t mine = 0;
#pragma unroll
        for (int j = 0; j < kJointWPW; ++j) {
            const int x = (w0 + j) * 32 + lane;
            bool pass = row_ok && x >= sc.x_lo && x <= sc.x_hi;
            for (int ar = 0; ar < a.n_areas && pass; ++ar)
                pass = member(a, a.areas[s * a.n_areas + ar], a.sets[ar], row + x);
            const uint32_t bits = __ballot_sync(0xffffffffu, pass);
            mine = lane == j ? bits : mine;
        }
        if (lane < kJointWPW && w0 + lane < a.Wwords)
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
