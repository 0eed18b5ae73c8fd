// Load-throughput probe behind the screening kernel's on-chip roofline: how
// many warp instructions per clock per SM the L1 data pipe sustains for the
// load shapes a corner read can take (32-bit coalesced, 128-byte aligned or
// not; 64- and 128-bit vectors), for warp shuffles and shared-memory loads,
// and for pairs of them issued together (whether they share the pipe).  Each
// kernel's warps read 8 loads per iteration from a small region (L1-resident)
// or a 32 MB region (mostly L2-served).  Two further kernels read through a
// texture object (tex1Dfetch) instead, alone and mixed with global loads, to
// see whether the texture input path of L1TEX adds bandwidth next to the load
// path.  Not part of libscreen.so: bench.py --workload l1probe builds and runs
// it and prints one JSON line.
// Every kernel reads only inside buf[0 .. words + PAD): the largest index read
// is off + 1027 with off <= words - 32 (see each load's comment).
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <vector>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e_), __LINE__); exit(1);} } while (0)

constexpr uint32_t PAD = 4096;   // words of slack after the power-of-two region

template <int M>
__global__ void __launch_bounds__(256) probe(const uint32_t *__restrict__ buf, cudaTextureObject_t tx,
                                             uint32_t wmask, int iters, uint32_t *out) {
    __shared__ uint32_t sm[2048 + 64];
    const int lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (M == 6 || M == 7) {
        for (int i = threadIdx.x; i < 2048 + 64; i += blockDim.x) sm[i] = buf[i] + i;
        __syncthreads();
    }
    uint32_t acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = lane + j;
    const uint32_t base = gw * 1024u;
    for (int it = 0; it < iters; ++it) {
        const uint32_t off = (base + (uint32_t)it * 288u) & wmask & ~31u;   // <= wmask - 31
        if (M == 0) {            // 8 coalesced 32-bit loads, start 1 word past a 128-B line
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] += __ldg(buf + off + 1 + lane + 32 * j);   // max off+1+31+224 < off+257
        } else if (M == 1) {     // 8 coalesced 32-bit loads, 128-B aligned
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] += __ldg(buf + off + lane + 32 * j);
        } else if (M == 2) {     // 8 coalesced 128-bit loads, aligned (512 B per warp each)
            const uint4 *b4 = reinterpret_cast<const uint4 *>(buf + off);
#pragma unroll
            for (int j = 0; j < 8; ++j) {   // words off + 4*(lane + 32 j) + 3 < off + 1024
                const uint4 v = __ldg(b4 + lane + 32 * j);
                acc[j] += v.x + v.y;
                acc[(j + 1) & 7] += v.z + v.w;
            }
        } else if (M == 3) {     // 8 warp shuffles
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] += __shfl_sync(0xffffffffu, acc[j] + it, (lane + j + 1) & 31);
        } else if (M == 4) {     // 8 LDG.128 + 8 shuffles
            const uint4 *b4 = reinterpret_cast<const uint4 *>(buf + off);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint4 v = __ldg(b4 + lane + 32 * j);
                const uint32_t s = __shfl_down_sync(0xffffffffu, v.x, 1);
                acc[j] += v.y + s;
                acc[(j + 1) & 7] += v.z + v.w;
            }
        } else if (M == 5) {     // 8 misaligned 32-bit loads + 8 shuffles
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t v = __ldg(buf + off + 1 + lane + 32 * j);
                acc[j] += v + __shfl_down_sync(0xffffffffu, v, 1);
            }
        } else if (M == 6) {     // 8 shared-memory 32-bit loads, misaligned start
            const uint32_t so = off & 1023u;   // so + 1 + 31 + 224 < 1280 <= 2048
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] += sm[so + 1 + lane + 32 * j];
        } else if (M == 7) {     // 8 LDS + 8 LDG misaligned
            const uint32_t so = off & 1023u;
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] += sm[so + 1 + lane + 32 * j] + __ldg(buf + off + 1 + lane + 32 * j);
        } else if (M == 8) {     // 8 coalesced 64-bit loads, aligned
            const uint2 *b2 = reinterpret_cast<const uint2 *>(buf + off);
#pragma unroll
            for (int j = 0; j < 8; ++j) {   // words off + 2*(lane+32j)+1 < off + 512
                const uint2 v = __ldg(b2 + lane + 32 * j);
                acc[j] += v.x + v.y;
            }
        } else if (M == 10) {    // 8 texture fetches, start 1 word past a 128-B line
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] += tex1Dfetch<unsigned int>(tx, (int)(off + 1 + lane + 32 * j));
        } else if (M == 11) {    // 8 texture fetches + 8 misaligned 32-bit loads of other words
#pragma unroll
            for (int j = 0; j < 8; ++j)   // largest index off + 513 + 31 + 224 < off + 1027
                acc[j] += tex1Dfetch<unsigned int>(tx, (int)(off + 1 + lane + 32 * j)) +
                          __ldg(buf + off + 513 + lane + 32 * j);
        } else if (M == 9) {     // 8 LDG.128 shifted by 16 B (16-B aligned, not line aligned)
            const uint4 *b4 = reinterpret_cast<const uint4 *>(buf + off + 4);
#pragma unroll
            for (int j = 0; j < 8; ++j) {   // < off + 4 + 1024
                const uint4 v = __ldg(b4 + lane + 32 * j);
                acc[j] += v.x + v.y;
                acc[(j + 1) & 7] += v.z + v.w;
            }
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) r += acc[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

template <int M>
float run(const uint32_t *buf, cudaTextureObject_t tx, uint32_t wmask, int iters, uint32_t *out, int blocks) {
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    probe<M><<<blocks, 256>>>(buf, tx, wmask, iters, out);
    CK(cudaGetLastError());
    CK(cudaEventRecord(a));
    for (int r = 0; r < 3; ++r) probe<M><<<blocks, 256>>>(buf, tx, wmask, iters, out);
    CK(cudaEventRecord(b));
    CK(cudaEventSynchronize(b));
    float ms;
    CK(cudaEventElapsedTime(&ms, a, b));
    return ms / 3;
}

int main() {
    int dev = 0, sms = 0, clk = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev));
    const uint32_t regions[2] = {1u << 13, 1u << 23};   // 32 KB (L1-resident), 32 MB (L2-served)
    const uint32_t maxw = (1u << 23) + PAD;
    uint32_t *buf, *out;
    CK(cudaMalloc(&buf, maxw * 4ull));
    CK(cudaMemset(buf, 1, maxw * 4ull));
    // a texture object over the same words (out-of-range fetches return 0)
    cudaResourceDesc rd = {};
    rd.resType = cudaResourceTypeLinear;
    rd.res.linear.devPtr = buf;
    rd.res.linear.desc = cudaCreateChannelDesc<unsigned int>();
    rd.res.linear.sizeInBytes = maxw * 4ull;
    cudaTextureDesc td = {};
    td.readMode = cudaReadModeElementType;
    cudaTextureObject_t tx;
    CK(cudaCreateTextureObject(&tx, &rd, &td, nullptr));
    const int blocks = sms * 8;
    CK(cudaMalloc(&out, blocks * 256 * 4ull));
    const int iters = 2000;
    const char *names[] = {"ldg32_misaligned", "ldg32_aligned", "ldg128_aligned", "shfl",
                           "ldg128_plus_shfl", "ldg32_misaligned_plus_shfl", "lds32_misaligned",
                           "lds32_plus_ldg32_misaligned", "ldg64_aligned", "ldg128_at_16B", "tex32_misaligned",
                           "tex32_plus_ldg32_misaligned"};
    printf("{\"sms\": %d, \"max_clock_mhz\": %.0f, \"unit\": \"warp instructions of each kind per clock per SM "
           "(at the maximum clock)\"", sms, clk / 1e3);
    for (uint32_t region : regions) {
        const uint32_t wmask = region - 1;
        float t[12];
        t[0] = run<0>(buf, tx, wmask, iters, out, blocks);
        t[1] = run<1>(buf, tx, wmask, iters, out, blocks);
        t[2] = run<2>(buf, tx, wmask, iters, out, blocks);
        t[3] = run<3>(buf, tx, wmask, iters, out, blocks);
        t[4] = run<4>(buf, tx, wmask, iters, out, blocks);
        t[5] = run<5>(buf, tx, wmask, iters, out, blocks);
        t[6] = run<6>(buf, tx, wmask, iters, out, blocks);
        t[7] = run<7>(buf, tx, wmask, iters, out, blocks);
        t[8] = run<8>(buf, tx, wmask, iters, out, blocks);
        t[9] = run<9>(buf, tx, wmask, iters, out, blocks);
        t[10] = run<10>(buf, tx, wmask, iters, out, blocks);
        t[11] = run<11>(buf, tx, wmask, iters, out, blocks);
        const double warps = blocks * 8.0;
        printf(", \"%s\": {", region < (1u << 20) ? "l1_resident_32KB" : "l2_served_32MB");
        for (int m = 0; m < 12; ++m) {
            const double per = warps * iters * 8.0 / sms / (t[m] * 1e-3 * clk * 1e3);
            printf("%s\"%s\": %.3f", m ? ", " : "", names[m], per);
        }
        printf("}");
    }
    printf("}\n");
    CK(cudaDestroyTextureObject(tx));
    CK(cudaFree(buf));
    CK(cudaFree(out));
    return 0;
}
