// probe.cu -- micro-benchmarks behind the rooflines (no counterpart in the
// paper).  An FP32 fused multiply-add loop gives the arithmetic ceiling of
// the hull and depth kernels, whose camera tests and triangle set-ups are
// chains of binary32 fused multiply-adds on the plain ALUs.  Two L2 probes
// give the memory side of the hull tests' roofline: a coalesced read of an
// L2-resident buffer and a random gather of 32-bit words from one.  A camera
// test gathers one 32-bit silhouette word (Sec. II-B-1 reads one silhouette
// pixel per projection), so the gather rate measured here is the rate of
// camera tests that L2 alone could feed.  Both read with ld.global.cg (cached
// in L2, not in L1).
#include <cuda_runtime.h>

#include "fvv.h"

namespace {

__global__ void k_probe_read(const uint4* __restrict__ buf, size_t n16, int reps, uint32_t* out) {
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    uint32_t acc = 0;
    for (int r = 0; r < reps; ++r)
        for (size_t i = tid; i < n16; i += stride) {
            const uint4 v = __ldcg(buf + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    out[tid] = acc;
}

// Word index of gather i of thread t: a 32-bit integer hash (multiply and
// xor-shift) of (t, i), masked to the buffer.
__device__ __forceinline__ uint32_t probe_index(uint32_t t, uint32_t i, uint32_t mask) {
    uint32_t x = t * 0x9E3779B9u + i * 0x85EBCA6Bu;
    x ^= x >> 16;
    x *= 0x7FEB352Du;
    x ^= x >> 15;
    return x & mask;
}

__global__ void k_probe_gather(const uint32_t* __restrict__ buf, uint32_t mask, int reps, uint32_t* out) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    int i = 0;
    for (; i + 4 <= reps; i += 4) {
        const uint32_t a = __ldcg(buf + probe_index(tid, i, mask));
        const uint32_t b = __ldcg(buf + probe_index(tid, i + 1, mask));
        const uint32_t c = __ldcg(buf + probe_index(tid, i + 2, mask));
        const uint32_t d = __ldcg(buf + probe_index(tid, i + 3, mask));
        acc ^= a ^ b ^ c ^ d;
    }
    for (; i < reps; ++i) acc ^= __ldcg(buf + probe_index(tid, i, mask));
    out[tid] = acc;
}

// kFmaChains independent chains x = fma(x, a, b) per thread, `reps` steps
// each; a and b come in as parameters so nothing is folded at compile time.
constexpr int kFmaChains = 16;
__global__ void k_probe_fma(int reps, float a, float b, float* out) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    float x[kFmaChains];
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) x[k] = (float)((tid + (uint32_t)k) & 7u);
    for (int r = 0; r < reps; ++r) {
#pragma unroll
        for (int k = 0; k < kFmaChains; ++k) x[k] = __fmaf_rn(x[k], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) s = __fadd_rn(s, x[k]);
    out[tid] = s;
}

}  // namespace

extern "C" fvv_status fvv_probe_fma(int reps, float a, float b, float* out, int blocks, int threads, void* stream) {
    if (!out || reps < 1 || blocks < 1 || threads < 32 || threads > 1024 || threads % 32) return FVV_ERR_INVALID_ARG;
    if ((unsigned long long)blocks * threads > 0xFFFFFFFFull) return FVV_ERR_INVALID_ARG;
    k_probe_fma<<<blocks, threads, 0, (cudaStream_t)stream>>>(reps, a, b, out);
    return cudaGetLastError() == cudaSuccess ? FVV_OK : FVV_ERR_CUDA;
}

extern "C" fvv_status fvv_probe_l2(int mode, const void* buf, size_t bytes, int reps, uint32_t* out, int blocks,
                                   int threads, void* stream) {
    if (!buf || !out || reps < 1 || blocks < 1 || threads < 32 || threads > 1024 || threads % 32)
        return FVV_ERR_INVALID_ARG;
    const cudaStream_t st = (cudaStream_t)stream;
    if (mode == 0) {
        if (bytes < 16 || bytes % 16 || (uintptr_t)buf % 16) return FVV_ERR_INVALID_ARG;
        k_probe_read<<<blocks, threads, 0, st>>>((const uint4*)buf, bytes / 16, reps, out);
    } else if (mode == 1) {
        const size_t words = bytes / 4;
        if (bytes % 4 || words < 1 || words > (1ull << 31) || (words & (words - 1)) || (uintptr_t)buf % 4)
            return FVV_ERR_INVALID_ARG;
        if ((unsigned long long)blocks * threads > 0xFFFFFFFFull) return FVV_ERR_INVALID_ARG;
        k_probe_gather<<<blocks, threads, 0, st>>>((const uint32_t*)buf, (uint32_t)(words - 1), reps, out);
    } else {
        return FVV_ERR_INVALID_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? FVV_OK : FVV_ERR_CUDA;
}
