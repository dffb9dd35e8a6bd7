// fvv_device.cuh -- device helpers shared by the kernels of libfvv: the
// silhouette predicate of Sec. II-B-1 and small warp/block reductions.
//
// All floating point uses the explicit round-to-nearest intrinsics
// (__fmul_rn, __fadd_rn, __fdiv_rn, __fsqrt_rn), which the compiler never
// fuses into an FMA, so every result has one fixed binary32 value.
#pragma once

#include "fvv_internal.h"

namespace fvv {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }

// (x', y', w') = P (X, Y, Z, 1), each row evaluated as ((p0 X + p1 Y) + p2 Z) + p3.
__device__ __forceinline__ void project(const float* p, float X, float Y, float Z, float& xp, float& yp,
                                        float& wp) {
    xp = fadd(fadd(fadd(fmul(p[0], X), fmul(p[1], Y)), fmul(p[2], Z)), p[3]);
    yp = fadd(fadd(fadd(fmul(p[4], X), fmul(p[5], Y)), fmul(p[6], Z)), p[7]);
    wp = fadd(fadd(fadd(fmul(p[8], X), fmul(p[9], Y)), fmul(p[10], Z)), p[11]);
}

// One camera's vote for a world point (Sec. II-B-1: project the voxel onto
// the silhouette): 1 foreground, 0 background, -1 abstain.  The pixel is
// (floor(x'/w'), floor(y'/w')); a point behind the camera or outside the
// image votes background under FVV_OOB_STRICT and abstains otherwise.
__device__ __forceinline__ int cam_vote(const Cam& c, int oob, const uint32_t* __restrict__ sil, float X,
                                        float Y, float Z) {
    float xp, yp, wp;
    project(c.P, X, Y, Z, xp, yp, wp);
    const int off = oob == FVV_OOB_ABSTAIN ? -1 : 0;
    if (!(wp > 0.0f)) return off;
    const float fu = floorf(__fdiv_rn(xp, wp));
    const float fv = floorf(__fdiv_rn(yp, wp));
    if (!(fu >= 0.0f && fu < (float)c.W && fv >= 0.0f && fv < (float)c.H)) return off;
    const int px = (int)fu, py = (int)fv;
    const uint32_t w = __ldg(sil + c.bit_off + (size_t)py * (unsigned)c.Wq + (unsigned)(px >> 5));
    return (int)((w >> (px & 31)) & 1u);
}

// Occupancy of one point, cameras in index order with exit at the first
// background vote; `tests` counts the camera tests made.
__device__ __forceinline__ bool point_on(const CamSet& cams, const uint32_t* __restrict__ sil, float X,
                                         float Y, float Z, uint32_t& tests) {
    bool voted = false;
    for (int n = 0; n < cams.n; ++n) {
        ++tests;
        const int v = cam_vote(cams.c[n], cams.oob, sil, X, Y, Z);
        if (v == 0) return false;
        voted |= (v == 1);
    }
    return voted;
}

// Sum over the block (blockDim.x a multiple of 32, <= 1024); result valid in
// thread 0.  `sh` needs 32 entries.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    T s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    return s;
}

// Exclusive prefix over the block of one uint32 per thread; `total` gets the
// block sum in every thread.  `sh` needs 33 entries.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* sh, uint32_t& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < nw ? sh[lane] : 0u;
        uint32_t t = s;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) sh[lane] = t - s;
        if (lane == 31) sh[32] = t;
    }
    __syncthreads();
    total = sh[32];
    return sh[wid] + x - v;
}

}  // namespace fvv
