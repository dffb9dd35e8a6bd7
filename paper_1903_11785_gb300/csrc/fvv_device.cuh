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

// Approximate reciprocal (PTX rcp.approx.ftz.f32: at most 1 ulp of error).
__device__ __forceinline__ float rcp_approx(float w) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(w));
    return r;
}

// floor(x / w) of the exact quotient, clamped to [-1, n] (w > 0, n < 2^22):
// k0 = trunc(clamp(x * rcp(w), 0, n)) is within one of the answer whenever
// the answer is in [0, n]; the signs of the residuals x - k0 w and
// x - (k0 + 1) w, each formed by one FMA and so exact in sign, move it to
// the answer (or out of [0, n) when the quotient is outside).  No branch and
// no conversion instruction: the integer part is taken by a round-toward-zero
// add of 2^23.
__device__ __forceinline__ int pixel_floor(float x, float w, float r, float n) {
    const float q = fminf(fmaxf(fmul(x, r), 0.0f), n);
    const float t = __fadd_rz(q, 8388608.0f);   // 2^23 + trunc(q)
    const float k0 = fsub(t, 8388608.0f);
    const float r0 = __fmaf_rn(-k0, w, x);
    const float r1 = __fmaf_rn(-fadd(k0, 1.0f), w, x);
    return (__float_as_int(t) - 0x4B000000) - (r0 < 0.0f ? 1 : 0) + (r1 >= 0.0f ? 1 : 0);
}

// One camera's vote for a world point (Sec. II-B-1: project the voxel onto
// the silhouette): 1 foreground, 0 background, -1 abstain.  The pixel is
// (floor(x'/w'), floor(y'/w')) of the exact quotients of the binary32
// homogeneous coordinates; a point behind the camera or outside the image
// votes background under FVV_OOB_STRICT and abstains otherwise.
__device__ __forceinline__ int cam_vote(const Cam& c, int oob, const uint32_t* __restrict__ sil, float X,
                                        float Y, float Z) {
    float xp, yp, wp;
    project(c.P, X, Y, Z, xp, yp, wp);
    const float r = rcp_approx(wp);
    const int px = pixel_floor(xp, wp, r, c.Wf);
    const int py = pixel_floor(yp, wp, r, c.Hf);
    const bool in = wp > 0.0f && px >= 0 && px < c.W && py >= 0 && py < c.H;
    const unsigned ix = in ? (unsigned)px : 0u, iy = in ? (unsigned)py : 0u;
    const uint32_t word = in ? __ldg(sil + c.bit_off + iy * (unsigned)c.Wq + (ix >> 5)) : 0u;
    const int off = oob == FVV_OOB_ABSTAIN ? -1 : 0;
    return in ? (int)((word >> (ix & 31)) & 1u) : off;
}

// The pixel a point falls in for camera c, or -1 in px/py if none (behind the
// camera or outside the image).  Same arithmetic as cam_vote.
__device__ __forceinline__ void cam_pixel(const Cam& c, float X, float Y, float Z, int& px, int& py) {
    float xp, yp, wp;
    project(c.P, X, Y, Z, xp, yp, wp);
    const float r = rcp_approx(wp);
    px = pixel_floor(xp, wp, r, c.Wf);
    py = pixel_floor(yp, wp, r, c.Hf);
    if (!(wp > 0.0f && px >= 0 && px < c.W && py >= 0 && py < c.H)) px = py = -1;
}

// Occupancy of the 32 points of a warp (one per lane; lanes with alive ==
// false take no part), cameras in index order, each lane stopping at its
// first background vote and the warp stopping when no lane is left; `tests`
// counts each lane's camera tests.  All 32 lanes must call it together.
// NC > 0 unrolls the camera loop for NC cameras, so the camera matrices are
// read as constant-bank operands instead of indexed constant loads.
template <int NC>
__device__ __forceinline__ bool warp_test(const CamSet& cams, const uint32_t* __restrict__ sil, float X, float Y,
                                          float Z, bool alive, uint32_t& tests) {
    bool voted = false;
    if constexpr (NC > 0) {
#pragma unroll
        for (int n = 0; n < NC; ++n) {
            if (!__any_sync(kFull, alive)) break;
            if (alive) {
                ++tests;
                const int v = cam_vote(cams.c[n], cams.oob, sil, X, Y, Z);
                alive = v != 0;
                voted |= (v == 1);
            }
        }
    } else {
        for (int n = 0; n < cams.n; ++n) {
            if (!__any_sync(kFull, alive)) break;
            if (alive) {
                ++tests;
                const int v = cam_vote(cams.c[n], cams.oob, sil, X, Y, Z);
                alive = v != 0;
                voted |= (v == 1);
            }
        }
    }
    return alive && voted;
}

// Camera counts with an unrolled instantiation of the hull-test kernels
// (anything else runs the generic loop).
#define FVV_DISPATCH_NC(n, F)   \
    switch (n) {                \
        case 4: F(4); break;    \
        case 6: F(6); break;    \
        case 8: F(8); break;    \
        case 10: F(10); break;  \
        case 12: F(12); break;  \
        case 16: F(16); break;  \
        default: F(0); break;   \
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

// The ROI holding fine word w: the last ROI whose first word is <= w.
__device__ __forceinline__ int roi_of_word(const DRoi* rois, int n, uint32_t w) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rois[mid].word_off <= w) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Position of fine word w in its ROI's padded grid, with the ROI fields the
// kernels need kept in registers; a new ROI is looked up only when w leaves
// the current one (grid-stride loops visit words in increasing order).
struct RoiCursor {
    int k = -1;
    uint32_t lo = 0, hi = 0;
    int fdim[3];
    int nxw;
    float fo[3];
    // word position
    int wx, yp, zp;

    __device__ __forceinline__ void seek(const DRoi* rois, int n, uint32_t w) {
        if (w >= hi || w < lo) {
            k = roi_of_word(rois, n, w);
            const DRoi& r = rois[k];
            lo = r.word_off;
            hi = lo + r.n_words;
            nxw = r.nxw;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                fdim[a] = r.fdim[a];
                fo[a] = r.fo[a];
            }
        }
        const uint32_t lw = w - lo;
        const uint32_t row = lw / (uint32_t)nxw;
        wx = (int)(lw - row * (uint32_t)nxw);
        yp = (int)(row % (uint32_t)(fdim[1] + 2));
        zp = (int)(row / (uint32_t)(fdim[1] + 2));
    }
};

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

// 64-bit version of block_exclusive_scan; `sh` needs 33 entries.
__device__ __forceinline__ unsigned long long block_exclusive_scan64(unsigned long long v, unsigned long long* sh,
                                                                     unsigned long long& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const unsigned long long s = lane < nw ? sh[lane] : 0ull;
        unsigned long long t = s;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, t, o);
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
