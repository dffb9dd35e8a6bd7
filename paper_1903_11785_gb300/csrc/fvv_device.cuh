// fvv_device.cuh -- device helpers shared by the kernels of libfvv: the
// silhouette predicate of Sec. II-B-1 and small warp/block reductions.
//
// All floating point uses the explicit round-to-nearest intrinsics
// (__fmul_rn, __fadd_rn, __fdiv_rn, __fsqrt_rn), which the compiler never
// fuses into an FMA, and explicit __fmaf_rn where a fused step is meant, so
// every result has one fixed binary32 value.
#pragma once

#include "fvv_internal.h"

namespace fvv {

constexpr unsigned kFull = 0xFFFFFFFFu;

// Programmatic dependent launch.  The kernels of a call are launched with
// launch_pdl, so that a kernel's blocks can be scheduled while the kernel
// before it in the stream is still finishing.  Every such kernel calls
// pdl_begin() first: it waits until the kernel before it has completed and
// its memory is visible (a no-op when the kernel was launched without the
// attribute), then lets the kernel after it be scheduled.
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }

// (x', y', w') = P (X, Y, Z, 1), each row evaluated as ((p3 + p2 Z) + p1 Y) + p0 X
// with three fused multiply-adds (one rounding per step).
__device__ __forceinline__ void project(const float* p, float X, float Y, float Z, float& xp, float& yp,
                                        float& wp) {
    xp = __fmaf_rn(p[0], X, __fmaf_rn(p[1], Y, __fmaf_rn(p[2], Z, p[3])));
    yp = __fmaf_rn(p[4], X, __fmaf_rn(p[5], Y, __fmaf_rn(p[6], Z, p[7])));
    wp = __fmaf_rn(p[8], X, __fmaf_rn(p[9], Y, __fmaf_rn(p[10], Z, p[11])));
}

// Approximate reciprocal (PTX rcp.approx.ftz.f32: at most 1 ulp of error).
__device__ __forceinline__ float rcp_approx(float w) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(w));
    return r;
}

// floor(x / w) of the exact quotient, clamped to [-1, n + 1] (w > 0,
// n < 2^22): k0 = trunc(clamp(x * rcp(w), 0, n)) is within one of the answer
// whenever the answer is in [0, n]; the residual r0 = x - k0 w, formed by one
// FMA, is exact when |r0| < w and rounds monotonically otherwise, so r0 < 0
// means k0 is one too big and r0 >= w means one too small (or the quotient
// is outside [0, n), which the result then shows).  No branch and no
// conversion instruction: the integer part comes from a round-toward-zero
// add of 2^23.
__device__ __forceinline__ int pixel_floor(float x, float w, float r, float n) {
    const float q = fminf(fmaxf(fmul(x, r), 0.0f), n);
    const float t = __fadd_rz(q, 8388608.0f);   // 2^23 + trunc(q)
    const float k0 = fsub(t, 8388608.0f);
    const float r0 = __fmaf_rn(-k0, w, x);
    return (__float_as_int(t) - 0x4B000000) - (r0 < 0.0f ? 1 : 0) + (r0 >= w ? 1 : 0);
}

// Silhouette bit of camera c at the pixel holding world point (X,Y,Z)
// (Sec. II-B-1: project the voxel onto the silhouette): the pixel is
// (floor(x'/w'), floor(y'/w')) of the exact quotients of the binary32
// homogeneous coordinates.  `in` says whether the point is in front of the
// camera and inside its image; the bit is 0 when it is not.
template <class CamT>
__device__ __forceinline__ uint32_t cam_bit(const CamT& c, const uint32_t* __restrict__ sil, float X, float Y,
                                            float Z, bool& in) {
    float xp, yp, wp;
    project(c.P, X, Y, Z, xp, yp, wp);
    const float r = rcp_approx(wp);
    const int px = pixel_floor(xp, wp, r, c.Wf);
    const int py = pixel_floor(yp, wp, r, c.Hf);
    in = wp > 0.0f && (unsigned)px < (unsigned)c.W && (unsigned)py < (unsigned)c.H;
    const uint32_t word = in ? __ldg(sil + c.bit_off + (unsigned)py * (unsigned)c.Wq + ((unsigned)px >> 5)) : 0u;
    return (word >> (px & 31)) & 1u;
}

// The pixel a point falls in for camera c, or -1 in px/py if none (behind the
// camera or outside the image).  Same arithmetic as cam_bit.
__device__ __forceinline__ void cam_pixel(const Cam& c, float X, float Y, float Z, int& px, int& py) {
    float xp, yp, wp;
    project(c.P, X, Y, Z, xp, yp, wp);
    const float r = rcp_approx(wp);
    px = pixel_floor(xp, wp, r, c.Wf);
    py = pixel_floor(yp, wp, r, c.Hf);
    if (!(wp > 0.0f && (unsigned)px < (unsigned)c.W && (unsigned)py < (unsigned)c.H)) px = py = -1;
}

// One camera's test of a live lane.  STRICT: a camera that does not see the
// point votes background, so the lane stays alive only on a foreground bit.
// ABSTAIN: such a camera does not vote; the lane must see one foreground vote.
template <bool ABSTAIN>
__device__ __forceinline__ void test_cam(const Cam& c, const uint32_t* __restrict__ sil, float X, float Y, float Z,
                                         bool& alive, bool& voted) {
    bool in;
    const uint32_t bit = cam_bit(c, sil, X, Y, Z, in);
    if constexpr (ABSTAIN) {
        alive = !in || bit;
        voted |= in && bit;
    } else {
        alive = bit != 0u;
    }
}

template <int NC, bool ABSTAIN>
__device__ __forceinline__ bool warp_test_p(const CamSet& cams, const uint32_t* __restrict__ sil, float X, float Y,
                                            float Z, bool alive, uint32_t& tests) {
    bool voted = !ABSTAIN;
    if constexpr (NC > 0) {
#pragma unroll
        for (int n = 0; n < NC; ++n) {
            if (!__any_sync(kFull, alive)) break;
            if (alive) {
                ++tests;
                test_cam<ABSTAIN>(cams.c[n], sil, X, Y, Z, alive, voted);
            }
        }
    } else {
        for (int n = 0; n < cams.n; ++n) {
            if (!__any_sync(kFull, alive)) break;
            if (alive) {
                ++tests;
                test_cam<ABSTAIN>(cams.c[n], sil, X, Y, Z, alive, voted);
            }
        }
    }
    return alive && voted;
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
    return cams.oob == FVV_OOB_ABSTAIN ? warp_test_p<NC, true>(cams, sil, X, Y, Z, alive, tests)
                                       : warp_test_p<NC, false>(cams, sil, X, Y, Z, alive, tests);
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

// A camera's fields for tests where lanes use different cameras, kept in
// shared memory (80 bytes: consecutive cameras fall in different banks).
struct __align__(16) SmemCam {
    float P[12];
    float Wf, Hf;
    int W, H, Wq;
    uint32_t bit_off;
    float du, dv;            // Cam::seg_du, seg_dv
};

// Copy the first n cameras into sc (all threads of the block; the caller
// synchronises).
__device__ __forceinline__ void load_smem_cams(const CamSet& cams, int n, SmemCam* sc) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const Cam& c = cams.c[i];
        for (int k = 0; k < 12; ++k) sc[i].P[k] = c.P[k];
        sc[i].Wf = c.Wf;
        sc[i].Hf = c.Hf;
        sc[i].W = c.W;
        sc[i].H = c.H;
        sc[i].Wq = c.Wq;
        sc[i].bit_off = c.bit_off;
        sc[i].du = c.seg_du;
        sc[i].dv = c.seg_dv;
    }
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
