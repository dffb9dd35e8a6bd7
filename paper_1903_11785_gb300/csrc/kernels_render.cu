// kernels_render.cu -- Sec. II-D: per-camera depth images (Eq. (4)) and the
// per-vertex visibility test and colour choice of Sec. II-D-2 and II-E.
//
// Depth images hold the binary32 bits of the squared distance (non-negative,
// so the unsigned order of the bits is the order of the values) and are
// merged with atomicMin; 0xFFFFFFFF means no triangle covered the pixel
// (+infinity).  Readers take the square root.
#include "fvv_device.cuh"

namespace fvv {
namespace {

__global__ void __launch_bounds__(256) k_clear_depth(const __grid_constant__ Layout L,
                                                     const __grid_constant__ SlotList sl, size_t n16) {
    const int slot = sl.s[blockIdx.y];
    uint4* d = slot_ptr<uint4>(L, slot, L.depth);
    const uint4 v = make_uint4(kEmptyDepth, kEmptyDepth, kEmptyDepth, kEmptyDepth);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
        __stcs(d + i, v);
}

// Eq. (4) for one triangle (world vertices X, Y, Z, squared centroid-camera
// distance d2 as float bits) in camera c.  The triangle is skipped if a vertex
// is not in front of the camera (w' <= 0) or its projected area is zero; its
// value goes into each pixel whose centre p lies in the closed box of the
// projection and on the inner side of (or on) all three edges, either winding.
// Everything is decided on the homogeneous image points (x', y', w') without
// dividing: the edge function of edge (i, j) at p is (p_x a - p_y b) + c with
// a = y_i w_j - w_i y_j, b = x_i w_j - w_i x_j, c = x_i y_j - y_i x_j (its
// sign is the image-plane one for w > 0), the area is zero iff
// (x_0 a_12 - y_0 b_12) + w_0 c_12 is, and the box test uses the exact signs
// of p w_j - x_j from one FMA each.
// `sink(pixel)` is called for each covered pixel (row-major index in c's
// image).
template <class Sink>
__device__ __forceinline__ void raster_tri(const Cam& c, const float* X, const float* Y, const float* Z,
                                           Sink&& sink) {
    float xh[3], yh[3], wh[3];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        project(c.P, X[j], Y[j], Z[j], xh[j], yh[j], wh[j]);
        ok &= wh[j] > 0.0f;
    }
    if (!ok) return;
    // candidate pixels: centres within 1/64 px of the box of the approximate
    // projections (their error is below 1e-3 px for images up to 65535 px;
    // the exact box test below decides)
    float umin = 3.0e38f, umax = -3.0e38f, vmin = 3.0e38f, vmax = -3.0e38f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float r = rcp_approx(wh[j]);
        const float u = fmul(xh[j], r), v = fmul(yh[j], r);
        umin = fminf(umin, u); umax = fmaxf(umax, u);
        vmin = fminf(vmin, v); vmax = fmaxf(vmax, v);
    }
    constexpr float kSlack = 0.5f + 1.0f / 64.0f;
    if (!(umax >= 0.0f && vmax >= 0.0f && umin <= c.Wf && vmin <= c.Hf)) return;
    const int x0 = max(0, (int)ceilf(fsub(umin, kSlack)));
    const int y0 = max(0, (int)ceilf(fsub(vmin, kSlack)));
    const int x1 = umax > c.Wf ? c.W - 1 : min(c.W - 1, (int)floorf(fsub(fadd(umax, 1.0f / 64.0f), 0.5f)));
    const int y1 = vmax > c.Hf ? c.H - 1 : min(c.H - 1, (int)floorf(fsub(fadd(vmax, 1.0f / 64.0f), 0.5f)));
    if (x0 > x1 || y0 > y1) return;      // no pixel centre near the box
    // homogeneous edge functions of edges (0,1), (1,2), (2,0): no division
    float ea[3], eb[3], ec[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int i = e, j = (e + 1) % 3;
        ea[e] = fsub(fmul(yh[i], wh[j]), fmul(wh[i], yh[j]));
        eb[e] = fsub(fmul(xh[i], wh[j]), fmul(wh[i], xh[j]));
        ec[e] = fsub(fmul(xh[i], yh[j]), fmul(yh[i], xh[j]));
    }
    const float det = fadd(fsub(fmul(xh[0], ea[1]), fmul(yh[0], eb[1])), fmul(wh[0], ec[1]));
    if (!(det > 0.0f || det < 0.0f)) return;
    for (int yy = y0; yy <= y1; ++yy) {
        const float pcy = fadd((float)yy, 0.5f);
        const float s0 = __fmaf_rn(pcy, wh[0], -yh[0]), s1 = __fmaf_rn(pcy, wh[1], -yh[1]),
                    s2 = __fmaf_rn(pcy, wh[2], -yh[2]);
        if (!((s0 >= 0.0f || s1 >= 0.0f || s2 >= 0.0f) && (s0 <= 0.0f || s1 <= 0.0f || s2 <= 0.0f))) continue;
        for (int xx = x0; xx <= x1; ++xx) {
            const float pcx = fadd((float)xx, 0.5f);
            const float r0 = __fmaf_rn(pcx, wh[0], -xh[0]), r1 = __fmaf_rn(pcx, wh[1], -xh[1]),
                        r2 = __fmaf_rn(pcx, wh[2], -xh[2]);
            if (!((r0 >= 0.0f || r1 >= 0.0f || r2 >= 0.0f) && (r0 <= 0.0f || r1 <= 0.0f || r2 <= 0.0f))) continue;
            const float e0 = fadd(fsub(fmul(pcx, ea[0]), fmul(pcy, eb[0])), ec[0]);
            const float e1 = fadd(fsub(fmul(pcx, ea[1]), fmul(pcy, eb[1])), ec[1]);
            const float e2 = fadd(fsub(fmul(pcx, ea[2]), fmul(pcy, eb[2])), ec[2]);
            const bool in = (e0 >= 0.0f && e1 >= 0.0f && e2 >= 0.0f) || (e0 <= 0.0f && e1 <= 0.0f && e2 <= 0.0f);
            if (in) sink((size_t)yy * (unsigned)c.W + xx);
        }
    }
}

// Grid (blocks, cameras, slots): the camera is uniform over a block, so its
// matrix is read through uniform registers, and blocks are issued frame by
// frame, so one frame's depth images are worked on together.  One thread per
// triangle; the centroid ((v0 + v1) + v2) / 3 was formed once per triangle
// when the triangle was emitted.
__global__ void __launch_bounds__(256) k_zbuffer(const __grid_constant__ CamSet cams, const __grid_constant__ Layout L,
                                                 const __grid_constant__ SlotList sl) {
    const int slot = sl.s[blockIdx.z];
    const Cam& c = cams.c[blockIdx.y];
    const SlotInfo* info = slot_ptr<SlotInfo>(L, slot, L.info);
    const uint32_t nt = info->n_words ? info->n_tris : 0u;
    const float* verts = slot_ptr<float>(L, slot, L.verts);
    const uint32_t* tris = slot_ptr<uint32_t>(L, slot, L.tris);
    const float* tcen = slot_ptr<float>(L, slot, L.tcen);
    uint32_t* depth = slot_ptr<uint32_t>(L, slot, L.depth);
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        float X[3], Y[3], Z[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const uint32_t vi = __ldg(tris + 3 * (size_t)t + j);
            X[j] = __ldg(verts + 3 * (size_t)vi);
            Y[j] = __ldg(verts + 3 * (size_t)vi + 1);
            Z[j] = __ldg(verts + 3 * (size_t)vi + 2);
        }
        const float dx = fsub(__ldg(tcen + 3 * (size_t)t), c.C[0]);
        const float dy = fsub(__ldg(tcen + 3 * (size_t)t + 1), c.C[1]);
        const float dz = fsub(__ldg(tcen + 3 * (size_t)t + 2), c.C[2]);
        const uint32_t d2 = __float_as_uint(fadd(fadd(fmul(dx, dx), fmul(dy, dy)), fmul(dz, dz)));
        // the buffer keeps the minimum of the squared distance: sqrt is
        // monotone, so the square root of that minimum is the minimum
        // distance itself, taken where the depth is read
        uint32_t* D = depth + c.pix_off;
        raster_tri(c, X, Y, Z, [&](size_t pix) {
            uint32_t* p = D + pix;
            if (__ldcg(p) > d2) atomicMin(p, d2);   // skip the atomic when already nearer
        });
    }
}

// Stored squared distance -> distance (+infinity for an empty pixel).
__device__ __forceinline__ float depth_of(uint32_t bits) {
    return bits == kEmptyDepth ? __int_as_float(0x7f800000) : __fsqrt_rn(__uint_as_float(bits));
}

// Sec. II-D-2 and II-E: the capture cameras ranked by squared distance of
// their centre to the viewpoint vp, ties to the lower index (thread m <
// cams.n places camera m; the caller synchronises).
__device__ __forceinline__ void rank_cameras(const CamSet& cams, const float* vp, int* rank_cam) {
    if (threadIdx.x < (unsigned)cams.n) {
        float d2[FVV_MAX_CAMS];
        const int me = threadIdx.x;
        int r = 0;
        for (int m = 0; m < cams.n; ++m) {
            const float ax = fsub(cams.c[m].C[0], vp[0]), ay = fsub(cams.c[m].C[1], vp[1]),
                        az = fsub(cams.c[m].C[2], vp[2]);
            d2[m] = fadd(fadd(fmul(ax, ax), fmul(ay, ay)), fmul(az, az));
        }
        for (int m = 0; m < cams.n; ++m) r += (d2[m] < d2[me]) || (d2[m] == d2[me] && m < me);
        rank_cam[r] = me;
    }
}

// The colour of world point (X,Y,Z): the first camera in rank order that has
// it in front, inside the image and with |X - C| - depth <= t_v, and that
// camera's RGB at the point's pixel.  Returns the camera, or -1 with (0,0,0).
__device__ __forceinline__ int colour_point(const CamSet& cams, const int* rank_cam,
                                            const uint32_t* __restrict__ depth, const uint8_t* const* rgb, float t_v,
                                            float X, float Y, float Z, uint8_t* col) {
    col[0] = col[1] = col[2] = 0;
    for (int k = 0; k < cams.n; ++k) {
        const int n = rank_cam[k];
        const Cam& c = cams.c[n];
        int px, py;
        cam_pixel(c, X, Y, Z, px, py);
        if (px < 0) continue;
        const size_t pix = (size_t)py * (unsigned)c.W + (size_t)px;
        const float dx = fsub(X, c.C[0]), dy = fsub(Y, c.C[1]), dz = fsub(Z, c.C[2]);
        const float dist = __fsqrt_rn(fadd(fadd(fmul(dx, dx), fmul(dy, dy)), fmul(dz, dz)));
        const float dep = depth_of(__ldg(depth + c.pix_off + pix));
        if (!(fsub(dist, dep) <= t_v)) continue;
        const uint8_t* src = rgb[n] + 3 * pix;
        col[0] = __ldg(src);
        col[1] = __ldg(src + 1);
        col[2] = __ldg(src + 2);
        return n;
    }
    return -1;
}

// Per vertex: colour_point with the cameras ranked for the slot's viewpoint.
__global__ void __launch_bounds__(256) k_colour(const __grid_constant__ CamSet cams, const __grid_constant__ Grid g,
                                                const __grid_constant__ Layout L,
                                                const __grid_constant__ ColourBatch cb) {
    __shared__ int rank_cam[FVV_MAX_CAMS];
    const int slot = cb.slot[blockIdx.y];
    rank_cameras(cams, cb.view[blockIdx.y], rank_cam);
    __syncthreads();
    const SlotInfo* info = slot_ptr<SlotInfo>(L, slot, L.info);
    const uint32_t nv = info->n_words ? info->n_verts : 0u;
    const float* verts = slot_ptr<float>(L, slot, L.verts);
    const uint32_t* depth = slot_ptr<uint32_t>(L, slot, L.depth);
    const uint8_t* const* rgb = cb.rgb[blockIdx.y];
    uint8_t* out = slot_ptr<uint8_t>(L, slot, L.vrgb);
    int* ocam = slot_ptr<int>(L, slot, L.vcam);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
        uint8_t col[3];
        const int chosen = colour_point(cams, rank_cam, depth, rgb, g.t_v, verts[3 * (size_t)i],
                                        verts[3 * (size_t)i + 1], verts[3 * (size_t)i + 2], col);
        out[3 * (size_t)i] = col[0];
        out[3 * (size_t)i + 1] = col[1];
        out[3 * (size_t)i + 2] = col[2];
        ocam[i] = chosen;
    }
}

// ---- Sec. II-E, step E: a novel view of the coloured mesh

__global__ void __launch_bounds__(256) k_view_clear(unsigned long long* __restrict__ key, size_t npix) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += (size_t)gridDim.x * blockDim.x)
        key[i] = ~0ull;
}

// Visibility in the virtual view: every covered pixel keeps the minimum of
// (squared distance from the triangle's centroid to the view centre, as float
// bits) << 32 | triangle index -- the nearest triangle, ties to the lower
// index.  One thread per triangle.
__global__ void __launch_bounds__(256) k_view_raster(const __grid_constant__ Layout L,
                                                     const __grid_constant__ ViewArgs va,
                                                     unsigned long long* __restrict__ key) {
    const Cam& v = va.v;
    const SlotInfo* info = slot_ptr<SlotInfo>(L, va.slot, L.info);
    const uint32_t nt = info->n_words ? info->n_tris : 0u;
    const float* verts = slot_ptr<float>(L, va.slot, L.verts);
    const uint32_t* tris = slot_ptr<uint32_t>(L, va.slot, L.tris);
    const float* tcen = slot_ptr<float>(L, va.slot, L.tcen);
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        float X[3], Y[3], Z[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const uint32_t vi = __ldg(tris + 3 * (size_t)t + j);
            X[j] = __ldg(verts + 3 * (size_t)vi);
            Y[j] = __ldg(verts + 3 * (size_t)vi + 1);
            Z[j] = __ldg(verts + 3 * (size_t)vi + 2);
        }
        const float dx = fsub(__ldg(tcen + 3 * (size_t)t), v.C[0]);
        const float dy = fsub(__ldg(tcen + 3 * (size_t)t + 1), v.C[1]);
        const float dz = fsub(__ldg(tcen + 3 * (size_t)t + 2), v.C[2]);
        const unsigned long long k =
            (unsigned long long)__float_as_uint(fadd(fadd(fmul(dx, dx), fmul(dy, dy)), fmul(dz, dz))) << 32 | t;
        raster_tri(v, X, Y, Z, [&](size_t pix) {
            unsigned long long* p = key + pix;
            if (__ldcg(p) > k) atomicMin(p, k);
        });
    }
}

// Colour of every pixel of the view: colour_point of its triangle's
// centroid, with the capture cameras ranked for the view centre, so the
// camera is chosen per pixel (Sec. II-E: the nearest camera where it sees
// the surface, its neighbours where it is occluded).
__global__ void __launch_bounds__(256) k_view_shade(const __grid_constant__ CamSet cams,
                                                    const __grid_constant__ Grid g, const __grid_constant__ Layout L,
                                                    const __grid_constant__ ViewArgs va,
                                                    const unsigned long long* __restrict__ key,
                                                    uint8_t* __restrict__ out_rgb, int32_t* __restrict__ out_cam) {
    __shared__ int rank_cam[FVV_MAX_CAMS];
    rank_cameras(cams, va.v.C, rank_cam);
    __syncthreads();
    const uint32_t* depth = slot_ptr<uint32_t>(L, va.slot, L.depth);
    const float* tcen = slot_ptr<float>(L, va.slot, L.tcen);
    const size_t npix = (size_t)va.v.W * (unsigned)va.v.H;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long k = key[i];
        uint8_t col[3] = {0, 0, 0};
        int chosen = -1;
        if (k != ~0ull) {
            const size_t t = (size_t)(uint32_t)k;
            chosen = colour_point(cams, rank_cam, depth, va.rgb, g.t_v, __ldg(tcen + 3 * t), __ldg(tcen + 3 * t + 1),
                                  __ldg(tcen + 3 * t + 2), col);
        }
        out_rgb[3 * i] = col[0];
        out_rgb[3 * i + 1] = col[1];
        out_rgb[3 * i + 2] = col[2];
        if (out_cam) out_cam[i] = chosen;
    }
}

__global__ void k_debug_depth(const __grid_constant__ Layout L, int slot, float* dst, size_t npix) {
    const uint32_t* d = slot_ptr<uint32_t>(L, slot, L.depth);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t b = d[i];
        dst[i] = depth_of(b);
    }
}

}  // namespace

cudaError_t launch_depth(const CamSet& cams, const Grid& g, const Layout& L, const SlotList& sl, int sms,
                         size_t depth_bytes, const Tuning& tu, cudaStream_t st) {
    const size_t n16 = depth_bytes / 16;
    const int gc = grid_x(sms, sl.n, (long long)n16, 256);
    k_clear_depth<<<dim3(gc, sl.n), 256, 0, st>>>(L, sl, n16);
    const int gz = tuned_grid(tu, FVV_TUNE_ZBUFFER, sms, sl.n, (long long)g.max_tris, cams.n);
    k_zbuffer<<<dim3(gz, cams.n, sl.n), tu.threads[FVV_TUNE_ZBUFFER], 0, st>>>(cams, L, sl);
    return cudaGetLastError();
}

cudaError_t launch_colour(const CamSet& cams, const Grid& g, const Layout& L, const ColourBatch& cb, int sms,
                          int total_slots, cudaStream_t st) {
    const int gv = grid_x(sms, total_slots, g.max_verts, 256);
    k_colour<<<dim3(gv, cb.n), 256, 0, st>>>(cams, g, L, cb);
    return cudaGetLastError();
}

cudaError_t launch_render_view(const CamSet& cams, const Grid& g, const Layout& L, const ViewArgs& va,
                              unsigned long long* key, uint8_t* out_rgb, int32_t* out_cam, int sms, cudaStream_t st) {
    const size_t npix = (size_t)va.v.W * (unsigned)va.v.H;
    const unsigned gp = (unsigned)std::max<size_t>(1, std::min<size_t>((npix + 255) / 256, (size_t)sms * 8));
    k_view_clear<<<gp, 256, 0, st>>>(key, npix);
    const unsigned gt = (unsigned)std::max<long long>(1, std::min<long long>((g.max_tris + 255) / 256, (long long)sms * 8));
    k_view_raster<<<gt, 256, 0, st>>>(L, va, key);
    k_view_shade<<<gp, 256, 0, st>>>(cams, g, L, va, key, out_rgb, out_cam);
    return cudaGetLastError();
}

cudaError_t launch_debug_depth(const CamSet& cams, const Layout& L, int slot, float* dst, size_t npix,
                               cudaStream_t st) {
    (void)cams;
    k_debug_depth<<<(unsigned)std::min<size_t>((npix + 255) / 256, 8192), 256, 0, st>>>(L, slot, dst, npix);
    return cudaGetLastError();
}

}  // namespace fvv
