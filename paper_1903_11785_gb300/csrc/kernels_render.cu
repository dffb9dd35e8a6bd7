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

// The depth images only ever hold values inside each camera's box (x0, x1,
// y0, y1, none when x1 < x0), which contains every pixel the slot's last
// z-buffer could write: a depth stage clears the previous box, sets the box
// for this frame (k_depth_box) and runs the z-buffer, so every pixel outside
// it is empty (+infinity) without clearing the whole image each frame.
__global__ void __launch_bounds__(256) k_init_depth(const __grid_constant__ Layout L, size_t n16,
                                                    int n_cams) {
    const int slot = blockIdx.y;
    uint4* d = slot_ptr<uint4>(L, slot, L.depth);
    const uint4 v = make_uint4(kEmptyDepth, kEmptyDepth, kEmptyDepth, kEmptyDepth);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
        d[i] = v;
    if (blockIdx.x == 0 && threadIdx.x < (unsigned)n_cams) {
        int4* box = slot_ptr<int4>(L, slot, L.dbox);
        box[threadIdx.x] = make_int4(INT_MAX, -1, INT_MAX, -1);
    }
}

// Clear each camera's written box (grid: blocks, cameras, slots).
__global__ void __launch_bounds__(256) k_clear_depth(const __grid_constant__ CamSet cams,
                                                     const __grid_constant__ Layout L,
                                                     const __grid_constant__ SlotList sl) {
    pdl_begin();
    const int slot = sl.s[blockIdx.z];
    const Cam& c = cams.c[blockIdx.y];
    const int4 b = slot_ptr<int4>(L, slot, L.dbox)[blockIdx.y];
    if (b.y < b.x || b.w < b.z) return;
    uint32_t* D = slot_ptr<uint32_t>(L, slot, L.depth) + c.pix_off;
    for (int y = b.z + (int)blockIdx.x; y <= b.w; y += (int)gridDim.x) {
        uint32_t* row = D + (size_t)y * (unsigned)c.W;
        for (int x = b.x + (int)threadIdx.x; x <= b.y; x += (int)blockDim.x) __stcs(row + x, kEmptyDepth);
    }
}

// The box each camera's z-buffer can write this frame (after k_clear_depth,
// before k_zbuffer): every mesh vertex lies in its ROI's fine grid box grown
// by one fine voxel (padding samples and bisection points), so every covered
// pixel centre lies in the convex hull of the projections of that box's
// eight corners; the union over the ROIs, widened by two pixels and clamped
// to the image, or the whole image if a corner is not in front of the
// camera.  One block per slot, a thread per (camera, ROI).
__global__ void k_depth_box(const __grid_constant__ CamSet cams, const __grid_constant__ Grid g,
                            const __grid_constant__ Layout L, const __grid_constant__ SlotList sl) {
    pdl_begin();
    const int slot = sl.s[blockIdx.x];
    int4* box = slot_ptr<int4>(L, slot, L.dbox);
    for (int n = threadIdx.x; n < cams.n; n += blockDim.x) box[n] = make_int4(INT_MAX, -1, INT_MAX, -1);
    __syncthreads();
    const SlotInfo* info = slot_ptr<SlotInfo>(L, slot, L.info);
    const int nrois = info->n_words ? info->n_rois : 0;
    const DRoi* rois = slot_ptr<DRoi>(L, slot, L.rois);
    for (int i = threadIdx.x; i < cams.n * nrois; i += blockDim.x) {
        const int n = i / nrois, k = i - n * nrois;
        const Cam& c = cams.c[n];
        const DRoi& r = rois[k];
        float lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = r.fo[a] - g.sf;
            hi[a] = r.fo[a] + (float)(r.fdim[a] + 1) * g.sf;
        }
        float umin = 3.0e38f, umax = -3.0e38f, vmin = 3.0e38f, vmax = -3.0e38f;
        bool front = true;
        for (int q = 0; q < 8; ++q) {
            float xh, yh, wh;
            project(c.P, (q & 1) ? hi[0] : lo[0], (q & 2) ? hi[1] : lo[1], (q & 4) ? hi[2] : lo[2], xh, yh, wh);
            front &= wh > 0.0f;
            const float u = __fdiv_rn(xh, wh), v = __fdiv_rn(yh, wh);
            umin = fminf(umin, u); umax = fmaxf(umax, u);
            vmin = fminf(vmin, v); vmax = fmaxf(vmax, v);
        }
        int x0 = 0, x1 = c.W - 1, y0 = 0, y1 = c.H - 1;
        if (front && umin > -1.0e6f && umax < 1.0e6f && vmin > -1.0e6f && vmax < 1.0e6f) {
            x0 = max(0, (int)floorf(umin) - 2);
            x1 = min(c.W - 1, (int)floorf(umax) + 2);
            y0 = max(0, (int)floorf(vmin) - 2);
            y1 = min(c.H - 1, (int)floorf(vmax) + 2);
        }
        if (x0 > x1 || y0 > y1) continue;
        int* b = reinterpret_cast<int*>(box + n);
        atomicMin(b + 0, x0);
        atomicMax(b + 1, x1);
        atomicMin(b + 2, y0);
        atomicMax(b + 3, y1);
    }
}

// Eq. (4) coverage of one triangle (world vertices X, Y, Z) in camera c, in
// two parts, raster_setup and raster_pixels (below).
// The first part: the homogeneous image points of the vertices
// and the candidate pixels (centres within 1/64 px of the box of the
// approximate projections; their error is below 1e-3 px for images up to
// 65535 px, and the exact box test in raster_pixels decides).  False if a
// vertex is not in front of the camera or no pixel centre is a candidate.
//
// The candidate columns are ceil(umin - 1/2 - 1/64) .. floor((umax + 1/64)
// - 1/2), clamped to the image (rows alike).  They are rounded on the FMA
// pipe: for |t| < 2^22, t + 1.5 * 2^23 rounded down (up) is 1.5 * 2^23 +
// floor(t) (ceil(t)) exactly, since floats in [2^23, 2^24) are the
// integers; the box ends are kept in that form (kMagic + integer), so that
// comparing them compares the integers, and the integer is the float's bits
// minus those of kMagic.  A clamped end is always in that range; an end
// outside it only arises for an empty box, which the comparison then shows.
constexpr float kMagic = 12582912.0f;        // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;
struct TriSetup {
    float xh[3], yh[3], wh[3];
    float x0, x1, y0, y1;                    // kMagic + first/last candidate column and row
};

__device__ __forceinline__ int magic_int(float m) { return __float_as_int(m) - kMagicBits; }

__device__ __forceinline__ bool raster_setup(const Cam& c, const float* X, const float* Y, const float* Z,
                                             TriSetup& s) {
    bool ok = true;
    float u[3], v[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        project(c.P, X[j], Y[j], Z[j], s.xh[j], s.yh[j], s.wh[j]);
        ok &= s.wh[j] > 0.0f;
        const float r = rcp_approx(s.wh[j]);
        u[j] = fmul(s.xh[j], r);
        v[j] = fmul(s.yh[j], r);
    }
    const float umin = fminf(u[0], fminf(u[1], u[2])), umax = fmaxf(u[0], fmaxf(u[1], u[2]));
    const float vmin = fminf(v[0], fminf(v[1], v[2])), vmax = fmaxf(v[0], fmaxf(v[1], v[2]));
    constexpr float kSlack = 0.5f + 1.0f / 64.0f;
    s.x0 = __fadd_ru(fmaxf(fsub(umin, kSlack), 0.0f), kMagic);
    s.y0 = __fadd_ru(fmaxf(fsub(vmin, kSlack), 0.0f), kMagic);
    s.x1 = __fadd_rd(fminf(fsub(fadd(umax, 1.0f / 64.0f), 0.5f), fsub(c.Wf, 1.0f)), kMagic);
    s.y1 = __fadd_rd(fminf(fsub(fadd(vmax, 1.0f / 64.0f), 0.5f), fsub(c.Hf, 1.0f)), kMagic);
    // (umax >= 0 and vmax >= 0 also turn away all-NaN image positions)
    return ok && umax >= 0.0f && vmax >= 0.0f && s.x0 <= s.x1 && s.y0 <= s.y1;
}

// The second part: the triangle is skipped if its projected area is zero;
// `sink(pixel)` is called for each candidate pixel (row-major index in an
// image W pixels wide) whose centre p lies in the closed box of the projection and on the
// inner side of (or on) all three edges, either winding.  Everything is
// decided on the homogeneous image points (x', y', w') without dividing: the
// edge function of edge (i, j) at p is (p_x a - p_y b) + c with
// a = y_i w_j - w_i y_j, b = x_i w_j - w_i x_j, c = x_i y_j - y_i x_j (its sign
// is the image-plane one for w > 0), the area is zero iff
// (x_0 a_12 - y_0 b_12) + w_0 c_12 is, and the box test uses the exact signs
// of p w_j - x_j from one FMA each.
template <class Sink>
__device__ __forceinline__ void raster_pixels(unsigned W, const TriSetup& s, Sink&& sink) {
    const float* xh = s.xh;
    const float* yh = s.yh;
    const float* wh = s.wh;
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
    const int x0 = magic_int(s.x0), x1 = magic_int(s.x1), y1 = magic_int(s.y1);
    for (int yy = magic_int(s.y0); yy <= y1; ++yy) {
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
            if (in) sink((size_t)yy * W + xx);
        }
    }
}

// Eq. (4) coverage of one triangle (world vertices X, Y, Z) in camera c.
template <class Sink>
__device__ __forceinline__ void raster_tri(const Cam& c, const float* X, const float* Y, const float* Z,
                                           Sink&& sink) {
    TriSetup s;
    if (raster_setup(c, X, Y, Z, s)) raster_pixels((unsigned)c.W, s, sink);
}

constexpr int kZQueue = 64;   // queue entries per camera and warp

// Draws the n (<= 32) queued triangles ids[0..n-1] in camera c, one per
// lane: each is set up again from its record (the same arithmetic as when
// it was queued, so the same candidate box) and its covered pixels keep the
// minimum of the squared centroid distance (sqrt is monotone, so the square
// root of that minimum is the minimum distance itself, taken where the
// depth is read).
__device__ __forceinline__ void zdraw_ids(const Cam& c, const uint32_t* ids, int n, const float4* tsoup,
                                          uint32_t* D) {
    const int lane = threadIdx.x & 31;
    if (lane >= n) return;
    const uint32_t t = ids[lane];
    const float4 r0 = __ldg(tsoup + 3 * (size_t)t), r1 = __ldg(tsoup + 3 * (size_t)t + 1),
                 r2 = __ldg(tsoup + 3 * (size_t)t + 2);
    const float X[3] = {r0.x, r0.w, r1.z}, Y[3] = {r0.y, r1.x, r1.w}, Z[3] = {r0.z, r1.y, r2.x};
    const float dx = fsub(r2.y, c.C[0]);
    const float dy = fsub(r2.z, c.C[1]);
    const float dz = fsub(r2.w, c.C[2]);
    const uint32_t d2 = __float_as_uint(fadd(fadd(fmul(dx, dx), fmul(dy, dy)), fmul(dz, dz)));
    TriSetup s;
    raster_setup(c, X, Y, Z, s);   // true, as when the triangle was queued
    uint32_t* img = D + c.pix_off;
    raster_pixels((unsigned)c.W, s, [&](size_t pix) {
        uint32_t* p = img + pix;
        if (__ldcg(p) > d2) atomicMin(p, d2);   // skip the atomic when already nearer
    });
}

// Eq. (4) depth images.  Grid (blocks, camera groups, slots): a block serves
// K cameras (blockIdx.y * K ...; K = 1, 2 or 4, the autotuner's choice), the
// same for all its threads, so their matrices are read through uniform
// registers, and blocks are issued frame by frame, so one frame's depth
// images are worked on together.  A warp takes 32 triangles at a time, one
// per lane, reads each triangle's 48-byte record once (vertices and the
// centroid ((v0 + v1) + v2) / 3 formed when the triangle was emitted) and
// sets it up for each camera of the group in turn (raster_setup).  About 70%
// of the (triangle, camera) pairs have no candidate pixel centre; the warp
// queues the indices of the others, per camera, and draws them 32 at a
// time, one per lane (zdraw_ids), instead of by 30% of the lanes while the
// rest wait.  A queue entry is 4 bytes: the set-up is done again at drawing,
// which costs less than keeping its 64 bytes in shared memory.
template <int K>
__global__ void __launch_bounds__(256, 4) k_zbuffer(const __grid_constant__ CamSet cams,
                                                    const __grid_constant__ Layout L,
                                                    const __grid_constant__ SlotList sl) {
    pdl_begin();
    __shared__ uint32_t zq[8][K * kZQueue];   // per warp (at most 256 threads), per camera
    const int slot = sl.s[blockIdx.z];
    const int n0 = blockIdx.y * K;
    const int kn = min(K, cams.n - n0);       // cameras of this group
    const SlotInfo* info = slot_ptr<SlotInfo>(L, slot, L.info);
    const uint32_t nt = info->n_words ? info->n_tris : 0u;
    const float4* tsoup = slot_ptr<float4>(L, slot, L.tsoup);
    uint32_t* D = slot_ptr<uint32_t>(L, slot, L.depth);
    const int lane = threadIdx.x & 31;
    uint32_t* q = zq[threadIdx.x >> 5];
    uint32_t qn = 0;   // queued triangles per camera, 8 bits each (the same in every lane; each < 64)
    for (uint32_t t0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); t0 < nt; t0 += gridDim.x * blockDim.x) {
        const uint32_t t = t0 + (uint32_t)lane;   // the loop condition is warp-uniform
        const bool have = t < nt;
        float4 r0, r1, r2;                        // read only where have
        if (have) {
            r0 = __ldg(tsoup + 3 * (size_t)t);
            r1 = __ldg(tsoup + 3 * (size_t)t + 1);
            r2 = __ldg(tsoup + 3 * (size_t)t + 2);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (k >= kn) break;                   // uniform
            const Cam& c = cams.c[n0 + k];
            TriSetup s;
            bool ok = false;
            if (have) {
                const float X[3] = {r0.x, r0.w, r1.z}, Y[3] = {r0.y, r1.x, r1.w}, Z[3] = {r0.z, r1.y, r2.x};
                ok = raster_setup(c, X, Y, Z, s);
            }
            const unsigned m = __ballot_sync(kFull, ok);
            if (ok) q[k * kZQueue + ((qn >> (8 * k)) & 0xFFu) + __popc(m & ((1u << lane) - 1u))] = t;
            qn += (uint32_t)__popc(m) << (8 * k);
        }
        __syncwarp();
#pragma unroll 1
        for (int k = 0; k < kn; ++k) {            // a camera with 32 queued: draw them
            const uint32_t cnt = (qn >> (8 * k)) & 0xFFu;
            if (cnt >= 32u) {
                qn -= 32u << (8 * k);
                zdraw_ids(cams.c[n0 + k], q + k * kZQueue + (cnt - 32u), 32, tsoup, D);
                __syncwarp();                     // read before the entries are reused
            }
        }
    }
#pragma unroll 1
    for (int k = 0; k < kn; ++k) {                // the rest, up to 32 at a time
        uint32_t cnt = (qn >> (8 * k)) & 0xFFu;
        while (cnt > 0u) {
            const uint32_t n = min(cnt, 32u);
            cnt -= n;
            zdraw_ids(cams.c[n0 + k], q + k * kZQueue + cnt, (int)n, tsoup, D);
            __syncwarp();
        }
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
    pdl_begin();
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
    const float4* tsoup = slot_ptr<float4>(L, va.slot, L.tsoup);
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        const float4 r0 = __ldg(tsoup + 3 * (size_t)t), r1 = __ldg(tsoup + 3 * (size_t)t + 1),
                     r2 = __ldg(tsoup + 3 * (size_t)t + 2);
        const float X[3] = {r0.x, r0.w, r1.z}, Y[3] = {r0.y, r1.x, r1.w}, Z[3] = {r0.z, r1.y, r2.x};
        const float dx = fsub(r2.y, v.C[0]);
        const float dy = fsub(r2.z, v.C[1]);
        const float dz = fsub(r2.w, v.C[2]);
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
    const float4* tsoup = slot_ptr<float4>(L, va.slot, L.tsoup);
    const size_t npix = (size_t)va.v.W * (unsigned)va.v.H;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long k = key[i];
        uint8_t col[3] = {0, 0, 0};
        int chosen = -1;
        if (k != ~0ull) {
            const float4 r2 = __ldg(tsoup + 3 * (size_t)(uint32_t)k + 2);   // (v2 z, centroid xyz)
            chosen = colour_point(cams, rank_cam, depth, va.rgb, g.t_v, r2.y, r2.z, r2.w, col);
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

cudaError_t launch_init_depth(const CamSet& cams, const Layout& L, int n_slots, int sms, cudaStream_t st) {
    size_t pix = 0;
    for (int n = 0; n < cams.n; ++n) pix += (size_t)cams.c[n].W * cams.c[n].H;
    const size_t n16 = (pix * 4 + 15) / 16;
    const unsigned gx = (unsigned)std::max<size_t>(1, std::min<size_t>((n16 + 255) / 256, (size_t)sms * 4));
    for (int s0 = 0; s0 < n_slots; s0 += 65535) {
        // slots s0.. in one launch (blockIdx.y is at most 65535)
        Layout Ls = L;
        Ls.base = L.base + (size_t)s0 * L.stride;
        k_init_depth<<<dim3(gx, std::min(65535, n_slots - s0)), 256, 0, st>>>(Ls, n16, cams.n);
    }
    return cudaGetLastError();
}

cudaError_t launch_depth(const CamSet& cams, const Grid& g, const Layout& L, const SlotList& sl, int sms,
                         size_t depth_bytes, const Tuning& tu, cudaStream_t st) {
    (void)depth_bytes;
    const int gc = std::max(1, sms * 4 / std::max(1, sl.n * cams.n));
    launch_pdl(k_clear_depth, dim3(gc, cams.n, sl.n), dim3(256), 0, st, cams, L, sl);
    launch_pdl(k_depth_box, dim3(sl.n), dim3(256), 0, st, cams, g, L, sl);
    const int K = tu.zb_cams;
    const int groups = (cams.n + K - 1) / K;
    const int gz = tuned_grid(tu, FVV_TUNE_ZBUFFER, sms, sl.n, (long long)g.max_tris, groups);
    const dim3 grid(gz, groups, sl.n), block(tu.threads[FVV_TUNE_ZBUFFER]);
    cudaError_t e;
    if (K == 4) e = launch_pdl(k_zbuffer<4>, grid, block, 0, st, cams, L, sl);
    else if (K == 2) e = launch_pdl(k_zbuffer<2>, grid, block, 0, st, cams, L, sl);
    else e = launch_pdl(k_zbuffer<1>, grid, block, 0, st, cams, L, sl);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_colour(const CamSet& cams, const Grid& g, const Layout& L, const ColourBatch& cb, int sms,
                          int total_slots, cudaStream_t st) {
    const int gv = grid_x(sms, total_slots, g.max_verts, 256);
    launch_pdl(k_colour, dim3(gv, cb.n), dim3(256), 0, st, cams, g, L, cb);
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
