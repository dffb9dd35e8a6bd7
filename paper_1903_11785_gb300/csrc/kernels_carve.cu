// kernels_carve.cu -- silhouette packing (step a0) and the coarse and fine
// visual hulls (Sec. II-B-1 and II-B-3).
//
// Silhouettes are kept as 1 bit per pixel (a 1080p camera is 260 KB, a
// 16-camera frame 4 MB, so a frame's silhouettes stay in L2).  A carve warp
// owns one 32-voxel word of the occupancy bitset: lane i tests voxel 32w+i,
// the warp walks the cameras in index order and stops as soon as a ballot
// shows no lane is still occupied, so the warp's loads stay coherent (the 32
// voxels of a row project close together) and empty space costs one camera.
#include "fvv_device.cuh"

namespace fvv {
namespace {

struct PackSrc {
    const uint8_t* src[FVV_MAX_CAMS];
};

// High bit of each nonzero byte of w, gathered into 4 bits (byte k -> bit k).
__device__ __forceinline__ uint32_t nonzero_bytes4(uint32_t w) {
    uint32_t t = (((w & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w) & 0x80808080u;
    return ((t >> 7) & 1u) | ((t >> 14) & 2u) | ((t >> 21) & 4u) | ((t >> 28) & 8u);
}

// Step a0: uint8 mask (nonzero = foreground) -> 1 bit per pixel, 32 pixels per
// word, bit x%32 of word x/32 of its row.  One thread per output word.
__global__ void __launch_bounds__(256) k_pack(const __grid_constant__ CamSet cams, const __grid_constant__ PackSrc a,
                                              uint32_t* __restrict__ sil) {
    const Cam& c = cams.c[blockIdx.y];
    const uint8_t* src = a.src[blockIdx.y];
    const size_t words = (size_t)c.H * (unsigned)c.Wq;
    const bool vec = (c.W % 32 == 0) && ((reinterpret_cast<uintptr_t>(src) & 15u) == 0);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / (unsigned)c.Wq;
        const int wq = (int)(i - row * (unsigned)c.Wq);
        const uint8_t* p = src + row * (unsigned)c.W + (size_t)wq * 32;
        uint32_t bits = 0;
        if (vec) {
            const uint4 a0 = __ldcs(reinterpret_cast<const uint4*>(p));
            const uint4 a1 = __ldcs(reinterpret_cast<const uint4*>(p) + 1);
            bits = nonzero_bytes4(a0.x) | nonzero_bytes4(a0.y) << 4 | nonzero_bytes4(a0.z) << 8 |
                   nonzero_bytes4(a0.w) << 12 | nonzero_bytes4(a1.x) << 16 | nonzero_bytes4(a1.y) << 20 |
                   nonzero_bytes4(a1.z) << 24 | nonzero_bytes4(a1.w) << 28;
        } else {
            const int nb = min(32, c.W - wq * 32);
            for (int b = 0; b < nb; ++b) bits |= (uint32_t)(p[b] != 0) << b;
        }
        sil[c.bit_off + i] = bits;
    }
}

// Sec. II-B-1: the coarse hull over the whole volume.  Occupied voxels also
// start their union-find tree (parent = own linear index) for Sec. II-B-2.
template <int NC>
__global__ void __launch_bounds__(256) k_coarse_carve(const __grid_constant__ CamSet cams,
                                                      const __grid_constant__ Grid g,
                                                      const __grid_constant__ Layout L,
                                                      const __grid_constant__ SlotList sl) {
    __shared__ unsigned long long sh_t[32];
    __shared__ unsigned long long sh_n[32];
    const int slot = sl.s[blockIdx.y];
    const uint32_t* __restrict__ sil = slot_ptr<uint32_t>(L, slot, L.sil);
    uint32_t* bits = slot_ptr<uint32_t>(L, slot, L.coarse);
    int* parent = slot_ptr<int>(L, slot, L.parent);
    const uint32_t nwords = (uint32_t)g.nz * (uint32_t)g.ny * (uint32_t)g.nxw;
    const int lane = threadIdx.x & 31;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    uint32_t tests = 0, on_count = 0;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nwords; w += nwarps) {
        const uint32_t row = w / (uint32_t)g.nxw;
        const int wx = (int)(w - row * (uint32_t)g.nxw);
        const int y = (int)(row % (uint32_t)g.ny), z = (int)(row / (uint32_t)g.ny);
        const int x = wx * 32 + lane;
        const float X = fadd(g.o[0], fmul(fadd((float)x, 0.5f), g.sc));
        const float Y = fadd(g.o[1], fmul(fadd((float)y, 0.5f), g.sc));
        const float Z = fadd(g.o[2], fmul(fadd((float)z, 0.5f), g.sc));
        const bool on = warp_test<NC>(cams, sil, X, Y, Z, x < g.nx, tests);
        const uint32_t word = __ballot_sync(kFull, on);
        if (on) {
            const int Lin = (int)(row * (uint32_t)g.nx) + x;
            parent[Lin] = Lin;
        }
        if (lane == 0) {
            bits[w] = word;
            on_count += __popc(word);
        }
    }
    const unsigned long long t = block_sum<unsigned long long>(tests, sh_t);
    const unsigned long long c = block_sum<unsigned long long>(on_count, sh_n);
    if (threadIdx.x == 0) {
        SlotInfo* info = slot_ptr<SlotInfo>(L, slot, L.info);
        if (t) atomicAdd(&info->tests_coarse, t);
        if (c) atomicAdd(&info->n_on, (uint32_t)c);
    }
}

__global__ void __launch_bounds__(256) k_clear_fine(const __grid_constant__ Layout L,
                                                    const __grid_constant__ SlotList sl) {
    const int slot = sl.s[blockIdx.y];
    const uint32_t nwords = slot_ptr<SlotInfo>(L, slot, L.info)->n_words;
    uint32_t* fine = slot_ptr<uint32_t>(L, slot, L.fine);
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += gridDim.x * blockDim.x) fine[w] = 0u;
}

// The ROI holding interior fine sample s: the last ROI whose first sample <= s.
__device__ __forceinline__ int roi_of_sample(const DRoi* rois, int n, uint32_t s) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rois[mid].samp_off <= s) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Levels of the fine carve: a sample at level j has passed cameras
// [0, lvb(j)) and tests cameras [lvb(j), lvb(j + 1)) next: [0,2), [2,4),
// [4,8), [8,N).
constexpr int kLevels = 4;
__host__ __device__ constexpr int lvb(int n, int j) {
    return j == 0 ? 0 : (j < kLevels && (1 << j) < n ? (1 << j) : n);
}

// Cameras [C0, C1) of the test (Sec. II-B-1) for the live lanes of a warp,
// in index order, each lane stopping at its first background vote and the
// warp at the first camera where no lane is left.
template <bool ABSTAIN, int C0, int C1>
__device__ __forceinline__ void test_span(const CamSet& cams, const uint32_t* __restrict__ sil, float X, float Y,
                                          float Z, bool& alive, bool& voted, uint32_t& tests) {
#pragma unroll
    for (int n = C0; n < C1; ++n) {
        if (!__any_sync(kFull, alive)) break;
        if (alive) {
            ++tests;
            test_cam<ABSTAIN>(cams.c[n], sil, X, Y, Z, alive, voted);
        }
    }
}

template <bool ABSTAIN>
__device__ __forceinline__ void test_span_rt(const CamSet& cams, const uint32_t* __restrict__ sil, int c0, int c1,
                                             float X, float Y, float Z, bool& alive, bool& voted, uint32_t& tests) {
    for (int n = c0; n < c1; ++n) {
        if (!__any_sync(kFull, alive)) break;
        if (alive) {
            ++tests;
            test_cam<ABSTAIN>(cams.c[n], sil, X, Y, Z, alive, voted);
        }
    }
}

template <int NC, bool ABSTAIN>
__device__ __forceinline__ void test_level(const CamSet& cams, const uint32_t* __restrict__ sil, int lv, float X,
                                           float Y, float Z, bool& alive, bool& voted, uint32_t& tests) {
    if constexpr (NC > 0) {
        switch (lv) {
            case 0: test_span<ABSTAIN, lvb(NC, 0), lvb(NC, 1)>(cams, sil, X, Y, Z, alive, voted, tests); break;
            case 1: test_span<ABSTAIN, lvb(NC, 1), lvb(NC, 2)>(cams, sil, X, Y, Z, alive, voted, tests); break;
            case 2: test_span<ABSTAIN, lvb(NC, 2), lvb(NC, 3)>(cams, sil, X, Y, Z, alive, voted, tests); break;
            default: test_span<ABSTAIN, lvb(NC, 3), NC>(cams, sil, X, Y, Z, alive, voted, tests); break;
        }
    } else {
        test_span_rt<ABSTAIN>(cams, sil, lvb(cams.n, lv), lvb(cams.n, lv + 1), X, Y, Z, alive, voted, tests);
    }
}

// Sec. II-B-3: the fine hull of every ROI, each treated as its own volume.
// Fine grids are stored padded by one unoccupied sample per side (index 0
// and fdim+1), rows of ceil((fdim_x+2)/32) words, cleared beforehand; only
// occupied samples are written, by OR into their word.
//
// Most samples are rejected by the first camera or two while the points
// inside the hull take every camera, so a warp that kept its 32 samples to
// the end would idle most lanes.  Each warp therefore moves samples through
// levels (cameras [0,2), [2,4), [4,8), [8,N)): a step takes 32 samples at
// one level (fresh interior samples of all ROIs, in order, at level 0),
// tests that level's cameras and queues the survivors in the warp's part of
// shared memory for the next level; the deepest level holding 32 goes
// first, so each queue stays under 64 entries.  The queue counts are the
// same in every lane (they follow from ballots), so the warp needs no
// shared counters and the block no barrier.  Each sample still tests the
// cameras in index order and stops at its first background vote, so
// occupancy and test counts are those of the plain per-sample loop.
template <int NC>
__global__ void __launch_bounds__(256) k_fine_carve(const __grid_constant__ CamSet cams,
                                                    const __grid_constant__ Grid g,
                                                    const __grid_constant__ Layout L,
                                                    const __grid_constant__ SlotList sl) {
    extern __shared__ float4 fq_all[];       // per warp: levels 1..3, 64 entries each
    __shared__ unsigned long long sh_t[32];
    const int slot = sl.s[blockIdx.y];
    const SlotInfo* info = slot_ptr<SlotInfo>(L, slot, L.info);
    const uint32_t nsamp = info->n_words ? info->n_samples : 0u;
    const int nrois = info->n_rois;
    const DRoi* rois = slot_ptr<DRoi>(L, slot, L.rois);
    const uint32_t* __restrict__ sil = slot_ptr<uint32_t>(L, slot, L.sil);
    uint32_t* fine = slot_ptr<uint32_t>(L, slot, L.fine);
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    float4* fq = fq_all + (threadIdx.x >> 5) * (kLevels - 1) * 64;
    const int ncam = NC > 0 ? NC : cams.n;
    const bool abstain = cams.oob == FVV_OOB_ABSTAIN;
    const uint32_t fresh_step = gridDim.x * blockDim.x;
    uint32_t fresh = blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
    int qn[kLevels] = {0, 0, 0, 0};          // entries queued per level (level 0 unused)
    uint32_t tests = 0;
    // per-lane ROI cursor for fresh samples
    uint32_t lo = 0, hi = 0, woff = 0;
    int fx = 1, fy = 1, nxw = 1;
    float fo0 = 0.f, fo1 = 0.f, fo2 = 0.f;
    for (;;) {
        int lv = -1;
#pragma unroll
        for (int j = 1; j < kLevels; ++j)
            if (qn[j] >= 32) lv = j;
        if (lv < 0 && fresh < nsamp) lv = 0;
        if (lv < 0) {
#pragma unroll
            for (int j = kLevels - 1; j >= 1; --j)
                if (qn[j] > 0) lv = j;
        }
        if (lv < 0) break;
        float X = 0.f, Y = 0.f, Z = 0.f;
        uint32_t wb = 0;                     // word << 6 | voted << 5 | bit
        bool act;
        if (lv == 0) {
            const uint32_t s = fresh + lane;
            fresh += fresh_step;
            act = s < nsamp;
            if (act && (s >= hi || s < lo)) {
                const DRoi& r = rois[roi_of_sample(rois, nrois, s)];
                lo = r.samp_off;
                fx = r.fdim[0];
                fy = r.fdim[1];
                hi = lo + (uint32_t)fx * (uint32_t)fy * (uint32_t)r.fdim[2];
                woff = r.word_off;
                nxw = r.nxw;
                fo0 = r.fo[0];
                fo1 = r.fo[1];
                fo2 = r.fo[2];
            }
            const uint32_t loc = act ? s - lo : 0u;
            const uint32_t row = loc / (uint32_t)fx;
            const int x = (int)(loc - row * (uint32_t)fx);
            const int y = (int)(row % (uint32_t)fy), z = (int)(row / (uint32_t)fy);
            X = fadd(fo0, fmul(fadd((float)x, 0.5f), g.sf));
            Y = fadd(fo1, fmul(fadd((float)y, 0.5f), g.sf));
            Z = fadd(fo2, fmul(fadd((float)z, 0.5f), g.sf));
            const uint32_t word = woff + ((uint32_t)(z + 1) * (uint32_t)(fy + 2) + (uint32_t)(y + 1)) * (uint32_t)nxw +
                                  (uint32_t)((x + 1) >> 5);
            wb = (word << 6) | (uint32_t)((x + 1) & 31);
        } else {
            const int take = min(qn[lv], 32);
            qn[lv] -= take;
            act = lane < take;
            if (act) {
                const float4 e = fq[(lv - 1) * 64 + qn[lv] + lane];
                X = e.x;
                Y = e.y;
                Z = e.z;
                wb = __float_as_uint(e.w);
            }
        }
        bool alive = act, voted = !abstain || ((wb >> 5) & 1u);
        if (abstain) test_level<NC, true>(cams, sil, lv, X, Y, Z, alive, voted, tests);
        else test_level<NC, false>(cams, sil, lv, X, Y, Z, alive, voted, tests);
        if (lvb(ncam, lv + 1) == ncam) {
            // every camera done: OR the occupied samples into their words,
            // one atomic per distinct word of the warp
            const bool on = alive && voted;
            const uint32_t word = wb >> 6, bit = 1u << (wb & 31u);
            uint32_t pend = __ballot_sync(kFull, on);
            while (pend) {
                const int leader = __ffs(pend) - 1;
                const uint32_t T = __shfl_sync(kFull, word, leader);
                const bool mine = on && word == T;
                const uint32_t ored = __reduce_or_sync(kFull, mine ? bit : 0u);
                if (lane == leader) atomicOr(fine + T, ored);
                pend &= ~__ballot_sync(kFull, mine);
            }
        } else {
            // the popped entries were read above, before any lane writes
            const uint32_t m = __ballot_sync(kFull, alive);
            if (alive)
                fq[lv * 64 + qn[lv + 1] + __popc(m & lt)] =
                    make_float4(X, Y, Z, __uint_as_float((wb & ~32u) | (voted ? 32u : 0u)));
            qn[lv + 1] += __popc(m);
        }
        __syncwarp();
    }
    const unsigned long long t = block_sum<unsigned long long>(tests, sh_t);
    if (threadIdx.x == 0 && t) atomicAdd(&slot_ptr<SlotInfo>(L, slot, L.info)->tests_fine, t);
}

// Test hook: the pixel each point falls in for one camera (-1, -1 if none).
__global__ void k_debug_pixels(const __grid_constant__ CamSet cams, int cam, long long n,
                               const float* __restrict__ pts, int32_t* px, int32_t* py) {
    const Cam& c = cams.c[cam];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int u, v;
        cam_pixel(c, pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], u, v);
        px[i] = u;
        py[i] = v;
    }
}

}  // namespace

cudaError_t launch_debug_pixels(const CamSet& cams, int cam, long long n, const float* pts, int32_t* px,
                                int32_t* py, cudaStream_t st) {
    const unsigned g = (unsigned)std::min<long long>((n + 255) / 256, 8192);
    k_debug_pixels<<<g, 256, 0, st>>>(cams, cam, n, pts, px, py);
    return cudaGetLastError();
}

cudaError_t launch_pack(const CamSet& cams, const Layout& L, int slot, const uint8_t* const* src, cudaStream_t st) {
    PackSrc a{};
    size_t max_words = 0;
    for (int n = 0; n < cams.n; ++n) {
        a.src[n] = src[n];
        max_words = std::max(max_words, (size_t)cams.c[n].H * (unsigned)cams.c[n].Wq);
    }
    const unsigned gx = (unsigned)std::min<size_t>((max_words + 255) / 256, 2048);
    k_pack<<<dim3(std::max(1u, gx), cams.n), 256, 0, st>>>(cams, a, slot_ptr<uint32_t>(L, slot, L.sil));
    return cudaGetLastError();
}

cudaError_t launch_coarse_carve(const CamSet& cams, const Grid& g, const Layout& L, const SlotList& sl, int sms,
                                const Tuning& tu, cudaStream_t st) {
    const long long words = (long long)g.nz * g.ny * g.nxw;
    const int th = tu.threads[FVV_TUNE_COARSE];
    const int gx = tuned_grid(tu, FVV_TUNE_COARSE, sms, sl.n, words * 32);
#define FVV_LAUNCH(NC) k_coarse_carve<NC><<<dim3(gx, sl.n), th, 0, st>>>(cams, g, L, sl)
    FVV_DISPATCH_NC(cams.n, FVV_LAUNCH)
#undef FVV_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_fine_carve(const CamSet& cams, const Grid& g, const Layout& L, const SlotList& sl, int sms,
                              const Tuning& tu, cudaStream_t st) {
    const int gc = grid_x(sms, sl.n, (long long)g.max_fine_words, 256);
    k_clear_fine<<<dim3(gc, sl.n), 256, 0, st>>>(L, sl);
    const int th = tu.threads[FVV_TUNE_FINE];
    const int gx = tuned_grid(tu, FVV_TUNE_FINE, sms, sl.n, (long long)g.max_fine_words * 32);
#define FVV_LAUNCH(NC) k_fine_carve<NC><<<dim3(gx, sl.n), th, (size_t)th / 32 * 3 * 64 * sizeof(float4), st>>>(cams, g, L, sl)
    FVV_DISPATCH_NC(cams.n, FVV_LAUNCH)
#undef FVV_LAUNCH
    return cudaGetLastError();
}

}  // namespace fvv
