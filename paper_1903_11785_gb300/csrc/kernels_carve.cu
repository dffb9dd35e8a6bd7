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
        bool alive = x < g.nx, voted = false;
        const float X = fadd(g.o[0], fmul(fadd((float)x, 0.5f), g.sc));
        const float Y = fadd(g.o[1], fmul(fadd((float)y, 0.5f), g.sc));
        const float Z = fadd(g.o[2], fmul(fadd((float)z, 0.5f), g.sc));
        for (int n = 0; n < cams.n; ++n) {
            if (!__any_sync(kFull, alive)) break;
            if (alive) {
                ++tests;
                const int v = cam_vote(cams.c[n], cams.oob, sil, X, Y, Z);
                alive = v != 0;
                voted |= (v == 1);
            }
        }
        const bool on = alive && voted;
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

// Index of the ROI holding fine word w: the last ROI whose first word <= w.
__device__ __forceinline__ int roi_of_word(const DRoi* rois, int n, uint32_t w) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rois[mid].word_off <= w) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Sec. II-B-3: the fine hull of every ROI, each treated as its own volume.
// Fine grids are stored padded by one unoccupied sample per side (index 0
// and fdim+1), rows of ceil((fdim_x+2)/32) words.
__global__ void __launch_bounds__(256) k_fine_carve(const __grid_constant__ CamSet cams,
                                                    const __grid_constant__ Grid g,
                                                    const __grid_constant__ Layout L,
                                                    const __grid_constant__ SlotList sl) {
    __shared__ unsigned long long sh_t[32];
    const int slot = sl.s[blockIdx.y];
    const SlotInfo* info = slot_ptr<SlotInfo>(L, slot, L.info);
    const uint32_t nwords = info->n_words;
    const int nrois = info->n_rois;
    const DRoi* rois = slot_ptr<DRoi>(L, slot, L.rois);
    const uint32_t* __restrict__ sil = slot_ptr<uint32_t>(L, slot, L.sil);
    uint32_t* fine = slot_ptr<uint32_t>(L, slot, L.fine);
    const int lane = threadIdx.x & 31;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    uint32_t tests = 0;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nwords; w += nwarps) {
        const DRoi& r = rois[roi_of_word(rois, nrois, w)];
        const uint32_t lw = w - r.word_off;
        const uint32_t row = lw / (uint32_t)r.nxw;
        const int wx = (int)(lw - row * (uint32_t)r.nxw);
        const int yp = (int)(row % (uint32_t)(r.fdim[1] + 2)), zp = (int)(row / (uint32_t)(r.fdim[1] + 2));
        const int xp = wx * 32 + lane;
        bool alive = xp >= 1 && xp <= r.fdim[0] && yp >= 1 && yp <= r.fdim[1] && zp >= 1 && zp <= r.fdim[2];
        bool voted = false;
        const float X = fadd(r.fo[0], fmul(fadd((float)(xp - 1), 0.5f), g.sf));
        const float Y = fadd(r.fo[1], fmul(fadd((float)(yp - 1), 0.5f), g.sf));
        const float Z = fadd(r.fo[2], fmul(fadd((float)(zp - 1), 0.5f), g.sf));
        for (int n = 0; n < cams.n; ++n) {
            if (!__any_sync(kFull, alive)) break;
            if (alive) {
                ++tests;
                const int v = cam_vote(cams.c[n], cams.oob, sil, X, Y, Z);
                alive = v != 0;
                voted |= (v == 1);
            }
        }
        const uint32_t word = __ballot_sync(kFull, alive && voted);
        if (lane == 0) fine[w] = word;
    }
    const unsigned long long t = block_sum<unsigned long long>(tests, sh_t);
    if (threadIdx.x == 0 && t) atomicAdd(&slot_ptr<SlotInfo>(L, slot, L.info)->tests_fine, t);
}

}  // namespace

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
                                cudaStream_t st) {
    const long long words = (long long)g.nz * g.ny * g.nxw;
    const int gx = grid_x(sms, sl.n, words * 32, 256);
    k_coarse_carve<<<dim3(gx, sl.n), 256, 0, st>>>(cams, g, L, sl);
    return cudaGetLastError();
}

cudaError_t launch_fine_carve(const CamSet& cams, const Grid& g, const Layout& L, const SlotList& sl, int sms,
                              cudaStream_t st) {
    const int gx = grid_x(sms, sl.n, (long long)g.max_fine_words * 32, 256);
    k_fine_carve<<<dim3(gx, sl.n), 256, 0, st>>>(cams, g, L, sl);
    return cudaGetLastError();
}

}  // namespace fvv
