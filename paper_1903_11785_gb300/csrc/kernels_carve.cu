// kernels_carve.cu -- silhouette packing (step a0) and the coarse and fine
// visual hulls (Sec. II-B-1 and II-B-3).
//
// Silhouettes are kept as 1 bit per pixel (a 1080p camera is 260 KB, a
// 16-camera frame 4 MB, so a frame's silhouettes stay in L2).  A coarse
// carve warp takes a row of the occupancy bitset one 32-voxel word at a time:
// lane i tests voxel 32w+i, the warp walks the cameras in index order and
// stops as soon as a ballot shows no lane is still occupied, so the warp's
// loads stay coherent (the 32 voxels of a word project close together) and
// empty space costs one camera.
#include "fvv_device.cuh"

namespace fvv {
namespace {

// The masks of up to kPackFrames frames (frame j: slot[j], camera n:
// src[j * n_cams + n]) packed by one launch.
constexpr int kPackPtrs = 2048;
struct PackSrc {
    const uint8_t* src[kPackPtrs];
    int slot[kPackPtrs / 4];
};

// High bit of each nonzero byte of w, gathered into 4 bits (byte k -> bit k).
__device__ __forceinline__ uint32_t nonzero_bytes4(uint32_t w) {
    uint32_t t = (((w & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w) & 0x80808080u;
    return ((t >> 7) & 1u) | ((t >> 14) & 2u) | ((t >> 21) & 4u) | ((t >> 28) & 8u);
}

// Step a0: uint8 mask (nonzero = foreground) -> 1 bit per pixel, 32 pixels per
// word, bit x%32 of word x/32 of its row.  One thread per output word; grid
// (blocks, cameras, frames).
__global__ void __launch_bounds__(256) k_pack(const __grid_constant__ CamSet cams, const __grid_constant__ PackSrc a,
                                              const __grid_constant__ Layout L) {
    pdl_begin();
    const Cam& c = cams.c[blockIdx.y];
    const uint8_t* src = a.src[blockIdx.z * (unsigned)cams.n + blockIdx.y];
    uint32_t* __restrict__ sil = slot_ptr<uint32_t>(L, a.slot[blockIdx.z], L.sil);
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
// start the union-find forest of Sec. II-B-2: each run of consecutive
// occupied voxels within a 32-voxel word is one tree, rooted at the run's
// first voxel (in this word), which is its smallest linear index.
template <int NC>
__global__ void __launch_bounds__(256) k_coarse_carve(const __grid_constant__ CamSet cams,
                                                      const __grid_constant__ Grid g,
                                                      const __grid_constant__ Layout L,
                                                      const __grid_constant__ SlotList sl) {
    pdl_begin();
    __shared__ unsigned long long sh_t[32];
    __shared__ unsigned long long sh_n[32];
    const int slot = sl.s[blockIdx.y];
    const uint32_t* __restrict__ sil = slot_ptr<uint32_t>(L, slot, L.sil);
    uint32_t* bits = slot_ptr<uint32_t>(L, slot, L.coarse);
    int* parent = slot_ptr<int>(L, slot, L.parent);
    const uint32_t nrows = (uint32_t)g.nz * (uint32_t)g.ny;
    const int lane = threadIdx.x & 31;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    uint32_t tests = 0, on_count = 0;
    // a warp takes a whole row (y, z) and walks its words, so the row is
    // decoded once and Y, Z are formed once
    for (uint32_t row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < nrows; row += nwarps) {
        const int y = (int)(row % (uint32_t)g.ny), z = (int)(row / (uint32_t)g.ny);
        const float Y = fadd(g.o[1], fmul(fadd((float)y, 0.5f), g.sc));
        const float Z = fadd(g.o[2], fmul(fadd((float)z, 0.5f), g.sc));
        for (int wx = 0; wx < g.nxw; ++wx) {
            const int x = wx * 32 + lane;
            const float X = fadd(g.o[0], fmul(fadd((float)x, 0.5f), g.sc));
            const bool on = warp_test<NC>(cams, sil, X, Y, Z, x < g.nx, tests);
            const uint32_t word = __ballot_sync(kFull, on);
            if (on) {
                const uint32_t starts = word & ~(word << 1);   // first voxel of each run
                const int run0 = 31 - __clz(starts & (0xFFFFFFFFu >> (31 - lane)));
                parent[(int)(row * (uint32_t)g.nx) + x] = (int)(row * (uint32_t)g.nx) + wx * 32 + run0;
            }
            if (lane == 0) {
                bits[row * (uint32_t)g.nxw + (uint32_t)wx] = word;
                on_count += __popc(word);
            }
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

// Clears the fine grids and the compaction's chunk states, and resets the
// fine carve's tile counter.
__global__ void __launch_bounds__(256) k_clear_fine(const __grid_constant__ Layout L,
                                                    const __grid_constant__ SlotList sl) {
    pdl_begin();
    const int slot = sl.s[blockIdx.y];
    SlotInfo* info = slot_ptr<SlotInfo>(L, slot, L.info);
    const uint32_t nwords = info->n_words;
    uint32_t* fine = slot_ptr<uint32_t>(L, slot, L.fine);
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += gridDim.x * blockDim.x) fine[w] = 0u;
    // the compaction's look-back states of this reconstruction's chunks, and
    // each chunk's slab: words lo .. hi-1, hi past the farthest neighbour of
    // its words, in whole 16-byte units (the fine array is padded to 256
    // bytes), or 0 when that is more than kSlabWords
    const uint32_t nchunks = info->n_chunks;
    const int nrois = info->n_rois;
    const DRoi* rois = slot_ptr<DRoi>(L, slot, L.rois);
    unsigned long long* cst = slot_ptr<unsigned long long>(L, slot, L.chunk_st);
    uint32_t* clen = slot_ptr<uint32_t>(L, slot, L.chunk_len);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nchunks; i += gridDim.x * blockDim.x) {
        cst[2 * (size_t)i] = 0ull;
        cst[2 * (size_t)i + 1] = 0ull;
        const uint32_t lo = i * kChunk, last = min(lo + (uint32_t)kChunk, nwords) - 1u;
        const int k0 = roi_of_word(rois, nrois, lo), k1 = roi_of_word(rois, nrois, last);
        uint32_t reach = 0;
        for (int k = k0; k <= k1; ++k) {
            const uint32_t rs = (uint32_t)rois[k].nxw;
            reach = max(reach, 1u + rs + rs * (uint32_t)(rois[k].fdim[1] + 2));
        }
        const uint32_t n4 = (min(nwords, last + 1u + reach) - lo + 3u) & ~3u;
        clen[i] = n4 <= kSlabWords ? n4 : 0u;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) info->next_tile = 0u;
}

// The ROI holding fine-carve tile t: the last ROI whose first tile is <= t.
__device__ __forceinline__ int roi_of_tile(const DRoi* rois, int n, uint32_t t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rois[mid].tile_off <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Bits 0, 2, 4, ... of x packed into bits 0..15.
__device__ __forceinline__ uint32_t even_bits(uint32_t x) {
    x &= 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0F0F0F0Fu;
    x = (x | (x >> 4)) & 0x00FF00FFu;
    return (x | (x >> 8)) & 0x0000FFFFu;
}

// What every sample of a fine-carve tile sees in camera c (two lanes per
// camera, `half` = 0 or 1, each projecting four of the tile's eight extreme
// samples (cx[i], cy[j], cz[k])).  The box of their image positions, widened
// by the camera's error margin (Cam::seg_du, seg_dv), holds the pixel of
// every sample of the tile (two lanes per camera; the caller has all lanes
// call it).  fg_all: the box is inside the image and every
// pixel of it is set, so every sample votes foreground.  bg_all: no pixel of
// the box inside the image is set and (under STRICT, where a point outside
// the image votes background) the rest lies outside it, or (under ABSTAIN)
// the box is inside the image: every sample votes background.
template <bool ABSTAIN>
__device__ __forceinline__ void classify_tile_camera(const SmemCam& c, const uint32_t* __restrict__ sil,
                                                     const float* cx, const float* cy, const float* cz, int half,
                                                     bool& fg_all, bool& bg_all, uint32_t& reads) {
    // the two lanes of a camera take the same path through this function, so
    // they exchange values among themselves only
    const unsigned pm = 3u << ((threadIdx.x & 31u) & ~1u);
    float umin = 3.0e38f, umax = -3.0e38f, vmin = 3.0e38f, vmax = -3.0e38f;
    bool wpos = true;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int kk = half * 4 + q;
        float xh, yh, wh;
        project(c.P, cx[kk & 1], cy[(kk >> 1) & 1], cz[kk >> 2], xh, yh, wh);
        wpos &= wh > 0.0f;
        const float r = rcp_approx(wh);
        const float u = fmul(xh, r), v = fmul(yh, r);
        umin = fminf(umin, u); umax = fmaxf(umax, u);
        vmin = fminf(vmin, v); vmax = fmaxf(vmax, v);
    }
    umin = fminf(umin, __shfl_xor_sync(pm, umin, 1));
    umax = fmaxf(umax, __shfl_xor_sync(pm, umax, 1));
    vmin = fminf(vmin, __shfl_xor_sync(pm, vmin, 1));
    vmax = fmaxf(vmax, __shfl_xor_sync(pm, vmax, 1));
    const int wpos_other = __shfl_xor_sync(pm, (int)wpos, 1);   // both lanes, unconditionally
    wpos = wpos && wpos_other != 0;
    fg_all = bg_all = false;
    if (!wpos || !(c.du >= 0.0f)) return;
    const float u0 = fsub(umin, c.du), u1 = fadd(umax, c.du), v0 = fsub(vmin, c.dv), v1 = fadd(vmax, c.dv);
    if (!(u0 > -1.0e6f && u1 < 1.0e6f && v0 > -1.0e6f && v1 < 1.0e6f)) return;   // also NaN
    const int bx0 = (int)floorf(u0), bx1 = (int)floorf(u1), by0 = (int)floorf(v0), by1 = (int)floorf(v1);
    const bool inside = bx0 >= 0 && by0 >= 0 && bx1 < c.W && by1 < c.H;
    // the part of the box inside the image
    const int x0 = max(bx0, 0), x1 = min(bx1, c.W - 1), y0 = max(by0, 0), y1 = min(by1, c.H - 1);
    if (x0 > x1 || y0 > y1) {            // entirely outside the image
        bg_all = !ABSTAIN;
        return;
    }
    if (x1 - x0 > 31 || y1 - y0 > 15) return;   // too large to scan: undecided
    const int w0 = x0 >> 5, w1 = x1 >> 5;
    const uint32_t m0 = ~0u << (x0 & 31), m1 = ~0u >> (31 - (x1 & 31));
    bool all = true, any = false;
    for (int y = y0 + half; y <= y1; y += 2) {     // the two lanes take alternate rows
        const uint32_t* row = sil + c.bit_off + (unsigned)y * (unsigned)c.Wq;
        if (w0 == w1) {
            const uint32_t m = m0 & m1, v = __ldg(row + w0) & m;
            all &= v == m;
            any |= v != 0u;
        } else {
            const uint32_t va = __ldg(row + w0) & m0, vb = __ldg(row + w1) & m1;
            all &= va == m0 && vb == m1;
            any |= (va | vb) != 0u;
        }
        reads += (unsigned)(w1 - w0 + 1);
    }
    const int all_other = __shfl_xor_sync(pm, (int)all, 1), any_other = __shfl_xor_sync(pm, (int)any, 1);
    all = all && all_other != 0;
    any = any || any_other != 0;
    fg_all = inside && all;
    bg_all = !any && (inside || !ABSTAIN);
}

// Sec. II-B-3: the fine hull of every ROI, each treated as its own volume.
// Fine grids are stored padded by one unoccupied sample per side (index 0
// and fdim+1), rows of ceil((fdim_x+2)/32) words, cleared beforehand; only
// occupied samples are written, by OR into their word.
//
// A warp takes a tile of 4 x 4 x 8 interior samples (x, y, z) and first
// decides, per camera, whether all of the tile's samples vote foreground or
// all vote background there (classify_tile_camera); then it takes the tile's
// samples 4 x 2 x 4 at a time, one per lane.  A
// sample's first background camera in index order is then either an
// undecided camera before the tile's first all-background camera, where it
// is tested, or that camera; so each sample projects and looks its pixel up
// only at those undecided cameras, and its test count (first background
// camera + 1, or N when occupied) and occupancy are those of the plain
// per-sample loop.
template <int NC, bool ABSTAIN, int TY, int TZ>
__device__ __forceinline__ void fine_tiles(const CamSet& cams, const Grid& g, const SmemCam* sc, int ncam,
                                           uint32_t ntiles, int nrois, const DRoi* rois,
                                           const uint32_t* __restrict__ sil, uint32_t* fine,
                                           uint32_t* next_tile, uint32_t& tests, uint32_t& reads) {
    const int lane = threadIdx.x & 31, half = lane & 1;
    const int xi = lane & 3, yi = (lane >> 2) & 1, zi = lane >> 3;
    // ROI of the current tile (the same in every lane)
    uint32_t lo = 0, hi = 0, woff = 0;
    int fx = 1, fy = 1, fz = 1, nxw = 1, ntx = 1, nty = 1;
    float fo0 = 0.f, fo1 = 0.f, fo2 = 0.f;
    // tiles differ a lot in cost (a surface tile tests many cameras, an
    // empty one few), so each warp claims its next tile from a counter
    for (;;) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(next_tile, 1u);
        t = __shfl_sync(kFull, t, 0);
        if (t >= ntiles) break;
        if (t >= hi || t < lo) {
            const DRoi& r = rois[roi_of_tile(rois, nrois, t)];
            lo = r.tile_off;
            fx = r.fdim[0];
            fy = r.fdim[1];
            fz = r.fdim[2];
            ntx = (fx + kTileX - 1) / kTileX;
            nty = (fy + TY - 1) / TY;
            hi = lo + (uint32_t)ntx * (uint32_t)nty * (uint32_t)((fz + TZ - 1) / TZ);
            woff = r.word_off;
            nxw = r.nxw;
            fo0 = r.fo[0];
            fo1 = r.fo[1];
            fo2 = r.fo[2];
        }
        const uint32_t lt = t - lo;
        const uint32_t r1 = lt / (uint32_t)ntx;
        const int tx = (int)(lt - r1 * (uint32_t)ntx), ty = (int)(r1 % (uint32_t)nty), tz = (int)(r1 / (uint32_t)nty);
        const int x0 = tx * kTileX, y0 = ty * TY, z0 = tz * TZ;
        // the tile's extreme samples
        const int xs[2] = {x0, min(x0 + kTileX - 1, fx - 1)};
        const int ys[2] = {y0, min(y0 + TY - 1, fy - 1)};
        const int zs[2] = {z0, min(z0 + TZ - 1, fz - 1)};
        float cx[2], cy[2], cz[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            cx[e] = fadd(fo0, fmul(fadd((float)xs[e], 0.5f), g.sf));
            cy[e] = fadd(fo1, fmul(fadd((float)ys[e], 0.5f), g.sf));
            cz[e] = fadd(fo2, fmul(fadd((float)zs[e], 0.5f), g.sf));
        }
        // bit n: every sample votes foreground (fgm) / background (bgm) in camera n
        uint64_t fgm = 0, bgm = 0;
        for (int cg = 0; cg < ncam; cg += 16) {
            const int cam = cg + (lane >> 1);
            bool fg, bg;
            uint32_t r = 0;
            classify_tile_camera<ABSTAIN>(sc[min(cam, ncam - 1)], sil, cx, cy, cz, half, fg, bg, r);
            if (cam < ncam) reads += r;
            fg = fg && cam < ncam;
            bg = bg && cam < ncam;
            fgm |= (uint64_t)even_bits(__ballot_sync(kFull, fg)) << cg;
            bgm |= (uint64_t)even_bits(__ballot_sync(kFull, bg)) << cg;
        }
        // the tile's samples, one sub-tile of 4 x 2 x 4 (one per lane) at a time
        const int nb = bgm ? __ffsll((long long)bgm) - 1 : ncam;
        const uint64_t before = nb >= 64 ? ~0ull : (1ull << nb) - 1ull;
        constexpr int kSubsY = TY / kSubY, kSubTiles = kSubsY * (TZ / kSubZ);
        if (nb < ncam && (~(fgm | bgm) & before) == 0ull) {
            // Every camera before the first all-background one votes
            // foreground on the whole tile: each sample stops at camera nb
            // (nb + 1 tests) and none is occupied.  Count this lane's samples
            // of the sub-tile walk below without walking it.
            const int dy = fy - y0 - yi, dz = fz - z0 - zi;
            const int ny_ = dy > 0 ? min((dy + kSubY - 1) / kSubY, kSubsY) : 0;
            const int nz_ = dz > 0 ? min((dz + kSubZ - 1) / kSubZ, TZ / kSubZ) : 0;
            if (x0 + xi < fx) tests += (unsigned)(ny_ * nz_ * (nb + 1));
            continue;
        }
        for (int sub = 0; sub < kSubTiles; ++sub) {
            const int sy0 = y0 + (sub % kSubsY) * kSubY, sz0 = z0 + (sub / kSubsY) * kSubZ;
            if (sy0 >= fy || sz0 >= fz) continue;          // the same in every lane
            // this lane's sample
            const int x = x0 + xi, y = sy0 + yi, z = sz0 + zi;
            const bool act = x < fx && y < fy && z < fz;
            const float X = fadd(fo0, fmul(fadd((float)x, 0.5f), g.sf));
            const float Y = fadd(fo1, fmul(fadd((float)y, 0.5f), g.sf));
            const float Z = fadd(fo2, fmul(fadd((float)z, 0.5f), g.sf));
            // In camera order: the first all-background camera nb stops every
            // sample still alive there; before it, all-foreground cameras pass
            // every sample and only the undecided ones are tested, per lane.
            uint64_t todo = ~(fgm | bgm) & before;
            bool alive = act, voted = !ABSTAIN || (fgm & before) != 0ull;
            int stop = -1;
            while (todo && __any_sync(kFull, alive)) {
                const int n = __ffsll((long long)todo) - 1;
                todo &= todo - 1ull;
                if (alive) {
                    bool in;
                    const uint32_t bit = cam_bit(sc[n], sil, X, Y, Z, in);
                    reads += in ? 1u : 0u;
                    if (ABSTAIN ? (in && !bit) : !bit) {
                        alive = false;
                        stop = n;
                    }
                    voted |= bit != 0u;
                }
            }
            if (act) tests += stop >= 0 ? (unsigned)(stop + 1) : (nb < ncam ? (unsigned)(nb + 1) : (unsigned)ncam);
            alive = alive && nb >= ncam;
            const bool on = alive && voted;
            // OR the occupied samples into their words: the four lanes of one
            // (y, z) row span at most two words
            if (__any_sync(kFull, on)) {
                const uint32_t word = woff + ((uint32_t)(z + 1) * (uint32_t)(fy + 2) + (uint32_t)(y + 1)) * (uint32_t)nxw +
                                      (uint32_t)((x + 1) >> 5);
                const uint32_t first = __shfl_sync(kFull, word, lane & ~3);
                const uint32_t bit = on ? 1u << ((x + 1) & 31) : 0u;
                uint32_t blo = word == first ? bit : 0u, bhi = word == first ? 0u : bit;
                blo |= __shfl_xor_sync(kFull, blo, 1);
                bhi |= __shfl_xor_sync(kFull, bhi, 1);
                blo |= __shfl_xor_sync(kFull, blo, 2);
                bhi |= __shfl_xor_sync(kFull, bhi, 2);
                if (xi == 0) {
                    if (blo) atomicOr(fine + first, blo);
                    if (bhi) atomicOr(fine + first + 1, bhi);
                }
            }
        }
    }
}

template <int NC, int TY, int TZ>
__global__ void __launch_bounds__(256) k_fine_carve(const __grid_constant__ CamSet cams,
                                                    const __grid_constant__ Grid g,
                                                    const __grid_constant__ Layout L,
                                                    const __grid_constant__ SlotList sl) {
    pdl_begin();
    __shared__ unsigned long long sh_t[32];
    __shared__ SmemCam sc[FVV_MAX_CAMS];
    const int ncam = NC > 0 ? NC : cams.n;
    load_smem_cams(cams, ncam, sc);
    __syncthreads();
    const int slot = sl.s[blockIdx.y];
    const SlotInfo* info = slot_ptr<SlotInfo>(L, slot, L.info);
    const uint32_t ntiles = info->n_words ? info->n_tiles : 0u;
    const int nrois = info->n_rois;
    const DRoi* rois = slot_ptr<DRoi>(L, slot, L.rois);
    const uint32_t* __restrict__ sil = slot_ptr<uint32_t>(L, slot, L.sil);
    uint32_t* fine = slot_ptr<uint32_t>(L, slot, L.fine);
    uint32_t* next_tile = &slot_ptr<SlotInfo>(L, slot, L.info)->next_tile;
    // per-lane counts stay below 2^30 (at most 2^24 tiles of 64 tests each)
    uint32_t tests = 0, reads = 0;
    if (cams.oob == FVV_OOB_ABSTAIN)
        fine_tiles<NC, true, TY, TZ>(cams, g, sc, ncam, ntiles, nrois, rois, sil, fine, next_tile, tests, reads);
    else
        fine_tiles<NC, false, TY, TZ>(cams, g, sc, ncam, ntiles, nrois, rois, sil, fine, next_tile, tests, reads);
    const unsigned long long t = block_sum<unsigned long long>((unsigned long long)tests, sh_t);
    const unsigned long long rd = block_sum<unsigned long long>((unsigned long long)reads, sh_t);
    if (threadIdx.x == 0 && t) atomicAdd(&slot_ptr<SlotInfo>(L, slot, L.info)->tests_fine, t);
    if (threadIdx.x == 0 && rd) atomicAdd(&slot_ptr<SlotInfo>(L, slot, L.info)->look_fine, rd);
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

cudaError_t launch_pack(const CamSet& cams, const Layout& L, int n_frames, const int* slots,
                        const uint8_t* const* src, bool host_src, int sms, cudaStream_t st) {
    size_t max_words = 0;
    for (int n = 0; n < cams.n; ++n) max_words = std::max(max_words, (size_t)cams.c[n].H * (unsigned)cams.c[n].Wq);
    const int per_launch = std::min(kPackPtrs / 4, kPackPtrs / std::max(1, cams.n));
    // Device sources: enough blocks to stream HBM at full rate.  Masks read in
    // place from host memory are bound by the host link, which about two
    // blocks per SM keep busy; the rest of the GPU stays free for the work
    // of other streams meanwhile.
    const size_t cap = host_src ? (size_t)std::max(1, 2 * sms / std::max(1, cams.n * std::min(n_frames, per_launch)))
                                : (size_t)2048;
    const unsigned gx = (unsigned)std::max<size_t>(1, std::min<size_t>((max_words + 255) / 256, cap));
    static_assert(sizeof(CamSet) + sizeof(PackSrc) + sizeof(Layout) <= 32764, "k_pack parameters");
    thread_local PackSrc a;   // 18 KB: kept off the stack
    for (int j0 = 0; j0 < n_frames; j0 += per_launch) {
        const int nf = std::min(per_launch, n_frames - j0);
        for (int j = 0; j < nf; ++j) {
            a.slot[j] = slots[j0 + j];
            for (int n = 0; n < cams.n; ++n) a.src[j * cams.n + n] = src[(size_t)(j0 + j) * cams.n + n];
        }
        const cudaError_t e = launch_pdl(k_pack, dim3(gx, cams.n, nf), dim3(256), 0, st, cams, a, L);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t launch_coarse_carve(const CamSet& cams, const Grid& g, const Layout& L, const SlotList& sl, int sms,
                                const Tuning& tu, cudaStream_t st) {
    const long long rows = (long long)g.nz * g.ny;    // a warp per row
    const int th = tu.threads[FVV_TUNE_COARSE];
    const int gx = tuned_grid(tu, FVV_TUNE_COARSE, sms, sl.n, rows * 32);
#define FVV_LAUNCH(NC) launch_pdl(k_coarse_carve<NC>, dim3(gx, sl.n), dim3(th), 0, st, cams, g, L, sl)
    FVV_DISPATCH_NC(cams.n, FVV_LAUNCH)
#undef FVV_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_fine_carve(const CamSet& cams, const Grid& g, const Layout& L, const SlotList& sl, int sms,
                              const Tuning& tu, cudaStream_t st) {
    const int gc = grid_x(sms, sl.n, (long long)g.max_fine_words, 256);
    launch_pdl(k_clear_fine, dim3(gc, sl.n), dim3(256), 0, st, L, sl);
    const int th = tu.threads[FVV_TUNE_FINE];
    const int gx = tuned_grid(tu, FVV_TUNE_FINE, sms, sl.n, (long long)g.max_fine_words * 32);
    // the tile shape (tile_y, tile_z) the k_filter of this sequence counted tiles with
    if (g.tile_y == 4 && g.tile_z == 4) {
#define FVV_LAUNCH(NC) launch_pdl(k_fine_carve<NC, 4, 4>, dim3(gx, sl.n), dim3(th), 0, st, cams, g, L, sl)
        FVV_DISPATCH_NC(cams.n, FVV_LAUNCH)
#undef FVV_LAUNCH
    } else if (g.tile_y == 8 && g.tile_z == 8) {
#define FVV_LAUNCH(NC) launch_pdl(k_fine_carve<NC, 8, 8>, dim3(gx, sl.n), dim3(th), 0, st, cams, g, L, sl)
        FVV_DISPATCH_NC(cams.n, FVV_LAUNCH)
#undef FVV_LAUNCH
    } else {
#define FVV_LAUNCH(NC) launch_pdl(k_fine_carve<NC, 4, 8>, dim3(gx, sl.n), dim3(th), 0, st, cams, g, L, sl)
        FVV_DISPATCH_NC(cams.n, FVV_LAUNCH)
#undef FVV_LAUNCH
    }
    return cudaGetLastError();
}

}  // namespace fvv
