// fvv_internal.h -- device-side data layout and kernel launchers of libfvv.
//
// Everything a kernel needs about the rig travels by value in kernel
// parameters (cameras, grid, per-slot arena layout); everything per frame
// lives in the slot's part of the arena.  Launchers enqueue on a stream and
// never synchronise.
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/fvv.h"

namespace fvv {

constexpr int kMaxComponents = 8192;  // raw components sortable by one block
// Words of the slab the MC compaction stages per 256-word chunk: the chunk
// and the neighbours its cells reach (a word in +x, a row in +y, a plane in
// +z).  Chunks whose ROIs reach further read global memory instead.
constexpr uint32_t kSlabWords = 6144;
constexpr int kMaxRois = 4096;
constexpr int kChunk = 256;           // fine words per scan chunk (= block size)
constexpr uint32_t kEmptyDepth = 0xFFFFFFFFu;  // depth-buffer bits meaning +inf
constexpr int kMaxTriPerCell = 12;

struct Cam {
    float P[12];
    float C[3];
    int W, H, Wq;        // Wq = 32-bit words per silhouette row
    float Wf, Hf;        // W and H as floats
    uint32_t bit_off;    // first silhouette word of this camera in a slot
    uint64_t pix_off;    // first pixel of this camera in per-slot pixel arrays
    // Bound (pixels) on how far the computed image position of any point the
    // bisection of a grid edge can test lies from the box of the edge ends'
    // approximate image positions; negative: no bound (the camera can see
    // part of the volume at w' <= 0).  See segment_margins in fvv_api.cu.
    float seg_du, seg_dv;
};

struct CamSet {
    int n;
    int oob;             // FVV_OOB_*
    Cam c[FVV_MAX_CAMS];
};

struct Grid {
    float o[3];          // volume origin (vol_min)
    float sc, sf;        // coarse and fine steps
    int nx, ny, nz, nxw; // coarse dims, words per coarse row
    long long coarse_um, fine_um;
    int steps;           // bisection steps
    int rule;            // FVV_SURFACE_*
    int t_np, t_nb;
    float t_v;
    int max_comp, max_rois;
    uint32_t max_fine_words, max_chunks;
    uint32_t max_verts, max_tris;
    int tile_y, tile_z;  // fine-carve tile shape of this launch sequence (kFineTiles)
};

// Fine-carve tiles: kTileX x tile_y x tile_z interior samples, classified
// per camera once and tested in sub-tiles of 4 x kSubY x kSubZ samples, one
// per lane.  The autotuner picks the shape among kFineTiles (FVV_TILE_*).
constexpr int kTileX = 4;
constexpr int kSubY = 2, kSubZ = 4;
constexpr int kFineTiles[FVV_N_TILES][2] = {{4, 8}, {4, 4}, {8, 8}};   // (tile_y, tile_z)

// Per-slot device bookkeeping (zeroed at the start of each reconstruction).
struct SlotInfo {
    unsigned int flags;
    int n_roots;
    int n_rois;
    uint32_t n_words;           // fine words in use
    uint32_t n_chunks;
    uint32_t n_tiles;           // fine-carve tiles of all ROIs
    uint32_t next_tile;         // the fine carve's next unclaimed tile
    uint32_t next_chunk;        // the compaction's next unclaimed 256-word chunk
    uint32_t n_verts, n_tris;
    uint32_t n_on;
    unsigned long long tests_coarse, tests_fine, tests_bisect;
    unsigned long long look_fine, look_bisect;   // silhouette words read
};

// Device ROI record (one per kept component).
struct DRoi {
    int cmin[3], cmax[3], gmin[3], gmax[3], fdim[3];
    float fo[3];
    int count;
    int nxw;                    // words per padded fine row
    uint32_t word_off;          // first fine word of this ROI in the slot
    uint32_t n_words;
    uint32_t tile_off;          // first fine-carve tile of this ROI in the slot
    uint32_t vert_off, tri_off; // filled after the scans (for fvv_roi)
};

// Offsets (bytes) of each per-slot array from the slot base.  All 256-aligned.
struct Layout {
    char* base;                 // arena + slots region
    size_t stride;              // bytes per slot
    size_t info;                // SlotInfo
    size_t sil;                 // uint32 silhouette bits
    size_t coarse;              // uint32 coarse bits (nz*ny*nxw)
    size_t parent;              // int32 union-find parents, nx*ny*nz
    size_t roots;               // int32 root linear indices, max_comp
    size_t cstat;               // int32 per component: count, min xyz, max xyz (7 each)
    size_t rois;                // DRoi, max_rois
    size_t roi_label;           // int32 label per sorted component (0 = removed)
    size_t fine;                // uint32 fine bits, max_fine_words
    size_t emask;               // uint32 x3 bipolar-edge masks per fine word
    size_t vpre;                // uint32 exclusive vertex prefix per fine word
    size_t chunk_st;            // uint64 x2 per 256-word chunk: look-back states (vertices, triangles)
    size_t chunk_len;           // uint32 per chunk: words of its staged slab (a multiple of 4), 0: not staged
    size_t vrec;                // uint64 vertex records, max_verts
    size_t verts;               // float x3, max_verts
    size_t tris;                // uint32 x3, max_tris
    size_t tsoup;               // float4 x3 per triangle: its vertices and centroid
                                // (v0 xyz, v1 xyz, v2 xyz, centroid xyz), max_tris
    size_t trec;                // uint64 triangle records (word, cell, case, triangle, ROI), max_tris
    size_t vrgb;                // uint8 x3, max_verts
    size_t vcam;                // int32, max_verts
    size_t depth;               // uint32 per pixel of all cameras
    size_t dbox;                // int32 x4 per camera: box of the depth pixels the last z-buffer wrote
    size_t mask_stage;          // uint8 per pixel (host uploads), or 0
    size_t rgb_stage;           // uint8 x3 per pixel (host uploads), or 0
};

template <typename T>
__host__ __device__ inline T* slot_ptr(const Layout& L, int slot, size_t off) {
    return reinterpret_cast<T*>(L.base + (size_t)slot * L.stride + off);
}

struct SlotList {
    int n;
    int s[FVV_MAX_BATCH];
};

// Marching-cubes table in device memory.
struct McTable {
    const uint8_t* ntri;        // [256]
    const uint8_t* edges;       // [256][12][3]
};

// Blocks per slot for a grid-stride kernel: enough for the work, at most
// about 8 blocks per SM over the whole batch.
inline int grid_x(int sms, int n_slots, long long work_items, int per_block) {
    const long long want = (work_items + per_block - 1) / per_block;
    const long long cap = std::max(1LL, (long long)sms * 8 / std::max(1, n_slots));
    return (int)std::max(1LL, std::min(want, cap));
}

// Launch shape of the tunable kernels (index FVV_TUNE_*): threads per block
// (a multiple of 32, <= 256) and resident blocks per SM over the whole batch.
struct Tuning {
    int threads[FVV_N_TUNE];
    int waves[FVV_N_TUNE];
    int fine_tile;       // index into kFineTiles
    int zb_cams;         // cameras per z-buffer block: 1, 2 or 4
};

// The grid with the tuned fine-carve tile shape.
inline Grid tuned_grid_params(const Grid& g, const Tuning& tu) {
    Grid out = g;
    out.tile_y = kFineTiles[tu.fine_tile][0];
    out.tile_z = kFineTiles[tu.fine_tile][1];
    return out;
}

inline Tuning default_tuning() {
    Tuning t;
    for (int k = 0; k < FVV_N_TUNE; ++k) {
        t.threads[k] = 256;
        t.waves[k] = 8;
    }
    t.waves[FVV_TUNE_ZBUFFER] = 16;
    t.fine_tile = FVV_TILE_4x4x8;
    t.zb_cams = 4;
    return t;
}

// Blocks per slot of a tuned grid-stride kernel: the tuned blocks per SM
// spread over the launch's slots, but never more than kMaxWavesPerSlot per
// SM for one slot (one frame's work is too little for more: with the
// shapes tuned on a 64-frame batch at 64 blocks per SM, one frame took
// 0.561 ms at p50 uncapped and 0.531 ms capped at 16).
constexpr int kMaxWavesPerSlot = 16;
inline int tuned_grid(const Tuning& tu, int knob, int sms, int n_slots, long long work_items, int parts = 1) {
    const long long per_block = tu.threads[knob];
    const long long want = (work_items + per_block - 1) / per_block;
    const long long cap = std::max(1LL, (long long)sms * std::min(tu.waves[knob], kMaxWavesPerSlot * n_slots) /
                                            std::max(1, n_slots * parts));
    return (int)std::max(1LL, std::min(want, cap));
}

// Builds the 256-case table from the face rule (host).
void build_mc_table(uint8_t ntri[256], uint8_t edges[256 * kMaxTriPerCell * 3]);

// ---- launchers (all enqueue on `st`)
// Packs frame j's masks (src[j * cams.n + n]) into slots[j], j < n_frames;
// host_src: the sources are mapped page-locked host memory.
cudaError_t launch_pack(const CamSet& cams, const Layout& L, int n_frames, const int* slots,
                        const uint8_t* const* src, bool host_src, int sms, cudaStream_t st);
cudaError_t launch_coarse_carve(const CamSet& cams, const Grid& g, const Layout& L, const SlotList& sl,
                                int sms, const Tuning& tu, cudaStream_t st);
cudaError_t launch_ccl(const Grid& g, const Layout& L, const SlotList& sl, int sms, cudaStream_t st);
// The filter and ROI table alone (k_filter), e.g. again for another fine-carve tile shape.
cudaError_t launch_filter(const Grid& g, const Layout& L, const SlotList& sl, cudaStream_t st);
cudaError_t launch_fine_carve(const CamSet& cams, const Grid& g, const Layout& L, const SlotList& sl,
                              int sms, const Tuning& tu, cudaStream_t st);
cudaError_t launch_mc_prefix(const Grid& g, const Layout& L, const SlotList& sl, const McTable& mc, int sms,
                             cudaStream_t st);
cudaError_t launch_bisect(const CamSet& cams, const Grid& g, const Layout& L, const SlotList& sl, int sms,
                          const Tuning& tu, cudaStream_t st);
cudaError_t launch_mc_triangles(const Grid& g, const Layout& L, const SlotList& sl, const McTable& mc, int sms,
                                const Tuning& tu, cudaStream_t st);
// Depth images of every slot to empty and their written boxes to none (once,
// when a rig is created).
cudaError_t launch_init_depth(const CamSet& cams, const Layout& L, int n_slots, int sms, cudaStream_t st);
cudaError_t launch_depth(const CamSet& cams, const Grid& g, const Layout& L, const SlotList& sl,
                         int sms, size_t depth_bytes, const Tuning& tu, cudaStream_t st);
// Colour-call arguments of up to kColourBatch slots, passed by value as a
// kernel parameter (so nothing is copied from host memory).
constexpr int kColourBatch = 48;
struct ColourBatch {
    int n;
    int slot[kColourBatch];
    float view[kColourBatch][3];
    const uint8_t* rgb[kColourBatch][FVV_MAX_CAMS];
};

cudaError_t launch_colour(const CamSet& cams, const Grid& g, const Layout& L, const ColourBatch& cb, int sms,
                          int total_slots, cudaStream_t st);

// A novel view (step E) of one reconstructed slot: the virtual camera as a
// Cam (P, C, W, H, Wf, Hf; the other fields unused) and the capture RGB.
struct ViewArgs {
    Cam v;
    int slot;
    const uint8_t* rgb[FVV_MAX_CAMS];
};

cudaError_t launch_render_view(const CamSet& cams, const Grid& g, const Layout& L, const ViewArgs& va,
                              unsigned long long* key, uint8_t* out_rgb, int32_t* out_cam, int sms, cudaStream_t st);
cudaError_t launch_debug_pixels(const CamSet& cams, int cam, long long n, const float* pts, int32_t* px,
                                int32_t* py, cudaStream_t st);
cudaError_t launch_debug_labels(const Grid& g, const Layout& L, int slot, int32_t* dst, cudaStream_t st);
// Writes a given coarse grid into slot and seeds its union-find forest as the
// coarse hull does (the slot's SlotInfo must be zeroed first).
cudaError_t launch_debug_seed(const Grid& g, const Layout& L, int slot, const uint32_t* src, cudaStream_t st);
cudaError_t launch_debug_depth(const CamSet& cams, const Layout& L, int slot, float* dst, size_t npix,
                               cudaStream_t st);

}  // namespace fvv
