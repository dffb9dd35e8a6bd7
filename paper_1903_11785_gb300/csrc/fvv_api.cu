// fvv_api.cu -- the C ABI of libfvv (include/fvv.h): rig creation and arena
// layout, argument checking, and the launch sequences of each call.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fvv_device.cuh"

using namespace fvv;

struct fvv_rig {
    CamSet cams;
    Grid grid;
    Layout L;
    int max_slots = 0;
    int host_staging = 0;
    int device = 0;
    int sms = 1;
    char* arena = nullptr;
    size_t arena_bytes = 0;
    bool own_arena = false;
    uint8_t* mc_ntri = nullptr;    // device
    uint8_t* mc_edges = nullptr;   // device
    size_t sil_words = 0, npix = 0;
    std::vector<int> state;        // per slot: 0 empty, 1 uploaded, 2 reconstructed
    std::string err;
    // per-stage timing: CUDA events around each stage, summed on request
    bool timing = false;
    std::vector<cudaEvent_t> events;   // pool, reused after every fvv_get_timing
    size_t events_used = 0;
    struct Interval { int stage; cudaEvent_t a, b; };
    std::vector<Interval> intervals;
    Tuning tune = default_tuning();
    // CUDA graphs of fvv_reconstruct, one per slot list (least recently used dropped)
    bool graphs = false;
    struct Graph { std::vector<int> slots; cudaGraphExec_t exec; unsigned long long used; };
    std::vector<Graph> graph_cache;
    unsigned long long graph_clock = 0;
    SlotInfo* host_info = nullptr;   // page-locked, FVV_MAX_BATCH entries: counts read by fvv_get_results_batch
};

namespace {

thread_local std::string g_create_err;

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

fvv_status fail(fvv_rig* rig, fvv_status st, const std::string& msg) {
    if (rig) rig->err = msg;
    else g_create_err = msg;
    return st;
}

fvv_status cuda_fail(fvv_rig* rig, cudaError_t e, const char* what) {
    return fail(rig, FVV_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

long long um_of(float m) { return llround((double)m * 1e6); }

// Per camera, the margins seg_du, seg_dv used by the bisection to decide,
// once per grid edge, that a camera sees every point of the edge in its
// silhouette.  Every point a bisection tests lies within 2^-19 |X| per
// coordinate of the edge (at most 30 midpoints, each rounded by half an ulp)
// and inside the box B = the grid grown by one coarse and two fine voxels
// (ROI overshoot and padding samples).  For a row r of P, the computed
// binary32 value ((p3 + p2 Z) + p1 Y) + p0 X (three fused multiply-adds)
// differs from the exact value at the nearest edge point by at most
// 2^-18 S_r, with S_r = sum |p_rj| max_B |X_j| + |p_r3| (three roundings of
// at most 2^-24 relative to S_r, plus the point's deviation).  With w' >= w_min - 2^-18 S_w > 0 on B and |u| <= W + 1
// inside the image, the computed u = x'/w' of a tested point lies within
// 2^-18 (S_x + (W + 1) S_w) / (w_min - 2^-18 S_w) of the exact projection of
// an edge point, which lies between the exact projections of the ends (a
// projective map keeps segments straight).  The ends' approximate positions
// carry the same error plus that of rcp.approx and one multiply (below
// (W + 2) 2^-21), so the margin is twice the first term plus that, plus 2^-12.
void segment_margins(CamSet& cs, const Grid& g) {
    double lo[3], hi[3];
    const int dims[3] = {g.nx, g.ny, g.nz};
    for (int a = 0; a < 3; ++a) {
        const double pad = (double)g.sc + 2.0 * (double)g.sf;
        lo[a] = (double)g.o[a] - pad;
        hi[a] = (double)g.o[a] + (double)dims[a] * (double)g.sc + pad;
    }
    const double e = std::ldexp(1.0, -18);
    for (int n = 0; n < cs.n; ++n) {
        Cam& c = cs.c[n];
        double S[3], wmin = 1e300;
        for (int r = 0; r < 3; ++r) {
            S[r] = std::fabs((double)c.P[4 * r + 3]);
            for (int j = 0; j < 3; ++j)
                S[r] += std::fabs((double)c.P[4 * r + j]) * std::max(std::fabs(lo[j]), std::fabs(hi[j]));
        }
        for (int k = 0; k < 8; ++k) {
            const double X = (k & 1) ? hi[0] : lo[0], Y = (k & 2) ? hi[1] : lo[1], Z = (k & 4) ? hi[2] : lo[2];
            wmin = std::min(wmin, (double)c.P[8] * X + (double)c.P[9] * Y + (double)c.P[10] * Z + (double)c.P[11]);
        }
        const double den = wmin - e * S[2];
        if (!(den > 0.0)) {
            c.seg_du = c.seg_dv = -1.0f;
            continue;
        }
        const double du = 2.0 * e * (S[0] + (c.W + 1.0) * S[2]) / den + (c.W + 2.0) * std::ldexp(1.0, -21) +
                          std::ldexp(1.0, -12);
        const double dv = 2.0 * e * (S[1] + (c.H + 1.0) * S[2]) / den + (c.H + 2.0) * std::ldexp(1.0, -21) +
                          std::ldexp(1.0, -12);
        c.seg_du = (float)(du * (1.0 + 1e-6));
        c.seg_dv = (float)(dv * (1.0 + 1e-6));
    }
}

struct Plan {
    CamSet cams;
    Grid grid;
    Layout L;        // offsets only (base unset)
    size_t common = 0;   // bytes before the slots region
    size_t total = 0;
    size_t sil_words = 0, npix = 0;
};

// Validate the arguments and lay out the arena.
fvv_status make_plan(const fvv_rig_desc* d, const fvv_recon_params* p, Plan& pl, std::string& err) {
    if (!d || !p) { err = "desc and params must not be NULL"; return FVV_ERR_INVALID_ARG; }
    if (d->n_cams < 1 || d->n_cams > FVV_MAX_CAMS) { err = "n_cams must be 1..64"; return FVV_ERR_INVALID_ARG; }
    if (!d->P || !d->centre || !d->width || !d->height) { err = "camera arrays must not be NULL"; return FVV_ERR_INVALID_ARG; }
    if (d->max_slots < 1 || d->max_slots > 65536) { err = "max_slots must be 1..65536"; return FVV_ERR_INVALID_ARG; }
    CamSet& cs = pl.cams;
    std::memset(&cs, 0, sizeof(cs));
    cs.n = d->n_cams;
    if (p->oob_policy != FVV_OOB_STRICT && p->oob_policy != FVV_OOB_ABSTAIN) { err = "bad oob_policy"; return FVV_ERR_INVALID_ARG; }
    cs.oob = p->oob_policy;
    size_t words = 0, pix = 0;
    for (int n = 0; n < cs.n; ++n) {
        Cam& c = cs.c[n];
        for (int k = 0; k < 12; ++k) {
            c.P[k] = d->P[12 * n + k];
            if (!std::isfinite(c.P[k])) { err = "P must be finite"; return FVV_ERR_INVALID_ARG; }
        }
        for (int k = 0; k < 3; ++k) {
            c.C[k] = d->centre[3 * n + k];
            if (!std::isfinite(c.C[k])) { err = "centre must be finite"; return FVV_ERR_INVALID_ARG; }
        }
        c.W = d->width[n];
        c.H = d->height[n];
        if (c.W < 1 || c.W > 65535 || c.H < 1 || c.H > 65535) { err = "image sizes must be 1..65535"; return FVV_ERR_INVALID_ARG; }
        c.Wq = (c.W + 31) / 32;
        c.Wf = (float)c.W;
        c.Hf = (float)c.H;
        c.bit_off = (uint32_t)words;
        c.pix_off = pix;
        words += (size_t)c.H * c.Wq;
        pix += (size_t)c.H * c.W;
        if (words >= (1ull << 32)) { err = "silhouettes too large"; return FVV_ERR_INVALID_ARG; }
    }
    pl.sil_words = words;
    pl.npix = pix;
    Grid& g = pl.grid;
    std::memset(&g, 0, sizeof(g));
    if (!(p->coarse_m > 0) || !(p->fine_m > 0) || !std::isfinite(p->coarse_m) || !std::isfinite(p->fine_m)) {
        err = "voxel sizes must be positive"; return FVV_ERR_INVALID_ARG;
    }
    g.coarse_um = um_of(p->coarse_m);
    g.fine_um = um_of(p->fine_m);
    if (g.coarse_um < 1 || g.fine_um < 1) { err = "voxel sizes must be >= 1 micrometre"; return FVV_ERR_INVALID_ARG; }
    int dims[3];
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(p->vol_min[a]) || !std::isfinite(p->vol_max[a])) { err = "volume must be finite"; return FVV_ERR_INVALID_ARG; }
        const long long span = um_of(p->vol_max[a]) - um_of(p->vol_min[a]);
        if (span <= 0) { err = "vol_max must exceed vol_min"; return FVV_ERR_INVALID_ARG; }
        const long long n = (span + g.coarse_um - 1) / g.coarse_um;
        if (n > 32767) { err = "coarse grid too large"; return FVV_ERR_INVALID_ARG; }
        dims[a] = (int)n;
        g.o[a] = p->vol_min[a];
    }
    g.nx = dims[0]; g.ny = dims[1]; g.nz = dims[2];
    if ((long long)g.nx * g.ny * g.nz >= (1ll << 31)) { err = "coarse grid too large"; return FVV_ERR_INVALID_ARG; }
    g.nxw = (g.nx + 31) / 32;
    g.sc = p->coarse_m;
    g.sf = p->fine_m;
    if (p->bisect_steps < 0 || p->bisect_steps > 30) { err = "bisect_steps must be 0..30"; return FVV_ERR_INVALID_ARG; }
    segment_margins(cs, g);
    g.steps = p->bisect_steps;
    if (p->surface_rule != FVV_SURFACE_BISECT && p->surface_rule != FVV_SURFACE_LAMBDA) {
        err = "bad surface_rule";
        return FVV_ERR_INVALID_ARG;
    }
    g.rule = p->surface_rule;
    g.t_np = p->t_np;
    g.t_nb = p->t_nb;
    g.t_v = p->t_v;
    if (std::isnan(p->t_v)) { err = "t_v must not be NaN"; return FVV_ERR_INVALID_ARG; }
    g.max_comp = p->max_components > 0 ? p->max_components : kMaxComponents;
    g.max_rois = p->max_rois > 0 ? p->max_rois : 256;
    if (g.max_comp > kMaxComponents || g.max_rois > kMaxRois) { err = "max_components <= 8192, max_rois <= 4096"; return FVV_ERR_INVALID_ARG; }
    long long fw = p->max_fine_words;
    if (fw <= 0) {
        // the whole volume at the fine step, in words, over 16; clamped
        double vol = 1.0;
        for (int a = 0; a < 3; ++a) vol *= (double)(um_of(p->vol_max[a]) - um_of(p->vol_min[a])) / (double)g.fine_um;
        fw = (long long)std::min(std::max(vol / 32.0 / 16.0, (double)(1 << 18)), (double)(1 << 23));
    }
    long long mv = p->max_verts > 0 ? p->max_verts : 2 * fw;
    long long mt = p->max_tris > 0 ? p->max_tris : 2 * mv;
    if (fw > (1ll << 26) || mv > (1ll << 30) || mt > (1ll << 30)) {
        err = "max_fine_words must be <= 2^26, max_verts and max_tris <= 2^30";
        return FVV_ERR_INVALID_ARG;
    }
    g.max_fine_words = (uint32_t)fw;
    g.max_chunks = (uint32_t)((fw + kChunk - 1) / kChunk);
    g.max_verts = (uint32_t)mv;
    g.max_tris = (uint32_t)mt;
    g.tile_y = kFineTiles[FVV_TILE_4x4x8][0];
    g.tile_z = kFineTiles[FVV_TILE_4x4x8][1];

    Layout& L = pl.L;
    std::memset(&L, 0, sizeof(L));
    size_t o = 0;
    auto take = [&](size_t& off, size_t bytes) { off = o; o = align_up(o + std::max<size_t>(bytes, 1)); };
    const size_t nvox = (size_t)g.nx * g.ny * g.nz;
    take(L.info, sizeof(SlotInfo));
    take(L.sil, words * 4);
    take(L.coarse, (size_t)g.nz * g.ny * g.nxw * 4);
    take(L.parent, nvox * 4);
    take(L.roots, (size_t)g.max_comp * 4);
    take(L.cstat, (size_t)g.max_comp * 7 * 4);
    take(L.rois, (size_t)g.max_rois * sizeof(DRoi));
    take(L.roi_label, (size_t)g.max_comp * 4);
    take(L.fine, (size_t)fw * 4);
    take(L.emask, (size_t)fw * 12);
    take(L.vpre, (size_t)fw * 4);
    take(L.chunk_st, (size_t)g.max_chunks * 16);
    take(L.chunk_len, (size_t)g.max_chunks * 4);
    take(L.vrec, (size_t)mv * 8);
    take(L.verts, (size_t)mv * 12);
    take(L.tris, (size_t)mt * 12);
    take(L.tsoup, (size_t)mt * 48);
    take(L.trec, (size_t)mt * 8);
    take(L.vrgb, (size_t)mv * 3);
    take(L.vcam, (size_t)mv * 4);
    take(L.depth, align_up(pix * 4));
    take(L.dbox, (size_t)FVV_MAX_CAMS * 4 * sizeof(int32_t));
    if (d->host_staging < 0 || d->host_staging > 2) { err = "host_staging must be 0, 1 or 2"; return FVV_ERR_INVALID_ARG; }
    if (d->host_staging) take(L.mask_stage, pix);
    if (d->host_staging == 1) take(L.rgb_stage, pix * 3);
    L.stride = o;
    pl.common = align_up(256) + align_up(256 * kMaxTriPerCell * 3) + align_up(FVV_MAX_BATCH * 3 * sizeof(float));
    pl.total = pl.common + (size_t)d->max_slots * L.stride;
    return FVV_OK;
}

bool check_slot(fvv_rig* rig, int slot) { return rig && slot >= 0 && slot < rig->max_slots; }

constexpr size_t kMaxIntervals = 1 << 16;

cudaEvent_t next_event(fvv_rig* rig) {
    if (rig->events_used == rig->events.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        rig->events.push_back(e);
    }
    return rig->events[rig->events_used++];
}

// Records the start of a timed stage; returns the interval index or -1.
int stage_begin(fvv_rig* rig, int stage, cudaStream_t st) {
    if (!rig->timing || rig->intervals.size() >= kMaxIntervals) return -1;
    cudaEvent_t a = next_event(rig), b = next_event(rig);
    if (!a || !b || cudaEventRecord(a, st) != cudaSuccess) return -1;
    rig->intervals.push_back({stage, a, b});
    return (int)rig->intervals.size() - 1;
}

void stage_end(fvv_rig* rig, int idx, cudaStream_t st) {
    if (idx >= 0) cudaEventRecord(rig->intervals[idx].b, st);
}

__global__ void k_zero_info(const __grid_constant__ Layout L, const __grid_constant__ SlotList sl) {
    pdl_begin();
    uint32_t* p = reinterpret_cast<uint32_t*>(slot_ptr<SlotInfo>(L, sl.s[blockIdx.x], L.info));
    for (unsigned i = threadIdx.x; i < sizeof(SlotInfo) / 4; i += blockDim.x) p[i] = 0u;
}

}  // namespace

extern "C" {

int fvv_version(void) { return FVV_VERSION; }

const char* fvv_status_string(fvv_status s) {
    switch (s) {
        case FVV_OK: return "FVV_OK";
        case FVV_ERR_INVALID_ARG: return "FVV_ERR_INVALID_ARG";
        case FVV_ERR_OUT_OF_MEMORY: return "FVV_ERR_OUT_OF_MEMORY";
        case FVV_ERR_CAPACITY: return "FVV_ERR_CAPACITY";
        case FVV_ERR_NOT_READY: return "FVV_ERR_NOT_READY";
        case FVV_ERR_TIMEOUT: return "FVV_ERR_TIMEOUT";
        case FVV_ERR_CUDA: return "FVV_ERR_CUDA";
    }
    return "unknown fvv_status";
}

const char* fvv_last_error(const fvv_rig* rig) { return rig ? rig->err.c_str() : g_create_err.c_str(); }

fvv_status fvv_mc_table(uint8_t* ntri, uint8_t* edges) {
    if (!ntri || !edges) return fail(nullptr, FVV_ERR_INVALID_ARG, "NULL table buffer");
    std::memset(edges, 0, 256 * kMaxTriPerCell * 3);
    build_mc_table(ntri, edges);
    return FVV_OK;
}

fvv_status fvv_query_arena(const fvv_rig_desc* desc, const fvv_recon_params* params, size_t* bytes) {
    Plan pl;
    std::string err;
    const fvv_status st = make_plan(desc, params, pl, err);
    if (st != FVV_OK) return fail(nullptr, st, err);
    if (!bytes) return fail(nullptr, FVV_ERR_INVALID_ARG, "bytes must not be NULL");
    *bytes = pl.total;
    return FVV_OK;
}

fvv_status fvv_create_rig(const fvv_rig_desc* desc, const fvv_recon_params* params, void* arena, size_t arena_bytes,
                          fvv_rig** out) {
    if (!out) return fail(nullptr, FVV_ERR_INVALID_ARG, "out must not be NULL");
    *out = nullptr;
    Plan pl;
    std::string err;
    fvv_status st = make_plan(desc, params, pl, err);
    if (st != FVV_OK) return fail(nullptr, st, err);
    if (arena && (arena_bytes < pl.total || (reinterpret_cast<uintptr_t>(arena) % kAlign) != 0))
        return fail(nullptr, FVV_ERR_INVALID_ARG, "arena too small or not 256-byte aligned (need " +
                                                      std::to_string(pl.total) + " bytes)");
    fvv_rig* rig = new (std::nothrow) fvv_rig();
    if (!rig) return fail(nullptr, FVV_ERR_OUT_OF_MEMORY, "host allocation failed");
    cudaError_t e = cudaGetDevice(&rig->device);
    if (e != cudaSuccess) { delete rig; return cuda_fail(nullptr, e, "cudaGetDevice"); }
    e = cudaDeviceGetAttribute(&rig->sms, cudaDevAttrMultiProcessorCount, rig->device);
    if (e != cudaSuccess) { delete rig; return cuda_fail(nullptr, e, "cudaDeviceGetAttribute"); }
    if (!arena) {
        e = cudaMalloc(&arena, pl.total);
        if (e != cudaSuccess) {
            delete rig;
            cudaGetLastError();
            return fail(nullptr, FVV_ERR_OUT_OF_MEMORY, "cudaMalloc of " + std::to_string(pl.total) + " bytes failed");
        }
        rig->own_arena = true;
    }
    rig->arena = static_cast<char*>(arena);
    rig->arena_bytes = pl.total;
    rig->cams = pl.cams;
    rig->grid = pl.grid;
    rig->L = pl.L;
    rig->L.base = rig->arena + pl.common;
    rig->max_slots = desc->max_slots;
    rig->host_staging = desc->host_staging;
    rig->sil_words = pl.sil_words;
    rig->npix = pl.npix;
    rig->state.assign(desc->max_slots, 0);
    rig->mc_ntri = reinterpret_cast<uint8_t*>(rig->arena);
    rig->mc_edges = reinterpret_cast<uint8_t*>(rig->arena + align_up(256));
    std::vector<uint8_t> ntri(256), edges(256 * kMaxTriPerCell * 3, 0);
    build_mc_table(ntri.data(), edges.data());
    e = cudaMemcpy(rig->mc_ntri, ntri.data(), ntri.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(rig->mc_edges, edges.data(), edges.size(), cudaMemcpyHostToDevice);
    // every depth image starts empty; each depth stage then clears only the
    // box its slot's previous z-buffer wrote
    if (e == cudaSuccess) e = launch_init_depth(rig->cams, rig->L, rig->max_slots, rig->sms, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&rig->host_info), FVV_MAX_BATCH * sizeof(SlotInfo),
                                            cudaHostAllocDefault);
    if (e != cudaSuccess) {
        if (rig->own_arena) cudaFree(rig->arena);
        if (rig->host_info) cudaFreeHost(rig->host_info);
        delete rig;
        return cuda_fail(nullptr, e, "initialising the rig");
    }
    *out = rig;
    return FVV_OK;
}

fvv_status fvv_destroy_rig(fvv_rig* rig) {
    if (!rig) return FVV_OK;
    cudaError_t e = cudaDeviceSynchronize();
    for (cudaEvent_t ev : rig->events) cudaEventDestroy(ev);
    for (auto& gr : rig->graph_cache) cudaGraphExecDestroy(gr.exec);
    if (rig->host_info) cudaFreeHost(rig->host_info);
    if (rig->own_arena) {
        cudaError_t f = cudaFree(rig->arena);
        if (e == cudaSuccess) e = f;
    }
    delete rig;
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "fvv_destroy_rig");
    return FVV_OK;
}

// The device address of a camera image of `bytes` bytes at host address p in
// page-locked, device-mapped host memory (FVV_MAPPED_HOST), or NULL if
// its first or last byte is not in such memory.
static const uint8_t* mapped_host(const uint8_t* p, size_t bytes) {
    cudaPointerAttributes a{}, b{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (cudaPointerGetAttributes(&b, p + bytes - 1) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
        return nullptr;
    const uint8_t* d = static_cast<const uint8_t*>(a.devicePointer);
    if (static_cast<const uint8_t*>(b.devicePointer) != d + bytes - 1) return nullptr;
    return d;
}

// Validates and stages the masks of frames j < n_frames (slots[j], masks
// masks[j * n_cams + n]), then packs them.
static fvv_status upload(fvv_rig* rig, int n_frames, const int* slots, const uint8_t* const* masks,
                         int masks_on_device, void* stream, const char* who) {
    if (!rig) return fail(nullptr, FVV_ERR_INVALID_ARG, "rig is NULL");
    if (!slots || n_frames < 1 || n_frames > FVV_MAX_BATCH)
        return fail(rig, FVV_ERR_INVALID_ARG, "slots must list 1..256 slots");
    if (!masks) return fail(rig, FVV_ERR_INVALID_ARG, "masks is NULL");
    if (masks_on_device < 0 || masks_on_device > FVV_MAPPED_HOST)
        return fail(rig, FVV_ERR_INVALID_ARG, "masks_on_device must be 0, 1 or FVV_MAPPED_HOST");
    if (!masks_on_device && !rig->host_staging)
        return fail(rig, FVV_ERR_INVALID_ARG, "host masks need a rig with host_staging");
    const int N = rig->cams.n;
    std::vector<char> seen(rig->max_slots, 0);
    for (int j = 0; j < n_frames; ++j) {
        if (!check_slot(rig, slots[j])) return fail(rig, FVV_ERR_INVALID_ARG, "slot out of range");
        if (seen[slots[j]]) return fail(rig, FVV_ERR_INVALID_ARG, "slots must be distinct");
        seen[slots[j]] = 1;
        for (int n = 0; n < N; ++n)
            if (!masks[(size_t)j * N + n]) return fail(rig, FVV_ERR_INVALID_ARG, "a mask pointer is NULL");
    }
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<const uint8_t*> src(masks, masks + (size_t)n_frames * N);
    if (masks_on_device == FVV_MAPPED_HOST) {
        for (int j = 0; j < n_frames; ++j)
            for (int n = 0; n < N; ++n) {
                const Cam& c = rig->cams.c[n];
                const uint8_t*& p = src[(size_t)j * N + n];
                p = mapped_host(p, (size_t)c.W * c.H);
                if (!p) return fail(rig, FVV_ERR_INVALID_ARG, "a mask is not in mapped page-locked host memory");
            }
    } else if (!masks_on_device) {
        for (int j = 0; j < n_frames; ++j) {
            uint8_t* stage = slot_ptr<uint8_t>(rig->L, slots[j], rig->L.mask_stage);
            for (int n = 0; n < N; ++n) {
                const Cam& c = rig->cams.c[n];
                const uint8_t*& p = src[(size_t)j * N + n];
                const cudaError_t e = cudaMemcpyAsync(stage + c.pix_off, p, (size_t)c.W * c.H,
                                                      cudaMemcpyHostToDevice, st);
                if (e != cudaSuccess) return cuda_fail(rig, e, "copying masks");
                p = stage + c.pix_off;
            }
        }
    }
    const int t = stage_begin(rig, FVV_STAGE_PACK, st);
    const cudaError_t e = launch_pack(rig->cams, rig->L, n_frames, slots, src.data(),
                                      masks_on_device == FVV_MAPPED_HOST, rig->sms, st);
    stage_end(rig, t, st);
    if (e != cudaSuccess) return cuda_fail(rig, e, who);
    for (int j = 0; j < n_frames; ++j) rig->state[slots[j]] = 1;
    return FVV_OK;
}

fvv_status fvv_upload_silhouettes(fvv_rig* rig, int slot, const uint8_t* const* masks, int masks_on_device,
                                  void* stream) {
    return upload(rig, 1, &slot, masks, masks_on_device, stream, "fvv_upload_silhouettes");
}

fvv_status fvv_upload_silhouettes_batch(fvv_rig* rig, const int* slots, int n_slots, const uint8_t* const* masks,
                                        int masks_on_device, void* stream) {
    return upload(rig, n_slots, slots, masks, masks_on_device, stream, "fvv_upload_silhouettes_batch");
}

static fvv_status make_slot_list(fvv_rig* rig, const int* slots, int n_slots, int need_state, SlotList& sl) {
    if (!slots || n_slots < 1 || n_slots > FVV_MAX_BATCH || n_slots > rig->max_slots)
        return fail(rig, FVV_ERR_INVALID_ARG, "slots must list 1..min(256, max_slots) slots");
    std::vector<char> seen(rig->max_slots, 0);
    sl.n = n_slots;
    for (int i = 0; i < n_slots; ++i) {
        if (!check_slot(rig, slots[i])) return fail(rig, FVV_ERR_INVALID_ARG, "slot out of range");
        if (seen[slots[i]]) return fail(rig, FVV_ERR_INVALID_ARG, "slots must be distinct");
        seen[slots[i]] = 1;
        if (rig->state[slots[i]] < need_state) return fail(rig, FVV_ERR_NOT_READY, "slot not ready for this call");
        sl.s[i] = slots[i];
    }
    return FVV_OK;
}

// The launch sequence of one reconstruction of the slots in `sl`.
static cudaError_t enqueue_reconstruct(fvv_rig* rig, const SlotList& sl, cudaStream_t st) {
    const Tuning& tu = rig->tune;
    const Grid g = tuned_grid_params(rig->grid, tu);
    const McTable mc{rig->mc_ntri, rig->mc_edges};
    cudaError_t e = launch_pdl(k_zero_info, dim3(sl.n), dim3(32), 0, st, rig->L, sl);
    int t;
#define FVV_STAGE(stage, call)                  \
    if (e == cudaSuccess) {                     \
        t = stage_begin(rig, stage, st);        \
        e = (call);                             \
        stage_end(rig, t, st);                  \
    }
    FVV_STAGE(FVV_STAGE_COARSE, launch_coarse_carve(rig->cams, g, rig->L, sl, rig->sms, tu, st));
    FVV_STAGE(FVV_STAGE_CCL, launch_ccl(g, rig->L, sl, rig->sms, st));
    FVV_STAGE(FVV_STAGE_FINE, launch_fine_carve(rig->cams, g, rig->L, sl, rig->sms, tu, st));
    FVV_STAGE(FVV_STAGE_MC, launch_mc_prefix(g, rig->L, sl, mc, rig->sms, st));
    FVV_STAGE(FVV_STAGE_BISECT, launch_bisect(rig->cams, g, rig->L, sl, rig->sms, tu, st));
    FVV_STAGE(FVV_STAGE_MC, launch_mc_triangles(g, rig->L, sl, mc, rig->sms, tu, st));
    FVV_STAGE(FVV_STAGE_DEPTH, launch_depth(rig->cams, g, rig->L, sl, rig->sms, align_up(rig->npix * 4), tu, st));
#undef FVV_STAGE
    return e;
}

static void drop_graphs(fvv_rig* rig) {
    for (auto& gr : rig->graph_cache) cudaGraphExecDestroy(gr.exec);
    rig->graph_cache.clear();
}

// Replay (or first record) the graph of this slot list on `st`.
static cudaError_t launch_graph(fvv_rig* rig, const SlotList& sl, cudaStream_t st) {
    std::vector<int> key(sl.s, sl.s + sl.n);
    for (auto& gr : rig->graph_cache)
        if (gr.slots == key) {
            gr.used = ++rig->graph_clock;
            return cudaGraphLaunch(gr.exec, st);
        }
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t le = enqueue_reconstruct(rig, sl, st);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(st, &graph);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return le != cudaSuccess ? le : e;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    if (rig->graph_cache.size() >= 16) {
        size_t lru = 0;
        for (size_t i = 1; i < rig->graph_cache.size(); ++i)
            if (rig->graph_cache[i].used < rig->graph_cache[lru].used) lru = i;
        cudaGraphExecDestroy(rig->graph_cache[lru].exec);
        rig->graph_cache.erase(rig->graph_cache.begin() + (long)lru);
    }
    rig->graph_cache.push_back({key, exec, ++rig->graph_clock});
    return cudaGraphLaunch(exec, st);
}

fvv_status fvv_reconstruct(fvv_rig* rig, const int* slots, int n_slots, void* stream) {
    if (!rig) return fail(nullptr, FVV_ERR_INVALID_ARG, "rig is NULL");
    SlotList sl;
    fvv_status s = make_slot_list(rig, slots, n_slots, 1, sl);
    if (s != FVV_OK) return s;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool use_graph = rig->graphs && !rig->timing && st != nullptr;
    const cudaError_t e = use_graph ? launch_graph(rig, sl, st) : enqueue_reconstruct(rig, sl, st);
    if (e != cudaSuccess) return cuda_fail(rig, e, "fvv_reconstruct launch");
    for (int i = 0; i < sl.n; ++i) rig->state[sl.s[i]] = 2;
    return FVV_OK;
}

fvv_status fvv_set_graphs(fvv_rig* rig, int enable) {
    if (!rig) return fail(nullptr, FVV_ERR_INVALID_ARG, "rig is NULL");
    rig->graphs = enable != 0;
    if (!rig->graphs) {
        cudaDeviceSynchronize();
        drop_graphs(rig);
    }
    return FVV_OK;
}

fvv_status fvv_get_tuning(fvv_rig* rig, int* config) {
    if (!rig || !config) return fail(rig, FVV_ERR_INVALID_ARG, "rig and config must not be NULL");
    for (int k = 0; k < FVV_N_TUNE; ++k) {
        config[k] = rig->tune.threads[k];
        config[FVV_N_TUNE + k] = rig->tune.waves[k];
    }
    config[2 * FVV_N_TUNE] = rig->tune.fine_tile;
    config[2 * FVV_N_TUNE + 1] = rig->tune.zb_cams;
    return FVV_OK;
}

fvv_status fvv_set_tuning(fvv_rig* rig, const int* config) {
    if (!rig || !config) return fail(rig, FVV_ERR_INVALID_ARG, "rig and config must not be NULL");
    for (int k = 0; k < FVV_N_TUNE; ++k) {
        const int th = config[k], wv = config[FVV_N_TUNE + k];
        if (th < 32 || th > 256 || th % 32 || wv < 1 || wv > 64)
            return fail(rig, FVV_ERR_INVALID_ARG, "threads must be 32..256 in steps of 32, blocks per SM 1..64");
    }
    const int tile = config[2 * FVV_N_TUNE];
    if (tile < 0 || tile >= FVV_N_TILES) return fail(rig, FVV_ERR_INVALID_ARG, "tile shape must be one of FVV_TILE_*");
    const int zc = config[2 * FVV_N_TUNE + 1];
    if (zc != 1 && zc != 2 && zc != 4) return fail(rig, FVV_ERR_INVALID_ARG, "z-buffer cameras per block must be 1, 2 or 4");
    for (int k = 0; k < FVV_N_TUNE; ++k) {
        rig->tune.threads[k] = config[k];
        rig->tune.waves[k] = config[FVV_N_TUNE + k];
    }
    rig->tune.fine_tile = tile;
    rig->tune.zb_cams = zc;
    cudaDeviceSynchronize();
    drop_graphs(rig);
    return FVV_OK;
}

fvv_status fvv_autotune(fvv_rig* rig, const int* slots, int n_slots, void* stream, int* config) {
    if (!rig) return fail(nullptr, FVV_ERR_INVALID_ARG, "rig is NULL");
    SlotList sl;
    fvv_status s = make_slot_list(rig, slots, n_slots, 2, sl);
    if (s != FVV_OK) return s;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool timing = rig->timing;
    rig->timing = false;
    const McTable mc{rig->mc_ntri, rig->mc_edges};
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    // one stage on its own, on the inputs the last reconstruction left (the
    // fine hull after the ROI table was laid out for its tile shape)
    auto run = [&](int knob, const Tuning& tu) -> cudaError_t {
        const Grid g = tuned_grid_params(rig->grid, tu);
        switch (knob) {
            case FVV_TUNE_COARSE: return launch_coarse_carve(rig->cams, g, rig->L, sl, rig->sms, tu, st);
            case FVV_TUNE_FINE: return launch_fine_carve(rig->cams, g, rig->L, sl, rig->sms, tu, st);
            case FVV_TUNE_BISECT: return launch_bisect(rig->cams, g, rig->L, sl, rig->sms, tu, st);
            case FVV_TUNE_ZBUFFER:
                return launch_depth(rig->cams, g, rig->L, sl, rig->sms, align_up(rig->npix * 4), tu, st);
            default: return launch_mc_triangles(g, rig->L, sl, mc, rig->sms, tu, st);
        }
    };
    const int threads[] = {64, 128, 256};
    const int waves[] = {2, 4, 8, 16, 32, 64};
    for (int knob = 0; knob < FVV_N_TUNE && e == cudaSuccess; ++knob) {
        float best = 1e30f;
        Tuning keep = rig->tune;
        // the fine hull also tries each tile shape, the z-buffer each number
        // of cameras per block (1, 2, 4)
        const int n_tiles = knob == FVV_TUNE_FINE ? FVV_N_TILES : knob == FVV_TUNE_ZBUFFER ? 3 : 1;
        for (int tile = 0; tile < n_tiles && e == cudaSuccess; ++tile)
        for (int th : threads)
            for (int wv : waves) {
                Tuning tu = rig->tune;
                tu.threads[knob] = th;
                tu.waves[knob] = wv;
                if (knob == FVV_TUNE_ZBUFFER) tu.zb_cams = 1 << tile;
                if (knob == FVV_TUNE_FINE) {
                    tu.fine_tile = tile;
                    // the ROI table's tile offsets for this shape (not timed)
                    if (th == threads[0] && wv == waves[0]) e = launch_filter(tuned_grid_params(rig->grid, tu), rig->L, sl, st);
                    if (e != cudaSuccess) break;
                }
                e = run(knob, tu);  // warm
                if (e == cudaSuccess) e = cudaEventRecord(a, st);
                for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) e = run(knob, tu);
                if (e == cudaSuccess) e = cudaEventRecord(b, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(b);
                float ms = 0.0f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
                if (e != cudaSuccess) break;
                if (ms < best) {
                    best = ms;
                    keep.threads[knob] = th;
                    keep.waves[knob] = wv;
                    keep.fine_tile = tu.fine_tile;
                    keep.zb_cams = tu.zb_cams;
                }
            }
        rig->tune = keep;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e == cudaSuccess) {
        drop_graphs(rig);
        e = enqueue_reconstruct(rig, sl, st);   // consistent results and counts again
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    rig->timing = timing;
    if (e != cudaSuccess) return cuda_fail(rig, e, "fvv_autotune");
    if (config) fvv_get_tuning(rig, config);
    return FVV_OK;
}

fvv_status fvv_colour(fvv_rig* rig, const int* slots, int n_slots, const uint8_t* const* rgb, int rgb_on_device,
                      const float* viewpoints, void* stream) {
    if (!rig) return fail(nullptr, FVV_ERR_INVALID_ARG, "rig is NULL");
    SlotList sl;
    fvv_status s = make_slot_list(rig, slots, n_slots, 2, sl);
    if (s != FVV_OK) return s;
    if (!rgb || !viewpoints) return fail(rig, FVV_ERR_INVALID_ARG, "rgb and viewpoints must not be NULL");
    if (rgb_on_device < 0 || rgb_on_device > FVV_MAPPED_HOST)
        return fail(rig, FVV_ERR_INVALID_ARG, "rgb_on_device must be 0, 1 or FVV_MAPPED_HOST");
    if (!rgb_on_device && rig->host_staging != 1)
        return fail(rig, FVV_ERR_INVALID_ARG, "copied host RGB needs host_staging = 1");
    for (int i = 0; i < 3 * n_slots; ++i)
        if (!std::isfinite(viewpoints[i])) return fail(rig, FVV_ERR_INVALID_ARG, "viewpoints must be finite");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int N = rig->cams.n;
    for (size_t i = 0; i < (size_t)n_slots * N; ++i)
        if (!rgb[i]) return fail(rig, FVV_ERR_INVALID_ARG, "an rgb pointer is NULL");
    if (rgb_on_device == FVV_MAPPED_HOST)
        for (int i = 0; i < n_slots; ++i)
            for (int n = 0; n < N; ++n) {
                const Cam& c = rig->cams.c[n];
                if (!mapped_host(rgb[(size_t)i * N + n], (size_t)3 * c.W * c.H))
                    return fail(rig, FVV_ERR_INVALID_ARG, "an rgb image is not in mapped page-locked host memory");
            }
    cudaError_t e = cudaSuccess;
    const int t = stage_begin(rig, FVV_STAGE_COLOUR, st);
    // slots go to the kernel in groups of kColourBatch, with their RGB sources
    // and viewpoints as kernel parameters
    for (int i0 = 0; i0 < n_slots && e == cudaSuccess; i0 += kColourBatch) {
        ColourBatch cb;
        cb.n = std::min(kColourBatch, n_slots - i0);
        for (int j = 0; j < cb.n && e == cudaSuccess; ++j) {
            const int i = i0 + j;
            cb.slot[j] = sl.s[i];
            for (int k = 0; k < 3; ++k) cb.view[j][k] = viewpoints[3 * i + k];
            for (int n = 0; n < N; ++n) {
                const uint8_t* src = rgb[(size_t)i * N + n];
                if (rgb_on_device == 1) {
                    cb.rgb[j][n] = src;
                } else if (rgb_on_device == FVV_MAPPED_HOST) {
                    const Cam& c = rig->cams.c[n];
                    cb.rgb[j][n] = mapped_host(src, (size_t)3 * c.W * c.H);   // checked above
                } else {
                    const Cam& c = rig->cams.c[n];
                    uint8_t* dst = slot_ptr<uint8_t>(rig->L, sl.s[i], rig->L.rgb_stage) + 3 * c.pix_off;
                    e = cudaMemcpyAsync(dst, src, (size_t)3 * c.W * c.H, cudaMemcpyHostToDevice, st);
                    if (e != cudaSuccess) break;
                    cb.rgb[j][n] = dst;
                }
            }
        }
        if (e == cudaSuccess) e = launch_colour(rig->cams, rig->grid, rig->L, cb, rig->sms, n_slots, st);
    }
    stage_end(rig, t, st);
    if (e != cudaSuccess) return cuda_fail(rig, e, "fvv_colour");
    return FVV_OK;
}

fvv_status fvv_render_view(fvv_rig* rig, int slot, const uint8_t* const* rgb, int rgb_on_device, const float* P,
                           const float* centre, int width, int height, uint64_t* key, uint8_t* out_rgb,
                           int32_t* out_cam, void* stream) {
    if (!rig) return fail(nullptr, FVV_ERR_INVALID_ARG, "rig is NULL");
    SlotList sl;
    fvv_status s = make_slot_list(rig, &slot, 1, 2, sl);
    if (s != FVV_OK) return s;
    if (!rgb || !P || !centre || !key || !out_rgb)
        return fail(rig, FVV_ERR_INVALID_ARG, "rgb, P, centre, key and out_rgb must not be NULL");
    if (width < 1 || height < 1 || width > 65535 || height > 65535)
        return fail(rig, FVV_ERR_INVALID_ARG, "view size must be 1..65535 pixels per side");
    if (rgb_on_device < 0 || rgb_on_device > FVV_MAPPED_HOST)
        return fail(rig, FVV_ERR_INVALID_ARG, "rgb_on_device must be 0, 1 or FVV_MAPPED_HOST");
    if (!rgb_on_device && rig->host_staging != 1)
        return fail(rig, FVV_ERR_INVALID_ARG, "copied host RGB needs host_staging = 1");
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(P[i])) return fail(rig, FVV_ERR_INVALID_ARG, "P must be finite");
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(centre[i])) return fail(rig, FVV_ERR_INVALID_ARG, "centre must be finite");
    const int N = rig->cams.n;
    for (int n = 0; n < N; ++n)
        if (!rgb[n]) return fail(rig, FVV_ERR_INVALID_ARG, "an rgb pointer is NULL");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    ViewArgs va;
    std::memset(&va, 0, sizeof(va));
    for (int i = 0; i < 12; ++i) va.v.P[i] = P[i];
    for (int i = 0; i < 3; ++i) va.v.C[i] = centre[i];
    va.v.W = width;
    va.v.H = height;
    va.v.Wf = (float)width;
    va.v.Hf = (float)height;
    va.slot = slot;
    cudaError_t e = cudaSuccess;
    for (int n = 0; n < N && e == cudaSuccess; ++n) {
        if (rgb_on_device == 1) {
            va.rgb[n] = rgb[n];
        } else if (rgb_on_device == FVV_MAPPED_HOST) {
            const Cam& c = rig->cams.c[n];
            va.rgb[n] = mapped_host(rgb[n], (size_t)3 * c.W * c.H);
            if (!va.rgb[n]) return fail(rig, FVV_ERR_INVALID_ARG, "an rgb image is not in mapped page-locked host memory");
        } else {
            const Cam& c = rig->cams.c[n];
            uint8_t* dst = slot_ptr<uint8_t>(rig->L, slot, rig->L.rgb_stage) + 3 * c.pix_off;
            e = cudaMemcpyAsync(dst, rgb[n], (size_t)3 * c.W * c.H, cudaMemcpyHostToDevice, st);
            va.rgb[n] = dst;
        }
    }
    if (e == cudaSuccess)
        e = launch_render_view(rig->cams, rig->grid, rig->L, va, reinterpret_cast<unsigned long long*>(key), out_rgb,
                               out_cam, rig->sms, st);
    if (e != cudaSuccess) return cuda_fail(rig, e, "fvv_render_view");
    return FVV_OK;
}

fvv_status fvv_set_timing(fvv_rig* rig, int enable) {
    if (!rig) return fail(nullptr, FVV_ERR_INVALID_ARG, "rig is NULL");
    rig->timing = enable != 0;
    rig->intervals.clear();
    rig->events_used = 0;
    return FVV_OK;
}

fvv_status fvv_get_timing(fvv_rig* rig, float* ms, int* calls) {
    if (!rig) return fail(nullptr, FVV_ERR_INVALID_ARG, "rig is NULL");
    if (!ms) return fail(rig, FVV_ERR_INVALID_ARG, "ms must not be NULL");
    for (int i = 0; i < FVV_N_STAGES; ++i) {
        ms[i] = 0.0f;
        if (calls) calls[i] = 0;
    }
    cudaError_t e = cudaSuccess;
    for (const auto& iv : rig->intervals) {
        float t = 0.0f;
        e = cudaEventSynchronize(iv.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, iv.a, iv.b);
        if (e != cudaSuccess) break;
        ms[iv.stage] += t;
        if (calls) calls[iv.stage] += 1;
    }
    rig->intervals.clear();
    rig->events_used = 0;
    if (e != cudaSuccess) return cuda_fail(rig, e, "fvv_get_timing");
    return FVV_OK;
}

}  // extern "C"

// The counts of a slot from its device bookkeeping; true if a capacity was exceeded.
static bool fill_counts(const SlotInfo& info, fvv_counts* out) {
    std::memset(out, 0, sizeof(*out));
    out->flags = info.flags;
    out->n_components = info.n_roots;
    out->n_rois = info.n_rois;
    out->n_coarse_on = info.n_on;
    out->n_fine_words = info.n_words;
    out->n_verts = info.n_words ? info.n_verts : 0;
    out->n_tris = info.n_words ? info.n_tris : 0;
    out->tests_coarse = (long long)info.tests_coarse;
    out->tests_fine = (long long)info.tests_fine;
    out->tests_bisect = (long long)info.tests_bisect;
    out->lookups_fine = (long long)info.look_fine;
    out->lookups_bisect = (long long)info.look_bisect;
    const unsigned cap = FVV_FLAG_ROOTS | FVV_FLAG_ROIS | FVV_FLAG_FINE | FVV_FLAG_VERTS | FVV_FLAG_TRIS | FVV_FLAG_LOOP;
    return (info.flags & cap) != 0u;
}

// Enqueue the copies of a slot's vertices, triangles, colours and cameras
// (counts c) into caller-owned buffers (any may be NULL).
static cudaError_t copy_results(fvv_rig* rig, int slot, const fvv_counts& c, float* verts, uint32_t* tris,
                                uint8_t* rgb, int32_t* cam, cudaMemcpyKind kind, cudaStream_t st) {
    const Layout& L = rig->L;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess && verts && c.n_verts)
        e = cudaMemcpyAsync(verts, slot_ptr<float>(L, slot, L.verts), 12 * (size_t)c.n_verts, kind, st);
    if (e == cudaSuccess && tris && c.n_tris)
        e = cudaMemcpyAsync(tris, slot_ptr<uint32_t>(L, slot, L.tris), 12 * (size_t)c.n_tris, kind, st);
    if (e == cudaSuccess && rgb && c.n_verts)
        e = cudaMemcpyAsync(rgb, slot_ptr<uint8_t>(L, slot, L.vrgb), 3 * (size_t)c.n_verts, kind, st);
    if (e == cudaSuccess && cam && c.n_verts)
        e = cudaMemcpyAsync(cam, slot_ptr<int32_t>(L, slot, L.vcam), 4 * (size_t)c.n_verts, kind, st);
    return e;
}

extern "C" {

fvv_status fvv_get_counts(fvv_rig* rig, int slot, fvv_counts* out, void* stream) {
    if (!rig) return fail(nullptr, FVV_ERR_INVALID_ARG, "rig is NULL");
    if (!check_slot(rig, slot) || !out) return fail(rig, FVV_ERR_INVALID_ARG, "bad slot or NULL counts");
    if (rig->state[slot] < 2) return fail(rig, FVV_ERR_NOT_READY, "slot was not reconstructed");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    SlotInfo info;
    cudaError_t e = cudaMemcpyAsync(&info, slot_ptr<SlotInfo>(rig->L, slot, rig->L.info), sizeof(info),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(rig, e, "fvv_get_counts");
    if (fill_counts(info, out)) return fail(rig, FVV_ERR_CAPACITY, "a capacity was exceeded (see flags)");
    return FVV_OK;
}

fvv_status fvv_get_results_batch(fvv_rig* rig, const int* slots, int n_slots, fvv_results_dst* dst,
                                 int dst_on_device, void* stream) {
    if (!rig) return fail(nullptr, FVV_ERR_INVALID_ARG, "rig is NULL");
    if (!slots || !dst || n_slots < 1 || n_slots > FVV_MAX_BATCH)
        return fail(rig, FVV_ERR_INVALID_ARG, "slots and dst must list 1..256 slots");
    for (int i = 0; i < n_slots; ++i) {
        if (!check_slot(rig, slots[i])) return fail(rig, FVV_ERR_INVALID_ARG, "slot out of range");
        if (rig->state[slots[i]] < 2) return fail(rig, FVV_ERR_NOT_READY, "slot was not reconstructed");
        if (dst[i].rois) return fail(rig, FVV_ERR_INVALID_ARG, "ROIs are read by fvv_get_results only");
    }
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n_slots && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(rig->host_info + i, slot_ptr<SlotInfo>(rig->L, slots[i], rig->L.info), sizeof(SlotInfo),
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the one wait of the call
    if (e != cudaSuccess) return cuda_fail(rig, e, "fvv_get_results_batch");
    bool over = false;
    const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int i = 0; i < n_slots && e == cudaSuccess; ++i) {
        fvv_results_dst& d = dst[i];
        if (fill_counts(rig->host_info[i], &d.counts)) {
            over = true;
            continue;
        }
        e = copy_results(rig, slots[i], d.counts, d.verts, d.tris, d.rgb, d.cam, kind, st);
    }
    if (e != cudaSuccess) return cuda_fail(rig, e, "fvv_get_results_batch");
    if (over) return fail(rig, FVV_ERR_CAPACITY, "a capacity was exceeded in some slot (see its flags)");
    return FVV_OK;
}

fvv_status fvv_get_results(fvv_rig* rig, int slot, fvv_roi* rois, float* verts, uint32_t* tris, uint8_t* rgb,
                           int32_t* cam, int dst_on_device, void* stream) {
    fvv_counts c;
    fvv_status s = fvv_get_counts(rig, slot, &c, stream);
    if (s != FVV_OK) return s;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaSuccess;
    if (rois && c.n_rois > 0) {
        std::vector<DRoi> d(c.n_rois);
        e = cudaMemcpyAsync(d.data(), slot_ptr<DRoi>(rig->L, slot, rig->L.rois), sizeof(DRoi) * c.n_rois,
                            cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(rig, e, "reading ROIs");
        std::vector<fvv_roi> h(c.n_rois);
        for (int k = 0; k < c.n_rois; ++k) {
            fvv_roi& r = h[k];
            for (int a = 0; a < 3; ++a) {
                r.cmin[a] = d[k].cmin[a]; r.cmax[a] = d[k].cmax[a];
                r.gmin[a] = d[k].gmin[a]; r.gmax[a] = d[k].gmax[a];
                r.fdim[a] = d[k].fdim[a]; r.forigin[a] = d[k].fo[a];
            }
            r.count = d[k].count;
            r.label = k + 1;
            r.vert_offset = d[k].vert_off;
            r.tri_offset = d[k].tri_off;
            r.n_verts = (k + 1 < c.n_rois ? (long long)d[k + 1].vert_off : c.n_verts) - r.vert_offset;
            r.n_tris = (k + 1 < c.n_rois ? (long long)d[k + 1].tri_off : c.n_tris) - r.tri_offset;
        }
        if (dst_on_device) e = cudaMemcpyAsync(rois, h.data(), sizeof(fvv_roi) * c.n_rois, cudaMemcpyHostToDevice, st);
        else std::memcpy(rois, h.data(), sizeof(fvv_roi) * c.n_rois);
    }
    if (e == cudaSuccess) e = copy_results(rig, slot, c, verts, tris, rgb, cam, kind, st);
    if (e != cudaSuccess) return cuda_fail(rig, e, "fvv_get_results");
    return FVV_OK;
}

fvv_status fvv_debug_pixels(fvv_rig* rig, int cam, long long n, const float* pts, int32_t* px, int32_t* py,
                            void* stream) {
    if (!rig) return fail(nullptr, FVV_ERR_INVALID_ARG, "rig is NULL");
    if (cam < 0 || cam >= rig->cams.n || n < 0 || (n > 0 && (!pts || !px || !py)))
        return fail(rig, FVV_ERR_INVALID_ARG, "bad camera, count or NULL buffer");
    if (n == 0) return FVV_OK;
    const cudaError_t e = launch_debug_pixels(rig->cams, cam, n, pts, px, py, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(rig, e, "fvv_debug_pixels");
    return FVV_OK;
}

fvv_status fvv_debug_label_coarse(fvv_rig* rig, int slot, const uint32_t* coarse_bits, void* stream) {
    if (!rig) return fail(nullptr, FVV_ERR_INVALID_ARG, "rig is NULL");
    if (!check_slot(rig, slot) || !coarse_bits) return fail(rig, FVV_ERR_INVALID_ARG, "bad slot or NULL grid");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    SlotList sl;
    sl.n = 1;
    sl.s[0] = slot;
    k_zero_info<<<1, 32, 0, st>>>(rig->L, sl);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_debug_seed(rig->grid, rig->L, slot, coarse_bits, st);
    if (e == cudaSuccess) e = launch_ccl(rig->grid, rig->L, sl, rig->sms, st);
    if (e != cudaSuccess) return cuda_fail(rig, e, "fvv_debug_label_coarse");
    rig->state[slot] = 2;
    return FVV_OK;
}

fvv_status fvv_debug_bytes(fvv_rig* rig, int slot, int what, size_t* bytes) {
    if (!rig) return fail(nullptr, FVV_ERR_INVALID_ARG, "rig is NULL");
    if (!check_slot(rig, slot) || !bytes) return fail(rig, FVV_ERR_INVALID_ARG, "bad slot or NULL bytes");
    const Grid& g = rig->grid;
    switch (what) {
        case FVV_DEBUG_SIL_BITS: *bytes = rig->sil_words * 4; return FVV_OK;
        case FVV_DEBUG_COARSE_BITS: *bytes = (size_t)g.nz * g.ny * g.nxw * 4; return FVV_OK;
        case FVV_DEBUG_LABELS: *bytes = (size_t)g.nz * g.ny * g.nx * 4; return FVV_OK;
        case FVV_DEBUG_DEPTH: *bytes = rig->npix * 4; return FVV_OK;
        case FVV_DEBUG_FINE_BITS: {
            SlotInfo info;
            const cudaError_t e = cudaMemcpy(&info, slot_ptr<SlotInfo>(rig->L, slot, rig->L.info), sizeof(info),
                                             cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(rig, e, "fvv_debug_bytes");
            *bytes = (size_t)info.n_words * 4;
            return FVV_OK;
        }
    }
    return fail(rig, FVV_ERR_INVALID_ARG, "unknown debug view");
}

fvv_status fvv_get_debug(fvv_rig* rig, int slot, int what, void* dst, size_t bytes, void* stream) {
    size_t need = 0;
    fvv_status s = fvv_debug_bytes(rig, slot, what, &need);
    if (s != FVV_OK) return s;
    if (!dst || bytes < need) return fail(rig, FVV_ERR_INVALID_ARG, "debug buffer too small");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Layout& L = rig->L;
    cudaError_t e = cudaSuccess;
    switch (what) {
        case FVV_DEBUG_SIL_BITS:
            e = cudaMemcpyAsync(dst, slot_ptr<void>(L, slot, L.sil), need, cudaMemcpyDeviceToDevice, st);
            break;
        case FVV_DEBUG_COARSE_BITS:
            e = cudaMemcpyAsync(dst, slot_ptr<void>(L, slot, L.coarse), need, cudaMemcpyDeviceToDevice, st);
            break;
        case FVV_DEBUG_FINE_BITS:
            if (need) e = cudaMemcpyAsync(dst, slot_ptr<void>(L, slot, L.fine), need, cudaMemcpyDeviceToDevice, st);
            break;
        case FVV_DEBUG_LABELS:
            e = cudaMemsetAsync(dst, 0, need, st);
            if (e == cudaSuccess) e = launch_debug_labels(rig->grid, L, slot, static_cast<int32_t*>(dst), st);
            break;
        case FVV_DEBUG_DEPTH:
            e = launch_debug_depth(rig->cams, L, slot, static_cast<float*>(dst), rig->npix, st);
            break;
    }
    if (e != cudaSuccess) return cuda_fail(rig, e, "fvv_get_debug");
    return FVV_OK;
}

}  // extern "C"
