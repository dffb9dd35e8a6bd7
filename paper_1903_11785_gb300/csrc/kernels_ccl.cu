// kernels_ccl.cu -- Sec. II-B-2: 26-connected component labelling of the
// coarse hull, the minimum 3D box of each component, the noise filter of
// Eq. (1) and the 3D ROI table.
//
// Union-find over the occupied voxels with atomics (Playne & Hawick style):
// parents live in a dense int32 array indexed by the linear voxel index and
// are only ever touched at occupied voxels (the coarse carve initialised
// them, each run of consecutive occupied voxels of a 32-voxel word as one
// tree rooted at its first voxel), so nothing is cleared per frame.  A
// union links the larger root
// below the smaller with atomicMin, so every root is the smallest linear
// index of its component; sorting the roots therefore numbers components in
// order of their smallest index, the canonical order of the oracle.  The
// paper's block-local-then-global scheme is replaced by this lock-free
// union, which needs no second pass over block borders.
#include "fvv_device.cuh"

namespace fvv {
namespace {

// Every thread gets a budget of find/union steps for the whole launch; valid
// input never comes near it, and a thread that exhausts it stops, sets
// FVV_FLAG_LOOP and returns, so no launch can run unbounded.
constexpr int kStepBudget = 1 << 22;

// Root of x during the union step, shortening the path on the way (each
// visited node is pointed at its grandparent).  Parents only ever point to
// smaller indices of the same tree, so while unions run the plain stores are
// benign: a store that overwrites a concurrent atomicMin link is made good by
// that union, which retries from the old parent it got back.  This holds for
// k_union only: once k_compress writes a voxel's final root, a shortening
// store from another thread's stale walk could replace it with an
// intermediate node, so k_compress uses find_root_readonly instead.
__device__ __forceinline__ int find_root(int* parent, int x, int& budget) {
    int cur = __ldcg(parent + x);
    if (cur == x || cur < 0) return x;
    int prev = x;
    while (budget > 0) {
        --budget;
        const int next = __ldcg(parent + cur);
        if (next == cur || next < 0) return cur;
        __stcg(parent + prev, next);
        prev = cur;
        cur = next;
    }
    return cur;
}

// Root of x once every union is done, without writing anything.  In
// k_compress the only store to parent[v] is v's own thread writing v's root,
// so a parent entry only ever changes from an ancestor to the root: a walk
// that reads either value still ends at the root, and the root that thread
// writes stays (each non-root voxel ends pointing straight at its root, which
// the two-step lookups of k_stats and k_debug_labels rely on).
__device__ __forceinline__ int find_root_readonly(const int* parent, int x, int& budget) {
    int cur = x;
    while (budget > 0) {
        --budget;
        const int next = __ldcg(parent + cur);
        if (next == cur || next < 0) return cur;
        cur = next;
    }
    return cur;
}

__device__ __forceinline__ void unite(int* parent, int a, int b, int& budget) {
    while (budget > 0) {
        a = find_root(parent, a, budget);
        b = find_root(parent, b, budget);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(parent + a, b);
        if (old == a) return;
        a = old;
    }
}

// Bit i of row `row` (y, z), word wx of the coarse bitset as seen from the
// 26-neighbourhood: 0 outside the grid.
__device__ __forceinline__ uint32_t coarse_word(const uint32_t* bits, const Grid& g, int y, int z, int wx) {
    if (y < 0 || z < 0 || y >= g.ny || z >= g.nz || wx < 0 || wx >= g.nxw) return 0u;
    return __ldg(bits + ((size_t)z * g.ny + y) * g.nxw + wx);
}

// The unions of Sec. II-B-2 (26-connectivity), a word at a time.  The coarse
// carve made each run of consecutive occupied voxels within a word one tree
// rooted at its first voxel, so what is left is to join runs:
//  - across a word boundary in the same row (the word's first voxel with
//    the last voxel of the word before it);
//  - with the four rows before it that touch it, (y-1, z) and (y-1..y+1,
//    z-1): a run R of this row and a run S of such a row N are 26-adjacent
//    iff some voxel l of R has a voxel of S among N's voxels l-1, l, l+1.
// For each pair (R, S) one union suffices.  Let l0 be R's first voxel whose
// window meets S.  Either l0 is R's first voxel, and S holds the leftmost
// occupied of N's l0-1, l0 or, failing both, starts at l0+1; or l0 is
// later, the window of l0-1 misses S, and S starts exactly at l0+1 with l0
// empty in N.  So each voxel l of R unites R with the run of N's leftmost
// occupied voxel among l-1, l if l starts R, and with the run starting at
// l+1 if N has l empty and l+1 occupied: at most two unions per voxel and
// row, almost all of them at run starts.  A warp reads 32 words of the
// bitset (a lane each) and then takes its non-empty words one at a time
// with a lane per voxel.
__global__ void __launch_bounds__(256) k_union(const __grid_constant__ Grid g, const __grid_constant__ Layout L,
                                               const __grid_constant__ SlotList sl) {
    pdl_begin();
    const int slot = sl.s[blockIdx.y];
    const uint32_t* bits = slot_ptr<uint32_t>(L, slot, L.coarse);
    int* parent = slot_ptr<int>(L, slot, L.parent);
    const uint32_t nwords = (uint32_t)g.nz * g.ny * g.nxw;
    const int lane = threadIdx.x & 31;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    int budget = kStepBudget;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (uint32_t base = 0; base < nwords; base += nwarps * 32u) {
        // words interleaved over the warps (lane l of warp k reads word
        // base + l * nwarps + k), so that neighbouring words, which often
        // belong to one object, are worked on by different warps
        const uint32_t mw = base + (uint32_t)lane * nwarps + gw;
        const uint32_t mine = mw < nwords ? __ldg(bits + mw) : 0u;
        uint32_t pending = __ballot_sync(kFull, mine != 0u);
        while (pending) {
            const int src = __ffs(pending) - 1;
            pending &= pending - 1u;
            const uint32_t w = base + (uint32_t)src * nwarps + gw;
            const uint32_t word = __shfl_sync(kFull, mine, src);
            if (!((word >> lane) & 1u) || budget <= 0) continue;
            const uint32_t row = w / (uint32_t)g.nxw;
            const int wx = (int)(w - row * g.nxw);
            const int y = (int)(row % (uint32_t)g.ny), z = (int)(row / (uint32_t)g.ny);
            const int x0 = wx * 32;
            const uint32_t starts = word & ~(word << 1);
            const bool first = (starts >> lane) & 1u;                      // lane starts its run
            const int run0 = (int)row * g.nx + x0 + (31 - __clz(starts & (0xFFFFFFFFu >> (31 - lane))));
            // the run across the boundary with the word before, same row
            if (lane == 0 && (coarse_word(bits, g, y, z, wx - 1) >> 31))
                unite(parent, run0, run0 - 1, budget);
            for (int k = 0; k < 4; ++k) {
                const int dy = k == 0 ? -1 : k - 2, dz = k == 0 ? 0 : -1;
                const uint32_t n = coarse_word(bits, g, y + dy, z + dz, wx);
                const uint32_t np = coarse_word(bits, g, y + dy, z + dz, wx - 1);
                const uint32_t nn = coarse_word(bits, g, y + dy, z + dz, wx + 1);
                const bool left = lane > 0 ? (n >> (lane - 1)) & 1u : np >> 31;
                const bool mid = (n >> lane) & 1u;
                const bool right = lane < 31 ? (n >> (lane + 1)) & 1u : nn & 1u;
                const int nrow = ((z + dz) * g.ny + (y + dy)) * g.nx + x0;
                if (first && (left || mid)) unite(parent, run0, nrow + (left ? lane - 1 : lane), budget);
                if (!mid && right) unite(parent, run0, nrow + lane + 1, budget);
            }
        }
    }
    if (budget <= 0) atomicOr(&slot_ptr<SlotInfo>(L, slot, L.info)->flags, (unsigned)FVV_FLAG_LOOP);
}

// Point every voxel at its root and list the roots (unordered); words are
// taken as in k_union, a lane per voxel.  A thread writes only its own
// voxel's entry (see find_root_readonly).
__global__ void __launch_bounds__(256) k_compress(const __grid_constant__ Grid g, const __grid_constant__ Layout L,
                                                  const __grid_constant__ SlotList sl) {
    pdl_begin();
    const int slot = sl.s[blockIdx.y];
    const uint32_t* bits = slot_ptr<uint32_t>(L, slot, L.coarse);
    int* parent = slot_ptr<int>(L, slot, L.parent);
    int* roots = slot_ptr<int>(L, slot, L.roots);
    SlotInfo* info = slot_ptr<SlotInfo>(L, slot, L.info);
    const uint32_t nwords = (uint32_t)g.nz * g.ny * g.nxw;
    const int lane = threadIdx.x & 31;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    int budget = kStepBudget;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (uint32_t base = 0; base < nwords; base += nwarps * 32u) {
        // words interleaved over the warps (lane l of warp k reads word
        // base + l * nwarps + k), so that neighbouring words, which often
        // belong to one object, are worked on by different warps
        const uint32_t mw = base + (uint32_t)lane * nwarps + gw;
        const uint32_t mine = mw < nwords ? __ldg(bits + mw) : 0u;
        uint32_t pending = __ballot_sync(kFull, mine != 0u);
        while (pending) {
            const int src = __ffs(pending) - 1;
            pending &= pending - 1u;
            const uint32_t w = base + (uint32_t)src * nwarps + gw;
            const uint32_t word = __shfl_sync(kFull, mine, src);
            if (!((word >> lane) & 1u) || budget <= 0) continue;
            const uint32_t row = w / (uint32_t)g.nxw;
            const int wx = (int)(w - row * g.nxw);
            const int Lin = (int)row * g.nx + wx * 32 + lane;
            const int r = find_root_readonly(parent, Lin, budget);
            if (r == Lin) {
                const int k = atomicAdd(&info->n_roots, 1);
                if (k < g.max_comp) roots[k] = Lin;
            } else {
                parent[Lin] = r;
            }
        }
    }
    if (budget <= 0) atomicOr(&info->flags, (unsigned)FVV_FLAG_LOOP);
}

// One block per slot: sort the roots (bitonic, in shared memory) so that
// component i is the one with the i-th smallest least index; tag each root's
// parent entry with -(i+1); reset the per-component statistics.
__global__ void __launch_bounds__(1024) k_sort_roots(const __grid_constant__ Grid g, const __grid_constant__ Layout L,
                                                     const __grid_constant__ SlotList sl) {
    pdl_begin();
    __shared__ int key[kMaxComponents];
    const int slot = sl.s[blockIdx.x];
    SlotInfo* info = slot_ptr<SlotInfo>(L, slot, L.info);
    int* roots = slot_ptr<int>(L, slot, L.roots);
    int* parent = slot_ptr<int>(L, slot, L.parent);
    int* cstat = slot_ptr<int>(L, slot, L.cstat);
    int n = info->n_roots;
    if (n > g.max_comp) {
        __syncthreads();
        if (threadIdx.x == 0) {
            info->flags |= FVV_FLAG_ROOTS;
            info->n_roots = 0;
        }
        return;
    }
    int m = 1;
    while (m < n) m <<= 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x) key[i] = i < n ? roots[i] : 0x7FFFFFFF;
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                const int p = i ^ j;
                if (p > i) {
                    const bool up = (i & k) == 0;
                    const int a = key[i], b = key[p];
                    if ((a > b) == up) {
                        key[i] = b;
                        key[p] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        roots[i] = key[i];
        parent[key[i]] = -(i + 1);
        int* s = cstat + 7 * i;
        s[0] = 0;
        s[1] = s[2] = s[3] = 0x7FFFFFFF;
        s[4] = s[5] = s[6] = -1;
    }
}

// Voxel count and inclusive box of every component (Sec. II-B-2 takes the
// smallest box holding each labelled set after labelling).  Words are taken
// as in k_union: a non-empty word (one row segment: y and z are the same for
// all its voxels) with a lane per voxel; lanes of the same component are
// merged (__match_any_sync) and the lowest of them makes the atomics for the
// group, whose x range is the span of its lanes.
__global__ void __launch_bounds__(256) k_stats(const __grid_constant__ Grid g, const __grid_constant__ Layout L,
                                               const __grid_constant__ SlotList sl) {
    pdl_begin();
    const int slot = sl.s[blockIdx.y];
    const SlotInfo* info = slot_ptr<SlotInfo>(L, slot, L.info);
    if (info->n_roots <= 0) return;
    const uint32_t* bits = slot_ptr<uint32_t>(L, slot, L.coarse);
    const int* parent = slot_ptr<int>(L, slot, L.parent);
    int* cstat = slot_ptr<int>(L, slot, L.cstat);
    const uint32_t nwords = (uint32_t)g.nz * g.ny * g.nxw;
    const int lane = threadIdx.x & 31;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (uint32_t base = 0; base < nwords; base += nwarps * 32u) {
        // words interleaved over the warps (lane l of warp k reads word
        // base + l * nwarps + k), so that neighbouring words, which often
        // belong to one object, are worked on by different warps
        const uint32_t mw = base + (uint32_t)lane * nwarps + gw;
        const uint32_t mine = mw < nwords ? __ldg(bits + mw) : 0u;
        uint32_t pending = __ballot_sync(kFull, mine != 0u);
        while (pending) {                             // the same in every lane
            const int src = __ffs(pending) - 1;
            pending &= pending - 1u;
            const uint32_t w = base + (uint32_t)src * nwarps + gw;
            const uint32_t word = __shfl_sync(kFull, mine, src);
            const uint32_t row = w / (uint32_t)g.nxw;
            const int wx = (int)(w - row * g.nxw);
            const int y = (int)(row % (uint32_t)g.ny), z = (int)(row / (uint32_t)g.ny);
            int idx = -1;
            if ((word >> lane) & 1u) {
                const int Lin = (int)row * g.nx + wx * 32 + lane;
                const int r = parent[Lin];
                const int t = r < 0 ? r : parent[r];
                if (t < 0) idx = -t - 1;              // else: roots were not tagged (capacity overflow)
            }
            const uint32_t grp = __match_any_sync(kFull, idx);
            if (idx >= 0 && lane == __ffs(grp) - 1) {
                int* st = cstat + 7 * idx;
                atomicAdd(st, __popc(grp));
                atomicMin(st + 1, wx * 32 + lane);
                atomicMax(st + 4, wx * 32 + 31 - __clz(grp));
                atomicMin(st + 2, y);
                atomicMax(st + 5, y);
                atomicMin(st + 3, z);
                atomicMax(st + 6, z);
            }
        }
    }
}

// One block per slot: Eq. (1) as its prose states it (keep iff
// t_np <= count <= t_nb), canonical labels 1..K in component order, and the
// ROI of each kept component: its box grown by one coarse voxel per side and
// clamped (Sec. II-B-3 treats it as a volume of its own), covered by whole
// fine voxels counted in integer micrometres, with the fine grid's origin and
// word layout.  Capacity overflows set a flag and leave the slot with no ROIs.
__global__ void __launch_bounds__(1024) k_filter(const __grid_constant__ Grid g, const __grid_constant__ Layout L,
                                                 const __grid_constant__ SlotList sl) {
    pdl_begin();
    __shared__ uint32_t sh[33];
    __shared__ unsigned long long sh64[33];
    __shared__ int s_fail;
    const int slot = sl.s[blockIdx.x];
    SlotInfo* info = slot_ptr<SlotInfo>(L, slot, L.info);
    const int n = info->n_roots;
    const int* cstat = slot_ptr<int>(L, slot, L.cstat);
    int* label = slot_ptr<int>(L, slot, L.roi_label);
    DRoi* rois = slot_ptr<DRoi>(L, slot, L.rois);
    if (threadIdx.x == 0) s_fail = 0;
    // pass 1: labels; components are processed in tiles of blockDim
    uint32_t base = 0;
    for (int t0 = 0; t0 < n; t0 += blockDim.x) {
        const int i = t0 + threadIdx.x;
        uint32_t keep = 0;
        if (i < n) {
            const int c = cstat[7 * i];
            keep = (c >= g.t_np && c <= g.t_nb) ? 1u : 0u;
        }
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(keep, sh, tot);
        if (i < n) label[i] = keep ? (int)(base + ex + 1) : 0;
        if (keep && base + ex < (uint32_t)g.max_rois) {
            DRoi r;
            const int* s = cstat + 7 * i;
            const int dims[3] = {g.nx, g.ny, g.nz};
            bool ok = true;
            for (int a = 0; a < 3; ++a) {
                r.cmin[a] = s[1 + a];
                r.cmax[a] = s[4 + a];
                r.gmin[a] = max(r.cmin[a] - 1, 0);
                r.gmax[a] = min(r.cmax[a] + 1, dims[a] - 1);
                const long long span = (long long)(r.gmax[a] - r.gmin[a] + 1) * g.coarse_um;
                const long long fd = (span + g.fine_um - 1) / g.fine_um;
                ok &= fd + 2 <= 32767;
                r.fdim[a] = (int)min(fd, 32765LL);
                r.fo[a] = fadd(g.o[a], fmul((float)r.gmin[a], g.sc));
            }
            r.count = s[0];
            r.nxw = (r.fdim[0] + 2 + 31) / 32;
            const unsigned long long nw = (unsigned long long)r.nxw * (r.fdim[1] + 2) * (r.fdim[2] + 2);
            ok &= nw <= g.max_fine_words;
            r.n_words = ok ? (uint32_t)nw : 0u;
            r.word_off = 0;
            r.vert_off = r.tri_off = 0;
            rois[base + ex] = r;
            if (!ok) s_fail = 1;
        }
        base += tot;
    }
    __syncthreads();
    const int K = (int)base;
    if (K > g.max_rois || s_fail) {
        if (threadIdx.x == 0) {
            info->flags |= (K > g.max_rois ? FVV_FLAG_ROIS : 0u) | (s_fail ? FVV_FLAG_FINE : 0u);
            info->n_rois = 0;
            info->n_words = 0;
        }
        return;
    }
    // pass 2: first fine word and first fine-carve tile of each ROI
    unsigned long long wbase = 0, sbase = 0;
    for (int t0 = 0; t0 < K; t0 += blockDim.x) {
        const int i = t0 + threadIdx.x;
        const unsigned long long nw = i < K ? rois[i].n_words : 0ull;
        const unsigned long long ns =
            i < K ? (unsigned long long)((rois[i].fdim[0] + kTileX - 1) / kTileX) *
                        ((rois[i].fdim[1] + g.tile_y - 1) / g.tile_y) * ((rois[i].fdim[2] + g.tile_z - 1) / g.tile_z)
                  : 0ull;
        unsigned long long tw, ts;
        const unsigned long long ew = block_exclusive_scan64(nw, sh64, tw);
        const unsigned long long es = block_exclusive_scan64(ns, sh64, ts);
        if (i < K) {
            rois[i].word_off = (uint32_t)min(wbase + ew, 0xFFFFFFFFull);
            rois[i].tile_off = (uint32_t)min(sbase + es, 0xFFFFFFFFull);
        }
        wbase += tw;
        sbase += ts;
    }
    if (threadIdx.x == 0) {
        if (wbase > g.max_fine_words || sbase > 0xFFFFFFFFull) {
            info->flags |= FVV_FLAG_FINE;
            info->n_rois = 0;
            info->n_words = 0;
        } else {
            info->n_rois = K;
            info->n_words = (uint32_t)wbase;
            info->n_tiles = (uint32_t)sbase;
            info->n_chunks = (uint32_t)((wbase + kChunk - 1) / kChunk);
        }
    }
}

}  // namespace

cudaError_t launch_ccl(const Grid& g, const Layout& L, const SlotList& sl, int sms, cudaStream_t st) {
    const long long words = (long long)g.nz * g.ny * g.nxw;
    const int gx = grid_x(sms, sl.n, words, 256);
    launch_pdl(k_union, dim3(gx, sl.n), dim3(256), 0, st, g, L, sl);
    launch_pdl(k_compress, dim3(gx, sl.n), dim3(256), 0, st, g, L, sl);
    launch_pdl(k_sort_roots, dim3(sl.n), dim3(1024), 0, st, g, L, sl);
    launch_pdl(k_stats, dim3(gx, sl.n), dim3(256), 0, st, g, L, sl);
    launch_pdl(k_filter, dim3(sl.n), dim3(1024), 0, st, g, L, sl);
    return cudaGetLastError();
}

cudaError_t launch_filter(const Grid& g, const Layout& L, const SlotList& sl, cudaStream_t st) {
    launch_pdl(k_filter, dim3(sl.n), dim3(1024), 0, st, g, L, sl);
    return cudaGetLastError();
}

// Canonical labels of every coarse voxel, for the parity tests; dst must be
// zeroed (nz*ny*nx int32).
namespace {
__global__ void k_debug_labels(const __grid_constant__ Grid g, const __grid_constant__ Layout L, int slot,
                               int32_t* dst) {
    const uint32_t* bits = slot_ptr<uint32_t>(L, slot, L.coarse);
    const int* parent = slot_ptr<int>(L, slot, L.parent);
    const int* label = slot_ptr<int>(L, slot, L.roi_label);
    const SlotInfo* info = slot_ptr<SlotInfo>(L, slot, L.info);
    if (info->n_roots <= 0) return;
    const uint32_t nwords = (uint32_t)g.nz * g.ny * g.nxw;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += gridDim.x * blockDim.x) {
        uint32_t word = bits[w];
        const uint32_t row = w / (uint32_t)g.nxw;
        const int wx = (int)(w - row * g.nxw);
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            const int Lin = (int)row * g.nx + wx * 32 + b;
            const int r = parent[Lin];
            const int t = r < 0 ? r : parent[r];
            if (t < 0) dst[Lin] = label[-t - 1];
        }
    }
}
}  // namespace

// A given coarse grid (parity tests of the labelling): copies the words into
// the slot with the bits past nx cleared, and starts the union-find forest
// exactly as k_coarse_carve does (each run of a word one tree rooted at its
// first voxel), counting the occupied voxels.  One thread per word.
namespace {
__global__ void k_debug_seed(const __grid_constant__ Grid g, const __grid_constant__ Layout L, int slot,
                             const uint32_t* src) {
    uint32_t* bits = slot_ptr<uint32_t>(L, slot, L.coarse);
    int* parent = slot_ptr<int>(L, slot, L.parent);
    SlotInfo* info = slot_ptr<SlotInfo>(L, slot, L.info);
    const uint32_t nwords = (uint32_t)g.nz * g.ny * g.nxw;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += gridDim.x * blockDim.x) {
        const uint32_t row = w / (uint32_t)g.nxw;
        const int wx = (int)(w - row * g.nxw);
        uint32_t word = src[w];
        if (wx == g.nxw - 1 && (g.nx & 31)) word &= (1u << (g.nx & 31)) - 1u;
        bits[w] = word;
        if (word) atomicAdd(&info->n_on, (uint32_t)__popc(word));
        const uint32_t starts = word & ~(word << 1);
        for (uint32_t m = word; m; m &= m - 1u) {
            const int b = __ffs(m) - 1;
            const int run0 = 31 - __clz(starts & (0xFFFFFFFFu >> (31 - b)));
            parent[(int)row * g.nx + wx * 32 + b] = (int)row * g.nx + wx * 32 + run0;
        }
    }
}
}  // namespace

cudaError_t launch_debug_seed(const Grid& g, const Layout& L, int slot, const uint32_t* src, cudaStream_t st) {
    const long long words = (long long)g.nz * g.ny * g.nxw;
    k_debug_seed<<<(unsigned)std::min<long long>((words + 255) / 256, 4096), 256, 0, st>>>(g, L, slot, src);
    return cudaGetLastError();
}

cudaError_t launch_debug_labels(const Grid& g, const Layout& L, int slot, int32_t* dst, cudaStream_t st) {
    const long long words = (long long)g.nz * g.ny * g.nxw;
    k_debug_labels<<<(unsigned)std::min<long long>((words + 255) / 256, 4096), 256, 0, st>>>(g, L, slot, dst);
    return cudaGetLastError();
}

}  // namespace fvv
