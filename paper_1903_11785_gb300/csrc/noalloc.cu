// noalloc.cu -- fvv_label_components_noalloc: 26-connected labelling of a
// coarse occupancy bitset with the size filter, for callers that cannot
// allocate device memory.
//
// Its scratch (union-find parents, the component list and per-component
// statistics) lives in one file-scope static __device__ array, so the call
// allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.
// The array is part of the library image, so every GPU that loads the
// library holds it (kScratchInts ints, about 32.4 MB) until the process exits.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so the first call on each device, with that
// device current, asks cudaGetSymbolAddress for the real address and keeps it.
// That first call should therefore come before any stream capture.
//
// Every call shares the one array: calls that overlap on the GPU (on
// different streams, or from different threads) race on it.  Each call
// clears what must start at zero; the rest is written before it is read.
#include <mutex>

#include "fvv_device.cuh"

namespace fvv {
namespace {

constexpr int kNaMaxVoxels = 8 * 1024 * 1024;       // 8,388,608 coarse voxels
constexpr int kNaMaxComponents = kMaxComponents;    // 8192 raw components
// layout, in ints: [0] root count, [1] flags, [64 ..) roots, then per-component
// statistics (7 each), then labels per component, then parents per voxel
constexpr int kNaRoots = 64;
constexpr int kNaStats = kNaRoots + kNaMaxComponents;
constexpr int kNaLabel = kNaStats + 7 * kNaMaxComponents;
constexpr int kNaParent = (kNaLabel + kNaMaxComponents + 63) / 64 * 64;
constexpr int kScratchInts = kNaParent + kNaMaxVoxels;

static __device__ __align__(256) int g_na_scratch[kScratchInts];

struct NaGrid {
    const uint32_t* bits;
    int nx, ny, nz, nxw;
    int t_np, t_nb;
};

constexpr int kNaBudget = 1 << 22;

// Root of x while unions run, shortening the path on the way; its plain
// stores are safe only in k_na_union (see na_find_readonly).
__device__ __forceinline__ int na_find(int* parent, int x, int& budget) {
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

// Root of x after the unions, writing nothing.  In k_na_compress each thread
// stores only its own voxel's root, so every entry changes at most once, from
// an ancestor to the root; no other store can overwrite that root afterwards
// (a shortening store here could, which would leave the voxel pointing at an
// intermediate node and out of its component's count and box).
__device__ __forceinline__ int na_find_readonly(const int* parent, int x, int& budget) {
    int cur = x;
    while (budget > 0) {
        --budget;
        const int next = __ldcg(parent + cur);
        if (next == cur || next < 0) return cur;
        cur = next;
    }
    return cur;
}

__device__ __forceinline__ void na_unite(int* parent, int a, int b, int& budget) {
    while (budget > 0) {
        a = na_find(parent, a, budget);
        b = na_find(parent, b, budget);
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

__device__ __forceinline__ bool na_on(const NaGrid& g, int x, int y, int z) {
    if (x < 0 || y < 0 || z < 0 || x >= g.nx || y >= g.ny || z >= g.nz) return false;
    return (__ldg(g.bits + ((size_t)z * g.ny + y) * g.nxw + (x >> 5)) >> (x & 31)) & 1u;
}

// Zero the counters, start a tree at every occupied voxel.
__global__ void k_na_init(NaGrid g, int* sc) {
    if (blockIdx.x == 0 && threadIdx.x < 64) sc[threadIdx.x] = 0;
    int* parent = sc + kNaParent;
    const uint32_t nwords = (uint32_t)g.nz * g.ny * g.nxw;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += gridDim.x * blockDim.x) {
        uint32_t word = __ldg(g.bits + w);
        const uint32_t row = w / (uint32_t)g.nxw;
        const int wx = (int)(w - row * g.nxw);
        if (wx == g.nxw - 1 && (g.nx & 31)) word &= (1u << (g.nx & 31)) - 1u;   // ignore bits past nx
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            const int L = (int)row * g.nx + wx * 32 + b;
            parent[L] = L;
        }
    }
}

__global__ void k_na_union(NaGrid g, int* sc) {
    int* parent = sc + kNaParent;
    const uint32_t nwords = (uint32_t)g.nz * g.ny * g.nxw;
    int budget = kNaBudget;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nwords && budget > 0; w += gridDim.x * blockDim.x) {
        uint32_t word = __ldg(g.bits + w);
        const uint32_t row = w / (uint32_t)g.nxw;
        const int wx = (int)(w - row * g.nxw);
        if (wx == g.nxw - 1 && (g.nx & 31)) word &= (1u << (g.nx & 31)) - 1u;
        const int y = (int)(row % (uint32_t)g.ny), z = (int)(row / (uint32_t)g.ny);
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            const int x = wx * 32 + b;
            const int L = (int)row * g.nx + x;
            for (int dz = -1; dz <= 0; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (dz == 0 && (dy > 0 || (dy == 0 && dx >= 0))) continue;
                        if (!na_on(g, x + dx, y + dy, z + dz)) continue;
                        na_unite(parent, L, ((z + dz) * g.ny + (y + dy)) * g.nx + (x + dx), budget);
                    }
        }
    }
    if (budget <= 0) atomicOr(sc + 1, (int)FVV_FLAG_LOOP);
}

__global__ void k_na_compress(NaGrid g, int* sc) {
    int* parent = sc + kNaParent;
    const uint32_t nwords = (uint32_t)g.nz * g.ny * g.nxw;
    int budget = kNaBudget;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nwords && budget > 0; w += gridDim.x * blockDim.x) {
        uint32_t word = __ldg(g.bits + w);
        const uint32_t row = w / (uint32_t)g.nxw;
        const int wx = (int)(w - row * g.nxw);
        if (wx == g.nxw - 1 && (g.nx & 31)) word &= (1u << (g.nx & 31)) - 1u;
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            const int L = (int)row * g.nx + wx * 32 + b;
            const int r = na_find_readonly(parent, L, budget);
            if (r == L) {
                const int k = atomicAdd(sc, 1);
                if (k < kNaMaxComponents) sc[kNaRoots + k] = L;
            } else {
                parent[L] = r;
            }
        }
    }
    if (budget <= 0) atomicOr(sc + 1, (int)FVV_FLAG_LOOP);
}

// One block: sort the roots, tag each root's parent entry with -(i+1), reset
// the statistics.
__global__ void __launch_bounds__(1024) k_na_sort(int* sc) {
    __shared__ int key[kNaMaxComponents];
    const int n = sc[0];
    if (n > kNaMaxComponents) return;
    int* parent = sc + kNaParent;
    int m = 1;
    while (m < n) m <<= 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x) key[i] = i < n ? sc[kNaRoots + i] : 0x7FFFFFFF;
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1)
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
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        parent[key[i]] = -(i + 1);
        int* s = sc + kNaStats + 7 * i;
        s[0] = 0;
        s[1] = s[2] = s[3] = 0x7FFFFFFF;
        s[4] = s[5] = s[6] = -1;
    }
}

// Component index of occupied voxel L after tagging, or -1.
__device__ __forceinline__ int na_comp(const int* parent, int L) {
    const int r = parent[L];
    const int t = r < 0 ? r : parent[r];
    return t < 0 ? -t - 1 : -1;
}

__global__ void k_na_stats(NaGrid g, int* sc) {
    if (sc[0] > kNaMaxComponents) return;
    const int* parent = sc + kNaParent;
    const uint32_t nwords = (uint32_t)g.nz * g.ny * g.nxw;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += gridDim.x * blockDim.x) {
        uint32_t word = __ldg(g.bits + w);
        const uint32_t row = w / (uint32_t)g.nxw;
        const int wx = (int)(w - row * g.nxw);
        if (wx == g.nxw - 1 && (g.nx & 31)) word &= (1u << (g.nx & 31)) - 1u;
        const int y = (int)(row % (uint32_t)g.ny), z = (int)(row / (uint32_t)g.ny);
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            const int x = wx * 32 + b;
            const int c = na_comp(parent, (int)row * g.nx + x);
            if (c < 0) continue;
            int* s = sc + kNaStats + 7 * c;
            atomicAdd(s, 1);
            atomicMin(s + 1, x); atomicMin(s + 2, y); atomicMin(s + 3, z);
            atomicMax(s + 4, x); atomicMax(s + 5, y); atomicMax(s + 6, z);
        }
    }
}

// One block: keep iff t_np <= count <= t_nb, labels 1..K in component order.
__global__ void __launch_bounds__(1024) k_na_filter(NaGrid g, int* sc, int32_t* counts) {
    __shared__ uint32_t sh[33];
    const int n = sc[0];
    const bool over = n > kNaMaxComponents;
    uint32_t base = 0;
    for (int t0 = 0; t0 < (over ? 0 : n); t0 += blockDim.x) {
        const int i = t0 + threadIdx.x;
        uint32_t keep = 0;
        if (i < n) {
            const int c = sc[kNaStats + 7 * i];
            keep = (c >= g.t_np && c <= g.t_nb) ? 1u : 0u;
        }
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(keep, sh, tot);
        if (i < n) sc[kNaLabel + i] = keep ? (int)(base + ex + 1) : 0;
        base += tot;
    }
    if (threadIdx.x == 0) {
        counts[0] = n;
        counts[1] = over ? 0 : (int)base;
        counts[2] = sc[1] | (over ? (int)FVV_FLAG_ROOTS : 0);
    }
}

// Every voxel of the output: its canonical label, 0 for empty or removed.
__global__ void k_na_labels(NaGrid g, const int* sc, int32_t* labels) {
    const bool ok = sc[0] <= kNaMaxComponents;
    const int* parent = sc + kNaParent;
    const uint32_t nwords = (uint32_t)g.nz * g.ny * g.nxw;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += gridDim.x * blockDim.x) {
        const uint32_t word = __ldg(g.bits + w);
        const uint32_t row = w / (uint32_t)g.nxw;
        const int wx = (int)(w - row * g.nxw);
        const int nb = min(32, g.nx - wx * 32);
        for (int b = 0; b < nb; ++b) {
            const int L = (int)row * g.nx + wx * 32 + b;
            int lab = 0;
            if (ok && ((word >> b) & 1u)) {
                const int c = na_comp(parent, L);
                lab = c >= 0 ? sc[kNaLabel + c] : 0;
            }
            labels[L] = lab;
        }
    }
}

std::mutex g_na_mutex;
int* g_na_ptr[256] = {};   // device address of g_na_scratch, per device ordinal

}  // namespace
}  // namespace fvv

using namespace fvv;

extern "C" fvv_status fvv_label_components_noalloc(const uint32_t* coarse_bits, int nx, int ny, int nz, int t_np,
                                                   int t_nb, int32_t* labels, int32_t* counts, void* stream) {
    if (!coarse_bits || !labels || !counts) return FVV_ERR_INVALID_ARG;
    if (nx < 1 || ny < 1 || nz < 1) return FVV_ERR_INVALID_ARG;
    if ((long long)nx * ny * nz > kNaMaxVoxels) return FVV_ERR_INVALID_ARG;   // beyond the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return FVV_ERR_CUDA;
    int* sc = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) return FVV_ERR_CUDA;
            g_na_ptr[dev] = static_cast<int*>(p);
        }
        sc = g_na_ptr[dev];
    }
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    NaGrid g{coarse_bits, nx, ny, nz, (nx + 31) / 32, t_np, t_nb};
    const long long words = (long long)nz * ny * g.nxw;
    const unsigned blocks = (unsigned)std::max(1LL, std::min((words + 255) / 256, 4096LL));
    k_na_init<<<blocks, 256, 0, st>>>(g, sc);
    k_na_union<<<blocks, 256, 0, st>>>(g, sc);
    k_na_compress<<<blocks, 256, 0, st>>>(g, sc);
    k_na_sort<<<1, 1024, 0, st>>>(sc);
    k_na_stats<<<blocks, 256, 0, st>>>(g, sc);
    k_na_filter<<<1, 1024, 0, st>>>(g, sc, counts);
    k_na_labels<<<blocks, 256, 0, st>>>(g, sc, labels);
    return cudaGetLastError() == cudaSuccess ? FVV_OK : FVV_ERR_CUDA;
}
