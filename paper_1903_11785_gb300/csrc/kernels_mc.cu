// kernels_mc.cu -- Sec. II-C: surface polygonisation of every fine grid.
//
// Each fine grid is padded by one unoccupied sample per side and stored as
// rows of 32-bit words, so one thread owns 32 cells (or 32 samples) and works
// with word-wide bit operations:
//   compact   bipolar-edge masks (x: w ^ w>>1, y: w ^ w(y+1), z: w ^ w(z+1)),
//             vertices = popcounts, triangles = table counts of mixed cells;
//             exclusive prefix per word (block scan + a look-back over the
//             earlier 256-word chunks) and one record per bipolar edge, in
//             edge-key order (3*Lpad + axis), and one per triangle; the
//             grid slab a chunk reads is staged in shared memory by a bulk
//             copy.
//   bisect    one thread per vertex: fixed-count bisection of its edge
//             against the silhouettes (the exact intersection of Eqs. (2)-(3)
//             read as the hull crossing on the edge).
//   triangles table triangles of each mixed cell, vertex ids = word prefix +
//             rank of the edge inside its word.
// Vertex and triangle order is therefore (ROI, key) and (ROI, cell, table
// order): independent of scheduling, identical to a serial scan.
#include <atomic>

#include "fvv_device.cuh"

namespace fvv {

// ------------------------------------------------------------ MC table (host)
//
// Corners are numbered x + 2y + 4z.  Cube edge e runs along axis e/4 from its
// lower corner, whose other two coordinates, in increasing axis order, are
// (e & 1, e >> 1 & 1).  On every face the bipolar edges are joined by
// segments (two bipolar edges: one segment; four, i.e. two diagonal ON
// corners: one segment around each ON corner, keeping ON corners apart), each
// directed so that the ON side is on its right seen from outside the cube;
// chaining them gives loops whose normals point from ON to OFF.  Loops are
// taken in order of their smallest edge, walked from it, and fanned from the
// first vertex that shares no face with a vertex it is not adjacent to.
namespace {

void edge_ends(int e, int& lo, int& hi) {
    const int axis = e >> 2;
    int other[2], k = 0;
    for (int b = 0; b < 3; ++b)
        if (b != axis) other[k++] = b;
    lo = ((e & 1) << other[0]) | (((e >> 1) & 1) << other[1]);
    hi = lo | (1 << axis);
}

int edge_of(int c0, int c1) {
    for (int e = 0; e < 12; ++e) {
        int lo, hi;
        edge_ends(e, lo, hi);
        if ((lo == c0 && hi == c1) || (lo == c1 && hi == c0)) return e;
    }
    return -1;
}

}  // namespace

void build_mc_table(uint8_t ntri[256], uint8_t edges[256 * kMaxTriPerCell * 3]) {
    // face membership of every edge, and each face's corner cycle
    int face_mask[12] = {0};
    int cyc[6][4];
    for (int f = 0; f < 6; ++f) {
        const int b = f >> 1, t = f & 1;
        const int p = b == 0 ? 1 : 0, q = b == 2 ? 1 : 2;
        const int uv[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
        for (int i = 0; i < 4; ++i) cyc[f][i] = (t << b) | (uv[i][0] << p) | (uv[i][1] << q);
        for (int i = 0; i < 4; ++i) face_mask[edge_of(cyc[f][i], cyc[f][(i + 1) & 3])] |= 1 << f;
    }
    for (int cs = 0; cs < 256; ++cs) {
        int nxt[12];
        for (int e = 0; e < 12; ++e) nxt[e] = -1;
        for (int f = 0; f < 6; ++f) {
            const int b = f >> 1, t = f & 1;
            const int hand = b == 1 ? -1 : 1;       // (p, q, b) right-handed?
            const int side = t ? 1 : -1;            // outward normal along b
            const int uv[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
            int s[4], fe[4], nb = 0;
            for (int i = 0; i < 4; ++i) s[i] = (cs >> cyc[f][i]) & 1;
            for (int i = 0; i < 4; ++i)
                if (s[i] != s[(i + 1) & 3]) fe[nb++] = i;  // face edge i joins corners i, i+1
            int seg[2][3], ns = 0;                          // (face edge, face edge, ON corner)
            if (nb == 2) {
                int on = 0;
                while (!s[on]) ++on;
                seg[0][0] = fe[0]; seg[0][1] = fe[1]; seg[0][2] = on;
                ns = 1;
            } else if (nb == 4) {
                for (int i = 0; i < 4; ++i)
                    if (s[i]) {
                        seg[ns][0] = (i + 3) & 3; seg[ns][1] = i; seg[ns][2] = i;
                        ++ns;
                    }
            }
            for (int k = 0; k < ns; ++k) {
                const int i0 = seg[k][0], i1 = seg[k][1], a = seg[k][2];
                // doubled face-plane coordinates of the two midpoints and the ON corner
                const int P[2] = {uv[i0][0] + uv[(i0 + 1) & 3][0], uv[i0][1] + uv[(i0 + 1) & 3][1]};
                const int Q[2] = {uv[i1][0] + uv[(i1 + 1) & 3][0], uv[i1][1] + uv[(i1 + 1) & 3][1]};
                const int A[2] = {2 * uv[a][0], 2 * uv[a][1]};
                const int cr = (Q[0] - P[0]) * (A[1] - P[1]) - (Q[1] - P[1]) * (A[0] - P[0]);
                const int ep = edge_of(cyc[f][i0], cyc[f][(i0 + 1) & 3]);
                const int eq = edge_of(cyc[f][i1], cyc[f][(i1 + 1) & 3]);
                if (cr * hand * side < 0) nxt[ep] = eq;
                else nxt[eq] = ep;
            }
        }
        int done = 0, nt = 0;
        for (int e0 = 0; e0 < 12; ++e0) {
            if (nxt[e0] < 0 || (done >> e0 & 1)) continue;
            int loop[12], n = 0;
            for (int e = e0; !(done >> e & 1); e = nxt[e]) {
                done |= 1 << e;
                loop[n++] = e;
            }
            int apex = 0;
            for (int i = 0; i < n; ++i) {
                bool ok = true;
                for (int d = 2; d + 1 < n && ok; ++d)
                    if (face_mask[loop[i]] & face_mask[loop[(i + d) % n]]) ok = false;
                if (ok) {
                    apex = i;
                    break;
                }
            }
            for (int d = 1; d + 1 < n; ++d) {
                uint8_t* o = edges + ((size_t)cs * kMaxTriPerCell + nt) * 3;
                o[0] = (uint8_t)loop[apex];
                o[1] = (uint8_t)loop[(apex + d) % n];
                o[2] = (uint8_t)loop[(apex + d + 1) % n];
                ++nt;
            }
        }
        ntri[cs] = (uint8_t)nt;
    }
}

// ------------------------------------------------------------------ kernels
namespace {

// The 8 words around fine word w (rows y, y+1 and planes z, z+1; this word
// and the next in x) as "samples at xp" (c*) and "samples at xp+1" (s*),
// indexed by corner bits (dy + 2dz).
struct Nbhd {
    uint32_t w[4];   // sample xp, corner dy + 2 dz
    uint32_t s[4];   // sample xp + 1
};

__device__ __forceinline__ void load_nbhd(const uint32_t* fine, const RoiCursor& r, uint32_t w, Nbhd& n) {
    const uint32_t rs = (uint32_t)r.nxw, ps = (uint32_t)r.nxw * (uint32_t)(r.fdim[1] + 2);
    const bool hx = r.wx + 1 < r.nxw, hy = r.yp + 1 < r.fdim[1] + 2, hz = r.zp + 1 < r.fdim[2] + 2;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool dy = k & 1, dz = k >> 1;
        const bool ok = (!dy || hy) && (!dz || hz);
        const uint32_t base = w + (dy ? rs : 0u) + (dz ? ps : 0u);
        const uint32_t a = ok ? __ldg(fine + base) : 0u;
        const uint32_t b = (ok && hx) ? __ldg(fine + base + 1) : 0u;
        n.w[k] = a;
        n.s[k] = (a >> 1) | (b << 31);
    }
}

__device__ __forceinline__ uint32_t mixed_cells(const Nbhd& n) {
    const uint32_t a = n.w[0];
    return (a ^ n.s[0]) | (a ^ n.w[1]) | (a ^ n.s[1]) | (a ^ n.w[2]) | (a ^ n.s[2]) | (a ^ n.w[3]) | (a ^ n.s[3]);
}

__device__ __forceinline__ int cell_case(const Nbhd& n, int b) {
    int c = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        c |= (int)((n.w[k] >> b) & 1u) << (2 * k);
        c |= (int)((n.s[k] >> b) & 1u) << (2 * k + 1);
    }
    return c;
}

// The 8 words of load_nbhd, read from a slab of the slot's fine words
// staged in shared memory (slab[i] = fine word lo + i).
__device__ __forceinline__ void load_nbhd_slab(const uint32_t* slab, uint32_t lo, const RoiCursor& r, uint32_t w,
                                               Nbhd& n) {
    const uint32_t rs = (uint32_t)r.nxw, ps = (uint32_t)r.nxw * (uint32_t)(r.fdim[1] + 2);
    const bool hx = r.wx + 1 < r.nxw, hy = r.yp + 1 < r.fdim[1] + 2, hz = r.zp + 1 < r.fdim[2] + 2;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool dy = k & 1, dz = k >> 1;
        const bool ok = (!dy || hy) && (!dz || hz);
        const uint32_t i = w - lo + (dy ? rs : 0u) + (dz ? ps : 0u);
        const uint32_t a = ok ? slab[i] : 0u;
        const uint32_t b = (ok && hx) ? slab[i + 1] : 0u;
        n.w[k] = a;
        n.s[k] = (a >> 1) | (b << 31);
    }
}

// ---- staging through the tensor memory accelerator (1-D bulk copies into
// shared memory, completion counted on an mbarrier)
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival that also expects `bytes` of copies to complete on the barrier.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0u;
}

// Copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from
// global to shared memory; completes on `bar`.  Shared memory that generic
// loads read before must be ordered before the copy (fence_proxy_async).
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Decoupled look-back state of a chunk, one word per count (vertices,
// triangles): bits 62-63 say what bits 0-61 hold -- 0 nothing yet, 1 the
// chunk's own count, 2 the count of chunks 0..c together.
constexpr unsigned long long kStAgg = 1ull << 62, kStInc = 2ull << 62, kStVal = (1ull << 62) - 1ull;

__device__ __forceinline__ void st_state(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_state(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Polls of a bounded wait (the slab copy, or the states of earlier chunks)
// before the kernel gives up on it and sets FVV_FLAG_LOOP.
constexpr int kMaxPolls = 1 << 22;

// Counts (vertices, triangles) of the chunks before chunk c, by warp 0: the
// lanes read the states of 32 earlier chunks at a time (lane i: chunk
// top - i), wait until all 32 are published, and add the values from the
// nearest chunk back to the first inclusive one; without an inclusive one
// in the window, all 32 and the window before.  False if the polls ran out.
__device__ __forceinline__ bool look_back_warp(const unsigned long long* st, uint32_t c, unsigned long long& sv,
                                               unsigned long long& stt) {
    const int lane = threadIdx.x & 31;
    sv = stt = 0;
    bool need_v = true, need_t = true;
    int polls = 0;
    for (long long top = (long long)c - 1; top >= 0 && (need_v || need_t);) {
        const long long q = top - lane;
        // chunks before chunk 0 read as an inclusive zero, which ends the walk
        const unsigned long long a = q >= 0 ? ld_state(st + 2 * q) : kStInc;
        const unsigned long long b = q >= 0 ? ld_state(st + 2 * q + 1) : kStInc;
        if (__any_sync(kFull, (a >> 62) == 0ull || (b >> 62) == 0ull)) {
            if (++polls > kMaxPolls) return false;
            continue;
        }
        const unsigned iv = __ballot_sync(kFull, (a >> 62) == 2ull), it = __ballot_sync(kFull, (b >> 62) == 2ull);
        const int lv = iv ? __ffs(iv) - 1 : 31, lt = it ? __ffs(it) - 1 : 31;
        unsigned long long xv = (need_v && lane <= lv) ? (a & kStVal) : 0ull;
        unsigned long long xt = (need_t && lane <= lt) ? (b & kStVal) : 0ull;
        for (int o = 16; o > 0; o >>= 1) {
            xv += __shfl_xor_sync(kFull, xv, o);
            xt += __shfl_xor_sync(kFull, xt, o);
        }
        sv += xv;
        stt += xt;
        need_v = need_v && !iv;
        need_t = need_t && !it;
        top -= 32;
    }
    return true;
}

// Vertex record: ROI (14 bits) | axis (2) | ON at lower sample (1) | xp, yp, zp (15 bits each).
__device__ __forceinline__ uint64_t pack_vrec(int k, int axis, int s0on, int xp, int yp, int zp) {
    return (uint64_t)k | (uint64_t)axis << 14 | (uint64_t)s0on << 16 | (uint64_t)xp << 17 | (uint64_t)yp << 32 |
           (uint64_t)zp << 47;
}

// Triangle record: fine word (26 bits) | cell bit (5) | triangle of the cell
// (4) | cell case (8) | ROI (14).
__device__ __forceinline__ uint64_t pack_trec(uint32_t w, int b, int j, int cs, int k) {
    return (uint64_t)w | (uint64_t)b << 26 | (uint64_t)j << 31 | (uint64_t)cs << 35 | (uint64_t)k << 43;
}

// Sec. II-C classify and compact, in one pass over each slot's fine words:
// 256-word chunks are claimed in order from a per-slot counter; a chunk's
// words and the neighbours its cells reach (a slab) are copied into shared
// memory by one bulk copy; each thread takes one word: its bipolar-edge
// masks (x: w ^ w>>1, y: w ^ w(y+1), z: w ^ w(z+1)), vertex count (their
// popcounts) and triangle count (table counts of its mixed cells).  Block
// scans give the offsets within the chunk, and a decoupled look-back over
// the earlier chunks' published counts gives the chunk's base, so vertex
// ids follow the edge-key order (3*Lpad + axis) and triangles (ROI, cell,
// table order) of a serial scan.  Each word then writes its prefix, masks,
// one record per vertex and one per triangle; the last chunk sets the
// totals and the capacity flags.  A chunk waits only on chunks claimed
// before it, whose blocks are running, so the look-back always ends.
__global__ void __launch_bounds__(kChunk) k_mc_compact(const __grid_constant__ Grid g,
                                                       const __grid_constant__ Layout L,
                                                       const __grid_constant__ SlotList sl,
                                                       const __grid_constant__ McTable mc) {
    pdl_begin();
    extern __shared__ __align__(128) uint32_t slab[];   // kSlabWords
    __shared__ uint8_t s_ntri[256];
    __shared__ uint32_t sh[33];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_c, s_use;
    __shared__ unsigned long long s_base[2];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) s_ntri[i] = mc.ntri[i];
    if (threadIdx.x == 0) mbar_init(&bar);
    __syncthreads();
    const int slot = sl.s[blockIdx.y];
    SlotInfo* info = slot_ptr<SlotInfo>(L, slot, L.info);
    const uint32_t nwords = info->n_words, nchunks = info->n_chunks;
    const int nrois = info->n_rois;
    DRoi* rois = slot_ptr<DRoi>(L, slot, L.rois);
    const uint32_t* fine = slot_ptr<uint32_t>(L, slot, L.fine);
    uint32_t* emask = slot_ptr<uint32_t>(L, slot, L.emask);
    uint32_t* vpre = slot_ptr<uint32_t>(L, slot, L.vpre);
    uint64_t* vrec = slot_ptr<uint64_t>(L, slot, L.vrec);
    uint64_t* trec = slot_ptr<uint64_t>(L, slot, L.trec);
    unsigned long long* cst = slot_ptr<unsigned long long>(L, slot, L.chunk_st);
    const uint32_t* clen = slot_ptr<uint32_t>(L, slot, L.chunk_len);
    uint32_t parity = 0;
    bool pending = false;   // a copy whose wait ran out may still be in flight (thread 0's view)
    RoiCursor p;
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t c = nchunks ? atomicAdd(&info->next_chunk, 1u) : 0u;
            s_c = c;
            s_use = 0;
            const uint32_t n4 = c < nchunks && !pending ? __ldcg(clen + c) : 0u;   // (k_clear_fine)
            if (n4) {
                s_use = 1;
                fence_proxy_async();
                mbar_expect_tx(&bar, n4 * 4u);
                bulk_copy_g2s(slab, fine + c * kChunk, n4 * 4u, &bar);
            }
        }
        __syncthreads();
        const uint32_t c = s_c;
        if (c >= nchunks) break;
        bool use = s_use != 0u;
        if (use) {
            bool done = false;
            for (int it = 0; it < kMaxPolls && !done; ++it) done = mbar_try_wait(&bar, parity);
            if (__syncthreads_or(!done)) {
                // the copy did not complete in time: this chunk and the later
                // ones read global memory, and the slot is flagged
                use = false;
                if (threadIdx.x == 0) {
                    pending = true;
                    atomicOr(&info->flags, (unsigned)FVV_FLAG_LOOP);
                }
            } else {
                parity ^= 1u;
            }
        }
        const uint32_t lo = c * kChunk, w = lo + threadIdx.x;
        const bool in = w < nwords;
        Nbhd n;
        uint32_t xm = 0, ym = 0, zm = 0, vc = 0, tc = 0;
        if (in) {
            p.seek(rois, nrois, w);
            if (use) load_nbhd_slab(slab, lo, p, w, n);
            else load_nbhd(fine, p, w, n);
            xm = n.w[0] ^ n.s[0];
            ym = n.w[0] ^ n.w[1];
            zm = n.w[0] ^ n.w[2];
            vc = __popc(xm) + __popc(ym) + __popc(zm);
            uint32_t mx = mixed_cells(n);
            while (mx) {
                const int b = __ffs(mx) - 1;
                mx &= mx - 1;
                tc += s_ntri[cell_case(n, b)];
            }
        }
        uint32_t tv, tt;
        const uint32_t ev = block_exclusive_scan(vc, sh, tv);
        const uint32_t et = block_exclusive_scan(tc, sh, tt);
        if (threadIdx.x < 32) {
            unsigned long long bv = 0, bt = 0;
            bool ok = true;
            if (c > 0) {
                if (threadIdx.x == 0) {
                    st_state(cst + 2 * (size_t)c, kStAgg | tv);
                    st_state(cst + 2 * (size_t)c + 1, kStAgg | tt);
                }
                ok = look_back_warp(cst, c, bv, bt);
            }
            if (threadIdx.x == 0) {
                st_state(cst + 2 * (size_t)c, kStInc | ((bv + tv) & kStVal));
                st_state(cst + 2 * (size_t)c + 1, kStInc | ((bt + tt) & kStVal));
                if (!ok) atomicOr(&info->flags, (unsigned)FVV_FLAG_LOOP);
                s_base[0] = bv;
                s_base[1] = bt;
                if (c == nchunks - 1u) {
                    // totals and capacities (the records past a capacity were not written)
                    const unsigned long long nv = bv + tv, nt = bt + tt;
                    unsigned fl = 0;
                    if (nv > g.max_verts) fl |= FVV_FLAG_VERTS;
                    if (nt > g.max_tris) fl |= FVV_FLAG_TRIS;
                    if (fl) atomicOr(&info->flags, fl);
                    info->n_verts = fl ? 0u : (uint32_t)nv;
                    info->n_tris = fl ? 0u : (uint32_t)nt;
                    if (fl) info->n_words = 0;   // nothing downstream runs on this frame
                }
            }
        }
        __syncthreads();
        if (in) {
            const unsigned long long vb = s_base[0] + ev, tb = s_base[1] + et;
            vpre[w] = (uint32_t)vb;
            if (w == p.lo) {
                rois[p.k].vert_off = (uint32_t)vb;
                rois[p.k].tri_off = (uint32_t)tb;
            }
            emask[3 * (size_t)w + 0] = xm;
            emask[3 * (size_t)w + 1] = ym;
            emask[3 * (size_t)w + 2] = zm;
            const uint32_t own = n.w[0];
            uint32_t any = xm | ym | zm;
            unsigned long long id = vb;
            while (any) {
                const int b = __ffs(any) - 1;
                any &= any - 1;
                const int s0 = (own >> b) & 1u, xp = p.wx * 32 + b;
                if (((xm >> b) & 1u) && id < g.max_verts) vrec[id] = pack_vrec(p.k, 0, s0, xp, p.yp, p.zp);
                id += (xm >> b) & 1u;
                if (((ym >> b) & 1u) && id < g.max_verts) vrec[id] = pack_vrec(p.k, 1, s0, xp, p.yp, p.zp);
                id += (ym >> b) & 1u;
                if (((zm >> b) & 1u) && id < g.max_verts) vrec[id] = pack_vrec(p.k, 2, s0, xp, p.yp, p.zp);
                id += (zm >> b) & 1u;
            }
            if (tc) {
                uint32_t mx = mixed_cells(n);
                unsigned long long t = tb;
                while (mx) {
                    const int b = __ffs(mx) - 1;
                    mx &= mx - 1;
                    const int cs = cell_case(n, b);
                    for (int j = 0; j < (int)s_ntri[cs]; ++j, ++t)
                        if (t < g.max_tris) trec[t] = pack_trec(w, b, j, cs, p.k);
                }
            }
        }
    }
    if (threadIdx.x == 0 && pending) {
        // a copy whose wait ran out: wait (bounded) before the block's shared memory goes
        for (int it = 0; it < kMaxPolls && !mbar_try_wait(&bar, parity); ++it) {
        }
    }
}

// Does camera c see every point the bisection of the edge (a, b) can test in
// its silhouette?  True when the pixels of the box spanned by the ends'
// approximate image positions, widened by the camera's margins (see
// segment_margins on the host), are all inside the image and set.  Boxes
// wider than 32 or taller than 8 pixels are not scanned (false).
template <class CamT>
__device__ __forceinline__ bool segment_all_fg(const CamT& c, const uint32_t* __restrict__ sil, const float* a,
                                               const float* b, unsigned long long& reads) {
    if (!(c.du >= 0.0f)) return false;
    float xa, ya, wa, xb, yb, wb;
    project(c.P, a[0], a[1], a[2], xa, ya, wa);
    project(c.P, b[0], b[1], b[2], xb, yb, wb);
    if (!(wa > 0.0f && wb > 0.0f)) return false;
    const float ra = rcp_approx(wa), rb = rcp_approx(wb);
    const float ua = fmul(xa, ra), va = fmul(ya, ra), ub = fmul(xb, rb), vb = fmul(yb, rb);
    const float u0 = fsub(fminf(ua, ub), c.du), u1 = fadd(fmaxf(ua, ub), c.du);
    const float v0 = fsub(fminf(va, vb), c.dv), v1 = fadd(fmaxf(va, vb), c.dv);
    if (!(u0 >= 0.0f && v0 >= 0.0f && u1 < c.Wf && v1 < c.Hf)) return false;
    const int x0 = (int)u0, x1 = (int)u1, y0 = (int)v0, y1 = (int)v1;   // truncation = floor here
    if (x1 - x0 > 31 || y1 - y0 > 7) return false;
    const int w0 = x0 >> 5, w1 = x1 >> 5;
    const uint32_t m0 = ~0u << (x0 & 31), m1 = ~0u >> (31 - (x1 & 31));
    const uint32_t* row = sil + c.bit_off + (unsigned)y0 * (unsigned)c.Wq;
    bool all = true;
    for (int y = y0; y <= y1; ++y, row += c.Wq) {
        if (w0 == w1) {
            all &= (__ldg(row + w0) & (m0 & m1)) == (m0 & m1);
        } else {
            all &= (__ldg(row + w0) & m0) == m0;
            all &= (__ldg(row + w1) & m1) == m1;
        }
    }
    reads += (unsigned)((y1 - y0 + 1) * (w1 - w0 + 1));
    return all;
}

// Sec. II-C, exact intersection: between the ON end a and the OFF end b of a
// bipolar edge, `steps` times m = (a+b)/2, a = m if m is occupied else b = m;
// the vertex is the final midpoint.
//
// Every point tested lies on the edge (up to rounding), so a camera that sees
// the whole edge inside its silhouette (segment_all_fg) votes foreground for
// all of them: it is decided once per edge, and only the other cameras are
// tested at each midpoint, from the vertex's list.  A midpoint's first
// background camera in index order is then the first listed camera that votes
// background, so the occupancy and the test count (that camera's index + 1,
// or N when the midpoint is occupied) are those of the plain early-exit loop
// over all cameras.

// The ends of vertex record `rec`'s grid edge: a the ON sample, b the OFF one.
__device__ __forceinline__ void bisect_ends(uint64_t rec, const DRoi* rois, const Grid& g, float* a, float* b) {
    const int k = (int)(rec & 0x3FFFu), axis = (int)(rec >> 14 & 3u), s0 = (int)(rec >> 16 & 1u);
    const int q[3] = {(int)(rec >> 17 & 0x7FFFu), (int)(rec >> 32 & 0x7FFFu), (int)(rec >> 47 & 0x7FFFu)};
    const DRoi& r = rois[k];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float c0 = fadd(r.fo[d], fmul(fadd((float)(q[d] - 1), 0.5f), g.sf));
        const float c1 = fadd(r.fo[d], fmul(fadd((float)(q[d] - 1 + (d == axis)), 0.5f), g.sf));
        a[d] = s0 ? c0 : c1;
        b[d] = s0 ? c1 : c0;
    }
}

// The cameras that must be tested at each midpoint of the edge (a, b) (bit n:
// camera n); seen_fg: some camera votes foreground on the whole edge.
__device__ __forceinline__ uint64_t bisect_undecided(const SmemCam* sc, int ncam, const uint32_t* __restrict__ sil,
                                                     const float* a, const float* b, bool& seen_fg,
                                                     unsigned long long& reads) {
    uint64_t undecided = 0;
    seen_fg = false;
    // one compact loop over the cameras' fields in shared memory (the camera
    // is the same in every lane): 16 inlined copies of this check cost more
    // in instruction-cache misses than the loads
#pragma unroll 1
    for (int n = 0; n < ncam; ++n) {
        const bool fg = segment_all_fg(sc[n], sil, a, b, reads);
        undecided |= fg ? 0ull : 1ull << n;
        seen_fg |= fg;
    }
    return undecided;
}

// The `steps` bisection steps of the edge (a, b) with the cameras of
// `undecided` tested at each midpoint; a and b end as the last bracket.
__device__ __forceinline__ void bisect_steps(const SmemCam* sc, int ncam, const uint32_t* __restrict__ sil, int steps,
                                             bool abstain, uint64_t undecided, bool seen_fg, float* a, float* b,
                                             unsigned long long& tests, unsigned long long& reads) {
    for (int it = 0; it < steps; ++it) {
        float m[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) m[d] = fmul(fadd(a[d], b[d]), 0.5f);
        int stop = -1;
        bool voted = !abstain || seen_fg;
        for (uint64_t u = undecided; u; u &= u - 1) {
            const int n = __ffsll((long long)u) - 1;
            const SmemCam& c = sc[n];
            float xp, yp, wp;
            project(c.P, m[0], m[1], m[2], xp, yp, wp);
            const float rw = rcp_approx(wp);
            const int px = pixel_floor(xp, wp, rw, c.Wf);
            const int py = pixel_floor(yp, wp, rw, c.Hf);
            const bool in = wp > 0.0f && (unsigned)px < (unsigned)c.W && (unsigned)py < (unsigned)c.H;
            const uint32_t word =
                in ? __ldg(sil + c.bit_off + (unsigned)py * (unsigned)c.Wq + ((unsigned)px >> 5)) : 0u;
            reads += in ? 1u : 0u;
            const bool bit = (word >> (px & 31)) & 1u;
            if (abstain ? (in && !bit) : !bit) {
                stop = n;
                break;
            }
            voted |= bit;
        }
        tests += stop < 0 ? (unsigned)ncam : (unsigned)(stop + 1);
        const bool on = stop < 0 && voted;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            a[d] = on ? m[d] : a[d];
            b[d] = on ? b[d] : m[d];
        }
    }
}

// Vertices a warp sorts at once, per lane, and the bucket of the sort that
// holds every list of kSortCap - 1 or more cameras (one more bucket, the
// last, holds the window's empty places).
constexpr int kBisectWin = 4;
constexpr int kSortCap = 7;
constexpr int kSortBuckets = kSortCap + 1;
constexpr int kSortPerLane = kSortBuckets * kBisectWin / 32;   // sort counters per lane
static_assert(kSortBuckets * kBisectWin % 32 == 0 && kBisectWin <= 8, "sort counters");

// Per-warp shared memory of the sorted path (dynamic shared memory, one per
// warp of the block).
struct BisectWarpSmem {
    unsigned long long und[32 * kBisectWin];   // undecided cameras, in window order
    uint32_t id[32 * kBisectWin];              // vertex | seen_fg << 31, or ~0u for an empty place
    uint8_t perm[32 * kBisectWin];             // window places in sorted order
    int cnt[kSortBuckets * kBisectWin];        // bucket-major counts, then their exclusive prefix
};

// One vertex per thread.  Lanes whose undecided lists differ in length idle in
// the midpoint loop while the longest list is walked (about 42% of the lanes
// busy there in vertex order, on a CPU model of a volleyball-shaped frame).
// When a slot has enough vertices for every warp of the launch that can be
// resident for it (`resident_warps`) to take two windows of 32 * kv
// consecutive vertices (kv = 2 or 4), each warp takes such windows instead:
// it finds every vertex's undecided cameras, sorts the window's vertices by
// the length of that list (a counting sort in the warp's shared memory, no
// block barrier) and then bisects them 32 at a time in that order, so that a
// warp's lanes walk lists of about the same length.  Each vertex's
// arithmetic is the same in both orders; only the lane that does it changes.
template <int NC>
__global__ void __launch_bounds__(256) k_bisect(const __grid_constant__ CamSet cams, const __grid_constant__ Grid g,
                                                const __grid_constant__ Layout L, const __grid_constant__ SlotList sl,
                                                uint32_t resident_warps) {
    pdl_begin();
    __shared__ unsigned long long sh_t[32];
    __shared__ SmemCam sc[FVV_MAX_CAMS];
    extern __shared__ __align__(16) unsigned char bisect_smem[];   // BisectWarpSmem per warp
    BisectWarpSmem* wsm = reinterpret_cast<BisectWarpSmem*>(bisect_smem);
    const int ncam = NC > 0 ? NC : cams.n;
    load_smem_cams(cams, ncam, sc);
    __syncthreads();
    const bool abstain = cams.oob == FVV_OOB_ABSTAIN;
    const int slot = sl.s[blockIdx.y];
    const SlotInfo* info = slot_ptr<SlotInfo>(L, slot, L.info);
    const uint32_t nv = info->n_words ? info->n_verts : 0u;
    const DRoi* rois = slot_ptr<DRoi>(L, slot, L.rois);
    const uint32_t* __restrict__ sil = slot_ptr<uint32_t>(L, slot, L.sil);
    const uint64_t* vrec = slot_ptr<uint64_t>(L, slot, L.vrec);
    float* verts = slot_ptr<float>(L, slot, L.verts);
    unsigned long long tests = 0, reads = 0;
    const uint32_t nthreads = gridDim.x * blockDim.x;
    int kv = 1;                                    // the same in every block of the slot
    for (int k = kBisectWin; k >= 2; k >>= 1)
        if (kv == 1 && (unsigned long long)nv >= 64ull * resident_warps * (unsigned)k) kv = k;
    if (kv == 1 || g.steps == 0) {
        for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += nthreads) {
            float a[3], b[3];
            bisect_ends(vrec[i], rois, g, a, b);
            bool seen_fg = false;
            const uint64_t undecided = g.steps > 0 ? bisect_undecided(sc, ncam, sil, a, b, seen_fg, reads) : 0ull;
            bisect_steps(sc, ncam, sil, g.steps, abstain, undecided, seen_fg, a, b, tests, reads);
#pragma unroll
            for (int d = 0; d < 3; ++d) verts[3 * (size_t)i + d] = fmul(fadd(a[d], b[d]), 0.5f);
        }
    } else {
        const int lane = threadIdx.x & 31;
        BisectWarpSmem& w = wsm[threadIdx.x >> 5];
        const uint32_t win = 32u * (uint32_t)kv;
        const uint32_t nwarps = nthreads >> 5;
        // windows of the slot's vertices, taken by the warps in turn (the loop
        // condition is the same in every lane)
        for (uint32_t base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * win; base < nv;
             base += nwarps * win) {
            // (1) each lane's kv vertices: their undecided cameras
            for (int j = 0; j < kv; ++j) {
                const uint32_t i = base + (uint32_t)(j * 32 + lane);
                uint64_t und = 0;
                uint32_t id = ~0u;
                if (i < nv) {
                    float a[3], b[3];
                    bisect_ends(vrec[i], rois, g, a, b);
                    bool seen_fg;
                    und = bisect_undecided(sc, ncam, sil, a, b, seen_fg, reads);
                    id = i | (seen_fg ? 0x80000000u : 0u);
                }
                w.und[j * 32 + lane] = und;
                w.id[j * 32 + lane] = id;
            }
            // (2) counting sort of the window's places by list length
#pragma unroll
            for (int e = 0; e < kSortPerLane; ++e) w.cnt[kSortPerLane * lane + e] = 0;
            __syncwarp();
            // a place's key and its rank among the lanes of its window row with
            // that key (worked out twice, so that nothing stays in registers)
            auto place = [&](int j, int& key, int& rank) {
                const int p = j * 32 + lane;
                key = w.id[p] == ~0u ? kSortCap : min(__popcll(w.und[p]), kSortCap - 1);
                const unsigned same = __match_any_sync(kFull, key);
                rank = __popc(same & ((1u << lane) - 1u));
                return __popc(same);
            };
            for (int j = 0; j < kv; ++j) {
                int key, rank;
                const int n = place(j, key, rank);
                if (rank == 0) w.cnt[key * kBisectWin + j] = n;
            }
            __syncwarp();
            {   // exclusive prefix of the counts (bucket-major, then window row)
                int c[kSortPerLane], incl = 0;
#pragma unroll
                for (int e = 0; e < kSortPerLane; ++e) incl += c[e] = w.cnt[kSortPerLane * lane + e];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += t;
                }
#pragma unroll
                for (int e = kSortPerLane - 1; e >= 0; --e) w.cnt[kSortPerLane * lane + e] = incl -= c[e];
            }
            __syncwarp();
            for (int j = 0; j < kv; ++j) {
                int key, rank;
                place(j, key, rank);
                w.perm[w.cnt[key * kBisectWin + j] + rank] = (uint8_t)(j * 32 + lane);
            }
            __syncwarp();
            // (3) the bisections, 32 at a time in sorted order (empty places last)
            for (int j = 0; j < kv; ++j) {
                const int p = w.perm[j * 32 + lane];
                const uint32_t id = w.id[p];
                if (__all_sync(kFull, id == ~0u)) break;
                if (id != ~0u) {
                    const uint32_t i = id & 0x7FFFFFFFu;
                    float a[3], b[3];
                    bisect_ends(vrec[i], rois, g, a, b);
                    bisect_steps(sc, ncam, sil, g.steps, abstain, w.und[p], (id >> 31) != 0u, a, b, tests, reads);
#pragma unroll
                    for (int d = 0; d < 3; ++d) verts[3 * (size_t)i + d] = fmul(fadd(a[d], b[d]), 0.5f);
                }
            }
            __syncwarp();   // the window's shared memory is read before the next one writes it
        }
    }
    const unsigned long long t = block_sum<unsigned long long>(tests, sh_t);
    const unsigned long long rd = block_sum<unsigned long long>(reads, sh_t);
    if (threadIdx.x == 0 && t) atomicAdd(&slot_ptr<SlotInfo>(L, slot, L.info)->tests_bisect, t);
    if (threadIdx.x == 0 && rd) atomicAdd(&slot_ptr<SlotInfo>(L, slot, L.info)->look_bisect, rd);
}

// Sec. II-C, Eq. (2), camera c, for the edge from the occupied end a to the
// unoccupied end b: walk the pixels of the line between their pixels in
// Bresenham order from a's end and stop at the first one outside the image
// or not in the silhouette; lambda = |centre of the last silhouette pixel -
// p_a| / |p_b - p_a| in the image plane, at most 1.  Cameras that bound
// nothing (an end behind the camera, the walk reaching b's pixel, a not
// seen, p_a = p_b) give 1.  `tests` counts the pixels visited.
__device__ __forceinline__ float cam_lambda(const Cam& c, const uint32_t* __restrict__ sil, const float* a,
                                           const float* b, uint32_t& tests) {
    float xa, ya, wa, xb, yb, wb;
    project(c.P, a[0], a[1], a[2], xa, ya, wa);
    project(c.P, b[0], b[1], b[2], xb, yb, wb);
    if (!(wa > 0.0f && wb > 0.0f)) return 1.0f;
    // end pixels: floor of the exact quotient, clamped to [-1, n + 1]
    const float ra = rcp_approx(wa), rb = rcp_approx(wb);
    int x = pixel_floor(xa, wa, ra, c.Wf), y = pixel_floor(ya, wa, ra, c.Hf);
    const int x1 = pixel_floor(xb, wb, rb, c.Wf), y1 = pixel_floor(yb, wb, rb, c.Hf);
    const int dx = abs(x1 - x), dy = -abs(y1 - y);
    const int sx = x < x1 ? 1 : -1, sy = y < y1 ? 1 : -1;
    int err = dx + dy;
    bool have = false;
    int lx = 0, ly = 0;
    for (;;) {   // at most max(dx, -dy) + 1 <= 65537 pixels
        ++tests;
        const bool in = (unsigned)x < (unsigned)c.W && (unsigned)y < (unsigned)c.H;
        const uint32_t word = in ? __ldg(sil + c.bit_off + (unsigned)y * (unsigned)c.Wq + ((unsigned)x >> 5)) : 0u;
        if (!((word >> (x & 31)) & 1u)) break;
        have = true;
        lx = x;
        ly = y;
        if (x == x1 && y == y1) return 1.0f;
        const int e2 = 2 * err;
        if (e2 >= dy) {
            err += dy;
            x += sx;
        }
        if (e2 <= dx) {
            err += dx;
            y += sy;
        }
    }
    if (!have) return 1.0f;
    const float ua = __fdiv_rn(xa, wa), va = __fdiv_rn(ya, wa), ub = __fdiv_rn(xb, wb), vb = __fdiv_rn(yb, wb);
    const float ex = fsub(fadd((float)lx, 0.5f), ua), ey = fsub(fadd((float)ly, 0.5f), va);
    const float fx = fsub(ub, ua), fy = fsub(vb, va);
    const float num = __fsqrt_rn(fadd(fmul(ex, ex), fmul(ey, ey)));
    const float den = __fsqrt_rn(fadd(fmul(fx, fx), fmul(fy, fy)));
    if (!(den > 0.0f)) return 1.0f;
    const float l = __fdiv_rn(num, den);
    return l < 1.0f ? l : 1.0f;
}

// Sec. II-C, Eq. (3): lambda = the minimum of Eq. (2) over the cameras; the
// vertex is a + lambda (b - a).  One vertex per thread.
template <int NC>
__global__ void __launch_bounds__(256) k_lambda(const __grid_constant__ CamSet cams, const __grid_constant__ Grid g,
                                                const __grid_constant__ Layout L, const __grid_constant__ SlotList sl) {
    pdl_begin();
    __shared__ unsigned long long sh_t[32];
    const int slot = sl.s[blockIdx.y];
    const SlotInfo* info = slot_ptr<SlotInfo>(L, slot, L.info);
    const uint32_t nv = info->n_words ? info->n_verts : 0u;
    const DRoi* rois = slot_ptr<DRoi>(L, slot, L.rois);
    const uint32_t* __restrict__ sil = slot_ptr<uint32_t>(L, slot, L.sil);
    const uint64_t* vrec = slot_ptr<uint64_t>(L, slot, L.vrec);
    float* verts = slot_ptr<float>(L, slot, L.verts);
    uint32_t tests = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
        const uint64_t rec = vrec[i];
        const int k = (int)(rec & 0x3FFFu), axis = (int)(rec >> 14 & 3u), s0 = (int)(rec >> 16 & 1u);
        const int q[3] = {(int)(rec >> 17 & 0x7FFFu), (int)(rec >> 32 & 0x7FFFu), (int)(rec >> 47 & 0x7FFFu)};
        const DRoi& r = rois[k];
        float a[3], b[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float c0 = fadd(r.fo[d], fmul(fadd((float)(q[d] - 1), 0.5f), g.sf));
            const float c1 = fadd(r.fo[d], fmul(fadd((float)(q[d] - 1 + (d == axis)), 0.5f), g.sf));
            a[d] = s0 ? c0 : c1;
            b[d] = s0 ? c1 : c0;
        }
        float lam = 1.0f;
        if constexpr (NC > 0) {
#pragma unroll
            for (int n = 0; n < NC; ++n) {
                const float l = cam_lambda(cams.c[n], sil, a, b, tests);
                if (l < lam) lam = l;
            }
        } else {
            for (int n = 0; n < cams.n; ++n) {
                const float l = cam_lambda(cams.c[n], sil, a, b, tests);
                if (l < lam) lam = l;
            }
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) verts[3 * (size_t)i + d] = fadd(a[d], fmul(lam, fsub(b[d], a[d])));
    }
    // every pixel visited is one silhouette word read
    const unsigned long long t = block_sum<unsigned long long>(tests, sh_t);
    if (threadIdx.x == 0 && t) {
        atomicAdd(&slot_ptr<SlotInfo>(L, slot, L.info)->tests_bisect, t);
        atomicAdd(&slot_ptr<SlotInfo>(L, slot, L.info)->look_bisect, t);
    }
}

// Sec. II-C: the triangles, one per thread from the triangle records: the
// table gives the triangle's three cube edges, and each edge's vertex id is
// its word's vertex offset plus the rank of the edge among the word's
// bipolar edges (x, y, z masks in canonical order).  Also the centroid
// ((v0 + v1) + v2) / 3 of each triangle, for the depth images (Sec. II-D-1).
__global__ void __launch_bounds__(256) k_mc_triangles(const __grid_constant__ Layout L,
                                                      const __grid_constant__ SlotList sl,
                                                      const __grid_constant__ McTable mc) {
    pdl_begin();
    __shared__ uint8_t s_edges[256 * kMaxTriPerCell * 3];
    for (int i = threadIdx.x; i < 256 * kMaxTriPerCell * 3; i += blockDim.x) s_edges[i] = mc.edges[i];
    __syncthreads();
    const int slot = sl.s[blockIdx.y];
    const SlotInfo* info = slot_ptr<SlotInfo>(L, slot, L.info);
    const uint32_t nt = info->n_words ? info->n_tris : 0u;
    const DRoi* rois = slot_ptr<DRoi>(L, slot, L.rois);
    const uint32_t* emask = slot_ptr<uint32_t>(L, slot, L.emask);
    const uint32_t* vpre = slot_ptr<uint32_t>(L, slot, L.vpre);
    const uint64_t* trec = slot_ptr<uint64_t>(L, slot, L.trec);
    uint32_t* tris = slot_ptr<uint32_t>(L, slot, L.tris);
    const float* verts = slot_ptr<float>(L, slot, L.verts);
    float4* tsoup = slot_ptr<float4>(L, slot, L.tsoup);
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        const uint64_t rec = trec[t];
        const uint32_t w = (uint32_t)(rec & 0x3FFFFFFu);
        const int b = (int)(rec >> 26 & 31u), j = (int)(rec >> 31 & 15u), cs = (int)(rec >> 35 & 255u);
        const int k = (int)(rec >> 43 & 0x3FFFu);
        const uint32_t rs = (uint32_t)rois[k].nxw, ps = rs * (uint32_t)(rois[k].fdim[1] + 2);
        uint32_t id[3];
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const int e = s_edges[(cs * kMaxTriPerCell + j) * 3 + v];
            const int axis = e >> 2;
            // offsets of the edge's lower corner (same convention as the table)
            const int o0 = e & 1, o1 = (e >> 1) & 1;
            const int dx = axis == 0 ? 0 : o0;
            const int dy = axis == 1 ? 0 : (axis == 0 ? o0 : o1);
            const int dz = axis == 2 ? 0 : o1;
            const uint32_t wi = w + (uint32_t)((b + dx) >> 5) + (dy ? rs : 0u) + (dz ? ps : 0u);
            const int bb = (b + dx) & 31;
            const uint32_t lm = (1u << bb) - 1u;
            const uint32_t xm = emask[3 * (size_t)wi], ym = emask[3 * (size_t)wi + 1], zm = emask[3 * (size_t)wi + 2];
            uint32_t rank = __popc(xm & lm) + __popc(ym & lm) + __popc(zm & lm);
            if (axis >= 1) rank += (xm >> bb) & 1u;
            if (axis >= 2) rank += (ym >> bb) & 1u;
            id[v] = vpre[wi] + rank;
        }
        tris[3 * (size_t)t + 0] = id[0];
        tris[3 * (size_t)t + 1] = id[1];
        tris[3 * (size_t)t + 2] = id[2];
        // the triangle's vertices and centroid ((v0 + v1) + v2) / 3, stored
        // together for the kernels that draw it
        float v[12];
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int d = 0; d < 3; ++d) v[3 * q + d] = verts[3 * (size_t)id[q] + d];
#pragma unroll
        for (int d = 0; d < 3; ++d) v[9 + d] = __fdiv_rn(fadd(fadd(v[d], v[3 + d]), v[6 + d]), 3.0f);
        tsoup[3 * (size_t)t + 0] = make_float4(v[0], v[1], v[2], v[3]);
        tsoup[3 * (size_t)t + 1] = make_float4(v[4], v[5], v[6], v[7]);
        tsoup[3 * (size_t)t + 2] = make_float4(v[8], v[9], v[10], v[11]);
    }
}

}  // namespace

cudaError_t launch_mc_prefix(const Grid& g, const Layout& L, const SlotList& sl, const McTable& mc, int sms,
                             cudaStream_t st) {
    const int gc = grid_x(sms, sl.n, g.max_chunks, 1);
    const cudaError_t e = launch_pdl(k_mc_compact, dim3(gc, sl.n), dim3(kChunk), kSlabWords * sizeof(uint32_t), st, g,
                                     L, sl, mc);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// Resident blocks per SM of a k_bisect instantiation (index nc: its camera
// count, 0 for the generic one) with `threads` threads and `smem` bytes of
// dynamic shared memory, asked of the runtime once per shape and kept.  The
// figure is that of the GPU current at the first call; on a host that mixes
// GPU models it may not fit the others, which changes only how the
// vertices are grouped into windows, never a result.
template <class K>
int bisect_blocks_per_sm(K kernel, int nc, int threads, size_t smem) {
    static std::atomic<int> known[FVV_MAX_CAMS + 1][9];   // [nc][threads / 32]; 0: not asked yet
    std::atomic<int>& slot = known[nc][threads / 32];
    int n = slot.load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) {
            (void)cudaGetLastError();
            n = 1;
        }
        slot.store(n, std::memory_order_relaxed);
    }
    return n;
}

cudaError_t launch_bisect(const CamSet& cams, const Grid& g, const Layout& L, const SlotList& sl, int sms,
                          const Tuning& tu, cudaStream_t st) {
    const int th = tu.threads[FVV_TUNE_BISECT];
    const int gv = tuned_grid(tu, FVV_TUNE_BISECT, sms, sl.n, g.max_verts);
    if (g.rule == FVV_SURFACE_LAMBDA) {
#define FVV_LAUNCH(NC) launch_pdl(k_lambda<NC>, dim3(gv, sl.n), dim3(th), 0, st, cams, g, L, sl)
        FVV_DISPATCH_NC(cams.n, FVV_LAUNCH)
#undef FVV_LAUNCH
    } else {
        // the warps that can be resident for each slot: those launched, or the
        // slot's share of what the GPU holds if that is fewer
        const size_t smem = (size_t)(th / 32) * sizeof(BisectWarpSmem);
        int per_sm = 0;
#define FVV_OCC(NC) per_sm = bisect_blocks_per_sm(k_bisect<NC>, NC, th, smem)
        FVV_DISPATCH_NC(cams.n, FVV_OCC)
#undef FVV_OCC
        const long long launched = (long long)gv * (th / 32);
        const long long fit = (long long)std::max(per_sm, 1) * sms * (th / 32) / std::max(sl.n, 1);
        const uint32_t resident = (uint32_t)std::max(1LL, std::min(launched, fit));
#define FVV_LAUNCH(NC) launch_pdl(k_bisect<NC>, dim3(gv, sl.n), dim3(th), smem, st, cams, g, L, sl, resident)
        FVV_DISPATCH_NC(cams.n, FVV_LAUNCH)
#undef FVV_LAUNCH
    }
    return cudaGetLastError();
}

cudaError_t launch_mc_triangles(const Grid& g, const Layout& L, const SlotList& sl, const McTable& mc, int sms,
                                const Tuning& tu, cudaStream_t st) {
    const int gw = tuned_grid(tu, FVV_TUNE_TRIANGLES, sms, sl.n, g.max_tris);
    launch_pdl(k_mc_triangles, dim3(gw, sl.n), dim3(tu.threads[FVV_TUNE_TRIANGLES]), 0, st, L, sl, mc);
    return cudaGetLastError();
}

}  // namespace fvv
