/*
 * fvv.h -- C ABI of the GB300 (sm_103a) coarse-to-fine visual-hull library.
 *
 * The library implements steps (B)-(D) of "A Fast Free-viewpoint Video
 * Synthesis Algorithm for Sports Scenes" (arXiv 1903.11785) for calibrated,
 * static cameras (Sec. II-A) and per-frame binary silhouettes:
 *
 *   B-1 coarse ("sparse") volumetric visual hull            Sec. II-B-1
 *   B-2 26-connected CCL, minimum 3D box, noise filter       Sec. II-B-2, Eq. (1)
 *   B-3 fine ("dense") hull inside each 3D ROI               Sec. II-B-3
 *   C   exact edge/hull intersection + marching cubes        Sec. II-C, Eqs. (2)-(3)
 *   D-1 per-camera depth image                               Sec. II-D-1, Eq. (4)
 *   D-2 visibility by T_v and colour from the nearest
 *       unoccluded camera (per vertex)                       Sec. II-D-2, II-E
 *
 * Conventions.  World coordinates in metres.  Camera n projects a world point
 * X through its row-major 3x4 matrix P_n: (x', y', w') = P_n (X, 1); the pixel
 * is (floor(x'/w'), floor(y'/w')), pixel (px, py) covering [px, px+1) x
 * [py, py+1); images are row-major, W pixels per row.  Voxel i of a grid with
 * origin o and step s is tested at its centre o + (i + 1/2) s.  Linear voxel
 * index L = (z*ny + y)*nx + x (x fastest).  All floating point on the device
 * is IEEE binary32, round to nearest, in a fixed order, so results are
 * reproducible bit for bit; each row of the projection is the three fused
 * multiply-adds ((p3 + p2 Z) + p1 Y) + p0 X, every other product and sum is
 * rounded on its own.
 *
 * Memory.  As the paper does (Sec. III-B), all device memory a rig needs is
 * taken once, at fvv_create_rig, as one arena: either a buffer the caller
 * passes (for example a torch tensor) or one the library allocates.  It never
 * grows.  A rig has max_slots frame slots; a slot holds one frame's packed
 * silhouettes, grids, mesh, depth images and colours.  Results of a slot stay
 * valid until that slot is uploaded to or reconstructed again.
 *
 * Streams.  Every call that takes `void* stream` (a cudaStream_t; NULL is the
 * legacy default stream) only enqueues work on it and returns (host inputs in
 * pageable memory are the exception: CUDA copies those before returning).
 * Everything a call touches on the device belongs to the slots it names, so
 * calls on disjoint slots may run concurrently on different streams; calls
 * on the same slot must be ordered (one stream, or the caller's events).
 * fvv_get_counts synchronises the stream it is given.
 *
 * Errors.  Every call returns an fvv_status and never throws.  A NULL or
 * inconsistent argument gives FVV_ERR_INVALID_ARG; a failed CUDA call gives
 * FVV_ERR_CUDA; work that exceeds a capacity chosen at creation is detected
 * on the device, skipped without writing out of bounds, and reported by
 * fvv_get_counts as FVV_ERR_CAPACITY with the overflowing capacity in
 * fvv_counts.flags.  fvv_last_error gives a message for the last failure.
 *
 * Thread safety.  A rig may be used by one host thread at a time.
 */
#ifndef FVV_H
#define FVV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FVV_VERSION 1
#define FVV_MAX_CAMS 64      /* cameras per rig                              */
#define FVV_MAX_BATCH 256    /* slots per fvv_reconstruct / fvv_colour call   */

typedef struct fvv_rig fvv_rig;

typedef enum {
    FVV_OK = 0,
    FVV_ERR_INVALID_ARG = 1,
    FVV_ERR_OUT_OF_MEMORY = 2,
    FVV_ERR_CAPACITY = 3,
    FVV_ERR_NOT_READY = 4,
    FVV_ERR_TIMEOUT = 5,
    FVV_ERR_CUDA = 6
} fvv_status;

/* What a camera whose image does not contain a point's projection (or that
 * has the point behind it) does.  STRICT: it votes background, the literal
 * reading of Sec. II-B, where a voxel projecting outside a silhouette is
 * empty.
 * ABSTAIN: it does not vote; a point no camera votes for is unoccupied. */
enum { FVV_OOB_STRICT = 0, FVV_OOB_ABSTAIN = 1 };

/* How a surface vertex is placed on a grid edge between an occupied sample
 * a and an unoccupied one b (Sec. II-C).
 * BISECT: bisect_steps times m = (a+b)/2, a = m if m is occupied else b = m;
 *   the vertex is the final midpoint (0 steps: the edge midpoint, the
 *   isovalue 0.5 of conventional marching cubes).
 * LAMBDA: the paper's form, Eqs. (2)-(3).  Per camera the pixels of the line
 *   from the pixel of a to the pixel of b (both clamped to [-1, W+1] x
 *   [-1, H+1]) are walked in Bresenham order from a's end; P_n is the last
 *   silhouette pixel before the first that is outside the image or not in
 *   the silhouette, lambda_n = |c(P_n) - p_a| / |p_b - p_a| in the image
 *   plane (c = pixel centre, p = x'/w', y'/w' in binary32), at most 1; a
 *   camera with an end behind it, whose walk reaches b's pixel, that does
 *   not see a (ABSTAIN only), or with p_a = p_b gives 1.  lambda is the
 *   minimum over the cameras and the vertex is a + lambda (b - a).  Every
 *   pixel visited counts as one test (fvv_counts.tests_bisect). */
enum { FVV_SURFACE_BISECT = 0, FVV_SURFACE_LAMBDA = 1 };

/* Input images in page-locked host memory that the device can address (for
 * example a pinned torch tensor), read in place by the kernels over the host
 * link, with no staging copy: a value of masks_on_device / rgb_on_device.
 * Both ends of every image must lie in such memory
 * (cudaPointerGetAttributes), else FVV_ERR_INVALID_ARG with nothing
 * launched; the memory must stay valid until the work has run. */
#define FVV_MAPPED_HOST 2
#define FVV_RGB_MAPPED_HOST FVV_MAPPED_HOST

/* Bits of fvv_counts.flags: which capacity a reconstruction exceeded. */
enum {
    FVV_FLAG_ROOTS = 1u << 0,      /* raw 26-connected components > max_components */
    FVV_FLAG_ROIS = 1u << 1,       /* kept components > max_rois                   */
    FVV_FLAG_FINE = 1u << 2,       /* fine grid words > max_fine_words, or a ROI
                                      side longer than 32765 fine voxels          */
    FVV_FLAG_VERTS = 1u << 3,      /* vertices > max_verts                         */
    FVV_FLAG_TRIS = 1u << 4,       /* triangles > max_tris                         */
    FVV_FLAG_LOOP = 1u << 5        /* an iteration bound of union-find, or of a
                                      * bounded wait in the compaction, was hit     */
};

/* The cameras (Sec. II-A: calibrated in advance, static).  All arrays are
 * host memory, read during fvv_create_rig only. */
typedef struct {
    int n_cams;            /* 1..FVV_MAX_CAMS                                 */
    const float *P;        /* n_cams x 12: row-major 3x4 world -> pixel       */
    const float *centre;   /* n_cams x 3: camera centres (depth, colour rank) */
    const int *width;      /* n_cams: image width in pixels, 1..65535         */
    const int *height;     /* n_cams: image height in pixels, 1..65535        */
    int max_slots;         /* frames that can be held at once, >= 1           */
    int host_staging;      /* 1: reserve per-slot buffers so masks and RGB can
                              be passed in host memory (copied); 2: masks
                              only (RGB then comes from the device or is read
                              in place, FVV_RGB_MAPPED_HOST); 0: none */
} fvv_rig_desc;

/* Reconstruction parameters.  The capacities are per slot; 0 picks a default
 * derived from the grid (see fvv_query_arena). */
typedef struct {
    float vol_min[3], vol_max[3]; /* the pre-defined 3D volume, metres        */
    float coarse_m;        /* coarse voxel step (Sec. II-B-1), metres          */
    float fine_m;          /* fine voxel step (Sec. II-B-3), metres            */
    int bisect_steps;      /* bisections per bipolar edge, 0..30 (0 = midpoint) */
    int t_np, t_nb;        /* Eq. (1): keep a component iff t_np <= voxels <= t_nb */
    float t_v;             /* Sec. II-D-2 occlusion threshold, metres          */
    int oob_policy;        /* FVV_OOB_STRICT or FVV_OOB_ABSTAIN                */
    int max_components;    /* raw components per frame (<= 8192)              */
    int max_rois;          /* kept components per frame (<= 4096)             */
    long long max_fine_words;  /* 32-sample words of all padded fine grids,
                                  <= 2^26                                    */
    long long max_verts;   /* mesh vertices per frame                          */
    long long max_tris;    /* mesh triangles per frame                         */
    int surface_rule;      /* FVV_SURFACE_BISECT or FVV_SURFACE_LAMBDA         */
} fvv_recon_params;

/* One kept object and its 3D ROI (Sec. II-B-2, II-B-3). */
typedef struct {
    int cmin[3], cmax[3];  /* inclusive coarse index box of the component     */
    int gmin[3], gmax[3];  /* the box grown by one coarse voxel, clamped      */
    int fdim[3];           /* fine voxels per axis covering the grown box     */
    float forigin[3];      /* world position of the grown box's lower corner  */
    int count;             /* coarse voxels in the component                  */
    int label;             /* canonical label, 1..n_rois                      */
    long long vert_offset, n_verts;  /* this object's vertices in the slot's mesh  */
    long long tri_offset, n_tris;    /* this object's triangles in the slot's mesh */
} fvv_roi;

typedef struct {
    unsigned int flags;    /* FVV_FLAG_* capacities exceeded (0 = none)        */
    int n_components;      /* 26-connected components before the filter       */
    int n_rois;            /* components kept                                 */
    int pad_;
    long long n_coarse_on; /* occupied coarse voxels                          */
    long long n_fine_words;
    long long n_verts, n_tris;
    long long tests_coarse, tests_fine, tests_bisect; /* camera tests, with the
                              per-point early exit at the first background vote */
    long long lookups_fine, lookups_bisect; /* silhouette words the fine-hull and
                              surface kernels actually read: they settle most
                              tests for a whole tile or grid edge at once (the
                              coarse hull reads one word per test) */
} fvv_counts;

/* Per-slot debug views for tests (fvv_get_debug). */
enum {
    FVV_DEBUG_SIL_BITS = 0,   /* uint32: per camera H rows of ceil(W/32) words  */
    FVV_DEBUG_COARSE_BITS = 1,/* uint32: nz*ny rows of ceil(nx/32) words        */
    FVV_DEBUG_LABELS = 2,     /* int32 nz*ny*nx canonical labels (0 = none)     */
    FVV_DEBUG_FINE_BITS = 3,  /* uint32: per ROI, (fz+2)*(fy+2) rows of
                                 ceil((fx+2)/32) words of the padded fine grid  */
    FVV_DEBUG_DEPTH = 4       /* float32: per camera H*W depth, +inf = empty     */
};

/* Bytes of device memory fvv_create_rig needs for these arguments (after the
 * defaults for zero capacities are applied): the memory that, as in
 * Sec. III-B, is taken once at start-up.  desc, params and bytes are host
 * pointers; NULL or an invalid argument gives FVV_ERR_INVALID_ARG. */
fvv_status fvv_query_arena(const fvv_rig_desc *desc, const fvv_recon_params *params,
                           size_t *bytes);

/* Create a rig for cameras calibrated in advance and static (Sec. II-A), with
 * all device memory taken at once (Sec. III-B): validate the cameras and
 * parameters, lay out the arena and build the marching-cubes table
 * (Sec. II-C).  `arena` is a device buffer of at least
 * fvv_query_arena bytes, aligned to 256 bytes, owned by the caller and kept
 * alive until fvv_destroy_rig; or NULL, in which case the library allocates
 * (and later frees) it.  On success *out is the new rig. */
fvv_status fvv_create_rig(const fvv_rig_desc *desc, const fvv_recon_params *params,
                          void *arena, size_t arena_bytes, fvv_rig **out);

/* Free the rig (and the arena if the library allocated it): the end of the
 * start-up allocation of Sec. III-B. Synchronises the device first.  NULL is
 * accepted. */
fvv_status fvv_destroy_rig(fvv_rig *rig);

/* Pack one frame's silhouettes into slot `slot` (step a0): masks[n] points
 * to camera n's H x W uint8 image, nonzero = foreground (Sec. II-A).  With
 * masks_on_device = 1 the pointers are device memory that must stay valid
 * until the work on `stream` has run; with 0 they are host memory (pinned
 * memory makes the copy asynchronous; pageable memory is copied before this
 * call returns) and the rig needs host_staging; with FVV_MAPPED_HOST the
 * packing kernel reads them in place from mapped page-locked host memory. */
fvv_status fvv_upload_silhouettes(fvv_rig *rig, int slot, const uint8_t *const *masks,
                                  int masks_on_device, void *stream);

/* fvv_upload_silhouettes (the silhouettes of Sec. II-A, step a0) for several
 * frames at once: frame j's masks (masks[j*n_cams + n] for camera n, memory
 * as for fvv_upload_silhouettes) go into slots[j], n_slots distinct slots
 * (1..256).  One packing launch
 * takes up to min(512, 2048 / n_cams) frames, so a batch costs a few
 * launches instead of one per frame.  Nothing is packed if an argument is
 * rejected. */
fvv_status fvv_upload_silhouettes_batch(fvv_rig *rig, const int *slots, int n_slots,
                                        const uint8_t *const *masks, int masks_on_device,
                                        void *stream);

/* Reconstruct the frames in `slots` (n_slots distinct slots, each uploaded):
 * coarse hull (Sec. II-B-1), 26-connected components, the filter of Eq. (1)
 * and the 3D ROIs (Sec. II-B-2), fine hull (Sec. II-B-3), marching-cubes
 * mesh with each vertex placed by the surface rule (Sec. II-C, Eqs. (2)-(3))
 * and per-camera depth images (Sec. II-D-1, Eq. (4)): steps a1..a9.  All
 * slots are processed by the same launches.  No host synchronisation
 * happens inside.  A NULL rig or slot list, a slot out of range or listed
 * twice gives FVV_ERR_INVALID_ARG, a slot not uploaded FVV_ERR_NOT_READY,
 * both with nothing launched. */
fvv_status fvv_reconstruct(fvv_rig *rig, const int *slots, int n_slots, void *stream);

/* Colour the meshes of `slots` for a virtual viewpoint (step a10, Sec. II-D-2
 * and II-E): cameras are ranked by distance to viewpoints[3*i..3*i+2]; each
 * vertex takes the colour of the first camera in that order that has it in
 * front, inside its image and not occluded (|v - C| - depth <= t_v), else
 * (0,0,0) and camera -1.  rgb[i*n_cams + n] is camera n's H x W x 3 uint8
 * image for slots[i]; device or host memory as for fvv_upload_silhouettes. */
fvv_status fvv_colour(fvv_rig *rig, const int *slots, int n_slots, const uint8_t *const *rgb,
                      int rgb_on_device, const float *viewpoints, void *stream);

/* Synchronise `stream` and read slot's counts; returns FVV_ERR_CAPACITY if a
 * capacity was exceeded (counts->flags says which), else FVV_OK.  The counts
 * are those the paper's pipeline produces and reports: components before and
 * after the noise filter of Eq. (1) (Sec. II-B-2), the occupied coarse
 * voxels of the sparse hull (Sec. II-B-1; the paper counts them for its
 * volleyball scene in Sec. II-B), the mesh's vertices and triangles
 * (Sec. II-C), and the camera tests of the hulls and the surface step, the
 * work behind Table II's stage times. */
fvv_status fvv_get_counts(fvv_rig *rig, int slot, fvv_counts *counts, void *stream);

/* The outputs of Sec. II-B to II-D for a slot: the objects with their 3D ROI
 * (Sec. II-B-2, II-B-3), the mesh of each (Sec. II-C: vertices on the hull
 * boundary, triangles of the marching-cubes table) and each vertex's colour
 * and source camera (Sec. II-D-2, II-E), which is what the paper sends to
 * the client for rendering.
 * Copy slot's results into caller-owned buffers (any may be NULL):
 * rois[n_rois], verts[n_verts*3] float, tris[n_tris*3] uint32 (indices into
 * the slot's vertices), rgb[n_verts*3] uint8, cam[n_verts] int32.  Sizes come
 * from fvv_get_counts.  dst_on_device says whether the buffers are device
 * memory.  The copies are enqueued on `stream` (ROIs are read synchronously). */
fvv_status fvv_get_results(fvv_rig *rig, int slot, fvv_roi *rois, float *verts, uint32_t *tris,
                           uint8_t *rgb, int32_t *cam, int dst_on_device, void *stream);

/* Destination of one slot's results for fvv_get_results_batch: caller-owned
 * buffers (any may be NULL; sized from an earlier fvv_get_counts of a
 * reconstruction of the same frame, or generously), and the slot's counts,
 * written by the call. */
typedef struct {
    fvv_counts counts;     /* out                                             */
    fvv_roi *rois;         /* must be NULL (ROIs: fvv_get_results)            */
    float *verts;          /* n_verts*3 float                                 */
    uint32_t *tris;        /* n_tris*3 uint32                                 */
    uint8_t *rgb;          /* n_verts*3 uint8                                 */
    int32_t *cam;          /* n_verts int32                                   */
} fvv_results_dst;

/* The outputs of Sec. II-C to II-E (as fvv_get_results returns them) for
 * several slots with one wait: the counts of all n_slots slots (1..256) are
 * read together, with one synchronisation of `stream`, then the copies of
 * every slot's vertices, triangles, colours and cameras into dst[i]'s
 * buffers are enqueued on `stream` (wait for the stream before reading
 * them).  A slot whose reconstruction exceeded a capacity gets its counts
 * but no copies, and the call returns FVV_ERR_CAPACITY; a slot not
 * reconstructed gives FVV_ERR_NOT_READY and a bad argument
 * FVV_ERR_INVALID_ARG, both with nothing copied.  For callers that read many
 * frames back (one wait per group of frames instead of one per frame). */
fvv_status fvv_get_results_batch(fvv_rig *rig, const int *slots, int n_slots, fvv_results_dst *dst,
                                 int dst_on_device, void *stream);

/* Size in bytes of a debug view of slot, an intermediate result of
 * Sec. II-A to II-D-1 (fvv_get_counts must have been called after the
 * reconstruction for FINE_BITS). */
fvv_status fvv_debug_bytes(fvv_rig *rig, int slot, int what, size_t *bytes);

/* Write a debug view of slot (silhouette bits of Sec. II-A, coarse occupancy
 * of Sec. II-B-1, labels of Sec. II-B-2, fine grids of Sec. II-B-3, depth
 * images of Sec. II-D-1) into device buffer dst (bytes from
 * fvv_debug_bytes), enqueued on `stream`. */
fvv_status fvv_get_debug(fvv_rig *rig, int slot, int what, void *dst, size_t bytes, void *stream);

/* Test hook for the projection of Sec. II-B-1: for camera `cam`, the pixel
 * (px[i], py[i]) = (floor(x'/w'), floor(y'/w')) that world point
 * pts[3i..3i+2] falls in, exactly as the hull tests compute it, or (-1, -1)
 * if w' <= 0 or the pixel is outside the image.  pts, px and py are device
 * arrays of n entries; the work is enqueued on `stream`. */
fvv_status fvv_debug_pixels(fvv_rig *rig, int cam, long long n, const float *pts, int32_t *px, int32_t *py,
                            void *stream);

/* Test hook for the labelling of Sec. II-B-2 on a grid that is given rather
 * than carved, so that the parity tests can feed it random and adversarial
 * occupancy (percolating random grids, long chains, spirals) that no set of
 * silhouettes produces.  coarse_bits is a device array in the
 * FVV_DEBUG_COARSE_BITS layout of the rig's grid (nz*ny rows of ceil(nx/32)
 * uint32, bit x%32 of word x/32; bits past nx are ignored).  The call copies
 * it into slot's coarse grid, starts the union-find forest as the coarse hull
 * does, and runs the same labelling, box, Eq. (1) filter and ROI kernels as
 * fvv_reconstruct.  Afterwards fvv_get_counts (components, ROIs, occupied
 * voxels, flags), fvv_get_results (rois only) and FVV_DEBUG_LABELS read the
 * outcome; the slot's fine grids, mesh and depth images are not computed
 * (zero vertices and triangles) and its silhouettes are left as they were.
 * Work is enqueued on `stream`; a NULL rig or grid, or a bad slot, gives
 * FVV_ERR_INVALID_ARG with nothing launched. */
fvv_status fvv_debug_label_coarse(fvv_rig *rig, int slot, const uint32_t *coarse_bits, void *stream);

/* Allocation-free labelling (the paper has no counterpart; it is a service of
 * this library).  For callers that cannot call cudaMalloc: code that runs
 * inside a host framework which owns all device memory, or real-time loops
 * in which an allocation (which may synchronise the device) is not allowed.
 * It labels the 26-connected components of a coarse occupancy bitset,
 * numbered by their smallest linear index, and applies the size filter of
 * Eq. (1) (keep iff t_np <= voxels <= t_nb), exactly as fvv_reconstruct does
 * for FVV_DEBUG_LABELS.
 *   coarse_bits  device, nz*ny rows of ceil(nx/32) uint32, bit x%32 of word
 *                x/32 (the FVV_DEBUG_COARSE_BITS layout); bits past nx ignored
 *   labels       device, nz*ny*nx int32 written in full: canonical label of
 *                every voxel, 0 for empty voxels and removed components
 *   counts       device int32[3]: components before the filter, components
 *                kept, FVV_FLAG_* bits (ROOTS if more than 8192 components,
 *                in which case every label is 0; LOOP if a union-find bound
 *                was hit)
 * Work is enqueued on `stream`; nothing is allocated.  Its scratch is one
 * static device array inside the library (about 32.4 MB, held on every GPU
 * that loads the library until the process exits), which limits the grid to
 * nx*ny*nz <= 8,388,608 voxels: larger grids, non-positive sizes or NULL
 * pointers give FVV_ERR_INVALID_ARG without launching anything.  The first
 * call on each device looks up the array's device address with that device
 * current, so make that first call before any stream capture.  All calls
 * share the array and each clears what it needs: calls whose work overlaps
 * on the GPU (different streams or host threads without ordering) race and
 * give wrong labels. */
fvv_status fvv_label_components_noalloc(const uint32_t *coarse_bits, int nx, int ny, int nz, int t_np, int t_nb,
                                        int32_t *labels, int32_t *counts, void *stream);

/* Per-stage device time, the buckets of the paper's Table II (plus packing,
 * the bisection kernel and colour on their own). */
enum {
    FVV_STAGE_PACK = 0,      /* step a0, silhouette packing (fvv_upload_silhouettes) */
    FVV_STAGE_COARSE = 1,    /* B-1 coarse hull                                       */
    FVV_STAGE_CCL = 2,       /* B-2 labelling, boxes, Eq. (1) filter, ROIs             */
    FVV_STAGE_FINE = 3,      /* B-3 fine hull                                          */
    FVV_STAGE_MC = 4,        /* C   marching cubes: edges, prefix sums, triangles      */
    FVV_STAGE_BISECT = 5,    /* C   exact intersection by bisection                    */
    FVV_STAGE_DEPTH = 6,     /* D-1 depth images                                       */
    FVV_STAGE_COLOUR = 7,    /* D-2 visibility and colour (fvv_colour)                 */
    FVV_N_STAGES = 8
};

/* Step E (Sec. II-E): render a novel view of a reconstructed slot's coloured
 * mesh into a headless image, from a virtual camera with row-major 3x4
 * matrix P (world -> pixel, as for the rig's cameras) and centre `centre`,
 * width x height pixels.  Visibility: each pixel keeps, among the mesh
 * triangles whose projection covers its centre (the coverage test of the
 * depth images), the one with the smallest squared distance from its
 * centroid to `centre`, ties to the lower triangle index.  Colour: that
 * triangle's centroid takes the colour rule of fvv_colour with the capture
 * cameras ranked for the viewpoint `centre` -- the nearest capture camera
 * that sees the point unoccluded (|X - C| - depth <= t_v), else the next
 * ones -- so the capture camera is chosen per pixel.
 *   rgb      n_cams capture images (H x W x 3 uint8 each), located as
 *            rgb_on_device says (see fvv_colour; with 0 they are copied into
 *            the slot's staging, which this call then overwrites);
 *   P, centre  host arrays of 12 and 3 finite floats;
 *   key      device, width*height uint64, written: per pixel (squared
 *            distance as float bits) << 32 | triangle index within the slot's
 *            mesh, all ones where no triangle covers the pixel;
 *   out_rgb  device, width*height*3 uint8, written ((0,0,0) where empty or
 *            no camera sees the point);
 *   out_cam  device, width*height int32, or NULL: the capture camera per
 *            pixel, -1 where none.
 * The slot must hold a reconstruction (FVV_ERR_NOT_READY otherwise); its
 * depth images and mesh are read, not changed.  All buffers are the caller's;
 * work is enqueued on `stream`. */
fvv_status fvv_render_view(fvv_rig *rig, int slot, const uint8_t *const *rgb, int rgb_on_device, const float *P,
                           const float *centre, int width, int height, uint64_t *key, uint8_t *out_rgb,
                           int32_t *out_cam, void *stream);

/* Switch per-stage timing (the stage buckets of Table II) on (1) or off
 * (0).  When on, each call records CUDA events around its stages on its
 * stream (no synchronisation). */
fvv_status fvv_set_timing(fvv_rig *rig, int enable);

/* Wait for the recorded events and return, per stage (Table II's buckets),
 * the summed device milliseconds (ms[FVV_N_STAGES]) and the number of timed
 * intervals (calls[FVV_N_STAGES], may be NULL) since the previous
 * fvv_get_timing or fvv_set_timing; then start a new accumulation. */
fvv_status fvv_get_timing(fvv_rig *rig, float *ms, int *calls);

/* Launch shapes of the five heaviest kernels, chosen per rig by fvv_autotune
 * (results never depend on them).  Batching, autotuning and graphs have no
 * counterpart in the paper, which runs one frame at a time with fixed launch
 * shapes; they are services of this library. */
enum {
    FVV_TUNE_COARSE = 0,     /* coarse hull                     */
    FVV_TUNE_FINE = 1,       /* fine hull                       */
    FVV_TUNE_BISECT = 2,     /* bisection                       */
    FVV_TUNE_ZBUFFER = 3,    /* depth images                    */
    FVV_TUNE_TRIANGLES = 4,  /* marching-cubes triangles        */
    FVV_N_TUNE = 5
};

/* Fine-hull tile shapes (x by y by z samples) the autotuner chooses among; a
 * tile is classified per camera once and tested 4 x 2 x 4 samples at a time. */
enum { FVV_TILE_4x4x8 = 0, FVV_TILE_4x4x4 = 1, FVV_TILE_4x8x8 = 2, FVV_N_TILES = 3 };

/* Ints of a tuning configuration: threads per block of each FVV_TUNE_*
 * kernel, then its resident blocks per SM, then the fine-hull tile shape
 * (FVV_TILE_*), then the cameras one z-buffer block serves (1, 2 or 4; each
 * triangle record is read once per that many cameras). */
#define FVV_TUNE_INTS (2 * FVV_N_TUNE + 2)

/* Autotuning (no counterpart in the paper).
 * Time candidate launch shapes (threads per block 64/128/256 x resident
 * blocks per SM 2/4/8/16/32/64) of each tunable kernel, for the fine hull
 * each tile shape too and for the z-buffer each number of cameras per block
 * (1, 2, 4), on the given slots, which must hold reconstructed
 * frames; keep the fastest, then reconstruct the slots once more with it so
 * that their results and counts are those of one reconstruction.  Results
 * never depend on the choice.  Synchronises `stream`.  config (may be NULL)
 * receives FVV_TUNE_INTS ints. */
fvv_status fvv_autotune(fvv_rig *rig, const int *slots, int n_slots, void *stream, int *config);

/* Read or set the configuration (no counterpart in the paper):
 * FVV_TUNE_INTS ints as for fvv_autotune; threads must be 32..256 in steps
 * of 32, blocks per SM 1..64, the tile shape one of FVV_TILE_*, the z-buffer
 * cameras per block 1, 2 or 4 (else FVV_ERR_INVALID_ARG). */
fvv_status fvv_get_tuning(fvv_rig *rig, int *config);
fvv_status fvv_set_tuning(fvv_rig *rig, const int *config);

/* CUDA graphs (no counterpart in the paper).
 * With graphs on (1), fvv_reconstruct records its launch sequence for each
 * distinct slot list into a CUDA graph the first time it sees the list and
 * replays that graph afterwards (up to 16 lists are kept).  Graphs are not
 * used on the legacy default stream (NULL), nor while per-stage timing is on;
 * a change of tuning drops them. */
fvv_status fvv_set_graphs(fvv_rig *rig, int enable);

/* The marching-cubes table (Sec. II-C) the library built from its face
 * rule: ntri[256] triangle counts and edges[256*12*3] cube-edge numbers
 * (corner c = dx + 2dy + 4dz; cube edge e has axis e/4 and lower corner with
 * the other two coordinates (e%4 & 1, e%4 >> 1) in axis order).  Host
 * memory; no GPU needed. */
fvv_status fvv_mc_table(uint8_t *ntri, uint8_t *edges);

/* L2 micro-benchmark (no counterpart in the paper): the memory side of the
 * roofline of the hull tests, each of which gathers one 32-bit silhouette
 * word.  Launches `blocks` x `threads` threads on `stream`; every load is
 * ld.global.cg (L2, not L1).
 *   mode 0: coalesced read of the `bytes` at buf (16-byte aligned, a multiple
 *           of 16), `reps` times over: bytes*reps bytes read;
 *   mode 1: `reps` random 32-bit gathers per thread from the bytes/4 words at
 *           buf (a power of two): blocks*threads*reps gathers.
 * buf and out are device pointers; out receives blocks*threads uint32 (an
 * XOR of what each thread read, so that the loads are not dropped).  Bad
 * arguments give FVV_ERR_INVALID_ARG with nothing launched.  Time it with
 * events on `stream`. */
fvv_status fvv_probe_l2(int mode, const void *buf, size_t bytes, int reps, uint32_t *out, int blocks, int threads,
                        void *stream);

/* FP32 micro-benchmark (no counterpart in the paper): the arithmetic ceiling
 * of the hull and depth kernels, whose camera tests and triangle set-ups are
 * chains of binary32 fused multiply-adds on the plain ALUs.  Launches
 * `blocks` x `threads` threads on `stream`; each runs 16 independent chains
 * x = fma(x, a, b) of `reps` steps (x starting at (thread + k) mod 8 for
 * chain k) and writes the sum of its chains (added in chain order, binary32)
 * to out[thread]: blocks*threads*reps*16 fused multiply-adds, two
 * floating-point operations each.  out is a device pointer of
 * blocks*threads floats.  Bad arguments give FVV_ERR_INVALID_ARG with
 * nothing launched.  Time it with events on `stream`. */
fvv_status fvv_probe_fma(int reps, float a, float b, float *out, int blocks, int threads, void *stream);

/* Error reporting (no counterpart in the paper).
 * Message of the last failure on rig (or of the last failed create if rig is
 * NULL).  The string stays valid until the next call on the rig. */
const char *fvv_last_error(const fvv_rig *rig);

/* Static name of a status code (no counterpart in the paper). */
const char *fvv_status_string(fvv_status status);

/* FVV_VERSION of the library (no counterpart in the paper). */
int fvv_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FVV_H */
