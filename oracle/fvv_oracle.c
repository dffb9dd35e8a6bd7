/*
 * fvv_oracle.c -- plain, slow, single-threaded CPU oracle of the coarse-to-fine
 * visual-hull path of "A Fast Free-viewpoint Video Synthesis Algorithm for
 * Sports Scenes" (arXiv 1903.11785).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: it is used by the tests, by the smoke check and by the CPU
 * baseline leg of the benchmark.  It shares no code, header, table or helper
 * with the CUDA library; the MC polygons in particular are derived per cell
 * from the face rule below, with no case table.
 *
 * The file is compiled twice: -DORC_REAL=float is the parity target (all
 * floating point is IEEE binary32 with round-to-nearest, evaluated in the
 * order written) and -DORC_REAL=double gives the flip count.  Build with
 * -ffp-contract=off so that only the explicit fma() calls are fused.
 *
 * Steps, in the paper's order:
 *   Sec. II-B-1  coarse ("sparse") visual hull        orc_coarse
 *   Sec. II-B-2  26-connected CCL, minimum 3D box,
 *                noise filter of Eq. (1)               orc_ccl_bfs, orc_filter
 *   Sec. II-B-3  fine ("dense") hull inside each ROI   orc_fine
 *   Sec. II-C    exact edge/hull intersection and
 *                marching cubes                        orc_mesh_roi
 *   Sec. II-D-1  depth image per camera, Eq. (4)       orc_depth
 *   Sec. II-D-2/E visibility by T_v and colour from the
 *                nearest visible camera               orc_colour
 *   Sec. II-E    a novel view of the coloured mesh    orc_render_view
 *
 * Readings of the paper used here (each is also listed with the design notes):
 *  - A voxel is tested at its centre c = o + (i + 1/2) s (Sec. II-B-1 says
 *    the voxel is projected; the paper does not say which point).
 *  - The projection (x', y', w') = P (X, Y, Z, 1) is evaluated per row as
 *    ((p_3 + p_2 Z) + p_1 Y) + p_0 X, three fused multiply-adds (the paper
 *    fixes no arithmetic; this is the cheapest fixed order).
 *  - A camera votes "foreground" iff w' > 0, the pixel (floor(x'/w'),
 *    floor(y'/w')) -- the floor of the exact quotient of the homogeneous
 *    coordinates as computed -- is inside the image and its silhouette bit
 *    is set.  STRICT: a projection
 *    outside the image votes background (Sec. II-B: a voxel outside the
 *    silhouettes is unoccupied).  ABSTAIN: such a camera does not vote, and a
 *    point no camera votes for is unoccupied.
 *  - Eq. (1) is printed with its inequality reversed; the prose after it is
 *    followed: a component is kept iff T_np <= count <= T_nb.
 *  - The ROI is the component's inclusive box grown by one coarse voxel per
 *    side and clamped to the grid; the fine grid covers it in whole fine
 *    voxels (counted in integer micrometres) and is padded by one layer of
 *    unoccupied samples so that every mesh is closed.
 *  - The exact intersection of Eqs. (2)-(3) is computed as a fixed number of
 *    3D bisection steps of the same all-cameras predicate; 0 steps gives the
 *    edge midpoint (isovalue 0.5).  The paper's own form (a pixel walk along
 *    each projected edge, Eq. (2) per camera, the minimum of Eq. (3)) is the
 *    alternative surface rule, edge_lambda below.
 *  - MC faces with two diagonal ON corners separate the ON corners.
 *  - The triangle depth is the distance from the triangle centroid to the
 *    camera centre (Sec. II-D-1), also used for the occlusion test of
 *    Sec. II-D-2, which is made per vertex.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <tgmath.h> /* sqrt/floor resolve to the float or double routine of R */

#ifndef ORC_REAL
#define ORC_REAL float
#endif
typedef ORC_REAL R;

#define ORC_STRICT 0
#define ORC_ABSTAIN 1

typedef struct {
    int n_cams;
    const float *P;      /* n_cams x 12: row-major 3x4 world -> pixel */
    const float *centre; /* n_cams x 3: camera centres in world metres */
    const int *width;    /* n_cams */
    const int *height;   /* n_cams */
    float vol_min[3], vol_max[3];
    float coarse_m, fine_m;
    int bisect_steps;
    int t_np, t_nb;
    float t_v;
    int oob_policy;
    int surface_rule;    /* ORC_SURFACE_BISECT or ORC_SURFACE_LAMBDA */
} orc_rig;

#define ORC_SURFACE_BISECT 0
#define ORC_SURFACE_LAMBDA 1

typedef struct {
    int cmin[3], cmax[3]; /* inclusive coarse box of the component          */
    int gmin[3], gmax[3]; /* the same grown by one voxel, clamped to grid   */
    int fdim[3];          /* fine samples per axis                          */
    double forigin[3];    /* fine grid origin (value of type R)             */
    long long count;      /* coarse voxels in the component                 */
} orc_roi;

typedef struct {
    int dims[3];
    uint8_t *coarse;      /* dims[0]*dims[1]*dims[2], index (z*ny+y)*nx+x   */
    int32_t *labels;      /* canonical labels after the filter, 0 = none   */
    int n_components;     /* components before the filter                  */
    int n_rois;
    orc_roi *rois;
    long long *fine_offset; /* n_rois+1 offsets into fine                   */
    uint8_t *fine;          /* per-ROI fine occupancy, x fastest            */
    long long n_verts, n_tris;
    long long *roi_vert_offset; /* n_rois+1 */
    long long *roi_tri_offset;  /* n_rois+1 */
    double *verts;        /* n_verts x 3 (values of type R)                 */
    uint64_t *vert_key;   /* n_verts: 3*Lpad+axis within its ROI           */
    double *vert_a;       /* n_verts x 3: final ON end of the bisection     */
    double *vert_b;       /* n_verts x 3: final OFF end of the bisection    */
    uint32_t *tris;       /* n_tris x 3, frame-wide vertex indices          */
    long long tests_coarse, tests_fine, tests_bisect;
} orc_frame;

/* ---------------------------------------------------------------- helpers */

static long long um_of(float m) { return llround((double)m * 1e6); }

static int grid_dim(float lo, float hi, float step)
{
    long long d = um_of(hi) - um_of(lo), s = um_of(step);
    if (s <= 0 || d <= 0) return 0;
    return (int)((d + s - 1) / s);
}

/* Index of the pixel holding the projected coordinate: floor of the exact
 * quotient x/w of the homogeneous coordinates as computed (w > 0).  For the
 * binary32 build the quotient is formed in double: a quotient of two binary32
 * numbers that is not an integer lies at least 2^-41 of its magnitude (for
 * magnitudes below 2^16) from every integer, far above double rounding, so
 * the double floor is the exact one. */
static double pixel_floor(R x, R w) { return floor((double)x / (double)w); }

/* Row r of the homogeneous projection, P_r . (X, Y, Z, 1), evaluated as
 * ((p_r3 + p_r2 Z) + p_r1 Y) + p_r0 X with every step one fused
 * multiply-add (one rounding each, from the innermost term out). */
static R proj_row(const float *p, int r, R X, R Y, R Z)
{
    const float *q = p + 4 * r;
    return fma((R)q[0], X, fma((R)q[1], Y, fma((R)q[2], Z, (R)q[3])));
}

/* One camera's vote for world point (X,Y,Z): 1 foreground, 0 background,
 * -1 abstain (Sec. II-B-1: project the voxel onto the silhouette). */
static int camera_vote(const orc_rig *rig, const uint8_t *const *masks, int n,
                       R X, R Y, R Z)
{
    const float *p = rig->P + 12 * n;
    R xp = proj_row(p, 0, X, Y, Z);
    R yp = proj_row(p, 1, X, Y, Z);
    R wp = proj_row(p, 2, X, Y, Z);
    int off = rig->oob_policy == ORC_ABSTAIN ? -1 : 0;
    if (!(wp > (R)0)) return off;
    double fu = pixel_floor(xp, wp), fv = pixel_floor(yp, wp);
    int W = rig->width[n], H = rig->height[n];
    if (!(fu >= 0.0 && fu < (double)W && fv >= 0.0 && fv < (double)H)) return off;
    int px = (int)fu, py = (int)fv;
    return masks[n][(size_t)py * (size_t)W + (size_t)px] != 0;
}

/* Occupancy of one point: ON iff no camera votes background (and, under
 * ABSTAIN, at least one votes foreground).  Cameras are taken in index
 * order and the test stops at the first background vote; *tests counts the
 * camera tests made. */
static int point_on(const orc_rig *rig, const uint8_t *const *masks,
                    R X, R Y, R Z, long long *tests)
{
    int voted = 0;
    for (int n = 0; n < rig->n_cams; ++n) {
        ++*tests;
        int v = camera_vote(rig, masks, n, X, Y, Z);
        if (v == 0) return 0;
        if (v == 1) voted = 1;
    }
    return voted;
}

/* Pixel index of a Bresenham end point: the floor of the exact quotient,
 * clamped to [-1, n + 1] (n = image width or height), so that an end point
 * far outside the image keeps the walk short. */
static long long end_pixel(R x, R w, int n)
{
    double f = pixel_floor(x, w);
    if (f < -1.0) return -1;
    if (f > (double)n + 1.0) return (long long)n + 1;
    return (long long)f;
}

/* Sec. II-C, Eq. (2), camera n, for the grid edge from the ON sample a to
 * the OFF sample b.  The end points project to the image positions
 * p_on = (x'/w', y'/w') and p_off (binary32 quotients) and to the pixels A
 * and B holding them.  The pixels of the line from A to B are visited in
 * Bresenham order starting at A; the walk stops at the first pixel that is
 * outside the image or not in the silhouette, and P_n is the last pixel
 * before it.  lambda_n = |c(P_n) - p_on| / |p_off - p_on| with c(P_n) the
 * pixel centre, clamped to at most 1.  A camera that has an end point behind
 * it, that does not see A in its silhouette (only possible under ABSTAIN),
 * whose walk reaches B, or for which p_on = p_off, bounds nothing: 1.
 * Every pixel visited counts as one test. */
static R camera_lambda(const orc_rig *rig, const uint8_t *const *masks, int n, const R *a, const R *b,
                       long long *tests)
{
    const float *p = rig->P + 12 * n;
    R xa = proj_row(p, 0, a[0], a[1], a[2]);
    R ya = proj_row(p, 1, a[0], a[1], a[2]);
    R wa = proj_row(p, 2, a[0], a[1], a[2]);
    R xb = proj_row(p, 0, b[0], b[1], b[2]);
    R yb = proj_row(p, 1, b[0], b[1], b[2]);
    R wb = proj_row(p, 2, b[0], b[1], b[2]);
    if (!(wa > (R)0 && wb > (R)0)) return (R)1;
    int W = rig->width[n], H = rig->height[n];
    long long x = end_pixel(xa, wa, W), y = end_pixel(ya, wa, H);
    long long x1 = end_pixel(xb, wb, W), y1 = end_pixel(yb, wb, H);
    long long dx = x1 > x ? x1 - x : x - x1, dy = y1 > y ? y - y1 : y1 - y; /* dy <= 0 */
    long long sx = x < x1 ? 1 : -1, sy = y < y1 ? 1 : -1, err = dx + dy;
    int have = 0;
    long long lx = 0, ly = 0;
    for (;;) {
        ++*tests;
        int fg = x >= 0 && x < W && y >= 0 && y < H && masks[n][(size_t)y * (size_t)W + (size_t)x] != 0;
        if (!fg) break;
        have = 1;
        lx = x;
        ly = y;
        if (x == x1 && y == y1) return (R)1;
        long long e2 = 2 * err;
        if (e2 >= dy) { err += dy; x += sx; }
        if (e2 <= dx) { err += dx; y += sy; }
    }
    if (!have) return (R)1;
    R ua = xa / wa, va = ya / wa, ub = xb / wb, vb = yb / wb;
    R cx = (R)lx + (R)0.5, cy = (R)ly + (R)0.5;
    R num = sqrt((cx - ua) * (cx - ua) + (cy - va) * (cy - va));
    R den = sqrt((ub - ua) * (ub - ua) + (vb - va) * (vb - va));
    if (!(den > (R)0)) return (R)1;
    R l = num / den;
    return l < (R)1 ? l : (R)1;
}

/* Sec. II-C, Eq. (3): lambda = the minimum of Eq. (2) over all cameras, in
 * index order; the vertex is a + lambda (b - a). */
static R edge_lambda(const orc_rig *rig, const uint8_t *const *masks, const R *a, const R *b, R *lam_n,
                     long long *tests)
{
    R lam = (R)1;
    for (int n = 0; n < rig->n_cams; ++n) {
        R l = camera_lambda(rig, masks, n, a, b, tests);
        if (lam_n) lam_n[n] = l;
        if (l < lam) lam = l;
    }
    return lam;
}

/* Public: Eqs. (2)-(3) for a list of edges (end points as double values of
 * type R); lam_n (may be NULL) receives n_edges x n_cams per-camera values. */
int orc_edge_lambda(const orc_rig *rig, const uint8_t *const *masks, long long n_edges, const double *a,
                    const double *b, double *lam, double *lam_n, long long *tests)
{
    long long t = 0;
    R *ln = (R *)malloc(sizeof(R) * (size_t)(rig->n_cams > 0 ? rig->n_cams : 1));
    if (!ln) return -1;
    for (long long i = 0; i < n_edges; ++i) {
        R ra[3] = {(R)a[3 * i], (R)a[3 * i + 1], (R)a[3 * i + 2]};
        R rb[3] = {(R)b[3 * i], (R)b[3 * i + 1], (R)b[3 * i + 2]};
        lam[i] = (double)edge_lambda(rig, masks, ra, rb, ln, &t);
        if (lam_n)
            for (int n = 0; n < rig->n_cams; ++n) lam_n[i * rig->n_cams + n] = (double)ln[n];
    }
    free(ln);
    if (tests) *tests = t;
    return 0;
}

/* Public: occupancy of a list of points (values of type R, given as double). */
int orc_points_on(const orc_rig *rig, const uint8_t *const *masks, long long n_pts,
                  const double *pts, uint8_t *on, long long *tests)
{
    long long t = 0;
    for (long long i = 0; i < n_pts; ++i)
        on[i] = (uint8_t)point_on(rig, masks, (R)pts[3 * i], (R)pts[3 * i + 1],
                                  (R)pts[3 * i + 2], &t);
    if (tests) *tests = t;
    return 0;
}

int orc_grid_dims(const orc_rig *rig, int *dims)
{
    for (int a = 0; a < 3; ++a)
        dims[a] = grid_dim(rig->vol_min[a], rig->vol_max[a], rig->coarse_m);
    return (dims[0] > 0 && dims[1] > 0 && dims[2] > 0) ? 0 : -1;
}

/* ------------------------------------------------ Sec. II-B-1: coarse hull */

int orc_coarse(const orc_rig *rig, const uint8_t *const *masks, uint8_t *occ,
               long long *tests)
{
    int d[3];
    if (orc_grid_dims(rig, d)) return -1;
    R s = (R)rig->coarse_m;
    R ox = (R)rig->vol_min[0], oy = (R)rig->vol_min[1], oz = (R)rig->vol_min[2];
    long long t = 0;
    for (int z = 0; z < d[2]; ++z) {
        R Z = oz + ((R)z + (R)0.5) * s;
        for (int y = 0; y < d[1]; ++y) {
            R Y = oy + ((R)y + (R)0.5) * s;
            for (int x = 0; x < d[0]; ++x) {
                R X = ox + ((R)x + (R)0.5) * s;
                occ[((size_t)z * d[1] + y) * d[0] + x] =
                    (uint8_t)point_on(rig, masks, X, Y, Z, &t);
            }
        }
    }
    *tests = t;
    return 0;
}

/* ------------------------------------------- Sec. II-B-2: 26-connected CCL */

/* Breadth-first flood fill over the 26-neighbourhood.  Components are
 * numbered 1..C in order of their smallest linear index (the first voxel
 * met in a scan in index order). Returns C. */
int orc_ccl_bfs(int nx, int ny, int nz, const uint8_t *occ, int32_t *lab)
{
    size_t n = (size_t)nx * ny * nz;
    for (size_t i = 0; i < n; ++i) lab[i] = 0;
    size_t *queue = (size_t *)malloc((n ? n : 1) * sizeof(size_t));
    if (!queue) return -1;
    int c = 0;
    for (size_t s = 0; s < n; ++s) {
        if (!occ[s] || lab[s]) continue;
        ++c;
        size_t head = 0, tail = 0;
        queue[tail++] = s;
        lab[s] = c;
        while (head < tail) {
            size_t v = queue[head++];
            int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((size_t)nx * ny));
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int X = x + dx, Y = y + dy, Z = z + dz;
                        if (X < 0 || Y < 0 || Z < 0 || X >= nx || Y >= ny || Z >= nz) continue;
                        size_t w = ((size_t)Z * ny + Y) * nx + X;
                        if (occ[w] && !lab[w]) {
                            lab[w] = c;
                            queue[tail++] = w;
                        }
                    }
        }
    }
    free(queue);
    return c;
}

/* A second, independent labelling inside the oracle: sequential union-find
 * (union by smaller index, path halving) over the 13 neighbours that precede
 * each voxel, then numbering by smallest index.  Used only to cross-check
 * orc_ccl_bfs. */
static size_t uf_find(size_t *par, size_t a)
{
    while (par[a] != a) {
        par[a] = par[par[a]];
        a = par[a];
    }
    return a;
}

int orc_ccl_uf(int nx, int ny, int nz, const uint8_t *occ, int32_t *lab)
{
    size_t n = (size_t)nx * ny * nz;
    size_t *par = (size_t *)malloc((n ? n : 1) * sizeof(size_t));
    if (!par) return -1;
    for (size_t i = 0; i < n; ++i) par[i] = i;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t v = ((size_t)z * ny + y) * nx + x;
                if (!occ[v]) continue;
                for (int dz = -1; dz <= 0; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            if (dz == 0 && (dy > 0 || (dy == 0 && dx >= 0))) continue;
                            int X = x + dx, Y = y + dy, Z = z + dz;
                            if (X < 0 || Y < 0 || Z < 0 || X >= nx || Y >= ny) continue;
                            size_t w = ((size_t)Z * ny + Y) * nx + X;
                            if (!occ[w]) continue;
                            size_t ra = uf_find(par, v), rb = uf_find(par, w);
                            if (ra < rb) par[rb] = ra;
                            else if (rb < ra) par[ra] = rb;
                        }
            }
    int c = 0;
    for (size_t i = 0; i < n; ++i) {
        if (!occ[i]) { lab[i] = 0; continue; }
        size_t r = uf_find(par, i);
        if (r == i) lab[i] = ++c;
        else lab[i] = lab[r]; /* r < i, so it is numbered already */
    }
    free(par);
    return c;
}

/* ----------------------- Sec. II-B-2: minimum box, Eq. (1) filter, 3D ROI */

/* From the raw labels 1..C: per component its voxel count and inclusive box;
 * keep iff t_np <= count <= t_nb (the prose reading of Eq. (1)); number the
 * kept ones 1..K in raw order; write the canonical labels (0 for removed and
 * background) and the ROI of each kept component: the box grown by one
 * coarse voxel per side, clamped, with its fine grid size and origin.
 * Returns K, or -1. */
int orc_filter(const orc_rig *rig, int nx, int ny, int nz, const int32_t *raw,
               int n_comp, int32_t *lab, orc_roi *rois, int max_rois)
{
    size_t n = (size_t)nx * ny * nz;
    long long *cnt = (long long *)calloc((size_t)n_comp + 1, sizeof(long long));
    int *bb = (int *)malloc(((size_t)n_comp + 1) * 6 * sizeof(int));
    int *newl = (int *)calloc((size_t)n_comp + 1, sizeof(int));
    if (!cnt || !bb || !newl) { free(cnt); free(bb); free(newl); return -1; }
    for (int c = 0; c <= n_comp; ++c) {
        bb[6 * c + 0] = bb[6 * c + 1] = bb[6 * c + 2] = 1 << 30;
        bb[6 * c + 3] = bb[6 * c + 4] = bb[6 * c + 5] = -1;
    }
    for (size_t i = 0; i < n; ++i) {
        int c = raw[i];
        if (!c) continue;
        int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((size_t)nx * ny));
        int q[3] = {x, y, z};
        ++cnt[c];
        for (int a = 0; a < 3; ++a) {
            if (q[a] < bb[6 * c + a]) bb[6 * c + a] = q[a];
            if (q[a] > bb[6 * c + 3 + a]) bb[6 * c + 3 + a] = q[a];
        }
    }
    int dims[3] = {nx, ny, nz};
    long long cu = um_of(rig->coarse_m), fu = um_of(rig->fine_m);
    R sc = (R)rig->coarse_m;
    int K = 0;
    for (int c = 1; c <= n_comp; ++c) {
        if (cnt[c] < (long long)rig->t_np || cnt[c] > (long long)rig->t_nb) continue;
        newl[c] = ++K;
        if (K > max_rois) continue;
        orc_roi *r = &rois[K - 1];
        r->count = cnt[c];
        for (int a = 0; a < 3; ++a) {
            r->cmin[a] = bb[6 * c + a];
            r->cmax[a] = bb[6 * c + 3 + a];
            r->gmin[a] = r->cmin[a] > 0 ? r->cmin[a] - 1 : 0;
            r->gmax[a] = r->cmax[a] < dims[a] - 1 ? r->cmax[a] + 1 : dims[a] - 1;
            long long span = (long long)(r->gmax[a] - r->gmin[a] + 1) * cu;
            r->fdim[a] = (int)((span + fu - 1) / fu);
            R o = (R)rig->vol_min[a];
            R off = (R)r->gmin[a] * sc;
            r->forigin[a] = (double)(o + off);
        }
    }
    for (size_t i = 0; i < n; ++i) lab[i] = raw[i] ? newl[raw[i]] : 0;
    free(cnt); free(bb); free(newl);
    return K;
}

/* --------------------------------------------- Sec. II-B-3: fine hull in ROI */

int orc_fine(const orc_rig *rig, const uint8_t *const *masks, const orc_roi *r,
             uint8_t *occ, long long *tests)
{
    R s = (R)rig->fine_m;
    R ox = (R)r->forigin[0], oy = (R)r->forigin[1], oz = (R)r->forigin[2];
    long long t = 0;
    for (int z = 0; z < r->fdim[2]; ++z) {
        R Z = oz + ((R)z + (R)0.5) * s;
        for (int y = 0; y < r->fdim[1]; ++y) {
            R Y = oy + ((R)y + (R)0.5) * s;
            for (int x = 0; x < r->fdim[0]; ++x) {
                R X = ox + ((R)x + (R)0.5) * s;
                occ[((size_t)z * r->fdim[1] + y) * r->fdim[0] + x] =
                    (uint8_t)point_on(rig, masks, X, Y, Z, &t);
            }
        }
    }
    *tests = t;
    return 0;
}

/* ---------------------------------- Sec. II-C: marching-cubes cell polygons */

/* Cube corners are numbered dx + 2dy + 4dz.  Cube edge e has axis e/4; its
 * two other coordinates (u, w) = (e%4 & 1, e%4 >> 1) are, in axis order, the
 * coordinates of its lower corner that are not along the axis. */
static void cube_edge_corners(int e, int *c0, int *c1)
{
    int a = e >> 2, u = e & 1, w = (e >> 1) & 1;
    if (a == 0) { *c0 = 2 * u + 4 * w; *c1 = *c0 + 1; }
    else if (a == 1) { *c0 = u + 4 * w; *c1 = *c0 + 2; }
    else { *c0 = u + 2 * w; *c1 = *c0 + 4; }
}

static int corner_coord(int c, int a) { return (c >> a) & 1; }

/* Each cube edge lies on the two faces (axis b, side t) with b not its axis
 * and t the lower corner's coordinate along b. */
static int cube_edges_share_face(int e, int f)
{
    int c0, c1, d0, d1;
    cube_edge_corners(e, &c0, &c1);
    cube_edge_corners(f, &d0, &d1);
    for (int b = 0; b < 3; ++b) {
        if (b == (e >> 2) || b == (f >> 2)) continue;
        if (corner_coord(c0, b) == corner_coord(d0, b)) return 1;
    }
    return 0;
}

/* Polygons of one cell with corner states given by bits of `cs`.  On each
 * cube face the bipolar edges are joined by segments: two bipolar edges are
 * joined; four (two diagonal ON corners) are joined in the pairs that cut off
 * each ON corner.  Each segment is directed so that, seen from outside the
 * cube, the ON side lies to its right; following the directed segments gives
 * closed polygons whose normals point from ON to OFF.  Polygons are listed in
 * order of their smallest cube-edge number; each is fanned from the first
 * vertex, in polygon order from the smallest, whose diagonals all leave the
 * cube faces (so no two cells draw the same diagonal on a shared face).
 * Writes up to 12 triangles (3 cube edges each) and returns their number, or
 * -1 if the segments do not form closed loops. */
int orc_mc_cell(int cs, int *tri_edges)
{
    int on[8], bip[12], next[12];
    for (int c = 0; c < 8; ++c) on[c] = (cs >> c) & 1;
    for (int e = 0; e < 12; ++e) {
        int c0, c1;
        cube_edge_corners(e, &c0, &c1);
        bip[e] = on[c0] != on[c1];
        next[e] = -1;
    }
    for (int f = 0; f < 6; ++f) {
        int a = f >> 1, t = f & 1;
        int fe[4], nfe = 0;
        for (int e = 0; e < 12; ++e) {
            if ((e >> 2) == a || !bip[e]) continue;
            int c0, c1;
            cube_edge_corners(e, &c0, &c1);
            if (corner_coord(c0, a) == t && corner_coord(c1, a) == t) fe[nfe++] = e;
        }
        if (nfe == 0) continue;
        /* pairs (p, q) with the ON corner that decides the direction */
        int pairs[2][3], npairs = 0;
        if (nfe == 2) {
            int onc = -1;
            for (int c = 0; c < 8; ++c)
                if (corner_coord(c, a) == t && on[c]) { onc = c; break; }
            pairs[0][0] = fe[0]; pairs[0][1] = fe[1]; pairs[0][2] = onc;
            npairs = 1;
        } else if (nfe == 4) {
            for (int c = 0; c < 8; ++c) {
                if (corner_coord(c, a) != t || !on[c]) continue;
                int k = 0, pe[2];
                for (int i = 0; i < 4; ++i) {
                    int c0, c1;
                    cube_edge_corners(fe[i], &c0, &c1);
                    if (c0 == c || c1 == c) pe[k++] = fe[i];
                }
                if (k != 2) return -1;
                pairs[npairs][0] = pe[0]; pairs[npairs][1] = pe[1]; pairs[npairs][2] = c;
                ++npairs;
            }
        } else {
            return -1;
        }
        for (int i = 0; i < npairs; ++i) {
            int p = pairs[i][0], q = pairs[i][1], A = pairs[i][2];
            int c0, c1, P2[3], Q2[3], A2[3];
            cube_edge_corners(p, &c0, &c1);
            for (int k = 0; k < 3; ++k) P2[k] = corner_coord(c0, k) + corner_coord(c1, k);
            cube_edge_corners(q, &c0, &c1);
            for (int k = 0; k < 3; ++k) Q2[k] = corner_coord(c0, k) + corner_coord(c1, k);
            for (int k = 0; k < 3; ++k) A2[k] = 2 * corner_coord(A, k);
            int d[3] = {Q2[0] - P2[0], Q2[1] - P2[1], Q2[2] - P2[2]};
            int g[3] = {A2[0] - P2[0], A2[1] - P2[1], A2[2] - P2[2]};
            int cr[3] = {d[1] * g[2] - d[2] * g[1], d[2] * g[0] - d[0] * g[2],
                         d[0] * g[1] - d[1] * g[0]};
            int sgn = cr[a] * (t ? 1 : -1);
            if (sgn == 0) return -1;
            int from = sgn < 0 ? p : q, to = sgn < 0 ? q : p;
            if (next[from] != -1) return -1;
            next[from] = to;
        }
    }
    int seen[12] = {0}, ntri = 0;
    for (int e0 = 0; e0 < 12; ++e0) {
        if (!bip[e0] || seen[e0]) continue;
        int poly[12], np = 0, e = e0;
        do {
            if (e < 0 || seen[e] || np >= 12) return -1;
            seen[e] = 1;
            poly[np++] = e;
            e = next[e];
        } while (e != e0);
        /* apex: the first vertex (from the smallest cube edge on, in polygon
         * order) that shares no cube face with a vertex it is not joined to;
         * a diagonal lying in a face could otherwise be drawn by the cell on
         * the other side of that face too. */
        int k = -1;
        for (int i = 0; i < np && k < 0; ++i) {
            int ok = 1;
            for (int j = 0; j < np && ok; ++j) {
                int d = (j - i + np) % np;
                if (d == 0 || d == 1 || d == np - 1) continue;
                if (cube_edges_share_face(poly[i], poly[j])) ok = 0;
            }
            if (ok) k = i;
        }
        if (k < 0) return -1;
        for (int i = 1; i + 1 < np; ++i) {
            tri_edges[3 * ntri + 0] = poly[k];
            tri_edges[3 * ntri + 1] = poly[(k + i) % np];
            tri_edges[3 * ntri + 2] = poly[(k + i + 1) % np];
            ++ntri;
        }
    }
    return ntri;
}

/* ----------------- Sec. II-C: bipolar edges, bisection, triangles of one ROI */

typedef struct {
    double *v, *a, *b; uint64_t *k; long long n, cap;
} vbuf;
typedef struct {
    uint32_t *t; long long n, cap;
} tbuf;

static int vpush(vbuf *b, const R *p, const R *pa, const R *pb, uint64_t key)
{
    if (b->n == b->cap) {
        long long nc = b->cap ? 2 * b->cap : 4096;
        double *nv = (double *)realloc(b->v, (size_t)nc * 3 * sizeof(double));
        if (!nv) return -1;
        b->v = nv;
        nv = (double *)realloc(b->a, (size_t)nc * 3 * sizeof(double));
        if (!nv) return -1;
        b->a = nv;
        nv = (double *)realloc(b->b, (size_t)nc * 3 * sizeof(double));
        if (!nv) return -1;
        b->b = nv;
        uint64_t *nk = (uint64_t *)realloc(b->k, (size_t)nc * sizeof(uint64_t));
        if (!nk) return -1;
        b->k = nk;
        b->cap = nc;
    }
    b->v[3 * b->n + 0] = (double)p[0];
    b->v[3 * b->n + 1] = (double)p[1];
    b->v[3 * b->n + 2] = (double)p[2];
    for (int i = 0; i < 3; ++i) {
        b->a[3 * b->n + i] = (double)pa[i];
        b->b[3 * b->n + i] = (double)pb[i];
    }
    b->k[b->n] = key;
    ++b->n;
    return 0;
}

static int tpush(tbuf *b, uint32_t i0, uint32_t i1, uint32_t i2)
{
    if (b->n == b->cap) {
        long long nc = b->cap ? 2 * b->cap : 8192;
        uint32_t *nt = (uint32_t *)realloc(b->t, (size_t)nc * 3 * sizeof(uint32_t));
        if (!nt) return -1;
        b->t = nt;
        b->cap = nc;
    }
    b->t[3 * b->n + 0] = i0;
    b->t[3 * b->n + 1] = i1;
    b->t[3 * b->n + 2] = i2;
    ++b->n;
    return 0;
}

/* Centre of padded sample (xp,yp,zp): the fine voxel (xp-1, yp-1, zp-1). */
static void sample_centre(const orc_roi *r, R s, int xp, int yp, int zp, R *c)
{
    c[0] = (R)r->forigin[0] + ((R)(xp - 1) + (R)0.5) * s;
    c[1] = (R)r->forigin[1] + ((R)(yp - 1) + (R)0.5) * s;
    c[2] = (R)r->forigin[2] + ((R)(zp - 1) + (R)0.5) * s;
}

/* Mesh of one ROI.  The fine occupancy is padded by one layer of unoccupied
 * samples.  Every grid edge whose two samples differ gets one vertex; vertices
 * are numbered in order of the key 3*Lpad + axis of the edge (Lpad is the
 * padded linear index of its lower sample).  Each vertex is placed by
 * `steps` bisections between the ON end a and the OFF end b: m = (a+b)/2,
 * a = m if m is occupied else b = m; the vertex is the final midpoint.
 * Triangles follow orc_mc_cell for the cells in padded index order of their
 * lower corner; indices are offset by vbase. */
static int mesh_roi(const orc_rig *rig, const uint8_t *const *masks, const orc_roi *r,
                    const uint8_t *occ, uint32_t vbase, vbuf *vb, tbuf *tb,
                    long long *tests)
{
    int nx = r->fdim[0], ny = r->fdim[1], nz = r->fdim[2];
    int px = nx + 2, py = ny + 2, pz = nz + 2;
    size_t np = (size_t)px * py * pz;
    int32_t *vid = (int32_t *)malloc(np * 3 * sizeof(int32_t));
    if (!vid) return -1;
    R s = (R)rig->fine_m;
    long long vstart = vb->n;
#define SAMPLE(X, Y, Z)                                                                  \
    (((X) >= 1 && (X) <= nx && (Y) >= 1 && (Y) <= ny && (Z) >= 1 && (Z) <= nz)          \
         ? occ[((size_t)((Z)-1) * ny + ((Y)-1)) * nx + ((X)-1)]                         \
         : 0)
    for (int zp = 0; zp < pz; ++zp)
        for (int yp = 0; yp < py; ++yp)
            for (int xp = 0; xp < px; ++xp) {
                size_t L = ((size_t)zp * py + yp) * px + xp;
                int s0 = SAMPLE(xp, yp, zp) != 0;
                for (int a = 0; a < 3; ++a) {
                    vid[3 * L + a] = -1;
                    int q[3] = {xp, yp, zp};
                    q[a] += 1;
                    if (q[0] >= px || q[1] >= py || q[2] >= pz) continue;
                    int s1 = SAMPLE(q[0], q[1], q[2]) != 0;
                    if (s0 == s1) continue;
                    R ca[3], cb[3], m[3];
                    if (s0) {
                        sample_centre(r, s, xp, yp, zp, ca);
                        sample_centre(r, s, q[0], q[1], q[2], cb);
                    } else {
                        sample_centre(r, s, q[0], q[1], q[2], ca);
                        sample_centre(r, s, xp, yp, zp, cb);
                    }
                    if (rig->surface_rule == ORC_SURFACE_LAMBDA) {
                        R lam = edge_lambda(rig, masks, ca, cb, NULL, tests);
                        for (int k = 0; k < 3; ++k) m[k] = ca[k] + lam * (cb[k] - ca[k]);
                    } else {
                        for (int it = 0; it < rig->bisect_steps; ++it) {
                            for (int k = 0; k < 3; ++k) m[k] = (ca[k] + cb[k]) * (R)0.5;
                            if (point_on(rig, masks, m[0], m[1], m[2], tests))
                                for (int k = 0; k < 3; ++k) ca[k] = m[k];
                            else
                                for (int k = 0; k < 3; ++k) cb[k] = m[k];
                        }
                        for (int k = 0; k < 3; ++k) m[k] = (ca[k] + cb[k]) * (R)0.5;
                    }
                    vid[3 * L + a] = (int32_t)(vb->n - vstart);
                    if (vpush(vb, m, ca, cb, 3ull * (uint64_t)L + (uint64_t)a)) { free(vid); return -1; }
                }
            }
    for (int cz = 0; cz <= nz; ++cz)
        for (int cy = 0; cy <= ny; ++cy)
            for (int cx = 0; cx <= nx; ++cx) {
                int cs = 0;
                for (int c = 0; c < 8; ++c)
                    if (SAMPLE(cx + (c & 1), cy + ((c >> 1) & 1), cz + ((c >> 2) & 1)))
                        cs |= 1 << c;
                if (cs == 0 || cs == 255) continue;
                int te[36];
                int nt = orc_mc_cell(cs, te);
                if (nt < 0) { free(vid); return -1; }
                for (int t = 0; t < nt; ++t) {
                    uint32_t id[3];
                    for (int j = 0; j < 3; ++j) {
                        int e = te[3 * t + j], c0, c1;
                        cube_edge_corners(e, &c0, &c1);
                        int X = cx + corner_coord(c0, 0), Y = cy + corner_coord(c0, 1),
                            Z = cz + corner_coord(c0, 2);
                        size_t L = ((size_t)Z * py + Y) * px + X;
                        int32_t v = vid[3 * L + (e >> 2)];
                        if (v < 0) { free(vid); return -1; }
                        id[j] = vbase + (uint32_t)v;
                    }
                    if (tpush(tb, id[0], id[1], id[2])) { free(vid); return -1; }
                }
            }
#undef SAMPLE
    free(vid);
    return 0;
}

/* ------------------------------------------------------ the whole frame */

void orc_frame_free(orc_frame *f)
{
    free(f->coarse); free(f->labels); free(f->rois); free(f->fine_offset);
    free(f->fine); free(f->roi_vert_offset); free(f->roi_tri_offset);
    free(f->verts); free(f->vert_key); free(f->vert_a); free(f->vert_b); free(f->tris);
    memset(f, 0, sizeof(*f));
}

/* Sec. II-B and II-C for one frame: coarse hull, CCL, filter and ROIs, fine
 * hull per ROI, mesh per ROI.  Returns 0, -1 on allocation failure or bad
 * grid, -2 if more than max_rois components are kept. */
int orc_reconstruct(const orc_rig *rig, const uint8_t *const *masks, int max_rois,
                    orc_frame *f)
{
    memset(f, 0, sizeof(*f));
    if (orc_grid_dims(rig, f->dims)) return -1;
    int nx = f->dims[0], ny = f->dims[1], nz = f->dims[2];
    size_t n = (size_t)nx * ny * nz;
    f->coarse = (uint8_t *)malloc(n);
    f->labels = (int32_t *)malloc(n * sizeof(int32_t));
    int32_t *raw = (int32_t *)malloc(n * sizeof(int32_t));
    if (!f->coarse || !f->labels || !raw) { free(raw); orc_frame_free(f); return -1; }
    orc_coarse(rig, masks, f->coarse, &f->tests_coarse);
    f->n_components = orc_ccl_bfs(nx, ny, nz, f->coarse, raw);
    f->rois = (orc_roi *)calloc((size_t)(max_rois > 0 ? max_rois : 1), sizeof(orc_roi));
    if (f->n_components < 0 || !f->rois) { free(raw); orc_frame_free(f); return -1; }
    int K = orc_filter(rig, nx, ny, nz, raw, f->n_components, f->labels, f->rois, max_rois);
    free(raw);
    if (K < 0) { orc_frame_free(f); return -1; }
    if (K > max_rois) { orc_frame_free(f); return -2; }
    f->n_rois = K;
    f->fine_offset = (long long *)calloc((size_t)K + 1, sizeof(long long));
    f->roi_vert_offset = (long long *)calloc((size_t)K + 1, sizeof(long long));
    f->roi_tri_offset = (long long *)calloc((size_t)K + 1, sizeof(long long));
    if (!f->fine_offset || !f->roi_vert_offset || !f->roi_tri_offset) { orc_frame_free(f); return -1; }
    for (int r = 0; r < K; ++r)
        f->fine_offset[r + 1] = f->fine_offset[r] +
            (long long)f->rois[r].fdim[0] * f->rois[r].fdim[1] * f->rois[r].fdim[2];
    f->fine = (uint8_t *)malloc((size_t)(f->fine_offset[K] ? f->fine_offset[K] : 1));
    if (!f->fine) { orc_frame_free(f); return -1; }
    vbuf vb = {0};
    tbuf tb = {0};
    for (int r = 0; r < K; ++r) {
        long long t = 0;
        orc_fine(rig, masks, &f->rois[r], f->fine + f->fine_offset[r], &t);
        f->tests_fine += t;
        f->roi_vert_offset[r] = vb.n;
        f->roi_tri_offset[r] = tb.n;
        if (mesh_roi(rig, masks, &f->rois[r], f->fine + f->fine_offset[r], (uint32_t)vb.n,
                     &vb, &tb, &f->tests_bisect)) {
            free(vb.v); free(vb.a); free(vb.b); free(vb.k); free(tb.t); orc_frame_free(f); return -1;
        }
    }
    f->roi_vert_offset[K] = vb.n;
    f->roi_tri_offset[K] = tb.n;
    f->n_verts = vb.n;
    f->n_tris = tb.n;
    f->verts = vb.v;
    f->vert_key = vb.k;
    f->vert_a = vb.a;
    f->vert_b = vb.b;
    f->tris = tb.t;
    return 0;
}

/* Sec. II-C for one ROI whose fine occupancy is given: fills the vertex and
 * triangle fields of *f (and its ROI offsets) only.  Returns 0 or -1. */
int orc_mesh_one(const orc_rig *rig, const uint8_t *const *masks, const orc_roi *roi,
                 const uint8_t *occ, orc_frame *f)
{
    memset(f, 0, sizeof(*f));
    vbuf vb = {0};
    tbuf tb = {0};
    if (mesh_roi(rig, masks, roi, occ, 0, &vb, &tb, &f->tests_bisect)) {
        free(vb.v); free(vb.a); free(vb.b); free(vb.k); free(tb.t);
        return -1;
    }
    f->n_verts = vb.n;
    f->n_tris = tb.n;
    f->verts = vb.v;
    f->vert_key = vb.k;
    f->vert_a = vb.a;
    f->vert_b = vb.b;
    f->tris = tb.t;
    return 0;
}

/* ------------------------ Sec. II-D-1: which pixels a projected triangle covers */

/* For camera n, every triangle whose three vertices are in front of it
 * (w' > 0) and whose projected area is non-zero writes, into each pixel whose
 * centre p = (px+1/2, py+1/2) lies inside or on it, the distance from its
 * centroid ((v0+v1)+v2)/3 to the camera centre; each pixel keeps the minimum
 * (Eq. (4)); a pixel no triangle covers stays +infinity.
 * The test is made on the homogeneous image points (x', y', w') of the
 * vertices, without dividing: for edge (i, j) the edge function at p is
 * (p_x a - p_y b) + c with a = y_i w_j - w_i y_j, b = x_i w_j - w_i x_j,
 * c = x_i y_j - y_i x_j (binary32, in that order) -- the determinant of the
 * two vertices and p, whose sign for w > 0 is that of the image-plane edge
 * function.  p is inside or on the triangle iff the three are all >= 0 or
 * all <= 0.  The projected area is zero iff (x_0 a_12 - y_0 b_12) + w_0 c_12
 * is.  Only pixel centres inside the closed box spanned by the projected
 * vertices are tested; that box is decided exactly, by the signs of
 * p_x w_j - x_j (and p_y w_j - y_j) formed with one fma each.
 *
 * tri_cover holds one projected triangle set up for that test: the
 * homogeneous image points of camera matrix p, the edge functions of edges
 * (0,1), (1,2), (2,0), and the candidate pixel box. */
typedef struct {
    R xh[3], yh[3], wh[3], ea[3], eb[3], ec[3];
    int x0, y0, x1, y1;
} tri_cover;

/* Set up triangle (X, Y, Z) in the view of matrix p (image W x H).  Returns
 * 0 if the triangle is skipped: a vertex not in front (w' <= 0), zero
 * projected area, or a box entirely off the image. */
static int cover_setup(const float *p, int W, int H, const R *X, const R *Y, const R *Z, tri_cover *t)
{
    for (int j = 0; j < 3; ++j) {
        t->xh[j] = proj_row(p, 0, X[j], Y[j], Z[j]);
        t->yh[j] = proj_row(p, 1, X[j], Y[j], Z[j]);
        t->wh[j] = proj_row(p, 2, X[j], Y[j], Z[j]);
        if (!(t->wh[j] > (R)0)) return 0;
    }
    for (int e = 0; e < 3; ++e) {
        int i = e, j = (e + 1) % 3;
        t->ea[e] = t->yh[i] * t->wh[j] - t->wh[i] * t->yh[j];
        t->eb[e] = t->xh[i] * t->wh[j] - t->wh[i] * t->xh[j];
        t->ec[e] = t->xh[i] * t->yh[j] - t->yh[i] * t->xh[j];
    }
    R det = (t->xh[0] * t->ea[1] - t->yh[0] * t->eb[1]) + t->wh[0] * t->ec[1];
    if (!(det > (R)0 || det < (R)0)) return 0;
    /* candidate pixels: the projected box widened by one pixel (any superset
     * of the box gives the same coverage) */
    double umin = 1e300, umax = -1e300, vmin = 1e300, vmax = -1e300;
    for (int j = 0; j < 3; ++j) {
        double u = (double)t->xh[j] / (double)t->wh[j], v = (double)t->yh[j] / (double)t->wh[j];
        if (u < umin) umin = u;
        if (u > umax) umax = u;
        if (v < vmin) vmin = v;
        if (v > vmax) vmax = v;
    }
    if (umax < 0.0 || vmax < 0.0 || umin > (double)W || vmin > (double)H) return 0;
    t->x0 = umin < 1.0 ? 0 : (int)floor(umin) - 1;
    t->y0 = vmin < 1.0 ? 0 : (int)floor(vmin) - 1;
    t->x1 = umax > (double)W - 2.0 ? W - 1 : (int)floor(umax) + 1;
    t->y1 = vmax > (double)H - 2.0 ? H - 1 : (int)floor(vmax) + 1;
    return 1;
}

/* Row yy of the candidate box: is the pixel-centre row inside the closed
 * box of the projection (signs of pcy*w_j - y_j, exact by one fma)? */
static int cover_row(const tri_cover *t, int yy)
{
    R pcy = (R)yy + (R)0.5;
    R s0 = fma(pcy, t->wh[0], -t->yh[0]), s1 = fma(pcy, t->wh[1], -t->yh[1]), s2 = fma(pcy, t->wh[2], -t->yh[2]);
    return (s0 >= (R)0 || s1 >= (R)0 || s2 >= (R)0) && (s0 <= (R)0 || s1 <= (R)0 || s2 <= (R)0);
}

/* Pixel (xx, yy) of a row that passed cover_row: centre in the closed box
 * and on the inner side of (or on) all three edges, either winding. */
static int cover_pixel(const tri_cover *t, int xx, int yy)
{
    R pcy = (R)yy + (R)0.5, pcx = (R)xx + (R)0.5;
    R r0 = fma(pcx, t->wh[0], -t->xh[0]), r1 = fma(pcx, t->wh[1], -t->xh[1]), r2 = fma(pcx, t->wh[2], -t->xh[2]);
    if (!((r0 >= (R)0 || r1 >= (R)0 || r2 >= (R)0) && (r0 <= (R)0 || r1 <= (R)0 || r2 <= (R)0))) return 0;
    R e0 = (pcx * t->ea[0] - pcy * t->eb[0]) + t->ec[0];
    R e1 = (pcx * t->ea[1] - pcy * t->eb[1]) + t->ec[1];
    R e2 = (pcx * t->ea[2] - pcy * t->eb[2]) + t->ec[2];
    return (e0 >= (R)0 && e1 >= (R)0 && e2 >= (R)0) || (e0 <= (R)0 && e1 <= (R)0 && e2 <= (R)0);
}

/* Triangle t's vertices and centroid ((v0 + v1) + v2) / 3 (Sec. II-D-1). */
static int tri_points(long long n_verts, const double *verts, const uint32_t *tris, long long t, R *X, R *Y, R *Z,
                      R *g)
{
    for (int j = 0; j < 3; ++j) {
        uint32_t vi = tris[3 * t + j];
        if ((long long)vi >= n_verts) return -1;
        X[j] = (R)verts[3 * vi]; Y[j] = (R)verts[3 * vi + 1]; Z[j] = (R)verts[3 * vi + 2];
    }
    g[0] = ((X[0] + X[1]) + X[2]) / (R)3;
    g[1] = ((Y[0] + Y[1]) + Y[2]) / (R)3;
    g[2] = ((Z[0] + Z[1]) + Z[2]) / (R)3;
    return 0;
}

/* ------------------------------------------ Sec. II-D-1: depth images, Eq. (4) */

/* Per camera, each pixel holds the minimum over the triangles covering it of
 * the distance from the triangle's centroid to the camera centre, +inf if
 * none.  A pixel is covered when its centre lies inside or on the projected
 * triangle, decided on the homogeneous image points without dividing
 * (cover_setup, cover_row, cover_pixel); triangles with a vertex behind the
 * camera or zero projected area are skipped. */
int orc_depth(const orc_rig *rig, long long n_verts, const double *verts,
              long long n_tris, const uint32_t *tris, R *depth)
{
    size_t off = 0;
    for (int n = 0; n < rig->n_cams; ++n) {
        int W = rig->width[n], H = rig->height[n];
        R *D = depth + off;
        off += (size_t)W * H;
        for (size_t i = 0; i < (size_t)W * H; ++i) D[i] = (R)INFINITY;
        const float *p = rig->P + 12 * n;
        R Cx = (R)rig->centre[3 * n], Cy = (R)rig->centre[3 * n + 1], Cz = (R)rig->centre[3 * n + 2];
        for (long long t = 0; t < n_tris; ++t) {
            R X[3], Y[3], Z[3], g[3];
            if (tri_points(n_verts, verts, tris, t, X, Y, Z, g)) return -1;
            tri_cover tc;
            if (!cover_setup(p, W, H, X, Y, Z, &tc)) continue;
            R dx = g[0] - Cx, dy = g[1] - Cy, dz = g[2] - Cz;
            R d = sqrt((dx * dx + dy * dy) + dz * dz);
            for (int yy = tc.y0; yy <= tc.y1; ++yy) {
                if (!cover_row(&tc, yy)) continue;
                for (int xx = tc.x0; xx <= tc.x1; ++xx) {
                    if (!cover_pixel(&tc, xx, yy)) continue;
                    R *px = &D[(size_t)yy * W + xx];
                    if (d < *px) *px = d;
                }
            }
        }
    }
    return 0;
}

/* ------------------------ Sec. II-D-2 and II-E: visibility and vertex colour */

/* Capture cameras ranked by squared distance from their centre to the
 * viewpoint ((dx*dx + dy*dy) + dz*dz), ties to the lower index; doff[n] is
 * camera n's first pixel in the concatenated depth images. */
static int rank_cameras(const orc_rig *rig, const float *viewpoint, int *rank, size_t *doff)
{
    int N = rig->n_cams;
    R *d2 = (R *)malloc((size_t)N * sizeof(R));
    if (!d2) return -1;
    size_t off = 0;
    for (int n = 0; n < N; ++n) {
        R dx = (R)rig->centre[3 * n] - (R)viewpoint[0];
        R dy = (R)rig->centre[3 * n + 1] - (R)viewpoint[1];
        R dz = (R)rig->centre[3 * n + 2] - (R)viewpoint[2];
        d2[n] = (dx * dx + dy * dy) + dz * dz;
        doff[n] = off;
        off += (size_t)rig->width[n] * rig->height[n];
    }
    for (int i = 0; i < N; ++i) rank[i] = i;
    for (int i = 1; i < N; ++i) { /* insertion sort: stable, so ties keep index order */
        int c = rank[i], j = i - 1;
        while (j >= 0 && d2[rank[j]] > d2[c]) { rank[j + 1] = rank[j]; --j; }
        rank[j + 1] = c;
    }
    free(d2);
    return 0;
}

/* The colour of world point (X,Y,Z): the first camera in rank order that
 * has it in front (w' > 0), inside the image, and not occluded:
 * |X - C| - depth[pixel] <= T_v.  Returns that camera (its RGB at the pixel
 * in out3) or -1 with (0,0,0). */
static int colour_point(const orc_rig *rig, const uint8_t *const *rgb, const int *rank, const size_t *doff,
                        const R *depth, R X, R Y, R Z, uint8_t *out3)
{
    out3[0] = out3[1] = out3[2] = 0;
    R tv = (R)rig->t_v;
    for (int r = 0; r < rig->n_cams; ++r) {
        int n = rank[r];
        const float *p = rig->P + 12 * n;
        R xp = proj_row(p, 0, X, Y, Z);
        R yp = proj_row(p, 1, X, Y, Z);
        R wp = proj_row(p, 2, X, Y, Z);
        if (!(wp > (R)0)) continue;
        double fu = pixel_floor(xp, wp), fv = pixel_floor(yp, wp);
        int W = rig->width[n], H = rig->height[n];
        if (!(fu >= 0.0 && fu < (double)W && fv >= 0.0 && fv < (double)H)) continue;
        size_t pix = (size_t)(int)fv * W + (size_t)(int)fu;
        R dx = X - (R)rig->centre[3 * n], dy = Y - (R)rig->centre[3 * n + 1], dz = Z - (R)rig->centre[3 * n + 2];
        R dist = sqrt((dx * dx + dy * dy) + dz * dz);
        if (!(dist - depth[doff[n] + pix] <= tv)) continue;
        out3[0] = rgb[n][3 * pix + 0];
        out3[1] = rgb[n][3 * pix + 1];
        out3[2] = rgb[n][3 * pix + 2];
        return n;
    }
    return -1;
}

/* Per vertex: colour_point with the cameras ranked for the viewpoint. */
int orc_colour(const orc_rig *rig, const uint8_t *const *rgb, const float *viewpoint,
               const R *depth, long long n_verts, const double *verts,
               uint8_t *out_rgb, int32_t *out_cam)
{
    int N = rig->n_cams;
    int *rank = (int *)malloc((size_t)N * sizeof(int));
    size_t *doff = (size_t *)malloc((size_t)N * sizeof(size_t));
    if (!rank || !doff || rank_cameras(rig, viewpoint, rank, doff)) { free(rank); free(doff); return -1; }
    for (long long i = 0; i < n_verts; ++i)
        out_cam[i] = colour_point(rig, rgb, rank, doff, depth, (R)verts[3 * i], (R)verts[3 * i + 1],
                                  (R)verts[3 * i + 2], out_rgb + 3 * i);
    free(rank); free(doff);
    return 0;
}

/* -------------------------------- Sec. II-E: rendering a novel view (step E) */

/* The coloured mesh seen from a virtual camera (matrix Pv, centre Cv, image
 * Wv x Hv).  Visibility: each pixel of the view keeps, among the triangles
 * covering it (the coverage test of the depth images), the one with the
 * smallest squared distance from its centroid to Cv ((dx*dx + dy*dy) +
 * dz*dz), ties to the lower triangle index; out_tri gets its index (-1 for
 * none) and out_d2 that squared distance (+inf for none).  Colour: the
 * pixel takes colour_point of that triangle's centroid with the capture
 * cameras ranked for the viewpoint Cv -- the nearest capture camera that
 * sees the surface point unoccluded, else the next ones (Sec. II-E) -- so
 * the camera is chosen per pixel; out_cam gets it (-1 for none or an empty
 * pixel, whose colour is (0,0,0)).  `depth` holds the capture cameras'
 * depth images (orc_depth). */
int orc_render_view(const orc_rig *rig, const uint8_t *const *rgb, const R *depth, long long n_verts,
                    const double *verts, long long n_tris, const uint32_t *tris, const float *Pv, const float *Cv,
                    int Wv, int Hv, int64_t *out_tri, R *out_d2, uint8_t *out_rgb, int32_t *out_cam)
{
    size_t np = (size_t)Wv * Hv;
    for (size_t i = 0; i < np; ++i) { out_tri[i] = -1; out_d2[i] = (R)INFINITY; }
    R cx = (R)Cv[0], cy = (R)Cv[1], cz = (R)Cv[2];
    for (long long t = 0; t < n_tris; ++t) {
        R X[3], Y[3], Z[3], g[3];
        if (tri_points(n_verts, verts, tris, t, X, Y, Z, g)) return -1;
        tri_cover tc;
        if (!cover_setup(Pv, Wv, Hv, X, Y, Z, &tc)) continue;
        R dx = g[0] - cx, dy = g[1] - cy, dz = g[2] - cz;
        R d2 = (dx * dx + dy * dy) + dz * dz;
        for (int yy = tc.y0; yy <= tc.y1; ++yy) {
            if (!cover_row(&tc, yy)) continue;
            for (int xx = tc.x0; xx <= tc.x1; ++xx) {
                if (!cover_pixel(&tc, xx, yy)) continue;
                size_t i = (size_t)yy * Wv + xx;
                if (d2 < out_d2[i]) { out_d2[i] = d2; out_tri[i] = t; } /* t increases: ties keep the lower */
            }
        }
    }
    int N = rig->n_cams;
    int *rank = (int *)malloc((size_t)N * sizeof(int));
    size_t *doff = (size_t *)malloc((size_t)N * sizeof(size_t));
    if (!rank || !doff || rank_cameras(rig, Cv, rank, doff)) { free(rank); free(doff); return -1; }
    for (size_t i = 0; i < np; ++i) {
        out_cam[i] = -1;
        out_rgb[3 * i] = out_rgb[3 * i + 1] = out_rgb[3 * i + 2] = 0;
        if (out_tri[i] < 0) continue;
        R X[3], Y[3], Z[3], g[3];
        tri_points(n_verts, verts, tris, out_tri[i], X, Y, Z, g);
        out_cam[i] = colour_point(rig, rgb, rank, doff, depth, g[0], g[1], g[2], out_rgb + 3 * i);
    }
    free(rank); free(doff);
    return 0;
}

int orc_real_bytes(void) { return (int)sizeof(R); }
