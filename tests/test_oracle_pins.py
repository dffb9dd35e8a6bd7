"""Pins of the CPU oracle against what the paper and the mathematics fix:
closed forms, library routines, brute force on tiny inputs and invariants.
None of these compares the oracle with itself or with the CUDA path."""
import itertools
import math

import numpy as np
import pytest
from scipy import ndimage

from oracle import Oracle
from oracle.oracle import Roi
from synth import ABSTAIN, STRICT, make_frame, make_rig, render, sphere_scene, inside_any
from tests.helpers import (affine_rig, canonical_labels, closed_oriented, cover_binary32_exact, edge_use,
                           euler_characteristic, fma32, mesh_shells, round32, signed_volume, sphere_rig)


# ------------------------------------------------------------------ Sec. II-B-1

def _box_rig(shift_side=0.0, policy=STRICT):
    # volume [-4,4]^2 x [0,4] at 0.25 m: voxel i has centre -4 + (i + 1/2)/4 and
    # projects to pixel coordinate i + 1/2 in each view (one pixel per voxel).
    top = [[4, 0, 0, 16], [0, 4, 0, 16], [0, 0, 0, 1]]
    front = [[4, 0, 0, 16], [0, 0, 4, 0], [0, 0, 0, 1]]
    side = [[0, 4, 0, 16 + shift_side], [0, 0, 4, 0], [0, 0, 0, 1]]
    return affine_rig([top, front, side], 32, 32, (-4, -4, 0), (4, 4, 4), 0.25, oob_policy=policy)


def _box_masks(xr, yr, zr, shift_side=0):
    m = np.zeros((3, 32, 32), np.uint8)
    m[0, yr[0]:yr[1], xr[0]:xr[1]] = 1
    m[1, zr[0]:zr[1], xr[0]:xr[1]] = 1
    lo, hi = max(yr[0] + shift_side, 0), max(yr[1] + shift_side, 0)
    m[2, zr[0]:zr[1], lo:hi] = 1
    return m


def test_orthographic_box_is_the_box():
    """Three axis-aligned orthographic views of a box whose faces lie on pixel
    edges and between voxel centres: the hull is exactly the box."""
    xr, yr, zr = (9, 21), (5, 30), (3, 11)
    o = Oracle(_box_rig())
    occ, tests = o.coarse(_box_masks(xr, yr, zr))
    z, y, x = np.meshgrid(np.arange(16), np.arange(32), np.arange(32), indexing="ij")
    inx, iny, inz = (x >= xr[0]) & (x < xr[1]), (y >= yr[0]) & (y < yr[1]), (z >= zr[0]) & (z < zr[1])
    assert occ.shape == (16, 32, 32)
    np.testing.assert_array_equal(occ, (inx & iny & inz).astype(np.uint8))
    # early exit in camera order: 1 test if the top view rejects, 2 if the front does, else 3
    v0, v1 = inx & iny, inx & inz
    expect = np.where(~v0, 1, np.where(~v1, 2, 3)).sum()
    assert tests == expect


def test_pixel_floor_is_exact():
    """The pixel of a projection is the floor of the exact quotient of two
    binary32 numbers.  The oracle forms it in double; checked here against
    exact rational arithmetic on quotients placed within a few ulps of
    integers (where a rounded binary32 quotient would round up to the
    integer) and on random ones, so the double floor equals the exact one."""
    from fractions import Fraction
    rng = np.random.default_rng(5)
    cases = []
    for _ in range(4000):
        k = int(rng.integers(0, 4096))
        w = np.float32(rng.uniform(0.5, 80.0))
        x = np.float32(k * np.float64(w))
        for d in range(-3, 4):
            cases.append((np.nextafter(x, np.float32(np.inf) if d > 0 else np.float32(-np.inf)) if d else x, w))
            x = cases[-1][0]
    for _ in range(4000):
        cases.append((np.float32(rng.uniform(-100, 5000) * rng.uniform(1, 60)), np.float32(rng.uniform(0.1, 60))))
    hits = 0
    for x, w in cases:
        exact = Fraction(float(x)) / Fraction(float(w))
        fl = exact.numerator // exact.denominator
        assert np.floor(np.float64(x) / np.float64(w)) == fl
        q32 = np.float32(x) / np.float32(w)
        hits += int(np.floor(q32) != fl)
    assert hits > 0          # binary32 rounding does cross integers on these inputs


def test_fma32_is_correctly_rounded():
    """The numpy fused multiply-add used by the projection pins, against
    exact rational arithmetic: random operands, sums that cancel, and sums
    whose binary64 rounding lands exactly halfway between two binary32
    numbers (where rounding twice would be wrong)."""
    from fractions import Fraction
    rng = np.random.default_rng(6)
    n = 3000
    a = (rng.standard_normal(n) * 10.0 ** rng.integers(-3, 4, n)).astype(np.float32)
    b = (rng.standard_normal(n) * 10.0 ** rng.integers(-3, 4, n)).astype(np.float32)
    c = (rng.standard_normal(n) * 10.0 ** rng.integers(-3, 4, n)).astype(np.float32)
    c[: n // 3] = (-(a[: n // 3].astype(np.float64) * b[: n // 3])).astype(np.float32)   # cancellation
    # a b = +-(2^-24 - 2^-60) and c = 2^q (1 + k 2^-23): the exact sum lies 2^-60 2^q
    # off a binary32 halfway point, which binary64 cannot hold
    k = np.arange(64)
    q = rng.integers(-4, 5, 64)
    sg = np.where(k % 4 < 2, 1.0, -1.0)
    a = np.concatenate([a, (2.0 ** (-12 + q) * (1 + 2.0 ** -18)).astype(np.float32)])
    b = np.concatenate([b, (sg * 2.0 ** -12 * (1 - 2.0 ** -18)).astype(np.float32)])
    c = np.concatenate([c, (2.0 ** q * (1 + k * 2.0 ** -23)).astype(np.float32)])
    got = fma32(a, b, c)
    twice = 0
    for x, y, z, g in zip(a, b, c, got):
        exact = Fraction(float(x)) * Fraction(float(y)) + Fraction(float(z))
        lo = np.float32(float(exact))                  # within one binary32 step of the exact value
        cands = [np.nextafter(lo, np.float32(-np.inf)), lo, np.nextafter(lo, np.float32(np.inf))]
        dist = [abs(Fraction(float(v)) - exact) for v in cands]
        near = [v for v, d in zip(cands, dist) if d == min(dist)]
        want = near[0] if len(near) == 1 else [v for v in near if (v.view(np.uint32) & 1) == 0][0]
        assert g == want, (x, y, z, g, want)
        twice += np.float32(np.float64(x) * np.float64(y) + np.float64(z)) != want
    assert twice > 0         # rounding the binary64 sum again is wrong on some of these


def test_round32_is_binary32_rounding():
    """The rational emulation's rounding (used to pin the depth coverage in
    its edge band) equals IEEE binary32 conversion of binary64 values (one
    rounding, so numpy's conversion is exact there), including halfway cases
    (ties to even) and subnormals."""
    from fractions import Fraction
    rng = np.random.default_rng(5)
    x = rng.normal(0, 1, 4000) * np.exp2(rng.integers(-140, 100, 4000).astype(np.float64))
    for v in x:
        assert round32(Fraction(float(v))) == Fraction(float(np.float32(v)))
    one = Fraction(1)
    ulp = Fraction(1, 2 ** 23)
    assert round32(one + ulp / 2) == one                      # tie, even below
    assert round32(one + 3 * ulp / 2) == one + 2 * ulp        # tie, even above
    assert round32(one + ulp / 2 + Fraction(1, 2 ** 80)) == one + ulp
    assert round32(-(one + 3 * ulp / 2)) == -(one + 2 * ulp)
    assert round32(Fraction(3, 2 ** 150)) == Fraction(4, 2 ** 150)   # 1.5 subnormal quanta: tie to even
    assert round32(Fraction(3, 2 ** 151)) == Fraction(2, 2 ** 150)   # 0.75 quanta: up to the smallest
    assert round32(Fraction(1, 3)) == Fraction(float(np.float32(1 / 3)))


def test_projection_is_fused_binary32():
    """Each row of the projection is ((p3 + p2 Z) + p1 Y) + p0 X in three
    fused multiply-adds (binary32), and the pixel is the floor of the exact
    quotient.  Checked through the oracle's vote on a checkerboard
    silhouette at points on rays through pixel corners (where one rounding
    decides the pixel); the unfused order puts some of them in other pixels."""
    from dataclasses import replace
    from fractions import Fraction
    from tests.helpers import project32
    base = make_rig("judo")
    rig = replace(base, P=base.P[:1], centre=base.centre[:1], width=base.width[:1], height=base.height[:1])
    W, H = int(rig.width[0]), int(rig.height[0])
    rng = np.random.default_rng(12)
    m = 6000
    uv = np.stack([rng.integers(0, W + 1, m).astype(float), rng.integers(0, H + 1, m).astype(float)], 1)
    d = (base.R64[0].T @ (np.linalg.inv(base.K64[0]) @ np.concatenate([uv, np.ones((m, 1))], 1).T)).T
    pts = (base.C64[0] + rng.uniform(2.0, 30.0, (m, 1)) * d).astype(np.float32)
    yy, xx = np.mgrid[0:H, 0:W]
    masks = ((xx + yy) % 2 == 0).astype(np.uint8)[None]
    on, _ = Oracle(rig).points_on(masks, pts.astype(np.float64))

    def vote(xp, wp, yp):
        out = np.zeros(len(pts), np.uint8)
        for i in range(len(pts)):
            if not wp[i] > 0:
                continue
            px = math.floor(Fraction(float(xp[i])) / Fraction(float(wp[i])))
            py = math.floor(Fraction(float(yp[i])) / Fraction(float(wp[i])))
            out[i] = 0 <= px < W and 0 <= py < H and (px + py) % 2 == 0
        return out
    xp, yp, wp = project32(rig.P[0], pts[:, 0], pts[:, 1], pts[:, 2])
    np.testing.assert_array_equal(np.asarray(on, np.uint8), vote(xp, wp, yp))
    P = rig.P[0].astype(np.float32)
    X, Y, Z = pts[:, 0], pts[:, 1], pts[:, 2]
    ux, uy, uw = (((P[r, 0] * X + P[r, 1] * Y) + P[r, 2] * Z) + P[r, 3] for r in range(3))
    assert int((vote(ux, uw, uy) != np.asarray(on, np.uint8)).sum()) > 0


def test_out_of_image_policy():
    """A view shifted so part of the volume falls outside its image: STRICT
    carves that part, ABSTAIN lets the other views decide."""
    xr, yr, zr = (4, 28), (2, 30), (1, 15)
    shift = -10   # side view pixel = y + 1/2 - 10: y < 10 falls left of the image
    strict, _ = Oracle(_box_rig(shift, STRICT)).coarse(_box_masks(xr, yr, zr, shift))
    abst, _ = Oracle(_box_rig(shift, ABSTAIN)).coarse(_box_masks(xr, yr, zr, shift))
    z, y, x = np.meshgrid(np.arange(16), np.arange(32), np.arange(32), indexing="ij")
    box = (x >= xr[0]) & (x < xr[1]) & (y >= yr[0]) & (y < yr[1]) & (z >= zr[0]) & (z < zr[1])
    np.testing.assert_array_equal(strict, (box & (y >= 10)).astype(np.uint8))
    np.testing.assert_array_equal(abst, box.astype(np.uint8))


@pytest.mark.parametrize("policy", [STRICT, ABSTAIN])
def test_hull_contains_shape_conservative(policy):
    """With conservative silhouettes (a pixel is foreground iff its square meets
    the exact image ellipse), every voxel whose centre lies inside the shape
    shrunk by 1 mm is occupied, in the coarse grid and in every fine grid."""
    rig = make_rig("tiny")
    rig.oob_policy = policy
    objs = __import__("synth").scene_objects("tiny", 0)
    fr = render(rig, objs, conservative=True, with_rgb=False)
    o = Oracle(rig)
    res = o.reconstruct(fr.masks.numpy())
    nx, ny, nz = res.dims
    s = rig.coarse_m
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cen = np.stack([np.float32(rig.vol_min[0]) + (xx + np.float32(0.5)) * np.float32(s),
                    np.float32(rig.vol_min[1]) + (yy + np.float32(0.5)) * np.float32(s),
                    np.float32(rig.vol_min[2]) + (zz + np.float32(0.5)) * np.float32(s)], -1).reshape(-1, 3)
    inside = inside_any(objs, cen.astype(np.float64), shrink=1e-3).reshape(nz, ny, nx)
    assert inside.sum() > 100
    assert np.all(res.coarse[inside] == 1)
    assert len(res.rois) == 1
    r, occ = res.rois[0], res.fine[0]
    fz, fy, fx = occ.shape
    zz, yy, xx = np.meshgrid(np.arange(fz), np.arange(fy), np.arange(fx), indexing="ij")
    f = rig.fine_m
    cen = np.stack([r.forigin[0] + (xx + 0.5) * f, r.forigin[1] + (yy + 0.5) * f,
                    r.forigin[2] + (zz + 0.5) * f], -1).reshape(-1, 3)
    inside = inside_any(objs, cen, shrink=1e-3).reshape(occ.shape)
    assert inside.sum() > 10000
    assert np.all(occ[inside] == 1)


def test_flip_count_fp32_vs_fp64():
    """Report (and bound) the voxels whose binary32 occupancy differs from binary64."""
    rig, fr = make_frame("tiny", 0)
    m = fr.masks.numpy()
    a, _ = Oracle(rig, "f32").coarse(m)
    b, _ = Oracle(rig, "f64").coarse(m)
    flips = int((a != b).sum())
    print(f"coarse flips fp32 vs fp64 (tiny): {flips} of {a.size}")
    assert flips <= a.size // 1000


# ------------------------------------------------------------------ Sec. II-B-2

def _scipy_labels(occ):
    lab, n = ndimage.label(occ, structure=np.ones((3, 3, 3), int))
    return canonical_labels(lab), n


@pytest.mark.parametrize("density", [0.05, 0.1, 0.2, 0.5])
def test_ccl_matches_scipy_26(density):
    """26-connected labels equal scipy.ndimage.label with the full 3x3x3
    structure, renumbered by smallest linear index; BFS and union-find agree."""
    rng = np.random.default_rng(int(density * 1000))
    occ = (rng.random((17, 23, 41)) < density).astype(np.uint8)
    o = Oracle(make_rig("tiny"))
    ref, n = _scipy_labels(occ)
    bfs, cb = o.ccl_bfs(occ)
    uf, cu = o.ccl_uf(occ)
    assert cb == cu == n
    np.testing.assert_array_equal(bfs, ref)
    np.testing.assert_array_equal(uf, ref)


def test_ccl_structured_cases():
    occ = np.zeros((8, 9, 10), np.uint8)
    occ[0, 0, 0] = occ[1, 1, 1] = 1            # corner-only contact: one component
    occ[7, 8, 9] = 1                            # grid corner, isolated
    occ[3, 0, 5] = occ[3, 0, 7] = 1             # a gap of one voxel: two components
    occ[5, 4, 0] = occ[5, 5, 9] = 0
    for t in range(30):                         # a spiral crossing the grid
        a = t * 0.4
        occ[2 + (t // 15), 4 + int(round(3 * math.sin(a))), int(round(4.5 + 4 * math.cos(a)))] = 1
    o = Oracle(make_rig("tiny"))
    ref, n = _scipy_labels(occ)
    bfs, cb = o.ccl_bfs(occ)
    assert cb == n
    np.testing.assert_array_equal(bfs, ref)
    assert bfs[0, 0, 0] == bfs[1, 1, 1] == 1


def test_filter_eq1_bounds_and_roi():
    """Eq. (1), prose reading: keep iff T_np <= count <= T_nb (both bounds
    inclusive); the ROI is the inclusive box grown by one voxel, clamped; the
    fine grid covers it in whole fine voxels."""
    rig = make_rig("tiny")
    rig.t_np, rig.t_nb = 8, 20
    nx, ny, nz = 30, 20, 12
    occ = np.zeros((nz, ny, nx), np.uint8)
    # size: block origin (z,y,x); each fills a 7x7 layer in raster order
    sizes = {7: (3, 2, 1), 8: (5, 11, 2), 20: (0, 0, nx - 7), 21: (nz - 1, 12, 12)}
    for size, (z, y, x) in sizes.items():
        for i in range(size):
            occ[z, y + i // 7, x + i % 7] = 1
    o = Oracle(rig)
    raw, n = o.ccl_bfs(occ)
    counts = np.bincount(raw.ravel())[1:]
    assert sorted(counts.tolist()) == [7, 8, 20, 21]
    lab, rois = o.filter(raw, n)
    kept = [c for c in range(1, n + 1) if 8 <= counts[c - 1] <= 20]
    assert len(rois) == 2 and lab.max() == 2
    for k, c in enumerate(kept, start=1):
        zz, yy, xx = np.nonzero(raw == c)
        np.testing.assert_array_equal(lab == k, raw == c)
        r = rois[k - 1]
        assert r.count == counts[c - 1]
        assert r.cmin == (xx.min(), yy.min(), zz.min()) and r.cmax == (xx.max(), yy.max(), zz.max())
        dims = (nx, ny, nz)
        for a in range(3):
            assert r.gmin[a] == max(r.cmin[a] - 1, 0)
            assert r.gmax[a] == min(r.cmax[a] + 1, dims[a] - 1)
            assert r.fdim[a] == 5 * (r.gmax[a] - r.gmin[a] + 1)     # 5 cm / 1 cm, exactly
            assert abs(r.forigin[a] - (rig.vol_min[a] + r.gmin[a] * rig.coarse_m)) < 1e-6
    assert np.all(lab[(raw > 0) & (lab == 0)] == 0)


def test_fine_dims_non_integer_ratio():
    rig = make_rig("tiny")
    rig.fine_m = 0.02                         # 5 cm / 2 cm = 2.5: ceil
    occ = np.zeros((6, 6, 6), np.uint8)
    occ[2, 2, 2] = occ[2, 2, 3] = 1
    rig.t_np = 1
    o = Oracle(rig)
    raw, n = o.ccl_bfs(occ)
    _, rois = o.filter(raw, n)
    r = rois[0]
    assert (r.gmax[0] - r.gmin[0] + 1, r.gmax[1] - r.gmin[1] + 1) == (4, 3)
    assert r.fdim[0] == 10 and r.fdim[1] == math.ceil(3 * 2.5) == 8


# ------------------------------------------------------------------ Sec. II-C

def _cube_edge_corners(e):
    a, u, w = e >> 2, e & 1, (e >> 1) & 1
    c0 = [2 * u + 4 * w, u + 4 * w, u + 2 * w][a]
    return c0, c0 + (1 << a)


def _corner_xyz(c):
    return np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1], float)


def _edge_mid(e):
    c0, c1 = _cube_edge_corners(e)
    return (_corner_xyz(c0) + _corner_xyz(c1)) / 2


def test_mc_every_case_closes_and_covers_bipolar_edges():
    for cs in range(256):
        tris = Oracle.mc_cell(cs)
        on = [(cs >> c) & 1 for c in range(8)]
        bip = {e for e in range(12) if on[_cube_edge_corners(e)[0]] != on[_cube_edge_corners(e)[1]]}
        used = {e for t in tris for e in t}
        assert used == bip, cs
        # every polygon edge is used once each way inside the cell or lies on a face
        if tris:
            assert len(tris) <= 12


@pytest.mark.parametrize("corner", range(8))
def test_mc_single_corner_orientation(corner):
    """One ON corner: one triangle through its three edges, normal pointing
    away from the ON corner (outward); one OFF corner: normal toward it."""
    for cs, sign in ((1 << corner, 1.0), (255 ^ (1 << corner), -1.0)):
        tris = Oracle.mc_cell(cs)
        assert len(tris) == 1
        p = [_edge_mid(e) for e in tris[0]]
        n = np.cross(p[1] - p[0], p[2] - p[0])
        g = (p[0] + p[1] + p[2]) / 3
        assert sign * float(n @ (g - _corner_xyz(corner))) > 0


def _cell_edges(cell_min, cs):
    """Triangles of a cell as triples of global edge ids (min-end sample, axis)."""
    out = []
    for t in Oracle.mc_cell(cs):
        tri = []
        for e in t:
            c0, _ = _cube_edge_corners(e)
            tri.append((tuple(int(v) for v in np.asarray(cell_min) + _corner_xyz(c0)), e >> 2))
        out.append(tuple(tri))
    return out


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_mc_two_cell_brute_force(axis):
    """All 2^12 states of two cells sharing a face: no edge is used more than
    twice, shared edges are used once in each direction, and edges used once
    lie on the outer boundary of the two-cell block."""
    shape = [2, 2, 2]
    shape[axis] = 3
    samples = list(itertools.product(range(shape[0]), range(shape[1]), range(shape[2])))
    cache = {cs: None for cs in range(256)}
    for state in range(1 << 12):
        on = {s: (state >> i) & 1 for i, s in enumerate(samples)}
        tris = []
        for k in range(2):
            mn = [0, 0, 0]
            mn[axis] = k
            cs = 0
            for c in range(8):
                p = (mn[0] + (c & 1), mn[1] + ((c >> 1) & 1), mn[2] + ((c >> 2) & 1))
                cs |= on[p] << c
            tris += _cell_edges(mn, cs)
        use = {}
        for t in tris:
            for i in range(3):
                a, b = t[i], t[(i + 1) % 3]
                key = (min(a, b), max(a, b))
                d = use.setdefault(key, [0, 0])
                d[0 if a < b else 1] += 1
        for (a, b), (f, r) in use.items():
            assert f + r <= 2, (axis, state)
            if f + r == 2:
                assert f == 1 and r == 1, (axis, state)
            else:
                # both endpoints on one outer face of the block
                ok = False
                for ax in range(3):
                    for val in (0, shape[ax] - 1):
                        if all(e[1] != ax and e[0][ax] == val for e in (a, b)):
                            ok = True
                assert ok, (axis, state, a, b)
    del cache


def _single_roi(fdim, forigin=(0.0, 0.0, 0.0)):
    return Roi((0, 0, 0), (0, 0, 0), (0, 0, 0), (0, 0, 0), tuple(fdim), np.array(forigin, float), 1)


def test_mc_octahedron_volume_and_closed_random_grids():
    """One ON sample meshed at edge midpoints (0 steps) is the octahedron of
    volume s^3/6 with outward normals; random grids mesh closed and oriented."""
    rig = make_rig("tiny")
    rig.bisect_steps = 0
    o = Oracle(rig)
    masks = np.zeros((rig.n_cams, 360, 640), np.uint8)
    occ = np.zeros((1, 1, 1), np.uint8)
    occ[0, 0, 0] = 1
    v, k, a, b, t, tests = o.mesh_one(masks, _single_roi((1, 1, 1)), occ)
    assert len(v) == 6 and len(t) == 8 and tests == 0
    s = rig.fine_m
    assert abs(signed_volume(v, t) - s ** 3 / 6) < 1e-12
    assert closed_oriented(t) and euler_characteristic(t) == 2
    rng = np.random.default_rng(7)
    for dens in (0.1, 0.3, 0.5, 0.7, 0.9):
        occ = (rng.random((5, 6, 7)) < dens).astype(np.uint8)
        v, k, a, b, t, _ = o.mesh_one(masks, _single_roi((7, 6, 5)), occ)
        assert closed_oriented(t), dens
        assert np.all(np.diff(k.astype(np.int64)) > 0)      # vertices sorted by edge key
        assert signed_volume(v, t) > 0


def test_bisection_zero_steps_is_edge_midpoint():
    rig, fr = make_frame("tiny", 0)
    rig.bisect_steps = 0
    res = Oracle(rig).reconstruct(fr.masks.numpy())
    assert res.tests_bisect == 0
    np.testing.assert_allclose(res.verts, (res.vert_a + res.vert_b) / 2, atol=1e-7)
    d = np.abs(res.vert_a - res.vert_b)
    assert np.allclose(np.sort(d, axis=1)[:, 2], rig.fine_m, atol=1e-6)
    assert np.allclose(np.sort(d, axis=1)[:, :2], 0.0, atol=0)


def test_bisection_bracket_invariant():
    """After k steps the bracket [a, b] has length edge/2^k, lies on the grid
    edge, a is occupied and b is not (unless b is still the padding sample),
    and the vertex is its midpoint: within one step of the hull boundary."""
    rig, fr = make_frame("tiny", 0)
    o = Oracle(rig)
    m = fr.masks.numpy()
    res = o.reconstruct(m)
    k = rig.bisect_steps
    h = rig.fine_m / 2 ** k
    d = np.abs(res.vert_a - res.vert_b)
    # binary32 midpoints round each end by at most half an ulp of the coordinate
    ulp = np.spacing(np.abs(res.vert_a).max(axis=1).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(d.max(axis=1) - h) <= 2 * k * ulp)
    assert np.all(np.sort(d, axis=1)[:, :2] == 0)
    on_a, _ = o.points_on(m, res.vert_a)
    on_b, _ = o.points_on(m, res.vert_b)
    assert np.all(on_a == 1)
    forced = on_b == 1
    # a forced vertex is one whose OFF end is the padding layer and stayed there
    assert forced.mean() < 0.01
    np.testing.assert_allclose(res.verts, (res.vert_a + res.vert_b) / 2, atol=1e-6)


def test_sphere_mesh_closed_genus0_and_radius():
    """A sphere seen by a ring of cameras with conservative silhouettes (so the
    hull contains the sphere): one closed, outward shell with Euler
    characteristic 2; every vertex is at radius >= R - edge/2^k, since its
    bracket's OFF end lies outside the hull; the enclosed volume agrees with
    the occupied fine-voxel volume."""
    rig = sphere_rig()
    R0 = 0.4
    fr = render(rig, sphere_scene((0.0, 0.0, 1.0), R0), conservative=True, with_rgb=False)
    res = Oracle(rig).reconstruct(fr.masks.numpy())
    assert len(res.rois) == 1
    t = res.tris
    assert closed_oriented(t)
    assert mesh_shells(len(res.verts), t) == 1
    assert euler_characteristic(t) == 2
    rad = np.linalg.norm(res.verts - np.array([0, 0, 1.0]), axis=1)
    assert rad.min() >= R0 - rig.fine_m / 2 ** rig.bisect_steps - 1e-5
    vol = signed_volume(res.verts, t)
    von = res.fine[0].sum() * rig.fine_m ** 3
    assert vol > 4 / 3 * math.pi * R0 ** 3 * 0.99
    assert abs(vol - von) / von < 0.05


def test_scene_mesh_closed_and_tests_bounded():
    rig, fr = make_frame("tiny", 0)
    res = Oracle(rig).reconstruct(fr.masks.numpy())
    assert closed_oriented(res.tris)
    nvox = int(np.prod(res.dims))
    assert nvox <= res.tests_coarse <= rig.n_cams * nvox
    nf = sum(f.size for f in res.fine)
    assert nf <= res.tests_fine <= rig.n_cams * nf
    assert res.tests_bisect <= rig.n_cams * rig.bisect_steps * len(res.verts)
    for r, (a, b) in enumerate(zip(res.roi_vert_offset[:-1], res.roi_vert_offset[1:])):
        tt = res.tris[res.roi_tri_offset[r]:res.roi_tri_offset[r + 1]]
        assert tt.min() >= a and tt.max() < b


# ------------------------------------------------------------------ Sec. II-D-1

def _brute_depth(P, C, W, H, verts, tris):
    """Per-pixel loop over all triangles, in float64 (coverage by barycentric
    sign with inclusive edges)."""
    D = np.full((H, W), np.inf)
    hv = np.concatenate([verts, np.ones((len(verts), 1))], 1) @ np.asarray(P, np.float64).T
    for t in tris:
        if np.any(hv[t, 2] <= 0):
            continue
        uv = hv[t, :2] / hv[t, 2:3]
        area = (uv[1, 0] - uv[0, 0]) * (uv[2, 1] - uv[0, 1]) - (uv[1, 1] - uv[0, 1]) * (uv[2, 0] - uv[0, 0])
        if area == 0:
            continue
        g = verts[t].mean(0)
        d = np.linalg.norm(g - C)
        for py in range(H):
            for px in range(W):
                p = np.array([px + 0.5, py + 0.5])
                s = []
                for i in range(3):
                    a, b = uv[i], uv[(i + 1) % 3]
                    s.append((b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0]))
                if all(x >= 0 for x in s) or all(x <= 0 for x in s):
                    D[py, px] = min(D[py, px], d)
    return D


def test_depth_matches_brute_force():
    """Eq. (4) on a small affine view where every edge function is exact:
    inclusive edges, both windings, overlaps keep the minimum, degenerate
    triangles are skipped, triangles leaving the image are clipped."""
    P = [[8, 0, 0, 8], [0, 8, 0, 8], [0, 0, 0, 1]]       # u = 8x + 8, v = 8y + 8
    C = np.array([0.25, -0.5, 3.0])
    rig = affine_rig([P], 24, 20, (-1, -1, 0), (1, 1, 1), 0.25, centres=[C])
    q = 1 / 16
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0.5],            # t0
                      [0.5, 0.25, 1], [-0.5, 0.75, 1], [0.25, 1.5, 1.2],   # t1 (other winding)
                      [-1, -1, 0], [2, 0, 0], [0.5, 0.5, 0],        # t2 leaves the image
                      [0, 0, 0], [1, 1, 0], [0.5, 0.5, 0],          # t3 degenerate (collinear)
                      [3 * q, 5 * q, 2], [19 * q, 5 * q, 2], [3 * q, 21 * q, 2]], float)  # t4: edges through centres
    tris = np.arange(15, dtype=np.uint32).reshape(5, 3)
    tris[1] = tris[1][::-1]
    D = Oracle(rig).depth(verts, tris)[0]
    ref = _brute_depth(P, C, 24, 20, verts, tris)
    np.testing.assert_array_equal(np.isfinite(D), np.isfinite(ref))
    np.testing.assert_allclose(D[np.isfinite(D)], ref[np.isfinite(ref)], rtol=1e-6)
    assert np.isfinite(D).sum() > 50


def _perspective_coverage(rig, n, verts, tris, band=1e-3):
    """Predicted coverage of the union of `tris` in camera n: at pixel centres
    farther than `band` px from every edge line of a triangle, float64
    image-plane geometry of its projection (exact far beyond its rounding
    error); at the others, the reading itself evaluated exactly
    (cover_binary32_exact).  Returns (coverage, number of (triangle, pixel)
    decisions taken by each route, band pixels covered)."""
    W, H = int(rig.width[n]), int(rig.height[n])
    P = rig.P[n].astype(np.float64)
    hv = np.concatenate([verts, np.ones((len(verts), 1))], 1) @ P.T
    uv = hv[:, :2] / hv[:, 2:3]
    cover = np.zeros((H, W), bool)
    n_geo = n_band = band_in = 0
    for t in tris:
        q = uv[t]
        x0, x1 = int(max(0, np.floor(q[:, 0].min()) - 2)), int(min(W - 1, np.ceil(q[:, 0].max()) + 2))
        y0, y1 = int(max(0, np.floor(q[:, 1].min()) - 2)), int(min(H - 1, np.ceil(q[:, 1].max()) + 2))
        if x0 > x1 or y0 > y1:
            continue
        ys, xs = np.mgrid[y0:y1 + 1, x0:x1 + 1]
        px, py = xs + 0.5, ys + 0.5
        e, dist = [], []
        for i in range(3):
            a, b = q[i], q[(i + 1) % 3]
            ei = (b[0] - a[0]) * (py - a[1]) - (b[1] - a[1]) * (px - a[0])
            e.append(ei)
            dist.append(np.abs(ei) / max(np.hypot(*(b - a)), 1e-12))
        inside = ((e[0] >= 0) & (e[1] >= 0) & (e[2] >= 0)) | ((e[0] <= 0) & (e[1] <= 0) & (e[2] <= 0))
        near = np.min(np.stack(dist), 0) < band
        n_geo += int((~near).sum())
        for yy, xx in zip(*np.nonzero(near)):
            n_band += 1
            c = cover_binary32_exact(rig.P[n], verts[t, 0], verts[t, 1], verts[t, 2], x0 + xx, y0 + yy)
            inside[yy, xx] = c
            band_in += int(c)
        cover[y0:y1 + 1, x0:x1 + 1] |= inside
    return cover, n_geo, n_band, band_in


def test_depth_perspective_matches_exact_geometry():
    """Perspective view, random triangles of a few pixels: the oracle's
    coverage equals exact image-plane geometry at every pixel centre farther
    than 1e-3 px from a triangle edge, and, at the centres nearer than that,
    the binary32 homogeneous test of the reading evaluated exactly with
    rationals (no pixel is exempt)."""
    rig = make_rig("tiny")
    rng = np.random.default_rng(3)
    n = 0
    base = np.array([0.2, -0.3, 1.0])
    tris = []
    verts = []
    for t in range(300):
        c = base + rng.normal(0, 0.5, 3)
        for k in range(3):
            verts.append(c + rng.normal(0, 0.02, 3))
        tris.append([3 * t, 3 * t + 1, 3 * t + 2])
    verts = np.array(verts, np.float32).astype(np.float64)
    tris = np.array(tris, np.uint32)
    D = Oracle(rig).depth(verts, tris)[n]
    cover, n_geo, n_band, _ = _perspective_coverage(rig, n, verts, tris)
    assert cover.sum() > 500 and n_geo > 5000
    np.testing.assert_array_equal(np.isfinite(D), cover)


def _on_centres(rig, n, pix, depth):
    """World points (binary32 values, as float64) that camera n sees at the
    image points `pix` (k, 2) at distance `depth` along each ray."""
    K, R, C = rig.K64[n], rig.R64[n], rig.C64[n]
    pts = []
    for (u, v), d in zip(pix, depth):
        ray = R.T @ np.linalg.solve(K, np.array([u, v, 1.0]))
        pts.append(C + d * ray / np.linalg.norm(ray))
    return np.array(pts, np.float32).astype(np.float64)


def test_depth_edge_band_matches_exact_binary32_reading():
    """Triangles whose edges run through rows, columns and diagonals of pixel
    centres (vertices projected within about 1e-5 px of pixel centres), so
    that hundreds of centres lie within 1e-3 px of an edge and rounding
    decides them: the oracle's coverage of every pixel equals the reading
    evaluated exactly with rationals there, and exact geometry elsewhere."""
    import dataclasses
    rig0 = make_rig("tiny")
    n = 0
    rig = dataclasses.replace(rig0, P=rig0.P[:1], centre=rig0.centre[:1], width=rig0.width[:1],
                              height=rig0.height[:1])
    rng = np.random.default_rng(11)
    verts, tris = [], []
    shapes = [((0, 0), (12, 0), (0, 7)), ((0, 0), (9, 9), (0, 9)), ((0, 0), (9, 9), (9, 0)),
              ((0, 0), (10, 5), (0, 5)), ((0, 0), (6, 0), (6, 6)), ((3, 0), (0, 4), (6, 4)),
              ((0, 0), (1, 0), (0, 1)), ((0, 0), (8, 3), (2, 7))]
    for k in range(40):
        u0, v0 = int(rng.integers(40, 580)), int(rng.integers(30, 320))
        a, b, c = shapes[k % len(shapes)]
        if k % 2:
            a, b, c = a, c, b                  # both windings
        pix = [(u0 + x + 0.5, v0 + y + 0.5) for x, y in (a, b, c)]
        depth = 6.0 + rng.uniform(-0.5, 0.5, 3) * (k % 3 != 0)
        verts.extend(_on_centres(rig, n, pix, depth))
        tris.append([3 * k, 3 * k + 1, 3 * k + 2])
    verts = np.array(verts)
    tris = np.array(tris, np.uint32)
    got = np.zeros((int(rig.height[0]), int(rig.width[0])), bool)
    cover = np.zeros_like(got)
    n_band = band_in = 0
    o = Oracle(rig)
    for t in tris:                              # one triangle at a time: no overlap hides a decision
        got |= np.isfinite(o.depth(verts, t[None])[0])
        c, _, nb, bi = _perspective_coverage(rig, 0, verts, t[None])
        cover |= c
        n_band += nb
        band_in += bi
    assert n_band > 200 and 50 < band_in < n_band - 50
    np.testing.assert_array_equal(got, cover)


def test_depth_perspective_behind_camera_skipped():
    rig = make_rig("tiny")
    C = rig.C64[0]
    fwd = rig.R64[0][2]
    verts = np.array([C + fwd * 2 + [0.1, 0, 0], C + fwd * 2 + [0, 0.1, 0], C - fwd * 1.0])
    D = Oracle(rig).depth(verts, np.array([[0, 1, 2]], np.uint32))
    assert not np.isfinite(D[0]).any()


# ------------------------------------------------------------- Sec. II-D-2, II-E

def test_colour_rank_occlusion_and_threshold():
    """Two affine cameras with hand-made depth images: the nearest camera to
    the viewpoint is taken unless |v - C| - depth > T_v (equality visible)."""
    P0 = [[8, 0, 0, 8], [0, 8, 0, 8], [0, 0, 0, 1]]
    P1 = [[8, 0, 0, 9], [0, 8, 0, 8], [0, 0, 0, 1]]   # shifted one pixel
    C0, C1 = np.array([0.0, 0.0, 4.0]), np.array([0.0, 0.0, -4.0])
    rig = affine_rig([P0, P1], 16, 16, (-1, -1, -1), (1, 1, 1), 0.25, centres=[C0, C1], t_v=0.5)
    verts = np.array([[0.5, 0.5, 0.0], [0.25, 0.5, 0.0], [0.5, 0.25, 0.0], [5.0, 5.0, 0.0]])
    rgb = [np.zeros((16, 16, 3), np.uint8), np.zeros((16, 16, 3), np.uint8)]
    rgb[0][..., 0] = 10
    rgb[1][..., 0] = 20
    rgb[0][12, 12] = (11, 12, 13)
    dist = np.sqrt(np.float32(16.5))   # |(0.5,0.5,0) - (0,0,4)|; 16.5 is exact in binary32
    d0 = np.full((16, 16), np.inf, np.float32)
    d1 = np.full((16, 16), np.inf, np.float32)
    d0[12, 12] = np.float32(dist) - np.float32(0.5)     # exactly at the threshold: visible
    d0[12, 10] = 1.0                                    # vertex 1 occluded in camera 0
    d1[12, 11] = 1.0                                    # ... and in camera 1
    o = Oracle(rig)
    col, cam = o.colour(rgb, np.array([0.0, 0.0, 10.0], np.float32), [d0, d1], verts)
    assert cam.tolist() == [0, -1, 0, -1]
    assert col[0].tolist() == [11, 12, 13] and col[1].tolist() == [0, 0, 0]
    # viewpoint near camera 1: it is ranked first
    col, cam = o.colour(rgb, np.array([0.0, 0.0, -10.0], np.float32), [d0, d1], verts)
    assert cam.tolist() == [1, -1, 1, -1]
    assert col[0].tolist() == [20, 0, 0]


def test_colour_scene_matches_surface_colour():
    """Flat-coloured ellipsoids: most vertices take the colour of the nearest
    ellipsoid surface (the rest sit where parts meet or behind noise)."""
    rig, fr = make_frame("tiny", 0)
    o = Oracle(rig)
    res = o.reconstruct(fr.masks.numpy())
    D = o.depth(res.verts, res.tris)
    col, cam = o.colour(fr.rgb.numpy(), fr.viewpoint, D, res.verts)
    assert np.all(cam >= 0)
    dist = []
    for e in fr.ellipsoids:
        q = (res.verts - e.centre) @ e.rot / e.axes[None, :]
        dist.append(np.abs(np.sqrt((q * q).sum(1)) - 1) * e.axes.min())
    near = np.argmin(np.stack(dist, 1), 1)
    want = np.array([fr.ellipsoids[i].colour for i in near], np.uint8)
    frac = float(np.mean(np.all(col == want, axis=1)))
    print(f"vertices coloured as their nearest ellipsoid: {frac:.3f}")
    assert frac > 0.6
