"""Pins of the oracle's novel view (Sec. II-E, step E): per pixel the nearest
covering triangle (squared centroid distance to the virtual camera, ties to
the lower index), coloured at that triangle's centroid by the nearest
capture camera that sees it unoccluded, else the next ones.  The expected
images are worked out from the geometry by hand."""
import numpy as np

from oracle import Oracle
from synth import make_frame
from tests.helpers import affine_rig

IDENT = [[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1]]


def _grid_quad(x0, x1, y0, y1, z, base=0):
    """Unit squares [x,x+1]x[y,y+1] at height z, two triangles each."""
    verts, tris = [], []
    idx = {}
    for y in range(y0, y1 + 1):
        for x in range(x0, x1 + 1):
            idx[x, y] = base + len(verts)
            verts.append((x, y, z))
    for y in range(y0, y1):
        for x in range(x0, x1):
            a, b, c, d = idx[x, y], idx[x + 1, y], idx[x + 1, y + 1], idx[x, y + 1]
            tris += [(a, b, c), (a, c, d)]
    return verts, tris


def _rig(views, centres, W=32, H=16):
    return affine_rig(views, W, H, (0, 0, -50), (W, H, 50), 1.0, centres=centres, t_v=0.5)


def test_nearest_triangle_wins_and_ties_keep_the_lower_index():
    rig = _rig([IDENT], [(0, 0, -100)])
    # triangle 0 far (z = 5), triangle 1 near (z = -5), overlapping; 2 and 3 identical
    verts = [(2, 2, 5), (20, 2, 5), (2, 12, 5), (8, 4, -5), (28, 4, -5), (8, 14, -5),
             (2, 13, 0), (6, 13, 0), (2, 15, 0)]
    tris = [(0, 1, 2), (3, 4, 5), (6, 7, 8), (6, 7, 8)]
    o = Oracle(rig)
    W, H = 32, 16
    masks = [np.zeros((H, W), np.uint8)]
    rgb = [np.zeros((H, W, 3), np.uint8)]
    depth = o.depth(np.array(verts, np.float64), np.array(tris, np.uint32))
    Pv = np.array(IDENT, np.float32)
    tri, d2, out, cam = o.render_view(rgb, depth, verts, tris, Pv, (10.0, 8.0, -30.0), W, H)

    def inside(p, a, b, c):
        def s(u, v, w):
            return (v[0] - u[0]) * (w[1] - u[1]) - (v[1] - u[1]) * (w[0] - u[0])
        d = [s(a, b, p), s(b, c, p), s(c, a, p)]
        return all(x >= 0 for x in d) or all(x <= 0 for x in d)
    want = np.full((H, W), -1)
    for y in range(H):
        for x in range(W):
            p = (x + 0.5, y + 0.5)
            t0 = inside(p, *[verts[i][:2] for i in tris[0]])
            t1 = inside(p, *[verts[i][:2] for i in tris[1]])
            t2 = inside(p, *[verts[i][:2] for i in tris[2]])
            # distances to (10, 8, -30): triangle 1 (z = -5) is nearer than 0 (z = 5)
            want[y, x] = 1 if t1 else (0 if t0 else (2 if t2 else -1))
    np.testing.assert_array_equal(tri, want)
    assert (want == 2).any() and (want == 1).any() and (want == 0).any()
    assert np.all(np.isinf(d2[want < 0])) and np.all(np.isfinite(d2[want >= 0]))


def test_colour_falls_back_to_the_next_camera_where_the_nearest_is_occluded():
    W, H = 32, 16
    # capture camera 0 looks straight (u = X), camera 1 obliquely (u = X + Z/2)
    P0 = IDENT
    P1 = [[1, 0, 0.5, 0], [0, 1, 0, 0], [0, 0, 0, 1]]
    rig = _rig([P0, P1], [(10, 8, -20), (10, 8, -40)], W, H)
    qv, qt = _grid_quad(2, 18, 2, 14, 0.0)
    # occluder: a 4 x 16 m wall at z = -10, in front of the quad for camera 0
    ov = [(12, 0, -10), (16, 0, -10), (16, 16, -10), (12, 16, -10)]
    b = len(qv)
    verts = np.array(qv + ov, np.float64)
    tris = np.array(qt + [(b, b + 1, b + 2), (b, b + 2, b + 3)], np.uint32)
    o = Oracle(rig)
    depth = o.depth(verts, tris)
    red = np.zeros((H, W, 3), np.uint8)
    red[..., 0] = 255
    green = np.zeros((H, W, 3), np.uint8)
    green[..., 1] = 255
    # the virtual camera sees the quad straight on and the wall off to the side
    Pv = np.array([[1, 0, -2, 0], [0, 1, 0, 0], [0, 0, 0, 1]], np.float32)
    tri, d2, out, cam = o.render_view([red, green], depth, verts, tris, Pv, (10.0, 8.0, -25.0), W, H)
    for y in range(H):
        for x in range(W):
            on_quad = 2 <= x <= 17 and 2 <= y <= 13
            if not on_quad:
                assert tri[y, x] == -1 and cam[y, x] == -1 and not out[y, x].any(), (x, y)
                continue
            assert 0 <= tri[y, x] < len(qt)
            if 12 <= x <= 15:      # hidden from camera 0 by the wall, seen by camera 1
                assert cam[y, x] == 1 and tuple(out[y, x]) == (0, 255, 0), (x, y)
            else:
                assert cam[y, x] == 0 and tuple(out[y, x]) == (255, 0, 0), (x, y)


def test_view_from_a_capture_camera_reproduces_its_depth_image():
    """Virtual camera = capture camera n at its own centre: the view's nearest
    squared distance is the square of Eq. (4)'s depth at every pixel."""
    rig, fr = make_frame("tiny", 0)
    o = Oracle(rig)
    ref = o.reconstruct(fr.masks.numpy())
    depth = o.depth(ref.verts, ref.tris)
    n = 3
    W, H = int(rig.width[n]), int(rig.height[n])
    tri, d2, out, cam = o.render_view(fr.rgb.numpy(), depth, ref.verts, ref.tris, rig.P[n], rig.centre[n], W, H)
    got = np.sqrt(d2.astype(np.float32))
    np.testing.assert_array_equal(np.isinf(got), np.isinf(depth[n]))
    fin = np.isfinite(got)
    assert fin.sum() > 1000
    np.testing.assert_array_equal(got[fin], depth[n][fin].astype(np.float32))
    # the nearest capture camera is camera n itself (distance 0)
    assert (cam[fin] == n).mean() > 0.9
