"""Pins of the oracle's form of the paper's own surface rule (Sec. II-C,
Eqs. (2)-(3)): per camera a Bresenham walk along the projected grid edge
from the ON end, P_i = the last silhouette pixel before the first one that
is not, lambda_i = |c(P_i) - p_on| / |p_off - p_on| (c = pixel centre), and
lambda = the minimum over the cameras.

The expected values are worked out by hand from the geometry (closed forms),
or from the pixels nearest the ideal line, which is the path Bresenham's
algorithm takes when no pixel centre lies exactly half-way."""
import numpy as np
import pytest

from oracle import Oracle
from tests.helpers import affine_rig, closed_oriented, sphere_rig
from synth import sphere_scene, render

# u = X, v = Y: world x/y are pixel coordinates directly
IDENT = [[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1]]


def _rig(views, W=32, H=16, **kw):
    return affine_rig(views, W, H, (0, 0, -1), (W, H, 1), 1.0, surface_rule=1, **kw)


def _mask(W, H, fg):
    yy, xx = np.mgrid[0:H, 0:W]
    return fg(xx, yy).astype(np.uint8)


def test_horizontal_walk_closed_form():
    rig = _rig([IDENT])
    m = _mask(32, 16, lambda x, y: x <= 12)
    lam, lam_n, tests = Oracle(rig).edge_lambda([m], [[10.3, 2.5, 0]], [[14.3, 2.5, 0]])
    # pixels 10, 11, 12 are foreground, 13 is not: P = 12, centre 12.5
    assert abs(lam[0] - (12.5 - 10.3) / 4.0) < 1e-6
    assert tests == 4


def _ideal_line(x0, y0, x1, y1):
    """Pixels nearest to the ideal line from (x0,y0) to (x1,y1), one per step
    of the longer axis (no half-way ties in the cases used)."""
    n = max(abs(x1 - x0), abs(y1 - y0))
    out = []
    for k in range(n + 1):
        t = k / n
        out.append((int(round(x0 + t * (x1 - x0))), int(round(y0 + t * (y1 - y0)))))
    return out


@pytest.mark.parametrize("a,b", [
    ((2.2, 1.7), (9.6, 5.1)),     # shallow, +x +y
    ((9.6, 5.1), (2.2, 1.7)),     # shallow, -x -y
    ((3.4, 1.2), (5.8, 12.9)),    # steep, +y
    ((20.7, 13.3), (11.1, 9.4)),  # shallow, -x -y, other slope
    ((6.5, 14.6), (9.2, 3.3)),    # steep, -y
])
def test_diagonal_walk_matches_nearest_pixel_path(a, b):
    W, H = 32, 16
    A = (int(np.floor(a[0])), int(np.floor(a[1])))
    B = (int(np.floor(b[0])), int(np.floor(b[1])))
    path = _ideal_line(*A, *B)
    for k in range(1, len(path) - 1):
        rig = _rig([IDENT], W, H)
        # foreground: exactly the first k pixels of the path
        m = np.zeros((H, W), np.uint8)
        for (x, y) in path[:k]:
            m[y, x] = 1
        lam, _, tests = Oracle(rig).edge_lambda([m], [[a[0], a[1], 0]], [[b[0], b[1], 0]])
        cx, cy = path[k - 1][0] + 0.5, path[k - 1][1] + 0.5
        want = min(1.0, np.hypot(cx - a[0], cy - a[1]) / np.hypot(b[0] - a[0], b[1] - a[1]))
        assert abs(lam[0] - want) < 2e-6, (k, lam[0], want)
        assert tests == k + 1


def test_minimum_over_cameras_and_unbounding_cameras():
    # camera 0 cuts at x <= 12, camera 1 sees the whole edge, camera 2 cuts at x <= 11
    rig = _rig([IDENT, IDENT, IDENT])
    ms = [_mask(32, 16, lambda x, y: x <= 12), np.ones((16, 32), np.uint8), _mask(32, 16, lambda x, y: x <= 11)]
    lam, lam_n, _ = Oracle(rig).edge_lambda(ms, [[10.3, 2.5, 0]], [[14.3, 2.5, 0]])
    assert abs(lam_n[0, 0] - 2.2 / 4) < 1e-6
    assert lam_n[0, 1] == 1.0                      # the walk reaches B
    assert abs(lam_n[0, 2] - 1.2 / 4) < 1e-6
    assert lam[0] == lam_n[0].min()


def test_image_border_and_far_end():
    rig = _rig([IDENT], W=16, H=4)
    m = np.ones((4, 16), np.uint8)
    lam, _, _ = Oracle(rig).edge_lambda([m], [[14.5, 1.5, 0]], [[20.5, 1.5, 0]])
    # pixels 14 and 15 are in the image, 16 is not: P = 15, centre 15.5
    assert abs(lam[0] - 1.0 / 6.0) < 1e-6
    # an end point very far outside: the walk still stops at the border
    lam, _, tests = Oracle(rig).edge_lambda([m], [[14.5, 1.5, 0]], [[1.0e6, 1.5, 0]])
    assert abs(lam[0] - 1.0 / (1.0e6 - 14.5)) < 1e-9
    assert tests == 3


def test_end_behind_camera_bounds_nothing():
    # perspective: w' = Z; the OFF end lies behind the camera
    P = [[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]]
    rig = _rig([P])
    m = _mask(32, 16, lambda x, y: x <= 3)
    lam, lam_n, _ = Oracle(rig).edge_lambda([m], [[2.5, 2.5, 1.0]], [[2.5, 2.5, -1.0]])
    assert lam[0] == 1.0


def test_degenerate_edge_projection():
    # both ends project to the same image point: no information, lambda 1
    P = [[0, 0, 1, 5.5], [0, 1, 0, 0], [0, 0, 0, 1]]  # u ignores x
    rig = _rig([P])
    m = np.ones((16, 32), np.uint8)
    lam, _, _ = Oracle(rig).edge_lambda([m], [[0.2, 2.5, 0.0]], [[0.8, 2.5, 0.0]])
    assert lam[0] == 1.0


def test_mesh_with_paper_rule_is_closed_and_near_the_sphere():
    rig = sphere_rig()
    rig.surface_rule = 1
    c, R = np.array([0.0, 0.0, 1.0]), 0.4
    fr = render(rig, sphere_scene(c, R), flip_prob=0.0, conservative=True, with_rgb=False)
    res = Oracle(rig).reconstruct(fr.masks.numpy())
    assert len(res.verts) > 0 and closed_oriented(res.tris)
    # each vertex lies on its grid edge between the ON and the OFF end
    a, b, v = res.vert_a.astype(np.float64), res.vert_b.astype(np.float64), res.verts.astype(np.float64)
    ab = b - a
    t = np.einsum("ij,ij->i", v - a, ab) / np.einsum("ij,ij->i", ab, ab)
    assert np.all(t >= -1e-5) and np.all(t <= 1 + 1e-5)
    assert np.allclose(a + t[:, None] * ab, v, atol=1e-5)
    # the ON end is inside the conservative hull of the sphere, so every
    # vertex is at least R - (one fine step) from the centre
    r = np.linalg.norm(v - c, axis=1)
    assert r.min() >= R - rig.fine_m * 1.01
