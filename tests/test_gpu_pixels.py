"""The projection used by every hull test (Sec. II-B-1), checked through the
fvv_debug_pixels hook against numpy: x' = ((p3 + p2 Z) + p1 Y) + p0 X (and
y', w') in three binary32 fused multiply-adds, pixel = floor of the exact
quotient x'/w'.  Points are
placed on rays through pixel corners, so many quotients fall within an ulp
or two of an integer, where the kernel's approximate reciprocal must be
corrected by its residual test."""
import ctypes as C

import numpy as np
import pytest
import torch

from synth import make_rig
from tests.helpers import project32

pytestmark = pytest.mark.gpu


def _numpy_pixels(P, W, H, pts):
    row = project32(P, pts[:, 0], pts[:, 1], pts[:, 2])
    xp, yp, wp = (a.astype(np.float64) for a in row)
    with np.errstate(divide="ignore", invalid="ignore"):
        u = np.floor(xp / wp)       # exact floor: see test_oracle_pins.test_pixel_floor_is_exact
        v = np.floor(yp / wp)
    ok = (wp > 0) & (u >= 0) & (u < W) & (v >= 0) & (v < H)
    return np.where(ok, u, -1).astype(np.int64), np.where(ok, v, -1).astype(np.int64)


@pytest.mark.parametrize("config", ["tiny", "judo"])
def test_pixel_index_matches_binary32_definition(config):
    from paper_1903_11785_gb300 import fvv
    rig = make_rig(config)
    rng = np.random.default_rng(11)
    W, H = int(rig.width[0]), int(rig.height[0])
    pts = []
    for n in range(rig.n_cams):
        Kinv = np.linalg.inv(rig.K64[n])
        # rays through pixel corners (integer u, v), and through random pixel positions
        m = 20000
        uv = np.stack([rng.integers(-2, W + 3, m).astype(float), rng.integers(-2, H + 3, m).astype(float)], 1)
        uv[m // 2:] += rng.random((m - m // 2, 2))
        d = (rig.R64[n].T @ (Kinv @ np.concatenate([uv, np.ones((m, 1))], 1).T)).T
        t = rng.uniform(1.0, 40.0, (m, 1))
        pts.append(rig.C64[n] + t * d)
    pts.append(rng.uniform(-50, 50, (20000, 3)))          # anywhere, including behind cameras
    pts = np.concatenate(pts).astype(np.float32)
    r = fvv.Rig(rig, max_slots=1, host_staging=0, max_fine_words=1 << 12, max_verts=1 << 12, max_tris=1 << 12)
    try:
        dp = torch.from_numpy(pts).cuda()
        px = torch.empty(len(pts), dtype=torch.int32, device="cuda")
        py = torch.empty(len(pts), dtype=torch.int32, device="cuda")
        near = 0
        for n in range(rig.n_cams):
            fvv._check(fvv._lib.fvv_debug_pixels(r.ptr, n, C.c_longlong(len(pts)), C.c_void_p(dp.data_ptr()),
                                                  C.c_void_p(px.data_ptr()), C.c_void_p(py.data_ptr()),
                                                  fvv._stream()), r.ptr)
            torch.cuda.synchronize()
            ru, rv = _numpy_pixels(rig.P[n], W, H, pts)
            np.testing.assert_array_equal(px.cpu().numpy(), ru)
            np.testing.assert_array_equal(py.cpu().numpy(), rv)
            # how many quotients sat within 1e-3 px of an integer (the slow path)
            xp, _, wp = project32(rig.P[n], pts[:, 0], pts[:, 1], pts[:, 2])
            with np.errstate(divide="ignore", invalid="ignore"):
                q = xp.astype(np.float64) / wp
            fr = np.abs(q - np.round(q))
            near += int(np.sum((wp > 0) & (fr < 1e-3) & (q > 0) & (q < W)))
        assert near > 1000
    finally:
        r.close()
