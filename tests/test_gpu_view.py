"""Parity of the novel view (Sec. II-E, step E) through the C ABI with the
oracle: per pixel the nearest triangle and its squared distance (the key),
the colour and the capture camera chosen, bit for bit."""
import numpy as np
import pytest
import torch

from oracle import Oracle
from synth import default_viewpoint, look_at_camera, make_frame

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    assert torch.cuda.is_available(), "the -m gpu tests need a CUDA GPU"
    from paper_1903_11785_gb300.build import build
    build()


def _view(rig, index, W, H, f, target):
    C = default_viewpoint(rig, index)
    _, _, P = look_at_camera(np.asarray(C, np.float64), np.asarray(target, np.float64), f, W, H)
    return P.astype(np.float32), np.asarray(C, np.float32)


def _compare(rig, fr, P, C, W, H, host=False, in_place=False):
    from paper_1903_11785_gb300 import fvv
    r = fvv.Rig(rig, max_slots=1, host_staging=int(host))
    try:
        r.upload_silhouettes(0, fr.masks.cuda())
        r.reconstruct([0])
        rgb = fr.rgb.pin_memory() if (host or in_place) else fr.rgb.cuda()
        key, out, cam = r.render_view(0, rgb, P, C, W, H, in_place=in_place)
        torch.cuda.synchronize()
        key, out, cam = key.cpu().numpy(), out.cpu().numpy(), cam.cpu().numpy()
    finally:
        r.close()
    o = Oracle(rig)
    ref = o.reconstruct(fr.masks.numpy())
    depth = o.depth(ref.verts, ref.tris)
    tri, d2, orgb, ocam = o.render_view(fr.rgb.numpy(), depth, ref.verts, ref.tris, P, C, W, H)
    k = key.view(np.uint64)
    empty = k == np.uint64(0xFFFFFFFFFFFFFFFF)
    np.testing.assert_array_equal(empty, tri < 0)
    np.testing.assert_array_equal((k[~empty] & np.uint64(0xFFFFFFFF)).astype(np.int64), tri[~empty])
    np.testing.assert_array_equal((k[~empty] >> np.uint64(32)).astype(np.uint32),
                                  d2[~empty].astype(np.float32).view(np.uint32))
    np.testing.assert_array_equal(out, orgb)
    np.testing.assert_array_equal(cam, ocam)
    return (~empty).sum(), ocam


def test_tiny_view_bit_exact():
    rig, fr = make_frame("tiny", 0)
    P, C = _view(rig, 0, 640, 360, 500.0, (0.0, 0.0, 0.9))
    covered, cam = _compare(rig, fr, P, C, 640, 360)
    assert covered > 2000 and (cam >= 0).sum() > 0.9 * covered


def test_tiny_view_host_rgb_and_ragged_size():
    rig, fr = make_frame("tiny", 1)
    P, C = _view(rig, 1, 333, 217, 300.0, (0.0, 0.0, 0.9))
    covered, _ = _compare(rig, fr, P, C, 333, 217, host=True)
    assert covered > 500


def test_view_reads_pinned_host_rgb_in_place():
    rig, fr = make_frame("tiny", 2)
    P, C = _view(rig, 2, 320, 180, 250.0, (0.0, 0.0, 0.9))
    covered, _ = _compare(rig, fr, P, C, 320, 180, in_place=True)
    assert covered > 300


def test_volleyball_view_bit_exact():
    rig, fr = make_frame("volleyball", 0)
    P, C = _view(rig, 0, 1920, 1080, 1800.0, (0.0, 0.0, 1.0))
    covered, cam = _compare(rig, fr, P, C, 1920, 1080)
    assert covered > 20000 and len(np.unique(cam[cam >= 0])) >= 2


def test_view_needs_a_reconstructed_slot():
    from paper_1903_11785_gb300 import fvv
    rig, fr = make_frame("tiny", 0)
    r = fvv.Rig(rig, max_slots=1, host_staging=0)
    try:
        P, C = _view(rig, 0, 64, 64, 50.0, (0.0, 0.0, 0.9))
        with pytest.raises(fvv.FvvError) as e:
            r.render_view(0, fr.rgb.cuda(), P, C, 64, 64)
        assert e.value.status == fvv.FVV_ERR_NOT_READY
        r.upload_silhouettes(0, fr.masks.cuda())
        r.reconstruct([0])
        with pytest.raises(fvv.FvvError):
            r.render_view(0, fr.rgb.cuda(), P, C, 0, 64)
    finally:
        r.close()
