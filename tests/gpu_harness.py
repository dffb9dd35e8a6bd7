"""Run frames through the C ABI and through the oracle, and compare every
output of the path element by element (used by the -m gpu tests)."""
import numpy as np
import torch

from oracle import Oracle


def unpack_rows(words: np.ndarray, shape_rows, width):
    """uint32 rows -> bits (little-endian bit order), cropped to `width`."""
    b = np.unpackbits(np.ascontiguousarray(words, np.uint32).view(np.uint8), bitorder="little")
    return b.reshape(*shape_rows, -1)[..., :width]


def run_gpu(rig, frames, host=False, caps=None, slots=None, batch=True, rgb_in_place=False, masks_in_place=False,
            upload_batch=False, tuning=None):
    """Upload (all slots in one call when upload_batch), reconstruct (all
    slots in one call when batch) and colour, with the launch shapes
    `tuning` (as Rig.set_tuning takes them) if given.  Returns one dict of
    numpy outputs per frame."""
    from paper_1903_11785_gb300 import fvv
    caps = dict(caps or {})
    n = len(frames)
    slots = list(slots) if slots is not None else list(range(n))
    r = fvv.Rig(rig, max_slots=max(slots) + 1, host_staging=int(host), **caps)
    try:
        if tuning is not None:
            r.set_tuning(tuning)
        ms = [fr.masks.pin_memory() if (host or masks_in_place) else fr.masks.cuda() for fr in frames]
        if upload_batch:
            r.upload_silhouettes_batch(slots, ms, in_place=masks_in_place)
        else:
            for s, m in zip(slots, ms):
                r.upload_silhouettes(s, m, in_place=masks_in_place)
        if batch:
            r.reconstruct(slots)
        else:
            for s in slots:
                r.reconstruct([s])
        rgbs = [fr.rgb.pin_memory() if (host or rgb_in_place) else fr.rgb.cuda() for fr in frames]
        vps = np.stack([fr.viewpoint for fr in frames])
        r.colour(slots, rgbs, vps, in_place=rgb_in_place)
        torch.cuda.synchronize()
        return [fetch_outputs(r, s) for s in slots]
    finally:
        r.close()


def fetch_outputs(r, s):
    """Every output of slot s of rig r (an fvv.Rig), as numpy arrays."""
    from paper_1903_11785_gb300 import fvv
    c = r.counts(s, allow_capacity=True)
    o = dict(counts=c)
    if c["flags"] == 0:
        res = r.results(s)
        o.update(rois=res["rois"], verts=res["verts"].cpu().numpy(), tris=res["tris"].cpu().numpy(),
                 rgb=res["rgb"].cpu().numpy(), cam=res["cam"].cpu().numpy())
        o["sil"] = r.debug(s, fvv.FVV_DEBUG_SIL_BITS).cpu().numpy().view(np.uint32)
        o["coarse"] = r.debug(s, fvv.FVV_DEBUG_COARSE_BITS).cpu().numpy().view(np.uint32)
        o["labels"] = r.debug(s, fvv.FVV_DEBUG_LABELS).cpu().numpy()
        o["fine"] = r.debug(s, fvv.FVV_DEBUG_FINE_BITS).cpu().numpy().view(np.uint32)
        o["depth"] = r.debug(s, fvv.FVV_DEBUG_DEPTH).cpu().numpy()
    return o


def run_oracle(rig, fr):
    o = Oracle(rig)
    ref = o.reconstruct(fr.masks.cpu().numpy())
    depth = o.depth(ref.verts, ref.tris)
    col, cam = o.colour(fr.rgb.cpu().numpy(), fr.viewpoint, depth, ref.verts)
    return ref, depth, col, cam


def compare(rig, fr, g, oracle_out=None):
    """Assert the GPU outputs `g` equal the oracle's, bit for bit."""
    ref, depth, col, cam = oracle_out or run_oracle(rig, fr)
    c = g["counts"]
    assert c["flags"] == 0
    # a0: packed silhouettes
    masks = fr.masks.cpu().numpy()
    N, H, W = masks.shape
    Wq = (W + 31) // 32
    sil = unpack_rows(g["sil"], (N, H), W)
    np.testing.assert_array_equal(sil, (masks != 0).astype(np.uint8))
    # a1: coarse occupancy and tests
    nx, ny, nz = ref.dims
    coarse = unpack_rows(g["coarse"], (nz, ny), nx)
    np.testing.assert_array_equal(coarse, ref.coarse)
    assert c["n_coarse_on"] == int(ref.coarse.sum())
    assert c["tests_coarse"] == ref.tests_coarse
    # a2-a4: labels, components, ROIs
    np.testing.assert_array_equal(g["labels"].reshape(nz, ny, nx), ref.labels)
    assert c["n_components"] == ref.n_components
    assert c["n_rois"] == len(ref.rois)
    for k, (gr, orr) in enumerate(zip(g["rois"], ref.rois)):
        assert gr["label"] == k + 1
        assert tuple(gr["cmin"]) == orr.cmin and tuple(gr["cmax"]) == orr.cmax
        assert tuple(gr["gmin"]) == orr.gmin and tuple(gr["gmax"]) == orr.gmax
        assert tuple(gr["fdim"]) == orr.fdim and gr["count"] == orr.count
        np.testing.assert_array_equal(np.asarray(gr["forigin"], np.float32).astype(np.float64), orr.forigin)
        assert gr["vert_offset"] == ref.roi_vert_offset[k] and gr["n_verts"] == (
            ref.roi_vert_offset[k + 1] - ref.roi_vert_offset[k])
        assert gr["tri_offset"] == ref.roi_tri_offset[k] and gr["n_tris"] == (
            ref.roi_tri_offset[k + 1] - ref.roi_tri_offset[k])
    # a5: fine occupancy (padded grids, pad samples unoccupied)
    off = 0
    for orr, focc in zip(ref.rois, ref.fine):
        fx, fy, fz = orr.fdim
        nxw = (fx + 2 + 31) // 32
        nw = nxw * (fy + 2) * (fz + 2)
        bits = unpack_rows(g["fine"][off:off + nw], (fz + 2, fy + 2), fx + 2)
        off += nw
        np.testing.assert_array_equal(bits[1:-1, 1:-1, 1:-1], focc)
        assert bits.sum() == focc.sum()
    assert off == len(g["fine"]) == c["n_fine_words"]
    assert c["tests_fine"] == ref.tests_fine
    # a6-a8: mesh topology bit-exact, vertices bit-exact (tolerance 1e-5 m allowed; none needed)
    assert c["n_verts"] == len(ref.verts) and c["n_tris"] == len(ref.tris)
    np.testing.assert_array_equal(g["tris"].astype(np.uint32), ref.tris)
    gv = g["verts"].astype(np.float64)
    assert np.abs(gv - ref.verts).max(initial=0.0) <= 1e-5
    np.testing.assert_array_equal(gv, ref.verts)
    assert c["tests_bisect"] == ref.tests_bisect
    # a9: depth images
    o = 0
    for n in range(N):
        d = g["depth"][o:o + H * W].reshape(H, W)
        o += H * W
        np.testing.assert_array_equal(d, depth[n])
    # a10: colours and chosen cameras
    np.testing.assert_array_equal(g["rgb"], col)
    np.testing.assert_array_equal(g["cam"], cam)
    return ref


# ---- digests: every output of a frame in the oracle's layouts, hashed, so
# that many frames can be compared without moving the arrays between processes

def _h(a) -> str:
    import hashlib
    a = np.ascontiguousarray(a)
    return hashlib.blake2b(a.view(np.uint8).reshape(-1).tobytes(), digest_size=16).hexdigest() + str(a.dtype) + \
        str(a.shape)


def oracle_digest(rig, masks, rgb, viewpoint) -> dict:
    """The oracle's outputs for one frame (numpy inputs), hashed."""
    o = Oracle(rig)
    ref = o.reconstruct(masks)
    depth = o.depth(ref.verts, ref.tris)
    col, cam = o.colour(rgb, viewpoint, depth, ref.verts)
    rois = [(r.cmin, r.cmax, r.gmin, r.gmax, r.fdim, r.count,
             tuple(np.asarray(r.forigin, np.float32).view(np.uint32).tolist())) for r in ref.rois]
    fine = np.concatenate([f.ravel() for f in ref.fine]) if ref.fine else np.zeros(0, np.uint8)
    return dict(counts=(ref.n_components, len(ref.rois), int(ref.coarse.sum()), ref.tests_coarse, ref.tests_fine,
                        ref.tests_bisect, len(ref.verts), len(ref.tris)),
                coarse=_h(ref.coarse.astype(np.uint8)), labels=_h(ref.labels.astype(np.int32)), rois=rois,
                fine=_h(fine.astype(np.uint8)), verts=_h(ref.verts.astype(np.float32)), tris=_h(ref.tris.astype(np.uint32)),
                depth=_h(np.concatenate([np.asarray(d, np.float32).ravel() for d in depth])),
                rgb=_h(col.astype(np.uint8)), cam=_h(cam.astype(np.int32)))


def gpu_digest(rig, g) -> dict:
    """The same digest of the GPU outputs `g` (fetch_outputs), converted to
    the oracle's layouts."""
    c = g["counts"]
    nx, ny, nz = rig.grid_dims()
    rois = [(tuple(r["cmin"]), tuple(r["cmax"]), tuple(r["gmin"]), tuple(r["gmax"]), tuple(r["fdim"]), r["count"],
             tuple(np.asarray(r["forigin"], np.float32).view(np.uint32).tolist())) for r in g["rois"]]
    fine, off = [], 0
    for r in g["rois"]:
        fx, fy, fz = r["fdim"]
        nw = ((fx + 2 + 31) // 32) * (fy + 2) * (fz + 2)
        bits = unpack_rows(g["fine"][off:off + nw], (fz + 2, fy + 2), fx + 2)
        off += nw
        fine.append(bits[1:-1, 1:-1, 1:-1].ravel())
    fine = np.concatenate(fine) if fine else np.zeros(0, np.uint8)
    return dict(counts=(c["n_components"], c["n_rois"], c["n_coarse_on"], c["tests_coarse"], c["tests_fine"],
                        c["tests_bisect"], c["n_verts"], c["n_tris"]),
                coarse=_h(unpack_rows(g["coarse"], (nz, ny), nx).astype(np.uint8)),
                labels=_h(g["labels"].reshape(nz, ny, nx).astype(np.int32)), rois=rois, fine=_h(fine.astype(np.uint8)),
                verts=_h(g["verts"].astype(np.float32)), tris=_h(g["tris"].astype(np.uint32)),
                depth=_h(g["depth"].astype(np.float32)), rgb=_h(g["rgb"].astype(np.uint8)),
                cam=_h(g["cam"].astype(np.int32)))


def _oracle_digest_job(job):
    """Worker: digest of frame i of the arrays saved at `path` (spawned pool)."""
    import os
    import sys
    path, config, i = job
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from synth import make_rig
    rig = make_rig(config)
    masks = np.load(os.path.join(path, "masks.npy"), mmap_mode="r")
    rgb = np.load(os.path.join(path, "rgb.npy"), mmap_mode="r")
    vps = np.load(os.path.join(path, "vps.npy"))
    return i, oracle_digest(rig, np.array(masks[i]), np.array(rgb[i]), vps[i])
