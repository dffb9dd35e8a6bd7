"""fvv_label_components_noalloc: labelling without any device allocation.

Some callers cannot call cudaMalloc -- code running inside a host framework
that owns all device memory, or a real-time loop in which an allocation
(which may synchronise the device) is not allowed.  For them the library
offers a labelling call whose scratch is a static device array inside the
library.  These tests check, through the C ABI, that it gives exactly the
labels and component counts that fvv_reconstruct computes for the same
coarse grid, and that the CPU oracle computes from the same silhouettes, on
two calls in a row (the second call must not see the first's leftovers),
and that grids larger than the static scratch are refused before anything
runs.  (Random and adversarial grids are run through both labellers many
times over in test_gpu_ccl_stress.py.)

The file is named to be collected last, so that a run stopping at the first
failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest
import torch

from synth import make_frame

MAX_VOXELS = 8 * 1024 * 1024


def _lib():
    from paper_1903_11785_gb300.build import build
    build()
    from paper_1903_11785_gb300 import fvv
    return fvv


def _reference(fvv, config, index):
    """Coarse bits, canonical labels and counts as fvv_reconstruct gives them;
    the labels and counts are checked against the oracle's on the way."""
    from oracle import Oracle
    rig, fr = make_frame(config, index)
    ref = Oracle(rig).reconstruct(fr.masks.numpy())
    r = fvv.Rig(rig, max_slots=1, host_staging=0)
    try:
        r.upload_silhouettes(0, fr.masks.cuda())
        r.reconstruct([0])
        c = r.counts(0)
        bits = r.debug(0, fvv.FVV_DEBUG_COARSE_BITS).clone()
        labels = r.debug(0, fvv.FVV_DEBUG_LABELS).clone()
    finally:
        r.close()
    np.testing.assert_array_equal(labels.cpu().numpy().reshape(ref.labels.shape), ref.labels)
    assert (c["n_components"], c["n_rois"]) == (ref.n_components, len(ref.rois))
    return rig, bits, labels, c


def _noalloc(fvv, rig, bits, fill):
    nx, ny, nz = rig.grid_dims()
    labels = torch.full((nx * ny * nz,), fill, dtype=torch.int32, device="cuda")
    counts = torch.full((3,), -1, dtype=torch.int32, device="cuda")
    st = fvv._lib.fvv_label_components_noalloc(C.c_void_p(bits.data_ptr()), nx, ny, nz, rig.t_np, rig.t_nb,
                                               C.c_void_p(labels.data_ptr()), C.c_void_p(counts.data_ptr()),
                                               fvv._stream())
    assert st == fvv.FVV_OK
    torch.cuda.synchronize()
    return labels, counts.cpu().numpy()


@pytest.mark.gpu
def test_noalloc_labels_match_reconstruct_two_calls():
    assert torch.cuda.is_available()
    fvv = _lib()
    # two different frames, one call each, then the first frame again: every
    # call must match the labels fvv_reconstruct produced for its grid
    refs = [_reference(fvv, "volleyball", 0), _reference(fvv, "tiny", 1)]
    for (rig, bits, ref_labels, c), fill in zip(refs + refs[:1], (7, -3, 11)):
        labels, counts = _noalloc(fvv, rig, bits, fill)
        assert torch.equal(labels, ref_labels)
        assert counts.tolist() == [c["n_components"], c["n_rois"], 0]
    assert refs[0][3]["n_rois"] == 13


@pytest.mark.gpu
def test_noalloc_same_grid_twice_in_a_row():
    fvv = _lib()
    rig, bits, ref_labels, c = _reference(fvv, "hd720", 0)
    a, ca = _noalloc(fvv, rig, bits, 5)
    b, cb = _noalloc(fvv, rig, bits, -5)
    assert torch.equal(a, ref_labels) and torch.equal(b, ref_labels)
    assert ca.tolist() == cb.tolist() == [c["n_components"], c["n_rois"], 0]
    assert int(ref_labels.max()) == c["n_rois"] >= 3


def test_noalloc_rejects_grids_beyond_its_scratch():
    """Refused on the host, before any GPU work (runs without a GPU)."""
    fvv = _lib()
    f = fvv._lib.fvv_label_components_noalloc
    dummy = C.c_void_p(256)
    assert f(dummy, 512, 512, 33, 8, 2**31 - 1, dummy, dummy, None) == fvv.FVV_ERR_INVALID_ARG
    assert f(dummy, MAX_VOXELS + 1, 1, 1, 8, 2**31 - 1, dummy, dummy, None) == fvv.FVV_ERR_INVALID_ARG
    assert f(dummy, 0, 10, 10, 8, 2**31 - 1, dummy, dummy, None) == fvv.FVV_ERR_INVALID_ARG
    assert f(None, 10, 10, 10, 8, 2**31 - 1, dummy, dummy, None) == fvv.FVV_ERR_INVALID_ARG
