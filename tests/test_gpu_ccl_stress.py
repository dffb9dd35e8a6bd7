"""Stress parity of the 26-connected labelling, the component boxes and the
Eq. (1) filter (Sec. II-B-2) against the oracle, on grids that no set of
silhouettes produces.

Both labellers of the library are run, through the C ABI, on the same
seeded grids: the one inside fvv_reconstruct (fed a given grid through the
fvv_debug_label_coarse hook, which then runs exactly the labelling, box,
filter and ROI kernels of a reconstruction) and the allocation-free
fvv_label_components_noalloc.  Their labels, component counts and ROI
tables must equal the oracle's BFS flood fill followed by its filter, bit
for bit.

The grids are i.i.d. random occupancy at densities 0.05, 0.1 (near the
26-neighbour site percolation threshold), 0.2 and 0.5, and single long
components (a serpentine chain, staircases crossing word boundaries, stacked
spirals, corner-only contacts) that build deep union-find trees, up to the
largest grid the allocation-free labeller takes.  Union-find with atomics is
timing dependent, so every grid is labelled many times in a row: a race that
loses a parent update shows up as a voxel missing from its component's label,
count or box in some of the repetitions."""
import ctypes as C
import dataclasses

import numpy as np
import pytest
import torch

from oracle import Oracle
from synth import make_rig
from synth.grids import (corner_contacts_grid, pack_words, random_grid, serpentine_grid, spiral_grid,
                         staircase_grid)

pytestmark = pytest.mark.gpu

REPEATS = 20
SMALL = (96, 64, 40)          # 245,760 voxels, three words per row
RAGGED = (70, 40, 33)         # rows end in a partial word
LARGE = (300, 300, 75)        # 6.75 M voxels: the judo-shaped coarse grid


@pytest.fixture(scope="module")
def fvv():
    assert torch.cuda.is_available(), "the -m gpu tests need a CUDA GPU"
    from paper_1903_11785_gb300.build import build
    build()
    from paper_1903_11785_gb300 import fvv as mod
    return mod


def grid_rig(dims, t_np=8, t_nb=2**31 - 1):
    """The tiny scene's cameras over a volume whose 5 cm grid has `dims`
    (nx, ny, nz); the fine step is 2.5 cm so that ROI sizing is exercised."""
    nx, ny, nz = dims
    rig = dataclasses.replace(make_rig("tiny"), vol_min=(-0.025 * nx, -0.025 * ny, 0.0),
                              vol_max=(0.025 * nx, 0.025 * ny, 0.05 * nz), coarse_m=0.05, fine_m=0.025,
                              t_np=t_np, t_nb=t_nb)
    assert rig.grid_dims() == tuple(dims)
    return rig


def oracle_labels(rig, occ):
    o = Oracle(rig)
    raw, n = o.ccl_bfs(occ)
    lab, rois = o.filter(raw, n, max_rois=4096)
    return lab, n, rois


def fine_words_needed(rois):
    return sum(((r.fdim[0] + 2 + 31) // 32) * (r.fdim[1] + 2) * (r.fdim[2] + 2) for r in rois)


def make_lib_rig(fvv, rig, rois):
    fw = min(1 << 26, max(1 << 16, fine_words_needed(rois)))
    return fvv.Rig(rig, max_slots=1, host_staging=0, max_rois=4096, max_fine_words=fw, max_verts=1024,
                   max_tris=1024)


def check_reconstruct_labeller(fvv, r, words, ref_lab, n_comp, rois, n_on):
    r.debug_label_coarse(0, words)
    c = r.counts(0)
    assert c["flags"] == 0
    assert c["n_components"] == n_comp
    assert c["n_rois"] == len(rois)
    assert c["n_coarse_on"] == n_on
    lab = r.debug(0, fvv.FVV_DEBUG_LABELS).cpu().numpy().reshape(ref_lab.shape)
    np.testing.assert_array_equal(lab, ref_lab)
    got = r.results(0)["rois"]
    assert len(got) == len(rois)
    for k, (g, o) in enumerate(zip(got, rois)):
        assert g["label"] == k + 1
        assert (tuple(g["cmin"]), tuple(g["cmax"]), g["count"]) == (o.cmin, o.cmax, o.count)
        assert (tuple(g["gmin"]), tuple(g["gmax"]), tuple(g["fdim"])) == (o.gmin, o.gmax, o.fdim)
        np.testing.assert_array_equal(np.asarray(g["forigin"], np.float32).astype(np.float64), o.forigin)


def run_noalloc(fvv, words, dims, t_np, t_nb, fill):
    nx, ny, nz = dims
    labels = torch.full((nx * ny * nz,), fill, dtype=torch.int32, device="cuda")
    counts = torch.full((3,), -1, dtype=torch.int32, device="cuda")
    st = fvv._lib.fvv_label_components_noalloc(C.c_void_p(words.data_ptr()), nx, ny, nz, t_np, t_nb,
                                               C.c_void_p(labels.data_ptr()), C.c_void_p(counts.data_ptr()),
                                               fvv._stream())
    assert st == fvv.FVV_OK
    torch.cuda.synchronize()
    return labels.cpu().numpy().reshape(nz, ny, nx), counts.cpu().numpy().tolist()


def grid_words(occ, junk_past_nx=False):
    w = pack_words(occ)
    nz, ny, nx = occ.shape
    if junk_past_nx and nx % 32:
        # bits past nx in each row's last word must be ignored by both labellers
        last = np.arange((nx + 31) // 32 - 1, w.size, (nx + 31) // 32)
        w[last] |= np.uint32(0xFFFFFFFF) << np.uint32(nx % 32)
    return torch.from_numpy(w.view(np.int32)).cuda()


CASES = [
    ("random", SMALL, 0.05, 3, 2**31 - 1),
    ("random", SMALL, 0.1, 3, 400),
    ("random", SMALL, 0.2, 8, 2**31 - 1),
    ("random", SMALL, 0.5, 8, 2**31 - 1),
    ("random", RAGGED, 0.1, 2, 50),
    ("random", LARGE, 0.2, 8, 2**31 - 1),
    ("random", LARGE, 0.5, 8, 2**31 - 1),
    ("serpentine", SMALL, None, 8, 2**31 - 1),
    ("staircase", SMALL, None, 8, 2**31 - 1),
    ("spiral", SMALL, None, 8, 2**31 - 1),
    ("corners", SMALL, None, 8, 2**31 - 1),
    ("serpentine", LARGE, None, 8, 2**31 - 1),
    ("staircase", LARGE, None, 8, 2**31 - 1),
    ("spiral", LARGE, None, 8, 2**31 - 1),
]
MAKERS = {"serpentine": serpentine_grid, "staircase": staircase_grid, "spiral": spiral_grid,
          "corners": corner_contacts_grid}


def _case_id(c):
    kind, dims, dens = c[:3]
    return f"{kind}-{'x'.join(map(str, dims))}" + (f"-{dens}" if dens is not None else "")


@pytest.mark.parametrize("case", CASES, ids=[_case_id(c) for c in CASES])
def test_labels_boxes_filter_match_oracle_repeatedly(fvv, case):
    kind, dims, dens, t_np, t_nb = case
    occ = random_grid(dims, dens, seed=len(kind)) if kind == "random" else MAKERS[kind](dims)
    rig = grid_rig(dims, t_np, t_nb)
    ref_lab, n_comp, rois = oracle_labels(rig, occ)
    assert 0 < n_comp <= 8192 and len(rois) <= 4096
    words = grid_words(occ, junk_past_nx=True)
    n_on = int(occ.sum())
    r = make_lib_rig(fvv, rig, rois)
    try:
        for rep in range(REPEATS):
            check_reconstruct_labeller(fvv, r, words, ref_lab, n_comp, rois, n_on)
            lab, counts = run_noalloc(fvv, words, dims, t_np, t_nb, fill=rep - 7)
            assert counts == [n_comp, len(rois), 0]
            np.testing.assert_array_equal(lab, ref_lab)
    finally:
        r.close()


def test_too_many_components_are_flagged(fvv):
    """More raw components than the 8192 one block can sort: the
    reconstruction path reports FVV_ERR_CAPACITY with FVV_FLAG_ROOTS and no
    ROI, the allocation-free labeller the same flag with every label 0."""
    occ = random_grid(LARGE, 0.05, seed=1)
    rig = grid_rig(LARGE)
    _, n_comp = Oracle(rig).ccl_bfs(occ)
    assert n_comp > 8192
    words = grid_words(occ)
    r = make_lib_rig(fvv, rig, [])
    try:
        r.debug_label_coarse(0, words)
        c = r.counts(0, allow_capacity=True)
        assert c["flags"] & 1 and c["n_rois"] == 0
        with pytest.raises(fvv.FvvError) as e:
            r.counts(0)
        assert e.value.status == fvv.FVV_ERR_CAPACITY
    finally:
        r.close()
    lab, counts = run_noalloc(fvv, words, LARGE, 8, 2**31 - 1, fill=9)
    assert counts[0] > 8192 and counts[1] == 0 and counts[2] & 1
    assert not lab.any()


def test_reconstruction_after_a_given_grid_is_unchanged(fvv):
    """The hook leaves nothing behind that a later reconstruction of the slot
    would read: a carved frame after a given grid equals the oracle."""
    from synth import make_frame
    from tests.gpu_harness import compare, fetch_outputs
    rig, fr = make_frame("tiny", 2)
    occ = random_grid(rig.grid_dims(), 0.2, seed=3)
    r = fvv.Rig(rig, max_slots=1, host_staging=0)
    try:
        r.debug_label_coarse(0, grid_words(occ))
        r.upload_silhouettes(0, fr.masks.cuda())
        r.reconstruct([0])
        r.colour([0], [fr.rgb.cuda()], fr.viewpoint[None])
        torch.cuda.synchronize()
        g = fetch_outputs(r, 0)
    finally:
        r.close()
    compare(rig, fr, g)
