"""CPU-side checks of the C ABI: the library loads, exports every function
include/fvv.h declares, validates arguments on the host, and builds the same
marching-cubes polygons as the oracle's face rule (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import Oracle
from synth import make_rig
from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "fvv.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fvv_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def fvv():
    from paper_1903_11785_gb300.build import build
    build()
    from paper_1903_11785_gb300 import fvv as mod
    return mod


def test_library_exports_every_declared_symbol(fvv):
    names = _declared()
    assert len(names) >= 14
    lib = C.CDLL(fvv.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(fvv.EXPORTED)
    assert fvv.fvv_version() == 1


def test_mc_table_matches_oracle_face_rule(fvv):
    ntri, edges = fvv.fvv_mc_table()
    for cs in range(256):
        ref = Oracle.mc_cell(cs)
        assert ntri[cs] == len(ref), cs
        got = [tuple(int(e) for e in edges[cs, j]) for j in range(ntri[cs])]
        assert got == ref, cs
    assert ntri.max() <= 12


def test_query_arena_and_validation(fvv):
    rig = make_rig("tiny")
    d = fvv.make_desc(rig, max_slots=2, host_staging=1)
    p = fvv.make_params(rig, max_fine_words=1 << 16)
    n1 = fvv.fvv_query_arena(d, p)
    d2 = fvv.make_desc(rig, max_slots=4, host_staging=1)
    n2 = fvv.fvv_query_arena(d2, p)
    assert n2 > n1 > 0
    # per-slot part includes the depth images and staging of every camera
    pix = int(np.sum(rig.width.astype(np.int64) * rig.height))
    assert (n2 - n1) // 2 >= pix * (4 + 1 + 3)
    bad = fvv.make_params(rig)
    bad.coarse_m = 0.0
    with pytest.raises(fvv.FvvError) as e:
        fvv.fvv_query_arena(d, bad)
    assert e.value.status == fvv.FVV_ERR_INVALID_ARG
    bad = fvv.make_params(rig)
    bad.bisect_steps = 31
    with pytest.raises(fvv.FvvError):
        fvv.fvv_query_arena(d, bad)
    bad = fvv.make_params(rig)
    bad.max_components = 9000
    with pytest.raises(fvv.FvvError):
        fvv.fvv_query_arena(d, bad)
    bad = fvv.make_params(rig)
    bad.surface_rule = 2
    with pytest.raises(fvv.FvvError):
        fvv.fvv_query_arena(d, bad)
    bad = fvv.make_params(rig, max_fine_words=(1 << 26) + 1)   # fine words are packed in 26 bits
    with pytest.raises(fvv.FvvError):
        fvv.fvv_query_arena(d, bad)
    n_masks_only = fvv.fvv_query_arena(fvv.make_desc(rig, max_slots=2, host_staging=2), p)
    assert n1 - n_masks_only >= 2 * pix * 3            # no RGB staging
    with pytest.raises(fvv.FvvError):
        fvv.fvv_query_arena(fvv.make_desc(rig, max_slots=2, host_staging=3), p)
    d0 = fvv.make_desc(rig, max_slots=0)
    with pytest.raises(fvv.FvvError):
        fvv.fvv_query_arena(d0, p)


def test_null_arguments_are_rejected(fvv):
    lib = C.CDLL(fvv.LIB_PATH)
    lib.fvv_query_arena.restype = C.c_int
    assert lib.fvv_query_arena(None, None, None) == fvv.FVV_ERR_INVALID_ARG
    assert fvv._lib.fvv_destroy_rig(None) == fvv.FVV_OK
    assert fvv._lib.fvv_reconstruct(None, None, 0, None) == fvv.FVV_ERR_INVALID_ARG
    assert fvv._lib.fvv_upload_silhouettes(None, 0, None, 1, None) == fvv.FVV_ERR_INVALID_ARG
    assert fvv._lib.fvv_upload_silhouettes_batch(None, None, 0, None, 1, None) == fvv.FVV_ERR_INVALID_ARG
    assert fvv._lib.fvv_colour(None, None, 0, None, 1, None, None) == fvv.FVV_ERR_INVALID_ARG
    assert fvv._lib.fvv_get_counts(None, 0, None, None) == fvv.FVV_ERR_INVALID_ARG
    assert fvv._lib.fvv_mc_table(None, None) == fvv.FVV_ERR_INVALID_ARG
    assert fvv._lib.fvv_debug_label_coarse(None, 0, None, None) == fvv.FVV_ERR_INVALID_ARG
    assert fvv._lib.fvv_get_results_batch(None, None, 0, None, 0, None) == fvv.FVV_ERR_INVALID_ARG
