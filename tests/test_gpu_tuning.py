"""Launch shapes and CUDA graphs change nothing in the results: the
autotuner's choice, unusual hand-set shapes and graph replay all give the
same bits as the default launches."""
import numpy as np
import pytest
import torch

from synth import make_frame, make_rig

pytestmark = pytest.mark.gpu


def _frames(n):
    rig = make_rig("tiny")
    return rig, [make_frame("tiny", i, rig=rig)[1] for i in range(n)]


def _run(r, frames, stream=None):
    from paper_1903_11785_gb300 import fvv
    slots = list(range(len(frames)))
    for s, fr in zip(slots, frames):
        r.upload_silhouettes(s, fr.masks.cuda(), stream=stream)
    r.reconstruct(slots, stream=stream)
    r.colour(slots, [fr.rgb.cuda() for fr in frames], np.stack([fr.viewpoint for fr in frames]), stream=stream)
    torch.cuda.synchronize()
    out = []
    for s in slots:
        res = r.results(s)
        out.append({k: res[k].cpu() for k in ("verts", "tris", "rgb", "cam")} | {"counts": res["counts"]}
                   | {"depth": r.debug(s, fvv.FVV_DEBUG_DEPTH).cpu()})
    return out


def _results(c):
    """Counts that are results of the method: everything but the silhouette
    words the kernels read (lookups_*), which depend on the tile shape."""
    return {k: v for k, v in c.items() if not k.startswith("lookups_")}


def _same(a, b):
    for x, y in zip(a, b):
        assert _results(x["counts"]) == _results(y["counts"])
        for k in ("verts", "tris", "rgb", "cam", "depth"):
            assert torch.equal(x[k], y[k]), k


def test_autotune_and_shapes_keep_results():
    from paper_1903_11785_gb300 import fvv
    from paper_1903_11785_gb300.build import build
    build()
    rig, frames = _frames(3)
    caps = dict(max_fine_words=1 << 17, max_verts=1 << 18, max_tris=1 << 19)
    r = fvv.Rig(rig, max_slots=3, host_staging=0, **caps)
    try:
        ref = _run(r, frames)
        chosen = r.autotune([0, 1, 2])
        assert set(chosen) == set(fvv.TUNE_KNOBS) | {"fine_tile", "zbuffer_cams"}
        assert chosen["fine_tile"] in fvv.FINE_TILES
        assert chosen["zbuffer_cams"] in fvv.ZBUFFER_CAMS
        for k in fvv.TUNE_KNOBS:
            th, wv = chosen[k]
            assert th in (64, 128, 256) and wv in (2, 4, 8, 16, 32, 64)
        # the autotuner leaves the slots freshly reconstructed
        after = [{k: r.results(s)[k].cpu() for k in ("verts", "tris")} | {"counts": r.counts(s)} for s in range(3)]
        for x, y in zip(after, ref):
            assert _results(x["counts"]) == _results(y["counts"]) and torch.equal(x["verts"], y["verts"])
        _same(_run(r, frames), ref)
        r.set_tuning({k: (32, 1) for k in fvv.TUNE_KNOBS})
        _same(_run(r, frames), ref)
        r.set_tuning({k: (64, 64) for k in fvv.TUNE_KNOBS})
        _same(_run(r, frames), ref)
        for tile in fvv.FINE_TILES:            # every fine-hull tile shape: the same bits
            r.set_tuning({k: (128, 8) for k in fvv.TUNE_KNOBS} | {"fine_tile": tile})
            assert r.get_tuning()["fine_tile"] == tile
            _same(_run(r, frames), ref)
        for zc in fvv.ZBUFFER_CAMS:            # cameras per z-buffer block: the same depth images
            r.set_tuning({k: (96, 4) for k in fvv.TUNE_KNOBS} | {"zbuffer_cams": zc})
            assert r.get_tuning()["zbuffer_cams"] == zc
            _same(_run(r, frames), ref)
        with pytest.raises(fvv.FvvError):
            r.set_tuning({k: (128, 8) for k in fvv.TUNE_KNOBS} | {"fine_tile": 3})
        with pytest.raises(fvv.FvvError):
            r.set_tuning({k: (128, 8) for k in fvv.TUNE_KNOBS} | {"zbuffer_cams": 3})
        with pytest.raises(fvv.FvvError):
            r.set_tuning({k: (48, 8) for k in fvv.TUNE_KNOBS})
    finally:
        r.close()


def test_graph_replay_matches_direct_launches():
    from paper_1903_11785_gb300 import fvv
    rig, frames = _frames(2)
    r = fvv.Rig(rig, max_slots=2, host_staging=0, max_fine_words=1 << 17)
    try:
        ref = _run(r, frames)
        r.set_graphs(True)
        st = torch.cuda.Stream()
        for _ in range(3):                     # record once, replay twice
            _same(_run(r, frames, stream=st), ref)
        # a different slot list gets its own graph
        one = _run(r, frames[1:], stream=st)
        _same(one, _run(fvv.Rig(rig, max_slots=1, host_staging=0, max_fine_words=1 << 17), frames[1:]))
        r.set_graphs(False)
        _same(_run(r, frames), ref)
    finally:
        r.close()
