"""Serving: requests from two rigs arrive (Poisson) while earlier ones are on
the GPU; they are admitted as slots free up, batched per rig and overlapped.
Every result must equal the same frame reconstructed and coloured alone."""
import numpy as np
import pytest
import torch

from synth import make_frame, make_rig

pytestmark = pytest.mark.gpu


def _pool(config, n):
    from paper_1903_11785_gb300.serve import RigPool
    rig = make_rig(config)
    frames = [make_frame(config, i, rig=rig)[1] for i in range(n)]
    return RigPool(scene_rig=rig, masks=[f.masks.pin_memory() for f in frames],
                   rgb=[f.rgb.pin_memory() for f in frames],
                   viewpoints=np.stack([f.viewpoint for f in frames])), frames


def _alone(rig, fr, caps):
    from paper_1903_11785_gb300 import fvv
    r = fvv.Rig(rig, max_slots=1, host_staging=0, **caps)
    try:
        r.upload_silhouettes(0, fr.masks.cuda())
        r.reconstruct([0])
        r.colour([0], [fr.rgb.cuda()], fr.viewpoint[None])
        out = r.results(0)
        return {k: out[k].cpu() for k in ("verts", "tris", "rgb", "cam")}
    finally:
        r.close()


@pytest.mark.parametrize("mask_copies", [False, True])
def test_served_results_equal_alone(mask_copies):
    from paper_1903_11785_gb300.build import build
    build()
    from paper_1903_11785_gb300.serve import Server, poisson_schedule, summarize
    caps = dict(max_fine_words=1 << 18, max_verts=1 << 19, max_tris=1 << 20)
    pa, fa = _pool("tiny", 4)
    pb, fb = _pool("hd720", 3)
    srv = Server([pa, pb], budget_bytes=3 << 30, max_slots_per_rig=3, caps=caps, mask_copies=mask_copies)
    got = {}

    def on_done(rs, q):
        out = rs.rig.results(q.slot)
        got[q.rid] = {k: out[k].cpu() for k in ("verts", "tris", "rgb", "cam")}

    try:
        # arrivals compressed 50x (20,000 requests/s per rig), so that requests
        # arrive while earlier batches are still on the GPU
        reqs = poisson_schedule(2, 400.0, 36, seed=3, pool_sizes=[4, 3])
        done = srv.run(reqs, on_done=on_done, time_scale=50.0)
    finally:
        srv.close()
    assert all(q.t_done > 0 and q.slot >= 0 for q in done)
    s = summarize(done)
    assert s["frames"] == 36 and s["batches"] < 36          # some requests shared a batch
    ref = {}
    for q in done:
        key = (q.rig, q.frame)
        if key not in ref:
            rig = pa.scene_rig if q.rig == 0 else pb.scene_rig
            fr = (fa if q.rig == 0 else fb)[q.frame]
            ref[key] = _alone(rig, fr, caps)
        for k, v in ref[key].items():
            assert torch.equal(got[q.rid][k], v), (q.rid, k)
