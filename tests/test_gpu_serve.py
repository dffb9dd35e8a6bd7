"""Serving: requests from several rigs arrive (Poisson) while earlier ones are
on the GPU; they are admitted as slots and the memory budget allow, batched
per group of rigs with the same calibration, and overlapped.  Every result
must equal the same frame reconstructed and coloured alone, also when slots
with fitted (small) capacities overflow and the frame is served again with
the default capacities."""
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
    srv = Server([pa, pb], budget_bytes=3 << 30, max_slots_per_group=3, caps=caps, mask_copies=mask_copies)
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


def test_rigs_with_one_calibration_are_batched_together_and_overflow_is_served_again():
    """Two rigs with the same calibration share one group, and their requests
    go into the same batches; a frame whose needs exceed the fitted
    capacities (here: fitted on a pool of one small frame) is served again by
    the overflow slot, with the same result as alone."""
    from paper_1903_11785_gb300.build import build
    build()
    from paper_1903_11785_gb300.serve import RigPool, Server, poisson_schedule, summarize
    caps = dict(max_fine_words=1 << 18, max_verts=1 << 19, max_tris=1 << 20)
    pa, fa = _pool("tiny", 4)
    pb, _ = _pool("tiny", 4)
    srv = Server([pa, pb], budget_bytes=3 << 30, max_slots_per_group=4, caps=caps)
    try:
        assert len(srv.groups) == 1 and srv.groups[0].members == [0, 1]
        reqs = poisson_schedule(2, 400.0, 24, seed=5, pool_sizes=[4, 4])
        got = {}
        done = srv.run(reqs, on_done=lambda g, q: got.__setitem__(q.rid, g.rig.results(q.slot)["verts"].cpu()),
                       time_scale=50.0)
        s = summarize(done)
        assert s["frames"] == 24 and s["overflowed"] == 0
        mixed = {}
        for q in done:
            mixed.setdefault(q.batch, set()).add(q.rig)
        assert any(len(v) == 2 for v in mixed.values())       # a batch held requests of both rigs
        for q in done:
            assert torch.equal(got[q.rid], _alone(pa.scene_rig, fa[q.frame], caps)["verts"])
    finally:
        srv.close()
    # capacities fitted to one frame's needs, then a frame that needs more
    import dataclasses
    small = RigPool(scene_rig=pa.scene_rig, masks=pa.masks[:1], rgb=pa.rgb[:1], viewpoints=pa.viewpoints[:1])
    srv = Server([small], budget_bytes=3 << 30, max_slots_per_group=2, caps=caps)
    try:
        g = srv.groups[0]
        fit = srv.caps[0]
        # force an overflow: shrink the fitted vertex capacity below what frame 0 needs
        g.rig.close()
        tight = dict(fit, max_verts=1 << 10)
        from paper_1903_11785_gb300 import fvv
        g.rig = fvv.Rig(pa.scene_rig, max_slots=g.n_slots, host_staging=0, **tight)
        full = RigPool(scene_rig=pa.scene_rig, masks=pa.masks, rgb=pa.rgb, viewpoints=pa.viewpoints)
        srv.groups[0].pools = [full]
        srv.overflow[0].pools = [full]
        got = {}
        reqs = poisson_schedule(1, 400.0, 6, seed=6, pool_sizes=[4])
        done = srv.run(reqs, on_done=lambda g, q: got.__setitem__(q.rid, g.rig.results(q.slot)["verts"].cpu()),
                       time_scale=50.0)
        assert all(q.overflowed for q in done) and srv.n_overflowed == 6
        for q in done:
            assert torch.equal(got[q.rid], _alone(pa.scene_rig, fa[q.frame], caps)["verts"])
    finally:
        srv.close()
