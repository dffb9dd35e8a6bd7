"""Parity of the sm_103a path (through the C ABI) with the CPU oracle.

Every output of every step is compared element by element on the same
seeded inputs: packed silhouettes, coarse occupancy and its test count,
canonical labels, ROIs, padded fine grids and their test count, vertices,
triangles, bisection test count, depth images, colours and chosen cameras.
All of them are bit-exact (the vertex tolerance of 1e-5 m is checked too)."""
import math
import os

import numpy as np
import pytest
import torch

from synth import ABSTAIN, make_frame, make_rig, render, scene_objects
from synth.scenes import _gen, _make_rig
from tests.gpu_harness import compare, fetch_outputs, run_gpu, run_oracle, unpack_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    assert torch.cuda.is_available(), "the -m gpu tests need a CUDA GPU"
    from paper_1903_11785_gb300.build import build
    build()


def test_tiny_frame_bit_exact():
    rig, fr = make_frame("tiny", 0)
    g = run_gpu(rig, [fr])[0]
    ref = compare(rig, fr, g)
    assert len(ref.rois) == 1 and len(ref.tris) > 10000


def test_tiny_host_buffers_match():
    rig, fr = make_frame("tiny", 1)
    g = run_gpu(rig, [fr], host=True)[0]
    compare(rig, fr, g)


def test_colour_reads_pinned_host_rgb_in_place():
    """FVV_RGB_MAPPED_HOST: the colour kernel reads pinned host images in
    place (no staging copy) and gives the oracle's colours; pageable host
    memory is refused without launching anything."""
    rig = make_rig("tiny")
    frames = [make_frame("tiny", i, rig=rig)[1] for i in range(2)]
    outs = run_gpu(rig, frames, rgb_in_place=True)
    for fr, g in zip(frames, outs):
        compare(rig, fr, g)
    from paper_1903_11785_gb300 import fvv
    r = fvv.Rig(rig, max_slots=1, host_staging=0)
    try:
        r.upload_silhouettes(0, frames[0].masks.cuda())
        r.reconstruct([0])
        pageable = [np.ascontiguousarray(frames[0].rgb[n].numpy()) for n in range(rig.n_cams)]
        ptrs = fvv._ptr_array([a.ctypes.data for a in pageable])
        vp = np.ascontiguousarray(frames[0].viewpoint, np.float32)
        arr = (fvv.C.c_int * 1)(0)
        st = fvv._lib.fvv_colour(r.ptr, arr, 1, ptrs, fvv.FVV_RGB_MAPPED_HOST,
                                 vp.ctypes.data_as(fvv.C.POINTER(fvv.C.c_float)), fvv._stream())
        assert st == fvv.FVV_ERR_INVALID_ARG
        torch.cuda.synchronize()
    finally:
        r.close()


def test_masks_read_in_place_including_ragged_rows():
    """FVV_MAPPED_HOST masks: the packing kernel reads pinned host images in
    place, on 640-pixel rows (16-byte loads) and on 630-pixel rows (byte
    loads, rows not 16-byte aligned)."""
    rig = make_rig("tiny")
    fr = make_frame("tiny", 3, rig=rig)[1]
    compare(rig, fr, run_gpu(rig, [fr], masks_in_place=True, rgb_in_place=True)[0])
    n, r, h = 6, 6.0, 3.0
    cs = [(r * math.cos(2 * math.pi * k / n), r * math.sin(2 * math.pi * k / n), h) for k in range(n)]
    rig = _make_rig("ragged", cs, [(0, 0, 0.9)] * n, 480.0, 630, 349, _gen("ragged/rig"),
                    (-2.0, -2.0, 0.0), (2.0, 2.0, 2.5), 0.05, 0.01, 6)
    fr = render(rig, scene_objects("tiny", 3), index=3, config_tag="ragged")
    compare(rig, fr, run_gpu(rig, [fr], masks_in_place=True)[0])


def test_slot_reuse_leaves_no_stale_depth():
    """A slot reconstructed again with a different frame: the depth stage
    clears only the box the previous z-buffer wrote, and every output (the
    whole depth images included) equals the oracle's for the new frame."""
    from paper_1903_11785_gb300 import fvv
    rig = make_rig("tiny")
    f0, f1 = make_frame("tiny", 0, rig=rig)[1], make_frame("tiny", 5, rig=rig)[1]
    r = fvv.Rig(rig, max_slots=1, host_staging=0)
    try:
        for fr in (f0, f1, f0):
            r.upload_silhouettes(0, fr.masks.cuda())
            r.reconstruct([0])
            r.colour([0], [fr.rgb.cuda()], fr.viewpoint[None])
            torch.cuda.synchronize()
            c = r.counts(0)
            res = r.results(0)
            g = dict(counts=c, rois=res["rois"], verts=res["verts"].cpu().numpy(), tris=res["tris"].cpu().numpy(),
                     rgb=res["rgb"].cpu().numpy(), cam=res["cam"].cpu().numpy(),
                     sil=r.debug(0, fvv.FVV_DEBUG_SIL_BITS).cpu().numpy().view(np.uint32),
                     coarse=r.debug(0, fvv.FVV_DEBUG_COARSE_BITS).cpu().numpy().view(np.uint32),
                     labels=r.debug(0, fvv.FVV_DEBUG_LABELS).cpu().numpy(),
                     fine=r.debug(0, fvv.FVV_DEBUG_FINE_BITS).cpu().numpy().view(np.uint32),
                     depth=r.debug(0, fvv.FVV_DEBUG_DEPTH).cpu().numpy())
            compare(rig, fr, g)
    finally:
        r.close()


def test_batched_slots_each_bit_exact():
    """Three frames in one reconstruct/colour call, slots listed out of order."""
    rig = make_rig("tiny")
    frames = [make_frame("tiny", i, rig=rig)[1] for i in range(3)]
    outs = run_gpu(rig, frames, slots=[2, 0, 1])
    for fr, g in zip(frames, outs):
        compare(rig, fr, g)


@pytest.mark.parametrize("mode", ["device", "host", "in_place"])
def test_batched_upload_each_bit_exact(mode):
    """Three frames packed by one fvv_upload_silhouettes_batch call, slots
    out of order, masks on the device, staged from host memory or read in
    place."""
    rig = make_rig("tiny")
    frames = [make_frame("tiny", i, rig=rig)[1] for i in range(3)]
    outs = run_gpu(rig, frames, slots=[1, 3, 0], upload_batch=True, host=mode == "host",
                   masks_in_place=mode == "in_place")
    for fr, g in zip(frames, outs):
        compare(rig, fr, g)


@pytest.mark.parametrize("W", [96, 100])
def test_batched_upload_spans_launches(W):
    """64 cameras (the most a rig takes), so one packing launch holds 32
    frames: 40 frames in one call, slots in reverse order, take two launches.
    Every slot's silhouette bits equal its masks packed 32 pixels per word
    (W = 96: whole 16-byte loads; W = 100: ragged rows)."""
    from paper_1903_11785_gb300 import fvv
    n, H, F = 64, 48, 40
    cs = [(6.0 * math.cos(2 * math.pi * k / n), 6.0 * math.sin(2 * math.pi * k / n), 3.0 + 0.3 * (k % 3))
          for k in range(n)]
    rig = _make_rig(f"ring64w{W}", cs, [(0, 0, 0.9)] * n, 60.0, W, H, _gen(f"ring64w{W}/rig"),
                    (-1.0, -1.0, 0.0), (1.0, 1.0, 2.0), 0.1, 0.05, 2)
    g = torch.Generator().manual_seed(W)
    masks = (torch.rand((F, n, H, W), generator=g) < 0.3).to(torch.uint8)
    r = fvv.Rig(rig, max_slots=F, host_staging=0, max_fine_words=1 << 12, max_verts=1 << 12, max_tris=1 << 12)
    try:
        slots = list(range(F))[::-1]
        r.upload_silhouettes_batch(slots, masks.cuda())
        torch.cuda.synchronize()
        for j, s in enumerate(slots):
            bits = r.debug(s, fvv.FVV_DEBUG_SIL_BITS).cpu().numpy().view(np.uint32)
            np.testing.assert_array_equal(unpack_rows(bits, (n, H), W), masks[j].numpy())
    finally:
        r.close()


def test_batched_upload_rejects_bad_arguments():
    from paper_1903_11785_gb300 import fvv
    rig = make_rig("tiny")
    frames = [make_frame("tiny", i, rig=rig)[1] for i in range(2)]
    r = fvv.Rig(rig, max_slots=2, host_staging=0, max_fine_words=1 << 16)
    try:
        ms = [fr.masks.cuda() for fr in frames]
        for bad in ([0, 0], [0, 2], [-1, 1]):
            with pytest.raises(fvv.FvvError) as e:
                r.upload_silhouettes_batch(bad, ms)
            assert e.value.status == fvv.FVV_ERR_INVALID_ARG
        with pytest.raises(fvv.FvvError):       # host masks need staging
            r.upload_silhouettes_batch([0, 1], [fr.masks for fr in frames])
        with pytest.raises(fvv.FvvError) as e:  # nothing was packed
            r.reconstruct([0])
        assert e.value.status == fvv.FVV_ERR_NOT_READY
    finally:
        r.close()


def test_batched_equals_one_by_one():
    rig = make_rig("tiny")
    frames = [make_frame("tiny", i, rig=rig)[1] for i in range(2)]
    a = run_gpu(rig, frames, batch=True)
    b = run_gpu(rig, frames, batch=False)
    for x, y in zip(a, b):
        for k in ("verts", "tris", "rgb", "cam", "depth", "labels", "fine"):
            np.testing.assert_array_equal(x[k], y[k])


def test_volleyball_frame_bit_exact():
    rig, fr = make_frame("volleyball", 0)
    g = run_gpu(rig, [fr])[0]
    ref = compare(rig, fr, g)
    assert len(ref.rois) == 13


def test_bench_batch_all_frames_bit_exact(tmp_path):
    """The benchmark's step at full size: 64 volleyball-shaped frames packed
    by one upload call and reconstructed and coloured by one call each, with
    the launch shapes the autotuner picks on that batch.  Every output of
    every one of the 64 frames (coarse grid, labels, ROI table, fine grids,
    test counts, vertices, triangles, depth images, colours, cameras) is
    compared with the oracle's through a hash of the oracle's layout; the
    oracle runs frame-parallel in spawned worker processes."""
    import multiprocessing as mp
    import bench
    from paper_1903_11785_gb300 import fvv
    from synth import Frame
    from tests.gpu_harness import _oracle_digest_job, gpu_digest
    import shutil
    import tempfile
    F = 64
    rig, masks, rgb, vps = bench.make_batch(F, 0, "cuda")
    # the workers read the inputs from files (memory-backed where there is room)
    shm = "/dev/shm"
    base = shm if os.path.isdir(shm) and shutil.disk_usage(shm).free > 24 << 30 else str(tmp_path)
    work = tempfile.mkdtemp(prefix="fvv_parity_", dir=base)
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(max(1, min(16, (os.cpu_count() or 2) - 1)))
    try:
        np.save(os.path.join(work, "masks.npy"), masks.cpu().numpy())
        np.save(os.path.join(work, "rgb.npy"), rgb.cpu().numpy())
        np.save(os.path.join(work, "vps.npy"), np.asarray(vps))
        pending = pool.map_async(_oracle_digest_job, [(work, bench.CONFIG, i) for i in range(F)])
        r = fvv.Rig(rig, max_slots=F, host_staging=0)
        try:
            slots = list(range(F))
            r.upload_silhouettes_batch(slots, masks)
            r.reconstruct(slots)
            r.autotune(slots)                 # times the shapes, then reconstructs once more
            r.colour(slots, rgb, vps)
            torch.cuda.synchronize()
            got = {i: gpu_digest(rig, fetch_outputs(r, i)) for i in slots}
            ref = dict(pending.get(timeout=1800))
            bad = [i for i in slots if got[i] != ref[i]]
            for i in bad[:1]:                     # element by element, for the message
                fr = Frame(masks=masks[i].cpu(), rgb=rgb[i].cpu(), ellipsoids=[], viewpoint=vps[i])
                compare(rig, fr, fetch_outputs(r, i))
            assert not bad, f"frames differing from the oracle: {bad}"
        finally:
            r.close()
    finally:
        pool.terminate()
        shutil.rmtree(work, ignore_errors=True)


@pytest.mark.parametrize("coarse,fine", [(0.02, 0.02), (0.05, 0.02)], ids=["coarse_eq_fine_20mm", "coarse50_fine20"])
def test_fig10_shapes_bit_exact(coarse, fine):
    """The end points of the Fig. 10 sweeps on the device, on a
    volleyball-shaped frame: coarse = fine = 20 mm, the coarse-to-fine scheme
    switched off (a 1000 x 550 x 200 coarse grid, ROIs carved again at the
    same step), and the paper's non-integer 50/20 mm ratio (fine sides of
    ceil(2.5 n) samples)."""
    from dataclasses import replace
    rig = replace(make_rig("volleyball"), coarse_m=coarse, fine_m=fine)
    _, fr = make_frame("volleyball", 5, rig=rig)
    g = run_gpu(rig, [fr])[0]
    ref = compare(rig, fr, g)
    assert len(ref.rois) >= 12
    if coarse != fine:
        spans = [r.gmax[a] - r.gmin[a] + 1 for r in ref.rois for a in range(3)]
        fdims = [r.fdim[a] for r in ref.rois for a in range(3)]
        assert fdims == [-(-5 * n // 2) for n in spans]


@pytest.mark.parametrize("config", ["volleyball_t1", "judo_t1"])
def test_table1_shapes_bit_exact(config):
    """The capture shapes of Table I on the device: volleyball with 10 cameras
    at 3840 x 2160 over an 18 x 18 x 9 m volume at 50/20 mm (the 360 x 360 x
    180 coarse grid, 2.33e7 voxels, that the paper counts), and judo with 16
    cameras at 1080p over 5 x 6 x 2.1 m at 80/40 mm."""
    rig, fr = make_frame(config, 0)
    g = run_gpu(rig, [fr])[0]
    ref = compare(rig, fr, g)
    assert len(ref.rois) >= (12 if config == "volleyball_t1" else 2)


def test_results_batch_equals_per_slot_results():
    """fvv_get_results_batch (one wait for a group of slots, copies into
    pinned host buffers and into device buffers) returns what fvv_get_results
    returns slot by slot; a slot over capacity gets its counts and no copies;
    a slot never reconstructed is refused."""
    from paper_1903_11785_gb300 import fvv
    rig = make_rig("tiny")
    frames = [make_frame("tiny", i, rig=rig)[1] for i in range(3)]
    r = fvv.Rig(rig, max_slots=4, host_staging=0, max_fine_words=1 << 16)
    try:
        for s, fr in enumerate(frames):
            r.upload_silhouettes(s, fr.masks.cuda())
        r.reconstruct([0, 1, 2])
        r.colour([0, 1, 2], [fr.rgb.cuda() for fr in frames], np.stack([fr.viewpoint for fr in frames]))
        torch.cuda.synchronize()
        ref = [r.results(s) for s in range(3)]
        for device in ("cpu", "cuda"):
            outs = []
            for c in (x["counts"] for x in ref):
                mk = (lambda shape, dt: torch.full(shape, 7, dtype=dt).pin_memory()) if device == "cpu" else \
                     (lambda shape, dt: torch.full(shape, 7, dtype=dt, device="cuda"))
                outs.append(dict(verts=mk((c["n_verts"], 3), torch.float32), tris=mk((c["n_tris"], 3), torch.int32),
                                 rgb=mk((c["n_verts"], 3), torch.uint8), cam=mk((c["n_verts"],), torch.int32)))
            counts = fvv.fvv_get_results_batch(r.ptr, [2, 0, 1], [outs[2], outs[0], outs[1]])
            torch.cuda.synchronize()
            assert [counts[1], counts[2], counts[0]] == [x["counts"] for x in ref]
            for o, x in zip(outs, ref):
                for k in ("verts", "tris", "rgb", "cam"):
                    assert torch.equal(o[k].cpu(), x[k].cpu()), k
        with pytest.raises(fvv.FvvError) as e:
            fvv.fvv_get_results_batch(r.ptr, [0, 3], [{}, {}])
        assert e.value.status == fvv.FVV_ERR_NOT_READY
    finally:
        r.close()
    # a slot over its vertex capacity: counts with the flag, nothing copied
    r = fvv.Rig(rig, max_slots=2, host_staging=0, max_fine_words=1 << 16, max_verts=1 << 10)
    try:
        r.upload_silhouettes(0, frames[0].masks.cuda())
        r.reconstruct([0])
        v = torch.full((8, 3), 5.0).pin_memory()
        with pytest.raises(fvv.FvvError) as e:
            fvv.fvv_get_results_batch(r.ptr, [0], [dict(verts=v)])
        assert e.value.status == fvv.FVV_ERR_CAPACITY
        torch.cuda.synchronize()
        assert bool((v == 5.0).all())
    finally:
        r.close()


def test_judo_frame_bit_exact():
    rig, fr = make_frame("judo", 0)
    g = run_gpu(rig, [fr])[0]
    compare(rig, fr, g)


def test_hd720_frame_bit_exact():
    rig, fr = make_frame("hd720", 0)
    g = run_gpu(rig, [fr])[0]
    compare(rig, fr, g)


def test_abstain_policy_and_zero_steps():
    rig, fr = make_frame("tiny", 2)
    rig.oob_policy = ABSTAIN
    rig.bisect_steps = 0
    g = run_gpu(rig, [fr])[0]
    ref = compare(rig, fr, g)
    assert ref.tests_bisect == 0


@pytest.mark.parametrize("config,index", [("tiny", 4), ("volleyball", 1), ("judo", 1)])
def test_paper_surface_rule_bit_exact(config, index):
    """Sec. II-C as printed: vertices from the pixel walks and the minimum
    ratio of Eqs. (2)-(3) (the lambda kernel) equal the oracle's, and so do
    the pixel counts, depth images and colours that follow."""
    rig, fr = make_frame(config, index)
    rig.surface_rule = 1
    g = run_gpu(rig, [fr])[0]
    ref = compare(rig, fr, g)
    assert ref.tests_bisect >= len(ref.verts) * rig.n_cams


def test_paper_surface_rule_abstain_ragged():
    """The lambda kernel under ABSTAIN (cameras that do not see the ON end
    bound nothing) on images 630 px wide, the walks crossing partial words."""
    n, r, h = 6, 6.0, 3.0
    cs = [(r * math.cos(2 * math.pi * k / n), r * math.sin(2 * math.pi * k / n), h) for k in range(n)]
    rig = _make_rig("ragged", cs, [(0, 0, 0.9)] * n, 480.0, 630, 349, _gen("ragged/rig"),
                    (-2.0, -2.0, 0.0), (2.0, 2.0, 2.5), 0.05, 0.01, 6)
    rig.oob_policy = ABSTAIN
    rig.surface_rule = 1
    fr = render(rig, scene_objects("tiny", 5), index=5, config_tag="ragged")
    g = run_gpu(rig, [fr])[0]
    compare(rig, fr, g)


def test_abstain_policy_with_bisection():
    """ABSTAIN with bisection on 630 px images: cameras that do not see a
    midpoint do not vote, and cameras decided once per edge are skipped."""
    n, r, h = 6, 6.0, 3.0
    cs = [(r * math.cos(2 * math.pi * k / n), r * math.sin(2 * math.pi * k / n), h) for k in range(n)]
    rig = _make_rig("ragged", cs, [(0, 0, 0.9)] * n, 480.0, 630, 349, _gen("ragged/rig"),
                    (-2.0, -2.0, 0.0), (2.0, 2.0, 2.5), 0.05, 0.01, 9)
    rig.oob_policy = ABSTAIN
    fr = render(rig, scene_objects("tiny", 6), index=6, config_tag="ragged")
    g = run_gpu(rig, [fr])[0]
    ref = compare(rig, fr, g)
    assert ref.tests_bisect > 0


def _bisect_window(n_verts, n_slots, threads, waves):
    """Vertices per lane that k_bisect sorts at once for a slot of n_verts
    vertices when the launch has these shapes and the default capacities (1:
    no sorting).  The kernel takes windows of 32 * k vertices (k = 4 or 2)
    when there are at least two per warp that can be resident for the slot;
    at the small grids used here that is every warp launched."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    warps = max(1, sms * min(waves, 16 * n_slots) // n_slots) * threads // 32
    return 4 if n_verts >= 2 * warps * 32 * 4 else 2 if n_verts >= 2 * warps * 32 * 2 else 1


@pytest.mark.parametrize("config,first,n_frames,threads,window",
                         [("tiny", 3, 1, 32, 2), ("tiny", 5, 2, 32, 4), ("volleyball", 3, 1, 256, 4)])
def test_bisection_in_sorted_windows_bit_exact(config, first, n_frames, threads, window):
    """Bisection launches small enough that every warp takes windows of
    32 x `window` vertices and sorts them by their number of undecided cameras
    before bisecting them (the path of batched launches): every output equals
    the oracle's, the last, partly filled window included."""
    from paper_1903_11785_gb300 import fvv
    rig = make_rig(config)
    frames = [make_frame(config, first + i, rig=rig)[1] for i in range(n_frames)]
    tuning = {k: (256, 8) for k in fvv.TUNE_KNOBS} | {"bisect": (threads, 1)}
    gs = run_gpu(rig, frames, tuning=tuning)
    for fr, g in zip(frames, gs):
        assert _bisect_window(g["counts"]["n_verts"], n_frames, threads, 1) == window
        assert g["counts"]["n_verts"] % (32 * window) != 0
        compare(rig, fr, g)


def test_bisection_in_sorted_windows_abstain():
    """The sorted windows under ABSTAIN on 630 px images: a vertex carries
    whether some camera saw its whole edge in the silhouette (its vote) into
    the lane that bisects it."""
    from paper_1903_11785_gb300 import fvv
    n, r, h = 6, 6.0, 3.0
    cs = [(r * math.cos(2 * math.pi * k / n), r * math.sin(2 * math.pi * k / n), h) for k in range(n)]
    rig = _make_rig("ragged", cs, [(0, 0, 0.9)] * n, 480.0, 630, 349, _gen("ragged/rig"),
                    (-2.0, -2.0, 0.0), (2.0, 2.0, 2.5), 0.05, 0.01, 9)
    rig.oob_policy = ABSTAIN
    fr = render(rig, scene_objects("tiny", 6), index=6, config_tag="ragged")
    g = run_gpu(rig, [fr], tuning={k: (256, 8) for k in fvv.TUNE_KNOBS} | {"bisect": (32, 1)})[0]
    assert _bisect_window(g["counts"]["n_verts"], 1, 32, 1) >= 2
    ref = compare(rig, fr, g)
    assert ref.tests_bisect > 0


@pytest.mark.parametrize("n_cams", [5, 20, 64])
def test_generic_and_large_camera_counts(n_cams):
    """5 cameras (no unrolled instantiation: the generic camera loops), 20
    cameras (two camera groups in the fine hull's per-tile decisions) and 64
    (the most a rig takes: four groups, every camera bit of the 64-bit
    masks), with bisection and with the paper's walk."""
    r, h = 6.0, 3.0
    cs = [(r * math.cos(2 * math.pi * k / n_cams), r * math.sin(2 * math.pi * k / n_cams), h + 0.3 * (k % 3))
          for k in range(n_cams)]
    rig = _make_rig(f"ring{n_cams}", cs, [(0, 0, 0.9)] * n_cams, 420.0, 480, 320, _gen(f"ring{n_cams}/rig"),
                    (-2.0, -2.0, 0.0), (2.0, 2.0, 2.5), 0.05, 0.01, 7)
    fr = render(rig, scene_objects("tiny", 7), index=7, config_tag=f"ring{n_cams}")
    compare(rig, fr, run_gpu(rig, [fr])[0])
    # z-buffer blocks serving 2 and 4 cameras (5 cameras: a last group of one)
    from paper_1903_11785_gb300 import fvv
    for zc in (2, 4):
        compare(rig, fr, run_gpu(rig, [fr], tuning={k: (128, 8) for k in fvv.TUNE_KNOBS} | {"zbuffer_cams": zc})[0])
    rig.surface_rule = 1
    compare(rig, fr, run_gpu(rig, [fr])[0])


def test_wide_roi_compaction_reads_global_memory():
    """A flat 4.6 m disc at 1 cm: its ROI's fine planes hold about 7,100
    words, more than a compaction chunk stages in shared memory, so its
    chunks read the grid from global memory; the ball's small ROI in the
    same frame is staged.  Both give the oracle's vertices and triangles."""
    from synth.scenes import Ellipsoid
    n, r, h = 8, 9.0, 5.0
    cs = [(r * math.cos(2 * math.pi * k / n), r * math.sin(2 * math.pi * k / n), h) for k in range(n)]
    rig = _make_rig("disc", cs, [(0, 0, 0.3)] * n, 500.0, 640, 360, _gen("disc/rig"),
                    (-3.0, -3.0, 0.0), (3.0, 3.0, 0.8), 0.05, 0.01, 7)
    objs = [Ellipsoid(centre=np.array([0.0, 0.0, 0.3]), rot=np.eye(3), axes=np.array([2.3, 2.3, 0.1]),
                      colour=(200, 60, 40), obj=0),
            Ellipsoid(centre=np.array([2.75, 2.75, 0.5]), rot=np.eye(3), axes=np.full(3, 0.12),
                      colour=(40, 60, 200), obj=1)]
    fr = render(rig, objs, index=0, config_tag="disc")
    caps = dict(max_fine_words=1 << 20, max_verts=1 << 21, max_tris=1 << 22)
    ref = compare(rig, fr, run_gpu(rig, [fr], caps=caps)[0])
    nxw = [(r.fdim[0] + 2 + 31) // 32 for r in ref.rois]
    assert max(w * (r.fdim[1] + 2) for w, r in zip(nxw, ref.rois)) > 6144
    assert min(w * (r.fdim[1] + 2) for w, r in zip(nxw, ref.rois)) < 1000


def test_ragged_image_width():
    """Images whose width is not a multiple of 32 (scalar packing path, partial
    last word of every silhouette row)."""
    n, r, h = 6, 6.0, 3.0
    cs = [(r * math.cos(2 * math.pi * k / n), r * math.sin(2 * math.pi * k / n), h) for k in range(n)]
    rig = _make_rig("ragged", cs, [(0, 0, 0.9)] * n, 480.0, 630, 349, _gen("ragged/rig"),
                    (-2.0, -2.0, 0.0), (2.0, 2.0, 2.5), 0.05, 0.01, 6)
    fr = render(rig, scene_objects("tiny", 3), index=3, config_tag="ragged")
    g = run_gpu(rig, [fr])[0]
    compare(rig, fr, g)


def test_empty_scene():
    rig, fr = make_frame("tiny", 0)
    fr.masks.zero_()
    g = run_gpu(rig, [fr])[0]
    c = g["counts"]
    assert c["n_components"] == 0 and c["n_rois"] == 0 and c["n_verts"] == 0 and c["n_tris"] == 0
    ref = compare(rig, fr, g)
    assert ref.coarse.sum() == 0
    assert np.isinf(g["depth"]).all()


def test_small_components_filtered():
    """Small floating specks next to the player give hull pieces of a few
    voxels that Eq. (1) removes (t_np = 8); heavy pixel noise (2% flips) is
    on top.  The GPU agrees on every component, label and ROI."""
    from synth import sphere_scene
    rig = make_rig("tiny")
    objs = scene_objects("tiny", 0)
    for k, rad in enumerate((0.02, 0.035, 0.05, 0.12)):
        objs += sphere_scene((-1.6 + 0.8 * k, 1.6, 1.8), rad)
    fr = render(rig, objs, flip_prob=0.02, config_tag="tiny-specks")
    g = run_gpu(rig, [fr])[0]
    ref = compare(rig, fr, g)
    assert ref.n_components > len(ref.rois) >= 2


def test_capacity_overflow_is_reported_and_recovers():
    """Everything foreground: the one component fills the volume and its fine
    grid exceeds max_fine_words; the call reports FVV_ERR_CAPACITY (flag FINE)
    without touching memory beyond the arena, and the coarse stage still
    matches the oracle.  A following normal frame on the same rig is exact."""
    from oracle import Oracle
    from paper_1903_11785_gb300 import fvv
    rig, fr = make_frame("tiny", 0)
    full = torch.ones_like(fr.masks)
    r = fvv.Rig(rig, max_slots=1, host_staging=0, max_fine_words=1 << 16)
    try:
        r.upload_silhouettes(0, full.cuda())
        r.reconstruct([0])
        with pytest.raises(fvv.FvvError) as e:
            r.counts(0)
        assert e.value.status == fvv.FVV_ERR_CAPACITY
        c = r.counts(0, allow_capacity=True)
        assert c["flags"] & 4 and c["n_rois"] == 0 and c["n_components"] == 1
        occ, tests = Oracle(rig).coarse(full.numpy())
        nx, ny, nz = rig.grid_dims()
        bits = unpack_rows(r.debug(0, fvv.FVV_DEBUG_COARSE_BITS).cpu().numpy().view(np.uint32), (nz, ny), nx)
        np.testing.assert_array_equal(bits, occ)
        assert c["tests_coarse"] == tests
        # the same rig recovers on a normal frame
        r.upload_silhouettes(0, fr.masks.cuda())
        r.reconstruct([0])
        c2 = r.counts(0)
        assert c2["flags"] == 0 and c2["n_rois"] == 1
    finally:
        r.close()


def test_vertex_capacity_overflow():
    from paper_1903_11785_gb300 import fvv
    rig, fr = make_frame("tiny", 0)
    r = fvv.Rig(rig, max_slots=1, host_staging=0, max_verts=1000)
    try:
        r.upload_silhouettes(0, fr.masks.cuda())
        r.reconstruct([0])
        c = r.counts(0, allow_capacity=True)
        assert c["flags"] & 8 and c["n_verts"] == 0
    finally:
        r.close()


def test_not_ready_and_bad_slots():
    from paper_1903_11785_gb300 import fvv
    rig, fr = make_frame("tiny", 0)
    r = fvv.Rig(rig, max_slots=2, host_staging=0, max_fine_words=1 << 16)
    try:
        with pytest.raises(fvv.FvvError) as e:
            r.reconstruct([0])
        assert e.value.status == fvv.FVV_ERR_NOT_READY
        r.upload_silhouettes(0, fr.masks.cuda())
        with pytest.raises(fvv.FvvError):
            r.reconstruct([0, 0])
        with pytest.raises(fvv.FvvError):
            r.reconstruct([5])
        with pytest.raises(fvv.FvvError):       # host masks need staging
            r.upload_silhouettes(1, fr.masks)
    finally:
        r.close()
