"""The autotuner's JSON cache (paper_1903_11785_gb300/tuning_cache.py): keys,
round trips, hits and misses, and files that are missing or damaged.  A fake
rig stands in for fvv.Rig, so no GPU is needed."""
import dataclasses
import json

from paper_1903_11785_gb300 import tuning_cache as tc
from synth import make_rig

SHAPES = {"coarse": (256, 64), "fine": (256, 32), "bisect": (128, 16), "zbuffer": (256, 64),
          "triangles": (64, 8), "fine_tile": (4, 8, 8), "zbuffer_cams": 2}


class FakeRig:
    """Records the calls tuned() makes; autotune 'picks' SHAPES."""

    def __init__(self):
        self.calls = []
        self.shapes = None

    def autotune(self, slots, stream=None):
        self.calls.append(("autotune", tuple(slots)))
        self.shapes = dict(SHAPES)
        return dict(SHAPES)

    def set_tuning(self, shapes):
        self.calls.append(("set_tuning",))
        self.shapes = dict(shapes)

    def get_tuning(self):
        return dict(self.shapes)


def test_keys_separate_gpus_workloads_and_batch_sizes():
    v = make_rig("volleyball")
    k = tc.workload_key(v, 64, "NVIDIA GB300")
    assert k == tc.workload_key(make_rig("volleyball"), 64, "NVIDIA GB300 ")
    assert k == tc.workload_key(dataclasses.replace(v, name="another rig of the same shape"), 64, "NVIDIA GB300")
    others = [tc.workload_key(v, 1, "NVIDIA GB300"), tc.workload_key(v, 64, "NVIDIA B200"),
              tc.workload_key(make_rig("judo"), 64, "NVIDIA GB300"),
              tc.workload_key(dataclasses.replace(v, fine_m=0.02), 64, "NVIDIA GB300"),
              tc.workload_key(dataclasses.replace(v, surface_rule=1), 64, "NVIDIA GB300"),
              tc.workload_key(dataclasses.replace(v, bisect_steps=12), 64, "NVIDIA GB300")]
    assert len(set(others)) == len(others) and k not in others


def test_miss_autotunes_and_stores_then_hit_applies(tmp_path):
    path = str(tmp_path / "sub" / "tuning.json")
    v = make_rig("volleyball")
    r1 = FakeRig()
    shapes, cached = tc.tuned(r1, v, [0, 1, 2, 3], path, "NVIDIA GB300")
    assert not cached and shapes == SHAPES and r1.calls == [("autotune", (0, 1, 2, 3))]
    r2 = FakeRig()
    shapes2, cached2 = tc.tuned(r2, v, [4, 5, 6, 7], path, "NVIDIA GB300")
    assert cached2 and r2.calls == [("set_tuning",)] and shapes2 == SHAPES
    # another batch size is another entry; both stay in the file
    r3 = FakeRig()
    assert not tc.tuned(r3, v, [0], path, "NVIDIA GB300")[1]
    data = json.load(open(path))
    assert len(data) == 2 and all(isinstance(e, dict) for e in data.values())
    assert tc.lookup(path, tc.workload_key(v, 4, "NVIDIA GB300")) == SHAPES


def test_missing_or_damaged_file_is_empty_and_replaced(tmp_path):
    path = str(tmp_path / "tuning.json")
    assert tc.load(path) == {} and tc.lookup(path, "x") is None
    open(path, "w").write("{not json")
    assert tc.load(path) == {}
    open(path, "w").write("[1, 2, 3]")
    assert tc.load(path) == {}
    tc.store(path, "k", SHAPES)
    assert tc.lookup(path, "k") == SHAPES
    # no temporary files are left beside it
    assert sorted(p.name for p in tmp_path.iterdir()) == ["tuning.json"]
