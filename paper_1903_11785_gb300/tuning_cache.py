"""A JSON file of autotuned launch shapes, keyed by GPU and workload.

fvv_autotune times candidate launch shapes on the caller's own frames, which
takes a few seconds.  A process that serves the same rig on the same kind of
GPU as an earlier one can take the shapes that process picked instead:
`tuned()` looks the workload up in the file, applies the stored shapes with
fvv_set_tuning if it finds them, and otherwise autotunes and stores the
result.  The shapes never change an output of the library (only how fast it
gets there), so a stale or foreign entry costs speed, not correctness.

The key names the GPU model, the cameras (count and image sizes), the grid
(volume, coarse and fine steps), the surface rule and its steps, and the
number of slots a call takes, which decides how the tuned blocks per SM are
spread.  The file is rewritten whole through a temporary file and
os.replace, so a reader never sees half of it; a file that does not parse is
treated as empty and replaced at the next store.
"""
from __future__ import annotations

import json
import os
import tempfile

import numpy as np

VERSION = 1


def workload_key(scene_rig, n_slots: int, gpu_name: str) -> str:
    """The cache key of a rig's reconstructions of `n_slots` frames per call
    on the GPU model `gpu_name`."""
    sizes = sorted({(int(w), int(h)) for w, h in zip(np.asarray(scene_rig.width), np.asarray(scene_rig.height))})
    parts = [f"v{VERSION}", gpu_name.strip(), f"cams={scene_rig.n_cams}",
             "img=" + ",".join(f"{w}x{h}" for w, h in sizes),
             "vol=" + ",".join(f"{float(np.float32(x)):.6g}" for x in (*scene_rig.vol_min, *scene_rig.vol_max)),
             f"coarse={float(np.float32(scene_rig.coarse_m)):.6g}", f"fine={float(np.float32(scene_rig.fine_m)):.6g}",
             f"rule={getattr(scene_rig, 'surface_rule', 0)}", f"steps={scene_rig.bisect_steps}",
             f"oob={scene_rig.oob_policy}", f"slots={int(n_slots)}"]
    return "|".join(parts)


def load(path: str) -> dict:
    """All entries of the file (empty if it is missing or does not parse)."""
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    return data if isinstance(data, dict) else {}


def lookup(path: str, key: str):
    """The shapes stored under `key`, as fvv.Rig.set_tuning takes them, or None."""
    entry = load(path).get(key)
    return _from_json(entry) if isinstance(entry, dict) else None


def store(path: str, key: str, tuning: dict) -> None:
    """Add or replace the entry `key` (read-modify-write of the whole file)."""
    data = load(path)
    data[key] = _to_json(tuning)
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(prefix=".tuning.", dir=d)
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def tuned(rig, scene_rig, slots, path: str, gpu_name: str, stream=None):
    """Launch shapes for `rig` (an fvv.Rig built from `scene_rig`) when it
    reconstructs len(slots) frames per call: the stored ones, applied with
    set_tuning, or else autotuned on `slots` (which must hold reconstructed
    frames) and stored.  Returns (shapes, True if they came from the file)."""
    key = workload_key(scene_rig, len(slots), gpu_name)
    found = lookup(path, key)
    if found is not None:
        rig.set_tuning(found)
        return rig.get_tuning(), True
    shapes = rig.autotune(list(slots), stream=stream)
    store(path, key, shapes)
    return shapes, False


def _to_json(tuning: dict) -> dict:
    return {k: [int(x) for x in v] if isinstance(v, (tuple, list)) else int(v) for k, v in tuning.items()}


def _from_json(entry: dict) -> dict:
    return {k: tuple(v) if isinstance(v, list) else v for k, v in entry.items()}
