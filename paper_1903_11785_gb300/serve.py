"""Serving: a continuous-batching request loop over several camera rigs.

Requests (one synchronized multi-camera frame each) arrive from several rigs
at their own times.  Rigs whose calibration and reconstruction parameters are
the same share one library rig (a group), so requests from all of them are
batched together.  As the paper does (Sec. III-B), all device memory is taken
at start-up: every group gets an arena of frame slots, and the slot counts
divide a memory budget among the groups in proportion to the number of rigs
each serves.

What a request costs in memory is its slot.  A slot's capacities (fine-grid
words, vertices, triangles) default to worst cases derived from the volume,
most of which a real frame never uses; with `fit_caps` the server sizes them
from the frames it is given at start-up (twice the largest need seen), so
that more slots, and more requests in flight, fit the same budget.  A request
is admitted when its group has a free slot and the bytes of all slots in use
stay within the budget.  A frame that still exceeds a fitted capacity (the
device reports it; nothing is written out of bounds) is served again by an
overflow slot with the default capacities, kept beside each group.

On every pass the loop gathers each group's newly admitted requests into one
batch and issues, on one of the group's streams, the packing of their
silhouettes, one fvv_reconstruct over the batch and one fvv_colour (pinned
masks and RGB images are read in place by the kernels, so a slot needs no
staging); batches of different groups, and successive batches of one group
(on alternating streams, disjoint slots), run concurrently on the GPU.  A
slot is freed when its batch's completion event has fired.  Latency is
measured from a request's scheduled arrival to the completion event of its
colour pass, on the GPU clock.

Results do not depend on what else is in flight: every kernel reads and
writes only the slots of its own call.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np
import torch

from . import fvv


@dataclass
class Request:
    rid: int
    rig: int
    frame: int            # index into the rig's frame pool
    t_arrival: float      # seconds after the start of the run
    slot: int = -1
    t_admit: float = -1.0
    t_done: float = -1.0  # seconds after the start, from the GPU clock
    batch: int = -1
    group: int = -1       # the group (or overflow group) that served it
    overflowed: bool = False


@dataclass
class RigPool:
    """One rig's cameras, parameters and pool of frames in pinned host memory."""
    scene_rig: object
    masks: list           # per frame: (N,H,W) uint8 pinned
    rgb: list             # per frame: (N,H,W,3) uint8 pinned
    viewpoints: np.ndarray  # (F,3) float32


def _staging(pool, mask_copies: bool = False) -> int:
    """Host staging a rig's slots need: none when the pool's masks and RGB are
    pinned and the masks are read in place by the packing kernel, masks only
    when the RGB is pinned and the masks are copied (mask_copies, or not
    pinned), else masks and RGB."""
    if _rgb_pinned(pool):
        return 0 if _masks_pinned(pool) and not mask_copies else 2
    return 1


def _rgb_pinned(pool) -> bool:
    return all(t.is_pinned() for t in pool.rgb)


def _masks_pinned(pool) -> bool:
    return all(t.is_pinned() for t in pool.masks)


def slot_bytes(scene_rig, staging: int = 1, **caps) -> int:
    """Device bytes one more slot costs for this rig (with that host staging)."""
    a = fvv.fvv_query_arena(fvv.make_desc(scene_rig, 1, staging), fvv.make_params(scene_rig, **caps))
    b = fvv.fvv_query_arena(fvv.make_desc(scene_rig, 2, staging), fvv.make_params(scene_rig, **caps))
    return b - a


def calibration_key(rig) -> tuple:
    """What must agree for two rigs to share one library rig: cameras, image
    sizes and every reconstruction parameter."""
    return (np.asarray(rig.P, np.float32).tobytes(), np.asarray(rig.centre, np.float32).tobytes(),
            np.asarray(rig.width, np.int32).tobytes(), np.asarray(rig.height, np.int32).tobytes(),
            tuple(np.float32(rig.vol_min).tolist()), tuple(np.float32(rig.vol_max).tolist()),
            float(np.float32(rig.coarse_m)), float(np.float32(rig.fine_m)), rig.bisect_steps, rig.t_np, rig.t_nb,
            float(np.float32(rig.t_v)), rig.oob_policy, getattr(rig, "surface_rule", 0))


def fitted_caps(pool, staging: int, base_caps: dict) -> dict:
    """Capacities from a pool's frames: twice the largest fine-grid words,
    vertices, triangles and ROIs that any of them needs (reconstructed once,
    alone, with the default capacities)."""
    r = fvv.Rig(pool.scene_rig, max_slots=1, host_staging=staging, **base_caps)
    need = dict(max_fine_words=1, max_verts=1, max_tris=1, max_rois=1)
    try:
        for m in pool.masks:
            r.upload_silhouettes(0, m, in_place=staging == 0 and m.is_pinned())
            r.reconstruct([0])
            c = r.counts(0)
            need["max_fine_words"] = max(need["max_fine_words"], c["n_fine_words"])
            need["max_verts"] = max(need["max_verts"], c["n_verts"])
            need["max_tris"] = max(need["max_tris"], c["n_tris"])
            need["max_rois"] = max(need["max_rois"], c["n_rois"])
    finally:
        r.close()
    caps = dict(base_caps)
    caps["max_fine_words"] = min(1 << 26, max(1 << 16, 2 * need["max_fine_words"]))
    caps["max_verts"] = max(1 << 16, 2 * need["max_verts"])
    caps["max_tris"] = max(1 << 17, 2 * need["max_tris"])
    caps["max_rois"] = min(4096, max(64, 2 * need["max_rois"]))
    return caps


def poisson_schedule(n_rigs, rate_hz, n_requests, seed, pool_sizes):
    """Merged Poisson arrivals (rate_hz per rig), frames cycling through each pool."""
    rng = np.random.default_rng(seed)
    per = [[] for _ in range(n_rigs)]
    t = np.zeros(n_rigs)
    reqs = []
    while len(reqs) < n_requests:
        k = int(np.argmin(t))
        reqs.append((t[k], k, len(per[k]) % pool_sizes[k]))
        per[k].append(t[k])
        t[k] += rng.exponential(1.0 / rate_hz)
    reqs.sort()
    return [Request(rid=i, rig=k, frame=f, t_arrival=float(ta)) for i, (ta, k, f) in enumerate(reqs)]


class _Group:
    """One library rig serving the rigs (pools) that share its calibration."""

    def __init__(self, pools, members, n_slots, n_streams, caps, staging, check_caps):
        self.members = members                     # pool indices
        self.pools = pools
        first = pools[members[0]]
        self.rgb_in_place = _rgb_pinned(first)
        self.masks_in_place = staging == 0
        self.rig = fvv.Rig(first.scene_rig, max_slots=n_slots, host_staging=staging, **caps)
        self.slot_bytes = slot_bytes(first.scene_rig, staging, **caps)
        self.n_slots = n_slots
        self.check_caps = check_caps               # fitted capacities: read each result's flags
        self.free = list(range(n_slots))
        self.queue = []            # waiting requests
        self.pending = []          # admitted, not yet issued
        self.inflight = []         # (done event, requests)
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.turn = 0


class Server:
    def __init__(self, pools, budget_bytes: int, max_slots_per_group: int = 64, n_streams: int = 2, caps=None,
                 mask_copies: bool = False, fit_caps: bool = True):
        """Group the rigs by calibration, size each group's slots (fitted to
        its pool's frames when fit_caps), and divide the memory budget among
        the groups in proportion to the rigs each serves.  mask_copies:
        pinned masks are copied to the slots by the copy engines (which need
        no SMs) instead of being read in place by the packing kernel."""
        base_caps = dict(caps or {})
        self.budget = int(budget_bytes)
        keys, members = [], []
        for k, p in enumerate(pools):
            key = calibration_key(p.scene_rig)
            if key in keys:
                members[keys.index(key)].append(k)
            else:
                keys.append(key)
                members.append([k])
        self.pool_group = {k: gi for gi, mem in enumerate(members) for k in mem}
        staging = [_staging(pools[mem[0]], mask_copies) for mem in members]
        gcaps = [fitted_caps(pools[mem[0]], st, base_caps) if fit_caps else dict(base_caps)
                 for mem, st in zip(members, staging)]
        # overflow slots (default capacities) beside fitted ones come out of the budget first
        over_bytes = [slot_bytes(pools[mem[0]].scene_rig, st, **base_caps) if fit_caps else 0
                      for mem, st in zip(members, staging)]
        sizes = [slot_bytes(pools[mem[0]].scene_rig, st, **c) for mem, st, c in zip(members, staging, gcaps)]
        left = self.budget - sum(over_bytes)
        demand = sum(len(mem) * s for mem, s in zip(members, sizes))
        n = [int(min(max_slots_per_group, max(0, left) * len(mem) // max(1, demand))) for mem in members]
        if any(x < 1 for x in n):
            raise MemoryError("memory budget too small for one slot of every group")
        self.groups = [_Group(pools, mem, ns, n_streams, c, st, fit_caps)
                       for mem, ns, c, st in zip(members, n, gcaps, staging)]
        self.overflow = [_Group(pools, mem, 1, 1, base_caps, st, False) if fit_caps else None
                         for mem, st in zip(members, staging)]
        self.caps = gcaps
        self.slots = n
        self.in_flight_bytes = 0
        self.n_overflowed = 0
        self.read_stream = torch.cuda.Stream()     # result flags are read here, apart from the work

    def close(self):
        for g in self.groups + [o for o in self.overflow if o is not None]:
            g.rig.close()

    def describe(self) -> dict:
        return {"groups": [{"rigs": g.members, "slots": g.n_slots, "slot_gb": g.slot_bytes / 1e9} for g in self.groups],
                "budget_gb": self.budget / 1e9,
                "overflow_slot_gb": [o.slot_bytes / 1e9 if o else 0.0 for o in self.overflow],
                "caps": self.caps}

    def _issue(self, g: _Group, batch_id):
        reqs, g.pending = g.pending, []
        st = g.streams[g.turn % len(g.streams)]
        g.turn += 1
        slots = [q.slot for q in reqs]
        pools = g.pools
        with torch.cuda.stream(st):
            g.rig.upload_silhouettes_batch(slots, [pools[q.rig].masks[q.frame] for q in reqs], stream=st,
                                           in_place=g.masks_in_place)
            g.rig.reconstruct(slots, stream=st)
            rgb = [pools[q.rig].rgb[q.frame] for q in reqs]
            g.rig.colour(slots, rgb, np.stack([pools[q.rig].viewpoints[q.frame] for q in reqs]), stream=st,
                         in_place=g.rgb_in_place)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(st)
        for q in reqs:
            q.batch = batch_id
        g.inflight.append((ev, reqs))

    def run(self, requests, on_done=None, time_scale: float = 1.0):
        """Serve `requests` (arrival times divided by time_scale); returns them
        with slot, admission and completion times filled in.  on_done(group,
        request) is called, before its slot is freed, for every completed
        request (group.rig holds its results in request.slot)."""
        order = sorted(requests, key=lambda q: q.t_arrival)
        t0_event = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0_event.record()
        t0_event.synchronize()
        t0 = time.perf_counter()
        i, done, batch_id = 0, 0, 0
        everyone = list(enumerate(self.groups)) + [(gi, o) for gi, o in enumerate(self.overflow) if o is not None]
        while done < len(order):
            now = time.perf_counter() - t0
            while i < len(order) and order[i].t_arrival / time_scale <= now:
                self.groups[self.pool_group[order[i].rig]].queue.append(order[i])
                i += 1
            progressed = False
            for gi, g in everyone:
                # completions free slots (and their bytes of the budget)
                still = []
                for ev, reqs in g.inflight:
                    if not ev.query():
                        still.append((ev, reqs))
                        continue
                    t_done = t0_event.elapsed_time(ev) / 1000.0
                    for q in reqs:
                        c = g.rig.counts(q.slot, stream=self.read_stream, allow_capacity=True) if g.check_caps else None
                        if c is not None and c["flags"]:
                            # a fitted capacity was too small: serve it again with the defaults
                            q.overflowed = True
                            self.n_overflowed += 1
                            self.overflow[gi].queue.append(q)
                        else:
                            q.t_done = t_done
                            q.group = gi
                            if on_done is not None:
                                on_done(g, q)
                            done += 1
                        g.free.append(q.slot)
                        self.in_flight_bytes -= g.slot_bytes
                    progressed = True
                g.inflight = still
                # admission: a free slot of the group, within the memory budget
                while g.queue and g.free and self.in_flight_bytes + g.slot_bytes <= self.budget:
                    q = g.queue.pop(0)
                    q.slot = g.free.pop()
                    q.t_admit = time.perf_counter() - t0
                    self.in_flight_bytes += g.slot_bytes
                    g.pending.append(q)
                if g.pending:
                    self._issue(g, batch_id)
                    batch_id += 1
                    progressed = True
            if not progressed:
                nxt = order[i].t_arrival / time_scale if i < len(order) else None
                busy = any(g.inflight for _, g in everyone)
                if nxt is not None and nxt - (time.perf_counter() - t0) > 2e-4 and not busy:
                    time.sleep(min(nxt - (time.perf_counter() - t0), 1e-3))
                else:
                    time.sleep(5e-5)
        torch.cuda.synchronize()
        return order


def summarize(requests, time_scale: float = 1.0) -> dict:
    lat = np.array([(q.t_done - q.t_arrival / time_scale) * 1000.0 for q in requests])
    span = max(q.t_done for q in requests) - min(q.t_arrival / time_scale for q in requests)
    batches = len({q.batch for q in requests})
    return {"frames": len(requests), "throughput_fps": len(requests) / span, "latency_ms_p50": float(np.percentile(lat, 50)),
            "latency_ms_p99": float(np.percentile(lat, 99)), "latency_ms_max": float(lat.max()),
            "batches": batches, "mean_batch": len(requests) / max(1, batches),
            "overflowed": int(sum(q.overflowed for q in requests))}


def summarize_per_rig(requests, n_rigs, time_scale: float = 1.0) -> dict:
    out = {}
    for k in range(n_rigs):
        lat = np.array([(q.t_done - q.t_arrival / time_scale) * 1000.0 for q in requests if q.rig == k])
        if len(lat):
            out[k] = {"frames": int(len(lat)), "latency_ms_p50": float(np.percentile(lat, 50)),
                      "latency_ms_p99": float(np.percentile(lat, 99))}
    return out
