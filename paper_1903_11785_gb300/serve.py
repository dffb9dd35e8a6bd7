"""Serving: a continuous-batching request loop over several camera rigs.

Requests (one synchronized multi-camera frame each) arrive from several rigs
at their own times.  Every rig has a fixed set of frame slots in its arena,
sized at start-up so that all rigs together stay within a memory budget
(the paper takes all device memory at start-up, Sec. III-B); a request is
admitted when its rig has a free slot, otherwise it waits in that rig's
queue.  On every pass the loop gathers the requests admitted since the last
pass into one batch per rig and issues, on one of the rig's streams, the
packing of their silhouettes, one fvv_reconstruct
over the batch and one fvv_colour (pinned masks and RGB images are read in
place by the kernels, so a slot needs no staging); batches of different rigs, and
successive batches of one rig (on alternating streams, disjoint slots), run
concurrently on the GPU.  A slot is freed when its batch's completion event
has fired.  Latency is measured from a request's scheduled arrival to the
completion event of its colour pass, on the GPU clock.

Results do not depend on what else is in flight: every kernel reads and
writes only the slots of its own call.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

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


class _RigState:
    def __init__(self, pool: RigPool, n_slots: int, n_streams: int, caps: dict, mask_copies: bool):
        self.pool = pool
        self.rgb_in_place = _rgb_pinned(pool)
        self.masks_in_place = _staging(pool, mask_copies) == 0
        self.rig = fvv.Rig(pool.scene_rig, max_slots=n_slots, host_staging=_staging(pool, mask_copies), **caps)
        self.free = list(range(n_slots))
        self.queue = []            # waiting requests
        self.pending = []          # admitted, not yet issued
        self.inflight = []         # (done event, requests)
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.turn = 0


class Server:
    def __init__(self, pools, budget_bytes: int, max_slots_per_rig: int = 32, n_streams: int = 2, caps=None,
                 mask_copies: bool = False):
        """Give every rig an equal share of the memory budget, in whole slots.
        mask_copies: pinned masks are copied to the slots by the copy engines
        (which need no SMs) instead of being read in place by the packing
        kernel."""
        caps = dict(caps or {})
        share = budget_bytes // max(1, len(pools))
        self.rigs = []
        self.slots = []
        for p in pools:
            n = int(min(max_slots_per_rig, share // slot_bytes(p.scene_rig, _staging(p, mask_copies), **caps)))
            if n < 1:
                raise MemoryError("memory budget too small for one slot of a rig")
            self.slots.append(n)
            self.rigs.append(_RigState(p, n, n_streams, caps, mask_copies))

    def close(self):
        for r in self.rigs:
            r.rig.close()

    def _issue(self, r: _RigState, batch_id, t0_event):
        reqs, r.pending = r.pending, []
        st = r.streams[r.turn % len(r.streams)]
        r.turn += 1
        slots = [q.slot for q in reqs]
        with torch.cuda.stream(st):
            r.rig.upload_silhouettes_batch(slots, [r.pool.masks[q.frame] for q in reqs], stream=st,
                                           in_place=r.masks_in_place)
            r.rig.reconstruct(slots, stream=st)
            rgb = [r.pool.rgb[q.frame] for q in reqs]
            r.rig.colour(slots, rgb, np.stack([r.pool.viewpoints[q.frame] for q in reqs]), stream=st,
                         in_place=r.rgb_in_place)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(st)
        for q in reqs:
            q.batch = batch_id
        r.inflight.append((ev, reqs))

    def run(self, requests, on_done=None, time_scale: float = 1.0):
        """Serve `requests` (arrival times divided by time_scale); returns them
        with slot, admission and completion times filled in.  on_done(rig
        state, request) is called, before its slot is freed, for every
        completed request."""
        order = sorted(requests, key=lambda q: q.t_arrival)
        t0_event = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0_event.record()
        t0_event.synchronize()
        t0 = time.perf_counter()
        i, done, batch_id = 0, 0, 0
        while done < len(order):
            now = time.perf_counter() - t0
            while i < len(order) and order[i].t_arrival / time_scale <= now:
                self.rigs[order[i].rig].queue.append(order[i])
                i += 1
            progressed = False
            for r in self.rigs:
                # completions free slots
                still = []
                for ev, reqs in r.inflight:
                    if ev.query():
                        t_done = t0_event.elapsed_time(ev) / 1000.0
                        for q in reqs:
                            q.t_done = t_done
                            if on_done is not None:
                                on_done(r, q)
                            r.free.append(q.slot)
                        done += len(reqs)
                        progressed = True
                    else:
                        still.append((ev, reqs))
                r.inflight = still
                # admission: as slots allow
                while r.queue and r.free:
                    q = r.queue.pop(0)
                    q.slot = r.free.pop()
                    q.t_admit = time.perf_counter() - t0
                    r.pending.append(q)
                if r.pending:
                    self._issue(r, batch_id, t0_event)
                    batch_id += 1
                    progressed = True
            if not progressed:
                nxt = order[i].t_arrival / time_scale if i < len(order) else None
                if nxt is not None and nxt - (time.perf_counter() - t0) > 2e-4 and not any(r.inflight for r in self.rigs):
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
            "batches": batches, "mean_batch": len(requests) / max(1, batches)}
