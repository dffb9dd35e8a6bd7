"""Host-side logic of the serving loop (paper_1903_11785_gb300/serve.py) that
needs no GPU: the seeded Poisson arrival schedule, the key under which rigs
share one library rig (and so one batch), and the latency and throughput
summary."""
import dataclasses

import numpy as np
import pytest

from synth import ABSTAIN, make_rig


@pytest.fixture(scope="module")
def serve():
    # serve.py imports the library binding, which needs libfvv.so (built
    # here for sm_103a; nothing runs on a GPU)
    from paper_1903_11785_gb300.build import build
    build()
    from paper_1903_11785_gb300 import serve as mod
    return mod


def test_poisson_schedule_rates_order_and_frame_cycling(serve):
    rate, n_rigs, pools = 30.0, 4, [8, 8, 5, 3]
    reqs = serve.poisson_schedule(n_rigs, rate, 8000, seed=7, pool_sizes=pools)
    assert len(reqs) == 8000
    assert [q.rid for q in reqs] == list(range(8000))
    t = np.array([q.t_arrival for q in reqs])
    assert np.all(np.diff(t) >= 0.0) and t[0] == 0.0
    horizon = t[-1]
    for k in range(n_rigs):
        mine = [q for q in reqs if q.rig == k]
        # the rigs' arrivals are merged Poisson streams: over the schedule's
        # span each rig has rate * span of them, within 5 standard deviations,
        # and its frames cycle through its pool in order
        assert abs(len(mine) - rate * horizon) < 5.0 * np.sqrt(rate * horizon)
        assert [q.frame for q in mine] == [i % pools[k] for i in range(len(mine))]
        # exponential gaps of mean 1 / rate: the sample mean is within 5 standard errors
        gaps = np.diff([q.t_arrival for q in mine])
        assert abs(gaps.mean() - 1.0 / rate) < 5.0 * (1.0 / rate) / np.sqrt(len(gaps))
        assert gaps.min() >= 0.0
    # the same seed gives the same schedule, another seed another one
    again = serve.poisson_schedule(n_rigs, rate, 8000, seed=7, pool_sizes=pools)
    assert [(q.rig, q.frame, q.t_arrival) for q in again] == [(q.rig, q.frame, q.t_arrival) for q in reqs]
    other = serve.poisson_schedule(n_rigs, rate, 8000, seed=8, pool_sizes=pools)
    assert [q.t_arrival for q in other] != [q.t_arrival for q in reqs]


def test_calibration_key_groups_only_identical_rigs(serve):
    key = serve.calibration_key
    v = make_rig("volleyball")
    assert key(v) == key(make_rig("volleyball"))
    assert key(v) == key(dataclasses.replace(v, name="second volleyball rig"))
    assert key(v) != key(make_rig("judo"))
    moved = v.P.copy()
    moved[3, 0, 3] = np.nextafter(moved[3, 0, 3], np.float32(np.inf))
    for other in (dataclasses.replace(v, P=moved), dataclasses.replace(v, t_v=0.25),
                  dataclasses.replace(v, bisect_steps=9), dataclasses.replace(v, oob_policy=ABSTAIN),
                  dataclasses.replace(v, surface_rule=1), dataclasses.replace(v, fine_m=0.02),
                  dataclasses.replace(v, t_np=9)):
        assert key(other) != key(v)


def _done(serve, rid, rig, t_arrival, t_done, batch):
    q = serve.Request(rid=rid, rig=rig, frame=0, t_arrival=t_arrival)
    q.t_done, q.batch = t_done, batch
    return q


def test_summary_latency_percentiles_throughput_and_batches(serve):
    # 100 requests 10 ms apart, each done 1 ms + (rid % 10) * 0.1 ms after it
    # arrived; ten requests per batch
    reqs = [_done(serve, i, i % 2, 0.01 * i, 0.01 * i + 1e-3 + (i % 10) * 1e-4, i // 10) for i in range(100)]
    s = serve.summarize(reqs)
    lat = np.array([1.0 + (i % 10) * 0.1 for i in range(100)])
    assert s["frames"] == 100 and s["batches"] == 10 and s["mean_batch"] == 10.0
    assert s["latency_ms_p50"] == pytest.approx(np.percentile(lat, 50))
    assert s["latency_ms_p99"] == pytest.approx(np.percentile(lat, 99))
    assert s["latency_ms_max"] == pytest.approx(1.9)
    assert s["throughput_fps"] == pytest.approx(100 / (0.99 + 1e-3 + 9e-4))
    per = serve.summarize_per_rig(reqs, 3)
    assert set(per) == {0, 1} and per[0]["frames"] == per[1]["frames"] == 50
    # arrival times are scaled as the loop scaled them
    s2 = serve.summarize([_done(serve, 0, 0, 2.0, 1.0015, 0)], time_scale=2.0)
    assert s2["latency_ms_p50"] == pytest.approx(1.5)
