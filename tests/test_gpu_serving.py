"""GPU tests of the run digest and of the rollout server (hase_serve.h),
through the C ABI: digests equal the oracle's; every served request's result
equals the oracle's run of that request and the same request served alone."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2604_27162_gb300 import hase
from paper_2604_27162_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _oracle_digest(req, skip=0):
    w = oracle.World(req["n_envs"], req["seed"], [req["desc"]])
    for _ in range(skip):
        w.step()
    return w.run_digest(req["steps"])


def small_requests(n, seed=7, rate=4000.0):
    """A scaled-down served stream: Poisson arrivals, a few to a few dozen
    envs, short horizons and short episodes (so resets happen)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t, reqs = 0.0, []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        agents = int(rng.integers(1, 11))
        reqs.append({
            "arrival": t,
            "seed": int(rng.integers(0, 2**62)) * 4 + 3,
            "n_envs": int(rng.integers(3, 40)),
            "steps": int(rng.integers(8, 70)),
            "desc": W.env_desc(int(rng.choice([8, 16, 32])), agents, (agents + 1) // 2, 3,
                               int(rng.integers(1, 4)), int(rng.integers(5, 40)), "0.15"),
        })
    return reqs


def test_digest_matches_oracle():
    c = W.ten1k()
    descs = [dict(c["descs"][0], cap=23)]
    eng = hase.Engine(20, c["seed"], descs, ring_steps=64)
    eng.step(50)
    dig, eps, rs, err, per_agent = eng.digest(50, per_agent=True)
    w = oracle.World(20, c["seed"], descs)
    ref = w.run_digest(50)
    assert err == 0
    assert dig == ref["digest"] and eps == ref["episodes"]
    assert rs == int(ref["reward_sum"].sum())
    assert np.array_equal(per_agent, ref["reward_sum"])
    eng.close()


def test_digest_of_ring_tail_matches_oracle():
    descs = W.uneven_descs(12, 9)
    eng = hase.Engine(12, 5, descs, ring_steps=16)
    eng.step(41)
    dig, eps, rs, err = eng.digest(16)
    w = oracle.World(12, 5, descs)
    for _ in range(25):
        w.step()
    ref = w.run_digest(16)
    assert (dig, eps, rs, err) == (ref["digest"], ref["episodes"], int(ref["reward_sum"].sum()), 0)
    with pytest.raises(hase.HaseError):
        eng.digest(17)  # longer than the ring
    eng.close()


def test_served_results_equal_oracle_and_alone():
    reqs = small_requests(48)
    budget = sum(hase.hase_request_bytes(r) for r in reqs)
    res, stats = hase.hase_serve(reqs, budget, n_streams=8, time_scale=1.0)
    assert all(r["status"] == hase.HASE_OK for r in res)
    assert stats["peak_inflight"] > 1, "no overlap: the test does not exercise the mix"
    for i in (0, 7, 23, 47):
        ref = _oracle_digest(reqs[i])
        assert res[i]["digest"] == ref["digest"], i
        assert res[i]["episodes"] == ref["episodes"], i
        assert res[i]["reward_sum"] == int(ref["reward_sum"].sum()), i
    for i in (3, 11, 30):
        alone = dict(reqs[i], arrival=0.0)
        r1, _ = hase.hase_serve([alone], budget, n_streams=1, time_scale=0.0)
        for k in ("digest", "episodes", "reward_sum", "status"):
            assert r1[0][k] == res[i][k], (i, k)
        assert res[i]["finished"] >= res[i]["admitted"] >= reqs[i]["arrival"] - 1e-3


def test_serving_respects_budget_and_rejects_oversize():
    reqs = small_requests(24, seed=8)
    sizes = [hase.hase_request_bytes(r) for r in reqs]
    budget = int(max(sizes) * 1.5)
    big = dict(reqs[-1], arrival=reqs[-1]["arrival"] + 1e-4, n_envs=4000, steps=1000)
    res, stats = hase.hase_serve(reqs + [big], budget, n_streams=4, time_scale=0.0)
    assert all(r["status"] == hase.HASE_OK for r in res[:-1])
    assert res[-1]["status"] == hase.HASE_ENOMEM and stats["rejected"] == 1
    assert stats["peak_bytes"] <= budget
    for i in (0, 5, 17):
        ref = _oracle_digest(reqs[i])
        assert res[i]["digest"] == ref["digest"]


def test_server_shared_batches_equal_oracle_and_alone():
    """Requests submitted from two threads while the server runs share
    batches (one handle, every step launch) and still give the oracle's
    result of each request run alone."""
    import threading

    reqs = small_requests(60, seed=11)
    budget = 4 * sum(hase.hase_request_bytes(r) for r in reqs)
    srv = hase.Server(budget, n_streams=4, max_inflight=256)
    ids = [None] * len(reqs)

    def submit(part):
        for i in part:
            ids[i] = srv.submit(reqs[i])

    threads = [threading.Thread(target=submit, args=(range(k, len(reqs), 2),)) for k in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    res = [srv.poll(rid, timeout_s=60.0) for rid in ids]
    stats = srv.stats()
    srv.shutdown()
    srv.close()
    assert all(r is not None and r["status"] == hase.HASE_OK for r in res)
    assert stats["requests"] == len(reqs) and stats["batches"] < len(reqs)
    assert max(r["batch_size"] for r in res) > 1, "no request shared a batch"
    for i in range(0, len(reqs), 6):
        ref = _oracle_digest(reqs[i])
        assert (res[i]["digest"], res[i]["episodes"], res[i]["reward_sum"]) == (
            ref["digest"], ref["episodes"], int(ref["reward_sum"].sum())), i
        assert res[i]["finished"] >= res[i]["admitted"] >= res[i]["submitted"]
    alone = hase.Server(budget, n_streams=1, max_batch=1)  # every request its own handle
    for i in (1, 8, 33):
        r1 = alone.poll(alone.submit(reqs[i]), timeout_s=60.0)
        assert r1["batch_size"] == 1
        for k in ("digest", "episodes", "reward_sum", "status"):
            assert r1[k] == res[i][k], (i, k)
    alone.close()


def test_server_status_codes():
    reqs = small_requests(8, seed=12)
    long = dict(reqs[0], n_envs=2000, steps=4000)
    budget = int(hase.hase_request_bytes(long) * 1.2)
    srv = hase.Server(budget, n_streams=1, max_inflight=4, queue_capacity=1)
    import time

    first = srv.submit(long)
    assert srv.poll(first, timeout_s=0.0) is None  # HASE_ETIMEOUT: not finished yet
    t = time.time()
    while srv.stats()["peak_inflight"] < 1:  # admitted (requests under admission count as queued)
        assert time.time() - t < 30
        time.sleep(1e-3)
    srv.submit(dict(long, seed=5))  # waits in the queue for memory
    busy = 0
    for r in reqs[1:]:
        try:
            srv.submit(r)
        except hase.HaseError as e:
            assert e.status == hase.HASE_EBUSY
            busy += 1
    assert busy > 0, "the one-slot queue never filled"
    with pytest.raises(hase.HaseError) as ei:  # an invalid request
        srv.submit(dict(reqs[1], desc=dict(reqs[1]["desc"], side=99)))
    assert ei.value.status == hase.HASE_EINVAL
    big = srv.submit(dict(long, n_envs=4000, steps=8000))  # never fits: finished at once
    assert srv.poll(big, timeout_s=1.0)["status"] == hase.HASE_ENOMEM
    with pytest.raises(hase.HaseError):
        srv.poll(big)  # already collected
    assert srv.poll(first, timeout_s=120.0)["status"] == hase.HASE_OK
    srv.shutdown()  # finishes the queued request
    with pytest.raises(hase.HaseError) as ei:
        srv.submit(reqs[2])
    assert ei.value.status == hase.HASE_ESTATE
    srv.close()
