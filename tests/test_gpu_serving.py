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
