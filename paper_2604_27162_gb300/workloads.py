"""Seeded synthetic workloads of the hide-and-seek environment step.

This module only generates inputs -- environment parameter tables and the
served request stream -- and holds none of the step's arithmetic.  Both the
CUDA engine and the oracle receive the same tables from here; nothing in it
depends on either implementation.

Workload shapes (the paper's maps are PNG files that are not available, so
Bernoulli obstacle maps stand in for them; the paper's throughput table uses
1024 environments with 1, 5 and 10 agents, Table A.1):

  plain16   16 envs, 16x16, p=0.15, 1 seeker + 1 hider (r=2), cap 64, seed 0
  single1k  1024 envs, 32x32, p=0.15, 1 observed seeker (r=3) + 1 scripted
            hider, cap 256, seed 1, packed + unpacked observations
  ten1k     1024 envs, 32x32, p=0.2, 5 seekers (r=3) + 5 hiders (r=2),
            cap 256, seed 2
  uneven64k 65,536 envs with side in {8,16,24,32,48,64}, 1..16 agents (half
            seekers, rounded up), density uniform in [0.05, 0.30], radius in
            {1,2,3,4} (both teams), cap = 4 x side, seed 3
  served    Poisson request stream, 2,000 requests/s for 60 s, seed 4
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

TWO32 = 1 << 32

# Observation emission flags (which teams write observations).
OBS_SEEKERS = 1
OBS_HIDERS = 2


def density_threshold(p) -> int:
    """floor(p * 2^32) in exact rational arithmetic (p given as str or
    Fraction so that 0.15 means 15/100 exactly)."""
    q = Fraction(p) if not isinstance(p, float) else Fraction(str(p))
    if q < 0 or q > 1:
        raise ValueError("density outside [0, 1]")
    v = (q.numerator * TWO32) // q.denominator
    return min(v, TWO32 - 1) if q < 1 else TWO32 - 1


def env_desc(side, n_agents, n_seekers, r_seek, r_hide, cap, density, obs_teams=3):
    return {
        "side": int(side),
        "n_agents": int(n_agents),
        "n_seekers": int(n_seekers),
        "r_seek": int(r_seek),
        "r_hide": int(r_hide),
        "cap": int(cap),
        "density_thr": density_threshold(density) if not isinstance(density, int) else density,
        "obs_teams": int(obs_teams),
    }


def plain16():
    return {
        "name": "plain16",
        "n_envs": 16,
        "seed": 0,
        "descs": [env_desc(16, 2, 1, 2, 2, 64, "0.15")],
        "steps": 1000,
        "unpacked": False,
    }


def single1k():
    return {
        "name": "single1k",
        "n_envs": 1024,
        "seed": 1,
        "descs": [env_desc(32, 2, 1, 3, 3, 256, "0.15", OBS_SEEKERS)],
        "steps": 10000,
        "unpacked": True,
    }


def ten1k():
    return {
        "name": "ten1k",
        "n_envs": 1024,
        "seed": 2,
        "descs": [env_desc(32, 10, 5, 3, 2, 256, "0.2")],
        "steps": 10000,
        "unpacked": False,
    }


SIDES = (8, 16, 24, 32, 48, 64)


def uneven_descs(n_envs, param_seed=3):
    """Per-env parameter table of the uneven batch, drawn with numpy's PCG64
    from param_seed (an input table; both implementations receive it)."""
    rng = np.random.Generator(np.random.PCG64(param_seed))
    side = rng.choice(np.array(SIDES), size=n_envs)
    agents = rng.integers(1, 17, size=n_envs)
    lo = density_threshold("0.05")
    hi = density_threshold("0.30")
    thr = rng.integers(lo, hi + 1, size=n_envs)
    radius = rng.integers(1, 5, size=n_envs)
    descs = []
    for i in range(n_envs):
        A = int(agents[i])
        descs.append({
            "side": int(side[i]),
            "n_agents": A,
            "n_seekers": (A + 1) // 2,
            "r_seek": int(radius[i]),
            "r_hide": int(radius[i]),
            "cap": 4 * int(side[i]),
            "density_thr": int(thr[i]),
            "obs_teams": 3,
        })
    return descs


def uneven64k(n_envs=65536):
    return {
        "name": "uneven64k",
        "n_envs": n_envs,
        "seed": 3,
        "descs": uneven_descs(n_envs, 3),
        "steps": 1000,
        "unpacked": False,
    }


def served_requests(rate=2000.0, duration=60.0, seed=4, max_requests=None):
    """Request stream of the served workload: Poisson arrivals at `rate`/s
    over `duration` s; each request draws n_envs log-uniform in [64, 4096],
    agents uniform in 1..10, side in {16, 32, 64}, horizon log-uniform in
    [128, 1024] steps and its own 64-bit seed.  Density 0.15 and radius 3
    are fixed.  Uses numpy's PCG64 (an input generator, not the method)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    reqs = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        n_envs = int(np.floor(64.0 * np.exp(rng.uniform(0.0, np.log(64.0)))))
        agents = int(rng.integers(1, 11))
        side = int(rng.choice(np.array([16, 32, 64])))
        horizon = int(np.floor(128.0 * np.exp(rng.uniform(0.0, np.log(8.0)))))
        rseed = int(rng.integers(0, 2**63 - 1)) * 2 + int(rng.integers(0, 2))
        reqs.append({
            "id": len(reqs),
            "arrival": t,
            "n_envs": min(max(n_envs, 64), 4096),
            "seed": rseed,
            "steps": min(max(horizon, 128), 1024),
            "desc": env_desc(side, agents, (agents + 1) // 2, 3, 3, 256, "0.15"),
        })
        if max_requests is not None and len(reqs) >= max_requests:
            break
    return reqs


WORKLOADS = {
    "plain16": plain16,
    "single1k": single1k,
    "ten1k": ten1k,
    "uneven64k": uneven64k,
}
