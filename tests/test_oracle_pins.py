"""Pins of the oracle against things other than itself (CPU only).

* Philox4x32-10: ATen's header-only Philox engine, compiled here and run as a
  black box, on random and corner counters/keys.
* Moves, rewards, observations: brute force on tiny grids against the
  independently written definition-level checker ``defcheck``.
* Statistics the definitions fix: action frequencies (chi-square), obstacle
  density, distinct and free start cells.
* Invariants over whole runs (paper Sec. 3.2: blocking tiles are impassable;
  Sec. 3.3: the window bounds what is seen; Sec. 4.2: a reset restores the
  pristine state): agents in bounds, on free cells and on distinct cells,
  plane popcounts bounded by the view area, planes pairwise disjoint, episode
  length equal to the cap, state after a reset equal to the state after
  create, env-range shards equal to the whole run.
"""
from __future__ import annotations

import itertools
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2604_27162_gb300 import workloads as W
from tests import defcheck


# --------------------------------------------------------------------------
# Philox4x32-10 against ATen's engine (black box).
# --------------------------------------------------------------------------
_ATEN_DRIVER = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdint>
int main() {
  unsigned c0, c1, c2, c3, k0, k1;
  while (std::scanf("%u %u %u %u %u %u", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
    uint64_t seed = (uint64_t)k0 | ((uint64_t)k1 << 32);
    uint64_t sub = (uint64_t)c2 | ((uint64_t)c3 << 32);
    uint64_t off = (uint64_t)c0 | ((uint64_t)c1 << 32);
    at::philox_engine e(seed, sub, off);
    unsigned a = e(), b = e(), c = e(), d = e();
    std::printf("%u %u %u %u\n", a, b, c, d);
  }
  return 0;
}
"""


def _aten_philox(cases, tmp_path):
    import torch

    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    src = tmp_path / "aten_philox.cpp"
    exe = tmp_path / "aten_philox"
    src.write_text(_ATEN_DRIVER)
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-I", inc, str(src), "-o", str(exe)])
    data = "\n".join(" ".join(str(int(v)) for v in c) for c in cases) + "\n"
    out = subprocess.run([str(exe)], input=data, capture_output=True, text=True, check=True)
    return [tuple(int(v) for v in line.split()) for line in out.stdout.strip().splitlines()]


def test_philox_matches_aten_engine(tmp_path):
    rng = np.random.default_rng(12345)
    cases = [(0, 0, 0, 0, 0, 0), (0xFFFFFFFF,) * 6, (1, 0, 0, 0, 0, 0), (0, 0, 0, 0, 1, 0),
             (0, 0, 0, 0, 0, 1), (0, 1, 0, 0, 0, 0), (0, 0, 1, 0, 0, 0), (0, 0, 0, 1, 0, 0)]
    cases += [tuple(int(v) for v in rng.integers(0, 2**32, size=6)) for _ in range(2000)]
    # counters of the shapes the engine uses: (t>>2, agent, env, stream)
    cases += [(t, a, e, s, 2, 0) for t in (0, 1, 2499) for a in (0, 9) for e in (0, 1023)
              for s in (0, 1, 2)]
    ref = _aten_philox(cases, tmp_path)
    for c, r in zip(cases, ref):
        got = tuple(int(v) for v in oracle.philox4x32_10(c[:4], c[4:]))
        assert got == r, (c, got, r)


# --------------------------------------------------------------------------
# Actions: uniform over 5 values, independent across agents and steps.
# --------------------------------------------------------------------------
def _chi2_sf_bound(counts, probs):
    counts = np.asarray(counts, dtype=np.float64)
    exp = counts.sum() * np.asarray(probs)
    return float(((counts - exp) ** 2 / exp).sum())


def test_action_frequencies_uniform():
    from scipy.stats import chi2

    seed = 7
    acts = np.array([oracle.action(seed, t, a, e) for t in range(400) for a in range(10)
                     for e in range(25)], dtype=np.int64)
    assert acts.min() == 0 and acts.max() == 4
    stat = _chi2_sf_bound(np.bincount(acts, minlength=5), [0.2] * 5)
    assert chi2.sf(stat, 4) > 1e-4, stat
    # joint of two neighbouring agents: 25 equiprobable cells
    a0 = np.array([oracle.action(seed, t, 0, e) for t in range(400) for e in range(25)])
    a1 = np.array([oracle.action(seed, t, 1, e) for t in range(400) for e in range(25)])
    stat = _chi2_sf_bound(np.bincount(a0 * 5 + a1, minlength=25), [1 / 25] * 25)
    assert chi2.sf(stat, 24) > 1e-4, stat
    # consecutive steps of one agent (steps within one Philox block and across)
    b0 = np.array([oracle.action(seed, t, 3, e) for t in range(0, 400, 1) for e in range(25)])
    b1 = np.array([oracle.action(seed, t + 1, 3, e) for t in range(0, 400, 1) for e in range(25)])
    stat = _chi2_sf_bound(np.bincount(b0 * 5 + b1, minlength=25), [1 / 25] * 25)
    assert chi2.sf(stat, 24) > 1e-4, stat


def test_action_mapping_is_multiply_shift():
    # word t&3 of the counter (t>>2, agent, env, 0), mapped by floor(u*5/2^32)
    seed = (3 << 32) | 11
    for t in (0, 1, 2, 3, 4, 7, 1001):
        u = oracle.philox4x32_10([t >> 2, 4, 9, 0], [11, 3])[t & 3]
        assert oracle.action(seed, t, 4, 9) == (int(u) * 5) >> 32


# --------------------------------------------------------------------------
# Moves: brute force against the definition-level checker.
# --------------------------------------------------------------------------
def _check_moves(S, grid, pos, act):
    x = [p[0] for p in pos]
    y = [p[1] for p in pos]
    nx, ny = oracle.move(S, grid.reshape(-1), x, y, act)
    got = list(zip(nx.tolist(), ny.tolist()))
    want = defcheck.moves(S, grid.tolist(), pos, act)
    assert got == want, (S, grid.tolist(), pos, act, got, want)
    assert defcheck.moves_are_legal(S, grid.tolist(), pos, act, got)


def test_moves_bruteforce_3x3_two_agents():
    S = 3
    cells = [(x, y) for y in range(S) for x in range(S)]
    masks = range(0, 1 << 9, 3)  # every third obstacle mask
    n = 0
    for mask in masks:
        grid = np.array([(mask >> i) & 1 for i in range(9)], np.uint8).reshape(S, S)
        free = [c for c in cells if not grid[c[1], c[0]]]
        for p0, p1 in itertools.permutations(free, 2):
            for a0 in range(5):
                for a1 in range(5):
                    _check_moves(S, grid, [p0, p1], [a0, a1])
                    n += 1
    assert n > 10000


def test_moves_sampled_three_to_six_agents():
    rng = np.random.default_rng(99)
    for _ in range(6000):
        S = int(rng.integers(2, 6))
        A = int(rng.integers(3, min(7, S * S) + 1))
        grid = (rng.random((S, S)) < 0.25).astype(np.uint8)
        cells = rng.permutation(S * S)[:A]
        grid.reshape(-1)[cells] = 0
        pos = [(int(c % S), int(c // S)) for c in cells]
        act = [int(v) for v in rng.integers(0, 5, size=A)]
        _check_moves(S, grid, pos, act)


def test_moves_chain_and_swap_are_blocked():
    grid = np.zeros((1, 4), np.uint8).reshape(1, 4)
    S = 4
    g = np.zeros((S, S), np.uint8)
    # agent 0 moves east into agent 1's cell while agent 1 also moves east: blocked
    nx, ny = oracle.move(S, g.reshape(-1), [0, 1], [0, 0], [3, 3])
    assert list(nx) == [0, 2] and list(ny) == [0, 0]
    # swap: both blocked
    nx, ny = oracle.move(S, g.reshape(-1), [0, 1], [0, 0], [3, 4])
    assert list(nx) == [0, 1]
    # equal targets: lowest index wins
    nx, ny = oracle.move(S, g.reshape(-1), [0, 2], [1, 1], [3, 4])
    assert list(nx) == [1, 2]
    del grid


# --------------------------------------------------------------------------
# Rewards: closed forms and brute force.
# --------------------------------------------------------------------------
def test_reward_closed_forms():
    # seeker at (5,5), r=3; hiders at Chebyshev 3 (seen) and 4 (not seen)
    x = [5, 8, 9, 2, 8]
    y = [5, 5, 5, 1, 8]
    rew = oracle.reward(1, 3, x, y)
    assert list(rew) == [2, -1, 0, 0, -1]
    # two seekers both seeing the same hider: counted once
    rew = oracle.reward(2, 1, [0, 2, 1], [0, 0, 1])
    assert list(rew) == [1, 1, -1]
    # no hiders: zero reward; lone seeker
    assert list(oracle.reward(1, 3, [4], [4])) == [0]
    # no seekers: nobody is seen
    assert list(oracle.reward(0, 3, [1, 2], [1, 1])) == [0, 0]


def test_reward_bruteforce_and_sums():
    rng = np.random.default_rng(5)
    for _ in range(3000):
        S = int(rng.integers(2, 12))
        A = int(rng.integers(1, min(12, S * S) + 1))
        ns = int(rng.integers(0, A + 1))
        r = int(rng.integers(0, 5))
        cells = rng.permutation(S * S)[:A]
        pos = [(int(c % S), int(c // S)) for c in cells]
        rew = oracle.reward(ns, r, [p[0] for p in pos], [p[1] for p in pos]).tolist()
        assert rew == defcheck.rewards(ns, r, pos)
        seen = -sum(rew[ns:])
        assert sum(rew[:ns]) == ns * seen


# --------------------------------------------------------------------------
# Observations: brute force against the padded-window checker.
# --------------------------------------------------------------------------
def test_observation_bruteforce():
    rng = np.random.default_rng(17)
    for S in (1, 2, 3, 5, 8):
        for r in (0, 1, 2, 3, 4):
            Wd = ((2 * r + 1) ** 2 + 63) // 64
            for _ in range(12):
                A = int(rng.integers(1, min(6, S * S) + 1))
                ns = int(rng.integers(0, A + 1))
                grid = (rng.random((S, S)) < 0.3).astype(np.uint8)
                cells = rng.permutation(S * S)[:A]
                grid.reshape(-1)[cells] = 0
                pos = [(int(c % S), int(c // S)) for c in cells]
                xs = [p[0] for p in pos]
                ys = [p[1] for p in pos]
                for a in range(A):
                    got = oracle.observe_agent(S, grid.reshape(-1), ns, xs, ys, a, r)
                    want = defcheck.observation(S, grid.tolist(), pos, ns, a, r)
                    for p in range(3):
                        assert [int(v) for v in got[p]] == defcheck.words_of(want[p], Wd), (
                            S, r, a, p)


def test_observation_every_cell_of_small_grid():
    # every agent position on a 6x6 grid, every radius, one fixed second agent
    S = 6
    grid = np.zeros((S, S), np.uint8)
    grid[2, 3] = 1
    grid[4, 0] = 1
    for r in range(1, 5):
        Wd = ((2 * r + 1) ** 2 + 63) // 64
        for cy in range(S):
            for cx in range(S):
                if grid[cy, cx] or (cx, cy) == (5, 5):
                    continue
                pos = [(cx, cy), (5, 5)]
                for ns in (1, 2):
                    got = oracle.observe_agent(S, grid.reshape(-1), ns, [cx, 5], [cy, 5], 0, r)
                    want = defcheck.observation(S, grid.tolist(), pos, ns, 0, r)
                    for p in range(3):
                        assert [int(v) for v in got[p]] == defcheck.words_of(want[p], Wd)


# --------------------------------------------------------------------------
# Generation.
# --------------------------------------------------------------------------
def test_generation_density_and_start_cells():
    c = W.ten1k()
    n_envs = 256
    w = oracle.World(n_envs, c["seed"], c["descs"])
    st = w.state()
    p = 0.2
    blocked = 0
    cells = 0
    for e in range(n_envs):
        g = w.grid(e)
        sx = st["sx"][e * 10:(e + 1) * 10]
        sy = st["sy"][e * 10:(e + 1) * 10]
        starts = set(zip(sx.tolist(), sy.tolist()))
        assert len(starts) == 10
        for (x, y) in starts:
            assert g[y, x] == 0
        mask = np.ones_like(g, dtype=bool)
        mask[sy, sx] = False
        blocked += int(g[mask].sum())
        cells += int(mask.sum())
    phat = blocked / cells
    sigma = (p * (1 - p) / cells) ** 0.5
    assert abs(phat - p) < 4 * sigma, (phat, sigma)


def test_density_threshold_exact():
    assert W.density_threshold("0.15") == 644245094
    assert W.density_threshold("0.2") == 858993459
    assert W.density_threshold("0") == 0
    # density 0 -> no obstacles at all; density 1 -> all but start cells
    d0 = W.env_desc(8, 3, 1, 1, 1, 10, 0)
    w = oracle.World(4, 9, [d0])
    assert all(w.grid(e).sum() == 0 for e in range(4))
    d1 = W.env_desc(8, 3, 1, 1, 1, 10, 2**32 - 1)
    w = oracle.World(4, 9, [d1])
    assert all(w.grid(e).sum() == 64 - 3 for e in range(4))


# --------------------------------------------------------------------------
# Whole runs: invariants, done / reset, determinism, shards.
# --------------------------------------------------------------------------
def _run_invariants(cfg, n_envs, n_steps, check_defcheck_every=7):
    descs = cfg["descs"]
    w = oracle.World(n_envs, cfg["seed"], descs)
    st0 = w.state()
    grids = [w.grid(e) for e in range(n_envs)]
    d = [descs[0 if len(descs) == 1 else e] for e in range(n_envs)]
    aoff = w.agent_off.astype(np.int64)
    ooff = w.obs_off.astype(np.int64)
    wpp = w.words_per_plane
    for t in range(n_steps):
        prev = w.state()
        out = w.step()
        st = w.state()
        for e in range(n_envs):
            p = d[e]
            S, A, ns = p["side"], p["n_agents"], p["n_seekers"]
            xs = st["x"][aoff[e]:aoff[e + 1]]
            ys = st["y"][aoff[e]:aoff[e + 1]]
            assert ((xs >= 0) & (xs < S) & (ys >= 0) & (ys < S)).all()
            assert not grids[e][ys, xs].any()
            assert len(set(zip(xs.tolist(), ys.tolist()))) == A
            done = int(out["done"][e])
            # episode length: done exactly every cap steps
            assert done == (3 if (t + 1) % p["cap"] == 0 else 0)
            if done:
                assert (xs == st0["x"][aoff[e]:aoff[e + 1]]).all()
                assert (ys == st0["y"][aoff[e]:aoff[e + 1]]).all()
            # obs invariants
            Wd = int(wpp[e])
            obs = out["obs"][ooff[e]:ooff[e + 1]].reshape(-1, 3, Wd) if Wd else None
            ai = 0
            for a in range(A):
                team = 0 if a < ns else 1
                if not (p["obs_teams"] >> team) & 1:
                    continue
                r = p["r_seek"] if team == 0 else p["r_hide"]
                V = (2 * r + 1) ** 2
                planes = [sum(int(v) << (64 * j) for j, v in enumerate(obs[ai, q]))
                          for q in range(3)]
                centre = 1 << (r * (2 * r + 1) + r)
                for q in range(3):
                    assert planes[q] >> V == 0
                    assert not planes[q] & centre
                assert not planes[0] & planes[1]
                assert not planes[0] & planes[2]
                assert not planes[1] & planes[2]
                if (e + t) % check_defcheck_every == 0:
                    pos = list(zip(xs.tolist(), ys.tolist()))
                    want = defcheck.observation(S, grids[e].tolist(), pos, ns, a, r)
                    assert planes == want
                ai += 1
            # rewards from the post-move, pre-reset positions
            if not done and (e + t) % check_defcheck_every == 0:
                pos = list(zip(xs.tolist(), ys.tolist()))
                assert out["reward"][aoff[e]:aoff[e + 1]].tolist() == defcheck.rewards(
                    ns, p["r_seek"], pos)
            # moves from the previous state and the exported actions
            if (e + t) % check_defcheck_every == 0:
                ppos = list(zip(prev["x"][aoff[e]:aoff[e + 1]].tolist(),
                                prev["y"][aoff[e]:aoff[e + 1]].tolist()))
                act = out["action"][aoff[e]:aoff[e + 1]].tolist()
                moved = defcheck.moves(S, grids[e].tolist(), ppos, act)
                if not done:
                    assert moved == list(zip(xs.tolist(), ys.tolist()))
                for a in range(A):
                    assert act[a] == oracle.action(cfg["seed"], t, a, e)
    return w


def test_run_invariants_ten_agents():
    c = W.ten1k()
    c = dict(c, descs=[dict(c["descs"][0], cap=40)])
    _run_invariants(c, 6, 130)


def test_run_invariants_plain16():
    _run_invariants(W.plain16(), 16, 140)


def test_run_invariants_uneven():
    descs = W.uneven_descs(24, 3)
    for d in descs:
        d["cap"] = min(d["cap"], 37)
    _run_invariants({"descs": descs, "seed": 3}, 24, 80)


def test_single_agent_unpacked_matches_packed():
    c = W.single1k()
    w = oracle.World(8, c["seed"], c["descs"])
    for _ in range(20):
        out = w.step(unpacked=True)
        obs = out["obs"].reshape(8, 1, 3, 1)
        unp = out["unpacked"].reshape(8, 1, 3, 7, 7)
        for e in range(8):
            for q in range(3):
                word = int(obs[e, 0, q, 0])
                bits = [(word >> k) & 1 for k in range(49)]
                assert unp[e, 0, q].reshape(-1).tolist() == bits
                assert word >> 49 == 0


def test_reset_restores_pristine_and_replays():
    c = W.ten1k()
    w = oracle.World(4, c["seed"], c["descs"])
    s0 = w.state()
    first = [w.step() for _ in range(9)]
    w.reset()
    s1 = w.state()
    for k in ("x", "y", "ep_t", "ep_idx"):
        assert (s0[k] == s1[k]).all()
    assert s1["t"] == 0
    again = [w.step() for _ in range(9)]
    for a, b in zip(first, again):
        for k in a:
            assert (a[k] == b[k]).all()


def test_shards_concatenate_to_whole_run():
    c = W.ten1k()
    n = 12
    whole = oracle.World(n, c["seed"], c["descs"])
    parts = [oracle.World(5, c["seed"], c["descs"], env_id_base=0),
             oracle.World(7, c["seed"], c["descs"], env_id_base=5)]
    for _ in range(30):
        o = whole.step()
        ps = [p.step() for p in parts]
        for k in o:
            assert (o[k] == np.concatenate([p[k] for p in ps])).all()


def test_digest_matches_step_outputs():
    c = W.plain16()
    w1 = oracle.World(3, 21, c["descs"])
    w2 = oracle.World(3, 21, c["descs"])
    res = w1.run_digest(70)
    rs = np.zeros(w2.n_agents_total, np.int64)
    eps = 0
    dig = 0
    M = (1 << 64) - 1

    def mix(z):  # splitmix64 output function (Steele, Lea, Flood 2014)
        z = (z + 0x9E3779B97F4A7C15) & M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)

    nw = w2.obs_words
    for s in range(70):
        o = w2.step()
        rs += o["reward"]
        eps += int((o["done"] & 1).sum())
        for j in range(nw):
            dig = (dig + mix(int(o["obs"][j]) ^ (s * nw + j))) & M
    assert (res["reward_sum"] == rs).all()
    assert res["episodes"] == eps == 3
    assert res["digest"] == dig


def test_splitmix64_known_answers():
    """The digest's mixing function reproduces the published splitmix64
    output sequence from state 0 (Steele, Lea, Flood 2014; the values in
    tests/golden/splitmix64_seed0.txt come with the reference implementation,
    not from this code)."""
    from tests.pin_battery import splitmix64_known_answers

    ka = splitmix64_known_answers()
    assert len(ka) == 5
    for z, v in ka:
        assert oracle.splitmix64(z) == v, (hex(z), hex(v))


def test_start_cells_and_obstacles_follow_keying():
    """Start cells and obstacles of worlds with odd sides and nonzero env-id
    bases, recomputed from the Philox block pinned against ATen."""
    from tests.pin_battery import _keying

    assert _keying(oracle.lib())


def test_invalid_params_rejected():
    with pytest.raises(ValueError):
        oracle.World(2, 0, [W.env_desc(0, 1, 1, 1, 1, 5, 0)])
    with pytest.raises(ValueError):
        oracle.World(2, 0, [W.env_desc(4, 2, 3, 1, 1, 5, 0)])
    with pytest.raises(ValueError):
        oracle.World(2, 0, [W.env_desc(4, 2, 1, 1, 1, 0, 0)])


def test_desynchronised_start():
    """Section 3.3 (last paragraph): with the desynchronised start the first
    episode of env e lasts cap - offset(e) steps, offsets spread uniformly over
    [0, cap), and every later episode lasts cap steps from the start cells."""
    cap = 16
    n = 4000
    descs = [W.env_desc(8, 3, 2, 1, 1, cap, "0.1")]
    plain = oracle.World(n, 21, descs)
    w = oracle.World(n, 21, descs, desync=True)
    s0, s1 = plain.state(), w.state()
    ep0, ep1 = s0["ep_t"].astype(np.int64), s1["ep_t"].astype(np.int64)
    assert np.array_equal(s0["sx"], s1["sx"]) and np.array_equal(s0["sy"], s1["sy"])  # same start cells
    assert (ep0 == 0).all() and ep1.min() >= 0 and ep1.max() < cap
    counts = np.bincount(ep1, minlength=cap)
    expected = n / cap
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert chi2 < 40.0, chi2  # 15 degrees of freedom, p ~ 5e-4
    ends = [[] for _ in range(n)]
    for t in range(3 * cap):
        d = w.step()["done"]
        for e in np.flatnonzero(d):
            ends[e].append(t)
            if len(ends[e]) == 1:  # the first reset puts the env back on its start cells
                st = w.state()
                sl = slice(3 * e, 3 * e + 3)
                assert np.array_equal(st["x"][sl], st["sx"][sl]) and np.array_equal(st["y"][sl], st["sy"][sl])
    for e in range(n):
        assert ends[e][0] == cap - 1 - ep1[e], e
        assert all(b - a == cap for a, b in zip(ends[e], ends[e][1:])), e


def _prestep_replay(seed, S, grid, sx, sy, n, env_id):
    """n pre-steps from (sx, sy) rebuilt from the pinned parts: Philox blocks
    of counter (tau / 4, agent, env, 4), word tau % 4 scaled to 0..4, and the
    simultaneous move rule."""
    x, y = np.array(sx, np.int32), np.array(sy, np.int32)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for tau in range(n):
        act = [(int(oracle.philox4x32_10((tau // 4, a, env_id, 4), key)[tau % 4]) * 5) >> 32 for a in range(len(x))]
        x, y = oracle.move(S, grid, x, y, np.array(act, np.uint8))
    return x, y


def test_desynchronised_start_steps_the_dynamics():
    """Section 3.3 (last paragraph): the envs are stepped stochastically at
    initialisation -- env e takes offset(e) moves from its start cells, with
    actions of their own Philox stream, before its first observation.  The
    positions equal a replay of those moves, stay legal (inside the grid, off
    obstacles, one agent per cell, within offset(e) cells of the start), an
    env with offset 0 stays on its start cells, and longer offsets carry the
    agents further on average."""
    cap, n, seed = 40, 300, 5
    A = 4
    descs = [W.env_desc(10, A, 2, 1, 1, cap, "0.15")]
    w = oracle.World(n, seed, descs, env_id_base=7, desync=True)
    st = w.state()
    x, y, sx, sy, off = st["x"], st["y"], st["sx"], st["sy"], st["ep_t"].astype(np.int64)
    dist = np.abs(x - sx) + np.abs(y - sy)
    moved = []
    for e in range(n):
        sl = slice(A * e, A * e + A)
        g = w.grid(e).reshape(10, 10)
        rx, ry = _prestep_replay(seed, 10, g, sx[sl], sy[sl], int(off[e]), 7 + e)
        assert np.array_equal(rx, x[sl]) and np.array_equal(ry, y[sl]), e
        assert ((x[sl] >= 0) & (x[sl] < 10) & (y[sl] >= 0) & (y[sl] < 10)).all()
        assert (g[y[sl], x[sl]] == 0).all()
        assert len(set(zip(x[sl].tolist(), y[sl].tolist()))) == A
        assert (dist[sl] <= off[e]).all()
        if off[e] == 0:
            assert (dist[sl] == 0).all()
        moved.append(dist[sl].mean())
    moved = np.array(moved)
    assert (off == 0).any() and moved[off >= 20].mean() > moved[off < 5].mean() + 1.0
    # the pre-step stream is not the step stream: counter word 3 is 4, not 0
    assert any(oracle.prestep_action(seed, t, 0, 7) != oracle.action(seed, t, 0, 7) for t in range(8))


def test_fog_of_war_equals_union_of_centralized_views():
    """The global discovery map is the OR of the centralized observation's
    seen plane over the episode so far, and the newly discovered plane is
    its difference to the previous step (the whole map at an episode start);
    per-agent maps OR to the global one, and each equals the seen plane of
    a centralized view of that agent alone (line of sight included)."""
    descs = [W.env_desc(9, 5, 3, 2, 1, 6, "0.25", 3),
             W.env_desc(12, 4, 2, 3, 2, 5, "0.3", 3 | 4),
             W.env_desc(7, 3, 1, 0, 2, 4, "0.2", 2),
             W.env_desc(10, 6, 3, 4, 4, 7, "0.2", 1 | 4)]
    n = len(descs)
    glob = oracle.World(n, 21, descs, fog=1)
    per = oracle.World(n, 21, descs, fog=2)
    grids = [glob.grid(e) for e in range(n)]
    acc = [None] * n
    done = np.ones(n, np.uint8)  # step -1 starts every episode
    for t in range(-1, 16):
        if t >= 0:
            done = glob.step()["done"]
            per.step()
        cen, fg, fp = glob.central(), glob.fog(), per.fog()
        st = glob.state()
        co = fo = po = ao = 0
        for e, d in enumerate(descs):
            S, A, ns = d["side"], d["n_agents"], d["n_seekers"]
            seen = cen[co:co + S]
            prev = np.zeros(S, np.uint64) if done[e] else acc[e]
            acc[e] = prev | seen
            assert np.array_equal(fg[fo:fo + S], acc[e]), (t, e)
            assert np.array_equal(fg[fo + S:fo + 2 * S], acc[e] & ~prev), (t, e)
            obs = [a for a in range(A) if (d["obs_teams"] >> (0 if a < ns else 1)) & 1]
            union = np.zeros(S, np.uint64)
            for j, a in enumerate(obs):
                m = fp[po + 2 * j * S:po + (2 * j + 1) * S]
                union |= m
                one = oracle.central_one(S, grids[e].reshape(-1), 1 if a < ns else 0, d["r_seek"], d["r_hide"],
                                         d["obs_teams"], st["x"][ao + a:ao + a + 1], st["y"][ao + a:ao + a + 1])
                if done[e]:
                    assert np.array_equal(m, one[0, :, 0]), (t, e, a)
                else:
                    assert not (one[0, :, 0] & ~m).any(), (t, e, a)  # this step's view is discovered
            assert np.array_equal(union, acc[e]), (t, e)
            co += 4 * S
            fo += 2 * S
            po += 2 * S * len(obs)
            ao += A
    assert (st["ep_idx"] > 0).all()  # every env went through an auto-reset
