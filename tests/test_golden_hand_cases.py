"""The oracle against the hand-worked cases in tests/golden/hand_cases.txt
(window bits, moves and rewards derived by hand from the paper's rules)."""
from __future__ import annotations

import os

import numpy as np

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _cases():
    cases, cur = [], None
    with open(os.path.join(HERE, "golden", "hand_cases.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, val = line.partition(" ")
            if key == "case":
                cur = {"name": val}
                cases.append(cur)
            else:
                cur[key] = val
    return cases


def _xy(s):
    pts = [tuple(int(v) for v in p.split(",")) for p in s.split()]
    return np.array([p[0] for p in pts]), np.array([p[1] for p in pts])


def _grid(c):
    S = int(c["side"])
    rows = c["grid"].split()
    assert len(rows) == S and all(len(r) == S for r in rows)
    return S, np.array([[int(ch) for ch in r] for r in rows], dtype=np.uint8).reshape(-1)


def test_hand_cases_cover_every_rule():
    names = [c["name"] for c in _cases()]
    assert {"obs_inside", "obs_corner", "obs_radius4_two_words", "obs_line_of_sight", "moves",
            "rewards", "central", "true_state", "fog", "fog_per_agent"} <= set(names)
    assert all("cite" in c for c in _cases())


def test_observation_windows():
    for c in _cases():
        if not c["name"].startswith("obs_"):
            continue
        S, grid = _grid(c)
        x, y = _xy(c["agents"])
        r = int(c["radius"])
        W = ((2 * r + 1) ** 2 + 63) // 64
        got = oracle.observe_agent(S, grid, int(c["seekers"]), x, y, int(c["observer"]), r, W,
                                   los=bool(int(c.get("los", "0"))))
        for p in range(3):
            want = [int(v) for v in c["plane%d" % p].split()]
            want += [0] * (W - len(want))
            assert [int(v) for v in got[p]] == want, (c["name"], p)


def test_moves():
    c = [c for c in _cases() if c["name"] == "moves"][0]
    S, grid = _grid(c)
    x, y = _xy(c["agents"])
    act = [int(v) for v in c["actions"].split()]
    nx, ny = oracle.move(S, grid, x, y, act)
    ex, ey = _xy(c["expect"])
    assert list(nx) == list(ex) and list(ny) == list(ey)


def test_rewards():
    c = [c for c in _cases() if c["name"] == "rewards"][0]
    x, y = _xy(c["agents"])
    got = oracle.reward(int(c["seekers"]), int(c["radius"]), x, y)
    assert list(got) == [int(v) for v in c["expect"].split()]


def test_line_of_sight_properties():
    """Without obstacles every window cell is visible; a full wall one row
    below the agent hides every cell two or more rows below it and leaves the
    cells straight below and diagonally adjacent visible."""
    S, r = 11, 4
    empty = np.zeros(S * S, np.uint8)
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            assert oracle.visible(S, empty, 5, 5, dx, dy)
    wall = np.zeros((S, S), np.uint8)
    wall[6, :] = 1
    wall = wall.reshape(-1)
    for dy in range(2, r + 1):
        for dx in range(-r, r + 1):
            assert not oracle.visible(S, wall, 5, 5, dx, dy), (dx, dy)
    for dx in (-1, 0, 1):
        assert oracle.visible(S, wall, 5, 5, dx, 1)
    # cells outside the grid block the view beyond them
    assert not oracle.visible(S, empty, 0, 5, -2, 0)
    assert oracle.visible(S, empty, 0, 5, -1, 0)


def test_centralized_observation():
    for c in _cases():
        if not c["name"].startswith("central"):
            continue
        S, grid = _grid(c)
        x, y = _xy(c["agents"])
        r = int(c["radius"])
        got = oracle.central_one(S, grid, int(c["seekers"]), r, r, int(c.get("teams", "3")), x, y)
        for p in range(4):
            assert [int(v) for v in got[p, :, 0]] == [int(v) for v in c["plane%d" % p].split()], (c["name"], p)


def test_centralized_observation_properties():
    """Seen = the union of the observing agents' windows (without line of
    sight); seen obstacles and agents are the map's restricted to it; with
    line of sight the seen plane only shrinks."""
    rng = np.random.default_rng(5)
    for _ in range(30):
        S = int(rng.integers(3, 20))
        grid = (rng.random(S * S) < 0.25).astype(np.uint8)
        A = int(rng.integers(1, 7))
        cells = rng.choice(S * S, size=A, replace=False)
        x, y = cells % S, cells // S
        ns, rs, rh, teams = int(rng.integers(0, A + 1)), int(rng.integers(0, 4)), int(rng.integers(0, 4)), int(rng.integers(0, 4))
        c = oracle.central_one(S, grid, ns, rs, rh, teams, x, y)
        seen = np.zeros((S, S), bool)
        for a in range(A):
            team = 0 if a < ns else 1
            if not (teams >> team) & 1:
                continue
            r = rs if team == 0 else rh
            seen[max(0, y[a] - r):y[a] + r + 1, max(0, x[a] - r):x[a] + r + 1] = True
        bits = lambda p: np.array([[(int(c[p, yy, xx // 64]) >> (xx % 64)) & 1 for xx in range(S)]
                                   for yy in range(S)], bool)
        assert np.array_equal(bits(0), seen)
        assert np.array_equal(bits(1), seen & grid.reshape(S, S).astype(bool))
        occ_s = np.zeros((S, S), bool)
        occ_h = np.zeros((S, S), bool)
        for a in range(A):
            (occ_s if a < ns else occ_h)[y[a], x[a]] = True
        assert np.array_equal(bits(2), seen & occ_s) and np.array_equal(bits(3), seen & occ_h)
        cl = oracle.central_one(S, grid, ns, rs, rh, teams | 4, x, y)
        assert not (bits(0) < np.array([[(int(cl[0, yy, xx // 64]) >> (xx % 64)) & 1 for xx in range(S)]
                                         for yy in range(S)], bool)).any()


def test_true_state_record():
    from paper_2604_27162_gb300 import workloads as W

    c = [c for c in _cases() if c["name"] == "true_state"][0]
    x, y = _xy(c["agents"])
    w = oracle.World(1, 1, [W.env_desc(int(c["side"]), len(x), int(c["seekers"]), 1, 1, 100, 0)])
    w.set_state(x, y, [int(c["ep_t"])], [0], 0)
    cells, ep_t = w.true_state()
    assert [int(v) for v in cells] == [int(v) for v in c["cells"].split()]
    assert [int(v) for v in ep_t] == [int(c["ep_t"])]


def test_true_state_against_full_view_central():
    """With radius 4 on a 4x4 grid every window covers the grid, so the
    centralized seeker and hider planes are exactly the true state's cells;
    the episode clock after k steps is k mod cap."""
    from paper_2604_27162_gb300 import workloads as W

    cap = 7
    descs = [W.env_desc(4, A, (A + 1) // 2, 4, 4, cap, "0.2") for A in (1, 3, 5, 6)]
    w = oracle.World(4, 9, descs)
    off = np.concatenate([[0], np.cumsum([d["n_agents"] for d in descs])])
    for k in range(1, 20):
        w.step()
        cells, ep_t = w.true_state()
        cen = w.central()
        assert [int(v) for v in ep_t] == [k % cap] * 4
        for e, d in enumerate(descs):
            S, ns = d["side"], d["n_seekers"]
            pl = cen[e * 4 * S:(e + 1) * 4 * S].reshape(4, S)
            sk = np.zeros(S, np.uint64)
            hd = np.zeros(S, np.uint64)
            for a in range(d["n_agents"]):
                v = int(cells[off[e] + a])
                cx, cy = v & 63, v >> 6
                assert 0 <= cx < S and 0 <= cy < S
                if a < ns:
                    sk[cy] |= np.uint64(1 << cx)
                else:
                    hd[cy] |= np.uint64(1 << cx)
            assert np.array_equal(pl[0], np.full(S, (1 << S) - 1, np.uint64))
            assert np.array_equal(pl[2], sk) and np.array_equal(pl[3], hd)


def _rows(m):
    """Rows of bits (bit x of row y) of one byte map [S][S]."""
    return [sum(int(v) << x for x, v in enumerate(row)) for row in m]


def test_fog_of_war_updates():
    c = [c for c in _cases() if c["name"] == "fog"][0]
    S, grid = _grid(c)
    r, ns, teams = int(c["radius"]), int(c["seekers"]), int(c["teams"])
    disc = np.zeros((1, S, S), np.uint8)
    for k in range(4):
        start, cells = c["update%d" % k].split(" ", 1)
        x, y = _xy(cells)
        fresh = oracle.fog_update(S, grid, ns, r, r, teams, False, x, y, int(start), disc)
        assert _rows(disc[0]) == [int(v) for v in c["disc%d" % k].split()], k
        assert _rows(fresh[0]) == [int(v) for v in c["fresh%d" % k].split()], k


def test_fog_of_war_per_agent_and_global():
    c = [c for c in _cases() if c["name"] == "fog_per_agent"][0]
    S, grid = _grid(c)
    r, ns, teams = int(c["radius"]), int(c["seekers"]), int(c["teams"])
    x, y = _xy(c["agents"])
    per = np.zeros((2, S, S), np.uint8)
    oracle.fog_update(S, grid, ns, r, r, teams, True, x, y, 1, per)
    glob = np.zeros((1, S, S), np.uint8)
    oracle.fog_update(S, grid, ns, r, r, teams, False, x, y, 1, glob)
    assert _rows(per[0]) == [int(v) for v in c["unit0"].split()]
    assert _rows(per[1]) == [int(v) for v in c["unit1"].split()]
    assert _rows(glob[0]) == [int(v) for v in c["global"].split()]
