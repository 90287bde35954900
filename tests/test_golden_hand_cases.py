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
            "rewards"} <= set(names)
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
