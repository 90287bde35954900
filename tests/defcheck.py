"""Second, independently written definition-level checker of the step rules.

Pure Python, written from the rules rather than from the oracle's code, with
different data structures (sets and dicts for the moves, a padded numpy
window for the observations).  The pin tests compare the oracle with these
functions by brute force on tiny inputs.

Rules (paper Sec. 3.2 blocking tiles, Sec. 3.3 decentralized observation,
Sec. 4.2 pristine reset; open points fixed by the repository's readings):
  * a move targets the neighbouring cell in the action's direction
    (1 N = row - 1, 2 S = row + 1, 3 E = column + 1, 4 W = column - 1);
  * it is valid iff the target is on the grid, not an obstacle and not the
    current cell of any agent; action 0 stays;
  * of the valid movers with one target only the lowest index moves;
  * a hider is seen iff a seeker is within Chebyshev distance r_seek;
  * the observation window of radius r is read row by row, outside cells are
    obstacles, the observer itself is not an ally.
"""
from __future__ import annotations

import numpy as np

STEP = {0: (0, 0), 1: (0, -1), 2: (0, 1), 3: (1, 0), 4: (-1, 0)}


def moves(S, grid, pos, act):
    """New positions (list of (x, y)) after one simultaneous move."""
    occupied = set(pos)
    wanted = []
    for (x, y), a in zip(pos, act):
        dx, dy = STEP[int(a)]
        tgt = (x + dx, y + dy)
        ok = (
            int(a) != 0
            and 0 <= tgt[0] < S
            and 0 <= tgt[1] < S
            and not grid[tgt[1]][tgt[0]]
            and tgt not in occupied
        )
        wanted.append(tgt if ok else None)
    first_claim = {}
    for i, tgt in enumerate(wanted):
        if tgt is not None and tgt not in first_claim:
            first_claim[tgt] = i
    out = []
    for i, tgt in enumerate(wanted):
        out.append(tgt if tgt is not None and first_claim[tgt] == i else pos[i])
    return out


def moves_are_legal(S, grid, pos, act, new):
    """Check an outcome against the rule statements one by one."""
    occupied = set(pos)
    if len(set(new)) != len(new):
        return False
    for i, ((x, y), a, n) in enumerate(zip(pos, act, new)):
        if n != (x, y):
            dx, dy = STEP[int(a)]
            if n != (x + dx, y + dy):
                return False
            if not (0 <= n[0] < S and 0 <= n[1] < S) or grid[n[1]][n[0]] or n in occupied:
                return False
            for j in range(i):
                ddx, ddy = STEP[int(act[j])]
                tj = (pos[j][0] + ddx, pos[j][1] + ddy)
                if (int(act[j]) != 0 and tj == n and 0 <= tj[0] < S and 0 <= tj[1] < S
                        and not grid[tj[1]][tj[0]] and tj not in occupied):
                    return False
    return True


def rewards(n_seekers, r_seek, pos):
    seekers = pos[:n_seekers]
    seen = [any(max(abs(h[0] - s[0]), abs(h[1] - s[1])) <= r_seek for s in seekers)
            for h in pos[n_seekers:]]
    n = sum(seen)
    return [n] * len(seekers) + [-1 if v else 0 for v in seen]


def observation(S, grid, pos, n_seekers, a, r):
    """Three planes as Python ints (bit k = window row * (2r+1) + column)."""
    D = 2 * r + 1
    pad = np.ones((S + 2 * r, S + 2 * r), dtype=np.int8)
    pad[r:r + S, r:r + S] = np.asarray(grid, dtype=np.int8)
    team = np.full((S + 2 * r, S + 2 * r), -1, dtype=np.int8)
    for b, (x, y) in enumerate(pos):
        if b != a:
            team[y + r, x + r] = 0 if b < n_seekers else 1
    x, y = pos[a]
    my_team = 0 if a < n_seekers else 1
    win_o = pad[y:y + D, x:x + D].reshape(-1)
    win_t = team[y:y + D, x:x + D].reshape(-1)
    planes = [win_o == 1, win_t == my_team, (win_t >= 0) & (win_t != my_team)]
    return [sum(1 << int(k) for k in np.flatnonzero(p)) for p in planes]


def words_of(value, W):
    return [(value >> (64 * j)) & 0xFFFFFFFFFFFFFFFF for j in range(W)]
