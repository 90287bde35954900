"""A fast battery of the oracle's pins, runnable against any build of the
oracle library (``python -m tests.pin_battery <libpath> <aten_driver>``).

Used by the mutation test: each planted mistake in the oracle must make at
least one of these checks fail, and the unmodified oracle must pass them all.
Prints one JSON list of the failed check names.
"""
from __future__ import annotations

import itertools
import json
import subprocess
import sys

import numpy as np

import oracle
from paper_2604_27162_gb300 import workloads as W
from tests import defcheck


def _philox(L, drv):
    rng = np.random.default_rng(1)
    cases = [tuple(int(v) for v in rng.integers(0, 2**32, size=6)) for _ in range(64)]
    cases.append((0, 0, 0, 0, 0, 0))
    data = "\n".join(" ".join(map(str, c)) for c in cases) + "\n"
    out = subprocess.run([drv], input=data, capture_output=True, text=True, check=True).stdout
    ref = [tuple(int(v) for v in ln.split()) for ln in out.strip().splitlines()]
    return all(tuple(int(v) for v in oracle.philox4x32_10(c[:4], c[4:], L=L)) == r
               for c, r in zip(cases, ref))


def _actions(L):
    from scipy.stats import chi2

    acts = np.array([oracle.action(5, t, a, e, L=L) for t in range(120) for a in range(6)
                     for e in range(12)])
    if acts.min() != 0 or acts.max() != 4:
        return False
    cnt = np.bincount(acts, minlength=5).astype(float)
    exp = cnt.sum() / 5
    if chi2.sf(((cnt - exp) ** 2 / exp).sum(), 4) <= 1e-4:
        return False
    # consecutive steps of one agent are independent (25 equiprobable pairs)
    b0 = np.array([oracle.action(5, t, 2, e, L=L) for t in range(200) for e in range(12)])
    b1 = np.array([oracle.action(5, t + 1, 2, e, L=L) for t in range(200) for e in range(12)])
    cnt = np.bincount(b0 * 5 + b1, minlength=25).astype(float)
    exp = cnt.sum() / 25
    if chi2.sf(((cnt - exp) ** 2 / exp).sum(), 24) <= 1e-4:
        return False
    # keying convention: word t&3 of the block at counter (t>>2, agent, env, 0)
    key = [5, 0]
    for t, a, e in ((0, 0, 0), (5, 3, 7), (10, 1, 2), (3, 9, 11)):
        u = int(oracle.philox4x32_10([t >> 2, a, e, 0], key, L=L)[t & 3])
        if oracle.action(5, t, a, e, L=L) != (u * 5) >> 32:
            return False
    return True


def _moves(L):
    rng = np.random.default_rng(2)
    S = 3
    cells = [(x, y) for y in range(S) for x in range(S)]
    for mask in range(0, 512, 37):
        grid = np.array([(mask >> i) & 1 for i in range(9)], np.uint8).reshape(S, S)
        free = [c for c in cells if not grid[c[1], c[0]]]
        for p0, p1 in itertools.permutations(free, 2):
            for a0, a1 in itertools.product(range(5), range(5)):
                nx, ny = oracle.move(S, grid.reshape(-1), [p0[0], p1[0]], [p0[1], p1[1]],
                                     [a0, a1], L=L)
                if list(zip(nx.tolist(), ny.tolist())) != defcheck.moves(
                        S, grid.tolist(), [p0, p1], [a0, a1]):
                    return False
    for _ in range(800):
        S = int(rng.integers(2, 6))
        A = int(rng.integers(3, min(6, S * S) + 1))
        grid = (rng.random((S, S)) < 0.25).astype(np.uint8)
        cc = rng.permutation(S * S)[:A]
        grid.reshape(-1)[cc] = 0
        pos = [(int(c % S), int(c // S)) for c in cc]
        act = [int(v) for v in rng.integers(0, 5, size=A)]
        nx, ny = oracle.move(S, grid.reshape(-1), [p[0] for p in pos], [p[1] for p in pos],
                             act, L=L)
        if list(zip(nx.tolist(), ny.tolist())) != defcheck.moves(S, grid.tolist(), pos, act):
            return False
    return True


def _rewards(L):
    rng = np.random.default_rng(3)
    if list(oracle.reward(1, 3, [5, 8, 9, 2, 8], [5, 5, 5, 1, 8], L=L)) != [2, -1, 0, 0, -1]:
        return False
    for _ in range(500):
        S = int(rng.integers(2, 12))
        A = int(rng.integers(1, min(10, S * S) + 1))
        ns = int(rng.integers(0, A + 1))
        r = int(rng.integers(0, 5))
        cc = rng.permutation(S * S)[:A]
        pos = [(int(c % S), int(c // S)) for c in cc]
        got = oracle.reward(ns, r, [p[0] for p in pos], [p[1] for p in pos], L=L).tolist()
        if got != defcheck.rewards(ns, r, pos):
            return False
    return True


def _observations(L):
    rng = np.random.default_rng(4)
    for S in (2, 5, 8):
        for r in (1, 2, 3, 4):
            Wd = ((2 * r + 1) ** 2 + 63) // 64
            for _ in range(6):
                A = int(rng.integers(2, min(6, S * S) + 1))
                ns = int(rng.integers(1, A))
                grid = (rng.random((S, S)) < 0.3).astype(np.uint8)
                cc = rng.permutation(S * S)[:A]
                grid.reshape(-1)[cc] = 0
                pos = [(int(c % S), int(c // S)) for c in cc]
                for a in range(A):
                    got = oracle.observe_agent(S, grid.reshape(-1), ns, [p[0] for p in pos],
                                               [p[1] for p in pos], a, r, L=L)
                    want = defcheck.observation(S, grid.tolist(), pos, ns, a, r)
                    for q in range(3):
                        if [int(v) for v in got[q]] != defcheck.words_of(want[q], Wd):
                            return False
    return True


def _generation(L):
    desc = W.ten1k()["descs"][0]
    n = 96
    w = oracle.World(n, 2, [desc], L=L)
    st = w.state()
    blocked = cells = pairs = both = 0
    for e in range(n):
        g = w.grid(e)
        sx = st["sx"][e * 10:(e + 1) * 10]
        sy = st["sy"][e * 10:(e + 1) * 10]
        if len(set(zip(sx.tolist(), sy.tolist()))) != 10 or g[sy, sx].any():
            return False
        m = np.ones_like(g, dtype=bool)
        m[sy, sx] = False
        blocked += int(g[m].sum())
        cells += int(m.sum())
        h = m[:, :-1] & m[:, 1:]
        both += int((g[:, :-1] & g[:, 1:])[h].sum())
        pairs += int(h.sum())
    p = 0.2
    if abs(blocked / cells - p) > 4 * (p * (1 - p) / cells) ** 0.5:
        return False
    q = p * p
    return abs(both / pairs - q) < 4 * (q * (1 - q) / pairs) ** 0.5


def _keying(L):
    """Start cells and obstacles recomputed from the Philox block (itself
    pinned against ATen's engine): start cell of agent a = floor(u S^2 / 2^32)
    with u = word 0 of counter (attempt, a, env, 2), row-major (x = cell mod S,
    y = cell div S), redrawn while taken; cell c is an obstacle iff word c mod 4
    of counter (c div 4, 0, env, 1) is below the threshold, start cells free.
    Odd sides and a nonzero env-id base make a transposed or shifted index
    visible."""
    for S, A, dens, seed, base in ((13, 5, "0.3", 11, 0), (32, 10, "0.2", 2, 1000),
                                   (7, 3, "0.5", (1 << 40) + 3, 77)):
        d = W.env_desc(S, A, (A + 1) // 2, 2, 2, 50, dens)
        n = 3
        w = oracle.World(n, seed, [d], env_id_base=base, L=L)
        st = w.state()
        key = (seed & 0xFFFFFFFF, seed >> 32)
        for e in range(n):
            env = base + e
            cells = []
            for a in range(A):
                att = 0
                while True:
                    u = int(oracle.philox4x32_10((att, a, env, 2), key, L=L)[0])
                    c = (u * S * S) >> 32
                    if c not in cells:
                        break
                    att += 1
                cells.append(c)
            sl = slice(e * A, (e + 1) * A)
            if [int(v) for v in st["sx"][sl]] != [c % S for c in cells]:
                return False
            if [int(v) for v in st["sy"][sl]] != [c // S for c in cells]:
                return False
            g = w.grid(e)
            for c in range(S * S):
                u = int(oracle.philox4x32_10((c >> 2, 0, env, 1), key, L=L)[c & 3])
                if int(g[c // S, c % S]) != (0 if c in cells else int(u < d["density_thr"])):
                    return False
    return True


def splitmix64_known_answers():
    """(state before the output, expected output) pairs of the published
    splitmix64 sequence from state 0 (tests/golden/splitmix64_seed0.txt)."""
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "splitmix64_seed0.txt")
    vals = [int(ln, 16) for ln in open(path) if ln.strip() and not ln.startswith("#")]
    gamma = 0x9E3779B97F4A7C15
    return [((k * gamma) & ((1 << 64) - 1), v) for k, v in enumerate(vals)]


def _digest(L):
    """The digest's mixing function against the published splitmix64
    outputs (the oracle's ho_splitmix64 adds the gamma itself)."""
    return all(oracle.splitmix64(z, L=L) == v for z, v in splitmix64_known_answers())


def _run(L):
    desc = dict(W.ten1k()["descs"][0], cap=20)
    n = 6
    w = oracle.World(n, 2, [desc], L=L)
    st0 = w.state()
    grids = [w.grid(e) for e in range(n)]
    for t in range(45):
        prev = w.state()
        out = w.step()
        st = w.state()
        for e in range(n):
            sl = slice(e * 10, (e + 1) * 10)
            xs, ys = st["x"][sl], st["y"][sl]
            d = int(out["done"][e])
            if d != (3 if (t + 1) % 20 == 0 else 0):
                return False
            if d and ((xs != st0["x"][sl]).any() or (ys != st0["y"][sl]).any()):
                return False
            act = out["action"][sl].tolist()
            ppos = list(zip(prev["x"][sl].tolist(), prev["y"][sl].tolist()))
            if not d and defcheck.moves(32, grids[e].tolist(), ppos, act) != list(
                    zip(xs.tolist(), ys.tolist())):
                return False
            if act != [oracle.action(2, t, a, e, L=L) for a in range(10)]:
                return False
    w.reset()
    s1 = w.state()
    return all((st0[k] == s1[k]).all() for k in ("x", "y", "ep_t", "ep_idx"))


def _modes(L):
    """Line of sight, the centralized observation, the desynchronised start
    and the true state (the hand-worked cases of tests/golden and their
    properties)."""
    from tests.test_golden_hand_cases import _cases, _grid, _xy

    cases = {c["name"]: c for c in _cases()}
    c = cases["obs_line_of_sight"]
    S, grid = _grid(c)
    x, y = _xy(c["agents"])
    got = oracle.observe_agent(S, grid, int(c["seekers"]), x, y, int(c["observer"]), int(c["radius"]), 1,
                               L=L, los=True)
    if [int(got[p, 0]) for p in range(3)] != [int(c["plane%d" % p]) for p in range(3)]:
        return False
    for name in ("central", "central_seekers_only"):
        c = cases[name]
        S, grid = _grid(c)
        x, y = _xy(c["agents"])
        r = int(c["radius"])
        got = oracle.central_one(S, grid, int(c["seekers"]), r, r, int(c.get("teams", "3")), x, y, L=L)
        for p in range(4):
            if [int(v) for v in got[p, :, 0]] != [int(v) for v in c["plane%d" % p].split()]:
                return False
    # desynchronised start: offset floor(u cap / 2^32), u = word 0 of Philox
    # counter (0, 0, env, 3); the first episode ends after cap - offset steps
    cap, n, seed = 9, 12, 77
    w = oracle.World(n, seed, [W.env_desc(8, 2, 1, 1, 1, cap, "0.1")], L=L, desync=True)
    key = (seed & 0xffffffff, seed >> 32)
    want = [(int(oracle.philox4x32_10((0, 0, e, 3), key, L=L)[0]) * cap) >> 32 for e in range(n)]
    if [int(v) for v in w.state()["ep_t"]] != want:
        return False
    first = [None] * n
    for t in range(cap):
        d = w.step()["done"]
        for e in range(n):
            if d[e] and first[e] is None:
                first[e] = t + 1
    if first != [cap - v for v in want]:
        return False
    # ... and the env took that many moves from its start cells, actions from
    # Philox counter (tau / 4, agent, env, 4), word tau % 4
    A, S = 3, 8
    w = oracle.World(n, seed, [W.env_desc(S, A, 1, 1, 1, cap, "0.1")], L=L, desync=True)
    st = w.state()
    for e in range(n):
        sl = slice(A * e, A * e + A)
        x, y = st["sx"][sl].astype(np.int32), st["sy"][sl].astype(np.int32)
        g = w.grid(e).reshape(S, S)
        for tau in range(int(st["ep_t"][e])):
            act = [(int(oracle.philox4x32_10((tau // 4, a, e, 4), key, L=L)[tau % 4]) * 5) >> 32 for a in range(A)]
            x, y = oracle.move(S, g, x, y, np.array(act, np.uint8), L=L)
        if not (np.array_equal(x, st["x"][sl]) and np.array_equal(y, st["y"][sl])):
            return False
    # true state: the hand case, and the full-view centralized planes
    c = cases["true_state"]
    x, y = _xy(c["agents"])
    w = oracle.World(1, 1, [W.env_desc(int(c["side"]), len(x), int(c["seekers"]), 1, 1, 100, 0)], L=L)
    w.set_state(x, y, [int(c["ep_t"])], [0], 0)
    cells, ep = w.true_state()
    if [int(v) for v in cells] != [int(v) for v in c["cells"].split()] or int(ep[0]) != int(c["ep_t"]):
        return False
    w = oracle.World(2, 4, [W.env_desc(4, 5, 3, 4, 4, 5, "0.2")], L=L)
    for k in range(1, 8):
        w.step()
        cells, ep = w.true_state()
        cen = w.central()
        if [int(v) for v in ep] != [k % 5] * 2:
            return False
        for e in range(2):
            pl = cen[e * 16:(e + 1) * 16].reshape(4, 4)
            occ = [[0] * 4 for _ in range(2)]
            for a in range(5):
                v = int(cells[e * 5 + a])
                occ[0 if a < 3 else 1][v >> 6] |= 1 << (v & 63)
            if [int(v) for v in pl[2]] != occ[0] or [int(v) for v in pl[3]] != occ[1]:
                return False
    # fog of war: the hand cases, and a run against the centralized views
    from tests.test_golden_hand_cases import _rows

    c = cases["fog"]
    S, grid = _grid(c)
    disc = np.zeros((1, S, S), np.uint8)
    for k in range(4):
        start, cl = c["update%d" % k].split(" ", 1)
        x, y = _xy(cl)
        fresh = oracle.fog_update(S, grid, 1, 1, 1, 1, False, x, y, int(start), disc, L=L)
        if _rows(disc[0]) != [int(v) for v in c["disc%d" % k].split()]:
            return False
        if _rows(fresh[0]) != [int(v) for v in c["fresh%d" % k].split()]:
            return False
    c = cases["fog_per_agent"]
    S, grid = _grid(c)
    x, y = _xy(c["agents"])
    per = np.zeros((2, S, S), np.uint8)
    oracle.fog_update(S, grid, 1, 1, 1, 3, True, x, y, 1, per, L=L)
    if _rows(per[0]) != [int(v) for v in c["unit0"].split()] or _rows(per[1]) != [int(v) for v in c["unit1"].split()]:
        return False
    d = W.env_desc(9, 4, 2, 2, 1, 5, "0.25", 3)
    w = oracle.World(1, 8, [d], L=L, fog=1)
    acc = None
    for t in range(12):
        done = w.step()["done"][0] if t else 1
        seen = w.central()[:9]
        prev = np.zeros(9, np.uint64) if done else acc
        acc = prev | seen
        f = w.fog()
        if not np.array_equal(f[:9], acc) or not np.array_equal(f[9:], acc & ~prev):
            return False
    return True


CHECKS = {
    "philox": None,
    "actions": _actions,
    "moves": _moves,
    "rewards": _rewards,
    "observations": _observations,
    "generation": _generation,
    "keying": _keying,
    "digest": _digest,
    "run": _run,
    "modes": _modes,
}


def battery(L, drv):
    failed = []
    for name, fn in CHECKS.items():
        try:
            ok = _philox(L, drv) if name == "philox" else fn(L)
        except Exception:  # noqa: BLE001 - a crash of a check is a failure
            ok = False
        if not ok:
            failed.append(name)
    return failed


if __name__ == "__main__":
    L = oracle.load_library(sys.argv[1])
    print(json.dumps(battery(L, sys.argv[2])))
