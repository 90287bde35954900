"""Python access to the plain-C oracle of the hide-and-seek environment step.

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product package
never imports this module, and this module imports nothing from the product
package: the two implementations share no code.  Every computation happens in
``hase_oracle.c`` (naive, single-threaded, index order); this file only builds
that library with gcc and marshals numpy arrays in and out of it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_DIR, "hase_oracle.c")
_LIB = os.path.join(_DIR, "libhase_oracle.so")


def build(force: bool = False) -> str:
    """Compile ``hase_oracle.c`` into ``libhase_oracle.so`` (plain gcc -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_DIR, "hase_oracle.h"))
    ):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", _SRC, "-o", tmp]
        )
        os.replace(tmp, _LIB)
    return _LIB


class HoEnv(C.Structure):
    _fields_ = [
        ("side", C.c_uint32),
        ("n_agents", C.c_uint32),
        ("n_seekers", C.c_uint32),
        ("r_seek", C.c_uint32),
        ("r_hide", C.c_uint32),
        ("cap", C.c_uint32),
        ("density_thr", C.c_uint32),
        ("obs_teams", C.c_uint32),
    ]


_lib = None


def load_library(path):
    """Load an oracle shared library and declare its signatures."""
    L = C.CDLL(path)
    P = C.c_void_p
    u32, u64 = C.c_uint32, C.c_uint64
    L.ho_philox4x32_10.argtypes = [P, P, P]
    L.ho_action.argtypes = [u64, u64, u32, u32]
    L.ho_action.restype = u32
    L.ho_prestep_action.argtypes = [u64, u32, u32, u32]
    L.ho_prestep_action.restype = u32
    L.ho_move.argtypes = [u32, P, u32, P, P, P, P, P]
    L.ho_reward.argtypes = [u32, u32, u32, P, P, P]
    L.ho_observe_agent.argtypes = [u32, P, u32, u32, P, P, u32, u32, u32, u32, P]
    L.ho_visible.argtypes = [u32, P, C.c_int32, C.c_int32, C.c_int32, C.c_int32]
    L.ho_visible.restype = C.c_int
    L.ho_create.argtypes = [u32, u32, u64, P, u32]
    L.ho_create.restype = P
    L.ho_destroy.argtypes = [P]
    L.ho_error.restype = C.c_char_p
    L.ho_reset.argtypes = [P]
    L.ho_set_desync.argtypes = [P, C.c_int]
    L.ho_central_words.argtypes = [P]
    L.ho_central_words.restype = u64
    L.ho_central.argtypes = [P, P]
    L.ho_central_one.argtypes = [u32, P, u32, u32, u32, u32, u32, P, P, P]
    L.ho_sizes.argtypes = [P, P, P, P]
    L.ho_offsets.argtypes = [P, P, P, P, P]
    L.ho_observe.argtypes = [P, P, P]
    L.ho_step.argtypes = [P, P, P, P, P, P]
    L.ho_state.argtypes = [P, P, P, P, P, P, P, P]
    L.ho_grid.argtypes = [P, u32, P]
    L.ho_true_state.argtypes = [P, P, P]
    L.ho_fog_units.argtypes = [u32, u32, u32, u32]
    L.ho_fog_units.restype = u32
    L.ho_fog_update.argtypes = [u32, P, u32, u32, u32, u32, u32, u32, P, P, u32, P, P]
    L.ho_set_fog.argtypes = [P, C.c_int]
    L.ho_fog_words.argtypes = [P]
    L.ho_fog_words.restype = u64
    L.ho_fog.argtypes = [P, P]
    L.ho_set_state.argtypes = [P, P, P, P, P, u64]
    L.ho_run_digest.argtypes = [P, u64, P, P, P]
    L.ho_splitmix64.argtypes = [u64]
    L.ho_splitmix64.restype = u64
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load_library(build())
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def env_array(descs):
    """Pack a list of dicts (keys as in ``HoEnv``) into a ctypes array."""
    arr = (HoEnv * len(descs))()
    for i, d in enumerate(descs):
        for k, _ in HoEnv._fields_:
            setattr(arr[i], k, int(d[k]))
    return arr


def philox4x32_10(ctr, key, L=None):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    (L or lib()).ho_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def action(seed, t, agent, env_id, L=None):
    return int((L or lib()).ho_action(seed, t, agent, env_id))


def prestep_action(seed, tau, agent, env_id, L=None):
    return int((L or lib()).ho_prestep_action(seed, tau, agent, env_id))


def splitmix64(z, L=None):
    return int((L or lib()).ho_splitmix64(z & 0xFFFFFFFFFFFFFFFF))


def move(S, grid, x, y, act, L=None):
    grid = np.ascontiguousarray(grid, dtype=np.uint8)
    x = np.ascontiguousarray(x, dtype=np.int32)
    y = np.ascontiguousarray(y, dtype=np.int32)
    act = np.ascontiguousarray(act, dtype=np.uint8)
    nx = np.zeros_like(x)
    ny = np.zeros_like(y)
    (L or lib()).ho_move(S, _p(grid), len(x), _p(x), _p(y), _p(act), _p(nx), _p(ny))
    return nx, ny


def reward(n_seekers, r_seek, x, y, L=None):
    x = np.ascontiguousarray(x, dtype=np.int32)
    y = np.ascontiguousarray(y, dtype=np.int32)
    rew = np.zeros(len(x), dtype=np.int32)
    (L or lib()).ho_reward(len(x), n_seekers, r_seek, _p(x), _p(y), _p(rew))
    return rew


def visible(S, grid, x, y, dx, dy, L=None):
    grid = np.ascontiguousarray(grid, dtype=np.uint8)
    return bool((L or lib()).ho_visible(S, _p(grid), x, y, dx, dy))


def central_one(S, grid, n_seekers, r_seek, r_hide, obs_teams, x, y, L=None):
    """Centralized observation of one env: array [4][S][ceil(S/64)]."""
    grid = np.ascontiguousarray(grid, dtype=np.uint8)
    x = np.ascontiguousarray(x, dtype=np.int32)
    y = np.ascontiguousarray(y, dtype=np.int32)
    rw = (S + 63) // 64
    out = np.zeros(4 * S * rw, dtype=np.uint64)
    (L or lib()).ho_central_one(S, _p(grid), len(x), n_seekers, r_seek, r_hide, obs_teams, _p(x), _p(y),
                                _p(out))
    return out.reshape(4, S, rw)


def fog_update(S, grid, n_seekers, r_seek, r_hide, obs_teams, per_agent, x, y, start, disc, L=None):
    """One fog-of-war update of one env (the discovery maps [units][S][S] as
    uint8, updated in place); returns the newly discovered cells."""
    L = L or lib()
    A = len(x)
    units = int(L.ho_fog_units(A, n_seekers, obs_teams, int(per_agent)))
    assert disc.shape == (units, S, S) and disc.dtype == np.uint8 and disc.flags["C_CONTIGUOUS"]
    fresh = np.zeros_like(disc)
    g = np.ascontiguousarray(grid, np.uint8)
    xs = np.ascontiguousarray(x, np.int32)
    ys = np.ascontiguousarray(y, np.int32)
    L.ho_fog_update(S, _p(g), A, n_seekers, r_seek, r_hide, obs_teams, int(per_agent), _p(xs), _p(ys),
                    int(start), _p(disc), _p(fresh))
    return fresh


def observe_agent(S, grid, n_seekers, x, y, a, r, W=None, L=None, los=False):
    if W is None:
        W = ((2 * r + 1) ** 2 + 63) // 64
    grid = np.ascontiguousarray(grid, dtype=np.uint8)
    x = np.ascontiguousarray(x, dtype=np.int32)
    y = np.ascontiguousarray(y, dtype=np.int32)
    out = np.zeros(3 * W, dtype=np.uint64)
    (L or lib()).ho_observe_agent(S, _p(grid), len(x), n_seekers, _p(x), _p(y), a, r, W, int(los), _p(out))
    return out.reshape(3, W)


class World:
    """A batch of environments stepped by the oracle, outputs as numpy."""

    def __init__(self, n_envs, seed, descs, env_id_base=0, L=None, desync=False, fog=0):
        self._L = L or lib()
        self._descs = env_array(descs)
        h = self._L.ho_create(n_envs, env_id_base, seed, C.cast(self._descs, C.c_void_p),
                              len(descs))
        if not h:
            raise ValueError(self._L.ho_error().decode())
        self._h = C.c_void_p(h)
        self.n_envs = n_envs
        a = np.zeros(1, np.uint64)
        o = np.zeros(1, np.uint64)
        u = np.zeros(1, np.uint64)
        self._L.ho_sizes(self._h, _p(a), _p(o), _p(u))
        self.n_agents_total = int(a[0])
        self.obs_words = int(o[0])
        self.unp_bytes = int(u[0])
        self.agent_off = np.zeros(n_envs + 1, np.uint64)
        self.obs_off = np.zeros(n_envs + 1, np.uint64)
        self.unp_off = np.zeros(n_envs + 1, np.uint64)
        self.words_per_plane = np.zeros(max(n_envs, 1), np.uint32)
        self._L.ho_offsets(self._h, _p(self.agent_off), _p(self.obs_off), _p(self.unp_off),
                           _p(self.words_per_plane))
        if desync:
            self._L.ho_set_desync(self._h, 1)
        if fog:  # 1 global, 2 per-agent discovery maps
            self._L.ho_set_fog(self._h, int(fog))

    def close(self):
        if getattr(self, "_h", None):
            self._L.ho_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        self._L.ho_reset(self._h)

    def observe(self, unpacked=False):
        obs = np.zeros(self.obs_words, np.uint64)
        unp = np.zeros(self.unp_bytes, np.uint8) if unpacked else None
        self._L.ho_observe(self._h, _p(obs), _p(unp))
        return (obs, unp) if unpacked else obs

    def step(self, unpacked=False, observe=True):
        """One step of every env; returns dict of obs, reward, done, action
        (and unpacked when asked).  observe=False skips the decentralized
        observation (its entry is then empty)."""
        obs = np.zeros(self.obs_words if observe else 0, np.uint64)
        rew = np.zeros(self.n_agents_total, np.int32)
        done = np.zeros(self.n_envs, np.uint8)
        act = np.zeros(self.n_agents_total, np.uint8)
        unp = np.zeros(self.unp_bytes, np.uint8) if unpacked else None
        self._L.ho_step(self._h, _p(obs) if observe else None, _p(rew), _p(done), _p(act), _p(unp))
        out = {"obs": obs, "reward": rew, "done": done, "action": act}
        if unpacked:
            out["unpacked"] = unp
        return out

    def central(self):
        """Centralized observation of the current state (all envs)."""
        out = np.zeros(max(1, int(self._L.ho_central_words(self._h))), np.uint64)
        self._L.ho_central(self._h, _p(out))
        return out[: int(self._L.ho_central_words(self._h))]

    def fog(self):
        """Fog-of-war maps of the current step: per env [units][2][side] rows
        (discovered, newly discovered)."""
        n = int(self._L.ho_fog_words(self._h))
        out = np.zeros(max(1, n), np.uint64)
        self._L.ho_fog(self._h, _p(out))
        return out[:n]

    def true_state(self):
        """True state of the current step (Sec. 3.3, modes 2, 4, 5): every
        agent's cell x | y << 6 and every env's episode clock."""
        cells = np.zeros(max(1, self.n_agents_total), np.uint16)
        ep_t = np.zeros(max(1, self.n_envs), np.uint32)
        self._L.ho_true_state(self._h, _p(cells), _p(ep_t))
        return cells[: self.n_agents_total], ep_t[: self.n_envs]

    def state(self):
        n = self.n_agents_total
        x = np.zeros(n, np.int32)
        y = np.zeros(n, np.int32)
        sx = np.zeros(n, np.int32)
        sy = np.zeros(n, np.int32)
        ep_t = np.zeros(self.n_envs, np.uint32)
        ep_idx = np.zeros(self.n_envs, np.uint32)
        t = np.zeros(1, np.uint64)
        self._L.ho_state(self._h, _p(x), _p(y), _p(sx), _p(sy), _p(ep_t), _p(ep_idx), _p(t))
        return {"x": x, "y": y, "sx": sx, "sy": sy, "ep_t": ep_t, "ep_idx": ep_idx,
                "t": int(t[0])}

    def set_state(self, x, y, ep_t, ep_idx, t):
        x = np.ascontiguousarray(x, np.int32)
        y = np.ascontiguousarray(y, np.int32)
        ep_t = np.ascontiguousarray(ep_t, np.uint32)
        ep_idx = np.ascontiguousarray(ep_idx, np.uint32)
        self._L.ho_set_state(self._h, _p(x), _p(y), _p(ep_t), _p(ep_idx), t)

    def grid(self, e):
        side = int(self._descs[0 if len(self._descs) == 1 else e].side)
        g = np.zeros(side * side, np.uint8)
        self._L.ho_grid(self._h, e, _p(g))
        return g.reshape(side, side)

    def run_digest(self, n_steps):
        rs = np.zeros(self.n_agents_total, np.int64)
        eps = np.zeros(1, np.uint64)
        dig = np.zeros(1, np.uint64)
        self._L.ho_run_digest(self._h, n_steps, _p(rs), _p(eps), _p(dig))
        return {"reward_sum": rs, "episodes": int(eps[0]), "digest": int(dig[0])}
