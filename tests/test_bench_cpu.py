"""CPU checks of the benchmark's bookkeeping: the algorithmic bytes of every
optional mode against hand-worked figures for the default workload, and the
flags and descriptors each mode applies.  No GPU."""
from __future__ import annotations

import bench
from paper_2604_27162_gb300 import hase
from paper_2604_27162_gb300 import workloads as W

# 1024 envs, 32 x 32, 5 seekers (r 3) + 5 hiders (r 2), both teams observe:
# obs 10 agents x 3 planes x 1 word x 8 B = 240, rewards 10 x 4 = 40, done 1;
# true state 10 cells x 2 B + clock 4 B = 24; centralized 4 planes x 32 rows
# x 8 B = 1024; fog 2 planes x 32 rows x 8 B = 512 a unit (1, or 10 per agent).
HAND = {
    "default": 281, "los": 281, "desync": 281,
    "state": 281 + 24,
    "central": 41 + 1024,
    "central-state": 41 + 1024 + 24,
    "state-only": 41 + 24,
    "void": 41,
    "fog": 281 + 512,
    "fog-agent": 281 + 10 * 512,
}


def test_mode_bytes_match_hand_worked_figures():
    c = W.ten1k()
    assert set(HAND) == set(bench.MODES)
    for mode, want in HAND.items():
        cc, flags = bench.apply_mode(c, mode)
        got = bench.algorithmic_bytes_per_env_step(cc["descs"], 1, cc["unpacked"], flags)
        assert got == want, (mode, got, want)


def test_mode_flags_and_descriptors():
    c = W.ten1k()
    cc, flags = bench.apply_mode(c, "los")
    assert flags == 0 and all(d["obs_teams"] & hase.HASE_OBS_LOS for d in cc["descs"])
    assert not any(d["obs_teams"] & hase.HASE_OBS_LOS for d in c["descs"])  # the input is untouched
    s = W.single1k()
    _, f_default = bench.apply_mode(s, "default")
    _, f_void = bench.apply_mode(s, "void")
    assert f_default & hase.HASE_EXPORT_UNPACKED  # the workload's unpacked export
    assert not f_void & hase.HASE_EXPORT_UNPACKED  # nothing to unpack without planes
    assert bench.oracle_fog(bench.MODES["fog"][0]) == 1
    assert bench.oracle_fog(bench.MODES["fog-agent"][0]) == 2
    assert bench.oracle_fog(bench.MODES["central"][0]) == 0


def test_single_agent_bytes():
    # one observing seeker (r 3): obs 3 words + unpacked 3 x 49 B + rewards of
    # 2 agents + done = 24 + 147 + 8 + 1
    s = W.single1k()
    cc, flags = bench.apply_mode(s, "default")
    assert bench.algorithmic_bytes_per_env_step(cc["descs"], 1, cc["unpacked"], flags) == 180
