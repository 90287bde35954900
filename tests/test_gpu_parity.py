"""GPU parity: the CUDA engine (through the C ABI) against the oracle, bit
for bit on every output of every step (integer and bit work: exact).

Sizes span several CTA groups, chunk boundaries, ring wrap-around and
episode resets; the full-size runs use the launch configuration of the
benchmark and compare sampled environments one by one (the oracle steps a
single env through its global env id) plus properties that hold at any size.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2604_27162_gb300 import hase
from paper_2604_27162_gb300 import workloads as W
from tests.gpu_helpers import compare_run, engine_outputs

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    hase.load()


# The two forms of the step kernel (identical outputs): the streaming one
# (one-thread families without line of sight, centralized observation or fog
# of war) and the chunked one.
FORMS = {"stream": hase.HASE_STREAM_STEP, "chunked": hase.HASE_CHUNKED_STEP}


@pytest.mark.parametrize("form", sorted(FORMS))
def test_plain16_full_run(form):
    c = W.plain16()
    compare_run(c["n_envs"], c["seed"], c["descs"], c["steps"], flags=hase.HASE_EXPORT_ACTIONS | FORMS[form])


@pytest.mark.parametrize("form", sorted(FORMS))
def test_ten_agents_1024_envs_600_steps(form):
    c = W.ten1k()
    compare_run(1024, c["seed"], c["descs"], 600, flags=hase.HASE_EXPORT_ACTIONS | FORMS[form])


@pytest.mark.parametrize("form", sorted(FORMS))
def test_single_agent_packed_and_unpacked(form):
    c = W.single1k()
    compare_run(1024, c["seed"], c["descs"], 300,
                flags=hase.HASE_EXPORT_ACTIONS | hase.HASE_EXPORT_UNPACKED | FORMS[form])


@pytest.mark.parametrize("form", sorted(FORMS))
def test_unpacked_export_every_radius(form):
    """The unpacked bytes of windows of 1, 9, 25 and 49 bits a plane, the
    envs' runs starting at every offset mod 16."""
    for r, A, S in ((0, 3, 9), (1, 4, 12), (2, 2, 16), (3, 5, 20)):
        descs = [W.env_desc(S, A, (A + 1) // 2, r, r, 40, "0.2", 3)]
        compare_run(37, 50 + r, descs, 90, ring=200, env_id_base=5,
                    flags=hase.HASE_EXPORT_ACTIONS | hase.HASE_EXPORT_UNPACKED | FORMS[form])


@pytest.mark.parametrize("form", sorted(FORMS))
def test_unpacked_export_uneven_and_waves(form):
    """The unpacked export where a group's envs are not consecutive in the
    layout (mixed shapes: written directly, not staged), and with more CTAs
    than SMs (staged groups of one family, CTAs in waves)."""
    fl = hase.HASE_EXPORT_ACTIONS | hase.HASE_EXPORT_UNPACKED | FORMS[form]
    compare_run(60, 8, W.uneven_descs(60, 11), 45, ring=180, flags=fl)
    compare_run(2600, 9, [W.env_desc(8, 2, 1, 2, 2, 20, "0.2", 1)], 25, ring=170, flags=fl, env_id_base=3)


@pytest.mark.parametrize("form", sorted(FORMS))
def test_uneven_batch(form):
    descs = W.uneven_descs(1500, 3)
    compare_run(1500, 3, descs, 300, flags=hase.HASE_EXPORT_ACTIONS | FORMS[form])


@pytest.mark.parametrize("tuning", [
    dict(chunk_steps=1, emit_warps=1),
    dict(chunk_steps=5, emit_warps=2, steps_per_launch=7),
    dict(chunk_steps=32, emit_warps=7, max_group_envs=1),
    dict(chunk_steps=13, emit_warps=12, steps_per_launch=1),
    dict(chunk_steps=4, emit_warps=4, max_group_envs=3),
])
@pytest.mark.parametrize("form", sorted(FORMS))
def test_launch_configurations_agree(tuning, form):
    c = W.ten1k()
    descs = [dict(c["descs"][0], cap=37)]
    fl = hase.HASE_EXPORT_ACTIONS | FORMS[form]
    compare_run(70, c["seed"], descs, 90, ring=200, flags=fl, **tuning)
    compare_run(40, 11, W.uneven_descs(40, 5), 90, ring=170, flags=fl, **tuning)


def test_graph_replays_match_oracle():
    c = W.ten1k()
    descs = [dict(c["descs"][0], cap=45)]
    # one graph replayed four times, mixed with plain launches and a second graph
    compare_run(50, c["seed"], descs, 180, launches=[("graph", 32), ("graph", 32), 5, ("graph", 32),
                                                     ("graph", 32), ("graph", 47)])
    compare_run(40, 11, W.uneven_descs(40, 5), 96, ring=10,
                launches=[("graph", 24)] * 4, steps_per_launch=7)


@pytest.mark.parametrize("cap", [32768, 65536, 98304])
def test_shared_memory_caps_agree(cap):
    compare_run(60, 12, W.uneven_descs(60, 6), 70, smem_cap=cap)


def test_shared_memory_cap_too_small_rejected():
    with pytest.raises(hase.HaseError):
        hase.Engine(2, 1, [W.env_desc(64, 16, 8, 4, 4, 10, "0.2")], 8, smem_cap=16384)


def test_desynchronised_start_matches_oracle():
    c = W.ten1k()
    descs = [dict(c["descs"][0], cap=29)]
    flags = hase.HASE_EXPORT_ACTIONS | hase.HASE_DESYNC_START
    compare_run(40, c["seed"], descs, 75, flags=flags)
    compare_run(30, 4, W.uneven_descs(30, 8), 60, flags=flags, launches=[7, 53])
    # a reset restores the same drawn offsets
    eng = hase.Engine(25, 9, descs, 64, flags)
    eng.step(40)
    eng.reset()
    eng.step(40)
    got = engine_outputs(eng)
    w = oracle.World(25, 9, descs, desync=True)
    for t in range(40):
        o = w.step()
        assert (got["done"][t] == o["done"]).all() and (got["obs"][t] == o["obs"]).all(), t
    eng.close()


@pytest.mark.parametrize("form", sorted(FORMS))
def test_desynchronised_start_moves_match_oracle(form):
    """The moves taken before the first observation (Sec. 3.3, last
    paragraph): the step -1 cells and clocks, then every step, with an
    env-id offset, in both step forms (the streaming form serves up to 16
    agents; 20 and 32 run chunked)."""
    flags = hase.HASE_EXPORT_STATE | hase.HASE_EXPORT_ACTIONS | hase.HASE_DESYNC_START | FORMS[form]
    for A, S, cap in ((2, 16, 40), (10, 32, 60), (20, 16, 50), (32, 24, 90)):
        descs = [W.env_desc(S, A, max(1, A // 2), 3, 2, cap, "0.2")]
        compare_run(24, 31, descs, 70, ring=200, flags=flags, env_id_base=1000, launches=[33, 37])


@pytest.mark.parametrize("desc", [
    W.env_desc(32, 10, 5, 3, 2, 40, "0.2", 3 | 4),     # one-thread emission, radius 3 / 2
    W.env_desc(24, 7, 4, 4, 4, 40, "0.25", 3 | 4),     # one-thread emission, radius 4 (two words)
    W.env_desc(16, 6, 2, 3, 1, 30, "0.3", 3 | 4),      # lane-per-agent emission
    W.env_desc(12, 5, 3, 2, 2, 30, "0.2", 2 | 4),      # hiders only emit
    W.env_desc(10, 3, 2, 2, 3, 30, "0.2", 1 | 4),      # one-thread emission, 1-4 agents
    W.env_desc(20, 16, 8, 3, 1, 30, "0.25", 3 | 4),    # one-thread emission, 13-16 agents
    W.env_desc(12, 3, 2, 4, 4, 30, "0.2", 1 | 4),      # two-word windows, 1-4 agents
    W.env_desc(20, 16, 8, 4, 2, 30, "0.25", 3 | 4),    # two-word windows, 13-16 agents
])
def test_line_of_sight_matches_oracle(desc):
    compare_run(36, 17, [desc], 70, flags=hase.HASE_EXPORT_ACTIONS | hase.HASE_EXPORT_UNPACKED)
    compare_run(20, 18, [desc], 40, smem_cap=32768)  # windows computed without tables


@pytest.mark.parametrize("desc", [
    W.env_desc(32, 10, 5, 3, 2, 40, "0.2"),            # both teams observe
    W.env_desc(64, 6, 3, 4, 1, 40, "0.2"),             # 64 columns: full-word rows
    W.env_desc(9, 4, 2, 2, 3, 20, "0.3", 1),           # seekers only
    W.env_desc(16, 8, 4, 3, 3, 25, "0.25", 3 | 4),     # line of sight
    W.env_desc(12, 5, 2, 0, 1, 30, "0.2", 2),          # hiders only, radius 0
])
def test_centralized_observation_matches_oracle(desc):
    compare_run(24, 23, [desc], 50, flags=hase.HASE_EXPORT_CENTRAL | hase.HASE_EXPORT_ACTIONS)


def test_centralized_observation_uneven():
    compare_run(30, 24, W.uneven_descs(30, 12), 45, flags=hase.HASE_EXPORT_CENTRAL, launches=[20, 25])


def test_line_of_sight_shared_table():
    """Seven 32x32 envs per CTA: the per-team window tables (radius 3 and 2,
    with visibility) do not fit, one radius-3 table serves both teams."""
    desc = W.env_desc(32, 10, 5, 3, 2, 40, "0.2", 3 | 4)
    compare_run(21, 23, [desc], 75, flags=hase.HASE_EXPORT_ACTIONS | hase.HASE_EXPORT_UNPACKED,
                max_group_envs=7, launches=[40, 35])
    compare_run(21, 24, [W.env_desc(32, 7, 4, 1, 3, 30, "0.3", 3 | 4)], 50, max_group_envs=7)


def test_line_of_sight_uneven():
    descs = [dict(d, obs_teams=3 | 4) for d in W.uneven_descs(40, 11)]
    compare_run(40, 19, descs, 60)


# Observability modes of Section 3.3 (mode 1 is the default everywhere else).
MODES = {
    2: hase.HASE_EXPORT_STATE,
    3: hase.HASE_SKIP_OBS | hase.HASE_EXPORT_CENTRAL,
    4: hase.HASE_SKIP_OBS | hase.HASE_EXPORT_CENTRAL | hase.HASE_EXPORT_STATE,
    5: hase.HASE_SKIP_OBS | hase.HASE_EXPORT_STATE,
    6: hase.HASE_SKIP_OBS,
}


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("desc", [
    W.env_desc(32, 10, 5, 3, 2, 40, "0.2"),            # one-thread emission, one word a plane
    W.env_desc(24, 7, 4, 4, 4, 40, "0.25"),            # one-thread emission, radius 4 (two words)
    W.env_desc(16, 6, 2, 3, 1, 30, "0.3"),             # lane-per-agent emission
    W.env_desc(16, 8, 4, 3, 3, 25, "0.25", 3 | 4),     # line of sight
], ids=["fast", "fast-r4", "lane", "los"])
def test_observability_modes_match_oracle(mode, desc):
    compare_run(24, 31, [desc], 70, flags=MODES[mode] | hase.HASE_EXPORT_ACTIONS, launches=[30, 40])


def test_true_state_uneven_desynchronised_and_reset():
    flags = hase.HASE_EXPORT_STATE | hase.HASE_DESYNC_START | hase.HASE_EXPORT_CENTRAL
    descs = W.uneven_descs(36, 13)
    compare_run(36, 6, descs, 90, flags=flags, launches=[11, ("graph", 40), 39])
    compare_run(36, 6, descs, 90, flags=flags | hase.HASE_SKIP_OBS, ring=17, launches=[50, 40])
    # hase_reset writes the true state of the reset (step -1) again
    eng = hase.Engine(36, 6, descs, 64, flags)
    eng.step(70)
    eng.reset()
    got = engine_outputs(eng)
    cells, ep_t = oracle.World(36, 6, descs, desync=True).true_state()
    assert (got["cells"][63] == cells).all() and (got["ep_t"][63] == ep_t).all()
    eng.close()


@pytest.mark.parametrize("per_agent", [False, True], ids=["global", "per-agent"])
@pytest.mark.parametrize("desc", [
    W.env_desc(32, 10, 5, 3, 2, 40, "0.2"),            # one-thread emission family
    W.env_desc(24, 7, 4, 4, 4, 31, "0.25"),            # radius 4
    W.env_desc(16, 6, 2, 3, 1, 30, "0.3", 2),          # lane-per-agent, hiders observe
    W.env_desc(16, 8, 4, 3, 3, 25, "0.25", 3 | 4),     # line of sight
    W.env_desc(64, 5, 3, 2, 4, 20, "0.15"),            # 64 columns
    W.env_desc(9, 4, 2, 2, 2, 33, "0.2", 0),           # nobody observes
], ids=["fast", "r4", "lane-hiders", "los", "side64", "none"])
def test_fog_of_war_matches_oracle(desc, per_agent):
    flags = hase.HASE_EXPORT_FOG | (hase.HASE_FOG_PER_AGENT if per_agent else 0)
    compare_run(20, 41, [desc], 80, flags=flags, launches=[13, 64, 3], chunk_steps=16)


def test_fog_of_war_uneven_graph_desync_and_reset():
    descs = W.uneven_descs(40, 14)
    flags = hase.HASE_EXPORT_FOG | hase.HASE_DESYNC_START | hase.HASE_EXPORT_CENTRAL
    compare_run(40, 9, descs, 70, flags=flags, launches=[("graph", 30), 40])
    compare_run(40, 9, descs, 70, flags=flags | hase.HASE_FOG_PER_AGENT | hase.HASE_SKIP_OBS, ring=23,
                launches=[35, ("graph", 35)])
    eng = hase.Engine(40, 9, descs, 64, flags | hase.HASE_FOG_PER_AGENT)
    eng.step(50)
    eng.reset()
    fog = engine_outputs(eng)["fog"]
    assert (fog[63] == oracle.World(40, 9, descs, desync=True, fog=2).fog()).all()
    eng.close()


def test_fog_of_war_checkpoint_resume():
    descs = [W.env_desc(16, 6, 3, 3, 2, 45, "0.2")]
    flags = hase.HASE_EXPORT_FOG
    a = hase.Engine(12, 3, descs, 100, flags)
    a.step(30)
    blob = hase.hase_get_state(a.h)
    a.step(30)
    want = engine_outputs(a)["fog"][30:60]
    b = hase.Engine(12, 3, descs, 100, flags)
    b.step(7)  # another history, then the checkpoint
    hase.hase_set_state(b.h, blob)
    b.step(30)
    got = engine_outputs(b)["fog"][30:60]
    assert (got == want).all()
    a.close()
    b.close()


@pytest.mark.parametrize("desc,flags", [
    (W.env_desc(6, 3, 2, 1, 2, 1, "0.2"), hase.HASE_EXPORT_FOG | hase.HASE_EXPORT_CENTRAL | hase.HASE_EXPORT_STATE),
    (W.env_desc(2, 3, 1, 2, 1, 5, "0.5"), hase.HASE_EXPORT_FOG | hase.HASE_FOG_PER_AGENT | hase.HASE_EXPORT_CENTRAL),
    (W.env_desc(12, 6, 3, 0, 0, 9, "0.2", 3 | 4), hase.HASE_EXPORT_FOG | hase.HASE_EXPORT_CENTRAL),
    (W.env_desc(64, 16, 8, 4, 4, 17, "0.3", 3 | 4), hase.HASE_EXPORT_FOG | hase.HASE_FOG_PER_AGENT | hase.HASE_SKIP_OBS),
    (W.env_desc(10, 4, 2, 2, 2, 30, 2**32 - 1, 1), hase.HASE_EXPORT_FOG | hase.HASE_EXPORT_STATE | hase.HASE_SKIP_OBS),
    (W.env_desc(16, 6, 3, 3, 2, 30, "0.2"), hase.HASE_EXPORT_STATE | hase.HASE_EXPORT_UNPACKED | hase.HASE_DESYNC_START),
], ids=["cap1-all-exports", "smallest-grid", "radius0-los", "largest-los-per-agent", "all-blocked", "state-unpacked"])
def test_optional_exports_edge_cases(desc, flags):
    compare_run(9, 77, [desc], 40, flags=flags | hase.HASE_EXPORT_ACTIONS, launches=[1, 17, 22], chunk_steps=8)


@pytest.mark.parametrize("teams", [3, 3 | 4], ids=["plain", "los"])
def test_mixed_sides_in_one_cta(teams):
    """Envs of one kernel shape but different sides share a CTA (the shape key
    holds the cell packing, not the side): every export must size its
    per-CTA buffers for the largest side."""
    descs = [W.env_desc(side, 6, 3, 2, 2, 30, "0.2", teams) for side in (8, 16, 24, 32, 12, 20)] * 4
    flags = (hase.HASE_EXPORT_CENTRAL | hase.HASE_EXPORT_FOG | hase.HASE_EXPORT_STATE
             | hase.HASE_EXPORT_ACTIONS)
    compare_run(24, 52, descs, 70, flags=flags, max_group_envs=6, launches=[33, 37])
    compare_run(24, 53, descs, 40, flags=flags | hase.HASE_FOG_PER_AGENT | hase.HASE_SKIP_OBS,
                max_group_envs=6)


def test_ring_wraparound_and_split_launches():
    c = W.ten1k()
    compare_run(64, c["seed"], c["descs"], 300, ring=7, launches=[1, 2, 97, 200])
    compare_run(64, c["seed"], c["descs"], 50, ring=1, launches=[3, 47])


@pytest.mark.parametrize("desc", [
    W.env_desc(8, 1, 1, 3, 3, 20, "0.15"),            # lone seeker
    W.env_desc(8, 5, 0, 2, 2, 20, "0.15"),            # hiders only
    W.env_desc(8, 5, 5, 2, 2, 20, "0.15"),            # seekers only
    W.env_desc(12, 6, 3, 0, 0, 9, "0.2"),             # radius 0
    W.env_desc(12, 9, 4, 4, 1, 17, "0.25"),           # radius 4: two words per plane
    W.env_desc(2, 3, 1, 2, 1, 5, "0.5"),              # smallest grid
    W.env_desc(64, 16, 8, 4, 4, 33, "0.3"),           # largest grid: two-word rows
    W.env_desc(57, 7, 3, 3, 2, 40, "0.1"),            # first side with two-word rows
    W.env_desc(56, 7, 3, 3, 2, 40, "0.1"),            # last side with one-word rows
    W.env_desc(16, 8, 4, 2, 3, 1, "0.15"),            # cap 1: reset every step
    W.env_desc(10, 4, 2, 2, 2, 30, 0),                # no obstacles
    W.env_desc(10, 4, 2, 2, 2, 30, 2**32 - 1),        # all blocked but start cells
    W.env_desc(4, 16, 8, 1, 2, 30, "0.2"),            # full grid: nobody can move
    W.env_desc(16, 6, 3, 3, 2, 30, "0.2", 0),         # void observations
    W.env_desc(16, 6, 3, 3, 2, 30, "0.2", 2),         # hiders only emit
])
def test_edge_cases(desc):
    compare_run(37, 5, [desc], 80, flags=hase.HASE_EXPORT_ACTIONS | hase.HASE_EXPORT_UNPACKED)


def test_checkpoint_resume_and_reset_replay():
    import torch

    c = W.ten1k()
    eng = hase.Engine(96, c["seed"], c["descs"], 400, hase.HASE_EXPORT_ACTIONS)
    eng.step(150)
    blob = eng.get_state()
    eng.step(150)
    first = engine_outputs(eng)
    eng.set_state(blob)
    assert eng.t == 150
    eng.step(150)
    second = engine_outputs(eng)
    for k in first:
        assert (first[k][150:300] == second[k][150:300]).all(), k
    eng.reset()
    assert eng.t == 0
    eng.step(300)
    third = engine_outputs(eng)
    for k in first:
        assert (first[k][:300] == third[k][:300]).all(), k
    torch.cuda.synchronize()
    eng.close()


def test_world_readback_matches_oracle():
    descs = W.uneven_descs(30, 9)
    eng = hase.Engine(30, 77, descs, 2)
    w = oracle.World(30, 77, descs)
    st = w.state()
    off = w.agent_off.astype(int)
    for e in range(30):
        d = descs[e]
        grid, start = hase.hase_get_world(eng.h, e, d["side"], d["n_agents"])
        assert (grid == w.grid(e)).all()
        assert (start[:, 0] == st["sx"][off[e]:off[e + 1]]).all()
        assert (start[:, 1] == st["sy"][off[e]:off[e + 1]]).all()
    eng.close()


def test_invalid_configs_rejected():
    good = W.ten1k()["descs"][0]
    for bad in (dict(good, side=65), dict(good, side=1), dict(good, n_agents=33),
                dict(good, n_agents=0), dict(good, n_seekers=11), dict(good, r_seek=5),
                dict(good, cap=0), dict(good, obs_teams=8)):
        with pytest.raises(hase.HaseError) as ei:
            hase.Engine(4, 0, [bad], 2)
        assert ei.value.status == hase.HASE_EINVAL
    with pytest.raises(hase.HaseError):
        hase.Engine(4, 0, [good], 0)
    with pytest.raises(hase.HaseError):
        hase.Engine(0, 0, [good], 2)
    with pytest.raises(hase.HaseError) as ei:  # no decentralized planes to unpack
        hase.Engine(4, 0, [good], 2, hase.HASE_SKIP_OBS | hase.HASE_EXPORT_UNPACKED)
    assert ei.value.status == hase.HASE_EINVAL
    with pytest.raises(hase.HaseError):
        hase.Engine(4, 0, [good], 2, 1 << 12)  # unknown flag
    with pytest.raises(hase.HaseError):  # two step forms at once
        hase.Engine(4, 0, [good], 2, hase.HASE_CHUNKED_STEP | hase.HASE_STREAM_STEP)
    with pytest.raises(hase.HaseError):  # per-agent maps without the fog export
        hase.Engine(4, 0, [good], 2, hase.HASE_FOG_PER_AGENT)


# ---------------------------------------------------------------------------
# Full-size runs in the benchmark's launch configuration.
# ---------------------------------------------------------------------------
def _full_size_check(cfg, n_steps, sample_envs, flags=0, setting=None, graph=False):
    """The workload at full size in the benchmark's launch configuration
    (setting: an autotuned launch setting; graph: the steps replayed as one
    CUDA graph), then: the done property over every env and step on the GPU,
    and every output of every step of the sampled envs against a one-env
    oracle (the unpacked export too when the flags ask for it)."""
    import torch

    n = cfg["n_envs"]
    descs = cfg["descs"]
    eng = hase.Engine(n, cfg["seed"], descs, n_steps, flags, **(setting or {}))
    if graph:
        eng.step_graph(n_steps)
    else:
        eng.step(n_steps)
    torch.cuda.synchronize()
    L = eng.layout
    aoff = L["agent_off"].astype(np.int64)
    ooff = L["obs_off"].astype(np.int64)
    uoff = L["unp_off"].astype(np.int64)
    unpacked = bool(flags & hase.HASE_EXPORT_UNPACKED)
    # properties over every env and step (on the GPU)
    done = eng.done
    caps = torch.tensor([descs[0 if len(descs) == 1 else e]["cap"] for e in range(n)],
                        device="cuda", dtype=torch.int64)
    steps = torch.arange(n_steps, device="cuda", dtype=torch.int64)[:, None]
    want_done = torch.where((steps + 1) % caps[None, :] == 0, 3, 0).to(torch.uint8)
    assert torch.equal(done, want_done)
    # sampled envs: every output of every step against a one-env oracle
    for e in sample_envs:
        d = descs[0 if len(descs) == 1 else e]
        rew = eng.reward[:, aoff[e]:aoff[e + 1]].cpu().numpy()
        obs = eng.obs[:, ooff[e]:ooff[e + 1]].cpu().numpy().view(np.uint64)
        unp = eng.unpacked[:, uoff[e]:uoff[e + 1]].cpu().numpy() if unpacked else None
        dn = eng.done[:, e].cpu().numpy()
        w = oracle.World(1, cfg["seed"], [d], env_id_base=e)
        for t in range(n_steps):
            o = w.step(unpacked=unpacked)
            assert (rew[t] == o["reward"]).all(), (e, t)
            assert (obs[t] == o["obs"]).all(), (e, t)
            assert dn[t] == o["done"][0], (e, t)
            if unpacked:
                assert (unp[t] == o["unpacked"]).all(), (e, t)
    eng.close()


def _full_size_exports_check(cfg, n_steps, sample_envs, flags):
    """The optional exports at full size, sampled: every step of the sampled
    envs' centralized observation, true state and fog of war against a
    one-env oracle (with the desynchronised start when asked: its offsets
    and pre-steps depend on the env id only)."""
    import torch

    n = cfg["n_envs"]
    descs = cfg["descs"]
    eng = hase.Engine(n, cfg["seed"], descs, n_steps, flags)
    eng.step(n_steps)
    torch.cuda.synchronize()
    L = eng.layout
    nxt = lambda off, total, e: int(off[e + 1]) if e + 1 < n else total
    fog = 0 if not flags & hase.HASE_EXPORT_FOG else (2 if flags & hase.HASE_FOG_PER_AGENT else 1)
    aoff = L["agent_off"].astype(np.int64)
    for e in sample_envs:
        d = descs[0 if len(descs) == 1 else e]
        w = oracle.World(1, cfg["seed"], [d], env_id_base=e, desync=bool(flags & hase.HASE_DESYNC_START), fog=fog)
        obs = eng.obs[:, int(L["obs_off"][e]):nxt(L["obs_off"], eng.obs.shape[1], e)].cpu().numpy().view(np.uint64)
        cen = fo = cells = ept = None
        if eng.central is not None:
            c0 = int(L["central_off"][e])
            cen = eng.central[:, c0:nxt(L["central_off"], eng.central.shape[1], e)].cpu().numpy().view(np.uint64)
        if eng.fog is not None:
            f0 = int(L["fog_off"][e])
            fo = eng.fog[:, f0:nxt(L["fog_off"], eng.fog.shape[1], e)].cpu().numpy().view(np.uint64)
        if eng.cells is not None:
            cells = eng.cells[:, aoff[e]:aoff[e + 1]].cpu().numpy().view(np.uint16)
            ept = eng.ep_t[:, e].cpu().numpy().view(np.uint32)
        for t in range(n_steps):
            o = w.step()
            assert (obs[t] == o["obs"]).all(), (e, t)
            if cen is not None:
                assert (cen[t] == w.central()).all(), (e, t)
            if fo is not None:
                assert (fo[t] == w.fog()).all(), (e, t)
            if cells is not None:
                c, ep = w.true_state()
                assert (cells[t] == c).all() and ept[t] == ep[0], (e, t)
    eng.close()


def test_full_size_optional_exports_sampled():
    """ten1k at the benchmark's size with the centralized observation, the
    true state and the desynchronised start, then with the per-agent fog of
    war, each sampled on four envs over 1,500 steps."""
    cfg = W.ten1k()
    _full_size_exports_check(cfg, 1500, [0, 5, 512, 1023],
                             hase.HASE_EXPORT_CENTRAL | hase.HASE_EXPORT_STATE | hase.HASE_DESYNC_START)
    _full_size_exports_check(cfg, 1500, [1, 700, 1022], hase.HASE_EXPORT_FOG | hase.HASE_FOG_PER_AGENT)


def test_full_size_ten_agents_sampled():
    cfg = W.ten1k()
    _full_size_check(cfg, cfg["steps"], [0, 1, 337, 511, 512, 1023])


def test_full_size_single_agent_sampled():
    """The whole 10,000-step run of the benchmark, packed and unpacked."""
    cfg = W.single1k()
    _full_size_check(cfg, cfg["steps"], [0, 5, 700, 1023], flags=hase.HASE_EXPORT_UNPACKED)


def test_full_size_line_of_sight_sampled():
    cfg = W.ten1k()
    cfg = dict(cfg, descs=[dict(cfg["descs"][0], obs_teams=3 | 4)])
    _full_size_check(cfg, 1500, [0, 338, 1023])


def test_full_size_uneven_sampled():
    cfg = W.uneven64k()
    _full_size_check(cfg, 200, [0, 1, 4097, 33333, 65535])


def _uneven_samples(descs, per_key=1):
    """Envs of the uneven table spread over sides, agent counts and radii."""
    picks, seen = [], set()
    for e, d in enumerate(descs):
        for key in (("side", d["side"]), ("agents", d["n_agents"]), ("radius", d["r_seek"])):
            if key not in seen:
                seen.add(key)
                picks.append(e)
    return sorted(set(picks))


def test_full_size_uneven_autotuned_graph():
    """The benchmark's batched form of the uneven workload: the autotuned
    setting, the 1,000-step rollout replayed as one CUDA graph."""
    from paper_2604_27162_gb300 import autotune

    cfg = W.uneven64k()
    setting, _ = autotune.tune(cfg["n_envs"], cfg["seed"], cfg["descs"])
    sample = _uneven_samples(cfg["descs"])
    assert len(sample) >= 8
    _full_size_check(cfg, cfg["steps"], sample, setting=setting, graph=True)


@pytest.mark.parametrize("form", sorted(FORMS))
@pytest.mark.parametrize("rank", [1, 3])
def test_rank_shards_match_oracle(rank, form):
    """The env range of rank 1 or 3 of a multi-GPU run (env ids from
    rank * 1024): its draws are keyed by the global env ids."""
    c = W.ten1k()
    compare_run(1024, c["seed"], c["descs"], 200, flags=hase.HASE_EXPORT_ACTIONS | FORMS[form],
                env_id_base=rank * 1024)


TWENTY_PLUS = [
    W.env_desc(32, 20, 10, 3, 2, 37, "0.2"),    # the paper's 20 searchers (seekers = ceil(A / 2))
    W.env_desc(24, 20, 12, 2, 3, 29, "0.15"),   # seekers != ceil(A / 2)
    W.env_desc(16, 32, 5, 1, 2, 23, "0.1"),     # 32 agents, few seekers
    W.env_desc(64, 32, 16, 4, 4, 41, "0.25"),   # 32 agents on the largest grid, radius 4
]


def test_twenty_and_thirty_two_agents():
    """Up to 32 agents an env (one dynamics lane each): the lane-per-agent
    emission, alone and mixed in one batch."""
    for d in TWENTY_PLUS:
        compare_run(12, 31, [d], 120)
    descs = [TWENTY_PLUS[e % 4] for e in range(40)]
    compare_run(40, 32, descs, 100, launches=[37, 63])


def test_thirty_two_agents_optional_exports():
    descs = [dict(TWENTY_PLUS[e % 4], obs_teams=3 | (4 if e % 2 else 0)) for e in range(16)]
    flags = (hase.HASE_EXPORT_ACTIONS | hase.HASE_EXPORT_CENTRAL | hase.HASE_EXPORT_STATE
             | hase.HASE_EXPORT_FOG | hase.HASE_EXPORT_UNPACKED)
    compare_run(16, 33, descs, 90, flags=flags)
    compare_run(16, 34, descs, 60, flags=flags | hase.HASE_FOG_PER_AGENT | hase.HASE_DESYNC_START)
