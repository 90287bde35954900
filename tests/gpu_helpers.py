"""Helpers of the GPU parity tests: run the CUDA engine through the C ABI and
the oracle on the same seeded inputs and compare every output bit for bit."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2604_27162_gb300 import hase


def engine_outputs(eng):
    import torch

    torch.cuda.synchronize()
    out = {
        "obs": eng.obs.cpu().numpy().view(np.uint64),
        "reward": eng.reward.cpu().numpy(),
        "done": eng.done.cpu().numpy(),
    }
    if eng.actions is not None:
        out["action"] = eng.actions.cpu().numpy()
    if eng.unpacked is not None:
        out["unpacked"] = eng.unpacked.cpu().numpy()
    if eng.central is not None:
        out["central"] = eng.central.cpu().numpy().view(np.uint64)
    if eng.fog is not None:
        out["fog"] = eng.fog.cpu().numpy().view(np.uint64)
    if eng.cells is not None:
        out["cells"] = eng.cells.cpu().numpy().view(np.uint16)
        out["ep_t"] = eng.ep_t.cpu().numpy().view(np.uint32)
    return out


def compare_run(n_envs, seed, descs, n_steps, ring=None, flags=hase.HASE_EXPORT_ACTIONS,
                env_id_base=0, launches=None, **tuning):
    """Step the engine n_steps (in the given launch sizes) and the oracle in
    lockstep; every slot still in the ring must match exactly."""
    ring = ring or n_steps + 1
    eng = hase.Engine(n_envs, seed, descs, ring, flags, env_id_base, **tuning)
    total = 0
    for item in (launches or [n_steps]):
        # an int: hase_step; ("graph", n): the same steps as a replayed CUDA graph
        if isinstance(item, tuple):
            eng.step_graph(item[1])
            total += item[1]
        else:
            eng.step(item)
            total += item
    assert total == n_steps
    got = engine_outputs(eng)
    if flags & hase.HASE_SKIP_OBS:  # no decentralized observation at all
        assert got["obs"].shape == (ring, 0), got["obs"].shape
        del got["obs"]
    unpacked = bool(flags & hase.HASE_EXPORT_UNPACKED)
    fog = 0 if not flags & hase.HASE_EXPORT_FOG else (2 if flags & hase.HASE_FOG_PER_AGENT else 1)
    w = oracle.World(n_envs, seed, descs, env_id_base=env_id_base,
                     desync=bool(flags & hase.HASE_DESYNC_START), fog=fog)
    if ring > n_steps:
        init = w.observe(unpacked=unpacked)
        o0 = init[0] if unpacked else init
        assert "obs" not in got or (got["obs"][ring - 1] == o0).all(), "initial observation"
        if unpacked:
            assert (got["unpacked"][ring - 1] == init[1]).all(), "initial unpacked"
        assert (got["reward"][ring - 1] == 0).all() and (got["done"][ring - 1] == 0).all()
        if "central" in got:
            assert (got["central"][ring - 1] == w.central()).all(), "initial centralized observation"
        if "fog" in got:
            assert (got["fog"][ring - 1] == w.fog()).all(), "initial fog of war"
        if "cells" in got:
            cells, ep_t = w.true_state()
            assert (got["cells"][ring - 1] == cells).all(), "initial true state (cells)"
            assert (got["ep_t"][ring - 1] == ep_t).all(), "initial true state (episode clocks)"
    for t in range(n_steps):
        o = w.step(unpacked=unpacked)
        if "central" in got:
            o["central"] = w.central()
        if "cells" in got:
            o["cells"], o["ep_t"] = w.true_state()
        if "fog" in got:
            o["fog"] = w.fog()
        if t < n_steps - ring:
            continue
        s = t % ring
        for k in ("obs", "reward", "done", "action", "unpacked", "central", "cells", "ep_t", "fog"):
            if k in got and k in o:
                if not (got[k][s] == o[k]).all():
                    bad = np.flatnonzero(got[k][s] != o[k])[:8]
                    raise AssertionError("%s differs at step %d, entries %s: gpu %s oracle %s" % (
                        k, t, bad.tolist(), got[k][s][bad].tolist(), o[k][bad].tolist()))
    st = w.state()
    eng_t = eng.t
    eng.close()
    assert eng_t == n_steps
    return st
