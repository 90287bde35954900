"""Launch-configuration autotuner of the batched step.

The knobs are the ones `hase_create` takes: the form of the step kernel
(chunked or streaming), the shared-memory cap of a CTA (which decides how
many envs share a CTA and whether the per-cell window tables fit, hence how
many CTAs an SM holds), the emission warps per CTA, the envs packed per CTA,
the steps per on-chip chunk and the steps fused per launch.  Each candidate
is measured on a rollout of the actual batch (by default 128 steps; give the
timed run's own length where the per-launch prologue matters, e.g. CTAs that
run in waves), replayed as a CUDA graph exactly as the timed run will be, and
the fastest is kept.  The search is coordinate descent from the engine's own defaults:
one knob at a time, keeping the best value before moving to the next.
"""
from __future__ import annotations

import time

from . import hase

KNOBS = [
    ("step_form", ["auto", "chunked", "stream"]),
    ("smem_cap", [0, 49152, 65536, 98304, 131072, 163840]),
    ("emit_warps", [0, 3, 4, 6, 8]),
    ("max_group_envs", [0, 1, 2, 4]),
    ("chunk_steps", [0, 16, 24]),
    ("steps_per_launch", [0, 64]),
]


def measure(n_envs, seed, descs, flags, setting, probe_steps, repeats=3, stream=None):
    """Seconds per probe rollout of one setting (None when it cannot be built)."""
    import torch

    try:
        eng = hase.Engine(n_envs, seed, descs, ring_steps=max(probe_steps, 160), flags=flags, stream=stream,
                          **{k: v for k, v in setting.items() if v})
    except hase.HaseError:
        return None
    try:
        eng.step_graph(probe_steps)  # capture + warm-up
        torch.cuda.synchronize()
        s = stream or torch.cuda.current_stream()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(s)
        for _ in range(repeats):
            eng.step_graph(probe_steps)
        t1.record(s)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / 1e3 / repeats
    finally:
        eng.close()


def tune(n_envs, seed, descs, flags=0, probe_steps=128, knobs=None, stream=None, log=None):
    """Returns (best setting, list of (setting, seconds)) for the batch."""
    knobs = knobs or KNOBS
    best = {k: vals[0] for k, vals in knobs}
    best_s = measure(n_envs, seed, descs, flags, best, probe_steps, stream=stream)
    if best_s is None:
        raise RuntimeError("the default launch configuration cannot be built")
    trials = [(dict(best), best_s)]
    t_start = time.perf_counter()
    for name, values in knobs:
        for v in values:
            if v == best[name]:
                continue
            cand = dict(best, **{name: v})
            s = measure(n_envs, seed, descs, flags, cand, probe_steps, stream=stream)
            if s is None:
                continue
            trials.append((cand, s))
            if log:
                log("autotune %s -> %.3f ms" % (cand, s * 1e3))
            if s < best_s:
                best, best_s = cand, s
    if log:
        log("autotune: best %s (%.3f ms per %d steps) after %d trials, %.1f s"
            % (best, best_s * 1e3, probe_steps, len(trials), time.perf_counter() - t_start))
    return {k: v for k, v in best.items() if v and v != "auto"}, trials
