"""Benchmark of the batched hide-and-seek environment step on GB300.

One benchmark step is one rollout of the workload's run length through the
whole hot path (actions, moves, collisions, observations, rewards, done,
auto-reset): for the default workload (1024 envs, 32x32, 5 seekers + 5
hiders) that is 10,000 env-steps of all 1024 envs.  Every env-step writes its
outputs into a 10,000-slot ring (2.9 GB, far above the 129 MB L2), so the
written bytes stream to HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   (the oracle on the host cores)

Prints one JSON line.  Multi-GPU (torchrun, one rank per GPU): every rank
steps its own independent env range (weak scaling, no collective on the
data path); rank 0 reports the max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2604_27162_gb300 import hase as H  # noqa: E402  (constants only; the library loads later)
from paper_2604_27162_gb300 import workloads as W  # noqa: E402

# Rollout length of one benchmark step per workload (the workload's run).
RUN_STEPS = {"plain16": 1000, "single1k": 10000, "ten1k": 10000, "uneven64k": 1000, "served": 0}

# Optional parts of the step, measured one at a time on a workload:
# name -> (engine flags, obs_teams bits added to every env).  "default" is
# observability mode 1 of Section 3.3; state / central / central-state /
# state-only / void are its modes 2-6; los, desync and fog the other
# optional layers.
MODES = {
    "default": (0, 0),
    "los": (0, H.HASE_OBS_LOS),
    "desync": (H.HASE_DESYNC_START, 0),
    "state": (H.HASE_EXPORT_STATE, 0),
    "central": (H.HASE_SKIP_OBS | H.HASE_EXPORT_CENTRAL, 0),
    "central-state": (H.HASE_SKIP_OBS | H.HASE_EXPORT_CENTRAL | H.HASE_EXPORT_STATE, 0),
    "state-only": (H.HASE_SKIP_OBS | H.HASE_EXPORT_STATE, 0),
    "void": (H.HASE_SKIP_OBS, 0),
    "fog": (H.HASE_EXPORT_FOG, 0),
    "fog-agent": (H.HASE_EXPORT_FOG | H.HASE_FOG_PER_AGENT, 0),
}


def apply_mode(c, mode):
    """The workload with the mode's obs_teams bits, and the mode's flags."""
    flags, teams = MODES[mode]
    if teams:
        c = dict(c, descs=[dict(d, obs_teams=d["obs_teams"] | teams) for d in c["descs"]])
    if c["unpacked"] and not flags & H.HASE_SKIP_OBS:
        flags |= H.HASE_EXPORT_UNPACKED
    return c, flags


def oracle_fog(flags):
    return 0 if not flags & H.HASE_EXPORT_FOG else (2 if flags & H.HASE_FOG_PER_AGENT else 1)


def algorithmic_bytes_per_env_step(descs, n_envs, unpacked, flags=0):
    """Bytes the method must deliver per env-step (obs + reward + done, and
    the exports the flags ask for: unpacked obs, centralized observation,
    true state, fog of war); padding bits are counted inside the obs words,
    the CTA-resident state is not (it is read once per launch)."""
    skip = bool(flags & H.HASE_SKIP_OBS)
    total = 0
    for e in range(n_envs):
        d = descs[0 if len(descs) == 1 else e]
        wmax = 0
        n_obs = 0
        unp = 0
        for a in range(d["n_agents"]):
            team = 0 if a < d["n_seekers"] else 1
            if not (d["obs_teams"] >> team) & 1:
                continue
            r = d["r_seek"] if team == 0 else d["r_hide"]
            D = 2 * r + 1
            wmax = max(wmax, (D * D + 63) // 64)
            n_obs += 1
            unp += 3 * D * D
        S, A = d["side"], d["n_agents"]
        total += 0 if skip else n_obs * 3 * wmax * 8
        total += A * 4 + 1 + (unp if unpacked and not skip else 0)
        if flags & H.HASE_EXPORT_CENTRAL:
            total += 4 * S * 8
        if flags & H.HASE_EXPORT_STATE:
            total += 2 * A + 4
        if flags & H.HASE_EXPORT_FOG:
            units = n_obs if flags & H.HASE_FOG_PER_AGENT else 1
            total += units * 2 * S * 8
    return total / n_envs


def oracle_step(w, flags, unpacked):
    """One oracle step with the mode's outputs (the fog maps are updated by
    the step itself; ho_fog packs them)."""
    w.step(unpacked=unpacked and not flags & H.HASE_SKIP_OBS, observe=not flags & H.HASE_SKIP_OBS)
    if flags & H.HASE_EXPORT_CENTRAL:
        w.central()
    if flags & H.HASE_EXPORT_STATE:
        w.true_state()
    if flags & H.HASE_EXPORT_FOG:
        w.fog()


def measured_traffic(workload_name, key="traffic_bytes_per_env_step"):
    """A per-env-step figure of step_kernel from the committed ncu summary of
    this workload (DRAM bytes, or with key="warp_inst_per_env_step" issued
    warp instructions), or None when the summary is missing or was taken on
    other kernel sources (the summary records their digest)."""
    from paper_2604_27162_gb300 import build as B

    path = os.path.join(ROOT, "profiles", "step_kernel_%s.md" % workload_name)
    try:
        with open(path) as f:
            text = f.read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        line = line.strip().strip("`")
        if "=" in line and line.split("=", 1)[0] in (key, "source_digest"):
            name, val = line.split("=", 1)
            vals[name] = val.strip()
    if vals.get("source_digest") != B.source_digest() or key not in vals:
        return None
    return float(vals[key])


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class NvmlSampler:
    """SM clock, power and clock-event reasons read through NVML (ctypes,
    read-only queries) every `period` seconds in a background thread."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, gpu_index, period=0.002):
        import ctypes

        self.gpu, self.period = gpu_index, period
        self.nv = ctypes.CDLL("libnvidia-ml.so.1")
        if self.nv.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(gpu_index), ctypes.byref(self.h)) != 0:
            raise RuntimeError("no NVML handle")
        self.rows, self.stop_flag, self.thread = [], False, None

    def _read(self):
        import ctypes

        mhz, mx, mw = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_uint()
        reasons = ctypes.c_ulonglong()
        self.nv.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(mhz))  # NVML_CLOCK_SM
        self.nv.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx))
        self.nv.nvmlDeviceGetPowerUsage(self.h, ctypes.byref(mw))
        self.nv.nvmlDeviceGetCurrentClocksEventReasons(self.h, ctypes.byref(reasons))
        return mhz.value, mx.value, mw.value / 1e3, reasons.value

    def start(self):
        import threading

        def loop():
            while not self.stop_flag:
                self.rows.append(self._read())
                time.sleep(self.period)

        self.rows.append(self._read())
        self.thread = threading.Thread(target=loop, daemon=True)
        self.thread.start()

    def stop(self):
        self.stop_flag = True
        if self.thread:
            self.thread.join()
        self.rows.append(self._read())
        sm = [r[0] for r in self.rows]
        reasons = sorted({name for r in self.rows for bit, name in self.REASONS.items() if r[3] & bit})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(r[1] for r in self.rows), "reasons": reasons,
                "samples": len(self.rows), "power_w_max": max(r[2] for r in self.rows), "source": "nvml",
                "period_ms": self.period * 1e3}


def clock_sampler(gpu_index):
    """NVML sampling when the library is there, else nvidia-smi."""
    try:
        return NvmlSampler(gpu_index)
    except Exception:
        return ClockSampler(gpu_index)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "source": "nvidia-smi"}


def issue_roofline(inst_per_env_step, env_steps_per_s, clk):
    if inst_per_env_step is None or not clk or not clk.get("sm_mhz"):
        return None
    import torch

    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak = 4.0 * sms * clk["sm_mhz"] * 1e6
    achieved = inst_per_env_step * env_steps_per_s
    return {"achieved": achieved, "peak": peak, "unit": "warp-inst/s", "frac": achieved / peak,
            "warp_inst_per_env_step": inst_per_env_step, "sms": sms,
            "peak_kind": "4 warp instructions per cycle per SM at the sampled SM clock"}


def workload(name):
    c = W.WORKLOADS[name]()
    return c


def shape_classes(descs, n_envs):
    """Env indices grouped by kernel shape (everything but the obstacle
    density): the 'per-config' form launches one engine per class."""
    classes = {}
    for e in range(n_envs):
        d = descs[0 if len(descs) == 1 else e]
        key = (d["side"], d["n_agents"], d["n_seekers"], d["r_seek"], d["r_hide"], d["cap"], d["obs_teams"])
        classes.setdefault(key, []).append(e)
    return classes


def build_form(form, c, run, flags, stream, base, log):
    """Engines and the benchmark step of one form of the workload.
    plain:      one engine, default launch configuration, hase_step;
    batched:    one engine, autotuned configuration, the rollout replayed as
                a CUDA graph (hase_step_graph);
    per-config: one engine per kernel-shape class of the batch, launched one
                after another on the stream (each class's envs get their
                own env-id range, so its trajectories differ from the
                batched run's while the workload is the same)."""
    from paper_2604_27162_gb300 import autotune, hase

    n_envs = c["n_envs"]
    extra = {"form": form}
    if form == "per-config":
        engines = []
        next_id = base
        for key, idx in sorted(shape_classes(c["descs"], n_envs).items()):
            descs = [c["descs"][0 if len(c["descs"]) == 1 else e] for e in idx]
            engines.append(hase.Engine(len(idx), c["seed"], descs, ring_steps=run, flags=flags,
                                       env_id_base=next_id, stream=stream))
            next_id += len(idx)
        extra["classes"] = len(engines)

        def step():
            for eng in engines:
                eng.step(run)
        launches = sum(math.ceil(run / (e.launch_info()["steps_per_launch"] or 65536)) + 1 for e in engines)
        return engines, step, launches, extra
    setting = {}
    if form == "batched":
        t = time.perf_counter()
        knobs = [(k, v) for k, v in autotune.KNOBS if k != "step_form" or not flags & (
            H.HASE_CHUNKED_STEP | H.HASE_STREAM_STEP)]  # a form given on the command line is kept
        # every candidate is timed on the run's own length: a shorter probe
        # overweights the per-launch prologue of CTAs that run in waves
        setting, trials = autotune.tune(n_envs, c["seed"], c["descs"], flags, probe_steps=run, stream=stream, log=log,
                                        knobs=knobs)
        extra["autotune"] = {"setting": setting, "trials": len(trials),
                             "seconds": round(time.perf_counter() - t, 1)}
    eng = hase.Engine(n_envs, c["seed"], c["descs"], ring_steps=run, flags=flags, env_id_base=base,
                      stream=stream, **setting)
    spl = eng.launch_info()["steps_per_launch"] or 65536
    if form == "batched":
        def step():
            eng.step_graph(run)
    else:
        def step():
            eng.step(run)
    return [eng], step, math.ceil(run / spl) + 1, extra


def time_form(step, steps, warmup, stream):
    import torch

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2604_27162_gb300 import hase
    from paper_2604_27162_gb300 import shard as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    hase.load()
    c, flags = apply_mode(workload(args.workload), args.mode)
    flags |= H.STEP_FORMS[args.step_form]
    n_envs = c["n_envs"]
    run = args.run_steps or RUN_STEPS[args.workload]
    # weak scaling: rank r steps envs [r*E, (r+1)*E) of the global batch
    stream = torch.cuda.current_stream()
    form = args.form or ("batched" if args.workload == "uneven64k" else "plain")
    log = (lambda m: print(m, file=sys.stderr)) if rank == 0 else None
    engines, one_step, launches_per_step, form_info = build_form(
        form, c, run, flags, stream, S.env_base(rank, n_envs), log)
    eng = engines[0]
    info = eng.launch_info()

    clocks = clock_sampler(local)  # from the warm-up on, through the timed region
    clocks.start()
    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0.record(stream)
    for _ in range(args.steps):
        one_step()
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1)
    ms = S.max_over_ranks(ms, device="cuda")
    agents = sum(c["descs"][0 if len(c["descs"]) == 1 else e]["n_agents"] for e in range(n_envs))
    value = S.weak_throughput(n_envs * run * args.steps, world, ms / 1e3)
    bpe = algorithmic_bytes_per_env_step(c["descs"], n_envs, c["unpacked"], flags)
    per_rank_bytes = bpe * n_envs * run * args.steps
    achieved = per_rank_bytes / (ms / 1e3) / 1e9
    peak, peak_kind = peaks()
    tpe = measured_traffic(args.workload) if args.mode == "default" else None
    ipe = measured_traffic(args.workload, "warp_inst_per_env_step") if args.mode == "default" else None
    traffic = tpe * n_envs * run if tpe is not None else None  # bytes per launch

    # end to end through the public API: every step's results copied to
    # pinned host memory inside the timed region (no per-step inputs exist:
    # actions are drawn on the device)
    e2e = None if args.no_e2e or len(engines) > 1 else run_e2e(eng, c, run, stream, args)
    # the batched form is reported against the other two forms on this GPU
    if form == "batched" and rank == 0 and not args.no_compare:
        cmp_steps = max(3, min(args.steps, 20))
        for other in ("plain", "per-config"):
            en2, st2, _, _ = build_form(other, c, run, flags, stream, 0, None)
            ms2 = time_form(st2, cmp_steps, 2, stream)
            form_info["%s_env_steps_per_s" % other.replace("-", "_")] = n_envs * run * cmp_steps / (ms2 / 1e3)
            for e2 in en2:
                e2.close()
    for e in engines:
        e.close()
    if rank == 0:
        out = {
            "metric": "env-steps/s",
            "value": value,
            "unit": "env-steps/s",
            "agent_steps_per_s": value * agents / n_envs,
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "u32",
            "data": "synthetic (seeded Bernoulli maps, Philox actions)",
            "config": {
                "workload": args.workload,
                "mode": args.mode,
                "step_form": args.step_form,
                "flags": flags,
                "n_envs_per_gpu": n_envs,
                "env_steps_per_bench_step": run,
                "descs": c["descs"] if len(c["descs"]) == 1 else "per-env table (%d)" % n_envs,
                "ring_steps": run,
                "l2": "outputs larger than L2 (ring %.2f GB)" % (per_rank_bytes / args.steps / 1e9),
                "ctas": info["ctas"],
                "threads_per_cta": info["threads"],
                "smem_per_cta": info["smem"],
                "parallelism": "env shards, one process per GPU" if world > 1 else "1 GPU",
                **form_info,
            },
            "roofline": {
                "bound": "hbm",
                "kernel": "step_kernel",
                "achieved": achieved,
                "peak": peak,
                "peak_kind": peak_kind + " (HBM copy burst, kernel timed alone)",
                "unit": "GB/s",
                "frac": achieved / peak,
                "algorithmic_bytes_per_env_step": bpe,
                "algorithmic_bytes_per_launch": bpe * n_envs * run,
                "traffic": traffic,
            },
            # the SM instruction-issue view of the same kernel: ncu warp
            # instructions per env-step x env-steps/s against 4 warp
            # instructions per cycle per SM at the sampled SM clock
            "issue": issue_roofline(ipe, value / world, clk),
            "gpu_launches": args.steps * launches_per_step,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu_baseline(c, args, flags) if world == 1 and not args.no_cpu else None,
        }
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def engine_exports(eng):
    """(name, device ring view) of every output the handle writes."""
    out = [("obs", eng.obs), ("reward", eng.reward), ("done", eng.done)]
    for k in ("unpacked", "central", "cells", "ep_t", "fog"):
        v = getattr(eng, k)
        if v is not None:
            out.append((k, v))
    return [(k, v) for k, v in out if v.shape[1] > 0]


def gpu_local_cpus():
    """The CPUs NVML names as closest to the current CUDA device (read-only
    query), intersected with this process's; None when unknown."""
    import ctypes

    import torch

    try:
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        nv = ctypes.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            return None
        h = ctypes.c_void_p()
        if nv.nvmlDeviceGetHandleByUUID(("GPU-%s" % props.uuid).encode(), ctypes.byref(h)) != 0:
            return None
        words = (ctypes.c_ulong * 64)()
        if nv.nvmlDeviceGetCpuAffinity(h, ctypes.c_uint(64), words) != 0:
            return None
        bits = 8 * ctypes.sizeof(ctypes.c_ulong)
        cpus = {bits * i + b for i in range(64) for b in range(bits) if (words[i] >> b) & 1}
        cpus &= os.sched_getaffinity(0)
        return cpus or None
    except Exception:
        return None


def pinned_near_gpu(make):
    """Run make() (pinned host allocations) on the GPU-local CPUs, so that
    the pages land in the memory next to the GPU's host link."""
    cpus = gpu_local_cpus()
    if not cpus:
        return make(), "default placement"
    old = os.sched_getaffinity(0)
    try:
        os.sched_setaffinity(0, cpus)
        return make(), "allocated on the %d GPU-local CPUs (NVML affinity)" % len(cpus)
    finally:
        os.sched_setaffinity(0, old)


def run_e2e(eng, c, run, stream, args):
    """The rollout through the public API with every step's outputs copied to
    pinned host memory inside the timed region: the steps of chunk k + 1 run
    on the compute stream while chunk k's slots are copied on a second stream
    (events order them; a chunk's slots are stepped again only after their
    copy).  Beside it: the pinned device-to-host copy rate of the same chunk
    bytes alone, the link's measured peak for this traffic."""
    import torch

    n_steps = run * max(1, min(args.steps, 3))
    ex = engine_exports(eng)
    per_step = sum(v.shape[1] * v.element_size() for _, v in ex)
    # chunks of at most 1,000 steps and 1 GiB of pinned staging a buffer, a
    # divisor of the ring so that no chunk wraps round it (one copy per ring)
    limit = max(1, min(1000, run, (1 << 30) // per_step))
    chunk = max(d for d in range(1, limit + 1) if eng.ring % d == 0)
    nbytes = chunk * per_step
    (host, hst), placement = pinned_near_gpu(lambda: (
        [[torch.empty((chunk, v.shape[1]), dtype=v.dtype, pin_memory=True) for _, v in ex] for _ in range(2)],
        torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)))
    copy = torch.cuda.Stream()
    done_copy = {}  # ring chunk index -> event after its copy
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    done_steps, k = 0, 0
    while done_steps < n_steps:
        n = min(chunk, n_steps - done_steps)
        s0 = eng.t % eng.ring
        idx = [(s0 + i) % eng.ring for i in range(n)]
        for sl in {i // chunk for i in idx}:  # the slots' previous copy must be done
            if sl in done_copy:
                stream.wait_event(done_copy[sl])
        eng.step(n)
        stepped = torch.cuda.Event()
        stepped.record(stream)
        copy.wait_event(stepped)
        hb = host[k % 2]
        with torch.cuda.stream(copy):
            for (_, v), h in zip(ex, hb):
                if idx[0] + n <= eng.ring:
                    h[:n].copy_(v[idx[0]:idx[0] + n], non_blocking=True)
                else:
                    for j, sl in enumerate(idx):
                        h[j].copy_(v[sl], non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(copy)
        for sl in {i // chunk for i in idx}:
            done_copy[sl] = ev
        done_steps += n
        k += 1
    stream.wait_stream(copy)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    # the same bytes copied alone (pinned, one stream): the link's rate for this traffic
    v0 = ex[0][1]
    dev = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    for _ in range(2):
        hst.copy_(dev, non_blocking=True)
    torch.cuda.synchronize()
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    reps = 5
    c0.record()
    for _ in range(reps):
        hst.copy_(dev, non_blocking=True)
    c1.record()
    torch.cuda.synchronize()
    link = reps * nbytes / (c0.elapsed_time(c1) / 1e3) / 1e9
    del dev, hst, v0
    achieved = per_step * n_steps / (ms / 1e3) / 1e9
    return {"value": eng.n_envs * n_steps / (ms / 1e3), "unit": "env-steps/s",
            "h2d_bytes_per_step": 0, "d2h_bytes_per_step": int(per_step),
            "d2h_gbs": achieved, "d2h_link_peak_gbs": link, "link_frac": achieved / link, "host_memory": placement,
            "note": "per env-step: every output ring slot (%s) copied to pinned host memory, overlapped with the "
                    "next chunk's steps; link peak = the same chunk bytes copied alone" % ", ".join(k for k, _ in ex)}


def _oracle_shard(job):
    """One host process of the multi-core oracle leg: its env range of the
    workload stepped for about `seconds`."""
    n, base, seed, descs, unpacked, seconds, flags = job
    sys.path.insert(0, ROOT)
    import oracle

    w = oracle.World(n, seed, descs, env_id_base=base, desync=bool(flags & H.HASE_DESYNC_START),
                     fog=oracle_fog(flags))
    t = time.perf_counter()
    steps = 0
    while time.perf_counter() - t < seconds:
        oracle_step(w, flags, unpacked)
        steps += 1
    dt = time.perf_counter() - t
    w.close()
    return n, steps, dt


def cpu_baseline(c, args, flags=0, target_s=8.0):
    """The oracle (single-threaded C, as it stands) on a bounded sample of the
    same workload: all envs of the batch for as many steps as fit target_s,
    on one core and as one process per host core over env shards (spawned:
    the parent holds a CUDA context)."""
    import multiprocessing as mp

    import oracle

    n = c["n_envs"]
    w = oracle.World(n, c["seed"], c["descs"], desync=bool(flags & H.HASE_DESYNC_START), fog=oracle_fog(flags))
    t = time.perf_counter()
    steps = 0
    while time.perf_counter() - t < target_s:
        oracle_step(w, flags, c["unpacked"])
        steps += 1
    dt = time.perf_counter() - t
    single = {"value": n * steps / dt, "unit": "env-steps/s", "cores": 1,
              "sample": "%d envs x %d steps (%.1f s)" % (n, steps, dt)}
    cores = max(1, min(os.cpu_count() or 1, n))
    jobs = []
    for i in range(cores):
        lo, hi = i * n // cores, (i + 1) * n // cores
        d = c["descs"] if len(c["descs"]) == 1 else c["descs"][lo:hi]
        jobs.append((hi - lo, lo, c["seed"], d, c["unpacked"], target_s, flags))
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_shard, jobs)
        value = sum(r[0] * r[1] / r[2] for r in res)
        return {"value": value, "unit": "env-steps/s", "cores": cores, "kind": "oracle",
                "sample": "%d envs in %d shards, %d-%d steps each (~%.0f s), one process per core"
                          % (n, cores, min(r[1] for r in res), max(r[1] for r in res), target_s),
                "single_core": single}
    except Exception as exc:  # no pool possible: report the single-core leg
        single.update({"kind": "oracle", "note": "multi-core leg failed: %s" % exc})
        return single


def request_bytes_algorithmic(r):
    d = r["desc"]
    return r["n_envs"] * r["steps"] * algorithmic_bytes_per_env_step([d], 1, False)


def run_served(args):
    """Served rollouts: the Poisson request stream through the rollout server
    (continuous batching into shared launches under the HBM budget); the
    server's capacity (the same stream submitted at once) and p50/p99 latency
    against the arrival rate; the stream served with every request in its own
    handle (no shared launches) for comparison; the oracle on a sample of the
    requests as the CPU baseline."""
    import torch

    from paper_2604_27162_gb300 import hase

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    hase.load()
    budget = int(args.budget_gb * (1 << 30))

    def summarize(res, reqs_):
        ok = [i for i, r in enumerate(res) if r["status"] == hase.HASE_OK]
        lat = sorted(res[i]["finished"] - res[i]["submitted"] for i in ok)
        span = max((res[i]["finished"] for i in ok), default=0.0) - min((res[i]["submitted"] for i in ok), default=0.0)
        env_steps = sum(reqs_[i]["n_envs"] * reqs_[i]["steps"] for i in ok)
        agent_steps = sum(reqs_[i]["n_envs"] * reqs_[i]["steps"] * reqs_[i]["desc"]["n_agents"] for i in ok)
        q = lambda p: lat[min(len(lat) - 1, int(p * len(lat)))] if lat else None
        return {"requests": len(reqs_), "ok": len(ok), "env_steps": env_steps, "agent_steps": agent_steps,
                "env_steps_per_s": env_steps / span if span else None,
                "agent_steps_per_s": agent_steps / span if span else None,
                "p50_ms": q(0.50) * 1e3 if lat else None, "p99_ms": q(0.99) * 1e3 if lat else None,
                "makespan_s": span,
                "mean_batch": sum(res[i]["batch_size"] for i in ok) / max(1, len(ok))}

    def serve(reqs_, time_scale, max_batch=0):
        res, st = hase.hase_serve(reqs_, budget, n_streams=args.streams, max_inflight=4096, time_scale=time_scale,
                                  max_batch=max_batch)
        return summarize(res, reqs_), st, res

    hase.hase_serve(W.served_requests(duration=0.05), budget, n_streams=args.streams)  # warm-up
    reqs = W.served_requests(duration=args.duration)
    clocks = clock_sampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    s, stats, res = serve(reqs, 1.0)  # the stream at its own pace: 2,000 requests/s
    clk = clocks.stop()
    # capacity: a few seconds of the stream submitted at once; latency against rate
    head = [r for r in reqs if r["arrival"] < args.sweep_seconds]
    cap, _, _ = serve(head, 0.0)
    sweep = []
    for rate in args.rates:
        sub = W.served_requests(rate=rate, duration=args.sweep_seconds)
        r_, _, _ = serve(sub, 1.0)
        sweep.append({"rate_per_s": rate, **{k: r_[k] for k in ("requests", "env_steps_per_s", "p50_ms", "p99_ms",
                                                                  "mean_batch")}})
    unshared, _, _ = serve(head, 0.0, max_batch=1)  # every request its own handle and launches
    alg = sum(request_bytes_algorithmic(reqs[i]) for i, r in enumerate(res) if r["status"] == hase.HASE_OK)
    achieved = alg / s["makespan_s"] / 1e9
    peak, peak_kind = peaks()
    out = {
        "metric": "env-steps/s",
        "value": s["env_steps_per_s"],
        "unit": "env-steps/s",
        "agent_steps_per_s": s["agent_steps_per_s"],
        "latency_ms": {"p50": s["p50_ms"], "p99": s["p99_ms"]},
        "n_gpus": 1,
        "steps": 1,
        "warmup": 1,
        "ms_per_step": s["makespan_s"] * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic (Poisson request stream, seeded Bernoulli maps, Philox actions)",
        "config": {
            "workload": "served",
            "rate_per_s": 2000.0, "duration_s": args.duration, "requests": s["requests"],
            "served_ok": s["ok"], "budget_gb": args.budget_gb, "streams": args.streams,
            "peak_bytes": stats["peak_bytes"], "peak_inflight": stats["peak_inflight"],
            "rejected": stats["rejected"], "batches": stats["batches"], "mean_batch": s["mean_batch"],
            "capacity": {"seconds_of_stream": args.sweep_seconds, "submitted_at_once": True, **cap},
            "capacity_env_steps_per_s": cap["env_steps_per_s"],
            "unshared": {"note": "the same requests, every one its own handle and launches", **unshared},
            "rate_sweep": sweep,
            "l2": "outputs of every request resident until its digest (far above L2 in total)",
        },
        "roofline": {"bound": "hbm", "kernel": "step_kernel", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "note": "offered load of the 2,000 requests/s stream, not capacity (see config.capacity)"},
        "gpu_launches": None,
        "clocks": clk,
        "e2e": {"value": s["env_steps_per_s"], "unit": "env-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 32,
                "note": "the server is the public API: per request the 32-byte digest comes back"},
        "cpu_baseline": None if args.no_cpu else served_cpu_baseline(reqs),
    }
    print(json.dumps(out))


def served_cpu_baseline(reqs, target_s=10.0):
    """The oracle on the host, one core: requests of the stream run back to
    back (every step of every env, digest included) for about target_s."""
    import oracle

    t0 = time.perf_counter()
    done_env = n = 0
    for r in reqs:
        w = oracle.World(r["n_envs"], r["seed"], [r["desc"]])
        w.run_digest(r["steps"])
        w.close()
        n += 1
        done_env += r["n_envs"] * r["steps"]
        if time.perf_counter() - t0 > target_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done_env / dt, "unit": "env-steps/s", "cores": 1, "kind": "oracle",
            "sample": "first %d requests of the stream, back to back (%.1f s)" % (n, dt)}


def run_reference_served(args, world):
    """Reference arm of the served workload: the oracle runs requests of the
    same stream one after another (digest of every step) for about a minute."""
    import oracle

    reqs = W.served_requests(duration=args.duration)
    budget = 60.0
    t0 = time.perf_counter()
    done_env_steps = done_agent_steps = n = 0
    for r in reqs:
        w = oracle.World(r["n_envs"], r["seed"], [r["desc"]])
        w.run_digest(r["steps"])
        w.close()
        n += 1
        done_env_steps += r["n_envs"] * r["steps"]
        done_agent_steps += r["n_envs"] * r["steps"] * r["desc"]["n_agents"]
        if time.perf_counter() - t0 > budget:
            break
    dt = time.perf_counter() - t0
    value = done_env_steps / dt
    print(json.dumps({
        "impl": "reference", "metric": "env-steps/s", "value": value, "unit": "env-steps/s",
        "agent_steps_per_s": done_agent_steps / dt, "n_gpus": world, "steps": 1, "warmup": 0,
        "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic (Poisson request stream)",
        "config": {"workload": "served", "requests_run": n},
        "cpu_baseline": {"value": value, "unit": "env-steps/s", "cores": 1, "kind": "oracle",
                         "sample": "first %d requests of the stream, run back to back" % n},
        "e2e": {"value": value, "unit": "env-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_reference(args):
    """Reference arm: the oracle timed on the host cores, same metric."""
    import oracle

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload == "served":
        return run_reference_served(args, world)
    c, flags = apply_mode(workload(args.workload), args.mode)
    n = c["n_envs"]
    desync, fog = bool(flags & H.HASE_DESYNC_START), oracle_fog(flags)
    # bounded sample: each benchmark step runs a sample of the rollout, sized
    # so that warmup + steps take about a minute in total
    probe = oracle.World(n, c["seed"], c["descs"], desync=desync, fog=fog)
    t = time.perf_counter()
    oracle_step(probe, flags, c["unpacked"])
    per_env_step = (time.perf_counter() - t) / n
    budget = 60.0 / max(1, args.steps + args.warmup)
    sample_envs = max(1, min(n, int(budget / max(per_env_step, 1e-9))))
    sample_steps = 1
    w = oracle.World(sample_envs, c["seed"], c["descs"][:1] if len(c["descs"]) == 1 else
                     c["descs"][:sample_envs], desync=desync, fog=fog)
    for _ in range(args.warmup):
        oracle_step(w, flags, c["unpacked"])
    t = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(sample_steps):
            oracle_step(w, flags, c["unpacked"])
    dt = time.perf_counter() - t
    value = sample_envs * sample_steps * args.steps / dt
    out = {
        "impl": "reference",
        "metric": "env-steps/s",
        "value": value,
        "unit": "env-steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic (seeded Bernoulli maps, Philox actions)",
        "config": {"workload": args.workload, "mode": args.mode, "flags": flags, "n_envs_per_gpu": n},
        "cpu_baseline": {"value": value, "unit": "env-steps/s", "cores": 1, "kind": "oracle",
                         "sample": "%d of %d envs, 1 env-step per benchmark step" % (sample_envs, n)},
        "e2e": {"value": value, "unit": "env-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="ten1k", choices=sorted(RUN_STEPS))
    ap.add_argument("--mode", default="default", choices=list(MODES),
                    help="optional part of the step to include (observability modes, line of sight, "
                         "desynchronised start, fog of war)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--run-steps", type=int, default=0,
                    help="override the env-steps per benchmark step (small profiling cases)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--form", choices=["plain", "batched", "per-config"], default=None,
                    help="launch form (default: batched for uneven64k, plain otherwise)")
    ap.add_argument("--duration", type=float, default=60.0, help="served: seconds of the request stream")
    ap.add_argument("--budget-gb", type=float, default=64.0, help="served: device memory budget")
    ap.add_argument("--streams", type=int, default=16, help="served: CUDA streams of the server")
    ap.add_argument("--sweep-seconds", type=float, default=2.0,
                    help="served: seconds of stream per capacity and rate-sweep point")
    ap.add_argument("--rates", type=float, nargs="*", default=[1000.0, 2000.0, 4000.0, 8000.0, 16000.0],
                    help="served: arrival rates of the latency sweep (requests/s)")
    ap.add_argument("--step-form", choices=sorted(H.STEP_FORMS), default="auto",
                    help="step kernel form: auto (the engine's choice; the batched form lets the autotuner "
                         "choose), chunked or stream")
    ap.add_argument("--no-compare", action="store_true",
                    help="batched form: skip timing the plain and per-config forms beside it")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "served":
        run_served(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
