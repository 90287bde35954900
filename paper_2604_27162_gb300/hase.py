"""Thin Python binding of the C ABI in ``include/hase.h`` (ctypes).

Every function here only marshals arguments: the environment step runs in
``libhase.so`` (CUDA kernels for sm_103a).  There is no CPU fallback: if the
library is missing or no CUDA device is present, the calls raise.

The C names are mirrored one to one (``hase_create``, ``hase_step``, ...).
``Engine`` is a convenience owner of one handle that exposes the device
output rings as zero-copy torch tensors (through ``__cuda_array_interface__``;
PyTorch is used for device memory views and streams only).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhase.so")

HASE_OK, HASE_EINVAL, HASE_ENOMEM, HASE_ECUDA, HASE_ETIMEOUT, HASE_EBUSY, HASE_ESTATE = range(7)
HASE_EXPORT_ACTIONS = 1
HASE_EXPORT_UNPACKED = 2
HASE_ASYNC_CREATE = 4
HASE_POOL_ALLOC = 8
HASE_DESYNC_START = 16
HASE_EXPORT_CENTRAL = 32
HASE_EXPORT_STATE = 64
HASE_SKIP_OBS = 128
HASE_EXPORT_FOG = 256
HASE_FOG_PER_AGENT = 512
HASE_CHUNKED_STEP = 1024
HASE_STREAM_STEP = 2048
STEP_FORMS = {"auto": 0, "chunked": HASE_CHUNKED_STEP, "stream": HASE_STREAM_STEP}
HASE_OBS_LOS = 4
HASE_OBS_SEEKERS = 1
HASE_OBS_HIDERS = 2
STATUS_NAMES = {0: "HASE_OK", 1: "HASE_EINVAL", 2: "HASE_ENOMEM", 3: "HASE_ECUDA",
                4: "HASE_ETIMEOUT", 5: "HASE_EBUSY", 6: "HASE_ESTATE"}

# Every symbol include/hase.h declares (the CPU tests check the export list).
EXPORTS = [
    "hase_create", "hase_reset", "hase_step", "hase_step_graph", "hase_digest", "hase_digest_range",
    "hase_digest_noalloc",
    "hase_obs_ptr", "hase_reward_ptr", "hase_done_ptr",
    "hase_actions_ptr", "hase_central_ptr", "hase_state_ptr", "hase_fog_ptr", "hase_layout_get", "hase_step_count", "hase_get_state", "hase_set_state",
    "hase_get_world", "hase_sync", "hase_launch_info", "hase_destroy", "hase_last_error",
    "hase_request_bytes", "hase_serve", "hase_server_create", "hase_server_submit", "hase_server_poll",
    "hase_server_stats", "hase_server_shutdown", "hase_server_destroy",
]


class HaseError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class hase_env_desc(C.Structure):
    _fields_ = [(n, C.c_uint32) for n in (
        "side", "n_agents", "n_seekers", "r_seek", "r_hide", "cap", "density_thr", "obs_teams")]


class hase_config(C.Structure):
    _fields_ = [
        ("n_envs", C.c_uint32),
        ("env_id_base", C.c_uint32),
        ("seed", C.c_uint64),
        ("envs", C.POINTER(hase_env_desc)),
        ("n_desc", C.c_uint32),
        ("ring_steps", C.c_uint32),
        ("flags", C.c_uint32),
        ("steps_per_launch", C.c_uint32),
        ("chunk_steps", C.c_uint32),
        ("emit_warps", C.c_uint32),
        ("max_group_envs", C.c_uint32),
        ("smem_cap", C.c_uint32),
        ("env_seeds", C.POINTER(C.c_uint64)),
        ("env_ids", C.POINTER(C.c_uint32)),
    ]


class hase_digest_out(C.Structure):
    _fields_ = [
        ("digest", C.c_uint64),
        ("episodes", C.c_uint64),
        ("reward_sum", C.c_int64),
        ("gen_error", C.c_uint32),
        ("pad", C.c_uint32),
    ]


class hase_request(C.Structure):
    _fields_ = [
        ("arrival", C.c_double),
        ("seed", C.c_uint64),
        ("n_envs", C.c_uint32),
        ("steps", C.c_uint32),
        ("desc", hase_env_desc),
    ]


class hase_serve_config(C.Structure):
    _fields_ = [
        ("budget_bytes", C.c_uint64),
        ("n_streams", C.c_uint32),
        ("max_inflight", C.c_uint32),
        ("time_scale", C.c_double),
        ("max_batch", C.c_uint32),
        ("pad", C.c_uint32),
    ]


class hase_server_config(C.Structure):
    _fields_ = [
        ("budget_bytes", C.c_uint64),
        ("n_streams", C.c_uint32),
        ("max_inflight", C.c_uint32),
        ("queue_capacity", C.c_uint32),
        ("max_batch_envs", C.c_uint32),
        ("max_batch", C.c_uint32),
        ("pad", C.c_uint32),
    ]


class hase_request_result(C.Structure):
    _fields_ = [
        ("submitted", C.c_double),
        ("admitted", C.c_double),
        ("finished", C.c_double),
        ("digest", C.c_uint64),
        ("episodes", C.c_uint64),
        ("reward_sum", C.c_int64),
        ("bytes", C.c_uint64),
        ("status", C.c_uint32),
        ("batch_size", C.c_uint32),
    ]


class hase_serve_stats(C.Structure):
    _fields_ = [
        ("makespan", C.c_double),
        ("peak_bytes", C.c_uint64),
        ("peak_inflight", C.c_uint32),
        ("rejected", C.c_uint32),
        ("batches", C.c_uint64),
        ("requests", C.c_uint64),
    ]


class hase_layout(C.Structure):
    _fields_ = [
        ("n_envs", C.c_uint32),
        ("ring_steps", C.c_uint32),
        ("agents", C.c_uint64),
        ("obs_words", C.c_uint64),
        ("unp_bytes", C.c_uint64),
        ("agent_off", C.POINTER(C.c_uint64)),
        ("obs_off", C.POINTER(C.c_uint64)),
        ("unp_off", C.POINTER(C.c_uint64)),
        ("central_words", C.c_uint64),
        ("central_off", C.POINTER(C.c_uint64)),
        ("fog_words", C.c_uint64),
        ("fog_off", C.POINTER(C.c_uint64)),
    ]


_lib = None


def load(path=LIB_PATH):
    """Load libhase.so (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libhase.so is not built (%s); run __graft_entry__.build()" % path)
    L = C.CDLL(path)
    P, H = C.c_void_p, C.c_void_p
    u32, u64 = C.c_uint32, C.c_uint64
    st = C.c_int
    L.hase_create.argtypes = [C.POINTER(hase_config), P, C.POINTER(H)]
    L.hase_reset.argtypes = [H, P]
    L.hase_step.argtypes = [H, u32, P]
    L.hase_step_graph.argtypes = [H, u32, P]
    L.hase_digest.argtypes = [H, u32, P, P, P]
    L.hase_digest_noalloc.argtypes = [H, u32, P, P, P]
    L.hase_digest_range.argtypes = [H, u64, u32, u32, u32, P, P, P]
    L.hase_request_bytes.argtypes = [C.POINTER(hase_request)]
    L.hase_server_create.argtypes = [C.POINTER(hase_server_config), C.POINTER(P)]
    L.hase_server_submit.argtypes = [P, C.POINTER(hase_request), C.POINTER(u64)]
    L.hase_server_poll.argtypes = [P, u64, C.c_double, C.POINTER(hase_request_result)]
    L.hase_server_stats.argtypes = [P, C.POINTER(hase_serve_stats)]
    L.hase_server_shutdown.argtypes = [P]
    L.hase_server_destroy.argtypes = [P]
    L.hase_server_destroy.restype = None
    L.hase_serve.argtypes = [C.POINTER(hase_request), u32, C.POINTER(hase_serve_config),
                             C.POINTER(hase_request_result), C.POINTER(hase_serve_stats)]
    L.hase_obs_ptr.argtypes = [H, C.POINTER(P), C.POINTER(P)]
    L.hase_reward_ptr.argtypes = [H, C.POINTER(P)]
    L.hase_done_ptr.argtypes = [H, C.POINTER(P)]
    L.hase_actions_ptr.argtypes = [H, C.POINTER(P)]
    L.hase_central_ptr.argtypes = [H, C.POINTER(P)]
    L.hase_state_ptr.argtypes = [H, C.POINTER(P), C.POINTER(P)]
    L.hase_fog_ptr.argtypes = [H, C.POINTER(P)]
    L.hase_layout_get.argtypes = [H, C.POINTER(hase_layout)]
    L.hase_step_count.argtypes = [H, C.POINTER(u64)]
    L.hase_get_state.argtypes = [H, P, C.POINTER(C.c_size_t), P]
    L.hase_set_state.argtypes = [H, P, C.c_size_t, P]
    L.hase_get_world.argtypes = [H, u32, P, P]
    L.hase_sync.argtypes = [H]
    L.hase_launch_info.argtypes = [H, C.POINTER(u32), C.POINTER(u32), C.POINTER(u32), C.POINTER(u32)]
    L.hase_destroy.argtypes = [H]
    L.hase_destroy.restype = None
    L.hase_last_error.argtypes = [H]
    L.hase_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("hase_destroy", "hase_last_error"):
            getattr(L, name).restype = st
    L.hase_request_bytes.restype = u64
    _lib = L
    return L


def _check(status, h=None):
    if status != HASE_OK:
        msg = load().hase_last_error(h)
        raise HaseError(status, msg.decode() if msg else "")


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------------------
# C names, one to one.
# ---------------------------------------------------------------------------
def make_config(n_envs, seed, descs, ring_steps, flags=0, env_id_base=0, steps_per_launch=0,
                chunk_steps=0, emit_warps=0, max_group_envs=0, smem_cap=0, env_seeds=None, env_ids=None):
    arr = (hase_env_desc * len(descs))()
    for i, d in enumerate(descs):
        for k, _ in hase_env_desc._fields_:
            setattr(arr[i], k, int(d[k]))
    seeds = ids = None
    if env_seeds is not None:
        seeds = (C.c_uint64 * n_envs)(*[int(v) & (2**64 - 1) for v in env_seeds])
    if env_ids is not None:
        ids = (C.c_uint32 * n_envs)(*[int(v) for v in env_ids])
    cfg = hase_config(n_envs=n_envs, env_id_base=env_id_base, seed=seed & (2**64 - 1),
                      envs=C.cast(arr, C.POINTER(hase_env_desc)), n_desc=len(descs),
                      ring_steps=ring_steps, flags=flags, steps_per_launch=steps_per_launch,
                      chunk_steps=chunk_steps, emit_warps=emit_warps, max_group_envs=max_group_envs,
                      smem_cap=smem_cap,
                      env_seeds=C.cast(seeds, C.POINTER(C.c_uint64)) if seeds is not None else None,
                      env_ids=C.cast(ids, C.POINTER(C.c_uint32)) if ids is not None else None)
    cfg._keep = (arr, seeds, ids)  # keep the host arrays alive
    return cfg


def hase_create(cfg, stream=None):
    h = C.c_void_p()
    _check(load().hase_create(C.byref(cfg), _stream(stream), C.byref(h)))
    return h


def hase_reset(h, stream=None):
    _check(load().hase_reset(h, _stream(stream)), h)


def hase_step(h, n_steps, stream=None):
    _check(load().hase_step(h, n_steps, _stream(stream)), h)


def hase_step_graph(h, n_steps, stream=None):
    _check(load().hase_step_graph(h, n_steps, _stream(stream)), h)


def hase_digest(h, n_steps, out_ptr, agent_rew_ptr=None, stream=None):
    """Enqueue the digest of the last n_steps steps into device memory at
    out_ptr (a hase_digest_out) and, optionally, per-agent reward sums."""
    _check(load().hase_digest(h, n_steps, C.c_void_p(out_ptr), C.c_void_p(agent_rew_ptr or 0),
                              _stream(stream)), h)


def _requests(reqs):
    arr = (hase_request * max(1, len(reqs)))()
    for i, r in enumerate(reqs):
        arr[i].arrival = float(r["arrival"])
        arr[i].seed = int(r["seed"]) & (2**64 - 1)
        arr[i].n_envs = int(r["n_envs"])
        arr[i].steps = int(r["steps"])
        for k, _ in hase_env_desc._fields_:
            setattr(arr[i].desc, k, int(r["desc"][k]))
    return arr


def hase_request_bytes(r):
    return int(load().hase_request_bytes(C.byref(_requests([r])[0])))


def hase_serve(reqs, budget_bytes, n_streams=16, max_inflight=1024, time_scale=1.0, max_batch=0):
    """Serve the request list (dicts with arrival, seed, n_envs, steps, desc)
    and return (per-request result dicts, stats dict)."""
    arr = _requests(reqs)
    cfg = hase_serve_config(budget_bytes=int(budget_bytes), n_streams=n_streams, max_inflight=max_inflight,
                            time_scale=float(time_scale), max_batch=max_batch)
    res = (hase_request_result * max(1, len(reqs)))()
    stats = hase_serve_stats()
    status = load().hase_serve(arr, len(reqs), C.byref(cfg), res, C.byref(stats))
    if status != HASE_OK:
        raise HaseError(status, "hase_serve failed")
    out = [{k: getattr(res[i], k) for k, _ in hase_request_result._fields_} for i in range(len(reqs))]
    return out, {k: getattr(stats, k) for k, _ in hase_serve_stats._fields_}


class Server:
    """A rollout server (hase_server_*): submit from any thread, poll by id."""

    def __init__(self, budget_bytes, n_streams=16, max_inflight=4096, queue_capacity=65536, max_batch_envs=0,
                 max_batch=0):
        cfg = hase_server_config(budget_bytes=int(budget_bytes), n_streams=n_streams, max_inflight=max_inflight,
                                 queue_capacity=queue_capacity, max_batch_envs=max_batch_envs, max_batch=max_batch)
        self.s = C.c_void_p()
        status = load().hase_server_create(C.byref(cfg), C.byref(self.s))
        if status != HASE_OK:
            raise HaseError(status, "hase_server_create failed")

    def submit(self, req):
        """Queue one request dict; returns its id (HaseError: HASE_EBUSY, HASE_ESTATE, HASE_EINVAL)."""
        rid = C.c_uint64()
        status = load().hase_server_submit(self.s, C.byref(_requests([dict(req, arrival=0.0)])[0]), C.byref(rid))
        if status != HASE_OK:
            raise HaseError(status, "hase_server_submit failed")
        return rid.value

    def poll(self, rid, timeout_s=0.0):
        """The result dict of request rid, or None when it has not finished within timeout_s."""
        res = hase_request_result()
        status = load().hase_server_poll(self.s, rid, float(timeout_s), C.byref(res))
        if status == HASE_ETIMEOUT:
            return None
        if status != HASE_OK:
            raise HaseError(status, "hase_server_poll failed")
        return {k: getattr(res, k) for k, _ in hase_request_result._fields_}

    def stats(self):
        st = hase_serve_stats()
        load().hase_server_stats(self.s, C.byref(st))
        return {k: getattr(st, k) for k, _ in hase_serve_stats._fields_}

    def shutdown(self):
        status = load().hase_server_shutdown(self.s)
        if status != HASE_OK:
            raise HaseError(status, "hase_server_shutdown failed")

    def close(self):
        if self.s:
            load().hase_server_destroy(self.s)
            self.s = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hase_digest_range(h, first_step, n_steps, env_first, env_count, out_ptr, agent_rew_ptr=None, stream=None):
    """hase_digest of steps [first_step, first_step + n_steps) of an env range."""
    _check(load().hase_digest_range(h, C.c_uint64(first_step), n_steps, env_first, env_count, C.c_void_p(out_ptr),
                                    C.c_void_p(agent_rew_ptr or 0), _stream(stream)), h)


def hase_digest_noalloc(h, n_steps, out_ptr, agent_rew_ptr=None, stream=None):
    """hase_digest with the partial sums in the library's fixed scratch."""
    _check(load().hase_digest_noalloc(h, n_steps, C.c_void_p(out_ptr), C.c_void_p(agent_rew_ptr or 0),
                                      _stream(stream)), h)


def hase_obs_ptr(h):
    a, b = C.c_void_p(), C.c_void_p()
    _check(load().hase_obs_ptr(h, C.byref(a), C.byref(b)), h)
    return a.value, b.value


def hase_reward_ptr(h):
    a = C.c_void_p()
    _check(load().hase_reward_ptr(h, C.byref(a)), h)
    return a.value


def hase_done_ptr(h):
    a = C.c_void_p()
    _check(load().hase_done_ptr(h, C.byref(a)), h)
    return a.value


def hase_actions_ptr(h):
    a = C.c_void_p()
    _check(load().hase_actions_ptr(h, C.byref(a)), h)
    return a.value


def hase_central_ptr(h):
    a = C.c_void_p()
    _check(load().hase_central_ptr(h, C.byref(a)), h)
    return a.value


def hase_fog_ptr(h):
    a = C.c_void_p()
    _check(load().hase_fog_ptr(h, C.byref(a)), h)
    return a.value


def hase_state_ptr(h):
    """(cells, ep_t) device pointers of the true-state rings, or (None, None)."""
    a, b = C.c_void_p(), C.c_void_p()
    _check(load().hase_state_ptr(h, C.byref(a), C.byref(b)), h)
    return a.value, b.value


def hase_layout_get(h):
    lay = hase_layout()
    _check(load().hase_layout_get(h, C.byref(lay)), h)
    n = lay.n_envs + 1
    return {
        "n_envs": lay.n_envs,
        "ring_steps": lay.ring_steps,
        "agents": lay.agents,
        "obs_words": lay.obs_words,
        "unp_bytes": lay.unp_bytes,
        "agent_off": np.ctypeslib.as_array(lay.agent_off, shape=(n,)).copy(),
        "obs_off": np.ctypeslib.as_array(lay.obs_off, shape=(n,)).copy(),
        "unp_off": np.ctypeslib.as_array(lay.unp_off, shape=(n,)).copy(),
        "central_words": lay.central_words,
        "central_off": np.ctypeslib.as_array(lay.central_off, shape=(n,)).copy(),
        "fog_words": lay.fog_words,
        "fog_off": np.ctypeslib.as_array(lay.fog_off, shape=(n,)).copy(),
    }


def hase_step_count(h):
    t = C.c_uint64()
    _check(load().hase_step_count(h, C.byref(t)), h)
    return t.value


def hase_get_state(h, stream=None):
    n = C.c_size_t()
    _check(load().hase_get_state(h, None, C.byref(n), _stream(stream)), h)
    buf = (C.c_uint8 * n.value)()
    _check(load().hase_get_state(h, buf, C.byref(n), _stream(stream)), h)
    return bytes(buf)


def hase_set_state(h, blob, stream=None):
    buf = (C.c_uint8 * len(blob)).from_buffer_copy(blob)
    _check(load().hase_set_state(h, buf, len(blob), _stream(stream)), h)


def hase_get_world(h, e, side, n_agents):
    grid = np.zeros(side * side, np.uint8)
    st = np.zeros(2 * n_agents, np.int32)
    _check(load().hase_get_world(h, e, grid.ctypes.data_as(C.c_void_p), st.ctypes.data_as(C.c_void_p)), h)
    return grid.reshape(side, side), st.reshape(n_agents, 2)


def hase_sync(h):
    _check(load().hase_sync(h), h)


def hase_launch_info(h):
    a, b, c, d = C.c_uint32(), C.c_uint32(), C.c_uint32(), C.c_uint32()
    _check(load().hase_launch_info(h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)), h)
    return {"ctas": a.value, "threads": b.value, "smem": c.value, "steps_per_launch": d.value}


def hase_destroy(h):
    if h:
        load().hase_destroy(h)


# ---------------------------------------------------------------------------
# Zero-copy torch views of device buffers.
# ---------------------------------------------------------------------------
class _DeviceArray:
    def __init__(self, ptr, shape, typestr, owner):
        self.__cuda_array_interface__ = {
            "shape": tuple(int(s) for s in shape),
            "typestr": typestr,
            "data": (int(ptr), False),
            "version": 2,
            "strides": None,
        }
        self._owner = owner


def device_view(ptr, shape, dtype, owner=None):
    """torch tensor aliasing device memory at ptr (no copy)."""
    import torch

    typestr = {"u8": "|u1", "i16": "<i2", "i32": "<i4", "i64": "<i8"}[dtype]
    if int(np.prod(shape)) == 0:
        tdt = {"u8": torch.uint8, "i16": torch.int16, "i32": torch.int32, "i64": torch.int64}[dtype]
        return torch.empty(shape, dtype=tdt, device="cuda")
    return torch.as_tensor(_DeviceArray(ptr, shape, typestr, owner), device="cuda")


class Engine:
    """One handle: create, step, and zero-copy torch views of the rings."""

    def __init__(self, n_envs, seed, descs, ring_steps, flags=0, env_id_base=0, stream=None,
                 step_form="auto", **tuning):
        flags |= STEP_FORMS[step_form]  # auto: the engine's choice of step kernel form
        self.cfg = make_config(n_envs, seed, descs, ring_steps, flags, env_id_base, **tuning)
        self.stream = stream
        self.h = hase_create(self.cfg, stream)
        self.layout = hase_layout_get(self.h)
        self.n_envs = n_envs
        self.ring = ring_steps
        obs, unp = hase_obs_ptr(self.h)
        L = self.layout
        self.obs = device_view(obs, (ring_steps, L["obs_words"]), "i64", self)  # uint64 bits
        self.reward = device_view(hase_reward_ptr(self.h), (ring_steps, L["agents"]), "i32", self)
        self.done = device_view(hase_done_ptr(self.h), (ring_steps, n_envs), "u8", self)
        act = hase_actions_ptr(self.h)
        self.actions = device_view(act, (ring_steps, L["agents"]), "u8", self) if act else None
        self.unpacked = device_view(unp, (ring_steps, L["unp_bytes"]), "u8", self) if unp else None
        cen = hase_central_ptr(self.h)
        self.central = device_view(cen, (ring_steps, L["central_words"]), "i64", self) if cen else None
        # true state: cells x | y << 6 (<= 4095) and episode clocks (< 2^31)
        cells, ept = hase_state_ptr(self.h)
        self.cells = device_view(cells, (ring_steps, L["agents"]), "i16", self) if cells else None
        self.ep_t = device_view(ept, (ring_steps, n_envs), "i32", self) if ept else None
        fog = hase_fog_ptr(self.h)
        self.fog = device_view(fog, (ring_steps, L["fog_words"]), "i64", self) if fog else None

    def slot(self, t):
        """Ring slot of global step t (t = -1: the observation after create/reset)."""
        return t % self.ring

    def step(self, n_steps=1):
        hase_step(self.h, n_steps, self.stream)

    def digest(self, n_steps, per_agent=False):
        """(digest, episodes, reward_sum, gen_error[, per-agent sums]) of the
        last n_steps steps, reduced on the device."""
        import numpy as np
        import torch

        out = torch.zeros(4, dtype=torch.int64, device="cuda")
        ag = torch.zeros(self.layout["agents"], dtype=torch.int64, device="cuda") if per_agent else None
        hase_digest(self.h, n_steps, out.data_ptr(), ag.data_ptr() if ag is not None else None, self.stream)
        torch.cuda.synchronize()
        v = out.cpu().numpy().view(np.uint64)
        res = (int(v[0]), int(v[1]), int(np.int64(v[2])), int(v[3] & 0xffffffff))
        return res + ((ag.cpu().numpy(),) if per_agent else ())

    def step_graph(self, n_steps=1):
        """The same steps replayed as one CUDA graph (captured on first use)."""
        hase_step_graph(self.h, n_steps, self.stream)

    def reset(self):
        hase_reset(self.h, self.stream)

    @property
    def t(self):
        return hase_step_count(self.h)

    def sync(self):
        hase_sync(self.h)

    def get_state(self):
        return hase_get_state(self.h, self.stream)

    def set_state(self, blob):
        hase_set_state(self.h, blob, self.stream)

    def launch_info(self):
        return hase_launch_info(self.h)

    def close(self):
        if getattr(self, "h", None):
            try:
                import torch

                torch.cuda.synchronize()
            except Exception:
                pass
            hase_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
