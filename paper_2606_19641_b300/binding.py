"""Thin Python binding of the C ABI in include/gigapixel.h (argument marshalling only).

Every computation runs in the CUDA library ``libgigapixel.so`` built in-tree from
``csrc/``; PyTorch only provides device memory and streams.  There is no CPU fallback:
if the library cannot be loaded, the first call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgigapixel.so")

GP_OK, GP_EINVAL, GP_ENOMEM, GP_ECUDA, GP_ELIMIT, GP_EDEVICE, GP_ESTATE = 0, -1, -2, -3, -4, -5, -6
KEY_F32, KEY_F16 = 0, 1
OUT_CLASS_U8, OUT_ONEHOT_BF16, OUT_RGB_U8 = 0, 1, 2
CLASS_SIGNAL = 4
SIGNAL_RED, SIGNAL_AMBER, SIGNAL_GREEN, SIGNAL_OFF = 0, 1, 2, 3
FLAG_COLLIDED, FLAG_OFFROAD, FLAG_HALTED, FLAG_DONE, FLAG_RED_LIGHT = 1, 2, 4, 8, 16
DEV_NONFINITE_STATE, DEV_CLIP_OVERFLOW, DEV_PIPELINE_TIMEOUT, DEV_INJECTED = 1, 2, 4, 1 << 31
MAX_CAMS = 8
DYN_DIRECT, DYN_JERK = 0, 1
STAT_NAMES = ("items", "clusters", "boxes", "signals", "quads", "tris_kept", "tris_clipped",
              "tris_from_clip", "batches", "row_items", "fragments")
EGO_DIM = 9
# App. A's discrete action set for DYN_JERK: (longitudinal, lateral) jerk in m/s^3.
JERK_ACTIONS = tuple((jl, jt) for jl in (-15.0, -4.0, 0.0, 4.0) for jt in (-4.0, 0.0, 4.0))

TRI_DTYPE = np.dtype([("X", "<i4", (3,)), ("Y", "<i4", (3,)), ("d", "<f4", (3,)),
                      ("prim", "<u4"), ("sub", "<u4")])

EXPORTED = ("gp_default_config", "gp_create_worlds", "gp_destroy", "gp_step", "gp_render", "gp_trace",
            "gp_step_render", "gp_step_render_host", "gp_step_trace", "gp_step_world", "gp_render_world", "gp_get_state",
            "gp_set_state", "gp_get_info", "gp_get_status", "gp_clear_status",
            "gp_get_rewards", "gp_set_reward_weights", "gp_observe_vec",
            "gp_get_dynamics", "gp_set_dynamics", "gp_set_signal_states", "gp_reset_worlds",
            "gp_get_render_stats", "gp_get_conditioning", "gp_get_reward_weights",
            "gp_debug_inject_status", "gp_debug_stall_pipeline", "gp_debug_dump_tris",
            "gp_debug_dump_tris_noalloc",
            "gp_last_error")
NOALLOC_MAX_TRIS = 16384


class WorldDesc(ctypes.Structure):
    _fields_ = [("n_worlds", ctypes.c_int32),
                ("box_off", ctypes.POINTER(ctypes.c_int32)),
                ("agent_count", ctypes.POINTER(ctypes.c_int32)),
                ("boxes", ctypes.POINTER(ctypes.c_float)),
                ("road_off", ctypes.POINTER(ctypes.c_int32)),
                ("road", ctypes.POINTER(ctypes.c_float)),
                ("line_off", ctypes.POINTER(ctypes.c_int32)),
                ("line", ctypes.POINTER(ctypes.c_float)),
                ("signal_off", ctypes.POINTER(ctypes.c_int32)),
                ("signal", ctypes.POINTER(ctypes.c_float)),
                ("signal_state", ctypes.POINTER(ctypes.c_uint8))]


class Config(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("n_cams", ctypes.c_int32),
                ("cam_yaw", ctypes.c_float * MAX_CAMS), ("hfov", ctypes.c_float),
                ("cam_height", ctypes.c_float), ("near_plane", ctypes.c_float),
                ("lane_line_z", ctypes.c_float), ("dt", ctypes.c_float), ("v_max", ctypes.c_float),
                ("key_precision", ctypes.c_int32), ("output", ctypes.c_int32),
                ("norm_mean", ctypes.c_float * 4), ("norm_std", ctypes.c_float * 4),
                ("autotune", ctypes.c_int32), ("band_rows", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("tri_capacity", ctypes.c_int32),
                ("producer_warps", ctypes.c_int32),
                ("light_dir", ctypes.c_float * 3), ("ambient", ctypes.c_float),
                ("colour", (ctypes.c_float * 3) * 4),
                ("rewards", ctypes.c_int32), ("lane_width", ctypes.c_float),
                ("v_limit", ctypes.c_float), ("dynamics", ctypes.c_int32),
                ("stats", ctypes.c_int32), ("episode_steps", ctypes.c_int32),
                ("reward_conditioning", ctypes.c_int32), ("conditioning_seed", ctypes.c_uint32),
                ("signal_colour", (ctypes.c_float * 3) * 4)]


class Info(ctypes.Structure):
    _fields_ = [("n_worlds", ctypes.c_int32), ("n_agents", ctypes.c_int32),
                ("n_boxes", ctypes.c_int32), ("n_views", ctypes.c_int32),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("n_cams", ctypes.c_int32),
                ("key_precision", ctypes.c_int32), ("output", ctypes.c_int32),
                ("out_bytes", ctypes.c_int64), ("depth_bytes", ctypes.c_int64),
                ("band_rows", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("tri_capacity", ctypes.c_int32), ("blocks", ctypes.c_int32),
                ("producer_warps", ctypes.c_int32)]


class GigapixelError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("gigapixel status %d: %s" % (status, msg))
        self.status = status


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library; raises if it is missing (there is no fallback)."""
    if not os.path.exists(path):
        raise ImportError("libgigapixel.so not built: run paper_2606_19641_b300/build.py")
    lib = ctypes.CDLL(path)
    vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    sigs = {
        "gp_default_config": [ctypes.POINTER(Config)],
        "gp_create_worlds": [ctypes.POINTER(WorldDesc), ctypes.POINTER(Config), ctypes.c_int,
                             ctypes.POINTER(vp)],
        "gp_destroy": [vp],
        "gp_step": [vp, vp, vp],
        "gp_render": [vp, vp, vp, vp],
        "gp_step_render": [vp, vp, vp, vp, vp],
        "gp_step_trace": [vp, vp, vp, vp, vp],
        "gp_step_render_host": [vp, vp, vp, vp, vp, vp, vp],
        "gp_step_world": [vp, i32, vp, vp],
        "gp_render_world": [vp, i32, vp, vp, vp],
        "gp_get_state": [vp, vp, vp, ctypes.c_int, vp],
        "gp_set_state": [vp, vp, vp, ctypes.c_int, vp],
        "gp_get_info": [vp, ctypes.POINTER(Info)],
        "gp_get_status": [vp, ctypes.POINTER(u32)],
        "gp_clear_status": [vp],
        "gp_debug_inject_status": [vp, u32],
        "gp_get_rewards": [vp, vp, vp, i32, vp],
        "gp_trace": [vp, vp, vp, vp],
        "gp_observe_vec": [vp, vp, vp, vp, vp],
        "gp_set_reward_weights": [vp, vp, i32, vp],
        "gp_get_dynamics": [vp, vp, i32, vp],
        "gp_set_signal_states": [vp, vp, i32, vp],
        "gp_reset_worlds": [vp, vp, i32, vp],
        "gp_get_render_stats": [vp, vp, i32],
        "gp_get_conditioning": [vp, vp, i32, vp],
        "gp_get_reward_weights": [vp, vp, i32, vp],
        "gp_set_dynamics": [vp, vp, i32, vp],
        "gp_debug_stall_pipeline": [vp, vp, vp, i64, vp],
        "gp_debug_dump_tris": [vp, i32, vp, vp, vp, i64, ctypes.POINTER(i64), vp],
        "gp_debug_dump_tris_noalloc": [vp, i32, vp, vp, vp, i64, ctypes.POINTER(i64), vp],
    }
    for name, args in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.gp_last_error.argtypes = []
    lib.gp_last_error.restype = ctypes.c_char_p
    return lib


_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def check(status: int) -> None:
    if status != GP_OK:
        raise GigapixelError(status, lib().gp_last_error().decode())


def default_config(**kw) -> Config:
    c = Config()
    check(lib().gp_default_config(ctypes.byref(c)))
    for k, v in kw.items():
        if k == "cam_yaw":
            vals = list(v)
            c.n_cams = len(vals)
            for i, y in enumerate(vals):
                c.cam_yaw[i] = y
        elif k in ("norm_mean", "norm_std", "light_dir"):
            arr = getattr(c, k)
            for i, y in enumerate(v):
                arr[i] = y
        elif k in ("colour", "signal_colour"):
            arr = getattr(c, k)
            for i, row in enumerate(v):
                for j, y in enumerate(row):
                    arr[i][j] = y
        else:
            setattr(c, k, v)
    return c


def _ptr(t) -> int:
    """Device/host address of a torch tensor or numpy array (None -> 0)."""
    if t is None:
        return 0
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Simulator:
    """A batch of worlds on one GPU (one gp_handle)."""

    def __init__(self, worlds, config: Config, device: int = 0):
        keep = []
        desc = WorldDesc()
        desc.n_worlds = worlds.n_worlds

        def arr(a, dtype, ct):
            a = np.ascontiguousarray(a, dtype=dtype)
            keep.append(a)
            return a.ctypes.data_as(ctypes.POINTER(ct))
        desc.box_off = arr(worlds.box_off, np.int32, ctypes.c_int32)
        desc.agent_count = arr(worlds.agent_count, np.int32, ctypes.c_int32)
        desc.boxes = arr(worlds.boxes, np.float32, ctypes.c_float)
        desc.road_off = arr(worlds.road_off, np.int32, ctypes.c_int32)
        desc.road = arr(worlds.road, np.float32, ctypes.c_float)
        desc.line_off = arr(worlds.line_off, np.int32, ctypes.c_int32)
        desc.line = arr(worlds.line, np.float32, ctypes.c_float)
        sig_off = getattr(worlds, "signal_off", None)
        if sig_off is not None:
            desc.signal_off = arr(sig_off, np.int32, ctypes.c_int32)
            desc.signal = arr(worlds.signal, np.float32, ctypes.c_float)
            desc.signal_state = arr(worlds.signal_state, np.uint8, ctypes.c_uint8)
        self.n_signals = 0 if sig_off is None else int(sig_off[-1])
        self.config = config
        self.device = device
        self._h = None
        h = ctypes.c_void_p()
        check(lib().gp_create_worlds(ctypes.byref(desc), ctypes.byref(config), device,
                                     ctypes.byref(h)))
        self._h = h
        self.info = Info()
        check(lib().gp_get_info(self._h, ctypes.byref(self.info)))

    def close(self) -> None:
        if self._h is not None and self._h.value:
            lib().gp_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_agents(self) -> int:
        return self.info.n_agents

    @property
    def n_views(self) -> int:
        return self.info.n_views

    def alloc_outputs(self, depth: bool = True):
        """Output tensors on the device in the layout gp_render writes."""
        import torch
        i = self.info
        dev = torch.device("cuda", self.device)
        if i.output == OUT_CLASS_U8:
            out = torch.empty((i.n_views, i.height, i.width), dtype=torch.uint8, device=dev)
        elif i.output == OUT_RGB_U8:
            out = torch.empty((i.n_views, 3, i.height, i.width), dtype=torch.uint8, device=dev)
        else:
            out = torch.empty((i.n_views, 4, i.height, i.width), dtype=torch.bfloat16, device=dev)
        d = None
        if depth:
            dt = torch.float32 if i.key_precision == KEY_F32 else torch.float16
            d = torch.empty((i.n_views, i.height, i.width), dtype=dt, device=dev)
        return out, d

    def _dev(self, t, dtype, numel: int, name: str) -> int:
        """Address of a device tensor the library will read or write, after checking that it
        is a contiguous tensor on this simulator's GPU with the dtype and element count of the
        layout the call expects (a host array or a short buffer would otherwise reach a
        kernel).  None passes through as a null pointer, which the library checks itself."""
        import torch
        if t is None:
            return 0
        if not isinstance(t, torch.Tensor):
            raise GigapixelError(GP_EINVAL, "%s: expected a torch tensor on cuda:%d, got %s"
                                 % (name, self.device, type(t).__name__))
        if t.device.type != "cuda" or t.device.index != self.device:
            raise GigapixelError(GP_EINVAL, "%s: tensor on %s, the simulator is on cuda:%d"
                                 % (name, t.device, self.device))
        if t.dtype != dtype:
            raise GigapixelError(GP_EINVAL, "%s: dtype %s, expected %s" % (name, t.dtype, dtype))
        if not t.is_contiguous():
            raise GigapixelError(GP_EINVAL, "%s: tensor is not contiguous" % name)
        if t.numel() != numel:
            raise GigapixelError(GP_EINVAL, "%s: %d elements (shape %s), expected %d"
                                 % (name, t.numel(), tuple(t.shape), numel))
        return t.data_ptr()

    def _host(self, t, dtype, numel: int, name: str) -> int:
        """Address of a pinned host tensor the library will copy from or to, after checking
        its dtype, element count and contiguity (the library refuses pageable memory)."""
        import torch
        if t is None:
            return 0
        if not isinstance(t, torch.Tensor) or t.device.type != "cpu":
            raise GigapixelError(GP_EINVAL, "%s: expected a pinned CPU tensor" % name)
        if not t.is_pinned():
            raise GigapixelError(GP_EINVAL, "%s: CPU tensor is not pinned" % name)
        if t.dtype != dtype:
            raise GigapixelError(GP_EINVAL, "%s: dtype %s, expected %s" % (name, t.dtype, dtype))
        if not t.is_contiguous():
            raise GigapixelError(GP_EINVAL, "%s: tensor is not contiguous" % name)
        if t.numel() != numel:
            raise GigapixelError(GP_EINVAL, "%s: %d elements (shape %s), expected %d"
                                 % (name, t.numel(), tuple(t.shape), numel))
        return t.data_ptr()

    def _actions(self, actions) -> int:
        import torch
        return self._dev(actions, torch.float32, 2 * self.n_agents, "actions")

    def _images(self, out, depth):
        """(out, depth) addresses checked against the configured output layout."""
        import torch
        i = self.info
        px = i.n_views * i.height * i.width
        if i.output == OUT_CLASS_U8:
            od, on = torch.uint8, px
        elif i.output == OUT_RGB_U8:
            od, on = torch.uint8, 3 * px
        else:
            od, on = torch.bfloat16, 4 * px
        dd = torch.float32 if i.key_precision == KEY_F32 else torch.float16
        return self._dev(out, od, on, "out"), self._dev(depth, dd, px, "depth")

    def step(self, actions, stream=None) -> None:
        check(lib().gp_step(self._h, self._actions(actions), _stream(stream)))

    def render(self, out, depth=None, stream=None) -> None:
        o, d = self._images(out, depth)
        check(lib().gp_render(self._h, o, d, _stream(stream)))

    def step_render(self, actions, out, depth=None, stream=None) -> None:
        a = self._actions(actions)
        o, d = self._images(out, depth)
        check(lib().gp_step_render(self._h, a, o, d, _stream(stream)))

    def step_render_host(self, actions, out, depth=None, state=None, flags=None,
                         stream=None) -> None:
        """One closed-loop step from pinned host actions to pinned host state (asynchronous:
        synchronise `stream` before reading state/flags or refilling actions)."""
        import torch
        a = self._host(actions, torch.float32, 2 * self.n_agents, "actions")
        o, d = self._images(out, depth)
        sp = self._host(state, torch.float32, 4 * self.n_agents, "state")
        fp = self._host(flags, torch.uint8, self.n_agents, "flags")
        check(lib().gp_step_render_host(self._h, a, o, d, sp, fp, _stream(stream)))

    def step_trace(self, actions, out, depth=None, stream=None) -> None:
        """One step then the ray-traced render, replayed from a CUDA graph."""
        a = self._actions(actions)
        o, d = self._images(out, depth)
        check(lib().gp_step_trace(self._h, a, o, d, _stream(stream)))

    def step_world(self, world: int, actions, stream=None) -> None:
        check(lib().gp_step_world(self._h, world, self._actions(actions), _stream(stream)))

    def render_world(self, world: int, out, depth=None, stream=None) -> None:
        o, d = self._images(out, depth)
        check(lib().gp_render_world(self._h, world, o, d, _stream(stream)))

    def get_state(self):
        """(state float32 [n_agents, 4] = x, y, yaw, v; flags uint8 [n_agents]) on the host."""
        st = np.zeros((self.n_agents, 4), np.float32)
        fl = np.zeros(self.n_agents, np.uint8)
        check(lib().gp_get_state(self._h, _ptr(st), _ptr(fl), 1, _stream(None)))
        return st, fl

    def get_state_device(self, state, flags, stream=None) -> None:
        check(lib().gp_get_state(self._h, _ptr(state), _ptr(flags), 0, _stream(stream)))

    def set_state(self, state, flags) -> None:
        st = np.ascontiguousarray(state, np.float32)
        fl = np.ascontiguousarray(flags, np.uint8)
        check(lib().gp_set_state(self._h, _ptr(st), _ptr(fl), 1, _stream(None)))

    def status(self) -> int:
        bits = ctypes.c_uint32()
        check(lib().gp_get_status(self._h, ctypes.byref(bits)))
        return bits.value

    def clear_status(self) -> None:
        check(lib().gp_clear_status(self._h))

    def inject_status(self, bits: int) -> None:
        check(lib().gp_debug_inject_status(self._h, bits))

    def trace(self, out, depth=None, stream=None) -> None:
        """Ray-traced render of every camera into the same tensors as render()."""
        o, d = self._images(out, depth)
        check(lib().gp_trace(self._h, o, d, _stream(stream)))

    def observe_vec(self, stream=None, out=None):
        """(agents [n_agents, 16, 8], roads [n_agents, 32, 8], signals [n_agents, 4, 8])
        float32 O_vec on the device (into `out`, a tuple of such tensors, if given)."""
        import torch
        if out is None:
            dev = torch.device("cuda", self.device)
            out = tuple(torch.empty((self.n_agents, k, 8), dtype=torch.float32, device=dev)
                        for k in (16, 32, 4))
        a, r, s = out
        n = self.n_agents
        pa = self._dev(a, torch.float32, n * 16 * 8, "agents")
        pr = self._dev(r, torch.float32, n * 32 * 8, "roads")
        ps = self._dev(s, torch.float32, n * 4 * 8, "signals")
        check(lib().gp_observe_vec(self._h, pa, pr, ps, _stream(stream)))
        return a, r, s

    def reward_weights(self) -> np.ndarray:
        """Reward weights in use, float32 [n_agents, 10] (host copy)."""
        w = np.zeros((self.n_agents, 10), np.float32)
        check(lib().gp_get_reward_weights(self._h, _ptr(w), 1, _stream(None)))
        return w

    def conditioning(self) -> np.ndarray:
        """Reward conditioning vectors float32 [n_agents, 12] in [-1, 1] (host copy)."""
        c = np.zeros((self.n_agents, 12), np.float32)
        check(lib().gp_get_conditioning(self._h, _ptr(c), 1, _stream(None)))
        return c

    def render_stats(self, reset: bool = False) -> dict:
        """GP_STAT_* render counters since create or the last reset (config stats = 1)."""
        c = np.zeros(16, np.uint64)
        check(lib().gp_get_render_stats(self._h, _ptr(c), int(reset)))
        return {k: int(c[i]) for i, k in enumerate(STAT_NAMES)}

    def reset_worlds(self, mask=None, stream=None) -> None:
        """Return the agents of the worlds selected by mask (uint8/bool [n_worlds], host
        array or device tensor; None = all) to their initial state."""
        if mask is None:
            check(lib().gp_reset_worlds(self._h, None, 1, _stream(stream)))
        elif isinstance(mask, np.ndarray):
            m = np.ascontiguousarray(mask, np.uint8)
            assert m.shape == (self.info.n_worlds,)
            check(lib().gp_reset_worlds(self._h, _ptr(m), 1, _stream(stream)))
        else:
            assert tuple(mask.shape) == (self.info.n_worlds,) and mask.is_contiguous()
            assert mask.element_size() == 1, "mask must be uint8 or bool"
            check(lib().gp_reset_worlds(self._h, _ptr(mask), 0, _stream(stream)))

    def set_signal_states(self, states) -> None:
        """Traffic-signal states uint8 [n_signals] (0 red, 1 amber, 2 green, 3 off): host
        array, or a device tensor."""
        if isinstance(states, np.ndarray):
            s = np.ascontiguousarray(states, np.uint8)
            assert s.shape == (self.n_signals,)
            check(lib().gp_set_signal_states(self._h, _ptr(s), 1, _stream(None)))
        else:
            assert tuple(states.shape) == (self.n_signals,) and states.is_contiguous()
            check(lib().gp_set_signal_states(self._h, _ptr(states), 0, _stream(None)))

    def get_dynamics(self) -> np.ndarray:
        """Jerk dynamics' actuator state float32 [n_agents, 3] = a_lon, a_lat, steer (host)."""
        d = np.zeros((self.n_agents, 3), np.float32)
        check(lib().gp_get_dynamics(self._h, _ptr(d), 1, _stream(None)))
        return d

    def set_dynamics(self, dyn) -> None:
        d = np.ascontiguousarray(dyn, np.float32)
        assert d.shape == (self.n_agents, 3)
        check(lib().gp_set_dynamics(self._h, _ptr(d), 1, _stream(None)))

    def rewards(self, stream=None):
        """(reward [n_agents], ego state [n_agents, EGO_DIM]) of the last step, float32 on
        the device (the handle must have been created with rewards = 1)."""
        import torch
        dev = torch.device("cuda", self.device)
        r = torch.empty((self.n_agents,), dtype=torch.float32, device=dev)
        e = torch.empty((self.n_agents, EGO_DIM), dtype=torch.float32, device=dev)
        check(lib().gp_get_rewards(self._h, _ptr(r), _ptr(e), 0, _stream(stream)))
        return r, e

    def set_reward_weights(self, weights) -> None:
        """Per-agent reward weights [n_agents, 10] (host array or device tensor)."""
        if isinstance(weights, np.ndarray):
            w = np.ascontiguousarray(weights, np.float32)
            assert w.shape == (self.n_agents, 10)
            check(lib().gp_set_reward_weights(self._h, w.ctypes.data, 1, _stream(None)))
        else:
            assert tuple(weights.shape) == (self.n_agents, 10) and weights.is_contiguous()
            check(lib().gp_set_reward_weights(self._h, _ptr(weights), 0, _stream(None)))

    def debug_stall_pipeline(self, out, depth=None, wait_ns: int = 50_000_000) -> None:
        """Run the pipelined render kernel with producers that publish nothing (its bounded
        handoff wait runs out and sets DEV_PIPELINE_TIMEOUT)."""
        check(lib().gp_debug_stall_pipeline(self._h, _ptr(out), _ptr(depth), wait_ns,
                                            _stream(None)))

    def dump_tris(self, view: int, out, depth=None, cap: int = 1 << 20) -> np.ndarray:
        """Render all views and return the snapped triangles view `view` rasterised."""
        buf = np.zeros(cap, TRI_DTYPE)
        n = ctypes.c_int64()
        check(lib().gp_debug_dump_tris(self._h, view, _ptr(out), _ptr(depth), buf.ctypes.data,
                                       cap, ctypes.byref(n), _stream(None)))
        assert n.value <= cap, "dump capacity exceeded"
        return buf[:n.value].copy()
