"""ORACLE -- test infrastructure only.

A plain, slow, CPU-only FP64 statement of the batched step-and-render (kinematic bicycle,
OBB collision, off-road, halt; per-camera transform, near/guard clipping, projection,
1/16-pixel snapping, and the integer + FP32 raster rule).  Only ``tests/``, the smoke
check and the benchmark's CPU-baseline leg may import this package; the product path
(the CUDA library and its binding) never does, and the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, compiled with -ffp-contract=off); this
module only marshals numpy arrays.  Every function cites the passage it follows in the
C source.  Parity pins: ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_oracle.so")

COLLIDED, OFFROAD, HALTED = 1, 2, 4

TRI_DTYPE = np.dtype([("X", "<i4", (3,)), ("Y", "<i4", (3,)), ("d", "<f4", (3,)),
                      ("prim", "<u4"), ("sub", "<u4")])


class OrCam(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("hfov", ctypes.c_double), ("cam_height", ctypes.c_double),
                ("near", ctypes.c_double), ("line_z", ctypes.c_double),
                ("guard", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, FP64 geometry, no fused multiply-adds but fmaf).

    ``ORACLE_SO`` in the environment names a prebuilt library to load instead (the
    mutation test uses it to load deliberately broken copies).
    """
    if os.environ.get("ORACLE_SO"):
        return os.environ["ORACLE_SO"]
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib_handle = None
P = ctypes.POINTER
c_f64p, c_f32p, c_u8p = P(ctypes.c_double), P(ctypes.c_float), P(ctypes.c_uint8)
c_u16p, c_u64p = P(ctypes.c_uint16), P(ctypes.c_uint64)


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        lib.or_bicycle.argtypes = [c_f64p, c_f64p, c_f64p, c_f64p] + [ctypes.c_double] * 5
        lib.or_jerk_bicycle.argtypes = [c_f64p, c_f64p, c_f64p, c_f64p] + [ctypes.c_double] * 3 + \
            [c_f64p, ctypes.c_double, ctypes.c_double]
        lib.or_step_world_jerk.argtypes = [ctypes.c_int32, ctypes.c_int32, c_f64p, c_f64p, c_u8p,
                                           c_f32p, ctypes.c_int32, c_f32p, ctypes.c_int32,
                                           c_f64p, c_u8p, ctypes.c_double, ctypes.c_double,
                                           c_f64p]
        lib.or_obb_overlap.argtypes = [c_f64p, c_f64p]
        lib.or_obb_overlap.restype = ctypes.c_int
        lib.or_point_in_quad.argtypes = [ctypes.c_double, ctypes.c_double, c_f32p]
        lib.or_point_in_quad.restype = ctypes.c_int
        lib.or_step_world.argtypes = [ctypes.c_int32, ctypes.c_int32, c_f64p, c_f64p, c_u8p,
                                      c_f32p, ctypes.c_int32, c_f32p, ctypes.c_int32, c_f64p,
                                      c_u8p, ctypes.c_double, ctypes.c_double]
        lib.or_camera_tris.argtypes = [P(OrCam), ctypes.c_int32, c_f64p, ctypes.c_int32,
                                       ctypes.c_int32, c_f32p, ctypes.c_int32, c_f32p,
                                       ctypes.c_int32, c_f64p,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_void_p, ctypes.c_int64]
        lib.or_camera_tris.restype = ctypes.c_int64
        for fn in (lib.or_raster, lib.or_raster_bruteforce):
            fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                           ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                           c_u64p, c_u8p, c_f32p, c_u16p]
        lib.or_f32_to_f16.argtypes = [ctypes.c_float]
        lib.or_f32_to_f16.restype = ctypes.c_uint16
        lib.or_f32_to_bf16.argtypes = [ctypes.c_float]
        lib.or_f32_to_bf16.restype = ctypes.c_uint16
        lib.or_onehot_bf16.argtypes = [c_u8p, ctypes.c_int64, c_f32p, c_f32p, c_u16p]
        lib.or_trace_view.argtypes = [P(OrCam), ctypes.c_int32, c_f64p, ctypes.c_int32,
                                      ctypes.c_int32, c_f32p, ctypes.c_int32, c_f32p,
                                      ctypes.c_int32, c_f64p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, c_u8p, c_f32p, P(ctypes.c_uint32)]
        lib.or_observe_world.argtypes = [ctypes.c_int32, ctypes.c_int32, c_f64p, c_f64p,
                                         ctypes.c_int32, c_f32p, ctypes.c_int32, c_f32p,
                                         ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                         ctypes.c_double, c_f64p, c_f64p, c_f64p]
        lib.or_observe_signals.argtypes = [ctypes.c_int32, c_f64p, ctypes.c_int32, c_f64p, c_u8p,
                                           ctypes.c_int32, ctypes.c_double, c_f64p, c_f64p]
        lib.or_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.or_splitmix64.restype = ctypes.c_uint64
        lib.or_conditioning.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_uint32, c_f64p, c_f64p]
        lib.or_lane_frame.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int32, c_f32p,
                                      ctypes.c_double, c_f64p, c_f64p]
        lib.or_lane_frame.restype = ctypes.c_int
        lib.or_rewards_world.argtypes = [ctypes.c_int32, c_f64p, c_u8p, c_f64p, c_u8p, c_f32p,
                                         c_f64p, c_f64p, c_f64p, ctypes.c_int32, c_f32p,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, c_f64p, ctypes.c_int32, c_f64p, c_u8p,
                                         c_f64p, c_f64p]
        lib.or_shade_rgb.argtypes = [c_u64p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32,
                                     ctypes.c_uint32, ctypes.c_uint32, c_f64p, c_f64p, c_u8p,
                                     c_f64p, c_f64p, c_f64p, ctypes.c_double, c_u8p]
        _lib_handle = lib
    return _lib_handle


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------------------------------
# Dynamics
# ---------------------------------------------------------------------------------------

def bicycle(x, y, yaw, v, L, accel, steer, dt=0.1, vmax=30.0):
    """One kinematic-bicycle step (App. A "Action Space and Dynamics"); returns x, y, yaw, v."""
    cx, cy, cyaw, cv = (ctypes.c_double(float(t)) for t in (x, y, yaw, v))
    _lib().or_bicycle(ctypes.byref(cx), ctypes.byref(cy), ctypes.byref(cyaw), ctypes.byref(cv),
                      float(L), float(accel), float(steer), float(dt), float(vmax))
    return cx.value, cy.value, cyaw.value, cv.value


# The paper's discrete action set: longitudinal x lateral jerk (m/s^3).
JERK_ACTIONS = tuple((jl, jt) for jl in (-15.0, -4.0, 0.0, 4.0) for jt in (-4.0, 0.0, 4.0))


def jerk_bicycle(x, y, yaw, v, L, j_lon, j_lat, st, dt=0.1, vmax=30.0):
    """One jerk-actuated bicycle step; st = [a_lon, a_lat, steer] (updated in place);
    returns x, y, yaw, v."""
    assert st.dtype == np.float64 and st.shape == (3,)
    cx, cy, cyaw, cv = (ctypes.c_double(float(t)) for t in (x, y, yaw, v))
    _lib().or_jerk_bicycle(ctypes.byref(cx), ctypes.byref(cy), ctypes.byref(cyaw), ctypes.byref(cv),
                           float(L), float(j_lon), float(j_lat), _p(st, c_f64p), float(dt), float(vmax))
    return cx.value, cy.value, cyaw.value, cv.value


def obb_overlap(a: Sequence[float], b: Sequence[float]) -> bool:
    """Footprint interiors intersect (x, y, yaw, L, W each)."""
    aa, bb = _c(a[:5], np.float64), _c(b[:5], np.float64)
    return bool(_lib().or_obb_overlap(_p(aa, c_f64p), _p(bb, c_f64p)))


def point_in_quad(px: float, py: float, quad: Sequence[float]) -> bool:
    q = _c(quad, np.float32)
    return bool(_lib().or_point_in_quad(float(px), float(py), _p(q, c_f32p)))


def step_world(boxes6: np.ndarray, state: np.ndarray, flags: np.ndarray, actions: np.ndarray,
               road: np.ndarray, dt: float = 0.1, vmax: float = 30.0,
               jerk: Optional[np.ndarray] = None, sph=None, sph_state=None) -> None:
    """One step of one world in place (App. A dynamics + infractions + halt).

    boxes6 float64 [n_boxes, 6]; state float64 [n_agents, 4]; flags uint8 [n_agents]
    (1 collided, 2 off-road, 4 halted, 16 red-light violation); actions float32
    [n_agents, 2] (accel, steer; or j_lon, j_lat when `jerk` is given); road float32
    [n_road, 8]; jerk float64 [n_agents, 3] (a_lon, a_lat, steer), updated; sph [n_sig, 4]
    signal spheres x, y, z, r with states sph_state [n_sig] (0 red; None = all red).
    """
    assert boxes6.dtype == np.float64 and boxes6.flags.c_contiguous
    assert state.dtype == np.float64 and state.flags.c_contiguous
    assert flags.dtype == np.uint8 and flags.flags.c_contiguous
    act = _c(actions, np.float32)
    rd = _c(road, np.float32).reshape(-1, 8)
    sp = _sph(sph)
    st = _c(np.zeros(sp.shape[0]) if sph_state is None else sph_state, np.uint8)
    assert st.shape == (sp.shape[0],)
    if jerk is None:
        _lib().or_step_world(boxes6.shape[0], state.shape[0], _p(boxes6, c_f64p),
                             _p(state, c_f64p), _p(flags, c_u8p), _p(act, c_f32p), rd.shape[0],
                             _p(rd, c_f32p), sp.shape[0], _p(sp, c_f64p), _p(st, c_u8p),
                             float(dt), float(vmax))
    else:
        assert jerk.dtype == np.float64 and jerk.flags.c_contiguous
        assert jerk.shape == (state.shape[0], 3)
        _lib().or_step_world_jerk(boxes6.shape[0], state.shape[0], _p(boxes6, c_f64p),
                                  _p(state, c_f64p), _p(flags, c_u8p), _p(act, c_f32p),
                                  rd.shape[0], _p(rd, c_f32p), sp.shape[0], _p(sp, c_f64p),
                                  _p(st, c_u8p), float(dt), float(vmax), _p(jerk, c_f64p))


# ---------------------------------------------------------------------------------------
# Geometry and raster
# ---------------------------------------------------------------------------------------

@dataclasses.dataclass
class CamConfig:
    width: int
    height: int
    hfov: float = math.pi / 2
    cam_height: float = 1.5
    near: float = 0.1
    line_z: float = 0.02
    guard: float = 4.0

    def c(self) -> OrCam:
        return OrCam(self.width, self.height, self.hfov, self.cam_height, self.near,
                     self.line_z, self.guard)


def _sph(sph) -> np.ndarray:
    return _c(np.zeros((0, 4)) if sph is None else sph, np.float64).reshape(-1, 4)


def camera_tris(cam: CamConfig, boxes6: np.ndarray, ego: int, road: np.ndarray,
                line: np.ndarray, ax: float, ay: float, ayaw: float, cam_yaw: float = 0.0,
                cap: Optional[int] = None, sph=None) -> np.ndarray:
    """FP64 scene triangles of one camera after clipping, snapping and back-face culling;
    sph [n, 4] = signal spheres (x, y, z, r)."""
    b = _c(boxes6, np.float64).reshape(-1, 6)
    rd = _c(road, np.float32).reshape(-1, 8)
    ln = _c(line, np.float32).reshape(-1, 8)
    sp = _sph(sph)
    lib = _lib()
    c = cam.c()
    if cap is None:
        cap = 6 * (12 * b.shape[0] + 2 * rd.shape[0] + 2 * ln.shape[0] + 64 * sp.shape[0]) + 16
    out = np.zeros(cap, TRI_DTYPE)
    n = lib.or_camera_tris(ctypes.byref(c), b.shape[0], _p(b, c_f64p), int(ego), rd.shape[0],
                           _p(rd, c_f32p), ln.shape[0], _p(ln, c_f32p), sp.shape[0],
                           _p(sp, c_f64p), float(ax), float(ay),
                           float(ayaw), float(cam_yaw), out.ctypes.data, cap)
    assert n <= cap
    return out[:n].copy()


@dataclasses.dataclass
class Traced:
    cls: np.ndarray      # uint8 [H, W]
    depth: np.ndarray    # float32 [H, W], near / t (0 on background)
    prim: np.ndarray     # uint32 [H, W], the hit's primitive id (0xFFFFFFFF background)

    def key(self, key_f16: bool = False) -> np.ndarray:
        """Keys in the raster's layout (for shade_rgb): id half only, 0 on background."""
        k = np.zeros(self.prim.shape, np.uint64)
        hit = self.prim != 0xFFFFFFFF
        full = 0xFFFF if key_f16 else 0xFFFFFFFF
        k[hit] = (np.uint64(1) << np.uint64(40)) | (full - self.prim[hit].astype(np.uint64))
        return k


def trace_view(cam: CamConfig, boxes6: np.ndarray, ego: int, road: np.ndarray, line: np.ndarray,
               ax: float, ay: float, ayaw: float, cam_yaw: float, sph=None) -> Traced:
    """Ray-traced view (see or_trace_view)."""
    b = _c(boxes6, np.float64).reshape(-1, 6)
    rd = _c(road, np.float32).reshape(-1, 8)
    ln = _c(line, np.float32).reshape(-1, 8)
    sp = _sph(sph)
    cls = np.zeros((cam.height, cam.width), np.uint8)
    dep = np.zeros((cam.height, cam.width), np.float32)
    pr = np.zeros((cam.height, cam.width), np.uint32)
    c = cam.c()
    _lib().or_trace_view(ctypes.byref(c), b.shape[0], _p(b, c_f64p), int(ego), rd.shape[0],
                         _p(rd, c_f32p), ln.shape[0], _p(ln, c_f32p), sp.shape[0],
                         _p(sp, c_f64p), float(ax), float(ay),
                         float(ayaw), float(cam_yaw), _p(cls, c_u8p), _p(dep, c_f32p),
                         pr.ctypes.data_as(P(ctypes.c_uint32)))
    return Traced(cls, dep, pr)


@dataclasses.dataclass
class Image:
    key: np.ndarray      # uint64 [H, W]
    cls: np.ndarray      # uint8 [H, W]
    depth: np.ndarray    # float32 [H, W] (FP32 key mode) or uint16 binary16 bits (FP16)


def raster(tris: np.ndarray, width: int, height: int, key_f16: bool, box_end: int,
           road_end: int, bruteforce: bool = False, line_end: Optional[int] = None) -> Image:
    """The raster rule on snapped triangles; box_end = 12 n_boxes, road_end = box_end + 2 n_road,
    line_end = road_end + 2 n_line (ids from it on are signal spheres; None: no spheres)."""
    t = _c(tris, TRI_DTYPE)
    if key_f16 and len(t):
        assert int(t["prim"].max()) <= 0xFFFE, "FP16 keys hold 16-bit primitive ids"
    key = np.zeros((height, width), np.uint64)
    cls = np.zeros((height, width), np.uint8)
    d32 = np.zeros((height, width), np.float32)
    d16 = np.zeros((height, width), np.uint16)
    fn = _lib().or_raster_bruteforce if bruteforce else _lib().or_raster
    le = 0xFFFFFFFF if line_end is None else int(line_end)
    fn(t.ctypes.data, len(t), width, height, int(key_f16), box_end, road_end, le,
       _p(key, c_u64p), _p(cls, c_u8p), _p(d32, c_f32p), _p(d16, c_u16p))
    return Image(key, cls, d16 if key_f16 else d32)


# Reward weights at inference (Table "Reward terms", rightmost column), in the order
# collision, off-road, comfort, alignment, centering, velocity, traffic light, time,
# reverse, overspeed.
REWARD_WEIGHTS = (3.0, 3.0, 0.05, 0.025, 3.8e-3, 2.5e-3, 1.0, 2.5e-5, 5e-3, 0.0)
LANE_WIDTH = 3.5


OBS_AGENTS, OBS_AGENT_RADIUS, OBS_ROADS, OBS_ROAD_RADIUS = 16, 100.0, 32, 30.0


def observe_world(boxes6, speed, road, line, K=OBS_AGENTS, r_agents=OBS_AGENT_RADIUS,
                  M=OBS_ROADS, r_roads=OBS_ROAD_RADIUS, n_agents=None):
    """O_vec of one world's agents: (agents [n_agents, K, 8], roads [n_agents, M, 8])."""
    b = _c(boxes6, np.float64).reshape(-1, 6)
    sp = _c(speed, np.float64)
    rd = _c(road, np.float32).reshape(-1, 8)
    ln = _c(line, np.float32).reshape(-1, 8)
    na = b.shape[0] if n_agents is None else n_agents
    ao = np.zeros((na, K, 8), np.float64)
    ro = np.zeros((na, M, 8), np.float64)
    scratch = np.zeros(2 * max(1, b.shape[0], rd.shape[0] + ln.shape[0]), np.float64)
    _lib().or_observe_world(b.shape[0], na, _p(b, c_f64p), _p(sp, c_f64p), rd.shape[0],
                            _p(rd, c_f32p), ln.shape[0], _p(ln, c_f32p), K, float(r_agents), M,
                            float(r_roads), _p(ao, c_f64p), _p(ro, c_f64p), _p(scratch, c_f64p))
    return ao, ro


def splitmix64(seed: int, n: int) -> int:
    """n-th output (n >= 1) of the SplitMix64 stream seeded with `seed`."""
    return int(_lib().or_splitmix64(seed & (2**64 - 1), n & (2**64 - 1)))


def conditioning(seed: int, world: int, episode: int, agent: int):
    """(reward weights [10], normalised conditioning vector [12]) of one agent and episode
    (see or_conditioning)."""
    w = np.zeros(10, np.float64)
    c = np.zeros(12, np.float64)
    _lib().or_conditioning(seed & (2**64 - 1), world, episode, agent, _p(w, c_f64p), _p(c, c_f64p))
    return w, c


OBS_SIGNALS, OBS_SIGNAL_RADIUS = 4, 50.0


def observe_signals(boxes6, n_agents, sph, state, S=OBS_SIGNALS, r_sig=OBS_SIGNAL_RADIUS):
    """Traffic controls of O_vec for a world's agents: [n_agents, S, 8] (or_observe_signals)."""
    b = _c(boxes6, np.float64).reshape(-1, 6)
    sp = _sph(sph)
    st = _c(np.zeros(sp.shape[0]) if state is None else state, np.uint8)
    out = np.zeros((n_agents, S, 8), np.float64)
    scratch = np.zeros(2 * max(1, sp.shape[0]), np.float64)
    _lib().or_observe_signals(n_agents, _p(b, c_f64p), sp.shape[0], _p(sp, c_f64p), _p(st, c_u8p),
                              S, float(r_sig), _p(out, c_f64p), _p(scratch, c_f64p))
    return out


def lane_frame(px: float, py: float, road: np.ndarray, lane_w: float = LANE_WIDTH):
    """(lane direction, lateral offset x_f) of a point, or None off the road."""
    rd = _c(road, np.float32).reshape(-1, 8)
    d, x = ctypes.c_double(), ctypes.c_double()
    ok = _lib().or_lane_frame(float(px), float(py), rd.shape[0], _p(rd, c_f32p), float(lane_w),
                              ctypes.byref(d), ctypes.byref(x))
    return (d.value, x.value) if ok else None


def rewards_world(before, fl_before, after, fl_after, actions, dims, acc, weights, road,
                  lane_w=LANE_WIDTH, v_lim=30.0, dt=0.1, vmax=30.0, jerk=None, sph=None,
                  sph_state=None):
    """Per-agent reward and ego state [n, 9] of one step (see or_rewards_world); `acc`
    [n, 2] (previous accelerations) is updated in place; `jerk` [n, 3] is the post-step
    jerk-dynamics state (a_lon, a_lat, steer) or None under direct control."""
    b = _c(before, np.float64).reshape(-1, 4)
    n = b.shape[0]
    a = _c(after, np.float64).reshape(-1, 4)
    fb, fa = _c(fl_before, np.uint8), _c(fl_after, np.uint8)
    act = _c(actions, np.float32).reshape(-1, 2)
    dm = _c(dims, np.float64).reshape(-1, 2)
    assert acc.dtype == np.float64 and acc.flags.c_contiguous and acc.shape == (n, 2)
    w = _c(weights, np.float64).reshape(-1, 10)
    rd = _c(road, np.float32).reshape(-1, 8)
    reward = np.zeros(n, np.float64)
    ego = np.zeros((n, 9), np.float64)
    jk = None if jerk is None else _c(jerk, np.float64).reshape(n, 3)
    sp = _sph(sph)
    st = _c(np.zeros(sp.shape[0]) if sph_state is None else sph_state, np.uint8)
    _lib().or_rewards_world(n, _p(b, c_f64p), _p(fb, c_u8p), _p(a, c_f64p), _p(fa, c_u8p),
                            _p(act, c_f32p), _p(dm, c_f64p), _p(acc, c_f64p), _p(w, c_f64p),
                            rd.shape[0], _p(rd, c_f32p), float(lane_w), float(v_lim), float(dt),
                            float(vmax), None if jk is None else _p(jk, c_f64p),
                            sp.shape[0], _p(sp, c_f64p), _p(st, c_u8p),
                            _p(reward, c_f64p), _p(ego, c_f64p))
    return reward, ego


# Default RGB appearance (readings; the paper gives only "blue" for vehicles and static
# objects): class colours in [0, 1] and the light direction towards the light.
RGB_COLOURS = ((0.55, 0.75, 0.95), (0.33, 0.33, 0.35), (0.92, 0.92, 0.85), (0.15, 0.35, 0.85))
RGB_LIGHT = (0.3, 0.4, 0.866)
RGB_AMBIENT = 0.35
# Signal-sphere colours by state 0 red, 1 amber, 2 green, 3 off (readings).
SIGNAL_COLOURS = ((0.9, 0.1, 0.1), (0.95, 0.7, 0.1), (0.1, 0.8, 0.3), (0.25, 0.25, 0.25))


def unit(v) -> np.ndarray:
    a = np.asarray(v, np.float64)
    return a / np.sqrt(float(np.dot(a, a)))


def shade_rgb(key: np.ndarray, key_f16: bool, box_end: int, road_end: int, boxes6: np.ndarray,
              colour=RGB_COLOURS, light=RGB_LIGHT, ambient: float = RGB_AMBIENT,
              line_end: Optional[int] = None, sph=None, sph_state=None,
              signal_colour=SIGNAL_COLOURS) -> np.ndarray:
    """uint8 [3, H, W] RGB observation from the raster's keys (see or_shade_rgb)."""
    k = _c(key, np.uint64)
    b = _c(boxes6, np.float64).reshape(-1, 6)
    col = _c(colour, np.float64).reshape(4, 3)
    sc = _c(signal_colour, np.float64).reshape(4, 3)
    sp = _sph(sph)
    st = _c(np.zeros(sp.shape[0]) if sph_state is None else sph_state, np.uint8)
    le = 0xFFFFFFFF if line_end is None else int(line_end)
    l = _c(unit(light), np.float64)
    out = np.zeros((3,) + k.shape, np.uint8)
    _lib().or_shade_rgb(_p(k, c_u64p), k.size, int(key_f16), box_end, road_end, le,
                        _p(b, c_f64p), _p(sp, c_f64p), _p(st, c_u8p), _p(col, c_f64p),
                        _p(sc, c_f64p), _p(l, c_f64p), float(ambient), _p(out, c_u8p))
    return out


def f32_to_f16_bits(x) -> np.ndarray:
    a = np.asarray(x, np.float32).ravel()
    lib = _lib()
    return np.array([lib.or_f32_to_f16(float(v)) for v in a], np.uint16)


def f32_to_bf16_bits(x) -> np.ndarray:
    a = np.asarray(x, np.float32).ravel()
    lib = _lib()
    return np.array([lib.or_f32_to_bf16(float(v)) for v in a], np.uint16)


def onehot_bf16(cls: np.ndarray, mean=(0.5,) * 4, std=(0.5,) * 4) -> np.ndarray:
    """bf16 bits [4, *cls.shape] of (onehot - mean) / std, per channel."""
    c = _c(cls, np.uint8)
    m, s = _c(mean, np.float32), _c(std, np.float32)
    out = np.zeros((4,) + c.shape, np.uint16)
    _lib().or_onehot_bf16(_p(c, c_u8p), c.size, _p(m, c_f32p), _p(s, c_f32p), _p(out, c_u16p))
    return out


# ---------------------------------------------------------------------------------------
# Batch driver over worlds (plain loops)
# ---------------------------------------------------------------------------------------

class Sim:
    """Oracle simulation of a batch of worlds: FP64 agent state, latched flags."""

    def __init__(self, worlds, dt: float = 0.1, vmax: float = 30.0, jerk_dynamics: bool = False,
                 episode_steps: int = 0, conditioning_seed: Optional[int] = None):
        self.w = worlds
        self.dt, self.vmax = dt, vmax
        na = worlds.n_agents
        self.agent_off = worlds.agent_offsets()
        self.state = np.zeros((na, 4), np.float64)
        self.flags = np.zeros(na, np.uint8)
        # jerk-dynamics actuator state a_lon, a_lat, steer (None under direct control)
        self.jerk = np.zeros((na, 3), np.float64) if jerk_dynamics else None
        st = getattr(worlds, "signal_state", None)
        self.signal_state = None if st is None else np.array(st, np.uint8)
        for w in range(worlds.n_worlds):
            b0 = int(worlds.box_off[w])
            a0, a1 = int(self.agent_off[w]), int(self.agent_off[w + 1])
            bx = worlds.boxes[b0:b0 + (a1 - a0)].astype(np.float64)
            self.state[a0:a1, 0:3] = bx[:, 0:3]
            self.state[a0:a1, 3] = bx[:, 6]
        # episodes (App. A "Other Details": episodes end after a fixed time): after
        # episode_steps steps a world's agents return to their initial state with only the
        # done flag (8) set; 0 = never
        self.episode_steps = episode_steps
        self.ep = np.zeros(worlds.n_worlds, np.int64)
        self.state0 = self.state.copy()
        # reward conditioning: per-agent weights and normalised vector, redrawn at every
        # episode start (episode index per world counts the restarts)
        self.cond_seed = conditioning_seed
        self.episode_index = np.zeros(worlds.n_worlds, np.int64)
        self.weights = np.tile(np.array(REWARD_WEIGHTS, np.float64), (na, 1))
        self.cond = np.zeros((na, 12), np.float64)
        if conditioning_seed is not None:
            for w in range(worlds.n_worlds):
                self._draw(w)

    def set_state(self, state, flags, jerk=None) -> None:
        self.state[:] = np.asarray(state, np.float64)
        self.flags[:] = np.asarray(flags, np.uint8)
        if self.jerk is not None:
            self.jerk[:] = 0.0 if jerk is None else np.asarray(jerk, np.float64)

    def boxes6(self, w: int) -> np.ndarray:
        b0, b1 = int(self.w.box_off[w]), int(self.w.box_off[w + 1])
        b = self.w.boxes[b0:b1, 0:6].astype(np.float64)
        a0, a1 = int(self.agent_off[w]), int(self.agent_off[w + 1])
        b[: a1 - a0, 0:3] = self.state[a0:a1, 0:3]
        return np.ascontiguousarray(b)

    def road(self, w: int) -> np.ndarray:
        return self.w.road[int(self.w.road_off[w]):int(self.w.road_off[w + 1])]

    def line(self, w: int) -> np.ndarray:
        return self.w.line[int(self.w.line_off[w]):int(self.w.line_off[w + 1])]

    def signals(self, w: int):
        """(spheres float64 [n, 4] x, y, z, r; states uint8 [n]) of world w."""
        off = getattr(self.w, "signal_off", None)
        if off is None:
            return np.zeros((0, 4)), np.zeros(0, np.uint8)
        s0, s1 = int(off[w]), int(off[w + 1])
        st = np.zeros(s1 - s0, np.uint8) if self.signal_state is None else self.signal_state[s0:s1]
        return self.w.signal[s0:s1].astype(np.float64), np.asarray(st, np.uint8)

    def step(self, actions: np.ndarray, worlds: Optional[Sequence[int]] = None) -> None:
        ws = range(self.w.n_worlds) if worlds is None else worlds
        for w in ws:
            a0, a1 = int(self.agent_off[w]), int(self.agent_off[w + 1])
            b = self.boxes6(w)
            st = np.ascontiguousarray(self.state[a0:a1])
            fl = np.ascontiguousarray(self.flags[a0:a1] & ~np.uint8(8))
            jk = None if self.jerk is None else np.ascontiguousarray(self.jerk[a0:a1])
            sp, ss = self.signals(w)
            step_world(b, st, fl, actions[a0:a1], self.road(w), self.dt, self.vmax, jk,
                       sph=sp, sph_state=ss)
            self.state[a0:a1] = st
            self.flags[a0:a1] = fl
            if jk is not None:
                self.jerk[a0:a1] = jk
            if self.episode_steps:
                self.ep[w] += 1
                if self.ep[w] >= self.episode_steps:
                    self._restart(w)
                    self.flags[a0:a1] = 8

    def _draw(self, w: int) -> None:
        a0, a1 = int(self.agent_off[w]), int(self.agent_off[w + 1])
        for i in range(a1 - a0):
            self.weights[a0 + i], self.cond[a0 + i] = conditioning(
                self.cond_seed, w, int(self.episode_index[w]), i)

    def _restart(self, w: int) -> None:
        """A new episode of world w: initial state, clear flags, next conditioning draw."""
        a0, a1 = int(self.agent_off[w]), int(self.agent_off[w + 1])
        self.ep[w] = 0
        self.state[a0:a1] = self.state0[a0:a1]
        self.flags[a0:a1] = 0
        if self.jerk is not None:
            self.jerk[a0:a1] = 0.0
        self.episode_index[w] += 1
        if self.cond_seed is not None:
            self._draw(w)

    def reset_worlds(self, mask=None) -> None:
        for w in range(self.w.n_worlds):
            if mask is None or mask[w]:
                self._restart(w)

    def camera_tris(self, cam: CamConfig, w: int, agent_local: int, cam_yaw: float) -> np.ndarray:
        a = int(self.agent_off[w]) + agent_local
        return camera_tris(cam, self.boxes6(w), agent_local, self.road(w), self.line(w),
                           self.state[a, 0], self.state[a, 1], self.state[a, 2], cam_yaw,
                           sph=self.signals(w)[0])

    def trace(self, cam: CamConfig, w: int, agent_local: int, cam_yaw: float) -> Traced:
        a = int(self.agent_off[w]) + agent_local
        return trace_view(cam, self.boxes6(w), agent_local, self.road(w), self.line(w),
                          self.state[a, 0], self.state[a, 1], self.state[a, 2], cam_yaw,
                          sph=self.signals(w)[0])

    def prim_ranges(self, w: int):
        nb = int(self.w.box_off[w + 1] - self.w.box_off[w])
        nr = int(self.w.road_off[w + 1] - self.w.road_off[w])
        return 12 * nb, 12 * nb + 2 * nr

    def line_end(self, w: int) -> int:
        nl = int(self.w.line_off[w + 1] - self.w.line_off[w])
        return self.prim_ranges(w)[1] + 2 * nl

    def render_rgb(self, cam: CamConfig, w: int, agent_local: int, cam_yaw: float,
                   key_f16: bool = False, **appearance) -> np.ndarray:
        """uint8 [3, H, W] RGB observation of one camera (FP64 pipeline)."""
        img = self.render(cam, w, agent_local, cam_yaw, key_f16)
        be, re = self.prim_ranges(w)
        sp, st = self.signals(w)
        return shade_rgb(img.key, key_f16, be, re, self.boxes6(w), line_end=self.line_end(w),
                         sph=sp, sph_state=st, **appearance)

    def render(self, cam: CamConfig, w: int, agent_local: int, cam_yaw: float,
               key_f16: bool = False) -> Image:
        tris = self.camera_tris(cam, w, agent_local, cam_yaw)
        be, re = self.prim_ranges(w)
        return raster(tris, cam.width, cam.height, key_f16, be, re, line_end=self.line_end(w))
