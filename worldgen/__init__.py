"""Seeded synthetic driving worlds and actions (input generator).

This module is the one piece shared by the CUDA path's tests/benchmarks and the CPU
oracle.  It holds none of the simulator's arithmetic: it lays out road pieces,
lane-line strips and boxes, and draws actions.  The paper trains on nuPlan scenarios
(App. A, "Other Details"), which are not available here; these synthetic worlds stand
in for them with the workload distributions stated in ``WORKLOADS``.

Layout of a batch of worlds (all host numpy arrays, CSR over worlds):

* ``box_off``  int32 [n_worlds+1]  boxes of world w are ``boxes[box_off[w]:box_off[w+1]]``
* ``agent_count`` int32 [n_worlds] the first ``agent_count[w]`` boxes of a world are agents
* ``boxes``    float32 [n_boxes, 7] x, y, yaw, L, W, H, v0
* ``road_off`` int32 [n_worlds+1], ``road`` float32 [n_road, 8] road-surface quads
* ``line_off`` int32 [n_worlds+1], ``line`` float32 [n_line, 8] lane-line strips
* ``signal_off`` int32 [n_worlds+1], ``signal`` float32 [n_signal, 4] traffic-signal
  spheres (x, y, z, radius), ``signal_state`` uint8 [n_signal] (0 red, 1 amber, 2 green,
  3 off)

Quads are four (x, y) corners, counter-clockwise seen from above.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "worldgen.c")
_SO = os.path.join(_HERE, "_worldgen.so")


class _Params(ctypes.Structure):
    _fields_ = [
        ("half_extent", ctypes.c_double),
        ("lane_w", ctypes.c_double),
        ("n_lanes", ctypes.c_int32),
        ("line_w", ctypes.c_double),
        ("seg_len_lo", ctypes.c_double),
        ("seg_len_hi", ctypes.c_double),
        ("p_straight", ctypes.c_double),
        ("arc_r_lo", ctypes.c_double),
        ("arc_r_hi", ctypes.c_double),
        ("arc_pieces", ctypes.c_int32),
        ("chain_max", ctypes.c_int32),
        ("box_l_lo", ctypes.c_double),
        ("box_l_hi", ctypes.c_double),
        ("box_w_lo", ctypes.c_double),
        ("box_w_hi", ctypes.c_double),
        ("box_h_lo", ctypes.c_double),
        ("box_h_hi", ctypes.c_double),
        ("box_gap", ctypes.c_double),
        ("heading_jitter", ctypes.c_double),
        ("v0_lo", ctypes.c_double),
        ("v0_hi", ctypes.c_double),
        ("max_tries", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile the generator's C source into a shared object next to it."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib_handle = None


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        lib.wg_default_params.argtypes = [P(_Params)]
        lib.wg_max_road_quads.argtypes = [P(_Params), ctypes.c_int32]
        lib.wg_max_road_quads.restype = ctypes.c_int64
        lib.wg_max_line_quads.argtypes = [P(_Params), ctypes.c_int32]
        lib.wg_max_line_quads.restype = ctypes.c_int64
        lib.wg_generate_world.argtypes = [
            P(_Params), ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
            ctypes.c_int32, P(ctypes.c_float), P(ctypes.c_float), P(ctypes.c_int64),
            P(ctypes.c_float), P(ctypes.c_int64), P(ctypes.c_double)]
        lib.wg_generate_world.restype = ctypes.c_int
        lib.wg_actions.argtypes = [
            ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            P(ctypes.c_float)]
        _lib_handle = lib
    return _lib_handle


def _fptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


@dataclasses.dataclass(frozen=True)
class Workload:
    """A synthetic workload: world batch shape, camera rig, output format, steps."""
    name: str
    n_worlds: int
    agents: Tuple[int, int]          # agents per world ~ U{lo..hi}
    segments: Tuple[int, int]        # road segments per world ~ U{lo..hi}
    boxes: Optional[int]             # boxes per world; None -> max(32, agents)
    width: int
    height: int
    cam_yaw_deg: Tuple[float, ...] = (0.0,)
    precision: str = "f32"           # depth key precision: "f32" or "f16"
    output: str = "class_u8"         # "class_u8", "onehot_bf16" or "rgb_u8"
    steps: int = 10
    seed: int = 1000
    dt: float = 0.1
    hfov_deg: float = 90.0
    cam_height: float = 1.5
    signals: int = 0                 # traffic-signal spheres per world

    @property
    def n_cams(self) -> int:
        return len(self.cam_yaw_deg)


# Workloads (names describe what they are).  Dimensions follow the stated synthetic
# recipe: 200 x 200 m world, 3.5 m lanes, boxes L~U[4,5] W~U[1.8,2.0] H~U[1.4,1.7] m,
# 90 deg horizontal FOV, camera 1.5 m above ground, dt = 0.1 s.
WORKLOADS = {
    "tiny": Workload("tiny: 1 world x 8 agents, 32 boxes, 200 segments, 64x64",
                     1, (8, 8), (200, 200), 32, 64, 64, steps=10, seed=1000),
    "uniform": Workload("uniform: 256 worlds x 32 agents, 32 boxes, 500 segments, 128x128",
                        256, (32, 32), (500, 500), 32, 128, 128, steps=100, seed=1001),
    "ragged": Workload("ragged: 1024 worlds, agents U{1..64}, segments U{100..2000}, 128x128",
                       1024, (1, 64), (100, 2000), None, 128, 128, steps=200, seed=1002),
    "ragged_precision": Workload(
        "ragged precision: 1024 worlds, agents U{1..64}, segments U{100..2000}, 256x144, "
        "f16 reversed-Z key, bf16 one-hot NCHW",
        1024, (1, 64), (100, 2000), None, 256, 144, precision="f16", output="onehot_bf16",
        steps=200, seed=1003),
    "sweep": Workload("sweep: 256 worlds x 32 agents x 3 cameras, 64 boxes, 1000 segments",
                      256, (32, 32), (1000, 1000), 64, 128, 128,
                      cam_yaw_deg=(0.0, 60.0, -60.0), steps=10, seed=1004),
    # The paper's observation rig (App. A rendering; training details): four cameras --
    # front, front-left, front-right (read as +-60 deg), rear -- at its two training
    # resolutions, shaded RGB with one directional light.
    "paper_rig_210x126": Workload(
        "paper rig: 256 worlds x 32 agents x 4 cameras (0, +-60, 180 deg), 8 signals, 210x126 RGB",
        256, (32, 32), (500, 500), 32, 210, 126, cam_yaw_deg=(0.0, 60.0, -60.0, 180.0),
        precision="f16", output="rgb_u8", steps=10, seed=1005, signals=8),
    "paper_rig_434x252": Workload(
        "paper rig: 256 worlds x 32 agents x 4 cameras (0, +-60, 180 deg), 8 signals, 434x252 RGB",
        256, (32, 32), (500, 500), 32, 434, 252, cam_yaw_deg=(0.0, 60.0, -60.0, 180.0),
        precision="f16", output="rgb_u8", steps=10, seed=1006, signals=8),
}


@dataclasses.dataclass
class Worlds:
    box_off: np.ndarray
    agent_count: np.ndarray
    boxes: np.ndarray
    road_off: np.ndarray
    road: np.ndarray
    line_off: np.ndarray
    line: np.ndarray
    signal_off: Optional[np.ndarray] = None
    signal: Optional[np.ndarray] = None
    signal_state: Optional[np.ndarray] = None

    def __post_init__(self):
        if self.signal_off is None:
            self.signal_off = np.zeros(self.n_worlds + 1, np.int32)
            self.signal = np.zeros((0, 4), np.float32)
            self.signal_state = np.zeros(0, np.uint8)

    @property
    def n_worlds(self) -> int:
        return int(self.agent_count.shape[0])

    @property
    def n_agents(self) -> int:
        return int(self.agent_count.sum())

    def world(self, w: int) -> "Worlds":
        """A one-world view (copies) of world w."""
        b0, b1 = int(self.box_off[w]), int(self.box_off[w + 1])
        r0, r1 = int(self.road_off[w]), int(self.road_off[w + 1])
        l0, l1 = int(self.line_off[w]), int(self.line_off[w + 1])
        s0, s1 = int(self.signal_off[w]), int(self.signal_off[w + 1])
        return Worlds(np.array([0, b1 - b0], np.int32), self.agent_count[w:w + 1].copy(),
                      self.boxes[b0:b1].copy(), np.array([0, r1 - r0], np.int32),
                      self.road[r0:r1].copy(), np.array([0, l1 - l0], np.int32),
                      self.line[l0:l1].copy(), np.array([0, s1 - s0], np.int32),
                      self.signal[s0:s1].copy(), self.signal_state[s0:s1].copy())

    def agent_offsets(self) -> np.ndarray:
        off = np.zeros(self.n_worlds + 1, np.int64)
        np.cumsum(self.agent_count, out=off[1:])
        return off


def default_params() -> _Params:
    p = _Params()
    _lib().wg_default_params(ctypes.byref(p))
    return p


def make_worlds(n_worlds: int, agents: Sequence[int], boxes: Sequence[int],
                segments: Sequence[int], seed: int, params: Optional[_Params] = None) -> Worlds:
    """Generate ``n_worlds`` worlds with the given per-world agent/box/segment counts."""
    lib = _lib()
    p = params if params is not None else default_params()
    agents = np.asarray(agents, np.int32)
    boxes_n = np.asarray(boxes, np.int32)
    segments = np.asarray(segments, np.int32)
    assert agents.shape == boxes_n.shape == segments.shape == (n_worlds,)
    assert np.all(boxes_n >= agents) and np.all(agents >= 0)
    box_off = np.zeros(n_worlds + 1, np.int32)
    np.cumsum(boxes_n, out=box_off[1:])
    box_arr = np.zeros((int(box_off[-1]), 7), np.float32)
    roads, lines = [], []
    mr = int(lib.wg_max_road_quads(ctypes.byref(p), int(segments.max(initial=0))))
    ml = int(lib.wg_max_line_quads(ctypes.byref(p), int(segments.max(initial=0))))
    rbuf = np.zeros((max(mr, 1), 8), np.float32)
    lbuf = np.zeros((max(ml, 1), 8), np.float32)
    scratch = np.zeros((max(mr, 1), 6), np.float64)
    nr, nl = ctypes.c_int64(), ctypes.c_int64()
    for w in range(n_worlds):
        bview = box_arr[box_off[w]:box_off[w + 1]]
        bview = np.ascontiguousarray(bview)
        rc = lib.wg_generate_world(ctypes.byref(p), ctypes.c_uint64(seed), w, int(agents[w]),
                                   int(boxes_n[w]), int(segments[w]), _fptr(bview), _fptr(rbuf),
                                   ctypes.byref(nr), _fptr(lbuf), ctypes.byref(nl),
                                   scratch.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        if rc != 0:
            raise RuntimeError("worldgen: could not place %d boxes in world %d" % (boxes_n[w], w))
        box_arr[box_off[w]:box_off[w + 1]] = bview
        roads.append(rbuf[:nr.value].copy())
        lines.append(lbuf[:nl.value].copy())
    road_off = np.zeros(n_worlds + 1, np.int32)
    np.cumsum([len(r) for r in roads], out=road_off[1:])
    line_off = np.zeros(n_worlds + 1, np.int32)
    np.cumsum([len(l) for l in lines], out=line_off[1:])
    road = np.concatenate(roads) if roads else np.zeros((0, 8), np.float32)
    line = np.concatenate(lines) if lines else np.zeros((0, 8), np.float32)
    return Worlds(box_off, agents, box_arr, road_off, np.ascontiguousarray(road, np.float32),
                  line_off, np.ascontiguousarray(line, np.float32))


def workload_counts(wl: Workload):
    """Per-world (agents, boxes, segments) counts for a workload (seeded)."""
    rng = np.random.default_rng(wl.seed)
    ag = rng.integers(wl.agents[0], wl.agents[1] + 1, size=wl.n_worlds).astype(np.int32)
    sg = rng.integers(wl.segments[0], wl.segments[1] + 1, size=wl.n_worlds).astype(np.int32)
    if wl.boxes is None:
        bx = np.maximum(32, ag).astype(np.int32)
    else:
        bx = np.maximum(wl.boxes, ag).astype(np.int32)
    return ag, bx, sg


def add_signals(worlds: Worlds, per_world: int, seed: int, height: float = 5.0,
                radius: float = 0.4) -> Worlds:
    """Place ``per_world`` traffic-signal spheres over each world's road: each hangs
    ``height`` m above the centroid of a road quad drawn uniformly (seeded per world), in a
    uniformly drawn state red / amber / green.  Worlds without road get none."""
    sig, st, counts = [], [], []
    for w in range(worlds.n_worlds):
        r0, r1 = int(worlds.road_off[w]), int(worlds.road_off[w + 1])
        k = per_world if r1 > r0 else 0
        rng = np.random.default_rng([seed, w, 7])
        q = worlds.road[r0 + rng.integers(0, max(r1 - r0, 1), size=k)].reshape(k, 4, 2)
        c = q.astype(np.float64).mean(axis=1)
        sig.append(np.column_stack([c, np.full(k, height), np.full(k, radius)]))
        st.append(rng.integers(0, 3, size=k))
        counts.append(k)
    worlds.signal_off = np.zeros(worlds.n_worlds + 1, np.int32)
    np.cumsum(counts, out=worlds.signal_off[1:])
    worlds.signal = np.ascontiguousarray(np.concatenate(sig) if sig else np.zeros((0, 4)),
                                         np.float32).reshape(-1, 4)
    worlds.signal_state = np.ascontiguousarray(np.concatenate(st) if st else np.zeros(0), np.uint8)
    return worlds


def make_workload(wl: Workload, n_worlds: Optional[int] = None) -> Worlds:
    """Worlds of a workload; ``n_worlds`` takes only the first worlds (same seeds)."""
    ag, bx, sg = workload_counts(wl)
    n = wl.n_worlds if n_worlds is None else n_worlds
    worlds = make_worlds(n, ag[:n], bx[:n], sg[:n], wl.seed)
    if wl.signals:
        add_signals(worlds, wl.signals, wl.seed)
    return worlds


def actions(seed: int, step: int, n_agents: int, gid0: int = 0,
            accel=(-3.0, 2.0), steer=(-0.3, 0.3)) -> np.ndarray:
    """Actions [n_agents, 2] (accel m/s^2, steer rad) for one step, counter-based."""
    out = np.zeros((n_agents, 2), np.float32)
    if n_agents:
        _lib().wg_actions(ctypes.c_uint64(seed), step, gid0, n_agents, accel[0], accel[1],
                          steer[0], steer[1], _fptr(out))
    return out


# App. A's discrete action set: (longitudinal, lateral) jerk in m/s^3.
JERK_TABLE = np.array([(jl, jt) for jl in (-15.0, -4.0, 0.0, 4.0) for jt in (-4.0, 0.0, 4.0)],
                      np.float32)


def jerk_actions(seed: int, step: int, n_agents: int) -> np.ndarray:
    """Jerk actions [n_agents, 2] for one step: a uniform pick from the twelve per agent."""
    rng = np.random.default_rng([seed, step, 12])
    return JERK_TABLE[rng.integers(0, 12, n_agents)]


def deg(x: float) -> float:
    return x * math.pi / 180.0
