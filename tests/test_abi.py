"""CPU checks of the C ABI: the library loads, exports every declared entry point, the
ctypes structures match the C header layout, and host-side validation rejects bad input
before touching a GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gigapixel.h")


@pytest.fixture(scope="module")
def gp():
    from paper_2606_19641_b300 import build, binding
    build.build()
    return binding


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:gp_status|const char \*)\s*(gp_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_symbol(gp):
    names = declared_functions()
    assert len(names) >= 15
    lib = gp.load_library()
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(gp.EXPORTED)


def test_struct_layout_matches_header(gp, tmp_path):
    c = tmp_path / "layout.c"
    c.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gigapixel.h"\n'
                 'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(gp_config),'
                 ' offsetof(gp_config, tri_capacity), offsetof(gp_config, norm_std),'
                 ' sizeof(gp_world_desc), offsetof(gp_world_desc, line), sizeof(gp_info),'
                 ' offsetof(gp_info, blocks)); return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I" + os.path.dirname(HEADER), str(c), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(gp.Config), gp.Config.tri_capacity.offset, gp.Config.norm_std.offset,
            ctypes.sizeof(gp.WorldDesc), gp.WorldDesc.line.offset, ctypes.sizeof(gp.Info),
            gp.Info.blocks.offset]
    assert got == want


def test_default_config_values(gp):
    c = gp.default_config()
    assert (c.width, c.height, c.n_cams) == (128, 128, 1)
    assert c.hfov == pytest.approx(np.pi / 2) and c.dt == pytest.approx(0.1)
    assert c.cam_height == pytest.approx(1.5) and c.near_plane == pytest.approx(0.1)
    assert list(c.norm_mean) == [0.5] * 4 and list(c.norm_std) == [0.5] * 4
    assert c.dynamics == gp.DYN_DIRECT and c.rewards == 0


def _desc(gp, worlds):
    keep = []

    def arr(a, dt, ct):
        a = np.ascontiguousarray(a, dt)
        keep.append(a)
        return a.ctypes.data_as(ctypes.POINTER(ct))
    d = gp.WorldDesc()
    d.n_worlds = worlds["n"]
    d.box_off = arr(worlds["box_off"], np.int32, ctypes.c_int32)
    d.agent_count = arr(worlds["agents"], np.int32, ctypes.c_int32)
    d.boxes = arr(worlds["boxes"], np.float32, ctypes.c_float)
    d.road_off = arr(worlds["road_off"], np.int32, ctypes.c_int32)
    d.road = arr(worlds["road"], np.float32, ctypes.c_float)
    d.line_off = arr(worlds["line_off"], np.int32, ctypes.c_int32)
    d.line = arr(worlds["line"], np.float32, ctypes.c_float)
    if "signal_off" in worlds:
        d.signal_off = arr(worlds["signal_off"], np.int32, ctypes.c_int32)
        d.signal = arr(worlds["signal"], np.float32, ctypes.c_float)
        d.signal_state = arr(worlds["signal_state"], np.uint8, ctypes.c_uint8)
    return d, keep


def _good():
    return dict(n=1, box_off=[0, 2], agents=[1], boxes=[[0, 0, 0, 4, 2, 1.5, 1], [10, 0, 0, 4, 2, 1.5, 0]],
                road_off=[0, 1], road=[[-50, -4, 50, -4, 50, 4, -50, 4]], line_off=[0, 0],
                line=np.zeros((0, 8)))


@pytest.mark.parametrize("mutate,status", [
    (lambda w, c: w.update(box_off=[0, -1]), -1),
    (lambda w, c: w.update(agents=[3]), -1),
    (lambda w, c: w.update(boxes=[[0, 0, 0, 4, 2, 1.5, 1], [10, 0, np.nan, 4, 2, 1.5, 0]]), -1),
    (lambda w, c: w.update(boxes=[[0, 0, 0, 4, 2, 1.5, 1], [10, 0, 0, 0, 2, 1.5, 0]]), -1),
    (lambda w, c: setattr(c, "width", 101), -1),
    (lambda w, c: setattr(c, "height", 63), -1),
    (lambda w, c: setattr(c, "output", 3), -1),
    (lambda w, c: (setattr(c, "output", 2), [c.light_dir.__setitem__(i, 0.0) for i in range(3)]), -1),
    (lambda w, c: (setattr(c, "output", 2), setattr(c, "ambient", -0.1)), -1),
    (lambda w, c: setattr(c, "width", 1024), -4),
    (lambda w, c: setattr(c, "n_cams", 9), -4),
    (lambda w, c: setattr(c, "key_precision", 7), -1),
    (lambda w, c: setattr(c, "threads", 100), -1),
    (lambda w, c: setattr(c, "dynamics", 2), -1),
    (lambda w, c: setattr(c, "stats", 2), -1),
    (lambda w, c: setattr(c, "episode_steps", -1), -1),
    (lambda w, c: setattr(c, "reward_conditioning", 3), -1),
    (lambda w, c: w.update(signal_off=[0, 1], signal=[[0, 0, 5, 0.0]], signal_state=[0]), -1),
    (lambda w, c: w.update(signal_off=[0, 1], signal=[[0, 0, 5, 0.4]], signal_state=[4]), -1),
    (lambda w, c: w.update(signal_off=[0, 1], signal=[[0, np.nan, 5, 0.4]], signal_state=[0]), -1),
    (lambda w, c: w.update(signal_off=[0, 33], signal=np.tile([0, 0, 5, 0.4], (33, 1)),
                           signal_state=np.zeros(33)), -4),
    (lambda w, c: w.update(box_off=[0, 130], agents=[1], boxes=np.tile([1, 1, 0, 4, 2, 1.5, 0], (130, 1))), -4),
])
def test_create_rejects_invalid_input_on_host(gp, mutate, status):
    w = _good()
    c = gp.default_config()
    mutate(w, c)
    d, keep = _desc(gp, w)
    h = ctypes.c_void_p()
    rc = gp.lib().gp_create_worlds(ctypes.byref(d), ctypes.byref(c), 0, ctypes.byref(h))
    assert rc == status
    assert h.value is None
    assert gp.lib().gp_last_error().decode()


def test_null_handle_calls_fail_cleanly(gp):
    L = gp.lib()
    assert L.gp_step(None, None, None) == -1
    assert L.gp_render(None, None, None, None) == -1
    assert L.gp_step_render_host(None, None, None, None, None, None, None) == -1
    assert L.gp_destroy(None) == 0
    assert L.gp_get_info(None, None) == -1
    assert L.gp_get_dynamics(None, None, 1, None) == -1
    assert L.gp_set_dynamics(None, None, 1, None) == -1
    assert L.gp_reset_worlds(None, None, 1, None) == -1
    assert L.gp_get_conditioning(None, None, 1, None) == -1
    assert L.gp_get_reward_weights(None, None, 1, None) == -1
    assert L.gp_get_render_stats(None, None, 0) == -1
    assert L.gp_set_signal_states(None, None, 1, None) == -1


def test_fp16_primitive_limit(gp):
    w = _good()
    w["road_off"] = [0, 32767]  # 2 boxes + 32767 quads -> 65558 primitive ids
    w["road"] = np.tile([-50, -4, 50, -4, 50, 4, -50, 4], (32767, 1))
    c = gp.default_config(key_precision=gp.KEY_F16)
    d, keep = _desc(gp, w)
    h = ctypes.c_void_p()
    assert gp.lib().gp_create_worlds(ctypes.byref(d), ctypes.byref(c), 0, ctypes.byref(h)) == -4


def test_binding_rejects_host_buffers_before_any_call(gp):
    """The Python layer hands the library raw addresses, so a host array or a tensor on
    another device must be refused before it could reach a kernel."""
    import types
    import torch
    sim = gp.Simulator.__new__(gp.Simulator)
    sim.device = 0
    sim.info = types.SimpleNamespace(n_agents=4, n_views=4, height=8, width=8,
                                     output=gp.OUT_CLASS_U8, key_precision=gp.KEY_F32)
    for bad in (np.zeros((4, 2), np.float32), torch.zeros((4, 2)), [0.0] * 8):
        with pytest.raises(gp.GigapixelError) as e:
            sim._actions(bad)
        assert e.value.status == gp.GP_EINVAL
    with pytest.raises(gp.GigapixelError):
        sim._images(torch.zeros((4, 8, 8), dtype=torch.uint8), None)
    assert sim._actions(None) == 0  # a null pointer is the library's to reject
