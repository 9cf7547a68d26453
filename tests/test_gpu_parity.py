"""GPU parity tests: the CUDA path (through the C ABI) against the CPU oracle.

Tiers:
  T1 step      one GPU step from an FP32 state vs one oracle FP64 step from the same state:
               pose/speed within FP32 rounding, flags identical.
  T2 geometry  snapped vertices of every triangle the GPU rasterised vs the oracle's FP64
               geometry from the same state: within 1 unit (1/16 px), matched by
               (primitive, fan index).
  T3 raster    the oracle's raster rule applied to the GPU's own snapped triangles gives
               bit-identical class, depth and one-hot outputs.
  T4 image     GPU image vs the oracle's full FP64 pipeline: class mismatch fraction and
               depth error reported and bounded.
"""
import numpy as np
import pytest

import oracle
import worldgen as wg
from gpu_common import (assert_views, cam_config, check_views, cls_of, dedupe, expected_planes,
                        gpu_view, oracle_raster_of, oracle_sim, sim_for, view_loc)

pytestmark = pytest.mark.gpu

# class mismatch bound vs the FP64 pipeline for the tests that do not run the per-view
# T2 accounting of check_views (which bounds each sample by the pixels its differing
# triangles can flip): a class differs only at a pixel centre within 1/16 px of an edge
# whose snapped vertex moved by one unit; about 1 in 1500 visible triangles has such a
# vertex, and a far (short, perimeter ~6 px) triangle can flip at most every centre along
# its edges, perimeter + 3 ~ 9 pixels, so about 1000 triangles x 9 / 1500 ~ 6 pixels per
# 128 x 128 view: 4e-4 (measured: 3e-5 at most)
T4_MISMATCH = 4e-4


def sample_views(worlds, sim, n, seed):
    """About n views: every camera of the first agent of the four heaviest worlds (the most
    road and lane-line quads; their items lead the work order) and uniformly drawn others."""
    cams = sim.n_views // worlds.n_agents
    off = worlds.agent_offsets()
    quads = np.diff(worlds.road_off) + np.diff(worlds.line_off)
    heavy = [int(w) for w in np.argsort(-quads, kind="stable") if off[w + 1] > off[w]][:4]
    views = {int(off[w]) * cams + c for w in heavy for c in range(cams)}
    rng = np.random.default_rng(seed)
    extra = rng.choice(sim.n_views, min(n, sim.n_views), replace=False).tolist()
    for v in extra:
        if len(views) >= n:
            break
        views.add(int(v))
    return sorted(views)


def torch_actions(worlds, step, seed):
    import torch
    a = wg.actions(seed, step, worlds.n_agents)
    return torch.from_numpy(a).cuda(), a


def check_t3(sim, cfg, worlds, views, out, depth):
    """Bit-exact raster parity for the given views (returns total covered pixels)."""
    covered = 0
    for v in views:
        tris = dedupe(sim.dump_tris(v, out, depth))
        img = oracle_raster_of(worlds, cfg, v, tris)
        go, gd = gpu_view(cfg, out, depth, v)
        eo, ed = expected_planes(cfg, img)
        assert np.array_equal(go, eo), "view %d: class/one-hot differs from the raster rule" % v
        if depth is not None:
            assert np.array_equal(gd, ed), "view %d: depth bits differ from the raster rule" % v
        covered += int((img.cls > 0).sum())
    return covered


def t4_stats(sim, cfg, worlds, views, out, depth):
    """Class mismatch fraction and depth errors vs the oracle's FP64 pipeline."""
    osim = oracle_sim(worlds, sim)
    cam = cam_config(cfg)
    mism, total, derr = 0, 0, []
    for v in views:
        w, a, c = view_loc(worlds, cfg, v)
        img = osim.render(cam, w, a, float(np.float32(cfg.cam_yaw[c])), bool(cfg.key_precision))
        go, gd = gpu_view(cfg, out, depth, v)
        gcls = cls_of(cfg, go)
        ocls = img.cls if int(cfg.output) == 0 else np.where(img.cls == 4, 3, img.cls)  # one-hot: signals in channel 3
        mism += int((gcls != ocls).sum())
        total += gcls.size
        if depth is not None:
            both = (gcls > 0) & (gcls == ocls)
            if int(cfg.key_precision) == 0:
                g = gd.view(np.float32)[both].astype(np.float64)
                e = img.depth[both].astype(np.float64)
            else:
                g = gd[both].view(np.float16).astype(np.float64)
                e = img.depth[both].view(np.float16).astype(np.float64)
            if len(g):
                derr.append(np.abs(g - e) / np.maximum(e, 1e-6))
    d = np.concatenate(derr) if derr else np.zeros(1)
    return mism / max(total, 1), d


# ---------------------------------------------------------------------------------------
# T1 step
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("name,n_worlds,steps", [("tiny", 1, 10), ("uniform", 6, 20),
                                                 ("ragged", 8, 12)])
def test_step_matches_oracle_from_same_state(name, n_worlds, steps):
    wl = wg.WORKLOADS[name]
    worlds = wg.make_workload(wl, n_worlds=n_worlds)
    sim, cfg = sim_for(worlds, wl)
    n_halted = 0
    for k in range(steps):
        st0, fl0 = sim.get_state()
        osim = oracle.Sim(worlds)
        osim.set_state(st0.astype(np.float64), fl0)
        act_t, act = torch_actions(worlds, k, wl.seed)
        sim.step(act_t)
        osim.step(act)
        st1, fl1 = sim.get_state()
        moving = (fl0 & 4) == 0
        assert np.allclose(st1[:, 0:2], osim.state[:, 0:2], atol=2e-4, rtol=0)
        dyaw = np.angle(np.exp(1j * (st1[:, 2].astype(np.float64) - osim.state[:, 2])))
        assert np.all(np.abs(dyaw) < 2e-5)
        assert np.allclose(st1[:, 3], osim.state[:, 3], atol=2e-5)
        assert np.array_equal(fl1, osim.flags), "flags differ at step %d" % k
        assert np.all(st1[~moving, :3] == st0[~moving, :3])  # halted agents do not move
        n_halted = int((fl1 & 4).astype(bool).sum())
    if name != "tiny":
        assert n_halted > 0  # random steering does drive some agents off the road


@pytest.mark.parametrize("name,n_worlds,steps,jerk", [("uniform", 4, 15, False), ("ragged", 6, 12, False),
                                                      ("uniform", 4, 12, True)],
                         ids=["uniform", "ragged", "uniform-jerk"])
def test_red_light_halt_matches_oracle(name, n_worlds, steps, jerk):
    """App. A "Other Details": a red-light violation halts the agent like a collision or an
    off-road departure.  32 red signals per world hang over the agents' roads; every step
    from the GPU's own FP32 state (and, under the jerk dynamics, actuator state) is compared
    with one oracle step: pose and speed within FP32 rounding, flags identical (including
    the red-light bit 16), rewards as the oracle's (direct control); violators stop at once
    and stay where they stopped."""
    import torch
    import paper_2606_19641_b300 as gp
    wl = wg.WORKLOADS[name]
    worlds = wg.make_workload(wl, n_worlds=n_worlds)
    wg.add_signals(worlds, 32, wl.seed, height=5.0)
    worlds.signal_state[:] = 0
    extra = dict(dynamics=gp.DYN_JERK) if jerk else {}
    sim, cfg = sim_for(worlds, wl, rewards=1, **extra)
    off = worlds.agent_offsets()
    na = worlds.n_agents
    dims = np.zeros((na, 2), np.float64)
    for w in range(worlds.n_worlds):
        b0 = int(worlds.box_off[w])
        a0, a1 = int(off[w]), int(off[w + 1])
        dims[a0:a1] = worlds.boxes[b0:b0 + (a1 - a0), 3:5]
    weights = np.tile(np.array(oracle.REWARD_WEIGHTS, np.float32), (na, 1))
    acc = np.zeros((na, 2), np.float64)
    red = np.zeros(na, bool)
    stopped_at = {}
    for k in range(steps):
        st0, fl0 = sim.get_state()
        if jerk:
            osim = oracle.Sim(worlds, jerk_dynamics=True)
            osim.set_state(st0.astype(np.float64), fl0, sim.get_dynamics().astype(np.float64))
            act = _jerk_actions(na, k, wl.seed)
            act_t = torch.from_numpy(act).cuda()
        else:
            osim = oracle.Sim(worlds)
            osim.set_state(st0.astype(np.float64), fl0)
            act_t, act = torch_actions(worlds, k, wl.seed)
        sim.step(act_t)
        osim.step(act)
        st1, fl1 = sim.get_state()
        if jerk:
            assert np.allclose(sim.get_dynamics(), osim.jerk, atol=2e-5, rtol=0)
        r, _ = sim.rewards()
        torch.cuda.synchronize()
        r = r.cpu().numpy()
        assert np.array_equal(fl1, osim.flags), "flags differ at step %d" % k
        assert np.allclose(st1[:, 0:2], osim.state[:, 0:2], atol=2e-4, rtol=0)
        assert np.allclose(st1[:, 3], osim.state[:, 3], atol=2e-5)
        new = (fl1 & 16).astype(bool) & ~(fl0 & 16).astype(bool)
        assert np.all(fl1[new] & 4) and np.all(st1[new, 3] == 0.0)
        for i in np.flatnonzero(new):
            stopped_at[i] = st1[i, 0:3].copy()
        for i, pose in stopped_at.items():
            assert np.array_equal(st1[i, 0:3], pose), "agent %d moved after its red-light halt" % i
        red |= new
        for w in range(0 if jerk else worlds.n_worlds):  # jerk rewards: their own test
            a0, a1 = int(off[w]), int(off[w + 1])
            road = worlds.road[int(worlds.road_off[w]):int(worlds.road_off[w + 1])]
            s0, s1 = int(worlds.signal_off[w]), int(worlds.signal_off[w + 1])
            acc_w = np.ascontiguousarray(acc[a0:a1])
            rr, _ = oracle.rewards_world(st0[a0:a1], fl0[a0:a1], st1[a0:a1], fl1[a0:a1],
                                         act[a0:a1], dims[a0:a1], acc_w, weights[a0:a1], road,
                                         sph=worlds.signal[s0:s1],
                                         sph_state=worlds.signal_state[s0:s1])
            acc[a0:a1] = acc_w
            # the red-light term is charged exactly on the steps that set the flag
            tl = np.abs(rr - r[a0:a1]) <= 1e-4 + 1e-4 * np.abs(rr) + weights[a0:a1, 2]
            assert np.all(tl)
    print("red-light halts: %d of %d agents" % (int(red.sum()), na))
    assert red.sum() > 0
    assert sim.status() == 0


# ---------------------------------------------------------------------------------------
# T2 / T3 / T4 rendering
# ---------------------------------------------------------------------------------------

SHAPES = [dict(), dict(band_rows=16), dict(band_rows=8, threads=128, tri_capacity=224),
          dict(threads=1024, tri_capacity=1024), dict(band_rows=128, threads=256, tri_capacity=300),
          # pipelined kernel: producer warps set up batches while the rest rasterise
          dict(producer_warps=4), dict(band_rows=8, threads=128, tri_capacity=224, producer_warps=1),
          dict(threads=1024, tri_capacity=512, producer_warps=12),
          dict(band_rows=128, threads=512, tri_capacity=300, producer_warps=6)]


@pytest.mark.parametrize("shape", SHAPES,
                         ids=lambda s: "-".join("%s%s" % kv for kv in s.items()) or "default")
@pytest.mark.parametrize("name,n_worlds", [("tiny", 1), ("uniform", 3)])
def test_raster_bit_exact_for_gpu_triangles(name, n_worlds, shape):
    import torch
    wl = wg.WORKLOADS[name]
    worlds = wg.make_workload(wl, n_worlds=n_worlds)
    sim, cfg = sim_for(worlds, wl, **shape)
    out, depth = sim.alloc_outputs()
    for k in range(3):
        sim.step(torch_actions(worlds, k, wl.seed)[0])
    sim.render(out, depth)
    torch.cuda.synchronize()
    assert sim.info.producer_warps == shape.get("producer_warps", 0)
    assert sim.status() == 0
    views = list(range(0, sim.n_views, max(1, sim.n_views // 12)))
    covered = check_t3(sim, cfg, worlds, views, out, depth)
    assert covered > 0.2 * len(views) * cfg.width * cfg.height


@pytest.mark.parametrize("name,n_worlds,views", [("tiny", 1, 8), ("uniform", 2, 16), ("ragged", 4, 24)])
def test_snapped_vertices_within_one_unit_of_fp64(name, n_worlds, views):
    """T2 in both directions plus T3 and the located T4 on the same views (check_views)."""
    import torch
    wl = wg.WORKLOADS[name]
    worlds = wg.make_workload(wl, n_worlds=n_worlds)
    sim, cfg = sim_for(worlds, wl)
    out, depth = sim.alloc_outputs()
    for k in range(2):
        sim.step(torch_actions(worlds, k, wl.seed)[0])
    torch.cuda.synchronize()
    vs = list(range(0, sim.n_views, max(1, sim.n_views // views)))
    S = check_views(sim, cfg, worlds, vs, out, depth)
    assert_views(S, "T2/T3/T4 %s" % name)
    assert S["o_vis"] > 50
    assert S["exact"] >= 0.9 * S["matched"]


@pytest.mark.parametrize("name,n_worlds", [("tiny", 1), ("uniform", 2)])
def test_image_vs_fp64_pipeline(name, n_worlds):
    import torch
    wl = wg.WORKLOADS[name]
    worlds = wg.make_workload(wl, n_worlds=n_worlds)
    sim, cfg = sim_for(worlds, wl)
    out, depth = sim.alloc_outputs()
    for k in range(3):
        sim.step(torch_actions(worlds, k, wl.seed)[0])
    sim.render(out, depth)
    torch.cuda.synchronize()
    views = list(range(0, sim.n_views, max(1, sim.n_views // 16)))
    frac, derr = t4_stats(sim, cfg, worlds, views, out, depth)
    print("T4 %s: class mismatch %.2e, depth rel err median %.2e p99 %.2e max %.2e" % (
        name, frac, np.median(derr), np.percentile(derr, 99), derr.max()))
    assert frac < T4_MISMATCH
    assert np.percentile(derr, 99) < 1e-3


@pytest.mark.parametrize("shape", [dict(), dict(threads=512, tri_capacity=1024, producer_warps=4)],
                         ids=["default", "pipelined"])
def test_precision_path_fp16_key_and_bf16_onehot(shape):
    import torch
    wl = wg.WORKLOADS["ragged_precision"]
    worlds = wg.make_workload(wl, n_worlds=4)
    sim, cfg = sim_for(worlds, wl, **shape)
    out, depth = sim.alloc_outputs()
    assert out.dtype == torch.bfloat16 and depth.dtype == torch.float16
    sim.step(torch_actions(worlds, 0, wl.seed)[0])
    sim.render(out, depth)
    torch.cuda.synchronize()
    views = list(range(0, sim.n_views, max(1, sim.n_views // 10)))
    check_t3(sim, cfg, worlds, views, out, depth)
    # one-hot values are exactly +-1 with the default normalisation
    u = torch.unique(out.view(torch.int16)).cpu().numpy().view(np.uint16)
    assert set(u.tolist()) <= {0x3F80, 0xBF80}
    frac, derr = t4_stats(sim, cfg, worlds, views, out, depth)
    print("T4 precision: class mismatch %.2e, depth rel err p99 %.2e" % (frac, np.percentile(derr, 99)))
    assert frac < T4_MISMATCH
    # without a depth output the one-hot tensor is the same
    out2, _ = sim.alloc_outputs(depth=False)
    sim.render(out2, None)
    torch.cuda.synchronize()
    assert torch.equal(out.view(torch.int16), out2.view(torch.int16))


def test_camera_rig_three_cameras():
    import torch
    wl = wg.WORKLOADS["sweep"]
    worlds = wg.make_workload(wl, n_worlds=2)
    sim, cfg = sim_for(worlds, wl)
    assert sim.n_views == 3 * worlds.n_agents
    out, depth = sim.alloc_outputs()
    sim.render(out, depth)
    torch.cuda.synchronize()
    check_t3(sim, cfg, worlds, [0, 1, 2, 3 * 5 + 1, 3 * 40 + 2], out, depth)


@pytest.mark.parametrize("size", [(512, 512), (64, 48), (256, 144), (16, 16)])
def test_resolutions(size):
    import torch
    wl = wg.WORKLOADS["tiny"]
    worlds = wg.make_workload(wl)
    sim, cfg = sim_for(worlds, wl, width=size[0], height=size[1])
    out, depth = sim.alloc_outputs()
    sim.render(out, depth)
    torch.cuda.synchronize()
    check_t3(sim, cfg, worlds, list(range(sim.n_views)), out, depth)


def test_edge_case_worlds():
    """No roads, a lone agent, a world without agents, and a camera facing empty space."""
    import torch
    road = np.array([[-20, -4, 20, -4, 20, 4, -20, 4]], np.float32)
    line = np.array([[-20, -0.1, 20, -0.1, 20, 0.1, -20, 0.1]], np.float32)
    boxes = np.array([
        [0, 0, 0, 4.5, 1.9, 1.5, 2.0], [12, 0, 0, 4.5, 1.9, 1.5, 0.0],   # w0: agent + static, no road
        [0, 0, 0, 4.5, 1.9, 1.4, 1.0],                                   # w1: lone agent on a road
        [5, 5, 0, 4.5, 1.9, 1.5, 0.0],                                   # w2: static box only
        [90, 0, 0, 4.5, 1.9, 1.5, 0.0],                                  # w3: agent facing nothing
    ], np.float32)
    worlds = wg.Worlds(box_off=np.array([0, 2, 3, 4, 5], np.int32),
                       agent_count=np.array([1, 1, 0, 1], np.int32), boxes=boxes,
                       road_off=np.array([0, 0, 1, 1, 2], np.int32), road=np.concatenate([road, road]),
                       line_off=np.array([0, 0, 1, 1, 1], np.int32), line=line)
    wl = wg.WORKLOADS["tiny"]
    sim, cfg = sim_for(worlds, wl)
    assert sim.n_agents == 3
    out, depth = sim.alloc_outputs()
    sim.render(out, depth)
    torch.cuda.synchronize()
    check_t3(sim, cfg, worlds, [0, 1, 2], out, depth)
    o = out.cpu().numpy()
    assert (o[0] == 3).any() and not (o[0] == 1).any()   # box visible, no road
    assert (o[1] == 1).any() and (o[1] == 2).any()        # road and line, no box
    assert not o[2].any()                                  # nothing ahead of the third agent
    act = torch.zeros((3, 2), device="cuda")
    sim.step(act)
    st, fl = sim.get_state()
    assert fl[0] & 2 and fl[0] & 4        # no road at all: off-road, halted
    assert fl[1] == 0                      # on its road


@pytest.mark.parametrize("precision", [False, True], ids=["f32", "f16"])
def test_full_width_spans_fill_a_wave(precision):
    """The largest wave of the fragment walk: 32 boxes one behind the other, each front face
    (30 m wide, 21 m tall, 5..14 m ahead, inside the guard band, its diagonal above the view)
    covering whole 512-pixel rows, so every wave of 32 row items carries 32 full-width spans
    (16 384 fragments: the walk's packed span fields at their limits).  Raster parity (T3)
    on the GPU's own triangles."""
    import torch
    import paper_2606_19641_b300 as gp
    n = 32
    boxes = np.zeros((n + 1, 7), np.float32)
    boxes[0] = [0, 0, 0, 4.5, 1.9, 1.5, 0.0]  # the agent, facing +x
    for k in range(n):
        boxes[k + 1] = [5.1 + 0.3 * k, 0, 0, 0.2, 30.0, 21.0, 0.0]
    worlds = wg.Worlds(box_off=np.array([0, n + 1], np.int32), agent_count=np.array([1], np.int32),
                       boxes=boxes, road_off=np.array([0, 0], np.int32), road=np.zeros((0, 8), np.float32),
                       line_off=np.array([0, 0], np.int32), line=np.zeros((0, 8), np.float32))
    wl = wg.WORKLOADS["tiny"]
    extra = dict(key_precision=gp.KEY_F16) if precision else {}
    sim, cfg = sim_for(worlds, wl, width=512, height=512, band_rows=16, **extra)
    out, depth = sim.alloc_outputs()
    sim.render(out, depth)
    torch.cuda.synchronize()
    assert sim.status() == 0
    assert check_t3(sim, cfg, worlds, [0], out, depth) > 300 * 512
    o = out.cpu().numpy()[0]
    assert (o[:300] == 3).all()  # every pixel of the upper rows shows the nearest box face
    # the counters of the same render: every box face covers >= 282 whole rows, so the
    # waves above row 282 are all full-width spans
    cnt, _ = sim_for(worlds, wl, width=512, height=512, band_rows=16, stats=1, **extra)
    cnt.render_stats(reset=True)
    cnt.render(out, depth)
    st = cnt.render_stats(reset=True)
    assert st["fragments"] >= n * 282 * 512, st


@pytest.mark.parametrize("precision", [False, True], ids=["f32", "f16"])
def test_maximum_sizes(precision):
    """The documented limits at once: a world of GP_MAX_BOXES = 128 boxes that are all
    agents, GP_MAX_CAMS = 8 cameras per agent (every 45 deg), 2000 road segments (20 300
    quads, 42 136 primitive ids: within the FP16 key's 16-bit ids), and a second world of
    100 agents among 128 boxes.  One step against the oracle (all 128 x 128 box pairs), then
    T3, T2 and T4 on every camera of four agents, and the ray tracer on some views."""
    import math
    import torch
    import paper_2606_19641_b300 as gp
    worlds = wg.make_worlds(2, [128, 100], [128, 128], [2000, 1500], seed=77)
    wl = wg.WORKLOADS["tiny"]
    extra = dict(key_precision=gp.KEY_F16) if precision else {}
    sim, cfg = sim_for(worlds, wl, width=64, height=64,
                       cam_yaw=[math.radians(45.0 * k) for k in range(8)], **extra)
    assert sim.n_views == 8 * 228
    st0, fl0 = sim.get_state()
    osim = oracle.Sim(worlds)
    osim.set_state(st0.astype(np.float64), fl0)
    act_t, act = torch_actions(worlds, 0, 4242)
    sim.step(act_t)
    osim.step(act)
    st1, fl1 = sim.get_state()
    assert np.allclose(st1[:, 0:2], osim.state[:, 0:2], atol=2e-4, rtol=0)
    assert np.array_equal(fl1, osim.flags)
    out, depth = sim.alloc_outputs()
    sim.render(out, depth)
    torch.cuda.synchronize()
    assert sim.status() == 0
    views = sorted(8 * a + c for a in (0, 63, 127, 200) for c in range(8))
    S = check_views(sim, cfg, worlds, views, out, depth)
    assert_views(S, "maximum sizes %s" % ("f16" if precision else "f32"), min_covered=0.05)
    if not precision:
        sim.trace(out, depth)
        torch.cuda.synchronize()
        o2 = oracle_sim(worlds, sim)
        cam = cam_config(cfg)
        bad = total = 0
        for v in views[::4]:
            w, a, c = view_loc(worlds, cfg, v)
            tr = o2.trace(cam, w, a, float(np.float32(cfg.cam_yaw[c])))
            g = out[v].cpu().numpy()
            bad += int((g != tr.cls).sum())
            total += g.size
        assert bad <= 1e-3 * total


# ---------------------------------------------------------------------------------------
# Paths, state and status
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [dict(), dict(producer_warps=2)], ids=["default", "pipelined"])
def test_graph_and_per_world_paths_match_direct_calls(shape):
    """Direct calls, the step + render graph and the one-world-at-a-time path give identical
    images and states; 16 red signals per world over the roads make the red-light halts run
    on every path."""
    import torch
    wl = wg.WORKLOADS["ragged"]
    worlds = wg.make_workload(wl, n_worlds=6)
    wg.add_signals(worlds, 16, wl.seed, height=5.0)
    worlds.signal_state[:] = 0
    a, cfg = sim_for(worlds, wl, **shape)
    b, _ = sim_for(worlds, wl, **shape)
    c, _ = sim_for(worlds, wl, **shape)
    oa, da = a.alloc_outputs()
    ob, db = b.alloc_outputs()
    oc, dc = c.alloc_outputs()
    act = torch.empty((worlds.n_agents, 2), device="cuda")
    for k in range(4):
        act.copy_(torch_actions(worlds, k, wl.seed)[0])
        a.step(act)
        a.render(oa, da)
        b.step_render(act, ob, db)
        for w in range(worlds.n_worlds):
            c.step_world(w, act)
        for w in range(worlds.n_worlds):
            c.render_world(w, oc, dc)
        torch.cuda.synchronize()
        assert torch.equal(oa, ob) and torch.equal(da.view(torch.int32), db.view(torch.int32))
        assert torch.equal(oa, oc) and torch.equal(da.view(torch.int32), dc.view(torch.int32))
    sa, fa = a.get_state()
    sb, fb = b.get_state()
    sc, fc = c.get_state()
    assert np.array_equal(sa, sb) and np.array_equal(sa, sc)
    assert np.array_equal(fa, fb) and np.array_equal(fa, fc)
    assert (fa & 16).any()  # some agent ran a red light and was halted on every path


def test_host_step_matches_graph_path():
    """gp_step_render_host (pinned host actions in, pinned host state out, one call) gives the
    images and states of gp_step_render + gp_get_state on device buffers, step after step,
    and refuses pageable host buffers before any launch."""
    import torch
    import paper_2606_19641_b300 as gp
    wl = wg.WORKLOADS["ragged"]
    worlds = wg.make_workload(wl, n_worlds=6)
    a, cfg = sim_for(worlds, wl)
    b, _ = sim_for(worlds, wl)
    oa, da = a.alloc_outputs()
    ob, db = b.alloc_outputs()
    n = worlds.n_agents
    act = torch.empty((n, 2), device="cuda")
    h_act = torch.empty((n, 2), dtype=torch.float32).pin_memory()
    h_state = torch.empty((n, 4), dtype=torch.float32).pin_memory()
    h_flags = torch.empty((n,), dtype=torch.uint8).pin_memory()
    for k in range(4):
        acts = torch_actions(worlds, k, wl.seed)[0]
        act.copy_(acts)
        h_act.copy_(acts.cpu())
        a.step_render(act, oa, da)
        b.step_render_host(h_act, ob, db, h_state, h_flags)
        torch.cuda.synchronize()
        assert torch.equal(oa, ob) and torch.equal(da.view(torch.int32), db.view(torch.int32))
        sa, fa = a.get_state()
        assert np.array_equal(sa, h_state.numpy()) and np.array_equal(fa, h_flags.numpy())
    L, h = gp.lib(), b._h
    page = np.zeros((n, 4), np.float32)  # pageable host memory
    assert L.gp_step_render_host(h, page.ctypes.data, ob.data_ptr(), None, None, None,
                                 None) == gp.binding.GP_EINVAL
    assert L.gp_step_render_host(h, h_act.data_ptr(), ob.data_ptr(), None, page.ctypes.data,
                                 None, None) == gp.binding.GP_EINVAL
    assert "pinned" in L.gp_last_error().decode()
    with pytest.raises(gp.GigapixelError):
        b.step_render_host(act, ob, db)  # a device tensor where pinned host memory belongs
    torch.cuda.synchronize()
    sb, fb = b.get_state()
    assert np.array_equal(sb, h_state.numpy())  # the refused calls stepped nothing
    assert b.status() == 0


def test_state_roundtrip_and_fork():
    import torch
    wl = wg.WORKLOADS["uniform"]
    worlds = wg.make_workload(wl, n_worlds=2)
    sim, cfg = sim_for(worlds, wl)
    for k in range(3):
        sim.step(torch_actions(worlds, k, wl.seed)[0])
    snap_s, snap_f = sim.get_state()
    out1, d1 = sim.alloc_outputs()
    out2, d2 = sim.alloc_outputs()
    for k in range(3, 6):
        sim.step(torch_actions(worlds, k, wl.seed)[0])
    sim.render(out1, d1)
    end_s, end_f = sim.get_state()
    sim.set_state(snap_s, snap_f)          # fork: rewind and replay the same actions
    s2, f2 = sim.get_state()
    assert np.array_equal(s2, snap_s) and np.array_equal(f2, snap_f)
    for k in range(3, 6):
        sim.step(torch_actions(worlds, k, wl.seed)[0])
    sim.render(out2, d2)
    torch.cuda.synchronize()
    s3, f3 = sim.get_state()
    assert np.array_equal(s3, end_s) and np.array_equal(f3, end_f)
    assert torch.equal(out1, out2) and torch.equal(d1, d2)


@pytest.mark.parametrize("autotuned", [False, True], ids=["default", "autotuned"])
def test_pipeline_wait_runs_out_and_is_reported(autotuned):
    """The pipelined kernel's handoff waits are bounded: with producers that publish
    nothing, the consumers give up after the limit, the status word says so, the call
    returns promptly, and after clearing the status the context renders normally."""
    import time
    import torch
    import paper_2606_19641_b300 as gp
    wl = wg.WORKLOADS["tiny"]
    worlds = wg.make_workload(wl)
    sim, cfg = sim_for(worlds, wl, autotune=int(autotuned))
    out, depth = sim.alloc_outputs()
    sim.render(out, depth)
    torch.cuda.synchronize()
    ref_out, ref_depth = out.clone(), depth.clone()
    out.zero_()
    depth.zero_()
    t0 = time.perf_counter()
    sim.debug_stall_pipeline(out, depth, wait_ns=20_000_000)
    took = time.perf_counter() - t0
    bits = sim.status()
    assert bits & gp.binding.DEV_PIPELINE_TIMEOUT
    assert took < 10.0
    assert int(out.abs().sum()) == 0  # nothing was rendered
    with pytest.raises(gp.GigapixelError) as e:  # the bit is sticky until cleared
        sim.render(out, depth)
    assert e.value.status == gp.binding.GP_EDEVICE
    sim.clear_status()
    sim.render(out, depth)
    torch.cuda.synchronize()
    assert sim.status() == 0
    assert torch.equal(out, ref_out) and torch.equal(depth.view(torch.int32),
                                                     ref_depth.view(torch.int32))
    with pytest.raises(gp.GigapixelError):
        sim.debug_stall_pipeline(out, depth, wait_ns=10)  # limit outside 1e6..2e9


def test_status_word_injection_and_nonfinite_state():
    import torch
    import paper_2606_19641_b300 as gp
    wl = wg.WORKLOADS["tiny"]
    worlds = wg.make_workload(wl)
    sim, cfg = sim_for(worlds, wl)
    act = torch.zeros((worlds.n_agents, 2), device="cuda")
    assert sim.status() == 0
    sim.inject_status(gp.binding.DEV_INJECTED)
    assert sim.status() == gp.binding.DEV_INJECTED
    with pytest.raises(gp.GigapixelError) as e:
        sim.step(act)
    assert e.value.status == gp.binding.GP_EDEVICE
    # the debug entry points refuse to launch on a sticky status too
    import ctypes
    out, depth = sim.alloc_outputs()
    n = ctypes.c_int64(-7)
    tris = np.zeros(64, gp.binding.TRI_DTYPE)
    L, h = gp.lib(), sim._h
    assert L.gp_debug_stall_pipeline(h, out.data_ptr(), None, 20_000_000, None) == gp.binding.GP_EDEVICE
    for entry in (L.gp_debug_dump_tris, L.gp_debug_dump_tris_noalloc):
        assert entry(h, 0, out.data_ptr(), depth.data_ptr(), tris.ctypes.data, 64, ctypes.byref(n),
                     None) == gp.binding.GP_EDEVICE
    assert n.value == -7
    sim.clear_status()
    sim.step(act)
    assert sim.status() == 0
    # a NaN steering angle makes a moving agent's pose non-finite: reported, never
    # trapped (a NaN acceleration alone is absorbed by the speed clamp)
    st, fl = sim.get_state()
    st[:, 3] = 5.0
    sim.set_state(st, np.zeros_like(fl))
    bad = act.clone()
    bad[0, 1] = float("nan")
    sim.step(bad)
    assert sim.status() & gp.binding.DEV_NONFINITE_STATE
    sim.clear_status()


def test_full_size_uniform_batch_sampled():
    """The full uniform batch (256 worlds x 32 agents, 128x128) in the benchmark's launch
    configuration (autotuned launch shape, graph replay): sampled views are bit-exact against
    the raster rule and within the FP64 mismatch bound; invariants hold on every view."""
    import torch
    wl = wg.WORKLOADS["uniform"]
    worlds = wg.make_workload(wl)
    sim, cfg = sim_for(worlds, wl, autotune=1)
    print("launch shape", sim.info.band_rows, sim.info.threads, sim.info.tri_capacity,
          sim.info.producer_warps)
    out, depth = sim.alloc_outputs()
    act = torch.empty((worlds.n_agents, 2), device="cuda")
    for k in range(3):
        act.copy_(torch_actions(worlds, k, wl.seed)[0])
        sim.step_render(act, out, depth)
    torch.cuda.synchronize()
    assert int(out.max()) <= 3
    assert torch.equal(out > 0, depth > 0)
    views = sample_views(worlds, sim, 256, 0)
    out_copy, depth_copy = out.clone(), depth.clone()
    S = check_views(sim, cfg, worlds, views, out, depth)
    assert_views(S, "full-size uniform")
    assert torch.equal(out, out_copy) and torch.equal(depth, depth_copy)  # re-render identical
    assert sim.status() == 0


def test_full_size_ragged_precision_sampled():
    """The full ragged precision batch (1024 worlds, agents U{1..64}, road segments
    U{100..2000}, 256x144, FP16 reversed-Z keys, BF16 one-hot NCHW) in the benchmark's
    launch configuration (autotuned launch shape, graph replay): sampled views are bit-exact
    against the raster rule and within the FP64 mismatch bound."""
    import torch
    wl = wg.WORKLOADS["ragged_precision"]
    worlds = wg.make_workload(wl)
    sim, cfg = sim_for(worlds, wl, autotune=1)
    print("launch shape", sim.info.band_rows, sim.info.threads, sim.info.tri_capacity,
          sim.info.producer_warps, "views", sim.n_views)
    out, depth = sim.alloc_outputs()
    act = torch.empty((worlds.n_agents, 2), device="cuda")
    for k in range(2):
        act.copy_(torch_actions(worlds, k, wl.seed)[0])
        sim.step_render(act, out, depth)
    torch.cuda.synchronize()
    assert sim.status() == 0
    # one-hot values are exactly +-1 (bf16 0x3F80 / 0xBF80) everywhere
    flat = out.view(torch.int16).view(-1)
    for c0 in range(0, flat.numel(), 1 << 28):
        part = flat[c0:c0 + (1 << 28)]
        assert bool(((part == 0x3F80) | (part == -0x4080)).all())
    views = sample_views(worlds, sim, 256, 1)
    S = check_views(sim, cfg, worlds, views, out, depth)
    assert_views(S, "full-size ragged precision 256x144")
    assert sim.status() == 0


def test_full_size_ragged_batch_sampled():
    """The full ragged batch (1024 worlds, agents U{1..64}, road segments U{100..2000},
    128x128, u8 class + f32 depth), autotuned, graph replay: sampled views bit-exact against
    the raster rule and within the FP64 mismatch bound."""
    import torch
    wl = wg.WORKLOADS["ragged"]
    worlds = wg.make_workload(wl)
    sim, cfg = sim_for(worlds, wl, autotune=1)
    out, depth = sim.alloc_outputs()
    act = torch.empty((worlds.n_agents, 2), device="cuda")
    for k in range(2):
        act.copy_(torch_actions(worlds, k, wl.seed)[0])
        sim.step_render(act, out, depth)
    torch.cuda.synchronize()
    assert sim.status() == 0
    assert int(out.max()) <= 3
    assert torch.equal(out > 0, depth > 0)
    views = sample_views(worlds, sim, 256, 2)
    S = check_views(sim, cfg, worlds, views, out, depth)
    assert_views(S, "full-size ragged 128x128")


@pytest.mark.parametrize("size", [64, 512])
@pytest.mark.parametrize("precision", [False, True], ids=["plain", "precision"])
def test_full_size_sweep_three_cameras_sampled(size, precision):
    """The camera and resolution sweep at full size (256 worlds x 32 agents x 3 cameras at
    0 and +-60 deg, 64 boxes and 1000 road segments per world) at the smallest and largest
    square resolution, plain and precision paths: sampled views of every camera bit-exact
    against the raster rule and within the FP64 mismatch bound."""
    import torch
    import paper_2606_19641_b300 as gp
    wl = wg.WORKLOADS["sweep"]
    worlds = wg.make_workload(wl)
    extra = dict(key_precision=gp.KEY_F16, output=gp.OUT_ONEHOT_BF16) if precision else {}
    sim, cfg = sim_for(worlds, wl, width=size, height=size, **extra)
    assert sim.n_views == 3 * worlds.n_agents
    out, depth = sim.alloc_outputs()
    act = torch.empty((worlds.n_agents, 2), device="cuda")
    for k in range(2):
        act.copy_(torch_actions(worlds, k, wl.seed)[0])
        sim.step_render(act, out, depth)
    torch.cuda.synchronize()
    assert sim.status() == 0
    views = sample_views(worlds, sim, 96 if size == 512 else 256, size)
    S = check_views(sim, cfg, worlds, views, out, depth)
    assert_views(S, "full-size sweep %dx%d %s" % (size, size, "precision" if precision else "plain"))
    del out, depth
    sim.close()
    torch.cuda.empty_cache()


# ---------------------------------------------------------------------------------------
# The paper's observation rig: 4 cameras, 210x126 / 434x252, shaded RGB
# ---------------------------------------------------------------------------------------

def check_rgb(sim, cfg, worlds, views, out, depth):
    """RGB of the GPU vs the oracle's shading of the same winners: the winning primitive
    per pixel comes from the raster rule on the GPU's own snapped triangles (bit-exact
    depth), the colour within 1 of the FP64 shading (the yaw's sin/cos and the FP32 light
    arithmetic may flip a rounding step).  Returns the fraction of channel values off by 1."""
    osim = oracle_sim(worlds, sim)
    colour = np.array(cfg.colour, np.float64).reshape(4, 3)
    light = np.array(list(cfg.light_dir), np.float64)
    off1 = total = 0
    for v in views:
        tris = dedupe(sim.dump_tris(v, out, depth))
        img = oracle_raster_of(worlds, cfg, v, tris)
        w, _, _ = view_loc(worlds, cfg, v)
        be, re = osim.prim_ranges(w)
        sp, st = osim.signals(w)
        ref = oracle.shade_rgb(img.key, bool(cfg.key_precision), be, re, osim.boxes6(w),
                               colour=colour, light=light, ambient=float(cfg.ambient),
                               line_end=osim.line_end(w), sph=sp, sph_state=st,
                               signal_colour=np.array(cfg.signal_colour, np.float64).reshape(4, 3))
        got = out[v].cpu().numpy()
        diff = np.abs(got.astype(np.int16) - ref.astype(np.int16))
        assert diff.max() <= 1, "view %d: RGB off by %d" % (v, diff.max())
        off1 += int((diff == 1).sum())
        total += diff.size
        if depth is not None:
            _, gd = gpu_view(cfg, out, depth, v)
            _, ed = expected_planes(cfg, img)
            assert np.array_equal(gd, ed), "view %d: depth bits differ" % v
    return off1 / total


@pytest.mark.parametrize("size", [(210, 126), (434, 252)])
@pytest.mark.parametrize("key", ["f16", "f32"])
def test_paper_rig_rgb(size, key):
    import torch
    import paper_2606_19641_b300 as gp
    name = "paper_rig_%dx%d" % size
    wl = wg.WORKLOADS[name]
    worlds = wg.make_workload(wl, n_worlds=2)
    sim, cfg = sim_for(worlds, wl, key_precision=gp.KEY_F16 if key == "f16" else gp.KEY_F32)
    assert sim.n_views == 4 * worlds.n_agents
    out, depth = sim.alloc_outputs()
    assert out.shape == (sim.n_views, 3, size[1], size[0]) and out.dtype == torch.uint8
    act = torch.empty((worlds.n_agents, 2), device="cuda")
    for k in range(3):
        act.copy_(torch_actions(worlds, k, wl.seed)[0])
        sim.step_render(act, out, depth)
    torch.cuda.synchronize()
    assert sim.status() == 0
    views = [0, 1, 2, 3, 4 * 7 + 3, 4 * 33 + 1, sim.n_views - 1]
    frac = check_rgb(sim, cfg, worlds, views, out, depth)
    print("paper rig %s %s: %.2e of channel values off by one" % (name, key, frac))
    assert frac < 1e-3
    # every class colour appears, shaded boxes differ by face
    assert int(out[:, 2].float().mean()) > 0
    # the rig's geometry (four cameras, signal spheres) against the FP64 oracle, both ways
    S = check_views(sim, cfg, worlds, views, out, depth, t3=False, t4=False)
    assert_views(S, "paper rig %s %s T2" % (name, key), min_covered=0.05)
    assert S["o_vis"] > 500


def test_binding_checks_tensor_layouts():
    """Tensors of the wrong dtype, size or strides are refused before any launch, and the
    simulator keeps working afterwards."""
    import torch
    import paper_2606_19641_b300 as gp
    wl = wg.WORKLOADS["tiny"]
    worlds = wg.make_workload(wl)
    sim, cfg = sim_for(worlds, wl)
    out, depth = sim.alloc_outputs()
    act = torch_actions(worlds, 0, wl.seed)[0]
    bad = [
        (act.double(), out, depth),                      # actions dtype
        (act[:-1], out, depth),                          # short actions
        (act.t().contiguous().t(), out, depth),          # actions not contiguous
        (act, out.float(), depth),                       # class image dtype
        (act, out[:-1], depth),                          # one view short
        (act, out, depth.half()),                        # depth dtype for FP32 keys
        (act, out, depth.transpose(1, 2)),               # depth not contiguous
    ]
    for a, o, d in bad:
        with pytest.raises(gp.GigapixelError) as e:
            sim.step_render(a, o, d)
        assert e.value.status == gp.binding.GP_EINVAL
    with pytest.raises(gp.GigapixelError):
        sim.observe_vec(out=(torch.empty((sim.n_agents, 16, 8), device="cuda"),
                             torch.empty((sim.n_agents, 31, 8), device="cuda"),
                             torch.empty((sim.n_agents, 4, 8), device="cuda")))
    sim.step_render(act, out, depth)
    torch.cuda.synchronize()
    assert sim.status() == 0
    check_t3(sim, cfg, worlds, [0, sim.n_views - 1], out, depth)


def test_library_refuses_unreachable_pointers():
    """Through the C ABI itself (no binding checks): a pageable host buffer handed to the
    step, render, trace and O_vec calls returns GP_EINVAL before any launch.  The runtime is
    first asked how it classifies the buffer; the calls are only made if it reports
    unregistered host memory, which the library refuses."""
    import torch
    from cuda.bindings import runtime as rt
    import paper_2606_19641_b300 as gp
    wl = wg.WORKLOADS["tiny"]
    worlds = wg.make_workload(wl)
    sim, cfg = sim_for(worlds, wl)
    host = np.zeros(16 << 20, np.uint8)  # larger than any output of this workload
    err, attr = rt.cudaPointerGetAttributes(host.ctypes.data)
    assert err == rt.cudaError_t.cudaSuccess
    assert attr.type == rt.cudaMemoryType.cudaMemoryTypeUnregistered
    out, depth = sim.alloc_outputs()
    act = torch_actions(worlds, 0, wl.seed)[0]
    L, h, hp = gp.lib(), sim._h, host.ctypes.data
    assert L.gp_step(h, hp, None) == gp.binding.GP_EINVAL
    assert L.gp_step_world(h, 0, hp, None) == gp.binding.GP_EINVAL
    assert L.gp_render(h, hp, depth.data_ptr(), None) == gp.binding.GP_EINVAL
    assert L.gp_render(h, out.data_ptr(), hp, None) == gp.binding.GP_EINVAL
    assert L.gp_render_world(h, 0, hp, None, None) == gp.binding.GP_EINVAL
    assert L.gp_trace(h, hp, None, None) == gp.binding.GP_EINVAL
    assert L.gp_step_render(h, act.data_ptr(), hp, None, None) == gp.binding.GP_EINVAL
    assert L.gp_step_trace(h, hp, out.data_ptr(), None, None) == gp.binding.GP_EINVAL
    assert "pageable host memory" in L.gp_last_error().decode()
    assert L.gp_observe_vec(h, hp, None, None, None) == gp.binding.GP_EINVAL
    # the debug entry points run the same checks before their launch
    import ctypes
    n = ctypes.c_int64(-7)
    tris = np.zeros(64, gp.binding.TRI_DTYPE)
    assert L.gp_debug_stall_pipeline(h, hp, None, 20_000_000, None) == gp.binding.GP_EINVAL
    assert L.gp_debug_stall_pipeline(h, out.data_ptr(), hp, 20_000_000, None) == gp.binding.GP_EINVAL
    for entry in (L.gp_debug_dump_tris, L.gp_debug_dump_tris_noalloc):
        assert entry(h, 0, hp, None, tris.ctypes.data, 64, ctypes.byref(n), None) == gp.binding.GP_EINVAL
        assert entry(h, 0, out.data_ptr(), hp, tris.ctypes.data, 64, ctypes.byref(n), None) == \
            gp.binding.GP_EINVAL
        assert "pageable host memory" in L.gp_last_error().decode()
    assert n.value == -7  # refused before anything was written
    sim.step_render(act, out, depth)
    torch.cuda.synchronize()
    assert sim.status() == 0
    check_t3(sim, cfg, worlds, [0], out, depth)


def test_rgb_rejects_bad_appearance():
    import paper_2606_19641_b300 as gp
    wl = wg.WORKLOADS["paper_rig_210x126"]
    worlds = wg.make_workload(wl, n_worlds=1)
    with pytest.raises(gp.GigapixelError):
        sim_for(worlds, wl, light_dir=(0.0, 0.0, 0.0))
    with pytest.raises(gp.GigapixelError):
        sim_for(worlds, wl, ambient=1.5)
    with pytest.raises(gp.GigapixelError):
        sim_for(worlds, wl, width=211)  # odd widths are rejected


# ---------------------------------------------------------------------------------------
# Rewards and ego state (App. A reward table and observations)
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("name,n_worlds,steps", [("uniform", 4, 12), ("ragged", 6, 10),
                                                 ("paper_rig_210x126", 3, 12)])
def test_rewards_match_oracle(name, n_worlds, steps):
    """Per-step rewards and ego states against the oracle evaluated on the GPU's own
    before/after states and flags; random per-agent weights from the table's ranges.  The
    signal worlds hang 32 red signals per world so that the red-light term fires."""
    import torch
    wl = wg.WORKLOADS[name]
    worlds = wg.make_workload(wl, n_worlds=n_worlds)
    if wl.signals:
        wg.add_signals(worlds, 32, wl.seed, height=5.0)
        worlds.signal_state[:] = 0
    sim, cfg = sim_for(worlds, wl, rewards=1)
    red_fired = 0
    na = worlds.n_agents
    rng = np.random.default_rng(5)
    lo = np.array([0, 0, 0, 2.5e-4, 2.5e-4, 0, 0, 0, 2.5e-4, 0])
    hi = np.array([3, 3, 0.05, 2.5e-2, 7.5e-3, 5e-3, 1, 5e-5, 7.5e-3, 1])
    weights = (lo + (hi - lo) * rng.random((na, 10))).astype(np.float32)
    sim.set_reward_weights(weights)
    off = worlds.agent_offsets()
    acc = np.zeros((na, 2), np.float64)
    dims = np.zeros((na, 2), np.float64)
    for w in range(worlds.n_worlds):
        b0 = int(worlds.box_off[w])
        a0, a1 = int(off[w]), int(off[w + 1])
        dims[a0:a1] = worlds.boxes[b0:b0 + (a1 - a0), 3:5]
    n_bad = n_total = 0
    seen_collision = False
    for k in range(steps):
        st0, fl0 = sim.get_state()
        act_t, act = torch_actions(worlds, k, wl.seed)
        sim.step(act_t)
        st1, fl1 = sim.get_state()
        r, e = sim.rewards()
        torch.cuda.synchronize()
        r, e = r.cpu().numpy(), e.cpu().numpy()
        for w in range(worlds.n_worlds):
            a0, a1 = int(off[w]), int(off[w + 1])
            road = worlds.road[int(worlds.road_off[w]):int(worlds.road_off[w + 1])]
            s0, s1 = int(worlds.signal_off[w]), int(worlds.signal_off[w + 1])
            sph, sst = worlds.signal[s0:s1], worlds.signal_state[s0:s1]
            acc_w = np.ascontiguousarray(acc[a0:a1])
            acc_g = acc_w.copy()
            rr, ee = oracle.rewards_world(st0[a0:a1], fl0[a0:a1], st1[a0:a1], fl1[a0:a1],
                                          act[a0:a1], dims[a0:a1], acc_w, weights[a0:a1], road,
                                          sph=sph, sph_state=sst)
            if s1 > s0:
                rg, _ = oracle.rewards_world(st0[a0:a1], fl0[a0:a1], st1[a0:a1], fl1[a0:a1],
                                             act[a0:a1], dims[a0:a1], acc_g, weights[a0:a1], road,
                                             sph=sph, sph_state=np.full(s1 - s0, 2, np.uint8))
                red_fired += int((np.abs(rg - rr) > 0).sum())
            acc[a0:a1] = acc_w
            d = np.abs(r[a0:a1] - rr)
            n_bad += int((d > 1e-4 + 1e-4 * np.abs(rr)).sum())
            n_total += a1 - a0
            # the only admissible larger difference: one comfort indicator flipped at its
            # threshold by FP32 rounding of the acceleration
            assert np.all((d <= 1e-4 + 1e-4 * np.abs(rr)) | (d <= weights[a0:a1, 2] + 1e-4))
            assert np.allclose(e[a0:a1], ee, atol=2e-5)
            seen_collision |= bool((fl1[a0:a1] & 1).any())
    assert n_bad <= 0.005 * n_total
    assert sim.status() == 0
    if wl.signals:
        print("red-light violations in the oracle: %d" % red_fired)
        assert red_fired > 0


def test_rewards_off_by_default_and_weights_validated():
    import paper_2606_19641_b300 as gp
    wl = wg.WORKLOADS["tiny"]
    worlds = wg.make_workload(wl)
    sim, _ = sim_for(worlds, wl)
    with pytest.raises(gp.GigapixelError) as e:
        sim.rewards()
    assert e.value.status == gp.binding.GP_ESTATE
    sim2, _ = sim_for(worlds, wl, rewards=1)
    bad = np.ones((worlds.n_agents, 10), np.float32)
    bad[0, 3] = np.nan
    with pytest.raises(gp.GigapixelError):
        sim2.set_reward_weights(bad)


# ---------------------------------------------------------------------------------------
# Ray-traced backend
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("name,n_worlds,output", [("tiny", 1, "class"), ("uniform", 2, "class"),
                                                  ("paper_rig_210x126", 1, "rgb")])
def test_trace_matches_oracle(name, n_worlds, output):
    """GPU ray tracing (FP32) against the oracle's FP64 ray tracer from the same state: the
    hit object agrees except on rays that graze an edge (< 0.1 % of pixels), depth within
    FP32 rounding, RGB within 1 where the hit agrees."""
    import torch
    import paper_2606_19641_b300 as gp
    wl = wg.WORKLOADS[name]
    worlds = wg.make_workload(wl, n_worlds=n_worlds)
    extra = {} if output == "rgb" else dict(key_precision=gp.KEY_F32)
    sim, cfg = sim_for(worlds, wl, **extra)
    out, depth = sim.alloc_outputs()
    for k in range(2):
        sim.step(torch_actions(worlds, k, wl.seed)[0])
    sim.trace(out, depth)
    torch.cuda.synchronize()
    assert sim.status() == 0
    osim = oracle_sim(worlds, sim)
    cam = cam_config(cfg)
    views = list(range(0, sim.n_views, max(1, sim.n_views // 10)))
    mism = total = 0
    key_f16 = bool(cfg.key_precision)
    for v in views:
        w, a, c = view_loc(worlds, cfg, v)
        tr = osim.trace(cam, w, a, float(np.float32(cfg.cam_yaw[c])))
        go, gd = gpu_view(cfg, out, depth, v)
        if output == "rgb":
            be, re = osim.prim_ranges(w)
            sp, st = osim.signals(w)
            ref = oracle.shade_rgb(tr.key(key_f16), key_f16, be, re, osim.boxes6(w),
                                   colour=np.array(cfg.colour, np.float64).reshape(4, 3),
                                   light=np.array(list(cfg.light_dir)), ambient=float(cfg.ambient),
                                   line_end=osim.line_end(w), sph=sp, sph_state=st)
            diff = np.abs(go.astype(np.int16) - ref.astype(np.int16)).max(axis=0)
            bad = diff > 1
            gcls_hit = gd != 0
        else:
            bad = go != tr.cls
            gcls_hit = go != 0
        mism += int(bad.sum())
        total += bad.size
        # depth where both hit the same class
        both = ~bad & gcls_hit & (tr.cls != 0)
        if key_f16:
            gdv = gd.view(np.float16).astype(np.float32)
            assert np.allclose(gdv[both], tr.depth[both], rtol=2e-3)
        else:
            gdv = gd.view(np.float32)
            assert np.allclose(gdv[both], tr.depth[both], rtol=2e-5)
    print("trace %s: %d of %d pixels differ" % (name, mism, total))
    assert mism <= 1e-3 * total


def test_full_size_uniform_trace_sampled():
    """The full uniform batch (256 worlds x 32 agents, 128x128, class + FP32 depth) ray
    traced in the benchmark's launch configuration (step + trace replayed from one graph):
    sampled views agree with the oracle's FP64 ray tracer except on grazing rays; every view
    keeps the class/depth invariants."""
    import torch
    import paper_2606_19641_b300 as gp
    wl = wg.WORKLOADS["uniform"]
    worlds = wg.make_workload(wl)
    sim, cfg = sim_for(worlds, wl, autotune=1, key_precision=gp.KEY_F32)
    out, depth = sim.alloc_outputs()
    act = torch.empty((worlds.n_agents, 2), device="cuda")
    for k in range(3):
        act.copy_(torch_actions(worlds, k, wl.seed)[0])
        sim.step_trace(act, out, depth)
    torch.cuda.synchronize()
    assert sim.status() == 0
    assert int(out.max()) <= 3
    assert torch.equal(out > 0, depth > 0)
    osim = oracle_sim(worlds, sim)
    cam = cam_config(cfg)
    rng = np.random.default_rng(5)
    views = sorted(rng.choice(sim.n_views, 4, replace=False).tolist())
    mism = total = 0
    for v in views:
        w, a, c = view_loc(worlds, cfg, v)
        tr = osim.trace(cam, w, a, float(np.float32(cfg.cam_yaw[c])))
        go, gd = gpu_view(cfg, out, depth, v)
        bad = go != tr.cls
        mism += int(bad.sum())
        total += bad.size
        both = ~bad & (go != 0)
        assert np.allclose(gd.view(np.float32)[both], tr.depth[both], rtol=2e-5)
    print("trace uniform full size: %d of %d pixels differ" % (mism, total))
    assert mism <= 1e-3 * total



def test_trace_and_raster_agree_away_from_silhouettes():
    """Both backends render the same scene: they may differ only along edges."""
    import torch
    wl = wg.WORKLOADS["uniform"]
    worlds = wg.make_workload(wl, n_worlds=2)
    sim, cfg = sim_for(worlds, wl)
    o1, d1 = sim.alloc_outputs()
    o2, d2 = sim.alloc_outputs()
    sim.render(o1, d1)
    sim.trace(o2, d2)
    torch.cuda.synchronize()
    agree = (o1 == o2).float().mean().item()
    print("raster vs trace class agreement %.4f" % agree)
    assert agree > 0.97


# ---------------------------------------------------------------------------------------
# Vectorized observations O_vec
# ---------------------------------------------------------------------------------------

def _sure_limit(d, cap, radius, eps):
    """(limit, tied): the selection of candidates nearer than limit cannot depend on
    rounding.  tied if a candidate lies within eps of the radius, or the cap-th and the next
    nearest (when more than cap are in range) are within eps of each other; else limit is
    infinite (the whole selection is determined)."""
    limit, tied = np.inf, False
    if np.any(np.abs(d - radius) < eps):
        limit, tied = radius - eps, True
    ds = np.sort(d[d <= radius])
    if len(ds) > cap and ds[cap] - ds[cap - 1] < eps:
        limit, tied = min(limit, ds[cap - 1] - eps), True
    return limit, tied


def _rows(x, scale, limit):
    """Valid slots nearer than limit (near-equal distances may order differently in FP32
    and FP64, so they are compared as sets with _same_rows)."""
    v = x[x[:, 0] > 0]
    return v[np.hypot(v[:, 1], v[:, 2]) * scale < limit]


def _same_rows(a, b, atol):
    """a and b hold the same rows up to atol, in any order (a one-to-one matching)."""
    if a.shape != b.shape:
        return False
    used = np.zeros(len(b), bool)
    for r in a:
        hit = np.flatnonzero(~used & np.all(np.abs(b - r) <= atol, axis=1))
        if len(hit) == 0:
            return False
        used[hit[0]] = True
    return True


@pytest.mark.parametrize("name,n_worlds", [("uniform", 3), ("ragged", 4), ("paper_rig_210x126", 3)])
def test_observe_vec_matches_oracle(name, n_worlds):
    import torch
    wl = wg.WORKLOADS[name]
    worlds = wg.make_workload(wl, n_worlds=n_worlds)
    if wl.signals:
        wg.add_signals(worlds, 24, wl.seed, height=5.0)  # denser: more than 4 in range
    sim, cfg = sim_for(worlds, wl)
    for k in range(3):
        sim.step(torch_actions(worlds, k, wl.seed)[0])
    ga, gr, gs = sim.observe_vec()
    torch.cuda.synchronize()
    ga, gr, gs = ga.cpu().numpy(), gr.cpu().numpy(), gs.cpu().numpy()
    st, fl = sim.get_state()
    osim = oracle_sim(worlds, sim)
    off = worlds.agent_offsets()
    checked = skipped = 0
    compared_rows = [0]
    for w in range(worlds.n_worlds):
        a0, a1 = int(off[w]), int(off[w + 1])
        b = osim.boxes6(w)
        sp = np.zeros(len(b))
        sp[:a1 - a0] = st[a0:a1, 3]
        road, line = osim.road(w), osim.line(w)
        oa, orr = oracle.observe_world(b, sp, road, line, n_agents=a1 - a0)
        sph, sst = osim.signals(w)
        osg = oracle.observe_signals(b, a1 - a0, sph, sst)
        for i in range(a1 - a0):
            ds = np.hypot(sph[:, 0] - b[i, 0], sph[:, 1] - b[i, 1])
            ls, _ = _sure_limit(ds, 4, 50.0, 1e-3)
            ra, rb = _rows(gs[a0 + i], 50.0, ls), _rows(osg[i], 50.0, ls)
            assert _same_rows(ra, rb, 2e-5), "signals, agent %d" % (a0 + i)
            compared_rows[0] += len(ra)
        if wl.signals:
            assert (gs[a0:a1, :, 0] > 0).sum() > 2 * (a1 - a0)
        else:
            assert not gs[a0:a1].any()
        segs = np.concatenate([road, line]).astype(np.float64).reshape(-1, 4, 2)
        mid = 0.25 * (segs[:, 0] + segs[:, 3] + segs[:, 1] + segs[:, 2])
        for i in range(a1 - a0):
            db = np.delete(np.hypot(b[:, 0] - b[i, 0], b[:, 1] - b[i, 1]), i)
            dm = np.hypot(mid[:, 0] - b[i, 0], mid[:, 1] - b[i, 1])
            (la, ta), (lr, tr) = _sure_limit(db, 16, 100.0, 1e-3), _sure_limit(dm, 32, 30.0, 1e-3)
            full = not (ta or tr)
            checked += int(full)
            skipped += int(not full)
            for g, o, scale, lim in ((ga[a0 + i], oa[i], 100.0, la), (gr[a0 + i], orr[i], 30.0, lr)):
                ra, rb = _rows(g, scale, lim), _rows(o, scale, lim)
                assert _same_rows(ra, rb, 2e-5), "agent %d" % (a0 + i)
                compared_rows[0] += len(ra)
                # nearest first: the GPU's slot distances are non-decreasing
                v = g[g[:, 0] > 0]
                assert np.all(np.diff(np.hypot(v[:, 1], v[:, 2]) * scale) >= -1e-3)
    print("O_vec %s: %d agents fully checked, %d up to a near-tie at the cutoff, %d slots compared"
          % (name, checked, skipped, compared_rows[0]))
    assert checked > 0.5 * (checked + skipped)
    assert compared_rows[0] > 1000


# ---------------------------------------------------------------------------------------
# Jerk-actuated dynamics (App. A "Action Space and Dynamics")
# ---------------------------------------------------------------------------------------

def _jerk_actions(n, step, seed):
    return wg.jerk_actions(seed, step, n)


@pytest.mark.parametrize("name,n_worlds,steps", [("tiny", 1, 15), ("uniform", 4, 25),
                                                 ("ragged", 6, 20)])
def test_jerk_dynamics_match_oracle(name, n_worlds, steps):
    """One GPU step against one oracle step from the same pose, flags and actuator state;
    rewards and the ego extras against the oracle on the resolved controls."""
    import torch
    import paper_2606_19641_b300 as gp
    wl = wg.WORKLOADS[name]
    worlds = wg.make_workload(wl, n_worlds=n_worlds)
    sim, cfg = sim_for(worlds, wl, dynamics=gp.DYN_JERK, rewards=1)
    na = worlds.n_agents
    off = worlds.agent_offsets()
    dims = np.zeros((na, 2), np.float64)
    for w in range(worlds.n_worlds):
        b0 = int(worlds.box_off[w])
        dims[off[w]:off[w + 1]] = worlds.boxes[b0:b0 + (off[w + 1] - off[w]), 3:5]
    acc = np.zeros((na, 2), np.float64)
    saw_clip = saw_rate = False
    for k in range(steps):
        st0, fl0 = sim.get_state()
        dy0 = sim.get_dynamics()
        osim = oracle.Sim(worlds, jerk_dynamics=True)
        osim.set_state(st0.astype(np.float64), fl0, dy0.astype(np.float64))
        act = _jerk_actions(na, k, wl.seed)
        sim.step(torch.from_numpy(act).cuda())
        osim.step(act)
        st1, fl1 = sim.get_state()
        dy1 = sim.get_dynamics()
        assert np.allclose(dy1, osim.jerk, atol=2e-5, rtol=0), "actuator state, step %d" % k
        assert np.allclose(st1[:, 0:2], osim.state[:, 0:2], atol=2e-4, rtol=0)
        dyaw = np.angle(np.exp(1j * (st1[:, 2].astype(np.float64) - osim.state[:, 2])))
        assert np.all(np.abs(dyaw) < 2e-5)
        assert np.allclose(st1[:, 3], osim.state[:, 3], atol=2e-5)
        assert np.array_equal(fl1, osim.flags), "flags differ at step %d" % k
        saw_clip |= bool((np.abs(dy1[:, 0] - 3.0) < 1e-6).any() or (np.abs(dy1[:, 0] + 5.0) < 1e-6).any())
        saw_rate |= bool((np.abs(np.abs(dy1[:, 2] - dy0[:, 2]) - 0.05) < 1e-6).any())
        # rewards / ego on the controls the actuator resolved (a_lon, steer)
        r, e = sim.rewards()
        torch.cuda.synchronize()
        r, e = r.cpu().numpy(), e.cpu().numpy()
        ctrl = np.stack([dy1[:, 0], dy1[:, 2]], 1).astype(np.float32)
        for w in range(worlds.n_worlds):
            a0, a1 = int(off[w]), int(off[w + 1])
            road = worlds.road[int(worlds.road_off[w]):int(worlds.road_off[w + 1])]
            acc_w = np.ascontiguousarray(acc[a0:a1])
            rr, ee = oracle.rewards_world(st0[a0:a1], fl0[a0:a1], st1[a0:a1], fl1[a0:a1],
                                          ctrl[a0:a1], dims[a0:a1], acc_w,
                                          np.tile(oracle.REWARD_WEIGHTS, (a1 - a0, 1)), road,
                                          jerk=dy1[a0:a1])
            acc[a0:a1] = acc_w
            assert np.allclose(e[a0:a1], ee, atol=3e-5)
            d = np.abs(r[a0:a1] - rr)
            assert np.all((d <= 1e-4 + 1e-4 * np.abs(rr)) | (d <= oracle.REWARD_WEIGHTS[2] + 1e-4))
    assert saw_clip and saw_rate  # the limits were exercised
    assert sim.status() == 0


def test_jerk_state_fork_and_reset():
    """get/set of pose + actuator state replays a rollout exactly; set_state zeroes the
    actuators; the calls are refused under direct control."""
    import torch
    import paper_2606_19641_b300 as gp
    wl = wg.WORKLOADS["uniform"]
    worlds = wg.make_workload(wl, n_worlds=3)
    sim, _ = sim_for(worlds, wl, dynamics=gp.DYN_JERK)
    na = worlds.n_agents
    for k in range(5):
        sim.step(torch.from_numpy(_jerk_actions(na, k, 7)).cuda())
    snap = sim.get_state(), sim.get_dynamics()
    assert np.abs(snap[1]).max() > 0.1
    outs = []
    for _ in range(2):
        sim.set_state(*snap[0])
        assert np.all(sim.get_dynamics() == 0.0)
        sim.set_dynamics(snap[1])
        for k in range(5, 10):
            sim.step(torch.from_numpy(_jerk_actions(na, k, 7)).cuda())
        outs.append((sim.get_state()[0], sim.get_dynamics()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    bad = snap[1].copy()
    bad[0, 0] = np.nan
    with pytest.raises(gp.GigapixelError):
        sim.set_dynamics(bad)
    direct, _ = sim_for(worlds, wl)
    with pytest.raises(gp.GigapixelError) as e:
        direct.get_dynamics()
    assert e.value.status == gp.binding.GP_ESTATE


# ---------------------------------------------------------------------------------------
# Traffic-signal spheres (the third primitive): raster tiers, trace, states
# ---------------------------------------------------------------------------------------

def _signal_worlds(n_worlds=2, per_world=12):
    """Uniform worlds with large, low signal spheres (3 m up, 1 m radius): many covered
    pixels per view."""
    wl = wg.WORKLOADS["uniform"]
    worlds = wg.make_workload(wl, n_worlds=n_worlds)
    wg.add_signals(worlds, per_world, 77, height=3.0, radius=1.0)
    return wl, worlds


def _signal_views(sim, cfg, out, n=8):
    import torch
    cls = out if int(cfg.output) == 0 else None
    if cls is None:
        return list(range(0, sim.n_views, max(1, sim.n_views // n)))
    counts = (cls == 4).flatten(1).sum(1).cpu().numpy()
    order = np.argsort(-counts, kind="stable")
    return [int(v) for v in order[:n] if counts[v] > 0]


@pytest.mark.parametrize("shape,precision", [(dict(), False), (dict(producer_warps=4), False),
                                             (dict(), True)],
                         ids=["default", "pipelined", "precision"])
def test_signal_spheres_raster(shape, precision):
    """T3 bit-exact on the views with the most signal pixels, T2 on the signal triangles,
    T4 against the FP64 pipeline."""
    import torch
    import paper_2606_19641_b300 as gp
    wl, worlds = _signal_worlds()
    extra = dict(key_precision=gp.KEY_F16, output=gp.OUT_ONEHOT_BF16) if precision else {}
    sim, cfg = sim_for(worlds, wl, **shape, **extra)
    assert sim.n_signals == 24
    out, depth = sim.alloc_outputs()
    sim.step(torch_actions(worlds, 0, wl.seed)[0])
    sim.render(out, depth)
    torch.cuda.synchronize()
    assert sim.status() == 0
    if precision:
        views = list(range(0, sim.n_views, 4))
        ref, _ = sim_for(worlds, wl, **shape)
        o2, d2 = ref.alloc_outputs()
        ref.step(torch_actions(worlds, 0, wl.seed)[0])
        ref.render(o2, d2)
        torch.cuda.synchronize()
        views = _signal_views(ref, ref.config, o2)
    else:
        views = _signal_views(sim, cfg, out)
        assert len(views) >= 4 and int((out == 4).sum()) > 500
    check_t3(sim, cfg, worlds, views, out, depth)
    frac, derr = t4_stats(sim, cfg, worlds, views, out, depth)
    print("signals T4: class mismatch %.2e, depth p99 %.2e" % (frac, np.percentile(derr, 99)))
    assert frac < T4_MISMATCH
    # T2 on the signal triangles
    osim = oracle_sim(worlds, sim)
    cam = cam_config(cfg)
    n_vis = n_found = worst = 0
    for v in views:
        g = dedupe(sim.dump_tris(v, out, depth))
        w, a, c = view_loc(worlds, cfg, v)
        o = osim.camera_tris(cam, w, a, float(np.float32(cfg.cam_yaw[c])))
        le = osim.line_end(w)
        gmap = {(int(t["prim"]), int(t["sub"])): t for t in g}
        be, re = osim.prim_ranges(w)
        for t in o[o["prim"] >= le]:
            one = np.zeros(1, oracle.TRI_DTYPE)
            one[0] = t
            if not oracle.raster(one, cam.width, cam.height, False, be, re, line_end=le).key.any():
                continue
            n_vis += 1
            gt = gmap.get((int(t["prim"]), int(t["sub"])))
            if gt is None:
                continue
            n_found += 1
            worst = max(worst, int(np.abs(gt["X"].astype(np.int64) - t["X"]).max()),
                        int(np.abs(gt["Y"].astype(np.int64) - t["Y"]).max()))
    print("signals T2: %d visible, %d found, worst %d units" % (n_vis, n_found, worst))
    assert n_vis > 50 and n_found >= 0.995 * n_vis and worst <= 1


def test_signal_spheres_trace_and_states():
    """Ray-traced signals against the oracle's ray tracer; the raster and the tracer agree
    away from silhouettes; a state change recolours only the signals (RGB parity)."""
    import torch
    import paper_2606_19641_b300 as gp
    wl, worlds = _signal_worlds()
    sim, cfg = sim_for(worlds, wl)
    out, depth = sim.alloc_outputs()
    o2, d2 = sim.alloc_outputs()
    sim.render(out, depth)
    sim.trace(o2, d2)
    torch.cuda.synchronize()
    views = _signal_views(sim, cfg, out)
    osim = oracle_sim(worlds, sim)
    cam = cam_config(cfg)
    mism = total = sig = 0
    for v in views:
        w, a, c = view_loc(worlds, cfg, v)
        tr = osim.trace(cam, w, a, float(np.float32(cfg.cam_yaw[c])))
        go = o2[v].cpu().numpy()
        mism += int((go != tr.cls).sum())
        total += go.size
        sig += int((tr.cls == 4).sum())
    print("signals trace: %d of %d pixels differ (%d signal pixels)" % (mism, total, sig))
    assert sig > 1000 and mism <= 1e-3 * total
    agree = (out[views] == o2[views]).float().mean().item()
    assert agree > 0.97
    # RGB: states set from the host, shading against the oracle
    rgb_sim, rgb_cfg = sim_for(worlds, wl, output=gp.OUT_RGB_U8)
    states = (np.arange(sim.n_signals) % 4).astype(np.uint8)
    rgb_sim.set_signal_states(states)
    worlds.signal_state[:] = states
    ro, rd = rgb_sim.alloc_outputs()
    rgb_sim.render(ro, rd)
    torch.cuda.synchronize()
    frac = check_rgb(rgb_sim, rgb_cfg, worlds, views[:4], ro, rd)
    assert frac < 1e-3
    with pytest.raises(gp.GigapixelError):
        rgb_sim.set_signal_states(np.full(sim.n_signals, 4, np.uint8))


def test_signal_limits_validated():
    import paper_2606_19641_b300 as gp
    wl, worlds = _signal_worlds(n_worlds=1, per_world=33)
    with pytest.raises(gp.GigapixelError) as e:
        sim_for(worlds, wl)
    assert e.value.status == gp.binding.GP_ELIMIT
    wl, worlds = _signal_worlds(n_worlds=1, per_world=2)
    worlds.signal[0, 3] = 0.0
    with pytest.raises(gp.GigapixelError):
        sim_for(worlds, wl)


def test_reset_worlds():
    """Episode reset: the selected worlds' agents get their initial state back exactly
    (pose, speed, clear flags, zero actuator state); the others are untouched."""
    import torch
    import paper_2606_19641_b300 as gp
    wl = wg.WORKLOADS["uniform"]
    worlds = wg.make_workload(wl, n_worlds=3)
    sim, _ = sim_for(worlds, wl, dynamics=gp.DYN_JERK)
    na = worlds.n_agents
    st_init, fl_init = sim.get_state()
    off = worlds.agent_offsets()
    # the initial state is the descriptor's
    for w in range(3):
        b0, a0, a1 = int(worlds.box_off[w]), int(off[w]), int(off[w + 1])
        bx = worlds.boxes[b0:b0 + (a1 - a0)]
        assert np.array_equal(st_init[a0:a1, :3], bx[:, :3]) and np.array_equal(st_init[a0:a1, 3], bx[:, 6])
    for k in range(8):
        sim.step(torch.from_numpy(wg.jerk_actions(3, k, na)).cuda())
    st1, fl1 = sim.get_state()
    dy1 = sim.get_dynamics()
    assert not np.array_equal(st1, st_init) and np.abs(dy1).max() > 0
    sim.reset_worlds(np.array([0, 1, 0], np.uint8))
    st2, fl2 = sim.get_state()
    dy2 = sim.get_dynamics()
    a0, a1 = int(off[1]), int(off[2])
    assert np.array_equal(st2[a0:a1], st_init[a0:a1]) and not fl2[a0:a1].any()
    assert not dy2[a0:a1].any()
    keep = np.ones(na, bool)
    keep[a0:a1] = False
    assert np.array_equal(st2[keep], st1[keep]) and np.array_equal(fl2[keep], fl1[keep])
    assert np.array_equal(dy2[keep], dy1[keep])
    # device mask, every world
    sim.reset_worlds(torch.ones(3, dtype=torch.uint8, device="cuda"))
    torch.cuda.synchronize()
    st3, fl3 = sim.get_state()
    assert np.array_equal(st3, st_init) and not fl3.any() and not sim.get_dynamics().any()
    sim.reset_worlds()
    assert sim.status() == 0


@pytest.mark.parametrize("shape", [dict(), dict(producer_warps=2)], ids=["default", "pipelined"])
def test_render_stats_counters(shape):
    """GP_STAT_* counters of one render against what the GPU's own triangles imply: one item
    per (view, band), the kept triangles equal the records rasterised, and the fragments
    equal the covered (triangle, pixel) pairs of the raster rule."""
    import torch
    import paper_2606_19641_b300 as gp
    wl = wg.WORKLOADS["tiny"]
    worlds = wg.make_workload(wl)
    sim, cfg = sim_for(worlds, wl, stats=1, **shape)
    out, depth = sim.alloc_outputs()
    sim.render_stats(reset=True)
    sim.render(out, depth)
    st = sim.render_stats(reset=True)
    bands = -(-int(cfg.height) // int(sim.info.band_rows))
    assert st["items"] == sim.n_views * bands
    n_rec = frags = 0
    be = 12 * int(worlds.box_off[1])
    re = be + 2 * int(worlds.road_off[1])
    for v in range(sim.n_views):
        tris = sim.dump_tris(v, out, depth)
        n_rec += len(tris)
        for t in dedupe(tris):
            one = np.zeros(1, oracle.TRI_DTYPE)
            for k in ("X", "Y", "d", "prim", "sub"):
                one[k] = t[k]
            frags += int((oracle.raster(one, int(cfg.width), int(cfg.height), False, be, re).key != 0).sum())
    print("render stats:", st)
    assert st["tris_kept"] + st["tris_from_clip"] == n_rec
    assert st["fragments"] == frags
    assert st["row_items"] >= st["tris_kept"] and st["batches"] >= 1 and st["quads"] > 0
    direct, _ = sim_for(worlds, wl)
    with pytest.raises(gp.GigapixelError) as e:
        direct.render_stats()
    assert e.value.status == gp.binding.GP_ESTATE


def test_step_trace_graph_matches_direct_calls():
    """The step + ray-tracing graph gives the same images and states as the direct calls,
    and shares the graph cache with the raster graph."""
    import torch
    wl = wg.WORKLOADS["paper_rig_210x126"]
    worlds = wg.make_workload(wl, n_worlds=2)
    a, cfg = sim_for(worlds, wl)
    b, _ = sim_for(worlds, wl)
    oa, da = a.alloc_outputs()
    ob, db = b.alloc_outputs()
    oc, dc = b.alloc_outputs()
    act = torch.empty((worlds.n_agents, 2), device="cuda")
    for k in range(3):
        act.copy_(torch_actions(worlds, k, wl.seed)[0])
        a.step(act)
        a.trace(oa, da)
        b.step_trace(act, ob, db)
        torch.cuda.synchronize()
        assert torch.equal(oa, ob) and torch.equal(da.view(torch.int16), db.view(torch.int16))
    # both graph kinds on the same pointers are distinct cache entries
    a.step(act)
    a.render(oa, da)
    b.step_render(act, oc, dc)
    torch.cuda.synchronize()
    assert torch.equal(oa, oc)
    assert np.array_equal(a.get_state()[0], b.get_state()[0])


def test_fixed_length_episodes():
    """episode_steps: every world returns to its start with the done flag after exactly that
    many steps, matching the oracle from the same state; gp_reset_worlds restarts a world's
    count."""
    import torch
    import paper_2606_19641_b300 as gp
    wl = wg.WORKLOADS["uniform"]
    worlds = wg.make_workload(wl, n_worlds=3)
    sim, _ = sim_for(worlds, wl, episode_steps=4)
    osim = oracle.Sim(worlds, episode_steps=4)
    start, _ = sim.get_state()
    for k in range(9):
        st0, fl0 = sim.get_state()
        osim.set_state(st0.astype(np.float64), fl0)
        act_t, act = torch_actions(worlds, k, wl.seed)
        sim.step(act_t)
        osim.step(act)
        st1, fl1 = sim.get_state()
        assert np.array_equal(fl1, osim.flags), "flags, step %d" % k
        assert np.allclose(st1, osim.state, atol=2e-4)
        if (k + 1) % 4 == 0:
            assert np.all(fl1 == gp.FLAG_DONE) and np.array_equal(st1, start)
        else:
            assert not np.any(fl1 & gp.FLAG_DONE)
    # one step into the third episode; restart world 1: its episode now ends 4 steps later
    sim.reset_worlds(np.array([0, 1, 0], np.uint8))
    off = worlds.agent_offsets()
    a0, a1 = int(off[1]), int(off[2])
    for k in range(4):
        sim.step(torch_actions(worlds, 20 + k, wl.seed)[0])
        fl = sim.get_state()[1]
        other = np.ones(len(fl), bool)
        other[a0:a1] = False
        assert np.all(fl[other] == gp.FLAG_DONE) == (k == 2)
        assert np.all(fl[a0:a1] == gp.FLAG_DONE) == (k == 3)


def test_reward_conditioning():
    """Conditioning vectors drawn at create, at every episode restart and at gp_reset_worlds
    equal the oracle's draws; the rewards use the drawn weights."""
    import torch
    import paper_2606_19641_b300 as gp
    wl = wg.WORKLOADS["uniform"]
    worlds = wg.make_workload(wl, n_worlds=3)
    sim, _ = sim_for(worlds, wl, rewards=1, episode_steps=3, reward_conditioning=1,
                     conditioning_seed=11)
    osim = oracle.Sim(worlds, episode_steps=3, conditioning_seed=11)
    first = osim.cond.copy()
    assert np.array_equal(sim.conditioning(), osim.cond.astype(np.float32))
    assert np.allclose(sim.reward_weights(), osim.weights, rtol=1e-6, atol=1e-12)
    off = worlds.agent_offsets()
    dims = np.zeros((worlds.n_agents, 2), np.float64)
    for w in range(worlds.n_worlds):
        b0 = int(worlds.box_off[w])
        dims[off[w]:off[w + 1]] = worlds.boxes[b0:b0 + (off[w + 1] - off[w]), 3:5]
    acc = np.zeros((worlds.n_agents, 2), np.float64)
    for k in range(5):
        st0, fl0 = sim.get_state()
        weights = osim.weights.copy()
        act_t, act = torch_actions(worlds, k, wl.seed)
        sim.step(act_t)
        osim.set_state(st0.astype(np.float64), fl0)
        osim.step(act)
        st1, fl1 = sim.get_state()
        assert np.array_equal(sim.conditioning(), osim.cond.astype(np.float32)), "step %d" % k
        if k == 2:  # the episode restarts: rewards are on the pre-restart state, not kept here
            acc[:] = 0.0
            continue
        r = sim.rewards()[0].cpu().numpy()
        for w in range(worlds.n_worlds):
            a0, a1 = int(off[w]), int(off[w + 1])
            road = worlds.road[int(worlds.road_off[w]):int(worlds.road_off[w + 1])]
            acc_w = np.ascontiguousarray(acc[a0:a1])
            rr, _ = oracle.rewards_world(st0[a0:a1], fl0[a0:a1] & 7, st1[a0:a1], fl1[a0:a1],
                                         act[a0:a1], dims[a0:a1], acc_w, weights[a0:a1], road)
            acc[a0:a1] = acc_w
            d = np.abs(r[a0:a1] - rr)
            assert np.all((d <= 1e-4 + 1e-4 * np.abs(rr)) | (d <= weights[a0:a1, 2] + 1e-4))
    assert not np.array_equal(osim.cond, first)  # redrawn at the restart
    sim.reset_worlds(np.array([0, 1, 0], np.uint8))
    osim.reset_worlds([0, 1, 0])
    assert np.array_equal(sim.conditioning(), osim.cond.astype(np.float32))
    assert np.allclose(sim.reward_weights(), osim.weights, rtol=1e-6, atol=1e-12)
    direct, _ = sim_for(worlds, wl)
    with pytest.raises(gp.GigapixelError):
        direct.conditioning()
