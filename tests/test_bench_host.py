"""Host-side pieces of bench.py: the roofline traffic comes from a committed ncu summary
only while that summary describes the current render source and launch shape."""
import hashlib
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _src_hash():
    src = open(os.path.join(ROOT, "paper_2606_19641_b300", "csrc", "gp_render.cu"), "rb").read()
    return hashlib.sha256(src).hexdigest()


def test_profiled_traffic_follows_the_render_source():
    import re
    for kernel, shape in (("render_kernel", None), ("trace_kernel", "trace")):
        text = open(os.path.join(ROOT, "profiles", kernel + "_uniform_128x128.md")).read()
        m = re.search(r"traffic_bytes_per_launch: (\d+) \(render source sha256 ([0-9a-f]+), "
                      r"shape ([0-9a-z,]+)\)", text)
        assert m, kernel
        b = _bench()
        # the bench reports the captured traffic only for the source the capture was of
        want = int(m.group(1)) if _src_hash().startswith(m.group(2)) else None
        assert b.profiled_traffic(m.group(3), kernel) == want
        assert b.profiled_traffic("1,2,3", kernel) is None  # another launch shape


def test_job_rate_and_reduction_on_one_rank():
    b = _bench()
    # 8192 agents x 100 steps in 200 ms -> 4.096 M agent-steps/s
    assert abs(b.job_rate(8192, 100, 200.0) - 4.096e6) < 1e-3


def test_algorithmic_bytes_follow_the_method_accounting():
    """Images written plus the world read once: 32 B per road segment, 40 B per agent and
    28 B per static box (not the implementation's triangle geometry)."""
    import types
    import worldgen as wg
    b = _bench()
    wl = wg.WORKLOADS["uniform"]
    worlds = wg.make_workload(wl, n_worlds=2)
    info = types.SimpleNamespace(out_bytes=1000, depth_bytes=400)
    sim = types.SimpleNamespace(info=info)
    want = 1000 + 400 + 32 * 2 * 500 + 40 * 64 + 28 * 0
    assert b.algorithmic_bytes(sim, worlds, wl) == want
    assert b.algorithmic_bytes(sim, worlds, wl, with_depth=False) == want - 400


def test_oracle_sampler_uses_every_core_it_is_given():
    import sys
    import worldgen as wg
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench as b  # importable by name, so the spawned workers can find its functions
    wl = wg.WORKLOADS["tiny"]
    s = b.OracleSampler(wg.make_workload(wl), wl, cores=2)
    try:
        rate, wall, done = s.sample(0.5)
    finally:
        s.close()
    assert s.cores == 2 and done > 0 and rate > 0 and 0.4 < wall < 5.0


def test_accuracy_vs_oracle_on_the_oracles_own_images():
    """The bench's accuracy leg on stand-in "GPU" planes made by the oracle itself from the
    same state: zero class mismatch and zero depth error, for the u8 class + FP32 depth,
    the BF16 one-hot + FP16 key and the class + FP16 key encodings."""
    import sys
    import types
    import numpy as np
    import torch
    import oracle
    import worldgen as wg
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench as b
    from paper_2606_19641_b300 import config_for
    wl = wg.WORKLOADS["tiny"]
    worlds = wg.make_workload(wl)
    o = oracle.Sim(worlds)
    o.step(wg.actions(wl.seed, 0, worlds.n_agents))
    st = o.state.astype(np.float32)
    fl = o.flags.copy()
    for kw in (dict(), dict(key_precision=1, output=1), dict(key_precision=1)):
        cfg = config_for(wl, **kw)
        osim = oracle.Sim(worlds)
        osim.set_state(st.astype(np.float64), fl)
        cam = oracle.CamConfig(wl.width, wl.height, float(np.float32(cfg.hfov)),
                               float(np.float32(cfg.cam_height)), float(np.float32(cfg.near_plane)),
                               float(np.float32(cfg.lane_line_z)))
        views = np.array([0, 3, 7])
        outs, deps = [], []
        for v in views:
            img = osim.render(cam, 0, int(v), 0.0, bool(cfg.key_precision))
            if int(cfg.output) == 1:
                outs.append(torch.from_numpy(oracle.onehot_bf16(img.cls).view(np.int16)))
            else:
                outs.append(torch.from_numpy(img.cls))
            d = img.depth
            deps.append(torch.from_numpy(d.view(np.int16) if d.dtype == np.uint16 else d.view(np.int32)))
        sample = dict(worlds=worlds, wl=wl, cfg=cfg, views=views, state=st, flags=fl,
                      out=torch.stack(outs), depth=torch.stack(deps))
        r = b.accuracy_vs_oracle(sample)
        assert r["class_mismatch_frac_vs_oracle_same_precision"] == 0.0
        assert r["pixels"] == 3 * wl.width * wl.height
        if not kw:
            assert r["depth_rel_err_vs_oracle_fp32_depth"]["max"] == 0.0
        else:
            assert r["depth_rel_err_vs_oracle_fp16_key"]["max"] == 0.0
            assert r["depth_rel_err_vs_oracle_fp32_depth"]["max"] < 2 ** -10  # binary16 rounding
