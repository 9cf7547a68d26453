"""Helpers shared by the GPU parity tests: build a simulator from a workload, mirror its
FP32 state into the oracle, and compare one view against the oracle."""
import numpy as np

import oracle


def sim_for(worlds, workload, **overrides):
    import paper_2606_19641_b300 as gp
    from paper_2606_19641_b300 import build
    build.build()
    cfg = gp.config_for(workload, **overrides)
    return gp.Simulator(worlds, cfg), cfg


def cam_config(cfg):
    return oracle.CamConfig(int(cfg.width), int(cfg.height), float(np.float32(cfg.hfov)),
                            float(np.float32(cfg.cam_height)), float(np.float32(cfg.near_plane)),
                            float(np.float32(cfg.lane_line_z)))


def oracle_sim(worlds, sim):
    """Oracle simulation holding the GPU's current FP32 state (as FP64)."""
    o = oracle.Sim(worlds)
    st, fl = sim.get_state()
    o.set_state(st.astype(np.float64), fl)
    return o


def view_loc(worlds, cfg, view):
    """view -> (world, agent index within the world, camera index)."""
    off = worlds.agent_offsets()
    agent, cam = divmod(view, int(cfg.n_cams))
    w = int(np.searchsorted(off, agent, side="right") - 1)
    return w, agent - int(off[w]), cam


def dedupe(tris):
    if len(tris) == 0:
        return tris
    u = np.unique(tris.view(np.dtype((np.void, tris.dtype.itemsize))))
    return u.view(tris.dtype)


def oracle_raster_of(worlds, cfg, view, tris):
    w, _, _ = view_loc(worlds, cfg, view)
    nb = int(worlds.box_off[w + 1] - worlds.box_off[w])
    nr = int(worlds.road_off[w + 1] - worlds.road_off[w])
    nl = int(worlds.line_off[w + 1] - worlds.line_off[w])
    t = np.zeros(len(tris), oracle.TRI_DTYPE)
    for k in ("X", "Y", "d", "prim", "sub"):
        t[k] = tris[k]
    return oracle.raster(t, int(cfg.width), int(cfg.height), bool(cfg.key_precision), 12 * nb,
                         12 * nb + 2 * nr, line_end=12 * nb + 2 * nr + 2 * nl)


def gpu_view(cfg, out, depth, view):
    """(class image or one-hot bits, depth bits) of one view as numpy."""
    import torch
    o = out[view]
    if o.dtype == torch.bfloat16:
        o = o.view(torch.int16).cpu().numpy().view(np.uint16)
    else:
        o = o.cpu().numpy()
    d = None
    if depth is not None:
        dv = depth[view]
        d = dv.view(torch.int32).cpu().numpy().view(np.uint32) if dv.dtype == torch.float32 \
            else dv.view(torch.int16).cpu().numpy().view(np.uint16)
    return o, d


def expected_planes(cfg, img):
    """Oracle image -> (class u8 or one-hot bf16 bits, depth bits) in the GPU's encodings."""
    if int(cfg.output) == 0:
        o = img.cls
    else:
        o = oracle.onehot_bf16(img.cls, list(cfg.norm_mean), list(cfg.norm_std))
    d = img.depth.view(np.uint32) if int(cfg.key_precision) == 0 else img.depth
    return o, d


def cls_of(cfg, o):
    """Class image from a GPU/oracle plane (class u8, or one-hot bf16 bits)."""
    if int(cfg.output) == 0:
        return o
    hot = [int(oracle.f32_to_bf16_bits(np.float32((1 - np.float32(m)) / np.float32(s)))[0])
           for m, s in zip(cfg.norm_mean, cfg.norm_std)]
    c = np.zeros(o.shape[1:], np.uint8)
    for k in range(4):
        c[o[k] == hot[k]] = k
    return c
