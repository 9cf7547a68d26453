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


def coverage(t, width, height):
    """Pixel centres that one snapped triangle covers under the raster rule (1/16 px
    vertices, pixel (i, j) sampled at (16 i + 8, 16 j + 8), top-left fill rule, either
    winding): (j0, i0, bool mask over the triangle's bounding box clipped to the image), or
    None if it covers none.  Used to sort out which triangles and pixels a snapping
    difference can touch; checked against oracle.raster in the CPU tests."""
    X = np.asarray(t["X"], np.int64)
    Y = np.asarray(t["Y"], np.int64)
    area = (X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0])
    if area == 0:
        return None
    if area < 0:  # orient to positive area (y down)
        X = X[[0, 2, 1]]
        Y = Y[[0, 2, 1]]
    i0 = max((int(X.min()) + 7) >> 4, 0)
    i1 = min((int(X.max()) - 8) >> 4, width - 1)
    j0 = max((int(Y.min()) + 7) >> 4, 0)
    j1 = min((int(Y.max()) - 8) >> 4, height - 1)
    if i0 > i1 or j0 > j1:
        return None
    px = 16 * np.arange(i0, i1 + 1, dtype=np.int64)[None, :] + 8
    py = 16 * np.arange(j0, j1 + 1, dtype=np.int64)[:, None] + 8
    m = np.ones((j1 - j0 + 1, i1 - i0 + 1), bool)
    for k in range(3):
        xa, ya, xb, yb = X[k], Y[k], X[(k + 1) % 3], Y[(k + 1) % 3]
        A, B = ya - yb, xb - xa
        bias = 0 if (A > 0 or (A == 0 and B > 0)) else 1
        m &= A * (px - xa) + B * (py - ya) - bias >= 0
    return (j0, i0, m) if m.any() else None


def edge_band(cov, width, height):
    """Pixels within one pixel of a covered region's boundary (the region dilated by one
    pixel minus the region eroded by one pixel), as a full-image bool mask."""
    full = np.zeros((height + 2, width + 2), bool)
    j0, i0, m = cov
    full[j0 + 1:j0 + 1 + m.shape[0], i0 + 1:i0 + 1 + m.shape[1]] = m
    dil = np.zeros_like(full)
    ero = np.ones_like(full)
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            sh = np.roll(np.roll(full, dj, 0), di, 1)
            dil |= sh
            ero &= sh
    return (dil & ~ero)[1:-1, 1:-1]


def tri_altitude_units(t):
    """Smallest altitude of a snapped triangle in 1/16-px units (twice the area over the
    longest side): at most a couple of units means a one-unit snap of a vertex can empty or
    flip its coverage."""
    X = np.asarray(t["X"], np.float64)
    Y = np.asarray(t["Y"], np.float64)
    area2 = abs((X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0]))
    longest = max(np.hypot(X[(k + 1) % 3] - X[k], Y[(k + 1) % 3] - Y[k]) for k in range(3))
    return float(area2 / max(longest, 1.0))


def max_centre_depth_units(t, cov):
    """Deepest covered pixel centre of a snapped triangle: the largest, over its covered
    centres, of the distance (in 1/16-px units) to the nearest of its edges.  A one-unit
    move of every vertex shifts each edge line by at most sqrt(2) units, so a centre deeper
    than that stays covered under any such snapping difference."""
    X = np.asarray(t["X"], np.float64)
    Y = np.asarray(t["Y"], np.float64)
    j0, i0, m = cov
    jj, ii = np.nonzero(m)
    px = 16.0 * (ii + i0) + 8.0
    py = 16.0 * (jj + j0) + 8.0
    dmin = np.full(len(px), np.inf)
    for k in range(3):
        xa, ya, xb, yb = X[k], Y[k], X[(k + 1) % 3], Y[(k + 1) % 3]
        ln = max(np.hypot(xb - xa, yb - ya), 1e-9)
        dist = np.abs((ya - yb) * (px - xa) + (xb - xa) * (py - ya)) / ln
        dmin = np.minimum(dmin, dist)
    return float(dmin.max()) if len(dmin) else 0.0


def tri_perimeter_px(t):
    X = np.asarray(t["X"], np.float64) / 16.0
    Y = np.asarray(t["Y"], np.float64) / 16.0
    return float(sum(np.hypot(X[(k + 1) % 3] - X[k], Y[(k + 1) % 3] - Y[k]) for k in range(3)))


def check_views(sim, cfg, worlds, views, out, depth, t2=True, t4=True, t3=True):
    """Per view, from one triangle dump of the GPU:
      T3  the raster rule on the GPU's own snapped triangles gives bit-identical planes;
      T2  (both directions) every triangle covering a pixel centre in one pipeline has a
          counterpart with the same (primitive, fan index) in the other -- the GPU's FP32
          geometry and the oracle's FP64 geometry from the same FP32 state -- with snapped
          vertices within one 1/16-px unit; a primitive that the two pipelines cut into
          different fan pieces (a vertex on a clip plane decided differently in FP32 and
          FP64) must cover the same pixel centres up to what a one-unit snap can flip; a
          primitive present on one side only may cover only pixel centres within 2 units
          (1/8 px) of its edges -- a one-unit snap of the vertices moves an edge by at most
          sqrt(2) units, so a deeper centre would be covered by the other pipeline too;
      T4  the GPU image against the oracle's full FP64 pipeline: class mismatches counted,
          bounded by the pixels a snapping difference can flip -- for every triangle whose
          snapped vertices differ (or that one side lacks or cuts differently), the pixel
          centres within 1/16 px of its edges: at worst every centre along them (an edge on
          a row of pixel centres), perimeter + 3 pixels -- and located (how many lie within
          one pixel of such a triangle's boundary).
    Returns a dict of totals."""
    osim = oracle_sim(worlds, sim)
    cam = cam_config(cfg)
    W, H = int(cfg.width), int(cfg.height)
    S = dict(views=0, pixels=0, covered=0, o_vis=0, g_vis=0, matched=0, exact=0, worst=0,
             missing=0, extra=0, differing=0, recut=0, mismatch=0, explained=0, ties=0, bound=0.0)
    derr = []
    for v in views:
        g = dedupe(sim.dump_tris(v, out, depth))
        # T3 (class or one-hot outputs; the RGB tests check their planes themselves)
        img = oracle_raster_of(worlds, cfg, v, g)
        go, gd = gpu_view(cfg, out, depth, v)
        if t3:
            eo, ed = expected_planes(cfg, img)
            assert np.array_equal(go, eo), "view %d: class/one-hot differs from the raster rule" % v
            if depth is not None:
                assert np.array_equal(gd, ed), "view %d: depth bits differ from the raster rule" % v
        S["covered"] += int((img.cls > 0).sum())
        S["views"] += 1
        S["pixels"] += W * H
        if not (t2 or t4):
            continue
        w, a, c = view_loc(worlds, cfg, v)
        yaw = float(np.float32(cfg.cam_yaw[c]))
        o = osim.camera_tris(cam, w, a, yaw)
        # visible pieces (covering a pixel centre) of every primitive on each side
        cov = {}
        gp_, op_ = {}, {}
        for side, tris, dst in (("g", g, gp_), ("o", o, op_)):
            for t in tris:
                cv = coverage(t, W, H)
                if cv is not None:
                    key = (side, int(t["prim"]), int(t["sub"]))
                    cov[key] = cv
                    dst.setdefault(int(t["prim"]), {})[int(t["sub"])] = t
        risky = []
        for pr in set(gp_) | set(op_):
            gd_, od_ = gp_.get(pr, {}), op_.get(pr, {})
            if sorted(gd_) == sorted(od_):
                for sb in gd_:
                    tg, to = gd_[sb], od_[sb]
                    dx = int(np.abs(tg["X"].astype(np.int64) - to["X"]).max())
                    dy = int(np.abs(tg["Y"].astype(np.int64) - to["Y"]).max())
                    S["o_vis"] += 1
                    S["g_vis"] += 1
                    S["matched"] += 1
                    S["exact"] += int(dx == 0 and dy == 0)
                    S["worst"] = max(S["worst"], dx, dy)
                    assert dx <= 1 and dy <= 1, "view %d prim %d sub %d: snapped vertex %d units from FP64" % (
                        v, pr, sb, max(dx, dy))
                    if dx or dy:
                        risky += [tg, to]
                        S["differing"] += 1
                continue
            pg, po = list(gd_.values()), list(od_.values())
            risky += pg + po
            if pg and po:
                # cut into different fan pieces (a vertex on a clip plane decided differently
                # in FP32 and FP64): the pieces must cover the same centres up to what a
                # one-unit snap of their vertices can flip
                S["recut"] += 1
                S["o_vis"] += 1
                S["g_vis"] += 1
                ug, uo = np.zeros((H, W), bool), np.zeros((H, W), bool)
                for side, d_, u in (("g", gd_, ug), ("o", od_, uo)):
                    for sb in d_:
                        j0, i0, m = cov[(side, pr, sb)]
                        u[j0:j0 + m.shape[0], i0:i0 + m.shape[1]] |= m
                allowed = sum(tri_perimeter_px(t) + 3.0 for t in pg + po)
                nd = int((ug ^ uo).sum())
                assert nd <= allowed, "view %d prim %d: recut pieces cover %d different centres (%s vs %s)" % (
                    v, pr, nd, sorted(gd_), sorted(od_))
            else:
                side = "g" if pg else "o"
                pieces = pg or po
                S["extra" if pg else "missing"] += 1
                S["g_vis" if pg else "o_vis"] += 1
                for sb in sorted(gd_ or od_):
                    t = (gd_ or od_)[sb]
                    cv = cov[(side, pr, sb)]
                    deep = max_centre_depth_units(t, cv)
                    assert deep <= 2.0, (
                        "view %d prim %d: a piece covers %d pixel centres in the %s pipeline only, "
                        "one of them %.2f units inside its edges (X %s, Y %s)" % (
                            v, pr, int(cv[2].sum()), "GPU" if pg else "oracle", deep,
                            list(t["X"]), list(t["Y"])))
        if not t4:
            continue
        ref = osim.render(cam, w, a, yaw, bool(cfg.key_precision))
        gcls = cls_of(cfg, go)
        ocls = ref.cls if int(cfg.output) == 0 else np.where(ref.cls == 4, 3, ref.cls)
        mis = gcls != ocls
        band = np.zeros((H, W), bool)
        for t in risky:
            cv = coverage(t, W, H)
            if cv is not None:
                band |= edge_band(cv, W, H)
                S["bound"] += tri_perimeter_px(t) + 3.0
        S["mismatch"] += int(mis.sum())
        S["explained"] += int((mis & band).sum())
        # the rest should be near-ties in depth between two surfaces (a box's base on the
        # road plane, a lane line far away): both pipelines cover the pixel, at depths
        # within the per-vertex n / z rounding of FP32 against FP64 (or one binary16 step)
        rest = mis & ~band & (gcls > 0) & (ocls > 0)
        if rest.any() and depth is not None:
            if int(cfg.key_precision) == 0:
                gz = gd.view(np.float32).astype(np.float64)
                oz = ref.depth.astype(np.float64)
                tol = 1e-5
            else:
                gz = gd.view(np.float16).astype(np.float64)
                oz = ref.depth.view(np.float16).astype(np.float64)
                tol = 2.0 ** -9
            tie = rest & (np.abs(gz - oz) <= tol * np.maximum(np.abs(oz), 1e-12))
            S["ties"] += int(tie.sum())
        if depth is not None:
            both = (gcls > 0) & (gcls == ocls)
            if int(cfg.key_precision) == 0:
                gg = gd.view(np.float32)[both].astype(np.float64)
                ee = ref.depth[both].astype(np.float64)
            else:
                gg = gd[both].view(np.float16).astype(np.float64)
                ee = ref.depth[both].view(np.float16).astype(np.float64)
            if len(gg):
                derr.append(np.abs(gg - ee) / np.maximum(ee, 1e-6))
    S["depth_rel_err"] = np.concatenate(derr) if derr else np.zeros(1)
    return S


def assert_views(S, label, min_covered=0.2):
    """Print the totals of check_views and apply its bounds."""
    d = S["depth_rel_err"]
    print("%s: %d views; T2 %d oracle / %d GPU visible triangles, %d matched (%d exact, worst "
          "%d units), %d missing, %d extra, %d differing, %d recut; T4 %d class mismatches of %d pixels "
          "(%.2e), %d within a pixel of a differing triangle's boundary, %d depth near-ties, bound %.0f; depth rel "
          "err p99 %.2e max %.2e" % (
              label, S["views"], S["o_vis"], S["g_vis"], S["matched"], S["exact"], S["worst"],
              S["missing"], S["extra"], S["differing"], S["recut"], S["mismatch"], S["pixels"],
              S["mismatch"] / max(S["pixels"], 1), S["explained"], S["ties"], S["bound"],
              np.percentile(d, 99), d.max()))
    assert S["covered"] > min_covered * S["pixels"]
    assert S["missing"] <= 0.002 * S["o_vis"] + 2 and S["extra"] <= 0.002 * S["g_vis"] + 2
    assert S["mismatch"] <= S["bound"]
    assert np.percentile(d, 99) < 1e-3
