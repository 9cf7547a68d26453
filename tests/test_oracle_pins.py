"""Pins for the CPU oracle: closed forms, invariants, brute force and independent methods.

Each test checks the oracle against something other than itself, chosen so that a
plausible slip in it (a dropped term, a flipped sign or index, a transposed operand, a
wrong fill rule) fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import CamConfig

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            vals[k] = [float(t) for t in v]
    return vals


def ego_box(x=0.0, y=0.0, yaw=0.0):
    return [x, y, yaw, 4.5, 1.9, 1.5]


def render_scene(cam, boxes, road=(), line=(), pose=(0.0, 0.0, 0.0), cam_yaw=0.0,
                 key_f16=False, ego=0, sph=None):
    b = np.array(boxes, np.float64).reshape(-1, 6)
    rd = np.array(road, np.float32).reshape(-1, 8)
    ln = np.array(line, np.float32).reshape(-1, 8)
    tris = oracle.camera_tris(cam, b, ego, rd, ln, pose[0], pose[1], pose[2], cam_yaw, sph=sph)
    re = 12 * len(b) + 2 * len(rd)
    img = oracle.raster(tris, cam.width, cam.height, key_f16, 12 * len(b), re,
                        line_end=re + 2 * len(ln))
    return img, tris


def rect_quad(x0, x1, y0, y1):
    """Axis-aligned rectangle as a quad, counter-clockwise from above."""
    return [x0, y0, x1, y0, x1, y1, x0, y1]


# ---------------------------------------------------------------------------------------
# Rendering closed forms
# ---------------------------------------------------------------------------------------

def test_empty_scene_is_background():
    cam = CamConfig(32, 24)
    img, tris = render_scene(cam, [ego_box()])
    assert len(tris) == 0
    assert not img.cls.any() and not img.depth.any() and not img.key.any()


def _box_face_expectation(W, H, D, hw, bh, cam_h=1.5):
    f = Fraction(W, 2)  # hfov = 90 deg
    x_lo, x_hi = Fraction(W, 2) - f * hw / D, Fraction(W, 2) + f * hw / D
    y_top, y_bot = Fraction(H, 2) - f * (bh - cam_h) / D, Fraction(H, 2) + f * cam_h / D
    cols = [i for i in range(W) if x_lo < i + Fraction(1, 2) < x_hi]
    rows = [j for j in range(H) if y_top < j + Fraction(1, 2) < y_bot]
    # every pixel centre must be >= 1/16 px from an edge, so snapping cannot flip it
    margin = min(min(abs(i + Fraction(1, 2) - e) for e in (x_lo, x_hi)) for i in range(W))
    margin = min(margin, min(min(abs(j + Fraction(1, 2) - e) for e in (y_top, y_bot))
                             for j in range(H)))
    return cols, rows, margin


def test_golden_box_face_rectangle():
    g = read_golden("box_front_face_64x64.txt")
    W, H = int(g["width"][0]), int(g["height"][0])
    D, hw, bh = (Fraction(str(g[k][0])) for k in ("distance", "half_width", "box_height"))
    cols, rows, margin = _box_face_expectation(W, H, D, hw, bh)
    # the derivation in the fixture and the exact arithmetic here agree
    assert (cols[0], cols[-1]) == tuple(int(v) for v in g["cols"])
    assert (rows[0], rows[-1]) == tuple(int(v) for v in g["rows"])
    assert margin >= Fraction(1, 16)
    L = 4.5
    cam = CamConfig(W, H)
    img, _ = render_scene(cam, [ego_box(), [float(D) + L / 2, 0.0, 0.0, L, 2 * float(hw), float(bh)]])
    expect = np.zeros((H, W), bool)
    expect[rows[0]:rows[-1] + 1, cols[0]:cols[-1] + 1] = True
    assert np.array_equal(img.cls == 3, expect)
    assert np.array_equal(img.cls != 0, expect)
    assert np.all(img.depth[expect] == np.float32(g["depth"][0]))
    assert np.all(img.depth[~expect] == 0)


def _generic_box_cases(n=6):
    """Seeded (W, H, D, half-width, height) cases with every pixel centre >= 1/8 px from
    the face's projected edges."""
    rng = np.random.default_rng(21)
    out = []
    while len(out) < n:
        W, H = [(64, 64), (128, 96), (48, 48), (256, 144), (96, 64), (512, 512)][len(out) % 6]
        D = Fraction(int(rng.integers(40, 300)), 10)
        hw = Fraction(int(rng.integers(90, 100)), 100)
        bh = Fraction(int(rng.integers(140, 170)), 100)
        if _box_face_expectation(W, H, D, hw, bh)[2] >= Fraction(1, 8):
            out.append((W, H, D, hw, bh))
    return out


@pytest.mark.parametrize("W,H,D,hw,bh", _generic_box_cases())
def test_box_face_rectangle_general(W, H, D, hw, bh):
    cols, rows, margin = _box_face_expectation(W, H, D, hw, bh)
    assert margin >= Fraction(1, 8) and cols and rows
    L = 4.2
    cam = CamConfig(W, H)
    img, _ = render_scene(cam, [ego_box(), [float(D) + L / 2, 0.0, 0.0, L, 2 * float(hw), float(bh)]])
    expect = np.zeros((H, W), bool)
    expect[rows[0]:rows[-1] + 1, cols[0]:cols[-1] + 1] = True
    assert np.array_equal(img.cls == 3, expect)
    assert np.all(img.depth[expect] == np.float32(0.1 / float(D)))


def test_ground_strip_vanishing_lines_and_row_depth():
    """A strip |y| < r ahead of the camera: edges are the lines u - W/2 = +-(r/h)(v - H/2)
    through the vanishing point, and the ground depth in row v is n (v - H/2) / (f h)."""
    W = H = 64
    f, h, n, r = 32.0, 1.5, 0.1, 1.3137
    cam = CamConfig(W, H)
    img, _ = render_scene(cam, [ego_box()], road=[rect_quad(-5.0, 200.0, -r, r)])
    u = np.arange(W) + 0.5
    v = np.arange(H) + 0.5 - H / 2
    checked = 0
    for j in range(H):
        if v[j] <= 0:
            assert not img.cls[j].any()
            continue
        half = r / h * v[j]
        dist = np.abs(np.abs(u - W / 2) - half)
        inside = np.abs(u - W / 2) < half
        sure = dist > 1 / 8
        assert np.array_equal(img.cls[j][sure] == 1, inside[sure])
        d_exact = n * v[j] / (f * h)
        tol = (n / (f * h)) / 16 + 1e-7  # depth gradient per px times 1/16 px of snapping
        cov = img.cls[j] == 1
        assert np.all(np.abs(img.depth[j][cov] - d_exact) <= tol)
        checked += int(sure.sum())
    assert checked > 1000


def test_mirror_symmetry_of_centred_scene():
    W = H = 64
    r, lw = 1.7321, 0.15
    cam = CamConfig(W, H)
    boxes = [ego_box(), [8.137 + 2.2, 0.0, 0.0, 4.4, 1.8913, 1.6217]]
    road = [rect_quad(-5.0, 150.0, -r, r)]
    line = [rect_quad(-5.0, 150.0, r - lw / 2, r + lw / 2),
            rect_quad(-5.0, 150.0, -r - lw / 2, -r + lw / 2)]
    img, _ = render_scene(cam, boxes, road, line)
    assert (img.cls == 3).sum() > 20 and (img.cls == 1).sum() > 100 and (img.cls == 2).sum() > 10
    assert np.array_equal(img.cls, img.cls[:, ::-1])


# ---------------------------------------------------------------------------------------
# Independent FP64 ray casting on tiny images
# ---------------------------------------------------------------------------------------

def _quad_contains(q, px, py):
    q = np.asarray(q, np.float64).reshape(4, 2)
    ok = np.ones_like(px, bool)
    for k in range(4):
        a, b = q[k], q[(k + 1) % 4]
        cr = (b[0] - a[0]) * (py - a[1]) - (b[1] - a[1]) * (px - a[0])
        ok &= cr >= 0
    return ok


def raycast(W, H, boxes, ego, road, line, pose, cam_yaw, jx=0.0, jy=0.0,
            h=1.5, near=0.1, line_z=0.02, hfov=math.pi / 2):
    """Nearest hit per pixel by slab tests (boxes) and plane hits (ground quads)."""
    psi = pose[2] + cam_yaw
    f = (W / 2) / math.tan(hfov / 2)
    uu = np.arange(W) + 0.5 + jx
    vv = np.arange(H) + 0.5 + jy
    xv = ((uu - W / 2) / f)[None, :]
    yv = (-(vv - H / 2) / f)[:, None]
    right = np.array([math.sin(psi), -math.cos(psi), 0.0])
    fwd = np.array([math.cos(psi), math.sin(psi), 0.0])
    D = xv[..., None] * right + yv[..., None] * np.array([0, 0, 1.0]) + fwd  # [H, W, 3]
    D = np.broadcast_to(D, (H, W, 3))
    O = np.array([pose[0], pose[1], h])
    best_t = np.full((H, W), np.inf)
    best_cls = np.zeros((H, W), np.uint8)
    best_obj = np.full((H, W), -1)
    for bi, b in enumerate(boxes):
        if bi == ego:
            continue
        cs, sn = math.cos(b[2]), math.sin(b[2])
        # ray in box-local frame
        ox, oy = O[0] - b[0], O[1] - b[1]
        lo_o = np.array([cs * ox + sn * oy, -sn * ox + cs * oy, O[2]])
        ld = np.stack([cs * D[..., 0] + sn * D[..., 1], -sn * D[..., 0] + cs * D[..., 1], D[..., 2]], -1)
        lo = np.array([-b[3] / 2, -b[4] / 2, 0.0])
        hi = np.array([b[3] / 2, b[4] / 2, b[5]])
        with np.errstate(divide="ignore", invalid="ignore"):
            t1 = (lo - lo_o) / ld
            t2 = (hi - lo_o) / ld
        tmin = np.nanmax(np.minimum(t1, t2), axis=-1)
        tmax = np.nanmin(np.maximum(t1, t2), axis=-1)
        hit = (tmin <= tmax) & (tmin >= near) & (tmin < best_t)
        best_t[hit], best_cls[hit], best_obj[hit] = tmin[hit], 3, bi
    for cls, quads, z, base in ((1, road, 0.0, 1000), (2, line, line_z, 100000)):
        for qi, q in enumerate(quads):
            with np.errstate(divide="ignore", invalid="ignore"):
                t = (z - h) / D[..., 2]
            px, py = O[0] + t * D[..., 0], O[1] + t * D[..., 1]
            hit = (D[..., 2] < 0) & (t >= near) & _quad_contains(q, px, py) & (t < best_t)
            best_t[hit], best_cls[hit], best_obj[hit] = t[hit], cls, base + qi
    depth = np.where(np.isfinite(best_t), near / best_t, 0.0)
    return best_cls, depth, best_obj


def _random_scene(rng):
    boxes = [ego_box(0.0, 0.0, 0.0)]
    want = rng.integers(2, 6)
    while len(boxes) < want + 1:
        ang = rng.uniform(-0.7, 0.7)
        dist = rng.uniform(4.0, 30.0)
        x, y = dist * math.cos(ang), dist * math.sin(ang)
        # bounding circles (radius <= 2.7 m) apart: boxes never interpenetrate
        if all(math.hypot(x - b[0], y - b[1]) > 5.5 for b in boxes):
            boxes.append([x, y, rng.uniform(-math.pi, math.pi), rng.uniform(4, 5),
                          rng.uniform(1.8, 2.0), rng.uniform(1.4, 1.7)])
    road, line = [], []
    for _ in range(rng.integers(2, 5)):
        cx, cy = rng.uniform(-10, 40), rng.uniform(-20, 20)
        hd = rng.uniform(-math.pi, math.pi)
        L, Wd = rng.uniform(10, 60), rng.uniform(3, 8)
        c, s = math.cos(hd), math.sin(hd)

        def corner(a, b):
            return [cx + c * a - s * b, cy + s * a + c * b]
        road.append(sum([corner(-L / 2, -Wd / 2), corner(L / 2, -Wd / 2), corner(L / 2, Wd / 2),
                         corner(-L / 2, Wd / 2)], []))
        for off in (-Wd / 2, 0.0, Wd / 2):
            line.append(sum([corner(-L / 2, off - 0.075), corner(L / 2, off - 0.075),
                             corner(L / 2, off + 0.075), corner(-L / 2, off + 0.075)], []))
    return boxes, road, line


def _outline_distance(W, H, boxes, ego, road, line, pose, cam_yaw, h=1.5, near=0.1,
                      line_z=0.02, hfov=math.pi / 2):
    """Distance (px) from each pixel centre to the nearest projected outline edge of any
    box face or ground quad, after cutting each polygon at the near plane."""
    psi = pose[2] + cam_yaw
    f = (W / 2) / math.tan(hfov / 2)
    right = np.array([math.sin(psi), -math.cos(psi), 0.0])
    fwd = np.array([math.cos(psi), math.sin(psi), 0.0])
    O = np.array([pose[0], pose[1], h])
    polys = []
    for bi, b in enumerate(boxes):
        if bi == ego:
            continue
        c, s = math.cos(b[2]), math.sin(b[2])
        P = {}
        for sx in (-1, 1):
            for sy in (-1, 1):
                for z in (0.0, b[5]):
                    lx, ly = sx * b[3] / 2, sy * b[4] / 2
                    P[(sx, sy, z)] = np.array([b[0] + c * lx - s * ly, b[1] + s * lx + c * ly, z])
        for axis in range(3):
            for sign in (0, 1):
                pts = [k for k in P if (k[axis] > 0 if axis < 2 else k[2] > 0) == bool(sign)]
                # order the 4 face corners around the face
                cen = np.mean([P[k] for k in pts], 0)
                nrm = cen - np.mean(list(P.values()), 0)  # face normal direction
                u = P[pts[0]] - cen
                v = np.cross(nrm, u)
                ang = [math.atan2(np.dot(P[k] - cen, v), np.dot(P[k] - cen, u)) for k in pts]
                polys.append([P[pts[i]] for i in np.argsort(ang)])
    for quads, z in ((road, 0.0), (line, line_z)):
        for q in quads:
            qq = np.asarray(q, np.float64).reshape(4, 2)
            polys.append([np.array([x, y, z]) for x, y in qq])
    cx = (np.arange(W) + 0.5)[None, :]
    cy = (np.arange(H) + 0.5)[:, None]
    best = np.full((H, W), np.inf)
    for poly in polys:
        vw = [np.array([np.dot(p - O, right), p[2] - O[2], np.dot(p - O, fwd)]) for p in poly]
        out = []
        for i in range(len(vw)):  # keep the part with z >= near
            a, b = vw[i], vw[(i + 1) % len(vw)]
            if a[2] >= near:
                out.append(a)
            if (a[2] >= near) != (b[2] >= near):
                t = (near - a[2]) / (b[2] - a[2])
                out.append(a + t * (b - a))
        if len(out) < 2:
            continue
        pts = [(W / 2 + f * p[0] / p[2], H / 2 - f * p[1] / p[2]) for p in out]
        for i in range(len(pts)):
            (ax, ay), (bx, by) = pts[i], pts[(i + 1) % len(pts)]
            dx, dy = bx - ax, by - ay
            L2 = dx * dx + dy * dy
            t = np.clip(((cx - ax) * dx + (cy - ay) * dy) / L2, 0, 1) if L2 > 0 else 0.0
            d = np.hypot(cx - (ax + t * dx), cy - (ay + t * dy))
            best = np.minimum(best, d)
    return best


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("W,H", [(16, 16), (32, 32), (40, 24)])
def test_raycast_agrees_away_from_edges(seed, W, H):
    """Every pixel whose centre is more than 1/16 px from all projected outlines (snapping
    moves a vertex by at most 1/32 px per axis) must show the ray-cast class, and the
    depth must match within the change of depth across 1/16 px."""
    rng = np.random.default_rng(100 + seed)
    boxes, road, line = _random_scene(rng)
    cam_yaw = rng.uniform(-0.3, 0.3)
    cam = CamConfig(W, H)
    img, _ = render_scene(cam, boxes, road, line, cam_yaw=cam_yaw)
    cls0, d0, obj0 = raycast(W, H, boxes, 0, road, line, (0, 0, 0), cam_yaw)
    sure = _outline_distance(W, H, boxes, 0, road, line, (0, 0, 0), cam_yaw) > 1 / 16
    dspread = np.zeros((H, W))
    for jx, jy in ((1 / 16, 0), (-1 / 16, 0), (0, 1 / 16), (0, -1 / 16)):
        c, d, o = raycast(W, H, boxes, 0, road, line, (0, 0, 0), cam_yaw, jx, jy)
        assert np.array_equal(o[sure], obj0[sure])  # no outline within 1/16 px
        dspread = np.maximum(dspread, np.abs(d - d0))
    assert sure.mean() > 0.5
    assert np.array_equal(img.cls[sure], cls0[sure])
    hit = sure & (cls0 > 0)
    assert np.all(np.abs(img.depth[hit] - d0[hit]) <= dspread[hit] + 1e-6 * d0[hit] + 1e-9)


# ---------------------------------------------------------------------------------------
# Raster rule: bounding-box loop == brute force; fill rule; watertightness
# ---------------------------------------------------------------------------------------

def _tris(rows):
    t = np.zeros(len(rows), oracle.TRI_DTYPE)
    for i, (X, Y, d, prim) in enumerate(rows):
        t[i]["X"], t[i]["Y"], t[i]["d"], t[i]["prim"] = X, Y, d, prim
    return t


@pytest.mark.parametrize("key_f16", [False, True])
def test_bbox_raster_equals_bruteforce(key_f16):
    rng = np.random.default_rng(7)
    rows = []
    for i in range(300):
        X = rng.integers(-300, 1300, 3)
        Y = rng.integers(-300, 900, 3)
        if i % 10 == 0:  # some vertices exactly on pixel centres
            X = 16 * rng.integers(-2, 66, 3) + 8
            Y = 16 * rng.integers(-2, 50, 3) + 8
        d = rng.uniform(1e-3, 1.0, 3).astype(np.float32)
        if i % 7 == 0:
            d[:] = d[0]  # equal depths -> exact ties between triangles
        rows.append((X, Y, d, int(rng.integers(0, 60000))))
    t = _tris(rows)
    a = oracle.raster(t, 64, 48, key_f16, 1000, 30000)
    b = oracle.raster(t, 64, 48, key_f16, 1000, 30000, bruteforce=True)
    assert np.array_equal(a.key, b.key)
    assert np.array_equal(a.cls, b.cls) and np.array_equal(a.depth, b.depth)
    assert (a.key != 0).mean() > 0.5


def test_fill_rule_top_left_cases():
    # the centre of pixel (0, 0) is (8, 8) in 1/16 units
    def covered(X, Y):
        img = oracle.raster(_tris([(X, Y, [0.5, 0.5, 0.5], 1)]), 4, 4, False, 0, 0)
        return bool(img.key[0, 0])
    assert covered([0, 32, 0], [8, 8, 40])        # on a top edge (triangle below it)
    assert not covered([0, 32, 0], [8, 8, -24])   # on a bottom edge
    assert covered([8, 8, 40], [0, 32, 16])       # on a left edge (triangle to its right)
    assert not covered([8, 8, -24], [0, 32, 16])  # on a right edge
    assert covered([8, 40, 8], [8, 8, 40])        # on the top-left corner vertex
    assert not covered([8, 40, 8], [8, 8, -24])   # vertex shared with a bottom edge
    # winding does not matter: either orientation gives the same coverage
    assert covered([0, 0, 32], [8, 40, 8]) == covered([0, 32, 0], [8, 8, 40])


@pytest.mark.parametrize("seed", range(4))
def test_mesh_is_watertight(seed):
    """A perturbed lattice mesh tiling a rectangle covers each centre inside exactly once,
    and on the boundary exactly the left/top lines (top-left rule)."""
    rng = np.random.default_rng(seed)
    W, H, nx, ny = 40, 32, 6, 5
    x0, x1 = 16 * 3 + 8, 16 * 36 + 8   # boundary lines through pixel centres
    y0, y1 = 16 * 2 + 8, 16 * 29 + 8
    gx = np.linspace(x0, x1, nx + 1).round().astype(np.int64)
    gy = np.linspace(y0, y1, ny + 1).round().astype(np.int64)
    VX = np.tile(gx, (ny + 1, 1))
    VY = np.tile(gy[:, None], (1, nx + 1))
    sx, sy = (x1 - x0) // nx, (y1 - y0) // ny
    for j in range(ny + 1):
        for i in range(nx + 1):
            if 0 < i < nx:
                VX[j, i] += rng.integers(-sx // 4, sx // 4 + 1)
            if 0 < j < ny:
                VY[j, i] += rng.integers(-sy // 4, sy // 4 + 1)
            if rng.random() < 0.3:  # snap some vertices onto pixel centres
                if 0 < i < nx:
                    VX[j, i] = 16 * (VX[j, i] // 16) + 8
                if 0 < j < ny:
                    VY[j, i] = 16 * (VY[j, i] // 16) + 8
    tris = []
    for j in range(ny):
        for i in range(nx):
            a, b, c, d = (j, i), (j, i + 1), (j + 1, i + 1), (j + 1, i)
            split = [(a, b, c), (a, c, d)] if rng.random() < 0.5 else [(a, b, d), (b, c, d)]
            for tri in split:
                tris.append(([VX[p] for p in tri], [VY[p] for p in tri]))
    count = np.zeros((H, W), int)
    for k, (X, Y) in enumerate(tris):
        img = oracle.raster(_tris([(X, Y, [0.3, 0.3, 0.3], k)]), W, H, False, 0, 0)
        count += img.key != 0
    cx = 16 * np.arange(W)[None, :] + 8
    cy = 16 * np.arange(H)[:, None] + 8
    expect = (cx >= x0) & (cx < x1) & (cy >= y0) & (cy < y1)
    assert np.array_equal(count, expect.astype(int))


def test_depth_plane_matches_vertex_values():
    """At pixel centres that coincide with vertices the plane returns the vertex depth
    (up to FP32 rounding of the plane evaluation)."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        P = 16 * rng.integers(0, 32, (3, 2)) + 8
        d = rng.uniform(0.01, 1.0, 3).astype(np.float32)
        t = _tris([(P[:, 0], P[:, 1], d, 5)])
        a2 = (P[1, 0] - P[0, 0]) * (P[2, 1] - P[0, 1]) - (P[2, 0] - P[0, 0]) * (P[1, 1] - P[0, 1])
        if a2 == 0:
            continue
        # the vertex pixel is covered unless it sits on a non-top-left edge: use the bruteforce
        # key of the lone triangle, and compare wherever the vertex pixel is covered
        img = oracle.raster(t, 32, 32, False, 100, 100)
        for k in range(3):
            i, j = (P[k] - 8) // 16
            if img.key[j, i]:
                assert abs(float(img.depth[j, i]) - float(d[k])) <= 4e-6 * max(1.0, float(d.max()))


# ---------------------------------------------------------------------------------------
# Number formats
# ---------------------------------------------------------------------------------------

def test_f16_rounding_matches_numpy():
    rng = np.random.default_rng(11)
    bits = rng.integers(0, 2 ** 32, 20000, dtype=np.uint64).astype(np.uint32)
    x = bits.view(np.float32)
    special = np.array([0.0, -0.0, 1.0, 65504.0, 65519.99, 65520.0, 1e-8, 2 ** -24, 2 ** -25,
                        3 * 2 ** -26, 2 ** -14, 2 ** -14 * (1 - 2 ** -11), 1 + 2 ** -11,
                        1 + 3 * 2 ** -11, 5.9604645e-08, np.inf, -np.inf], np.float32)
    x = np.concatenate([x, special, rng.uniform(0, 1, 5000).astype(np.float32)])
    ours = oracle.f32_to_f16_bits(x)
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).view(np.uint16)
    nan = np.isnan(x)
    assert np.array_equal(ours[~nan], ref[~nan])
    assert np.all(np.isnan(ours[nan].view(np.float16)))


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(12)
    bits = rng.integers(0, 2 ** 32, 20000, dtype=np.uint64).astype(np.uint32)
    x = np.concatenate([bits.view(np.float32), np.array([1.0, -1.0, 0.5, 1 + 2 ** -8,
                                                         1 + 3 * 2 ** -8, 3.4e38], np.float32)])
    x = x[~np.isnan(x)]
    ours = oracle.f32_to_bf16_bits(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, ref)


def test_onehot_default_normalisation_is_plus_minus_one():
    cls = np.array([[0, 1, 2, 3]], np.uint8)
    out = oracle.onehot_bf16(cls)
    assert out.shape == (4, 1, 4)
    for c in range(4):
        for p in range(4):
            assert out[c, 0, p] == (0x3F80 if p == c else 0xBF80)
    out2 = oracle.onehot_bf16(cls, mean=(0.1, 0.2, 0.3, 0.4), std=(0.25, 0.5, 2.0, 4.0))
    import torch
    for c, (m, s) in enumerate(zip((0.1, 0.2, 0.3, 0.4), (0.25, 0.5, 2.0, 4.0))):
        hot = (np.float32(1) - np.float32(m)) / np.float32(s)
        cold = (np.float32(0) - np.float32(m)) / np.float32(s)
        want = torch.tensor([cold, hot], dtype=torch.float32).to(torch.bfloat16)
        want = want.view(torch.int16).numpy().view(np.uint16)
        assert out2[c, 0, c] == want[1] and out2[c, 0, (c + 1) % 4] == want[0]


# ---------------------------------------------------------------------------------------
# Dynamics and infractions
# ---------------------------------------------------------------------------------------

def test_paper_constants_golden():
    g = read_golden("paper_constants.txt")
    # a straight step with steer -> the wheelbase enters through l_r = wheelbase / 2
    L, v, steer, dt = 4.0, 10.0, 0.2, g["dt"][0]
    x, y, yaw, v1 = oracle.bicycle(0, 0, 0, v, L, 0.0, steer, dt)
    wb = g["wheelbase_fraction"][0] * L
    beta = math.atan(0.5 * math.tan(steer))
    assert yaw == pytest.approx(v / (wb / 2) * math.sin(beta) * dt, rel=1e-12)


def test_bicycle_straight_closed_form():
    x0, y0, yaw, v0, a, dt, vmax = 1.0, -2.0, 0.3, 5.0, 1.5, 0.1, 12.0
    st = (x0, y0, yaw, v0)
    n = 80
    for _ in range(n):
        st = oracle.bicycle(*st, 4.5, a, 0.0, dt, vmax)
    vs = [min(v0 + k * a * dt, vmax) for k in range(n)]
    assert st[0] == pytest.approx(x0 + dt * math.cos(yaw) * sum(vs), rel=1e-12)
    assert st[1] == pytest.approx(y0 + dt * math.sin(yaw) * sum(vs), rel=1e-12)
    assert st[2] == pytest.approx(yaw, abs=1e-15)
    assert st[3] == pytest.approx(vmax)
    # braking clamps at zero
    st = (0, 0, 0, 1.0)
    for _ in range(10):
        st = oracle.bicycle(*st, 4.5, -3.0, 0.0, dt, vmax)
    assert st[3] == 0.0 and st[0] == pytest.approx(dt * (1.0 + 0.7 + 0.4 + 0.1))


def test_bicycle_constant_steer_sum_of_cosines():
    """Constant speed and steer: heading advances by phi = v sin(beta)/l_r dt per step, so the
    position is a geometric sum of cosines with the textbook closed form."""
    x0, y0, th0, v, L, steer, dt = 3.0, 4.0, -0.4, 7.0, 4.6, 0.25, 0.1
    beta = math.atan(0.5 * math.tan(steer))
    phi = v * math.sin(beta) / (0.3 * L) * dt
    n = 37
    st = (x0, y0, th0, v)
    pts = [st[:2]]
    for _ in range(n):
        st = oracle.bicycle(*st, L, 0.0, steer, dt, 30.0)
        pts.append(st[:2])
    k = math.sin(n * phi / 2) / math.sin(phi / 2)
    mid = th0 + beta + (n - 1) * phi / 2
    assert st[0] == pytest.approx(x0 + v * dt * k * math.cos(mid), abs=1e-10)
    assert st[1] == pytest.approx(y0 + v * dt * k * math.sin(mid), abs=1e-10)
    # the discrete path lies on a circle of radius v dt / (2 sin(phi/2)) (chord v dt, angle phi)
    rho = v * dt / (2 * math.sin(phi / 2))
    p = np.array(pts)
    A = np.c_[2 * p, np.ones(len(p))]
    sol, *_ = np.linalg.lstsq(A, (p ** 2).sum(1), rcond=None)
    c = sol[:2]
    assert np.allclose(np.linalg.norm(p - c, axis=1), rho, rtol=1e-9)
    # heading wraps into (-pi, pi]
    st = (0, 0, math.pi - 0.01, 10.0)
    st = oracle.bicycle(*st, 4.0, 0.0, 0.3, 0.1, 30.0)
    assert -math.pi < st[2] <= math.pi and st[2] < 0


def _poly_clip_area(p, q):
    """Area of the intersection of two convex CCW polygons (Sutherland-Hodgman)."""
    out = [tuple(v) for v in p]
    for k in range(len(q)):
        a, b = q[k], q[(k + 1) % len(q)]
        inp, out = out, []
        if not inp:
            break

        def side(v):
            return (b[0] - a[0]) * (v[1] - a[1]) - (b[1] - a[1]) * (v[0] - a[0])
        for i in range(len(inp)):
            cur, nxt = inp[i], inp[(i + 1) % len(inp)]
            sc, sn = side(cur), side(nxt)
            if sc >= 0:
                out.append(cur)
            if (sc >= 0) != (sn >= 0):
                t = sc / (sc - sn)
                out.append((cur[0] + t * (nxt[0] - cur[0]), cur[1] + t * (nxt[1] - cur[1])))
    if len(out) < 3:
        return 0.0
    o = np.array(out)
    return 0.5 * float(np.sum(o[:, 0] * np.roll(o[:, 1], -1) - np.roll(o[:, 0], -1) * o[:, 1]))


def _corners(b):
    c, s = math.cos(b[2]), math.sin(b[2])
    return [(b[0] + c * lx - s * ly, b[1] + s * lx + c * ly)
            for lx, ly in ((-b[3] / 2, -b[4] / 2), (b[3] / 2, -b[4] / 2), (b[3] / 2, b[4] / 2),
                           (-b[3] / 2, b[4] / 2))]


def test_sat_matches_polygon_intersection_area():
    rng = np.random.default_rng(5)
    seen = {True: 0, False: 0}
    for _ in range(3000):
        a = [0.0, 0.0, rng.uniform(-math.pi, math.pi), rng.uniform(3, 6), rng.uniform(1, 3)]
        b = [rng.uniform(-6, 6), rng.uniform(-6, 6), rng.uniform(-math.pi, math.pi),
             rng.uniform(3, 6), rng.uniform(1, 3)]
        area = _poly_clip_area(_corners(a), _corners(b))
        if 0 < area < 1e-6:
            continue
        got = oracle.obb_overlap(a, b)
        assert got == (area > 0), (a, b, area)
        seen[got] += 1
    assert seen[True] > 300 and seen[False] > 300


def test_sat_axis_aligned_intervals_and_touching():
    for dx, dy, want in ((4.0, 0.0, False), (3.999, 0.0, True), (0.0, 2.0, False),
                         (0.0, 1.99, True), (4.0, 2.0, False), (-3.5, 1.5, True)):
        assert oracle.obb_overlap([0, 0, 0, 4.0, 2.0], [dx, dy, 0, 4.0, 2.0]) == want


def _winding(q, px, py):
    q = np.asarray(q, np.float64).reshape(4, 2)
    ang = 0.0
    for k in range(4):
        a = math.atan2(q[k][1] - py, q[k][0] - px)
        b = math.atan2(q[(k + 1) % 4][1] - py, q[(k + 1) % 4][0] - px)
        d = b - a
        while d > math.pi:
            d -= 2 * math.pi
        while d < -math.pi:
            d += 2 * math.pi
        ang += d
    return round(ang / (2 * math.pi))


def test_point_in_quad_matches_winding_number():
    rng = np.random.default_rng(9)
    n_in = 0
    for _ in range(400):
        c, s = math.cos(t := rng.uniform(-math.pi, math.pi)), math.sin(t)
        L, Wd = rng.uniform(2, 20), rng.uniform(2, 8)
        sk = rng.uniform(-1, 1)
        pts = [(-L / 2, -Wd / 2), (L / 2, -Wd / 2 + sk), (L / 2, Wd / 2 - sk), (-L / 2, Wd / 2)]
        q = np.array([[c * x - s * y, s * x + c * y] for x, y in pts], np.float32).ravel()
        for _ in range(10):
            px, py = rng.uniform(-12, 12), rng.uniform(-12, 12)
            qq = q.astype(np.float64).reshape(4, 2)
            dmin = min(abs((qq[(k + 1) % 4][0] - qq[k][0]) * (py - qq[k][1]) -
                           (qq[(k + 1) % 4][1] - qq[k][1]) * (px - qq[k][0]))
                       for k in range(4))
            if dmin < 1e-6:
                continue
            w = _winding(q, px, py)
            got = oracle.point_in_quad(px, py, q)
            assert got == (w == 1)
            n_in += got
    assert n_in > 200


def test_step_offroad_halts_and_latches():
    R = 3.5
    road = np.array([rect_quad(-50, 50, -R, R)], np.float32)
    # agent 0 centred, agent 1 with its left side 0.05 m inside the edge, agent 2 outside
    boxes = np.array([[0, 0, 0, 4.0, 2.0, 1.5], [10, R - 1.05, 0, 4.0, 2.0, 1.5],
                      [20, R - 0.95, 0, 4.0, 2.0, 1.5]], np.float64)
    state = np.array([[0, 0, 0, 0], [10, R - 1.05, 0, 0], [20, R - 0.95, 0, 0]], np.float64)
    flags = np.zeros(3, np.uint8)
    act = np.zeros((3, 2), np.float32)
    oracle.step_world(boxes, state, flags, act, road)
    assert list(flags) == [0, 0, oracle.OFFROAD | oracle.HALTED]
    # the halted agent ignores actions and stays put; flags latch
    act[:, 0] = 2.0
    before = state[2].copy()
    for _ in range(3):
        oracle.step_world(boxes, state, flags, act, road)
    assert np.array_equal(state[2, :3], before[:3]) and state[2, 3] == 0
    assert flags[2] == oracle.OFFROAD | oracle.HALTED
    assert state[0, 3] == pytest.approx(0.6) and flags[0] == 0


def test_step_collision_flags_agents_only():
    road = np.array([rect_quad(-100, 100, -10, 10)], np.float32)
    # agents 0 and 1 drive into each other; agent 2 drives into static box 3
    boxes = np.array([[0, 0, 0, 4, 2, 1.5], [4.2, 0, math.pi, 4, 2, 1.5],
                      [30, 5, 0, 4, 2, 1.5], [34.1, 5, 0, 4, 2, 1.5]], np.float64)
    state = np.array([[0, 0, 0, 2.0], [4.2, 0, math.pi, 2.0], [30, 5, 0, 2.0]], np.float64)
    flags = np.zeros(3, np.uint8)
    oracle.step_world(boxes, state, flags, np.zeros((3, 2), np.float32), road)
    c = oracle.COLLIDED | oracle.HALTED
    assert list(flags) == [c, c, c]
    assert np.all(state[:, 3] == 0)
    assert boxes[3, 0] == 34.1  # static boxes never move


def test_bicycle_heading_uses_speed_at_step_start():
    """With constant steer and acceleration, the heading after n steps is
    theta0 + sin(beta)/l_r * dt * sum_k v_k with v_k the speed at the start of step k."""
    L, steer, a, dt, v0 = 4.4, 0.2, 1.3, 0.1, 3.0
    beta = math.atan(0.5 * math.tan(steer))
    st = (0.0, 0.0, 0.1, v0)
    n = 20
    for _ in range(n):
        st = oracle.bicycle(*st, L, a, steer, dt, 30.0)
    vs = [v0 + k * a * dt for k in range(n)]
    assert st[2] == pytest.approx(0.1 + math.sin(beta) / (0.3 * L) * dt * sum(vs), abs=1e-12)


def test_offroad_boundary_counts_as_inside():
    # corner exactly on the road edge (all values exact in binary): still on the road
    road = np.array([rect_quad(-50, 50, -3.5, 3.5)], np.float32)
    assert oracle.point_in_quad(10.0, 3.5, road[0]) and oracle.point_in_quad(50.0, 3.5, road[0])
    assert not oracle.point_in_quad(10.0, 3.5000001, road[0])
    boxes = np.array([[0, 2.5, 0, 4.0, 2.0, 1.5]], np.float64)
    state = np.array([[0, 2.5, 0, 0]], np.float64)
    flags = np.zeros(1, np.uint8)
    oracle.step_world(boxes, state, flags, np.zeros((1, 2), np.float32), road)
    assert flags[0] == 0


def test_visible_faces_of_a_box():
    """A viewpoint sees exactly the faces whose planes it is strictly in front of; a face
    whose plane contains the camera is edge-on (zero area) and is culled."""
    cam = CamConfig(64, 64)
    D, L, Wd, H = 9.0, 4.0, 2.0, 1.25
    # camera at y = 0 lies in the plane of the box's -y face (y = 0); top face below camera
    boxes = [ego_box(), [D + L / 2, Wd / 2, 0.0, L, Wd, H]]
    img, tris = render_scene(cam, boxes)
    faces = sorted({(int(p) - 12) // 2 for p in tris["prim"]})
    assert faces == [1, 4]  # -x face and +z (top) face; -y face edge-on, rest back-facing
    assert (img.cls == 3).any()


def test_ego_box_is_not_drawn():
    # a low ego box (top face below the camera) would cover the bottom of its own image
    cam = CamConfig(32, 32)
    img, tris = render_scene(cam, [[0.0, 0.0, 0.0, 4.5, 1.9, 1.4]])
    assert len(tris) == 0 and not img.cls.any()
    img2, tris2 = render_scene(cam, [[0.0, 0.0, 0.0, 4.5, 1.9, 1.4]], ego=-1)
    assert (img2.cls == 3).sum() > 100  # the same box drawn (no ego) shows its top face


def test_snapped_vertices_stay_inside_guard_band():
    """Guard-band clipping bounds every snapped coordinate to the band of 4x the viewport
    half-extent around its centre, which keeps edge functions inside 32-bit range."""
    import worldgen as wg
    w = wg.make_workload(wg.WORKLOADS["tiny"])
    sim = oracle.Sim(w)
    for W, H in ((64, 64), (256, 144)):
        cam = CamConfig(W, H)
        n_near = 0
        for a in range(8):
            for yaw in (0.0, 1.0, -1.0):
                t = sim.camera_tris(cam, 0, a, yaw)
                X, Y = t["X"].astype(np.int64), t["Y"].astype(np.int64)
                assert np.all(np.abs(X - 8 * W) <= 4 * 8 * W + 1)
                assert np.all(np.abs(Y - 8 * H) <= 4 * 8 * H + 1)
                n_near += int((np.abs(Y - 8 * H) > 3 * 8 * H).sum())
        assert n_near > 0  # some ground really is clipped by the guard band


# ---------------------------------------------------------------------------------------
# RGB observation: one directional light, a colour per class (closed forms)
# ---------------------------------------------------------------------------------------

def _rgb8(v):
    """Expected 8-bit channel value: round half to even of 255 * clamp(v, 0, 1)."""
    return int(np.rint(255.0 * min(max(v, 0.0), 1.0)))


def test_rgb_empty_scene_is_unshaded_background():
    cam = CamConfig(32, 24)
    boxes = [ego_box()]
    img, _ = render_scene(cam, boxes)
    col = ((0.2, 0.4, 0.6), (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, 0.0))
    rgb = oracle.shade_rgb(img.key, False, 12, 12, np.array(boxes), colour=col,
                           light=(0.0, 0.0, -1.0), ambient=0.1)
    assert rgb.shape == (3, 24, 32)
    for ch, v in enumerate((51, 102, 153)):  # 255 * (0.2, 0.4, 0.6), no light involved
        assert np.all(rgb[ch] == v)


@pytest.mark.parametrize("box_yaw,light,lit", [
    (0.0, (-0.6, 0.0, 0.8), 0.6),      # the visible face (-x of the box) faces the light
    (math.pi, (-0.6, 0.0, 0.8), 0.6),  # turned round: the box's +x face now faces the camera
    (0.0, (0.6, 0.0, 0.8), 0.0),       # light from behind the face: ambient only
    (math.pi, (0.6, 0.0, 0.8), 0.0),
])
def test_rgb_front_face_lambert(box_yaw, light, lit):
    W, H, D, hw, bh = 64, 64, Fraction(10), Fraction(1), Fraction(16, 10)
    cols, rows, margin = _box_face_expectation(W, H, D, hw, bh)
    assert margin >= Fraction(1, 16)
    L = 4.5
    boxes = [ego_box(), [float(D) + L / 2, 0.0, box_yaw, L, 2 * float(hw), float(bh)]]
    img, _ = render_scene(CamConfig(W, H), boxes)
    face = np.zeros((H, W), bool)
    face[rows[0]:rows[-1] + 1, cols[0]:cols[-1] + 1] = True
    assert np.array_equal(img.cls == 3, face)
    bg, blue, ambient = (0.5, 0.5, 0.5), (0.1, 0.3, 0.9), 0.25
    col = (bg, (0.3, 0.3, 0.3), (0.9, 0.9, 0.9), blue)
    rgb = oracle.shade_rgb(img.key, False, 24, 24, np.array(boxes), colour=col, light=light,
                           ambient=ambient)
    shade = ambient + (1.0 - ambient) * lit
    for ch in range(3):
        assert np.all(rgb[ch][face] == _rgb8(blue[ch] * shade))
        assert np.all(rgb[ch][~face] == _rgb8(bg[ch]))


def test_rgb_ground_is_lit_from_above():
    """Road pieces are horizontal: their shade is ambient + (1 - ambient) * l_z."""
    W, H = 48, 32
    boxes = [ego_box()]
    road = [rect_quad(-5.0, 200.0, -3.5, 3.5)]
    img, _ = render_scene(CamConfig(W, H), boxes, road=road)
    ground = img.cls == 1
    assert ground.sum() > 100
    light = oracle.unit((0.5, -0.2, 0.7))
    col = ((0.0, 0.0, 0.0), (0.4, 0.5, 0.6), (1.0, 1.0, 1.0), (0.0, 0.0, 1.0))
    rgb = oracle.shade_rgb(img.key, False, 12, 14, np.array(boxes), colour=col, light=light,
                           ambient=0.3)
    shade = 0.3 + 0.7 * float(light[2])
    for ch in range(3):
        assert np.all(rgb[ch][ground] == _rgb8(col[1][ch] * shade))
        assert np.all(rgb[ch][~ground] == 0)


def test_rgb_side_face_normal_follows_box_yaw():
    """A box seen from its side: its +y face (normal (-sin yaw, cos yaw, 0)) faces a camera
    placed on the box's +y side; a light along that normal gives full shade."""
    W, H = 64, 64
    yaw = 0.7
    n = np.array([-math.sin(yaw), math.cos(yaw), 0.0])
    centre = np.array([0.0, 0.0])
    cam_pos = centre + 12.0 * n[:2]
    cam_heading = math.atan2(-n[1], -n[0])  # looking back at the box along -n
    boxes = [ego_box(cam_pos[0], cam_pos[1], cam_heading), [0.0, 0.0, yaw, 4.5, 1.9, 1.6]]
    img, _ = render_scene(CamConfig(W, H), boxes, pose=(cam_pos[0], cam_pos[1], cam_heading))
    side = img.cls == 3
    assert side.sum() > 20
    col = ((0.0, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), (0.2, 0.6, 1.0))
    rgb = oracle.shade_rgb(img.key, False, 24, 24, np.array(boxes), colour=col,
                           light=tuple(n), ambient=0.5)
    prim = 0xFFFFFFFF - (img.key[side] & 0xFFFFFFFF).astype(np.uint64)
    faces = set(((prim % 12) // 2).tolist())
    assert faces == {2}  # only the +y face is visible
    for ch in range(3):
        assert np.all(rgb[ch][side] == _rgb8(col[3][ch]))


# ---------------------------------------------------------------------------------------
# Reward terms (Table "Reward terms") and ego state: closed forms on a two-lane road
# ---------------------------------------------------------------------------------------

W_INF = oracle.REWARD_WEIGHTS  # collision, off-road, comfort, alignment, centering,
#                                velocity, traffic light, time, reverse, overspeed
STRAIGHT = np.array([rect_quad(-100.0, 100.0, -3.5, 3.5)], np.float32)  # runs along +x


def _reward_step(y, yaw, v0, accel=0.0, steer=0.0, fl_after=0, fl_before=0, acc=(0.0, 0.0),
                 road=STRAIGHT, x=0.0, L=4.5, Wd=1.9, weights=W_INF):
    before = np.array([[x, y, yaw, v0]], np.float64)
    after = before.copy()
    if not fl_before & 4:
        after[0] = oracle.bicycle(x, y, yaw, v0, L, accel, steer)
    if fl_after & 3:
        after[0, 3] = 0.0  # halted this step
    a = np.array([acc], np.float64)
    r, ego = oracle.rewards_world(before, [fl_before], after, [fl_after | (4 if fl_after & 3 else 0)],
                                  [[accel, steer]], [[L, Wd]], a, [weights], road)
    return float(r[0]), ego[0], a[0]


def _lane_terms(theta, v, xf, dt=0.1, w=W_INF):
    ct = math.cos(theta)
    aln = w[3] * dt * (min(ct, 0.0) + min(v * ct, 0.0) + 0.0025 * (1 - 2 * theta / math.pi))
    ctr = -w[4] * dt * ((abs(xf) if ct > 0.5 else 0.0) - 0.05 * math.exp(0.5 - abs(xf)))
    vel = w[5] * dt * max(ct, 0.0) if abs(v) > 2.5 else 0.0
    return aln + ctr + vel


def test_reward_cruising_in_lane():
    r, _, _ = _reward_step(-1.75, 0.0, 10.0)
    assert r == pytest.approx(_lane_terms(0.0, 10.0, 0.0) - W_INF[7] * 0.1, rel=1e-12, abs=1e-15)


def test_reward_wrong_way_lane():
    # right-hand traffic: the left half of the road runs against the quad's direction
    r, _, _ = _reward_step(+1.75, 0.0, 10.0)
    assert r == pytest.approx(_lane_terms(math.pi, 10.0, 0.0) - W_INF[7] * 0.1, rel=1e-12)
    assert r < -0.02  # wrong-way driving is penalised


def test_reward_lateral_offset_and_misalignment():
    r, _, _ = _reward_step(-1.75 + 0.6, -0.2, 10.0)
    th, xf = 0.2, 0.6 + 10.0 * math.sin(-0.2) * 0.1  # the step moves the agent sideways
    assert r == pytest.approx(_lane_terms(th, 10.0, xf) - W_INF[7] * 0.1, rel=1e-9)


def test_reward_slow_agent_gets_no_velocity_term():
    r, _, _ = _reward_step(-1.75, 0.0, 2.0)
    assert r == pytest.approx(_lane_terms(0.0, 2.0, 0.0) - W_INF[7] * 0.1, rel=1e-12)
    assert _lane_terms(0.0, 2.0, 0.0) < _lane_terms(0.0, 3.0, 0.0)


def test_reward_harsh_braking_and_jerk():
    r, ego, acc = _reward_step(-1.75, 0.0, 10.0, accel=-5.0)
    assert acc[0] == pytest.approx(-5.0) and acc[1] == 0.0
    base = _lane_terms(0.0, 9.5, 0.0) - W_INF[7] * 0.1
    assert r == pytest.approx(base - 2 * W_INF[2], rel=1e-9)  # |a_lon| > 3 and jerk > 5
    # the same deceleration again: no jerk, still harsh
    r2, _, _ = _reward_step(-1.75, 0.0, 10.0, accel=-5.0, acc=(-5.0, 0.0))
    assert r2 == pytest.approx(base - W_INF[2], rel=1e-9)
    assert ego[1] == pytest.approx(-0.5)


def test_reward_collision_scales_with_speed_and_offroad():
    r, ego, _ = _reward_step(-1.75, 0.0, 10.0, fl_after=1)
    assert r == pytest.approx(_lane_terms(0.0, 10.0, 0.0) - W_INF[7] * 0.1 - (W_INF[0] + 0.1 * 10.0),
                              rel=1e-9)
    assert ego[5] == 1.0 and ego[0] == 0.0  # collided; speed zeroed by the halt
    r, _, _ = _reward_step(50.0, 0.0, 10.0, fl_after=2)  # off the road: no lane terms
    assert r == pytest.approx(-W_INF[1] - W_INF[7] * 0.1, rel=1e-12)


def test_reward_halted_agent_earns_nothing():
    r, ego, acc = _reward_step(-1.75, 0.0, 0.0, fl_before=4 | 1, fl_after=4 | 1, acc=(3.0, 1.0))
    assert r == 0.0 and acc[0] == 0.0 and acc[1] == 0.0
    assert ego[5] == 1.0


def test_lane_frame_follows_road_direction():
    phi = 0.9
    c, s = math.cos(phi), math.sin(phi)
    local = [(-20, -3.5), (20, -3.5), (20, 3.5), (-20, 3.5)]
    quad = np.array([[v for (u, w) in local for v in (u * c - w * s, u * s + w * c)]], np.float32)
    for lat, want_dir, want_xf in ((-1.75, phi, 0.0), (-1.0, phi, 0.75), (2.0, phi - math.pi, 0.25)):
        px, py = -lat * s, lat * c
        d, xf = oracle.lane_frame(px, py, quad)
        assert math.cos(d - want_dir) == pytest.approx(1.0, abs=1e-9)
        assert xf == pytest.approx(want_xf, abs=1e-6)
    assert oracle.lane_frame(100.0, 100.0, quad) is None


def test_ego_state_normalisation():
    _, ego, _ = _reward_step(-1.75, 0.0, 15.0, accel=1.0, L=4.2, Wd=1.8)
    assert ego[0] == pytest.approx(15.1 / 30.0)
    assert ego[1] == pytest.approx(0.1) and ego[2] == 0.0
    assert ego[3] == pytest.approx(0.42) and ego[4] == pytest.approx(0.36) and ego[5] == 0.0


# ---------------------------------------------------------------------------------------
# Ray-traced view: closed forms and the independent NumPy ray caster above
# ---------------------------------------------------------------------------------------

def trace_scene(cam, boxes, road=(), line=(), pose=(0.0, 0.0, 0.0), cam_yaw=0.0, ego=0):
    b = np.array(boxes, np.float64).reshape(-1, 6)
    rd = np.array(road, np.float32).reshape(-1, 8)
    ln = np.array(line, np.float32).reshape(-1, 8)
    return oracle.trace_view(cam, b, ego, rd, ln, pose[0], pose[1], pose[2], cam_yaw)


@pytest.mark.parametrize("W,H,D,hw,bh", _generic_box_cases())
def test_trace_box_face_rectangle(W, H, D, hw, bh):
    cols, rows, margin = _box_face_expectation(W, H, D, hw, bh)
    L = 4.2
    tr = trace_scene(CamConfig(W, H), [ego_box(), [float(D) + L / 2, 0.0, 0.0, L, 2 * float(hw), float(bh)]])
    expect = np.zeros((H, W), bool)
    expect[rows[0]:rows[-1] + 1, cols[0]:cols[-1] + 1] = True
    assert np.array_equal(tr.cls == 3, expect) and np.array_equal(tr.cls != 0, expect)
    assert np.all(tr.depth[expect] == np.float32(0.1 / float(D)))
    assert np.all(tr.prim[expect] == 12 * 1 + 2 * 1)  # box 1, its -x face
    assert np.all(tr.prim[~expect] == 0xFFFFFFFF) and np.all(tr.depth[~expect] == 0)


def test_trace_ground_rows_and_lines_above_road():
    W = H = 64
    f, h, n, r = 32.0, 1.5, 0.1, 1.3137
    road = [rect_quad(-5.0, 200.0, -r, r)]
    line = [rect_quad(-5.0, 200.0, -0.075, 0.075)]
    tr = trace_scene(CamConfig(W, H), [ego_box()], road=road, line=line)
    u = np.arange(W) + 0.5
    v = np.arange(H) + 0.5 - H / 2
    for j in range(H):
        if v[j] <= 0:
            assert not tr.cls[j].any()
            continue
        half = r / h * v[j]
        sure = np.abs(np.abs(u - W / 2) - half) > 1e-6
        inside = np.abs(u - W / 2) < half
        assert np.array_equal(tr.cls[j][sure] != 0, inside[sure])
        road_px = tr.cls[j] == 1
        assert np.allclose(tr.depth[j][road_px], n * v[j] / (f * h), rtol=1e-6)
        # the lane line (raised by line_z) is nearer: its depth is n (v - H/2 ...) / (f (h - z))
        line_px = tr.cls[j] == 2
        assert np.allclose(tr.depth[j][line_px], n * v[j] / (f * (h - 0.02)), rtol=1e-6)
    assert (tr.cls == 2).sum() > 20


def test_trace_entry_faces_follow_box_yaw():
    W, H, L = 64, 64, 4.5
    # the face whose outward normal points back at the camera (along -x): -x at yaw 0, +x
    # at yaw pi, +y (normal (-sin, cos)) at yaw pi/2, -y at yaw -pi/2
    for yaw, face in ((0.0, 1), (math.pi, 0), (math.pi / 2, 2), (-math.pi / 2, 3)):
        tr = trace_scene(CamConfig(W, H), [ego_box(), [10.0 + L / 2, 0.0, yaw, L, 1.9, 1.6]])
        hit = tr.cls == 3
        assert hit.sum() > 20
        assert set(((tr.prim[hit] - 12) // 2).tolist()) == {face}


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("W,H", [(16, 16), (40, 24)])
def test_trace_equals_numpy_raycast(seed, W, H):
    rng = np.random.default_rng(300 + seed)
    boxes, road, line = _random_scene(rng)
    cam_yaw = rng.uniform(-0.3, 0.3)
    tr = trace_scene(CamConfig(W, H), boxes, road, line, cam_yaw=cam_yaw)
    cls0, d0, obj0 = raycast(W, H, boxes, 0, road, line, (0, 0, 0), cam_yaw)
    assert np.array_equal(tr.cls, cls0)
    assert np.allclose(tr.depth, d0.astype(np.float32), rtol=1e-6, atol=0)
    nb, nr = len(boxes), len(road)
    box = cls0 == 3
    assert np.array_equal((tr.prim[box] // 12), obj0[box])
    rd = cls0 == 1
    assert np.array_equal((tr.prim[rd] - 12 * nb) // 2, obj0[rd] - 1000)
    ln = cls0 == 2
    assert np.array_equal((tr.prim[ln] - 12 * nb - 2 * nr) // 2, obj0[ln] - 100000)


def test_trace_ignores_boxes_behind_the_camera():
    """A box behind the camera (or nearer than the near plane along the ray) is not hit."""
    W = H = 32
    tr = trace_scene(CamConfig(W, H), [ego_box(), [-10.0, 0.0, 0.3, 4.5, 1.9, 1.6],
                                       [-6.0, 1.0, 0.0, 4.5, 1.9, 2.5]])
    assert not tr.cls.any() and np.all(tr.prim == 0xFFFFFFFF)


def test_trace_overlapping_road_quads_tie_to_lower_index():
    W = H = 32
    road = [rect_quad(-5.0, 100.0, -4.0, 4.0), rect_quad(-5.0, 100.0, -4.0, 4.0),
            rect_quad(0.0, 50.0, -2.0, 3.0)]  # inside quad 0
    tr = trace_scene(CamConfig(W, H), [ego_box()], road=road)
    rd = tr.cls == 1
    assert rd.sum() > 100
    assert np.all(tr.prim[rd] == 12)  # road quad 0 wins every tie


# ---------------------------------------------------------------------------------------
# Vectorized observations O_vec: hand-computed slots and an independent brute force
# ---------------------------------------------------------------------------------------

def test_ovec_agents_in_ego_frame():
    # ego at the origin facing +y: world +y is ego-forward (x), world -x is ego-left (y)
    boxes = [[0.0, 0.0, math.pi / 2, 4.5, 1.9, 1.5],
             [0.0, 20.0, math.pi / 2 + 0.3, 4.2, 1.8, 1.5],   # 20 m ahead
             [-10.0, 0.0, 0.0, 4.0, 2.0, 1.6],                 # 10 m to the left
             [0.0, -100.5, 0.0, 4.0, 2.0, 1.6]]                # beyond 100 m
    speed = [10.0, 12.0, 0.0, 0.0]
    ao, _ = oracle.observe_world(boxes, speed, np.zeros((0, 8)), np.zeros((0, 8)), n_agents=1)
    s = ao[0]
    # nearest: the box 10 m to the left (heading 0 = -90 deg relative to the ego)
    assert s[0] == pytest.approx([1, 0.0, 10 / 100, 0.4, 2.0 / 5, 0.0, -1.0, -10 / 30], abs=1e-12)
    assert s[1] == pytest.approx([1, 0.2, 0.0, 0.42, 0.36, math.cos(0.3), math.sin(0.3), 2 / 30], abs=1e-12)
    assert not s[2:].any()


def test_ovec_ties_and_truncation():
    boxes = [[0.0, 0.0, 0.0, 4.5, 1.9, 1.5]] + [[10.0 * math.cos(a), 10.0 * math.sin(a), 0.0, 4.0, 2.0, 1.5]
                                                for a in np.linspace(0, 2 * math.pi, 20, endpoint=False)]
    ao, _ = oracle.observe_world(boxes, np.zeros(21), np.zeros((0, 8)), np.zeros((0, 8)), K=16,
                                 n_agents=1)
    # all at 10 m (to rounding): the 16 lowest indices after nearest-first ordering
    x = ao[0, :, 1] * 100
    y = ao[0, :, 2] * 100
    assert np.allclose(np.hypot(x, y), 10.0)
    ang = np.arctan2(y, x) % (2 * math.pi)
    assert ao[0, :, 0].all() and len(set(np.round(ang, 6))) == 16


def test_ovec_road_segment_features():
    road = np.array([rect_quad(-20.0, 20.0, -3.5, 3.5)], np.float32)
    line = np.array([rect_quad(-20.0, 20.0, -0.075, 0.075), rect_quad(100.0, 140.0, -0.1, 0.1)],
                    np.float32)
    boxes = [[5.0, 1.0, math.pi, 4.5, 1.9, 1.5]]
    _, ro = oracle.observe_world(boxes, [0.0], road, line, n_agents=1)
    r = ro[0]
    # midpoint (0, 0) seen from (5, 1) facing -x: 5 m ahead, 1 m to the right
    assert r[0] == pytest.approx([1, 5 / 30, 1 / 30, 40 / 30, -1.0, 0.0, 1, 0], abs=1e-6)
    assert r[1] == pytest.approx([1, 5 / 30, 1 / 30, 40 / 30, -1.0, 0.0, 0, 1], abs=1e-6)
    assert not r[2:].any()  # the far line is beyond 30 m


@pytest.mark.parametrize("seed", range(3))
def test_ovec_matches_numpy_brute_force(seed):
    rng = np.random.default_rng(500 + seed)
    nb = 40
    boxes = np.column_stack([rng.uniform(-120, 120, nb), rng.uniform(-120, 120, nb),
                             rng.uniform(-math.pi, math.pi, nb), rng.uniform(4, 5, nb),
                             rng.uniform(1.8, 2, nb), rng.uniform(1.4, 1.7, nb)])
    speed = rng.uniform(0, 20, nb)
    def quads(n):
        c = rng.uniform(-60, 60, (n, 2))
        h = rng.uniform(-math.pi, math.pi, n)
        L, Wd = rng.uniform(5, 30, n), rng.uniform(0.1, 7, n)
        out = []
        for (cx, cy), hh, l, w in zip(c, h, L, Wd):
            cc, ss = math.cos(hh), math.sin(hh)
            pts = [(-l / 2, -w / 2), (l / 2, -w / 2), (l / 2, w / 2), (-l / 2, w / 2)]
            out.append([v for (a, b) in pts for v in (cx + cc * a - ss * b, cy + ss * a + cc * b)])
        return np.array(out, np.float32)
    road, line = quads(60), quads(90)
    na = 12
    ao, ro = oracle.observe_world(boxes, speed, road, line, n_agents=na)
    segs = np.concatenate([road, line]).astype(np.float64).reshape(-1, 4, 2)
    a = 0.5 * (segs[:, 0] + segs[:, 3])
    b = 0.5 * (segs[:, 1] + segs[:, 2])
    mid, vec = 0.5 * (a + b), b - a
    for i in range(na):
        x, y, th = boxes[i, :3]
        c, s = math.cos(th), math.sin(th)
        d = np.hypot(boxes[:, 0] - x, boxes[:, 1] - y)
        order = [j for j in np.lexsort((np.arange(nb), d)) if j != i and d[j] <= 100][:16]
        for k, j in enumerate(order):
            dx, dy = boxes[j, 0] - x, boxes[j, 1] - y
            want = [1, (dx * c + dy * s) / 100, (-dx * s + dy * c) / 100, boxes[j, 3] / 10,
                    boxes[j, 4] / 5, math.cos(boxes[j, 2] - th), math.sin(boxes[j, 2] - th),
                    (speed[j] - speed[i]) / 30]
            assert ao[i, k] == pytest.approx(want, abs=1e-9)
        assert not ao[i, len(order):].any()
        dm = np.hypot(mid[:, 0] - x, mid[:, 1] - y)
        sel = [q for q in np.lexsort((np.arange(len(dm)), dm)) if dm[q] <= 30][:32]
        for k, q in enumerate(sel):
            dx, dy = mid[q, 0] - x, mid[q, 1] - y
            phi = math.atan2(vec[q, 1], vec[q, 0])
            want = [1, (dx * c + dy * s) / 30, (-dx * s + dy * c) / 30,
                    math.hypot(*vec[q]) / 30, math.cos(phi - th), math.sin(phi - th),
                    float(q < 60), float(q >= 60)]
            assert ro[i, k] == pytest.approx(want, abs=1e-9)
        assert not ro[i, len(sel):].any()


# ---------------------------------------------------------------------------------------
# Jerk-actuated bicycle (App. A "Action Space and Dynamics"): closed forms of the
# integration chain jerk -> acceleration -> speed / steering, its limits and symmetry
# ---------------------------------------------------------------------------------------

def _jerk_roll(j_lon, j_lat, n, v0=0.0, L=4.5, st0=(0.0, 0.0, 0.0), yaw0=0.0):
    st = np.array(st0, np.float64)
    x, y, yaw, v = 0.0, 0.0, yaw0, v0
    traj = []
    for _ in range(n):
        x, y, yaw, v = oracle.jerk_bicycle(x, y, yaw, v, L, j_lon, j_lat, st)
        traj.append((x, y, yaw, v, *st))
    return np.array(traj)


def test_jerk_action_set_is_the_papers_twelve():
    assert len(oracle.JERK_ACTIONS) == 12
    assert sorted({a for a, _ in oracle.JERK_ACTIONS}) == [-15.0, -4.0, 0.0, 4.0]
    assert sorted({b for _, b in oracle.JERK_ACTIONS}) == [-4.0, 0.0, 4.0]


def test_jerk_zero_from_rest_state_is_straight_cruise():
    t = _jerk_roll(0.0, 0.0, 20, v0=12.0)
    assert np.all(t[:, 3] == 12.0) and np.all(t[:, 1] == 0.0) and np.all(t[:, 2] == 0.0)
    assert t[-1, 0] == pytest.approx(20 * 12.0 * 0.1, rel=1e-12)


def test_jerk_longitudinal_ramp_and_acceleration_limit():
    # a_k = min(0.4 k, 3): 0.4 .. 2.8 over seven steps, then held at the 3 m/s^2 limit
    n = 12
    t = _jerk_roll(4.0, 0.0, n)
    a = np.minimum(0.4 * np.arange(1, n + 1), 3.0)
    assert np.allclose(t[:, 4], a, atol=1e-12)
    v = np.cumsum(a) * 0.1  # speed after each step (Euler on the new acceleration)
    assert np.allclose(t[:, 3], v, atol=1e-12)
    # positions advance with the speed at the start of each step
    x = np.cumsum(np.concatenate([[0.0], v[:-1]])) * 0.1
    assert np.allclose(t[:, 0], x, atol=1e-12)
    assert t[6, 3] == pytest.approx(1.12, abs=1e-12)  # sum 0.4 .. 2.8 = 11.2 -> 1.12 m/s


def test_jerk_hard_braking_hits_the_deceleration_limit_and_stops():
    t = _jerk_roll(-15.0, 0.0, 30, v0=10.0)
    assert t[0, 4] == pytest.approx(-1.5) and t[1, 4] == pytest.approx(-3.0)
    assert t[2, 4] == pytest.approx(-4.5) and np.all(t[3:, 4] == -5.0)
    assert t[1, 3] == pytest.approx(10.0 - 0.15 - 0.30)
    assert np.all(np.diff(t[:, 3]) <= 0.0) and t[-1, 3] == 0.0  # no reversing


def test_jerk_steering_rate_and_angle_bounds():
    # at walking pace the curvature target exceeds every bound: the steering angle moves
    # by exactly 0.05 rad (0.5 rad/s x 0.1 s) per step and then holds at 0.5 rad
    t = _jerk_roll(0.0, 4.0, 14, v0=0.5)
    steer = t[:, 6]
    assert np.allclose(steer[:10], 0.05 * np.arange(1, 11), atol=1e-12)
    assert np.allclose(steer[9:], 0.5, atol=1e-12) and np.all(steer <= 0.5)
    assert np.all(np.abs(t[:, 5]) <= 4.0) and t[-1, 5] == 4.0  # lateral limit


def test_jerk_lateral_acceleration_is_realised_on_the_bicycle():
    # at speed the steering settles to the curvature kappa = a_lat / v^2; the bicycle's
    # yaw rate v sin(beta) / l_r then reproduces a_lat up to the small-angle error
    v, L = 20.0, 4.5
    t = _jerk_roll(0.0, 4.0, 5, v0=v, L=L)  # a_lat ramps 0.4 .. 2.0
    st = np.array([0.0, 2.0, t[-1, 6]], np.float64)
    x, y, yaw, vv = oracle.jerk_bicycle(0.0, 0.0, 0.0, v, L, 0.0, 0.0, st)
    assert st[1] == pytest.approx(2.0)
    kappa = 2.0 / v ** 2
    assert st[2] == pytest.approx(math.atan(kappa * 0.6 * L), rel=1e-12)
    a_lat = v * (yaw / 0.1)
    assert a_lat == pytest.approx(2.0, rel=2e-4)


def test_jerk_mirror_symmetry():
    a = _jerk_roll(4.0, 4.0, 25, v0=8.0)
    b = _jerk_roll(4.0, -4.0, 25, v0=8.0)
    assert np.allclose(a[:, 0], b[:, 0], atol=1e-12) and np.allclose(a[:, 3], b[:, 3], atol=1e-12)
    assert np.allclose(a[:, 1], -b[:, 1], atol=1e-12) and np.allclose(a[:, 2], -b[:, 2], atol=1e-12)
    assert np.allclose(a[:, 6], -b[:, 6], atol=1e-12) and np.allclose(a[:, 5], -b[:, 5], atol=1e-12)
    assert a[-1, 1] > 1.0  # it did turn left


def test_jerk_step_world_halted_agent_resets_actuators():
    # two agents in one world; the second starts halted: it neither moves nor keeps
    # its actuator state, the first follows jerk_bicycle exactly
    road = np.array([rect_quad(-100.0, 100.0, -10.0, 10.0)], np.float32)
    boxes = np.array([[0.0, -5.0, 0.0, 4.5, 1.9, 1.6], [0.0, 5.0, 0.0, 4.5, 1.9, 1.6]], np.float64)
    state = np.array([[0.0, -5.0, 0.0, 5.0], [0.0, 5.0, 0.0, 0.0]], np.float64)
    flags = np.array([0, 4 | 1], np.uint8)
    jerk = np.array([[0.5, 0.2, 0.01], [1.0, 1.0, 0.3]], np.float64)
    oracle.step_world(boxes, state, flags, np.array([[4.0, -4.0], [4.0, 4.0]], np.float32), road,
                      jerk=jerk)
    st = np.array([0.5, 0.2, 0.01])
    want = oracle.jerk_bicycle(0.0, -5.0, 0.0, 5.0, 4.5, 4.0, -4.0, st)
    assert np.allclose(state[0], want, atol=1e-12) and np.allclose(jerk[0], st, atol=1e-15)
    assert np.all(jerk[1] == 0.0) and np.all(state[1] == [0.0, 5.0, 0.0, 0.0])
    assert flags[0] == 0


def test_jerk_ego_extras():
    before = np.array([[0.0, -1.75, 0.0, 10.0]], np.float64)
    after = before.copy()
    after[0] = oracle.bicycle(0.0, -1.75, 0.0, 10.0, 4.5, -2.5, 0.1)
    _, ego = oracle.rewards_world(before, [0], after, [0], [[-2.5, 0.1]], [[4.5, 1.9]],
                                  np.zeros((1, 2)), [W_INF], STRAIGHT, jerk=[[-2.5, 2.0, 0.1]])
    assert ego[0, 6] == pytest.approx(0.2) and ego[0, 7] == pytest.approx(-0.5)
    assert ego[0, 8] == pytest.approx(0.5)
    _, ego = oracle.rewards_world(before, [0], after, [0], [[-2.5, 0.1]], [[4.5, 1.9]],
                                  np.zeros((1, 2)), [W_INF], STRAIGHT)
    assert np.all(ego[0, 6:] == 0.0)


# ---------------------------------------------------------------------------------------
# Traffic-signal spheres (Sec. 3.1 / App. A third primitive): the drawn polyhedron lies
# between its inscribed and circumscribed spheres; faces, depth and ids against an
# independent ray/triangle intersection; shading against the faces' closed-form normals
# ---------------------------------------------------------------------------------------

SPH_IN = 0.8628  # inscribed-sphere radius of the 4 x 8 polyhedron, in units of r (below the exact 0.86286)


def _rays(W, H, psi, jx=0.0, jy=0.0, hfov=math.pi / 2):
    f = (W / 2) / math.tan(hfov / 2)
    xv = ((np.arange(W) + 0.5 + jx - W / 2) / f)[None, :, None]
    yv = (-(np.arange(H) + 0.5 + jy - H / 2) / f)[:, None, None]
    right = np.array([math.sin(psi), -math.cos(psi), 0.0])
    fwd = np.array([math.cos(psi), math.sin(psi), 0.0])
    return np.broadcast_to(xv * right + yv * np.array([0.0, 0.0, 1.0]) + fwd, (H, W, 3))


def _sphere_entry(O, D, c, R):
    """Entry parameter of rays O + t D into the sphere (c, R); nan where they miss."""
    oc = O - np.asarray(c, np.float64)
    a = np.einsum("hwk,hwk->hw", D, D)
    b = 2.0 * np.einsum("hwk,k->hw", D, oc)
    cc = float(oc @ oc) - R * R
    disc = b * b - 4 * a * cc
    with np.errstate(invalid="ignore"):
        return np.where(disc >= 0, (-b - np.sqrt(disc)) / (2 * a), np.nan)


def _fmin(arrays):
    out = arrays[0]
    for a in arrays[1:]:
        out = np.fmin(out, a)
    return out


def _sphere_mesh(c, r):
    """The polyhedron's quads from its definition: [32, 4, 3] corners."""
    def V(i, j):
        th, ph = -math.pi / 2 + i * math.pi / 4, (j % 8) * math.pi / 4
        ct = 0.0 if i in (0, 4) else math.cos(th)
        return np.array([c[0] + r * ct * math.cos(ph), c[1] + r * ct * math.sin(ph), c[2] + r * math.sin(th)])
    return np.array([[V(q // 8, q % 8), V(q // 8, q % 8 + 1), V(q // 8 + 1, q % 8 + 1), V(q // 8 + 1, q % 8)]
                     for q in range(32)])


def _mt_cast(O, D, quads):
    """Nearest hit per ray over the quads' triangles (Moller-Trumbore): (t, quad, edge
    margin = smallest barycentric coordinate), t = inf on a miss."""
    H, W, _ = D.shape
    best = np.full((H, W), np.inf)
    bq = np.full((H, W), -1)
    marg = np.zeros((H, W))
    for q, c in enumerate(quads):
        for tri in ((c[0], c[1], c[2]), (c[0], c[2], c[3])):
            e1, e2 = tri[1] - tri[0], tri[2] - tri[0]
            if np.linalg.norm(np.cross(e1, e2)) < 1e-12:
                continue  # degenerate pole triangle
            pv = np.cross(D, e2)
            det = pv @ e1
            with np.errstate(divide="ignore", invalid="ignore"):
                inv = 1.0 / det
                tv = O - tri[0]
                u = np.einsum("hwk,k->hw", pv, tv) * inv
                qv = np.cross(tv, e1)
                v = (D @ qv) * inv
                t = (qv @ e2) * inv
            ok = (np.abs(det) > 1e-15) & (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 0) & (t < best)
            best[ok], bq[ok] = t[ok], q
            marg[ok] = np.minimum(np.minimum(u, v), 1 - u - v)[ok]
    return best, bq, marg


SPH_SCENE = dict(boxes=[ego_box()], sph=np.array([[5.0, 0.6, 2.0, 1.8], [12.0, -2.5, 1.2, 1.0],
                                                   [7.0, -3.2, 4.2, 1.2]]))


@pytest.mark.parametrize("W,H,yaw", [(48, 48, 0.0), (64, 40, 0.15), (40, 24, -0.2)])
def test_signal_sphere_between_insphere_and_circumsphere(W, H, yaw):
    cam = CamConfig(W, H)
    sph = SPH_SCENE["sph"]
    img, _ = render_scene(cam, SPH_SCENE["boxes"], cam_yaw=yaw, sph=sph)
    tr = oracle.trace_view(cam, np.array(SPH_SCENE["boxes"], np.float64), 0, np.zeros((0, 8)),
                           np.zeros((0, 8)), 0.0, 0.0, 0.0, yaw, sph=sph)
    O = np.array([0.0, 0.0, 1.5])
    D = _rays(W, H, yaw)
    t_in = _fmin([_sphere_entry(O, D, s[:3], SPH_IN * s[3]) for s in sph])
    t_out = _fmin([_sphere_entry(O, D, s[:3], s[3]) for s in sph])
    inner, outer = np.isfinite(t_in), np.isfinite(t_out)
    assert inner.sum() > 100
    # ray tracing: exact containment
    assert np.all(tr.cls[inner] == 4) and not np.any(tr.cls[~outer])
    hit = tr.cls == 4
    with np.errstate(divide="ignore"):
        assert np.all(tr.depth[hit] <= 0.1 / t_out[hit] * (1 + 1e-6))
        assert np.all(tr.depth[inner] >= 0.1 / t_in[inner] * (1 - 1e-6))
    # raster: the same up to snapping (1/32 px per axis): use spheres 3 % apart
    t_in2 = _fmin([_sphere_entry(O, D, s[:3], 0.97 * SPH_IN * s[3]) for s in sph])
    t_out2 = _fmin([_sphere_entry(O, D, s[:3], 1.03 * s[3]) for s in sph])
    assert np.all(img.cls[np.isfinite(t_in2)] == 4) and not np.any(img.cls[~np.isfinite(t_out2)])
    near = np.isfinite(t_in2)
    assert np.all(img.depth[near] >= 0.1 / t_in2[near] * (1 - 1e-3))
    assert np.all(img.depth[near] <= 0.1 / t_out2[near] * (1 + 1e-3))


@pytest.mark.parametrize("W,H,yaw", [(48, 48, 0.0), (56, 32, 0.1)])
def test_signal_faces_against_ray_triangle_intersection(W, H, yaw):
    """Trace: every ray class, depth and entry quad as Moller-Trumbore on the mesh; raster:
    the drawn quad at every pixel whose neighbourhood (+-1/16 px) hits one quad only."""
    cam = CamConfig(W, H)
    sph = SPH_SCENE["sph"]
    quads = np.concatenate([_sphere_mesh(s[:3], s[3]) for s in sph])
    O = np.array([0.0, 0.0, 1.5])
    t, q, marg = _mt_cast(O, _rays(W, H, yaw), quads)
    tr = oracle.trace_view(cam, np.array(SPH_SCENE["boxes"], np.float64), 0, np.zeros((0, 8)),
                           np.zeros((0, 8)), 0.0, 0.0, 0.0, yaw, sph=sph)
    hit = np.isfinite(t)
    assert np.array_equal(tr.cls == 4, hit)
    assert np.allclose(tr.depth[hit], (0.1 / t[hit]).astype(np.float32), rtol=1e-6)
    base = 12  # one box, no ground quads
    rel = tr.prim[hit].astype(np.int64) - base
    clear = marg[hit] > 1e-6
    assert np.array_equal((rel // 64 * 32 + rel % 64 // 2)[clear], q[hit][clear])
    img, _ = render_scene(cam, SPH_SCENE["boxes"], cam_yaw=yaw, sph=sph)
    same = hit.copy()
    for jx, jy in ((1 / 16, 0), (-1 / 16, 0), (0, 1 / 16), (0, -1 / 16)):
        _, qj, _ = _mt_cast(O, _rays(W, H, yaw, jx, jy), quads)
        same &= qj == q
    assert same.sum() > 200
    full = 0xFFFFFFFF
    prim = full - (img.key & np.uint64(0xFFFFFFFF)).astype(np.int64)
    rel = prim[same] - base
    assert np.all(img.cls[same] == 4)
    assert np.array_equal(rel // 64 * 32 + rel % 64 // 2, q[same])
    # a pole-band quad has one drawn triangle: the trace reports that triangle's id
    pole = same & clear_map(hit, clear) & ((q % 32 < 8) | (q % 32 >= 24))
    assert pole.sum() >= 5
    assert np.array_equal(prim[pole], tr.prim[pole].astype(np.int64))


def test_signal_prim_ids_follow_lane_lines():
    cam = CamConfig(48, 48)
    road = [rect_quad(1.0, 30.0, -4.0, 4.0), rect_quad(30.0, 60.0, -4.0, 4.0)]
    line = [rect_quad(1.0, 60.0, -0.1, 0.1)]
    boxes = [ego_box(), [20.0, 5.0, 0.3, 4.5, 1.9, 1.6]]
    sph = np.array([[9.0, 0.0, 3.0, 0.8], [16.0, 1.0, 3.5, 0.8]])
    _, tris = render_scene(cam, boxes, road, line, sph=sph)
    _, plain = render_scene(cam, boxes, road, line)
    base = 12 * 2 + 2 * 2 + 2 * 1
    # the spheres add ids [base, base + 128) only; every other triangle is unchanged
    assert np.array_equal(tris[tris["prim"] < base], plain)
    sp = tris["prim"][tris["prim"] >= base].astype(np.int64) - base
    assert set(sp // 64) == {0, 1} and sp.max() < 128
    # the same spheres without ground quads: the same triangles, ids shifted by the 6
    # ground ids only
    _, bare = render_scene(cam, boxes, sph=sph)
    _, bare_plain = render_scene(cam, boxes)
    a, b = tris[len(plain):], bare[len(bare_plain):]
    assert len(a) == len(b) > 30
    assert np.array_equal(a["X"], b["X"]) and np.array_equal(a["Y"], b["Y"])
    assert np.array_equal(a["prim"].astype(np.int64) - base, b["prim"].astype(np.int64) - 24)


def clear_map(hit, clear):
    m = np.zeros(hit.shape, bool)
    m[hit] = clear
    return m


def _face_normal(q):
    """Closed form: a band quad is a planar isosceles trapezoid whose normal lies in the
    meridian plane of its middle longitude, perpendicular to the line joining the midpoints
    of its two horizontal edges."""
    i, j = divmod(q, 8)
    th0, th1 = -math.pi / 2 + i * math.pi / 4, -math.pi / 2 + (i + 1) * math.pi / 4
    ph = (j + 0.5) * math.pi / 4
    drho = math.cos(math.pi / 8) * (math.cos(th1) - math.cos(th0))
    dz = math.sin(th1) - math.sin(th0)
    n = np.array([dz * math.cos(ph), dz * math.sin(ph), -drho])
    return n / np.linalg.norm(n)


@pytest.mark.parametrize("state", [0, 1, 2, 3])
def test_signal_shading_uses_state_colour_and_face_normal(state):
    nb, nr, nl = 1, 2, 1
    line_end = 12 * nb + 2 * nr + 2 * nl
    sph = np.array([[0.0, 0.0, 4.0, 0.5], [3.0, 0.0, 4.0, 0.5]])
    states = np.array([3 - state, state], np.uint8)
    prims = line_end + 64 + np.arange(64)  # every triangle of the second sphere
    key = ((np.uint64(1) << np.uint64(40)) | (np.uint64(0xFFFFFFFF) - prims.astype(np.uint64)))
    rgb = oracle.shade_rgb(key[None, :], False, 12 * nb, 12 * nb + 2 * nr,
                           np.array([ego_box()], np.float64), line_end=line_end, sph=sph,
                           sph_state=states)
    l = oracle.unit(oracle.RGB_LIGHT)
    for t in range(64):
        n = _face_normal(t // 2)
        shade = oracle.RGB_AMBIENT + (1 - oracle.RGB_AMBIENT) * max(0.0, float(n @ l))
        want = [round(255 * min(1.0, max(0.0, c * shade))) for c in oracle.SIGNAL_COLOURS[state]]
        assert list(rgb[:, 0, t]) == pytest.approx(want, abs=1), t


def test_signal_class_and_onehot_channel():
    cls = np.array([0, 1, 2, 3, 4], np.uint8)
    oh = oracle.onehot_bf16(cls)
    hot, cold = oracle.f32_to_bf16_bits([1.0])[0], oracle.f32_to_bf16_bits([-1.0])[0]
    assert list(oh[3]) == [cold, cold, cold, hot, hot]
    assert list(oh[0]) == [hot, cold, cold, cold, cold]
    img, _ = render_scene(CamConfig(32, 32), [ego_box()], sph=np.array([[6.0, 0.0, 1.5, 1.0]]))
    assert (img.cls == 4).sum() > 10 and set(np.unique(img.cls)) == {0, 4}


def test_ovec_signals_frame_order_and_state():
    # ego at the origin facing +y: world +y is ego-forward (x), world -x is ego-left (y)
    boxes = np.array([[0.0, 0.0, math.pi / 2, 4.5, 1.9, 1.5]])
    sph = [[-10.0, 0.0, 5.0, 0.4],    # 10 m left, red
           [0.0, 30.0, 4.0, 0.4],     # 30 m ahead, green
           [10.0, 0.0, 6.0, 0.4],     # 10 m right, amber: ties with signal 0, higher index
           [0.0, -50.0, 5.0, 0.4],    # exactly at the radius: included
           [0.0, 50.001, 5.0, 0.4],   # just outside
           [3.0, 4.0, 5.0, 0.4]]      # 5 m: the nearest, off
    st = [0, 2, 1, 0, 0, 3]
    o = oracle.observe_signals(boxes, 1, sph, st)[0]
    assert o.shape == (4, 8)
    # order: 5 m (index 5), 10 m (index 0 before 2), then 30 m; the 50 m one is 5th
    want = [[1, 4 / 50, -3 / 50, 0.5, 0, 0, 0, 1],
            [1, 0.0, 10 / 50, 0.5, 1, 0, 0, 0],
            [1, 0.0, -10 / 50, 0.6, 0, 1, 0, 0],
            [1, 30 / 50, 0.0, 0.4, 0, 0, 1, 0]]
    assert np.allclose(o, want, atol=1e-12)
    # with fewer candidates the 50 m signal appears and the rest stays zero
    o2 = oracle.observe_signals(boxes, 1, [sph[3], sph[4]], [2, 1])[0]
    assert np.allclose(o2[0], [1, -1.0, 0.0, 0.5, 0, 0, 1, 0], atol=1e-12)
    assert not o2[1:].any()


def test_red_light_violation_term():
    """Reward table, traffic-light row: -w6 when the agent's centre enters, during the
    step, the road quad controlled by a red signal (the quad of smallest index under the
    signal's centre); nothing for green/amber/off, for staying inside, for leaving, or for
    a signal over no road."""
    road = [rect_quad(-100.0, 0.0, -3.5, 3.5), rect_quad(0.0, 100.0, -3.5, 3.5)]
    over_b = [[50.0, 0.0, 5.0, 0.4]]
    w = [list(W_INF)]

    def r_of(x0, x1, state, sph=over_b, fl_before=0):
        before = np.array([[x0, -1.75, 0.0, 10.0]])
        after = np.array([[x1, -1.75, 0.0, 10.0]])
        r, _ = oracle.rewards_world(before, [fl_before], after, [fl_before], [[0.0, 0.0]],
                                    [[4.5, 1.9]], np.zeros((1, 2)), w, road, sph=sph,
                                    sph_state=state)
        return float(r[0])
    base = r_of(-0.5, 0.5, [2])
    assert r_of(-0.5, 0.5, [0]) == pytest.approx(base - W_INF[6], abs=1e-15)
    for st in ([1], [2], [3]):
        assert r_of(-0.5, 0.5, st) == base
    assert r_of(0.5, 1.5, [0]) == r_of(0.5, 1.5, [2])      # already inside
    assert r_of(0.5, -0.5, [0]) == r_of(0.5, -0.5, [2])    # leaving
    assert r_of(-0.5, 0.0, [0]) == pytest.approx(r_of(-0.5, 0.0, [2]) - W_INF[6])  # edge is inside
    assert r_of(-0.5, 0.5, [0], sph=[[50.0, 40.0, 5.0, 0.4]]) == base  # over no road
    two = over_b + [[60.0, 1.0, 5.0, 0.4]]
    assert r_of(-0.5, 0.5, [0, 0], sph=two) == pytest.approx(base - W_INF[6])  # counted once
    # the signal controls the quad of smallest index under it: over quad A it fires on entering A
    assert r_of(0.5, -0.5, [0], sph=[[-50.0, 0.0, 5.0, 0.4]]) == pytest.approx(
        r_of(0.5, -0.5, [2], sph=[[-50.0, 0.0, 5.0, 0.4]]) - W_INF[6])
    assert r_of(-0.5, 0.5, [0], fl_before=4 | 1) == 0.0  # halted agents earn nothing


def test_red_light_violator_is_halted():
    """App. A "Other Details": a red-light violation halts the agent in place like a
    collision or an off-road departure.  An agent whose centre enters, during the step, the
    road quad under a red signal gets the red-light flag (16) and the halt flag (4), speed
    0, and keeps its post-move pose; later steps leave it there whatever the action.  Green,
    amber and off signals, staying inside, leaving, and a signal over no road halt
    nothing; both dynamics halt."""
    road = np.array([rect_quad(-100.0, 0.0, -3.5, 3.5), rect_quad(0.0, 100.0, -3.5, 3.5)],
                    np.float32)
    over_b = [[50.0, 0.0, 5.0, 0.4]]

    def run(x0, yaw, state, sph=over_b, jerk=None, flags0=0, steps=1, accel=0.0):
        boxes = np.array([[x0, -1.75, yaw, 4.5, 1.9, 1.5]], np.float64)
        st = np.array([[x0, -1.75, yaw, 15.0]], np.float64)
        fl = np.array([flags0], np.uint8)
        for _ in range(steps):
            boxes[0, 0:3] = st[0, 0:3]
            oracle.step_world(boxes, st, fl, np.array([[accel, 0.0]], np.float32), road,
                              jerk=jerk, sph=sph, sph_state=state)
        return st[0].copy(), int(fl[0])

    s1, f1 = run(-1.0, 0.0, [0])
    assert f1 == 16 | 4 and s1[3] == 0.0
    assert s1[0] == pytest.approx(0.5, abs=1e-12) and s1[1] == -1.75   # moved, then halted
    s3, f3 = run(-1.0, 0.0, [0], steps=3, accel=2.0)                      # stays put
    assert f3 == 16 | 4 and np.array_equal(s3, s1)
    for st in ([1], [2], [3]):
        s, f = run(-1.0, 0.0, st)
        assert f == 0 and s[3] == 15.0 and s[0] == pytest.approx(0.5, abs=1e-12)
    assert run(0.5, 0.0, [0])[1] == 0                                     # already inside
    s, f = run(1.0, math.pi, [0])                                         # leaving B for A
    assert f == 0 and s[0] == pytest.approx(-0.5, abs=1e-12)
    assert run(-1.5, 0.0, [0])[1] == 16 | 4                              # lands on the edge
    assert run(-1.0, 0.0, [0], sph=[[50.0, 40.0, 5.0, 0.4]])[1] == 0     # over no road
    assert run(-1.0, 0.0, [0], flags0=4)[1] == 4                          # halted: no move
    # the signal controls the quad of smallest index under it: over A, entering A halts
    assert run(1.0, math.pi, [0], sph=[[-50.0, 0.0, 5.0, 0.4]])[1] == 16 | 4
    s, f = run(-1.0, 0.0, [0], jerk=np.zeros((1, 3)))
    assert f == 16 | 4 and s[3] == 0.0


def test_batch_driver_halts_red_light_violators_per_world():
    """The batch driver hands each world its own signals to the step: two identical worlds
    whose one agent crosses into the quad under a signal, red in world 1 and green in world
    0; only world 1's agent is halted with the red-light flag."""
    import worldgen as wg
    road = np.array([rect_quad(-100.0, 0.0, -3.5, 3.5), rect_quad(0.0, 100.0, -3.5, 3.5)] * 2,
                    np.float32)
    box = [-1.0, -1.75, 0.0, 4.5, 1.9, 1.5, 15.0]
    worlds = wg.Worlds(np.array([0, 1, 2], np.int32), np.array([1, 1], np.int32),
                       np.array([box, box], np.float32), np.array([0, 2, 4], np.int32), road,
                       np.array([0, 0, 0], np.int32), np.zeros((0, 8), np.float32),
                       np.array([0, 1, 2], np.int32),
                       np.array([[50.0, 0.0, 5.0, 0.4]] * 2, np.float32),
                       np.array([2, 0], np.uint8))
    sim = oracle.Sim(worlds)
    sim.step(np.zeros((2, 2), np.float32))
    assert list(sim.flags) == [0, 16 | 4]
    assert sim.state[0, 3] == 15.0 and sim.state[1, 3] == 0.0
    assert sim.state[0, 0] == pytest.approx(0.5, abs=1e-6) and sim.state[1, 0] == sim.state[0, 0]


def test_episode_end_returns_worlds_to_their_start():
    """A world's agents are back at the descriptor's poses and speeds, with only the done
    flag, exactly every episode_steps steps; other steps keep moving."""
    import worldgen as wg
    wl = wg.WORKLOADS["tiny"]
    worlds = wg.make_workload(wl)
    sim = oracle.Sim(worlds, episode_steps=3)
    b0 = worlds.boxes[:worlds.n_agents]
    start = np.column_stack([b0[:, 0:3], b0[:, 6]]).astype(np.float64)
    assert np.array_equal(sim.state, start)
    for k in range(7):
        sim.step(wg.actions(wl.seed, k, worlds.n_agents))
        if (k + 1) % 3 == 0:
            assert np.array_equal(sim.state, start) and np.all(sim.flags == 8)
        else:
            assert not np.array_equal(sim.state, start) and not np.any(sim.flags & 8)


def test_splitmix64_known_outputs():
    # the first outputs of the SplitMix64 stream seeded with 0, as published with the
    # generator; the n-th output depends only on (seed, n)
    assert [oracle.splitmix64(0, n) for n in (1, 2, 3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert oracle.splitmix64(12345, 7) == oracle.splitmix64(12345, 7)
    assert oracle.splitmix64(12345, 7) != oracle.splitmix64(12346, 7)


REWARD_TERMS = ("collision", "offroad", "comfort", "alignment", "centering", "velocity",
                "traffic_light", "time", "reverse", "overspeed", "goal_radius",
                "goal_speed_tolerance")


def reward_table():
    """(lo, hi, inference) arrays of the twelve coefficients, from the golden table."""
    g = read_golden("reward_table.txt")
    assert list(g) == list(REWARD_TERMS)
    t = np.array([g[k] for k in REWARD_TERMS], np.float64)
    return t[:, 0], t[:, 1], t[:, 2]


def test_reward_table_golden():
    """The oracle's default weights are the table's inference column, and its conditioning
    draws fill each coefficient's training range (uniform on [lo, hi))."""
    lo, hi, inf = reward_table()
    assert np.array_equal(np.array(oracle.REWARD_WEIGHTS, np.float64), inf[:10])
    draws = np.array([oracle.conditioning(3, w, 0, i)[1] for w in range(4) for i in range(250)])
    vals = lo + (hi - lo) * (draws + 1) / 2
    assert np.all(vals >= lo) and np.all(vals < hi)
    span = hi - lo
    assert np.all(vals.min(axis=0) - lo < 0.01 * span) and np.all(hi - vals.max(axis=0) < 0.01 * span)


def test_reward_conditioning_ranges_and_normalisation():
    lo, hi, _ = reward_table()
    cs = []
    for w in range(3):
        for e in range(3):
            for i in range(40):
                wt, c = oracle.conditioning(99, w, e, i)
                assert np.all(c >= -1.0) and np.all(c < 1.0)
                assert np.allclose(wt, lo[:10] + (hi[:10] - lo[:10]) * (c[:10] + 1) / 2, rtol=1e-12)
                assert np.all((c + 1) * 2 ** 23 == np.round((c + 1) * 2 ** 23))  # 24-bit uniforms
                cs.append(c)
    cs = np.array(cs)
    assert abs(cs.mean()) < 0.02 and abs(cs.var() - 1 / 3) < 0.02  # U(-1, 1)
    assert len({tuple(c) for c in cs}) == len(cs)  # every (world, episode, agent) differs
    # the oracle's episode restarts redraw: episode 0 at start, 1 after the first restart
    import worldgen as wg
    wl = wg.WORKLOADS["tiny"]
    worlds = wg.make_workload(wl)
    sim = oracle.Sim(worlds, episode_steps=2, conditioning_seed=5)
    assert np.allclose(sim.cond[3], oracle.conditioning(5, 0, 0, 3)[1])
    for k in range(2):
        sim.step(wg.actions(wl.seed, k, worlds.n_agents))
    assert np.allclose(sim.cond[3], oracle.conditioning(5, 0, 1, 3)[1])
    assert np.allclose(sim.weights[3], oracle.conditioning(5, 0, 1, 3)[0])


def test_reset_worlds_by_mask_and_per_world_draws():
    """A masked reset returns only the chosen worlds to their own start (state, cleared
    flags, actuators, episode clock) and redraws their conditioning for the next episode;
    each world's draws are keyed by its own index and its agents' local indices."""
    import worldgen as wg
    wl = wg.WORKLOADS["uniform"]
    worlds = wg.make_workload(wl, n_worlds=3)
    off = worlds.agent_offsets()
    sim = oracle.Sim(worlds, jerk_dynamics=True, episode_steps=50, conditioning_seed=21)
    start = sim.state.copy()
    for w in range(3):
        for i in range(int(off[w + 1] - off[w])):
            wt, c = oracle.conditioning(21, w, 0, i)
            assert np.array_equal(sim.cond[off[w] + i], c)
            assert np.array_equal(sim.weights[off[w] + i], wt)
    for k in range(4):
        sim.step(wg.jerk_actions(wl.seed, k, worlds.n_agents))
    a0, a1 = int(off[1]), int(off[2])
    assert np.any(sim.jerk[a0:a1]) and not np.array_equal(sim.state[a0:a1], start[a0:a1])
    before = sim.state.copy(), sim.flags.copy(), sim.jerk.copy(), sim.cond.copy()
    sim.reset_worlds([0, 1, 0])
    assert np.array_equal(sim.state[a0:a1], start[a0:a1])
    assert not np.any(sim.flags[a0:a1]) and not np.any(sim.jerk[a0:a1])
    assert list(sim.ep) == [4, 0, 4] and list(sim.episode_index) == [0, 1, 0]
    for i in range(a1 - a0):
        assert np.array_equal(sim.cond[a0 + i], oracle.conditioning(21, 1, 1, i)[1])
    keep = np.r_[0:a0, a1:worlds.n_agents]
    for now, then in zip((sim.state, sim.flags, sim.jerk, sim.cond), before):
        assert np.array_equal(now[keep], then[keep])
    # the reset world runs its next episode from the start: one step from a fresh
    # simulator with the same draw gives the same state
    fresh = oracle.Sim(worlds, jerk_dynamics=True)
    act = wg.jerk_actions(wl.seed, 9, worlds.n_agents)
    sim.step(act)
    fresh.step(act)
    assert np.array_equal(sim.state[a0:a1], fresh.state[a0:a1])


def test_batch_driver_keeps_worlds_apart():
    """The batch driver gives each world its own agents' actions, draws agents at their
    current poses and reads each world's own signals: world 1 with zero actions goes
    straight at constant speed (the bicycle's closed form) while world 0 steers; an agent
    moved in front of another's camera is the box under the image centre; every signal of
    a world hangs over one of that world's road quads."""
    import worldgen as wg
    wl = wg.WORKLOADS["paper_rig_210x126"]
    worlds = wg.make_workload(wl, n_worlds=3)
    off = worlds.agent_offsets()
    sim = oracle.Sim(worlds)
    a0, a1 = int(off[1]), int(off[2])
    act = wg.actions(wl.seed, 0, worlds.n_agents).copy()
    act[a0:a1] = 0.0
    before = sim.state.copy()
    sim.step(act)
    b, s, ok = before[a0:a1], sim.state[a0:a1], sim.flags[a0:a1] == 0
    assert ok.sum() >= 10
    assert np.allclose(s[ok, 0], b[ok, 0] + 0.1 * b[ok, 3] * np.cos(b[ok, 2]), rtol=0, atol=1e-12)
    assert np.allclose(s[ok, 1], b[ok, 1] + 0.1 * b[ok, 3] * np.sin(b[ok, 2]), rtol=0, atol=1e-12)
    assert np.array_equal(s[ok, 2:4], b[ok, 2:4])
    # agent 1 of world 0 parked 6 m in front of agent 0, same heading
    st = sim.state.copy()
    x, y, yaw = st[0, 0:3]
    st[1, 0:3] = (x + 6.0 * np.cos(yaw), y + 6.0 * np.sin(yaw), yaw)
    sim.set_state(st, np.zeros_like(sim.flags))
    cam = oracle.CamConfig(wl.width, wl.height, math.radians(wl.hfov_deg), wl.cam_height)
    img = sim.render(cam, 0, 0, 0.0)
    f = 0.5 * wl.width / math.tan(0.5 * cam.hfov)
    row = int(0.5 * wl.height + f * 0.5 / 6.0)  # 1.0 m above the ground, 6 m ahead
    col = wl.width // 2
    prim = 0xFFFFFFFF - (int(img.key[row, col]) & 0xFFFFFFFF)
    assert img.cls[row, col] == 3 and 12 <= prim < 24  # one of agent 1's 12 triangles
    for w in range(3):
        sph, _ = sim.signals(w)
        road = sim.road(w)
        assert len(sph) == 8
        for c in sph:
            assert any(oracle.point_in_quad(c[0], c[1], q) for q in road)


def test_unclipped_vertices_are_snapped_pinhole_projections():
    """With nothing clipped, every triangle vertex is a box corner's pinhole projection
    (x right, y up, z forward; x_px = W/2 + f x / z, y_px = H/2 - f y / z, f = (W/2) /
    tan(hfov/2)) rounded half-to-even to 1/16 px."""
    cam = CamConfig(128, 96)
    f = 0.5 * cam.width / math.tan(0.5 * cam.hfov)
    for box in ([20.0, 1.3, 0.4, 4.5, 1.9, 1.6], [13.0, -2.2, -1.1, 4.2, 1.8, 1.5]):
        _, tris = render_scene(cam, [box], ego=-1)
        assert len(tris) >= 4
        bx, by, yaw, L, W, H = box
        snapped, frac = set(), []
        for sl in (-0.5, 0.5):
            for sw in (-0.5, 0.5):
                cx = bx + sl * L * math.cos(yaw) - sw * W * math.sin(yaw)
                cy = by + sl * L * math.sin(yaw) + sw * W * math.cos(yaw)
                for cz in (0.0, H):
                    xr, yu, zf = -cy, cz - cam.cam_height, cx  # camera at the origin, yaw 0
                    xs = 0.5 * cam.width + f * xr / zf
                    ys = 0.5 * cam.height - f * yu / zf
                    snapped.add((int(np.rint(16 * xs)), int(np.rint(16 * ys))))
                    frac += [(16 * xs) % 1.0, (16 * ys) % 1.0]
        assert any(0.5 < q < 1.0 for q in frac)  # some corner rounds up
        for t in tris:
            for i in range(3):
                assert (int(t["X"][i]), int(t["Y"][i])) in snapped


def test_guard_band_clips_near_tall_and_wide_boxes():
    """A box too tall and too wide for the guard band, 2 m ahead: clipping against all four
    guard planes keeps every snapped coordinate within 4x the viewport half-extent."""
    cam = CamConfig(64, 64)
    _, tris = render_scene(cam, [[2.5, 0.0, 0.0, 1.0, 30.0, 12.0]], ego=-1)
    assert len(tris) > 0
    X, Y = tris["X"].astype(np.int64), tris["Y"].astype(np.int64)
    assert np.all(np.abs(X - 8 * 64) <= 4 * 8 * 64 + 1)
    assert np.all(np.abs(Y - 8 * 64) <= 4 * 8 * 64 + 1)
    # each of the four guard lines is reached
    lim = 4 * 8 * 64
    assert (X - 8 * 64).min() <= -lim + 1 and (X - 8 * 64).max() >= lim - 1
    assert (Y - 8 * 64).min() <= -lim + 1


def test_lane_frame_takes_the_smallest_index_quad():
    """Where road quads overlap (a junction), the lane frame comes from the containing quad
    of smallest index; a point in only the later quad takes that quad's frame."""
    east = rect_quad(-20.0, 20.0, -3.5, 3.5)                       # runs along +x
    north = [3.5, -20.0, 3.5, 20.0, -3.5, 20.0, -3.5, -20.0]       # runs along +y
    # (-1, -1) lies in both: the right half of the east-running quad, the left half (against
    # the quad's direction) of the north-running one
    for first, second, want in ((east, north, 0.0), (north, east, -0.5 * math.pi)):
        road = np.array([first, second], np.float32)
        d, _ = oracle.lane_frame(-1.0, -1.0, road)
        assert math.cos(d - want) == pytest.approx(1.0, abs=1e-9)
    road = np.array([east, north], np.float32)
    d, _ = oracle.lane_frame(1.0, 10.0, road)  # only in the north-running quad
    assert math.cos(d - 0.5 * math.pi) == pytest.approx(1.0, abs=1e-9)


def test_offroad_when_any_single_corner_leaves_the_road():
    """An agent (4 x 2 m at the origin, at rest) is off the road as soon as any one of its
    four footprint corners lies outside every road quad, whichever corner it is."""
    for sx in (-1.0, 1.0):
        for sy in (-1.0, 1.0):
            # two quads covering the footprint except the corner (2 sx, 1 sy)
            road = np.array([rect_quad(-3.0, 3.0, -3.0, 0.5) if sy > 0 else rect_quad(-3.0, 3.0, -0.5, 3.0),
                             rect_quad(-3.0, 0.0, 0.0, 3.0) if sx > 0 else rect_quad(0.0, 3.0, 0.0, 3.0)],
                            np.float32)
            if sy < 0:
                road[1] = rect_quad(-3.0, 0.0, -3.0, 0.0) if sx > 0 else rect_quad(0.0, 3.0, -3.0, 0.0)
            covered = [any(oracle.point_in_quad(2 * ax, ay, q) for q in road)
                       for ax in (-1, 1) for ay in (-1, 1)]
            assert sum(covered) == 3 and not any(
                oracle.point_in_quad(2 * sx, sy, q) for q in road)
            state = np.zeros((1, 4), np.float64)
            flags = np.zeros(1, np.uint8)
            boxes = np.array([[0.0, 0.0, 0.0, 4.0, 2.0, 1.5]], np.float64)
            oracle.step_world(boxes, state, flags, np.zeros((1, 2), np.float32), road)
            assert flags[0] & 2, (sx, sy)
