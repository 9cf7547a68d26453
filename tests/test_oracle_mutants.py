"""Plant one mistake at a time in a copy of the oracle's C source and check that the pins
in test_oracle_pins.py fail for every one of them (so the pins constrain the oracle)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "near plane sign": ("case 0: return v.z - cfg->near;", "case 0: return cfg->near - v.z;"),
    "fill rule mirrored": ("r->tl[k] = (dy == 0 && dx > 0) || (dy < 0);",
                           "r->tl[k] = (dy == 0 && dx < 0) || (dy > 0);"),
    "no top-left rule": ("if (e < 0 || (e == 0 && !r->tl[k])) return 0;", "if (e <= 0) return 0;"),
    "screen y not flipped": ("double ys = 0.5 * cfg->height - cm->f",
                             "double ys = 0.5 * cfg->height + cm->f"),
    "depth plane operand": ("nb = nb - e1 * fx2;", "nb = nb - e1 * fy2;"),
    "slip angle factor": ("double beta = atan(0.5 * tan(steer));", "double beta = atan(tan(steer));"),
    "rear axle distance": ("double lr = 0.3 * L;", "double lr = 0.6 * L;"),
    "heading with new speed": ("*yaw = wrap_pi(*yaw + (v0 / lr)",
                               "*yaw = wrap_pi(*yaw + ((v0 + accel * dt) / lr)"),
    "touching collides": ("if (!(lo < hi)) return 0;", "if (!(lo <= hi)) return 0;"),
    "road edge outside": ("if (cr < 0.0) return 0;", "if (cr <= 0.0) return 0;"),
    "ties to larger id": ("| (uint64_t)(0xFFFFFFFFu - r->prim);", "| (uint64_t)(r->prim);"),
    "zero area kept": ("if (area2 >= 0) continue;", "if (area2 > 0) continue;"),
    "camera right axis": ("v3 v = {dx * cm->s - dy * cm->c, dz,", "v3 v = {dy * cm->c - dx * cm->s, dz,"),
    "half not rounded": ("if (rem > 0x1000u || (rem == 0x1000u && (h & 1u))) ++h;", ""),
    "halt keeps speed": ("            state[4 * i + 3] = 0.0;\n        }\n    }\n}", "        }\n    }\n}"),
    "lane lines on road plane": ("double z = pass ? cfg->line_z : 0.0;", "double z = 0.0;"),
    "ego drawn": ("if (b == ego) continue;", ""),
    "guard band off": ("double g = cfg->guard;", "double g = 1e9;"),
    "near clip t flipped": ("double t = di / (di - dov);", "double t = dov / (dov - di);"),
    "shade ignores box yaw": ("const double c = cos(boxes[6 * b + 2]), sn = sin(boxes[6 * b + 2]);",
                              "const double c = 1.0, sn = 0.0;"),
    "shade no light floor": ("if (ndl < 0.0) ndl = 0.0;", ""),
    "shade +x/-x normals swapped": ("case 0: nx = c; ny = sn;", "case 0: nx = -c; ny = -sn;"),
    "shade +y normal rotated wrong": ("case 2: nx = -sn; ny = c;", "case 2: nx = sn; ny = c;"),
    "shade ground faces down": ("double nx = 0.0, ny = 0.0, nz = 1.0;", "double nx = 0.0, ny = 0.0, nz = -1.0;"),
    "shade background lit": ("double shade = 1.0;", "double shade = 0.5;"),
    "left-hand traffic": ("        if (s < 0.0) {\n            *lane_dir = atan2(dy, dx);",
                          "        if (s > 0.0) {\n            *lane_dir = atan2(dy, dx);"),
    "lane centre offset sign": ("*xf = s + 0.5 * lane_w;", "*xf = s - 0.5 * lane_w;"),
    "collision ignores speed": ("r -= w[0] + 0.1 * fabs(v0);", "r -= w[0];"),
    "jerk needs both axes": ("(fabs(j_lon) > 5.0 || fabs(j_lat) > 5.0)", "(fabs(j_lon) > 5.0 && fabs(j_lat) > 5.0)"),
    "centering sign": ("r -= w[4] * dt * ((ct > 0.5", "r += w[4] * dt * ((ct > 0.5"),
    "velocity without threshold": ("if (fabs(vn) > 2.5) r += w[5]", "if (fabs(vn) > 0.0) r += w[5]"),
    "misalignment signed": ("const double th = fabs(wrap_pi(after[4 * i + 2] - lane_dir));",
                            "const double th = wrap_pi(after[4 * i + 2] - lane_dir);"),
    "halted agents rewarded": ("if (!(fl_before[i] & OR_HALTED)) {\n            const double v0",
                               "if (1) {\n            const double v0"),
    "trace entry face mirrored": ("int fa = 2 * k + 1, fb = 2 * k;", "int fa = 2 * k, fb = 2 * k + 1;"),
    "trace lines on road plane": ("const double z = pass ? cfg->line_z : 0.0;", "const double z = 0.0;"),
    "trace near ignored": ("t0 > t1 || t0 < cfg->near ||", "t0 > t1 ||"),
    "trace last road quad wins": ("                            pr = (uint32_t)(12 * n_boxes + (pass ? 2 * n_road + 2 * q : 2 * q));\n                            break;",
                                  "                            pr = (uint32_t)(12 * n_boxes + (pass ? 2 * n_road + 2 * q : 2 * q));"),
    "ovec lateral sign": ("            o[2] = (-dx * sn + dy * c) / r_agents;", "            o[2] = (dx * sn - dy * c) / r_agents;"),
    "ovec radius exclusive of far": ("            if (d <= r_agents) {", "            if (d <= 1.5 * r_agents) {"),
    "ovec speed difference sign": ("(speed[(int32_t)scratch[2 * k + 1]] - speed[i]) / 30.0;", "(speed[i] - speed[(int32_t)scratch[2 * k + 1]]) / 30.0;"),
    "ovec segment from quad edge": ("const double ax = 0.5 * ((double)q[0] + q[6]), ay = 0.5 * ((double)q[1] + q[7]);", "const double ax = q[0], ay = q[1];"),
    "ovec self included": ("            if (j == i) continue;\n            const double d = hypot", "            const double d = hypot"),
    "ego speed unnormalised": ("const double e[5] = {after[4 * i + 3] / vmax,", "const double e[5] = {after[4 * i + 3],"),
    "jerk accel cap": ("    if (a_lon > 3.0) a_lon = 3.0;\n", ""),
    "jerk braking cap": ("    if (a_lon < -5.0) a_lon = -5.0;\n", ""),
    "jerk steer rate unbounded": ("    if (target > st[2] + step) target = st[2] + step;\n", ""),
    "jerk steer angle unbounded": ("    if (target > 0.5) target = 0.5;\n", ""),
    "jerk curvature on wheelbase/2": ("double target = atan((a_lat / v2) * 0.6 * L);",
                                      "double target = atan((a_lat / v2) * 0.3 * L);"),
    "jerk lateral unclipped": ("    if (a_lat > 4.0) a_lat = 4.0;\n", ""),
    "jerk halted state kept": ("            if (jerk_state) jerk_state[3 * i] = jerk_state[3 * i + 1] = jerk_state[3 * i + 2] = 0.0;\n", ""),
    "sphere latitude step": ("const double th = -0.5 * M_PI + 0.25 * M_PI * i,", "const double th = -0.5 * M_PI + 0.24 * M_PI * i,"),
    "sphere x and y swapped": ("const v3 v = {sp[0] + sp[3] * ct * cos(ph), sp[1] + sp[3] * ct * sin(ph),", "const v3 v = {sp[0] + sp[3] * ct * sin(ph), sp[1] + sp[3] * ct * cos(ph),"),
    "sphere radius ignored in z": ("sp[2] + sp[3] * sin(th)};", "sp[2] + sin(th)};"),
    "sphere face from wrong corners": ("const v3 a = c[0], b = q < 8 ? c[2] : c[1], d = q < 8 ? c[3] : c[2];", "const v3 a = c[0], b = c[1], d = c[2];"),
    "trace sphere exit face": ("                    if (den < 0.0) {\n                        if (t > t0) {", "                    if (den > 0.0) {\n                        if (t > t0) {"),
    "trace sphere id band": ("64 * s + 2 * face +\n                                (face < 8 ? 1 : 0));", "64 * s + 2 * face);"),
    "signal drawn as box": ("return prim < box_end ? 3 : (prim < road_end ? 1 : (prim < line_end ? 2 : 4));", "return prim < box_end ? 3 : (prim < road_end ? 1 : (prim < line_end ? 2 : 3));"),
    "signal colour ignores state": ("                base = sig_colour + 3 * sph_state[s];", "                base = sig_colour;"),
    "signal one-hot channel": ("val[c][cls[p] == c || (c == 3 && cls[p] == 4)]", "val[c][cls[p] == c]"),
    "sphere ids overlap lines": ("const uint32_t sbase = (uint32_t)(12 * n_boxes + 2 * n_road + 2 * n_line);", "const uint32_t sbase = (uint32_t)(12 * n_boxes + 2 * n_road);"),
    "ovec signal lateral sign": ("            o[2] = (-dx * sn + dy * c) / r_sig;", "            o[2] = (dx * sn - dy * c) / r_sig;"),
    "ovec signal state slot": ("            o[4 + (state[s] & 3)] = 1.0;", "            o[4 + ((state[s] + 1) & 3)] = 1.0;"),
    "ovec signal radius": ("            if (d <= r_sig) {", "            if (d < r_sig) {"),
    "red light fires on leaving": ("                if (!or_point_in_quad(before[4 * i], before[4 * i + 1], road + 8 * q) &&\n                    or_point_in_quad(after[4 * i], after[4 * i + 1], road + 8 * q)) {", "                if (or_point_in_quad(before[4 * i], before[4 * i + 1], road + 8 * q) &&\n                    !or_point_in_quad(after[4 * i], after[4 * i + 1], road + 8 * q)) {"),
    "red light any state": ("                if (sig_state[s] != 0) continue;", "                if (sig_state[s] > 1) continue;"),
    "red light counted per signal": ("                    r -= w[6];\n                    break;", "                    r -= w[6];"),
    "splitmix mix constant": ("    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;", "    z = (z ^ (z >> 27)) * 0x94D049BB133111EDull;"),
    "conditioning range swapped": ("static const double COND_HI[12] = {3.0, 3.0, 0.05,", "static const double COND_HI[12] = {3.0, 3.0, 0.5,"),
    "ovec road radius doubled": ("            if (d <= r_roads) {", "            if (d <= 2.0 * r_roads) {"),
    "ovec road heading unrotated": ("            o[4] = cos(phi - bi[2]);", "            o[4] = cos(phi);"),
    "ovec road type swapped": ("            o[6] = s < n_road ? 1.0 : 0.0;", "            o[6] = s < n_road ? 0.0 : 1.0;"),
    "ovec road length unscaled": ("            o[3] = len / r_roads;", "            o[3] = len;"),
    "bf16 truncates": ("    x += 0x7FFFu + ((x >> 16) & 1u);\n", ""),
    "bf16 ties away from even": ("    x += 0x7FFFu + ((x >> 16) & 1u);", "    x += 0x8000u;"),
    "f16 subnormal truncated": ("    if (rem > half || (rem == half && (h & 1u))) ++h;\n    return (uint16_t)(sign | h);\n}",
                                "    return (uint16_t)(sign | h);\n}"),
    "f16 overflow threshold": ("if (ax >= 0x477FF000u) return", "if (ax >= 0x477FE000u) return"),
    "onehot mean subtracted twice": ("float t = ((float)hot - mean[c]) / std_[c];",
                                     "float t = ((float)hot - 2.0f * mean[c]) / std_[c];"),
    "snap to whole pixels": ("        X[i] = (int32_t)rint(16.0 * xs);", "        X[i] = 16 * (int32_t)rint(xs);"),
    "snap truncates": ("        Y[i] = (int32_t)rint(16.0 * ys);", "        Y[i] = (int32_t)(16.0 * ys);"),
    "depth is view z": ("        d[i] = (float)(cfg->near / poly[i].z);", "        d[i] = (float)(poly[i].z);"),
    "fan from the wrong corner": ("        int i0 = 0, i1 = k, i2 = k + 1;", "        int i0 = k, i1 = 0, i2 = k + 1;"),
    "one clip plane skipped": ("    for (int k = 0; k < 5 && m >= 3; ++k) {", "    for (int k = 0; k < 4 && m >= 3; ++k) {"),
    "second agent of a pair not flagged": ("                if (j < n_agents) flags[j] |= OR_COLLIDED;\n", ""),
    "off-road needs every corner out": ("            if (!inside) {\n                flags[i] |= OR_OFFROAD;\n                break;",
                                        "            if (!inside && k == 3) {\n                flags[i] |= OR_OFFROAD;\n                break;"),
    "halt keeps off-road agents moving": ("        if (flags[i] & (OR_COLLIDED | OR_OFFROAD | OR_RED_LIGHT)) {", "        if (flags[i] & (OR_COLLIDED | OR_RED_LIGHT)) {"),
    "red light does not halt": ("        if (flags[i] & (OR_COLLIDED | OR_OFFROAD | OR_RED_LIGHT)) {", "        if (flags[i] & (OR_COLLIDED | OR_OFFROAD)) {"),
    "red-light halt on leaving": ("            if (!or_point_in_quad(before[2 * i], before[2 * i + 1], road + 8 * q) &&\n                or_point_in_quad(state[4 * i], state[4 * i + 1], road + 8 * q)) {", "            if (or_point_in_quad(before[2 * i], before[2 * i + 1], road + 8 * q) &&\n                !or_point_in_quad(state[4 * i], state[4 * i + 1], road + 8 * q)) {"),
    "red-light halt for any state": ("            if (sig_state[s] != 0) continue;\n            int32_t q = 0;\n            while (q < n_road && !or_point_in_quad(sph[4 * s], sph[4 * s + 1], road + 8 * q)) ++q;\n            if (q == n_road) continue;\n            if (!or_point_in_quad(before", "            int32_t q = 0;\n            while (q < n_road && !or_point_in_quad(sph[4 * s], sph[4 * s + 1], road + 8 * q)) ++q;\n            if (q == n_road) continue;\n            if (!or_point_in_quad(before"),
    "lane frame from the quad's last match": ("        if (!or_point_in_quad(px, py, q)) continue;", "        if (!or_point_in_quad(px, py, q) || r + 1 < n_road) continue;"),
    "lane direction normalised by x only": ("        dy /= len;\n", ""),
    "jerk ego steer scale": ("ego[9 * i + 6] = jerk ? jerk[3 * i + 2] / 0.5 : 0.0;", "ego[9 * i + 6] = jerk ? jerk[3 * i + 2] : 0.0;"),
}


# Mistakes in the oracle's Python batch driver (episodes, resets, conditioning draws); the
# C library is left intact for these.
PY_MUTANTS = {
    "episode ends a step late": ("if self.ep[w] >= self.episode_steps:",
                                 "if self.ep[w] > self.episode_steps:"),
    "done flag kept into the next step": (
        "fl = np.ascontiguousarray(self.flags[a0:a1] & ~np.uint8(8))",
        "fl = np.ascontiguousarray(self.flags[a0:a1])"),
    "restart keeps actuators": ("            self.jerk[a0:a1] = 0.0\n        self.episode_index[w] += 1",
                                "            pass\n        self.episode_index[w] += 1"),
    "restart keeps the episode index": ("        self.episode_index[w] += 1\n", ""),
    "draw keyed by batch agent index": ("self.cond_seed, w, int(self.episode_index[w]), i)",
                                        "self.cond_seed, w, int(self.episode_index[w]), a0 + i)"),
    "reset ignores the mask": ("if mask is None or mask[w]:", "if True:"),
    "restart from world 0's start": ("self.state[a0:a1] = self.state0[a0:a1]",
                                     "self.state[a0:a1] = self.state0[:a1 - a0]"),
    "restart keeps the episode clock": ("        self.ep[w] = 0\n", ""),
    "agents drawn at their start poses": ("        b[: a1 - a0, 0:3] = self.state[a0:a1, 0:3]\n", ""),
    "every world reads world 0's signals": ("        s0, s1 = int(off[w]), int(off[w + 1])",
                                             "        s0, s1 = int(off[0]), int(off[1])"),
    "every world takes world 0's actions": ("actions[a0:a1], self.road(w)",
                                            "actions[:a1 - a0], self.road(w)"),
    "initial speed from box height": ("self.state[a0:a1, 3] = bx[:, 6]",
                                      "self.state[a0:a1, 3] = bx[:, 5]"),
    "signals ignored by the step": ("jk,\n                       sph=sp, sph_state=ss)", "jk)"),
}
ALL = sorted(MUTANTS) + sorted("py: " + k for k in PY_MUTANTS)
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")


def _run_mutant(name, workdir):
    """Plant one mistake in a copy of the oracle (its C source, or for "py: " names its Python
    driver) and run the pins against it; returns the pins' exit status and the end of their
    output."""
    d = os.path.join(workdir, "m%d" % ALL.index(name))
    os.makedirs(d, exist_ok=True)
    if name.startswith("py: "):
        import oracle
        so = oracle.build()  # the intact C library
        src = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
        a, b = PY_MUTANTS[name[4:]]
        if a not in src:
            return None, "mutation site not found: " + name
        pkg = os.path.join(d, "oracle")
        os.makedirs(pkg, exist_ok=True)
        with open(os.path.join(pkg, "__init__.py"), "w") as fh:
            fh.write(src.replace(a, b, 1))
        # import the mutated package first, so the pins' own import finds it loaded
        cmd = [sys.executable, "-c",
               "import sys; sys.path.insert(0, %r); import oracle; "
               "assert oracle.__file__.startswith(%r); import pytest; "
               "sys.exit(pytest.main(['-q', '-x', '-p', 'no:cacheprovider', %r]))" % (d, d, PINS)]
    else:
        src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
        a, b = MUTANTS[name]
        if a not in src:
            return None, "mutation site not found: " + name
        c, so = os.path.join(d, "mut.c"), os.path.join(d, "mut.so")
        with open(c, "w") as fh:
            fh.write(src.replace(a, b, 1))
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", so,
                               c, "-lm"])
        cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", PINS]
    env = dict(os.environ, ORACLE_SO=so)
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def mutant_results(tmp_path_factory):
    """Every mutant's pin run, several at a time (each is an independent process); under
    pytest-xdist the workers already run in parallel, so each test runs its own."""
    import concurrent.futures
    if os.environ.get("PYTEST_XDIST_WORKER"):
        return None
    work = str(tmp_path_factory.mktemp("mutants"))
    names = ALL
    with concurrent.futures.ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1))) as ex:
        return dict(zip(names, ex.map(lambda n: _run_mutant(n, work), names)))


@pytest.mark.parametrize("name", ALL)
def test_pins_catch_mutant(name, mutant_results, tmp_path):
    rc, out = mutant_results[name] if mutant_results is not None else _run_mutant(name, str(tmp_path))
    assert rc is not None, out
    assert rc != 0, "pins did not catch mutant %r:\n%s" % (name, out)
    assert " failed" in out, "the pins did not run to a failure for %r:\n%s" % (name, out)
