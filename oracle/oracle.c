/*
 * ORACLE -- test infrastructure only.  A plain, slow, CPU-only FP64 statement of what
 * the batched step-and-render computes, used by tests/, the smoke check and the CPU
 * baseline leg of the benchmark.  The product path never calls it; it shares no code,
 * header, table or constant with the CUDA library.
 *
 * What it follows (paper: "Scaling Self-Play for End-to-End Driving", Gigapixel):
 *   Sec. 3.1 and App. A "High-Throughput Batched Rendering": the world is agent/static
 *     cuboids plus flat road planes and thin lane-line strips; each agent gets an
 *     ego-centric perspective image.
 *   App. A "Action Space and Dynamics": kinematic bicycle, wheelbase 60 % of length,
 *     simulation step 0.1 s.
 *   App. A "Reward Functions" and "Other Details": vehicle collisions and leaving the
 *     drivable area are infractions; an infracting agent is halted in place (velocity
 *     zeroed) and keeps being observed/rendered.
 * The paper gives no rasterisation rule; the rule below is this project's reading
 * (listed as such in the design notes): 1/16-pixel round-half-even snapping, pixel-centre
 * sampling, top-left fill rule, back-face culling, near plane + 4x guard band clipping
 * (Sutherland-Hodgman, planes in the order near, left, right, bottom, top), reversed-Z
 * depth d = n / z_view interpolated by a fixed FP32 plane formula, nearest (largest d)
 * wins, ties to the smaller primitive id.
 *
 * Precision: geometry and dynamics in FP64.  The raster stage applies the rule on
 * snapped integer vertices and FP32 per-vertex depths; its depth-plane arithmetic is the
 * fixed IEEE FP32 sequence the rule defines (compile with -ffp-contract=off so no
 * operation is fused that the rule does not fuse).
 *
 * Parity pins: see tests/test_oracle_pins.py (closed forms, symmetry, brute-force ray
 * casting, watertightness, bicycle closed forms, SAT vs polygon clipping, point-in-quad vs
 * winding number, half/bfloat16 rounding vs numpy/torch).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------
 * Dynamics (App. A "Action Space and Dynamics"; "Other Details")
 * ------------------------------------------------------------------------------------ */

enum { OR_COLLIDED = 1, OR_OFFROAD = 2, OR_HALTED = 4, OR_RED_LIGHT = 16 };

static double wrap_pi(double a) {
    /* to (-pi, pi] */
    while (a > M_PI) a -= 2.0 * M_PI;
    while (a <= -M_PI) a += 2.0 * M_PI;
    return a;
}

/*
 * Kinematic bicycle, centre reference point, wheelbase 0.6 L split evenly
 * (l_r = l_f = 0.3 L): slip angle beta = atan(l_r / (l_f + l_r) * tan(steer)); explicit
 * Euler with the speed of the start of the step; then v += a dt clipped to [0, v_max].
 */
void or_bicycle(double *x, double *y, double *yaw, double *v, double L, double accel,
                double steer, double dt, double vmax) {
    double lr = 0.3 * L;
    double beta = atan(0.5 * tan(steer));
    double v0 = *v;
    *x += v0 * cos(*yaw + beta) * dt;
    *y += v0 * sin(*yaw + beta) * dt;
    *yaw = wrap_pi(*yaw + (v0 / lr) * sin(beta) * dt);
    double vn = v0 + accel * dt;
    if (vn < 0.0) vn = 0.0;
    if (vn > vmax) vn = vmax;
    *v = vn;
}

/*
 * Jerk-actuated kinematic bicycle (App. A "Action Space and Dynamics": the selected
 * longitudinal and lateral jerks are integrated into accelerations and then into velocity
 * and steering, accelerations clipped to g-force limits, speed to the speed limit, steering
 * angle and rate bounded; wheelbase 60 % of the length).  The paper defers the limits to
 * Gigaflow; readings: a_lon in [-5, 3] m/s^2, |a_lat| <= 4 m/s^2, |steer| <= 0.5 rad,
 * |d steer / dt| <= 0.5 rad/s; the steering target realises a_lat on the bicycle's curvature,
 * steer* = atan(kappa * 0.6 L) with kappa = a_lat / max(v^2, 1); then the bicycle above with
 * accel = a_lon and the limited steer.  st[3] = a_lon, a_lat, steer (updated).
 */
void or_jerk_bicycle(double *x, double *y, double *yaw, double *v, double L, double j_lon,
                     double j_lat, double *st, double dt, double vmax) {
    double a_lon = st[0] + j_lon * dt, a_lat = st[1] + j_lat * dt;
    if (a_lon < -5.0) a_lon = -5.0;
    if (a_lon > 3.0) a_lon = 3.0;
    if (a_lat < -4.0) a_lat = -4.0;
    if (a_lat > 4.0) a_lat = 4.0;
    const double v2 = (*v) * (*v) > 1.0 ? (*v) * (*v) : 1.0;
    double target = atan((a_lat / v2) * 0.6 * L);
    const double step = 0.5 * dt;
    if (target > st[2] + step) target = st[2] + step;
    if (target < st[2] - step) target = st[2] - step;
    if (target > 0.5) target = 0.5;
    if (target < -0.5) target = -0.5;
    st[0] = a_lon;
    st[1] = a_lat;
    st[2] = target;
    or_bicycle(x, y, yaw, v, L, a_lon, target, dt, vmax);
}

/* Footprint corners of a box (x, y, yaw, L, W), counter-clockwise from above. */
static void footprint(double x, double y, double yaw, double L, double W, double c[4][2]) {
    double cs = cos(yaw), sn = sin(yaw);
    const double sx[4] = {-0.5, 0.5, 0.5, -0.5};
    const double sy[4] = {-0.5, -0.5, 0.5, 0.5};
    for (int k = 0; k < 4; ++k) {
        double lx = sx[k] * L, ly = sy[k] * W;
        c[k][0] = x + cs * lx - sn * ly;
        c[k][1] = y + sn * lx + cs * ly;
    }
}

/*
 * Two footprints collide iff their interiors intersect.  For convex polygons this holds
 * iff no edge normal separates them (separating-axis theorem): on every one of the four
 * axes the projected intervals overlap with positive length.  Touching is not a collision.
 */
int or_obb_overlap(const double a[5], const double b[5]) {
    double ca[4][2], cb[4][2];
    footprint(a[0], a[1], a[2], a[3], a[4], ca);
    footprint(b[0], b[1], b[2], b[3], b[4], cb);
    double axes[4][2] = {{cos(a[2]), sin(a[2])}, {-sin(a[2]), cos(a[2])},
                         {cos(b[2]), sin(b[2])}, {-sin(b[2]), cos(b[2])}};
    for (int k = 0; k < 4; ++k) {
        double amin = INFINITY, amax = -INFINITY, bmin = INFINITY, bmax = -INFINITY;
        for (int i = 0; i < 4; ++i) {
            double pa = ca[i][0] * axes[k][0] + ca[i][1] * axes[k][1];
            double pb = cb[i][0] * axes[k][0] + cb[i][1] * axes[k][1];
            if (pa < amin) amin = pa;
            if (pa > amax) amax = pa;
            if (pb < bmin) bmin = pb;
            if (pb > bmax) bmax = pb;
        }
        double lo = amin > bmin ? amin : bmin;
        double hi = amax < bmax ? amax : bmax;
        if (!(lo < hi)) return 0;
    }
    return 1;
}

/* Point in a convex quad (corners counter-clockwise from above); boundary counts inside. */
int or_point_in_quad(double px, double py, const float *q) {
    for (int k = 0; k < 4; ++k) {
        double ax = q[2 * k], ay = q[2 * k + 1];
        double bx = q[2 * ((k + 1) & 3)], by = q[2 * ((k + 1) & 3) + 1];
        double cr = (bx - ax) * (py - ay) - (by - ay) * (px - ax);
        if (cr < 0.0) return 0;
    }
    return 1;
}

/*
 * One simulation step of one world, in place.
 *   boxes  [n_boxes][6]  x, y, yaw, L, W, H  (rows of agents are overwritten from state)
 *   state  [n_agents][4] x, y, yaw, v        (FP64)
 *   flags  [n_agents]    bit0 collided, bit1 off-road, bit2 halted, bit4 red-light
 *                        violation (all latched)
 *   actions[n_agents][2] accel (m/s^2), steer (rad)
 *   road   [n_road][8]   road-surface quads
 *   sph    [n_sig][4]    traffic-signal spheres x, y, z, r; sig_state [n_sig] (0 = red)
 * Order: move every non-halted agent; then flag collisions among all pairs that contain
 * an agent; then flag agents with a footprint corner outside every road quad; then flag
 * red-light violations (a halted agent does not move, so it cannot enter a quad); then
 * halt every flagged agent (v = 0).  Halted agents stay in
 * place and stay in the scene (App. A "Other Details": a collision, an off-road departure
 * or a red-light violation halts the agent in place, velocity zeroed).
 * Red-light violation (reading): a signal controls the road quad of smallest index that
 * contains its centre (none if no quad does); an agent that moved this step violates when
 * its centre went from outside a red signal's quad to inside it (boundary inside).
 */
static void step_world_impl(int32_t n_boxes, int32_t n_agents, double *boxes, double *state,
                            uint8_t *flags, const float *actions, int32_t n_road,
                            const float *road, int32_t n_sig, const double *sph,
                            const uint8_t *sig_state, double dt, double vmax,
                            double *jerk_state);

void or_step_world(int32_t n_boxes, int32_t n_agents, double *boxes, double *state,
                   uint8_t *flags, const float *actions, int32_t n_road, const float *road,
                   int32_t n_sig, const double *sph, const uint8_t *sig_state, double dt,
                   double vmax) {
    step_world_impl(n_boxes, n_agents, boxes, state, flags, actions, n_road, road, n_sig, sph,
                    sig_state, dt, vmax, 0);
}

/* The same step with the jerk-actuated bicycle: actions are (j_lon, j_lat) in m/s^3 and
 * jerk_state [n_agents][3] (a_lon, a_lat, steer) is updated for moving agents. */
void or_step_world_jerk(int32_t n_boxes, int32_t n_agents, double *boxes, double *state,
                        uint8_t *flags, const float *actions, int32_t n_road, const float *road,
                        int32_t n_sig, const double *sph, const uint8_t *sig_state, double dt,
                        double vmax, double *jerk_state) {
    step_world_impl(n_boxes, n_agents, boxes, state, flags, actions, n_road, road, n_sig, sph,
                    sig_state, dt, vmax, jerk_state);
}

static void step_world_impl(int32_t n_boxes, int32_t n_agents, double *boxes, double *state,
                            uint8_t *flags, const float *actions, int32_t n_road,
                            const float *road, int32_t n_sig, const double *sph,
                            const uint8_t *sig_state, double dt, double vmax,
                            double *jerk_state) {
    double *before = (double *)malloc(sizeof(double) * 2 * (size_t)(n_agents > 0 ? n_agents : 1));
    for (int32_t i = 0; i < n_agents; ++i) {
        double *s = state + 4 * i;
        before[2 * i] = s[0];
        before[2 * i + 1] = s[1];
        if (!(flags[i] & OR_HALTED)) {
            if (jerk_state)
                or_jerk_bicycle(&s[0], &s[1], &s[2], &s[3], boxes[6 * i + 3], actions[2 * i],
                                actions[2 * i + 1], jerk_state + 3 * i, dt, vmax);
            else
                or_bicycle(&s[0], &s[1], &s[2], &s[3], boxes[6 * i + 3], actions[2 * i],
                           actions[2 * i + 1], dt, vmax);
        } else {
            s[3] = 0.0;
            if (jerk_state) jerk_state[3 * i] = jerk_state[3 * i + 1] = jerk_state[3 * i + 2] = 0.0;
        }
        boxes[6 * i + 0] = s[0];
        boxes[6 * i + 1] = s[1];
        boxes[6 * i + 2] = s[2];
    }
    for (int32_t i = 0; i < n_agents; ++i) {
        for (int32_t j = i + 1; j < n_boxes; ++j) {
            double a[5] = {boxes[6 * i], boxes[6 * i + 1], boxes[6 * i + 2], boxes[6 * i + 3],
                           boxes[6 * i + 4]};
            double b[5] = {boxes[6 * j], boxes[6 * j + 1], boxes[6 * j + 2], boxes[6 * j + 3],
                           boxes[6 * j + 4]};
            if (or_obb_overlap(a, b)) {
                flags[i] |= OR_COLLIDED;
                if (j < n_agents) flags[j] |= OR_COLLIDED;
            }
        }
    }
    for (int32_t i = 0; i < n_agents; ++i) {
        double c[4][2];
        footprint(boxes[6 * i], boxes[6 * i + 1], boxes[6 * i + 2], boxes[6 * i + 3],
                  boxes[6 * i + 4], c);
        for (int k = 0; k < 4; ++k) {
            int inside = 0;
            for (int32_t r = 0; r < n_road && !inside; ++r)
                inside = or_point_in_quad(c[k][0], c[k][1], road + 8 * r);
            if (!inside) {
                flags[i] |= OR_OFFROAD;
                break;
            }
        }
    }
    for (int32_t i = 0; i < n_agents; ++i) {
        for (int32_t s = 0; s < n_sig; ++s) {
            if (sig_state[s] != 0) continue;
            int32_t q = 0;
            while (q < n_road && !or_point_in_quad(sph[4 * s], sph[4 * s + 1], road + 8 * q)) ++q;
            if (q == n_road) continue;
            if (!or_point_in_quad(before[2 * i], before[2 * i + 1], road + 8 * q) &&
                or_point_in_quad(state[4 * i], state[4 * i + 1], road + 8 * q)) {
                flags[i] |= OR_RED_LIGHT;
                break;
            }
        }
    }
    free(before);
    for (int32_t i = 0; i < n_agents; ++i) {
        if (flags[i] & (OR_COLLIDED | OR_OFFROAD | OR_RED_LIGHT)) {
            flags[i] |= OR_HALTED;
            state[4 * i + 3] = 0.0;
        }
    }
}

/*
 * Lane frame of a point: the road quad of smallest index that contains it (boundary
 * inside).  Road quads run from their q0-q3 edge to their q1-q2 edge; with right-hand
 * traffic on a two-lane road the half right of the centre line (lateral offset s < 0,
 * measured along the left normal from the quad centre) runs along that direction and the
 * left half against it; x_f is the offset from the lane's centre line (+-lane_w / 2).
 * Returns 0 if no road quad contains the point.
 */
int or_lane_frame(double px, double py, int32_t n_road, const float *road, double lane_w,
                  double *lane_dir, double *xf) {
    for (int32_t r = 0; r < n_road; ++r) {
        const float *q = road + 8 * r;
        if (!or_point_in_quad(px, py, q)) continue;
        const double m0x = 0.5 * ((double)q[0] + q[6]), m0y = 0.5 * ((double)q[1] + q[7]);
        const double m1x = 0.5 * ((double)q[2] + q[4]), m1y = 0.5 * ((double)q[3] + q[5]);
        double dx = m1x - m0x, dy = m1y - m0y;
        const double len = sqrt(dx * dx + dy * dy);
        dx /= len;
        dy /= len;
        const double cx = 0.25 * ((double)q[0] + q[2] + q[4] + q[6]);
        const double cy = 0.25 * ((double)q[1] + q[3] + q[5] + q[7]);
        const double s = (px - cx) * (-dy) + (py - cy) * dx;
        if (s < 0.0) {
            *lane_dir = atan2(dy, dx);
            *xf = s + 0.5 * lane_w;
        } else {
            *lane_dir = atan2(-dy, -dx);
            *xf = s - 0.5 * lane_w;
        }
        return 1;
    }
    return 0;
}

/*
 * Per-step reward and ego state of one world's agents (App. A "Reward Functions and Reward
 * Conditioning", Table "Reward terms"; "Observations": ego state), evaluated for a step of
 * or_step_world.  Readings:
 *   - a_lon = (v' - v) / dt and a_lat = v * dyaw / dt with v the speed at the step start,
 *     v' = clip(v + a dt, 0, v_max) and dyaw = (v / l_r) sin(beta) dt the bicycle's
 *     increments (before any halt); jerks are their differences to the previous step / dt;
 *   - collision and off-road are this step's new flags, the collision scaled by |v|;
 *   - theta_f in [0, pi] is the heading's misalignment with the lane of the post-step
 *     position (or_lane_frame) and x_f the lateral offset from its centre line; the lane
 *     terms are 0 off the road;
 *   - red-light violation: a signal controls the road quad of smallest index that
 *     contains its centre (none if no quad does); an agent violates when its centre moves
 *     during the step from outside a red signal's quad to inside it (boundary inside);
 *   - the goal term is 0: the synthetic worlds have no goals; an agent halted before the
 *     step earns 0 and has zero accelerations;
 *   - ego state: v'' / v_max (v'' the post-step speed), a_lon / 10, a_lat / 10, L / 10,
 *     W / 5 (each clipped to [-1, 1]) and the collision flag (0 or 1); under the jerk
 *     dynamics also the post-step steering angle / 0.5, and the actuator accelerations
 *     a_lon / 5 and a_lat / 4 of or_jerk_bicycle (zero under direct control).
 *   before/after [n][4] x, y, yaw, v; fl_before/fl_after [n]; actions [n][2] accel, steer
 *   (under the jerk dynamics: the resolved a_lon and steer of the step); dims [n][2] L, W;
 *   acc [n][2] previous a_lon, a_lat (overwritten with this step's); weights [n][10]
 *   collision, off-road, comfort, alignment, centering, velocity, traffic light, time,
 *   reverse, overspeed; jerk [n][3] post-step a_lon, a_lat, steer or NULL; signals
 *   sph [n_sig][4] x, y, z, r with states sig_state [n_sig] (0 = red)
 *   -> reward [n], ego [n][9]
 */
void or_rewards_world(int32_t n, const double *before, const uint8_t *fl_before,
                      const double *after, const uint8_t *fl_after, const float *actions,
                      const double *dims, double *acc, const double *weights, int32_t n_road,
                      const float *road, double lane_w, double v_lim, double dt, double vmax,
                      const double *jerk, int32_t n_sig, const double *sph,
                      const uint8_t *sig_state, double *reward, double *ego) {
    for (int32_t i = 0; i < n; ++i) {
        const double *w = weights + 10 * i;
        double a_lon = 0.0, a_lat = 0.0, r = 0.0;
        if (!(fl_before[i] & OR_HALTED)) {
            const double v0 = before[4 * i + 3];
            const double lr = 0.3 * dims[2 * i];
            const double beta = atan(0.5 * tan((double)actions[2 * i + 1]));
            double vn = v0 + (double)actions[2 * i] * dt;
            if (vn < 0.0) vn = 0.0;
            if (vn > vmax) vn = vmax;
            const double dyaw = (v0 / lr) * sin(beta) * dt;
            a_lon = (vn - v0) / dt;
            a_lat = v0 * dyaw / dt;
            const double j_lon = (a_lon - acc[2 * i]) / dt, j_lat = (a_lat - acc[2 * i + 1]) / dt;
            if (fl_after[i] & OR_COLLIDED) r -= w[0] + 0.1 * fabs(v0);
            if (fl_after[i] & OR_OFFROAD) r -= w[1];
            r -= w[2] * ((fabs(a_lon) > 3.0) + (fabs(a_lat) > 3.0) +
                         (fabs(j_lon) > 5.0 || fabs(j_lat) > 5.0));
            double lane_dir, xf;
            if (or_lane_frame(after[4 * i], after[4 * i + 1], n_road, road, lane_w, &lane_dir,
                              &xf)) {
                const double th = fabs(wrap_pi(after[4 * i + 2] - lane_dir));
                const double ct = cos(th);
                r += w[3] * dt * (fmin(ct, 0.0) + fmin(vn * ct, 0.0) + 0.0025 * (1.0 - 2.0 * th / M_PI));
                r -= w[4] * dt * ((ct > 0.5 ? fabs(xf) : 0.0) - 0.05 * exp(0.5 - fabs(xf)));
                if (fabs(vn) > 2.5) r += w[5] * dt * fmax(ct, 0.0);
            }
            if (fabs(vn) > 0.0 || a_lon != 0.0 || a_lat != 0.0) r -= w[7] * dt;
            if (vn < 0.0) r -= w[8] * dt;
            if (fabs(vn) > v_lim) r -= w[9];
            for (int32_t s = 0; s < n_sig; ++s) {
                if (sig_state[s] != 0) continue;
                int32_t q = 0;
                while (q < n_road && !or_point_in_quad(sph[4 * s], sph[4 * s + 1], road + 8 * q)) ++q;
                if (q == n_road) continue;
                if (!or_point_in_quad(before[4 * i], before[4 * i + 1], road + 8 * q) &&
                    or_point_in_quad(after[4 * i], after[4 * i + 1], road + 8 * q)) {
                    r -= w[6];
                    break;
                }
            }
        }
        acc[2 * i] = a_lon;
        acc[2 * i + 1] = a_lat;
        reward[i] = r;
        const double e[5] = {after[4 * i + 3] / vmax, a_lon / 10.0, a_lat / 10.0,
                             dims[2 * i] / 10.0, dims[2 * i + 1] / 5.0};
        for (int k = 0; k < 5; ++k) ego[9 * i + k] = fmax(-1.0, fmin(1.0, e[k]));
        ego[9 * i + 5] = (fl_after[i] & OR_COLLIDED) ? 1.0 : 0.0;
        ego[9 * i + 6] = jerk ? jerk[3 * i + 2] / 0.5 : 0.0;
        ego[9 * i + 7] = jerk ? jerk[3 * i] / 5.0 : 0.0;
        ego[9 * i + 8] = jerk ? jerk[3 * i + 1] / 4.0 : 0.0;
    }
}

/*
 * Vectorized observations O_vec (App. A "Observations": surrounding agents and road
 * geometry; no traffic controls in the synthetic worlds).  Readings, per agent i with
 * centre c_i, heading th_i, speed v_i and the ego frame (x forward, y left):
 *   agents: the other boxes j (agents and static boxes, speed 0 for static ones) with
 *     |c_j - c_i| <= r_agents, nearest first (ties to the lower index), at most K; slot =
 *     [1, x / r_agents, y / r_agents, L_j / 10, W_j / 5, cos(th_j - th_i), sin(th_j - th_i),
 *     (v_j - v_i) / 30];
 *   roads: segments = the centre lines of the road quads (type 0) and of the lane-line
 *     strips (type 1), each from the midpoint of its q0-q3 edge to that of its q1-q2 edge;
 *     those with midpoint within r_roads, nearest midpoint first (ties: road quads before
 *     lines, then lower index), at most M; slot = [1, x / r_roads, y / r_roads,
 *     length / r_roads, cos(phi - th_i), sin(phi - th_i), 1[type 0], 1[type 1]] with phi
 *     the segment's direction;
 *   unused slots are all zero.
 *   boxes [n_boxes][6] x, y, yaw, L, W, H; speed [n_boxes] -> agents_out [n_agents][K][8],
 *   roads_out [n_agents][M][8]
 */
static int cmp_key(const void *a, const void *b) {
    const double *x = (const double *)a, *y = (const double *)b;
    if (x[0] < y[0]) return -1;
    if (x[0] > y[0]) return 1;
    return (x[1] < y[1]) ? -1 : (x[1] > y[1]);
}

static void seg_of(const float *q, double *mx, double *my, double *len, double *phi) {
    const double ax = 0.5 * ((double)q[0] + q[6]), ay = 0.5 * ((double)q[1] + q[7]);
    const double bx = 0.5 * ((double)q[2] + q[4]), by = 0.5 * ((double)q[3] + q[5]);
    *mx = 0.5 * (ax + bx);
    *my = 0.5 * (ay + by);
    *len = sqrt((bx - ax) * (bx - ax) + (by - ay) * (by - ay));
    *phi = atan2(by - ay, bx - ax);
}

void or_observe_world(int32_t n_boxes, int32_t n_agents, const double *boxes, const double *speed,
                      int32_t n_road, const float *road, int32_t n_line, const float *line,
                      int32_t K, double r_agents, int32_t M, double r_roads, double *agents_out,
                      double *roads_out, double *scratch /* >= 2 * max(n_boxes, n_road + n_line) */) {
    for (int32_t i = 0; i < n_agents; ++i) {
        const double *bi = boxes + 6 * i;
        const double c = cos(bi[2]), sn = sin(bi[2]);
        double *ao = agents_out + (int64_t)i * K * 8;
        double *ro = roads_out + (int64_t)i * M * 8;
        memset(ao, 0, sizeof(double) * K * 8);
        memset(ro, 0, sizeof(double) * M * 8);
        int32_t n = 0;
        for (int32_t j = 0; j < n_boxes; ++j) {
            if (j == i) continue;
            const double d = hypot(boxes[6 * j] - bi[0], boxes[6 * j + 1] - bi[1]);
            if (d <= r_agents) {
                scratch[2 * n] = d;
                scratch[2 * n + 1] = j;
                ++n;
            }
        }
        qsort(scratch, (size_t)n, 2 * sizeof(double), cmp_key);
        for (int32_t k = 0; k < n && k < K; ++k) {
            const double *bj = boxes + 6 * (int32_t)scratch[2 * k + 1];
            const double dx = bj[0] - bi[0], dy = bj[1] - bi[1];
            double *o = ao + 8 * k;
            o[0] = 1.0;
            o[1] = (dx * c + dy * sn) / r_agents;
            o[2] = (-dx * sn + dy * c) / r_agents;
            o[3] = bj[3] / 10.0;
            o[4] = bj[4] / 5.0;
            o[5] = cos(bj[2] - bi[2]);
            o[6] = sin(bj[2] - bi[2]);
            o[7] = (speed[(int32_t)scratch[2 * k + 1]] - speed[i]) / 30.0;
        }
        n = 0;
        for (int32_t s = 0; s < n_road + n_line; ++s) {
            const float *q = s < n_road ? road + 8 * s : line + 8 * (s - n_road);
            double mx, my, len, phi;
            seg_of(q, &mx, &my, &len, &phi);
            const double d = hypot(mx - bi[0], my - bi[1]);
            if (d <= r_roads) {
                scratch[2 * n] = d;
                scratch[2 * n + 1] = s;
                ++n;
            }
        }
        qsort(scratch, (size_t)n, 2 * sizeof(double), cmp_key);
        for (int32_t k = 0; k < n && k < M; ++k) {
            const int32_t s = (int32_t)scratch[2 * k + 1];
            const float *q = s < n_road ? road + 8 * s : line + 8 * (s - n_road);
            double mx, my, len, phi;
            seg_of(q, &mx, &my, &len, &phi);
            const double dx = mx - bi[0], dy = my - bi[1];
            double *o = ro + 8 * k;
            o[0] = 1.0;
            o[1] = (dx * c + dy * sn) / r_roads;
            o[2] = (-dx * sn + dy * c) / r_roads;
            o[3] = len / r_roads;
            o[4] = cos(phi - bi[2]);
            o[5] = sin(phi - bi[2]);
            o[6] = s < n_road ? 1.0 : 0.0;
            o[7] = s < n_road ? 0.0 : 1.0;
        }
    }
}

/*
 * SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014; the 64-bit variant as published with xoroshiro): the n-th output (n >= 1) of
 * the stream seeded with s is mix(s + n * 0x9E3779B97F4A7C15), mix the variant-13 finaliser.
 */
uint64_t or_splitmix64(uint64_t seed, uint64_t n) {
    uint64_t z = seed + n * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/*
 * Reward conditioning (App. A "Reward Functions and Reward Conditioning", Table "Reward
 * terms", training distribution): at every episode start each agent's twelve coefficients
 * are drawn independently and uniformly from the table's ranges; the policy sees them
 * normalised to [-1, 1].  Readings: coefficient k of agent i (index within its world) of
 * world w in episode e uses u = top 24 bits of SplitMix64 output n = 1 + (w << 40 | e << 20 |
 * i << 4 | k) of the stream seeded with `seed`, scaled by 2^-24; value = lo + (hi - lo) u,
 * normalised 2 u - 1.  Coefficients 0..9 are the reward weights (collision .. overspeed);
 * 10 and 11 (goal radius, goal speed tolerance) are only observed (no goals here).
 *   -> w10 [10], c12 [12]
 */
static const double COND_LO[12] = {0.0, 0.0, 0.0, 2.5e-4, 2.5e-4, 0.0, 0.0, 0.0, 2.5e-4, 0.0, 2.0, 1.0};
static const double COND_HI[12] = {3.0, 3.0, 0.05, 2.5e-2, 7.5e-3, 5e-3, 1.0, 5e-5, 7.5e-3, 1.0, 12.0, 5.0};

void or_conditioning(uint64_t seed, uint32_t world, uint32_t episode, uint32_t agent, double *w10,
                     double *c12) {
    for (int k = 0; k < 12; ++k) {
        const uint64_t c = ((uint64_t)world << 40) | ((uint64_t)(episode & 0xFFFFFu) << 20) |
                           ((uint64_t)(agent & 0xFFFFu) << 4) | (uint64_t)k;
        const double u = (double)(or_splitmix64(seed, c + 1) >> 40) / 16777216.0;
        if (k < 10) w10[k] = COND_LO[k] + (COND_HI[k] - COND_LO[k]) * u;
        c12[k] = 2.0 * u - 1.0;
    }
}

/*
 * Traffic controls of O_vec (App. A "Observations": the vectorized observation also holds
 * traffic-control states).  Reading: per agent i the signal spheres s whose centre is
 * within r_sig of c_i on the ground plane, nearest first (ties to the lower index), at
 * most S; slot = [1, x / r_sig, y / r_sig (ego frame, x forward, y left), z_s / 10,
 * 1[red], 1[amber], 1[green], 1[off]]; unused slots zero.
 *   boxes [n_agents..][6]; sph [n_sph][4] x, y, z, r; state [n_sph] -> out [n_agents][S][8]
 */
void or_observe_signals(int32_t n_agents, const double *boxes, int32_t n_sph, const double *sph,
                        const uint8_t *state, int32_t S, double r_sig, double *out,
                        double *scratch /* >= 2 * n_sph */) {
    for (int32_t i = 0; i < n_agents; ++i) {
        const double *bi = boxes + 6 * i;
        const double c = cos(bi[2]), sn = sin(bi[2]);
        double *so = out + (int64_t)i * S * 8;
        memset(so, 0, sizeof(double) * S * 8);
        int32_t n = 0;
        for (int32_t s = 0; s < n_sph; ++s) {
            const double d = hypot(sph[4 * s] - bi[0], sph[4 * s + 1] - bi[1]);
            if (d <= r_sig) {
                scratch[2 * n] = d;
                scratch[2 * n + 1] = s;
                ++n;
            }
        }
        qsort(scratch, (size_t)n, 2 * sizeof(double), cmp_key);
        for (int32_t k = 0; k < n && k < S; ++k) {
            const int32_t s = (int32_t)scratch[2 * k + 1];
            const double dx = sph[4 * s] - bi[0], dy = sph[4 * s + 1] - bi[1];
            double *o = so + 8 * k;
            o[0] = 1.0;
            o[1] = (dx * c + dy * sn) / r_sig;
            o[2] = (-dx * sn + dy * c) / r_sig;
            o[3] = sph[4 * s + 2] / 10.0;
            o[4 + (state[s] & 3)] = 1.0;
        }
    }
}

/* ------------------------------------------------------------------------------------
 * Geometry: camera, scene triangles, clipping, projection, snapping (FP64)
 * ------------------------------------------------------------------------------------ */

typedef struct {
    int32_t X[3], Y[3]; /* snapped positions, 1/16 pixel units, y down */
    float d[3];         /* per-vertex reversed-Z depth n / z_view, rounded to FP32 */
    uint32_t prim;      /* primitive id (see below) */
    uint32_t sub;       /* index of the triangle in the clipped polygon's fan */
} or_tri;

typedef struct {
    int32_t width, height;
    double hfov;        /* horizontal field of view, rad */
    double cam_height;  /* camera height above ground, m */
    double near;        /* near plane distance, m */
    double line_z;      /* lane-line strip height above the road, m */
    double guard;       /* guard band, in multiples of the viewport half-extent */
} or_cam;

typedef struct { double x, y, z; } v3;

/* Box corner k: x = +-L/2 (bit 0), y = +-W/2 (bit 1), z = 0 or H (bit 2). */
static v3 box_corner(const double *b, int k) {
    double lx = (k & 1) ? 0.5 * b[3] : -0.5 * b[3];
    double ly = (k & 2) ? 0.5 * b[4] : -0.5 * b[4];
    double cs = cos(b[2]), sn = sin(b[2]);
    v3 p = {b[0] + cs * lx - sn * ly, b[1] + sn * lx + cs * ly, (k & 4) ? b[5] : 0.0};
    return p;
}

/* Faces as corner quads, counter-clockwise seen from outside, in the order
 * +x, -x, +y, -y, +z, -z.  Face quad (q0 q1 q2 q3) -> triangles (q0 q1 q2), (q0 q2 q3). */
static const int BOX_FACES[6][4] = {
    {1, 3, 7, 5}, {0, 4, 6, 2}, {2, 6, 7, 3}, {0, 1, 5, 4}, {4, 5, 7, 6}, {0, 2, 3, 1}};

/*
 * Traffic-signal sphere (Sec. 3.1 / App. A: spheres are the world's third primitive, used
 * for traffic lights).  Reading: a sphere of centre c and radius r is drawn as the convex
 * polyhedron with vertices on it at latitudes th_i = -pi/2 + i pi/4 (i = 0..4) and
 * longitudes ph_j = j pi/4 (j = 0..7): V(i, j) = c + r (cos th_i cos ph_j, cos th_i sin ph_j,
 * sin th_i), the poles exactly (0, 0, -+1).  Quad q = 8 i + j (i = 0..3) has the corners
 * V(i, j), V(i, j+1), V(i+1, j+1), V(i+1, j), counter-clockwise seen from outside; its
 * triangles (q0 q1 q2) and (q0 q2 q3) are primitives 2 q and 2 q + 1 of the sphere (64 ids
 * per sphere).  In the two pole bands one triangle of each quad is degenerate.
 *   sp [4] = x, y, z, r
 */
static v3 sphere_vertex(const double *sp, int i, int j) {
    const double th = -0.5 * M_PI + 0.25 * M_PI * i, ph = 0.25 * M_PI * (j % 8);
    const double ct = (i == 0 || i == 4) ? 0.0 : cos(th);
    const v3 v = {sp[0] + sp[3] * ct * cos(ph), sp[1] + sp[3] * ct * sin(ph), sp[2] + sp[3] * sin(th)};
    return v;
}

static void sphere_quad(const double *sp, int q, v3 c[4]) {
    const int i = q / 8, j = q % 8;
    c[0] = sphere_vertex(sp, i, j);
    c[1] = sphere_vertex(sp, i, j + 1);
    c[2] = sphere_vertex(sp, i + 1, j + 1);
    c[3] = sphere_vertex(sp, i + 1, j);
}

/* Outward unit normal of sphere quad q and its plane offset n . V (the plane through the
 * quad's distinct corners). */
static v3 sphere_face(const double *sp, int q, double *off) {
    v3 c[4];
    sphere_quad(sp, q, c);
    /* three distinct corners: the south-pole band repeats corner 0 as corner 1 */
    const v3 a = c[0], b = q < 8 ? c[2] : c[1], d = q < 8 ? c[3] : c[2];
    const double ux = b.x - a.x, uy = b.y - a.y, uz = b.z - a.z;
    const double wx = d.x - a.x, wy = d.y - a.y, wz = d.z - a.z;
    double nx = uy * wz - uz * wy, ny = uz * wx - ux * wz, nz = ux * wy - uy * wx;
    const double len = sqrt(nx * nx + ny * ny + nz * nz);
    nx /= len;
    ny /= len;
    nz /= len;
    *off = nx * a.x + ny * a.y + nz * a.z;
    const v3 n = {nx, ny, nz};
    return n;
}

typedef struct {
    double s, c;   /* sin, cos of camera yaw */
    double px, py, pz;
    double f;      /* focal length in pixels */
    double tx, ty; /* viewport half-extent over focal length */
} camera;

static v3 to_view(const camera *cm, v3 p) {
    double dx = p.x - cm->px, dy = p.y - cm->py, dz = p.z - cm->pz;
    v3 v = {dx * cm->s - dy * cm->c, dz, dx * cm->c + dy * cm->s};
    return v;
}

/* Signed distance-like value to clip plane k (inside >= 0). */
static double plane_dist(const or_cam *cfg, const camera *cm, int k, v3 v) {
    double g = cfg->guard;
    switch (k) {
    case 0: return v.z - cfg->near;
    case 1: return v.x + g * cm->tx * v.z;
    case 2: return g * cm->tx * v.z - v.x;
    case 3: return v.y + g * cm->ty * v.z;
    default: return g * cm->ty * v.z - v.y;
    }
}

/* Sutherland-Hodgman against one plane; the crossing point is always interpolated from
 * the inside vertex towards the outside one.  A convex polygon gains at most one vertex
 * per plane (at most 8 after five planes); the 16-entry bound only guards rounding on
 * near-degenerate input. */
static int clip_plane(const or_cam *cfg, const camera *cm, int k, const v3 *in, int n, v3 *out) {
    int m = 0;
    for (int i = 0; i < n; ++i) {
        v3 a = in[i], b = in[(i + 1) % n];
        double da = plane_dist(cfg, cm, k, a), db = plane_dist(cfg, cm, k, b);
        int ia = da >= 0.0, ib = db >= 0.0;
        if (ia && m < 16) out[m++] = a;
        if (ia != ib && m < 16) {
            v3 vi = ia ? a : b, vo = ia ? b : a;
            double di = ia ? da : db, dov = ia ? db : da;
            double t = di / (di - dov);
            v3 p = {vi.x + t * (vo.x - vi.x), vi.y + t * (vo.y - vi.y), vi.z + t * (vo.z - vi.z)};
            out[m++] = p;
        }
    }
    return m;
}

static int64_t emit_triangle(const or_cam *cfg, const camera *cm, v3 a, v3 b, v3 c, uint32_t prim,
                             or_tri *out, int64_t n, int64_t cap) {
    v3 poly[16], tmp[16];
    poly[0] = to_view(cm, a);
    poly[1] = to_view(cm, b);
    poly[2] = to_view(cm, c);
    int m = 3;
    for (int k = 0; k < 5 && m >= 3; ++k) {
        m = clip_plane(cfg, cm, k, poly, m, tmp);
        memcpy(poly, tmp, sizeof(v3) * (size_t)m);
    }
    if (m < 3) return n;
    int32_t X[16], Y[16];
    float d[16];
    for (int i = 0; i < m; ++i) {
        double xs = 0.5 * cfg->width + cm->f * poly[i].x / poly[i].z;
        double ys = 0.5 * cfg->height - cm->f * poly[i].y / poly[i].z;
        X[i] = (int32_t)rint(16.0 * xs); /* default rounding mode: round half to even */
        Y[i] = (int32_t)rint(16.0 * ys);
        d[i] = (float)(cfg->near / poly[i].z);
    }
    for (int k = 1; k + 1 < m; ++k) {
        int i0 = 0, i1 = k, i2 = k + 1;
        int64_t area2 = (int64_t)(X[i1] - X[i0]) * (Y[i2] - Y[i0]) -
                        (int64_t)(X[i2] - X[i0]) * (Y[i1] - Y[i0]);
        if (area2 >= 0) continue; /* back-facing or degenerate in y-down screen space */
        if (n < cap) {
            or_tri *t = out + n;
            t->X[0] = X[i0]; t->X[1] = X[i1]; t->X[2] = X[i2];
            t->Y[0] = Y[i0]; t->Y[1] = Y[i1]; t->Y[2] = Y[i2];
            t->d[0] = d[i0]; t->d[1] = d[i1]; t->d[2] = d[i2];
            t->prim = prim;
            t->sub = (uint32_t)(k - 1);
        }
        ++n;
    }
    return n;
}

/*
 * Scene triangles of one camera, FP64 geometry.
 *   boxes [n_boxes][6] x, y, yaw, L, W, H (current poses); box `ego` is skipped
 *   road/line quads [n][8]; roads at z = 0, lane lines at z = cfg->line_z
 *   agent pose (ax, ay, ayaw), camera yaw offset cam_yaw
 *   signal spheres sph [n_sph][4] x, y, z, r (sphere_vertex)
 * Primitive ids: box b face-triangle t -> 12 b + t; road quad r triangle t ->
 * 12 n_boxes + 2 r + t; lane-line quad l triangle t -> 12 n_boxes + 2 n_road + 2 l + t;
 * sphere s quad q triangle t -> 12 n_boxes + 2 n_road + 2 n_line + 64 s + 2 q + t.
 * Writes at most `cap` triangles; returns the number produced.
 */
int64_t or_camera_tris(const or_cam *cfg, int32_t n_boxes, const double *boxes, int32_t ego,
                       int32_t n_road, const float *road, int32_t n_line, const float *line,
                       int32_t n_sph, const double *sph, double ax, double ay, double ayaw,
                       double cam_yaw, or_tri *out, int64_t cap) {
    camera cm;
    double yaw = ayaw + cam_yaw;
    cm.s = sin(yaw);
    cm.c = cos(yaw);
    cm.px = ax;
    cm.py = ay;
    cm.pz = cfg->cam_height;
    cm.f = 0.5 * cfg->width / tan(0.5 * cfg->hfov);
    cm.tx = 0.5 * cfg->width / cm.f;
    cm.ty = 0.5 * cfg->height / cm.f;
    int64_t n = 0;
    for (int32_t b = 0; b < n_boxes; ++b) {
        if (b == ego) continue;
        const double *bx = boxes + 6 * b;
        v3 cn[8];
        for (int k = 0; k < 8; ++k) cn[k] = box_corner(bx, k);
        for (int f = 0; f < 6; ++f) {
            const int *q = BOX_FACES[f];
            n = emit_triangle(cfg, &cm, cn[q[0]], cn[q[1]], cn[q[2]], (uint32_t)(12 * b + 2 * f),
                              out, n, cap);
            n = emit_triangle(cfg, &cm, cn[q[0]], cn[q[2]], cn[q[3]],
                              (uint32_t)(12 * b + 2 * f + 1), out, n, cap);
        }
    }
    for (int pass = 0; pass < 2; ++pass) {
        int32_t nq = pass ? n_line : n_road;
        const float *qs = pass ? line : road;
        double z = pass ? cfg->line_z : 0.0;
        uint32_t base = (uint32_t)(12 * n_boxes + (pass ? 2 * n_road : 0));
        for (int32_t i = 0; i < nq; ++i) {
            const float *q = qs + 8 * i;
            v3 c[4];
            for (int k = 0; k < 4; ++k) {
                c[k].x = q[2 * k];
                c[k].y = q[2 * k + 1];
                c[k].z = z;
            }
            n = emit_triangle(cfg, &cm, c[0], c[1], c[2], base + 2 * i, out, n, cap);
            n = emit_triangle(cfg, &cm, c[0], c[2], c[3], base + 2 * i + 1, out, n, cap);
        }
    }
    const uint32_t sbase = (uint32_t)(12 * n_boxes + 2 * n_road + 2 * n_line);
    for (int32_t s = 0; s < n_sph; ++s)
        for (int q = 0; q < 32; ++q) {
            v3 c[4];
            sphere_quad(sph + 4 * s, q, c);
            const uint32_t pr = sbase + (uint32_t)(64 * s + 2 * q);
            n = emit_triangle(cfg, &cm, c[0], c[1], c[2], pr, out, n, cap);
            n = emit_triangle(cfg, &cm, c[0], c[2], c[3], pr + 1, out, n, cap);
        }
    return n;
}

/* ------------------------------------------------------------------------------------
 * Ray-traced view (App. A: the renderer's ray-traced backend)
 * ------------------------------------------------------------------------------------ */

/*
 * One ray per pixel centre from the camera: direction right * x + up * y + forward with
 * x = (i + 1/2 - W/2) / f, y = (H/2 - j - 1/2) / f, so the ray parameter t is the view
 * depth z.  Nearest hit with t >= near among every box except the ego's (slab test in the
 * box frame, z from 0 to H), road quads on z = 0 and lane-line strips on z = line_z (plane
 * hit, point in quad with the boundary inside) and signal spheres (the polyhedron of
 * sphere_vertex as the intersection of its 32 face half-spaces: entry at the largest
 * entering-face parameter, the first such face on ties); ties go to the lower object
 * (boxes by index, then road quads, then lines, then spheres).  Per pixel: class
 * (0 background, 1 road, 2 lane line, 3 box, 4 signal), reversed-Z depth near / t rounded to
 * FP32 (0 background), and the hit's primitive id in the raster's numbering -- box b's entry
 * face f gives 12 b + 2 f (faces +x, -x, +y, -y, +z, -z), road quad r gives 12 n_boxes + 2 r,
 * line l gives 12 n_boxes + 2 n_road + 2 l, sphere s's entry quad q the id of its
 * non-degenerate triangle (2 q + 1 in the south-pole band, else 2 q) -- or 0xFFFFFFFF on
 * background, so the RGB shading applies unchanged.
 */
void or_trace_view(const or_cam *cfg, int32_t n_boxes, const double *boxes, int32_t ego,
                   int32_t n_road, const float *road, int32_t n_line, const float *line,
                   int32_t n_sph, const double *sph, double ax, double ay, double ayaw,
                   double cam_yaw, uint8_t *cls, float *depth, uint32_t *prim) {
    const double yaw = ayaw + cam_yaw;
    const double fx = cos(yaw), fy = sin(yaw);  /* forward */
    const double rx = sin(yaw), ry = -cos(yaw); /* right */
    const double f = 0.5 * cfg->width / tan(0.5 * cfg->hfov);
    const double oz = cfg->cam_height;
    for (int32_t j = 0; j < cfg->height; ++j)
        for (int32_t i = 0; i < cfg->width; ++i) {
            const double x = (i + 0.5 - 0.5 * cfg->width) / f;
            const double y = (0.5 * cfg->height - j - 0.5) / f;
            const double dx = rx * x + fx, dy = ry * x + fy, dz = y;
            double best = INFINITY;
            int c = 0;
            uint32_t pr = 0xFFFFFFFFu;
            for (int32_t b = 0; b < n_boxes; ++b) {
                if (b == ego) continue;
                const double *bx = boxes + 6 * b;
                const double cs = cos(bx[2]), sn = sin(bx[2]);
                const double px = ax - bx[0], py = ay - bx[1];
                const double o[3] = {cs * px + sn * py, -sn * px + cs * py, oz};
                const double d[3] = {cs * dx + sn * dy, -sn * dx + cs * dy, dz};
                const double lo[3] = {-0.5 * bx[3], -0.5 * bx[4], 0.0};
                const double hi[3] = {0.5 * bx[3], 0.5 * bx[4], bx[5]};
                double t0 = -INFINITY, t1 = INFINITY;
                int face = -1, inside = 1;
                for (int k = 0; k < 3 && inside; ++k) {
                    if (d[k] == 0.0) {
                        if (o[k] < lo[k] || o[k] > hi[k]) inside = 0;
                        continue;
                    }
                    double ta = (lo[k] - o[k]) / d[k], tb = (hi[k] - o[k]) / d[k];
                    /* entering through the low side (face -k) when moving up the axis */
                    int fa = 2 * k + 1, fb = 2 * k;
                    if (ta > tb) {
                        const double tt = ta;
                        ta = tb;
                        tb = tt;
                        fa = 2 * k;
                        fb = 2 * k + 1;
                    }
                    (void)fb;
                    if (ta > t0) {
                        t0 = ta;
                        face = fa;
                    }
                    if (tb < t1) t1 = tb;
                }
                if (!inside || face < 0 || t0 > t1 || t0 < cfg->near || !(t0 < best)) continue;
                best = t0;
                c = 3;
                pr = (uint32_t)(12 * b + 2 * face);
            }
            if (dz < 0.0) {
                for (int pass = 0; pass < 2; ++pass) {
                    const double z = pass ? cfg->line_z : 0.0;
                    const double t = (z - oz) / dz;
                    if (t < cfg->near || !(t < best)) continue;
                    const double hx = ax + t * dx, hy = ay + t * dy;
                    const int32_t nq = pass ? n_line : n_road;
                    const float *qs = pass ? line : road;
                    for (int32_t q = 0; q < nq; ++q)
                        if (or_point_in_quad(hx, hy, qs + 8 * q)) {
                            best = t;
                            c = pass ? 2 : 1;
                            pr = (uint32_t)(12 * n_boxes + (pass ? 2 * n_road + 2 * q : 2 * q));
                            break;
                        }
                }
            }
            for (int32_t s = 0; s < n_sph; ++s) {
                double t0 = -INFINITY, t1 = INFINITY;
                int face = -1, inside = 1;
                for (int q = 0; q < 32 && inside; ++q) {
                    double off;
                    const v3 n = sphere_face(sph + 4 * s, q, &off);
                    const double den = n.x * dx + n.y * dy + n.z * dz;
                    const double num = off - (n.x * ax + n.y * ay + n.z * oz);
                    if (den == 0.0) {
                        if (num < 0.0) inside = 0;
                        continue;
                    }
                    const double t = num / den;
                    if (den < 0.0) {
                        if (t > t0) {
                            t0 = t;
                            face = q;
                        }
                    } else if (t < t1) {
                        t1 = t;
                    }
                }
                if (!inside || face < 0 || t0 > t1 || t0 < cfg->near || !(t0 < best)) continue;
                best = t0;
                c = 4;
                pr = (uint32_t)(12 * n_boxes + 2 * n_road + 2 * n_line + 64 * s + 2 * face +
                                (face < 8 ? 1 : 0));
            }
            const int64_t pix = (int64_t)j * cfg->width + i;
            cls[pix] = (uint8_t)c;
            depth[pix] = c ? (float)(cfg->near / best) : 0.0f;
            prim[pix] = pr;
        }
}

/* ------------------------------------------------------------------------------------
 * Raster rule on snapped triangles (integer coverage + FP32 depth)
 * ------------------------------------------------------------------------------------ */

/* IEEE binary32 -> binary16, round to nearest even (subnormals, overflow, NaN handled). */
uint16_t or_f32_to_f16(float f) {
    uint32_t x;
    memcpy(&x, &f, 4);
    uint32_t sign = (x >> 16) & 0x8000u;
    uint32_t ax = x & 0x7FFFFFFFu;
    if (ax >= 0x7F800000u) return (uint16_t)(sign | 0x7C00u | (ax > 0x7F800000u ? 0x200u : 0u));
    if (ax >= 0x477FF000u) return (uint16_t)(sign | 0x7C00u); /* >= 65520 rounds to inf */
    int32_t e = (int32_t)(ax >> 23);
    uint32_t mant = ax & 0x7FFFFFu;
    if (e >= 113) { /* normal half: value >= 2^-14 */
        uint32_t h = ((uint32_t)(e - 112) << 10) | (mant >> 13);
        uint32_t rem = mant & 0x1FFFu;
        if (rem > 0x1000u || (rem == 0x1000u && (h & 1u))) ++h;
        return (uint16_t)(sign | h);
    }
    /* subnormal half (or zero): value / 2^-24, rounded */
    if (e == 0) return (uint16_t)sign; /* float subnormals are far below half's range */
    uint32_t m24 = mant | 0x800000u;
    int32_t shift = 126 - e; /* >= 14 */
    if (shift > 24) return (uint16_t)sign;
    uint32_t h = m24 >> shift;
    uint32_t rem = m24 & ((1u << shift) - 1u);
    uint32_t half = 1u << (shift - 1);
    if (rem > half || (rem == half && (h & 1u))) ++h;
    return (uint16_t)(sign | h);
}

/* IEEE binary32 -> bfloat16, round to nearest even. */
uint16_t or_f32_to_bf16(float f) {
    uint32_t x;
    memcpy(&x, &f, 4);
    if ((x & 0x7FFFFFFFu) > 0x7F800000u) return (uint16_t)((x >> 16) | 0x40u);
    x += 0x7FFFu + ((x >> 16) & 1u);
    return (uint16_t)(x >> 16);
}

/* Triangle in raster form: positive-area vertex order, edge top-left flags, depth plane. */
typedef struct {
    int64_t X[3], Y[3];
    int tl[3];
    float d0, a, b;
    uint32_t prim;
} rtri;

static int setup_rtri(const or_tri *t, rtri *r) {
    int64_t area2 = (int64_t)(t->X[1] - t->X[0]) * (t->Y[2] - t->Y[0]) -
                    (int64_t)(t->X[2] - t->X[0]) * (t->Y[1] - t->Y[0]);
    if (area2 == 0) return 0;
    int o[3] = {0, 1, 2};
    if (area2 < 0) { o[1] = 2; o[2] = 1; area2 = -area2; }
    float dv[3];
    for (int k = 0; k < 3; ++k) {
        r->X[k] = t->X[o[k]];
        r->Y[k] = t->Y[o[k]];
        dv[k] = t->d[o[k]];
    }
    for (int k = 0; k < 3; ++k) {
        int64_t dx = r->X[(k + 1) % 3] - r->X[k], dy = r->Y[(k + 1) % 3] - r->Y[k];
        /* with area2 > 0 in y-down space: top edge = horizontal going +x; left = going up */
        r->tl[k] = (dy == 0 && dx > 0) || (dy < 0);
    }
    /* depth plane d(X, Y) = d0 + a (X - X0) + b (Y - Y0), fixed FP32 sequence */
    float fx1 = (float)(r->X[1] - r->X[0]), fy1 = (float)(r->Y[1] - r->Y[0]);
    float fx2 = (float)(r->X[2] - r->X[0]), fy2 = (float)(r->Y[2] - r->Y[0]);
    float e1 = dv[1] - dv[0], e2 = dv[2] - dv[0];
    float fa = (float)area2;
    float na = e1 * fy2;
    na = na - e2 * fy1;
    float nb = e2 * fx1;
    nb = nb - e1 * fx2;
    r->a = na / fa;
    r->b = nb / fa;
    r->d0 = dv[0];
    r->prim = t->prim;
    return 1;
}

static int64_t floor16(int64_t a) { return a >= 0 ? a / 16 : -((-a + 15) / 16); }

/* Coverage of the pixel with centre (Xp, Yp) (1/16 units) by the triangle. */
static int covers(const rtri *r, int64_t Xp, int64_t Yp) {
    for (int k = 0; k < 3; ++k) {
        int64_t xa = r->X[k], ya = r->Y[k], xb = r->X[(k + 1) % 3], yb = r->Y[(k + 1) % 3];
        int64_t e = (xb - xa) * (Yp - ya) - (yb - ya) * (Xp - xa);
        if (e < 0 || (e == 0 && !r->tl[k])) return 0;
    }
    return 1;
}

static uint64_t pixel_key(const rtri *r, int64_t Xp, int64_t Yp, int key_f16) {
    float gx = (float)(Xp - r->X[0]), gy = (float)(Yp - r->Y[0]);
    float dp = fmaf(r->a, gx, fmaf(r->b, gy, r->d0));
    if (!(dp > 0.0f)) dp = 0.0f;
    if (key_f16) {
        uint16_t h = or_f32_to_f16(dp);
        return ((uint64_t)h << 16) | (uint64_t)(0xFFFFu - (r->prim & 0xFFFFu));
    }
    uint32_t bits;
    memcpy(&bits, &dp, 4);
    return ((uint64_t)bits << 32) | (uint64_t)(0xFFFFFFFFu - r->prim);
}

/* Class of a primitive id: 3 vehicle/box, 1 road, 2 lane line, 4 signal sphere. */
static uint8_t prim_class(uint32_t prim, uint32_t box_end, uint32_t road_end,
                          uint32_t line_end) {
    return prim < box_end ? 3 : (prim < road_end ? 1 : (prim < line_end ? 2 : 4));
}

static void resolve(const uint64_t *key, int64_t npx, int key_f16, uint32_t box_end,
                    uint32_t road_end, uint32_t line_end, uint8_t *cls, float *depth,
                    uint16_t *depth16) {
    for (int64_t p = 0; p < npx; ++p) {
        uint64_t k = key[p];
        uint8_t c = 0;
        float dv = 0.0f;
        uint16_t h = 0;
        if (k) {
            uint32_t prim = key_f16 ? (0xFFFFu - (uint32_t)(k & 0xFFFFu))
                                    : (0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFu));
            c = prim_class(prim, box_end, road_end, line_end);
            if (key_f16) h = (uint16_t)(k >> 16);
            else {
                uint32_t bits = (uint32_t)(k >> 32);
                memcpy(&dv, &bits, 4);
            }
        }
        if (cls) cls[p] = c;
        if (depth) depth[p] = dv;
        if (depth16) depth16[p] = h;
    }
}

/*
 * Rasterise snapped triangles into W x H.  Pixel (i, j) samples (16 i + 8, 16 j + 8).
 * Output per pixel: the max key (0 = background), the class (0 background, 1 road,
 * 2 lane line, 3 box, 4 signal: ids from line_end on) and the winner's depth (FP32 mode) or
 * its binary16 bits (FP16 mode).
 * The loop visits each triangle's snapped bounding box; or_raster_bruteforce visits every
 * pixel for every triangle and must give the same result.
 */
void or_raster(const or_tri *tris, int64_t n, int32_t W, int32_t H, int32_t key_f16,
               uint32_t box_end, uint32_t road_end, uint32_t line_end, uint64_t *key,
               uint8_t *cls, float *depth, uint16_t *depth16) {
    memset(key, 0, sizeof(uint64_t) * (size_t)W * (size_t)H);
    for (int64_t t = 0; t < n; ++t) {
        rtri r;
        if (!setup_rtri(tris + t, &r)) continue;
        int64_t xmin = r.X[0], xmax = r.X[0], ymin = r.Y[0], ymax = r.Y[0];
        for (int k = 1; k < 3; ++k) {
            if (r.X[k] < xmin) xmin = r.X[k];
            if (r.X[k] > xmax) xmax = r.X[k];
            if (r.Y[k] < ymin) ymin = r.Y[k];
            if (r.Y[k] > ymax) ymax = r.Y[k];
        }
        /* pixel i has centre 16 i + 8: i in [ceil((xmin-8)/16), floor((xmax-8)/16)] */
        int64_t i0 = -floor16(-(xmin - 8)), i1 = floor16(xmax - 8);
        int64_t j0 = -floor16(-(ymin - 8)), j1 = floor16(ymax - 8);
        if (i0 < 0) i0 = 0;
        if (j0 < 0) j0 = 0;
        if (i1 > W - 1) i1 = W - 1;
        if (j1 > H - 1) j1 = H - 1;
        for (int64_t j = j0; j <= j1; ++j)
            for (int64_t i = i0; i <= i1; ++i) {
                int64_t Xp = 16 * i + 8, Yp = 16 * j + 8;
                if (!covers(&r, Xp, Yp)) continue;
                uint64_t k = pixel_key(&r, Xp, Yp, key_f16);
                if (k > key[j * W + i]) key[j * W + i] = k;
            }
    }
    resolve(key, (int64_t)W * H, key_f16, box_end, road_end, line_end, cls, depth, depth16);
}

void or_raster_bruteforce(const or_tri *tris, int64_t n, int32_t W, int32_t H, int32_t key_f16,
                          uint32_t box_end, uint32_t road_end, uint32_t line_end, uint64_t *key,
                          uint8_t *cls, float *depth, uint16_t *depth16) {
    for (int32_t j = 0; j < H; ++j)
        for (int32_t i = 0; i < W; ++i) {
            uint64_t best = 0;
            for (int64_t t = 0; t < n; ++t) {
                rtri r;
                if (!setup_rtri(tris + t, &r)) continue;
                int64_t Xp = 16 * (int64_t)i + 8, Yp = 16 * (int64_t)j + 8;
                if (!covers(&r, Xp, Yp)) continue;
                uint64_t k = pixel_key(&r, Xp, Yp, key_f16);
                if (k > best) best = k;
            }
            key[(int64_t)j * W + i] = best;
        }
    resolve(key, (int64_t)W * H, key_f16, box_end, road_end, line_end, cls, depth, depth16);
}

/*
 * RGB observation (App. A "High-Throughput Batched Rendering": minimal shading, one
 * directional light per agent, a colour per instance -- blue for every vehicle and static
 * object in the paper's experiments).  Reading: a pixel's colour is
 *     base * (ambient + (1 - ambient) * max(0, n . l))
 * with base the winning primitive's class colour (all boxes share one colour), n its
 * outward unit normal in the world frame -- a box face's normal turned by the box's yaw,
 * +z for road and lane-line strips, a signal sphere's face normal (sphere_face) -- and l
 * the unit direction towards the light (the same light in every world).  A signal sphere's
 * base colour is that of its state (0 red, 1 amber, 2 green, 3 off).  Background pixels take
 * the background colour unshaded.  Each channel is quantised as rint(255 * clamp(v, 0, 1))
 * (round half to even).
 *   key [npx]: the raster's per-pixel keys; boxes [n][6]: x, y, yaw, L, W, H of the world's
 *   boxes (post-step); sph [n][4], sph_state [n]: its signal spheres; colour [4][3]: classes
 *   0 background, 1 road, 2 lane line, 3 box; sig_colour [4][3]: signal states;
 *   light [3] unit -> rgb [3][npx]
 */
void or_shade_rgb(const uint64_t *key, int64_t npx, int32_t key_f16, uint32_t box_end,
                  uint32_t road_end, uint32_t line_end, const double *boxes, const double *sph,
                  const uint8_t *sph_state, const double *colour, const double *sig_colour,
                  const double *light, double ambient, uint8_t *rgb) {
    for (int64_t p = 0; p < npx; ++p) {
        const uint64_t k = key[p];
        int cls = 0;
        double shade = 1.0;
        const double *base = colour;
        if (k) {
            const uint32_t prim = key_f16 ? (0xFFFFu - (uint32_t)(k & 0xFFFFu))
                                          : (0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFu));
            cls = prim_class(prim, box_end, road_end, line_end);
            double nx = 0.0, ny = 0.0, nz = 1.0;
            if (cls == 4) {
                const uint32_t s = (prim - line_end) / 64, q = ((prim - line_end) % 64) / 2;
                double off;
                const v3 n = sphere_face(sph + 4 * s, (int)q, &off);
                nx = n.x;
                ny = n.y;
                nz = n.z;
                base = sig_colour + 3 * sph_state[s];
            } else if (cls == 3) {
                const uint32_t b = prim / 12, face = (prim % 12) / 2;
                const double c = cos(boxes[6 * b + 2]), sn = sin(boxes[6 * b + 2]);
                switch (face) { /* +x, -x, +y, -y, +z, -z in the box frame */
                case 0: nx = c; ny = sn; nz = 0.0; break;
                case 1: nx = -c; ny = -sn; nz = 0.0; break;
                case 2: nx = -sn; ny = c; nz = 0.0; break;
                case 3: nx = sn; ny = -c; nz = 0.0; break;
                case 4: nx = 0.0; ny = 0.0; nz = 1.0; break;
                default: nx = 0.0; ny = 0.0; nz = -1.0; break;
                }
            }
            double ndl = nx * light[0] + ny * light[1] + nz * light[2];
            if (ndl < 0.0) ndl = 0.0;
            shade = ambient + (1.0 - ambient) * ndl;
        }
        if (cls != 4) base = colour + 3 * cls;
        for (int ch = 0; ch < 3; ++ch) {
            double v = base[ch] * shade;
            if (v < 0.0) v = 0.0;
            if (v > 1.0) v = 1.0;
            rgb[(int64_t)ch * npx + p] = (uint8_t)rint(255.0 * v);
        }
    }
}

/*
 * Policy-input encoding: 4-channel one-hot of the class image, normalised per channel,
 * bfloat16, NCHW.  value(c) = bf16((onehot_c - mean_c) / std_c), computed in FP32.  Signal
 * spheres (class 4) count as objects: channel 3, with the boxes.
 *   cls [n] -> out [4][n]
 */
void or_onehot_bf16(const uint8_t *cls, int64_t n, const float *mean, const float *std_,
                    uint16_t *out) {
    uint16_t val[4][2];
    for (int c = 0; c < 4; ++c)
        for (int hot = 0; hot < 2; ++hot) {
            float t = ((float)hot - mean[c]) / std_[c];
            val[c][hot] = or_f32_to_bf16(t);
        }
    for (int c = 0; c < 4; ++c)
        for (int64_t p = 0; p < n; ++p)
            out[(int64_t)c * n + p] = val[c][cls[p] == c || (c == 3 && cls[p] == 4)];
}
