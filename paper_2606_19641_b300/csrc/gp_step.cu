// Step kernel: one CTA per world (persistent over worlds), one thread per box slot.
//
// Per world (App. A "Action Space and Dynamics", "Other Details"):
//   1. every non-halted agent advances by a kinematic bicycle with wheelbase 0.6 L,
//      centre reference point (l_r = l_f = 0.3 L), explicit Euler with the speed at the
//      start of the step, then v += a dt clamped to [0, v_max]; under the jerk dynamics the
//      action's jerks first move the actuator state (a_lon, a_lat, steer), which then gives
//      the bicycle's acceleration and steering (jerk_actuate);
//   2. footprint collisions: all pairs (agent, box) by the separating-axis test on the
//      four box axes, strict overlap (touching is no collision);
//   3. off-road: an agent whose footprint has a corner outside every road quad (boundary
//      counts as inside); candidate quads come from a per-world uniform grid;
//   4. red light: an agent whose centre enters, during the step, the road quad controlled
//      by a red signal (the quad of smallest index under the signal's centre) is flagged;
//   5. halt: collided, off-road or red-light agents are latched halted with v = 0.  Halted
//      agents keep their pose and stay in the scene as obstacles.
// All arithmetic is FP32 with full-precision libm (no fast-math).
#include "gp_internal.h"

namespace gpk {

namespace {

constexpr float kPi = 3.14159265358979f;

struct Footprint {
    float x, y, c, s, hl, hw;  // centre, heading cos/sin, half length/width
};

__device__ __forceinline__ float axis_radius(const Footprint &b, float ux, float uy) {
    return b.hl * fabsf(b.c * ux + b.s * uy) + b.hw * fabsf(-b.s * ux + b.c * uy);
}

// Interiors intersect iff on each of the four axes the centre distance is strictly less
// than the sum of the projected half-extents.
__device__ bool footprints_overlap(const Footprint &a, const Footprint &b) {
    const float ax[4] = {a.c, -a.s, b.c, -b.s};
    const float ay[4] = {a.s, a.c, b.s, b.c};
    const float dx = b.x - a.x, dy = b.y - a.y;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float d = fabsf(dx * ax[k] + dy * ay[k]);
        if (!(d < axis_radius(a, ax[k], ay[k]) + axis_radius(b, ax[k], ay[k]))) return false;
    }
    return true;
}

__device__ __forceinline__ bool in_quad(float px, float py, float4 g0, float4 g1) {
    const float qx[4] = {g0.x, g0.z, g1.x, g1.z};
    const float qy[4] = {g0.y, g0.w, g1.y, g1.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int n = (k + 1) & 3;
        const float cr = (qx[n] - qx[k]) * (py - qy[k]) - (qy[n] - qy[k]) * (px - qx[k]);
        if (cr < 0.f) return false;
    }
    return true;
}

__device__ __forceinline__ float wrap_pi(float a) {
    if (a > kPi) a -= 2.f * kPi;
    if (a <= -kPi) a += 2.f * kPi;
    return a;
}

// Lane frame of a point: the road quad of smallest index containing it (boundary inside);
// the quad runs from its q0-q3 edge to its q1-q2 edge; with right-hand traffic on two lanes
// the half right of the centre line runs along that direction, the left half against it.
// x_f = offset from the lane's centre line.  False off the road.
__device__ bool lane_frame(const StepParams &p, const WorldInfo &wi, float px, float py,
                           float &lane_dir, float &xf) {
    const float fx = floorf((px - wi.gx0) * wi.ginv);
    const float fy = floorf((py - wi.gy0) * wi.ginv);
    if (!(fx >= 0.f && fy >= 0.f && fx < (float)wi.gnx && fy < (float)wi.gny)) return false;
    const int cell = wi.cell_begin + (int)fy * wi.gnx + (int)fx;
    int best = 0x7FFFFFFF;
    for (int q = p.cell_off[cell]; q < p.cell_off[cell + 1]; ++q) {
        const int r = p.cell_quads[q];
        if (r < best && in_quad(px, py, p.road_geo[2 * r], p.road_geo[2 * r + 1])) best = r;
    }
    if (best == 0x7FFFFFFF) return false;
    const float4 g0 = p.road_geo[2 * best], g1 = p.road_geo[2 * best + 1];  // q0 q1 | q2 q3
    const float m0x = 0.5f * (g0.x + g1.z), m0y = 0.5f * (g0.y + g1.w);
    const float m1x = 0.5f * (g0.z + g1.x), m1y = 0.5f * (g0.w + g1.y);
    float dx = m1x - m0x, dy = m1y - m0y;
    const float inv = rsqrtf(dx * dx + dy * dy);
    dx *= inv;
    dy *= inv;
    const float cx = 0.25f * (g0.x + g0.z + g1.x + g1.z), cy = 0.25f * (g0.y + g0.w + g1.y + g1.w);
    const float s = (px - cx) * (-dy) + (py - cy) * dx;
    if (s < 0.f) {
        lane_dir = atan2f(dy, dx);
        xf = s + 0.5f * p.lane_w;
    } else {
        lane_dir = atan2f(-dy, -dx);
        xf = s - 0.5f * p.lane_w;
    }
    return true;
}

// Reward conditioning (App. A "Reward Functions and Reward Conditioning", Table "Reward
// terms", training distribution): coefficient k of the agent with index i in world w, in
// its episode e, is lo_k + (hi_k - lo_k) u with u the top 24 bits of output
// n = 1 + (w << 40 | e << 20 | i << 4 | k) of the SplitMix64 stream seeded with `seed`
// (the stream's n-th output is its finaliser applied to seed + n * golden gamma), scaled by
// 2^-24; the policy sees 2 u - 1.  Coefficients 0..9 are the reward weights, 10..11 the goal
// radius and goal speed tolerance (observed only).
__device__ __forceinline__ uint32_t splitmix_top24(unsigned long long seed, unsigned long long n) {
    unsigned long long z = seed + n * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return (uint32_t)((z ^ (z >> 31)) >> 40);
}

__device__ __forceinline__ void draw_conditioning(unsigned long long seed, int world, int episode,
                                                  int agent, float *w10, float *c12) {
    const float lo[12] = {0.f, 0.f, 0.f, 2.5e-4f, 2.5e-4f, 0.f, 0.f, 0.f, 2.5e-4f, 0.f, 2.f, 1.f};
    const float hi[12] = {3.f, 3.f, 0.05f, 2.5e-2f, 7.5e-3f, 5e-3f, 1.f, 5e-5f, 7.5e-3f, 1.f, 12.f, 5.f};
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const unsigned long long c = ((unsigned long long)world << 40) |
                                     ((unsigned long long)(episode & 0xFFFFF) << 20) |
                                     ((unsigned long long)(agent & 0xFFFF) << 4) | (unsigned long long)k;
        const float u = (float)splitmix_top24(seed, c + 1) * (1.f / 16777216.f);
        if (k < 10) w10[k] = lo[k] + (hi[k] - lo[k]) * u;
        c12[k] = 2.f * u - 1.f;
    }
}

// Jerk-actuated control (App. A "Action Space and Dynamics"): the longitudinal and lateral
// jerks move the accelerations, clipped to a_lon in [-5, 3] and |a_lat| <= 4 m/s^2; the
// steering angle follows the curvature a_lat / max(v^2, 1) through tan(steer) = kappa 0.6 L,
// limited to 0.5 rad/s of change and to |steer| <= 0.5 rad.  Returns the bicycle's
// (acceleration, steering) and updates the state st = (a_lon, a_lat, steer).
__device__ __forceinline__ float2 jerk_actuate(float2 jerk, float v, float L, float dt, float *st) {
    const float a_lon = fminf(fmaxf(st[0] + jerk.x * dt, -5.f), 3.f);
    const float a_lat = fminf(fmaxf(st[1] + jerk.y * dt, -4.f), 4.f);
    const float v2 = fmaxf(v * v, 1.f);
    float steer = atanf((a_lat / v2) * 0.6f * L);
    const float step = 0.5f * dt;
    steer = fmaxf(fminf(steer, st[2] + step), st[2] - step);
    steer = fmaxf(fminf(steer, 0.5f), -0.5f);
    st[0] = a_lon;
    st[1] = a_lat;
    st[2] = steer;
    return make_float2(a_lon, steer);
}

// Red-light violation of one step: the centre moved from outside to inside the road quad
// controlled by a red signal of the world (signal states are read modulo 4).
__device__ bool entered_red(const StepParams &p, const WorldInfo &wi, float px0, float py0,
                            float px, float py) {
    for (int s = 0; s < wi.n_sig; ++s) {
        const int q = p.sig_quad[wi.sig_begin + s];
        if (q < 0 || (p.sig_state[wi.sig_begin + s] & 3) != GP_SIGNAL_RED) continue;
        const float4 g0 = p.road_geo[2 * q], g1 = p.road_geo[2 * q + 1];
        if (!in_quad(px0, py0, g0, g1) && in_quad(px, py, g0, g1)) return true;
    }
    return false;
}

// Reward terms of one agent's step (App. A reward table; inference weights by default) and
// its ego state.  Accelerations are the bicycle's increments of the step (speed before any
// halt); an agent halted before the step earns 0.  The traffic-light term charges the
// step's red-light violation (`ran_red`, charged once however many red signals it crossed);
// the goal term is 0.
__device__ void agent_reward(const StepParams &p, const WorldInfo &wi, int a, float px, float py,
                             float yaw, float v_after, float v0, float2 act, float L, float W,
                             unsigned int fl0, unsigned int fl1, bool ran_red) {
    const float *w = p.weights + 10 * a;
    float a_lon = 0.f, a_lat = 0.f, r = 0.f;
    if (!(fl0 & GP_FLAG_HALTED)) {
        const float lr = 0.3f * L;
        const float beta = atanf(0.5f * tanf(act.y));
        const float vn = fminf(fmaxf(v0 + act.x * p.dt, 0.f), p.vmax);
        const float dyaw = (v0 / lr) * sinf(beta) * p.dt;
        a_lon = (vn - v0) / p.dt;
        a_lat = v0 * dyaw / p.dt;
        const float2 ap = p.acc[a];
        const float j_lon = (a_lon - ap.x) / p.dt, j_lat = (a_lat - ap.y) / p.dt;
        if (fl1 & GP_FLAG_COLLIDED) r -= w[0] + 0.1f * fabsf(v0);
        if (fl1 & GP_FLAG_OFFROAD) r -= w[1];
        r -= w[2] * (float)((fabsf(a_lon) > 3.f) + (fabsf(a_lat) > 3.f) +
                            (fabsf(j_lon) > 5.f || fabsf(j_lat) > 5.f));
        float lane_dir, xf;
        if (lane_frame(p, wi, px, py, lane_dir, xf)) {
            const float th = fabsf(wrap_pi(yaw - lane_dir));
            const float ct = cosf(th);
            r += w[3] * p.dt * (fminf(ct, 0.f) + fminf(vn * ct, 0.f) + 0.0025f * (1.f - 2.f * th / kPi));
            r -= w[4] * p.dt * ((ct > 0.5f ? fabsf(xf) : 0.f) - 0.05f * expf(0.5f - fabsf(xf)));
            if (fabsf(vn) > 2.5f) r += w[5] * p.dt * fmaxf(ct, 0.f);
        }
        if (fabsf(vn) > 0.f || a_lon != 0.f || a_lat != 0.f) r -= w[7] * p.dt;
        if (vn < 0.f) r -= w[8] * p.dt;
        if (fabsf(vn) > p.vlim) r -= w[9];
        if (ran_red) r -= w[6];
    }
    p.acc[a] = make_float2(a_lon, a_lat);
    p.reward[a] = r;
    float *e = p.ego + GP_EGO_DIM * a;
    e[0] = fmaxf(-1.f, fminf(1.f, v_after / p.vmax));
    e[1] = fmaxf(-1.f, fminf(1.f, a_lon / 10.f));
    e[2] = fmaxf(-1.f, fminf(1.f, a_lat / 10.f));
    e[3] = fmaxf(-1.f, fminf(1.f, L / 10.f));
    e[4] = fmaxf(-1.f, fminf(1.f, W / 5.f));
    e[5] = (fl1 & GP_FLAG_COLLIDED) ? 1.f : 0.f;
    // jerk dynamics: steering angle and actuator accelerations, each over its limit
    const float *js = p.dynamics ? p.jerk + 3 * a : nullptr;
    e[6] = js ? js[2] / 0.5f : 0.f;
    e[7] = js ? js[0] / 5.f : 0.f;
    e[8] = js ? js[1] / 4.f : 0.f;
}

__global__ void __launch_bounds__(kMaxBoxes) step_kernel(StepParams p) {
    __shared__ Footprint fp[kMaxBoxes];
    __shared__ unsigned int sflag[kMaxBoxes];
    const int tid = threadIdx.x;
    // the render launched after this step in the same graph takes its work items from this
    // counter (saves a memset node between the two kernels)
    if (p.render_counter && blockIdx.x == 0 && tid == 0) *p.render_counter = 0;

    for (int wl = blockIdx.x; wl < p.n_worlds; wl += gridDim.x) {
        const WorldInfo wi = p.worlds[p.world_begin + wl];
        float4 pose = make_float4(0.f, 0.f, 0.f, 0.f), dim = pose;
        float v = 0.f, v0 = 0.f;
        unsigned int fl = 0, fl0 = 0;
        float2 act = make_float2(0.f, 0.f);
        if (tid < wi.n_boxes) {
            pose = p.box_pose[wi.box_begin + tid];
            dim = p.box_dim[wi.box_begin + tid];
        }
        const float x0 = pose.x, y0 = pose.y;  // centre before the step (red-light test)
        if (tid < wi.n_agents) {
            const int a = wi.agent_begin + tid;
            fl = p.flags[a] & ~GP_FLAG_DONE;  // the done flag lasts one step
            fl0 = fl;
            v = p.speed[a];
            v0 = v;
            if (!(fl & GP_FLAG_HALTED)) {
                act = p.actions[a];
                if (p.dynamics) {
                    float st[3] = {p.jerk[3 * a], p.jerk[3 * a + 1], p.jerk[3 * a + 2]};
                    act = jerk_actuate(act, v, dim.x, p.dt, st);
                    p.jerk[3 * a] = st[0];
                    p.jerk[3 * a + 1] = st[1];
                    p.jerk[3 * a + 2] = st[2];
                }
                const float lr = 0.3f * dim.x;
                const float beta = atanf(0.5f * tanf(act.y));
                float sb, cb;
                sincosf(pose.z + beta, &sb, &cb);
                pose.x += v * cb * p.dt;
                pose.y += v * sb * p.dt;
                float yaw = pose.z + (v / lr) * sinf(beta) * p.dt;
                if (yaw > kPi) yaw -= 2.f * kPi;
                if (yaw <= -kPi) yaw += 2.f * kPi;
                pose.z = yaw;
                v = fminf(fmaxf(v + act.x * p.dt, 0.f), p.vmax);
            } else {
                v = 0.f;
                if (p.dynamics) p.jerk[3 * a] = p.jerk[3 * a + 1] = p.jerk[3 * a + 2] = 0.f;
            }
            if (!isfinite(pose.x) || !isfinite(pose.y) || !isfinite(pose.z) || !isfinite(v))
                atomicOr(p.status, GP_DEV_NONFINITE_STATE);
        }
        if (tid < wi.n_boxes) {
            float s, c;
            sincosf(pose.z, &s, &c);
            fp[tid] = Footprint{pose.x, pose.y, c, s, 0.5f * dim.x, 0.5f * dim.y};
        }
        sflag[tid] = 0;
        __syncthreads();

        // collisions: pairs (i, j), i an agent, j > i any box
        const int na = wi.n_agents, nb = wi.n_boxes;
        for (int idx = tid; idx < na * nb; idx += blockDim.x) {
            const int i = idx / nb, j = idx - i * nb;
            if (j <= i) continue;
            if (footprints_overlap(fp[i], fp[j])) {
                atomicOr(&sflag[i], GP_FLAG_COLLIDED);
                if (j < na) atomicOr(&sflag[j], GP_FLAG_COLLIDED);
            }
        }

        // off-road: every footprint corner must lie in some road quad; one (agent, corner)
        // pair per thread, so the candidate-quad searches of an agent's corners run side by
        // side
        for (int pc = tid; pc < 4 * na; pc += blockDim.x) {
            const int i = pc >> 2, k = pc & 3;
            const Footprint b = fp[i];
            const float lx = ((k == 1 || k == 2) ? 1.f : -1.f) * b.hl;
            const float ly = (k >= 2 ? 1.f : -1.f) * b.hw;
            const float px = b.x + b.c * lx - b.s * ly;
            const float py = b.y + b.s * lx + b.c * ly;
            const float fx = floorf((px - wi.gx0) * wi.ginv);
            const float fy = floorf((py - wi.gy0) * wi.ginv);
            bool inside = false;
            if (fx >= 0.f && fy >= 0.f && fx < (float)wi.gnx && fy < (float)wi.gny) {
                const int cell = wi.cell_begin + (int)fy * wi.gnx + (int)fx;
                // four candidates per round trip: their loads are independent
                const int q1 = p.cell_off[cell + 1];
                for (int q = p.cell_off[cell]; q < q1 && !inside; q += 4) {
                    int r[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) r[u] = q + u < q1 ? p.cell_quads[q + u] : -1;
                    float4 g0[4], g1[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        g0[u] = g1[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (r[u] >= 0) {
                            g0[u] = p.road_geo[2 * r[u]];
                            g1[u] = p.road_geo[2 * r[u] + 1];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (r[u] >= 0 && in_quad(px, py, g0[u], g1[u])) inside = true;
                }
            }
            if (!inside) atomicOr(&sflag[i], GP_FLAG_OFFROAD);
        }
        __syncthreads();

        if (tid < na) {
            const int a = wi.agent_begin + tid;
            fl |= sflag[tid];
            // a halted agent did not move, so it cannot have entered a quad
            const bool ran_red = !(fl0 & GP_FLAG_HALTED) && entered_red(p, wi, x0, y0, pose.x, pose.y);
            if (ran_red) fl |= GP_FLAG_RED_LIGHT;
            if (fl & (GP_FLAG_COLLIDED | GP_FLAG_OFFROAD | GP_FLAG_RED_LIGHT)) {
                fl |= GP_FLAG_HALTED;
                v = 0.f;
            }
            p.box_pose[wi.box_begin + tid] = pose;
            p.speed[a] = v;
            p.flags[a] = (uint8_t)fl;
            if (p.rewards)
                agent_reward(p, wi, a, pose.x, pose.y, pose.z, v, v0, act, dim.x, dim.y, fl0, fl,
                             ran_red);
        }
        if (p.episode_steps > 0) {
            // end of the world's episode: its agents return to their initial state (the
            // step's rewards stand); the done flag marks it for one step
            __shared__ int s_done;
            __syncthreads();
            if (tid == 0) {
                int *c = p.ep_counter + p.world_begin + wl;
                const int n = *c + 1 >= p.episode_steps ? 0 : *c + 1;
                *c = n;
                s_done = n == 0;
            }
            __syncthreads();
            if (s_done && tid < na) {
                const int a = wi.agent_begin + tid;
                p.box_pose[wi.box_begin + tid] = p.pose0[wi.box_begin + tid];
                p.speed[a] = p.speed0[a];
                p.flags[a] = GP_FLAG_DONE;
                p.acc[a] = make_float2(0.f, 0.f);
                if (p.dynamics) p.jerk[3 * a] = p.jerk[3 * a + 1] = p.jerk[3 * a + 2] = 0.f;
                const int e = ++p.ep_index[a];
                if (p.conditioning)
                    draw_conditioning(p.cond_seed, p.world_begin + wl, e, tid, p.weights + 10 * a,
                                      p.cond + 12 * a);
            }
        }
        __syncthreads();
    }
}

// Gather (to_state = 1) or scatter (0) agent state rows x, y, yaw, v and flags.
__global__ void state_kernel(float *state, uint8_t *flags, float4 *pose, float *speed,
                             uint8_t *fl, const int *agent_box, int n, int to_state) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    const int b = agent_box[a];
    if (to_state) {
        const float4 q = pose[b];
        state[4 * a + 0] = q.x;
        state[4 * a + 1] = q.y;
        state[4 * a + 2] = q.z;
        state[4 * a + 3] = speed[a];
        flags[a] = fl[a];
    } else {
        pose[b] = make_float4(state[4 * a + 0], state[4 * a + 1], state[4 * a + 2], 0.f);
        speed[a] = state[4 * a + 3];
        fl[a] = flags[a];
    }
}

// Episode reset: the agents of every world whose mask byte is non-zero (every world if
// mask is null) get their initial pose and speed back, with clear flags, zero previous-step
// accelerations and zero actuator state.
__global__ void reset_kernel(ResetParams p) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (p.draw_only) {
        if (a < p.n_agents && p.conditioning) {
            const int w = p.agent_world[a];
            draw_conditioning(p.cond_seed, w, p.ep_index[a], a - p.worlds[w].agent_begin,
                              p.weights + 10 * a, p.cond + 12 * a);
        }
        return;
    }
    if (a < p.n_worlds && (!p.mask || p.mask[a])) p.ep_counter[a] = 0;
    if (a >= p.n_agents) return;
    if (p.mask && !p.mask[p.agent_world[a]]) return;
    {
        const int w = p.agent_world[a];
        const int e = ++p.ep_index[a];
        if (p.conditioning)
            draw_conditioning(p.cond_seed, w, e, a - p.worlds[w].agent_begin, p.weights + 10 * a,
                              p.cond + 12 * a);
    }
    const int b = p.agent_box[a];
    p.pose[b] = p.pose0[b];
    p.speed[a] = p.speed0[a];
    p.flags[a] = 0;
    p.acc[a] = make_float2(0.f, 0.f);
    p.jerk[3 * a] = p.jerk[3 * a + 1] = p.jerk[3 * a + 2] = 0.f;
}

}  // namespace

cudaError_t launch_reset(const ResetParams &p, cudaStream_t s) {
    const int n = p.n_agents > p.n_worlds ? p.n_agents : p.n_worlds;
    if (n <= 0) return cudaSuccess;
    reset_kernel<<<(n + 255) / 256, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_step(const StepParams &p, int max_blocks, cudaStream_t s) {
    if (p.n_worlds <= 0) return cudaSuccess;
    const int blocks = p.n_worlds < max_blocks ? p.n_worlds : max_blocks;
    step_kernel<<<blocks, kMaxBoxes, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_state(float *state, uint8_t *flags, float4 *pose, float *speed, uint8_t *fl,
                         const int *agent_box, int n, int to_state, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    state_kernel<<<(n + 255) / 256, 256, 0, s>>>(state, flags, pose, speed, fl, agent_box, n,
                                                 to_state);
    return cudaGetLastError();
}

}  // namespace gpk
