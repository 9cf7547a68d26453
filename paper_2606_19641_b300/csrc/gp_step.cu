// Step kernel: one CTA per world (persistent over worlds), one thread per box slot.
//
// Per world (App. A "Action Space and Dynamics", "Other Details"):
//   1. every non-halted agent advances by a kinematic bicycle with wheelbase 0.6 L,
//      centre reference point (l_r = l_f = 0.3 L), explicit Euler with the speed at the
//      start of the step, then v += a dt clamped to [0, v_max];
//   2. footprint collisions: all pairs (agent, box) by the separating-axis test on the
//      four box axes, strict overlap (touching is no collision);
//   3. off-road: an agent whose footprint has a corner outside every road quad (boundary
//      counts as inside); candidate quads come from a per-world uniform grid;
//   4. halt: collided or off-road agents are latched halted with v = 0.  Halted agents keep
//      their pose and stay in the scene as obstacles.
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

__global__ void __launch_bounds__(kMaxBoxes) step_kernel(StepParams p) {
    __shared__ Footprint fp[kMaxBoxes];
    __shared__ unsigned int sflag[kMaxBoxes];
    const int tid = threadIdx.x;

    for (int wl = blockIdx.x; wl < p.n_worlds; wl += gridDim.x) {
        const WorldInfo wi = p.worlds[p.world_begin + wl];
        float4 pose = make_float4(0.f, 0.f, 0.f, 0.f), dim = pose;
        float v = 0.f;
        unsigned int fl = 0;
        if (tid < wi.n_boxes) {
            pose = p.box_pose[wi.box_begin + tid];
            dim = p.box_dim[wi.box_begin + tid];
        }
        if (tid < wi.n_agents) {
            const int a = wi.agent_begin + tid;
            fl = p.flags[a];
            v = p.speed[a];
            if (!(fl & GP_FLAG_HALTED)) {
                const float2 act = p.actions[a];
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
            if (fl & (GP_FLAG_COLLIDED | GP_FLAG_OFFROAD)) {
                fl |= GP_FLAG_HALTED;
                v = 0.f;
            }
            p.box_pose[wi.box_begin + tid] = pose;
            p.speed[a] = v;
            p.flags[a] = (uint8_t)fl;
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

}  // namespace

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
