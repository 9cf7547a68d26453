// Vectorized observations O_vec (App. A "Observations": surrounding agents and road
// geometry; the synthetic worlds have no traffic controls).  One CTA per world (persistent
// over worlds), one thread per agent; each thread keeps its nearest-first candidate list in
// shared memory (thread-major, so the lanes of a warp hit different banks).
//   agents: the other boxes (agents and static boxes, speed 0 for static ones) within
//     GP_OBS_AGENT_RADIUS, nearest first (ties to the lower index), at most GP_OBS_AGENTS;
//     slot = [1, x / R, y / R, L / 10, W / 5, cos(dth), sin(dth), dv / 30] in the ego frame
//     (x forward, y left);
//   roads: the centre lines of the road quads (type 0) and lane-line strips (type 1), each
//     from the midpoint of its q0-q3 edge to that of its q1-q2 edge, with midpoint within
//     GP_OBS_ROAD_RADIUS, nearest first (ties: roads before lines, then lower index), at most
//     GP_OBS_ROADS; candidates come from the world's grid cells that overlap the disc, each
//     segment counted in the cell of its midpoint only;
//     slot = [1, x / R, y / R, length / R, cos(dphi), sin(dphi), 1[road], 1[line]].
//   Unused slots are zero.
#include "gp_internal.h"

namespace gpk {

namespace {

constexpr int kObsThreads = kMaxBoxes;  // one thread per box slot of a world

struct ObsBox {
    float x, y, yaw, L, W, v;
};

// Insert (d, id) into a thread's nearest-first list of at most cap entries (thread-major
// arrays, stride kObsThreads), ordered by (d, id).
__device__ __forceinline__ void list_insert(float *ld, int *li, int &n, int cap, float d, int id) {
    const int tid = threadIdx.x;
    if (n == cap) {
        const float dl = ld[(cap - 1) * kObsThreads + tid];
        const int il = li[(cap - 1) * kObsThreads + tid];
        if (d > dl || (d == dl && id > il)) return;
    }
    int k = n < cap ? n : cap - 1;
    while (k > 0) {
        const float dp = ld[(k - 1) * kObsThreads + tid];
        const int ip = li[(k - 1) * kObsThreads + tid];
        if (dp < d || (dp == d && ip < id)) break;
        ld[k * kObsThreads + tid] = dp;
        li[k * kObsThreads + tid] = ip;
        --k;
    }
    ld[k * kObsThreads + tid] = d;
    li[k * kObsThreads + tid] = id;
    if (n < cap) ++n;
}

__device__ __forceinline__ void segment_of(float4 g0, float4 g1, float &mx, float &my, float &len,
                                           float &dx, float &dy) {
    // corners q0 q1 | q2 q3: from the midpoint of q0-q3 to the midpoint of q1-q2
    const float ax = 0.5f * (g0.x + g1.z), ay = 0.5f * (g0.y + g1.w);
    const float bx = 0.5f * (g0.z + g1.x), by = 0.5f * (g0.w + g1.y);
    dx = bx - ax;
    dy = by - ay;
    mx = 0.5f * (ax + bx);
    my = 0.5f * (ay + by);
    len = sqrtf(dx * dx + dy * dy);
}

__global__ void __launch_bounds__(kObsThreads) obs_kernel(ObsParams p) {
    __shared__ ObsBox bx[kMaxBoxes];
    __shared__ float ld[GP_OBS_ROADS * kObsThreads];
    __shared__ int li[GP_OBS_ROADS * kObsThreads];
    const int tid = threadIdx.x;
    for (int wl = blockIdx.x; wl < p.n_worlds; wl += gridDim.x) {
        const WorldInfo wi = p.worlds[wl];
        if (tid < wi.n_boxes) {
            const float4 q = p.box_pose[wi.box_begin + tid];
            const float4 d = p.box_dim[wi.box_begin + tid];
            bx[tid] = ObsBox{q.x, q.y, q.z, d.x, d.y,
                             tid < wi.n_agents ? p.speed[wi.agent_begin + tid] : 0.f};
        }
        __syncthreads();
        if (tid < wi.n_agents) {
            const ObsBox me = bx[tid];
            float sn, cs;
            sincosf(me.yaw, &sn, &cs);
            const int a = wi.agent_begin + tid;
            // surrounding agents
            int n = 0;
            for (int j = 0; j < wi.n_boxes; ++j) {
                if (j == tid) continue;
                const float dx = bx[j].x - me.x, dy = bx[j].y - me.y;
                const float d = sqrtf(dx * dx + dy * dy);
                if (d <= GP_OBS_AGENT_RADIUS) list_insert(ld, li, n, GP_OBS_AGENTS, d, j);
            }
            if (p.agents_out) {
                float *o = p.agents_out + (size_t)a * GP_OBS_AGENTS * 8;
                for (int k = 0; k < GP_OBS_AGENTS; ++k) {
                    float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                    if (k < n) {
                        const ObsBox b = bx[li[k * kObsThreads + tid]];
                        const float dx = b.x - me.x, dy = b.y - me.y;
                        float rs, rc;
                        sincosf(b.yaw - me.yaw, &rs, &rc);
                        f[0] = 1.f;
                        f[1] = (dx * cs + dy * sn) / GP_OBS_AGENT_RADIUS;
                        f[2] = (-dx * sn + dy * cs) / GP_OBS_AGENT_RADIUS;
                        f[3] = b.L / 10.f;
                        f[4] = b.W / 5.f;
                        f[5] = rc;
                        f[6] = rs;
                        f[7] = (b.v - me.v) / 30.f;
                    }
                    float4 *o4 = (float4 *)(o + 8 * k);
                    o4[0] = make_float4(f[0], f[1], f[2], f[3]);
                    o4[1] = make_float4(f[4], f[5], f[6], f[7]);
                }
            }
            // road geometry through the grid
            n = 0;
            const float R = GP_OBS_ROAD_RADIUS;
            const int cx0 = max(0, (int)floorf((me.x - R - wi.gx0) * wi.ginv));
            const int cx1 = min(wi.gnx - 1, (int)floorf((me.x + R - wi.gx0) * wi.ginv));
            const int cy0 = max(0, (int)floorf((me.y - R - wi.gy0) * wi.ginv));
            const int cy1 = min(wi.gny - 1, (int)floorf((me.y + R - wi.gy0) * wi.ginv));
            for (int cy = cy0; cy <= cy1; ++cy)
                for (int cx = cx0; cx <= cx1; ++cx)
                    for (int pass = 0; pass < 2; ++pass) {
                        const int *off = pass ? p.lcell_off : p.cell_off;
                        const int *list = pass ? p.lcell_quads : p.cell_quads;
                        const float4 *geo = pass ? p.line_geo : p.road_geo;
                        const int cell = (pass ? wi.lcell_begin : wi.cell_begin) + cy * wi.gnx + cx;
                        const int base = pass ? wi.line_begin : wi.road_begin;
                        for (int q = off[cell]; q < off[cell + 1]; ++q) {
                            const int r = list[q];
                            float mx, my, len, dx, dy;
                            segment_of(geo[2 * r], geo[2 * r + 1], mx, my, len, dx, dy);
                            // each segment is counted in the cell of its midpoint only
                            if ((int)floorf((mx - wi.gx0) * wi.ginv) != cx ||
                                (int)floorf((my - wi.gy0) * wi.ginv) != cy)
                                continue;
                            const float ex = mx - me.x, ey = my - me.y;
                            const float d = sqrtf(ex * ex + ey * ey);
                            if (d <= R)
                                list_insert(ld, li, n, GP_OBS_ROADS, d,
                                            pass ? wi.n_road + (r - base) : r - base);
                        }
                    }
            if (p.roads_out) {
                float *o = p.roads_out + (size_t)a * GP_OBS_ROADS * 8;
                for (int k = 0; k < GP_OBS_ROADS; ++k) {
                    float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                    if (k < n) {
                        const int s = li[k * kObsThreads + tid];
                        const bool is_line = s >= wi.n_road;
                        const int r = is_line ? wi.line_begin + (s - wi.n_road) : wi.road_begin + s;
                        const float4 *geo = is_line ? p.line_geo : p.road_geo;
                        float mx, my, len, dx, dy;
                        segment_of(geo[2 * r], geo[2 * r + 1], mx, my, len, dx, dy);
                        const float ex = mx - me.x, ey = my - me.y;
                        const float inv = len > 0.f ? 1.f / len : 0.f;
                        const float ux = dx * inv, uy = dy * inv;  // segment direction
                        f[0] = 1.f;
                        f[1] = (ex * cs + ey * sn) / R;
                        f[2] = (-ex * sn + ey * cs) / R;
                        f[3] = len / R;
                        f[4] = ux * cs + uy * sn;   // cos(phi - yaw)
                        f[5] = uy * cs - ux * sn;   // sin(phi - yaw)
                        f[6] = is_line ? 0.f : 1.f;
                        f[7] = is_line ? 1.f : 0.f;
                    }
                    float4 *o4 = (float4 *)(o + 8 * k);
                    o4[0] = make_float4(f[0], f[1], f[2], f[3]);
                    o4[1] = make_float4(f[4], f[5], f[6], f[7]);
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_obs(const ObsParams &p, int max_blocks, cudaStream_t s) {
    if (p.n_worlds <= 0) return cudaSuccess;
    const int blocks = p.n_worlds < max_blocks ? p.n_worlds : max_blocks;
    obs_kernel<<<blocks, kObsThreads, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace gpk
