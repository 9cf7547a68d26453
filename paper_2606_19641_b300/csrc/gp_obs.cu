// Vectorized observations O_vec (App. A "Observations": surrounding agents, road geometry
// and traffic controls).  One warp per agent.  Each of the three selections keeps the
// nearest candidates as a sorted list spread over the warp's lanes (lane i holds the i-th
// nearest, as a 64-bit key: distance bits above the candidate id, so keys order by distance
// and then by id); candidates that beat the current K-th are staged in shared memory, and
// every 32 of them are sorted across the lanes (bitonic network on shuffles) and merged into
// the list (bitonic merge).  Slots:
//   agents: the other boxes (agents and static boxes, speed 0 for static ones) within
//     GP_OBS_AGENT_RADIUS, nearest first (ties to the lower index), at most GP_OBS_AGENTS;
//     slot = [1, x / R, y / R, L / 10, W / 5, cos(dth), sin(dth), dv / 30] in the ego frame
//     (x forward, y left);
//   roads: the centre lines of the road quads (type 0) and lane-line strips (type 1), each
//     from the midpoint of its q0-q3 edge to that of its q1-q2 edge, with midpoint within
//     GP_OBS_ROAD_RADIUS, nearest first (ties: roads before lines, then lower index), at most
//     GP_OBS_ROADS; candidates come from the world's grid cells that overlap the disc, each
//     segment listed once, in the cell of its midpoint;
//     slot = [1, x / R, y / R, length / R, cos(dphi), sin(dphi), 1[road], 1[line]];
//   signals: the traffic-signal spheres with centre within GP_OBS_SIGNAL_RADIUS on the
//     ground plane, nearest first (ties to the lower index), at most GP_OBS_SIGNALS;
//     slot = [1, x / R, y / R, z / 10, 1[red], 1[amber], 1[green], 1[off]].
//   Unused slots are zero.
#include "gp_internal.h"

namespace gpk {

namespace {

constexpr int kObsWarps = 4;  // agents per block
constexpr unsigned long long kNone = ~0ull;

__device__ __forceinline__ unsigned long long shfl_xor64(unsigned long long v, int m) {
    return ((unsigned long long)__shfl_xor_sync(0xffffffffu, (unsigned int)(v >> 32), m) << 32) |
           __shfl_xor_sync(0xffffffffu, (unsigned int)v, m);
}

__device__ __forceinline__ unsigned long long shfl64(unsigned long long v, int src) {
    return ((unsigned long long)__shfl_sync(0xffffffffu, (unsigned int)(v >> 32), src) << 32) |
           __shfl_sync(0xffffffffu, (unsigned int)v, src);
}

// Ascending sort of one key per lane across the warp (bitonic network).
__device__ __forceinline__ unsigned long long warp_sort32(unsigned long long k) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
        const bool up = (lane & size) == 0 || size == 32;
#pragma unroll
        for (int j = size >> 1; j > 0; j >>= 1) {
            const unsigned long long o = shfl_xor64(k, j);
            const bool keep_min = ((lane & j) == 0) == up;
            k = keep_min ? (o < k ? o : k) : (o > k ? o : k);
        }
    }
    return k;
}

// The 32 smallest of two ascending lane-spread lists, ascending.
__device__ __forceinline__ unsigned long long warp_merge32(unsigned long long a, unsigned long long b) {
    const int lane = threadIdx.x & 31;
    const unsigned long long br = shfl64(b, 31 - lane);
    unsigned long long k = a < br ? a : br;  // bitonic: rises then falls
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        const unsigned long long o = shfl_xor64(k, j);
        k = (lane & j) == 0 ? (o < k ? o : k) : (o > k ? o : k);
    }
    return k;
}

// Nearest-K selection of one warp: the sorted list, its admission threshold (the K-th key)
// and the staging area of admitted candidates not yet merged.
struct NearestK {
    unsigned long long list = kNone, thr = kNone;
    int ns = 0;  // staged keys (warp-uniform)
    int K;
    unsigned long long *stage;  // 64 keys of this warp

    __device__ explicit NearestK(int k, unsigned long long *st) : K(k), stage(st) {}

    __device__ __forceinline__ void flush32() {
        const int lane = threadIdx.x & 31;
        __syncwarp();
        const unsigned long long b = warp_sort32(lane < ns ? stage[lane] : kNone);
        list = warp_merge32(list, b);
        thr = shfl64(list, K - 1);
        __syncwarp();
        if (lane + 32 < ns) stage[lane] = stage[lane + 32];
        ns = ns > 32 ? ns - 32 : 0;
        __syncwarp();
    }

    // Offer one key per lane (ok = false: none); warp-uniform call.
    __device__ __forceinline__ void offer(bool ok, unsigned long long key) {
        const int lane = threadIdx.x & 31;
        ok = ok && key < thr;
        const unsigned int m = __ballot_sync(0xffffffffu, ok);
        if (ok) stage[ns + __popc(m & ((1u << lane) - 1u))] = key;
        ns += __popc(m);
        if (ns >= 32) flush32();
    }

    __device__ __forceinline__ void finish() {
        if (ns > 0) flush32();
    }
};

__device__ __forceinline__ unsigned long long make_key(float d, uint32_t id) {
    return ((unsigned long long)__float_as_uint(d) << 32) | id;
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

__device__ __forceinline__ void store_slot(float *o, const float f[8]) {
    float4 *o4 = (float4 *)o;
    o4[0] = make_float4(f[0], f[1], f[2], f[3]);
    o4[1] = make_float4(f[4], f[5], f[6], f[7]);
}

__global__ void __launch_bounds__(32 * kObsWarps) obs_kernel(ObsParams p) {
    __shared__ unsigned long long stage[kObsWarps][64];
    const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    const int a = blockIdx.x * kObsWarps + wb;
    if (a >= p.n_agents) return;  // whole warps leave together
    const WorldInfo wi = p.worlds[p.agent_world[a]];
    const int me_box = wi.box_begin + (a - wi.agent_begin);
    const float4 me = p.box_pose[me_box];
    const float me_v = p.speed[a];
    float sn, cs;
    sincosf(me.z, &sn, &cs);

    // surrounding agents
    if (p.agents_out) {
        NearestK sel(GP_OBS_AGENTS, stage[wb]);
        for (int base = 0; base < wi.n_boxes; base += 32) {
            const int j = base + lane;
            bool ok = false;
            float d = 0.f;
            if (j < wi.n_boxes && wi.box_begin + j != me_box) {
                const float4 q = p.box_pose[wi.box_begin + j];
                const float dx = q.x - me.x, dy = q.y - me.y;
                d = sqrtf(dx * dx + dy * dy);
                ok = d <= GP_OBS_AGENT_RADIUS;
            }
            sel.offer(ok, make_key(d, (uint32_t)j));
        }
        sel.finish();
        if (lane < GP_OBS_AGENTS) {
            float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (sel.list != kNone) {
                const int j = (int)(sel.list & 0xFFFFFFFFu);
                const float4 q = p.box_pose[wi.box_begin + j];
                const float4 dm = p.box_dim[wi.box_begin + j];
                const float v = j < wi.n_agents ? p.speed[wi.agent_begin + j] : 0.f;
                const float dx = q.x - me.x, dy = q.y - me.y;
                float rs, rc;
                sincosf(q.z - me.z, &rs, &rc);
                f[0] = 1.f;
                f[1] = (dx * cs + dy * sn) / GP_OBS_AGENT_RADIUS;
                f[2] = (-dx * sn + dy * cs) / GP_OBS_AGENT_RADIUS;
                f[3] = dm.x / 10.f;
                f[4] = dm.y / 5.f;
                f[5] = rc;
                f[6] = rs;
                f[7] = (v - me_v) / 30.f;
            }
            store_slot(p.agents_out + ((size_t)a * GP_OBS_AGENTS + lane) * 8, f);
        }
    }

    // road geometry: the rows of grid cells overlapping the disc's bounding square; the
    // cells of one row are adjacent in the midpoint lists, so each row is one range
    if (p.roads_out) {
        NearestK sel(GP_OBS_ROADS, stage[wb]);
        const float R = GP_OBS_ROAD_RADIUS;
        const int cx0 = max(0, (int)floorf((me.x - R - wi.gx0) * wi.ginv));
        const int cx1 = min(wi.gnx - 1, (int)floorf((me.x + R - wi.gx0) * wi.ginv));
        const int cy0 = max(0, (int)floorf((me.y - R - wi.gy0) * wi.ginv));
        const int cy1 = min(wi.gny - 1, (int)floorf((me.y + R - wi.gy0) * wi.ginv));
        for (int cy = cy0; cy <= cy1 && cx0 <= cx1; ++cy) {
            const int c0 = wi.scell_begin + cy * wi.gnx;
            const int e0 = p.seg_off[c0 + cx0], e1 = p.seg_off[c0 + cx1 + 1];
            for (int e = e0; e < e1; e += 32) {
                bool ok = false;
                float d = 0.f;
                uint32_t s = 0;
                if (e + lane < e1) {
                    s = (uint32_t)p.seg_list[e + lane];
                    const bool is_line = (int)s >= wi.n_road;
                    const int r = is_line ? wi.line_begin + ((int)s - wi.n_road) : wi.road_begin + (int)s;
                    const float4 *geo = is_line ? p.line_geo : p.road_geo;
                    float mx, my, len, dx, dy;
                    segment_of(geo[2 * r], geo[2 * r + 1], mx, my, len, dx, dy);
                    const float ex = mx - me.x, ey = my - me.y;
                    d = sqrtf(ex * ex + ey * ey);
                    ok = d <= R;
                }
                sel.offer(ok, make_key(d, s));
            }
        }
        sel.finish();
        float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (sel.list != kNone) {
            const int s = (int)(sel.list & 0xFFFFFFFFu);
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
            f[4] = ux * cs + uy * sn;  // cos(phi - yaw)
            f[5] = uy * cs - ux * sn;  // sin(phi - yaw)
            f[6] = is_line ? 0.f : 1.f;
            f[7] = is_line ? 1.f : 0.f;
        }
        store_slot(p.roads_out + ((size_t)a * GP_OBS_ROADS + lane) * 8, f);
    }

    // traffic controls
    if (p.signals_out) {
        NearestK sel(GP_OBS_SIGNALS, stage[wb]);
        for (int base = 0; base < wi.n_sig; base += 32) {
            const int s = base + lane;
            bool ok = false;
            float d = 0.f;
            if (s < wi.n_sig) {
                const float4 q = p.sig[wi.sig_begin + s];
                const float dx = q.x - me.x, dy = q.y - me.y;
                d = sqrtf(dx * dx + dy * dy);
                ok = d <= GP_OBS_SIGNAL_RADIUS;
            }
            sel.offer(ok, make_key(d, (uint32_t)s));
        }
        sel.finish();
        if (lane < GP_OBS_SIGNALS) {
            float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (sel.list != kNone) {
                const int s = (int)(sel.list & 0xFFFFFFFFu);
                const float4 q = p.sig[wi.sig_begin + s];
                const float dx = q.x - me.x, dy = q.y - me.y;
                f[0] = 1.f;
                f[1] = (dx * cs + dy * sn) / GP_OBS_SIGNAL_RADIUS;
                f[2] = (-dx * sn + dy * cs) / GP_OBS_SIGNAL_RADIUS;
                f[3] = q.z / 10.f;
                f[4 + (p.sig_state[wi.sig_begin + s] & 3)] = 1.f;
            }
            store_slot(p.signals_out + ((size_t)a * GP_OBS_SIGNALS + lane) * 8, f);
        }
    }
}

}  // namespace

cudaError_t launch_obs(const ObsParams &p, cudaStream_t s) {
    if (p.n_agents <= 0) return cudaSuccess;
    const int blocks = (p.n_agents + kObsWarps - 1) / kObsWarps;
    obs_kernel<<<blocks, 32 * kObsWarps, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace gpk
