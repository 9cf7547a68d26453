// Internal device-side layout of the batched step-and-render library.  Host runtime
// (gp_api.cu) builds these arrays once at create time; the step and render kernels read
// them.  Nothing here is shared with the CPU oracle.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gigapixel.h"

namespace gpk {

constexpr int kMaxBoxes = GP_MAX_BOXES;
constexpr int kClusterQuads = 32;  // quads per culling cluster = one quad per lane of a warp
constexpr int kMaxClustersPerWorld = 4096;
constexpr int kMaxBandRows = 128;  // rows per screen band (raster records pack band-relative rows)
constexpr int kMaxSignals = GP_MAX_SIGNALS;
// The ray-tracing kernel (128 threads, four warps) stages one box per thread and compacts
// them with one ballot per warp.
static_assert(kMaxBoxes <= 128, "trace_kernel keeps at most one box per thread");
constexpr int kSignalQuads = 32;   // faces of a signal polyhedron = one setup unit

// Per-world table (device).
struct WorldInfo {
    int box_begin, n_boxes;      // global box range; the first n_agents are agents
    int agent_begin, n_agents;   // global agent range
    int cl_begin, n_cl;          // culling clusters
    int road_begin, n_road;      // road quads in original order (off-road test)
    int line_begin, n_line;      // lane-line quads in original order (ray tracing)
    int cell_begin;              // off-road grid: cells [cell_begin, cell_begin + gnx*gny)
    int lcell_begin;             // a finer grid over lane-line quads (same origin)
    int lgnx, lgny;
    float lginv;
    int rcell_begin;             // a finer grid over road quads for the ray tracer (same origin)
    int rgnx, rgny;
    float rginv;
    int scell_begin;             // the same grid listing each road/line segment once, in the
                                 // cell of its centre-line midpoint (ids: road r, n_road + line l)
    int gnx, gny;
    float gx0, gy0, ginv;        // grid origin and inverse cell size
    int sig_begin, n_sig;        // traffic-signal spheres
    uint32_t box_end, road_end;  // primitive-id class boundaries: box < box_end <= road < road_end
    uint32_t line_end;           // <= line < line_end <= signal
};

// A culling cluster: up to kClusterQuads ground quads of one grid cell.
struct Cluster {
    float cx, cy, hx, hy;  // xy bounding box (centre, half extents)
    float zlo, zhi;        // z range of the quads
    int q0, nq;            // quads [q0, q0 + nq) of the cluster-ordered quad arrays
};

struct StepParams {
    const WorldInfo *worlds;
    int world_begin, n_worlds;
    float4 *box_pose;       // x, y, yaw, 0 (agents updated in place)
    const float4 *box_dim;  // L, W, H, 0
    float *speed;           // [n_agents]
    uint8_t *flags;         // [n_agents]
    const float2 *actions;  // [n_agents] accel, steer (jerk dynamics: j_lon, j_lat)
    const float4 *road_geo; // 2 per road quad (original order)
    const int *cell_off;    // CSR of road quads per grid cell
    const int *cell_quads;
    float dt, vmax;
    uint32_t *status;
    // per-step reward terms and ego state (only if rewards != 0)
    int rewards;
    float lane_w, vlim;
    float *weights;         // [n_agents][10] (redrawn at episode starts with conditioning)
    float2 *acc;            // [n_agents] previous a_lon, a_lat (updated)
    float *reward;          // [n_agents]
    float *ego;             // [n_agents][GP_EGO_DIM]
    // jerk-actuated dynamics (dynamics == GP_DYN_JERK): actuator state per agent
    int dynamics;
    float *jerk;            // [n_agents][3] a_lon, a_lat, steer (updated)
    // traffic signals for the red-light term: centre, state, controlled road quad (-1: none)
    const float4 *sig;
    const uint8_t *sig_state;
    const int *sig_quad;
    // fixed-length episodes (episode_steps > 0): per-world step counter, initial state
    int episode_steps;
    int *ep_counter;       // [n_worlds]
    const float4 *pose0;   // [n_boxes]
    const float *speed0;   // [n_agents]
    // reward conditioning: coefficients redrawn at every episode start
    int conditioning;
    unsigned long long cond_seed;
    int *ep_index;         // [n_agents] episodes started so far
    float *cond;           // [n_agents][12] normalised coefficients
    int *render_counter;   // non-null: zeroed for the render launch that follows (graphs)
};

// Vectorized observations (gp_observe_vec).
struct ObsParams {
    const WorldInfo *worlds;
    const int *agent_world;
    int n_agents;
    const float4 *box_pose, *box_dim;
    const float *speed;
    const float4 *road_geo, *line_geo;
    const int *seg_off, *seg_list;  // midpoint grid (WorldInfo::scell_begin)
    const float4 *sig;
    const uint8_t *sig_state;
    float *agents_out;   // [n_agents][GP_OBS_AGENTS][8] or null
    float *roads_out;    // [n_agents][GP_OBS_ROADS][8] or null
    float *signals_out;  // [n_agents][GP_OBS_SIGNALS][8] or null
};
cudaError_t launch_obs(const ObsParams &p, cudaStream_t s);

// Snapped triangle as dumped for parity checks (matches gp_debug_dump_tris records).
struct DumpTri {
    int X[3], Y[3];
    float d[3];
    uint32_t prim, sub;
};

struct RenderParams {
    const WorldInfo *worlds;
    const float4 *box_pose;
    const float4 *box_dim;
    const int *agent_world;  // [n_agents]
    const Cluster *clusters;
    const float4 *quad_geo;  // 2 per quad, cluster order
    const uint32_t *quad_prim;
    const int2 *items;       // (view, band)
    int item_begin, n_items;
    int *work_counter;       // persistent mode if non-null, else one item per block

    int W, H, n_cams, band_rows;
    float cam_yaw[GP_MAX_CAMS];
    float f;                 // focal length, px
    float near_plane, cam_h, line_z;
    float tx, ty;            // viewport half-extent / f
    float guard;             // guard band factor

    int key_f16, out_mode;
    float light[3], ambient;  // RGB output: unit direction towards the light, ambient term
    float colour[4][3];       // RGB output: class colours in [0, 1]
    float sig_colour[4][3];   // RGB output: signal colours by state
    const float4 *sig;        // signal spheres: x, y, z, r
    const uint8_t *sig_state; // their states
    int has_signals;          // some world of the batch has signal spheres
    void *out;
    void *depth;
    int view_mod;            // 0, or write view v at slot v % view_mod (tuning scratch)
    uint16_t onehot[4][2];   // bf16 values per channel: [cold, hot]

    // ray tracing: ground quads in original order and their per-world grids
    const float4 *road_geo, *line_geo;
    const int *cell_off, *cell_quads, *lcell_off, *lcell_quads, *rcell_off, *rcell_quads;
    int trace_view0;         // first view of a ray-tracing launch

    int tri_cap;             // triangles per raster batch
    int max_cl;              // most culling clusters in any world of the batch
    int prod_warps;          // > 0: pipelined kernel with this many producer warps
    unsigned long long wait_ns;  // pipelined kernel: a handoff wait gives up after this long
    int debug_stall;         // pipelined kernel: producers publish nothing (timeout test)
    uint32_t *status;

    unsigned long long *stats;  // GP_STAT_* counters, or null (off)
    int dump_view;           // -1 = off
    DumpTri *dump;
    int *dump_count;
    int dump_cap;
};

// Shared-memory bytes the render kernel needs for a launch shape (max_cl: most culling
// clusters in any world of the batch).
size_t render_smem_bytes(int W, int band_rows, int key_f16, int threads, int tri_cap, int max_cl,
                         int prod_warps);

cudaError_t launch_step(const StepParams &p, int max_blocks, cudaStream_t s);

// Episode reset of selected worlds (gp_reset_worlds).
struct ResetParams {
    int n_agents, n_worlds;
    int draw_only;        // 1: draw the current episode's conditioning, change nothing else
    int *ep_counter;      // [n_worlds] episode step counters (zeroed for reset worlds)
    const WorldInfo *worlds;
    int conditioning;
    unsigned long long cond_seed;
    int *ep_index;        // [n_agents]
    float *weights;       // [n_agents][10]
    float *cond;          // [n_agents][12]
    const uint8_t *mask;  // [n_worlds] or null = all
    const int *agent_world, *agent_box;
    const float4 *pose0;  // initial box poses
    const float *speed0;  // initial agent speeds
    float4 *pose;
    float *speed;
    uint8_t *flags;
    float2 *acc;
    float *jerk;
};
cudaError_t launch_reset(const ResetParams &p, cudaStream_t s);
cudaError_t launch_state(float *state, uint8_t *flags, float4 *pose, float *speed, uint8_t *fl,
                         const int *agent_box, int n, int to_state, cudaStream_t s);
cudaError_t launch_render(const RenderParams &p, int blocks, int threads, size_t smem,
                          cudaStream_t s);
cudaError_t render_configure(size_t max_smem);
int render_occupancy(int key_f16, int threads, size_t smem, int prod_warps);
// Ray-traced views [0, n_views) in the render output formats (grid rows of 65535 views).
cudaError_t launch_trace(const RenderParams &p, int n_views, cudaStream_t s);

}  // namespace gpk
