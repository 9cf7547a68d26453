// Host runtime and C ABI (include/gigapixel.h): validation, device world layout, launch
// shapes, CUDA-graph replay, autotuning, state/status/debug calls.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gp_internal.h"

using namespace gpk;

namespace {

// Cell size (m) of the ray tracer's road grid (A/B on the uniform batch, outputs identical:
// 8 m 2.135 ms, 4 m 1.994 ms, 2 m 1.927 ms per trace launch).
constexpr float kTraceRoadCell = 2.f;

// NVTX range over a public call (visible in a timeline tool; free when none is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

thread_local std::string g_err;

gp_status fail(gp_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(GP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
    } while (0)

template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    cudaError_t alloc(size_t count) {
        n = count;
        if (count == 0) return cudaSuccess;
        return cudaMalloc(&p, sizeof(T) * count);
    }
    cudaError_t upload(const std::vector<T> &v) {
        cudaError_t e = alloc(v.size());
        if (e != cudaSuccess || v.empty()) return e;
        return cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

struct Shape {
    int threads = 512, band_rows = 32, tri_cap = 512, blocks = 0, prod_warps = 0;
    size_t smem = 0;
};

struct GraphKey {
    const void *a, *o, *d;
    int backend;  // 0: step + raster, 1: step + ray tracing
    bool operator<(const GraphKey &k) const {
        if (backend != k.backend) return backend < k.backend;
        if (a != k.a) return a < k.a;
        if (o != k.o) return o < k.o;
        return d < k.d;
    }
};

}  // namespace

struct gp_handle {
    int device = 0, sms = 148;
    gp_config cfg{};
    int n_worlds = 0, n_agents = 0, n_boxes = 0, n_views = 0, n_signals = 0;
    int max_cl = 1;  // most culling clusters in one world
    std::vector<WorldInfo> worlds_h;
    std::vector<int> world_item_begin, world_item_count;
    DevBuf<WorldInfo> worlds;
    DevBuf<float4> box_pose, box_dim, quad_geo, road_geo, line_geo, sig;
    DevBuf<uint8_t> sig_state;
    DevBuf<int> sig_quad;
    DevBuf<unsigned long long> stats;  // GP_STAT_* counters (gp_config.stats)
    DevBuf<int> ep_counter;            // per-world episode step counter
    DevBuf<int> ep_index;              // per-agent episodes started (conditioning draws)
    DevBuf<float> cond;                // per-agent conditioning vector [n_agents][12]  // road quad (road_geo index) each signal controls, -1 if none
    DevBuf<float> speed, speed0;
    DevBuf<float4> pose0;  // initial poses and speeds (gp_reset_worlds)
    DevBuf<uint8_t> flags;
    DevBuf<int> agent_world, agent_box, cell_off, cell_quads, lcell_off, lcell_quads, rcell_off,
        rcell_quads, seg_off,
        seg_list, counter, dump_count;
    DevBuf<Cluster> clusters;
    DevBuf<uint32_t> quad_prim, status;
    DevBuf<int2> items;
    DevBuf<DumpTri> dump;
    DevBuf<float> state_stage;
    DevBuf<float> reward, ego, weights;  // per-step rewards: [n_agents], [n_agents][GP_EGO_DIM], [n_agents][10]
    DevBuf<float> jerk;                  // jerk dynamics' actuator state [n_agents][3]
    DevBuf<float2> acc;                  // previous-step accelerations
    DevBuf<float2> act_stage;            // actions copied in by gp_step_render_host
    DevBuf<uint8_t> flag_stage, world_stage;  // host-copy staging: per agent, per world
    Shape shape;
    uint16_t onehot[4][2];
    cudaStream_t capture_stream = nullptr;
    std::map<GraphKey, cudaGraphExec_t> graphs;
    bool sticky = false;
};

namespace {

bool finite_all(const float *p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

gp_status validate(const gp_world_desc *d, const gp_config *c) {
    if (!d || !c) return fail(GP_EINVAL, "null descriptor or config");
    if (d->n_worlds <= 0) return fail(GP_EINVAL, "n_worlds must be positive");
    if (!d->box_off || !d->agent_count || !d->road_off || !d->line_off)
        return fail(GP_EINVAL, "null CSR array");
    if (c->width < 16 || c->height < 16 || c->width > GP_MAX_WIDTH || c->height > GP_MAX_WIDTH)
        return fail(GP_ELIMIT, "image size must be within 16..512");
    if (c->width % 2 || c->height % 2) return fail(GP_EINVAL, "image width and height must be even");
    if (c->n_cams < 1 || c->n_cams > GP_MAX_CAMS) return fail(GP_ELIMIT, "n_cams must be 1..8");
    if (!(c->hfov > 0.01f && c->hfov < 3.0f)) return fail(GP_EINVAL, "hfov out of range");
    if (!(c->near_plane > 0.f) || !(c->cam_height > 0.f) || !(c->dt > 0.f) || !(c->v_max >= 0.f))
        return fail(GP_EINVAL, "near_plane, cam_height, dt must be positive, v_max >= 0");
    if (c->key_precision != GP_KEY_F32 && c->key_precision != GP_KEY_F16)
        return fail(GP_EINVAL, "key_precision");
    if (c->output != GP_OUT_CLASS_U8 && c->output != GP_OUT_ONEHOT_BF16 && c->output != GP_OUT_RGB_U8)
        return fail(GP_EINVAL, "output");
    if (c->rewards != 0 && c->rewards != 1) return fail(GP_EINVAL, "rewards must be 0 or 1");
    if (c->stats != 0 && c->stats != 1) return fail(GP_EINVAL, "stats must be 0 or 1");
    if (c->episode_steps < 0) return fail(GP_EINVAL, "episode_steps must be >= 0");
    if (c->reward_conditioning != 0 && c->reward_conditioning != 1)
        return fail(GP_EINVAL, "reward_conditioning must be 0 or 1");
    if (c->dynamics != GP_DYN_DIRECT && c->dynamics != GP_DYN_JERK)
        return fail(GP_EINVAL, "dynamics must be GP_DYN_DIRECT or GP_DYN_JERK");
    if (c->rewards && !(c->lane_width > 0.f && c->v_limit >= 0.f))
        return fail(GP_EINVAL, "lane_width must be positive, v_limit >= 0");
    if (c->output == GP_OUT_RGB_U8) {
        const double l2 = (double)c->light_dir[0] * c->light_dir[0] +
                          (double)c->light_dir[1] * c->light_dir[1] +
                          (double)c->light_dir[2] * c->light_dir[2];
        if (!(l2 > 1e-12) || !finite_all(c->light_dir, 3) || !(c->ambient >= 0.f && c->ambient <= 1.f) ||
            !finite_all(&c->colour[0][0], 12) || !finite_all(&c->signal_colour[0][0], 12))
            return fail(GP_EINVAL, "RGB appearance: light_dir non-zero, ambient in 0..1, finite colours");
    }
    if (c->threads < 0 || c->threads > 1024 || c->threads % 32 || c->band_rows < 0 ||
        c->tri_capacity < 0 || c->tri_capacity > 4096)
        return fail(GP_EINVAL, "threads (multiple of 32, <= 1024), band_rows, tri_capacity");
    for (int k = 0; k < 4; ++k)
        if (!(c->norm_std[k] != 0.f) || !std::isfinite(c->norm_mean[k]) || !std::isfinite(c->norm_std[k]))
            return fail(GP_EINVAL, "norm_mean/norm_std");
    for (int k = 0; k < c->n_cams; ++k)
        if (!std::isfinite(c->cam_yaw[k])) return fail(GP_EINVAL, "cam_yaw");
    const int nw = d->n_worlds;
    if (d->box_off[0] != 0 || d->road_off[0] != 0 || d->line_off[0] != 0)
        return fail(GP_EINVAL, "CSR offsets must start at 0");
    for (int w = 0; w < nw; ++w) {
        const int nb = d->box_off[w + 1] - d->box_off[w];
        const int na = d->agent_count[w];
        const int nr = d->road_off[w + 1] - d->road_off[w];
        const int nl = d->line_off[w + 1] - d->line_off[w];
        if (nb < 0 || nr < 0 || nl < 0) return fail(GP_EINVAL, "CSR offsets must be non-decreasing");
        if (na < 0 || na > nb) return fail(GP_EINVAL, "agent_count must be in [0, boxes]");
        if (nb > GP_MAX_BOXES) return fail(GP_ELIMIT, "more than 128 boxes in a world");
        if (nr + nl > GP_MAX_QUADS) return fail(GP_ELIMIT, "more than 32767 quads in a world");
        const int ns = d->signal_off ? d->signal_off[w + 1] - d->signal_off[w] : 0;
        if (ns < 0) return fail(GP_EINVAL, "CSR offsets must be non-decreasing");
        if (ns > GP_MAX_SIGNALS) return fail(GP_ELIMIT, "more than 32 signals in a world");
        const long long prims = 12LL * nb + 2LL * (nr + nl) + 64LL * ns;
        if (c->key_precision == GP_KEY_F16 && prims > 65535)
            return fail(GP_ELIMIT, "FP16 keys hold at most 65535 primitive ids per world");
    }
    const size_t nb = d->box_off[nw], nr = d->road_off[nw], nl = d->line_off[nw];
    if ((nb && !d->boxes) || (nr && !d->road) || (nl && !d->line))
        return fail(GP_EINVAL, "null geometry array");
    // ground-quad codes of the render kernel keep bits 30..31 free
    if (nr + nl >= (size_t)1 << 29) return fail(GP_ELIMIT, "more than 2^29 quads in the batch");
    if (d->signal_off) {
        if (d->signal_off[0] != 0) return fail(GP_EINVAL, "CSR offsets must start at 0");
        const size_t ns = d->signal_off[nw];
        if (ns && !d->signal) return fail(GP_EINVAL, "null geometry array");
        if (!finite_all(d->signal, ns * 4)) return fail(GP_EINVAL, "non-finite geometry");
        for (size_t s = 0; s < ns; ++s) {
            if (!(d->signal[4 * s + 3] > 0.f)) return fail(GP_EINVAL, "signal radius must be positive");
            if (d->signal_state && d->signal_state[s] > GP_SIGNAL_OFF)
                return fail(GP_EINVAL, "signal state must be 0..3");
        }
    }
    if (!finite_all(d->boxes, nb * 7) || !finite_all(d->road, nr * 8) || !finite_all(d->line, nl * 8))
        return fail(GP_EINVAL, "non-finite geometry");
    for (size_t b = 0; b < nb; ++b)
        if (!(d->boxes[7 * b + 3] > 0.f && d->boxes[7 * b + 4] > 0.f && d->boxes[7 * b + 5] > 0.f))
            return fail(GP_EINVAL, "box dimensions must be positive");
    return GP_OK;
}

uint16_t bf16_bits(float x) {
    __nv_bfloat16 b = __float2bfloat16_rn(x);
    uint16_t u;
    std::memcpy(&u, &b, 2);
    return u;
}

size_t smem_limit(int device) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    return (size_t)v;
}

// Complete a launch shape: shared memory and resident blocks (0 blocks = does not fit).
bool finish_shape(gp_handle *h, Shape &s) {
    const gp_config &c = h->cfg;
    if (s.band_rows > c.height) s.band_rows = c.height;
    if (s.band_rows < 1 || s.band_rows > kMaxBandRows) return false;
    // 4-pixel vector stores: every band must hold a multiple of 4 pixels
    if (c.width % 4 && s.band_rows % 2) return false;
    if (s.threads < 32 || s.threads > 1024 || s.threads % 32) return false;
    // a setup unit needs at most 32 batch slots; a clip job needs 6
    if (s.tri_cap < 64) return false;
    // the pipelined kernel needs at least one producer and one consumer warp
    if (s.prod_warps < 0 || (s.prod_warps > 0 && s.prod_warps >= s.threads / 32)) return false;
    s.smem = render_smem_bytes(c.width, s.band_rows, c.key_precision, s.threads, s.tri_cap,
                               h->max_cl, s.prod_warps);
    if (s.smem + 1024 > smem_limit(h->device)) return false;  // leave room for static smem
    const int per_sm = render_occupancy(c.key_precision, s.threads, s.smem, s.prod_warps);
    if (per_sm < 1) return false;
    s.blocks = per_sm * h->sms;
    return true;
}

Shape default_shape(gp_handle *h) {
    const gp_config &c = h->cfg;
    Shape best;
    const int rows_opts[] = {128, 64, 48, 32, 16, 8};
    for (int r : rows_opts) {
        Shape s;
        s.threads = c.threads ? c.threads : 256;
        s.tri_cap = c.tri_capacity ? c.tri_capacity : std::max(1024, 2 * s.threads);
        s.prod_warps = c.producer_warps > 0 ? c.producer_warps : 0;
        s.band_rows = c.band_rows ? c.band_rows : r;
        if (!finish_shape(h, s)) {
            if (c.band_rows) break;
            continue;
        }
        // prefer >= 2 resident blocks per SM, then the tallest band
        if (best.blocks == 0 || (s.blocks >= 2 * h->sms && best.blocks < 2 * h->sms)) best = s;
        if (c.band_rows) break;
        if (best.blocks >= 2 * h->sms) break;
    }
    return best;
}

RenderParams render_params(gp_handle *h, void *out, void *depth) {
    RenderParams p{};
    const gp_config &c = h->cfg;
    p.worlds = h->worlds.p;
    p.box_pose = h->box_pose.p;
    p.box_dim = h->box_dim.p;
    p.agent_world = h->agent_world.p;
    p.clusters = h->clusters.p;
    p.quad_geo = h->quad_geo.p;
    p.quad_prim = h->quad_prim.p;
    p.items = h->items.p;
    p.item_begin = 0;
    p.n_items = (int)h->items.n;
    p.work_counter = h->counter.p;
    p.W = c.width;
    p.H = c.height;
    p.n_cams = c.n_cams;
    p.band_rows = h->shape.band_rows;
    for (int k = 0; k < GP_MAX_CAMS; ++k) p.cam_yaw[k] = c.cam_yaw[k];
    const double f = 0.5 * c.width / std::tan(0.5 * (double)c.hfov);
    p.f = (float)f;
    p.near_plane = c.near_plane;
    p.cam_h = c.cam_height;
    p.line_z = c.lane_line_z;
    p.tx = (float)(0.5 * c.width / f);
    p.ty = (float)(0.5 * c.height / f);
    p.guard = 4.0f;
    p.key_f16 = c.key_precision;
    p.out_mode = c.output;
    {
        const double l0 = c.light_dir[0], l1 = c.light_dir[1], l2 = c.light_dir[2];
        const double n = std::sqrt(l0 * l0 + l1 * l1 + l2 * l2);
        p.light[0] = n > 0 ? (float)(l0 / n) : 0.f;
        p.light[1] = n > 0 ? (float)(l1 / n) : 0.f;
        p.light[2] = n > 0 ? (float)(l2 / n) : 1.f;
        p.ambient = c.ambient;
        std::memcpy(p.colour, c.colour, sizeof(p.colour));
        std::memcpy(p.sig_colour, c.signal_colour, sizeof(p.sig_colour));
    }
    p.sig = h->sig.p;
    p.sig_state = h->sig_state.p;
    p.has_signals = h->n_signals > 0;
    p.out = out;
    p.depth = depth;
    p.view_mod = 0;
    std::memcpy(p.onehot, h->onehot, sizeof(p.onehot));
    p.tri_cap = h->shape.tri_cap;
    p.max_cl = h->max_cl;
    p.prod_warps = h->shape.prod_warps;
    p.road_geo = h->road_geo.p;
    p.line_geo = h->line_geo.p;
    p.cell_off = h->cell_off.p;
    p.cell_quads = h->cell_quads.p;
    p.lcell_off = h->lcell_off.p;
    p.lcell_quads = h->lcell_quads.p;
    p.rcell_off = h->rcell_off.p;
    p.rcell_quads = h->rcell_quads.p;
    p.trace_view0 = 0;
    p.wait_ns = 2000000000ull;  // 2 s: far beyond any legitimate handoff
    p.debug_stall = 0;
    p.status = h->status.p;
    p.stats = h->cfg.stats ? h->stats.p : nullptr;
    p.dump_view = -1;
    return p;
}

StepParams step_params(gp_handle *h, const float *actions) {
    StepParams p{};
    p.worlds = h->worlds.p;
    p.world_begin = 0;
    p.n_worlds = h->n_worlds;
    p.box_pose = h->box_pose.p;
    p.box_dim = h->box_dim.p;
    p.speed = h->speed.p;
    p.flags = h->flags.p;
    p.actions = (const float2 *)actions;
    p.road_geo = h->road_geo.p;
    p.cell_off = h->cell_off.p;
    p.cell_quads = h->cell_quads.p;
    p.dt = h->cfg.dt;
    p.vmax = h->cfg.v_max;
    p.status = h->status.p;
    p.rewards = h->cfg.rewards;
    p.lane_w = h->cfg.lane_width;
    p.vlim = h->cfg.v_limit;
    p.weights = h->weights.p;
    p.acc = h->acc.p;
    p.reward = h->reward.p;
    p.ego = h->ego.p;
    p.dynamics = h->cfg.dynamics;
    p.jerk = h->jerk.p;
    p.sig = h->sig.p;
    p.sig_state = h->sig_state.p;
    p.sig_quad = h->sig_quad.p;
    p.episode_steps = h->cfg.episode_steps;
    p.ep_counter = h->ep_counter.p;
    p.conditioning = h->cfg.reward_conditioning;
    p.cond_seed = h->cfg.conditioning_seed;
    p.ep_index = h->ep_index.p;
    p.cond = h->cond.p;
    p.pose0 = h->pose0.p;
    p.speed0 = h->speed0.p;
    return p;
}

ResetParams reset_params(gp_handle *h) {
    ResetParams p{};
    p.n_agents = h->n_agents;
    p.n_worlds = h->n_worlds;
    p.ep_counter = h->ep_counter.p;
    p.worlds = h->worlds.p;
    p.conditioning = h->cfg.reward_conditioning;
    p.cond_seed = h->cfg.conditioning_seed;
    p.ep_index = h->ep_index.p;
    p.weights = h->weights.p;
    p.cond = h->cond.p;
    p.mask = nullptr;
    p.agent_world = h->agent_world.p;
    p.agent_box = h->agent_box.p;
    p.pose0 = h->pose0.p;
    p.speed0 = h->speed0.p;
    p.pose = h->box_pose.p;
    p.speed = h->speed.p;
    p.flags = h->flags.p;
    p.acc = h->acc.p;
    p.jerk = h->jerk.p;
    return p;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

gp_status check_out(void *out, void *depth) {
    if (!out) return fail(GP_EINVAL, "out_dev is null");
    if (!aligned16(out) || (depth && !aligned16(depth)))
        return fail(GP_EINVAL, "output pointers must be 16-byte aligned");
    return GP_OK;
}

// Can kernels on the handle's GPU address p?  Device memory of that GPU, managed memory and
// mapped pinned host memory qualify; pageable host memory and another GPU's memory do not
// (a kernel touching them would fault), so they are refused before any launch.  Null passes.
gp_status check_reach(const gp_handle *h, const void *p, const char *what) {
    if (!p) return GP_OK;
    cudaPointerAttributes a{};
    const cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(GP_EINVAL, std::string(what) + ": not a CUDA-addressable pointer (" +
                                   cudaGetErrorString(e) + ")");
    }
    if (a.type == cudaMemoryTypeUnregistered)
        return fail(GP_EINVAL, std::string(what) + " is pageable host memory");
    if (a.type == cudaMemoryTypeDevice && a.device != h->device)
        return fail(GP_EINVAL, std::string(what) + " is on another GPU");
    if (a.type == cudaMemoryTypeHost && !a.devicePointer)
        return fail(GP_EINVAL, std::string(what) + " is pinned host memory without a device mapping");
    return GP_OK;
}

// Is p page-locked host memory (so that a copy from or to it is asynchronous)?  Null passes.
gp_status check_pinned(const void *p, const char *what) {
    if (!p) return GP_OK;
    cudaPointerAttributes a{};
    const cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(GP_EINVAL, std::string(what) + ": not a pointer CUDA knows (" +
                                   cudaGetErrorString(e) + ")");
    }
    if (a.type != cudaMemoryTypeHost)
        return fail(GP_EINVAL, std::string(what) + " must be pinned (page-locked) host memory");
    return GP_OK;
}

gp_status check_reach(const gp_handle *h, const void *actions, const void *out,
                      const void *depth) {
    gp_status st = check_reach(h, actions, "actions_dev");
    if (st == GP_OK) st = check_reach(h, out, "out_dev");
    if (st == GP_OK) st = check_reach(h, depth, "depth_dev");
    return st;
}

cudaError_t enqueue_render(gp_handle *h, const RenderParams &p, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(h->counter.p, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    return launch_render(p, h->shape.blocks, h->shape.threads, h->shape.smem, s);
}

// Work items: worlds in decreasing cost order (ragged batches start with the heaviest
// worlds), every view of a world together, every band of a view together.
void build_items(gp_handle *h, int band_rows, std::vector<int2> &items) {
    const gp_config &c = h->cfg;
    const int nb = (c.height + band_rows - 1) / band_rows;
    std::vector<int> order(h->n_worlds);
    for (int w = 0; w < h->n_worlds; ++w) order[w] = w;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const WorldInfo &A = h->worlds_h[a], &B = h->worlds_h[b];
        return (long long)A.n_cl * 16 + A.n_boxes + 5 * A.n_sig >
               (long long)B.n_cl * 16 + B.n_boxes + 5 * B.n_sig;
    });
    items.clear();
    items.reserve((size_t)h->n_views * nb);
    h->world_item_begin.assign(h->n_worlds, 0);
    h->world_item_count.assign(h->n_worlds, 0);
    for (int w : order) {
        const WorldInfo &wi = h->worlds_h[w];
        h->world_item_begin[w] = (int)items.size();
        for (int a = 0; a < wi.n_agents; ++a)
            for (int cam = 0; cam < c.n_cams; ++cam)
                for (int b = 0; b < nb; ++b)
                    items.push_back(make_int2((wi.agent_begin + a) * c.n_cams + cam, b));
        h->world_item_count[w] = (int)items.size() - h->world_item_begin[w];
    }
}

std::string cache_key(gp_handle *h) {
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, h->device);
    const gp_config &c = h->cfg;
    long long quads = 0;
    for (auto &w : h->worlds_h) quads += w.n_cl;
    std::ostringstream k;
    k << prop.name << "|" << c.width << "x" << c.height << "|cams" << c.n_cams << "|key"
      << c.key_precision << "|out" << c.output << "|views" << h->n_views << "|clusters" << quads;
    return k.str();
}

// Flat JSON object of "key": "threads,band_rows,tri_cap,producer_warps" strings.
std::map<std::string, std::string> read_cache(const char *path) {
    std::map<std::string, std::string> m;
    std::ifstream f(path);
    if (!f) return m;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string s = ss.str();
    size_t i = 0;
    while (true) {
        const size_t a = s.find('"', i);
        if (a == std::string::npos) break;
        const size_t b = s.find('"', a + 1);
        if (b == std::string::npos) break;
        const size_t c = s.find('"', b + 1);
        if (c == std::string::npos) break;
        const size_t d = s.find('"', c + 1);
        if (d == std::string::npos) break;
        m[s.substr(a + 1, b - a - 1)] = s.substr(c + 1, d - c - 1);
        i = d + 1;
    }
    return m;
}

void write_cache(const char *path, const std::map<std::string, std::string> &m) {
    std::ofstream f(path);
    f << "{\n";
    size_t i = 0;
    for (auto &kv : m)
        f << "  \"" << kv.first << "\": \"" << kv.second << "\"" << (++i < m.size() ? ",\n" : "\n");
    f << "}\n";
}

// Time candidate launch shapes on the real worlds (render only, into a scratch output of
// at most 1 GiB that views share round-robin).  The best shape is cached in the JSON file
// named by GP_AUTOTUNE_CACHE, if set.
gp_status autotune(gp_handle *h) {
    const char *cache_path = std::getenv("GP_AUTOTUNE_CACHE");
    const std::string key = cache_key(h);
    if (cache_path) {
        auto m = read_cache(cache_path);
        auto it = m.find(key);
        if (it != m.end()) {
            Shape s;
            const int got = std::sscanf(it->second.c_str(), "%d,%d,%d,%d", &s.threads,
                                        &s.band_rows, &s.tri_cap, &s.prod_warps);
            if ((got == 3 || got == 4) && finish_shape(h, s)) {
                h->shape = s;
                return GP_OK;
            }
        }
    }
    const gp_config &c = h->cfg;
    const size_t px = (size_t)c.width * c.height;
    const size_t out_pv = px * (c.output == GP_OUT_CLASS_U8 ? 1 : (c.output == GP_OUT_RGB_U8 ? 3 : 8));
    const size_t dep_pv = px * (c.key_precision == GP_KEY_F32 ? 4 : 2);
    size_t views = std::min<size_t>((size_t)h->n_views, ((size_t)1 << 30) / (out_pv + dep_pv));
    views = std::max<size_t>(views, 1);
    uint8_t *scratch = nullptr;
    const size_t out_bytes = (views * out_pv + 255) / 256 * 256;
    CK(cudaMalloc(&scratch, out_bytes + views * dep_pv));
    uint8_t *depth = scratch + out_bytes;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    Shape best;
    float best_ms = 1e30f;
    const Shape saved = h->shape;
    const int thr[] = {256, 512, 1024};
    const int caps[] = {512, 768, 1024, 1536, 2048};
    const int rows[] = {8, 16, 32, 48, 64, 128};
    for (int t : thr)
        for (int cap : caps)
            for (int r : rows)
                for (int pk = 0; pk < 3; ++pk) {
                // producer warps: the configured count, else none, a quarter or three
                // eighths of the block's warps
                int pw;
                if (c.producer_warps > 0) {
                    if (pk > 0) continue;
                    pw = c.producer_warps;
                } else {
                    pw = pk == 0 ? 0 : (pk == 1 ? t / 128 : 3 * t / 256);
                    if (c.producer_warps < 0 && pw > 0) continue;
                }
                if (r > c.height && r != rows[0]) continue;
                Shape s;
                s.threads = t;
                s.tri_cap = cap;
                s.band_rows = r;
                s.prod_warps = pw;
                if (!finish_shape(h, s)) continue;
                std::vector<int2> items;
                build_items(h, s.band_rows, items);
                DevBuf<int2> ditems;
                if (ditems.upload(items) != cudaSuccess) continue;
                h->shape = s;
                RenderParams p = render_params(h, scratch, depth);
                p.items = ditems.p;
                p.n_items = (int)items.size();
                p.view_mod = (int)views;
                float ms = 1e30f;
                bool ok = true;
                for (int rep = 0; rep < 3 && ok; ++rep) {
                    cudaEventRecord(e0, 0);
                    ok = enqueue_render(h, p, 0) == cudaSuccess;
                    cudaEventRecord(e1, 0);
                    ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
                    float t_ms = 0;
                    cudaEventElapsedTime(&t_ms, e0, e1);
                    if (rep > 0) ms = std::min(ms, t_ms);
                }
                ditems.release();
                h->shape = saved;
                if (!ok) continue;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = s;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(scratch);
    if (best.blocks == 0) return fail(GP_ECUDA, "autotune found no launch shape");
    h->shape = best;
    if (cache_path) {
        auto m = read_cache(cache_path);
        char buf[64];
        std::snprintf(buf, sizeof buf, "%d,%d,%d,%d", best.threads, best.band_rows, best.tri_cap,
                      best.prod_warps);
        m[key] = buf;
        write_cache(cache_path, m);
    }
    return GP_OK;
}

void release_all(gp_handle *h) {
    for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    h->capture_stream = nullptr;
    h->worlds.release();
    h->box_pose.release();
    h->box_dim.release();
    h->quad_geo.release();
    h->road_geo.release();
    h->speed.release();
    h->speed0.release();
    h->pose0.release();
    h->reward.release();
    h->ego.release();
    h->weights.release();
    h->acc.release();
    h->jerk.release();
    h->sig.release();
    h->sig_state.release();
    h->sig_quad.release();
    h->stats.release();
    h->ep_counter.release();
    h->ep_index.release();
    h->cond.release();
    h->flags.release();
    h->agent_world.release();
    h->agent_box.release();
    h->cell_off.release();
    h->cell_quads.release();
    h->line_geo.release();
    h->lcell_off.release();
    h->lcell_quads.release();
    h->rcell_off.release();
    h->rcell_quads.release();
    h->seg_off.release();
    h->seg_list.release();
    h->counter.release();
    h->dump_count.release();
    h->clusters.release();
    h->quad_prim.release();
    h->status.release();
    h->items.release();
    h->dump.release();
    h->state_stage.release();
    h->flag_stage.release();
    h->act_stage.release();
    h->world_stage.release();
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Scratch of the triangle dump that allocates nothing (gp_debug_dump_tris_noalloc).
// ---------------------------------------------------------------------------------------

// Fixed scratch of the allocation-free dump: bytes [0, 4) work counter, [4, 8) record
// count, records from byte 256.  One copy per device, alive until the process exits.
static __device__ __align__(256) unsigned char gp_noalloc_scratch[256 + GP_NOALLOC_MAX_TRIS * sizeof(DumpTri)];

namespace {

constexpr int kNoAllocDevices = 64;
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_addr[kNoAllocDevices] = {};

// Set-up, with `device` current: look up the device address of the scratch array (the
// host-side name of the array is not a device address; the lookup allocates nothing).
// Done by gp_create_worlds for its device, and again at every later creation on that
// device, so the address is that of the context the live handles were created in (a
// cudaDeviceReset ends that context and every handle made before it).
gp_status noalloc_setup(int device) {
    if (device < 0 || device >= kNoAllocDevices) return GP_OK;  // no allocation-free dump there
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, gp_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return fail(GP_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    g_noalloc_addr[device] = (unsigned char *)p;
    return GP_OK;
}

// The address found by the last set-up on `device`, or null.
unsigned char *noalloc_scratch(int device) {
    if (device < 0 || device >= kNoAllocDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    return g_noalloc_addr[device];
}

}  // namespace

extern "C" {

const char *gp_last_error(void) { return g_err.c_str(); }

gp_status gp_default_config(gp_config *c) {
    if (!c) return fail(GP_EINVAL, "null config");
    std::memset(c, 0, sizeof *c);
    c->width = 128;
    c->height = 128;
    c->n_cams = 1;
    c->hfov = 1.5707963267948966f;
    c->cam_height = 1.5f;
    c->near_plane = 0.1f;
    c->lane_line_z = 0.02f;
    c->dt = 0.1f;
    c->v_max = 30.f;
    c->key_precision = GP_KEY_F32;
    c->output = GP_OUT_CLASS_U8;
    c->light_dir[0] = 0.3f;
    c->light_dir[1] = 0.4f;
    c->light_dir[2] = 0.866f;
    c->ambient = 0.35f;
    c->rewards = 0;
    c->lane_width = 3.5f;
    c->v_limit = 30.f;
    c->dynamics = GP_DYN_DIRECT;
    const float col[4][3] = {{0.55f, 0.75f, 0.95f}, {0.33f, 0.33f, 0.35f}, {0.92f, 0.92f, 0.85f},
                             {0.15f, 0.35f, 0.85f}};
    std::memcpy(c->colour, col, sizeof col);
    const float sig[4][3] = {{0.9f, 0.1f, 0.1f}, {0.95f, 0.7f, 0.1f}, {0.1f, 0.8f, 0.3f},
                             {0.25f, 0.25f, 0.25f}};
    std::memcpy(c->signal_colour, sig, sizeof sig);
    for (int k = 0; k < 4; ++k) {
        c->norm_mean[k] = 0.5f;
        c->norm_std[k] = 0.5f;
    }
    return GP_OK;
}

gp_status gp_destroy(gp_handle *h) {
    if (!h) return GP_OK;
    cudaSetDevice(h->device);
    release_all(h);
    delete h;
    return GP_OK;
}

gp_status gp_create_worlds(const gp_world_desc *d, const gp_config *cfg, int device,
                           gp_handle **out) {
    NvtxRange range("gp_create_worlds");
    if (!out) return fail(GP_EINVAL, "null out handle");
    *out = nullptr;
    gp_status st = validate(d, cfg);
    if (st != GP_OK) return st;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(GP_EINVAL, "invalid device");
    CK(cudaSetDevice(device));
    gp_handle *h = new gp_handle();
    h->device = device;
    h->cfg = *cfg;
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, device);
    const int nw = d->n_worlds;
    h->n_worlds = nw;
    const int nbox = d->box_off[nw];

    std::vector<float4> pose(nbox), dim(nbox);
    std::vector<float> speed;
    std::vector<int> agent_world, agent_box;
    for (int b = 0; b < nbox; ++b) {
        const float *s = d->boxes + 7 * (size_t)b;
        pose[b] = make_float4(s[0], s[1], s[2], 0.f);
        dim[b] = make_float4(s[3], s[4], s[5], 0.f);
    }
    std::vector<Cluster> clusters;
    std::vector<float4> quad_geo, road_geo, line_geo;
    std::vector<uint32_t> quad_prim;
    std::vector<int> cell_off(1, 0), cell_quads, lcell_off(1, 0), lcell_quads, rcell_off(1, 0),
        rcell_quads, seg_off(1, 0),
        seg_list;
    // The ground grids of every world (8 m off-road grid, 1 m lane-line grid, the tracer's
    // road grid): queued by the world loop below, built in parallel after it and appended in
    // world order.
    struct GridJob {
        int grid, w;
        const float *quads;
        int n, index_base;
        float ginv;
        int gnx, gny;
        float bx0, by0;
    };
    std::vector<GridJob> grid_jobs;
    // Built in two passes over the quads (count per cell, then fill at the scanned
    // offsets), each cell's list in increasing quad index.
    auto build_cells = [](const float *quads, int n, int index_base, float ginv, int gnx,
                          int gny, float bx0, float by0, std::vector<int> &off,
                          std::vector<int> &list) {
        const double eps = 1e-3, cell = 1.0 / ginv;
        // calls row(r, cy, cx0, cx1) for every row of cells quad r overlaps
        auto visit = [&](auto &&row) {
            for (int r = 0; r < n; ++r) {
                const float *q = quads + 8 * (size_t)r;
                double qy0 = q[1], qy1 = q[1];
                for (int k = 1; k < 4; ++k) {
                    qy0 = std::min(qy0, (double)q[2 * k + 1]);
                    qy1 = std::max(qy1, (double)q[2 * k + 1]);
                }
                const int cy0 = std::max(0, (int)std::floor(((float)(qy0 - eps) - by0) * ginv));
                const int cy1 = std::min(gny - 1, (int)std::floor(((float)(qy1 + eps) - by0) * ginv));
                for (int cy = cy0; cy <= cy1; ++cy) {
                    const double ya = by0 + cy * cell - eps, yb = by0 + (cy + 1) * cell + eps;
                    double xa = INFINITY, xb = -INFINITY;
                    for (int k = 0; k < 4; ++k) {
                        const double x0 = q[2 * k], y0 = q[2 * k + 1];
                        const double x1 = q[(2 * k + 2) % 8], y1 = q[(2 * k + 3) % 8];
                        if (y0 >= ya && y0 <= yb) {
                            xa = std::min(xa, x0);
                            xb = std::max(xb, x0);
                        }
                        for (const double yc : {ya, yb})
                            if ((y0 - yc) * (y1 - yc) < 0.0) {
                                const double x = x0 + (x1 - x0) * (yc - y0) / (y1 - y0);
                                xa = std::min(xa, x);
                                xb = std::max(xb, x);
                            }
                    }
                    if (!(xa <= xb)) continue;  // the quad misses this row's band
                    const int cx0 = std::max(0, (int)std::floor(((float)(xa - eps) - bx0) * ginv));
                    const int cx1 = std::min(gnx - 1, (int)std::floor(((float)(xb + eps) - bx0) * ginv));
                    row(r, cy, cx0, cx1);
                }
            }
        };
        const size_t nc = (size_t)gnx * gny, base = list.size();
        std::vector<int> pos(nc + 1, 0);
        visit([&](int, int cy, int cx0, int cx1) {
            for (int cx = cx0; cx <= cx1; ++cx) ++pos[(size_t)cy * gnx + cx + 1];
        });
        for (size_t c = 0; c < nc; ++c) pos[c + 1] += pos[c];
        list.resize(base + (size_t)pos[nc]);
        for (size_t c = 0; c < nc; ++c) off.push_back((int)(base + (size_t)pos[c + 1]));
        visit([&](int r, int cy, int cx0, int cx1) {
            for (int cx = cx0; cx <= cx1; ++cx)
                list[base + (size_t)pos[(size_t)cy * gnx + cx]++] = index_base + r;
        });
    };
    h->worlds_h.resize(nw);
    for (int w = 0; w < nw; ++w) {
        WorldInfo wi{};
        wi.box_begin = d->box_off[w];
        wi.n_boxes = d->box_off[w + 1] - d->box_off[w];
        wi.agent_begin = (int)agent_world.size();
        wi.n_agents = d->agent_count[w];
        for (int a = 0; a < wi.n_agents; ++a) {
            agent_world.push_back(w);
            agent_box.push_back(wi.box_begin + a);
            speed.push_back(d->boxes[7 * (size_t)(wi.box_begin + a) + 6]);
        }
        const int r0 = d->road_off[w], nr = d->road_off[w + 1] - r0;
        const int l0 = d->line_off[w], nl = d->line_off[w + 1] - l0;
        wi.box_end = 12u * wi.n_boxes;
        wi.road_end = wi.box_end + 2u * nr;
        wi.line_end = wi.road_end + 2u * nl;
        wi.sig_begin = d->signal_off ? d->signal_off[w] : 0;
        wi.n_sig = d->signal_off ? d->signal_off[w + 1] - d->signal_off[w] : 0;
        wi.road_begin = (int)road_geo.size() / 2;
        wi.n_road = nr;
        float bx0 = 1e30f, by0 = 1e30f, bx1 = -1e30f, by1 = -1e30f;
        wi.line_begin = (int)line_geo.size() / 2;
        wi.n_line = nl;
        for (int r = 0; r < nr + nl; ++r) {
            const float *q = r < nr ? d->road + 8 * (size_t)(r0 + r) : d->line + 8 * (size_t)(l0 + r - nr);
            std::vector<float4> &geo = r < nr ? road_geo : line_geo;
            geo.push_back(make_float4(q[0], q[1], q[2], q[3]));
            geo.push_back(make_float4(q[4], q[5], q[6], q[7]));
            for (int k = 0; k < 4; ++k) {
                bx0 = std::min(bx0, q[2 * k]);
                bx1 = std::max(bx1, q[2 * k]);
                by0 = std::min(by0, q[2 * k + 1]);
                by1 = std::max(by1, q[2 * k + 1]);
            }
        }
        // off-road grid: 8 m cells over the bounding box of the road and lane-line quads; a
        // quad is listed in every cell its bounding box touches (widened by 1 mm), so any
        // point inside it finds it.  A second CSR over the same cells lists the lane lines.
        const float cs = 8.f;
        if (nr + nl == 0) {
            bx0 = by0 = 0.f;
            bx1 = by1 = 1.f;
        }
        wi.gx0 = bx0;
        wi.gy0 = by0;
        wi.ginv = 1.f / cs;
        wi.gnx = std::max(1, (int)std::ceil((bx1 - bx0) / cs) + 1);
        wi.gny = std::max(1, (int)std::ceil((by1 - by0) / cs) + 1);
        // A quad is listed in every cell it overlaps, widened by 1 mm: per row of cells, the
        // x-extent of the quad within the row's y-band.  A point that passes the kernels'
        // FP32 containment test lies within rounding (far below 1 mm) of the quad, and their
        // cell index floor((p - origin) * ginv) is monotone in p, so it finds the quad.
        grid_jobs.push_back(GridJob{0, w, d->road + 8 * (size_t)r0, nr, wi.road_begin, wi.ginv,
                                    wi.gnx, wi.gny, bx0, by0});
        // lane-line strips are thin: a finer grid (1 m cells, at most 256 per side) keeps
        // their per-cell lists short for the ray tracer's lookups
        {
            const float lcs = std::max(1.f, std::max(bx1 - bx0, by1 - by0) / 255.f);
            wi.lginv = 1.f / lcs;
            wi.lgnx = std::max(1, (int)std::ceil((bx1 - bx0) / lcs) + 1);
            wi.lgny = std::max(1, (int)std::ceil((by1 - by0) / lcs) + 1);
        }
        grid_jobs.push_back(GridJob{1, w, d->line + 8 * (size_t)l0, nl, wi.line_begin, wi.lginv,
                                    wi.lgnx, wi.lgny, bx0, by0});
        // the road quads again on a finer grid for the ray tracer, whose lookup scans a cell's
        // list up to the first quad holding the point: the overlapping roads of these worlds
        // put about a dozen quads in an 8 m cell (kTraceRoadCell cells, at most 256 a side);
        // the first holding quad in index order is the same on any grid that lists, in index
        // order, every quad overlapping a cell
        {
            const float rcs = std::max(kTraceRoadCell, std::max(bx1 - bx0, by1 - by0) / 255.f);
            wi.rginv = 1.f / rcs;
            wi.rgnx = std::max(1, (int)std::ceil((bx1 - bx0) / rcs) + 1);
            wi.rgny = std::max(1, (int)std::ceil((by1 - by0) / rcs) + 1);
        }
        grid_jobs.push_back(GridJob{2, w, d->road + 8 * (size_t)r0, nr, wi.road_begin, wi.rginv,
                                    wi.rgnx, wi.rgny, bx0, by0});
        // each road/line segment once, in the cell of its centre-line midpoint (the same
        // FP32 expressions as the observation kernel's, so both agree on the cell)
        {
            wi.scell_begin = (int)seg_off.size() - 1;
            std::vector<std::vector<int>> cells((size_t)wi.gnx * wi.gny);
            for (int s = 0; s < nr + nl; ++s) {
                const float *q = s < nr ? d->road + 8 * (size_t)(r0 + s) : d->line + 8 * (size_t)(l0 + s - nr);
                const float ax = 0.5f * (q[0] + q[6]), ay = 0.5f * (q[1] + q[7]);
                const float bx = 0.5f * (q[2] + q[4]), by = 0.5f * (q[3] + q[5]);
                const float mx = 0.5f * (ax + bx), my = 0.5f * (ay + by);
                const int cx = std::min(wi.gnx - 1, std::max(0, (int)std::floor((mx - wi.gx0) * wi.ginv)));
                const int cy = std::min(wi.gny - 1, std::max(0, (int)std::floor((my - wi.gy0) * wi.ginv)));
                cells[(size_t)cy * wi.gnx + cx].push_back(s);
            }
            for (auto &cl : cells) {
                seg_list.insert(seg_list.end(), cl.begin(), cl.end());
                seg_off.push_back((int)seg_list.size());
            }
        }
        // culling clusters: quads bucketed by the 16 m cell of their centroid, chunks of 16
        {
            const float cc = 16.f;
            struct QRef {
                long long key;
                int src;  // index into the combined road + line list
            };
            std::vector<QRef> refs;
            refs.reserve(nr + nl);
            auto quad_ptr = [&](int i) {
                return i < nr ? d->road + 8 * (size_t)(r0 + i) : d->line + 8 * (size_t)(l0 + i - nr);
            };
            for (int i = 0; i < nr + nl; ++i) {
                const float *q = quad_ptr(i);
                const float mx = 0.25f * (q[0] + q[2] + q[4] + q[6]);
                const float my = 0.25f * (q[1] + q[3] + q[5] + q[7]);
                const long long kx = (long long)std::floor(mx / cc) + (1 << 20);
                const long long ky = (long long)std::floor(my / cc) + (1 << 20);
                refs.push_back({ky * (1LL << 22) + kx, i});
            }
            std::stable_sort(refs.begin(), refs.end(),
                             [](const QRef &a, const QRef &b) { return a.key < b.key; });
            wi.cl_begin = (int)clusters.size();
            size_t i = 0;
            while (i < refs.size()) {
                size_t j = i;
                while (j < refs.size() && refs[j].key == refs[i].key && j - i < (size_t)kClusterQuads) ++j;
                Cluster c{};
                float x0 = 1e30f, y0 = 1e30f, x1 = -1e30f, y1 = -1e30f, z0 = 1e30f, z1 = -1e30f;
                c.q0 = (int)quad_prim.size();
                c.nq = (int)(j - i);
                for (size_t k = i; k < j; ++k) {
                    const int src = refs[k].src;
                    const float *q = quad_ptr(src);
                    quad_geo.push_back(make_float4(q[0], q[1], q[2], q[3]));
                    quad_geo.push_back(make_float4(q[4], q[5], q[6], q[7]));
                    const uint32_t prim = src < nr ? wi.box_end + 2u * src : wi.road_end + 2u * (src - nr);
                    quad_prim.push_back(prim);
                    const float z = src < nr ? 0.f : cfg->lane_line_z;
                    for (int t = 0; t < 4; ++t) {
                        x0 = std::min(x0, q[2 * t]);
                        x1 = std::max(x1, q[2 * t]);
                        y0 = std::min(y0, q[2 * t + 1]);
                        y1 = std::max(y1, q[2 * t + 1]);
                    }
                    z0 = std::min(z0, z);
                    z1 = std::max(z1, z);
                }
                // pad the bounds so that FP32 culling stays conservative
                const float pad = 1e-3f + 1e-5f * std::max(std::max(std::fabs(x0), std::fabs(x1)),
                                                           std::max(std::fabs(y0), std::fabs(y1)));
                c.cx = 0.5f * (x0 + x1);
                c.cy = 0.5f * (y0 + y1);
                c.hx = 0.5f * (x1 - x0) + pad;
                c.hy = 0.5f * (y1 - y0) + pad;
                c.zlo = z0 - 1e-4f;
                c.zhi = z1 + 1e-4f;
                clusters.push_back(c);
                i = j;
            }
            wi.n_cl = (int)clusters.size() - wi.cl_begin;
            h->max_cl = std::max(h->max_cl, wi.n_cl);
            if (wi.n_cl > kMaxClustersPerWorld) {
                delete h;
                return fail(GP_ELIMIT, "too many culling clusters in a world");
            }
        }
        h->worlds_h[w] = wi;
    }
    {
        // the queued grids on the host's cores, then appended in world order
        const size_t nj = grid_jobs.size();
        std::vector<std::vector<int>> joff(nj), jlist(nj);
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const size_t nt = std::min<size_t>(std::min(hw, 32u), std::max<size_t>(nj, 1));
        auto work = [&](size_t t) {
            for (size_t j = t; j < nj; j += nt) {
                const GridJob &g = grid_jobs[j];
                build_cells(g.quads, g.n, g.index_base, g.ginv, g.gnx, g.gny, g.bx0, g.by0,
                            joff[j], jlist[j]);
            }
        };
        std::vector<std::thread> pool;
        for (size_t t = 1; t < nt; ++t) pool.emplace_back(work, t);
        work(0);
        for (auto &th : pool) th.join();
        std::vector<int> *offs[3] = {&cell_off, &lcell_off, &rcell_off};
        std::vector<int> *lists[3] = {&cell_quads, &lcell_quads, &rcell_quads};
        for (size_t j = 0; j < nj; ++j) {
            const GridJob &g = grid_jobs[j];
            std::vector<int> &off = *offs[g.grid], &list = *lists[g.grid];
            WorldInfo &wi = h->worlds_h[g.w];
            (g.grid == 0 ? wi.cell_begin : (g.grid == 1 ? wi.lcell_begin : wi.rcell_begin)) =
                (int)off.size() - 1;
            const int base = (int)list.size();
            for (const int e : joff[j]) off.push_back(base + e);
            list.insert(list.end(), jlist[j].begin(), jlist[j].end());
            std::vector<int>().swap(joff[j]);
            std::vector<int>().swap(jlist[j]);
        }
    }
    h->n_agents = (int)agent_world.size();
    h->n_boxes = nbox;
    h->n_views = h->n_agents * cfg->n_cams;

    for (int c = 0; c < 4; ++c) {
        h->onehot[c][0] = bf16_bits((0.f - cfg->norm_mean[c]) / cfg->norm_std[c]);
        h->onehot[c][1] = bf16_bits((1.f - cfg->norm_mean[c]) / cfg->norm_std[c]);
    }

#define UP(buf, vec)                                                                        \
    do {                                                                                    \
        cudaError_t e_ = h->buf.upload(vec);                                                \
        if (e_ != cudaSuccess) {                                                            \
            gp_destroy(h);                                                                  \
            return fail(e_ == cudaErrorMemoryAllocation ? GP_ENOMEM : GP_ECUDA,             \
                        std::string("upload " #buf ": ") + cudaGetErrorString(e_));         \
        }                                                                                   \
    } while (0)
    UP(worlds, h->worlds_h);
    UP(box_pose, pose);
    UP(pose0, pose);
    UP(box_dim, dim);
    UP(speed, speed);
    UP(speed0, speed);
    std::vector<uint8_t> zeros(h->n_agents, 0);
    UP(flags, zeros);
    UP(agent_world, agent_world);
    UP(agent_box, agent_box);
    UP(clusters, clusters);
    UP(quad_geo, quad_geo);
    UP(quad_prim, quad_prim);
    UP(road_geo, road_geo);
    UP(cell_off, cell_off);
    UP(cell_quads, cell_quads);
    UP(line_geo, line_geo);
    UP(lcell_off, lcell_off);
    UP(lcell_quads, lcell_quads);
    UP(rcell_off, rcell_off);
    UP(rcell_quads, rcell_quads);
    if (seg_list.empty()) seg_list.push_back(0);
    UP(seg_off, seg_off);
    UP(seg_list, seg_list);
    {
        const size_t ns = d->signal_off ? (size_t)d->signal_off[nw] : 0;
        std::vector<float4> sig(std::max<size_t>(ns, 1), make_float4(0.f, 0.f, 0.f, 1.f));
        std::vector<uint8_t> sst(std::max<size_t>(ns, 1), 0);
        std::vector<int> sq(std::max<size_t>(ns, 1), -1);
        for (size_t s = 0; s < ns; ++s) {
            const float *q = d->signal + 4 * s;
            sig[s] = make_float4(q[0], q[1], q[2], q[3]);
            sst[s] = d->signal_state ? d->signal_state[s] : (uint8_t)GP_SIGNAL_RED;
        }
        // the road quad each signal controls: the one of smallest index under its centre
        for (int w = 0; w < nw && d->signal_off; ++w) {
            const WorldInfo &wi = h->worlds_h[w];
            for (int s = d->signal_off[w]; s < d->signal_off[w + 1]; ++s) {
                const float px = d->signal[4 * s], py = d->signal[4 * s + 1];
                for (int r = 0; r < wi.n_road; ++r) {
                    const float *q = d->road + 8 * (size_t)(d->road_off[w] + r);
                    bool in = true;
                    for (int k = 0; k < 4 && in; ++k) {
                        const int n = (k + 1) & 3;
                        in = (q[2 * n] - q[2 * k]) * (py - q[2 * k + 1]) -
                                 (q[2 * n + 1] - q[2 * k + 1]) * (px - q[2 * k]) >= 0.f;
                    }
                    if (in) {
                        sq[s] = wi.road_begin + r;
                        break;
                    }
                }
            }
        }
        h->n_signals = (int)ns;
        UP(sig, sig);
        UP(sig_state, sst);
        UP(sig_quad, sq);
    }
    {
        std::vector<unsigned long long> z(GP_STAT_COUNT, 0ull);
        UP(stats, z);
        std::vector<int> ep(std::max(1, nw), 0);
        UP(ep_counter, ep);
        std::vector<int> ei(std::max(1, h->n_agents), 0);
        UP(ep_index, ei);
        std::vector<float> c0(12 * (size_t)std::max(1, h->n_agents), 0.f);
        UP(cond, c0);
    }
    std::vector<int> one(1, 0);
    UP(counter, one);
    UP(dump_count, one);
    std::vector<uint32_t> st0(1, 0);
    UP(status, st0);
    std::vector<float> stage(4 * (size_t)std::max(1, h->n_agents), 0.f);
    UP(state_stage, stage);
    std::vector<uint8_t> fstage(std::max(1, h->n_agents), 0);
    UP(flag_stage, fstage);
    std::vector<float2> astage(std::max(1, h->n_agents), make_float2(0.f, 0.f));
    UP(act_stage, astage);
    std::vector<uint8_t> wstage(std::max(1, nw), 0);
    UP(world_stage, wstage);
    {
        const size_t na = (size_t)std::max(1, h->n_agents);
        std::vector<float> r0(na, 0.f), e0(GP_EGO_DIM * na, 0.f), w0(10 * na), j0(3 * na, 0.f);
        const float inference[10] = {3.f, 3.f, 0.05f, 0.025f, 3.8e-3f, 2.5e-3f, 1.f, 2.5e-5f, 5e-3f, 0.f};
        for (size_t i = 0; i < na; ++i)
            for (int k = 0; k < 10; ++k) w0[10 * i + k] = inference[k];
        std::vector<float2> a0(na, make_float2(0.f, 0.f));
        UP(reward, r0);
        UP(ego, e0);
        UP(weights, w0);
        UP(acc, a0);
        UP(jerk, j0);
    }
#undef UP

    if (render_configure(smem_limit(device) - 1024) != cudaSuccess) {
        gp_destroy(h);
        return fail(GP_ECUDA, "cannot configure render kernel shared memory");
    }
    st = noalloc_setup(device);
    if (st != GP_OK) {
        gp_destroy(h);
        return st;
    }
    h->shape = default_shape(h);
    if (h->shape.blocks == 0) {
        gp_destroy(h);
        return fail(GP_ELIMIT, "no launch shape fits this configuration");
    }
    if (cfg->autotune) {
        st = autotune(h);
        if (st != GP_OK) {
            gp_destroy(h);
            return st;
        }
    }
    std::vector<int2> items;
    build_items(h, h->shape.band_rows, items);
    if (h->items.upload(items) != cudaSuccess) {
        gp_destroy(h);
        return fail(GP_ENOMEM, "upload items");
    }
    if (cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
        gp_destroy(h);
        return fail(GP_ECUDA, "stream create");
    }
    if (h->cfg.reward_conditioning) {  // episode 0's conditioning draws
        ResetParams rp = reset_params(h);
        rp.draw_only = 1;
        if (launch_reset(rp, 0) != cudaSuccess) {
            gp_destroy(h);
            return fail(GP_ECUDA, "create: conditioning draw");
        }
    }
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemset(h->stats.p, 0, sizeof(unsigned long long) * GP_STAT_COUNT) != cudaSuccess) {
        gp_destroy(h);
        return fail(GP_ECUDA, "create: device error");
    }
    *out = h;
    return GP_OK;
}

gp_status gp_step(gp_handle *h, const float *actions, void *stream) {
    NvtxRange range("gp_step");
    if (!h) return fail(GP_EINVAL, "null handle");
    if (!actions) return fail(GP_EINVAL, "actions_dev is null");
    if (h->sticky) return fail(GP_EDEVICE, "device status word has an error bit set");
    CK(cudaSetDevice(h->device));
    gp_status st = check_reach(h, actions, nullptr, nullptr);
    if (st != GP_OK) return st;
    CK(launch_step(step_params(h, actions), 8 * h->sms, (cudaStream_t)stream));
    return GP_OK;
}

gp_status gp_render(gp_handle *h, void *out, void *depth, void *stream) {
    NvtxRange range("gp_render");
    if (!h) return fail(GP_EINVAL, "null handle");
    gp_status st = check_out(out, depth);
    if (st != GP_OK) return st;
    if (h->sticky) return fail(GP_EDEVICE, "device status word has an error bit set");
    CK(cudaSetDevice(h->device));
    st = check_reach(h, nullptr, out, depth);
    if (st != GP_OK) return st;
    CK(enqueue_render(h, render_params(h, out, depth), (cudaStream_t)stream));
    return GP_OK;
}

// One step followed by one render (backend 0: raster, 1: ray tracing), replayed from a
// CUDA graph cached per (backend, actions, out, depth).
static gp_status step_then_render(gp_handle *h, const float *actions, void *out, void *depth,
                                  void *stream, int backend) {
    if (!h) return fail(GP_EINVAL, "null handle");
    if (!actions) return fail(GP_EINVAL, "actions_dev is null");
    gp_status st = check_out(out, depth);
    if (st != GP_OK) return st;
    if (h->sticky) return fail(GP_EDEVICE, "device status word has an error bit set");
    CK(cudaSetDevice(h->device));
    GraphKey key{actions, out, depth, backend};
    auto it = h->graphs.find(key);
    if (it == h->graphs.end()) {
        // checked once per pointer triple: replays of a cached graph reuse the same pointers
        st = check_reach(h, actions, out, depth);
        if (st != GP_OK) return st;
        if (h->graphs.size() >= 4) {
            cudaGraphExecDestroy(h->graphs.begin()->second);
            h->graphs.erase(h->graphs.begin());
        }
        cudaStream_t cs = h->capture_stream;
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        StepParams sp = step_params(h, actions);
        if (!backend && h->n_worlds > 0) sp.render_counter = h->counter.p;  // no memset node
        cudaError_t e1 = launch_step(sp, 8 * h->sms, cs);
        cudaError_t e2 = e1;
        if (e1 == cudaSuccess)
            e2 = backend ? (h->n_views ? launch_trace(render_params(h, out, depth), h->n_views, cs)
                                       : cudaSuccess)
                         : (sp.render_counter
                                ? launch_render(render_params(h, out, depth), h->shape.blocks,
                                                h->shape.threads, h->shape.smem, cs)
                                : enqueue_render(h, render_params(h, out, depth), cs));
        cudaGraph_t g = nullptr;
        cudaError_t e3 = cudaStreamEndCapture(cs, &g);
        if (e2 != cudaSuccess || e3 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail(GP_ECUDA, std::string("graph capture: ") +
                                      cudaGetErrorString(e2 != cudaSuccess ? e2 : e3));
        }
        cudaGraphExec_t ge = nullptr;
        cudaError_t e4 = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e4 != cudaSuccess)
            return fail(GP_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e4));
        it = h->graphs.emplace(key, ge).first;
    }
    CK(cudaGraphLaunch(it->second, (cudaStream_t)stream));
    return GP_OK;
}

gp_status gp_step_render(gp_handle *h, const float *actions, void *out, void *depth,
                         void *stream) {
    NvtxRange range("gp_step_render");
    return step_then_render(h, actions, out, depth, stream, 0);
}

gp_status gp_step_render_host(gp_handle *h, const float *actions_host, void *out, void *depth,
                              float *state_host, uint8_t *flags_host, void *stream) {
    NvtxRange range("gp_step_render_host");
    if (!h) return fail(GP_EINVAL, "null handle");
    if (!actions_host) return fail(GP_EINVAL, "actions_host is null");
    CK(cudaSetDevice(h->device));
    gp_status st = check_pinned(actions_host, "actions_host");
    if (st == GP_OK) st = check_pinned(state_host, "state_host");
    if (st == GP_OK) st = check_pinned(flags_host, "flags_host");
    if (st != GP_OK) return st;
    if (h->sticky) return fail(GP_EDEVICE, "device status word has an error bit set");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = h->n_agents;
    if (n) CK(cudaMemcpyAsync(h->act_stage.p, actions_host, sizeof(float2) * n, cudaMemcpyHostToDevice, s));
    st = step_then_render(h, (const float *)h->act_stage.p, out, depth, stream, 0);
    if (st != GP_OK) return st;
    if (n && (state_host || flags_host)) {
        CK(launch_state(h->state_stage.p, h->flag_stage.p, h->box_pose.p, h->speed.p, h->flags.p,
                        h->agent_box.p, n, 1, s));
        if (state_host)
            CK(cudaMemcpyAsync(state_host, h->state_stage.p, sizeof(float) * 4 * n, cudaMemcpyDeviceToHost, s));
        if (flags_host) CK(cudaMemcpyAsync(flags_host, h->flag_stage.p, n, cudaMemcpyDeviceToHost, s));
    }
    return GP_OK;
}

gp_status gp_step_trace(gp_handle *h, const float *actions, void *out, void *depth,
                        void *stream) {
    NvtxRange range("gp_step_trace");
    return step_then_render(h, actions, out, depth, stream, 1);
}

gp_status gp_step_world(gp_handle *h, int32_t world, const float *actions, void *stream) {
    if (!h) return fail(GP_EINVAL, "null handle");
    if (world < 0 || world >= h->n_worlds) return fail(GP_EINVAL, "world out of range");
    if (!actions) return fail(GP_EINVAL, "actions_dev is null");
    if (h->sticky) return fail(GP_EDEVICE, "device status word has an error bit set");
    CK(cudaSetDevice(h->device));
    gp_status st = check_reach(h, actions, nullptr, nullptr);
    if (st != GP_OK) return st;
    StepParams p = step_params(h, actions);
    p.world_begin = world;
    p.n_worlds = 1;
    CK(launch_step(p, 1, (cudaStream_t)stream));
    return GP_OK;
}

gp_status gp_trace(gp_handle *h, void *out, void *depth, void *stream) {
    NvtxRange range("gp_trace");
    if (!h) return fail(GP_EINVAL, "null handle");
    gp_status st = check_out(out, depth);
    if (st != GP_OK) return st;
    if (h->sticky) return fail(GP_EDEVICE, "device status word has an error bit set");
    CK(cudaSetDevice(h->device));
    st = check_reach(h, nullptr, out, depth);
    if (st != GP_OK) return st;
    if (h->n_views) CK(launch_trace(render_params(h, out, depth), h->n_views, (cudaStream_t)stream));
    return GP_OK;
}

gp_status gp_render_world(gp_handle *h, int32_t world, void *out, void *depth, void *stream) {
    if (!h) return fail(GP_EINVAL, "null handle");
    if (world < 0 || world >= h->n_worlds) return fail(GP_EINVAL, "world out of range");
    gp_status st = check_out(out, depth);
    if (st != GP_OK) return st;
    if (h->sticky) return fail(GP_EDEVICE, "device status word has an error bit set");
    CK(cudaSetDevice(h->device));
    st = check_reach(h, nullptr, out, depth);
    if (st != GP_OK) return st;
    RenderParams p = render_params(h, out, depth);
    p.item_begin = h->world_item_begin[world];
    p.n_items = h->world_item_count[world];
    p.work_counter = nullptr;
    CK(launch_render(p, std::max(1, p.n_items), h->shape.threads, h->shape.smem,
                     (cudaStream_t)stream));
    return GP_OK;
}

gp_status gp_get_state(gp_handle *h, float *state, uint8_t *flags, int on_host, void *stream) {
    if (!h) return fail(GP_EINVAL, "null handle");
    if (!state && !flags) return fail(GP_EINVAL, "state and flags are both null");
    CK(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int n = h->n_agents;
    float *ds = (on_host || !state) ? h->state_stage.p : state;
    uint8_t *df = (on_host || !flags) ? h->flag_stage.p : flags;
    CK(launch_state(ds, df, h->box_pose.p, h->speed.p, h->flags.p, h->agent_box.p, n, 1, s));
    if (on_host) {
        if (state && n) CK(cudaMemcpyAsync(state, ds, sizeof(float) * 4 * n, cudaMemcpyDeviceToHost, s));
        if (flags && n) CK(cudaMemcpyAsync(flags, df, n, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return GP_OK;
}

gp_status gp_set_state(gp_handle *h, const float *state, const uint8_t *flags, int on_host,
                       void *stream) {
    if (!h) return fail(GP_EINVAL, "null handle");
    if (!state || !flags) return fail(GP_EINVAL, "state and flags are required");
    CK(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int n = h->n_agents;
    if (on_host) {
        if (!finite_all(state, 4 * (size_t)n)) return fail(GP_EINVAL, "non-finite state");
        if (n) {
            CK(cudaMemcpyAsync(h->state_stage.p, state, sizeof(float) * 4 * n, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(h->flag_stage.p, flags, n, cudaMemcpyHostToDevice, s));
        }
        CK(launch_state(h->state_stage.p, h->flag_stage.p, h->box_pose.p, h->speed.p, h->flags.p,
                        h->agent_box.p, n, 0, s));
        CK(cudaStreamSynchronize(s));
    } else {
        CK(launch_state(const_cast<float *>(state), const_cast<uint8_t *>(flags), h->box_pose.p,
                        h->speed.p, h->flags.p, h->agent_box.p, n, 0, s));
    }
    if (n) CK(cudaMemsetAsync(h->acc.p, 0, sizeof(float2) * n, s));  // accelerations restart
    if (n) CK(cudaMemsetAsync(h->jerk.p, 0, sizeof(float) * 3 * n, s));
    return GP_OK;
}

gp_status gp_get_conditioning(gp_handle *h, float *cond, int on_host, void *stream) {
    if (!h || !cond) return fail(GP_EINVAL, "null argument");
    if (!h->cfg.reward_conditioning)
        return fail(GP_ESTATE, "reward conditioning is off (gp_config.reward_conditioning = 0)");
    CK(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)h->n_agents;
    if (n)
        CK(cudaMemcpyAsync(cond, h->cond.p, sizeof(float) * 12 * n,
                           on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    if (on_host) CK(cudaStreamSynchronize(s));
    return GP_OK;
}

gp_status gp_get_render_stats(gp_handle *h, uint64_t *out, int reset) {
    if (!h || !out) return fail(GP_EINVAL, "null argument");
    if (!h->cfg.stats) return fail(GP_ESTATE, "stats are off (gp_config.stats = 0)");
    CK(cudaSetDevice(h->device));
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(out, h->stats.p, sizeof(uint64_t) * GP_STAT_COUNT, cudaMemcpyDeviceToHost));
    if (reset) CK(cudaMemset(h->stats.p, 0, sizeof(uint64_t) * GP_STAT_COUNT));
    return GP_OK;
}

gp_status gp_reset_worlds(gp_handle *h, const uint8_t *mask, int on_host, void *stream) {
    if (!h) return fail(GP_EINVAL, "null handle");
    CK(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    ResetParams p = reset_params(h);
    p.mask = mask;
    if (mask && on_host) {
        if (h->n_worlds) CK(cudaMemcpyAsync(h->world_stage.p, mask, h->n_worlds, cudaMemcpyHostToDevice, s));
        p.mask = h->world_stage.p;
    }
    CK(launch_reset(p, s));
    if (on_host) CK(cudaStreamSynchronize(s));
    return GP_OK;
}

gp_status gp_set_signal_states(gp_handle *h, const uint8_t *state, int on_host, void *stream) {
    if (!h || !state) return fail(GP_EINVAL, "null argument");
    CK(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)h->n_signals;
    if (on_host)
        for (size_t i = 0; i < n; ++i)
            if (state[i] > GP_SIGNAL_OFF) return fail(GP_EINVAL, "signal state must be 0..3");
    if (n)
        CK(cudaMemcpyAsync(h->sig_state.p, state, n,
                           on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    if (on_host) CK(cudaStreamSynchronize(s));
    return GP_OK;
}

gp_status gp_get_dynamics(gp_handle *h, float *dyn, int on_host, void *stream) {
    if (!h || !dyn) return fail(GP_EINVAL, "null argument");
    if (h->cfg.dynamics != GP_DYN_JERK) return fail(GP_ESTATE, "dynamics is not GP_DYN_JERK");
    CK(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)h->n_agents;
    if (n)
        CK(cudaMemcpyAsync(dyn, h->jerk.p, sizeof(float) * 3 * n,
                           on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    if (on_host) CK(cudaStreamSynchronize(s));
    return GP_OK;
}

gp_status gp_set_dynamics(gp_handle *h, const float *dyn, int on_host, void *stream) {
    if (!h || !dyn) return fail(GP_EINVAL, "null argument");
    if (h->cfg.dynamics != GP_DYN_JERK) return fail(GP_ESTATE, "dynamics is not GP_DYN_JERK");
    CK(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)h->n_agents;
    if (on_host && !finite_all(dyn, 3 * n)) return fail(GP_EINVAL, "non-finite dynamics state");
    if (n)
        CK(cudaMemcpyAsync(h->jerk.p, dyn, sizeof(float) * 3 * n,
                           on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    if (on_host) CK(cudaStreamSynchronize(s));
    return GP_OK;
}

gp_status gp_observe_vec(gp_handle *h, float *agents, float *roads, float *signals, void *stream) {
    NvtxRange range("gp_observe_vec");
    if (!h) return fail(GP_EINVAL, "null handle");
    if ((agents && !aligned16(agents)) || (roads && !aligned16(roads)) ||
        (signals && !aligned16(signals)))
        return fail(GP_EINVAL, "outputs must be 16-byte aligned");
    CK(cudaSetDevice(h->device));
    gp_status st = check_reach(h, agents, "agents_dev");
    if (st == GP_OK) st = check_reach(h, roads, "roads_dev");
    if (st == GP_OK) st = check_reach(h, signals, "signals_dev");
    if (st != GP_OK) return st;
    ObsParams p{};
    p.worlds = h->worlds.p;
    p.agent_world = h->agent_world.p;
    p.n_agents = h->n_agents;
    p.box_pose = h->box_pose.p;
    p.box_dim = h->box_dim.p;
    p.speed = h->speed.p;
    p.road_geo = h->road_geo.p;
    p.line_geo = h->line_geo.p;
    p.seg_off = h->seg_off.p;
    p.seg_list = h->seg_list.p;
    p.sig = h->sig.p;
    p.sig_state = h->sig_state.p;
    p.agents_out = agents;
    p.roads_out = roads;
    p.signals_out = signals;
    CK(launch_obs(p, (cudaStream_t)stream));
    return GP_OK;
}

gp_status gp_get_rewards(gp_handle *h, float *reward, float *ego, int on_host, void *stream) {
    if (!h) return fail(GP_EINVAL, "null handle");
    if (!h->cfg.rewards) return fail(GP_ESTATE, "rewards are off (gp_config.rewards = 0)");
    CK(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)h->n_agents;
    const cudaMemcpyKind k = on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (reward && n) CK(cudaMemcpyAsync(reward, h->reward.p, sizeof(float) * n, k, s));
    if (ego && n) CK(cudaMemcpyAsync(ego, h->ego.p, sizeof(float) * GP_EGO_DIM * n, k, s));
    if (on_host) CK(cudaStreamSynchronize(s));
    return GP_OK;
}

gp_status gp_set_reward_weights(gp_handle *h, const float *weights, int on_host, void *stream) {
    if (!h || !weights) return fail(GP_EINVAL, "null argument");
    CK(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)h->n_agents;
    if (on_host) {
        if (!finite_all(weights, 10 * n)) return fail(GP_EINVAL, "non-finite reward weights");
        if (n) CK(cudaMemcpyAsync(h->weights.p, weights, sizeof(float) * 10 * n, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    } else if (n) {
        CK(cudaMemcpyAsync(h->weights.p, weights, sizeof(float) * 10 * n, cudaMemcpyDeviceToDevice, s));
    }
    return GP_OK;
}

gp_status gp_get_reward_weights(gp_handle *h, float *weights, int on_host, void *stream) {
    if (!h || !weights) return fail(GP_EINVAL, "null argument");
    CK(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)h->n_agents;
    if (n)
        CK(cudaMemcpyAsync(weights, h->weights.p, sizeof(float) * 10 * n,
                           on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    if (on_host) CK(cudaStreamSynchronize(s));
    return GP_OK;
}

gp_status gp_get_info(gp_handle *h, gp_info *info) {
    if (!h || !info) return fail(GP_EINVAL, "null argument");
    info->n_worlds = h->n_worlds;
    info->n_agents = h->n_agents;
    info->n_boxes = h->n_boxes;
    info->n_views = h->n_views;
    info->width = h->cfg.width;
    info->height = h->cfg.height;
    info->n_cams = h->cfg.n_cams;
    info->key_precision = h->cfg.key_precision;
    info->output = h->cfg.output;
    const long long px = (long long)h->cfg.width * h->cfg.height * h->n_views;
    info->out_bytes = px * (h->cfg.output == GP_OUT_CLASS_U8 ? 1 : (h->cfg.output == GP_OUT_RGB_U8 ? 3 : 8));
    info->depth_bytes = px * (h->cfg.key_precision == GP_KEY_F32 ? 4 : 2);
    info->band_rows = h->shape.band_rows;
    info->threads = h->shape.threads;
    info->tri_capacity = h->shape.tri_cap;
    info->blocks = h->shape.blocks;
    info->producer_warps = h->shape.prod_warps;
    return GP_OK;
}

gp_status gp_get_status(gp_handle *h, uint32_t *bits) {
    if (!h || !bits) return fail(GP_EINVAL, "null argument");
    CK(cudaSetDevice(h->device));
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(bits, h->status.p, 4, cudaMemcpyDeviceToHost));
    h->sticky = *bits != 0;
    return GP_OK;
}

gp_status gp_clear_status(gp_handle *h) {
    if (!h) return fail(GP_EINVAL, "null handle");
    CK(cudaSetDevice(h->device));
    CK(cudaDeviceSynchronize());
    CK(cudaMemset(h->status.p, 0, 4));
    h->sticky = false;
    return GP_OK;
}

gp_status gp_debug_inject_status(gp_handle *h, uint32_t bits) {
    if (!h) return fail(GP_EINVAL, "null handle");
    CK(cudaSetDevice(h->device));
    uint32_t cur = 0;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(&cur, h->status.p, 4, cudaMemcpyDeviceToHost));
    cur |= bits;
    CK(cudaMemcpy(h->status.p, &cur, 4, cudaMemcpyHostToDevice));
    return GP_OK;
}

gp_status gp_debug_stall_pipeline(gp_handle *h, void *out, void *depth, int64_t wait_ns,
                                  void *stream) {
    if (!h) return fail(GP_EINVAL, "null handle");
    if (wait_ns < 1000000 || wait_ns > 2000000000) return fail(GP_EINVAL, "wait_ns outside 1e6..2e9");
    gp_status st = check_out(out, depth);
    if (st != GP_OK) return st;
    CK(cudaSetDevice(h->device));
    if (h->sticky) return fail(GP_EDEVICE, "device status word has an error bit set");
    st = check_reach(h, nullptr, out, depth);
    if (st != GP_OK) return st;
    Shape s = h->shape;  // same bands as the handle's work list
    s.prod_warps = std::max(1, s.threads / 128);
    if (!finish_shape(h, s)) {
        s.tri_cap = 256;
        if (!finish_shape(h, s)) return fail(GP_ELIMIT, "no pipelined launch shape fits");
    }
    RenderParams p = render_params(h, out, depth);
    p.prod_warps = s.prod_warps;
    p.tri_cap = s.tri_cap;
    p.wait_ns = (unsigned long long)wait_ns;
    p.debug_stall = 1;
    CK(launch_render(p, s.blocks, s.threads, s.smem, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    return GP_OK;
}

gp_status gp_debug_dump_tris(gp_handle *h, int32_t view, void *out, void *depth, void *host_tris,
                             int64_t cap, int64_t *n, void *stream) {
    if (!h || !n) return fail(GP_EINVAL, "null argument");
    if (view < 0 || view >= h->n_views) return fail(GP_EINVAL, "view out of range");
    if (cap < 0 || (cap > 0 && !host_tris)) return fail(GP_EINVAL, "bad capacity/buffer");
    gp_status st = check_out(out, depth);
    if (st != GP_OK) return st;
    CK(cudaSetDevice(h->device));
    if (h->sticky) return fail(GP_EDEVICE, "device status word has an error bit set");
    st = check_reach(h, nullptr, out, depth);
    if (st != GP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t want = (size_t)std::max<int64_t>(std::min<int64_t>(cap, 1 << 24), 1);
    if (h->dump.n < want) {
        h->dump.release();
        CK(h->dump.alloc(want));
    }
    CK(cudaMemsetAsync(h->dump_count.p, 0, sizeof(int), s));
    RenderParams p = render_params(h, out, depth);
    p.dump_view = view;
    p.dump = h->dump.p;
    p.dump_count = h->dump_count.p;
    p.dump_cap = (int)want;
    CK(enqueue_render(h, p, s));
    int cnt = 0;
    CK(cudaMemcpyAsync(&cnt, h->dump_count.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *n = cnt;
    const int64_t take = std::min<int64_t>(std::min<int64_t>(cnt, cap), (int64_t)want);
    if (take > 0) CK(cudaMemcpy(host_tris, h->dump.p, sizeof(DumpTri) * take, cudaMemcpyDeviceToHost));
    return GP_OK;
}

}  // extern "C"

extern "C" gp_status gp_debug_dump_tris_noalloc(gp_handle *h, int32_t view, void *out,
                                                void *depth, void *host_tris, int64_t cap,
                                                int64_t *n, void *stream) {
    if (!h || !n) return fail(GP_EINVAL, "null argument");
    if (view < 0 || view >= h->n_views) return fail(GP_EINVAL, "view out of range");
    if (cap < 0 || (cap > 0 && !host_tris)) return fail(GP_EINVAL, "bad capacity/buffer");
    if (cap > GP_NOALLOC_MAX_TRIS)
        return fail(GP_ELIMIT, "cap exceeds GP_NOALLOC_MAX_TRIS (16384 records), the size of the "
                               "fixed scratch of the allocation-free dump");
    gp_status st = check_out(out, depth);
    if (st != GP_OK) return st;
    CK(cudaSetDevice(h->device));
    if (h->sticky) return fail(GP_EDEVICE, "device status word has an error bit set");
    st = check_reach(h, nullptr, out, depth);
    if (st != GP_OK) return st;
    // set up when the handle was created on this device (no lookup or allocation here)
    unsigned char *scratch = noalloc_scratch(h->device);
    if (!scratch) return fail(GP_ESTATE, "no allocation-free scratch on this device");
    cudaStream_t s = (cudaStream_t)stream;
    int *counters = (int *)scratch;
    // the work counter and the record count must start at zero; the records need no clearing
    CK(cudaMemsetAsync(counters, 0, 2 * sizeof(int), s));
    RenderParams p = render_params(h, out, depth);
    p.work_counter = counters;
    p.dump_count = counters + 1;
    p.dump = (DumpTri *)(scratch + 256);
    p.dump_cap = (int)cap;
    p.dump_view = view;
    CK(launch_render(p, h->shape.blocks, h->shape.threads, h->shape.smem, s));
    int cnt = 0;
    CK(cudaMemcpyAsync(&cnt, counters + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *n = cnt;
    const int64_t take = std::min<int64_t>(cnt, cap);
    if (take > 0) {
        CK(cudaMemcpyAsync(host_tris, p.dump, sizeof(DumpTri) * take, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return GP_OK;
}
