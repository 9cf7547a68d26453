/*
 * gigapixel.h -- C ABI of the batched step-and-render library (B300, sm_103a).
 *
 * The library simulates thousands of independent driving worlds on one GPU and renders
 * every agent's ego-centric perspective camera of a bounding-box world into a caller-owned
 * device tensor.  It follows the problem statement of "Scaling Self-Play for End-to-End
 * Driving" (Gigapixel): the simulator state is agent boxes plus static map geometry
 * (Sec. 3.1), each agent receives a rendered ego-centric view, many worlds are stepped and
 * rendered together in one batched launch, and images stay on the GPU as a batched tensor
 * with no per-step host transfer (App. A, "High-Throughput Batched Rendering").  Dynamics
 * and infractions follow App. A ("Action Space and Dynamics", "Other Details").
 *
 * Conventions for every entry point:
 *  - Device pointers are raw CUDA device addresses on the handle's device, contiguous, in
 *    the layout stated at each call.  The library never frees or keeps a caller pointer
 *    after a call returns (except inside a captured graph, see gp_step_render).  Pointers
 *    that the handle's GPU cannot address (pageable host memory, another GPU's memory)
 *    return GP_EINVAL before any launch; the sizes behind a pointer cannot be checked.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  All work
 *    is enqueued asynchronously on it; the call returns before the GPU finishes.  Calls on
 *    one handle must be ordered (one stream, or caller-side events).
 *  - Errors detectable on the host return a negative gp_status immediately and leave the
 *    handle unchanged; gp_last_error() then describes the failure.  Conditions found on
 *    the device (non-finite agent state, internal capacity limits) set bits in a device
 *    status word read by gp_get_status; kernels never trap and never spin.
 */
#ifndef GIGAPIXEL_H
#define GIGAPIXEL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gp_handle gp_handle; /* opaque, owned by the library */

typedef enum gp_status {
    GP_OK = 0,
    GP_EINVAL = -1,   /* invalid argument or descriptor */
    GP_ENOMEM = -2,   /* device or host allocation failed */
    GP_ECUDA = -3,    /* a CUDA runtime call failed */
    GP_ELIMIT = -4,   /* a size exceeds a documented limit */
    GP_EDEVICE = -5,  /* the device status word has a sticky error bit set */
    GP_ESTATE = -6    /* call not valid in the handle's current state */
} gp_status;

/* Depth-key precision of the rasteriser. */
enum { GP_KEY_F32 = 0, GP_KEY_F16 = 1 };
/* Image encoding written by gp_render. */
enum { GP_OUT_CLASS_U8 = 0, GP_OUT_ONEHOT_BF16 = 1, GP_OUT_RGB_U8 = 2 };
/* Per-agent flag bits (latched for the lifetime of the handle or until gp_set_state). */
enum { GP_FLAG_COLLIDED = 1, GP_FLAG_OFFROAD = 2, GP_FLAG_HALTED = 4,
       GP_FLAG_DONE = 8, /* set for one step: the world's episode ended and it was reset */
       GP_FLAG_RED_LIGHT = 16 /* the agent ran a red light (App. A "Other Details") */ };
/* Device status bits (sticky until gp_clear_status). */
enum {
    GP_DEV_NONFINITE_STATE = 1u << 0, /* an agent's state became NaN/inf */
    GP_DEV_CLIP_OVERFLOW = 1u << 1,   /* internal clip capacity exceeded (image may be incomplete) */
    GP_DEV_PIPELINE_TIMEOUT = 1u << 2, /* a pipelined render block gave up waiting for its other
                                          side after 2 s and left its items unfinished */
    GP_DEV_INJECTED = 1u << 31        /* set by gp_debug_inject_status */
};

/* Pixel classes of the class image / one-hot channels (signals share channel 3). */
enum { GP_CLASS_BACKGROUND = 0, GP_CLASS_ROAD = 1, GP_CLASS_LANE_LINE = 2, GP_CLASS_VEHICLE = 3,
       GP_CLASS_SIGNAL = 4 };
/* Traffic-signal states (gp_world_desc.signal_state, gp_set_signal_states). */
enum { GP_SIGNAL_RED = 0, GP_SIGNAL_AMBER = 1, GP_SIGNAL_GREEN = 2, GP_SIGNAL_OFF = 3 };

/* Limits (GP_ELIMIT beyond them). */
#define GP_MAX_CAMS 8            /* cameras per agent */
#define GP_MAX_BOXES 128         /* boxes (agents + static) per world */
#define GP_MAX_QUADS 32767       /* road + lane-line quads per world */
#define GP_MAX_WIDTH 512         /* image width and height */
#define GP_MAX_SIGNALS 32        /* traffic-signal spheres per world */
/* Vectorized observations (gp_observe_vec) */
#define GP_OBS_AGENTS 16         /* surrounding-agent slots per agent */
#define GP_OBS_AGENT_RADIUS 100.0f
#define GP_OBS_ROADS 32          /* road-segment slots per agent */
#define GP_OBS_ROAD_RADIUS 30.0f
#define GP_OBS_SIGNALS 4         /* traffic-signal slots per agent */
#define GP_OBS_SIGNAL_RADIUS 50.0f
/* Render counters (gp_config.stats = 1, read with gp_get_render_stats), summed over
 * every render launch since the last reset; a triangle spanning several screen bands is
 * set up once per band. */
enum {
    GP_STAT_ITEMS = 0,          /* (view, band) work items */
    GP_STAT_CLUSTERS = 1,       /* culling clusters visible in an item's band */
    GP_STAT_BOXES = 2,          /* boxes visible in an item's band */
    GP_STAT_SIGNALS = 3,        /* signal spheres visible in an item's band */
    GP_STAT_QUADS = 4,          /* quads set up (visible clusters' quads, box faces, sphere faces) */
    GP_STAT_TRIS_KEPT = 5,      /* triangles kept without clipping */
    GP_STAT_TRIS_CLIPPED = 6,   /* triangles sent to near/guard-band clipping */
    GP_STAT_TRIS_FROM_CLIP = 7, /* triangles kept out of clipping */
    GP_STAT_BATCHES = 8,        /* raster batches */
    GP_STAT_ROW_ITEMS = 9,      /* (triangle, row) raster items */
    GP_STAT_FRAGMENTS = 10,     /* covered (triangle, pixel) pairs depth-tested */
    GP_STAT_COUNT = 16
};

/* Ego-state width (gp_get_rewards) */
#define GP_EGO_DIM 9

/* Vehicle dynamics (gp_config.dynamics). */
enum {
    GP_DYN_DIRECT = 0,  /* actions are (acceleration m/s^2, steering angle rad) */
    GP_DYN_JERK = 1     /* actions are (longitudinal, lateral jerk m/s^3); App. A's discrete set
                           is {-15, -4, 0, 4} x {-4, 0, 4} */
};

/*
 * Worlds, as host arrays in CSR form over worlds; copied to the device at create time.
 * Geometry is in metres, world frame x/y on the ground, z up, angles in radians.
 *   box_off[n_worlds+1]    boxes of world w: [box_off[w], box_off[w+1])
 *   agent_count[n_worlds]  the first agent_count[w] boxes of world w are agents (each
 *                          carries the cameras); the rest are static obstacles
 *   boxes[n_boxes][7]      x, y (footprint centre), yaw, length, width, height, v0
 *                          (initial speed, agents only)
 *   road_off/road          road-surface quads [n][8]: four (x, y) corners, counter-clockwise
 *                          seen from above, on the ground plane z = 0 (class road)
 *   line_off/line          lane-line strips [n][8], same layout, at z = lane_line_z
 *                          (class lane line)
 *   signal_off/signal      traffic-signal spheres [n][4]: centre x, y, z and radius > 0
 *                          (class signal); NULL signal_off = none.  A sphere is drawn as
 *                          the polyhedron with vertices on it at latitudes -90, -45, 0, 45,
 *                          90 deg and longitudes k 45 deg: quad q = 8 i + j (band i = 0..3
 *                          from the south pole, sector j) with corners (i, j), (i, j+1),
 *                          (i+1, j+1), (i+1, j), split into (q0 q1 q2), (q0 q2 q3)
 *   signal_state[n]        GP_SIGNAL_* state of each sphere (RGB colour); NULL = all red
 * Primitive ids of a world (used for the depth tie-break): box b face triangle t ->
 * 12 b + t; road quad r triangle t -> 12 n_boxes + 2 r + t; lane-line quad l triangle t ->
 * 12 n_boxes + 2 n_road + 2 l + t; signal s quad q triangle t -> 12 n_boxes + 2 n_road +
 * 2 n_line + 64 s + 2 q + t.
 */
typedef struct gp_world_desc {
    int32_t n_worlds;
    const int32_t *box_off;
    const int32_t *agent_count;
    const float *boxes;
    const int32_t *road_off;
    const float *road;
    const int32_t *line_off;
    const float *line;
    const int32_t *signal_off;
    const float *signal;
    const uint8_t *signal_state;
} gp_world_desc;

/*
 * Simulation and camera configuration.  gp_default_config fills the defaults listed here.
 */
typedef struct gp_config {
    int32_t width, height;        /* image size, 16..GP_MAX_WIDTH each, both even
                                     (default 128 x 128) */
    int32_t n_cams;               /* cameras per agent, 1..GP_MAX_CAMS (default 1) */
    float cam_yaw[GP_MAX_CAMS];   /* camera yaw offsets from the agent heading (default 0) */
    float hfov;                   /* horizontal field of view (default pi/2) */
    float cam_height;             /* camera height above ground (default 1.5 m) */
    float near_plane;             /* near clip distance (default 0.1 m) */
    float lane_line_z;            /* lane-line strip height above the road (default 0.02 m) */
    float dt;                     /* simulation step (default 0.1 s, App. A) */
    float v_max;                  /* speed clamp (default 30 m/s) */
    int32_t key_precision;        /* GP_KEY_F32 (default) or GP_KEY_F16 (reversed-Z binary16) */
    int32_t output;               /* GP_OUT_CLASS_U8 (default), GP_OUT_ONEHOT_BF16 or
                                     GP_OUT_RGB_U8 */
    float norm_mean[4];           /* one-hot normalisation (default 0.5 each) */
    float norm_std[4];            /* (default 0.5 each -> values are exactly +-1) */
    int32_t autotune;             /* 1: time candidate launch shapes at create (default 0) */
    int32_t band_rows;            /* rows per screen band (1..128), 0 = auto */
    int32_t threads;              /* render threads per block, 0 = auto */
    int32_t tri_capacity;         /* triangles per raster batch, 0 = auto */
    int32_t producer_warps;       /* pipelined render: warps per block that cull, set up and
                                     clip while the others rasterise (double-buffered batches);
                                     0 = auto (the autotuner may pick it; off otherwise),
                                     -1 = off, n > 0 = on with n warps */
    /* GP_OUT_RGB_U8 appearance (App. A: one directional light per agent, a colour per
     * instance).  colour = class colour * (ambient + (1 - ambient) * max(0, n . l)), n the
     * surface's outward normal (box faces turn with the box yaw; the ground faces +z), l
     * the unit direction towards the light (normalised at create); background unshaded;
     * channels rint(255 * clamp(., 0, 1)). */
    float light_dir[3];           /* towards the light, world frame (default 0.3 0.4 0.866) */
    float ambient;                /* 0..1 (default 0.35) */
    float colour[4][3];           /* RGB in 0..1 of classes background, road, lane line,
                                     vehicle/static box (defaults: sky, grey, off-white, blue) */
    /* Per-step reward terms and ego state (App. A reward table and observations), computed
     * in gp_step when rewards = 1 (default 0) and read with gp_get_rewards. */
    int32_t rewards;
    float lane_width;             /* lane width of the two-lane roads (default 3.5 m) */
    float v_limit;                /* speed limit of the overspeed term (default 30 m/s) */
    int32_t dynamics;             /* GP_DYN_DIRECT (default) or GP_DYN_JERK */
    int32_t stats;                /* 1: count GP_STAT_* events in every render (default 0) */
    int32_t episode_steps;        /* > 0: after this many steps of a world its agents return to
                                     their initial state, flags = GP_FLAG_DONE (default 0 =
                                     never; 200 is the paper's 20 s at dt = 0.1 s) */
    int32_t reward_conditioning;  /* 1: draw every agent's twelve reward coefficients from the
                                     reward table's training distribution at each episode start
                                     (App. A reward conditioning); 0 (default): the weights of
                                     gp_set_reward_weights / the inference column */
    uint32_t conditioning_seed;   /* seed of those draws (default 0) */
    float signal_colour[4][3];    /* RGB in 0..1 of signal states red, amber, green, off
                                     (defaults 0.9 0.1 0.1 / 0.95 0.7 0.1 / 0.1 0.8 0.3 /
                                     0.25 0.25 0.25); shaded like every surface */
} gp_config;

/* Fill `cfg` with the defaults above.  The paper fixes only dt = 0.1 s (App. A "Action
 * Space and Dynamics") and the reward weights' inference column (App. A, Table "Reward
 * terms"); every other default is this library's reading. */
gp_status gp_default_config(gp_config *cfg);

/*
 * Create a batch of worlds on CUDA device `device`: each world is the paper's simulator
 * state S_t = (A_t, M, L_t) -- agent bounding boxes, static map geometry (road planes and
 * lane-line strips) and traffic-light states (Sec. 3.1 "Gigapixel"), rendered as cuboids,
 * planes and spheres (App. A "High-Throughput Batched Rendering").  Copies the descriptor, builds the
 * device-side world layout (culling clusters, off-road grid, work list), optionally runs
 * the autotuner, and returns a handle in *out.  Synchronous.  Limits: GP_MAX_BOXES boxes,
 * GP_MAX_QUADS quads per world; with GP_KEY_F16 a world holds at most 65535 primitive ids.
 * Errors: GP_EINVAL (malformed CSR, non-finite values, bad config), GP_ELIMIT, GP_ENOMEM,
 * GP_ECUDA.
 */
gp_status gp_create_worlds(const gp_world_desc *desc, const gp_config *cfg, int device,
                           gp_handle **out);

/* Release every device and host resource of the handle.  NULL is accepted.  The paper has
 * no counterpart (resource management of this library). */
gp_status gp_destroy(gp_handle *h);

/*
 * Advance every world by one step (App. A "Action Space and Dynamics", "Other Details"):
 * kinematic bicycle (wheelbase 0.6 L) for each non-halted agent, then footprint collisions
 * among all box pairs that contain an agent, then the off-road test (a footprint corner
 * outside every road quad), then the red-light test (the agent's centre entered, during
 * the step, the road quad of smallest index under a red signal's centre), then halt: an
 * agent flagged by any of the three gets v = 0 and ignores later actions but stays in the
 * scene.
 *   actions_dev  float [n_agents][2] device: acceleration (m/s^2), steering angle (rad);
 *                agents ordered by world, then by agent index within the world.
 *                With GP_DYN_JERK: longitudinal and lateral jerk (m/s^3) of the
 *                jerk-actuated bicycle (App. A "Action Space and Dynamics"): the jerks move
 *                the actuator state a_lon in [-5, 3], a_lat in [-4, 4] m/s^2; the steering
 *                angle tracks atan(0.6 L a_lat / max(v^2, 1)) at most 0.5 rad/s, |steer| <=
 *                0.5 rad; the bicycle then runs on (a_lon, steer).  Halted agents' actuator
 *                state is zeroed.
 * Returns GP_EDEVICE if a previous gp_get_status saw an error bit (until gp_clear_status).
 */
gp_status gp_step(gp_handle *h, const float *actions_dev, void *stream);

/*
 * Render every camera of every agent from the current state (App. A rendering; Sec. 3.1
 * scene).  Cameras are ordered [world][agent][camera]; n_views = n_agents * n_cams.
 *   out_dev    GP_OUT_CLASS_U8:    uint8  [n_views][height][width] class ids
 *              GP_OUT_ONEHOT_BF16: bf16   [n_views][4][height][width], channel c holds
 *                                  (1[class == c] - norm_mean[c]) / norm_std[c]
 *              GP_OUT_RGB_U8:      uint8  [n_views][3][height][width] shaded RGB
 *   depth_dev  NULL, or reversed-Z depth n / z_view of the visible surface (0 on
 *              background): float [n_views][height][width] with GP_KEY_F32, binary16 bits
 *              (uint16) with GP_KEY_F16.
 * Both pointers must be 16-byte aligned.
 */
gp_status gp_render(gp_handle *h, void *out_dev, void *depth_dev, void *stream);

/*
 * Ray-traced render (App. A: the renderer's ray-traced backend): one ray per pixel centre
 * from each camera; the nearest hit at or beyond the near plane among the boxes (exact box
 * slabs), the lane-line strips and the road quads (exact plane hits, point in quad, boundary
 * inside); ties go to the lower object.  Same output formats and layouts as gp_render; the
 * depth is near / t of the hit (FP32, or its binary16 bits with GP_KEY_F16), and RGB
 * shading uses the hit surface's normal.  Unlike the raster there is no snapping, fill rule
 * or clipping, so the two differ only along silhouettes.  Asynchronous on `stream`.
 */
gp_status gp_trace(gp_handle *h, void *out_dev, void *depth_dev, void *stream);

/*
 * gp_step followed by gp_render, replayed from a CUDA graph (captured on the first call
 * for this (actions, out, depth) pointer triple; up to 4 graphs are cached, shared with
 * gp_step_trace).  The pointers must stay valid while their graph is cached (until
 * gp_destroy).  gp_step_trace is the same with gp_trace as the renderer.
 */
gp_status gp_step_render(gp_handle *h, const float *actions_dev, void *out_dev,
                         void *depth_dev, void *stream);
gp_status gp_step_trace(gp_handle *h, const float *actions_dev, void *out_dev,
                        void *depth_dev, void *stream);

/*
 * One closed-loop step for a policy that runs on the host (Sec. 3.1: actions in, the next
 * state and the images out): copies actions_host[n_agents][2] (pinned host memory, layout
 * as gp_step) to a library-owned device buffer, replays the gp_step_render graph on it,
 * and copies the post-step agent state (as gp_get_state: x, y, yaw, v per agent) and flags
 * to state_host / flags_host (pinned; either may be NULL).  The images stay on the device
 * in out_dev / depth_dev.  One call instead of five (copy in, step+render, state export,
 * two copies out).  Asynchronous on `stream`: synchronise it before reading state_host or
 * flags_host, and before overwriting actions_host.  Pageable host memory is refused with
 * GP_EINVAL (its copies would not be asynchronous).
 */
gp_status gp_step_render_host(gp_handle *h, const float *actions_host, void *out_dev,
                              void *depth_dev, float *state_host, uint8_t *flags_host,
                              void *stream);

/*
 * Per-world path: step or render one world only (one launch each), writing the world's
 * slice of the same tensors (actions/out/depth point at the start of the FULL arrays).
 * The paper has no counterpart: it is the plain one-world-at-a-time baseline against which
 * the batched launch of App. A "High-Throughput Batched Rendering" is measured.
 */
gp_status gp_step_world(gp_handle *h, int32_t world, const float *actions_dev, void *stream);
gp_status gp_render_world(gp_handle *h, int32_t world, void *out_dev, void *depth_dev,
                          void *stream);

/*
 * Agent state: state[n_agents][4] = x, y, yaw, v (float) and flags[n_agents] (uint8).
 * on_host = 1: host pointers (the call synchronises the stream); 0: device pointers.
 * gp_set_state also forks/resumes a simulation: the paper rolls the teacher out in a
 * parallel simulator instance initialised at the current state S (Sec. 3.2 "Pixel-based
 * student training"; App. B.2: a forked copy of the simulator, horizon 4 s);
 * it zeroes the jerk dynamics' actuator state (restore it with gp_set_dynamics after) and
 * leaves the per-world episode step counters alone (gp_reset_worlds restarts them).
 */
gp_status gp_get_state(gp_handle *h, float *state, uint8_t *flags, int on_host, void *stream);
gp_status gp_set_state(gp_handle *h, const float *state, const uint8_t *flags, int on_host,
                       void *stream);

/*
 * Episode reset (App. A "Other Details": an episode runs for up to 20 s and then ends;
 * the scenario's initial states start the next one): the agents
 * of every world w with mask[w] != 0 (every world if mask is
 * NULL) return to their initial pose and speed from gp_create_worlds, with clear flags and
 * zero previous-step accelerations and actuator state, and the world's episode step
 * counter restarts; other worlds are untouched.
 *   mask  uint8 [n_worlds]; on_host != 0: host memory (synchronous), else device memory
 *         (asynchronous on `stream`, so it can follow a device-side "done" test).
 */
gp_status gp_reset_worlds(gp_handle *h, const uint8_t *mask, int on_host, void *stream);

/*
 * The paper has no counterpart (instrumentation of this library).
 * Render counters out[GP_STAT_COUNT] (host, uint64) summed since create or the last reset
 * (reset != 0 clears them after reading).  Synchronises the device.  GP_ESTATE unless
 * gp_config.stats = 1.
 */
gp_status gp_get_render_stats(gp_handle *h, uint64_t *out, int reset);

/*
 * Reward conditioning vector cond[n_agents][12] (float): the agent's twelve coefficients of
 * its current episode normalised to [-1, 1] -- collision, off-road, comfort, alignment,
 * centering, velocity, traffic light, time, reverse, overspeed (the reward weights in use),
 * goal radius, goal speed tolerance (observed only).  Coefficient k of the agent with index i
 * in world w, episode e (0 at create, +1 at every restart) is lo_k + (hi_k - lo_k) u, u the
 * top 24 bits of output 1 + (w << 40 | e << 20 | i << 4 | k) of the SplitMix64 stream seeded
 * with conditioning_seed, times 2^-24; the normalised value is 2 u - 1.  GP_ESTATE unless
 * gp_config.reward_conditioning = 1.  on_host as for gp_get_state.
 */
gp_status gp_get_conditioning(gp_handle *h, float *cond, int on_host, void *stream);

/*
 * Actuator state of the jerk dynamics, dyn[n_agents][3] float = a_lon, a_lat (m/s^2),
 * steering angle (rad); GP_ESTATE unless gp_config.dynamics = GP_DYN_JERK.  on_host as for
 * gp_get_state.  gp_set_dynamics rejects non-finite host values (GP_EINVAL); device values
 * are taken as given.
 */
gp_status gp_get_dynamics(gp_handle *h, float *dyn, int on_host, void *stream);
gp_status gp_set_dynamics(gp_handle *h, const float *dyn, int on_host, void *stream);

/*
 * Traffic-signal states state[n_signals] (uint8, GP_SIGNAL_*; signals ordered by world),
 * seen from the next call on: RGB colours, the red-light reward term and the traffic
 * controls of O_vec.  on_host as for gp_get_state; host values above GP_SIGNAL_OFF are
 * rejected (GP_EINVAL), device values are taken modulo 4.
 */
gp_status gp_set_signal_states(gp_handle *h, const uint8_t *state, int on_host, void *stream);

/* Sizes of a handle (no counterpart in the paper). */
typedef struct gp_info {
    int32_t n_worlds, n_agents, n_boxes, n_views, width, height, n_cams;
    int32_t key_precision, output;
    int64_t out_bytes, depth_bytes;    /* bytes gp_render writes to out_dev / depth_dev */
    int32_t band_rows, threads, tri_capacity, blocks; /* chosen launch shape */
    int32_t producer_warps;            /* 0 = one-phase-at-a-time render kernel */
} gp_info;
gp_status gp_get_info(gp_handle *h, gp_info *info);

/*
 * Rewards and ego state of the last gp_step (gp_config.rewards = 1, else GP_ESTATE).
 * reward [n_agents] float: the weighted sum of the reward table's terms (App. A) --
 *   collision -(w0 + 0.1 |v|), off-road -w1, comfort -w2 (1[|a_lon| > 3] + 1[|a_lat| > 3]
 *   + 1[|jerk_lon| > 5 or |jerk_lat| > 5]), lane alignment, lane centering and velocity
 *   (w3..w5, from the lane frame of the road quad of smallest index under the agent,
 *   right-hand traffic, 0 off the road), time -w7 dt, reverse -w8 dt, overspeed -w9
 *   (|v| > v_limit), red-light violation -w6 (the agent's centre enters, during the step,
 *   the road quad of smallest index under a red signal's centre); the goal term is 0.
 *   Accelerations are the bicycle's increments of the step (speed before any halt):
 *   a_lon = (v' - v) / dt, a_lat = v dyaw / dt; an agent halted before the step earns 0.
 * ego [n_agents][GP_EGO_DIM] float: speed / v_max, a_lon / 10, a_lat / 10, L / 10, W / 5
 *   (clipped to [-1, 1]) and the collision flag (0 or 1); then, with GP_DYN_JERK, the
 *   post-step steering angle / 0.5 and the actuator accelerations a_lon / 5, a_lat / 4
 *   (0 under GP_DYN_DIRECT).  With GP_DYN_JERK the reward's accelerations are those of the
 *   bicycle driven by the resolved (a_lon, steer).
 * Either pointer may be NULL.  on_host != 0: host memory, synchronous; else device
 * memory, asynchronous on `stream`.
 */
gp_status gp_get_rewards(gp_handle *h, float *reward, float *ego, int on_host, void *stream);
/*
 * Per-agent reward weights [n_agents][10] in the order collision, off-road, comfort,
 * alignment, centering, velocity, traffic light, time, reverse, overspeed (positive
 * magnitudes; defaults: the table's inference column 3, 3, 0.05, 0.025, 0.0038, 0.0025,
 * 1, 2.5e-5, 0.005, 0).  on_host as above.  gp_set_state resets the previous-step
 * accelerations to 0.
 */
gp_status gp_set_reward_weights(gp_handle *h, const float *weights, int on_host, void *stream);
/*
 * Copies the weights in use, float [n_agents][10] in the order above, into the caller's
 * buffer: those last set by gp_set_reward_weights, or with reward_conditioning the ones
 * drawn at each world's latest episode start.  on_host != 0: host memory, the call waits
 * for `stream`; else device memory, asynchronous on `stream`.  GP_EINVAL for a null handle
 * or buffer.
 */
gp_status gp_get_reward_weights(gp_handle *h, float *weights, int on_host, void *stream);

/*
 * Vectorized observations O_vec of every agent from the current state (App. A
 * "Observations"), one warp per agent.  Ego frame: x forward, y left.
 *   agents_dev  float [n_agents][GP_OBS_AGENTS][8]: the other boxes (agents and static
 *               boxes) within GP_OBS_AGENT_RADIUS, nearest first (ties to the lower index);
 *               slot = [1, x / R, y / R, L / 10, W / 5, cos dth, sin dth, (v_j - v_i) / 30]
 *   roads_dev   float [n_agents][GP_OBS_ROADS][8]: the centre lines of the road quads and
 *               lane-line strips (from the midpoint of the q0-q3 edge to that of q1-q2)
 *               with midpoint within GP_OBS_ROAD_RADIUS, nearest first (ties: roads before
 *               lines, then lower index), found through the world's spatial grid;
 *               slot = [1, x / R, y / R, length / R, cos dphi, sin dphi, 1[road], 1[line]]
 *   signals_dev float [n_agents][GP_OBS_SIGNALS][8]: the traffic-signal spheres with
 *               centre within GP_OBS_SIGNAL_RADIUS on the ground plane, nearest first
 *               (ties to the lower index); slot = [1, x / R, y / R, z / 10, 1[red],
 *               1[amber], 1[green], 1[off]] (traffic controls)
 * Unused slots are zero.  Any pointer may be NULL; all 16-byte aligned.  Asynchronous.
 */
gp_status gp_observe_vec(gp_handle *h, float *agents_dev, float *roads_dev, float *signals_dev,
                         void *stream);

/* Read (synchronously) / clear the device status word; set bits for tests.  The paper has
 * no counterpart: this is this library's device-side error reporting. */
gp_status gp_get_status(gp_handle *h, uint32_t *bits);
gp_status gp_clear_status(gp_handle *h);
gp_status gp_debug_inject_status(gp_handle *h, uint32_t bits);

/*
 * Failure-path test of the pipelined render kernel: launch it (with the handle's bands and
 * a pipelined launch shape) with producer warps that publish nothing, so every consumer's
 * first handoff wait runs out after wait_ns nanoseconds (1e6..2e9, else GP_EINVAL).  The
 * kernel then sets GP_DEV_PIPELINE_TIMEOUT in the status word and returns; nothing is
 * written to out_dev/depth_dev and the context stays usable.  Synchronous.  GP_ELIMIT if no
 * pipelined shape fits.  The paper has no counterpart; this is a test aid of this library.
 */
gp_status gp_debug_stall_pipeline(gp_handle *h, void *out_dev, void *depth_dev, int64_t wait_ns,
                                  void *stream);

/*
 * The paper has no counterpart: a parity aid of this library (the "identical snapped
 * vertices" comparison with the CPU oracle).
 * Render all cameras (like gp_render) and copy the snapped triangles that camera `view`
 * rasterised to host memory: records of int32 X[3], Y[3] (1/16 pixel, y down), float d[3]
 * (n / z_view), uint32 prim, uint32 sub (fan index after clipping); 44 bytes each.  A
 * triangle that spans several screen bands appears once per band.  *n receives the number
 * produced (records beyond cap are dropped).  Synchronous.
 */
gp_status gp_debug_dump_tris(gp_handle *h, int32_t view, void *out_dev, void *depth_dev,
                             void *host_tris, int64_t cap, int64_t *n, void *stream);

/*
 * Same result as gp_debug_dump_tris, but the call allocates no memory: its scratch (the
 * work counter, the record count and up to GP_NOALLOC_MAX_TRIS records, ~0.7 MB) lives in
 * one fixed device array inside the library, which every GPU that loads the library keeps
 * until the process exits.  This serves callers that cannot allocate device memory at
 * this point: a process whose caching allocator (PyTorch's, for example) already holds
 * nearly all free HBM, where a fresh cudaMalloc can fail although the caller's pool has
 * room, and hooks inside a running loop that cannot afford the device-wide
 * synchronisation that cudaMalloc/cudaFree imply.  The paper has no counterpart; this is
 * a debugging aid of this library.
 *  - cap must be at most GP_NOALLOC_MAX_TRIS, otherwise GP_ELIMIT (nothing is launched).
 *  - The array's device address is looked up (no allocation) when a handle is created on
 *    the device, and again at every later creation there, so it belongs to the context of
 *    the live handles; the call itself does no set-up.  Like every handle, it does not
 *    survive a cudaDeviceReset: create a new handle after one.
 *  - All calls share the one array (the counters are cleared at the start of every call;
 *    the records keep the last call's contents): calls that overlap on the GPU, from
 *    several threads or streams, race.  Synchronous, like gp_debug_dump_tris.
 */
#define GP_NOALLOC_MAX_TRIS 16384
gp_status gp_debug_dump_tris_noalloc(gp_handle *h, int32_t view, void *out_dev, void *depth_dev,
                                     void *host_tris, int64_t cap, int64_t *n, void *stream);

/* Description of the last error on the calling thread ("" if none).  No counterpart in the
 * paper. */
const char *gp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GIGAPIXEL_H */
