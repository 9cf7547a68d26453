/*
 * Seeded synthetic driving worlds: the input generator shared by the CUDA path's
 * tests/benchmarks and the CPU oracle.  It holds none of the simulator's arithmetic
 * (no dynamics, collision, projection or rasterisation); it only lays out a map and
 * boxes and draws actions.  The paper's scenes come from nuPlan logs, which are not
 * available here; these worlds stand in for them with the stated distributions.
 *
 * World (Sec. 3.1, App. A "High-Throughput Batched Rendering"): agent/static cuboids
 * plus flat road pieces and thin lane-line strips.  Road pieces and lane-line strips
 * are emitted as convex quads in world coordinates, corners counter-clockwise seen
 * from above (+z).
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood 2014) seeds one PCG32 stream per
 * world (O'Neill 2014, "PCG: a family of simple fast space-efficient statistically
 * good algorithms", XSH-RR output).  Actions come from a counter-based SplitMix64
 * hash of (seed, step, global agent id) so any step can be regenerated on its own.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define WG_PI 3.14159265358979323846

static uint64_t splitmix64_next(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t mix64(uint64_t z) {
    uint64_t s = z;
    return splitmix64_next(&s);
}

typedef struct {
    uint64_t state, inc;
} pcg32;

static uint32_t pcg32_next(pcg32 *r) {
    uint64_t old = r->state;
    r->state = old * 6364136223846793005ull + r->inc;
    uint32_t xorshifted = (uint32_t)(((old >> 18u) ^ old) >> 27u);
    uint32_t rot = (uint32_t)(old >> 59u);
    return (xorshifted >> rot) | (xorshifted << ((-rot) & 31));
}

static void pcg32_seed(pcg32 *r, uint64_t initstate, uint64_t initseq) {
    r->state = 0u;
    r->inc = (initseq << 1u) | 1u;
    pcg32_next(r);
    r->state += initstate;
    pcg32_next(r);
}

/* uniform double in [0, 1) with 53 random bits */
static double unif(pcg32 *r) {
    uint64_t hi = pcg32_next(r) >> 5;  /* 27 bits */
    uint64_t lo = pcg32_next(r) >> 6;  /* 26 bits */
    return (double)((hi << 26) | lo) * (1.0 / 9007199254740992.0);
}
static double unif_ab(pcg32 *r, double a, double b) { return a + (b - a) * unif(r); }
static uint32_t unif_int(pcg32 *r, uint32_t n) { return (uint32_t)(unif(r) * n); }

/* Generator parameters (all lengths in metres, angles in radians). */
typedef struct {
    double half_extent;     /* world is [-h, h]^2 */
    double lane_w;          /* lane width */
    int32_t n_lanes;        /* lanes per road */
    double line_w;          /* lane-line strip width */
    double seg_len_lo, seg_len_hi;
    double p_straight;
    double arc_r_lo, arc_r_hi;
    int32_t arc_pieces;
    int32_t chain_max;      /* max segments per chain */
    double box_l_lo, box_l_hi, box_w_lo, box_w_hi, box_h_lo, box_h_hi;
    double box_gap;         /* minimum gap between box footprints */
    double heading_jitter;  /* box heading = lane direction +- U[-j, j] */
    double v0_lo, v0_hi;    /* initial agent speed */
    int32_t max_tries;      /* rejection-sampling tries per box */
} wg_params;

void wg_default_params(wg_params *p) {
    p->half_extent = 100.0;
    p->lane_w = 3.5;
    p->n_lanes = 2;
    p->line_w = 0.15;
    p->seg_len_lo = 20.0;
    p->seg_len_hi = 60.0;
    p->p_straight = 0.5;
    p->arc_r_lo = 30.0;
    p->arc_r_hi = 150.0;
    p->arc_pieces = 4;
    p->chain_max = 16;
    p->box_l_lo = 4.0;  p->box_l_hi = 5.0;
    p->box_w_lo = 1.8;  p->box_w_hi = 2.0;
    p->box_h_lo = 1.4;  p->box_h_hi = 1.7;
    p->box_gap = 6.0;
    p->heading_jitter = 5.0 * WG_PI / 180.0;
    p->v0_lo = 0.0;
    p->v0_hi = 10.0;
    p->max_tries = 20000;
}

/* Upper bounds on the per-world outputs, so that callers can size buffers. */
int64_t wg_max_road_quads(const wg_params *p, int32_t n_segments) {
    return (int64_t)n_segments * (p->arc_pieces > 1 ? p->arc_pieces : 1);
}
int64_t wg_max_line_quads(const wg_params *p, int32_t n_segments) {
    return wg_max_road_quads(p, n_segments) * (p->n_lanes + 1);
}

/* A cross-section of the road: centre point and heading. */
typedef struct { double x, y, h; } xsec;

static void emit_strip(const xsec *a, const xsec *b, double off_lo, double off_hi, float *q) {
    /* Quad between lateral offsets off_lo < off_hi (measured along the left normal)
     * of two cross-sections; corners counter-clockwise seen from above. */
    double nax = -sin(a->h), nay = cos(a->h);
    double nbx = -sin(b->h), nby = cos(b->h);
    q[0] = (float)(a->x + off_lo * nax); q[1] = (float)(a->y + off_lo * nay);
    q[2] = (float)(b->x + off_lo * nbx); q[3] = (float)(b->y + off_lo * nby);
    q[4] = (float)(b->x + off_hi * nbx); q[5] = (float)(b->y + off_hi * nby);
    q[6] = (float)(a->x + off_hi * nax); q[7] = (float)(a->y + off_hi * nay);
}

/* Lane placement record for boxes: a piece between two cross-sections. */
typedef struct { xsec a, b; } piece;

/*
 * Generate one world.  Outputs (caller-allocated):
 *   boxes [n_boxes][7]  x, y, yaw, L, W, H, v0  (first n_agents boxes are agents;
 *                       static boxes get v0 = 0)
 *   road  [<= wg_max_road_quads][8]  road-surface quads
 *   line  [<= wg_max_line_quads][8]  lane-line strips (edges + lane dividers)
 *   pieces_scratch [<= wg_max_road_quads][6] doubles of scratch
 * Returns 0 on success, -1 if the boxes could not be placed.
 */
int wg_generate_world(const wg_params *p, uint64_t seed, int32_t world_index,
                      int32_t n_agents, int32_t n_boxes, int32_t n_segments,
                      float *boxes, float *road, int64_t *n_road, float *line, int64_t *n_line,
                      double *pieces_scratch) {
    uint64_t s = seed ^ (0x5851F42D4C957F2Dull * (uint64_t)(world_index + 1));
    uint64_t st = splitmix64_next(&s);
    uint64_t sq = splitmix64_next(&s);
    pcg32 rng;
    pcg32_seed(&rng, st, sq);

    const double H = p->half_extent;
    const double hw = 0.5 * p->n_lanes * p->lane_w;
    piece *pcs = (piece *)pieces_scratch;
    int64_t npc = 0, nr = 0, nl = 0;

    int32_t done = 0;
    while (done < n_segments) {
        xsec cur;
        cur.x = unif_ab(&rng, -H, H);
        cur.y = unif_ab(&rng, -H, H);
        cur.h = unif_ab(&rng, -WG_PI, WG_PI);
        int32_t chain_len = 1 + (int32_t)unif_int(&rng, (uint32_t)p->chain_max);
        for (int32_t k = 0; k < chain_len && done < n_segments; ++k) {
            int straight = unif(&rng) < p->p_straight;
            double len = unif_ab(&rng, p->seg_len_lo, p->seg_len_hi);
            int np = 1;
            double radius = 0.0, sgn = 1.0;
            if (!straight) {
                radius = unif_ab(&rng, p->arc_r_lo, p->arc_r_hi);
                sgn = unif(&rng) < 0.5 ? -1.0 : 1.0;
                np = p->arc_pieces;
            }
            /* centre of curvature for arcs */
            double qx = cur.x + sgn * radius * (-sin(cur.h));
            double qy = cur.y + sgn * radius * cos(cur.h);
            xsec a = cur;
            for (int i = 1; i <= np; ++i) {
                double t = len * (double)i / (double)np;
                xsec b;
                if (straight) {
                    b.x = cur.x + t * cos(cur.h);
                    b.y = cur.y + t * sin(cur.h);
                    b.h = cur.h;
                } else {
                    b.h = cur.h + sgn * t / radius;
                    b.x = qx + sgn * radius * sin(b.h);
                    b.y = qy - sgn * radius * cos(b.h);
                }
                emit_strip(&a, &b, -hw, hw, road + 8 * nr);
                ++nr;
                for (int l = 0; l <= p->n_lanes; ++l) {
                    double o = -hw + l * p->lane_w;
                    emit_strip(&a, &b, o - 0.5 * p->line_w, o + 0.5 * p->line_w, line + 8 * nl);
                    ++nl;
                }
                pcs[npc].a = a;
                pcs[npc].b = b;
                ++npc;
                a = b;
            }
            cur = a;
            cur.h = atan2(sin(cur.h), cos(cur.h));
            ++done;
            if (fabs(cur.x) > H || fabs(cur.y) > H) break; /* left the world: new chain */
        }
    }
    *n_road = nr;
    *n_line = nl;

    /* Boxes on lane centres, headings along the lane, rejection-sampled gaps. */
    int32_t placed = 0, tries = 0;
    while (placed < n_boxes) {
        if (++tries > p->max_tries * (n_boxes + 1)) return -1;
        const piece *pc = &pcs[unif_int(&rng, (uint32_t)npc)];
        double u = unif(&rng);
        int lane = (int)unif_int(&rng, (uint32_t)p->n_lanes);
        /* interpolate the piece's cross-sections (pieces are short; linear is fine) */
        double cx = pc->a.x + u * (pc->b.x - pc->a.x);
        double cy = pc->a.y + u * (pc->b.y - pc->a.y);
        double dh = atan2(sin(pc->b.h - pc->a.h), cos(pc->b.h - pc->a.h));
        double ch = pc->a.h + u * dh;
        double off = -hw + (lane + 0.5) * p->lane_w;
        cx += off * (-sin(ch));
        cy += off * cos(ch);
        /* right-hand traffic: lanes right of the centre line run along the piece */
        double heading = (off < 0.0) ? ch : ch + WG_PI;
        heading += unif_ab(&rng, -p->heading_jitter, p->heading_jitter);
        heading = atan2(sin(heading), cos(heading));
        double L = unif_ab(&rng, p->box_l_lo, p->box_l_hi);
        double Wd = unif_ab(&rng, p->box_w_lo, p->box_w_hi);
        double Hh = unif_ab(&rng, p->box_h_lo, p->box_h_hi);
        double r = 0.5 * sqrt(L * L + Wd * Wd);
        int ok = 1;
        for (int32_t j = 0; j < placed && ok; ++j) {
            const float *b = boxes + 7 * j;
            double rj = 0.5 * sqrt((double)b[3] * b[3] + (double)b[4] * b[4]);
            double dx = cx - b[0], dy = cy - b[1];
            double need = r + rj + p->box_gap;
            if (dx * dx + dy * dy < need * need) ok = 0;
        }
        if (!ok) continue;
        float *b = boxes + 7 * placed;
        b[0] = (float)cx; b[1] = (float)cy; b[2] = (float)heading;
        b[3] = (float)L;  b[4] = (float)Wd; b[5] = (float)Hh;
        b[6] = placed < n_agents ? (float)unif_ab(&rng, p->v0_lo, p->v0_hi) : 0.0f;
        ++placed;
    }
    return 0;
}

/*
 * Actions for agents [gid0, gid0 + n) at a step: accel ~ U[a_lo, a_hi] m/s^2,
 * steer ~ U[s_lo, s_hi] rad, out[n][2].  Counter-based, so any step can be
 * regenerated independently of the others.
 */
void wg_actions(uint64_t seed, int64_t step, int64_t gid0, int64_t n,
                double a_lo, double a_hi, double s_lo, double s_hi, float *out) {
    uint64_t ks = mix64(seed ^ 0xA0761D6478BD642Full);
    uint64_t kst = mix64(ks ^ (uint64_t)step);
    for (int64_t i = 0; i < n; ++i) {
        uint64_t k = mix64(kst ^ (uint64_t)(gid0 + i) * 0xE7037ED1A0B428DBull);
        double u1 = (double)(k >> 40) * (1.0 / 16777216.0);
        double u2 = (double)((k >> 16) & 0xFFFFFFull) * (1.0 / 16777216.0);
        out[2 * i + 0] = (float)(a_lo + (a_hi - a_lo) * u1);
        out[2 * i + 1] = (float)(s_lo + (s_hi - s_lo) * u2);
    }
}
