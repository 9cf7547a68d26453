// Render kernel: batched perspective rasterisation of bounding-box worlds.
//
// One work item = one screen band (full image width, band_rows rows) of one agent camera.
// Persistent CTAs pull items from a global counter.  Per item:
//   1. cull: per-world clusters of ground quads and the world's boxes are tested as
//      axis-aligned boxes against the band's frustum (left/right planes, near plane and the
//      band's pixel-centre rows; conservative by 1/16 px for snapping);
//   2. setup: warps pull units of 32 quads (the visible clusters' ground quads packed back
//      to back, or box faces) from a shared counter, with no block barrier between units.
//      Each lane transforms its quad's corners to view space and rejects a triangle if all
//      three vertices lie beyond one plane through the eye (near, guard band, or the band's
//      pixel-centre extent widened by 1/4 px); otherwise it projects, snaps to 1/16 px
//      (round half to even), back-face culls and keeps the triangle if its snapped bounding
//      box holds a pixel centre of the band.  A triangle crossing the near plane or the 4x
//      guard band is queued and later clipped by an 8-lane warp segment (Sutherland-Hodgman,
//      planes in the order near, left, right, bottom, top) and fan-triangulated.  A warp
//      reserves batch slots for its unit with one atomic; when the batch is full it is
//      rasterised and setup continues;
//   3. raster: kept triangles are expanded into (triangle, row) items, dealt out so that
//      one triangle's rows land in different warps; each item computes the exact covered
//      span of its row from the integer edge functions (top-left fill rule); a warp then
//      walks its spans' pixels -- with FP32 keys each lane its own span when the spans are
//      even, else 32 fragments at a time found by binary search over the spans' prefix
//      sums; with FP16 keys each lane one odd-length run of the concatenated fragments, the
//      spans' parameters read from a per-warp table -- and resolves depth per pixel in
//      shared memory with atomicMax on a key: (FP32 depth bits << 32 | ~prim), or
//      (binary16 depth << 16 | ~prim) in FP16 mode; the nearest surface wins, ties go to
//      the smaller primitive id;
//   4. encode: keys become class ids (uint8) + depth, a normalised one-hot BF16 NCHW
//      tensor, or shaded RGB; the band is one contiguous range of every output plane, written
//      with coalesced streaming stores: per lane 16 B of FP32 depth, 4 B of class ids (or of
//      each RGB channel), and with FP16 keys 16 B per one-hot channel and of binary16 depth
//      (8 pixels per lane when the width is a multiple of 8; else 8 B for 4 pixels).
// A pipelined variant splits the block into producer warps (steps 1-2) and consumer warps
// (steps 3-4) that hand double-buffered triangle batches to each other.
// The depth plane d = d0 + a (X - X0) + b (Y - Y0) and its per-pixel evaluation follow a
// fixed IEEE FP32 operation sequence (explicit _rn intrinsics), so identical snapped
// triangles give bit-identical keys on any implementation that follows the same sequence.
#include <algorithm>
#include <cmath>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "gp_internal.h"

namespace gpk {

namespace {

constexpr int kItemsPerThread = 8;  // raster items per thread per raster sub-pass
constexpr int kClipQueue = 256;     // queued clip jobs per block

// A triangle ready for raster.  The edge functions are rebuilt from the vertices per row;
// snapped coordinates stay within the 4x guard band, |X|, |Y| <= 5 * 8 * 512 < 2^15.
struct __align__(16) TriRec {
    int xy[3];      // snapped vertices, positive area (y down): X low 16 bits, Y high 16 bits
    uint32_t low;   // low half of the key: inverted primitive id
    float d0, a, b; // depth plane d0 + a (X - X0) + b (Y - Y0), per 1/16 px, origin vertex 0
    uint32_t span;  // pixel-centre bounds: i0 | i1 << 9 | (j0 - by0) << 18 | (j1 - j0) << 25
};
static_assert(sizeof(TriRec) == 32, "TriRec layout");
static_assert(kMaxBandRows <= 128, "(j0 - by0) and (j1 - j0) have 7 bits each");
static_assert(kMaxBandRows * GP_MAX_WIDTH <= 65536, "a band's key index fits 16 bits");

// A warp's non-empty spans, compacted (one 640-byte table per warp): the key index and the
// pixel offset of fragment f of the warp's concatenated spans are kb + f and gb + 16 f for
// the span holding f, which ends before fragment `end`.
struct __align__(16) FragEnt {
    uint32_t w0;     // kb + kKbBias (bits 0..16) | end (bits 17..31)
    int gb;          // pixel-centre offset (1/16 px) from vertex 0 of fragment 0 along this row
    float a, inner;  // depth plane along the row
};
constexpr int kKbBias = 1 << 14;  // kb = kofs - start > -2^14: a wave holds <= 2^14 fragments
static_assert(32 * GP_MAX_WIDTH <= (1 << 14), "a wave's fragment count fits 15 bits");
constexpr int kFragTabBytes = 32 * (sizeof(FragEnt) + 4);  // entries + inverted ids, per warp

__device__ __forceinline__ int span_i0(uint32_t s) { return (int)(s & 511u); }
__device__ __forceinline__ int span_i1(uint32_t s) { return (int)((s >> 9) & 511u); }
__device__ __forceinline__ int span_j0(uint32_t s) { return (int)((s >> 18) & 127u); }  // band-relative
__device__ __forceinline__ int span_nj(uint32_t s) { return (int)(s >> 25) + 1; }     // rows
__device__ __forceinline__ int vtx_x(int xy) { return (int)(short)(xy & 0xFFFF); }
__device__ __forceinline__ int vtx_y(int xy) { return xy >> 16; }

struct Cam {
    float px, py, s, c;  // camera position and yaw sin/cos
    int by0, by1;        // band rows, inclusive
    uint32_t box_end, road_end, line_end;
    int sig_begin;       // the world's first signal sphere
    int box_begin, ego, cl_begin;
    float gtx, gty;      // guard-band planes |x| <= gtx z, |y| <= gty z
    float vl, vt, vb;    // band edges widened by 1/4 px: |x| <= vl z, vb z <= y <= vt z
};

struct Smem {
    size_t keys, tris, rowoff, map, ftab, clipscratch, vq0, vpre, vnq, visbox, vissig, clipq, total;
};

// Traffic-signal polyhedron (4 latitude bands x 8 longitude sectors, vertices on the
// sphere): cos/sin of the latitudes -90..90 deg (poles exact) and longitudes 0..315 deg;
// per face q = 8 i + j the outward unit normal (xyz) and the plane's distance from the
// centre in radii (w).  Filled by render_configure.
__constant__ float c_lat_c[5], c_lat_s[5], c_lon_c[8], c_lon_s[8];
__constant__ float4 c_sig_face[kSignalQuads];

// Vertex (i, j) of a signal sphere (x, y, z, r); one rounding order for every caller, so
// the triangles of a face and their clipped pieces share exact corners.
__device__ __forceinline__ void sig_vertex(float4 sp, int i, int j, float &x, float &y, float &z) {
    const float rc = __fmul_rn(sp.w, c_lat_c[i]);
    x = __fadd_rn(sp.x, __fmul_rn(rc, c_lon_c[j & 7]));
    y = __fadd_rn(sp.y, __fmul_rn(rc, c_lon_s[j & 7]));
    z = __fadd_rn(sp.z, __fmul_rn(sp.w, c_lat_s[i]));
}

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Shared memory of a block.  In the one-phase-at-a-time kernel the raster bookkeeping
// (rowoff, map) and the clip scratch are live in different phases and share one region; the
// pipelined kernel (prod_warps > 0) keeps them apart and double-buffers the batch.
__host__ __device__ inline Smem smem_layout(int W, int band_rows, int key_f16, int threads,
                                            int tri_cap, int max_cl, int prod_warps) {
    Smem s;
    size_t o = 0;
    s.keys = o;
    o += (size_t)W * band_rows * (key_f16 ? 4 : 8);
    o = align_up(o, 16);
    s.tris = o;
    o += (size_t)(prod_warps ? 2 : 1) * tri_cap * sizeof(TriRec);
    const size_t shared_base = o;
    const int raster_threads = threads - 32 * prod_warps;
    const int clip_warps = prod_warps ? prod_warps : threads / 32;
    s.rowoff = o;
    o += (size_t)(tri_cap + 1) * 4;
    o = align_up(o, 16);
    s.map = o;
    o += (size_t)raster_threads * kItemsPerThread * 2;
    o = align_up(o, 16);
    s.ftab = o;  // the raster warps' span tables (FP16 keys only)
    if (key_f16) o += (size_t)(raster_threads / 32) * kFragTabBytes;
    // per clipping warp: 4 jobs x 8 vertices x 3 floats; shares space with the raster
    // bookkeeping unless both sides run at once (pipelined kernel)
    s.clipscratch = prod_warps ? o : shared_base;
    const size_t clip_end = s.clipscratch + (size_t)clip_warps * 4 * 24 * 4;
    o = clip_end > o ? clip_end : o;
    o = align_up(o, 16);
    s.vq0 = o;  // first quad of each visible cluster
    o += (size_t)max_cl * 4;
    s.vpre = o;  // visible quads before it (exclusive prefix of the counts)
    o += (size_t)max_cl * 4;
    s.vnq = o;  // its quad count
    o += (size_t)max_cl;
    s.visbox = o;
    o += kMaxBoxes;
    s.vissig = o;
    o += kMaxSignals;
    o = align_up(o, 16);
    s.clipq = o;
    o += (size_t)kClipQueue * 4;
    s.total = align_up(o, 16);
    return s;
}

__device__ __forceinline__ float3 to_view(const RenderParams &p, const Cam &cm, float x, float y,
                                          float z) {
    const float dx = __fsub_rn(x, cm.px), dy = __fsub_rn(y, cm.py);
    return make_float3(__fsub_rn(__fmul_rn(dx, cm.s), __fmul_rn(dy, cm.c)), __fsub_rn(z, p.cam_h),
                       __fadd_rn(__fmul_rn(dx, cm.c), __fmul_rn(dy, cm.s)));
}

// Clip-plane values, inside >= 0: near, left, right, bottom, top.
__device__ __forceinline__ float plane_dist(const RenderParams &p, int k, float x, float y,
                                            float z) {
    const float gx = __fmul_rn(__fmul_rn(p.guard, p.tx), z);
    const float gy = __fmul_rn(__fmul_rn(p.guard, p.ty), z);
    switch (k) {
    case 0: return __fsub_rn(z, p.near_plane);
    case 1: return __fadd_rn(x, gx);
    case 2: return __fsub_rn(gx, x);
    case 3: return __fadd_rn(y, gy);
    default: return __fsub_rn(gy, y);
    }
}

// Outcode bits: 0 near, 1-4 guard band (left, right, bottom, top) -- the clip planes --
// and 5-8 the band's pixel-centre extent widened by 1/4 px (left, right, top, bottom).  All
// planes pass through the eye, so a triangle with every vertex beyond one plane has no
// visible part on the inner side.
__device__ __forceinline__ int outcode(const RenderParams &p, const Cam &cm, float x, float y,
                                       float z) {
    int oc = (z < p.near_plane) ? 1 : 0;
    const float gx = cm.gtx * z, gy = cm.gty * z;
    oc |= (x < -gx) ? 2 : 0;
    oc |= (x > gx) ? 4 : 0;
    oc |= (y < -gy) ? 8 : 0;
    oc |= (y > gy) ? 16 : 0;
    const float vx = cm.vl * z;
    oc |= (x < -vx) ? 32 : 0;
    oc |= (x > vx) ? 64 : 0;
    oc |= (y > cm.vt * z) ? 128 : 0;
    oc |= (y < cm.vb * z) ? 256 : 0;
    return oc;
}

// Projection and 1/16-px snap (round half to even) with one reciprocal per vertex; also
// the vertex's reversed-Z depth n / z.
__device__ __forceinline__ void project(const RenderParams &p, float x, float y, float z, int &X,
                                        int &Y, float &d) {
    const float r = __fdividef(1.f, z);
    const float f16 = 16.f * p.f;
    X = __float2int_rn(__fmaf_rn(f16, __fmul_rn(x, r), 8.f * (float)p.W));
    Y = __float2int_rn(__fmaf_rn(-f16, __fmul_rn(y, r), 8.f * (float)p.H));
    d = __fmul_rn(p.near_plane, r);
}

// Box corner k: x = +-L/2 (bit 0), y = +-W/2 (bit 1), z = 0 or H (bit 2).
__device__ __forceinline__ void box_corner(float4 pose, float4 dim, float s, float c, int k,
                                           float &x, float &y, float &z) {
    const float lx = (k & 1) ? 0.5f * dim.x : -0.5f * dim.x;
    const float ly = (k & 2) ? 0.5f * dim.y : -0.5f * dim.y;
    x = pose.x + (c * lx - s * ly);
    y = pose.y + (s * lx + c * ly);
    z = (k & 4) ? dim.z : 0.f;
}

// Face triangles (corner indices), counter-clockwise seen from outside; faces +x, -x, +y,
// -y, +z, -z, each quad (q0 q1 q2 q3) split into (q0 q1 q2), (q0 q2 q3).
__device__ __forceinline__ void box_tri(int t, int &a, int &b, int &c) {
    // packed 4-bit corner ids per face (q0 q1 q2 q3), faces 0..3 in one word, 4..5 in another
    const int face = t >> 1;
    const unsigned int f = face < 4 ? (unsigned int)(0x0154267304621375ull >> (16 * face)) & 0xFFFFu
                                    : (0x02314576u >> (16 * (face - 4))) & 0xFFFFu;
    const int q0 = (f >> 12) & 15, q1 = (f >> 8) & 15, q2 = (f >> 4) & 15, q3 = f & 15;
    a = q0;
    b = (t & 1) ? q2 : q1;
    c = (t & 1) ? q3 : q2;
}

// a * b + c in 32-bit two's-complement wrap-around (exact whenever the true result fits).
__device__ __forceinline__ unsigned int wrap_mul_add(int a, int b, unsigned int c) {
    return (unsigned int)a * (unsigned int)b + c;
}

// Build a raster record from a front-facing snapped triangle (area2 < 0 in y-down space)
// with pixel-centre bounds i0..i1, j0..j1 (j within the band starting at row by0).
__device__ __forceinline__ void build_rec(TriRec &r, const int X[3], const int Y[3], const float d[3],
                                          uint32_t prim, int key_f16, int i0, int i1, int j0,
                                          int j1, int by0) {
    // orient to positive area: keep vertex 0, swap 1 and 2
    const int vx[3] = {X[0], X[2], X[1]};
    const int vy[3] = {Y[0], Y[2], Y[1]};
    const float dv[3] = {d[0], d[2], d[1]};
#pragma unroll
    for (int k = 0; k < 3; ++k) r.xy[k] = (vx[k] & 0xFFFF) | (vy[k] << 16);
    const float fx1 = (float)(vx[1] - vx[0]), fy1 = (float)(vy[1] - vy[0]);
    const float fx2 = (float)(vx[2] - vx[0]), fy2 = (float)(vy[2] - vy[0]);
    const int area2 = (int)(wrap_mul_add(vx[1] - vx[0], vy[2] - vy[0], 0u) -
                            wrap_mul_add(vx[2] - vx[0], vy[1] - vy[0], 0u));
    const float e1 = __fsub_rn(dv[1], dv[0]), e2 = __fsub_rn(dv[2], dv[0]);
    const float fa = __int2float_rn(area2);
    const float na = __fsub_rn(__fmul_rn(e1, fy2), __fmul_rn(e2, fy1));
    const float nb = __fsub_rn(__fmul_rn(e2, fx1), __fmul_rn(e1, fx2));
    r.a = __fdiv_rn(na, fa);
    r.b = __fdiv_rn(nb, fa);
    r.d0 = dv[0];
    r.low = key_f16 ? (0xFFFFu - (prim & 0xFFFFu)) : (0xFFFFFFFFu - prim);
    r.span = (uint32_t)i0 | ((uint32_t)i1 << 9) | ((uint32_t)(j0 - by0) << 18) |
             ((uint32_t)(j1 - j0) << 25);
}

// Snapped triangle -> keep? (front-facing, bbox holds a pixel centre of the band).
__device__ __forceinline__ bool tri_bbox(const RenderParams &p, const Cam &cm, const int X[3],
                                         const int Y[3], int &i0, int &i1, int &j0, int &j1) {
    const int area2 = (int)(wrap_mul_add(X[1] - X[0], Y[2] - Y[0], 0u) -
                            wrap_mul_add(X[2] - X[0], Y[1] - Y[0], 0u));
    if (area2 >= 0) return false;
    const int mnx = min(X[0], min(X[1], X[2])), mxx = max(X[0], max(X[1], X[2]));
    const int mny = min(Y[0], min(Y[1], Y[2])), mxy = max(Y[0], max(Y[1], Y[2]));
    i0 = max((mnx + 7) >> 4, 0);
    i1 = min((mxx - 8) >> 4, p.W - 1);
    j0 = max((mny + 7) >> 4, cm.by0);
    j1 = min((mxy - 8) >> 4, cm.by1);
    return i0 <= i1 && j0 <= j1;
}

__device__ __forceinline__ void dump_tri(const RenderParams &p, const int X[3], const int Y[3],
                                         const float d[3], uint32_t prim, uint32_t sub) {
    const int k = atomicAdd(p.dump_count, 1);
    if (k < p.dump_cap) {
        DumpTri &t = p.dump[k];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            t.X[i] = X[i];
            t.Y[i] = Y[i];
            t.d[i] = d[i];
        }
        t.prim = prim;
        t.sub = sub;
    }
}

// Is an axis-aligned box (xy centre/half extents, z range) possibly visible in the band?
__device__ bool aabb_visible(const RenderParams &p, const Cam &cm, float cx, float cy, float hx,
                             float hy, float zlo, float zhi) {
    const float dx = cx - cm.px, dy = cy - cm.py;
    const float as = fabsf(cm.s), ac = fabsf(cm.c);
    const float zc = dx * cm.c + dy * cm.s, ze = hx * ac + hy * as;
    const float zmax = zc + ze;
    if (zmax < p.near_plane) return false;
    const float zmin = fmaxf(zc - ze, p.near_plane);
    const float xc = dx * cm.s - dy * cm.c;
    // left plane x + tx z >= 0 and right plane tx z - x >= 0 (viewport, not guard band)
    const float lv = xc + p.tx * zc + hx * fabsf(cm.s + p.tx * cm.c) + hy * fabsf(p.tx * cm.s - cm.c);
    const float rv = p.tx * zc - xc + hx * fabsf(p.tx * cm.c - cm.s) + hy * fabsf(p.tx * cm.s + cm.c);
    if (lv < 0.f || rv < 0.f) return false;
    // rows: y_px = H/2 - f y / z over y in [zlo - h, zhi - h], z in [zmin, zmax]
    const float ylo = zlo - p.cam_h, yhi = zhi - p.cam_h;
    const float hh = 0.5f * (float)p.H;
    const float ymax = hh - p.f * ylo / (ylo < 0.f ? zmin : zmax);
    const float ymin = hh - p.f * yhi / (yhi > 0.f ? zmin : zmax);
    const float margin = 0.0625f + 1e-5f * fmaxf(fabsf(ymin), fabsf(ymax));
    const float jlo = ceilf(ymin - 0.5f - margin), jhi = floorf(ymax - 0.5f + margin);
    return fmaxf(jlo, (float)cm.by0) <= fminf(jhi, (float)cm.by1);
}

// FP16 mode key: binary16 depth bits above the inverted primitive id.
__device__ __forceinline__ unsigned int key16(float d, uint32_t low) {
    return ((unsigned int)__half_as_ushort(__float2half_rn(d)) << 16) | low;
}

// Raster items of a triangle: one per row of its bounding box (none for an empty slot,
// whose i1 < i0).
__device__ __forceinline__ int tri_items(uint32_t s) {
    return span_i1(s) < span_i0(s) ? 0 : span_nj(s);
}

// Exact covered span of one row of a triangle within columns [lo, hi] (narrowed in place;
// empty if lo > hi afterwards).  Edge k runs from vertex a = k to b = k + 1; its function
// at pixel centre (16 i + 8, py) is E = A (16 i + 8 - X_a) + B (py - Y_a) - bias with
// A = Y_a - Y_b, B = X_b - X_a, and bias 0 on a top or left edge, else 1 (top-left fill
// rule); the pixel is covered if E >= 0 on all three edges.  An edge with A > 0 bounds the
// span from below (smallest i with E >= 0), one with A < 0 from above; the latter is the
// former in the mirrored frame i -> -i, X_a -> 16 - X_a, so every edge runs the same
// instructions (no divergence between the lanes of a warp).  The crossing is estimated in
// float (within one pixel wherever it matters) and fixed by one exact integer check on each
// side.  A horizontal edge (A = 0) keeps or empties the whole row.
__device__ __forceinline__ void row_span(const TriRec &T, int row, int &lo, int &hi) {
    const int py = 16 * row + 8;
    int vx[3], vy[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        vx[k] = vtx_x(T.xy[k]);
        vy[k] = vtx_y(T.xy[k]);
    }
    int L = lo, U = hi;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int xa = vx[k], ya = vy[k], xb = vx[(k + 1) % 3], yb = vy[(k + 1) % 3];
        const int A = ya - yb, B = xb - xa;
        const bool top_left = A > 0 || (A == 0 && B > 0);
        const int R = (int)wrap_mul_add(B, py - ya, top_left ? 0u : 0xFFFFFFFFu);
        const bool up = A < 0;
        const int Am = up ? -A : A;
        const int xm = up ? 16 - xa : xa;
        const int lm = up ? -U : L, hm = up ? -L : U;
        // smallest i in [lm, hm + 1] with Am (16 i + 8 - xm) + R >= 0
        const float q = ((float)(xm - 8) - __fdividef((float)R, (float)Am)) * 0.0625f;
        int c = __float2int_ru(fminf(fmaxf(q, -1e6f), 1e6f));
        c = min(max(c, lm), hm + 1);
        const int e = (int)wrap_mul_add(Am, 16 * c + 8 - xm, (unsigned int)R);  // E at c
        const int em = e - 16 * Am;                                            // E at c - 1
        c = (c > lm && em >= 0) ? c - 1 : ((c <= hm && e < 0) ? c + 1 : c);
        if (A == 0) c = R >= 0 ? lm : hm + 1;
        if (up) U = min(U, -c);
        else L = max(L, c);
    }
    lo = L;
    hi = U;
}

// Depth test of one fragment: the key's maximum wins per pixel -- FP32 mode one 64-bit key
// (FP32 depth bits << 32 | inverted id), FP16 mode one 32-bit key (binary16 depth bits << 16
// | inverted id) -- so the nearest surface wins and ties go to the smaller primitive id.  The
// shared-memory atomic is issued unconditionally (its result is unused): reading the key
// first to skip losing fragments cost about 2 % more time.
// Depth is a * g + inner, clamped to >= 0, g the pixel centre's offset (1/16 px) from the
// triangle's vertex 0.
template <bool F32>
__device__ __forceinline__ void depth_test(void *keys, int ko, int g, float a, float inner,
                                           uint32_t low) {
    float d = __fmaf_rn(a, (float)g, inner);
    d = d > 0.f ? d : 0.f;
    if (F32) {
        unsigned long long *rk = (unsigned long long *)keys + ko;
        const unsigned long long key = ((unsigned long long)__float_as_uint(d) << 32) | low;
        atomicMax(rk, key);
    } else {
        unsigned int *rk = (unsigned int *)keys + ko;
        const unsigned int key = key16(d, low);
        atomicMax(rk, key);
    }
}

// Relative cost of one cooperative round (32 fragments) against one per-lane iteration:
// 64-bit key updates favour the cooperative walk.
constexpr int kCoopCostF32 = 1;

// Depth resolution of a warp's spans with FP32 keys (warp-uniform call).  Lane k brings a
// span of `cnt` pixels starting at key index `kofs`, whose first pixel centre lies gx0
// (1/16 px) right of the triangle's vertex 0.  If the spans are even, each lane walks its
// own span; if a few long spans dominate, the warp scans the counts and walks the
// concatenated fragments 32 at a time, each lane finding its span by binary search over the
// prefix sums, so the cost follows the number of fragments rather than the longest span.
// Consecutive lanes take consecutive fragments, so the 64-bit key atomics of a round land
// on adjacent keys (distinct banks); this walk needs no shared table, which the FP32 key
// buffer leaves no room for.
__device__ __forceinline__ void warp_fragments_coop(int cnt, int kofs, int gx0, float a,
                                                    float inner, uint32_t low, void *keys) {
    const int lane = threadIdx.x & 31;
    const int maxc = __reduce_max_sync(0xffffffffu, cnt);
    const int total = __reduce_add_sync(0xffffffffu, cnt);
    if (maxc <= ((total + 31) >> 5) * kCoopCostF32) {
        for (int t = 0; t < cnt; ++t) depth_test<true>(keys, kofs + t, gx0 + 16 * t, a, inner, low);
        return;
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    // key index and pixel offset in one word: kofs < band rows x W <= 2^16, |gx0| < 2^15
    const int kg = (int)(((unsigned int)gx0 << 16) | ((unsigned int)kofs & 0xFFFFu));
    // Each lane finds the first lane whose inclusive prefix exceeds its fragment index f by
    // binary search; the last probe that moved the search right holds that lane's exclusive
    // prefix (0 if none did).  Two rounds per iteration (independent searches overlap their
    // shuffle latency), then at most one single round for a tail of up to 32 fragments.
    int f0 = 0;
    for (; f0 + 32 < total; f0 += 64) {
        const int fA = f0 + lane, fB = fA + 32;
        int oA = 0, oB = 0, eA = 0, eB = 0;
#pragma unroll
        for (int st = 16; st > 0; st >>= 1) {
            const int vA = __shfl_sync(0xffffffffu, incl, oA + st - 1);
            const int vB = __shfl_sync(0xffffffffu, incl, oB + st - 1);
            if (vA <= fA) {
                oA += st;
                eA = vA;
            }
            if (vB <= fB) {
                oB += st;
                eB = vB;
            }
        }
        const int tA = fA - eA, tB = fB - eB;
        const int kgA = __shfl_sync(0xffffffffu, kg, oA);
        const int kgB = __shfl_sync(0xffffffffu, kg, oB);
        const float aA = __shfl_sync(0xffffffffu, a, oA), aB = __shfl_sync(0xffffffffu, a, oB);
        const float iA = __shfl_sync(0xffffffffu, inner, oA);
        const float iB = __shfl_sync(0xffffffffu, inner, oB);
        const uint32_t lA = __shfl_sync(0xffffffffu, low, oA);
        const uint32_t lB = __shfl_sync(0xffffffffu, low, oB);
        // fA < total here
        depth_test<true>(keys, (kgA & 0xFFFF) + tA, (kgA >> 16) + 16 * tA, aA, iA, lA);
        if (fB < total)
            depth_test<true>(keys, (kgB & 0xFFFF) + tB, (kgB >> 16) + 16 * tB, aB, iB, lB);
    }
    if (f0 < total) {
        const int f = f0 + lane;
        int o = 0, e = 0;
#pragma unroll
        for (int st = 16; st > 0; st >>= 1) {
            const int v = __shfl_sync(0xffffffffu, incl, o + st - 1);
            if (v <= f) {
                o += st;
                e = v;
            }
        }
        const int t = f - e;
        const int kgo = __shfl_sync(0xffffffffu, kg, o);
        const float fa = __shfl_sync(0xffffffffu, a, o);
        const float fi = __shfl_sync(0xffffffffu, inner, o);
        const uint32_t lw = __shfl_sync(0xffffffffu, low, o);
        if (f < total) depth_test<true>(keys, (kgo & 0xFFFF) + t, (kgo >> 16) + 16 * t, fa, fi, lw);
    }
}

// Depth resolution of a warp's spans with FP16 keys (warp-uniform call), arguments as for
// warp_fragments_coop plus the warp's span table.  The warp concatenates its spans (prefix
// sums) and cuts the fragments into 32 runs of equal, odd length, one per lane: each lane
// walks its run pixel by pixel and moves to the next span from the table when it crosses
// one, so the cost follows the number of fragments, not the longest span, with no search
// per fragment.  The odd run length puts the lanes that share one long span on different
// shared-memory banks at every step.
__device__ __forceinline__ void warp_fragments_runs(int cnt, int kofs, int gx0, float a,
                                                    float inner, uint32_t low, void *keys,
                                                    FragEnt *ent, uint32_t *lows) {
    const int lane = threadIdx.x & 31;
    const unsigned int nz = __ballot_sync(0xffffffffu, cnt > 0);
    if (!nz) return;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (cnt > 0) {
        const int k = __popc(nz & ((1u << lane) - 1u));
        const int start = incl - cnt;
        ent[k] = FragEnt{(uint32_t)(kofs - start + kKbBias) | ((uint32_t)incl << 17), gx0 - 16 * start,
                         a, inner};
        lows[k] = low;
    }
    __syncwarp();
    const int L = ((total + 31) >> 5) | 1;
    int f = lane * L;
    // the lane holding fragment f: the number of inclusive prefixes <= f (f < total)
    int o = 0;
#pragma unroll
    for (int st = 16; st > 0; st >>= 1) {
        const int v = __shfl_sync(0xffffffffu, incl, o + st - 1);
        if (v <= f) o += st;
    }
    if (f < total) {
        const int fe = min(f + L, total);
        int k = __popc(nz & ((1u << o) - 1u));
        FragEnt e = ent[k];
        uint32_t lw = lows[k];
        int end = (int)(e.w0 >> 17), kb = (int)(e.w0 & 0x1FFFFu) - kKbBias;
        for (; f < fe; ++f) {
            if (f == end) {
                ++k;
                e = ent[k];
                lw = lows[k];
                end = (int)(e.w0 >> 17);
                kb = (int)(e.w0 & 0x1FFFFu) - kKbBias;
            }
            depth_test<false>(keys, kb + f, e.gb + 16 * f, e.a, e.inner, lw);
        }
    }
    __syncwarp();  // the next wave rewrites the table
}

// Warp-aggregated append: returns this lane's slot (valid where keep is true).
__device__ __forceinline__ int warp_append(bool keep, int *counter) {
    const unsigned int lane = threadIdx.x & 31;
    const unsigned int m = __ballot_sync(0xffffffffu, keep);
    int base = 0;
    if (lane == 0 && m) base = atomicAdd(counter, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    return base + __popc(m & ((1u << lane) - 1u));
}

// Consecutive warps of the block that synchronise among themselves on one hardware
// barrier: the whole block (barrier 0), or one side of the pipelined kernel.
struct Group {
    int tid, nt, bar;  // thread index within the group, group size (multiple of 32), barrier id
    __device__ __forceinline__ int warp() const { return tid >> 5; }
    __device__ __forceinline__ int nw() const { return nt >> 5; }
    // The barrier instruction requires each warp to arrive converged: for a named barrier,
    // reconverge first and use the compiler's barrier intrinsic, which keeps it converged.
    __device__ __forceinline__ void sync() const {
        if (bar == 0) {
            __syncthreads();
        } else {
            __syncwarp();
            __barrier_sync_count((unsigned)bar, (unsigned)nt);
        }
    }
};

// Group-wide exclusive scan of per-thread sums (all group threads call; returns own prefix).
__device__ __forceinline__ int group_exclusive_scan(int v, int *s_warp, int &total, const Group &g) {
    const int lane = g.tid & 31, warp = g.warp(), nw = g.nw();
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    g.sync();
    if (warp == 0) {
        int w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) s_warp[lane] = w;  // inclusive prefix of warp totals
    }
    g.sync();
    total = s_warp[nw - 1];
    const int before = warp > 0 ? s_warp[warp - 1] : 0;
    g.sync();
    return before + x - v;
}

// Group-wide exclusive max-scan of per-thread values (0 for thread 0).
__device__ __forceinline__ int group_exclusive_max(int v, int *s_warp, const Group &g) {
    const int lane = g.tid & 31, warp = g.warp(), nw = g.nw();
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x = max(x, y);
    }
    if (lane == 31) s_warp[warp] = x;
    g.sync();
    if (warp == 0) {
        int w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w = max(w, y);
        }
        if (lane < nw) s_warp[lane] = w;
    }
    g.sync();
    const int prev_lane = __shfl_up_sync(0xffffffffu, x, 1);
    const int before_warp = warp > 0 ? s_warp[warp - 1] : 0;
    g.sync();
    return lane > 0 ? max(before_warp, prev_lane) : before_warp;
}

// Block state of the setup side (the whole block, or the producer warps).
struct Shared {
    int item, resv, next_unit, npend, nvcl, nvbox, nvsig, cq_n, nvq;
};

// Rasterise a batch of n triangles into the key buffer of the band of rows by0..by1 (all
// threads of group g call; ends with a group barrier).
template <bool F32, bool ST>
__device__ void flush(const RenderParams &p, int by0, int by1, int n, void *keys, TriRec *tris,
                      int *rowoff, unsigned short *map, unsigned char *ftab, int *s_warp,
                      const Group &g) {
    n = min(n, p.tri_cap);
    const int tid = g.tid, nt = g.nt;
    // row counts -> exclusive scan (each thread owns a contiguous slice of triangles)
    const int per = (n + nt - 1) / nt;
    const int t0 = min(tid * per, n), t1 = min(t0 + per, n);
    int local = 0;
    for (int t = t0; t < t1; ++t) local += tri_items(tris[t].span);
    int total = 0;
    int run = group_exclusive_scan(local, s_warp, total, g);
    for (int t = t0; t < t1; ++t) {
        rowoff[t] = run;
        run += tri_items(tris[t].span);
    }
    if (tid == 0) {
        rowoff[n] = total;
        if (ST && p.stats) {
            atomicAdd(&p.stats[GP_STAT_BATCHES], 1ull);
            atomicAdd(&p.stats[GP_STAT_ROW_ITEMS], (unsigned long long)total);
        }
    }
    g.sync();

    const int chunk = nt * kItemsPerThread;
    for (int start = 0; start < total; start += chunk) {
        const int len = min(chunk, total - start);
        for (int i = tid; i < len; i += nt) map[i] = 0;
        g.sync();
        for (int t = tid; t < n; t += nt) {
            const int o = rowoff[t], c = rowoff[t + 1] - o;
            if (c > 0) {
                if (o >= start && o < start + len) map[o - start] = (unsigned short)t;
                else if (o < start && o + c > start) map[0] = (unsigned short)t;
            }
        }
        g.sync();
        // max-scan of the head map: every item gets the triangle it belongs to (heads are
        // increasing with position, so the running maximum is the latest head)
        const int m0 = tid * kItemsPerThread;
        int own = 0;
#pragma unroll
        for (int k = 0; k < kItemsPerThread; ++k)
            if (m0 + k < len) own = max(own, (int)map[m0 + k]);
        int cur = group_exclusive_max(own, s_warp, g);
#pragma unroll
        for (int k = 0; k < kItemsPerThread; ++k) {
            if (m0 + k < len) {
                cur = max(cur, (int)map[m0 + k]);
                map[m0 + k] = (unsigned short)cur;
            }
        }
        g.sync();
        // Consecutive items (the rows of one triangle) go to different warps, so a large
        // triangle is spread over the block instead of holding up one warp.  The warp order
        // is rotated per group of lanes so that a warp's 32 reads of the map fall on distinct
        // banks (lane l reads entry l nw + its rotated warp index).
        const int nw = nt >> 5, lane = tid & 31;
        const int mine = lane * nw + ((tid >> 5) + 2 * ((lane * nw) >> 6)) % nw;
        FragEnt *ent = (FragEnt *)(ftab + (size_t)(tid >> 5) * kFragTabBytes);
        uint32_t *lows = (uint32_t *)(ent + 32);
        for (int ib = 0; ib < len; ib += nt) {  // warp-uniform trip count
            const int i = ib + mine;
            int cnt = 0, kofs = 0, gx0 = 0;
            float a = 0.f, inner = 0.f;
            uint32_t low = 0;
            if (i < len) {
                const int t = map[i];
                const TriRec &T = tris[t];
                const uint32_t sp = T.span;
                const int row = by0 + span_j0(sp) + (start + i - rowoff[t]);
                int lo = span_i0(sp), hi = span_i1(sp);
                if (row >= by0 && row <= by1 && lo >= 0 && hi < p.W) {
                    row_span(T, row, lo, hi);
                    if (lo <= hi) {
                        const int X0 = vtx_x(T.xy[0]), Y0 = vtx_y(T.xy[0]);
                        cnt = hi - lo + 1;
                        kofs = (row - by0) * p.W + lo;
                        gx0 = 16 * lo + 8 - X0;
                        a = T.a;
                        inner = __fmaf_rn(T.b, (float)(16 * row + 8 - Y0), T.d0);
                        low = T.low;
                    }
                }
            }
            if (ST && p.stats) {
                const int fr = __reduce_add_sync(0xffffffffu, cnt);
                if ((tid & 31) == 0 && fr)
                    atomicAdd(&p.stats[GP_STAT_FRAGMENTS], (unsigned long long)fr);
            }
            if (F32) warp_fragments_coop(cnt, kofs, gx0, a, inner, low, keys);
            else warp_fragments_runs(cnt, kofs, gx0, a, inner, low, keys, ent, lows);
        }
        g.sync();
    }
}

// World-space vertices and primitive id of a source triangle.
//   code bit 31 set: box triangle, bits 4..11 local box index, bits 0..3 face triangle
//   code bit 30 set: signal triangle, bits 6..10 local signal index, bits 0..5 2 q + t
//   otherwise: quad (cluster order) << 1 | triangle
__device__ __forceinline__ void source_tri(const RenderParams &p, const Cam &cm, uint32_t code,
                                           float vx[3], float vy[3], float vz[3],
                                           uint32_t &prim) {
    if (code & 0x80000000u) {
        const int b = (code >> 4) & 0xFF, t = code & 15;
        const float4 pose = p.box_pose[cm.box_begin + b];
        const float4 dim = p.box_dim[cm.box_begin + b];
        float s, c;
        sincosf(pose.z, &s, &c);
        int k[3];
        box_tri(t, k[0], k[1], k[2]);
#pragma unroll
        for (int i = 0; i < 3; ++i) box_corner(pose, dim, s, c, k[i], vx[i], vy[i], vz[i]);
        prim = 12u * b + t;
    } else if (code & 0x40000000u) {
        const int sg = (code >> 6) & 31, q = (code >> 1) & 31, t = code & 1;
        const float4 sp = p.sig[cm.sig_begin + sg];
        const int i = q >> 3, j = q & 7;
        // quad corners (i, j) (i, j+1) (i+1, j+1) (i+1, j); triangles (0 1 2), (0 2 3)
        sig_vertex(sp, i, j, vx[0], vy[0], vz[0]);
        sig_vertex(sp, t ? i + 1 : i, j + 1, vx[1], vy[1], vz[1]);
        sig_vertex(sp, i + 1, t ? j : j + 1, vx[2], vy[2], vz[2]);
        prim = cm.line_end + 64u * sg + 2u * q + t;
    } else {
        const int q = code >> 1, t = code & 1;
        const float4 g0 = p.quad_geo[2 * q], g1 = p.quad_geo[2 * q + 1];
        const uint32_t base = p.quad_prim[q];
        const float z = base < cm.road_end ? 0.f : p.line_z;
        vx[0] = g0.x;
        vy[0] = g0.y;
        vx[1] = t ? g1.x : g0.z;
        vy[1] = t ? g1.y : g0.w;
        vx[2] = t ? g1.z : g1.x;
        vy[2] = t ? g1.w : g1.y;
        vz[0] = vz[1] = vz[2] = z;
        prim = base + t;
    }
}

// A batch slot that holds no triangle (zero rows).
__device__ __forceinline__ void empty_rec(TriRec &r) { r.span = 1u; }  // i0 = 1 > i1 = 0

// Clip queued triangles cooperatively: an 8-lane segment per job (4 jobs per warp), one
// polygon vertex per lane.  For every plane the triangle crosses (near, then guard left,
// right, bottom, top; planes no vertex lies beyond cannot change it), each lane emits its
// vertex if inside and the crossing point of its edge to the next vertex if the edge
// crosses (interpolated from the inside vertex), in edge order -- Sutherland-Hodgman --
// and the segment compacts the outputs through shared scratch.  The polygon is then
// fan-triangulated from its first vertex, one fan triangle per lane, into slots[6 j ..).
// Called by all threads of group grp for jobs [0, njobs) of `jobs`.
template <bool ST>
__device__ void clip_jobs(const RenderParams &p, const Cam &cm, int view, const uint32_t *jobs,
                          int njobs, TriRec *slots, float *scratch, const Group &grp) {
    const int lane = grp.tid & 31, warp = grp.warp(), nw = grp.nw();
    const int g = lane >> 3, gl = lane & 7, seg0 = lane & ~7;
    const unsigned int segmask = 0xFFu << seg0, lt = (1u << lane) - 1u;
    float *sc = scratch + (warp * 4 + g) * 24;  // 8 vertices x (x, y, z) per segment
    for (int jb = warp * 4; jb < njobs; jb += nw * 4) {
        const int job = jb + g;
        const bool active = job < njobs;
        float x = 0.f, y = 0.f, z = 1.f;
        uint32_t prim = 0;
        int n = 0, oc = 0;
        if (active) {
            float wx[3], wy[3], wz[3];
            source_tri(p, cm, jobs[job], wx, wy, wz, prim);
            n = 3;
            if (gl < 3) {
                const float3 v = to_view(p, cm, gl == 0 ? wx[0] : (gl == 1 ? wx[1] : wx[2]),
                                         gl == 0 ? wy[0] : (gl == 1 ? wy[1] : wy[2]),
                                         gl == 0 ? wz[0] : (gl == 1 ? wz[1] : wz[2]));
                x = v.x;
                y = v.y;
                z = v.z;
                oc = outcode(p, cm, x, y, z);
            }
        }
        oc |= __shfl_xor_sync(0xffffffffu, oc, 1);
        oc |= __shfl_xor_sync(0xffffffffu, oc, 2);
        oc |= __shfl_xor_sync(0xffffffffu, oc, 4);
        const int planes = oc & 0x1F;
#pragma unroll 1
        for (int k = 0; k < 5; ++k) {
            const bool do_k = active && n >= 3 && (planes & (1 << k));  // segment-uniform
            if (!__any_sync(0xffffffffu, do_k)) continue;  // no job of this warp crosses plane k
            const float dk = plane_dist(p, k, x, y, z);
            const int nxt = seg0 + ((gl + 1 < n) ? gl + 1 : 0);
            const float xn = __shfl_sync(0xffffffffu, x, nxt);
            const float yn = __shfl_sync(0xffffffffu, y, nxt);
            const float zn = __shfl_sync(0xffffffffu, z, nxt);
            const float dn = __shfl_sync(0xffffffffu, dk, nxt);
            const bool in_i = dk >= 0.f, in_n = dn >= 0.f;
            const bool ev = do_k && gl < n && in_i;
            const bool ex = do_k && gl < n && in_i != in_n;
            const unsigned int bv = __ballot_sync(0xffffffffu, ev);
            const unsigned int bx = __ballot_sync(0xffffffffu, ex);
            const int pos = __popc(bv & segmask & lt) + __popc(bx & segmask & lt);
            int nn = __popc(bv & segmask) + __popc(bx & segmask);
            if (ev && pos < 8) {
                sc[3 * pos] = x;
                sc[3 * pos + 1] = y;
                sc[3 * pos + 2] = z;
            }
            if (ex && pos + (ev ? 1 : 0) < 8) {
                const float xi = in_i ? x : xn, yi = in_i ? y : yn, zi = in_i ? z : zn;
                const float xo = in_i ? xn : x, yo = in_i ? yn : y, zo = in_i ? zn : z;
                const float di = in_i ? dk : dn, dov = in_i ? dn : dk;
                const float t = __fdiv_rn(di, __fsub_rn(di, dov));
                const int q = pos + (ev ? 1 : 0);
                sc[3 * q] = __fmaf_rn(t, __fsub_rn(xo, xi), xi);
                sc[3 * q + 1] = __fmaf_rn(t, __fsub_rn(yo, yi), yi);
                sc[3 * q + 2] = __fmaf_rn(t, __fsub_rn(zo, zi), zi);
            }
            __syncwarp();
            if (do_k) {
                if (nn > 8) {  // not reachable for exact input: a plane adds at most one vertex
                    if (gl == 0) atomicOr(p.status, GP_DEV_CLIP_OVERFLOW);
                    nn = 8;
                }
                if (gl < nn) {
                    x = sc[3 * gl];
                    y = sc[3 * gl + 1];
                    z = sc[3 * gl + 2];
                }
                n = nn;
            }
            __syncwarp();
        }
        int X = 0, Y = 0;
        float d = 0.f;
        if (active && n >= 3 && gl < n) project(p, x, y, z, X, Y, d);
        const int s1 = seg0 + min(gl + 1, 7), s2 = seg0 + min(gl + 2, 7);
        const int tX[3] = {__shfl_sync(0xffffffffu, X, seg0), __shfl_sync(0xffffffffu, X, s1),
                           __shfl_sync(0xffffffffu, X, s2)};
        const int tY[3] = {__shfl_sync(0xffffffffu, Y, seg0), __shfl_sync(0xffffffffu, Y, s1),
                           __shfl_sync(0xffffffffu, Y, s2)};
        const float td[3] = {__shfl_sync(0xffffffffu, d, seg0), __shfl_sync(0xffffffffu, d, s1),
                             __shfl_sync(0xffffffffu, d, s2)};
        bool built = false;
        if (active && gl < 6) {
            TriRec &r = slots[6 * job + gl];
            int i0, i1, j0, j1;
            if (n >= 3 && gl + 2 < n && tri_bbox(p, cm, tX, tY, i0, i1, j0, j1)) {
                build_rec(r, tX, tY, td, prim, p.key_f16, i0, i1, j0, j1, cm.by0);
                if (view == p.dump_view) dump_tri(p, tX, tY, td, prim, (uint32_t)gl);
                built = true;
            } else {
                empty_rec(r);
            }
        }
        if (ST && p.stats) {
            const unsigned int b = __ballot_sync(0xffffffffu, built);
            if ((threadIdx.x & 31) == 0 && b)
                atomicAdd(&p.stats[GP_STAT_TRIS_FROM_CLIP], (unsigned long long)__popc(b));
        }
    }
}

// Reserve [base, base + n) of a counter if it stays within cap; returns base or -1.  The
// counter only ever grows by successful reservations.
__device__ __forceinline__ int cas_reserve(int *counter, int n, int cap) {
    int cur = *(volatile int *)counter;
    for (;;) {
        if (cur + n > cap) return -1;
        const int prev = atomicCAS(counter, cur, cur + n);
        if (prev == cur) return cur;
        cur = prev;
    }
}

// World-space corners of a source quad and the primitive id of its first triangle.
//   code bit 31 set: box face, bits 4..11 local box index, bits 0..3 face index
//   code bit 30 set: signal face, bits 5..9 local signal index, bits 0..4 face q
//   otherwise: ground quad index (cluster order)
// The quad's triangles are (q0 q1 q2) and (q0 q2 q3), primitive ids prim0 and prim0 + 1.
__device__ __forceinline__ void source_quad(const RenderParams &p, const Cam &cm, uint32_t code,
                                            float qx[4], float qy[4], float qz[4],
                                            uint32_t &prim0) {
    if (code & 0x80000000u) {
        const int b = (code >> 4) & 0xFF, face = code & 15;
        const float4 pose = p.box_pose[cm.box_begin + b];
        const float4 dim = p.box_dim[cm.box_begin + b];
        float s, c;
        sincosf(pose.z, &s, &c);
        int k0, k1, k2, k3;
        box_tri(2 * face, k0, k1, k2);      // (q0 q1 q2)
        box_tri(2 * face + 1, k0, k2, k3);  // (q0 q2 q3)
        box_corner(pose, dim, s, c, k0, qx[0], qy[0], qz[0]);
        box_corner(pose, dim, s, c, k1, qx[1], qy[1], qz[1]);
        box_corner(pose, dim, s, c, k2, qx[2], qy[2], qz[2]);
        box_corner(pose, dim, s, c, k3, qx[3], qy[3], qz[3]);
        prim0 = 12u * b + 2u * face;
    } else if (code & 0x40000000u) {
        const int sg = (code >> 5) & 31, q = code & 31;
        const float4 sp = p.sig[cm.sig_begin + sg];
        const int i = q >> 3, j = q & 7;
        sig_vertex(sp, i, j, qx[0], qy[0], qz[0]);
        sig_vertex(sp, i, j + 1, qx[1], qy[1], qz[1]);
        sig_vertex(sp, i + 1, j + 1, qx[2], qy[2], qz[2]);
        sig_vertex(sp, i + 1, j, qx[3], qy[3], qz[3]);
        prim0 = cm.line_end + 64u * sg + 2u * q;
    } else {
        const float4 g0 = p.quad_geo[2 * code], g1 = p.quad_geo[2 * code + 1];
        prim0 = p.quad_prim[code];
        const float z = prim0 < cm.road_end ? 0.f : p.line_z;
        qx[0] = g0.x;
        qy[0] = g0.y;
        qx[1] = g0.z;
        qy[1] = g0.w;
        qx[2] = g1.x;
        qy[2] = g1.y;
        qx[3] = g1.z;
        qy[3] = g1.w;
        qz[0] = qz[1] = qz[2] = qz[3] = z;
    }
}

// One setup unit: 32 quads (box faces, the 32 faces of one signal sphere, or the visible
// clusters' ground quads packed back to back), one per lane, two triangles each
// (warp-uniform call).  Returns false if the clip queue or the batch has no room;
// `clips_queued` tells the retry (after a flush) whether this unit's clip jobs are already
// queued.
template <bool ST>
__device__ bool setup_unit(const RenderParams &p, const Cam &cm, Shared &sh, TriRec *tris,
                           uint32_t *clipq, const int *vq0, const int *vpre, int nvcl, int nvq,
                           const unsigned char *visbox, const unsigned char *vissig, int view,
                           int unit, int n_box_units, int nbox_items, int n_sig_units,
                           bool clips_done, bool &clips_queued) {
    const int lane = threadIdx.x & 31;
    uint32_t qcode = 0, tcode = 0;  // quad code; triangle-code base for the clip queue
    bool valid;
    if (unit < n_box_units) {
        const int item = unit * 32 + lane;
        valid = item < nbox_items;
        if (valid) {
            const uint32_t b = visbox[item / 6], face = item % 6;
            qcode = 0x80000000u | (b << 4) | face;
            tcode = 0x80000000u | (b << 4) | (2u * face);
        }
    } else if (unit < n_box_units + n_sig_units) {
        const uint32_t sg = vissig[unit - n_box_units];
        valid = true;
        qcode = 0x40000000u | (sg << 5) | (uint32_t)lane;
        tcode = 0x40000000u | (sg << 6) | (2u * lane);
    } else {
        // the visible clusters' quads, packed 32 per unit: find this lane's cluster (the
        // last one whose first packed index is <= gq)
        const int gq = (unit - n_box_units - n_sig_units) * 32 + lane;
        valid = gq < nvq;
        int lo = 0, hi = nvcl - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (vpre[mid] <= gq) lo = mid;
            else hi = mid - 1;
        }
        qcode = valid ? (uint32_t)(vq0[lo] + (gq - vpre[lo])) : 0u;
        tcode = qcode << 1;
    }
    bool keep0 = false, keep1 = false, clip0 = false, clip1 = false;
    int X[4] = {0, 0, 0, 0}, Y[4] = {0, 0, 0, 0};
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    int b0[4] = {0, 0, 0, 0}, b1[4] = {0, 0, 0, 0};  // bounding rows/columns per triangle
    uint32_t prim0 = 0;
    if (valid) {
        float wx[4], wy[4], wz[4];
        source_quad(p, cm, qcode, wx, wy, wz, prim0);
        float vx[4], vy[4], vz[4];
        int oc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float3 v = to_view(p, cm, wx[i], wy[i], wz[i]);
            vx[i] = v.x;
            vy[i] = v.y;
            vz[i] = v.z;
            oc[i] = outcode(p, cm, v.x, v.y, v.z);
        }
        const int and0 = oc[0] & oc[1] & oc[2], or0 = oc[0] | oc[1] | oc[2];
        const int and1 = oc[0] & oc[2] & oc[3], or1 = oc[0] | oc[2] | oc[3];
        const bool fast0 = and0 == 0 && (or0 & 0x1F) == 0;
        const bool fast1 = and1 == 0 && (or1 & 0x1F) == 0;
        clip0 = and0 == 0 && !fast0;
        clip1 = and1 == 0 && !fast1;
        if (fast0 || fast1) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if ((oc[i] & 0x1F) == 0) project(p, vx[i], vy[i], vz[i], X[i], Y[i], d[i]);
            if (fast0) {
                const int tX[3] = {X[0], X[1], X[2]}, tY[3] = {Y[0], Y[1], Y[2]};
                keep0 = tri_bbox(p, cm, tX, tY, b0[0], b0[1], b0[2], b0[3]);
            }
            if (fast1) {
                const int tX[3] = {X[0], X[2], X[3]}, tY[3] = {Y[0], Y[2], Y[3]};
                keep1 = tri_bbox(p, cm, tX, tY, b1[0], b1[1], b1[2], b1[3]);
            }
        }
    }
    const unsigned int k0 = __ballot_sync(0xffffffffu, keep0);
    const unsigned int k1 = __ballot_sync(0xffffffffu, keep1);
    const unsigned int c0 = __ballot_sync(0xffffffffu, clip0);
    const unsigned int c1 = __ballot_sync(0xffffffffu, clip1);
    const unsigned int lt = (1u << lane) - 1u;
    // Triangles that need clipping go to the block's clip queue (clipped later by whole
    // warps).  Reservations never exceed their capacity, so every reserved slot is written.
    clips_queued = clips_done;
    if (!clips_done && (c0 | c1)) {
        const int n0 = __popc(c0), nc = n0 + __popc(c1);
        int qb = 0;
        if (lane == 0) qb = cas_reserve(&sh.cq_n, nc, kClipQueue);
        qb = __shfl_sync(0xffffffffu, qb, 0);
        if (qb < 0) return false;
        if (clip0) clipq[qb + __popc(c0 & lt)] = tcode;
        if (clip1) clipq[qb + n0 + __popc(c1 & lt)] = tcode + 1u;
        if (ST && p.stats && lane == 0) atomicAdd(&p.stats[GP_STAT_TRIS_CLIPPED], (unsigned long long)nc);
    }
    clips_queued = true;
    if (!(k0 | k1)) return true;
    const int nk0 = __popc(k0), nk = nk0 + __popc(k1);
    int base = 0;
    if (lane == 0) base = cas_reserve(&sh.resv, nk, p.tri_cap);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base < 0) return false;
    if (ST && p.stats && lane == 0) atomicAdd(&p.stats[GP_STAT_TRIS_KEPT], (unsigned long long)nk);
    if (keep0) {
        const int tX[3] = {X[0], X[1], X[2]}, tY[3] = {Y[0], Y[1], Y[2]};
        const float td[3] = {d[0], d[1], d[2]};
        build_rec(tris[base + __popc(k0 & lt)], tX, tY, td, prim0, p.key_f16, b0[0], b0[1], b0[2],
                  b0[3], cm.by0);
        if (view == p.dump_view) dump_tri(p, tX, tY, td, prim0, 0u);
    }
    if (keep1) {
        const int tX[3] = {X[0], X[2], X[3]}, tY[3] = {Y[0], Y[2], Y[3]};
        const float td[3] = {d[0], d[2], d[3]};
        build_rec(tris[base + nk0 + __popc(k1 & lt)], tX, tY, td, prim0 + 1u, p.key_f16, b1[0], b1[1],
                  b1[2], b1[3], cm.by0);
        if (view == p.dump_view) dump_tri(p, tX, tY, td, prim0 + 1u, 0u);
    }
    return true;
}

// Class of an inverted primitive id (0 = nothing covered): 3 box, 1 road, 2 lane line,
// 4 signal.
__device__ __forceinline__ uint32_t class_of_low(uint32_t low, uint32_t full, const Cam &cm) {
    if (!low) return 0;
    const uint32_t prim = full - low;
    return prim < cm.box_end ? 3u : (prim < cm.road_end ? 1u : (prim < cm.line_end ? 2u : 4u));
}

// RGB observation of one pixel, 8 bits per channel in bytes 0..2 (App. A: one directional
// light, a colour per instance): class colour x (ambient + (1 - ambient) max(0, n . l)), n
// the winning surface's outward normal -- a box face's normal turned by the box yaw, +z for
// the ground strips, a signal face's normal (signals take their state's colour) -- and the
// background unshaded; each channel rint(255 clamp(v, 0, 1)).
// low = inverted primitive id (0 = background), full = the id's all-ones value.
__device__ __forceinline__ uint32_t shade_rgb(const RenderParams &p, const Cam &cm, uint32_t low,
                                              uint32_t full) {
    uint32_t cls = 0, state = 0;
    float shade = 1.f;
    if (low) {
        const uint32_t prim = full - low;
        cls = prim < cm.box_end ? 3u : (prim < cm.road_end ? 1u : (prim < cm.line_end ? 2u : 4u));
        float nx = 0.f, ny = 0.f, nz = 1.f;
        if (cls == 4u) {
            const uint32_t rel = prim - cm.line_end;
            const float4 fn = c_sig_face[(rel & 63u) >> 1];
            nx = fn.x;
            ny = fn.y;
            nz = fn.z;
            state = p.sig_state[cm.sig_begin + (rel >> 6)] & 3u;
        } else if (cls == 3u) {
            const uint32_t b = prim / 12u, face = (prim % 12u) >> 1;
            float sn, c;
            sincosf(p.box_pose[cm.box_begin + b].z, &sn, &c);
            // faces +x, -x, +y, -y, +z, -z of the box frame
            nx = face == 0 ? c : (face == 1 ? -c : (face == 2 ? -sn : (face == 3 ? sn : 0.f)));
            ny = face == 0 ? sn : (face == 1 ? -sn : (face == 2 ? c : (face == 3 ? -c : 0.f)));
            nz = face == 4 ? 1.f : (face == 5 ? -1.f : 0.f);
        }
        const float ndl = fmaxf(nx * p.light[0] + ny * p.light[1] + nz * p.light[2], 0.f);
        shade = p.ambient + (1.f - p.ambient) * ndl;
    }
    uint32_t rgb = 0;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float base = cls == 4u ? p.sig_colour[state][ch]
                                     : (cls == 0u ? p.colour[0][ch]
                                                  : (cls == 1u ? p.colour[1][ch]
                                                               : (cls == 2u ? p.colour[2][ch] : p.colour[3][ch])));
        const float v = fminf(fmaxf(base * shade, 0.f), 1.f);
        rgb |= (uint32_t)__float2int_rn(255.f * v) << (8 * ch);
    }
    return rgb;
}

// Store one group of four adjacent pixels: class ids, normalised one-hot channels, or RGB.
// c: classes; low: inverted primitive ids (full: the id's all-ones value).
__device__ __forceinline__ void store_classes(const RenderParams &p, const Cam &cm, long long slot,
                                              long long plane, long long px, const uint32_t c[4],
                                              const uint32_t low[4], uint32_t full) {
    if (p.out_mode == GP_OUT_CLASS_U8) {
        __stcs((unsigned int *)((uint8_t *)p.out + slot * plane + px),
               c[0] | (c[1] << 8) | (c[2] << 16) | (c[3] << 24));
    } else if (p.out_mode == GP_OUT_RGB_U8) {
        uint32_t q[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) q[k] = shade_rgb(p, cm, low[k], full);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const int sh = 8 * ch;
            __stcs((unsigned int *)((uint8_t *)p.out + (slot * 3 + ch) * plane + px),
                   ((q[0] >> sh) & 0xFFu) | (((q[1] >> sh) & 0xFFu) << 8) |
                       (((q[2] >> sh) & 0xFFu) << 16) | (((q[3] >> sh) & 0xFFu) << 24));
        }
    } else {
        // signals (class 4) share the object channel 3 with the boxes
        const uint32_t o[4] = {c[0] == 4u ? 3u : c[0], c[1] == 4u ? 3u : c[1], c[2] == 4u ? 3u : c[2],
                               c[3] == 4u ? 3u : c[3]};
        for (int ch = 0; ch < 4; ++ch) {
            const uint32_t lo = (uint32_t)p.onehot[ch][o[0] == (uint32_t)ch] |
                                ((uint32_t)p.onehot[ch][o[1] == (uint32_t)ch] << 16);
            const uint32_t hi = (uint32_t)p.onehot[ch][o[2] == (uint32_t)ch] |
                                ((uint32_t)p.onehot[ch][o[3] == (uint32_t)ch] << 16);
            __stcs((uint2 *)((uint16_t *)p.out + (slot * 4 + ch) * plane + px), make_uint2(lo, hi));
        }
    }
}

// Encode the band into the output tensors and clear the planes for the next item.  Each
// lane reads four adjacent words of a plane with one 16-byte shared load (conflict-free)
// and writes the matching adjacent outputs, so a warp's stores cover contiguous sectors.
// FP32 mode: one 64-bit key per pixel, FP32 depth bits above the inverted primitive id.
__device__ void encode_f32(const RenderParams &p, const Cam &cm, unsigned long long *keys,
                           int view, const Group &g) {
    const int band_px = (cm.by1 - cm.by0 + 1) * p.W;
    const long long slot = p.view_mod ? (view % p.view_mod) : view;
    const long long plane = (long long)p.H * p.W;
    const long long row0 = (long long)cm.by0 * p.W;
    for (int b = 4 * g.tid; b < band_px; b += 4 * g.nt) {
        const ulonglong2 k01 = *(const ulonglong2 *)(keys + b);
        const ulonglong2 k23 = *(const ulonglong2 *)(keys + b + 2);
        *(ulonglong2 *)(keys + b) = make_ulonglong2(0ull, 0ull);
        *(ulonglong2 *)(keys + b + 2) = make_ulonglong2(0ull, 0ull);
        const uint32_t low[4] = {(uint32_t)k01.x, (uint32_t)k01.y, (uint32_t)k23.x, (uint32_t)k23.y};
        const uint32_t c[4] = {class_of_low(low[0], 0xFFFFFFFFu, cm), class_of_low(low[1], 0xFFFFFFFFu, cm),
                               class_of_low(low[2], 0xFFFFFFFFu, cm), class_of_low(low[3], 0xFFFFFFFFu, cm)};
        store_classes(p, cm, slot, plane, row0 + b, c, low, 0xFFFFFFFFu);
        if (p.depth)
            __stcs((uint4 *)((float *)p.depth + slot * plane + row0 + b),
                   make_uint4((uint32_t)(k01.x >> 32), (uint32_t)(k01.y >> 32),
                              (uint32_t)(k23.x >> 32), (uint32_t)(k23.y >> 32)));
    }
}

// FP16 mode: one key per pixel, binary16 depth bits above the inverted primitive id.  With
// the one-hot output and a width that is a multiple of 8, a lane takes eight pixels, so each
// channel (and the depth plane) is written with one 16-byte store per lane.
__device__ void encode_f16(const RenderParams &p, const Cam &cm, unsigned int *keys, int view,
                           const Group &g) {
    const int band_px = (cm.by1 - cm.by0 + 1) * p.W;
    const long long slot = p.view_mod ? (view % p.view_mod) : view;
    const long long plane = (long long)p.H * p.W;
    const long long row0 = (long long)cm.by0 * p.W;
    if (p.out_mode == GP_OUT_ONEHOT_BF16 && (p.W & 7) == 0) {
        for (int b = 8 * g.tid; b < band_px; b += 8 * g.nt) {
            const uint4 ka = *(const uint4 *)(keys + b);
            const uint4 kb = *(const uint4 *)(keys + b + 4);
            *(uint4 *)(keys + b) = make_uint4(0u, 0u, 0u, 0u);
            *(uint4 *)(keys + b + 4) = make_uint4(0u, 0u, 0u, 0u);
            const uint32_t k[8] = {ka.x, ka.y, ka.z, ka.w, kb.x, kb.y, kb.z, kb.w};
            uint32_t o[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const uint32_t c = class_of_low(k[q] & 0xFFFFu, 0xFFFFu, cm);
                o[q] = c == 4u ? 3u : c;  // signals share the object channel 3 with the boxes
            }
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
                uint32_t w[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    w[q] = (uint32_t)p.onehot[ch][o[2 * q] == (uint32_t)ch] |
                           ((uint32_t)p.onehot[ch][o[2 * q + 1] == (uint32_t)ch] << 16);
                __stcs((uint4 *)((uint16_t *)p.out + (slot * 4 + ch) * plane + row0 + b),
                       make_uint4(w[0], w[1], w[2], w[3]));
            }
            if (p.depth)
                __stcs((uint4 *)((uint16_t *)p.depth + slot * plane + row0 + b),
                       make_uint4((k[0] >> 16) | (k[1] & 0xFFFF0000u), (k[2] >> 16) | (k[3] & 0xFFFF0000u),
                                  (k[4] >> 16) | (k[5] & 0xFFFF0000u), (k[6] >> 16) | (k[7] & 0xFFFF0000u)));
        }
        return;
    }
    for (int b = 4 * g.tid; b < band_px; b += 4 * g.nt) {
        const uint4 k = *(const uint4 *)(keys + b);
        *(uint4 *)(keys + b) = make_uint4(0u, 0u, 0u, 0u);
        const uint32_t low[4] = {k.x & 0xFFFFu, k.y & 0xFFFFu, k.z & 0xFFFFu, k.w & 0xFFFFu};
        const uint32_t c[4] = {class_of_low(low[0], 0xFFFFu, cm), class_of_low(low[1], 0xFFFFu, cm),
                               class_of_low(low[2], 0xFFFFu, cm), class_of_low(low[3], 0xFFFFu, cm)};
        store_classes(p, cm, slot, plane, row0 + b, c, low, 0xFFFFu);
        if (p.depth)
            __stcs((uint2 *)((uint16_t *)p.depth + slot * plane + row0 + b),
                   make_uint2((k.x >> 16) | (k.y & 0xFFFF0000u), (k.z >> 16) | (k.w & 0xFFFF0000u)));
    }
}

// ------------------------------------------------------------------------------------
// Ray-traced backend: one ray per pixel centre, nearest hit among the boxes (slab test),
// the lane-line strips and the road quads (plane hit, point in quad); ties go to the lower
// object (boxes by index, then lines over the road below them, then roads).  The result is
// written in the same formats as the raster; the primitive id of a hit follows the raster's
// numbering (box b's entry face f: 12 b + 2 f), so the RGB shading applies unchanged.
// ------------------------------------------------------------------------------------

// Camera of a view (agent pose + rig yaw) and its world.
__device__ __forceinline__ void view_cam(const RenderParams &p, int view, Cam &cm, WorldInfo &wi) {
    const int agent = view / p.n_cams, cam = view - agent * p.n_cams;
    wi = p.worlds[p.agent_world[agent]];
    cm.ego = agent - wi.agent_begin;
    cm.box_begin = wi.box_begin;
    cm.cl_begin = wi.cl_begin;
    cm.box_end = wi.box_end;
    cm.road_end = wi.road_end;
    cm.line_end = wi.line_end;
    cm.sig_begin = wi.sig_begin;
    const float4 pose = p.box_pose[wi.box_begin + cm.ego];
    cm.px = pose.x;
    cm.py = pose.y;
    sincosf(pose.z + p.cam_yaw[cam], &cm.s, &cm.c);
}

__device__ __forceinline__ bool quad_contains(float px, float py, float4 g0, float4 g1) {
    const float qx[4] = {g0.x, g0.z, g1.x, g1.z};
    const float qy[4] = {g0.y, g0.w, g1.y, g1.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int n = (k + 1) & 3;
        if ((qx[n] - qx[k]) * (py - qy[k]) - (qy[n] - qy[k]) * (px - qx[k]) < 0.f) return false;
    }
    return true;
}

// The quad of smallest index among those listed in the point's grid cell that contain it;
// -1 if none.  A cell lists its quads in increasing index order, so the first that contains
// the point is the one.
__device__ int ground_quad(const WorldInfo &wi, float px, float py, const int *off,
                           const int *list, int cell_base, float ginv, int gnx, int gny,
                           const float4 *geo) {
    const float fx = floorf((px - wi.gx0) * ginv), fy = floorf((py - wi.gy0) * ginv);
    if (!(fx >= 0.f && fy >= 0.f && fx < (float)gnx && fy < (float)gny)) return -1;
    const int cell = cell_base + (int)fy * gnx + (int)fx;
    for (int q = off[cell]; q < off[cell + 1]; ++q) {
        const int r = list[q];
        if (quad_contains(px, py, geo[2 * r], geo[2 * r + 1])) return r;
    }
    return -1;
}

// A box as one view's rays see it: yaw cos/sin, the camera position in the box frame, half
// extents and height; skipped (the ego's box, or entirely behind the camera) if hl < 0.
struct TraceBox {
    float cs, sn, ox, oy, hl, hw, h, pad;
};

// Ray-traced class (0 background) and, on a hit, primitive id and view depth t of pixel (i, j).
// blist[0, nb): the boxes that can appear in this block's rows, in index order; ts: the
// world's signal spheres as (camera - centre, radius), radius < 0 if culled.
__device__ int trace_pixel(const RenderParams &p, const Cam &cm, const WorldInfo &wi, int i, int j,
                           const TraceBox *tb, const unsigned char *blist, int nb,
                           const float4 *ts, uint32_t &prim, float &t_hit) {
    const float x = ((float)i + 0.5f - 0.5f * (float)p.W) / p.f;
    const float y = (0.5f * (float)p.H - (float)j - 0.5f) / p.f;
    // right = (sin psi, -cos psi, 0), up = +z, forward = (cos psi, sin psi, 0)
    const float dx = cm.s * x + cm.c, dy = -cm.c * x + cm.s, dz = y;
    const float oz = p.cam_h;
    float best = INFINITY;
    int cls = 0;
    prim = 0xFFFFFFFFu;
    for (int k = 0; k < nb; ++k) {
        const int b = blist[k];
        const TraceBox B = tb[b];
        const float cs = B.cs, sn = B.sn;
        const float o[3] = {B.ox, B.oy, oz};
        const float d[3] = {cs * dx + sn * dy, -sn * dx + cs * dy, dz};
        const float lo[3] = {-B.hl, -B.hw, 0.f};
        const float hi[3] = {B.hl, B.hw, B.h};
        float t0 = -INFINITY, t1 = INFINITY;
        int face = -1;
        bool inside = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (d[k] == 0.f) {
                if (o[k] < lo[k] || o[k] > hi[k]) inside = false;
                continue;
            }
            const float rd = __frcp_rn(d[k]);  // one reciprocal, two products
            float ta = (lo[k] - o[k]) * rd, tb = (hi[k] - o[k]) * rd;
            int fa = 2 * k + 1;  // entering through the low side: face -k
            if (ta > tb) {
                const float tt = ta;
                ta = tb;
                tb = tt;
                fa = 2 * k;
            }
            if (ta > t0) {
                t0 = ta;
                face = fa;
            }
            t1 = fminf(t1, tb);
        }
        if (!inside || face < 0 || t0 > t1 || t0 < p.near_plane || !(t0 < best)) continue;
        best = t0;
        cls = 3;
        prim = (uint32_t)(12 * b + 2 * face);
    }
    if (dz < 0.f) {
        // lane-line strips lie above the road: a line hit is nearer than the road below it
        const float tl = (p.line_z - oz) / dz;
        bool line_hit = false;
        if (tl >= p.near_plane && tl < best) {
            const int q = ground_quad(wi, cm.px + tl * dx, cm.py + tl * dy, p.lcell_off,
                                      p.lcell_quads, wi.lcell_begin, wi.lginv, wi.lgnx, wi.lgny,
                                      p.line_geo);
            if (q >= 0) {
                best = tl;
                cls = 2;
                prim = wi.road_end + 2u * (uint32_t)(q - wi.line_begin);
                line_hit = true;
            }
        }
        const float tr = -oz / dz;
        if (!line_hit && tr >= p.near_plane && tr < best) {
            const int q = ground_quad(wi, cm.px + tr * dx, cm.py + tr * dy, p.rcell_off,
                                      p.rcell_quads, wi.rcell_begin, wi.rginv, wi.rgnx, wi.rgny,
                                      p.road_geo);
            if (q >= 0) {
                best = tr;
                cls = 1;
                prim = wi.box_end + 2u * (uint32_t)(q - wi.road_begin);
            }
        }
    }
    // signal spheres: the polyhedron as the intersection of its face half-spaces (entry at
    // the largest entering-face parameter, the first such face on ties), after a reject
    // against the circumscribed sphere
    const float dd = dx * dx + dy * dy + dz * dz;
    for (int sg = 0; sg < wi.n_sig; ++sg) {
        const float4 S = ts[sg];
        if (S.w < 0.f) continue;
        const float b = S.x * dx + S.y * dy + S.z * dz;
        const float c0 = S.x * S.x + S.y * S.y + S.z * S.z - S.w * S.w * 1.0001f - 1e-6f;
        if (b * b < dd * c0) continue;  // the ray's line misses the circumsphere
        float t0 = -INFINITY, t1 = INFINITY;
        int face = -1;
        bool inside = true;
        for (int q = 0; q < kSignalQuads; ++q) {
            const float4 F = c_sig_face[q];
            const float den = F.x * dx + F.y * dy + F.z * dz;
            const float num = F.w * S.w - (F.x * S.x + F.y * S.y + F.z * S.z);
            if (den == 0.f) {
                if (num < 0.f) inside = false;
                continue;
            }
            const float t = num * __frcp_rn(den);
            if (den < 0.f) {
                if (t > t0) {
                    t0 = t;
                    face = q;
                }
            } else {
                t1 = fminf(t1, t);
            }
        }
        if (!inside || face < 0 || t0 > t1 || t0 < p.near_plane || !(t0 < best)) continue;
        best = t0;
        cls = 4;
        prim = wi.line_end + 64u * (uint32_t)sg + 2u * (uint32_t)face + (face < 8 ? 1u : 0u);
    }
    t_hit = best;
    return cls;
}

// One thread traces four consecutive pixels of one view and stores them like the raster's
// encode (class / one-hot / RGB, and FP32 depth or its binary16 bits).
// 14 blocks of 128 threads per SM caps the kernel at 32 registers: the latency of its grid
// and quad loads hides better with more resident warps than it loses to a few spills
// (A/B: 2.59 -> 2.38 ms per launch on the uniform batch).
// PAIRS: the four pixels are traced two at a time (interleaved, for instruction-level
// parallelism) -- used when no world has signal spheres; with spheres the larger tracing
// code runs one pixel at a time, which stalls less on instruction fetch (A/B on B300:
// uniform 2.31 -> 2.13 ms with pairs; the 210 x 126 rig with signals 19.9 -> 21.1 ms).
template <bool PAIRS>
__global__ void __launch_bounds__(128, 14) trace_kernel(RenderParams p) {
    __shared__ TraceBox tb[kMaxBoxes];
    __shared__ float4 ts[kMaxSignals];
    __shared__ unsigned char blist[kMaxBoxes];
    __shared__ int wcount[4];
    const int view = p.trace_view0 + (int)blockIdx.y;
    const long long plane = (long long)p.H * p.W;
    const int px0 = 4 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    Cam cm;
    WorldInfo wi;
    view_cam(p, view, cm, wi);
    // this block's pixel rows
    const long long first = 4LL * blockIdx.x * blockDim.x;
    const int row0 = (int)(first / p.W);
    const int row1 = (int)(min(first + 4LL * blockDim.x, (long long)p.H * p.W) - 1) / p.W;
    // the world's boxes in index order (ties keep going to the lower index), each once per
    // block: yaw sin/cos and the camera in the box frame
    bool keep = false;
    for (int b = threadIdx.x; b < wi.n_boxes; b += blockDim.x) {
        const float4 bp = p.box_pose[wi.box_begin + b];
        const float4 bd = p.box_dim[wi.box_begin + b];
        TraceBox B;
        sincosf(bp.z, &B.sn, &B.cs);
        const float ox = cm.px - bp.x, oy = cm.py - bp.y;
        B.ox = B.cs * ox + B.sn * oy;
        B.oy = -B.sn * ox + B.cs * oy;
        B.hl = 0.5f * bd.x;
        B.hw = 0.5f * bd.y;
        B.h = bd.z;
        B.pad = 0.f;
        // no ray can hit a box whose footprint circle (radius = half diagonal) lies wholly
        // behind the near plane or wholly outside the left or right frustum plane
        const float fwd = -(ox * cm.c + oy * cm.s), side = -ox * cm.s + oy * cm.c;
        const float rad = sqrtf(B.hl * B.hl + B.hw * B.hw);
        const float nrm = sqrtf(1.f + p.tx * p.tx);
        const bool culled = fwd + rad < p.near_plane || (side + p.tx * fwd) < -rad * nrm ||
                            (p.tx * fwd - side) < -rad * nrm;
        if (b == cm.ego || culled) B.hl = -1.f;
        tb[b] = B;
        keep = B.hl >= 0.f;
        if (keep) {
            // rows the box can cover: its corners' projected rows when all lie beyond the
            // near plane (else every row), widened by a pixel for rounding
            float jlo = INFINITY, jhi = -INFINITY;
            bool behind = false;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float lx = (k & 1) ? B.hl : -B.hl, ly = (k & 2) ? B.hw : -B.hw;
                const float wx = bp.x + B.cs * lx - B.sn * ly - cm.px;
                const float wy = bp.y + B.sn * lx + B.cs * ly - cm.py;
                const float z = wx * cm.c + wy * cm.s;
                const float yv = ((k & 4) ? B.h : 0.f) - p.cam_h;
                behind |= !(z > p.near_plane);
                const float j = 0.5f * (float)p.H - p.f * yv / z - 0.5f;
                jlo = fminf(jlo, j);
                jhi = fmaxf(jhi, j);
            }
            keep = behind || (jhi + 1.f >= (float)row0 && jlo - 1.f <= (float)row1);
        }
    }
    for (int sg = threadIdx.x; sg < wi.n_sig; sg += blockDim.x) {
        const float4 sp = p.sig[wi.sig_begin + sg];
        const float ox = cm.px - sp.x, oy = cm.py - sp.y, oz = p.cam_h - sp.z;
        // the same frustum test on the sphere's footprint circle
        const float fwd = -(ox * cm.c + oy * cm.s), side = -ox * cm.s + oy * cm.c;
        const float nrm = sqrtf(1.f + p.tx * p.tx);
        const bool culled = fwd + sp.w < p.near_plane || (side + p.tx * fwd) < -sp.w * nrm ||
                            (p.tx * fwd - side) < -sp.w * nrm;
        ts[sg] = make_float4(ox, oy, oz, culled ? -1.f : sp.w);
    }
    // compact the kept boxes, in index order (one box per thread: n_boxes <= blockDim)
    const unsigned int kb = __ballot_sync(0xffffffffu, keep);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) wcount[warp] = __popc(kb);
    __syncthreads();
    int pos = 0, nbk = 0;
    for (int w = 0; w < 4; ++w) {
        pos += w < warp ? wcount[w] : 0;
        nbk += wcount[w];
    }
    if (keep) blist[pos + __popc(kb & ((1u << lane) - 1u))] = (unsigned char)threadIdx.x;
    __syncthreads();
    if (px0 >= plane) return;
    const uint32_t full = p.key_f16 ? 0xFFFFu : 0xFFFFFFFFu;
    // the four pixels in a rolled loop (one or two copies of the tracing code: the fully
    // unrolled kernel stalled on instruction fetch), their results gathered in scalars
    uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0, l0 = 0, l1 = 0, l2 = 0, l3 = 0;
    float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
#pragma unroll(PAIRS ? 2 : 1)
    for (int k = 0; k < 4; ++k) {
        const int pix = px0 + k, j = pix / p.W, i = pix - j * p.W;
        uint32_t prim;
        float t;
        const uint32_t ck = (uint32_t)trace_pixel(p, cm, wi, i, j, tb, blist, nbk, ts, prim, t);
        const uint32_t lk = ck ? full - prim : 0u;
        const float dk = ck ? __fdiv_rn(p.near_plane, t) : 0.f;
        c0 = k == 0 ? ck : c0;
        c1 = k == 1 ? ck : c1;
        c2 = k == 2 ? ck : c2;
        c3 = k == 3 ? ck : c3;
        l0 = k == 0 ? lk : l0;
        l1 = k == 1 ? lk : l1;
        l2 = k == 2 ? lk : l2;
        l3 = k == 3 ? lk : l3;
        d0 = k == 0 ? dk : d0;
        d1 = k == 1 ? dk : d1;
        d2 = k == 2 ? dk : d2;
        d3 = k == 3 ? dk : d3;
    }
    const uint32_t c[4] = {c0, c1, c2, c3}, low[4] = {l0, l1, l2, l3};
    const float d[4] = {d0, d1, d2, d3};
    const long long slot = view;
    store_classes(p, cm, slot, plane, px0, c, low, full);
    if (p.depth) {
        if (p.key_f16) {
            const uint32_t h0 = __half_as_ushort(__float2half_rn(d[0])), h1 = __half_as_ushort(__float2half_rn(d[1]));
            const uint32_t h2 = __half_as_ushort(__float2half_rn(d[2])), h3 = __half_as_ushort(__float2half_rn(d[3]));
            __stcs((uint2 *)((uint16_t *)p.depth + slot * plane + px0), make_uint2(h0 | (h1 << 16), h2 | (h3 << 16)));
        } else {
            __stcs((float4 *)((float *)p.depth + slot * plane + px0), make_float4(d[0], d[1], d[2], d[3]));
        }
    }
}

// Camera and band of a work item.
__device__ __forceinline__ void make_cam(const RenderParams &p, int item, Cam &cm, WorldInfo &wi,
                                         int &view) {
    const int2 wv = p.items[p.item_begin + item];
    view = wv.x;
    const int band = wv.y;
    const int agent = view / p.n_cams, cam = view - agent * p.n_cams;
    wi = p.worlds[p.agent_world[agent]];
    cm.ego = agent - wi.agent_begin;
    cm.box_begin = wi.box_begin;
    cm.cl_begin = wi.cl_begin;
    cm.box_end = wi.box_end;
    cm.road_end = wi.road_end;
    cm.line_end = wi.line_end;
    cm.sig_begin = wi.sig_begin;
    const float4 pose = p.box_pose[wi.box_begin + cm.ego];
    cm.px = pose.x;
    cm.py = pose.y;
    sincosf(pose.z + p.cam_yaw[cam], &cm.s, &cm.c);
    cm.by0 = band * p.band_rows;
    cm.by1 = min(cm.by0 + p.band_rows, p.H) - 1;
    cm.gtx = __fmul_rn(p.guard, p.tx);
    cm.gty = __fmul_rn(p.guard, p.ty);
    // pixel centres of the band lie in x in [0.5, W - 0.5], y in [by0 + 0.5, by1 + 0.5];
    // a 1/4 px margin covers snapping (at most 1/32 px) and rounding
    cm.vl = (0.5f * (float)p.W - 0.25f) / p.f;
    cm.vt = (0.5f * (float)p.H - (float)cm.by0 - 0.25f) / p.f;
    cm.vb = (0.5f * (float)p.H - (float)cm.by1 - 0.75f) / p.f;
}

// Take the next work item (thread 0 of g) and reset the setup state; all of g call.
__device__ __forceinline__ int next_item(const RenderParams &p, Shared &sh, int iter, const Group &g) {
    if (g.tid == 0) {
        int it;
        if (p.work_counter) it = atomicAdd(p.work_counter, 1);
        else it = iter == 0 ? (int)blockIdx.x : p.n_items;
        sh.item = it;
        sh.resv = 0;
        sh.next_unit = 0;
        sh.npend = 0;
        sh.nvcl = 0;
        sh.nvbox = 0;
        sh.nvsig = 0;
        sh.cq_n = 0;
    }
    g.sync();
    return sh.item;
}

// Shared memory of the setup side.
struct SetupMem {
    TriRec *tris;  // batch being filled
    uint32_t *clipq;
    float *clipscratch;
    int *vq0, *vpre;
    unsigned char *vnq, *visbox, *vissig;
};

// Cull, set up and clip one (view, band) work item on group g.  Kept triangles fill the
// current batch m.tris[0, sh.resv).  emit(last) hands the batch over -- whenever it is
// full, and once with last = true when the item is done (that batch may be empty) -- and
// returns the batch to fill next, or nullptr to abandon the item; all threads of g call it
// after a group barrier, and it ends with one.  Returns false if the item was abandoned.
template <bool ST, class Emit>
__device__ bool produce_item(const RenderParams &p, const Cam &cm, const WorldInfo &wi, int view,
                             Shared &sh, SetupMem &m, const Group &g, Emit &emit) {
    // 1. cull clusters and boxes against the band frustum.  The clusters hold only ground
    //    quads; when the ground lies below the eye, each of their vertices (clipped ones
    //    too) projects below the horizon (snapped Y >= 8 H), so a band whose pixel-centre
    //    rows all lie above it (by1 < H / 2) can show none of them.
    const int n_cl = (cm.by1 < (p.H >> 1) && fmaxf(0.f, p.line_z) < p.cam_h) ? 0 : wi.n_cl;
    for (int base = 0; base < n_cl; base += g.nt) {
        const int c = base + g.tid;
        bool keep = false;
        Cluster cl{};
        if (c < n_cl) {
            cl = p.clusters[wi.cl_begin + c];
            keep = aabb_visible(p, cm, cl.cx, cl.cy, cl.hx, cl.hy, cl.zlo, cl.zhi);
        }
        const int k = warp_append(keep, &sh.nvcl);
        if (keep) {  // the cluster's quad range, so setup needs no further lookup
            m.vq0[k] = cl.q0;
            m.vnq[k] = (unsigned char)cl.nq;
        }
    }
    for (int base = 0; base < wi.n_boxes; base += g.nt) {
        const int b = base + g.tid;
        bool keep = false;
        if (b < wi.n_boxes && b != cm.ego) {
            const float4 bp = p.box_pose[wi.box_begin + b];
            const float4 bd = p.box_dim[wi.box_begin + b];
            float s, c;
            sincosf(bp.z, &s, &c);
            const float hx = 0.5f * (fabsf(c) * bd.x + fabsf(s) * bd.y);
            const float hy = 0.5f * (fabsf(s) * bd.x + fabsf(c) * bd.y);
            keep = aabb_visible(p, cm, bp.x, bp.y, hx * 1.0001f + 1e-4f, hy * 1.0001f + 1e-4f,
                                -1e-4f, bd.z + 1e-4f);
        }
        const int k = warp_append(keep, &sh.nvbox);
        if (keep) m.visbox[k] = (unsigned char)b;
    }
    for (int base = 0; base < wi.n_sig; base += g.nt) {
        const int sg = base + g.tid;
        bool keep = false;
        if (sg < wi.n_sig) {
            const float4 sp = p.sig[wi.sig_begin + sg];
            const float h = sp.w * 1.0001f + 1e-4f;
            keep = aabb_visible(p, cm, sp.x, sp.y, h, h, sp.z - h, sp.z + h);
        }
        const int k = warp_append(keep, &sh.nvsig);
        if (keep) m.vissig[k] = (unsigned char)sg;
    }
    g.sync();
    // packed positions of the visible clusters' quads (warp 0 scans the counts)
    if (g.warp() == 0) {
        const int lane = g.tid & 31, nv = sh.nvcl;
        int run = 0;
        for (int base = 0; base < nv; base += 32) {
            const int c = base + lane;
            const int v = c < nv ? (int)m.vnq[c] : 0;
            int x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (c < nv) m.vpre[c] = run + x - v;
            run += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) sh.nvq = run;
    }
    g.sync();
    if (ST && p.stats && g.tid == 0) {
        atomicAdd(&p.stats[GP_STAT_ITEMS], 1ull);
        atomicAdd(&p.stats[GP_STAT_CLUSTERS], (unsigned long long)sh.nvcl);
        atomicAdd(&p.stats[GP_STAT_BOXES], (unsigned long long)sh.nvbox);
        atomicAdd(&p.stats[GP_STAT_SIGNALS], (unsigned long long)sh.nvsig);
        atomicAdd(&p.stats[GP_STAT_QUADS], (unsigned long long)(sh.nvq + 6 * sh.nvbox + 32 * sh.nvsig));
    }

    // 2. setup: warps pull units until the units run out or the batch is full; then the
    //    batch is handed over; repeat until every unit is placed.
    const int nbox_items = sh.nvbox * 6;  // one box face (two triangles) per lane
    const int n_box_units = (nbox_items + 31) / 32;
    const int nvcl = sh.nvcl, nvq = sh.nvq;
    const int n_sig_units = sh.nvsig;  // one signal sphere (32 faces) per unit
    const int n_units = n_box_units + n_sig_units + (nvq + 31) / 32;
    int pend = -1;            // unit this warp could not place (warp-uniform)
    bool pend_clips = false;  // its clip jobs are already queued
    for (;;) {
        for (;;) {
            int u;
            bool done_clips = false;
            if (pend >= 0) {
                u = pend;
                done_clips = pend_clips;
                pend = -1;
            } else {
                u = 0;
                if ((g.tid & 31) == 0) u = atomicAdd(&sh.next_unit, 1);
                u = __shfl_sync(0xffffffffu, u, 0);
            }
            if (u >= n_units) break;
            bool queued = false;
            if (!setup_unit<ST>(p, cm, sh, m.tris, m.clipq, m.vq0, m.vpre, nvcl, nvq, m.visbox,
                            m.vissig, view, u, n_box_units, nbox_items, n_sig_units, done_clips,
                            queued)) {
                pend = u;
                pend_clips = queued;
                if ((g.tid & 31) == 0) atomicAdd(&sh.npend, 1);
                break;
            }
        }
        g.sync();
        // clip the queued triangles (8 lanes per job), handing the batch over when full
        for (;;) {
            const int nq = sh.cq_n, rv = sh.resv;
            if (nq == 0) break;
            const int room = (p.tri_cap - rv) / 6;
            if (room == 0) {
                m.tris = emit(false);
                if (!m.tris) return false;
                continue;
            }
            const int take = min(nq, room);
            clip_jobs<ST>(p, cm, view, m.clipq + (nq - take), take, m.tris + rv, m.clipscratch, g);
            g.sync();
            if (g.tid == 0) {
                sh.cq_n = nq - take;
                sh.resv = rv + 6 * take;
            }
            g.sync();
        }
        const bool more = sh.next_unit < n_units || sh.npend > 0;
        const bool full = sh.resv > 0;
        g.sync();
        if (g.tid == 0) sh.npend = 0;
        if (!more) {
            m.tris = emit(true);
            return m.tris != nullptr;
        }
        if (full) {
            m.tris = emit(false);
            if (!m.tris) return false;
        } else {
            g.sync();
        }
    }
}

// One block does everything for its items: setup, then raster of each full batch, then
// the encode of the band.
template <bool F32, bool ST>
__global__ void __launch_bounds__(1024, 1) render_kernel(RenderParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Shared sh;
    __shared__ int s_warp[32];
    const Group g{(int)threadIdx.x, (int)blockDim.x, 0};
    const Smem L = smem_layout(p.W, p.band_rows, p.key_f16, g.nt, p.tri_cap, p.max_cl, 0);
    unsigned int *keys = (unsigned int *)(smem + L.keys);  // 8 B per pixel (FP32) or 4 B
    TriRec *tris = (TriRec *)(smem + L.tris);
    int *rowoff = (int *)(smem + L.rowoff);
    unsigned short *map = (unsigned short *)(smem + L.map);
    unsigned char *ftab = smem + L.ftab;
    SetupMem m{tris, (uint32_t *)(smem + L.clipq), (float *)(smem + L.clipscratch),
               (int *)(smem + L.vq0), (int *)(smem + L.vpre), smem + L.vnq,
               smem + L.visbox, smem + L.vissig};

    for (int b = g.tid; b < (F32 ? 2 : 1) * p.band_rows * p.W; b += g.nt) keys[b] = 0;

    Cam cm;
    WorldInfo wi;
    int view = 0;
    auto emit = [&](bool last) -> TriRec * {
        const int n = sh.resv;
        if (n > 0) flush<F32, ST>(p, cm.by0, cm.by1, n, keys, tris, rowoff, map, ftab, s_warp, g);
        if (g.tid == 0) {
            sh.resv = 0;
            // The item's last batch: fetch the next item and reset the block state now, so
            // that after the encode each warp goes straight on to the next item's cull
            // (which touches neither the keys nor this item's camera; the keys are written
            // again only after that cull's barrier).
            if (last) {
                sh.item = p.work_counter ? atomicAdd(p.work_counter, 1) : p.n_items;
                sh.next_unit = 0;
                sh.npend = 0;
                sh.nvcl = 0;
                sh.nvbox = 0;
                sh.nvsig = 0;
                sh.cq_n = 0;
            }
        }
        g.sync();
        if (last) {  // 3. encode and store the band
            if (F32) encode_f32(p, cm, (unsigned long long *)keys, view, g);
            else encode_f16(p, cm, keys, view, g);
        }
        return tris;
    };
    for (int item = next_item(p, sh, 0, g); item < p.n_items; item = sh.item) {
        make_cam(p, item, cm, wi, view);
        produce_item<ST>(p, cm, wi, view, sh, m, g, emit);
    }
}

// What a raster batch of the pipelined kernel carries besides its triangles.
struct BatchMeta {
    int n, view, by0, by1, box_begin, sig_begin;
    uint32_t box_end, road_end, line_end;
    int flags;  // kBatchLast: the item's last batch (encode after it); kBatchEnd: no more work
};
constexpr int kBatchLast = 1, kBatchEnd = 2;

__device__ __forceinline__ uint32_t smem_u32(const void *ptr) {
    return (uint32_t)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    unsigned long long state;
    asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];"
                 : "=l"(state)
                 : "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait until the phase of parity `parity` of an mbarrier completes; false (and a status bit)
// if it does not within wait_ns.  Warp-collective: all 32 lanes call it, poll in lock step
// and return the same answer together, so the warp leaves converged.
__device__ bool mbar_wait(unsigned long long *bar, uint32_t parity, unsigned long long wait_ns,
                          uint32_t *status) {
    bool done = mbar_try_wait(bar, parity);
    if (__all_sync(0xffffffffu, done)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        done = done || mbar_try_wait(bar, parity);
        if (__all_sync(0xffffffffu, done)) return true;
        const bool late = global_ns() - t0 > wait_ns;
        if (__shfl_sync(0xffffffffu, late, 0)) {
            if ((threadIdx.x & 31) == 0) atomicOr(status, GP_DEV_PIPELINE_TIMEOUT);
            return false;
        }
    }
}

// Pipelined variant: the first p.prod_warps warps (producers) cull, set up and clip; the
// other warps (consumers) rasterise and encode.  Two triangle batches alternate between
// them: the producers fill one while the consumers rasterise the other.  Batch s lives in
// buffer s & 1; full[b] completes when the producers have written a batch into buffer b,
// empty[b] when the consumers are done with it.  Each side synchronises internally on its
// own hardware barrier (1 producers, 2 consumers).  Every handoff wait is bounded (p.wait_ns):
// on a timeout the side records it, sets GP_DEV_PIPELINE_TIMEOUT and leaves as a whole, and
// the other side then times out too.
template <bool F32, bool ST>
__global__ void __launch_bounds__(1024, 1) render_kernel_ws(RenderParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Shared sh;
    __shared__ int s_warp[32];
    __shared__ BatchMeta meta[2];
    __shared__ __align__(8) unsigned long long bars[4];  // full[0], full[1], empty[0], empty[1]
    __shared__ int gave_up[3];  // producers; consumers, by parity of the batch they waited for
    const int nprod = 32 * p.prod_warps, ncons = (int)blockDim.x - nprod;
    const Smem L = smem_layout(p.W, p.band_rows, p.key_f16, blockDim.x, p.tri_cap, p.max_cl,
                               p.prod_warps);
    unsigned int *keys = (unsigned int *)(smem + L.keys);
    TriRec *tris0 = (TriRec *)(smem + L.tris);  // two batches of tri_cap records
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], nprod);
        mbar_init(&bars[1], nprod);
        mbar_init(&bars[2], ncons);
        mbar_init(&bars[3], ncons);
        gave_up[0] = 0;
        gave_up[1] = 0;
        gave_up[2] = 0;
    }
    for (int b = threadIdx.x; b < (F32 ? 2 : 1) * p.band_rows * p.W; b += blockDim.x) keys[b] = 0;
    __syncthreads();

    if ((int)threadIdx.x < nprod) {
        if (p.debug_stall) return;  // test mode: the consumers' first wait runs out
        const Group g{(int)threadIdx.x, nprod, 1};
        SetupMem m{tris0, (uint32_t *)(smem + L.clipq), (float *)(smem + L.clipscratch),
                   (int *)(smem + L.vq0), (int *)(smem + L.vpre), smem + L.vnq,
               smem + L.visbox, smem + L.vissig};
        Cam cm;
        WorldInfo wi;
        int view = 0;
        int s = 0;  // batches published
        auto emit = [&](bool last) -> TriRec * {
            // every producer thread has read the batch state it acted on before thread 0
            // changes it
            g.sync();
            const int b = s & 1;
            if (g.tid == 0) {
                meta[b] = BatchMeta{sh.resv, view, cm.by0, cm.by1, cm.box_begin, cm.sig_begin,
                                    cm.box_end, cm.road_end, cm.line_end, last ? kBatchLast : 0};
                sh.resv = 0;
            }
            mbar_arrive(&bars[b]);  // release: this thread's records (and thread 0's meta)
            ++s;
            const int nb = s & 1;
            // batch s - 2 used buffer nb: wait until the consumers are done with it
            if (s >= 2 && !mbar_wait(&bars[2 + nb], (uint32_t)(((s >> 1) - 1) & 1), p.wait_ns,
                                     p.status))
                gave_up[0] = 1;
            g.sync();
            if (gave_up[0]) return nullptr;
            return tris0 + (size_t)nb * p.tri_cap;
        };
        bool ok = true;
        for (int iter = 0;; ++iter) {
            const int item = next_item(p, sh, iter, g);
            if (item >= p.n_items) break;
            make_cam(p, item, cm, wi, view);
            if (!produce_item<ST>(p, cm, wi, view, sh, m, g, emit)) {
                ok = false;
                break;
            }
        }
        if (ok) {  // end marker; its buffer is free (emit waited for it)
            if (g.tid == 0) meta[s & 1].flags = kBatchEnd;
            mbar_arrive(&bars[s & 1]);
        }
    } else {
        const Group g{(int)threadIdx.x - nprod, ncons, 2};
        int *rowoff = (int *)(smem + L.rowoff);
        unsigned short *map = (unsigned short *)(smem + L.map);
        unsigned char *ftab = smem + L.ftab;
        for (int s = 0;; ++s) {
            const int b = s & 1;
            // a flag per batch parity: a thread already waiting for batch s + 1 cannot change
            // the flag the others still read for batch s
            if (!mbar_wait(&bars[b], (uint32_t)((s >> 1) & 1), p.wait_ns, p.status))
                gave_up[1 + b] = 1;
            g.sync();
            if (gave_up[1 + b]) break;
            const BatchMeta mt = meta[b];
            if (mt.flags & kBatchEnd) break;
            if (mt.n > 0)
                flush<F32, ST>(p, mt.by0, mt.by1, mt.n, keys, tris0 + (size_t)b * p.tri_cap, rowoff,
                               map, ftab, s_warp, g);
            mbar_arrive(&bars[2 + b]);  // release: this thread is done reading buffer b
            if (mt.flags & kBatchLast) {
                Cam cm;
                cm.by0 = mt.by0;
                cm.by1 = mt.by1;
                cm.box_begin = mt.box_begin;
                cm.box_end = mt.box_end;
                cm.road_end = mt.road_end;
                cm.line_end = mt.line_end;
                cm.sig_begin = mt.sig_begin;
                if (F32) encode_f32(p, cm, (unsigned long long *)keys, mt.view, g);
                else encode_f16(p, cm, keys, mt.view, g);
                g.sync();
            }
        }
    }
}

}  // namespace

cudaError_t launch_trace(const RenderParams &p, int n_views, cudaStream_t s) {
    const long long plane = (long long)p.H * p.W;
    const int bx = (int)((plane / 4 + 127) / 128);
    for (int v0 = 0; v0 < n_views; v0 += 65535) {
        RenderParams q = p;
        q.trace_view0 = v0;
        const dim3 grid(bx, (unsigned)std::min(65535, n_views - v0));
        if (p.has_signals) trace_kernel<false><<<grid, 128, 0, s>>>(q);
        else trace_kernel<true><<<grid, 128, 0, s>>>(q);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

size_t render_smem_bytes(int W, int band_rows, int key_f16, int threads, int tri_cap, int max_cl,
                         int prod_warps) {
    return smem_layout(W, band_rows, key_f16, threads, tri_cap, max_cl, prod_warps).total;
}

// The signal polyhedron's tables, computed in double on the host and rounded once.
static cudaError_t upload_signal_tables() {
    const double pi = 3.14159265358979323846;
    float lat_c[5], lat_s[5], lon_c[8], lon_s[8];
    double V[5][8][3];
    for (int i = 0; i < 5; ++i) {
        const double th = -0.5 * pi + 0.25 * pi * i;
        const double ct = (i == 0 || i == 4) ? 0.0 : std::cos(th), st = std::sin(th);
        lat_c[i] = (float)ct;
        lat_s[i] = (float)st;
        for (int j = 0; j < 8; ++j) {
            const double ph = 0.25 * pi * j;
            V[i][j][0] = ct * std::cos(ph);
            V[i][j][1] = ct * std::sin(ph);
            V[i][j][2] = st;
        }
    }
    for (int j = 0; j < 8; ++j) {
        lon_c[j] = (float)std::cos(0.25 * pi * j);
        lon_s[j] = (float)std::sin(0.25 * pi * j);
    }
    float4 face[kSignalQuads];
    for (int q = 0; q < kSignalQuads; ++q) {
        const int i = q / 8, j = q % 8, j1 = (j + 1) % 8;
        // three distinct corners of the face: the south-pole band's corners 0 and 1 coincide
        const double *a = V[i][j];
        const double *b = i == 0 ? V[i + 1][j1] : V[i][j1];
        const double *c = i == 0 ? V[i + 1][j] : V[i + 1][j1];
        const double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        const double w[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        double n[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
        const double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (double &x : n) x /= len;
        face[q] = make_float4((float)n[0], (float)n[1], (float)n[2],
                              (float)(n[0] * a[0] + n[1] * a[1] + n[2] * a[2]));
    }
    cudaError_t e;
    if ((e = cudaMemcpyToSymbol(c_lat_c, lat_c, sizeof lat_c)) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_lat_s, lat_s, sizeof lat_s)) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_lon_c, lon_c, sizeof lon_c)) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_lon_s, lon_s, sizeof lon_s)) != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_sig_face, face, sizeof face);
}

cudaError_t render_configure(size_t max_smem) {
    // the ST = true instances count GP_STAT_* events (gp_config.stats)
    const void *fns[8] = {(const void *)render_kernel<true, false>, (const void *)render_kernel<false, false>,
                          (const void *)render_kernel_ws<true, false>, (const void *)render_kernel_ws<false, false>,
                          (const void *)render_kernel<true, true>, (const void *)render_kernel<false, true>,
                          (const void *)render_kernel_ws<true, true>, (const void *)render_kernel_ws<false, true>};
    for (const void *f : fns) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)max_smem);
        if (e != cudaSuccess) return e;
    }
    return upload_signal_tables();
}

static const void *render_fn(int key_f16, int prod_warps) {
    if (prod_warps > 0)
        return key_f16 ? (const void *)render_kernel_ws<false, false> : (const void *)render_kernel_ws<true, false>;
    return key_f16 ? (const void *)render_kernel<false, false> : (const void *)render_kernel<true, false>;
}

int render_occupancy(int key_f16, int threads, size_t smem, int prod_warps) {
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &n, render_fn(key_f16, prod_warps), threads, smem);
    return e == cudaSuccess ? n : 0;
}

cudaError_t launch_render(const RenderParams &p, int blocks, int threads, size_t smem,
                          cudaStream_t s) {
    if (p.n_items <= 0) return cudaSuccess;
    if (p.prod_warps > 0) {
        if (p.stats) {
            if (p.key_f16) render_kernel_ws<false, true><<<blocks, threads, smem, s>>>(p);
            else render_kernel_ws<true, true><<<blocks, threads, smem, s>>>(p);
        } else if (p.key_f16) {
            render_kernel_ws<false, false><<<blocks, threads, smem, s>>>(p);
        } else {
            render_kernel_ws<true, false><<<blocks, threads, smem, s>>>(p);
        }
    } else {
        if (p.stats) {
            if (p.key_f16) render_kernel<false, true><<<blocks, threads, smem, s>>>(p);
            else render_kernel<true, true><<<blocks, threads, smem, s>>>(p);
        } else if (p.key_f16) {
            render_kernel<false, false><<<blocks, threads, smem, s>>>(p);
        } else {
            render_kernel<true, false><<<blocks, threads, smem, s>>>(p);
        }
    }
    return cudaGetLastError();
}

}  // namespace gpk
