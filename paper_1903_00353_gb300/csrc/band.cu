// Extrusion, scan conversion and merge (Sections 5, 8, 9 and 10; Algorithms 1 and 2).
//
// Every feature (face, non-flat edge, non-flat vertex) owns a convex characteristic region
// clipped to the band:
//   face   : prism over the triangle, three side planes with inward normals n x (edge)
//            (Section 8.1), |n.(p - a)| <= w; one extrusion covers both signs;
//   edge   : wedge between the two face normals, (p - a).m1 <= 0, (p - a).m2 <= 0, end caps
//            0 <= t.(p - a) <= L (Section 8.2); the convex / concave side follows from the
//            planes themselves;
//   vertex : {p : (p - v).e_j <= 0 for every incident edge e_j} within the ball |p - v| <= w,
//            the set where no incident edge leads closer than v.  It contains the closest-point
//            region of v for every vertex type, so saddle and ruff vertices (Sections 3.2, 3.3)
//            need no special cone; its sign is taken per point from N_alpha (Section 4.3).
// Each region is a superset of the points whose closest surface point lies on its feature
// (Section 4), so the union covers the band without gaps.
//
// GB300 schedule (replacing the paper's thread-per-extrusion cell loop, Section 9), for a batch of
// one or more (mesh, grid) problems described by a device table of Prob entries:
//   1. bin: every region's integer bounding box is split over 32xTYxTZ-point tiles (8x8 by
//      default; 4x4 and 16x8 for the autotuner) and the (tile, region) pairs, each with the
//      region's box clipped to the tile, are bucketed per tile and type (count, scan, fill;
//      a warp's pairs share one atomic per bin); tiles of all problems share one numbering;
//   2. tile kernel: a persistent grid (4 CTAs of 256 threads per SM) takes work items from one
//      atomic ticket: a band tile plus its share of the empty tiles (band tiles largest first
//      for batches).  A band tile keeps the packed keys (|d| bits << 32 | id << 1 | sign) of
//      its points in shared memory.  Warps take chunks of at most 32 of the tile's regions
//      without block barriers: one lane per region computes its scan axis and per-plane span
//      coefficients (Algorithm 2 restricted to grid lines, with the inclusion tolerance of
//      Section 10), a warp scan numbers the rows, each lane evaluates one row's span, and the
//      span points are flattened across lanes, evaluated against the feature and merged with a
//      shared-memory 64-bit atomicMin (Algorithm 1's min-magnitude rule).  The CTA then writes
//      its tile of the dense output (coalesced 16-byte rows), +inf outside the band, optionally
//      the winners or the compact band list, and queues the few points whose band membership
//      or sign lies inside the FP32 error window.  Empty tiles are written +inf;
//   3. patch kernel: re-decides the queued points in FP64 from the winner's neighbourhood (and
//      appends those it puts in the band to the band list).
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "sdf_internal.cuh"

namespace sdf {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int NT = 256;  // threads per tile CTA (and regions per pass)
enum { FACE = 0, EDGE = 1, VERT = 2 };

struct GridP {
    int nx, ny, nz;
    int kofs;    // index of the first z layer within the whole grid (sdf_grid::k0)
    int ntx, nty, ntz;
    FastDiv div_ntx, div_nty, div_nx, div_ny;  // tile and grid index decomposition
    float ox, oy, oz, h, inv_h;
    float w;     // band half-width: in band iff |d| < w
    float Mg;    // coordinate magnitude of the grid (and w)
    // FP32 error windows (set_windows: from the coordinate magnitude and the mesh's shape terms)
    float derr;  // bound on the FP32 distance error (delta)
    float W;     // candidate cutoff w + delta
    float dlo;   // w - delta: points with |d| in [dlo, W) are re-decided in FP64
    float ds;    // sign window: a candidate whose sign predicate lies within ds (per unit normal) of 0
    float ds2;   //   is marked uncertain; ds2 (edges) and dsv (vertices) add the pseudonormal's
    float dsv;   //   own direction error
    float eps;   // inclusion tolerance of the half-space tests (world units)
};

// The FP32 error windows of a problem (see the derivation in the design notes of this library):
//   delta = (2^-20 M + tau_a + tau_b w) / (1 - 2 tau_b),  i.e.  delta = 2^-20 M + tau_a + tau_b (w + 2 delta),
// with M the largest coordinate magnitude of the grid and the mesh.  2^-20 M = 16 u M bounds the
// rounding of every FP32 plane test, span bound and distance (at most 12.2 u M: the grid point
// carries u M per coordinate, a three-term dot product with p and the plane offset -n.a each
// 3 sqrt(3) u M, and the subtraction u W); tau_a + tau_b W bounds the error of the FP32 normals
// and planes themselves at points within W + eps of the feature (k_face_records).  The inclusion
// tolerance is eps = delta; candidates with FP32 |d| >= W = w + delta are dropped (their true
// distance is >= w), and points whose FP32 winner lies in [w - delta, W) are re-decided in FP64.
// A candidate's sign is certain when its sign predicate (p - q).N exceeds ds |N| (+ ds2 for
// edges, + dsv for vertices), ds = 2 delta: moving p by at most eps into the feature's exact
// region changes (p - q).N^ by at most eps, the FP32 evaluation errs by at most delta (plus the
// pseudonormal's own direction error), and there the sign of the closest feature's predicate
// is the sign of the distance (Baerentzen-Aanaes, Section 4.3); otherwise the candidate is
// marked uncertain and, if it wins, re-decided in FP64.
__host__ __device__ inline void set_windows(GridP &g, float m_mesh, float tau_a, float tau_b, float tau_v) {
    const float M = fmaxf(g.Mg, m_mesh);
    const float tb = fminf(tau_b, 0.25f);
    const float delta = (M * 0x1p-20f + tau_a + tau_b * g.w) / (1.f - 2.f * tb) * 1.0001f;
    const float reach = g.w + 2.f * delta;  // largest distance of an evaluated point from its feature
    g.derr = delta;
    g.eps = delta;
    g.W = g.w + delta;
    g.dlo = g.w - delta;
    g.ds = 2.f * delta;
    g.ds2 = 1.1f * tau_b * reach;
    g.dsv = fminf(tau_v, 1.f) * reach;
}

struct Feat {
    int T, E, V;
    const float4 *face_rec, *face_box, *edge_rec, *vert_rec, *vert_plane;
    const int8_t *edge_class, *vert_class;
    const int32_t *face_vid, *face_edge, *vert_start, *vert_corner;
    const int4 *edge_vf;
    const float *vpos;
    const unsigned *prec;  // the handle's precision terms (DevCounters::prec)
    int skip_saddle;
    int vmode;  // vertex regions of the cell-loop schedule: VM_EXACT, VM_CONE or VM_HEMISPHERE
};

// Packed merge key of a candidate (Algorithm 1's minimum-magnitude rule as one 64-bit minimum):
// |d| bits << 32 | feature id << 2 | sign uncertain << 1 | negative.  Feature ids are < 2^30.
__device__ __forceinline__ unsigned long long make_key(float d, int fid, bool unc, bool neg) {
    return ((unsigned long long)__float_as_uint(d) << 32) | ((unsigned long long)(unsigned)fid << 2) |
           ((unsigned long long)unc << 1) | (unsigned long long)neg;
}
__device__ __forceinline__ int key_fid(unsigned long long key) { return (int)((key >> 2) & 0x3fffffffu); }

// Vertex extrusions (cell-loop schedule only).  VM_EXACT: the exact vertex region of the tile path.
// VM_CONE: the paper's cone (Sections 3.3, 8.3): axis N_alpha, half-angle to the most diverging
// face normal on the positive side of the pseudonormal plane, height w; convex vertices get the
// positive cone, concave ones the negative cone (axis -N_alpha), saddles both (the negative one the
// reflection of the positive one).  VM_HEMISPHERE: the half-balls on the N_alpha side and on the
// -N_alpha side (Section 4.3), by the same class rule.
enum { VM_EXACT = 0, VM_CONE = 1, VM_HEMISPHERE = 2 };

struct PatchEntry {
    long long idx;  // linear grid index inside its problem
    int fid;        // FP32 winner feature
    int prob;       // problem of the batch
};

// one (mesh, grid, outputs) problem of a batch; the single-problem call is a batch of one
struct Prob {
    Feat F;
    GridP g;
    float *dist;
    int32_t *winner;
    int vec;  // rows 16-byte aligned: x-rows of 4 points are stored with one vector store
    // compact band list (null: not requested): one (point index, winner) entry per band point;
    // list_count receives the number of band points, entries at or beyond list_cap are not written
    uint2 *list = nullptr;
    unsigned long long *list_count = nullptr;
    long long list_cap = 0;
    float *list_dist = nullptr;  // nullable: the signed distance of every list entry
};

// largest p in [0, n) with base[p] <= x (base ascending, base[0] = 0)
__device__ __forceinline__ int find_prob(const long long *base, int n, long long x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

struct Outputs {
    const int2 *pairs;
    const uint32_t *bin_start;
    int64_t pair_cap;
    PatchEntry *patch;
    int64_t patch_cap;
    DevCounters *ctr;
    // split tiles (see k_tile_lists): work items, per-slot merged keys and finished-item counts
    const int2 *split_items = nullptr;
    unsigned long long *split_keys = nullptr;
    unsigned *split_done = nullptr;
};

// ----------------------------------------------------------------------------- boxes
__device__ __forceinline__ bool to_index_box(float lx, float ly, float lz, float hx, float hy, float hz,
                                             const GridP &g, int &i0, int &i1, int &j0, int &j1, int &k0, int &k1) {
    const float sl = 1.f / 4096.f;  // index slack against rounding of the conversion
    float a0 = fmaxf((lx - g.ox) * g.inv_h - 0.5f - sl, -1.f), a1 = fminf((hx - g.ox) * g.inv_h - 0.5f + sl, (float)g.nx);
    float b0 = fmaxf((ly - g.oy) * g.inv_h - 0.5f - sl, -1.f), b1 = fminf((hy - g.oy) * g.inv_h - 0.5f + sl, (float)g.ny);
    const float kz = (float)g.kofs;
    float c0 = fmaxf((lz - g.oz) * g.inv_h - 0.5f - kz - sl, -1.f), c1 = fminf((hz - g.oz) * g.inv_h - 0.5f - kz + sl, (float)g.nz);
    i0 = max((int)ceilf(a0), 0); i1 = min((int)floorf(a1), g.nx - 1);
    j0 = max((int)ceilf(b0), 0); j1 = min((int)floorf(b1), g.ny - 1);
    k0 = max((int)ceilf(c0), 0); k1 = min((int)floorf(c1), g.nz - 1);
    return i0 <= i1 && j0 <= j1 && k0 <= k1;
}

__device__ __forceinline__ void box_add(float3 &lo, float3 &hi, float3 p) {
    lo.x = fminf(lo.x, p.x); lo.y = fminf(lo.y, p.y); lo.z = fminf(lo.z, p.z);
    hi.x = fmaxf(hi.x, p.x); hi.y = fmaxf(hi.y, p.y); hi.z = fmaxf(hi.z, p.z);
}

// extent of the spherical cone {y : angle(y, axis) <= theta, |y| <= 1} along +e (unit axis comp. ca)
__device__ __forceinline__ float cone_reach(float ca, float cth, float sth) {
    if (ca >= cth) return 1.f;
    float sa = sqrtf(fmaxf(0.f, 1.f - ca * ca));
    return fmaxf(0.f, ca * cth + sa * sth);  // cos(angle(e, axis) - theta), or the apex
}

// integer box of the clipped region of feature `id` of type TYPE; false if the feature has none.
//   face  : triangle box grown by W |n| per axis (the prism is the triangle swept along +-W n);
//   edge  : segment box plus the box of the sector of radius W between the two face normals
//           (u1, u2 on the region's side), which lies in the kite {0, u1, u2, m / cos(theta/2)};
//   vertex: the spherical cone of the vertex region when one bounds it, else the ball of radius W.
template <int TYPE>
__device__ __forceinline__ bool feature_box(const Feat &F, const GridP &g, int id, int &i0, int &i1, int &j0,
                                            int &j1, int &k0, int &k1) {
    const float R = g.W + g.eps;
    const float slack = R * 1e-5f + g.eps;
    if (TYPE == FACE) {
        float4 n = __ldg(F.face_rec + 4 * id), lo = __ldg(F.face_box + 2 * id), hi = __ldg(F.face_box + 2 * id + 1);
        float ex = R * fabsf(n.x) + slack, ey = R * fabsf(n.y) + slack, ez = R * fabsf(n.z) + slack;
        return to_index_box(lo.x - ex, lo.y - ey, lo.z - ez, hi.x + ex, hi.y + ey, hi.z + ez, g, i0, i1, j0, j1, k0, k1);
    } else if (TYPE == EDGE) {
        const int8_t c = F.edge_class[id];
        if (c == CLS_FLAT) return false;
        const float4 a = __ldg(F.edge_rec + 5 * id), t = __ldg(F.edge_rec + 5 * id + 1);
        const float4 r2 = __ldg(F.edge_rec + 5 * id + 2), r3 = __ldg(F.edge_rec + 5 * id + 3);
        const float3 tt = f3(t);
        // n1 = t x m1, n2 = (-t) x m2 with the stored planes holding -m1, -m2
        float3 u1 = cross3(f3(r2), tt), u2 = cross3(tt, f3(r3));
        if (c == CLS_CONCAVE) { u1 = -1.f * u1; u2 = -1.f * u2; }
        const float3 ms = u1 + u2;
        const float lm = sqrtf(dot3(ms, ms));
        float3 slo = make_float3(0.f, 0.f, 0.f), shi = slo;
        if (lm > 0.2f) {  // sector angle < ~168 degrees: kite bound
            box_add(slo, shi, u1);
            box_add(slo, shi, u2);
            box_add(slo, shi, (2.f / (lm * lm)) * ms);  // m / cos(theta/2), |ms| = 2 cos(theta/2)
        } else {
            slo = make_float3(-1.f, -1.f, -1.f);
            shi = make_float3(1.f, 1.f, 1.f);
        }
        const float bx = fmaf(a.w, t.x, a.x), by = fmaf(a.w, t.y, a.y), bz = fmaf(a.w, t.z, a.z);
        return to_index_box(fminf(a.x, bx) + R * slo.x - slack, fminf(a.y, by) + R * slo.y - slack,
                            fminf(a.z, bz) + R * slo.z - slack, fmaxf(a.x, bx) + R * shi.x + slack,
                            fmaxf(a.y, by) + R * shi.y + slack, fmaxf(a.z, bz) + R * shi.z + slack, g, i0, i1, j0,
                            j1, k0, k1);
    } else {
        const int8_t c = F.vert_class[id];
        if (c == CLS_FLAT || (F.skip_saddle && c == CLS_SADDLE)) return false;
        const float4 v = __ldg(F.vert_rec + 3 * id), cone = __ldg(F.vert_rec + 3 * id + 2);
        float3 lo = make_float3(-1.f, -1.f, -1.f), hi = make_float3(1.f, 1.f, 1.f);
        if (cone.w > -1.f) {
            const float cth = fminf(cone.w, 1.f), sth = sqrtf(fmaxf(0.f, 1.f - cth * cth));
            hi = make_float3(cone_reach(cone.x, cth, sth), cone_reach(cone.y, cth, sth), cone_reach(cone.z, cth, sth));
            lo = make_float3(-cone_reach(-cone.x, cth, sth), -cone_reach(-cone.y, cth, sth),
                             -cone_reach(-cone.z, cth, sth));
        }
        return to_index_box(v.x + R * lo.x - slack, v.y + R * lo.y - slack, v.z + R * lo.z - slack,
                            v.x + R * hi.x + slack, v.y + R * hi.y + slack, v.z + R * hi.z + slack, g, i0, i1, j0,
                            j1, k0, k1);
    }
}

// ----------------------------------------------------------------------------- binning
// The region's integer box clipped to tile (tx, ty, tz), in tile-local indices, packed in 26 bits:
// x lo, hi (5 bits each), y lo, hi, z lo, hi (4 bits each; TY, TZ <= 16).
template <int TY, int TZ>
__device__ __forceinline__ int pack_box(int i0, int i1, int j0, int j1, int k0, int k1, int tx, int ty, int tz) {
    static_assert(TY <= 16 && TZ <= 16, "tile-local box packing");
    const int x0 = tx * TILE_X, y0 = ty * TY, z0 = tz * TZ;
    const int a0 = max(i0 - x0, 0), a1 = min(i1 - x0, TILE_X - 1);
    const int b0 = max(j0 - y0, 0), b1 = min(j1 - y0, TY - 1);
    const int c0 = max(k0 - z0, 0), c1 = min(k1 - z0, TZ - 1);
    return a0 | (a1 << 5) | (b0 << 10) | (b1 << 14) | (c0 << 18) | (c1 << 22);
}

// ----------------------------------------------------------------------------- warp helpers
__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    return v;
}
// number of lanes whose (non-decreasing) inclusive prefix is <= r; valid for r < prefix of lane 31
__device__ __forceinline__ int warp_owner(int incl, int r) {
    int lo = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        int v = __shfl_sync(FULL, incl, lo + s - 1);
        if (v <= r) lo += s;
    }
    return lo;
}

// Binning of the regions into tiles, one thread per feature, its (feature, tile) pairs flattened
// over the warp: in each round every lane takes one pair, lanes whose pairs fall in the same bin
// (neighbouring features share tiles: faces, edges and vertices are numbered in spatial order)
// are grouped by __match_any_sync, and one atomic per group takes their slots.  The count pass
// (FILL false) and the fill pass walk the same pairs; the fill pass takes each bin's slots by
// counting its count back down to 0 (so the counts need no clearing in between, and end cleared).
template <bool FILL, int TY, int TZ>
__global__ void k_bin(const Prob *P, const long long *feat_base, const long long *tile_base, int n, long long f_tot,
                      uint32_t *cnt, const uint32_t *start, int2 *pairs, int64_t pair_cap, DevCounters *ctr) {
    dep_wait();
    dep_next();
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int p = 0, type = 0, fid = 0, ntile = 0;
    int i0 = 0, i1 = -1, j0 = 0, j1 = -1, k0 = 0, k1 = -1;
    if (gid < f_tot) {
        p = find_prob(feat_base, n, gid);
        const Feat &F = P[p].F;
        const GridP &g = P[p].g;
        const int64_t lid = gid - feat_base[p];
        bool ok;
        int id;
        if (lid < F.T) { type = FACE; id = (int)lid; ok = feature_box<FACE>(F, g, id, i0, i1, j0, j1, k0, k1); }
        else if (lid < (int64_t)F.T + F.E) { type = EDGE; id = (int)(lid - F.T); ok = feature_box<EDGE>(F, g, id, i0, i1, j0, j1, k0, k1); }
        else { type = VERT; id = (int)(lid - F.T - F.E); ok = feature_box<VERT>(F, g, id, i0, i1, j0, j1, k0, k1); }
        fid = (int)lid;  // face f -> f, edge e -> T + e, vertex v -> T + E + v (within its problem)
        if (ok)
            ntile = (i1 / TILE_X - i0 / TILE_X + 1) * (j1 / TY - j0 / TY + 1) * (k1 / TZ - k0 / TZ + 1);
    }
    const int incl = warp_incl_scan(ntile);
    const int total = __shfl_sync(FULL, incl, 31);
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int r0 = 0; r0 < total; r0 += 32) {
        const int r = r0 + lane;
        const bool has = r < total;
        const int o = warp_owner(incl, has ? r : total - 1);  // every lane takes part in the search
        const int o_incl = __shfl_sync(FULL, incl, o), o_n = __shfl_sync(FULL, ntile, o);
        const int op = __shfl_sync(FULL, p, o), otype = __shfl_sync(FULL, type, o), ofid = __shfl_sync(FULL, fid, o);
        const int oi0 = __shfl_sync(FULL, i0, o), oi1 = __shfl_sync(FULL, i1, o);
        const int oj0 = __shfl_sync(FULL, j0, o), oj1 = __shfl_sync(FULL, j1, o);
        const int ok0 = __shfl_sync(FULL, k0, o), ok1 = __shfl_sync(FULL, k1, o);
        unsigned long long bin = (1ull << 63) | (unsigned)lane;  // inactive lanes: a group of their own
        int tx = 0, ty = 0, tz = 0;
        if (has) {
            const int k = r - (o_incl - o_n);  // the owner's k-th tile, x fastest
            const int nx = oi1 / TILE_X - oi0 / TILE_X + 1, ny = oj1 / TY - oj0 / TY + 1;
            tx = oi0 / TILE_X + k % nx;
            ty = oj0 / TY + (k / nx) % ny;
            tz = ok0 / TZ + k / (nx * ny);
            const GridP &g = P[op].g;
            const int64_t tile = tile_base[op] + ((int64_t)tz * g.nty + ty) * g.ntx + tx;
            bin = (unsigned long long)(3 * tile + otype);
        }
        const unsigned peers = __match_any_sync(FULL, bin);
        const int leader = __ffs(peers) - 1;
        unsigned base = 0;
        if (has && lane == leader) {
            const unsigned k = (unsigned)__popc(peers);
            base = FILL ? atomicSub(cnt + bin, k) - k : atomicAdd(cnt + bin, k);
        }
        base = __shfl_sync(FULL, base, leader);
        if (FILL && has) {
            const int64_t pos = (int64_t)start[bin] + base + __popc(peers & lt_mask);
            if (pos < pair_cap) pairs[pos] = make_int2(ofid, pack_box<TY, TZ>(oi0, oi1, oj0, oj1, ok0, ok1, tx, ty, tz));
            else atomicOr(&ctr->nb_status, ST_PAIR_OVERFLOW);
        }
    }
}

__device__ __forceinline__ float comp(float4 P, int ax) { return ax == 0 ? P.x : (ax == 1 ? P.y : P.z); }
__device__ __forceinline__ float comp3(float3 P, int ax) { return ax == 0 ? P.x : (ax == 1 ? P.y : P.z); }

// FP32 distance to the triangle boundary (three clamped segments); used for points of the face
// prism's tolerance margin, whose closest triangle point lies on the boundary
__device__ float tri_boundary_dist(float3 p, float3 a, float3 b, float3 c) {
    float best = INFINITY;
    float3 P[3] = {a, b, c};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        float3 s = P[k], ev = P[(k + 1) % 3] - s, u = p - s;
        float t = fminf(fmaxf(dot3(u, ev) / dot3(ev, ev), 0.f), 1.f);
        float3 r = u - t * ev;
        best = fminf(best, dot3(r, r));
    }
    return sqrtf(best);
}

// distance from grid point (i, j, k) to feature `id`, the sign from the feature's pseudonormal
// (face normal / n1 + n2 / N_alpha, Section 4.3), and whether that sign is within the FP32 sign
// window (unc: the predicate (p - q).N is smaller than the window allows, see set_windows)
template <int TYPE>
__device__ __forceinline__ float eval_point(const Feat &F, const GridP &g, int id, int i, int j, int k, bool &neg,
                                            bool &unc) {
    const float3 p = make_float3(fmaf((float)i + 0.5f, g.h, g.ox), fmaf((float)j + 0.5f, g.h, g.oy),
                                 fmaf((float)(k + g.kofs) + 0.5f, g.h, g.oz));
    if (TYPE == FACE) {
        const float4 *r = F.face_rec + 4 * id;
        float4 n = __ldg(r), s1 = __ldg(r + 1), s2 = __ldg(r + 2), s3 = __ldg(r + 3);
        float sd = dot3(f3(n), p) + n.w;
        neg = sd < 0.f;
        unc = fabsf(sd) < g.ds;
        float v1 = dot3(f3(s1), p) + s1.w, v2 = dot3(f3(s2), p) + s2.w, v3 = dot3(f3(s3), p) + s3.w;
        if (v1 >= 0.f && v2 >= 0.f && v3 >= 0.f) return fabsf(sd);
        return tri_boundary_dist(p, load_vpos(F.vpos, F.face_vid[3 * id]), load_vpos(F.vpos, F.face_vid[3 * id + 1]),
                                 load_vpos(F.vpos, F.face_vid[3 * id + 2]));
    } else if (TYPE == EDGE) {
        const float4 *r = F.edge_rec + 5 * id;
        float4 a = __ldg(r), t = __ldg(r + 1), np = __ldg(r + 4);
        float3 u = p - f3(a);
        float s = fminf(fmaxf(dot3(u, f3(t)), 0.f), a.w);
        float3 d = u - s * f3(t);
        const float P = dot3(d, f3(np));
        neg = P < 0.f;
        unc = fabsf(P) < fmaf(g.ds, np.w, g.ds2);
        return sqrtf(dot3(d, d));
    } else {
        float4 v = __ldg(F.vert_rec + 3 * id), nv = __ldg(F.vert_rec + 3 * id + 1);
        float3 u = p - f3(v);
        const float P = dot3(u, f3(nv));
        neg = P < 0.f;
        unc = fabsf(P) < g.ds + g.dsv;
        return sqrtf(dot3(u, u));
    }
}

// ----------------------------------------------------------------------------- type dispatch
__device__ __forceinline__ int feat_type(const Feat &F, int fid) { return fid < F.T ? FACE : (fid < F.T + F.E ? EDGE : VERT); }
__device__ __forceinline__ int feat_local(const Feat &F, int fid, int type) {
    return type == FACE ? fid : (type == EDGE ? fid - F.T : fid - F.T - F.E);
}
__device__ __forceinline__ float eval_any(const Feat &F, const GridP &g, int type, int id, int i, int j, int k,
                                          bool &neg, bool &unc) {
    if (type == FACE) return eval_point<FACE>(F, g, id, i, j, k, neg, unc);
    if (type == EDGE) return eval_point<EDGE>(F, g, id, i, j, k, neg, unc);
    return eval_point<VERT>(F, g, id, i, j, k, neg, unc);
}

// ----------------------------------------------------------------------------- per-tile row coefficients
// For a region and its scan axis a (other axes b < c), every half-space m.p + w >= -eps becomes,
// on the row with relative indices (ib, ic), a bound on the relative index j along a that is
// linear in (ib, ic):  j >= A + B ib + C ic (lower, m_a > 0) or j <= A + B ib + C ic (upper,
// m_a < 0).  When m_a = 0 the half-space is a gate G = A + B ib + C ic >= 0 that opens or empties
// the whole row; it is stored as the lower bound j >= -2^100 G, which is <= 0 (no restriction) for
// G >= 0 and beyond the tile for every G < -2^-95.  Scaling by a power of two is exact, so the
// sign of G is kept; a negative G of smaller magnitude (a row on the plane, inside the inclusion
// tolerance) may leave part of the row open, which only adds candidates.  The vertex ball adds
// |j - j_v| <= sqrt(R^2 - (db0 + ib)^2 - (dc0 + ic)^2) in index units.  The coefficients are
// computed once per (region, tile) and kept in shared memory, lower bounds from the front and
// upper bounds from the back of the region's slots, so a row costs one FMA pair and a min or max
// per plane (unused slots hold the neutral upper bound +1e30, so every row runs all KMAX slots
// without branching).  Vertex regions keep at most MAXVP of their planes: dropping planes only enlarges the
// region, and a point outside the exact vertex region has a strictly closer point on an incident
// edge.  Faces have 5 planes, edges 4.
constexpr int KMAX = 6, MAXVP = 6;
constexpr float Q_NONE = 0.f, Q_EDGE = 1.f, Q_VERT = 2.f;  // kinds of quadratic row bound

template <int TY, int TZ>
struct TileSmem {
    unsigned long long key[TILE_X * TY * TZ];  // packed (|d| bits << 32 | id << 2 | unc << 1 | neg) per point
    float4 coef[NT][KMAX];             // span coefficients (A, B, C, -): nl lower bounds, then upper bounds
    float4 quad[NT][2];                // quadratic bound of a region's rows: vertex ball, edge cylinder
    uint2 rinfo[NT];                   // row set-up of each region, packed (see setup_region)
    int fid[NT];                       // regions of the current pass (global feature ids)
    unsigned char ax[NT];              // scan axis
    unsigned char qkind[NT];           // kind of quadratic row bound: Q_NONE, Q_EDGE or Q_VERT
    unsigned rowq[NT / 32][64];        // per-warp ring of non-empty rows waiting for point evaluation
    int next;                          // next chunk of the tile's regions to hand to a warp
    long long work;
};



__device__ __forceinline__ void add_coef(float4 *E, int &nl, int &nu, float4 P, int ax, int bx, int cx, float pb0,
                                         float pc0, float K, const GridP &g) {
    const float ma = comp(P, ax), mb = comp(P, bx), mc = comp(P, cx);
    const float r0 = fmaf(mb, pb0, fmaf(mc, pc0, P.w)) + g.eps;
    if (ma > 0.f) {
        const float inv = 1.f / ma;
        E[nl++] = make_float4(fmaf(-r0 * inv, g.inv_h, -K), -mb * inv, -mc * inv, 0.f);
    } else if (ma < 0.f) {
        const float inv = 1.f / ma;
        E[KMAX - 1 - nu++] = make_float4(fmaf(-r0 * inv, g.inv_h, -K), -mb * inv, -mc * inv, 0.f);
    } else {
        const float s = -0x1p100f;
        E[nl++] = make_float4(s * r0, s * (mb * g.h), s * (mc * g.h), 0.f);
    }
}

// Points of n (<= 32) queued rows, starting at ring slot q0, flattened over the lanes of the warp:
// distance to the row's feature, and the merge into the tile's keys (Algorithm 1).
template <int TY, int TZ>
__device__ __forceinline__ void eval_rows(const Feat &F, const GridP &g, TileSmem<TY, TZ> &S, const unsigned *Q,
                                          int q0, int n, int x0, int y0, int z0, unsigned &cand) {
    const int lane = threadIdx.x & 31;
    const unsigned e = lane < n ? Q[(q0 + lane) & 63] : 0u;
    const int len = (int)((e >> 13) & 63u);
    const int pincl = warp_incl_scan(len);
    const int ptotal = __shfl_sync(FULL, pincl, 31);
    for (int p0 = 0; p0 < ptotal; p0 += 32) {
        const int pp = p0 + lane;
        const int ro = min(warp_owner(pincl, pp), 31);
        const unsigned re = __shfl_sync(FULL, e, ro);
        const int rfirst = __shfl_sync(FULL, pincl - len, ro);  // points before this row
        if (pp < ptotal) {
            const int slot = (int)(re & 255u);
            const int la = (int)((re >> 8) & 31u) + (pp - rfirst), lb = (int)((re >> 19) & 31u), lc = (int)((re >> 24) & 31u);
            const int ax = S.ax[slot];
            const int lx = ax == 0 ? la : lb;
            const int ly = ax == 1 ? la : (ax == 0 ? lb : lc);
            const int lz = ax == 2 ? la : lc;
            const int fid = S.fid[slot];
            const int type = feat_type(F, fid), id = feat_local(F, fid, type);
            bool neg, unc;
            const float d = eval_any(F, g, type, id, x0 + lx, y0 + ly, z0 + lz, neg, unc);
            if (d < g.W) {
                atomicMin(S.key + (lz * TY + ly) * TILE_X + lx, make_key(d, fid, unc, neg));
                cand++;
            }
        }
    }
}

// Set-up of one region of a band tile (pair q of the tile's list; none when q >= qend) into slot
// `slot` of the tile's shared arrays: its scan axis (the longest side of its box in the tile), its
// row count (returned) and its span coefficients (Algorithm 2's half-spaces as bounds linear in a
// row's two indices, plus the quadratic bound of a vertex ball or an edge cylinder).
template <int TY, int TZ>
__device__ __forceinline__ int setup_region(const Feat &F, const GridP &g, const int2 *pairs, int64_t q, int64_t qend,
                                            int x0, int y0, int z0, TileSmem<TY, TZ> &S, int slot) {
    const float3 org = make_float3(g.ox, g.oy, g.oz);
    int fid = 0, lo[3] = {0, 0, 0}, hi[3] = {-1, -1, -1}, type = FACE, id = 0;
    if (q < qend) {
        const int2 pr = __ldg(pairs + q);
        fid = pr.x;
        type = feat_type(F, fid);
        id = feat_local(F, fid, type);
        const unsigned bx = (unsigned)pr.y;
        lo[0] = x0 + (int)(bx & 31u); hi[0] = x0 + (int)((bx >> 5) & 31u);
        lo[1] = y0 + (int)((bx >> 10) & 15u); hi[1] = y0 + (int)((bx >> 14) & 15u);
        lo[2] = z0 + (int)((bx >> 18) & 15u); hi[2] = z0 + (int)((bx >> 22) & 15u);
    }
    const int n0 = hi[0] - lo[0] + 1, n1 = hi[1] - lo[1] + 1, n2 = hi[2] - lo[2] + 1;
    const int ax = (n0 >= n1 && n0 >= n2) ? 0 : (n1 >= n2 ? 1 : 2);
    const int bx = ax == 0 ? 1 : 0, cx = ax == 2 ? 1 : 2;
    const int nb = bx == 0 ? n0 : n1, nc = cx == 1 ? n1 : n2;
    const int nrows = (n0 > 0 && n1 > 0 && n2 > 0) ? nb * nc : 0;
    const int la = ax == 0 ? lo[0] : (ax == 1 ? lo[1] : lo[2]);
    const int ha = ax == 0 ? hi[0] : (ax == 1 ? hi[1] : hi[2]);
    const int lb = bx == 0 ? lo[0] : lo[1];
    const int lc = cx == 1 ? lo[1] : lo[2];
    S.fid[slot] = fid;
    S.ax[slot] = (unsigned char)ax;
    // tile-local starts: a row's points are (a, b, c) = (lo_a + j, lo_b + ib, lo_c + ic)
    const int loa = la - (ax == 0 ? x0 : (ax == 1 ? y0 : z0));
    const int lob = lb - (bx == 0 ? x0 : y0);
    const int loc = lc - (cx == 1 ? y0 : z0);
    const int nbc = max(nb, 1);
    int nl = 0, nu = 0;
    // quadratic row bound in index units: vertex (j_v, db0, dc0, R^2); edge (Qa, Qb, Qc, R^2),
    // (t_a, t_b, t_c, -) with Q the edge point a seen from the row origin; faces none (their
    // slab planes bound the distance)
    float4 q0v = make_float4(0.f, 0.f, 0.f, 0.f), q1v = make_float4(0.f, 0.f, 0.f, Q_NONE);
    if (nrows > 0) {
        // whole-grid indices of the box's first row (z indices carry the slab's first layer)
        const int la_g = la + (ax == 2 ? g.kofs : 0), lc_g = lc + (cx == 2 ? g.kofs : 0);
        const float pb0 = fmaf((float)lb + 0.5f, g.h, comp3(org, bx));
        const float pc0 = fmaf((float)lc_g + 0.5f, g.h, comp3(org, cx));
        const float K = comp3(org, ax) * g.inv_h + 0.5f + (float)la_g;  // j = (p_a - o_a)/h - 1/2 - lo_a
        float4 *E = S.coef[slot];  // written directly to shared memory
        if (type == FACE) {
            const float4 *r = F.face_rec + 4 * id;
            const float4 n = __ldg(r);
            add_coef(E, nl, nu, make_float4(n.x, n.y, n.z, n.w + g.W), ax, bx, cx, pb0, pc0, K, g);
            add_coef(E, nl, nu, make_float4(-n.x, -n.y, -n.z, g.W - n.w), ax, bx, cx, pb0, pc0, K, g);
            add_coef(E, nl, nu, __ldg(r + 1), ax, bx, cx, pb0, pc0, K, g);
            add_coef(E, nl, nu, __ldg(r + 2), ax, bx, cx, pb0, pc0, K, g);
            add_coef(E, nl, nu, __ldg(r + 3), ax, bx, cx, pb0, pc0, K, g);
        } else if (type == EDGE) {
            const float4 *r = F.edge_rec + 5 * id;
            const float4 a = __ldg(r), tt = __ldg(r + 1);
            add_coef(E, nl, nu, make_float4(tt.x, tt.y, tt.z, -tt.w), ax, bx, cx, pb0, pc0, K, g);
            add_coef(E, nl, nu, make_float4(-tt.x, -tt.y, -tt.z, tt.w + a.w), ax, bx, cx, pb0, pc0, K, g);
            add_coef(E, nl, nu, __ldg(r + 2), ax, bx, cx, pb0, pc0, K, g);
            add_coef(E, nl, nu, __ldg(r + 3), ax, bx, cx, pb0, pc0, K, g);
            // the wedge planes do not bound the distance to the edge line: add the cylinder
            // |(p - a) x t| <= W (+ tolerance and a slack of 1/64 cell), which only removes
            // points the merge would reject (d >= W)
            const float3 av = f3(a), tv = f3(tt);
            const float Rs = (g.W + g.eps) * g.inv_h + 1.f / 64.f;
            q0v = make_float4((comp3(org, ax) - comp3(av, ax)) * g.inv_h + 0.5f + (float)la_g,
                              (pb0 - comp3(av, bx)) * g.inv_h, (pc0 - comp3(av, cx)) * g.inv_h, Rs * Rs);
            q1v = make_float4(comp3(tv, ax), comp3(tv, bx), comp3(tv, cx), Q_EDGE);
        } else {
            const float4 v = __ldg(F.vert_rec + 3 * id), nv = __ldg(F.vert_rec + 3 * id + 1);
            const int s0 = __float_as_int(v.w), cnt = min(__float_as_int(nv.w), MAXVP);
            for (int k = 0; k < cnt; k++)
                add_coef(E, nl, nu, __ldg(F.vert_plane + s0 + k), ax, bx, cx, pb0, pc0, K, g);
            const float3 vv = f3(v);
            const float Rh = (g.W + g.eps) * g.inv_h;
            q0v = make_float4((comp3(vv, ax) - comp3(org, ax)) * g.inv_h - 0.5f - (float)la_g,
                              (pb0 - comp3(vv, bx)) * g.inv_h, (pc0 - comp3(vv, cx)) * g.inv_h, Rh * Rh);
            q1v.w = Q_VERT;
        }
    }
    for (int k = nl; k < KMAX - nu; k++) S.coef[slot][k] = make_float4(1e30f, 0.f, 0.f, 0.f);
    S.quad[slot][0] = q0v;
    S.quad[slot][1] = q1v;
    S.qkind[slot] = (unsigned char)q1v.w;
    // rinfo: x = nb | nl << 8 | span_hi << 12 | lo_a << 17 | lo_b << 22 | lo_c << 27 (tile-local,
    // 5 bits each), y = 1 / nb
    S.rinfo[slot] = make_uint2((unsigned)(nbc | (nl << 8) | (max(ha - la, 0) << 12) | (loa << 17) | (lob << 22) |
                                       (loc << 27)),
                            __float_as_uint(1.f / (float)nbc));
    return nrows;
}

// The span of row `local` (in the region's row order) of the region in slot reg: its length (0 for
// an empty row) and, in `packed`, its queue record slot | start along a << 8 | len << 13 |
// b << 19 | c << 24 (tile-local).
template <int TY, int TZ>
__device__ __forceinline__ int row_span(const TileSmem<TY, TZ> &S, int reg, int local, int &packed) {
    const uint2 ri = S.rinfo[reg];
    const int nbv = (int)(ri.x & 255u), nl = (int)((ri.x >> 8) & 15u);
    const int ic = (int)(((float)local + 0.5f) * __uint_as_float(ri.y));  // exact for these sizes
    const int ib = local - ic * nbv;
    const float fb = (float)ib, fc = (float)ic;
    float lo_f = -1e30f, hi_f = 1e30f;
    bool open = true;
    const float4 *E = S.coef[reg];
#pragma unroll
    for (int k = 0; k < KMAX; k++) {
        const float4 c = E[k];
        const float v = fmaf(c.y, fb, fmaf(c.z, fc, c.x));
        if (k < nl) lo_f = fmaxf(lo_f, v);
        else hi_f = fminf(hi_f, v);
    }
    const int qk = S.qkind[reg];
    if (qk == (int)Q_VERT) {  // ball around the vertex
        const float4 bl = S.quad[reg][0];
        const float db = bl.y + fb, dc = bl.z + fc;
        const float q2 = bl.w - db * db - dc * dc;
        if (q2 < 0.f) {
            open = false;
        } else {
            const float sq = sqrtf(q2);
            lo_f = fmaxf(lo_f, bl.x - sq);
            hi_f = fminf(hi_f, bl.x + sq);
        }
    } else if (qk == (int)Q_EDGE && hi_f - lo_f > 2.f) {
        // cylinder around the edge line, c2 j^2 + c1 j + c0 <= 0: only for spans of more than
        // a few points (long spans come from wide wedges, whose planes leave the radius open)
        const float4 cq = S.quad[reg][0], q1 = S.quad[reg][1];
        const float ub = cq.y + fb, uc = cq.z + fc;
        const float k0 = fmaf(q1.x, cq.x, fmaf(q1.y, ub, q1.z * uc));
        const float c2 = fmaf(-q1.x, q1.x, 1.f);
        const float c1 = 2.f * fmaf(-q1.x, k0, cq.x);
        const float c0 = fmaf(cq.x, cq.x, fmaf(ub, ub, fmaf(uc, uc, fmaf(-k0, k0, -cq.w))));
        if (c2 > 1e-6f) {
            const float disc = fmaf(c1, c1, -4.f * c2 * c0);
            if (disc < 0.f) {
                open = false;
            } else {  // roots by the cancellation-free form
                const float qq = -0.5f * (c1 + copysignf(sqrtf(disc), c1));
                const float r1 = qq / c2, r2 = qq != 0.f ? c0 / qq : r1;
                lo_f = fmaxf(lo_f, fminf(r1, r2));
                hi_f = fminf(hi_f, fmaxf(r1, r2));
            }
        } else if (c1 == 0.f || fabsf(c1) < 1e-6f) {  // the edge runs along the row
            if (c0 > 0.f) open = false;
        } else {  // linear: c1 j + c0 <= 0
            const float r = -c0 / c1;
            if (c1 > 0.f) hi_f = fminf(hi_f, r); else lo_f = fmaxf(lo_f, r);
        }
    }
    const float sl = 1.f / 4096.f;
    const float span_hi = (float)((ri.x >> 12) & 31u);
    const float fa = fminf(fmaxf(lo_f - sl, 0.f), span_hi + 1.f);
    const float fz = fmaxf(fminf(hi_f + sl, span_hi), -1.f);
    const int ja = (int)ceilf(fa), jb = (int)floorf(fz);
    const int len = open ? max(jb - ja + 1, 0) : 0;
    packed = reg | ((int)((ri.x >> 17) & 31u) + ja) << 8 | (len << 13) |
             (((int)((ri.x >> 22) & 31u) + ib) << 19) | (((int)(ri.x >> 27) + ic) << 24);
    return len;
}

// Queue a row (len > 0) in the warp's ring; once 32 rows wait, evaluate their points.
template <int TY, int TZ>
__device__ __forceinline__ void queue_row(const Feat &F, const GridP &g, TileSmem<TY, TZ> &S, int len, int packed,
                                          int &qh, int &qn, int x0, int y0, int z0, unsigned &cand) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned hit = __ballot_sync(FULL, len > 0);
    if (len > 0) S.rowq[warp][(qh + qn + __popc(hit & ((1u << lane) - 1u))) & 63] = (unsigned)packed;
    qn += __popc(hit);
    __syncwarp();
    if (qn >= 32) {
        eval_rows<TY, TZ>(F, g, S, S.rowq[warp], qh, 32, x0, y0, z0, cand);
        qh = (qh + 32) & 63;
        qn -= 32;
    }
}
// the rest of the warp's queue
template <int TY, int TZ>
__device__ __forceinline__ void flush_rows(const Feat &F, const GridP &g, TileSmem<TY, TZ> &S, int &qh, int &qn,
                                           int x0, int y0, int z0, unsigned &cand) {
    const int warp = threadIdx.x >> 5;
    while (qn > 0) {
        const int m = min(qn, 32);
        eval_rows<TY, TZ>(F, g, S, S.rowq[warp], qh, m, x0, y0, z0, cand);
        qh = (qh + m) & 63;
        qn -= m;
    }
}

// All regions of one band tile.  Per region: its box in the tile (packed in the pair by the
// binning), its scan axis, its row count and its span coefficients (setup_region); per row: the
// span (row_span, Algorithm 2 on a grid line); non-empty rows wait in a per-warp queue until 32
// are ready, then their points are flattened over the lanes, evaluated and merged into the tile's
// keys with a shared-memory atomicMin (Algorithm 1, eval_rows).  The warps take equal chunks of
// at most 32 regions (a multiple of the warp count of them, so that a tile with few regions still
// uses every warp) from a shared counter and work on them without block barriers: one lane per
// region sets it up, a warp scan numbers the chunk's rows, and each lane takes one row, found by a
// shuffle search of the scan.  (Handing out a tile's rows block-wide in batches of 32 was measured
// slower on the knot tube and no faster on the torus.)
template <int TY, int TZ>
__device__ void process_band_tile(const Feat &F, const GridP &g, const int2 *pairs, int64_t q0, int64_t q3,
                                  int x0, int y0, int z0, TileSmem<TY, TZ> &S, unsigned &cand, unsigned &rows,
                                  unsigned &hits) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, t = threadIdx.x;
    const int64_t npairs = q3 - q0;
    if (npairs <= 0) return;  // (after a pair-list overflow a band tile may have no stored pairs)
    int qh = 0, qn = 0;       // head and length of this warp's row queue
    const int64_t nchunks = (NT / 32) * ((npairs + NT - 1) / NT);  // >= NT / 32
    const int cs = (int)((npairs + nchunks - 1) / nchunks);          // >= 1: every chunk advances
    for (;;) {
        int chunk = 0;  // this warp's next chunk of the tile's regions
        if (lane == 0) chunk = atomicAdd(&S.next, 1);
        chunk = __shfl_sync(FULL, chunk, 0);
        const int64_t base = q0 + (int64_t)cs * chunk;
        if (base >= q3) break;
        const int nrows = setup_region<TY, TZ>(F, g, pairs, base + lane, min(base + cs, q3), x0, y0, z0, S, t);
        // rows of the warp's regions, numbered by a warp scan
        const int incl = warp_incl_scan(nrows);
        const int R = __shfl_sync(FULL, incl, 31);
        __syncwarp();
        for (int rbase = 0; rbase < R; rbase += 32) {
            const int r = rbase + lane;
            const int own = min(warp_owner(incl, r), 31);  // lane whose region holds row r
            const int r0 = __shfl_sync(FULL, incl - nrows, own);
            int len = 0, packed = 0;
            if (r < R) {
                len = row_span<TY, TZ>(S, warp * 32 + own, r - r0, packed);
                rows++;
                hits += len > 0;
            }
            queue_row<TY, TZ>(F, g, S, len, packed, qh, qn, x0, y0, z0, cand);
        }
        flush_rows<TY, TZ>(F, g, S, qh, qn, x0, y0, z0, cand);  // region slots are rewritten by the next chunk
        __syncwarp();
    }
}

// decode one merged key into the output value / winner, queueing FP64 re-decisions; entry tells
// whether the point goes to the compact band list here (a band point outside the FP32 window)
__device__ __forceinline__ float decode_key(unsigned long long key, const GridP &g, const Outputs &o, int64_t idx,
                                            int prob, int &wid, unsigned &band, bool &overflow, bool &entry) {
    wid = -1;
    entry = false;
    if (key == ~0ull) return INFINITY;
    const float d = __uint_as_float((unsigned)(key >> 32));
    const int fid = key_fid(key);
    float val = INFINITY;
    if (d < g.w) {
        val = (key & 1ull) ? -d : d;
        wid = fid;
        band++;
    }
    const bool window = (key & 2ull) || d >= g.dlo;  // sign uncertain, or near the band edge
    entry = wid >= 0 && !window;
    if (window) {  // inside the FP32 error window: re-decide in FP64
        unsigned long long slot = atomicAdd(&o.ctr->n_patch, 1ull);
        if ((int64_t)slot < o.patch_cap) {
            PatchEntry pe;
            pe.idx = idx;
            pe.fid = fid;
            pe.prob = prob;
            o.patch[slot] = pe;
        } else {
            overflow = true;
        }
    }
    return val;
}

// Append the band-list entries of a band tile.  During the decode each thread marks in emask
// which of its points (bit k: the k-th point of its decode loop) are entries; here every warp
// takes consecutive slots for its entries with one atomicAdd (no block barrier, so the atomic's
// latency overlaps the other warps' work) and its threads write their entries, re-reading the
// winners from the tile's keys, which stay in shared memory until the tile's end.
template <int TY, int TZ>
__device__ __forceinline__ void list_write(const Prob &pr, const TileSmem<TY, TZ> &S, unsigned emask, int x0, int y0,
                                           int z0, bool vec_rows, bool &overflow) {
    const int lane = threadIdx.x & 31;
    const unsigned c = __popc(emask);
    unsigned incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;
    unsigned long long base = 0;
    if (lane == 31) base = atomicAdd(pr.list_count, (unsigned long long)total);
    unsigned long long pos = __shfl_sync(0xffffffffu, base, 31) + incl - c;
    const GridP &g = pr.g;
    const int64_t plane = (int64_t)g.nx * g.ny;
    while (emask) {
        const int k = __ffs(emask) - 1;
        emask &= emask - 1;
        int e, gi, gj, gk;
        if (vec_rows) {  // decode loop: rows r = threadIdx.x / 8 + (k / 4) * (NT / 8), 4 points from x
            const int r = (threadIdx.x >> 3) + (k >> 2) * (NT / 8);
            const int x = (threadIdx.x & 7) * 4 + (k & 3);
            e = r * TILE_X + x;
            gi = x0 + x;
            gj = y0 + r % TY;
            gk = z0 + r / TY;
        } else {  // decode loop: points e = threadIdx.x + k * NT
            e = threadIdx.x + k * NT;
            gi = x0 + e % TILE_X;
            gj = y0 + (e / TILE_X) % TY;
            gk = z0 + e / (TILE_X * TY);
        }
        const int64_t idx = (int64_t)gk * plane + (int64_t)gj * g.nx + gi;
        if ((long long)pos < pr.list_cap) {
            const unsigned long long key = S.key[e];
            pr.list[pos] = make_uint2((uint32_t)idx, (uint32_t)key_fid(key));
            if (pr.list_dist) {
                const float d = __uint_as_float((unsigned)(key >> 32));
                pr.list_dist[pos] = (key & 1ull) ? -d : d;
            }
        } else {
            overflow = true;
        }
        pos++;
    }
}

// Cost class of a band tile with np >= 1 (tile, region) pairs: 15 - floor(log2 np), clamped to
// [0, 15], so class 0 holds the tiles with the most pairs.
constexpr int N_COST_CLASSES = 16;
__device__ __forceinline__ int tile_cost_class(uint32_t np) { return N_COST_CLASSES - 1 - min(15, 31 - __clz(np)); }

__global__ void k_band_flags(const uint32_t *bin_start, int64_t n_tiles, uint32_t *flag, DevCounters *ctr, int lpt) {
    dep_wait();
    dep_next();
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    const uint32_t np = bin_start[3 * t + 3] - bin_start[3 * t];
    flag[t] = np ? 1u : 0u;
    if (lpt && np) atomicAdd(&ctr->tile_hist[tile_cost_class(np)], 1u);
}

// Work list of the tile kernel: first the band tiles (tiles that some region meets), then chunks
// of FILL_CHUNK empty tiles; empty_list comes from one scan of the band flags.  For a batch (lpt)
// the band tiles are listed heaviest cost class first (largest-first order, so that the last work
// items of the persistent kernel are short and its CTAs finish together; within a class the order
// is that of the atomic cursor); for one problem they stay in tile order, where neighbouring
// tiles, taken at the same time, share feature records in L2.  A tile's output depends on neither.
constexpr int FILL_CHUNK = 32;

//
// A band tile with more than SPLIT_MIN pairs (a densely subdivided part of a mesh puts tens of
// thousands of regions into a few tiles) is split: while slots last (split_cap), it takes a slot
// and becomes S = min(ceil(np / SPLIT_PAIRS), SPLIT_MAX_ITEMS) work items, each a contiguous part
// of its pairs, listed in split_items for the SPLIT launch of the tile kernel; its own entry in
// band_list becomes -1 (skipped).  An item packs (tile, slot | item << 12 | S << 20).  Tiles of a
// few thousand pairs (the knot tube at 512^3 has some) stay whole: their split items, run in a
// launch of their own, cost more than they gain.
constexpr int SPLIT_MIN = 8192, SPLIT_PAIRS = 2048, SPLIT_MAX_ITEMS = 64, SPLIT_SLOTS = 256;
// the launch clears tile_hist, tile_cursor, n_split and n_split_items with one memset
static_assert(offsetof(DevCounters, n_split_items) == offsetof(DevCounters, tile_hist) + 33 * sizeof(unsigned),
              "the per-launch tile-list counters must be contiguous");

__global__ void k_tile_lists(const uint32_t *bin_start, int64_t n_tiles, const uint32_t *band_pos,
                             int32_t *band_list, int32_t *empty_list, DevCounters *ctr, int lpt, int2 *split_items,
                             int split_cap) {
    dep_wait();
    dep_next();
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    const uint32_t np = bin_start[3 * t + 3] - bin_start[3 * t];
    if (!np) {
        empty_list[t - band_pos[t]] = (int32_t)t;
        return;
    }
    int32_t entry = (int32_t)t;
    if (np > (uint32_t)SPLIT_MIN && split_cap > 0) {
        const unsigned slot = atomicAdd(&ctr->n_split, 1u);
        if (slot < (unsigned)split_cap) {
            const int S = (int)min((np + SPLIT_PAIRS - 1) / SPLIT_PAIRS, (uint32_t)SPLIT_MAX_ITEMS);
            const unsigned base = atomicAdd(&ctr->n_split_items, (unsigned)S);  // < split_cap * SPLIT_MAX_ITEMS
            for (int i = 0; i < S; i++) split_items[base + i] = make_int2((int)t, (int)(slot | i << 12 | S << 20));
            entry = -1;
        }
    }
    if (!lpt) {
        band_list[band_pos[t]] = entry;
    } else {
        const int c = tile_cost_class(np);
        uint32_t base = 0;
        for (int k = 0; k < c; k++) base += ctr->tile_hist[k];
        band_list[base + atomicAdd(&ctr->tile_cursor[c], 1u)] = entry;
    }
}

// One chunk of empty tiles (tile ids empty_list[e0 .. e1)): +inf, and winner -1 when winners are
// kept.  The problem's sizes and pointers are loaded once per problem met (every tile of a
// single-problem call, and most chunks of a batch, belong to one), so a whole tile costs its index
// arithmetic and, per thread, TY * TZ / 32 coalesced 16-byte stores; tiles cut by the grid's edge
// or rows not 16-byte aligned take the per-point path.
template <int TY, int TZ>
__device__ __forceinline__ void fill_chunk(const Prob *P, const long long *tile_base, int n, const int32_t *empty_list,
                                           int64_t e0, int64_t e1) {
    long long tb_lo = 1, tb_hi = 0;  // tile range of the loaded problem (empty: load on first use)
    int nx = 0, ny = 0, nz = 0, ntx = 0, nty = 0, vec = 0;
    FastDiv dtx, dty;
    float *dist = nullptr;
    int32_t *winner = nullptr;
    const float4 inf4 = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
    for (int64_t e = e0; e < e1; e++) {
        const long long tile = empty_list[e];
        if (tile < tb_lo || tile >= tb_hi) {
            const int p = find_prob(tile_base, n, tile);
            const GridP &g = P[p].g;
            tb_lo = tile_base[p];
            tb_hi = tile_base[p + 1];
            nx = g.nx; ny = g.ny; nz = g.nz; ntx = g.ntx; nty = g.nty;
            dtx = g.div_ntx; dty = g.div_nty;
            dist = P[p].dist;
            winner = P[p].winner;
            vec = P[p].vec;
        }
        if (!dist) continue;  // a sparse problem: no dense field
        const uint32_t tu = (uint32_t)(tile - tb_lo), r1 = dtx.div(tu), tz = dty.div(r1);
        const int x0 = (int)(tu - r1 * (uint32_t)ntx) * TILE_X, y0 = (int)(r1 - tz * (uint32_t)nty) * TY,
                  z0 = (int)tz * TZ;
        const int64_t plane = (int64_t)nx * ny;
        if (vec && x0 + TILE_X <= nx && y0 + TY <= ny && z0 + TZ <= nz) {
            const int64_t org = (int64_t)z0 * plane + (int64_t)y0 * nx + x0 + (threadIdx.x & 7) * 4;
#pragma unroll
            for (int pass = 0; pass < (TY * TZ + NT / 8 - 1) / (NT / 8); pass++) {
                const int r = (int)(threadIdx.x >> 3) + pass * (NT / 8);
                if ((TY * TZ) % (NT / 8) == 0 || r < TY * TZ) {
                    const int64_t idx = org + (int64_t)(r / TY) * plane + (int64_t)(r % TY) * nx;
                    __stcs(reinterpret_cast<float4 *>(dist + idx), inf4);
                    if (winner) __stcs(reinterpret_cast<int4 *>(winner + idx), make_int4(-1, -1, -1, -1));
                }
            }
        } else {
            for (int q = threadIdx.x; q < TILE_X * TY * TZ; q += NT) {
                const int gi = x0 + q % TILE_X, gj = y0 + (q / TILE_X) % TY, gk = z0 + q / (TILE_X * TY);
                if (gi >= nx || gj >= ny || gk >= nz) continue;
                const int64_t idx = (int64_t)gk * plane + (int64_t)gj * nx + gi;
                __stcs(dist + idx, INFINITY);
                if (winner) __stcs(winner + idx, -1);
            }
        }
    }
}

// An item of a split tile: its keys go into the slot's keys in global memory (atomicMin, the same
// minimum as in shared memory); the CTA that finishes the tile's last item takes the merged keys
// back into shared memory (and clears the slot for the next launch) and returns true: it decodes
// the tile.  No CTA waits for another.  Kept out of line, so that the band work of the tile kernel
// compiles as without it (inlined, it cost the kernel about 12 %).
template <int TP>
__device__ __noinline__ bool split_merge(const Outputs &o, unsigned long long *key, int slot, int n_items, int &s_last) {
    unsigned long long *gk = o.split_keys + (size_t)slot * TP;
    for (int e = threadIdx.x; e < TP; e += NT) {
        const unsigned long long kv = key[e];
        if (kv != ~0ull) atomicMin(gk + e, kv);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(o.split_done + slot, 1u) == (unsigned)(n_items - 1) ? 1 : 0;
    __syncthreads();
    if (!s_last) return false;  // (uniform over the CTA)
    __threadfence();
    for (int e = threadIdx.x; e < TP; e += NT) {
        key[e] = __ldcg(gk + e);
        gk[e] = ~0ull;
    }
    if (threadIdx.x == 0) o.split_done[slot] = 0u;
    __syncthreads();
    return true;
}

// Persistent tile kernel over all tiles of all problems of a batch.  Two work queues, each with
// its own atomic ticket: the band tiles (one per item, largest first for batches) and chunks of
// FILL_CHUNK empty tiles.  The CTAs of a fifth of the SMs start on the empty chunks, the others on
// the band tiles, and a CTA whose queue runs dry takes work from the other one.  A band tile merges its
// regions' candidates in shared memory and writes its points; an empty tile is written +inf
// (Algorithm 1's initial value).  The dense output goes out with streaming (evict-first) stores,
// so that the write stream does not push the feature records that the band work reads out of
// L2.  LIST: some problem of the launch writes a compact band list (compiled apart, so that the
// plain kernel carries none of its code).  SPLIT: the launch that works on the items of split
// tiles (k_tile_lists) alone, before the launch of the band tiles and the fill; compiled apart
// too, since the split path in the same kernel cost the band work about 12 %.
template <int TY, int TZ, bool LIST, bool SPLIT>
__global__ void __launch_bounds__(NT, 4) k_tile(const Prob *P, const long long *tile_base, int n, Outputs o,
                                                int64_t n_tiles, const int32_t *band_list,
                                                const int32_t *empty_list, const uint32_t *n_band_ptr,
                                                unsigned long long *ticket, int dense) {
    dep_wait();
    dep_next();
    constexpr int TP = TILE_X * TY * TZ;
    extern __shared__ __align__(16) unsigned char tile_smem[];
    TileSmem<TY, TZ> &S = *reinterpret_cast<TileSmem<TY, TZ> *>(tile_smem);
    __shared__ unsigned s_cand, s_band, s_ovf, s_rows, s_hits, s_pairs;
    __shared__ int s_kind, s_last;
    if (threadIdx.x == 0) { s_cand = 0; s_band = 0; s_ovf = 0; s_rows = 0; s_hits = 0; s_pairs = 0; }
    unsigned cand = 0, band = 0, rows = 0, hits = 0, pairs = 0;
    bool overflow = false, list_ovf = false;
    const int64_t n_band = *n_band_ptr, n_empty = n_tiles - n_band;
    // the items of split tiles (the SPLIT launch's only work; the other launch skips those tiles)
    const int64_t n_items = SPLIT ? min((int64_t)o.ctr->n_split_items, (int64_t)SPLIT_SLOTS * SPLIT_MAX_ITEMS) : 0;
    if (SPLIT) ticket += 2;  // its own ticket
    const int64_t n_chunks = dense && !SPLIT ? (n_empty + FILL_CHUNK - 1) / FILL_CHUNK : 0;  // no field: no +inf fill
    for (;;) {
        if (threadIdx.x == 0) {
            // The CTAs of every fifth SM start on the fill queue, the others on the band tiles.  An
            // SM that writes +inf at full rate slows the band work of its other CTAs nearly as much
            // as the fill is worth, so the fill goes to a few SMs, which take band tiles once it
            // is done (measured on the 2.1 M-triangle knot at 1024^3: 1.91 ms against 2.01 ms with
            // half of the CTAs of every SM filling, and 1.37 ms for the band work alone).
            unsigned smid;
            asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
            const bool filler = smid % 5 == 0;
            long long w = -1;
            int kind = 0;
            for (int q = 0; q < 2 && w < 0; q++) {
                const int k = (q == 0) == filler ? 1 : 0;  // 1: empty chunks, 0: band tiles
                const long long lim = k ? n_chunks : (SPLIT ? n_items : n_band);
                if ((long long)*(volatile unsigned long long *)(ticket + k) >= lim) continue;
                const long long t = (long long)atomicAdd(ticket + k, 1ull);
                if (t < lim) {
                    w = t;
                    kind = k;
                }
            }
            S.work = w;
            s_kind = kind;
        }
        __syncthreads();
        const int64_t w = S.work;
        const int kind = s_kind;
        __syncthreads();
        if (w < 0) break;
        if (kind) {  // a chunk of empty tiles
            fill_chunk<TY, TZ>(P, tile_base, n, empty_list, w * FILL_CHUNK, min((w + 1) * FILL_CHUNK, n_empty));
            continue;
        }
        {  // a band tile, or an item of a split tile
            const bool is_band = true;
            int64_t tile;
            int split_slot = -1, split_i = 0, split_n = 1;
            if (SPLIT) {
                const int2 it = o.split_items[w];
                tile = it.x;
                split_slot = it.y & 0xfff;
                split_i = (it.y >> 12) & 0xff;
                split_n = it.y >> 20;
            } else {
                tile = band_list[w];
                if (tile < 0) continue;  // a split tile's own entry: the SPLIT launch does its work
            }
            const int p = find_prob(tile_base, n, tile);
            const Prob &pr = P[p];
            const GridP &g = pr.g;
            const uint32_t tu = (uint32_t)(tile - tile_base[p]), r1 = g.div_ntx.div(tu), tz = g.div_nty.div(r1);
            const int tx = (int)(tu - r1 * (uint32_t)g.ntx), ty = (int)(r1 - tz * (uint32_t)g.nty);
            const int x0 = tx * TILE_X, y0 = ty * TY, z0 = (int)tz * TZ;
            const int cx1 = min(x0 + TILE_X, g.nx) - 1, cy1 = min(y0 + TY, g.ny) - 1, cz1 = min(z0 + TZ, g.nz) - 1;
            const int64_t plane = (int64_t)g.nx * g.ny;
            float *dist = pr.dist;
            int32_t *winner = pr.winner;
            if (is_band) {
                const uint32_t *st = o.bin_start + 3 * tile;
                int64_t q0 = min((int64_t)st[0], o.pair_cap), q3 = min((int64_t)st[3], o.pair_cap);
                if (SPLIT) {  // this item's contiguous part of the tile's pairs
                    const int64_t np = q3 - q0;
                    const int64_t qa = q0 + np * split_i / split_n, qb = q0 + np * (split_i + 1) / split_n;
                    q0 = qa;
                    q3 = qb;
                }
                for (int e = threadIdx.x; e < TP; e += NT) S.key[e] = ~0ull;
                if (threadIdx.x == 0) S.next = 0;
                __syncthreads();
                process_band_tile<TY, TZ>(pr.F, g, o.pairs, q0, q3, x0, y0, z0, S, cand, rows, hits);
                __syncthreads();  // every merge is in before the decode
                if (threadIdx.x == 0) pairs += (unsigned)(q3 - q0);
                if (SPLIT && !split_merge<TP>(o, S.key, split_slot, split_n, s_last)) continue;
            }
            const bool list = LIST && is_band && pr.list != nullptr;
            const bool vec_rows = pr.vec && cx1 == x0 + TILE_X - 1;
            unsigned emask = 0;  // this thread's points that go to the band list (bit: decode order)
            if (vec_rows) {
                // 8 threads per 32-point row, 4 points each
                for (int r = threadIdx.x >> 3; r < TY * TZ; r += NT / 8) {
                    const int y = r % TY, z = r / TY;
                    const int gj = y0 + y, gk = z0 + z;
                    if (gj > cy1 || gk > cz1) continue;
                    const int x = (threadIdx.x & 7) * 4;
                    const int64_t idx = (int64_t)gk * plane + (int64_t)gj * g.nx + x0 + x;
                    float4 v = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
                    int4 wv = make_int4(-1, -1, -1, -1);
                    if (is_band) {
                        const unsigned long long *kp = S.key + r * TILE_X + x;
                        bool e0, e1, e2, e3;
                        v.x = decode_key(kp[0], g, o, idx, p, wv.x, band, overflow, e0);
                        v.y = decode_key(kp[1], g, o, idx + 1, p, wv.y, band, overflow, e1);
                        v.z = decode_key(kp[2], g, o, idx + 2, p, wv.z, band, overflow, e2);
                        v.w = decode_key(kp[3], g, o, idx + 3, p, wv.w, band, overflow, e3);
                        if (list) {
                            const int sh = 4 * ((r - (int)(threadIdx.x >> 3)) / (NT / 8));
                            emask |= ((unsigned)e0 | (unsigned)e1 << 1 | (unsigned)e2 << 2 | (unsigned)e3 << 3) << sh;
                        }
                    }
                    if (dist) __stcs(reinterpret_cast<float4 *>(dist + idx), v);
                    if (winner) __stcs(reinterpret_cast<int4 *>(winner + idx), wv);
                }
            } else {
                for (int e = threadIdx.x; e < TP; e += NT) {
                    const int x = e % TILE_X, y = (e / TILE_X) % TY, z = e / (TILE_X * TY);
                    const int gi = x0 + x, gj = y0 + y, gk = z0 + z;
                    if (gi > cx1 || gj > cy1 || gk > cz1) continue;
                    const int64_t idx = (int64_t)gk * plane + (int64_t)gj * g.nx + gi;
                    int wid = -1;
                    bool en = false;
                    const float val = is_band ? decode_key(S.key[e], g, o, idx, p, wid, band, overflow, en) : INFINITY;
                    if (list && en) emask |= 1u << ((e - (int)threadIdx.x) / NT);
                    if (dist) __stcs(dist + idx, val);
                    if (winner) __stcs(winner + idx, wid);
                }
            }
            if (list) list_write<TY, TZ>(pr, S, emask, x0, y0, z0, vec_rows, list_ovf);
            if (is_band) __syncthreads();  // keys are reused by the next band tile
        }
    }
    atomicAdd(&s_cand, cand);
    atomicAdd(&s_band, band);
    atomicAdd(&s_rows, rows);
    atomicAdd(&s_hits, hits);
    atomicAdd(&s_pairs, pairs);
    if (overflow) atomicOr(&s_ovf, 1u);
    if (list_ovf) atomicOr(&s_ovf, 2u);
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&o.ctr->n_candidates, (unsigned long long)s_cand);
        atomicAdd(&o.ctr->n_band, (unsigned long long)s_band);
        atomicAdd(&o.ctr->n_rows, (unsigned long long)s_rows);
        atomicAdd(&o.ctr->n_rows_hit, (unsigned long long)s_hits);
        atomicAdd(&o.ctr->n_pairs, (unsigned long long)s_pairs);
        if (s_ovf & 1u) atomicOr(&o.ctr->nb_status, ST_PATCH_OVERFLOW);
        if (s_ovf & 2u) atomicOr(&o.ctr->nb_status, ST_LIST_OVERFLOW);
    }
}

// ----------------------------------------------------------------------------- FP64 re-decision
// closest point of triangle (a, b, c) to p by Voronoi-region classification of the corner,
// edge and face regions; region 0 face, 1 + k edge (corner k -> k+1), 4 + k corner k.  The
// published method of C. Ericson, Real-Time Collision Detection (2005), Section 5.1.5, in FP64.
__device__ double closest_on_tri(double3 p, double3 a, double3 b, double3 c, int &region, double3 &lam) {
    double3 ab = b - a, ac = c - a, ap = p - a;
    double d1 = ddot3(ab, ap), d2 = ddot3(ac, ap);
    double3 r;
    if (d1 <= 0.0 && d2 <= 0.0) { region = 4; lam = make_double3(1, 0, 0); r = ap; return ddot3(r, r); }
    double3 bp = p - b;
    double d3v = ddot3(ab, bp), d4 = ddot3(ac, bp);
    if (d3v >= 0.0 && d4 <= d3v) { region = 5; lam = make_double3(0, 1, 0); r = bp; return ddot3(r, r); }
    double vc = d1 * d4 - d3v * d2;
    if (vc <= 0.0 && d1 >= 0.0 && d3v <= 0.0) {
        double v = d1 / (d1 - d3v);
        region = 1; lam = make_double3(1.0 - v, v, 0);
        r = ap - v * ab;
        return ddot3(r, r);
    }
    double3 cp = p - c;
    double d5 = ddot3(ab, cp), d6 = ddot3(ac, cp);
    if (d6 >= 0.0 && d5 <= d6) { region = 6; lam = make_double3(0, 0, 1); r = cp; return ddot3(r, r); }
    double vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
        double wv = d2 / (d2 - d6);
        region = 3; lam = make_double3(1.0 - wv, 0, wv);
        r = ap - wv * ac;
        return ddot3(r, r);
    }
    double va = d3v * d6 - d5 * d4;
    if (va <= 0.0 && (d4 - d3v) >= 0.0 && (d5 - d6) >= 0.0) {
        double wv = (d4 - d3v) / ((d4 - d3v) + (d5 - d6));
        region = 2; lam = make_double3(0, 1.0 - wv, wv);
        r = bp - wv * (c - b);
        return ddot3(r, r);
    }
    double den = 1.0 / (va + vb + vc);
    double v = vb * den, wv = vc * den;
    region = 0;
    lam = make_double3(1.0 - v - wv, v, wv);
    r = ap - v * ab - wv * ac;
    return ddot3(r, r);
}

__device__ double3 tri_normal64(const Feat &F, int t) {
    double3 a = d3(load_vpos(F.vpos, F.face_vid[3 * t])), b = d3(load_vpos(F.vpos, F.face_vid[3 * t + 1])),
            c = d3(load_vpos(F.vpos, F.face_vid[3 * t + 2]));
    double3 cr = dcross3(b - a, c - a);
    return (1.0 / sqrt(ddot3(cr, cr))) * cr;
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// An FP64 candidate of the re-decision: squared distance, the feature holding the closest point q
// in its relative interior (global feature id: face, edge or vertex), and p - q.
struct Cand64 {
    double d2;
    int id;
    double3 pq;
};

__device__ __forceinline__ bool cand_less(double d2, int id, double bd2, int bid) {
    return d2 < bd2 || (d2 == bd2 && id < bid);
}

// closest point of the closed triangle t (Voronoi regions of closest_on_tri), as a candidate
__device__ __forceinline__ Cand64 face_cand64(const Feat &F, double3 p, int t) {
    const double3 A = d3(load_vpos(F.vpos, F.face_vid[3 * t])), B = d3(load_vpos(F.vpos, F.face_vid[3 * t + 1])),
                  C = d3(load_vpos(F.vpos, F.face_vid[3 * t + 2]));
    int reg;
    double3 lam;
    Cand64 c;
    c.d2 = closest_on_tri(p, A, B, C, reg, lam);
    if (reg == 0) {  // (p - A).n equals (p - q).n for q in the face
        c.id = t;
        c.pq = p - A;
    } else if (reg <= 3) {
        c.id = F.T + F.face_edge[3 * t + reg - 1];
        c.pq = (p - A) - lam.y * (B - A) - lam.z * (C - A);
    } else {
        c.id = F.T + F.E + F.face_vid[3 * t + reg - 4];
        c.pq = p - (reg == 4 ? A : (reg == 5 ? B : C));
    }
    return c;
}

// closest point of the closed edge e (segment va - vb), as a candidate
__device__ __forceinline__ Cand64 edge_cand64(const Feat &F, double3 p, int e) {
    const int4 q = F.edge_vf[e];
    const double3 a = d3(load_vpos(F.vpos, q.x)), b = d3(load_vpos(F.vpos, q.y));
    const double3 ab = b - a, ap = p - a;
    const double t = ddot3(ap, ab) / ddot3(ab, ab);
    Cand64 c;
    if (t <= 0.0) {
        c.id = F.T + F.E + q.x;
        c.pq = ap;
    } else if (t >= 1.0) {
        c.id = F.T + F.E + q.y;
        c.pq = p - b;
    } else {
        c.id = F.T + e;
        c.pq = ap - t * ab;
    }
    c.d2 = ddot3(c.pq, c.pq);
    return c;
}

__device__ __forceinline__ Cand64 vert_cand64(const Feat &F, double3 p, int v) {
    Cand64 c;
    c.id = F.T + F.E + v;
    c.pq = p - d3(load_vpos(F.vpos, v));
    c.d2 = ddot3(c.pq, c.pq);
    return c;
}

// One warp per queued point.  The point's FP32 winner may be wrong by the FP32 error (band edge)
// or carry an uncertain sign; here the exact FP64 minimum is taken over every feature whose
// characteristic region can contain the point: those of the (tile, region) pairs of the point's
// tile whose tile-local box contains it (every region containing the point is listed there, so
// the true closest feature is among them, Section 4).  A first FP32 pass over these candidates
// finds the smallest FP32 distance d0; only candidates within d0 + 3 delta are evaluated in FP64
// (the true closest one's FP32 distance is within delta of the minimum, and d0 is at most delta
// below it, plus the plane distance's under-estimate in the inclusion margin, at most delta).
// Without a pair list (the paper's cell-loop schedule) the candidates are the triangles of the
// fans of the FP32 winner's vertices.  The sign is that of (p - q).N with N the FP64 pseudonormal
// of the feature holding the closest point q (face normal, n1 + n2, or N_alpha, Eq. 8).
template <int TY, int TZ>
__global__ void __launch_bounds__(256) k_patch(const Prob *P, const long long *tile_base, Outputs o) {
    dep_wait();
    dep_next();
    const int lane = threadIdx.x & 31;
    const int64_t wid0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t n = min((int64_t)o.ctr->n_patch, o.patch_cap);
    for (int64_t e = wid0; e < n; e += nwarps) {
        PatchEntry pe = o.patch[e];
        const int64_t idx = pe.idx;
        const int fid = pe.fid;
        const Feat &F = P[pe.prob].F;
        const GridP &g = P[pe.prob].g;
        float *const dist = P[pe.prob].dist;
        int32_t *const winner = P[pe.prob].winner;
        const int64_t plane = (int64_t)g.nx * g.ny;
        int gi, gj, gk;
        if (idx < (int64_t(1) << 31)) {
            const uint32_t iu = (uint32_t)idx, r1 = g.div_nx.div(iu), r2 = g.div_ny.div(r1);
            gi = (int)(iu - r1 * (uint32_t)g.nx);
            gj = (int)(r1 - r2 * (uint32_t)g.ny);
            gk = (int)r2;
        } else {
            gk = (int)(idx / plane);
            gj = (int)((idx - (int64_t)gk * plane) / g.nx);
            gi = (int)(idx - (int64_t)gk * plane - (int64_t)gj * g.nx);
        }
        const double h = g.h;
        const double3 p = make_double3((double)g.ox + (gi + 0.5) * h, (double)g.oy + (gj + 0.5) * h,
                                       (double)g.oz + (gk + g.kofs + 0.5) * h);
        Cand64 best;
        best.d2 = INFINITY;
        best.id = 0x7fffffff;
        best.pq = make_double3(0, 0, 0);
        if (o.pairs) {
            const int tx = gi / TILE_X, ty = gj / TY, tz = gk / TZ;
            const int64_t tile = tile_base[pe.prob] + ((int64_t)tz * g.nty + ty) * g.ntx + tx;
            const uint32_t *st = o.bin_start + 3 * tile;
            const int64_t q0 = min((int64_t)st[0], o.pair_cap), q3 = min((int64_t)st[3], o.pair_cap);
            const unsigned lx = (unsigned)(gi - tx * TILE_X), ly = (unsigned)(gj - ty * TY), lz = (unsigned)(gk - tz * TZ);
            // pass 1: the smallest FP32 distance over the regions whose box holds the point
            float d0 = INFINITY;
            for (int64_t q = q0 + lane; q < q3; q += 32) {
                const int2 pr = __ldg(o.pairs + q);
                const unsigned bx = (unsigned)pr.y;
                if (lx < (bx & 31u) || lx > ((bx >> 5) & 31u) || ly < ((bx >> 10) & 15u) || ly > ((bx >> 14) & 15u) ||
                    lz < ((bx >> 18) & 15u) || lz > ((bx >> 22) & 15u))
                    continue;
                const int type = feat_type(F, pr.x);
                bool neg, unc;
                d0 = fminf(d0, eval_any(F, g, type, feat_local(F, pr.x, type), gi, gj, gk, neg, unc));
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) d0 = fminf(d0, __shfl_xor_sync(FULL, d0, off));
            const float thr = d0 + 3.f * g.derr;
            // pass 2: FP64 closest points of the candidates within the threshold
            for (int64_t q = q0 + lane; q < q3; q += 32) {
                const int2 pr = __ldg(o.pairs + q);
                const unsigned bx = (unsigned)pr.y;
                if (lx < (bx & 31u) || lx > ((bx >> 5) & 31u) || ly < ((bx >> 10) & 15u) || ly > ((bx >> 14) & 15u) ||
                    lz < ((bx >> 18) & 15u) || lz > ((bx >> 22) & 15u))
                    continue;
                const int type = feat_type(F, pr.x), id = feat_local(F, pr.x, type);
                bool neg, unc;
                if (!(eval_any(F, g, type, id, gi, gj, gk, neg, unc) <= thr)) continue;
                const Cand64 c = type == FACE ? face_cand64(F, p, id) : (type == EDGE ? edge_cand64(F, p, id)
                                                                                       : vert_cand64(F, p, id));
                if (cand_less(c.d2, c.id, best.d2, best.id)) best = c;
            }
        } else {
            // the fans of the winner's vertices, concatenated; lanes take one corner (triangle) each
            int vs[3], nv;
            if (fid < F.T) { vs[0] = F.face_vid[3 * fid]; vs[1] = F.face_vid[3 * fid + 1]; vs[2] = F.face_vid[3 * fid + 2]; nv = 3; }
            else if (fid < F.T + F.E) { int4 q = F.edge_vf[fid - F.T]; vs[0] = q.x; vs[1] = q.y; vs[2] = 0; nv = 2; }
            else { vs[0] = fid - F.T - F.E; vs[1] = vs[2] = 0; nv = 1; }
            int c0[3], cn[3];
            for (int a = 0; a < 3; a++) {
                c0[a] = a < nv ? F.vert_start[vs[a]] : 0;
                cn[a] = a < nv ? F.vert_start[vs[a] + 1] - c0[a] : 0;
            }
            const int total = cn[0] + cn[1] + cn[2];
            for (int slot = lane; slot < total; slot += 32) {
                const int a = slot < cn[0] ? 0 : (slot < cn[0] + cn[1] ? 1 : 2);
                const int c = c0[a] + slot - (a == 0 ? 0 : (a == 1 ? cn[0] : cn[0] + cn[1]));
                const Cand64 cd = face_cand64(F, p, F.vert_corner[c] / 3);
                if (cand_less(cd.d2, cd.id, best.d2, best.id)) best = cd;
            }
        }
        // warp argmin over (d2, feature id)
        int src = lane;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double od = __shfl_xor_sync(FULL, best.d2, off);
            const int oid = __shfl_xor_sync(FULL, best.id, off);
            const int os = __shfl_xor_sync(FULL, src, off);
            if (cand_less(od, oid, best.d2, best.id)) { best.d2 = od; best.id = oid; src = os; }
        }
        const double3 pq = make_double3(__shfl_sync(FULL, best.pq.x, src), __shfl_sync(FULL, best.pq.y, src),
                                        __shfl_sync(FULL, best.pq.z, src));
        const int out_id = best.id;
        // The sign: (p - q).N with the feature's stored FP32 pseudonormal (face normal, n1 + n2, unit
        // N_alpha) when that cannot flip it, i.e. when |(p - q).N| exceeds |p - q| times the stored
        // normal's direction error (u for faces and edges, rounded from FP64 normals; tau_v for
        // N_alpha); otherwise the FP64 pseudonormal (Eq. 8 for a vertex).  The fallback is rare: it
        // needs p within about 1e-6 |p - q| of the pseudonormal's plane.
        const double pq2 = ddot3(pq, pq);
        double3 N = make_double3(0, 0, 0);
        double nerr = 0.0;
        if (out_id < F.T) {
            N = d3(f3(__ldg(F.face_rec + 4 * out_id)));
            nerr = 4e-7;
        } else if (out_id < F.T + F.E) {
            N = d3(f3(__ldg(F.edge_rec + 5 * (out_id - F.T) + 4)));
            nerr = 8e-7;
        } else if (out_id != 0x7fffffff) {
            N = d3(f3(__ldg(F.vert_rec + 3 * (out_id - F.T - F.E) + 1)));
            nerr = (double)__uint_as_float(F.prec[PREC_TAU_V]) + 4e-7;
        }
        // |(p - q).N| > 2 nerr |p - q| |N|, squared (no FP64 square roots: they are long sequences
        // on this part's FP64 pipe, which bounds this kernel)
        const double sN = ddot3(pq, N);
        const bool sure = sN * sN > 4.0 * nerr * nerr * pq2 * ddot3(N, N) + 1e-300;
        if (sure) {
            // the stored normal decides
        } else if (out_id < F.T) {
            N = tri_normal64(F, out_id);
        } else if (out_id < F.T + F.E) {
            const int4 q = F.edge_vf[out_id - F.T];
            N = tri_normal64(F, q.z) + tri_normal64(F, q.w);
        } else if (out_id != 0x7fffffff) {
            const int u = out_id - F.T - F.E;
            const int c0 = F.vert_start[u], c1 = F.vert_start[u + 1];
            const double3 Pv = d3(load_vpos(F.vpos, u));
            double3 acc = make_double3(0, 0, 0);
            for (int c = c0 + lane; c < c1; c += 32) {  // N_alpha = sum alpha_i n_i, lanes over the fan
                const int cc = F.vert_corner[c];
                const int ft = cc / 3, kk = cc - 3 * ft;
                double3 e1 = d3(load_vpos(F.vpos, F.face_vid[3 * ft + (kk + 1) % 3])) - Pv;
                double3 e2 = d3(load_vpos(F.vpos, F.face_vid[3 * ft + (kk + 2) % 3])) - Pv;
                double3 cr = dcross3(e1, e2);
                double alpha = atan2(sqrt(ddot3(cr, cr)), ddot3(e1, e2));
                acc = acc + alpha * tri_normal64(F, ft);
            }
            N = make_double3(wsum(acc.x), wsum(acc.y), wsum(acc.z));
        }
        const double s = ddot3(pq, N);
        if (lane == 0) {
            float val = INFINITY;
            int w = -1;
            // |d| < w decided on the squares (w^2 is exact in FP64); the value is the FP32 square root
            // of the FP64 square distance (within an FP32 ulp of the rounded FP64 distance)
            if (best.d2 < (double)g.w * (double)g.w) {
                const float d = sqrtf((float)best.d2);
                val = s < 0.0 ? -d : d;
                w = out_id;
            }
            if (dist) dist[idx] = val;
            if (winner) winner[idx] = w;
            const Prob &pr = P[pe.prob];
            if (pr.list && w >= 0) {
                const unsigned long long pos = atomicAdd(pr.list_count, 1ull);
                if ((long long)pos < pr.list_cap) {
                    pr.list[pos] = make_uint2((uint32_t)idx, (uint32_t)w);
                    if (pr.list_dist) pr.list_dist[pos] = val;
                } else {
                    atomicOr(&o.ctr->nb_status, ST_LIST_OVERFLOW);
                }
            }
        }
    }
}

// The FP32 error windows of every problem of a launch, from its grid and the current precision
// terms of its mesh (set_windows); the first kernel of every narrow-band launch.
__global__ void k_windows(Prob *P, int n) {
    dep_wait();
    dep_next();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const unsigned *pr = P[p].F.prec;
    set_windows(P[p].g, __uint_as_float(pr[PREC_MESH_M]), __uint_as_float(pr[PREC_TAU_A]),
                __uint_as_float(pr[PREC_TAU_B]), __uint_as_float(pr[PREC_TAU_V]));
}

// Start of a tile launch: the FP32 error windows of every problem (set_windows), and the launch's
// bin counts, overflow status, statistics, cost-class counters and work tickets cleared, in one
// launch instead of k_windows and five memsets (each an operation of its own on the stream).
__global__ void k_front(Prob *P, int n, uint32_t *cnt, int64_t n_bins, DevCounters *ctr,
                        unsigned long long *ticket, int n_tickets) {
    dep_wait();
    dep_next();
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (t < n) {
        const unsigned *pr = P[t].F.prec;
        set_windows(P[t].g, __uint_as_float(pr[PREC_MESH_M]), __uint_as_float(pr[PREC_TAU_A]),
                    __uint_as_float(pr[PREC_TAU_B]), __uint_as_float(pr[PREC_TAU_V]));
    }
    if (t == 0) {
        ctr->nb_status = 0;
        unsigned long long *stats = &ctr->n_candidates;  // n_candidates .. n_rows_hit
        for (int k = 0; k < 6; k++) stats[k] = 0;
        for (int k = 0; k < 2 * N_COST_CLASSES + 2; k++) ctr->tile_hist[k] = 0;  // .. n_split_items
        for (int k = 0; k < n_tickets; k++) ticket[k] = 0;
    }
    const int64_t n4 = n_bins / 4;  // cnt is 16-byte aligned
    for (int64_t i = t; i < n4; i += stride) reinterpret_cast<uint4 *>(cnt)[i] = make_uint4(0, 0, 0, 0);
    for (int64_t i = 4 * n4 + t; i < n_bins; i += stride) cnt[i] = 0;
}

inline unsigned nblk(int64_t n, int bt) { return (unsigned)((n + bt - 1) / bt); }

}  // namespace

// ----------------------------------------------------------------------------- the paper's schedule
// The schedule of Section 9, kept for the schedule ablation (SDF_FLAG_CELL_LOOP): one thread per
// characteristic region walks every grid point of the region's box, tests it against the region's
// half-spaces (and the vertex ball) with the inclusion tolerance, and merges the distance into a
// 64-bit key per grid point with a global atomicMin (the paper's atomicCAS loop on a packed value);
// a second kernel decodes every key into the dense output.  Same regions, distances, keys and
// FP64 re-decision as the tile path; only the work decomposition differs.
template <int TYPE>
__device__ __forceinline__ bool region_contains(const Feat &F, const GridP &g, int id, float3 p) {
    const float e = g.eps;
    if (TYPE == FACE) {
        const float4 *r = F.face_rec + 4 * id;
        const float4 n = __ldg(r), s1 = __ldg(r + 1), s2 = __ldg(r + 2), s3 = __ldg(r + 3);
        const float sd = dot3(f3(n), p) + n.w;
        return sd + g.W >= -e && g.W - sd >= -e && dot3(f3(s1), p) + s1.w >= -e && dot3(f3(s2), p) + s2.w >= -e &&
               dot3(f3(s3), p) + s3.w >= -e;
    } else if (TYPE == EDGE) {
        const float4 *r = F.edge_rec + 5 * id;
        const float4 a = __ldg(r), t = __ldg(r + 1), p2 = __ldg(r + 2), p3 = __ldg(r + 3);
        const float tp = dot3(f3(t), p);
        return tp - t.w >= -e && t.w + a.w - tp >= -e && dot3(f3(p2), p) + p2.w >= -e &&
               dot3(f3(p3), p) + p3.w >= -e;
    } else {
        const float4 v = __ldg(F.vert_rec + 3 * id), nv = __ldg(F.vert_rec + 3 * id + 1);
        const float3 u = p - f3(v);
        const float R = g.W + e;
        if (dot3(u, u) > R * R) return false;
        const int s0 = __float_as_int(v.w), cnt = min(__float_as_int(nv.w), MAXVP);
        for (int k = 0; k < cnt; k++) {
            const float4 P = __ldg(F.vert_plane + s0 + k);
            if (dot3(f3(P), p) + P.w < -e) return false;
        }
        return true;
    }
}

// the paper's vertex extrusions: which sides the vertex gets, and the cone's cos(half-angle)
__device__ __forceinline__ bool paper_vertex(const Feat &F, int id, bool &pos, bool &neg, float &cth, float3 &axis) {
    const int8_t c = F.vert_class[id];
    if (c == CLS_FLAT || (F.skip_saddle && c == CLS_SADDLE)) return false;
    pos = c == CLS_CONVEX || c == CLS_SADDLE;
    neg = c == CLS_CONCAVE || c == CLS_SADDLE;
    axis = f3(__ldg(F.vert_rec + 3 * id + 1));  // unit N_alpha
    cth = 1.f;
    if (F.vmode == VM_CONE) {  // most diverging face normal among those on the positive side
        const int s0 = F.vert_start[id], s1 = F.vert_start[id + 1];
        for (int i = s0; i < s1; i++) {
            const float cn = dot3(f3(__ldg(F.face_rec + 4 * (F.vert_corner[i] / 3))), axis);
            if (cn > 0.f) cth = fminf(cth, cn);
        }
    } else {
        cth = 0.f;  // hemisphere: angle 90 degrees
    }
    return pos || neg;
}

template <int TYPE>
__device__ __forceinline__ unsigned walk_region(const Feat &F, const GridP &g, int id, int fid,
                                                unsigned long long *keys) {
    int i0, i1, j0, j1, k0, k1;
    bool vpos = false, vneg = false;
    float vcth = 0.f;
    float3 vaxis = make_float3(0.f, 0.f, 0.f), vv = vaxis;
    if (TYPE == VERT && F.vmode != VM_EXACT) {
        if (!paper_vertex(F, id, vpos, vneg, vcth, vaxis)) return 0;
        vv = f3(__ldg(F.vert_rec + 3 * id));
        const float R = g.W + g.eps + g.eps;
        if (!to_index_box(vv.x - R, vv.y - R, vv.z - R, vv.x + R, vv.y + R, vv.z + R, g, i0, i1, j0, j1, k0, k1))
            return 0;
    } else if (!feature_box<TYPE>(F, g, id, i0, i1, j0, j1, k0, k1)) {
        return 0;
    }
    unsigned cand = 0;
    for (int k = k0; k <= k1; k++)
        for (int j = j0; j <= j1; j++)
            for (int i = i0; i <= i1; i++) {
                const float3 p = make_float3(fmaf((float)i + 0.5f, g.h, g.ox), fmaf((float)j + 0.5f, g.h, g.oy),
                                             fmaf((float)(k + g.kofs) + 0.5f, g.h, g.oz));
                if (TYPE == VERT && F.vmode != VM_EXACT) {
                    const float3 u = p - vv;
                    const float R = g.W + g.eps, lu2 = dot3(u, u);
                    if (lu2 > R * R) continue;
                    const float ua = dot3(u, vaxis), lim = sqrtf(lu2) * vcth - g.eps;
                    if (!((vpos && ua >= lim) || (vneg && -ua >= lim))) continue;
                } else if (!region_contains<TYPE>(F, g, id, p)) {
                    continue;
                }
                bool neg, unc;
                const float d = eval_point<TYPE>(F, g, id, i, j, k, neg, unc);
                if (d < g.W) {
                    atomicMin(keys + ((int64_t)k * g.ny + j) * g.nx + i, make_key(d, fid, unc, neg));
                    cand++;
                }
            }
    return cand;
}

__global__ void k_cell_loop(const Prob *P, const long long *feat_base, const long long *pbase, int n, long long f_tot,
                            unsigned long long *keys, DevCounters *ctr) {
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned cand = 0;
    if (gid < f_tot) {
        const int p = find_prob(feat_base, n, gid);
        const Feat &F = P[p].F;
        const GridP &g = P[p].g;
        const int64_t lid = gid - feat_base[p];
        unsigned long long *kp = keys + pbase[p];
        if (lid < F.T) cand = walk_region<FACE>(F, g, (int)lid, (int)lid, kp);
        else if (lid < (int64_t)F.T + F.E) cand = walk_region<EDGE>(F, g, (int)(lid - F.T), (int)lid, kp);
        else cand = walk_region<VERT>(F, g, (int)(lid - F.T - F.E), (int)lid, kp);
    }
    const unsigned c = __reduce_add_sync(0xffffffffu, cand);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&ctr->n_candidates, (unsigned long long)c);
}

// every grid point of every problem: its key to the dense output (and the FP64 queue)
__global__ void k_decode_keys(const Prob *P, const long long *pbase, int n, long long p_tot,
                              const unsigned long long *keys, Outputs o) {
    unsigned band = 0;
    bool overflow = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < p_tot; q += stride) {
        const int p = find_prob(pbase, n, q);
        const int64_t idx = q - pbase[p];
        int wid = -1;
        bool en;
        const float v = decode_key(__ldg(keys + q), P[p].g, o, idx, p, wid, band, overflow, en);
        __stcs(P[p].dist + idx, v);
        if (P[p].winner) __stcs(P[p].winner + idx, wid);
    }
    const unsigned b = __reduce_add_sync(0xffffffffu, band);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(&o.ctr->n_band, (unsigned long long)b);
    if (overflow) atomicOr(&o.ctr->nb_status, ST_PATCH_OVERFLOW);
}

// ----------------------------------------------------------------------------- host side
// Tile shapes the kernels are instantiated for: 32 x TY x TZ points.  8 x 8 is the default; a
// batch created with SDF_FLAG_AUTOTUNE times all of them on its own problems and keeps the fastest.
constexpr int N_SHAPES = 3;
static const int SHAPE_TY[N_SHAPES] = {8, 4, 16};
static const int SHAPE_TZ[N_SHAPES] = {8, 4, 8};

static int make_grid(const sdf_grid &gr, float w, int shape, GridP &g) {
    if (gr.nx < 1 || gr.ny < 1 || gr.nz < 1 || !(gr.h > 0.f) || !isfinite(gr.h) || !(w > 0.f) || !isfinite(w) ||
        gr.k0 < 0 || (int64_t)gr.k0 + gr.nz >= (int64_t(1) << 24))
        return SDF_ERR_INVALID_ARG;
    for (int j = 0; j < 3; j++)
        if (!isfinite(gr.origin[j])) return SDF_ERR_INVALID_ARG;
    if ((int64_t)gr.nx * gr.ny >= (int64_t(1) << 40)) return SDF_ERR_TOO_LARGE;
    g.nx = gr.nx; g.ny = gr.ny; g.nz = gr.nz;
    g.kofs = gr.k0;
    g.ntx = (gr.nx + TILE_X - 1) / TILE_X;
    g.nty = (gr.ny + SHAPE_TY[shape] - 1) / SHAPE_TY[shape];
    g.ntz = (gr.nz + SHAPE_TZ[shape] - 1) / SHAPE_TZ[shape];
    if ((int64_t)g.ntx * g.nty * g.ntz * 3 >= (int64_t(1) << 31)) return SDF_ERR_TOO_LARGE;
    g.div_ntx = FastDiv((uint32_t)g.ntx);
    g.div_nty = FastDiv((uint32_t)g.nty);
    g.div_nx = FastDiv((uint32_t)gr.nx);
    g.div_ny = FastDiv((uint32_t)gr.ny);
    g.ox = gr.origin[0]; g.oy = gr.origin[1]; g.oz = gr.origin[2];
    g.h = gr.h;
    g.inv_h = 1.0f / gr.h;
    // coordinate magnitude M of the problem: FP32 errors of dot products scale with it
    double M = 0.0;
    for (int j = 0; j < 3; j++) {
        const int lo = j == 2 ? gr.k0 : 0, n = j == 0 ? gr.nx : (j == 1 ? gr.ny : gr.nz);
        M = fmax(M, fabs((double)gr.origin[j] + (double)lo * gr.h));
        M = fmax(M, fabs((double)gr.origin[j] + (double)(lo + n) * gr.h));
    }
    M = fmax(M, (double)w);
    g.w = w;
    g.Mg = (float)M;
    // provisional windows of the grid alone; every launch finalises them on the device with the
    // mesh's current precision terms (k_windows)
    set_windows(g, 0.f, 0.f, 0.f, 0.f);
    return SDF_OK;
}

// Expected number of (tile, region) pairs of one problem, from the build's face-box moments, so
// that a call that does not synchronise (and so cannot grow its scratch and repeat) starts with
// enough room on meshes of large triangles.  A box of extent e cells meets about e / t + 1 tiles of
// t cells along an axis; a face's region box lies within its bounding box widened by the band
// (plus one cell of rounding), so a face meets about prod_a (b_a / (h t_a) + c_a) tiles with
// c_a = (2 w / h + 1) / t_a + 1, which the moments sum over the faces.  Every edge's box lies in the
// box of either of its faces (1.5 edges per face), and a vertex's box is a cube of side 2 w.
static int64_t pair_estimate(const sdf_features_s *f, const GridP &g, int shape) {
    const double h = g.h, w = 1.001 * g.w;
    const double t[3] = {(double)TILE_X, (double)SHAPE_TY[shape], (double)SHAPE_TZ[shape]};
    double c[3], sc[3];
    for (int a = 0; a < 3; a++) {
        c[a] = (2.0 * w / h + 1.0) / t[a] + 1.0;
        sc[a] = 1.0 / (h * t[a]);
    }
    const double *M = f->box_mom;  // bx, by, bz, bx by, bx bz, by bz, bx by bz
    const double faces = sc[0] * sc[1] * sc[2] * M[6] + sc[0] * sc[1] * c[2] * M[3] + sc[0] * c[1] * sc[2] * M[4] +
                         c[0] * sc[1] * sc[2] * M[5] + sc[0] * c[1] * c[2] * M[0] + c[0] * sc[1] * c[2] * M[1] +
                         c[0] * c[1] * sc[2] * M[2] + c[0] * c[1] * c[2] * (double)f->T;
    const double est = 2.5 * faces + c[0] * c[1] * c[2] * (double)f->V;
    return est < 2147483648.0 ? (int64_t)est : (int64_t(1) << 31);  // pair positions are 32-bit
}

static Feat make_feat(const sdf_features_s *f) {
    Feat F;
    F.T = (int)f->T; F.E = (int)f->E; F.V = (int)f->V;
    F.face_rec = f->face_rec; F.face_box = f->face_box; F.edge_rec = f->edge_rec;
    F.vert_rec = f->vert_rec; F.vert_plane = f->vert_plane;
    F.edge_class = f->edge_class; F.vert_class = f->vert_class;
    F.face_vid = f->face_vid; F.face_edge = f->face_edge; F.vert_start = f->vert_start;
    F.vert_corner = f->vert_corner; F.edge_vf = f->edge_vf; F.vpos = f->vpos;
    F.prec = f->ctr->prec;
    F.skip_saddle = (f->flags & SDF_FLAG_DISABLE_SADDLE) ? 1 : 0;
    F.vmode = VM_EXACT;
    return F;
}

static int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 152;
    }
    return n;
}

template <int TY, int TZ, bool LIST, bool SPLIT = false> static int tile_blocks_per_sm() {
    static int b = 0;
    if (!b) {
        cudaFuncSetAttribute(k_tile<TY, TZ, LIST, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(TileSmem<TY, TZ>));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_tile<TY, TZ, LIST, SPLIT>, NT, sizeof(TileSmem<TY, TZ>));
        if (b <= 0) b = 1;
    }
    return b;
}

// CTAs of k_patch resident at once on the device: its grid, so that its grid-stride loop over the
// queued points runs in a single wave
template <int TY, int TZ> static int patch_blocks() {
    static int b = 0;
    if (!b) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_patch<TY, TZ>, 256, 0);
        if (b <= 0) b = 1;
        b *= num_sms();
    }
    return b;
}

// an event record that becomes an event node (with its timestamp) when the stream is being captured
static cudaError_t record_event(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t err = cudaStreamIsCapturing(s, &cs);
    if (err != cudaSuccess) return err;
    return cudaEventRecordWithFlags(e, s, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                             : cudaEventRecordDefault);
}

int ensure_events(sdf_features_s *f) {
    for (int i = 0; i < 6; i++)
        if (!f->ev[i]) SDF_TRY(cudaEventCreate(&f->ev[i]));
    return SDF_OK;
}

int resolve_timing(sdf_features_s *f) {
    if (f->fwd_pending) {
        SDF_TRY(cudaEventSynchronize(f->ev[3]));
        for (int i = 0; i < 3; i++) {
            float ms = 0.f;
            SDF_TRY(cudaEventElapsedTime(&ms, f->ev[i], f->ev[i + 1]));
            f->t_ms[i] += ms;
            f->t_calls[i]++;
        }
        f->fwd_pending = false;
    }
    if (f->adj_pending) {
        SDF_TRY(cudaEventSynchronize(f->ev[5]));
        float ms = 0.f;
        SDF_TRY(cudaEventElapsedTime(&ms, f->ev[4], f->ev[5]));
        f->t_ms[3] += ms;
        f->t_calls[3]++;
        f->adj_pending = false;
    }
    return SDF_OK;
}

// A batch of (mesh, grid, outputs) problems: host description, device tables and scratch.
struct Plan {
    int n = 0, shape = 0;
    std::vector<Prob> probs;
    std::vector<long long> fbase, tbase;  // prefix sums of features and tiles over the problems
    long long f_tot = 0, n_tiles = 0;
    // sign beyond the band (SDF_FLAG_FILL_SIGN): output table, prefix sums of x-rows, z- and y-lines
    bool fill = false;
    std::vector<FillProb> fprobs;
    std::vector<long long> rbase, zbase, ybase;
    long long r_tot = 0, z_tot = 0, y_tot = 0;
    // the paper's schedule (SDF_FLAG_CELL_LOOP): prefix sums of grid points, one key per point
    bool cell_loop = false;
    int vmode = VM_EXACT;
    std::vector<long long> pbase;
    long long p_tot = 0;
    DevBuf tables, bins, pairs, patch, scan_tmp, lists, rowsign, keys, split;
    DevCounters *ctr = nullptr;
    bool own_ctr = false;
    int64_t pair_cap = 0, patch_cap = 0;
    int64_t pair_est = 0;  // expected (tile, region) pairs of the described problems (pair_estimate)
    double tuned_ms = 0.0;
    sdf_features_s *events = nullptr;  // handle whose events time the stages (SDF_FLAG_TIMING)
    // the last uploaded table (host copy), the device address it went to, and a pinned staging
    // buffer with an event marking the end of its last copy
    std::vector<char> uploaded;
    const void *uploaded_to = nullptr;
    char *pinned = nullptr;
    size_t pinned_bytes = 0;
    cudaEvent_t pinned_ev = nullptr;
    bool pageable = false;  // one-shot plans copy the table from pageable memory
    bool batch_timing = false;  // record bev[0..3] around the stages of every launch
    cudaEvent_t bev[4] = {nullptr, nullptr, nullptr, nullptr};
};

// Pinned staging blocks for the problem tables, kept for reuse by later plans (a plan per handle
// is created on the first call, and pinning host memory is slow).  A block is returned only after
// its last copy has completed.
static std::mutex g_pin_mu;
static std::vector<std::pair<char *, size_t>> g_pin_free;

static cudaError_t pinned_get(size_t bytes, char **p, size_t *got) {
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        for (size_t i = 0; i < g_pin_free.size(); i++)
            if (g_pin_free[i].second >= bytes) {
                *p = g_pin_free[i].first;
                *got = g_pin_free[i].second;
                g_pin_free.erase(g_pin_free.begin() + (long)i);
                return cudaSuccess;
            }
    }
    const size_t want = bytes < 4096 ? 4096 : bytes;
    count_host_alloc();
    cudaError_t e = cudaMallocHost(reinterpret_cast<void **>(p), want);
    *got = e == cudaSuccess ? want : 0;
    return e;
}

static void pinned_put(char *p, size_t bytes) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (g_pin_free.size() < 64) g_pin_free.emplace_back(p, bytes);
    else cudaFreeHost(p);
}

void plan_free(Plan *pl, cudaStream_t s) {
    if (!pl) return;
    pl->tables.release(s);
    pl->bins.release(s);
    pl->pairs.release(s);
    pl->patch.release(s);
    pl->split.release(s);
    pl->scan_tmp.release(s);
    pl->lists.release(s);
    pl->rowsign.release(s);
    pl->keys.release(s);
    if (pl->own_ctr && pl->ctr) pool_free(pl->ctr, s);
    if (pl->pinned_ev) {
        cudaEventSynchronize(pl->pinned_ev);
        cudaEventDestroy(pl->pinned_ev);
    }
    pinned_put(pl->pinned, pl->pinned_bytes);
    for (cudaEvent_t e : pl->bev)
        if (e) cudaEventDestroy(e);
    delete pl;
}

// Plans of destroyed handles, kept with their scratch for the next handle's first call on the same
// device (a handle per step, as in a loop that rebuilds its mesh, would otherwise allocate the
// pair list, the bins and the lists afresh every step: 0.3-0.5 ms of host time for the 2.1 M-
// triangle knot tube at 1024^3, against 0.07 ms with the scratch in place).  At most two per device.
static std::mutex g_park_mu;
static std::vector<std::pair<int, Plan *>> g_parked;

void plan_park(Plan *pl, cudaStream_t s) {
    if (!pl) return;
    int dev = -1;
    if (pl->own_ctr || pl->batch_timing || cudaGetDevice(&dev) != cudaSuccess) {
        plan_free(pl, s);
        return;
    }
    pl->ctr = nullptr;
    pl->events = nullptr;
    pl->uploaded.clear();
    pl->uploaded_to = nullptr;
    pl->keys.release(s);  // the cell-loop schedule's 8 bytes per grid point are not kept
    Plan *evict = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_park_mu);
        int same = 0;
        for (auto &e : g_parked) same += e.first == dev;
        if (same >= 2) {
            for (auto it = g_parked.begin(); it != g_parked.end(); ++it)
                if (it->first == dev) {
                    evict = it->second;
                    g_parked.erase(it);
                    break;
                }
        }
        g_parked.emplace_back(dev, pl);
    }
    if (evict) plan_free(evict, s);
}

// a parked plan of the current device for a handle's first call, or a new one
static Plan *plan_take() {
    int dev = -1;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        std::lock_guard<std::mutex> lk(g_park_mu);
        for (auto it = g_parked.rbegin(); it != g_parked.rend(); ++it)
            if (it->first == dev) {
                Plan *pl = it->second;
                g_parked.erase(std::next(it).base());
                return pl;
            }
    }
    return new Plan();
}

static int plan_describe(Plan &pl, const sdf_features *feats, const sdf_grid *grids, const float *band_w, int n,
                         float *const *out_dist, int32_t *const *out_winner, int shape, bool fill,
                         const ListOut *lists = nullptr) {
    if (!feats || !grids || !band_w || n < 1 || !out_dist) return SDF_ERR_INVALID_ARG;
    pl.n = n;
    pl.shape = shape;
    pl.fill = fill;
    pl.probs.resize(n);
    pl.fbase.assign(n + 1, 0);
    pl.tbase.assign(n + 1, 0);
    pl.fprobs.resize(n);
    pl.rbase.assign(n + 1, 0);
    pl.zbase.assign(n + 1, 0);
    pl.ybase.assign(n + 1, 0);
    pl.pbase.assign(n + 1, 0);
    pl.pair_est = 0;
    for (int p = 0; p < n; p++) {
        // the dense field may be left out only by a sparse forward (a list with its distances)
        const bool sparse = lists && lists[p].list && lists[p].dist;
        if (!feats[p] || (!out_dist[p] && !sparse) || (!out_dist[p] && fill)) return SDF_ERR_INVALID_ARG;
        Prob &pr = pl.probs[p];
        int st = make_grid(grids[p], band_w[p], shape, pr.g);
        if (st) return st;
        pr.F = make_feat(feats[p]);
        pr.F.vmode = pl.vmode;
        pl.pair_est += pair_estimate(feats[p], pr.g, shape);
        pr.dist = out_dist[p];
        pr.winner = out_winner ? out_winner[p] : nullptr;
        pr.vec = ((pr.g.nx & 3) == 0) && ((reinterpret_cast<uintptr_t>(pr.dist) & 15) == 0) &&
                 ((reinterpret_cast<uintptr_t>(pr.winner) & 15) == 0);
        pr.list = nullptr;
        pr.list_count = nullptr;
        pr.list_cap = 0;
        pr.list_dist = nullptr;
        if (lists && lists[p].list) {
            // entries hold 32-bit point indices; the paper's own schedule writes no list
            if (!lists[p].count || lists[p].cap < 0 || pl.cell_loop) return SDF_ERR_INVALID_ARG;
            if ((long long)grids[p].nx * grids[p].ny * grids[p].nz > (long long)UINT32_MAX) return SDF_ERR_TOO_LARGE;
            pr.list = reinterpret_cast<uint2 *>(lists[p].list);
            pr.list_count = lists[p].count;
            pr.list_cap = lists[p].cap;
            pr.list_dist = lists[p].dist;
        }
        if (feats[p]->T + feats[p]->E + feats[p]->V >= (int64_t(1) << 30)) return SDF_ERR_TOO_LARGE;  // key ids
        pl.fbase[p + 1] = pl.fbase[p] + feats[p]->T + feats[p]->E + feats[p]->V;
        pl.tbase[p + 1] = pl.tbase[p] + (long long)pr.g.ntx * pr.g.nty * pr.g.ntz;
        // the fill's argument (rows outside the band run uncrossed) needs w > h, and the whole grid
        if (fill && (!(band_w[p] > grids[p].h) || grids[p].k0 != 0)) return SDF_ERR_INVALID_ARG;
        pl.fprobs[p] = FillProb{out_dist[p], grids[p].nx, grids[p].ny, grids[p].nz};
        pl.rbase[p + 1] = pl.rbase[p] + (long long)grids[p].ny * grids[p].nz;
        pl.zbase[p + 1] = pl.zbase[p] + grids[p].nz;
        pl.ybase[p + 1] = pl.ybase[p] + grids[p].ny;
        pl.pbase[p + 1] = pl.pbase[p] + (long long)grids[p].nx * grids[p].ny * grids[p].nz;
    }
    pl.f_tot = pl.fbase[n];
    pl.n_tiles = pl.tbase[n];
    pl.r_tot = pl.rbase[n];
    pl.z_tot = pl.zbase[n];
    pl.y_tot = pl.ybase[n];
    pl.p_tot = pl.pbase[n];
    if (3 * pl.n_tiles >= (int64_t(1) << 31) || pl.f_tot >= (int64_t(1) << 31)) return SDF_ERR_TOO_LARGE;
    return SDF_OK;
}

// Layout of a plan's split-tile buffer: the keys of SPLIT_SLOTS tiles (sized for the largest tile
// shape), the work items, the finished-item counts.
static constexpr size_t SPLIT_TP_MAX = (size_t)TILE_X * 16 * 8;
static constexpr size_t split_items_offset() { return sizeof(unsigned long long) * SPLIT_TP_MAX * SPLIT_SLOTS; }
static constexpr size_t split_done_offset() {
    return split_items_offset() + sizeof(int2) * (size_t)SPLIT_SLOTS * SPLIT_MAX_ITEMS;
}
static constexpr size_t split_bytes() { return split_done_offset() + sizeof(unsigned) * SPLIT_SLOTS; }

// allocate scratch for the current capacities and upload the tables (not allowed while capturing)
static int plan_reserve(Plan &pl, cudaStream_t s) {
    const int64_t n_bins = 3 * pl.n_tiles;
    const size_t tb = sizeof(Prob) * pl.n + 2 * sizeof(long long) * (pl.n + 1) + sizeof(FillProb) * pl.n +
                      4 * sizeof(long long) * (pl.n + 1) + 256;
    SDF_TRY(pl.tables.reserve(tb, s));
    if (pl.fill) SDF_TRY(pl.rowsign.reserve((size_t)pl.r_tot + 64, s));
    if (pl.cell_loop) SDF_TRY(pl.keys.reserve(sizeof(unsigned long long) * (size_t)pl.p_tot, s));
    SDF_TRY(pl.bins.reserve(sizeof(uint32_t) * (size_t)(2 * n_bins + 64), s));
    if (!pl.cell_loop) {  // split tiles: items, per-slot keys (kept at ~0 between launches) and counts
        void *const before = pl.split.p;
        SDF_TRY(pl.split.reserve(split_bytes(), s));
        if (pl.split.p != before) {
            SDF_TRY(cudaMemsetAsync(pl.split.p, 0xff, split_bytes(), s));
            SDF_TRY(cudaMemsetAsync(static_cast<char *>(pl.split.p) + split_done_offset(), 0,
                                    sizeof(unsigned) * SPLIT_SLOTS, s));
        }
    }
    {  // the scan state starts cleared whenever its memory is new (see scan_exclusive_u32)
        void *const before = pl.scan_tmp.p;
        SDF_TRY(pl.scan_tmp.reserve(scan_state_bytes(n_bins), s));
        if (pl.scan_tmp.p != before) SDF_TRY(cudaMemsetAsync(pl.scan_tmp.p, 0, pl.scan_tmp.bytes, s));
    }
    SDF_TRY(pl.lists.reserve(32 + sizeof(uint32_t) * (size_t)(3 * pl.n_tiles + 256), s));
    // room for the expected pairs (with a quarter to spare), and never less than 8 per feature;
    // a synchronising call grows it further when the binning finds more.  SDF_PAIR_CAPACITY, when
    // set, replaces the first capacity (to exercise that growth in tests).
    const char *env = getenv("SDF_PAIR_CAPACITY");
    const int64_t forced = env ? (int64_t)atoll(env) : 0;
    if (forced > 0) {
        if (pl.pair_cap == 0) pl.pair_cap = forced;
    } else {
        pl.pair_cap = std::max<int64_t>(pl.pair_cap, std::max<int64_t>(8 * pl.f_tot, pl.pair_est + pl.pair_est / 4) + 4096);
    }
    if (pl.patch_cap == 0) pl.patch_cap = pl.f_tot / 8 + 65536;
    SDF_TRY(pl.pairs.reserve(sizeof(int2) * (size_t)pl.pair_cap, s));
    SDF_TRY(pl.patch.reserve(sizeof(PatchEntry) * (size_t)pl.patch_cap, s));
    if (!pl.ctr) {
        SDF_TRY(pool_alloc(reinterpret_cast<void **>(&pl.ctr), sizeof(DevCounters), s));
        SDF_TRY(cudaMemsetAsync(pl.ctr, 0, sizeof(DevCounters), s));
        pl.own_ctr = true;
    }
    // the table: Prob[n], feature and tile prefix sums, FillProb[n], row / z-line / y-line prefix
    // sums; uploaded only when it changed
    const size_t pb = sizeof(Prob) * pl.n, lb = sizeof(long long) * (pl.n + 1), fb = sizeof(FillProb) * pl.n;
    std::vector<char> tab(pb + 2 * lb + fb + 4 * lb);
    memcpy(tab.data(), pl.probs.data(), pb);
    memcpy(tab.data() + pb, pl.fbase.data(), lb);
    memcpy(tab.data() + pb + lb, pl.tbase.data(), lb);
    memcpy(tab.data() + pb + 2 * lb, pl.fprobs.data(), fb);
    memcpy(tab.data() + pb + 2 * lb + fb, pl.rbase.data(), lb);
    memcpy(tab.data() + pb + 3 * lb + fb, pl.zbase.data(), lb);
    memcpy(tab.data() + pb + 4 * lb + fb, pl.ybase.data(), lb);
    memcpy(tab.data() + pb + 5 * lb + fb, pl.pbase.data(), lb);
    if (pl.uploaded_to == pl.tables.p && pl.uploaded == tab) return SDF_OK;
    if (pl.pageable) {
        pl.uploaded.swap(tab);
        pl.uploaded_to = pl.tables.p;
        SDF_TRY(cudaMemcpyAsync(pl.tables.p, pl.uploaded.data(), pl.uploaded.size(), cudaMemcpyHostToDevice, s));
        return SDF_OK;
    }
    if (!pl.pinned_ev) SDF_TRY(cudaEventCreateWithFlags(&pl.pinned_ev, cudaEventDisableTiming));
    SDF_TRY(cudaEventSynchronize(pl.pinned_ev));  // the previous copy out of the staging buffer
    if (pl.pinned_bytes < tab.size()) {
        pinned_put(pl.pinned, pl.pinned_bytes);
        pl.pinned = nullptr;
        pl.pinned_bytes = 0;
        SDF_TRY(pinned_get(tab.size() + 1024, &pl.pinned, &pl.pinned_bytes));
    }
    memcpy(pl.pinned, tab.data(), tab.size());
    SDF_TRY(cudaMemcpyAsync(pl.tables.p, pl.pinned, tab.size(), cudaMemcpyHostToDevice, s));
    SDF_TRY(cudaEventRecord(pl.pinned_ev, s));
    pl.uploaded.swap(tab);
    pl.uploaded_to = pl.tables.p;
    return SDF_OK;
}

struct Scratch {  // device pointers used by one launch of the pipeline
    const Prob *probs;
    bool any_list = false;  // some problem writes a compact band list
    bool any_dense = true;  // some problem writes a dense field (else the +inf fill is skipped)
    const long long *fbase, *tbase;
    uint32_t *cnt, *start;
    void *scan_tmp;
    unsigned long long *ticket;
    uint32_t *band_pos;
    int32_t *band_list, *empty_list;
    int2 *pairs;
    int64_t pair_cap;
    PatchEntry *patch;
    int64_t patch_cap;
    DevCounters *ctr;
    // sign beyond the band (null fprobs: not requested)
    const FillProb *fprobs = nullptr;
    const long long *rbase = nullptr, *zbase = nullptr, *ybase = nullptr;
    long long r_tot = 0, z_tot = 0, y_tot = 0;
    int8_t *rowsign = nullptr;
    // the paper's schedule (null keys: the tile path)
    const long long *pbase = nullptr;
    long long p_tot = 0;
    unsigned long long *keys = nullptr;
    // split tiles (null: not used, as in the allocation-free entry point)
    unsigned long long *split_keys = nullptr;
    int2 *split_items = nullptr;
    unsigned *split_done = nullptr;
};

static Scratch plan_scratch(const Plan &pl) {
    Scratch sc;
    sc.any_dense = false;
    for (const Prob &pr : pl.probs) {
        sc.any_list |= pr.list != nullptr;
        sc.any_dense |= pr.dist != nullptr || pr.winner != nullptr;
    }
    const char *t = pl.tables.as<char>();
    sc.probs = reinterpret_cast<const Prob *>(t);
    sc.fbase = reinterpret_cast<const long long *>(t + sizeof(Prob) * pl.n);
    sc.tbase = sc.fbase + pl.n + 1;
    if (pl.cell_loop) {
        sc.pbase = reinterpret_cast<const long long *>(reinterpret_cast<const char *>(sc.tbase + pl.n + 1) +
                                                       sizeof(FillProb) * pl.n) + 3 * (pl.n + 1);
        sc.p_tot = pl.p_tot;
        sc.keys = pl.keys.as<unsigned long long>();
    }
    if (pl.fill) {
        sc.fprobs = reinterpret_cast<const FillProb *>(sc.tbase + pl.n + 1);
        sc.rbase = reinterpret_cast<const long long *>(sc.fprobs + pl.n);
        sc.zbase = sc.rbase + pl.n + 1;
        sc.ybase = sc.zbase + pl.n + 1;
        sc.r_tot = pl.r_tot;
        sc.z_tot = pl.z_tot;
        sc.y_tot = pl.y_tot;
        sc.rowsign = pl.rowsign.as<int8_t>();
    }
    sc.cnt = pl.bins.as<uint32_t>();
    sc.start = sc.cnt + 3 * pl.n_tiles + 32;
    sc.scan_tmp = pl.scan_tmp.p;
    sc.ticket = pl.lists.as<unsigned long long>();  // 8-byte aligned (allocation start)
    sc.band_pos = reinterpret_cast<uint32_t *>(sc.ticket + 4);  // tickets: band, fill, split items
    sc.band_list = reinterpret_cast<int32_t *>(sc.band_pos + pl.n_tiles + 32);
    sc.empty_list = sc.band_list + pl.n_tiles + 32;
    sc.pairs = pl.pairs.as<int2>();
    sc.pair_cap = pl.pair_cap;
    sc.patch = pl.patch.as<PatchEntry>();
    sc.patch_cap = pl.patch_cap;
    sc.ctr = pl.ctr;
    if (pl.split.p) {
        char *b = static_cast<char *>(pl.split.p);
        sc.split_keys = reinterpret_cast<unsigned long long *>(b);
        sc.split_items = reinterpret_cast<int2 *>(b + split_items_offset());
        sc.split_done = reinterpret_cast<unsigned *>(b + split_done_offset());
    }
    return sc;
}

// the whole pipeline of one batch: kernels and memsets only (no allocation, no synchronisation)
template <int TY, int TZ>
static int launch_shape(int n, long long f_tot, int64_t n_tiles, const Scratch &sc, cudaStream_t s,
                        cudaEvent_t *ev) {
    const int64_t n_bins = 3 * n_tiles;
    if (ev) SDF_TRY(record_event(ev[0], s));
    {  // windows, counters, tickets (band, fill and, where split tiles are possible, split items)
        const unsigned blocks = std::max(nblk(n, 256), std::min(nblk(n_bins / 4, 256), (unsigned)(2 * num_sms())));
        SDF_TRY(launch_dep(k_front, dim3(blocks), dim3(256), 0, s, const_cast<Prob *>(sc.probs), n, sc.cnt, n_bins,
                           sc.ctr, sc.ticket, sc.split_items ? 3 : 2));
    }
    SDF_TRY(launch_dep(k_bin<false, TY, TZ>, dim3(nblk(f_tot, 256)), dim3(256), 0, s, sc.probs, sc.fbase, sc.tbase, n,
                       f_tot, sc.cnt, (const uint32_t *)nullptr, (int2 *)nullptr, (int64_t)0, sc.ctr));
    SDF_TRY(scan_exclusive_u32(sc.cnt, sc.start, n_bins, true, sc.scan_tmp, s, &sc.ctr->nb_status));
    SDF_TRY(launch_dep(k_bin<true, TY, TZ>, dim3(nblk(f_tot, 256)), dim3(256), 0, s, sc.probs, sc.fbase, sc.tbase, n,
                       f_tot, sc.cnt, (const uint32_t *)sc.start, sc.pairs, sc.pair_cap, sc.ctr));
    // band / empty tile lists for the persistent tile kernel (one scan of the band flags)
    uint32_t *flags = sc.cnt;  // the fill cursors are no longer needed
    const int lpt = n > 1;  // largest-first order of the band tiles for batches
    SDF_TRY(launch_dep(k_band_flags, dim3(nblk(n_tiles, 256)), dim3(256), 0, s, (const uint32_t *)sc.start, n_tiles,
                       flags, sc.ctr, lpt));
    SDF_TRY(scan_exclusive_u32(flags, sc.band_pos, n_tiles, true, sc.scan_tmp, s, &sc.ctr->nb_status));
    SDF_TRY(launch_dep(k_tile_lists, dim3(nblk(n_tiles, 256)), dim3(256), 0, s, (const uint32_t *)sc.start, n_tiles,
                       (const uint32_t *)sc.band_pos, sc.band_list, sc.empty_list, sc.ctr, lpt, sc.split_items,
                       sc.split_items ? SPLIT_SLOTS : 0));
    Outputs o;
    o.pairs = sc.pairs;
    o.bin_start = sc.start;
    o.pair_cap = sc.pair_cap;
    o.patch = sc.patch;
    o.patch_cap = sc.patch_cap;
    o.ctr = sc.ctr;
    o.split_items = sc.split_items;
    o.split_keys = sc.split_keys;
    o.split_done = sc.split_done;
    if (ev) SDF_TRY(record_event(ev[1], s));
    if (sc.any_list) {
        const int64_t ctas = std::min<int64_t>(n_tiles, (int64_t)tile_blocks_per_sm<TY, TZ, true>() * num_sms());
        if (sc.split_items) {  // the items of split tiles (none in most launches: the CTAs then return at once)
            // one CTA per SM: a few tiles' items at most, and a cheap launch when there are none
            tile_blocks_per_sm<TY, TZ, true, true>();  // (sets the kernel's shared-memory limit once)
            const int64_t sctas = std::min<int64_t>(n_tiles, (int64_t)num_sms());
            SDF_TRY(launch_dep(k_tile<TY, TZ, true, true>, dim3((unsigned)sctas), dim3(NT),
                               sizeof(TileSmem<TY, TZ>), s, sc.probs, sc.tbase, n, o, n_tiles,
                               (const int32_t *)sc.band_list, (const int32_t *)sc.empty_list,
                               sc.band_pos + n_tiles, sc.ticket, sc.any_dense ? 1 : 0));
        }
        SDF_TRY(launch_dep(k_tile<TY, TZ, true, false>, dim3((unsigned)ctas), dim3(NT), sizeof(TileSmem<TY, TZ>), s,
                           sc.probs, sc.tbase, n, o, n_tiles, (const int32_t *)sc.band_list,
                           (const int32_t *)sc.empty_list, sc.band_pos + n_tiles, sc.ticket, sc.any_dense ? 1 : 0));
    } else {
        const int64_t ctas = std::min<int64_t>(n_tiles, (int64_t)tile_blocks_per_sm<TY, TZ, false>() * num_sms());
        if (sc.split_items) {
            // one CTA per SM: a few tiles' items at most, and a cheap launch when there are none
            tile_blocks_per_sm<TY, TZ, false, true>();  // (sets the kernel's shared-memory limit once)
            const int64_t sctas = std::min<int64_t>(n_tiles, (int64_t)num_sms());
            SDF_TRY(launch_dep(k_tile<TY, TZ, false, true>, dim3((unsigned)sctas), dim3(NT),
                               sizeof(TileSmem<TY, TZ>), s, sc.probs, sc.tbase, n, o, n_tiles,
                               (const int32_t *)sc.band_list, (const int32_t *)sc.empty_list,
                               sc.band_pos + n_tiles, sc.ticket, sc.any_dense ? 1 : 0));
        }
        SDF_TRY(launch_dep(k_tile<TY, TZ, false, false>, dim3((unsigned)ctas), dim3(NT), sizeof(TileSmem<TY, TZ>), s,
                           sc.probs, sc.tbase, n, o, n_tiles, (const int32_t *)sc.band_list,
                           (const int32_t *)sc.empty_list, sc.band_pos + n_tiles, sc.ticket, sc.any_dense ? 1 : 0));
    }
    if (ev) SDF_TRY(record_event(ev[2], s));
    SDF_TRY(launch_dep(k_patch<TY, TZ>, dim3(patch_blocks<TY, TZ>()), dim3(256), 0, s, sc.probs, sc.tbase, o));
    if (sc.fprobs)
        SDF_TRY(fill_sign(sc.fprobs, sc.rbase, sc.zbase, sc.ybase, n, sc.r_tot, sc.z_tot, sc.y_tot, sc.rowsign,
                          num_sms(), s));
    if (ev) SDF_TRY(record_event(ev[3], s));
    return SDF_OK;
}

// the paper's schedule: clear the keys, one thread per region, decode, FP64 re-decision (and the fill)
static int launch_cell_loop(int n, long long f_tot, const Scratch &sc, cudaStream_t s, cudaEvent_t *ev) {
    if (ev) SDF_TRY(record_event(ev[0], s));
    k_windows<<<nblk(n, 64), 64, 0, s>>>(const_cast<Prob *>(sc.probs), n);
    SDF_LAUNCHED(1);
    SDF_TRY(cudaMemsetAsync(sc.keys, 0xff, sizeof(unsigned long long) * (size_t)sc.p_tot, s));
    SDF_TRY(cudaMemsetAsync(&sc.ctr->nb_status, 0, sizeof(unsigned), s));
    SDF_TRY(cudaMemsetAsync(&sc.ctr->n_candidates, 0, 6 * sizeof(unsigned long long), s));
    if (ev) SDF_TRY(record_event(ev[1], s));
    k_cell_loop<<<nblk(f_tot, 128), 128, 0, s>>>(sc.probs, sc.fbase, sc.pbase, n, f_tot, sc.keys, sc.ctr);
    SDF_LAUNCHED(1);
    SDF_TRY(cudaGetLastError());
    Outputs o;
    o.pairs = nullptr;
    o.bin_start = nullptr;
    o.pair_cap = 0;
    o.patch = sc.patch;
    o.patch_cap = sc.patch_cap;
    o.ctr = sc.ctr;
    k_decode_keys<<<16 * num_sms(), 256, 0, s>>>(sc.probs, sc.pbase, n, sc.p_tot, sc.keys, o);
    SDF_LAUNCHED(1);
    SDF_TRY(cudaGetLastError());
    if (ev) SDF_TRY(record_event(ev[2], s));
    k_patch<8, 8><<<patch_blocks<8, 8>(), 256, 0, s>>>(sc.probs, sc.tbase, o);  // no pairs: fan search
    SDF_LAUNCHED(1);
    SDF_TRY(cudaGetLastError());
    if (sc.fprobs)
        SDF_TRY(fill_sign(sc.fprobs, sc.rbase, sc.zbase, sc.ybase, n, sc.r_tot, sc.z_tot, sc.y_tot, sc.rowsign,
                          num_sms(), s));
    if (ev) SDF_TRY(record_event(ev[3], s));
    return SDF_OK;
}

static int launch_any(int shape, int n, long long f_tot, int64_t n_tiles, const Scratch &sc, cudaStream_t s,
                      cudaEvent_t *ev) {
    if (sc.keys) return launch_cell_loop(n, f_tot, sc, s, ev);
    switch (shape) {
    case 1: return launch_shape<4, 4>(n, f_tot, n_tiles, sc, s, ev);
    case 2: return launch_shape<16, 8>(n, f_tot, n_tiles, sc, s, ev);
    default: return launch_shape<8, 8>(n, f_tot, n_tiles, sc, s, ev);
    }
}

// Single-problem calls with SDF_FLAG_TIMING time the stages with the handle's events and wait for
// them; a batch created with SDF_FLAG_TIMING records its own events on every run (also inside a
// graph capture, as event nodes) and leaves the reading to sdf_batch_timing.
static int plan_launch(Plan &pl, cudaStream_t s, bool timing) {
    cudaEvent_t *ev = nullptr;
    if (pl.batch_timing) {
        ev = pl.bev;
    } else if (timing && pl.events) {
        if (ensure_events(pl.events)) return SDF_ERR_CUDA;
        SDF_TRY_ST(resolve_timing(pl.events));  // the previous timed call's events are reused
        ev = pl.events->ev;
    }
    for (const Prob &pr : pl.probs)  // band-list lengths count up from 0 in every launch
        if (pr.list_count) SDF_TRY(cudaMemsetAsync(pr.list_count, 0, sizeof(unsigned long long), s));
    int st = launch_any(pl.shape, pl.n, pl.f_tot, pl.n_tiles, plan_scratch(pl), s, ev);
    if (st) return st;
    if (ev && !pl.batch_timing) pl.events->fwd_pending = true;  // read later (resolve_timing)
    return SDF_OK;
}

// synchronise, read the counters, and grow the capacities that overflowed (retry set)
static int plan_check(Plan &pl, const sdf_features *feats, cudaStream_t s, bool *retry) {
    DevCounters c;
    uint32_t total_pairs = 0;
    {
        const HostRead rd[2] = {{&c, pl.ctr, sizeof(DevCounters)},
                                {&total_pairs, plan_scratch(pl).start + 3 * pl.n_tiles, sizeof(uint32_t)}};
        SDF_TRY(read_small(rd, 2, s));
    }
    *retry = false;
    // degenerate positions are flagged in each handle's own status word (batches: four per read)
    for (int p0 = 0; p0 < pl.n; p0 += 4) {
        unsigned st[4] = {0, 0, 0, 0};
        HostRead rd[4];
        int m = 0;
        for (int p = p0; p < pl.n && p < p0 + 4; p++)
            if (feats[p]->ctr != pl.ctr) {
                rd[m] = HostRead{&st[m], &feats[p]->ctr->status, sizeof(unsigned)};
                m++;
            }
        if (m) SDF_TRY(read_small(rd, m, s));
        for (int i = 0; i < m; i++)
            if (st[i] & ST_DEGENERATE) return SDF_ERR_DEGENERATE;
    }
    if (c.status & ST_DEGENERATE) return SDF_ERR_DEGENERATE;
    if (c.nb_status & ST_TIMEOUT) return SDF_ERR_TIMEOUT;
    if (c.nb_status & ST_PAIR_OVERFLOW) {
        pl.pair_cap = (int64_t)total_pairs + total_pairs / 4 + 4096;
        *retry = true;
    }
    if (c.nb_status & ST_PATCH_OVERFLOW) {
        pl.patch_cap = (int64_t)c.n_patch + c.n_patch / 2 + 4096;
        *retry = true;
    }
    // the caller's band list is too short: its count holds the length needed (no retry here, the
    // caller owns the list)
    if (!*retry && (c.nb_status & ST_LIST_OVERFLOW)) return SDF_ERR_LIST_OVERFLOW;
    return SDF_OK;
}

// describe (already done), reserve, launch and, when synchronising, retry with grown scratch
static int plan_execute(Plan &pl, const sdf_features *feats, cudaStream_t s, bool sync, bool timing) {
    for (int attempt = 0; attempt < 4; attempt++) {
        SDF_TRY_ST(plan_reserve(pl, s));
        SDF_TRY_ST(plan_launch(pl, s, timing));
        if (!sync) return SDF_OK;
        bool retry = false;
        SDF_TRY_ST(plan_check(pl, feats, s, &retry));
        if (!retry) return SDF_OK;
    }
    return SDF_ERR_OOM;
}

// stats of the last call (host), used by sdf_features_status
int narrow_band_stats(sdf_features_s *f, int64_t *stats, cudaStream_t s) {
    DevCounters c;
    {
        const HostRead rd[1] = {{&c, f->ctr, sizeof(DevCounters)}};
        SDF_TRY(read_small(rd, 1, s));
    }
    if (stats) {
        stats[0] = (int64_t)c.n_candidates;
        stats[1] = (int64_t)c.n_band;
        stats[2] = (int64_t)c.n_patch;
        stats[3] = (int64_t)c.n_pairs;
        stats[4] = (int64_t)c.n_rows;
        stats[5] = (int64_t)c.n_rows_hit;
    }
    if (c.status & ST_DEGENERATE) return SDF_ERR_DEGENERATE;
    if (c.nb_status & ST_TIMEOUT) return SDF_ERR_TIMEOUT;
    if (c.nb_status & (ST_PAIR_OVERFLOW | ST_PATCH_OVERFLOW)) return SDF_ERR_OOM;
    if (c.nb_status & ST_LIST_OVERFLOW) return SDF_ERR_LIST_OVERFLOW;
    return SDF_OK;
}

static std::mutex g_tune_mu;
static std::map<std::tuple<int, long long, long long>, int> g_tuned;  // (n, features, grid points) -> shape

static std::tuple<int, long long, long long> tune_key(const sdf_features *feats, const sdf_grid *grids, int n) {
    long long nf = 0, np = 0;
    for (int p = 0; p < n; p++) {
        nf += feats[p]->T + feats[p]->E + feats[p]->V;
        np += (long long)grids[p].nx * grids[p].ny * grids[p].nz;
    }
    return std::make_tuple(n, nf, np);
}

int narrow_band_all(const sdf_features *feats, const sdf_grid *grids, const float *band_w, int32_t n,
                    float *const *out_dist, int32_t *const *out_winner, uint32_t flags, cudaStream_t s,
                    const ListOut *lists) {
    if (!feats || !grids || !band_w || n < 1 || !out_dist) return SDF_ERR_INVALID_ARG;
    for (int p = 0; p < n; p++)
        if (!feats[p] || (!out_dist[p] && !(lists && lists[p].list && lists[p].dist))) return SDF_ERR_INVALID_ARG;
    const bool sync = !(flags & SDF_FLAG_NO_SYNC), timing = (flags & SDF_FLAG_TIMING) != 0;
    const bool fill = (flags & SDF_FLAG_FILL_SIGN) != 0, cell_loop = (flags & SDF_FLAG_CELL_LOOP) != 0;
    const int vmode = (flags & SDF_FLAG_VERTEX_CONE) ? VM_CONE : ((flags & SDF_FLAG_VERTEX_HEMISPHERE) ? VM_HEMISPHERE : VM_EXACT);
    if (vmode != VM_EXACT && (!cell_loop || (flags & SDF_FLAG_VERTEX_CONE && flags & SDF_FLAG_VERTEX_HEMISPHERE)))
        return SDF_ERR_INVALID_ARG;  // the paper's vertex extrusions exist in the cell-loop schedule only
    if (n == 1) {  // a batch of one, with the plan (and its scratch) cached in the handle
        sdf_features_s *f = feats[0];
        if (!f->plan) {
            f->plan = plan_take();
            f->plan->ctr = f->ctr;
            f->plan->events = f;
        }
        Plan &pl = *f->plan;
        pl.cell_loop = cell_loop;
        pl.vmode = vmode;
        SDF_TRY_ST(plan_describe(pl, feats, grids, band_w, 1, out_dist, out_winner, 0, fill, lists));
        return plan_execute(pl, feats, s, sync, timing);
    }
    int shape = 0;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(tune_key(feats, grids, n));
        if (it != g_tuned.end()) shape = it->second;
    }
    Plan pl;
    pl.pageable = true;
    pl.cell_loop = cell_loop;
    pl.vmode = vmode;
    int st = plan_describe(pl, feats, grids, band_w, n, out_dist, out_winner, shape, fill, lists);
    if (!st) st = plan_execute(pl, feats, s, true, false);
    // the temporary plan's memory returns to the pool in stream order
    plan_free(new Plan(std::move(pl)), s);
    return st;
}

}  // namespace sdf

extern "C" int sdf_narrow_band(const sdf_features *feats, const sdf_grid *grids, const float *band_w, int32_t n,
                               float *const *out_dist, int32_t *const *out_winner, uint32_t flags, void *stream) {
    return sdf::narrow_band_all(feats, grids, band_w, n, out_dist, out_winner, flags,
                                reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int sdf_narrow_band_list(sdf_features f, const sdf_grid *grid, float band_w, float *out_dist,
                                    int32_t *out_winner, sdf_band_entry *list, int64_t list_cap,
                                    unsigned long long *list_count, uint32_t flags, void *stream) {
    if (!f || !grid || !out_dist || !list || !list_count || list_cap < 0) return SDF_ERR_INVALID_ARG;
    if (flags & SDF_FLAG_CELL_LOOP) return SDF_ERR_INVALID_ARG;
    const sdf_features fl[1] = {f};
    float *const dl[1] = {out_dist};
    int32_t *const wl[1] = {out_winner};
    const sdf::ListOut lo[1] = {{list, (long long)list_cap, list_count}};
    return sdf::narrow_band_all(fl, grid, &band_w, 1, dl, wl, flags, reinterpret_cast<cudaStream_t>(stream), lo);
}

extern "C" int sdf_narrow_band_sparse(sdf_features f, const sdf_grid *grid, float band_w, sdf_band_entry *list,
                                      float *list_dist, int64_t list_cap, unsigned long long *list_count,
                                      uint32_t flags, void *stream) {
    if (!f || !grid || !list || !list_dist || !list_count || list_cap < 0) return SDF_ERR_INVALID_ARG;
    if (flags & (SDF_FLAG_CELL_LOOP | SDF_FLAG_FILL_SIGN)) return SDF_ERR_INVALID_ARG;
    const sdf_features fl[1] = {f};
    float *const dl[1] = {nullptr};
    int32_t *const wl[1] = {nullptr};
    sdf::ListOut lo[1] = {{list, (long long)list_cap, list_count}};
    lo[0].dist = list_dist;
    return sdf::narrow_band_all(fl, grid, &band_w, 1, dl, wl, flags, reinterpret_cast<cudaStream_t>(stream), lo);
}

extern "C" int sdf_narrow_band_lists(const sdf_features *feats, const sdf_grid *grids, const float *band_w, int32_t n,
                                     float *const *out_dist, int32_t *const *out_winner, sdf_band_entry *const *lists,
                                     const int64_t *list_caps, unsigned long long *const *list_counts, uint32_t flags,
                                     void *stream) {
    if (!feats || !grids || !band_w || n < 1 || !out_dist || !lists || !list_caps || !list_counts)
        return SDF_ERR_INVALID_ARG;
    if (flags & SDF_FLAG_CELL_LOOP) return SDF_ERR_INVALID_ARG;
    std::vector<sdf::ListOut> lo((size_t)n);
    for (int p = 0; p < n; p++) {
        if (!lists[p] || !list_counts[p] || list_caps[p] < 0) return SDF_ERR_INVALID_ARG;
        lo[p] = sdf::ListOut{lists[p], (long long)list_caps[p], list_counts[p]};
    }
    return sdf::narrow_band_all(feats, grids, band_w, n, out_dist, out_winner, flags,
                                reinterpret_cast<cudaStream_t>(stream), lo.data());
}

// ----------------------------------------------------------------------------- batches for CUDA graphs
struct sdf_batch_s {
    sdf::Plan plan;
    std::vector<sdf_features> feats;
};

extern "C" int sdf_batch_create(const sdf_features *feats, const sdf_grid *grids, const float *band_w, int32_t n,
                                float *const *out_dist, int32_t *const *out_winner, uint32_t flags, void *stream,
                                sdf_batch *out) {
    using namespace sdf;
    if (!out) return SDF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!feats || !grids || !band_w || n < 1 || !out_dist) return SDF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    sdf_batch_s *b = new sdf_batch_s();
    b->feats.assign(feats, feats + n);
    int best = 0;
    double best_ms = 0.0;
    const int n_try = (flags & SDF_FLAG_AUTOTUNE) ? N_SHAPES : 1;
    const bool fill = (flags & SDF_FLAG_FILL_SIGN) != 0;
    b->plan.cell_loop = (flags & SDF_FLAG_CELL_LOOP) != 0;
    b->plan.vmode = (flags & SDF_FLAG_VERTEX_CONE) ? VM_CONE : ((flags & SDF_FLAG_VERTEX_HEMISPHERE) ? VM_HEMISPHERE : VM_EXACT);
    if (b->plan.vmode != VM_EXACT && (!b->plan.cell_loop || (flags & SDF_FLAG_VERTEX_CONE && flags & SDF_FLAG_VERTEX_HEMISPHERE))) {
        delete b;
        return SDF_ERR_INVALID_ARG;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = SDF_OK;
    if (n_try > 1 && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) st = SDF_ERR_CUDA;
    for (int shape = 0; shape < n_try && !st; shape++) {
        st = plan_describe(b->plan, feats, grids, band_w, n, out_dist, out_winner, shape, fill);
        if (!st) st = plan_execute(b->plan, b->feats.data(), s, true, false);  // sizes the scratch
        if (st || n_try == 1) break;
        const int reps = 3;
        if (cudaEventRecord(e0, s) != cudaSuccess) { st = SDF_ERR_CUDA; break; }
        for (int r = 0; r < reps && !st; r++) st = plan_launch(b->plan, s, false);
        float ms = 0.f;
        if (!st && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            st = SDF_ERR_CUDA;
        if (!st && (shape == 0 || ms / reps < best_ms)) {
            best = shape;
            best_ms = ms / reps;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (!st && (flags & SDF_FLAG_TIMING)) {
        for (int i = 0; i < 4 && !st; i++)
            if (cudaEventCreate(&b->plan.bev[i]) != cudaSuccess) st = SDF_ERR_CUDA;
        b->plan.batch_timing = !st;
    }
    if (!st && n_try > 1) {  // rebuild the plan for the fastest shape and leave its outputs filled
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tuned[tune_key(feats, grids, n)] = best;
        }
        b->plan.pair_cap = 0;
        b->plan.patch_cap = 0;
        st = plan_describe(b->plan, feats, grids, band_w, n, out_dist, out_winner, best, fill);
        if (!st) st = plan_execute(b->plan, b->feats.data(), s, true, false);
        b->plan.tuned_ms = best_ms;
    }
    if (st) {
        plan_free(new Plan(std::move(b->plan)), s);
        delete b;
        return st;
    }
    *out = b;
    return SDF_OK;
}

extern "C" int sdf_batch_run(sdf_batch b, void *stream) {
    if (!b) return SDF_ERR_INVALID_ARG;
    return sdf::plan_launch(b->plan, reinterpret_cast<cudaStream_t>(stream), false);
}

extern "C" int sdf_batch_status(sdf_batch b, int64_t *stats, void *stream) {
    using namespace sdf;
    if (!b) return SDF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DevCounters c;
    {
        const HostRead rd[1] = {{&c, b->plan.ctr, sizeof(DevCounters)}};
        SDF_TRY(read_small(rd, 1, s));
    }
    if (stats) {
        stats[0] = (int64_t)c.n_candidates;
        stats[1] = (int64_t)c.n_band;
        stats[2] = (int64_t)c.n_patch;
        stats[3] = (int64_t)c.n_pairs;
        stats[4] = (int64_t)c.n_rows;
        stats[5] = (int64_t)c.n_rows_hit;
    }
    if (c.nb_status & ST_TIMEOUT) return SDF_ERR_TIMEOUT;
    if (c.nb_status & (ST_PAIR_OVERFLOW | ST_PATCH_OVERFLOW)) return SDF_ERR_OOM;
    if (c.nb_status & ST_LIST_OVERFLOW) return SDF_ERR_LIST_OVERFLOW;
    return SDF_OK;
}

extern "C" int sdf_batch_timing(sdf_batch b, float *ms) {
    if (!b || !ms) return SDF_ERR_INVALID_ARG;
    if (!b->plan.batch_timing) return SDF_ERR_INVALID_ARG;
    for (int i = 0; i < 3; i++) {
        SDF_TRY(cudaEventSynchronize(b->plan.bev[i + 1]));
        SDF_TRY(cudaEventElapsedTime(&ms[i], b->plan.bev[i], b->plan.bev[i + 1]));
    }
    return SDF_OK;
}

extern "C" int sdf_batch_info(sdf_batch b, int32_t *tile_shape, double *tuned_ms) {
    if (!b) return SDF_ERR_INVALID_ARG;
    if (tile_shape) {
        tile_shape[0] = sdf::TILE_X;
        tile_shape[1] = sdf::SHAPE_TY[b->plan.shape];
        tile_shape[2] = sdf::SHAPE_TZ[b->plan.shape];
    }
    if (tuned_ms) *tuned_ms = b->plan.tuned_ms;
    return SDF_OK;
}

extern "C" void sdf_batch_destroy(sdf_batch b) {
    if (!b) return;
    cudaDeviceSynchronize();
    sdf::plan_free(new sdf::Plan(std::move(b->plan)), 0);
    delete b;
}

extern "C" int sdf_features_error_bound(sdf_features f, const sdf_grid *grid, float band_w, double *bounds,
                                        void *stream) {
    using namespace sdf;
    if (!f || !grid || !bounds) return SDF_ERR_INVALID_ARG;
    GridP g;
    SDF_TRY_ST(make_grid(*grid, band_w, 0, g));
    unsigned prec[4] = {0, 0, 0, 0};
    {
        const HostRead rd[1] = {{prec, f->ctr->prec, sizeof(prec)}};
        SDF_TRY(read_small(rd, 1, reinterpret_cast<cudaStream_t>(stream)));
    }
    float v[4];
    memcpy(v, prec, sizeof(v));
    set_windows(g, v[PREC_MESH_M], v[PREC_TAU_A], v[PREC_TAU_B], v[PREC_TAU_V]);
    bounds[0] = g.derr;
    bounds[1] = g.eps;
    bounds[2] = g.ds;
    bounds[3] = fmax(g.ds2, g.dsv);
    return SDF_OK;
}

extern "C" int sdf_features_status(sdf_features f, int64_t *stats, void *stream) {
    if (!f) return SDF_ERR_INVALID_ARG;
    return sdf::narrow_band_stats(f, stats, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int sdf_features_timing(sdf_features f, double *ms, int64_t *calls, int reset) {
    if (!f) return SDF_ERR_INVALID_ARG;
    SDF_TRY_ST(sdf::resolve_timing(f));
    for (int i = 0; i < 4; i++) {
        if (ms) ms[i] = f->t_ms[i];
        if (calls) calls[i] = f->t_calls[i];
        if (reset) {
            f->t_ms[i] = 0.0;
            f->t_calls[i] = 0;
        }
    }
    return SDF_OK;
}

// ============================================================================= allocation-free variant
// sdf_narrow_band_static: the narrow band of one (mesh, grid) problem without any device
// allocation.  It exists for callers that must not allocate device memory during the call: a
// process whose device memory is handed out by another runtime or a fixed budget (where an
// unexpected cudaMalloc can fail or steal memory), or a real-time loop where the latency of an
// allocation is not acceptable.  The regular sdf_narrow_band grows scratch buffers inside the
// handle on demand, which allocates.  The first call on a device looks up the address of the
// scratch array (which also makes the driver load this module's device data); make that first
// call before any stream capture.
//
// All per-call scratch (bin counters, the (tile, region) pair list, the tile work lists, the
// FP64 re-decision list, counters and the work ticket) lives in this one file-scope device
// array.  Every device that loads the library holds it until the process exits.
namespace sdf {
namespace {
static_assert(sizeof(Prob) + 16 * 4 <= 2048, "problem table slot");
constexpr int64_t ST_MAX_TILES = 65536;                 // 32x8x8-point tiles (512^3 points)
constexpr int64_t ST_MAX_PAIRS = int64_t(2) << 20;      // (tile, region) pairs
constexpr int64_t ST_MAX_PATCH = 131072;                // points re-decided in FP64
constexpr size_t ST_OFF_CTR = 0;                        // DevCounters
constexpr size_t ST_OFF_TICKET = 1024;                  // work tickets (two, 16 bytes)
constexpr size_t ST_OFF_TABLE = 2048;                   // one Prob, then long long [4] prefix sums
constexpr size_t ST_PROB_BYTES = (sizeof(Prob) + 15) / 16 * 16;
constexpr size_t ST_OFF_CNT = ST_OFF_TABLE + 2048;      // uint32 [3 * max tiles]
constexpr size_t ST_OFF_START = ST_OFF_CNT + 4 * (3 * ST_MAX_TILES + 256);      // uint32 [3 * max tiles + 1]
constexpr size_t ST_OFF_BANDPOS = ST_OFF_START + 4 * (3 * ST_MAX_TILES + 256);  // uint32 [max tiles + 1]
constexpr size_t ST_OFF_BANDLIST = ST_OFF_BANDPOS + 4 * (ST_MAX_TILES + 256);   // int32 [max tiles]
constexpr size_t ST_OFF_EMPTYLIST = ST_OFF_BANDLIST + 4 * (ST_MAX_TILES + 256); // int32 [max tiles]
constexpr size_t ST_OFF_SCAN = ST_OFF_EMPTYLIST + 4 * (ST_MAX_TILES + 256);     // scan temporaries
constexpr size_t ST_SCAN_BYTES = 65536;
constexpr size_t ST_OFF_PAIRS = ST_OFF_SCAN + ST_SCAN_BYTES;                     // int2 [max pairs]
constexpr size_t ST_OFF_PATCH = ST_OFF_PAIRS + 8 * ST_MAX_PAIRS;                 // PatchEntry [max patch]
constexpr size_t ST_BYTES = ST_OFF_PATCH + sizeof(PatchEntry) * ST_MAX_PATCH;    // about 20.3 MiB
}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[ST_BYTES];

// device address of g_static_scratch for each device, looked up once with that device current
// (under a lock: two host threads may make their first calls at the same time)
static std::mutex g_static_mu;
static unsigned char *static_scratch_ptr(int *err) {
    static unsigned char *ptrs[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        *err = SDF_ERR_CUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!ptrs[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
            *err = SDF_ERR_CUDA;
            return nullptr;
        }
        ptrs[dev] = static_cast<unsigned char *>(p);
    }
    *err = SDF_OK;
    return ptrs[dev];
}
}  // namespace sdf

extern "C" int sdf_narrow_band_static(sdf_features f, const sdf_grid *grid, float band_w, float *out_dist,
                                      int32_t *out_winner, void *stream) {
    using namespace sdf;
    if (!f || !grid || !out_dist) return SDF_ERR_INVALID_ARG;
    GridP g;
    int st = make_grid(*grid, band_w, 0, g);
    if (st) return st;
    const int64_t n_tiles = (int64_t)g.ntx * g.nty * g.ntz, n_bins = 3 * n_tiles;
    if (n_tiles > ST_MAX_TILES) return SDF_ERR_TOO_LARGE;  // grid beyond the static scratch
    if (scan_state_bytes(n_bins) > ST_SCAN_BYTES) return SDF_ERR_TOO_LARGE;
    unsigned char *base = static_scratch_ptr(&st);
    if (st) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n_feat = f->T + f->E + f->V;
    // the one-problem table: Prob, feature prefix sums {0, n_feat}, tile prefix sums {0, n_tiles}
    Prob pr;
    pr.F = make_feat(f);
    pr.g = g;
    pr.dist = out_dist;
    pr.winner = out_winner;
    pr.vec = ((g.nx & 3) == 0) && ((reinterpret_cast<uintptr_t>(out_dist) & 15) == 0) &&
             ((reinterpret_cast<uintptr_t>(out_winner) & 15) == 0);
    const long long bases[4] = {0, n_feat, 0, n_tiles};
    Scratch sc;
    sc.probs = reinterpret_cast<const Prob *>(base + ST_OFF_TABLE);
    sc.fbase = reinterpret_cast<const long long *>(base + ST_OFF_TABLE + ST_PROB_BYTES);
    sc.tbase = sc.fbase + 2;
    sc.ctr = reinterpret_cast<DevCounters *>(base + ST_OFF_CTR);
    sc.ticket = reinterpret_cast<unsigned long long *>(base + ST_OFF_TICKET);
    sc.cnt = reinterpret_cast<uint32_t *>(base + ST_OFF_CNT);
    sc.start = reinterpret_cast<uint32_t *>(base + ST_OFF_START);
    sc.band_pos = reinterpret_cast<uint32_t *>(base + ST_OFF_BANDPOS);
    sc.band_list = reinterpret_cast<int32_t *>(base + ST_OFF_BANDLIST);
    sc.empty_list = reinterpret_cast<int32_t *>(base + ST_OFF_EMPTYLIST);
    sc.scan_tmp = base + ST_OFF_SCAN;
    sc.pairs = reinterpret_cast<int2 *>(base + ST_OFF_PAIRS);
    sc.pair_cap = ST_MAX_PAIRS;
    sc.patch = reinterpret_cast<PatchEntry *>(base + ST_OFF_PATCH);
    sc.patch_cap = ST_MAX_PATCH;
    // host-to-device copies of a few hundred bytes (staged by the driver, no device allocation)
    SDF_TRY(cudaMemcpyAsync(base + ST_OFF_TABLE, &pr, sizeof(Prob), cudaMemcpyHostToDevice, s));
    SDF_TRY(cudaMemcpyAsync(base + ST_OFF_TABLE + ST_PROB_BYTES, bases, sizeof(bases), cudaMemcpyHostToDevice, s));
    // the array keeps the previous call's contents: clear the counters (the pipeline clears the rest)
    SDF_TRY(cudaMemsetAsync(sc.ctr, 0, sizeof(DevCounters), s));
    SDF_TRY(cudaMemsetAsync(sc.scan_tmp, 0, scan_state_bytes(n_bins), s));  // the scans' state starts cleared
    SDF_TRY_ST((launch_shape<8, 8>(1, n_feat, n_tiles, sc, s, nullptr)));
    // The status words, read into host stack memory: this call's list overflows and the handle's
    // own status (a face that sdf_features_update_positions made degenerate).  A device-to-host
    // copy into pageable memory returns once the data has arrived and allocates nothing.
    unsigned status[2] = {0, 0};
    SDF_TRY(cudaMemcpyAsync(&status[0], &sc.ctr->nb_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    SDF_TRY(cudaMemcpyAsync(&status[1], &f->ctr->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    SDF_TRY(cudaStreamSynchronize(s));
    if (status[1] & ST_DEGENERATE) return SDF_ERR_DEGENERATE;
    if (status[0] & ST_TIMEOUT) return SDF_ERR_TIMEOUT;
    if (status[0] & (ST_PAIR_OVERFLOW | ST_PATCH_OVERFLOW)) return SDF_ERR_TOO_LARGE;
    return SDF_OK;
}
