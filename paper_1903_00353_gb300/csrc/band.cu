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
// GB300 schedule (replacing the paper's thread-per-extrusion cell loop, Section 9):
//   1. bin: every region's integer bounding box is split over 32x8x8-point tiles and the
//      (tile, region) pairs are bucketed per tile and type (count, scan, fill);
//   2. tile kernel: one CTA per tile keeps the packed keys (|d| bits << 32 | id << 1 | sign) of
//      its 2048 points in shared memory; warps take 32 regions at a time, flatten their grid
//      rows across lanes, intersect each row with the region's half-spaces (Algorithm 2, with
//      the inclusion tolerance of Section 10) to get an x-span, flatten the span points across
//      lanes again, evaluate the distance to the feature and merge with a shared-memory 64-bit
//      atomicMin (Algorithm 1's min-magnitude rule).  The CTA then writes its tile of the dense
//      output (coalesced rows), +inf outside the band, and queues the few points whose band
//      membership or sign lies inside the FP32 error window;
//   3. patch kernel: re-decides the queued points in FP64 from the winner's neighbourhood.
#include <math.h>

#include "sdf_internal.cuh"

namespace sdf {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int NT = 256;  // threads per tile CTA
enum { FACE = 0, EDGE = 1, VERT = 2 };

struct GridP {
    int nx, ny, nz;
    int ntx, nty, ntz;
    float ox, oy, oz, h, inv_h;
    float w;     // band half-width: in band iff |d| < w
    float W;     // candidate cutoff w + dw
    float dlo;   // w - dw: points with |d| in [dlo, W) are re-decided in FP64
    float ds;    // points with |d| < ds are re-decided in FP64 (sign)
    float eps;   // inclusion tolerance of the half-space tests (world units)
};

struct Feat {
    int T, E, V;
    const float4 *face_rec, *face_box, *edge_rec, *vert_rec, *vert_plane;
    const int8_t *edge_class, *vert_class;
    const int32_t *face_vid, *face_edge, *vert_start, *vert_corner;
    const int4 *edge_vf;
    const float *vpos;
    int skip_saddle;
};

struct PatchEntry {
    long long idx;
    int fid;
    int pad;
};

struct Outputs {
    float *dist;
    int32_t *winner;
    const int32_t *pairs;
    const uint32_t *bin_start;
    int64_t pair_cap;
    PatchEntry *patch;
    int64_t patch_cap;
    DevCounters *ctr;
};

// ----------------------------------------------------------------------------- boxes
__device__ __forceinline__ bool to_index_box(float lx, float ly, float lz, float hx, float hy, float hz,
                                             const GridP &g, int &i0, int &i1, int &j0, int &j1, int &k0, int &k1) {
    const float sl = 1.f / 4096.f;  // index slack against rounding of the conversion
    float a0 = fmaxf((lx - g.ox) * g.inv_h - 0.5f - sl, -1.f), a1 = fminf((hx - g.ox) * g.inv_h - 0.5f + sl, (float)g.nx);
    float b0 = fmaxf((ly - g.oy) * g.inv_h - 0.5f - sl, -1.f), b1 = fminf((hy - g.oy) * g.inv_h - 0.5f + sl, (float)g.ny);
    float c0 = fmaxf((lz - g.oz) * g.inv_h - 0.5f - sl, -1.f), c1 = fminf((hz - g.oz) * g.inv_h - 0.5f + sl, (float)g.nz);
    i0 = max((int)ceilf(a0), 0); i1 = min((int)floorf(a1), g.nx - 1);
    j0 = max((int)ceilf(b0), 0); j1 = min((int)floorf(b1), g.ny - 1);
    k0 = max((int)ceilf(c0), 0); k1 = min((int)floorf(c1), g.nz - 1);
    return i0 <= i1 && j0 <= j1 && k0 <= k1;
}

// integer box of the clipped region of feature `id` of type TYPE; false if the feature has none
template <int TYPE>
__device__ __forceinline__ bool feature_box(const Feat &F, const GridP &g, int id, int &i0, int &i1, int &j0,
                                            int &j1, int &k0, int &k1) {
    const float R = g.W + g.eps;
    if (TYPE == FACE) {
        float4 n = __ldg(F.face_rec + 4 * id), lo = __ldg(F.face_box + 2 * id), hi = __ldg(F.face_box + 2 * id + 1);
        float ex = R * fabsf(n.x) + g.eps, ey = R * fabsf(n.y) + g.eps, ez = R * fabsf(n.z) + g.eps;
        return to_index_box(lo.x - ex, lo.y - ey, lo.z - ez, hi.x + ex, hi.y + ey, hi.z + ez, g, i0, i1, j0, j1, k0, k1);
    } else if (TYPE == EDGE) {
        int8_t c = F.edge_class[id];
        if (c == CLS_FLAT) return false;
        float4 a = __ldg(F.edge_rec + 5 * id), t = __ldg(F.edge_rec + 5 * id + 1);
        float bx = fmaf(a.w, t.x, a.x), by = fmaf(a.w, t.y, a.y), bz = fmaf(a.w, t.z, a.z);
        return to_index_box(fminf(a.x, bx) - R, fminf(a.y, by) - R, fminf(a.z, bz) - R, fmaxf(a.x, bx) + R,
                            fmaxf(a.y, by) + R, fmaxf(a.z, bz) + R, g, i0, i1, j0, j1, k0, k1);
    } else {
        int8_t c = F.vert_class[id];
        if (c == CLS_FLAT || (F.skip_saddle && c == CLS_SADDLE)) return false;
        float4 v = __ldg(F.vert_rec + 2 * id);
        return to_index_box(v.x - R, v.y - R, v.z - R, v.x + R, v.y + R, v.z + R, g, i0, i1, j0, j1, k0, k1);
    }
}

// ----------------------------------------------------------------------------- binning
template <bool FILL>
__global__ void k_bin(Feat F, GridP g, uint32_t *cnt, const uint32_t *start, int32_t *pairs, int64_t pair_cap,
                      DevCounters *ctr) {
    int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t total = (int64_t)F.T + F.E + F.V;
    if (gid >= total) return;
    int type, id;
    bool ok;
    int i0, i1, j0, j1, k0, k1;
    if (gid < F.T) { type = FACE; id = (int)gid; ok = feature_box<FACE>(F, g, id, i0, i1, j0, j1, k0, k1); }
    else if (gid < (int64_t)F.T + F.E) { type = EDGE; id = (int)(gid - F.T); ok = feature_box<EDGE>(F, g, id, i0, i1, j0, j1, k0, k1); }
    else { type = VERT; id = (int)(gid - F.T - F.E); ok = feature_box<VERT>(F, g, id, i0, i1, j0, j1, k0, k1); }
    if (!ok) return;
    int fid = (int)gid;  // face f -> f, edge e -> T + e, vertex v -> T + E + v
    for (int tz = k0 / TILE_Z; tz <= k1 / TILE_Z; tz++)
        for (int ty = j0 / TILE_Y; ty <= j1 / TILE_Y; ty++)
            for (int tx = i0 / TILE_X; tx <= i1 / TILE_X; tx++) {
                int64_t tile = ((int64_t)tz * g.nty + ty) * g.ntx + tx;
                int64_t bin = 3 * tile + type;
                if (!FILL) {
                    atomicAdd(cnt + bin, 1u);
                } else {
                    int64_t pos = (int64_t)start[bin] + atomicAdd(cnt + bin, 1u);
                    if (pos < pair_cap) pairs[pos] = fid;
                    else atomicOr(&ctr->status, ST_PAIR_OVERFLOW);
                }
            }
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

// half-space P.xyz . (X, Y, Z) + P.w >= -eps along the row (Y, Z): shrink [xa, xb]
__device__ __forceinline__ void clip_plane(float4 P, float Y, float Z, float eps, float &xa, float &xb) {
    float r = fmaf(P.y, Y, fmaf(P.z, Z, P.w)) + eps;
    if (P.x > 0.f) xa = fmaxf(xa, -r / P.x);
    else if (P.x < 0.f) xb = fminf(xb, -r / P.x);
    else if (r < 0.f) xa = INFINITY;
}

// x-span of the region of feature `id` on the row (j, k), intersected with [bi0, bi1]
template <int TYPE>
__device__ __forceinline__ void row_span(const Feat &F, const GridP &g, int id, int j, int k, int bi0, int bi1,
                                         int &ia, int &ib) {
    const float Y = fmaf((float)j + 0.5f, g.h, g.oy), Z = fmaf((float)k + 0.5f, g.h, g.oz);
    float xa = -INFINITY, xb = INFINITY;
    const float e = g.eps;
    if (TYPE == FACE) {
        const float4 *r = F.face_rec + 4 * id;
        float4 n = __ldg(r);
        clip_plane(make_float4(n.x, n.y, n.z, n.w + g.W), Y, Z, e, xa, xb);      // n.p + c >= -W
        clip_plane(make_float4(-n.x, -n.y, -n.z, g.W - n.w), Y, Z, e, xa, xb);   // n.p + c <= W
        clip_plane(__ldg(r + 1), Y, Z, e, xa, xb);
        clip_plane(__ldg(r + 2), Y, Z, e, xa, xb);
        clip_plane(__ldg(r + 3), Y, Z, e, xa, xb);
    } else if (TYPE == EDGE) {
        const float4 *r = F.edge_rec + 5 * id;
        float4 a = __ldg(r), t = __ldg(r + 1);
        clip_plane(make_float4(t.x, t.y, t.z, -t.w), Y, Z, e, xa, xb);           // t.(p - a) >= 0
        clip_plane(make_float4(-t.x, -t.y, -t.z, t.w + a.w), Y, Z, e, xa, xb);   // t.(p - a) <= L
        clip_plane(__ldg(r + 2), Y, Z, e, xa, xb);                               // (p - a).m1 <= 0
        clip_plane(__ldg(r + 3), Y, Z, e, xa, xb);                               // (p - a).m2 <= 0
    } else {
        float4 v = __ldg(F.vert_rec + 2 * id), nv = __ldg(F.vert_rec + 2 * id + 1);
        float dy = Y - v.y, dz = Z - v.z;
        float R = g.W + e;
        float r2 = R * R - dy * dy - dz * dz;
        if (r2 < 0.f) { ia = 1; ib = 0; return; }
        float sq = sqrtf(r2);
        xa = v.x - sq;
        xb = v.x + sq;
        int s0 = __float_as_int(v.w), cnt = __float_as_int(nv.w);
        for (int q = 0; q < cnt; q++) clip_plane(__ldg(F.vert_plane + s0 + q), Y, Z, e, xa, xb);
    }
    const float sl = 1.f / 4096.f;
    float fa = fminf(fmaxf((xa - g.ox) * g.inv_h - 0.5f - sl, (float)bi0), (float)bi1 + 1.f);
    float fb = fmaxf(fminf((xb - g.ox) * g.inv_h - 0.5f + sl, (float)bi1), (float)bi0 - 1.f);
    ia = (int)ceilf(fa);
    ib = (int)floorf(fb);
}

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

// distance from grid point (i, j, k) to feature `id` and the sign from the feature's
// pseudonormal (face normal / n1 + n2 / N_alpha, Section 4.3)
template <int TYPE>
__device__ __forceinline__ float eval_point(const Feat &F, const GridP &g, int id, int i, int j, int k, bool &neg) {
    const float3 p = make_float3(fmaf((float)i + 0.5f, g.h, g.ox), fmaf((float)j + 0.5f, g.h, g.oy),
                                 fmaf((float)k + 0.5f, g.h, g.oz));
    if (TYPE == FACE) {
        const float4 *r = F.face_rec + 4 * id;
        float4 n = __ldg(r), s1 = __ldg(r + 1), s2 = __ldg(r + 2), s3 = __ldg(r + 3);
        float sd = dot3(f3(n), p) + n.w;
        neg = sd < 0.f;
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
        neg = dot3(d, f3(np)) < 0.f;
        return sqrtf(dot3(d, d));
    } else {
        float4 v = __ldg(F.vert_rec + 2 * id), nv = __ldg(F.vert_rec + 2 * id + 1);
        float3 u = p - f3(v);
        neg = dot3(u, f3(nv)) < 0.f;
        return sqrtf(dot3(u, u));
    }
}

template <int TYPE>
__device__ __forceinline__ void process_regions(const Feat &F, const GridP &g, const int32_t *pairs, int64_t q_begin,
                                                int64_t q_end, int tx0, int ty0, int tz0, int cx1, int cy1, int cz1,
                                                unsigned long long *skey, unsigned &cand) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int id_base = TYPE == FACE ? 0 : (TYPE == EDGE ? F.T : F.T + F.E);
    for (int64_t qb = q_begin + (int64_t)warp * 32; qb < q_end; qb += (int64_t)nw * 32) {
        int64_t q = qb + lane;
        int id = 0, bi0 = 0, bi1 = -1, bj0 = 0, bj1 = -1, bk0 = 0, bk1 = -1;
        if (q < q_end) {
            id = __ldg(pairs + q) - id_base;
            if (feature_box<TYPE>(F, g, id, bi0, bi1, bj0, bj1, bk0, bk1)) {
                bi0 = max(bi0, tx0); bi1 = min(bi1, cx1);
                bj0 = max(bj0, ty0); bj1 = min(bj1, cy1);
                bk0 = max(bk0, tz0); bk1 = min(bk1, cz1);
            } else {
                bi1 = -1;
            }
        }
        const int nj = bj1 - bj0 + 1;
        const int nrows = (bi0 <= bi1 && bj0 <= bj1 && bk0 <= bk1) ? nj * (bk1 - bk0 + 1) : 0;
        const int incl = warp_incl_scan(nrows);
        const int total = __shfl_sync(FULL, incl, 31);
        for (int r0 = 0; r0 < total; r0 += 32) {
            const int r = r0 + lane;
            const int o = min(warp_owner(incl, r), 31);
            const int o_excl = __shfl_sync(FULL, incl - nrows, o);
            const int o_id = __shfl_sync(FULL, id, o), o_nj = __shfl_sync(FULL, nj, o);
            const int o_bj0 = __shfl_sync(FULL, bj0, o), o_bk0 = __shfl_sync(FULL, bk0, o);
            const int o_bi0 = __shfl_sync(FULL, bi0, o), o_bi1 = __shfl_sync(FULL, bi1, o);
            int rj = 0, rk = 0, ia = 0, len = 0;
            if (r < total) {
                const int local = r - o_excl;
                rk = o_bk0 + local / o_nj;
                rj = o_bj0 + (local - (rk - o_bk0) * o_nj);
                int ib;
                row_span<TYPE>(F, g, o_id, rj, rk, o_bi0, o_bi1, ia, ib);
                len = max(ib - ia + 1, 0);
            }
            const int pincl = warp_incl_scan(len);
            const int ptotal = __shfl_sync(FULL, pincl, 31);
            for (int p0 = 0; p0 < ptotal; p0 += 32) {
                const int pp = p0 + lane;
                const int ro = min(warp_owner(pincl, pp), 31);
                const int r_start = __shfl_sync(FULL, ia - (pincl - len), ro);
                const int r_j = __shfl_sync(FULL, rj, ro), r_k = __shfl_sync(FULL, rk, ro);
                const int r_id = __shfl_sync(FULL, o_id, ro);
                if (pp < ptotal) {
                    const int pi = r_start + pp;
                    bool neg;
                    float d = eval_point<TYPE>(F, g, r_id, pi, r_j, r_k, neg);
                    if (d < g.W) {
                        unsigned long long key = ((unsigned long long)__float_as_uint(d) << 32) |
                                                 ((unsigned long long)(unsigned)(r_id + id_base) << 1) |
                                                 (unsigned long long)neg;
                        int loc = ((r_k - tz0) * TILE_Y + (r_j - ty0)) * TILE_X + (pi - tx0);
                        atomicMin(skey + loc, key);
                        cand++;
                    }
                }
            }
        }
    }
}

__global__ void __launch_bounds__(NT) k_tile(Feat F, GridP g, Outputs o) {
    __shared__ unsigned long long skey[TILE_PTS];
    __shared__ unsigned s_cand, s_band, s_patch_overflow;
    const int64_t tile = blockIdx.x;
    const int tx = (int)(tile % g.ntx), ty = (int)((tile / g.ntx) % g.nty), tz = (int)(tile / ((int64_t)g.ntx * g.nty));
    const int x0 = tx * TILE_X, y0 = ty * TILE_Y, z0 = tz * TILE_Z;
    const uint32_t *st = o.bin_start + 3 * tile;
    int64_t q0 = st[0], q1 = st[1], q2 = st[2], q3 = st[3];
    q0 = min(q0, o.pair_cap); q1 = min(q1, o.pair_cap); q2 = min(q2, o.pair_cap); q3 = min(q3, o.pair_cap);
    const int64_t plane = (int64_t)g.nx * g.ny;
    if (q0 == q3) {  // no region meets this tile: +inf everywhere (Algorithm 1's initial value)
        for (int e = threadIdx.x; e < TILE_PTS; e += NT) {
            int x = e % TILE_X, y = (e / TILE_X) % TILE_Y, z = e / (TILE_X * TILE_Y);
            int gi = x0 + x, gj = y0 + y, gk = z0 + z;
            if (gi < g.nx && gj < g.ny && gk < g.nz) {
                int64_t idx = (int64_t)gk * plane + (int64_t)gj * g.nx + gi;
                o.dist[idx] = INFINITY;
                if (o.winner) o.winner[idx] = -1;
            }
        }
        return;
    }
    for (int e = threadIdx.x; e < TILE_PTS; e += NT) skey[e] = ~0ull;
    if (threadIdx.x == 0) { s_cand = 0; s_band = 0; s_patch_overflow = 0; }
    __syncthreads();
    const int cx1 = min(x0 + TILE_X, g.nx) - 1, cy1 = min(y0 + TILE_Y, g.ny) - 1, cz1 = min(z0 + TILE_Z, g.nz) - 1;
    unsigned cand = 0;
    process_regions<FACE>(F, g, o.pairs, q0, q1, x0, y0, z0, cx1, cy1, cz1, skey, cand);
    process_regions<EDGE>(F, g, o.pairs, q1, q2, x0, y0, z0, cx1, cy1, cz1, skey, cand);
    process_regions<VERT>(F, g, o.pairs, q2, q3, x0, y0, z0, cx1, cy1, cz1, skey, cand);
    __syncthreads();
    unsigned band = 0;
    for (int e = threadIdx.x; e < TILE_PTS; e += NT) {
        int x = e % TILE_X, y = (e / TILE_X) % TILE_Y, z = e / (TILE_X * TILE_Y);
        int gi = x0 + x, gj = y0 + y, gk = z0 + z;
        if (gi >= g.nx || gj >= g.ny || gk >= g.nz) continue;
        int64_t idx = (int64_t)gk * plane + (int64_t)gj * g.nx + gi;
        unsigned long long key = skey[e];
        float val = INFINITY;
        int wid = -1;
        if (key != ~0ull) {
            float d = __uint_as_float((unsigned)(key >> 32));
            int fid = (int)((key >> 1) & 0x7fffffffu);
            if (d < g.w) {
                val = (key & 1ull) ? -d : d;
                wid = fid;
                band++;
            }
            if (d < g.ds || d >= g.dlo) {  // inside the FP32 error window: re-decide in FP64
                unsigned long long slot = atomicAdd(&o.ctr->n_patch, 1ull);
                if ((int64_t)slot < o.patch_cap) {
                    PatchEntry pe;
                    pe.idx = idx;
                    pe.fid = fid;
                    pe.pad = 0;
                    o.patch[slot] = pe;
                } else {
                    s_patch_overflow = 1;
                }
            }
        }
        o.dist[idx] = val;
        if (o.winner) o.winner[idx] = wid;
    }
    atomicAdd(&s_cand, cand);
    atomicAdd(&s_band, band);
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&o.ctr->n_candidates, (unsigned long long)s_cand);
        atomicAdd(&o.ctr->n_band, (unsigned long long)s_band);
        if (s_patch_overflow) atomicOr(&o.ctr->status, ST_PATCH_OVERFLOW);
    }
}

// ----------------------------------------------------------------------------- FP64 re-decision
// closest point of triangle (a, b, c) to p by Voronoi-region classification of the corner,
// edge and face regions; region 0 face, 1 + k edge (corner k -> k+1), 4 + k corner k
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

// one warp per queued point: FP64 minimum over the triangles around the winner's vertices, sign
// from the pseudonormal of the closest feature (face normal, n1 + n2, or N_alpha, Eq. 8)
__global__ void k_patch(Feat F, GridP g, Outputs o) {
    const int lane = threadIdx.x & 31;
    const int64_t wid0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t n = min((int64_t)o.ctr->n_patch, o.patch_cap);
    const double h = g.h;
    for (int64_t e = wid0; e < n; e += nwarps) {
        PatchEntry pe = o.patch[e];
        const int64_t idx = pe.idx;
        const int fid = pe.fid;
        const int64_t plane = (int64_t)g.nx * g.ny;
        const int gk = (int)(idx / plane), gj = (int)((idx - (int64_t)gk * plane) / g.nx),
                  gi = (int)(idx - (int64_t)gk * plane - (int64_t)gj * g.nx);
        const double3 p = make_double3((double)g.ox + (gi + 0.5) * h, (double)g.oy + (gj + 0.5) * h,
                                       (double)g.oz + (gk + 0.5) * h);
        int vs[3], nv;
        if (fid < F.T) { vs[0] = F.face_vid[3 * fid]; vs[1] = F.face_vid[3 * fid + 1]; vs[2] = F.face_vid[3 * fid + 2]; nv = 3; }
        else if (fid < F.T + F.E) { int4 q = F.edge_vf[fid - F.T]; vs[0] = q.x; vs[1] = q.y; vs[2] = 0; nv = 2; }
        else { vs[0] = fid - F.T - F.E; vs[1] = vs[2] = 0; nv = 1; }
        double bd = INFINITY;
        int bt = 0x7fffffff, breg = 0;
        double3 blam = make_double3(0, 0, 0);
        for (int a = 0; a < nv; a++) {
            const int c0 = F.vert_start[vs[a]], c1 = F.vert_start[vs[a] + 1];
            for (int c = c0 + lane; c < c1; c += 32) {
                const int t = F.vert_corner[c] / 3;
                int reg;
                double3 lam;
                double d2 = closest_on_tri(p, d3(load_vpos(F.vpos, F.face_vid[3 * t])),
                                           d3(load_vpos(F.vpos, F.face_vid[3 * t + 1])),
                                           d3(load_vpos(F.vpos, F.face_vid[3 * t + 2])), reg, lam);
                if (d2 < bd || (d2 == bd && t < bt)) { bd = d2; bt = t; breg = reg; blam = lam; }
            }
        }
        // warp argmin over (d2, triangle)
        int src = lane;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            double od = __shfl_xor_sync(FULL, bd, off);
            int ot = __shfl_xor_sync(FULL, bt, off);
            int os = __shfl_xor_sync(FULL, src, off);
            if (od < bd || (od == bd && ot < bt)) { bd = od; bt = ot; src = os; }
        }
        breg = __shfl_sync(FULL, breg, src);
        blam.x = __shfl_sync(FULL, blam.x, src);
        blam.y = __shfl_sync(FULL, blam.y, src);
        blam.z = __shfl_sync(FULL, blam.z, src);
        const int t = bt;
        const double3 A = d3(load_vpos(F.vpos, F.face_vid[3 * t])), B = d3(load_vpos(F.vpos, F.face_vid[3 * t + 1])),
                      C = d3(load_vpos(F.vpos, F.face_vid[3 * t + 2]));
        double3 N;
        int out_id;
        if (breg == 0) {
            N = tri_normal64(F, t);
            out_id = t;
        } else if (breg <= 3) {
            const int k = breg - 1;
            const int ee = F.face_edge[3 * t + k];
            const int4 q = F.edge_vf[ee];
            N = tri_normal64(F, q.z) + tri_normal64(F, q.w);
            out_id = F.T + ee;
        } else {
            const int u = F.face_vid[3 * t + (breg - 4)];
            const int c0 = F.vert_start[u], c1 = F.vert_start[u + 1];
            const double3 P = d3(load_vpos(F.vpos, u));
            double3 acc = make_double3(0, 0, 0);
            for (int c = c0 + lane; c < c1; c += 32) {  // N_alpha = sum alpha_i n_i, lanes over the fan
                const int cc = F.vert_corner[c];
                const int ft = cc / 3, kk = cc - 3 * ft;
                double3 e1 = d3(load_vpos(F.vpos, F.face_vid[3 * ft + (kk + 1) % 3])) - P;
                double3 e2 = d3(load_vpos(F.vpos, F.face_vid[3 * ft + (kk + 2) % 3])) - P;
                double3 cr = dcross3(e1, e2);
                double alpha = atan2(sqrt(ddot3(cr, cr)), ddot3(e1, e2));
                acc = acc + alpha * tri_normal64(F, ft);
            }
            N = make_double3(wsum(acc.x), wsum(acc.y), wsum(acc.z));
            out_id = F.T + F.E + u;
        }
        // p - q relative to corner A: (p - A) - lam_b (B - A) - lam_c (C - A)
        double3 pq = (p - A) - blam.y * (B - A) - blam.z * (C - A);
        if (breg == 0) pq = p - A;
        const double s = ddot3(pq, N);
        const double d = sqrt(bd);
        if (lane == 0) {
            float val = INFINITY;
            int w = -1;
            if (d < (double)g.w) {
                val = (float)(s < 0.0 ? -d : d);
                w = out_id;
            }
            o.dist[idx] = val;
            if (o.winner) o.winner[idx] = w;
        }
    }
}

inline unsigned nblk(int64_t n, int bt) { return (unsigned)((n + bt - 1) / bt); }

}  // namespace

// ----------------------------------------------------------------------------- host side
static int make_grid(const sdf_grid &gr, float w, GridP &g) {
    if (gr.nx < 1 || gr.ny < 1 || gr.nz < 1 || !(gr.h > 0.f) || !isfinite(gr.h) || !(w > 0.f) || !isfinite(w))
        return SDF_ERR_INVALID_ARG;
    for (int j = 0; j < 3; j++)
        if (!isfinite(gr.origin[j])) return SDF_ERR_INVALID_ARG;
    g.nx = gr.nx; g.ny = gr.ny; g.nz = gr.nz;
    g.ntx = (gr.nx + TILE_X - 1) / TILE_X;
    g.nty = (gr.ny + TILE_Y - 1) / TILE_Y;
    g.ntz = (gr.nz + TILE_Z - 1) / TILE_Z;
    if ((int64_t)g.ntx * g.nty * g.ntz * 3 >= (int64_t(1) << 31)) return SDF_ERR_TOO_LARGE;
    g.ox = gr.origin[0]; g.oy = gr.origin[1]; g.oz = gr.origin[2];
    g.h = gr.h;
    g.inv_h = 1.0f / gr.h;
    // coordinate magnitude M of the problem: FP32 errors of dot products scale with it
    double M = 0.0;
    for (int j = 0; j < 3; j++) {
        int n = j == 0 ? gr.nx : (j == 1 ? gr.ny : gr.nz);
        M = fmax(M, fabs((double)gr.origin[j]));
        M = fmax(M, fabs((double)gr.origin[j] + (double)n * gr.h));
    }
    M = fmax(M, (double)w);
    g.w = w;
    g.eps = (float)(M * 0x1p-21);          // inclusion tolerance, about 8 ulp(M)
    const float dw = (float)(M * 0x1p-21);  // bound on the FP32 distance error
    g.W = w + dw;
    g.dlo = w - dw;
    g.ds = (float)(M * 0x1p-19);           // sign window, 4x the inclusion tolerance
    return SDF_OK;
}

static Feat make_feat(const sdf_features_s *f) {
    Feat F;
    F.T = (int)f->T; F.E = (int)f->E; F.V = (int)f->V;
    F.face_rec = f->face_rec; F.face_box = f->face_box; F.edge_rec = f->edge_rec;
    F.vert_rec = f->vert_rec; F.vert_plane = f->vert_plane;
    F.edge_class = f->edge_class; F.vert_class = f->vert_class;
    F.face_vid = f->face_vid; F.face_edge = f->face_edge; F.vert_start = f->vert_start;
    F.vert_corner = f->vert_corner; F.edge_vf = f->edge_vf; F.vpos = f->vpos;
    F.skip_saddle = (f->flags & SDF_FLAG_DISABLE_SADDLE) ? 1 : 0;
    return F;
}

// one (mesh, grid) problem; returns SDF_OK or an error; sets *retry when scratch was too small
int ensure_events(sdf_features_s *f) {
    for (int i = 0; i < 6; i++)
        if (!f->ev[i]) SDF_TRY(cudaEventCreate(&f->ev[i]));
    return SDF_OK;
}

static int narrow_band_one(sdf_features_s *f, const sdf_grid &gr, float w, float *out, int32_t *win,
                           cudaStream_t s, bool sync, bool timing, bool *retry) {
    GridP g;
    int st = make_grid(gr, w, g);
    if (st) return st;
    Feat F = make_feat(f);
    const int64_t n_tiles = (int64_t)g.ntx * g.nty * g.ntz, n_bins = 3 * n_tiles;
    const int64_t n_feat = f->T + f->E + f->V;
    // scratch: cnt [n_bins], start [n_bins + 1], scan temporaries
    size_t bins_bytes = sizeof(uint32_t) * (size_t)(2 * n_bins + 64);
    SDF_TRY(f->bins.reserve(bins_bytes));
    SDF_TRY(f->scan_tmp.reserve(scan_tmp_bytes(n_bins)));
    if (f->pair_cap == 0) f->pair_cap = 8 * n_feat + 4096;
    if (f->patch_cap == 0) f->patch_cap = n_feat / 8 + 65536;
    SDF_TRY(f->pairs.reserve(sizeof(int32_t) * (size_t)f->pair_cap));
    SDF_TRY(f->patch.reserve(sizeof(PatchEntry) * (size_t)f->patch_cap));
    uint32_t *cnt = f->bins.as<uint32_t>(), *start = cnt + n_bins + 32;
    if (timing) {
        if (ensure_events(f)) return SDF_ERR_CUDA;
        SDF_TRY(cudaEventRecord(f->ev[0], s));
    }
    SDF_TRY(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * n_bins, s));
    SDF_TRY(cudaMemsetAsync(&f->ctr->status, 0, sizeof(unsigned), s));
    SDF_TRY(cudaMemsetAsync(&f->ctr->n_candidates, 0, 4 * sizeof(unsigned long long), s));
    k_bin<false><<<nblk(n_feat, 256), 256, 0, s>>>(F, g, cnt, nullptr, nullptr, 0, f->ctr);
    SDF_LAUNCHED(1);
    SDF_TRY(cudaGetLastError());
    SDF_TRY(scan_exclusive_u32(cnt, start, n_bins, true, f->scan_tmp.p, s));
    SDF_TRY(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * n_bins, s));
    k_bin<true><<<nblk(n_feat, 256), 256, 0, s>>>(F, g, cnt, start, f->pairs.as<int32_t>(), f->pair_cap, f->ctr);
    SDF_LAUNCHED(1);
    SDF_TRY(cudaGetLastError());
    Outputs o;
    o.dist = out;
    o.winner = win;
    o.pairs = f->pairs.as<int32_t>();
    o.bin_start = start;
    o.pair_cap = f->pair_cap;
    o.patch = f->patch.as<PatchEntry>();
    o.patch_cap = f->patch_cap;
    o.ctr = f->ctr;
    if (timing) SDF_TRY(cudaEventRecord(f->ev[1], s));
    k_tile<<<(unsigned)n_tiles, NT, 0, s>>>(F, g, o);
    SDF_LAUNCHED(1);
    SDF_TRY(cudaGetLastError());
    if (timing) SDF_TRY(cudaEventRecord(f->ev[2], s));
    k_patch<<<4 * 152, 256, 0, s>>>(F, g, o);
    SDF_LAUNCHED(1);
    SDF_TRY(cudaGetLastError());
    if (timing) {
        SDF_TRY(cudaEventRecord(f->ev[3], s));
        SDF_TRY(cudaEventSynchronize(f->ev[3]));
        for (int i = 0; i < 3; i++) {
            float ms = 0.f;
            SDF_TRY(cudaEventElapsedTime(&ms, f->ev[i], f->ev[i + 1]));
            f->t_ms[i] += ms;
            f->t_calls[i]++;
        }
    }
    if (!sync) return SDF_OK;
    DevCounters c;
    uint32_t total_pairs = 0;
    SDF_TRY(cudaMemcpyAsync(&c, f->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
    SDF_TRY(cudaMemcpyAsync(&total_pairs, start + n_bins, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    SDF_TRY(cudaStreamSynchronize(s));
    *retry = false;
    if (c.status & ST_PAIR_OVERFLOW) {
        f->pair_cap = (int64_t)total_pairs + total_pairs / 4 + 4096;
        *retry = true;
    }
    if (c.status & ST_PATCH_OVERFLOW) {
        f->patch_cap = (int64_t)c.n_patch + c.n_patch / 2 + 4096;
        *retry = true;
    }
    return SDF_OK;
}

// stats of the last call (host), used by sdf_features_status
int narrow_band_stats(sdf_features_s *f, int64_t *stats, cudaStream_t s) {
    DevCounters c;
    SDF_TRY(cudaMemcpyAsync(&c, f->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
    SDF_TRY(cudaStreamSynchronize(s));
    if (stats) {
        stats[0] = (int64_t)c.n_candidates;
        stats[1] = (int64_t)c.n_band;
        stats[2] = (int64_t)c.n_patch;
        stats[3] = 0;
    }
    if (c.status & (ST_PAIR_OVERFLOW | ST_PATCH_OVERFLOW)) return SDF_ERR_OOM;
    return SDF_OK;
}

int narrow_band_all(const sdf_features *feats, const sdf_grid *grids, const float *band_w, int32_t n,
                    float *const *out_dist, int32_t *const *out_winner, uint32_t flags, cudaStream_t s) {
    if (!feats || !grids || !band_w || n < 1 || !out_dist) return SDF_ERR_INVALID_ARG;
    for (int p = 0; p < n; p++)
        if (!feats[p] || !out_dist[p]) return SDF_ERR_INVALID_ARG;
    const bool sync = !(flags & SDF_FLAG_NO_SYNC), timing = (flags & SDF_FLAG_TIMING) != 0;
    for (int p = 0; p < n; p++) {
        int32_t *win = out_winner ? out_winner[p] : nullptr;
        bool retry = false;
        int st = narrow_band_one(feats[p], grids[p], band_w[p], out_dist[p], win, s, sync, timing, &retry);
        if (st) return st;
        for (int attempt = 0; retry && attempt < 3; attempt++) {
            st = narrow_band_one(feats[p], grids[p], band_w[p], out_dist[p], win, s, sync, timing, &retry);
            if (st) return st;
        }
        if (retry) return SDF_ERR_OOM;
    }
    return SDF_OK;
}

}  // namespace sdf

extern "C" int sdf_narrow_band(const sdf_features *feats, const sdf_grid *grids, const float *band_w, int32_t n,
                               float *const *out_dist, int32_t *const *out_winner, uint32_t flags, void *stream) {
    return sdf::narrow_band_all(feats, grids, band_w, n, out_dist, out_winner, flags,
                                reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int sdf_features_status(sdf_features f, int64_t *stats, void *stream) {
    if (!f) return SDF_ERR_INVALID_ARG;
    return sdf::narrow_band_stats(f, stats, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int sdf_features_timing(sdf_features f, double *ms, int64_t *calls, int reset) {
    if (!f) return SDF_ERR_INVALID_ARG;
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
