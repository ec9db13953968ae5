// Adjoint of the narrow band with respect to the welded vertex positions (a project addition:
// the paper computes no gradients).
//
// A band value is d(p) = s * |p - q(X)|, q the closest point of the winning feature (Eq. 1 with
// the minimum attained on that feature).  With the closest-point weights lam held at the
// minimiser (envelope theorem), d d / d x_k = -s * lam_k * (p - q) / |p - q| for the feature's
// vertices x_k: lam are the barycentric weights on a face, (1 - t, t) on an edge, 1 at a vertex.
// Inside a face region s * (p - q)/|p - q| is the face normal n, so no sign is needed there.
//
// Band points come either from the dense winner array (k_adjoint: compacted over the lanes of a
// warp in grid order) or from a compact band list (k_adjoint_list, which can also form the
// fitting loss's upstream gradient itself); lanes that hit the same vertex in a run are merged by
// a segmented warp scan before the atomicAdd (warp-aggregated atomics), since neighbouring band
// points usually share their winner.  The sums are FP32, or FP64 with SDF_FLAG_GRAD_F64.  The
// file ends with the dense fused loss (sdf_band_l2_loss).
#include "sdf_internal.cuh"

namespace sdf {
namespace {

constexpr unsigned FULL = 0xffffffffu;

struct AdjArgs {
    int T, E, V;
    int nx, ny, nz;
    int kofs;  // index of the first z layer within the whole grid
    FastDiv div_nx, div_ny;
    float ox, oy, oz, h;
    const float *grad;
    const int32_t *winner;
    float *gv;
    float4 *g4;    // FP32 sums per vertex (the handle's grad4), added into gv by k_grad_out
    double *gv64;  // SDF_FLAG_GRAD_F64: the vertex gradient accumulated in FP64 instead
    const float4 *face_rec, *edge_rec, *vert_rec;
    const int32_t *face_vid;
    const int4 *edge_vf;
    const float *vpos;
    const int32_t *vert_start, *vert_corner;
};

// One coordinate of p - x for the grid point p = o + (i + 1/2) h and a vertex coordinate x, with
// relative rather than absolute rounding: o - x is split exactly into hi + lo (Knuth's two-sum),
// hi + (i + 1/2) h is formed by one fused multiply-add, then lo is added.  A plain FP32 p - x
// errs by about u |p|, which near the surface (|p - x| small) ruins the direction (p - q)/|p - q|.
__device__ __forceinline__ float rel_coord(float o, float h, int i, float x) {
    const float a = o, b = -x;
    const float hi = a + b;
    const float bv = hi - a;
    const float lo = (a - (hi - bv)) + (b - bv);
    return fmaf((float)i + 0.5f, h, hi) + lo;
}
__device__ __forceinline__ float3 rel_point(const AdjArgs &a, int i, int j, int k, float3 x) {
    return make_float3(rel_coord(a.ox, a.h, i, x.x), rel_coord(a.oy, a.h, j, x.y), rel_coord(a.oz, a.h, k + a.kofs, x.z));
}

__device__ double3 face_normal64(const AdjArgs &a, int f) {
    const double3 A = d3(load_vpos(a.vpos, a.face_vid[3 * f])), B = d3(load_vpos(a.vpos, a.face_vid[3 * f + 1])),
                  C = d3(load_vpos(a.vpos, a.face_vid[3 * f + 2]));
    const double3 cr = dcross3(B - A, C - A);
    return (1.0 / sqrt(ddot3(cr, cr))) * cr;
}

// FP64 sign of (p - q).N for an edge (N = n1 + n2) or a vertex (N = N_alpha, Eq. 8), taken when the
// FP32 predicate is within 1e-3 |N| |p - q| of zero (its FP32 error is far smaller, so elsewhere the
// FP32 sign is the FP64 one); p is the grid point (i, j, k) in FP64.
__device__ float sign64_edge(const AdjArgs &a, int e, int i, int j, int k) {
    const int4 q = a.edge_vf[e];
    const double3 p = make_double3((double)a.ox + (i + 0.5) * (double)a.h, (double)a.oy + (j + 0.5) * (double)a.h,
                                   (double)a.oz + (k + a.kofs + 0.5) * (double)a.h);
    const double3 A = d3(load_vpos(a.vpos, q.x)), B = d3(load_vpos(a.vpos, q.y));
    const double3 ab = B - A, ap = p - A;
    double t = ddot3(ap, ab) / ddot3(ab, ab);
    t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
    const double3 d = ap - t * ab;
    return ddot3(d, face_normal64(a, q.z) + face_normal64(a, q.w)) < 0.0 ? -1.f : 1.f;
}
__device__ float sign64_vertex(const AdjArgs &a, int v, int i, int j, int k) {
    const double3 p = make_double3((double)a.ox + (i + 0.5) * (double)a.h, (double)a.oy + (j + 0.5) * (double)a.h,
                                   (double)a.oz + (k + a.kofs + 0.5) * (double)a.h);
    const double3 P = d3(load_vpos(a.vpos, v));
    double3 N = make_double3(0, 0, 0);
    for (int c = a.vert_start[v]; c < a.vert_start[v + 1]; c++) {
        const int cc = a.vert_corner[c];
        const int f = cc / 3, kk = cc - 3 * f;
        const double3 e1 = d3(load_vpos(a.vpos, a.face_vid[3 * f + (kk + 1) % 3])) - P;
        const double3 e2 = d3(load_vpos(a.vpos, a.face_vid[3 * f + (kk + 2) % 3])) - P;
        const double3 cr = dcross3(e1, e2);
        N = N + atan2(sqrt(ddot3(cr, cr)), ddot3(e1, e2)) * face_normal64(a, f);
    }
    return ddot3(p - P, N) < 0.0 ? -1.f : 1.f;
}

// add (gx, gy, gz) to vertex v, merged over runs of consecutive lanes that target the same vertex
// (band points arrive in grid order, so neighbours with a common winner sit in adjacent lanes): a
// segmented warp scan sums each run and its last lane issues the atomics.  T is the accumulation
// type (float, or double for SDF_FLAG_GRAD_F64, where the run sums are taken in FP64 as well).
template <typename T>
__device__ __forceinline__ void warp_add(T *gv, int v, T gx, T gy, T gz, bool active) {
    const int lane = threadIdx.x & 31;
    const int key = active ? v : -1;
    const int prev = __shfl_up_sync(FULL, key, 1), next = __shfl_down_sync(FULL, key, 1);
    const unsigned heads = __ballot_sync(FULL, lane == 0 || prev != key);
    const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));  // first lane of this run
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T tx = __shfl_up_sync(FULL, gx, o), ty = __shfl_up_sync(FULL, gy, o),
                tz = __shfl_up_sync(FULL, gz, o);
        if (lane - o >= start) {
            gx += tx;
            gy += ty;
            gz += tz;
        }
    }
    if (active && (lane == 31 || next != key)) {
        atomicAdd(gv + 3 * v, gx);
        atomicAdd(gv + 3 * v + 1, gy);
        atomicAdd(gv + 3 * v + 2, gz);
    }
}

// The FP32 sums go to a float4 per vertex, one vector atomic (red.global.add.v4.f32) per run
// instead of three scalar ones: on the 50 k-triangle torus the list adjoint took 0.118 instead of
// 0.157 ms, close to the 0.113 ms of a copy with no atomics at all.  k_grad_out then adds the
// float4 sums into the caller's float[V][3] gradient and clears them.
__device__ __forceinline__ void warp_add4(float4 *g4, int v, float gx, float gy, float gz, bool active) {
    const int lane = threadIdx.x & 31;
    const int key = active ? v : -1;
    const int prev = __shfl_up_sync(FULL, key, 1), next = __shfl_down_sync(FULL, key, 1);
    const unsigned heads = __ballot_sync(FULL, lane == 0 || prev != key);
    const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));  // first lane of this run
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float tx = __shfl_up_sync(FULL, gx, o), ty = __shfl_up_sync(FULL, gy, o),
                    tz = __shfl_up_sync(FULL, gz, o);
        if (lane - o >= start) {
            gx += tx;
            gy += ty;
            gz += tz;
        }
    }
    if (active && (lane == 31 || next != key)) atomicAdd(g4 + v, make_float4(gx, gy, gz, 0.f));
}

// the contributions of one point (from point_adjoint) into the FP32 or FP64 vertex gradient
template <bool F64>
__device__ __forceinline__ void add_point(const AdjArgs &a, const int *vtx, const float (*c)[3], int nv) {
    for (int q = 0; q < 3; q++) {
        if (F64)
            warp_add<double>(a.gv64, vtx[q], (double)c[q][0], (double)c[q][1], (double)c[q][2], q < nv);
        else
            warp_add4(a.g4, vtx[q], c[q][0], c[q][1], c[q][2], q < nv);
    }
}

// adds the FP32 sums of an adjoint call into the caller's float[V][3] gradient and clears them
__global__ void k_grad_out(float4 *g4, float *gv, int64_t V) {
    dep_wait();
    dep_next();
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= V) return;
    const float4 t = g4[v];
    if (t.x != 0.f || t.y != 0.f || t.z != 0.f) {
        gv[3 * v] += t.x;
        gv[3 * v + 1] += t.y;
        gv[3 * v + 2] += t.z;
        g4[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// contribution of band point idx (winner wid, upstream gradient g) to at most 3 vertices
__device__ __forceinline__ int point_adjoint(const AdjArgs &a, int64_t idx, int wid, float g, int *vtx, float (*c)[3]) {
    int i, j, k;
    if (idx < (int64_t(1) << 31)) {
        const uint32_t iu = (uint32_t)idx, r1 = a.div_nx.div(iu), r2 = a.div_ny.div(r1);
        i = (int)(iu - r1 * (uint32_t)a.nx);
        j = (int)(r1 - r2 * (uint32_t)a.ny);
        k = (int)r2;
    } else {
        const int64_t plane = (int64_t)a.nx * a.ny;
        k = (int)(idx / plane);
        j = (int)((idx - (int64_t)k * plane) / a.nx);
        i = (int)(idx - (int64_t)k * plane - (int64_t)j * a.nx);
    }
    if (wid < a.T) {
        // barycentric weights of the projection of p onto the face plane; s (p - q)/|p - q| = n
        const int f = wid;
        const float3 A = load_vpos(a.vpos, a.face_vid[3 * f]), B = load_vpos(a.vpos, a.face_vid[3 * f + 1]),
                     C = load_vpos(a.vpos, a.face_vid[3 * f + 2]);
        const float3 n = f3(a.face_rec[4 * f]);
        const float3 ab = B - A, ac = C - A, ap = rel_point(a, i, j, k, A);
        const float d00 = dot3(ab, ab), d01 = dot3(ab, ac), d11 = dot3(ac, ac);
        const float d20 = dot3(ap, ab), d21 = dot3(ap, ac);
        const float den = d00 * d11 - d01 * d01;
        const float lb = (d11 * d20 - d01 * d21) / den, lc = (d00 * d21 - d01 * d20) / den;
        if (lb >= 0.f && lc >= 0.f && lb + lc <= 1.f) {
            const float lam[3] = {1.f - lb - lc, lb, lc};
            for (int q = 0; q < 3; q++) {
                vtx[q] = a.face_vid[3 * f + q];
                c[q][0] = -g * lam[q] * n.x;
                c[q][1] = -g * lam[q] * n.y;
                c[q][2] = -g * lam[q] * n.z;
            }
            return 3;
        }
        // a point of the inclusion margin: its closest point of the closed triangle lies on the
        // boundary, q = A + lb ab + lc ac on the nearest of the three edges, and the contribution
        // takes the direction (p - q)/|p - q| with the face's sign, as at an edge
        float best = INFINITY, bb = 0.f, bc = 0.f;
        {
            const float t = fminf(fmaxf(d20 / d00, 0.f), 1.f);  // edge AB
            const float3 r = ap - t * ab;
            const float e = dot3(r, r);
            if (e < best) { best = e; bb = t; bc = 0.f; }
        }
        {
            const float t = fminf(fmaxf(d21 / d11, 0.f), 1.f);  // edge AC
            const float3 r = ap - t * ac;
            const float e = dot3(r, r);
            if (e < best) { best = e; bb = 0.f; bc = t; }
        }
        {
            const float3 bcv = ac - ab, bp = ap - ab;  // edge BC
            const float t = fminf(fmaxf(dot3(bp, bcv) / dot3(bcv, bcv), 0.f), 1.f);
            const float3 r = bp - t * bcv;
            const float e = dot3(r, r);
            if (e < best) { best = e; bb = 1.f - t; bc = t; }
        }
        const float3 d = ap - bb * ab - bc * ac;
        const float len = sqrtf(dot3(d, d));
        if (!(len > 0.f)) return 0;
        const float s = dot3(d, n) < 0.f ? -1.f : 1.f;
        const float lam[3] = {1.f - bb - bc, bb, bc};
        const float k0 = -g * s / len;
        for (int q = 0; q < 3; q++) {
            vtx[q] = a.face_vid[3 * f + q];
            c[q][0] = k0 * lam[q] * d.x;
            c[q][1] = k0 * lam[q] * d.y;
            c[q][2] = k0 * lam[q] * d.z;
        }
        return 3;
    } else if (wid < a.T + a.E) {
        const int e = wid - a.T;
        const int4 q = a.edge_vf[e];
        const float4 r0 = a.edge_rec[5 * e], r1 = a.edge_rec[5 * e + 1], np = a.edge_rec[5 * e + 4];
        const float3 u = rel_point(a, i, j, k, f3(r0));
        const float t = fminf(fmaxf(dot3(u, f3(r1)), 0.f), r0.w);
        const float3 d = u - t * f3(r1);
        const float len = sqrtf(dot3(d, d));
        if (!(len > 0.f)) return 0;
        const float P = dot3(d, f3(np));
        const float s = fabsf(P) < 1e-3f * np.w * len ? sign64_edge(a, e, i, j, k) : (P < 0.f ? -1.f : 1.f);
        const float tt = t / r0.w;
        const float lam[2] = {1.f - tt, tt};
        const float k0 = -g * s / len;
        for (int qq = 0; qq < 2; qq++) {
            vtx[qq] = qq == 0 ? q.x : q.y;
            c[qq][0] = k0 * lam[qq] * d.x;
            c[qq][1] = k0 * lam[qq] * d.y;
            c[qq][2] = k0 * lam[qq] * d.z;
        }
        return 2;
    } else {
        const int v = wid - a.T - a.E;
        const float4 r0 = a.vert_rec[3 * v], r1 = a.vert_rec[3 * v + 1];
        const float3 d = rel_point(a, i, j, k, f3(r0));
        const float len = sqrtf(dot3(d, d));
        if (!(len > 0.f)) return 0;
        const float P = dot3(d, f3(r1));
        const float s = fabsf(P) < 1e-3f * len ? sign64_vertex(a, v, i, j, k) : (P < 0.f ? -1.f : 1.f);
        const float k0 = -g * s / len;
        vtx[0] = v;
        c[0][0] = k0 * d.x;
        c[0][1] = k0 * d.y;
        c[0][2] = k0 * d.z;
        return 1;
    }
}

__device__ __forceinline__ int warp_incl_scan_i(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Each lane reads the winners of 4 consecutive grid points (one int4 when vec is set).  The band
// points among a warp's 128 points are appended, in grid order, to a per-warp ring in shared
// memory; whenever 32 are waiting, each lane takes one, computes its vertex contributions, and
// neighbouring points, which mostly share a winner, are merged by warp_add before the atomics.
// The band is a thin shell, so most passes hold only a few band points: the ring keeps the
// contribution step on full warps.
constexpr int ADJ_RING = 256;  // > 31 waiting + 128 appended per pass

template <bool F64>
__device__ __forceinline__ void adjoint_batch(const AdjArgs &a, const long long *ridx, const int *rwid, int q0,
                                              int m) {
    const int lane = threadIdx.x & 31;
    bool act = false;
    int wid = -1;
    int64_t idx = 0;
    float g = 0.f;
    if (lane < m) {
        const int e = (q0 + lane) & (ADJ_RING - 1);
        idx = ridx[e];
        wid = rwid[e];
        g = __ldg(a.grad + idx);
        act = g != 0.f;
    }
    int vtx[3] = {0, 0, 0};
    float c[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    const int nv = act ? point_adjoint(a, idx, wid, g, vtx, c) : 0;
    add_point<F64>(a, vtx, c, nv);
}

template <bool F64>
__global__ void __launch_bounds__(256) k_adjoint(AdjArgs a, int vec) {
    __shared__ long long s_idx[8][ADJ_RING];
    __shared__ int s_wid[8][ADJ_RING];
    const int warp = threadIdx.x >> 5;
    long long *ridx = s_idx[warp];
    int *rwid = s_wid[warp];
    const int64_t n = (int64_t)a.nx * a.ny * a.nz;
    const int64_t n4 = (n + 3) / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int qh = 0, qn = 0;  // ring head and length (warp-uniform)
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n4; base += stride) {
        const int64_t q4 = base + threadIdx.x;
        int w4[4] = {-1, -1, -1, -1};
        if (q4 < n4) {
            if (vec) {
                const int4 w = __ldg(reinterpret_cast<const int4 *>(a.winner) + q4);
                w4[0] = w.x; w4[1] = w.y; w4[2] = w.z; w4[3] = w.w;
            } else {
                for (int u = 0; u < 4; u++)
                    if (4 * q4 + u < n) w4[u] = __ldg(a.winner + 4 * q4 + u);
            }
        }
        const int cnt = (w4[0] >= 0) + (w4[1] >= 0) + (w4[2] >= 0) + (w4[3] >= 0);
        const int incl = warp_incl_scan_i(cnt);
        const int total = __shfl_sync(FULL, incl, 31);
        if (total == 0) continue;
        int pos = qh + qn + incl - cnt;
        for (int u = 0; u < 4; u++) {
            if (w4[u] >= 0) {
                ridx[pos & (ADJ_RING - 1)] = 4 * q4 + u;
                rwid[pos & (ADJ_RING - 1)] = w4[u];
                pos++;
            }
        }
        qn += total;
        __syncwarp();
        while (qn >= 32) {
            adjoint_batch<F64>(a, ridx, rwid, qh, 32);
            qh = (qh + 32) & (ADJ_RING - 1);
            qn -= 32;
        }
        __syncwarp();  // ring slots are rewritten by the next pass
    }
    if (qn > 0) adjoint_batch<F64>(a, ridx, rwid, qh, qn);
}

// The adjoint over a compact band list: a warp takes 32 consecutive entries (one per lane; the
// list holds a tile's band points in tile order, so neighbours mostly share a winner for
// warp_add).  The upstream gradient is read at the listed point (a.grad), or, when target is
// set, formed there as 2 (d - target) with the loss (d - target)^2 summed in FP64 (the
// shape-fitting loss fused with its adjoint).
template <bool F64>
__global__ void __launch_bounds__(256) k_adjoint_list(AdjArgs a, const uint2 *list, const unsigned long long *count,
                                                      long long cap, const float *dist, const float *target,
                                                      double *loss, unsigned long long *band_out) {
    const long long n = min((long long)*count, cap);
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    double acc = 0.0;
    unsigned cnt = 0;
    // warp-uniform trip count: warp_add votes over all 32 lanes
    for (long long e0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) & ~31ll; e0 < n; e0 += stride) {
        const long long e = e0 + lane;
        bool act = false;
        uint2 en = make_uint2(0u, 0u);
        float g = 0.f;
        if (e < n) {
            en = __ldcs(list + e);
            if (target) {
                const float df = __ldg(dist + en.x) - __ldg(target + en.x);
                g = 2.f * df;
                acc += (double)df * df;
                cnt++;
            } else {
                g = __ldg(a.grad + en.x);
            }
            act = g != 0.f;
        }
        int vtx[3] = {0, 0, 0};
        float c[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        const int nv = act ? point_adjoint(a, (int64_t)en.x, (int)en.y, g, vtx, c) : 0;
        add_point<F64>(a, vtx, c, nv);
    }
    if (!target) return;
    // loss and count: warp sums, then one atomic per block
    cnt = __reduce_add_sync(FULL, cnt);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    __shared__ double s_acc[8];
    __shared__ unsigned s_cnt[8];
    if (lane == 0) {
        s_acc[threadIdx.x >> 5] = acc;
        s_cnt[threadIdx.x >> 5] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        unsigned long long c = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            b += s_acc[w];
            c += s_cnt[w];
        }
        if (c) {
            atomicAdd(loss, b);
            if (band_out) atomicAdd(band_out, c);
        }
    }
}

AdjArgs make_adj_args(const sdf_features_s *f, const sdf_grid &gr) {
    AdjArgs a;
    a.T = (int)f->T; a.E = (int)f->E; a.V = (int)f->V;
    a.nx = gr.nx; a.ny = gr.ny; a.nz = gr.nz;
    a.kofs = gr.k0;
    a.div_nx = FastDiv((uint32_t)gr.nx);
    a.div_ny = FastDiv((uint32_t)gr.ny);
    a.ox = gr.origin[0]; a.oy = gr.origin[1]; a.oz = gr.origin[2]; a.h = gr.h;
    a.grad = nullptr;
    a.winner = nullptr;
    a.gv = nullptr;
    a.g4 = f->grad4;
    a.gv64 = nullptr;
    a.face_rec = f->face_rec; a.edge_rec = f->edge_rec; a.vert_rec = f->vert_rec;
    a.face_vid = f->face_vid; a.edge_vf = f->edge_vf; a.vpos = f->vpos;
    a.vert_start = f->vert_start; a.vert_corner = f->vert_corner;
    return a;
}

int list_adjoint(sdf_features_s *f, const sdf_grid *grid, const sdf_band_entry *list, int64_t list_cap,
                 const unsigned long long *list_count, const float *grad_dist, const float *dist,
                 const float *target, float *grad_vertices, double *loss_out, unsigned long long *band_out,
                 uint32_t flags, cudaStream_t s) {
    if (!f || !grid || !list || !list_count || list_cap < 0 || !grad_vertices) return SDF_ERR_INVALID_ARG;
    const sdf_grid &gr = *grid;
    if (gr.nx < 1 || gr.ny < 1 || gr.nz < 1 || !(gr.h > 0.f) || gr.k0 < 0) return SDF_ERR_INVALID_ARG;
    if ((long long)gr.nx * gr.ny * gr.nz > (long long)UINT32_MAX) return SDF_ERR_TOO_LARGE;
    AdjArgs a = make_adj_args(f, gr);
    a.grad = grad_dist;
    const bool f64 = (flags & SDF_FLAG_GRAD_F64) != 0;
    a.gv = f64 ? nullptr : grad_vertices;
    a.gv64 = f64 ? reinterpret_cast<double *>(grad_vertices) : nullptr;
    if (target) {
        SDF_TRY(cudaMemsetAsync(loss_out, 0, sizeof(double), s));
        if (band_out) SDF_TRY(cudaMemsetAsync(band_out, 0, sizeof(unsigned long long), s));
    }
    static int n_sm = 0;
    if (!n_sm) {
        int dev = 0;
        SDF_TRY(cudaGetDevice(&dev));
        SDF_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    }
    const bool timing = (flags & SDF_FLAG_TIMING) != 0;
    if (timing) {
        if (ensure_events(f)) return SDF_ERR_CUDA;
        SDF_TRY_ST(resolve_timing(f));
        SDF_TRY(cudaEventRecord(f->ev[4], s));
    }
    // the length is known on the device only: a grid of 8 CTAs per SM strides over the list
    if (f64)
        k_adjoint_list<true><<<8 * n_sm, 256, 0, s>>>(a, reinterpret_cast<const uint2 *>(list), list_count,
                                                       (long long)list_cap, dist, target, loss_out, band_out);
    else
        k_adjoint_list<false><<<8 * n_sm, 256, 0, s>>>(a, reinterpret_cast<const uint2 *>(list), list_count,
                                                        (long long)list_cap, dist, target, loss_out, band_out);
    SDF_LAUNCHED(1);
    SDF_TRY(cudaGetLastError());
    if (!f64)
        SDF_TRY(launch_dep(k_grad_out, dim3((unsigned)((f->V + 255) / 256)), dim3(256), 0, s, f->grad4,
                           grad_vertices, (int64_t)f->V));
    if (timing) {
        SDF_TRY(cudaEventRecord(f->ev[5], s));
        f->adj_pending = true;  // read later (resolve_timing)
    }
    return SDF_OK;
}

}  // namespace


}  // namespace sdf

using namespace sdf;

extern "C" int sdf_band_list_backward(sdf_features f, const sdf_grid *grid, const sdf_band_entry *list,
                                      int64_t list_cap, const unsigned long long *list_count, const float *grad_dist,
                                      float *grad_vertices, uint32_t flags, void *stream) {
    if (!grad_dist) return SDF_ERR_INVALID_ARG;
    return list_adjoint(f, grid, list, list_cap, list_count, grad_dist, nullptr, nullptr, grad_vertices, nullptr,
                        nullptr, flags, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int sdf_band_list_l2(sdf_features f, const sdf_grid *grid, const sdf_band_entry *list, int64_t list_cap,
                                const unsigned long long *list_count, const float *dist, const float *target,
                                float *grad_vertices, double *loss_out, unsigned long long *band_out, uint32_t flags,
                                void *stream) {
    if (!dist || !target || !loss_out) return SDF_ERR_INVALID_ARG;
    return list_adjoint(f, grid, list, list_cap, list_count, nullptr, dist, target, grad_vertices, loss_out, band_out,
                        flags, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int sdf_narrow_band_backward(const sdf_features *feats, const sdf_grid *grids, const float *band_w,
                                        int32_t n, const float *const *grad_dist, const int32_t *const *winner,
                                        float *const *grad_vertices, uint32_t flags, void *stream) {
    if (!feats || !grids || n < 1 || !grad_dist || !grad_vertices) return SDF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    for (int p = 0; p < n; p++) {
        sdf_features_s *f = feats[p];
        const sdf_grid &gr = grids[p];
        if (!f || !grad_dist[p] || !grad_vertices[p]) return SDF_ERR_INVALID_ARG;
        if (gr.nx < 1 || gr.ny < 1 || gr.nz < 1 || !(gr.h > 0.f) || gr.k0 < 0) return SDF_ERR_INVALID_ARG;
        const int64_t npts = (int64_t)gr.nx * gr.ny * gr.nz;
        const int32_t *win = winner ? winner[p] : nullptr;
        if (!win) {  // recompute the winners with a forward pass into library scratch
            if (!band_w) return SDF_ERR_INVALID_ARG;
            SDF_TRY(f->fwd_winner.reserve((size_t)npts * (sizeof(int32_t) + sizeof(float)), s));
            int32_t *w = f->fwd_winner.as<int32_t>();
            float *dscratch = reinterpret_cast<float *>(w + npts);
            float *const dl[1] = {dscratch};
            int32_t *const wl[1] = {w};
            sdf_features fl[1] = {f};
            int st = narrow_band_all(fl, &gr, band_w + p, 1, dl, wl, flags, s);
            if (st) return st;
            win = w;
        }
        AdjArgs a = make_adj_args(f, gr);
        a.grad = grad_dist[p];
        a.winner = win;
        const bool f64 = (flags & SDF_FLAG_GRAD_F64) != 0;
        a.gv = f64 ? nullptr : grad_vertices[p];
        a.gv64 = f64 ? reinterpret_cast<double *>(grad_vertices[p]) : nullptr;
        int64_t blocks = ((npts + 3) / 4 + 255) / 256;
        if (blocks > 152 * 16) blocks = 152 * 16;
        const int vec = (npts % 4 == 0) && ((reinterpret_cast<uintptr_t>(win) & 15) == 0);
        const bool timing = (flags & SDF_FLAG_TIMING) != 0;
        if (timing) {
            if (ensure_events(f)) return SDF_ERR_CUDA;
            SDF_TRY_ST(resolve_timing(f));
            SDF_TRY(cudaEventRecord(f->ev[4], s));
        }
        if (f64)
            k_adjoint<true><<<(unsigned)blocks, 256, 0, s>>>(a, vec);
        else
            k_adjoint<false><<<(unsigned)blocks, 256, 0, s>>>(a, vec);
        SDF_LAUNCHED(1);
        SDF_TRY(cudaGetLastError());
        if (!f64)
            SDF_TRY(launch_dep(k_grad_out, dim3((unsigned)((f->V + 255) / 256)), dim3(256), 0, s, f->grad4,
                               grad_vertices[p], (int64_t)f->V));
        if (timing) {
            SDF_TRY(cudaEventRecord(f->ev[5], s));
            f->adj_pending = true;  // read later (resolve_timing)
        }
    }
    return SDF_OK;
}

// ----------------------------------------------------------------------------- band L2 loss
// L = sum over band points of (d - target)^2 and its gradient dL/dd = 2 (d - target) on the band,
// 0 elsewhere, in one pass over the grid (the loss of the shape-fitting workload; the paper has no
// loss).  Points outside the band hold +-inf in d and contribute nothing.
namespace sdf {
namespace {
__global__ void __launch_bounds__(256) k_band_l2(const float *dist, const float *target, int64_t n, float *grad,
                                                 double *loss, unsigned long long *band, int vec) {
    double acc = 0.0;
    unsigned cnt = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (vec) {
        const int64_t n4 = n / 4;
        // the trip count is uniform across each warp (the warp vote below needs all 32 lanes)
        for (int64_t q0 = t0 & ~(int64_t)31; q0 < n4; q0 += stride) {
            const int64_t q = q0 + (threadIdx.x & 31);
            const bool in = q < n4;
            const float4 d = in ? __ldcs(reinterpret_cast<const float4 *>(dist) + q)
                                : make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
            const float4 t = in ? __ldcs(reinterpret_cast<const float4 *>(target) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 gq;
            const float dx = d.x - t.x, dy = d.y - t.y, dz = d.z - t.z, dw = d.w - t.w;
            gq.x = isfinite(d.x) ? 2.f * dx : 0.f;
            gq.y = isfinite(d.y) ? 2.f * dy : 0.f;
            gq.z = isfinite(d.z) ? 2.f * dz : 0.f;
            gq.w = isfinite(d.w) ? 2.f * dw : 0.f;
            const unsigned fin = isfinite(d.x) | isfinite(d.y) << 1 | isfinite(d.z) << 2 | isfinite(d.w) << 3;
            // FP64 runs at a small fraction of the FP32 rate on this part and band points are a few
            // percent of the grid: the FP64 sum is taken only by warps that hold a band point
            if (__any_sync(0xffffffffu, fin != 0u)) {
                acc += ((fin & 1u) ? (double)dx * dx : 0.0) + ((fin & 2u) ? (double)dy * dy : 0.0) +
                       ((fin & 4u) ? (double)dz * dz : 0.0) + ((fin & 8u) ? (double)dw * dw : 0.0);
                cnt += __popc(fin);
            }
            if (grad && in) __stcs(reinterpret_cast<float4 *>(grad) + q, gq);
        }
        for (int64_t q = 4 * n4 + t0; q < n; q += stride) {  // tail of a length that is not a multiple of 4
            const float d = dist[q], t = target[q], df = d - t;
            if (grad) grad[q] = isfinite(d) ? 2.f * df : 0.f;
            if (isfinite(d)) { acc += (double)df * df; cnt++; }
        }
    } else {
        for (int64_t q0 = t0 & ~(int64_t)31; q0 < n; q0 += stride) {  // warp-uniform trip count
            const int64_t q = q0 + (threadIdx.x & 31);
            const float d = q < n ? dist[q] : INFINITY, t = q < n ? target[q] : 0.f, df = d - t;
            if (grad && q < n) grad[q] = isfinite(d) ? 2.f * df : 0.f;
            if (__any_sync(0xffffffffu, isfinite(d)) && isfinite(d)) { acc += (double)df * df; cnt++; }
        }
    }
    // band points: one atomic per warp
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (band && (threadIdx.x & 31) == 0 && cnt) atomicAdd(band, (unsigned long long)cnt);
    // block sum in FP64, one atomic per block
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double s_acc[8];
    if ((threadIdx.x & 31) == 0) s_acc[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) b += s_acc[w];
        atomicAdd(loss, b);
    }
}
}  // namespace
}  // namespace sdf

extern "C" int sdf_band_l2_loss(const float *dist, const float *target, int64_t n, float *grad_out, double *loss_out,
                                unsigned long long *band_out, void *stream) {
    using namespace sdf;
    if (!dist || !target || !loss_out || n < 0) return SDF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    SDF_TRY(cudaMemsetAsync(loss_out, 0, sizeof(double), s));
    if (band_out) SDF_TRY(cudaMemsetAsync(band_out, 0, sizeof(unsigned long long), s));
    if (n == 0) return SDF_OK;
    static int n_sm = 0;
    if (!n_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (n_sm <= 0) n_sm = 152;
    }
    const int vec = ((reinterpret_cast<uintptr_t>(dist) | reinterpret_cast<uintptr_t>(target) |
                      reinterpret_cast<uintptr_t>(grad_out)) & 15) == 0;
    int64_t blocks = (n / (vec ? 4 : 1) + 255) / 256;
    if (blocks > 8 * (int64_t)n_sm) blocks = 8 * (int64_t)n_sm;
    if (blocks < 1) blocks = 1;
    k_band_l2<<<(unsigned)blocks, 256, 0, s>>>(dist, target, n, grad_out, loss_out, band_out, vec);
    SDF_LAUNCHED(1);
    SDF_TRY(cudaGetLastError());
    return SDF_OK;
}
