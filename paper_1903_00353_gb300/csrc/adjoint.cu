// Adjoint of the narrow band with respect to the welded vertex positions (a project addition:
// the paper computes no gradients).
//
// A band value is d(p) = s * |p - q(X)|, q the closest point of the winning feature (Eq. 1 with
// the minimum attained on that feature).  With the closest-point weights lam held at the
// minimiser (envelope theorem), d d / d x_k = -s * lam_k * (p - q) / |p - q| for the feature's
// vertices x_k: lam are the barycentric weights on a face, (1 - t, t) on an edge, 1 at a vertex.
// Inside a face region s * (p - q)/|p - q| is the face normal n, so no sign is needed there.
//
// One thread per grid point; threads of a warp that hit the same vertex are merged with
// __match_any_sync before the atomicAdd (warp-aggregated atomics), since neighbouring band
// points usually share their winner.
#include "sdf_internal.cuh"

namespace sdf {
namespace {

constexpr unsigned FULL = 0xffffffffu;

struct AdjArgs {
    int T, E, V;
    int nx, ny, nz;
    float ox, oy, oz, h;
    const float *grad;
    const int32_t *winner;
    float *gv;
    const float4 *face_rec, *edge_rec, *vert_rec;
    const int32_t *face_vid;
    const int4 *edge_vf;
    const float *vpos;
};

// add (gx, gy, gz) to vertex v, merged across the lanes of the warp that target the same vertex
__device__ __forceinline__ void warp_add(float *gv, int v, float gx, float gy, float gz, bool active) {
    const int lane = threadIdx.x & 31;
    int key = active ? v : -1 - lane;  // inactive lanes form singleton groups
    unsigned peers = __match_any_sync(FULL, key);
    int leader = __ffs(peers) - 1;
    // reduce within the peer group: each lane walks its group with shuffles
    float sx = 0.f, sy = 0.f, sz = 0.f;
    unsigned m = peers;
    while (m) {
        int src = __ffs(m) - 1;
        m &= m - 1;
        sx += __shfl_sync(peers, gx, src);
        sy += __shfl_sync(peers, gy, src);
        sz += __shfl_sync(peers, gz, src);
    }
    if (active && lane == leader) {
        atomicAdd(gv + 3 * v, sx);
        atomicAdd(gv + 3 * v + 1, sy);
        atomicAdd(gv + 3 * v + 2, sz);
    }
}

__global__ void k_adjoint(AdjArgs a) {
    const int64_t n = (int64_t)a.nx * a.ny * a.nz;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += stride) {
        const int64_t idx = base + threadIdx.x;
        int wid = -1;
        float g = 0.f;
        if (idx < n) {
            wid = a.winner[idx];
            if (wid >= 0) g = a.grad[idx];
        }
        bool act = wid >= 0 && g != 0.f;
        if (!__any_sync(FULL, act)) continue;
        int vtx[3] = {0, 0, 0};
        float c[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        int nv = 0;
        if (act) {
            const int64_t plane = (int64_t)a.nx * a.ny;
            const int k = (int)(idx / plane), j = (int)((idx - (int64_t)k * plane) / a.nx),
                      i = (int)(idx - (int64_t)k * plane - (int64_t)j * a.nx);
            const float3 p = make_float3(fmaf((float)i + 0.5f, a.h, a.ox), fmaf((float)j + 0.5f, a.h, a.oy),
                                         fmaf((float)k + 0.5f, a.h, a.oz));
            if (wid < a.T) {
                // barycentric weights of the projection of p onto the face plane
                const int f = wid;
                float3 A = load_vpos(a.vpos, a.face_vid[3 * f]), B = load_vpos(a.vpos, a.face_vid[3 * f + 1]),
                       C = load_vpos(a.vpos, a.face_vid[3 * f + 2]);
                float3 n = f3(a.face_rec[4 * f]);
                float3 ab = B - A, ac = C - A, ap = p - A;
                float d00 = dot3(ab, ab), d01 = dot3(ab, ac), d11 = dot3(ac, ac);
                float d20 = dot3(ap, ab), d21 = dot3(ap, ac);
                float den = d00 * d11 - d01 * d01;
                float lb = (d11 * d20 - d01 * d21) / den, lc = (d00 * d21 - d01 * d20) / den;
                // points of the inclusion margin project just outside: clamp onto the triangle
                lb = fmaxf(lb, 0.f);
                lc = fmaxf(lc, 0.f);
                float sum = lb + lc;
                if (sum > 1.f) { lb /= sum; lc /= sum; }
                float la = 1.f - lb - lc;
                float lam[3] = {la, lb, lc};
                for (int q = 0; q < 3; q++) {
                    vtx[q] = a.face_vid[3 * f + q];
                    c[q][0] = -g * lam[q] * n.x;
                    c[q][1] = -g * lam[q] * n.y;
                    c[q][2] = -g * lam[q] * n.z;
                }
                nv = 3;
            } else if (wid < a.T + a.E) {
                const int e = wid - a.T;
                const int4 q = a.edge_vf[e];
                float4 r0 = a.edge_rec[5 * e], r1 = a.edge_rec[5 * e + 1], np = a.edge_rec[5 * e + 4];
                float3 u = p - f3(r0);
                float t = fminf(fmaxf(dot3(u, f3(r1)), 0.f), r0.w);
                float3 d = u - t * f3(r1);
                float len = sqrtf(dot3(d, d));
                if (len > 0.f) {
                    float s = dot3(d, f3(np)) < 0.f ? -1.f : 1.f;
                    float tt = t / r0.w;
                    float lam[2] = {1.f - tt, tt};
                    float k0 = -g * s / len;
                    for (int qq = 0; qq < 2; qq++) {
                        vtx[qq] = qq == 0 ? q.x : q.y;
                        c[qq][0] = k0 * lam[qq] * d.x;
                        c[qq][1] = k0 * lam[qq] * d.y;
                        c[qq][2] = k0 * lam[qq] * d.z;
                    }
                    nv = 2;
                }
            } else {
                const int v = wid - a.T - a.E;
                float4 r0 = a.vert_rec[3 * v], r1 = a.vert_rec[3 * v + 1];
                float3 d = p - f3(r0);
                float len = sqrtf(dot3(d, d));
                if (len > 0.f) {
                    float s = dot3(d, f3(r1)) < 0.f ? -1.f : 1.f;
                    float k0 = -g * s / len;
                    vtx[0] = v;
                    c[0][0] = k0 * d.x;
                    c[0][1] = k0 * d.y;
                    c[0][2] = k0 * d.z;
                    nv = 1;
                }
            }
        }
        for (int q = 0; q < 3; q++) warp_add(a.gv, vtx[q], c[q][0], c[q][1], c[q][2], act && q < nv);
    }
}

}  // namespace

int narrow_band_all(const sdf_features *feats, const sdf_grid *grids, const float *band_w, int32_t n,
                    float *const *out_dist, int32_t *const *out_winner, uint32_t flags, cudaStream_t s);
int ensure_events(sdf_features_s *f);

}  // namespace sdf

using namespace sdf;

extern "C" int sdf_narrow_band_backward(const sdf_features *feats, const sdf_grid *grids, const float *band_w,
                                        int32_t n, const float *const *grad_dist, const int32_t *const *winner,
                                        float *const *grad_vertices, uint32_t flags, void *stream) {
    if (!feats || !grids || n < 1 || !grad_dist || !grad_vertices) return SDF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    for (int p = 0; p < n; p++) {
        sdf_features_s *f = feats[p];
        const sdf_grid &gr = grids[p];
        if (!f || !grad_dist[p] || !grad_vertices[p]) return SDF_ERR_INVALID_ARG;
        if (gr.nx < 1 || gr.ny < 1 || gr.nz < 1 || !(gr.h > 0.f)) return SDF_ERR_INVALID_ARG;
        const int64_t npts = (int64_t)gr.nx * gr.ny * gr.nz;
        const int32_t *win = winner ? winner[p] : nullptr;
        if (!win) {  // recompute the winners with a forward pass into library scratch
            if (!band_w) return SDF_ERR_INVALID_ARG;
            SDF_TRY(f->fwd_winner.reserve((size_t)npts * (sizeof(int32_t) + sizeof(float))));
            int32_t *w = f->fwd_winner.as<int32_t>();
            float *dscratch = reinterpret_cast<float *>(w + npts);
            float *const dl[1] = {dscratch};
            int32_t *const wl[1] = {w};
            sdf_features fl[1] = {f};
            int st = narrow_band_all(fl, &gr, band_w + p, 1, dl, wl, flags, s);
            if (st) return st;
            win = w;
        }
        AdjArgs a;
        a.T = (int)f->T; a.E = (int)f->E; a.V = (int)f->V;
        a.nx = gr.nx; a.ny = gr.ny; a.nz = gr.nz;
        a.ox = gr.origin[0]; a.oy = gr.origin[1]; a.oz = gr.origin[2]; a.h = gr.h;
        a.grad = grad_dist[p];
        a.winner = win;
        a.gv = grad_vertices[p];
        a.face_rec = f->face_rec; a.edge_rec = f->edge_rec; a.vert_rec = f->vert_rec;
        a.face_vid = f->face_vid; a.edge_vf = f->edge_vf; a.vpos = f->vpos;
        int64_t blocks = (npts + 255) / 256;
        if (blocks > 152 * 16) blocks = 152 * 16;
        const bool timing = (flags & SDF_FLAG_TIMING) != 0;
        if (timing) {
            if (ensure_events(f)) return SDF_ERR_CUDA;
            SDF_TRY(cudaEventRecord(f->ev[4], s));
        }
        k_adjoint<<<(unsigned)blocks, 256, 0, s>>>(a);
        SDF_LAUNCHED(1);
        SDF_TRY(cudaGetLastError());
        if (timing) {
            SDF_TRY(cudaEventRecord(f->ev[5], s));
            SDF_TRY(cudaEventSynchronize(f->ev[5]));
            float ms = 0.f;
            SDF_TRY(cudaEventElapsedTime(&ms, f->ev[4], f->ev[5]));
            f->t_ms[3] += ms;
            f->t_calls[3]++;
        }
    }
    return SDF_OK;
}
