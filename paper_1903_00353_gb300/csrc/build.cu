// Mesh-connectivity stage and feature records (Sections 7 and 8 of the paper).
//
//   soup --(bounds, weld keys)--> radix sort --> vertex runs --> welded vertices + CSR of corners
//        --(smallest vertex id)--> spatial face order --> edge twins found in the vertex fans
//        --> face / edge / vertex records (normals, side planes, pseudonormals, classes)
//
// Welding (Section 7.2).  The paper sorts 30-bit Morton codes and then groups identical
// vertices serially inside each equal-code run.  Here the sort key is 40 bits (five 8-bit radix
// passes): the 30-bit Morton code of the quantised position (over the soup's bounding box,
// Section 7.1) in the high bits and a 10-bit hash of the exact coordinate bits in the low bits, so
// equal vertices always share a key and distinct vertices rarely do.  Runs of equal keys holding different coordinates (hash
// collisions, or distinct vertices in one Morton cell) are re-ordered by exact coordinates by one
// thread per such run, the only serial step left of the paper's fix-up.
//
// Edge pairing (Section 7.1): the twin of the directed edge a->b is the corner of b whose next
// vertex is a, found in b's fan of the vertex CSR; a->b must occur once around a and b->a once
// around b, else the surface is not a closed oriented 2-manifold.  No second sort is needed.
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "sdf_internal.cuh"

namespace sdf {
namespace {

constexpr int BT = 256;

__device__ __forceinline__ void atomic_min_f(float *a, float v) {
    if (v >= 0.f) atomicMin(reinterpret_cast<int *>(a), __float_as_int(v));
    else atomicMax(reinterpret_cast<unsigned *>(a), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_f(float *a, float v) {
    if (v >= 0.f) atomicMax(reinterpret_cast<int *>(a), __float_as_int(v));
    else atomicMin(reinterpret_cast<unsigned *>(a), __float_as_uint(v));
}
__device__ __forceinline__ float canon_zero(float x) { return x == 0.f ? 0.f : x; }  // -0 -> +0

// ----------------------------------------------------------------------------- soup bounds + finiteness
__global__ void k_soup_bounds(const float *soup, int64_t n3, float *bb, DevCounters *ctr) {
    dep_wait();
    dep_next();
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n3; s += (int64_t)gridDim.x * blockDim.x) {
        for (int j = 0; j < 3; j++) {
            float x = soup[3 * s + j];
            if (!isfinite(x)) bad = true;
            else { lo[j] = fminf(lo[j], x); hi[j] = fmaxf(hi[j], x); }
        }
    }
    if (bad) atomicOr(&ctr->status, ST_NONFINITE);
    // warp, then block reduction; six atomics per block (same-address atomics serialise in L2)
    for (int j = 0; j < 3; j++) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[j] = fminf(lo[j], __shfl_xor_sync(0xffffffffu, lo[j], o));
            hi[j] = fmaxf(hi[j], __shfl_xor_sync(0xffffffffu, hi[j], o));
        }
    }
    __shared__ float s_lo[3][32], s_hi[3][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0)
        for (int j = 0; j < 3; j++) {
            s_lo[j][warp] = lo[j];
            s_hi[j][warp] = hi[j];
        }
    __syncthreads();
    if (warp == 0) {
        for (int j = 0; j < 3; j++) {
            float l = lane < nw ? s_lo[j][lane] : INFINITY, h = lane < nw ? s_hi[j][lane] : -INFINITY;
            for (int o = 16; o > 0; o >>= 1) {
                l = fminf(l, __shfl_xor_sync(0xffffffffu, l, o));
                h = fmaxf(h, __shfl_xor_sync(0xffffffffu, h, o));
            }
            if (lane == 0 && l <= h) {
                atomic_min_f(bb + j, l);
                atomic_max_f(bb + 3 + j, h);
            }
        }
    }
}

__device__ __forceinline__ uint32_t expand10(uint32_t x) {  // spread 10 bits to every third bit
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {  // SplitMix64 finaliser
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void k_weld_keys(const float *soup, int64_t n3, const float *bb, uint64_t *keys, uint32_t *vals) {
    dep_wait();
    dep_next();
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n3) return;
    float x = canon_zero(soup[3 * s]), y = canon_zero(soup[3 * s + 1]), z = canon_zero(soup[3 * s + 2]);
    uint32_t q[3];
    float c[3] = {x, y, z};
    for (int j = 0; j < 3; j++) {
        float ext = bb[3 + j] - bb[j];
        float t = ext > 0.f ? (c[j] - bb[j]) / ext * 1024.f : 0.f;
        int qi = (int)t;
        q[j] = (uint32_t)min(max(qi, 0), 1023);
    }
    uint64_t morton = (uint64_t)(expand10(q[0]) | (expand10(q[1]) << 1) | (expand10(q[2]) << 2));
    uint64_t hsh = mix64(((uint64_t)__float_as_uint(x) << 32 | __float_as_uint(y)) ^ mix64(__float_as_uint(z) + 0x9e3779b97f4a7c15ull));
    keys[s] = (morton << 10) | (hsh & ((1ull << 10) - 1));  // 40-bit key: 5 radix passes
    vals[s] = (uint32_t)s;
}

__device__ __forceinline__ bool same_xyz(const float *soup, uint32_t a, uint32_t b) {
    return canon_zero(soup[3 * (int64_t)a]) == canon_zero(soup[3 * (int64_t)b]) &&
           canon_zero(soup[3 * (int64_t)a + 1]) == canon_zero(soup[3 * (int64_t)b + 1]) &&
           canon_zero(soup[3 * (int64_t)a + 2]) == canon_zero(soup[3 * (int64_t)b + 2]);
}
__device__ __forceinline__ bool less_xyz(const float *soup, uint32_t a, uint32_t b) {
    for (int j = 0; j < 3; j++) {
        uint32_t ua = __float_as_uint(canon_zero(soup[3 * (int64_t)a + j]));
        uint32_t ub = __float_as_uint(canon_zero(soup[3 * (int64_t)b + j]));
        if (ua != ub) return ua < ub;
    }
    return a < b;
}

// One thread per run of equal keys.  A run that mixes distinct coordinates (a hash collision, or
// distinct vertices in one Morton cell, as in a dense cluster of small triangles) is re-ordered by
// (coordinate bits, soup index) so that equal vertices become contiguous: runs of up to
// WELD_SHORT entries by the thread itself (insertion sort), longer ones are listed for
// k_weld_sort_runs, one block per run.
constexpr int WELD_SHORT = 32, WELD_BLOCK_MAX = 2048;
__global__ void k_weld_fix(const uint64_t *keys, uint32_t *vals, const float *soup, int64_t n, int2 *long_runs,
                           int64_t long_cap, unsigned *n_long) {
    dep_wait();
    dep_next();
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || (i > 0 && keys[i] == keys[i - 1])) return;
    int64_t e = i + 1;
    bool mixed = false;
    while (e < n && keys[e] == keys[i]) {
        mixed |= !same_xyz(soup, vals[e], vals[i]);
        e++;
    }
    if (!mixed) return;
    if (e - i > WELD_SHORT && e - i <= WELD_BLOCK_MAX) {
        const unsigned slot = atomicAdd(n_long, 1u);
        if ((int64_t)slot < long_cap) {
            long_runs[slot] = make_int2((int)i, (int)(e - i));
            return;
        }
    }
    for (int64_t a = i + 1; a < e; a++) {  // short runs (and runs beyond the block sort's size)
        uint32_t v = vals[a];
        int64_t b = a - 1;
        while (b >= i && less_xyz(soup, v, vals[b])) { vals[b + 1] = vals[b]; b--; }
        vals[b + 1] = v;
    }
}

// The listed long mixed runs, one block per run (grid-stride over the device-side count): the
// run's (x, y, z bits, soup index) records are sorted in shared memory by a bitonic network over
// the next power of two (padding sorts last), then written back.  Any total order of the
// coordinate bits makes equal vertices contiguous; -0 is read as +0.
__global__ void __launch_bounds__(256) k_weld_sort_runs(const int2 *long_runs, const unsigned *n_long, int64_t long_cap,
                                                        uint32_t *vals, const float *soup) {
    dep_wait();
    dep_next();
    __shared__ uint4 rec[WELD_BLOCK_MAX];
    const int64_t nl = min((int64_t)*n_long, long_cap);
    for (int64_t r = blockIdx.x; r < nl; r += gridDim.x) {
        const int2 run = long_runs[r];
        int m = 1;
        while (m < run.y) m <<= 1;
        for (int t = threadIdx.x; t < m; t += blockDim.x) {
            if (t < run.y) {
                const uint32_t v = vals[run.x + t];
                rec[t] = make_uint4(__float_as_uint(canon_zero(soup[3 * (int64_t)v])),
                                    __float_as_uint(canon_zero(soup[3 * (int64_t)v + 1])),
                                    __float_as_uint(canon_zero(soup[3 * (int64_t)v + 2])), v);
            } else {
                rec[t] = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
            }
        }
        __syncthreads();
        for (int k = 2; k <= m; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int t = threadIdx.x; t < m; t += blockDim.x) {
                    const int u = t ^ j;
                    if (u > t) {
                        const uint4 a = rec[t], b = rec[u];
                        const bool gt = a.x != b.x ? a.x > b.x : (a.y != b.y ? a.y > b.y : (a.z != b.z ? a.z > b.z : a.w > b.w));
                        if (gt == ((t & k) == 0)) {  // ascending where t & k == 0
                            rec[t] = b;
                            rec[u] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int t = threadIdx.x; t < run.y; t += blockDim.x) vals[run.x + t] = rec[t].w;
        __syncthreads();
    }
}

__global__ void k_weld_heads(const uint64_t *keys, const uint32_t *vals, const float *soup, int64_t n,
                             uint32_t *head) {
    dep_wait();
    dep_next();
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    head[i] = (i == 0 || keys[i] != keys[i - 1] || !same_xyz(soup, vals[i], vals[i - 1])) ? 1u : 0u;
}

// head[] holds the exclusive scan of the run heads; vid = that + is_head - 1
__global__ void k_weld_scatter(const uint32_t *vals, const uint32_t *hscan, const uint64_t *keys, const float *soup,
                               int64_t n, int32_t *soup_vid, int32_t *vert_start, int32_t *vert_corner,
                               float *vpos, float4 *grad4) {
    dep_wait();
    dep_next();
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool is_head = hscan[i + 1] != hscan[i];
    int32_t vid = (int32_t)hscan[i + 1] - 1;
    uint32_t s = vals[i];
    soup_vid[s] = vid;
    vert_corner[i] = (int32_t)s;
    if (is_head) {
        vert_start[vid] = (int32_t)i;
        for (int j = 0; j < 3; j++) vpos[3 * vid + j] = canon_zero(soup[3 * (int64_t)s + j]);
        grad4[vid] = make_float4(0.f, 0.f, 0.f, 0.f);  // the adjoints' sums start cleared
    }
    if (i == n - 1) vert_start[vid + 1] = (int32_t)n;
}

// ----------------------------------------------------------------------------- spatial face order
// key of a face: its smallest welded vertex id (vertex ids follow the Morton order of the weld),
// so faces that are close in space get close ids and their records share cache lines
__global__ void k_face_keys(const int32_t *soup_vid, int64_t T, uint64_t *keys, uint32_t *vals) {
    dep_wait();
    dep_next();
    int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= T) return;
    int32_t a = soup_vid[3 * f], b = soup_vid[3 * f + 1], c = soup_vid[3 * f + 2];
    keys[f] = (uint64_t)(uint32_t)min(a, min(b, c));
    vals[f] = (uint32_t)f;
}

// face_soup[f] = soup triangle of library face f; face_vid in library order; inv: soup -> library
__global__ void k_face_perm(const uint32_t *order, const int32_t *soup_vid, int64_t T, int32_t *face_soup,
                            int32_t *face_vid, uint32_t *inv) {
    dep_wait();
    dep_next();
    int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= T) return;
    uint32_t sf = order[f];
    face_soup[f] = (int32_t)sf;
    inv[sf] = (uint32_t)f;
    for (int k = 0; k < 3; k++) face_vid[3 * f + k] = soup_vid[3 * (int64_t)sf + k];
}

__global__ void k_corner_remap(int32_t *vert_corner, const uint32_t *inv, int64_t n) {
    dep_wait();
    dep_next();
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t c = vert_corner[i];
    int32_t sf = c / 3;
    vert_corner[i] = 3 * (int32_t)inv[sf] + (c - 3 * sf);
}

// ----------------------------------------------------------------------------- edge pairing
// Directed edge h (corner k of face f, from vertex a to the next corner's vertex b) must meet
// exactly one directed edge b -> a, found among the corners of b, and a -> b must occur once
// among the corners of a (closed, consistently oriented 2-manifold).  Edges get ids in the
// order of their smaller end point's corners, which keeps them spatially ordered too.
__global__ void k_pair_fans(const int32_t *vert_start, const int32_t *vert_corner, const int32_t *face_vid, int64_t n,
                            int32_t *twin, uint32_t *canon, DevCounters *ctr) {
    dep_wait();
    dep_next();
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t h = vert_corner[i];
    const int32_t f = h / 3, k = h - 3 * f;
    const int32_t a = face_vid[h], b = face_vid[3 * f + (k + 1) % 3];
    if (a == b) {
        atomicOr(&ctr->status, ST_DEGENERATE);
        canon[i] = 0;
        return;
    }
    int32_t found = -1, nfound = 0;
    for (int32_t q = vert_start[b]; q < vert_start[b + 1]; q++) {
        const int32_t c = vert_corner[q];
        const int32_t g = c / 3, kk = c - 3 * g;
        if (face_vid[3 * g + (kk + 1) % 3] == a) {
            found = c;
            nfound++;
        }
    }
    int32_t same = 0;
    for (int32_t q = vert_start[a]; q < vert_start[a + 1]; q++) {
        const int32_t c = vert_corner[q];
        const int32_t g = c / 3, kk = c - 3 * g;
        same += face_vid[3 * g + (kk + 1) % 3] == b;
    }
    if (nfound != 1 || same != 1) {
        atomicOr(&ctr->status, ST_NONMANIFOLD);
        canon[i] = 0;
        return;
    }
    twin[h] = found;
    canon[i] = a < b ? 1u : 0u;
}

// canonical directed edges (va < vb) create the edge records; eid = exclusive scan of canon
__global__ void k_edge_emit(const int32_t *vert_corner, const int32_t *face_vid, const int32_t *twin,
                            const uint32_t *canon, const uint32_t *eid, int64_t n, int4 *edge_vf,
                            int32_t *face_edge) {
    dep_wait();
    dep_next();
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || !canon[i]) return;
    const int32_t h = vert_corner[i];
    const int32_t f = h / 3, k = h - 3 * f;
    const int32_t e = (int32_t)eid[i];
    const int32_t t = twin[h];
    edge_vf[e] = make_int4(face_vid[h], face_vid[3 * f + (k + 1) % 3], f, t / 3);
    face_edge[h] = e;
    face_edge[t] = e;
}

// ----------------------------------------------------------------------------- records (geometry)
// FP64 check of a (filtered) zero-area predicate
__device__ __forceinline__ float4 plane_through(float3 m, float3 p) {  // (m, -m.p): value m.x + w
    return make_float4(m.x, m.y, m.z, -dot3(m, p));
}
__device__ __forceinline__ float3 normalized(float3 v) {
    float r = rsqrtf(dot3(v, v));
    return r * v;
}

// Block-wide reductions of one value per thread into a device counter, one atomic per block (the
// records kernels loop over their items with a fixed grid, so a build makes a few thousand
// atomics on these few words instead of one per warp: same-address atomics serialise in L2).
// Every thread of the block must call them.
__device__ __forceinline__ float block_reduce_max(float v) {  // v >= 0; the result is in thread 0
    __shared__ float part[BT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();  // the array may still be read by a previous reduction
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < BT / 32; w++) v = fmaxf(v, part[w]);
    return v;
}
// the largest value (v >= 0) into a word holding FP32 bits, skipping the atomic when it is no larger
__device__ __forceinline__ void block_max_into(unsigned *word, float v) {
    v = block_reduce_max(v);
    if (threadIdx.x == 0 && v > 0.f && __float_as_uint(v) > *(volatile unsigned *)word)
        atomicMax(word, __float_as_uint(v));
}
__device__ __forceinline__ void block_count_into(unsigned long long *word, unsigned c) {
    __shared__ unsigned part[BT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < BT / 32; w++) c += part[w];
        if (c) atomicAdd(word, (unsigned long long)c);
    }
}

// Sums of K values over a block of BT threads, added to K counters with one atomic each (FP32
// within the block, FP64 across blocks).
template <int K>
__device__ __forceinline__ void block_sums_into(double *words, float (&v)[K]) {
    __shared__ float part[BT / 32][K];
#pragma unroll
    for (int k = 0; k < K; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < K; k++) part[threadIdx.x >> 5][k] = v[k];
    __syncthreads();
    if (threadIdx.x < K) {
        double t = 0.0;
        for (int w = 0; w < BT / 32; w++) t += part[w][threadIdx.x];
        if (t != 0.0) atomicAdd(&words[threadIdx.x], t);
    }
}

// Face records, and the precision terms and box moments of the faces (a fixed grid looping over
// the faces; the block reductions at the end take every thread).  The unit normal and the plane
// offset -n.a are computed in FP64 from the FP32 corners (their differences are exact in FP64)
// and rounded once, so the stored normal is within about u = 2^-24 of the exact normal of the
// corners however thin the triangle.  The side planes n x (edge) are formed in FP32 from it: the
// edge difference, the cross product and the normalisation add at most 8 u to the direction, so
// a side-plane test at a point p of the prism errs by at most 8 u |p - a| <= 8 u (D + W) beyond
// the rounding of its evaluation (D the face's longest edge, W the band cutoff).  The edge wedge
// planes (k_edge_records) have the same bound with the edge length.  The records kernels keep the
// maxima of tau_a = 10 u D and tau_b = 10 u (with margin) and of the coordinate magnitude; the
// narrow band adds tau_a + tau_b W to its FP32 error bound (the windows in band.cu).
__global__ void __launch_bounds__(BT) k_face_records(const int32_t *face_vid, const float *vpos, int64_t T,
                                                     float4 *face_rec, float4 *face_box, DevCounters *ctr) {
    dep_wait();
    dep_next();
    float m_abs = 0.f, tau_a = 0.f;
    float mom[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    bool degenerate = false;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < T; f += (int64_t)gridDim.x * blockDim.x) {
        float3 a = load_vpos(vpos, face_vid[3 * f]), b = load_vpos(vpos, face_vid[3 * f + 1]),
               c = load_vpos(vpos, face_vid[3 * f + 2]);
        const double3 A = d3(a), E1 = d3(b) - A, E2 = d3(c) - A;
        const double3 CR = dcross3(E1, E2);
        double len = sqrt(ddot3(CR, CR));
        if (!(len > 1e-14 * (ddot3(E1, E1) + ddot3(E2, E2)))) {  // zero area (Section 4)
            degenerate = true;
            len = fmax(len, 1e-300);
        }
        const double3 N = (1.0 / len) * CR;
        const float3 n = make_float3((float)N.x, (float)N.y, (float)N.z);
        // plane of the face, and the three side planes with inward normals n x (edge) (Section 8.1)
        face_rec[4 * f + 0] = make_float4(n.x, n.y, n.z, (float)-ddot3(N, A));
        face_rec[4 * f + 1] = plane_through(normalized(cross3(n, b - a)), a);
        face_rec[4 * f + 2] = plane_through(normalized(cross3(n, c - b)), b);
        face_rec[4 * f + 3] = plane_through(normalized(cross3(n, a - c)), c);
        const float3 lo = make_float3(fminf(a.x, fminf(b.x, c.x)), fminf(a.y, fminf(b.y, c.y)), fminf(a.z, fminf(b.z, c.z)));
        const float3 hi = make_float3(fmaxf(a.x, fmaxf(b.x, c.x)), fmaxf(a.y, fmaxf(b.y, c.y)), fmaxf(a.z, fmaxf(b.z, c.z)));
        face_box[2 * f + 0] = make_float4(lo.x, lo.y, lo.z, 0.f);
        face_box[2 * f + 1] = make_float4(hi.x, hi.y, hi.z, 0.f);
        m_abs = fmaxf(m_abs, fmaxf(fmaxf(fmaxf(fabsf(lo.x), fabsf(hi.x)), fmaxf(fabsf(lo.y), fabsf(hi.y))),
                                   fmaxf(fabsf(lo.z), fabsf(hi.z))));
        const float3 e3 = c - b;
        const float diam = sqrtf(fmaxf(fmaxf(dot3(b - a, b - a), dot3(c - a, c - a)), dot3(e3, e3)));
        tau_a = fmaxf(tau_a, 10.f * U32 * diam * 1.001f);
        const float bx = hi.x - lo.x, by = hi.y - lo.y, bz = hi.z - lo.z;
        mom[0] += bx; mom[1] += by; mom[2] += bz;
        mom[3] += bx * by; mom[4] += bx * bz; mom[5] += by * bz; mom[6] += bx * by * bz;
    }
    if (degenerate) atomicOr(&ctr->status, ST_DEGENERATE);
    block_max_into(&ctr->prec[PREC_MESH_M], m_abs);
    block_max_into(&ctr->prec[PREC_TAU_A], tau_a);
    block_max_into(&ctr->prec[PREC_TAU_B], T > 0 ? 10.f * U32 : 0.f);
    block_sums_into<7>(ctr->box_mom, mom);
}

__device__ double3 face_normal_fp64(const int32_t *face_vid, const float *vpos, int f) {
    double3 a = d3(load_vpos(vpos, face_vid[3 * f])), b = d3(load_vpos(vpos, face_vid[3 * f + 1])),
            c = d3(load_vpos(vpos, face_vid[3 * f + 2]));
    double3 cr = dcross3(b - a, c - a);
    return (1.0 / sqrt(ddot3(cr, cr))) * cr;
}

// edge wedge (Section 8.2): unit direction t (va -> vb, the direction in face f1), the planes
// (p - a).m1 <= 0 and (p - a).m2 <= 0 with m1 = n1 x t into face 1 and m2 = n2 x (-t) into face 2,
// and the edge pseudonormal n1 + n2.  Class from d = (ab x n1) . n2 (FP32, FP64 when near zero).
__global__ void __launch_bounds__(BT) k_edge_records(const int4 *edge_vf, const int32_t *face_vid, const float *vpos,
                                                     const float4 *face_rec, int64_t E, float4 *edge_rec,
                                                     int8_t *edge_class, DevCounters *ctr) {
    dep_wait();
    dep_next();
    unsigned ncv = 0, ncc = 0;  // class counts of this thread's edges
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const int4 q = edge_vf[e];
        if (q.x < 0 || q.y < 0 || q.z < 0 || q.w < 0) {  // not paired (a broken mesh, rejected by the build)
            edge_class[e] = CLS_FLAT;
            continue;
        }
        const float3 a = load_vpos(vpos, q.x), b = load_vpos(vpos, q.y);
        const float3 n1 = f3(face_rec[4 * q.z]), n2 = f3(face_rec[4 * q.w]);
        const float3 ab = b - a;
        const float L = sqrtf(dot3(ab, ab));
        const float3 t = (1.f / L) * ab;
        const float3 m1 = normalized(cross3(n1, t));
        const float3 m2 = normalized(cross3(n2, make_float3(-t.x, -t.y, -t.z)));
        const float3 np = n1 + n2;
        edge_rec[5 * e + 0] = make_float4(a.x, a.y, a.z, L);
        edge_rec[5 * e + 1] = make_float4(t.x, t.y, t.z, dot3(t, a));
        edge_rec[5 * e + 2] = make_float4(-m1.x, -m1.y, -m1.z, dot3(m1, a));
        edge_rec[5 * e + 3] = make_float4(-m2.x, -m2.y, -m2.z, dot3(m2, a));
        edge_rec[5 * e + 4] = make_float4(np.x, np.y, np.z, sqrtf(dot3(np, np)));  // (n1 + n2, |n1 + n2|)
        const float d = dot3(cross3(t, n1), n2);
        int8_t cls;
        if (fabsf(d) > 2e-6f) {
            cls = d > 0.f ? CLS_CONVEX : CLS_CONCAVE;
        } else {  // filtered predicate: decide near-flat edges in FP64
            const double3 A = d3(a), B = d3(b);
            const double3 N1 = face_normal_fp64(face_vid, vpos, q.z), N2 = face_normal_fp64(face_vid, vpos, q.w);
            const double3 AB = B - A;
            const double dd = ddot3(dcross3(AB, N1), N2);
            const double tol = 1e-12 * sqrt(ddot3(AB, AB));
            cls = dd > tol ? CLS_CONVEX : (dd < -tol ? CLS_CONCAVE : CLS_FLAT);
        }
        edge_class[e] = cls;
        ncv += cls == CLS_CONVEX;
        ncc += cls == CLS_CONCAVE;
    }
    block_count_into(&ctr->cls[6], ncv);
    block_count_into(&ctr->cls[7], ncc);
}

__device__ __forceinline__ float corner_angle(float3 e1, float3 e2) {
    float3 cr = cross3(e1, e2);
    return atan2f(sqrtf(dot3(cr, cr)), dot3(e1, e2));
}

constexpr int VL = 8;      // lanes per vertex in k_vertex_records
constexpr int VMAXS = 24;  // corners of a fan staged in shared memory (and cone-searched)

__device__ __forceinline__ float gsum8(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 4, VL);
    v += __shfl_xor_sync(0xffffffffu, v, 2, VL);
    v += __shfl_xor_sync(0xffffffffu, v, 1, VL);
    return v;
}
__device__ __forceinline__ float gmin8(float v) {
    v = fminf(v, __shfl_xor_sync(0xffffffffu, v, 4, VL));
    v = fminf(v, __shfl_xor_sync(0xffffffffu, v, 2, VL));
    v = fminf(v, __shfl_xor_sync(0xffffffffu, v, 1, VL));
    return v;
}
__device__ __forceinline__ bool gor8(bool b) {
    int v = b;
    v |= __shfl_xor_sync(0xffffffffu, v, 4, VL);
    v |= __shfl_xor_sync(0xffffffffu, v, 2, VL);
    v |= __shfl_xor_sync(0xffffffffu, v, 1, VL);
    return v != 0;
}

// vertex records (Section 8.3), 8 lanes per vertex, each lane taking every 8th corner of the fan:
// N_alpha = sum alpha_i n_i (Eq. 8); one plane (p - v).e_j <= 0 per incident edge (the region where
// no incident edge leads closer than v); the class from the signs of (v_n - v).N_alpha over the
// neighbours (FP32 when clear, FP64 otherwise); and a cone bounding the vertex region.
__global__ void __launch_bounds__(BT) k_vertex_records(const int32_t *vert_start, const int32_t *vert_corner,
                                                       const int32_t *face_vid, const float *vpos,
                                                       const float4 *face_rec, int64_t V, float4 *vert_rec,
                                                       float4 *vert_plane, int8_t *vert_class, DevCounters *ctr) {
    dep_wait();
    dep_next();
    // the planes and face normals of each group's fan, staged for the classification and the cone
    // search (fans of more than VMAXS corners read them from global memory and skip the search)
    __shared__ float4 s_plane[BT / VL][VMAXS];
    __shared__ float3 s_nf[BT / VL][VMAXS];
    const int grp = (int)(threadIdx.x / VL);
    float tv_max = 0.f;
    unsigned ncls[4] = {0, 0, 0, 0};  // convex, concave, flat and saddle vertices of this thread
    // a warp-uniform loop (the groups' shuffles take the whole warp): item gl is lane gl % VL of
    // vertex gl / VL
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31u); g0 < V * VL; g0 += stride) {
        const int64_t gl = g0 + (threadIdx.x & 31);
        const int64_t v = gl / VL;
        const int sub = (int)(gl % VL);
        const bool valid = v < V;
        const int s0 = valid ? vert_start[v] : 0, s1 = valid ? vert_start[v + 1] : 0;
        const float3 p = valid ? load_vpos(vpos, (int)v) : make_float3(0.f, 0.f, 0.f);
        // pass 1: pseudonormal and region planes
        float3 N = make_float3(0.f, 0.f, 0.f);
        float asum = 0.f;
        const bool staged = s1 - s0 <= VMAXS;  // the fan's planes and normals fit the group's slots
        for (int i = s0 + sub; i < s1; i += VL) {
            const int c = vert_corner[i];
            const int f = c / 3, k = c - 3 * f;
            const float3 xn = load_vpos(vpos, face_vid[3 * f + (k + 1) % 3]);
            const float3 xp = load_vpos(vpos, face_vid[3 * f + (k + 2) % 3]);
            const float3 e1 = xn - p, e2 = xp - p;
            const float alpha = corner_angle(e1, e2);
            asum += alpha;
            const float3 nf = f3(face_rec[4 * f]);
            N = N + alpha * nf;
            const float3 ej = normalized(e1);
            const float4 pl = make_float4(-ej.x, -ej.y, -ej.z, dot3(ej, p));
            vert_plane[i] = pl;
            if (staged) {
                s_plane[grp][i - s0] = pl;
                s_nf[grp][i - s0] = nf;
            }
        }
        N = make_float3(gsum8(N.x), gsum8(N.y), gsum8(N.z));
        asum = gsum8(asum);
        const float Nlen = sqrtf(dot3(N, N));
        const float3 Nu = (Nlen > 0.f ? 1.f / Nlen : 0.f) * N;
        // Direction error of the unit pseudonormal: each term alpha_i n_i errs by at most
        // alpha_i 10 u (the stored face normal within u, the angle's rounding) and the sum of deg terms
        // adds deg u sum(alpha); the normalisation at most doubles the relative error.
        // tau_v = 2 sum(alpha) (deg + 10) u / |N_alpha|, kept as a maximum (per unit distance: the sign
        // predicate N^.(p - v) errs by tau_v |p - v| from it).
        {
            float tv = 0.f;
            if (valid && sub == 0 && s1 > s0)
                tv = Nlen > 0.f ? fminf(2.f * asum * (float)(s1 - s0 + 10) * U32 / Nlen * 1.001f, 1.f) : 1.f;
            tv_max = fmaxf(tv_max, tv);
        }
        __syncwarp();  // the group's planes are written before they are read back
        // pass 2: classification (FP32 with an error margin), convexity and the normal spread
        bool below = false, above = false, unsure = false, cvx = true, ccv = true;
        float cmin = 1.f;
        for (int i = s0 + sub; i < s1; i += VL) {
            // unit direction e_j to the next neighbour (the plane holds -e_j): the sign of
            // (v_n - v).N_alpha is that of e_j.N_alpha, tested against 2e-6 |N_alpha|
            const float3 ej = -1.f * (staged ? f3(s_plane[grp][i - s0]) : f3(vert_plane[i]));
            const float d = dot3(ej, N);
            const float bound = 2e-6f * Nlen;
            if (d < -bound) below = true;
            else if (d > bound) above = true;
            else unsure = true;
            const float3 nf = staged ? s_nf[grp][i - s0] : f3(face_rec[4 * (vert_corner[i] / 3)]);
            cmin = fminf(cmin, dot3(nf, Nu));
            for (int b = 0; b < s1 - s0; b++) {  // every incident edge against this face's plane
                const float dd = -dot3(nf, staged ? f3(s_plane[grp][b]) : f3(vert_plane[s0 + b]));
                cvx = cvx && dd <= 1e-4f;
                ccv = ccv && dd >= -1e-4f;
            }
        }
        below = gor8(below);
        above = gor8(above);
        unsure = gor8(unsure);
        cvx = !gor8(!cvx);
        ccv = !gor8(!ccv);
        cmin = gmin8(cmin);
        // Bound of the vertex region {y : y.e_j <= 0}.  Locally convex (every incident edge below every
        // incident face plane): the cone spanned by the face normals; locally concave: by their
        // negatives; otherwise the extreme rays are searched among +-(e_j x e_l): the deg (deg - 1) / 2
        // plane pairs are spread over the group's 8 lanes, and each candidate ray is tested against
        // every plane without early exit, so the lanes of a group stay converged.  A cone is kept only
        // if all its rays lie within 89 degrees of +N_alpha (or of -N_alpha).  The flags and bounds
        // below are uniform over the 8 lanes of a vertex after the group reductions.
        const int deg = s1 - s0;
        const bool conv_cone = cvx && !ccv && cmin > 0.02f, conc_cone = ccv && !cvx && cmin > 0.02f;
        const bool search = valid && Nlen > 0.f && !conv_cone && !conc_cone && staged;
        bool any = false, all_pos = true, all_neg = true;
        float cpos = 1.f, cng = 1.f;
        if (search) {
            const int npairs = deg * (deg - 1) / 2;
            for (int pidx = sub; pidx < npairs; pidx += VL) {
                int a = 0, rem = pidx;  // pair pidx = (a, b), a < b, in row-major order
                while (rem >= deg - 1 - a) {
                    rem -= deg - 1 - a;
                    a++;
                }
                const int b = a + 1 + rem;
                float3 y = cross3(f3(s_plane[grp][a]), f3(s_plane[grp][b]));  // planes hold -e
                const float ly = sqrtf(dot3(y, y));
                const bool ok = ly > 1e-6f;
                y = (ok ? 1.f / ly : 0.f) * y;
                bool fp = ok, fn = ok;  // +y and -y feasible
                for (int m = 0; m < deg; m++) {
                    const float dm = dot3(y, f3(s_plane[grp][m]));
                    fp = fp && dm >= -1e-4f;
                    fn = fn && -dm >= -1e-4f;
                }
                const float cc = dot3(y, Nu);
                if (fp) {
                    any = true;
                    if (cc > 0.02f) cpos = fminf(cpos, cc); else all_pos = false;
                    if (cc < -0.02f) cng = fminf(cng, -cc); else all_neg = false;
                }
                if (fn) {
                    any = true;
                    if (-cc > 0.02f) cpos = fminf(cpos, -cc); else all_pos = false;
                    if (-cc < -0.02f) cng = fminf(cng, cc); else all_neg = false;
                }
            }
        }
        any = gor8(any);
        all_pos = !gor8(!all_pos);
        all_neg = !gor8(!all_neg);
        cpos = gmin8(cpos);
        cng = gmin8(cng);
        int8_t my_cls = 99;  // class of the vertex held by lane sub == 0
        if (valid && sub == 0) {
            if (unsure) {  // FP64 filtered predicate (rare): recompute N_alpha and the signs in FP64
                below = above = false;
                const double3 P = d3(p);
                double3 ND = make_double3(0, 0, 0);
                for (int i = s0; i < s1; i++) {
                    const int c = vert_corner[i];
                    const int f = c / 3, k = c - 3 * f;
                    const double3 e1 = d3(load_vpos(vpos, face_vid[3 * f + (k + 1) % 3])) - P;
                    const double3 e2 = d3(load_vpos(vpos, face_vid[3 * f + (k + 2) % 3])) - P;
                    const double3 cr = dcross3(e1, e2);
                    const double alpha = atan2(sqrt(ddot3(cr, cr)), ddot3(e1, e2));
                    ND = ND + alpha * face_normal_fp64(face_vid, vpos, f);
                }
                const double NL = sqrt(ddot3(ND, ND));
                for (int i = s0; i < s1; i++) {
                    const int c = vert_corner[i];
                    const int f = c / 3, k = c - 3 * f;
                    const double3 dv = d3(load_vpos(vpos, face_vid[3 * f + (k + 1) % 3])) - P;
                    const double d = ddot3(dv, ND);
                    const double tol = 1e-12 * sqrt(ddot3(dv, dv)) * NL;
                    if (d < -tol) below = true;
                    else if (d > tol) above = true;
                }
            }
            const int8_t cls = below && above ? CLS_SADDLE : (below ? CLS_CONVEX : (above ? CLS_CONCAVE : CLS_FLAT));
            vert_class[v] = cls;
            float4 cone = make_float4(0.f, 0.f, 0.f, -2.f);
            if (Nlen > 0.f) {
                if (conv_cone) cone = make_float4(Nu.x, Nu.y, Nu.z, cmin - 2e-3f);
                else if (conc_cone) cone = make_float4(-Nu.x, -Nu.y, -Nu.z, cmin - 2e-3f);
                else if (search && any && all_pos) cone = make_float4(Nu.x, Nu.y, Nu.z, cpos - 2e-3f);
                else if (search && any && all_neg) cone = make_float4(-Nu.x, -Nu.y, -Nu.z, cng - 2e-3f);
            }
            vert_rec[3 * v + 0] = make_float4(p.x, p.y, p.z, __int_as_float(s0));
            vert_rec[3 * v + 1] = make_float4(Nu.x, Nu.y, Nu.z, __int_as_float(s1 - s0));
            vert_rec[3 * v + 2] = cone;
            my_cls = cls;
        }
        ncls[0] += my_cls == CLS_CONVEX;
        ncls[1] += my_cls == CLS_CONCAVE;
        ncls[2] += my_cls == CLS_FLAT;
        ncls[3] += my_cls == CLS_SADDLE;
        __syncwarp();  // the group's staged fan is read to the end before the next one is written
    }
    block_max_into(&ctr->prec[PREC_TAU_V], tv_max);
    for (int c = 0; c < 4; c++) block_count_into(&ctr->cls[2 + c], ncls[c]);
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + BT - 1) / BT); }

// the build's small state: counters and scan state cleared, the bounding box at (+inf, -inf)
__global__ void k_build_init(unsigned *ctr, int64_t ctr_words, float *bb, unsigned *n_long, unsigned *scan,
                             int64_t scan_words) {
    dep_wait();
    dep_next();
    for (int64_t i = threadIdx.x; i < ctr_words; i += blockDim.x) ctr[i] = 0u;
    for (int64_t i = threadIdx.x; i < scan_words; i += blockDim.x) scan[i] = 0u;
    if (threadIdx.x < 6) bb[threadIdx.x] = threadIdx.x < 3 ? INFINITY : -INFINITY;
    if (threadIdx.x == 0) *n_long = 0u;
}

// grid of a records kernel over n threads' worth of items: the blocks resident on the device at
// once (a single wave of the grid-stride loop), fewer when the items need fewer
template <class K> unsigned rec_grid(K kernel, int64_t n) {
    static int resident = 0;  // per kernel (one instance of this function per kernel type)
    if (!resident) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, BT, 0);
        resident = std::max(1, per_sm) * std::max(1, sms);
    }
    return (unsigned)std::min<int64_t>(nblk(n), resident);
}

}  // namespace

int build_records(sdf_features_s *f, cudaStream_t s) {
    if (f->T > 0) {
        SDF_TRY(launch_dep(k_face_records, dim3(rec_grid(k_face_records, f->T)), dim3(BT), 0, s, f->face_vid, f->vpos,
                           f->T, f->face_rec, f->face_box, f->ctr));
        SDF_TRY(launch_dep(k_edge_records, dim3(rec_grid(k_edge_records, f->E)), dim3(BT), 0, s, f->edge_vf, f->face_vid,
                           f->vpos, f->face_rec, f->E, f->edge_rec, f->edge_class, f->ctr));
        SDF_TRY(launch_dep(k_vertex_records, dim3(rec_grid(k_vertex_records, f->V * VL)), dim3(BT), 0, s, f->vert_start,
                           f->vert_corner, f->face_vid, f->vpos, f->face_rec, f->V, f->vert_rec, f->vert_plane,
                           f->vert_class, f->ctr));
    }
    SDF_TRY(cudaGetLastError());
    return SDF_OK;
}

}  // namespace sdf

using namespace sdf;

static int status_to_code(unsigned st) {
    if (st & ST_TIMEOUT) return SDF_ERR_TIMEOUT;
    if (st & ST_NONFINITE) return SDF_ERR_NONFINITE;
    if (st & ST_DEGENERATE) return SDF_ERR_DEGENERATE;
    if (st & ST_NONMANIFOLD) return SDF_ERR_NONMANIFOLD;
    return SDF_OK;
}

// Device blocks kept for the next build on the device: a destroyed handle's array block and
// counters, and a finished build's scratch (at most four per device, each taken only by a request
// of at least half its size).  A loop that builds a handle per step (a fitting or benchmark loop)
// then takes no memory from the pool: its allocations of the handle block took 0.08 ms every few
// builds of a 200 k-triangle mesh and once 2.3 ms, when the pool rearranged its cached blocks.
// Only idle blocks are kept (after the device synchronisation of a destroy, or after the build's
// own final synchronisation), so a later build may take one on any stream.
namespace {
struct KeptBlock {
    int dev;
    void *p;
    size_t bytes;
};
constexpr int KEEP_PER_DEVICE = 4;
std::mutex g_keep_mu;
std::vector<KeptBlock> g_kept;

cudaError_t take_block(size_t need, void **p, size_t *bytes, cudaStream_t s) {
    int dev = -1;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        std::lock_guard<std::mutex> lk(g_keep_mu);
        int best = -1;
        for (int i = 0; i < (int)g_kept.size(); i++) {
            const KeptBlock &k = g_kept[i];
            if (k.dev == dev && k.bytes >= need && k.bytes <= 2 * need + (size_t(1) << 20) &&
                (best < 0 || k.bytes < g_kept[best].bytes))
                best = i;
        }
        if (best >= 0) {
            *p = g_kept[best].p;
            *bytes = g_kept[best].bytes;
            g_kept.erase(g_kept.begin() + best);
            return cudaSuccess;
        }
    }
    *bytes = need;
    return pool_alloc(p, need, s);
}

void keep_block(void *p, size_t bytes, cudaStream_t s) {
    if (!p) return;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        pool_free(p, s);
        return;
    }
    void *evict = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_keep_mu);
        int same = 0, oldest = -1;
        for (int i = 0; i < (int)g_kept.size(); i++)
            if (g_kept[i].dev == dev) {
                if (oldest < 0) oldest = i;
                same++;
            }
        if (same >= KEEP_PER_DEVICE) {
            evict = g_kept[oldest].p;
            g_kept.erase(g_kept.begin() + oldest);
        }
        g_kept.push_back({dev, p, bytes});
    }
    if (evict) pool_free(evict, s);
}
}  // namespace

// frees on the legacy default stream, after the caller's work on the handle has completed
static void free_handle(sdf_features_s *f) {
    if (!f) return;
    // on the handle's own device (the caller's current device may be another one), restored after
    int cur = -1;
    const bool other = f->dev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != f->dev &&
                       cudaSetDevice(f->dev) == cudaSuccess;
    cudaDeviceSynchronize();  // no work may still use the handle's memory
    cudaStream_t s0 = 0;
    keep_block(f->block, f->block_bytes, s0);  // every array of the handle (kept for the next build)
    keep_block(f->ctr, f->ctr_bytes, s0);
    sdf::plan_park(f->plan, s0);
    f->plan = nullptr;
    f->fwd_winner.release(s0);
    for (cudaEvent_t e : f->ev)
        if (e) cudaEventDestroy(e);
    delete f;
    if (other) cudaSetDevice(cur);
}


// Offsets of a handle's arrays within one allocation, each on a 256-byte boundary.
struct HandleLayout {
    size_t bytes = 0;
    std::vector<std::pair<void **, size_t>> slots;
    template <class T> void add(T *&p, int64_t n) {
        slots.emplace_back(reinterpret_cast<void **>(&p), bytes);
        bytes += (sizeof(T) * (size_t)(n > 0 ? n : 1) + 255) & ~(size_t)255;
    }
    void place(void *base) {
        for (auto &sl : slots) *sl.first = static_cast<char *>(base) + sl.second;
    }
};

#define B_TRY(expr)                                       \
    do {                                                  \
        cudaError_t e_ = (expr);                          \
        if (e_ != cudaSuccess) {                          \
            tmp.release(s);                                \
            free_handle(f);                               \
            return e_ == cudaErrorMemoryAllocation ? SDF_ERR_OOM : SDF_ERR_CUDA; \
        }                                                 \
    } while (0)

extern "C" int sdf_build_features(const float *soup, int64_t n_tri, uint32_t flags, void *stream, sdf_features *out) {
    if (!out) return SDF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!soup || n_tri <= 0) return SDF_ERR_INVALID_ARG;
    if (n_tri >= (int64_t(1) << 28)) return SDF_ERR_TOO_LARGE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t T = n_tri, n = 3 * T;
    sdf_features_s *f = new sdf_features_s();
    if (cudaGetDevice(&f->dev) != cudaSuccess) {
        delete f;
        return SDF_ERR_CUDA;
    }
    f->T = T;
    f->flags = flags;
    DevBuf tmp;
    // scratch: keys, vals (+ alternates), heads/scan, sort and scan temporaries, bounds
    const int64_t long_cap = n / (WELD_SHORT + 1) + 1;  // long mixed runs (each > WELD_SHORT entries)
    size_t off_keys = 0, off_kalt = off_keys + 8 * n, off_vals = off_kalt + 8 * n, off_valt = off_vals + 4 * n,
           off_head = off_valt + 4 * n, off_bb = off_head + 4 * (n + 1) + 64,
           off_long = (off_bb + 64 + 15) & ~(size_t)15,               // int2: 8-byte aligned (16 here)
           off_rtmp = (off_long + 8 * long_cap + 64 + 15) & ~(size_t)15;
    // one scan state for the build's scans and sorts, cleared once here (see scan_exclusive_u32)
    const size_t scan_bytes = std::max(scan_state_bytes(n + 1), radix_scan_state_bytes(n));
    const size_t off_scan = (off_rtmp + radix_tmp_bytes(n) + 255) & ~(size_t)255;
    size_t need = off_scan + scan_bytes + 1024;
    B_TRY(take_block(need, &tmp.p, &tmp.bytes, s));
    char *base = tmp.as<char>();
    uint64_t *keys = reinterpret_cast<uint64_t *>(base + off_keys), *kalt = reinterpret_cast<uint64_t *>(base + off_kalt);
    uint32_t *vals = reinterpret_cast<uint32_t *>(base + off_vals), *valt = reinterpret_cast<uint32_t *>(base + off_valt);
    uint32_t *head = reinterpret_cast<uint32_t *>(base + off_head);
    float *bb = reinterpret_cast<float *>(base + off_bb);
    unsigned *n_long = reinterpret_cast<unsigned *>(base + off_bb + 32);
    int2 *long_runs = reinterpret_cast<int2 *>(base + off_long);
    void *rtmp = base + off_rtmp;
    void *scan_state = base + off_scan;

    B_TRY(take_block(sizeof(DevCounters), reinterpret_cast<void **>(&f->ctr), &f->ctr_bytes, s));
    unsigned *const err = &f->ctr->status;  // a scan whose look-back ran out marks ST_TIMEOUT here
    // counters, the bounding box, the long-run count and the scan state start cleared (one launch)
    B_TRY(launch_dep(k_build_init, dim3(1), dim3(BT), 0, s, reinterpret_cast<unsigned *>(f->ctr),
                     (int64_t)(sizeof(DevCounters) / sizeof(unsigned)), bb, n_long,
                     reinterpret_cast<unsigned *>(scan_state), (int64_t)(scan_bytes / sizeof(unsigned))));
    // about four corners per thread, at most four blocks per SM of this part
    B_TRY(launch_dep(k_soup_bounds, dim3((unsigned)std::min<int64_t>((n + 4 * BT - 1) / (4 * BT), 4 * 152)), dim3(BT),
                     0, s, soup, n, bb, f->ctr));
    B_TRY(launch_dep(k_weld_keys, dim3(nblk(n)), dim3(BT), 0, s, soup, n, bb, keys, vals));
    B_TRY(radix_sort_u64(keys, vals, kalt, valt, n, 40, rtmp, scan_state, s, err));
    B_TRY(launch_dep(k_weld_fix, dim3(nblk(n)), dim3(BT), 0, s, keys, vals, soup, n, long_runs, long_cap, n_long));
    B_TRY(launch_dep(k_weld_sort_runs, dim3(2 * 152), dim3(256), 0, s, long_runs, n_long, long_cap, vals, soup));
    B_TRY(launch_dep(k_weld_heads, dim3(nblk(n)), dim3(BT), 0, s, keys, vals, soup, n, valt));
    // head[i] = number of run heads before i, head[n] = V (so head[i+1] is the inclusive count at i)
    B_TRY(scan_exclusive_u32(valt, head, n, true, scan_state, s, err));
    uint32_t Vh = 0;
    unsigned st_h = 0;
    {
        const HostRead rd[2] = {{&Vh, head + n, sizeof(uint32_t)}, {&st_h, &f->ctr->status, sizeof(unsigned)}};
        B_TRY(read_small(rd, 2, s));
    }
    if (st_h) {
        tmp.release(s);
        free_handle(f);
        return status_to_code(st_h);
    }
    const int64_t V = Vh;
    f->V = V;
    if (n % 2) {  // a closed 2-manifold has 3T/2 edges
        tmp.release(s);
        free_handle(f);
        return SDF_ERR_NONMANIFOLD;
    }
    const int64_t E = n / 2;
    f->E = E;
    {  // the handle's arrays, carved from one allocation (one pool call per build instead of 16)
        HandleLayout L;
        L.add(f->soup_vid, n);
        L.add(f->face_vid, n);
        L.add(f->face_soup, T);
        L.add(f->face_edge, n);
        L.add(f->vert_start, V + 1);
        L.add(f->vert_corner, n);
        L.add(f->vpos, 3 * V);
        L.add(f->edge_vf, E);
        L.add(f->face_rec, 4 * T);
        L.add(f->face_box, 2 * T);
        L.add(f->edge_rec, 5 * E);
        L.add(f->edge_class, E);
        L.add(f->vert_rec, 3 * V);
        L.add(f->vert_plane, n);
        L.add(f->vert_class, V);
        L.add(f->grad4, V);
        B_TRY(take_block(L.bytes, &f->block, &f->block_bytes, s));
        L.place(f->block);
    }
    B_TRY(launch_dep(k_weld_scatter, dim3(nblk(n)), dim3(BT), 0, s, vals, head, keys, soup, n, f->soup_vid,
                     f->vert_start, f->vert_corner, f->vpos, f->grad4));
    // spatial face order: sort faces by their smallest (Morton-ordered) vertex id
    int nb = 1;
    while ((int64_t(1) << nb) < V) nb++;
    B_TRY(launch_dep(k_face_keys, dim3(nblk(T)), dim3(BT), 0, s, f->soup_vid, T, keys, vals));
    B_TRY(radix_sort_u64(keys, vals, kalt, valt, T, nb, rtmp, scan_state, s, err));
    B_TRY(launch_dep(k_face_perm, dim3(nblk(T)), dim3(BT), 0, s, vals, f->soup_vid, T, f->face_soup, f->face_vid,
                     valt));
    B_TRY(launch_dep(k_corner_remap, dim3(nblk(n)), dim3(BT), 0, s, f->vert_corner, valt, n));
    // edge pairing through the vertex fans
    int32_t *twin = reinterpret_cast<int32_t *>(kalt);  // kalt is free again
    uint32_t *canon = valt;
    B_TRY(launch_dep(k_pair_fans, dim3(nblk(n)), dim3(BT), 0, s, f->vert_start, f->vert_corner, f->face_vid, n, twin,
                     canon, f->ctr));
    B_TRY(scan_exclusive_u32(canon, head, n, true, scan_state, s, err));
    // entries that no canonical edge writes (a broken mesh) stay -1 and are skipped by the records
    B_TRY(cudaMemsetAsync(f->edge_vf, 0xff, sizeof(int4) * (size_t)E, s));
    B_TRY(launch_dep(k_edge_emit, dim3(nblk(n)), dim3(BT), 0, s, f->vert_corner, f->face_vid, twin, canon, head, n,
                     f->edge_vf, f->face_edge));
    // The records are built without first reading the connectivity status (one host round trip
    // fewer): on a broken mesh they only see valid indices (the weld's are valid by construction,
    // unpaired edges are skipped) and the status read below rejects the handle.
    if (build_records(f, s) != SDF_OK) B_TRY(cudaErrorUnknown);
    DevCounters c;
    uint32_t n_canon = 0;
    {
        const HostRead rd[2] = {{&c, f->ctr, sizeof(DevCounters)}, {&n_canon, head + n, sizeof(uint32_t)}};
        B_TRY(read_small(rd, 2, s));
    }
    keep_block(tmp.p, tmp.bytes, s);  // idle after the read above synchronised the stream
    tmp.p = nullptr;
    tmp.bytes = 0;
    if (!c.status && (int64_t)n_canon != E) c.status |= ST_NONMANIFOLD;
    if (c.status) {
        int code = status_to_code(c.status);
        free_handle(f);
        return code;
    }
    f->counts[0] = V;
    f->counts[1] = E;
    for (int i = 2; i < 8; i++) f->counts[i] = (int64_t)c.cls[i];
    for (int i = 0; i < 7; i++) f->box_mom[i] = c.box_mom[i];
    *out = f;
    return SDF_OK;
}

extern "C" int sdf_features_update_positions(sdf_features f, const float *vertices, void *stream) {
    if (!f || !vertices) return SDF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    SDF_TRY(cudaMemcpyAsync(f->vpos, vertices, sizeof(float) * 3 * f->V, cudaMemcpyDeviceToDevice, s));
    SDF_TRY(cudaMemsetAsync(f->ctr->cls, 0, sizeof(f->ctr->cls), s));
    SDF_TRY(cudaMemsetAsync(&f->ctr->status, 0, sizeof(unsigned), s));  // re-evaluated below
    SDF_TRY(cudaMemsetAsync(f->ctr->prec, 0, sizeof(f->ctr->prec), s));  // precision terms, likewise
    SDF_TRY(cudaMemsetAsync(f->ctr->box_mom, 0, sizeof(f->ctr->box_mom), s));
    return build_records(f, s);
}

extern "C" void sdf_features_destroy(sdf_features f) {
    if (!f) return;
    cudaDeviceSynchronize();
    free_handle(f);
}

extern "C" int sdf_features_info(sdf_features f, int64_t *n_tri, int64_t *counts) {
    if (!f) return SDF_ERR_INVALID_ARG;
    if (n_tri) *n_tri = f->T;
    if (counts)
        for (int i = 0; i < 8; i++) counts[i] = f->counts[i];
    return SDF_OK;
}

extern "C" int sdf_features_vertex_map(sdf_features f, int32_t *soup_to_vertex, void *stream) {
    if (!f || !soup_to_vertex) return SDF_ERR_INVALID_ARG;
    SDF_TRY(cudaMemcpyAsync(soup_to_vertex, f->soup_vid, sizeof(int32_t) * 3 * f->T, cudaMemcpyDeviceToDevice,
                            reinterpret_cast<cudaStream_t>(stream)));
    return SDF_OK;
}

extern "C" int sdf_features_face_map(sdf_features f, int32_t *face_to_soup, void *stream) {
    if (!f || !face_to_soup) return SDF_ERR_INVALID_ARG;
    SDF_TRY(cudaMemcpyAsync(face_to_soup, f->face_soup, sizeof(int32_t) * f->T, cudaMemcpyDeviceToDevice,
                            reinterpret_cast<cudaStream_t>(stream)));
    return SDF_OK;
}

extern "C" int sdf_features_edges(sdf_features f, int32_t *out, void *stream) {
    if (!f || !out) return SDF_ERR_INVALID_ARG;
    SDF_TRY(cudaMemcpyAsync(out, f->edge_vf, sizeof(int4) * f->E, cudaMemcpyDeviceToDevice,
                            reinterpret_cast<cudaStream_t>(stream)));
    return SDF_OK;
}

extern "C" int sdf_features_vertices(sdf_features f, float *outp, void *stream) {
    if (!f || !outp) return SDF_ERR_INVALID_ARG;
    SDF_TRY(cudaMemcpyAsync(outp, f->vpos, sizeof(float) * 3 * f->V, cudaMemcpyDeviceToDevice,
                            reinterpret_cast<cudaStream_t>(stream)));
    return SDF_OK;
}

extern "C" const char *sdf_status_string(int status) {
    switch (status) {
    case SDF_OK: return "ok";
    case SDF_ERR_INVALID_ARG: return "invalid argument";
    case SDF_ERR_NONMANIFOLD: return "surface is not a closed, consistently oriented 2-manifold";
    case SDF_ERR_DEGENERATE: return "degenerate triangle or edge";
    case SDF_ERR_NONFINITE: return "non-finite coordinate";
    case SDF_ERR_TOO_LARGE: return "size beyond the supported index range";
    case SDF_ERR_OOM: return "device out of memory";
    case SDF_ERR_CUDA: return "CUDA runtime error";
    case SDF_ERR_TIMEOUT: return "bounded device wait gave up";
    case SDF_ERR_LIST_OVERFLOW: return "band list too short for the band";
    default: return "unknown status";
    }
}
