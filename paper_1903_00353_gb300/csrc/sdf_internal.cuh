// Internal declarations shared by the CUDA translation units of the library.
// Nothing here is part of the C ABI (include/sdf.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sdf.h"

namespace sdf {

// ----------------------------------------------------------------------------- status bits (device word)
enum : unsigned {
    ST_NONFINITE = 1u,
    ST_DEGENERATE = 2u,
    ST_NONMANIFOLD = 4u,
    ST_PAIR_OVERFLOW = 8u,   // (tile, region) pair list too small: grow and rerun
    ST_PATCH_OVERFLOW = 16u, // FP64 re-decision list too small: grow and rerun
    ST_LIST_OVERFLOW = 32u,  // the caller's compact band list is too short (its count holds the length)
    ST_TIMEOUT = 64u,        // a bounded device wait (the scan's look-back) ran out
};

// vertex / edge classes (Section 3.1, Section 3.2)
enum : int8_t { CLS_FLAT = 0, CLS_CONVEX = 1, CLS_CONCAVE = -1, CLS_SADDLE = 2 };

// tile of the narrow-band kernel: TX x TY x TZ grid points (x fastest)
constexpr int TILE_X = 32, TILE_Y = 8, TILE_Z = 8;
constexpr int TILE_PTS = TILE_X * TILE_Y * TILE_Z;

// ----------------------------------------------------------------------------- device memory
// All library allocations come from one stream-ordered memory pool per device that keeps freed
// memory cached (release threshold = unlimited), so a build or a call that needs scratch of a
// size seen before does not reach the driver's allocator.
cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s);
cudaError_t pool_free(void *p, cudaStream_t s);
// counts a pinned host allocation (reported by sdf_memory_stats)
void count_host_alloc();

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaError_t reserve(size_t need, cudaStream_t s) {
        if (need <= bytes) return cudaSuccess;
        if (p) pool_free(p, s);
        p = nullptr;
        bytes = 0;
        size_t want = need + need / 4 + 256;
        cudaError_t e = pool_alloc(&p, want, s);
        if (e == cudaSuccess) bytes = want;
        return e;
    }
    void release(cudaStream_t s) {
        if (p) pool_free(p, s);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

// ----------------------------------------------------------------------------- device status / counters
struct DevCounters {
    unsigned status;     // build / position-update errors (ST_NONFINITE, ST_DEGENERATE, ST_NONMANIFOLD)
    unsigned nb_status;  // narrow-band overflows (ST_PAIR_OVERFLOW, ST_PATCH_OVERFLOW, ST_LIST_OVERFLOW)
    unsigned long long n_candidates;   // (point, region) pairs merged
    unsigned long long n_band;         // band points written
    unsigned long long n_patch;        // points re-decided in FP64
    unsigned long long n_pairs;        // (tile, region) pairs scheduled
    unsigned long long n_rows;         // grid rows intersected with a region
    unsigned long long n_rows_hit;     // of which non-empty
    unsigned long long cls[8];         // classification counts
    unsigned tile_hist[16];            // band tiles per cost class (class 0: the most pairs)
    unsigned tile_cursor[16];          // fill cursors of the classes in the band tile list
    unsigned n_split;                  // band tiles split over several CTAs (slots taken)
    unsigned n_split_items;            // their work items
    // Precision terms of the current positions (FP32 bits of non-negative floats, so an unsigned
    // atomicMax takes their maximum), written by the records kernels: PREC_MESH_M the largest
    // vertex coordinate magnitude, PREC_TAU_A / PREC_TAU_B the shape term of the FP32 plane
    // and normal errors, tau_a + tau_b * W (see k_face_records), PREC_TAU_V the direction error
    // of the unit pseudonormals per unit distance (see k_vertex_records).
    unsigned prec[4];
    // Sums over the faces of the extents (bx, by, bz) of their bounding boxes, written by the build:
    // bx, by, bz, bx by, bx bz, by bz, bx by bz.  They give the expected number of (tile, region)
    // pairs of a grid before any kernel runs (pair_estimate in band.cu).
    double box_mom[7];
};
enum { PREC_MESH_M = 0, PREC_TAU_A = 1, PREC_TAU_B = 2, PREC_TAU_V = 3 };
// unit roundoff of FP32 (2^-24)
constexpr float U32 = 5.9604644775390625e-8f;

struct Plan;
void plan_free(Plan *pl, cudaStream_t s);
// keep a destroyed handle's plan (with its scratch) for the next handle on the device
void plan_park(Plan *pl, cudaStream_t s);

// compact band list of one problem (see sdf_narrow_band_list)
struct ListOut {
    sdf_band_entry *list;
    long long cap;
    unsigned long long *count;
    float *dist = nullptr;  // nullable: the signed distance of every entry (the sparse forward)
};

// the narrow band of n problems (sdf_narrow_band), with optional band lists (host array [n] or
// null; an entry with a null list asks for none)
int narrow_band_all(const sdf_features *feats, const sdf_grid *grids, const float *band_w, int32_t n,
                    float *const *out_dist, int32_t *const *out_winner, uint32_t flags, cudaStream_t s,
                    const ListOut *lists = nullptr);
int ensure_events(sdf_features_s *f);
// add the durations of pending timed calls to the handle's totals (waits for their events)
int resolve_timing(sdf_features_s *f);

}  // namespace sdf

// ----------------------------------------------------------------------------- the handle
struct sdf_features_s {
    int64_t T = 0, V = 0, E = 0;
    uint32_t flags = 0;
    int dev = -1;  // the device the handle was built on (its memory, kept blocks and plan belong to it)
    // connectivity (fixed after the build); faces are stored in a spatial order (by smallest
    // welded vertex id), face_soup maps them back to soup triangles
    int32_t *soup_vid = nullptr;    // [3T] welded vertex of each soup corner (soup order)
    int32_t *face_soup = nullptr;   // [T] soup triangle of each library face
    int32_t *face_vid = nullptr;    // [3T] welded vertex of each library face corner
    int32_t *face_edge = nullptr;   // [3T] edge id of the edge from corner k to corner k+1
    int4 *edge_vf = nullptr;        // [E] (va < vb, f1 holding va->vb, f2 holding vb->va)
    int32_t *vert_start = nullptr;  // [V+1] CSR into vert_corner
    int32_t *vert_corner = nullptr; // [3T] face corners (3 f + k) grouped by vertex
    // geometry (re-evaluated by sdf_features_update_positions)
    float *vpos = nullptr;          // [V][3]
    float4 *face_rec = nullptr;     // [T][4] (n, c0) and three inward side planes (m, c)
    float4 *face_box = nullptr;     // [T][2] vertex bounding box lo, hi
    float4 *edge_rec = nullptr;     // [E][5] (a, L) (t, t.a) (-m1, m1.a) (-m2, m2.a) (n1+n2, |n1+n2|)
    float4 *vert_rec = nullptr;     // [V][3] (v, start) (unit N_alpha, count) (cone axis, cos theta)
    float4 *vert_plane = nullptr;   // [3T] (-e_j, e_j.v) per incident edge, CSR by vert_start
    int8_t *edge_class = nullptr;   // [E]
    int8_t *vert_class = nullptr;   // [V]
    int64_t counts[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double box_mom[7] = {0, 0, 0, 0, 0, 0, 0};  // the build's face-box moments (DevCounters::box_mom)
    float4 *grad4 = nullptr;        // [V] FP32 vertex-gradient sums of an adjoint call (x, y, z, 0),
                                    // zero between calls
    void *block = nullptr;           // one allocation holding every array above
    size_t block_bytes = 0;
    sdf::DevCounters *ctr = nullptr; // device counters
    size_t ctr_bytes = 0;
    // narrow-band scratch of single-problem calls (problem table, bins, pairs), grown on demand
    sdf::Plan *plan = nullptr;
    sdf::DevBuf fwd_winner;  // winners recomputed by a backward call that was given none
    // stage timing (SDF_FLAG_TIMING)
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    double t_ms[4] = {0, 0, 0, 0};
    int64_t t_calls[4] = {0, 0, 0, 0};
    // events recorded by the last timed forward (ev[0..3]) / adjoint (ev[4..5]) and not read yet:
    // they are read when the next timed call needs the events or when sdf_features_timing asks,
    // so that timing never makes a call wait for its own work
    bool fwd_pending = false, adj_pending = false;
};

namespace sdf {

// ----------------------------------------------------------------------------- launch counter
void count_launches(int64_t n);
#define SDF_LAUNCHED(n) ::sdf::count_launches(n)

// ----------------------------------------------------------------------------- dependent launches
// The build and the scans are chains of short kernels on one stream, each waiting for the last.
// They are launched with programmatic stream serialisation: a kernel may be scheduled while its
// predecessor still runs and waits at its top (griddepcontrol.wait) until the predecessor has
// finished and its writes are visible, so each launch's latency hides behind the kernel before it.
// Every kernel launched by launch_dep calls dep_wait() before it touches memory, then dep_next()
// to let its successor be scheduled (after the wait: at most one launch waits at a time).  Both are
// no-ops in a kernel launched without the attribute.  SDF_PDL=0 in the environment launches every
// kernel without it.
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void dep_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
bool pdl_enabled();

template <typename... P, typename... A>
cudaError_t launch_dep(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    count_launches(1);
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ----------------------------------------------------------------------------- scans and sorts (scan_sort.cu)
// Exclusive scan of n uint32 values (in may equal out); out[n] receives the total when
// write_total is set.  One launch (decoupled look-back).  state holds scan_state_bytes(n) bytes,
// zeroed before its first scan; every scan leaves it ready for the next one issued after it on
// the same stream (any n up to the size it was made for).  A look-back wait that runs out sets
// ST_TIMEOUT in *err (nullable).
size_t scan_state_bytes(int64_t n);
cudaError_t scan_exclusive_u32(const uint32_t *in, uint32_t *out, int64_t n, bool write_total, void *state,
                               cudaStream_t s, unsigned *err);
// Stable LSD radix sort of (keys, vals) on bits [0, bits).  Buffers *_alt are ping-pong
// scratch of the same size; the result ends in keys/vals.  tmp holds radix_tmp_bytes(n) bytes of
// histograms; scan_state is a scan state (as above) of radix_scan_state_bytes(n) bytes.  A sort
// whose tiles fit on the device at once is one cooperative launch (its grid barrier uses words 2
// and 3 of the scan state, which every completed sort leaves ready); a barrier wait that runs out
// sets ST_TIMEOUT in *err.  Otherwise three launches per 8-bit pass.
size_t radix_tmp_bytes(int64_t n);
size_t radix_scan_state_bytes(int64_t n);
cudaError_t radix_sort_u64(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, int64_t n,
                           int bits, void *tmp, void *scan_state, cudaStream_t s, unsigned *err);

// ----------------------------------------------------------------------------- small reads (scan_sort.cu)
// Reads up to 4 small device values (counters, sizes, status words) into host variables and
// synchronises the stream.  A one-block kernel writes them into pinned host memory, so the read
// does not queue behind large copies that the caller may have in flight on the copy engines.
struct HostRead {
    void *dst;
    const void *src;
    unsigned bytes;
};
cudaError_t read_small(const HostRead *reads, int n, cudaStream_t s);

// ----------------------------------------------------------------------------- sign beyond the band (fill.cu)
// One problem's dense output, float[nz][ny][nx].
struct FillProb {
    float *dist;
    int nx, ny, nz;
};
// Writes -inf to the points outside the band that lie inside the surface (points outside the band
// hold +inf on entry).  rbase / zbase / ybase: prefix sums over the n problems of ny * nz (x-rows),
// nz and ny, with totals r_tot, z_tot, y_tot; rowsign: int8 scratch of r_tot entries.
cudaError_t fill_sign(const FillProb *P, const long long *rbase, const long long *zbase, const long long *ybase, int n,
                      long long r_tot, long long z_tot, long long y_tot, int8_t *rowsign, int n_sm, cudaStream_t s);

// ----------------------------------------------------------------------------- geometry stage (build.cu)
int build_records(sdf_features_s *f, cudaStream_t s);

// ----------------------------------------------------------------------------- division by a grid size
// Unsigned division by an invariant divisor d >= 1 as a multiply-high and a shift (round-up
// multiplier method of Granlund and Montgomery, 1994): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (umulhi(n, m) + n) >> l for every n < 2^31.
struct FastDiv {
    uint32_t d = 1, m = 1, l = 0;
    FastDiv() = default;
    explicit FastDiv(uint32_t dv) : d(dv) {
        while ((uint64_t(1) << l) < dv) l++;
        m = (uint32_t)(((uint64_t(1) << 32) * ((uint64_t(1) << l) - dv)) / dv + 1);
    }
    __device__ __forceinline__ uint32_t div(uint32_t n) const { return (__umulhi(n, m) + n) >> l; }
};

// ----------------------------------------------------------------------------- small device helpers
__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double3 d3(float3 a) { return make_double3(a.x, a.y, a.z); }
__device__ __forceinline__ double3 operator-(double3 a, double3 b) { return make_double3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ double3 operator+(double3 a, double3 b) { return make_double3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ double3 operator*(double s, double3 a) { return make_double3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ double ddot3(double3 a, double3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ double3 dcross3(double3 a, double3 b) {
    return make_double3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 load_vpos(const float *vpos, int v) {
    return make_float3(vpos[3 * v], vpos[3 * v + 1], vpos[3 * v + 2]);
}

}  // namespace sdf

#define SDF_TRY(expr)                                  \
    do {                                               \
        cudaError_t e_ = (expr);                       \
        if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? SDF_ERR_OOM : SDF_ERR_CUDA; \
    } while (0)
// propagate a library status code
#define SDF_TRY_ST(expr)                               \
    do {                                               \
        int st_ = (expr);                              \
        if (st_ != SDF_OK) return st_;                 \
    } while (0)
