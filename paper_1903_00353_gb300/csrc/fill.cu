// Sign of the grid points beyond the band (the fill the paper names as the step after the narrow
// band, Section 11.3): every point outside the band gets -inf inside the surface and +inf outside,
// so the whole grid carries the inside/outside sign.
//
// The band half-width w exceeds the grid step h, so the surface never passes between two
// neighbouring grid points that are both outside the band: if it crossed the segment between
// them, both would lie within h < w of it.  Hence
//   (1) along an x-row, every run of points outside the band has the sign of the band point next
//       to it (left or right);
//   (2) a row with no band point at all has one sign along its whole length, and it is the sign
//       of the point next to it in a neighbouring row (y or z), whichever row that is;
//   (3) a grid without any band point is taken as outside.
// Kernels: k_fill_rows applies (1) and records per row the sign at x = 0 (0 for a row without band
// points); k_fill_lines resolves (2) by nearest-known propagation along y, then along z;
// k_fill_empty writes the rows of (2) that lie inside.  Points start at +inf (written by the tile
// kernel), so only inside points are written.
#include <math.h>
#include <stdint.h>

#include "sdf_internal.cuh"

namespace sdf {
namespace {

constexpr unsigned FULL_MASK = 0xffffffffu;

__device__ __forceinline__ int find_row_prob(const long long *rbase, int n, long long r) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rbase[mid] <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// negative in the sense of the field: d < 0, or -0
__device__ __forceinline__ bool is_neg(float v) { return signbit(v); }

// One warp per x-row.  rowsign[r] = sign at x = 0 (+1 / -1), or 0 if the row has no band point.
__global__ void k_fill_rows(const FillProb *P, const long long *rbase, int n, long long r_tot, int8_t *rowsign) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < r_tot; r += warps) {
        const int p = find_row_prob(rbase, n, r);
        const FillProb pr = P[p];
        float *row = pr.dist + (r - rbase[p]) * (long long)pr.nx;
        // sign of the first band point of the row
        int first = 0;  // 0: none yet, +1 / -1
        for (int x0 = 0; x0 < pr.nx && first == 0; x0 += 32) {
            const int x = x0 + lane;
            const float v = x < pr.nx ? row[x] : INFINITY;
            const bool band = isfinite(v);
            const unsigned bm = __ballot_sync(FULL_MASK, band), nm = __ballot_sync(FULL_MASK, band && is_neg(v));
            if (bm) {
                const int l = __ffs(bm) - 1;
                first = ((nm >> l) & 1u) ? -1 : 1;
            }
        }
        if (lane == 0) rowsign[r] = (int8_t)first;
        if (first == 0) continue;  // row without band points: resolved by the line passes
        int carry = first;         // sign of the nearest band point to the left (or the first one)
        for (int x0 = 0; x0 < pr.nx; x0 += 32) {
            const int x = x0 + lane;
            const float v = x < pr.nx ? row[x] : INFINITY;
            const bool band = isfinite(v);
            const unsigned bm = __ballot_sync(FULL_MASK, band), nm = __ballot_sync(FULL_MASK, band && is_neg(v));
            if (!band && x < pr.nx) {
                const unsigned left = bm & (0xffffffffu >> (31 - lane));  // band lanes <= this one
                const int s = left ? (((nm >> (31 - __clz(left))) & 1u) ? -1 : 1) : carry;
                if (s < 0) row[x] = -INFINITY;
            }
            if (bm) carry = ((nm >> (31 - __clz(bm))) & 1u) ? -1 : 1;
        }
    }
}

// Nearest-known propagation of the row signs along one line of the (y, z) row grid of each problem:
// along y for every (problem, z) when ALONG_Y, else along z for every (problem, y).  Unknown entries
// (0) take the sign of the nearest known entry before them, else after them; after the z pass the
// entries still unknown (a problem without band points) become outside.  Resolved rows are marked
// +-2 so that k_fill_empty can tell them from rows with band points.
template <bool ALONG_Y>
__global__ void k_fill_lines(const FillProb *P, const long long *lbase, int n, long long l_tot,
                             const long long *rbase, int8_t *rowsign) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long L = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); L < l_tot; L += warps) {
        const int p = find_row_prob(lbase, n, L);
        const FillProb pr = P[p];
        const long long li = L - lbase[p];
        // line li: ALONG_Y -> z = li, entries j = 0..ny-1 (stride 1); else y = li, entries k (stride ny)
        const int len = ALONG_Y ? pr.ny : pr.nz;
        const long long stride = ALONG_Y ? 1 : pr.ny;
        int8_t *e = rowsign + rbase[p] + (ALONG_Y ? li * pr.ny : li);
        // pass 1 (forward): carry the last known sign; pass 2 (backward) fills what is still unknown
        int carry = 0;
        for (int i0 = 0; i0 < len; i0 += 32) {
            const int i = i0 + lane;
            const int v = i < len ? (int)e[i * stride] : 0;
            const unsigned km = __ballot_sync(FULL_MASK, v != 0), nm = __ballot_sync(FULL_MASK, v < 0);
            if (i < len && v == 0) {
                const unsigned left = km & (0xffffffffu >> (31 - lane));
                const int s = left ? (((nm >> (31 - __clz(left))) & 1u) ? -1 : 1) : carry;
                if (s != 0) e[i * stride] = (int8_t)(2 * s);
            }
            if (km) carry = ((nm >> (31 - __clz(km))) & 1u) ? -1 : 1;
        }
        __syncwarp();
        carry = 0;
        for (int i0 = ((len - 1) / 32) * 32; i0 >= 0; i0 -= 32) {
            const int i = i0 + lane;
            const int v = i < len ? (int)e[i * stride] : 0;
            const unsigned km = __ballot_sync(FULL_MASK, v != 0), nm = __ballot_sync(FULL_MASK, v < 0);
            if (i < len && v == 0) {
                const unsigned right = km & (0xffffffffu << lane);  // known lanes >= this one
                int s = right ? (((nm >> (__ffs(right) - 1)) & 1u) ? -1 : 1) : carry;
                if (!ALONG_Y && s == 0) s = 1;  // no band point in the whole problem: outside
                if (s != 0) e[i * stride] = (int8_t)(2 * s);
            }
            if (km) carry = ((nm >> (__ffs(km) - 1)) & 1u) ? -1 : 1;
        }
    }
}

// rows without band points that lie inside: the whole row becomes -inf
__global__ void k_fill_empty(const FillProb *P, const long long *rbase, int n, long long r_tot,
                             const int8_t *rowsign) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < r_tot; r += warps) {
        if (rowsign[r] != -2) continue;
        const int p = find_row_prob(rbase, n, r);
        const FillProb pr = P[p];
        float *row = pr.dist + (r - rbase[p]) * (long long)pr.nx;
        for (int x = lane; x < pr.nx; x += 32) row[x] = -INFINITY;
    }
}

}  // namespace

cudaError_t fill_sign(const FillProb *P, const long long *rbase, const long long *zbase, const long long *ybase, int n,
                      long long r_tot, long long z_tot, long long y_tot, int8_t *rowsign, int n_sm, cudaStream_t s) {
    const int blocks = 8 * n_sm;  // 8 warps per block, grid-stride over rows / lines
    k_fill_rows<<<blocks, 256, 0, s>>>(P, rbase, n, r_tot, rowsign);
    SDF_LAUNCHED(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_fill_lines<true><<<blocks, 256, 0, s>>>(P, zbase, n, z_tot, rbase, rowsign);
    SDF_LAUNCHED(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_fill_lines<false><<<blocks, 256, 0, s>>>(P, ybase, n, y_tot, rbase, rowsign);
    SDF_LAUNCHED(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_fill_empty<<<blocks, 256, 0, s>>>(P, rbase, n, r_tot, rowsign);
    SDF_LAUNCHED(1);
    return cudaGetLastError();
}

}  // namespace sdf
