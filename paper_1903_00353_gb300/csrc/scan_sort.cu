// Device-wide exclusive scan and stable LSD radix sort.
//
// The paper orders edge and vertex entries with a library sort_by_key followed by
// a gather and a serial per-group fix-up (Section 7.1).  Here both steps are one
// hand-written stable radix sort of (64-bit key, 32-bit payload) pairs: 8-bit
// digits, a per-tile histogram pass, a device-wide scan of the digit offsets and a
// scatter pass that ranks keys inside each warp with __match_any_sync and stages
// the tile in shared memory so global writes of one digit run are contiguous.  A
// sort whose tiles all fit on the GPU at once runs every pass in one cooperative
// launch instead.
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "sdf_internal.cuh"

namespace sdf {

// ============================================================================= scan
namespace {
constexpr int SC_THREADS = 256, SC_ITEMS = 16, SC_TILE = SC_THREADS * SC_ITEMS;

__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// block-wide exclusive scan of one value per thread; returns the block total via *total
__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t *total) {
    __shared__ uint32_t warp_tot[SC_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = warp_incl_scan_u32(v);
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < SC_THREADS / 32 ? warp_tot[lane] : 0u;
        uint32_t ti = warp_incl_scan_u32(t);
        if (lane < SC_THREADS / 32) warp_tot[lane] = ti - t;
        if (lane == SC_THREADS / 32 - 1) *total = ti;
    }
    __syncthreads();
    uint32_t r = warp_tot[warp] + inc - v;
    __syncthreads();
    return r;
}

// exclusive scan of each tile (blocked arrangement: thread t owns SC_ITEMS consecutive items),
// offset by offs[blockIdx.x] (nullable)
__global__ void __launch_bounds__(SC_THREADS) k_scan_apply(const uint32_t *in, uint32_t *out, int64_t n,
                                                           const uint32_t *offs, uint32_t *total_out) {
    dep_wait();
    dep_next();
    int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
    uint32_t v[SC_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < SC_ITEMS; i++) {
        v[i] = (base + i < n) ? in[base + i] : 0u;
        s += v[i];
    }
    __shared__ uint32_t tot;
    uint32_t run = block_excl_scan_u32(s, &tot) + (offs ? offs[blockIdx.x] : 0u);
#pragma unroll
    for (int i = 0; i < SC_ITEMS; i++) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (total_out && blockIdx.x == gridDim.x - 1 && threadIdx.x == SC_THREADS - 1) *total_out = run;
}

// Single-pass scan with decoupled look-back (D. Merrill and M. Garland, "Single-pass Parallel
// Prefix Scan with Decoupled Look-back", NVIDIA technical report NVR-2016-002).  Each CTA draws
// its tile from a ticket, so it only ever waits for tiles whose CTAs have already started; it
// publishes its tile's total (AGGREGATE), then sums its predecessors' words walking back 32 at a
// time until one carries an inclusive prefix (PREFIX), and publishes its own inclusive prefix.
// The state region: [0] ticket, [1] epoch, [2] and [3] the one-launch radix sort's grid barrier
// (below; unused here), then one 64-bit word per tile, epoch << 34 | flag << 32 | value.  Words of earlier scans carry an older epoch and count as not yet published.  The CTA
// that draws the last ticket puts the ticket back to 0, and the one holding the last tile
// advances the epoch when it is done (by then every CTA has read it), so the region is ready for
// the next scan issued after this one on the stream.  A wait that runs out of polls marks
// ST_TIMEOUT in *err (nullable) and leaves the scan unfinished instead of hanging.
constexpr unsigned long long SCAN_AGG = 1ull << 32, SCAN_PFX = 2ull << 32;
constexpr unsigned SCAN_POLL_LIMIT = 1u << 20;

__global__ void __launch_bounds__(SC_THREADS) k_scan_chained(const uint32_t *in, uint32_t *out, int64_t n,
                                                             unsigned *hdr, unsigned long long *status,
                                                             uint32_t *total_out, unsigned *err) {
    dep_wait();
    dep_next();
    __shared__ unsigned s_tile, s_epoch;
    __shared__ uint32_t s_prefix, s_tot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        s_epoch = *(volatile unsigned *)(hdr + 1) & 0x3fffffffu;
        const unsigned t = atomicAdd(hdr, 1u);
        if (t == gridDim.x - 1) atomicExch(hdr, 0u);  // every ticket is drawn: ready for the next scan
        s_tile = t;
    }
    __syncthreads();
    const unsigned tile = s_tile;
    const unsigned long long tag = (unsigned long long)s_epoch << 34;
    const int64_t base = (int64_t)tile * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
    uint32_t v[SC_ITEMS];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < SC_ITEMS; i++) {
        v[i] = (base + i < n) ? in[base + i] : 0u;
        sum += v[i];
    }
    uint32_t run = block_excl_scan_u32(sum, &s_tot);  // ends with a barrier: s_tot is set
    const uint32_t tot = s_tot;
    if (threadIdx.x == 0) {
        atomicExch(status + tile, tag | (tile == 0 ? SCAN_PFX : SCAN_AGG) | tot);
        if (tile == 0) s_prefix = 0;
    }
    if (warp == 0 && tile > 0) {
        uint32_t acc = 0;
        int64_t j = (int64_t)tile - 1;  // the nearest predecessor not yet added
        unsigned polls = 0;
        bool ok = true;
        for (;;) {
            const int64_t idx = j - lane;
            // before the first tile: an inclusive prefix of 0
            const unsigned long long w = idx >= 0 ? __ldcv(status + idx) : (tag | SCAN_PFX);
            const bool valid = (w >> 34) == (tag >> 34) && (w & (3ull << 32)) != 0;
            const unsigned vmask = __ballot_sync(0xffffffffu, valid);
            const unsigned pmask = __ballot_sync(0xffffffffu, valid && (w & SCAN_PFX) != 0);
            const int p = pmask ? __ffs(pmask) - 1 : 31;  // the nearest prefix ends the walk
            const unsigned need = p == 31 ? 0xffffffffu : (2u << p) - 1u;
            if ((vmask & need) == need) {
                uint32_t x = lane <= p ? (uint32_t)w : 0u;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                acc += x;
                if (pmask) break;
                j -= 32;
                continue;
            }
            if (++polls > SCAN_POLL_LIMIT) {
                ok = false;
                break;
            }
        }
        if (lane == 0) {
            atomicExch(status + tile, tag | SCAN_PFX | (acc + tot));
            s_prefix = acc;
            if (!ok && err) atomicOr(err, ST_TIMEOUT);
        }
    }
    __syncthreads();
    run += s_prefix;
#pragma unroll
    for (int i = 0; i < SC_ITEMS; i++) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (tile == gridDim.x - 1 && threadIdx.x == 0) {
        if (total_out) *total_out = s_prefix + tot;
        atomicAdd(hdr + 1, 1u);  // every CTA has read the epoch: the next scan takes the next one
    }
}
}  // namespace

size_t scan_state_bytes(int64_t n) {
    const int64_t tiles = (n + SC_TILE - 1) / SC_TILE;
    return 16 + sizeof(unsigned long long) * (size_t)(tiles + 2);
}

cudaError_t scan_exclusive_u32(const uint32_t *in, uint32_t *out, int64_t n, bool write_total, void *state,
                               cudaStream_t s, unsigned *err) {
    if (n <= 0) {
        if (write_total) return cudaMemsetAsync(out, 0, sizeof(uint32_t), s);
        return cudaSuccess;
    }
    const int64_t nb = (n + SC_TILE - 1) / SC_TILE;
    uint32_t *total = write_total ? out + n : nullptr;
    if (nb == 1)
        return launch_dep(k_scan_apply, dim3(1), dim3(SC_THREADS), 0, s, in, out, n, (const uint32_t *)nullptr, total);
    unsigned *hdr = reinterpret_cast<unsigned *>(state);
    return launch_dep(k_scan_chained, dim3((unsigned)nb), dim3(SC_THREADS), 0, s, in, out, n, hdr,
                      reinterpret_cast<unsigned long long *>(hdr + 4), total, err);
}

// ============================================================================= radix sort
// LSD radix sort of 64-bit keys with 32-bit values, 8 bits per pass: per pass a digit histogram
// per tile of keys, one scan of the digit-major histograms, and a stable scatter (ranks within
// each warp by match_any, then across the warps of the tile, the tile staged in shared memory so
// that the global writes of each digit run are contiguous).  The tile holds 256 x ITEMS keys;
// ITEMS is chosen per sort so that small sorts (the weld of a 50 k-triangle mesh sorts 150 k
// keys) still spread over every SM instead of a few dozen CTAs.
namespace {
constexpr int RS_THREADS = 256, RS_WARPS = RS_THREADS / 32, RADIX = 256;
template <int ITEMS>
constexpr size_t rs_smem() {
    return (size_t)RS_THREADS * ITEMS * (sizeof(uint64_t) + sizeof(uint32_t)) +
           (size_t)RS_WARPS * RADIX * sizeof(uint32_t) + 2 * RADIX * sizeof(uint32_t);
}

template <int ITEMS>
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint64_t *keys, int64_t n, int shift,
                                                        uint32_t *hist, int64_t nb) {
    dep_wait();
    dep_next();
    constexpr int TILE = RS_THREADS * ITEMS;
    __shared__ uint32_t h[RADIX];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * TILE;
    for (int i = 0; i < ITEMS; i++) {
        int64_t idx = base + (int64_t)i * RS_THREADS + threadIdx.x;
        if (idx < n) atomicAdd(&h[(unsigned)(keys[idx] >> shift) & (RADIX - 1)], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];  // digit-major
}

template <int ITEMS>
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint64_t *kin, const uint32_t *vin,
                                                           uint64_t *kout, uint32_t *vout, int64_t n, int shift,
                                                           const uint32_t *offs, int64_t nb) {
    dep_wait();
    dep_next();
    constexpr int TILE = RS_THREADS * ITEMS;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *skey = reinterpret_cast<uint64_t *>(smem);
    uint32_t *sval = reinterpret_cast<uint32_t *>(skey + TILE);
    uint32_t *wcnt = sval + TILE;               // [RS_WARPS][RADIX]
    uint32_t *bstart = wcnt + RS_WARPS * RADIX; // [RADIX]
    uint32_t *btot = bstart + RADIX;           // [RADIX]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RADIX; i += RS_THREADS) wcnt[i] = 0;
    __syncthreads();

    const int64_t tile0 = (int64_t)blockIdx.x * TILE;
    const int64_t wbase = tile0 + (int64_t)warp * (32 * ITEMS);
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint64_t k[ITEMS];
    uint32_t v[ITEMS], rank[ITEMS];
    uint32_t *mycnt = wcnt + warp * RADIX;
#pragma unroll
    for (int it = 0; it < ITEMS; it++) {
        int64_t idx = wbase + it * 32 + lane;
        bool valid = idx < n;
        k[it] = valid ? kin[idx] : 0ull;
        v[it] = valid ? vin[idx] : 0u;
        unsigned d = valid ? ((unsigned)(k[it] >> shift) & (RADIX - 1)) : (RADIX + lane);  // invalid: own group
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = valid ? mycnt[d] : 0u;
        __syncwarp();
        if (valid && (peers & lt_mask) == 0u) mycnt[d] = before + __popc(peers);
        __syncwarp();
        rank[it] = before + __popc(peers & lt_mask);
    }
    __syncthreads();
    {   // thread t owns digit t: prefix over warps, then block totals
        uint32_t run = 0;
        for (int w = 0; w < RS_WARPS; w++) {
            uint32_t c = wcnt[w * RADIX + threadIdx.x];
            wcnt[w * RADIX + threadIdx.x] = run;
            run += c;
        }
        btot[threadIdx.x] = run;
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive scan of 256 digit totals by one warp (8 per lane)
        uint32_t loc[8], s = 0;
#pragma unroll
        for (int i = 0; i < 8; i++) { loc[i] = btot[lane * 8 + i]; s += loc[i]; }
        uint32_t inc = warp_incl_scan_u32(s);
        uint32_t run = inc - s;
#pragma unroll
        for (int i = 0; i < 8; i++) { bstart[lane * 8 + i] = run; run += loc[i]; }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < ITEMS; it++) {
        int64_t idx = wbase + it * 32 + lane;
        if (idx < n) {
            unsigned d = (unsigned)(k[it] >> shift) & (RADIX - 1);
            uint32_t lp = bstart[d] + mycnt[d] + rank[it];
            skey[lp] = k[it];
            sval[lp] = v[it];
        }
    }
    __syncthreads();
    int cnt = (n - tile0 < (int64_t)TILE) ? (int)(n - tile0) : TILE;
    for (int i = threadIdx.x; i < cnt; i += RS_THREADS) {
        uint64_t key = skey[i];
        unsigned d = (unsigned)(key >> shift) & (RADIX - 1);
        int64_t g = (int64_t)offs[(int64_t)d * nb + blockIdx.x] + (i - (int64_t)bstart[d]);
        kout[g] = key;
        vout[g] = sval[i];
    }
}

// ---------------------------------------------------------------------------- one-launch sort
// A sort whose tiles can all be resident at once runs every pass in one cooperative launch, one
// CTA per tile.  Per pass: (1) each CTA loads its tile's keys into registers, ranks them by digit
// as the scatter pass above does, and writes its 256 digit counts (digit-major); grid barrier;
// (2) the counts of each digit are scanned over the tiles, one CTA per digit, and the digit's
// total is stored; grid barrier; (3) each CTA adds the digits' global starts to its own prefixes
// and scatters its keys in place: every key of the pass is already in registers, so the pass
// needs no second buffer; grid barrier (the next pass reads what the others wrote).  Data written
// by other CTAs is read past L1 (ld.global.cg).  Against the three launches per pass above (a
// histogram, a scan and a scatter) this makes 1 launch per sort.
constexpr unsigned RS_POLL_LIMIT = 1u << 20;

// Grid barrier of a cooperative launch on bar[0] (arrivals, 0 between barriers) and bar[1]
// (generation): the last CTA to arrive clears the arrivals and advances the generation; the others
// wait until it reaches `target`.  A wait that runs out of polls marks ST_TIMEOUT in *err and
// returns false (the CTA then ends; the others run out at their next barrier).
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned target, unsigned *err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();  // the CTA's writes (ordered before this thread by the block barrier) first
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned polls = 0;
            while ((int)(*(volatile unsigned *)(bar + 1) - target) < 0) {
                if (++polls > RS_POLL_LIMIT) {
                    ok = 0;
                    if (err) atomicOr(err, ST_TIMEOUT);
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <int ITEMS>
constexpr size_t rs_one_smem() {
    return (size_t)RS_THREADS * ITEMS * (sizeof(uint64_t) + sizeof(uint32_t)) +
           (size_t)RS_WARPS * RADIX * sizeof(uint32_t) + 2 * RADIX * sizeof(uint32_t);
}

template <int ITEMS>
__global__ void __launch_bounds__(RS_THREADS) k_rs_one(uint64_t *keys, uint32_t *vals, int64_t n, int passes,
                                                       uint32_t *counts, uint32_t *totals, unsigned *bar,
                                                       unsigned *err) {
    constexpr int TILE = RS_THREADS * ITEMS;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *skey = reinterpret_cast<uint64_t *>(smem);
    uint32_t *sval = reinterpret_cast<uint32_t *>(skey + TILE);
    uint32_t *wcnt = sval + TILE;                // [RS_WARPS][RADIX]
    uint32_t *bstart = wcnt + RS_WARPS * RADIX;  // [RADIX] start of each digit's run in the tile
    uint32_t *gofs = bstart + RADIX;             // [RADIX] where that run goes in the output
    __shared__ unsigned s_gen;
    __shared__ uint32_t s_tot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned nb = gridDim.x, t = blockIdx.x;
    if (threadIdx.x == 0) s_gen = *(volatile unsigned *)(bar + 1);  // before the first arrival
    __syncthreads();
    unsigned target = s_gen;
    const int64_t tile0 = (int64_t)t * TILE;
    const int64_t wbase = tile0 + (int64_t)warp * (32 * ITEMS);
    const int cnt = (int)(n - tile0 < (int64_t)TILE ? n - tile0 : (int64_t)TILE);
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint32_t *mycnt = wcnt + warp * RADIX;
    for (int p = 0; p < passes; p++) {
        const int shift = 8 * p;
        // (1) ranks within the tile: lanes in order within a warp, warps in order (stable)
        for (int i = threadIdx.x; i < RS_WARPS * RADIX; i += RS_THREADS) wcnt[i] = 0;
        __syncthreads();
        uint64_t k[ITEMS];
        uint32_t v[ITEMS], rank[ITEMS];
#pragma unroll
        for (int it = 0; it < ITEMS; it++) {
            const int64_t idx = wbase + it * 32 + lane;
            const bool valid = idx < n;
            k[it] = valid ? __ldcg(keys + idx) : 0ull;
            v[it] = valid ? __ldcg(vals + idx) : 0u;
            const unsigned d = valid ? ((unsigned)(k[it] >> shift) & (RADIX - 1)) : (RADIX + lane);
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const uint32_t before = valid ? mycnt[d] : 0u;
            __syncwarp();
            if (valid && (peers & lt_mask) == 0u) mycnt[d] = before + __popc(peers);
            __syncwarp();
            rank[it] = before + __popc(peers & lt_mask);
        }
        __syncthreads();
        {  // thread d: prefix of digit d over the warps, the tile's count, its start in the tile
            uint32_t run = 0;
            for (int w = 0; w < RS_WARPS; w++) {
                const uint32_t c = wcnt[w * RADIX + threadIdx.x];
                wcnt[w * RADIX + threadIdx.x] = run;
                run += c;
            }
            counts[(int64_t)threadIdx.x * nb + t] = run;
            bstart[threadIdx.x] = block_excl_scan_u32(run, &s_tot);
        }
        if (!grid_barrier(bar, ++target, err)) return;
        // (2) exclusive scan of digit d's counts over the tiles, in place, and the digit's total
        for (unsigned d = t; d < (unsigned)RADIX; d += nb) {
            uint32_t *row = counts + (int64_t)d * nb;
            const unsigned per = (nb + RS_THREADS - 1) / RS_THREADS;
            const unsigned j0 = min(threadIdx.x * per, nb), j1 = min(j0 + per, nb);
            uint32_t s = 0;
            for (unsigned j = j0; j < j1; j++) s += __ldcg(row + j);
            uint32_t run = block_excl_scan_u32(s, &s_tot);
            for (unsigned j = j0; j < j1; j++) {
                const uint32_t c = __ldcg(row + j);
                row[j] = run;
                run += c;
            }
            if (threadIdx.x == 0) totals[d] = s_tot;
        }
        if (!grid_barrier(bar, ++target, err)) return;
        // (3) global start of the tile's run of digit d: the totals of the smaller digits plus the
        // counts of digit d in the tiles before this one
        {
            const uint32_t start = block_excl_scan_u32(__ldcg(totals + threadIdx.x), &s_tot);
            gofs[threadIdx.x] = start + __ldcg(counts + (int64_t)threadIdx.x * nb + t);
        }
#pragma unroll
        for (int it = 0; it < ITEMS; it++) {
            const int64_t idx = wbase + it * 32 + lane;
            if (idx < n) {
                const unsigned d = (unsigned)(k[it] >> shift) & (RADIX - 1);
                const uint32_t lp = bstart[d] + mycnt[d] + rank[it];
                skey[lp] = k[it];
                sval[lp] = v[it];
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += RS_THREADS) {
            const uint64_t key = skey[i];
            const unsigned d = (unsigned)(key >> shift) & (RADIX - 1);
            const int64_t g = (int64_t)gofs[d] + (i - (int64_t)bstart[d]);
            keys[g] = key;
            vals[g] = sval[i];
        }
        if (p + 1 < passes && !grid_barrier(bar, ++target, err)) return;  // the kernel's end orders the last
    }
}

// keys per thread: the largest of 8, 4, 2 that still gives at least one tile per SM (the SM
// count of this part; the count only changes the choice, not the result).  16 keys per thread
// would need 127 registers, two CTAs per SM: the 6.3 M-key sort of the knot tube ran its scatter
// passes faster with 8.
int rs_items(int64_t n) {
    for (int items = 8; items > 2; items >>= 1)
        if ((n + RS_THREADS * items - 1) / (RS_THREADS * items) >= 152) return items;
    return 2;
}

template <int ITEMS>
cudaError_t rs_passes(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, int64_t n, int bits,
                      void *tmp, void *scan_state, cudaStream_t s, unsigned *err) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_rs_scatter<ITEMS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)rs_smem<ITEMS>());
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    constexpr int TILE = RS_THREADS * ITEMS;
    int64_t nb = (n + TILE - 1) / TILE;
    uint32_t *hist = reinterpret_cast<uint32_t *>(tmp);
    int passes = (bits + 7) / 8;
    uint64_t *ki = keys, *ko = keys_alt;
    uint32_t *vi = vals, *vo = vals_alt;
    for (int p = 0; p < passes; p++) {
        int shift = 8 * p;
        cudaError_t e = launch_dep(k_rs_hist<ITEMS>, dim3((unsigned)nb), dim3(RS_THREADS), 0, s,
                                   (const uint64_t *)ki, n, shift, hist, nb);
        if (e != cudaSuccess) return e;
        e = scan_exclusive_u32(hist, hist, nb * RADIX, false, scan_state, s, err);
        if (e != cudaSuccess) return e;
        e = launch_dep(k_rs_scatter<ITEMS>, dim3((unsigned)nb), dim3(RS_THREADS), rs_smem<ITEMS>(), s,
                       (const uint64_t *)ki, (const uint32_t *)vi, ko, vo, n, shift, (const uint32_t *)hist, nb);
        if (e != cudaSuccess) return e;
        uint64_t *tk = ki; ki = ko; ko = tk;
        uint32_t *tv = vi; vi = vo; vo = tv;
    }
    if (ki != keys) {
        cudaError_t e = cudaMemcpyAsync(keys, ki, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(vals, vi, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// CTAs of k_rs_one<ITEMS> that the current device can hold at once (0 where it has no cooperative
// launch), found once per device
template <int ITEMS>
cudaError_t rs_one_capacity(int64_t *cap) {
    static std::atomic<int> known[64];  // static storage: starts at 0, "not yet known"
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    int c = known[dev].load(std::memory_order_relaxed);
    if (c == 0) {
        int per_sm = 0, n_sm = 0, coop = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rs_one<ITEMS>, RS_THREADS, rs_one_smem<ITEMS>());
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        if (e != cudaSuccess) return e;
        c = coop && per_sm > 0 ? per_sm * n_sm : -1;
        known[dev].store(c, std::memory_order_relaxed);
    }
    *cap = c > 0 ? c : 0;
    return cudaSuccess;
}

// The one-launch sort when its tiles fit on the device at once (*ran set), else nothing.
template <int ITEMS>
cudaError_t rs_one(uint64_t *keys, uint32_t *vals, int64_t n, int bits, void *tmp, void *scan_state, cudaStream_t s,
                   unsigned *err, bool *ran) {
    *ran = false;
    constexpr int TILE = RS_THREADS * ITEMS;
    const int64_t nb = (n + TILE - 1) / TILE;
    int64_t cap = 0;
    cudaError_t e = rs_one_capacity<ITEMS>(&cap);
    if (e != cudaSuccess || nb > cap) return e;
    uint32_t *counts = reinterpret_cast<uint32_t *>(tmp);
    uint32_t *totals = counts + nb * RADIX;
    unsigned *bar = reinterpret_cast<unsigned *>(scan_state) + 2;  // words 2 and 3 of the scan state
    int passes = (bits + 7) / 8;
    void *args[] = {&keys, &vals, &n, &passes, &counts, &totals, &bar, &err};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_rs_one<ITEMS>), dim3((unsigned)nb),
                                    dim3(RS_THREADS), args, rs_one_smem<ITEMS>(), s);
    if (e == cudaErrorCooperativeLaunchTooLarge) {  // not resident at once after all: the launches per pass
        (void)cudaGetLastError();
        return cudaSuccess;
    }
    if (e != cudaSuccess) return e;
    SDF_LAUNCHED(1);
    *ran = true;
    return cudaSuccess;
}
}  // namespace

// histograms of a sort of at most n keys: sized for the smallest tile (the most tiles), so that
// they also hold those of any shorter sort, whatever tile size that one picks
size_t radix_tmp_bytes(int64_t n) {
    const int64_t tile = (int64_t)RS_THREADS * 2;
    int64_t nb = (n + tile - 1) / tile;
    return ((size_t)nb * RADIX + RADIX + 64) * sizeof(uint32_t);  // + the one-launch sort's digit totals
}

// the scan state a sort of at most n keys needs (its digit histograms are scanned)
size_t radix_scan_state_bytes(int64_t n) {
    const int64_t tile = (int64_t)RS_THREADS * 2;
    return scan_state_bytes(((n + tile - 1) / tile) * RADIX);
}

cudaError_t radix_sort_u64(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, int64_t n,
                           int bits, void *tmp, void *scan_state, cudaStream_t s, unsigned *err) {
    if (n <= 1 || bits <= 0) return cudaSuccess;
    const int items = rs_items(n);
    // SDF_RADIX_ONE_LAUNCH=0 keeps every sort on the launches per pass (the two give the same order)
    const char *env = getenv("SDF_RADIX_ONE_LAUNCH");
    if (!(env && env[0] == '0')) {
        bool ran = false;
        const cudaError_t e =
            items == 8 ? rs_one<8>(keys, vals, n, bits, tmp, scan_state, s, err, &ran)
                       : (items == 4 ? rs_one<4>(keys, vals, n, bits, tmp, scan_state, s, err, &ran)
                                     : rs_one<2>(keys, vals, n, bits, tmp, scan_state, s, err, &ran));
        if (e != cudaSuccess || ran) return e;
    }
    switch (items) {
    case 8: return rs_passes<8>(keys, vals, keys_alt, vals_alt, n, bits, tmp, scan_state, s, err);
    case 4: return rs_passes<4>(keys, vals, keys_alt, vals_alt, n, bits, tmp, scan_state, s, err);
    default: return rs_passes<2>(keys, vals, keys_alt, vals_alt, n, bits, tmp, scan_state, s, err);
    }
}

}  // namespace sdf

// ============================================================================= launch counter
namespace sdf {
static std::atomic<int64_t> g_launches{0};
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
bool pdl_enabled() {
    static const bool on = [] {
        const char *e = getenv("SDF_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}
}  // namespace sdf
extern "C" int64_t sdf_kernel_launches(void) { return sdf::g_launches.load(); }

// ============================================================================= memory pool
namespace sdf {
static cudaMemPool_t g_pools[64] = {nullptr};
static std::mutex g_pool_mu;  // guards the creation of the per-device pools
static std::atomic<int64_t> g_pool_allocs{0}, g_host_allocs{0};
void count_host_alloc() { g_host_allocs.fetch_add(1, std::memory_order_relaxed); }

static cudaMemPool_t pool_for_current_device(cudaError_t *err) {
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        *err = cudaMemPoolCreate(&pool, &props);
        if (*err != cudaSuccess) return nullptr;
        uint64_t threshold = ~0ull;  // keep freed blocks cached in the pool
        *err = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
        if (*err != cudaSuccess) return nullptr;
        g_pools[dev] = pool;
    }
    return g_pools[dev];
}

cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s) {
    cudaError_t e;
    cudaMemPool_t pool = pool_for_current_device(&e);
    if (!pool) return e;
    g_pool_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMallocFromPoolAsync(p, bytes > 0 ? bytes : 1, pool, s);
}

cudaError_t pool_free(void *p, cudaStream_t s) { return p ? cudaFreeAsync(p, s) : cudaSuccess; }
}  // namespace sdf

extern "C" int sdf_memory_stats(int64_t *out) {
    using namespace sdf;
    if (!out) return SDF_ERR_INVALID_ARG;
    out[0] = g_pool_allocs.load();
    out[1] = out[2] = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
        cudaMemPool_t pool = nullptr;
        {
            std::lock_guard<std::mutex> lk(g_pool_mu);
            pool = g_pools[dev];
        }
        if (pool) {
            uint64_t used = 0, reserved = 0;
            if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess ||
                cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) != cudaSuccess)
                return SDF_ERR_CUDA;
            out[1] = (int64_t)used;
            out[2] = (int64_t)reserved;
        }
    }
    out[3] = g_host_allocs.load();
    return SDF_OK;
}

// ----------------------------------------------------------------------------- small reads
namespace sdf {
namespace {
constexpr int MAX_READS = 4;
constexpr unsigned MAX_READ_BYTES = 1024;
struct SmallReads {
    const unsigned char *src[MAX_READS];
    unsigned bytes[MAX_READS];
    unsigned off[MAX_READS];
    int n;
};
__global__ void k_read_small(SmallReads r, unsigned char *out) {
    dep_wait();
    dep_next();
    for (int i = 0; i < r.n; i++)
        for (unsigned b = threadIdx.x; b < r.bytes[i]; b += blockDim.x) out[r.off[i] + b] = r.src[i][b];
}
std::mutex g_small_mu;
std::vector<unsigned char *> g_small_free;  // pinned blocks of MAX_READ_BYTES
}  // namespace

cudaError_t read_small(const HostRead *reads, int n, cudaStream_t s) {
    if (n < 1 || n > MAX_READS) return cudaErrorInvalidValue;
    SmallReads r;
    r.n = n;
    unsigned total = 0;
    for (int i = 0; i < n; i++) {
        r.src[i] = static_cast<const unsigned char *>(reads[i].src);
        r.bytes[i] = reads[i].bytes;
        r.off[i] = total;
        total += (reads[i].bytes + 15u) & ~15u;
    }
    if (total > MAX_READ_BYTES) return cudaErrorInvalidValue;
    unsigned char *buf = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_small_mu);
        if (!g_small_free.empty()) {
            buf = g_small_free.back();
            g_small_free.pop_back();
        }
    }
    cudaError_t e = cudaSuccess;
    if (!buf) {
        e = cudaMallocHost(reinterpret_cast<void **>(&buf), MAX_READ_BYTES);
        count_host_alloc();
    }
    if (e != cudaSuccess) return e;
    // pinned host memory is device-addressable (unified addressing)
    e = launch_dep(k_read_small, dim3(1), dim3(128), 0, s, r, buf);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess)
        for (int i = 0; i < n; i++) memcpy(reads[i].dst, buf + r.off[i], reads[i].bytes);
    std::lock_guard<std::mutex> lk(g_small_mu);
    g_small_free.push_back(buf);
    return e;
}
}  // namespace sdf
