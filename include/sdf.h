/*
 * sdf.h -- C ABI of the GB300 narrow-band signed distance field library
 * (Characteristic/Scan Conversion method, Roosing, Strickson & Nikiforakis,
 * "Fast Distance Fields for Fluid Dynamics Mesh Generation on Graphics
 * Hardware", arXiv:1903.00353).
 *
 * Problem statement (Section 6, Section 7): the input is a closed, oriented
 * triangulated surface whose triangles list their vertices counter-clockwise
 * seen from outside, with no gaps, overlaps or flipped faces.  The output is
 * the signed distance (interior negative, Section 3.1) at every cell centre of
 * a logically Cartesian grid that lies within a user-given distance w of the
 * surface (Section 9, Section 10); every other cell holds +infinity
 * (Algorithm 1 starts from d = infinity).
 *
 * Conventions for every call:
 *   - Pointers are DEVICE pointers unless marked "host".  Float data is FP32.
 *   - Calls are asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *     default stream) unless stated otherwise; they may synchronise `stream`
 *     once to read a device status word or a size.
 *   - The caller owns every input and output buffer.  The library owns the
 *     sdf_features handle and the scratch memory cached in it, released by
 *     sdf_features_destroy.  No call keeps a pointer to caller memory after it
 *     returns.
 *   - Every call returns an sdf_status; no exception crosses the ABI.  On an
 *     error the outputs are unspecified.
 *   - Calls on one handle must not overlap in time (they share its scratch).
 *   - The library's short kernels (the build, the scans, the narrow band's
 *     set-up and FP64 re-decision) are launched as programmatic dependent
 *     launches: each may be scheduled while its predecessor on `stream` runs
 *     and waits on the device for it, so stream order is kept.  The
 *     environment variable SDF_PDL=0 launches them plainly.
 *
 * Grid layout (Section 10, a row-major 1D float array): point (i,j,k) sits at
 * origin + ((i+1/2) h, (j+1/2) h, (k0+k+1/2) h) and is stored at
 * i + nx*(j + ny*k) (x fastest); k0 = 0 except for a z-slab of a larger grid.
 *
 * Feature ids (Section 2: faces, edges and vertices are the features):
 *   face f in [0, T); edge e -> T + e; vertex v -> T + E + v,
 * with T triangles, E = 3T/2 unique edges and V unique vertices.  Faces,
 * edges and vertices are numbered in a spatial (Morton) order chosen by the
 * library; sdf_features_face_map and sdf_features_vertex_map relate them to
 * the soup.  Winner ids name the feature whose characteristic region produced
 * the stored value; -1 outside the band.
 */
#ifndef GB300_SDF_H
#define GB300_SDF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sdf_status {
    SDF_OK = 0,
    SDF_ERR_INVALID_ARG = 1,  /* null pointer, negative size, bad grid, w <= 0             */
    SDF_ERR_NONMANIFOLD = 2,  /* an edge is not shared by exactly two oppositely directed
                                 triangle edges: open, non-manifold or inconsistently
                                 oriented surface (Section 6 assumes a closed surface)     */
    SDF_ERR_DEGENERATE = 3,   /* zero-area triangle or zero-length edge (Section 4)        */
    SDF_ERR_NONFINITE = 4,    /* NaN or infinite coordinate                               */
    SDF_ERR_TOO_LARGE = 5,    /* sizes beyond the index ranges (2^31 features, 2^31 rows)  */
    SDF_ERR_OOM = 6,          /* device allocation failed                                 */
    SDF_ERR_CUDA = 7,         /* a CUDA runtime call failed                               */
    SDF_ERR_TIMEOUT = 8,      /* a bounded device wait gave up (a look-back or a barrier) */
    SDF_ERR_LIST_OVERFLOW = 9 /* the caller's band list holds fewer entries than the band
                                 has points; its count holds the length needed             */
} sdf_status;

/* Grid description (host struct, passed by pointer).  k0 places the grid inside a larger one
 * along z (a z-slab of it): point (i,j,k) sits at origin + ((i+1/2) h, (j+1/2) h, (k0+k+1/2) h) and
 * is stored at i + nx*(j + ny*k).  A slab with the same origin, h and a first layer k0 that is a
 * multiple of 8 gives bitwise the values of those layers of the whole grid, whatever h is. */
typedef struct sdf_grid {
    int32_t nx, ny, nz;  /* points per axis, each >= 1                        */
    float origin[3];     /* lower corner of the (whole) grid box              */
    float h;             /* cell size > 0                                     */
    int32_t k0;          /* index of the first z layer, >= 0 (0: the whole grid) */
} sdf_grid;

/* Opaque, library-owned feature set of one mesh. */
typedef struct sdf_features_s *sdf_features;

/* Flags for sdf_build_features / sdf_narrow_band. */
#define SDF_FLAG_DISABLE_SADDLE 0x1u /* debug ablation (Section 11.1, Fig. ear): give saddle
                                        vertices no extrusion; the field then has gaps      */
#define SDF_FLAG_NO_SYNC 0x2u        /* sdf_narrow_band: skip the final status read; call
                                        sdf_features_status later (needed inside graphs)     */
#define SDF_FLAG_TIMING 0x4u         /* record CUDA events on `stream` around the stages of
                                        sdf_narrow_band(_list) and the adjoints; no call waits
                                        for them: sdf_features_timing (or the next timed call
                                        on the handle) reads them                            */
#define SDF_FLAG_AUTOTUNE 0x8u       /* sdf_batch_create: time every tile shape on the batch
                                        and keep the fastest (also remembered for later
                                        sdf_narrow_band calls with n > 1 of the same sizes)  */
#define SDF_FLAG_FILL_SIGN 0x10u     /* sdf_narrow_band / sdf_batch_create: points outside the
                                        band get -inf inside the surface and +inf outside
                                        (the sign fill beyond the band, Section 11.3);
                                        requires w > h and k0 = 0 on every grid              */
#define SDF_FLAG_CELL_LOOP 0x20u     /* sdf_narrow_band / sdf_batch_create: run the paper's own
                                        schedule (Section 9: one thread per characteristic
                                        region walking its box, a global 64-bit atomicMin per
                                        grid point, then a decode pass) instead of the binned
                                        tile kernel; same regions, distances and FP64
                                        re-decision.  For the schedule comparison; needs
                                        8 bytes of scratch per grid point                    */
#define SDF_FLAG_VERTEX_CONE 0x40u   /* with SDF_FLAG_CELL_LOOP: the paper's vertex extrusions
                                        (Sections 3.3, 8.3): a cone of height w around N_alpha
                                        opening to the most diverging face normal on the
                                        positive side; convex vertices the positive cone,
                                        concave the negative one, saddles both.  For the
                                        coverage comparison: the paper leaves its correctness
                                        open (Section 11.1), so gaps are possible            */
#define SDF_FLAG_VERTEX_HEMISPHERE 0x80u /* with SDF_FLAG_CELL_LOOP: half-balls on the N_alpha
                                        and -N_alpha sides (Section 4.3), same class rule    */
#define SDF_FLAG_GRAD_F64 0x100u     /* the adjoints (sdf_narrow_band_backward, sdf_band_list_backward,
                                        sdf_band_list_l2): grad_vertices points to double[V][3] and
                                        the per-point contributions (FP32) are summed in FP64, for
                                        comparisons where the order of FP32 atomics would blur the
                                        result                                               */

/*
 * sdf_build_features -- mesh-connectivity stage (Section 7, Section 8).
 *
 * From an unordered triangle soup, welds equal vertices by sorting (Section
 * 7.2; "identical" read as bitwise-equal FP32 coordinates, -0 == +0), pairs
 * the two directed copies of every edge (Section 7.1), and builds the face,
 * edge and vertex records: unit face normals, edge convexity
 * d = (ab x n1) . n2 (Section 8.2), angle-weighted pseudonormals
 * N_alpha = sum alpha_i n_i (Eq. 8) and the convex / concave / flat / saddle
 * class of every vertex (Section 3.1, Section 3.2, Section 8.3).
 *
 *   soup   device float[n_tri][3][3], corners counter-clockwise seen from
 *          outside; read only during the call.
 *   n_tri  number of triangles, 1 <= n_tri < 2^28.
 *   flags  0 or SDF_FLAG_DISABLE_SADDLE.
 *   out    host pointer receiving the new handle (NULL on error).
 *
 * Synchronises `stream` twice (the welded vertex count; the sizes and the
 * status word at the end).  The two sorts (the weld's and the spatial face
 * order) each run in one cooperative launch when their tiles fit on the
 * device at once, else in three launches per 8-bit pass; the environment
 * variable SDF_RADIX_ONE_LAUNCH=0 selects the latter always (both give the
 * same result).  Errors: SDF_ERR_INVALID_ARG, SDF_ERR_NONFINITE,
 * SDF_ERR_DEGENERATE, SDF_ERR_NONMANIFOLD, SDF_ERR_TOO_LARGE, SDF_ERR_OOM,
 * SDF_ERR_CUDA, SDF_ERR_TIMEOUT (a bounded device wait of a scan or a sort
 * ran out).
 */
int sdf_build_features(const float *soup, int64_t n_tri, uint32_t flags, void *stream, sdf_features *out);

/*
 * sdf_features_update_positions -- re-evaluate the geometry of an existing
 * handle for new welded vertex positions (same connectivity): normals,
 * pseudonormals, classification and extrusion records (Section 8).  Used by
 * shape optimisation, where only the positions change between steps.
 *
 *   vertices  device float[V][3] in the handle's vertex order (see
 *             sdf_features_vertices / sdf_features_vertex_map).
 * Errors: SDF_ERR_INVALID_ARG, SDF_ERR_CUDA; a zero-area triangle at the new
 * positions is reported as SDF_ERR_DEGENERATE by the next synchronising
 * sdf_narrow_band or sdf_features_status call.
 */
int sdf_features_update_positions(sdf_features f, const float *vertices, void *stream);

/*
 * sdf_narrow_band -- extrusion, scan conversion and merge (Sections 5, 8, 9,
 * 10; Algorithm 1 and Algorithm 2).
 *
 * For every feature, builds its characteristic region clipped to distance w
 * (face prism, edge wedge, vertex region), finds the grid points inside it
 * row by row (half-space tests against the region's planes, Algorithm 2),
 * computes the distance of each point to the feature and its sign, and keeps
 * per point the value of smallest magnitude (Algorithm 1) through a packed
 * 64-bit atomicMin of (|d| bits, feature id).  Distances and scan conversion
 * run in FP32; points whose band membership or sign falls inside the FP32
 * error window are re-decided in FP64 from the winner's neighbourhood.
 *
 *   feats       host array [n] of handles.
 *   grids       host array [n] of grids.
 *   band_w      host array [n] of band half-widths w > 0 (a point is in the
 *               band iff |d| < w).
 *   n           number of (mesh, grid) problems; n > 1 runs them as one batch.
 *   out_dist    host array [n] of device float[nz][ny][nx] outputs.
 *   out_winner  host array [n] of device int32[nz][ny][nx] (winner feature
 *               id, -1 outside the band); the array or any entry may be NULL.
 *   flags       0, SDF_FLAG_NO_SYNC, SDF_FLAG_TIMING, SDF_FLAG_FILL_SIGN, SDF_FLAG_CELL_LOOP
 *               (any combination), and with SDF_FLAG_CELL_LOOP one of SDF_FLAG_VERTEX_CONE,
 *               SDF_FLAG_VERTEX_HEMISPHERE.
 *               With SDF_FLAG_FILL_SIGN, points outside the band hold -inf inside the
 *               surface and +inf outside (Section 11.3's fill beyond the band): along each
 *               x-row a run of points outside the band takes the sign of the band point
 *               next to it, and a row without band points the sign of a neighbouring row
 *               (exact whenever w > h; a grid without any band point is taken as outside).
 *
 * Errors: SDF_ERR_INVALID_ARG (also w <= h with SDF_FLAG_FILL_SIGN), SDF_ERR_TOO_LARGE,
 * SDF_ERR_OOM, SDF_ERR_CUDA, SDF_ERR_DEGENERATE (positions set by
 * sdf_features_update_positions).
 */
int sdf_narrow_band(const sdf_features *feats, const sdf_grid *grids, const float *band_w, int32_t n,
                    float *const *out_dist, int32_t *const *out_winner, uint32_t flags, void *stream);

/*
 * sdf_narrow_band_backward -- adjoint of the narrow band with respect to the
 * welded vertex positions (a project addition; the paper has no adjoint).
 *
 * For L with upstream gradient g = dL/dd on the grid, every band point p with
 * winner feature F and closest point q = sum_k lam_k x_k on F (barycentric on a
 * face, (1-t, t) on an edge, 1 at a vertex) contributes
 *     dL/dx_k += -g(p) * s(p) * lam_k * (p - q)/|p - q|,
 * s = sign d(p): the envelope theorem applied to d = s * min |p - q| (Eq. 1).
 *
 *   grad_dist      host array [n] of device float[nz][ny][nx] (dL/dd).
 *   winner         host array [n] of device int32 winners from the forward, or
 *                  NULL (array or entry) to recompute them.
 *   grad_vertices  host array [n] of device float[V][3] (double[V][3] with
 *                  SDF_FLAG_GRAD_F64); ACCUMULATED into (the caller zeroes it first).
 * Errors: SDF_ERR_INVALID_ARG, SDF_ERR_OOM, SDF_ERR_CUDA.
 */
int sdf_narrow_band_backward(const sdf_features *feats, const sdf_grid *grids, const float *band_w, int32_t n,
                             const float *const *grad_dist, const int32_t *const *winner,
                             float *const *grad_vertices, uint32_t flags, void *stream);

/*
 * sdf_features_info -- sizes and classification counts (host outputs, any may
 * be NULL).  Table 2 of the paper reports total, unique and saddle vertices.
 *   counts[0..7] = V, E, convex vertices, concave vertices, flat vertices,
 *                  saddle vertices, convex edges, concave edges.
 */
int sdf_features_info(sdf_features f, int64_t *n_tri, int64_t *counts /* host [8] */);

/* Welded vertex id of every soup corner: device int32[3*n_tri]. */
int sdf_features_vertex_map(sdf_features f, int32_t *soup_to_vertex, void *stream);

/* Soup triangle of every library face id: device int32[n_tri]. */
int sdf_features_face_map(sdf_features f, int32_t *face_to_soup, void *stream);

/* Edge table: device int32[E][4] = (va, vb, f1, f2) per library edge id e: the welded end
 * points va < vb, the face f1 holding the directed edge va -> vb and the face f2 holding vb -> va
 * (library face ids).  Relates edge winners (feature id T + e) to the mesh. */
int sdf_features_edges(sdf_features f, int32_t *edges, void *stream);

/*
 * sdf_features_error_bound -- the FP32 error windows the narrow band uses for this mesh at its
 * current positions on the given grid and band (host outputs, synchronises `stream`):
 *   bounds[0] delta: bound on | |d_fp32| - |d| | for every FP32 distance the tile kernel keeps,
 *             delta = (2^-20 M + tau_a + tau_b w) / (1 - 2 tau_b), M the largest coordinate
 *             magnitude of the grid and the mesh, tau_a, tau_b the mesh's normal-error terms;
 *   bounds[1] the inclusion tolerance of the region tests (world units);
 *   bounds[2] the sign window: a candidate whose sign predicate is within it of zero is
 *             re-decided in FP64;
 *   bounds[3] the largest extra sign-window term of the edge and vertex pseudonormals.
 * A point whose FP32 distance lies within delta of w, or whose sign is uncertain, is re-decided
 * in FP64, so the band mask and the sign are exact elsewhere and |d| errs by at most delta.
 * Errors: SDF_ERR_INVALID_ARG, SDF_ERR_CUDA.
 */
int sdf_features_error_bound(sdf_features f, const sdf_grid *grid, float band_w, double *bounds, void *stream);

/* Welded vertex positions: device float[V][3]. */
int sdf_features_vertices(sdf_features f, float *out, void *stream);

/*
 * Status word and counters of the last single-problem (n = 1) sdf_narrow_band on this handle
 * (synchronises `stream`).  stats (host, nullable) [6] = candidate (point,
 * region) pairs merged by atomicMin, band points decided in FP32, points
 * re-decided in FP64, (tile, region) pairs scheduled, grid rows intersected
 * with a region, of which non-empty.
 * Errors: those of the call, among them SDF_ERR_OOM when a call made with SDF_FLAG_NO_SYNC
 * outgrew its scratch.  A synchronising call grows the scratch (the (tile, region) pair list and
 * the FP64 re-decision list) and repeats its launch when it overflows; a call with
 * SDF_FLAG_NO_SYNC cannot, so its first capacities are sized from the mesh: the expected pairs
 * of the grid, from the build's sums of the faces' bounding-box extents, with a quarter to spare
 * and at least 8 per feature.  The environment variable SDF_PAIR_CAPACITY, when set to a
 * positive count, replaces the first capacity of the pair list (for testing the growth path).
 */
int sdf_features_status(sdf_features f, int64_t *stats, void *stream);

/*
 * Accumulated device time (milliseconds, from CUDA events recorded on the calls' stream) of the
 * stages of calls made with SDF_FLAG_TIMING, and the number of timed calls:
 *   ms[0] binning (region boxes -> tiles), ms[1] tile kernel (scan conversion, merge and the
 *   dense write), ms[2] FP64 re-decision, ms[3] adjoint kernel.  Host outputs [4], nullable.
 * reset != 0 zeroes the accumulators after reading.
 */
int sdf_features_timing(sdf_features f, double *ms, int64_t *calls, int reset);

/* Process-wide number of CUDA kernels this library has launched (diagnostics). */
int64_t sdf_kernel_launches(void);

/*
 * Memory the library has taken (diagnostics; host outputs [4]): out[0] the number of device
 * allocations it has made from its stream-ordered pool (process-wide), out[1] and out[2] the
 * bytes in use and reserved in the current device's pool, out[3] the number of pinned host
 * allocations it has made (staging blocks for small reads and table uploads).
 * Errors: SDF_ERR_INVALID_ARG, SDF_ERR_CUDA.
 */
int sdf_memory_stats(int64_t *out);

/*
 * sdf_narrow_band_static -- the same narrow band as sdf_narrow_band for one (mesh, grid) problem,
 * but the call allocates no device memory.  The paper has no counterpart: this entry point is
 * for callers that cannot allocate during the call, such as a process whose device memory is
 * owned by another runtime or a fixed budget, or a latency-bound loop.
 *
 * Its scratch is one library-owned device array of about 20.3 MiB that every device holding
 * this library keeps until the process exits.  Limits: at most 65536 tiles of 32x8x8 points
 * (e.g. a 512^3 grid), 2097152 (tile, region) pairs and 131072 points re-decided in FP64;
 * beyond them the call returns SDF_ERR_TOO_LARGE (the grid limit before any work, the list
 * limits after it, with the outputs unspecified).
 *
 * All calls share the array, and each call clears what it needs at its start.  Two calls
 * whose work overlaps on the GPU (for example on two streams) race on it and must not be made.
 * The first call on a device performs the set-up (it looks up the array's device address with
 * that device current); make that first call before any stream capture.  The call
 * synchronises `stream` once to read its status words, by a copy into host stack memory: it
 * allocates neither device memory nor pinned host memory (sdf_memory_stats counts both).
 *
 *   f           handle from sdf_build_features.
 *   grid        host pointer to the grid.
 *   band_w      band half-width w > 0.
 *   out_dist    device float[nz][ny][nx].
 *   out_winner  device int32[nz][ny][nx] or NULL.
 * Errors: SDF_ERR_INVALID_ARG, SDF_ERR_TOO_LARGE, SDF_ERR_CUDA, SDF_ERR_DEGENERATE (positions set by
 * sdf_features_update_positions).
 */
int sdf_narrow_band_static(sdf_features f, const sdf_grid *grid, float band_w, float *out_dist,
                           int32_t *out_winner, void *stream);

/*
 * Batches for repeated evaluation -- the same computation as sdf_narrow_band with n problems,
 * split into a set-up call and a replayable launch (a project addition; the paper evaluates one
 * mesh at a time).
 *
 * sdf_batch_create describes the n (mesh, grid, output) problems, sizes and allocates all scratch
 * (the problem table, bins, the (tile, region) pair list, tile work lists and the FP64
 * re-decision list), runs the batch once (so the outputs hold the result on return) and, with
 * SDF_FLAG_AUTOTUNE, times the tile shapes 32x8x8, 32x4x4 and 32x16x8 and keeps the fastest.
 * It synchronises `stream`.  The handles, grids, widths and output pointers are fixed for the
 * batch's lifetime; the handles' positions may change (sdf_features_update_positions) as long
 * as the band stays within the scratch sized at creation.
 *
 * sdf_batch_run enqueues the whole batch on `stream`: a fixed sequence of kernels and memsets,
 * with no allocation, no host synchronisation and no host-to-device copy, so it may be captured
 * in a CUDA graph and replayed.  All problems share one persistent tile-kernel launch.
 *
 * sdf_batch_status (synchronises `stream`) returns the counters of the last run (layout of
 * sdf_features_status) and SDF_ERR_OOM if the band of that run outgrew the scratch sized at
 * creation (the outputs of that run are then unspecified; create a new batch).
 *
 * sdf_batch_info returns the tile shape in use (host int32[3], points per tile along x, y, z)
 * and the per-run time measured while autotuning (ms; 0 without SDF_FLAG_AUTOTUNE).
 *
 * sdf_batch_timing (batches created with SDF_FLAG_TIMING, which then record four CUDA events on
 * every run, as event nodes when captured in a graph) waits for the last run and returns its
 * stage times in ms (host float[3]): binning, tile kernel, FP64 re-decision.  Without the flag
 * it returns SDF_ERR_INVALID_ARG.
 *
 * Arguments of sdf_batch_create are those of sdf_narrow_band; flags 0 or any of
 * SDF_FLAG_AUTOTUNE, SDF_FLAG_TIMING, SDF_FLAG_FILL_SIGN.
 * Errors: SDF_ERR_INVALID_ARG, SDF_ERR_TOO_LARGE, SDF_ERR_OOM, SDF_ERR_CUDA, SDF_ERR_DEGENERATE.
 * sdf_batch_destroy synchronises the device and releases the batch (NULL is a no-op); the
 * handles outlive the batch and are not released by it.
 */
typedef struct sdf_batch_s *sdf_batch;
int sdf_batch_create(const sdf_features *feats, const sdf_grid *grids, const float *band_w, int32_t n,
                     float *const *out_dist, int32_t *const *out_winner, uint32_t flags, void *stream,
                     sdf_batch *out);
int sdf_batch_run(sdf_batch b, void *stream);
int sdf_batch_status(sdf_batch b, int64_t *stats, void *stream);
int sdf_batch_info(sdf_batch b, int32_t *tile_shape, double *tuned_ms);
int sdf_batch_timing(sdf_batch b, float *ms);
void sdf_batch_destroy(sdf_batch b);

/*
 * sdf_band_l2_loss -- the loss of the shape-fitting workload and its gradient in one pass (a project
 * addition; the paper has no loss): L = sum over band points (finite d) of (d - target)^2, written
 * to *loss_out (device double, overwritten), and dL/dd = 2 (d - target) on the band, 0 elsewhere,
 * written to grad_out (device float[n], nullable), ready for sdf_narrow_band_backward; the number
 * of band points to *band_out (device uint64, nullable, overwritten).
 *   dist, target  device float[n]; n >= 0 points.
 * No synchronisation.  Errors: SDF_ERR_INVALID_ARG, SDF_ERR_CUDA.
 */
int sdf_band_l2_loss(const float *dist, const float *target, int64_t n, float *grad_out, double *loss_out,
                     unsigned long long *band_out, void *stream);

/*
 * Compact band list (a project addition).  The dense field keeps one value per grid point, but
 * the band is a thin shell (a few percent of the points at 512^3); a list of the band points
 * lets a later pass (loss, adjoint) touch only them instead of streaming the whole grid again.
 * One entry per band point: its linear index (x fastest, as in the dense outputs) and its winner
 * feature id (the value the dense winner array holds there).
 */
typedef struct sdf_band_entry {
    uint32_t idx;    /* point index k * ny * nx + j * nx + i */
    int32_t winner;  /* winning feature: face t, edge T + e, or vertex T + E + v */
} sdf_band_entry;

/*
 * sdf_narrow_band_list -- sdf_narrow_band for one problem that also writes the band as a compact
 * list (the tile kernel appends each tile's band points, the FP64 re-decision appends the points
 * it decides into the band).
 *   out_dist     device float[nz][ny][nx] (as sdf_narrow_band).
 *   out_winner   device int32[nz][ny][nx] or NULL (the list carries the winners).
 *   list         device sdf_band_entry[list_cap]; entries in no particular order (tiles finish in
 *                any order), each band point exactly once.
 *   list_count   device uint64, overwritten with the number of band points (also when that
 *                exceeds list_cap; entries from list_cap on are then not written).
 *   flags        as sdf_narrow_band, but not SDF_FLAG_CELL_LOOP.
 * The grid must have at most 2^32 - 1 points.  With SDF_FLAG_NO_SYNC an overflow of the list is
 * reported by the next sdf_features_status.
 * Errors: those of sdf_narrow_band, and SDF_ERR_LIST_OVERFLOW.
 */
int sdf_narrow_band_list(sdf_features f, const sdf_grid *grid, float band_w, float *out_dist,
                         int32_t *out_winner, sdf_band_entry *list, int64_t list_cap,
                         unsigned long long *list_count, uint32_t flags, void *stream);

/*
 * sdf_narrow_band_sparse -- the narrow band of one problem as the compact band list alone, with no
 * dense field (a project addition: the paper writes the dense row-major array, Section 10).  Each
 * band point is listed once, with its signed distance in list_dist at the same position; nothing
 * is written for the points outside the band, so the output costs 12 bytes per band point
 * instead of 4 bytes per grid point.  The same tile kernel, merge and FP64 re-decision as
 * sdf_narrow_band_list.
 *   list        device sdf_band_entry[list_cap] (as sdf_narrow_band_list).
 *   list_dist   device float[list_cap]: the signed distance of entry i.
 *   list_count  device uint64, overwritten with the number of band points.
 *   flags       0, SDF_FLAG_NO_SYNC, SDF_FLAG_TIMING (not SDF_FLAG_CELL_LOOP or SDF_FLAG_FILL_SIGN).
 * The grid must have at most 2^32 - 1 points.
 * Errors: those of sdf_narrow_band_list.
 */
int sdf_narrow_band_sparse(sdf_features f, const sdf_grid *grid, float band_w, sdf_band_entry *list,
                           float *list_dist, int64_t list_cap, unsigned long long *list_count, uint32_t flags,
                           void *stream);

/*
 * sdf_narrow_band_lists -- the same for n problems in one batch (as sdf_narrow_band with n > 1:
 * one persistent tile launch over all problems, synchronous): problem p writes its field to
 * out_dist[p] and its band list to lists[p] (list_caps[p] entries, length to *list_counts[p],
 * point indices within its own grid).  out_winner as for sdf_narrow_band (nullable).  A list that
 * is too short makes the call return SDF_ERR_LIST_OVERFLOW; every count still holds the length
 * its problem needs.
 * Errors: those of sdf_narrow_band, and SDF_ERR_LIST_OVERFLOW.
 */
int sdf_narrow_band_lists(const sdf_features *feats, const sdf_grid *grids, const float *band_w, int32_t n,
                          float *const *out_dist, int32_t *const *out_winner, sdf_band_entry *const *lists,
                          const int64_t *list_caps, unsigned long long *const *list_counts, uint32_t flags,
                          void *stream);

/*
 * sdf_band_list_backward -- the adjoint of sdf_narrow_band_backward over the entries of a band
 * list: grad_vertices += sum over entries e of g(idx_e) * d d(p) / d X at p = point idx_e with
 * winner winner_e (the same per-point contribution as sdf_narrow_band_backward).
 *   list, list_cap, list_count  as written by sdf_narrow_band_list (min(count, cap) entries used;
 *                                the count is read on the device, so the call never synchronises).
 *   grad_dist      device float[nz][ny][nx] (dL/dd; read at the listed points only).
 *   grad_vertices  device float[V][3] (double[V][3] with SDF_FLAG_GRAD_F64), ACCUMULATED into.
 * Errors: SDF_ERR_INVALID_ARG, SDF_ERR_TOO_LARGE (a grid of more than 2^32 - 1 points),
 * SDF_ERR_CUDA.
 */
int sdf_band_list_backward(sdf_features f, const sdf_grid *grid, const sdf_band_entry *list, int64_t list_cap,
                           const unsigned long long *list_count, const float *grad_dist, float *grad_vertices,
                           uint32_t flags, void *stream);

/*
 * sdf_band_list_l2 -- the loss of the shape-fitting workload and its vertex gradient in one pass
 * over a band list: L = sum over the listed points of (d - target)^2 with d = dist[idx] (the same
 * L as sdf_band_l2_loss), dL/dX = sum of 2 (d - target) d d / d X accumulated into grad_vertices
 * (float[V][3], or double[V][3] with SDF_FLAG_GRAD_F64), without a dense gradient field.
 *   dist, target   device float[nz][ny][nx] (read at the listed points only).
 *   loss_out       device double, overwritten (FP64 sum of the FP32 squared differences).
 *   band_out       device uint64 or NULL, overwritten with the number of listed points used.
 * No synchronisation.  Errors: SDF_ERR_INVALID_ARG, SDF_ERR_TOO_LARGE (as above), SDF_ERR_CUDA.
 */
int sdf_band_list_l2(sdf_features f, const sdf_grid *grid, const sdf_band_entry *list, int64_t list_cap,
                     const unsigned long long *list_count, const float *dist, const float *target,
                     float *grad_vertices, double *loss_out, unsigned long long *band_out, uint32_t flags,
                     void *stream);

/* Release the handle and its device memory (NULL is a no-op).  Waits for the device.  The scratch
 * of its narrow-band calls (pair list, bins, tile lists) is kept for the next handle's first call
 * on the same device, at most two such sets per device, and its array block and counters for the
 * next sdf_build_features on the device (with the builds' own scratch, at most four blocks per
 * device): a loop that builds a handle per step then takes no memory from the pool per step. */
void sdf_features_destroy(sdf_features f);

/* Static description of a status code. */
const char *sdf_status_string(int status);

/*
 * sdf_probe_rate -- one launch of a rate probe for the roofline of the narrow band (a measurement
 * helper with no counterpart in the paper).  The merge of Algorithm 1 is a 64-bit atomicMin of
 * the packed key (|d|, feature id): in shared memory in the tile kernel, in global memory in the
 * paper's own schedule (Section 9, one thread per region walking its cells); the filtered
 * re-decision runs in FP64.  The launch runs 4 CTAs of 256 threads per SM, each thread `iters`
 * steps, on `stream`, with no synchronisation; the caller times it (CUDA events on the same
 * stream) and divides *ops by the time.
 *
 *   kind     SDF_PROBE_SMEM_ATOMIC_MIN: atomicMin(u64) on a 32 KB shared-memory array per CTA,
 *            lane l of a warp on word l + 32 m; buf: device uint64[n_words], n_words >= the
 *            number of CTAs (one result word per CTA is written).
 *            SDF_PROBE_GLOBAL_ATOMIC_MIN: atomicMin(u64) on pseudo-random words of buf, device
 *            uint64[n_words] with n_words a power of two (within L2 or larger than L2); its
 *            contents are overwritten with smaller values.
 *            SDF_PROBE_FP64_FMA: FP64 fused multiply-adds, 8 independent chains per thread;
 *            buf: device double[n_words], n_words >= 1 (not written in practice).
 *   iters    steps per thread, >= 1.
 *   ops      host int64, set to the launch's operation count (atomics, or FP64 flops).
 * Errors: SDF_ERR_INVALID_ARG, SDF_ERR_CUDA.
 */
enum { SDF_PROBE_SMEM_ATOMIC_MIN = 0, SDF_PROBE_GLOBAL_ATOMIC_MIN = 1, SDF_PROBE_FP64_FMA = 2 };
int sdf_probe_rate(int32_t kind, void *buf, int64_t n_words, int64_t iters, int64_t *ops, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GB300_SDF_H */
