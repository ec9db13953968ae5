/*
 * FP64 CPU oracle for the narrow-band signed distance field of a closed,
 * oriented triangle mesh.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and
 * bench.py's CPU-baseline / reference leg may load or call this library.  It
 * shares no code with the CUDA path (no headers, helpers or tables).
 *
 * What it computes is the plain definition, written out:
 *
 *   d(p) = s(p) * min_t dist(p, triangle_t)                 (Eq. 1, Section 2)
 *
 * in double precision on the float32 input values promoted exactly.  The
 * minimum over triangles is a literal loop (ties go to the lowest triangle
 * index).  The sign follows the paper's convention (interior negative,
 * Section 3.1) and is taken from the pseudonormal of the feature that holds
 * the closest point q (Section 4.3, angle-weighted pseudonormal Eq. 8):
 *   q inside the triangle  -> the face normal,
 *   q inside an edge       -> n1 + n2 (the two incident face normals),
 *   q at a vertex          -> N_alpha = sum_i alpha_i n_i.
 * s = sign((p - q) . N).  A grid point is in the band iff |d| < w (Section 10,
 * "smaller than a user defined maximum"); outside the band the value is +inf
 * (Algorithm 1 initialises d = infinity).
 *
 * Sample points are cell centres origin + (i+1/2) h (Section 10), stored x
 * fastest: idx = i + nx*(j + ny*k).
 *
 * The only acceleration is an exact pruning of the triangle loop: triangles
 * are binned by bounding box into a uniform cell grid and cells are visited in
 * growing Chebyshev rings; the loop stops once a lower bound on the distance
 * to every unvisited triangle exceeds the best distance found (or the band
 * width).  Skipped triangles provably cannot win, and visited triangles are
 * compared in increasing index order with the same strict "<" as the literal
 * loop, so the result is bitwise that of the literal loop (checked by tests).
 *
 * Mesh connectivity (Section 7): soup vertices with equal coordinates are
 * welded (qsort on the exact values; -0 == +0), and each directed edge must
 * meet exactly one opposite directed edge (closed 2-manifold), else an error.
 *
 * The adjoint (a project addition) is the envelope-theorem derivative of d = s |p - q(X)|
 * with respect to the welded vertices, either at each point's own closest feature
 * (om_adjoint_points) or at a feature the caller gives per point (om_adjoint_features), so
 * that another implementation's winners can be evaluated in FP64.
 *
 * Parity pins: see tests/test_oracle_*.py (exact-rational brute force,
 * closed forms of a box and a regular tetrahedron, Eikonal, translation and
 * rotation covariance, ray-parity inside test, finite differences).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_NONMANIFOLD 2
#define OR_ERR_DEGENERATE 3
#define OR_ERR_NONFINITE 4
#define OR_ERR_OOM 6

typedef struct {
    int64_t T, V, E;
    double *X;         /* [V][3] welded vertex positions                           */
    int32_t *tri;      /* [T][3] vertex ids, CCW seen from outside                 */
    int32_t *soup_vid; /* [3T] soup corner -> vertex id                            */
    double *fn;        /* [T][3] unit face normals                                 */
    int32_t *adj;      /* [T][3] face across the edge from corner k to corner k+1  */
    double *vn;        /* [V][3] angle-weighted pseudonormals (not normalised)     */
    int8_t *vclass;    /* [V] 1 convex, -1 concave, 0 flat, 2 saddle               */
    int8_t *eclass;    /* [T][3] per directed edge: 1 convex, -1 concave, 0 flat   */
    /* bin grid for the pruned search */
    double blo[3], bcs;
    int32_t bn[3];
    int64_t *bstart;   /* [ncells+1] */
    int32_t *bitems;   /* triangle ids, ascending inside each cell */
} om_mesh;

/* ------------------------------------------------------------------ small vector helpers */
static inline void v_sub(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static inline double v_dot(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void v_cross(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double v_norm(const double *a) { return sqrt(v_dot(a, a)); }

/* ------------------------------------------------------------------ welding (Section 7.2) */
typedef struct { double x, y, z; int64_t idx; } wrec;
static int wrec_cmp(const void *pa, const void *pb) {
    const wrec *a = (const wrec *)pa, *b = (const wrec *)pb;
    if (a->x != b->x) return a->x < b->x ? -1 : 1;
    if (a->y != b->y) return a->y < b->y ? -1 : 1;
    if (a->z != b->z) return a->z < b->z ? -1 : 1;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}

/* half-edge key for pairing (Section 7.1): (min vid, max vid) */
typedef struct { int64_t lo, hi; int64_t h; } erec;
static int erec_cmp(const void *pa, const void *pb) {
    const erec *a = (const erec *)pa, *b = (const erec *)pb;
    if (a->lo != b->lo) return a->lo < b->lo ? -1 : 1;
    if (a->hi != b->hi) return a->hi < b->hi ? -1 : 1;
    return (a->h < b->h) ? -1 : (a->h > b->h);
}

void om_free(om_mesh *m);

static int finish_mesh(om_mesh *m);

/* Build from an indexed mesh (X [V][3] doubles, tri [T][3]).  Used directly by the
 * finite-difference checks, and by om_build_soup after welding. */
int om_build_indexed(const double *X, int64_t V, const int32_t *tri, int64_t T, om_mesh **out) {
    om_mesh *m = (om_mesh *)calloc(1, sizeof(om_mesh));
    if (!m) return OR_ERR_OOM;
    m->T = T; m->V = V;
    m->X = (double *)malloc(sizeof(double) * 3 * V);
    m->tri = (int32_t *)malloc(sizeof(int32_t) * 3 * T);
    m->soup_vid = (int32_t *)malloc(sizeof(int32_t) * 3 * T);
    if (!m->X || !m->tri || !m->soup_vid) { om_free(m); return OR_ERR_OOM; }
    memcpy(m->X, X, sizeof(double) * 3 * V);
    memcpy(m->tri, tri, sizeof(int32_t) * 3 * T);
    memcpy(m->soup_vid, tri, sizeof(int32_t) * 3 * T);
    for (int64_t i = 0; i < 3 * V; i++) if (!isfinite(m->X[i])) { om_free(m); return OR_ERR_NONFINITE; }
    int st = finish_mesh(m);
    if (st) { om_free(m); return st; }
    *out = m;
    return OR_OK;
}

/* Build from an FP32 soup [T][3][3]: weld equal coordinates, then connectivity. */
int om_build_soup(const float *soup, int64_t T, om_mesh **out) {
    int64_t n = 3 * T;
    wrec *w = (wrec *)malloc(sizeof(wrec) * (n ? n : 1));
    if (!w) return OR_ERR_OOM;
    for (int64_t i = 0; i < n; i++) {
        w[i].x = (double)soup[3 * i + 0];
        w[i].y = (double)soup[3 * i + 1];
        w[i].z = (double)soup[3 * i + 2];
        w[i].idx = i;
        if (!isfinite(w[i].x) || !isfinite(w[i].y) || !isfinite(w[i].z)) { free(w); return OR_ERR_NONFINITE; }
    }
    qsort(w, (size_t)n, sizeof(wrec), wrec_cmp);
    int32_t *vid = (int32_t *)malloc(sizeof(int32_t) * (n ? n : 1));
    double *X = (double *)malloc(sizeof(double) * 3 * (n ? n : 1));
    if (!vid || !X) { free(w); free(vid); free(X); return OR_ERR_OOM; }
    int64_t V = 0;
    for (int64_t i = 0; i < n; i++) {
        /* == on doubles treats -0 and +0 as equal */
        if (i == 0 || !(w[i].x == w[i - 1].x && w[i].y == w[i - 1].y && w[i].z == w[i - 1].z)) {
            X[3 * V + 0] = w[i].x; X[3 * V + 1] = w[i].y; X[3 * V + 2] = w[i].z;
            V++;
        }
        vid[w[i].idx] = (int32_t)(V - 1);
    }
    free(w);
    int st = om_build_indexed(X, V, vid, T, out);
    free(X); free(vid);
    return st;
}

static int finish_mesh(om_mesh *m) {
    int64_t T = m->T, V = m->V, n = 3 * T;
    m->fn = (double *)malloc(sizeof(double) * 3 * (T ? T : 1));
    m->adj = (int32_t *)malloc(sizeof(int32_t) * 3 * (T ? T : 1));
    m->vn = (double *)calloc((size_t)(3 * (V ? V : 1)), sizeof(double));
    m->vclass = (int8_t *)malloc((size_t)(V ? V : 1));
    m->eclass = (int8_t *)malloc((size_t)(n ? n : 1));
    if (!m->fn || !m->adj || !m->vn || !m->vclass || !m->eclass) return OR_ERR_OOM;
    /* face normals; zero area is rejected (Section 4 disallows zero-area faces) */
    for (int64_t t = 0; t < T; t++) {
        const double *a = m->X + 3 * m->tri[3 * t], *b = m->X + 3 * m->tri[3 * t + 1], *c = m->X + 3 * m->tri[3 * t + 2];
        double ab[3], ac[3], cr[3];
        v_sub(b, a, ab); v_sub(c, a, ac); v_cross(ab, ac, cr);
        double len = v_norm(cr);
        double scale = v_dot(ab, ab) + v_dot(ac, ac);
        if (!(len > 1e-14 * scale) || m->tri[3 * t] == m->tri[3 * t + 1] || m->tri[3 * t + 1] == m->tri[3 * t + 2] ||
            m->tri[3 * t] == m->tri[3 * t + 2])
            return OR_ERR_DEGENERATE;
        for (int k = 0; k < 3; k++) m->fn[3 * t + k] = cr[k] / len;
    }
    /* edge pairing: every directed edge meets exactly one opposite directed edge */
    if (n % 2) return OR_ERR_NONMANIFOLD;
    erec *e = (erec *)malloc(sizeof(erec) * (n ? n : 1));
    if (!e) return OR_ERR_OOM;
    for (int64_t h = 0; h < n; h++) {
        int64_t t = h / 3, k = h % 3;
        int64_t a = m->tri[3 * t + k], b = m->tri[3 * t + (k + 1) % 3];
        e[h].lo = a < b ? a : b; e[h].hi = a < b ? b : a; e[h].h = h;
    }
    qsort(e, (size_t)n, sizeof(erec), erec_cmp);
    for (int64_t i = 0; i < n; i += 2) {
        if (e[i].lo != e[i + 1].lo || e[i].hi != e[i + 1].hi) { free(e); return OR_ERR_NONMANIFOLD; }
        if (i + 2 < n && e[i + 2].lo == e[i].lo && e[i + 2].hi == e[i].hi) { free(e); return OR_ERR_NONMANIFOLD; }
        int64_t h0 = e[i].h, h1 = e[i + 1].h;
        int64_t a0 = m->tri[3 * (h0 / 3) + h0 % 3], a1 = m->tri[3 * (h1 / 3) + h1 % 3];
        if (a0 == a1) { free(e); return OR_ERR_NONMANIFOLD; } /* same direction twice: not oriented */
        m->adj[h0] = (int32_t)(h1 / 3);
        m->adj[h1] = (int32_t)(h0 / 3);
    }
    free(e);
    m->E = n / 2;
    /* angle-weighted pseudonormals N_alpha = sum alpha_i n_i (Eq. 8) */
    for (int64_t t = 0; t < T; t++) {
        for (int k = 0; k < 3; k++) {
            const double *p = m->X + 3 * m->tri[3 * t + k];
            const double *q = m->X + 3 * m->tri[3 * t + (k + 1) % 3];
            const double *r = m->X + 3 * m->tri[3 * t + (k + 2) % 3];
            double e1[3], e2[3], cr[3];
            v_sub(q, p, e1); v_sub(r, p, e2); v_cross(e1, e2, cr);
            double alpha = atan2(v_norm(cr), v_dot(e1, e2));
            double *N = m->vn + 3 * m->tri[3 * t + k];
            for (int j = 0; j < 3; j++) N[j] += alpha * m->fn[3 * t + j];
        }
    }
    /* edge classification (Section 8.2): d = (ab x n1) . n2, ab directed as in face 1 */
    for (int64_t h = 0; h < n; h++) {
        int64_t t = h / 3, k = h % 3;
        const double *a = m->X + 3 * m->tri[3 * t + k], *b = m->X + 3 * m->tri[3 * t + (k + 1) % 3];
        double ab[3], cr[3];
        v_sub(b, a, ab);
        v_cross(ab, m->fn + 3 * t, cr);
        double d = v_dot(cr, m->fn + 3 * m->adj[h]);
        double tol = 1e-12 * v_norm(ab);
        m->eclass[h] = (int8_t)(d > tol ? 1 : (d < -tol ? -1 : 0));
    }
    /* vertex classification (Section 8.3): neighbours all below the pseudonormal plane -> convex,
     * all above -> concave, all on it -> flat, otherwise saddle.  "Below" is (v_n - v).N < 0. */
    int8_t *below = (int8_t *)calloc((size_t)(V ? V : 1), 1), *above = (int8_t *)calloc((size_t)(V ? V : 1), 1);
    if (!below || !above) { free(below); free(above); return OR_ERR_OOM; }
    for (int64_t h = 0; h < n; h++) {
        int64_t t = h / 3, k = h % 3;
        int64_t v = m->tri[3 * t + k], vn = m->tri[3 * t + (k + 1) % 3];
        double dv[3];
        v_sub(m->X + 3 * vn, m->X + 3 * v, dv);
        double d = v_dot(dv, m->vn + 3 * v);
        double tol = 1e-12 * v_norm(dv) * v_norm(m->vn + 3 * v);
        if (d < -tol) below[v] = 1;
        else if (d > tol) above[v] = 1;
    }
    for (int64_t v = 0; v < V; v++)
        m->vclass[v] = (int8_t)(below[v] && above[v] ? 2 : (below[v] ? 1 : (above[v] ? -1 : 0)));
    free(below); free(above);
    /* bin grid for the exact pruned search */
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double elen = 0.0;
    for (int64_t t = 0; t < T; t++) {
        for (int k = 0; k < 3; k++) {
            const double *p = m->X + 3 * m->tri[3 * t + k];
            for (int j = 0; j < 3; j++) { if (p[j] < lo[j]) lo[j] = p[j]; if (p[j] > hi[j]) hi[j] = p[j]; }
            double d[3];
            v_sub(m->X + 3 * m->tri[3 * t + (k + 1) % 3], p, d);
            elen += v_norm(d);
        }
    }
    elen /= (double)(3 * (T ? T : 1));
    double ext = 0.0;
    for (int j = 0; j < 3; j++) ext = fmax(ext, hi[j] - lo[j]);
    double cs = fmax(2.0 * elen, ext / 256.0);
    if (!(cs > 0)) cs = 1.0;
    int64_t ncell = 1;
    for (int j = 0; j < 3; j++) {
        m->blo[j] = lo[j];
        m->bn[j] = (int32_t)fmax(1.0, ceil((hi[j] - lo[j]) / cs));
        ncell *= m->bn[j];
    }
    m->bcs = cs;
    m->bstart = (int64_t *)calloc((size_t)(ncell + 1), sizeof(int64_t));
    if (!m->bstart) return OR_ERR_OOM;
    int32_t (*box)[6] = (int32_t(*)[6])malloc(sizeof(int32_t) * 6 * (T ? T : 1));
    if (!box) return OR_ERR_OOM;
    for (int64_t t = 0; t < T; t++) {
        for (int j = 0; j < 3; j++) {
            double a = m->X[3 * m->tri[3 * t] + j], b = m->X[3 * m->tri[3 * t + 1] + j], c = m->X[3 * m->tri[3 * t + 2] + j];
            double mn = fmin(a, fmin(b, c)) - 1e-9 * cs, mx = fmax(a, fmax(b, c)) + 1e-9 * cs;
            int32_t c0 = (int32_t)floor((mn - m->blo[j]) / cs), c1 = (int32_t)floor((mx - m->blo[j]) / cs);
            c0 = c0 < 0 ? 0 : (c0 >= m->bn[j] ? m->bn[j] - 1 : c0);
            c1 = c1 < 0 ? 0 : (c1 >= m->bn[j] ? m->bn[j] - 1 : c1);
            box[t][j] = c0; box[t][3 + j] = c1;
        }
        for (int32_t z = box[t][2]; z <= box[t][5]; z++)
            for (int32_t y = box[t][1]; y <= box[t][4]; y++)
                for (int32_t x = box[t][0]; x <= box[t][3]; x++)
                    m->bstart[((int64_t)z * m->bn[1] + y) * m->bn[0] + x + 1]++;
    }
    for (int64_t c = 0; c < ncell; c++) m->bstart[c + 1] += m->bstart[c];
    m->bitems = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m->bstart[ncell] ? m->bstart[ncell] : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    if (!m->bitems || !fill) { free(box); free(fill); return OR_ERR_OOM; }
    memcpy(fill, m->bstart, sizeof(int64_t) * (size_t)ncell);
    for (int64_t t = 0; t < T; t++) /* ascending t: cells list triangles in index order */
        for (int32_t z = box[t][2]; z <= box[t][5]; z++)
            for (int32_t y = box[t][1]; y <= box[t][4]; y++)
                for (int32_t x = box[t][0]; x <= box[t][3]; x++)
                    m->bitems[fill[((int64_t)z * m->bn[1] + y) * m->bn[0] + x]++] = (int32_t)t;
    free(fill); free(box);
    return OR_OK;
}

void om_free(om_mesh *m) {
    if (!m) return;
    free(m->X); free(m->tri); free(m->soup_vid); free(m->fn); free(m->adj); free(m->vn);
    free(m->vclass); free(m->eclass); free(m->bstart); free(m->bitems);
    free(m);
}

/* ------------------------------------------------------------------ accessors */
void om_counts(const om_mesh *m, int64_t *out /* [8] */) {
    int64_t nc = 0, ncc = 0, nf = 0, ns = 0, ec = 0, ecc = 0, ef = 0;
    for (int64_t v = 0; v < m->V; v++) {
        nc += m->vclass[v] == 1; ncc += m->vclass[v] == -1; nf += m->vclass[v] == 0; ns += m->vclass[v] == 2;
    }
    for (int64_t h = 0; h < 3 * m->T; h++) {
        int64_t t = h / 3, k = h % 3;
        if (m->tri[3 * t + k] < m->tri[3 * t + (k + 1) % 3]) { /* count each undirected edge once */
            ec += m->eclass[h] == 1; ecc += m->eclass[h] == -1; ef += m->eclass[h] == 0;
        }
    }
    out[0] = m->V; out[1] = m->E; out[2] = nc; out[3] = ncc; out[4] = nf; out[5] = ns; out[6] = ec; out[7] = ecc;
    (void)ef;
}
void om_vertices(const om_mesh *m, double *out) { memcpy(out, m->X, sizeof(double) * 3 * m->V); }
void om_triangles(const om_mesh *m, int32_t *out) { memcpy(out, m->tri, sizeof(int32_t) * 3 * m->T); }
void om_soup_vid(const om_mesh *m, int32_t *out) { memcpy(out, m->soup_vid, sizeof(int32_t) * 3 * m->T); }
void om_vclass(const om_mesh *m, int8_t *out) { memcpy(out, m->vclass, (size_t)m->V); }
void om_pseudonormals(const om_mesh *m, double *out) { memcpy(out, m->vn, sizeof(double) * 3 * m->V); }

/* ------------------------------------------------------------------ point-triangle distance
 * The closest point of a triangle to p is the orthogonal projection of p onto the
 * triangle's plane when that projection lies inside the triangle; otherwise it lies
 * on the boundary, i.e. on one of the three closed segments.  region: 0 interior,
 * 1+k the open edge from corner k to corner k+1, 4+k corner k.  lam: barycentric
 * weights of the closest point on corners (0,1,2).  Returns the squared distance. */
static double pt_tri(const double *p, const double *A, const double *B, const double *C, const double *n,
                     int *region, double *lam) {
    /* all arithmetic on differences from corner A, so the result is unchanged bitwise
     * when p and the triangle are shifted together by an exactly representable vector */
    double ap[3], q[3], P[3][3];
    v_sub(p, A, ap);
    P[0][0] = P[0][1] = P[0][2] = 0.0;
    v_sub(B, A, P[1]);
    v_sub(C, A, P[2]);
    double h = v_dot(ap, n);
    for (int j = 0; j < 3; j++) q[j] = ap[j] - h * n[j]; /* projection, relative to A */
    double wgt[3];
    int inside = 1;
    for (int k = 0; k < 3; k++) {
        /* signed area of (P[k+1], P[k+2], q) along n: barycentric weight of corner k */
        double e[3], f[3], cr[3];
        v_sub(P[(k + 2) % 3], P[(k + 1) % 3], e);
        v_sub(q, P[(k + 1) % 3], f);
        v_cross(e, f, cr);
        wgt[k] = v_dot(cr, n);
        if (wgt[k] < 0) inside = 0;
    }
    if (inside) {
        double s = wgt[0] + wgt[1] + wgt[2];
        for (int k = 0; k < 3; k++) lam[k] = wgt[k] / s;
        *region = 0;
        return h * h;
    }
    double best = INFINITY;
    for (int k = 0; k < 3; k++) {
        const double *S = P[k], *E = P[(k + 1) % 3];
        double se[3], sp[3];
        v_sub(E, S, se);
        v_sub(ap, S, sp);
        double t = v_dot(sp, se) / v_dot(se, se);
        t = t < 0 ? 0 : (t > 1 ? 1 : t);
        double r[3] = {sp[0] - t * se[0], sp[1] - t * se[1], sp[2] - t * se[2]};
        double d2 = v_dot(r, r);
        if (d2 < best) {
            best = d2;
            lam[0] = lam[1] = lam[2] = 0.0;
            lam[k] = 1.0 - t; lam[(k + 1) % 3] = t;
            *region = t == 0.0 ? 4 + k : (t == 1.0 ? 4 + (k + 1) % 3 : 1 + k);
        }
    }
    return best;
}

/* signed value at p given the winning triangle t, its region and squared distance */
static double signed_from(const om_mesh *m, const double *p, int64_t t, int region, const double *lam, double d2) {
    if (d2 == 0.0) return 0.0;
    const int32_t *tv = m->tri + 3 * t;
    const double *A = m->X + 3 * tv[0];
    double pq[3], N[3];
    v_sub(p, A, pq); /* p - q = (p - A) - sum_k lam_k (X_k - A) */
    for (int k = 1; k < 3; k++) {
        double xk[3];
        v_sub(m->X + 3 * tv[k], A, xk);
        for (int j = 0; j < 3; j++) pq[j] -= lam[k] * xk[j];
    }
    if (region == 0) {
        /* p - q is parallel to the face normal: the sign of (p - A).n is the sign of (p - q).n */
        v_sub(p, A, pq);
        for (int j = 0; j < 3; j++) N[j] = m->fn[3 * t + j];
    } else if (region <= 3) {
        int k = region - 1;
        int64_t g = m->adj[3 * t + k];
        for (int j = 0; j < 3; j++) N[j] = m->fn[3 * t + j] + m->fn[3 * g + j];
    } else {
        int k = region - 4;
        for (int j = 0; j < 3; j++) N[j] = m->vn[3 * tv[k] + j];
    }
    double d = sqrt(d2);
    return v_dot(pq, N) < 0 ? -d : d;
}

typedef struct { double d2; int64_t t; int region; double lam[3]; } hit;

static void consider(const om_mesh *m, const double *p, int64_t t, hit *best) {
    const int32_t *tv = m->tri + 3 * t;
    int region = 0;
    double lam[3] = {0, 0, 0};
    double d2 = pt_tri(p, m->X + 3 * tv[0], m->X + 3 * tv[1], m->X + 3 * tv[2], m->fn + 3 * t, &region, lam);
    if (d2 < best->d2 || (d2 == best->d2 && t < best->t)) {
        best->d2 = d2; best->t = t; best->region = region;
        memcpy(best->lam, lam, sizeof(lam));
    }
}

/* literal loop over every triangle (the definition, Eq. 1) */
static hit query_brute(const om_mesh *m, const double *p) {
    hit b = {INFINITY, -1, -1, {0, 0, 0}};
    for (int64_t t = 0; t < m->T; t++) consider(m, p, t, &b);
    return b;
}

/* exact pruned loop; stops early (returning t = -1) once every triangle is provably
 * at distance >= cutoff.  With cutoff = inf it returns the same hit as query_brute. */
static hit query_pruned(const om_mesh *m, const double *p, double cutoff) {
    hit b = {INFINITY, -1, -1, {0, 0, 0}};
    int32_t c[3];
    for (int j = 0; j < 3; j++) {
        double f = floor((p[j] - m->blo[j]) / m->bcs);
        if (f < 0) f = 0;
        if (f > m->bn[j] - 1) f = m->bn[j] - 1;
        c[j] = (int32_t)f;
    }
    int32_t rmax = m->bn[0];
    if (m->bn[1] > rmax) rmax = m->bn[1];
    if (m->bn[2] > rmax) rmax = m->bn[2];
    /* a triangle id may appear in several cells: visiting it twice is harmless (same value) */
    for (int32_t r = 0; r <= rmax; r++) {
        int32_t lo[3], hi[3];
        for (int j = 0; j < 3; j++) { lo[j] = c[j] - r; hi[j] = c[j] + r; }
        for (int32_t z = lo[2]; z <= hi[2]; z++) {
            if (z < 0 || z >= m->bn[2]) continue;
            for (int32_t y = lo[1]; y <= hi[1]; y++) {
                if (y < 0 || y >= m->bn[1]) continue;
                for (int32_t x = lo[0]; x <= hi[0]; x++) {
                    if (x < 0 || x >= m->bn[0]) continue;
                    if (z != lo[2] && z != hi[2] && y != lo[1] && y != hi[1] && x != lo[0] && x != hi[0]) continue;
                    int64_t cell = ((int64_t)z * m->bn[1] + y) * m->bn[0] + x;
                    for (int64_t i = m->bstart[cell]; i < m->bstart[cell + 1]; i++) consider(m, p, m->bitems[i], &b);
                }
            }
        }
        /* every unvisited cell lies beyond the visited cube along some axis, and every
         * triangle is listed in all cells its (slightly grown) bounding box meets, so an
         * unvisited triangle is at least lb away from p */
        double lb = INFINITY;
        for (int j = 0; j < 3; j++) {
            if (hi[j] < m->bn[j] - 1) lb = fmin(lb, m->blo[j] + (hi[j] + 1) * m->bcs - p[j]);
            if (lo[j] > 0) lb = fmin(lb, p[j] - (m->blo[j] + lo[j] * m->bcs));
        }
        if (lb == INFINITY) break; /* all cells visited */
        double lbs = lb * (1.0 - 1e-9) - 1e-15 * m->bcs; /* conservative against rounding */
        if (lbs > 0 && lbs * lbs > b.d2) break;         /* unvisited triangles are strictly farther */
        if (lbs >= cutoff) break; /* unvisited triangles cannot be in the band; best keeps its own test */
    }
    return b;
}

/* ------------------------------------------------------------------ public queries */

/* Signed distance at arbitrary points (double [n][3]).  pruned: 0 literal loop, 1 exact pruned.
 * out_tri / out_region (nullable) give the winning triangle and region. */
void om_sdf_points(const om_mesh *m, const double *pts, int64_t n, int pruned,
                   double *out_d, int32_t *out_tri, int32_t *out_region) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        const double *p = pts + 3 * i;
        hit b = pruned ? query_pruned(m, p, INFINITY) : query_brute(m, p);
        out_d[i] = signed_from(m, p, b.t, b.region, b.lam, b.d2);
        if (out_tri) out_tri[i] = (int32_t)b.t;
        if (out_region) out_region[i] = b.region;
    }
}

/* Narrow-band value at grid points given by linear index (x fastest).  +inf when
 * |d| >= w.  pruned as above (the literal loop is used when pruned == 0). */
void om_band_points(const om_mesh *m, const int32_t *dims, const double *origin, double h, double w,
                    const int64_t *idx, int64_t n, int pruned, double *out_d, int32_t *out_tri, int32_t *out_region) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t s = 0; s < n; s++) {
        int64_t id = idx[s];
        int64_t i = id % dims[0], j = (id / dims[0]) % dims[1], k = id / ((int64_t)dims[0] * dims[1]);
        double p[3] = {origin[0] + (i + 0.5) * h, origin[1] + (j + 0.5) * h, origin[2] + (k + 0.5) * h};
        hit b = pruned ? query_pruned(m, p, w) : query_brute(m, p);
        double d = (b.t >= 0) ? signed_from(m, p, b.t, b.region, b.lam, b.d2) : INFINITY;
        if (!(fabs(d) < w)) { d = INFINITY; b.t = -1; b.region = -1; }
        out_d[s] = d;
        if (out_tri) out_tri[s] = (int32_t)b.t;
        if (out_region) out_region[s] = b.region;
    }
}

/* Dense narrow band over the whole grid.  Points outside the mesh bounding box grown
 * by w cannot be in the band and are written +inf without a query. */
void om_narrow_band(const om_mesh *m, const int32_t *dims, const double *origin, double h, double w,
                    int pruned, double *out, int32_t *out_tri) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t v = 0; v < m->V; v++)
        for (int j = 0; j < 3; j++) { lo[j] = fmin(lo[j], m->X[3 * v + j]); hi[j] = fmax(hi[j], m->X[3 * v + j]); }
    int64_t nx = dims[0], ny = dims[1], nz = dims[2];
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int64_t k = 0; k < nz; k++) {
        for (int64_t j = 0; j < ny; j++) {
            for (int64_t i = 0; i < nx; i++) {
                int64_t id = i + nx * (j + ny * k);
                double p[3] = {origin[0] + (i + 0.5) * h, origin[1] + (j + 0.5) * h, origin[2] + (k + 0.5) * h};
                int far = 0;
                for (int a = 0; a < 3; a++) far |= (p[a] < lo[a] - w) || (p[a] > hi[a] + w);
                double d = INFINITY;
                int64_t t = -1;
                if (!far) {
                    hit b = pruned ? query_pruned(m, p, w) : query_brute(m, p);
                    if (b.t >= 0) {
                        d = signed_from(m, p, b.t, b.region, b.lam, b.d2);
                        t = b.t;
                    }
                    if (!(fabs(d) < w)) { d = INFINITY; t = -1; }
                }
                out[id] = d;
                if (out_tri) out_tri[id] = (int32_t)t;
            }
        }
    }
}

/* Contribution of one point to the adjoint of L = sum_p g_p d(p): for d = s |p - q(X)| with
 * q = sum_k lam_k X_k the closest point of the triangle's feature (lam fixed at the minimiser:
 * envelope theorem), dd/dX_k = -s lam_k (p - q)/|p - q|.  b is the point's hit (triangle, region
 * label, weights, squared distance) and d its signed value; mine [V][3] is accumulated into. */
static void add_point_adjoint(const om_mesh *m, const double *p, double g, const hit *b, double d, double *mine) {
    const int32_t *tv = m->tri + 3 * b->t;
    const double *A = m->X + 3 * tv[0];
    double pq[3];
    v_sub(p, A, pq);
    for (int k = 1; k < 3; k++)
        for (int j = 0; j < 3; j++) pq[j] -= b->lam[k] * (m->X[3 * tv[k] + j] - A[j]);
    double u[3];
    if (b->region == 0) {
        /* (p - q)/|p - q| = s n inside the face region */
        for (int j = 0; j < 3; j++) u[j] = m->fn[3 * b->t + j] * (d < 0 ? -1.0 : 1.0);
    } else {
        double r = sqrt(b->d2);
        for (int j = 0; j < 3; j++) u[j] = pq[j] / r;
    }
    double s = d < 0 ? -1.0 : 1.0;
    for (int k = 0; k < 3; k++)
        for (int j = 0; j < 3; j++) mine[3 * tv[k] + j] += -g * s * b->lam[k] * u[j];
}

/* Per-thread accumulators summed into out_grad [V][3] (overwritten) in thread order. */
static double *adjoint_acc(const om_mesh *m, int *nth) {
    *nth = 1;
#ifdef _OPENMP
    *nth = omp_get_max_threads();
#endif
    return (double *)calloc((size_t)*nth * 3 * (m->V ? m->V : 1), sizeof(double));
}
static void adjoint_sum(const om_mesh *m, double *acc, int nth, double *out_grad) {
    memset(out_grad, 0, sizeof(double) * 3 * m->V);
    for (int t = 0; t < nth; t++)
        for (int64_t v = 0; v < 3 * m->V; v++) out_grad[v] += acc[(size_t)t * 3 * m->V + v];
    free(acc);
}

/* Adjoint of L = sum_p g_p d(p) with respect to the welded vertex positions, at the given
 * points (their band membership and winners as found here).  For d = s |p - q(X)| with
 * q = sum_k lam_k X_k the closest point (lam fixed at the minimiser: envelope theorem),
 * dd/dX_k = -s lam_k (p - q)/|p - q|.  out_grad [V][3] is overwritten. */
void om_adjoint_points(const om_mesh *m, const double *pts, const double *g, int64_t n, double w,
                       double *out_grad) {
    int nth;
    double *acc = adjoint_acc(m, &nth);
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *mine = acc + (size_t)tid * 3 * m->V;
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; i++) {
            const double *p = pts + 3 * i;
            hit b = query_pruned(m, p, w);
            if (b.t < 0 || g[i] == 0.0 || b.d2 == 0.0) continue;
            double d = signed_from(m, p, b.t, b.region, b.lam, b.d2);
            if (!(fabs(d) < w)) continue;
            add_point_adjoint(m, p, g[i], &b, d, mine);
        }
    }
    adjoint_sum(m, acc, nth, out_grad);
}

/* The closest point of p on one given feature of triangle t: region 0 the closed triangle,
 * 1 + k its closed edge from corner k to corner k + 1, 4 + k its corner k (the labels of
 * pt_tri).  Returns the hit (whose region labels where on the feature the closest point lies:
 * the feature's relative interior or one of its end points) and sets *d to the signed
 * distance, the sign from the pseudonormal of that feature (Section 4.3, Eq. 8).
 *
 * If the closest point of the whole triangle lies on the given feature, it is also the
 * feature's closest point (the feature is a subset of the triangle), so pt_tri's result is
 * taken as it is; otherwise the feature's own closest point is computed on the segment (with
 * the arithmetic of pt_tri's segment loop, relative to corner 0) or is the corner itself. */
static hit feature_hit(const om_mesh *m, const double *p, int64_t t, int region, double *d) {
    const int32_t *tv = m->tri + 3 * t;
    const double *A = m->X + 3 * tv[0];
    hit b = {INFINITY, t, -1, {0, 0, 0}};
    b.d2 = pt_tri(p, A, m->X + 3 * tv[1], m->X + 3 * tv[2], m->fn + 3 * t, &b.region, b.lam);
    int on_feature;
    if (region == 0) on_feature = 1;
    else if (region <= 3) on_feature = b.region == region || b.region == 4 + (region - 1) || b.region == 4 + region % 3;
    else on_feature = b.region == region;
    if (!on_feature) {
        double ap[3], P[3][3];
        v_sub(p, A, ap);
        P[0][0] = P[0][1] = P[0][2] = 0.0;
        v_sub(m->X + 3 * tv[1], A, P[1]);
        v_sub(m->X + 3 * tv[2], A, P[2]);
        b.lam[0] = b.lam[1] = b.lam[2] = 0.0;
        if (region <= 3) {
            int k = region - 1;
            const double *S = P[k], *E = P[(k + 1) % 3];
            double se[3], sp[3];
            v_sub(E, S, se);
            v_sub(ap, S, sp);
            double tt = v_dot(sp, se) / v_dot(se, se);
            tt = tt < 0 ? 0 : (tt > 1 ? 1 : tt);
            double r[3] = {sp[0] - tt * se[0], sp[1] - tt * se[1], sp[2] - tt * se[2]};
            b.d2 = v_dot(r, r);
            b.lam[k] = 1.0 - tt;
            b.lam[(k + 1) % 3] = tt;
            b.region = tt == 0.0 ? 4 + k : (tt == 1.0 ? 4 + (k + 1) % 3 : 1 + k);
        } else {
            int k = region - 4;
            double r[3];
            v_sub(ap, P[k], r);
            b.d2 = v_dot(r, r);
            b.lam[k] = 1.0;
            b.region = region;
        }
    }
    *d = signed_from(m, p, t, b.region, b.lam, b.d2);
    return b;
}

/* The adjoint of L = sum_p g_p d_F(p) where d_F(p) is the signed distance of point p to a
 * GIVEN feature (tri[i], region[i]) (labels as in feature_hit), not to its own closest one:
 * the same per-point contribution as om_adjoint_points with the winner fixed by the caller, so
 * that another implementation's choice of winners can be evaluated in FP64.  No band test.
 * out_grad [V][3] is overwritten; out_d [n] (nullable) receives d_F(p). */
void om_adjoint_features(const om_mesh *m, const double *pts, const double *g, const int32_t *tri,
                         const int32_t *region, int64_t n, double *out_grad, double *out_d) {
    int nth;
    double *acc = adjoint_acc(m, &nth);
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *mine = acc + (size_t)tid * 3 * m->V;
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; i++) {
            const double *p = pts + 3 * i;
            double d = INFINITY;
            hit b = feature_hit(m, p, tri[i], region[i], &d);
            if (out_d) out_d[i] = d;
            if (g[i] == 0.0 || b.d2 == 0.0) continue;
            add_point_adjoint(m, p, g[i], &b, d, mine);
        }
    }
    adjoint_sum(m, acc, nth, out_grad);
}

/* Number of OpenMP threads of the following calls (tests compare sums in one fixed order). */
void om_set_num_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int om_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
