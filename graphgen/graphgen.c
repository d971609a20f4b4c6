/*
 * graphgen.c -- seeded synthetic graph generators (input side only).
 *
 * This module produces the CSR inputs that both the CUDA library and the
 * oracle consume.  It holds none of the traversal arithmetic: no distances,
 * no frontiers, no reachability.  Every random number is a counter-based
 * draw (SplitMix64 finaliser of seed + counter, Steele, Lea & Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014), so the
 * output is a pure function of the arguments and does not depend on the
 * number of OpenMP threads or on the machine (x86 or Arm).
 *
 * Output format: CSR with uint32 offsets[n+1] and indices[m]; every
 * neighbour list sorted ascending, duplicates and self-loops removed
 * (except by gg_random, which can keep them on purpose for tests).
 *
 * Graph families (shapes of the paper's inputs, Table 1 of the paper):
 *   gg_grid   undirected rows x cols 4-neighbour grid, row-major ids
 *             (REC-like synthetic grids; rows = 1 gives a path / strip)
 *   gg_dgrid  directed grid: each grid edge kept in both directions with
 *             probability p_both, else in one random direction, plus a
 *             number of random long-range directed shortcut arcs
 *   gg_knn    exact k-nearest-neighbour graph of uniform points in the unit
 *             square, symmetrised (GeoLife / Chem / Cosmo-like kNN graphs)
 *   gg_rmat   R-MAT power-law graph, symmetrised, ids randomly permuted
 *             (social / web low-diameter graphs)
 *   gg_random tiny uniform random graphs for brute-force checks
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GG_OK 0
#define GG_ERR_ARG 1
#define GG_ERR_OOM 2
#define GG_ERR_TOO_LARGE 3

typedef struct {
    uint32_t n;
    uint32_t m;
    uint32_t *offsets; /* n+1 */
    uint32_t *indices; /* m   */
} gg_csr;

/* ---------------------------------------------------------------- PRNG -- */

static inline uint64_t gg_mix64(uint64_t z) {
    /* SplitMix64 output function (published constants of the finaliser). */
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* i-th draw of the stream identified by (seed, stream). */
static inline uint64_t gg_draw(uint64_t seed, uint64_t stream, uint64_t i) {
    uint64_t key = gg_mix64(seed ^ gg_mix64(stream + 0x632be59bd9b4e019ULL));
    return gg_mix64(key + (i + 1) * 0x9e3779b97f4a7c15ULL);
}

static inline double gg_unit(uint64_t x) { /* [0,1) with 53 bits */
    return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

/* exported for tests: the raw draw function */
uint64_t gg_rand(uint64_t seed, uint64_t stream, uint64_t i) { return gg_draw(seed, stream, i); }

enum { S_DGRID_KEEP = 1, S_DGRID_DIR = 2, S_DGRID_SC = 3, S_KNN_X = 4, S_KNN_Y = 5,
       S_RMAT = 6, S_PERM = 7, S_SRC = 8, S_RAND = 9 };

/* ------------------------------------------------------- arc list -> CSR -- */

static int cmp_u32(const void *a, const void *b) {
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

static void sort_small(uint32_t *a, uint32_t len) {
    if (len > 48) { qsort(a, len, sizeof(uint32_t), cmp_u32); return; }
    for (uint32_t i = 1; i < len; i++) {
        uint32_t x = a[i], j = i;
        while (j > 0 && a[j - 1] > x) { a[j] = a[j - 1]; j--; }
        a[j] = x;
    }
}

/*
 * Build a canonical CSR from M arcs (src[i] -> dst[i]).  If symmetrize, the
 * reverse of every arc is added.  Self-loops and duplicates are removed when
 * `clean` is set.  The result does not depend on arc order or thread count.
 */
static int csr_from_arcs(uint32_t n, uint64_t M, const uint32_t *src, const uint32_t *dst,
                         int symmetrize, int clean, gg_csr *out) {
    uint64_t total = symmetrize ? 2 * M : M;
    if (total > 0xFFFFFFF0ULL) return GG_ERR_TOO_LARGE;
    uint32_t *deg = (uint32_t *)calloc((size_t)n + 1, sizeof(uint32_t));
    if (!deg) return GG_ERR_OOM;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)M; i++) {
        uint32_t u = src[i], v = dst[i];
        if (clean && u == v) continue;
        __atomic_fetch_add(&deg[u], 1u, __ATOMIC_RELAXED);
        if (symmetrize) __atomic_fetch_add(&deg[v], 1u, __ATOMIC_RELAXED);
    }
    uint32_t *off = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    if (!off) { free(deg); return GG_ERR_OOM; }
    uint64_t acc = 0;
    for (uint32_t v = 0; v < n; v++) { off[v] = (uint32_t)acc; acc += deg[v]; }
    off[n] = (uint32_t)acc;
    uint32_t *tmp = (uint32_t *)malloc((size_t)(acc ? acc : 1) * sizeof(uint32_t));
    if (!tmp) { free(deg); free(off); return GG_ERR_OOM; }
    /* reuse deg as per-vertex cursor */
    memcpy(deg, off, (size_t)n * sizeof(uint32_t));
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)M; i++) {
        uint32_t u = src[i], v = dst[i];
        if (clean && u == v) continue;
        uint32_t p = __atomic_fetch_add(&deg[u], 1u, __ATOMIC_RELAXED);
        tmp[p] = v;
        if (symmetrize) {
            uint32_t q = __atomic_fetch_add(&deg[v], 1u, __ATOMIC_RELAXED);
            tmp[q] = u;
        }
    }
    /* sort + dedupe each list; deg[v] becomes the cleaned degree */
    #pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < (int64_t)n; v++) {
        uint32_t b = off[v], e = off[v + 1];
        sort_small(tmp + b, e - b);
        uint32_t w = b;
        for (uint32_t i = b; i < e; i++) {
            if (clean && i > b && tmp[i] == tmp[i - 1]) continue;
            tmp[w++] = tmp[i];
        }
        deg[v] = w - b;
    }
    uint32_t *noff = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    if (!noff) { free(deg); free(off); free(tmp); return GG_ERR_OOM; }
    acc = 0;
    for (uint32_t v = 0; v < n; v++) { noff[v] = (uint32_t)acc; acc += deg[v]; }
    noff[n] = (uint32_t)acc;
    uint32_t *idx = (uint32_t *)malloc((size_t)(acc ? acc : 1) * sizeof(uint32_t));
    if (!idx) { free(deg); free(off); free(tmp); free(noff); return GG_ERR_OOM; }
    #pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < (int64_t)n; v++)
        memcpy(idx + noff[v], tmp + off[v], (size_t)deg[v] * sizeof(uint32_t));
    free(deg); free(off); free(tmp);
    out->n = n; out->m = (uint32_t)acc; out->offsets = noff; out->indices = idx;
    return GG_OK;
}

void gg_free(gg_csr *g) {
    if (!g) return;
    free(g->offsets); free(g->indices);
    g->offsets = g->indices = NULL; g->n = g->m = 0;
}

/* ------------------------------------------------------------ families -- */

/* Undirected 4-neighbour grid, vertex (r,c) has id r*cols + c. */
int gg_grid(uint32_t rows, uint32_t cols, gg_csr *out) {
    if (!out || rows == 0 || cols == 0) return GG_ERR_ARG;
    uint64_t n = (uint64_t)rows * cols;
    if (n >= 0xFFFFFFFFULL) return GG_ERR_TOO_LARGE;
    uint64_t m = 2ULL * ((uint64_t)rows * (cols - 1) + (uint64_t)(rows - 1) * cols);
    if (m > 0xFFFFFFF0ULL) return GG_ERR_TOO_LARGE;
    uint32_t *off = (uint32_t *)malloc((n + 1) * sizeof(uint32_t));
    uint32_t *idx = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
    if (!off || !idx) { free(off); free(idx); return GG_ERR_OOM; }
    /* degree of (r,c) depends only on whether it is on a border, so the
       offsets have a closed form per row; fill row by row in parallel. */
    #pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < (int64_t)rows; r++) {
        uint64_t base = 0;
        /* edges before row r: each earlier row contributes its arcs */
        uint64_t row_h = 2ULL * (cols - 1);                 /* horizontal arcs in a row */
        /* vertical arcs: every row r' < r contributes "down" arcs from r' and
           "up" arcs from r'+... count arcs with source in rows < r */
        uint64_t up_down_before = 0;
        if (r > 0) up_down_before = (uint64_t)cols * (2ULL * (uint64_t)r - 1); /* row0: down; rows1..r-1: up+down */
        if (rows == 1) up_down_before = 0;
        base = (uint64_t)r * row_h + up_down_before;
        uint64_t p = base;
        for (uint32_t c = 0; c < cols; c++) {
            uint64_t v = (uint64_t)r * cols + c;
            off[v] = (uint32_t)p;
            /* ascending order: up, left, right, down */
            if (r > 0) idx[p++] = (uint32_t)(v - cols);
            if (c > 0) idx[p++] = (uint32_t)(v - 1);
            if (c + 1 < cols) idx[p++] = (uint32_t)(v + 1);
            if ((uint32_t)r + 1 < rows) idx[p++] = (uint32_t)(v + cols);
        }
    }
    off[n] = (uint32_t)m;
    out->n = (uint32_t)n; out->m = (uint32_t)m; out->offsets = off; out->indices = idx;
    return GG_OK;
}

/*
 * Directed grid.  Undirected grid edge e (horizontal edges numbered first,
 * row-major, then vertical ones) is kept in both directions when
 * draw(KEEP,e) < p_both, otherwise in one direction chosen by the low bit of
 * draw(DIR,e).  Then `shortcuts` extra arcs with endpoints drawn uniformly;
 * a draw that is a self-loop or repeats an existing arc is redrawn.
 */
int gg_dgrid(uint32_t rows, uint32_t cols, double p_both, uint64_t seed, uint32_t shortcuts,
             gg_csr *out) {
    if (!out || rows == 0 || cols == 0 || !(p_both >= 0.0 && p_both <= 1.0)) return GG_ERR_ARG;
    uint64_t n = (uint64_t)rows * cols;
    if (n >= 0xFFFFFFFFULL) return GG_ERR_TOO_LARGE;
    uint64_t H = (uint64_t)rows * (cols - 1), V = (uint64_t)(rows - 1) * cols, E = H + V;
    uint64_t maxarcs = 2 * E + shortcuts;
    if (maxarcs > 0xFFFFFFF0ULL) return GG_ERR_TOO_LARGE;
    uint32_t *src = (uint32_t *)malloc((maxarcs ? maxarcs : 1) * sizeof(uint32_t));
    uint32_t *dst = (uint32_t *)malloc((maxarcs ? maxarcs : 1) * sizeof(uint32_t));
    uint8_t *kind = (uint8_t *)malloc(E ? E : 1);
    if (!src || !dst || !kind) { free(src); free(dst); free(kind); return GG_ERR_OOM; }
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < (int64_t)E; e++) {
        double u = gg_unit(gg_draw(seed, S_DGRID_KEEP, (uint64_t)e));
        kind[e] = (u < p_both) ? 2 : (uint8_t)(gg_draw(seed, S_DGRID_DIR, (uint64_t)e) & 1);
    }
    /* prefix over kinds (arcs per edge = 2 if both else 1) */
    uint64_t *pos = (uint64_t *)malloc((E + 1) * sizeof(uint64_t));
    if (!pos) { free(src); free(dst); free(kind); return GG_ERR_OOM; }
    uint64_t acc = 0;
    for (uint64_t e = 0; e < E; e++) { pos[e] = acc; acc += (kind[e] == 2) ? 2 : 1; }
    pos[E] = acc;
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < (int64_t)E; e++) {
        uint32_t a, b;
        if ((uint64_t)e < H) {
            uint64_t r = (uint64_t)e / (cols - 1), c = (uint64_t)e % (cols - 1);
            a = (uint32_t)(r * cols + c); b = a + 1;
        } else {
            uint64_t f = (uint64_t)e - H;
            uint64_t r = f / cols, c = f % cols;
            a = (uint32_t)(r * cols + c); b = a + cols;
        }
        uint64_t p = pos[e];
        if (kind[e] == 2) { src[p] = a; dst[p] = b; src[p + 1] = b; dst[p + 1] = a; }
        else if (kind[e] == 0) { src[p] = a; dst[p] = b; }
        else { src[p] = b; dst[p] = a; }
    }
    free(pos); free(kind);
    uint64_t M = acc;
    gg_csr base;
    int rc = csr_from_arcs((uint32_t)n, M, src, dst, 0, 1, &base);
    if (rc) { free(src); free(dst); return rc; }
    if (shortcuts == 0) { free(src); free(dst); *out = base; return GG_OK; }
    /* shortcut arcs, drawn sequentially so redraws are deterministic */
    uint32_t *ss = src, *sd = dst; /* reuse buffers (size >= shortcuts) */
    uint64_t drawn = 0, i = 0;
    while (drawn < shortcuts) {
        uint32_t a = (uint32_t)(gg_draw(seed, S_DGRID_SC, 2 * i) % n);
        uint32_t b = (uint32_t)(gg_draw(seed, S_DGRID_SC, 2 * i + 1) % n);
        i++;
        if (a == b) continue;
        int dup = 0;
        for (uint32_t q = base.offsets[a]; q < base.offsets[a + 1]; q++)
            if (base.indices[q] == b) { dup = 1; break; }
        for (uint64_t q = 0; q < drawn && !dup; q++)
            if (ss[q] == a && sd[q] == b) dup = 1;
        if (dup) continue;
        ss[drawn] = a; sd[drawn] = b; drawn++;
    }
    /* merge: rebuild from base arcs + shortcuts */
    uint64_t Mt = (uint64_t)base.m + shortcuts;
    uint32_t *s2 = (uint32_t *)malloc(Mt * sizeof(uint32_t));
    uint32_t *d2 = (uint32_t *)malloc(Mt * sizeof(uint32_t));
    if (!s2 || !d2) { free(s2); free(d2); free(src); free(dst); gg_free(&base); return GG_ERR_OOM; }
    #pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < (int64_t)n; v++)
        for (uint32_t q = base.offsets[v]; q < base.offsets[v + 1]; q++) { s2[q] = (uint32_t)v; d2[q] = base.indices[q]; }
    for (uint64_t q = 0; q < shortcuts; q++) { s2[base.m + q] = ss[q]; d2[base.m + q] = sd[q]; }
    free(src); free(dst); gg_free(&base);
    rc = csr_from_arcs((uint32_t)n, Mt, s2, d2, 0, 1, out);
    free(s2); free(d2);
    return rc;
}

/* ----------------------------------------------------------------- kNN -- */

typedef struct { double d2; uint32_t id; } knn_cand;

static inline int cand_less(double d2a, uint32_t ia, double d2b, uint32_t ib) {
    return d2a < d2b || (d2a == d2b && ia < ib);
}

/*
 * Points: x_i = (draw(X,i) >> 40) * 2^-24, y_i likewise (exact fp32 values on
 * a 2^-24 lattice).  Squared distances are computed in fp64 from the fp32
 * coordinates; on this lattice they are exact, so "nearest" is unambiguous
 * and ties are broken by the smaller point index.  Each point is linked to
 * its k nearest other points; the arc set is then symmetrised.
 */
int gg_knn(uint32_t npts, uint32_t k, uint64_t seed, gg_csr *out, float *xy_out) {
    if (!out || npts < 2 || k == 0 || k >= npts || k > 64) return GG_ERR_ARG;
    if ((uint64_t)npts * k * 2 > 0xFFFFFFF0ULL) return GG_ERR_TOO_LARGE;
    float *xy = xy_out ? xy_out : (float *)malloc((size_t)npts * 2 * sizeof(float));
    if (!xy) return GG_ERR_OOM;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)npts; i++) {
        xy[2 * i] = (float)((double)(gg_draw(seed, S_KNN_X, (uint64_t)i) >> 40) * (1.0 / 16777216.0));
        xy[2 * i + 1] = (float)((double)(gg_draw(seed, S_KNN_Y, (uint64_t)i) >> 40) * (1.0 / 16777216.0));
    }
    uint32_t G = (uint32_t)ceil(sqrt((double)npts / 2.0));
    if (G < 1) G = 1;
    uint64_t ncell = (uint64_t)G * G;
    uint32_t *cell_start = (uint32_t *)calloc(ncell + 1, sizeof(uint32_t));
    uint32_t *cell_of = (uint32_t *)malloc((size_t)npts * sizeof(uint32_t));
    uint32_t *bucket = (uint32_t *)malloc((size_t)npts * sizeof(uint32_t));
    uint32_t *src = (uint32_t *)malloc((size_t)npts * k * sizeof(uint32_t));
    uint32_t *dst = (uint32_t *)malloc((size_t)npts * k * sizeof(uint32_t));
    if (!cell_start || !cell_of || !bucket || !src || !dst) {
        free(cell_start); free(cell_of); free(bucket); free(src); free(dst);
        if (!xy_out) free(xy);
        return GG_ERR_OOM;
    }
    for (uint32_t i = 0; i < npts; i++) {
        uint32_t cx = (uint32_t)((double)xy[2 * i] * G), cy = (uint32_t)((double)xy[2 * i + 1] * G);
        if (cx >= G) cx = G - 1;
        if (cy >= G) cy = G - 1;
        cell_of[i] = cy * G + cx;
        cell_start[cell_of[i] + 1]++;
    }
    for (uint64_t c = 0; c < ncell; c++) cell_start[c + 1] += cell_start[c];
    {
        uint32_t *cur = (uint32_t *)malloc(ncell * sizeof(uint32_t));
        if (!cur) { free(cell_start); free(cell_of); free(bucket); free(src); free(dst); if (!xy_out) free(xy); return GG_ERR_OOM; }
        memcpy(cur, cell_start, ncell * sizeof(uint32_t));
        for (uint32_t i = 0; i < npts; i++) bucket[cur[cell_of[i]]++] = i; /* ascending ids per cell */
        free(cur);
    }
    const double cs = 1.0 / (double)G;
    #pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t ii = 0; ii < (int64_t)npts; ii++) {
        uint32_t i = (uint32_t)ii;
        knn_cand best[64];
        uint32_t have = 0;
        double xi = xy[2 * i], yi = xy[2 * i + 1];
        int32_t cx = (int32_t)(cell_of[i] % G), cy = (int32_t)(cell_of[i] / G);
        for (int32_t r = 0;; r++) {
            /* visit cells with Chebyshev distance exactly r from (cx,cy) */
            for (int32_t dy = -r; dy <= r; dy++) {
                int32_t y = cy + dy;
                if (y < 0 || y >= (int32_t)G) continue;
                int32_t step = (dy == -r || dy == r) ? 1 : 2 * r;
                if (r == 0) step = 1;
                for (int32_t dx = -r; dx <= r; dx += step) {
                    int32_t x = cx + dx;
                    if (x < 0 || x >= (int32_t)G) continue;
                    uint32_t c = (uint32_t)y * G + (uint32_t)x;
                    for (uint32_t q = cell_start[c]; q < cell_start[c + 1]; q++) {
                        uint32_t j = bucket[q];
                        if (j == i) continue;
                        double ddx = (double)xy[2 * j] - xi, ddy = (double)xy[2 * j + 1] - yi;
                        double d2 = ddx * ddx + ddy * ddy;
                        if (have == k && !cand_less(d2, j, best[k - 1].d2, best[k - 1].id)) continue;
                        uint32_t p = (have < k) ? have++ : k - 1;
                        while (p > 0 && cand_less(d2, j, best[p - 1].d2, best[p - 1].id)) { best[p] = best[p - 1]; p--; }
                        best[p].d2 = d2; best[p].id = j;
                    }
                }
            }
            /* every point outside rings 0..r is farther than r*cs */
            double bound = (double)r * cs;
            if (have == k && best[k - 1].d2 < bound * bound * (1.0 - 1e-12)) break;
            if (r > (int32_t)G + 1) break;
        }
        for (uint32_t t = 0; t < k; t++) { src[(uint64_t)i * k + t] = i; dst[(uint64_t)i * k + t] = best[t].id; }
    }
    free(cell_start); free(cell_of); free(bucket);
    if (!xy_out) free(xy);
    int rc = csr_from_arcs(npts, (uint64_t)npts * k, src, dst, 1, 1, out);
    free(src); free(dst);
    return rc;
}

/* ---------------------------------------------------------------- RMAT -- */

/*
 * R-MAT (Chakrabarti, Zhan & Faloutsos 2004): each of 2^scale * edge_factor
 * draws picks, at each of `scale` levels, quadrant a (0,0), b (0,1), c (1,0)
 * or d (1,1) from one uniform draw.  Self-loops are dropped, the arcs are
 * symmetrised and deduplicated, and ids are relabelled by a Fisher-Yates
 * permutation when `permute` is set.
 */
int gg_rmat(uint32_t scale, uint32_t edge_factor, double a, double b, double c, uint64_t seed,
            int permute, gg_csr *out) {
    if (!out || scale == 0 || scale > 30 || edge_factor == 0) return GG_ERR_ARG;
    if (!(a >= 0 && b >= 0 && c >= 0 && a + b + c <= 1.0)) return GG_ERR_ARG;
    uint64_t n = 1ULL << scale, M = n * edge_factor;
    if (2 * M > 0xFFFFFFF0ULL) return GG_ERR_TOO_LARGE;
    uint32_t *src = (uint32_t *)malloc(M * sizeof(uint32_t));
    uint32_t *dst = (uint32_t *)malloc(M * sizeof(uint32_t));
    if (!src || !dst) { free(src); free(dst); return GG_ERR_OOM; }
    const double ab = a + b, abc = a + b + c;
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < (int64_t)M; e++) {
        uint32_t u = 0, v = 0;
        for (uint32_t l = 0; l < scale; l++) {
            double r = gg_unit(gg_draw(seed, S_RMAT, (uint64_t)e * scale + l));
            uint32_t bu, bv;
            if (r < a) { bu = 0; bv = 0; }
            else if (r < ab) { bu = 0; bv = 1; }
            else if (r < abc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu; v = (v << 1) | bv;
        }
        src[e] = u; dst[e] = v;
    }
    if (permute) {
        uint32_t *perm = (uint32_t *)malloc(n * sizeof(uint32_t));
        if (!perm) { free(src); free(dst); return GG_ERR_OOM; }
        for (uint64_t i = 0; i < n; i++) perm[i] = (uint32_t)i;
        for (uint64_t i = n - 1; i > 0; i--) {
            uint64_t j = gg_draw(seed, S_PERM, i) % (i + 1);
            uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        }
        #pragma omp parallel for schedule(static)
        for (int64_t e = 0; e < (int64_t)M; e++) { src[e] = perm[src[e]]; dst[e] = perm[dst[e]]; }
        free(perm);
    }
    int rc = csr_from_arcs((uint32_t)n, M, src, dst, 1, 1, out);
    free(src); free(dst);
    return rc;
}

/* -------------------------------------------------------------- random -- */

/*
 * Tiny random graphs for brute-force checks: `draws` arcs with uniform
 * endpoints.  keep_raw != 0 keeps self-loops and duplicate arcs (the CSR is
 * still grouped by source, lists sorted); directed == 0 symmetrises.
 */
int gg_random(uint32_t n, uint32_t draws, int directed, int keep_raw, uint64_t seed, gg_csr *out) {
    if (!out || n == 0) return GG_ERR_ARG;
    uint32_t *src = (uint32_t *)malloc((size_t)(draws ? draws : 1) * sizeof(uint32_t));
    uint32_t *dst = (uint32_t *)malloc((size_t)(draws ? draws : 1) * sizeof(uint32_t));
    if (!src || !dst) { free(src); free(dst); return GG_ERR_OOM; }
    for (uint32_t i = 0; i < draws; i++) {
        src[i] = (uint32_t)(gg_draw(seed, S_RAND, 2ULL * i) % n);
        dst[i] = (uint32_t)(gg_draw(seed, S_RAND, 2ULL * i + 1) % n);
    }
    int rc = csr_from_arcs(n, draws, src, dst, !directed, !keep_raw, out);
    free(src); free(dst);
    return rc;
}

/* Arbitrary arc list -> canonical CSR (used by tests and file readers). */
int gg_from_arcs(uint32_t n, uint32_t M, const uint32_t *src, const uint32_t *dst, int symmetrize,
                 int clean, gg_csr *out) {
    if (!out || n == 0 || (M && (!src || !dst))) return GG_ERR_ARG;
    for (uint32_t i = 0; i < M; i++) if (src[i] >= n || dst[i] >= n) return GG_ERR_ARG;
    return csr_from_arcs(n, M, src, dst, symmetrize, clean, out);
}

/* ------------------------------------------------------------- sources -- */

/* k distinct sources drawn uniformly, rejecting vertices with no out-arcs. */
int gg_pick_sources(uint32_t n, const uint32_t *offsets, uint32_t k, uint64_t seed, uint32_t *out) {
    if (!offsets || !out || n == 0) return GG_ERR_ARG;
    uint64_t nonempty = 0;
    for (uint32_t v = 0; v < n; v++) nonempty += offsets[v + 1] > offsets[v];
    if (nonempty < k) return GG_ERR_ARG;
    uint32_t got = 0;
    for (uint64_t i = 0; got < k; i++) {
        uint32_t v = (uint32_t)(gg_draw(seed, S_SRC, i) % n);
        if (offsets[v + 1] == offsets[v]) continue;
        int dup = 0;
        for (uint32_t q = 0; q < got; q++) if (out[q] == v) { dup = 1; break; }
        if (!dup) out[got++] = v;
    }
    return GG_OK;
}

int gg_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------ file input -- */
/* The PBBS "AdjacencyGraph" text format (the problem-based benchmark
 * suite's graph format, also read by GBBS): the header line
 * "AdjacencyGraph", then n, m, the n offsets and the m targets, one
 * decimal number per line (any whitespace separates).  The graph is read
 * as given (arcs u -> indices[...]); lists are not re-sorted or deduplicated. */

#define GG_ERR_IO 4
#define GG_ERR_FORMAT 5

static int read_u64(FILE *f, uint64_t *x) {
    int c;
    do { c = fgetc(f); } while (c == ' ' || c == '\n' || c == '\r' || c == '\t');
    if (c < '0' || c > '9') return -1;
    uint64_t v = 0;
    while (c >= '0' && c <= '9') {
        v = v * 10u + (uint64_t)(c - '0');
        if (v > 0xFFFFFFFFull) return -1;
        c = fgetc(f);
    }
    *x = v;
    return 0;
}

int gg_read_adj(const char *path, gg_csr *out) {
    if (!path || !out) return GG_ERR_ARG;
    memset(out, 0, sizeof(*out));
    FILE *f = fopen(path, "rb");
    if (!f) return GG_ERR_IO;
    char head[32] = {0};
    if (fscanf(f, "%31s", head) != 1 || strcmp(head, "AdjacencyGraph") != 0) { fclose(f); return GG_ERR_FORMAT; }
    uint64_t n = 0, m = 0;
    if (read_u64(f, &n) || read_u64(f, &m) || n == 0 || n >= 0x80000000ull) { fclose(f); return GG_ERR_FORMAT; }
    uint32_t *off = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint32_t *idx = (uint32_t *)malloc((size_t)(m ? m : 1) * sizeof(uint32_t));
    if (!off || !idx) { free(off); free(idx); fclose(f); return GG_ERR_OOM; }
    int bad = 0;
    for (uint64_t v = 0; v < n && !bad; v++) {
        uint64_t x;
        if (read_u64(f, &x) || x > m || (v == 0 && x != 0) || (v > 0 && x < off[v - 1])) bad = 1;
        else off[v] = (uint32_t)x;
    }
    off[n] = (uint32_t)m;
    for (uint64_t e = 0; e < m && !bad; e++) {
        uint64_t x;
        if (read_u64(f, &x) || x >= n) bad = 1;
        else idx[e] = (uint32_t)x;
    }
    fclose(f);
    if (bad) { free(off); free(idx); return GG_ERR_FORMAT; }
    out->n = (uint32_t)n; out->m = (uint32_t)m; out->offsets = off; out->indices = idx;
    return GG_OK;
}

int gg_write_adj(const char *path, uint32_t n, uint32_t m, const uint32_t *offsets, const uint32_t *indices) {
    if (!path || !offsets || (m && !indices)) return GG_ERR_ARG;
    FILE *f = fopen(path, "wb");
    if (!f) return GG_ERR_IO;
    int ok = fprintf(f, "AdjacencyGraph\n%u\n%u\n", n, m) > 0;
    for (uint32_t v = 0; v < n && ok; v++) ok = fprintf(f, "%u\n", offsets[v]) > 0;
    for (uint32_t e = 0; e < m && ok; e++) ok = fprintf(f, "%u\n", indices[e]) > 0;
    if (fclose(f) != 0) ok = 0;
    return ok ? GG_OK : GG_ERR_IO;
}

/* The GBBS binary graph layout (the binary format the paper's experiments
 * read, Sec. 4 Setup; the paper names it but does not print it).  Read here
 * as: three little-endian 64-bit header words n, m and the file's size in
 * bytes, then n + 1 64-bit offsets, then m 32-bit targets.  The file must
 * hold exactly 24 + 8(n+1) + 4m bytes; the third header word is checked
 * against that size.  Offsets must start at 0, not decrease and end at m;
 * targets must be < n.  n < 2^31 and m < 2^32 (this library's ids). */
static int read_exact(FILE *f, void *p, size_t bytes) { return fread(p, 1, bytes, f) == bytes ? 0 : -1; }

int gg_read_gbbs_bin(const char *path, gg_csr *out) {
    if (!path || !out) return GG_ERR_ARG;
    memset(out, 0, sizeof(*out));
    FILE *f = fopen(path, "rb");
    if (!f) return GG_ERR_IO;
    uint64_t h[3];
    if (read_exact(f, h, sizeof(h))) { fclose(f); return GG_ERR_FORMAT; }
    const uint64_t n = h[0], m = h[1];
    if (n == 0 || n >= 0x80000000ull || m > 0xFFFFFFFFull) { fclose(f); return GG_ERR_FORMAT; }
    const uint64_t want = 24u + 8u * (n + 1u) + 4u * m;
    if (h[2] != want || fseek(f, 0, SEEK_END) != 0) { fclose(f); return GG_ERR_FORMAT; }
    const long size = ftell(f);
    if (size < 0 || (uint64_t)size != want || fseek(f, 24, SEEK_SET) != 0) { fclose(f); return GG_ERR_FORMAT; }
    uint64_t *o64 = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint32_t *off = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint32_t *idx = (uint32_t *)malloc((size_t)(m ? m : 1) * sizeof(uint32_t));
    if (!o64 || !off || !idx) { free(o64); free(off); free(idx); fclose(f); return GG_ERR_OOM; }
    int bad = read_exact(f, o64, ((size_t)n + 1) * sizeof(uint64_t)) ||
              (m && read_exact(f, idx, (size_t)m * sizeof(uint32_t)));
    fclose(f);
    if (!bad && (o64[0] != 0 || o64[n] != m)) bad = 1;
    for (uint64_t v = 0; v < n && !bad; v++)
        if (o64[v + 1] < o64[v]) bad = 1;
    for (uint64_t v = 0; v <= n && !bad; v++) off[v] = (uint32_t)o64[v];
    for (uint64_t e = 0; e < m && !bad; e++)
        if (idx[e] >= n) bad = 1;
    free(o64);
    if (bad) { free(off); free(idx); return GG_ERR_FORMAT; }
    out->n = (uint32_t)n; out->m = (uint32_t)m; out->offsets = off; out->indices = idx;
    return GG_OK;
}

int gg_write_gbbs_bin(const char *path, uint32_t n, uint32_t m, const uint32_t *offsets,
                      const uint32_t *indices) {
    if (!path || !offsets || (m && !indices) || n == 0) return GG_ERR_ARG;
    FILE *f = fopen(path, "wb");
    if (!f) return GG_ERR_IO;
    const uint64_t h[3] = {n, m, 24u + 8u * ((uint64_t)n + 1u) + 4u * (uint64_t)m};
    int ok = fwrite(h, sizeof(uint64_t), 3, f) == 3;
    for (uint32_t v = 0; v <= n && ok; v++) {
        const uint64_t o = offsets[v];
        ok = fwrite(&o, sizeof(o), 1, f) == 1;
    }
    if (ok && m) ok = fwrite(indices, sizeof(uint32_t), m, f) == m;
    if (fclose(f) != 0) ok = 0;
    return ok ? GG_OK : GG_ERR_IO;
}

/* ------------------------------------------------------------ edge weights -- */
/* Seeded positive weights in [lo, hi] for every arc of a CSR, drawn per
 * unordered vertex pair {u, w}: the two arcs of an undirected edge (stored
 * both ways) get the same weight.  out[e] is the weight of arc e. */
int gg_edge_weights(uint32_t n, const uint32_t *offsets, const uint32_t *indices, uint32_t lo,
                    uint32_t hi, uint64_t seed, uint32_t *out) {
    if (!offsets || !out || lo == 0 || hi < lo) return GG_ERR_ARG;
    const uint64_t span = (uint64_t)hi - lo + 1u;
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < (int64_t)n; v++) {
        for (uint32_t e = offsets[v]; e < offsets[v + 1]; e++) {
            const uint32_t w = indices[e];
            const uint64_t a = (uint64_t)v < w ? (uint64_t)v : w, b = (uint64_t)v < w ? w : (uint64_t)v;
            out[e] = lo + (uint32_t)(gg_draw(seed, 0x77u, (a << 32) | b) % span);
        }
    }
    return GG_OK;
}
